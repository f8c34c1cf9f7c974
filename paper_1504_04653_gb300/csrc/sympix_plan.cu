// Support, symmetry classes and block plan.
//
// Pixel c of ring j (n_j pixels, longitude 2 pi (c + 1/2) / n_j) and pixel p
// of ring rho differ in longitude by pi z g / (n_j n_rho) with the integer
// z = (2c+1) Q - (2p+1) P, P = n_j / g, Q = n_rho / g, g = gcd(n_j, n_rho).
// Their separation therefore depends only on (j, rho, |z|): every distinct
// |z| of a ring pair is one symmetry class (Sec. 2.3: distances repeat along
// the ring with period P), evaluated once (Sec. 4.1, 4.2).  The transposed
// pair (rho, j) and the north/south mirror (N-1-j, N-1-rho) have the same
// classes, so only canonical pairs own table slots.  A pair couples when its
// angular distance is <= r_s (the truncation of Eq. f); |z| grows with the
// distance, so the coupled classes of a ring pair are |z| <= mmax.
#include <math.h>

#include <algorithm>
#include <numeric>
#include <unordered_map>

#include "sympix_internal.cuh"

namespace sympix {

// u = 1 - cos(gamma) of separation index m on canonical pair (a, b), by the
// haversine identity 2 sin^2(dtheta/2) + 2 sin th_a sin th_b sin^2(dphi/2),
// dphi / 2 = pi m g / (2 n_a n_b).
__device__ __forceinline__ double class_u(double base, double st, double denom, long mg) {
    double h = sin(0.5 * kPi * (double)mg / denom);
    return base + st * h * h;
}

// One thread per (canonical pair, operator): the largest coupled |z|, and
// the pair's smallest relative distance |u - u_s| / u_s over the classes
// next to the threshold (the last coupled and the first uncoupled one, or
// the nearest class when none couples; +inf when r_s >= pi).
__global__ void k_support_mmax(int npairs, int nops, const CanonPair *__restrict__ pairs,
                               const double *__restrict__ theta, const double *__restrict__ rs,
                               int32_t *__restrict__ mmax, double *__restrict__ margin) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npairs * nops) return;
    const int pi = i / nops, o = i % nops;
    const CanonPair cp = pairs[pi];
    const long P = cp.na / cp.g, Q = cp.nb / cp.g;
    const long PQg = P * Q * cp.g;
    const long par = (P + Q) & 1;
    const long mcap = PQg - ((PQg - par) & 1);  // |dphi| <= pi
    const double r = rs[o];
    if (r >= kPi) {
        mmax[i] = (int32_t)mcap;
        margin[i] = INFINITY;
        return;
    }
    const double hs = sin(0.5 * r);
    const double us = 2.0 * hs * hs;
    const double ta = theta[cp.a], tb = theta[cp.b];
    const double da = sin(0.5 * (ta - tb));
    const double base = 2.0 * da * da;
    const double st = 2.0 * sin(ta) * sin(tb);
    const double denom = (double)cp.na * (double)cp.nb;
    const double u0 = class_u(base, st, denom, par * cp.g);
    if (u0 > us) {
        mmax[i] = -1;
        margin[i] = (u0 - us) / us;
        return;
    }
    long m = par;
    double um = u0, un = INFINITY;
    while (m + 2 <= mcap) {
        const double u = class_u(base, st, denom, (m + 2) * cp.g);
        if (u > us) {
            un = u;
            break;
        }
        m += 2;
        um = u;
    }
    mmax[i] = (int32_t)m;
    margin[i] = fmin(us - um, un - us) / us;
}

// One thread per canonical pair: u of each stored class.
__global__ void k_support_slots(int npairs, const CanonPair *__restrict__ pairs, const double *__restrict__ theta,
                                double *__restrict__ slot_u, int32_t *__restrict__ slot_pair) {
    int pi = blockIdx.x * blockDim.x + threadIdx.x;
    if (pi >= npairs) return;
    const CanonPair cp = pairs[pi];
    const long P = cp.na / cp.g, Q = cp.nb / cp.g;
    const long par = (P + Q) & 1;
    const double ta = theta[cp.a], tb = theta[cp.b];
    const double da = sin(0.5 * (ta - tb));
    const double base = 2.0 * da * da;
    const double st = 2.0 * sin(ta) * sin(tb);
    const double denom = (double)cp.na * (double)cp.nb;
    for (int k = 0; k < cp.kmax; ++k) {
        slot_u[cp.slot0 + k] = class_u(base, st, denom, (par + 2L * k) * cp.g);
        slot_pair[cp.slot0 + k] = pi;
    }
}

// Largest offset d >= 0 such that some pixel couples to both c and c - d
// (for some class c), i.e. some z = (2c+1)Q - (2p+1)P lies in
// [2 d Q - m, m]; -1 if none.
static long entry_width(long P, long Q, long m) {
    long w = -1;
    for (long d = 0;; ++d) {
        const long lo = 2 * d * Q - m;
        if (lo > m) break;
        for (long c = 0; c < P; ++c) {
            long z0 = ((2 * c + 1) * Q - P) % (2 * P);
            if (z0 < 0) z0 += 2 * P;
            long r = ((z0 - lo) % (2 * P) + 2 * P) % (2 * P);
            if (lo + r <= m) {
                w = d;
                break;
            }
        }
    }
    return w;
}

// Work of one entry over one period of P columns: multiply-adds (pixels p
// coupled to both c and c - d, summed over d = 0..w and c) and products
// B^_pq N^-1_p (pixels coupled to c).
static void entry_work(long P, long Q, long m, long w, int64_t *triples, int64_t *mults) {
    int64_t t = 0, mu = 0;
    for (long c = 0; c < P; ++c) {
        long z0 = ((2 * c + 1) * Q - P) % (2 * P);
        if (z0 < 0) z0 += 2 * P;
        auto count = [&](long lo, long hi) -> int64_t {  // lattice points z0 + 2P k in [lo, hi]
            if (lo > hi) return 0;
            long first = lo + (((z0 - lo) % (2 * P)) + 2 * P) % (2 * P);
            if (first > hi) return 0;
            return (hi - first) / (2 * P) + 1;
        };
        mu += count(-m, m);
        for (long d = 0; d <= w; ++d) t += count(2 * d * Q - m, m);
    }
    *triples = t;
    *mults = mu;
}

static long gcdl(long a, long b) {
    while (b) {
        long t = a % b;
        a = b;
        b = t;
    }
    return a;
}

}  // namespace sympix

using namespace sympix;

extern "C" int sympix_support(sympix_grid_t grid, int nops, const double *r_s, int ring0, int ring1,
                              sympix_plan_t *out) {
    if (!out) return set_error(SYMPIX_EINVAL, "sympix_support: out is NULL");
    *out = nullptr;
    if (!grid || !r_s) return set_error(SYMPIX_EINVAL, "sympix_support: NULL argument");
    const int N = grid->nrings;
    // DP grids with k > 1: band blocks under tile adjacency (sympix_tiles.cu)
    const bool tiles = grid->k > 1;
    if (tiles && (grid->k > kTileKMax || ring0 % grid->k || ring1 % grid->k))
        return set_error(SYMPIX_EUNSUPPORTED, "sympix_support: k = %d grids need k <= %d and band-aligned rings",
                         grid->k, kTileKMax);
    if (nops < 1 || nops > 4096) return set_error(SYMPIX_EINVAL, "sympix_support: nops %d out of [1, 4096]", nops);
    if (ring0 < 0 || ring1 > N || ring0 >= ring1)
        return set_error(SYMPIX_EINVAL, "sympix_support: ring range [%d, %d) not inside [0, %d)", ring0, ring1, N);
    for (int o = 0; o < nops; ++o)
        if (!(r_s[o] > 0.0) || !std::isfinite(r_s[o]))
            return set_error(SYMPIX_EINVAL, "sympix_support: r_s[%d] must be positive and finite", o);
    if (grid->max_ring > 30000)
        return set_error(SYMPIX_EUNSUPPORTED, "sympix_support: rings above 30000 pixels overflow 32-bit indices");

    sympix_plan_s *pl = new sympix_plan_s();
    auto fail = [&](int code) {
        delete pl;
        return code;
    };
    pl->grid = grid;
    pl->nops = nops;
    pl->ring0 = ring0;
    pl->ring1 = ring1;
    pl->r_s.assign(r_s, r_s + nops);
    pl->tiles = tiles;
    pl->all_d = tiles;  // D^ of a band block couples different rings: d at every class
    const std::vector<double> &th = grid->theta;
    const std::vector<int32_t> &nr = grid->nring;
    double hmin = kPi;
    for (int j = 0; j + 1 < N; ++j) hmin = std::min(hmin, th[j + 1] - th[j]);
    int rmax = 0;
    for (int o = 0; o < nops; ++o) {
        int R = (r_s[o] >= kPi) ? N : (int)std::min<double>(N, ceil(r_s[o] / hmin) + 1);
        pl->radius.push_back(R);
        rmax = std::max(rmax, R);
    }

    // canonical ring pairs met by the planned blocks
    std::unordered_map<int64_t, int> index;
    auto canon = [&](int j, int rho) { return canon_pair(N, j, rho); };
    const int kk = grid->k;
    for (int j = ring0; j < ring1; ++j)
        for (int rho = tiles ? std::max(0, (j / kk - 1) * kk) : std::max(0, j - rmax);
             rho <= (tiles ? std::min(N - 1, (j / kk + 2) * kk - 1) : std::min(N - 1, j + rmax)); ++rho) {
            auto ab = canon(j, rho);
            int64_t key = (int64_t)ab.first * N + ab.second;
            if (index.count(key)) continue;
            CanonPair cp{};
            cp.a = ab.first;
            cp.b = ab.second;
            cp.na = nr[cp.a];
            cp.nb = nr[cp.b];
            cp.g = (int32_t)gcdl(cp.na, cp.nb);
            index[key] = (int)pl->pairs.size();
            pl->pairs.push_back(cp);
        }
    const int npairs = (int)pl->pairs.size();

    // device: coupled classes per pair and operator.  Coupling is an FP64
    // comparison u <= u_s; a class whose u lies within 1e-12 (relative) of
    // u_s could fall either way under another correct sin, so such a radius
    // is scaled by (1 - 1e-9) until no class is that close (the same rule,
    // applied the same way, in every implementation of the support).
    int rc;
    DevBuf<double> d_rs, d_margin;
    DevBuf<int32_t> d_mmax;
    if (tiles) {  // the largest |z| of a tile-coupled pixel pair; no radius, no threshold
        pl->pair_mmax.resize((size_t)npairs * nops);
        pl->margin.assign(nops, INFINITY);
        std::map<std::pair<int, int>, long> seen;
        for (int pi = 0; pi < npairs; ++pi) {
            const CanonPair &cp = pl->pairs[pi];
            const int ga = cp.a / kk, gb = cp.b / kk;
            const bool all = ga == gb && (ga == 0 || ga == N / kk - 1);
            auto key = std::make_pair(all ? -cp.na : cp.na, cp.nb);
            if (!seen.count(key)) seen[key] = tile_pair_mmax(cp.na, cp.nb, kk, all);
            for (int o = 0; o < nops; ++o) pl->pair_mmax[(size_t)pi * nops + o] = (int32_t)seen[key];
        }
    } else {
        const int tot = npairs * nops;
        if ((rc = pl->d_pairs.upload(pl->pairs)) || (rc = d_mmax.alloc((size_t)tot)) ||
            (rc = d_margin.alloc((size_t)tot)))
            return fail(rc);
        pl->pair_mmax.resize((size_t)tot);
        std::vector<double> marg((size_t)tot);
        pl->margin.assign(nops, INFINITY);
        for (int it = 0;; ++it) {
            if ((rc = d_rs.upload(pl->r_s))) return fail(rc);
            k_support_mmax<<<(tot + 127) / 128, 128>>>(npairs, nops, pl->d_pairs.p, grid->d_theta.p, d_rs.p,
                                                       d_mmax.p, d_margin.p);
            cudaError_t e = cudaMemcpy(pl->pair_mmax.data(), d_mmax.p, (size_t)tot * sizeof(int32_t),
                                       cudaMemcpyDeviceToHost);
            if (e == cudaSuccess)
                e = cudaMemcpy(marg.data(), d_margin.p, (size_t)tot * sizeof(double), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return fail(cuda_error(e, "sympix_support: class search"));
            bool again = false;
            for (int o = 0; o < nops; ++o) {
                double mo = INFINITY;
                for (int pi = 0; pi < npairs; ++pi) mo = std::min(mo, marg[(size_t)pi * nops + o]);
                pl->margin[o] = mo;
                if (mo <= kSupportMargin && it < 8) {
                    pl->r_s[o] *= 1.0 - 1e-9;
                    again = true;
                }
            }
            if (!again) break;
        }
    }
    // slots: levels 0..kmax-1 of every canonical pair (max over operators);
    // the same-ring pairs' slots first, so that the kernel table's warps that
    // evaluate d (needed there only, unless blocks between rings are planned)
    // are a leading range and the others skip d's multiply-adds as a whole
    int64_t nslots = 0;
    for (int pass = 0; pass < 2; ++pass)
        for (int pi = 0; pi < npairs; ++pi) {
            CanonPair &cp = pl->pairs[pi];
            if ((cp.a == cp.b) != (pass == 0)) continue;
            int kmax = 0;
            for (int o = 0; o < nops; ++o) {
                int m = pl->pair_mmax[(size_t)pi * nops + o];
                if (m >= 0) kmax = std::max(kmax, m / 2 + 1);
            }
            cp.kmax = kmax;
            cp.slot0 = nslots;
            nslots += kmax;
        }
    pl->nslots = nslots;
    if ((rc = pl->d_pairs.upload(pl->pairs)) || (rc = pl->d_slot_u.alloc(std::max<int64_t>(nslots, 1))) ||
        (rc = pl->d_slot_pair.alloc(std::max<int64_t>(nslots, 1))))
        return fail(rc);
    k_support_slots<<<(npairs + 127) / 128, 128>>>(npairs, pl->d_pairs.p, grid->d_theta.p, pl->d_slot_u.p,
                                                   pl->d_slot_pair.p);

    // blocks and their coupled neighbour rings (DP grids: one block per band)
    if (tiles && (rc = plan_tile_blocks(pl, index, ring0 / kk, ring1 / kk))) return fail(rc);
    const int nb = ring1 - ring0;
    int64_t offp = 0, offd = 0;
    for (int o = 0; o < (tiles ? 0 : nops); ++o) {
        for (int j = ring0; j < ring1; ++j) {
            BlockDesc bd{};
            bd.op = o;
            bd.ring = j;
            bd.n = nr[j];
            bd.pair0 = (int64_t)pl->entries.size();
            bd.dtab = -1;
            long w = 0;
            bool wrap = false;
            const int R = pl->radius[o];
            for (int rho = std::max(0, j - R); rho <= std::min(N - 1, j + R); ++rho) {
                auto ab = canon(j, rho);
                const int pi = index.at((int64_t)ab.first * N + ab.second);
                const int m = pl->pair_mmax[(size_t)pi * nops + o];
                if (m < 0) continue;
                const long g = gcdl(nr[j], nr[rho]);
                PairEntry pe{};
                pe.rho = rho;
                pe.P = (int32_t)(nr[j] / g);
                pe.Q = (int32_t)(nr[rho] / g);
                pe.mmax = m;
                pe.par = (pe.P + pe.Q) & 1;
                pe.nrho = nr[rho];
                pe.nstride = grid->stride[rho];
                pe.tab = pl->pairs[pi].slot0;
                pe.noff = grid->offset[rho];
                if ((long)m >= (long)pe.P * pe.Q * g - pe.P) wrap = true;
                w = std::max(w, entry_width(pe.P, pe.Q, m));
                if (rho == j) {
                    bd.dtab = pe.tab;
                    bd.dK = m / 2 + 1;
                }
                pl->entries.push_back(pe);
            }
            bd.npairs = (int32_t)((int64_t)pl->entries.size() - bd.pair0);
            bd.w = (int32_t)w;
            if (!(wrap || 2 * w + 1 >= bd.n || w > 64)) {
                for (int e = 0; e < bd.npairs; ++e) {
                    const PairEntry &pe = pl->entries[bd.pair0 + e];
                    int64_t t, mu;
                    entry_work(pe.P, pe.Q, pe.mmax, w, &t, &mu);
                    pl->ntriples += t * (bd.n / pe.P);
                    pl->nmults += mu * (bd.n / pe.P);
                }
            }
            bd.format = (wrap || 2 * w + 1 >= bd.n || w > 64) ? SYMPIX_BLOCK_DENSE : SYMPIX_BLOCK_PBAND;
            const int64_t n = bd.n;
            // every block starts on a 32-byte boundary (a DRAM sector)
            offp = (offp + 3) & ~int64_t(3);
            offd = (offd + 3) & ~int64_t(3);
            bd.off_pband = offp;
            bd.off_dense = offd;
            if (bd.format == SYMPIX_BLOCK_PBAND) {
                offp += n * (2 * w + 1);
                pl->elems_pband += n * (w + 1);
                pl->max_w = std::max<int>(pl->max_w, (int)w);
            } else {
                if (n > 8192) {
                    return fail(set_error(SYMPIX_EUNSUPPORTED,
                                          "sympix_support: ring %d (%d pixels) couples too widely for a band", j, bd.n));
                }
                offp += n * n;
                pl->elems_pband += n * (n + 1) / 2;
            }
            offd += n * n;
            pl->elems_dense += n * (n + 1) / 2;
            pl->blocks.push_back(bd);
        }
    }
    if (!tiles) {
        pl->size_pband = offp;
        pl->size_dense = offd;
    }

    // sampling work items: pband blocks in tiles of 128 columns, bucketed by
    // band width; dense blocks of up to 64 pixels in tiles of 8 elements (a
    // warp each), larger ones in tiles of 256 (a thread each)
    for (size_t b = 0; b < (tiles ? 0 : pl->blocks.size()); ++b) {
        const BlockDesc &bd = pl->blocks[b];
        if (bd.format == SYMPIX_BLOCK_PBAND) {
            int bucket = bd.w <= 8 ? 0 : bd.w <= 16 ? 1 : bd.w <= 32 ? 2 : 3;
            for (int q0 = 0; q0 < bd.n; q0 += 128) pl->items_pband[bucket].push_back({(int32_t)b, q0});
        } else {
            const int64_t ne = (int64_t)bd.n * bd.n;
            if (bd.n <= 64)
                for (int64_t e0 = 0; e0 < ne; e0 += kDenseItemElems) pl->items_dense.push_back({(int32_t)b, (int32_t)e0});
            else
                for (int64_t e0 = 0; e0 < ne; e0 += 256) pl->items_dense_rows.push_back({(int32_t)b, (int32_t)e0});
        }
    }
    // convolution work items: every block's ring in tiles of 128 pixels
    for (size_t b = 0; b < (tiles ? 0 : pl->blocks.size()); ++b) {
        const BlockDesc &bd = pl->blocks[b];
        for (int q0 = 0; q0 < bd.n; q0 += 128)
            pl->items_conv.push_back({(int32_t)b, q0, grid->offset[bd.ring], grid->stride[bd.ring], 0});
    }
    // factorisation work lists, most expensive blocks first
    std::vector<int32_t> order(pl->blocks.size());
    std::iota(order.begin(), order.end(), 0);
    auto cost = [&](int b) {
        const BlockDesc &bd = pl->blocks[b];
        double n = bd.n, w = bd.w;
        return bd.format == SYMPIX_BLOCK_PBAND ? n * (w + 1) * (3 * w + 1) : n * n * n / 3.0;
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
    for (int b : order) {
        const BlockDesc &bd = pl->blocks[b];
        int list;
        if (bd.format == SYMPIX_BLOCK_PBAND)
            list = bd.w <= 8 ? 0 : bd.w <= 12 ? 1 : bd.w <= 16 ? 2 : bd.w <= 64 ? 5 : 4;
        else
            list = bd.n <= 1024 ? 3 : 4;
        pl->factor_items[list].push_back(b);
    }
    // wide bands: one launch per CTA size (a multiple of 32 threads, capped),
    // most expensive blocks first within each
    {
        auto &l5 = pl->factor_items[5];
        auto cta = [&](int b) {
            const int t = (wide_threads(pl->blocks[b].w) + 31) / 32 * 32;
            return std::min(t, kWideMaxThreads);
        };
        std::stable_sort(l5.begin(), l5.end(), [&](int x, int y) { return cta(x) > cta(y); });
        pl->wide_cls.clear();
        for (size_t i = 0; i < l5.size(); ++i) {
            const int t = cta(l5[i]);
            if (pl->wide_cls.empty() || pl->wide_cls.back().threads != t)
                pl->wide_cls.push_back({(int)i, 0, t, 0});
            WideClass &c = pl->wide_cls.back();
            ++c.count;
            c.wmax = std::max(c.wmax, pl->blocks[l5[i]].w);
        }
    }

    // FP32 factorisation on a band shadow: blocks by exact width (most
    // expensive first, so a slice holds blocks of similar length), slices of
    // up to 32, each with its lane-interleaved shadow region.  The slices of
    // w > 12 take the first shadow offsets: the narrow-band factor covers
    // w <= 12, so by default only those are allocated.
    {
        std::vector<int32_t> byw[17];
        for (int b : order) {
            const BlockDesc &bd = pl->blocks[b];
            if (bd.format == SYMPIX_BLOCK_PBAND && bd.w <= 16) byw[bd.w].push_back(b);
        }
        int64_t sh = 0, l21 = 0;
        auto rows_of = [&](int w, int i, int cnt) {
            int r = 0;
            for (int j = 0; j < cnt; ++j) r = std::max(r, pl->blocks[byw[w][i + j]].n);
            return r;
        };
        std::vector<int64_t> sh_at[17], l21_at[17];
        for (int pass = 0; pass < 2; ++pass)
            for (int w = 0; w <= 16; ++w) {
                if ((pass == 0) != (w > 12)) continue;
                for (int i = 0; i < (int)byw[w].size(); i += 32) {
                    const int rows = rows_of(w, i, std::min(32, (int)byw[w].size() - i));
                    sh_at[w].push_back(sh);
                    l21_at[w].push_back(l21);
                    sh += 32 * (int64_t)rows * (w + 1);
                    l21 += 32 * (int64_t)w * (rows - w);
                }
                if (pass == 0 && w == 16) {
                    pl->size_shadow_hi = sh;
                    pl->size_l21_hi = l21;
                }
            }
        std::vector<int2> tiles21, tiles21_hi, tiles21_lo;
        for (int w = 0; w <= 16; ++w) {
            const int first = (int)pl->f32_items.size(), cnt = (int)byw[w].size();
            pl->f32_items.insert(pl->f32_items.end(), byw[w].begin(), byw[w].end());
            for (int i = 0, si = 0; i < cnt; i += 32, ++si) {
                F32Slice sl;
                sl.w = w;
                sl.first = first + i;
                sl.count = std::min(32, cnt - i);
                sl.rows = rows_of(w, i, sl.count);
                sl.sh = sh_at[w][si];
                sl.l21 = l21_at[w][si];
                const int64_t elems = (int64_t)sl.rows * (w + 1), elems21 = (int64_t)w * (sl.rows - w);
                const int idx = (int)pl->f32_slices.size();
                for (int64_t e0 = 0; e0 < elems; e0 += kTileE) {
                    pl->f32_tiles.push_back(make_int2(idx, (int)e0));
                    if (w > 12) pl->f32_tiles_hi.push_back(make_int2(idx, (int)e0));
                    else pl->f32_tiles_lo.push_back(make_int2(idx, (int)e0));
                }
                for (int64_t e0 = 0; e0 < elems21; e0 += kTileE) {
                    tiles21.push_back(make_int2(idx, (int)(-1 - e0)));
                    if (w > 12) tiles21_hi.push_back(make_int2(idx, (int)(-1 - e0)));
                    else tiles21_lo.push_back(make_int2(idx, (int)(-1 - e0)));
                }
                if (w <= 12) ++pl->f32_slices_fused;
                if (w <= 8) ++pl->f32_slices_w8;
                pl->f32_slices.push_back(sl);
            }
        }
        pl->size_shadow_il = sh;
        pl->size_l21_il = l21;
        pl->f32_out_tiles = pl->f32_tiles;
        pl->f32_out_tiles.insert(pl->f32_out_tiles.end(), tiles21.begin(), tiles21.end());
        pl->f32_out_tiles_hi = pl->f32_tiles_hi;
        pl->f32_out_tiles_hi.insert(pl->f32_out_tiles_hi.end(), tiles21_hi.begin(), tiles21_hi.end());
        pl->f32_out_tiles_lo = pl->f32_tiles_lo;
        pl->f32_out_tiles_lo.insert(pl->f32_out_tiles_lo.end(), tiles21_lo.begin(), tiles21_lo.end());
    }
    if (cudaEventCreateWithFlags(&pl->chol_fork, cudaEventDisableTiming) != cudaSuccess)
        return fail(set_error(SYMPIX_ECUDA, "sympix_support: event of the narrow-band factor"));
    if (pl->f32_slices_w8 > 0 && pl->f32_slices_fused > pl->f32_slices_w8 &&
        (cudaStreamCreateWithFlags(&pl->f32_side, cudaStreamNonBlocking) != cudaSuccess ||
         cudaEventCreateWithFlags(&pl->f32_fork, cudaEventDisableTiming) != cudaSuccess ||
         cudaEventCreateWithFlags(&pl->f32_join, cudaEventDisableTiming) != cudaSuccess))
        return fail(set_error(SYMPIX_ECUDA, "sympix_support: stream of the FP32 factor"));
    if ((!pl->factor_items[1].empty() || !pl->factor_items[2].empty()) &&
        (cudaStreamCreateWithFlags(&pl->chol_side, cudaStreamNonBlocking) != cudaSuccess ||
         cudaEventCreateWithFlags(&pl->chol_side_join, cudaEventDisableTiming) != cudaSuccess))
        return fail(set_error(SYMPIX_ECUDA, "sympix_support: stream of the lane-group factor"));
    // narrow-band factor (w <= 12): blocks by width, most expensive first;
    // FP32 slices of 4 blocks (8 lanes each), FP64 / split-FP32 slices of
    // 8 blocks (4 lanes) up to w = 8 and 2 blocks (16 lanes) above; commit tiles over
    // the band rows of every block
    {
        std::vector<int32_t> byw[kNarrowWMax + 1];
        for (int b : order) {
            const BlockDesc &bd = pl->blocks[b];
            if (bd.format == SYMPIX_BLOCK_PBAND && bd.w <= kNarrowWMax) byw[bd.w].push_back(b);
        }
        for (int w = 0; w <= kNarrowWMax; ++w) {
            const int first = (int)pl->chol_items.size(), cnt = (int)byw[w].size();
            if (!cnt) continue;
            pl->chol_wmax = w;
            pl->chol_items.insert(pl->chol_items.end(), byw[w].begin(), byw[w].end());
            const int g64 = w <= 8 ? 4 : 16;
            pl->chol_f32[w] = (int)pl->chol_sl32.size();
            pl->chol_f64[w] = (int)pl->chol_sl64.size();
            for (int i = 0; i < cnt; i += 32 / 8) pl->chol_sl32.push_back({w, first + i, std::min(32 / 8, cnt - i), 8});
            for (int i = 0; i < cnt; i += 32 / g64)
                pl->chol_sl64.push_back({w, first + i, std::min(32 / g64, cnt - i), g64});
            pl->chol_n32[w] = (int)pl->chol_sl32.size() - pl->chol_f32[w];
            pl->chol_n64[w] = (int)pl->chol_sl64.size() - pl->chol_f64[w];
            if (cudaStreamCreateWithFlags(&pl->chol_st[w], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&pl->chol_join[w], cudaEventDisableTiming) != cudaSuccess)
                return fail(set_error(SYMPIX_ECUDA, "sympix_support: stream of the narrow-band factor"));
            for (int b : byw[w]) {
                const BlockDesc &bd = pl->blocks[b];
                const int64_t lim = (int64_t)(bd.n - bd.w) * (bd.w + 1);
                for (int64_t e0 = 0; e0 < lim; e0 += kCommitTileElems) pl->chol_tiles.push_back(make_int2(b, (int)e0));
            }
        }
    }
    // chunked border solve of the fused-range slices (1 <= w <= 12)
    pl->l21_first.assign(pl->f32_slices_fused, -1);
    pl->l21_nch.assign(pl->f32_slices_fused, 0);
    for (int si = 0; si < pl->f32_slices_fused; ++si) {
        const F32Slice &sl = pl->f32_slices[si];
        const int kc = sl.rows - sl.w;
        if (sl.w < 1 || kc <= 0) continue;
        const int cols = l21_chunk_cols_host(sl.w), nch = (kc + cols - 1) / cols;
        pl->l21_slices.push_back(si);
        pl->l21_first[si] = (int32_t)pl->l21_items.size();
        pl->l21_nch[si] = nch;
        for (int q = 0; q < nch; ++q) pl->l21_items.push_back(make_int2(si, q));
        if (sl.w <= 8) {
            pl->l21_items_w8 = (int)pl->l21_items.size();
            pl->l21_slices_w8 = (int)pl->l21_slices.size();
        }
    }
    if (!pl->l21_items.empty()) {
        const int64_t ni = (int64_t)pl->l21_items.size();
        if ((rc = pl->d_l21_items.upload(pl->l21_items)) || (rc = pl->d_l21_slices.upload(pl->l21_slices)) ||
            (rc = pl->d_l21_first.upload(pl->l21_first)) || (rc = pl->d_l21_nch.upload(pl->l21_nch)) ||
            (rc = pl->d_l21_T.alloc(2 * ni * l21_mat_floats())) || (rc = pl->d_l21_P.alloc(2 * ni * l21_mat_floats())) ||
            (rc = pl->d_l21_S.alloc(2 * ni * l21_mat_floats())) || (rc = pl->d_l21_C.alloc(2 * ni * l21_pair_floats())))
            return fail(rc);
    }
    if (pl->f32_slices_fused > 0) {
        if ((rc = pl->d_split_flags.alloc(2 * (int64_t)pl->f32_slices_fused)) ||
            (rc = pl->d_split_bandres.alloc(32 * (int64_t)pl->f32_slices_fused)))
            return fail(rc);
        SPX_CUDA(cudaMemset(pl->d_split_flags.p, 0, 2 * sizeof(int) * pl->f32_slices_fused));
    }
    if ((rc = pl->d_f32_items.upload(pl->f32_items)) || (rc = pl->d_f32_slices.upload(pl->f32_slices)) ||
        (rc = pl->d_f32_tiles.upload(pl->f32_tiles)) || (rc = pl->d_f32_out_tiles.upload(pl->f32_out_tiles)) ||
        (rc = pl->d_f32_tiles_hi.upload(pl->f32_tiles_hi)) ||
        (rc = pl->d_f32_out_tiles_hi.upload(pl->f32_out_tiles_hi)) ||
        (rc = pl->d_f32_tiles_lo.upload(pl->f32_tiles_lo)) ||
        (rc = pl->d_f32_out_tiles_lo.upload(pl->f32_out_tiles_lo)) ||
        (rc = pl->d_shadow_il.alloc(std::max<int64_t>(2 * pl->size_shadow_il, 2))) ||
        (rc = pl->d_l21_il.alloc(std::max<int64_t>(2 * pl->size_l21_il, 2))) ||
        (rc = pl->d_chol_items.upload(pl->chol_items)) || (rc = pl->d_chol_sl32.upload(pl->chol_sl32)) ||
        (rc = pl->d_chol_sl64.upload(pl->chol_sl64)) || (rc = pl->d_chol_tiles.upload(pl->chol_tiles)) ||
        (rc = pl->d_shadow.alloc((pl->factor_items[5].empty() && pl->chol_items.empty())
                                     ? 1
                                     : std::max<int64_t>(pl->size_pband, 1))))
        return fail(rc);
    if (tiles && ((rc = pl->d_tile_blocks.upload(pl->tile_blocks)) || (rc = pl->d_tile_items.upload(pl->tile_items)) ||
                  (rc = pl->d_tile_slot0.upload(pl->tile_slot0)) || (rc = pl->d_tile_noff.upload(pl->tile_noff))))
        return fail(rc);
    if ((rc = pl->d_blocks.upload(pl->blocks)) || (rc = pl->d_entries.upload(pl->entries)) ||
        (rc = pl->d_items_dense.upload(pl->items_dense)) || (rc = pl->d_items_dense_rows.upload(pl->items_dense_rows)) || (rc = pl->d_items_conv.upload(pl->items_conv)))
        return fail(rc);
    for (int bkt = 0; bkt < 5; ++bkt)
        if ((rc = pl->d_items_pband[bkt].upload(pl->items_pband[bkt]))) return fail(rc);
    for (int l = 0; l < 6; ++l)
        if ((rc = pl->d_factor_items[l].upload(pl->factor_items[l]))) return fail(rc);
    if ((rc = pl->d_status.alloc(1)) || (rc = pl->d_ring_off.upload(grid->offset)) ||
        (rc = pl->d_ring_stride.upload(grid->stride)))
        return fail(rc);
    if (cudaMemset(pl->d_status.p, 0, sizeof(int32_t)) != cudaSuccess)
        return fail(set_error(SYMPIX_ECUDA, "sympix_support: status word"));
    const size_t tabn = (size_t)nops * std::max<int64_t>(nslots, 1);
    const size_t nn = (size_t)nops * grid->npix;
    if ((rc = pl->d_tab_b.alloc(tabn)) || (rc = pl->d_tab_d.alloc(tabn)) || (rc = pl->d_tab_b32.alloc(tabn)) ||
        (rc = pl->d_tab_blo.alloc(tabn)) || (rc = pl->d_tab_d32.alloc(tabn)) || (rc = pl->d_tab_dlo.alloc(tabn)) ||
        (rc = pl->d_ninv32.alloc(nn)) || (rc = pl->d_ninvlo.alloc(nn)))
        return fail(rc);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail(cuda_error(e, "sympix_support"));
    (void)nb;
    *out = pl;
    return SYMPIX_OK;
}

constexpr int kTraceCap = 256;

extern "C" int sympix_plan_option(sympix_plan_t pl, int option, double value) {
    if (!pl) return set_error(SYMPIX_EINVAL, "sympix_plan_option: NULL plan");
    if (option == SYMPIX_OPT_FP32_PIVOT_FLOOR) {
        if (!(value >= 0.0) || !std::isfinite(value))
            return set_error(SYMPIX_EINVAL, "sympix_plan_option: pivot floor must be finite and >= 0");
        pl->fp32_pivot_floor = value;
        return SYMPIX_OK;
    }
    if (option == SYMPIX_OPT_TABLE_CTA) {
        if (value != 32.0 && value != 64.0 && value != 128.0)
            return set_error(SYMPIX_EINVAL, "sympix_plan_option: table CTA size is 32, 64 or 128");
        pl->table_cta = (int)value;
        return SYMPIX_OK;
    }
    if (option == SYMPIX_OPT_BORDER_THREADS) {
        if (value != 256.0 && value != 512.0)
            return set_error(SYMPIX_EINVAL, "sympix_plan_option: border threads are 256 or 512");
        pl->border_threads = (int)value;
        return SYMPIX_OK;
    }
    if (option == SYMPIX_OPT_NARROW_FACTOR) {
        if (value != 0.0 && value != 1.0 && value != 2.0 && value != 3.0 && value != -1.0)
            return set_error(SYMPIX_EINVAL, "sympix_plan_option: narrow factor kernel is -1, 0, 1, 2 or 3");
        if (value == -1.0) {
            pl->narrow_pref[SYMPIX_PREC_FP64] = 2;
            pl->narrow_pref[SYMPIX_PREC_FP32] = 3;
            pl->narrow_pref[SYMPIX_PREC_FP32X2] = 2;
        } else if (value == 2.0 || value == 3.0) {
            // the chunked border solve (every arithmetic) and the split kernel (FP32)
            pl->narrow_pref[SYMPIX_PREC_FP64] = 2;
            pl->narrow_pref[SYMPIX_PREC_FP32] = (int)value;
            pl->narrow_pref[SYMPIX_PREC_FP32X2] = 2;
        } else {
            for (int &v : pl->narrow_pref) v = (int)value;
        }
        return SYMPIX_OK;
    }
    if (option == SYMPIX_OPT_WAIT_LIMIT) {
        if (!(value >= 1.0) || value > 2147483647.0 || value != floor(value))
            return set_error(SYMPIX_EINVAL, "sympix_plan_option: wait limit is an integer in [1, 2^31)");
        pl->wait_limit = (int)value;
        return SYMPIX_OK;
    }
    if (option == SYMPIX_OPT_TRACE) {
        if (value != 0.0 && value != 1.0) return set_error(SYMPIX_EINVAL, "sympix_plan_option: trace is 0 or 1");
        if (value == 1.0 && pl->trace_ev.empty()) {
            pl->trace_ev.resize(kTraceCap, nullptr);
            pl->trace_name.resize(kTraceCap, nullptr);
            for (auto &e : pl->trace_ev) SPX_CUDA(cudaEventCreate(&e));
        }
        pl->trace = value == 1.0;
        pl->trace_n = 0;
        return SYMPIX_OK;
    }
    return set_error(SYMPIX_EINVAL, "sympix_plan_option: unknown option %d", option);
}

namespace sympix {
void trace_mark(sympix_plan_t pl, cudaStream_t st, const char *name) {
    if (!pl->trace || pl->trace_n >= kTraceCap) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    if (cudaEventRecord(pl->trace_ev[pl->trace_n], st) != cudaSuccess) return;
    pl->trace_name[pl->trace_n++] = name;
}
}  // namespace sympix

extern "C" int sympix_plan_tuning(sympix_plan_t pl, int *table_cta, int *border_threads, int *narrow) {
    if (!pl) return set_error(SYMPIX_EINVAL, "sympix_plan_tuning: NULL plan");
    if (table_cta) *table_cta = pl->table_cta;
    if (border_threads) *border_threads = pl->border_threads;
    if (narrow)
        for (int i = 0; i < 3; ++i) narrow[i] = pl->narrow_pref[i];
    return SYMPIX_OK;
}

extern "C" int sympix_autotune(sympix_plan_t pl, const double *bl, const double *dl, const double *ninv, int storage,
                               int sample_precision, int factor_precision, double *blocks, int32_t *info,
                               void *stream) {
    if (!pl || !bl || !dl || !ninv || !blocks || !info) return set_error(SYMPIX_EINVAL, "sympix_autotune: NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    SPX_CUDA(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_error(ce, "sympix_autotune: cudaEventCreate");
    }
    const bool tr = pl->trace;
    pl->trace = false;
    int rc = SYMPIX_OK;
    // time `run` once after one warm-up call
    auto timed = [&](auto run, float *ms) -> int {
        int r = run();
        if (r) return r;
        if (cudaEventRecord(e0, st) != cudaSuccess) return set_error(SYMPIX_ECUDA, "sympix_autotune: event");
        if ((r = run())) return r;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
            return set_error(SYMPIX_ECUDA, "sympix_autotune: event timing");
        return SYMPIX_OK;
    };
    float best = 1e30f;
    int best_cta = pl->table_cta;
    for (int cta : {32, 64, 128}) {
        pl->table_cta = cta;
        float ms = 0.0f;
        if ((rc = timed([&] { return sympix_kernel_table(pl, bl, dl, st); }, &ms))) break;
        if (ms < best) {
            best = ms;
            best_cta = cta;
        }
    }
    pl->table_cta = best_cta;
    // the w <= 12 factor kernel of this arithmetic (periodic-band storage)
    if (!rc && storage == SYMPIX_STORE_PBAND && !pl->chol_items.empty() && factor_precision >= 0 &&
        factor_precision <= 2) {
        best = 1e30f;
        int best_k = pl->narrow_pref[factor_precision];
        for (int kk : {0, 1, 2, 3}) {
            if (kk == 3 && factor_precision != SYMPIX_PREC_FP32) continue;
            pl->narrow_pref[factor_precision] = kk;
            float ms = 0.0f;
            auto run = [&] {
                int r = sympix_sample_blocks(pl, ninv, sample_precision, storage, blocks, st);
                return r ? r : sympix_factor_blocks(pl, storage, factor_precision, blocks, info, st);
            };
            if ((rc = timed(run, &ms))) break;
            if (ms < best) {
                best = ms;
                best_k = kk;
            }
        }
        pl->narrow_pref[factor_precision] = best_k;
    }
    if (!rc && factor_precision == SYMPIX_PREC_FP32 && storage == SYMPIX_STORE_PBAND && !pl->f32_slices.empty() &&
        pl->narrow_pref[SYMPIX_PREC_FP32] == 1) {
        best = 1e30f;
        int best_nt = pl->border_threads;
        for (int nt : {256, 512}) {
            pl->border_threads = nt;
            float ms = 0.0f;
            auto run = [&] {
                int r = sympix_sample_blocks(pl, ninv, sample_precision, storage, blocks, st);
                return r ? r : sympix_factor_blocks(pl, storage, factor_precision, blocks, info, st);
            };
            if ((rc = timed(run, &ms))) break;
            if (ms < best) {
                best = ms;
                best_nt = nt;
            }
        }
        pl->border_threads = best_nt;
    }
    pl->trace = tr;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

extern "C" int sympix_trace_read(sympix_plan_t pl, int cap, const char **names, float *ms, int *count) {
    if (!pl || !count || (cap > 0 && (!names || !ms))) return set_error(SYMPIX_EINVAL, "sympix_trace_read: NULL argument");
    int k = 0;
    if (pl->trace_n > 0) SPX_CUDA(cudaEventSynchronize(pl->trace_ev[pl->trace_n - 1]));
    for (int i = 1; i < pl->trace_n; ++i) {
        if (!pl->trace_name[i]) continue;
        if (k < cap) {
            float t = 0.0f;
            SPX_CUDA(cudaEventElapsedTime(&t, pl->trace_ev[i - 1], pl->trace_ev[i]));
            names[k] = pl->trace_name[i];
            ms[k] = t;
        }
        ++k;
    }
    *count = k;
    pl->trace_n = 0;
    return SYMPIX_OK;
}

extern "C" int sympix_plan_counts(sympix_plan_t pl, int64_t *nslots, int64_t *npairs, int64_t *ntriples,
                                  int64_t *nmults) {
    if (!pl) return set_error(SYMPIX_EINVAL, "sympix_plan_counts: NULL plan");
    if (nslots) *nslots = pl->nslots;
    if (npairs) *npairs = (int64_t)pl->entries.size();
    if (ntriples) *ntriples = pl->ntriples;
    if (nmults) *nmults = pl->nmults;
    return SYMPIX_OK;
}

extern "C" int sympix_plan_launches(sympix_plan_t pl, int storage, int sample_precision, int factor_precision,
                                    int32_t *table, int32_t *sample, int32_t *factor) {
    if (!pl) return set_error(SYMPIX_EINVAL, "sympix_plan_launches: NULL plan");
    if (table) {
        int chunks = 0;
        for (int op0 = 0; op0 < pl->nops;) {
            const int left = pl->nops - op0;
            op0 += left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
            ++chunks;
        }
        *table = 1 + (pl->nslots > 0 ? chunks : 0);
    }
    int s = sample_precision != SYMPIX_PREC_FP64 ? 1 : 0;  // the N^-1 split
    s += pl->tile_items.empty() ? 0 : 1;                     // band blocks of a DP grid
    for (int b = 0; b < 4; ++b) s += pl->items_pband[b].empty() ? 0 : 1;
    s += pl->items_dense.empty() ? 0 : 1;
    s += pl->items_dense_rows.empty() ? 0 : 1;
    if (sample) *sample = s;
    // mirrors the launch sequence of sympix_factor_blocks
    int f = 0;
    const bool pband = storage == SYMPIX_STORE_PBAND;
    const bool narrow = pband && pl->narrow_pref[factor_precision] == 0;
    const bool l0 = !pl->factor_items[0].empty(), l1 = !pl->factor_items[1].empty(),
               l2 = !pl->factor_items[2].empty();
    if (narrow && !pl->chol_items.empty()) {
        // one launch per width present (FP32: then its commit and the FP64
        // rescue, again one launch per width)
        int n32 = 0, n64 = 0;
        for (int w = 0; w <= kNarrowWMax; ++w) {
            n32 += pl->chol_n32[w] > 0 ? 1 : 0;
            n64 += pl->chol_n64[w] > 0 ? 1 : 0;
        }
        int n64lo = 0;  // FP64 / split FP32: the G-lane kernel below kCholGroupFrom (9)
        for (int w = 0; w < 9; ++w) n64lo += pl->chol_n64[w] > 0 ? 1 : 0;
        f += factor_precision == SYMPIX_PREC_FP32 ? n32 + 1 + n64 : n64lo;
    }
    if (factor_precision == SYMPIX_PREC_FP32 && pband) {
        const int nsl = (int)pl->f32_slices.size(), nfu = pl->f32_slices_fused;
        if (narrow) {
            // slices with w > 12: shadow in, band pass, border pass, write-back, FP64 rescue of list 2
            if (nsl > nfu) f += 4 + (l2 ? 1 : 0);
        } else if (nsl > 0) {
            // shadow in, the fused kernels (w <= 8 and 9 <= w <= 12), band and
            // border passes, FP64 write-back, then the FP64 rescue launches
            // (which return at once for blocks that need none)
            const int n8 = pl->f32_slices_w8;
            const int nhi_items = (int)pl->l21_items.size() - pl->l21_items_w8;
            if (pl->narrow_pref[SYMPIX_PREC_FP32] == 3 && f32_split_fits(pl))
                // the split launch (w <= 8); band pass and the five chunked kernels of 9 <= w <= 12
                f += 2 + (n8 > 0 ? 1 : 0) + (nfu > n8 ? 1 + (nhi_items > 0 ? 5 : 0) : 0) + (nsl > nfu ? 2 : 0);
            else if (pl->narrow_pref[SYMPIX_PREC_FP32] == 2)  // band pass, then transfer, carry, solve, corner sums, corners
                f += 2 + (nfu > 0 ? 1 : 0) + (nsl > nfu ? 2 : 0) +
                     (pl->l21_items.empty() ? 0
                                            : 2 + 2 * (pl->l21_items_w8 > 0 ? 1 : 0) +
                                                  3 * ((int)pl->l21_items.size() > pl->l21_items_w8 ? 1 : 0));
            else
                f += 2 + (n8 > 0 ? 1 : 0) + (nfu > n8 ? 1 : 0) + (nsl > nfu ? 2 : 0);
            f += (l0 ? 2 : 0) + (l1 ? 1 : 0) + (l2 ? 1 : 0);
        }
    } else if (factor_precision == SYMPIX_PREC_FP32) {
        f += (l0 || l1 || l2) ? 2 : 0;  // both passes for every width up to 16
    } else if (factor_precision != SYMPIX_PREC_FP32 && pband && pl->narrow_pref[factor_precision] == 2) {
        // w <= 12 on the FP64 / split-FP32 shadow: transpose in, band pass, transfer, carry,
        // solve and corner sums of each width range, corners, write-back; then
        // the lane groups of 12 < w <= 16
        const int ni = (int)pl->l21_items.size(), nlo = pl->l21_items_w8;
        if (pl->f32_slices_fused > 0 && !pl->f32_tiles_lo.empty())
            f += 3 + (ni > 0 ? 2 + 3 * (nlo > 0 ? 1 : 0) + 3 * (ni > nlo ? 1 : 0) : 0);
        f += l2 ? 1 : 0;
    } else if (narrow) {
        f += (l1 ? 1 : 0) + (l2 ? 1 : 0);  // lane groups for 8 < w <= 16, beside the G-lane kernel
    } else {
        f += (l0 ? 2 : 0) + (l1 ? 1 : 0) + (l2 ? 1 : 0);
    }
    f += (int)pl->wide_cls.size() * ((factor_precision == SYMPIX_PREC_FP32 && pband) ? 2 : 1);
    for (int l = 3; l < 5; ++l) f += pl->factor_items[l].empty() ? 0 : 1;
    if (factor) *factor = f;
    return SYMPIX_OK;
}

extern "C" int sympix_blocks_size(sympix_plan_t pl, int storage, size_t *bytes, int64_t *elements) {
    if (!pl) return set_error(SYMPIX_EINVAL, "sympix_blocks_size: NULL plan");
    if (storage != SYMPIX_STORE_PBAND && storage != SYMPIX_STORE_DENSE)
        return set_error(SYMPIX_EINVAL, "sympix_blocks_size: unknown storage %d", storage);
    const bool pb = storage == SYMPIX_STORE_PBAND;
    if (bytes) *bytes = (size_t)(pb ? pl->size_pband : pl->size_dense) * sizeof(double);
    if (elements) *elements = pb ? pl->elems_pband : pl->elems_dense;
    return SYMPIX_OK;
}

extern "C" int sympix_block_layout(sympix_plan_t pl, int storage, int op, int ring, int64_t *offset, int32_t *n,
                                   int32_t *w, int32_t *format) {
    if (!pl) return set_error(SYMPIX_EINVAL, "sympix_block_layout: NULL plan");
    // DP-grid plans: `ring` is the band index (one block per band of k rings)
    const int kk = pl->tiles ? pl->grid->k : 1, lo = pl->ring0 / kk, hi = pl->ring1 / kk;
    if (op < 0 || op >= pl->nops || ring < lo || ring >= hi)
        return set_error(SYMPIX_EINVAL, "sympix_block_layout: (op %d, ring %d) not planned", op, ring);
    const BlockDesc &bd = pl->blocks[(size_t)op * (hi - lo) + (ring - lo)];
    const bool pb = storage == SYMPIX_STORE_PBAND;
    if (offset) *offset = pb ? bd.off_pband : bd.off_dense;
    if (n) *n = bd.n;
    if (w) *w = bd.w;
    if (format) *format = pb ? bd.format : SYMPIX_BLOCK_DENSE;
    return SYMPIX_OK;
}

extern "C" int sympix_plan_status(sympix_plan_t pl, void *stream) {
    if (!pl) return set_error(SYMPIX_EINVAL, "sympix_plan_status: NULL plan");
    cudaStream_t st = (cudaStream_t)stream;
    int32_t v = 0;
    SPX_CUDA(cudaMemcpyAsync(&v, pl->d_status.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SPX_CUDA(cudaMemsetAsync(pl->d_status.p, 0, sizeof(int32_t), st));
    SPX_CUDA(cudaStreamSynchronize(st));
    if (v & 1) return set_error(SYMPIX_ETIMEOUT, "a bounded device wait of the factorisation ran out");
    return SYMPIX_OK;
}

extern "C" int sympix_plan_radius(sympix_plan_t pl, int op, double *r_s, double *margin) {
    if (!pl) return set_error(SYMPIX_EINVAL, "sympix_plan_radius: NULL plan");
    if (op < 0 || op >= pl->nops) return set_error(SYMPIX_EINVAL, "sympix_plan_radius: op %d not planned", op);
    if (r_s) *r_s = pl->r_s[op];
    if (margin) *margin = pl->margin[op];
    return SYMPIX_OK;
}

extern "C" int sympix_plan_device_bytes(sympix_plan_t pl, size_t *bytes, size_t *staging) {
    if (!pl) return set_error(SYMPIX_EINVAL, "sympix_plan_device_bytes: NULL plan");
    size_t b = pl->d_pairs.bytes() + pl->d_slot_u.bytes() + pl->d_slot_pair.bytes() + pl->d_tab_b.bytes() +
               pl->d_tab_d.bytes() + pl->d_tab_b32.bytes() + pl->d_tab_blo.bytes() + pl->d_tab_d32.bytes() +
               pl->d_tab_dlo.bytes() + pl->d_ninv32.bytes() + pl->d_ninvlo.bytes() + pl->d_rec.bytes() +
               pl->d_blocks.bytes() + pl->d_entries.bytes() + pl->d_items_dense.bytes() +
               pl->d_items_dense_rows.bytes() + pl->d_items_conv.bytes() + pl->d_f32_items.bytes() +
               pl->d_f32_slices.bytes() + pl->d_f32_tiles.bytes() + pl->d_shadow_il.bytes() +
               pl->d_l21_il.bytes() + pl->d_f32_out_tiles.bytes() + pl->d_shadow.bytes() + pl->d_chol_items.bytes() +
               pl->d_chol_sl32.bytes() + pl->d_chol_sl64.bytes() + pl->d_chol_tiles.bytes() +
               pl->d_f32_tiles_hi.bytes() + pl->d_f32_out_tiles_hi.bytes() + pl->d_status.bytes() +
               pl->d_ring_off.bytes() + pl->d_ring_stride.bytes() + pl->d_l21_items.bytes() +
               pl->d_l21_slices.bytes() + pl->d_l21_first.bytes() + pl->d_l21_nch.bytes() + pl->d_l21_T.bytes() +
               pl->d_l21_P.bytes() + pl->d_l21_S.bytes() + pl->d_l21_C.bytes() + pl->d_split_flags.bytes() +
               pl->d_split_bandres.bytes() + pl->d_f32_tiles_lo.bytes() + pl->d_f32_out_tiles_lo.bytes();
    for (const auto &kv : pl->coupling) b += kv.second.d_desc.bytes();
    for (int i = 0; i < 5; ++i) b += pl->d_items_pband[i].bytes();
    for (int i = 0; i < 6; ++i) b += pl->d_factor_items[i].bytes();
    if (bytes) *bytes = b;
    if (staging) *staging = pl->d_rec.bytes();
    return SYMPIX_OK;
}

extern "C" int sympix_support_copy(sympix_plan_t pl, int op, int ring, int radius, int32_t *mmax) {
    if (!pl || !mmax) return set_error(SYMPIX_EINVAL, "sympix_support_copy: NULL argument");
    if (pl->tiles) return set_error(SYMPIX_EUNSUPPORTED, "sympix_support_copy: ring blocks only (k = 1)");
    if (op < 0 || op >= pl->nops || ring < pl->ring0 || ring >= pl->ring1 || radius < 0)
        return set_error(SYMPIX_EINVAL, "sympix_support_copy: (op %d, ring %d) not planned", op, ring);
    for (int i = 0; i <= 2 * radius; ++i) mmax[i] = -1;
    const BlockDesc &bd = pl->blocks[(size_t)op * (pl->ring1 - pl->ring0) + (ring - pl->ring0)];
    for (int e = 0; e < bd.npairs; ++e) {
        const PairEntry &pe = pl->entries[bd.pair0 + e];
        const int d = pe.rho - ring;
        if (d >= -radius && d <= radius) mmax[d + radius] = pe.mmax;
    }
    return SYMPIX_OK;
}

extern "C" void sympix_plan_free(sympix_plan_t pl) { delete pl; }
