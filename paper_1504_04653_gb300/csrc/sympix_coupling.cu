// Blocks between rings, and the block preconditioner applied to a vector.
//
// Off-diagonal blocks (Eq. system-rewritten, Eq. Dhat with rows on ring j
// and columns on ring k = j + delta):
//   M_qr = [gamma_qr <= r_s] d(x_qr) + sum_p B^_pq N^-1_p B^_pr,
// p over the pixels of every ring coupled to both.  Pixel q of ring j and
// pixel r of ring k are at separation index z = (2q+1) Q - (2r+1) P with
// P = n_j / g, Q = n_k / g, g = gcd(n_j, n_k).  M_qr vanishes unless
// gamma_qr <= 2 r_s (a pixel coupled to both is within r_s of each), so row
// q stores the columns with |z| <= zmax, zmax the largest separation index
// within 2 r_s: r = r0(q) + t (mod n_k), t = 0 .. K-1, with
//   r0(q) = ceil(((2q+1) Q - zmax - P) / (2P)),  K = floor(zmax / P) + 1,
// entries past the row's own count stored as zero; when K >= n_k the row
// holds every column (r0 = 0, K = n_k).  One thread per stored entry walks,
// for every ring rho coupled to both rings, the contiguous arc of pixels p
// coupled to q and adds b(q,p) N^-1_p b(r,p) where p also couples to r.
// Unwrapped pixel indices (longitudes continued past 2 pi) keep every
// separation index in one piece.
//
// The preconditioner M^-1 x applied block by block (the diagonal ring
// blocks, block Jacobi): y = L^-T L^-1 x with the factor of
// sympix_factor_blocks, one warp per block.  Periodic band: the band rows by
// substitution along the band (one lane, from rows staged in shared memory),
// the border rows as dense dot products; the back substitution first takes
// the border rows' entries out of every band row, in parallel.
#include <cmath>

#include "sympix_internal.cuh"

namespace sympix {

__device__ __forceinline__ int fdiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
__device__ __forceinline__ int cdiv(int a, int b) { return -fdiv(-a, b); }

// z reduced to its nearest image in (-half, half] (the separation of the
// nearest copies of the two pixels, |dphi| <= pi).
__device__ __forceinline__ int near_image(int z, int half) {
    z %= 2 * half;
    if (z < 0) z += 2 * half;
    return z > half ? z - 2 * half : z;
}

__global__ void __launch_bounds__(128) k_sample_coupling(int64_t total, const CoupDesc *__restrict__ cds, int ncd,
                                                         const BlockDesc *__restrict__ blocks,
                                                         const PairEntry *__restrict__ entries, int64_t nslots,
                                                         int64_t npix, const double *__restrict__ tb,
                                                         const double *__restrict__ td,
                                                         const double *__restrict__ ninv, double *__restrict__ out) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= total) return;
    // the descriptor holding this entry (descriptors in offset order)
    int lo = 0, hi = ncd - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cds[mid].off <= gid) lo = mid;
        else hi = mid - 1;
    }
    const CoupDesc cd = cds[lo];
    const int64_t e = gid - cd.off;
    const int q = (int)(e / cd.K), t = (int)(e - (int64_t)q * cd.K);
    const int Z = (2 * q + 1) * cd.Q;
    const int ru = cd.dense ? t : cdiv(Z - cd.zmax - cd.P, 2 * cd.P) + t;  // column, unwrapped
    const int zqr = Z - (2 * ru + 1) * cd.P;
    double acc = 0.0;
    if (cd.dense || (zqr <= cd.zmax && zqr >= -cd.zmax)) {
        const BlockDesc bj = blocks[cd.bj], bk = blocks[cd.bk];
        const int64_t tbase = (int64_t)bj.op * nslots;
        const double *nv = ninv + (int64_t)bj.op * npix;
        // D^ between the two rings (the same support as B^)
        if (cd.dpair >= 0) {
            const PairEntry pd = entries[cd.dpair];
            // reduce the separation to the nearest image (|dphi| <= pi)
            const int64_t half = (int64_t)pd.P * pd.nrho;
            int64_t z = ((int64_t)(2 * q + 1) * pd.Q - (int64_t)(2 * ru + 1) * pd.P) % (2 * half);
            if (z < 0) z += 2 * half;
            if (z > half) z -= 2 * half;
            const int az = (int)(z < 0 ? -z : z);
            if (az <= pd.mmax) acc += td[tbase + pd.tab + ((az - pd.par) >> 1)];
        }
        for (int a = 0; a < bj.npairs; ++a) {
            const PairEntry p1 = entries[bj.pair0 + a];
            // the same neighbour ring in ring k's list
            int ib = -1;
            for (int b = 0; b < bk.npairs; ++b)
                if (entries[bk.pair0 + b].rho == p1.rho) {
                    ib = b;
                    break;
                }
            if (ib < 0) continue;
            const PairEntry p2 = entries[bk.pair0 + ib];
            // pixels p coupled to q: |Z1 - (2p+1) P1| <= m1, p unwrapped near q
            const int Z1 = (2 * q + 1) * p1.Q;
            const int plo = cdiv(Z1 - p1.mmax - p1.P, 2 * p1.P), phi = fdiv(Z1 + p1.mmax - p1.P, 2 * p1.P);
            // r's separation to p: z2 = (2 ru + 1) Q2 - (2 p + 1) P2 (the pair
            // constants of ring k with rho), the longitude difference of (r, p)
            // being pi z2 g2 / (n_k n_rho), taken at its nearest image
            const int Z2 = (2 * ru + 1) * p2.Q;
            int pm = plo % p1.nrho;
            if (pm < 0) pm += p1.nrho;
            // an arc as long as the ring (polar rings) holds every pixel once
            const int pend = min(phi, plo + p1.nrho - 1);
            double s = 0.0;
            for (int p = plo; p <= pend; ++p) {
                const int z1 = near_image(Z1 - (2 * p + 1) * p1.P, p1.P * p1.nrho);
                const int z2 = near_image(Z2 - (2 * p + 1) * p2.P, p2.P * p2.nrho);
                const int a1 = z1 < 0 ? -z1 : z1, a2 = z2 < 0 ? -z2 : z2;
                if (a1 <= p1.mmax && a2 <= p2.mmax) {
                    const double b1 = tb[tbase + p1.tab + ((a1 - p1.par) >> 1)];
                    const double b2 = tb[(int64_t)bk.op * nslots + p2.tab + ((a2 - p2.par) >> 1)];
                    s = fma(b1 * nv[p1.noff + (int64_t)pm * p1.nstride], b2, s);
                }
                if (++pm == p1.nrho) pm = 0;
            }
            acc += s;
        }
    }
    out[gid] = acc;
}

// y = M^-1 x on every planned block (one warp per block): forward
// substitution L z = x, back substitution L^T y = z, in FP64.  Blocks whose
// factorisation failed (info != 0) pass x through unchanged.  The band
// recurrences are sequential: 32 band rows at a time are staged into shared
// memory by the warp (with their reciprocal diagonals), then one lane runs
// the rows from there; the border rows (dense dot products) and their
// contribution to every band row of the back substitution are formed by the
// whole warp.
constexpr int kApplyRows = 32;

__global__ void __launch_bounds__(32) k_apply(const BlockDesc *__restrict__ blocks, const int32_t *__restrict__ info,
                                              const double *__restrict__ Lbuf, int dense_storage,
                                              const int64_t *__restrict__ roff, const int32_t *__restrict__ rstr,
                                              int64_t npix, int max_ring, const double *__restrict__ x,
                                              double *__restrict__ y) {
    extern __shared__ double smem_apply[];
    double *v = smem_apply;           // the block's vector, n values
    double *stg = v + max_ring;       // staged band rows
    const int bi = blockIdx.x, lane = threadIdx.x;
    const BlockDesc bd = blocks[bi];
    const int n = bd.n;
    const int64_t px0 = (int64_t)bd.op * npix + roff[bd.ring];
    const int64_t ps = rstr[bd.ring];
    const double *xin = x + px0;
    double *yout = y + px0;
    if (info[bi] != 0) {
        for (int c = lane; c < n; c += 32) yout[c * ps] = xin[c * ps];
        return;
    }
    for (int c = lane; c < n; c += 32) v[c] = xin[c * ps];
    __syncwarp();
    auto wsum = [](double s) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        return s;
    };
    const bool pband = !dense_storage && bd.format == SYMPIX_BLOCK_PBAND;
    if (pband) {
        const int w = bd.w, RL = w + 1, m = n - w;
        const double *band = Lbuf + bd.off_pband;
        const double *bord = band + (int64_t)n * RL;
        double *rinv = stg + (kApplyRows + w) * RL;  // 1 / L[i][i] of the staged rows
        // stage band rows [r0, r1) and their reciprocal diagonals
        auto stage = [&](int r0, int r1) {
            const int cnt = (r1 - r0) * RL;
            for (int e = lane; e < cnt; e += 32) stg[e] = band[(int64_t)r0 * RL + e];
            for (int r = lane; r < r1 - r0; r += 32) rinv[r] = 1.0 / band[(int64_t)(r0 + r) * RL];
            __syncwarp();
        };
        // forward: band rows i < m
        for (int r0 = 0; r0 < m; r0 += kApplyRows) {
            const int r1 = min(m, r0 + kApplyRows);
            stage(r0, r1);
            if (lane == 0)
                for (int i = r0; i < r1; ++i) {
                    const double *row = stg + (i - r0) * RL;
                    double s = v[i];
                    for (int d = 1; d <= w && d <= i; ++d) s = fma(-row[d], v[i - d], s);
                    v[i] = s * rinv[i - r0];
                }
            __syncwarp();
        }
        // forward: the border rows (dense dot products)
        for (int b = 0; b < w; ++b) {
            const int i = m + b;
            double s = 0.0;
            for (int c = lane; c < i; c += 32) s = fma(bord[(int64_t)b * n + c], v[c], s);
            s = wsum(s);
            if (lane == 0) v[i] = (v[i] - s) / bord[(int64_t)b * n + i];
            __syncwarp();
        }
        // back: the border rows (columns i >= m of L^T)
        if (lane == 0)
            for (int i = n - 1; i >= m; --i) {
                double s = v[i];
                for (int c = i + 1; c < n; ++c) s = fma(-bord[(int64_t)(c - m) * n + i], v[c], s);
                v[i] = s / bord[(int64_t)(i - m) * n + i];
            }
        __syncwarp();
        // their contribution to every band row: v_i -= sum_b L21[b][i] v_{m+b}
        for (int i = lane; i < m; i += 32) {
            double s = v[i];
            for (int b = 0; b < w; ++b) s = fma(-bord[(int64_t)b * n + i], v[m + b], s);
            v[i] = s;
        }
        __syncwarp();
        // back: band rows, from the bottom; a chunk needs the w rows below it
        for (int r1 = m; r1 > 0; r1 -= kApplyRows) {
            const int r0 = max(0, r1 - kApplyRows);
            const int re = min(m, r1 + w);
            stage(r0, re);
            if (lane == 0)
                for (int i = r1 - 1; i >= r0; --i) {
                    double s = v[i];
                    for (int d = 1; d <= w && i + d < m; ++d) s = fma(-stg[(i + d - r0) * RL + d], v[i + d], s);
                    v[i] = s * rinv[i - r0];
                }
            __syncwarp();
        }
    } else {
        const double *A = Lbuf + (dense_storage ? bd.off_dense : bd.off_pband);
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int c = lane; c < i; c += 32) s = fma(A[(int64_t)i * n + c], v[c], s);
            s = wsum(s);
            if (lane == 0) v[i] = (v[i] - s) / A[(int64_t)i * n + i];
            __syncwarp();
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = 0.0;
            for (int c = i + 1 + lane; c < n; c += 32) s = fma(A[(int64_t)c * n + i], v[c], s);
            s = wsum(s);
            if (lane == 0) v[i] = (v[i] - s) / A[(int64_t)i * n + i];
            __syncwarp();
        }
    }
    for (int c = lane; c < n; c += 32) yout[c * ps] = v[c];
}

static long gcd_h(long a, long b) {
    while (b) {
        long t = a % b;
        a = b;
        b = t;
    }
    return a;
}

}  // namespace sympix

using namespace sympix;

extern "C" int sympix_coupling_size(sympix_plan_t pl, int delta, size_t *bytes, int64_t *elements) {
    if (!pl) return set_error(SYMPIX_EINVAL, "sympix_coupling_size: NULL plan");
    if (pl->tiles) return set_error(SYMPIX_EUNSUPPORTED, "sympix_coupling_size: ring blocks only (k = 1)");
    if (delta < 1 || delta >= pl->grid->nrings)
        return set_error(SYMPIX_EINVAL, "sympix_coupling_size: ring offset %d out of [1, nrings)", delta);
    auto it = pl->coupling.find(delta);
    if (it == pl->coupling.end()) {
        it = pl->coupling.emplace(delta, CouplingPlan{}).first;  // built in place
        CouplingPlan &cp = it->second;
        const sympix_grid_s *g = pl->grid;
        const int nb = pl->ring1 - pl->ring0;
        int64_t off = 0;
        for (int o = 0; o < pl->nops; ++o) {
            const double r2 = std::min(2.0 * pl->r_s[o], kPi);
            const double h2 = std::sin(0.5 * r2), u2 = 2.0 * h2 * h2 * (1.0 + 1e-9);
            for (int j = pl->ring0; j + delta < pl->ring1; ++j) {
                const int k = j + delta;
                CoupDesc cd{};
                cd.bj = o * nb + (j - pl->ring0);
                cd.bk = o * nb + (k - pl->ring0);
                const long nj = g->nring[j], nk = g->nring[k], gg = gcd_h(nj, nk);
                cd.P = (int32_t)(nj / gg);
                cd.Q = (int32_t)(nk / gg);
                // largest separation index within 2 r_s (u grows with |z| up to |dphi| = pi)
                const double ta = g->theta[j], tb = g->theta[k];
                const double da = std::sin(0.5 * (ta - tb));
                const double base = 2.0 * da * da, st = 2.0 * std::sin(ta) * std::sin(tb);
                const long par = (cd.P + cd.Q) & 1, PQg = (long)cd.P * cd.Q * gg;
                const long mcap = PQg - ((PQg - par) & 1);
                long zmax = -1;
                for (long z = par; z <= mcap; z += 2) {
                    const double hh = std::sin(0.5 * kPi * (double)(z * gg) / ((double)nj * (double)nk));
                    if (r2 < kPi && base + st * hh * hh > u2) break;
                    zmax = z;
                }
                cd.zmax = (int32_t)std::max<long>(zmax, 0);
                const long K = zmax < 0 ? 1 : zmax / cd.P + 1;
                cd.dense = K >= nk ? 1 : 0;
                cd.K = (int32_t)(cd.dense ? nk : K);
                cd.n = (int32_t)nj;
                cd.off = off;
                cd.dpair = -1;
                const BlockDesc &bd = pl->blocks[cd.bj];
                for (int e = 0; e < bd.npairs; ++e)
                    if (pl->entries[bd.pair0 + e].rho == k) cd.dpair = (int32_t)(bd.pair0 + e);
                off += (int64_t)cd.n * cd.K;
                cp.desc.push_back(cd);
            }
        }
        cp.total = off;
        int rc;
        if ((rc = cp.d_desc.upload(cp.desc))) {
            pl->coupling.erase(it);
            return rc;
        }
        pl->all_d = true;  // D^ between rings needs d at every slot: the next table call evaluates it
    }
    if (bytes) *bytes = (size_t)it->second.total * sizeof(double);
    if (elements) *elements = it->second.total;
    return SYMPIX_OK;
}

extern "C" int sympix_coupling_layout(sympix_plan_t pl, int delta, int op, int ring, int64_t *offset, int32_t *geom) {
    if (!pl || !geom) return set_error(SYMPIX_EINVAL, "sympix_coupling_layout: NULL argument");
    if (pl->tiles) return set_error(SYMPIX_EUNSUPPORTED, "sympix_coupling_layout: ring blocks only (k = 1)");
    auto it = pl->coupling.find(delta);
    if (it == pl->coupling.end())
        return set_error(SYMPIX_EINVAL, "sympix_coupling_layout: call sympix_coupling_size(%d) first", delta);
    const int nb = pl->ring1 - pl->ring0;
    for (const CoupDesc &cd : it->second.desc) {
        const BlockDesc &bj = pl->blocks[cd.bj];
        if (bj.op != op || bj.ring != ring) continue;
        if (offset) *offset = cd.off;
        geom[0] = cd.n;
        geom[1] = pl->blocks[cd.bk].n;
        geom[2] = cd.K;
        geom[3] = cd.zmax;
        geom[4] = cd.P;
        geom[5] = cd.Q;
        geom[6] = cd.dense;
        return SYMPIX_OK;
    }
    (void)nb;
    return set_error(SYMPIX_EINVAL, "sympix_coupling_layout: no block (op %d, ring %d) for offset %d", op, ring, delta);
}

extern "C" int sympix_sample_coupling(sympix_plan_t pl, const double *ninv, int delta, double *out, void *stream) {
    if (!pl || !ninv || !out) return set_error(SYMPIX_EINVAL, "sympix_sample_coupling: NULL argument");
    if (pl->tiles) return set_error(SYMPIX_EUNSUPPORTED, "sympix_sample_coupling: ring blocks only (k = 1)");
    auto it = pl->coupling.find(delta);
    if (it == pl->coupling.end())
        return set_error(SYMPIX_EINVAL, "sympix_sample_coupling: call sympix_coupling_size(%d) first", delta);
    if (!pl->table_all_d)
        return set_error(SYMPIX_EINVAL,
                         "sympix_sample_coupling: call sympix_kernel_table after sympix_coupling_size "
                         "(the blocks between rings need d at every class)");
    cudaStream_t st = (cudaStream_t)stream;
    const CouplingPlan &cp = it->second;
    trace_mark(pl, st, nullptr);
    if (cp.total > 0)
        k_sample_coupling<<<(unsigned)((cp.total + 127) / 128), 128, 0, st>>>(
            cp.total, cp.d_desc.p, (int)cp.desc.size(), pl->d_blocks.p, pl->d_entries.p, pl->nslots,
            pl->grid->npix, pl->d_tab_b.p, pl->d_tab_d.p, ninv, out);
    trace_mark(pl, st, "k_sample_coupling");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "sympix_sample_coupling: launch");
    return SYMPIX_OK;
}

extern "C" int sympix_apply(sympix_plan_t pl, int storage, const double *blocks, const int32_t *info, const double *x,
                            double *y, void *stream) {
    if (!pl || !blocks || !info || !x || !y) return set_error(SYMPIX_EINVAL, "sympix_apply: NULL argument");
    if (pl->tiles) return set_error(SYMPIX_EUNSUPPORTED, "sympix_apply: ring blocks only (k = 1)");
    if (storage != SYMPIX_STORE_PBAND && storage != SYMPIX_STORE_DENSE)
        return set_error(SYMPIX_EINVAL, "sympix_apply: unknown storage %d", storage);
    if (x == y) return set_error(SYMPIX_EINVAL, "sympix_apply: x and y must not alias");
    cudaStream_t st = (cudaStream_t)stream;
    // the vector, then kApplyRows + w staged rows of w + 1 values and their
    // reciprocal diagonals (the widest periodic band planned)
    const size_t W1 = (size_t)pl->max_w + 1;
    const size_t smem = ((size_t)pl->grid->max_ring + (kApplyRows + W1) * (W1 + 1)) * sizeof(double);
    cudaFuncSetAttribute(k_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    trace_mark(pl, st, nullptr);
    k_apply<<<(unsigned)pl->blocks.size(), 32, smem, st>>>(pl->d_blocks.p, info, blocks,
                                                           storage == SYMPIX_STORE_DENSE ? 1 : 0, pl->d_ring_off.p,
                                                           pl->d_ring_stride.p, pl->grid->npix, pl->grid->max_ring,
                                                           x, y);
    trace_mark(pl, st, "k_apply");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "sympix_apply: launch");
    return SYMPIX_OK;
}
