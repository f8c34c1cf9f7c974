// Blocks on DP grids (k > 1): one dense block per band of k rings under tile
// adjacency (Sec. 2.3 tiling; Sec. 4.2, the locality approximation: D^_ij
// and B^_ij vanish unless pixels i and j lie in the same or neighbouring
// k x k tiles).  Reading of "neighbouring": tiles of bands at most one apart
// in latitude whose closed longitude arcs [a/T, (a+1)/T] of a turn meet, and
// every two tiles of a polar band (they meet across the pole).
//
// The kernel values come from the same class table as the ring blocks: the
// separation of pixel c of a ring of n_a pixels and pixel p of a ring of n_b
// depends only on the ring pair and |z|, z = (2c+1) Q - (2p+1) P (P = n_a/g,
// Q = n_b/g, g = gcd), so a plan over a DP grid stores, per canonical ring
// pair of neighbouring bands, the classes up to the largest |z| any
// tile-coupled pixel pair reaches.  The sampler then forms each k^2 x k^2
// tile pair of a band block as a small dense product over the pixels of the
// tiles coupled to both, B_a^T diag(N^-1) B_a2, plus D^ where the two tiles
// are neighbours.
#include <algorithm>
#include <set>
#include <unordered_map>

#include "sympix_factor_kernels.cuh"

namespace sympix {

// Tiles of a band of Tb tiles coupled to tile a of a band of Ta tiles: the
// circular range lo, lo+1, ..., lo+cnt-1 (mod Tb).  The arcs meet iff
// ceil(a Tb / Ta) - 1 <= b <= floor((a+1) Tb / Ta) for some turn of b.
__host__ __device__ inline void tile_range(long a, long Ta, long Tb, bool all, long *lo, long *cnt) {
    if (!all) {
        const long l = (a * Tb + Ta - 1) / Ta - 1, h = ((a + 1) * Tb) / Ta;
        if (h - l + 1 < Tb) {
            *lo = (l + Tb) % Tb;
            *cnt = h - l + 1;
            return;
        }
    }
    *lo = 0;
    *cnt = Tb;
}

// z reduced to (-half, half]
__host__ __device__ inline long reduce_z(long z, long half) {
    const long t = 2 * half;
    z %= t;
    if (z <= -half) z += t;
    if (z > half) z -= t;
    return z;
}

static long gcd_l(long a, long b) {
    while (b) {
        const long t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Largest |z| over the tile-coupled pixel pairs of a ring of na pixels
// (band of Ta = na / k tiles) and a ring of nb pixels.
long tile_pair_mmax(int na, int nb, int k, bool all) {
    const long g = gcd_l(na, nb), P = na / g, Q = nb / g, half = P * Q * g;
    const long Ta = na / k, Tb = nb / k;
    long m = -1;
    for (long a = 0; a < Ta; ++a) {
        long lo, cnt;
        tile_range(a, Ta, Tb, all, &lo, &cnt);
        for (long i = 0; i < cnt; ++i) {
            const long b = (lo + i) % Tb;
            for (long c = a * k; c < a * k + k; ++c)
                for (long p = b * k; p < b * k + k; ++p) {
                    const long z = reduce_z((2 * c + 1) * Q - (2 * p + 1) * P, half);
                    m = std::max(m, z < 0 ? -z : z);
                }
        }
    }
    return m;
}

// Band blocks, their per-block tables and the lower tile pairs with some
// coupling, for bands [g0, g1) and every operator.
int plan_tile_blocks(sympix_plan_t pl, const std::unordered_map<int64_t, int> &index, int g0, int g1) {
    const sympix_grid_s *grid = pl->grid;
    const int N = grid->nrings, k = grid->k, G = N / k;
    const std::vector<int32_t> &nr = grid->nring;
    auto band_start = [&](int g) {
        int64_t s = grid->offset[g * k];
        for (int r = g * k; r < g * k + k; ++r) s = std::min<int64_t>(s, grid->offset[r]);
        return s;
    };
    // ring of band g at row order r (pixel c of it at row c k + r)
    auto ring_at = [&](int g, int r) {
        const int64_t s = band_start(g);
        for (int j = g * k; j < g * k + k; ++j)
            if (grid->offset[j] - s == r) return j;
        return -1;
    };
    int64_t off = 0;
    for (int o = 0; o < pl->nops; ++o)
        for (int g = g0; g < g1; ++g) {
            const int n = nr[g * k];
            const int64_t K = (int64_t)k * n;
            if (K > 16384)  // also keeps every separation index z of the sampler within 32 bits
                return set_error(SYMPIX_EUNSUPPORTED, "sympix_support: band %d has %lld pixels, above 16384", g,
                                 (long long)K);
            TileBlock tb{};
            tb.op = o;
            tb.g = g;
            tb.K = (int32_t)K;
            tb.T = n / k;
            tb.k = k;
            tb.G = G;
            tb.meta0 = (int64_t)pl->tile_slot0.size();
            for (int d = 0; d < 3; ++d) {
                const int gd = g - 1 + d;
                tb.gnb[d] = (gd >= 0 && gd < G) ? gd : -1;
                if (tb.gnb[d] < 0) {
                    for (int i = 0; i < k * k; ++i) pl->tile_slot0.push_back(0);
                    continue;
                }
                const int nd = nr[gd * k];
                const long gg = gcd_l(n, nd);
                tb.Tnb[d] = nd / k;
                tb.P[d] = (int32_t)(n / gg);
                tb.Q[d] = (int32_t)(nd / gg);
                tb.par[d] = (tb.P[d] + tb.Q[d]) & 1;
                tb.half[d] = (int64_t)tb.P[d] * tb.Q[d] * gg;
                for (int r = 0; r < k; ++r)
                    for (int r2 = 0; r2 < k; ++r2) {
                        const auto ab = canon_pair(N, ring_at(g, r), ring_at(gd, r2));
                        pl->tile_slot0.push_back(pl->pairs[index.at((int64_t)ab.first * N + ab.second)].slot0);
                    }
            }
            for (int d = 0; d < 3; ++d)
                for (int r2 = 0; r2 < k; ++r2)
                    pl->tile_noff.push_back(tb.gnb[d] < 0 ? 0 : grid->offset[ring_at(tb.gnb[d], r2)]);
            off = (off + 3) & ~int64_t(3);
            tb.off = off;
            off += K * K;

            BlockDesc bd{};
            bd.op = o;
            bd.ring = g;
            bd.n = (int32_t)K;
            bd.w = (int32_t)(K - 1);
            bd.format = SYMPIX_BLOCK_DENSE;
            bd.dtab = -1;
            bd.off_pband = bd.off_dense = tb.off;
            pl->elems_pband += K * (K + 1) / 2;
            pl->elems_dense += K * (K + 1) / 2;
            const int bi = (int)pl->blocks.size();
            pl->blocks.push_back(bd);

            // lower tile pairs (a2 <= a) with D^ or a common neighbour tile
            const bool polar = g == 0 || g == G - 1;
            for (long a = 0; a < tb.T; ++a) {
                std::set<long> mates;
                long lo, cnt;
                tile_range(a, tb.T, tb.T, polar, &lo, &cnt);
                for (long i = 0; i < cnt; ++i) mates.insert((lo + i) % tb.T);
                for (int d = 0; d < 3; ++d) {
                    if (tb.gnb[d] < 0) continue;
                    const bool all = tb.gnb[d] == g && polar;
                    long lb, cb;
                    tile_range(a, tb.T, tb.Tnb[d], all, &lb, &cb);
                    for (long i = 0; i < cb; ++i) {
                        const long b = (lb + i) % tb.Tnb[d];
                        long la, ca;
                        tile_range(b, tb.Tnb[d], tb.T, all, &la, &ca);
                        for (long t = 0; t < ca; ++t) mates.insert((la + t) % tb.T);
                    }
                }
                for (long a2 : mates) {
                    if (a2 > a) continue;
                    pl->tile_items.push_back({bi, (int32_t)a, (int32_t)a2, 0});
                    // work of the item: k^2 x k^2 multiply-adds per pixel of a
                    // common tile (k^2 pixels), two gathered products per pixel pair
                    int64_t common = 0;
                    for (int d = 0; d < 3; ++d) {
                        if (tb.gnb[d] < 0) continue;
                        const bool all = tb.gnb[d] == g && polar;
                        long l1, c1, l2, c2;
                        tile_range(a, tb.T, tb.Tnb[d], all, &l1, &c1);
                        tile_range(a2, tb.T, tb.Tnb[d], all, &l2, &c2);
                        for (long i = 0; i < c1; ++i)
                            if (((l1 + i) % tb.Tnb[d] - l2 + tb.Tnb[d]) % tb.Tnb[d] < c2) ++common;
                    }
                    const int64_t k2 = (int64_t)k * k;
                    pl->ntriples += common * k2 * k2 * k2;
                    pl->nmults += common * 2 * k2 * k2;
                }
            }
            pl->tile_blocks.push_back(tb);
        }
    pl->size_pband = off;
    pl->size_dense = off;
    return SYMPIX_OK;
}

// -- the sampler ---------------------------------------------------------------
// Kernel values, N^-1 and accumulation in one arithmetic: FP64, FP32, or
// split FP32 (hi + lo tables and maps).
struct TileSrcF64 {
    typedef double V;
    const double *b, *d, *nv;
    __device__ V tb(int64_t i) const { return b[i]; }
    __device__ V td(int64_t i) const { return d[i]; }
    __device__ V n(int64_t i) const { return nv[i]; }
    __device__ static V fma_(V x, V y, V z) { return fma(x, y, z); }
    __device__ static V mul(V x, V y) { return x * y; }
    __device__ static V add(V x, V y) { return x + y; }
    __device__ static double out(V x) { return x; }
};
struct TileSrcF32 {
    typedef float V;
    const float *b, *d, *nv;
    __device__ V tb(int64_t i) const { return b[i]; }
    __device__ V td(int64_t i) const { return d[i]; }
    __device__ V n(int64_t i) const { return nv[i]; }
    __device__ static V fma_(V x, V y, V z) { return fmaf(x, y, z); }
    __device__ static V mul(V x, V y) { return x * y; }
    __device__ static V add(V x, V y) { return x + y; }
    __device__ static double out(V x) { return f32_to_f64_bits(x); }
};
struct TileSrcF2 {
    typedef DF V;
    const float *b, *blo, *d, *dlo, *nv, *nvlo;
    __device__ V tb(int64_t i) const { return DF(b[i], blo[i]); }
    __device__ V td(int64_t i) const { return DF(d[i], dlo[i]); }
    __device__ V n(int64_t i) const { return DF(nv[i], nvlo[i]); }
    __device__ static V fma_(V x, V y, V z) { return df_fma(x, y, z); }
    __device__ static V mul(V x, V y) { return x * y; }
    __device__ static V add(V x, V y) { return x + y; }
    __device__ static double out(V x) { return elem_to_f64(x); }
};

// z = (2c+1) Q - (2p+1) P of pixels c < n_a, p < n_b lies in (-2 half,
// 2 half) (half = n_a n_b / g), so one correction reduces it to
// (-half, half].
__device__ __forceinline__ int reduce_z_near(int z, int half) {
    return z > half ? z - 2 * half : (z <= -half ? z + 2 * half : z);
}

// One CTA per lower tile pair (a, a2) of a band block: the k^2 x k^2 tile
// of rows a and columns a2 (and its transpose), summed over the pixels p of
// every tile coupled to both, one such tile at a time: Ba[p][i] =
// b(p, row i) N^-1_p and Bb[p][j] = b(p, column j) are gathered from the
// class table into shared memory, then each of the 16 x 16 threads adds an
// MU x MU piece of Ba^T Bb (MU = ceil(k^2 / 16)).  Band sizes stay below
// 2^15 pixels, so every z fits 32 bits.
template <class S, int K>
__global__ void __launch_bounds__(256) k_sample_tiles(const TileItem *__restrict__ items,
                                                      const TileBlock *__restrict__ tbs,
                                                      const int64_t *__restrict__ slot0s,
                                                      const int64_t *__restrict__ noffs, int64_t nslots,
                                                      int64_t npix, S src, double *__restrict__ out) {
    typedef typename S::V V;
    constexpr int KK = K * K, MU = (KK + 15) / 16;
    extern __shared__ __align__(16) unsigned char tile_smem[];
    V *Ba = reinterpret_cast<V *>(tile_smem), *Bb = Ba + KK * KK;  // [p][row], [p][column]
    const TileItem it = items[blockIdx.x];
    const TileBlock tb = tbs[it.block];
    const int64_t tbase = (int64_t)tb.op * nslots, nbase = (int64_t)tb.op * npix;
    const int64_t *slot0 = slot0s + tb.meta0;
    const int64_t *noff = noffs + tb.meta0 / K;  // 3 k^2 slots, 3 k offsets per block
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    V acc[MU][MU];
#pragma unroll
    for (int u = 0; u < MU; ++u)
#pragma unroll
        for (int v = 0; v < MU; ++v) acc[u][v] = V(0);
    const bool polar = tb.g == 0 || tb.g == tb.G - 1;
    for (int d = 0; d < 3; ++d) {
        if (tb.gnb[d] < 0) continue;
        const bool all = tb.gnb[d] == tb.g && polar;
        const long Td = tb.Tnb[d];
        long l1, c1, l2, c2;
        tile_range(it.a, tb.T, Td, all, &l1, &c1);
        tile_range(it.a2, tb.T, Td, all, &l2, &c2);
        const int P = tb.P[d], Q = tb.Q[d], half = (int)tb.half[d], par = tb.par[d];
        for (long i1 = 0; i1 < c1; ++i1) {
            long b = l1 + i1;
            if (b >= Td) b -= Td;
            long rel = b - l2;
            if (rel < 0) rel += Td;
            if (rel >= c2) continue;  // not coupled to tile a2
            __syncthreads();
            for (int e = threadIdx.x; e < KK * KK; e += 256) {
                const int pi = e / KK, qi = e % KK;
                const int r2 = pi % K, r = qi % K;
                const int cp = (int)b * K + pi / K;
                const int ca = it.a * K + qi / K, cb = it.a2 * K + qi / K;
                const V nv = src.n(nbase + noff[d * K + r2] + (int64_t)cp * K);
                int za = reduce_z_near((2 * ca + 1) * Q - (2 * cp + 1) * P, half);
                int zb = reduce_z_near((2 * cb + 1) * Q - (2 * cp + 1) * P, half);
                za = za < 0 ? -za : za;
                zb = zb < 0 ? -zb : zb;
                const int64_t s0 = tbase + slot0[(d * K + r) * K + r2];
                Ba[pi * KK + qi] = S::mul(src.tb(s0 + ((za - par) >> 1)), nv);
                Bb[pi * KK + qi] = src.tb(s0 + ((zb - par) >> 1));
            }
            __syncthreads();
#pragma unroll 4
            for (int pi = 0; pi < KK; ++pi) {
                V x[MU], y[MU];
#pragma unroll
                for (int u = 0; u < MU; ++u) {
                    x[u] = MU * ty + u < KK ? Ba[pi * KK + MU * ty + u] : V(0);
                    y[u] = MU * tx + u < KK ? Bb[pi * KK + MU * tx + u] : V(0);
                }
#pragma unroll
                for (int u = 0; u < MU; ++u)
#pragma unroll
                    for (int v = 0; v < MU; ++v) acc[u][v] = S::fma_(x[u], y[v], acc[u][v]);
            }
        }
    }
    // D^ where the two tiles are neighbours (same band: a2 = a, a +- 1, or any in a polar band)
    long ld, cd;
    tile_range(it.a, tb.T, tb.T, polar, &ld, &cd);
    long rel = it.a2 - ld;
    if (rel < 0) rel += tb.T;
    const bool dcoup = rel < cd;
    const int64_t Kr = tb.K;
#pragma unroll
    for (int u = 0; u < MU; ++u)
#pragma unroll
        for (int v = 0; v < MU; ++v) {
            const int i = MU * ty + u, j = MU * tx + v;
            if (i >= KK || j >= KK) continue;
            V val = acc[u][v];
            if (dcoup) {
                const int ci = it.a * K + i / K, cj = it.a2 * K + j / K;
                int z = reduce_z_near(2 * (ci - cj), (int)tb.half[1]);
                z = z < 0 ? -z : z;
                val = S::add(val, src.td(tbase + slot0[(K + i % K) * K + j % K] + (z >> 1)));
            }
            const int64_t row = (int64_t)it.a * KK + i, col = (int64_t)it.a2 * KK + j;
            const double w = S::out(val);
            out[tb.off + row * Kr + col] = w;
            if (it.a != it.a2) out[tb.off + col * Kr + row] = w;
        }
}

template <class S, int K>
static void launch_tiles_k(sympix_plan_t pl, S src, double *blocks, cudaStream_t st) {
    const size_t smem = (size_t)2 * K * K * K * K * sizeof(typename S::V);
    cudaFuncSetAttribute(k_sample_tiles<S, K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_sample_tiles<S, K><<<(unsigned)pl->tile_items.size(), 256, smem, st>>>(
        pl->d_tile_items.p, pl->d_tile_blocks.p, pl->d_tile_slot0.p, pl->d_tile_noff.p, pl->nslots, pl->grid->npix,
        src, blocks);
}

template <class S>
static void launch_tiles_with(sympix_plan_t pl, S src, double *blocks, cudaStream_t st) {
    switch (pl->grid->k) {
    case 2: launch_tiles_k<S, 2>(pl, src, blocks, st); break;
    case 3: launch_tiles_k<S, 3>(pl, src, blocks, st); break;
    case 4: launch_tiles_k<S, 4>(pl, src, blocks, st); break;
    case 5: launch_tiles_k<S, 5>(pl, src, blocks, st); break;
    case 6: launch_tiles_k<S, 6>(pl, src, blocks, st); break;
    case 7: launch_tiles_k<S, 7>(pl, src, blocks, st); break;
    default: launch_tiles_k<S, 8>(pl, src, blocks, st); break;
    }
}

// Zeroes the blocks, then writes every tile pair with some coupling.
int launch_tiles(sympix_plan_t pl, const double *ninv, int precision, double *blocks, cudaStream_t st) {
    SPX_CUDA(cudaMemsetAsync(blocks, 0, (size_t)pl->size_pband * sizeof(double), st));
    if (pl->tile_items.empty()) return SYMPIX_OK;
    if (precision == SYMPIX_PREC_FP64)
        launch_tiles_with(pl, TileSrcF64{pl->d_tab_b.p, pl->d_tab_d.p, ninv}, blocks, st);
    else if (precision == SYMPIX_PREC_FP32)
        launch_tiles_with(pl, TileSrcF32{pl->d_tab_b32.p, pl->d_tab_d32.p, pl->d_ninv32.p}, blocks, st);
    else
        launch_tiles_with(pl,
                          TileSrcF2{pl->d_tab_b32.p, pl->d_tab_blo.p, pl->d_tab_d32.p, pl->d_tab_dlo.p,
                                    pl->d_ninv32.p, pl->d_ninvlo.p},
                          blocks, st);
    trace_mark(pl, st, "k_sample_tiles");
    return SYMPIX_OK;
}

}  // namespace sympix
