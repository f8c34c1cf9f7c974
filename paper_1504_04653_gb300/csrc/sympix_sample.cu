// Block sampling: M_qr = D^_qr + sum_p B^_pq N^-1_p B^_pr for q, r on the
// block's ring (Eq. Dhat, Eq. system-rewritten; Y2 = Y1).
//
// For a coupled neighbour ring rho with pair constants (P, Q, mmax) pixel q
// couples to the pixels p with |z| <= mmax, z = (2q+1)Q - (2p+1)P (a
// contiguous arc), and r = q - d couples to p iff |z - 2dQ| <= mmax.  The
// kernel value of (q, p) is table[(|z| - par) / 2].  One thread owns one
// column q of its block and accumulates the whole lower band row
// M[q][q-d], d = 0..w, in registers: per pixel p it forms w_p = B^_pq N^-1_p
// once and adds w_p B^_pr to every d whose arc holds p.
//
// Arithmetic (template PREC):
//   0  FP64 products and sums;
//   1  FP32 products and sums (kernel values and N^-1 rounded to FP32);
//   2  split FP32: every value is an unevaluated sum hi + lo of two floats,
//      products by the exact FMA-based two-product, sums by two-sum with
//      renormalisation, i.e. ~44-bit significands on the FP32 pipes.
#include "sympix_arith.cuh"
#include "sympix_internal.cuh"

namespace sympix {

template <int PREC, bool DENSE_OUT>
void launch_pband(sympix_plan_t pl, const double *ninv, double *blocks, cudaStream_t st);

// N^-1 split once per call into FP32 (hi, lo) planes, so the contraction
// never converts from FP64 in its inner loops.
__global__ void k_split_ninv(int64_t count, const double *__restrict__ ninv, float *__restrict__ n32,
                             float *__restrict__ nlo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const F2 v = f2_from_bits(ninv[i]);
    n32[i] = v.hi;
    nlo[i] = v.lo;
}

// z reduced to (-half, half] (T2 = 2 half): the longitude separation index
// of a pixel pair on a pair of rings, as the kernel table is indexed.
__device__ __forceinline__ int64_t wrap_half(int64_t z, int64_t half, int64_t T2) {
    z %= T2;
    if (z > half) z -= T2;
    if (z <= -half) z += T2;
    return z;
}

// Small or wrapping blocks (every pixel pair of the ring may couple): one
// warp per element (q, r), its lanes sharing the pixels coupled to q on
// every coupled ring (the arc |z_q| <= mmax, or the whole ring when the
// support covers it), separation indices reduced to |dphi| <= pi; the
// partial sums meet in a fixed-order shuffle tree.  FP64.
__global__ void __launch_bounds__(32 * kDenseItemElems) k_sample_dense(const SampleItem *__restrict__ items,
                                                                   const BlockDesc *__restrict__ blocks,
                                                                   const PairEntry *__restrict__ entries,
                                                                   int64_t nslots, int64_t npix,
                                                                   const double *__restrict__ tb,
                                                                   const double *__restrict__ td,
                                                                   const double *__restrict__ ninv,
                                                                   double *__restrict__ out, int dense_storage) {
    const SampleItem it = items[blockIdx.x];
    const BlockDesc bd = blocks[it.block];
    const int n = bd.n, lane = threadIdx.x & 31;
    const int64_t eidx = (int64_t)it.q0 + (threadIdx.x >> 5);
    if (eidx >= (int64_t)n * n) return;  // uniform per warp
    const int q = (int)(eidx / n), r = (int)(eidx % n);
    const int64_t tbase = (int64_t)bd.op * nslots;
    const double *nv = ninv + (int64_t)bd.op * npix;
    double acc = 0.0;
    for (int e = 0; e < bd.npairs; ++e) {
        const PairEntry pe = entries[bd.pair0 + e];
        const int64_t P = pe.P, Q = pe.Q, m = pe.mmax;
        const int64_t half = P * pe.nrho;  // P Q g
        const int64_t T2 = 2 * half;
        const double *trow = tb + tbase + pe.tab;
        // the pixels coupled to q: the whole ring when the support covers it,
        // else the arc |z_q| <= mmax (each pixel once)
        const bool full = m >= half;
        const int64_t Zq = (2 * (int64_t)q + 1) * Q;
        int64_t lo = 0, hi = pe.nrho - 1;
        if (!full) {  // ceil((Z - m - P) / 2P) .. floor((Z + m - P) / 2P)
            const int64_t a = Zq - m - P, b = Zq + m - P, d2 = 2 * P;
            lo = a >= 0 ? (a + d2 - 1) / d2 : -((-a) / d2);
            hi = b >= 0 ? b / d2 : -((-b + d2 - 1) / d2);
        }
        // z of q and of r against pixel pm, reduced to (-half, half]; the
        // lane's next pixel is 32 on (mod nrho), so both z move by a fixed
        // step reduced once
        const int64_t nr = pe.nrho;
        int64_t pm = (lo + lane) % nr;
        if (pm < 0) pm += nr;
        const int64_t s32 = 32 % nr, dz = 2 * P * s32;
        int64_t zq = wrap_half(Zq - (2 * pm + 1) * P, half, T2);
        int64_t zr = wrap_half((2 * (int64_t)r + 1) * Q - (2 * pm + 1) * P, half, T2);
        for (int64_t pp = lo + lane; pp <= hi; pp += 32) {
            if (zq <= m && -zq <= m && zr <= m && -zr <= m) {
                const double bq = trow[((zq < 0 ? -zq : zq) - pe.par) >> 1];
                const double br = trow[((zr < 0 ? -zr : zr) - pe.par) >> 1];
                acc = fma(bq * nv[pe.noff + pm * pe.nstride], br, acc);
            }
            pm += s32;
            if (pm >= nr) pm -= nr;
            zq -= dz;
            if (zq <= -half) zq += T2;
            zr -= dz;
            if (zr <= -half) zr += T2;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) {
        int k = q > r ? q - r : r - q;
        if (n - k < k) k = n - k;
        if (k < bd.dK) acc += td[tbase + bd.dtab + k];
        out[(dense_storage ? bd.off_dense : bd.off_pband) + (int64_t)q * n + r] = acc;
    }
}

// Large dense-format blocks: one thread per element (q, r), 256 elements of
// a row-major block per CTA, every pixel of every coupled ring tested (the
// warp's 32 elements share their row q, so the q test is uniform), the
// separation index reduced to |dphi| <= pi.  FP64.
__global__ void __launch_bounds__(256) k_sample_dense_rows(const SampleItem *__restrict__ items,
                                                      const BlockDesc *__restrict__ blocks,
                                                      const PairEntry *__restrict__ entries, int64_t nslots,
                                                      int64_t npix, const double *__restrict__ tb,
                                                      const double *__restrict__ td, const double *__restrict__ ninv,
                                                      double *__restrict__ out, int dense_storage) {
    const SampleItem it = items[blockIdx.x];
    const BlockDesc bd = blocks[it.block];
    const int n = bd.n;
    const int64_t eidx = (int64_t)it.q0 + threadIdx.x;
    if (eidx >= (int64_t)n * n) return;
    const int q = (int)(eidx / n), r = (int)(eidx % n);
    const int64_t tbase = (int64_t)bd.op * nslots;
    const double *nv = ninv + (int64_t)bd.op * npix;
    double acc = 0.0;
    for (int e = 0; e < bd.npairs; ++e) {
        const PairEntry pe = entries[bd.pair0 + e];
        const int64_t P = pe.P, Q = pe.Q, m = pe.mmax;
        const int64_t half = P * pe.nrho;  // P Q g
        const int64_t T2 = 2 * half;
        const double *trow = tb + tbase + pe.tab;
        // z of q and of r against pixel p, reduced to (-half, half], moved
        // by -2P per pixel
        int64_t zq = wrap_half((2 * (int64_t)q + 1) * Q - P, half, T2);
        int64_t zr = wrap_half((2 * (int64_t)r + 1) * Q - P, half, T2);
        for (int p = 0; p < pe.nrho; ++p) {
            if (zq <= m && -zq <= m && zr <= m && -zr <= m) {
                const double bq = trow[((zq < 0 ? -zq : zq) - pe.par) >> 1];
                const double br = trow[((zr < 0 ? -zr : zr) - pe.par) >> 1];
                acc = fma(bq * nv[pe.noff + (int64_t)p * pe.nstride], br, acc);
            }
            zq -= 2 * P;
            if (zq <= -half) zq += T2;
            zr -= 2 * P;
            if (zr <= -half) zr += T2;
        }
    }
    int k = q > r ? q - r : r - q;
    if (n - k < k) k = n - k;
    if (k < bd.dK) acc += td[tbase + bd.dtab + k];
    out[(dense_storage ? bd.off_dense : bd.off_pband) + (int64_t)q * n + r] = acc;
}

}  // namespace sympix

using namespace sympix;

extern "C" int sympix_sample_blocks(sympix_plan_t pl, const double *ninv, int precision, int storage,
                                    double *blocks, void *stream) {
    if (!pl || !ninv || !blocks) return set_error(SYMPIX_EINVAL, "sympix_sample_blocks: NULL argument");
    if (precision < SYMPIX_PREC_FP64 || precision > SYMPIX_PREC_FP32X2)
        return set_error(SYMPIX_EINVAL, "sympix_sample_blocks: unknown precision %d", precision);
    if (storage != SYMPIX_STORE_PBAND && storage != SYMPIX_STORE_DENSE)
        return set_error(SYMPIX_EINVAL, "sympix_sample_blocks: unknown storage %d", storage);
    if (!pl->table_ready)
        return set_error(SYMPIX_EINVAL, "sympix_sample_blocks: sympix_kernel_table has not been called");
    cudaStream_t st = (cudaStream_t)stream;
    const bool dense = storage == SYMPIX_STORE_DENSE;
    trace_mark(pl, st, nullptr);
    if (dense) SPX_CUDA(cudaMemsetAsync(blocks, 0, (size_t)pl->size_dense * sizeof(double), st));
    if (precision != SYMPIX_PREC_FP64) {
        const int64_t cnt = (int64_t)pl->nops * pl->grid->npix;
        k_split_ninv<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(cnt, ninv, pl->d_ninv32.p, pl->d_ninvlo.p);
        trace_mark(pl, st, "k_split_ninv");
    }
    if (pl->tiles) {  // band blocks of a DP grid
        int rc = launch_tiles(pl, ninv, precision, blocks, st);
        if (rc) return rc;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_error(e, "sympix_sample_blocks: launch");
        return SYMPIX_OK;
    }
    if (precision == SYMPIX_PREC_FP64) {
        dense ? launch_pband<0, true>(pl, ninv, blocks, st) : launch_pband<0, false>(pl, ninv, blocks, st);
    } else if (precision == SYMPIX_PREC_FP32) {
        dense ? launch_pband<1, true>(pl, ninv, blocks, st) : launch_pband<1, false>(pl, ninv, blocks, st);
    } else {
        dense ? launch_pband<2, true>(pl, ninv, blocks, st) : launch_pband<2, false>(pl, ninv, blocks, st);
    }
    trace_mark(pl, st, "k_sample_pband");
    if (!pl->items_dense.empty())
        k_sample_dense<<<(unsigned)pl->items_dense.size(), 32 * kDenseItemElems, 0, st>>>(
            pl->d_items_dense.p, pl->d_blocks.p, pl->d_entries.p, pl->nslots, pl->grid->npix, pl->d_tab_b.p,
            pl->d_tab_d.p, ninv, blocks, dense ? 1 : 0);
    if (!pl->items_dense_rows.empty())
        k_sample_dense_rows<<<(unsigned)pl->items_dense_rows.size(), 256, 0, st>>>(
            pl->d_items_dense_rows.p, pl->d_blocks.p, pl->d_entries.p, pl->nslots, pl->grid->npix, pl->d_tab_b.p,
            pl->d_tab_d.p, ninv, blocks, dense ? 1 : 0);
    trace_mark(pl, st, "k_sample_dense");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "sympix_sample_blocks: launch");
    return SYMPIX_OK;
}
