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
#include "sympix_internal.cuh"

namespace sympix {

struct F2 {
    float hi, lo;
};

__device__ __forceinline__ F2 f2_fast_two_sum(float a, float b) {
    float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
    float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return f2_fast_two_sum(p, e);
}

__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    float s = a.hi + b.hi;
    float bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    e += a.lo + b.lo;
    return f2_fast_two_sum(s, e);
}

__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
__device__ __forceinline__ int ceil_div(int a, int b) { return -floor_div(-a, b); }

template <int PREC>
struct Arith;

template <>
struct Arith<0> {
    typedef double V;
    __device__ static V zero() { return 0.0; }
    __device__ static V tab(const double *tb, const float *, const float *, int64_t i) { return tb[i]; }
    __device__ static V from(double x) { return x; }
    __device__ static V mul(V a, V b) { return a * b; }
    __device__ static V fma_(V a, V b, V c) { return fma(a, b, c); }
    __device__ static double to_double(V a) { return a; }
};

template <>
struct Arith<1> {
    typedef float V;
    __device__ static V zero() { return 0.0f; }
    __device__ static V tab(const double *, const float *t32, const float *, int64_t i) { return t32[i]; }
    __device__ static V from(double x) { return (float)x; }
    __device__ static V mul(V a, V b) { return a * b; }
    __device__ static V fma_(V a, V b, V c) { return fmaf(a, b, c); }
    __device__ static double to_double(V a) { return (double)a; }
};

template <>
struct Arith<2> {
    typedef F2 V;
    __device__ static V zero() { return {0.0f, 0.0f}; }
    __device__ static V tab(const double *, const float *t32, const float *tlo, int64_t i) {
        return {t32[i], tlo[i]};
    }
    __device__ static V from(double x) {
        float h = (float)x;
        return {h, (float)(x - (double)h)};
    }
    __device__ static V mul(V a, V b) { return f2_mul(a, b); }
    __device__ static V fma_(V a, V b, V c) { return f2_add(f2_mul(a, b), c); }
    __device__ static double to_double(V a) { return (double)a.hi + (double)a.lo; }
};

template <int PREC, int WMAX, bool DENSE_OUT>
__global__ void __launch_bounds__(128) k_sample_pband(const SampleItem *__restrict__ items,
                                                      const BlockDesc *__restrict__ blocks,
                                                      const PairEntry *__restrict__ entries, int64_t nslots,
                                                      int64_t npix, const double *__restrict__ tb,
                                                      const float *__restrict__ tb32, const float *__restrict__ tblo,
                                                      const double *__restrict__ td, const double *__restrict__ ninv,
                                                      double *__restrict__ out) {
    typedef Arith<PREC> A;
    typedef typename A::V V;
    const SampleItem it = items[blockIdx.x];
    const BlockDesc bd = blocks[it.block];
    const int q = it.q0 + (int)threadIdx.x;
    if (q >= bd.n) return;
    const int w = bd.w;
    V acc[WMAX + 1];
#pragma unroll
    for (int d = 0; d <= WMAX; ++d) acc[d] = A::zero();
    const int64_t tbase = (int64_t)bd.op * nslots;
    const double *nv = ninv + (int64_t)bd.op * npix;
    for (int e = 0; e < bd.npairs; ++e) {
        const PairEntry pe = entries[bd.pair0 + e];
        const int P = pe.P, Q = pe.Q, m = pe.mmax, par = pe.par;
        const int Z = (2 * q + 1) * Q;
        const int p_lo = ceil_div(Z - m - P, 2 * P);
        const int p_hi = floor_div(Z + m - P, 2 * P);
        const int64_t tab = tbase + pe.tab;
        for (int p = p_lo; p <= p_hi; ++p) {
            const int z = Z - (2 * p + 1) * P;
            const int lq = (abs(z) - par) >> 1;
            int pm = p % pe.nrho;
            if (pm < 0) pm += pe.nrho;
            const V wq = A::mul(A::tab(tb, tb32, tblo, tab + lq), A::from(nv[pe.noff + (int64_t)pm * pe.nstride]));
            const int d_lo = max(0, ceil_div(z - m, 2 * Q));
            const int d_hi = min(w, floor_div(z + m, 2 * Q));
#pragma unroll
            for (int d = 0; d <= WMAX; ++d) {
                if (d >= d_lo && d <= d_hi) {
                    const int lr = (abs(z - 2 * d * Q) - par) >> 1;
                    acc[d] = A::fma_(wq, A::tab(tb, tb32, tblo, tab + lr), acc[d]);
                }
            }
        }
    }
    const int n = bd.n;
#pragma unroll
    for (int d = 0; d <= WMAX; ++d) {
        if (d <= w) {
            double v = A::to_double(acc[d]);
            if (d < bd.dK) v += td[tbase + bd.dtab + d];
            if (DENSE_OUT) {
                int r = q - d;
                if (r < 0) r += n;
                out[bd.off_dense + (int64_t)q * n + r] = v;
                out[bd.off_dense + (int64_t)r * n + q] = v;
            } else {
                out[bd.off_pband + (int64_t)q * (w + 1) + d] = v;
            }
        }
    }
}

// Small or wrapping blocks (every pixel pair of the ring may couple): one
// thread per element (q, r), every pixel of every coupled ring tested, the
// separation index reduced to |dphi| <= pi.  FP64.
__global__ void __launch_bounds__(256) k_sample_dense(const SampleItem *__restrict__ items,
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
        for (int p = 0; p < pe.nrho; ++p) {
            int64_t zq = ((2 * q + 1) * Q - (2 * (int64_t)p + 1) * P) % T2;
            if (zq > half) zq -= T2;
            if (zq <= -half) zq += T2;
            if (zq > m || -zq > m) continue;
            int64_t zr = ((2 * r + 1) * Q - (2 * (int64_t)p + 1) * P) % T2;
            if (zr > half) zr -= T2;
            if (zr <= -half) zr += T2;
            if (zr > m || -zr > m) continue;
            const double bq = trow[((zq < 0 ? -zq : zq) - pe.par) >> 1];
            const double br = trow[((zr < 0 ? -zr : zr) - pe.par) >> 1];
            acc = fma(bq * nv[pe.noff + (int64_t)p * pe.nstride], br, acc);
        }
    }
    int k = q > r ? q - r : r - q;
    if (n - k < k) k = n - k;
    if (k < bd.dK) acc += td[tbase + bd.dtab + k];
    out[(dense_storage ? bd.off_dense : bd.off_pband) + (int64_t)q * n + r] = acc;
}

}  // namespace sympix

using namespace sympix;

template <int PREC, bool DENSE_OUT>
static void launch_pband(sympix_plan_t pl, const double *ninv, double *blocks, cudaStream_t st) {
    const int64_t npix = pl->grid->npix;
    const int wm[4] = {8, 16, 32, 64};
    for (int b = 0; b < 4; ++b) {
        const size_t ni = pl->items_pband[b].size();
        if (!ni) continue;
#define SPX_ARGS                                                                                            \
    pl->d_items_pband[b].p, pl->d_blocks.p, pl->d_entries.p, pl->nslots, npix, pl->d_tab_b.p, pl->d_tab_b32.p, \
        pl->d_tab_blo.p, pl->d_tab_d.p, ninv, blocks
        switch (wm[b]) {
            case 8: k_sample_pband<PREC, 8, DENSE_OUT><<<(unsigned)ni, 128, 0, st>>>(SPX_ARGS); break;
            case 16: k_sample_pband<PREC, 16, DENSE_OUT><<<(unsigned)ni, 128, 0, st>>>(SPX_ARGS); break;
            case 32: k_sample_pband<PREC, 32, DENSE_OUT><<<(unsigned)ni, 128, 0, st>>>(SPX_ARGS); break;
            default: k_sample_pband<PREC, 64, DENSE_OUT><<<(unsigned)ni, 128, 0, st>>>(SPX_ARGS); break;
        }
#undef SPX_ARGS
    }
}

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
    if (dense) SPX_CUDA(cudaMemsetAsync(blocks, 0, (size_t)pl->size_dense * sizeof(double), st));
    if (precision == SYMPIX_PREC_FP64) {
        dense ? launch_pband<0, true>(pl, ninv, blocks, st) : launch_pband<0, false>(pl, ninv, blocks, st);
    } else if (precision == SYMPIX_PREC_FP32) {
        dense ? launch_pband<1, true>(pl, ninv, blocks, st) : launch_pband<1, false>(pl, ninv, blocks, st);
    } else {
        dense ? launch_pband<2, true>(pl, ninv, blocks, st) : launch_pband<2, false>(pl, ninv, blocks, st);
    }
    if (!pl->items_dense.empty())
        k_sample_dense<<<(unsigned)pl->items_dense.size(), 256, 0, st>>>(
            pl->d_items_dense.p, pl->d_blocks.p, pl->d_entries.p, pl->nslots, pl->grid->npix, pl->d_tab_b.p,
            pl->d_tab_d.p, ninv, blocks, dense ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "sympix_sample_blocks: launch");
    return SYMPIX_OK;
}
