#pragma once
// Block-sampling kernels, included by one translation unit per arithmetic.
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

__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
__device__ __forceinline__ int ceil_div(int a, int b) { return -floor_div(-a, b); }

// Table loads per arithmetic: the FP64 table, its FP32 rounding, or the
// FP32 (hi, lo) split of each FP64 value.
template <int PREC>
struct Arith;

template <>
struct Arith<0> : ArF64 {
    __device__ static V tab(const double *tb, const float *, const float *, int64_t i) { return tb[i]; }
    __device__ static V nval(const double *n64, const float *, const float *, int64_t i) { return n64[i]; }
};

template <>
struct Arith<1> : ArF32 {
    __device__ static V tab(const double *, const float *t32, const float *, int64_t i) { return t32[i]; }
    __device__ static V nval(const double *, const float *n32, const float *, int64_t i) { return n32[i]; }
};

template <>
struct Arith<2> : ArF2 {
    __device__ static V tab(const double *, const float *t32, const float *tlo, int64_t i) {
        return {t32[i], tlo[i]};
    }
    __device__ static V nval(const double *, const float *n32, const float *nlo, int64_t i) {
        return {n32[i], nlo[i]};
    }
};

// Neighbour ring with the same pixel count (P = Q = 1): with s = p - q the
// levels are |s| and |s + d|, so the row is a correlation of the N^-1 ring
// with K kernel values,  acc[d] += sum_s T[|s|] N[q+s] T[|s+d|],
// |s|, |s+d| <= K-1.  K is a template parameter: every index is static, the
// kernel values and the N^-1 window sit in registers, one FMA per triple.
template <class A, int WMAX, int K>
__device__ __forceinline__ void same_count_entry(typename A::V (&acc)[WMAX + 1], int q, int n, int w,
                                                 const double *__restrict__ n64, const float *__restrict__ n32,
                                                 const float *__restrict__ nlo, int nstride,
                                                 const double *__restrict__ tb, const float *__restrict__ tb32,
                                                 const float *__restrict__ tblo, int64_t tab) {
    typedef typename A::V V;
    V t[K];
#pragma unroll
    for (int k = 0; k < K; ++k) t[k] = A::tab(tb, tb32, tblo, tab + k);
    V wv[2 * K - 1];
    const int p0 = q - (K - 1);
    if (nstride == 1 && p0 >= 0 && p0 + 2 * K - 2 < n) {
        // the window does not wrap: one base pointer, immediate offsets
#pragma unroll
        for (int i = 0; i < 2 * K - 1; ++i) {
            const int s = i - (K - 1);
            wv[i] = A::mul(t[s < 0 ? -s : s], A::nval(n64 + p0, n32 + p0, nlo + p0, i));
        }
    } else {
#pragma unroll
        for (int i = 0; i < 2 * K - 1; ++i) {
            const int s = i - (K - 1);
            int p = q + s;
            p += p < 0 ? n : 0;
            p -= p >= n ? n : 0;
            wv[i] = A::mul(t[s < 0 ? -s : s], A::nval(n64, n32, nlo, (int64_t)p * nstride));
        }
    }
#pragma unroll
    for (int d = 0; d <= 2 * K - 2; ++d) {
        if (d > w) break;  // offsets past the stored band (uniform per block)
#pragma unroll
        for (int i = 0; i < 2 * K - 1; ++i) {
            const int a = i - (K - 1) + d;
            if (a >= -(K - 1) && a <= K - 1) acc[d] = A::fma_(wv[i], t[a < 0 ? -a : a], acc[d]);
        }
    }
}

template <class A, int WMAX, int K>
struct SameCount {
    __device__ static bool run(int Kr, typename A::V (&acc)[WMAX + 1], int q, int n, int w, const double *n64,
                               const float *n32, const float *nlo, int nstride, const double *tb, const float *tb32,
                               const float *tblo, int64_t tab) {
        if (Kr == K) {
            same_count_entry<A, WMAX, K>(acc, q, n, w, n64, n32, nlo, nstride, tb, tb32, tblo, tab);
            return true;
        }
        return SameCount<A, WMAX, K - 1>::run(Kr, acc, q, n, w, n64, n32, nlo, nstride, tb, tb32, tblo, tab);
    }
};
template <class A, int WMAX>
struct SameCount<A, WMAX, 0> {
    __device__ static bool run(int, typename A::V (&)[WMAX + 1], int, int, int, const double *, const float *,
                               const float *, int, const double *, const float *, const float *, int64_t) {
        return false;
    }
};

// Any ring pair: for each stored offset d (static) the pixels coupled to both
// q and q - d form one contiguous run, (2p+1)P in [Z - m, Z - 2dQ + m]: a
// prefix of q's own arc (d = 0).  With a cache (this thread's column of a
// shared array, stride 128) the weights b(q, p) N^-1_p of the arc are formed
// once, in the same rounding, and every d walks its prefix of them; arcs
// longer than the cache take the direct walk.
constexpr int kArcCache = 88;  // cached arc length per thread (w > 16; 44 KB per CTA in FP32, 88 KB else)

template <class A, int WMAX, bool CACHE>
__device__ __forceinline__ void general_entry(typename A::V (&acc)[WMAX + 1], int q, int w, const PairEntry &pe,
                                              const double *__restrict__ n64, const float *__restrict__ n32,
                                              const float *__restrict__ nlo, const double *__restrict__ tb,
                                              const float *__restrict__ tb32, const float *__restrict__ tblo,
                                              int64_t tab, typename A::V *wc) {
    typedef typename A::V V;
    const int P = pe.P, Q = pe.Q, m = pe.mmax, par = pe.par;
    const int Z = (2 * q + 1) * Q;
    const int p_lo = ceil_div(Z - m - P, 2 * P);
    int pm0 = p_lo % pe.nrho;
    if (pm0 < 0) pm0 += pe.nrho;
    if constexpr (CACHE) {
        const int narc = floor_div(Z + m - P, 2 * P) - p_lo + 1;
        if (narc <= kArcCache) {
            int pm = pm0, z = Z - (2 * p_lo + 1) * P;
            for (int j = 0; j < narc; ++j) {
                const int lq = (abs(z) - par) >> 1;
                wc[j * 128] = A::mul(A::tab(tb, tb32, tblo, tab + lq),
                                     A::nval(n64, n32, nlo, pe.noff + (int64_t)pm * pe.nstride));
                z -= 2 * P;
                if (++pm == pe.nrho) pm = 0;
            }
#pragma unroll
            for (int d = 0; d <= WMAX; ++d) {
                if (d > w || 2 * d * Q > 2 * m) break;
                const int cnt = floor_div(Z - 2 * d * Q + m - P, 2 * P) - p_lo + 1;
                int zd = Z - 2 * d * Q - (2 * p_lo + 1) * P;
                V a = A::zero();
#pragma unroll 4
                for (int j = 0; j < cnt; ++j) {
                    const int lr = (abs(zd) - par) >> 1;
                    a = A::fma_(wc[j * 128], A::tab(tb, tb32, tblo, tab + lr), a);
                    zd -= 2 * P;
                }
                acc[d] = A::add(acc[d], a);
            }
            return;
        }
    }
#pragma unroll
    for (int d = 0; d <= WMAX; ++d) {
        if (d > w || 2 * d * Q > 2 * m) break;
        const int p_hi = floor_div(Z - 2 * d * Q + m - P, 2 * P);
        int pm = pm0;
        V a = A::zero();
        for (int p = p_lo; p <= p_hi; ++p) {
            const int z = Z - (2 * p + 1) * P;
            const int lq = (abs(z) - par) >> 1;
            const int lr = (abs(z - 2 * d * Q) - par) >> 1;
            const V bq = A::tab(tb, tb32, tblo, tab + lq);
            const V nv = A::nval(n64, n32, nlo, pe.noff + (int64_t)pm * pe.nstride);
            a = A::fma_(A::mul(bq, nv), A::tab(tb, tb32, tblo, tab + lr), a);
            if (++pm == pe.nrho) pm = 0;
        }
        acc[d] = A::add(acc[d], a);
    }
}

template <int PREC, int WMAX, bool DENSE_OUT>
__global__ void __launch_bounds__(128) k_sample_pband(const SampleItem *__restrict__ items,
                                                      const BlockDesc *__restrict__ blocks,
                                                      const PairEntry *__restrict__ entries, int64_t nslots,
                                                      int64_t npix, const double *__restrict__ tb,
                                                      const float *__restrict__ tb32, const float *__restrict__ tblo,
                                                      const double *__restrict__ td, const float *__restrict__ td32,
                                                      const float *__restrict__ tdlo, const double *__restrict__ ninv,
                                                      const float *__restrict__ ninv32, const float *__restrict__ ninvlo,
                                                      double *__restrict__ out) {
    typedef Arith<PREC> A;
    typedef typename A::V V;
    // same-count fast path up to KTOP levels (FP32 covers wide beams; the
    // wider arithmetics keep register pressure and code size bounded)
    constexpr int KCAP = PREC == 1 ? 17 : 9;
    constexpr int KTOP = (WMAX / 2 + 1) < KCAP ? (WMAX / 2 + 1) : KCAP;
    constexpr bool STAGE = !DENSE_OUT && WMAX <= 16;
    constexpr bool CACHE = WMAX > 16;  // arc weights in dynamic shared memory
    __shared__ double stage[STAGE ? 128 * (WMAX + 1) : 1];
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    V *wc = reinterpret_cast<V *>(dyn_smem) + threadIdx.x;
    const SampleItem it = items[blockIdx.x];
    const BlockDesc bd = blocks[it.block];
    const int q = it.q0 + (int)threadIdx.x;
    const int n = bd.n;
    const int w = bd.w;
    const bool live = q < n;
    V acc[WMAX + 1];
#pragma unroll
    for (int d = 0; d <= WMAX; ++d) acc[d] = A::zero();
    const int64_t tbase = (int64_t)bd.op * nslots;
    const int64_t nbase = (int64_t)bd.op * npix;
    const double *n64 = ninv + nbase;
    const float *n32 = ninv32 + nbase;
    const float *nlo = ninvlo + nbase;
    if (live) {
        for (int e = 0; e < bd.npairs; ++e) {
            const PairEntry pe = entries[bd.pair0 + e];
            const int64_t tab = tbase + pe.tab;
            bool done = false;
            if (pe.P == 1 && pe.Q == 1)
                done = SameCount<A, WMAX, KTOP>::run(pe.mmax / 2 + 1, acc, q, n, w, n64 + pe.noff, n32 + pe.noff,
                                                     nlo + pe.noff, pe.nstride, tb, tb32, tblo, tab);
            if (!done) general_entry<A, WMAX, CACHE>(acc, q, w, pe, n64, n32, nlo, tb, tb32, tblo, tab, wc);
        }
        // D^ on the same ring, in the contraction's arithmetic
#pragma unroll
        for (int d = 0; d <= WMAX; ++d)
            if (d < bd.dK) acc[d] = A::add(acc[d], A::tab(td, td32, tdlo, tbase + bd.dtab + d));
    }
    if (STAGE) {
        // stage the rows and write the tile's contiguous band slice coalesced
#pragma unroll
        for (int d = 0; d <= WMAX; ++d) {
            if (d <= w && live) stage[threadIdx.x * (w + 1) + d] = A::to_double(acc[d]);
        }
        __syncthreads();
        const int nq = min(128, n - it.q0);
        const int tot = nq * (w + 1);
        double *dst = out + bd.off_pband + (int64_t)it.q0 * (w + 1);
        for (int i = threadIdx.x; i < tot; i += 128) dst[i] = stage[i];
        return;
    }
    if (!live) return;
#pragma unroll
    for (int d = 0; d <= WMAX; ++d) {
        if (d <= w) {
            const double v = A::to_double(acc[d]);
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

// -- FP32, two columns per thread on the packed FP32 pipe -------------------
// fma.rn.f32x2 / mul.rn.f32x2 apply the FP32 operation to both halves of a
// register pair with the same rounding as the scalar instruction, so the two
// columns q, q+1 of a thread come out exactly as the one-column kernel's.
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) {
    unsigned long long ua = *reinterpret_cast<unsigned long long *>(&a), ub = *reinterpret_cast<unsigned long long *>(&b),
                       ud;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(ud) : "l"(ua), "l"(ub));
    return *reinterpret_cast<float2 *>(&ud);
}
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) {
    unsigned long long ua = *reinterpret_cast<unsigned long long *>(&a), ub = *reinterpret_cast<unsigned long long *>(&b),
                       uc = *reinterpret_cast<unsigned long long *>(&c), ud;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(ud) : "l"(ua), "l"(ub), "l"(uc));
    return *reinterpret_cast<float2 *>(&ud);
}

// Same-count neighbour ring for columns q and q+1: one window of 2K map
// values serves both (column q+1's window is column q's shifted by one).
template <int WMAX, int K>
__device__ __forceinline__ void same_count2(float2 (&acc)[WMAX + 1], int q, int n, int w,
                                            const float *__restrict__ n32, int nstride, const float *__restrict__ t32) {
    float t[K];
#pragma unroll
    for (int k = 0; k < K; ++k) t[k] = t32[k];
    float v[2 * K];
    const int p0 = q - (K - 1);
    if (nstride == 1 && p0 >= 0 && p0 + 2 * K - 1 < n) {
#pragma unroll
        for (int j = 0; j < 2 * K; ++j) v[j] = n32[p0 + j];
    } else {
#pragma unroll
        for (int j = 0; j < 2 * K; ++j) {
            int p = p0 + j;
            p += p < 0 ? n : 0;
            p -= p >= n ? n : 0;
            v[j] = n32[(int64_t)p * nstride];
        }
    }
    float2 wv[2 * K - 1];
#pragma unroll
    for (int i = 0; i < 2 * K - 1; ++i) {
        const int sv = i - (K - 1);
        const float ts = t[sv < 0 ? -sv : sv];
        wv[i] = f2mul(make_float2(v[i], v[i + 1]), make_float2(ts, ts));
    }
#pragma unroll
    for (int d = 0; d <= 2 * K - 2; ++d) {
        if (d > w) break;  // offsets past the stored band (uniform per block)
#pragma unroll
        for (int i = 0; i < 2 * K - 1; ++i) {
            const int a = i - (K - 1) + d;
            if (a >= -(K - 1) && a <= K - 1) {
                const float ta = t[a < 0 ? -a : a];
                acc[d] = f2fma(wv[i], make_float2(ta, ta), acc[d]);
            }
        }
    }
}

template <int WMAX, int K>
struct SameCount2 {
    __device__ static bool run(int Kr, float2 (&acc)[WMAX + 1], int q, int n, int w, const float *n32, int nstride,
                               const float *t32) {
        if (Kr == K) {
            same_count2<WMAX, K>(acc, q, n, w, n32, nstride, t32);
            return true;
        }
        return SameCount2<WMAX, K - 1>::run(Kr, acc, q, n, w, n32, nstride, t32);
    }
};
template <int WMAX>
struct SameCount2<WMAX, 0> {
    __device__ static bool run(int, float2 (&)[WMAX + 1], int, int, int, const float *, int, const float *) {
        return false;
    }
};

// FP32 periodic-band sampling, 64 threads per 128-column tile, columns
// q0 + 2t and q0 + 2t + 1 in thread t; output staged and written as the
// tile's contiguous band slice.
template <int WMAX>
__global__ void __launch_bounds__(64) k_sample_pband_f32x2(const SampleItem *__restrict__ items,
                                                           const BlockDesc *__restrict__ blocks,
                                                           const PairEntry *__restrict__ entries, int64_t nslots,
                                                           int64_t npix, const float *__restrict__ tb32,
                                                           const float *__restrict__ td32,
                                                           const float *__restrict__ ninv32,
                                                           double *__restrict__ out) {
    constexpr int KTOP = (WMAX / 2 + 1) < 17 ? (WMAX / 2 + 1) : 17;
    __shared__ double stage[128 * (WMAX + 1)];
    const SampleItem it = items[blockIdx.x];
    const BlockDesc bd = blocks[it.block];
    const int n = bd.n, w = bd.w;
    const int q = it.q0 + 2 * (int)threadIdx.x;
    const bool live0 = q < n, live1 = q + 1 < n;
    float2 acc[WMAX + 1];
#pragma unroll
    for (int d = 0; d <= WMAX; ++d) acc[d] = make_float2(0.0f, 0.0f);
    const int64_t tbase = (int64_t)bd.op * nslots;
    const float *n32 = ninv32 + (int64_t)bd.op * npix;
    if (live0) {
        for (int e = 0; e < bd.npairs; ++e) {
            const PairEntry pe = entries[bd.pair0 + e];
            const int64_t tab = tbase + pe.tab;
            bool done = false;
            if (pe.P == 1 && pe.Q == 1)
                done = SameCount2<WMAX, KTOP>::run(pe.mmax / 2 + 1, acc, q, n, w, n32 + pe.noff, pe.nstride, tb32 + tab);
            if (!done) {  // any other ring pair: each column on its own
                float a0[WMAX + 1], a1[WMAX + 1];
#pragma unroll
                for (int d = 0; d <= WMAX; ++d) {
                    a0[d] = acc[d].x;
                    a1[d] = acc[d].y;
                }
                general_entry<Arith<1>, WMAX, false>(a0, q, w, pe, nullptr, n32, nullptr, nullptr, tb32, nullptr, tab,
                                                     nullptr);
                if (live1)
                    general_entry<Arith<1>, WMAX, false>(a1, q + 1, w, pe, nullptr, n32, nullptr, nullptr, tb32, nullptr,
                                                         tab, nullptr);
#pragma unroll
                for (int d = 0; d <= WMAX; ++d) acc[d] = make_float2(a0[d], a1[d]);
            }
        }
#pragma unroll
        for (int d = 0; d <= WMAX; ++d)
            if (d < bd.dK) {
                const float dv = td32[tbase + bd.dtab + d];
                acc[d].x += dv;
                acc[d].y += dv;
            }
    }
    const int t2 = 2 * (int)threadIdx.x;
#pragma unroll
    for (int d = 0; d <= WMAX; ++d) {
        if (d <= w) {
            if (live0) stage[t2 * (w + 1) + d] = f32_to_f64_bits(acc[d].x);
            if (live1) stage[(t2 + 1) * (w + 1) + d] = f32_to_f64_bits(acc[d].y);
        }
    }
    __syncthreads();
    const int nq = min(128, n - it.q0);
    const int tot = nq * (w + 1);
    double *dst = out + bd.off_pband + (int64_t)it.q0 * (w + 1);
    for (int i = threadIdx.x; i < tot; i += 64) dst[i] = stage[i];
}

template <int PREC, bool DENSE_OUT>
void launch_pband(sympix_plan_t pl, const double *ninv, double *blocks, cudaStream_t st) {
    const int64_t npix = pl->grid->npix;
    const int wm[4] = {8, 16, 32, 64};
    for (int b = 0; b < 4; ++b) {
        const size_t ni = pl->items_pband[b].size();
        if (!ni) continue;
#define SPX_ARGS                                                                                            \
    pl->d_items_pband[b].p, pl->d_blocks.p, pl->d_entries.p, pl->nslots, npix, pl->d_tab_b.p, pl->d_tab_b32.p, \
        pl->d_tab_blo.p, pl->d_tab_d.p, pl->d_tab_d32.p, pl->d_tab_dlo.p, ninv, pl->d_ninv32.p, pl->d_ninvlo.p, blocks
        if (PREC == 1 && !DENSE_OUT && wm[b] == 8) {  // two columns per thread, packed FP32 (faster here;
                                                       // the one-column kernel is faster for wider bands)
            k_sample_pband_f32x2<8><<<(unsigned)ni, 64, 0, st>>>(pl->d_items_pband[b].p, pl->d_blocks.p, pl->d_entries.p, pl->nslots, npix,
                                            pl->d_tab_b32.p, pl->d_tab_d32.p, pl->d_ninv32.p, blocks);
            continue;
        }
        // wide bands: the arc-weight cache, kArcCache values per thread
        const size_t wcs = (size_t)128 * kArcCache * sizeof(typename Arith<PREC>::V);
        switch (wm[b]) {
            case 8: k_sample_pband<PREC, 8, DENSE_OUT><<<(unsigned)ni, 128, 0, st>>>(SPX_ARGS); break;
            case 16: k_sample_pband<PREC, 16, DENSE_OUT><<<(unsigned)ni, 128, 0, st>>>(SPX_ARGS); break;
            case 32:
                cudaFuncSetAttribute(k_sample_pband<PREC, 32, DENSE_OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)wcs);
                k_sample_pband<PREC, 32, DENSE_OUT><<<(unsigned)ni, 128, wcs, st>>>(SPX_ARGS);
                break;
            default:
                cudaFuncSetAttribute(k_sample_pband<PREC, 64, DENSE_OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)wcs);
                k_sample_pband<PREC, 64, DENSE_OUT><<<(unsigned)ni, 128, wcs, st>>>(SPX_ARGS);
                break;
        }
#undef SPX_ARGS
    }
}

}  // namespace sympix
