// Shared pieces of the Cholesky factorisation kernels (sympix_factor*.cu):
// block views, staging helpers, and the templated FP32 band / border
// passes that both the separate and the fused FP32 kernels run.
#pragma once

#include <type_traits>
#include <utility>

#include "sympix_arith.cuh"
#include "sympix_internal.cuh"

namespace sympix {

// Element access of one block in its storage.
struct PBandView {
    double *band;  // n x (w+1)
    double *bord;  // w x n
    int n, w, m;
    // original A[i][j], i >= j
    __device__ double a(int i, int j) const {
        const int d = i - j;
        if (d <= w) return band[(int64_t)i * (w + 1) + d];
        const int dw = j - i + n;  // wrapped: A[j][(j - dw) mod n]
        if (dw <= w) return band[(int64_t)j * (w + 1) + dw];
        return 0.0;
    }
    __device__ void put_l(int i, int j, double x) const { band[(int64_t)i * (w + 1) + (i - j)] = x; }
    __device__ double get_l(int i, int j) const { return band[(int64_t)i * (w + 1) + (i - j)]; }
    __device__ void put_b(int b, int j, double x) const { bord[(int64_t)b * n + j] = x; }
    __device__ double get_b(int b, int j) const { return bord[(int64_t)b * n + j]; }
    // A[rr][rr - w + c], c = 0..w (a band row, rr >= w)
    __device__ const double *row_elem(int rr, int c) const { return band + (int64_t)rr * (w + 1) + (w - c); }
};

struct DenseView {
    double *p;
    int n, w, m;
    __device__ double a(int i, int j) const { return p[(int64_t)i * n + j]; }
    __device__ void put_l(int i, int j, double x) const { p[(int64_t)i * n + j] = x; }
    __device__ double get_l(int i, int j) const { return p[(int64_t)i * n + j]; }
    __device__ void put_b(int b, int j, double x) const { p[(int64_t)(m + b) * n + j] = x; }
    __device__ double get_b(int b, int j) const { return p[(int64_t)(m + b) * n + j]; }
    __device__ const double *row_elem(int rr, int c) const { return p + (int64_t)rr * n + (rr - w + c); }
};

template <bool DENSE>
struct ViewOf;
template <>
struct ViewOf<false> {
    typedef PBandView T;
    __device__ static T make(double *out, const BlockDesc &bd) {
        double *base = out + bd.off_pband;
        return PBandView{base, base + (int64_t)bd.n * (bd.w + 1), bd.n, bd.w, bd.n - bd.w};
    }
};
template <>
struct ViewOf<true> {
    typedef DenseView T;
    __device__ static T make(double *out, const BlockDesc &bd) {
        return DenseView{out + bd.off_dense, bd.n, bd.w, bd.n - bd.w};
    }
};

// info value of a block whose FP32 pivots shrank below the floor: it is
// refactored in FP64 from the untouched FP64 input (kRescued marks a
// rescued block between the FP64 band and border passes).
constexpr int32_t kRescue = 0x40000000;
constexpr int32_t kRescued = 0x20000000;

// Asynchronous global -> shared copies (no register round trip), used to
// prefetch band rows several elimination steps ahead.
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int kPrefetch = 6;  // band rows in flight ahead of the elimination
constexpr int kRing = 8;      // ring slots per group (> kPrefetch)

// ---------------------------------------------------------------------------
// Two-pass factorisation of periodic-band blocks.
//
// Pass 1 (band): one lane per block factors the band part A11 = L11 L11^T.
// The lane keeps the active (w+1) x (w+1) triangle W[r][c] (rows k..k+w,
// columns k..k+r) in registers; per column k it forms 1/sqrt(pivot),
// scales column k, applies the rank-1 update and shifts the window, the
// band row entering the window having been loaded two columns ahead.
// Pass 2 (border): one lane per border row, G2 lanes per block, runs the
// forward substitution L21 = A21 L11^-T along the band, the band row of L11
// broadcast by shuffles, and accumulates the corner S = A22 - L21 L21^T on
// the fly; the w x w corner is then factored by one lane.
// ---------------------------------------------------------------------------

constexpr int kChunk = 16;  // band rows per staged chunk

// ---------------------------------------------------------------------------
// FP32 factorisation on a shadow of the band.
//
// Blocks of one exact width W <= 16 are factored in slices of up to 32.  A
// slice's band rows are converted once to an FP32 copy (the shadow) laid out
// lane-interleaved: element e (row e / (W+1), offset e % (W+1)) of the
// slice's block L sits at 32 e + L.  With one lane per block every warp
// access of the band pass then covers 32 consecutive floats, and the
// border pass stages the rows of all 32 blocks with contiguous copies.
//   1. k_f32_shadow_in   FP64 rows -> interleaved FP32 (a shared-memory
//                        transpose, coalesced on both sides);
//   2. k_f32_band_pass   A11 = L11 L11^T, one lane per block;
//   3. k_f32_border_pass L21 = A21 L11^-T into an interleaved FP32 buffer,
//                        S = L21 L21^T and the corner A22 - S = L22 L22^T;
//   4. k_f32_out         L11 and L21 back to the FP64 blocks.
// Kernels are specialised on W (a slice holds one width), so every window
// index is static.
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// f(integral_constant<int, I>) for I = B .. E-1, expanded at compile time.
template <int B, int E>
struct StaticFor {
    template <class F>
    __device__ __forceinline__ static void run(F &&f) {
        f(std::integral_constant<int, B>{});
        StaticFor<B + 1, E>::run(f);
    }
};
template <int E>
struct StaticFor<E, E> {
    template <class F>
    __device__ __forceinline__ static void run(F &&) {}
};

// Band pass of one block in one lane, exact width W.
//
// The active window is the lower triangle of rows k..k+W at columns k..k+r
// (row k+r).  Row i and column j are kept in register slot i mod (W+1) and
// j mod (W+1), and the column loop is unrolled by one period of W+1 steps,
// so every slot index is static and moving the window costs nothing: the
// row retiring at step k frees the slot the row k+1+W enters.  During
// period p (steps k = p(W+1) .. p(W+1)+W) the entering rows are exactly the
// W+1 rows of period p+1, which the warp stages into shared memory one
// period ahead with contiguous 16-byte copies.  Inside a period the code is
// straight-line, so the scheduler overlaps the next pivot's rsqrt with the
// rest of the update.  Pivots are checked against the floor as they come;
// a block that fell below it stops and is recomputed from its FP64 input.
//
// shs: the slice's interleaved shadow; m: this lane's A11 size (0 for an
// idle lane); mmax: the slice's largest m (every lane runs mmax's periods,
// so that all take part in the staging); stage: the CTA's two period
// buffers, laid out like the shadow.
// T = float: FP32, pivots checked against the floor (a block below it
// returns kRescue and is refactored in FP64).  T = double (FP64) or DF
// (split FP32), on a shadow of that element: the return value is LAPACK's
// info (i + 1 for the first row i whose pivot is not positive; the lane
// stops there).
// An element of the FP64 input in a shadow's arithmetic (FP32 on the integer
// ALU, see sympix_arith.cuh), and back to FP64.
template <class V>
__device__ __forceinline__ V elem_from_f64(double x);
template <>
__device__ __forceinline__ float elem_from_f64<float>(double x) { return f64_to_f32_bits(x); }
template <>
__device__ __forceinline__ double elem_from_f64<double>(double x) { return x; }
template <>
__device__ __forceinline__ DF elem_from_f64<DF>(double x) { return to_df(f2_from_bits(x)); }
__device__ __forceinline__ double elem_to_f64(float x) { return f32_to_f64_bits(x); }
__device__ __forceinline__ double elem_to_f64(double x) { return x; }
// split FP32: hi + lo is exact in FP64 (one FP64 add)
__device__ __forceinline__ double elem_to_f64(DF x) { return f32_to_f64_bits(x.hi) + f32_to_f64_bits(x.lo); }
// A 16-byte group of consecutive elements (four floats, two doubles or two
// split-FP32 values).
__device__ __forceinline__ void store16(float *p, const float *v) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store16(double *p, const double *v) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
}
__device__ __forceinline__ void load16(const float *p, float *v) {
    const float4 e = *reinterpret_cast<const float4 *>(p);
    v[0] = e.x;
    v[1] = e.y;
    v[2] = e.z;
    v[3] = e.w;
}
__device__ __forceinline__ void load16(const double *p, double *v) {
    const double2 e = *reinterpret_cast<const double2 *>(p);
    v[0] = e.x;
    v[1] = e.y;
}
__device__ __forceinline__ void store16(DF *p, const DF *v) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo);
}
__device__ __forceinline__ void load16(const DF *p, DF *v) {
    const float4 e = *reinterpret_cast<const float4 *>(p);
    v[0] = DF(e.x, e.y);
    v[1] = DF(e.z, e.w);
}
// a read-only load through the non-coherent cache
__device__ __forceinline__ float ldg_elem(const float *p) { return __ldg(p); }
__device__ __forceinline__ double ldg_elem(const double *p) { return __ldg(p); }
__device__ __forceinline__ DF ldg_elem(const DF *p) {
    const float2 e = __ldg(reinterpret_cast<const float2 *>(p));
    return DF(e.x, e.y);
}

__device__ __forceinline__ float band_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double band_rsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ float band_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double band_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ DF band_rsqrt(DF x) { return to_df(f2_rsqrt(to_f2(x))); }
__device__ __forceinline__ DF band_fma(DF a, DF b, DF c) { return df_fma(a, b, c); }

template <class T, int W>
__device__ __forceinline__ int band_lanes(T *shs, int lane, int m, int mmax, T *stage, float floor,
                                          volatile int *prog) {
    constexpr int RL = W + 1, CH = RL * RL;
    constexpr bool EXACT = !std::is_same<T, float>::value;  // FP64 or split FP32: LAPACK's info
    constexpr int PER16 = 16 / (int)sizeof(T);  // elements per 16-byte copy
    T *band = shs + lane;  // element e at band[32 e]
    auto issue = [&](int per) {
        const int r0 = per * RL;
        if (r0 < mmax) {  // rows r0 .. r0 + W < the slice's rows
            T *dst = stage + (per & 1) * CH * 32;
            const T *src = shs + (int64_t)r0 * RL * 32;
            for (int i = lane; i < CH * 32 / PER16; i += 32) cp_async16(dst + PER16 * i, src + PER16 * i);
        }
        cp_async_commit();
    };
    issue(1);
    T Wn[RL][RL];  // [row slot][column slot]
    T od[RL];      // original diagonal per row slot
#pragma unroll
    for (int r = 0; r <= W; ++r) {
#pragma unroll
        for (int c = 0; c <= r; ++c) Wn[r][c] = r < m ? band[((int64_t)r * RL + (r - c)) * 32] : T(0);
        od[r] = Wn[r][r];
    }
    // One elimination step at phase PH (k = p RL + PH).  lrow = band row
    // p RL; src = this lane's staged rows of period p + 1.  Rows >= m only
    // ever feed rows >= m, which nothing reads, so they need no masking.
    // The pivot d of row k and rs = 1/sqrt(d) arrive from the previous
    // step: each step forms the next pivot first (one product) and starts
    // its rsqrt before the rest of the update.
    // FP32: the floor test; FP64 and split FP32: the first non-positive pivot (row + 1)
    auto fails = [&](T dv, T odv) { return EXACT ? !(dv > T(0)) : !(dv > T(floor) * odv); };
    bool bad = m > 0 && fails(Wn[0][0], od[0]);
    int info = bad ? 1 : 0;
    T d = Wn[0][0], rs = band_rsqrt(Wn[0][0]);
    auto step = [&](auto PHc, T *lrow, const T *src, bool live, int kbase) {
        constexpr int PH = decltype(PHc)::value;
        constexpr int P1 = (PH + 1) % RL;
        if (!live) return;
        lrow[PH * RL * 32] = d * rs;
        T l[RL];
        T dn = T(0), rsn = T(0);
        if constexpr (W >= 1) {
            l[1] = Wn[P1][PH] * rs;
            dn = band_fma(-l[1], l[1], Wn[P1][P1]);
            rsn = band_rsqrt(dn);
        }
#pragma unroll
        for (int r = 2; r <= W; ++r) l[r] = Wn[(PH + r) % RL][PH] * rs;
#pragma unroll
        for (int r = 1; r <= W; ++r) lrow[((PH + r) * RL + r) * 32] = l[r];
#pragma unroll
        for (int r = 1; r <= W; ++r)
#pragma unroll
            for (int c = 1; c <= r; ++c)
                if (r > 1 || c > 1)
                    Wn[(PH + r) % RL][(PH + c) % RL] = band_fma(-l[r], l[c], Wn[(PH + r) % RL][(PH + c) % RL]);
        // row k+1+W enters slot PH at columns k+1 .. k+1+W
#pragma unroll
        for (int c = 0; c <= W; ++c) Wn[PH][(PH + 1 + c) % RL] = src[(PH * RL + (W - c)) * 32];
        od[PH] = Wn[PH][PH];
        if constexpr (W >= 1) {
            d = dn;
            rs = rsn;
        } else {  // a diagonal block: the next pivot is the entering row's
            (void)dn;
            (void)rsn;
            d = Wn[0][0];
            rs = band_rsqrt(d);
        }
        // the next pivot (rows >= m are not A11's); includes d <= 0 and NaN
        const bool f = kbase + PH + 1 < m && fails(d, od[P1]);
        if (f && !bad) info = kbase + PH + 2;
        bad |= f;
    };
    const int PW = mmax / RL;  // the slice's last period
    for (int p = 0; p <= PW; ++p) {
        issue(p + 2);
        cp_async_wait<1>();  // period p + 1 has landed
        __syncwarp();        // ... for every lane's copies
        const T *src = stage + ((p + 1) & 1) * CH * 32 + lane;
        T *lrow = band + (int64_t)p * RL * RL * 32;
        const int left = m - p * RL;  // this lane's steps left
        const int kbase = p * RL;
        if (left >= RL) {
            auto full = [&](auto PHc) { step(PHc, lrow, src, true, kbase); };
            StaticFor<0, RL>::run(full);
        } else if (left > 0) {
            auto part = [&](auto PHc) { step(PHc, lrow, src, decltype(PHc)::value < left, kbase); };
            StaticFor<0, RL>::run(part);
        }
        if (bad) m = 0;  // stop this lane; the warp keeps staging
        // every 8th period: this period's L rows reach L2 (where the border
        // pass stages from) before the flag says rows < (p+1)(W+1) are final
        const bool publish = prog && (p & 7) == 7;
        if (publish) __threadfence();
        __syncwarp();    // every lane is done with the buffer the next copies overwrite
        if (publish && lane == 0) *prog = p + 1;
    }
    cp_async_wait<0>();
    if (prog) {
        __threadfence();
        __syncwarp();
        if (lane == 0) *prog = 0x7fffffff;
    }
    if constexpr (EXACT)
        return info;
    else
        return bad ? kRescue : 0;
}

// The same band pass for FP64 (T = double) and split FP32 (T = DF), whose
// steps are several times longer: a period unrolled as above would not fit
// the instruction cache, so the steps run as a loop over one body, and the
// window moves through the registers instead (Wn[r][c] holds rows k+r,
// columns k+c; after the update every entry shifts up and left by one,
// W (W+1)/2 moves, and row k+1+W enters at the bottom).  Same staging, same
// order of operations per entry, same return value (LAPACK's info).
template <class T, int W>
__device__ __forceinline__ int band_lanes_loop(T *shs, int lane, int m, int mmax, T *stage) {
    constexpr int RL = W + 1, CH = RL * RL;
    constexpr int PER16 = 16 / (int)sizeof(T);
    T *band = shs + lane;
    auto issue = [&](int per) {
        const int r0 = per * RL;
        if (r0 < mmax) {
            T *dst = stage + (per & 1) * CH * 32;
            const T *src = shs + (int64_t)r0 * RL * 32;
            for (int i = lane; i < CH * 32 / PER16; i += 32) cp_async16(dst + PER16 * i, src + PER16 * i);
        }
        cp_async_commit();
    };
    issue(1);
    T Wn[RL][RL];
#pragma unroll
    for (int r = 0; r <= W; ++r)
#pragma unroll
        for (int c = 0; c <= r; ++c) Wn[r][c] = r < m ? band[((int64_t)r * RL + (r - c)) * 32] : T(0);
    bool bad = m > 0 && !(Wn[0][0] > T(0));
    int info = bad ? 1 : 0;
    T d = Wn[0][0], rs = band_rsqrt(Wn[0][0]);
    const int PW = mmax / RL;
    for (int p = 0; p <= PW; ++p) {
        issue(p + 2);
        cp_async_wait<1>();
        __syncwarp();
        const T *src = stage + ((p + 1) & 1) * CH * 32 + lane;
        T *lrow = band + (int64_t)p * RL * RL * 32;
        const int kend = min(RL, m - p * RL);  // this lane's steps in the period
#pragma unroll 1
        for (int ph = 0; ph < kend; ++ph) {
            lrow[ph * RL * 32] = d * rs;
            T l[RL];
            T dn = T(0), rsn = T(0);
            if constexpr (W >= 1) {
                l[1] = Wn[1][0] * rs;
                dn = band_fma(-l[1], l[1], Wn[1][1]);
                rsn = band_rsqrt(dn);
            }
#pragma unroll
            for (int r = 2; r <= W; ++r) l[r] = Wn[r][0] * rs;
#pragma unroll
            for (int r = 1; r <= W; ++r) lrow[((ph + r) * RL + r) * 32] = l[r];
#pragma unroll
            for (int r = 1; r <= W; ++r)
#pragma unroll
                for (int c = 1; c <= r; ++c)
                    if (r > 1 || c > 1) Wn[r][c] = band_fma(-l[r], l[c], Wn[r][c]);
            // shift by one row and column; row k+1+W enters at the bottom
#pragma unroll
            for (int r = 0; r < W; ++r)
#pragma unroll
                for (int c = 0; c <= r; ++c) Wn[r][c] = Wn[r + 1][c + 1];
#pragma unroll
            for (int c = 0; c <= W; ++c) Wn[W][c] = src[(ph * RL + (W - c)) * 32];
            if constexpr (W >= 1) {
                d = dn;
                rs = rsn;
            } else {
                d = Wn[0][0];
                rs = band_rsqrt(d);
            }
            const int k = p * RL + ph;
            const bool f = k + 1 < m && !(d > T(0));
            if (f && !bad) info = k + 2;
            bad |= f;
        }
        if (bad) m = 0;
        __syncwarp();
    }
    cp_async_wait<0>();
    return info;
}

// The band pass of the exact arithmetics over the four schedulers of an SM:
// four warps per slice, each lane still one block.  A warp's FP64 or
// split-FP32 instructions issue on its own scheduler only (a DFMA costs that
// scheduler 64 cycles whatever the other warps do), so one warp per slice
// leaves three quarters of the SM idle and every step's whole chain on one
// pipe.  Here the window's entries are dealt out by diagonal: Wn[r][c] with
// r - c = delta belongs to warp band4_owner(W, delta).  The window's shift
// moves each entry along its own diagonal, so ownership never changes and
// each warp keeps its entries in registers.  Per step:
//   A. the owner of diagonal delta >= 1 forms l[delta] = Wn[delta][0] rs
//      (and stores it as L); warp 0 (the main diagonal) stores L's diagonal;
//   B. every warp reads l from shared memory and updates its entries;
//      warp 0 first forms the next pivot Wn[1][1] - l1^2 and its rsqrt;
//      then the shift, and the entering row's entries of each diagonal.
// Named barrier 1 (all 128 threads) separates A and B and the steps.  Same
// operations per entry, in the same order, as band_lanes_loop.
__host__ __device__ constexpr int band4_owner(int W, int delta) {
    if (delta == 0) return 0;
    int load[4] = {0, 0, 0, 0};
    int own = 1;
    for (int d = 1; d <= W; ++d) {  // most entries first (diagonal d has W - d + 1)
        int best = 1;
        for (int q = 2; q < 4; ++q)
            if (load[q] < load[best]) best = q;
        load[best] += W - d + 1;
        if (d == delta) own = best;
    }
    return own;
}

__device__ __forceinline__ void band4_sync() { asm volatile("bar.sync 1, 128;\n" ::: "memory"); }

// Shared memory of band_lanes4: the staging of band_lanes_loop, then l[W+1][32],
// rs[32] and the lanes' failure flags.
template <class T, int W>
constexpr size_t band4_smem() {
    return (size_t)(2 * (W + 1) * (W + 1) * 32 + (W + 1) * 32 + 32) * sizeof(T) + 32 * sizeof(int);
}

template <class T, int W, int Q>
__device__ __forceinline__ int band_lanes4(T *shs, int lane, int m, int mmax, unsigned char *smem) {
    constexpr int RL = W + 1, CH = RL * RL;
    constexpr int PER16 = 16 / (int)sizeof(T);
    T *stage = reinterpret_cast<T *>(smem);
    T *ls = stage + 2 * CH * 32;  // l[delta][lane]
    T *rss = ls + RL * 32;        // rs[lane]
    int *bads = reinterpret_cast<int *>(rss + 32);
    const int tid = Q * 32 + lane;
    T *band = shs + lane;
    auto issue = [&](int per) {
        const int r0 = per * RL;
        if (r0 < mmax) {
            T *dst = stage + (per & 1) * CH * 32;
            const T *src = shs + (int64_t)r0 * RL * 32;
            for (int i = tid; i < CH * 32 / PER16; i += 128) cp_async16(dst + PER16 * i, src + PER16 * i);
        }
        cp_async_commit();
    };
    issue(1);
    // e[delta][j]: entry (delta + j, j) of the window, for the owned diagonals
    T e[RL][RL];
    StaticFor<0, RL>::run([&](auto Dc) {
        constexpr int D = decltype(Dc)::value;
        if constexpr (band4_owner(W, D) == Q) {
#pragma unroll
            for (int j = 0; j + D <= W; ++j) e[D][j] = D + j < m ? band[((int64_t)(D + j) * RL + D) * 32] : T(0);
        }
    });
    bool bad = false;
    int info = 0;
    T d = T(0);
    if constexpr (Q == 0) {
        d = e[0][0];
        bad = m > 0 && !(d > T(0));
        info = bad ? 1 : 0;
        rss[lane] = band_rsqrt(d);
    }
    band4_sync();
    T rs = rss[lane];
    const int PW = mmax / RL;
    for (int p = 0; p <= PW; ++p) {
        issue(p + 2);
        cp_async_wait<1>();
        band4_sync();  // period p + 1 has landed for every thread's copies
        const T *src = stage + ((p + 1) & 1) * CH * 32 + lane;
        T *lrow = band + (int64_t)p * RL * RL * 32;
        const int left = m - p * RL;
#pragma unroll 1
        for (int ph = 0; ph < RL; ++ph) {
            const bool live = ph < left;
            // A: L's column k
            if (live) {
                if constexpr (Q == 0) lrow[ph * RL * 32] = d * rs;
                StaticFor<1, RL>::run([&](auto Dc) {
                    constexpr int D = decltype(Dc)::value;
                    if constexpr (band4_owner(W, D) == Q) {
                        const T l = e[D][0] * rs;
                        ls[D * 32 + lane] = l;
                        lrow[((ph + D) * RL + D) * 32] = l;
                    }
                });
            }
            band4_sync();
            // B: the updates, the next pivot, the shift
            if (live) {
                T lv[RL];
#pragma unroll
                for (int c = 1; c <= W; ++c) lv[c] = ls[c * 32 + lane];
                if constexpr (Q == 0) {
                    if constexpr (W >= 1) {
                        const T dn = band_fma(-lv[1], lv[1], e[0][1]);
                        rss[lane] = band_rsqrt(dn);
                        e[0][1] = dn;
                    }
                }
                StaticFor<0, RL>::run([&](auto Dc) {
                    constexpr int D = decltype(Dc)::value;
                    if constexpr (band4_owner(W, D) == Q) {
#pragma unroll
                        for (int j = (D == 0 ? 2 : 1); j + D <= W; ++j) e[D][j] = band_fma(-lv[D + j], lv[j], e[D][j]);
#pragma unroll
                        for (int j = 0; j + D < W; ++j) e[D][j] = e[D][j + 1];
                        e[D][W - D] = src[(ph * RL + D) * 32];
                    }
                });
                if constexpr (Q == 0) {
                    d = e[0][0];
                    if constexpr (W == 0) rss[lane] = band_rsqrt(d);
                    const int k = p * RL + ph;
                    const bool f = k + 1 < m && !(d > T(0));
                    if (f && !bad) info = k + 2;
                    bad |= f;
                }
            }
            band4_sync();
            rs = rss[lane];
        }
        // a lane whose pivot failed stops (every warp of it)
        if constexpr (Q == 0) bads[lane] = bad ? 1 : 0;
        band4_sync();
        if (bads[lane]) m = 0;
    }
    cp_async_wait<0>();
    return info;
}

template <class T, int W>
__device__ __forceinline__ int band_lanes4_any(T *shs, int lane, int m, int mmax, unsigned char *smem) {
    switch (threadIdx.x >> 5) {
    case 0: return band_lanes4<T, W, 0>(shs, lane, m, mmax, smem);
    case 1: return band_lanes4<T, W, 1>(shs, lane, m, mmax, smem);
    case 2: return band_lanes4<T, W, 2>(shs, lane, m, mmax, smem);
    default: return band_lanes4<T, W, 3>(shs, lane, m, mmax, smem);
    }
}

template <int W>
__device__ __forceinline__ int f32_band(float *shs, int lane, int m, int mmax, float *stage, float floor,
                                        volatile int *prog) {
    return band_lanes<float, W>(shs, lane, m, mmax, stage, floor, prog);
}

template <int W, class T = float>
struct F32BandDispatch {
    __device__ static int run(int w, T *shs, int lane, int m, int mmax, T *stage, float floor,
                              volatile int *prog = nullptr) {
        if (w == W) return band_lanes<T, W>(shs, lane, m, mmax, stage, floor, prog);
        return F32BandDispatch<W - 1, T>::run(w, shs, lane, m, mmax, stage, floor, prog);
    }
};
template <class T>
struct F32BandDispatch<0, T> {
    __device__ static int run(int w, T *shs, int lane, int m, int mmax, T *stage, float floor,
                              volatile int *prog = nullptr) {
        return w == 0 ? band_lanes<T, 0>(shs, lane, m, mmax, stage, floor, prog) : -1;
    }
};

constexpr int kF32BandStage = 2 * 17 * 17 * 32;  // floats: two periods of W = 16, 32 lanes

// Border pass of one slice, exact width W: the forward substitution
// L21 = A21 L11^-T,
//   L21[b][k] = (A21[b][k] - sum_c L21[b][k-W+c] L11[k][k-W+c]) / L11[k][k],
// with A21 zero except in its first W columns (the wrap) and its last W.
// One CTA per slice; lane = block, warp q owns border rows R q .. R q + R-1
// of all 32 blocks (R = 1 for W <= 8, 2 above).  Like the band pass it
// walks the columns by periods of W+1 with the L11 rows staged one period
// ahead, and keeps each row's last W values in register slot
// (column mod W+1), so every index is static.  L21 goes to the
// lane-interleaved FP32 border buffer (element (b, k) of block L at
// 32 (b kc + k) + L, kc = the slice's largest m) and, a period at a time,
// through shared memory to the corner sums S = L21 L21^T, which the 8 warps
// share pair by pair.  At the end one thread per block factors its corner
// A22 - S = L22 L22^T in FP64.
// FUSED: the CTA's warp 0 runs the band pass of the same slice at the same
// time; this function's NT threads are threads 32 .. 32+NT-1, synchronise
// among themselves on named barrier 1, stage only rows the band warp has
// published as final (*prog = periods done), meet the band warp on named
// barrier 2 (all 32+NT threads) at the end, and take the blocks' band-pass
// results from bandres there.  Each wait for a published period polls at
// most `limit` times; a wait that runs out sets the CTA's abort flag and
// the device status bit kStatusTimeout, the sweep stops at the next
// barrier (every thread reads the flag after the same barrier), waits for
// its copies in flight, and reports kInfoTimeout for the slice's blocks.
// SPLIT: the band pass runs in another CTA of the same (cooperative)
// launch; the progress and a done flag are global words of the slice, the
// function's NT threads are the whole CTA, and the band-pass results are read
// from global memory once the done flag is seen (that wait is bounded too).
constexpr int32_t kStatusTimeout = 1;  // bit of the plan's device status word
constexpr int32_t kInfoTimeout = -1;   // info of a block whose factor a timed-out wait left incomplete
struct FusedWait {
    volatile int *prog;    // periods of L11 rows the band warp has published
    const int *bandres;    // band-pass result per block
    volatile int *abort;   // set when a wait ran out (shared, starts 0)
    int32_t *status;       // device status word of the plan
    int limit;             // polls per wait
    volatile int *done;    // split mode: set once bandres is final
};

// How the border role meets its band pass: after it (a separate kernel),
// beside it in the same CTA (warp 0, shared-memory progress and a named
// barrier at the end), or beside it in another CTA of the same launch
// (global progress and done flags, each poll bounded).
constexpr int kBorderAfter = 0, kBorderFused = 1, kBorderSplit = 2;

// Barrier of all 32 + NT threads of the fused kernel (the band warp and the
// border threads arrive from different code paths, which the non-aligned
// form allows; every warp arrives as a whole).
template <int NT>
__device__ __forceinline__ void fused_barrier_all() {
    asm volatile("barrier.sync 2, %0;\n" ::"n"(32 + NT) : "memory");
}

template <int W, int NT, int MODE>
__device__ __forceinline__ void f32_border(const F32Slice &sl, const float *__restrict__ shs, float *__restrict__ l21,
                                           const double *__restrict__ out, const int64_t *s_off, const int *s_n,
                                           const int *s_live, float *stage, int *binfo, const FusedWait *fw) {
    constexpr int RL = W + 1, CH = RL * RL;
    constexpr int NWARP = NT / 32;
    constexpr int R = (W + NWARP - 1) / NWARP;  // border rows per lane
    constexpr bool FUSED = MODE == kBorderFused, WAITS = MODE != kBorderAfter;
    const int tb = (int)threadIdx.x - (FUSED ? 32 : 0);
    auto bsync = [] {
        if (FUSED)
            asm volatile("bar.sync 1, %0;\n" ::"n"(NT) : "memory");
        else
            __syncthreads();
    };
    const int lane = tb & 31, b0 = (tb >> 5) * R;
    const bool rows = b0 < W;       // warp-uniform: this warp owns border rows
    const int n = s_n[lane], m = n - W;
    const bool live = s_live[lane];
    const PBandView view{const_cast<double *>(out) + s_off[lane],
                         const_cast<double *>(out) + s_off[lane] + (int64_t)n * RL, n, W, m};
    const int kc = sl.rows - W;
    int seen = 0;  // the largest progress value this thread has read
    auto issue = [&](int per) {
        const int r0 = per * RL;
        if (r0 < kc) {  // rows r0 .. r0 + W < the slice's rows
            bool ready = true;
            if (WAITS && seen < per + 1) {  // wait until the band warp has finished these rows
                int spins = 0, v = *fw->prog;
                while (v < per + 1 && ++spins < fw->limit) {
                    __nanosleep(64);
                    v = *fw->prog;
                }
                if (v < per + 1) {  // ran out: stop the sweep at the next barrier
                    ready = false;
                    *fw->abort = 1;
                    atomicOr(fw->status, kStatusTimeout);
                } else {  // a newly published value: order the row reads after it (once per value)
                    seen = v;
                    if (FUSED)
                        __threadfence_block();
                    else
                        __threadfence();  // the rows come from another SM's writes
                }
            }
            if (ready) {
                float *dst = stage + (per % 3) * CH * 32;
                const float *src = shs + (int64_t)r0 * RL * 32;
                for (int i = tb; i < CH * 8; i += NT) cp_async16(dst + 4 * i, src + 4 * i);
            }
        }
        cp_async_commit();
    };
    float *vbuf = stage + 3 * CH * 32;  // two periods of L21 values, [b][column][lane]
    float *vb = vbuf;                   // the current period's
    float *abuf = vbuf + 2 * W * RL * 32;  // A21 at the last W columns, [b][c][lane]: A[m+b][m-W+c]
    for (int i = tb; i < W * W * 32; i += NT) {
        const int L = i & 31, bc = i >> 5, bb = bc / (W > 0 ? W : 1), c = bc - bb * W;
        float v = 0.0f;
        if (s_live[L]) {
            const int nL = s_n[L], mL = nL - W;
            double *o = const_cast<double *>(out) + s_off[L];
            const PBandView vL{o, o + (int64_t)nL * RL, nL, W, mL};
            v = f64_to_f32_bits(vL.a(mL + bb, mL - W + c));
        }
        abuf[i] = v;
    }
    float aw[R][W];  // A21 of my rows at columns < W (the wrap part)
    float y[R][RL];  // L21 of my rows at the last W columns, slot = column mod RL
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
        for (int c = 0; c < W; ++c)
            aw[r][c] = (rows && live && b0 + r < W) ? f64_to_f32_bits(view.a(m + b0 + r, c)) : 0.0f;
#pragma unroll
        for (int c = 0; c < RL; ++c) y[r][c] = 0.0f;
    }
    // corner sums S[b][b2] = sum_k L21[b][k] L21[b2][k], b2 <= b, lane =
    // block; each period's L21 values pass through vbuf.  With one border
    // row per warp (R = 1) a pair goes to the warp owning one of its rows
    // (b when b + b2 is odd or b = b2, else b2), which takes that operand
    // from its own registers: one shared load per FMA, about (W+1)/2 + 1
    // pairs per warp.  Otherwise the pairs are dealt round-robin.
    // With a single border warp (R = W) every pair's operands are the lane's
    // own registers: the sums are formed per column, no shared memory.
    constexpr int NPAIR = W * (W + 1) / 2, NP = (NPAIR + NWARP - 1) / NWARP;
    constexpr bool REG = NWARP == 1;
    constexpr bool OWN = R == 1 && !REG;
    constexpr int NPC = REG ? (NPAIR > 0 ? NPAIR : 1) : OWN ? (W + 1) / 2 + 1 : (NP > 0 ? NP : 1);
    const int wq = tb >> 5;
    int pb[NPC], pb2[NPC], po[NPC];
    float sacc[NPC];
    int npw = 0;  // pairs of this warp
    if constexpr (REG) {
#pragma unroll
        for (int i = 0; i < NPC; ++i) {
            pb[i] = pb2[i] = po[i] = 0;
            sacc[i] = 0.0f;
        }
        npw = NPAIR;
    } else if constexpr (OWN) {
#pragma unroll
        for (int i = 0; i < NPC; ++i) {
            pb[i] = pb2[i] = po[i] = 0;
            sacc[i] = 0.0f;
        }
        for (int bb = 0; bb < W; ++bb)
            for (int b2 = 0; b2 <= bb; ++b2) {
                const int owner = (bb == b2 || ((bb + b2) & 1)) ? bb : b2;
                if (owner != wq) continue;
#pragma unroll
                for (int i = 0; i < NPC; ++i)
                    if (i == npw) {
                        pb[i] = bb;
                        pb2[i] = b2;
                        po[i] = bb == wq ? b2 : bb;
                    }
                ++npw;
            }
    } else {
#pragma unroll
        for (int i = 0; i < NPC; ++i) {
            int j = wq + NWARP * i, bb = 0;
            while (j > bb) {  // pair j = bb (bb+1)/2 + b2
                j -= bb + 1;
                ++bb;
            }
            pb[i] = bb < W ? bb : 0;
            pb2[i] = bb < W ? j : 0;
            po[i] = 0;
            sacc[i] = 0.0f;
            if (wq + NWARP * i < NPAIR) npw = i + 1;
        }
    }
    // column k = p RL + PH; src = this lane's staged rows of period p
    // TAIL: some block of the warp reaches its last W columns (A21's band
    // part) or its end in this period; otherwise no select is needed
    auto column = [&](auto PHc, auto FIRSTc, auto TAILc, const float *src, int kbase) {
        constexpr int PH = decltype(PHc)::value;
        constexpr bool FIRST = decltype(FIRSTc)::value;  // p == 0: mask the columns left of 0
        constexpr bool TAIL = decltype(TAILc)::value;
        const int k = kbase + PH;
        const float *row = src + PH * RL * 32;  // L11 row k: offset d at row[32 d]
        float lr[RL];
#pragma unroll
        for (int d = 0; d < RL; ++d) lr[d] = row[d * 32];
        const float rd = rsqrtf(lr[0]);
        const float rcp = rd * rd;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int b = b0 + r;
            float acc = 0.0f;
            if constexpr (FIRST && PH < W) acc = aw[r][PH < W ? PH : 0];
            if constexpr (TAIL) {  // the last W columns, without a branch
                const int c = k - (m - W);
                const float a = abuf[((b < W ? b : W - 1) * W + min(max(c, 0), W - 1)) * 32 + lane];
                acc = (c >= 0 && c < W) ? a : acc;
            }
#pragma unroll
            for (int cc = 0; cc < W; ++cc) {
                if (FIRST && PH - W + cc < 0) continue;  // left of column 0
                acc = fmaf(-y[r][(PH - W + cc + RL) % RL], lr[W - cc], acc);
            }
            const float val = (!TAIL || (live && b < W && k < m)) ? acc * rcp : 0.0f;
            y[r][PH] = val;
            if (b < W) {
                if constexpr (!REG) vb[(b * RL + PH) * 32 + lane] = val;
                if (!TAIL || k < kc) l21[((int64_t)b * kc + k) * 32 + lane] = val;
            }
        }
        if constexpr (REG) {  // S[b][b2] += L21[b][k] L21[b2][k], pair index b (b+1)/2 + b2
#pragma unroll
            for (int b = 0; b < W; ++b)
#pragma unroll
                for (int b2 = 0; b2 <= b; ++b2)
                    sacc[b * (b + 1) / 2 + b2] = fmaf(y[b][PH], y[b2][PH], sacc[b * (b + 1) / 2 + b2]);
        }
    };
    auto accumulate = [&](const float *v) {
        if constexpr (!REG) {
#pragma unroll
            for (int i = 0; i < NPC; ++i) {
                if (i >= npw) break;
                if constexpr (OWN) {
                    const float *z = v + po[i] * RL * 32 + lane;
#pragma unroll
                    for (int c = 0; c < RL; ++c) sacc[i] = fmaf(y[0][c], z[c * 32], sacc[i]);
                } else {
                    const float *x = v + pb[i] * RL * 32 + lane, *z = v + pb2[i] * RL * 32 + lane;
#pragma unroll
                    for (int c = 0; c < RL; ++c) sacc[i] = fmaf(x[c * 32], z[c * 32], sacc[i]);
                }
            }
        } else {
            (void)v;
        }
    };
    issue(0);
    issue(1);
    const int PW = (kc - 1) / RL;  // the last period
    bool aborted = false;
    for (int p = 0; p <= PW; ++p) {
        cp_async_wait<1>();  // period p has landed
        bsync();             // ... for every thread's copies; period p-1's buffer is free
        if (WAITS && *fw->abort) {  // read by every thread after the same barrier
            aborted = true;
            break;
        }
        issue(p + 2);
        if (p > 0) accumulate(vbuf + ((p - 1) & 1) * W * RL * 32);
        vb = vbuf + (p & 1) * W * RL * 32;
        if (rows) {
            const float *src = stage + (p % 3) * CH * 32 + lane;
            const int kbase = p * RL;
            // warp-uniform: does any block of the warp need the tail handling?
            const bool tail = kbase + RL > kc - W || __any_sync(0xffffffffu, live && kbase + RL > m - W);
            if (p == 0) {
                auto f = [&](auto PHc) { column(PHc, std::true_type{}, std::true_type{}, src, kbase); };
                StaticFor<0, RL>::run(f);
            } else if (tail) {
                auto f = [&](auto PHc) { column(PHc, std::false_type{}, std::true_type{}, src, kbase); };
                StaticFor<0, RL>::run(f);
            } else {
                auto f = [&](auto PHc) { column(PHc, std::false_type{}, std::false_type{}, src, kbase); };
                StaticFor<0, RL>::run(f);
            }
        }
    }
    cp_async_wait<0>();
    if (FUSED) {
        fused_barrier_all<NT>();  // the band warp is done too, bandres is final
    } else if (WAITS) {           // the band CTA's results: wait for its done flag
        if (threadIdx.x == 0) {
            int spins = 0;
            while (*fw->done == 0 && ++spins < fw->limit) __nanosleep(64);
            if (*fw->done == 0) {
                *fw->abort = 1;
                atomicOr(fw->status, kStatusTimeout);
            }
            __threadfence();
        }
        __syncthreads();
        aborted = aborted || *fw->abort;
    } else {
        __syncthreads();
    }
    if (aborted) {
        if (tb < 32) binfo[lane] = kInfoTimeout;
        return;
    }
    accumulate(vbuf + (PW & 1) * W * RL * 32);
    // the corner: sums to shared memory [block][b][b2], then one thread per
    // block factors C = A22 - S = L22 L22^T in FP64
    float *sS = stage;  // the staging is free now
    bsync();
    if constexpr (REG) {
#pragma unroll
        for (int b = 0; b < W; ++b)
#pragma unroll
            for (int b2 = 0; b2 <= b; ++b2) sS[(lane * W + b) * W + b2] = sacc[b * (b + 1) / 2 + b2];
    } else {
#pragma unroll
        for (int i = 0; i < NPC; ++i)
            if (i < npw) sS[(lane * W + pb[i]) * W + pb2[i]] = sacc[i];
    }
    bsync();
    const bool live_end = WAITS ? (live && ((volatile const int *)fw->bandres)[lane] == 0) : live;
    if (tb < 32 && live_end) {
        double *C = reinterpret_cast<double *>(stage + 32 * 16 * 16) + lane * (W * W + 1);  // odd stride
        double *outp = const_cast<double *>(out);
        const PBandView v{outp + s_off[lane], outp + s_off[lane] + (int64_t)n * RL, n, W, m};
        for (int i = 0; i < W; ++i)
            for (int j = 0; j <= i; ++j) C[i * W + j] = v.a(m + i, m + j) - f32_to_f64_bits(sS[(lane * W + i) * W + j]);
        int inf = 0;
        for (int i = 0; i < W && inf == 0; ++i) {
            for (int j = 0; j <= i; ++j) {
                double sv = C[i * W + j];
                for (int k = 0; k < j; ++k) sv -= C[i * W + k] * C[j * W + k];
                if (j < i) {
                    C[i * W + j] = sv / C[j * W + j];
                } else {
                    if (!(sv > 0.0)) {
                        inf = m + i + 1;
                        break;
                    }
                    C[i * W + i] = sqrt(sv);
                }
            }
        }
        for (int i = 0; i < W; ++i)
            for (int j = 0; j <= i; ++j) v.put_b(i, m + j, C[i * W + j]);
        binfo[lane] = inf;
    }
}

template <int W, int WMIN, int NT, int FUSED = kBorderAfter>
struct F32BorderDispatch {
    __device__ static void run(int w, const F32Slice &sl, const float *shs, float *l21, const double *out,
                               const int64_t *s_off, const int *s_n, const int *s_live, float *stage, int *binfo,
                               const FusedWait *fw = nullptr) {
        if (w == W) {
            f32_border<W, NT, FUSED>(sl, shs, l21, out, s_off, s_n, s_live, stage, binfo, fw);
            return;
        }
        F32BorderDispatch<W - 1, WMIN, NT, FUSED>::run(w, sl, shs, l21, out, s_off, s_n, s_live, stage, binfo, fw);
    }
};
template <int WMIN, int NT, int FUSED>
struct F32BorderDispatch<WMIN - 1, WMIN, NT, FUSED> {
    __device__ static void run(int, const F32Slice &, const float *, float *, const double *, const int64_t *,
                               const int *, const int *, float *, int *, const FusedWait * = nullptr) {}
};

// floats: three staged periods, two periods of L21 values and the last W
// columns of A21, W = 16
constexpr int kF32BorderStage = 3 * 17 * 17 * 32 + 2 * 16 * 17 * 32 + 16 * 16 * 32;

// Per-slice block table in shared memory: offsets, sizes, and whether the
// block is still factored in FP32 (its band pass passed the pivot floor).
struct SliceBlocks {
    int64_t off[32];
    int n[32], live[32], bi[32];
};

__device__ __forceinline__ void load_slice_blocks(SliceBlocks &t, const F32Slice &sl, const int32_t *items,
                                                  const BlockDesc *blocks, const int32_t *info) {
    // info == nullptr: every block of the slice counts as live
    if (threadIdx.x < 32) {
        const int L = threadIdx.x;
        int64_t off = 0;
        int n = 2 * sl.w + 2, live = 0, bi = 0;
        if (L < sl.count) {
            bi = items[sl.first + L];
            const BlockDesc bd = blocks[bi];
            off = bd.off_pband;
            n = bd.n;
            live = info ? info[bi] == 0 : 1;
        }
        t.off[L] = off;
        t.n[L] = n;
        t.live[L] = live;
        t.bi[L] = bi;
    }
    __syncthreads();
}


// One CTA of NT threads per slice (256 or 512, the plan's border_threads):
// warp q owns border rows R q .. R q + R-1, R = ceil(w / (NT / 32)).
template <int NT>
__global__ void __launch_bounds__(NT) k_f32_border_pass(const F32Slice *__restrict__ slices,
                                                        const int32_t *__restrict__ items,
                                                        const BlockDesc *__restrict__ blocks,
                                                        const float *__restrict__ sh, float *__restrict__ l21,
                                                        const double *__restrict__ out, int32_t *__restrict__ info) {
    extern __shared__ __align__(16) float bsm[];
    __shared__ SliceBlocks t;
    __shared__ int binfo[32];
    const F32Slice sl = slices[blockIdx.x];
    load_slice_blocks(t, sl, items, blocks, info);
    F32BorderDispatch<16, 1, NT>::run(sl.w, sl, sh + sl.sh, l21 + sl.l21, out, t.off, t.n, t.live, bsm, binfo);
    if (threadIdx.x < 32 && t.live[threadIdx.x] && sl.w > 0) info[t.bi[threadIdx.x]] = binfo[threadIdx.x];
}

// -- launch helpers (one translation unit each) ---------------------------------
// the separate border pass of slices [first, first+count), NT threads per CTA
template <int NT>
void launch_f32_border(sympix_plan_t pl, int first, int count, double *blocks, int32_t *info, cudaStream_t st);
// skip_narrow: lists 0 and 1 (w <= 12) are factored by the narrow-band kernel
template <class A>
void launch_band(sympix_plan_t pl, bool dense, double *blocks, int32_t *info, cudaStream_t st, int rescue = 0,
                 bool skip_narrow = false);
// the 32-lane group kernel on lists 1 and 2 (8 < w <= 16, periodic band) on `st`
template <class A>
void launch_band_groups(sympix_plan_t pl, double *blocks, int32_t *info, cudaStream_t st);
// hi_only: only the slices with w > 12 (the narrow-band kernel has the rest)
void launch_f32_slices(sympix_plan_t pl, double *blocks, int32_t *info, cudaStream_t st, bool hi_only);
void launch_f32_fused(sympix_plan_t pl, int nf, double *blocks, int32_t *info, cudaStream_t st);
// band and border passes of the w <= 8 slices in two CTAs of one
// cooperative launch per slice (sympix_factor_split.cu), and whether that
// launch's CTAs can all be resident at once
bool f32_split_fits(sympix_plan_t pl);
void launch_f32_split_w8(sympix_plan_t pl, double *blocks, int32_t *info, cudaStream_t st);

// the border rows and corners of the fused-range slices by column chunks,
// after their band pass (sympix_l21.cu); hi_only: only the slices with
// 9 <= w <= 12, everything on `st`, no trace marks
void launch_f32_l21(sympix_plan_t pl, double *blocks, int32_t *info, cudaStream_t st, bool hi_only = false);
// the same in FP64 on the FP64 band shadow (every fused-range slice)
void launch_f64_l21(sympix_plan_t pl, double *blocks, int32_t *info, cudaStream_t st);
void launch_df_l21(sympix_plan_t pl, double *blocks, int32_t *info, cudaStream_t st);
// the FP64 / split-FP32 factor of the periodic bands up to w = 16 on a
// shadow of that arithmetic (sympix_factor_f32.cu)
void launch_f64_slices(sympix_plan_t pl, double *blocks, int32_t *info, cudaStream_t st);
void launch_df_slices(sympix_plan_t pl, double *blocks, int32_t *info, cudaStream_t st);
constexpr int kDefaultWaitLimit = 1 << 22;  // polls of a bounded device wait (about 0.3 s)
void launch_factor_wide_dense(sympix_plan_t pl, int precision, bool dense, double *blocks, int32_t *info,
                              cudaStream_t st);

}  // namespace sympix
