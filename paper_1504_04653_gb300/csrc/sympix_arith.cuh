// Arithmetic policies shared by the contraction and the factorisation.
//
//   ArF64   IEEE FP64.
//   ArF32   IEEE FP32.
//   ArF2    split FP32: a value is the unevaluated sum hi + lo of two floats
//           (|lo| <= ulp(hi)/2).  Products use the exact FMA two-product
//           (Dekker / Ogita-Rump-Oishi "TwoProduct"), sums Knuth's two-sum
//           followed by a fast renormalisation, giving ~44-48 significant
//           bits on the FP32 pipes, which run 61x faster than FP64 on GB300.
#pragma once

#include <cuda_runtime.h>

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

__device__ __forceinline__ F2 f2_neg(F2 a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ F2 f2_from(double x) {
    float h = (float)x;
    return {h, (float)(x - (double)h)};
}

// 1/sqrt(x): FP32 estimate refined by one Newton-Raphson step
// y <- y + y (1 - x y^2) / 2, with the residual formed in split precision.
__device__ __forceinline__ F2 f2_rsqrt(F2 x) {
    float y = rsqrtf(x.hi);
    F2 t = f2_mul(x, F2{y, 0.0f});
    t = f2_mul(t, F2{y, 0.0f});
    F2 r = f2_add(F2{1.0f, 0.0f}, f2_neg(t));  // 1 - x y^2, small
    float corr = 0.5f * y * r.hi;
    return f2_fast_two_sum(y, corr);
}

// A split-FP32 value as an arithmetic type, for the kernels templated on
// their element type (the one-lane band pass and the chunked border rows):
// the operations above behind operators.
struct __align__(8) DF {  // one 8-byte access per value
    float hi, lo;
    DF() = default;
    __host__ __device__ constexpr DF(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr explicit DF(float h) : hi(h), lo(0.0f) {}
};
__device__ __forceinline__ F2 to_f2(DF a) { return {a.hi, a.lo}; }
__device__ __forceinline__ DF to_df(F2 a) { return {a.hi, a.lo}; }
__device__ __forceinline__ DF operator-(DF a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ DF operator+(DF a, DF b) { return to_df(f2_add(to_f2(a), to_f2(b))); }
__device__ __forceinline__ DF operator-(DF a, DF b) { return to_df(f2_add(to_f2(a), f2_neg(to_f2(b)))); }
__device__ __forceinline__ DF operator*(DF a, DF b) { return to_df(f2_mul(to_f2(a), to_f2(b))); }
__device__ __forceinline__ DF &operator+=(DF &a, DF b) { return a = a + b; }
__device__ __forceinline__ bool operator>(DF a, DF b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
// a b + c: the exact product of the high parts (TwoProduct) and the cross
// terms, added to c by a two-sum, then one renormalisation
__device__ __forceinline__ DF df_fma(DF a, DF b, DF c) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float s = p + c.hi, bb = s - p;
    float t = (p - (s - bb)) + (c.hi - bb);
    t += e + c.lo;
    return to_df(f2_fast_two_sum(s, t));
}

// -- FP32 <-> FP64 on the integer ALU --------------------------------------
// Type conversions to and from 64-bit floating point issue on the FP64 pipe,
// which runs at 1/64 of the FP32 rate on GB300.  These helpers move the
// IEEE-754 sign, exponent and significand fields with integer instructions
// instead.  Normal numbers and zeros are handled exactly as the IEEE
// conversions do (round to nearest even for FP64 -> FP32); values in the
// FP32 subnormal range are flushed to signed zero, overflow gives infinity.

__device__ __forceinline__ double f32_to_f64_bits(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xFFu;
    const unsigned sh = u & 0x80000000u;
    const unsigned ee = (e == 0xFFu) ? 0x7FFu : e + 896u;
    unsigned hi = sh | (ee << 20) | ((u & 0x7FFFFFu) >> 3);
    unsigned lo = (u & 0x7u) << 29;
    if (e == 0u) {
        hi = sh;
        lo = 0u;
    }
    return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float f64_to_f32_bits(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned sgn = hi & 0x80000000u;
    const int E = (int)((hi >> 20) & 0x7FFu);
    const int e = E - 896;
    unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1FFFFFFFu;
    m += (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
    unsigned r = ((unsigned)e << 23) + m;  // a carry out of m bumps the exponent
    if (e <= 0) r = 0u;
    if (e >= 255) r = 0x7F800000u;
    if (E == 0x7FF) r = 0x7F800000u | (((hi & 0xFFFFFu) | lo) ? 0x400000u : 0u);
    return __uint_as_float(sgn | r);
}

// x = hi + lo with hi = RN_f32(x) and lo = RN_f32(x - hi), integer ALU only.
// The residual x - hi is the dropped 29-bit tail (minus 2^29 when hi was
// rounded up) in units of x's last bit; lo is flushed to zero when that unit
// lies below the FP32 normal range (|x| < 2^-74).
__device__ __forceinline__ F2 f2_from_bits(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int E = (int)((hi >> 20) & 0x7FFu);
    const float h = f64_to_f32_bits(x);
    const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1FFFFFFFu;
    const bool up = rem > 0x10000000u || (rem == 0x10000000u && (m & 1u));
    int r = up ? (int)rem - 0x20000000 : (int)rem;
    if (hi & 0x80000000u) r = -r;
    const int se = E - 1075 + 127;  // FP32 exponent field of x's last-bit unit
    float l = 0.0f;
    if (se >= 1 && se <= 254 && E != 0x7FF) l = (float)r * __uint_as_float((unsigned)se << 23);
    return {h, l};
}

struct ArF64 {
    typedef double V;
    __device__ static V zero() { return 0.0; }
    __device__ static V from(double x) { return x; }
    __device__ static double to_double(V a) { return a; }
    __device__ static V mul(V a, V b) { return a * b; }
    __device__ static V fma_(V a, V b, V c) { return fma(a, b, c); }
    __device__ static V fnma(V a, V b, V c) { return fma(-a, b, c); }
    __device__ static V sub(V a, V b) { return a - b; }
    __device__ static V rsqrt_(V a) { return rsqrt(a); }
    __device__ static bool positive(V a) { return a > 0.0; }
    __device__ static V shfl(V a, int src, unsigned mask) { return __shfl_sync(mask, a, src); }
    __device__ static V shfl_xor(V a, int m, unsigned mask) { return __shfl_xor_sync(mask, a, m); }
    __device__ static V add(V a, V b) { return a + b; }
};

struct ArF32 {
    typedef float V;
    __device__ static V zero() { return 0.0f; }
    __device__ static V from(double x) { return f64_to_f32_bits(x); }
    __device__ static double to_double(V a) { return f32_to_f64_bits(a); }
    __device__ static V mul(V a, V b) { return a * b; }
    __device__ static V fma_(V a, V b, V c) { return fmaf(a, b, c); }
    __device__ static V fnma(V a, V b, V c) { return fmaf(-a, b, c); }
    __device__ static V sub(V a, V b) { return a - b; }
    __device__ static V rsqrt_(V a) { return rsqrtf(a); }
    __device__ static bool positive(V a) { return a > 0.0f; }
    __device__ static V shfl(V a, int src, unsigned mask) { return __shfl_sync(mask, a, src); }
    __device__ static V shfl_xor(V a, int m, unsigned mask) { return __shfl_xor_sync(mask, a, m); }
    __device__ static V add(V a, V b) { return a + b; }
};

struct ArF2 {
    typedef F2 V;
    __device__ static V zero() { return {0.0f, 0.0f}; }
    __device__ static V from(double x) { return f2_from_bits(x); }
    // one FP64 add per value: both halves convert exactly on the integer ALU
    __device__ static double to_double(V a) { return f32_to_f64_bits(a.hi) + f32_to_f64_bits(a.lo); }
    __device__ static V mul(V a, V b) { return f2_mul(a, b); }
    __device__ static V fma_(V a, V b, V c) { return f2_add(f2_mul(a, b), c); }
    __device__ static V fnma(V a, V b, V c) { return f2_add(c, f2_neg(f2_mul(a, b))); }
    __device__ static V sub(V a, V b) { return f2_add(a, f2_neg(b)); }
    __device__ static V rsqrt_(V a) { return f2_rsqrt(a); }
    __device__ static bool positive(V a) { return a.hi > 0.0f || (a.hi == 0.0f && a.lo > 0.0f); }
    __device__ static V shfl(V a, int src, unsigned mask) {
        return {__shfl_sync(mask, a.hi, src), __shfl_sync(mask, a.lo, src)};
    }
    __device__ static V shfl_xor(V a, int m, unsigned mask) {
        return {__shfl_xor_sync(mask, a.hi, m), __shfl_xor_sync(mask, a.lo, m)};
    }
    __device__ static V add(V a, V b) { return f2_add(a, b); }
};

}  // namespace sympix
