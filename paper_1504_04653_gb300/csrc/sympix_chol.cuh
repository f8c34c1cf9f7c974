// Periodic-band Cholesky of narrow bands (w <= 12) with G lanes per block.
//
// A periodic-band block (n rows, half-width w, m = n - w) is factored as
//   A11 = L11 L11^T (band),  L21 = A21 L11^-T (the w border rows),
//   A22 - L21 L21^T = L22 L22^T (the w x w corner, FP64).
// One warp factors a slice of up to 32 / G blocks of one width W; the G
// lanes of a block all run the band elimination (the (W+1) x (W+1) active
// triangle in registers, the column loop unrolled by one period of W+1
// steps so that every register slot index is static), so the pivot chain
// needs no shuffle, and split the border: lane g owns border rows
// b = g, g + G, ... and their share of the corner sums S = L21 L21^T.
// Column k of L, finished at step k, is written into a per-block ring of
// L rows in shared memory (three periods deep); the border sweep runs one
// period behind the band, on rows the previous period completed, so the
// warp synchronises once per period, and the same ring gives each row of
// L11 to write out.
// The band rows that enter the window during period p are staged one period
// ahead with cp.async from the FP64 blocks and converted once, cooperatively.
//
// Compared with one lane per block (32 blocks per warp) this puts 4-8x more
// warps on the machine, each with a short instruction stream per step and
// no waits on other warps; compared with splitting the window over lanes it
// keeps shuffles off the pivot chain.
//
// Output: FP64 and split FP32 write L in place (L11 into the band rows,
// L21 and L22 into the border rows).  FP32 writes L11 as floats into the
// plan's float scratch (same offsets as the blocks) and L21 / L22 into the
// border rows, so the band rows keep the FP64 input until the commit pass:
// a block whose FP32 pivot fell below the floor is then refactored in FP64
// from its untouched input (rescue mode: only blocks marked kRescue).
#pragma once

#include <algorithm>

#include "sympix_factor_kernels.cuh"

namespace sympix {

constexpr int kCholWMax = kNarrowWMax;

// Lanes per block for an arithmetic and width: FP32 8; FP64 and split FP32
// (twice the registers, and FP64 replicated across the lanes costs FP64
// issue) 4 up to w = 8, else 16 (one border row per lane).  The FP64 rescue of the FP32 pass runs on the
// FP64 slices.
template <class A>
__host__ __device__ constexpr int chol_lanes(int w) {
    return std::is_same<A, ArF32>::value ? 8 : (w <= 8 ? 4 : 16);
}

template <class A, int W, int G>
__host__ __device__ constexpr size_t chol_smem_bytes() {
    constexpr int RL = W + 1, CH = RL * RL, B = 32 / G;
    // raw FP64 staging of two periods, the converted period, the L row ring
    // (3 (W+1) rows of W+2: the row of L and 1 / L[k][k]); the corner sums
    // reuse the raw staging
    return (size_t)2 * B * CH * sizeof(double) + (size_t)B * CH * sizeof(typename A::V) +
           (size_t)B * 3 * RL * (RL + 1) * sizeof(typename A::V);
}

// One slice of width W with G lanes per block (one warp).
template <class A, int W, int G>
__device__ __forceinline__ void chol_slice(const CholSlice &sl, const int32_t *__restrict__ items,
                                           const BlockDesc *__restrict__ blocks, double *__restrict__ out,
                                           float *__restrict__ l11f, int32_t *__restrict__ info, float floor,
                                           int rescue, unsigned char *smem) {
    typedef typename A::V V;
    constexpr bool F32 = std::is_same<A, ArF32>::value;
    constexpr int RL = W + 1, CH = RL * RL, B = 32 / G, NR = (W + G - 1) / G;
    constexpr unsigned FULL = 0xffffffffu;
    double *s64 = reinterpret_cast<double *>(smem);
    V *sv = reinterpret_cast<V *>(s64 + 2 * B * CH);
    V *ring_all = sv + B * CH;
    __shared__ int64_t s_off[32];
    __shared__ int s_n[32];

    const int lane = threadIdx.x & 31, grp = lane / G, g = lane % G, gbase = grp * G;
    int bi = -1, n = 0;
    int64_t off = 0;
    if (grp < sl.count) {
        bi = items[sl.first + grp];
        const BlockDesc bd = blocks[bi];
        n = bd.n;
        off = bd.off_pband;
    }
    bool live = bi >= 0;
    if (rescue && live) live = info[bi] == kRescue;
    if (g == 0 && grp < B) {
        s_off[grp] = live ? off : 0;
        s_n[grp] = live ? n : 0;
    }
    const int m = n - W;
    const int mmax = (int)__reduce_max_sync(FULL, (unsigned)(live ? m : 0));
    __syncwarp();
    if (mmax == 0) return;  // nothing to factor in this warp
    double *band = out + off;
    double *bord = band + (int64_t)n * RL;
    constexpr int RS = RL + 1;  // ring row: L[k][k-e], e = 0..W, then 1 / L[k][k]
    V *ring = ring_all + grp * 3 * RL * RS;
    for (int i = lane; i < B * 3 * RL * RS; i += 32) ring_all[i] = A::zero();

    // stage band rows [per (W+1), per (W+1) + W] of every block (raw FP64)
    auto issue = [&](int per) {
        const int r0 = per * RL;
        if (r0 < mmax) {
            double *dst = s64 + (per & 1) * B * CH;
            for (int i = lane; i < B * CH; i += 32) {
                const int bl = i / CH, e = i - bl * CH;
                if (r0 + e / RL < s_n[bl]) cp_async8(dst + i, out + s_off[bl] + (int64_t)r0 * RL + e);
            }
        }
        cp_async_commit();
    };
    issue(1);

    // the window: rows 0..W at columns 0..r (row i, column j in slot i, j mod RL)
    V Wn[RL][RL];
    V od[RL];
#pragma unroll
    for (int r = 0; r <= W; ++r) {
#pragma unroll
        for (int c = 0; c <= r; ++c) Wn[r][c] = live ? A::from(band[(int64_t)r * RL + (r - c)]) : A::zero();
        od[r] = Wn[r][r];
    }
    // border rows b = g + G t
    V y[NR > 0 ? NR : 1][RL];                // the last W+1 values of L21 row b, slot = column mod RL
    V sacc[NR > 0 ? NR : 1][W > 0 ? W : 1];  // corner sums S[b][b2], b2 <= b
#pragma unroll
    for (int t = 0; t < NR; ++t) {
#pragma unroll
        for (int c = 0; c < W; ++c) sacc[t][c] = A::zero();
#pragma unroll
        for (int c = 0; c < RL; ++c) y[t][c] = A::zero();
    }
    V d = Wn[0][0], rs = A::rsqrt_(Wn[0][0]);
    bool bad = false;  // FP32: a pivot fell below floor x its original diagonal
    int inf = 0;       // FP64 / split FP32: first non-positive pivot, row + 1
    if constexpr (F32) {
        bad = !(d > floor * od[0]);
    } else {
        if (!A::positive(d)) inf = 1;
    }

    // Band step k = p (W+1) + PH writes column k of L into the ring (row k+r,
    // offset r, row slot (k+r) mod 3(W+1)); the border sweep runs one period
    // behind, on rows that the previous period completed, so the two never
    // touch the same ring rows within a period and the warp synchronises once
    // per period.
    auto band_step = [&](auto PHc, int kbase, int sb0, int sb1) {
        constexpr int PH = decltype(PHc)::value;
        constexpr int P1 = (PH + 1) % RL;
        const int k = kbase + PH;
        V l[RL];
        l[0] = A::mul(d, rs);
        V dn = A::zero(), rsn = A::zero();
        if constexpr (W >= 1) {
            l[1] = A::mul(Wn[P1][PH], rs);
            dn = A::fnma(l[1], l[1], Wn[P1][P1]);
            rsn = A::rsqrt_(dn);
        }
#pragma unroll
        for (int r = 2; r <= W; ++r) l[r] = A::mul(Wn[(PH + r) % RL][PH], rs);
#pragma unroll
        for (int r = 0; r <= W; ++r)
            if (r % G == g) ring[((PH + r) < RL ? sb0 + PH + r : sb1 + PH + r - RL) * RS + r] = l[r];
        if (g == G - 1) ring[(sb0 + PH) * RS + RL] = rs;
        // rank-1 update of the window
#pragma unroll
        for (int r = 1; r <= W; ++r)
#pragma unroll
            for (int c = 1; c <= r; ++c)
                if (r > 1 || c > 1)
                    Wn[(PH + r) % RL][(PH + c) % RL] = A::fnma(l[r], l[c], Wn[(PH + r) % RL][(PH + c) % RL]);
        // band row k+1+W enters slot PH at columns k+1 .. k+1+W
        const V *er = sv + grp * CH + PH * RL;
#pragma unroll
        for (int c = 0; c <= W; ++c) Wn[PH][(PH + 1 + c) % RL] = er[W - c];
        if constexpr (F32) od[PH] = Wn[PH][PH];
        if constexpr (W >= 1) {
            d = dn;
            rs = rsn;
        } else {  // a diagonal block: the next pivot is the entering row's
            d = Wn[0][0];
            rs = A::rsqrt_(d);
        }
        if (k + 1 < m) {  // the pivot of row k+1
            if constexpr (F32)
                bad |= !(d > floor * od[P1]);
            else if (inf == 0 && !A::positive(d))
                inf = k + 2;
        }
    };
    // border step: column k of L21 (and row k of L11 out), k in the previous period
    auto border_step = [&](auto PHc, int kbase, int sbp) {
        constexpr int PH = decltype(PHc)::value;
        const int k = kbase + PH;
        V lr[RL];  // row k of L: lr[e] = L[k][k-e]
#pragma unroll
        for (int e = 0; e <= W; ++e) lr[e] = ring[(sbp + PH) * RS + e];
        const V rsk = ring[(sbp + PH) * RS + RL];  // 1 / L[k][k], the pivot's rsqrt
        const bool inb = k < m;
        const bool wr = live && inf == 0 && inb;
        // L21[b][k] = (A21[b][k] - sum_e L21[b][k-e] L[k][k-e]) / L[k][k].
        // A21[b][k] = A[m+b][k] is nonzero for k <= b (the wrap, stored in band
        // row k at offset W - b + k) and for m + b - W <= k < m (band row m+b
        // at offset m + b - k); neither slot is ever overwritten by L11.
        V val[NR > 0 ? NR : 1];
#pragma unroll
        for (int t = 0; t < NR; ++t) {
            const int b = g + G * t;
            V acc = A::zero();
            const int rr = m + b - k;
            if (live && b < W && k <= b) acc = A::from(band[(int64_t)k * RL + (W - b + k)]);
            if (live && b < W && inb && rr <= W) acc = A::from(band[(int64_t)(m + b) * RL + rr]);
#pragma unroll
            for (int e = 1; e <= W; ++e) acc = A::fnma(y[t][(PH - e + RL) % RL], lr[e], acc);
            V v = A::mul(acc, rsk);
            v = inb ? v : A::zero();  // past the block's end nothing more enters the sums
            val[t] = v;
            y[t][PH] = v;
            if (wr && b < W) bord[(int64_t)b * n + k] = A::to_double(v);
        }
        // corner sums: every lane of the group needs this column's W values
#pragma unroll
        for (int b2 = 0; b2 < W; ++b2) {
            const V v2 = A::shfl(val[b2 / G], gbase + b2 % G, FULL);
#pragma unroll
            for (int t = 0; t < NR; ++t) {
                const int b = g + G * t;
                if (b < W && b2 <= b) sacc[t][b2] = A::fma_(val[t], v2, sacc[t][b2]);
            }
        }
        // row k of L11 out (lane g: offsets e = g mod G; offsets e > k keep A's wrap values)
#pragma unroll
        for (int e = 0; e <= W; ++e) {
            if (e % G == g && wr && e <= k) {
                if constexpr (F32)
                    l11f[off + (int64_t)k * RL + e] = lr[e];
                else
                    band[(int64_t)k * RL + e] = A::to_double(lr[e]);
            }
        }
    };
    const int PW = (mmax - 1) / RL;
    for (int p = 0; p <= PW + 1; ++p) {
        cp_async_wait<0>();  // period p+1's rows have landed
        __syncwarp();        // ... and the ring rows of period p-1 are complete
        if (p <= PW) {
            const double *src = s64 + ((p + 1) & 1) * B * CH;
            for (int i = lane; i < B * CH; i += 32) sv[i] = A::from(src[i]);
        }
        __syncwarp();
        issue(p + 2);
        const int kbase = p * RL;
        const int sb0 = (p % 3) * RL, sb1 = ((p + 1) % 3) * RL, sbp = ((p + 2) % 3) * RL;
        if (p == 0) {
            auto f = [&](auto PHc) { band_step(PHc, kbase, sb0, sb1); };
            StaticFor<0, RL>::run(f);
        } else if (p <= PW) {
            auto f = [&](auto PHc) {
                band_step(PHc, kbase, sb0, sb1);
                border_step(PHc, kbase - RL, sbp);
            };
            StaticFor<0, RL>::run(f);
        } else {
            auto f = [&](auto PHc) { border_step(PHc, kbase - RL, sbp); };
            StaticFor<0, RL>::run(f);
        }
    }
    cp_async_wait<0>();
    __syncwarp();

    // the corner C = A22 - S, factored in FP64 by the group's first lane
    double *cs = s64 + grp * (W > 0 ? W * W : 1);
#pragma unroll
    for (int t = 0; t < NR; ++t) {
        const int b = g + G * t;
#pragma unroll
        for (int b2 = 0; b2 < W; ++b2)
            if (b < W && b2 <= b) cs[b * W + b2] = A::to_double(sacc[t][b2]);
    }
    __syncwarp();
    if (g == 0 && live) {
        int res = inf;
        if (F32 && bad) {
            res = kRescue;
        } else if (res == 0 && W > 0) {
            for (int i = 0; i < W; ++i)
                for (int j = 0; j <= i; ++j) cs[i * W + j] = band[(int64_t)(m + i) * RL + (i - j)] - cs[i * W + j];
            for (int i = 0; i < W && res == 0; ++i) {
                for (int j = 0; j <= i; ++j) {
                    double sv2 = cs[i * W + j];
                    for (int q = 0; q < j; ++q) sv2 -= cs[i * W + q] * cs[j * W + q];
                    if (j < i) {
                        cs[i * W + j] = sv2 / cs[j * W + j];
                    } else if (!(sv2 > 0.0)) {
                        res = m + i + 1;
                        break;
                    } else {
                        cs[i * W + i] = sqrt(sv2);
                    }
                }
            }
            if (res == 0)
                for (int i = 0; i < W; ++i)
                    for (int j = 0; j <= i; ++j) bord[(int64_t)i * n + m + j] = cs[i * W + j];
        }
        info[bi] = res;
    }
}

// One warp per slice of blocks of width W, G lanes per block.
template <class A, int W, int G>
__global__ void __launch_bounds__(32) k_pband_chol(const CholSlice *__restrict__ slices,
                                                   const int32_t *__restrict__ items,
                                                   const BlockDesc *__restrict__ blocks, double *__restrict__ out,
                                                   float *__restrict__ l11f, int32_t *__restrict__ info, float floor,
                                                   int rescue) {
    extern __shared__ __align__(16) unsigned char csm[];
    chol_slice<A, W, G>(slices[blockIdx.x], items, blocks, out, l11f, info, floor, rescue, csm);
}

// f(integral_constant<int, I>) for I = B .. E-1 on the host (the launchers'
// loop over the instantiated widths).
template <int B, int E>
struct HostStaticFor {
    template <class F>
    static void run(F &f) {
        f(std::integral_constant<int, B>{});
        HostStaticFor<B + 1, E>::run(f);
    }
};
template <int E>
struct HostStaticFor<E, E> {
    template <class F>
    static void run(F &) {}
};

// The FP32 pass's L11 (floats, at the blocks' offsets) into the FP64 blocks,
// for the blocks that were not sent to the FP64 rescue: entries with offset
// d <= row of rows < m.  One CTA of 256 threads per tile of kCommitTile
// elements of one block's band rows.
constexpr int kCommitTile = kCommitTileElems;
__global__ void __launch_bounds__(256) k_chol_commit(const int2 *__restrict__ tiles, const BlockDesc *__restrict__ blocks,
                                                     const int32_t *__restrict__ info, const float *__restrict__ l11f,
                                                     double *__restrict__ out);

// The launches of k_pband_chol<A, W, chol_lanes(W)> for every width present
// (slices [first, first + count) of the FP32 or the FP64 list), each on its
// own stream so that the widths run side by side; one translation unit per
// arithmetic.
void launch_chol_f32(sympix_plan_t pl, double *blocks, int32_t *info, int rescue, int wmax);
void launch_chol_f64(sympix_plan_t pl, double *blocks, int32_t *info, int rescue, int wmax);
void launch_chol_f2(sympix_plan_t pl, double *blocks, int32_t *info, int rescue, int wmax);

// FP64 and split FP32: widths up to kCholGroupFrom - 1 on k_pband_chol, wider
// bands (up to 16) on the 32-lane group kernel, side by side (measured at
// l_max 3000: the G-lane kernel is faster for w <= 8, the lane groups for
// w = 9 .. 11, whose few long chains the G-lane kernel runs on one warp each)
constexpr int kCholGroupFrom = 9;

// Launch the narrow-band factor of `precision`: FP32 over the plan's w <= 12
// periodic-band blocks (the pass, the commit, then the FP64 rescue); FP64 and
// split FP32 over w <= 16 (the G-lane kernel below kCholGroupFrom, the lane
// groups above, on a side stream).
void launch_pband_chol(sympix_plan_t pl, int precision, double *blocks, int32_t *info, cudaStream_t st);

}  // namespace sympix
