// Cholesky factorisation M = L L^T of every sampled block.
//
// A periodic-band block (half-width w, 2w+1 < n) couples only |i-j| <= w or
// |i-j| >= n-w.  With m = n - w its leading m x m part A11 is a plain band
// matrix, so L11 keeps the band; the last w rows (the border) fill in
// completely.  Work is O(n w^2) per block instead of O(n^3):
//   L11 L11^T = A11,   L21 = A21 L11^-T,   L22 L22^T = A22 - L21 L21^T.
//
// Kernels, by band width and arithmetic (the plan sorts blocks into lists):
//   w <= 8 (FP64, split FP32) and w <= 16 (FP32 on pband storage):
//       two passes.  The band pass runs one lane per block with the active
//       (w+1) x (w+1) triangle in registers and band rows staged into
//       shared memory a chunk ahead with cp.async; the border pass runs one
//       lane per border row (the forward substitution) and accumulates the
//       corner S on the fly, then one lane factors the w x w corner.
//       FP32 eliminates on a float copy of the band (the "shadow"),
//       converted once on the way in and once on the way out.
//   8 < w <= 16 (FP64, split FP32): one group of 32 lanes per block carries
//       the band window and the border rows in registers, one column per
//       step (band and border in one pass).
//   16 < w <= 64: one CTA per block, window, border columns and S in shared
//       memory indexed mod (w+1).
//   dense-format blocks with n <= 1024: a warp per block, right-looking,
//   FP64; larger ones: a CTA per block, blocked right-looking, FP64.
//
// FP32 rescue: an FP32 elimination whose pivot falls below a floor times the
// original diagonal marks its block, and the block is refactored in FP64
// from the untouched FP64 input.  A non-positive pivot in FP64 stops the
// block and records info = row + 1.
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

// One group of G lanes per periodic-band block with w <= G/2.
template <class A, int G, bool DENSE>
__global__ void __launch_bounds__(128) k_factor_band(int nitems, const int32_t *__restrict__ items,
                                                     const BlockDesc *__restrict__ blocks, double *__restrict__ out,
                                                     int32_t *__restrict__ info, int rescue) {
    typedef typename A::V V;
    constexpr int HW = G / 2;
    constexpr int RB = (G == 16) ? 8 : 2;  // corner rows per pass
    const int lane = threadIdx.x & 31;
    const int t = lane % G;
    const int gbase = lane - t;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (0xffffu << gbase);
    const int idx = (int)((blockIdx.x * blockDim.x + threadIdx.x) / G);
    if (idx >= nitems) return;  // uniform within the group
    const int bi = items[idx];
    if (rescue && info[bi] != kRescue) return;  // uniform within the group
    const BlockDesc bd = blocks[bi];
    const typename ViewOf<DENSE>::T v = ViewOf<DENSE>::make(out, bd);
    const int w = bd.w, m = bd.n - bd.w;
    const bool wl = t < HW;  // window lane or border lane
    const int r = wl ? t : t - HW;
    const bool used = r < w;

    // ring of prefetched band rows for this group: row rr in slot rr % kRing,
    // element c = column rr - w + c
    __shared__ double ring[128 / G][kRing][HW + 1];
    double(*myring)[HW + 1] = ring[threadIdx.x / G];
    auto prefetch = [&](int rr) {
        if (t <= w && rr < m) cp_async8(&myring[rr % kRing][t], v.row_elem(rr, t));
        cp_async_commit();
    };
#pragma unroll
    for (int s = 0; s < kPrefetch; ++s) prefetch(1 + w + s);

    V win[HW + 1];
#pragma unroll
    for (int c = 0; c <= HW; ++c) win[c] = A::zero();
    if (used) {
        if (wl) {
            const int i = 1 + r;
            if (i < m) {
#pragma unroll
                for (int c = 0; c <= HW; ++c)
                    if (c <= r + 1) win[c] = A::from(v.a(i, c));
            }
        } else {
#pragma unroll
            for (int c = 0; c <= HW; ++c)
                if (c <= w && c < m) win[c] = A::from(v.a(m + r, c));
        }
    }
    V d = A::from(v.a(0, 0));
    int inf = 0;
    for (int k = 0; k < m; ++k) {
        prefetch(k + 1 + w + kPrefetch);
        if (!A::positive(d)) {
            inf = k + 1;
            break;
        }
        const V rs = A::rsqrt_(d);
        if (t == 0) v.put_l(k, k, A::to_double(A::mul(d, rs)));
        const bool act = used && (!wl || k + 1 + r < m);
        const V l = act ? A::mul(win[0], rs) : A::zero();
        if (act) {
            if (wl)
                v.put_l(k + 1 + r, k, A::to_double(l));
            else
                v.put_b(r, k, A::to_double(l));
        }
        // rank-1 update of the band columns k+1..k+w
#pragma unroll
        for (int c = 1; c <= HW; ++c) {
            if (c > w) break;
            const V lc = A::shfl(l, gbase + c - 1, gmask);
            if (act && (!wl || c <= r + 1)) win[c] = A::fnma(l, lc, win[c]);
        }
        // row k+1's diagonal (a diagonal block, w = 0, reads it from memory)
        d = A::shfl(win[1], gbase, gmask);
        if (w == 0 && k + 1 < m) d = A::from(v.a(k + 1, k + 1));
        // shift the window one row down and one column right
        const int src = t + 1 < G ? gbase + t + 1 : gbase + t;
#pragma unroll
        for (int c = 0; c < HW; ++c) {
            const V nx = A::shfl(win[c + 1], src, gmask);
            win[c] = wl ? nx : win[c + 1];
        }
        win[HW] = A::zero();
        const int nc = k + 1 + w;  // row (window) and column (border) entering
        // the new window row arrived kPrefetch steps ago: each lane converts
        // one element, the bottom window lane gathers them
        cp_async_wait<kPrefetch>();
        __syncwarp(gmask);
        const V mine = (t <= w && nc < m) ? A::from(myring[nc % kRing][t]) : A::zero();
#pragma unroll
        for (int c = 0; c <= HW; ++c) {
            if (c > w) break;
            const V x = A::shfl(mine, gbase + c, gmask);
            if (wl && used && r == w - 1) win[c] = x;
        }
        if (!wl && used) {
            const V x = nc < m ? A::from(v.a(m + r, nc)) : A::zero();
#pragma unroll
            for (int c = 0; c <= HW; ++c)
                if (c == w) win[c] = x;
        }
    }
    cp_async_wait<0>();
    __syncwarp(gmask);
    if (inf == 0 && w > 0) {
        // corner S = A22 - L21 L21^T, lanes over the column index k
#pragma unroll
        for (int b0 = 0; b0 < HW; b0 += RB) {
            if (b0 >= w) break;
            V acc[RB][HW];
#pragma unroll
            for (int i = 0; i < RB; ++i)
#pragma unroll
                for (int bp = 0; bp < HW; ++bp) acc[i][bp] = A::zero();
            for (int k0 = 0; k0 < m; k0 += G) {
                const int k = k0 + t;
                V y[HW];
#pragma unroll
                for (int bb = 0; bb < HW; ++bb)
                    y[bb] = (bb < w && bb < b0 + RB && k < m) ? A::from(v.get_b(bb, k)) : A::zero();
#pragma unroll
                for (int i = 0; i < RB; ++i) {
                    const int b = b0 + i;
                    if (b < HW) {
#pragma unroll
                        for (int bp = 0; bp < HW; ++bp)
                            if (bp <= b) acc[i][bp] = A::fma_(y[b], y[bp], acc[i][bp]);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < RB; ++i) {
                const int b = b0 + i;
#pragma unroll
                for (int bp = 0; bp < HW; ++bp) {
                    if (bp <= b && b < HW) {
#pragma unroll
                        for (int off = G / 2; off > 0; off >>= 1)
                            acc[i][bp] = A::add(acc[i][bp], A::shfl_xor(acc[i][bp], off, gmask));
                        if (t == 0 && b < w)
                            v.put_b(b, m + bp, v.a(m + b, m + bp) - A::to_double(acc[i][bp]));
                    }
                }
            }
        }
        __syncwarp(gmask);
        if (t == 0) {
            // dense Cholesky of the w x w corner, FP64
            for (int i = 0; i < w && inf == 0; ++i) {
                for (int j = 0; j <= i; ++j) {
                    double s = v.get_b(i, m + j);
                    for (int k = 0; k < j; ++k) s -= v.get_b(i, m + k) * v.get_b(j, m + k);
                    if (j < i) {
                        v.put_b(i, m + j, s / v.get_b(j, m + j));
                    } else {
                        if (!(s > 0.0)) {
                            inf = m + i + 1;
                            break;
                        }
                        v.put_b(i, m + i, sqrt(s));
                    }
                }
            }
        }
    }
    if (t == 0) info[bi] = inf;
}

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

// Band pass for one block in one lane.  `stage` (pband storage only) is
// this lane's shared-memory area of 2 x kChunk x (w+1) doubles: band rows
// are copied into it a chunk ahead with cp.async, so no global load sits on
// the elimination chain.  DENSE storage reads rows from global directly.
template <class A, int WB, class View, bool STAGED>
__device__ __forceinline__ int band_pass(const View &v, double *stage) {
    typedef typename A::V V;
    const int w = v.w, m = v.m, RL = w + 1;
    auto issue = [&](int j) {
        if (STAGED) {
            const int r0 = j * kChunk;
            if (r0 < m) {
                const int cnt = min(kChunk, m - r0) * RL;
                double *dst = stage + (j & 1) * kChunk * RL;
                const double *src = v.row_elem(r0, w);  // element 0 of row r0
                for (int i = 0; i < cnt; ++i) cp_async8(dst + i, src + i);
            }
            cp_async_commit();
        }
    };
    // A[R][R - w + c] of a band row R < m (entering the window)
    auto row_val = [&](int R, int c) -> double {
        if (STAGED) return stage[((R / kChunk) & 1) * kChunk * RL + (R % kChunk) * RL + (w - c)];
        return *v.row_elem(R, c);
    };
    issue(0);
    issue(1);
    if (STAGED) cp_async_wait<1>();
    V W[WB + 1][WB + 1];
#pragma unroll
    for (int r = 0; r <= WB; ++r)
#pragma unroll
        for (int c = 0; c <= r; ++c) W[r][c] = (r <= w && r < m) ? A::from(v.a(r, c)) : A::zero();
    int next = 2;  // next chunk to issue
    for (int k = 0; k < m; ++k) {
        const V d = W[0][0];
        if (!A::positive(d)) {
            if (STAGED) cp_async_wait<0>();
            return k + 1;
        }
        const V rs = A::rsqrt_(d);
        v.put_l(k, k, A::to_double(A::mul(d, rs)));
        V l[WB + 1];
#pragma unroll
        for (int r = 1; r <= WB; ++r) {
            const bool on = r <= w && k + r < m;
            l[r] = on ? A::mul(W[r][0], rs) : A::zero();
            if (on) v.put_l(k + r, k, A::to_double(l[r]));
        }
#pragma unroll
        for (int r = 1; r <= WB; ++r)
#pragma unroll
            for (int c = 1; c <= r; ++c) W[r][c] = A::fnma(l[r], l[c], W[r][c]);
#pragma unroll
        for (int r = 0; r < WB; ++r)
#pragma unroll
            for (int c = 0; c <= r; ++c) W[r][c] = W[r + 1][c + 1];
        // row R = k + 1 + w enters the window
        const int R = k + 1 + w;
        if (STAGED && R < m && R % kChunk == 0) {
            // chunk R / kChunk was issued a chunk ago; the buffer of the
            // chunk before it is free for the one after
            if (R / kChunk + 1 >= next) {
                issue(next);
                ++next;
            }
            cp_async_wait<1>();
        }
#pragma unroll
        for (int c = 0; c <= WB; ++c) {
            const V x = (c <= w && R < m) ? A::from(row_val(R, c)) : A::zero();
#pragma unroll
            for (int r = 0; r <= WB; ++r)
                if (c <= r) {
                    if (r == w) W[r][c] = x;
                    if (r == WB && r != w) W[r][c] = A::zero();
                }
        }
    }
    if (STAGED) cp_async_wait<0>();
    return 0;
}

// Blocks of up to three width classes in one launch: CTAs [0, c0) take
// items0 (w <= 8, 32 lanes), the next c1 items1 (w <= 12) and the rest
// items2 (w <= 16), 16 lanes each for those.  Dynamic shared memory holds
// each lane's staging area (pband storage).
template <class A, bool DENSE, bool WIDE>
__global__ void __launch_bounds__(32) k_factor_band_pass(int n0, int n1, int n2, const int32_t *__restrict__ items0,
                                                         const int32_t *__restrict__ items1,
                                                         const int32_t *__restrict__ items2,
                                                         const BlockDesc *__restrict__ blocks, double *__restrict__ out,
                                                         int32_t *__restrict__ info, int rescue) {
    extern __shared__ double dsm[];
    const int c0 = (n0 + 31) / 32, c1 = (n1 + 15) / 16;
    int cta = blockIdx.x, list = 0, per = 32;
    if (cta >= c0) {
        cta -= c0;
        list = 1;
        per = 16;
        if (cta >= c1) {
            cta -= c1;
            list = 2;
        }
    }
    if ((int)threadIdx.x >= per) return;
    const int idx = cta * per + threadIdx.x;
    const int nl = list == 0 ? n0 : list == 1 ? n1 : n2;
    if (idx >= nl) return;
    const int bi = (list == 0 ? items0 : list == 1 ? items1 : items2)[idx];
    if (rescue && info[bi] != kRescue) return;
    const BlockDesc bd = blocks[bi];
    typedef typename ViewOf<DENSE>::T View;
    const View v = ViewOf<DENSE>::make(out, bd);
    // lane area: 2 chunks of kChunk rows of up to 9 (list 0) or 17 values,
    // padded by one double to spread the lanes over the banks
    const int area = (list == 0 ? 2 * kChunk * 9 : 2 * kChunk * 17) + 1;
    double *stage = DENSE ? nullptr : dsm + threadIdx.x * area;
    int res;
    if constexpr (WIDE) {
        res = list == 0   ? band_pass<A, 8, View, !DENSE>(v, stage)
              : list == 1 ? band_pass<A, 12, View, !DENSE>(v, stage)
                          : band_pass<A, 16, View, !DENSE>(v, stage);
    } else {
        res = band_pass<A, 8, View, !DENSE>(v, stage);
    }
    info[bi] = (rescue && res == 0) ? kRescued : res;
}

template <class A, int G2, int WB, class View, bool STAGED>
__device__ __forceinline__ void border_pass(const View &v, int t, int gbase, unsigned gmask, double *stage,
                                            int32_t *info_bi) {
    typedef typename A::V V;
    const int w = v.w, m = v.m, RL = w + 1;
    const int b = t;  // border row m + b
    const bool used = b < w;
    // the group's lanes stage the block's L band rows a chunk ahead
    auto issue = [&](int j) {
        if (STAGED) {
            const int r0 = j * kChunk;
            if (r0 < m) {
                const int cnt = min(kChunk, m - r0) * RL;
                double *dst = stage + (j & 1) * kChunk * RL;
                const double *src = v.row_elem(r0, w);
                for (int i = t; i < cnt; i += G2) cp_async8(dst + i, src + i);
            }
            cp_async_commit();
        }
    };
    auto lval = [&](int k, int col) -> double {  // L[k][col], col in [k-w, k]
        if (STAGED) return stage[((k / kChunk) & 1) * kChunk * RL + (k % kChunk) * RL + (k - col)];
        return v.get_l(k, col);
    };
    issue(0);
    issue(1);
    int next = 2;
    V y[WB];     // L[m+b][k-w+c], c = 0..w-1
    V sacc[WB];  // sum_k L[m+b][k] L[m+b'][k], b' <= b
#pragma unroll
    for (int c = 0; c < WB; ++c) {
        y[c] = A::zero();
        sacc[c] = A::zero();
    }
    const int kband = ((m - w) / kChunk) * kChunk;
    for (int k = 0; k < m; ++k) {
        if (STAGED && k % kChunk == 0) {
            // exact zeros in every lane's window: skip to the band part
            if (k > w && k < kband) {
                bool zero = true;
#pragma unroll
                for (int c = 0; c < WB; ++c) zero = zero && A::to_double(y[c]) == 0.0;
                if (__all_sync(gmask, zero)) {
                    if (used)
                        for (int kk = k; kk < kband; ++kk) v.put_b(b, kk, 0.0);
                    k = kband;
                    cp_async_wait<0>();
                    __syncwarp(gmask);
                    issue(k / kChunk);
                    issue(k / kChunk + 1);
                    next = k / kChunk + 2;
                }
            }
            if (k / kChunk + 1 >= next) {
                issue(next);
                ++next;
            }
            cp_async_wait<1>();
            __syncwarp(gmask);
        }
        // band row k of L11: entries c = 0..w at columns k-w+c (c = w: diagonal)
        const V e0 = (t <= w && k - w + t >= 0) ? A::from(lval(k, k - w + t)) : A::zero();
        const int t2 = t + G2;
        const V e1 = (t2 <= w && k - w + t2 >= 0) ? A::from(lval(k, k - w + t2)) : A::zero();
        V acc = A::zero();
        if (used && (k <= b || k >= m + b - w)) acc = A::from(v.a(m + b, k));
        V diag = A::zero();
#pragma unroll
        for (int c = 0; c <= WB; ++c) {
            if (c > w) break;
            const V lc = c < G2 ? A::shfl(e0, gbase + c, gmask) : A::shfl(e1, gbase + c - G2, gmask);
            if (c < w) {
#pragma unroll
                for (int cc = 0; cc < WB; ++cc)
                    if (cc == c) acc = A::fnma(y[cc], lc, acc);
            } else {
                diag = lc;
            }
        }
        const V rd = A::rsqrt_(diag);
        const V val = used ? A::mul(acc, A::mul(rd, rd)) : A::zero();
        if (used) v.put_b(b, k, A::to_double(val));
#pragma unroll
        for (int c = 0; c < WB; ++c) {
            if (c >= w) break;
            const V vc = A::shfl(val, gbase + c, gmask);
            if (c <= b) sacc[c] = A::fma_(val, vc, sacc[c]);
        }
#pragma unroll
        for (int c = 0; c + 1 < WB; ++c) y[c] = y[c + 1];
#pragma unroll
        for (int c = 0; c < WB; ++c)
            if (c == w - 1) y[c] = val;
        if (STAGED && (k + 1) % kChunk == 0) __syncwarp(gmask);  // chunk consumed by every lane
    }
    if (STAGED) cp_async_wait<0>();
    if (used) {
#pragma unroll
        for (int c = 0; c < WB; ++c)
            if (c <= b) v.put_b(b, m + c, v.a(m + b, m + c) - A::to_double(sacc[c]));
    }
    __syncwarp(gmask);
    if (t == 0) {
        // dense Cholesky of the w x w corner, FP64
        int inf = 0;
        for (int i = 0; i < w && inf == 0; ++i) {
            for (int j = 0; j <= i; ++j) {
                double s = v.get_b(i, m + j);
                for (int k = 0; k < j; ++k) s -= v.get_b(i, m + k) * v.get_b(j, m + k);
                if (j < i) {
                    v.put_b(i, m + j, s / v.get_b(j, m + j));
                } else {
                    if (!(s > 0.0)) {
                        inf = m + i + 1;
                        break;
                    }
                    v.put_b(i, m + i, sqrt(s));
                }
            }
        }
        *info_bi = inf;
    }
}

// Pass 2: CTAs [0, c0) run 8-lane groups on items0; the rest 16-lane groups
// on items1 then items2.  Each group stages its block's L band rows in
// shared memory (2 chunks).
template <class A, bool DENSE, bool WIDE>
__global__ void __launch_bounds__(128) k_factor_border_pass(int n0, int n1, int n2, const int32_t *__restrict__ items0,
                                                            const int32_t *__restrict__ items1,
                                                            const int32_t *__restrict__ items2,
                                                            const BlockDesc *__restrict__ blocks,
                                                            double *__restrict__ out, int32_t *__restrict__ info,
                                                            int rescue) {
    const int32_t want = rescue ? kRescued : 0;
    // 16 groups x 2 chunks x kChunk rows x 9 values (8-lane groups, w <= 8),
    // or 8 groups x 2 x kChunk x 17 (16-lane groups)
    __shared__ double stg[16 * 2 * kChunk * 9];
    typedef typename ViewOf<DENSE>::T View;
    const int c0 = (n0 + 15) / 16;
    const int lane = threadIdx.x & 31;
    if ((int)blockIdx.x < c0) {
        const int t = lane & 7, gbase = lane - t;
        const unsigned gmask = 0xFFu << gbase;
        const int grp = threadIdx.x / 8;
        const int idx = blockIdx.x * 16 + grp;
        if (idx >= n0) return;
        const int bi = items0[idx];
        if (info[bi] != want) return;  // a bad pivot in the band pass, or not this pass's block
        const BlockDesc bd = blocks[bi];
        const View v = ViewOf<DENSE>::make(out, bd);
        if (bd.w > 0) border_pass<A, 8, 8, View, !DENSE>(v, t, gbase, gmask, stg + grp * 2 * kChunk * 9, info + bi);
        return;
    }
    if constexpr (WIDE) {
        const int t = lane & 15, gbase = lane - t;
        const unsigned gmask = 0xFFFFu << gbase;
        const int grp = threadIdx.x / 16;
        const int idx = (blockIdx.x - c0) * 8 + grp;
        if (idx >= n1 + n2) return;
        const int bi = idx < n1 ? items1[idx] : items2[idx - n1];
        if (info[bi] != want) return;
        const BlockDesc bd = blocks[bi];
        const View v = ViewOf<DENSE>::make(out, bd);
        border_pass<A, 16, 16, View, !DENSE>(v, t, gbase, gmask, stg + grp * 2 * kChunk * 17, info + bi);
    }
}

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

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// One CTA per kTileE elements x 32 blocks of a slice.
__global__ void __launch_bounds__(256) k_f32_shadow_in(const int2 *__restrict__ tiles,
                                                       const F32Slice *__restrict__ slices,
                                                       const int32_t *__restrict__ items,
                                                       const BlockDesc *__restrict__ blocks,
                                                       const double *__restrict__ out, float *__restrict__ sh) {
    __shared__ float tile[kTileE][33];
    __shared__ int64_t s_off[32];
    __shared__ int s_cnt[32];
    const int2 tl = tiles[blockIdx.x];
    const F32Slice sl = slices[tl.x];
    const int RL = sl.w + 1, e0 = tl.y;
    if (threadIdx.x < 32) {
        int64_t off = 0;
        int cnt = 0;
        if ((int)threadIdx.x < sl.count) {
            const BlockDesc bd = blocks[items[sl.first + threadIdx.x]];
            off = bd.off_pband;
            cnt = bd.n * RL;
        }
        s_off[threadIdx.x] = off;
        s_cnt[threadIdx.x] = cnt;
    }
    __syncthreads();
#pragma unroll
    for (int i = threadIdx.x; i < 32 * kTileE; i += 256) {
        const int L = i / kTileE, e = i % kTileE;
        float v = 0.0f;
        if (e0 + e < s_cnt[L]) v = f64_to_f32_bits(out[s_off[L] + e0 + e]);
        tile[e][L] = v;
    }
    __syncthreads();
    const int lim = sl.rows * RL;
    float *dst = sh + sl.sh + (int64_t)e0 * 32;
#pragma unroll
    for (int i = threadIdx.x; i < 32 * kTileE; i += 256) {
        const int e = i >> 5, L = i & 31;
        if (e0 + e < lim) dst[e * 32 + L] = tile[e][L];
    }
}

// f(integral_constant<int, I>) for I = B .. E-1, expanded at compile time.
template <int B, int E>
struct StaticFor {
    template <class F>
    __device__ __forceinline__ static void run(F &f) {
        f(std::integral_constant<int, B>{});
        StaticFor<B + 1, E>::run(f);
    }
};
template <int E>
struct StaticFor<E, E> {
    template <class F>
    __device__ __forceinline__ static void run(F &) {}
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
template <int W>
__device__ __forceinline__ int f32_band(float *shs, int lane, int m, int mmax, float *stage, float floor,
                                        volatile int *prog) {
    constexpr int RL = W + 1, CH = RL * RL;
    float *band = shs + lane;  // element e at band[32 e]
    auto issue = [&](int per) {
        const int r0 = per * RL;
        if (r0 < mmax) {  // rows r0 .. r0 + W < the slice's rows
            float *dst = stage + (per & 1) * CH * 32;
            const float *src = shs + (int64_t)r0 * RL * 32;
            for (int i = lane; i < CH * 8; i += 32) cp_async16(dst + 4 * i, src + 4 * i);
        }
        cp_async_commit();
    };
    issue(1);
    float Wn[RL][RL];  // [row slot][column slot]
    float od[RL];      // original diagonal per row slot
#pragma unroll
    for (int r = 0; r <= W; ++r) {
#pragma unroll
        for (int c = 0; c <= r; ++c) Wn[r][c] = r < m ? band[((int64_t)r * RL + (r - c)) * 32] : 0.0f;
        od[r] = Wn[r][r];
    }
    // One elimination step at phase PH (k = p RL + PH).  lrow = band row
    // p RL; src = this lane's staged rows of period p + 1.  Rows >= m only
    // ever feed rows >= m, which nothing reads, so they need no masking.
    // The pivot d of row k and rs = 1/sqrt(d) arrive from the previous
    // step: each step forms the next pivot first (one product) and starts
    // its rsqrt before the rest of the update.
    bool bad = !(Wn[0][0] > floor * od[0]);
    float d = Wn[0][0], rs = rsqrtf(Wn[0][0]);
    auto step = [&](auto PHc, float *lrow, const float *src, bool live, int kbase) {
        constexpr int PH = decltype(PHc)::value;
        constexpr int P1 = (PH + 1) % RL;
        if (!live) return;
        lrow[PH * RL * 32] = d * rs;
        float l[RL];
        float dn = 0.0f, rsn = 0.0f;
        if constexpr (W >= 1) {
            l[1] = Wn[P1][PH] * rs;
            dn = fmaf(-l[1], l[1], Wn[P1][P1]);
            rsn = rsqrtf(dn);
        }
#pragma unroll
        for (int r = 2; r <= W; ++r) l[r] = Wn[(PH + r) % RL][PH] * rs;
#pragma unroll
        for (int r = 1; r <= W; ++r) lrow[((PH + r) * RL + r) * 32] = l[r];
#pragma unroll
        for (int r = 1; r <= W; ++r)
#pragma unroll
            for (int c = 1; c <= r; ++c)
                if (r > 1 || c > 1) Wn[(PH + r) % RL][(PH + c) % RL] = fmaf(-l[r], l[c], Wn[(PH + r) % RL][(PH + c) % RL]);
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
            rs = rsqrtf(d);
        }
        // the next pivot (rows >= m are not A11's); includes d <= 0 and NaN
        bad |= kbase + PH + 1 < m && !(d > floor * od[P1]);
    };
    const int PW = mmax / RL;  // the slice's last period
    for (int p = 0; p <= PW; ++p) {
        issue(p + 2);
        cp_async_wait<1>();  // period p + 1 has landed
        __syncwarp();        // ... for every lane's copies
        const float *src = stage + ((p + 1) & 1) * CH * 32 + lane;
        float *lrow = band + (int64_t)p * RL * RL * 32;
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
        // every 4th period: this period's L rows reach L2 (where the border
        // pass stages from) before the flag says rows < (p+1)(W+1) are final
        const bool publish = prog && (p & 3) == 3;
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
    return bad ? kRescue : 0;
}

template <int W>
struct F32BandDispatch {
    __device__ static int run(int w, float *shs, int lane, int m, int mmax, float *stage, float floor,
                              volatile int *prog = nullptr) {
        if (w == W) return f32_band<W>(shs, lane, m, mmax, stage, floor, prog);
        return F32BandDispatch<W - 1>::run(w, shs, lane, m, mmax, stage, floor, prog);
    }
};
template <>
struct F32BandDispatch<0> {
    __device__ static int run(int w, float *shs, int lane, int m, int mmax, float *stage, float floor,
                              volatile int *prog = nullptr) {
        return w == 0 ? f32_band<0>(shs, lane, m, mmax, stage, floor, prog) : -1;
    }
};

constexpr int kF32BandStage = 2 * 17 * 17 * 32;  // floats: two periods of W = 16, 32 lanes

// One warp per slice, one lane per block.
__global__ void __launch_bounds__(32) k_f32_band_pass(const F32Slice *__restrict__ slices,
                                                      const int32_t *__restrict__ items,
                                                      const BlockDesc *__restrict__ blocks, float *__restrict__ sh,
                                                      int32_t *__restrict__ info, float floor) {
    extern __shared__ __align__(16) float fsm[];
    const F32Slice sl = slices[blockIdx.x];
    const int lane = threadIdx.x;
    int m = 0, bi = -1;
    if (lane < sl.count) {
        bi = items[sl.first + lane];
        m = blocks[bi].n - sl.w;
    }
    const int r = F32BandDispatch<16>::run(sl.w, sh + sl.sh, lane, m, sl.rows - sl.w, fsm, floor);
    if (bi >= 0) info[bi] = r;
}

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
// published as final (*prog = periods done), and take the blocks' band-pass
// results from bandres at the end.
template <int W, int NT, bool FUSED>
__device__ __forceinline__ void f32_border(const F32Slice &sl, const float *__restrict__ shs, float *__restrict__ l21,
                                           const double *__restrict__ out, const int64_t *s_off, const int *s_n,
                                           const int *s_live, float *stage, int *binfo, volatile int *prog,
                                           const int *bandres) {
    constexpr int RL = W + 1, CH = RL * RL;
    constexpr int NWARP = NT / 32;
    constexpr int R = (W + NWARP - 1) / NWARP;  // border rows per lane
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
    auto issue = [&](int per) {
        const int r0 = per * RL;
        if (r0 < kc) {  // rows r0 .. r0 + W < the slice's rows
            if (FUSED) {  // wait until the band warp has finished these rows
                int spins = 0;
                while (*prog < per + 1 && ++spins < (1 << 22)) __nanosleep(64);
                __threadfence_block();
            }
            float *dst = stage + (per % 3) * CH * 32;
            const float *src = shs + (int64_t)r0 * RL * 32;
            for (int i = tb; i < CH * 8; i += NT) cp_async16(dst + 4 * i, src + 4 * i);
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
                vb[(b * RL + PH) * 32 + lane] = val;
                if (!TAIL || k < kc) l21[((int64_t)b * kc + k) * 32 + lane] = val;
            }
        }
    };
    // corner sums S[b][b2] = sum_k L21[b][k] L21[b2][k], b2 <= b: the
    // W (W+1)/2 pairs are dealt round-robin to the warps, lane = block;
    // each period's L21 values pass through vbuf
    constexpr int NPAIR = W * (W + 1) / 2, NP = (NPAIR + NWARP - 1) / NWARP;
    const int wq = tb >> 5;
    int pb[NP > 0 ? NP : 1], pb2[NP > 0 ? NP : 1];
    float sacc[NP > 0 ? NP : 1];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
        int j = wq + NWARP * i, bb = 0;
        while (j > bb) {  // pair j = bb (bb+1)/2 + b2
            j -= bb + 1;
            ++bb;
        }
        pb[i] = bb < W ? bb : 0;
        pb2[i] = bb < W ? j : 0;
        sacc[i] = 0.0f;
    }
    auto accumulate = [&](const float *v) {
#pragma unroll
        for (int i = 0; i < NP; ++i) {
            if (wq + NWARP * i >= NPAIR) break;
            const float *x = v + pb[i] * RL * 32 + lane, *z = v + pb2[i] * RL * 32 + lane;
#pragma unroll
            for (int c = 0; c < RL; ++c) sacc[i] = fmaf(x[c * 32], z[c * 32], sacc[i]);
        }
    };
    issue(0);
    issue(1);
    const int PW = (kc - 1) / RL;  // the last period
    for (int p = 0; p <= PW; ++p) {
        cp_async_wait<1>();  // period p has landed
        bsync();             // ... for every thread's copies; period p-1's buffer is free
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
    __syncthreads();  // (fused: the band warp is done too, bandres is final)
    accumulate(vbuf + (PW & 1) * W * RL * 32);
    // the corner: sums to shared memory [block][b][b2], then one thread per
    // block factors C = A22 - S = L22 L22^T in FP64
    float *sS = stage;  // the staging is free now
    bsync();
#pragma unroll
    for (int i = 0; i < NP; ++i)
        if (wq + NWARP * i < NPAIR) sS[(lane * W + pb[i]) * W + pb2[i]] = sacc[i];
    bsync();
    const bool live_end = FUSED ? (live && bandres[lane] == 0) : live;
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

template <int W, int WMIN, int NT, bool FUSED = false>
struct F32BorderDispatch {
    __device__ static void run(int w, const F32Slice &sl, const float *shs, float *l21, const double *out,
                               const int64_t *s_off, const int *s_n, const int *s_live, float *stage, int *binfo,
                               volatile int *prog = nullptr, const int *bandres = nullptr) {
        if (w == W) {
            f32_border<W, NT, FUSED>(sl, shs, l21, out, s_off, s_n, s_live, stage, binfo, prog, bandres);
            return;
        }
        F32BorderDispatch<W - 1, WMIN, NT, FUSED>::run(w, sl, shs, l21, out, s_off, s_n, s_live, stage, binfo, prog,
                                                       bandres);
    }
};
template <int WMIN, int NT, bool FUSED>
struct F32BorderDispatch<WMIN - 1, WMIN, NT, FUSED> {
    __device__ static void run(int, const F32Slice &, const float *, float *, const double *, const int64_t *,
                               const int *, const int *, float *, int *, volatile int * = nullptr,
                               const int * = nullptr) {}
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

// Band and border passes of one slice in one CTA, widths 1..kFusedWMax:
// warp 0 eliminates the band (f32_band) and publishes after every period
// how many periods of L11 rows are final; kFusedBorderThreads threads run
// the border sweep (f32_border, FUSED) behind it, so the two latency-bound
// chains overlap instead of running one after the other.  The border's waits
// are bounded (a wait that runs out lets the sweep proceed; it cannot run
// out unless the band warp stalls for ~0.3 s).
constexpr int kFusedWMax = 12, kFusedBorderThreads = 320;
constexpr int kFusedBandStage = 2 * 13 * 13 * 32;  // floats: two periods of W = 12
// floats: band stage, then three staged periods, two periods of L21 values
// and the last W columns of A21, W = 12
constexpr int kFusedSmem = kFusedBandStage + 3 * 13 * 13 * 32 + 2 * 12 * 13 * 32 + 12 * 12 * 32;

__global__ void __launch_bounds__(32 + kFusedBorderThreads)
    k_f32_fused(const F32Slice *__restrict__ slices, const int32_t *__restrict__ items,
                const BlockDesc *__restrict__ blocks, float *__restrict__ sh, float *__restrict__ l21,
                const double *__restrict__ out, int32_t *__restrict__ info, float floor) {
    extern __shared__ __align__(16) float fsm[];
    __shared__ SliceBlocks t;
    __shared__ int binfo[32], bandres[32];
    __shared__ int prog_s;
    volatile int *prog = &prog_s;
    const F32Slice sl = slices[blockIdx.x];
    load_slice_blocks(t, sl, items, blocks, nullptr);
    if (threadIdx.x == 0) *prog = 0;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int L = threadIdx.x;
        const int m = L < sl.count ? t.n[L] - sl.w : 0;
        bandres[L] = F32BandDispatch<kFusedWMax>::run(sl.w, sh + sl.sh, L, m, sl.rows - sl.w, fsm, floor, prog);
        __syncthreads();  // the border sweep's end
    } else if (sl.w == 0) {
        __syncthreads();
    } else {
        F32BorderDispatch<kFusedWMax, 1, kFusedBorderThreads, true>::run(
            sl.w, sl, sh + sl.sh, l21 + sl.l21, out, t.off, t.n, t.live, fsm + kFusedBandStage, binfo, prog,
            bandres);
    }
    __syncthreads();
    if (threadIdx.x < 32 && threadIdx.x < sl.count) {
        const int L = threadIdx.x;
        info[t.bi[L]] = (bandres[L] != 0 || sl.w == 0) ? bandres[L] : binfo[L];
    }
}

// The factor back to the FP64 blocks: L11 rows from the band shadow and
// L21 rows from the border buffer, 64 elements x 32 blocks per CTA, through
// a shared-memory transpose (coalesced on both sides).  Blocks sent to the
// FP64 rescue are skipped.
__global__ void __launch_bounds__(256) k_f32_out(const int2 *__restrict__ tiles, const F32Slice *__restrict__ slices,
                                                 const int32_t *__restrict__ items,
                                                 const BlockDesc *__restrict__ blocks,
                                                 const int32_t *__restrict__ info, const float *__restrict__ sh,
                                                 const float *__restrict__ l21, double *__restrict__ out) {
    __shared__ float tile[kTileE][33];
    __shared__ int64_t s_off[32];
    __shared__ int s_n[32], s_live[32];
    const int2 tl = tiles[blockIdx.x];
    const F32Slice sl = slices[tl.x];
    const int W = sl.w, RL = W + 1;
    const bool part21 = tl.y < 0;
    const int e0 = part21 ? -1 - tl.y : tl.y;
    if (threadIdx.x < 32) {
        const int L = threadIdx.x;
        int64_t off = 0;
        int n = 0, live = 0;
        if (L < sl.count) {
            const int bi = items[sl.first + L];
            const BlockDesc bd = blocks[bi];
            off = bd.off_pband;
            n = bd.n;
            live = info[bi] != kRescue;
        }
        s_off[L] = off;
        s_n[L] = n;
        s_live[L] = live;
    }
    const int kc = sl.rows - W;
    const int lim = part21 ? W * kc : sl.rows * RL;
    const float *src = (part21 ? l21 + sl.l21 : sh + sl.sh) + (int64_t)e0 * 32;
#pragma unroll
    for (int i = threadIdx.x; i < kTileE * 32; i += 256) {
        const int e = i >> 5, L = i & 31;
        tile[e][L] = (e0 + e < lim) ? src[e * 32 + L] : 0.0f;
    }
    __syncthreads();
    // every element of this thread has the same e (its lanes differ): the
    // element's (row, offset) or (border row, column) is formed once
    const int e = threadIdx.x % kTileE, ee = e0 + e;
    if (ee >= lim) return;
    const int q = part21 ? ee / kc : ee / RL;          // border row b, or band row
    const int r = part21 ? ee - q * kc : ee - q * RL;  // column k, or offset d
#pragma unroll
    for (int L = threadIdx.x / kTileE; L < 32; L += 256 / kTileE) {
        const int n = s_n[L], m = n - W;
        const bool ok = s_live[L] && (part21 ? r < m : (q < m && r <= q));
        if (ok) {
            const int64_t dst = part21 ? s_off[L] + (int64_t)n * RL + (int64_t)q * n + r : s_off[L] + ee;
            out[dst] = f32_to_f64_bits(tile[e][L]);
        }
    }
}

// ---------------------------------------------------------------------------
// Wide bands (16 < w <= 64): one CTA per block.
//
// The active band window (rows k..k+w, columns k..k+w), the w border rows at
// columns k..k+w and the corner accumulator S live in shared memory; rows
// and columns are stored at index mod (w+1), so moving the window to column
// k+1 costs nothing: the slot of row/column k is reused for k+1+w.  Per
// column: thread 0 forms the pivot, the threads scale the column (band and
// border), then apply the rank-1 update to the band window, the border rows
// and S while the next band row and border column, loaded one column ahead,
// go into the freed slots.  T = double or float; the float version sends a
// block whose pivot falls below the floor to the FP64 rescue.
// ---------------------------------------------------------------------------
constexpr int kWideMax = 64;

template <typename T>
__device__ __forceinline__ T wide_from(double x);
template <>
__device__ __forceinline__ double wide_from<double>(double x) { return x; }
template <>
__device__ __forceinline__ float wide_from<float>(double x) { return f64_to_f32_bits(x); }
__device__ __forceinline__ double wide_to(double x) { return x; }
__device__ __forceinline__ double wide_to(float x) { return f32_to_f64_bits(x); }

// Where the wide kernel writes L: straight into the FP64 blocks (FP64), or
// into the FP32 band shadow, copied to the FP64 blocks only once the block
// has factored without reaching the pivot floor (so an FP64 rescue still
// finds its input intact).
template <typename T, class View>
struct WideSink;
template <class View>
struct WideSink<double, View> {
    View v;
    __device__ void put_l(int i, int j, double x) const { v.put_l(i, j, x); }
    __device__ void put_b(int b, int j, double x) const { v.put_b(b, j, x); }
    __device__ double get_b(int b, int j) const { return v.get_b(b, j); }
};
template <class View>
struct WideSink<float, View> {
    float *band;  // shadow: n x (w+1) band, then w x n border
    int n, w;
    __device__ void put_l(int i, int j, float x) const { band[(int64_t)i * (w + 1) + (i - j)] = x; }
    __device__ void put_b(int b, int j, float x) const { band[(int64_t)n * (w + 1) + (int64_t)b * n + j] = x; }
    __device__ double get_b(int b, int j) const {
        return f32_to_f64_bits(band[(int64_t)n * (w + 1) + (int64_t)b * n + j]);
    }
};

template <typename T, bool DENSE>
__global__ void __launch_bounds__(256) k_factor_wide(int nitems, const int32_t *__restrict__ items,
                                                     const BlockDesc *__restrict__ blocks, double *__restrict__ out,
                                                     int32_t *__restrict__ info, int rescue, float floor,
                                                     float *__restrict__ shadow) {
    extern __shared__ double wsm_raw[];
    T *wsm = reinterpret_cast<T *>(wsm_raw);
    const int bi = items[blockIdx.x];
    if (rescue && info[bi] != kRescue) return;
    const BlockDesc bd = blocks[bi];
    typedef typename ViewOf<DENSE>::T View;
    const View v = ViewOf<DENSE>::make(out, bd);
    const int w = bd.w, m = bd.n - bd.w, S = w + 1;
    auto make_sink = [&]() {
        if constexpr (sizeof(T) == 4)
            return WideSink<T, View>{shadow + bd.off_pband, bd.n, w};
        else
            return WideSink<T, View>{v};
    };
    const WideSink<T, View> sink = make_sink();
    T *Wn = wsm;         // S x S, [row mod S][col mod S]
    T *Bd = Wn + S * S;  // w x S, [b][col mod S]
    T *Sc = Bd + w * S;  // w x w corner accumulator
    T *lc = Sc + w * w;  // S: column k of L (band rows k..k+w)
    T *lb = lc + S;      // w: column k of L (border rows)
    T *od = lb + w;      // S: original diagonal of the window rows
    __shared__ T piv;
    __shared__ int fail;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < S * S; e += nt) {
        const int r = e / S, c = e % S;
        Wn[e] = (c <= r && r < m) ? wide_from<T>(v.a(r, c)) : T(0);
        if (c == r) od[r] = Wn[e];
    }
    for (int e = tid; e < w * S; e += nt) {
        const int b = e / S, c = e % S;
        Bd[e] = c < m ? wide_from<T>(v.a(m + b, c)) : T(0);
    }
    for (int e = tid; e < w * w; e += nt) {
        const int b = e / w, c = e % w;
        Sc[e] = c <= b ? wide_from<T>(v.a(m + b, m + c)) : T(0);
    }
    if (tid == 0) fail = 0;
    const int nband = w * (w + 1) / 2, nbord = w * w, ncorner = w * (w + 1) / 2;
    const int e0 = nband + nbord + ncorner, total = e0 + S;
    // the new-row element this thread stores each column (c < S), if any
    int myc = -1;
    for (int e = tid; e < total; e += nt)
        if (e >= e0) myc = e - e0;
    auto fetch = [&](int nc, T &pa, T &pb) {
        pa = (myc >= 0 && nc < m) ? wide_from<T>(v.a(nc, nc - w + myc)) : T(0);
        pb = (myc >= 0 && myc < w && nc < m) ? wide_from<T>(v.a(m + myc, nc)) : T(0);
    };
    T pa, pb;
    fetch(1 + w, pa, pb);
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        const int ks = k % S;
        if (tid == 0) {
            const T d = Wn[ks * S + ks];
            if (!(d > T(floor) * od[ks])) {
                fail = (sizeof(T) == 4) ? kRescue : k + 1;
            } else {
                const T lkk = sqrt(d);
                piv = T(1) / lkk;
                sink.put_l(k, k, lkk);
            }
        }
        __syncthreads();
        if (fail) break;
        const T rs = piv;
        for (int r = tid; r < S + w; r += nt) {
            if (r == 0) {
                lc[0] = T(0);
            } else if (r <= w) {
                const int row = k + r;
                const T l = row < m ? Wn[(row % S) * S + ks] * rs : T(0);
                lc[r] = l;
                if (row < m) sink.put_l(row, k, l);
            } else {
                const int b = r - S;
                const T l = Bd[b * S + ks] * rs;
                lb[b] = l;
                sink.put_b(b, k, l);
            }
        }
        __syncthreads();
        const int nc = k + 1 + w;
        for (int e = tid; e < total; e += nt) {
            if (e < nband) {
                int r = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f) + 1;
                while (r * (r - 1) / 2 > e) --r;
                while ((r + 1) * r / 2 <= e) ++r;
                const int c = e - r * (r - 1) / 2 + 1;
                const int row = k + r;
                if (row < m) Wn[(row % S) * S + (k + c) % S] -= lc[r] * lc[c];
            } else if (e < nband + nbord) {
                const int f = e - nband, b = f / w, c = f % w + 1;
                Bd[b * S + (k + c) % S] -= lb[b] * lc[c];
            } else if (e < e0) {
                const int f = e - nband - nbord;
                int b = (int)((sqrtf(8.0f * f + 1.0f) - 1.0f) * 0.5f);
                while (b * (b + 1) / 2 > f) --b;
                while ((b + 1) * (b + 2) / 2 <= f) ++b;
                const int c = f - b * (b + 1) / 2;
                Sc[b * w + c] -= lb[b] * lb[c];
            } else {
                // band row nc (columns k+1..nc) and the border rows' column nc
                // into the slot freed by row/column k
                const int c = e - e0;
                if (nc < m) {
                    Wn[ks * S + (k + 1 + c) % S] = pa;
                    if (c == w) od[ks] = pa;
                }
                if (c < w) Bd[c * S + ks] = pb;
            }
        }
        fetch(nc + 1, pa, pb);
        __syncthreads();
    }
    if (fail) {
        if (tid == 0) info[bi] = fail;
        return;
    }
    __shared__ int cinf;
    if (tid == 0) {
        // the w x w corner, FP64 arithmetic
        int inf = 0;
        for (int i = 0; i < w && inf == 0; ++i) {
            for (int j = 0; j <= i; ++j) {
                double s = wide_to(Sc[i * w + j]);
                for (int q = 0; q < j; ++q) s -= sink.get_b(i, m + q) * sink.get_b(j, m + q);
                if (j < i) {
                    sink.put_b(i, m + j, T(s / sink.get_b(j, m + j)));
                } else {
                    if (!(s > 0.0)) {
                        inf = m + i + 1;
                        break;
                    }
                    sink.put_b(i, m + i, T(sqrt(s)));
                }
            }
        }
        if (sizeof(T) == 4 && inf) inf = kRescue;  // let FP64 decide
        cinf = inf;
        info[bi] = inf;
    }
    if constexpr (sizeof(T) == 4) {
        // the block factored in FP32: copy L from the shadow
        __syncthreads();
        if (cinf) return;
        const int64_t nb = (int64_t)m * S;  // band rows < m
        for (int64_t e = tid; e < nb; e += nt) {
            const int row = (int)(e / S), d = (int)(e % S);
            if (d <= row) out[bd.off_pband + e] = f32_to_f64_bits(sink.band[e]);
        }
        const int64_t bo = (int64_t)bd.n * S;
        for (int64_t e = tid; e < (int64_t)w * bd.n; e += nt) {
            const int b = (int)(e / bd.n), j = (int)(e % bd.n);
            if (j <= m + b) out[bd.off_pband + bo + e] = f32_to_f64_bits(sink.band[bo + e]);
        }
    }
}

// One warp per dense-format block: right-looking, FP64, in place.
__global__ void __launch_bounds__(128) k_factor_dense(int nitems, const int32_t *__restrict__ items,
                                                      const BlockDesc *__restrict__ blocks, double *__restrict__ out,
                                                      int dense_storage, int32_t *__restrict__ info) {
    const int lane = threadIdx.x & 31;
    const int idx = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (idx >= nitems) return;
    const int bi = items[idx];
    const BlockDesc bd = blocks[bi];
    const int n = bd.n;
    double *p = out + (dense_storage ? bd.off_dense : bd.off_pband);
    int inf = 0;
    for (int k = 0; k < n; ++k) {
        const double dkk = p[(int64_t)k * n + k];
        if (!(dkk > 0.0)) {
            inf = k + 1;
            break;
        }
        const double lkk = sqrt(dkk);
        const double rl = 1.0 / lkk;
        __syncwarp();
        if (lane == 0) p[(int64_t)k * n + k] = lkk;
        for (int i = k + 1 + lane; i < n; i += 32) p[(int64_t)i * n + k] *= rl;
        __syncwarp();
        for (int j = k + 1; j < n; ++j) {
            const double ljk = p[(int64_t)j * n + k];
            for (int i = j + lane; i < n; i += 32) p[(int64_t)i * n + j] -= p[(int64_t)i * n + k] * ljk;
        }
        __syncwarp();
    }
    if (lane == 0) info[bi] = inf;
}

// Dense blocks with n > 1024: one CTA of 256 threads per block, right-looking
// blocked Cholesky in FP64 with panels of 32 columns.  Per panel: warp 0
// factors the 32 x 32 diagonal block in shared memory; the rows below solve
// against it (forward substitution, 64 rows at a time staged in shared
// memory); the trailing lower triangle takes the rank-32 update in 64 x 64
// tiles, each thread a 4 x 4 sub-tile.  The matrix stays in global memory
// (row-major n x n at the block's offset; the lower triangle is read and
// written).  info = first non-positive pivot row + 1, or 0.
constexpr int kDenseNB = 32, kDenseT = 64;

__global__ void __launch_bounds__(256) k_factor_dense_cta(int nitems, const int32_t *__restrict__ items,
                                                          const BlockDesc *__restrict__ blocks,
                                                          double *__restrict__ out, int dense_storage,
                                                          int32_t *__restrict__ info) {
    __shared__ double sd[kDenseNB][kDenseNB + 1];
    __shared__ double pa[kDenseT][kDenseNB + 1], pb[kDenseT][kDenseNB + 1];
    __shared__ int s_inf;
    if ((int)blockIdx.x >= nitems) return;
    const int bi = items[blockIdx.x];
    const BlockDesc bd = blocks[bi];
    const int n = bd.n;
    double *A = out + (dense_storage ? bd.off_dense : bd.off_pband);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_inf = 0;
    __syncthreads();
    for (int k0 = 0; k0 < n; k0 += kDenseNB) {
        const int nb = min(kDenseNB, n - k0);
        // (1) diagonal block
        for (int e = tid; e < kDenseNB * kDenseNB; e += 256) {
            const int r = e / kDenseNB, c = e % kDenseNB;
            sd[r][c] = (r < nb && c <= r) ? A[(int64_t)(k0 + r) * n + k0 + c] : 0.0;
        }
        __syncthreads();
        if (warp == 0) {
            for (int k = 0; k < nb; ++k) {
                const double dkk = sd[k][k];
                if (!(dkk > 0.0)) {  // uniform across the warp
                    if (lane == 0) s_inf = k0 + k + 1;
                    break;
                }
                const double lkk = sqrt(dkk), rl = 1.0 / lkk;
                __syncwarp();
                if (lane == 0) sd[k][k] = lkk;
                if (lane > k && lane < nb) sd[lane][k] *= rl;
                __syncwarp();
                for (int j = k + 1; j < nb; ++j) {
                    const double ljk = sd[j][k];
                    if (lane >= j && lane < nb) sd[lane][j] -= sd[lane][k] * ljk;
                }
                __syncwarp();
            }
        }
        __syncthreads();
        if (s_inf) break;  // uniform: read after the barrier
        for (int e = tid; e < nb * nb; e += 256) {
            const int r = e / nb, c = e % nb;
            if (c <= r) A[(int64_t)(k0 + r) * n + k0 + c] = sd[r][c];
        }
        const int r0 = k0 + nb;
        // (2) panel: L[i][k0..] = A[i][k0..] L_kk^-T, 64 rows at a time
        for (int i0 = r0; i0 < n; i0 += kDenseT) {
            const int ni = min(kDenseT, n - i0);
            __syncthreads();
            for (int e = tid; e < kDenseT * kDenseNB; e += 256) {
                const int r = e / kDenseNB, c = e % kDenseNB;
                pa[r][c] = (r < ni && c < nb) ? A[(int64_t)(i0 + r) * n + k0 + c] : 0.0;
            }
            __syncthreads();
            if (tid < ni) {
                for (int c = 0; c < nb; ++c) {
                    double x = pa[tid][c];
                    for (int t = 0; t < c; ++t) x -= pa[tid][t] * sd[c][t];
                    pa[tid][c] = x / sd[c][c];
                }
            }
            __syncthreads();
            for (int e = tid; e < kDenseT * kDenseNB; e += 256) {
                const int r = e / kDenseNB, c = e % kDenseNB;
                if (r < ni && c < nb) A[(int64_t)(i0 + r) * n + k0 + c] = pa[r][c];
            }
        }
        // (3) trailing update of the lower triangle, 64 x 64 tiles
        const int ty = tid / 16, tx = tid % 16;  // rows 4 ty .. 4 ty + 3, columns 4 tx .. 4 tx + 3
        for (int i0 = r0; i0 < n; i0 += kDenseT) {
            for (int j0 = r0; j0 <= i0; j0 += kDenseT) {
                __syncthreads();
                for (int e = tid; e < kDenseT * kDenseNB; e += 256) {
                    const int r = e / kDenseNB, c = e % kDenseNB;
                    pa[r][c] = (i0 + r < n && c < nb) ? A[(int64_t)(i0 + r) * n + k0 + c] : 0.0;
                    pb[r][c] = (j0 + r < n && c < nb) ? A[(int64_t)(j0 + r) * n + k0 + c] : 0.0;
                }
                __syncthreads();
                double acc[4][4];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
                for (int c = 0; c < nb; ++c) {
                    double xa[4], xb[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        xa[a] = pa[4 * ty + a][c];
                        xb[a] = pb[4 * tx + a][c];
                    }
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] = fma(xa[a], xb[b], acc[a][b]);
                }
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int i = i0 + 4 * ty + a;
                    if (i >= n) continue;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int j = j0 + 4 * tx + b;
                        if (j <= i) A[(int64_t)i * n + j] -= acc[a][b];
                    }
                }
            }
        }
        __syncthreads();
    }
    if (tid == 0) info[bi] = s_inf;
}

}  // namespace sympix

using namespace sympix;

// FP32 runs both passes for every band width up to 16; FP64 and split FP32
// (twice the registers) run them for w <= 8 and factor wider bands with
// lane groups.
template <class A>
static void launch_band(sympix_plan_t pl, bool dense, double *blocks, int32_t *info, cudaStream_t st,
                        int rescue = 0) {
    constexpr bool wide = std::is_same<A, ArF32>::value;
    const int n0 = (int)pl->factor_items[0].size();
    const int n1 = (int)pl->factor_items[1].size(), n2 = (int)pl->factor_items[2].size();
    const int w1 = wide ? n1 : 0, w2 = wide ? n2 : 0;
    const int32_t *i0 = pl->d_factor_items[0].p, *i1 = pl->d_factor_items[1].p, *i2 = pl->d_factor_items[2].p;
    if (n0 + w1 + w2 > 0) {
        const unsigned g1 = (unsigned)((n0 + 31) / 32 + (w1 + 15) / 16 + (w2 + 15) / 16);
        const unsigned g2 = (unsigned)((n0 + 15) / 16 + (w1 + w2 + 7) / 8);
        const size_t smem = (size_t)32 * (2 * kChunk * 17 + 1) * sizeof(double);
        if (dense) {
            k_factor_band_pass<A, true, wide><<<g1, 32, 0, st>>>(n0, w1, w2, i0, i1, i2, pl->d_blocks.p, blocks, info,
                                                                 rescue);
            k_factor_border_pass<A, true, wide><<<g2, 128, 0, st>>>(n0, w1, w2, i0, i1, i2, pl->d_blocks.p, blocks, info,
                                                                    rescue);
        } else {
            cudaFuncSetAttribute(k_factor_band_pass<A, false, wide>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
            k_factor_band_pass<A, false, wide><<<g1, 32, smem, st>>>(n0, w1, w2, i0, i1, i2, pl->d_blocks.p, blocks,
                                                                     info, rescue);
            k_factor_border_pass<A, false, wide><<<g2, 128, 0, st>>>(n0, w1, w2, i0, i1, i2, pl->d_blocks.p, blocks,
                                                                     info, rescue);
        }
    }
    if constexpr (!wide) {
        // wider bands: lane groups of 32 (band and border in one pass)
        for (int l = 1; l <= 2; ++l) {
            const int nl = (int)pl->factor_items[l].size();
            if (!nl) continue;
            const unsigned grid = (unsigned)((nl * 32 + 127) / 128);
            if (dense)
                k_factor_band<A, 32, true><<<grid, 128, 0, st>>>(nl, pl->d_factor_items[l].p, pl->d_blocks.p, blocks,
                                                                info, rescue);
            else
                k_factor_band<A, 32, false><<<grid, 128, 0, st>>>(nl, pl->d_factor_items[l].p, pl->d_blocks.p, blocks,
                                                                 info, rescue);
        }
    }
}

extern "C" int sympix_factor_blocks(sympix_plan_t pl, int storage, int precision, double *blocks, int32_t *info,
                                    void *stream) {
    if (!pl || !blocks || !info) return set_error(SYMPIX_EINVAL, "sympix_factor_blocks: NULL argument");
    if (storage != SYMPIX_STORE_PBAND && storage != SYMPIX_STORE_DENSE)
        return set_error(SYMPIX_EINVAL, "sympix_factor_blocks: unknown storage %d", storage);
    if (precision < SYMPIX_PREC_FP64 || precision > SYMPIX_PREC_FP32X2)
        return set_error(SYMPIX_EINVAL, "sympix_factor_blocks: unknown precision %d", precision);
    cudaStream_t st = (cudaStream_t)stream;
    const bool dense = storage == SYMPIX_STORE_DENSE;
    trace_mark(pl, st, nullptr);
    if (precision == SYMPIX_PREC_FP64) {
        launch_band<ArF64>(pl, dense, blocks, info, st);
        trace_mark(pl, st, "k_factor_band");
    }
    else if (precision == SYMPIX_PREC_FP32 && !dense) {
        const int ns = (int)pl->f32_slices.size();
        if (ns) {
            const F32Slice *sl = pl->d_f32_slices.p;
            k_f32_shadow_in<<<(unsigned)pl->f32_tiles.size(), 256, 0, st>>>(
                pl->d_f32_tiles.p, sl, pl->d_f32_items.p, pl->d_blocks.p, blocks, pl->d_shadow_il.p);
            trace_mark(pl, st, "k_f32_shadow_in");
            const int nf = pl->f32_slices_fused;  // slices with w <= kFusedWMax (they come first)
            if (nf > 0) {
                const size_t fs = (size_t)kFusedSmem * sizeof(float);
                cudaFuncSetAttribute(k_f32_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fs);
                k_f32_fused<<<(unsigned)nf, 32 + kFusedBorderThreads, fs, st>>>(
                    sl, pl->d_f32_items.p, pl->d_blocks.p, pl->d_shadow_il.p, pl->d_l21_il.p, blocks, info,
                    (float)pl->fp32_pivot_floor);
                trace_mark(pl, st, "k_f32_fused");
            }
            if (ns > nf) {
                const size_t smem = (size_t)kF32BandStage * sizeof(float);
                cudaFuncSetAttribute(k_f32_band_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                k_f32_band_pass<<<(unsigned)(ns - nf), 32, smem, st>>>(sl + nf, pl->d_f32_items.p, pl->d_blocks.p,
                                                                      pl->d_shadow_il.p, info,
                                                                      (float)pl->fp32_pivot_floor);
                trace_mark(pl, st, "k_f32_band_pass");
                const size_t bs = (size_t)kF32BorderStage * sizeof(float);
                auto kb = pl->border_threads == 256 ? k_f32_border_pass<256> : k_f32_border_pass<512>;
                cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bs);
                kb<<<(unsigned)(ns - nf), pl->border_threads, bs, st>>>(sl + nf, pl->d_f32_items.p, pl->d_blocks.p,
                                                                       pl->d_shadow_il.p, pl->d_l21_il.p, blocks,
                                                                       info);
                trace_mark(pl, st, "k_f32_border_pass");
            }
            k_f32_out<<<(unsigned)pl->f32_out_tiles.size(), 256, 0, st>>>(
                pl->d_f32_out_tiles.p, sl, pl->d_f32_items.p, pl->d_blocks.p, info, pl->d_shadow_il.p,
                pl->d_l21_il.p, blocks);
            trace_mark(pl, st, "k_f32_out");
            // near-degenerate blocks: FP64 from the untouched FP64 input
            launch_band<ArF64>(pl, false, blocks, info, st, 1);
            trace_mark(pl, st, "k_factor_rescue");
        }
    } else if (precision == SYMPIX_PREC_FP32) {
        launch_band<ArF32>(pl, dense, blocks, info, st);
        trace_mark(pl, st, "k_factor_band");
    } else {
        launch_band<ArF2>(pl, dense, blocks, info, st);
        trace_mark(pl, st, "k_factor_band");
    }
    const int nw = (int)pl->factor_items[5].size();
    if (nw) {
        const size_t smem = (size_t)((kWideMax + 1) * (kWideMax + 1) + kWideMax * (kWideMax + 1) +
                                     kWideMax * kWideMax + 3 * (kWideMax + 1)) *
                            sizeof(double);
        const int32_t *it = pl->d_factor_items[5].p;
        // FP32 arithmetic for the FP32 factor (near-degenerate blocks then
        // rescued in FP64), FP64 otherwise
        if (precision == SYMPIX_PREC_FP32 && !dense) {
            auto kf = k_factor_wide<float, false>;
            auto kd = dense ? k_factor_wide<double, true> : k_factor_wide<double, false>;
            cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaFuncSetAttribute(kd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            kf<<<nw, 256, smem, st>>>(nw, it, pl->d_blocks.p, blocks, info, 0, (float)pl->fp32_pivot_floor,
                                      pl->d_shadow.p);
            kd<<<nw, 256, smem, st>>>(nw, it, pl->d_blocks.p, blocks, info, 1, 0.0f, nullptr);
        } else {
            auto kd = dense ? k_factor_wide<double, true> : k_factor_wide<double, false>;
            cudaFuncSetAttribute(kd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            kd<<<nw, 256, smem, st>>>(nw, it, pl->d_blocks.p, blocks, info, 0, 0.0f, nullptr);
        }
    }
    if (nw) trace_mark(pl, st, "k_factor_wide");
    const int nd = (int)pl->factor_items[3].size(), ns = (int)pl->factor_items[4].size();
    if (nd)
        k_factor_dense<<<(unsigned)((nd * 32 + 127) / 128), 128, 0, st>>>(nd, pl->d_factor_items[3].p, pl->d_blocks.p,
                                                                        blocks, dense ? 1 : 0, info);
    if (nd) trace_mark(pl, st, "k_factor_dense");
    if (ns)
        k_factor_dense_cta<<<(unsigned)ns, 256, 0, st>>>(ns, pl->d_factor_items[4].p, pl->d_blocks.p, blocks,
                                                         dense ? 1 : 0, info);
    if (ns) trace_mark(pl, st, "k_factor_dense_cta");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "sympix_factor_blocks: launch");
    return SYMPIX_OK;
}
