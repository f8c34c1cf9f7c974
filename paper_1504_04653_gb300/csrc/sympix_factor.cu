// Cholesky factorisation M = L L^T of every sampled block.
//
// A periodic-band block (half-width w, 2w+1 < n) couples only |i-j| <= w or
// |i-j| >= n-w.  With m = n - w its leading m x m part A11 is a plain band
// matrix, so L11 keeps the band; the last w rows (the border) fill in
// completely.  Right-looking elimination of column k touches only rows
// k+1..k+w of the band and the w border rows, so one lane group carries
// the whole active part in registers:
//   * window lanes r = 0..w-1 hold rows k+1+r of A11 at columns k..k+1+r;
//   * border lanes r = 0..w-1 hold border row m+r at columns k..k+w;
//   * the pivot is row k's updated diagonal, broadcast to the group.
// Each step forms 1/sqrt(pivot), scales column k (L[k+1+r][k] and
// L[m+r][k]), applies the rank-1 update to the band columns k+1..k+w and
// shifts the window by one row, loading one new row of the band.  The
// border lanes thus do the forward substitution L21 = A21 L11^-T in the
// same instructions.  Afterwards the group forms the corner
// S = A22 - L21 L21^T with lanes over the column index and factors it.
// Work O(n w^2) per block instead of O(n^3).
//
// Arithmetic: FP64, split FP32 (near-FP64 on the FP32 pipes) or FP32.
// Dense-format blocks (small or fully coupled rings) use a warp-parallel
// right-looking dense factorisation in FP64; blocks wider than the lane
// groups allow fall back to one thread per block.
//
// A non-positive pivot stops the block and records info = row + 1.
#include <type_traits>

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
                                                     int32_t *__restrict__ info) {
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

// One lane per periodic-band block with w <= WB, 32 blocks per warp (the
// blocks of a warp are adjacent in the plan's cost order, so the lanes run
// in step).  Everything the elimination of column k touches stays in the
// lane's registers:
//   W[r][c]  band rows k..k+w at columns k..k+r (r = 0 is the pivot row);
//   B[b][c]  border rows m+b at columns k..k+w;
//   S[b][c]  the corner A22 - L21 L21^T, accumulated as the border rows'
//            column-k entries of L are produced.
// Per column: 1/sqrt of the pivot, scale the column, rank-1 update of the
// band and border windows and of S, shift both windows by one column; the
// band row entering the window is loaded two columns ahead.  After the last
// column the w x w corner S is factored in registers.
template <class A, int WB, bool DENSE>
__global__ void __launch_bounds__(32) k_factor_lane(int nitems, const int32_t *__restrict__ items,
                                                    const BlockDesc *__restrict__ blocks, double *__restrict__ out,
                                                    int32_t *__restrict__ info) {
    typedef typename A::V V;
    const int idx = blockIdx.x * 32 + threadIdx.x;
    if (idx >= nitems) return;
    const int bi = items[idx];
    const BlockDesc bd = blocks[bi];
    const typename ViewOf<DENSE>::T v = ViewOf<DENSE>::make(out, bd);
    const int w = bd.w, m = bd.n - bd.w;

    V W[WB + 1][WB + 1];
    V B[WB][WB + 1];
    V S[WB][WB];
#pragma unroll
    for (int r = 0; r <= WB; ++r)
#pragma unroll
        for (int c = 0; c <= WB; ++c) W[r][c] = (r <= w && c <= r && r < m) ? A::from(v.a(r, c)) : A::zero();
#pragma unroll
    for (int b = 0; b < WB; ++b) {
#pragma unroll
        for (int c = 0; c <= WB; ++c) B[b][c] = (b < w && c <= w) ? A::from(v.a(m + b, c)) : A::zero();
#pragma unroll
        for (int c = 0; c < WB; ++c) S[b][c] = (b < w && c <= b) ? A::from(v.a(m + b, m + c)) : A::zero();
    }
    // rows entering the window one and two columns ahead
    double nx1[WB + 1], nx2[WB + 1];
#pragma unroll
    for (int c = 0; c <= WB; ++c) {
        const int r1 = 1 + w, r2 = 2 + w;
        nx1[c] = (c <= w && r1 < m) ? *v.row_elem(r1, c) : 0.0;
        nx2[c] = (c <= w && r2 < m) ? *v.row_elem(r2, c) : 0.0;
    }
    int inf = 0;
    for (int k = 0; k < m; ++k) {
        const V d = W[0][0];
        if (!A::positive(d)) {
            inf = k + 1;
            break;
        }
        const V rs = A::rsqrt_(d);
        v.put_l(k, k, A::to_double(A::mul(d, rs)));
        V l[WB + 1], lb[WB];
#pragma unroll
        for (int r = 1; r <= WB; ++r) {
            l[r] = (r <= w && k + r < m) ? A::mul(W[r][0], rs) : A::zero();
            if (r <= w && k + r < m) v.put_l(k + r, k, A::to_double(l[r]));
        }
#pragma unroll
        for (int b = 0; b < WB; ++b) {
            lb[b] = b < w ? A::mul(B[b][0], rs) : A::zero();
            if (b < w) v.put_b(b, k, A::to_double(lb[b]));
        }
        // rank-1 updates
#pragma unroll
        for (int r = 1; r <= WB; ++r)
#pragma unroll
            for (int c = 1; c <= r; ++c) W[r][c] = A::fnma(l[r], l[c], W[r][c]);
#pragma unroll
        for (int b = 0; b < WB; ++b) {
#pragma unroll
            for (int c = 1; c <= WB; ++c) B[b][c] = A::fnma(lb[b], l[c], B[b][c]);
#pragma unroll
            for (int c = 0; c <= b; ++c) S[b][c] = A::fnma(lb[b], lb[c], S[b][c]);
        }
        // shift: column k+1 becomes column 0; row k+1+w enters the band
        // window, column k+1+w enters the border windows
        const int nc = k + 1 + w;
#pragma unroll
        for (int r = 0; r < WB; ++r)
#pragma unroll
            for (int c = 0; c <= r; ++c) W[r][c] = W[r + 1][c + 1];
#pragma unroll
        for (int c = 0; c <= WB; ++c) W[WB][c] = A::zero();
#pragma unroll
        for (int c = 0; c <= WB; ++c)
            if (c <= w) {
#pragma unroll
                for (int r = 0; r <= WB; ++r)
                    if (r == w) W[r][c] = A::from(nx1[c]);
            }
#pragma unroll
        for (int b = 0; b < WB; ++b) {
#pragma unroll
            for (int c = 0; c < WB; ++c) B[b][c] = B[b][c + 1];
            B[b][WB] = A::zero();
            if (b < w) {
                const V x = nc < m ? A::from(v.a(m + b, nc)) : A::zero();
#pragma unroll
                for (int c = 0; c <= WB; ++c)
                    if (c == w) B[b][c] = x;
            }
        }
        // prefetch the row entering two columns from now
        const int r3 = k + 3 + w;
#pragma unroll
        for (int c = 0; c <= WB; ++c) {
            nx1[c] = nx2[c];
            nx2[c] = (c <= w && r3 < m) ? *v.row_elem(r3, c) : 0.0;
        }
    }
    if (inf == 0) {
        // the w x w corner: S = L22 L22^T, in registers
#pragma unroll
        for (int j = 0; j < WB; ++j) {
            if (j < w && inf == 0) {
                const V dj = S[j][j];
                if (!A::positive(dj)) {
                    inf = m + j + 1;
                } else {
                    const V rs = A::rsqrt_(dj);
                    S[j][j] = A::mul(dj, rs);
#pragma unroll
                    for (int i = j + 1; i < WB; ++i) S[i][j] = A::mul(S[i][j], rs);
#pragma unroll
                    for (int i = j + 1; i < WB; ++i)
#pragma unroll
                        for (int c = j + 1; c <= i; ++c) S[i][c] = A::fnma(S[i][j], S[c][j], S[i][c]);
                }
            }
        }
        if (inf == 0) {
#pragma unroll
            for (int b = 0; b < WB; ++b)
#pragma unroll
                for (int c = 0; c <= b; ++c)
                    if (b < w) v.put_b(b, m + c, A::to_double(S[b][c]));
        }
    }
    info[bi] = inf;
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

// Fallback: one thread per block, FP64 (wide bands beyond the lane groups).
template <class View>
__device__ int factor_band_border_serial(const View &v) {
    const int n = v.n, w = v.w, m = v.m;
    for (int i = 0; i < m; ++i) {
        const int j0 = max(0, i - w);
        for (int j = j0; j <= i; ++j) {
            double s = v.a(i, j);
            for (int k = max(j0, j - w); k < j; ++k) s -= v.get_l(i, k) * v.get_l(j, k);
            if (j < i) {
                v.put_l(i, j, s / v.get_l(j, j));
            } else {
                if (!(s > 0.0)) return i + 1;
                v.put_l(i, i, sqrt(s));
            }
        }
    }
    for (int b = 0; b < w; ++b) {
        const int i = m + b;
        for (int j = 0; j < m; ++j) {
            double s = v.a(i, j);
            for (int k = max(0, j - w); k < j; ++k) s -= v.get_b(b, k) * v.get_l(j, k);
            v.put_b(b, j, s / v.get_l(j, j));
        }
    }
    for (int b = 0; b < w; ++b) {
        const int i = m + b;
        for (int bp = 0; bp <= b; ++bp) {
            const int j = m + bp;
            double s = v.a(i, j);
            for (int k = 0; k < j; ++k) s -= v.get_b(b, k) * v.get_b(bp, k);
            if (bp < b) {
                v.put_b(b, j, s / v.get_b(bp, j));
            } else {
                if (!(s > 0.0)) return i + 1;
                v.put_b(b, j, sqrt(s));
            }
        }
    }
    return 0;
}

__global__ void k_factor_serial(int nitems, const int32_t *__restrict__ items, const BlockDesc *__restrict__ blocks,
                                double *__restrict__ out, int dense_storage, int32_t *__restrict__ info) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nitems) return;
    const int bi = items[t];
    const BlockDesc bd = blocks[bi];
    int res;
    if (dense_storage) {
        DenseView v{out + bd.off_dense, bd.n, bd.w, bd.n - bd.w};
        res = factor_band_border_serial(v);
    } else {
        double *base = out + bd.off_pband;
        PBandView v{base, base + (int64_t)bd.n * (bd.w + 1), bd.n, bd.w, bd.n - bd.w};
        res = factor_band_border_serial(v);
    }
    info[bi] = res;
}

}  // namespace sympix

using namespace sympix;

// FP32 keeps the whole elimination state of a block in one lane's registers;
// FP64 and split FP32 need twice the registers and use lane groups.
template <class A>
static void launch_band(sympix_plan_t pl, bool dense, double *blocks, int32_t *info, cudaStream_t st) {
    constexpr bool lane_kernel = std::is_same<A, ArF32>::value;
    const int n16 = (int)pl->factor_items[0].size(), n32 = (int)pl->factor_items[1].size();
    if constexpr (lane_kernel) {
        if (n16) {
            const unsigned grid = (unsigned)((n16 + 31) / 32);
            if (dense)
                k_factor_lane<A, 8, true><<<grid, 32, 0, st>>>(n16, pl->d_factor_items[0].p, pl->d_blocks.p, blocks,
                                                               info);
            else
                k_factor_lane<A, 8, false><<<grid, 32, 0, st>>>(n16, pl->d_factor_items[0].p, pl->d_blocks.p, blocks,
                                                                info);
        }
    } else if (n16) {
        const unsigned grid = (unsigned)((n16 * 16 + 127) / 128);
        if (dense)
            k_factor_band<A, 16, true><<<grid, 128, 0, st>>>(n16, pl->d_factor_items[0].p, pl->d_blocks.p, blocks, info);
        else
            k_factor_band<A, 16, false><<<grid, 128, 0, st>>>(n16, pl->d_factor_items[0].p, pl->d_blocks.p, blocks, info);
    }
    if (n32) {
        const unsigned grid = (unsigned)((n32 * 32 + 127) / 128);
        if (dense)
            k_factor_band<A, 32, true><<<grid, 128, 0, st>>>(n32, pl->d_factor_items[1].p, pl->d_blocks.p, blocks, info);
        else
            k_factor_band<A, 32, false><<<grid, 128, 0, st>>>(n32, pl->d_factor_items[1].p, pl->d_blocks.p, blocks, info);
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
    if (precision == SYMPIX_PREC_FP64)
        launch_band<ArF64>(pl, dense, blocks, info, st);
    else if (precision == SYMPIX_PREC_FP32)
        launch_band<ArF32>(pl, dense, blocks, info, st);
    else
        launch_band<ArF2>(pl, dense, blocks, info, st);
    const int nd = (int)pl->factor_items[2].size(), ns = (int)pl->factor_items[3].size();
    if (nd)
        k_factor_dense<<<(unsigned)((nd * 32 + 127) / 128), 128, 0, st>>>(nd, pl->d_factor_items[2].p, pl->d_blocks.p,
                                                                        blocks, dense ? 1 : 0, info);
    if (ns)
        k_factor_serial<<<(unsigned)((ns + 31) / 32), 32, 0, st>>>(ns, pl->d_factor_items[3].p, pl->d_blocks.p, blocks,
                                                                  dense ? 1 : 0, info);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "sympix_factor_blocks: launch");
    return SYMPIX_OK;
}
