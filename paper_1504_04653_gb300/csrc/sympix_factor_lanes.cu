// Periodic-band Cholesky in FP64, split FP32 and FP32 (dense storage):
// two-pass band/border kernels for narrow bands and 32-lane groups for
// 8 < w <= 16, and their launcher.
#include "sympix_factor_kernels.cuh"

namespace sympix {

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

// FP32 runs both passes for every band width up to 16; FP64 and split FP32
// (twice the registers) run them for w <= 8 and factor wider bands with
// lane groups.
template <class A>
void launch_band(sympix_plan_t pl, bool dense, double *blocks, int32_t *info, cudaStream_t st, int rescue,
                 bool skip_narrow) {
    constexpr bool wide = std::is_same<A, ArF32>::value;
    const int n0 = skip_narrow ? 0 : (int)pl->factor_items[0].size();
    const int n1 = skip_narrow ? 0 : (int)pl->factor_items[1].size(), n2 = (int)pl->factor_items[2].size();
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
        for (int l = skip_narrow ? 2 : 1; l <= 2; ++l) {
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

template <class A>
void launch_band_groups(sympix_plan_t pl, double *blocks, int32_t *info, cudaStream_t st) {
    for (int l = 1; l <= 2; ++l) {
        const int nl = (int)pl->factor_items[l].size();
        if (!nl) continue;
        k_factor_band<A, 32, false><<<(unsigned)((nl * 32 + 127) / 128), 128, 0, st>>>(
            nl, pl->d_factor_items[l].p, pl->d_blocks.p, blocks, info, 0);
    }
}
template void launch_band_groups<ArF64>(sympix_plan_t, double *, int32_t *, cudaStream_t);
template void launch_band_groups<ArF2>(sympix_plan_t, double *, int32_t *, cudaStream_t);

template void launch_band<ArF64>(sympix_plan_t, bool, double *, int32_t *, cudaStream_t, int, bool);
template void launch_band<ArF32>(sympix_plan_t, bool, double *, int32_t *, cudaStream_t, int, bool);
template void launch_band<ArF2>(sympix_plan_t, bool, double *, int32_t *, cudaStream_t, int, bool);

}  // namespace sympix
