// FP32 factor of periodic-band blocks on the lane-interleaved shadow: the
// transposes in and out, the separate band and border passes (widths above
// the fused kernel's), and the launcher of the whole FP32 path.
#include "sympix_factor_kernels.cuh"

namespace sympix {

// One CTA per kTileE elements x 32 blocks of a slice; V = float (the FP32
// factor's shadow) or double (the FP64 one).
template <class V>
__global__ void __launch_bounds__(256) k_f32_shadow_in(const int2 *__restrict__ tiles,
                                                       const F32Slice *__restrict__ slices,
                                                       const int32_t *__restrict__ items,
                                                       const BlockDesc *__restrict__ blocks,
                                                       const double *__restrict__ out, V *__restrict__ sh) {
    constexpr int P16 = 16 / (int)sizeof(V);  // lanes per 16-byte shadow access
    __shared__ V tile[kTileE][33];
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
    // FP64 side: two consecutive elements of one block per thread (blocks
    // start on 32-byte boundaries and e0 is even, so the pair is aligned)
#pragma unroll
    for (int i = threadIdx.x; i < 16 * kTileE; i += 256) {
        const int L = i / (kTileE / 2), e = 2 * (i % (kTileE / 2));
        V v0 = V(0), v1 = V(0);
        const int cnt = s_cnt[L];
        if (e0 + e + 1 < cnt) {
            const double2 d = *reinterpret_cast<const double2 *>(out + s_off[L] + e0 + e);
            v0 = elem_from_f64<V>(d.x);
            v1 = elem_from_f64<V>(d.y);
        } else if (e0 + e < cnt) {
            v0 = elem_from_f64<V>(out[s_off[L] + e0 + e]);
        }
        tile[e][L] = v0;
        tile[e + 1][L] = v1;
    }
    __syncthreads();
    // shadow side: P16 consecutive blocks of one element per thread
    const int lim = sl.rows * RL;
    V *dst = sh + sl.sh + (int64_t)e0 * 32;
#pragma unroll
    for (int i = threadIdx.x; i < (32 / P16) * kTileE; i += 256) {
        const int e = i / (32 / P16), L = P16 * (i % (32 / P16));
        if (e0 + e < lim) store16(dst + e * 32 + L, &tile[e][L]);
    }
}

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

// Band pass on an FP64 (V = double) or split-FP32 (V = DF) shadow, widths
// up to 12: one CTA of four warps per slice, one lane per block; from w = 4
// the four warps share each block's window (band_lanes4), below it warp 0
// runs the one-warp loop alone.  info = i + 1 for the first row whose pivot
// is not positive (the border kernels then leave the block alone).
template <class V, int W>
__device__ __forceinline__ int exact_band_w(V *shs, int lane, int m, int mmax, unsigned char *smem) {
    if constexpr (W >= 4) {
        return band_lanes4_any<V, W>(shs, lane, m, mmax, smem);
    } else {
        if (threadIdx.x >= 32) return 0;
        return band_lanes_loop<V, W>(shs, lane, m, mmax, reinterpret_cast<V *>(smem));
    }
}

template <class V>
__global__ void __launch_bounds__(128) k_exact_band_pass(const F32Slice *__restrict__ slices,
                                                         const int32_t *__restrict__ items,
                                                         const BlockDesc *__restrict__ blocks, V *__restrict__ sh,
                                                         int32_t *__restrict__ info) {
    extern __shared__ __align__(16) unsigned char exact_smem[];
    const F32Slice sl = slices[blockIdx.x];
    const int lane = threadIdx.x & 31;
    int m = 0, bi = -1;
    if (lane < sl.count) {
        bi = items[sl.first + lane];
        m = blocks[bi].n - sl.w;
    }
    V *shs = sh + sl.sh;
    const int mmax = sl.rows - sl.w;
    int r = 0;
    StaticFor<0, 13>::run([&](auto Wc) {
        constexpr int W = decltype(Wc)::value;
        if (sl.w == W) r = exact_band_w<V, W>(shs, lane, m, mmax, exact_smem);
    });
    if (bi >= 0 && threadIdx.x < 32) info[bi] = r;
}

// The factor back to the FP64 blocks: L11 rows from the band shadow and
// L21 rows from the border buffer, 64 elements x 32 blocks per CTA, through
// a shared-memory transpose (coalesced on both sides).  Blocks sent to the
// FP64 rescue are skipped.  V: the shadow's element (float or double).
template <class V>
__global__ void __launch_bounds__(256) k_f32_out(const int2 *__restrict__ tiles, const F32Slice *__restrict__ slices,
                                                 const int32_t *__restrict__ items,
                                                 const BlockDesc *__restrict__ blocks,
                                                 const int32_t *__restrict__ info, const V *__restrict__ sh,
                                                 const V *__restrict__ l21, double *__restrict__ out) {
    constexpr int P16 = 16 / (int)sizeof(V);  // lanes per 16-byte shadow access
    __shared__ V tile[kTileE][33];
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
    const V *src = (part21 ? l21 + sl.l21 : sh + sl.sh) + (int64_t)e0 * 32;
    // shadow side: P16 consecutive blocks of one element per thread
#pragma unroll
    for (int i = threadIdx.x; i < (32 / P16) * kTileE; i += 256) {
        const int e = i / (32 / P16), L = P16 * (i % (32 / P16));
        V v[P16];
#pragma unroll
        for (int u = 0; u < P16; ++u) v[u] = V(0);
        if (e0 + e < lim) load16(src + e * 32 + L, v);
#pragma unroll
        for (int u = 0; u < P16; ++u) tile[e][L + u] = v[u];
    }
    __syncthreads();
    // FP64 side: two consecutive elements of one block per thread; their
    // (row, offset) or (border row, column) are formed once for all blocks.
    // A pair that is contiguous and 16-byte aligned in the block (always in
    // the band part: blocks start on 32-byte boundaries, e0 is even) goes as
    // one 16-byte store.
    const int e = 2 * (threadIdx.x % (kTileE / 2)), ee = e0 + e;
    if (ee >= lim) return;
    const bool has2 = ee + 1 < lim;
    const int q0 = part21 ? ee / kc : ee / RL;           // border row b, or band row
    const int r0 = part21 ? ee - q0 * kc : ee - q0 * RL;  // column k, or offset d
    const int q1 = part21 ? (ee + 1) / kc : (ee + 1) / RL;
    const int r1 = part21 ? ee + 1 - q1 * kc : ee + 1 - q1 * RL;
#pragma unroll
    for (int L = threadIdx.x / (kTileE / 2); L < 32; L += 256 / (kTileE / 2)) {
        const int n = s_n[L], m = n - W;
        const bool ok0 = s_live[L] && (part21 ? r0 < m : (q0 < m && r0 <= q0));
        const bool ok1 = has2 && s_live[L] && (part21 ? r1 < m : (q1 < m && r1 <= q1));
        const int64_t d0 = part21 ? s_off[L] + (int64_t)n * RL + (int64_t)q0 * n + r0 : s_off[L] + ee;
        const int64_t d1 = part21 ? s_off[L] + (int64_t)n * RL + (int64_t)q1 * n + r1 : s_off[L] + ee + 1;
        if (ok0 && ok1 && d1 == d0 + 1 && (d0 & 1) == 0) {
            *reinterpret_cast<double2 *>(out + d0) = make_double2(elem_to_f64(tile[e][L]), elem_to_f64(tile[e + 1][L]));
        } else {
            if (ok0) out[d0] = elem_to_f64(tile[e][L]);
            if (ok1) out[d1] = elem_to_f64(tile[e + 1][L]);
        }
    }
}

void launch_f32_slices(sympix_plan_t pl, double *blocks, int32_t *info, cudaStream_t st, bool hi_only) {
    const int ns = (int)pl->f32_slices.size();
    const int nf = pl->f32_slices_fused;  // slices with w <= 12 (they come first)
    if (hi_only ? ns == nf : ns == 0) return;
    const F32Slice *sl = pl->d_f32_slices.p;
    const size_t nin = hi_only ? pl->f32_tiles_hi.size() : pl->f32_tiles.size();
    const size_t nout = hi_only ? pl->f32_out_tiles_hi.size() : pl->f32_out_tiles.size();
    const int2 *tin = hi_only ? pl->d_f32_tiles_hi.p : pl->d_f32_tiles.p;
    const int2 *tout = hi_only ? pl->d_f32_out_tiles_hi.p : pl->d_f32_out_tiles.p;
    k_f32_shadow_in<float><<<(unsigned)nin, 256, 0, st>>>(tin, sl, pl->d_f32_items.p, pl->d_blocks.p, blocks,
                                                   pl->d_shadow_il.p);
    trace_mark(pl, st, "k_f32_shadow_in");
    if (nf > 0 && !hi_only) {
        if (pl->narrow_pref[SYMPIX_PREC_FP32] == 2) {  // band pass, then the border rows by column chunks
            const size_t smem = (size_t)kF32BandStage * sizeof(float);
            cudaFuncSetAttribute(k_f32_band_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_f32_band_pass<<<(unsigned)nf, 32, smem, st>>>(sl, pl->d_f32_items.p, pl->d_blocks.p, pl->d_shadow_il.p,
                                                           info, (float)pl->fp32_pivot_floor);
            trace_mark(pl, st, "k_f32_band_pass");
            launch_f32_l21(pl, blocks, info, st);
        } else if (pl->narrow_pref[SYMPIX_PREC_FP32] == 3 && f32_split_fits(pl)) {
            // w <= 8: band and border passes in separate CTAs of one launch;
            // 9 <= w <= 12 (a few slices): band pass, then the chunked border
            // kernels, on the side stream at the same time (a second
            // cooperative launch would wait for the first to finish)
            const int n8 = pl->f32_slices_w8;
            const bool side = n8 > 0 && nf > n8 && pl->f32_side;
            cudaStream_t sh = side ? pl->f32_side : st;
            if (side) {
                cudaEventRecord(pl->f32_fork, st);
                cudaStreamWaitEvent(sh, pl->f32_fork, 0);
            }
            if (nf > n8) {
                const size_t smem = (size_t)kF32BandStage * sizeof(float);
                cudaFuncSetAttribute(k_f32_band_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                k_f32_band_pass<<<(unsigned)(nf - n8), 32, smem, sh>>>(sl + n8, pl->d_f32_items.p, pl->d_blocks.p,
                                                                      pl->d_shadow_il.p, info,
                                                                      (float)pl->fp32_pivot_floor);
                launch_f32_l21(pl, blocks, info, sh, true);
            }
            launch_f32_split_w8(pl, blocks, info, st);
            if (side) trace_mark(pl, st, "k_f32_split_w8");
            if (side) {
                cudaEventRecord(pl->f32_join, sh);
                cudaStreamWaitEvent(st, pl->f32_join, 0);
            }
            trace_mark(pl, st, "k_f32_split");
        } else {
            launch_f32_fused(pl, nf, blocks, info, st);
        }
    }
    if (ns > nf) {
        const size_t smem = (size_t)kF32BandStage * sizeof(float);
        cudaFuncSetAttribute(k_f32_band_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_f32_band_pass<<<(unsigned)(ns - nf), 32, smem, st>>>(sl + nf, pl->d_f32_items.p, pl->d_blocks.p,
                                                              pl->d_shadow_il.p, info, (float)pl->fp32_pivot_floor);
        trace_mark(pl, st, "k_f32_band_pass");
        if (pl->border_threads == 256)
            launch_f32_border<256>(pl, nf, ns - nf, blocks, info, st);
        else
            launch_f32_border<512>(pl, nf, ns - nf, blocks, info, st);
        trace_mark(pl, st, "k_f32_border_pass");
    }
    k_f32_out<float><<<(unsigned)nout, 256, 0, st>>>(tout, sl, pl->d_f32_items.p, pl->d_blocks.p, info, pl->d_shadow_il.p,
                                             pl->d_l21_il.p, blocks);
    trace_mark(pl, st, "k_f32_out");
    // near-degenerate blocks: FP64 from the untouched FP64 input
    launch_band<ArF64>(pl, false, blocks, info, st, 1, hi_only);
    trace_mark(pl, st, "k_factor_rescue");
}

// The FP64 (V = double) or split-FP32 (V = DF) factor of the periodic bands
// up to w = 16 on a shadow of that element: for w <= 12 the transposes
// around the one-lane-per-block band pass and the chunked border solve (every
// instruction does 32 blocks' work), for 12 < w <= 16 the lane-group kernel.
// The shadow and the chunk scratch are the FP32 path's buffers, which the
// plan sizes for 8-byte elements.
template <class V>
static void launch_exact_slices(sympix_plan_t pl, double *blocks, int32_t *info, cudaStream_t st) {
    const int nf = pl->f32_slices_fused;
    const size_t nin = pl->f32_tiles_lo.size(), nout = pl->f32_out_tiles_lo.size();
    if (nf > 0 && nin > 0) {
        const F32Slice *sl = pl->d_f32_slices.p;
        V *sh = reinterpret_cast<V *>(pl->d_shadow_il.p), *l21 = reinterpret_cast<V *>(pl->d_l21_il.p);
        k_f32_shadow_in<V><<<(unsigned)nin, 256, 0, st>>>(pl->d_f32_tiles_lo.p, sl, pl->d_f32_items.p, pl->d_blocks.p,
                                                          blocks, sh);
        trace_mark(pl, st, "k_f32_shadow_in");
        const size_t smem = band4_smem<V, 12>();  // >= the one-warp loop's two periods of w = 3
        cudaFuncSetAttribute(k_exact_band_pass<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_exact_band_pass<V><<<(unsigned)nf, 128, smem, st>>>(sl, pl->d_f32_items.p, pl->d_blocks.p, sh, info);
        trace_mark(pl, st, std::is_same<V, double>::value ? "k_f64_band_pass" : "k_df_band_pass");
        if constexpr (std::is_same<V, double>::value)
            launch_f64_l21(pl, blocks, info, st);
        else
            launch_df_l21(pl, blocks, info, st);
        k_f32_out<V><<<(unsigned)nout, 256, 0, st>>>(pl->d_f32_out_tiles_lo.p, sl, pl->d_f32_items.p, pl->d_blocks.p,
                                                     info, sh, l21, blocks);
        trace_mark(pl, st, "k_f32_out");
    }
    if constexpr (std::is_same<V, double>::value)
        launch_band<ArF64>(pl, false, blocks, info, st, 0, true);  // 12 < w <= 16
    else
        launch_band<ArF2>(pl, false, blocks, info, st, 0, true);
    trace_mark(pl, st, "k_factor_band");
}

void launch_f64_slices(sympix_plan_t pl, double *blocks, int32_t *info, cudaStream_t st) {
    launch_exact_slices<double>(pl, blocks, info, st);
}
void launch_df_slices(sympix_plan_t pl, double *blocks, int32_t *info, cudaStream_t st) {
    launch_exact_slices<DF>(pl, blocks, info, st);
}

}  // namespace sympix
