// FP32 factor: band and border passes of one slice fused in one CTA.
#include "sympix_factor_kernels.cuh"

namespace sympix {

// Band and border passes of one slice in one CTA, widths 1..kFusedWMax:
// warp 0 eliminates the band (f32_band) and publishes after every fourth
// period how many periods of L11 rows are final; kFusedBorderThreads threads
// run the border sweep (f32_border, FUSED) behind it, so the two
// latency-bound chains overlap instead of running one after the other.  The
// border's waits poll at most `wait_limit` times (a wait cannot run out
// unless the band warp stalls for a long time); one that runs out stops the
// sweep, sets the plan's device status and reports info = -1 for the
// slice's blocks.  The two roles meet on named barrier 2 (all threads)
// before the results are written.
constexpr int kFusedWMax = 12, kFusedBorderThreads = 320;
constexpr int kFusedBandStage = 2 * 13 * 13 * 32;  // floats: two periods of W = 12
// floats: band stage, then three staged periods, two periods of L21 values
// and the last W columns of A21, W = 12
constexpr int kFusedSmem = kFusedBandStage + 3 * 13 * 13 * 32 + 2 * 12 * 13 * 32 + 12 * 12 * 32;

__global__ void __launch_bounds__(32 + kFusedBorderThreads)
    k_f32_fused(const F32Slice *__restrict__ slices, const int32_t *__restrict__ items,
                const BlockDesc *__restrict__ blocks, float *__restrict__ sh, float *__restrict__ l21,
                const double *__restrict__ out, int32_t *__restrict__ info, float floor, int32_t *status,
                int wait_limit) {
    extern __shared__ __align__(16) float fsm[];
    __shared__ SliceBlocks t;
    __shared__ int binfo[32], bandres[32];
    __shared__ int prog_s, abort_s;
    volatile int *prog = &prog_s;
    const F32Slice sl = slices[blockIdx.x];
    load_slice_blocks(t, sl, items, blocks, nullptr);
    if (threadIdx.x == 0) {
        *prog = 0;
        abort_s = 0;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const int L = threadIdx.x;
        const int m = L < sl.count ? t.n[L] - sl.w : 0;
        bandres[L] = F32BandDispatch<kFusedWMax>::run(sl.w, sh + sl.sh, L, m, sl.rows - sl.w, fsm, floor, prog);
        fused_barrier_all<kFusedBorderThreads>();  // the border sweep's end
    } else if (sl.w == 0) {
        fused_barrier_all<kFusedBorderThreads>();
    } else {
        const FusedWait fw{prog, bandres, &abort_s, status, wait_limit};
        F32BorderDispatch<kFusedWMax, 1, kFusedBorderThreads, true>::run(
            sl.w, sl, sh + sl.sh, l21 + sl.l21, out, t.off, t.n, t.live, fsm + kFusedBandStage, binfo, &fw);
    }
    __syncthreads();
    if (threadIdx.x < 32 && threadIdx.x < sl.count) {
        const int L = threadIdx.x;
        info[t.bi[L]] = (bandres[L] != 0 || sl.w == 0) ? bandres[L] : binfo[L];
    }
}

void launch_f32_fused(sympix_plan_t pl, int nf, double *blocks, int32_t *info, cudaStream_t st) {
    const size_t fs = (size_t)kFusedSmem * sizeof(float);
    cudaFuncSetAttribute(k_f32_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fs);
    k_f32_fused<<<(unsigned)nf, 32 + kFusedBorderThreads, fs, st>>>(pl->d_f32_slices.p, pl->d_f32_items.p,
                                                                   pl->d_blocks.p, pl->d_shadow_il.p, pl->d_l21_il.p,
                                                                   blocks, info, (float)pl->fp32_pivot_floor,
                                                                   pl->d_status.p, pl->wait_limit);
    trace_mark(pl, st, "k_f32_fused");
}

}  // namespace sympix
