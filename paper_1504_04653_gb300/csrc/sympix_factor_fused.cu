// FP32 factor: band and border passes of one slice fused in one CTA.
#include "sympix_factor_kernels.cuh"

namespace sympix {

// Band and border passes of one slice in one CTA, widths 1..WMAX: warp 0
// eliminates the band (f32_band) and publishes after every eighth period how
// many periods of L11 rows are final; NT threads run the border sweep
// (f32_border, FUSED) behind it, so the two latency-bound chains overlap
// instead of running one after the other.  The border's waits poll at most
// `wait_limit` times (a wait cannot run out unless the band warp stalls for a
// long time); one that runs out stops the sweep, sets the plan's device
// status and reports info = -1 for the slice's blocks.  The two roles meet on
// named barrier 2 (all threads) before the results are written.
//
// Two shapes: widths 1..8 with one border warp that keeps all W border rows
// and the corner sums in registers (each column's L11 row is loaded once
// and no pair goes through shared memory, which matters because every
// shared or global access costs an issue slot of the memory pipe, the
// resource both roles queue on), and widths 9..12 with ten border warps of
// one or two rows each, which the register budget of W rows per lane rules
// out there.
template <int WMAX, int NT>
struct FusedShape {
    static constexpr int kBandStage = 2 * (WMAX + 1) * (WMAX + 1) * 32;  // floats: two periods
    // floats: band stage, then three staged periods, two periods of L21
    // values and the last W columns of A21
    static constexpr int kSmem = kBandStage + 3 * (WMAX + 1) * (WMAX + 1) * 32 + 2 * WMAX * (WMAX + 1) * 32 +
                                 WMAX * WMAX * 32;
};

template <int WMAX, int NT>
__global__ void __launch_bounds__(32 + NT)
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
        bandres[L] = F32BandDispatch<WMAX>::run(sl.w, sh + sl.sh, L, m, sl.rows - sl.w, fsm, floor, prog);
        fused_barrier_all<NT>();  // the border sweep's end
    } else if (sl.w == 0) {
        fused_barrier_all<NT>();
    } else {
        const FusedWait fw{prog, bandres, &abort_s, status, wait_limit, nullptr};
        F32BorderDispatch<WMAX, 1, NT, kBorderFused>::run(sl.w, sl, sh + sl.sh, l21 + sl.l21, out, t.off, t.n, t.live,
                                                  fsm + FusedShape<WMAX, NT>::kBandStage, binfo, &fw);
    }
    __syncthreads();
    if (threadIdx.x < 32 && threadIdx.x < sl.count) {
        const int L = threadIdx.x;
        info[t.bi[L]] = (bandres[L] != 0 || sl.w == 0) ? bandres[L] : binfo[L];
    }
}

template <int WMAX, int NT>
static void launch_fused_shape(sympix_plan_t pl, int first, int count, double *blocks, int32_t *info,
                               cudaStream_t st) {
    if (count <= 0) return;
    const size_t fs = (size_t)FusedShape<WMAX, NT>::kSmem * sizeof(float);
    cudaFuncSetAttribute(k_f32_fused<WMAX, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fs);
    k_f32_fused<WMAX, NT><<<(unsigned)count, 32 + NT, fs, st>>>(
        pl->d_f32_slices.p + first, pl->d_f32_items.p, pl->d_blocks.p, pl->d_shadow_il.p, pl->d_l21_il.p, blocks,
        info, (float)pl->fp32_pivot_floor, pl->d_status.p, pl->wait_limit);
}

// Slices [0, f32_slices_w8) have w <= 8, [f32_slices_w8, nf) 9 <= w <= 12;
// the second group runs on a side stream beside the first.
void launch_f32_fused(sympix_plan_t pl, int nf, double *blocks, int32_t *info, cudaStream_t st) {
    const int n8 = pl->f32_slices_w8;
    const bool side = n8 > 0 && nf > n8 && pl->f32_side;
    if (side) {
        cudaEventRecord(pl->f32_fork, st);
        cudaStreamWaitEvent(pl->f32_side, pl->f32_fork, 0);
    }
    launch_fused_shape<8, 32>(pl, 0, n8, blocks, info, st);
    if (side) trace_mark(pl, st, "k_f32_fused_w8");
    launch_fused_shape<12, 320>(pl, n8, nf - n8, blocks, info, side ? pl->f32_side : st);
    if (side) {
        cudaEventRecord(pl->f32_join, pl->f32_side);
        cudaStreamWaitEvent(st, pl->f32_join, 0);
    }
    trace_mark(pl, st, "k_f32_fused");
}

}  // namespace sympix
