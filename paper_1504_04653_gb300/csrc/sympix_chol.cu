// Launcher of the narrow-band factor (sympix_chol.cuh) and its FP32 commit.
#include "sympix_chol.cuh"

namespace sympix {

__global__ void __launch_bounds__(256) k_chol_commit(const int2 *__restrict__ tiles, const BlockDesc *__restrict__ blocks,
                                                     const int32_t *__restrict__ info, const float *__restrict__ l11f,
                                                     double *__restrict__ out) {
    const int2 tl = tiles[blockIdx.x];
    const BlockDesc bd = blocks[tl.x];
    if (info[tl.x] == kRescue) return;  // refactored in FP64 from its input
    const int RL = bd.w + 1;
    const int64_t lim = (int64_t)(bd.n - bd.w) * RL;  // band rows < m
    const int64_t e1 = lim < (int64_t)tl.y + kCommitTile ? lim : (int64_t)tl.y + kCommitTile;
    for (int64_t e = tl.y + threadIdx.x; e < e1; e += 256) {
        const int row = (int)(e / RL), d = (int)(e - (int64_t)row * RL);
        if (d <= row) out[bd.off_pband + e] = f32_to_f64_bits(l11f[bd.off_pband + e]);
    }
}


// the widths present run on their own streams (and the lane groups on a side
// stream): fork from `st`, join back
static void chol_fork(sympix_plan_t pl, cudaStream_t st) {
    cudaEventRecord(pl->chol_fork, st);
    for (int w = 0; w <= kNarrowWMax; ++w)
        if (pl->chol_st[w]) cudaStreamWaitEvent(pl->chol_st[w], pl->chol_fork, 0);
    if (pl->chol_side) cudaStreamWaitEvent(pl->chol_side, pl->chol_fork, 0);
}
static void chol_join(sympix_plan_t pl, cudaStream_t st) {
    for (int w = 0; w <= kNarrowWMax; ++w)
        if (pl->chol_st[w]) {
            cudaEventRecord(pl->chol_join[w], pl->chol_st[w]);
            cudaStreamWaitEvent(st, pl->chol_join[w], 0);
        }
    if (pl->chol_side) {
        cudaEventRecord(pl->chol_side_join, pl->chol_side);
        cudaStreamWaitEvent(st, pl->chol_side_join, 0);
    }
}

void launch_pband_chol(sympix_plan_t pl, int precision, double *blocks, int32_t *info, cudaStream_t st) {
    if (pl->chol_items.empty() && pl->factor_items[2].empty()) return;
    chol_fork(pl, st);
    if (precision == SYMPIX_PREC_FP32) {
        launch_chol_f32(pl, blocks, info, 0, kCholWMax);
    } else if (precision == SYMPIX_PREC_FP64) {
        launch_chol_f64(pl, blocks, info, 0, kCholGroupFrom - 1);
        if (pl->chol_side) launch_band_groups<ArF64>(pl, blocks, info, pl->chol_side);
    } else {
        launch_chol_f2(pl, blocks, info, 0, kCholGroupFrom - 1);
        if (pl->chol_side) launch_band_groups<ArF2>(pl, blocks, info, pl->chol_side);
    }
    chol_join(pl, st);
    trace_mark(pl, st, "k_pband_chol");
    if (precision == SYMPIX_PREC_FP32 && !pl->chol_items.empty()) {
        k_chol_commit<<<(unsigned)pl->chol_tiles.size(), 256, 0, st>>>(pl->d_chol_tiles.p, pl->d_blocks.p, info,
                                                                      pl->d_shadow.p, blocks);
        trace_mark(pl, st, "k_chol_commit");
        // blocks whose FP32 pivots fell below the floor: FP64 from their input
        chol_fork(pl, st);
        launch_chol_f64(pl, blocks, info, 1, kCholWMax);
        chol_join(pl, st);
        trace_mark(pl, st, "k_pband_chol_rescue");
    }
}

}  // namespace sympix
