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
//   16 < w <= 64: one CTA per block, the window and border rows in
//       registers (24 entries of one column slot per thread), one barrier
//       per column; the corner from the stored L21 at the end.
//   dense-format blocks with n <= 1024: a warp per block, right-looking,
//   FP64; larger ones: a CTA per block, blocked right-looking, FP64.
//
// FP32 rescue: an FP32 elimination whose pivot falls below a floor times the
// original diagonal marks its block, and the block is refactored in FP64
// from the untouched FP64 input.  A non-positive pivot in FP64 stops the
// block and records info = row + 1.
//
// Files: sympix_factor_kernels.cuh (views, staging, the templated FP32
// passes), sympix_factor_lanes.cu (FP64 / split FP32 band and border
// kernels), sympix_factor_f32.cu and sympix_factor_fused.cu (the FP32
// path), sympix_factor_wide.cu (wide bands, dense blocks), this file (the
// entry point).
#include "sympix_chol.cuh"
#include "sympix_factor_kernels.cuh"

using namespace sympix;

extern "C" int sympix_factor_blocks(sympix_plan_t pl, int storage, int precision, double *blocks, int32_t *info,
                                    void *stream) {
    if (!pl || !blocks || !info) return set_error(SYMPIX_EINVAL, "sympix_factor_blocks: NULL argument");
    if ((reinterpret_cast<uintptr_t>(blocks) & 15) != 0)
        return set_error(SYMPIX_EINVAL, "sympix_factor_blocks: blocks must be 16-byte aligned");
    if (storage != SYMPIX_STORE_PBAND && storage != SYMPIX_STORE_DENSE)
        return set_error(SYMPIX_EINVAL, "sympix_factor_blocks: unknown storage %d", storage);
    if (precision < SYMPIX_PREC_FP64 || precision > SYMPIX_PREC_FP32X2)
        return set_error(SYMPIX_EINVAL, "sympix_factor_blocks: unknown precision %d", precision);
    cudaStream_t st = (cudaStream_t)stream;
    const bool dense = storage == SYMPIX_STORE_DENSE;
    trace_mark(pl, st, nullptr);
    // periodic-band storage: bands up to w = 12 go to the narrow-band kernel
    // or (every arithmetic) to the one-lane-per-block shadow path, as the plan
    // selects, 12 < w <= 16 to the lane kernels; dense storage keeps the lane
    // kernels for every w <= 16
    const bool narrow = !dense && pl->narrow_pref[precision] == 0;
    if (narrow) launch_pband_chol(pl, precision, blocks, info, st);
    if (precision == SYMPIX_PREC_FP64 && !dense && pl->narrow_pref[precision] == 2) {
        launch_f64_slices(pl, blocks, info, st);  // w <= 12 on the FP64 shadow, lane groups above
    } else if (precision == SYMPIX_PREC_FP32X2 && !dense && pl->narrow_pref[precision] == 2) {
        launch_df_slices(pl, blocks, info, st);  // w <= 12 on a split-FP32 shadow, lane groups above
    } else if (precision == SYMPIX_PREC_FP64) {
        if (!narrow) launch_band<ArF64>(pl, dense, blocks, info, st);  // (narrow: every w <= 16 done)
        trace_mark(pl, st, "k_factor_band");
    } else if (precision == SYMPIX_PREC_FP32 && !dense) {
        launch_f32_slices(pl, blocks, info, st, narrow);
    } else if (precision == SYMPIX_PREC_FP32) {
        launch_band<ArF32>(pl, dense, blocks, info, st);
        trace_mark(pl, st, "k_factor_band");
    } else {
        if (!narrow) launch_band<ArF2>(pl, dense, blocks, info, st);
        trace_mark(pl, st, "k_factor_band");
    }
    launch_factor_wide_dense(pl, precision, dense, blocks, info, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "sympix_factor_blocks: launch");
    return SYMPIX_OK;
}
