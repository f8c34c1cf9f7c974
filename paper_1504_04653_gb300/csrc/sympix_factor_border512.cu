// FP32 border pass of periodic-band slices, 512 threads per CTA (one
// translation unit per thread count, so the build compiles them in parallel).
#include "sympix_factor_kernels.cuh"

namespace sympix {

template <>
void launch_f32_border<512>(sympix_plan_t pl, int first, int count, double *blocks, int32_t *info, cudaStream_t st) {
    const size_t bs = (size_t)kF32BorderStage * sizeof(float);
    cudaFuncSetAttribute(k_f32_border_pass<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bs);
    k_f32_border_pass<512><<<(unsigned)count, 512, bs, st>>>(pl->d_f32_slices.p + first, pl->d_f32_items.p,
                                                        pl->d_blocks.p, pl->d_shadow_il.p, pl->d_l21_il.p, blocks,
                                                        info);
}

}  // namespace sympix
