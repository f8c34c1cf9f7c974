// FP64 instantiation of the block-sampling kernels (one translation unit
// per arithmetic so that the build compiles them in parallel).
#include "sympix_sample_kernels.cuh"

namespace sympix {
template void launch_pband<0, true>(sympix_plan_t pl, const double *ninv, double *blocks, cudaStream_t st);
template void launch_pband<0, false>(sympix_plan_t pl, const double *ninv, double *blocks, cudaStream_t st);
}  // namespace sympix
