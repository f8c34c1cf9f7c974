// Chunked border solve, widths 1..8: the transfer and solve kernels
// (one translation unit per width range, compiled in parallel).
#include "sympix_l21.cuh"

namespace sympix {

void launch_l21_transfer_lo(const L21Ctx &c, const int2 *items, const int32_t *nch, float *T, float *P, float *S,
                            float *Cs, int it0, int count, cudaStream_t st) {
    const size_t smem = (size_t)l21_stage_floats<8>() * sizeof(float);
    cudaFuncSetAttribute(k_l21_transfer<1, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_l21_transfer<1, 8><<<(unsigned)count, 32 * L21Split<8>::NWARP, smem, st>>>(c, items, nch, T, P, S, Cs, it0);
}

void launch_l21_solve_lo(const L21Ctx &c, const int2 *items, const float *S, float *Cs, int it0, int count,
                         cudaStream_t st) {
    const size_t smem = (size_t)l21_stage_floats<8>() * sizeof(float);
    cudaFuncSetAttribute(k_l21_solve<1, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_l21_solve<1, 8><<<(unsigned)count, 32 * L21Split<8>::NWARP, smem, st>>>(c, items, S, Cs, it0);
}

}  // namespace sympix
