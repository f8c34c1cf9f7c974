// Chunked border solve, widths 9..12: the transfer and solve kernels
// (one translation unit per width range, compiled in parallel).
#include "sympix_l21.cuh"

namespace sympix {

void launch_l21_transfer_hi(const L21Ctx &c, const int2 *items, const int32_t *nch, float *T, float *P, float *S,
                            float *Cs, int it0, int count, cudaStream_t st) {
    const size_t smem = (size_t)l21_stage_floats<12>() * sizeof(float);
    cudaFuncSetAttribute(k_l21_transfer<9, 12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_l21_transfer<9, 12><<<(unsigned)count, 32 * L21Split<12>::NWARP, smem, st>>>(c, items, nch, T, P, S, Cs, it0);
}

void launch_l21_solve_hi(const L21Ctx &c, const int2 *items, const float *S, float *Cs, int it0, int count,
                         cudaStream_t st) {
    const size_t smem = (size_t)l21_stage_floats<12>() * sizeof(float);
    cudaFuncSetAttribute(k_l21_solve<9, 12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_l21_solve<9, 12><<<(unsigned)count, 32 * L21Split<12>::NWARP, smem, st>>>(c, items, S, Cs, it0);
}

}  // namespace sympix
