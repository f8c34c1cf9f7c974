// Chunked border solve, widths 1..8: the transfer and solve kernels in FP32,
// FP64 and split FP32 (one translation unit per width range, compiled in parallel).
#include "sympix_l21.cuh"

namespace sympix {

template <class V>
void launch_l21_transfer_lo(const L21Ctx<V> &c, const int2 *items, const int32_t *nch, V *T, V *P, V *S, V *Cs,
                            int it0, int count, cudaStream_t st) {
    auto kern = k_l21_transfer<V, 1, 8>;
    const size_t smem = (size_t)l21_stage_elems<8>() * sizeof(V);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<(unsigned)count, l21_cta_threads<V, 8>(), smem, st>>>(c, items, nch, T, P, S, Cs, it0);
}

template <class V>
void launch_l21_solve_lo(const L21Ctx<V> &c, const int2 *items, const V *S, V *Cs, int it0, int count,
                         cudaStream_t st) {
    auto kern = k_l21_solve<V, 1, 8>;
    const size_t smem = (size_t)l21_stage_elems<8>() * sizeof(V);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<(unsigned)count, l21_cta_threads<V, 8>(), smem, st>>>(c, items, S, Cs, it0);
}

template void launch_l21_transfer_lo<float>(const L21Ctx<float> &, const int2 *, const int32_t *, float *, float *,
                                            float *, float *, int, int, cudaStream_t);
template void launch_l21_transfer_lo<double>(const L21Ctx<double> &, const int2 *, const int32_t *, double *,
                                             double *, double *, double *, int, int, cudaStream_t);
template void launch_l21_solve_lo<float>(const L21Ctx<float> &, const int2 *, const float *, float *, int, int,
                                         cudaStream_t);
template void launch_l21_solve_lo<double>(const L21Ctx<double> &, const int2 *, const double *, double *, int, int,
                                          cudaStream_t);

template void launch_l21_transfer_lo<DF>(const L21Ctx<DF> &, const int2 *, const int32_t *, DF *, DF *, DF *, DF *, int,
                                      int, cudaStream_t);
template void launch_l21_solve_lo<DF>(const L21Ctx<DF> &, const int2 *, const DF *, DF *, int, int, cudaStream_t);

}  // namespace sympix
