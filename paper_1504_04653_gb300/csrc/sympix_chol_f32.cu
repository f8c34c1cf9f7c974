// Narrow-band factor, ArF32 instantiation (one translation unit per
// arithmetic, compiled in parallel).
#include "sympix_chol.cuh"

namespace sympix {

void launch_chol_f32(sympix_plan_t pl, double *blocks, int32_t *info, int rescue, int wmax) {
    auto one = [&](auto WWc) {
        constexpr int WW = decltype(WWc)::value;
        const int cnt = pl->chol_n32[WW];
        if (!cnt || WW > wmax) return;
        constexpr int G = chol_lanes<ArF32>(WW);
        constexpr size_t smem = chol_smem_bytes<ArF32, WW, G>();
        auto kern = k_pband_chol<ArF32, WW, G>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<(unsigned)cnt, 32, smem, pl->chol_st[WW]>>>(pl->d_chol_sl32.p + pl->chol_f32[WW],
                                                           pl->d_chol_items.p, pl->d_blocks.p, blocks, pl->d_shadow.p,
                                                           info, (float)pl->fp32_pivot_floor, rescue);
    };
    HostStaticFor<0, kCholWMax + 1>::run(one);
}

}  // namespace sympix
