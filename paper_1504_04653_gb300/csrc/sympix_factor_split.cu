// FP32 factor: the band pass and the border sweep of a slice in two CTAs of
// one cooperative launch.
//
// In the fused kernel both roles share one SM, and so its shared-memory and
// load/store pipe, which both queue on: each runs at about half the speed it
// has alone.  Here CTAs [0, ns) run the band passes (warp 0; the other warps
// leave at once) and CTAs [ns, 2 ns) the border sweeps, so every role has an
// SM's pipes to itself.  The band CTA publishes how many periods of L11 rows
// are final in a global word of its slice (after a fence), then its results
// and a done flag; the border CTA polls them (each wait bounded, see
// f32_border).  Both words are zeroed before every launch.  The launch is
// cooperative, so every CTA is resident at once and no border CTA can wait
// on a band CTA that has not started.
#include "sympix_factor_kernels.cuh"

namespace sympix {

template <int WMAX, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_f32_split(const F32Slice *__restrict__ slices, const int32_t *__restrict__ items,
                const BlockDesc *__restrict__ blocks, float *__restrict__ sh, float *__restrict__ l21,
                const double *__restrict__ out, int32_t *__restrict__ info, float floor, int32_t *status,
                int wait_limit, int ns, int *flags, int *bandres) {
    extern __shared__ __align__(16) float fsm[];
    __shared__ SliceBlocks t;
    __shared__ int binfo[32];
    __shared__ int abort_s;
    const bool band = (int)blockIdx.x < ns;
    const int s = band ? (int)blockIdx.x : (int)blockIdx.x - ns;
    const F32Slice sl = slices[s];
    volatile int *prog = flags + 2 * s, *done = flags + 2 * s + 1;
    if (band) {
        if (threadIdx.x >= 32) return;
        const int L = threadIdx.x;
        int m = 0;
        if (L < sl.count) m = blocks[items[sl.first + L]].n - sl.w;
        const int r = F32BandDispatch<WMAX>::run(sl.w, sh + sl.sh, L, m, sl.rows - sl.w, fsm, floor, prog);
        bandres[s * 32 + L] = r;
        __threadfence();
        __syncwarp();
        if (L == 0) *done = 1;
        return;
    }
    load_slice_blocks(t, sl, items, blocks, nullptr);
    if (threadIdx.x == 0) abort_s = 0;
    __syncthreads();
    const FusedWait fw{prog, bandres + s * 32, &abort_s, status, wait_limit, done};
    if (sl.w > 0) {
        F32BorderDispatch<WMAX, 1, NT, kBorderSplit>::run(sl.w, sl, sh + sl.sh, l21 + sl.l21, out, t.off, t.n, t.live,
                                                          fsm, binfo, &fw);
    } else if (threadIdx.x == 0) {  // a diagonal block: only the band pass' result
        int spins = 0;
        while (*done == 0 && ++spins < wait_limit) __nanosleep(64);
        if (*done == 0) {
            abort_s = 1;
            atomicOr(status, kStatusTimeout);
        }
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x < 32 && threadIdx.x < sl.count) {
        const int L = threadIdx.x;
        const int br = ((volatile const int *)bandres)[s * 32 + L];
        info[t.bi[L]] = abort_s ? kInfoTimeout : ((br != 0 || sl.w == 0) ? br : binfo[L]);
    }
}

// floats of one CTA: the border role's staging (three periods, two periods
// of L21 values, the last W columns of A21), which covers the band role's two
// periods
template <int WMAX>
constexpr int split_smem_floats() {
    return 3 * (WMAX + 1) * (WMAX + 1) * 32 + 2 * WMAX * (WMAX + 1) * 32 + WMAX * WMAX * 32;
}

template <int WMAX, int NT, int MINB>
static bool split_fits(int count) {
    if (count <= 0) return true;
    auto kern = k_f32_split<WMAX, NT, MINB>;
    const size_t fs = (size_t)split_smem_floats<WMAX>() * sizeof(float);
    int dev = 0, sms = 0, per = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fs) != cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, NT, fs) != cudaSuccess)
        return false;
    return (int64_t)per * sms >= 2 * (int64_t)count;  // every CTA resident at once
}

template <int WMAX, int NT, int MINB>
static void launch_split_shape(sympix_plan_t pl, int first, int count, double *blocks, int32_t *info,
                               cudaStream_t st) {
    if (count <= 0) return;
    auto kern = k_f32_split<WMAX, NT, MINB>;
    const size_t fs = (size_t)split_smem_floats<WMAX>() * sizeof(float);
    const F32Slice *sl = pl->d_f32_slices.p + first;
    const int32_t *items = pl->d_f32_items.p;
    const BlockDesc *bd = pl->d_blocks.p;
    float *sh = pl->d_shadow_il.p, *l21 = pl->d_l21_il.p;
    const double *out = blocks;
    float floor = (float)pl->fp32_pivot_floor;
    int32_t *status = pl->d_status.p;
    int limit = pl->wait_limit, ns = count;
    int *flags = pl->d_split_flags.p + 2 * first, *bres = pl->d_split_bandres.p + 32 * first;
    void *args[] = {&sl, &items, &bd, &sh, &l21, &out, &info, &floor, &status, &limit, &ns, &flags, &bres};
    // every launch starts from zero words, whatever an earlier one that ran
    // out of waits left behind
    cudaMemsetAsync(flags, 0, 2 * sizeof(int) * (size_t)count, st);
    cudaLaunchCooperativeKernel((const void *)kern, dim3(2 * count), dim3(NT), args, fs, st);
}

// Whether the split launch of slices [0, f32_slices_w8) (w <= 8: eight
// border warps, one row each) can have every CTA resident at once.
bool f32_split_fits(sympix_plan_t pl) { return split_fits<8, 256, 2>(pl->f32_slices_w8); }

// The split launch of slices [0, f32_slices_w8).
void launch_f32_split_w8(sympix_plan_t pl, double *blocks, int32_t *info, cudaStream_t st) {
    launch_split_shape<8, 256, 2>(pl, 0, pl->f32_slices_w8, blocks, info, st);
}

}  // namespace sympix
