// FP32 border rows of the periodic-band factor, L21 = A21 L11^-T, in
// parallel over column chunks.
//
// With L11 known (the band pass has run), each border row obeys the linear
// recurrence
//   L21[b][k] = (A21[b][k] - sum_{c=1..W} L21[b][k-c] L11[k][k-c]) / L11[k][k],
// where A21 is nonzero only in the first W columns (the wrap) and the last W
// (the band part).  A linear recurrence can be cut into chunks exactly:
// over a chunk of columns the window of the last W values maps affinely,
//   window_end = window_start T + P,
// where row j of T is the end window that the unit start window e_j gives
// without A21 terms, and P is the end window from a zero start with the
// chunk's A21 terms.  So:
//   transfer  every chunk after the first, in parallel: T (and P where some
//             block has A21 terms in it); the first chunk runs the real
//             recurrence from the zero window and writes its L21 at once;
//   carry     per block, sequentially over the chunks: S_{q+1} = S_q T_q + P_q
//             (W x W x W per chunk, a few dozen chunks);
//   solve     every chunk after the first, in parallel: the real recurrence
//             from S_q, writing L21;
//   corner    the sums S = L21 L21^T per chunk, then per block the corner
//             A22 - S = L22 L22^T in FP64 (LAPACK info m + i + 1 on failure).
// The result is the same L21 as the column-by-column sweep (the same
// recurrence, evaluated from exact carries), up to FP32 rounding order.
// Chunks are whole periods of W+1 columns (the unit of the row staging).
//
// One warp per (slice, chunk), lane = block of the slice; the L11 rows come
// from the lane-interleaved FP32 band shadow (element e of block L at
// 32 e + L), so every load of the warp covers 32 consecutive floats.
#pragma once

#include "sympix_factor_kernels.cuh"

namespace sympix {

constexpr int kL21WMax = 12;
constexpr int kL21Mat = kL21WMax * kL21WMax * 32;                // floats of one W x W matrix per item
constexpr int kL21Pairs = kL21WMax * (kL21WMax + 1) / 2 * 32;  // floats of the corner sums per item

__host__ __device__ constexpr int l21_chunk_cols(int w) { return (288 / (w + 1)) * (w + 1); }
// A W x W matrix of an item is stored lane-major: lane L's W*W values
// (row-major) at L * l21_lane_stride(W), a multiple of 4 floats, so a lane
// moves its matrix with 16-byte accesses.
__host__ __device__ constexpr int l21_lane_stride(int w) { return (w * w + 3) / 4 * 4; }
template <int W>
__device__ __forceinline__ void l21_store_mat(float *mat, int lane, const float (&v)[W][W]) {
    float4 *d = reinterpret_cast<float4 *>(mat + lane * l21_lane_stride(W));
    constexpr int NV = l21_lane_stride(W) / 4;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        float e[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int x = 4 * q + t;
            e[t] = x < W * W ? v[x / W][x % W] : 0.0f;
        }
        d[q] = make_float4(e[0], e[1], e[2], e[3]);
    }
}
template <int W>
__device__ __forceinline__ void l21_load_mat(const float *mat, int lane, float (&v)[W * W]) {
    const float4 *s = reinterpret_cast<const float4 *>(mat + lane * l21_lane_stride(W));
    constexpr int NV = l21_lane_stride(W) / 4;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const float4 e = s[q];
        const float t[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (4 * q + u < W * W) v[4 * q + u] = t[u];
    }
}

struct L21Ctx {
    const F32Slice *slices;
    const int32_t *items, *info;
    const BlockDesc *blocks;
    const float *sh;
    float *l21;
    const double *out;
};

// Slice geometry of one lane.
struct L21Lane {
    int w, m, kc, bi;
    bool live;
    PBandView view;
};

__device__ __forceinline__ L21Lane l21_lane(const L21Ctx &c, const F32Slice &sl, int lane) {
    L21Lane r;
    r.w = sl.w;
    r.kc = sl.rows - sl.w;
    r.bi = -1;
    r.m = 0;
    r.live = false;
    r.view = PBandView{nullptr, nullptr, 0, sl.w, 0};
    if (lane < sl.count) {
        r.bi = c.items[sl.first + lane];
        const BlockDesc bd = c.blocks[r.bi];
        r.m = bd.n - sl.w;
        r.live = c.info[r.bi] == 0;
        double *base = const_cast<double *>(c.out) + bd.off_pband;
        r.view = PBandView{base, base + (int64_t)bd.n * (sl.w + 1), bd.n, sl.w, r.m};
    }
    return r;
}

// The recurrence of W rows over columns [k0, k1) (k0 a multiple of W+1).
// The window y[b][c] holds row b's values at columns k-W+c, c = 0..W-1, and
// shifts by one column per step: a runtime loop over the columns whose body
// (W rows of W FMAs) stays small enough for the instruction cache, where a
// period-long unrolled ring would not.  REAL: A21 terms of the lane's block,
// values masked to 0 from column m on (and for blocks that are not live);
// otherwise the homogeneous recurrence.  WRITE: L21 stored.  CORNER: the
// pair sums sum_k L21[b][k] L21[b2][k] (index b (b+1)/2 + b2) added to sacc.
// The L11 rows of each period of W+1 columns are staged into `stage` (two
// period buffers of the warp) by asynchronous copies one period ahead.
// Columns left of 0 read zeros from the window (it starts at zero), so the
// unused slots of the first rows (which hold finite input values) add nothing.
template <int W>
struct L21Pairs {
    static constexpr int N = W * (W + 1) / 2;
};
template <int W>
constexpr int l21_stage_floats() { return 2 * (W + 1) * (W + 1) * 32; }

// NR rows b0 .. b0+NR-1 of the W (rows >= W are computed on zeros and not
// stored); the CTA's NWARP warps share the staging (each warp its own rows).
template <int W, int NR, int NWARP, bool REAL, bool WRITE, bool CORNER>
__device__ __forceinline__ void l21_run(float (&y)[NR][W], int b0, const float *__restrict__ shs, int lane, int k0,
                                        int k1, const L21Lane &ln, float *__restrict__ l21, float *stage,
                                        float (&sacc)[L21Pairs<W>::N]) {
    constexpr int RL = W + 1, CH = RL * RL;
    const int m = ln.m;
    const int p0 = k0 / RL, p1 = (k1 + RL - 1) / RL;  // periods [p0, p1)
    auto sync = [] {
        if constexpr (NWARP == 1)
            __syncwarp();
        else
            __syncthreads();
    };
    auto issue = [&](int p) {
        if (p < p1) {  // rows p RL .. p RL + W, all lanes: CH * 32 contiguous floats
            float *dst = stage + (p & 1) * CH * 32;
            const float *src = shs + (int64_t)p * RL * RL * 32;
            for (int i = threadIdx.x; i < CH * 8; i += 32 * NWARP) cp_async16(dst + 4 * i, src + 4 * i);
        }
        cp_async_commit();
    };
    issue(p0);
    for (int p = p0; p < p1; ++p) {
        sync();              // every thread is done with period p-1's buffer
        issue(p + 1);
        cp_async_wait<1>();  // period p has landed
        sync();              // ... for every thread's copies
        const float *prow = stage + (p & 1) * CH * 32 + lane;
        const int kend = min(RL, k1 - p * RL);
#pragma unroll 1
        for (int ph = 0; ph < kend; ++ph) {
            const int k = p * RL + ph;
            const float *row = prow + ph * RL * 32;  // L11 row k: offset d at row[32 d]
            float lr[RL];
#pragma unroll
            for (int d = 0; d < RL; ++d) lr[d] = row[d * 32];
            const float rd = rsqrtf(lr[0]);
            const float rcp = rd * rd;
            const bool in = REAL && ln.live && k < m;
            const bool a21 = in && (k < W || k >= m - W);  // the wrap or the band part of A21
            float val[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int b = b0 + r;
                float acc = 0.0f;
                if (REAL && a21 && b < W) acc = f64_to_f32_bits(ln.view.a(m + b, k));
#pragma unroll
                for (int c = 0; c < W; ++c) acc = fmaf(-y[r][c], lr[W - c], acc);
                val[r] = acc * rcp;
                if constexpr (REAL) val[r] = in ? val[r] : 0.0f;
                if constexpr (WRITE)
                    if (b < W) l21[((int64_t)b * ln.kc + k) * 32 + lane] = val[r];
#pragma unroll
                for (int c = 0; c + 1 < W; ++c) y[r][c] = y[r][c + 1];
                y[r][W - 1] = val[r];
            }
            if constexpr (CORNER) {  // NR == W, b0 == 0
#pragma unroll
                for (int b = 0; b < NR; ++b)
#pragma unroll
                    for (int b2 = 0; b2 <= b; ++b2)
                        sacc[b * (b + 1) / 2 + b2] = fmaf(val[b], val[b2], sacc[b * (b + 1) / 2 + b2]);
            }
        }
    }
    cp_async_wait<0>();
    sync();
}

// Rows per warp and warps per item of a width: up to 8 one warp holds all
// rows (and forms the pair sums); wider bands spread 3 rows over each of 4
// warps, which shortens the per-item chain those few blocks would set.
template <int W>
struct L21Split {
    static constexpr int NWARP = W <= 8 ? 1 : 4;
    static constexpr int NR = W <= 8 ? W : 3;
};

// Rows b0 .. b0+NR-1 of a lane-major W x W item matrix (scalar accesses:
// a row range need not start on a 16-byte boundary).
template <int W, int NR>
__device__ __forceinline__ void l21_store_rows(float *mat, int lane, int b0, const float (&v)[NR][W]) {
    float *d = mat + lane * l21_lane_stride(W);
#pragma unroll
    for (int r = 0; r < NR; ++r)
        if (b0 + r < W)
#pragma unroll
            for (int i = 0; i < W; ++i) d[(b0 + r) * W + i] = v[r][i];
}

template <int W>
__device__ __forceinline__ void l21_store_pairs(float *cs, int lane, const float (&sacc)[L21Pairs<W>::N]) {
#pragma unroll
    for (int i = 0; i < L21Pairs<W>::N; ++i) cs[i * 32 + lane] = sacc[i];
}

// Widths whose pair sums are formed in the recurrence (registers allow it);
// wider ones get them from a pass over the stored L21.
template <int W>
struct L21FusedCorner {
    static constexpr bool value = W <= 8;
};

// Width dispatch: F<W>::run(args...) for the slice's w in [WLO, W].
template <template <int> class F, int WLO, int W>
struct L21Dispatch {
    template <class... A>
    __device__ static void run(int w, A &&...a) {
        if (w == W)
            F<W>::run(std::forward<A>(a)...);
        else
            L21Dispatch<F, WLO, W - 1>::run(w, std::forward<A>(a)...);
    }
};
template <template <int> class F, int WLO>
struct L21Dispatch<F, WLO, WLO - 1> {
    template <class... A>
    __device__ static void run(int, A &&...) {}
};

// --- transfer ----------------------------------------------------------------
template <int W>
struct L21Transfer {
    __device__ static void run(const L21Ctx &c, int it, int2 item, int nchunks, float *T, float *P, float *S,
                               float *Cs, float *stage) {
        constexpr int C = l21_chunk_cols(W), NR = L21Split<W>::NR, NW = L21Split<W>::NWARP;
        constexpr bool FC = L21FusedCorner<W>::value;
        static_assert(!FC || (NW == 1 && NR == W), "the pair sums need every row in one warp");
        const int lane = threadIdx.x & 31, b0 = (threadIdx.x >> 5) * NR;
        float sacc[L21Pairs<W>::N];
#pragma unroll
        for (int i = 0; i < L21Pairs<W>::N; ++i) sacc[i] = 0.0f;
        const F32Slice sl = c.slices[item.x];
        const L21Lane ln = l21_lane(c, sl, lane);
        const int q = item.y, k0 = q * C, k1 = min(ln.kc, k0 + C);
        const float *shs = c.sh + sl.sh;
        float *l21 = c.l21 + sl.l21;
        float y[NR][W];
        if (q == 0) {  // the real recurrence from the zero window, L21 written
#pragma unroll
            for (int r = 0; r < NR; ++r)
#pragma unroll
                for (int i = 0; i < W; ++i) y[r][i] = 0.0f;
            l21_run<W, NR, NW, true, true, FC>(y, b0, shs, lane, k0, k1, ln, l21, stage, sacc);
            if (nchunks > 1) l21_store_rows<W, NR>(S + (int64_t)(it + 1) * kL21Mat, lane, b0, y);  // chunk 1's start
            if constexpr (FC) l21_store_pairs<W>(Cs + (int64_t)it * kL21Pairs, lane, sacc);
            return;
        }
        if (q == nchunks - 1) return;  // nothing follows the last chunk
        // T: the unit start windows, homogeneous
#pragma unroll
        for (int r = 0; r < NR; ++r)
#pragma unroll
            for (int i = 0; i < W; ++i) y[r][i] = (i == b0 + r) ? 1.0f : 0.0f;
        l21_run<W, NR, NW, false, false, false>(y, b0, shs, lane, k0, k1, ln, nullptr, stage, sacc);
        l21_store_rows<W, NR>(T + (int64_t)it * kL21Mat, lane, b0, y);
        // P: zero start with the band part of A21, where some block has it in
        // this chunk (zero elsewhere)
        const bool has = ln.live && ln.m > k0 && ln.m - W < k1;
#pragma unroll
        for (int r = 0; r < NR; ++r)
#pragma unroll
            for (int i = 0; i < W; ++i) y[r][i] = 0.0f;
        if (__syncthreads_or(has))
            l21_run<W, NR, NW, true, false, false>(y, b0, shs, lane, k0, k1, ln, nullptr, stage, sacc);
        l21_store_rows<W, NR>(P + (int64_t)it * kL21Mat, lane, b0, y);
    }
};

template <int WLO, int WHI>
__global__ void __launch_bounds__(128) k_l21_transfer(L21Ctx c, const int2 *__restrict__ items,
                                                     const int32_t *__restrict__ nch, float *T, float *P, float *S,
                                                     float *Cs, int it0) {
    extern __shared__ __align__(16) float l21_stage[];
    const int it = it0 + blockIdx.x;
    const int2 item = items[it];
    const int w = c.slices[item.x].w;
    L21Dispatch<L21Transfer, WLO, WHI>::run(w, c, it, item, nch[item.x], T, P, S, Cs, l21_stage);
}

// --- solve -------------------------------------------------------------------
template <int W>
struct L21Solve {
    __device__ static void run(const L21Ctx &c, int it, int2 item, const float *S, float *Cs, float *stage) {
        constexpr int C = l21_chunk_cols(W), NR = L21Split<W>::NR, NW = L21Split<W>::NWARP;
        constexpr bool FC = L21FusedCorner<W>::value;
        const int lane = threadIdx.x & 31, b0 = (threadIdx.x >> 5) * NR;
        float sacc[L21Pairs<W>::N];
#pragma unroll
        for (int i = 0; i < L21Pairs<W>::N; ++i) sacc[i] = 0.0f;
        const F32Slice sl = c.slices[item.x];
        const L21Lane ln = l21_lane(c, sl, lane);
        const int q = item.y, k0 = q * C, k1 = min(ln.kc, k0 + C);
        // blocks that ended before this chunk only write zeros: their start window is not carried
        const bool carried = ln.live && ln.m > k0;
        const float *s = S + (int64_t)it * kL21Mat + lane * l21_lane_stride(W);
        float y[NR][W];
#pragma unroll
        for (int r = 0; r < NR; ++r)
#pragma unroll
            for (int i = 0; i < W; ++i) y[r][i] = (carried && b0 + r < W) ? s[(b0 + r) * W + i] : 0.0f;
        l21_run<W, NR, NW, true, true, FC>(y, b0, c.sh + sl.sh, lane, k0, k1, ln, c.l21 + sl.l21, stage, sacc);
        if constexpr (FC) l21_store_pairs<W>(Cs + (int64_t)it * kL21Pairs, lane, sacc);
    }
};

template <int WLO, int WHI>
__global__ void __launch_bounds__(128) k_l21_solve(L21Ctx c, const int2 *__restrict__ items, const float *S, float *Cs,
                                                  int it0) {
    extern __shared__ __align__(16) float l21_stage[];
    const int it = it0 + blockIdx.x;
    const int2 item = items[it];
    if (item.y == 0) return;  // written by the transfer kernel
    L21Dispatch<L21Solve, WLO, WHI>::run(c.slices[item.x].w, c, it, item, S, Cs, l21_stage);
}

// launchers of the two width ranges (sympix_l21_lo.cu: 1..8, sympix_l21_hi.cu: 9..12)
void launch_l21_transfer_lo(const L21Ctx &c, const int2 *items, const int32_t *nch, float *T, float *P, float *S,
                            float *Cs, int it0, int count, cudaStream_t st);
void launch_l21_transfer_hi(const L21Ctx &c, const int2 *items, const int32_t *nch, float *T, float *P, float *S,
                            float *Cs, int it0, int count, cudaStream_t st);
void launch_l21_solve_lo(const L21Ctx &c, const int2 *items, const float *S, float *Cs, int it0, int count,
                         cudaStream_t st);
void launch_l21_solve_hi(const L21Ctx &c, const int2 *items, const float *S, float *Cs, int it0, int count,
                         cudaStream_t st);

}  // namespace sympix
