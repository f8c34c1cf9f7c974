// Border rows of the periodic-band factor, L21 = A21 L11^-T, in parallel
// over column chunks, in FP32 (V = float), FP64 (V = double) or split FP32
// (V = DF).
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
// recurrence, evaluated from exact carries), up to rounding order.  Chunks
// are whole periods of W+1 columns (the unit of the row staging).
//
// One warp per (slice, chunk), lane = block of the slice; the L11 rows come
// from the lane-interleaved band shadow (element e of block L at 32 e + L),
// so every load of the warp covers 32 consecutive elements.
#pragma once

#include "sympix_factor_kernels.cuh"

namespace sympix {

constexpr int kL21WMax = 12;
constexpr int kL21Mat = kL21WMax * kL21WMax * 32;                // elements of one W x W matrix per item
constexpr int kL21Pairs = kL21WMax * (kL21WMax + 1) / 2 * 32;  // elements of the corner sums per item

__host__ __device__ constexpr int l21_chunk_cols(int w) { return (288 / (w + 1)) * (w + 1); }
// A W x W matrix of an item is stored lane-major: lane L's W*W values
// (row-major) at L * l21_lane_stride<V>(W), a whole number of 16-byte
// units, so a lane moves its matrix with 16-byte accesses.
template <class V>
__host__ __device__ constexpr int l21_lane_stride(int w) {
    return (w * w + 16 / (int)sizeof(V) - 1) / (16 / (int)sizeof(V)) * (16 / (int)sizeof(V));
}

template <class V>
__device__ __forceinline__ V l21_from_f64(double x) { return elem_from_f64<V>(x); }
template <class V>
__device__ __forceinline__ double l21_to_f64(V x) { return elem_to_f64(x); }

template <class V, int W>
__device__ __forceinline__ void l21_store_mat(V *mat, int lane, const V (&v)[W][W]) {
    V *d = mat + lane * l21_lane_stride<V>(W);
    constexpr int P16 = 16 / (int)sizeof(V), NV = l21_lane_stride<V>(W) / P16;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        V e[P16];
#pragma unroll
        for (int t = 0; t < P16; ++t) {
            const int x = P16 * q + t;
            e[t] = x < W * W ? v[x / W][x % W] : V(0);
        }
        store16(d + P16 * q, e);
    }
}
template <class V, int W>
__device__ __forceinline__ void l21_load_mat(const V *mat, int lane, V (&v)[W * W]) {
    const V *s = mat + lane * l21_lane_stride<V>(W);
    constexpr int P16 = 16 / (int)sizeof(V), NV = l21_lane_stride<V>(W) / P16;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        V t[P16];
        load16(s + P16 * q, t);
#pragma unroll
        for (int u = 0; u < P16; ++u)
            if (P16 * q + u < W * W) v[P16 * q + u] = t[u];
    }
}

template <class V>
struct L21Ctx {
    const F32Slice *slices;
    const int32_t *items, *info;
    const BlockDesc *blocks;
    const V *sh;
    V *l21;
    const double *out;
};

// Slice geometry of one lane.
struct L21Lane {
    int w, m, kc, bi;
    bool live;
    PBandView view;
};

template <class V>
__device__ __forceinline__ L21Lane l21_lane(const L21Ctx<V> &c, const F32Slice &sl, int lane) {
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

template <int W>
struct L21Pairs {
    static constexpr int N = W * (W + 1) / 2;
};
// elements of a CTA's staging: two periods of W+1 rows, 32 blocks
template <int W>
constexpr int l21_stage_elems() { return 2 * (W + 1) * (W + 1) * 32; }

// The recurrence of W rows over columns [k0, k1) (k0 a multiple of W+1).
// The window y[b][c] holds row b's values at columns k-W+c, c = 0..W-1, and
// shifts by one column per step: a runtime loop over the columns whose body
// (W rows of W FMAs) stays small enough for the instruction cache, where a
// period-long unrolled ring would not.  REAL: A21 terms of the lane's block,
// values masked to 0 from column m on (and for blocks that are not live);
// otherwise the homogeneous recurrence.  WRITE: L21 stored.  CORNER: the
// pair sums sum_k L21[b][k] L21[b2][k] (index b (b+1)/2 + b2) added to sacc.
// The L11 rows of each period of W+1 columns are staged into `stage` (two
// period buffers of the CTA) by asynchronous copies one period ahead.
// Columns left of 0 read zeros from the window (it starts at zero), so the
// unused slots of the first rows (which hold finite input values) add nothing.
// NR rows b0 .. b0+NR-1 of the W (rows >= W are computed on zeros and not
// stored); the CTA's NWARP warps share the staging (each warp its own rows).
template <class V, int W, int NR, int NWARP, bool REAL, bool WRITE, bool CORNER>
__device__ __forceinline__ void l21_run(V (&y)[NR][W], int b0, const V *__restrict__ shs, int lane, int k0, int k1,
                                        const L21Lane &ln, V *__restrict__ l21, V *stage,
                                        V (&sacc)[L21Pairs<W>::N]) {
    constexpr int RL = W + 1, CH = RL * RL, P16 = 16 / (int)sizeof(V);
    const int m = ln.m;
    const int p0 = k0 / RL, p1 = (k1 + RL - 1) / RL;  // periods [p0, p1)
    auto sync = [] {
        if constexpr (NWARP == 1)
            __syncwarp();
        else
            __syncthreads();
    };
    auto issue = [&](int p) {
        if (p < p1) {  // rows p RL .. p RL + W, all lanes: CH * 32 contiguous elements
            V *dst = stage + (p & 1) * CH * 32;
            const V *src = shs + (int64_t)p * RL * RL * 32;
            for (int i = threadIdx.x; i < CH * 32 / P16; i += 32 * NWARP) cp_async16(dst + P16 * i, src + P16 * i);
        }
        cp_async_commit();
    };
    issue(p0);
    for (int p = p0; p < p1; ++p) {
        sync();              // every thread is done with period p-1's buffer
        issue(p + 1);
        cp_async_wait<1>();  // period p has landed
        sync();              // ... for every thread's copies
        const V *prow = stage + (p & 1) * CH * 32 + lane;
        const int kend = min(RL, k1 - p * RL);
#pragma unroll 1
        for (int ph = 0; ph < kend; ++ph) {
            const int k = p * RL + ph;
            const V *row = prow + ph * RL * 32;  // L11 row k: offset d at row[32 d]
            V lr[RL];
#pragma unroll
            for (int d = 0; d < RL; ++d) lr[d] = row[d * 32];
            const V rd = band_rsqrt(lr[0]);
            const V rcp = rd * rd;
            const bool in = REAL && ln.live && k < m;
            const bool a21 = in && (k < W || k >= m - W);  // the wrap or the band part of A21
            V val[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int b = b0 + r;
                V acc = V(0);
                if (REAL && a21 && b < W) acc = l21_from_f64<V>(ln.view.a(m + b, k));
#pragma unroll
                for (int c = 0; c < W; ++c) acc = band_fma(-y[r][c], lr[W - c], acc);
                val[r] = acc * rcp;
                if constexpr (REAL) val[r] = in ? val[r] : V(0);
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
                        sacc[b * (b + 1) / 2 + b2] = band_fma(val[b], val[b2], sacc[b * (b + 1) / 2 + b2]);
            }
        }
    }
    cp_async_wait<0>();
    sync();
}

// Rows per warp and warps per item of a width.  FP32: up to 8 one warp
// holds all rows (and forms the pair sums); wider bands spread 3 rows over
// each of 4 warps, which shortens the per-item chain those few blocks would
// set.  FP64 and split FP32 (twice the registers per value): up to 8 rows
// over 2 warps, 9 to 12 over 4.  The warp count is the same for
// every width of one launch range (1..8, 9..12): it is the CTA's, and all
// its warps take part in the staging and its barriers.
template <class V, int W>
struct L21Split {
    static constexpr bool WIDE = sizeof(V) == 8;  // two registers a value
    static constexpr int NWARP = W <= 8 ? (WIDE ? 2 : 1) : 4;
    static constexpr int NR = (W + NWARP - 1) / NWARP;
};

// Widths whose pair sums are formed in the recurrence (registers allow it:
// FP32 up to 8); the rest get them from a pass over the stored L21.
template <class V, int W>
struct L21FusedCorner {
    static constexpr bool value = sizeof(V) == 4 && W <= 8;
};

// Rows b0 .. b0+NR-1 of a lane-major W x W item matrix (scalar accesses:
// a row range need not start on a 16-byte boundary).
template <class V, int W, int NR>
__device__ __forceinline__ void l21_store_rows(V *mat, int lane, int b0, const V (&v)[NR][W]) {
    V *d = mat + lane * l21_lane_stride<V>(W);
#pragma unroll
    for (int r = 0; r < NR; ++r)
        if (b0 + r < W)
#pragma unroll
            for (int i = 0; i < W; ++i) d[(b0 + r) * W + i] = v[r][i];
}

template <class V, int W>
__device__ __forceinline__ void l21_store_pairs(V *cs, int lane, const V (&sacc)[L21Pairs<W>::N]) {
#pragma unroll
    for (int i = 0; i < L21Pairs<W>::N; ++i) cs[i * 32 + lane] = sacc[i];
}

// Width dispatch: F<V, W>::run(args...) for the slice's w in [WLO, W].
template <template <class, int> class F, class V, int WLO, int W>
struct L21Dispatch {
    template <class... A>
    __device__ static void run(int w, A &&...a) {
        if (w == W)
            F<V, W>::run(std::forward<A>(a)...);
        else
            L21Dispatch<F, V, WLO, W - 1>::run(w, std::forward<A>(a)...);
    }
};
template <template <class, int> class F, class V, int WLO>
struct L21Dispatch<F, V, WLO, WLO - 1> {
    template <class... A>
    __device__ static void run(int, A &&...) {}
};

// Threads of a transfer / solve CTA for the widths up to WHI (every width
// of the range has this many warps; rows >= W are computed on zeros and
// not stored).
template <class V, int WHI>
constexpr int l21_cta_threads() { return 32 * L21Split<V, WHI>::NWARP; }

// --- transfer ----------------------------------------------------------------
template <class V, int W>
struct L21Transfer {
    __device__ static void run(const L21Ctx<V> &c, int it, int2 item, int nchunks, V *T, V *P, V *S, V *Cs,
                               V *stage) {
        constexpr int C = l21_chunk_cols(W), NR = L21Split<V, W>::NR, NW = L21Split<V, W>::NWARP;
        static_assert(NW == L21Split<V, (W <= 8 ? 8 : kL21WMax)>::NWARP, "the CTA's warp count");
        constexpr bool FC = L21FusedCorner<V, W>::value;
        static_assert(!FC || (NW == 1 && NR == W), "the pair sums need every row in one warp");
        const int lane = threadIdx.x & 31, b0 = (threadIdx.x >> 5) * NR;
        V sacc[L21Pairs<W>::N];
#pragma unroll
        for (int i = 0; i < L21Pairs<W>::N; ++i) sacc[i] = V(0);
        const F32Slice sl = c.slices[item.x];
        const L21Lane ln = l21_lane(c, sl, lane);
        const int q = item.y, k0 = q * C, k1 = min(ln.kc, k0 + C);
        const V *shs = c.sh + sl.sh;
        V *l21 = c.l21 + sl.l21;
        V y[NR][W];
        if (q == 0) {  // the real recurrence from the zero window, L21 written
#pragma unroll
            for (int r = 0; r < NR; ++r)
#pragma unroll
                for (int i = 0; i < W; ++i) y[r][i] = V(0);
            l21_run<V, W, NR, NW, true, true, FC>(y, b0, shs, lane, k0, k1, ln, l21, stage, sacc);
            if (nchunks > 1) l21_store_rows<V, W, NR>(S + (int64_t)(it + 1) * kL21Mat, lane, b0, y);  // chunk 1's start
            if constexpr (FC) l21_store_pairs<V, W>(Cs + (int64_t)it * kL21Pairs, lane, sacc);
            return;
        }
        if (q == nchunks - 1) return;  // nothing follows the last chunk
        // T: the unit start windows, homogeneous
#pragma unroll
        for (int r = 0; r < NR; ++r)
#pragma unroll
            for (int i = 0; i < W; ++i) y[r][i] = (i == b0 + r) ? V(1) : V(0);
        l21_run<V, W, NR, NW, false, false, false>(y, b0, shs, lane, k0, k1, ln, nullptr, stage, sacc);
        l21_store_rows<V, W, NR>(T + (int64_t)it * kL21Mat, lane, b0, y);
        // P: zero start with the band part of A21, where some block has it in
        // this chunk (zero elsewhere)
        const bool has = ln.live && ln.m > k0 && ln.m - W < k1;
#pragma unroll
        for (int r = 0; r < NR; ++r)
#pragma unroll
            for (int i = 0; i < W; ++i) y[r][i] = V(0);
        if (__syncthreads_or(has))
            l21_run<V, W, NR, NW, true, false, false>(y, b0, shs, lane, k0, k1, ln, nullptr, stage, sacc);
        l21_store_rows<V, W, NR>(P + (int64_t)it * kL21Mat, lane, b0, y);
    }
};

template <class V, int WLO, int WHI>
__global__ void __launch_bounds__(128) k_l21_transfer(L21Ctx<V> c, const int2 *__restrict__ items,
                                                     const int32_t *__restrict__ nch, V *T, V *P, V *S, V *Cs,
                                                     int it0) {
    extern __shared__ __align__(16) unsigned char l21_smem[];
    V *stage = reinterpret_cast<V *>(l21_smem);
    const int it = it0 + blockIdx.x;
    const int2 item = items[it];
    const int w = c.slices[item.x].w;
    L21Dispatch<L21Transfer, V, WLO, WHI>::run(w, c, it, item, nch[item.x], T, P, S, Cs, stage);
}

// --- solve -------------------------------------------------------------------
template <class V, int W>
struct L21Solve {
    __device__ static void run(const L21Ctx<V> &c, int it, int2 item, const V *S, V *Cs, V *stage) {
        constexpr int C = l21_chunk_cols(W), NR = L21Split<V, W>::NR, NW = L21Split<V, W>::NWARP;
        static_assert(NW == L21Split<V, (W <= 8 ? 8 : kL21WMax)>::NWARP, "the CTA's warp count");
        constexpr bool FC = L21FusedCorner<V, W>::value;
        const int lane = threadIdx.x & 31, b0 = (threadIdx.x >> 5) * NR;
        V sacc[L21Pairs<W>::N];
#pragma unroll
        for (int i = 0; i < L21Pairs<W>::N; ++i) sacc[i] = V(0);
        const F32Slice sl = c.slices[item.x];
        const L21Lane ln = l21_lane(c, sl, lane);
        const int q = item.y, k0 = q * C, k1 = min(ln.kc, k0 + C);
        // blocks that ended before this chunk only write zeros: their start window is not carried
        const bool carried = ln.live && ln.m > k0;
        const V *s = S + (int64_t)it * kL21Mat + lane * l21_lane_stride<V>(W);
        V y[NR][W];
#pragma unroll
        for (int r = 0; r < NR; ++r)
#pragma unroll
            for (int i = 0; i < W; ++i) y[r][i] = (carried && b0 + r < W) ? s[(b0 + r) * W + i] : V(0);
        l21_run<V, W, NR, NW, true, true, FC>(y, b0, c.sh + sl.sh, lane, k0, k1, ln, c.l21 + sl.l21, stage, sacc);
        if constexpr (FC) l21_store_pairs<V, W>(Cs + (int64_t)it * kL21Pairs, lane, sacc);
    }
};

template <class V, int WLO, int WHI>
__global__ void __launch_bounds__(128) k_l21_solve(L21Ctx<V> c, const int2 *__restrict__ items, const V *S, V *Cs,
                                                  int it0) {
    extern __shared__ __align__(16) unsigned char l21_smem[];
    V *stage = reinterpret_cast<V *>(l21_smem);
    const int it = it0 + blockIdx.x;
    const int2 item = items[it];
    if (item.y == 0) return;  // written by the transfer kernel
    L21Dispatch<L21Solve, V, WLO, WHI>::run(c.slices[item.x].w, c, it, item, S, Cs, stage);
}

// launchers of the two width ranges (sympix_l21_lo.cu: 1..8, sympix_l21_hi.cu: 9..12)
template <class V>
void launch_l21_transfer_lo(const L21Ctx<V> &c, const int2 *items, const int32_t *nch, V *T, V *P, V *S, V *Cs,
                            int it0, int count, cudaStream_t st);
template <class V>
void launch_l21_transfer_hi(const L21Ctx<V> &c, const int2 *items, const int32_t *nch, V *T, V *P, V *S, V *Cs,
                            int it0, int count, cudaStream_t st);
template <class V>
void launch_l21_solve_lo(const L21Ctx<V> &c, const int2 *items, const V *S, V *Cs, int it0, int count,
                         cudaStream_t st);
template <class V>
void launch_l21_solve_hi(const L21Ctx<V> &c, const int2 *items, const V *S, V *Cs, int it0, int count,
                         cudaStream_t st);

}  // namespace sympix
