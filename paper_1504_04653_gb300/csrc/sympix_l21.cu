// Chunked border solve: the carry between chunks, the corner sums and
// corners, and the launchers in FP32 and FP64 (sympix_l21.cuh has the
// recurrence, the transfer and the solve).
#include "sympix_l21.cuh"

namespace sympix {

// --- carry -------------------------------------------------------------------
// Per block (lane), chunk by chunk: S_{q+1} = S_q T_q + P_q, one row of S at
// a time (the row in registers; T_q's entries read back from the item, which
// stays in L1 across the rows), from and to the lane-major item matrices.
template <class V, int W>
struct L21Carry {
    __device__ static void run(const L21Ctx<V> &c, int slice, int first, int nchunks, const V *T, const V *P,
                               V *S) {
        constexpr int C = l21_chunk_cols(W), LS = l21_lane_stride<V>(W);
        const int lane = threadIdx.x;
        const F32Slice sl = c.slices[slice];
        const L21Lane ln = l21_lane(c, sl, lane);
        for (int q = 1; q + 1 < nchunks; ++q) {
            if (!(ln.live && ln.m > (q + 1) * C)) break;  // the block ends in chunk q: nothing to carry
            const V *t = T + (int64_t)(first + q) * kL21Mat + lane * LS;
            const V *p = P + (int64_t)(first + q) * kL21Mat + lane * LS;
            const V *s = S + (int64_t)(first + q) * kL21Mat + lane * LS;
            V *sn = S + (int64_t)(first + q + 1) * kL21Mat + lane * LS;
#pragma unroll 1
            for (int b = 0; b < W; ++b) {
                V sb[W], r[W];
#pragma unroll
                for (int j = 0; j < W; ++j) sb[j] = s[b * W + j];
#pragma unroll
                for (int i = 0; i < W; ++i) r[i] = p[b * W + i];
#pragma unroll 2
                for (int j = 0; j < W; ++j) {
                    const V sj = sb[j];
#pragma unroll
                    for (int i = 0; i < W; ++i) r[i] = band_fma(sj, ldg_elem(t + j * W + i), r[i]);
                }
#pragma unroll
                for (int i = 0; i < W; ++i) sn[b * W + i] = r[i];
            }
        }
    }
};

template <class V>
__global__ void __launch_bounds__(32) k_l21_carry(L21Ctx<V> c, const int32_t *__restrict__ slice_ids,
                                                  const int32_t *__restrict__ first, const int32_t *__restrict__ nch,
                                                  const V *T, const V *P, V *S) {
    const int s = slice_ids[blockIdx.x];
    if (nch[s] < 3) return;  // chunks 0 and 1 need no carry
    L21Dispatch<L21Carry, V, 1, kL21WMax>::run(c.slices[s].w, c, s, first[s], nch[s], T, P, S);
}

// --- corner ------------------------------------------------------------------
// Per chunk, for widths whose recurrence does not form them: the pair sums
// sum_k L21[b][k] L21[b2][k] (b2 <= b, index b (b+1)/2 + b2) over the
// chunk's columns, from the stored L21.
template <class V, int W>
struct L21CornerPart {
    __device__ static void run(const L21Ctx<V> &c, int it, int2 item, V *Cs) {
        constexpr int C = l21_chunk_cols(W), NP = L21Pairs<W>::N;
        if constexpr (L21FusedCorner<V, W>::value) return;  // formed in the recurrence
        const int lane = threadIdx.x;
        const F32Slice sl = c.slices[item.x];
        const int kc = sl.rows - sl.w, k0 = item.y * C, k1 = min(kc, k0 + C);
        const V *l21 = c.l21 + sl.l21;
        V acc[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) acc[i] = V(0);
#pragma unroll 4
        for (int k = k0; k < k1; ++k) {
            V v[W];
#pragma unroll
            for (int b = 0; b < W; ++b) v[b] = l21[((int64_t)b * kc + k) * 32 + lane];
#pragma unroll
            for (int b = 0; b < W; ++b)
#pragma unroll
                for (int b2 = 0; b2 <= b; ++b2)
                    acc[b * (b + 1) / 2 + b2] = band_fma(v[b], v[b2], acc[b * (b + 1) / 2 + b2]);
        }
        l21_store_pairs<V, W>(Cs + (int64_t)it * kL21Pairs, lane, acc);
    }
};

template <class V>
__global__ void __launch_bounds__(32) k_l21_cornerpart(L21Ctx<V> c, const int2 *__restrict__ items, V *Cs, int it0) {
    const int it = it0 + blockIdx.x;
    const int2 item = items[it];
    L21Dispatch<L21CornerPart, V, 1, kL21WMax>::run(c.slices[item.x].w, c, it, item, Cs);
}

// Per block (lane): C = A22 - the pair sums over its chunks (summed in the
// working arithmetic, chunk by chunk, as the column sweep accumulates them),
// then the FP64 Cholesky C = L22 L22^T into the border rows' last W columns;
// LAPACK info m + i + 1 when pivot i is not positive.
template <class V, int W>
struct L21Corner {
    __device__ static void run(const L21Ctx<V> &c, int s, int first, int nchunks, const V *Cs, int32_t *info,
                               double *cm) {
        constexpr int NP = L21Pairs<W>::N;
        const int lane = threadIdx.x;
        const F32Slice sl = c.slices[s];
        const L21Lane ln = l21_lane(c, sl, lane);
        V sum[NP];
#pragma unroll
        for (int i = 0; i < NP; ++i) sum[i] = V(0);
        for (int q = 0; q < nchunks; ++q) {
            const V *cs = Cs + (int64_t)(first + q) * kL21Pairs + lane;
#pragma unroll
            for (int i = 0; i < NP; ++i) sum[i] += cs[i * 32];
        }
        if (!ln.live) return;
        const int m = ln.m;
        double *C = cm + lane * (W * W + 1);  // odd stride
#pragma unroll
        for (int i = 0; i < W; ++i)
#pragma unroll
            for (int j = 0; j <= i; ++j) C[i * W + j] = ln.view.a(m + i, m + j) - l21_to_f64(sum[i * (i + 1) / 2 + j]);
        int inf = 0;
        for (int i = 0; i < W && inf == 0; ++i) {
            for (int j = 0; j <= i; ++j) {
                double sv = C[i * W + j];
                for (int k = 0; k < j; ++k) sv -= C[i * W + k] * C[j * W + k];
                if (j < i) {
                    C[i * W + j] = sv / C[j * W + j];
                } else {
                    if (!(sv > 0.0)) {
                        inf = m + i + 1;
                        break;
                    }
                    C[i * W + i] = sqrt(sv);
                }
            }
        }
        for (int i = 0; i < W; ++i)
            for (int j = 0; j <= i; ++j) ln.view.put_b(i, m + j, C[i * W + j]);
        info[ln.bi] = inf;
    }
};

template <class V>
__global__ void __launch_bounds__(32) k_l21_corner(L21Ctx<V> c, const int32_t *__restrict__ slice_ids,
                                                   const int32_t *__restrict__ first,
                                                   const int32_t *__restrict__ nch, const V *Cs,
                                                   int32_t *__restrict__ info) {
    __shared__ double cm[32 * (kL21WMax * kL21WMax + 1)];
    const int s = slice_ids[blockIdx.x];
    L21Dispatch<L21Corner, V, 1, kL21WMax>::run(c.slices[s].w, c, s, first[s], nch[s], Cs, info, cm);
}

// The border rows and corners of slices [0, nf) after their band pass:
// transfer, carry, solve, corner sums, corners.  Items of slices with w <= 8
// come first (slices are in width order); the two width ranges of the
// transfer and the solve are separate kernels, run side by side.  hi_only:
// only the slices with 9 <= w <= 12, everything on `st`, no trace marks.
template <class V>
static void launch_l21(sympix_plan_t pl, const L21Ctx<V> &c, V *T, V *P, V *S, V *Cs, int32_t *info, cudaStream_t st,
                       bool hi_only) {
    constexpr bool FC8 = L21FusedCorner<V, 8>::value;  // the w <= 8 recurrence forms its pair sums
    const int ni = (int)pl->l21_items.size(), ns = (int)pl->l21_slices.size(), nlo = pl->l21_items_w8;
    const int2 *items = pl->d_l21_items.p;
    if (ni == 0) return;
    if (hi_only) {  // slices with 9 <= w <= 12 (the tail of both lists)
        const int s0 = pl->l21_slices_w8, nhs = ns - s0;
        if (ni == nlo) return;
        launch_l21_transfer_hi<V>(c, items, pl->d_l21_nch.p, T, P, S, Cs, nlo, ni - nlo, st);
        k_l21_carry<V><<<(unsigned)nhs, 32, 0, st>>>(c, pl->d_l21_slices.p + s0, pl->d_l21_first.p, pl->d_l21_nch.p,
                                                     T, P, S);
        launch_l21_solve_hi<V>(c, items, S, Cs, nlo, ni - nlo, st);
        k_l21_cornerpart<V><<<(unsigned)(ni - nlo), 32, 0, st>>>(c, items, Cs, nlo);
        k_l21_corner<V><<<(unsigned)nhs, 32, 0, st>>>(c, pl->d_l21_slices.p + s0, pl->d_l21_first.p,
                                                      pl->d_l21_nch.p, Cs, info);
        return;
    }
    // the two width ranges side by side: w <= 8 on `st`, 9..12 on the side stream
    const bool side = nlo > 0 && ni > nlo && pl->f32_side;
    cudaStream_t sh = side ? pl->f32_side : st;
    auto fork = [&] {
        if (!side) return;
        cudaEventRecord(pl->f32_fork, st);
        cudaStreamWaitEvent(sh, pl->f32_fork, 0);
    };
    auto join = [&] {
        if (!side) return;
        cudaEventRecord(pl->f32_join, sh);
        cudaStreamWaitEvent(st, pl->f32_join, 0);
    };
    fork();
    if (ni > nlo) launch_l21_transfer_hi<V>(c, items, pl->d_l21_nch.p, T, P, S, Cs, nlo, ni - nlo, sh);
    if (nlo > 0) launch_l21_transfer_lo<V>(c, items, pl->d_l21_nch.p, T, P, S, Cs, 0, nlo, st);
    join();
    trace_mark(pl, st, "k_l21_transfer");
    k_l21_carry<V><<<(unsigned)ns, 32, 0, st>>>(c, pl->d_l21_slices.p, pl->d_l21_first.p, pl->d_l21_nch.p, T, P, S);
    trace_mark(pl, st, "k_l21_carry");
    fork();
    if (ni > nlo) {  // then the pair sums of these widths (their recurrence does not form them)
        launch_l21_solve_hi<V>(c, items, S, Cs, nlo, ni - nlo, sh);
        k_l21_cornerpart<V><<<(unsigned)(ni - nlo), 32, 0, sh>>>(c, items, Cs, nlo);
    }
    if (nlo > 0) {
        launch_l21_solve_lo<V>(c, items, S, Cs, 0, nlo, st);
        if (!FC8) k_l21_cornerpart<V><<<(unsigned)nlo, 32, 0, st>>>(c, items, Cs, 0);
    }
    join();
    trace_mark(pl, st, "k_l21_solve");
    k_l21_corner<V><<<(unsigned)ns, 32, 0, st>>>(c, pl->d_l21_slices.p, pl->d_l21_first.p, pl->d_l21_nch.p, Cs,
                                                 info);
    trace_mark(pl, st, "k_l21_corner");
}

void launch_f32_l21(sympix_plan_t pl, double *blocks, int32_t *info, cudaStream_t st, bool hi_only) {
    const L21Ctx<float> c{pl->d_f32_slices.p, pl->d_f32_items.p, info, pl->d_blocks.p, pl->d_shadow_il.p,
                          pl->d_l21_il.p, blocks};
    launch_l21<float>(pl, c, pl->d_l21_T.p, pl->d_l21_P.p, pl->d_l21_S.p, pl->d_l21_C.p, info, st, hi_only);
}

// FP64: the same buffers hold twice the elements' bytes (the plan sizes them
// for it), read as doubles.
void launch_f64_l21(sympix_plan_t pl, double *blocks, int32_t *info, cudaStream_t st) {
    const L21Ctx<double> c{pl->d_f32_slices.p, pl->d_f32_items.p, info, pl->d_blocks.p,
                           reinterpret_cast<double *>(pl->d_shadow_il.p), reinterpret_cast<double *>(pl->d_l21_il.p),
                           blocks};
    launch_l21<double>(pl, c, reinterpret_cast<double *>(pl->d_l21_T.p), reinterpret_cast<double *>(pl->d_l21_P.p),
                       reinterpret_cast<double *>(pl->d_l21_S.p), reinterpret_cast<double *>(pl->d_l21_C.p), info, st,
                       false);
}

// Split FP32: the same buffers, read as (hi, lo) float pairs.
void launch_df_l21(sympix_plan_t pl, double *blocks, int32_t *info, cudaStream_t st) {
    const L21Ctx<DF> c{pl->d_f32_slices.p, pl->d_f32_items.p, info, pl->d_blocks.p,
                       reinterpret_cast<DF *>(pl->d_shadow_il.p), reinterpret_cast<DF *>(pl->d_l21_il.p), blocks};
    launch_l21<DF>(pl, c, reinterpret_cast<DF *>(pl->d_l21_T.p), reinterpret_cast<DF *>(pl->d_l21_P.p),
                   reinterpret_cast<DF *>(pl->d_l21_S.p), reinterpret_cast<DF *>(pl->d_l21_C.p), info, st, false);
}

int l21_chunk_cols_host(int w) { return l21_chunk_cols(w); }
int l21_mat_floats() { return kL21Mat; }
int l21_pair_floats() { return kL21Pairs; }

}  // namespace sympix
