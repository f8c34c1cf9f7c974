// Cholesky of wide bands (16 < w <= 64, a CTA per block) and of dense-format
// blocks (a warp per block up to n = 1024, a blocked CTA per block above),
// and their launcher.
#include "sympix_factor_kernels.cuh"

namespace sympix {

// ---------------------------------------------------------------------------
// Wide bands (16 < w <= 64): one CTA per block.
//
// The active band window (rows k..k+w, columns k..k+w), the w border rows at
// columns k..k+w and the corner accumulator S live in shared memory; rows
// and columns are stored at index mod (w+1), so moving the window to column
// k+1 costs nothing: the slot of row/column k is reused for k+1+w.  Per
// column: thread 0 forms the pivot, the threads scale the column (band and
// border), then apply the rank-1 update to the band window, the border rows
// and S while the next band row and border column, loaded one column ahead,
// go into the freed slots.  T = double or float; the float version sends a
// block whose pivot falls below the floor to the FP64 rescue.
// ---------------------------------------------------------------------------
constexpr int kWideMax = 64;

template <typename T>
__device__ __forceinline__ T wide_from(double x);
template <>
__device__ __forceinline__ double wide_from<double>(double x) { return x; }
template <>
__device__ __forceinline__ float wide_from<float>(double x) { return f64_to_f32_bits(x); }
__device__ __forceinline__ double wide_to(double x) { return x; }
__device__ __forceinline__ double wide_to(float x) { return f32_to_f64_bits(x); }

// Where the wide kernel writes L: straight into the FP64 blocks (FP64), or
// into the FP32 band shadow, copied to the FP64 blocks only once the block
// has factored without reaching the pivot floor (so an FP64 rescue still
// finds its input intact).
template <typename T, class View>
struct WideSink;
template <class View>
struct WideSink<double, View> {
    View v;
    __device__ void put_l(int i, int j, double x) const { v.put_l(i, j, x); }
    __device__ void put_b(int b, int j, double x) const { v.put_b(b, j, x); }
    __device__ double get_b(int b, int j) const { return v.get_b(b, j); }
};
template <class View>
struct WideSink<float, View> {
    float *band;  // shadow: n x (w+1) band, then w x n border
    int n, w;
    __device__ void put_l(int i, int j, float x) const { band[(int64_t)i * (w + 1) + (i - j)] = x; }
    __device__ void put_b(int b, int j, float x) const { band[(int64_t)n * (w + 1) + (int64_t)b * n + j] = x; }
    __device__ double get_b(int b, int j) const {
        return f32_to_f64_bits(band[(int64_t)n * (w + 1) + (int64_t)b * n + j]);
    }
};

template <typename T, bool DENSE>
__global__ void __launch_bounds__(256) k_factor_wide(int nitems, const int32_t *__restrict__ items,
                                                     const BlockDesc *__restrict__ blocks, double *__restrict__ out,
                                                     int32_t *__restrict__ info, int rescue, float floor,
                                                     float *__restrict__ shadow) {
    extern __shared__ double wsm_raw[];
    T *wsm = reinterpret_cast<T *>(wsm_raw);
    const int bi = items[blockIdx.x];
    if (rescue && info[bi] != kRescue) return;
    const BlockDesc bd = blocks[bi];
    typedef typename ViewOf<DENSE>::T View;
    const View v = ViewOf<DENSE>::make(out, bd);
    const int w = bd.w, m = bd.n - bd.w, S = w + 1;
    auto make_sink = [&]() {
        if constexpr (sizeof(T) == 4)
            return WideSink<T, View>{shadow + bd.off_pband, bd.n, w};
        else
            return WideSink<T, View>{v};
    };
    const WideSink<T, View> sink = make_sink();
    T *Wn = wsm;         // S x S, [row mod S][col mod S]
    T *Bd = Wn + S * S;  // w x S, [b][col mod S]
    T *Sc = Bd + w * S;  // w x w corner accumulator
    T *lc = Sc + w * w;  // S: column k of L (band rows k..k+w)
    T *lb = lc + S;      // w: column k of L (border rows)
    T *od = lb + w;      // S: original diagonal of the window rows
    __shared__ T piv;
    __shared__ int fail;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < S * S; e += nt) {
        const int r = e / S, c = e % S;
        Wn[e] = (c <= r && r < m) ? wide_from<T>(v.a(r, c)) : T(0);
        if (c == r) od[r] = Wn[e];
    }
    for (int e = tid; e < w * S; e += nt) {
        const int b = e / S, c = e % S;
        Bd[e] = c < m ? wide_from<T>(v.a(m + b, c)) : T(0);
    }
    for (int e = tid; e < w * w; e += nt) {
        const int b = e / w, c = e % w;
        Sc[e] = c <= b ? wide_from<T>(v.a(m + b, m + c)) : T(0);
    }
    if (tid == 0) fail = 0;
    const int nband = w * (w + 1) / 2, nbord = w * w, ncorner = w * (w + 1) / 2;
    const int e0 = nband + nbord + ncorner, total = e0 + S;
    // the new-row element this thread stores each column (c < S), if any
    int myc = -1;
    for (int e = tid; e < total; e += nt)
        if (e >= e0) myc = e - e0;
    auto fetch = [&](int nc, T &pa, T &pb) {
        pa = (myc >= 0 && nc < m) ? wide_from<T>(v.a(nc, nc - w + myc)) : T(0);
        pb = (myc >= 0 && myc < w && nc < m) ? wide_from<T>(v.a(m + myc, nc)) : T(0);
    };
    T pa, pb;
    fetch(1 + w, pa, pb);
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        const int ks = k % S;
        if (tid == 0) {
            const T d = Wn[ks * S + ks];
            if (!(d > T(floor) * od[ks])) {
                fail = (sizeof(T) == 4) ? kRescue : k + 1;
            } else {
                const T lkk = sqrt(d);
                piv = T(1) / lkk;
                sink.put_l(k, k, lkk);
            }
        }
        __syncthreads();
        if (fail) break;
        const T rs = piv;
        for (int r = tid; r < S + w; r += nt) {
            if (r == 0) {
                lc[0] = T(0);
            } else if (r <= w) {
                const int row = k + r;
                const T l = row < m ? Wn[(row % S) * S + ks] * rs : T(0);
                lc[r] = l;
                if (row < m) sink.put_l(row, k, l);
            } else {
                const int b = r - S;
                const T l = Bd[b * S + ks] * rs;
                lb[b] = l;
                sink.put_b(b, k, l);
            }
        }
        __syncthreads();
        const int nc = k + 1 + w;
        for (int e = tid; e < total; e += nt) {
            if (e < nband) {
                int r = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f) + 1;
                while (r * (r - 1) / 2 > e) --r;
                while ((r + 1) * r / 2 <= e) ++r;
                const int c = e - r * (r - 1) / 2 + 1;
                const int row = k + r;
                if (row < m) Wn[(row % S) * S + (k + c) % S] -= lc[r] * lc[c];
            } else if (e < nband + nbord) {
                const int f = e - nband, b = f / w, c = f % w + 1;
                Bd[b * S + (k + c) % S] -= lb[b] * lc[c];
            } else if (e < e0) {
                const int f = e - nband - nbord;
                int b = (int)((sqrtf(8.0f * f + 1.0f) - 1.0f) * 0.5f);
                while (b * (b + 1) / 2 > f) --b;
                while ((b + 1) * (b + 2) / 2 <= f) ++b;
                const int c = f - b * (b + 1) / 2;
                Sc[b * w + c] -= lb[b] * lb[c];
            } else {
                // band row nc (columns k+1..nc) and the border rows' column nc
                // into the slot freed by row/column k
                const int c = e - e0;
                if (nc < m) {
                    Wn[ks * S + (k + 1 + c) % S] = pa;
                    if (c == w) od[ks] = pa;
                }
                if (c < w) Bd[c * S + ks] = pb;
            }
        }
        fetch(nc + 1, pa, pb);
        __syncthreads();
    }
    if (fail) {
        if (tid == 0) info[bi] = fail;
        return;
    }
    __shared__ int cinf;
    if (tid == 0) {
        // the w x w corner, FP64 arithmetic
        int inf = 0;
        for (int i = 0; i < w && inf == 0; ++i) {
            for (int j = 0; j <= i; ++j) {
                double s = wide_to(Sc[i * w + j]);
                for (int q = 0; q < j; ++q) s -= sink.get_b(i, m + q) * sink.get_b(j, m + q);
                if (j < i) {
                    sink.put_b(i, m + j, T(s / sink.get_b(j, m + j)));
                } else {
                    if (!(s > 0.0)) {
                        inf = m + i + 1;
                        break;
                    }
                    sink.put_b(i, m + i, T(sqrt(s)));
                }
            }
        }
        if (sizeof(T) == 4 && inf) inf = kRescue;  // let FP64 decide
        cinf = inf;
        info[bi] = inf;
    }
    if constexpr (sizeof(T) == 4) {
        // the block factored in FP32: copy L from the shadow
        __syncthreads();
        if (cinf) return;
        const int64_t nb = (int64_t)m * S;  // band rows < m
        for (int64_t e = tid; e < nb; e += nt) {
            const int row = (int)(e / S), d = (int)(e % S);
            if (d <= row) out[bd.off_pband + e] = f32_to_f64_bits(sink.band[e]);
        }
        const int64_t bo = (int64_t)bd.n * S;
        for (int64_t e = tid; e < (int64_t)w * bd.n; e += nt) {
            const int b = (int)(e / bd.n), j = (int)(e % bd.n);
            if (j <= m + b) out[bd.off_pband + bo + e] = f32_to_f64_bits(sink.band[bo + e]);
        }
    }
}

// One warp per dense-format block: right-looking, FP64, in place.
__global__ void __launch_bounds__(128) k_factor_dense(int nitems, const int32_t *__restrict__ items,
                                                      const BlockDesc *__restrict__ blocks, double *__restrict__ out,
                                                      int dense_storage, int32_t *__restrict__ info) {
    const int lane = threadIdx.x & 31;
    const int idx = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (idx >= nitems) return;
    const int bi = items[idx];
    const BlockDesc bd = blocks[bi];
    const int n = bd.n;
    double *p = out + (dense_storage ? bd.off_dense : bd.off_pband);
    int inf = 0;
    for (int k = 0; k < n; ++k) {
        const double dkk = p[(int64_t)k * n + k];
        if (!(dkk > 0.0)) {
            inf = k + 1;
            break;
        }
        const double lkk = sqrt(dkk);
        const double rl = 1.0 / lkk;
        __syncwarp();
        if (lane == 0) p[(int64_t)k * n + k] = lkk;
        for (int i = k + 1 + lane; i < n; i += 32) p[(int64_t)i * n + k] *= rl;
        __syncwarp();
        for (int j = k + 1; j < n; ++j) {
            const double ljk = p[(int64_t)j * n + k];
            for (int i = j + lane; i < n; i += 32) p[(int64_t)i * n + j] -= p[(int64_t)i * n + k] * ljk;
        }
        __syncwarp();
    }
    if (lane == 0) info[bi] = inf;
}

// Dense blocks with n > 1024: one CTA of 256 threads per block, right-looking
// blocked Cholesky in FP64 with panels of 32 columns.  Per panel: warp 0
// factors the 32 x 32 diagonal block in shared memory; the rows below solve
// against it (forward substitution, 64 rows at a time staged in shared
// memory); the trailing lower triangle takes the rank-32 update in 64 x 64
// tiles, each thread a 4 x 4 sub-tile.  The matrix stays in global memory
// (row-major n x n at the block's offset; the lower triangle is read and
// written).  info = first non-positive pivot row + 1, or 0.
constexpr int kDenseNB = 32, kDenseT = 64;

__global__ void __launch_bounds__(256) k_factor_dense_cta(int nitems, const int32_t *__restrict__ items,
                                                          const BlockDesc *__restrict__ blocks,
                                                          double *__restrict__ out, int dense_storage,
                                                          int32_t *__restrict__ info) {
    __shared__ double sd[kDenseNB][kDenseNB + 1];
    __shared__ double pa[kDenseT][kDenseNB + 1], pb[kDenseT][kDenseNB + 1];
    __shared__ int s_inf;
    if ((int)blockIdx.x >= nitems) return;
    const int bi = items[blockIdx.x];
    const BlockDesc bd = blocks[bi];
    const int n = bd.n;
    double *A = out + (dense_storage ? bd.off_dense : bd.off_pband);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_inf = 0;
    __syncthreads();
    for (int k0 = 0; k0 < n; k0 += kDenseNB) {
        const int nb = min(kDenseNB, n - k0);
        // (1) diagonal block
        for (int e = tid; e < kDenseNB * kDenseNB; e += 256) {
            const int r = e / kDenseNB, c = e % kDenseNB;
            sd[r][c] = (r < nb && c <= r) ? A[(int64_t)(k0 + r) * n + k0 + c] : 0.0;
        }
        __syncthreads();
        if (warp == 0) {
            for (int k = 0; k < nb; ++k) {
                const double dkk = sd[k][k];
                if (!(dkk > 0.0)) {  // uniform across the warp
                    if (lane == 0) s_inf = k0 + k + 1;
                    break;
                }
                const double lkk = sqrt(dkk), rl = 1.0 / lkk;
                __syncwarp();
                if (lane == 0) sd[k][k] = lkk;
                if (lane > k && lane < nb) sd[lane][k] *= rl;
                __syncwarp();
                for (int j = k + 1; j < nb; ++j) {
                    const double ljk = sd[j][k];
                    if (lane >= j && lane < nb) sd[lane][j] -= sd[lane][k] * ljk;
                }
                __syncwarp();
            }
        }
        __syncthreads();
        if (s_inf) break;  // uniform: read after the barrier
        for (int e = tid; e < nb * nb; e += 256) {
            const int r = e / nb, c = e % nb;
            if (c <= r) A[(int64_t)(k0 + r) * n + k0 + c] = sd[r][c];
        }
        const int r0 = k0 + nb;
        // (2) panel: L[i][k0..] = A[i][k0..] L_kk^-T, 64 rows at a time
        for (int i0 = r0; i0 < n; i0 += kDenseT) {
            const int ni = min(kDenseT, n - i0);
            __syncthreads();
            for (int e = tid; e < kDenseT * kDenseNB; e += 256) {
                const int r = e / kDenseNB, c = e % kDenseNB;
                pa[r][c] = (r < ni && c < nb) ? A[(int64_t)(i0 + r) * n + k0 + c] : 0.0;
            }
            __syncthreads();
            if (tid < ni) {
                for (int c = 0; c < nb; ++c) {
                    double x = pa[tid][c];
                    for (int t = 0; t < c; ++t) x -= pa[tid][t] * sd[c][t];
                    pa[tid][c] = x / sd[c][c];
                }
            }
            __syncthreads();
            for (int e = tid; e < kDenseT * kDenseNB; e += 256) {
                const int r = e / kDenseNB, c = e % kDenseNB;
                if (r < ni && c < nb) A[(int64_t)(i0 + r) * n + k0 + c] = pa[r][c];
            }
        }
        // (3) trailing update of the lower triangle, 64 x 64 tiles
        const int ty = tid / 16, tx = tid % 16;  // rows 4 ty .. 4 ty + 3, columns 4 tx .. 4 tx + 3
        for (int i0 = r0; i0 < n; i0 += kDenseT) {
            for (int j0 = r0; j0 <= i0; j0 += kDenseT) {
                __syncthreads();
                for (int e = tid; e < kDenseT * kDenseNB; e += 256) {
                    const int r = e / kDenseNB, c = e % kDenseNB;
                    pa[r][c] = (i0 + r < n && c < nb) ? A[(int64_t)(i0 + r) * n + k0 + c] : 0.0;
                    pb[r][c] = (j0 + r < n && c < nb) ? A[(int64_t)(j0 + r) * n + k0 + c] : 0.0;
                }
                __syncthreads();
                double acc[4][4];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
                for (int c = 0; c < nb; ++c) {
                    double xa[4], xb[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        xa[a] = pa[4 * ty + a][c];
                        xb[a] = pb[4 * tx + a][c];
                    }
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] = fma(xa[a], xb[b], acc[a][b]);
                }
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int i = i0 + 4 * ty + a;
                    if (i >= n) continue;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int j = j0 + 4 * tx + b;
                        if (j <= i) A[(int64_t)i * n + j] -= acc[a][b];
                    }
                }
            }
        }
        __syncthreads();
    }
    if (tid == 0) info[bi] = s_inf;
}

void launch_factor_wide_dense(sympix_plan_t pl, int precision, bool dense, double *blocks, int32_t *info,
                              cudaStream_t st) {
    const int nw = (int)pl->factor_items[5].size();
    if (nw) {
        const size_t smem = (size_t)((kWideMax + 1) * (kWideMax + 1) + kWideMax * (kWideMax + 1) +
                                     kWideMax * kWideMax + 3 * (kWideMax + 1)) *
                            sizeof(double);
        const int32_t *it = pl->d_factor_items[5].p;
        // FP32 arithmetic for the FP32 factor (near-degenerate blocks then
        // rescued in FP64), FP64 otherwise
        if (precision == SYMPIX_PREC_FP32 && !dense) {
            auto kf = k_factor_wide<float, false>;
            auto kd = dense ? k_factor_wide<double, true> : k_factor_wide<double, false>;
            cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaFuncSetAttribute(kd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            kf<<<nw, 256, smem, st>>>(nw, it, pl->d_blocks.p, blocks, info, 0, (float)pl->fp32_pivot_floor,
                                      pl->d_shadow.p);
            kd<<<nw, 256, smem, st>>>(nw, it, pl->d_blocks.p, blocks, info, 1, 0.0f, nullptr);
        } else {
            auto kd = dense ? k_factor_wide<double, true> : k_factor_wide<double, false>;
            cudaFuncSetAttribute(kd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            kd<<<nw, 256, smem, st>>>(nw, it, pl->d_blocks.p, blocks, info, 0, 0.0f, nullptr);
        }
    }
    if (nw) trace_mark(pl, st, "k_factor_wide");
    const int nd = (int)pl->factor_items[3].size(), ns = (int)pl->factor_items[4].size();
    if (nd)
        k_factor_dense<<<(unsigned)((nd * 32 + 127) / 128), 128, 0, st>>>(nd, pl->d_factor_items[3].p, pl->d_blocks.p,
                                                                        blocks, dense ? 1 : 0, info);
    if (nd) trace_mark(pl, st, "k_factor_dense");
    if (ns)
        k_factor_dense_cta<<<(unsigned)ns, 256, 0, st>>>(ns, pl->d_factor_items[4].p, pl->d_blocks.p, blocks,
                                                         dense ? 1 : 0, info);
    if (ns) trace_mark(pl, st, "k_factor_dense_cta");
}

}  // namespace sympix
