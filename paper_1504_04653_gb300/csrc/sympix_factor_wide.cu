// Cholesky of wide bands (16 < w <= 64, a CTA per block) and of dense-format
// blocks (a warp per block up to n = 1024, a blocked CTA per block above),
// and their launcher.
#include "sympix_factor_kernels.cuh"

namespace sympix {

// ---------------------------------------------------------------------------
// Wide bands (16 < w <= 64): one CTA per block, the elimination state in
// registers.
//
// The active band window (rows k..k+w, each with its columns row-w..row) and
// the w border rows at columns k..k+w are stored by slot: row R and column C
// sit at slots R mod (w+1) and C mod (w+1), so moving the window to column
// k+1 only reuses the slot of row/column k for row/column k+1+w.  The
// 2w+1 entries of a column slot (w+1 band rows by row slot, then the w
// border rows) are split over G threads of kWideE consecutive entries each.
//
// One barrier per column.  Before the barrier of step k the group owning
// column slot k mod (w+1) has published its raw column a = A(., k) (after
// the updates of steps < k), 1/a_kk, sqrt(a_kk) and 1/sqrt(a_kk) to shared
// memory; after it every thread applies A(R, C) -= a_R a_C / a_kk to its
// entries (stale entries of eliminated columns take harmless garbage), the
// new band row k+1+w and border column k+1+w go into the freed slot, and
// the group of the next column publishes its column.  Every kWideKC columns
// the CTA writes the finished columns of L = a / sqrt(a_kk) out together,
// row by row.  Band rows and border columns arrive through a shared-memory
// ring filled by cp.async kWideD steps ahead (FP32: converted once by the
// thread that staged them).  After the band the corner
// S = A22 - L21 L21^T is formed from the stored L21 in 4 x 4 register tiles
// and factored in FP64 in shared memory.  T = double or float; the float
// version sends a block whose pivot falls below the floor to the FP64
// rescue.
// ---------------------------------------------------------------------------
constexpr int kWideD = 6;             // band rows staged ahead of the elimination
constexpr int kWideNR = kWideD + 1;   // staging ring slots
constexpr int kWideKC = 8;            // columns of L written out together
constexpr int kWideNB = kWideKC + 1;  // raw-column buffers
constexpr int kWideKS = 32;           // L21 columns per corner-update chunk

// FP32 verdict on a band pivot that failed the floor test (row1 = its row
// + 1): the FP32 pivot lies within about (w+1) 2^-24 of the original
// diagonal of the FP64 one (every earlier pivot having passed the floor), so
// a pivot at or below -1e-3 of the original diagonal is negative in FP64
// too and fails the block at the same row; anything else is left to the
// FP64 refactor.
constexpr float kWideDecisive = 1e-3f;
template <typename T>
__device__ __forceinline__ int wide_verdict(T d, T od, int row1) {
    if constexpr (sizeof(T) == 8)
        return row1;
    else
        return d <= T(-kWideDecisive) * od ? row1 : kRescue;
}

// Shared-memory layout of a wide CTA (byte offsets) for band width w and
// element size tsz.
struct WideLayout {
    int S, NV, LP;
    size_t la, piv, ring, ringt, corner, total;
};
__host__ __device__ inline size_t wide_al16(size_t x) { return (x + 15) / 16 * 16; }
__host__ __device__ inline WideLayout wide_layout(int w, int tsz) {
    WideLayout L;
    L.S = w + 1;
    L.NV = 2 * w + 1;
    L.LP = (L.NV + kWideE - 1) / kWideE * kWideE;
    size_t o = 0;
    L.la = o;  // kWideNB x LP raw columns
    o = wide_al16(o + (size_t)kWideNB * L.LP * tsz);
    L.piv = o;  // 1/a_kk, sqrt(a_kk), 1/sqrt(a_kk) per raw-column buffer
    o = wide_al16(o + 3 * (size_t)kWideNB * tsz);
    L.ring = o;  // kWideNR x LP staged FP64 rows
    o = wide_al16(o + (size_t)kWideNR * L.LP * sizeof(double));
    L.ringt = o;  // 2 x LP staged rows in T
    o = wide_al16(o + 2 * (size_t)L.LP * tsz);
    L.corner = o;  // L21 staging, then the w x w corner in FP64
    const size_t a = (size_t)w * w * sizeof(double), b = (size_t)w * (kWideKS + 1) * tsz;
    o = wide_al16(o + (a > b ? a : b));
    L.total = o;
    return L;
}

template <typename T>
__device__ __forceinline__ T wide_from(double x);
template <>
__device__ __forceinline__ double wide_from<double>(double x) { return x; }
template <>
__device__ __forceinline__ float wide_from<float>(double x) { return f64_to_f32_bits(x); }
__device__ __forceinline__ double wide_to(double x) { return x; }
__device__ __forceinline__ double wide_to(float x) { return f32_to_f64_bits(x); }

// kWideE consecutive entries from / to shared memory (16-byte aligned).
__device__ __forceinline__ void wide_lds(const double *p, double (&r)[kWideE]) {
#pragma unroll
    for (int q = 0; q < kWideE / 2; ++q) {
        const double2 v = reinterpret_cast<const double2 *>(p)[q];
        r[2 * q] = v.x;
        r[2 * q + 1] = v.y;
    }
}
__device__ __forceinline__ void wide_lds(const float *p, float (&r)[kWideE]) {
#pragma unroll
    for (int q = 0; q < kWideE / 4; ++q) {
        const float4 v = reinterpret_cast<const float4 *>(p)[q];
        r[4 * q] = v.x;
        r[4 * q + 1] = v.y;
        r[4 * q + 2] = v.z;
        r[4 * q + 3] = v.w;
    }
}
__device__ __forceinline__ void wide_sts(double *p, const double (&r)[kWideE]) {
#pragma unroll
    for (int q = 0; q < kWideE / 2; ++q) reinterpret_cast<double2 *>(p)[q] = make_double2(r[2 * q], r[2 * q + 1]);
}
__device__ __forceinline__ void wide_sts(float *p, const float (&r)[kWideE]) {
#pragma unroll
    for (int q = 0; q < kWideE / 4; ++q)
        reinterpret_cast<float4 *>(p)[q] = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
}

// x[e] = v / return x[e] for a run-time e in [LO, HI): a binary branch tree
// (the owning lanes of a warp share e), not a select per register.
template <int LO, int HI, typename T>
__device__ __forceinline__ void wide_set(T (&x)[kWideE], int e, T v) {
    if constexpr (HI - LO == 1) {
        x[LO] = v;
    } else {
        constexpr int MID = (LO + HI) / 2;
        if (e < MID)
            wide_set<LO, MID>(x, e, v);
        else
            wide_set<MID, HI>(x, e, v);
    }
}
template <int LO, int HI, typename T>
__device__ __forceinline__ T wide_get(const T (&x)[kWideE], int e) {
    if constexpr (HI - LO == 1) {
        return x[LO];
    } else {
        constexpr int MID = (LO + HI) / 2;
        return e < MID ? wide_get<LO, MID>(x, e) : wide_get<MID, HI>(x, e);
    }
}

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
    __device__ float get_b(int b, int j) const { return band[(int64_t)n * (w + 1) + (int64_t)b * n + j]; }
};

template <typename T, bool DENSE>
__global__ void __launch_bounds__(kWideMaxThreads)
    k_factor_wide(int nitems, const int32_t *__restrict__ items, const BlockDesc *__restrict__ blocks,
                  double *__restrict__ out, int32_t *__restrict__ info, int rescue, float floor,
                  float *__restrict__ shadow) {
    extern __shared__ __align__(16) unsigned char wsm[];
    __shared__ int s_fail;
    if ((int)blockIdx.x >= nitems) return;
    const int bi = items[blockIdx.x];
    if (rescue && info[bi] != kRescue) return;
    const BlockDesc bd = blocks[bi];
    typedef typename ViewOf<DENSE>::T View;
    const View v = ViewOf<DENSE>::make(out, bd);
    const int w = bd.w, n = bd.n, m = n - w;
    const WideLayout lay = wide_layout(w, (int)sizeof(T));
    const int S = lay.S, NV = lay.NV, LP = lay.LP, G = LP / kWideE;
    auto make_sink = [&]() {
        if constexpr (sizeof(T) == 4)
            return WideSink<T, View>{shadow + bd.off_pband, n, w};
        else
            return WideSink<T, View>{v};
    };
    const WideSink<T, View> sink = make_sink();
    T *la = reinterpret_cast<T *>(wsm + lay.la);
    T *pinv = reinterpret_cast<T *>(wsm + lay.piv), *plkk = pinv + kWideNB, *prs = plkk + kWideNB;
    double *ring = reinterpret_cast<double *>(wsm + lay.ring);
    T *ringt = reinterpret_cast<T *>(wsm + lay.ringt);
    double *csh = reinterpret_cast<double *>(wsm + lay.corner);
    const int tid = threadIdx.x, nt = blockDim.x, nthr = G * S;
    const int cs = tid / G, g = tid - cs * G, i0 = g * kWideE;
    const bool live = tid < nthr;
    const bool diag_owner = live && cs >= i0 && cs < i0 + kWideE;

    // A(r, r - d) of band row r and A(m + b, r) of border row b, w < r < m
    auto row_src = [&](int r, int d) -> const double * {
        if constexpr (DENSE)
            return v.p + (int64_t)r * n + (r - d);
        else
            return v.band + (int64_t)r * S + d;
    };
    auto bord_src = [&](int b, int r) -> const double * {
        if constexpr (DENSE) {
            return v.p + (int64_t)(m + b) * n + r;
        } else {
            const int d = m + b - r;  // r > w > b: no wrapped entry
            return d <= w ? v.band + (int64_t)(m + b) * S + d : nullptr;
        }
    };
    // the band row and border column entering the window at step kk
    auto stage = [&](int kk) {
        const int r = kk + 1 + w;
        if (tid < NV) {
            double *dst = ring + (kk % kWideNR) * LP + tid;
            const double *src = nullptr;
            if (r < m) src = tid < S ? row_src(r, tid) : bord_src(tid - S, r);
            if (src)
                cp_async8(dst, src);
            else
                *dst = 0.0;
        }
        cp_async_commit();
    };
    // the staged row of step kk in T (FP32: converted by the thread that
    // staged it, once its copy has landed)
    auto convert = [&](int kk) {
        if constexpr (sizeof(T) == 4)
            if (tid < NV) ringt[(kk & 1) * LP + tid] = wide_from<T>(ring[(kk % kWideNR) * LP + tid]);
    };
    // L columns [j0, j1) out of the raw-column buffers: band rows row by
    // row (consecutive threads on consecutive columns of one row), then the
    // border rows
    auto flush = [&](int j0, int j1) {
        const int nc = j1 - j0;
        const int nband = (nc + w) * nc, nall = nband + w * nc;
        for (int e = tid; e < nall; e += nt) {
            if (e < nband) {
                const int R = j0 + e / nc, j = j0 + e % nc, d = R - j;
                if (d < 0 || d > w || R >= m) continue;
                const int jb = j % kWideNB;
                sink.put_l(R, j, d == 0 ? plkk[jb] : la[jb * LP + R % S] * prs[jb]);
            } else {
                const int f = e - nband, b = f / nc, j = j0 + f % nc, jb = j % kWideNB;
                sink.put_b(b, j, la[jb * LP + S + b] * prs[jb]);
            }
        }
    };

    // window rows 0..w (row R's column at slot cs is cs, or cs - S < 0 before
    // the start) and border columns 0..w
    T x[kWideE];
    T od = T(0);  // original diagonal of the row in slot cs (diag owner)
#pragma unroll
    for (int e = 0; e < kWideE; ++e) {
        const int i = i0 + e;
        T val = T(0);
        if (live) {
            if (i < S) {
                const int C = cs <= i ? cs : cs - S;
                if (C >= 0) val = wide_from<T>(v.a(i, C));
            } else if (i < NV) {
                val = wide_from<T>(v.a(m + i - S, cs));
            }
        }
        x[e] = val;
        if (i == cs) od = val;
    }
    // column slot cs publishes column kn (after its updates) into buffer
    // nb; its diagonal owner tests the pivot
    auto publish = [&](int kn, int nb) {
        wide_sts(la + nb * LP + i0, x);
        if (diag_owner) {
            const T dn = wide_get<0, kWideE>(x, cs - i0);
            if (!(dn > T(floor) * od)) {
                s_fail = wide_verdict(dn, od, kn + 1);
            } else {
                const T lkk = sqrt(dn);
                pinv[nb] = T(1) / dn;
                plkk[nb] = lkk;
                prs[nb] = T(1) / lkk;
            }
        }
    };
    // padding of the staging rows stays zero
    for (int e = tid; e < kWideNR * LP; e += nt)
        if (e % LP >= NV) ring[e] = 0.0;
    for (int e = tid; e < 2 * LP; e += nt)
        if (e % LP >= NV) ringt[e] = T(0);
    for (int kk = 0; kk < kWideD; ++kk) stage(kk);
    if (tid == 0) s_fail = 0;
    __syncthreads();
    if (live && cs == 0) publish(0, 0);
    cp_async_wait<kWideD - 1>();
    convert(0);

    int ks = 0, rslot = 0, kb = 0, kflush = 0;
    for (int k = 0; k < m; ++k) {
        __syncthreads();  // column k, its pivot values and the staged row k are in place
        if (s_fail) break;
        const T *lk = la + kb * LP;
        int kb1 = kb + 1;
        if (kb1 == kWideNB) kb1 = 0;
        if (live) {
            // rank-1 update of this thread's entries
            const T t = lk[cs] * pinv[kb];
            T a[kWideE];
            wide_lds(lk + i0, a);
#pragma unroll
            for (int e = 0; e < kWideE; ++e) x[e] = fma(-a[e], t, x[e]);
            // column slot ks becomes column k+1+w: its border rows take the
            // staged column (its band entries are stale, the one of row slot
            // ks is set next); row slot ks of every column slot takes the
            // staged band row k+1+w
            const T *rg;
            if constexpr (sizeof(T) == 4)
                rg = ringt + (k & 1) * LP;
            else
                rg = ring + rslot * LP;
            if (cs == ks) wide_lds(rg + i0, x);
            if (ks >= i0 && ks < i0 + kWideE) {
                int dd = ks - cs;
                if (dd < 0) dd += S;
                const T val = rg[dd];
                wide_set<0, kWideE>(x, ks - i0, val);
                if (cs == ks) od = val;
            }
            int c1 = ks + 1;
            if (c1 == S) c1 = 0;
            if (cs == c1 && k + 1 < m) publish(k + 1, kb1);
        }
        if (k + 1 - kflush == kWideKC) {
            flush(kflush, k + 1);
            kflush = k + 1;
        }
        stage(k + kWideD);
        cp_async_wait<kWideD - 1>();
        convert(k + 1);
        if (++ks == S) ks = 0;
        if (++rslot == kWideNR) rslot = 0;
        kb = kb1;
    }
    cp_async_wait<0>();
    int fail = s_fail;  // set before the last barrier the loop passed, or 0
    if (!fail) {
        if (kflush < m) flush(kflush, m);
        // S = A22 - L21 L21^T from the stored L21, 4 x 4 tiles of the lower
        // triangle, L21 staged kWideKS columns at a time
        const int n4 = (w + 3) / 4, ntiles = n4 * (n4 + 1) / 2;
        int tb = -1, tc = 0;
        if (tid < ntiles) {
            tb = (int)((sqrtf(8.0f * tid + 1.0f) - 1.0f) * 0.5f);
            while (tb * (tb + 1) / 2 > tid) --tb;
            while ((tb + 1) * (tb + 2) / 2 <= tid) ++tb;
            tc = tid - tb * (tb + 1) / 2;
        }
        T acc[4][4];
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[p][q] = T(0);
        T *stg = reinterpret_cast<T *>(csh);  // w x (kWideKS + 1)
        for (int k0 = 0; k0 < m; k0 += kWideKS) {
            const int kn = min(kWideKS, m - k0);
            __syncthreads();  // L21 stored (first chunk) / the previous chunk used
            for (int e = tid; e < w * kWideKS; e += nt) {
                const int b = e / kWideKS, kk = e % kWideKS;
                stg[b * (kWideKS + 1) + kk] = kk < kn ? sink.get_b(b, k0 + kk) : T(0);
            }
            __syncthreads();
            if (tb >= 0) {
                for (int kk = 0; kk < kn; ++kk) {
                    T xa[4], xb[4];
#pragma unroll
                    for (int p = 0; p < 4; ++p) {
                        const int ra = 4 * tb + p, rb = 4 * tc + p;
                        xa[p] = ra < w ? stg[ra * (kWideKS + 1) + kk] : T(0);
                        xb[p] = rb < w ? stg[rb * (kWideKS + 1) + kk] : T(0);
                    }
#pragma unroll
                    for (int p = 0; p < 4; ++p)
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[p][q] = fma(xa[p], xb[q], acc[p][q]);
                }
            }
        }
        __syncthreads();  // staging done: the corner goes where it was
        if (tb >= 0) {
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int i = 4 * tb + p, j = 4 * tc + q;
                    if (i < w && j <= i) csh[i * w + j] = v.a(m + i, m + j) - wide_to(acc[p][q]);
                }
        }
        __syncthreads();
        // the corner, factored in FP64 in shared memory (right-looking)
        for (int j = 0; j < w; ++j) {
            if (tid == 0) {
                const double dj = csh[j * w + j];
                if (!(dj > 0.0))
                    s_fail = sizeof(T) == 4 ? kRescue : m + j + 1;  // the FP32 path lets FP64 decide
                else
                    csh[j * w + j] = sqrt(dj);
            }
            __syncthreads();
            if (s_fail) break;
            const double ljj = csh[j * w + j];
            for (int i = j + 1 + tid; i < w; i += nt) csh[i * w + j] /= ljj;
            __syncthreads();
            const int nr = w - j - 1;
            for (int e = tid; e < nr * nr; e += nt) {
                const int i = j + 1 + e / nr, c = j + 1 + e % nr;
                if (c <= i) csh[i * w + c] -= csh[i * w + j] * csh[c * w + j];
            }
            __syncthreads();
        }
        fail = s_fail;
        if (!fail)
            for (int e = tid; e < w * w; e += nt) {
                const int b = e / w, c = e % w;
                if (c <= b) sink.put_b(b, m + c, T(csh[e]));
            }
    }
    if (tid == 0) info[bi] = fail;
    if constexpr (sizeof(T) == 4) {
        // the block factored in FP32: copy L from the shadow, rows of the
        // band (d <= row) then the border (columns <= m + b)
        if (fail) return;
        __syncthreads();
        const float *sb = sink.band;
        double *ob = out + bd.off_pband;
        const int dq = nt / S, dr = nt % S;
        for (int row = tid / S, d = tid % S; row < m;) {
            if (d <= row) ob[(int64_t)row * S + d] = f32_to_f64_bits(sb[(int64_t)row * S + d]);
            row += dq;
            d += dr;
            if (d >= S) {
                d -= S;
                ++row;
            }
        }
        const int64_t bo = (int64_t)n * S;
        const int eq = nt / n, er = nt % n;
        for (int b = tid / n, j = tid % n; b < w;) {
            if (j <= m + b) ob[bo + (int64_t)b * n + j] = f32_to_f64_bits(sb[bo + (int64_t)b * n + j]);
            b += eq;
            j += er;
            if (j >= n) {
                j -= n;
                ++b;
            }
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
        // FP32 arithmetic for the FP32 factor (near-degenerate blocks then
        // rescued in FP64), FP64 otherwise; one launch per CTA size
        // the shared-memory limit is a property of the function, not of a
        // launch: set it once to the largest class's need, so that every
        // launch (and every node of a captured graph) stays within it
        auto launch = [&](auto kern, size_t tsz, int rescue, float floor) {
            size_t smax = 0;
            for (const WideClass &c : pl->wide_cls) smax = std::max(smax, wide_layout(c.wmax, (int)tsz).total);
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
            for (const WideClass &c : pl->wide_cls) {
                const size_t smem = wide_layout(c.wmax, (int)tsz).total;
                kern<<<(unsigned)c.count, (unsigned)c.threads, smem, st>>>(
                    c.count, pl->d_factor_items[5].p + c.begin, pl->d_blocks.p, blocks, info, rescue, floor,
                    pl->d_shadow.p);
            }
        };
        auto kd = dense ? k_factor_wide<double, true> : k_factor_wide<double, false>;
        if (precision == SYMPIX_PREC_FP32 && !dense) {
            launch(k_factor_wide<float, false>, sizeof(float), 0, (float)pl->fp32_pivot_floor);
            trace_mark(pl, st, "k_factor_wide");
            launch(kd, sizeof(double), 1, 0.0f);
            trace_mark(pl, st, "k_factor_wide_rescue");
        } else {
            launch(kd, sizeof(double), 0, 0.0f);
            trace_mark(pl, st, "k_factor_wide");
        }
    }
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
