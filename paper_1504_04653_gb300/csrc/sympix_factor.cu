// Cholesky factorisation M = L L^T of every sampled block, FP64.
//
// A periodic-band block (half-width w, 2w+1 < n) couples only |i-j| <= w or
// |i-j| >= n-w.  With m = n - w its leading m x m part is a plain band
// matrix, so L11 keeps the band; the last w rows fill in completely.  The
// factor is computed in three phases:
//   1. L11 = chol(A11), band of width w, row by row;
//   2. L21 = A21 L11^-T by forward substitution along each border row;
//   3. L22 = chol(A22 - L21 L21^T).
// Work O(n w^2) instead of O(n^3).  Dense-format blocks (small or fully
// coupled rings) use the textbook left-looking algorithm.  The same
// band-and-border algorithm runs on DENSE storage, so a large ring stored
// densely still costs O(n w^2).
//
// A non-positive pivot stops the block and records info = row + 1.
#include "sympix_internal.cuh"

namespace sympix {

// Element access of one block in its storage.
struct PBandView {
    double *band;   // n x (w+1)
    double *bord;   // w x n
    int n, w, m;
    // A[i][j] (i >= j) before factorisation
    __device__ double a(int i, int j) const {
        const int d = i - j;
        if (d <= w) return band[(int64_t)i * (w + 1) + d];
        const int dw = j - i + n;  // wrapped: A[j][(j - dw) mod n]
        if (dw <= w) return band[(int64_t)j * (w + 1) + dw];
        return 0.0;
    }
    __device__ double &l_band(int i, int j) const { return band[(int64_t)i * (w + 1) + (i - j)]; }
    __device__ double &l_bord(int i, int j) const { return bord[(int64_t)(i - m) * n + j]; }
};

struct DenseView {
    double *p;
    int n, w, m;
    __device__ double a(int i, int j) const { return p[(int64_t)i * n + j]; }
    __device__ double &l_band(int i, int j) const { return p[(int64_t)i * n + j]; }
    __device__ double &l_bord(int i, int j) const { return p[(int64_t)i * n + j]; }
};

template <class View>
__device__ int factor_band_border(const View &v) {
    const int n = v.n, w = v.w, m = v.m;
    // phase 1: band rows 0..m-1
    for (int i = 0; i < m; ++i) {
        const int j0 = max(0, i - w);
        for (int j = j0; j <= i; ++j) {
            double s = v.a(i, j);
            for (int k = max(j0, j - w); k < j; ++k) s -= v.l_band(i, k) * v.l_band(j, k);
            if (j < i) {
                v.l_band(i, j) = s / v.l_band(j, j);
            } else {
                if (!(s > 0.0)) return i + 1;
                v.l_band(i, i) = sqrt(s);
            }
        }
    }
    // phase 2: border rows m..n-1 against the band columns 0..m-1
    for (int i = m; i < n; ++i) {
        for (int j = 0; j < m; ++j) {
            double s = v.a(i, j);
            for (int k = max(0, j - w); k < j; ++k) s -= v.l_bord(i, k) * v.l_band(j, k);
            v.l_bord(i, j) = s / v.l_band(j, j);
        }
    }
    // phase 3: the dense w x w corner
    for (int i = m; i < n; ++i) {
        for (int j = m; j <= i; ++j) {
            double s = v.a(i, j);
            for (int k = 0; k < j; ++k) s -= v.l_bord(i, k) * v.l_bord(j, k);
            if (j < i) {
                v.l_bord(i, j) = s / v.l_bord(j, j);
            } else {
                if (!(s > 0.0)) return i + 1;
                v.l_bord(i, i) = sqrt(s);
            }
        }
    }
    return 0;
}

// Textbook left-looking Cholesky on an n x n row-major block.
__device__ int factor_dense(double *p, int n) {
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = p[(int64_t)i * n + j];
            for (int k = 0; k < j; ++k) s -= p[(int64_t)i * n + k] * p[(int64_t)j * n + k];
            if (j < i) {
                p[(int64_t)i * n + j] = s / p[(int64_t)j * n + j];
            } else {
                if (!(s > 0.0)) return i + 1;
                p[(int64_t)i * n + i] = sqrt(s);
            }
        }
    }
    return 0;
}

// One thread per block, blocks taken in the plan's cost order so that the
// lanes of a warp carry blocks of similar size.
__global__ void k_factor(int nblocks, const int32_t *__restrict__ order, const BlockDesc *__restrict__ blocks,
                         double *__restrict__ out, int dense_storage, int32_t *__restrict__ info) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nblocks) return;
    const int b = order[t];
    const BlockDesc bd = blocks[b];
    int res;
    if (bd.format == SYMPIX_BLOCK_DENSE) {
        res = factor_dense(out + (dense_storage ? bd.off_dense : bd.off_pband), bd.n);
    } else if (dense_storage) {
        DenseView v{out + bd.off_dense, bd.n, bd.w, bd.n - bd.w};
        res = factor_band_border(v);
    } else {
        double *base = out + bd.off_pband;
        PBandView v{base, base + (int64_t)bd.n * (bd.w + 1), bd.n, bd.w, bd.n - bd.w};
        res = factor_band_border(v);
    }
    info[b] = res;
}

}  // namespace sympix

using namespace sympix;

extern "C" int sympix_factor_blocks(sympix_plan_t pl, int storage, double *blocks, int32_t *info, void *stream) {
    if (!pl || !blocks || !info) return set_error(SYMPIX_EINVAL, "sympix_factor_blocks: NULL argument");
    if (storage != SYMPIX_STORE_PBAND && storage != SYMPIX_STORE_DENSE)
        return set_error(SYMPIX_EINVAL, "sympix_factor_blocks: unknown storage %d", storage);
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = (int)pl->blocks.size();
    k_factor<<<(nb + 31) / 32, 32, 0, st>>>(nb, pl->d_factor_order.p, pl->d_blocks.p, blocks,
                                            storage == SYMPIX_STORE_DENSE ? 1 : 0, info);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "sympix_factor_blocks: launch");
    return SYMPIX_OK;
}
