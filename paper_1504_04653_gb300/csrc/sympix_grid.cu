// SymPix grid construction on the device (Sec. 2 of the paper):
//   ring colatitudes at the roots of P_{N_rings}(cos theta) (Sec. 1, 2.1),
//   per-ring pixel counts (greedy per-ring layout, or the dynamic programme
//   of Fig. Optimal-SymPix-Grid, Sec. 2.5),
//   pixel numbering with interleaved hemispheres (Sec. 2.4).
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>

#include "sympix_internal.cuh"

namespace sympix {

static thread_local std::string g_last_error;

int set_error(int code, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_error(cudaError_t e, const char *what) {
    (void)cudaGetLastError();
    return set_error(SYMPIX_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// Ring colatitudes
// ---------------------------------------------------------------------------

// rinv[l] = 1 / (l + 1), l = 0..N-1: turns the recurrence's divisions into
// products inside the Newton loop.
__global__ void k_recip(int N, double *rinv) {
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l < N) rinv[l] = 1.0 / (double)(l + 1);
}

// One thread per northern root theta_j, j < N/2.  Newton in theta on
// f = P_N(cos theta) with f' = -N (P_{N-1} - x P_N) / sin theta; P_N at
// x = 1 - u, u = 2 sin^2(theta/2), advanced on the differences
// D_l = P_l - P_{l-1} so that polar roots keep their relative accuracy.
__global__ void k_gl_theta(int N, const double *__restrict__ rinv, double *__restrict__ theta) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    int half = N / 2;
    if (j >= half) return;
    double t = kPi * ((double)j + 0.75) / ((double)N + 0.5);
    for (int it = 0; it < 60; ++it) {
        double sh = sin(0.5 * t);
        double u = 2.0 * sh * sh;
        double pm1 = 1.0, p = 1.0 - u, dlt = -u;
        for (int l = 1; l < N; ++l) {
            double fl = (double)l;
            dlt = (fl * dlt - (fl + fl + 1.0) * u * p) * rinv[l];
            pm1 = p;
            p += dlt;
        }
        double step = p * sin(t) / ((double)N * (pm1 - cos(t) * p));
        t += step;
        if (fabs(step) <= 1e-16 * t) break;
    }
    theta[j] = t;
    theta[N - 1 - j] = kPi - t;
    if ((N & 1) && j == 0) theta[half] = 0.5 * kPi;
}

// ---------------------------------------------------------------------------
// Ring counts
// ---------------------------------------------------------------------------

__device__ bool smooth235(long v) {
    if (v <= 0) return false;
    while (v % 2 == 0) v /= 2;
    while (v % 3 == 0) v /= 3;
    while (v % 5 == 0) v /= 5;
    return v == 1;
}

__device__ long next_smooth235(long v) {
    if (v < 1) v = 1;
    while (!smooth235(v)) ++v;
    return v;
}

// Greedy per-ring counts (one thread): equator-most northern ring gets the
// least 5-smooth count >= max(8, ceil(2 (lmax+1) sin theta)); toward the
// pole each ring takes the least n_{j+1} / x, x in {1, 6/5, 5/4, 4/3, 2, 3},
// that is an integer, >= 8 and >= 2 (lmax+1) sin theta_j; south mirrors.
__global__ void k_layout_greedy(int lmax, const double *__restrict__ theta, int32_t *__restrict__ nring) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int N = lmax + 1;
    const int e = (N & 1) ? (N - 1) / 2 : N / 2 - 1;
    const double scale = 2.0 * (double)(lmax + 1);
    long ce = (long)ceil(scale * sin(theta[e]));
    nring[e] = (int32_t)next_smooth235(ce < 8 ? 8 : ce);
    const int dn[5] = {6, 5, 4, 2, 3};
    const int nm[5] = {5, 4, 3, 1, 1};
    for (int j = e - 1; j >= 0; --j) {
        const double t = scale * sin(theta[j]);
        const long prev = nring[j + 1];
        long best = prev;
        for (int x = 0; x < 5; ++x) {
            if ((prev * nm[x]) % dn[x]) continue;
            long c = prev * nm[x] / dn[x];
            if (c >= 8 && (double)c >= t && c < best) best = c;
        }
        nring[j] = (int32_t)best;
    }
    for (int j = 0; j <= e; ++j) nring[N - 1 - j] = nring[j];
}

// alpha_i = ceil((2 m + 1) / k) with m the least order that Eq.
// polar-optimization omits at the equator-side ring of band i.
__global__ void k_dp_alpha(int lmax, int k, int nb, double thr, const double *__restrict__ theta,
                           int32_t *__restrict__ alpha) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    const double th = theta[i * k + k - 1];
    const double c = cos(th), s = (double)lmax * sin(th);
    int m = lmax + 1;
    for (int mm = 0; mm <= lmax; ++mm) {
        double a = (double)mm * (double)mm - 2.0 * (double)mm * c;
        if (a >= 0.0 && sqrt(a) - s > thr) {
            m = mm;
            break;
        }
    }
    alpha[i] = (2 * m + 1 + k - 1) / k;
}

// The dynamic programme of Fig. Optimal-SymPix-Grid in one CTA.  State
// (band i, tiles t) holds key = cost << 20 | t_prev; atomicMin keeps the
// least cost and, among equal costs, the least t_prev.  The start state is
// (0, T0) with t_prev = T0, so that band 1 may differ from band 0.
__global__ void k_dp_layout(int nb, int W, const int32_t *__restrict__ alpha,
                            unsigned long long *__restrict__ key, int32_t *__restrict__ T,
                            int32_t *__restrict__ status) {
    const unsigned long long NONE = ~0ull;
    const unsigned long long MASK = (1ull << 20) - 1;
    if (threadIdx.x == 0) {
        long t0 = next_smooth235(alpha[0]);
        unsigned long long c0 = (unsigned long long)((t0 - alpha[0]) * (t0 - alpha[0]));
        key[t0] = (c0 << 20) | (unsigned long long)t0;
    }
    __syncthreads();
    const int num[6] = {3, 2, 1, 4, 5, 6};
    const int den[6] = {1, 1, 1, 3, 4, 5};
    for (int i = 1; i < nb; ++i) {
        const int a = alpha[i];
        for (int tp = threadIdx.x + 1; tp < W; tp += blockDim.x) {
            unsigned long long kp = key[(size_t)(i - 1) * W + tp];
            if (kp == NONE) continue;
            const unsigned long long cprev = kp >> 20;
            const int pprev = (int)(kp & MASK);
            for (int x = 0; x < 6; ++x) {
                if ((tp * num[x]) % den[x]) continue;
                const int t = tp * num[x] / den[x];
                if (t < a || t > 3 * a || t >= W) continue;
                if (!(pprev == tp || num[x] == den[x])) continue;
                const unsigned long long c = cprev + (unsigned long long)((long)(a - t) * (a - t));
                atomicMin(&key[(size_t)i * W + t], (c << 20) | (unsigned long long)tp);
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int best = -1;
        unsigned long long bc = NONE;
        for (int t = 1; t < W; ++t) {
            unsigned long long kk = key[(size_t)(nb - 1) * W + t];
            if (kk != NONE && (kk >> 20) < bc) {
                bc = kk >> 20;
                best = t;
            }
        }
        if (best < 0) {
            *status = 1;
            return;
        }
        T[nb - 1] = best;
        for (int i = nb - 2; i >= 0; --i) T[i] = (int32_t)(key[(size_t)(i + 1) * W + T[i + 1]] & MASK);
        *status = 0;
    }
}

__global__ void k_dp_expand(int N, int k, int nb, const int32_t *__restrict__ T, int32_t *__restrict__ nring) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N / 2) return;
    int v = k * T[j / k];
    nring[j] = v;
    nring[N - 1 - j] = v;
}

// Pixel numbering (Sec. 2.4), one thread: bands north 0, south 0, north 1,
// ...; inside a band pixel c of its r-th ring (counted from the band's pole)
// is band_start + c k + r; with k = 1 an odd equatorial ring comes last.
__global__ void k_ordering(int N, int k, const int32_t *__restrict__ nring, int64_t *__restrict__ off,
                           int32_t *__restrict__ stride, int64_t *__restrict__ npix) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int nb = (k == 1) ? N / 2 : N / (2 * k);
    int64_t pos = 0;
    for (int i = 0; i < nb; ++i) {
        for (int r = 0; r < k; ++r) {
            off[i * k + r] = pos + r;
            stride[i * k + r] = k;
        }
        pos += (int64_t)nring[i * k] * k;
        for (int r = 0; r < k; ++r) {
            off[N - 1 - i * k - r] = pos + r;
            stride[N - 1 - i * k - r] = k;
        }
        pos += (int64_t)nring[N - 1 - i * k] * k;
    }
    if (k == 1 && (N & 1)) {
        off[N / 2] = pos;
        stride[N / 2] = 1;
        pos += nring[N / 2];
    }
    *npix = pos;
}

}  // namespace sympix

using namespace sympix;

extern "C" const char *sympix_last_error(void) { return g_last_error.c_str(); }

extern "C" const char *sympix_version(void) { return "sympix-gb300 0.1 (sm_103a)"; }

extern "C" int sympix_grid(int lmax, int k, int layout, double polar_thr, sympix_grid_t *out) {
    if (!out) return set_error(SYMPIX_EINVAL, "sympix_grid: out is NULL");
    *out = nullptr;
    if (lmax < 1 || lmax > 16383) return set_error(SYMPIX_EINVAL, "sympix_grid: lmax %d out of [1, 16383]", lmax);
    if (layout == SYMPIX_LAYOUT_GREEDY) {
        if (k != 1) return set_error(SYMPIX_EINVAL, "sympix_grid: the greedy layout has k = 1 (got %d)", k);
    } else if (layout == SYMPIX_LAYOUT_DP) {
        if (k < 1 || k > 64) return set_error(SYMPIX_EINVAL, "sympix_grid: k %d out of [1, 64]", k);
    } else {
        return set_error(SYMPIX_EINVAL, "sympix_grid: unknown layout %d", layout);
    }
    int N = lmax + 1;
    if (layout == SYMPIX_LAYOUT_DP && N % (2 * k)) N += 2 * k - N % (2 * k);
    if (N < 2) return set_error(SYMPIX_EINVAL, "sympix_grid: need at least 2 rings");

    sympix_grid_s *g = new sympix_grid_s();
    g->lmax = lmax;
    g->k = k;
    g->layout = layout;
    g->nrings = N;
    int rc = SYMPIX_OK;
    DevBuf<double> rinv;
    DevBuf<int32_t> nring, stride, alpha, T, status;
    DevBuf<int64_t> off, npix;
    DevBuf<unsigned long long> key;
    auto fail = [&](int code) {
        delete g;
        return code;
    };
    if ((rc = g->d_theta.alloc(N)) || (rc = rinv.alloc(N)) || (rc = nring.alloc(N)) || (rc = stride.alloc(N)) ||
        (rc = off.alloc(N)) || (rc = npix.alloc(1)))
        return fail(rc);
    k_recip<<<(N + 255) / 256, 256>>>(N, rinv.p);
    k_gl_theta<<<(N / 2 + 127) / 128, 128>>>(N, rinv.p, g->d_theta.p);
    if (layout == SYMPIX_LAYOUT_GREEDY) {
        k_layout_greedy<<<1, 1>>>(lmax, g->d_theta.p, nring.p);
    } else {
        const int nb = N / (2 * k);
        if ((rc = alpha.alloc(nb)) || (rc = T.alloc(nb)) || (rc = status.alloc(1))) return fail(rc);
        k_dp_alpha<<<(nb + 127) / 128, 128>>>(lmax, k, nb, polar_thr < 0.0 ? fmax(100.0, lmax / 100.0) : polar_thr,
                                              g->d_theta.p, alpha.p);
        std::vector<int32_t> ha(nb);
        cudaError_t e = cudaMemcpy(ha.data(), alpha.p, nb * sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail(cuda_error(e, "sympix_grid: alpha"));
        int amax = *std::max_element(ha.begin(), ha.end());
        long t0 = ha[0];
        auto smooth = [](long v) {
            for (int f : {2, 3, 5})
                while (v % f == 0) v /= f;
            return v == 1;
        };
        while (!smooth(t0)) ++t0;
        int W = (int)std::max<long>(3L * amax, t0) + 1;
        if ((rc = key.alloc((size_t)nb * W))) return fail(rc);
        e = cudaMemset(key.p, 0xFF, (size_t)nb * W * sizeof(unsigned long long));
        if (e != cudaSuccess) return fail(cuda_error(e, "sympix_grid: memset"));
        k_dp_layout<<<1, 1024>>>(nb, W, alpha.p, key.p, T.p, status.p);
        int32_t st = 1;
        e = cudaMemcpy(&st, status.p, sizeof st, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail(cuda_error(e, "sympix_grid: dp layout"));
        if (st) return fail(set_error(SYMPIX_EINVAL, "sympix_grid: no DP layout satisfies the constraints"));
        k_dp_expand<<<(N / 2 + 127) / 128, 128>>>(N, k, nb, T.p, nring.p);
    }
    k_ordering<<<1, 1>>>(N, k, nring.p, off.p, stride.p, npix.p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(cuda_error(e, "sympix_grid: launch"));
    g->theta.resize(N);
    g->nring.resize(N);
    g->stride.resize(N);
    g->offset.resize(N);
    if ((e = cudaMemcpy(g->theta.data(), g->d_theta.p, N * sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(g->nring.data(), nring.p, N * sizeof(int32_t), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(g->stride.data(), stride.p, N * sizeof(int32_t), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(g->offset.data(), off.p, N * sizeof(int64_t), cudaMemcpyDeviceToHost)) != cudaSuccess ||
        (e = cudaMemcpy(&g->npix, npix.p, sizeof(int64_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return fail(cuda_error(e, "sympix_grid: copy back"));
    g->nbands = (k == 1) ? N : N / k;
    g->max_ring = *std::max_element(g->nring.begin(), g->nring.end());
    *out = g;
    return SYMPIX_OK;
}

extern "C" int sympix_grid_describe(sympix_grid_t g, sympix_grid_desc *d) {
    if (!g || !d) return set_error(SYMPIX_EINVAL, "sympix_grid_describe: NULL argument");
    d->lmax = g->lmax;
    d->k = g->k;
    d->layout = g->layout;
    d->nrings = g->nrings;
    d->nbands = g->nbands;
    d->max_ring = g->max_ring;
    d->npix = g->npix;
    return SYMPIX_OK;
}

extern "C" int sympix_grid_copy(sympix_grid_t g, double *theta, int32_t *nring, int64_t *ring_offset,
                                int32_t *ring_stride) {
    if (!g) return set_error(SYMPIX_EINVAL, "sympix_grid_copy: NULL grid");
    if (theta) std::copy(g->theta.begin(), g->theta.end(), theta);
    if (nring) std::copy(g->nring.begin(), g->nring.end(), nring);
    if (ring_offset) std::copy(g->offset.begin(), g->offset.end(), ring_offset);
    if (ring_stride) std::copy(g->stride.begin(), g->stride.end(), ring_stride);
    return SYMPIX_OK;
}

extern "C" void sympix_grid_free(sympix_grid_t g) { delete g; }
