// Kernel tables: b(x) = sum_{l=0}^{lmax} (2l+1)/(4 pi) b_l P_l(x) (Eq.
// addition-theorem) and d(x) likewise, at every symmetry-class slot, in FP64.
//
// x is carried as u = 1 - x (exact haversine form from the plan).  P_l is
// advanced on its scaled differences E_l = l (P_l - P_{l-1}):
//   E_{l+1} = E_l - (2l+1) u P_l,  P_{l+1} = P_l + E_{l+1} / (l+1),
// which is the three-term recurrence (l+1) P_{l+1} = (2l+1) x P_l - l P_{l-1}
// rearranged for x near 1, where the kernel is steep (d b / d x ~ b / sigma^2)
// and rounding x itself would cost ~1e-10.  One step is a product and three
// fused multiply-adds on the FP64 pipe, the slowest pipe this kernel uses.
// The coefficients (-(2l+1), 1/(l+1)) and the scaled c'_l = (2l+1) c_l / (4 pi)
// are staged once per launch in global memory and read as warp-uniform loads.
#include "sympix_internal.cuh"

namespace sympix {

__global__ void k_table_coeffs(int lmax, int nops, const double *__restrict__ bl, const double *__restrict__ dl,
                               double *__restrict__ rec, double *__restrict__ cb, double *__restrict__ cd) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int L1 = lmax + 1;
    if (i < L1) {
        double l = (double)i;
        rec[2 * i] = -(2.0 * l + 1.0);
        rec[2 * i + 1] = 1.0 / (l + 1.0);
    }
    if (i < nops * L1) {
        const double f = (2.0 * (double)(i % L1) + 1.0) / (4.0 * kPi);
        cb[i] = f * bl[i];
        cd[i] = f * dl[i];
    }
}

// kTableSpt slots per thread, blockDim.x (the plan's table_cta: 32, 64 or
// 128) threads per CTA; the same-ring slots also get d.  nops operators are
// summed from one pass of the recurrence.  The kernel is bound by each SM's
// FP64 pipe, so what matters is an even spread: small CTAs give every SM
// nearly the same number of slots.
constexpr int kTableSpt = 1;

template <int NOPS>
__global__ void __launch_bounds__(128) k_table(int64_t nslots, int nops_total, int op0, int lmax,
                                               const double *__restrict__ slot_u,
                                               const int32_t *__restrict__ slot_pair,
                                               const CanonPair *__restrict__ pairs,
                                               const double *__restrict__ rec, const double *__restrict__ cb,
                                               const double *__restrict__ cd, double *__restrict__ tb,
                                               double *__restrict__ td, float *__restrict__ tb32,
                                               float *__restrict__ tblo, float *__restrict__ td32,
                                               float *__restrict__ tdlo, int all_d) {
    constexpr int J = kTableSpt;
    const int L1 = lmax + 1;
    const int nops = min(NOPS, nops_total - op0);
    int64_t s[J];
    bool ok[J], same[J];
    double u[J], p[J], dlt[J], sb[J][NOPS], sd[J][NOPS];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        s[j] = ((int64_t)blockIdx.x * J + j) * blockDim.x + threadIdx.x;
        ok[j] = s[j] < nslots;
        u[j] = ok[j] ? slot_u[s[j]] : 0.0;
        // d at the same-ring classes (the diagonal blocks), or at every class
        // once blocks between rings are planned
        same[j] = ok[j] && (all_d || pairs[slot_pair[s[j]]].a == pairs[slot_pair[s[j]]].b);
        p[j] = 1.0;
        dlt[j] = -u[j];
#pragma unroll
        for (int o = 0; o < NOPS; ++o) {
            sb[j][o] = 0.0;
            sd[j][o] = 0.0;
            if (o < nops) {
                sb[j][o] = cb[(op0 + o) * L1];
                if (same[j]) sd[j][o] = cd[(op0 + o) * L1];
            }
        }
    }
    if (lmax >= 1) {
#pragma unroll
        for (int j = 0; j < J; ++j) {
            p[j] = 1.0 - u[j];
#pragma unroll
            for (int o = 0; o < NOPS; ++o)
                if (o < nops) {
                    sb[j][o] = fma(cb[(op0 + o) * L1 + 1], p[j], sb[j][o]);
                    if (same[j]) sd[j][o] = fma(cd[(op0 + o) * L1 + 1], p[j], sd[j][o]);
                }
        }
    }
    // the recurrence; a warp none of whose slots needs d (the plan puts the
    // same-ring slots first) leaves d's multiply-adds out altogether
    auto recur = [&](auto HASDc) {
        constexpr bool HASD = decltype(HASDc)::value;
        for (int l = 1; l < lmax; ++l) {  // dlt = E_l on entry (E_1 = -u)
            const double a = rec[2 * l], r = rec[2 * l + 1];
#pragma unroll
            for (int j = 0; j < J; ++j) {
                dlt[j] = fma(a, u[j] * p[j], dlt[j]);
                p[j] = fma(dlt[j], r, p[j]);
            }
#pragma unroll
            for (int o = 0; o < NOPS; ++o)
                if (o < nops) {
                    const double c = cb[(op0 + o) * L1 + l + 1];
#pragma unroll
                    for (int j = 0; j < J; ++j) sb[j][o] = fma(c, p[j], sb[j][o]);
                    if constexpr (HASD) {
                        const double e = cd[(op0 + o) * L1 + l + 1];
#pragma unroll
                        for (int j = 0; j < J; ++j)
                            if (same[j]) sd[j][o] = fma(e, p[j], sd[j][o]);
                    }
                }
        }
    };
    bool anyd = false;
#pragma unroll
    for (int j = 0; j < J; ++j) anyd |= same[j];
    if (__any_sync(0xffffffffu, anyd))
        recur(std::true_type{});
    else
        recur(std::false_type{});
#pragma unroll
    for (int j = 0; j < J; ++j) {
        if (!ok[j]) continue;
#pragma unroll
        for (int o = 0; o < NOPS; ++o)
            if (o < nops) {
                const int64_t idx = (int64_t)(op0 + o) * nslots + s[j];
                tb[idx] = sb[j][o];
                td[idx] = same[j] ? sd[j][o] : 0.0;
                const float hi = (float)sb[j][o];
                tb32[idx] = hi;
                tblo[idx] = (float)(sb[j][o] - (double)hi);
                const double dv = same[j] ? sd[j][o] : 0.0;
                const float dh = (float)dv;
                td32[idx] = dh;
                tdlo[idx] = (float)(dv - (double)dh);
            }
    }
}

// The launches of one kernel-table call with the coefficient staging at
// `rec` (2 (lmax+1) (nops+1) doubles): the coefficients, then the table in
// chunks of 8, 4, 2 or 1 operators sharing one recurrence, with a trace
// mark after each.  Both entry points run exactly this sequence.
static int launch_table(sympix_plan_t pl, const double *bl, const double *dl, double *rec, cudaStream_t st,
                        const char *who) {
    const int lmax = pl->grid->lmax;
    const size_t L1 = (size_t)lmax + 1;
    double *cb = rec + 2 * L1;
    double *cd = cb + (size_t)pl->nops * L1;
    const int tot = pl->nops * (int)L1;
    trace_mark(pl, st, nullptr);
    // every staging entry read below is written first by k_table_coeffs
    k_table_coeffs<<<(tot + 255) / 256, 256, 0, st>>>(lmax, pl->nops, bl, dl, rec, cb, cd);
    trace_mark(pl, st, "k_table_coeffs");
    if (pl->nslots > 0) {
        const int cta = pl->table_cta;
        const unsigned grid = (unsigned)((pl->nslots + cta * kTableSpt - 1) / (cta * kTableSpt));
        for (int op0 = 0; op0 < pl->nops;) {
            const int left = pl->nops - op0;
            const int chunk = left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
#define SPX_TABLE(NO)                                                                                              \
    k_table<NO><<<grid, cta, 0, st>>>(pl->nslots, pl->nops, op0, lmax, pl->d_slot_u.p, pl->d_slot_pair.p,          \
                                      pl->d_pairs.p, rec, cb, cd, pl->d_tab_b.p, pl->d_tab_d.p, pl->d_tab_b32.p, \
                                      pl->d_tab_blo.p, pl->d_tab_d32.p, pl->d_tab_dlo.p, pl->all_d ? 1 : 0)
            if (chunk == 8)
                SPX_TABLE(8);
            else if (chunk == 4)
                SPX_TABLE(4);
            else if (chunk == 2)
                SPX_TABLE(2);
            else
                SPX_TABLE(1);
#undef SPX_TABLE
            op0 += chunk;
        }
    }
    trace_mark(pl, st, "k_table");
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, who);
    pl->table_ready = true;
    pl->table_all_d = pl->all_d;
    return SYMPIX_OK;
}

}  // namespace sympix

using namespace sympix;

extern "C" int sympix_kernel_table(sympix_plan_t pl, const double *bl, const double *dl, void *stream) {
    if (!pl || !bl || !dl) return set_error(SYMPIX_EINVAL, "sympix_kernel_table: NULL argument");
    const size_t L1 = (size_t)pl->grid->lmax + 1;
    const size_t need = 2 * L1 + 2 * (size_t)pl->nops * L1;
    int rc;
    if (pl->d_rec.n < need) {
        if ((rc = pl->d_rec.alloc(need))) return rc;
    }
    return launch_table(pl, bl, dl, pl->d_rec.p, (cudaStream_t)stream, "sympix_kernel_table: launch");
}

extern "C" int sympix_table_copy(sympix_plan_t pl, int op, int ring, int rho, int count, double *b, double *d) {
    if (!pl || !b) return set_error(SYMPIX_EINVAL, "sympix_table_copy: NULL argument");
    if (pl->tiles) return set_error(SYMPIX_EUNSUPPORTED, "sympix_table_copy: ring blocks only (k = 1)");
    if (op < 0 || op >= pl->nops || ring < pl->ring0 || ring >= pl->ring1)
        return set_error(SYMPIX_EINVAL, "sympix_table_copy: (op %d, ring %d) not planned", op, ring);
    const BlockDesc &bd = pl->blocks[(size_t)op * (pl->ring1 - pl->ring0) + (ring - pl->ring0)];
    for (int e = 0; e < bd.npairs; ++e) {
        const PairEntry &pe = pl->entries[bd.pair0 + e];
        if (pe.rho != rho) continue;
        const int K = pe.mmax / 2 + 1;
        if (count > K) return set_error(SYMPIX_EINVAL, "sympix_table_copy: %d values requested, %d stored", count, K);
        SPX_CUDA(cudaMemcpy(b, pl->d_tab_b.p + (size_t)op * pl->nslots + pe.tab, count * sizeof(double),
                            cudaMemcpyDeviceToHost));
        if (d && rho == ring)
            SPX_CUDA(cudaMemcpy(d, pl->d_tab_d.p + (size_t)op * pl->nslots + pe.tab, count * sizeof(double),
                                cudaMemcpyDeviceToHost));
        return SYMPIX_OK;
    }
    return set_error(SYMPIX_EINVAL, "sympix_table_copy: ring %d does not couple to ring %d", rho, ring);
}

// ---------------------------------------------------------------------------
// Allocation-free variant of sympix_kernel_table.
//
// The coefficient staging of the kernel-table launch (recurrence
// coefficients and the scaled c'_l) normally lives in a buffer the library
// allocates on first use.  This variant keeps it in one file-scope device
// array instead, so the call itself allocates nothing.  The array is loaded
// with the module and stays resident on every GPU that loads the library
// until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

namespace sympix {

constexpr size_t kStaticTableScratch = 262144;  // doubles (2 MiB)
static __device__ __align__(256) double g_table_scratch[kStaticTableScratch];

}  // namespace sympix

extern "C" int sympix_kernel_table_static(sympix_plan_t pl, const double *bl, const double *dl, void *stream) {
    if (!pl || !bl || !dl) return set_error(SYMPIX_EINVAL, "sympix_kernel_table_static: NULL argument");
    const int lmax = pl->grid->lmax;
    const size_t L1 = (size_t)lmax + 1;
    const size_t need = 2 * L1 + 2 * (size_t)pl->nops * L1;
    if (need > kStaticTableScratch)
        return set_error(SYMPIX_EINVAL,
                         "sympix_kernel_table_static: needs %zu scratch doubles (2 (lmax+1) (nops+1)), "
                         "the static array holds %zu",
                         need, kStaticTableScratch);
    // Host code only sees a stand-in for the device array: fetch its device
    // address once per device, with that device current.
    static std::mutex mu;
    static double *addr[64] = {nullptr};
    int dev = 0;
    SPX_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(SYMPIX_EINVAL, "sympix_kernel_table_static: device %d", dev);
    double *scratch;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_table_scratch);
            if (e != cudaSuccess) return cuda_error(e, "sympix_kernel_table_static: cudaGetSymbolAddress");
            addr[dev] = (double *)p;
        }
        scratch = addr[dev];
    }
    return launch_table(pl, bl, dl, scratch, (cudaStream_t)stream, "sympix_kernel_table_static: launch");
}
