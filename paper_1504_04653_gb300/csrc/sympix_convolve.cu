// Pixel-domain convolution g = B^ f (Eq. convolution-pixel):
//   g_q = sum over pixels p within r_s of b(n_q . n_p) f_p,
// with b from the plan's class tables (Eq. addition-theorem), so the kernel
// values come from the same symmetry-reduced slots as the blocks.  For a
// coupled ring pair (P, Q, mmax) pixel q of ring j meets the pixels p of ring
// rho with |z| <= mmax, z = (2q+1) Q - (2p+1) P: a contiguous arc, walked
// once, unless the support covers the whole ring (mmax >= P n_rho, half a
// turn), when every pixel is visited once with z reduced to (-half, half].
// One thread per output pixel, 128 pixels of one ring per CTA, every
// operator's map with its own kernel.
#include "sympix_sample_kernels.cuh"

namespace sympix {

template <int PREC>
__global__ void __launch_bounds__(128) k_convolve(const ConvItem *__restrict__ items,
                                                  const BlockDesc *__restrict__ blocks,
                                                  const PairEntry *__restrict__ entries, int64_t nslots,
                                                  int64_t npix, const double *__restrict__ tb,
                                                  const float *__restrict__ tb32, const float *__restrict__ tblo,
                                                  const double *__restrict__ f64, const float *__restrict__ f32,
                                                  const float *__restrict__ flo, double *__restrict__ g) {
    typedef Arith<PREC> A;
    typedef typename A::V V;
    const ConvItem it = items[blockIdx.x];
    const BlockDesc bd = blocks[it.block];
    const int q = it.q0 + (int)threadIdx.x;
    if (q >= bd.n) return;
    const int64_t tbase = (int64_t)bd.op * nslots, fbase = (int64_t)bd.op * npix;
    const double *F64 = f64 + fbase;
    const float *F32 = f32 + fbase, *FLO = flo + fbase;
    V acc = A::zero();
    for (int e = 0; e < bd.npairs; ++e) {
        const PairEntry pe = entries[bd.pair0 + e];
        const int P = pe.P, m = pe.mmax, par = pe.par, nr = pe.nrho;
        const int64_t tab = tbase + pe.tab;
        const int64_t Z = (int64_t)(2 * q + 1) * pe.Q;
        const int64_t half = (int64_t)P * nr;
        if (m >= half) {
            // z reduced to (-half, half] once, then moved by -2P per pixel
            const int64_t T2 = 2 * half;
            int64_t z = (Z - (int64_t)P) % T2;
            if (z > half) z -= T2;
            if (z <= -half) z += T2;
            for (int p = 0; p < nr; ++p) {
                if (z <= m && -z <= m) {
                    const int lv = (int)(((z < 0 ? -z : z) - par) >> 1);
                    acc = A::fma_(A::tab(tb, tb32, tblo, tab + lv),
                                  A::nval(F64, F32, FLO, pe.noff + (int64_t)p * pe.nstride), acc);
                }
                z -= 2 * (int64_t)P;
                if (z <= -half) z += T2;
            }
        } else {
            // one contiguous arc; table and map read through per-pair bases,
            // z stepped by -2P in 32-bit integers
            const double *T64 = tb + tab;
            const float *T32 = tb32 + tab, *TLO = tblo + tab;
            const double *M64 = F64 + pe.noff;
            const float *M32 = F32 + pe.noff, *MLO = FLO + pe.noff;
            const int ns = pe.nstride;
            if (P == 1 && pe.Q == 1 && ns == 1 && q - m / 2 >= 0 && q + m / 2 < nr) {
                // same pixel count, no wrap: p = q + s, table level |s|
                const int K = m / 2;
                for (int s = -K; s <= K; ++s)
                    acc = A::fma_(A::tab(T64, T32, TLO, s < 0 ? -s : s), A::nval(M64, M32, MLO, q + s), acc);
            } else {
                const int p_lo = ceil_div((int)(Z - m - P), 2 * P), p_hi = floor_div((int)(Z + m - P), 2 * P);
                int pm = p_lo % nr;
                if (pm < 0) pm += nr;
                int z = (int)(Z - (int64_t)(2 * p_lo + 1) * P);
                for (int p = p_lo; p <= p_hi; ++p) {
                    const int lv = ((z < 0 ? -z : z) - par) >> 1;
                    acc = A::fma_(A::tab(T64, T32, TLO, lv), A::nval(M64, M32, MLO, pm * ns), acc);
                    z -= 2 * P;
                    if (++pm == nr) pm = 0;
                }
            }
        }
    }
    g[fbase + it.goff + (int64_t)q * it.gstride] = A::to_double(acc);
}

}  // namespace sympix

using namespace sympix;

extern "C" int sympix_convolve(sympix_plan_t pl, const double *f, int precision, double *g, void *stream) {
    if (!pl || !f || !g) return set_error(SYMPIX_EINVAL, "sympix_convolve: NULL argument");
    if (pl->tiles) return set_error(SYMPIX_EUNSUPPORTED, "sympix_convolve: ring blocks only (k = 1)");
    if (precision < SYMPIX_PREC_FP64 || precision > SYMPIX_PREC_FP32X2)
        return set_error(SYMPIX_EINVAL, "sympix_convolve: unknown precision %d", precision);
    if (!pl->table_ready)
        return set_error(SYMPIX_EINVAL, "sympix_convolve: sympix_kernel_table has not been called");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t npix = pl->grid->npix, cnt = (int64_t)pl->nops * npix;
    trace_mark(pl, st, nullptr);
    if (precision != SYMPIX_PREC_FP64) {
        k_split_ninv<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(cnt, f, pl->d_ninv32.p, pl->d_ninvlo.p);
        trace_mark(pl, st, "k_split_ninv");
    }
    const unsigned ni = (unsigned)pl->items_conv.size();
    if (ni) {
#define SPX_CONV(PREC)                                                                                        \
    k_convolve<PREC><<<ni, 128, 0, st>>>(pl->d_items_conv.p, pl->d_blocks.p, pl->d_entries.p, pl->nslots, npix, \
                                         pl->d_tab_b.p, pl->d_tab_b32.p, pl->d_tab_blo.p, f, pl->d_ninv32.p,   \
                                         pl->d_ninvlo.p, g)
        if (precision == SYMPIX_PREC_FP64)
            SPX_CONV(0);
        else if (precision == SYMPIX_PREC_FP32)
            SPX_CONV(1);
        else
            SPX_CONV(2);
#undef SPX_CONV
        trace_mark(pl, st, "k_convolve");
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "sympix_convolve: launch");
    return SYMPIX_OK;
}
