/*
 * SymPix oracle: plain, slow, FP64 CPU restatement of what the preconditioner
 * block path computes (Seljebotn & Eriksen, "SymPix: a spherical grid for
 * efficient sampling of rotationally invariant operators").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so and is
 * called by the tests, by __graft_entry__.smoke() and by the cpu_baseline /
 * reference arm of bench.py.  The product path (the CUDA library) neither
 * links nor calls it, and it shares no code with that library.
 *
 * Every function states the passage it follows.  Nothing here exploits the
 * grid's symmetries: each kernel value is evaluated for its own pixel pair and
 * each B^T N^-1 B triple is summed explicitly.
 *
 * Readings where the paper is silent or inconsistent (each also listed in the
 * design notes):
 *   - rings sit at the roots of P_{N_rings}(cos theta) (Sec. 1, Sec. 2.1);
 *   - the kernel argument x = n1.n2 is carried as u = 1 - x, formed by the
 *     haversine identity, and P_l(1-u) is advanced by the three-term
 *     recurrence rewritten for the differences P_l - P_{l-1}; this is the
 *     same recurrence, arranged so that x close to 1 loses no digits;
 *   - the support of both D^ and B^ is gamma <= r_s for a radius r_s that the
 *     caller passes in (the truncation of Eq. f with one radius for both
 *     operators, Sec. 4.2);
 *   - a block is one ring (tile size k = 1); its entries are
 *     D^_qr + sum_p B^_pq N^-1_p B^_pr over pixels p of the same grid
 *     (Eq. Dhat with Y2 = Y1), or, for Y2 != Y1, over the pixels of an
 *     auxiliary grid carrying the noise of Eq. degrade;
 *   - in Eq. degrade, N_2^-1 is built from theta_2 as N^-1 is from theta:
 *     here both are the diagonal itself (N^-1 = diag(theta)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Legendre polynomials near x = 1                                           */
/* ------------------------------------------------------------------------ */

/* P_N(1-u) and P_{N-1}(1-u) by Bonnet's recurrence
 *   (l+1) P_{l+1} = (2l+1) x P_l - l P_{l-1}
 * rewritten for D_l = P_l - P_{l-1}:
 *   D_{l+1} = (l D_l - (2l+1) u P_l) / (l+1),   P_{l+1} = P_l + D_{l+1}.
 * (Substitute x = 1-u and subtract (l+1) P_l from both sides.) */
static void legendre_pair_u(int N, double u, double *pN, double *pNm1)
{
    if (N == 0) { *pN = 1.0; *pNm1 = 0.0; return; }
    double p_prev = 1.0, p = 1.0 - u, d = -u;
    for (int l = 1; l < N; ++l) {
        double dl = (double)l;
        d = (dl * d - (2.0 * dl + 1.0) * u * p) / (dl + 1.0);
        p_prev = p;
        p = p + d;
    }
    *pN = p;
    *pNm1 = p_prev;
}

/* Eq. addition-theorem: b(x) = sum_{l=0}^{lmax} (2l+1)/(4 pi) b_l P_l(x),
 * evaluated at x = 1 - u term by term with the recurrence above. */
double sympix_oracle_kernel_u(int lmax, const double *cl, double u)
{
    double p = 1.0, d = 0.0;
    double s = cl[0] / (4.0 * ORACLE_PI);
    if (lmax >= 1) {
        d = -u;
        p = 1.0 - u;
        s += 3.0 * cl[1] / (4.0 * ORACLE_PI) * p;
    }
    for (int l = 1; l < lmax; ++l) {
        double dl = (double)l;
        d = (dl * d - (2.0 * dl + 1.0) * u * p) / (dl + 1.0);
        p = p + d;
        s += (2.0 * (dl + 1.0) + 1.0) * cl[l + 1] / (4.0 * ORACLE_PI) * p;
    }
    return s;
}

/* ------------------------------------------------------------------------ */
/* Ring latitudes (Sec. 1 and Sec. 2.1: P_{N_rings}(cos theta_j) = 0)        */
/* ------------------------------------------------------------------------ */

/* theta_j for j = 0..N-1, north to south.  Newton's method in theta on
 * f(theta) = P_N(cos theta), df/dtheta = -N (P_{N-1} - x P_N) / sin(theta),
 * started from pi (j + 3/4) / (N + 1/2).  The northern roots are found; the
 * southern ones are pi - theta by the reflection P_N(-x) = (-1)^N P_N(x), and
 * an odd N has theta = pi/2 in the middle. */
int sympix_oracle_gl_theta(int N, double *theta)
{
    if (N <= 0) return -1;
    int half = N / 2;
    for (int j = 0; j < half; ++j) {
        double t = ORACLE_PI * ((double)j + 0.75) / ((double)N + 0.5);
        for (int it = 0; it < 100; ++it) {
            double s = sin(0.5 * t);
            double u = 2.0 * s * s;
            double pN, pNm1;
            legendre_pair_u(N, u, &pN, &pNm1);
            double x = cos(t);
            double step = pN * sin(t) / ((double)N * (pNm1 - x * pN));
            t += step;
            if (fabs(step) <= 1e-16 * t) break;
        }
        theta[j] = t;
        theta[N - 1 - j] = ORACLE_PI - t;
    }
    if (N % 2 == 1) theta[half] = 0.5 * ORACLE_PI;
    return 0;
}

/* Gauss-Legendre weights w_j = 2 (1 - x_j^2) / (N P_{N-1}(x_j))^2, the
 * quadrature weights of Eq. shdef (they integrate over x in [-1, 1]). */
int sympix_oracle_gl_weights(int N, const double *theta, double *w)
{
    for (int j = 0; j < N; ++j) {
        double th = theta[j] <= 0.5 * ORACLE_PI ? theta[j] : ORACLE_PI - theta[j];
        double s = sin(0.5 * th);
        double pN, pNm1;
        legendre_pair_u(N, 2.0 * s * s, &pN, &pNm1);
        double st = sin(th);
        w[j] = 2.0 * st * st / ((double)N * (double)N * pNm1 * pNm1);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Ring pixel counts                                                         */
/* ------------------------------------------------------------------------ */

static int is_5smooth(long v)
{
    if (v <= 0) return 0;
    while (v % 2 == 0) v /= 2;
    while (v % 3 == 0) v /= 3;
    while (v % 5 == 0) v /= 5;
    return v == 1;
}

static long smallest_5smooth_at_least(long v)
{
    if (v < 1) v = 1;
    while (!is_5smooth(v)) ++v;
    return v;
}

/* Greedy per-ring layout (not in the paper; the measured workloads use it):
 * N = lmax + 1 rings; target t_j = 2 (lmax+1) sin theta_j.  The equator-most
 * northern ring (the equatorial ring when N is odd) gets the smallest
 * 5-smooth count >= max(8, ceil t).  Moving to the pole, each ring takes the
 * smallest n_{j+1}/x over x in {1, 6/5, 5/4, 4/3, 2, 3} that is an integer,
 * >= 8 and >= t_j (the ratio set of Sec. 2.3).  The south mirrors the north. */
int sympix_oracle_layout_greedy(int lmax, const double *theta, int32_t *nring)
{
    int N = lmax + 1;
    int e = (N % 2 == 1) ? (N - 1) / 2 : N / 2 - 1;
    double te = 2.0 * (double)(lmax + 1) * sin(theta[e]);
    long ce = (long)ceil(te);
    if (ce < 8) ce = 8;
    nring[e] = (int32_t)smallest_5smooth_at_least(ce);
    static const int num[6] = {1, 5, 4, 3, 1, 1};
    static const int den[6] = {1, 6, 5, 4, 2, 3};
    for (int j = e - 1; j >= 0; --j) {
        double t = 2.0 * (double)(lmax + 1) * sin(theta[j]);
        long best = -1;
        long prev = nring[j + 1];
        for (int x = 0; x < 6; ++x) {
            if ((prev * num[x]) % den[x] != 0) continue;
            long c = prev * num[x] / den[x];
            if (c < 8) continue;
            if ((double)c < t) continue;
            if (best < 0 || c < best) best = c;
        }
        nring[j] = (int32_t)best;
    }
    for (int j = 0; j <= e; ++j) nring[N - 1 - j] = nring[j];
    return 0;
}

/* Smallest m >= 0 with sqrt(m^2 - 2 m cos theta) - lmax sin theta > thr
 * (Eq. polar-optimization); lmax + 1 when no m <= lmax qualifies. */
static int first_omitted_m(int lmax, double theta, double thr)
{
    for (int m = 0; m <= lmax; ++m) {
        double a = (double)m * (double)m - 2.0 * (double)m * cos(theta);
        if (a < 0.0) continue;
        if (sqrt(a) - (double)lmax * sin(theta) > thr) return m;
    }
    return lmax + 1;
}

/* Dynamic-programming layout of Fig. "Optimal-SymPix-Grid" (Sec. 2.5).
 * Inputs lmax, k, the threshold of Eq. polar-optimization (thr < 0 selects
 * the paper's max(100, lmax/100)) and the N = N_rings latitudes, where N is
 * lmax+1 rounded up to a multiple of 2k.  Output T[i], tiles per northern
 * band i = 0..N/(2k)-1 (pixels per ring = k T_i).  Readings of the figure:
 *   alpha_i uses the equator-side ring i k + k - 1 of band i;
 *   the start condition is C_{0,T0} = (T0-alpha_0)^2 with P_{0,T0} = T0, so
 *   that T1 != T0 is allowed as the caption says;
 *   the cost recursion adds (alpha_i - t)^2 to C_{i-1,t_prev};
 *   the last band takes argmin_t C_{n-1,t}; ties keep the first candidate
 *   found, scanning t_prev upward and x in the order 3, 2, 1, 4/3, 5/4, 6/5.
 * Returns 0, or -2 when no layout satisfies the constraints. */
int sympix_oracle_layout_dp(int lmax, int k, double thr, const double *theta,
                            int32_t *T, int32_t *alpha_out)
{
    int N = lmax + 1;
    if (N % (2 * k)) N += 2 * k - N % (2 * k);
    int n = N / (2 * k);
    if (thr < 0.0) thr = fmax(100.0, (double)lmax / 100.0);
    int *alpha = (int *)malloc(sizeof(int) * n);
    int tmax = 1;
    for (int i = 0; i < n; ++i) {
        int m = first_omitted_m(lmax, theta[i * k + k - 1], thr);
        alpha[i] = (2 * m + 1 + k - 1) / k;
        if (3 * alpha[i] > tmax) tmax = 3 * alpha[i];
        if (alpha_out) alpha_out[i] = alpha[i];
    }
    long T0 = smallest_5smooth_at_least(alpha[0]);
    if (T0 > tmax) tmax = (int)T0;
    int W = tmax + 1;
    double *C = (double *)malloc(sizeof(double) * (size_t)n * W);
    int *P = (int *)malloc(sizeof(int) * (size_t)n * W);
    for (size_t i = 0; i < (size_t)n * W; ++i) { C[i] = INFINITY; P[i] = -1; }
    C[T0] = (double)(T0 - alpha[0]) * (double)(T0 - alpha[0]);
    P[T0] = (int)T0;
    static const int num[6] = {3, 2, 1, 4, 5, 6};
    static const int den[6] = {1, 1, 1, 3, 4, 5};
    for (int i = 1; i < n; ++i) {
        for (int tp = 1; tp < W; ++tp) {
            double cprev = C[(size_t)(i - 1) * W + tp];
            if (!(cprev < INFINITY)) continue;
            for (int x = 0; x < 6; ++x) {
                if ((tp * num[x]) % den[x] != 0) continue;
                int t = tp * num[x] / den[x];
                if (t < alpha[i] || t > 3 * alpha[i] || t >= W) continue;
                int same = (num[x] == den[x]);
                if (!(P[(size_t)(i - 1) * W + tp] == tp || same)) continue;
                double c = cprev + (double)(alpha[i] - t) * (double)(alpha[i] - t);
                if (c < C[(size_t)i * W + t]) {
                    C[(size_t)i * W + t] = c;
                    P[(size_t)i * W + t] = tp;
                }
            }
        }
    }
    int best = -1;
    for (int t = 1; t < W; ++t)
        if (C[(size_t)(n - 1) * W + t] < INFINITY &&
            (best < 0 || C[(size_t)(n - 1) * W + t] < C[(size_t)(n - 1) * W + best]))
            best = t;
    int rc = 0;
    if (best < 0) {
        rc = -2;
    } else {
        T[n - 1] = best;
        for (int i = n - 2; i >= 0; --i) T[i] = P[(size_t)(i + 1) * W + T[i + 1]];
    }
    free(alpha); free(C); free(P);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Geometry of a pixel pair                                                  */
/* ------------------------------------------------------------------------ */

/* u = 1 - n1.n2 for pixel c1 of a ring (theta1, n1) and pixel c2 of a ring
 * (theta2, n2), with phi = 2 pi (c + 1/2) / n (first pixel at half a pixel
 * spacing, Sec. 2.3).  Haversine identity:
 *   1 - cos g = 2 sin^2((theta1-theta2)/2) + 2 sin th1 sin th2 sin^2(dphi/2),
 * and dphi = phi1 - phi2 = pi ((2c1+1) n2 - (2c2+1) n1) / (n1 n2). */
double sympix_oracle_u(double theta1, int n1, long c1, double theta2, int n2, long c2)
{
    double num = (double)((2 * c1 + 1) * (long)n2 - (2 * c2 + 1) * (long)n1);
    double half_dphi = 0.5 * ORACLE_PI * num / ((double)n1 * (double)n2);
    double a = sin(0.5 * (theta1 - theta2));
    double b = sin(half_dphi);
    return 2.0 * a * a + 2.0 * sin(theta1) * sin(theta2) * b * b;
}

/* The support gamma <= r_s as u <= 1 - cos r_s = 2 sin^2(r_s/2); a radius of
 * pi or more admits every pair (gamma never exceeds pi). */
static double support_u(double r_s)
{
    if (r_s >= ORACLE_PI) return INFINITY;
    double hs = sin(0.5 * r_s);
    return 2.0 * hs * hs;
}

/* Pixels p of ring rho coupled to pixel c of ring j: those with
 * u(q, p) <= 1 - cos r_s (support of Eq. f, one radius for D^ and B^).
 * Writes the ascending list of column indices into out (capacity n_rho) and
 * returns its length. */
int sympix_oracle_coupled(const double *theta, const int32_t *nring, int j, long c,
                          int rho, double r_s, int32_t *out)
{
    double us = support_u(r_s);
    int cnt = 0;
    for (long p = 0; p < nring[rho]; ++p) {
        double u = sympix_oracle_u(theta[j], nring[j], c, theta[rho], nring[rho], p);
        if (u <= us) out[cnt++] = (int32_t)p;
    }
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* Determinism of the support decision at its threshold                      */
/* ------------------------------------------------------------------------ */

static long gcd_l(long a, long b)
{
    while (b) { long t = a % b; a = b; b = t; }
    return a;
}

/* Smallest relative distance |u - u_s| / u_s between the support threshold
 * u_s = 2 sin^2(r_s / 2) and the u of any pixel pair (c on ring j, p on ring
 * rho) with j in [ring0, ring1) and rho any ring.  Coupling (u <= u_s) is an
 * FP64 comparison; two correct implementations (different sin routines) can
 * only disagree on a pair whose u lies within a few ulps of u_s, so a margin
 * well above that makes the coupled sets, and every integer derived from
 * them, implementation-independent.
 * Pairs: rotating both rings by 2 pi / g, g = gcd(n_j, n_rho), maps pixel c
 * to c + n_j/g and p to p + n_rho/g and keeps every separation, so columns
 * c < n_j / g of ring j meet every separation of the ring pair.  A ring whose
 * nearest possible pair (same longitude, u = 2 sin^2(dtheta/2)) lies above
 * 2 u_s cannot hold a pair near the threshold and is skipped.
 * Returns +inf when r_s >= pi (every pair couples, no comparison is made). */
double sympix_oracle_support_margin(int nrings, const double *theta, const int32_t *nring,
                                    double r_s, int ring0, int ring1)
{
    double us = support_u(r_s);
    if (!(us < INFINITY)) return INFINITY;
    double best = INFINITY;
    for (int j = ring0; j < ring1; ++j) {
        for (int rho = 0; rho < nrings; ++rho) {
            double a = sin(0.5 * (theta[j] - theta[rho]));
            if (2.0 * a * a > 2.0 * us) continue;
            long g = gcd_l(nring[j], nring[rho]);
            long P = nring[j] / g;
            for (long c = 0; c < P; ++c)
                for (long p = 0; p < nring[rho]; ++p) {
                    double u = sympix_oracle_u(theta[j], nring[j], c, theta[rho], nring[rho], p);
                    double m = fabs(u - us) / us;
                    if (m < best) best = m;
                }
        }
    }
    return best;
}

/* The radius both implementations use (reading C5 of the support): r_s
 * itself when every pair is more than 1e-12 (relative) away from the
 * threshold, else r_s scaled by (1 - 1e-9), repeatedly, until that holds.
 * *margin receives the final smallest relative distance. */
double sympix_oracle_guarded_radius(int nrings, const double *theta, const int32_t *nring,
                                    double r_s, int ring0, int ring1, double *margin)
{
    double m = sympix_oracle_support_margin(nrings, theta, nring, r_s, ring0, ring1);
    for (int it = 0; it < 8 && m <= 1e-12; ++it) {
        r_s *= 1.0 - 1e-9;
        m = sympix_oracle_support_margin(nrings, theta, nring, r_s, ring0, ring1);
    }
    if (margin) *margin = m;
    return r_s;
}

/* ------------------------------------------------------------------------ */
/* One preconditioner block (Eq. system-rewritten, Eq. Dhat)                */
/* ------------------------------------------------------------------------ */

/* Dense M (n_j x n_j, row-major) for ring j:
 *   M_qr = [u_qr <= u_s] d(1-u_qr)
 *        + sum over pixels p of every ring with u_pq <= u_s and u_pr <= u_s of
 *          b(1-u_pq) N^-1_p b(1-u_pr).
 * b and d follow Eq. addition-theorem with coefficients bl and dl.  ninv is
 * indexed by the grid's pixel numbering: pixel c of ring r is
 * ring_offset[r] + c * ring_stride[r].  The sum is taken p by p: for each p
 * the coupled pixels of ring j are listed with their kernel values, and every
 * pair of them receives its product (each triple once per ordered pair).
 * Returns the number of triples summed. */
long sympix_oracle_block(int nrings, const double *theta, const int32_t *nring,
                         const int64_t *ring_offset, const int32_t *ring_stride,
                         int lmax, const double *bl, const double *dl, double r_s,
                         const double *ninv, int j, double *M)
{
    int n = nring[j];
    double us = support_u(r_s);
    memset(M, 0, sizeof(double) * (size_t)n * n);

    /* D^ on the block's own ring */
    for (long q = 0; q < n; ++q)
        for (long r = 0; r < n; ++r) {
            double u = sympix_oracle_u(theta[j], n, q, theta[j], n, r);
            if (u <= us) M[q * n + r] += sympix_oracle_kernel_u(lmax, dl, u);
        }

    /* B^T N^-1 B^, summed over every pixel p of every ring */
    long triples = 0;
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * n);
    double *val = (double *)malloc(sizeof(double) * n);
    for (int rho = 0; rho < nrings; ++rho) {
        double a = sin(0.5 * (theta[j] - theta[rho]));
        if (2.0 * a * a > us) continue; /* u >= 2 sin^2(dtheta/2) for every pair */
        for (long p = 0; p < nring[rho]; ++p) {
            int cnt = 0;
            for (long q = 0; q < n; ++q) {
                double u = sympix_oracle_u(theta[j], n, q, theta[rho], nring[rho], p);
                if (u <= us) {
                    idx[cnt] = (int32_t)q;
                    val[cnt] = sympix_oracle_kernel_u(lmax, bl, u);
                    ++cnt;
                }
            }
            double np = ninv[ring_offset[rho] + p * (int64_t)ring_stride[rho]];
            for (int x = 0; x < cnt; ++x)
                for (int y = 0; y < cnt; ++y)
                    M[(size_t)idx[x] * n + idx[y]] += val[x] * np * val[y];
            triples += (long)cnt * cnt;
        }
    }
    free(idx); free(val);
    return triples;
}

/* The block of the same operator between two rings (Eq. system-rewritten,
 * Eq. Dhat), dense n_j x n_k, row-major, rows on ring j and columns on ring
 * k:
 *   M_qr = [u_qr <= u_s] d(1-u_qr)
 *        + sum over pixels p of every ring with u_pq <= u_s and u_pr <= u_s of
 *          b(1-u_pq) N^-1_p b(1-u_pr).
 * With k = j this is sympix_oracle_block.  Summed p by p as there: for each
 * p the coupled pixels of both rings are listed with their kernel values and
 * every (q, r) pair of them receives its product.  Returns the triples. */
long sympix_oracle_block_pair(int nrings, const double *theta, const int32_t *nring,
                              const int64_t *ring_offset, const int32_t *ring_stride,
                              int lmax, const double *bl, const double *dl, double r_s,
                              const double *ninv, int j, int k, double *M)
{
    int nj = nring[j], nk = nring[k];
    double us = support_u(r_s);
    memset(M, 0, sizeof(double) * (size_t)nj * nk);

    /* D^ between the two rings */
    for (long q = 0; q < nj; ++q)
        for (long r = 0; r < nk; ++r) {
            double u = sympix_oracle_u(theta[j], nj, q, theta[k], nk, r);
            if (u <= us) M[q * nk + r] += sympix_oracle_kernel_u(lmax, dl, u);
        }

    /* B^T N^-1 B^, summed over every pixel p of every ring */
    long triples = 0;
    int32_t *iq = (int32_t *)malloc(sizeof(int32_t) * nj);
    int32_t *ir = (int32_t *)malloc(sizeof(int32_t) * nk);
    double *vq = (double *)malloc(sizeof(double) * nj);
    double *vr = (double *)malloc(sizeof(double) * nk);
    for (int rho = 0; rho < nrings; ++rho) {
        double a1 = sin(0.5 * (theta[j] - theta[rho]));
        double a2 = sin(0.5 * (theta[k] - theta[rho]));
        if (2.0 * a1 * a1 > us || 2.0 * a2 * a2 > us) continue; /* no pixel of rho reaches both */
        for (long p = 0; p < nring[rho]; ++p) {
            int cq = 0, cr = 0;
            for (long q = 0; q < nj; ++q) {
                double u = sympix_oracle_u(theta[j], nj, q, theta[rho], nring[rho], p);
                if (u <= us) {
                    iq[cq] = (int32_t)q;
                    vq[cq] = sympix_oracle_kernel_u(lmax, bl, u);
                    ++cq;
                }
            }
            if (!cq) continue;
            for (long r = 0; r < nk; ++r) {
                double u = sympix_oracle_u(theta[k], nk, r, theta[rho], nring[rho], p);
                if (u <= us) {
                    ir[cr] = (int32_t)r;
                    vr[cr] = sympix_oracle_kernel_u(lmax, bl, u);
                    ++cr;
                }
            }
            double np = ninv[ring_offset[rho] + p * (int64_t)ring_stride[rho]];
            for (int x = 0; x < cq; ++x)
                for (int y = 0; y < cr; ++y)
                    M[(size_t)iq[x] * nk + ir[y]] += vq[x] * np * vr[y];
            triples += (long)cq * cr;
        }
    }
    free(iq); free(ir); free(vq); free(vr);
    return triples;
}

/* ------------------------------------------------------------------------ */
/* Triangular solves with a Cholesky factor (applying M^-1 = L^-T L^-1)      */
/* ------------------------------------------------------------------------ */

/* Solve L y = b (trans = 0, forward substitution) or L^T y = b (trans = 1,
 * back substitution) for a lower-triangular n x n row-major L.  Returns 0, or
 * i+1 for the first zero diagonal met. */
int sympix_oracle_trisolve(int n, const double *L, const double *b, int trans, double *y)
{
    if (!trans) {
        for (int i = 0; i < n; ++i) {
            double s = b[i];
            for (int c = 0; c < i; ++c) s -= L[(size_t)i * n + c] * y[c];
            if (L[(size_t)i * n + i] == 0.0) return i + 1;
            y[i] = s / L[(size_t)i * n + i];
        }
    } else {
        for (int i = n - 1; i >= 0; --i) {
            double s = b[i];
            for (int c = i + 1; c < n; ++c) s -= L[(size_t)c * n + i] * y[c];
            if (L[(size_t)i * n + i] == 0.0) return i + 1;
            y[i] = s / L[(size_t)i * n + i];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Pixel-domain convolution (Eq. convolution-pixel)                          */
/* ------------------------------------------------------------------------ */

/* g at nq output pixels (ring q_ring[i], column q_col[i]):
 *   g_i = sum over every pixel p of every ring with u_ip <= u_s of
 *         b(1 - u_ip) f_p,
 * b by Eq. addition-theorem with coefficients bl, truncated at the radius r_s
 * (the approximation b = 0 beyond the support, Sec. 3).  f is indexed by the
 * grid's pixel numbering (pixel c of ring r is ring_offset[r] +
 * c * ring_stride[r]).  Returns the number of coupled pairs summed. */
long sympix_oracle_convolve(int nrings, const double *theta, const int32_t *nring,
                            const int64_t *ring_offset, const int32_t *ring_stride,
                            int lmax, const double *bl, double r_s, const double *f,
                            int nq, const int32_t *q_ring, const int32_t *q_col, double *g)
{
    double us = support_u(r_s);
    long pairs = 0;
    for (int i = 0; i < nq; ++i) {
        int j = q_ring[i];
        double acc = 0.0;
        for (int rho = 0; rho < nrings; ++rho) {
            double a = sin(0.5 * (theta[j] - theta[rho]));
            if (2.0 * a * a > us) continue; /* no pixel of this ring is close enough */
            for (long p = 0; p < nring[rho]; ++p) {
                double u = sympix_oracle_u(theta[j], nring[j], q_col[i], theta[rho], nring[rho], p);
                if (u <= us) {
                    acc += sympix_oracle_kernel_u(lmax, bl, u) *
                           f[ring_offset[rho] + p * (int64_t)ring_stride[rho]];
                    ++pairs;
                }
            }
        }
        g[i] = acc;
    }
    return pairs;
}

/* ------------------------------------------------------------------------ */
/* Cholesky                                                                  */
/* ------------------------------------------------------------------------ */

/* Textbook left-looking dense Cholesky A = L L^T of an n x n row-major
 * matrix; L is written to the lower triangle of L (upper set to zero).
 * Returns 0, or i+1 for the first row i whose pivot is not positive. */
int sympix_oracle_cholesky(int n, const double *A, double *L)
{
    memset(L, 0, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            if (i == j) {
                if (!(s > 0.0)) return i + 1;
                L[(size_t)i * n + i] = sqrt(s);
            } else {
                L[(size_t)i * n + j] = s / L[(size_t)j * n + j];
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Pixel ordering (Sec. 2.4)                                                 */
/* ------------------------------------------------------------------------ */

/* Bands of k rings are listed north band 0, south band 0, north band 1,
 * south band 1, ... (hemispheres interleaved band by band).  Inside a band
 * the index runs fastest along theta: pixel c of the r-th ring of the band
 * is band_start + c k + r.  A northern band counts its rings from the pole
 * (rings i k .. i k + k - 1); a southern band also counts from its pole
 * (rings N-1-i k, N-2-i k, ...), i.e. it mirrors the northern band (the
 * paper's ordering figure is missing; this is the reading used).  With k = 1
 * and N odd the equatorial ring comes last.  Outputs, per ring j (geometric
 * order, north to south): ring_offset[j] = index of its pixel c = 0 and
 * ring_stride[j] = k, so pixel c sits at ring_offset[j] + c ring_stride[j].
 * Returns the pixel count, or -1 when N and k do not fit together. */
long sympix_oracle_ordering(int N, int k, const int32_t *nring, int64_t *ring_offset,
                            int32_t *ring_stride)
{
    int nb;
    int odd = 0;
    if (k == 1) {
        nb = N / 2;
        odd = N % 2;
    } else {
        if (N % (2 * k)) return -1;
        nb = N / (2 * k);
    }
    long pos = 0;
    for (int i = 0; i < nb; ++i) {
        for (int hemi = 0; hemi < 2; ++hemi) {
            int cnt = nring[hemi == 0 ? i * k : N - 1 - i * k];
            for (int r = 0; r < k; ++r) {
                int ring = hemi == 0 ? i * k + r : N - 1 - i * k - r;
                if (nring[ring] != cnt) return -1;
                ring_offset[ring] = pos + r;
                ring_stride[ring] = k;
            }
            pos += (long)cnt * k;
        }
    }
    if (odd) {
        int ring = N / 2;
        ring_offset[ring] = pos;
        ring_stride[ring] = 1;
        pos += nring[ring];
    }
    return pos;
}

/* ------------------------------------------------------------------------ */
/* Tile adjacency on a DP grid, and the block of one band (Sec. 2.3 tiling, */
/* Sec. 4.2 locality approximation)                                         */
/* ------------------------------------------------------------------------ */

/* The paper partitions a grid of k-ring bands into k x k tiles (k columns of
 * the band's k rings) and takes D^_ij = B^_ij = 0 unless pixels i and j lie
 * in the same or in neighbouring tiles.  It does not say which tiles of two
 * bands with different tile counts are neighbours.  Reading used here:
 *   - bands are numbered by latitude, g = ring / k (north pole to south
 *     pole); tiles of bands g and g' can be neighbours only if |g - g'| <= 1
 *     (so the two bands next to the equator are neighbours);
 *   - tile a of a band with T tiles spans the longitudes [a/T, (a+1)/T] of a
 *     turn; two tiles are neighbours when these closed arcs meet (overlap or
 *     touch) on the circle;
 *   - inside a polar band (g = 0 or the last) every two tiles are
 *     neighbours: the tiles meet across the pole.
 * Returns 1 when pixel ca of ring ra and pixel cb of ring rb are coupled. */
int sympix_oracle_tiles_coupled(int nrings, int k, const int32_t *nring, int ra, long ca, int rb, long cb)
{
    int ga = ra / k, gb = rb / k;
    int G = nrings / k;
    if (ga - gb > 1 || gb - ga > 1) return 0;
    if (ga == gb && (ga == 0 || ga == G - 1)) return 1;
    long Ta = nring[ra] / k, Tb = nring[rb] / k;
    long a = ca / k, b = cb / k;
    /* arcs [a/Ta, (a+1)/Ta] and [(b+s Tb)/Tb, (b+s Tb+1)/Tb] for a turn s */
    for (long s = -1; s <= 1; ++s) {
        long bb = b + s * Tb;
        if (a * Tb <= (bb + 1) * Ta && bb * Ta <= (a + 1) * Tb) return 1;
    }
    return 0;
}

/* Dense block M (K x K, row-major, K = k n_g) of band g of a DP grid, in the
 * band's own pixel order: row i is the pixel with grid index
 * band_start + i, band_start the smallest grid index of the band's pixels.
 *   M_qr = [q, r coupled] d(q.r)
 *        + sum over pixels p of the grid coupled to both q and r of
 *          b(p.q) N^-1_p b(p.r),
 * "coupled" as sympix_oracle_tiles_coupled says (Eq. system-rewritten,
 * Eq. Dhat with Y2 = Y1 under the tile truncation).  Summed p by p as
 * sympix_oracle_block does.  Returns the triples summed, or -1 when g is not
 * a band of the grid. */
long sympix_oracle_band_block(int nrings, const double *theta, const int32_t *nring,
                              const int64_t *ring_offset, const int32_t *ring_stride, int k,
                              int lmax, const double *bl, const double *dl, const double *ninv,
                              int g, double *M)
{
    if (k < 1 || nrings % k || g < 0 || g >= nrings / k) return -1;
    int r0 = g * k;
    long nb = nring[r0];
    long K = (long)k * nb;
    int64_t start = ring_offset[r0];
    for (int r = r0; r < r0 + k; ++r)
        if (ring_offset[r] < start) start = ring_offset[r];
    memset(M, 0, sizeof(double) * (size_t)K * K);
    /* row index of pixel c of ring r of the band */
#define BAND_ROW(r, c) ((long)(ring_offset[(r)] + (c) * (int64_t)ring_stride[(r)] - start))

    /* D^ inside the band */
    for (int ra = r0; ra < r0 + k; ++ra)
        for (long ca = 0; ca < nb; ++ca)
            for (int rb = r0; rb < r0 + k; ++rb)
                for (long cb = 0; cb < nb; ++cb) {
                    if (!sympix_oracle_tiles_coupled(nrings, k, nring, ra, ca, rb, cb)) continue;
                    double u = sympix_oracle_u(theta[ra], (int)nb, ca, theta[rb], (int)nb, cb);
                    M[BAND_ROW(ra, ca) * K + BAND_ROW(rb, cb)] += sympix_oracle_kernel_u(lmax, dl, u);
                }

    /* B^T N^-1 B^ */
    long triples = 0;
    long *idx = (long *)malloc(sizeof(long) * K);
    double *val = (double *)malloc(sizeof(double) * K);
    for (int rho = 0; rho < nrings; ++rho) {
        if (rho / k < g - 1 || rho / k > g + 1) continue; /* no tile of band g has a neighbour there */
        for (long p = 0; p < nring[rho]; ++p) {
            long cnt = 0;
            for (int ra = r0; ra < r0 + k; ++ra)
                for (long ca = 0; ca < nb; ++ca) {
                    if (!sympix_oracle_tiles_coupled(nrings, k, nring, rho, p, ra, ca)) continue;
                    double u = sympix_oracle_u(theta[ra], (int)nb, ca, theta[rho], nring[rho], p);
                    idx[cnt] = BAND_ROW(ra, ca);
                    val[cnt] = sympix_oracle_kernel_u(lmax, bl, u);
                    ++cnt;
                }
            double np = ninv[ring_offset[rho] + p * (int64_t)ring_stride[rho]];
            for (long x = 0; x < cnt; ++x)
                for (long y = 0; y < cnt; ++y) M[(size_t)idx[x] * K + idx[y]] += val[x] * np * val[y];
            triples += cnt * cnt;
        }
    }
#undef BAND_ROW
    free(idx);
    free(val);
    return triples;
}

/* ------------------------------------------------------------------------ */
/* Y2 != Y1: the noise on an auxiliary grid (Sec. 4.2, Eq. substitution,     */
/* Eq. degrade)                                                              */
/* ------------------------------------------------------------------------ */

/* 1 - cos of the angle between (t1, f1) and (t2, f2), by the haversine form:
 * sin^2(gamma/2) = sin^2(dt/2) + sin t1 sin t2 sin^2(df/2). */
static double u_angles(double t1, double f1, double t2, double f2)
{
    double a = sin(0.5 * (t1 - t2)), b = sin(0.5 * (f1 - f2));
    return 2.0 * (a * a + sin(t1) * sin(t2) * b * b);
}

/* Eq. degrade: theta_2 = W_2 Y_2 Y_obs^T theta.  Y_obs^T theta is the
 * unweighted adjoint synthesis a_lm = sum_i Y_lm(n_i) theta_i over the
 * observation points i; Y_2 synthesises a_lm (l <= lmax2) on the auxiliary
 * grid; W_2 multiplies pixel p by its quadrature weight w_p (the weight of its
 * ring in cos theta times 2 pi / n_ring).  The sum over m is the addition
 * theorem, so
 *   theta_2[p] = w_p sum_i theta_i K(n_p . n_i),
 *   K(x) = sum_{l <= lmax2} (2l+1)/(4 pi) P_l(x)
 * (Eq. addition-theorem with every coefficient 1), evaluated per pair.
 * Grid 2: nrings2 rings at theta2 with nring2 pixels each (pixel c at
 * phi = 2 pi (c + 1/2) / n), ring weights wring2, pixel numbering
 * ring_offset2 + c * ring_stride2.  Observation points: (obs_theta,
 * obs_phi) with values obs_val.  Returns the pixels written, -1 on
 * allocation failure. */
long sympix_oracle_degrade(int lmax2, long nobs, const double *obs_theta, const double *obs_phi,
                           const double *obs_val, int nrings2, const double *theta2, const int32_t *nring2,
                           const double *wring2, const int64_t *ring_offset2, const int32_t *ring_stride2,
                           double *out)
{
    double *ones = (double *)malloc(sizeof(double) * (size_t)(lmax2 + 1));
    if (!ones) return -1;
    for (int l = 0; l <= lmax2; ++l) ones[l] = 1.0;
    long written = 0;
    for (int rho = 0; rho < nrings2; ++rho) {
        int n = nring2[rho];
        double w = wring2[rho] * 2.0 * ORACLE_PI / (double)n;
        for (long c = 0; c < n; ++c) {
            double phi = 2.0 * ORACLE_PI * ((double)c + 0.5) / (double)n;
            double s = 0.0;
            for (long i = 0; i < nobs; ++i)
                s += obs_val[i] * sympix_oracle_kernel_u(lmax2, ones, u_angles(theta2[rho], phi, obs_theta[i], obs_phi[i]));
            out[ring_offset2[rho] + c * (int64_t)ring_stride2[rho]] = w * s;
            ++written;
        }
    }
    free(ones);
    return written;
}

/* Eq. system-rewritten and Eq. Dhat with B^ = Y_2 B Y_1^T: the block of ring
 * j of grid 1 (dense n_j x n_j, row-major), with the noise N_2^-1 = ninv2 on
 * the pixels p of grid 2:
 *   M_qr = [u_qr <= u_s] d(1-u_qr)
 *        + sum over pixels p of grid 2 with u_pq <= u_s and u_pr <= u_s of
 *          b(1-u_pq) N2^-1_p b(1-u_pr).
 * With grid 2 = grid 1 this is sympix_oracle_block.  Returns the triples
 * summed, -1 on allocation failure. */
long sympix_oracle_block_y2(const double *theta1, const int32_t *nring1, int j, int nrings2,
                            const double *theta2, const int32_t *nring2, const int64_t *ring_offset2,
                            const int32_t *ring_stride2, int lmax, const double *bl, const double *dl,
                            double r_s, const double *ninv2, double *M)
{
    int n = nring1[j];
    double us = support_u(r_s);
    memset(M, 0, sizeof(double) * (size_t)n * n);
    for (long q = 0; q < n; ++q)
        for (long r = 0; r < n; ++r) {
            double u = sympix_oracle_u(theta1[j], n, q, theta1[j], n, r);
            if (u <= us) M[q * n + r] += sympix_oracle_kernel_u(lmax, dl, u);
        }
    long triples = 0;
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * n);
    double *val = (double *)malloc(sizeof(double) * n);
    if (!idx || !val) { free(idx); free(val); return -1; }
    for (int rho = 0; rho < nrings2; ++rho)
        for (long p = 0; p < nring2[rho]; ++p) {
            int cnt = 0;
            for (long q = 0; q < n; ++q) {
                double u = sympix_oracle_u(theta1[j], n, q, theta2[rho], nring2[rho], p);
                if (u <= us) {
                    idx[cnt] = (int32_t)q;
                    val[cnt] = sympix_oracle_kernel_u(lmax, bl, u);
                    ++cnt;
                }
            }
            double np = ninv2[ring_offset2[rho] + p * (int64_t)ring_stride2[rho]];
            for (int x = 0; x < cnt; ++x)
                for (int y = 0; y < cnt; ++y)
                    M[(size_t)idx[x] * n + idx[y]] += val[x] * np * val[y];
            triples += (long)cnt * cnt;
        }
    free(idx); free(val);
    return triples;
}
