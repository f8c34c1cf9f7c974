/*
 * sympix.h -- C ABI of the GB300 SymPix preconditioner-block library.
 *
 * The library samples the rotationally invariant operators D^ = Y D Y^T and
 * B^ = Y B Y^T in pixel space on a SymPix grid and forms, per ring, the
 * preconditioner block  M = D^ + B^T N^-1 B^  (Seljebotn & Eriksen,
 * "SymPix: a spherical grid for efficient sampling of rotationally
 * invariant operators", Sec. 4.2, Eq. system-rewritten and Eq. Dhat), then
 * Cholesky-factors every block.
 *
 * Conventions shared by every call:
 *   - Every call returns SYMPIX_OK (0) or a positive error code; the text of
 *     the last error of the calling thread is sympix_last_error().  No call
 *     aborts the process.
 *   - Device pointers are plain CUDA device addresses of the current device;
 *     host pointers are ordinary host memory.  The caller owns every pointer
 *     it passes; the library owns the handles it returns and frees them in
 *     the matching *_free call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that take a stream only enqueue work on it and return;
 *     their launch errors are reported at once, device-side failures of the
 *     factorisation through the per-block `info` array.
 *   - Indices: rings j = 0 .. nrings-1 run north to south; the pixels of
 *     ring j are columns c = 0 .. n_j-1 at longitude 2 pi (c + 1/2) / n_j.
 *   - There is no CPU fallback: if no CUDA device is usable every compute
 *     call fails with SYMPIX_ECUDA.
 */
#ifndef SYMPIX_H
#define SYMPIX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SYMPIX_OK 0
#define SYMPIX_EINVAL 1   /* bad argument (size, range, null pointer)         */
#define SYMPIX_ENOMEM 2   /* a device or host allocation of the library failed */
#define SYMPIX_ECUDA 3    /* a CUDA call failed (message names it)             */
#define SYMPIX_ETIMEOUT 4 /* a bounded device wait ran out                      */
#define SYMPIX_EUNSUPPORTED 5 /* combination not implemented (message says which) */

/* grid layouts */
#define SYMPIX_LAYOUT_GREEDY 0 /* per-ring counts, k = 1, N_rings = lmax + 1      */
#define SYMPIX_LAYOUT_DP 1     /* bands of k rings chosen by dynamic programming  */

/* arithmetic of the B^T N^-1 B^ contraction */
#define SYMPIX_PREC_FP64 0   /* FP64 products and sums                           */
#define SYMPIX_PREC_FP32 1   /* FP32 products, FP32 accumulation                 */
#define SYMPIX_PREC_FP32X2 2 /* split FP32 (hi + lo pairs): near-FP64 on FP32 pipes */

/* block storage */
#define SYMPIX_STORE_PBAND 0 /* periodic band + border, dense for small rings   */
#define SYMPIX_STORE_DENSE 1 /* every block n x n                              */

/* block formats reported by sympix_block_layout */
#define SYMPIX_BLOCK_PBAND 0
#define SYMPIX_BLOCK_DENSE 1

typedef struct sympix_grid_s *sympix_grid_t;
typedef struct sympix_plan_s *sympix_plan_t;
typedef struct sympix_step_s *sympix_step_t;

/* stages of a captured step (sympix_step_launch) */
#define SYMPIX_STAGE_TABLE 1  /* sympix_kernel_table  */
#define SYMPIX_STAGE_SAMPLE 2 /* sympix_sample_blocks */
#define SYMPIX_STAGE_FACTOR 4 /* sympix_factor_blocks */
#define SYMPIX_STAGE_ALL 7

typedef struct {
    int lmax;       /* band limit the grid was built for                    */
    int k;          /* tile size (rings per band)                            */
    int layout;     /* SYMPIX_LAYOUT_*                                       */
    int nrings;     /* number of rings                                       */
    int nbands;     /* number of bands of k rings (an odd equator ring counts as one) */
    int max_ring;   /* largest ring pixel count                              */
    int64_t npix;   /* number of pixels                                      */
} sympix_grid_desc;

/* ------------------------------------------------------------------------ */
/* Grid (Sec. 2; Fig. Optimal-SymPix-Grid)                                   */
/* ------------------------------------------------------------------------ */

/* Build a SymPix grid.
 *   lmax       band limit (>= 1, <= 16383).
 *   k          tile size: 1 for SYMPIX_LAYOUT_GREEDY; >= 1 for SYMPIX_LAYOUT_DP.
 *   layout     SYMPIX_LAYOUT_GREEDY: N_rings = lmax + 1, per-ring counts from
 *              the equator outward, target 2 (lmax+1) sin theta_j, neighbour
 *              ratios in {1, 6/5, 5/4, 4/3, 2, 3}, at least 8 per ring.
 *              SYMPIX_LAYOUT_DP: the dynamic programme of Fig.
 *              Optimal-SymPix-Grid (Sec. 2.5) with N_rings = lmax + 1 rounded
 *              up to a multiple of 2k.
 *   polar_thr  threshold of Eq. polar-optimization (Sec. 2.1); < 0 selects
 *              the paper's max(100, lmax/100).  Ignored by GREEDY.
 *   out        receives a library-owned handle (free with sympix_grid_free).
 * Ring colatitudes are the roots of P_{N_rings}(cos theta) (Sec. 1, 2.1),
 * found on the device in FP64.  Pixel numbering (Sec. 2.4): bands of k rings
 * in the order north 0, south 0, north 1, south 1, ...; inside a band the
 * index runs fastest along theta; a southern band counts its rings from its
 * pole; an odd equatorial ring (GREEDY) comes last.  Synchronous. */
int sympix_grid(int lmax, int k, int layout, double polar_thr, sympix_grid_t *out);

/* Sizes of a grid. */
int sympix_grid_describe(sympix_grid_t grid, sympix_grid_desc *desc);

/* Copy the ring tables to host arrays of length nrings (any may be NULL):
 * theta[j] colatitude, nring[j] pixel count, ring_offset[j] index of the
 * ring's pixel c = 0, ring_stride[j] index step between its columns (pixel
 * c of ring j is ring_offset[j] + c * ring_stride[j]). */
int sympix_grid_copy(sympix_grid_t grid, double *theta, int32_t *nring,
                     int64_t *ring_offset, int32_t *ring_stride);

void sympix_grid_free(sympix_grid_t grid);

/* ------------------------------------------------------------------------ */
/* Support, symmetry classes and block plan (Eq. f; Sec. 2.3; Sec. 4.2)     */
/* ------------------------------------------------------------------------ */

/* Plan `nops` operators on `grid` for the blocks of rings [ring0, ring1).
 *   r_s   host array [nops]: support radius (radians) of operator o; a pixel
 *         pair couples when its angular distance is <= r_s[o] (the truncation
 *         of Eq. f, one radius for D^ and B^ of the operator).  r_s >= pi
 *         couples every pair.  A radius within 1e-12 (relative, in
 *         1 - cos) of some pixel pair's separation is scaled by (1 - 1e-9)
 *         first, so that no coupling decision rests on the last bits of a
 *         sin (sympix_plan_radius reports the radius used).
 * The device computes, for every coupled pair of rings, the distinct pixel
 * separations (one symmetry class per distinct |phi_1 - phi_2|, shared by
 * the transposed and the north/south-mirrored ring pair) and the band width
 * of every block; the host-side plan keeps the block sizes and offsets.
 * On a GREEDY grid (k = 1) a block is one ring.  On a DP grid with
 * 2 <= k <= 8 a block is one band of k rings (Sec. 2.3 tiling), and the
 * support is tile adjacency instead of a radius (Sec. 4.2, the locality
 * approximation): two pixels couple when their k x k tiles lie in bands at
 * most one apart in latitude and their closed longitude arcs [a/T, (a+1)/T]
 * of a turn meet, and every two tiles of a polar band couple; r_s is checked
 * but not used.  Such a plan needs ring0 and ring1 to be multiples of k and
 * bands of at most 16384 pixels; its blocks are dense (SYMPIX_BLOCK_DENSE,
 * rows in the band's pixel order, ring_offset - the band's first index), and
 * sympix_convolve, sympix_support_copy, sympix_table_copy and the calls on
 * blocks between rings return SYMPIX_EUNSUPPORTED.
 * Allocates the class and kernel tables on the device.  Synchronous.
 * out receives a library-owned handle (free with sympix_plan_free). */
int sympix_support(sympix_grid_t grid, int nops, const double *r_s, int ring0, int ring1,
                   sympix_plan_t *out);

/* Plan options (sympix_plan_option). */
#define SYMPIX_OPT_FP32_PIVOT_FLOOR 1 /* FP32 factor: a block is refactored in FP64 when a pivot
                                          falls below floor x its row's original diagonal
                                          (default 0.05; 0 never, > 1 always) */
#define SYMPIX_OPT_TRACE 2            /* 1: record a CUDA event after every kernel launch of
                                          sympix_kernel_table / _sample_blocks / _factor_blocks
                                          (direct calls, not stream capture); 0: off (default) */
#define SYMPIX_OPT_TABLE_CTA 3        /* threads per CTA of the kernel-table launch: 32, 64 or
                                          128 (default 32) */
#define SYMPIX_OPT_BORDER_THREADS 4   /* threads per CTA of the FP32 border pass: 256 or 512
                                          (default 512) */
#define SYMPIX_OPT_NARROW_FACTOR 6    /* periodic-band blocks with w <= 12: 0 one warp per 4-8
                                          blocks, G lanes per block sharing the band window; 1 the
                                          earlier kernels (FP32: one lane per block on an FP32
                                          band copy, a band warp and border warps per CTA; FP64 /
                                          split FP32: lane groups); 2 every arithmetic: the band
                                          pass alone (one lane per block on a band copy of the
                                          arithmetic), then the border rows solved in parallel
                                          over column chunks; 3 FP32: for w <= 8 band and border
                                          passes in two CTAs of one cooperative launch (the
                                          kernel of 1 where they cannot all be resident),
                                          9 <= w <= 12 as 2 beside it (3: FP64 and split FP32
                                          as 2); -1 (default) per
                                          arithmetic, as measured at l_max 3000: FP64 2, FP32 3,
                                          split FP32 2.  sympix_autotune times the candidates for
                                          its factor arithmetic */
#define SYMPIX_OPT_WAIT_LIMIT 5       /* polls of a bounded device wait (default 2^22, about
                                          0.3 s): the FP32 factor's border warps wait for rows
                                          the band warp of the same CTA publishes */

/* Set a plan option; takes effect for the following calls on the plan. */
int sympix_plan_option(sympix_plan_t plan, int option, double value);

/* Autotune the launch shapes (SYMPIX_OPT_TABLE_CTA, SYMPIX_OPT_BORDER_THREADS)
 * and the w <= 12 factor kernel of factor_precision (SYMPIX_OPT_NARROW_FACTOR)
 * on the caller's data: each candidate runs the calls it affects
 * (sympix_kernel_table with bl, dl; sympix_sample_blocks and
 * sympix_factor_blocks with ninv, storage, the precisions, blocks and info)
 * once to warm up and once timed with CUDA events on `stream`; the fastest is
 * kept in the plan.  Results are identical for every candidate; blocks and
 * info are overwritten.  Synchronous.  The paper has no counterpart: this
 * chooses how the same operations are launched. */
int sympix_autotune(sympix_plan_t plan, const double *bl, const double *dl, const double *ninv, int storage,
                    int sample_precision, int factor_precision, double *blocks, int32_t *info, void *stream);

/* The plan's launch shapes (any pointer may be NULL); narrow[3] receives
 * the w <= 12 factor kernel per arithmetic (index SYMPIX_PREC_*). */
int sympix_plan_tuning(sympix_plan_t plan, int *table_cta, int *border_threads, int *narrow);

/* Per-kernel device times of the traced calls since the last read
 * (SYMPIX_OPT_TRACE): waits for the last recorded event, then writes up to
 * `cap` spans, each the kernel (or group of launches) `names[i]` (static
 * strings) and its duration `ms[i]` in milliseconds, in launch order;
 * *count receives the number of spans recorded (at most 256 per read).
 * Clears the trace.  Not part of the method: a measurement aid. */
int sympix_trace_read(sympix_plan_t plan, int cap, const char **names, float *ms, int *count);

/* Counts of a plan (any pointer may be NULL): nslots symmetry-class slots
 * (kernel values per operator); npairs coupled ordered ring pairs summed over
 * operators; ntriples the pixel triples (q, r, p) with r in the stored lower
 * band of q and p coupled to both, summed over all periodic-band blocks (the
 * algorithmic multiply-adds of the B^T N^-1 B^ contraction); nmults the
 * products B^_pq N^-1_p formed once per coupled pair (q, p). */
int sympix_plan_counts(sympix_plan_t plan, int64_t *nslots, int64_t *npairs, int64_t *ntriples,
                       int64_t *nmults);

/* Number of library kernel launches one call of sympix_kernel_table,
 * sympix_sample_blocks and sympix_factor_blocks enqueues for a storage mode
 * and the contraction / factor arithmetic (SYMPIX_PREC_*). */
int sympix_plan_launches(sympix_plan_t plan, int storage, int sample_precision, int factor_precision,
                         int32_t *table, int32_t *sample, int32_t *factor);

/* Output size of sample/factor for a storage mode: bytes of the blocks
 * buffer (doubles) and the number of stored lower-triangle elements
 * (periodic band including the diagonal; n (n+1) / 2 for dense blocks). */
int sympix_blocks_size(sympix_plan_t plan, int storage, size_t *bytes, int64_t *elements);

/* Where block (op, ring) sits in the blocks buffer of a storage mode (on a
 * DP-grid plan `ring` is the band index, ring / k):
 * offset in doubles (a multiple of 4: every block starts on a 32-byte
 * boundary), ring size n, lower band half-width w, format
 * SYMPIX_BLOCK_PBAND or SYMPIX_BLOCK_DENSE.
 *   PBAND format: n (2w+1) doubles.  Sampled: band[q*(w+1) + d] =
 *   M[q][(q-d) mod n] for d = 0..w (the other entries follow by symmetry).
 *   Factored: with m = n - w, rows i < m of L as band[i*(w+1)+d] = L[i][i-d]
 *   (d <= min(i, w)); rows m..n-1 of L in the border that follows the band,
 *   border[(i-m)*n + c] = L[i][c] for c <= i.
 *   DENSE format: n*n doubles, row-major M; factored: L in the lower
 *   triangle (the strict upper triangle keeps M). */
int sympix_block_layout(sympix_plan_t plan, int storage, int op, int ring, int64_t *offset,
                        int32_t *n, int32_t *w, int32_t *format);

/* Device-side failures of the calls on a plan since the last query: waits
 * for the work on `stream` (and what precedes it), then reads and clears
 * the plan's device status word.  Returns SYMPIX_ETIMEOUT if a bounded wait
 * ran out (the FP32 factor then also set info = -1 for the blocks whose
 * factor it left incomplete), else SYMPIX_OK.  Synchronous.  The paper has
 * no counterpart: this reports on the execution, not the method. */
int sympix_plan_status(sympix_plan_t plan, void *stream);

/* The support radius operator `op` is planned with, and its margin (either
 * pointer may be NULL).  Coupling is the FP64 comparison
 * u <= u_s = 2 sin^2(r_s / 2) with u = 1 - cos(gamma) (the truncation of
 * Eq. f).  A pixel pair whose u lies within a few ulps of u_s could be
 * decided either way by another correct implementation (another sin), so
 * sympix_support measures, over every class of every coupled ring pair, the
 * smallest relative distance |u - u_s| / u_s; while it is <= 1e-12 the
 * radius is scaled by (1 - 1e-9) (at most 8 times).  *r_s receives the
 * radius used (the caller's unless that happened), *margin the final
 * smallest distance (+inf for r_s >= pi, where nothing is compared). */
int sympix_plan_radius(sympix_plan_t plan, int op, double *r_s, double *margin);

/* Device memory held by a plan (either pointer may be NULL): *bytes all of
 * it, *staging the part sympix_kernel_table allocates on its first call
 * (0 before that call).  For memory accounting and tests. */
int sympix_plan_device_bytes(sympix_plan_t plan, size_t *bytes, size_t *staging);

/* Per coupled ring pair (ring j of a planned block, neighbour ring rho):
 * the largest coupled separation index m (pixel pairs with
 * |(2c+1) n_rho - (2p+1) n_j| / gcd(n_j, n_rho) <= m couple), written for
 * every rho in [ring - radius, ring + radius] into mmax[rho - ring + radius]
 * (-1 where nothing couples).  For tests and diagnostics. */
int sympix_support_copy(sympix_plan_t plan, int op, int ring, int radius, int32_t *mmax);

/* ------------------------------------------------------------------------ */
/* Kernel table (Eq. addition-theorem)                                       */
/* ------------------------------------------------------------------------ */

/* Evaluate b(x) = sum_l (2l+1)/(4 pi) b_l P_l(x) at every symmetry-class
 * slot of every operator, and d(x) likewise at the same-ring slots.
 *   bl, dl  device arrays [nops][lmax+1] of b_l and d_l (row o = operator o).
 * FP64, O(lmax) per slot (Sec. 4.2).  Writes the plan's kernel tables; must
 * precede sympix_sample_blocks.  Asynchronous on `stream`. */
int sympix_kernel_table(sympix_plan_t plan, const double *bl, const double *dl, void *stream);

/* Same computation and outputs as sympix_kernel_table, for callers that
 * must not allocate device memory at the time of the call (for example
 * code that runs under a fixed device-memory budget reserved up front, or
 * whose allocator forbids the implicit device synchronisation cudaMalloc
 * brings).  sympix_kernel_table allocates its coefficient staging buffer on
 * first use; this entry point calls no cudaMalloc, cudaFree or other
 * allocating routine and stages the coefficients in one static device
 * array of 262144 doubles (2 MiB) that every GPU which loads the library
 * holds until the process exits.  (The paper has no counterpart; this is a
 * deployment variant.)
 *   Limit: 2 (lmax + 1) (nops + 1) <= 262144, else SYMPIX_EINVAL and
 *   nothing is launched.
 *   The plan (and its kernel tables) must already exist: create it with
 *   sympix_support beforehand.
 *   The first call on a device looks up the array's device address with
 *   that device current (a host-side query, done once per device); make
 *   that first call before any stream capture.
 *   Every call shares the one array and it keeps the last call's contents;
 *   nothing in it needs to start at zero (each launch writes every entry it
 *   reads).  Calls whose work overlaps on the GPU race on the array: issue
 *   them on one stream, or otherwise order them.
 * Asynchronous on `stream`. */
int sympix_kernel_table_static(sympix_plan_t plan, const double *bl, const double *dl, void *stream);

/* Copy operator `op`'s kernel values to the host: b at every slot of ring
 * pair (ring, rho) for separation indices m = par, par+2, ..., mmax
 * (par = mmax mod 2), count values; d likewise for rho == ring (NULL to
 * skip).  Synchronous.  For tests. */
int sympix_table_copy(sympix_plan_t plan, int op, int ring, int rho, int count, double *b,
                      double *d);

/* ------------------------------------------------------------------------ */
/* Blocks (Eq. Dhat, Eq. system-rewritten)                                   */
/* ------------------------------------------------------------------------ */

/* Sample every planned block  M = D^_jj + sum_p B^_pq N^-1_p B^_pr  (q, r on
 * ring j, p over all pixels; Y2 = Y1) for every operator.
 *   ninv       device [nops][npix] inverse noise N^-1 in pixel numbering.
 *   precision  SYMPIX_PREC_*: arithmetic of the contraction (the kernel
 *              values are FP64 in every mode; outputs are FP64).
 *   storage    SYMPIX_STORE_*.
 *   blocks     device buffer of sympix_blocks_size(storage) bytes.
 * One grouped launch covers every (operator, block, tile).  Asynchronous. */
int sympix_sample_blocks(sympix_plan_t plan, const double *ninv, int precision, int storage,
                         double *blocks, void *stream);

/* Cholesky-factor every sampled block in place, M = L L^T.
 *   blocks     the sampled blocks (sympix_sample_blocks), 16-byte aligned
 *              (cudaMalloc and PyTorch allocations are); SYMPIX_EINVAL
 *              otherwise.
 *   precision  arithmetic of the periodic-band factorisation:
 *              SYMPIX_PREC_FP64, SYMPIX_PREC_FP32X2 (split FP32, near-FP64
 *              accuracy on the FP32 pipes) or SYMPIX_PREC_FP32.  With FP32
 *              (PBAND storage) a block whose pivots shrink below the plan's
 *              pivot floor (SYMPIX_OPT_FP32_PIVOT_FLOOR) relative to their
 *              original diagonal is near-degenerate and is refactored in FP64
 *              on the device, except that a band wider than 16 whose FP32
 *              pivot falls to -1e-3 of its original diagonal or below fails
 *              at that row without the refactor (the FP32 pivot is within
 *              about (w+1) 2^-24 of the diagonal of the FP64 one, so FP64
 *              fails there too; the block is left as sampled).  Dense-format blocks (small or fully coupled
 *              rings) are factored in FP64 always; with FP32X2, bands wider
 *              than 16 are factored in FP64.
 *   info       device int32 [nops * nblocks] (operator-major, blocks in ring
 *              order): 0, or i+1 for the first row i whose pivot is not
 *              positive (that block's factor is then incomplete), or -1
 *              when a bounded device wait ran out before the block was
 *              factored (sympix_plan_status then reports SYMPIX_ETIMEOUT).
 * Asynchronous. */
int sympix_factor_blocks(sympix_plan_t plan, int storage, int precision, double *blocks, int32_t *info,
                         void *stream);

/* Pixel-domain convolution (Eq. convolution-pixel) of every operator's map
 * with its own kernel b (Eq. addition-theorem, from sympix_kernel_table),
 * truncated at the operator's radius r_s:
 *   g_q = sum over the pixels p with gamma_qp <= r_s of b(n_q . n_p) f_p.
 *   f, g       device FP64 [nops][npix] in the grid's pixel numbering; g is
 *              written at the pixels of the planned rings [ring0, ring1).
 *   precision  SYMPIX_PREC_*: arithmetic of the sums (FP64, FP32, or split
 *              FP32); f is split into FP32 planes in the plan's scratch, so
 *              calls on one plan must not overlap on the GPU.
 * Asynchronous. */
int sympix_convolve(sympix_plan_t plan, const double *f, int precision, double *g, void *stream);

/* ------------------------------------------------------------------------ */
/* Blocks between rings, and the preconditioner applied to a vector         */
/* ------------------------------------------------------------------------ */

/* Lay out the blocks M_jk between ring j and ring k = j + delta (delta >= 1)
 * of every operator, for every ring j with both j and k in the planned range
 * (Eq. system-rewritten and Eq. Dhat with rows on ring j and columns on ring
 * k: M_qr = [gamma_qr <= r_s] d(x_qr) + sum_p B^_pq N^-1_p B^_pr, p over
 * every pixel; M_kj = M_jk^T).  Entries vanish unless gamma_qr <= 2 r_s; row
 * q of a block stores the columns r = r0(q) + t (mod n_k), t = 0 .. K-1,
 * whose separation index z = (2q+1) Q - (2r+1) P (P = n_j / g, Q = n_k / g,
 * g = gcd(n_j, n_k)) satisfies |z| <= zmax, with
 * r0(q) = ceil(((2q+1) Q - zmax - P) / (2P)), zero past the row's own count;
 * a block with K >= n_k stores every column (r0 = 0, K = n_k).  *bytes and
 * *elements receive the size of the output buffer of sympix_sample_coupling.
 * Host bookkeeping plus one upload; synchronous.  After the first call for
 * any delta, sympix_kernel_table also evaluates d at the classes of
 * different rings (D^ between rings); call it again before sampling. */
int sympix_coupling_size(sympix_plan_t plan, int delta, size_t *bytes, int64_t *elements);

/* Layout of the block (op, ring j) for ring offset delta: *offset (doubles)
 * in the buffer and geom[7] = {rows n_j, columns n_k, K, zmax, P, Q,
 * dense (1: every column stored)}. */
int sympix_coupling_layout(sympix_plan_t plan, int delta, int op, int ring, int64_t *offset, int32_t *geom);

/* Sample every block between ring j and ring j + delta (FP64) into out
 * (device, sympix_coupling_size bytes) from ninv (device [nops][npix]) and the
 * plan's kernel tables.  Asynchronous. */
int sympix_sample_coupling(sympix_plan_t plan, const double *ninv, int delta, double *out, void *stream);

/* The block preconditioner applied to x: y_j = M_jj^-1 x_j on every planned
 * ring j of every operator (block Jacobi with the diagonal ring blocks), by
 * forward and back substitution with the factors of sympix_factor_blocks.
 *   blocks, info  the factored blocks of `storage` and their info array;
 *   x, y          device FP64 [nops][npix] in pixel numbering (must not
 *                 alias); y is written at the planned rings' pixels.  A block
 *                 whose factorisation failed (info != 0) passes x through.
 * FP64, one warp per block.  Asynchronous. */
int sympix_apply(sympix_plan_t plan, int storage, const double *blocks, const int32_t *info, const double *x,
                 double *y, void *stream);

void sympix_plan_free(sympix_plan_t plan);

/* ------------------------------------------------------------------------ */
/* Captured step (batching: one graph launch per stage)                     */
/* ------------------------------------------------------------------------ */

/* Capture the three calls above -- sympix_kernel_table(bl, dl),
 * sympix_sample_blocks(ninv, sample_precision, storage, blocks) and
 * sympix_factor_blocks(storage, factor_precision, blocks, info) -- into one
 * CUDA graph per stage on the current device, and instantiate them.  Nothing
 * runs.  The graphs keep the pointers: a replay reads bl, dl and ninv as they
 * are when it runs, so callers update inputs in place between replays.  The
 * device buffers, and the plan, must outlive the step.  The plan's scratch
 * (FP32 copies of N^-1, the factor's band shadow) is shared by the plan's
 * steps and direct calls: work on one plan must not overlap on the GPU.
 * Allocates the table's coefficient staging if no call has yet.  The paper
 * describes the method, not its launch; this is the grouped, graph-replayed
 * execution of the same three operations. */
int sympix_step_create(sympix_plan_t plan, const double *bl, const double *dl, const double *ninv,
                       int storage, int sample_precision, int factor_precision, double *blocks,
                       int32_t *info, sympix_step_t *out);

/* Replay the stages in `stages` (SYMPIX_STAGE_* bits, in the order table,
 * sample, factor) on `stream` (any stream of the step's device, including
 * the default stream).  Sampling without the table stage requires the plan's
 * table to have been computed.  Asynchronous. */
int sympix_step_launch(sympix_step_t step, int stages, void *stream);

/* Number of kernel launches one replay of `stages` performs. */
int sympix_step_kernels(sympix_step_t step, int stages, int64_t *count);

void sympix_step_free(sympix_step_t step);

/* Text of the calling thread's last error ("" if none). */
const char *sympix_last_error(void);

/* Library version string. */
const char *sympix_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SYMPIX_H */
