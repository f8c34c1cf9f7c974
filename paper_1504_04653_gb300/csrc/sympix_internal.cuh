// Internal types shared by the translation units of libsympix.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include "../../include/sympix.h"

namespace sympix {

constexpr double kPi = 3.14159265358979323846;

// -- errors ------------------------------------------------------------------
int set_error(int code, const char *fmt, ...);
int cuda_error(cudaError_t e, const char *what);

#define SPX_CUDA(call)                                        \
    do {                                                      \
        cudaError_t e__ = (call);                             \
        if (e__ != cudaSuccess) return cuda_error(e__, #call); \
    } while (0)

// Record a trace event on `st` (no-op unless the plan traces and `st` is not
// capturing); `name` labels the span since the previous mark, null starts a call.
void trace_mark(sympix_plan_t pl, cudaStream_t st, const char *name);
// The canonical form of ring pair (j, rho) of a grid of N rings: a <= b and
// a <= N-1-b (transposed and north/south-mirrored pairs share kernel values).
// DP-grid plans (sympix_tiles.cu): the largest |z| of a tile-coupled pixel
// pair of two ring sizes; the band blocks of bands [g0, g1); their sampler.
long tile_pair_mmax(int na, int nb, int k, bool all);
int plan_tile_blocks(sympix_plan_t pl, const std::unordered_map<int64_t, int> &index, int g0, int g1);
int launch_tiles(sympix_plan_t pl, const double *ninv, int precision, double *blocks, cudaStream_t st);
inline std::pair<int, int> canon_pair(int N, int j, int rho) {
    int a = j < rho ? j : rho, b = j < rho ? rho : j;
    if (a > N - 1 - b) {
        const int a2 = N - 1 - b, b2 = N - 1 - a;
        a = a2;
        b = b2;
    }
    return {a, b};
}
// columns per chunk of the chunked border solve for width w, and the floats
// of its per-item scratch (a W x W matrix, the corner sums) for 32 lanes
int l21_chunk_cols_host(int w);
int l21_mat_floats();
int l21_pair_floats();
// whether the split FP32 launch of a plan's w <= 8 slices can have every CTA
// resident at once (sympix_factor_split.cu)
bool f32_split_fits(sympix_plan_t pl);

// Widest band of the narrow-band factor (k_pband_chol), and the elements of
// one tile of its FP32 commit.
constexpr int kNarrowWMax = 12;
constexpr int kCommitTileElems = 2048;

// Smallest relative distance |u - u_s| / u_s a support class may have from
// the coupling threshold before the radius is scaled by (1 - 1e-9).
constexpr double kSupportMargin = 1e-12;

// Elements of a dense-format block sampled by one CTA (a warp each).
constexpr int kDenseItemElems = 8;

// Elements per block in one CTA of the FP32 shadow transposes (x 32 blocks).
constexpr int kTileE = 128;

// Wide-band factor kernel (16 < w <= 64): each thread holds kWideE entries of
// one column slot of the window (G = ceil((2w+1) / kWideE) threads per slot,
// w+1 slots); CTAs of up to kWideMaxThreads threads.
constexpr int kWideE = 24;
constexpr int kWideMaxThreads = 416;
inline int wide_threads(int w) {
    const int t = (2 * w + 1 + kWideE - 1) / kWideE * (w + 1);
    return t;
}
// One launch of the wide kernel: items [begin, begin + count) of list 5,
// CTAs of `threads`, shared memory sized for the widest band `wmax`.
struct WideClass {
    int begin, count, threads, wmax;
};

// FP64 [count] -> FP32 hi and lo planes (integer-ALU split; sympix_sample.cu).
__global__ void k_split_ninv(int64_t count, const double *__restrict__ ninv, float *__restrict__ n32,
                             float *__restrict__ nlo);

// Device buffer owned by a handle.  Movable, not copyable: a copy would free
// the memory twice.
template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), n(o.n) {
        o.p = nullptr;
        o.n = 0;
    }
    DevBuf &operator=(DevBuf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p;
            n = o.n;
            o.p = nullptr;
            o.n = 0;
        }
        return *this;
    }
    int alloc(size_t count) {
        release();
        if (count == 0) return SYMPIX_OK;
        cudaError_t e = cudaMalloc(&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            (void)cudaGetLastError();
            return set_error(SYMPIX_ENOMEM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                             cudaGetErrorString(e));
        }
        n = count;
        return SYMPIX_OK;
    }
    int upload(const std::vector<T> &v) {
        int rc = alloc(v.size());
        if (rc) return rc;
        if (!v.empty()) SPX_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
        return SYMPIX_OK;
    }
    size_t bytes() const { return n * sizeof(T); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    ~DevBuf() { release(); }
};

}  // namespace sympix

// -- grid ---------------------------------------------------------------------
struct sympix_grid_s {
    int lmax = 0, k = 1, layout = 0, nrings = 0, nbands = 0, max_ring = 0;
    int64_t npix = 0;
    std::vector<double> theta;          // ring colatitudes, north to south
    std::vector<int32_t> nring, stride; // pixels per ring; column step in the numbering
    std::vector<int64_t> offset;        // pixel index of column 0
    sympix::DevBuf<double> d_theta;
};

// One coupled ordered ring pair (ring j of a block, neighbour ring rho).
// Pixel c of ring j and pixel p of ring rho are at separation index
// z = (2c+1) Q - (2p+1) P, with P = n_j / g, Q = n_rho / g, g = gcd; they
// couple iff |z| <= mmax, and their kernel value is table[tab + (|z|-par)/2].
struct PairEntry {
    int32_t rho;
    int32_t P, Q;
    int32_t mmax;
    int32_t par;
    int32_t nrho;
    int32_t nstride;
    int32_t pad;
    int64_t tab;
    int64_t noff;
};

// One planned block (operator op, ring ring).
struct BlockDesc {
    int32_t op, ring, n, w;
    int32_t format;   // SYMPIX_BLOCK_PBAND / SYMPIX_BLOCK_DENSE
    int32_t npairs;   // coupled neighbour rings
    int64_t pair0;    // first PairEntry
    int64_t off_pband, off_dense;  // offsets (doubles) in the two storage modes
    int64_t dtab;     // slot of level 0 of the same-ring pair
    int32_t dK;       // same-ring levels (D support)
    int32_t pad;
};

// One canonical ring pair (a <= b, a <= N-1-b): the kernel values of the
// transposed and the north/south mirrored pair are the same.
struct CanonPair {
    int32_t a, b;
    int32_t na, nb;
    int32_t g;
    int32_t kmax;   // levels stored (max over operators)
    int64_t slot0;  // first slot
};

// DP grids (k > 1): one dense block per band of k rings, under tile
// adjacency.  A block's rows are the band's pixels in grid order (pixel c
// of the band's r-th ring at row c k + r), so tile a (columns a k .. a k +
// k - 1) is rows a k^2 .. a k^2 + k^2 - 1.
constexpr int kTileKMax = 8;  // k^2 <= 64 pixels per tile
struct TileBlock {
    int32_t op, g;         // operator, band (latitude order, g = ring / k)
    int32_t K, T;          // rows (k n_g), tiles of the band
    int32_t k, G;          // tile size, bands of the grid
    int32_t gnb[3];        // bands g-1, g, g+1 (-1 where none)
    int32_t Tnb[3];        // their tiles
    int32_t P[3], Q[3];    // separation-index steps against each (ring of band g first)
    int32_t par[3], pad;
    int64_t half[3];       // P Q gcd: z reduced to (-half, half]
    int64_t off;           // first element of the block (dense K x K, row-major)
    int64_t meta0;         // first of its 3 k^2 slot bases and 3 k ring offsets
};
// One lower tile pair (a2 <= a) of a block with some coupling.
struct TileItem {
    int32_t block, a, a2, pad;
};

// Work item of the sampling launches.
struct SampleItem {
    int32_t block;
    int32_t q0;
};

// Up to 32 periodic-band blocks of one width w <= 16 factored together in
// FP32: blocks f32_items[first .. first+count), at most `rows` rows each.
// Their lane-interleaved band shadow starts at float offset `sh` (rows x
// (w+1) x 32) and their FP32 border rows L21 at `l21` (w x (rows-w) x 32).
struct F32Slice {
    int32_t w, first, count, rows;
    int64_t sh, l21;
};

// One warp of the narrow-band factor: blocks chol_items[first .. first+count)
// of exact width w <= 12, factored with g lanes each (count <= 32 / g).
struct CholSlice {
    int32_t w, first, count, g;
};

// One tile of the pixel-domain convolution: pixels q0 .. q0+127 of block
// `block`'s ring, whose column c is output pixel goff + c * gstride.
struct ConvItem {
    int32_t block, q0;
    int64_t goff;
    int32_t gstride, pad;
};

// One off-diagonal block (rows on ring j of block bj, columns on ring k of
// block bk): pair constants P = n_j / g, Q = n_k / g, stored separations
// |z| <= zmax in rows of K entries (every column when dense), at offset off;
// dpair: the (j, k) entry of block bj (D^ between the rings), or -1.
struct CoupDesc {
    int64_t off;
    int32_t bj, bk, n, K, zmax, P, Q, dense, dpair, pad;
};

struct CouplingPlan {
    std::vector<CoupDesc> desc;
    int64_t total = 0;  // stored entries
    sympix::DevBuf<CoupDesc> d_desc;
};

struct sympix_plan_s {
    sympix_grid_t grid = nullptr;
    int nops = 0, ring0 = 0, ring1 = 0;
    std::vector<double> r_s;            // radius used per operator (after the margin guard)
    std::vector<double> margin;         // smallest |u - u_s| / u_s per operator
    std::vector<int> radius;            // ring offset bound per operator
    std::vector<CanonPair> pairs;       // canonical pairs
    std::vector<int32_t> pair_mmax;     // [pair][op]
    std::vector<BlockDesc> blocks;      // [op][ring1-ring0]
    std::vector<PairEntry> entries;
    int64_t nslots = 0;
    int64_t ntriples = 0, nmults = 0;
    int64_t elems_pband = 0, elems_dense = 0;
    int64_t size_pband = 0, size_dense = 0;  // doubles
    int max_w = 0;
    // sampling schedule (built once)
    std::vector<SampleItem> items_pband[5];  // buckets of WMAX = 8,16,32,64,128
    std::vector<SampleItem> items_dense;       // dense-format blocks with n <= 64: a warp per element
    std::vector<SampleItem> items_dense_rows;  // larger ones: a thread per element, 256 per CTA
    std::vector<ConvItem> items_conv;  // every block in tiles of 128 pixels
    // factorisation work lists, each most expensive first: periodic band with
    // [0] w <= 8, [1] 8 < w <= 12, [2] 12 < w <= 16, [5] 16 < w <= 64;
    // [3] dense format with n <= 1024; [4] everything else
    std::vector<int32_t> factor_items[6];
    std::vector<sympix::WideClass> wide_cls;  // list 5 by CTA size
    // FP32 factorisation on a band shadow: periodic-band blocks with w <= 16
    // grouped by exact width into slices of up to 32 blocks; each slice's
    // shadow is lane-interleaved (element e of its block L at 32 e + L)
    std::vector<int32_t> f32_items;
    std::vector<F32Slice> f32_slices;
    std::vector<int2> f32_tiles;  // (slice, first element) of the band shadow transposes
    std::vector<int2> f32_out_tiles;  // the same, then (slice, -1 - first element) of L21
    int f32_slices_fused = 0;     // slices with w <= 12, band and border fused (they come first)
    int f32_slices_w8 = 0;        // of those, the slices with w <= 8 (they come first)
    // border rows of the fused-range slices by column chunks: work items
    // (slice, chunk) with each slice's chunks consecutive, the slices with
    // w >= 1, each slice's first item and chunk count, and per item the
    // W x W transfer, particular and start windows and the corner sums
    std::vector<int2> l21_items;
    std::vector<int32_t> l21_slices, l21_first, l21_nch;
    int l21_items_w8 = 0;   // items of slices with w <= 8 (they come first)
    int l21_slices_w8 = 0;  // entries of l21_slices with w <= 8 (they come first)
    sympix::DevBuf<int2> d_l21_items;
    sympix::DevBuf<int32_t> d_l21_slices, d_l21_first, d_l21_nch;
    sympix::DevBuf<float> d_l21_T, d_l21_P, d_l21_S, d_l21_C;
    // the split FP32 factor: per fused-range slice a progress and a done word
    // (zero between launches) and the band passes' results
    sympix::DevBuf<int> d_split_flags, d_split_bandres;
    cudaStream_t f32_side = nullptr;  // the fused 9 <= w <= 12 slices beside the w <= 8 ones
    cudaEvent_t f32_fork = nullptr, f32_join = nullptr;
    // the f32 transposes of slices with w > 12 only (the narrow-band factor
    // covers w <= 12 unless the two-role fused kernel is selected)
    std::vector<int2> f32_tiles_hi, f32_out_tiles_hi;
    // ... and of slices with w <= 12 only (the FP64 path's shadow)
    std::vector<int2> f32_tiles_lo, f32_out_tiles_lo;
    int64_t size_shadow_hi = 0, size_l21_hi = 0;  // floats of the w > 12 slices (they come first in the buffers)
    // narrow-band factor (w <= 12, periodic-band storage): blocks by width,
    // most expensive first; slices for FP32 (8 lanes) and for FP64 / split
    // FP32 (4 lanes up to w = 8, then 8); commit tiles (block, first element)
    std::vector<int32_t> chol_items;
    std::vector<CholSlice> chol_sl32, chol_sl64;
    std::vector<int2> chol_tiles;
    int chol_wmax = -1;
    // per width: the slices [chol_f32[w], + chol_n32[w]) of chol_sl32 and
    // [chol_f64[w], + chol_n64[w]) of chol_sl64; a stream per width present
    // (the widths run side by side) and the fork / join events
    int chol_f32[sympix::kNarrowWMax + 1] = {0}, chol_n32[sympix::kNarrowWMax + 1] = {0};
    int chol_f64[sympix::kNarrowWMax + 1] = {0}, chol_n64[sympix::kNarrowWMax + 1] = {0};
    cudaStream_t chol_st[sympix::kNarrowWMax + 1] = {nullptr};
    cudaEvent_t chol_fork = nullptr, chol_join[sympix::kNarrowWMax + 1] = {nullptr};
    cudaStream_t chol_side = nullptr;  // the lane-group kernel beside the narrow kernels (FP64, split FP32)
    cudaEvent_t chol_side_join = nullptr;
    // kernel for periodic bands w <= 12, per factor arithmetic (SYMPIX_PREC_*):
    // 0 k_pband_chol (G lanes per block), 1 the earlier kernels (FP32: the
    // two-role kernel on an FP32 band copy; FP64 / split FP32: lane groups),
    // 2 band pass and chunked border solve on a shadow of the arithmetic,
    // 3 (FP32) band and border CTAs of one cooperative launch for w <= 8, 2
    // for 9 <= w <= 12.  Defaults from measurement at l_max = 3000 (factor
    // stage): FP64 2 (12.9 ms; 0: 20.1 ms), FP32 3, split FP32 2 (6.0 ms;
    // 1: 30.2 ms).
    int narrow_pref[3] = {2, 3, 2};
    // DP-grid plans (k > 1): band blocks under tile adjacency
    bool tiles = false;
    std::vector<TileBlock> tile_blocks;
    std::vector<TileItem> tile_items;
    std::vector<int64_t> tile_slot0;  // per block: [3][k][k] slot of (ring r of g, ring r2 of band d)
    std::vector<int64_t> tile_noff;   // per block: [3][k] pixel index of column 0 of ring r2 of band d
    sympix::DevBuf<TileBlock> d_tile_blocks;
    sympix::DevBuf<TileItem> d_tile_items;
    sympix::DevBuf<int64_t> d_tile_slot0, d_tile_noff;
    int64_t size_shadow_il = 0, size_l21_il = 0;  // floats
    // device
    sympix::DevBuf<CanonPair> d_pairs;
    sympix::DevBuf<double> d_slot_u;         // u = 1 - cos(gamma) per slot
    sympix::DevBuf<int32_t> d_slot_pair;     // canonical pair of each slot
    sympix::DevBuf<double> d_tab_b, d_tab_d; // [op][nslots] FP64
    sympix::DevBuf<float> d_tab_b32;         // [op][nslots] FP32 (rounded)
    sympix::DevBuf<float> d_tab_blo;         // [op][nslots] FP32 remainder b - hi
    sympix::DevBuf<float> d_tab_d32, d_tab_dlo; // the same split of d
    sympix::DevBuf<float> d_ninv32, d_ninvlo;   // [op][npix] split of N^-1, per sampling call
    sympix::DevBuf<double> d_rec;            // recurrence coefficients
    sympix::DevBuf<BlockDesc> d_blocks;
    sympix::DevBuf<PairEntry> d_entries;
    sympix::DevBuf<SampleItem> d_items_pband[5];
    sympix::DevBuf<SampleItem> d_items_dense, d_items_dense_rows;
    sympix::DevBuf<ConvItem> d_items_conv;
    sympix::DevBuf<int32_t> d_factor_items[6];
    sympix::DevBuf<int32_t> d_f32_items;
    sympix::DevBuf<F32Slice> d_f32_slices;
    sympix::DevBuf<int2> d_f32_tiles;
    sympix::DevBuf<float> d_shadow_il;  // lane-interleaved FP32 band rows, w <= 16
    sympix::DevBuf<float> d_l21_il;     // lane-interleaved FP32 border rows, w <= 16
    sympix::DevBuf<int2> d_f32_out_tiles;
    sympix::DevBuf<float> d_shadow;     // FP32 band rows of wide blocks / FP32 L11 of narrow ones, at their pband offsets
    sympix::DevBuf<int32_t> d_chol_items;
    sympix::DevBuf<CholSlice> d_chol_sl32, d_chol_sl64;
    sympix::DevBuf<int2> d_chol_tiles, d_f32_tiles_hi, d_f32_out_tiles_hi, d_f32_tiles_lo, d_f32_out_tiles_lo;
    bool table_ready = false;
    // blocks between rings: their layouts per ring offset; d evaluated at every
    // class (not only the same-ring ones) once such a layout exists
    std::map<int, CouplingPlan> coupling;
    bool all_d = false, table_all_d = false;
    sympix::DevBuf<int64_t> d_ring_off;  // the grid's ring offsets and strides (the apply's pixel addresses)
    sympix::DevBuf<int32_t> d_ring_stride;
    // tracing (SYMPIX_OPT_TRACE): an event after every launch of a traced
    // call; a null name marks the start of a call
    int table_cta = 32, border_threads = 512;  // launch shapes (autotuned)
    bool trace = false;
    std::vector<cudaEvent_t> trace_ev;
    std::vector<const char *> trace_name;
    int trace_n = 0;
    ~sympix_plan_s() {
        for (cudaEvent_t e : trace_ev) cudaEventDestroy(e);
        for (int w = 0; w <= sympix::kNarrowWMax; ++w) {
            if (chol_st[w]) cudaStreamDestroy(chol_st[w]);
            if (chol_join[w]) cudaEventDestroy(chol_join[w]);
        }
        if (chol_fork) cudaEventDestroy(chol_fork);
        if (chol_side) cudaStreamDestroy(chol_side);
        if (chol_side_join) cudaEventDestroy(chol_side_join);
        if (f32_side) cudaStreamDestroy(f32_side);
        if (f32_fork) cudaEventDestroy(f32_fork);
        if (f32_join) cudaEventDestroy(f32_join);
    }
    double fp32_pivot_floor = 0.05;  // FP32 factor: rescue in FP64 below this pivot ratio
    // device status word (bit 1: a bounded wait ran out), read and cleared by
    // sympix_plan_status; polls per bounded wait (SYMPIX_OPT_WAIT_LIMIT)
    sympix::DevBuf<int32_t> d_status;
    int wait_limit = 1 << 22;
};
