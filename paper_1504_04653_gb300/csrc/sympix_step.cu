// The whole per-problem step -- kernel table, block sampling, Cholesky --
// captured once into CUDA graphs and replayed.
//
// A step of the method is a fixed sequence of launches whose shapes depend
// only on the plan, so after the first capture a replay costs one graph
// launch per stage instead of a dozen kernel launches and their host-side
// argument set-up.  Each stage (table, sample, factor) is captured into its
// own graph so a caller may replay a subset (e.g. resample and refactor for
// a new N^-1 with the same beams) or time the stages separately.
#include <cuda_runtime.h>

#include "sympix_internal.cuh"

struct sympix_step_s {
    sympix_plan_t plan = nullptr;
    int device = 0;
    cudaGraph_t graph[3] = {nullptr, nullptr, nullptr};
    cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};
};

using namespace sympix;

static void step_destroy(sympix_step_t s) {
    if (!s) return;
    for (int i = 0; i < 3; ++i) {
        if (s->exec[i]) cudaGraphExecDestroy(s->exec[i]);
        if (s->graph[i]) cudaGraphDestroy(s->graph[i]);
    }
    delete s;
}

extern "C" int sympix_step_create(sympix_plan_t pl, const double *bl, const double *dl, const double *ninv,
                                  int storage, int sample_precision, int factor_precision, double *blocks,
                                  int32_t *info, sympix_step_t *out) {
    if (!pl || !bl || !dl || !ninv || !blocks || !info || !out)
        return set_error(SYMPIX_EINVAL, "sympix_step_create: NULL argument");
    *out = nullptr;
    if (storage != SYMPIX_STORE_PBAND && storage != SYMPIX_STORE_DENSE)
        return set_error(SYMPIX_EINVAL, "sympix_step_create: unknown storage %d", storage);
    if (sample_precision < SYMPIX_PREC_FP64 || sample_precision > SYMPIX_PREC_FP32X2 ||
        factor_precision < SYMPIX_PREC_FP64 || factor_precision > SYMPIX_PREC_FP32X2)
        return set_error(SYMPIX_EINVAL, "sympix_step_create: unknown precision (%d, %d)", sample_precision,
                         factor_precision);
    // the table call allocates its coefficient staging on first use, which a
    // capture must not do: allocate it here
    const size_t L1 = (size_t)pl->grid->lmax + 1;
    const size_t need = 2 * L1 + 2 * (size_t)pl->nops * L1;
    int rc;
    if (pl->d_rec.n < need && (rc = pl->d_rec.alloc(need))) return rc;

    sympix_step_s *s = new sympix_step_s;
    s->plan = pl;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) {
        delete s;
        return cuda_error(e, "sympix_step_create: cudaGetDevice");
    }
    // capture on a private stream: the legacy default stream cannot be captured
    cudaStream_t cs = nullptr;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete s;
        return cuda_error(e, "sympix_step_create: cudaStreamCreateWithFlags");
    }
    const bool was_ready = pl->table_ready;
    rc = SYMPIX_OK;
    for (int stage = 0; stage < 3 && rc == SYMPIX_OK; ++stage) {
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            rc = cuda_error(e, "sympix_step_create: cudaStreamBeginCapture");
            break;
        }
        int crc;
        if (stage == 0)
            crc = sympix_kernel_table(pl, bl, dl, cs);
        else if (stage == 1)
            crc = sympix_sample_blocks(pl, ninv, sample_precision, storage, blocks, cs);
        else
            crc = sympix_factor_blocks(pl, storage, factor_precision, blocks, info, cs);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cs, &g);
        if (crc != SYMPIX_OK) {
            if (g) cudaGraphDestroy(g);
            rc = crc;  // the failing call's message stands
            break;
        }
        if (e != cudaSuccess) {
            rc = cuda_error(e, "sympix_step_create: cudaStreamEndCapture");
            break;
        }
        s->graph[stage] = g;
        e = cudaGraphInstantiate(&s->exec[stage], g, 0);
        if (e != cudaSuccess) rc = cuda_error(e, "sympix_step_create: cudaGraphInstantiate");
    }
    // capturing the table stage ran nothing: the table is as ready as before
    pl->table_ready = was_ready;
    cudaStreamDestroy(cs);
    if (rc != SYMPIX_OK) {
        step_destroy(s);
        return rc;
    }
    *out = s;
    return SYMPIX_OK;
}

extern "C" int sympix_step_launch(sympix_step_t s, int stages, void *stream) {
    if (!s) return set_error(SYMPIX_EINVAL, "sympix_step_launch: NULL step");
    if (stages <= 0 || (stages & ~SYMPIX_STAGE_ALL))
        return set_error(SYMPIX_EINVAL, "sympix_step_launch: stage mask %d", stages);
    if (!(stages & SYMPIX_STAGE_TABLE) && (stages & SYMPIX_STAGE_SAMPLE) && !s->plan->table_ready)
        return set_error(SYMPIX_EINVAL, "sympix_step_launch: sampling without a kernel table");
    int dev = 0;
    SPX_CUDA(cudaGetDevice(&dev));
    if (dev != s->device)
        return set_error(SYMPIX_EINVAL, "sympix_step_launch: step captured on device %d, device %d is current",
                         s->device, dev);
    cudaStream_t st = (cudaStream_t)stream;
    const int bits[3] = {SYMPIX_STAGE_TABLE, SYMPIX_STAGE_SAMPLE, SYMPIX_STAGE_FACTOR};
    for (int i = 0; i < 3; ++i)
        if (stages & bits[i]) {
            cudaError_t e = cudaGraphLaunch(s->exec[i], st);
            if (e != cudaSuccess) return cuda_error(e, "sympix_step_launch: cudaGraphLaunch");
            if (i == 0) s->plan->table_ready = true;
        }
    return SYMPIX_OK;
}

extern "C" int sympix_step_kernels(sympix_step_t s, int stages, int64_t *count) {
    if (!s || !count) return set_error(SYMPIX_EINVAL, "sympix_step_kernels: NULL argument");
    if (stages <= 0 || (stages & ~SYMPIX_STAGE_ALL))
        return set_error(SYMPIX_EINVAL, "sympix_step_kernels: stage mask %d", stages);
    const int bits[3] = {SYMPIX_STAGE_TABLE, SYMPIX_STAGE_SAMPLE, SYMPIX_STAGE_FACTOR};
    int64_t total = 0;
    for (int i = 0; i < 3; ++i) {
        if (!(stages & bits[i])) continue;
        size_t nn = 0;
        SPX_CUDA(cudaGraphGetNodes(s->graph[i], nullptr, &nn));
        if (nn == 0) continue;
        cudaGraphNode_t *nodes = new cudaGraphNode_t[nn];
        cudaError_t e = cudaGraphGetNodes(s->graph[i], nodes, &nn);
        if (e != cudaSuccess) {
            delete[] nodes;
            return cuda_error(e, "sympix_step_kernels: cudaGraphGetNodes");
        }
        for (size_t k = 0; k < nn; ++k) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[k], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++total;
        }
        delete[] nodes;
    }
    *count = total;
    return SYMPIX_OK;
}

extern "C" void sympix_step_free(sympix_step_t s) { step_destroy(s); }
