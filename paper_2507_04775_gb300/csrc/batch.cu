// Batched path: many HMult / HRotate / Rescale operations on ciphertexts at
// uneven levels, executed with one launch per step of the key switch for the
// whole batch instead of one launch per step per operation.
//
// The paper hides the CPU's launch overhead with limb batching over streams
// (Sec. III-F1).  Here every step of every operation of a batch becomes part
// of one launch: fides_batch_create builds, once, device-resident tables of
// NTT segments, base-conversion jobs and element-wise descriptors for all
// operations (with their own scratch), and fides_batch_run replays the fixed
// sequence of launches -- about ten per stage however many operations the
// stage holds -- optionally as one captured CUDA graph.  Operations are
// grouped in stages: an operation of stage s may read the outputs of stages
// < s; operations of one stage are independent.
#include <algorithm>
#include <cstring>
#include <vector>

#include "fides_internal.cuh"
#include "launchplan.cuh"

struct fides_batch {
    fides_ctx *ctx;
    std::vector<Launch> launches;
    unsigned char *dmem;      // device tables
    u64 *scratch;             // scratch of every operation
    size_t table_bytes, scratch_bytes;
    cudaGraphExec_t exec;     // captured run, or null
};

extern "C" int fides_batch_create(fides_ctx *c, fides_op *ops, int n_ops, fides_batch **out)
{
    if (!out) return fides_set_error(FIDES_ERR_ARG, "fides_batch_create: out is NULL");
    *out = nullptr;
    if (!c || (n_ops > 0 && !ops) || n_ops < 0) return fides_set_error(FIDES_ERR_ARG, "fides_batch_create: bad arguments");
    int nstage = 0;
    for (int i = 0; i < n_ops; ++i) {
        if (int rc = plan_validate(c, ops[i], i, "fides_batch_create")) return rc;
        nstage = std::max(nstage, ops[i].stage + 1);
    }
    // scratch of every operation
    std::vector<size_t> soff(n_ops);
    size_t words = 0;
    for (int i = 0; i < n_ops; ++i) {
        soff[i] = words;
        words += op_scratch_words(c->N, c->K, c->alpha, ops[i].type, ops[i].a.n_limbs);
    }

    fides_batch *b = new fides_batch();
    b->ctx = c;
    b->dmem = nullptr;
    b->exec = nullptr;
    b->scratch = nullptr;
    b->scratch_bytes = words * sizeof(u64);
    if (words) {
        int rc = fides_check_cuda(cudaMalloc((void **)&b->scratch, b->scratch_bytes), "fides_batch_create: scratch");
        if (rc) { delete b; return rc; }
    }
    std::vector<u64 *> scr(n_ops);
    for (int i = 0; i < n_ops; ++i) scr[i] = b->scratch + soff[i];
    Plan P;
    for (int s = 0; s < nstage; ++s) plan_stage(c, ops, n_ops, s, scr.data(), P);
    b->table_bytes = P.image.size();
    if (b->table_bytes) {
        int rc = fides_check_cuda(cudaMalloc((void **)&b->dmem, b->table_bytes), "fides_batch_create: tables");
        if (!rc) rc = fides_check_cuda(cudaMemcpy(b->dmem, P.image.data(), b->table_bytes, cudaMemcpyHostToDevice),
                                       "fides_batch_create: upload");
        if (rc) { fides_batch_destroy(b); return rc; }
    }
    plan_patch(P, b->dmem);
    b->launches.swap(P.launches);
    *out = b;
    return FIDES_OK;
}

extern "C" void fides_batch_destroy(fides_batch *b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    cudaFree(b->dmem);
    cudaFree(b->scratch);
    delete b;
}

extern "C" int fides_batch_run(fides_batch *b, void *stream)
{
    if (!b) return fides_set_error(FIDES_ERR_ARG, "fides_batch_run: NULL batch");
    cudaStream_t st = (cudaStream_t)stream;
    OpTrace op("op_batch", st);
    if (b->exec) return fides_check_cuda(cudaGraphLaunch(b->exec, st), "fides_batch_run: graph launch");
    return plan_run(b->ctx, b->launches, st);
}

extern "C" int fides_batch_capture(fides_batch *b, void *stream)
{
    if (!b) return fides_set_error(FIDES_ERR_ARG, "fides_batch_capture: NULL batch");
    if (!stream) return fides_set_error(FIDES_ERR_ARG, "fides_batch_capture: needs a non-default stream");
    cudaStream_t st = (cudaStream_t)stream;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    const int was = fides_trace_set(0);   // no event records inside the graph
    cudaGraph_t g = nullptr;
    int rc = fides_check_cuda(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (!rc) {
        int rc2 = plan_run(b->ctx, b->launches, st);
        rc = fides_check_cuda(cudaStreamEndCapture(st, &g), "end capture");
        if (!rc) rc = rc2;
    }
    if (!rc) rc = fides_check_cuda(cudaGraphInstantiate(&b->exec, g, 0), "graph instantiate");
    if (g) cudaGraphDestroy(g);
    fides_trace_set(was);
    return rc;
}

extern "C" int fides_batch_info(const fides_batch *b, int *launches, size_t *scratch_bytes, size_t *table_bytes)
{
    if (!b) return fides_set_error(FIDES_ERR_ARG, "fides_batch_info: NULL batch");
    const int n = plan_kernel_count(b->ctx, b->launches);
    if (launches) *launches = n;
    if (scratch_bytes) *scratch_bytes = b->scratch_bytes;
    if (table_bytes) *table_bytes = b->table_bytes;
    return FIDES_OK;
}
