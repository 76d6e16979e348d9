// Batched path: many HMult / HRotate / Rescale operations on ciphertexts at
// uneven levels, executed with one launch per step of the key switch for a
// whole launch group instead of one launch per step per operation.
//
// The paper hides the CPU's launch overhead with limb batching over streams
// and notes that the batch size trades parallelism against cache locality
// (Sec. III-F1, Sec. IV).  Here the operations of a stage are split into
// launch groups of at most `group_limbs` ciphertext limbs (0: the whole stage
// is one group); every step of every operation of a group becomes part of one
// launch.  fides_batch_create builds, once, device-resident tables of NTT
// segments, base-conversion jobs and element-wise descriptors for all groups,
// and fides_batch_run replays the fixed sequence of launches -- about ten per
// group -- optionally as one captured CUDA graph.  Groups run one after
// another, so they share one scratch pool sized for the largest group (a
// stage's groups and the groups of later stages reuse it).  Operations are
// grouped in stages: an operation of stage s may read the outputs of stages
// < s; operations of one stage are independent.
//
// fides_batch_autotune times candidate group sizes, both placements of the
// HMult tensor product (its own pass, or fused into the first INTT pass) and
// both limb orders of the NTT launches (as planned, or by prime) on the batch
// itself and keeps the fastest.
#include <algorithm>
#include <cstring>
#include <vector>

#include "fides_internal.cuh"
#include "launchplan.cuh"

struct fides_batch {
    fides_ctx *ctx;
    std::vector<fides_op> ops;   // the operations (out.scale set)
    int nstage;
    int group_limbs;             // limbs per launch group, 0: one group per stage
    int tensor_split;            // HMult tensor product as its own pass (1) or fused (0)
    int prime_order;             // NTT launches visit their limbs by prime (1) or as planned (0)
    int groups;                  // launch groups of the current plan
    std::vector<Launch> launches;
    unsigned char *dmem;         // device tables
    size_t dmem_cap;
    u64 *scratch;                // one launch group's scratch, shared by all groups
    size_t scratch_cap;          // words allocated
    size_t table_bytes, scratch_bytes;
    cudaGraphExec_t exec;        // captured run, or null
};

namespace {

// Groups of op indices: per stage in order, consecutive ops of the stage while
// their limbs fit in group_limbs (at least one op per group).
std::vector<std::vector<int>> batch_groups(const std::vector<fides_op> &ops, int nstage, int group_limbs)
{
    std::vector<std::vector<int>> gs;
    for (int s = 0; s < nstage; ++s) {
        std::vector<int> cur;
        int limbs = 0;
        for (int i = 0; i < (int)ops.size(); ++i) {
            if (ops[i].stage != s) continue;
            const int nl = ops[i].a.n_limbs;
            if (!cur.empty() && group_limbs > 0 && limbs + nl > group_limbs) {
                gs.push_back(cur);
                cur.clear();
                limbs = 0;
            }
            cur.push_back(i);
            limbs += nl;
        }
        if (!cur.empty()) gs.push_back(cur);
    }
    return gs;
}

// (Re)builds the launch plan for a group size and tensor placement: grows the
// scratch pool and the table buffer when needed (shrink: also reallocates a
// pool larger than the plan needs), uploads the tables and drops a captured
// graph.  Synchronises the device before it frees anything.
int batch_build(fides_batch *b, int group_limbs, int tensor_split, int prime_order, bool shrink = true)
{
    const fides_ctx *c = b->ctx;
    const std::vector<std::vector<int>> gs = batch_groups(b->ops, b->nstage, group_limbs);
    size_t words = 0;
    for (const std::vector<int> &g : gs) {
        size_t w = 0;
        for (int i : g) w += op_scratch_words(c->N, c->K, c->alpha, b->ops[i].type, b->ops[i].a.n_limbs);
        words = std::max(words, w);
    }
    if (int rc = fides_check_cuda(cudaDeviceSynchronize(), "fides_batch: synchronise")) return rc;
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (words > b->scratch_cap || (shrink && words < b->scratch_cap)) {
        cudaFree(b->scratch);
        b->scratch = nullptr;
        b->scratch_cap = 0;
        if (int rc = fides_check_cuda(cudaMalloc((void **)&b->scratch, words * sizeof(u64)), "fides_batch: scratch"))
            return rc;
        b->scratch_cap = words;
    }
    Plan P;
    for (const std::vector<int> &g : gs) {
        std::vector<fides_op> gops;
        std::vector<u64 *> scr;
        size_t off = 0;
        for (int i : g) {
            gops.push_back(b->ops[i]);
            scr.push_back(b->scratch + off);
            off += op_scratch_words(c->N, c->K, c->alpha, b->ops[i].type, b->ops[i].a.n_limbs);
        }
        plan_stage(c, gops.data(), (int)gops.size(), gops[0].stage, scr.data(), P, tensor_split != 0, prime_order != 0);
        for (size_t k = 0; k < g.size(); ++k) b->ops[g[k]].out.scale = gops[k].out.scale;
    }
    if (P.image.size() > b->dmem_cap) {
        cudaFree(b->dmem);
        b->dmem = nullptr;
        b->dmem_cap = 0;
        if (int rc = fides_check_cuda(cudaMalloc((void **)&b->dmem, P.image.size()), "fides_batch: tables")) return rc;
        b->dmem_cap = P.image.size();
    }
    if (!P.image.empty())
        if (int rc = fides_check_cuda(cudaMemcpy(b->dmem, P.image.data(), P.image.size(), cudaMemcpyHostToDevice),
                                      "fides_batch: upload"))
            return rc;
    plan_patch(P, b->dmem);
    b->launches.swap(P.launches);
    b->table_bytes = P.image.size();
    b->scratch_bytes = b->scratch_cap * sizeof(u64);
    b->group_limbs = group_limbs;
    b->tensor_split = tensor_split;
    b->prime_order = prime_order;
    b->groups = (int)gs.size();
    return FIDES_OK;
}

}  // namespace

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
    fides_batch *b = new fides_batch();
    b->ctx = c;
    b->ops.assign(ops, ops + n_ops);
    b->nstage = nstage;
    b->dmem = nullptr;
    b->dmem_cap = 0;
    b->scratch = nullptr;
    b->scratch_cap = 0;
    b->exec = nullptr;
    if (int rc = batch_build(b, 0, 1, 0)) {
        fides_batch_destroy(b);
        return rc;
    }
    for (int i = 0; i < n_ops; ++i) ops[i].out.scale = b->ops[i].out.scale;
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

extern "C" int fides_batch_configure(fides_batch *b, int group_limbs, int tensor_split, int prime_order)
{
    if (!b) return fides_set_error(FIDES_ERR_ARG, "fides_batch_configure: NULL batch");
    if (group_limbs < 0 || (tensor_split != 0 && tensor_split != 1) || (prime_order != 0 && prime_order != 1))
        return fides_set_error(FIDES_ERR_ARG,
                               "fides_batch_configure: group_limbs >= 0, tensor_split and prime_order 0 or 1");
    return batch_build(b, group_limbs, tensor_split, prime_order);
}

extern "C" int fides_batch_tuning(const fides_batch *b, int *group_limbs, int *tensor_split, int *prime_order,
                                  int *groups)
{
    if (!b) return fides_set_error(FIDES_ERR_ARG, "fides_batch_tuning: NULL batch");
    if (group_limbs) *group_limbs = b->group_limbs;
    if (tensor_split) *tensor_split = b->tensor_split;
    if (prime_order) *prime_order = b->prime_order;
    if (groups) *groups = b->groups;
    return FIDES_OK;
}

extern "C" int fides_batch_autotune(fides_batch *b, void *stream, double *best_ms)
{
    if (!b) return fides_set_error(FIDES_ERR_ARG, "fides_batch_autotune: NULL batch");
    cudaStream_t st = (cudaStream_t)stream;
    int most = 0;   // limbs of the largest stage
    for (int s = 0; s < b->nstage; ++s) {
        int l = 0;
        for (const fides_op &o : b->ops)
            if (o.stage == s) l += o.a.n_limbs;
        most = std::max(most, l);
    }
    std::vector<int> sizes(1, 0);
    for (int g = 32; g < most; g *= 2) sizes.push_back(g);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = fides_check_cuda(cudaEventCreate(&e0), "fides_batch_autotune: event");
    if (!rc) rc = fides_check_cuda(cudaEventCreate(&e1), "fides_batch_autotune: event");
    const int was = fides_trace_set(0);
    float best = 0.f;
    int best_g = b->group_limbs, best_t = b->tensor_split, best_o = b->prime_order;
    for (size_t k = 0; !rc && k < sizes.size(); ++k) {
        for (int cand = 0; !rc && cand < 4; ++cand) {
            const int ts = 1 - (cand & 1), po = cand >> 1;
            rc = batch_build(b, sizes[k], ts, po, false);
            if (!rc) rc = plan_run(b->ctx, b->launches, st);   // warm-up
            if (!rc) rc = fides_check_cuda(cudaEventRecord(e0, st), "fides_batch_autotune: event");
            for (int r = 0; !rc && r < 2; ++r) rc = plan_run(b->ctx, b->launches, st);
            if (!rc) rc = fides_check_cuda(cudaEventRecord(e1, st), "fides_batch_autotune: event");
            if (!rc) rc = fides_check_cuda(cudaEventSynchronize(e1), "fides_batch_autotune: event");
            float ms = 0.f;
            if (!rc) rc = fides_check_cuda(cudaEventElapsedTime(&ms, e0, e1), "fides_batch_autotune: event");
            ms /= 2;
            if (!rc && (best == 0.f || ms < best)) {
                best = ms;
                best_g = sizes[k];
                best_t = ts;
                best_o = po;
            }
        }
    }
    fides_trace_set(was);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc) return rc;
    if (best_ms) *best_ms = best;
    return batch_build(b, best_g, best_t, best_o);
}
