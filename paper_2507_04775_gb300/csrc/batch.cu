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
#include "plan.cuh"

namespace {

enum LaunchKind { L_INTT, L_BCONV, L_NTT, L_INNER, L_NTT_SUBMUL, L_NTT_SWITCH_SUBMUL };

struct Launch {
    LaunchKind kind;
    LimbSet set;       // NTT kinds (device segments)
    BConvArgs bc;      // L_BCONV (device jobs)
    int ns, max_dst;
    IPArgs ip;         // L_INNER
    int max_beta;      // L_INNER
    int total;         // grid.y of L_INNER
};

// Host image of the device tables, with their offsets in the device buffer.
struct Tables {
    std::vector<unsigned char> host;
    size_t add(const void *p, size_t bytes)
    {
        size_t off = (host.size() + 15) & ~(size_t)15;
        host.resize(off + bytes);
        if (bytes) memcpy(host.data() + off, p, bytes);
        return off;
    }
};

}  // namespace

struct fides_batch {
    fides_ctx *ctx;
    std::vector<Launch> launches;
    unsigned char *dmem;      // device tables
    u64 *scratch;             // scratch of every operation
    size_t table_bytes, scratch_bytes;
    cudaGraphExec_t exec;     // captured run, or null
};

namespace {

// Pending table references: the device address of a table is known only after
// the buffer is allocated, so launches record offsets and are patched later.
struct Pending {
    int launch;
    int which;        // 0: set.dseg, 1: set.dpre, 2: bc.djob, 3: ip.dop, 4: ip.dpre
    size_t off;
};

void add_ntt(std::vector<Launch> &L, std::vector<Pending> &P, Tables &T, LaunchKind kind, const std::vector<Seg> &segs)
{
    if (segs.empty()) return;
    Launch l;
    memset(&l, 0, sizeof(l));
    l.kind = kind;
    l.set.nseg = (int)segs.size();
    std::vector<int> pre(segs.size());
    int tot = 0;
    for (size_t i = 0; i < segs.size(); ++i) { pre[i] = tot; tot += segs[i].count; }
    l.set.total = tot;
    L.push_back(l);
    const int id = (int)L.size() - 1;
    P.push_back(Pending{id, 0, T.add(segs.data(), sizeof(Seg) * segs.size())});
    P.push_back(Pending{id, 1, T.add(pre.data(), sizeof(int) * pre.size())});
}

void add_bconv(std::vector<Launch> &L, std::vector<Pending> &P, Tables &T, const std::vector<BConvJob> &jobs)
{
    std::vector<bool> done(jobs.size(), false);
    for (size_t j = 0; j < jobs.size(); ++j) {
        if (done[j]) continue;
        std::vector<BConvJob> g;
        int max_dst = 0;
        for (size_t k = j; k < jobs.size(); ++k) {
            if (done[k] || jobs[k].n_src != jobs[j].n_src) continue;
            done[k] = true;
            g.push_back(jobs[k]);
            max_dst = std::max(max_dst, bconv_targets(jobs[k]));
        }
        Launch l;
        memset(&l, 0, sizeof(l));
        l.kind = L_BCONV;
        l.bc.njob = (int)g.size();
        l.ns = jobs[j].n_src;
        l.max_dst = max_dst;
        L.push_back(l);
        P.push_back(Pending{(int)L.size() - 1, 2, T.add(g.data(), sizeof(BConvJob) * g.size())});
    }
}

void add_inner(std::vector<Launch> &L, std::vector<Pending> &P, Tables &T, const std::vector<IPOp> &ops,
               const std::vector<int> &rows)
{
    if (ops.empty()) return;
    Launch l;
    memset(&l, 0, sizeof(l));
    l.kind = L_INNER;
    std::vector<int> pre(ops.size());
    int tot = 0;
    for (size_t i = 0; i < ops.size(); ++i) { pre[i] = tot; tot += rows[i]; }
    l.total = tot;
    l.ip.nop = (int)ops.size();
    for (const IPOp &o : ops) l.max_beta = std::max(l.max_beta, o.beta);
    L.push_back(l);
    const int id = (int)L.size() - 1;
    P.push_back(Pending{id, 3, T.add(ops.data(), sizeof(IPOp) * ops.size())});
    P.push_back(Pending{id, 4, T.add(pre.data(), sizeof(int) * pre.size())});
}

int validate(const fides_ctx *c, const fides_op &o, int i)
{
    const int nl = o.a.n_limbs;
    if (!o.a.data || !o.out.data || o.stage < 0)
        return fides_set_error(FIDES_ERR_ARG, "fides_batch_create: op %d: NULL buffer or negative stage", i);
    if (nl < 1 || nl > c->L) return fides_set_error(FIDES_ERR_ARG, "fides_batch_create: op %d: bad level %d", i, nl);
    switch (o.type) {
    case FIDES_OP_HMULT:
        if (!o.b.data || o.b.n_limbs != nl || o.out.n_limbs != nl || !o.key)
            return fides_set_error(FIDES_ERR_ARG, "fides_batch_create: op %d: HMULT needs b, key and equal levels", i);
        return FIDES_OK;
    case FIDES_OP_ROTATE:
        if (o.out.n_limbs != nl || !o.key)
            return fides_set_error(FIDES_ERR_ARG, "fides_batch_create: op %d: ROTATE needs a key and equal levels", i);
        return FIDES_OK;
    case FIDES_OP_RESCALE:
        if (nl < 2 || o.out.n_limbs != nl - 1)
            return fides_set_error(FIDES_ERR_ARG, "fides_batch_create: op %d: RESCALE needs n_limbs >= 2 -> n_limbs-1", i);
        return FIDES_OK;
    default:
        return fides_set_error(FIDES_ERR_ARG, "fides_batch_create: op %d: unknown type %d", i, o.type);
    }
}

int run_launches(fides_batch *b, cudaStream_t st)
{
    const fides_ctx *c = b->ctx;
    for (const Launch &l : b->launches) {
        int rc = FIDES_OK;
        switch (l.kind) {
        case L_INTT: rc = ntt_inverse(c, l.set, ProSrc{}, EpiCanon{}, st); break;
        case L_NTT: rc = ntt_forward(c, l.set, ProSrc{}, EpiCanon{}, st); break;
        case L_NTT_SUBMUL: rc = ntt_forward(c, l.set, ProSrc{}, EpiSubMul{}, st); break;
        case L_NTT_SWITCH_SUBMUL: rc = ntt_forward(c, l.set, ProSwitchMod{}, EpiSubMul{}, st); break;
        case L_BCONV: rc = launch_bconv_group(c, l.bc, l.ns, l.max_dst, st); break;
        case L_INNER: rc = launch_inner(c, l.ip, l.total, l.max_beta, st); break;
        }
        if (rc) return rc;
    }
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
        if (int rc = validate(c, ops[i], i)) return rc;
        nstage = std::max(nstage, ops[i].stage + 1);
    }
    const size_t N = c->N;

    // scratch of every operation
    std::vector<size_t> soff(n_ops);
    size_t words = 0;
    for (int i = 0; i < n_ops; ++i) {
        soff[i] = words;
        const int nl = ops[i].a.n_limbs;
        words += ops[i].type == FIDES_OP_RESCALE ? 2 * N : (size_t)nl * N + ks_scratch_words(c, nl);
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
    u64 *scratch = b->scratch;
    // launches, with table addresses patched once the table buffer exists
    std::vector<Pending> pend;
    Tables T;
    for (int s = 0; s < nstage; ++s) {
        std::vector<Seg> intt, ntt, pinv, fin, rsfin;
        std::vector<BConvJob> up, down;
        std::vector<IPOp> ip;
        std::vector<int> ip_rows;
        for (int i = 0; i < n_ops; ++i) {
            fides_op &o = ops[i];
            if (o.stage != s) continue;
            const int nl = o.a.n_limbs;
            const size_t S = (size_t)nl * N;
            u64 *base = scratch + soff[i];
            if (o.type == FIDES_OP_RESCALE) {
                rs_intt_segs(c, o.a.data, nl, base, intt);
                rs_final_segs(c, o.a.data, nl, base, o.out.data, rsfin);
                o.out.scale = o.a.scale / (double)c->primes[nl - 1];
                continue;
            }
            const bool hm = o.type == FIDES_OP_HMULT;
            u64 *dsrc = base;
            KsBuffers B;
            memset(&B, 0, sizeof(B));
            B.d = dsrc; B.nl = nl; B.evk = o.key;
            B.out0 = o.out.data; B.out1 = o.out.data + S;
            B.mode0 = 1; B.mode1 = hm ? 1 : 0;
            B.prep = hm ? 1 : 2;
            B.pa = o.a.data;
            B.pb = hm ? o.b.data : nullptr;
            B.pout = o.out.data;
            B.g = hm ? 0 : fides_galois_elt(c, o.steps);
            ks_carve(c, B, dsrc + S);
            ks_intt_segs(c, B, intt);
            ks_modup_jobs(c, B, up);
            ks_modup_ntt_segs(c, B, ntt);
            ip.push_back(ks_ip_op(c, B));
            ip_rows.push_back(nl + c->K);
            ks_pinv_segs(c, B, pinv);
            ks_moddown_jobs(c, B, down);
            ks_final_segs(c, B, fin);
            o.out.scale = hm ? o.a.scale * o.b.scale : o.a.scale;
        }
        std::vector<Launch> &L = b->launches;
        add_ntt(L, pend, T, L_INTT, intt);
        add_bconv(L, pend, T, up);
        add_ntt(L, pend, T, L_NTT, ntt);
        add_inner(L, pend, T, ip, ip_rows);
        add_ntt(L, pend, T, L_INTT, pinv);
        add_bconv(L, pend, T, down);
        add_ntt(L, pend, T, L_NTT_SUBMUL, fin);
        add_ntt(L, pend, T, L_NTT_SWITCH_SUBMUL, rsfin);
    }
    b->table_bytes = T.host.size();
    if (b->table_bytes) {
        int rc = fides_check_cuda(cudaMalloc((void **)&b->dmem, b->table_bytes), "fides_batch_create: tables");
        if (!rc) rc = fides_check_cuda(cudaMemcpy(b->dmem, T.host.data(), b->table_bytes, cudaMemcpyHostToDevice),
                                       "fides_batch_create: upload");
        if (rc) { fides_batch_destroy(b); return rc; }
    }
    for (const Pending &p : pend) {
        Launch &l = b->launches[p.launch];
        void *a = b->dmem + p.off;
        switch (p.which) {
        case 0: l.set.dseg = (const Seg *)a; break;
        case 1: l.set.dpre = (const int *)a; break;
        case 2: l.bc.djob = (const BConvJob *)a; break;
        case 3: l.ip.dop = (const IPOp *)a; break;
        case 4: l.ip.dpre = (const int *)a; break;
        }
    }
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
    return run_launches(b, st);
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
        int rc2 = run_launches(b, st);
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
    int n = 0;
    for (const Launch &l : b->launches) {
        n += (l.kind == L_INTT || l.kind == L_NTT || l.kind == L_NTT_SUBMUL || l.kind == L_NTT_SWITCH_SUBMUL)
                 ? (b->ctx->logN == 16 ? 2 : 1)
                 : 1;
    }
    if (launches) *launches = n;
    if (scratch_bytes) *scratch_bytes = b->scratch_bytes;
    if (table_bytes) *table_bytes = b->table_bytes;
    return FIDES_OK;
}
