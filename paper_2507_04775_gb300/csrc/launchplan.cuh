// Launch plans: the fixed sequence of launches that runs a group of HMult,
// HRotate and Rescale operations with one launch per step of the key switch
// (and of the rescale) for the whole group, together with the host image of
// the device tables those launches read (NTT segments, base-conversion jobs,
// inner-product descriptors).  Used by the batched path (a fixed batch replayed
// many times) and by the request server (a new group per launch).
#pragma once

#include <algorithm>
#include <cstring>
#include <vector>

#include "plan.cuh"

namespace {

enum LaunchKind { L_INTT, L_BCONV, L_NTT, L_INNER, L_NTT_SUBMUL, L_NTT_SWITCH_SUBMUL, L_TENSOR };

struct Launch {
    LaunchKind kind;
    LimbSet set;       // NTT kinds (device segments)
    BConvArgs bc;      // L_BCONV (device jobs)
    int ns, max_dst;
    IPArgs ip;         // L_INNER
    int max_beta;      // L_INNER
    int ip_pairs;      // L_INNER: every op can take the paired path
    int total;         // grid.y of L_INNER and L_TENSOR
    TensorArgs tp;     // L_TENSOR (device ops)
};

// Table references: a launch records the offset of each of its tables in the
// table image; the device addresses are patched in once the image has a home.
struct Pending {
    int launch;
    int which;        // 0: set.dseg, 1: set.dpre, 2: bc.djob, 3: ip.dop, 4: ip.drow, 5: tp.dop, 6: tp.dpre
    size_t off;
};

struct Plan {
    std::vector<Launch> launches;
    std::vector<Pending> pend;
    std::vector<unsigned char> image;   // host image of the device tables

    size_t add(const void *p, size_t bytes)
    {
        size_t off = (image.size() + 15) & ~(size_t)15;
        image.resize(off + bytes);
        if (bytes) memcpy(image.data() + off, p, bytes);
        return off;
    }
};

// One launch for the segments.  prime_major: every limb becomes a segment of
// its own and the limbs are ordered by prime, so that the CTAs in flight work
// on few primes and their row twiddle tables stay in L2 (a table per prime
// and direction, 16 N bytes); the kernels then index the table directly.
void plan_ntt(Plan &P, LaunchKind kind, const std::vector<Seg> &segs, size_t N, bool prime_major = false)
{
    if (segs.empty()) return;
    std::vector<Seg> v;
    if (prime_major) {
        for (const Seg &g : segs)
            for (int k = 0; k < g.count; ++k) v.push_back(limb_of(g, k, N));
        std::stable_sort(v.begin(), v.end(), [](const Seg &a, const Seg &b) { return a.prime0 < b.prime0; });
    } else {
        v = segs;
    }
    Launch l;
    memset(&l, 0, sizeof(l));
    l.kind = kind;
    l.set.nseg = (int)v.size();
    std::vector<int> pre(v.size());
    int tot = 0;
    for (size_t i = 0; i < v.size(); ++i) { pre[i] = tot; tot += v[i].count; l.set.modes |= v[i].mode; }
    l.set.total = tot;
    P.launches.push_back(l);
    const int id = (int)P.launches.size() - 1;
    P.pend.push_back(Pending{id, 0, P.add(v.data(), sizeof(Seg) * v.size())});
    P.pend.push_back(Pending{id, 1, P.add(pre.data(), sizeof(int) * pre.size())});
}

// One launch for the tensor-core jobs, one per distinct source count of the
// others (the integer conversion kernel is templated on it).
// Tensor-core jobs go to two launches by target count: with at most 16
// targets an accumulator has at most 128 tensor-memory columns, and a launch
// of such jobs keeps four of them per CTA instead of two (bconv_tc.cuh).
inline int plan_bconv_key(const BConvJob &j)
{
    const int key = bconv_group_key(j);
    return key < 0 && bconv_targets(j) > 16 ? -2 : key;
}

void plan_bconv(Plan &P, const std::vector<BConvJob> &jobs)
{
    std::vector<bool> done(jobs.size(), false);
    for (size_t j = 0; j < jobs.size(); ++j) {
        if (done[j]) continue;
        const int key = plan_bconv_key(jobs[j]);
        std::vector<BConvJob> g;
        int max_dst = 0, ns = 0;
        for (size_t k = j; k < jobs.size(); ++k) {
            if (done[k] || plan_bconv_key(jobs[k]) != key) continue;
            done[k] = true;
            g.push_back(jobs[k]);
            max_dst = std::max(max_dst, bconv_targets(jobs[k]));
            ns = std::max(ns, jobs[k].n_src);
        }
        Launch l;
        memset(&l, 0, sizeof(l));
        l.kind = L_BCONV;
        l.bc.njob = (int)g.size();
        l.bc.tc = key < 0;
        if (l.bc.tc)
            for (const BConvJob &x : g) l.bc.tc_smem = std::max(l.bc.tc_smem, bconv_tc_smem(x));
        l.ns = ns;
        l.max_dst = max_dst;
        P.launches.push_back(l);
        P.pend.push_back(Pending{(int)P.launches.size() - 1, 2, P.add(g.data(), sizeof(BConvJob) * g.size())});
    }
}

void plan_inner(Plan &P, const std::vector<IPOp> &ops, const std::vector<int> &rows)
{
    if (ops.empty()) return;
    Launch l;
    memset(&l, 0, sizeof(l));
    l.kind = L_INNER;
    // rows (op, limb) ordered by key, then by the key limb the row reads,
    // then by op: the ops sharing a key read each of its limbs back to back
    struct Row { const u64 *evk; int pz, op, z; };
    std::vector<Row> order;
    for (size_t i = 0; i < ops.size(); ++i)
        for (int z = 0; z < rows[i]; ++z)
            order.push_back(Row{ops[i].evk, z < ops[i].nl ? z : 1024 + (z - ops[i].nl), (int)i, z});
    std::stable_sort(order.begin(), order.end(), [](const Row &a, const Row &b) {
        if (a.evk != b.evk) return a.evk < b.evk;
        return a.pz < b.pz;
    });
    std::vector<int> rowtab(order.size());
    for (size_t r = 0; r < order.size(); ++r) rowtab[r] = (order[r].op << 7) | order[r].z;
    l.total = (int)order.size();
    l.ip.nop = (int)ops.size();
    l.ip_pairs = 1;
    for (const IPOp &o : ops) {
        l.max_beta = std::max(l.max_beta, o.beta);
        if (!ip_pairs_ok(o)) l.ip_pairs = 0;
    }
    P.launches.push_back(l);
    const int id = (int)P.launches.size() - 1;
    P.pend.push_back(Pending{id, 3, P.add(ops.data(), sizeof(IPOp) * ops.size())});
    P.pend.push_back(Pending{id, 4, P.add(rowtab.data(), sizeof(int) * rowtab.size())});
}

void plan_tensor(Plan &P, const std::vector<TensorOp> &ops)
{
    if (ops.empty()) return;
    Launch l;
    memset(&l, 0, sizeof(l));
    l.kind = L_TENSOR;
    std::vector<int> pre(ops.size());
    int tot = 0;
    for (size_t i = 0; i < ops.size(); ++i) { pre[i] = tot; tot += ops[i].nl; }
    l.total = tot;
    l.tp.nop = (int)ops.size();
    P.launches.push_back(l);
    const int id = (int)P.launches.size() - 1;
    P.pend.push_back(Pending{id, 5, P.add(ops.data(), sizeof(TensorOp) * ops.size())});
    P.pend.push_back(Pending{id, 6, P.add(pre.data(), sizeof(int) * pre.size())});
}

// Checks one operation's descriptor (levels, buffers, key); `fn` names the
// caller in the error message.
int plan_validate(const fides_ctx *c, const fides_op &o, int i, const char *fn)
{
    const int nl = o.a.n_limbs;
    if (!o.a.data || !o.out.data || o.stage < 0)
        return fides_set_error(FIDES_ERR_ARG, "%s: op %d: NULL buffer or negative stage", fn, i);
    if (nl < 1 || nl > c->L) return fides_set_error(FIDES_ERR_ARG, "%s: op %d: bad level %d", fn, i, nl);
    switch (o.type) {
    case FIDES_OP_HMULT:
        if (!o.b.data || o.b.n_limbs != nl || o.out.n_limbs != nl || !o.key)
            return fides_set_error(FIDES_ERR_ARG, "%s: op %d: HMULT needs b, key and equal levels", fn, i);
        if (fides_check_key(c, o.key, FIDES_GALOIS_RELIN, fn))
            return fides_set_error(FIDES_ERR_KEY, "%s: op %d: the key is not this context's relinearisation key", fn, i);
        return FIDES_OK;
    case FIDES_OP_ROTATE:
        if (o.out.n_limbs != nl || !o.key)
            return fides_set_error(FIDES_ERR_ARG, "%s: op %d: ROTATE needs a key and equal levels", fn, i);
        if (fides_check_key(c, o.key, fides_galois_elt(c, o.steps), fn))
            return fides_set_error(FIDES_ERR_KEY, "%s: op %d: the key is not this context's key of Galois element %llu",
                                   fn, i, (unsigned long long)fides_galois_elt(c, o.steps));
        return FIDES_OK;
    case FIDES_OP_RESCALE:
        if (nl < 2 || o.out.n_limbs != nl - 1)
            return fides_set_error(FIDES_ERR_ARG, "%s: op %d: RESCALE needs n_limbs >= 2 -> n_limbs-1", fn, i);
        return FIDES_OK;
    default:
        return fides_set_error(FIDES_ERR_ARG, "%s: op %d: unknown type %d", fn, i, o.type);
    }
}

// Scratch words one operation needs: the key-switch input and one key switch
// for HMult / HRotate, the dropped limb of both polynomials for Rescale.
inline size_t op_scratch_words(int N, int K, int alpha, int type, int nl)
{
    if (type == FIDES_OP_RESCALE) return 2 * (size_t)N;
    return (size_t)nl * N + ks_scratch_words_of(N, K, alpha, nl);
}

// Appends the launches of one stage: the operations ops[i] with ops[i].stage
// == stage, each with its scratch at scratch[i].  Sets each op's out.scale.
// tensor_split: HMult's tensor product runs as its own 16-byte pass (where
// the buffers allow) instead of fused into the first INTT pass; a fusion
// boundary the batch autotuner chooses.
void plan_stage(const fides_ctx *c, fides_op *ops, int n_ops, int stage, u64 *const *scratch, Plan &P,
                bool tensor_split = true, bool prime_major = false)
{
    const size_t N = c->N;
    std::vector<Seg> intt, ntt, pinv, fin, rsfin;
    std::vector<BConvJob> up, down;
    std::vector<IPOp> ip;
    std::vector<int> ip_rows;
    std::vector<TensorOp> tens;
    for (int i = 0; i < n_ops; ++i) {
        fides_op &o = ops[i];
        if (o.stage != stage) continue;
        const int nl = o.a.n_limbs;
        const size_t S = (size_t)nl * N;
        u64 *base = scratch[i];
        if (o.type == FIDES_OP_RESCALE) {
            rs_intt_segs(c, o.a.data, nl, base, intt);
            rs_final_segs(c, o.a.data, nl, base, o.out.data, rsfin, c->round_nearest != 0);
            o.out.scale = o.a.scale / (double)c->primes[nl - 1];
            continue;
        }
        const bool hm = o.type == FIDES_OP_HMULT;
        u64 *dsrc = base;
        KsBuffers B;
        memset(&B, 0, sizeof(B));
        B.d = dsrc; B.nl = nl; B.evk = o.key->data;
        B.out0 = o.out.data; B.out1 = o.out.data + S;
        B.mode0 = 1; B.mode1 = hm ? 1 : 0;
        if (hm && tensor_split && tensor_pass_ok(o.a.data, o.b.data, o.out.data, dsrc)) {
            tens.push_back(TensorOp{o.a.data, o.b.data, o.out.data, dsrc, nl});   // d2 in dsrc, plain INTT
        } else {
            B.prep = hm ? 1 : 2;
            B.pa = o.a.data;
            B.pb = hm ? o.b.data : nullptr;
            B.pout = o.out.data;
        }
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
    plan_tensor(P, tens);
    plan_ntt(P, L_INTT, intt, N, prime_major);
    plan_bconv(P, up);
    plan_ntt(P, L_NTT, ntt, N, prime_major);
    plan_inner(P, ip, ip_rows);
    plan_ntt(P, L_INTT, pinv, N, prime_major);
    plan_bconv(P, down);
    plan_ntt(P, L_NTT_SUBMUL, fin, N, prime_major);
    plan_ntt(P, L_NTT_SWITCH_SUBMUL, rsfin, N, prime_major);
}

// Points every launch at the device copy of the table image.
void plan_patch(Plan &P, unsigned char *dmem)
{
    for (const Pending &p : P.pend) {
        Launch &l = P.launches[p.launch];
        void *a = dmem + p.off;
        switch (p.which) {
        case 0: l.set.dseg = (const Seg *)a; break;
        case 1: l.set.dpre = (const int *)a; break;
        case 2: l.bc.djob = (const BConvJob *)a; break;
        case 3: l.ip.dop = (const IPOp *)a; break;
        case 4: l.ip.drow = (const int *)a; break;
        case 5: l.tp.dop = (const TensorOp *)a; break;
        case 6: l.tp.dpre = (const int *)a; break;
        }
    }
}

int plan_run(const fides_ctx *c, const std::vector<Launch> &launches, cudaStream_t st)
{
    for (const Launch &l : launches) {
        int rc = FIDES_OK;
        switch (l.kind) {
        case L_INTT: rc = ntt_inverse(c, l.set, ProSrc{}, EpiCanon{}, st); break;
        case L_NTT: rc = ntt_forward(c, l.set, ProSrc{}, EpiCanon{}, st); break;
        case L_NTT_SUBMUL: rc = ntt_forward(c, l.set, ProSrc{}, EpiSubMul{}, st); break;
        case L_NTT_SWITCH_SUBMUL: rc = ntt_forward(c, l.set, ProSwitchMod{}, EpiSubMul{}, st); break;
        case L_BCONV: rc = launch_bconv_group(c, l.bc, l.ns, l.max_dst, st); break;
        case L_INNER: rc = launch_inner(c, l.ip, l.total, l.max_beta, st, l.ip_pairs); break;
        case L_TENSOR: rc = launch_tensor_args(c, l.tp, l.total, st); break;
        }
        if (rc) return rc;
    }
    return FIDES_OK;
}

// Kernels one run of the plan launches (an NTT at logN=16 is two passes).
int plan_kernel_count(const fides_ctx *c, const std::vector<Launch> &launches)
{
    int n = 0;
    for (const Launch &l : launches) {
        const bool ntt = l.kind == L_INTT || l.kind == L_NTT || l.kind == L_NTT_SUBMUL ||
                         l.kind == L_NTT_SWITCH_SUBMUL;
        n += ntt ? (c->logN == 12 ? 1 : 2) : 1;
    }
    return n;
}

}  // namespace
