// Homomorphic programs: a list of instructions over ciphertext registers,
// executed on the device through the library's operations.  Bootstrapping
// (Sec. III-F7) is such a program -- ModRaise, three linear transforms for
// CoeffToSlot, the conjugation split, the EvalMod polynomial and double-angle
// steps, three linear transforms for SlotToCoeff -- whose constants (the
// transforms' plaintext diagonals, scalar constants) are the precomputation
// that the paper takes from OpenFHE (Sec. III-B).
//
// Registers are virtual and written once; at creation the program is checked
// (operands defined before use, levels consistent, keys present) and the
// virtual registers are mapped onto as few device buffers as their lifetimes
// allow, never giving an instruction's result the buffer of one of its
// operands.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "fides_internal.cuh"
#include "ops_ws.h"

struct fides_program {
    fides_ctx *ctx;
    std::vector<fides_instr> instr;
    int n_regs, in_reg, out_reg, in_limbs;
    double out_scale;
    struct Lt {
        std::vector<int> idx;
        std::vector<const uint64_t *> pts;
        int n1;
        double pt_scale;
    };
    std::vector<Lt> lt;
    std::vector<std::vector<uint64_t>> consts;
    std::vector<double> const_scale;
    u64 *dconst = nullptr;                      // device copy of the constants, [n_const][L]
    std::vector<int> lin_start, lin_reg, lin_const;   // CMAC term lists
    const uint64_t *relin, *conj;               // key buffers (null: none)
    std::vector<const fides_key *> rot_keys;    // rotation-key handles, found by Galois element
    // analysis
    std::vector<int> level;     // limbs of each virtual register
    std::vector<int> phys;      // buffer of each virtual register (-1: the input)
    int n_phys;
    size_t lt_words;
    // fuse[i]: instruction i is an HMULT whose product only the RESCALE at
    // i + 1 reads; the pair runs as one fides_hmult_rescale
    std::vector<char> fuse;
};

namespace {

bool reads_b(int op) { return op == FIDES_I_HADD || op == FIDES_I_HSUB || op == FIDES_I_HMULT; }

// The key of the rotation by `steps` among the program's handles: the one
// registered with Galois element 5^steps mod 2N, or null.
const uint64_t *rot_key(const fides_program *p, int64_t steps)
{
    const u64 want = fides_galois_elt(p->ctx, steps);
    for (const fides_key *k : p->rot_keys)
        if (k && k->g == want) return k->data;
    return nullptr;
}

// registers an instruction reads
std::vector<int> operands(const fides_program *p, const fides_instr &I)
{
    if (I.op == FIDES_I_CMAC)
        return std::vector<int>(p->lin_reg.begin() + p->lin_start[I.arg], p->lin_reg.begin() + p->lin_start[I.arg + 1]);
    std::vector<int> r(1, I.a);
    if (reads_b(I.op) && I.b != I.a) r.push_back(I.b);
    return r;
}

// Registers are written once, so an instruction may move earlier as long as
// its operands are defined before it.  Every RESCALE that is the only reader
// of an HMULT's product moves to just after that HMULT, where the executor
// runs the pair as one fused call.  Out-of-range registers are left for
// analyse() to report.
void hoist_rescales(fides_program *p)
{
    const int n = (int)p->instr.size();
    auto readers = [&](std::vector<int> &count, std::vector<int> &at) {
        count.assign(p->n_regs, 0);
        at.assign(p->n_regs, -1);
        for (int i = 0; i < n; ++i) {
            const fides_instr &I = p->instr[i];
            if (I.op == FIDES_I_CMAC && (I.arg < 0 || I.arg + 1 >= (int)p->lin_start.size())) continue;
            for (int r : operands(p, I))
                if (r >= 0 && r < p->n_regs) { ++count[r]; at[r] = i; }
        }
    };
    std::vector<int> count, at;
    readers(count, at);
    for (int i = 0; i < n; ++i) {
        const fides_instr I = p->instr[i];
        if (I.op != FIDES_I_HMULT || I.dst < 0 || I.dst >= p->n_regs || I.dst == p->out_reg) continue;
        if (count[I.dst] != 1) continue;
        const int j = at[I.dst];
        if (j <= i + 1 || p->instr[j].op != FIDES_I_RESCALE || p->instr[j].a != I.dst) continue;
        std::rotate(p->instr.begin() + i + 1, p->instr.begin() + j, p->instr.begin() + j + 1);
        readers(count, at);
    }
}

int analyse(fides_program *p)
{
    const fides_ctx *c = p->ctx;
    const int n = (int)p->instr.size();
    p->level.assign(p->n_regs, 0);
    std::vector<int> def(p->n_regs, -1), last(p->n_regs, -1);
    p->level[p->in_reg] = p->in_limbs;
    def[p->in_reg] = -2;
    for (int i = 0; i < n; ++i) {
        const fides_instr &I = p->instr[i];
        auto bad = [&](const char *why) {
            return fides_set_error(FIDES_ERR_ARG, "fides_program_create: instruction %d (op %d): %s", i, I.op, why);
        };
        if (I.op == FIDES_I_CMAC) {
            if (I.arg < 0 || I.arg + 1 >= (int)p->lin_start.size()) return bad("no such term list");
            const int t0 = p->lin_start[I.arg], t1 = p->lin_start[I.arg + 1];
            if (t1 - t0 < 1 || t1 - t0 > FIDES_MAC_TERMS) return bad("a term list holds 1..32 terms");
            if (I.dst < 0 || I.dst >= p->n_regs || def[I.dst] != -1) return bad("bad or reused destination");
            if (I.b < 1 || I.b > c->L) return bad("bad target level");
            for (int t = t0; t < t1; ++t) {
                const int r = p->lin_reg[t], k = p->lin_const[t];
                if (r < 0 || r >= p->n_regs || def[r] == -1) return bad("term register not defined");
                if (p->level[r] < I.b) return bad("term below the target level");
                if (k < 0 || k >= (int)p->consts.size()) return bad("no such constant");
                last[r] = i;
            }
            p->level[I.dst] = I.b;
            def[I.dst] = i;
            continue;
        }
        if (I.dst < 0 || I.dst >= p->n_regs || I.a < 0 || I.a >= p->n_regs) return bad("register out of range");
        if (def[I.a] == -1) return bad("operand a is not defined yet");
        if (reads_b(I.op) && (I.b < 0 || I.b >= p->n_regs || def[I.b] == -1)) return bad("operand b is not defined");
        if (def[I.dst] != -1) return bad("register written twice");
        const int la = p->level[I.a];
        int ld = la;
        switch (I.op) {
        case FIDES_I_MODRAISE:
            if (la != 1 || I.arg < 1 || I.arg > c->L) return bad("ModRaise needs one limb in and 1..L out");
            ld = I.arg;
            break;
        case FIDES_I_LT:
            if (I.arg < 0 || I.arg >= (int)p->lt.size()) return bad("no such linear transform");
            break;
        case FIDES_I_RESCALE:
            if (la < 2) return bad("rescale needs two limbs");
            ld = la - 1;
            break;
        case FIDES_I_DROP:
            if (I.arg < 1 || I.arg > la) return bad("drop to more limbs than the operand has");
            ld = I.arg;
            break;
        case FIDES_I_HADD:
        case FIDES_I_HSUB:
        case FIDES_I_HMULT:
            if (p->level[I.b] != la) return bad("operands at different levels");
            if (I.op == FIDES_I_HMULT && !p->relin) return bad("no relinearisation key");
            break;
        case FIDES_I_CONJ:
            if (!p->conj) return bad("no conjugation key");
            break;
        case FIDES_I_ROT:
            if (!rot_key(p, I.arg)) return bad("no rotation key for the step");
            break;
        case FIDES_I_MULI:
            if (I.arg != 1 && I.arg != -1) return bad("MULI takes +1 or -1");
            break;
        case FIDES_I_CMULT:
        case FIDES_I_CADD:
            if (I.arg < 0 || I.arg >= (int)p->consts.size()) return bad("no such constant");
            break;
        case FIDES_I_COPY:
            break;
        default:
            return bad("unknown instruction");
        }
        p->level[I.dst] = ld;
        def[I.dst] = i;
        last[I.a] = i;
        if (reads_b(I.op)) last[I.b] = i;
    }
    if (def[p->out_reg] == -1) return fides_set_error(FIDES_ERR_ARG, "fides_program_create: output never written");
    last[p->out_reg] = n;
    // buffers: the destination is taken before the operands are released, so
    // no instruction writes a buffer it reads
    p->phys.assign(p->n_regs, -1);
    std::vector<int> free_list;
    int count = 0;
    for (int i = 0; i < n; ++i) {
        const fides_instr &I = p->instr[i];
        int b;
        if (!free_list.empty()) { b = free_list.back(); free_list.pop_back(); }
        else b = count++;
        p->phys[I.dst] = b;
        std::vector<int> ops = operands(p, I);
        std::sort(ops.begin(), ops.end());
        ops.erase(std::unique(ops.begin(), ops.end()), ops.end());
        for (int r : ops) {
            if (r == p->in_reg) continue;
            if (last[r] == i) free_list.push_back(p->phys[r]);
        }
        if (last[I.dst] < 0) free_list.push_back(b);   // never read
    }
    p->n_phys = count;
    p->fuse.assign(n, 0);
    for (int i = 0; i + 1 < n; ++i) {
        const fides_instr &I = p->instr[i], &J = p->instr[i + 1];
        if (I.op != FIDES_I_HMULT || J.op != FIDES_I_RESCALE || J.a != I.dst || I.dst == p->out_reg) continue;
        if (last[I.dst] != i + 1) continue;
        const int pd = p->phys[J.dst];
        auto buf = [&](int r) { return r == p->in_reg ? -1 : p->phys[r]; };
        if (pd == buf(I.a) || pd == buf(I.b)) continue;
        p->fuse[i] = 1;
    }
    // linear-transform scratch at the top level
    p->lt_words = 0;
    for (const fides_program::Lt &t : p->lt) {
        size_t w = 0;
        if (int rc = fides_linear_transform_work_words(p->ctx, c->L, (int)t.idx.size(), t.idx.data(), t.n1, &w))
            return rc;
        p->lt_words = std::max(p->lt_words, w);
    }
    return FIDES_OK;
}

}  // namespace

extern "C" int fides_program_create(fides_ctx *c, const fides_program_desc *d, fides_program **out)
{
    if (!out) return fides_set_error(FIDES_ERR_ARG, "fides_program_create: out is NULL");
    *out = nullptr;
    if (!c || !d || d->n_instr < 1 || !d->instr || d->n_regs < 1)
        return fides_set_error(FIDES_ERR_ARG, "fides_program_create: bad arguments");
    if (d->in_reg < 0 || d->in_reg >= d->n_regs || d->out_reg < 0 || d->out_reg >= d->n_regs ||
        d->in_limbs < 1 || d->in_limbs > c->L)
        return fides_set_error(FIDES_ERR_ARG, "fides_program_create: bad input/output register or limbs");
    if ((d->n_lt > 0 && !d->lt) || (d->n_const > 0 && (!d->consts || !d->const_scale)) ||
        d->n_rot_keys < 0 || (d->n_rot_keys > 0 && !d->rot_keys))
        return fides_set_error(FIDES_ERR_ARG, "fides_program_create: NULL table");
    // keys: the relinearisation key of Galois element 0, the conjugation key
    // of 2N - 1, rotation keys of this context (each found by its element)
    if (d->relin_key)
        if (int rc = fides_check_key(c, d->relin_key, FIDES_GALOIS_RELIN, "fides_program_create: relin_key")) return rc;
    if (d->conj_key)
        if (int rc = fides_check_key(c, d->conj_key, 2 * (u64)c->N - 1, "fides_program_create: conj_key")) return rc;
    for (int k = 0; k < d->n_rot_keys; ++k)
        if (int rc = fides_check_key(c, d->rot_keys[k], FIDES_GALOIS_ANY, "fides_program_create: rot_keys")) return rc;
    fides_program *p = new fides_program();
    p->ctx = c;
    p->instr.assign(d->instr, d->instr + d->n_instr);
    p->n_regs = d->n_regs;
    p->in_reg = d->in_reg;
    p->out_reg = d->out_reg;
    p->in_limbs = d->in_limbs;
    p->out_scale = d->out_scale;
    for (int k = 0; k < d->n_lt; ++k) {
        const fides_lt &t = d->lt[k];
        if (t.n_diag < 1 || !t.diag_idx || !t.dev_pts) {
            delete p;
            return fides_set_error(FIDES_ERR_ARG, "fides_program_create: linear transform %d is empty", k);
        }
        fides_program::Lt l;
        l.idx.assign(t.diag_idx, t.diag_idx + t.n_diag);
        l.pts.assign(t.dev_pts, t.dev_pts + t.n_diag);
        l.n1 = t.n1;
        l.pt_scale = t.pt_scale;
        p->lt.push_back(std::move(l));
    }
    for (int k = 0; k < d->n_const; ++k) {
        p->consts.emplace_back(d->consts[k], d->consts[k] + c->L);
        p->const_scale.push_back(d->const_scale[k]);
    }
    if (d->n_lin > 0) {
        if (!d->lin_start || !d->lin_reg || !d->lin_const) {
            delete p;
            return fides_set_error(FIDES_ERR_ARG, "fides_program_create: NULL term lists");
        }
        p->lin_start.assign(d->lin_start, d->lin_start + d->n_lin + 1);
        const int nt = p->lin_start.back();
        if (p->lin_start[0] != 0 || nt < 0) {
            delete p;
            return fides_set_error(FIDES_ERR_ARG, "fides_program_create: bad term list offsets");
        }
        for (int k = 0; k < d->n_lin; ++k)
            if (p->lin_start[k + 1] < p->lin_start[k]) {
                delete p;
                return fides_set_error(FIDES_ERR_ARG, "fides_program_create: bad term list offsets");
            }
        p->lin_reg.assign(d->lin_reg, d->lin_reg + nt);
        p->lin_const.assign(d->lin_const, d->lin_const + nt);
    } else {
        p->lin_start.assign(1, 0);
    }
    p->relin = d->relin_key ? d->relin_key->data : nullptr;
    p->conj = d->conj_key ? d->conj_key->data : nullptr;
    p->rot_keys.assign(d->rot_keys, d->rot_keys + d->n_rot_keys);
    hoist_rescales(p);
    if (int rc = analyse(p)) {
        delete p;
        return rc;
    }
    if (!p->consts.empty()) {
        std::vector<uint64_t> flat;
        for (const auto &k : p->consts) flat.insert(flat.end(), k.begin(), k.end());
        int rc = fides_check_cuda(cudaMalloc((void **)&p->dconst, flat.size() * sizeof(u64)), "fides_program_create");
        if (!rc) rc = fides_check_cuda(cudaMemcpy(p->dconst, flat.data(), flat.size() * sizeof(u64), cudaMemcpyHostToDevice),
                                       "fides_program_create");
        if (rc) {
            fides_program_destroy(p);
            return rc;
        }
    }
    *out = p;
    return FIDES_OK;
}

extern "C" void fides_program_destroy(fides_program *p)
{
    if (!p) return;
    cudaFree(p->dconst);
    delete p;
}

extern "C" int fides_program_info(const fides_program *p, size_t *work_words, int *buffers, int *out_limbs)
{
    if (!p) return fides_set_error(FIDES_ERR_ARG, "fides_program_info: NULL program");
    const size_t ct = 2 * (size_t)p->ctx->L * p->ctx->N;
    // registers, linear-transform buffers, and the program's own scratch pool
    // for its key-switching operations (so that programs on one context can
    // run concurrently on several streams)
    if (work_words) *work_words = (size_t)p->n_phys * ct + p->lt_words + p->ctx->scratch_words;
    if (buffers) *buffers = p->n_phys;
    if (out_limbs) *out_limbs = p->level[p->out_reg];
    return FIDES_OK;
}

extern "C" int fides_program_run(fides_program *p, const fides_ct *in, fides_ct *out, uint64_t *work,
                                 size_t work_words, void *stream)
{
    const char *fn = "fides_program_run";
    if (!p || !in || !in->data || !out || !out->data) return fides_set_error(FIDES_ERR_ARG, "%s: NULL argument", fn);
    fides_ctx *c = p->ctx;
    const size_t N = c->N, ct_words = 2 * (size_t)c->L * N;
    size_t need = 0;
    fides_program_info(p, &need, nullptr, nullptr);
    if (!work || work_words < need) return fides_set_error(FIDES_ERR_ARG, "%s: work buffer needs %zu words", fn, need);
    if (in->n_limbs != p->in_limbs) return fides_set_error(FIDES_ERR_ARG, "%s: input must have %d limbs", fn, p->in_limbs);
    if (out->n_limbs != p->level[p->out_reg])
        return fides_set_error(FIDES_ERR_ARG, "%s: output must have %d limbs", fn, p->level[p->out_reg]);
    if (out->data == in->data) return fides_set_error(FIDES_ERR_ARG, "%s: out may not alias in", fn);
    cudaStream_t st = (cudaStream_t)stream;
    OpTrace tr("op_program", st);
    uint64_t *lt_work = work + (size_t)p->n_phys * ct_words;
    u64 *ws = lt_work + p->lt_words;
    std::vector<double> scale(p->n_regs, 0.0);
    scale[p->in_reg] = in->scale;
    auto reg = [&](int r) {
        fides_ct x;
        x.data = r == p->in_reg ? in->data : work + (size_t)p->phys[r] * ct_words;
        x.n_limbs = p->level[r];
        x.scale = scale[r];
        return x;
    };
    for (size_t i = 0; i < p->instr.size(); ++i) {
        const fides_instr &I = p->instr[i];
        if (p->fuse[i]) {
            const fides_instr &J = p->instr[i + 1];
            fides_ct a = reg(I.a), b = reg(I.b), d = reg(J.dst);
            if (int rc = fides_hmult_rescale_ws(c, &a, &b, p->relin, &d, stream, ws)) {
                char msg[400];
                snprintf(msg, sizeof(msg), "%s", fides_last_error());
                return fides_set_error(rc, "%s: instructions %zu-%zu (HMULT+RESCALE): %s", fn, i, i + 1, msg);
            }
            scale[I.dst] = a.scale * b.scale;
            scale[J.dst] = d.scale;
            ++i;
            continue;
        }
        fides_ct d = reg(I.dst), a, b;
        if (I.op != FIDES_I_CMAC) a = reg(I.a);
        if (reads_b(I.op)) b = reg(I.b);
        int rc = FIDES_OK;
        switch (I.op) {
        case FIDES_I_CMAC: {
            const int t0 = p->lin_start[I.arg], nt = p->lin_start[I.arg + 1] - t0;
            std::vector<const u64 *> x(nt);
            std::vector<int> xl(nt), ci(nt);
            double sc = 0.0;
            for (int t = 0; t < nt; ++t) {
                const fides_ct r = reg(p->lin_reg[t0 + t]);
                x[t] = r.data;
                xl[t] = r.n_limbs;
                ci[t] = p->lin_const[t0 + t];
                if (t == 0) sc = r.scale * p->const_scale[ci[t]];
            }
            rc = launch_cmac(c, x.data(), xl.data(), ci.data(), nt, p->dconst, c->L, d.data, d.n_limbs, st);
            d.scale = sc;
            break;
        }
        case FIDES_I_MODRAISE: rc = fides_modraise_ws(c, &a, &d, stream, ws); break;
        case FIDES_I_LT: {
            const fides_program::Lt &t = p->lt[I.arg];
            rc = fides_linear_transform_ws(c, &a, (int)t.idx.size(), t.idx.data(), t.pts.data(), t.pt_scale, t.n1,
                                           (int)p->rot_keys.size(), p->rot_keys.data(),
                                           lt_work, p->lt_words, &d, stream, ws);
            break;
        }
        case FIDES_I_RESCALE: rc = fides_rescale_ws(c, &a, &d, stream, ws); break;
        case FIDES_I_DROP:
            for (int t = 0; t < 2 && !rc; ++t)
                rc = fides_check_cuda(cudaMemcpyAsync(d.data + (size_t)t * d.n_limbs * N, a.data + (size_t)t * a.n_limbs * N,
                                                      sizeof(uint64_t) * d.n_limbs * N, cudaMemcpyDeviceToDevice, st),
                                      "program: drop");
            d.scale = a.scale;
            break;
        case FIDES_I_COPY:
            rc = fides_check_cuda(cudaMemcpyAsync(d.data, a.data, sizeof(uint64_t) * 2 * a.n_limbs * N,
                                                  cudaMemcpyDeviceToDevice, st),
                                  "program: copy");
            d.scale = a.scale;
            break;
        case FIDES_I_HADD: rc = fides_hadd(c, &a, &b, &d, stream); break;
        case FIDES_I_HSUB: rc = fides_hsub(c, &a, &b, &d, stream); break;
        case FIDES_I_HMULT: rc = fides_hmult_ws(c, &a, &b, p->relin, &d, stream, ws); break;
        case FIDES_I_CONJ: rc = fides_conjugate_ws(c, &a, p->conj, &d, stream, ws); break;
        case FIDES_I_ROT: rc = fides_rotate_ws(c, &a, I.arg, rot_key(p, I.arg), &d, stream, ws); break;
        case FIDES_I_MULI: rc = fides_mul_i(c, &a, I.arg, &d, stream); break;
        case FIDES_I_CMULT:
            rc = fides_scalar_mult(c, &a, p->consts[I.arg].data(), p->const_scale[I.arg], &d, stream);
            break;
        case FIDES_I_CADD: rc = fides_scalar_add(c, &a, p->consts[I.arg].data(), &d, stream); break;
        }
        if (rc) {
            char msg[400];
            snprintf(msg, sizeof(msg), "%s", fides_last_error());
            return fides_set_error(rc, "%s: instruction %zu (op %d): %s", fn, i, I.op, msg);
        }
        scale[I.dst] = d.scale;
    }
    fides_ct o = reg(p->out_reg);
    int rc = fides_check_cuda(cudaMemcpyAsync(out->data, o.data, sizeof(uint64_t) * 2 * o.n_limbs * N,
                                              cudaMemcpyDeviceToDevice, st),
                              "program: output");
    if (!rc) out->scale = p->out_scale;
    return rc;
}
