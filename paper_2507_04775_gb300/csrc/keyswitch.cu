// Single-operation path: hybrid key switching and the CKKS operations built on
// it -- ModUp, key inner product, ModDown (Sec. II-A, Sec. III-F3),
// HMult + relinearisation, HRotate and Rescale (Table I) -- one launch per
// step of the operation, and the C ABI entry points for them.
#include <algorithm>
#include <cstring>
#include <vector>

#include "fides_internal.cuh"
#include "ops_ws.h"
#include "plan.cuh"

namespace {

// Scratch layout of one operation (words from the caller's pool, by default
// the pool of the call's stream, scratch_for):
//   dsrc  [L]      key-switch input of HMult (d2) or HRotate (sigma(c1))
//   key switch     coeff, ext, acc, pc, conv at the top level (ks_carve)
//   last  [2]      Rescale: coefficient form of the dropped limb
//   dd    [2][L]   HMult fused with Rescale: the tensor product d0, d1
//   lastc [4]      ... and the coefficient forms of d0, d1, acc0, acc1 at the dropped limb
struct Scratch {
    u64 *dsrc, *ks, *last, *dd, *lastc;
};

Scratch carve(const fides_ctx *c, u64 *ws, void *stream)
{
    Scratch s;
    s.dsrc = ws ? ws : scratch_for(c, stream);
    s.ks = s.dsrc + (size_t)c->L * c->N;
    s.last = s.ks + ks_scratch_words(c, c->L);
    s.dd = s.last + 2 * (size_t)c->N;
    s.lastc = s.dd + 2 * (size_t)c->L * c->N;
    return s;
}

// HMult fused with Rescale: the coefficient form of the dropped limb l of the
// HMult result, last_t = INTT(d_t,l) + P^-1 (INTT(acc_t,l) - conv_t,l) mod q_l
// (canonical), for t = 0, 1; lastc = [INTT(d0), INTT(d1), INTT(acc0),
// INTT(acc1)] at limb l, conv_t,l < 4 q_l.
__global__ void __launch_bounds__(256) k_hr_last(const u64 *lastc, const u64 *conv0,
                                                 const u64 *conv1, u64 *__restrict__ last,
                                                 const TwPair *__restrict__ md_pinv, const PrimeInfo *__restrict__ P,
                                                 int l, int N)
{
    pdl_enter();
    const TwPair pinv = md_pinv[l];
    const PrimeInfo p = P[l];
    const int t = blockIdx.y;
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (size_t)N) return;
    const u64 dv = lastc[(size_t)t * N + n], av = lastc[(size_t)(2 + t) * N + n];
    const u64 cv = (t ? conv1 : conv0)[n];
    const u64 x = mul_shoup(av + 4 * p.q - cv, pinv, p.q) + dv;   // < 3q
    last[(size_t)t * N + n] = csub(csub(x, p.q2), p.q);
}

int run_modup(const fides_ctx *c, const KsBuffers &B, cudaStream_t st)
{
    std::vector<Seg> v;
    std::vector<BConvJob> jb;
    ks_intt_segs(c, B, v);
    if (int rc = ntt_inverse(c, inline_set(v), ProSrc{}, EpiCanon{}, st)) return rc;
    ks_modup_jobs(c, B, jb);
    if (int rc = launch_bconv(c, inline_bconv(jb), st)) return rc;
    v.clear();
    ks_modup_ntt_segs(c, B, v);
    return ntt_forward(c, inline_set(v), ProSrc{}, EpiCanon{}, st);
}

int run_keyswitch(const fides_ctx *c, const KsBuffers &B, cudaStream_t st)
{
    if (int rc = run_modup(c, B, st)) return rc;
    IPArgs ip;
    memset(&ip, 0, sizeof(ip));
    ip.one = ks_ip_op(c, B);
    if (int rc = launch_inner(c, ip, B.nl + c->K, ks_beta(c, B.nl), st)) return rc;
    std::vector<Seg> v;
    std::vector<BConvJob> jb;
    ks_pinv_segs(c, B, v);
    if (int rc = ntt_inverse(c, inline_set(v), ProSrc{}, EpiCanon{}, st)) return rc;
    ks_moddown_jobs(c, B, jb);
    if (int rc = launch_bconv(c, inline_bconv(jb), st)) return rc;
    v.clear();
    ks_final_segs(c, B, v);
    return ntt_forward(c, inline_set(v), ProSrc{}, EpiSubMul{}, st);
}

KsBuffers ks_buffers(const fides_ctx *c, const u64 *d, int nl, const u64 *evk, u64 *out0, u64 *out1, int mode0,
                     int mode1, const Scratch &s)
{
    KsBuffers B;
    memset(&B, 0, sizeof(B));
    B.d = d; B.nl = nl; B.evk = evk;
    B.out0 = out0; B.out1 = out1; B.mode0 = mode0; B.mode1 = mode1;
    ks_carve(c, B, s.ks);
    return B;
}

int check_ctx(const fides_ctx *c, const char *fn)
{
    if (!c) return fides_set_error(FIDES_ERR_ARG, "%s: ctx is NULL", fn);
    return FIDES_OK;
}

int check_level(const fides_ctx *c, int nl, const char *fn)
{
    if (nl < 1 || nl > c->L) return fides_set_error(FIDES_ERR_ARG, "%s: n_limbs=%d outside [1, %d]", fn, nl, c->L);
    return FIDES_OK;
}

cudaStream_t as_stream(void *s) { return (cudaStream_t)s; }

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
static int ntt_entry(fides_ctx *c, uint64_t *dev, int first_prime, int n_limbs, int batch, void *stream, bool inv)
{
    const char *fn = inv ? "fides_intt" : "fides_ntt";
    if (int rc = check_ctx(c, fn)) return rc;
    if (!dev || n_limbs < 1 || batch < 1 || first_prime < 0 || first_prime + n_limbs > c->L + c->K)
        return fides_set_error(FIDES_ERR_ARG, "%s: bad arguments", fn);
    const size_t N = c->N;
    for (int b0 = 0; b0 < batch; b0 += FIDES_MAX_SEG) {
        LimbSet S = empty_set();
        for (int b = b0; b < std::min(batch, b0 + FIDES_MAX_SEG); ++b) {
            u64 *p = dev + (size_t)b * n_limbs * N;
            add_seg(S, seg_of(p, p, n_limbs, first_prime));
        }
        int rc = inv ? ntt_inverse(c, S, ProSrc{}, EpiCanon{}, as_stream(stream))
                     : ntt_forward(c, S, ProSrc{}, EpiCanon{}, as_stream(stream));
        if (rc) return rc;
    }
    return FIDES_OK;
}

namespace {

// A wait that runs out: one thread waits on an mbarrier that nothing arrives
// on, with the given limit, and reports the timeout the way the tensor-core
// conversion does.
__global__ void k_wait_selftest(u64 limit_ns, int *status)
{
    __shared__ __align__(8) u64 bar;
    const u32 b = smem_addr(&bar);
    mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(b, 0, limit_ns)) atomicOr(status, FIDES_STATUS_WAIT_TIMEOUT);
}

}  // namespace

extern "C" int fides_ctx_selftest_wait(fides_ctx *c, int limit_us, void *stream)
{
    if (!c || limit_us < 1 || limit_us > 100000)
        return fides_set_error(FIDES_ERR_ARG, "fides_ctx_selftest_wait: limit_us must be 1..100000");
    k_wait_selftest<<<1, 1, 0, (cudaStream_t)stream>>>((u64)limit_us * 1000, c->d_status);
    return fides_check_cuda(cudaGetLastError(), "fides_ctx_selftest_wait");
}

extern "C" int fides_ctx_selftest_conversion(fides_ctx *c, int limit_us, void *stream)
{
    if (!c || limit_us < 1 || limit_us > 100000)
        return fides_set_error(FIDES_ERR_ARG, "fides_ctx_selftest_conversion: limit_us must be 1..100000");
    if (!(c->tc_on & 1))
        return fides_set_error(FIDES_ERR_UNSUPPORTED, "fides_ctx_selftest_conversion: ModUp converts on the integer "
                                                      "kernel on this context");
    // the top-level ModUp conversion on the scratch pool of `stream`: its
    // sources hold whatever the pool holds, and only the status word is the
    // result
    KsBuffers B = ks_buffers(c, nullptr, c->L, nullptr, nullptr, nullptr, 0, 0, carve(c, nullptr, stream));
    std::vector<BConvJob> jb;
    ks_modup_jobs(c, B, jb);
    BConvArgs G = inline_bconv(jb);
    G.tc = 1;
    int max_ns = 0, max_dst = 0;
    for (const BConvJob &j : jb) {
        G.tc_smem = std::max(G.tc_smem, bconv_tc_smem(j));
        max_ns = std::max(max_ns, j.n_src);
        max_dst = std::max(max_dst, bconv_targets(j));
    }
    return launch_bconv_tc(c, G, max_ns, max_dst, as_stream(stream), (u64)limit_us * 1000, 1);
}

extern "C" int fides_ntt(fides_ctx *c, uint64_t *dev, int first_prime, int n_limbs, int batch, void *stream)
{
    return ntt_entry(c, dev, first_prime, n_limbs, batch, stream, false);
}

extern "C" int fides_intt(fides_ctx *c, uint64_t *dev, int first_prime, int n_limbs, int batch, void *stream)
{
    return ntt_entry(c, dev, first_prime, n_limbs, batch, stream, true);
}

extern "C" int fides_modup(fides_ctx *c, const uint64_t *d, int nl, uint64_t *ext, void *stream)
{
    if (int rc = check_ctx(c, "fides_modup")) return rc;
    if (int rc = check_level(c, nl, "fides_modup")) return rc;
    if (!d || !ext) return fides_set_error(FIDES_ERR_ARG, "fides_modup: NULL buffer");
    cudaStream_t st = as_stream(stream);
    KsBuffers B = ks_buffers(c, d, nl, nullptr, nullptr, nullptr, 0, 0, carve(c, nullptr, stream));
    B.ext = ext;
    if (int rc = run_modup(c, B, st)) return rc;
    // the digits' own limbs are the input's limbs
    const size_t N = c->N, ne = (size_t)nl + c->K;
    for (int j = 0; j < ks_beta(c, nl); ++j) {
        const int lo = j * c->alpha, hi = std::min(lo + c->alpha, nl);
        int rc = fides_check_cuda(cudaMemcpyAsync(ext + (j * ne + lo) * N, d + (size_t)lo * N,
                                                  sizeof(u64) * (size_t)(hi - lo) * N, cudaMemcpyDeviceToDevice, st),
                                  "fides_modup: copy");
        if (rc) return rc;
    }
    return FIDES_OK;
}

extern "C" int fides_moddown(fides_ctx *c, const uint64_t *x, int nl, uint64_t *out, void *stream)
{
    if (int rc = check_ctx(c, "fides_moddown")) return rc;
    if (int rc = check_level(c, nl, "fides_moddown")) return rc;
    if (!x || !out) return fides_set_error(FIDES_ERR_ARG, "fides_moddown: NULL buffer");
    cudaStream_t st = as_stream(stream);
    KsBuffers B = ks_buffers(c, nullptr, nl, nullptr, out, nullptr, 0, 0, carve(c, nullptr, stream));
    const size_t N = c->N;
    std::vector<Seg> v(1, seg_of(x + (size_t)nl * N, B.pc, c->K, c->L, nullptr, nullptr, 1, 0, c->d_md_nscale));
    if (int rc = ntt_inverse(c, inline_set(v), ProSrc{}, EpiCanon{}, st)) return rc;
    std::vector<BConvJob> jb;
    ks_moddown_jobs(c, B, jb);
    jb.resize(1);
    if (int rc = launch_bconv(c, inline_bconv(jb), st)) return rc;
    v.assign(1, seg_of(B.conv, B.conv, nl, 0, x, out, 1, 0, c->d_md_pinv));
    return ntt_forward(c, inline_set(v), ProSrc{}, EpiSubMul{}, st);
}

extern "C" int fides_keyswitch(fides_ctx *c, const uint64_t *d, int nl, const fides_key *evk, uint64_t *out0,
                               uint64_t *out1, void *stream)
{
    if (int rc = check_ctx(c, "fides_keyswitch")) return rc;
    if (int rc = check_level(c, nl, "fides_keyswitch")) return rc;
    if (!d || !out0 || !out1) return fides_set_error(FIDES_ERR_ARG, "fides_keyswitch: NULL buffer");
    if (int rc = fides_check_key(c, evk, FIDES_GALOIS_ANY, "fides_keyswitch")) return rc;
    OpTrace op("op_keyswitch", as_stream(stream));
    return run_keyswitch(c, ks_buffers(c, d, nl, evk->data, out0, out1, 0, 0, carve(c, nullptr, stream)),
                         as_stream(stream));
}

extern "C" int fides_hmult(fides_ctx *c, const fides_ct *a, const fides_ct *b, const fides_key *rlk, fides_ct *out,
                           void *stream)
{
    if (int rc = check_ctx(c, "fides_hmult")) return rc;
    if (int rc = fides_check_key(c, rlk, FIDES_GALOIS_RELIN, "fides_hmult")) return rc;
    return fides_hmult_ws(c, a, b, rlk->data, out, stream, nullptr);
}

int fides_hmult_ws(fides_ctx *c, const fides_ct *a, const fides_ct *b, const uint64_t *rlk, fides_ct *out,
                   void *stream, u64 *ws)
{
    if (int rc = check_ctx(c, "fides_hmult")) return rc;
    if (!a || !b || !out || !rlk || !a->data || !b->data || !out->data)
        return fides_set_error(FIDES_ERR_ARG, "fides_hmult: NULL argument");
    const int nl = a->n_limbs;
    if (int rc = check_level(c, nl, "fides_hmult")) return rc;
    if (b->n_limbs != nl || out->n_limbs != nl)
        return fides_set_error(FIDES_ERR_ARG, "fides_hmult: level mismatch (%d, %d, %d)", nl, b->n_limbs,
                               out->n_limbs);
    if (out->data == a->data || out->data == b->data)
        return fides_set_error(FIDES_ERR_ARG, "fides_hmult: out may not alias a or b");
    const size_t S = (size_t)nl * c->N;
    cudaStream_t st = as_stream(stream);
    OpTrace op("op_hmult", st);
    const Scratch sc = carve(c, ws, stream);
    KsBuffers B = ks_buffers(c, sc.dsrc, nl, rlk, out->data, out->data + S, 1, 1, sc);
    if (tensor_pass_ok(a->data, b->data, out->data, sc.dsrc)) {
        if (int rc = launch_tensor(c, a->data, b->data, out->data, sc.dsrc, nl, st)) return rc;
    } else {
        B.prep = 1;
        B.pa = a->data;
        B.pb = b->data;
        B.pout = out->data;
    }
    int rc = run_keyswitch(c, B, st);
    if (!rc) out->scale = a->scale * b->scale;
    return rc;
}

extern "C" int fides_hmult_rescale(fides_ctx *c, const fides_ct *a, const fides_ct *b, const fides_key *rlk,
                                   fides_ct *out, void *stream)
{
    if (int rc = check_ctx(c, "fides_hmult_rescale")) return rc;
    if (int rc = fides_check_key(c, rlk, FIDES_GALOIS_RELIN, "fides_hmult_rescale")) return rc;
    return fides_hmult_rescale_ws(c, a, b, rlk->data, out, stream, nullptr);
}

// Rescale(HMult(a, b)) in one key switch: the tensor product goes to scratch;
// the ModDown's INTT also transforms limb l = nl - 1 of d0, d1, acc0, acc1;
// k_hr_last forms the coefficient form of the dropped limb; one forward NTT
// over the remaining limbs gives q_l^-1 (d + P^-1 acc - NTT(P^-1 conv +
// [last])) (ProHmRs / EpiHmRs).  Residues equal fides_hmult then
// fides_rescale.
int fides_hmult_rescale_ws(fides_ctx *c, const fides_ct *a, const fides_ct *b, const uint64_t *rlk, fides_ct *out,
                           void *stream, u64 *ws)
{
    const char *fn = "fides_hmult_rescale";
    if (int rc = check_ctx(c, fn)) return rc;
    if (!a || !b || !out || !rlk || !a->data || !b->data || !out->data)
        return fides_set_error(FIDES_ERR_ARG, "%s: NULL argument", fn);
    const int nl = a->n_limbs, l = nl - 1;
    if (int rc = check_level(c, nl, fn)) return rc;
    if (nl < 2 || b->n_limbs != nl || out->n_limbs != l)
        return fides_set_error(FIDES_ERR_ARG,
                               "%s: needs n_limbs >= 2, equal input levels and out->n_limbs = n_limbs - 1", fn);
    if (out->data == a->data || out->data == b->data)
        return fides_set_error(FIDES_ERR_ARG, "%s: out may not alias a or b", fn);
    const size_t N = c->N, S = (size_t)nl * N, ne = (size_t)nl + c->K;
    cudaStream_t st = as_stream(stream);
    OpTrace op("op_hmult_rescale", st);
    const Scratch sc = carve(c, ws, stream);
    KsBuffers B = ks_buffers(c, sc.dsrc, nl, rlk, sc.dd, sc.dd + S, 1, 1, sc);
    if (tensor_pass_ok(a->data, b->data, sc.dd, sc.dsrc)) {
        if (int rc = launch_tensor(c, a->data, b->data, sc.dd, sc.dsrc, nl, st)) return rc;
    } else {
        B.prep = 1;
        B.pa = a->data;
        B.pb = b->data;
        B.pout = sc.dd;
    }
    if (int rc = run_modup(c, B, st)) return rc;
    IPArgs ip;
    memset(&ip, 0, sizeof(ip));
    ip.one = ks_ip_op(c, B);
    if (int rc = launch_inner(c, ip, nl + c->K, ks_beta(c, nl), st)) return rc;
    // ModDown INTT of the special limbs, plus limb l of d0, d1, acc0, acc1
    std::vector<Seg> v;
    ks_pinv_segs(c, B, v);
    for (int t = 0; t < 2; ++t) v.push_back(seg_of(sc.dd + t * S + (size_t)l * N, sc.lastc + t * N, 1, l));
    for (int t = 0; t < 2; ++t)
        v.push_back(seg_of(B.acc + (t * ne + l) * N, sc.lastc + (2 + t) * N, 1, l));
    if (int rc = ntt_inverse(c, inline_set(v), ProSrc{}, EpiCanon{}, st)) return rc;
    std::vector<BConvJob> jb;
    ks_moddown_jobs(c, B, jb);
    if (int rc = launch_bconv(c, inline_bconv(jb), st)) return rc;
    FIDES_LAUNCH("k_hr_last", st, k_hr_last, dim3((c->N + 255) / 256, 2), dim3(256), (const u64 *)sc.lastc,
                 (const u64 *)(B.conv + (size_t)l * N), (const u64 *)(B.conv + (size_t)(nl + l) * N), sc.last,
                 (const TwPair *)c->d_md_pinv, (const PrimeInfo *)c->d_prime, l, c->N);
    if (int rc = fides_check_cuda(cudaGetLastError(), "fides_hmult_rescale: last limb")) return rc;
    // one forward NTT over limbs 0 .. l-1 of both polynomials
    v.clear();
    for (int t = 0; t < 2; ++t) {
        u64 *cv = B.conv + (size_t)t * nl * N;
        Seg g = seg_of(sc.last + t * N, cv, l, 0, B.acc + t * ne * N, out->data + (size_t)t * l * N, 0, 0,
                       c->d_hr + (size_t)l * c->L * 2);
        g.side = sc.dd + t * S;
        g.g = c->round_nearest ? c->primes[l] : 0;   // centred lift of the dropped limb (round to nearest)
        v.push_back(g);
    }
    int rc = ntt_forward(c, inline_set(v), ProHmRs{}, EpiHmRs{}, st);
    if (!rc) out->scale = a->scale * b->scale / (double)c->primes[l];
    return rc;
}

// sigma_g of a ciphertext with key switching (HRotate, Conjugate)
static int automorph_entry(fides_ctx *c, const fides_ct *a, u64 g, const uint64_t *rk, fides_ct *out, void *stream,
                           const char *fn, const char *trace, u64 *ws)
{
    if (int rc = check_ctx(c, fn)) return rc;
    if (!a || !out || !rk || !a->data || !out->data) return fides_set_error(FIDES_ERR_ARG, "%s: NULL argument", fn);
    const int nl = a->n_limbs;
    if (int rc = check_level(c, nl, fn)) return rc;
    if (out->n_limbs != nl) return fides_set_error(FIDES_ERR_ARG, "%s: level mismatch", fn);
    if (out->data == a->data) return fides_set_error(FIDES_ERR_ARG, "%s: out may not alias a", fn);
    const size_t S = (size_t)nl * c->N;
    cudaStream_t st = as_stream(stream);
    OpTrace op(trace, st);
    const Scratch sc = carve(c, ws, stream);
    KsBuffers B = ks_buffers(c, sc.dsrc, nl, rk, out->data, out->data + S, 1, 0, sc);
    B.prep = 2;
    B.pa = a->data;
    B.pout = out->data;
    B.g = g;
    int rc = run_keyswitch(c, B, st);
    if (!rc) out->scale = a->scale;
    return rc;
}

int fides_rotate_ws(fides_ctx *c, const fides_ct *a, int64_t steps, const uint64_t *rk, fides_ct *out, void *stream,
                    u64 *ws)
{
    if (int rc = check_ctx(c, "fides_rotate")) return rc;
    return automorph_entry(c, a, fides_galois_elt(c, steps), rk, out, stream, "fides_rotate", "op_rotate", ws);
}

extern "C" int fides_rotate(fides_ctx *c, const fides_ct *a, int64_t steps, const fides_key *rk, fides_ct *out,
                            void *stream)
{
    if (int rc = check_ctx(c, "fides_rotate")) return rc;
    if (int rc = fides_check_key(c, rk, fides_galois_elt(c, steps), "fides_rotate")) return rc;
    return fides_rotate_ws(c, a, steps, rk->data, out, stream, nullptr);
}

int fides_conjugate_ws(fides_ctx *c, const fides_ct *a, const uint64_t *ck, fides_ct *out, void *stream, u64 *ws)
{
    if (int rc = check_ctx(c, "fides_conjugate")) return rc;
    return automorph_entry(c, a, 2 * (u64)c->N - 1, ck, out, stream, "fides_conjugate", "op_conjugate", ws);
}

extern "C" int fides_conjugate(fides_ctx *c, const fides_ct *a, const fides_key *ck, fides_ct *out, void *stream)
{
    if (int rc = check_ctx(c, "fides_conjugate")) return rc;
    if (int rc = fides_check_key(c, ck, 2 * (u64)c->N - 1, "fides_conjugate")) return rc;
    return fides_conjugate_ws(c, a, ck->data, out, stream, nullptr);
}

extern "C" int fides_hsquare(fides_ctx *c, const fides_ct *a, const fides_key *rlk, fides_ct *out, void *stream)
{
    return fides_hmult(c, a, a, rlk, out, stream);
}

extern "C" int fides_rotate_hoisted(fides_ctx *c, const fides_ct *a, int n_rot, const int64_t *steps,
                                    const fides_key *const *rks, fides_ct *outs, void *stream)
{
    const char *fn = "fides_rotate_hoisted";
    if (int rc = check_ctx(c, fn)) return rc;
    if (!steps || !rks) return fides_set_error(FIDES_ERR_ARG, "%s: NULL argument", fn);
    if (n_rot < 1 || n_rot > 64) return fides_set_error(FIDES_ERR_ARG, "%s: n_rot=%d outside [1, 64]", fn, n_rot);
    const uint64_t *keys[64];
    for (int k = 0; k < n_rot; ++k) {
        if (int rc = fides_check_key(c, rks[k], fides_galois_elt(c, steps[k]), fn)) return rc;
        keys[k] = rks[k]->data;
    }
    return fides_rotate_hoisted_ws(c, a, n_rot, steps, keys, outs, stream, nullptr);
}

int fides_rotate_hoisted_ws(fides_ctx *c, const fides_ct *a, int n_rot, const int64_t *steps,
                            const uint64_t *const *rks, fides_ct *outs, void *stream, u64 *ws)
{
    const char *fn = "fides_rotate_hoisted";
    if (int rc = check_ctx(c, fn)) return rc;
    if (!a || !a->data || !steps || !rks || !outs) return fides_set_error(FIDES_ERR_ARG, "%s: NULL argument", fn);
    if (n_rot < 1 || n_rot > 64) return fides_set_error(FIDES_ERR_ARG, "%s: n_rot=%d outside [1, 64]", fn, n_rot);
    const int nl = a->n_limbs;
    if (int rc = check_level(c, nl, fn)) return rc;
    for (int k = 0; k < n_rot; ++k) {
        if (!rks[k] || !outs[k].data) return fides_set_error(FIDES_ERR_ARG, "%s: rotation %d: NULL key or output", fn, k);
        if (outs[k].n_limbs != nl) return fides_set_error(FIDES_ERR_ARG, "%s: rotation %d: level mismatch", fn, k);
    }
    const size_t S = (size_t)nl * c->N;
    cudaStream_t st = as_stream(stream);
    OpTrace op("op_rotate_hoisted", st);
    // one ModUp of c1 (the INTT reads c1 itself; the digits' own limbs are c1's)
    KsBuffers B = ks_buffers(c, a->data + S, nl, nullptr, nullptr, nullptr, 0, 0, carve(c, ws, stream));
    if (int rc = run_modup(c, B, st)) return rc;
    for (int k = 0; k < n_rot; ++k) {
        B.evk = rks[k];
        B.out0 = outs[k].data;
        B.out1 = outs[k].data + S;
        const u64 g = fides_galois_elt(c, steps[k]);
        IPArgs ip;
        memset(&ip, 0, sizeof(ip));
        ip.one = ks_ip_op(c, B);
        ip.one.g = g;
        if (int rc = launch_inner(c, ip, nl + c->K, ks_beta(c, nl), st)) return rc;
        std::vector<Seg> v;
        std::vector<BConvJob> jb;
        ks_pinv_segs(c, B, v);
        if (int rc = ntt_inverse(c, inline_set(v), ProSrc{}, EpiCanon{}, st)) return rc;
        ks_moddown_jobs(c, B, jb);
        if (int rc = launch_bconv(c, inline_bconv(jb), st)) return rc;
        v.clear();
        ks_final_segs(c, B, v);
        v[0].mode = 2;                  // out0 = sigma_g(c0) + P^-1 (acc0 - conv0)
        v[0].side = const_cast<u64 *>(a->data);
        v[0].g = g;
        v[1].mode = 0;                  // out1 = P^-1 (acc1 - conv1)
        if (int rc = ntt_forward(c, inline_set(v), ProSrc{}, EpiSubMulRot{}, st)) return rc;
        outs[k].scale = a->scale;
    }
    return FIDES_OK;
}

// Rescale (Table I): floor(x / q_l), or round(x / q_l) with nearest (the
// centred SwitchModulo of the dropped limb) -- asked for, or the context's
// rounding mode.
static int rescale_entry(fides_ctx *c, const fides_ct *a, fides_ct *out, void *stream, u64 *ws, bool nearest)
{
    const char *fn = nearest ? "fides_rescale_round" : "fides_rescale";
    if (int rc = check_ctx(c, fn)) return rc;
    if (!a || !out || !a->data || !out->data) return fides_set_error(FIDES_ERR_ARG, "%s: NULL argument", fn);
    const int nl = a->n_limbs;
    if (int rc = check_level(c, nl, fn)) return rc;
    if (nl < 2 || out->n_limbs != nl - 1)
        return fides_set_error(FIDES_ERR_ARG, "%s: needs n_limbs >= 2 and out->n_limbs = n_limbs - 1", fn);
    cudaStream_t st = as_stream(stream);
    OpTrace op(nearest ? "op_rescale_round" : "op_rescale", st);
    Scratch s = carve(c, ws, stream);
    std::vector<Seg> v;
    rs_intt_segs(c, a->data, nl, s.last, v);
    if (int rc = ntt_inverse(c, inline_set(v), ProSrc{}, EpiCanon{}, st)) return rc;
    v.clear();
    rs_final_segs(c, a->data, nl, s.last, out->data, v, nearest || c->round_nearest);
    int rc = ntt_forward(c, inline_set(v), ProSwitchMod{}, EpiSubMul{}, st);
    if (!rc) out->scale = a->scale / (double)c->primes[nl - 1];
    return rc;
}

extern "C" int fides_rescale(fides_ctx *c, const fides_ct *a, fides_ct *out, void *stream)
{
    return fides_rescale_ws(c, a, out, stream, nullptr);
}

extern "C" int fides_rescale_round(fides_ctx *c, const fides_ct *a, fides_ct *out, void *stream)
{
    return rescale_entry(c, a, out, stream, nullptr, true);
}

int fides_rescale_ws(fides_ctx *c, const fides_ct *a, fides_ct *out, void *stream, u64 *ws)
{
    return rescale_entry(c, a, out, stream, ws, false);
}

extern "C" int fides_modraise(fides_ctx *c, const fides_ct *a, fides_ct *out, void *stream)
{
    return fides_modraise_ws(c, a, out, stream, nullptr);
}

int fides_modraise_ws(fides_ctx *c, const fides_ct *a, fides_ct *out, void *stream, u64 *ws)
{
    const char *fn = "fides_modraise";
    if (int rc = check_ctx(c, fn)) return rc;
    if (!a || !out || !a->data || !out->data) return fides_set_error(FIDES_ERR_ARG, "%s: NULL argument", fn);
    if (a->n_limbs != 1) return fides_set_error(FIDES_ERR_ARG, "%s: input must have one limb", fn);
    const int nl = out->n_limbs;
    if (int rc = check_level(c, nl, fn)) return rc;
    if (out->data == a->data) return fides_set_error(FIDES_ERR_ARG, "%s: out may not alias a", fn);
    const size_t N = c->N;
    cudaStream_t st = as_stream(stream);
    OpTrace op("op_modraise", st);
    Scratch s = carve(c, ws, stream);
    std::vector<Seg> v;
    for (int t = 0; t < 2; ++t) v.push_back(seg_of(a->data + (size_t)t * N, s.last + (size_t)t * N, 1, 0));
    if (int rc = ntt_inverse(c, inline_set(v), ProSrc{}, EpiCanon{}, st)) return rc;
    v.clear();
    for (int t = 0; t < 2; ++t) {
        Seg g = seg_of(s.last + (size_t)t * N, out->data + (size_t)t * nl * N, nl, 0, nullptr, nullptr, 0, 0, c->d_raise);
        g.g = c->primes[0];
        v.push_back(g);
    }
    int rc = ntt_forward(c, inline_set(v), ProRaise{}, EpiCanon{}, st);
    if (!rc) out->scale = a->scale;
    return rc;
}
