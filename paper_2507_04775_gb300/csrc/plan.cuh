// Host-side description of the work of one operation, as lists of NTT
// segments, base-conversion jobs and element-wise descriptors.  The single-
// operation path turns each list into one inline launch; the batched path
// concatenates the lists of many operations into device-resident tables so
// that one launch per stage covers the whole batch.
#pragma once

#include <vector>

#include "kernels.cuh"

namespace {

// Buffers of one hybrid key switch of d (nl limbs, evaluation form) with key
// evk (Sec. II-A): the ModUp (Sec. III-F3), the key inner product and the
// ModDown of both accumulators, whose results are stored (mode 0) or added
// (mode 1) into out0 / out1.
struct KsBuffers {
    const u64 *d;       // [nl]  key-switch input (written by a fused prep, see below)
    int nl;
    // optional element-wise step fused into the first INTT (ProPrep): 0 none,
    // 1 HMult tensor product of ciphertexts pa, pb (d0, d1 into pout, d2 into
    // d), 2 HRotate automorphism g of ciphertext pa (sigma(c0) into pout,
    // sigma(c1) into d)
    int prep;
    const u64 *pa, *pb;
    u64 *pout;
    u64 g;
    const u64 *evk;     // [dnum][2][L+K]
    u64 *out0, *out1;   // [nl] each
    int mode0, mode1;
    u64 *coeff;         // [nl]          coefficient form of d
    u64 *ext;           // [beta][nl+K]  ModUp output
    u64 *acc;           // [2][nl+K]     inner-product accumulators
    u64 *pc;            // [2][K]        coefficient form of the special limbs
    u64 *conv;          // [2][nl]       converted limbs (NTT intermediate)
};

inline int ks_beta(const fides_ctx *c, int nl) { return (nl + c->alpha - 1) / c->alpha; }

// Words of scratch one key switch at nl limbs needs (coeff, ext, acc, pc, conv),
// for ring degree N, K special primes and digits of alpha limbs.
inline size_t ks_scratch_words_of(int N, int K, int alpha, int nl)
{
    const size_t ne = (size_t)nl + K, beta = (size_t)(nl + alpha - 1) / alpha;
    return (size_t)N * ((size_t)nl + beta * ne + 2 * ne + 2 * (size_t)K + 2 * (size_t)nl);
}

inline size_t ks_scratch_words(const fides_ctx *c, int nl) { return ks_scratch_words_of(c->N, c->K, c->alpha, nl); }

// Lays out the scratch of one key switch from `p`; returns the end.
inline u64 *ks_carve(const fides_ctx *c, KsBuffers &B, u64 *p)
{
    const size_t N = c->N, nl = B.nl, ne = nl + c->K;
    B.coeff = p; p += nl * N;
    B.ext = p; p += ks_beta(c, B.nl) * ne * N;
    B.acc = p; p += 2 * ne * N;
    B.pc = p; p += 2 * (size_t)c->K * N;
    B.conv = p; p += 2 * nl * N;
    return p;
}

// 1. ModUp, INTT of d into coefficient form, with the conversion's scaling
//    qhat_i^-1 folded into the final N^-1 (the conversion reads [x_i qhat_i^-1]),
//    and with the preparation of d fused into its first pass.
inline void ks_intt_segs(const fides_ctx *c, const KsBuffers &B, std::vector<Seg> &v)
{
    const size_t nl = B.nl;
    Seg g = seg_of(B.prep ? B.pa : B.d, B.coeff, B.nl, 0, B.pb, B.pout, 1, B.prep,
                   c->d_mu_nscale + nl * (nl - 1));   // pairs: 2 (nl(nl-1)/2) entries precede level nl
    g.side = B.prep ? const_cast<u64 *>(B.d) : nullptr;
    g.g = B.g;
    g.pstride = (int)(nl * c->N);
    v.push_back(g);
}

// 2. ModUp, base conversion of every digit D_j (contiguous blocks of alpha
//    limbs from limb 0, the last one partial) to its complement in Q_l and to P.
inline void ks_modup_jobs(const fides_ctx *c, const KsBuffers &B, std::vector<BConvJob> &v)
{
    const int N = c->N, K = c->K, L = c->L, nl = B.nl, ne = nl + K, alpha = c->alpha;
    for (int j = 0; j < ks_beta(c, nl); ++j) {
        const int lo = j * alpha, hi = std::min(lo + alpha, nl);
        u64 *e = B.ext + (size_t)j * ne * N;
        BConvJob J;
        memset(&J, 0, sizeof(J));
        J.src = B.coeff + (size_t)lo * N;
        J.n_src = hi - lo;
        J.prescaled = 1;
        J.src_prime0 = lo;
        const size_t off = ((size_t)(nl - 1) * c->dnum + j) * alpha;
        J.scale = c->d_mu_scale + off;
        J.mat = c->d_mu_mat + off * (L + K);
        J.ld = L + K;
        if (c->tc_on & 1) J.tc = (const unsigned char *)c->d_tc + c->tc_mu_off[nl - 1][j];
        if (lo > 0) J.run[J.nrun++] = BConvRun{e, lo, 0};
        if (hi < nl) J.run[J.nrun++] = BConvRun{e + (size_t)hi * N, nl - hi, hi};
        J.run[J.nrun++] = BConvRun{e + (size_t)nl * N, K, L};
        v.push_back(J);
    }
}

// 3. ModUp, NTT of the converted limbs (in place).
inline void ks_modup_ntt_segs(const fides_ctx *c, const KsBuffers &B, std::vector<Seg> &v)
{
    const int N = c->N, K = c->K, L = c->L, nl = B.nl, ne = nl + K, alpha = c->alpha;
    for (int j = 0; j < ks_beta(c, nl); ++j) {
        const int lo = j * alpha, hi = std::min(lo + alpha, nl);
        u64 *e = B.ext + (size_t)j * ne * N;
        if (lo > 0) v.push_back(seg_of(e, e, lo, 0));
        if (hi < nl) v.push_back(seg_of(e + (size_t)hi * N, e + (size_t)hi * N, nl - hi, hi));
        v.push_back(seg_of(e + (size_t)nl * N, e + (size_t)nl * N, K, L));
    }
}

// 4. Key inner product.
inline IPOp ks_ip_op(const fides_ctx *c, const KsBuffers &B)
{
    IPOp o;
    o.ext = B.ext; o.dsrc = B.d; o.evk = B.evk; o.acc = B.acc;
    o.nl = B.nl; o.ne = B.nl + c->K; o.beta = ks_beta(c, B.nl); o.alpha = c->alpha;
    o.g = 0;
    return o;
}

// 5. ModDown, INTT of both accumulators' special limbs.
inline void ks_pinv_segs(const fides_ctx *c, const KsBuffers &B, std::vector<Seg> &v)
{
    const size_t N = c->N, ne = (size_t)B.nl + c->K;
    for (int t = 0; t < 2; ++t)
        v.push_back(seg_of(B.acc + (t * ne + B.nl) * N, B.pc + (size_t)t * c->K * N, c->K, c->L, nullptr, nullptr, 1,
                           0, c->d_md_nscale));
}

// 6. ModDown, base conversion P -> Q_l of both accumulators.
inline void ks_moddown_jobs(const fides_ctx *c, const KsBuffers &B, std::vector<BConvJob> &v)
{
    const size_t N = c->N;
    for (int t = 0; t < 2; ++t) {
        BConvJob J;
        memset(&J, 0, sizeof(J));
        J.src = B.pc + (size_t)t * c->K * N;
        J.n_src = c->K;
        J.prescaled = 1;
        J.src_prime0 = c->L;
        J.scale = c->d_md_scale;
        J.mat = c->d_md_mat;
        J.ld = c->L + c->K;
        J.nrun = 1;
        J.run[0] = BConvRun{B.conv + (size_t)t * B.nl * N, B.nl, 0};
        if (c->tc_on & 2) J.tc = (const unsigned char *)c->d_tc + c->tc_md_off;
        J.tc_corr = 1;
        J.centred = c->round_nearest;   // round-to-nearest: convert the centred residues
        J.corr = c->d_md_negp;
        v.push_back(J);
    }
}

// 7. ModDown, NTT of the converted limbs with the fused epilogue
//    out_t (+)= P^-1 (acc_t - NTT(conv_t)) (Sec. III-F5 "ModDown fusion").
inline void ks_final_segs(const fides_ctx *c, const KsBuffers &B, std::vector<Seg> &v)
{
    const size_t N = c->N, ne = (size_t)B.nl + c->K;
    u64 *outs[2] = {B.out0, B.out1};
    const int modes[2] = {B.mode0, B.mode1};
    for (int t = 0; t < 2; ++t) {
        u64 *cv = B.conv + (size_t)t * B.nl * N;
        v.push_back(seg_of(cv, cv, B.nl, 0, B.acc + t * ne * N, outs[t], 1, modes[t], c->d_md_pinv));
    }
}

// Rescale of a ciphertext x ([2][nl]) into out ([2][nl-1]); `last` is two
// limbs of scratch.  (a) INTT of the dropped limb of both polynomials;
// (b) NTT under q_i of its SwitchModulo with the fused epilogue
// out_i = q_l^-1 (x_i - .) (Sec. III-F5 "Rescale fusion").
// V: any sink with push_back(const Seg &) -- a std::vector, or SetSink,
// which fills a LimbSet in place without touching the heap.
template <class V>
inline void rs_intt_segs(const fides_ctx *c, const u64 *x, int nl, u64 *last, V &v)
{
    const size_t N = c->N;
    for (int t = 0; t < 2; ++t) v.push_back(seg_of(x + ((size_t)t * nl + nl - 1) * N, last + t * N, 1, nl - 1));
}

// nearest: round-to-nearest Rescale (the centred SwitchModulo, ProSwitchMod
// with g = q_l) instead of floor.
template <class V>
inline void rs_final_segs(const fides_ctx *c, const u64 *x, int nl, u64 *last, u64 *out, V &v,
                          bool nearest = false)
{
    const size_t N = c->N;
    const int l = nl - 1;
    for (int t = 0; t < 2; ++t) {
        u64 *o = out + (size_t)t * l * N;
        Seg g = seg_of(last + t * N, o, l, 0, x + (size_t)t * nl * N, o, 0, 0, c->d_rs_qlinv + (size_t)l * c->L);
        g.g = nearest ? c->primes[l] : 0;
        v.push_back(g);
    }
}

// A sink for the segment builders that appends to a LimbSet (no heap use).
struct SetSink {
    LimbSet &S;
    void push_back(const Seg &g) { add_seg(S, g); }
};

// Inline limb set of at most FIDES_MAX_SEG segments.
inline LimbSet inline_set(const std::vector<Seg> &v)
{
    LimbSet S = empty_set();
    for (const Seg &g : v) add_seg(S, g);
    return S;
}

inline BConvArgs inline_bconv(const std::vector<BConvJob> &v)
{
    BConvArgs A;
    memset(&A, 0, sizeof(A));
    for (const BConvJob &j : v) A.job[A.njob++] = j;
    return A;
}

}  // namespace
