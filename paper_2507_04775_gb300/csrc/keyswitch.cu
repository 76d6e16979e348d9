// Hybrid key switching and the CKKS operations built on it, for sm_103a:
// fast base conversion (Sec. III-F3, Eq. 1), ModUp, the key inner product
// (Sec. III-F5 "Dot product fusion"), ModDown, HMult + relinearisation,
// HRotate and Rescale (Table I), and the C ABI entry points for them.
#include <algorithm>
#include <cstring>

#include "fides_internal.cuh"
#include "ntt.cuh"

namespace {

// ---------------------------------------------------------------------------
// Fast base conversion (Eq. 1): for every target prime p and coefficient n,
//   y_p[n] = ( sum_i [x_i[n] * qhat_i^-1]_{q_i} * [qhat_i]_p ) mod p.
// One thread per coefficient and per group of up to BCONV_TG targets: the
// scaled source values stay in registers and are reused for every target of
// the group; the partial dot products accumulate in 128 bits (four 32-bit
// words, one carry chain per partial product) and are reduced once per output
// (Sec. III-F3: lazy 128-bit accumulation, one reduction before the
// write-back).  The conversion matrix of the group is staged in shared memory
// (every thread reads the same entry).  NS is the exact number of source limbs
// (0: any number up to FIDES_MAX_SRC, with guarded loops).
// ---------------------------------------------------------------------------
struct BConvRun {
    u64 *dst;
    int count;
    int prime0;
};

struct BConvJob {
    const u64 *src;          // n_src contiguous coefficient-form limbs
    int n_src;
    int src_prime0;
    const TwPair *scale;     // [n_src] qhat_i^-1 mod q_i
    const u64 *mat;          // [n_src][ld]: [qhat_i]_{prime z}
    int ld;
    int nrun;
    BConvRun run[3];
};

struct BConvArgs {
    int njob;
    BConvJob job[FIDES_MAX_DIGITS];
};

constexpr int BCONV_TG = 16;     // targets per CTA

struct Acc128 {
    u32 w0, w1, w2, w3;
};

// c += a * b for 64-bit a, b (the full 128-bit product), as three carry chains
// of 32-bit multiply-adds.
__device__ __forceinline__ void mac_wide(Acc128 &c, u64 a, u64 b)
{
    const u32 a0 = (u32)a, a1 = (u32)(a >> 32), b0 = (u32)b, b1 = (u32)(b >> 32);
    asm("mad.lo.cc.u32 %0, %4, %6, %0;\n\t"
        "madc.hi.cc.u32 %1, %4, %6, %1;\n\t"
        "madc.lo.cc.u32 %2, %5, %7, %2;\n\t"
        "madc.hi.u32 %3, %5, %7, %3;\n\t"
        "mad.lo.cc.u32 %1, %4, %7, %1;\n\t"
        "madc.hi.cc.u32 %2, %4, %7, %2;\n\t"
        "addc.u32 %3, %3, 0;\n\t"
        "mad.lo.cc.u32 %1, %5, %6, %1;\n\t"
        "madc.hi.cc.u32 %2, %5, %6, %2;\n\t"
        "addc.u32 %3, %3, 0;"
        : "+r"(c.w0), "+r"(c.w1), "+r"(c.w2), "+r"(c.w3)
        : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
}

__device__ __forceinline__ u64 reduce_acc(const Acc128 &c, const PrimeInfo &p)
{
    return reduce128(((u64)c.w3 << 32) | c.w2, ((u64)c.w1 << 32) | c.w0, p);
}

template <int NS>
__global__ void __launch_bounds__(256) k_bconv(BConvArgs A, const PrimeInfo *__restrict__ P, int logN)
{
    constexpr int MS = NS > 0 ? NS : FIDES_MAX_SRC;
    pdl_enter();
    const BConvJob &B = A.job[blockIdx.y];
    __shared__ u64 smat[BCONV_TG * MS];
    __shared__ PrimeInfo sp[BCONV_TG];
    __shared__ u64 *sdst[BCONV_TG];
    const int N = 1 << logN;
    const int ns = NS > 0 ? NS : B.n_src;

    int ndst = 0;
    for (int r = 0; r < B.nrun; ++r) ndst += B.run[r].count;
    const int d0 = blockIdx.z * BCONV_TG;
    const int nd = min(BCONV_TG, ndst - d0);
    if (nd <= 0) return;
    if (threadIdx.x < nd) {
        int rem = d0 + threadIdx.x, pz = 0;
        u64 *ptr = nullptr;
        for (int r = 0; r < B.nrun; ++r) {
            if (rem < B.run[r].count) {
                pz = B.run[r].prime0 + rem;
                ptr = B.run[r].dst + (size_t)rem * N;
                break;
            }
            rem -= B.run[r].count;
        }
        sp[threadIdx.x] = P[pz];
        sdst[threadIdx.x] = ptr;
        for (int i = 0; i < ns; ++i) smat[threadIdx.x * MS + i] = B.mat[(size_t)i * B.ld + pz];
    }
    __syncthreads();

    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    u64 v[MS];
#pragma unroll
    for (int i = 0; i < MS; ++i) {
        if (NS > 0 || i < ns) {
            const u64 qi = P[B.src_prime0 + i].q;
            const u64 x = B.src[(size_t)i * N + n];
            v[i] = csub(mul_shoup(x, B.scale[i], qi), qi);
        } else {
            v[i] = 0;
        }
    }
    int d = 0;
    for (; d + 1 < nd; d += 2) {
        Acc128 c0 = {0, 0, 0, 0}, c1 = {0, 0, 0, 0};
        const u64 *m0 = smat + d * MS, *m1 = m0 + MS;
#pragma unroll
        for (int i = 0; i < MS; ++i) {
            if (NS > 0 || i < ns) {
                mac_wide(c0, v[i], m0[i]);
                mac_wide(c1, v[i], m1[i]);
            }
        }
        sdst[d][n] = reduce_acc(c0, sp[d]);
        sdst[d + 1][n] = reduce_acc(c1, sp[d + 1]);
    }
    if (d < nd) {
        Acc128 c0 = {0, 0, 0, 0};
        const u64 *m0 = smat + d * MS;
#pragma unroll
        for (int i = 0; i < MS; ++i)
            if (NS > 0 || i < ns) mac_wide(c0, v[i], m0[i]);
        sdst[d][n] = reduce_acc(c0, sp[d]);
    }
}

template <int NS>
void launch_bconv_ns(const fides_ctx *c, const BConvArgs &A, int max_dst, cudaStream_t st)
{
    dim3 grid(c->N / 256, A.njob, (max_dst + BCONV_TG - 1) / BCONV_TG), block(256);
    FIDES_LAUNCH("k_bconv", st, k_bconv<NS>, grid, block, A, c->d_prime, c->logN);
}

// Launches one conversion per distinct source count (a ragged last digit
// gets its own launch, so every launch runs fully unrolled loops).
int launch_bconv(const fides_ctx *c, const BConvArgs &A, int /*max_src*/, cudaStream_t st)
{
    if (A.njob == 0) return FIDES_OK;
    bool done[FIDES_MAX_DIGITS] = {false};
    for (int j = 0; j < A.njob; ++j) {
        if (done[j]) continue;
        const int ns = A.job[j].n_src;
        BConvArgs G;
        memset(&G, 0, sizeof(G));
        int max_dst = 0;
        for (int k = j; k < A.njob; ++k) {
            if (done[k] || A.job[k].n_src != ns) continue;
            done[k] = true;
            G.job[G.njob++] = A.job[k];
            int nd = 0;
            for (int r = 0; r < A.job[k].nrun; ++r) nd += A.job[k].run[r].count;
            max_dst = std::max(max_dst, nd);
        }
        switch (ns) {
        case 1: launch_bconv_ns<1>(c, G, max_dst, st); break;
        case 2: launch_bconv_ns<2>(c, G, max_dst, st); break;
        case 3: launch_bconv_ns<3>(c, G, max_dst, st); break;
        case 4: launch_bconv_ns<4>(c, G, max_dst, st); break;
        case 5: launch_bconv_ns<5>(c, G, max_dst, st); break;
        case 6: launch_bconv_ns<6>(c, G, max_dst, st); break;
        case 7: launch_bconv_ns<7>(c, G, max_dst, st); break;
        case 8: launch_bconv_ns<8>(c, G, max_dst, st); break;
        case 9: launch_bconv_ns<9>(c, G, max_dst, st); break;
        case 10: launch_bconv_ns<10>(c, G, max_dst, st); break;
        case 11: launch_bconv_ns<11>(c, G, max_dst, st); break;
        case 12: launch_bconv_ns<12>(c, G, max_dst, st); break;
        default: launch_bconv_ns<0>(c, G, max_dst, st); break;
        }
        if (int rc = fides_check_cuda(cudaGetLastError(), "bconv launch")) return rc;
    }
    return FIDES_OK;
}

// ---------------------------------------------------------------------------
// Key inner product: acc_t[z] = sum_j ext_j[z] * evk_{j,t}[key limb of z],
// t = 0, 1, over the nl q-limbs and the K special limbs; 128-bit lazy sums.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_inner(const u64 *__restrict__ ext, int beta, int nl, int ne,
                                               const u64 *__restrict__ evk, int L, int nfull,
                                               u64 *__restrict__ acc, const PrimeInfo *__restrict__ P, int logN)
{
    pdl_enter();
    const int N = 1 << logN;
    const int z = blockIdx.y;
    const int pz = z < nl ? z : L + (z - nl);
    const PrimeInfo pr = P[pz];
    const size_t n = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    U128 a0 = {0, 0}, a1 = {0, 0};
    for (int j = 0; j < beta; ++j) {
        const u64 e = ext[((size_t)j * ne + z) * N + n];
        const u64 k0 = evk[(((size_t)j * 2 + 0) * nfull + pz) * N + n];
        const u64 k1 = evk[(((size_t)j * 2 + 1) * nfull + pz) * N + n];
        mac128(a0, e, k0);
        mac128(a1, e, k1);
    }
    acc[(size_t)z * N + n] = reduce128(a0.hi, a0.lo, pr);
    acc[((size_t)ne + z) * N + n] = reduce128(a1.hi, a1.lo, pr);
}

// ---------------------------------------------------------------------------
// Element-wise kernels
// ---------------------------------------------------------------------------
// Tensor product (Table I HMult): d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1.
__global__ void __launch_bounds__(256) k_tensor(const u64 *__restrict__ a, const u64 *__restrict__ b, int nl,
                                                u64 *__restrict__ d0, u64 *__restrict__ d1, u64 *__restrict__ d2,
                                                const PrimeInfo *__restrict__ P, int logN)
{
    pdl_enter();
    const int N = 1 << logN;
    const int i = blockIdx.y;
    const PrimeInfo pr = P[i];
    const size_t o = (size_t)i * N + (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t S = (size_t)nl * N;
    const u64 a0 = a[o], a1 = a[S + o], b0 = b[o], b1 = b[S + o];
    d0[o] = mul_mod(a0, b0, pr);
    U128 m = {0, 0};
    mac128(m, a0, b1);
    mac128(m, a1, b0);
    d1[o] = reduce128(m.hi, m.lo, pr);
    d2[o] = mul_mod(a1, b1, pr);
}

// Automorphism sigma_g in evaluation form (Sec. III-F1: a dependency within
// one limb): out[j] = in[brv(((2 brv(j) + 1) g mod 2N - 1) / 2)].
__global__ void __launch_bounds__(256) k_permute(const u64 *__restrict__ in, u64 *__restrict__ out,
                                                 int n_limbs, u64 g, int logN)
{
    pdl_enter();
    const int N = 1 << logN;
    const u32 j = blockIdx.x * blockDim.x + threadIdx.x;
    const u32 rj = __brev(j) >> (32 - logN);
    const u64 e = ((2 * (u64)rj + 1) * g) & (2 * (u64)N - 1);
    const u32 src = __brev((u32)((e - 1) >> 1)) >> (32 - logN);
    for (int z = 0; z < n_limbs; ++z) out[(size_t)z * N + j] = in[(size_t)z * N + src];
}

Seg seg_of(const u64 *src, u64 *dst, int count, int prime0, const u64 *aux = nullptr, u64 *out = nullptr,
           int src_step = 1, int mode = 0)
{
    Seg s;
    s.src = src; s.dst = dst; s.aux = aux; s.out = out;
    s.count = count; s.prime0 = prime0; s.src_step = src_step; s.mode = mode;
    return s;
}

void add_seg(LimbSet &S, const Seg &g)
{
    if (g.count <= 0) return;
    S.seg[S.nseg++] = g;
    S.total += g.count;
}

LimbSet empty_set()
{
    LimbSet S;
    memset(&S, 0, sizeof(S));
    return S;
}

// Scratch layout of one operation (words from ctx->scratch):
//   dsrc  [L]        materialised input of the key switch (d2 or sigma(c1))
//   coeff [L]        coefficient form of the key-switch input
//   ext   [beta][ne] ModUp output
//   acc   [2][ne]    inner-product accumulators
//   pc    [2][K]     coefficient form of the accumulators' special limbs
//   conv  [2][L]     base-converted P -> Q limbs (NTT intermediate)
//   last  [2]        Rescale: coefficient form of the dropped limb
struct Scratch {
    u64 *dsrc, *coeff, *ext, *acc, *pc, *conv, *last;
};

Scratch carve(const fides_ctx *c)
{
    const size_t N = c->N, L = c->L, K = c->K, ne = L + K;
    const size_t beta = (L + c->alpha - 1) / c->alpha;
    Scratch s;
    u64 *p = c->scratch;
    s.dsrc = p; p += L * N;
    s.coeff = p; p += L * N;
    s.ext = p; p += beta * ne * N;
    s.acc = p; p += 2 * ne * N;
    s.pc = p; p += 2 * K * N;
    s.conv = p; p += 2 * L * N;
    s.last = p;
    return s;
}

// ModUp of d (nl limbs, evaluation form) into ext [beta][nl+K][N].
int do_modup(const fides_ctx *c, const u64 *d, int nl, u64 *ext, const Scratch &s, cudaStream_t st)
{
    const int N = c->N, K = c->K, L = c->L, ne = nl + K, alpha = c->alpha;
    const int beta = (nl + alpha - 1) / alpha;
    int rc;
    // 1. coefficient form of d (canonical residues, as Eq. 1 requires)
    LimbSet in = empty_set();
    add_seg(in, seg_of(d, s.coeff, nl, 0));
    if ((rc = ntt_inverse(c, in, ProSrc{}, EpiCanon{}, st))) return rc;
    // 2. base conversion of every digit to its complement in Q_l and to P
    BConvArgs A;
    memset(&A, 0, sizeof(A));
    A.njob = beta;
    LimbSet out = empty_set();
    int max_src = 0;
    for (int j = 0; j < beta; ++j) {
        const int lo = j * alpha, hi = std::min(lo + alpha, nl);
        u64 *e = ext + (size_t)j * ne * N;
        BConvJob &B = A.job[j];
        B.src = s.coeff + (size_t)lo * N;
        B.n_src = hi - lo;
        B.src_prime0 = lo;
        const size_t off = ((size_t)(nl - 1) * c->dnum + j) * alpha;
        B.scale = c->d_mu_scale + off;
        B.mat = c->d_mu_mat + off * (L + K);
        B.ld = L + K;
        B.nrun = 0;
        if (lo > 0) B.run[B.nrun++] = BConvRun{e, lo, 0};
        if (hi < nl) B.run[B.nrun++] = BConvRun{e + (size_t)hi * N, nl - hi, hi};
        B.run[B.nrun++] = BConvRun{e + (size_t)nl * N, K, L};
        for (int r = 0; r < B.nrun; ++r) {
            u64 *p = B.run[r].dst;
            add_seg(out, seg_of(p, p, B.run[r].count, B.run[r].prime0));
        }
        max_src = std::max(max_src, hi - lo);
        // the digit's own limbs are the input limbs (evaluation form)
        rc = fides_check_cuda(cudaMemcpyAsync(e + (size_t)lo * N, d + (size_t)lo * N,
                                              sizeof(u64) * (size_t)(hi - lo) * N, cudaMemcpyDeviceToDevice, st),
                              "modup copy");
        if (rc) return rc;
    }
    if ((rc = launch_bconv(c, A, max_src, st))) return rc;
    // 3. new limbs to evaluation form
    return ntt_forward(c, out, ProSrc{}, EpiCanon{}, st);
}

// ModDown of npoly extended polynomials x_t ([nl+K][N] each) into out_t,
// mode_t = 0 store, 1 accumulate.
int do_moddown(const fides_ctx *c, int npoly, const u64 *const *x, int nl, u64 *const *outp, const int *mode,
               const Scratch &s, cudaStream_t st)
{
    const int N = c->N, K = c->K, L = c->L;
    int rc;
    LimbSet pin = empty_set();
    for (int t = 0; t < npoly; ++t) add_seg(pin, seg_of(x[t] + (size_t)nl * N, s.pc + (size_t)t * K * N, K, L));
    if ((rc = ntt_inverse(c, pin, ProSrc{}, EpiCanon{}, st))) return rc;
    BConvArgs A;
    memset(&A, 0, sizeof(A));
    A.njob = npoly;
    for (int t = 0; t < npoly; ++t) {
        BConvJob &B = A.job[t];
        B.src = s.pc + (size_t)t * K * N;
        B.n_src = K;
        B.src_prime0 = L;
        B.scale = c->d_md_scale;
        B.mat = c->d_md_mat;
        B.ld = L + K;
        B.nrun = 1;
        B.run[0] = BConvRun{s.conv + (size_t)t * L * N, nl, 0};
    }
    if ((rc = launch_bconv(c, A, K, st))) return rc;
    LimbSet fin = empty_set();
    for (int t = 0; t < npoly; ++t) {
        u64 *cv = s.conv + (size_t)t * L * N;
        add_seg(fin, seg_of(cv, cv, nl, 0, x[t], outp[t], 1, mode[t]));
    }
    return ntt_forward(c, fin, ProSrc{}, EpiSubMul{c->d_md_pinv}, st);
}

int do_keyswitch(const fides_ctx *c, const u64 *d, int nl, const u64 *evk, u64 *out0, u64 *out1, int mode0,
                 int mode1, const Scratch &s, cudaStream_t st)
{
    const int N = c->N, K = c->K, ne = nl + K;
    const int beta = (nl + c->alpha - 1) / c->alpha;
    int rc;
    if ((rc = do_modup(c, d, nl, s.ext, s, st))) return rc;
    dim3 grid(N / 256, ne);
    FIDES_LAUNCH("k_inner", st, k_inner, grid, dim3(256), (const u64 *)s.ext, beta, nl, ne, evk, c->L, c->L + K, s.acc,
                 (const PrimeInfo *)c->d_prime, c->logN);
    if ((rc = fides_check_cuda(cudaGetLastError(), "inner product launch"))) return rc;
    const u64 *xs[2] = {s.acc, s.acc + (size_t)ne * N};
    u64 *outs[2] = {out0, out1};
    int modes[2] = {mode0, mode1};
    return do_moddown(c, 2, xs, nl, outs, modes, s, st);
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
    return do_modup(c, d, nl, ext, carve(c), as_stream(stream));
}

extern "C" int fides_moddown(fides_ctx *c, const uint64_t *x, int nl, uint64_t *out, void *stream)
{
    if (int rc = check_ctx(c, "fides_moddown")) return rc;
    if (int rc = check_level(c, nl, "fides_moddown")) return rc;
    if (!x || !out) return fides_set_error(FIDES_ERR_ARG, "fides_moddown: NULL buffer");
    const u64 *xs[1] = {x};
    u64 *outs[1] = {out};
    int modes[1] = {0};
    return do_moddown(c, 1, xs, nl, outs, modes, carve(c), as_stream(stream));
}

extern "C" int fides_keyswitch(fides_ctx *c, const uint64_t *d, int nl, const uint64_t *evk, uint64_t *out0,
                               uint64_t *out1, void *stream)
{
    if (int rc = check_ctx(c, "fides_keyswitch")) return rc;
    if (int rc = check_level(c, nl, "fides_keyswitch")) return rc;
    if (!d || !evk || !out0 || !out1) return fides_set_error(FIDES_ERR_ARG, "fides_keyswitch: NULL buffer");
    OpTrace op("op_keyswitch", as_stream(stream));
    return do_keyswitch(c, d, nl, evk, out0, out1, 0, 0, carve(c), as_stream(stream));
}

extern "C" int fides_hmult(fides_ctx *c, const fides_ct *a, const fides_ct *b, const uint64_t *rlk, fides_ct *out,
                           void *stream)
{
    if (int rc = check_ctx(c, "fides_hmult")) return rc;
    if (!a || !b || !out || !rlk || !a->data || !b->data || !out->data)
        return fides_set_error(FIDES_ERR_ARG, "fides_hmult: NULL argument");
    const int nl = a->n_limbs;
    if (int rc = check_level(c, nl, "fides_hmult")) return rc;
    if (b->n_limbs != nl || out->n_limbs != nl)
        return fides_set_error(FIDES_ERR_ARG, "fides_hmult: level mismatch (%d, %d, %d)", nl, b->n_limbs,
                               out->n_limbs);
    const size_t S = (size_t)nl * c->N;
    cudaStream_t st = as_stream(stream);
    OpTrace op("op_hmult", st);
    Scratch s = carve(c);
    FIDES_LAUNCH("k_tensor", st, k_tensor, dim3(c->N / 256, nl), dim3(256), (const u64 *)a->data, (const u64 *)b->data, nl,
                 out->data, out->data + S, s.dsrc, (const PrimeInfo *)c->d_prime, c->logN);
    if (int rc = fides_check_cuda(cudaGetLastError(), "tensor launch")) return rc;
    int rc = do_keyswitch(c, s.dsrc, nl, rlk, out->data, out->data + S, 1, 1, s, st);
    if (!rc) out->scale = a->scale * b->scale;
    return rc;
}

extern "C" int fides_rotate(fides_ctx *c, const fides_ct *a, int64_t steps, const uint64_t *rk, fides_ct *out,
                            void *stream)
{
    if (int rc = check_ctx(c, "fides_rotate")) return rc;
    if (!a || !out || !rk || !a->data || !out->data) return fides_set_error(FIDES_ERR_ARG, "fides_rotate: NULL argument");
    const int nl = a->n_limbs;
    if (int rc = check_level(c, nl, "fides_rotate")) return rc;
    if (out->n_limbs != nl) return fides_set_error(FIDES_ERR_ARG, "fides_rotate: level mismatch");
    const size_t S = (size_t)nl * c->N;
    cudaStream_t st = as_stream(stream);
    OpTrace op("op_rotate", st);
    Scratch s = carve(c);
    const u64 g = fides_galois_elt(c, steps);
    FIDES_LAUNCH("k_permute", st, k_permute, dim3(c->N / 256), dim3(256), (const u64 *)a->data, out->data, nl, g, c->logN);
    FIDES_LAUNCH("k_permute", st, k_permute, dim3(c->N / 256), dim3(256), (const u64 *)(a->data + S), s.dsrc, nl, g,
                 c->logN);
    if (int rc = fides_check_cuda(cudaGetLastError(), "permute launch")) return rc;
    int rc = do_keyswitch(c, s.dsrc, nl, rk, out->data, out->data + S, 1, 0, s, st);
    if (!rc) out->scale = a->scale;
    return rc;
}

extern "C" int fides_rescale(fides_ctx *c, const fides_ct *a, fides_ct *out, void *stream)
{
    if (int rc = check_ctx(c, "fides_rescale")) return rc;
    if (!a || !out || !a->data || !out->data) return fides_set_error(FIDES_ERR_ARG, "fides_rescale: NULL argument");
    const int nl = a->n_limbs;
    if (int rc = check_level(c, nl, "fides_rescale")) return rc;
    if (nl < 2 || out->n_limbs != nl - 1)
        return fides_set_error(FIDES_ERR_ARG, "fides_rescale: needs n_limbs >= 2 and out->n_limbs = n_limbs - 1");
    const int l = nl - 1;
    const size_t N = c->N, Sin = (size_t)nl * N, Sout = (size_t)l * N;
    cudaStream_t st = as_stream(stream);
    OpTrace op("op_rescale", st);
    Scratch s = carve(c);
    int rc;
    LimbSet last = empty_set();
    for (int t = 0; t < 2; ++t) add_seg(last, seg_of(a->data + t * Sin + (size_t)l * N, s.last + t * N, 1, l));
    if ((rc = ntt_inverse(c, last, ProSrc{}, EpiCanon{}, st))) return rc;
    LimbSet fin = empty_set();
    for (int t = 0; t < 2; ++t)
        add_seg(fin, seg_of(s.last + t * N, out->data + t * Sout, l, 0, a->data + t * Sin, out->data + t * Sout, 0, 0));
    rc = ntt_forward(c, fin, ProSwitchMod{}, EpiSubMul{c->d_rs_qlinv + (size_t)l * c->L}, st);
    if (!rc) out->scale = a->scale / (double)c->primes[l];
    return rc;
}
