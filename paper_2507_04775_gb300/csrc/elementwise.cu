// Element-wise CKKS operations (Table I): HAdd, HSub, PtAdd, PtMult,
// ScalarAdd and ScalarMult on ciphertexts in evaluation form, where a
// polynomial product is the slot-wise product of evaluations and a constant
// polynomial evaluates to itself everywhere.
//
// One kernel covers all six: a grid-stride loop over both polynomials of the
// ciphertext, two words per thread per step with 16-byte loads and stores
// (8-byte ones when a buffer is not 16-byte aligned).  The work is bound by
// HBM: per word it reads one or two operands and writes one result.
#include <algorithm>
#include <cstring>

#include "fides_internal.cuh"

namespace {

enum ElemOp { E_HADD, E_HSUB, E_PTADD, E_PTMULT, E_SCALAR_ADD, E_SCALAR_MULT, E_MULI };

struct ElemArgs {
    const u64 *a;     // [2][nl][N]
    const u64 *b;     // HADD / HSUB: [2][nl][N]; PTADD / PTMULT: [nl][N]
    u64 *out;         // [2][nl][N] (may alias a or b: each word is read and written by one thread)
    int nl, logN;
    int neg;                      // E_MULI: 0 multiplies by X^(N/2) (slots by i), 1 by X^(3N/2) (slots by -i)
    TwPair k[FIDES_MAX_PRIMES];   // scalar ops: residue of the constant per limb, with its Shoup companion;
                                  // E_MULI: i_q = psi^(N/2) mod q_i
};

template <int OP>
__device__ __forceinline__ u64 elem(u64 x, u64 y, int poly, const TwPair &k, const PrimeInfo &p)
{
    switch (OP) {
    case E_HADD: return csub(x + y, p.q);
    case E_HSUB: return csub(x + p.q - y, p.q);
    case E_PTADD: return poly == 0 ? csub(x + y, p.q) : x;
    case E_PTMULT: return mul_mod_small(x, y, p);
    case E_SCALAR_ADD: return poly == 0 ? csub(x + k.w, p.q) : x;
    default: return csub(mul_shoup(x, k, p.q), p.q);   // E_SCALAR_MULT, E_MULI
    }
}

template <bool VEC>
__device__ __forceinline__ void load2(const u64 *p, u64 &x0, u64 &x1)
{
    if (VEC) {
        const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(p);
        x0 = v.x; x1 = v.y;
    } else {
        x0 = p[0]; x1 = p[1];
    }
}

template <bool VEC>
__device__ __forceinline__ void store2(u64 *p, u64 x0, u64 x1)
{
    if (VEC) {
        *reinterpret_cast<ulonglong2 *>(p) = make_ulonglong2(x0, x1);
    } else {
        p[0] = x0; p[1] = x1;
    }
}

// Each thread step handles two consecutive words at the same position of both
// polynomials, so a plaintext operand is read once for both.
template <int OP, bool VEC>
__global__ void __launch_bounds__(256) k_elem(ElemArgs A, const PrimeInfo *__restrict__ P)
{
    pdl_enter();
    const size_t S = (size_t)A.nl << A.logN;     // words of one polynomial
    const bool two_b = OP == E_HADD || OP == E_HSUB;
    const bool pt_b = OP == E_PTADD || OP == E_PTMULT;
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < S / 2; v += (size_t)gridDim.x * blockDim.x) {
        const size_t wi = 2 * v;
        const int z = (int)(wi >> A.logN);
        const PrimeInfo p = P[z];
        const TwPair k = (OP == E_SCALAR_ADD || OP == E_SCALAR_MULT || OP == E_MULI) ? A.k[z] : TwPair{0, 0};
        u64 x[4], y[4] = {0, 0, 0, 0};
        load2<VEC>(A.a + wi, x[0], x[1]);
        load2<VEC>(A.a + S + wi, x[2], x[3]);
        if (two_b) {
            load2<VEC>(A.b + wi, y[0], y[1]);
            load2<VEC>(A.b + S + wi, y[2], y[3]);
        } else if (pt_b) {
            load2<VEC>(A.b + wi, y[0], y[1]);
            y[2] = y[0];
            y[3] = y[1];
        }
        u64 r[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) r[i] = elem<OP>(x[i], y[i], i >> 1, k, p);
        if (OP == E_MULI) {
            // X^(N/2) at the point psi^(2 brv(j) + 1) is i_q^(2 brv(j) + 1) = i_q (-1)^brv(j), and brv(j)
            // is odd exactly in the upper half of the limb
            if ((int)((wi >> (A.logN - 1)) & 1) != A.neg) {
#pragma unroll
                for (int i = 0; i < 4; ++i) r[i] = r[i] ? p.q - r[i] : 0;
            }
        }
        store2<VEC>(A.out + wi, r[0], r[1]);
        store2<VEC>(A.out + S + wi, r[2], r[3]);
    }
}

template <int OP>
int launch_elem(const fides_ctx *c, const ElemArgs &A, cudaStream_t st)
{
    const size_t pairs = ((size_t)A.nl << A.logN) / 2;
    const size_t want = (pairs + 255) / 256;
    const unsigned blocks = (unsigned)std::min<size_t>(want, (size_t)c->sms * 8);
    const bool vec = (((uintptr_t)A.a | (uintptr_t)A.b | (uintptr_t)A.out) & 15) == 0;
    if (vec) FIDES_LAUNCH("k_elem", st, (k_elem<OP, true>), dim3(blocks), dim3(256), A, (const PrimeInfo *)c->d_prime);
    else FIDES_LAUNCH("k_elem", st, (k_elem<OP, false>), dim3(blocks), dim3(256), A, (const PrimeInfo *)c->d_prime);
    return fides_check_cuda(cudaGetLastError(), "element-wise launch");
}

int run_elem(fides_ctx *c, int op, const fides_ct *a, const uint64_t *b, const uint64_t *k, fides_ct *out,
             double out_scale, void *stream, const char *fn, int neg = 0)
{
    if (!c || !a || !out || !a->data || !out->data) return fides_set_error(FIDES_ERR_ARG, "%s: NULL argument", fn);
    const int nl = a->n_limbs;
    if (nl < 1 || nl > c->L) return fides_set_error(FIDES_ERR_ARG, "%s: n_limbs=%d outside [1, %d]", fn, nl, c->L);
    if (out->n_limbs != nl) return fides_set_error(FIDES_ERR_ARG, "%s: out->n_limbs must equal a->n_limbs", fn);
    ElemArgs A;
    memset(&A, 0, sizeof(A));
    A.a = a->data;
    A.b = b;
    A.out = out->data;
    A.nl = nl;
    A.logN = c->logN;
    if (op == E_SCALAR_ADD || op == E_SCALAR_MULT) {
        if (!k) return fides_set_error(FIDES_ERR_ARG, "%s: constant is NULL", fn);
        for (int i = 0; i < nl; ++i) {
            const u64 q = c->primes[i];
            if (k[i] >= q) return fides_set_error(FIDES_ERR_ARG, "%s: constant residue %d not below q_%d", fn, i, i);
            A.k[i].w = k[i];
            A.k[i].wp = (u64)(((unsigned __int128)k[i] << 64) / q);
        }
    } else if (op == E_MULI) {
        for (int i = 0; i < nl; ++i) A.k[i] = c->iroot[i];
        A.neg = neg;
    } else if (!b) {
        return fides_set_error(FIDES_ERR_ARG, "%s: second operand is NULL", fn);
    }
    cudaStream_t st = (cudaStream_t)stream;
    OpTrace tr(fn, st);
    int rc;
    switch (op) {
    case E_HADD: rc = launch_elem<E_HADD>(c, A, st); break;
    case E_HSUB: rc = launch_elem<E_HSUB>(c, A, st); break;
    case E_PTADD: rc = launch_elem<E_PTADD>(c, A, st); break;
    case E_PTMULT: rc = launch_elem<E_PTMULT>(c, A, st); break;
    case E_SCALAR_ADD: rc = launch_elem<E_SCALAR_ADD>(c, A, st); break;
    case E_MULI: rc = launch_elem<E_MULI>(c, A, st); break;
    default: rc = launch_elem<E_SCALAR_MULT>(c, A, st); break;
    }
    if (!rc) out->scale = out_scale;
    return rc;
}

int check_b(const fides_ct *a, const fides_ct *b, const char *fn)
{
    if (!b || !b->data) return fides_set_error(FIDES_ERR_ARG, "%s: b is NULL", fn);
    if (a && b->n_limbs != a->n_limbs) return fides_set_error(FIDES_ERR_ARG, "%s: a and b at different levels", fn);
    return FIDES_OK;
}

}  // namespace

extern "C" int fides_hadd(fides_ctx *c, const fides_ct *a, const fides_ct *b, fides_ct *out, void *stream)
{
    if (int rc = check_b(a, b, "fides_hadd")) return rc;
    return run_elem(c, E_HADD, a, b->data, nullptr, out, a ? a->scale : 0.0, stream, "op_hadd");
}

extern "C" int fides_hsub(fides_ctx *c, const fides_ct *a, const fides_ct *b, fides_ct *out, void *stream)
{
    if (int rc = check_b(a, b, "fides_hsub")) return rc;
    return run_elem(c, E_HSUB, a, b->data, nullptr, out, a ? a->scale : 0.0, stream, "op_hsub");
}

extern "C" int fides_ptadd(fides_ctx *c, const fides_ct *a, const uint64_t *pt, fides_ct *out, void *stream)
{
    return run_elem(c, E_PTADD, a, pt, nullptr, out, a ? a->scale : 0.0, stream, "op_ptadd");
}

extern "C" int fides_ptmult(fides_ctx *c, const fides_ct *a, const uint64_t *pt, double pt_scale, fides_ct *out,
                            void *stream)
{
    return run_elem(c, E_PTMULT, a, pt, nullptr, out, a ? a->scale * pt_scale : 0.0, stream, "op_ptmult");
}

extern "C" int fides_scalar_add(fides_ctx *c, const fides_ct *a, const uint64_t *k, fides_ct *out, void *stream)
{
    return run_elem(c, E_SCALAR_ADD, a, nullptr, k, out, a ? a->scale : 0.0, stream, "op_scalar_add");
}

extern "C" int fides_scalar_mult(fides_ctx *c, const fides_ct *a, const uint64_t *k, double k_scale, fides_ct *out,
                                 void *stream)
{
    return run_elem(c, E_SCALAR_MULT, a, nullptr, k, out, a ? a->scale * k_scale : 0.0, stream, "op_scalar_mult");
}

extern "C" int fides_mul_i(fides_ctx *c, const fides_ct *a, int sign, fides_ct *out, void *stream)
{
    if (sign != 1 && sign != -1) return fides_set_error(FIDES_ERR_ARG, "fides_mul_i: sign must be +1 or -1");
    return run_elem(c, E_MULI, a, nullptr, nullptr, out, a ? a->scale : 0.0, stream, "op_mul_i", sign < 0 ? 1 : 0);
}

// ---------------------------------------------------------------------------
// Plaintext multiply-accumulate: out = sum_t ct_t (.) pt_t (+ out), the inner
// sum of a baby-step giant-step linear transform, with one 128-bit
// accumulator per word and one reduction at the end.
// ---------------------------------------------------------------------------
namespace {

struct MacArgs {
    const u64 *ct[FIDES_MAC_TERMS];   // [2][nl][N] each
    const u64 *pt[FIDES_MAC_TERMS];   // [nl][N] each
    u64 *out;                         // [2][nl][N]
    int nt, nl, logN, accumulate;
};

template <bool VEC>
__global__ void __launch_bounds__(256) k_ptmac(MacArgs A, const PrimeInfo *__restrict__ P)
{
    pdl_enter();
    const size_t S = (size_t)A.nl << A.logN;
    // two consecutive words at the same position of both polynomials per
    // step: each plaintext word is read once
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < S / 2; v += (size_t)gridDim.x * blockDim.x) {
        const size_t wi = 2 * v;
        const PrimeInfo p = P[(int)(wi >> A.logN)];
        U128 s[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
        if (A.accumulate) {
            load2<VEC>(A.out + wi, s[0].lo, s[1].lo);
            load2<VEC>(A.out + S + wi, s[2].lo, s[3].lo);
        }
#pragma unroll 2
        for (int t = 0; t < A.nt; ++t) {
            u64 x[4], y0, y1;
            load2<VEC>(A.ct[t] + wi, x[0], x[1]);
            load2<VEC>(A.ct[t] + S + wi, x[2], x[3]);
            load2<VEC>(A.pt[t] + wi, y0, y1);
            mac128(s[0], x[0], y0);
            mac128(s[1], x[1], y1);
            mac128(s[2], x[2], y0);
            mac128(s[3], x[3], y1);
        }
        store2<VEC>(A.out + wi, reduce128(s[0].hi, s[0].lo, p), reduce128(s[1].hi, s[1].lo, p));
        store2<VEC>(A.out + S + wi, reduce128(s[2].hi, s[2].lo, p), reduce128(s[3].hi, s[3].lo, p));
    }
}

}  // namespace

int launch_ptmac(const fides_ctx *c, const u64 *const *cts, const u64 *const *pts, int nt, u64 *out, int nl,
                 bool accumulate, cudaStream_t st)
{
    for (int t0 = 0; t0 < nt; t0 += FIDES_MAC_TERMS) {
        MacArgs A;
        memset(&A, 0, sizeof(A));
        A.nt = std::min(FIDES_MAC_TERMS, nt - t0);
        uintptr_t align = (uintptr_t)out;
        for (int t = 0; t < A.nt; ++t) {
            A.ct[t] = cts[t0 + t];
            A.pt[t] = pts[t0 + t];
            align |= (uintptr_t)A.ct[t] | (uintptr_t)A.pt[t];
        }
        A.out = out;
        A.nl = nl;
        A.logN = c->logN;
        A.accumulate = (accumulate || t0 > 0) ? 1 : 0;
        const size_t pairs = ((size_t)nl << c->logN) / 2;
        const unsigned blocks = (unsigned)std::min<size_t>((pairs + 255) / 256, (size_t)c->sms * 8);
        if ((align & 15) == 0)
            FIDES_LAUNCH("k_ptmac", st, k_ptmac<true>, dim3(blocks), dim3(256), A, (const PrimeInfo *)c->d_prime);
        else
            FIDES_LAUNCH("k_ptmac", st, k_ptmac<false>, dim3(blocks), dim3(256), A, (const PrimeInfo *)c->d_prime);
        if (int rc = fides_check_cuda(cudaGetLastError(), "plaintext multiply-accumulate launch")) return rc;
    }
    return FIDES_OK;
}

// ---------------------------------------------------------------------------
// Multiply-accumulate of ciphertexts by scalar constants:
//   out = sum_t k_t (.) x_t   at nl limbs,
// where x_t may have more limbs than nl (its first nl limbs of each polynomial
// are read in place, with its own polynomial stride) and k_t is row cidx[t]
// of a device table of per-limb residues.  One 128-bit accumulator per word,
// one reduction.
// ---------------------------------------------------------------------------
namespace {

struct CmacArgs {
    const u64 *x[FIDES_MAC_TERMS];
    int xl[FIDES_MAC_TERMS];        // limbs of x_t (its polynomial stride in limbs)
    int cidx[FIDES_MAC_TERMS];      // row of k_t in the constant table
    const u64 *k;                   // [rows][kld] residues
    int kld;
    u64 *out;                       // [2][nl][N]
    int nt, nl, logN;
};

template <bool VEC>
__global__ void __launch_bounds__(256) k_cmac(const CmacArgs A, const PrimeInfo *__restrict__ P)
{
    pdl_enter();
    const size_t S = (size_t)A.nl << A.logN;
    // two words per thread and step (both in one limb: N is even)
    for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < S; v += (size_t)gridDim.x * blockDim.x) {
        const size_t w = 2 * v;
        const int poly = w >= S;
        const size_t wi = w - (poly ? S : 0);
        const int z = (int)(wi >> A.logN);
        const PrimeInfo p = P[z];
        U128 s0 = {0, 0}, s1 = {0, 0};
#pragma unroll 4
        for (int t = 0; t < A.nt; ++t) {
            const u64 *src = A.x[t] + (poly ? ((size_t)A.xl[t] << A.logN) + wi : wi);
            const u64 k = __ldg(A.k + (size_t)A.cidx[t] * A.kld + z);
            u64 x0, x1;
            if (VEC) {
                const ulonglong2 xv = *reinterpret_cast<const ulonglong2 *>(src);
                x0 = xv.x; x1 = xv.y;
            } else {
                x0 = src[0]; x1 = src[1];
            }
            mac128(s0, x0, k);
            mac128(s1, x1, k);
        }
        const u64 r0 = reduce128(s0.hi, s0.lo, p), r1 = reduce128(s1.hi, s1.lo, p);
        if (VEC) {
            *reinterpret_cast<ulonglong2 *>(A.out + w) = make_ulonglong2(r0, r1);
        } else {
            A.out[w] = r0;
            A.out[w + 1] = r1;
        }
    }
}

}  // namespace

int launch_cmac(const fides_ctx *c, const u64 *const *x, const int *xl, const int *cidx, int nt, const u64 *k,
                int kld, u64 *out, int nl, cudaStream_t st)
{
    if (nt < 1 || nt > FIDES_MAC_TERMS)
        return fides_set_error(FIDES_ERR_ARG, "constant multiply-accumulate: %d terms outside [1, %d]", nt,
                               FIDES_MAC_TERMS);
    CmacArgs A;
    memset(&A, 0, sizeof(A));
    for (int t = 0; t < nt; ++t) {
        A.x[t] = x[t];
        A.xl[t] = xl[t];
        A.cidx[t] = cidx[t];
    }
    A.k = k;
    A.kld = kld;
    A.out = out;
    A.nt = nt;
    A.nl = nl;
    A.logN = c->logN;
    const size_t pairs = (size_t)nl << c->logN;
    const unsigned blocks = (unsigned)std::min<size_t>((pairs + 255) / 256, (size_t)c->sms * 8);
    uintptr_t align = (uintptr_t)out;
    for (int t = 0; t < nt; ++t) align |= (uintptr_t)x[t];
    if ((align & 15) == 0)
        FIDES_LAUNCH("k_cmac", st, k_cmac<true>, dim3(blocks), dim3(256), A, (const PrimeInfo *)c->d_prime);
    else
        FIDES_LAUNCH("k_cmac", st, k_cmac<false>, dim3(blocks), dim3(256), A, (const PrimeInfo *)c->d_prime);
    return fides_check_cuda(cudaGetLastError(), "constant multiply-accumulate launch");
}
