// Key-switching kernels shared by the single-operation path (keyswitch.cu)
// and the batched path (batch.cu): fast base conversion (Sec. III-F3, Eq. 1),
// and the key inner product (Sec. III-F5 "Dot product fusion").  Every kernel
// reads its work descriptors
// either inline from its parameters (one operation) or from a device-resident
// table built once for a batch.
#pragma once

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
    int prescaled;           // 1: the sources already hold [x_i qhat_i^-1]_{q_i}
    int src_prime0;
    const TwPair *scale;     // [n_src] qhat_i^-1 mod q_i
    const u64 *mat;          // [n_src][ld]: [qhat_i]_{prime z}
    int ld;
    int nrun;
    BConvRun run[3];
    const void *tc;          // tensor-core image of the conversion matrix (bconv_tc.cuh), or null
    int tc_corr;             // the image has the correction block (ModDown images)
    int centred;             // convert the centred residues: add c * corr[z], c = #{i: x_i > (q_i - 1) / 2}
    const u64 *corr;         // [prime z] the correction constant, -Q_src mod prime z (centred jobs)
};

// Jobs inline (djob == nullptr) or in device memory (djob[0..njob)).
struct BConvArgs {
    int njob;
    int tc;                  // 1: every job has a tensor-core image (k_bconv_tc)
    int tc_smem;             // k_bconv_tc: dynamic shared memory of the largest job (bconv_tc_smem)
    const BConvJob *djob;
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

// the same for a sum of at most two products of canonical residues
__device__ __forceinline__ u64 reduce_acc2(const Acc128 &c, const PrimeInfo &p)
{
    return csub(csub(reduce_prod(((u64)c.w3 << 32) | c.w2, ((u64)c.w1 << 32) | c.w0, p), p.q2), p.q);
}

// The same for a sum of m products of canonical residues: the Barrett form
// where its bound holds, m q^2 < 2^(k+63) for m at most 2^(63-k) (k the bit
// length of q: m <= 4 at 61-bit primes, 8 at 60-bit), reduce128 otherwise.
__device__ __forceinline__ bool reduce_prod_ok(int m, const PrimeInfo &p)
{
    return (u64)m <= (1ull << (__clzll((long long)p.q) - 1));   // 2^(63-k), k = 64 - clz(q)
}
__device__ __forceinline__ u64 reduce_accm(const Acc128 &c, const PrimeInfo &p, bool barrett)
{
    const u64 hi = ((u64)c.w3 << 32) | c.w2, lo = ((u64)c.w1 << 32) | c.w0;
    return barrett ? csub(csub(reduce_prod(hi, lo, p), p.q2), p.q) : reduce128(hi, lo, p);
}

template <int NS>
__device__ __forceinline__ void bconv_body(const BConvJob &B, const PrimeInfo *__restrict__ P, int logN, int tg)
{
    constexpr int MS = NS > 0 ? NS : FIDES_MAX_SRC;
    __shared__ u64 smat[BCONV_TG * MS];
    __shared__ PrimeInfo sp[BCONV_TG];
    __shared__ u64 *sdst[BCONV_TG];
    __shared__ u64 scorr[BCONV_TG];
    const int N = 1 << logN;
    const int ns = NS > 0 ? NS : B.n_src;

    int ndst = 0;
    for (int r = 0; r < B.nrun; ++r) ndst += B.run[r].count;
    const int d0 = blockIdx.z * tg;
    const int nd = min(tg, ndst - d0);
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
        scorr[threadIdx.x] = B.centred ? B.corr[pz] : 0;
        for (int i = 0; i < ns; ++i) smat[threadIdx.x * MS + i] = B.mat[(size_t)i * B.ld + pz];
    }
    __syncthreads();

    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const u64 *src = B.src;
    u64 v[MS];
#pragma unroll
    for (int i = 0; i < MS; ++i) {
        if (NS > 0 || i < ns) {
            const u64 x = src[(size_t)i * N + n];
            if (B.prescaled) {
                v[i] = x;
            } else {
                const u64 qi = P[B.src_prime0 + i].q;
                v[i] = csub(mul_shoup(x, B.scale[i], qi), qi);
            }
        } else {
            v[i] = 0;
        }
    }
    // centred conversion: the residues in the upper half stand for v - q_i,
    // which adds (their count) x (-Q_src) to every target
    u64 cnt = 0;
    if (B.centred) {
#pragma unroll
        for (int i = 0; i < MS; ++i)
            if (NS > 0 || i < ns) cnt += v[i] > (P[B.src_prime0 + i].q >> 1) ? 1 : 0;
    }
    int d = 0;
    for (; d + 1 < nd; d += 2) {
        Acc128 c0 = {0, 0, 0, 0}, c1 = {0, 0, 0, 0};
        if (cnt) {
            mac_wide(c0, cnt, scorr[d]);
            mac_wide(c1, cnt, scorr[d + 1]);
        }
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
        if (cnt) mac_wide(c0, cnt, scorr[d]);
        const u64 *m0 = smat + d * MS;
#pragma unroll
        for (int i = 0; i < MS; ++i)
            if (NS > 0 || i < ns) mac_wide(c0, v[i], m0[i]);
        sdst[d][n] = reduce_acc(c0, sp[d]);
    }
}

template <int NS>
__global__ void __launch_bounds__(256) k_bconv(BConvArgs A, const PrimeInfo *__restrict__ P, int logN, int tg)
{
    pdl_enter();
    if (A.djob) bconv_body<NS>(A.djob[blockIdx.y], P, logN, tg);
    else bconv_body<NS>(A.job[blockIdx.y], P, logN, tg);
}

// Targets per CTA: the group size minimising (waves of CTAs) x (per-CTA time),
// with a CTA's time modelled as tg + 4 target-equivalents (the scaling of the
// sources and the loads are paid once per CTA) and 4 resident CTAs per SM.
inline int bconv_group(const fides_ctx *c, int njob, int max_dst)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const long slots = 4L * sms, cols = (long)(c->N / 256) * njob;
    int best = BCONV_TG;
    long best_cost = -1;
    for (int tg = BCONV_TG; tg >= 1; --tg) {
        const long ctas = cols * ((max_dst + tg - 1) / tg);
        const long cost = ((ctas + slots - 1) / slots) * (tg + 4);
        if (best_cost < 0 || cost < best_cost) { best_cost = cost; best = tg; }
    }
    return best;
}

template <int NS>
void launch_bconv_ns(const fides_ctx *c, const BConvArgs &A, int max_dst, cudaStream_t st)
{
    const int tg = bconv_group(c, A.njob, max_dst);
    dim3 grid(c->N / 256, A.njob, (max_dst + tg - 1) / tg), block(256);
    FIDES_LAUNCH("k_bconv", st, k_bconv<NS>, grid, block, A, c->d_prime, c->logN, tg);
}

}  // namespace

#include "bconv_tc.cuh"

namespace {

// One launch for jobs that all have `ns` source limbs (inline or device jobs);
// tensor-core jobs (G.tc) may mix source counts up to ns.
inline int launch_bconv_group(const fides_ctx *c, const BConvArgs &G, int ns, int max_dst, cudaStream_t st)
{
    if (G.tc) return launch_bconv_tc(c, G, ns, max_dst, st);
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
    return fides_check_cuda(cudaGetLastError(), "bconv launch");
}

inline int bconv_targets(const BConvJob &j)
{
    int nd = 0;
    for (int r = 0; r < j.nrun; ++r) nd += j.run[r].count;
    return nd;
}

// Launch group of a job: every job with a tensor-core image goes to one
// k_bconv_tc launch (-1); the integer kernel gets one launch per distinct
// source count (a ragged last digit gets its own, so every launch runs fully
// unrolled loops).
// (The tensor-core kernel copies its sources in with bulk copies, which need
// 16-byte alignment; a job whose sources lack it goes to the integer kernel.)
inline int bconv_group_key(const BConvJob &j)
{
    return j.tc && ((uintptr_t)j.src & 15) == 0 ? -1 : j.n_src;
}

inline int launch_bconv(const fides_ctx *c, const BConvArgs &A, cudaStream_t st)
{
    if (A.njob == 0) return FIDES_OK;
    bool done[FIDES_MAX_DIGITS] = {false};
    for (int j = 0; j < A.njob; ++j) {
        if (done[j]) continue;
        const int key = bconv_group_key(A.job[j]);
        BConvArgs G;
        memset(&G, 0, sizeof(G));
        G.tc = key < 0;
        int max_dst = 0, ns = 0;
        for (int k = j; k < A.njob; ++k) {
            if (done[k] || bconv_group_key(A.job[k]) != key) continue;
            done[k] = true;
            G.job[G.njob++] = A.job[k];
            max_dst = std::max(max_dst, bconv_targets(A.job[k]));
            ns = std::max(ns, A.job[k].n_src);
        }
        if (G.tc)
            for (int k = 0; k < G.njob; ++k) G.tc_smem = std::max(G.tc_smem, bconv_tc_smem(G.job[k]));
        if (int rc = launch_bconv_group(c, G, ns, max_dst, st)) return rc;
    }
    return FIDES_OK;
}

// ---------------------------------------------------------------------------
// Key inner product: acc_t[z] = sum_j d~_j[z] * evk_{j,t}[key limb of z],
// t = 0, 1, over the nl q-limbs and the K special limbs; 128-bit lazy sums.
// d~_j[z] is the ModUp output ext_j[z], except on the limbs of digit j itself,
// where it is the key-switch input d[z] (read from dsrc, no copy is made).
// ---------------------------------------------------------------------------
struct IPOp {
    const u64 *ext;     // [beta][ne][N]
    const u64 *dsrc;    // [nl][N] evaluation-form input
    const u64 *evk;     // [dnum][2][L+K][N]
    u64 *acc;           // [2][ne][N]
    int nl, ne, beta, alpha;
    u64 g;              // 0, or the Galois element through which the digits are read (hoisted rotation)
};

// One op inline (dop == nullptr; grid.y = its ne limbs) or a device table of
// ops with a row table: row r (grid.y) computes limb drow[r] & 127 of op
// drow[r] >> 7 (an op has at most FIDES_MAX_PRIMES limbs).  The batched path orders the rows by key and key limb, so
// that the ops sharing a key (every HMult of a batch shares the
// relinearisation key) read each key limb while it is in L2.
struct IPArgs {
    const IPOp *dop;
    const int *drow;
    int nop;
    IPOp one;
};

// V2: two consecutive coefficients per thread with 16-byte loads and stores
// (only without an automorphism and with 16-byte-aligned buffers).
template <int MAXB, bool V2>
__device__ __forceinline__ void inner_body(const IPOp &op, int z, int L, int nfull, const PrimeInfo *__restrict__ P,
                                           int logN)
{
    const int N = 1 << logN;
    const int nl = op.nl, ne = op.ne, beta = op.beta;
    const int pz = z < nl ? z : L + (z - nl);
    const int own = z < nl ? z / op.alpha : -1;
    const PrimeInfo pr = P[pz];
    const size_t n = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * (V2 ? 2 : 1);
    const u64 *ext = op.ext;     // written by the kernels before this one: coherent loads
    const u64 *__restrict__ evk = op.evk;
    const u64 *dsrc = op.dsrc;
    u64 *acc = op.acc;
    if (V2) {
        // issue every load before the first product (the kernel is bound by
        // HBM); the keys, which no kernel writes, before the wait for the
        // previous kernel, so that they stream during its last wave
        ulonglong2 e[MAXB], k0[MAXB], k1[MAXB];
#pragma unroll
        for (int j = 0; j < MAXB; ++j) {
            if (j < beta) {
                k0[j] = *reinterpret_cast<const ulonglong2 *>(evk + (((size_t)j * 2 + 0) * nfull + pz) * N + n);
                k1[j] = *reinterpret_cast<const ulonglong2 *>(evk + (((size_t)j * 2 + 1) * nfull + pz) * N + n);
            }
        }
        pdl_wait();
#pragma unroll
        for (int j = 0; j < MAXB; ++j) {
            if (j < beta) {
                const u64 *src = (j == own) ? dsrc + (size_t)z * N : ext + ((size_t)j * ne + z) * N;
                e[j] = *reinterpret_cast<const ulonglong2 *>(src + n);
            }
        }
        // 128-bit sums as 32-bit carry chains (each product < 2^122, at most
        // FIDES_MAX_DIGITS of them)
        Acc128 a0 = {0, 0, 0, 0}, a1 = {0, 0, 0, 0}, b0 = {0, 0, 0, 0}, b1 = {0, 0, 0, 0};
#pragma unroll
        for (int j = 0; j < MAXB; ++j) {
            if (j < beta) {
                mac_wide(a0, e[j].x, k0[j].x);
                mac_wide(b0, e[j].y, k0[j].y);
                mac_wide(a1, e[j].x, k1[j].x);
                mac_wide(b1, e[j].y, k1[j].y);
            }
        }
        const bool bar = reduce_prod_ok(beta, pr);
        *reinterpret_cast<ulonglong2 *>(acc + (size_t)z * N + n) =
            make_ulonglong2(reduce_accm(a0, pr, bar), reduce_accm(b0, pr, bar));
        *reinterpret_cast<ulonglong2 *>(acc + ((size_t)ne + z) * N + n) =
            make_ulonglong2(reduce_accm(a1, pr, bar), reduce_accm(b1, pr, bar));
        return;
    }
    // hoisted rotation: the digits are read through sigma_g (evaluation form:
    // slot n takes slot brv(((2 brv(n) + 1) g mod 2N - 1) / 2))
    size_t sn = n;
    if (op.g) {
        const u32 rn = __brev((u32)n) >> (32 - logN);
        const u64 e2 = ((2 * (u64)rn + 1) * op.g) & ((2ull << logN) - 1);
        sn = __brev((u32)((e2 - 1) >> 1)) >> (32 - logN);
    }
    // issue every load before the first product (the kernel is bound by HBM),
    // the keys before the wait for the previous kernel
    u64 e[MAXB], k0[MAXB], k1[MAXB];
#pragma unroll
    for (int j = 0; j < MAXB; ++j) {
        if (j < beta) {
            k0[j] = evk[(((size_t)j * 2 + 0) * nfull + pz) * N + n];
            k1[j] = evk[(((size_t)j * 2 + 1) * nfull + pz) * N + n];
        }
    }
    pdl_wait();
#pragma unroll
    for (int j = 0; j < MAXB; ++j) {
        if (j < beta) {
            const u64 *src = (j == own) ? dsrc + (size_t)z * N : ext + ((size_t)j * ne + z) * N;
            e[j] = src[sn];
        }
    }
    Acc128 a0 = {0, 0, 0, 0}, a1 = {0, 0, 0, 0};
#pragma unroll
    for (int j = 0; j < MAXB; ++j) {
        if (j < beta) {
            mac_wide(a0, e[j], k0[j]);
            mac_wide(a1, e[j], k1[j]);
        }
    }
    acc[(size_t)z * N + n] = reduce_acc(a0, pr);
    acc[((size_t)ne + z) * N + n] = reduce_acc(a1, pr);
}

// whether an op can take the paired path
inline bool ip_pairs_ok(const IPOp &o)
{
    return o.g == 0 && ((((uintptr_t)o.ext | (uintptr_t)o.dsrc | (uintptr_t)o.evk | (uintptr_t)o.acc) & 15) == 0);
}

// index of the op holding row z in a table with exclusive prefix sums
__device__ __forceinline__ int find_op(const int *__restrict__ pre, int nop, int z)
{
    int lo = 0, hi = nop - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(pre + mid) <= z) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// MAXB: the largest digit count of the ops in the launch (loads for digits
// >= an op's own count are predicated off).  Up to three digits the kernel
// keeps to 64 registers, so that four CTAs share an SM and keep their loads
// in flight.
template <int MAXB, bool V2>
__global__ void __launch_bounds__(256, (MAXB <= 3 ? 4 : 1))
    k_inner(IPArgs A, int L, int nfull, const PrimeInfo *__restrict__ P, int logN)
{
    pdl_trigger();   // inner_body waits after issuing its key loads
    const int z = blockIdx.y;
    if (A.dop) {
        const int r = __ldg(A.drow + z);
        inner_body<MAXB, V2>(A.dop[r >> 7], r & 127, L, nfull, P, logN);
    } else {
        inner_body<MAXB, V2>(A.one, z, L, nfull, P, logN);
    }
}

template <int MAXB>
void launch_inner_b(const fides_ctx *c, const IPArgs &A, int total_limbs, bool pairs, cudaStream_t st)
{
    if (pairs) {
        dim3 grid(c->N / 512, total_limbs);
        FIDES_LAUNCH("k_inner", st, (k_inner<MAXB, true>), grid, dim3(256), A, c->L, c->L + c->K,
                     (const PrimeInfo *)c->d_prime, c->logN);
    } else {
        dim3 grid(c->N / 256, total_limbs);
        FIDES_LAUNCH("k_inner", st, (k_inner<MAXB, false>), grid, dim3(256), A, c->L, c->L + c->K,
                     (const PrimeInfo *)c->d_prime, c->logN);
    }
}

// pairs: < 0 decides from the inline op; the batched path passes what it
// found for all ops of the table
inline int launch_inner(const fides_ctx *c, const IPArgs &A, int total_limbs, int max_beta, cudaStream_t st,
                        int pairs = -1)
{
    const bool p2 = pairs < 0 ? (!A.dop && ip_pairs_ok(A.one)) : pairs != 0;
    switch (max_beta) {
    case 1: launch_inner_b<1>(c, A, total_limbs, p2, st); break;
    case 2: launch_inner_b<2>(c, A, total_limbs, p2, st); break;
    case 3: launch_inner_b<3>(c, A, total_limbs, p2, st); break;
    case 4: launch_inner_b<4>(c, A, total_limbs, p2, st); break;
    default: launch_inner_b<FIDES_MAX_DIGITS>(c, A, total_limbs, p2, st); break;
    }
    return fides_check_cuda(cudaGetLastError(), "inner product launch");
}

// ---------------------------------------------------------------------------
// Tensor product of HMult (Table I) in evaluation form, as its own pass:
// d0 = a0 b0 and d1 = a0 b1 + a1 b0 into out, d2 = a1 b1 into d2 (the
// key-switch input), two words per thread with 16-byte accesses: four words
// read and three written per coefficient, and three 128-bit reductions, which
// take the Barrett form of reduce_prod (the operands are canonical residues);
// with reduce128 the multiply pipe bounded the pass.  The INTT of d2 that
// follows runs without a prologue.  One op inline, or a device table of ops
// with exclusive prefix sums of their limb counts (grid.y = the total).
// ---------------------------------------------------------------------------
struct TensorOp {
    const u64 *a, *b;   // [2][nl][N]
    u64 *out;           // [2][nl][N]: d0, d1
    u64 *d2;            // [nl][N]
    int nl;
};

struct TensorArgs {
    const TensorOp *dop;
    const int *dpre;
    int nop;
    TensorOp one;
};

__device__ __forceinline__ void tensor_body(const TensorOp &o, int limb, const PrimeInfo *__restrict__ P, int logN)
{
    const size_t S = (size_t)o.nl << logN;
    const size_t i = ((size_t)limb << logN) + ((size_t)blockIdx.x * blockDim.x + threadIdx.x) * 2;
    const PrimeInfo p = P[limb];
    auto ld = [](const u64 *q) { return *reinterpret_cast<const ulonglong2 *>(q); };
    const ulonglong2 a0 = ld(o.a + i), a1 = ld(o.a + S + i), b0 = ld(o.b + i), b1 = ld(o.b + S + i);
    Acc128 mx = {0, 0, 0, 0}, my = {0, 0, 0, 0};
    mac_wide(mx, a0.x, b1.x);
    mac_wide(mx, a1.x, b0.x);
    mac_wide(my, a0.y, b1.y);
    mac_wide(my, a1.y, b0.y);
    *reinterpret_cast<ulonglong2 *>(o.out + i) = make_ulonglong2(mul_mod_small(a0.x, b0.x, p), mul_mod_small(a0.y, b0.y, p));
    *reinterpret_cast<ulonglong2 *>(o.out + S + i) = make_ulonglong2(reduce_acc2(mx, p), reduce_acc2(my, p));
    *reinterpret_cast<ulonglong2 *>(o.d2 + i) = make_ulonglong2(mul_mod_small(a1.x, b1.x, p), mul_mod_small(a1.y, b1.y, p));
}

__global__ void __launch_bounds__(256) k_tensor(TensorArgs A, const PrimeInfo *__restrict__ P, int logN)
{
    pdl_enter();
    const int z = blockIdx.y;
    if (A.dop) {
        const int k = find_op(A.dpre, A.nop, z);
        tensor_body(A.dop[k], z - __ldg(A.dpre + k), P, logN);
    } else {
        tensor_body(A.one, z, P, logN);
    }
}

// whether an HMult's tensor product can take the 16-byte pass
inline bool tensor_pass_ok(const void *a, const void *b, const void *out, const void *d2)
{
    return ((((uintptr_t)a | (uintptr_t)b | (uintptr_t)out | (uintptr_t)d2) & 15) == 0);
}

inline int launch_tensor_args(const fides_ctx *c, const TensorArgs &A, int total_limbs, cudaStream_t st)
{
    FIDES_LAUNCH("k_tensor", st, k_tensor, dim3(c->N / 512, total_limbs), dim3(256), A, (const PrimeInfo *)c->d_prime,
                 c->logN);
    return fides_check_cuda(cudaGetLastError(), "tensor product");
}

inline int launch_tensor(const fides_ctx *c, const u64 *a, const u64 *b, u64 *out, u64 *d2, int nl, cudaStream_t st)
{
    TensorArgs A;
    memset(&A, 0, sizeof(A));
    A.one = TensorOp{a, b, out, d2, nl};
    return launch_tensor_args(c, A, nl, st);
}

// ---------------------------------------------------------------------------
// Limb-set helpers
// ---------------------------------------------------------------------------
inline Seg seg_of(const u64 *src, u64 *dst, int count, int prime0, const u64 *aux = nullptr, u64 *out = nullptr,
                  int src_step = 1, int mode = 0, const TwPair *cst = nullptr)
{
    Seg s;
    s.src = src; s.dst = dst; s.aux = aux; s.out = out; s.side = nullptr; s.cst = cst; s.g = 0;
    s.count = count; s.prime0 = prime0; s.src_step = src_step; s.mode = mode; s.pstride = 0;
    return s;
}

// limb k of a segment as a segment of its own (the pointers job_of would
// compute for it, ring degree N)
inline Seg limb_of(const Seg &g, int k, size_t N)
{
    Seg s = g;
    s.src = g.src + (size_t)k * g.src_step * N;
    s.dst = g.dst ? g.dst + (size_t)k * N : nullptr;
    s.aux = g.aux ? g.aux + (size_t)k * N : nullptr;
    s.out = g.out ? g.out + (size_t)k * N : nullptr;
    s.side = g.side ? g.side + (size_t)k * N : nullptr;
    s.prime0 = g.prime0 + k;
    s.count = 1;
    return s;
}

inline void add_seg(LimbSet &S, const Seg &g)
{
    if (g.count <= 0) return;
    S.seg[S.nseg++] = g;
    S.total += g.count;
    S.modes |= g.mode;
}

inline LimbSet empty_set()
{
    LimbSet S;
    memset(&S, 0, sizeof(S));
    return S;
}

}  // namespace
