// Internal definitions of the GB300 CKKS key-switching engine: context layout,
// per-prime constants, job descriptors and 64-bit modular arithmetic.
//
// Modular arithmetic (Sec. III-F2 and its Table "mod_red"):
//   - Shoup multiplication by a fixed operand w with companion
//     w' = floor(w * 2^64 / q): one high and two low 64-bit products, result in
//     [0, 2q) for any 64-bit input (used for twiddles and per-prime constants).
//   - Reduction of a full 128-bit value (hi, lo): hi * 2^64 is folded with a
//     Shoup product by 2^64 mod q and lo with a one-word Barrett step
//     (mu = floor(2^64 / q)); two high and three low products in total.
//   - Additions keep values in [0, 2q) (lazy) or [0, q) (canonical) with one
//     conditional subtraction.
// All primes are below 2^61, so 4q < 2^63 and sums of up to 32 products of
// canonical residues fit in 128 bits.
#pragma once

#include <cstddef>
#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

#include "fides.h"

typedef uint64_t u64;
typedef uint32_t u32;

#define FIDES_MAX_PRIMES 64
#define FIDES_MAX_SEG 24
#define FIDES_MAX_DIGITS 8
#define FIDES_MAX_STREAMS 16   // streams with their own scratch pool (fides_ctx_add_stream)
#define FIDES_MAX_SRC 32
#define FIDES_TUNE_MAX 128   // NTT tile variants are kept per limb count up to this
#define FIDES_MAC_TERMS 32   // products one plaintext multiply-accumulate launch sums (each < 2^122)
#define FIDES_TC_MAX_SRC 16  // source primes of a tensor-core base conversion (K extent 8 x 16 = 128)

// A twiddle or constant with its Shoup companion.
struct __align__(16) TwPair {
    u64 w, wp;
};

// Per-prime constants.
struct __align__(16) PrimeInfo {
    u64 q;      // the prime
    u64 q2;     // 2q
    u64 mu;     // floor(2^64 / q)
    u64 r64;    // 2^64 mod q
    u64 r64p;   // Shoup companion of r64
    u64 ninv;   // N^-1 mod q
    u64 ninvp;  // Shoup companion of ninv
    u64 ninvw;  // N^-1 w1 mod q, w1 the twiddle of the last inverse stage (psi^-N/2)
    u64 ninvwp; // Shoup companion of ninvw
    u64 bmu;    // floor(2^(63+k) / q), k the bit length of q (reduce_prod)
};

// One contiguous run of limbs processed by a kernel: limb k of the run reads
// src + k*src_step*N, writes dst + k*N, optionally reads aux + k*N and writes
// out + k*N, and uses prime index prime0 + k.  `mode` selects an epilogue
// variant (see the functors in kernels.cu).
struct Seg {
    const u64 *src;
    u64 *dst;
    const u64 *aux;
    u64 *out;
    u64 *side;          // second output of a fused prologue (the key-switch input), or null
    const TwPair *cst;  // per-prime constants of a fused step (indexed by prime), or null
    u64 g;              // Galois element of a fused automorphism
    int count;
    int prime0;
    int src_step;   // 1: src advances one limb per limb; 0: every limb reads the same src limb
    int mode;       // prologue (inverse NTT) or epilogue (forward NTT) variant
    int pstride;    // words from polynomial 0 to polynomial 1 of a ciphertext operand
};

// The segments of a launch: inline (dseg == nullptr) or, for batches, a
// device-resident table dseg[0..nseg) with exclusive prefix sums dpre of the
// segment counts.
struct LimbSet {
    int nseg;
    int total;
    int modes;          // OR of the segments' modes (0: every inverse prologue is the plain load)
    const Seg *dseg;
    const int *dpre;
    Seg seg[FIDES_MAX_SEG];
};

// A job resolved for limb z of a LimbSet.
struct Job {
    const u64 *src;
    u64 *dst;
    const u64 *aux;
    u64 *out;
    u64 *side;
    const TwPair *cst;
    u64 g;
    int prime;
    int mode;
    int pstride;
};

struct fides_ctx {
    int device;
    int logN;
    int N;
    int L, K, dnum, alpha;
    u64 primes[FIDES_MAX_PRIMES];
    u64 psi[FIDES_MAX_PRIMES];

    PrimeInfo *d_prime;   // [L+K]
    TwPair *d_tw;         // [L+K][N]   psi^brv(k)
    TwPair *d_itw;        // [L+K][N]   psi^-brv(k)

    // ModUp base conversion, per (nl, digit j) at index (nl-1)*dnum + j:
    //   d_mu_scale[off .. off+alpha)        qhat_i^-1 mod q_i (Shoup pairs)
    //   d_mu_mat[off*(L+K) ..]              [alpha][L+K]: [qhat_i]_{prime z}
    TwPair *d_mu_scale;
    u64 *d_mu_mat;

    // ModDown base conversion P -> Q (independent of the level)
    TwPair *d_md_scale;   // [K]      Phat_k^-1 mod p_k
    u64 *d_md_mat;        // [K][L+K] [Phat_k]_{prime z}
    TwPair *d_md_pinv;    // [L]      P^-1 mod q_i
    u64 *d_md_negp;       // [L+K]    -P mod prime z (q-primes; the special ones unused)
    int round_nearest;    // FIDES_ROUND_NEAREST: ModDown converts centred residues, Rescale lifts the centred one

    // Rescale: [L][L], entry (l, i) = q_l^-1 mod q_i
    TwPair *d_rs_qlinv;
    // HMult fused with Rescale: [L][L][2], entry (l, i) = (P^-1 mod q_i,
    // q_l^-1 mod q_i)
    TwPair *d_hr;

    // Combined final constants of the inverse NTTs that feed a base conversion
    // (the N^-1 of the INTT times the conversion's qhat^-1), each c followed
    // by c w1 (w1 the twiddle of the last inverse stage, folded into it):
    //   d_mu_nscale[2 (nl(nl-1)/2 + i) + {0, 1}] = N^-1 qhat_{j(i),i}^-1 {1, w1} mod q_i, i < nl
    //   d_md_nscale[2 (L + k) + {0, 1}]          = N^-1 Phat_k^-1 {1, w1} mod p_k
    TwPair *d_mu_nscale;
    TwPair *d_md_nscale;

    // ModRaise: [L] q_0 mod q_i; host copy of i_q = psi_i^(N/2) mod q_i (X^(N/2) in evaluation form)
    TwPair *d_raise;
    TwPair iroot[FIDES_MAX_PRIMES];

    // Base conversion on the tensor cores (bconv_tc.cuh): the conversion
    // matrix of every ModUp job (nl, digit j) and of ModDown, as fp16 bytes
    // in the tensor cores' shared-memory operand layout, at byte offsets
    // tc_mu_off[nl-1][j] and tc_md_off of d_tc.  tc_on bit 0: ModUp images
    // exist (alpha <= FIDES_TC_MAX_SRC), bit 1: the ModDown image exists
    // (K <= FIDES_TC_MAX_SRC); without one the integer kernel converts.
    // d_c32[z] = 2^32 mod prime z with its Shoup companion.
    uint16_t *d_tc;
    size_t tc_mu_off[FIDES_MAX_PRIMES][FIDES_MAX_DIGITS];
    size_t tc_md_off;
    int tc_on;
    int tc_big;           // every prime >= 2^48 (the conversion's short epilogue)
    TwPair *d_c32;

    // Device status word: bits set by kernels whose bounded waits ran out
    // (FIDES_STATUS_*), read and cleared by fides_ctx_status.
    int *d_status;

    // Scratch pool for one operation at the top level.
    u64 *scratch;
    size_t scratch_words;

    // Streams registered with fides_ctx_add_stream, each with a scratch pool
    // of scratch_words words; n_spool is published with a release store after
    // its entry is written, and read with an acquire load (scratch_for).
    int n_spool;
    void *spool_stream[FIDES_MAX_STREAMS];
    u64 *spool[FIDES_MAX_STREAMS];

    // NTT tile variant per pass kind (forward columns, forward rows, inverse
    // rows, inverse columns) and limb count (ntt.cu)
    int sms;
    unsigned char ntt_var[4][FIDES_TUNE_MAX + 1];
};

// Scratch pool of a single-operation call on `stream`: the stream's own pool
// if it was registered, else the context's.
inline u64 *scratch_for(const fides_ctx *c, void *stream)
{
    const int n = __atomic_load_n(&c->n_spool, __ATOMIC_ACQUIRE);
    for (int i = 0; i < n; ++i)
        if (c->spool_stream[i] == stream) return c->spool[i];
    return c->scratch;
}

// A registered switching key: the caller's buffer [dnum][2][L+K][N] and the
// Galois element it switches from (0: relinearisation, s^2).
struct fides_key {
    const fides_ctx *ctx;
    const u64 *data;
    u64 g;
};

// Galois element any key is accepted for (fides_keyswitch)
#define FIDES_GALOIS_ANY (~(u64)0)

// ---------------------------------------------------------------------------
// Device modular arithmetic
// ---------------------------------------------------------------------------
__device__ __forceinline__ u64 mulhi64(u64 a, u64 b) { return __umul64hi(a, b); }

// a >= m ? a - m : a, for a, m < 2^63 (the sign of a - m decides)
__device__ __forceinline__ u64 csub(u64 a, u64 m)
{
    const long long d = (long long)(a - m);
    return d < 0 ? a : (u64)d;
}

// a * w mod q in [0, 2q) for any 64-bit a (Shoup).
__device__ __forceinline__ u64 mul_shoup(u64 a, u64 w, u64 wp, u64 q)
{
    return a * w - mulhi64(a, wp) * q;
}

__device__ __forceinline__ u64 mul_shoup(u64 a, const TwPair &t, u64 q)
{
    return mul_shoup(a, t.w, t.wp, q);
}

// x mod q in [0, 2q) for a 64-bit x (one-word Barrett).
__device__ __forceinline__ u64 reduce64_lazy(u64 x, const PrimeInfo &p)
{
    return x - mulhi64(x, p.mu) * p.q;
}

// (hi * 2^64 + lo) mod q, canonical.
__device__ __forceinline__ u64 reduce128(u64 hi, u64 lo, const PrimeInfo &p)
{
    u64 a = mul_shoup(hi, p.r64, p.r64p, p.q);   // [0, 2q)
    u64 b = reduce64_lazy(lo, p);                  // [0, 2q)
    u64 s = csub(a + b, p.q2);                     // [0, 2q)
    return csub(s, p.q);
}

// a * b mod q, canonical, for any 64-bit a, b.
__device__ __forceinline__ u64 mul_mod(u64 a, u64 b, const PrimeInfo &p)
{
    return reduce128(mulhi64(a, b), a * b, p);
}

// x mod q in [0, 3q) for x = hi * 2^64 + lo below 2^(k+63), k the bit length
// of q: a product of two values below 2q, or the sum of two products of
// canonical residues (primes below 2^61).  Barrett reduction whose quotient is
// the high word of one 64 x 64 product: q1 = floor(x / 2^(k-1)) fits in 64
// bits, and with bmu = floor(2^(63+k) / q) (below 2^64, since q > 2^(k-1))
// mulhi(q1, bmu) falls short of floor(x / q) by at most 2 -- one from each
// floor and one from truncating x.  Against reduce128 it drops the Shoup
// product by 2^64 mod q and one of the two high products.
__device__ __forceinline__ u64 reduce_prod(u64 hi, u64 lo, const PrimeInfo &p)
{
    const int s = 63 - __clzll((long long)p.q);   // k - 1, at least 1
    const u64 q1 = (hi << (64 - s)) | (lo >> s);
    return lo - mulhi64(q1, p.bmu) * p.q;
}

// a * b mod q, canonical, for a, b below 2q.
__device__ __forceinline__ u64 mul_mod_small(u64 a, u64 b, const PrimeInfo &p)
{
    return csub(csub(reduce_prod(mulhi64(a, b), a * b, p), p.q2), p.q);
}

// 128-bit accumulator
struct U128 {
    u64 lo, hi;
};

__device__ __forceinline__ void mac128(U128 &acc, u64 a, u64 b)
{
    u64 lo = a * b;
    u64 hi = mulhi64(a, b);
    acc.lo += lo;
    acc.hi += hi + (acc.lo < lo ? 1 : 0);
}

__device__ __forceinline__ Job job_of(const Seg &g, int z, int N)
{
    Job j;
    j.src = g.src + (size_t)z * g.src_step * N;
    j.dst = g.dst ? g.dst + (size_t)z * N : nullptr;
    j.aux = g.aux ? g.aux + (size_t)z * N : nullptr;
    j.out = g.out ? g.out + (size_t)z * N : nullptr;
    j.side = g.side ? g.side + (size_t)z * N : nullptr;
    j.cst = g.cst;
    j.g = g.g;
    j.prime = g.prime0 + z;
    j.mode = g.mode;
    j.pstride = g.pstride;
    return j;
}

__device__ __forceinline__ Job get_job(const LimbSet &S, int z, int N)
{
    if (S.dseg && S.nseg == S.total) return job_of(S.dseg[z], 0, N);   // one limb per segment
    if (S.dseg) {
        int lo = 0, hi = S.nseg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(S.dpre + mid) <= z) lo = mid; else hi = mid - 1;
        }
        return job_of(S.dseg[lo], z - __ldg(S.dpre + lo), N);
    }
    #pragma unroll 1
    for (int s = 0; s < S.nseg; ++s) {
        if (z < S.seg[s].count) return job_of(S.seg[s], z, N);
        z -= S.seg[s].count;
    }
    return job_of(S.seg[0], 0, N);
}

// ---------------------------------------------------------------------------
// Host-side helpers shared by the translation units
// ---------------------------------------------------------------------------
int fides_set_error(int code, const char *fmt, ...);
int fides_check_cuda(cudaError_t e, const char *what);

// Checks that `k` is a key of context c registered with Galois element g
// (FIDES_GALOIS_ANY: any element); FIDES_ERR_ARG for a NULL handle,
// FIDES_ERR_KEY for another context or element.  `what` names the caller.
int fides_check_key(const fides_ctx *c, const fides_key *k, u64 g, const char *what);

// out = sum_t cts[t] (.) pts[t] (+ out when accumulate), ciphertexts [2][nl][N]
// and plaintexts [nl][N] in evaluation form (elementwise.cu)
int launch_ptmac(const fides_ctx *c, const u64 *const *cts, const u64 *const *pts, int nt, u64 *out, int nl,
                 bool accumulate, cudaStream_t st);

// out = sum_t k[cidx[t]] (.) x[t] at nl limbs; x[t] has xl[t] >= nl limbs and is
// read in place; k is a device table of rows of kld per-limb residues
// (elementwise.cu)
int launch_cmac(const fides_ctx *c, const u64 *const *x, const int *xl, const int *cidx, int nt, const u64 *k,
                int kld, u64 *out, int nl, cudaStream_t st);

// tracing (trace.cu)
int fides_trace_begin(const char *name, cudaStream_t st);
void fides_trace_end(int id, cudaStream_t st);
void fides_count_launch();
int fides_trace_set(int on);

// Programmatic dependent launch: every kernel of the library lets the next
// kernel in its stream launch as soon as all of its CTAs are running, and waits
// for the previous kernel to finish (and its memory to be visible) before it
// reads anything a kernel produced.  The next kernel's CTAs thus occupy SMs
// freed during this kernel's last wave instead of after a launch gap.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// The two halves of pdl_enter, for kernels that first read data no kernel
// writes (twiddles, conversion matrices, keys, launch tables uploaded by the
// host) so that those reads overlap the previous kernel's last wave: trigger
// at entry, wait before the first read of anything a kernel produces.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... Params, typename... Args>
inline cudaError_t fides_launch_kernel(void (*kern)(Params...), dim3 grid, dim3 block, cudaStream_t st,
                                       Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <typename... Params, typename... Args>
inline cudaError_t fides_launch_kernel_smem(void (*kern)(Params...), dim3 grid, dim3 block, size_t smem,
                                            cudaStream_t st, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// Launch a kernel (with programmatic dependent launch): count it and, when
// tracing is on, bracket it with events.
#define FIDES_LAUNCH(name, st, kern, grid, block, ...)                  \
    do {                                                                \
        int fides_trace_id_ = fides_trace_begin(name, st);              \
        fides_launch_kernel(kern, grid, block, st, __VA_ARGS__);        \
        fides_trace_end(fides_trace_id_, st);                           \
        fides_count_launch();                                           \
    } while (0)

#define FIDES_LAUNCH_SMEM(name, st, kern, grid, block, smem, ...)            \
    do {                                                                    \
        int fides_trace_id_ = fides_trace_begin(name, st);                  \
        fides_launch_kernel_smem(kern, grid, block, smem, st, __VA_ARGS__); \
        fides_trace_end(fides_trace_id_, st);                               \
        fides_count_launch();                                               \
    } while (0)

// Bracket a whole public operation with events when tracing is on.
struct OpTrace {
    int id;
    cudaStream_t st;
    OpTrace(const char *name, cudaStream_t s) : id(fides_trace_begin(name, s)), st(s) {}
    ~OpTrace() { fides_trace_end(id, st); }
};
