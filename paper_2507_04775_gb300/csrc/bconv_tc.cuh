// Fast base conversion (Eq. 1) on the tensor cores (tcgen05, TMEM, bulk TMA).
//
// A job converts ns source limbs x_s (coefficient form, canonical, already
// scaled by qhat_s^-1) to nd target primes p_t:
//   y_t[n] = sum_s x_s[n] c_{s,t} mod p_t,   c_{s,t} = [qhat_s]_{p_t}.
// With the bytes x_s = sum_a x_{s,a} 2^(8a) and
// e_{s,t,a} = c_{s,t} 2^(8a) mod p_t = sum_b e_{s,t,a,b} 2^(8b),
//   y_t[n] = sum_b 2^(8b) D[n][8t + b] mod p_t,
//   D[n][8t + b] = sum_{s,a} x_{s,a}[n] e_{s,t,a,b},
// the product of a [coefficients x 8 ns] byte matrix with a [8 ns x 8 nd] byte
// matrix.  Bytes are exact in fp16 and every partial sum is an integer below
// 8 * 16 * 255^2 < 2^23 (2^24 with the offset below), exact in the fp32
// accumulator whatever the order of the additions, so the MMA gives D
// exactly.  The epilogue folds the eight sums of a target into a value below
// 2^80 and reduces it to [0, 4p_t), the range the forward NTT that follows
// takes; after that NTT the residues equal the integer kernel's.
//
// Persistent CTAs of 512 threads, each on one job with the job's matrix image
// resident in shared memory (one bulk TMA copy, completing on an mbarrier) and
// one accumulator of 8 nd columns in tensor memory; the CTAs of a job take its
// tiles of 128 coefficients (M = 128) round robin.  Per tile:
//   1. every thread writes the bytes of its prefetched source words (row m,
//      sources s0, s0 + 4, ...), as fp16, into the A operand;
//   2. thread 0 issues nsp/2 MMAs (K = 16: two columns of sources each) per
//      32 targets (N = 8 targets <= 256 per instruction) and commits them to
//      an mbarrier;
//   3. every thread issues the loads of its words of the next tile; thread 0
//      polls the mbarrier while the others wait at the CTA barrier; then
//      warp w reads accumulator lanes 32 (w mod 4) .. +31 (tcgen05.ld) for a
//      quarter of the targets, reduces and stores (coalesced 256-byte rows).
//      Two CTAs per SM overlap one's MMAs with the other's epilogue.
// Operand layout (K-major, no swizzle): 8-row x 16-byte core matrices, row r
// of a core matrix at +16 r; core matrices adjacent along K (one source: its
// eight bytes) 128 bytes apart (leading byte offset), adjacent 8-row groups
// 128 nsp bytes apart (stride byte offset); nsp = ns + 1 rounded up to even:
// after the sources, an offset column (A = 256, B = 2^15 for every output byte,
// both exact) starts every accumulator at 2^23, so that its fp32 bits read
// 0x4B000000 + D with no conversion.
//
// Centred conversion (round-to-nearest ModDown): the sources in the upper half
// of their range stand for x - q, which adds c (-Q_src) to every target, c
// their count.  ModDown images carry a correction block after the offset
// column (byte b of -Q_src mod p_t in elements 0..3 of row b); each of the
// four threads of a row puts the count among its own sources (0..4) into
// element s0 of that column of A, so the MMA adds c (-Q_src) byte by byte.
// It adds at most 16 x 255 to a sum, which keeps every sum below 2^23 for up
// to 16 sources (8 x 16 x 255^2 + 4080 < 2^23).  Floor jobs put zeros there.
//
// Every wait is bounded (about 2 s of %globaltimer): on a timeout the CTA sets
// FIDES_STATUS_WAIT_TIMEOUT in the context's status word, skips its outputs,
// frees its tensor memory and returns.
#pragma once

namespace {

constexpr int TC_M = 128;
constexpr int TC_THREADS = 512;

__device__ __forceinline__ u32 smem_addr(const void *p) { return (u32)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading / stride byte offsets,
// descriptor version 1, no swizzle
__device__ __forceinline__ u64 tc_desc(u32 addr, u32 lbo, u32 sbo)
{
    return (u64)((addr & 0x3FFFF) >> 4) | ((u64)(lbo >> 4) << 16) | ((u64)(sbo >> 4) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: fp32 accumulator, fp16 A and B, both
// K-major, M = 128, N = n
__device__ __forceinline__ u32 tc_idesc(int n)
{
    return (1u << 4) | ((u32)(n >> 3) << 17) | ((u32)(TC_M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(u32 bar, u32 count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_test(u32 bar, u32 parity)
{
    u32 ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ u64 global_ns()
{
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// true once the phase of `parity` has completed; false after `limit_ns`
// (about 2 s by default) or 2^26 polls
__device__ __forceinline__ bool mbar_wait(u32 bar, u32 parity, u64 limit_ns = 2000000000ull)
{
    if (mbar_test(bar, parity)) return true;
    const u64 t0 = global_ns();
    for (u32 it = 1; it < (1u << 26); ++it) {
        if (mbar_test(bar, parity)) return true;
        if ((it & 255) == 0 && global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// bulk copy global -> shared (16-byte aligned, a multiple of 16 bytes),
// completing `bytes` transactions on the mbarrier
__device__ __forceinline__ void bulk_load(u32 dst, const void *src, u32 bytes, u32 bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_alloc(u32 slot, u32 ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_free(u32 taddr, u32 ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(u32 d, u64 a, u64 b, u32 idesc, u32 accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(u32 bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 16 consecutive accumulator columns of the warp's 32 lanes; the wait names
// the registers so that no use of them is scheduled before it
__device__ __forceinline__ void tc_ld16(u32 taddr, u32 (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

// bytes k and k+1 of w as an fp16 pair: the permute builds the halves
// 0x64kk = 1024 + kk, and subtracting 1024 leaves kk exactly
__device__ __forceinline__ u32 f16_pair(u32 w, u32 sel)
{
    u32 r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(w), "r"(0x64646464u), "r"(sel));
    asm("sub.f16x2 %0, %0, %1;" : "+r"(r) : "r"(0x64006400u));
    return r;
}

// the eight bytes of x as fp16, byte a at element a
__device__ __forceinline__ uint4 bytes_f16(u64 x)
{
    const u32 w0 = (u32)x, w1 = (u32)(x >> 32);
    return make_uint4(f16_pair(w0, 0x4140u), f16_pair(w0, 0x4342u), f16_pair(w1, 0x4140u), f16_pair(w1, 0x4342u));
}

// Per-target constants of the epilogue.
struct TcTarget {
    u64 *dst;
    u64 p;
    u64 wp;      // floor(2^64 (2^32 mod p) / p): Shoup companion of 2^32 mod p
    u64 w;       // 2^32 mod p
};

// sum_b 2^(8b) D_b mod p, in [0, 4p) (the forward NTT's input range), from
// the accumulators f_b = bits(2^23 + D_b) = 0x4B000000 + D_b (the offset
// column adds 2^23 to every sum; D_b < 2^23).  w'_k = 2^8 f_2k+1 + f_2k = D_2k + 2^8 D_2k+1 + 0x4B000000
// (mod 2^32; the exponent bits of f_2k+1 shift out of the word, and the sum
// stays below 2^32); value = lo + 2^32 hi with lo, hi < 2^47.01.
// BIG (every target prime >= 2^48): 2^32 mod p = 2^32, and the Shoup quotient
// floor(hi wp / 2^64) is formed from 32-bit halves without the low x low
// product, so it may be one too small: hi 2^32 - q p in [0, 3p), and adding
// lo < p keeps the result below 4p.  Otherwise: full Shoup product and a
// reduction of lo.
template <bool BIG>
__device__ __forceinline__ u64 tc_reduce(const u32 *r, const TcTarget &T, const PrimeInfo &P)
{
    u32 w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) w[k] = r[2 * k + 1] * 256u + r[2 * k];
    constexpr u64 OFF = 0x4B000000ull * (1 + (1ull << 16));
    if constexpr (BIG) {
        // 32-bit limbs: lo = (l1, l0), hi = (h1, h0), wp = (v1, v0), p = (p1, p0)
        u32 l0, l1, h0, h1, m0, m1, q, x0, x1;
        const u32 v0 = (u32)T.wp, v1 = (u32)(T.wp >> 32), p0 = (u32)T.p, p1 = (u32)(T.p >> 32);
        asm("{\n\t.reg .u32 s;\n\t"
            // lo = w0 + 2^16 w1 - OFF, hi = w2 + 2^16 w3 - OFF
            "shl.b32 s, %10, 16;\n\t"
            "add.cc.u32 %0, %9, s;\n\t"
            "shr.u32 s, %10, 16;\n\t"
            "addc.u32 %1, s, 0;\n\t"
            "sub.cc.u32 %0, %0, 0x4B000000;\n\t"
            "subc.u32 %1, %1, 0x4B00;\n\t"
            "shl.b32 s, %12, 16;\n\t"
            "add.cc.u32 %2, %11, s;\n\t"
            "shr.u32 s, %12, 16;\n\t"
            "addc.u32 %3, s, 0;\n\t"
            "sub.cc.u32 %2, %2, 0x4B000000;\n\t"
            "subc.u32 %3, %3, 0x4B00;\n\t"
            // mid = h1 v0 + h0 v1 (< 2^49); q = h1 v1 + mid / 2^32
            "mul.lo.u32 %4, %3, %13;\n\t"
            "mul.hi.u32 %5, %3, %13;\n\t"
            "mad.lo.cc.u32 %4, %2, %14, %4;\n\t"
            "madc.hi.u32 %5, %2, %14, %5;\n\t"
            "mad.lo.u32 %6, %3, %14, %5;\n\t"
            // x = lo + 2^32 h0 - q p (mod 2^64)
            "mul.lo.u32 s, %6, %15;\n\t"
            "sub.cc.u32 %7, %0, s;\n\t"
            "mul.hi.u32 s, %6, %15;\n\t"
            "add.u32 %8, %1, %2;\n\t"
            "subc.u32 %8, %8, s;\n\t"
            "mul.lo.u32 s, %6, %16;\n\t"
            "sub.u32 %8, %8, s;\n\t"
            "}"
            : "=&r"(l0), "=&r"(l1), "=&r"(h0), "=&r"(h1), "=&r"(m0), "=&r"(m1), "=&r"(q), "=&r"(x0), "=&r"(x1)
            : "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(v0), "r"(v1), "r"(p0), "r"(p1));
        return ((u64)x1 << 32) | x0;
    } else {
        const u64 lo = (u64)w[0] + ((u64)w[1] << 16) - OFF;
        const u64 hi = (u64)w[2] + ((u64)w[3] << 16) - OFF;
        const u64 x = hi * T.w - mulhi64(hi, T.wp) * T.p;       // [0, 2p)
        return x + reduce64_lazy(lo, P);                        // < 4p
    }
}

// One CTA: the job's matrix image resident in shared memory and one
// accumulator in tensor memory; tiles blockIdx.x, + gridDim.x, ... of the
// job's N / 128.  Per tile: the source words prefetched during the previous
// tile are written as bf16 bytes into the A operand; thread 0 issues the MMAs;
// every thread issues the loads of the next tile's words, waits for the MMAs,
// then reduces and stores its share of the accumulator.
template <bool BIG>
__device__ __forceinline__ void bconv_tc_body(const BConvJob &B, const PrimeInfo *__restrict__ P,
                                              const TwPair *__restrict__ c32, int logN, u32 ncols, int *status)
{
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ __align__(8) u64 bar[2];
    __shared__ u32 tslot;
    __shared__ int sok;
    __shared__ TcTarget stg[FIDES_MAX_PRIMES];
    __shared__ PrimeInfo sp[BIG ? 1 : FIDES_MAX_PRIMES];

    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const int N = 1 << logN, ntiles = N / TC_M;
    const int ns = B.n_src, nsp = (ns + 2 + B.tc_corr) & ~1;   // sources, offset and correction columns, even
    int nd = 0;
    for (int r = 0; r < B.nrun; ++r) nd += B.run[r].count;
    const int ndp = (nd + 1) & ~1;
    unsigned char *sA = tsm;
    unsigned char *sB = tsm + 2048 * nsp;
    const u32 bar0 = smem_addr(&bar[0]), bar1 = smem_addr(&bar[1]);

    if (t == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (t < nd) {
        int rem = t, pz = 0;
        u64 *ptr = nullptr;
        for (int r = 0; r < B.nrun; ++r) {
            if (rem < B.run[r].count) {
                pz = B.run[r].prime0 + rem;
                ptr = B.run[r].dst + (size_t)rem * N;
                break;
            }
            rem -= B.run[r].count;
        }
        const TwPair cw = c32[pz];
        stg[t] = TcTarget{ptr, P[pz].q, cw.wp, cw.w};
        if (!BIG) sp[t] = P[pz];
    }
    __syncthreads();
    if (t == 0) bulk_load(smem_addr(sB), B.tc, (u32)ndp * nsp * 128, bar0);
    // everything above reads only the job and the context's tables; the
    // sources below are the previous kernel's output, and no tensor memory is
    // taken before it has finished (an early-launched conversion must not
    // hold it while this one waits)
    pdl_wait();
    __syncwarp();
    if (w == 0) tmem_alloc(smem_addr(&tslot), ncols);

    // this thread's A rows and sources: row m, sources s0, s0 + 4, ...
    constexpr int SPT = FIDES_TC_MAX_SRC / (TC_THREADS / TC_M);
    const int m = t & (TC_M - 1), s0 = t / TC_M;
    unsigned char *arow = sA + (m >> 3) * (nsp * 128) + (m & 7) * 16;
    u64 xr[SPT];
    u64 half[SPT];   // (q_s - 1) / 2 of this thread's sources (centred jobs)
#pragma unroll
    for (int k = 0; k < SPT; ++k) {
        const int s = s0 + k * (TC_THREADS / TC_M);
        half[k] = (B.centred && s < ns) ? (P[B.src_prime0 + s].q >> 1) : ~0ull;
    }
    int tile = blockIdx.x;
    if (tile < ntiles) {
#pragma unroll
        for (int k = 0; k < SPT; ++k) {
            const int s = s0 + k * (TC_THREADS / TC_M);
            xr[k] = s < ns ? B.src[(size_t)s * N + (size_t)tile * TC_M + m] : 0;
        }
    }
    // constant columns of A: the offset column (fp16 256 in element 0 of row
    // m; the image holds 2^15 there for every output byte) and a zero column
    if (t < TC_M) {
        *(uint4 *)(arow + ns * 128) = make_uint4(0x5C00u, 0, 0, 0);
        for (int col = ns + 1; col < nsp; ++col) *(uint4 *)(arow + col * 128) = make_uint4(0, 0, 0, 0);
    }
    // one thread polls each mbarrier; the others wait at the CTA barrier
    if (t == 0) {
        sok = mbar_wait(bar0, 0);
        if (!sok) {
            atomicOr(status, FIDES_STATUS_WAIT_TIMEOUT);
            mbar_wait(bar0, 0);   // the copy may still be in flight
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    bool ok = sok != 0;
    const u32 tm = tslot;

    const u32 a0 = smem_addr(sA), b0 = smem_addr(sB), sbo = (u32)nsp * 128;
    const int q4 = w & 3, grp = w >> 2;
    constexpr int GROUPS = TC_THREADS / 128;
    for (u32 phase = 0; ok && tile < ntiles; tile += gridDim.x, phase ^= 1) {
        u32 cnt = 0;
#pragma unroll
        for (int k = 0; k < SPT; ++k) {
            const int s = s0 + k * (TC_THREADS / TC_M);
            if (s < ns) *(uint4 *)(arow + s * 128) = bytes_f16(xr[k]);
            cnt += xr[k] > half[k] ? 1u : 0u;   // half = ~0: never (floor jobs, missing sources)
        }
        if (B.centred) {
            // fp16 of 0..4
            const u32 f = cnt == 0 ? 0u : (cnt == 1 ? 0x3C00u : (cnt == 2 ? 0x4000u : (cnt == 3 ? 0x4200u : 0x4400u)));
            *(uint16_t *)(arow + (ns + 1) * 128 + 2 * s0) = (uint16_t)f;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (t == 0) {
            for (int s = 0; s < nsp / 2; ++s)
                for (int c = 0; 32 * c < ndp; ++c)
                    tc_mma(tm + 256 * c, tc_desc(a0 + 256 * s, 128, sbo),
                           tc_desc(b0 + c * 32 * sbo + 256 * s, 128, sbo), tc_idesc(8 * min(32, ndp - 32 * c)),
                           s > 0);
            tc_commit(bar1);
        }
        const int next = tile + gridDim.x;
        if (next < ntiles) {
#pragma unroll
            for (int k = 0; k < SPT; ++k) {
                const int s = s0 + k * (TC_THREADS / TC_M);
                xr[k] = s < ns ? B.src[(size_t)s * N + (size_t)next * TC_M + m] : 0;
            }
        }
        if (t == 0) {
            sok = mbar_wait(bar1, phase);
            if (!sok) atomicOr(status, FIDES_STATUS_WAIT_TIMEOUT);
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        ok = sok != 0;
        if (!ok) break;
        const size_t n = (size_t)tile * TC_M + 32 * q4 + lane;
        const u32 lanes = (u32)(32 * q4) << 16;
        for (int pr = grp; 2 * pr < nd; pr += GROUPS) {   // targets 2 pr, 2 pr + 1
            u32 r[16];
            tc_ld16(tm + lanes + 16 * pr, r);
            const int t0 = 2 * pr;
            const TcTarget T0 = stg[t0];
            T0.dst[n] = tc_reduce<BIG>(r, T0, sp[BIG ? 0 : t0]);
            if (t0 + 1 < nd) {
                const TcTarget T1 = stg[t0 + 1];
                T1.dst[n] = tc_reduce<BIG>(r + 8, T1, sp[BIG ? 0 : t0 + 1]);
            }
        }
        tc_fence_before();   // the next tile's MMAs follow its conversion barrier
    }
    tc_fence_before();
    __syncthreads();
    if (w == 0) tmem_free(tm, ncols);
}

template <bool BIG>
__global__ void __launch_bounds__(TC_THREADS, 2) k_bconv_tc(BConvArgs A, const PrimeInfo *__restrict__ P,
                                                            const TwPair *__restrict__ c32, int logN, u32 ncols,
                                                            int *status)
{
    // the dependents may launch now; the body waits for the previous kernel
    // after staging the job's constants
    pdl_trigger();
    if (A.djob) bconv_tc_body<BIG>(A.djob[blockIdx.y], P, c32, logN, ncols, status);
    else bconv_tc_body<BIG>(A.job[blockIdx.y], P, c32, logN, ncols, status);
}

// One launch for the tensor-core jobs of G (any mix of source counts up to
// FIDES_TC_MAX_SRC).  Tensor memory per CTA: 8 nd columns rounded up to a power
// of two (at least 32); at most as many CTAs per SM as tensor memory holds (the
// dynamic shared memory is raised so that no more fit: a CTA beyond that would
// wait in its allocation) and two by registers.  The CTAs of a job take its
// N / 128 tiles round robin.
// Dynamic shared memory of one job: A operand and matrix image.
inline int bconv_tc_smem(const BConvJob &j)
{
    int nd = 0;
    for (int r = 0; r < j.nrun; ++r) nd += j.run[r].count;
    const int nsp = (j.n_src + 2 + j.tc_corr) & ~1, ndp = (nd + 1) & ~1;
    return 2048 * nsp + 128 * ndp * nsp;
}

template <bool BIG>
inline int launch_bconv_tc_t(const fides_ctx *c, const BConvArgs &G, int max_ns, int max_dst, cudaStream_t st)
{
    static int static_smem = -1;
    if (static_smem < 0) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, k_bconv_tc<BIG>) != cudaSuccess)
            return fides_check_cuda(cudaGetLastError(), "bconv tc");
        static_smem = (int)fa.sharedSizeBytes;
        cudaFuncSetAttribute(k_bconv_tc<BIG>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024 - static_smem);
    }
    (void)max_ns;
    const int ndp = (max_dst + 1) & ~1;
    u32 ncols = 32;
    while (ncols < (u32)(8 * ndp)) ncols <<= 1;
    const int cap = std::min(2, (int)(512 / ncols));          // resident CTAs per SM
    const size_t need = (size_t)G.tc_smem;
    if (need + static_smem > 227 * 1024)
        return fides_set_error(FIDES_ERR_UNSUPPORTED, "bconv tc: %zu bytes of shared memory", need);
    const size_t sm_bytes = 228 * 1024, per_cta = sm_bytes / (cap + 1) + 1;   // cap + 1 CTAs must not fit
    size_t smem = std::max(need, per_cta > (size_t)static_smem + 1024 ? per_cta - static_smem - 1024 : 0);
    smem = (smem + 127) & ~(size_t)127;
    const int tiles = c->N / TC_M;
    const int per_job = std::max(1, std::min(tiles, cap * c->sms / G.njob));   // one wave
    dim3 grid(per_job, G.njob), block(TC_THREADS);
    FIDES_LAUNCH_SMEM("k_bconv_tc", st, k_bconv_tc<BIG>, grid, block, smem, G, (const PrimeInfo *)c->d_prime,
                      (const TwPair *)c->d_c32, c->logN, ncols, c->d_status);
    return fides_check_cuda(cudaGetLastError(), "bconv tc launch");
}

inline int launch_bconv_tc(const fides_ctx *c, const BConvArgs &G, int max_ns, int max_dst, cudaStream_t st)
{
    return c->tc_big ? launch_bconv_tc_t<true>(c, G, max_ns, max_dst, st)
                     : launch_bconv_tc_t<false>(c, G, max_ns, max_dst, st);
}

}  // namespace
