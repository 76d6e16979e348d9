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
// One CTA per SM on one job, with the job's matrix image resident in shared
// memory (one bulk copy, completing on an mbarrier); the CTAs of a job take
// its tiles of 128 coefficients (M = 128) round robin.  Inside a CTA, warps
// have roles that hand tiles over through mbarriers (see bconv_tc_body): a
// loader brings each tile's source rows in with bulk copies, ahead of use;
// producers write their bytes as fp16 into the A operand (two buffers); one
// thread issues nsp/2 MMAs (K = 16: two columns of sources each) per 32
// targets (N = 8 targets <= 256 per instruction) into one of two
// accumulators in tensor memory; and twelve epilogue warps read the
// accumulator (tcgen05.ld), reduce and store coalesced 256-byte rows, while
// the next tile's MMAs run.
// Operand layout (K-major, no swizzle): 8-row x 16-byte core matrices, row r
// of a core matrix at +16 r; core matrices adjacent along K (one source: its
// eight bytes) 128 bytes apart (leading byte offset), adjacent 8-row groups
// 128 nsp bytes apart (stride byte offset); nsp = ns + 2 (+ 1 with the
// correction column) rounded down to even: after the sources, an offset column (A = 256, B = 2^15 for every output byte,
// both exact) starts every accumulator at 2^23, so that its fp32 bits read
// 0x4B000000 + D with no conversion.
//
// Centred conversion (round-to-nearest ModDown): the sources in the upper half
// of their range stand for x - q, which adds c (-Q_src) to every target, c
// their count.  ModDown images carry a correction block after the offset
// column (byte b of -Q_src mod p_t in elements 0..3 of row b); the producer
// thread of a row puts the count c (0..16) into element 0 of that column of A
// (elements 1..3 stay zero), so the MMA adds c (-Q_src) byte by byte.
// It adds at most 16 x 255 to a sum, which keeps every sum below 2^23 for up
// to 16 sources (8 x 16 x 255^2 + 4080 < 2^23).  Floor jobs put zeros there.
//
// Every wait is bounded (about 2 s of %globaltimer): on a timeout the role
// sets FIDES_STATUS_WAIT_TIMEOUT in the context's status word and a CTA-wide
// abort flag, every role leaves its loop (skipping the outputs it has not
// written), the loader and the MMA thread wait (again bounded) for their
// copies and products in flight, and the CTA frees its tensor memory and
// returns.
#pragma once

namespace {

constexpr int TC_M = 128;
constexpr int TC_PROD_WARPS = 4;                                   // warps 0-3: A rows
constexpr int TC_LOAD_WARP = 4;                                    // bulk copies of the sources
constexpr int TC_MMA_WARP = 5;                                     // MMA issue
constexpr int TC_EPI_WARP0 = 6;                                    // warps 6..: epilogue
constexpr int TC_EPI_GROUPS = 3;                                   // of four warps each
constexpr int TC_THREADS = 32 * (TC_EPI_WARP0 + 4 * TC_EPI_GROUPS);   // 576
constexpr int TC_MAX_DEPTH = 4;                                    // source stages

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

// Shape of a launch's pipeline (the same for all its CTAs).
struct TcPipe {
    int depth;      // source stages: tiles whose bulk copies may be in flight
    int na;         // A operand buffers
    int nbuf;       // accumulators in tensor memory
    u32 acc_cols;   // tensor-memory columns of one accumulator (a power of two)
    u32 ncols;      // columns allocated: nbuf x acc_cols
    u64 limit_ns;   // limit of every pipeline wait (about 2 s)
    int stall;      // self-test: CTA (0, 0) never copies its first tile in
};

// mbarriers of a CTA: source stage full / empty, A buffer full / empty,
// accumulator full / empty, matrix image
constexpr int TC_MAX_ACC = 4;   // accumulators in tensor memory (four of at most 128 columns)
constexpr int TB_SF = 0, TB_SE = TC_MAX_DEPTH, TB_AF = 2 * TC_MAX_DEPTH, TB_AE = TB_AF + 2, TB_CF = TB_AE + 2,
              TB_CE = TB_CF + TC_MAX_ACC, TB_IMG = TB_CE + TC_MAX_ACC, TB_COUNT = TB_IMG + 1;

__device__ __forceinline__ void mbar_arrive(u32 bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// bulk copy global -> shared completing on an mbarrier whose transaction
// count the caller has already raised
__device__ __forceinline__ void bulk_copy(u32 dst, const void *src, u32 bytes, u32 bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// A pipeline wait: true once the phase of `parity` has completed.  False when
// another role has given up (abort set), or after limit_ns of %globaltimer,
// which sets abort and the status bit, so that every role leaves its loop.
// Lanes of one warp may disagree (abort set as the phase completes), so warps
// that go on to warp-wide instructions combine their lanes' results first.
__device__ __forceinline__ bool pipe_wait(u32 bar, u32 parity, volatile int *abort, int *status, u64 limit_ns)
{
    if (mbar_test(bar, parity)) return true;
    const u64 t0 = global_ns();
    for (u32 it = 1;; ++it) {
        if (mbar_test(bar, parity)) return true;
        if ((it & 63) == 0) {
            if (*abort) return false;
            if (global_ns() - t0 > limit_ns || it >= (1u << 26)) {
                *abort = 1;
                atomicOr(status, FIDES_STATUS_WAIT_TIMEOUT);
                return false;
            }
        }
    }
}

// One CTA on one job, over tiles blockIdx.x, + gridDim.x, ... of its N / 128.
// Four roles run at their own pace, handing tiles over through mbarriers:
//   warp 4, one thread:   bulk copies of a tile's ns source rows (1 KB each)
//                         into a ring of `depth` stages;
//   warps 0-3:            thread m writes the bytes of row m of every source
//                         as fp16 into one of `na` A buffers;
//   warp 5, one thread:   the MMAs of a tile into one of `nbuf` accumulators;
//   warps 6-17:           tcgen05.ld of the accumulator (warp w reads lanes
//                         32 (w mod 4) ..), reduction and coalesced stores,
//                         three groups of four warps splitting the targets.
// So a tile's epilogue overlaps the next tile's MMAs and the bulk copies of
// the tiles after it.
template <bool BIG>
__device__ __forceinline__ void bconv_tc_body(const BConvJob &B, const PrimeInfo *__restrict__ P,
                                              const TwPair *__restrict__ c32, int logN, const TcPipe &pp,
                                              int *status)
{
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ __align__(8) u64 bars[TB_COUNT];
    __shared__ u32 tslot;
    __shared__ volatile int sabort;
    __shared__ TcTarget stg[FIDES_MAX_PRIMES];
    __shared__ PrimeInfo sp[BIG ? 1 : FIDES_MAX_PRIMES];
    __shared__ u64 shalf[FIDES_TC_MAX_SRC];

    const int t = threadIdx.x, w = t >> 5, lane = t & 31;
    const int N = 1 << logN, ntiles = N / TC_M;
    const int ns = B.n_src, nsp = (ns + 2 + B.tc_corr) & ~1;   // sources, offset and correction columns, even
    int nd = 0;
    for (int r = 0; r < B.nrun; ++r) nd += B.run[r].count;
    const int ndp = (nd + 1) & ~1;
    const int T = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const u32 szA = 2048u * nsp, szS = 1024u * ns;
    unsigned char *sB = tsm;
    unsigned char *sA = tsm + (size_t)ndp * nsp * 128;
    unsigned char *sS = sA + (size_t)pp.na * szA;
    const u32 bar0 = smem_addr(&bars[0]);
    auto bar = [&](int i) -> u32 { return bar0 + 8u * i; };

    if (t == 0) {
        for (int d = 0; d < pp.depth; ++d) {
            mbar_init(bar(TB_SF + d), 1);
            mbar_init(bar(TB_SE + d), TC_PROD_WARPS);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(bar(TB_AF + i), TC_PROD_WARPS);
            mbar_init(bar(TB_AE + i), 1);
        }
        for (int i = 0; i < pp.nbuf; ++i) {
            mbar_init(bar(TB_CF + i), 1);
            mbar_init(bar(TB_CE + i), 4 * TC_EPI_GROUPS);
        }
        mbar_init(bar(TB_IMG), 1);
        sabort = 0;
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
    // (q_s - 1) / 2 of the sources (centred jobs; ~0: never above)
    if (t < ns) shalf[t] = B.centred ? (P[B.src_prime0 + t].q >> 1) : ~0ull;
    // constant columns of every A buffer: the offset column (fp16 256 in
    // element 0 of row m; the image holds 2^15 there for every output byte),
    // the correction column (element 0 takes the row's count in centred
    // jobs) and padding
    if (t < TC_M) {
        for (int b = 0; b < pp.na; ++b) {
            unsigned char *arow = sA + b * szA + (t >> 3) * (nsp * 128) + (t & 7) * 16;
            *(uint4 *)(arow + ns * 128) = make_uint4(0x5C00u, 0, 0, 0);
            for (int col = ns + 1; col < nsp; ++col) *(uint4 *)(arow + col * 128) = make_uint4(0, 0, 0, 0);
        }
    }
    __syncthreads();
    if (t == 0) bulk_load(smem_addr(sB), B.tc, (u32)ndp * nsp * 128, bar(TB_IMG));
    // everything above reads only the job and the context's tables; the
    // sources are the previous kernel's output, and no tensor memory is taken
    // before it has finished (an early-launched conversion must not hold it
    // while this one waits)
    pdl_wait();
    __syncwarp();
    if (w == 0) tmem_alloc(smem_addr(&tslot), pp.ncols);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the constant columns, for the MMAs
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const u32 tm = tslot;
    const u64 lim = pp.limit_ns;

    if (w < TC_PROD_WARPS) {
        const int m = t;
        unsigned char *arow0 = sA + (m >> 3) * (nsp * 128) + (m & 7) * 16;
        for (int k = 0; k < T; ++k) {
            const int ss = k % pp.depth, sa = k % pp.na;
            bool ok = pipe_wait(bar(TB_SF + ss), (u32)(k / pp.depth) & 1, &sabort, status, lim);
            if (ok && k >= pp.na) ok = pipe_wait(bar(TB_AE + sa), (u32)(k / pp.na - 1) & 1, &sabort, status, lim);
            if (!__all_sync(0xffffffffu, ok)) break;   // one decision per warp (it synchronises below)
            const u64 *src = (const u64 *)(sS + ss * szS) + m;
            unsigned char *arow = arow0 + sa * szA;
            u32 cnt = 0;
#pragma unroll 4
            for (int s = 0; s < ns; ++s) {
                const u64 x = src[s * TC_M];
                *(uint4 *)(arow + s * 128) = bytes_f16(x);
                cnt += x > shalf[s] ? 1u : 0u;
            }
            if (B.centred) {
                unsigned short h;   // fp16 of the count, 0..16 (exact)
                asm("cvt.rn.f16.u32 %0, %1;" : "=h"(h) : "r"(cnt));
                *(unsigned short *)(arow + (ns + 1) * 128) = h;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(bar(TB_AF + sa));
                mbar_arrive(bar(TB_SE + ss));
            }
        }
    } else if (w == TC_LOAD_WARP) {
        if (lane == 0) {
            int last[TC_MAX_DEPTH];   // the last tile copied into each stage, -1: none
            for (int d = 0; d < TC_MAX_DEPTH; ++d) last[d] = -1;
            for (int k = 0; k < T; ++k) {
                const int ss = k % pp.depth;
                if (k >= pp.depth && !pipe_wait(bar(TB_SE + ss), (u32)(k / pp.depth - 1) & 1, &sabort, status, lim))
                    break;
                if (pp.stall && k == 0 && blockIdx.x == 0 && blockIdx.y == 0) continue;   // self-test
                const size_t tile = (size_t)blockIdx.x + (size_t)k * gridDim.x;
                const u32 dst = smem_addr(sS + ss * szS);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar(TB_SF + ss)),
                             "r"(szS)
                             : "memory");
                for (int s = 0; s < ns; ++s)
                    bulk_copy(dst + 1024u * s, B.src + (size_t)s * N + tile * TC_M, 1024u, bar(TB_SF + ss));
                last[ss] = k;
            }
            // copies still in flight land before the CTA leaves
            for (int ss = 0; ss < pp.depth; ++ss)
                if (last[ss] >= 0) mbar_wait(bar(TB_SF + ss), (u32)(last[ss] / pp.depth) & 1);
        }
    } else if (w == TC_MMA_WARP) {
        if (lane == 0) {
            int issued = 0;
            const bool img = pipe_wait(bar(TB_IMG), 0, &sabort, status, lim);
            const u32 a0 = smem_addr(sA), b0 = smem_addr(sB), sbo = (u32)nsp * 128;
            for (int k = 0; img && k < T; ++k) {
                const int sa = k % pp.na, sb = k % pp.nbuf;
                if (!pipe_wait(bar(TB_AF + sa), (u32)(k / pp.na) & 1, &sabort, status, lim)) break;
                if (k >= pp.nbuf && !pipe_wait(bar(TB_CE + sb), (u32)(k / pp.nbuf - 1) & 1, &sabort, status, lim))
                    break;
                tc_fence_after();
                const u32 acc = tm + sb * pp.acc_cols, ab = a0 + sa * szA;
                for (int s = 0; s < nsp / 2; ++s)
                    for (int c = 0; 32 * c < ndp; ++c)
                        tc_mma(acc + 256 * c, tc_desc(ab + 256 * s, 128, sbo),
                               tc_desc(b0 + c * 32 * sbo + 256 * s, 128, sbo), tc_idesc(8 * min(32, ndp - 32 * c)),
                               s > 0);
                tc_commit(bar(TB_AE + sa));
                tc_commit(bar(TB_CF + sb));
                issued = k + 1;
            }
            // the image copy and the issued products finish before the
            // tensor memory is freed and the CTA leaves
            mbar_wait(bar(TB_IMG), 0);
            if (issued > 0) mbar_wait(bar(TB_CF + (issued - 1) % pp.nbuf), (u32)((issued - 1) / pp.nbuf) & 1);
        }
    } else {
        const int grp = (w - TC_EPI_WARP0) >> 2, q4 = w & 3;
        const u32 lanes = (u32)(32 * q4) << 16;
        for (int k = 0; k < T; ++k) {
            const int sb = k % pp.nbuf;
            const bool ok = pipe_wait(bar(TB_CF + sb), (u32)(k / pp.nbuf) & 1, &sabort, status, lim);
            if (!__all_sync(0xffffffffu, ok)) break;   // one decision per warp (tcgen05.ld is warp-wide)
            tc_fence_after();
            const size_t n = ((size_t)blockIdx.x + (size_t)k * gridDim.x) * TC_M + 32 * q4 + lane;
            const u32 acc = tm + sb * pp.acc_cols + lanes;
            for (int pr = grp; 2 * pr < nd; pr += TC_EPI_GROUPS) {
                u32 r[16];
                tc_ld16(acc + 16 * pr, r);
                const int t0 = 2 * pr;
                const TcTarget T0 = stg[t0];
                T0.dst[n] = tc_reduce<BIG>(r, T0, sp[BIG ? 0 : t0]);
                if (t0 + 1 < nd) {
                    const TcTarget T1 = stg[t0 + 1];
                    T1.dst[n] = tc_reduce<BIG>(r + 8, T1, sp[BIG ? 0 : t0 + 1]);
                }
            }
            tc_fence_before();   // the accumulator's reads are done before it is handed back
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(TB_CE + sb));
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (w == 0) tmem_free(tm, pp.ncols);
}

template <bool BIG>
__global__ void __launch_bounds__(TC_THREADS, 1) k_bconv_tc(BConvArgs A, const PrimeInfo *__restrict__ P,
                                                            const TwPair *__restrict__ c32, int logN, TcPipe pp,
                                                            int *status)
{
    // the dependents may launch now; the body waits for the previous kernel
    // after staging the job's constants
    pdl_trigger();
    if (A.djob) bconv_tc_body<BIG>(A.djob[blockIdx.y], P, c32, logN, pp, status);
    else bconv_tc_body<BIG>(A.job[blockIdx.y], P, c32, logN, pp, status);
}

// Dynamic shared memory of one job with one A buffer and no source stage:
// A operand and matrix image.
inline int bconv_tc_smem(const BConvJob &j)
{
    int nd = 0;
    for (int r = 0; r < j.nrun; ++r) nd += j.run[r].count;
    const int nsp = (j.n_src + 2 + j.tc_corr) & ~1, ndp = (nd + 1) & ~1;
    return 2048 * nsp + 128 * ndp * nsp;
}

// One launch for the tensor-core jobs of G (any mix of source counts up to
// FIDES_TC_MAX_SRC), one CTA per SM: its tensor memory holds two
// accumulators of 8 nd columns each (rounded up to a power of two, at least
// 32), or one when two would exceed the 512 columns, and the dynamic shared
// memory is raised to more than half the SM's so that no second CTA of a
// conversion shares the SM (it would wait in its allocation).  The source
// ring is as deep as shared memory allows, up to TC_MAX_DEPTH tiles, with two
// A buffers, else one.  The CTAs of a job take its N / 128 tiles round robin.
template <bool BIG>
inline int launch_bconv_tc_t(const fides_ctx *c, const BConvArgs &G, int max_ns, int max_dst, cudaStream_t st,
                             u64 limit_ns, int stall)
{
    static int static_smem = -1;
    if (static_smem < 0) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, k_bconv_tc<BIG>) != cudaSuccess)
            return fides_check_cuda(cudaGetLastError(), "bconv tc");
        static_smem = (int)fa.sharedSizeBytes;
        cudaFuncSetAttribute(k_bconv_tc<BIG>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024 - static_smem);
    }
    const int ndp = (max_dst + 1) & ~1;
    TcPipe pp;
    pp.acc_cols = 32;
    while (pp.acc_cols < (u32)(8 * ndp)) pp.acc_cols <<= 1;
    pp.nbuf = std::min<int>(TC_MAX_ACC, 512 / pp.acc_cols);
    pp.ncols = pp.nbuf * pp.acc_cols;
    pp.limit_ns = limit_ns;
    pp.stall = stall;
    // a bound on every job's layout: image + one A buffer (G.tc_smem), the
    // second A buffer and the stages at the largest source count
    const size_t budget = 227 * 1024 - (size_t)static_smem;
    const size_t a_max = 2048 * (size_t)((max_ns + 3) & ~1), s_max = 1024 * (size_t)max_ns;
    size_t need = 0;
    pp.depth = 0;
    pp.na = 1;
    for (int na = 2; na >= 1 && pp.depth == 0; --na)
        for (int depth = TC_MAX_DEPTH; depth >= 1; --depth) {
            const size_t m = (size_t)G.tc_smem + (na - 1) * a_max + depth * s_max;
            if (m <= budget) {
                pp.depth = depth;
                pp.na = na;
                need = m;
                break;
            }
        }
    if (pp.depth == 0)
        return fides_set_error(FIDES_ERR_UNSUPPORTED, "bconv tc: %d bytes of shared memory", G.tc_smem);
    const size_t half_sm = 228 * 1024 / 2 + 1;   // a second CTA must not fit
    size_t smem = std::max(need, half_sm > (size_t)static_smem + 1024 ? half_sm - static_smem - 1024 + 128 : 0);
    smem = std::min((smem + 127) & ~(size_t)127, budget);
    // CTAs per job: the fewest waves x (tiles per CTA + a CTA's fixed cost,
    // about three tiles: image copy, pipeline fill); one wave when the jobs
    // are fewer than the SMs, and with many jobs (batches) a split whose last
    // wave is full
    const int tiles = c->N / TC_M;
    int per_job = 1;
    long best = -1;
    for (int pj = 1; pj <= tiles; ++pj) {
        const long waves = ((long)G.njob * pj + c->sms - 1) / c->sms;
        const long cost = waves * ((tiles + pj - 1) / pj + 3);
        if (best < 0 || cost < best) {
            best = cost;
            per_job = pj;
        }
    }
    dim3 grid(per_job, G.njob), block(TC_THREADS);
    FIDES_LAUNCH_SMEM("k_bconv_tc", st, k_bconv_tc<BIG>, grid, block, smem, G, (const PrimeInfo *)c->d_prime,
                      (const TwPair *)c->d_c32, c->logN, pp, c->d_status);
    return fides_check_cuda(cudaGetLastError(), "bconv tc launch");
}

// limit_ns: the limit of every pipeline wait; stall: the self-test in which
// CTA (0, 0) never copies its first tile in (fides_ctx_selftest_conversion)
inline int launch_bconv_tc(const fides_ctx *c, const BConvArgs &G, int max_ns, int max_dst, cudaStream_t st,
                           u64 limit_ns = 2000000000ull, int stall = 0)
{
    return c->tc_big ? launch_bconv_tc_t<true>(c, G, max_ns, max_dst, st, limit_ns, stall)
                     : launch_bconv_tc_t<false>(c, G, max_ns, max_dst, st, limit_ns, stall);
}

}  // namespace
