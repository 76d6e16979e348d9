// Negacyclic NTT engine for sm_103a (Sec. III-F4).
//
// Convention: slot j of a limb holds a(psi^(2 brv(j) + 1)); the forward
// transform uses Cooley-Tukey butterflies (natural in, bit-reversed out) and
// the inverse Gentleman-Sande butterflies (bit-reversed in, natural out), so no
// explicit bit reversal is needed.  Stage s (m = 2^s blocks) of the forward
// transform pairs j and j + N/2^(s+1) and uses twiddle psi^brv(m + (j >> (logN-s))).
//
// Decomposition.  A CTA of 256 threads transforms a 4096-element tile held in
// registers (16 elements per thread) and shared memory:
//   * logN = 12: the whole limb is one tile (KIND 2, one pass);
//   * logN = 16: two passes as in the paper's hierarchical 2-D NTT -- a column
//     pass (KIND 0) runs stages 0..7 on 16 columns of stride 256, a row pass
//     (KIND 1) runs stages 8..15 on 16 contiguous rows of 256.  Four global
//     accesses per element, as in the paper.
// Inside a pass, stages are grouped four at a time ("rounds"): in a round every
// thread owns 16 elements whose local indices differ only in the round's four
// bits, so four radix-2 stages run in registers; rounds exchange data through
// shared memory (k-major for columns, XOR-swizzled rows otherwise, both free
// of bank conflicts).  Loads and stores are coalesced: where the thread-to-
// element map of the first/last round is strided, the tile is staged through
// shared memory instead.
//
// Arithmetic is lazy: values stay in [0, 2q) between butterflies (primes are
// below 2^61, so 4q fits in 64 bits); each butterfly costs one Shoup product.
// Prologue and epilogue functors let callers fuse element-wise work into the
// first load and the last store (Sec. III-F5 "Operation Fusions").
#pragma once

#include "fides_internal.cuh"

// k with its four bits [b, b+3] set to r and the other bits taken from u
__device__ __forceinline__ int kmap(int u, int r, int b)
{
    return ((u >> b) << (b + 4)) | (r << b) | (u & ((1 << b) - 1));
}

__device__ __forceinline__ void ct_bfly(u64 &x, u64 &y, const TwPair &w, u64 q, u64 q2)
{
    u64 t = mul_shoup(y, w, q);          // [0, 2q)
    u64 a = x;                            // [0, 2q)
    x = csub(a + t, q2);
    y = csub(a + q2 - t, q2);
}

__device__ __forceinline__ void gs_bfly(u64 &x, u64 &y, const TwPair &w, u64 q, u64 q2)
{
    u64 a = x, b = y;
    x = csub(a + b, q2);
    y = mul_shoup(a + q2 - b, w, q);
}

// ---- prologue functors: value of input element j, in [0, 2q) ----
struct ProSrc {
    __device__ __forceinline__ u64 operator()(const Job &J, u32 j, const PrimeInfo &) const { return J.src[j]; }
};
struct ProDst {
    __device__ __forceinline__ u64 operator()(const Job &J, u32 j, const PrimeInfo &) const { return J.dst[j]; }
};
// reduce a value of another prime's range (SwitchModulo of Rescale)
struct ProSwitchMod {
    __device__ __forceinline__ u64 operator()(const Job &J, u32 j, const PrimeInfo &p) const
    {
        return reduce64_lazy(J.src[j], p);
    }
};

// ---- epilogue functors: v in [0, 2q) ----
struct EpiLazy {
    __device__ __forceinline__ void operator()(const Job &J, u32 j, u64 v, const PrimeInfo &) const { J.dst[j] = v; }
};
struct EpiCanon {
    __device__ __forceinline__ void operator()(const Job &J, u32 j, u64 v, const PrimeInfo &p) const
    {
        J.dst[j] = csub(v, p.q);
    }
};
// out = c_i (aux - v) mod q_i, or out += that when the segment's mode is 1
// (ModDown with c = P^-1, Rescale with c = q_l^-1; Sec. III-F5).
struct EpiSubMul {
    const TwPair *cst;
    __device__ __forceinline__ void operator()(const Job &J, u32 j, u64 v, const PrimeInfo &p) const
    {
        u64 y = csub(v, p.q);
        u64 r = csub(mul_shoup(J.aux[j] + p.q - y, cst[J.prime], p.q), p.q);
        if (J.mode == 1) r = csub(r + J.out[j], p.q);
        J.out[j] = r;
    }
};

// KIND: 0 = column pass (16 strided columns), 1 = row pass (16 rows),
//       2 = whole limb (S == LOGN == 12).
// INV selects Gentleman-Sande stages in reverse order; NINV multiplies by
// N^-1 before the epilogue.
template <int LOGN, int S, int KIND, bool INV, bool NINV, class Pro, class Epi>
__global__ void __launch_bounds__(256) k_ntt(LimbSet set, const PrimeInfo *__restrict__ P,
                                             const TwPair *__restrict__ TW, Pro pro, Epi epi)
{
    constexpr int C = 4096 >> S;                  // sub-transforms per tile
    constexpr int R = S / 4;                      // rounds of four stages
    constexpr int S0 = (KIND == 1) ? (LOGN - S) : 0;
    constexpr int SH = LOGN - S;                  // column stride shift
    static_assert(S % 4 == 0 && C * (1 << S) == 4096, "tile shape");
    __shared__ u64 sm[4096];

    const int t = threadIdx.x;
    const Job J = get_job(set, blockIdx.y, 1 << LOGN);
    const PrimeInfo pr = P[J.prime];
    const TwPair *__restrict__ tw = TW + ((size_t)J.prime << LOGN);
    const u64 q = pr.q, q2 = pr.q2;

    int c, u;
    if (KIND == 0) { c = t % C; u = t / C; }
    else if (KIND == 1) { u = t & 15; c = t >> 4; }
    else { u = t; c = 0; }
    const int cbase = (KIND == 2) ? 0 : (int)blockIdx.x * C + c;

    auto gidx = [&](int cb, int k) -> u32 {
        if (KIND == 0) return (u32)(cb + (k << SH));
        if (KIND == 1) return (u32)((cb << S) + k);
        return (u32)k;
    };
    auto widx = [&](int cc, int k) -> int {
        if (KIND == 0) return k * C + cc;
        return cc * (1 << S) + (k ^ ((k >> 4) & 15));
    };

    u64 x[16];

    // ---------------- load ----------------
    if (!INV || KIND == 0) {
        const int b0 = INV ? 0 : S - 4;
#pragma unroll
        for (int r = 0; r < 16; ++r) x[r] = pro(J, gidx(cbase, kmap(u, r, b0)), pr);
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            int e = t + 256 * i;
            int cc = e >> S, k = e & ((1 << S) - 1);
            int cb = (KIND == 2) ? 0 : (int)blockIdx.x * C + cc;
            sm[widx(cc, k)] = pro(J, gidx(cb, k), pr);
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 16; ++r) x[r] = sm[widx(c, kmap(u, r, 0))];
    }

    // ---------------- rounds ----------------
#pragma unroll
    for (int rho = 0; rho < R; ++rho) {
        const int b = INV ? 4 * rho : S - 4 - 4 * rho;
        if (rho > 0) {
#pragma unroll
            for (int r = 0; r < 16; ++r) x[r] = sm[widx(c, kmap(u, r, b))];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int s = INV ? S0 + S - 1 - (4 * rho + a) : S0 + 4 * rho + a;
            const int h = INV ? (1 << a) : (8 >> a);
#pragma unroll
            for (int r = 0; r < 16; ++r) {
                if (r & h) continue;
                const u32 j = gidx(cbase, kmap(u, r, b));
                const TwPair w = tw[(1u << s) + (j >> (LOGN - s))];
                if (INV) gs_bfly(x[r], x[r + h], w, q, q2);
                else ct_bfly(x[r], x[r + h], w, q, q2);
            }
        }
        if (rho < R - 1) {
#pragma unroll
            for (int r = 0; r < 16; ++r) sm[widx(c, kmap(u, r, b))] = x[r];
            __syncthreads();
        }
    }

    // ---------------- store ----------------
    if (NINV) {
#pragma unroll
        for (int r = 0; r < 16; ++r) x[r] = mul_shoup(x[r], pr.ninv, pr.ninvp, q);
    }
    if (INV || KIND == 0) {
        const int bl = INV ? S - 4 : 0;
#pragma unroll
        for (int r = 0; r < 16; ++r) epi(J, gidx(cbase, kmap(u, r, bl)), x[r], pr);
    } else {
        if (R > 1) __syncthreads();   // every thread has read its last-round inputs
#pragma unroll
        for (int r = 0; r < 16; ++r) sm[widx(c, kmap(u, r, 0))] = x[r];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            int e = t + 256 * i;
            int cc = e >> S, k = e & ((1 << S) - 1);
            int cb = (KIND == 2) ? 0 : (int)blockIdx.x * C + cc;
            epi(J, gidx(cb, k), sm[widx(cc, k)], pr);
        }
    }
}

// Forward NTT of every limb of `set`: prologue `pro` on the input, epilogue
// `epi` on the output.  The intermediate of a two-pass transform is written
// to each job's dst.
template <class Pro, class Epi>
int ntt_forward(const fides_ctx *c, const LimbSet &set, Pro pro, Epi epi, cudaStream_t st)
{
    if (set.total == 0) return FIDES_OK;
    dim3 block(256);
    if (c->logN == 16) {
        dim3 grid(16, set.total);
        FIDES_LAUNCH("k_ntt_fwd_cols", st, k_ntt<16, 8, 0, false, false><<<grid, block, 0, st>>>(set, c->d_prime, c->d_tw, pro, EpiLazy{}));
        FIDES_LAUNCH("k_ntt_fwd_rows", st, k_ntt<16, 8, 1, false, false><<<grid, block, 0, st>>>(set, c->d_prime, c->d_tw, ProDst{}, epi));
    } else {
        dim3 grid(1, set.total);
        FIDES_LAUNCH("k_ntt_fwd_limb", st, k_ntt<12, 12, 2, false, false><<<grid, block, 0, st>>>(set, c->d_prime, c->d_tw, pro, epi));
    }
    return fides_check_cuda(cudaGetLastError(), "ntt forward launch");
}

template <class Pro, class Epi>
int ntt_inverse(const fides_ctx *c, const LimbSet &set, Pro pro, Epi epi, cudaStream_t st)
{
    if (set.total == 0) return FIDES_OK;
    dim3 block(256);
    if (c->logN == 16) {
        dim3 grid(16, set.total);
        FIDES_LAUNCH("k_ntt_inv_rows", st, k_ntt<16, 8, 1, true, false><<<grid, block, 0, st>>>(set, c->d_prime, c->d_itw, pro, EpiLazy{}));
        FIDES_LAUNCH("k_ntt_inv_cols", st, k_ntt<16, 8, 0, true, true><<<grid, block, 0, st>>>(set, c->d_prime, c->d_itw, ProDst{}, epi));
    } else {
        dim3 grid(1, set.total);
        FIDES_LAUNCH("k_ntt_inv_limb", st, k_ntt<12, 12, 2, true, true><<<grid, block, 0, st>>>(set, c->d_prime, c->d_itw, pro, epi));
    }
    return fides_check_cuda(cudaGetLastError(), "ntt inverse launch");
}
