// Negacyclic NTT engine for sm_103a (Sec. III-F4).
//
// Convention: slot j of a limb holds a(psi^(2 brv(j) + 1)); the forward
// transform uses Cooley-Tukey butterflies (natural in, bit-reversed out) and
// the inverse Gentleman-Sande butterflies (bit-reversed in, natural out), so no
// explicit bit reversal is needed.  Stage s (m = 2^s blocks) of the forward
// transform pairs j and j + N/2^(s+1) and uses twiddle psi^brv(m + (j >> (logN-s))).
//
// Decomposition.  A CTA transforms a tile held in registers (16 elements per
// thread) and shared memory:
//   * logN = 12: the whole limb is one tile of 256 threads (KIND 2, one pass);
//   * logN = 13..17: two passes as in the paper's hierarchical 2-D NTT -- a
//     column pass (KIND 0) runs the first S_col stages on CT columns of stride
//     2^(logN - S_col), a row pass (KIND 1) runs the other S_row stages on CT
//     contiguous rows (S_col, S_row = 7+6, 7+7, 8+7, 8+8, 9+8 for logN 13..17).
//     Four global accesses per element, as in the paper.  CT is 16, 8 or 4;
//     narrower tiles split a small launch into more CTAs so its last wave
//     costs less (the choice per pass and limb count is autotuned, see
//     ntt.cu).
// Inside a pass, stages are grouped four at a time ("rounds"): in a round every
// thread owns 16 elements whose local indices differ only in the round's four
// bits, so four radix-2 stages run in registers (a pass whose stage count is
// not a multiple of four ends with a partial round, see ntt_round); rounds exchange data through
// shared memory (k-major for columns, XOR-swizzled rows otherwise, both free
// of bank conflicts).  Loads and stores are coalesced: where the thread-to-
// element map of the first/last round is strided, the tile is staged through
// shared memory instead.  The column pass reads its 255 twiddles (shared by
// every column) from shared memory; the row pass reads per-row twiddles
// through L1.
//
// Twiddle index of a butterfly.  In round rho (bit offset b of the round's four
// bits in the local index k) the thread's elements are k(r) = X' | r << b | low
// bits, and the forward stage s = S0 + 4 rho + a of the lower element r uses
// index 2^s + (X << a) + (r >> (4 - a)); the inverse stage s = S0 + S - 1 -
// 4 rho - a uses 2^s + (X << (3 - a)) + (r >> (a + 1)).  X collects the bits of
// the global index above the round's bits (the row for row passes).
//
// Arithmetic is lazy (Harvey): forward values stay in [0, 6q) at round
// boundaries and [0, 8q) in between (one conditional subtraction every other
// stage), inverse values in [0, 2q); primes are below 2^61, so 8q < 2^64.
// Each butterfly costs one Shoup product, and at most one conditional
// subtraction.
// Prologue and epilogue functors let callers fuse element-wise work into the
// first load and the last store (Sec. III-F5 "Operation Fusions"); epilogues
// receive values in [0, 2q), except the raw intermediate store of a forward
// column pass, which keeps [0, 6q) (the row pass accepts it).
#pragma once

#include <type_traits>

#include "fides_internal.cuh"

// k with its four bits [b, b+3] set to r and the other bits taken from u
__device__ __forceinline__ int kmap(int u, int r, int b)
{
    return ((u >> b) << (b + 4)) | (r << b) | (u & ((1 << b) - 1));
}

// Forward butterfly, reducing x on every other stage only (red): with
// t = w y in [0, 2q), a reducing stage maps inputs in [0, 8q) to [0, 6q)
// (x -> csub(x, 4q) in [0, 4q)), a skipping one maps [0, 6q) to [0, 8q);
// 8q < 2^64 for primes below 2^61, and the Shoup product takes any 64-bit
// input.  Rounds start and end on [0, 6q).
// (red is a constant once the stage loop is unrolled)
__device__ __forceinline__ void ct_bfly(u64 &x, u64 &y, const TwPair &w, u64 q, u64 q2, u64 q4, bool red)
{
    u64 a = red ? csub(x, q4) : x;
    u64 t = mul_shoup(y, w, q);           // [0, 2q)
    x = a + t;
    y = a + q2 - t;
}

// Inverse butterfly: x, y in [0, 2q) -> x + y, (x - y) w in [0, 2q).
__device__ __forceinline__ void gs_bfly(u64 &x, u64 &y, const TwPair &w, u64 q, u64 q2)
{
    u64 a = x, b = y;
    x = csub(a + b, q2);
    y = mul_shoup(a + q2 - b, w, q);
}

// The last inverse stage (one twiddle w1) with the final scale c folded in:
// (x + y) c and (x - y) (w1 c), both in [0, 2q) -- two Shoup products in
// place of the stage's product, its subtraction and two scalings.
__device__ __forceinline__ void gs_bfly_scaled(u64 &x, u64 &y, const TwPair &c, const TwPair &cw, u64 q, u64 q2)
{
    u64 a = x, b = y;
    x = mul_shoup(a + b, c, q);
    y = mul_shoup(a + q2 - b, cw, q);
}

// ---- prologue functors: value of input element j, in [0, 4q) ----
struct ProSrc {
    __device__ __forceinline__ u64 operator()(const Job &J, u32 j, const PrimeInfo &) const { return J.src[j]; }
};
struct ProDst {
    __device__ __forceinline__ u64 operator()(const Job &J, u32 j, const PrimeInfo &) const { return J.dst[j]; }
};
// reduce a value of another prime's range (SwitchModulo of Rescale): the
// canonical representative v in [0, q_l), or, when the segment's g holds q_l
// (round-to-nearest Rescale), the centred one v - q_l for v > (q_l - 1) / 2.
struct ProSwitchMod {
    __device__ __forceinline__ u64 operator()(const Job &J, u32 j, const PrimeInfo &p) const
    {
        const u64 v = J.src[j];
        u64 r = reduce64_lazy(v, p);                                     // [0, 2q)
        if (J.g && v > (J.g >> 1)) r += p.q - csub(reduce64_lazy(J.g, p), p.q);   // v - q_l mod q, < 3q
        return r;
    }
};

// ModRaise (bootstrapping, Sec. III-F7): src is a coefficient of the limb
// modulo q_0 (canonical); its centred representative in (-q_0/2, q_0/2] is
// reduced modulo this limb's prime.  g holds q_0, cst[prime].w = q_0 mod q.
struct ProRaise {
    __device__ __forceinline__ u64 operator()(const Job &J, u32 j, const PrimeInfo &p) const
    {
        const u64 v = J.src[j];
        const u64 r = reduce64_lazy(v, p);                                  // [0, 2q)
        if (v > (J.g >> 1)) return csub(r + p.q - J.cst[J.prime].w, p.q2);  // v - q_0 mod q, in [0, 2q)
        return r;
    }
};

// Inverse-NTT prologue with a run-time variant (the segment's mode), which
// fuses the element-wise step that produces a key-switch input:
//   0: the input limb as is;
//   1: HMult tensor product (Table I): src / aux are limbs of ciphertexts a
//      and b (polynomial 1 at +pstride words); d0 = a0 b0 goes to out,
//      d1 = a0 b1 + a1 b0 to out + pstride, d2 = a1 b1 to side, and d2 is
//      transformed;
//   2: HRotate automorphism sigma_g in evaluation form (Sec. III-F1):
//      sigma_g(a)[j] = a[brv(((2 brv(j) + 1) g mod 2N - 1) / 2)]; sigma_g(c0)
//      goes to out, sigma_g(c1) to side, and sigma_g(c1) is transformed.
// A prologue in two steps, so that the kernel can issue the loads of several
// elements before it computes and stores any of them (each call reads up to
// four words and stores up to three): load() reads what element j needs,
// apply() computes, stores the side outputs and returns the value.  Outputs
// may not alias inputs.  The operands are read with coherent loads, not the
// non-coherent path (ld.global.nc): PTX allows that path only for data that
// stays unchanged for the kernel's whole lifetime, and under programmatic
// dependent launch a kernel starts while the one before it still writes.
struct ProPrep {
    int logN;
    __device__ __forceinline__ void load(const Job &J, u32 j, u64 (&v)[4]) const
    {
        const size_t S = (size_t)J.pstride;
        if (J.mode == 0) {
            v[0] = J.src[j];
        } else if (J.mode == 1) {
            v[0] = J.src[j];
            v[1] = J.src[S + j];
            v[2] = J.aux[j];
            v[3] = J.aux[S + j];
        } else {
            const u32 rj = __brev(j) >> (32 - logN);
            const u64 e = ((2 * (u64)rj + 1) * J.g) & ((2ull << logN) - 1);
            const u32 src = __brev((u32)((e - 1) >> 1)) >> (32 - logN);
            v[0] = J.src[src];
            v[1] = J.src[S + src];
        }
    }
    __device__ __forceinline__ u64 apply(const Job &J, u32 j, const u64 (&v)[4], const PrimeInfo &p) const
    {
        if (J.mode == 0) return v[0];
        const size_t S = (size_t)J.pstride;
        if (J.mode == 1) {
            J.out[j] = mul_mod_small(v[0], v[2], p);
            U128 m = {0, 0};
            mac128(m, v[0], v[3]);
            mac128(m, v[1], v[2]);
            J.out[S + j] = csub(csub(reduce_prod(m.hi, m.lo, p), p.q2), p.q);
            const u64 d2 = mul_mod_small(v[1], v[3], p);
            J.side[j] = d2;
            return d2;
        }
        J.out[j] = v[0];
        J.side[j] = v[1];
        return v[1];
    }
    __device__ __forceinline__ u64 operator()(const Job &J, u32 j, const PrimeInfo &p) const
    {
        u64 v[4];
        load(J, j, v);
        return apply(J, j, v, p);
    }
};

// The plain inverse-NTT input (every segment of mode 0): the row pass issues
// all sixteen of a thread's loads before it stores any of them to shared
// memory (coherent loads, as for ProPrep).
struct ProPlain {
    __device__ __forceinline__ u64 operator()(const Job &J, u32 j, const PrimeInfo &) const { return J.src[j]; }
};

// ---- epilogue functors ----
// Each epilogue has a load step (the global reads it needs for element j) and
// a store step, so that the kernel can issue the loads of several elements
// before computing any of them.
// intermediate store of the first pass (raw: forward values stay in [0, 6q))
struct EpiLazy {
    static constexpr bool kRaw = true;
    __device__ __forceinline__ void load(const Job &, u32, u64 &, u64 &) const {}
    __device__ __forceinline__ void store(const Job &J, u32 j, u64 v, u64, u64, const PrimeInfo &) const
    {
        J.dst[j] = v;
    }
};
struct EpiCanon {
    static constexpr bool kRaw = false;
    __device__ __forceinline__ void load(const Job &, u32, u64 &, u64 &) const {}
    __device__ __forceinline__ void store(const Job &J, u32 j, u64 v, u64, u64, const PrimeInfo &p) const
    {
        J.dst[j] = csub(v, p.q);
    }
};
// out = c_i (aux - v) mod q_i, or out += that when the segment's mode is 1,
// with c from the segment's constant table (ModDown with c = P^-1, Rescale
// with c = q_l^-1; Sec. III-F5).
struct EpiSubMul {
    static constexpr bool kRaw = false;
    __device__ __forceinline__ void load(const Job &J, u32 j, u64 &a, u64 &o) const
    {
        a = J.aux[j];
        o = J.mode == 1 ? J.out[j] : 0;
    }
    __device__ __forceinline__ void store(const Job &J, u32 j, u64 v, u64 a, u64 o, const PrimeInfo &p) const
    {
        u64 y = csub(v, p.q);
        u64 r = csub(mul_shoup(a + p.q - y, J.cst[J.prime], p.q), p.q);
        if (J.mode == 1) r = csub(r + o, p.q);
        J.out[j] = r;
    }
};

// As EpiSubMul, but a segment of mode 2 adds side[sigma_g(j)], the
// automorphism of another polynomial gathered in evaluation form (the
// ModDown of a hoisted rotation adds sigma(c0) this way).  A separate functor
// so that the common epilogue keeps its registers.
struct EpiSubMulRot {
    static constexpr bool kRaw = false;
    int logN;
    __device__ __forceinline__ void load(const Job &J, u32 j, u64 &a, u64 &o) const
    {
        a = J.aux[j];
        o = 0;
        if (J.mode == 2) {
            const u32 rj = __brev(j) >> (32 - logN);
            const u64 e = ((2 * (u64)rj + 1) * J.g) & ((2ull << logN) - 1);
            o = J.side[__brev((u32)((e - 1) >> 1)) >> (32 - logN)];
        }
    }
    __device__ __forceinline__ void store(const Job &J, u32 j, u64 v, u64 a, u64 o, const PrimeInfo &p) const
    {
        u64 y = csub(v, p.q);
        u64 r = csub(mul_shoup(a + p.q - y, J.cst[J.prime], p.q), p.q);
        if (J.mode == 2) r = csub(r + o, p.q);
        J.out[j] = r;
    }
};

// HMult followed by Rescale in one pass (fides_hmult_rescale).  By linearity
// of the NTT, Rescale(HMult) gives for every remaining limb i < l
//   res_i = q_l^-1 (d_i + P^-1 acc_i - NTT(P^-1 conv_i + [last]_{q_i})),
// with d the tensor product, acc the key inner product, conv the ModDown
// conversion (coefficient form, < 4q) and last the coefficient form of the
// dropped limb l of the HMult result.  The segment's src is `last` (src_step
// 0: one limb for every limb of the run), dst holds conv_i (the pass works in
// place), aux = acc_i, side = d_i, out = res_i; cst holds two constants per
// prime: cst[2i] = P^-1 mod q_i, cst[2i + 1] = q_l^-1 mod q_i.  When the
// segment's g holds q_l (round-to-nearest), `last` is lifted from its centred
// representative, as ProSwitchMod does.
struct ProHmRs {
    __device__ __forceinline__ u64 operator()(const Job &J, u32 j, const PrimeInfo &p) const
    {
        const u64 x = mul_shoup(J.dst[j], J.cst[2 * J.prime], p.q);   // [0, 2q)
        const u64 v = J.src[j];
        u64 r = reduce64_lazy(v, p);                                  // [0, 2q)
        if (J.g && v > (J.g >> 1)) r = csub(r + p.q - csub(reduce64_lazy(J.g, p), p.q), p.q2);   // v - q_l, [0, 2q)
        return x + r;                                                 // [0, 4q)
    }
};
struct EpiHmRs {
    static constexpr bool kRaw = false;
    __device__ __forceinline__ void load(const Job &J, u32 j, u64 &a, u64 &o) const
    {
        a = J.aux[j];
        o = J.side[j];
    }
    __device__ __forceinline__ void store(const Job &J, u32 j, u64 v, u64 a, u64 o, const PrimeInfo &p) const
    {
        const u64 y = csub(v, p.q);
        const u64 r = o + mul_shoup(a, J.cst[2 * J.prime], p.q) + p.q - y;   // < 4q
        J.out[j] = csub(mul_shoup(r, J.cst[2 * J.prime + 1], p.q), p.q);
    }
};

// One round of up to four radix-2 stages on the thread's 16 registers, whose
// local indices differ in the four bits [B, B+3] (the round's window).  A full
// round runs the four stages of the window; the last round of a pass whose
// stage count is not a multiple of four runs only the stages a = A0..3 (its
// window is the lowest four bits for a forward pass, the highest four for an
// inverse one, and the window bits an earlier round transformed act as
// independent lanes).  X: the global-index bits above the window; TWS:
// twiddles come from shared memory instead of global.
// SCALED: an inverse pass that ends with stage 0 multiplies by the final
// constant there (gs_bfly_scaled with c, cw = c w1) instead of after it.
template <bool INV, int S0, int S, int B, int A0, bool TWS, bool SCALED>
__device__ __forceinline__ void ntt_round(u64 (&x)[16], int X, const TwPair *__restrict__ tw,
                                          const TwPair *stw, u64 q, u64 q2, const TwPair &c, const TwPair &cw)
{
    const u64 q4 = 2 * q2;
#pragma unroll
    for (int a = A0; a < 4; ++a) {
        const int s = INV ? S0 + S - 1 - B - a : S0 + (S - 4 - B) + a;
        const int h = INV ? (1 << a) : (8 >> a);
        const int base = (1 << s) + (INV ? (X << (3 - a)) : (X << a));
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            if (r & h) continue;
            if (INV && SCALED && s == 0) {
                gs_bfly_scaled(x[r], x[r + h], c, cw, q, q2);
                continue;
            }
            const int idx = base + (INV ? (r >> (a + 1)) : (r >> (4 - a)));
            const TwPair w = TWS ? stw[idx] : tw[idx];
            if (INV) gs_bfly(x[r], x[r + h], w, q, q2);
            else ct_bfly(x[r], x[r + h], w, q, q2, q4, (a & 1) != 0);   // stages a = 1, 3 reduce
        }
    }
}

// Window and first stage of round rho of a pass of S stages (see ntt_round).
template <int S, bool INV>
__host__ __device__ constexpr int round_window(int rho)
{
    return (rho == (S + 3) / 4 - 1 && S % 4 != 0) ? (INV ? S - 4 : 0) : (INV ? 4 * rho : S - 4 - 4 * rho);
}
template <int S>
__host__ __device__ constexpr int round_first(int rho)
{
    return (rho == (S + 3) / 4 - 1 && S % 4 != 0) ? 4 - S % 4 : 0;
}

// Threads of a tile: 16 elements each.
template <int S, int KIND, int CT>
__host__ __device__ constexpr int ntt_threads()
{
    return ((KIND == 2 ? 1 : CT) << S) / 16;
}

// KIND: 0 = column pass (CT strided columns of 2^S elements, stages 0..S-1),
//       1 = row pass (CT contiguous rows of 2^S elements, stages LOGN-S..LOGN-1),
//       2 = whole limb (S == LOGN == 12, 256 threads; CT ignored).
// INV selects Gentleman-Sande stages in reverse order; NINV applies N^-1 (or
// the segment's constant) within the last stage, before the epilogue.  MINB
// is the resident-CTA target per SM.
template <int LOGN, int S, int KIND, bool INV, bool NINV, int CT, int MINB, class Pro, class Epi>
__global__ void __launch_bounds__(ntt_threads<S, KIND, CT>(), MINB)
    k_ntt(LimbSet set, const PrimeInfo *__restrict__ P, const TwPair *__restrict__ TW, Pro pro, Epi epi)
{
    constexpr int C = (KIND == 2) ? 1 : CT;            // sub-transforms per tile
    constexpr int THREADS = ntt_threads<S, KIND, CT>();
    constexpr int RT = (1 << S) / 16;                  // threads per sub-transform
    constexpr int R = (S + 3) / 4;                     // rounds (the last one may be partial)
    constexpr int S0 = (KIND == 1) ? (LOGN - S) : 0;
    constexpr int SH = LOGN - S;                       // column stride shift
    constexpr bool TWS = (KIND == 0);                  // column twiddles staged in shared memory
    static_assert(S >= 5 && R <= 3, "tile shape");
    static_assert(!NINV || (INV && KIND != 1), "the final scale is applied in stage 0, which only this pass holds");
    __shared__ u64 sm[C << S];
    __shared__ TwPair stw[TWS ? (1 << S) : 1];

    // the job table, the primes and the twiddles are the context's or the
    // host's: read (and the column twiddles staged) before waiting for the
    // previous kernel, whose output is read only below
    pdl_trigger();
    const int t = threadIdx.x;
    const Job J = get_job(set, blockIdx.y, 1 << LOGN);
    const PrimeInfo pr = P[J.prime];
    const TwPair *__restrict__ tw = TW + ((size_t)J.prime << LOGN);
    const u64 q = pr.q, q2 = pr.q2;
    if (TWS) {
        for (int i = t; i < (1 << S); i += THREADS) stw[i] = tw[i];
    }
    pdl_wait();

    int c, u;
    if (KIND == 0) { c = t % C; u = t / C; }
    else if (KIND == 1) { u = t % RT; c = t / RT; }
    else { u = t; c = 0; }
    const int cbase = (KIND == 2) ? 0 : (int)blockIdx.x * C + c;   // column (KIND 0) or row (KIND 1)

    auto gidx = [&](int cb, int k) -> u32 {
        if (KIND == 0) return (u32)(cb + (k << SH));
        if (KIND == 1) return (u32)((cb << S) + k);
        return (u32)k;
    };
    auto widx = [&](int cc, int k) -> int {
        if (KIND == 0) return k * C + cc;
        return cc * (1 << S) + (k ^ ((k >> 4) & 15));
    };
    // the global-index bits above a round's window of four bits starting at b
    auto Xof = [&](int b) -> int { return (KIND == 1 ? (cbase << (S - 4 - b)) : 0) | (u >> b); };

    u64 x[16];

    // ---------------- load ----------------
    if (!INV || KIND == 0) {
        const int b0 = INV ? 0 : S - 4;
#pragma unroll
        for (int r = 0; r < 16; ++r) x[r] = pro(J, gidx(cbase, kmap(u, r, b0)), pr);
        if (TWS) __syncthreads();
    } else if constexpr (std::is_same<Pro, ProPlain>::value) {
        // all sixteen loads in flight before the first shared-memory store
        u64 v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int e = t + THREADS * i;
            const int cc = e >> S, k = e & ((1 << S) - 1);
            const int cb = (KIND == 2) ? 0 : (int)blockIdx.x * C + cc;
            v[i] = pro(J, gidx(cb, k), pr);
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int e = t + THREADS * i;
            sm[widx(e >> S, e & ((1 << S) - 1))] = v[i];
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 16; ++r) x[r] = sm[widx(c, kmap(u, r, 0))];
    } else if constexpr (std::is_same<Pro, ProPrep>::value) {
        // four elements' loads in flight before any of them is computed
#pragma unroll
        for (int g = 0; g < 16; g += 4) {
            u32 jj[4];
            int ww[4];
            u64 v[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int e = t + THREADS * (g + i);
                const int cc = e >> S, k = e & ((1 << S) - 1);
                const int cb = (KIND == 2) ? 0 : (int)blockIdx.x * C + cc;
                jj[i] = gidx(cb, k);
                ww[i] = widx(cc, k);
                pro.load(J, jj[i], v[i]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) sm[ww[i]] = pro.apply(J, jj[i], v[i], pr);
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 16; ++r) x[r] = sm[widx(c, kmap(u, r, 0))];
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            int e = t + THREADS * i;
            int cc = e >> S, k = e & ((1 << S) - 1);
            int cb = (KIND == 2) ? 0 : (int)blockIdx.x * C + cc;
            sm[widx(cc, k)] = pro(J, gidx(cb, k), pr);
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 16; ++r) x[r] = sm[widx(c, kmap(u, r, 0))];
    }

    // The final constant of an inverse pass (NINV): N^-1, or the segment's
    // combined constant (N^-1 times the qhat^-1 of the base conversion that
    // reads this output, Eq. 1), with its product by the last stage's twiddle;
    // applied in that stage (gs_bfly_scaled).
    TwPair nc = {0, 0}, nw = {0, 0};
    if (NINV) {
        if (J.cst) {
            nc = J.cst[2 * J.prime];
            nw = J.cst[2 * J.prime + 1];
        } else {
            nc = TwPair{pr.ninv, pr.ninvp};
            nw = TwPair{pr.ninvw, pr.ninvwp};
        }
    }

    // ---------------- rounds ----------------
#define FIDES_NTT_ROUND(RHO)                                                                 \
    if (RHO < R) {                                                                           \
        constexpr int b = round_window<S, INV>(RHO < R ? RHO : 0);                          \
        if (RHO > 0) {                                                                       \
            _Pragma("unroll") for (int r = 0; r < 16; ++r) x[r] = sm[widx(c, kmap(u, r, b))]; \
        }                                                                                    \
        ntt_round<INV, S0, S, b, round_first<S>(RHO < R ? RHO : 0), TWS, NINV>(x, Xof(b), tw, stw, q, q2, nc, nw); \
        if (RHO < R - 1) {                                                                   \
            _Pragma("unroll") for (int r = 0; r < 16; ++r) sm[widx(c, kmap(u, r, b))] = x[r]; \
            __syncthreads();                                                                 \
        }                                                                                    \
    }
    FIDES_NTT_ROUND(0)
    FIDES_NTT_ROUND(1)
    FIDES_NTT_ROUND(2)
#undef FIDES_NTT_ROUND

    // ---------------- store ----------------
    if (!INV && !Epi::kRaw) {
#pragma unroll
        for (int r = 0; r < 16; ++r) x[r] = csub(csub(x[r], 2 * q2), q2);   // [0, 6q) -> [0, 2q)
    }
    if (INV || KIND == 0) {
        const int bl = INV ? S - 4 : 0;
#pragma unroll
        for (int h = 0; h < 16; h += 8) {
            u64 pa[8], po[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) epi.load(J, gidx(cbase, kmap(u, h + r, bl)), pa[r], po[r]);
#pragma unroll
            for (int r = 0; r < 8; ++r) epi.store(J, gidx(cbase, kmap(u, h + r, bl)), x[h + r], pa[r], po[r], pr);
        }
    } else {
        __syncthreads();   // the last round's shared-memory reads are done
#pragma unroll
        for (int r = 0; r < 16; ++r) sm[widx(c, kmap(u, r, 0))] = x[r];
        __syncthreads();
#pragma unroll
        for (int h = 0; h < 16; h += 8) {
            u64 pa[8], po[8];
            u32 jj[8];
            int ww[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int e = t + THREADS * (h + i);
                const int cc = e >> S, k = e & ((1 << S) - 1);
                const int cb = (KIND == 2) ? 0 : (int)blockIdx.x * C + cc;
                jj[i] = gidx(cb, k);
                ww[i] = widx(cc, k);
                epi.load(J, jj[i], pa[i], po[i]);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) epi.store(J, jj[i], sm[ww[i]], pa[i], po[i], pr);
        }
    }
}

// ---------------------------------------------------------------------------
// Launchers (ntt.cu).  Forward: prologue on the input, the intermediate of a
// two-pass transform in each job's dst, epilogue on the output.  Inverse:
// includes N^-1.
// ---------------------------------------------------------------------------
int ntt_fwd_canon(const fides_ctx *c, const LimbSet &set, cudaStream_t st);           // ProSrc, EpiCanon
int ntt_fwd_submul(const fides_ctx *c, const LimbSet &set, cudaStream_t st);          // ProSrc, EpiSubMul
int ntt_fwd_switch_submul(const fides_ctx *c, const LimbSet &set, cudaStream_t st);   // ProSwitchMod, EpiSubMul
int ntt_fwd_submul_rot(const fides_ctx *c, const LimbSet &set, cudaStream_t st);      // ProSrc, EpiSubMulRot
int ntt_fwd_raise(const fides_ctx *c, const LimbSet &set, cudaStream_t st);           // ProRaise, EpiCanon
int ntt_fwd_hmrs(const fides_ctx *c, const LimbSet &set, cudaStream_t st);            // ProHmRs, EpiHmRs
int ntt_inv_canon(const fides_ctx *c, const LimbSet &set, cudaStream_t st);           // ProPrep (ProPlain), EpiCanon

inline int ntt_forward(const fides_ctx *c, const LimbSet &s, ProSrc, EpiCanon, cudaStream_t st)
{
    return ntt_fwd_canon(c, s, st);
}
inline int ntt_forward(const fides_ctx *c, const LimbSet &s, ProSrc, EpiSubMul, cudaStream_t st)
{
    return ntt_fwd_submul(c, s, st);
}
inline int ntt_forward(const fides_ctx *c, const LimbSet &s, ProSwitchMod, EpiSubMul, cudaStream_t st)
{
    return ntt_fwd_switch_submul(c, s, st);
}
inline int ntt_forward(const fides_ctx *c, const LimbSet &s, ProSrc, EpiSubMulRot, cudaStream_t st)
{
    return ntt_fwd_submul_rot(c, s, st);
}
inline int ntt_forward(const fides_ctx *c, const LimbSet &s, ProRaise, EpiCanon, cudaStream_t st)
{
    return ntt_fwd_raise(c, s, st);
}
inline int ntt_forward(const fides_ctx *c, const LimbSet &s, ProHmRs, EpiHmRs, cudaStream_t st)
{
    return ntt_fwd_hmrs(c, s, st);
}
inline int ntt_inverse(const fides_ctx *c, const LimbSet &s, ProSrc, EpiCanon, cudaStream_t st)
{
    return ntt_inv_canon(c, s, st);
}

// Default NTT tile variant of each pass kind for each limb count (ntt.cu).
void ntt_default_variants(fides_ctx *c);
