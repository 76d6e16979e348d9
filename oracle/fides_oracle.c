/*
 * Plain CPU oracle for the CKKS hybrid key-switching path described in
 * "FIDESlib: A Fully-Fledged Open-Source FHE Library for Efficient CKKS on
 * GPUs" (arXiv 2507.04775).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file.  It shares no code, header,
 * table or constant generator with the CUDA library; the two agree only
 * because both follow the same definitions.
 *
 * Every modular product is ((unsigned __int128)a * b) % q, every transform is
 * the textbook one, and nothing is fused, blocked or reordered beyond what the
 * definition states.  Loops over limbs carry an OpenMP pragma (independent
 * limbs, same arithmetic), so the same code can be timed on one core or on all
 * host cores.
 *
 * Layout: a polynomial with n limbs is a limb-major array u64[n][N]; limb i of
 * a ciphertext-level polynomial lives modulo q_i, and the K special limbs of an
 * extended polynomial follow the q limbs.  All residues are canonical [0, q).
 *
 * Parity status: every function below is pinned by the tests in
 * tests/test_oracle_pins.py (closed forms, brute force on tiny inputs,
 * big-integer CRT identities, decryption-error bounds).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <omp.h>

typedef uint64_t u64;
typedef int64_t i64;
typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------
 * Modular arithmetic by definition (Sec. III-F2 "Modular arithmetic": the
 * result of a product must be brought back to [0, p); here with a plain %).
 * ---------------------------------------------------------------------- */
static u64 mul_mod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static u64 add_mod(u64 a, u64 b, u64 q) { return (u64)(((u128)a + b) % q); }
static u64 sub_mod(u64 a, u64 b, u64 q) { return (u64)(((u128)(a % q) + q - (b % q)) % q); }

static u64 pow_mod(u64 a, u64 e, u64 q)
{
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mul_mod(r, a, q);
        a = mul_mod(a, a, q);
        e >>= 1;
    }
    return r;
}

/* inverse modulo a prime by Fermat's little theorem */
static u64 inv_mod(u64 a, u64 q) { return pow_mod(a, q - 2, q); }

static u64 neg_mod(u64 a, u64 q) { a %= q; return a ? q - a : 0; }

/* a signed small integer as a residue modulo q */
static u64 from_signed(i64 v, u64 q)
{
    if (v >= 0) return (u64)v % q;
    u64 m = (u64)(-(v + 1)) + 1;      /* |v| without overflow */
    return neg_mod(m % q, q);
}

u64 or_mul_mod(u64 a, u64 b, u64 q) { return mul_mod(a, b, q); }
u64 or_pow_mod(u64 a, u64 e, u64 q) { return pow_mod(a, e, q); }

/* ------------------------------------------------------------------------
 * Primes: deterministic Miller-Rabin with the first twelve prime bases, which
 * is exact for every n < 3.3e24 (so for every 64-bit n).
 * ---------------------------------------------------------------------- */
int or_is_prime(u64 n)
{
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n % bases[i] == 0) return n == bases[i];
    }
    u64 d = n - 1;
    int r = 0;
    while ((d & 1) == 0) { d >>= 1; r++; }
    for (int i = 0; i < 12; i++) {
        u64 x = pow_mod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int witness = 1;
        for (int k = 1; k < r; k++) {
            x = mul_mod(x, x, n);
            if (x == n - 1) { witness = 0; break; }
        }
        if (witness) return 0;
    }
    return 1;
}

/*
 * NTT-friendly primes (Sec. II, Table II: q_i ~ Delta, word-sized moduli):
 * walk downward from 2^bits over q = 1 (mod 2N), keep primes not in
 * `exclude`, in the order met.  Returns how many were found.
 */
int or_find_primes(int logN, int bits, int count, const u64 *exclude, int n_exclude, u64 *out)
{
    if (bits < logN + 2 || bits > 62 || count < 0) return -1;
    u64 step = (u64)2 << logN;
    u64 q = ((u64)1 << bits) - step + 1;
    int found = 0;
    while (found < count && q > step) {
        int skip = 0;
        for (int i = 0; i < n_exclude; i++) if (exclude[i] == q) skip = 1;
        if (!skip && or_is_prime(q)) out[found++] = q;
        q -= step;
    }
    return found;
}

/* distinct prime factors of n by trial division */
static int prime_factors(u64 n, u64 *f)
{
    int k = 0;
    for (u64 p = 2; p * p <= n; p += (p == 2 ? 1 : 2)) {
        if (n % p == 0) {
            f[k++] = p;
            while (n % p == 0) n /= p;
        }
    }
    if (n > 1) f[k++] = n;
    return k;
}

/* smallest generator of the multiplicative group modulo a prime q */
u64 or_smallest_generator(u64 q)
{
    u64 f[64];
    int k = prime_factors(q - 1, f);
    for (u64 g = 2; g < q; g++) {
        int ok = 1;
        for (int i = 0; i < k && ok; i++) if (pow_mod(g, (q - 1) / f[i], q) == 1) ok = 0;
        if (ok) return g;
    }
    return 0;
}

/* bit reversal of the low `bits` bits */
static u64 brv(u64 x, int bits)
{
    u64 r = 0;
    for (int i = 0; i < bits; i++) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

/* ------------------------------------------------------------------------
 * Context: the primes and the per-prime constants the definitions need
 * (Sec. III-E "Precomputation" lists the same kind of values).
 * ---------------------------------------------------------------------- */
typedef struct {
    int logN;
    u64 N;
    int nq, nk, dnum, alpha;
    u64 *primes;     /* nq q-primes then nk special p-primes */
    u64 *psi;        /* psi_i: primitive 2N-th root modulo prime i */
    u64 *psi_brv;    /* [np][N]: psi^brv(k) */
    u64 *ipsi_brv;   /* [np][N]: psi^-brv(k) */
    u64 *n_inv;      /* N^-1 mod prime i */
    int nearest;     /* rounding of ModDown and Rescale: 0 floor, 1 nearest (or_ctx_set_rounding) */
} or_ctx;

/* Thread count of the OpenMP loops over limbs and digits, for timing the
 * oracle on one core or on all of them; no result depends on it.  Returns the
 * count now in effect. */
int or_set_threads(int n)
{
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
}

void or_ctx_free(or_ctx *c)
{
    if (!c) return;
    free(c->primes); free(c->psi); free(c->psi_brv); free(c->ipsi_brv); free(c->n_inv);
    free(c);
}

/*
 * psi (Table II: the 2N-th root of unity used by the (i)NTT).  The paper does
 * not say which root; this oracle reads it as g^((q-1)/2N) with g the
 * smallest generator of Z_q^*.
 */
or_ctx *or_ctx_create(int logN, int nq, int nk, int dnum, const u64 *primes)
{
    if (logN < 1 || logN > 17 || nq < 1 || nk < 1 || dnum < 1 || dnum > nq) return NULL;
    or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
    int np = nq + nk;
    c->logN = logN;
    c->N = (u64)1 << logN;
    c->nq = nq; c->nk = nk; c->dnum = dnum;
    c->alpha = (nq + dnum - 1) / dnum;
    c->primes = (u64 *)malloc(sizeof(u64) * np);
    c->psi = (u64 *)malloc(sizeof(u64) * np);
    c->n_inv = (u64 *)malloc(sizeof(u64) * np);
    c->psi_brv = (u64 *)malloc(sizeof(u64) * np * c->N);
    c->ipsi_brv = (u64 *)malloc(sizeof(u64) * np * c->N);
    memcpy(c->primes, primes, sizeof(u64) * np);
    for (int i = 0; i < np; i++) {
        u64 q = primes[i];
        if (!or_is_prime(q) || (q - 1) % (2 * c->N) != 0) { or_ctx_free(c); return NULL; }
        u64 g = or_smallest_generator(q);
        u64 psi = pow_mod(g, (q - 1) / (2 * c->N), q);
        u64 ipsi = inv_mod(psi, q);
        c->psi[i] = psi;
        c->n_inv[i] = inv_mod(c->N % q, q);
        for (u64 k = 0; k < c->N; k++) {
            u64 e = brv(k, logN);
            c->psi_brv[i * c->N + k] = pow_mod(psi, e, q);
            c->ipsi_brv[i * c->N + k] = pow_mod(ipsi, e, q);
        }
    }
    return c;
}

u64 or_ctx_psi(const or_ctx *c, int pi) { return c->psi[pi]; }

/*
 * Rounding of the two divisions of the path (the paper's ModDown and Rescale
 * fusions, Sec. III-F5, state the formulas without a rounding offset):
 * 0 = floor, the literal reading (canonical representatives); 1 = nearest
 * (centred representatives: ModDown converts the centred residues of the
 * special limbs, Rescale lifts the centred residue of the dropped limb).
 */
void or_ctx_set_rounding(or_ctx *c, int nearest) { c->nearest = nearest ? 1 : 0; }
int or_ctx_alpha(const or_ctx *c) { return c->alpha; }

/* prime index of limb z of an extended polynomial over q_0..q_{nl-1}, p_0.. */
static int ext_prime(const or_ctx *c, int nl, int z) { return z < nl ? z : c->nq + (z - nl); }

/* ------------------------------------------------------------------------
 * NTT (Sec. III-F4).  Evaluation slot j of a limb holds a(psi^(2 brv(j) + 1))
 * (forward output in bit-reversed order, inverse input in bit-reversed order).
 * ---------------------------------------------------------------------- */

/* the definition, O(N^2): out[j] = sum_i a_i psi^((2 brv(j) + 1) i) */
void or_ntt_naive(const or_ctx *c, int pi, const u64 *a, u64 *out)
{
    u64 q = c->primes[pi], N = c->N;
    for (u64 j = 0; j < N; j++) {
        u64 root = pow_mod(c->psi[pi], 2 * brv(j, c->logN) + 1, q);
        u64 acc = 0, x = 1;
        for (u64 i = 0; i < N; i++) {
            acc = add_mod(acc, mul_mod(a[i], x, q), q);
            x = mul_mod(x, root, q);
        }
        out[j] = acc;
    }
}

/* the definition of the inverse: a_i = N^-1 sum_j A_j psi^(-(2 brv(j) + 1) i) */
void or_intt_naive(const or_ctx *c, int pi, const u64 *A, u64 *out)
{
    u64 q = c->primes[pi], N = c->N;
    u64 ipsi = inv_mod(c->psi[pi], q);
    for (u64 i = 0; i < N; i++) out[i] = 0;
    for (u64 j = 0; j < N; j++) {
        u64 root = pow_mod(ipsi, 2 * brv(j, c->logN) + 1, q);
        u64 x = 1;
        for (u64 i = 0; i < N; i++) {
            out[i] = add_mod(out[i], mul_mod(A[j], x, q), q);
            x = mul_mod(x, root, q);
        }
    }
    for (u64 i = 0; i < N; i++) out[i] = mul_mod(out[i], c->n_inv[pi], q);
}

/*
 * Textbook radix-2 negacyclic NTT, in place: Cooley-Tukey butterflies,
 * natural-order input, bit-reversed output (Sec. III-F4).  Stage m has m
 * blocks of 2t elements; block i uses twiddle psi^brv(m + i).
 */
void or_ntt(const or_ctx *c, int pi, u64 *a)
{
    u64 q = c->primes[pi], N = c->N;
    const u64 *w = c->psi_brv + (u64)pi * N;
    u64 t = N;
    for (u64 m = 1; m < N; m <<= 1) {
        t >>= 1;
        for (u64 i = 0; i < m; i++) {
            u64 W = w[m + i];
            for (u64 j = 2 * i * t; j < 2 * i * t + t; j++) {
                u64 U = a[j], V = mul_mod(a[j + t], W, q);
                a[j] = add_mod(U, V, q);
                a[j + t] = sub_mod(U, V, q);
            }
        }
    }
}

/*
 * Textbook radix-2 inverse: Gentleman-Sande butterflies, bit-reversed input,
 * natural-order output, then the N^-1 scaling (Sec. III-F4).  Each stage undoes
 * the forward stage with the same (m, i): (U, V) <- (U + V, (U - V) psi^-brv(m+i)).
 */
void or_intt(const or_ctx *c, int pi, u64 *a)
{
    u64 q = c->primes[pi], N = c->N;
    const u64 *w = c->ipsi_brv + (u64)pi * N;
    u64 t = 1;
    for (u64 m = N >> 1; m >= 1; m >>= 1) {
        for (u64 i = 0; i < m; i++) {
            u64 W = w[m + i];
            for (u64 j = 2 * i * t; j < 2 * i * t + t; j++) {
                u64 U = a[j], V = a[j + t];
                a[j] = add_mod(U, V, q);
                a[j + t] = mul_mod(sub_mod(U, V, q), W, q);
            }
        }
        t <<= 1;
    }
    for (u64 j = 0; j < N; j++) a[j] = mul_mod(a[j], c->n_inv[pi], q);
}

/* batched helpers: limbs z0..z0+n-1 of `a`, limb z under prime pidx[z] */
void or_ntt_limbs(const or_ctx *c, u64 *a, const int *pidx, int n)
{
    #pragma omp parallel for schedule(dynamic)
    for (int z = 0; z < n; z++) or_ntt(c, pidx[z], a + (u64)z * c->N);
}

void or_intt_limbs(const or_ctx *c, u64 *a, const int *pidx, int n)
{
    #pragma omp parallel for schedule(dynamic)
    for (int z = 0; z < n; z++) or_intt(c, pidx[z], a + (u64)z * c->N);
}

/* ------------------------------------------------------------------------
 * Fast base conversion, Eq. (1) (Sec. III-F3): for every target prime p,
 *   y_p = ( sum_i [x_i * qhat_i^-1]_{q_i} * [qhat_i]_p ) mod p,
 * qhat_i = prod_{k != i} q_k over the source base.  Coefficient domain.
 * ---------------------------------------------------------------------- */
/* The conversion with each [x_i qhat_i^-1]_{q_i} taken as its canonical
 * representative v in [0, q_i) (centred = 0) or as its centred one, v - q_i
 * when v > (q_i - 1) / 2 (centred = 1). */
static void bconv_impl(const or_ctx *c, const u64 *src, const int *src_idx, int n_src,
                       u64 *dst, const int *dst_idx, int n_dst, int centred)
{
    u64 N = c->N;
    u64 *qhat_inv = (u64 *)malloc(sizeof(u64) * n_src);
    u64 *qhat_mod = (u64 *)malloc(sizeof(u64) * n_src * n_dst);
    for (int i = 0; i < n_src; i++) {
        u64 qi = c->primes[src_idx[i]];
        u64 prod = 1;
        for (int k = 0; k < n_src; k++) if (k != i) prod = mul_mod(prod, c->primes[src_idx[k]] % qi, qi);
        qhat_inv[i] = inv_mod(prod, qi);
        for (int d = 0; d < n_dst; d++) {
            u64 p = c->primes[dst_idx[d]];
            u64 h = 1;
            for (int k = 0; k < n_src; k++) if (k != i) h = mul_mod(h, c->primes[src_idx[k]] % p, p);
            qhat_mod[i * n_dst + d] = h;
        }
    }
    #pragma omp parallel for schedule(static)
    for (int d = 0; d < n_dst; d++) {
        u64 p = c->primes[dst_idx[d]];
        for (u64 n = 0; n < N; n++) {
            u64 acc = 0;
            for (int i = 0; i < n_src; i++) {
                u64 qi = c->primes[src_idx[i]];
                u64 v = mul_mod(src[(u64)i * N + n], qhat_inv[i], qi);
                u64 vp = (centred && v > (qi - 1) / 2) ? sub_mod(0, (qi - v) % p, p)   /* v - q_i, negative */
                                                        : v % p;
                acc = add_mod(acc, mul_mod(vp, qhat_mod[i * n_dst + d], p), p);
            }
            dst[(u64)d * N + n] = acc;
        }
    }
    free(qhat_inv);
    free(qhat_mod);
}

void or_bconv(const or_ctx *c, const u64 *src, const int *src_idx, int n_src,
              u64 *dst, const int *dst_idx, int n_dst)
{
    bconv_impl(c, src, src_idx, n_src, dst, dst_idx, n_dst, 0);
}

void or_bconv_centred(const or_ctx *c, const u64 *src, const int *src_idx, int n_src,
                      u64 *dst, const int *dst_idx, int n_dst)
{
    bconv_impl(c, src, src_idx, n_src, dst, dst_idx, n_dst, 1);
}

/* number of digits in use at nl limbs: beta = ceil(nl / alpha) */
int or_beta(const or_ctx *c, int nl) { return (nl + c->alpha - 1) / c->alpha; }

/*
 * ModUp (Sec. III-F3, Sec. II hybrid key switching): bring d (nl limbs,
 * evaluation form) to coefficient form; for each digit D_j (contiguous blocks
 * of alpha limbs from limb 0, the last one partial) convert D_j to every other
 * prime of Q_l and to every special prime, then NTT the new limbs.  The limbs
 * of D_j are the input's own evaluation limbs.  ext: [beta][nl + K][N].
 */
void or_modup(const or_ctx *c, const u64 *d, int nl, u64 *ext)
{
    u64 N = c->N;
    int K = c->nk, ne = nl + K, beta = or_beta(c, nl);
    u64 *coeff = (u64 *)malloc(sizeof(u64) * nl * N);
    memcpy(coeff, d, sizeof(u64) * nl * N);
    int *pidx = (int *)malloc(sizeof(int) * ne);
    for (int z = 0; z < ne; z++) pidx[z] = ext_prime(c, nl, z);
    or_intt_limbs(c, coeff, pidx, nl);
    for (int j = 0; j < beta; j++) {
        int lo = j * c->alpha, hi = lo + c->alpha < nl ? lo + c->alpha : nl;
        u64 *e = ext + (u64)j * ne * N;
        int n_src = hi - lo, n_dst = 0;
        int *src_idx = (int *)malloc(sizeof(int) * n_src);
        int *dst_idx = (int *)malloc(sizeof(int) * ne);
        int *dst_limb = (int *)malloc(sizeof(int) * ne);
        for (int i = 0; i < n_src; i++) src_idx[i] = lo + i;
        for (int z = 0; z < ne; z++) {
            if (z >= lo && z < hi) continue;
            dst_idx[n_dst] = pidx[z];
            dst_limb[n_dst] = z;
            n_dst++;
        }
        u64 *conv = (u64 *)malloc(sizeof(u64) * n_dst * N);
        or_bconv(c, coeff + (u64)lo * N, src_idx, n_src, conv, dst_idx, n_dst);
        or_ntt_limbs(c, conv, dst_idx, n_dst);
        for (int z = lo; z < hi; z++) memcpy(e + (u64)z * N, d + (u64)z * N, sizeof(u64) * N);
        for (int k = 0; k < n_dst; k++) memcpy(e + (u64)dst_limb[k] * N, conv + (u64)k * N, sizeof(u64) * N);
        free(conv); free(src_idx); free(dst_idx); free(dst_limb);
    }
    free(coeff);
    free(pidx);
}

/*
 * ModDown (Sec. III-F3 and the "ModDown fusion" item of Sec. III-F5):
 * x has nl q-limbs then K p-limbs, evaluation form.  INTT the p-limbs,
 * base-convert P -> Q_l, NTT, and return P^-1 (x_i - conv_i) mod q_i.
 * Floor (the context's default): the conversion takes canonical residues, so
 * conv = [x]_P + u P with 0 <= u < K and the result is floor(x / P) - u.
 * Nearest: it takes centred residues, so conv = x - P r with |conv| < K P / 2
 * and the result r is within K / 2 of x / P, with a mean error of zero.
 */
void or_moddown(const or_ctx *c, const u64 *x, int nl, u64 *out)
{
    u64 N = c->N;
    int K = c->nk;
    u64 *xp = (u64 *)malloc(sizeof(u64) * K * N);
    memcpy(xp, x + (u64)nl * N, sizeof(u64) * K * N);
    int *pk = (int *)malloc(sizeof(int) * K);
    int *qi = (int *)malloc(sizeof(int) * nl);
    for (int k = 0; k < K; k++) pk[k] = c->nq + k;
    for (int i = 0; i < nl; i++) qi[i] = i;
    or_intt_limbs(c, xp, pk, K);
    u64 *conv = (u64 *)malloc(sizeof(u64) * nl * N);
    bconv_impl(c, xp, pk, K, conv, qi, nl, c->nearest);
    or_ntt_limbs(c, conv, qi, nl);
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < nl; i++) {
        u64 q = c->primes[i];
        u64 P = 1;
        for (int k = 0; k < K; k++) P = mul_mod(P, c->primes[c->nq + k] % q, q);
        u64 pinv = inv_mod(P, q);
        for (u64 n = 0; n < N; n++)
            out[(u64)i * N + n] = mul_mod(sub_mod(x[(u64)i * N + n], conv[(u64)i * N + n], q), pinv, q);
    }
    free(xp); free(pk); free(qi); free(conv);
}

/*
 * Hybrid key switching (Sec. II, Sec. III-F3): ModUp, key inner product
 * acc_t = sum_j d~_j * evk_{j,t} over Q_l and P, then ModDown of each
 * accumulator.  evk: [dnum][2][nq + K][N] (component 0 = b, 1 = a), stored
 * at the full level; at nl limbs the q-limbs 0..nl-1 and the K p-limbs are used.
 */
void or_keyswitch(const or_ctx *c, const u64 *d, int nl, const u64 *evk, u64 *out0, u64 *out1)
{
    u64 N = c->N;
    int K = c->nk, ne = nl + K, beta = or_beta(c, nl), nfull = c->nq + K;
    u64 *ext = (u64 *)malloc(sizeof(u64) * beta * ne * N);
    or_modup(c, d, nl, ext);
    u64 *acc = (u64 *)calloc((size_t)2 * ne * N, sizeof(u64));
    #pragma omp parallel for schedule(static)
    for (int z = 0; z < ne; z++) {
        int pi = ext_prime(c, nl, z);
        int kz = z < nl ? z : c->nq + (z - nl);       /* limb of the full-level key */
        u64 q = c->primes[pi];
        for (int t = 0; t < 2; t++) {
            u64 *a = acc + ((u64)t * ne + z) * N;
            for (int j = 0; j < beta; j++) {
                const u64 *e = ext + ((u64)j * ne + z) * N;
                const u64 *k = evk + (((u64)j * 2 + t) * nfull + kz) * N;
                for (u64 n = 0; n < N; n++) a[n] = add_mod(a[n], mul_mod(e[n], k[n], q), q);
            }
        }
    }
    or_moddown(c, acc, nl, out0);
    or_moddown(c, acc + (u64)ne * N, nl, out1);
    free(ext);
    free(acc);
}

/*
 * HMult with relinearisation (Table I; Sec. III-F5 "HMult fusion" names the
 * same three tensor products): d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1,
 * then (d0, d1) + KeySwitch(d2) with the relinearisation key.
 * a, b, out: [2][nl][N] evaluation form.
 */
void or_hmult(const or_ctx *c, const u64 *a, const u64 *b, int nl, const u64 *rlk, u64 *out)
{
    u64 N = c->N, S = (u64)nl * N;
    u64 *d = (u64 *)malloc(sizeof(u64) * 3 * S);
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < nl; i++) {
        u64 q = c->primes[i];
        for (u64 n = 0; n < N; n++) {
            u64 o = (u64)i * N + n;
            u64 a0 = a[o], a1 = a[S + o], b0 = b[o], b1 = b[S + o];
            d[o] = mul_mod(a0, b0, q);
            d[S + o] = add_mod(mul_mod(a0, b1, q), mul_mod(a1, b0, q), q);
            d[2 * S + o] = mul_mod(a1, b1, q);
        }
    }
    u64 *ks0 = (u64 *)malloc(sizeof(u64) * S), *ks1 = (u64 *)malloc(sizeof(u64) * S);
    or_keyswitch(c, d + 2 * S, nl, rlk, ks0, ks1);
    for (int i = 0; i < nl; i++) {
        u64 q = c->primes[i];
        for (u64 n = 0; n < N; n++) {
            u64 o = (u64)i * N + n;
            out[o] = add_mod(d[o], ks0[o], q);
            out[S + o] = add_mod(d[S + o], ks1[o], q);
        }
    }
    free(d); free(ks0); free(ks1);
}

/* ------------------------------------------------------------------------
 * Automorphism X -> X^g (Sec. III-F1: a dependency within one limb; Table I
 * HRotate/Conjugate).  Rotation by k slots uses g = 5^k mod 2N (negative k
 * taken modulo N/2, the order of 5); conjugation uses g = 2N - 1.
 * ---------------------------------------------------------------------- */
u64 or_galois_elt(const or_ctx *c, i64 steps)
{
    i64 half = (i64)(c->N / 2);
    i64 k = ((steps % half) + half) % half;
    return pow_mod(5, (u64)k, 2 * c->N);
}

/* coefficient form: a_i X^i -> a_i X^(i g mod 2N), negated when that is >= N */
void or_automorph_coeff(const or_ctx *c, const u64 *in, u64 *out, int nl, const int *pidx, u64 g)
{
    u64 N = c->N;
    for (int z = 0; z < nl; z++) {
        u64 q = c->primes[pidx[z]];
        for (u64 i = 0; i < N; i++) {
            u64 e = (u64)(((u128)i * g) % (2 * N));
            u64 v = in[(u64)z * N + i];
            if (e < N) out[(u64)z * N + e] = v;
            else out[(u64)z * N + (e - N)] = neg_mod(v, q);
        }
    }
}

/* evaluation form: slot j holds a(psi^(2 brv(j)+1)); sigma_g(a) there equals
 * a(psi^((2 brv(j)+1) g)), i.e. the slot j' with 2 brv(j')+1 = (2 brv(j)+1) g. */
void or_automorph_eval(const or_ctx *c, const u64 *in, u64 *out, int nl, u64 g)
{
    u64 N = c->N, twoN = 2 * N;
    for (u64 j = 0; j < N; j++) {
        u64 e = (u64)(((u128)(2 * brv(j, c->logN) + 1) * g) % twoN);
        u64 src = brv((e - 1) / 2, c->logN);
        for (int z = 0; z < nl; z++) out[(u64)z * N + j] = in[(u64)z * N + src];
    }
}

/* Automorphism of a ciphertext with key switching (Table I HRotate and
 * Conjugate): (sigma_g(c0), sigma_g(c1)) then key-switch sigma_g(c1) with the
 * key of s(X^g); out = (sigma_g(c0) + ks0, ks1).  a, out: [2][nl][N]. */
void or_automorph_ct(const or_ctx *c, const u64 *a, int nl, u64 g, const u64 *rk, u64 *out)
{
    u64 N = c->N, S = (u64)nl * N;
    u64 *r = (u64 *)malloc(sizeof(u64) * 2 * S);
    or_automorph_eval(c, a, r, nl, g);
    or_automorph_eval(c, a + S, r + S, nl, g);
    u64 *ks0 = (u64 *)malloc(sizeof(u64) * S);
    or_keyswitch(c, r + S, nl, rk, ks0, out + S);
    for (int i = 0; i < nl; i++) {
        u64 q = c->primes[i];
        for (u64 n = 0; n < N; n++) out[(u64)i * N + n] = add_mod(r[(u64)i * N + n], ks0[(u64)i * N + n], q);
    }
    free(r); free(ks0);
}

/* HRotate by `steps` slots: g = 5^steps mod 2N. */
void or_rotate(const or_ctx *c, const u64 *a, int nl, i64 steps, const u64 *rk, u64 *out)
{
    or_automorph_ct(c, a, nl, or_galois_elt(c, steps), rk, out);
}

/* Conjugate (Table I): g = 2N - 1 maps every slot to its complex conjugate. */
void or_conjugate(const or_ctx *c, const u64 *a, int nl, const u64 *ck, u64 *out)
{
    or_automorph_ct(c, a, nl, 2 * c->N - 1, ck, out);
}

/*
 * Hoisted rotations (Sec. III-F6): one ModUp of c1 serves every rotation.
 * The automorphism permutes evaluation points the same way under every
 * prime, so sigma_g is applied to each limb of each ModUp digit (q- and
 * special limbs alike); then the inner product with that rotation's key, the
 * ModDown of both accumulators (not hoisted), and out_k = (sigma_g(c0) + ks0,
 * ks1).  a: [2][nl][N]; rks: [n_rot][dnum][2][nq + K][N]; outs: [n_rot][2][nl][N].
 */
void or_rotate_hoisted(const or_ctx *c, const u64 *a, int nl, int n_rot, const i64 *steps, const u64 *rks, u64 *outs)
{
    u64 N = c->N, S = (u64)nl * N;
    int K = c->nk, ne = nl + K, beta = or_beta(c, nl), nfull = c->nq + K;
    u64 *ext = (u64 *)malloc(sizeof(u64) * beta * ne * N);
    u64 *rext = (u64 *)malloc(sizeof(u64) * beta * ne * N);
    u64 *acc = (u64 *)malloc(sizeof(u64) * 2 * ne * N);
    u64 *r0 = (u64 *)malloc(sizeof(u64) * S);
    or_modup(c, a + S, nl, ext);
    for (int r = 0; r < n_rot; r++) {
        u64 g = or_galois_elt(c, steps[r]);
        const u64 *rk = rks + (u64)r * c->dnum * 2 * nfull * N;
        u64 *out = outs + (u64)r * 2 * S;
        for (int j = 0; j < beta; j++) or_automorph_eval(c, ext + (u64)j * ne * N, rext + (u64)j * ne * N, ne, g);
        memset(acc, 0, sizeof(u64) * 2 * ne * N);
        #pragma omp parallel for schedule(static)
        for (int z = 0; z < ne; z++) {
            int pi = ext_prime(c, nl, z);
            int kz = z < nl ? z : c->nq + (z - nl);
            u64 q = c->primes[pi];
            for (int t = 0; t < 2; t++) {
                u64 *ac = acc + ((u64)t * ne + z) * N;
                for (int j = 0; j < beta; j++) {
                    const u64 *e = rext + ((u64)j * ne + z) * N;
                    const u64 *k = rk + (((u64)j * 2 + t) * nfull + kz) * N;
                    for (u64 n = 0; n < N; n++) ac[n] = add_mod(ac[n], mul_mod(e[n], k[n], q), q);
                }
            }
        }
        or_moddown(c, acc, nl, r0);
        or_moddown(c, acc + (u64)ne * N, nl, out + S);
        u64 *sc0 = (u64 *)malloc(sizeof(u64) * S);
        or_automorph_eval(c, a, sc0, nl, g);
        for (int i = 0; i < nl; i++) {
            u64 q = c->primes[i];
            for (u64 n = 0; n < N; n++) out[(u64)i * N + n] = add_mod(sc0[(u64)i * N + n], r0[(u64)i * N + n], q);
        }
        free(sc0);
    }
    free(ext); free(rext); free(acc); free(r0);
}

/*
 * ModRaise (bootstrapping, Sec. III-F7): a is a ciphertext [2][1][N] modulo
 * q_0; out [2][nl][N] holds, for every coefficient, its centred
 * representative in (-q_0/2, q_0/2] reduced modulo q_0 .. q_{nl-1}
 * (coefficient form after INTT, evaluation form again after NTT).
 */
void or_from_signed(const or_ctx *c, const i64 *v, const int *pidx, int n, u64 *out);

void or_modraise(const or_ctx *c, const u64 *a, int nl, u64 *out)
{
    u64 N = c->N, q0 = c->primes[0];
    u64 *coef = (u64 *)malloc(sizeof(u64) * N);
    i64 *v = (i64 *)malloc(sizeof(i64) * N);
    int *pidx = (int *)malloc(sizeof(int) * nl);
    for (int i = 0; i < nl; i++) pidx[i] = i;
    for (int t = 0; t < 2; t++) {
        memcpy(coef, a + (u64)t * N, sizeof(u64) * N);
        or_intt(c, 0, coef);
        for (u64 n = 0; n < N; n++) v[n] = coef[n] > q0 / 2 ? (i64)coef[n] - (i64)q0 : (i64)coef[n];
        u64 *o = out + (u64)t * nl * N;
        or_from_signed(c, v, pidx, nl, o);
        or_ntt_limbs(c, o, pidx, nl);
    }
    free(coef); free(v); free(pidx);
}

/* Multiplication by the monomial X^k, 0 <= k < 2N, of both polynomials of a
 * ciphertext [2][nl][N]: in coefficient form a_i X^i -> a_i X^(i+k), negated
 * once for every wrap past X^N (X^N = -1). */
void or_mul_monomial(const or_ctx *c, const u64 *a, int nl, u64 k, u64 *out)
{
    u64 N = c->N;
    int *pidx = (int *)malloc(sizeof(int) * nl);
    for (int i = 0; i < nl; i++) pidx[i] = i;
    u64 *x = (u64 *)malloc(sizeof(u64) * nl * N);
    for (int t = 0; t < 2; t++) {
        memcpy(x, a + (u64)t * nl * N, sizeof(u64) * nl * N);
        or_intt_limbs(c, x, pidx, nl);
        u64 *o = out + (u64)t * nl * N;
        for (int z = 0; z < nl; z++) {
            u64 q = c->primes[z];
            for (u64 i = 0; i < N; i++) {
                u64 e = i + k, val = x[(u64)z * N + i];
                int neg = 0;
                while (e >= N) { e -= N; neg ^= 1; }
                o[(u64)z * N + e] = neg ? neg_mod(val, q) : val;
            }
        }
        or_ntt_limbs(c, o, pidx, nl);
    }
    free(x); free(pidx);
}

/* ------------------------------------------------------------------------
 * Element-wise operations of Table I on ciphertexts [2][nl][N] in evaluation
 * form, where a product of polynomials is the slot-wise product of their
 * evaluations and a constant polynomial evaluates to itself at every point.
 * Plaintexts are [nl][N] (evaluation form); constants are given by their
 * residues c[i] mod q_i.
 * ---------------------------------------------------------------------- */
void or_hadd(const or_ctx *c, const u64 *a, const u64 *b, int nl, u64 *out)
{
    u64 N = c->N, S = (u64)nl * N;
    for (int t = 0; t < 2; t++)
        for (int i = 0; i < nl; i++)
            for (u64 n = 0; n < N; n++) {
                u64 o = t * S + (u64)i * N + n;
                out[o] = add_mod(a[o], b[o], c->primes[i]);
            }
}

void or_hsub(const or_ctx *c, const u64 *a, const u64 *b, int nl, u64 *out)
{
    u64 N = c->N, S = (u64)nl * N;
    for (int t = 0; t < 2; t++)
        for (int i = 0; i < nl; i++)
            for (u64 n = 0; n < N; n++) {
                u64 o = t * S + (u64)i * N + n;
                out[o] = sub_mod(a[o], b[o], c->primes[i]);
            }
}

/* (c0 + pt, c1) */
void or_ptadd(const or_ctx *c, const u64 *a, const u64 *pt, int nl, u64 *out)
{
    u64 N = c->N, S = (u64)nl * N;
    for (int i = 0; i < nl; i++)
        for (u64 n = 0; n < N; n++) {
            u64 o = (u64)i * N + n;
            out[o] = add_mod(a[o], pt[o], c->primes[i]);
            out[S + o] = a[S + o];
        }
}

/* (c0 pt, c1 pt) */
void or_ptmult(const or_ctx *c, const u64 *a, const u64 *pt, int nl, u64 *out)
{
    u64 N = c->N, S = (u64)nl * N;
    for (int t = 0; t < 2; t++)
        for (int i = 0; i < nl; i++)
            for (u64 n = 0; n < N; n++) {
                u64 o = (u64)i * N + n;
                out[t * S + o] = mul_mod(a[t * S + o], pt[o], c->primes[i]);
            }
}

/* (c0 + k, c1) for the constant k with residues k[i] */
void or_scalar_add(const or_ctx *c, const u64 *a, const u64 *k, int nl, u64 *out)
{
    u64 N = c->N, S = (u64)nl * N;
    for (int i = 0; i < nl; i++)
        for (u64 n = 0; n < N; n++) {
            u64 o = (u64)i * N + n;
            out[o] = add_mod(a[o], k[i], c->primes[i]);
            out[S + o] = a[S + o];
        }
}

/* (k c0, k c1) */
void or_scalar_mult(const or_ctx *c, const u64 *a, const u64 *k, int nl, u64 *out)
{
    u64 N = c->N, S = (u64)nl * N;
    for (int t = 0; t < 2; t++)
        for (int i = 0; i < nl; i++)
            for (u64 n = 0; n < N; n++) {
                u64 o = t * S + (u64)i * N + n;
                out[o] = mul_mod(a[o], k[i], c->primes[i]);
            }
}

/*
 * Linear transform of the slots with the baby-step giant-step split of the
 * diagonal method (Sec. III-F7 bootstrapping's CoeffToSlot / SlotToCoeff,
 * whose baby steps are the hoisted rotations of Sec. III-F6):
 *   y = sum_i d_i (.) rot_i(z) = sum_g rot_{n1 g}( sum_b pt_{g,b} (.) rot_b(z) ),
 * i = n1 g + b, 0 <= b < n1, with pt_{g,b} the plaintext of rot_{-n1 g}(d_i)
 * (the caller encodes it pre-rotated).  The baby-step rotations b != 0 share
 * one ModUp (or_rotate_hoisted); each giant step g != 0 is one HRotate.
 *   diag_idx[n_diag]   : diagonal indices i in [0, N/2), distinct
 *   pts                : [n_diag][nl][N], pts[k] the plaintext of diagonal diag_idx[k]
 *   key_steps, keys    : n_keys rotation keys [dnum][2][nq + K][N] by step count
 *   out                : [2][nl][N]
 * Returns 0, or -1 if a needed rotation key is missing.
 */
static const u64 *find_key(const or_ctx *c, int n_keys, const i64 *key_steps, const u64 *keys, i64 steps)
{
    i64 half = (i64)(c->N / 2), want = ((steps % half) + half) % half;
    u64 key_words = (u64)c->dnum * 2 * (c->nq + c->nk) * c->N;
    for (int k = 0; k < n_keys; k++)
        if ((((key_steps[k] % half) + half) % half) == want) return keys + (u64)k * key_words;
    return NULL;
}

int or_linear_transform(const or_ctx *c, const u64 *a, int nl, int n_diag, const int *diag_idx, const u64 *pts,
                        int n1, int n_keys, const i64 *key_steps, const u64 *keys, u64 *out)
{
    u64 N = c->N, S = (u64)nl * N;
    int half = (int)(N / 2), n_giant = (half + n1 - 1) / n1;
    u64 key_words = (u64)c->dnum * 2 * (c->nq + c->nk) * N;
    /* baby steps in use */
    int *baby_used = (int *)calloc(n1, sizeof(int));
    for (int k = 0; k < n_diag; k++) baby_used[diag_idx[k] % n1] = 1;
    int n_rot = 0;
    i64 *steps = (i64 *)malloc(sizeof(i64) * n1);
    u64 *rkeys = (u64 *)malloc(sizeof(u64) * (n1 > 1 ? n1 : 1) * key_words);
    for (int b = 1; b < n1; b++) {
        if (!baby_used[b]) continue;
        const u64 *k = find_key(c, n_keys, key_steps, keys, b);
        if (!k) { free(baby_used); free(steps); free(rkeys); return -1; }
        memcpy(rkeys + (u64)n_rot * key_words, k, sizeof(u64) * key_words);
        steps[n_rot++] = b;
    }
    u64 *rot = (u64 *)malloc(sizeof(u64) * (n_rot > 0 ? n_rot : 1) * 2 * S);
    if (n_rot) or_rotate_hoisted(c, a, nl, n_rot, steps, rkeys, rot);
    /* rotated copy of b, by baby step */
    const u64 **baby = (const u64 **)calloc(n1, sizeof(u64 *));
    baby[0] = a;
    for (int r = 0; r < n_rot; r++) baby[steps[r]] = rot + (u64)r * 2 * S;
    u64 *inner = (u64 *)malloc(sizeof(u64) * 2 * S);
    u64 *term = (u64 *)malloc(sizeof(u64) * 2 * S);
    u64 *prod = (u64 *)malloc(sizeof(u64) * 2 * S);
    int have_out = 0, rc = 0;
    for (int g = 0; g < n_giant && !rc; g++) {
        int have_inner = 0;
        for (int k = 0; k < n_diag; k++) {
            if (diag_idx[k] / n1 != g) continue;
            or_ptmult(c, baby[diag_idx[k] % n1], pts + (u64)k * S, nl, prod);
            if (have_inner) or_hadd(c, inner, prod, nl, inner);
            else memcpy(inner, prod, sizeof(u64) * 2 * S);
            have_inner = 1;
        }
        if (!have_inner) continue;
        if (g == 0) {
            memcpy(term, inner, sizeof(u64) * 2 * S);
        } else {
            const u64 *k = find_key(c, n_keys, key_steps, keys, (i64)n1 * g);
            if (!k) { rc = -1; break; }
            or_rotate(c, inner, nl, (i64)n1 * g, k, term);
        }
        if (have_out) or_hadd(c, out, term, nl, out);
        else memcpy(out, term, sizeof(u64) * 2 * S);
        have_out = 1;
    }
    if (!have_out && !rc) memset(out, 0, sizeof(u64) * 2 * S);
    free(baby_used); free(steps); free(rkeys); free(rot); free(baby); free(inner); free(term); free(prod);
    return rc;
}

/*
 * Rescale (Table I; Sec. III-F5 "Rescale fusion"): with l = nl - 1, INTT limb
 * l, take a representative of each of its coefficients modulo each q_i
 * (SwitchModulo), NTT under q_i, and return q_l^-1 (x_i - that) mod q_i for
 * i < l.  Floor (or_rescale): the canonical representative r in [0, q_l), so
 * the result is floor(x / q_l).  Nearest (or_rescale_round): the centred one,
 * r - q_l when r > (q_l - 1) / 2, so the result is round(x / q_l) (q_l odd:
 * no ties).
 * a: [2][nl][N] -> out: [2][nl-1][N].
 */
static void rescale_impl(const or_ctx *c, const u64 *a, int nl, u64 *out, int nearest)
{
    u64 N = c->N;
    int l = nl - 1;
    u64 ql = c->primes[l];
    for (int poly = 0; poly < 2; poly++) {
        const u64 *x = a + (u64)poly * nl * N;
        u64 *o = out + (u64)poly * l * N;
        u64 *last = (u64 *)malloc(sizeof(u64) * N);
        memcpy(last, x + (u64)l * N, sizeof(u64) * N);
        or_intt(c, l, last);
        #pragma omp parallel for schedule(dynamic)
        for (int i = 0; i < l; i++) {
            u64 q = c->primes[i];
            u64 *y = (u64 *)malloc(sizeof(u64) * N);
            for (u64 n = 0; n < N; n++) {
                u64 r = last[n];
                if (nearest && r > (ql - 1) / 2)
                    y[n] = sub_mod(0, (ql - r) % q, q);   /* r - q_l, a negative integer, mod q */
                else
                    y[n] = r % q;
            }
            or_ntt(c, i, y);
            u64 qinv = inv_mod(ql % q, q);
            for (u64 n = 0; n < N; n++)
                o[(u64)i * N + n] = mul_mod(sub_mod(x[(u64)i * N + n], y[n], q), qinv, q);
            free(y);
        }
        free(last);
    }
}

void or_rescale(const or_ctx *c, const u64 *a, int nl, u64 *out) { rescale_impl(c, a, nl, out, 0); }
void or_rescale_round(const or_ctx *c, const u64 *a, int nl, u64 *out) { rescale_impl(c, a, nl, out, 1); }

/* ------------------------------------------------------------------------
 * Client side (KeyGen / Encrypt / Decrypt are OpenFHE's job in the paper,
 * Sec. III-A; written here only to make test inputs and check results).
 * ---------------------------------------------------------------------- */

/* signed coefficients -> residues of limbs 0..n-1 under primes pidx[] */
void or_from_signed(const or_ctx *c, const i64 *v, const int *pidx, int n, u64 *out)
{
    for (int z = 0; z < n; z++) {
        u64 q = c->primes[pidx[z]];
        for (u64 i = 0; i < c->N; i++) out[(u64)z * c->N + i] = from_signed(v[i], q);
    }
}

/*
 * Hybrid switching key for s' (Sec. II, hybrid key switching of [hk2020]):
 * for each digit j, evk_j = (b_j, a_j) over all nq + K primes with
 *   b_j = -a_j s + e_j + [P]_{q_i} s'   on q-limbs i in D_j,
 *   b_j = -a_j s + e_j                  on the other q-limbs and on p-limbs,
 * i.e. b_j = -a_j s + e_j + P * Qtilde_j * s' with Qtilde_j = 1 mod D_j and
 * 0 mod the other q_i.  s, sp: [nq+K][N] evaluation form; a: [dnum][nq+K][N]
 * uniform (evaluation form); e: [dnum][N] signed coefficients.
 */
void or_keygen(const or_ctx *c, const u64 *s, const u64 *sp, const u64 *a, const i64 *e, u64 *evk)
{
    u64 N = c->N;
    int np = c->nq + c->nk;
    int *pidx = (int *)malloc(sizeof(int) * np);
    for (int z = 0; z < np; z++) pidx[z] = z;
    u64 *ee = (u64 *)malloc(sizeof(u64) * np * N);
    for (int j = 0; j < c->dnum; j++) {
        or_from_signed(c, e + (u64)j * N, pidx, np, ee);
        or_ntt_limbs(c, ee, pidx, np);
        int lo = j * c->alpha, hi = lo + c->alpha < c->nq ? lo + c->alpha : c->nq;
        u64 *b = evk + ((u64)j * 2 + 0) * np * N;
        u64 *ak = evk + ((u64)j * 2 + 1) * np * N;
        for (int z = 0; z < np; z++) {
            u64 q = c->primes[z];
            u64 P = 1;
            for (int k = 0; k < c->nk; k++) P = mul_mod(P, c->primes[c->nq + k] % q, q);
            int in_digit = (z >= lo && z < hi);
            for (u64 n = 0; n < N; n++) {
                u64 o = (u64)z * N + n;
                u64 aj = a[(u64)j * np * N + o];
                u64 v = add_mod(neg_mod(mul_mod(aj, s[o], q), q), ee[o], q);
                if (in_digit) v = add_mod(v, mul_mod(P, sp[o], q), q);
                b[o] = v;
                ak[o] = aj;
            }
        }
    }
    free(ee);
    free(pidx);
}

/* secret-key RLWE encryption: ct = (-a s + m + e, a) on limbs 0..nl-1;
 * m, e signed coefficients, a uniform (evaluation form), s evaluation form. */
void or_encrypt(const or_ctx *c, int nl, const i64 *m, const i64 *e, const u64 *a, const u64 *s, u64 *ct)
{
    u64 N = c->N, S = (u64)nl * N;
    int *pidx = (int *)malloc(sizeof(int) * nl);
    for (int z = 0; z < nl; z++) pidx[z] = z;
    i64 *me = (i64 *)malloc(sizeof(i64) * N);
    for (u64 i = 0; i < N; i++) me[i] = m[i] + e[i];
    u64 *p = (u64 *)malloc(sizeof(u64) * S);
    or_from_signed(c, me, pidx, nl, p);
    or_ntt_limbs(c, p, pidx, nl);
    for (int z = 0; z < nl; z++) {
        u64 q = c->primes[z];
        for (u64 n = 0; n < N; n++) {
            u64 o = (u64)z * N + n;
            ct[o] = add_mod(neg_mod(mul_mod(a[o], s[o], q), q), p[o], q);
            ct[S + o] = a[o];
        }
    }
    free(pidx); free(me); free(p);
}

/* decryption residues: INTT(c0 + c1 s) on limbs 0..nl-1 (coefficient form) */
void or_decrypt(const or_ctx *c, const u64 *ct, int nl, const u64 *s, u64 *out)
{
    u64 N = c->N, S = (u64)nl * N;
    int *pidx = (int *)malloc(sizeof(int) * nl);
    for (int z = 0; z < nl; z++) {
        pidx[z] = z;
        u64 q = c->primes[z];
        for (u64 n = 0; n < N; n++) {
            u64 o = (u64)z * N + n;
            out[o] = add_mod(ct[o], mul_mod(ct[S + o], s[o], q), q);
        }
    }
    or_intt_limbs(c, out, pidx, nl);
    free(pidx);
}

/* pointwise product of limbs under primes pidx[] (evaluation form) */
void or_pointwise_mul(const or_ctx *c, const u64 *a, const u64 *b, const int *pidx, int n, u64 *out)
{
    for (int z = 0; z < n; z++) {
        u64 q = c->primes[pidx[z]];
        for (u64 i = 0; i < c->N; i++) out[(u64)z * c->N + i] = mul_mod(a[(u64)z * c->N + i], b[(u64)z * c->N + i], q);
    }
}
