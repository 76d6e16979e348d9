/*
 * fides.h -- C ABI of the GB300 CKKS key-switching engine.
 *
 * The engine implements the server-side hot path of CKKS described in
 * "FIDESlib: A Fully-Fledged Open-Source FHE Library for Efficient CKKS on
 * GPUs" (arXiv 2507.04775): the 64-bit negacyclic (i)NTT over RNS limbs
 * (Sec. III-F4), fast base conversion (Sec. III-F3, Eq. 1), ModUp / ModDown,
 * the key inner product and hybrid key switching (Sec. II), HMult with
 * relinearisation, HRotate and Rescale (Table I; fusions of Sec. III-F5).
 *
 * Conventions (all entry points)
 * ------------------------------
 *  - Residues are uint64_t in canonical form [0, q).  Inputs outside [0, q)
 *    give unspecified (but memory-safe) results.
 *  - Polynomials are limb-major: limb z of an n-limb polynomial occupies
 *    words [z*N, (z+1)*N).  Limb i of a ciphertext-level polynomial lives
 *    modulo q_i.  An "extended" polynomial at nl limbs has nl + K limbs: q_0 ..
 *    q_{nl-1} followed by the K special primes p_0 .. p_{K-1}.
 *  - Evaluation ("NTT") form: word j of a limb holds a(psi^(2 brv(j) + 1)) mod
 *    q, psi = g^((q-1)/2N) with g the smallest generator of Z_q^*; i.e. the
 *    forward transform maps natural order to bit-reversed order (Sec. III-F4).
 *  - A ciphertext is two polynomials (c0, c1) stored back to back:
 *    [2][nl][N], evaluation form, decrypting to c0 + c1 s.
 *  - A switching key is [dnum][2][L + K][N] (component 0 = b, 1 = a),
 *    evaluation form, at the full level; at nl limbs the first nl q-limbs and
 *    the K special limbs are read.  Digit j covers q-limbs [j*alpha,
 *    min((j+1)*alpha, nl)), alpha = ceil(L / dnum).
 *  - Pointers named dev_* are device pointers owned by the caller; they must be
 *    8-byte aligned and must stay valid until the work queued on `stream`
 *    completes.  Outputs may not alias inputs unless the entry point says so.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Every compute
 *    entry point is asynchronous with respect to the host.
 *  - Calls on one context use the context's scratch memory and must not run
 *    concurrently, except on streams registered with fides_ctx_add_stream,
 *    which have pools of their own (or create one context per stream).
 *    Programs (fides_program_run) need no registration: each run uses the
 *    scratch inside its own work buffer, so runs with different work buffers
 *    may overlap on several streams of one context.
 *  - Switching keys (relinearisation, rotation, conjugation) are passed as
 *    handles from fides_key_register, which binds a caller-owned key buffer
 *    to the Galois element it switches from.  A key's contents must be final
 *    when it is registered and must not change while the handle exists: the
 *    key switch reads key words before it waits for the kernels queued ahead
 *    of it (they stream in during the previous kernel's last wave), and every
 *    fides_* kernel lets the next one start early (programmatic dependent
 *    launch), so a key written by a kernel still in flight -- a fides_ntt on
 *    the same stream, say -- could be read half-written.  Registration
 *    synchronises the context's device, which ends any such writer.
 *  - Return value: FIDES_OK (0) or a negative FIDES_ERR_* code; the message of
 *    the last error on the calling thread is available from fides_last_error().
 *    Argument errors are detected before anything is queued.
 */
#ifndef FIDES_H
#define FIDES_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FIDES_OK 0
#define FIDES_ERR_ARG (-1)          /* bad argument (null pointer, size, level) */
#define FIDES_ERR_UNSUPPORTED (-2)  /* parameter set outside what the kernels handle */
#define FIDES_ERR_NOMEM (-3)        /* device or host allocation failed */
#define FIDES_ERR_CUDA (-4)         /* a CUDA call failed */
#define FIDES_ERR_TIMEOUT (-5)      /* a bounded device-side wait gave up */
#define FIDES_ERR_PRIME (-6)        /* a modulus is not an NTT-friendly prime */
#define FIDES_ERR_KEY (-7)          /* no key for a request or a rotation the operation needs */
#define FIDES_ERR_BUSY (-8)         /* request server: queue full, or request no longer queued */
#define FIDES_ERR_CANCELLED (-9)    /* request server: the request was cancelled before it ran */

typedef struct fides_ctx fides_ctx;

/* A ciphertext descriptor: `data` is a device buffer [2][n_limbs][N]. The
 * scale is tracked on the host (Sec. II: scaling factors are tracked per
 * level); the library updates it in outputs. */
typedef struct {
    uint64_t *data;
    int n_limbs;
    double scale;
} fides_ct;

/*
 * Switching-key handles (Sec. II hybrid key switching; Table I: HMult
 * relinearises with the key of s^2, HRotate by k slots needs the key of
 * s(X^g) with g = 5^k mod 2N, Conjugate the key of s(X^(2N-1))).
 *   dev_key    : device buffer [dnum][2][L + K][N] of the context's shape (see
 *                the conventions above), 8-byte aligned, owned by the caller,
 *                valid and unchanged until fides_key_destroy.
 *   galois_elt : FIDES_GALOIS_RELIN (0) for a relinearisation key, otherwise
 *                the odd Galois element g in [1, 2N) of the automorphism the
 *                key undoes (fides_galois_elt for rotations, 2N - 1 for
 *                conjugation).
 * fides_key_register checks the arguments (FIDES_ERR_ARG: NULL or unaligned
 * buffer, memory that is not on the context's device, a Galois element that is
 * not 0 or odd below 2N), synchronises the context's device (so that whatever
 * filled the buffer has finished) and returns a handle, a small host object;
 * the buffer is referenced, not copied.  Every entry point that switches keys
 * checks the handle before it queues anything and returns FIDES_ERR_KEY when
 * the key belongs to another context or to another Galois element than the
 * operation needs.  Destroy handles after the work that uses them completes;
 * fides_key_destroy(NULL) does nothing.
 */
typedef struct fides_key fides_key;
#define FIDES_GALOIS_RELIN 0

/* Last error message of the calling thread ("" if none). */
const char *fides_last_error(void);

/* Library version string. */
const char *fides_version(void);

/*
 * NTT-friendly primes (Table II: word-sized q_i ~ Delta): walks downward from
 * 2^bits over q = 1 (mod 2N) and writes the first `count` primes that are not
 * in exclude[0..n_exclude).  Host only.  bits in [logN + 2, 61].
 */
int fides_find_primes(int logN, int bits, int count, const uint64_t *exclude, int n_exclude,
                      uint64_t *out);

/*
 * Creates a context on the current CUDA device (Sec. III-E "Precomputation":
 * per-prime constants are computed once at context creation).
 *   logN   : ring degree N = 2^logN, 12 <= logN <= 17 (one tile per limb at
 *            12; two-pass NTTs above).
 *   L      : number of q-primes (maximum ciphertext limbs), 1 <= L.
 *   dnum   : number of key-switching digits, 1 <= dnum <= L.
 *   primes : host array of L q-primes then K special primes, each prime,
 *            = 1 mod 2N, < 2^61, all distinct.
 *   K      : number of special primes, 1 <= K, L + K <= 64.
 * Owns device tables (twiddles with Shoup companions, base-conversion
 * matrices) and a scratch pool sized for one operation at the top level.
 */
int fides_ctx_create(int logN, int L, int dnum, const uint64_t *primes, int K, fides_ctx **out);
void fides_ctx_destroy(fides_ctx *ctx);

/*
 * Gives `stream` (a cudaStream_t; NULL, the legacy default stream, is
 * allowed) its own scratch pool, the size of the context's, allocated now on
 * the context's device.  Single-operation calls of this context on a
 * registered stream then use that pool, so they may overlap calls on other
 * registered streams, or on one unregistered stream, which uses the
 * context's pool.  The paper overlaps independent work on CUDA streams
 * (Sec. III-F1, stream handling); this is how independent operations of one
 * context do it.  Batches, servers and programs have scratch of their own
 * and are unaffected.
 *   - A stream stays registered, and its pool allocated, until the context is
 *     destroyed; registering it again does nothing and returns FIDES_OK.
 *   - At most 16 streams per context (FIDES_ERR_ARG beyond that, or for a
 *     NULL ctx); FIDES_ERR_CUDA if the allocation fails.
 *   - Call it from one host thread at a time per context, before the stream's
 *     first call; calls on other streams may run meanwhile.
 */
int fides_ctx_add_stream(fides_ctx *ctx, void *stream);

/*
 * Autotuner of the NTT launch shape (Sec. III-F1 tunes a limb-batch parameter
 * per GPU; every launch here covers all limbs of a step, and what is tuned is
 * the tile width of each pass, which sets the CTA count and hence how full the
 * last wave is).  Times each tile variant (16, 8 or 4 columns or rows per CTA,
 * with a 64- or 80-register budget) of each logN=16 pass for every limb count 1..max_limbs (at most 128; larger
 * launches use the choice for 128) on this context's scratch, and keeps the
 * fastest.  Without it 8 columns / 4 rows per CTA are used.  Results are unchanged
 * by the choice.  Synchronises `stream`; do not run it while other work uses
 * this context.  logN = 12 has a single variant (returns FIDES_OK at once).
 * fides_ctx_ntt_tile reports the variant chosen for pass 0..3 (forward
 * columns, forward rows, inverse rows, inverse columns) at n_limbs as
 * (tile width << 8) | resident CTAs per SM.
 */
int fides_ctx_autotune(fides_ctx *ctx, int max_limbs, void *stream);
int fides_ctx_ntt_tile(const fides_ctx *ctx, int pass, int n_limbs);

/*
 * The tuned table itself, for an autotuner cache: FIDES_TUNE_ENTRIES bytes,
 * the variant index per pass kind (4) and limb count (0..128).  set = 0
 * copies the context's table out; set = 1 installs `table` (FIDES_ERR_ARG,
 * nothing changed, if an entry is not a variant index).
 */
#define FIDES_TUNE_ENTRIES (4 * 129)
int fides_ctx_tune_table(fides_ctx *ctx, unsigned char *table, int set);

/*
 * Device status of the context: kernels never spin without a limit.  A
 * tensor-core base conversion whose wait for its operand copy or for its
 * matrix products runs out (about 2 s) sets FIDES_STATUS_WAIT_TIMEOUT, skips
 * its outputs, frees its tensor memory and returns.  Writes the bits seen
 * since the last call to *flags (0: none) and clears them.  Synchronises the
 * device.  Returns FIDES_OK or FIDES_ERR_CUDA.
 */
#define FIDES_STATUS_WAIT_TIMEOUT 1
int fides_ctx_status(fides_ctx *ctx, int *flags);

/*
 * Self-test of the bounded device waits: launches one thread that waits on an
 * mbarrier nothing arrives on, for limit_us (1..100000) microseconds, then
 * sets FIDES_STATUS_WAIT_TIMEOUT in the context's status word and returns.
 * The context stays usable.  Asynchronous on `stream`.
 */
int fides_ctx_selftest_wait(fides_ctx *ctx, int limit_us, void *stream);

/*
 * Self-test of the tensor-core conversion's abort path: runs the top-level
 * ModUp conversion (Eq. 1) on the scratch pool of `stream`, with every
 * pipeline wait limited to limit_us (1..100000) microseconds, and with the
 * first CTA never copying its first tile's sources in.  That CTA's waits run
 * out; it sets FIDES_STATUS_WAIT_TIMEOUT, every role of it leaves its loop,
 * it waits for the copies and products it did issue, frees its tensor memory
 * and returns; the other CTAs convert normally.  Its outputs are scratch
 * only.  The context stays usable.  Asynchronous on `stream`.  Returns
 * FIDES_ERR_UNSUPPORTED when this context's ModUp converts on the integer
 * kernel (a digit of more than 16 primes).
 */
int fides_ctx_selftest_conversion(fides_ctx *ctx, int limit_us, void *stream);

/*
 * Rounding of the two divisions of the path -- ModDown's division by P and
 * Rescale's division by q_l -- for every operation of this context (single
 * operations, batches, the server and programs).  The paper's ModDown and
 * Rescale fusion formulas (Sec. III-F5) state no rounding offset.
 *   FIDES_ROUND_FLOOR (the default): canonical residues.  Rescale gives
 *     floor(x / q_l); ModDown gives floor(x / P) - u with the conversion term
 *     0 <= u < K.  Both errors have a nonzero mean, which decoding sums
 *     coherently into the slots whose evaluation point is near 1: at
 *     logN=16, K=10, scale 2^40 a rotation decrypts within about 2^-14 there.
 *   FIDES_ROUND_NEAREST: centred residues.  Rescale gives round(x / q_l)
 *     (as fides_rescale_round); ModDown converts the centred residues of the
 *     special limbs, so its result is within K/2 of x / P with a mean error
 *     of zero (same work: the correction rides in a spare column of the
 *     tensor-core conversion).  The same rotation decrypts within 2^-20.
 * Affects calls issued after it returns; set it before building batches,
 * servers or programs, which capture the mode when they plan.  Returns
 * FIDES_OK or FIDES_ERR_ARG.  fides_ctx_rounding reads the mode.
 */
#define FIDES_ROUND_FLOOR 0
#define FIDES_ROUND_NEAREST 1
int fides_ctx_set_rounding(fides_ctx *ctx, int mode);
int fides_ctx_rounding(const fides_ctx *ctx);

/*
 * Whether base conversions of this context run on the tensor cores (1: every
 * digit and K have at most 16 primes) or on the integer pipes (0).  Results
 * are identical.
 */
int fides_ctx_tensor_bconv(const fides_ctx *ctx);

/* Number of digits in use at n_limbs limbs: ceil(n_limbs / alpha). */
int fides_ctx_beta(const fides_ctx *ctx, int n_limbs);
/* psi of prime index i (0..L+K-1), or 0 for a bad index. */
uint64_t fides_ctx_psi(const fides_ctx *ctx, int prime_index);
/* Galois element of a left rotation by `steps` slots: 5^steps mod 2N. */
uint64_t fides_galois_elt(const fides_ctx *ctx, int64_t steps);

int fides_key_register(fides_ctx *ctx, const uint64_t *dev_key, uint64_t galois_elt, fides_key **out);
void fides_key_destroy(fides_key *key);
/* Galois element a handle was registered with (0 for a NULL handle). */
uint64_t fides_key_galois(const fides_key *key);

/*
 * Forward / inverse negacyclic NTT (Sec. III-F4), in place, on `batch`
 * polynomials of n_limbs limbs each stored back to back; limb z of every
 * polynomial uses prime index first_prime + z.  Forward: natural order in,
 * bit-reversed out.  Inverse: bit-reversed in, natural out, includes N^-1.
 * first_prime + n_limbs <= L + K.
 */
int fides_ntt(fides_ctx *ctx, uint64_t *dev, int first_prime, int n_limbs, int batch, void *stream);
int fides_intt(fides_ctx *ctx, uint64_t *dev, int first_prime, int n_limbs, int batch, void *stream);

/*
 * ModUp (Sec. III-F3; Sec. II hybrid key switching): dev_d is an n_limbs-limb
 * polynomial in evaluation form.  For each digit D_j, the limbs of D_j are
 * copied and every other prime of q_0..q_{n_limbs-1} and every special prime
 * is filled by fast base conversion (Eq. 1) of D_j in coefficient form
 * followed by an NTT.  dev_ext receives [beta][n_limbs + K][N].
 */
int fides_modup(fides_ctx *ctx, const uint64_t *dev_d, int n_limbs, uint64_t *dev_ext, void *stream);

/*
 * ModDown (Sec. III-F3, Sec. III-F5 "ModDown fusion"): dev_x is an extended
 * polynomial [n_limbs + K][N] in evaluation form; dev_out [n_limbs][N]
 * receives P^-1 (x_i - NTT(Conv_{P->Q}(INTT(x_P))))_i mod q_i, the conversion
 * taking canonical residues (FIDES_ROUND_FLOOR) or centred ones
 * (FIDES_ROUND_NEAREST), per fides_ctx_set_rounding.
 */
int fides_moddown(fides_ctx *ctx, const uint64_t *dev_x, int n_limbs, uint64_t *dev_out, void *stream);

/*
 * Hybrid key switching of one polynomial d (n_limbs limbs, evaluation form)
 * with key evk (any registered key of this context): ModUp, key inner product
 * acc_t = sum_j d~_j evk_{j,t} (Sec. III-F5 "Dot product fusion"), ModDown of
 * both accumulators.  Output (dev_out0, dev_out1), each [n_limbs][N], with
 * out0 + out1 s ~= d s', s' the secret the key switches from.
 */
int fides_keyswitch(fides_ctx *ctx, const uint64_t *dev_d, int n_limbs, const fides_key *evk,
                    uint64_t *dev_out0, uint64_t *dev_out1, void *stream);

/*
 * HMult with relinearisation (Table I): d0 = a0 b0, d1 = a0 b1 + a1 b0,
 * d2 = a1 b1, out = (d0, d1) + KeySwitch(d2, rlk).  a, b and out have the
 * same n_limbs; out->scale = a->scale * b->scale.  out may not alias a or b.
 * rlk: a key registered with FIDES_GALOIS_RELIN (FIDES_ERR_KEY otherwise).
 */
int fides_hmult(fides_ctx *ctx, const fides_ct *a, const fides_ct *b, const fides_key *rlk,
                fides_ct *out, void *stream);

/*
 * HMult with relinearisation followed by Rescale, in one key switch: out
 * (a->n_limbs - 1 limbs, n_limbs >= 2) receives exactly the residues of
 * fides_hmult then fides_rescale; out->scale = a->scale * b->scale / q_l.
 * By linearity of the NTT the Rescale folds into the ModDown (Sec. III-F5
 * "ModDown fusion" and "Rescale fusion" combined): the ModDown's INTT also
 * transforms the dropped limb of the tensor product and of the accumulators,
 * and one forward NTT over the remaining limbs computes
 * q_l^-1 (d_i + P^-1 acc_i - NTT(P^-1 conv_i + [last]_{q_i})).  out may not
 * alias a or b.
 */
int fides_hmult_rescale(fides_ctx *ctx, const fides_ct *a, const fides_ct *b, const fides_key *rlk,
                        fides_ct *out, void *stream);

/*
 * HRotate (Table I): rotation of the slots left by `steps` (g = 5^steps mod
 * 2N); out = (sigma_g(c0) + ks0, ks1) with (ks0, ks1) = KeySwitch(sigma_g(c1),
 * rk) and rk the switching key of s(X^g), registered with that g
 * (FIDES_ERR_KEY otherwise, nothing queued).  out may not alias a.
 */
int fides_rotate(fides_ctx *ctx, const fides_ct *a, int64_t steps, const fides_key *rk,
                 fides_ct *out, void *stream);

/*
 * Rescale (Table I, Sec. III-F5 "Rescale fusion"): drops the last limb q_l,
 * l = a->n_limbs - 1 >= 1: out_i = q_l^-1 (x_i - NTT_{q_i}([INTT(x_l)]_{q_i}))
 * mod q_i, which is floor(x / q_l) limb-wise (FIDES_ROUND_FLOOR), or
 * round(x / q_l) with the centred lift (FIDES_ROUND_NEAREST, see
 * fides_ctx_set_rounding).  out->n_limbs must equal a->n_limbs - 1;
 * out->scale = a->scale / q_l.  out may not alias a.
 */
int fides_rescale(fides_ctx *ctx, const fides_ct *a, fides_ct *out, void *stream);

/*
 * Rescale rounding to nearest instead of down: as fides_rescale, but
 * SwitchModulo takes the centred representative of each coefficient r of
 * INTT(x_l) (r - q_l when r > (q_l - 1) / 2), which gives round(x / q_l)
 * limb-wise (q_l is odd, so there are no ties; a value just below Q_l rounds
 * to Q_{l-1}, that is 0), whatever the context's rounding mode.  Same
 * arguments, layout, errors and scale as fides_rescale.
 */
int fides_rescale_round(fides_ctx *ctx, const fides_ct *a, fides_ct *out, void *stream);

/*
 * HSquare (Table I): HMult+relin of a with itself, identical to
 * fides_hmult(ctx, a, a, rlk, out, stream).  out may not alias a.
 */
int fides_hsquare(fides_ctx *ctx, const fides_ct *a, const fides_key *rlk, fides_ct *out, void *stream);

/*
 * Conjugate (Table I): the automorphism g = 2N - 1 (every slot to its
 * complex conjugate) with key switching by ck, the switching key of
 * s(X^(2N-1)) registered with g = 2N - 1; otherwise as fides_rotate.  out may
 * not alias a.
 */
int fides_conjugate(fides_ctx *ctx, const fides_ct *a, const fides_key *ck, fides_ct *out, void *stream);

/*
 * Hoisted rotations (Sec. III-F6): n_rot rotations of one ciphertext sharing
 * a single ModUp of c1.  The automorphism permutes evaluation points alike
 * under every prime, so rotation k applies sigma_{g_k} (g_k = 5^steps[k] mod
 * 2N) to every limb of every ModUp digit as the key inner product reads it,
 * then runs its own ModDown (ModDown is not hoisted):
 *   outs[k] = (sigma(c0) + ModDown(acc0_k), ModDown(acc1_k)),
 *   acc_t,k = sum_j sigma(ModUp(c1)_j) * rks[k]_{j,t}.
 * The residues differ from fides_rotate's (ModUp's approximate base
 * conversion does not commute with the automorphism's sign flips), but both
 * decrypt to the rotated message with the same noise bound.
 *   steps : host array [n_rot]
 *   rks   : host array [n_rot] of key handles, rks[k] registered with g_k
 *   outs  : host array [n_rot] of output descriptors at a->n_limbs; none may
 *           alias a.  out scales are set to a->scale.
 * 1 <= n_rot <= 64.  Uses the context's scratch (one ModUp + one key
 * switch's accumulators); rotations run one after another on `stream`.
 */
int fides_rotate_hoisted(fides_ctx *ctx, const fides_ct *a, int n_rot, const int64_t *steps,
                         const fides_key *const *rks, fides_ct *outs, void *stream);

/*
 * Linear transform of the slots (the diagonal method with a baby-step
 * giant-step split; bootstrapping's CoeffToSlot / SlotToCoeff, Sec. III-F7,
 * with hoisted baby steps, Sec. III-F6):
 *   y = sum_i d_i (.) rot_i(z) = sum_g rot_{n1 g}( sum_b pt_{g,b} (.) rot_b(z) ),
 * i = n1 g + b, 0 <= b < n1, rot_k = rotation left by k slots.
 *   diag_idx : host [n_diag], the diagonal indices i in use, in [0, N/2), distinct
 *   pts      : host [n_diag] of device plaintexts [n_limbs][N] (evaluation form):
 *              pts[k] encodes rot_{-n1 floor(i/n1)}(d_i) for i = diag_idx[k]
 *              at scale pt_scale (pre-rotated, as the split requires)
 *   keys     : host array [n_keys] of rotation-key handles; a key of Galois
 *              element 5^b mod 2N is needed for every baby step b != 0 and one
 *              of 5^(n1 g) for every giant step n1 g != 0 in use (FIDES_ERR_KEY
 *              before anything is queued if one is missing)
 *   work     : device scratch of fides_linear_transform_work_words() words
 *   out      : result at a's level, scale a->scale * pt_scale; may not alias a
 * The residues equal those of: hoisted rotations of a by the baby steps, a
 * plaintext multiply-accumulate per giant step, HRotate by n1 g, HAdd.
 */
int fides_linear_transform_work_words(fides_ctx *ctx, int n_limbs, int n_diag, const int *diag_idx, int n1,
                                      size_t *words);
int fides_linear_transform(fides_ctx *ctx, const fides_ct *a, int n_diag, const int *diag_idx,
                           const uint64_t *const *dev_pts, double pt_scale, int n1, int n_keys,
                           const fides_key *const *keys, uint64_t *dev_work, size_t work_words, fides_ct *out,
                           void *stream);

/*
 * ModRaise (bootstrapping, Sec. III-F7): a ciphertext at one limb (modulo
 * q_0) is lifted to out->n_limbs limbs: each coefficient's centred
 * representative in (-q_0/2, q_0/2] is reduced modulo q_0 .. q_{n-1} (INTT of
 * limb 0, centred lift, NTT per limb).  The result decrypts to m + q_0 I for
 * a small integer polynomial I.  a->n_limbs must be 1; out may not alias a;
 * out->scale = a->scale.
 */
int fides_modraise(fides_ctx *ctx, const fides_ct *a, fides_ct *out, void *stream);

/*
 * Multiplication of every slot by i (sign = +1: the monomial X^(N/2)) or by
 * -i (sign = -1: X^(3N/2)), exactly, without a level: in evaluation form the
 * monomial X^(N/2) is i_q (-1)^brv(j) at point j, i_q = psi^(N/2) mod q.
 * out may alias a; out->scale = a->scale.
 */
int fides_mul_i(fides_ctx *ctx, const fides_ct *a, int sign, fides_ct *out, void *stream);

/*
 * Element-wise operations (Table I) on ciphertexts in evaluation form; out
 * may alias a (and b).  out->n_limbs must equal a->n_limbs.
 *   fides_hadd / fides_hsub : out = a +/- b (b at a's level); out->scale = a->scale
 *                             (operands must carry the same scale).
 *   fides_ptadd   : out = (c0 + pt, c1); pt is a device plaintext [n_limbs][N]
 *                   in evaluation form encoded at a->scale.
 *   fides_ptmult  : out = (c0 pt, c1 pt); out->scale = a->scale * pt_scale.
 *   fides_scalar_add  : out = (c0 + k, c1), k a constant given by its residues
 *                       k[i] mod q_i (host array [n_limbs], each < q_i).
 *   fides_scalar_mult : out = (k c0, k c1); out->scale = a->scale * k_scale.
 */
int fides_hadd(fides_ctx *ctx, const fides_ct *a, const fides_ct *b, fides_ct *out, void *stream);
int fides_hsub(fides_ctx *ctx, const fides_ct *a, const fides_ct *b, fides_ct *out, void *stream);
int fides_ptadd(fides_ctx *ctx, const fides_ct *a, const uint64_t *dev_pt, fides_ct *out, void *stream);
int fides_ptmult(fides_ctx *ctx, const fides_ct *a, const uint64_t *dev_pt, double pt_scale, fides_ct *out,
                 void *stream);
int fides_scalar_add(fides_ctx *ctx, const fides_ct *a, const uint64_t *k, fides_ct *out, void *stream);
int fides_scalar_mult(fides_ctx *ctx, const fides_ct *a, const uint64_t *k, double k_scale, fides_ct *out,
                      void *stream);

/*
 * Batched operations (Sec. III-F1 hides launch overhead with limb batching;
 * here whole operations are batched).  A batch is a fixed list of HMult,
 * HRotate and Rescale operations on ciphertexts at any levels; each op names
 * its caller-owned input and output buffers, which must stay allocated and at
 * the same addresses for the life of the batch.  Ops carry a stage number:
 * every op of stage s runs after every op of stages < s and may read their
 * outputs; ops of one stage must be independent (no op writes what another
 * op of its stage reads or writes).
 *
 * The ops of a stage run in launch groups of at most `group_limbs` ciphertext
 * limbs (consecutive ops of the stage, at least one per group; 0 = the whole
 * stage is one group): one launch per step of the key switch covers every op
 * of a group, and groups run one after another, sharing one scratch pool
 * sized for the largest group (one key switch's worth per HMult/HRotate, two
 * limbs per Rescale).  The group size trades launch size against cache
 * locality (the paper's limb-batch trade-off, Sec. III-F1 and Sec. IV).
 *
 * fides_batch_create validates every op (FIDES_ERR_ARG naming the op on
 * error; FIDES_ERR_KEY for a key handle of another context or Galois
 * element), sets each op's out.scale, plans one group per stage with the
 * HMult tensor product as its own pass, allocates the scratch and uploads
 * device tables describing every launch; it synchronises.
 * fides_batch_run enqueues the whole batch on `stream`.  Results are
 * identical to calling fides_hmult / fides_rotate / fides_rescale op by op,
 * whatever the grouping.
 * fides_batch_capture records one run into a CUDA graph (stream must not be
 * NULL); later fides_batch_run calls launch that graph.
 * fides_batch_info reports the kernels one run launches and the device bytes
 * the batch owns.  Runs of one batch must not overlap on the GPU.
 * fides_batch_configure re-plans with a group size, tensor_split (1: the
 * tensor product as its own 16-byte pass where the buffers allow, 0: fused
 * into the first INTT pass) and prime_order (1: every NTT launch visits its
 * limbs ordered by prime, so that the CTAs in flight share the per-prime
 * twiddle tables in L2; 0: in plan order); fides_batch_autotune runs the
 * batch on `stream` for each group size 0, 32, 64, ... below the largest
 * stage's limbs and each of the four (tensor_split, prime_order) pairs, keeps
 * the fastest (its time per run in *best_ms, may be NULL) and shrinks the
 * scratch to it; fides_batch_tuning reports the current choice and the
 * number of launch groups.  The inner product always visits its rows by key
 * and key limb (the ops sharing a key read each limb while it is in L2).  Configure and autotune
 * synchronise the device, overwrite the ops' outputs (autotune runs the
 * batch) and drop a captured graph (capture again afterwards).
 */
#define FIDES_OP_HMULT 1    /* out = HMult+relin(a, b) with key = relinearisation key (Galois element 0) */
#define FIDES_OP_ROTATE 2   /* out = HRotate(a, steps) with key = rotation key of 5^steps mod 2N */
#define FIDES_OP_RESCALE 3  /* out = Rescale(a), out.n_limbs = a.n_limbs - 1 */

typedef struct {
    int type;
    int stage;
    fides_ct a;
    fides_ct b;
    fides_ct out;
    const fides_key *key;   /* HMULT, ROTATE (FIDES_ERR_KEY at creation if it does not fit) */
    int64_t steps;
} fides_op;

typedef struct fides_batch fides_batch;

int fides_batch_create(fides_ctx *ctx, fides_op *ops, int n_ops, fides_batch **out);
int fides_batch_run(fides_batch *batch, void *stream);
int fides_batch_capture(fides_batch *batch, void *stream);
int fides_batch_info(const fides_batch *batch, int *launches, size_t *scratch_bytes, size_t *table_bytes);
void fides_batch_destroy(fides_batch *batch);
int fides_batch_configure(fides_batch *batch, int group_limbs, int tensor_split, int prime_order);
int fides_batch_autotune(fides_batch *batch, void *stream, double *best_ms);
int fides_batch_tuning(const fides_batch *batch, int *group_limbs, int *tensor_split, int *prime_order,
                       int *groups);

/*
 * Request server: continuous batching of HMult+relin, HRotate and Rescale
 * requests (the paper runs one operation at a time, Sec. III-F1; this is the
 * serving loop around that hot path).  The caller keeps ciphertexts and keys
 * resident in device memory and submits requests that name them; a dispatcher
 * thread owned by the server
 *   - admits queued requests in arrival order while their device memory
 *     (output ciphertext + key-switch scratch) fits in the server's arena, a
 *     device allocation of cfg.arena_bytes made at creation: the arena size is
 *     the admission budget, and the head of the queue waits (no overtaking)
 *     until completed work or released outputs free enough of it;
 *   - launches the admitted requests, up to cfg.max_batch, as one launch group
 *     on the first free of cfg.n_lanes CUDA streams: one launch per step of the
 *     key switch for the whole group (the batched path's planner), so requests
 *     that arrive while groups run are admitted as lanes and memory free up and
 *     their work overlaps on the device;
 *   - queues a completion record for each request when its group finishes.
 * Each result is bit-identical to the single-operation entry point's
 * (fides_hmult / fides_rotate / fides_rescale) on the same inputs, whatever
 * group it ran in.
 *
 * Creation: ctx may be NULL only in simulation (cfg.simulate = 1), where no
 * device memory is touched and a group "runs" for sim_ns_per_limb x its
 * ciphertext limbs; the shape then comes from cfg.logN/L/K/dnum.  Simulation
 * computes no results (completions carry out.data = NULL); it exists to
 * exercise admission, batching, cancellation, time-outs and fault injection
 * without a GPU.  Real servers allocate the arena, cfg.n_lanes streams and
 * per-lane launch tables, and use the context's tables (not its scratch):
 * single-operation calls on the same context may run alongside, but
 * fides_ctx_autotune must not.
 *
 * Keys: fides_server_set_relin_key takes the relinearisation key and
 * fides_server_add_rotation_key the key of rotations by `steps` (modulo N/2),
 * both as handles (fides_key_register) of the server's context registered with
 * Galois element 0 and 5^steps mod 2N respectively (FIDES_ERR_KEY otherwise).
 * Handles and their buffers must stay valid until destroy.  In simulation
 * there is no context, and handles are tokens that are never dereferenced.
 *
 * fides_server_submit validates and queues one request and returns its id:
 *   FIDES_ERR_ARG       bad type, NULL input, level outside [1, L] (Rescale:
 *                       [2, L]), b at another level, or the server stopping;
 *   FIDES_ERR_KEY       no key for the request;
 *   FIDES_ERR_NOMEM     the request alone is larger than the arena;
 *   FIDES_ERR_BUSY      cfg.max_pending requests already queued.
 * Nothing is queued on error.  Inputs must stay valid and unchanged until the
 * request's completion is delivered.
 * fides_server_poll moves up to `max` completion records to out (waits up to
 * timeout_us for the first, < 0 = forever, 0 = no wait); *n_out = count.
 * Statuses: FIDES_OK (out.data points into the arena and stays valid until
 * fides_server_release(id)), FIDES_ERR_CANCELLED, FIDES_ERR_TIMEOUT (the group
 * ran longer than cfg.timeout_us; its memory is reclaimed when the device
 * finishes it), FIDES_ERR_CUDA or another launch error.
 * fides_server_release returns a completed request's output memory
 * (FIDES_ERR_ARG if the id holds no output).
 * fides_server_cancel removes a still-queued request (its completion carries
 * FIDES_ERR_CANCELLED); FIDES_ERR_BUSY once it has been admitted.
 * fides_server_pause(1) holds admission (requests queue), pause(0) resumes.
 * fides_server_inject arms a host-side fault: FIDES_FAULT_LAUNCH_ERROR makes
 * the next `arg` groups fail at launch (nothing is enqueued; their requests
 * complete with FIDES_ERR_CUDA), FIDES_FAULT_STALL hides the next group's
 * completion from the dispatcher for `arg` microseconds (as a slow device
 * would), which the time-out watchdog then sees.
 * fides_server_destroy cancels queued requests, waits for running groups and
 * frees everything, including unreleased outputs.
 * All calls are thread-safe.  Timestamps are CLOCK_MONOTONIC nanoseconds, the
 * clock of fides_now_ns().
 */
#define FIDES_SERVER_MAX_LANES 8
#define FIDES_SERVER_MAX_BATCH 512
#define FIDES_FAULT_LAUNCH_ERROR 1
#define FIDES_FAULT_STALL 2

typedef struct {
    size_t arena_bytes;       /* admission budget: device memory for outputs + scratch */
    int n_lanes;              /* streams with a group in flight at once, 1..8 */
    int max_batch;            /* requests per launch group, 1..512 */
    int max_pending;          /* queue bound, >= 1 */
    int64_t timeout_us;       /* watchdog per group, 0 = none */
    int simulate;             /* 1 = no device work (see above) */
    int64_t sim_ns_per_limb;  /* simulated device time per ciphertext limb */
    int logN, L, K, dnum;     /* shape when ctx is NULL (simulation only) */
} fides_server_config;

typedef struct {
    int type;          /* FIDES_OP_HMULT, FIDES_OP_ROTATE or FIDES_OP_RESCALE */
    fides_ct a, b;     /* resident device inputs (b: HMULT only) */
    int64_t steps;     /* HRotate: slots to rotate left */
    uint64_t tag;      /* caller's data, returned in the completion */
} fides_request;

typedef struct {
    uint64_t id, tag;
    int type;
    int status;
    fides_ct out;      /* result (n_limbs and scale always set; data NULL unless status is FIDES_OK) */
    int64_t t_submit_ns, t_admit_ns, t_launch_ns, t_done_ns;
    int group_ops;     /* requests in the launch group it ran in */
    int lane;          /* lane it ran on, -1 if it never ran */
} fides_completion;

typedef struct {
    uint64_t submitted, rejected, cancelled, completed, failed, timed_out;
    uint64_t groups, grouped_ops, max_group;   /* launch groups, requests in them, largest */
    uint64_t pending, in_flight, held;         /* queued, on the device, outputs not released */
    uint64_t arena_bytes, arena_used, arena_peak;
    uint64_t admission_stalls;                 /* requests that waited at the head for memory */
    uint64_t kernel_launches;                  /* kernels launched by the server */
    double device_ms;                          /* summed device time of finished groups */
    int max_lanes_busy;
} fides_server_stats;

typedef struct fides_server fides_server;

int fides_server_create(fides_ctx *ctx, const fides_server_config *cfg, fides_server **out);
void fides_server_destroy(fides_server *srv);
int fides_server_set_relin_key(fides_server *srv, const fides_key *key);
int fides_server_add_rotation_key(fides_server *srv, int64_t steps, const fides_key *key);
int fides_server_submit(fides_server *srv, const fides_request *req, uint64_t *id_out);
int fides_server_poll(fides_server *srv, fides_completion *out, int max, int64_t timeout_us, int *n_out);
int fides_server_release(fides_server *srv, uint64_t id);
int fides_server_cancel(fides_server *srv, uint64_t id);
int fides_server_pause(fides_server *srv, int paused);
int fides_server_inject(fides_server *srv, int fault, int64_t arg);
int fides_server_stats_read(fides_server *srv, fides_server_stats *out);
int64_t fides_now_ns(void);

/*
 * Homomorphic programs (bootstrapping, Sec. III-F7).  A program is a list of
 * instructions over virtual ciphertext registers, each written once, with the
 * tables they use: linear transforms (diagonal indices, device plaintexts in
 * evaluation form pre-rotated for the baby-step giant-step split, n1,
 * plaintext scale; see fides_linear_transform), scalar constants (host
 * residues, one per q-limb; entries beyond an instruction's level unused) and
 * keys.  Bootstrapping is the program ModRaise -> three linear transforms
 * (CoeffToSlot) -> conjugation split -> EvalMod polynomial and double-angle
 * steps -> three linear transforms (SlotToCoeff); with fewer slots than N/2
 * (sparse packing, Table IV) ModRaise is followed by a trace of ROT and HADD
 * steps.  Its tables are the precomputation the paper takes from OpenFHE
 * (Sec. III-B).
 *
 * Instructions (dst <- ...):
 *   MODRAISE a to `arg` limbs (a has one limb)     LT #arg of a
 *   RESCALE a                                      DROP a to its first `arg` limbs
 *   HADD / HSUB / HMULT a, b (same level; HMULT relinearises with the relin key)
 *   CONJ a (conjugation key)                       MULI a by i (arg = 1) or -i (arg = -1)
 *   CMULT a by constant #arg (scale times const_scale[arg])
 *   CADD constant #arg to a                        COPY a
 *   ROT a by `arg` slots (the rotation key of Galois element 5^arg mod 2N)
 *   CMAC: dst <- sum_t const[c_t] * reg[r_t] at `b` limbs, over term list #arg
 *         (terms r_t, c_t: lin_reg / lin_const[lin_start[arg] .. lin_start[arg+1]),
 *         1..32 terms, each register with at least b limbs, read in place;
 *         scale = scale(r_0) * const_scale[c_0])
 * fides_program_create checks the program (operands defined before use,
 * levels consistent, keys present; FIDES_ERR_ARG naming the instruction; a key
 * of another context or element: FIDES_ERR_KEY),
 * copies every host table (device plaintexts and keys are referenced and must
 * outlive the program) and maps the virtual registers onto as few
 * ciphertext-sized buffers as their lifetimes allow.
 * fides_program_info reports the device work buffer the program needs (words:
 * the register buffers, the linear transforms' buffers and a key-switching
 * scratch pool of the context's size), the buffer count and the output's limb
 * count.
 * fides_program_run executes it on `stream` from `in` (in_limbs limbs) into
 * `out` (the output register's limbs; out->scale = desc->out_scale).  It
 * touches no context scratch: runs of one or several programs on one context
 * with distinct work buffers may proceed concurrently on different streams.
 */
#define FIDES_I_MODRAISE 1
#define FIDES_I_LT 2
#define FIDES_I_RESCALE 3
#define FIDES_I_DROP 4
#define FIDES_I_HADD 5
#define FIDES_I_HSUB 6
#define FIDES_I_HMULT 7
#define FIDES_I_CONJ 8
#define FIDES_I_MULI 9
#define FIDES_I_CMULT 10
#define FIDES_I_CADD 11
#define FIDES_I_COPY 12
#define FIDES_I_CMAC 13
#define FIDES_I_ROT 14

typedef struct {
    int op, dst, a, b, arg;
} fides_instr;

typedef struct {
    int n_diag;
    const int *diag_idx;
    const uint64_t *const *dev_pts;
    int n1;
    double pt_scale;
} fides_lt;

typedef struct {
    int n_instr;
    const fides_instr *instr;
    int n_regs, in_reg, out_reg, in_limbs;
    double out_scale;
    int n_lt;
    const fides_lt *lt;
    int n_const;
    const uint64_t *const *consts;   /* host [n_const] arrays of L residues */
    const double *const_scale;
    const fides_key *relin_key, *conj_key;    /* NULL when the program needs none */
    int n_rot_keys;
    const fides_key *const *rot_keys;         /* found by Galois element (5^k mod 2N for a rotation by k) */
    int n_lin;                       /* CMAC term lists */
    const int *lin_start;            /* [n_lin + 1] offsets */
    const int *lin_reg, *lin_const;  /* [lin_start[n_lin]] */
} fides_program_desc;

typedef struct fides_program fides_program;

int fides_program_create(fides_ctx *ctx, const fides_program_desc *desc, fides_program **out);
int fides_program_info(const fides_program *prog, size_t *work_words, int *buffers, int *out_limbs);
int fides_program_run(fides_program *prog, const fides_ct *in, fides_ct *out, uint64_t *dev_work, size_t work_words,
                      void *stream);
void fides_program_destroy(fides_program *prog);

/*
 * Rescale that allocates nothing.  The paper has no counterpart: this entry
 * point serves callers that cannot allocate device memory when they call it
 * (a host application that owns every device allocation and hands the library
 * fixed buffers, or a service that reserves all device memory at start-up).
 * It computes exactly what fides_rescale computes, with the same arguments and
 * rules, but its scratch (2 * N words) lives in a static device array of
 * FIDES_NOALLOC_SCRATCH_WORDS = 2 * 65536 words (1 MiB) instead of the
 * context's pool; every GPU that loads the library holds that array until the
 * process exits.  The caller passes the inputs and outputs.
 *   - N above 65536 is rejected with FIDES_ERR_UNSUPPORTED.
 *   - The context's device must be current (FIDES_ERR_ARG otherwise).
 *   - The first call on a device looks up the array's device address with
 *     cudaGetSymbolAddress; make that first call before any stream capture.
 *     The address is kept until the process exits, so a device reset
 *     (cudaDeviceReset) after the first call is not supported (it also
 *     invalidates every context on that device).
 *   - It calls no cudaMalloc, cudaFree or other allocating routine.
 *   - Every call shares the one array, which keeps the last call's contents:
 *     calls whose work overlaps on the GPU (other streams, other threads)
 *     race on it.  Each call writes every scratch word before reading it.
 */
int fides_rescale_noalloc(fides_ctx *ctx, const fides_ct *a, fides_ct *out, void *stream);

/*
 * Tracing (a profiling aid, not part of the method).  While enabled, every
 * kernel launch and every public operation is bracketed by CUDA events on its
 * stream.  fides_trace_read() waits for the recorded events and writes one
 * entry per name (kernel names start with "k_", operations with "op_") in
 * first-seen order to out[0..max); *n_out receives the number of names.
 * `name` points to static storage.  fides_trace_reset() drops the records.
 * fides_kernel_launches() counts every kernel launched by the library since
 * it was loaded, traced or not.
 */
typedef struct {
    const char *name;
    uint64_t launches;
    double total_ms;
} fides_trace_stat;

/*
 * Measured ALU roofline (a profiling aid): the sustained rate, in 10^9
 * modular products per second, of the library's 64-bit Shoup product
 * (Sec. III-F2) run register-resident on every SM of the current device.
 * *ms_out (optional) receives the duration of one measurement launch.
 * Allocates a small device buffer for the kernel's output and synchronises.
 */
int fides_measure_modmul_peak(double *gmodmul_per_s, double *ms_out);

int fides_trace_enable(int on);
void fides_trace_reset(void);
int fides_trace_read(fides_trace_stat *out, int max, int *n_out);
uint64_t fides_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* FIDES_H */
