// Context creation: validates the primes, finds psi for each of them and
// precomputes every per-prime table the kernels read (Sec. III-E
// "Precomputation": constants are computed once, when the context is built).
// Unlike the paper's singleton, every context owns its device tables, so
// several parameter sets can live in one process.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "fides_internal.cuh"
#include "ntt.cuh"

typedef unsigned __int128 u128;

// ---------------------------------------------------------------------------
// Error state (thread-local message of the last failure)
// ---------------------------------------------------------------------------
static thread_local char g_err[512] = "";

int fides_set_error(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int fides_check_cuda(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return FIDES_OK;
    return fides_set_error(e == cudaErrorMemoryAllocation ? FIDES_ERR_NOMEM : FIDES_ERR_CUDA,
                           "%s: %s", what, cudaGetErrorString(e));
}

extern "C" const char *fides_last_error(void) { return g_err; }
extern "C" const char *fides_version(void) { return "fides-gb300 0.1 (sm_103a)"; }

// ---------------------------------------------------------------------------
// Host number theory (u128 products)
// ---------------------------------------------------------------------------
namespace {

u64 hmul(u64 a, u64 b, u64 q) { return (u64)((u128)a * b % q); }

u64 hpow(u64 a, u64 e, u64 q)
{
    u64 r = 1 % q;
    a %= q;
    for (; e; e >>= 1) {
        if (e & 1) r = hmul(r, a, q);
        a = hmul(a, a, q);
    }
    return r;
}

u64 hinv(u64 a, u64 q) { return hpow(a, q - 2, q); }

// Shoup companion floor(w * 2^64 / q) for w < q
u64 shoup_of(u64 w, u64 q) { return (u64)(((u128)w << 64) / q); }

TwPair pair_of(u64 w, u64 q) { return TwPair{w % q, shoup_of(w % q, q)}; }

// Miller-Rabin with the first twelve prime bases: exact below 3.3e24.
bool is_prime(u64 n)
{
    static const u64 B[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (u64 b : B)
        if (n % b == 0) return n == b;
    u64 d = n - 1;
    int s = 0;
    while (!(d & 1)) { d >>= 1; ++s; }
    for (u64 b : B) {
        u64 x = hpow(b, d, n);
        if (x == 1 || x == n - 1) continue;
        bool composite = true;
        for (int r = 1; r < s && composite; ++r) {
            x = hmul(x, x, n);
            if (x == n - 1) composite = false;
        }
        if (composite) return false;
    }
    return true;
}

// smallest generator of Z_q^* (q prime): test g^((q-1)/f) != 1 for every
// prime factor f of q - 1
u64 smallest_generator(u64 q)
{
    std::vector<u64> f;
    u64 n = q - 1;
    for (u64 p = 2; p * p <= n; p = (p == 2 ? 3 : p + 2)) {
        if (n % p == 0) {
            f.push_back(p);
            while (n % p == 0) n /= p;
        }
    }
    if (n > 1) f.push_back(n);
    for (u64 g = 2; g < q; ++g) {
        bool ok = true;
        for (u64 p : f)
            if (hpow(g, (q - 1) / p, q) == 1) { ok = false; break; }
        if (ok) return g;
    }
    return 0;
}

u64 bitrev(u64 x, int bits)
{
    u64 r = 0;
    for (int i = 0; i < bits; ++i) { r = (r << 1) | (x & 1); x >>= 1; }
    return r;
}

template <class T>
int upload(T **dptr, const std::vector<T> &h, const char *what)
{
    size_t bytes = sizeof(T) * (h.empty() ? 1 : h.size());
    int rc = fides_check_cuda(cudaMalloc((void **)dptr, bytes), what);
    if (rc) return rc;
    if (!h.empty()) rc = fides_check_cuda(cudaMemcpy(*dptr, h.data(), bytes, cudaMemcpyHostToDevice), what);
    return rc;
}

}  // namespace

extern "C" int fides_find_primes(int logN, int bits, int count, const uint64_t *exclude, int n_exclude,
                                 uint64_t *out)
{
    if (logN < 1 || logN > 20 || bits < logN + 2 || bits > 61 || count < 0 || (count && !out) ||
        n_exclude < 0 || (n_exclude && !exclude))
        return fides_set_error(FIDES_ERR_ARG, "fides_find_primes: bad arguments");
    u64 step = (u64)2 << logN;
    u64 q = ((u64)1 << bits) - step + 1;
    int found = 0;
    while (found < count && q > step) {
        bool skip = false;
        for (int i = 0; i < n_exclude; ++i) skip |= (exclude[i] == q);
        if (!skip && is_prime(q)) out[found++] = q;
        q -= step;
    }
    if (found < count) return fides_set_error(FIDES_ERR_PRIME, "fides_find_primes: only %d primes", found);
    return FIDES_OK;
}

extern "C" void fides_ctx_destroy(fides_ctx *c)
{
    if (!c) return;
    cudaFree(c->d_prime);
    cudaFree(c->d_tw);
    cudaFree(c->d_itw);
    cudaFree(c->d_mu_scale);
    cudaFree(c->d_mu_mat);
    cudaFree(c->d_md_scale);
    cudaFree(c->d_md_mat);
    cudaFree(c->d_md_pinv);
    cudaFree(c->d_md_negp);
    cudaFree(c->d_rs_qlinv);
    cudaFree(c->d_hr);
    cudaFree(c->d_mu_nscale);
    cudaFree(c->d_md_nscale);
    cudaFree(c->d_raise);
    cudaFree(c->d_tc);
    cudaFree(c->d_c32);
    cudaFree(c->d_status);
    cudaFree(c->scratch);
    for (int i = 0; i < c->n_spool; ++i) cudaFree(c->spool[i]);
    free(c);
}

extern "C" int fides_ctx_status(fides_ctx *c, int *flags)
{
    if (!c || !flags) return fides_set_error(FIDES_ERR_ARG, "fides_ctx_status: NULL argument");
    *flags = 0;
    int rc = fides_check_cuda(cudaDeviceSynchronize(), "fides_ctx_status");
    if (!rc) rc = fides_check_cuda(cudaMemcpy(flags, c->d_status, sizeof(int), cudaMemcpyDeviceToHost), "fides_ctx_status");
    if (!rc) rc = fides_check_cuda(cudaMemset(c->d_status, 0, sizeof(int)), "fides_ctx_status");
    return rc;
}

extern "C" int fides_ctx_add_stream(fides_ctx *c, void *stream)
{
    if (!c) return fides_set_error(FIDES_ERR_ARG, "fides_ctx_add_stream: ctx is NULL");
    static std::mutex reg;   // registrations of every context, one at a time
    std::lock_guard<std::mutex> lock(reg);
    const int n = c->n_spool;
    for (int i = 0; i < n; ++i)
        if (c->spool_stream[i] == stream) return FIDES_OK;
    if (n == FIDES_MAX_STREAMS)
        return fides_set_error(FIDES_ERR_ARG, "fides_ctx_add_stream: at most %d streams", FIDES_MAX_STREAMS);
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != c->device) cudaSetDevice(c->device);
    u64 *pool = nullptr;
    const int rc = fides_check_cuda(cudaMalloc((void **)&pool, c->scratch_words * sizeof(u64)),
                                    "fides_ctx_add_stream: scratch pool");
    if (prev != c->device) cudaSetDevice(prev);
    if (rc) return rc;
    c->spool_stream[n] = stream;
    c->spool[n] = pool;
    __atomic_store_n(&c->n_spool, n + 1, __ATOMIC_RELEASE);   // scratch_for reads the entry after this
    return FIDES_OK;
}

extern "C" int fides_ctx_set_rounding(fides_ctx *c, int mode)
{
    if (!c || (mode != FIDES_ROUND_FLOOR && mode != FIDES_ROUND_NEAREST))
        return fides_set_error(FIDES_ERR_ARG, "fides_ctx_set_rounding: mode must be FIDES_ROUND_FLOOR or _NEAREST");
    c->round_nearest = mode == FIDES_ROUND_NEAREST;
    return FIDES_OK;
}

extern "C" int fides_ctx_rounding(const fides_ctx *c)
{
    return c && c->round_nearest ? FIDES_ROUND_NEAREST : FIDES_ROUND_FLOOR;
}

extern "C" int fides_ctx_tensor_bconv(const fides_ctx *c)
{
    return c && c->tc_on == 3 ? 1 : 0;
}

extern "C" int fides_ctx_beta(const fides_ctx *c, int n_limbs)
{
    if (!c || n_limbs < 1) return 0;
    return (n_limbs + c->alpha - 1) / c->alpha;
}

extern "C" uint64_t fides_ctx_psi(const fides_ctx *c, int i)
{
    if (!c || i < 0 || i >= c->L + c->K) return 0;
    return c->psi[i];
}

extern "C" uint64_t fides_galois_elt(const fides_ctx *c, int64_t steps)
{
    if (!c) return 0;
    int64_t half = c->N / 2;
    int64_t k = ((steps % half) + half) % half;
    return hpow(5, (u64)k, 2 * (u64)c->N);
}

// ---------------------------------------------------------------------------
// Switching-key handles
// ---------------------------------------------------------------------------
int fides_check_key(const fides_ctx *c, const fides_key *k, u64 g, const char *what)
{
    if (!k) return fides_set_error(FIDES_ERR_ARG, "%s: key handle is NULL", what);
    if (k->ctx != c) return fides_set_error(FIDES_ERR_KEY, "%s: the key was registered with another context", what);
    if (g != FIDES_GALOIS_ANY && k->g != g)
        return fides_set_error(FIDES_ERR_KEY, "%s: the key switches from Galois element %llu, the operation needs %llu",
                               what, (unsigned long long)k->g, (unsigned long long)g);
    return FIDES_OK;
}

extern "C" int fides_key_register(fides_ctx *c, const uint64_t *dev_key, uint64_t g, fides_key **out)
{
    const char *fn = "fides_key_register";
    if (!out) return fides_set_error(FIDES_ERR_ARG, "%s: out is NULL", fn);
    *out = nullptr;
    if (!c || !dev_key) return fides_set_error(FIDES_ERR_ARG, "%s: NULL argument", fn);
    if ((uintptr_t)dev_key % 8) return fides_set_error(FIDES_ERR_ARG, "%s: key buffer not 8-byte aligned", fn);
    if (g != 0 && (g % 2 == 0 || g >= 2 * (u64)c->N))
        return fides_set_error(FIDES_ERR_ARG, "%s: Galois element %llu is neither 0 nor odd below 2N = %d", fn,
                               (unsigned long long)g, 2 * c->N);
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, dev_key) != cudaSuccess) {
        cudaGetLastError();
        return fides_set_error(FIDES_ERR_ARG, "%s: the key buffer is not CUDA memory", fn);
    }
    const bool on_dev = (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == c->device;
    if (!on_dev) return fides_set_error(FIDES_ERR_ARG, "%s: the key buffer is not memory of device %d", fn, c->device);
    // whatever filled the buffer (a copy, a kernel of this library still
    // running under programmatic launch) finishes before the key is used
    int cur = -1;
    if (int rc = fides_check_cuda(cudaGetDevice(&cur), fn)) return rc;
    if (cur != c->device && fides_check_cuda(cudaSetDevice(c->device), fn)) return FIDES_ERR_CUDA;
    int rc = fides_check_cuda(cudaDeviceSynchronize(), fn);
    if (cur != c->device) cudaSetDevice(cur);
    if (rc) return rc;
    fides_key *k = (fides_key *)calloc(1, sizeof(fides_key));
    if (!k) return fides_set_error(FIDES_ERR_NOMEM, "%s: host allocation", fn);
    k->ctx = c;
    k->data = dev_key;
    k->g = g;
    *out = k;
    return FIDES_OK;
}

extern "C" void fides_key_destroy(fides_key *k) { free(k); }

extern "C" uint64_t fides_key_galois(const fides_key *k) { return k ? k->g : 0; }

// fp16 bits of an integer 0 <= k < 256 (exact: at most 8 significant bits).
static uint16_t f16_of_byte(unsigned k)
{
    if (k == 0) return 0;
    int e = 7;
    while (!(k >> e)) --e;
    return (uint16_t)(((e + 15) << 10) | ((k << (10 - e)) & 0x3FF));
}

// Appends the tensor-core image of one conversion matrix to img (bconv_tc.cuh):
// for target t (prime targets[t]) and source s (constant cst(s, z)), one 8 x 8
// core matrix of fp16 values in 16-byte rows, row b, column a = byte b of
// (cst(s, z) * 2^(8a) mod p_z); then, per target, the offset block (2^15 in
// column 0 of every row, zeros elsewhere) and, with corr, the correction block
// (byte b of corr[z] in columns 0..3 of row b: the conversion kernel puts up
// to four partial counts there, see bconv_tc.cuh).  Targets are padded to an
// even count, and the source, offset and correction blocks to an even count,
// with zero blocks.  Returns the image's byte offset.
template <class F>
static size_t tc_image(const u64 *primes, const std::vector<int> &targets, int ns, F cst,
                       std::vector<uint16_t> &img, const u64 *corr = nullptr)
{
    const size_t off = img.size() * 2;
    const int nd = (int)targets.size(), ndp = (nd + 1) & ~1, nsp = (ns + 2 + (corr ? 1 : 0)) & ~1;
    img.resize(img.size() + (size_t)ndp * nsp * 64, 0);
    uint16_t *base = img.data() + off / 2;
    for (int t = 0; t < nd; ++t) {
        const int z = targets[t];
        const u64 p = primes[z];
        for (int src = 0; src < ns; ++src) {
            uint16_t *blk = base + ((size_t)t * nsp + src) * 64;
            u64 v = cst(src, z) % p;
            for (int a = 0; a < 8; ++a) {
                for (int b = 0; b < 8; ++b) blk[b * 8 + a] = f16_of_byte((unsigned)((v >> (8 * b)) & 255));
                v = (u64)(((u128)v << 8) % p);
            }
        }
        // offset column: 2^15 (fp16 0x7800) against A's 256 adds 2^23 to every sum
        uint16_t *blk = base + ((size_t)t * nsp + ns) * 64;
        for (int b = 0; b < 8; ++b) blk[b * 8] = 0x7800;
        if (corr) {
            uint16_t *cb = base + ((size_t)t * nsp + ns + 1) * 64;
            for (int b = 0; b < 8; ++b)
                for (int a = 0; a < 4; ++a) cb[b * 8 + a] = f16_of_byte((unsigned)((corr[z] >> (8 * b)) & 255));
        }
    }
    return off;
}

// Scratch words one top-level operation needs (layout: keyswitch.cu, plan.cuh).
static size_t scratch_words_for(int L, int K, int dnum, int alpha, int N)
{
    int beta = (L + alpha - 1) / alpha;
    (void)dnum;
    size_t ne = (size_t)(L + K);
    // d2 / rotated c1 (L) + coeff copy (L) + ext (beta*ne) + acc (2*ne)
    // + P-limb INTT (2K) + conversion outputs (2L) + two spare limbs
    // + HMult fused with Rescale: the tensor product d0, d1 (2L) and the
    //   coefficient forms of their and the accumulators' dropped limb (4)
    return (size_t)N * (2 * (size_t)L + beta * ne + 2 * ne + 2 * (size_t)K + 2 * (size_t)L + 2 + 2 * (size_t)L + 4);
}

extern "C" int fides_ctx_create(int logN, int L, int dnum, const uint64_t *primes, int K, fides_ctx **out)
{
    if (!out) return fides_set_error(FIDES_ERR_ARG, "fides_ctx_create: out is NULL");
    *out = nullptr;
    if (!primes || L < 1 || K < 1 || L + K > FIDES_MAX_PRIMES || dnum < 1 || dnum > L)
        return fides_set_error(FIDES_ERR_ARG, "fides_ctx_create: bad sizes (L=%d K=%d dnum=%d)", L, K, dnum);
    if (logN < 12 || logN > 17)
        return fides_set_error(FIDES_ERR_UNSUPPORTED, "fides_ctx_create: logN=%d (supported: 12..17)", logN);
    int alpha = (L + dnum - 1) / dnum;
    if (alpha > FIDES_MAX_SRC || K > FIDES_MAX_SRC)
        return fides_set_error(FIDES_ERR_UNSUPPORTED, "fides_ctx_create: digit size %d or K=%d above %d",
                               alpha, K, FIDES_MAX_SRC);
    if ((L + alpha - 1) / alpha > FIDES_MAX_DIGITS)
        return fides_set_error(FIDES_ERR_UNSUPPORTED, "fides_ctx_create: more than %d digits", FIDES_MAX_DIGITS);
    const int N = 1 << logN, np = L + K;
    for (int i = 0; i < np; ++i) {
        u64 q = primes[i];
        if (q >= ((u64)1 << 61) || !is_prime(q) || (q - 1) % (2 * (u64)N) != 0)
            return fides_set_error(FIDES_ERR_PRIME, "fides_ctx_create: primes[%d]=%llu is not an NTT prime < 2^61",
                                   i, (unsigned long long)q);
        for (int k = 0; k < i; ++k)
            if (primes[k] == q) return fides_set_error(FIDES_ERR_PRIME, "fides_ctx_create: repeated prime");
    }

    fides_ctx *c = (fides_ctx *)calloc(1, sizeof(fides_ctx));
    if (!c) return fides_set_error(FIDES_ERR_NOMEM, "fides_ctx_create: host allocation");
    cudaGetDevice(&c->device);
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
    c->logN = logN; c->N = N; c->L = L; c->K = K; c->dnum = dnum; c->alpha = alpha;
    memcpy(c->primes, primes, sizeof(u64) * np);

    // per-prime constants and twiddles
    std::vector<PrimeInfo> pinfo(np);
    std::vector<TwPair> tw((size_t)np * N), itw((size_t)np * N);
    for (int i = 0; i < np; ++i) {
        u64 q = primes[i];
        u64 g = smallest_generator(q);
        u64 psi = hpow(g, (q - 1) / (2 * (u64)N), q);
        c->psi[i] = psi;
        u64 ipsi = hinv(psi, q);
        PrimeInfo &P = pinfo[i];
        P.q = q; P.q2 = 2 * q;
        P.mu = (u64)(((u128)1 << 64) / q);
        P.r64 = (u64)(((u128)1 << 64) % q);
        P.r64p = shoup_of(P.r64, q);
        P.ninv = hinv((u64)N % q, q);
        P.ninvp = shoup_of(P.ninv, q);
        P.ninvw = P.ninvwp = 0;   // after the twiddles
        P.bmu = (u64)(((u128)1 << (63 + (64 - __builtin_clzll(q)))) / q);
        // powers in natural order, then scattered to bit-reversed positions
        u64 x = 1, y = 1;
        for (int k = 0; k < N; ++k) {
            size_t at = (size_t)i * N + bitrev(k, logN);
            tw[at] = pair_of(x, q);
            itw[at] = pair_of(y, q);
            x = hmul(x, psi, q);
            y = hmul(y, ipsi, q);
        }
        P.ninvw = hmul(P.ninv, itw[(size_t)i * N + 1].w, q);
        P.ninvwp = shoup_of(P.ninvw, q);
    }

    // ModUp tables per (nl, j)
    std::vector<TwPair> mu_scale((size_t)L * dnum * alpha);
    std::vector<u64> mu_mat((size_t)L * dnum * alpha * np);
    for (int nl = 1; nl <= L; ++nl) {
        int beta = (nl + alpha - 1) / alpha;
        for (int j = 0; j < beta; ++j) {
            int lo = j * alpha, hi = std::min(lo + alpha, nl);
            size_t off = ((size_t)(nl - 1) * dnum + j) * alpha;
            for (int i = lo; i < hi; ++i) {
                u64 qi = primes[i];
                u64 prod = 1;
                for (int k = lo; k < hi; ++k)
                    if (k != i) prod = hmul(prod, primes[k] % qi, qi);
                mu_scale[off + (i - lo)] = pair_of(hinv(prod, qi), qi);
                for (int z = 0; z < np; ++z) {
                    u64 p = primes[z], h = 1;
                    for (int k = lo; k < hi; ++k)
                        if (k != i) h = hmul(h, primes[k] % p, p);
                    mu_mat[(off + (i - lo)) * np + z] = h;
                }
            }
        }
    }

    // ModDown tables
    std::vector<TwPair> md_scale(K), md_pinv(L);
    std::vector<u64> md_mat((size_t)K * np);
    for (int k = 0; k < K; ++k) {
        u64 pk = primes[L + k], prod = 1;
        for (int m = 0; m < K; ++m)
            if (m != k) prod = hmul(prod, primes[L + m] % pk, pk);
        md_scale[k] = pair_of(hinv(prod, pk), pk);
        for (int z = 0; z < np; ++z) {
            u64 p = primes[z], h = 1;
            for (int m = 0; m < K; ++m)
                if (m != k) h = hmul(h, primes[L + m] % p, p);
            md_mat[(size_t)k * np + z] = h;
        }
    }
    // md_negp[z] = -P mod prime z: the ModDown conversion from centred
    // residues is the canonical one plus c (-P), c the number of residues in
    // the upper half (round-to-nearest mode)
    std::vector<u64> md_negp((size_t)np, 0);
    for (int i = 0; i < L; ++i) {
        u64 qi = primes[i], P = 1;
        for (int k = 0; k < K; ++k) P = hmul(P, primes[L + k] % qi, qi);
        md_pinv[i] = pair_of(hinv(P, qi), qi);
        md_negp[i] = P ? qi - P : 0;
    }

    // Tensor-core conversion images: ModUp per (nl, j) with targets in the
    // order of the job's runs ([0, lo), [hi, nl), P), ModDown with targets
    // [0, L) (a level nl uses the first nl).
    std::vector<uint16_t> tc_img;
    c->tc_on = (alpha <= FIDES_TC_MAX_SRC ? 1 : 0) | (K <= FIDES_TC_MAX_SRC ? 2 : 0);
    c->tc_big = 1;
    for (int z = 0; z < np; ++z)
        if (primes[z] < ((u64)1 << 48)) c->tc_big = 0;
    if (c->tc_on & 1) {
        for (int nl = 1; nl <= L; ++nl) {
            int beta = (nl + alpha - 1) / alpha;
            for (int j = 0; j < beta; ++j) {
                int lo = j * alpha, hi = std::min(lo + alpha, nl);
                size_t off = ((size_t)(nl - 1) * dnum + j) * alpha;
                std::vector<int> tg;
                for (int z = 0; z < lo; ++z) tg.push_back(z);
                for (int z = hi; z < nl; ++z) tg.push_back(z);
                for (int z = L; z < np; ++z) tg.push_back(z);
                c->tc_mu_off[nl - 1][j] = tc_image(primes, tg, hi - lo,
                                                   [&](int src, int z) { return mu_mat[(off + src) * np + z]; },
                                                   tc_img);
            }
        }
    }
    if (c->tc_on & 2) {
        std::vector<int> tg;
        for (int z = 0; z < L; ++z) tg.push_back(z);
        c->tc_md_off = tc_image(primes, tg, K, [&](int src, int z) { return md_mat[(size_t)src * np + z]; }, tc_img,
                                md_negp.data());
    }
    if (tc_img.empty()) tc_img.resize(64, 0);
    std::vector<TwPair> c32((size_t)np);
    for (int z = 0; z < np; ++z) c32[z] = pair_of((u64)(((u128)1 << 32) % primes[z]), primes[z]);

    // Rescale tables
    std::vector<TwPair> rs((size_t)L * L);
    for (int l = 1; l < L; ++l)
        for (int i = 0; i < l; ++i) rs[(size_t)l * L + i] = pair_of(hinv(primes[l] % primes[i], primes[i]), primes[i]);

    // HMult fused with Rescale: (P^-1, q_l^-1) mod q_i
    std::vector<TwPair> hr((size_t)L * L * 2);
    for (int l = 1; l < L; ++l)
        for (int i = 0; i < l; ++i) {
            hr[((size_t)l * L + i) * 2] = md_pinv[i];
            hr[((size_t)l * L + i) * 2 + 1] = rs[(size_t)l * L + i];
        }

    // ModRaise: q_0 mod q_i (the centred lift subtracts q_0 from the upper half)
    std::vector<TwPair> raise((size_t)L);
    for (int i = 0; i < L; ++i) raise[i] = pair_of(primes[0] % primes[i], primes[i]);
    // multiplication by X^(N/2): i_q = psi^(N/2) mod q_i (a square root of -1)
    std::vector<TwPair> iroot((size_t)L);
    for (int i = 0; i < L; ++i) iroot[i] = pair_of(hpow(c->psi[i], (u64)N / 2, primes[i]), primes[i]);

    // combined N^-1 * qhat^-1 constants of the inverse NTTs feeding a conversion
    std::vector<TwPair> mu_ns((size_t)L * (L + 1)), md_ns(2 * (size_t)np);
    auto with_w1 = [&](std::vector<TwPair> &t, size_t at, u64 cval, int pi) {
        const u64 q = primes[pi];
        t[2 * at] = pair_of(cval, q);
        t[2 * at + 1] = pair_of(hmul(cval, itw[(size_t)pi * N + 1].w, q), q);
    };
    for (int nl = 1; nl <= L; ++nl) {
        for (int i = 0; i < nl; ++i) {
            const int j = i / alpha, lo = j * alpha, hi = std::min(lo + alpha, nl);
            u64 qi = primes[i], prod = 1;
            for (int k = lo; k < hi; ++k)
                if (k != i) prod = hmul(prod, primes[k] % qi, qi);
            with_w1(mu_ns, (size_t)nl * (nl - 1) / 2 + i, hmul(hinv(prod, qi), pinfo[i].ninv, qi), i);
        }
    }
    for (int k = 0; k < K; ++k) {
        u64 pk = primes[L + k];
        with_w1(md_ns, (size_t)L + k, hmul(md_scale[k].w, pinfo[L + k].ninv, pk), L + k);
    }

    int rc = FIDES_OK;
    if (!rc) rc = upload(&c->d_prime, pinfo, "tables");
    if (!rc) rc = upload(&c->d_tw, tw, "twiddles");
    if (!rc) rc = upload(&c->d_itw, itw, "twiddles");
    if (!rc) rc = upload(&c->d_mu_scale, mu_scale, "modup tables");
    if (!rc) rc = upload(&c->d_mu_mat, mu_mat, "modup tables");
    if (!rc) rc = upload(&c->d_md_scale, md_scale, "moddown tables");
    if (!rc) rc = upload(&c->d_md_mat, md_mat, "moddown tables");
    if (!rc) rc = upload(&c->d_md_pinv, md_pinv, "moddown tables");
    if (!rc) rc = upload(&c->d_md_negp, md_negp, "moddown tables");
    if (!rc) rc = upload(&c->d_rs_qlinv, rs, "rescale tables");
    if (!rc) rc = upload(&c->d_hr, hr, "rescale tables");
    if (!rc) rc = upload(&c->d_mu_nscale, mu_ns, "modup tables");
    if (!rc) rc = upload(&c->d_md_nscale, md_ns, "moddown tables");
    if (!rc) rc = upload(&c->d_raise, raise, "modraise tables");
    if (!rc) rc = upload(&c->d_tc, tc_img, "tensor-core conversion tables");
    if (!rc) rc = upload(&c->d_c32, c32, "tensor-core conversion tables");
    if (!rc) {
        std::vector<int> zero(1, 0);
        rc = upload(&c->d_status, zero, "status word");
    }
    for (int i = 0; i < L; ++i) c->iroot[i] = iroot[i];
    if (!rc) {
        c->scratch_words = scratch_words_for(L, K, dnum, alpha, N);
        rc = fides_check_cuda(cudaMalloc((void **)&c->scratch, c->scratch_words * sizeof(u64)), "scratch pool");
    }
    if (rc) {
        fides_ctx_destroy(c);
        return rc;
    }
    ntt_default_variants(c);
    *out = c;
    return FIDES_OK;
}
