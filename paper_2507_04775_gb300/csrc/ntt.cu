// NTT launchers and the tile-width autotuner.
//
// The paper trades launch overhead against locality with a "limb batch"
// context parameter (Sec. III-F1) whose best value depends on the GPU
// (Sec. IV).  Here one launch always covers every limb of a step; what is left
// to tune is the tile width of each pass, which decides how many CTAs a launch
// has and so how much of its last wave is empty.  Three variants of each
// logN=16 pass are compiled -- 16, 8 or 4 columns/rows per CTA (256, 128 or 64
// threads) with up to 80 registers (3, 6 or 12 resident CTAs per SM), and 4
// or 8 per CTA with up to 64 registers (16 or 8 per SM) -- and the context keeps, per pass
// kind and limb count, the variant to launch: a fixed default, or the fastest
// measured one after fides_ctx_autotune.
#include <algorithm>
#include <cstring>
#include <vector>

#include "fides_internal.cuh"
#include "ntt.cuh"

namespace {

constexpr int NVAR = 5;
constexpr int VAR_CT[NVAR] = {16, 8, 4, 4, 8};
constexpr int VAR_MINB[NVAR] = {3, 6, 12, 16, 8};   // 3/6/12: up to 80 registers; 16/8: up to 64

enum PassKind { FWD_COLS = 0, FWD_ROWS = 1, INV_ROWS = 2, INV_COLS = 3 };

int variant_of(const fides_ctx *c, int kind, int total)
{
    return c->ntt_var[kind][total > FIDES_TUNE_MAX ? FIDES_TUNE_MAX : total];
}

template <int V, int KIND, bool INV, bool NINV, class Pro, class Epi>
void launch_pass(const fides_ctx *c, const LimbSet &set, const TwPair *tw, Pro pro, Epi epi, cudaStream_t st,
                 const char *name)
{
    constexpr int CT = VAR_CT[V], MINB = VAR_MINB[V];
    auto k = k_ntt<16, 8, KIND, INV, NINV, CT, MINB, Pro, Epi>;
    dim3 grid(256 / CT, set.total), block(16 * CT);
    FIDES_LAUNCH(name, st, k, grid, block, set, (const PrimeInfo *)c->d_prime, tw, pro, epi);
}

template <int KIND, bool INV, bool NINV, class Pro, class Epi>
void launch_pass_v(int v, const fides_ctx *c, const LimbSet &set, const TwPair *tw, Pro pro, Epi epi,
                   cudaStream_t st, const char *name)
{
    switch (v) {
    case 0: launch_pass<0, KIND, INV, NINV>(c, set, tw, pro, epi, st, name); break;
    case 1: launch_pass<1, KIND, INV, NINV>(c, set, tw, pro, epi, st, name); break;
    case 2: launch_pass<2, KIND, INV, NINV>(c, set, tw, pro, epi, st, name); break;
    case 3: launch_pass<3, KIND, INV, NINV>(c, set, tw, pro, epi, st, name); break;
    default: launch_pass<4, KIND, INV, NINV>(c, set, tw, pro, epi, st, name); break;
    }
}

template <class Pro, class Epi>
int forward(const fides_ctx *c, const LimbSet &set, Pro pro, Epi epi, cudaStream_t st)
{
    if (set.total == 0) return FIDES_OK;
    if (c->logN == 16) {
        launch_pass_v<0, false, false>(variant_of(c, FWD_COLS, set.total), c, set, c->d_tw, pro, EpiLazy{}, st,
                                       "k_ntt_fwd_cols");
        launch_pass_v<1, false, false>(variant_of(c, FWD_ROWS, set.total), c, set, c->d_tw, ProDst{}, epi, st,
                                       "k_ntt_fwd_rows");
    } else {
        auto k = k_ntt<12, 12, 2, false, false, 16, 3, Pro, Epi>;
        FIDES_LAUNCH("k_ntt_fwd_limb", st, k, dim3(1, set.total), dim3(256), set, (const PrimeInfo *)c->d_prime,
                     (const TwPair *)c->d_tw, pro, epi);
    }
    return fides_check_cuda(cudaGetLastError(), "ntt forward launch");
}

template <class Pro, class Epi>
int inverse(const fides_ctx *c, const LimbSet &set, Pro pro, Epi epi, cudaStream_t st)
{
    if (set.total == 0) return FIDES_OK;
    if (c->logN == 16) {
        launch_pass_v<1, true, false>(variant_of(c, INV_ROWS, set.total), c, set, c->d_itw, pro, EpiLazy{}, st,
                                      "k_ntt_inv_rows");
        launch_pass_v<0, true, true>(variant_of(c, INV_COLS, set.total), c, set, c->d_itw, ProDst{}, epi, st,
                                     "k_ntt_inv_cols");
    } else {
        auto k = k_ntt<12, 12, 2, true, true, 16, 3, Pro, Epi>;
        FIDES_LAUNCH("k_ntt_inv_limb", st, k, dim3(1, set.total), dim3(256), set, (const PrimeInfo *)c->d_prime,
                     (const TwPair *)c->d_itw, pro, epi);
    }
    return fides_check_cuda(cudaGetLastError(), "ntt inverse launch");
}

// one pass of kind `kind` with variant v (for the autotuner)
void launch_one(const fides_ctx *c, int kind, int v, const LimbSet &set, cudaStream_t st)
{
    switch (kind) {
    case FWD_COLS: launch_pass_v<0, false, false>(v, c, set, c->d_tw, ProSrc{}, EpiLazy{}, st, "k_ntt_tune"); break;
    case FWD_ROWS: launch_pass_v<1, false, false>(v, c, set, c->d_tw, ProDst{}, EpiCanon{}, st, "k_ntt_tune"); break;
    case INV_ROWS: launch_pass_v<1, true, false>(v, c, set, c->d_itw, ProPrep{16}, EpiLazy{}, st, "k_ntt_tune"); break;
    default: launch_pass_v<0, true, true>(v, c, set, c->d_itw, ProDst{}, EpiCanon{}, st, "k_ntt_tune"); break;
    }
}

}  // namespace

int ntt_fwd_canon(const fides_ctx *c, const LimbSet &s, cudaStream_t st) { return forward(c, s, ProSrc{}, EpiCanon{}, st); }
int ntt_fwd_submul(const fides_ctx *c, const LimbSet &s, cudaStream_t st) { return forward(c, s, ProSrc{}, EpiSubMul{}, st); }
int ntt_fwd_switch_submul(const fides_ctx *c, const LimbSet &s, cudaStream_t st)
{
    return forward(c, s, ProSwitchMod{}, EpiSubMul{}, st);
}
int ntt_fwd_submul_rot(const fides_ctx *c, const LimbSet &s, cudaStream_t st)
{
    return forward(c, s, ProSrc{}, EpiSubMulRot{c->logN}, st);
}
int ntt_fwd_raise(const fides_ctx *c, const LimbSet &s, cudaStream_t st)
{
    return forward(c, s, ProRaise{}, EpiCanon{}, st);
}
int ntt_inv_canon(const fides_ctx *c, const LimbSet &s, cudaStream_t st)
{
    return inverse(c, s, ProPrep{c->logN}, EpiCanon{}, st);
}

// Default variants before autotuning: 8 columns per CTA for column passes and
// 4 rows per CTA for row passes (the choice the autotuner makes on GB300 for
// almost every limb count between 1 and 128).
void ntt_default_variants(fides_ctx *c)
{
    for (int n = 0; n <= FIDES_TUNE_MAX; ++n) {
        c->ntt_var[FWD_COLS][n] = 1;
        c->ntt_var[INV_COLS][n] = 1;
        c->ntt_var[FWD_ROWS][n] = 2;
        c->ntt_var[INV_ROWS][n] = 2;
    }
}

extern "C" int fides_ctx_autotune(fides_ctx *c, int max_limbs, void *stream)
{
    if (!c) return fides_set_error(FIDES_ERR_ARG, "fides_ctx_autotune: ctx is NULL");
    if (c->logN != 16) return FIDES_OK;   // one variant only
    const int np = c->L + c->K;
    const size_t limbs_avail = c->scratch_words / c->N;
    int maxn = std::min(std::min(max_limbs, FIDES_TUNE_MAX), (int)limbs_avail);
    if (maxn < 1) return fides_set_error(FIDES_ERR_ARG, "fides_ctx_autotune: max_limbs < 1");
    cudaStream_t st = (cudaStream_t)stream;
    const int was = fides_trace_set(0);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = FIDES_OK;
    for (int n = 1; n <= maxn && !rc; ++n) {
        LimbSet S;
        memset(&S, 0, sizeof(S));
        for (int z0 = 0; z0 < n && S.nseg < FIDES_MAX_SEG; z0 += np) {
            Seg &g = S.seg[S.nseg++];
            u64 *p = c->scratch + (size_t)z0 * c->N;
            g.src = p; g.dst = p; g.aux = nullptr; g.out = nullptr; g.side = nullptr; g.cst = nullptr; g.g = 0;
            g.count = std::min(np, n - z0); g.prime0 = 0; g.src_step = 1; g.mode = 0; g.pstride = 0;
            S.total += g.count;
        }
        for (int kind = 0; kind < 4 && !rc; ++kind) {
            float best_ms = 0.f;
            int best = 0;
            for (int v = 0; v < NVAR && !rc; ++v) {
                float tmin = 0.f;
                for (int r = 0; r < 4; ++r) {
                    cudaEventRecord(e0, st);
                    launch_one(c, kind, v, S, st);
                    cudaEventRecord(e1, st);
                    rc = fides_check_cuda(cudaEventSynchronize(e1), "fides_ctx_autotune");
                    if (rc) break;
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (r > 0 && (r == 1 || ms < tmin)) tmin = ms;   // the first run warms up
                }
                if (v == 0 || tmin < best_ms) { best_ms = tmin; best = v; }
            }
            c->ntt_var[kind][n] = (unsigned char)best;
        }
    }
    // counts above the tuned range keep the widest tile when it won at the top
    for (int kind = 0; kind < 4; ++kind)
        for (int n = maxn + 1; n <= FIDES_TUNE_MAX; ++n) c->ntt_var[kind][n] = c->ntt_var[kind][maxn];
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    fides_trace_set(was);
    return rc;
}

extern "C" int fides_ctx_ntt_tile(const fides_ctx *c, int pass, int n_limbs)
{
    if (!c || pass < 0 || pass > 3 || n_limbs < 0) return 0;
    if (c->logN != 16) return (1 << 8) | 3;
    const int v = variant_of(c, pass, n_limbs);
    return (VAR_CT[v] << 8) | VAR_MINB[v];
}

extern "C" int fides_ctx_tune_table(fides_ctx *c, unsigned char *table, int set)
{
    if (!c || !table) return fides_set_error(FIDES_ERR_ARG, "fides_ctx_tune_table: NULL argument");
    const size_t n = sizeof(c->ntt_var);
    if (!set) {
        memcpy(table, c->ntt_var, n);
        return FIDES_OK;
    }
    for (size_t i = 0; i < n; ++i)
        if (table[i] >= NVAR) return fides_set_error(FIDES_ERR_ARG, "fides_ctx_tune_table: variant %d out of range", table[i]);
    memcpy(c->ntt_var, table, n);
    return FIDES_OK;
}
