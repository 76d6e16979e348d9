// NTT launchers and the tile-width autotuner.
//
// The paper trades launch overhead against locality with a "limb batch"
// context parameter (Sec. III-F1) whose best value depends on the GPU
// (Sec. IV).  Here one launch always covers every limb of a step; what is left
// to tune is the tile width of each pass, which decides how many CTAs a launch
// has and so how much of its last wave is empty.  Five variants of each pass
// of a two-pass transform (logN 13..17) are compiled -- at logN=16, 16, 8 or
// 4 columns/rows per CTA (256, 128 or 64 threads) with up to 80 registers (3,
// 6 or 12 resident CTAs per SM), and 4 or 8 per CTA with up to 64 registers
// (16 or 8 per SM); other sizes scale the resident-CTA target to the same
// register budget (ntt_impl.cuh) -- and the context keeps, per pass kind and
// limb count, the variant to launch: a fixed default, or the fastest measured
// one after fides_ctx_autotune.  The launchers of each ring degree live in
// ntt_l12.cu .. ntt_l17.cu; this file dispatches on the context's logN.
#include <algorithm>
#include <cstring>
#include <vector>

#include "ntt_impl.cuh"

#define FIDES_NTT_DISPATCH(fn, ...)                                  \
    switch (c->logN) {                                               \
    case 12: return fn##_12(__VA_ARGS__);                            \
    case 13: return fn##_13(__VA_ARGS__);                            \
    case 14: return fn##_14(__VA_ARGS__);                            \
    case 15: return fn##_15(__VA_ARGS__);                            \
    case 16: return fn##_16(__VA_ARGS__);                            \
    default: return fn##_17(__VA_ARGS__);                            \
    }

int ntt_fwd_canon(const fides_ctx *c, const LimbSet &s, cudaStream_t st) { FIDES_NTT_DISPATCH(ntt_fwd_canon, c, s, st) }
int ntt_fwd_submul(const fides_ctx *c, const LimbSet &s, cudaStream_t st) { FIDES_NTT_DISPATCH(ntt_fwd_submul, c, s, st) }
int ntt_fwd_switch_submul(const fides_ctx *c, const LimbSet &s, cudaStream_t st)
{
    FIDES_NTT_DISPATCH(ntt_fwd_switch_submul, c, s, st)
}
int ntt_fwd_submul_rot(const fides_ctx *c, const LimbSet &s, cudaStream_t st)
{
    FIDES_NTT_DISPATCH(ntt_fwd_submul_rot, c, s, st)
}
int ntt_fwd_raise(const fides_ctx *c, const LimbSet &s, cudaStream_t st) { FIDES_NTT_DISPATCH(ntt_fwd_raise, c, s, st) }
int ntt_fwd_hmrs(const fides_ctx *c, const LimbSet &s, cudaStream_t st) { FIDES_NTT_DISPATCH(ntt_fwd_hmrs, c, s, st) }
int ntt_inv_canon(const fides_ctx *c, const LimbSet &s, cudaStream_t st) { FIDES_NTT_DISPATCH(ntt_inv_canon, c, s, st) }

namespace {
void tune_one(const fides_ctx *c, int kind, int v, const LimbSet &s, cudaStream_t st)
{
    FIDES_NTT_DISPATCH(ntt_tune_one, c, kind, v, s, st)
}
}  // namespace

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
    if (c->logN == 12) return FIDES_OK;   // one variant only
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
                    tune_one(c, kind, v, S, st);
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
    if (c->logN == 12) return (1 << 8) | 3;
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
