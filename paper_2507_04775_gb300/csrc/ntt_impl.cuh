// NTT launchers for one ring degree, instantiated once per logN in its own
// translation unit (ntt_l12.cu .. ntt_l17.cu) so that the many kernel
// instances compile in parallel; ntt.cu dispatches on the context's logN.
//
// logN = 12: one tile per limb (KIND 2).  logN = 13..17: the paper's two-pass
// decomposition (Sec. III-F4) with a column pass of S_col stages on columns
// of stride 2^(logN - S_col) and a row pass of S_row stages on contiguous rows:
//   logN   13   14   15   16   17
//   S_col   7    7    8    8    9
//   S_row   6    7    7    8    8
// Each pass has five compiled tile variants (columns/rows per CTA and the
// resident-CTA target, chosen per pass kind and limb count; see ntt.cu).
#pragma once

#include <algorithm>
#include <cstring>

#include "fides_internal.cuh"
#include "ntt.cuh"

namespace {

constexpr int NVAR = 5;
constexpr int VAR_CT[NVAR] = {16, 8, 4, 4, 8};
constexpr int VAR_MINB[NVAR] = {3, 6, 12, 16, 8};   // at 256-element passes: 3/6/12 up to 80 registers, 16/8 up to 64

enum PassKind { FWD_COLS = 0, FWD_ROWS = 1, INV_ROWS = 2, INV_COLS = 3 };

inline int variant_of(const fides_ctx *c, int kind, int total)
{
    return c->ntt_var[kind][total > FIDES_TUNE_MAX ? FIDES_TUNE_MAX : total];
}

template <int LOGN>
struct Split {
    static constexpr int COL = LOGN <= 14 ? 7 : (LOGN <= 16 ? 8 : 9);
    static constexpr int ROW = LOGN - COL;
};

// Tile of variant V for a pass of S stages: at most 8 sub-transforms per CTA
// when they have 512 elements (static shared memory), and the resident-CTA
// target that keeps the threads per SM (hence the register budget) of the
// variant's 256-element form.
template <int V, int S>
struct Tile {
    static constexpr int CT = (S >= 9 && VAR_CT[V] > 8) ? 8 : VAR_CT[V];
    static constexpr int THREADS = (CT << S) / 16;
    static constexpr int WANT = (16 * VAR_CT[V] * VAR_MINB[V]) / THREADS;
    static constexpr int MINB = WANT < 1 ? 1 : (WANT > 32 ? 32 : WANT);
};

template <int LOGN, int V, int KIND, bool INV, bool NINV, class Pro, class Epi>
void launch_pass(const fides_ctx *c, const LimbSet &set, const TwPair *tw, Pro pro, Epi epi, cudaStream_t st,
                 const char *name)
{
    constexpr int S = KIND == 0 ? Split<LOGN>::COL : Split<LOGN>::ROW;
    using T = Tile<V, S>;
    auto k = k_ntt<LOGN, S, KIND, INV, NINV, T::CT, T::MINB, Pro, Epi>;
    dim3 grid((1 << (LOGN - S)) / T::CT, set.total), block(T::THREADS);
    FIDES_LAUNCH(name, st, k, grid, block, set, (const PrimeInfo *)c->d_prime, tw, pro, epi);
}

template <int LOGN, int KIND, bool INV, bool NINV, class Pro, class Epi>
void launch_pass_v(int v, const fides_ctx *c, const LimbSet &set, const TwPair *tw, Pro pro, Epi epi,
                   cudaStream_t st, const char *name)
{
    switch (v) {
    case 0: launch_pass<LOGN, 0, KIND, INV, NINV>(c, set, tw, pro, epi, st, name); break;
    case 1: launch_pass<LOGN, 1, KIND, INV, NINV>(c, set, tw, pro, epi, st, name); break;
    case 2: launch_pass<LOGN, 2, KIND, INV, NINV>(c, set, tw, pro, epi, st, name); break;
    case 3: launch_pass<LOGN, 3, KIND, INV, NINV>(c, set, tw, pro, epi, st, name); break;
    default: launch_pass<LOGN, 4, KIND, INV, NINV>(c, set, tw, pro, epi, st, name); break;
    }
}

template <int LOGN, class Pro, class Epi>
int forward(const fides_ctx *c, const LimbSet &set, Pro pro, Epi epi, cudaStream_t st)
{
    if (set.total == 0) return FIDES_OK;
    if constexpr (LOGN == 12) {
        auto k = k_ntt<12, 12, 2, false, false, 16, 3, Pro, Epi>;
        FIDES_LAUNCH("k_ntt_fwd_limb", st, k, dim3(1, set.total), dim3(256), set, (const PrimeInfo *)c->d_prime,
                     (const TwPair *)c->d_tw, pro, epi);
    } else {
        launch_pass_v<LOGN, 0, false, false>(variant_of(c, FWD_COLS, set.total), c, set, c->d_tw, pro, EpiLazy{},
                                             st, "k_ntt_fwd_cols");
        launch_pass_v<LOGN, 1, false, false>(variant_of(c, FWD_ROWS, set.total), c, set, c->d_tw, ProDst{}, epi, st,
                                             "k_ntt_fwd_rows");
    }
    return fides_check_cuda(cudaGetLastError(), "ntt forward launch");
}

template <int LOGN, class Pro, class Epi>
int inverse(const fides_ctx *c, const LimbSet &set, Pro pro, Epi epi, cudaStream_t st)
{
    if (set.total == 0) return FIDES_OK;
    if constexpr (LOGN == 12) {
        auto k = k_ntt<12, 12, 2, true, true, 16, 3, Pro, Epi>;
        FIDES_LAUNCH("k_ntt_inv_limb", st, k, dim3(1, set.total), dim3(256), set, (const PrimeInfo *)c->d_prime,
                     (const TwPair *)c->d_itw, pro, epi);
    } else {
        launch_pass_v<LOGN, 1, true, false>(variant_of(c, INV_ROWS, set.total), c, set, c->d_itw, pro, EpiLazy{}, st,
                                            "k_ntt_inv_rows");
        launch_pass_v<LOGN, 0, true, true>(variant_of(c, INV_COLS, set.total), c, set, c->d_itw, ProDst{}, epi, st,
                                           "k_ntt_inv_cols");
    }
    return fides_check_cuda(cudaGetLastError(), "ntt inverse launch");
}

// one pass of kind `kind` with variant v (for the autotuner)
template <int LOGN>
void launch_one(const fides_ctx *c, int kind, int v, const LimbSet &set, cudaStream_t st)
{
    switch (kind) {
    case FWD_COLS:
        launch_pass_v<LOGN, 0, false, false>(v, c, set, c->d_tw, ProSrc{}, EpiLazy{}, st, "k_ntt_tune");
        break;
    case FWD_ROWS:
        launch_pass_v<LOGN, 1, false, false>(v, c, set, c->d_tw, ProDst{}, EpiCanon{}, st, "k_ntt_tune");
        break;
    case INV_ROWS:
        launch_pass_v<LOGN, 1, true, false>(v, c, set, c->d_itw, ProPlain{}, EpiLazy{}, st, "k_ntt_tune");
        break;
    default:
        launch_pass_v<LOGN, 0, true, true>(v, c, set, c->d_itw, ProDst{}, EpiCanon{}, st, "k_ntt_tune");
        break;
    }
}

}  // namespace

// The launchers of one ring degree (defined by FIDES_NTT_DEGREE in ntt_lNN.cu).
#define FIDES_NTT_DECLARE(L)                                                                      \
    int ntt_fwd_canon_##L(const fides_ctx *, const LimbSet &, cudaStream_t);                      \
    int ntt_fwd_submul_##L(const fides_ctx *, const LimbSet &, cudaStream_t);                     \
    int ntt_fwd_switch_submul_##L(const fides_ctx *, const LimbSet &, cudaStream_t);              \
    int ntt_fwd_submul_rot_##L(const fides_ctx *, const LimbSet &, cudaStream_t);                 \
    int ntt_fwd_raise_##L(const fides_ctx *, const LimbSet &, cudaStream_t);                      \
    int ntt_fwd_hmrs_##L(const fides_ctx *, const LimbSet &, cudaStream_t);                       \
    int ntt_inv_canon_##L(const fides_ctx *, const LimbSet &, cudaStream_t);                      \
    void ntt_tune_one_##L(const fides_ctx *, int, int, const LimbSet &, cudaStream_t);

#define FIDES_NTT_DEGREE(L)                                                                                       \
    int ntt_fwd_canon_##L(const fides_ctx *c, const LimbSet &s, cudaStream_t st)                                \
    {                                                                                                             \
        return forward<L>(c, s, ProSrc{}, EpiCanon{}, st);                                                        \
    }                                                                                                             \
    int ntt_fwd_submul_##L(const fides_ctx *c, const LimbSet &s, cudaStream_t st)                               \
    {                                                                                                             \
        return forward<L>(c, s, ProSrc{}, EpiSubMul{}, st);                                                       \
    }                                                                                                             \
    int ntt_fwd_switch_submul_##L(const fides_ctx *c, const LimbSet &s, cudaStream_t st)                        \
    {                                                                                                             \
        return forward<L>(c, s, ProSwitchMod{}, EpiSubMul{}, st);                                                 \
    }                                                                                                             \
    int ntt_fwd_submul_rot_##L(const fides_ctx *c, const LimbSet &s, cudaStream_t st)                           \
    {                                                                                                             \
        return forward<L>(c, s, ProSrc{}, EpiSubMulRot{c->logN}, st);                                             \
    }                                                                                                             \
    int ntt_fwd_raise_##L(const fides_ctx *c, const LimbSet &s, cudaStream_t st)                                \
    {                                                                                                             \
        return forward<L>(c, s, ProRaise{}, EpiCanon{}, st);                                                      \
    }                                                                                                             \
    int ntt_fwd_hmrs_##L(const fides_ctx *c, const LimbSet &s, cudaStream_t st)                                 \
    {                                                                                                             \
        return forward<L>(c, s, ProHmRs{}, EpiHmRs{}, st);                                                        \
    }                                                                                                             \
    int ntt_inv_canon_##L(const fides_ctx *c, const LimbSet &s, cudaStream_t st)                                \
    {                                                                                                             \
        if (s.modes == 0) return inverse<L>(c, s, ProPlain{}, EpiCanon{}, st);                                    \
        return inverse<L>(c, s, ProPrep{c->logN}, EpiCanon{}, st);                                                \
    }                                                                                                             \
    void ntt_tune_one_##L(const fides_ctx *c, int kind, int v, const LimbSet &s, cudaStream_t st)               \
    {                                                                                                             \
        if constexpr (L != 12) launch_one<L>(c, kind, v, s, st);                                                  \
    }

FIDES_NTT_DECLARE(12)
FIDES_NTT_DECLARE(13)
FIDES_NTT_DECLARE(14)
FIDES_NTT_DECLARE(15)
FIDES_NTT_DECLARE(16)
FIDES_NTT_DECLARE(17)
