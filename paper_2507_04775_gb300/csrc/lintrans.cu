// Linear transforms of the slots by the diagonal method with a baby-step
// giant-step split, the building block of bootstrapping's CoeffToSlot and
// SlotToCoeff (Sec. III-F7), whose baby steps are hoisted rotations
// (Sec. III-F6):
//   y = sum_i d_i (.) rot_i(z) = sum_g rot_{n1 g}( sum_b pt_{g,b} (.) rot_b(z) ),
// i = n1 g + b with 0 <= b < n1, pt_{g,b} the plaintext of rot_{-n1 g}(d_i).
// The baby-step rotations share one ModUp; each giant step is one inner sum
// (a single multiply-accumulate launch over its baby steps) and one HRotate.
#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "fides_internal.cuh"
#include "ops_ws.h"

namespace {

struct LtPlan {
    std::vector<int> baby;                      // baby steps b != 0 in use, ascending
    std::map<int, std::vector<int>> giant;      // g -> indices k of the diagonals with i / n1 == g
};

int lt_plan(const fides_ctx *c, int n_diag, const int *diag_idx, int n1, LtPlan &P, const char *fn)
{
    const int half = c->N / 2;
    if (n_diag < 1 || !diag_idx) return fides_set_error(FIDES_ERR_ARG, "%s: no diagonals", fn);
    if (n1 < 1) return fides_set_error(FIDES_ERR_ARG, "%s: n1=%d < 1", fn, n1);
    std::vector<bool> seen(half, false), used(std::min(n1, half), false);
    for (int k = 0; k < n_diag; ++k) {
        const int i = diag_idx[k];
        if (i < 0 || i >= half || seen[i])
            return fides_set_error(FIDES_ERR_ARG, "%s: diagonal %d out of range or repeated", fn, i);
        seen[i] = true;
        used[i % n1] = true;
        P.giant[i / n1].push_back(k);
    }
    for (int b = 1; b < (int)used.size(); ++b)
        if (used[b]) P.baby.push_back(b);
    return FIDES_OK;
}

// The key of the rotation by `steps` among the handles: the one registered
// with Galois element 5^steps mod 2N (of this context), or null.
const uint64_t *lt_key(const fides_ctx *c, int n_keys, const fides_key *const *keys, int64_t steps)
{
    const u64 want = fides_galois_elt(c, steps);
    for (int k = 0; k < n_keys; ++k)
        if (keys[k] && keys[k]->ctx == c && keys[k]->g == want) return keys[k]->data;
    return nullptr;
}

}  // namespace

extern "C" int fides_linear_transform_work_words(fides_ctx *c, int n_limbs, int n_diag, const int *diag_idx, int n1,
                                                 size_t *words)
{
    const char *fn = "fides_linear_transform_work_words";
    if (!c || !words) return fides_set_error(FIDES_ERR_ARG, "%s: NULL argument", fn);
    if (n_limbs < 1 || n_limbs > c->L) return fides_set_error(FIDES_ERR_ARG, "%s: bad n_limbs", fn);
    LtPlan P;
    if (int rc = lt_plan(c, n_diag, diag_idx, n1, P, fn)) return rc;
    // baby-step ciphertexts, one inner sum and one rotated inner sum
    *words = (P.baby.size() + 2) * 2 * (size_t)n_limbs * c->N;
    return FIDES_OK;
}

extern "C" int fides_linear_transform(fides_ctx *c, const fides_ct *a, int n_diag, const int *diag_idx,
                                      const uint64_t *const *pts, double pt_scale, int n1, int n_keys,
                                      const fides_key *const *keys, uint64_t *work, size_t work_words, fides_ct *out,
                                      void *stream)
{
    return fides_linear_transform_ws(c, a, n_diag, diag_idx, pts, pt_scale, n1, n_keys, keys, work, work_words, out,
                                     stream, nullptr);
}

int fides_linear_transform_ws(fides_ctx *c, const fides_ct *a, int n_diag, const int *diag_idx,
                              const uint64_t *const *pts, double pt_scale, int n1, int n_keys,
                              const fides_key *const *keys, uint64_t *work, size_t work_words, fides_ct *out,
                              void *stream, u64 *ws)
{
    const char *fn = "fides_linear_transform";
    if (!c || !a || !a->data || !out || !out->data || !pts || n_keys < 0 || (n_keys > 0 && !keys))
        return fides_set_error(FIDES_ERR_ARG, "%s: NULL argument", fn);
    const int nl = a->n_limbs;
    if (nl < 1 || nl > c->L || out->n_limbs != nl) return fides_set_error(FIDES_ERR_ARG, "%s: bad levels", fn);
    if (out->data == a->data) return fides_set_error(FIDES_ERR_ARG, "%s: out may not alias a", fn);
    LtPlan P;
    if (int rc = lt_plan(c, n_diag, diag_idx, n1, P, fn)) return rc;
    for (int k = 0; k < n_diag; ++k)
        if (!pts[k]) return fides_set_error(FIDES_ERR_ARG, "%s: plaintext %d is NULL", fn, k);
    const size_t ct_words = 2 * (size_t)nl * c->N;
    if (!work || work_words < (P.baby.size() + 2) * ct_words)
        return fides_set_error(FIDES_ERR_ARG, "%s: work buffer needs %zu words", fn, (P.baby.size() + 2) * ct_words);
    // every key first, so that nothing is queued when one is missing
    std::vector<const uint64_t *> baby_keys;
    for (int b : P.baby) {
        const uint64_t *k = lt_key(c, n_keys, keys, b);
        if (!k) return fides_set_error(FIDES_ERR_KEY, "%s: no rotation key for baby step %d", fn, b);
        baby_keys.push_back(k);
    }
    std::map<int, const uint64_t *> giant_keys;
    for (auto &kv : P.giant) {
        if (kv.first == 0) continue;
        const uint64_t *k = lt_key(c, n_keys, keys, (int64_t)n1 * kv.first);
        if (!k) return fides_set_error(FIDES_ERR_KEY, "%s: no rotation key for giant step %d", fn, n1 * kv.first);
        giant_keys[kv.first] = k;
    }
    cudaStream_t st = (cudaStream_t)stream;
    OpTrace tr("op_linear_transform", st);

    // baby steps: rotations of a sharing one ModUp
    std::vector<const u64 *> baby(std::min(n1, c->N / 2), nullptr);
    baby[0] = a->data;
    if (!P.baby.empty()) {
        std::vector<int64_t> steps(P.baby.begin(), P.baby.end());
        std::vector<fides_ct> outs(P.baby.size());
        for (size_t r = 0; r < P.baby.size(); ++r) {
            outs[r].data = work + r * ct_words;
            outs[r].n_limbs = nl;
            outs[r].scale = 0.0;
            baby[P.baby[r]] = outs[r].data;
        }
        if (int rc = fides_rotate_hoisted_ws(c, a, (int)steps.size(), steps.data(), baby_keys.data(), outs.data(),
                                             stream, ws))
            return rc;
    }
    u64 *inner = work + P.baby.size() * ct_words;
    u64 *term = inner + ct_words;

    // giant steps
    bool have_out = false;
    for (auto &kv : P.giant) {
        const int g = kv.first;
        std::vector<const u64 *> cts, ps;
        for (int k : kv.second) {
            cts.push_back(baby[diag_idx[k] % n1]);
            ps.push_back(pts[k]);
        }
        if (g == 0) {
            // the unrotated group accumulates straight into out
            if (int rc = launch_ptmac(c, cts.data(), ps.data(), (int)cts.size(), out->data, nl, have_out, st)) return rc;
            have_out = true;
            continue;
        }
        if (int rc = launch_ptmac(c, cts.data(), ps.data(), (int)cts.size(), inner, nl, false, st)) return rc;
        fides_ct ci = {inner, nl, a->scale * pt_scale};
        fides_ct ct = {have_out ? term : out->data, nl, 0.0};
        if (int rc = fides_rotate_ws(c, &ci, (int64_t)n1 * g, giant_keys[g], &ct, stream, ws)) return rc;
        if (have_out) {
            fides_ct co = {out->data, nl, 0.0};
            if (int rc = fides_hadd(c, &co, &ct, &co, stream)) return rc;
        }
        have_out = true;
    }
    out->scale = a->scale * pt_scale;
    return FIDES_OK;
}
