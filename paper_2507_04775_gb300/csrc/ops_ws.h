// Operations with an explicit scratch pool of ctx->scratch_words words (null:
// the context's own), defined in keyswitch.cu and lintrans.cu.  Calls that run
// concurrently on one context (programs on several streams, program.cu) each
// pass their own pool; the C entry points pass null.
#pragma once

#include "fides_internal.cuh"

int fides_hmult_ws(fides_ctx *c, const fides_ct *a, const fides_ct *b, const uint64_t *rlk, fides_ct *out,
                   void *stream, u64 *ws);
int fides_rotate_ws(fides_ctx *c, const fides_ct *a, int64_t steps, const uint64_t *rk, fides_ct *out, void *stream,
                    u64 *ws);
int fides_conjugate_ws(fides_ctx *c, const fides_ct *a, const uint64_t *ck, fides_ct *out, void *stream, u64 *ws);
int fides_rotate_hoisted_ws(fides_ctx *c, const fides_ct *a, int n_rot, const int64_t *steps,
                            const uint64_t *const *rks, fides_ct *outs, void *stream, u64 *ws);
int fides_rescale_ws(fides_ctx *c, const fides_ct *a, fides_ct *out, void *stream, u64 *ws);
int fides_modraise_ws(fides_ctx *c, const fides_ct *a, fides_ct *out, void *stream, u64 *ws);
int fides_linear_transform_ws(fides_ctx *c, const fides_ct *a, int n_diag, const int *diag_idx,
                              const uint64_t *const *pts, double pt_scale, int n1, int n_keys,
                              const fides_key *const *keys, uint64_t *work, size_t work_words, fides_ct *out,
                              void *stream, u64 *ws);
int fides_hmult_rescale_ws(fides_ctx *c, const fides_ct *a, const fides_ct *b, const uint64_t *rlk, fides_ct *out,
                           void *stream, u64 *ws);
