// Rescale that allocates nothing.
//
// Some callers cannot call cudaMalloc: code that runs while another component
// owns every device allocation (a host application that hands a plugin fixed
// buffers), services that reserve all device memory at start-up and forbid
// allocation afterwards, and callers that must not touch the allocator at a
// given point.  fides_rescale uses the context's scratch pool, which the
// context allocated when it was created; this variant instead keeps its
// scratch -- the coefficient form of the dropped limb of both polynomials,
// 2 x N words -- in a file-scope device array that exists as soon as the
// library is loaded on a GPU.
//
// The array holds FIDES_NOALLOC_SCRATCH_WORDS = 2 * 65536 words (1 MiB), so
// ring degrees up to N = 65536 are accepted; every GPU that loads the library
// keeps it until the process exits.  Every call shares the array: calls whose
// work overlaps on the GPU race on it.  Each call writes the words it later
// reads, so nothing has to start at zero.
#include <cstring>
#include <mutex>

#include "fides_internal.cuh"
#include "plan.cuh"

#define FIDES_NOALLOC_SCRATCH_WORDS (2 * 65536)
#define FIDES_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) u64 g_noalloc_scratch[FIDES_NOALLOC_SCRATCH_WORDS];

namespace {

std::mutex g_mu;
u64 *g_addr[FIDES_NOALLOC_MAX_DEVICES];

// Device address of the array on `dev`, looked up once per device with that
// device current (the first call on the device does it).  In host code the
// array's name is only a host-side stand-in, so kernels must be given this
// address.  The address is kept for the life of the process: a device reset
// (cudaDeviceReset) after the first call is not supported -- it frees every
// context of this library on that device as well.
int scratch_address(int dev, u64 **out)
{
    if (dev < 0 || dev >= FIDES_NOALLOC_MAX_DEVICES)
        return fides_set_error(FIDES_ERR_UNSUPPORTED, "fides_rescale_noalloc: device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return fides_check_cuda(e, "fides_rescale_noalloc: cudaGetSymbolAddress");
        g_addr[dev] = (u64 *)p;
    }
    *out = g_addr[dev];
    return FIDES_OK;
}

}  // namespace

extern "C" int fides_rescale_noalloc(fides_ctx *c, const fides_ct *a, fides_ct *out, void *stream)
{
    if (!c) return fides_set_error(FIDES_ERR_ARG, "fides_rescale_noalloc: ctx is NULL");
    if (!a || !out || !a->data || !out->data)
        return fides_set_error(FIDES_ERR_ARG, "fides_rescale_noalloc: NULL argument");
    const int nl = a->n_limbs;
    if (nl < 2 || nl > c->L || out->n_limbs != nl - 1)
        return fides_set_error(FIDES_ERR_ARG,
                               "fides_rescale_noalloc: needs 2 <= n_limbs <= %d and out->n_limbs = n_limbs - 1", c->L);
    if ((size_t)2 * c->N > FIDES_NOALLOC_SCRATCH_WORDS)
        return fides_set_error(FIDES_ERR_UNSUPPORTED,
                               "fides_rescale_noalloc: N = %d needs %d scratch words, the static array holds %d",
                               c->N, 2 * c->N, FIDES_NOALLOC_SCRATCH_WORDS);
    int dev = -1;
    if (int rc = fides_check_cuda(cudaGetDevice(&dev), "fides_rescale_noalloc: cudaGetDevice")) return rc;
    if (dev != c->device)
        return fides_set_error(FIDES_ERR_ARG, "fides_rescale_noalloc: the context's device (%d) must be current, not %d",
                               c->device, dev);
    u64 *scr = nullptr;
    if (int rc = scratch_address(dev, &scr)) return rc;

    const int l = nl - 1;
    cudaStream_t st = (cudaStream_t)stream;
    OpTrace op("op_rescale_noalloc", st);
    // the segments of fides_rescale, built into inline limb sets (no heap use)
    // with the static array in place of the context's scratch
    LimbSet last = empty_set(), fin = empty_set();
    SetSink sl{last}, sf{fin};
    rs_intt_segs(c, a->data, nl, scr, sl);
    int rc = ntt_inverse(c, last, ProSrc{}, EpiCanon{}, st);
    if (rc) return rc;
    rs_final_segs(c, a->data, nl, scr, out->data, sf, c->round_nearest != 0);
    rc = ntt_forward(c, fin, ProSwitchMod{}, EpiSubMul{}, st);
    if (!rc) out->scale = a->scale / (double)c->primes[l];
    return rc;
}
