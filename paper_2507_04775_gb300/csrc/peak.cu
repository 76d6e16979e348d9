// Measured ALU roofline of the library's modular arithmetic.
//
// The key-switching kernels are bound by 64-bit modular products on the
// integer multiply pipe, not by a dense contraction, so their roofline is the
// rate at which the device sustains the library's own Shoup product (the
// product every NTT butterfly and per-prime scaling uses).  This kernel runs
// eight independent chains of that product per thread, entirely in registers,
// over a grid of 8 CTAs of 256 threads per SM.
#include "fides_internal.cuh"

namespace {

__global__ void __launch_bounds__(256) k_modmul_peak(u64 *out, u64 q, u64 w, u64 wp, int iters)
{
    const u64 t = (u64)blockIdx.x * blockDim.x + threadIdx.x;
    u64 x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (t * 0x9E3779B97F4A7C15ull + (u64)k) % q;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = mul_shoup(x[k], w, wp, q);
    }
    u64 acc = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) acc ^= x[k];
    out[t] = acc;
}

}  // namespace

extern "C" int fides_measure_modmul_peak(double *gmodmul_per_s, double *ms_out)
{
    if (!gmodmul_per_s) return fides_set_error(FIDES_ERR_ARG, "fides_measure_modmul_peak: NULL output");
    int dev = 0, nsm = 0;
    if (int rc = fides_check_cuda(cudaGetDevice(&dev), "cudaGetDevice")) return rc;
    if (int rc = fides_check_cuda(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "attribute"))
        return rc;
    const int blocks = nsm * 8, threads = 256, iters = 4096;
    u64 *out = nullptr;
    if (int rc = fides_check_cuda(cudaMalloc(&out, sizeof(u64) * blocks * threads), "cudaMalloc")) return rc;
    // a 60-bit prime = 1 mod 2^17 and an arbitrary twiddle with its Shoup companion
    const u64 q = 1152921504606584833ull;
    const u64 w = 123456789012345678ull % q;
    const u64 wp = (u64)(((unsigned __int128)w << 64) / q);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_modmul_peak<<<blocks, threads>>>(out, q, w, wp, iters);   // warm-up
    cudaEventRecord(e0);
    const int reps = 5;
    for (int r = 0; r < reps; ++r) k_modmul_peak<<<blocks, threads>>>(out, q, w, wp, iters);
    cudaEventRecord(e1);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (int rc = fides_check_cuda(e, "fides_measure_modmul_peak")) return rc;
    const double ops = (double)blocks * threads * iters * 8.0 * reps;
    *gmodmul_per_s = ops / (ms * 1e-3) / 1e9;
    if (ms_out) *ms_out = ms / reps;
    return FIDES_OK;
}
