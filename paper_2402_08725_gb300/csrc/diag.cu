// Diagnostic: measured FP32 fused-multiply-add throughput of the current GPU (sm_103a).
//
// The denominator of the direct form's roofline: its tile kernels are bound by FP32 FMA issue,
// whose peak (SMs x 128 lanes x 2 FLOP x clock) depends on the clock the GPU sustains.  Each
// thread runs eight independent register-resident chains a <- a b + c (b slightly below 1, so
// the values stay normal and bounded); 2048 threads per SM keep every FMA pipe busy.
#include "common.cuh"

namespace sr {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(256) ffma_peak_kernel(float *out, int iters, float b, float c) {
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1e-3f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == -1.f) out[0] = s;  // never true; keeps the chains live
}

}  // namespace
}  // namespace sr

using namespace sr;

extern "C" sr_status sr_measure_fp32_peak(double *tflops) {
    if (!tflops) {
        set_error("sr_measure_fp32_peak: tflops is NULL");
        return SR_ERR_ARG;
    }
    int dev = 0, sms = 0;
    SR_CUDA(cudaGetDevice(&dev));
    SR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int grid = sms * 8, block = 256, iters = 8192;
    cudaEvent_t e0, e1;
    SR_CUDA(cudaEventCreate(&e0));
    SR_CUDA(cudaEventCreate(&e1));
    float *sink = nullptr;  // never written (see the kernel); a null pointer is never dereferenced
    ffma_peak_kernel<<<grid, block>>>(sink, iters / 8, 0.9999999f, 1e-7f);  // warm-up
    cudaEventRecord(e0);
    ffma_peak_kernel<<<grid, block>>>(sink, iters, 0.9999999f, 1e-7f);
    cudaEventRecord(e1);
    const cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    SR_CUDA(e);
    SR_CUDA(cudaGetLastError());
    const double flop = 2.0 * (double)grid * block * (double)iters * kUnroll * kChains;
    *tflops = ms > 0.f ? flop / (ms * 1e-3) / 1e12 : 0.0;
    return SR_OK;
}
