// Measurement aid (no counterpart in the paper): the FP32 fused multiply-add rate of the
// current device, the denominator of the plain FP32 SRP-PHAT kernel's roofline (Eq. 9 is
// 4 Q L flops per frame of FP32 multiply-adds).  Every thread runs 8 independent chains of
// dependent FMAs so that the FMA pipes, not their latency, bound the rate; one CTA per SM
// per 8 warps of each scheduler.
#include <cuda_runtime.h>

#include "common.h"

namespace sp {
namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

__global__ void __launch_bounds__(512) fma_peak_kernel(float *out, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1.2345f) out[threadIdx.x] = s;   // never true for the arguments used; keeps the work
}

}  // namespace
}  // namespace sp

using namespace sp;

extern "C" int sp_fp32_fma_peak(double *tflops) {
    SP_CHECK(tflops, SP_EINVAL, "sp_fp32_fma_peak: null pointer");
    float *out = nullptr;
    SP_CUDA(cudaMalloc(&out, 512 * sizeof(float)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = 4 * num_sms();
    const int threads = 512;
    fma_peak_kernel<<<blocks, threads>>>(out, 0.999f, 0.001f);   // warm-up
    cudaEventRecord(e0);
    const int reps = 20;
    for (int r = 0; r < reps; ++r) fma_peak_kernel<<<blocks, threads>>>(out, 0.999f, 0.001f);
    cudaEventRecord(e1);
    const cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    SP_CHECK(e == cudaSuccess && ms > 0.f, SP_ECUDA, std::string("sp_fp32_fma_peak: ") + cudaGetErrorString(e));
    const double flops = 2.0 * kChains * kIters * (double)threads * blocks * reps;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return SP_OK;
}
