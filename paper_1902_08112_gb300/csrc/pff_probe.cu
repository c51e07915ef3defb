// Measured FP32 FMA issue rate of the GPU: the denominator of the arithmetic roofline of the
// double-float applies (they run on the FP32 pipes).  Each thread runs 8 independent FMA chains
// (enough independent work to fill the pipes at one CTA of 256 threads per scheduler slot), the
// grid fills every SM several times over, and the result is stored only under a condition that
// never holds for the inputs used, so the compiler keeps the arithmetic.
#include "pff_internal.cuh"

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fma_rate(float a, float b, int iters, float* __restrict__ sink) {
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = __fmaf_rn(v[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == 1234.5678f) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" pff_status pff_fp32_fma_tflops(void* cuda_stream, double* tflops) {
    if (!tflops) return PFF_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PFF_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PFF_ECUDA;
    const int blocks = sms * 8, threads = 256, iters = 1 << 14;
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    pff_status st = PFF_ECUDA;
    if (cudaMalloc(&sink, sizeof(float) * blocks) != cudaSuccess) return PFF_ENOMEM;
    if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        // a = 1 - 2^-20, b = 2^-10: every chain stays finite and normal
        const float a = 1.0f - 0x1.0p-20f, b = 0x1.0p-10f;
        k_fma_rate<<<blocks, threads, 0, s>>>(a, b, iters / 4, sink);   // warm-up (clocks up)
        float best = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, s);
            k_fma_rate<<<blocks, threads, 0, s>>>(a, b, iters, sink);
            cudaEventRecord(e1, s);
            float ms = 0.f;
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                best = 0.f;
                break;
            }
            if (best == 0.f || ms < best) best = ms;
        }
        if (best > 0.f && cudaGetLastError() == cudaSuccess) {
            const double flops = 2.0 * kChains * (double)iters * blocks * threads;
            *tflops = flops / (best * 1e-3) / 1e12;
            st = PFF_OK;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return st;
}
