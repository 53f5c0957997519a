// probe.cu -- ucp_probe_alu: measured FP64 FMA, FP32 FMA and FP32 ex2 (SFU)
// throughput of the current GPU, the denominators of the roofline fractions
// reported for the ALU-bound kernels of this library.
//
// Each thread runs kChains independent multiply-add chains (enough
// instruction-level parallelism to cover the pipe latency) for kIters
// iterations; the grid fills every SM several times over.  The results are
// written to a device buffer so the compiler cannot drop the work.
#include "ucp_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

__global__ void k_dfma(double* out, double a, double b) {
    double v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = threadIdx.x * 1e-3 + c;
    for (int it = 0; it < kIters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = fma(v[c], a, b);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_ffma(float* out, float a, float b) {
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = threadIdx.x * 1e-3f + c;
    for (int it = 0; it < kIters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = fmaf(v[c], a, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_ex2(float* out, float a) {
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = -1e-3f * (threadIdx.x + c);
    for (int it = 0; it < kIters; ++it)
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float r;
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v[c]));
            v[c] = r * a - 1.0f;
        }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" UCP_API ucp_status ucp_probe_alu(double* fp64_tflops, double* fp32_tflops,
                                            double* ex2_gops, void* stream) {
    if (!fp64_tflops || !fp32_tflops || !ex2_gops) return UCP_E_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return UCP_E_CUDA;
    const int threads = 256, blocks = sms * 8;
    const size_t n = (size_t)threads * blocks;
    void* buf = nullptr;
    if (cudaMalloc(&buf, n * sizeof(double)) != cudaSuccess) return UCP_E_NOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float ms[3] = {0, 0, 0};
    for (int rep = 0; rep < 2; ++rep) {  // first pass warms up clocks
        cudaEventRecord(e0, s);
        k_dfma<<<blocks, threads, 0, s>>>((double*)buf, 0.999999, 1e-7);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms[0], e0, e1);
        cudaEventRecord(e0, s);
        k_ffma<<<blocks, threads, 0, s>>>((float*)buf, 0.999f, 1e-4f);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms[1], e0, e1);
        cudaEventRecord(e0, s);
        k_ex2<<<blocks, threads, 0, s>>>((float*)buf, 0.5f);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms[2], e0, e1);
    }
    const double ops = (double)n * kIters * kChains;
    *fp64_tflops = 2.0 * ops / (ms[0] * 1e-3) / 1e12;
    *fp32_tflops = 2.0 * ops / (ms[1] * 1e-3) / 1e12;
    *ex2_gops = ops / (ms[2] * 1e-3) / 1e9;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    return cudaGetLastError() == cudaSuccess ? UCP_OK : UCP_E_CUDA;
}
