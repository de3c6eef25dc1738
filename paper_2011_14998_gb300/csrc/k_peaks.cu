// k_peaks.cu -- throughput microbenchmarks of the arithmetic pipes the formal
// solution runs on: FP32 fused multiply-add, FP64 fused multiply-add, and the
// special-function unit's approximate exp2 and reciprocal.  Each kernel runs
// eight independent dependency chains per thread on every SM, long enough
// (tens of milliseconds) for CUDA-event timing; the results are written so
// that nothing is optimised away.
#include "mgx_internal.cuh"

namespace mgx {

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(256) k_peak_ffma(float *out, int iters, float s) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = float(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kUnroll; ++k)
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], s, 0.5f);
    }
    float t = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) t += a[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

__global__ void __launch_bounds__(256) k_peak_dfma(double *out, int iters, double s) {
    double a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = double(threadIdx.x + c) * 1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kUnroll; ++k)
#pragma unroll
            for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], s, 0.5);
    }
    double t = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) t += a[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

// kind 0: x <- 2^(-x) (ex2.approx.ftz.f32), kind 1: x <- 1/(x + 1) (rcp.approx.ftz.f32 of an add)
__global__ void __launch_bounds__(256) k_peak_mufu(float *out, int iters, int kind) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = float(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kUnroll; ++k)
#pragma unroll
            for (int c = 0; c < kChains; ++c) {
                float r;
                if (kind == 0) asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-a[c]));
                else asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[c]));
                a[c] = r;
            }
    }
    float t = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) t += a[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

}  // namespace

// out: [0] FP32 FMA TFLOP/s (2 flops per FMA), [1] FP64 FMA TFLOP/s, [2] ex2
// Gop/s, [3] rcp Gop/s; each the best of `reps` timed launches.
cudaError_t alu_peaks(cudaStream_t st, int reps, double out[4]) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int blocks = sms * 8, threads = 256;
    const int64_t n = int64_t(blocks) * threads;
    void *buf = nullptr;
    if ((e = cudaMalloc(&buf, size_t(n) * sizeof(double))) != cudaSuccess) return e;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int it32 = 256, it64 = 4, itmu = 8192;  // about 0.25 s, 0.25 s and 0.07 s per launch on GB300
    const double per_thread = double(kChains) * kUnroll;
    for (int kind = 0; kind < 4; ++kind) {
        double best = 0.0;
        for (int r = 0; r < reps + 1; ++r) {  // the first launch warms up
            cudaEventRecord(a, st);
            if (kind == 0) k_peak_ffma<<<blocks, threads, 0, st>>>(static_cast<float *>(buf), it32, 0.9999f);
            else if (kind == 1) k_peak_dfma<<<blocks, threads, 0, st>>>(static_cast<double *>(buf), it64, 0.9999);
            else k_peak_mufu<<<blocks, threads, 0, st>>>(static_cast<float *>(buf), itmu, kind - 2);
            cudaEventRecord(b, st);
            if ((e = cudaEventSynchronize(b)) != cudaSuccess) break;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            const int iters = kind == 0 ? it32 : kind == 1 ? it64 : itmu;
            const double ops = double(n) * per_thread * iters * (kind < 2 ? 2.0 : 1.0);
            const double rate = ops / (double(ms) * 1e-3) / (kind < 2 ? 1e12 : 1e9);
            if (r > 0 && rate > best) best = rate;
        }
        out[kind] = best;
        if (e != cudaSuccess) break;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    const cudaError_t e2 = cudaFree(buf);
    return e != cudaSuccess ? e : e2;
}

}  // namespace mgx
