// Pipe-rate probes: FP32 FMA and MUFU ex2 results per SM per clock, and FP64
// FMA (DFMA) results per SM per clock.
//
// The pair kernels are bound by the first two pipes, so their roofline is
// derived from measured rates rather than datasheet figures; the FP64 rate
// bounds the FP64 precision path.  Each CTA runs
// independent dependency chains long enough to hide latency, times itself
// with the SM clock counter, and reports operations per SM per clock.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "hawkes.h"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

__device__ __forceinline__ float ex2a(float x)
{
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// kind 0: FFMA chains; kind 1: ex2 chains (each step ex2 of a bounded value).
__global__ void probe_kernel(int kind, float seed, float *sink, long long *cycles)
{
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        v[c] = seed * (float)(threadIdx.x + c + 1) * 1e-6f;
    __syncthreads();
    const long long t0 = clock64();
    if (kind == 0) {
        const float a = 0.999999f, b = 1e-7f;
        for (int i = 0; i < kIters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c)
                v[c] = fmaf(v[c], a, b);
        }
    } else {
        for (int i = 0; i < kIters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c)
                v[c] = ex2a(v[c]) - 1.0f;  // stays in (-1, 1]
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += v[c];
    if (s == 12345.678f)
        sink[threadIdx.x] = s;
    if (threadIdx.x == 0)
        cycles[blockIdx.x] = t1 - t0;
}

constexpr int kIters64 = 256;  // FP64 runs at a small fraction of the FP32 rate

__global__ void probe_fp64_kernel(double seed, double *sink, long long *cycles)
{
    double v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        v[c] = seed * (double)(threadIdx.x + c + 1) * 1e-6;
    __syncthreads();
    const long long t0 = clock64();
    const double a = 0.999999, b = 1e-7;
    for (int i = 0; i < kIters64; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            v[c] = fma(v[c], a, b);
    }
    __syncthreads();
    const long long t1 = clock64();
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += v[c];
    if (s == 12345.678)
        sink[threadIdx.x] = s;
    if (threadIdx.x == 0)
        cycles[blockIdx.x] = t1 - t0;
}

}  // namespace

extern "C" hawkes_status hawkes_probe_dfma_rate(int32_t device, double *dfma_per_sm_clk)
{
    if (cudaSetDevice(device) != cudaSuccess)
        return HAWKES_ERR_CUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int threads = 512, per_sm = 2, grid = sms * per_sm;
    double *sink = nullptr;
    long long *cyc = nullptr;
    if (cudaMalloc(&sink, sizeof(double) * threads) != cudaSuccess ||
        cudaMalloc(&cyc, sizeof(long long) * grid) != cudaSuccess) {
        cudaFree(sink);
        return HAWKES_ERR_OOM;
    }
    probe_fp64_kernel<<<grid, threads>>>(1.0, sink, cyc);  // warm-up
    probe_fp64_kernel<<<grid, threads>>>(1.0, sink, cyc);
    std::vector<long long> c(grid);
    const cudaError_t e = cudaMemcpy(c.data(), cyc, sizeof(long long) * grid, cudaMemcpyDeviceToHost);
    cudaFree(sink);
    cudaFree(cyc);
    if (e != cudaSuccess)
        return HAWKES_ERR_CUDA;
    const double span = (double)*std::max_element(c.begin(), c.end());
    if (dfma_per_sm_clk)
        *dfma_per_sm_clk = (double)per_sm * threads * kChains * kIters64 / span;
    return HAWKES_OK;
}

extern "C" hawkes_status hawkes_probe_pipe_rates(int32_t device, double *fma_per_sm_clk, double *ex2_per_sm_clk,
                                                 double *sm_clock_mhz)
{
    if (cudaSetDevice(device) != cudaSuccess)
        return HAWKES_ERR_CUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int threads = 512, per_sm = 2, grid = sms * per_sm;
    float *sink = nullptr;
    long long *cyc = nullptr;
    if (cudaMalloc(&sink, sizeof(float) * threads) != cudaSuccess ||
        cudaMalloc(&cyc, sizeof(long long) * grid) != cudaSuccess) {
        cudaFree(sink);
        return HAWKES_ERR_OOM;
    }
    double rate[2] = {0, 0}, mhz = 0;
    for (int kind = 0; kind < 2; ++kind) {
        probe_kernel<<<grid, threads>>>(kind, 1.0f, sink, cyc);  // warm-up
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a);
        probe_kernel<<<grid, threads>>>(kind, 1.0f, sink, cyc);
        cudaEventRecord(b);
        if (cudaEventSynchronize(b) != cudaSuccess) {
            cudaFree(sink);
            cudaFree(cyc);
            return HAWKES_ERR_CUDA;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        std::vector<long long> c(grid);
        cudaMemcpy(c.data(), cyc, sizeof(long long) * grid, cudaMemcpyDeviceToHost);
        // the CTAs of one SM run concurrently: take the slowest as that SM's span
        const double span = (double)*std::max_element(c.begin(), c.end());
        const double ops_per_sm = (double)per_sm * threads * kChains * kIters;
        rate[kind] = ops_per_sm / span;
        if (kind == 0)
            mhz = span / (ms * 1e3);
    }
    cudaFree(sink);
    cudaFree(cyc);
    if (fma_per_sm_clk)
        *fma_per_sm_clk = rate[0];
    if (ex2_per_sm_clk)
        *ex2_per_sm_clk = rate[1];
    if (sm_clock_mhz)
        *sm_clock_mhz = mhz;
    return HAWKES_OK;
}
