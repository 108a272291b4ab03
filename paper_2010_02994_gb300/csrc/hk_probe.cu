// Pipe-rate probes: FP32 FMA and MUFU ex2 results per SM per clock, and FP64
// FMA (DFMA) results per SM per clock; and an evaluation entry for the FP64
// pair kernels' base-2 exponential, so tests can check it against the host.
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
#include "hk_exp2.cuh"

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

constexpr int kIters64 = 2048;

// FP64 FMA chains; each CTA records its clock-counter and global-timer spans
// (the ratio is the SM clock).
__global__ void probe_fp64_kernel(double seed, double *sink, long long *cycles, unsigned long long *nanos)
{
    double v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        v[c] = seed * (double)(threadIdx.x + c + 1) * 1e-6;
    const long long t0 = clock64();
    unsigned long long g0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g0));
    const double a = 0.999999, b = 1e-7;
    for (int i = 0; i < kIters64; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            v[c] = fma(v[c], a, b);
    }
    const long long t1 = clock64();
    unsigned long long g1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g1));
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += v[c];
    if (s == 12345.678)
        sink[threadIdx.x] = s;
    if (threadIdx.x == 0) {
        cycles[blockIdx.x] = t1 - t0;
        nanos[blockIdx.x] = g1 - g0;
    }
}

}  // namespace

// The whole kernel is timed with events and divided by the SM clock: on
// this GPU the longest clock-counter span of single CTAs overstated the
// FP64 rate two-fold.
extern "C" hawkes_status hawkes_probe_dfma_rate(int32_t device, double *dfma_per_sm_clk)
{
    if (cudaSetDevice(device) != cudaSuccess)
        return HAWKES_ERR_CUDA;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int threads = 512, per_sm = 2, grid = sms * per_sm;
    double *sink = nullptr;
    long long *cyc = nullptr;
    unsigned long long *ns = nullptr;
    if (cudaMalloc(&sink, sizeof(double) * threads) != cudaSuccess ||
        cudaMalloc(&cyc, sizeof(long long) * grid) != cudaSuccess ||
        cudaMalloc(&ns, sizeof(unsigned long long) * grid) != cudaSuccess) {
        cudaFree(sink);
        cudaFree(cyc);
        return HAWKES_ERR_OOM;
    }
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    probe_fp64_kernel<<<grid, threads>>>(1.0, sink, cyc, ns);  // warm-up
    cudaEventRecord(a);
    probe_fp64_kernel<<<grid, threads>>>(1.0, sink, cyc, ns);
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.0f;
    std::vector<long long> c(grid);
    std::vector<unsigned long long> g(grid);
    if (e == cudaSuccess)
        e = cudaEventElapsedTime(&ms, a, b);
    if (e == cudaSuccess)
        e = cudaMemcpy(c.data(), cyc, sizeof(long long) * grid, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(g.data(), ns, sizeof(unsigned long long) * grid, cudaMemcpyDeviceToHost);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    cudaFree(cyc);
    cudaFree(ns);
    if (e != cudaSuccess || ms <= 0.0f)
        return HAWKES_ERR_CUDA;
    // SM clock (cycles per nanosecond) from the CTA with the longest span
    const int k = (int)(std::max_element(g.begin(), g.end()) - g.begin());
    if (g[k] == 0)
        return HAWKES_ERR_CUDA;
    const double ghz = (double)c[k] / (double)g[k];
    const double ops = (double)grid * threads * kChains * kIters64;
    if (dfma_per_sm_clk)
        *dfma_per_sm_clk = ops / sms / (ms * 1e6 * ghz);
    return HAWKES_OK;
}

namespace {

__global__ void exp2_probe_kernel(const double *__restrict__ y, double *__restrict__ out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = hk::exp2_neg_lane(y[i], hk::kExp2Tab);
}

}  // namespace

extern "C" hawkes_status hawkes_probe_exp2_fp64(const double *y, double *out, int64_t n, hawkes_stream stream)
{
    if (n < 0 || (n > 0 && (!y || !out)))
        return HAWKES_ERR_INVALID_ARG;
    if (n == 0)
        return HAWKES_OK;
    const int grid = (int)std::min<int64_t>(4096, (n + 255) / 256);
    exp2_probe_kernel<<<grid, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(y, out, n);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ERR_CUDA;
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
