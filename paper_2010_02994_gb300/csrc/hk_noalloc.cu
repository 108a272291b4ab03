// hawkes_loglik_noalloc: the FP64 log-likelihood of hawkes_loglik without any
// device memory allocation (the paper has no counterpart of this entry point).
//
// Some callers cannot call cudaMalloc: code that runs inside a framework or
// plugin host that owns every device allocation (a custom allocator or memory
// pool that raw cudaMalloc would bypass or fragment), and real-time or
// embedded callers whose rules forbid allocating after start-up.  For them
// this entry point keeps its scratch -- one FP64 partial rate sum per event and
// column split -- in a file-scope __device__ array of fixed size, which every
// GPU that loads the library holds until the process exits.  The caller still
// owns the inputs and the output.
//
// The arithmetic is that of the FP64 rate pass: ordered pairs, every
// operation in double, the spatial and temporal Gaussians of the background
// term merged into one exp, partial sums added in a fixed order.  Times need
// not be sorted (each ordered pair applies the indicators of Section 2.1
// directly), so no sort and no other scratch is needed.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "hawkes.h"

namespace {

constexpr int kTile = 128;      // rows per CTA and columns per staged tile
constexpr int kMaxSplit = 16;   // column splits
constexpr int kMaxDim = 8;
constexpr int kFinishThreads = 1024;
constexpr size_t kScratchDoubles = (size_t)kMaxSplit * HAWKES_NOALLOC_MAX_N + 32;

// [0, kMaxSplit * max_n): partial rate sums, split-major; then status words.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mu;

// The scratch array's device address belongs to the CUDA context that loaded
// the library's module: the primary context of a device, a context that the
// host program created itself on the same device, or the primary context
// created again after cudaDeviceReset all have their own copy.  So the
// address is cached per context, keyed by the context's ID (unique for the
// life of the process), not per device number.  The driver entry points are
// fetched through the runtime, so the library needs no link to libcuda.
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);
constexpr int kMaxContexts = 64;
struct ScratchEntry {
    unsigned long long ctx_id;
    double *ptr;
};
ScratchEntry g_cache[kMaxContexts] = {};
int g_cached = 0;
CtxGetCurrentFn g_get_current = nullptr;
CtxGetIdFn g_get_id = nullptr;
bool g_entry_points_tried = false;

// ID of the calling thread's current context; false if there is none (or the
// driver offers no cuCtxGetId), in which case nothing is cached.
bool current_context_id(unsigned long long *id)
{
    if (!g_entry_points_tried) {
        g_entry_points_tried = true;
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            g_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
            g_get_id = reinterpret_cast<CtxGetIdFn>(f2);
        }
        cudaGetLastError();
    }
    if (!g_get_current || !g_get_id)
        return false;
    CUcontext c = nullptr;
    if (g_get_current(&c) != CUDA_SUCCESS || !c)
        return false;
    return g_get_id(c, id) == CUDA_SUCCESS;
}

// Device address of the scratch array in the calling thread's current
// context (its device is current), looked up once per context.  In host
// code the array's name only stands in for the symbol; kernels must be
// given this address.
hawkes_status scratch_in_current_context(double **out)
{
    std::lock_guard<std::mutex> g(g_mu);
    unsigned long long id = 0;
    bool have_id = current_context_id(&id);
    if (have_id)
        for (int k = 0; k < g_cached; ++k)
            if (g_cache[k].ctx_id == id) {
                *out = g_cache[k].ptr;
                return HAWKES_OK;
            }
    // the lookup also makes the device's primary context current if no
    // context was current yet
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return HAWKES_ERR_CUDA;
    }
    if (!have_id)
        have_id = current_context_id(&id);
    if (have_id && g_cached < kMaxContexts)
        g_cache[g_cached++] = {id, static_cast<double *>(p)};
    *out = static_cast<double *>(p);
    return HAWKES_OK;
}

struct Consts {
    double a, b, c, Cmu, Cxi, omega, mu0, tau_t, theta;
};

struct Nsum {
    double s = 0.0, c = 0.0;
    __device__ void add(double x)
    {
        const double t = s + x;
        if (!isfinite(t)) {
            s = t;
            c = 0.0;
            return;
        }
        if (fabs(s) >= fabs(x))
            c += (s - t) + x;
        else
            c += (x - t) + s;
        s = t;
    }
    __device__ double value() const { return isfinite(s) ? s + c : s; }
};

// lambda_n partial sums over one column split (ordered pairs, FP64).
__global__ void __launch_bounds__(kTile) noalloc_rates_kernel(const double *__restrict__ t,
                                                              const double *__restrict__ X, int n, int d, Consts k,
                                                              int fsplit, double *__restrict__ part,
                                                              unsigned *status)
{
    __shared__ double st[kTile];
    __shared__ double sx[kTile * kMaxDim];
    const int row = blockIdx.x * kTile + threadIdx.x;
    const int sp = blockIdx.y;
    const bool valid = row < n;
    double tn = 0.0, xn[kMaxDim];
    for (int q = 0; q < kMaxDim; ++q)
        xn[q] = 0.0;
    if (valid) {
        tn = t[row];
        bool bad = !(tn >= 0.0) || !isfinite(tn);
        for (int q = 0; q < d; ++q) {
            xn[q] = X[(int64_t)row * d + q];
            bad |= !isfinite(xn[q]);
        }
        if (bad && sp == 0)
            atomicOr(status, 1u);
    }
    const int tiles = (n + kTile - 1) / kTile;
    const int per = (tiles + fsplit - 1) / fsplit;
    const int lo = min(sp * per * kTile, n), hi = min((sp + 1) * per * kTile, n);
    Nsum tot;
    for (int c0 = lo; c0 < hi; c0 += kTile) {
        const int cnt = min(kTile, hi - c0);
        __syncthreads();
        if (threadIdx.x < cnt) {
            st[threadIdx.x] = t[c0 + threadIdx.x];
            for (int q = 0; q < d; ++q)
                sx[threadIdx.x * kMaxDim + q] = X[(int64_t)(c0 + threadIdx.x) * d + q];
        }
        __syncthreads();
        if (!valid)
            continue;
        double acc = 0.0;
        for (int j = 0; j < cnt; ++j) {
            const double tm = st[j];
            double r2 = 0.0;
            for (int q = 0; q < d; ++q) {
                const double df = xn[q] - sx[j * kMaxDim + q];
                r2 += df * df;
            }
            const double dt = tn - tm;
            if (tn != tm)
                acc += k.Cmu * exp(-(r2 * k.a + dt * dt * k.b));
            if (tm < tn)
                acc += k.Cxi * exp(-(k.omega * dt + r2 * k.c));
        }
        tot.add(acc);
    }
    if (valid)
        part[(size_t)sp * HAWKES_NOALLOC_MAX_N + row] = tot.value();
}

__device__ double block_sum(double v, double *sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = kFinishThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// ell = sum_n log(lambda_n) - Lambda_n in one CTA, fixed summation order.
__global__ void __launch_bounds__(kFinishThreads) noalloc_finish_kernel(const double *__restrict__ t, int n,
                                                                        Consts k, int fsplit,
                                                                        const double *__restrict__ part,
                                                                        const unsigned *status, double *out)
{
    __shared__ double sh[kFinishThreads];
    double tmax = -INFINITY;
    for (int i = threadIdx.x; i < n; i += kFinishThreads)
        tmax = fmax(tmax, t[i]);
    sh[threadIdx.x] = tmax;
    __syncthreads();
    for (int o = kFinishThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    const double T = sh[0];
    __syncthreads();
    Nsum acc;
    for (int i = threadIdx.x; i < n; i += kFinishThreads) {
        Nsum lam;
        for (int sp = 0; sp < fsplit; ++sp)
            lam.add(part[(size_t)sp * HAWKES_NOALLOC_MAX_N + i]);
        const double a = T - t[i];
        const double Lam = k.mu0 * (normcdf(a / k.tau_t) - normcdf(-t[i] / k.tau_t)) - k.theta * expm1(-k.omega * a);
        acc.add(log(lam.value()) - Lam);
    }
    const double ell = block_sum(acc.value(), sh);
    if (threadIdx.x == 0)
        *out = (*status != 0u) ? nan("") : ell;
}

}  // namespace

extern "C" hawkes_status hawkes_loglik_noalloc(const double *t, const double *X, int64_t n, int32_t d,
                                               const hawkes_params *params, hawkes_stream stream,
                                               double *out_loglik)
{
    if (!t || !X || !out_loglik || !params || d < 1 || d > kMaxDim || n < 1 || n > HAWKES_NOALLOC_MAX_N)
        return HAWKES_ERR_INVALID_ARG;
    const double v[6] = {params->mu0, params->tau_x, params->tau_t, params->theta, params->omega, params->h};
    for (double x : v)
        if (!(x > 0.0) || !std::isfinite(x))
            return HAWKES_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return HAWKES_ERR_CUDA;
    double *scratch = nullptr;
    hawkes_status st = scratch_in_current_context(&scratch);
    if (st != HAWKES_OK)
        return st;
    double *part = scratch;
    unsigned *status = reinterpret_cast<unsigned *>(scratch + (size_t)kMaxSplit * HAWKES_NOALLOC_MAX_N);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    const double two_pi = 6.283185307179586476925286766559;
    const hawkes_params &p = *params;
    Consts k;
    k.a = 0.5 / (p.tau_x * p.tau_x);
    k.b = 0.5 / (p.tau_t * p.tau_t);
    k.c = 0.5 / (p.h * p.h);
    k.Cmu = p.mu0 / (std::pow(p.tau_x, d) * p.tau_t * std::pow(two_pi, 0.5 * (d + 1)));
    k.Cxi = p.theta * p.omega / (std::pow(p.h, d) * std::pow(two_pi, 0.5 * d));
    k.omega = p.omega;
    k.mu0 = p.mu0;
    k.tau_t = p.tau_t;
    k.theta = p.theta;

    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = (int)((n + kTile - 1) / kTile);
    int fsplit = sms > 0 ? (8 * sms + tiles - 1) / tiles : 1;
    fsplit = fsplit < 1 ? 1 : (fsplit > kMaxSplit ? kMaxSplit : fsplit);
    if (fsplit > tiles)
        fsplit = tiles;

    // the status word must start at zero; the partial sums are all rewritten
    if (cudaMemsetAsync(status, 0, sizeof(unsigned), s) != cudaSuccess)
        return HAWKES_ERR_CUDA;
    noalloc_rates_kernel<<<dim3(tiles, fsplit), kTile, 0, s>>>(t, X, (int)n, d, k, fsplit, part, status);
    noalloc_finish_kernel<<<1, kFinishThreads, 0, s>>>(t, (int)n, k, fsplit, part, status, out_loglik);
    return cudaGetLastError() == cudaSuccess ? HAWKES_OK : HAWKES_ERR_CUDA;
}
