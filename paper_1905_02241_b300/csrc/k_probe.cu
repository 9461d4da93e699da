// k_probe.cu -- throughput probes of the arithmetic pipes that bound the
// mechanism kernels (the FP64 FMA pipe for the plain FP64 path; the FP32 FMA
// and exp2 (MUFU) pipes for the mixed path).  Each thread runs independent
// dependency chains so that the pipe, not latency, limits the rate.  The
// grid is a multiple of the SM count.
#include <algorithm>

#include "kernels.cuh"
#include "runtime.cuh"
#include "tcgen05.cuh"

namespace nmodl {

constexpr int kChains = 8;

__global__ void k_probe_dfma(double* sink, int iters, double a, double b) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (threadIdx.x + c) * 1e-3;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    double s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678) sink[0] = s;
}

__global__ void k_probe_ffma(float* sink, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    float s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) sink[0] = s;
}

__global__ void k_probe_ex2(float* sink, int iters) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = -(threadIdx.x % 7 + c) * 1e-3f;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = exp2f(x[c]) - 1.0f;  // stays in [-1, 0]
    float s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) sink[0] = s;
}

__global__ void k_math_eval(int fn, int64_t n, const double* __restrict__ x, double* y) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    y[i] = fn == 0   ? exp_tang(x[i])
           : fn == 1 ? exp(x[i])
           : fn == 2 ? f2d_int(d2f_int(x[i]))
           : fn == 3 ? rcp_fast(x[i])
           : fn == 4 ? ddiv_fast(x[2 * i], x[2 * i + 1])
           : fn == 5 ? one_pm_exp<1>(x[i])
                     : one_pm_exp<-1>(x[i]);
}

// The bounded mbarrier wait of the tensor-core kernels, on a barrier that
// nothing arrives at: every thread polls it `polls` times, gives up, and the
// block latches NMODL_ERR_TIMEOUT -- the path a stalled MMA completion would
// take, exercised without stalling anything.  The barrier lives in this
// block's shared memory and is invalidated before the block exits.
__global__ void k_probe_wait(uint32_t polls, int32_t* err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0, polls);
    const bool any_timeout = __syncthreads_or(!ok);
    if (threadIdx.x == 0) {
        if (any_timeout) latch_error(err, NMODL_ERR_TIMEOUT);
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_u32(&bar)) : "memory");
    }
}

}  // namespace nmodl

using namespace nmodl;

// Run the bounded wait on the context's stream; the timeout is latched in the
// context like any device error and returned by the next nmodl_sync.
extern "C" NMODL_API int nmodl_probe_wait(nmodl_ctx* ctx, int32_t polls) {
    if (!ctx || polls < 1 || polls > (1 << 20)) return NMODL_ERR_ARG;
    DeviceGuard g(ctx->device);
    k_probe_wait<<<1, 128, 0, ctx->stream>>>((uint32_t)polls, ctx->d_err);
    return cudaGetLastError() == cudaSuccess ? NMODL_OK : NMODL_ERR_CUDA;
}

// fn 0: the library's table-driven FP64 exp; fn 1: CUDA exp (for comparison);
// fn 2: rounding to float and back through the integer-pipe conversions;
// fn 3: the refined hardware reciprocal of the gate and node updates
extern "C" NMODL_API int nmodl_math_eval(int fn, int64_t n, const double* x, double* y,
                                         void* stream) {
    if (fn < 0 || fn > 6 || n < 0 || (n > 0 && (!x || !y))) return NMODL_ERR_ARG;
    if (n == 0) return NMODL_OK;
    k_math_eval<<<(int)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(fn, n, x, y);
    return cudaGetLastError() == cudaSuccess ? NMODL_OK : NMODL_ERR_CUDA;
}

// kind 0: FP64 FMA, 1: FP32 FMA (ops = lane FMAs / s), 2: exp2 (lane ops / s)
extern "C" NMODL_API int nmodl_probe_peak(int device, int kind, double* ops_per_s) {
    if (!ops_per_s || kind < 0 || kind > 2) return NMODL_ERR_ARG;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    double* sink = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = NMODL_OK;
    if (cudaMalloc(&sink, 64) != cudaSuccess || cudaStreamCreate(&s) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = NMODL_ERR_CUDA;
    } else {
        const int block = 256;
        const int grid = sms * 8;
        int iters = kind == 0 ? 512 : 8192;
        double best = 0.0;
        for (int rep = 0; rep < 7 && rc == NMODL_OK; ++rep) {
            cudaEventRecord(e0, s);
            if (kind == 0) k_probe_dfma<<<grid, block, 0, s>>>(sink, iters, 0.999999, 1e-7);
            else if (kind == 1) k_probe_ffma<<<grid, block, 0, s>>>((float*)sink, iters, 0.9999f, 1e-5f);
            else k_probe_ex2<<<grid, block, 0, s>>>((float*)sink, iters);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = NMODL_ERR_CUDA; break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            const double ops = (double)grid * block * iters * kChains;
            if (rep > 0) best = std::max(best, ops / (ms * 1e-3));
            if (ms < 20.f) iters *= 2;  // grow until the launch runs >= 20 ms
        }
        *ops_per_s = best;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (sink) cudaFree(sink);
    cudaSetDevice(prev);
    return rc;
}
