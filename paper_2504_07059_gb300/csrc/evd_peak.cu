// evd_peak.cu -- arithmetic throughput of this GPU (a diagnostic beside the
// step): independent FMA chains on every SM, timed with CUDA events, in
// double, float, and float pairs (f32x2).  The step's FP64 path is bound by
// the double-precision rate, so its roofline is this rate, not HBM.
#include <cuda_runtime.h>

#include <string>

#include "evd.h"
#include "evd_internal.h"

namespace {

constexpr int PK_BLOCK = 256;
constexpr int PK_CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(PK_BLOCK) evd_k_fma_chains(T* __restrict__ out, int iters, T a, T b)
{
    T x[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = (T)(threadIdx.x + c);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) x[c] = fma(x[c], a, b);
    T s = x[0];
#pragma unroll
    for (int c = 1; c < PK_CHAINS; ++c) s += x[c];
    out[blockIdx.x * PK_BLOCK + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PK_BLOCK) evd_k_fma2_chains(float2* __restrict__ out, int iters, float2 a, float2 b)
{
    float2 x[PK_CHAINS];
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = make_float2((float)threadIdx.x, (float)c);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int c = 0; c < PK_CHAINS; ++c) x[c] = __ffma2_rn(x[c], a, b);
    float2 s = x[0];
#pragma unroll
    for (int c = 1; c < PK_CHAINS; ++c) s = __fadd2_rn(s, x[c]);
    out[blockIdx.x * PK_BLOCK + threadIdx.x] = s;
}

}  // namespace

extern "C" evd_status evd_fma_rate(int kind, int iters, double* flops, double* ms, void* cuda_stream)
{
    if (!flops || !ms) { evd::set_thread_error("flops and ms must not be NULL"); return EVD_ERR_ARG; }
    if (kind < 0 || kind > 2) { evd::set_thread_error("kind must be 0 (FP64), 1 (FP32) or 2 (FP32 pairs)"); return EVD_ERR_ARG; }
    if (iters < 1 || iters > (1 << 24)) { evd::set_thread_error("iters must be 1 .. 2^24"); return EVD_ERR_ARG; }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8;
    const size_t n = (size_t)blocks * PK_BLOCK;
    void* out = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (e == cudaSuccess) e = cudaMalloc(&out, n * 8);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    auto launch = [&]() {
        if (kind == 0) evd_k_fma_chains<double><<<blocks, PK_BLOCK, 0, st>>>((double*)out, iters, 0.9999999, 1e-7);
        else if (kind == 1) evd_k_fma_chains<float><<<blocks, PK_BLOCK, 0, st>>>((float*)out, iters, 0.9999f, 1e-4f);
        else evd_k_fma2_chains<<<blocks, PK_BLOCK, 0, st>>>((float2*)out, iters, make_float2(0.9999f, 0.9998f),
                                                            make_float2(1e-4f, 2e-4f));
    };
    float t = 0.0f;
    if (e == cudaSuccess) {
        launch();   // warm-up
        e = cudaEventRecord(a, st);
    }
    if (e == cudaSuccess) {
        launch();
        e = cudaEventRecord(b, st);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (out) cudaFree(out);
    if (e != cudaSuccess) {
        evd::set_thread_error(std::string("evd_fma_rate: ") + cudaGetErrorString(e));
        return EVD_ERR_CUDA;
    }
    // two flops per fused multiply-add, two lanes per pair
    *flops = 2.0 * (kind == 2 ? 2.0 : 1.0) * (double)n * PK_CHAINS * (double)iters;
    *ms = (double)t;
    return EVD_OK;
}
