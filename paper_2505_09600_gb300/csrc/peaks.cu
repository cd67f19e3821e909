// Arithmetic peak microbenchmarks: fused multiply-add throughput of the FP32
// and FP64 pipes, measured by the caller around one launch.
//
// Each thread runs kChains independent recurrences x <- x m + a for `iters`
// steps (2 flop per step), so the pipe is never waiting on one chain's
// latency.  m and a come from the arguments, which keeps the compiler from
// folding the loop; every chain's final value is summed into one store per
// thread, so no step is dead code.  The FP32 kernel issues the steps as
// packed pairs (__ffma2_rn, two multiply-adds per instruction) or as scalar
// multiply-adds; the caller takes the better of the two.  The grid is
// `blocks_per_sm` CTAs of 256 threads on every SM.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lisa_internal.cuh"

namespace lisa {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(T m, T a, int64_t iters, T* sink)
{
    T x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], m, a);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += x[k];
    sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) fma2_peak_kernel(float m, float a, int64_t iters, float* sink)
{
    float2 x[kChains / 2];
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k) x[k] = make_float2(float(threadIdx.x + 2 * k) * 1e-3f, float(threadIdx.x + 2 * k + 1) * 1e-3f);
    const float2 m2 = make_float2(m, m), a2 = make_float2(a, a);
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < kChains / 2; ++k) x[k] = __ffma2_rn(x[k], m2, a2);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains / 2; ++k) s += x[k].x + x[k].y;
    sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace lisa

using namespace lisa;

extern "C" int lisa_peak_fma_blocks(int blocks_per_sm, int64_t* blocks)
{
    if (blocks_per_sm < 1 || blocks_per_sm > 64 || !blocks) {
        set_error("lisa_peak_fma_blocks: blocks_per_sm must be in 1..64");
        return LISA_EINVAL;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_status(e, "cudaDeviceGetAttribute");
    *blocks = (int64_t)sms * blocks_per_sm;
    return LISA_OK;
}

extern "C" int lisa_peak_fma(int kind, int64_t iters, int blocks_per_sm, void* sink, double* flop, void* stream)
{
    if (kind < 0 || kind > 2 || iters < 1 || !sink || !flop) {
        set_error("lisa_peak_fma: kind 0 (FP64), 1 (FP32) or 2 (FP32 pairs), iters >= 1, sink and flop non-NULL");
        return LISA_EINVAL;
    }
    int64_t blocks = 0;
    int rc = lisa_peak_fma_blocks(blocks_per_sm, &blocks);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    prof_before(kind == 0 ? "peak_fma_f64" : "peak_fma_f32", st);
    if (kind == 0)
        fma_peak_kernel<double><<<(unsigned)blocks, 256, 0, st>>>(0.9999999, 1e-7, iters, (double*)sink);
    else if (kind == 1)
        fma_peak_kernel<float><<<(unsigned)blocks, 256, 0, st>>>(0.9999f, 1e-4f, iters, (float*)sink);
    else
        fma2_peak_kernel<<<(unsigned)blocks, 256, 0, st>>>(0.9999f, 1e-4f, iters, (float*)sink);
    prof_after(st);
    *flop = 2.0 * (double)kChains * (double)iters * 256.0 * (double)blocks;
    return cuda_status(cudaGetLastError(), "fma_peak_kernel launch");
}
