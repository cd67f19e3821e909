// Device status word of the bounded waits (see async_copy.cuh) and its query.
#include "lisa_common.cuh"
#include "lisa_internal.cuh"
#include "async_copy.cuh"

#include <mutex>

namespace lisa {

static __device__ unsigned int g_device_status = 0u;

unsigned int* device_status_ptr()
{
    static std::mutex mu;
    static unsigned int* addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_device_status) != cudaSuccess) return nullptr;
        addr[dev] = (unsigned int*)p;
    }
    return addr[dev];
}

// Test of the bounded-wait path: thread 0 of one CTA waits on an mbarrier
// that expects one arrival and gets none; the wait gives up after its bound
// (kAsyncSpinLimit polls, about a second), flags the status word and the
// kernel returns.
__global__ void wait_timeout_selftest_kernel(unsigned int* status)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
        if (!mbar_wait_bounded(&bar, 0)) flag_timeout(status);
    }
}

}  // namespace lisa

using namespace lisa;

extern "C" int lisa_selftest_wait_timeout(void* stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    unsigned int* status = device_status_ptr();
    if (!status) { set_error("device status word unavailable"); return LISA_ECUDA; }
    prof_before("wait_timeout_selftest", st);
    wait_timeout_selftest_kernel<<<1, 32, 0, st>>>(status);
    prof_after(st);
    return cuda_status(cudaGetLastError(), "wait_timeout_selftest_kernel");
}

extern "C" int lisa_device_status(unsigned int* status, int reset)
{
    unsigned int h = 0;
    LISA_TRY(cuda_status(cudaDeviceSynchronize(), "cudaDeviceSynchronize"));
    LISA_TRY(cuda_status(cudaMemcpyFromSymbol(&h, g_device_status, sizeof(h)), "cudaMemcpyFromSymbol"));
    if (status) *status = h;
    if (reset) {
        const unsigned int z = 0;
        LISA_TRY(cuda_status(cudaMemcpyToSymbol(g_device_status, &z, sizeof(z)), "cudaMemcpyToSymbol"));
    }
    if (h & 1u) {
        set_error("a bounded device-side wait timed out (status 0x%x)", h);
        return LISA_ETIMEOUT;
    }
    return LISA_OK;
}
