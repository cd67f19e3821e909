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

}  // namespace lisa

using namespace lisa;

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
