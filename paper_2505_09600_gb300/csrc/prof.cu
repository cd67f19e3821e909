// Launch accounting and optional per-launch device timing (CUDA event pairs
// recorded on each launch's own stream).
#include <atomic>
#include <mutex>
#include <string.h>
#include <vector>

#include "lisa_internal.cuh"

namespace lisa {

namespace {
struct Rec {
    const char* name;
    cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::atomic<int64_t> g_launches{0};
thread_local Rec t_pending{nullptr, nullptr, nullptr};
}  // namespace

void prof_before(const char* name, cudaStream_t st)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return;
    Rec r{name, nullptr, nullptr};
    if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) return;
    cudaEventRecord(r.a, st);
    t_pending = r;
}

void prof_after(cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on || !t_pending.name) return;
    cudaEventRecord(t_pending.b, st);
    g_recs.push_back(t_pending);
    t_pending = Rec{nullptr, nullptr, nullptr};
}

static void clear_locked()
{
    for (auto& r : g_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    g_recs.clear();
}

}  // namespace lisa

using namespace lisa;

extern "C" int lisa_profile_enable(int enable)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (enable) clear_locked();
    g_on = enable != 0;
    return LISA_OK;
}

extern "C" int lisa_profile_query(const char* name, double* total_ms, int64_t* launches)
{
    std::lock_guard<std::mutex> lk(g_mu);
    double tot = 0.0;
    int64_t cnt = 0;
    for (auto& r : g_recs) {
        if (name && !strstr(r.name, name)) continue;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return cuda_status(e, "cudaEventSynchronize");
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) return cuda_status(e, "cudaEventElapsedTime");
        tot += ms;
        ++cnt;
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = cnt;
    return LISA_OK;
}

extern "C" int64_t lisa_launch_count(void) { return g_launches.load(); }
