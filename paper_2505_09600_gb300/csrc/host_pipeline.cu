// lisa_response_hybrid_host: the hybrid response (Sec. IV, Eq. hybridized_xs)
// of series held in host memory, with the host<->device copies overlapped
// with the computation.
//
// The output grid is cut into K chunks whose boundaries fall on the LFA
// kernel's tile groups, so every kernel sees exactly the tiles it would see in
// one call.  Three streams run a pipeline:
//   copy-in (internal stream):  h+, hx of chunk c and the halo its retarded
//                               times reach ahead of it;
//   compute (the caller's stream and an internal one, chunks alternating):
//                               LFA / links / TDI of chunk c once its input
//                               copy has landed (event);
//   copy-out (internal stream): X, Y, Z (or A, E, T) of chunk c once it is
//                               computed (event).
// With pinned host buffers the copies of chunk c+1 and the read-back of
// chunk c-1 overlap the kernels of chunk c.  The device buffers come from the
// stream-ordered allocator on the caller's stream and are released there
// after the last read-back.
#include <math.h>

#include <mutex>
#include <vector>

#include "lisa_common.cuh"
#include "lisa_internal.cuh"

using namespace lisa;

#ifndef LISA_HOST_CHUNKS
#define LISA_HOST_CHUNKS 8
#endif
#ifndef LISA_HOST_EDGE
#define LISA_HOST_EDGE 1
#endif

namespace {

constexpr int kMaxChunks = 16;
constexpr int kChunks = LISA_HOST_CHUNKS;
static_assert(kChunks >= 1 && kChunks <= kMaxChunks, "LISA_HOST_CHUNKS out of range");

// Streams and events of one pipeline.  They live for the process and are
// reused by later calls on the same device (creating three streams and 2K+2
// events per call cost tens of microseconds of host time before the first
// copy could be queued).  A set is held by one call at a time; work a
// previous call left queued on its streams runs before the next call's.
struct PipeRes {
    int device = -1;
    bool busy = false;
    cudaStream_t s_in = nullptr, s_out = nullptr, s_cmp2 = nullptr;
    cudaEvent_t e_ready = nullptr, e_tab = nullptr, e_done = nullptr;
    cudaEvent_t e_in[kMaxChunks] = {}, e_cmp[kMaxChunks] = {};
};

std::mutex g_pipe_mu;
std::vector<PipeRes*> g_pipes;

void pipe_destroy(PipeRes* p)
{
    for (int c = 0; c < kMaxChunks; ++c) {
        if (p->e_in[c]) cudaEventDestroy(p->e_in[c]);
        if (p->e_cmp[c]) cudaEventDestroy(p->e_cmp[c]);
    }
    if (p->e_ready) cudaEventDestroy(p->e_ready);
    if (p->e_tab) cudaEventDestroy(p->e_tab);
    if (p->e_done) cudaEventDestroy(p->e_done);
    if (p->s_in) cudaStreamDestroy(p->s_in);
    if (p->s_out) cudaStreamDestroy(p->s_out);
    if (p->s_cmp2) cudaStreamDestroy(p->s_cmp2);
    delete p;
}

PipeRes* pipe_acquire(int& rc)
{
    int dev = 0;
    rc = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return nullptr;
    {
        std::lock_guard<std::mutex> lk(g_pipe_mu);
        for (PipeRes* p : g_pipes)
            if (!p->busy && p->device == dev) {
                p->busy = true;
                return p;
            }
    }
    PipeRes* p = new PipeRes;
    p->device = dev;
    rc = cuda_status(cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking), "cudaStreamCreate");
    if (!rc) rc = cuda_status(cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking), "cudaStreamCreate");
    if (!rc) rc = cuda_status(cudaStreamCreateWithFlags(&p->s_cmp2, cudaStreamNonBlocking), "cudaStreamCreate");
    if (!rc) rc = cuda_status(cudaEventCreateWithFlags(&p->e_ready, cudaEventDisableTiming), "cudaEventCreate");
    if (!rc) rc = cuda_status(cudaEventCreateWithFlags(&p->e_tab, cudaEventDisableTiming), "cudaEventCreate");
    if (!rc) rc = cuda_status(cudaEventCreateWithFlags(&p->e_done, cudaEventDisableTiming), "cudaEventCreate");
    for (int c = 0; c < kMaxChunks && !rc; ++c) {
        rc = cuda_status(cudaEventCreateWithFlags(&p->e_in[c], cudaEventDisableTiming), "cudaEventCreate");
        if (!rc) rc = cuda_status(cudaEventCreateWithFlags(&p->e_cmp[c], cudaEventDisableTiming), "cudaEventCreate");
    }
    if (rc) {
        pipe_destroy(p);
        return nullptr;
    }
    p->busy = true;
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    g_pipes.push_back(p);
    return p;
}

void pipe_release(PipeRes* p)
{
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    p->busy = false;
}

}  // namespace

extern "C" int lisa_response_hybrid_host(const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid grid,
                                         const void* hp_host, const void* hc_host, int precision, int tdi_gen,
                                         int lfa_kind, int channels, double t_hyb, double T_win, double sigma,
                                         void* xyz_host, void* stream)
{
    LISA_TRY(check_orbit(orbit));
    LISA_TRY(check_grid(grid, "grid"));
    LISA_TRY(check_common(precision, tdi_gen, channels));
    if (!lfa_kind_ok(lfa_kind)) { set_error("lfa_kind %d unknown", lfa_kind); return LISA_EINVAL; }
    if (!sky) { set_error("sky is NULL"); return LISA_EINVAL; }
    if (!isfinite(t_hyb)) { set_error("t_hyb must be finite"); return LISA_EINVAL; }
    if (grid.n == 0) return LISA_OK;
    if (!xyz_host || !hp_host || !hc_host) { set_error("NULL series pointer"); return LISA_EINVAL; }
    const double Tw = T_win > 0.0 ? T_win : 800.0 * grid.dt;
    const double sg = sigma > 0.0 ? sigma : Tw / 40.0;
    const int64_t n = grid.n;
    const size_t rs = real_size(precision);
    int64_t iL, iF;
    hybrid_split(grid, t_hyb, Tw, iL, iF);

    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc(st);
    char* hp = (char*)sc.alloc((size_t)n * rs);
    char* hc = (char*)sc.alloc((size_t)n * rs);
    char* xyz = (char*)sc.alloc(3 * (size_t)n * rs);
    // one link buffer per compute stream (their chunks' link ranges overlap)
    char* ybuf[2] = {nullptr, nullptr};
    for (int q = 0; q < 2 && iF < n; ++q) ybuf[q] = (char*)sc.alloc(6 * (size_t)n * rs);
    if (!hp || !hc || !xyz || (iF < n && (!ybuf[0] || !ybuf[1]))) return sc.status();

    // chunks: whole LFA tile groups, at most kChunks.  With LISA_HOST_EDGE
    // the first and last chunks are half as long as the others: the first
    // copy-in and the last read-back are the parts of the pipeline that
    // nothing overlaps.
    const int64_t gt = (int64_t)lfa_group_host(grid.dt, precision) * kTile;
    const int64_t groups = (n + gt - 1) / gt;
    const int K = (int)(groups < kChunks ? groups : kChunks);
    int64_t cb[kMaxChunks + 1];   // chunk c = samples [cb[c], cb[c + 1])
    {
        const int edge = (LISA_HOST_EDGE && K >= 3) ? 1 : 2;
        const int64_t wsum = 2 * (int64_t)K - 2 * (2 - edge);
        int64_t acc = 0;
        cb[0] = 0;
        for (int c = 0; c < K; ++c) {
            acc += (c == 0 || c == K - 1) ? edge : 2;
            const int64_t g = groups * acc / wsum;
            cb[c + 1] = g * gt < n ? g * gt : n;
        }
        cb[K] = n;
    }
    // samples the retarded times reach ahead of (and behind) an output sample:
    // |k.R/c| <= 1.01 AU/c, the light times, the stencils and window margins
    const double Tmax = max_light_time(orbit, grid);
    const int64_t halo = (int64_t)ceil((1.01 * kAU / kC + 3.0 * Tmax) / grid.dt) + 160;
    const int64_t back = (int64_t)ceil(8.0 * Tmax / grid.dt) + 40;   // TDI delays (as lisa_response_hybrid)
    const int64_t lo_links = iF - back > 0 ? iF - back : 0;

    // chunks alternate between two compute streams (the caller's and an
    // internal one), so that one chunk's kernels fill the SMs left idle by
    // the other's tail
    int rc = 0;
    PipeRes* R = pipe_acquire(rc);
    if (!R) return rc;
    cudaStream_t s_in = R->s_in, s_out = R->s_out, s_cmp2 = R->s_cmp2;
    cudaEvent_t e_ready = R->e_ready;
    cudaEvent_t* e_in = R->e_in;
    cudaEvent_t* e_cmp = R->e_cmp;
    // the copy streams start after the allocations on the caller's stream;
    // the first input copy overlaps the orbit table, which the second compute
    // stream waits for
    rc = cuda_status(cudaEventRecord(e_ready, st), "cudaEventRecord");
    if (!rc) rc = cuda_status(cudaStreamWaitEvent(s_in, e_ready, 0), "cudaStreamWaitEvent");
    if (!rc) rc = cuda_status(cudaStreamWaitEvent(s_out, e_ready, 0), "cudaStreamWaitEvent");
    SegTable tab;
    if (!rc) rc = make_table(orbit, grid, sc, tab, st);
    const SkyDev skyd = make_sky_dev(*sky);
    if (!rc) rc = cuda_status(cudaEventRecord(R->e_tab, st), "cudaEventRecord");
    if (!rc) rc = cuda_status(cudaStreamWaitEvent(s_cmp2, R->e_tab, 0), "cudaStreamWaitEvent");
    const cudaStream_t cs[2] = {st, s_cmp2};

    int64_t h_done = 0;
    for (int c = 0; c < K && !rc; ++c) {
        const int64_t a = cb[c], b = cb[c + 1];
        if (a >= b) continue;
        // copy-in: h up to b + halo
        int64_t h_to = b + halo < n ? b + halo : n;
        if (c == K - 1) h_to = n;
        if (h_to > h_done) {
            const size_t off = (size_t)h_done * rs, bytes = (size_t)(h_to - h_done) * rs;
            rc = cuda_status(cudaMemcpyAsync(hp + off, (const char*)hp_host + off, bytes, cudaMemcpyHostToDevice, s_in),
                             "cudaMemcpyAsync(h+)");
            if (!rc)
                rc = cuda_status(cudaMemcpyAsync(hc + off, (const char*)hc_host + off, bytes, cudaMemcpyHostToDevice, s_in),
                                 "cudaMemcpyAsync(hx)");
            h_done = h_to;
        }
        const cudaStream_t sc_c = cs[c & 1];
        char* y = ybuf[c & 1];
        if (!rc) rc = cuda_status(cudaEventRecord(e_in[c], s_in), "cudaEventRecord");
        if (!rc) rc = cuda_status(cudaStreamWaitEvent(sc_c, e_in[c], 0), "cudaStreamWaitEvent");
        if (rc) break;
        // compute chunk [a, b)
        if (a <= iL) {
            BlendSpec bl{1, t_hyb, sg, +1.0, 0, 0};
            const int64_t e = b < iL + 1 ? b : iL + 1;
            rc = launch_lfa(tab, skyd, orbit->L_m, grid, hp, hc, precision, tdi_gen, lfa_kind, channels, grid, nullptr,
                            xyz, a, e, bl, sc_c);
        }
        if (!rc && iF > iL + 1) {
            const int64_t z0 = iL + 1 > a ? iL + 1 : a, z1 = iF < b ? iF : b;
            for (int q = 0; q < 3 && !rc && z1 > z0; ++q)
                rc = cuda_status(cudaMemsetAsync(xyz + ((size_t)q * n + (size_t)z0) * rs, 0, (size_t)(z1 - z0) * rs, sc_c),
                                 "cudaMemsetAsync");
        }
        if (!rc && b > iF) {
            int64_t l0 = a - back > lo_links ? a - back : lo_links;
            int64_t l1 = b + 40 < n ? b + 40 : n;
            rc = launch_links_full(tab, skyd, grid, hp, hc, precision, grid, y, l0, l1, sc_c);
            if (!rc) {
                BlendSpec bl{1, t_hyb, sg, -1.0, iF, iL + 1};
                rc = launch_tdi(tab, grid, y, precision, tdi_gen, LISA_FROZEN, channels, grid, xyz, a > iF ? a : iF, b, bl,
                                sc_c);
            }
        }
        if (!rc) rc = cuda_status(cudaEventRecord(e_cmp[c], sc_c), "cudaEventRecord");
        // copy-out of chunk c
        if (!rc) rc = cuda_status(cudaStreamWaitEvent(s_out, e_cmp[c], 0), "cudaStreamWaitEvent");
        if (!rc)
            rc = cuda_status(cudaMemcpy2DAsync((char*)xyz_host + (size_t)a * rs, (size_t)n * rs, xyz + (size_t)a * rs,
                                               (size_t)n * rs, (size_t)(b - a) * rs, 3, cudaMemcpyDeviceToHost, s_out),
                             "cudaMemcpy2DAsync(xyz)");
    }
    // the caller's stream (and the scratch release on it) waits for the last read-back
    if (!rc) rc = cuda_status(cudaEventRecord(R->e_done, s_out), "cudaEventRecord");
    if (!rc) rc = cuda_status(cudaStreamWaitEvent(st, R->e_done, 0), "cudaStreamWaitEvent");
    if (rc) {
        // an error after work was queued: let the queued work finish before
        // the scratch goes back to the pool
        cudaStreamSynchronize(s_in);
        cudaStreamSynchronize(s_cmp2);
        cudaStreamSynchronize(s_out);
        cudaStreamSynchronize(st);
    }
    pipe_release(R);
    return rc;
}
