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

#include "lisa_common.cuh"
#include "lisa_internal.cuh"

using namespace lisa;

extern "C" int lisa_response_hybrid_host(const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid grid,
                                         const void* hp_host, const void* hc_host, int precision, int tdi_gen,
                                         int lfa_kind, int channels, double t_hyb, double T_win, double sigma,
                                         void* xyz_host, void* stream)
{
    LISA_TRY(check_orbit(orbit));
    LISA_TRY(check_grid(grid, "grid"));
    LISA_TRY(check_common(precision, tdi_gen, channels));
    if (lfa_kind != LISA_LFA_UNEQUAL && lfa_kind != LISA_LFA_EQUAL) { set_error("lfa_kind %d unknown", lfa_kind); return LISA_EINVAL; }
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
    SegTable tab;
    LISA_TRY(make_table(orbit, grid, sc, tab, st));
    const SkyDev skyd = make_sky_dev(*sky);
    char* hp = (char*)sc.alloc((size_t)n * rs);
    char* hc = (char*)sc.alloc((size_t)n * rs);
    char* xyz = (char*)sc.alloc(3 * (size_t)n * rs);
    // one link buffer per compute stream (their chunks' link ranges overlap)
    char* ybuf[2] = {nullptr, nullptr};
    for (int q = 0; q < 2 && iF < n; ++q) ybuf[q] = (char*)sc.alloc(6 * (size_t)n * rs);
    if (!hp || !hc || !xyz || (iF < n && (!ybuf[0] || !ybuf[1]))) return sc.status();

    // chunks: whole LFA tile groups, at most 8
    const int64_t gt = (int64_t)lfa_group_host(grid.dt) * kTile;
    const int64_t groups = (n + gt - 1) / gt;
    const int K = (int)(groups < 8 ? groups : 8);
    const int64_t C = (groups + K - 1) / K * gt;
    // samples the retarded times reach ahead of (and behind) an output sample:
    // |k.R/c| <= 1.01 AU/c, the light times, the stencils and window margins
    const double Tmax = max_light_time(orbit, grid);
    const int64_t halo = (int64_t)ceil((1.01 * kAU / kC + 3.0 * Tmax) / grid.dt) + 160;
    const int64_t back = (int64_t)ceil(8.0 * Tmax / grid.dt) + 40;   // TDI delays (as lisa_response_hybrid)
    const int64_t lo_links = iF - back > 0 ? iF - back : 0;

    // chunks alternate between two compute streams (the caller's and an
    // internal one), so that one chunk's kernels fill the SMs left idle by
    // the other's tail
    cudaStream_t s_in = nullptr, s_out = nullptr, s_cmp2 = nullptr;
    cudaEvent_t e_ready = nullptr, e_in[8] = {}, e_cmp[8] = {};
    int rc = cuda_status(cudaStreamCreateWithFlags(&s_in, cudaStreamNonBlocking), "cudaStreamCreate");
    if (!rc) rc = cuda_status(cudaStreamCreateWithFlags(&s_out, cudaStreamNonBlocking), "cudaStreamCreate");
    if (!rc) rc = cuda_status(cudaStreamCreateWithFlags(&s_cmp2, cudaStreamNonBlocking), "cudaStreamCreate");
    if (!rc) rc = cuda_status(cudaEventCreateWithFlags(&e_ready, cudaEventDisableTiming), "cudaEventCreate");
    for (int c = 0; c < K && !rc; ++c) {
        rc = cuda_status(cudaEventCreateWithFlags(&e_in[c], cudaEventDisableTiming), "cudaEventCreate");
        if (!rc) rc = cuda_status(cudaEventCreateWithFlags(&e_cmp[c], cudaEventDisableTiming), "cudaEventCreate");
    }
    // the copy streams start after the allocations on the caller's stream
    if (!rc) rc = cuda_status(cudaEventRecord(e_ready, st), "cudaEventRecord");
    if (!rc) rc = cuda_status(cudaStreamWaitEvent(s_in, e_ready, 0), "cudaStreamWaitEvent");
    if (!rc) rc = cuda_status(cudaStreamWaitEvent(s_out, e_ready, 0), "cudaStreamWaitEvent");
    if (!rc) rc = cuda_status(cudaStreamWaitEvent(s_cmp2, e_ready, 0), "cudaStreamWaitEvent");
    const cudaStream_t cs[2] = {st, s_cmp2};

    int64_t h_done = 0;
    for (int c = 0; c < K && !rc; ++c) {
        const int64_t a = (int64_t)c * C;
        const int64_t b = a + C < n ? a + C : n;
        if (a >= b) break;
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
    if (!rc) rc = cuda_status(cudaEventRecord(e_ready, s_out), "cudaEventRecord");
    if (!rc) rc = cuda_status(cudaStreamWaitEvent(st, e_ready, 0), "cudaStreamWaitEvent");
    if (rc) {
        // an error after work was queued: let the queued work finish before
        // the scratch goes back to the pool
        cudaStreamSynchronize(s_in);
        cudaStreamSynchronize(s_cmp2);
        cudaStreamSynchronize(s_out);
        cudaStreamSynchronize(st);
    }
    for (int c = 0; c < K; ++c) {
        if (e_in[c]) cudaEventDestroy(e_in[c]);
        if (e_cmp[c]) cudaEventDestroy(e_cmp[c]);
    }
    if (e_ready) cudaEventDestroy(e_ready);
    if (s_in) cudaStreamDestroy(s_in);
    if (s_out) cudaStreamDestroy(s_out);
    if (s_cmp2) cudaStreamDestroy(s_cmp2);
    return rc;
}
