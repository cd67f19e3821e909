// Batched hybrid response: many sources of uneven duration in one persistent
// launch (mixed precision).
//
// A plan owns, in device memory allocated once at creation:
//   - one orbit polynomial table holding the segments of every source's grid
//     (built by one batched kernel per execution),
//   - a descriptor per source and the prefix of their tile counts,
//   - a work counter.
// The persistent kernel runs (SMs x CTAs per SM) blocks.  Each block takes the
// next work item -- a run of `tiles_per_item` consecutive output tiles of one
// source -- with one atomicAdd and, for every tile:
//   - computes the LFA channels of its samples with t <= t_hyb + T/2
//     (the same tile function as lisa_response_lfa),
//   - computes the full-response channels of its samples with
//     t >= t_hyb - T/2 by evaluating the six links over the window its TDI
//     delays reach directly into shared memory, then the TDI from there,
//   - blends them with the sigmoid weights of Eq. hybridized_xs and stores
//     X, Y, Z or A, E, T.
// Blocks never wait on each other (no spin, no grid barrier), so uneven
// sources are balanced by the queue alone.  The whole execution (counter
// reset, tables, persistent kernel) can be captured in a CUDA graph.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "lfa_tile.cuh"
#include "links_tile.cuh"
#include "tdi_tile.cuh"

struct lisa_plan;

namespace lisa {

struct BatchSrc {
    SegTable tab;
    SkyDev sky;
    GridMap hm;          // output grid -> h grid (identity here)
    const void* hp;
    const void* hc;
    void* out;
    int64_t n;
    double t0, dt;
    double t_hyb, sigma;
    float dtf, inv12dtf;  // FP32 copies of dt and 1/(12 dt)
    float c1f, c2f;       // 1/(12 dt), 1/(12 dt^2)
    int64_t iL, iF;      // LFA on samples <= iL, full response on samples >= iF
    int64_t tile_begin;  // first work tile of this source
    int64_t ntiles;
};

struct BatchKernelArgs {
    const BatchSrc* srcs;
    int nsrc;
    int64_t total_tiles;
    int tiles_per_item;
    unsigned long long* counter;
    int gen, kind, channels;
    double Lc;
    float Lcf;
};

struct BatchSmem {
    LfaSmem<true> lfa;        // also provides the tile geometry of the full part
    LinksTile<true> links;
    TdiTile<true> tdi;
    int64_t item;
    int src;
    float barg_c, barg_d;     // (t - t_hyb)/sigma at the tile centre, per sample
};

__device__ __forceinline__ void batch_full_part(const BatchKernelArgs& ka, const BatchSrc& b, int64_t i0,
                                                BatchSmem& sm, float (&Xf)[3])
{
    const int64_t ic = i0 + kTile / 2;
    const TileGeo& g = sm.lfa.g;
    TdiArgs ta;
    ta.tab = b.tab;
    ta.ym = b.hm;            // links live on the output grid: identity map
    ta.y = nullptr;
    ta.ny = b.n;
    ta.xyz = nullptr;
    ta.nout = b.n;
    ta.nterm = ka.gen == LISA_TDI20 ? 16 : 8;
    ta.mode = LISA_FROZEN;
    ta.channels = ka.channels;
    ta.i_begin = 0;
    ta.i_end = b.n;
    ta.tile0 = 0;
    ta.bl = BlendSpec{};
    ta.t0_out = b.t0;
    ta.dt_out = b.dt;
    tdi_tile_prologue<true>(ta, g, ic, i0, sm.tdi);
    LinksArgs la;
    la.tab = b.tab;
    la.sky = b.sky;
    la.hm = b.hm;
    la.hp = b.hp;
    la.hc = b.hc;
    la.y = nullptr;
    la.ny = b.n;
    la.i_begin = 0;
    la.i_end = b.n;
    la.tile0 = 0;
    const int64_t ylo = sm.tdi.wlo;
    const int ylen = sm.tdi.wlen;
    links_tile_prologue<true>(la, g, ic, ylo, ylo + (ylen > 0 ? ylen - 1 : 0), sm.links);
    for (int k = threadIdx.x; k < ylen; k += blockDim.x) {
        const int64_t m = ylo + k;
        if (m >= 0 && m < b.n) {
            links_sample<true>(la, g, ic, m, sm.links, &sm.tdi.win[0][k], kWinY);
        } else {
#pragma unroll
            for (int li = 0; li < 6; ++li) sm.tdi.win[li][k] = 0.f;
        }
    }
    __syncthreads();
    tdi_sample<true>(ta, g, ic, i0 + threadIdx.x, sm.tdi, Xf);
}

__global__ void __launch_bounds__(kTile) batch_hybrid_kernel(BatchKernelArgs ka)
{
    __shared__ BatchSmem sm;
    const int t = threadIdx.x;
    for (;;) {
        __syncthreads();   // the previous item is done with shared memory
        if (t == 0) {
            sm.item = (int64_t)atomicAdd(ka.counter, 1ull);
            const int64_t first = sm.item * ka.tiles_per_item;
            int lo = 0, hi = ka.nsrc - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (ka.srcs[mid].tile_begin <= first) lo = mid; else hi = mid - 1;
            }
            sm.src = lo;
        }
        __syncthreads();
        const int64_t first = sm.item * ka.tiles_per_item;
        if (first >= ka.total_tiles) break;
        int src = sm.src;
        for (int r = 0; r < ka.tiles_per_item; ++r) {
            const int64_t gt = first + r;
            if (gt >= ka.total_tiles) break;
            // an item may run into the next source: advance (uniform in the block)
            while (src + 1 < ka.nsrc && ka.srcs[src + 1].tile_begin <= gt) ++src;
            const BatchSrc& b = ka.srcs[src];
            const int64_t tile = gt - b.tile_begin;
            const int64_t i0 = tile * kTile;
            if (t == 0) {
                const double tc = b.t0 + (double)(i0 + kTile / 2) * b.dt;
                sm.barg_c = (float)((tc - b.t_hyb) / b.sigma);
                sm.barg_d = (float)(b.dt / b.sigma);
            }
            const bool need_lfa = i0 <= b.iL;
            const bool need_full = i0 + kTile - 1 >= b.iF;
            float Xl[3] = {0.f, 0.f, 0.f}, Xf[3] = {0.f, 0.f, 0.f};
            if (need_lfa) {
                LfaArgs a;
                a.tab = b.tab;
                a.sky = b.sky;
                a.hm = b.hm;
                a.Lc = ka.Lc;
                a.gen = ka.gen;
                a.kind = ka.kind;
                a.channels = ka.channels;
                a.hp = b.hp;
                a.hc = b.hc;
                a.z = nullptr;
                a.xyz = nullptr;
                a.nout = b.n;
                a.t0_out = b.t0;
                a.dt_out = b.dt;
                a.i_begin = 0;
                a.i_end = b.n;
                a.tile0 = 0;
                a.bl = BlendSpec{};
                a.Lcf = ka.Lcf;
                a.dtf = b.dtf;
                a.inv12dtf = b.inv12dtf;
                a.c1f = b.c1f;
                a.c2f = b.c2f;
                a.h_aligned = 0;
                a.status = nullptr;
                lfa_tile_compute<true>(a, i0, sm.lfa, Xl);
            } else {
                tile_geo_load(sm.lfa.g, b.tab, i0 + kTile / 2, b.sky);
            }
            if (need_full) {
                __syncthreads();
                batch_full_part(ka, b, i0, sm, Xf);
            }
            const int64_t i = i0 + t;
            if (i < b.n) {
                // X = S(+1) X_LFA [i <= iL] + S(-1) X_Full [i >= iF]
                const float arg = fmaf((float)(int)(i - (i0 + kTile / 2)), sm.barg_d, sm.barg_c);
                float o[3];
                const float wl = (i <= b.iL) ? 1.f / (1.f + expf(arg)) : 0.f;
                const float wf = (i >= b.iF) ? 1.f / (1.f + expf(-arg)) : 0.f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float v = 0.f;
                    if (wl != 0.f) v += wl * Xl[c];
                    if (wf != 0.f) v += wf * Xf[c];
                    o[c] = v;
                }
                float* out = (float*)b.out;
                if (ka.channels == LISA_AET) {
                    out[i] = (o[2] - o[0]) * 0.70710678118654752440f;
                    out[b.n + i] = (o[0] - 2.f * o[1] + o[2]) * 0.40824829046386301637f;
                    out[2 * b.n + i] = (o[0] + o[1] + o[2]) * 0.57735026918962576451f;
                } else {
                    out[i] = o[0];
                    out[b.n + i] = o[1];
                    out[2 * b.n + i] = o[2];
                }
            }
            __syncthreads();
        }
    }
}

}  // namespace lisa

using namespace lisa;

struct lisa_plan {
    int device = 0;
    int num_sms = 0;
    lisa_orbit orbit{};
    OrbitDev orb{};
    int gen = 20, kind = 0, channels = 1;
    int nsrc = 0;
    BatchSrc* d_srcs = nullptr;
    SegSource* d_segsrc = nullptr;
    double* d_coef = nullptr;
    unsigned long long* d_counter = nullptr;
    int64_t total_segs = 0, total_tiles = 0, total_samples = 0;
    int ctas_per_sm = 2, tiles_per_item = 1;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static int plan_enqueue(lisa_plan* p, cudaStream_t st)
{
    int rc = cuda_status(cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned long long), st), "cudaMemsetAsync");
    if (rc) return rc;
    rc = build_seg_tables_batched(p->orb, p->d_segsrc, p->nsrc, p->total_segs, p->d_coef, st);
    if (rc) return rc;
    BatchKernelArgs ka;
    ka.srcs = p->d_srcs;
    ka.nsrc = p->nsrc;
    ka.total_tiles = p->total_tiles;
    ka.tiles_per_item = p->tiles_per_item;
    ka.counter = p->d_counter;
    ka.gen = p->gen;
    ka.kind = p->kind;
    ka.channels = p->channels;
    ka.Lc = p->orbit.L_m / kC;
    ka.Lcf = (float)ka.Lc;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_hybrid_kernel, kTile, 0);
    const int cps = per_sm > 0 && p->ctas_per_sm > per_sm ? per_sm : p->ctas_per_sm;
    const int64_t items = (p->total_tiles + p->tiles_per_item - 1) / p->tiles_per_item;
    int64_t grid = (int64_t)p->num_sms * (cps > 0 ? cps : 1);
    if (grid > items) grid = items > 0 ? items : 1;
    prof_before("batch_hybrid_mixed", st);
    batch_hybrid_kernel<<<(unsigned)grid, kTile, 0, st>>>(ka);
    prof_after(st);
    return cuda_status(cudaGetLastError(), "batch_hybrid_kernel launch");
}

static void plan_free(lisa_plan* p)
{
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    cudaFree(p->d_srcs);
    cudaFree(p->d_segsrc);
    cudaFree(p->d_coef);
    cudaFree(p->d_counter);
    delete p;
}

extern "C" {

int lisa_plan_create(lisa_plan** out, const lisa_orbit* orbit, int precision, int tdi_gen, int lfa_kind,
                     int channels, const lisa_source* sources, int nsrc)
{
    if (!out) { set_error("plan output pointer is NULL"); return LISA_EINVAL; }
    *out = nullptr;
    if (!orbit || !sources || nsrc <= 0) { set_error("need an orbit and at least one source"); return LISA_EINVAL; }
    if (precision != LISA_MIXED) { set_error("batched plans run the mixed-precision form (precision=LISA_MIXED)"); return LISA_EINVAL; }
    if (tdi_gen != LISA_TDI15 && tdi_gen != LISA_TDI20) { set_error("tdi_gen must be 15 or 20"); return LISA_EINVAL; }
    if (lfa_kind != LISA_LFA_UNEQUAL && lfa_kind != LISA_LFA_EQUAL) { set_error("lfa_kind unknown"); return LISA_EINVAL; }
    if (channels != LISA_XYZ && channels != LISA_AET) { set_error("channels unknown"); return LISA_EINVAL; }
    if (orbit->kind < 0 || orbit->kind > 2 || orbit->delay < 0 || orbit->delay > 3 || !(orbit->L_m > 0.0)) {
        set_error("invalid orbit");
        return LISA_EINVAL;
    }
    lisa_plan* p = new (std::nothrow) lisa_plan();
    if (!p) { set_error("host allocation failed"); return LISA_ENOMEM; }
    cudaGetDevice(&p->device);
    cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    p->orbit = *orbit;
    p->orb = make_orbit_dev(*orbit);
    p->gen = tdi_gen;
    p->kind = lfa_kind;
    p->channels = channels;
    p->nsrc = nsrc;
    std::vector<BatchSrc> hs(nsrc);
    std::vector<SegSource> ss(nsrc);
    int64_t segs = 0, tiles = 0, samples = 0;
    for (int k = 0; k < nsrc; ++k) {
        const lisa_source& s = sources[k];
        const lisa_grid& g = s.grid;
        if (!(g.dt >= 0.5) || !isfinite(g.t0) || g.n <= 0 || !s.hp || !s.hc || !s.out || !isfinite(s.t_hyb)) {
            set_error("source %d: need dt >= 0.5 s, n > 0, device pointers and a finite t_hyb", k);
            delete p;
            return LISA_EINVAL;
        }
        // the fused full-response tile keeps the links over its TDI window in
        // shared memory: the largest TDI delay must fit that window
        double Tmax = 1.6 * orbit->L_m / kC;
        if (orbit->delay == LISA_DELAY_LINEAR) {
            const double span = fmax(fabs(g.t0 - orbit->t_ref), fabs(g.t0 + g.n * g.dt - orbit->t_ref));
            Tmax = 0.0;
            for (int q = 0; q < 6; ++q) Tmax = fmax(Tmax, fabs(orbit->lin_T0[q]) + fabs(orbit->lin_Tdot[q]) * span);
        }
        if ((7.0 * Tmax + 1.0) / g.dt + 40.0 > (double)(kWinY - kTile)) {
            set_error("source %d: dt=%g s is too small for the on-chip TDI window of batched plans", k, g.dt);
            delete p;
            return LISA_EINVAL;
        }
        const int S = seg_samples(g.dt);
        ss[k] = SegSource{g.t0, g.dt, S, segs};
        BatchSrc& b = hs[k];
        memset(&b, 0, sizeof(b));
        b.tab = SegTable{nullptr, seg_count(g.n, S), S, g.t0, g.dt};
        b.sky = make_sky_dev(s.sky);
        b.hm = make_grid_map(g, g);
        b.hp = s.hp;
        b.hc = s.hc;
        b.out = s.out;
        b.n = g.n;
        b.t0 = g.t0;
        b.dt = g.dt;
        b.dtf = (float)g.dt;
        b.inv12dtf = (float)(1.0 / (12.0 * g.dt));
        b.c1f = b.inv12dtf;
        b.c2f = (float)(1.0 / (12.0 * g.dt * g.dt));
        const double Tw = s.T_win > 0.0 ? s.T_win : 800.0 * g.dt;
        b.sigma = s.sigma > 0.0 ? s.sigma : Tw / 40.0;
        b.t_hyb = s.t_hyb;
        // same FP64 comparisons as lisa_response_hybrid
        volatile double hi_thr = s.t_hyb + 0.5 * Tw, lo_thr = s.t_hyb - 0.5 * Tw;
        auto t_at = [&](int64_t i) { volatile double q = (double)i * g.dt; return g.t0 + q; };
        int64_t iL = (int64_t)floor((hi_thr - g.t0) / g.dt);
        iL = iL < -1 ? -1 : (iL > g.n - 1 ? g.n - 1 : iL);
        while (iL + 1 <= g.n - 1 && t_at(iL + 1) <= hi_thr) ++iL;
        while (iL >= 0 && !(t_at(iL) <= hi_thr)) --iL;
        int64_t iF = (int64_t)ceil((lo_thr - g.t0) / g.dt);
        iF = iF < 0 ? 0 : (iF > g.n ? g.n : iF);
        while (iF - 1 >= 0 && t_at(iF - 1) >= lo_thr) --iF;
        while (iF < g.n && !(t_at(iF) >= lo_thr)) ++iF;
        b.iL = iL;
        b.iF = iF;
        b.tile_begin = tiles;
        b.ntiles = (g.n + kTile - 1) / kTile;
        segs += b.tab.nseg;
        tiles += b.ntiles;
        samples += g.n;
    }
    p->total_segs = segs;
    p->total_tiles = tiles;
    p->total_samples = samples;
    int rc = LISA_OK;
    rc = cuda_status(cudaMalloc(&p->d_coef, sizeof(double) * (size_t)segs * kNQ * kNC), "cudaMalloc(table)");
    if (!rc) rc = cuda_status(cudaMalloc(&p->d_srcs, sizeof(BatchSrc) * nsrc), "cudaMalloc(sources)");
    if (!rc) rc = cuda_status(cudaMalloc(&p->d_segsrc, sizeof(SegSource) * nsrc), "cudaMalloc(segments)");
    if (!rc) rc = cuda_status(cudaMalloc(&p->d_counter, sizeof(unsigned long long)), "cudaMalloc(counter)");
    if (rc) { plan_free(p); return rc; }
    for (int k = 0; k < nsrc; ++k) hs[k].tab.coef = p->d_coef + (size_t)ss[k].seg_begin * kNQ * kNC;
    rc = cuda_status(cudaMemcpy(p->d_srcs, hs.data(), sizeof(BatchSrc) * nsrc, cudaMemcpyHostToDevice), "cudaMemcpy");
    if (!rc) rc = cuda_status(cudaMemcpy(p->d_segsrc, ss.data(), sizeof(SegSource) * nsrc, cudaMemcpyHostToDevice),
                              "cudaMemcpy");
    if (rc) { plan_free(p); return rc; }
    *out = p;
    return LISA_OK;
}

int lisa_plan_destroy(lisa_plan* plan)
{
    plan_free(plan);
    return LISA_OK;
}

int lisa_plan_execute(lisa_plan* plan, void* stream)
{
    if (!plan) { set_error("plan is NULL"); return LISA_EINVAL; }
    return plan_enqueue(plan, (cudaStream_t)stream);
}

int lisa_plan_capture_graph(lisa_plan* plan, void* stream)
{
    if (!plan) { set_error("plan is NULL"); return LISA_EINVAL; }
    if (!stream) { set_error("graph capture needs a non-default stream"); return LISA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    if (plan->exec) { cudaGraphExecDestroy(plan->exec); plan->exec = nullptr; }
    if (plan->graph) { cudaGraphDestroy(plan->graph); plan->graph = nullptr; }
    int rc = cuda_status(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    if (rc) return rc;
    const int rc_enq = plan_enqueue(plan, st);
    cudaGraph_t g = nullptr;
    rc = cuda_status(cudaStreamEndCapture(st, &g), "cudaStreamEndCapture");
    if (rc_enq) { if (g) cudaGraphDestroy(g); return rc_enq; }
    if (rc) return rc;
    plan->graph = g;
    return cuda_status(cudaGraphInstantiate(&plan->exec, g, 0), "cudaGraphInstantiate");
}

int lisa_plan_replay(lisa_plan* plan, void* stream)
{
    if (!plan || !plan->exec) { set_error("plan has no captured graph"); return LISA_EINVAL; }
    return cuda_status(cudaGraphLaunch(plan->exec, (cudaStream_t)stream), "cudaGraphLaunch");
}

int lisa_plan_set_launch(lisa_plan* plan, int ctas_per_sm, int tiles_per_item)
{
    if (!plan || ctas_per_sm < 1 || ctas_per_sm > 8 || tiles_per_item < 1 || tiles_per_item > 64) {
        set_error("ctas_per_sm must be 1..8 and tiles_per_item 1..64");
        return LISA_EINVAL;
    }
    plan->ctas_per_sm = ctas_per_sm;
    plan->tiles_per_item = tiles_per_item;
    if (plan->exec) { cudaGraphExecDestroy(plan->exec); plan->exec = nullptr; }
    if (plan->graph) { cudaGraphDestroy(plan->graph); plan->graph = nullptr; }
    return LISA_OK;
}

int lisa_plan_info(const lisa_plan* plan, int64_t* total_samples, int64_t* total_tiles, int* ctas_per_sm,
                   int* tiles_per_item)
{
    if (!plan) { set_error("plan is NULL"); return LISA_EINVAL; }
    if (total_samples) *total_samples = plan->total_samples;
    if (total_tiles) *total_tiles = plan->total_tiles;
    if (ctas_per_sm) *ctas_per_sm = plan->ctas_per_sm;
    if (tiles_per_item) *tiles_per_item = plan->tiles_per_item;
    return LISA_OK;
}

int lisa_plan_autotune(lisa_plan* plan, void* stream, lisa_tune_result* best)
{
    if (!plan) { set_error("plan is NULL"); return LISA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    const int cps_opts[] = {1, 2, 3, 4};
    const int tpi_opts[] = {1, 2, 4, 8};
    float best_ms = 1e30f;
    int best_cps = plan->ctas_per_sm, best_tpi = plan->tiles_per_item;
    cudaEvent_t a, b;
    int rc = cuda_status(cudaEventCreate(&a), "cudaEventCreate");
    if (rc) return rc;
    rc = cuda_status(cudaEventCreate(&b), "cudaEventCreate");
    if (rc) { cudaEventDestroy(a); return rc; }
    for (int cps : cps_opts) {
        for (int tpi : tpi_opts) {
            plan->ctas_per_sm = cps;
            plan->tiles_per_item = tpi;
            rc = plan_enqueue(plan, st);     // warm-up
            if (rc) break;
            float tot = 0.f;
            for (int rep = 0; rep < 3 && !rc; ++rep) {
                cudaEventRecord(a, st);
                rc = plan_enqueue(plan, st);
                cudaEventRecord(b, st);
                rc = rc ? rc : cuda_status(cudaEventSynchronize(b), "cudaEventSynchronize");
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, b);
                tot += ms;
            }
            if (rc) break;
            if (tot / 3.f < best_ms) {
                best_ms = tot / 3.f;
                best_cps = cps;
                best_tpi = tpi;
            }
        }
        if (rc) break;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    lisa_plan_set_launch(plan, best_cps, best_tpi);
    if (rc) return rc;
    if (best) {
        best->ctas_per_sm = best_cps;
        best->tiles_per_item = best_tpi;
        best->ms = best_ms;
    }
    return LISA_OK;
}

}  // extern "C"
