// Batched hybrid response: many sources of uneven duration in one persistent
// launch (mixed precision).
//
// A plan owns, in device memory allocated once at creation:
//   - one orbit polynomial table holding the segments of every source's grid
//     (built by one batched kernel per execution),
//   - a descriptor per source with the prefix of its work items,
//   - a work counter and, per CTA of the persistent kernel, a link scratch.
// A source's tiles form groups of up to 8 consecutive tiles from its start
// (the grouping of lisa_response_lfa, fixed so that the results do not
// depend on the launch shape); a work item is a run of groups of one source.
// Each block takes the next item with one atomicAdd and runs the same code as
// the single-source calls on each group:
//   - the LFA channels of its samples with t <= t_hyb + T/2 (the grouped LFA
//     of lisa_response_lfa: one FP64 prologue, sub-blocks of two tiles, bulk
//     copies of the h windows), weighted by S(+1);
//   - the six links over the samples the TDI delays of its full-response part
//     reach (t >= t_hyb - T/2), into the block's scratch (L2-resident), then
//     the TDI combination on per-link combined filters (as lisa_tdi), weighted
//     by S(-1) and added where both parts contribute (Eq. hybridized_xs).
// Blocks never wait on each other (no spin, no grid barrier), so uneven
// sources are balanced by the queue alone.  The whole execution (counter
// reset, tables, persistent kernel) can be captured in a CUDA graph.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "lfa_tile.cuh"
#include "links_group.cuh"
#include "tdi_comb.cuh"

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
    int64_t lo_links;    // first sample whose links the full part may read
    int dm_links;        // samples the TDI delays reach back (plus margin)
    int G;               // tiles per group (fixed: the results do not depend on the launch shape)
    int gpi;             // groups per work item
    int h_aligned;       // hp, hc on 16-byte boundaries (bulk copies)
    int64_t ntiles, ngroups;
    int64_t item_begin;  // first work item of this source
};

struct BatchKernelArgs {
    const BatchSrc* srcs;
    int nsrc;
    int64_t total_items;
    unsigned long long* counter;
    float* scratch;      // per CTA: six link rows of scr_len samples
    int scr_len;
    int gen, kind, channels;
    double Lc;
    float Lcf;
    unsigned int* status;
};

// The three parts of an item use the block's shared memory one after the
// other.
union BatchShared {
    Lfa2Smem lfa;
    CombSmem tdi;
    LinksGroupSmem lg;
};

#ifndef LISA_BATCH_MINB
#define LISA_BATCH_MINB 3   // resident CTAs per SM the register budget is set for (85 registers)
#endif
__global__ void __launch_bounds__(kTile, LISA_BATCH_MINB) batch_hybrid_kernel(BatchKernelArgs ka)
{
    __shared__ BatchShared u;
    __shared__ int64_t s_item;
    __shared__ int s_src;
    const int t = threadIdx.x;
    float* scr = ka.scratch + (size_t)blockIdx.x * 6 * (size_t)ka.scr_len;
    for (;;) {
        __syncthreads();   // the previous item is done with shared memory and the scratch
        if (t == 0) {
            const int64_t item = (int64_t)atomicAdd(ka.counter, 1ull);
            int lo = 0, hi = ka.nsrc - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (ka.srcs[mid].item_begin <= item) lo = mid; else hi = mid - 1;
            }
            s_item = item;
            s_src = lo;
        }
        __syncthreads();
        const int64_t item = s_item;
        if (item >= ka.total_items) break;
        const BatchSrc& b = ka.srcs[s_src];
        const int64_t g0 = (item - b.item_begin) * b.gpi;
        const int64_t g1 = g0 + b.gpi < b.ngroups ? g0 + b.gpi : b.ngroups;
        for (int64_t grp = g0; grp < g1; ++grp) {
        if (grp > g0) __syncthreads();   // the previous group is done with shared memory and the scratch
        const int64_t t0 = grp * b.G;
        const int nt = (int)(b.ntiles - t0 < b.G ? b.ntiles - t0 : b.G);
        const int64_t i_lo = t0 * kTile, i_hi = (t0 + nt) * (int64_t)kTile;   // group samples [i_lo, i_hi)

        // LFA part, weight S(+1), samples [i_lo, min(i_hi, iL + 1))
        if (i_lo <= b.iL) {
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
            a.xyz = b.out;
            a.nout = b.n;
            a.t0_out = b.t0;
            a.dt_out = b.dt;
            a.i_begin = 0;
            a.i_end = b.iL + 1;
            a.tile0 = 0;
            a.bl = BlendSpec{1, b.t_hyb, b.sigma, +1.0, 0, 0};
            a.Lcf = ka.Lcf;
            a.dtf = b.dtf;
            a.inv12dtf = b.inv12dtf;
            a.c1f = b.c1f;
            a.c2f = b.c2f;
            a.h_aligned = b.h_aligned;
            a.status = ka.status;
            const int64_t last = b.iL / kTile;
            const int nl = (int)(last - t0 + 1 < nt ? last - t0 + 1 : nt);
            if (t == 0) {
                mbar_init(&u.lfa.bar[0], 1);
                mbar_init(&u.lfa.bar[1], 1);
                mbar_init_fence();
            }
            uint32_t ph0 = 0u, ph1 = 0u;
            const bool ok = lfa2_group(a, t0, nl, b.G, u.lfa, ph0, ph1);
            // every copy has landed: the barriers are invalidated before the
            // memory holds other data
            __syncthreads();
            if (t == 0) {
                mbar_inval(&u.lfa.bar[0]);
                mbar_inval(&u.lfa.bar[1]);
            }
            if (!ok) return;   // a bounded wait timed out (status word flagged)
        }
        // samples covered by neither part are zero
        if (b.iF > b.iL + 1) {
            const int64_t z0 = b.iL + 1 > i_lo ? b.iL + 1 : i_lo, z1 = b.iF < i_hi ? b.iF : i_hi;
            float* out = (float*)b.out;
            for (int64_t i = z0 + t; i < z1; i += blockDim.x) {
                out[i] = 0.f;
                out[b.n + i] = 0.f;
                out[2 * b.n + i] = 0.f;
            }
        }
        // full part, weight S(-1), samples [max(i_lo, iF), i_hi)
        const int64_t tf0 = b.iF / kTile > t0 ? b.iF / kTile : t0;
        if (b.iF < b.n && tf0 < t0 + nt) {
            const int nf = (int)(t0 + nt - tf0);
            int64_t ys = tf0 * kTile - b.dm_links;
            ys = ys > b.lo_links ? ys : b.lo_links;
            int64_t ye = i_hi + 40;
            ye = ye < b.n ? ye : b.n;
            LinksArgs la;
            la.tab = b.tab;
            la.sky = b.sky;
            la.hm = b.hm;
            la.hp = b.hp;
            la.hc = b.hc;
            la.y = scr;
            la.y0 = ys;
            la.ny = ka.scr_len;
            la.i_begin = ys;
            la.i_end = ye;
            la.tile0 = 0;
            // the links of [ys, ye) into the scratch, in groups of the source's G
            // tiles around one FP64 set-up each (as the links kernel)
            __syncthreads();   // the LFA part is done with the shared memory
            const int64_t tl0 = ys / kTile, tl1 = (ye - 1) / kTile;
            for (int64_t tg = tl0; tg <= tl1; tg += b.G) {
                const int ng = (int)(tl1 - tg + 1 < b.G ? tl1 - tg + 1 : b.G);
                links_group(la, tg, ng, b.G, u.lg);   // synchronises; the scratch is visible after it
            }
            TdiArgs ta;
            ta.tab = b.tab;
            ta.ym = GridMap{1.0, -ys, 0.0, b.dt, ye - ys, 1};
            ta.y = scr;
            ta.ny = ka.scr_len;
            ta.xyz = b.out;
            ta.nout = b.n;
            ta.nterm = ka.gen == LISA_TDI20 ? 16 : 8;
            ta.mode = LISA_FROZEN;
            ta.channels = ka.channels;
            ta.i_begin = b.iF;
            ta.i_end = b.n;
            ta.tile0 = 0;
            ta.bl = BlendSpec{1, b.t_hyb, b.sigma, -1.0, b.iF, b.iL + 1};
            ta.t0_out = b.t0;
            ta.dt_out = b.dt;
            comb_group(ta, tf0, nf, nf, u.tdi);
        }
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
    std::vector<BatchSrc> hsrc;
    BatchSrc* d_srcs = nullptr;
    SegSource* d_segsrc = nullptr;
    double* d_coef = nullptr;
    unsigned long long* d_counter = nullptr;
    float* d_scratch = nullptr;
    int scr_len = 0, max_ctas = 0;
    int64_t total_segs = 0, total_tiles = 0, total_samples = 0, total_items = 0;
    int ctas_per_sm = 2, tiles_per_item = 8;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

// Work items of every source for the plan's tiles_per_item, uploaded to the
// device descriptors.
static int plan_items(lisa_plan* p)
{
    int64_t items = 0;
    for (BatchSrc& b : p->hsrc) {
        b.G = lfa_group(b.dt);
        b.ngroups = (b.ntiles + b.G - 1) / b.G;
        b.gpi = p->tiles_per_item / b.G > 1 ? p->tiles_per_item / b.G : 1;
        b.item_begin = items;
        items += (b.ngroups + b.gpi - 1) / b.gpi;
    }
    p->total_items = items;
    return cuda_status(cudaMemcpy(p->d_srcs, p->hsrc.data(), sizeof(BatchSrc) * p->hsrc.size(), cudaMemcpyHostToDevice),
                       "cudaMemcpy(sources)");
}

static int plan_enqueue(lisa_plan* p, cudaStream_t st)
{
    int rc = cuda_status(cudaMemsetAsync(p->d_counter, 0, sizeof(unsigned long long), st), "cudaMemsetAsync");
    if (rc) return rc;
    rc = build_seg_tables_batched(p->orb, p->d_segsrc, p->nsrc, p->total_segs, p->d_coef, st);
    if (rc) return rc;
    BatchKernelArgs ka;
    ka.srcs = p->d_srcs;
    ka.nsrc = p->nsrc;
    ka.total_items = p->total_items;
    ka.counter = p->d_counter;
    ka.scratch = p->d_scratch;
    ka.scr_len = p->scr_len;
    ka.gen = p->gen;
    ka.kind = p->kind;
    ka.channels = p->channels;
    ka.Lc = p->orbit.L_m / kC;
    ka.Lcf = (float)ka.Lc;
    ka.status = device_status_ptr();
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_hybrid_kernel, kTile, 0);
    const int cps = per_sm > 0 && p->ctas_per_sm > per_sm ? per_sm : p->ctas_per_sm;
    int64_t grid = (int64_t)p->num_sms * (cps > 0 ? cps : 1);
    if (grid > p->max_ctas) grid = p->max_ctas;
    if (grid > p->total_items) grid = p->total_items > 0 ? p->total_items : 1;
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
    cudaFree(p->d_scratch);
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
    if (!lfa_kind_lo(lfa_kind)) { set_error("lfa_kind unknown (batched plans take the leading-order kinds)"); return LISA_EINVAL; }
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
    int scr_len = 0;
    for (int k = 0; k < nsrc; ++k) {
        const lisa_source& s = sources[k];
        const lisa_grid& g = s.grid;
        if (!(g.dt >= 0.5) || !isfinite(g.t0) || g.n <= 0 || !s.hp || !s.hc || !s.out || !isfinite(s.t_hyb)) {
            set_error("source %d: need dt >= 0.5 s, n > 0, device pointers and a finite t_hyb", k);
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
        // links from the earliest sample the TDI delays of [iF, n) can reach
        // (as lisa_response_hybrid)
        const double Dmax = 8.0 * max_light_time(orbit, g);
        b.dm_links = (int)ceil(Dmax / g.dt) + 40;
        b.lo_links = iF - b.dm_links > 0 ? iF - b.dm_links : 0;
        b.h_aligned = ((uintptr_t)s.hp % 16 == 0) && ((uintptr_t)s.hc % 16 == 0);
        b.ntiles = (g.n + kTile - 1) / kTile;
        const int need = 8 * kTile + 40 + b.dm_links;
        scr_len = need > scr_len ? need : scr_len;
        segs += b.tab.nseg;
        tiles += b.ntiles;
        samples += g.n;
    }
    p->total_segs = segs;
    p->total_tiles = tiles;
    p->total_samples = samples;
    p->scr_len = (scr_len + 31) / 32 * 32;
    p->max_ctas = 4 * (p->num_sms > 0 ? p->num_sms : 1);
    int rc = LISA_OK;
    rc = cuda_status(cudaMalloc(&p->d_coef, sizeof(double) * (size_t)segs * kNQ * kNC), "cudaMalloc(table)");
    if (!rc) rc = cuda_status(cudaMalloc(&p->d_srcs, sizeof(BatchSrc) * nsrc), "cudaMalloc(sources)");
    if (!rc) rc = cuda_status(cudaMalloc(&p->d_segsrc, sizeof(SegSource) * nsrc), "cudaMalloc(segments)");
    if (!rc) rc = cuda_status(cudaMalloc(&p->d_counter, sizeof(unsigned long long)), "cudaMalloc(counter)");
    if (!rc)
        rc = cuda_status(cudaMalloc(&p->d_scratch, sizeof(float) * 6 * (size_t)p->scr_len * (size_t)p->max_ctas),
                         "cudaMalloc(link scratch)");
    if (rc) { plan_free(p); return rc; }
    for (int k = 0; k < nsrc; ++k) hs[k].tab.coef = p->d_coef + (size_t)ss[k].seg_begin * kNQ * kNC;
    p->hsrc = hs;
    rc = plan_items(p);
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
    return plan_items(plan);
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
    // tiles per item: 1, 2, 4 or 8 whole groups of 8 tiles (an item holds at
    // least one group, so fewer tiles than a group would change nothing)
    const int tpi_opts[] = {8, 16, 32, 64};
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
            rc = plan_items(plan);
            if (!rc) rc = plan_enqueue(plan, st);     // warm-up
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
