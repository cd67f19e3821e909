// C ABI of liblisa: argument validation, scratch management and the
// orchestration of the kernels for each call declared in include/lisa.h.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "lisa_common.cuh"
#include "lisa_internal.cuh"

namespace lisa {

// ---------------------------------------------------------------------------
// scratch from the device's stream-ordered pool
// ---------------------------------------------------------------------------
static std::once_flag g_pool_once[64];

static void keep_pool_memory()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::call_once(g_pool_once[dev], [dev]() {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;  // keep freed blocks in the pool between calls
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    });
}

Scratch::Scratch(cudaStream_t st) : st_(st) { keep_pool_memory(); }

Scratch::~Scratch()
{
    for (int k = 0; k < n_; ++k) cudaFreeAsync(ptrs_[k], st_);
}

void* Scratch::alloc(size_t bytes)
{
    if (n_ >= 16) {
        rc_ = LISA_ENOMEM;
        set_error("too many scratch buffers");
        return nullptr;
    }
    void* p = nullptr;
    cudaError_t e = cudaMallocAsync(&p, bytes < 256 ? 256 : bytes, st_);
    if (e != cudaSuccess) {
        rc_ = cuda_status(e, "cudaMallocAsync");
        return nullptr;
    }
    ptrs_[n_++] = p;
    return p;
}

// ---------------------------------------------------------------------------
// validation
// ---------------------------------------------------------------------------
int check_grid(const lisa_grid& g, const char* name)
{
    if (!(g.dt > 0.0) || !isfinite(g.dt) || !isfinite(g.t0) || g.n < 0) {
        set_error("%s: need dt > 0, finite t0 and n >= 0 (t0=%g dt=%g n=%lld)", name, g.t0, g.dt, (long long)g.n);
        return LISA_EINVAL;
    }
    if (g.n > ((int64_t)1 << 40)) {
        set_error("%s: n=%lld too large", name, (long long)g.n);
        return LISA_EINVAL;
    }
    return LISA_OK;
}

int check_orbit(const lisa_orbit* o)
{
    if (!o) { set_error("orbit is NULL"); return LISA_EINVAL; }
    if (o->kind < LISA_ORB_KEPLER1 || o->kind > LISA_ORB_STATIC) { set_error("orbit kind %d unknown", o->kind); return LISA_EINVAL; }
    if (o->delay < LISA_DELAY_LIGHTTIME || o->delay > LISA_DELAY_LINEAR) { set_error("delay model %d unknown", o->delay); return LISA_EINVAL; }
    if (!(o->L_m > 0.0) || !isfinite(o->L_m)) { set_error("L_m must be positive"); return LISA_EINVAL; }
    if (o->kind == LISA_ORB_KEPLER2) {
        const double si = sqrt(3.0) * o->L_m / (2.0 * sqrt(3.0) * kAU) * o->kepler_tilt;
        if (!(si > -1.0 && si < 1.0)) { set_error("kepler_tilt gives |sin(inclination)| >= 1"); return LISA_EINVAL; }
    }
    return LISA_OK;
}

int check_common(int precision, int gen, int channels)
{
    if (precision != LISA_F64 && precision != LISA_MIXED && precision != LISA_DF) {
        set_error("precision %d unknown", precision);
        return LISA_EINVAL;
    }
    if (gen != LISA_TDI15 && gen != LISA_TDI20) { set_error("tdi_gen must be 15 or 20 (got %d)", gen); return LISA_EINVAL; }
    if (channels != LISA_XYZ && channels != LISA_AET) { set_error("channels %d unknown", channels); return LISA_EINVAL; }
    return LISA_OK;
}

size_t real_size(int precision) { return precision == LISA_MIXED ? sizeof(float) : sizeof(double); }

// Orbit polynomial table on grid g, in scratch.
int make_table(const lisa_orbit* orbit, const lisa_grid& g, Scratch& sc, SegTable& tab, cudaStream_t st)
{
    const int S = seg_samples(g.dt);
    const int64_t nseg = seg_count(g.n > 0 ? g.n : 1, S);
    double* coef = (double*)sc.alloc(sizeof(double) * (size_t)nseg * kNQ * kNC);
    if (!coef) return sc.status();
    LISA_TRY(build_seg_table(make_orbit_dev(*orbit), g, S, coef, nseg, st));
    tab = SegTable{coef, nseg, S, g.t0, g.dt};
    return LISA_OK;
}

// The tables of two grids (one launch).
int make_table_pair(const lisa_orbit* orbit, const lisa_grid& g1, const lisa_grid& g2, Scratch& sc, SegTable& tab1,
                    SegTable& tab2, cudaStream_t st)
{
    const int S1 = seg_samples(g1.dt), S2 = seg_samples(g2.dt);
    const int64_t n1 = seg_count(g1.n > 0 ? g1.n : 1, S1), n2 = seg_count(g2.n > 0 ? g2.n : 1, S2);
    double* c1 = (double*)sc.alloc(sizeof(double) * (size_t)(n1 + n2) * kNQ * kNC);
    if (!c1) return sc.status();
    double* c2 = c1 + (size_t)n1 * kNQ * kNC;
    LISA_TRY(build_seg_table_pair(make_orbit_dev(*orbit), g1, S1, c1, n1, g2, S2, c2, n2, st));
    tab1 = SegTable{c1, n1, S1, g1.t0, g1.dt};
    tab2 = SegTable{c2, n2, S2, g2.t0, g2.dt};
    return LISA_OK;
}

// Upper bound of any single light time (for halo sizing).
double max_light_time(const lisa_orbit* o, const lisa_grid& g)
{
    if (o->delay == LISA_DELAY_LINEAR) {
        const double span = fmax(fabs(g.t0 - o->t_ref), fabs(g.t0 + g.n * g.dt - o->t_ref)) + 1e3;
        double m = 0.0;
        for (int q = 0; q < 6; ++q) m = fmax(m, fabs(o->lin_T0[q]) + fabs(o->lin_Tdot[q]) * span);
        return m;
    }
    double flex = 1.0 + 3.0 * fmax(fabs(o->kepler_tilt - 1.0), 0.0) * 60.0 + 0.05 * fabs(o->flex_scale);
    return 1.5 * flex * o->L_m / kC;
}

// First sample of the full links a hybrid needs: the earliest sample that the
// TDI delays of the full part [iF, n) can reach (8 light times and a margin).
int64_t hybrid_links_begin(const lisa_orbit* orbit, const lisa_grid& out, int64_t iF)
{
    const double Dmax = 8.0 * max_light_time(orbit, out);
    const int64_t lo = iF - (int64_t)ceil(Dmax / out.dt) - 40;
    return lo < 0 ? 0 : lo;
}

// LFA samples: t_i <= t_hyb + Tw/2 -> [0, iL]; full samples: t_i >= t_hyb - Tw/2
// -> [iF, n) (the same FP64 comparisons as the definition).
void hybrid_split(const lisa_grid& out, double t_hyb, double Tw, int64_t& iL_out, int64_t& iF_out)
{
    const int64_t n = out.n;
    volatile double hi_thr = t_hyb + 0.5 * Tw, lo_thr = t_hyb - 0.5 * Tw;
    auto t_at = [&](int64_t i) { volatile double p = (double)i * out.dt; return out.t0 + p; };
    // clamped in FP64 before the conversions (a far switch time stays defined)
    const double lim = (double)n + 2.0;
    double fl = floor((hi_thr - out.t0) / out.dt);
    fl = fl < -2.0 ? -2.0 : (fl > lim ? lim : fl);
    int64_t iL = (int64_t)fl;
    iL = iL < -1 ? -1 : (iL > n - 1 ? n - 1 : iL);
    while (iL + 1 <= n - 1 && t_at(iL + 1) <= hi_thr) ++iL;
    while (iL >= 0 && !(t_at(iL) <= hi_thr)) --iL;
    double cl = ceil((lo_thr - out.t0) / out.dt);
    cl = cl < -1.0 ? -1.0 : (cl > lim ? lim : cl);
    int64_t iF = (int64_t)cl;
    iF = iF < 0 ? 0 : (iF > n ? n : iF);
    while (iF - 1 >= 0 && t_at(iF - 1) >= lo_thr) --iF;
    while (iF < n && !(t_at(iF) >= lo_thr)) ++iF;
    iL_out = iL;
    iF_out = iF;
}

}  // namespace lisa

using namespace lisa;

// ---------------------------------------------------------------------------
// side stream of the hybrid call
// ---------------------------------------------------------------------------
// The full-response links of a hybrid call depend only on the orbit table and
// h, not on the LFA part: they run on a second stream beside the LFA kernel,
// whose last wave leaves SMs idle, and the TDI waits for them (here and in the
// corrected hybrid).  A set (stream,
// fork and join events) serves one call at a time and is reused by later
// calls on the same device; it is released once the caller's stream has been
// told to wait for the join (a wait takes the event's state when it is
// queued, so a later call may re-record it).
namespace lisa {

static std::mutex g_side_mu;
static std::vector<SideRes*> g_side;

SideRes* side_acquire()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    {
        std::lock_guard<std::mutex> lk(g_side_mu);
        for (SideRes* r : g_side)
            if (!r->busy && r->device == dev) {
                r->busy = true;
                return r;
            }
    }
    SideRes* r = new SideRes;
    r->device = dev;
    bool ok = cudaStreamCreateWithFlags(&r->s, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&r->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&r->join, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        if (r->fork) cudaEventDestroy(r->fork);
        if (r->join) cudaEventDestroy(r->join);
        if (r->s) cudaStreamDestroy(r->s);
        delete r;
        cudaGetLastError();   // the caller falls back to one stream
        return nullptr;
    }
    r->busy = true;
    std::lock_guard<std::mutex> lk(g_side_mu);
    g_side.push_back(r);
    return r;
}

void side_release(SideRes* r)
{
    std::lock_guard<std::mutex> lk(g_side_mu);
    r->busy = false;
}

}  // namespace lisa

extern "C" {

int lisa_version(void) { return 10000; }

const char* lisa_strerror(int status)
{
    switch (status) {
    case LISA_OK: return "ok";
    case LISA_EINVAL: return "invalid argument";
    case LISA_ERANGE: return "time outside the valid range";
    case LISA_ECUDA: return "CUDA error";
    case LISA_ETIMEOUT: return "bounded device wait timed out";
    case LISA_ENOMEM: return "out of device memory";
    case LISA_ECORRECTOR: return "corrector spot check failed; full-response fallback used";
    default: return "unknown status";
    }
}

const char* lisa_last_error_message(void) { return last_error(); }

double lisa_t_hyb_from_f(double f_hyb, double mc_s, double tc)
{
    return tc - pow(f_hyb, -8.0 / 3.0) * 5.0 / pow(8.0 * kPi, 8.0 / 3.0) * pow(mc_s, -5.0 / 3.0);
}

int lisa_orbits(const lisa_orbit* orbit, lisa_grid g, double* R, double* T, double* nhat, void* stream)
{
    LISA_TRY(check_orbit(orbit));
    LISA_TRY(check_grid(g, "grid"));
    if (g.n == 0) return LISA_OK;
    return run_orbits(orbit, g, R, T, nhat, (cudaStream_t)stream);
}

int lisa_links_full(const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid h_grid, const void* hp, const void* hc,
                    int precision, lisa_grid y_grid, void* y, void* stream)
{
    LISA_TRY(check_orbit(orbit));
    LISA_TRY(check_grid(h_grid, "h_grid"));
    LISA_TRY(check_grid(y_grid, "y_grid"));
    LISA_TRY(check_common(precision, LISA_TDI15, LISA_XYZ));
    if (!sky) { set_error("sky is NULL"); return LISA_EINVAL; }
    if (y_grid.n == 0) return LISA_OK;
    if (!y || (h_grid.n > 0 && (!hp || !hc))) { set_error("NULL series pointer"); return LISA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc(st);
    SegTable tab;
    LISA_TRY(make_table(orbit, y_grid, sc, tab, st));
    return launch_links_full(tab, make_sky_dev(*sky), h_grid, hp, hc, precision, y_grid, y, 0, y_grid.n, st);
}

int lisa_tdi(const lisa_orbit* orbit, lisa_grid y_grid, const void* y, int precision, int tdi_gen, int delay_mode,
             int channels, lisa_grid out, void* xyz, void* stream)
{
    LISA_TRY(check_orbit(orbit));
    LISA_TRY(check_grid(y_grid, "y_grid"));
    LISA_TRY(check_grid(out, "out"));
    LISA_TRY(check_common(precision, tdi_gen, channels));
    if (delay_mode != LISA_FROZEN && delay_mode != LISA_NESTED) { set_error("delay_mode %d unknown", delay_mode); return LISA_EINVAL; }
    if (out.n == 0) return LISA_OK;
    if (!xyz || (y_grid.n > 0 && !y)) { set_error("NULL series pointer"); return LISA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc(st);
    SegTable tab;
    LISA_TRY(make_table(orbit, out, sc, tab, st));
    BlendSpec bl{};
    return launch_tdi(tab, y_grid, y, precision, tdi_gen, delay_mode, channels, out, xyz, 0, out.n, bl, st);
}

int lisa_response_full(const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid h_grid, const void* hp, const void* hc,
                       int precision, int tdi_gen, int channels, lisa_grid out, void* xyz, void* stream)
{
    LISA_TRY(check_orbit(orbit));
    LISA_TRY(check_grid(h_grid, "h_grid"));
    LISA_TRY(check_grid(out, "out"));
    LISA_TRY(check_common(precision, tdi_gen, channels));
    if (!sky) { set_error("sky is NULL"); return LISA_EINVAL; }
    if (out.n == 0) return LISA_OK;
    if (!xyz || (h_grid.n > 0 && (!hp || !hc))) { set_error("NULL series pointer"); return LISA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc(st);
    SegTable tab;
    LISA_TRY(make_table(orbit, out, sc, tab, st));
    void* y = sc.alloc(6 * (size_t)out.n * real_size(precision));
    if (!y) return sc.status();
    LISA_TRY(launch_links_full(tab, make_sky_dev(*sky), h_grid, hp, hc, precision, out, y, 0, out.n, st));
    BlendSpec bl{};
    return launch_tdi(tab, out, y, precision, tdi_gen, LISA_FROZEN, channels, out, xyz, 0, out.n, bl, st);
}

int lisa_links_lfa(const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid h_grid, const void* hp, const void* hc,
                   int precision, int tdi_gen, int lfa_kind, lisa_grid out, void* z, void* stream)
{
    LISA_TRY(check_orbit(orbit));
    LISA_TRY(check_grid(h_grid, "h_grid"));
    LISA_TRY(check_grid(out, "out"));
    LISA_TRY(check_common(precision, tdi_gen, LISA_XYZ));
    if (!lfa_kind_series_ok(lfa_kind)) { set_error("lfa_kind %d unknown or without link series", lfa_kind); return LISA_EINVAL; }
    if (!sky) { set_error("sky is NULL"); return LISA_EINVAL; }
    if (out.n == 0) return LISA_OK;
    if (!z || (h_grid.n > 0 && (!hp || !hc))) { set_error("NULL series pointer"); return LISA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc(st);
    SegTable tab;
    LISA_TRY(make_table(orbit, out, sc, tab, st));
    BlendSpec bl{};
    return launch_lfa(tab, make_sky_dev(*sky), orbit->L_m, h_grid, hp, hc, precision, tdi_gen, lfa_kind, LISA_XYZ, out,
                      z, nullptr, 0, out.n, bl, st);
}

int lisa_links_lfa_own(const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid h_grid, const void* hp, const void* hc,
                       int precision, int lfa_kind, lisa_grid out, void* y, void* stream)
{
    LISA_TRY(check_orbit(orbit));
    LISA_TRY(check_grid(h_grid, "h_grid"));
    LISA_TRY(check_grid(out, "out"));
    LISA_TRY(check_common(precision, LISA_TDI15, LISA_XYZ));
    if (!lfa_kind_series_ok(lfa_kind)) { set_error("lfa_kind %d unknown or without link series", lfa_kind); return LISA_EINVAL; }
    if (!sky) { set_error("sky is NULL"); return LISA_EINVAL; }
    if (out.n == 0) return LISA_OK;
    if (!y || (h_grid.n > 0 && (!hp || !hc))) { set_error("NULL series pointer"); return LISA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc(st);
    SegTable tab;
    LISA_TRY(make_table(orbit, out, sc, tab, st));
    BlendSpec bl{};
    return launch_lfa(tab, make_sky_dev(*sky), orbit->L_m, h_grid, hp, hc, precision, kLfaOwnTime, lfa_kind, LISA_XYZ,
                      out, y, nullptr, 0, out.n, bl, st);
}

int lisa_tdi_lfa(const lisa_orbit* orbit, lisa_grid z_grid, const void* z, int precision, int tdi_gen, int lfa_kind,
                 int channels, void* xyz, void* stream)
{
    LISA_TRY(check_orbit(orbit));
    LISA_TRY(check_grid(z_grid, "z_grid"));
    LISA_TRY(check_common(precision, tdi_gen, channels));
    if (!lfa_kind_series_ok(lfa_kind)) { set_error("lfa_kind %d unknown or without link series", lfa_kind); return LISA_EINVAL; }
    if (z_grid.n == 0) return LISA_OK;
    if (!z || !xyz) { set_error("NULL series pointer"); return LISA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc(st);
    SegTable tab;
    LISA_TRY(make_table(orbit, z_grid, sc, tab, st));
    return launch_tdi_lfa(tab, orbit->L_m, z_grid, z, precision, tdi_gen, lfa_kind, channels, xyz, st);
}

int lisa_response_lfa(const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid h_grid, const void* hp, const void* hc,
                      int precision, int tdi_gen, int lfa_kind, int channels, lisa_grid out, void* xyz, void* stream)
{
    LISA_TRY(check_orbit(orbit));
    LISA_TRY(check_grid(h_grid, "h_grid"));
    LISA_TRY(check_grid(out, "out"));
    LISA_TRY(check_common(precision, tdi_gen, channels));
    if (!lfa_kind_ok(lfa_kind)) { set_error("lfa_kind %d unknown", lfa_kind); return LISA_EINVAL; }
    if (!sky) { set_error("sky is NULL"); return LISA_EINVAL; }
    if (out.n == 0) return LISA_OK;
    if (!xyz || (h_grid.n > 0 && (!hp || !hc))) { set_error("NULL series pointer"); return LISA_EINVAL; }
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc(st);
    SegTable tab;
    LISA_TRY(make_table(orbit, out, sc, tab, st));
    BlendSpec bl{};
    return launch_lfa(tab, make_sky_dev(*sky), orbit->L_m, h_grid, hp, hc, precision, tdi_gen, lfa_kind, channels, out,
                      nullptr, xyz, 0, out.n, bl, st);
}

int lisa_response_hybrid(const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid h_grid, const void* hp, const void* hc,
                         int precision, int tdi_gen, int lfa_kind, int channels, double t_hyb, double T_win,
                         double sigma, lisa_grid out, void* xyz, void* stream)
{
    LISA_TRY(check_orbit(orbit));
    LISA_TRY(check_grid(h_grid, "h_grid"));
    LISA_TRY(check_grid(out, "out"));
    LISA_TRY(check_common(precision, tdi_gen, channels));
    if (!lfa_kind_ok(lfa_kind)) { set_error("lfa_kind %d unknown", lfa_kind); return LISA_EINVAL; }
    if (!sky) { set_error("sky is NULL"); return LISA_EINVAL; }
    if (!isfinite(t_hyb)) { set_error("t_hyb must be finite"); return LISA_EINVAL; }
    if (out.n == 0) return LISA_OK;
    if (!xyz || (h_grid.n > 0 && (!hp || !hc))) { set_error("NULL series pointer"); return LISA_EINVAL; }
    const double Tw = T_win > 0.0 ? T_win : 800.0 * out.dt;
    const double sg = sigma > 0.0 ? sigma : Tw / 40.0;
    const int64_t n = out.n;
    int64_t iL, iF;
    hybrid_split(out, t_hyb, Tw, iL, iF);

    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc(st);
    SegTable tab;
    LISA_TRY(make_table(orbit, out, sc, tab, st));
    const SkyDev skyd = make_sky_dev(*sky);
    const size_t rs = real_size(precision);
    // samples covered by neither part are zero
    if (iF > iL + 1) {
        for (int c = 0; c < 3; ++c) {
            LISA_TRY(cuda_status(cudaMemsetAsync((char*)xyz + ((size_t)c * n + (size_t)(iL + 1)) * rs, 0,
                                                 (size_t)(iF - iL - 1) * rs, st), "cudaMemsetAsync"));
        }
    }
    void* y = nullptr;
    int64_t lo = 0;
    if (iF < n) {
        lo = hybrid_links_begin(orbit, out, iF);
        // the links are held for samples [lo, n) only
        y = sc.alloc(6 * (size_t)(n - lo) * rs);
        if (!y) return sc.status();
    }
    // both parts: the links go on the side stream, forked after the table and
    // the link buffer are ready on the caller's stream; the caller's stream
    // joins it after the LFA launch (also after an error, so that nothing
    // queued there outlives the call's scratch)
    SideGuard side{(iL >= 0 && iF < n) ? side_acquire() : nullptr};
    int rc_links = 0, rc_join = 0;
    if (side.r) {
        LISA_TRY(cuda_status(cudaEventRecord(side.r->fork, st), "cudaEventRecord"));
        LISA_TRY(cuda_status(cudaStreamWaitEvent(side.r->s, side.r->fork, 0), "cudaStreamWaitEvent"));
        rc_links = launch_links_full(tab, skyd, h_grid, hp, hc, precision, out, y, lo, n, side.r->s, lo);
        rc_join = cuda_status(cudaEventRecord(side.r->join, side.r->s), "cudaEventRecord");
    }
    int rc_lfa = 0;
    if (iL >= 0 && !rc_links && !rc_join) {
        BlendSpec bl{1, t_hyb, sg, +1.0, 0, 0};
        rc_lfa = launch_lfa(tab, skyd, orbit->L_m, h_grid, hp, hc, precision, tdi_gen, lfa_kind, channels, out, nullptr,
                            xyz, 0, iL + 1, bl, st);
    }
    if (side.r && !rc_join) rc_join = cuda_status(cudaStreamWaitEvent(st, side.r->join, 0), "cudaStreamWaitEvent");
    if (rc_links) return rc_links;
    if (rc_join) return rc_join;
    if (rc_lfa) return rc_lfa;
    if (iF < n) {
        if (!side.r) LISA_TRY(launch_links_full(tab, skyd, h_grid, hp, hc, precision, out, y, lo, n, st, lo));
        BlendSpec bl{1, t_hyb, sg, -1.0, iF, iL + 1};
        LISA_TRY(launch_tdi(tab, out, y, precision, tdi_gen, LISA_FROZEN, channels, out, xyz, iF, n, bl, st, lo));
    }
    return LISA_OK;
}

}  // extern "C"
