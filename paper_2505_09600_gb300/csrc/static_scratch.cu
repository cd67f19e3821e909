// lisa_response_hybrid_static: the hybrid response with its scratch memory
// taken from a fixed, file-scope device array instead of being allocated.
//
// Who needs it: callers that may not allocate device memory while they run --
// for example an application that hands all device memory to its own pool at
// start-up and forbids later driver allocations, a latency-bound loop that
// must not wait on an allocator, or a platform where the stream-ordered
// allocator (cudaMallocAsync) is unavailable.  They pass inputs and outputs as
// usual; the orbit tables and link series live in g_static_scratch.
//
// The array is LISA_STATIC_SCRATCH_BYTES long and is resident on every GPU
// that loads the library, until the process exits.  Every call on a device
// shares it and leaves the last call's contents behind: calls that overlap on
// the GPU (different streams, or different host threads) race on it and must
// be serialised by the caller.  Nothing in it needs to start at zero: each
// call writes every table coefficient and link sample before it reads them.
// The scratch holds what lisa_response_hybrid allocates (the orbit table on
// the output grid and the full links of the samples the TDI part reaches), in
// the same layout, so the two calls give the same bits.
#include <math.h>
#include <string.h>

#include <mutex>

#include "lisa_common.cuh"
#include "lisa_internal.cuh"

namespace lisa {

static __device__ __align__(256) unsigned char g_static_scratch[LISA_STATIC_SCRATCH_BYTES];

// Device address of g_static_scratch on the current device.  In host code the
// symbol is only a host-side stand-in, so the address is looked up once per
// device, with that device current, and cached.
static int static_scratch_address(void** out)
{
    static std::mutex mu;
    static void* addr[64] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) {
        set_error("device %d out of range for the static scratch", dev);
        return LISA_EINVAL;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(g_static_scratch)");
        addr[dev] = p;
    }
    *out = addr[dev];
    return LISA_OK;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace lisa

using namespace lisa;

extern "C" int lisa_response_hybrid_static(const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid h_grid,
                                           const void* hp, const void* hc, int precision, int tdi_gen, int lfa_kind,
                                           int channels, double t_hyb, double T_win, double sigma, lisa_grid out,
                                           void* xyz, void* stream)
{
    // same argument checks as lisa_response_hybrid
    if (!orbit || !sky) { set_error("orbit or sky is NULL"); return LISA_EINVAL; }
    if (orbit->kind < LISA_ORB_KEPLER1 || orbit->kind > LISA_ORB_STATIC || orbit->delay < LISA_DELAY_LIGHTTIME ||
        orbit->delay > LISA_DELAY_LINEAR || !(orbit->L_m > 0.0) || !isfinite(orbit->L_m)) {
        set_error("invalid orbit");
        return LISA_EINVAL;
    }
    for (const lisa_grid* g : {&h_grid, &out}) {
        if (!(g->dt > 0.0) || !isfinite(g->dt) || !isfinite(g->t0) || g->n < 0) {
            set_error("grids need dt > 0, finite t0 and n >= 0");
            return LISA_EINVAL;
        }
    }
    if (precision != LISA_F64 && precision != LISA_MIXED && precision != LISA_DF) {
        set_error("precision unknown");
        return LISA_EINVAL;
    }
    if (tdi_gen != LISA_TDI15 && tdi_gen != LISA_TDI20) { set_error("tdi_gen must be 15 or 20"); return LISA_EINVAL; }
    if (!lfa_kind_ok(lfa_kind)) { set_error("lfa_kind unknown"); return LISA_EINVAL; }
    if (channels != LISA_XYZ && channels != LISA_AET) { set_error("channels unknown"); return LISA_EINVAL; }
    if (!isfinite(t_hyb)) { set_error("t_hyb must be finite"); return LISA_EINVAL; }
    if (out.n == 0) return LISA_OK;
    if (!xyz || (h_grid.n > 0 && (!hp || !hc))) { set_error("NULL series pointer"); return LISA_EINVAL; }

    const double Tw = T_win > 0.0 ? T_win : 800.0 * out.dt;
    const double sg = sigma > 0.0 ? sigma : Tw / 40.0;
    const int64_t n = out.n;
    int64_t iL, iF;
    hybrid_split(out, t_hyb, Tw, iL, iF);

    // scratch layout: [orbit table on `out`] [links of samples [lo, n)], the
    // same table and link range as lisa_response_hybrid, so the two calls
    // launch the same kernels on the same values
    const size_t rs = precision == LISA_MIXED ? sizeof(float) : sizeof(double);
    const int S = seg_samples(out.dt);
    const int64_t nseg = seg_count(n, S);
    const int64_t lo = iF < n ? hybrid_links_begin(orbit, out, iF) : n;
    const size_t b_tab = align256(sizeof(double) * (size_t)nseg * kNQ * kNC);
    const size_t b_y = align256(6 * (size_t)(n - lo) * rs);
    const size_t need = b_tab + b_y;
    if (need > (size_t)LISA_STATIC_SCRATCH_BYTES) {
        set_error("lisa_response_hybrid_static needs %zu bytes of scratch for this call; the static scratch holds "
                  "%zu bytes (LISA_STATIC_SCRATCH_BYTES): use lisa_response_hybrid or a shorter grid",
                  need, (size_t)LISA_STATIC_SCRATCH_BYTES);
        return LISA_EINVAL;
    }
    void* base = nullptr;
    int rc = static_scratch_address(&base);
    if (rc) return rc;
    double* coef = (double*)base;
    void* y = (char*)base + b_tab;

    cudaStream_t st = (cudaStream_t)stream;
    rc = build_seg_table(make_orbit_dev(*orbit), out, S, coef, nseg, st);
    if (rc) return rc;
    const SegTable tab{coef, nseg, S, out.t0, out.dt};
    const SkyDev skyd = make_sky_dev(*sky);
    if (iF > iL + 1) {
        for (int c = 0; c < 3; ++c) {
            rc = cuda_status(cudaMemsetAsync((char*)xyz + ((size_t)c * n + (size_t)(iL + 1)) * rs, 0,
                                             (size_t)(iF - iL - 1) * rs, st), "cudaMemsetAsync");
            if (rc) return rc;
        }
    }
    if (iL >= 0) {
        BlendSpec bl{1, t_hyb, sg, +1.0, 0, 0};
        rc = launch_lfa(tab, skyd, orbit->L_m, h_grid, hp, hc, precision, tdi_gen, lfa_kind, channels, out, nullptr,
                        xyz, 0, iL + 1, bl, st);
        if (rc) return rc;
    }
    if (iF < n) {
        rc = launch_links_full(tab, skyd, h_grid, hp, hc, precision, out, y, lo, n, st, lo);
        if (rc) return rc;
        BlendSpec bl{1, t_hyb, sg, -1.0, iF, iL + 1};
        rc = launch_tdi(tab, out, y, precision, tdi_gen, LISA_FROZEN, channels, out, xyz, iF, n, bl, st, lo);
        if (rc) return rc;
    }
    return LISA_OK;
}
