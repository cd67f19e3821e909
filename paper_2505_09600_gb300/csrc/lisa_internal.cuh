// Host-side internals shared by the translation units of liblisa.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lisa_common.cuh"

namespace lisa {

const char* last_error();

// Every kernel launch is bracketed by these (launch counter; optional timing).
void prof_before(const char* name, cudaStream_t st);
void prof_after(cudaStream_t st);

// Stream-ordered scratch: every allocation is released on the same stream
// (cudaFreeAsync) when the owner goes out of scope, i.e. after the kernels
// already enqueued have consumed it.
class Scratch {
public:
    explicit Scratch(cudaStream_t st);
    ~Scratch();
    void* alloc(size_t bytes);
    int status() const { return rc_; }

private:
    cudaStream_t st_;
    void* ptrs_[16];
    int n_ = 0;
    int rc_ = 0;
};

// Tile size (output samples per CTA) of the response kernels.
constexpr int kTile = 256;

// Known LFA kinds (central unequal / equal arms, non-central backward /
// forward, next-to-leading order, strain-derivative form).
inline bool lfa_kind_ok(int k)
{
    return k == LISA_LFA_UNEQUAL || k == LISA_LFA_EQUAL || k == LISA_LFA_BACKWARD || k == LISA_LFA_FORWARD ||
           k == LISA_LFA_NLO || k == LISA_LFA_STRAIN;
}
// Kinds with link / z series (all but the strain-derivative form).
inline bool lfa_kind_series_ok(int k) { return lfa_kind_ok(k) && k != LISA_LFA_STRAIN; }
// Kinds of the batched plans (leading order).
inline bool lfa_kind_lo(int k)
{
    return k == LISA_LFA_UNEQUAL || k == LISA_LFA_EQUAL || k == LISA_LFA_BACKWARD || k == LISA_LFA_FORWARD;
}

// Segment tables of many grids in one launch (batched plans).
struct SegSource {
    double t0, dt;
    int S;
    int64_t seg_begin;   // index of the first segment of this grid in the shared table
};
int build_seg_tables_batched(const OrbitDev& orb, const SegSource* srcs_dev, int nsrc, int64_t total_segs,
                             double* coef_dev, cudaStream_t st);

int run_orbits(const lisa_orbit* orbit, lisa_grid g, double* R, double* T, double* nh, cudaStream_t st);

// Full links on y-grid samples [i_begin, i_end) using a segment table built
// on the y grid.  y holds the samples [y0, yg.n) of the grid: link li, sample
// i at y[li (yg.n - y0) + i - y0] (y0 = 0: the whole grid).
int launch_links_full(const SegTable& tab, const SkyDev& sky, const lisa_grid& hg, const void* hp, const void* hc,
                      int precision, const lisa_grid& yg, void* y, int64_t i_begin, int64_t i_end, cudaStream_t st,
                      int64_t y0 = 0);

// TDI on out-grid samples [i_begin, i_end).  Hybrid support: each output is
// multiplied by the sigmoid weight S(t; t_hyb, sigma, -1) if `blend` is set,
// and the value already in xyz is added where `accumulate_until` > i.
struct BlendSpec {
    int enabled;        // 0: plain output
    double t_hyb, sigma, eps;   // weight S(t; t_hyb, sigma, eps)
    int64_t acc_begin, acc_end; // samples where the existing output is added
    int lerp;           // TDI stores only: on [acc_begin, acc_end) the output
                        // becomes S x + (1 - S) out instead of S x + out
};
// y holds the samples [y0, yg.n) of the link grid yg, laid out as in
// launch_links_full; samples below y0 read as zero.
int launch_tdi(const SegTable& tab, const lisa_grid& yg, const void* y, int precision, int gen, int mode, int channels,
               const lisa_grid& og, void* xyz, int64_t i_begin, int64_t i_end, const BlendSpec& bl, cudaStream_t st,
               int64_t y0 = 0);

// LFA: z series (optional) and channels (optional) on out-grid samples
// [i_begin, i_end), z recomputed with its 2-sample halo inside each tile.
// gen = kLfaOwnTime evaluates the LFA link formula for each of the six links
// at its own reception time (no TDI shift): z[6][og.n] in link order (xyz
// must be null).
constexpr int kLfaOwnTime = 0;
// group: tiles per CTA of the mixed kernel (0: lfa_group_mixed of the grid step).
int launch_lfa(const SegTable& tab, const SkyDev& sky, double L_nominal, const lisa_grid& hg, const void* hp,
               const void* hc, int precision, int gen, int kind, int channels, const lisa_grid& og, void* z,
               void* xyz, int64_t i_begin, int64_t i_end, const BlendSpec& bl, cudaStream_t st, int group = 0);
int launch_tdi_lfa(const SegTable& tab, double L_nominal, const lisa_grid& zg, const void* z, int precision, int gen,
                   int kind, int channels, void* xyz, cudaStream_t st);

// Shared host helpers of the C ABI (validation and orchestration).
#define LISA_TRY(x)                     \
    do {                                \
        int _rc = (x);                  \
        if (_rc != LISA_OK) return _rc; \
    } while (0)
int check_grid(const lisa_grid& g, const char* name);
int check_orbit(const lisa_orbit* o);
int check_common(int precision, int gen, int channels);
size_t real_size(int precision);
// Orbit polynomial table on grid g, in scratch.
int make_table(const lisa_orbit* orbit, const lisa_grid& g, Scratch& sc, SegTable& tab, cudaStream_t st);
int make_table_pair(const lisa_orbit* orbit, const lisa_grid& g1, const lisa_grid& g2, Scratch& sc, SegTable& tab1,
                    SegTable& tab2, cudaStream_t st);
// Upper bound of any single light time (halo sizing).
double max_light_time(const lisa_orbit* o, const lisa_grid& g);
// Tiles per CTA group of the mixed LFA kernel for a grid step dt (host side).
// A second stream (with a fork and a join event) for work of a call that does
// not depend on the work queued before it on the caller's stream after the
// fork; one set per concurrent call and device, reused (api.cu).  nullptr if
// none can be created: the caller then stays on its own stream.
struct SideRes {
    int device = -1;
    bool busy = false;
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};
SideRes* side_acquire();
void side_release(SideRes* r);
struct SideGuard {
    SideRes* r;
    ~SideGuard()
    {
        if (r) side_release(r);
    }
};

int lfa_group_host(double dt);
// tiles per LFA group of the kernel that serves the precision (chunk boundaries)
int lfa_group_host(double dt, int precision);
// Hybrid regions on grid `out`: LFA samples [0, iL] (t <= t_hyb + Tw/2), full
// samples [iF, n) (t >= t_hyb - Tw/2).
void hybrid_split(const lisa_grid& out, double t_hyb, double Tw, int64_t& iL, int64_t& iF);
// First sample of the full links a hybrid needs for its full samples [iF, n).
int64_t hybrid_links_begin(const lisa_orbit* orbit, const lisa_grid& out, int64_t iF);

}  // namespace lisa
