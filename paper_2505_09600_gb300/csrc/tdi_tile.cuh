// Per-tile prologue and per-sample body of the Michelson TDI combination,
// shared by the TDI kernel and the fused full-response tile of the batched
// kernel.  See tdi.cu for the definitions.
#pragma once

#include <type_traits>

#include "lisa_common.cuh"
#include "lisa_internal.cuh"
#include "tile_geo.cuh"

namespace lisa {


constexpr int kWinY = kTile + 256;

struct TdiTerm {
    int sign, link, nd;
    int d[8];
};

static __constant__ TdiTerm c_terms[16] = {
    {+1, 5, 3, {3, 2, 4}},              {-1, 5, 1, {4}},
    {+1, 4, 2, {3, 2}},                 {-1, 4, 0, {0}},
    {+1, 2, 1, {3}},                    {-1, 2, 3, {4, 5, 3}},
    {+1, 3, 0, {0}},                    {-1, 3, 2, {4, 5}},
    {+1, 5, 5, {3, 2, 4, 5, 4}},        {-1, 5, 7, {4, 5, 3, 2, 3, 2, 4}},
    {+1, 4, 4, {3, 2, 4, 5}},           {-1, 4, 6, {4, 5, 3, 2, 3, 2}},
    {+1, 2, 7, {3, 2, 4, 5, 4, 5, 3}},  {-1, 2, 5, {4, 5, 3, 2, 3}},
    {+1, 3, 6, {3, 2, 4, 5, 4, 5}},     {-1, 3, 4, {4, 5, 3, 2}},
};
static __constant__ int c_cyc[3][6] = {{0, 1, 2, 3, 4, 5}, {2, 3, 4, 5, 0, 1}, {4, 5, 0, 1, 2, 3}};

struct TdiArgs {
    SegTable tab;
    GridMap ym;
    const void* y;
    int64_t ny;
    void* xyz;
    int64_t nout;
    int nterm, mode, channels;
    int64_t i_begin, i_end, tile0;
    BlendSpec bl;
    double t0_out, dt_out;
};

template <typename Real>
__device__ __forceinline__ Real interp_one(const Real* win, int64_t wlo, int wlen, const Real* __restrict__ yg,
                                           int64_t n, int64_t j, Real eps)
{
    if (eps == Real(0)) {
        const int64_t o = j - wlo;
        if (o >= 0 && o < wlen) return win[o];
        return (j >= 0 && j < n) ? yg[j] : Real(0);
    }
    Real w[32];
    lagrange32_weights(eps, w);
    Real acc = Real(0);
    const int64_t base = j - 15 - wlo;
    if (base >= 0 && base + 32 <= wlen) {
        const Real* p = win + base;
#pragma unroll
        for (int k = 0; k < 32; ++k) acc = fma(w[k], p[k], acc);
    } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const int64_t idx = j - 15 + k;
            if (idx >= 0 && idx < n) acc = fma(w[k], yg[idx], acc);
        }
    }
    return acc;
}

// Epilogue shared by the full and LFA channel kernels: optional AET, optional
// sigmoid weight, optional accumulation onto the existing output.
// Mixed-precision store: the sigmoid argument comes from per-tile FP32
// constants (|error| < 1e-5 in the argument, < 3e-6 in the weight).
__device__ __forceinline__ void store_channels_f32(float X, float Y, float Z, int channels, const BlendSpec& bl,
                                                   float barg_c, float barg_d, int di, int64_t i, float* __restrict__ out,
                                                   int64_t n)
{
    float o0 = X, o1 = Y, o2 = Z;
    if (channels == LISA_AET) {
        o0 = (Z - X) * 0.70710678118654752440f;
        o1 = (X - 2.f * Y + Z) * 0.40824829046386301637f;
        o2 = (X + Y + Z) * 0.57735026918962576451f;
    }
    if (bl.enabled) {
        const float e = expf(fmaf((float)di, barg_d, barg_c));
        const float wgt = 1.f / (1.f + e);
        o0 *= wgt;
        o1 *= wgt;
        o2 *= wgt;
        if (i >= bl.acc_begin && i < bl.acc_end) {
            // 1 - S = e S, formed without the cancellation of 1 - S
            const float keep = bl.lerp ? e * wgt : 1.f;
            o0 = fmaf(keep, out[i], o0);
            o1 = fmaf(keep, out[n + i], o1);
            o2 = fmaf(keep, out[2 * n + i], o2);
        }
    }
    out[i] = o0;
    out[n + i] = o1;
    out[2 * n + i] = o2;
}

template <typename Real>
__device__ __forceinline__ void store_channels(Real X, Real Y, Real Z, int channels, const BlendSpec& bl,
                                               double t0, double dt, int64_t i, Real* __restrict__ out, int64_t n)
{
    Real o0 = X, o1 = Y, o2 = Z;
    if (channels == LISA_AET) {
        o0 = (Z - X) * Real(0.70710678118654752440);
        o1 = (X - Real(2) * Y + Z) * Real(0.40824829046386301637);
        o2 = (X + Y + Z) * Real(0.57735026918962576451);
    }
    if (bl.enabled) {
        const double ti = t0 + (double)i * dt;
        const double arg = bl.eps * (ti - bl.t_hyb) / bl.sigma;
        Real wgt, e;
        if constexpr (sizeof(Real) == 8) {
            e = exp(arg);
            wgt = 1.0 / (1.0 + e);
        } else {
            e = expf((float)arg);
            wgt = 1.f / (1.f + e);
        }
        o0 *= wgt;
        o1 *= wgt;
        o2 *= wgt;
        if (i >= bl.acc_begin && i < bl.acc_end) {
            if (bl.lerp) {
                const Real keep = e * wgt;   // 1 - S
                o0 += keep * out[i];
                o1 += keep * out[n + i];
                o2 += keep * out[2 * n + i];
            } else {
                o0 += out[i];
                o1 += out[n + i];
                o2 += out[2 * n + i];
            }
        }
    }
    out[i] = o0;
    out[n + i] = o1;
    out[2 * n + i] = o2;
}


// Shared memory of one TDI tile: the six link series over the window the
// tile's delays reach, and for the mixed frozen form the per-(channel, term)
// tile-centre split of the delay and its in-tile cubic.
template <bool MIXED>
struct TdiTile {
    using Real = typename std::conditional<MIXED, float, double>::type;
    Real win[6][kWinY];
    int64_t wlo;
    int wlen;
    int64_t J[48];
    float f[48];
    Cubic dD[48];
    float inv_half, inv_dt;        // FP32 constants
    float barg_c, barg_d;          // sigmoid argument at the tile centre and per sample
};

// Window range and mixed per-term data.  Every thread must call it.
template <bool MIXED>
__device__ void tdi_tile_prologue(const TdiArgs& a, const TileGeo& g, int64_t ic, int64_t i0, TdiTile<MIXED>& s)
{
    const double half = 0.5 * a.tab.S;
    const int t = threadIdx.x;
    if constexpr (MIXED) {
        if (t == 1) {
            s.inv_half = (float)(2.0 / a.tab.S);
            s.inv_dt = (float)(1.0 / a.ym.dt_in);
            const double tc = a.t0_out + (double)ic * a.dt_out;
            s.barg_c = (float)(a.bl.enabled ? a.bl.eps * (tc - a.bl.t_hyb) / a.bl.sigma : 0.0);
            s.barg_d = (float)(a.bl.enabled ? a.bl.eps * a.dt_out / a.bl.sigma : 0.0);
        }
        if (a.mode == LISA_FROZEN && t >= 64 && t < 64 + 3 * a.nterm) {
            const int w = t - 64, ch = w / a.nterm, q = w % a.nterm;
            const TdiTerm& tm = c_terms[q];
            double Dc = 0.0;
            Cubic cv{0.f, 0.f, 0.f};
            for (int k = 0; k < tm.nd; ++k) {
                const int row = kQT + c_cyc[ch][tm.d[k]];
                Dc += g.b[row][0];
                const Cubic cr = tg_cubic(g, row);
                cv.c1 += cr.c1; cv.c2 += cr.c2; cv.c3 += cr.c3;
            }
            int64_t j;
            double eps;
            split_f64(a.ym, ic, Dc, j, eps);
            s.J[w] = j;
            s.f[w] = (float)eps;
            s.dD[w] = cv;
        }
    }
    if (t == 0) {
        // largest delay of any term: up to 7 light times, +1 s of margin
        double Tmax = 0.0;
        for (int li = 0; li < 6; ++li) {
            const double a0 = tg_eval(g, kQT + li, (double)(i0 - ic) / half);
            const double a1 = tg_eval(g, kQT + li, (double)(i0 + kTile - 1 - ic) / half);
            Tmax = fmax(Tmax, fmax(a0, a1));
        }
        const double Dmax = (a.nterm == 16 ? 7.0 : 3.0) * Tmax + 1.0;
        int64_t jlo, jhi;
        double e;
        split_f64(a.ym, i0, Dmax, jlo, e);
        split_f64(a.ym, i0 + kTile - 1, -1.0, jhi, e);
        s.wlo = jlo - 15 - 2;
        const int64_t len = (jhi + 16 + 2) - s.wlo + 1;
        s.wlen = len <= kWinY ? (int)len : 0;
    }
    __syncthreads();
}

// Fill the window from the link series in global memory.
template <bool MIXED>
__device__ void tdi_fill_global(const TdiArgs& a, TdiTile<MIXED>& s)
{
    using Real = typename std::conditional<MIXED, float, double>::type;
    const Real* __restrict__ yg = (const Real*)a.y;
    const int64_t wlo = s.wlo;
    const int wlen = s.wlen;
    for (int li = 0; li < 6; ++li)
        for (int o = threadIdx.x; o < wlen; o += blockDim.x) {
            const int64_t idx = wlo + o;
            s.win[li][o] = (idx >= 0 && idx < a.ym.n_in) ? yg[(int64_t)li * a.ny + idx] : Real(0);
        }
    __syncthreads();
}

// X, Y, Z at output sample i (before AET, blend and store).
template <bool MIXED>
__device__ __forceinline__ void tdi_sample(const TdiArgs& a, const TileGeo& g, int64_t ic, int64_t i,
                                           const TdiTile<MIXED>& s,
                                           typename std::conditional<MIXED, float, double>::type (&acc)[3])
{
    using Real = typename std::conditional<MIXED, float, double>::type;
    const Real* __restrict__ yg = (const Real*)a.y;
    const double half = 0.5 * a.tab.S;
    const int64_t wlo = s.wlo;
    const int wlen = s.wlen;
    acc[0] = acc[1] = acc[2] = Real(0);
    if (!MIXED || a.mode == LISA_NESTED) {
        const double u = (double)(i - ic) / half;
        double T[6];
#pragma unroll
        for (int li = 0; li < 6; ++li) T[li] = tg_eval(g, kQT + li, u);
#pragma unroll 1
        for (int ch = 0; ch < 3; ++ch) {
#pragma unroll 1
            for (int q = 0; q < a.nterm; ++q) {
                const TdiTerm& tm = c_terms[q];
                double D = 0.0;
                for (int k = 0; k < tm.nd; ++k) {
                    const int li = c_cyc[ch][tm.d[k]];
                    if (a.mode == LISA_NESTED) {
                        D += tg_eval(g, kQT + li, u - D / (a.dt_out * half));
                    } else {
                        double Tl = T[0];
                        for (int r = 1; r < 6; ++r) Tl = (li == r) ? T[r] : Tl;
                        D += Tl;
                    }
                }
                int64_t j;
                double eps;
                split_f64(a.ym, i, D, j, eps);
                const int ls = c_cyc[ch][tm.link];
                const Real v = interp_one<Real>(s.win[ls], wlo, wlen, yg ? yg + (int64_t)ls * a.ny : nullptr,
                                                yg ? a.ym.n_in : 0, j, (Real)eps);
                acc[ch] += (tm.sign > 0) ? v : -v;
            }
        }
    } else if constexpr (MIXED) {
        const float u = (float)(int)(i - ic) * s.inv_half;
        int64_t jp;
        float fp;
        if (a.ym.unit_rho) {
            jp = i - ic;
            fp = 0.f;
        } else {
            const double P = (double)(i - ic) * a.ym.rho;
            const double fl = floor(P);
            jp = (int64_t)fl;
            fp = (float)(P - fl);
        }
        const float inv_dt = s.inv_dt;
#pragma unroll 1
        for (int ch = 0; ch < 3; ++ch) {
#pragma unroll 1
            for (int q = 0; q < a.nterm; ++q) {
                const int w = ch * a.nterm + q;
                const float v = (fp + s.f[w]) - s.dD[w](u) * inv_dt;
                const float fv = floorf(v);
                const int64_t j = s.J[w] + jp + (int)fv;
                const float eps = v - fv;
                const TdiTerm& tm = c_terms[q];
                const int ls = c_cyc[ch][tm.link];
                const float val = interp_one<float>(s.win[ls], wlo, wlen, yg ? yg + (int64_t)ls * a.ny : nullptr,
                                                    yg ? a.ym.n_in : 0, j, eps);
                acc[ch] += (tm.sign > 0) ? val : -val;
            }
        }
    }
}

}  // namespace lisa
