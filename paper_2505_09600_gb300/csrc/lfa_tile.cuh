// Per-tile body of the low-frequency approximation, shared by the LFA kernel
// and the batched persistent kernel.  See lfa.cu for the method.
#pragma once

#include <type_traits>

#include "lisa_common.cuh"
#include "lisa_internal.cuh"
#include "tile_geo.cuh"

namespace lisa {

constexpr int kWinH = kTile + 384;
constexpr int kZW = kTile + 4;

template <typename Real>
struct PairT;
template <>
struct PairT<double> { using T = double2; };
template <>
struct PairT<float> { using T = float2; };

struct LfaArgs {
    SegTable tab;
    SkyDev sky;
    GridMap hm;
    double Lc;
    int gen, kind, channels;
    const void* hp;
    const void* hc;
    void* z;
    void* xyz;
    int64_t nout;
    double t0_out, dt_out;
    int64_t i_begin, i_end, tile0;
    BlendSpec bl;
    float Lcf, dtf, inv12dtf;   // FP32 copies of Lc, dt_out and 1/(12 dt_in) (mixed form)
};

// Fill the FP32 copies of LfaArgs (host side).
inline void lfa_args_f32(LfaArgs& a)
{
    a.Lcf = (float)a.Lc;
    a.dtf = (float)a.dt_out;
    a.inv12dtf = (float)(1.0 / (12.0 * a.hm.dt_in));
}


// Channel ch: links a = cyc(+2), b = cyc(+3); arms T_a = cyc(+3), T_b = cyc(+2).
__device__ __forceinline__ int lfa_link(int ch, int which) { return link_cycle(which ? 4 : 2, ch); }
__device__ __forceinline__ int lfa_arm(int ch, int which) { return link_cycle(which ? 2 : 4, ch); }

__device__ __forceinline__ double lfa_shift(int gen, double Ta, double Tb)
{
    return gen == LISA_TDI20 ? 2.0 * Ta + 1.5 * Tb : gen == LISA_TDI15 ? Ta + 0.5 * Tb : 0.0;
}

template <typename Real>
__device__ __forceinline__ Real interp_pair_w(const typename PairT<Real>::T* win, int64_t wlo, int wlen,
                                              const typename PairT<Real>::T* __restrict__ dummy, int64_t j, Real eps,
                                              Real& oc, bool& ok)
{
    const int64_t base = j - 15 - wlo;
    ok = (base >= 0 && base + 32 <= wlen);
    if (!ok) { oc = Real(0); return Real(0); }
    if (eps == Real(0)) {
        oc = win[j - wlo].y;
        return win[j - wlo].x;
    }
    Real w[32];
    lagrange32_weights(eps, w);
    Real ap = Real(0), ac = Real(0);
    const typename PairT<Real>::T* p = win + base;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        const typename PairT<Real>::T v = p[k];
        ap = fma(w[k], v.x, ap);
        ac = fma(w[k], v.y, ac);
    }
    oc = ac;
    return ap;
}

// hdot at grid sample idx straight from global memory (fallback path).
template <typename Real>
__device__ __forceinline__ Real hdot_global(const Real* __restrict__ h, int64_t n, int64_t idx, Real inv12dt)
{
    if (idx < 0 || idx >= n) return Real(0);
    auto at = [&](int64_t k) { return (k >= 0 && k < n) ? h[k] : Real(0); };
    return ((at(idx + 1) - at(idx - 1)) * Real(8) - (at(idx + 2) - at(idx - 2))) * inv12dt;
}

template <typename Real>
__device__ __forceinline__ void interp_hdot_global(const Real* __restrict__ hp, const Real* __restrict__ hc, int64_t n,
                                                   int64_t j, Real eps, Real inv12dt, Real& op, Real& oc)
{
    if (eps == Real(0)) {
        op = hdot_global(hp, n, j, inv12dt);
        oc = hdot_global(hc, n, j, inv12dt);
        return;
    }
    Real w[32];
    lagrange32_weights(eps, w);
    Real ap = Real(0), ac = Real(0);
#pragma unroll
    for (int k = 0; k < 32; ++k) {
        ap = fma(w[k], hdot_global(hp, n, j - 15 + k, inv12dt), ap);
        ac = fma(w[k], hdot_global(hc, n, j - 15 + k, inv12dt), ac);
    }
    op = ap;
    oc = ac;
}

template <bool MIXED>
struct LfaSmem {
    using Real = typename std::conditional<MIXED, float, double>::type;
    using Real2 = typename PairT<Real>::T;
    TileGeo g;
    Real2 hw[kWinH];      // h window (+2 each side)
    Real2 dw[kWinH];      // hdot window
    Real zs[6][kZW];
    int64_t jends[12];
    int64_t wlo;
    int wlen;
    // mixed: FP32 rows (centre value, cubic) and per-series centre splits
    float c0[kRows];
    Cubic cu[kRows];
    double ac[6];
    Cubic da[6];
    int64_t J[6];
    float f[6];
    float acu[6];                 // centre shift in segment units
    float inv_half, inv_dt, u_per_s;   // FP32 constants
    float barg_c, barg_d;         // sigmoid argument at the tile centre and per sample
};

// FP64 per-tile set-up around the centre sample ic: the orbit geometry
// (Taylor shift of the segment polynomials) and, for the mixed form, the FP32
// constants of every z series (centre delay split, in-tile cubics).  Every
// thread of the block must call it (it synchronises).
template <bool MIXED>
__device__ void lfa_tile_prologue(const LfaArgs& a, int64_t ic, LfaSmem<MIXED>& sm)
{
    TileGeo& g = sm.g;
    const double half = 0.5 * a.tab.S;
    const double u_per_s = 1.0 / (a.dt_out * half);
    const int t = threadIdx.x;
    const bool equal = (a.kind == LISA_LFA_EQUAL);
    tile_geo_load(g, a.tab, ic, a.sky);
    if constexpr (MIXED) {
        if (t == 12) {
            sm.inv_half = (float)(2.0 / a.tab.S);
            sm.inv_dt = (float)(1.0 / a.hm.dt_in);
            sm.u_per_s = (float)u_per_s;
            const double tc = a.t0_out + (double)ic * a.dt_out;
            sm.barg_c = (float)(a.bl.enabled ? a.bl.eps * (tc - a.bl.t_hyb) / a.bl.sigma : 0.0);
            sm.barg_d = (float)(a.bl.enabled ? a.bl.eps * a.dt_out / a.bl.sigma : 0.0);
        }
        if (t >= 32 && t < 32 + kRows) {
            const int r = t - 32;
            sm.c0[r] = (float)g.b[r][0];
            sm.cu[r] = tg_cubic(g, r);
        }
        if (t >= 96 && t < 102) {
            const int c = t - 96, ch = c >> 1, which = c & 1;
            const int ra = kQT + lfa_arm(ch, 0), rb = kQT + lfa_arm(ch, 1);
            const double Ta = equal ? a.Lc : g.b[ra][0], Tb = equal ? a.Lc : g.b[rb][0];
            const double ac = which ? lfa_shift(a.gen, Tb, Ta) : lfa_shift(a.gen, Ta, Tb);
            Cubic da{0.f, 0.f, 0.f};
            if (!equal) {
                const Cubic ca = tg_cubic(g, ra), cb = tg_cubic(g, rb);
                float fa = which ? (a.gen == LISA_TDI20 ? 1.5f : 0.5f) : (a.gen == LISA_TDI20 ? 2.f : 1.f);
                float fb = which ? (a.gen == LISA_TDI20 ? 2.f : 1.f) : (a.gen == LISA_TDI20 ? 1.5f : 0.5f);
                if (a.gen == kLfaOwnTime) fa = fb = 0.f;
                da = Cubic{fa * ca.c1 + fb * cb.c1, fa * ca.c2 + fb * cb.c2, fa * ca.c3 + fb * cb.c3};
            }
            const int l = a.gen == kLfaOwnTime ? c : lfa_link(ch, which);
            const double Tl = equal ? a.Lc : g.b[kQT + l][0];
            const double dc = ac + 0.5 * Tl + 0.5 * (g.b[kRowKR + link_sender(l)][0] + g.b[kRowKR + link_receiver(l)][0]);
            int64_t j;
            double eps;
            split_f64(a.hm, ic, dc, j, eps);
            sm.ac[c] = ac;
            sm.acu[c] = (float)(ac * u_per_s);
            sm.da[c] = da;
            sm.J[c] = j;
            sm.f[c] = (float)eps;
        }
    }
    __syncthreads();
}

// Mixed form: integer sample and fraction of the retarded time of series c
// at output sample m, from the FP32 constants of the tile centre ic.
__device__ __forceinline__ void lfa_locate_f32(const LfaArgs& a, const LfaSmem<true>& sm, int c, int64_t m,
                                               int64_t ic, bool equal, int64_t& j, float& eps, float& Tl,
                                               float (&n3)[3])
{
    const int ch = c >> 1, which = c & 1;
    const int l = a.gen == kLfaOwnTime ? c : lfa_link(ch, which);
    // in-tile offsets are 32-bit: no 64-bit conversions (FP64 pipe) per sample
    const float u = (float)(int)(m - ic) * sm.inv_half;
    const float da = sm.da[c](u);
    const float up = u - sm.acu[c] - da * sm.u_per_s;
    const float dT = equal ? 0.f : sm.cu[kQT + l](up);
    Tl = equal ? a.Lcf : sm.c0[kQT + l] + dT;
    const float ddt = da + 0.5f * dT + 0.5f * (sm.cu[kRowKR + link_sender(l)](up) + sm.cu[kRowKR + link_receiver(l)](up));
    for (int q = 0; q < 3; ++q) n3[q] = sm.c0[kQN + 3 * l + q] + sm.cu[kQN + 3 * l + q](up);
    int64_t jp;
    float fp;
    if (a.hm.unit_rho) {
        jp = m - ic;
        fp = 0.f;
    } else {
        const double P = (double)(m - ic) * a.hm.rho;
        const double fl = floor(P);
        jp = (int64_t)fl;
        fp = (float)(P - fl);
    }
    const float v = (fp + sm.f[c]) - ddt * sm.inv_dt;
    const float fv = floorf(v);
    j = sm.J[c] + jp + (int)fv;
    eps = v - fv;
}

// One tile [i0, i0 + kTile) of LFA channels, after lfa_tile_prologue at the
// centre ic (the tile's own centre, or that of a group of tiles sharing one
// prologue): on return thread t holds X, Y, Z of sample i0 + t (before AET,
// blend and store) and z has been written if requested.  With reuse_halo the
// previous tile [i0 - kTile, i0) was the last one computed in this block, and
// its last four z values are this tile's leading halo: the block then
// computes exactly kTile values per series (no straggling round for the
// halo).  Every thread of the block must call it; it does not return early,
// so it can run inside a persistent loop.
template <bool MIXED>
__device__ void lfa_tile_body(const LfaArgs& a, int64_t i0, int64_t ic, LfaSmem<MIXED>& sm,
                              typename std::conditional<MIXED, float, double>::type (&X)[3], bool reuse_halo = false)
{
    using Real = typename std::conditional<MIXED, float, double>::type;
    using Real2 = typename PairT<Real>::T;
    TileGeo& g = sm.g;
    const Real* __restrict__ hp = (const Real*)a.hp;
    const Real* __restrict__ hc = (const Real*)a.hc;
    const double half = 0.5 * a.tab.S;
    const double u_per_s = 1.0 / (a.dt_out * half);
    const int t = threadIdx.x;
    const bool equal = (a.kind == LISA_LFA_EQUAL);
    __syncthreads();   // the previous tile's readers of the windows are done
    // z of samples i0-2 .. i0+1 were computed as the previous tile's i0'+256 .. i0'+259
    if (reuse_halo && t < 24) {
        const int c = t >> 2, o = t & 3;
        sm.zs[c][o] = sm.zs[c][kTile + o];
    }

    // --- window of h this tile reaches: the retarded samples of the 6 series
    //     at the tile's two ends (2-sample halo included)
    if (t < 12) {
        const int c = t % 6;
        const int64_t m = (t < 6) ? i0 - 2 : i0 + kTile + 1;
        int64_t j;
        if constexpr (MIXED) {
            float eps, Tl, n3[3];
            lfa_locate_f32(a, sm, c, m, ic, equal, j, eps, Tl, n3);
        } else {
            const double u = (double)(m - ic) / half;
            const int ch = c >> 1, which = c & 1;
            const double Ta = equal ? a.Lc : tg_eval(g, kQT + lfa_arm(ch, 0), u);
            const double Tb = equal ? a.Lc : tg_eval(g, kQT + lfa_arm(ch, 1), u);
            const double sh = which ? lfa_shift(a.gen, Tb, Ta) : lfa_shift(a.gen, Ta, Tb);
            const int l = a.gen == kLfaOwnTime ? c : lfa_link(ch, which);
            const double up = u - sh * u_per_s;
            const double Tl = equal ? a.Lc : tg_eval(g, kQT + l, up);
            const double d = sh + 0.5 * Tl
                           + 0.5 * (tg_eval(g, kRowKR + link_sender(l), up) + tg_eval(g, kRowKR + link_receiver(l), up));
            double eps;
            split_f64(a.hm, m, d, j, eps);
        }
        sm.jends[t] = j;
    }
    __syncthreads();
    if (t == 0) {
        int64_t lo = sm.jends[0], hi = sm.jends[0];
        for (int k = 1; k < 12; ++k) {
            lo = sm.jends[k] < lo ? sm.jends[k] : lo;
            hi = sm.jends[k] > hi ? sm.jends[k] : hi;
        }
        sm.wlo = lo - 15 - 3;
        const int64_t len = (hi + 16 + 3) - sm.wlo + 1;
        sm.wlen = (len + 4 <= kWinH) ? (int)len : 0;
    }
    __syncthreads();
    const int64_t wlo = sm.wlo;
    const int wlen = sm.wlen;
    Real inv12dt;
    if constexpr (MIXED) inv12dt = a.inv12dtf;
    else inv12dt = 1.0 / (12.0 * a.hm.dt_in);
    // h over [wlo-2, wlo+wlen+2), then hdot over [wlo, wlo+wlen)
    for (int k = t; k < wlen + 4; k += blockDim.x) {
        const int64_t idx = wlo - 2 + k;
        Real2 v;
        v.x = (idx >= 0 && idx < a.hm.n_in) ? hp[idx] : Real(0);
        v.y = (idx >= 0 && idx < a.hm.n_in) ? hc[idx] : Real(0);
        sm.hw[k] = v;
    }
    __syncthreads();
    for (int k = t; k < wlen; k += blockDim.x) {
        // hdot is defined on the h grid only and is zero outside it, like h
        const int64_t idx = wlo + k;
        const Real2 m2 = sm.hw[k], m1 = sm.hw[k + 1], p1 = sm.hw[k + 3], p2 = sm.hw[k + 4];
        Real2 d;
        const bool in = (idx >= 0 && idx < a.hm.n_in);
        d.x = in ? ((p1.x - m1.x) * Real(8) - (p2.x - m2.x)) * inv12dt : Real(0);
        d.y = in ? ((p1.y - m1.y) * Real(8) - (p2.y - m2.y)) * inv12dt : Real(0);
        sm.dw[k] = d;
    }
    __syncthreads();

    Real c2, s2, ku[3], kv[3];
    if constexpr (MIXED) {
        c2 = a.sky.c2f; s2 = a.sky.s2f;
        for (int q = 0; q < 3; ++q) { ku[q] = a.sky.uf[q]; kv[q] = a.sky.vf[q]; }
    } else {
        c2 = a.sky.c2p; s2 = a.sky.s2p;
        for (int q = 0; q < 3; ++q) { ku[q] = a.sky.u[q]; kv[q] = a.sky.v[q]; }
    }
    const float Lcf = a.Lcf;

    // --- z on the tile and its halo: (kTile + 4) x 6 values ----------------
    const int per = reuse_halo ? kTile : kZW;
    for (int w = t; w < 6 * per; w += blockDim.x) {
        // constant divisors: kTile values per series after a reused halo, else kZW
        const int c = reuse_halo ? w / kTile : w / kZW;
        const int o = reuse_halo ? 4 + w % kTile : w % kZW;
        const int64_t m = i0 - 2 + o;
        Real zval = Real(0);
        if (m >= 0 && m < a.nout) {
            const int ch = c >> 1, which = c & 1;
            const int l = a.gen == kLfaOwnTime ? c : lfa_link(ch, which);
            Real Tl, n3[3];
            int64_t j;
            Real eps;
            if constexpr (!MIXED) {
                const double u = (double)(m - ic) / half;
                const double Ta = equal ? a.Lc : tg_eval(g, kQT + lfa_arm(ch, 0), u);
                const double Tb = equal ? a.Lc : tg_eval(g, kQT + lfa_arm(ch, 1), u);
                const double sh = which ? lfa_shift(a.gen, Tb, Ta) : lfa_shift(a.gen, Ta, Tb);
                const double up = u - sh * u_per_s;
                Tl = equal ? a.Lc : tg_eval(g, kQT + l, up);
                const double dtau = sh + 0.5 * Tl
                                  + 0.5 * (tg_eval(g, kRowKR + link_sender(l), up) + tg_eval(g, kRowKR + link_receiver(l), up));
                for (int q = 0; q < 3; ++q) n3[q] = tg_eval(g, kQN + 3 * l + q, up);
                double e;
                split_f64(a.hm, m, dtau, j, e);
                eps = e;
            } else {
                float e, T32, n32[3];
                lfa_locate_f32(a, sm, c, m, ic, equal, j, e, T32, n32);
                eps = e;
                Tl = T32;
                n3[0] = n32[0];
                n3[1] = n32[1];
                n3[2] = n32[2];
            }
            const Real un = ku[0] * n3[0] + ku[1] * n3[1] + ku[2] * n3[2];
            const Real vn = kv[0] * n3[0] + kv[1] * n3[1] + kv[2] * n3[2];
            const Real xp = un * un - vn * vn, xc = Real(2) * un * vn;
            Real dp, dc;
            bool ok;
            dp = interp_pair_w<Real>(sm.dw, wlo, wlen, nullptr, j, eps, dc, ok);
            if (!ok) interp_hdot_global<Real>(hp, hc, a.hm.n_in, j, eps, inv12dt, dp, dc);
            zval = Real(-0.5) * Tl * (dp * (xp * c2 + xc * s2) + dc * (xc * c2 - xp * s2));
        }
        sm.zs[c][o] = zval;
    }
    __syncthreads();

    const int64_t i = i0 + t;
    if (a.z && i >= a.i_begin && i < a.i_end) {
        Real* zo = (Real*)a.z;
        for (int c = 0; c < 6; ++c) zo[(int64_t)c * a.nout + i] = sm.zs[c][t + 2];
    }
    Real dt;
    if constexpr (MIXED) dt = a.dtf;
    else dt = a.dt_out;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        Real Ta, Tb;
        if constexpr (!MIXED) {
            const double u = (double)(i - ic) / half;
            Ta = equal ? a.Lc : tg_eval(g, kQT + lfa_arm(ch, 0), u);
            Tb = equal ? a.Lc : tg_eval(g, kQT + lfa_arm(ch, 1), u);
        } else {
            const float u = (float)(int)(i - ic) * sm.inv_half;
            Ta = equal ? Lcf : sm.c0[kQT + lfa_arm(ch, 0)] + sm.cu[kQT + lfa_arm(ch, 0)](u);
            Tb = equal ? Lcf : sm.c0[kQT + lfa_arm(ch, 1)] + sm.cu[kQT + lfa_arm(ch, 1)](u);
        }
        const Real* za = sm.zs[2 * ch] + t;       // za[0..4] = z at i-2..i+2
        const Real* zb = sm.zs[2 * ch + 1] + t;
        if (a.gen == LISA_TDI20) {
            // 5-point second derivative as (14 d2_0 - d2_-1 - d2_1)/12, d2 from first differences
            auto d2 = [&](const Real* z) {
                const Real e0 = z[1] - z[0], e1 = z[2] - z[1], e2 = z[3] - z[2], e3 = z[4] - z[3];
                const Real m1 = e1 - e0, c0 = e2 - e1, p1 = e3 - e2;
                return (Real(14) * c0 - m1 - p1) / (Real(12) * dt * dt);
            };
            X[ch] = Real(8) * (Ta + Tb) * (Ta * d2(za) - Tb * d2(zb));
        } else {
            auto d1 = [&](const Real* z) { return ((z[3] - z[1]) * Real(8) - (z[4] - z[0])) / (Real(12) * dt); };
            X[ch] = Real(4) * (Ta * d1(za) - Tb * d1(zb));
        }
    }
}

// Prologue and body of one tile around its own centre.
template <bool MIXED>
__device__ __forceinline__ void lfa_tile_compute(const LfaArgs& a, int64_t i0, LfaSmem<MIXED>& sm,
                                                 typename std::conditional<MIXED, float, double>::type (&X)[3])
{
    const int64_t ic = i0 + kTile / 2;
    lfa_tile_prologue<MIXED>(a, ic, sm);
    lfa_tile_body<MIXED>(a, i0, ic, sm, X);
}

// AET, sigmoid weight (LFA side: eps = +1) and store of one sample.
template <typename Real>
__device__ __forceinline__ void lfa_store(const LfaArgs& a, int64_t i, const Real (&X)[3], float barg_c = 0.f,
                                          float barg_d = 0.f, int di = 0)
{
    Real* out = (Real*)a.xyz;
    Real o0 = X[0], o1 = X[1], o2 = X[2];
    if (a.channels == LISA_AET) {
        o0 = (X[2] - X[0]) * Real(0.70710678118654752440);
        o1 = (X[0] - Real(2) * X[1] + X[2]) * Real(0.40824829046386301637);
        o2 = (X[0] + X[1] + X[2]) * Real(0.57735026918962576451);
    }
    if (a.bl.enabled) {
        double arg = 0.0;
        if constexpr (sizeof(Real) == 8) {
            const double ti = a.t0_out + (double)i * a.dt_out;
            arg = a.bl.eps * (ti - a.bl.t_hyb) / a.bl.sigma;
        }
        Real wgt;
        if constexpr (sizeof(Real) == 4) wgt = 1.f / (1.f + expf(fmaf((float)di, barg_d, barg_c)));
        else wgt = 1.0 / (1.0 + exp(arg));
        o0 *= wgt;
        o1 *= wgt;
        o2 *= wgt;
    }
    out[i] = o0;
    out[a.nout + i] = o1;
    out[2 * a.nout + i] = o2;
}

}  // namespace lisa
