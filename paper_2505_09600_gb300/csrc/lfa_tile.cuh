// Per-tile body of the low-frequency approximation, shared by the LFA kernel
// and the batched persistent kernel.  See lfa.cu for the method.
#pragma once

#include <type_traits>

#include "async_copy.cuh"
#include "lisa_common.cuh"
#include "lisa_internal.cuh"
#include "tile_geo.cuh"

namespace lisa {

constexpr int kWinH = kTile + 384;
constexpr int kZW = kTile + 4;
constexpr int kWinP = kWinH + 8;   // planar h buffers: room for 16-byte alignment of the copy
#ifndef LISA_LFA_UNROLL
#define LISA_LFA_UNROLL 2
#endif
constexpr int kLfaUnroll = LISA_LFA_UNROLL;   // series per unrolled step of the mixed z loop
#ifndef LISA_LFA_DUNROLL
#define LISA_LFA_DUNROLL 1
#endif
constexpr int kLfaDUnroll = LISA_LFA_DUNROLL;   // series per unrolled step of the differenced channel loop
#ifndef LISA_LFA_PAIR
#define LISA_LFA_PAIR 1   // staged z loop: 1 = a thread's two samples share packed weight instructions, 2 = adjacent samples also share the taps
#endif

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
    float c1f, c2f;             // 1/(12 dt_out) and 1/(12 dt_out^2): the channels' stencil scales
    int h_aligned;              // hp, hc start on 16-byte boundaries (bulk copies allowed)
    unsigned int* status;       // device status word (bounded waits)
};

// Fill the FP32 copies of LfaArgs (host side).
inline void lfa_args_f32(LfaArgs& a)
{
    a.Lcf = (float)a.Lc;
    a.dtf = (float)a.dt_out;
    a.inv12dtf = (float)(1.0 / (12.0 * a.hm.dt_in));
    a.c1f = (float)(1.0 / (12.0 * a.dt_out));
    a.c2f = (float)(1.0 / (12.0 * a.dt_out * a.dt_out));
}


// Channel ch: links a = cyc(+2), b = cyc(+3); arms T_a = cyc(+3), T_b = cyc(+2).
__device__ __forceinline__ int lfa_link(int ch, int which) { return link_cycle(which ? 4 : 2, ch); }
__device__ __forceinline__ int lfa_arm(int ch, int which) { return link_cycle(which ? 2 : 4, ch); }

// Delay of the LFA link's expansion point after the TDI shift sh, from T_l,
// k.R_s/c and k.R_r/c: the central point T_l/2 + k.(R_s + R_r)/(2c)
// (Eq. tau_t_dependence), or, for the non-central variants of App. B, the
// sender end T_l + k.R_s/c (backward) or the receiver end k.R_r/c (forward).
__device__ __forceinline__ double lfa_point_delay(int kind, double sh, double Tl, double ks, double kr)
{
    if (kind == LISA_LFA_BACKWARD) return sh + Tl + ks;
    if (kind == LISA_LFA_FORWARD) return sh + kr;
    return sh + 0.5 * Tl + 0.5 * (ks + kr);
}

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

// Third derivative of h at grid sample idx straight from global memory: the
// 5-point second derivative of hdot, both zero off the grid (fallback path).
template <typename Real>
__device__ __forceinline__ Real hthird_global(const Real* __restrict__ h, int64_t n, int64_t idx, Real inv12dt,
                                             Real inv_dt)
{
    if (idx < 0 || idx >= n) return Real(0);
    return (-hdot_global(h, n, idx - 2, inv12dt) + Real(16) * hdot_global(h, n, idx - 1, inv12dt)
            - Real(30) * hdot_global(h, n, idx, inv12dt) + Real(16) * hdot_global(h, n, idx + 1, inv12dt)
            - hdot_global(h, n, idx + 2, inv12dt)) * inv12dt * inv_dt;
}

// NLO coefficient of the m = 1 link term: for a TDI-shifted series the mean
// over the link and its reverse, (T/2)^2 (1 + (k.n)^2) / 6; for a link at its
// own time (own != 0) [T (1 - k.n)/2]^2 / 6.
template <typename Real>
__device__ __forceinline__ Real nlo_kappa(Real T, Real kn, bool own)
{
    return own ? Real(0.25) * T * T * (Real(1) - kn) * (Real(1) - kn) / Real(6)
               : Real(0.25) * T * T * (Real(1) + kn * kn) / Real(6);
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

// Mixed form: each z series (link l evaluated at tau = t - sh - T_l/2 -
// k.(R_s + R_r)/2c with the TDI shift sh, Sec. III) as FP32 cubics in the
// block's coordinate u = (m - ic) * 2/S around the centre sample ic: the
// total delay d(u) = D0 + d1 u + d2 u^2 + d3 u^3 (D0 split exactly into J, f
// in FP64), and the two projection factors of the link,
//   F+(u) = -(T_l/2) (xi+ cos 2psi + xix sin 2psi),
//   Fx(u) = -(T_l/2) (xix cos 2psi - xi+ sin 2psi),
// so that z = F+ hdot+ + Fx hdotx (xi+ = (u.n)^2 - (v.n)^2, xix = 2 (u.n)(v.n),
// geometry at the retarded coordinate).  The factors are products of the
// composed T_l and n_l cubics, truncated at u^3 in FP64: over a group
// (|u| < 0.04) the dropped terms are below 1e-12 of the factors.
struct __align__(16) SerF32 {
    float f, d1, d2, d3;      // centre fraction, in-block delay variation (s)
    float Fp[4];              // F+(u) = Fp[0] + Fp[1] u + Fp[2] u^2 + Fp[3] u^3
    float Fc[4];              // Fx(u), same form
};

// Truncated product of two cubics: (a b) mod u^4.
__device__ __forceinline__ void cubic_mul(const double (&a)[4], const double (&b)[4], double (&c)[4])
{
    c[0] = a[0] * b[0];
    c[1] = a[0] * b[1] + a[1] * b[0];
    c[2] = a[0] * b[2] + a[1] * b[1] + a[2] * b[0];
    c[3] = a[0] * b[3] + a[1] * b[2] + a[2] * b[1] + a[3] * b[0];
}

// Staged window of one tile: hdot on samples [wlo, wlo + wlen) of the h grid
// (wlen = 0: not staged, stencils read global memory), built from h on
// [a0, a0 + nh) held in a planar buffer.
struct LfaWin {
    int64_t wlo, a0;
    int wlen, nh;
    int bulk;                 // filled by an asynchronous bulk copy
    int diff;                 // mixed form: the differenced window may be formed (interior, unit ratio)
    int jrel[6];              // mixed form: J_c - wlo - 15
};

// Shared memory of the FP64 form (one tile at a time).
struct LfaSmem64 {
    TileGeo g;
    double hb[2][kWinP];      // h+ and hx on the window
    double2 dw[kWinH];        // hdot window (interleaved pairs)
    double2 d3w[kWinH];       // NLO: third derivative of h on the window (pairs)
    double zs[6][kZW];
    LfaWin win;
    int64_t jends[12];
};

// FP64 set-up around the centre sample ic: the orbit geometry (Taylor shift
// of the segment polynomials) and, for the mixed form, the FP32 records of
// the six z series.  Every thread of the block must call it (it
// synchronises).
template <bool MIXED, class SM>
__device__ void lfa_tile_prologue(const LfaArgs& a, int64_t ic, SM& sm)
{
    TileGeo& g = sm.g;
    const int t = threadIdx.x;
    tile_geo_load(g, a.tab, ic, a.sky);
    if constexpr (MIXED) {
        const bool equal = (a.kind == LISA_LFA_EQUAL);
        const double u_per_s = 1.0 / (a.dt_out * 0.5 * a.tab.S);
        if (t < 36) {
            // series c, quantity r: 0 T_l, 1 k.R_s/c, 2 k.R_r/c, 3..5 n_l
            // composed with the retarded coordinate up(u) = u - sh(u)/(dt S/2):
            // r(up(u)) to cubic order by a Taylor shift to up(0) and the chain
            // rule (a1, a2, a3: the u, u^2, u^3 coefficients of up).
            const int c = t / 6, r = t % 6;
            const int ch = c >> 1, which = c & 1;
            const int l = a.gen == kLfaOwnTime ? c : lfa_link(ch, which);
            double sh[4] = {0.0, 0.0, 0.0, 0.0};
            if (a.gen != kLfaOwnTime) {
                const double al = which ? (a.gen == LISA_TDI20 ? 1.5 : 0.5) : (a.gen == LISA_TDI20 ? 2.0 : 1.0);
                const double be = which ? (a.gen == LISA_TDI20 ? 2.0 : 1.0) : (a.gen == LISA_TDI20 ? 1.5 : 0.5);
                const int ra = kQT + lfa_arm(ch, 0), rb = kQT + lfa_arm(ch, 1);
                for (int k = 0; k < 4; ++k)
                    sh[k] = equal ? (k == 0 ? (al + be) * a.Lc : 0.0) : al * g.b[ra][k] + be * g.b[rb][k];
            }
            const double a0 = -u_per_s * sh[0], a1 = 1.0 - u_per_s * sh[1], a2 = -u_per_s * sh[2],
                         a3 = -u_per_s * sh[3];
            double out[4];
            if (r == 0 && equal) {
                out[0] = a.Lc; out[1] = 0.0; out[2] = 0.0; out[3] = 0.0;
            } else {
                const int row = r == 0 ? kQT + l : r == 1 ? kRowKR + link_sender(l)
                              : r == 2 ? kRowKR + link_receiver(l) : kQN + 3 * l + (r - 3);
                double b[7];
                taylor_shift7(g.b[row], a0, b);
                out[0] = b[0];
                out[1] = b[1] * a1;
                out[2] = b[1] * a2 + b[2] * a1 * a1;
                out[3] = b[1] * a3 + 2.0 * b[2] * a1 * a2 + b[3] * a1 * a1 * a1;
            }
            for (int k = 0; k < 4; ++k) sm.comp[c][r][k] = out[k];
        }
        if (t == 40) {
            sm.inv_half = (float)(2.0 / a.tab.S);
            sm.inv_dt = (float)(1.0 / a.hm.dt_in);
            const double tc = a.t0_out + (double)ic * a.dt_out;
            sm.barg_c = (float)(a.bl.enabled ? a.bl.eps * (tc - a.bl.t_hyb) / a.bl.sigma : 0.0);
            sm.barg_d = (float)(a.bl.enabled ? a.bl.eps * a.dt_out / a.bl.sigma : 0.0);
        }
        if (t >= 64 && t < 64 + kRows) {
            const int r = t - 64;
            sm.c0[r] = (float)g.b[r][0];
            sm.cu[r] = tg_cubic(g, r);
        }
        __syncthreads();
        if (t < 6) {
            const int c = t, ch = c >> 1, which = c & 1;
            double sh[4] = {0.0, 0.0, 0.0, 0.0};
            if (a.gen != kLfaOwnTime) {
                const double al = which ? (a.gen == LISA_TDI20 ? 1.5 : 0.5) : (a.gen == LISA_TDI20 ? 2.0 : 1.0);
                const double be = which ? (a.gen == LISA_TDI20 ? 2.0 : 1.0) : (a.gen == LISA_TDI20 ? 1.5 : 0.5);
                const int ra = kQT + lfa_arm(ch, 0), rb = kQT + lfa_arm(ch, 1);
                for (int k = 0; k < 4; ++k)
                    sh[k] = equal ? (k == 0 ? (al + be) * a.Lc : 0.0) : al * g.b[ra][k] + be * g.b[rb][k];
            }
            // delay of the expansion point: central, or the sender / receiver end
            double d[4];
            for (int k = 0; k < 4; ++k)
                d[k] = a.kind == LISA_LFA_BACKWARD ? sh[k] + sm.comp[c][0][k] + sm.comp[c][1][k]
                     : a.kind == LISA_LFA_FORWARD ? sh[k] + sm.comp[c][2][k]
                     : sh[k] + 0.5 * (sm.comp[c][0][k] + sm.comp[c][1][k] + sm.comp[c][2][k]);
            int64_t j;
            double eps;
            split_f64(a.hm, ic, d[0], j, eps);
            SerF32& R = sm.ser[c];
            R.f = (float)eps;
            R.d1 = (float)d[1];
            R.d2 = (float)d[2];
            R.d3 = (float)d[3];
            // projection factors: (u.n), (v.n) cubics, then xi+, xix, times -T_l/2
            double un[4], vn[4], T[4];
            for (int k = 0; k < 4; ++k) {
                un[k] = a.sky.u[0] * sm.comp[c][3][k] + a.sky.u[1] * sm.comp[c][4][k] + a.sky.u[2] * sm.comp[c][5][k];
                vn[k] = a.sky.v[0] * sm.comp[c][3][k] + a.sky.v[1] * sm.comp[c][4][k] + a.sky.v[2] * sm.comp[c][5][k];
                T[k] = -0.5 * sm.comp[c][0][k];
            }
            double uu[4], vv[4], uv[4], xp[4], xc[4], gp[4], gc[4], Fp[4], Fc[4];
            cubic_mul(un, un, uu);
            cubic_mul(vn, vn, vv);
            cubic_mul(un, vn, uv);
            for (int k = 0; k < 4; ++k) {
                xp[k] = uu[k] - vv[k];
                xc[k] = 2.0 * uv[k];
                gp[k] = xp[k] * a.sky.c2p + xc[k] * a.sky.s2p;
                gc[k] = xc[k] * a.sky.c2p - xp[k] * a.sky.s2p;
            }
            cubic_mul(T, gp, Fp);
            cubic_mul(T, gc, Fc);
            for (int k = 0; k < 4; ++k) {
                R.Fp[k] = (float)Fp[k];
                R.Fc[k] = (float)Fc[k];
            }
            sm.J[c] = j;
        }
    }
    __syncthreads();
}

// Mixed form: retarded sample j (relative: jr = j - J) and fraction of series c
// at block offset dm = m - ic.
__device__ __forceinline__ void lfa_ser_locate(const LfaArgs& a, const SerF32& R, float inv_half, float inv_dt, int dm,
                                               int& jr, float& eps, float& u)
{
    u = (float)dm * inv_half;
    const float D = u * fmaf(u, fmaf(u, R.d3, R.d2), R.d1);
    int jp;
    float fp;
    if (a.hm.unit_rho) {
        jp = dm;
        fp = 0.f;
    } else {
        const double P = (double)dm * a.hm.rho;
        const double fl = floor(P);
        jp = (int)fl;
        fp = (float)(P - fl);
    }
    const float v = fmaf(-D, inv_dt, fp + R.f);
    const float fv = floorf(v);
    jr = jp + (int)fv;
    eps = v - fv;
}

__device__ __forceinline__ float cubic4(const float (&c)[4], float u)
{
    return fmaf(u, fmaf(u, fmaf(u, c[3], c[2]), c[1]), c[0]);
}

// hdot interpolated straight from global memory (stencils outside the staged
// window; kept out of line).
static __device__ __noinline__ float2 interp_hdot_global_ool(const float* __restrict__ hp, const float* __restrict__ hc,
                                                      int64_t n, int64_t j, float eps, float inv12dt)
{
    float p, q;
    interp_hdot_global<float>(hp, hc, n, j, eps, inv12dt, p, q);
    return make_float2(p, q);
}

// FP64 form: window of the tile starting at i0 (prologue centre ic): the
// retarded samples of the six series at the tile's two ends (2-sample halo
// included) bound the hdot window.  Every thread must call it (it
// synchronises twice).
__device__ inline void lfa_window(const LfaArgs& a, int64_t i0, int64_t ic, LfaSmem64& sm)
{
    const int t = threadIdx.x;
    const bool equal = (a.kind == LISA_LFA_EQUAL);
    if (t < 12) {
        const int c = t % 6;
        const int64_t m = (t < 6) ? i0 - 2 : i0 + kTile + 1;
        const TileGeo& g = sm.g;
        const double half = 0.5 * a.tab.S;
        const double u_per_s = 1.0 / (a.dt_out * half);
        const double u = (double)(m - ic) / half;
        const int ch = c >> 1, which = c & 1;
        const double Ta = equal ? a.Lc : tg_eval(g, kQT + lfa_arm(ch, 0), u);
        const double Tb = equal ? a.Lc : tg_eval(g, kQT + lfa_arm(ch, 1), u);
        const double sh = which ? lfa_shift(a.gen, Tb, Ta) : lfa_shift(a.gen, Ta, Tb);
        const int l = a.gen == kLfaOwnTime ? c : lfa_link(ch, which);
        const double up = u - sh * u_per_s;
        const double Tl = equal ? a.Lc : tg_eval(g, kQT + l, up);
        const double d = lfa_point_delay(a.kind, sh, Tl, tg_eval(g, kRowKR + link_sender(l), up),
                                         tg_eval(g, kRowKR + link_receiver(l), up));
        int64_t j;
        double eps;
        split_f64(a.hm, m, d, j, eps);
        sm.jends[t] = j;
    }
    __syncthreads();
    if (t == 0) {
        int64_t lo = sm.jends[0], hi = sm.jends[0];
        for (int k = 1; k < 12; ++k) {
            lo = sm.jends[k] < lo ? sm.jends[k] : lo;
            hi = sm.jends[k] > hi ? sm.jends[k] : hi;
        }
        LfaWin& w = sm.win;
        w.wlo = lo - 15 - 3;
        const int64_t len = (hi + 16 + 3) - w.wlo + 1;
        w.wlen = (len + 4 <= kWinH) ? (int)len : 0;
        // h needed on [wlo - 2, wlo + wlen + 2) for hdot, [wlo - 4, wlo + wlen + 4)
        // for the third derivative (NLO)
        w.bulk = 0;
        w.a0 = w.wlo - 4;
        w.nh = w.wlen > 0 ? w.wlen + 8 : 0;
    }
    __syncthreads();
}

// FP64 form: stage h on the window with plain loads (zero off the h grid),
// then form hdot (5-point central stencil).  Synchronises the block twice.
__device__ inline void lfa_stage_hdot(const LfaArgs& a, LfaSmem64& sm)
{
    const LfaWin& w = sm.win;
    const double* __restrict__ hp = (const double*)a.hp;
    const double* __restrict__ hc = (const double*)a.hc;
    for (int k = threadIdx.x; k < w.nh; k += blockDim.x) {
        const int64_t idx = w.a0 + k;
        const bool in = idx >= 0 && idx < a.hm.n_in;
        sm.hb[0][k] = in ? hp[idx] : 0.0;
        sm.hb[1][k] = in ? hc[idx] : 0.0;
    }
    __syncthreads();
    const double inv12dt = 1.0 / (12.0 * a.hm.dt_in);
    const double* P = sm.hb[0];   // P[q] = h+ at sample wlo - 4 + q
    const double* C = sm.hb[1];
    for (int k = threadIdx.x; k < w.wlen; k += blockDim.x) {
        const int64_t idx = w.wlo + k;
        const bool in = (idx >= 0 && idx < a.hm.n_in);
        double2 d;
        d.x = in ? ((P[k + 5] - P[k + 3]) * 8.0 - (P[k + 6] - P[k + 2])) * inv12dt : 0.0;
        d.y = in ? ((C[k + 5] - C[k + 3]) * 8.0 - (C[k + 6] - C[k + 2])) * inv12dt : 0.0;
        sm.dw[k] = d;
    }
    if (a.kind == LISA_LFA_NLO) {
        // third derivative: the 5-point second derivative of hdot (hdot zero
        // off the h grid), zero off the grid
        const double k2 = inv12dt / a.hm.dt_in;
        auto hd = [&](const double* X, int q) -> double {   // hdot at sample wlo - 4 + q
            const int64_t idx = w.wlo - 4 + q;
            if (idx < 0 || idx >= a.hm.n_in) return 0.0;
            return ((X[q + 1] - X[q - 1]) * 8.0 - (X[q + 2] - X[q - 2])) * inv12dt;
        };
        for (int k = threadIdx.x; k < w.wlen; k += blockDim.x) {
            const int64_t idx = w.wlo + k;
            double2 d = make_double2(0.0, 0.0);
            if (idx >= 0 && idx < a.hm.n_in) {
                d.x = (-hd(P, k + 2) + 16.0 * hd(P, k + 3) - 30.0 * hd(P, k + 4) + 16.0 * hd(P, k + 5) - hd(P, k + 6)) * k2;
                d.y = (-hd(C, k + 2) + 16.0 * hd(C, k + 3) - 30.0 * hd(C, k + 4) + 16.0 * hd(C, k + 5) - hd(C, k + 6)) * k2;
            }
            sm.d3w[k] = d;
        }
    }
    __syncthreads();
}

// Mixed form: block offset dm of an output sample -> block coordinate u and
// the sample's own position on the h grid (integer part jp, fraction fp).
__device__ __forceinline__ void lfa_sample_pos(const LfaArgs& a, float inv_half, int dm, float& u, int& jp, float& fp)
{
    u = (float)dm * inv_half;
    if (a.hm.unit_rho) {
        jp = dm;
        fp = 0.f;
    } else {
        const double P = (double)dm * a.hm.rho;
        const double fl = floor(P);
        jp = (int)fl;
        fp = (float)(P - fl);
    }
}

// Mixed form: z of series c at one sample (block coordinate u, own position
// jp + fp).  With the window staged (a decision uniform over the block) every
// stencil lies inside it: the retarded sample index is monotonic in the
// sample (|d delay/dt| << 1) and the window spans the indices at the tile's
// two ends plus margins; the clamp only keeps shared-memory reads in bounds.
// Without a window the stencils read global memory.
// STAGED: 1 = the window is staged (stencils from shared memory), 0 = global
// memory, -1 = decided here from W.wlen (a choice uniform over the block).
template <int STAGED = -1, class SM>
__device__ __forceinline__ float lfa_z_mixed(const LfaArgs& a, const SM& sm, const LfaWin& W, int c,
                                             float u, int jp, float fp)
{
    const float4* rp = reinterpret_cast<const float4*>(&sm.ser[c]);
    const float4 r0 = rp[0];   // f, d1, d2, d3
    const float D = u * fmaf(u, fmaf(u, r0.w, r0.z), r0.y);
    const float v = fmaf(-D, sm.inv_dt, fp + r0.x);
    const float fv = floorf(v);
    const int jr = jp + (int)fv;
    const float eps = v - fv;
    float dp, dc;
    if (STAGED == 1 || (STAGED < 0 && W.wlen > 0)) {
        const int base = min(max(W.jrel[c] + jr, 0), W.wlen - 32);
        lagrange32_dot2(eps, sm.dw + base, dp, dc);
    } else {
        const float2 r2 = interp_hdot_global_ool((const float*)a.hp, (const float*)a.hc, a.hm.n_in, sm.J[c] + jr, eps,
                                                 a.inv12dtf);
        dp = r2.x;
        dc = r2.y;
    }
    const float4 rp1 = rp[1], rp2 = rp[2];
    const float Fp = fmaf(u, fmaf(u, fmaf(u, rp1.w, rp1.z), rp1.y), rp1.x);
    const float Fc = fmaf(u, fmaf(u, fmaf(u, rp2.w, rp2.z), rp2.y), rp2.x);
    return fmaf(Fp, dp, Fc * dc);
}

// Mixed form, window staged: z of series c at two samples of the sub-block
// (block coordinates u.x, u.y; own positions jp + fp), the Lagrange weights of
// both formed together (lagrange32_dot2_pair).  Same arithmetic per sample as
// lfa_z_mixed<1>.  ADJ: the samples are adjacent, and where every lane's
// two stencils start one node apart (the common case on a unit-ratio grid)
// the warp reads the 33 values once for both.  Every lane of the warp must
// call it.
template <bool ADJ, class SM>
__device__ __forceinline__ float2 lfa_z_mixed_pair(const SM& sm, const LfaWin& W, int c, float2 u, int2 jp,
                                                   float2 fp)
{
    const float4* rp = reinterpret_cast<const float4*>(&sm.ser[c]);
    const float4 r0 = rp[0];   // f, d1, d2, d3
    const float Da = u.x * fmaf(u.x, fmaf(u.x, r0.w, r0.z), r0.y);
    const float Db = u.y * fmaf(u.y, fmaf(u.y, r0.w, r0.z), r0.y);
    const float va = fmaf(-Da, sm.inv_dt, fp.x + r0.x);
    const float vb = fmaf(-Db, sm.inv_dt, fp.y + r0.x);
    const float fa = floorf(va), fb = floorf(vb);
    const int ba = min(max(W.jrel[c] + jp.x + (int)fa, 0), W.wlen - 32);
    const int bb = min(max(W.jrel[c] + jp.y + (int)fb, 0), W.wlen - 32);
    float2 ha, hb;
    if (ADJ && __all_sync(0xffffffffu, bb == ba + 1))
        lagrange32_dot2_adjacent(make_float2(va - fa, vb - fb), sm.dw + ba, ha, hb);
    else
        lagrange32_dot2_pair(make_float2(va - fa, vb - fb), sm.dw + ba, sm.dw + bb, ha, hb);
    const float4 rp1 = rp[1], rp2 = rp[2];
    const float Fpa = fmaf(u.x, fmaf(u.x, fmaf(u.x, rp1.w, rp1.z), rp1.y), rp1.x);
    const float Fca = fmaf(u.x, fmaf(u.x, fmaf(u.x, rp2.w, rp2.z), rp2.y), rp2.x);
    const float Fpb = fmaf(u.y, fmaf(u.y, fmaf(u.y, rp1.w, rp1.z), rp1.y), rp1.x);
    const float Fcb = fmaf(u.y, fmaf(u.y, fmaf(u.y, rp2.w, rp2.z), rp2.y), rp2.x);
    return make_float2(fmaf(Fpa, ha.x, Fca * ha.y), fmaf(Fpb, hb.x, Fcb * hb.y));
}

// FP64 form: z values of the tile starting at i0 and its 2-sample halo (hdot
// in sm.dw).  Synchronises the block at the end.
__device__ inline void lfa_zvalues(const LfaArgs& a, int64_t i0, int64_t ic, LfaSmem64& sm)
{
    const double* __restrict__ hp = (const double*)a.hp;
    const double* __restrict__ hc = (const double*)a.hc;
    const TileGeo& g = sm.g;
    const int64_t wlo = sm.win.wlo;
    const int wlen = sm.win.wlen;
    const double half = 0.5 * a.tab.S;
    const double u_per_s = 1.0 / (a.dt_out * half);
    const bool equal = (a.kind == LISA_LFA_EQUAL);
    const double inv12dt = 1.0 / (12.0 * a.hm.dt_in);
    const double c2 = a.sky.c2p, s2 = a.sky.s2p;
    const double* ku = a.sky.u;
    const double* kv = a.sky.v;
    // On interior tiles no sample of the tile or its halo is off the grid.
    const bool interior = i0 - 2 >= 0 && i0 + kTile + 2 <= a.nout;
    for (int w = threadIdx.x; w < 6 * kZW; w += blockDim.x) {
        const int c = w / kZW, o = w % kZW;
        const int64_t m = i0 - 2 + o;
        double zval = 0.0;
        if (interior || (m >= 0 && m < a.nout)) {
            const int ch = c >> 1, which = c & 1;
            const int l = a.gen == kLfaOwnTime ? c : lfa_link(ch, which);
            const double u = (double)(m - ic) / half;
            const double Ta = equal ? a.Lc : tg_eval(g, kQT + lfa_arm(ch, 0), u);
            const double Tb = equal ? a.Lc : tg_eval(g, kQT + lfa_arm(ch, 1), u);
            const double sh = which ? lfa_shift(a.gen, Tb, Ta) : lfa_shift(a.gen, Ta, Tb);
            const double up = u - sh * u_per_s;
            const double Tl = equal ? a.Lc : tg_eval(g, kQT + l, up);
            const double dtau = lfa_point_delay(a.kind, sh, Tl, tg_eval(g, kRowKR + link_sender(l), up),
                                                tg_eval(g, kRowKR + link_receiver(l), up));
            double n3[3];
            for (int q = 0; q < 3; ++q) n3[q] = tg_eval(g, kQN + 3 * l + q, up);
            int64_t j;
            double eps;
            split_f64(a.hm, m, dtau, j, eps);
            const double un = ku[0] * n3[0] + ku[1] * n3[1] + ku[2] * n3[2];
            const double vn = kv[0] * n3[0] + kv[1] * n3[1] + kv[2] * n3[2];
            const double xp = un * un - vn * vn, xc = 2.0 * un * vn;
            double dp, dc;
            bool ok;
            dp = interp_pair_w<double>(sm.dw, wlo, wlen, nullptr, j, eps, dc, ok);
            if (!ok) interp_hdot_global<double>(hp, hc, a.hm.n_in, j, eps, inv12dt, dp, dc);
            if (a.kind == LISA_LFA_NLO) {
                const double kn = a.sky.k[0] * n3[0] + a.sky.k[1] * n3[1] + a.sky.k[2] * n3[2];
                const double kap = nlo_kappa<double>(Tl, kn, a.gen == kLfaOwnTime);
                double tp, tc;
                bool ok3;
                tp = interp_pair_w<double>(sm.d3w, wlo, wlen, nullptr, j, eps, tc, ok3);
                if (!ok3) {
                    tp = tc = 0.0;
                    double w32[32];
                    lagrange32_weights(eps, w32);
                    const double idt = 1.0 / a.hm.dt_in;
                    if (eps == 0.0) {
                        tp = hthird_global<double>(hp, a.hm.n_in, j, inv12dt, idt);
                        tc = hthird_global<double>(hc, a.hm.n_in, j, inv12dt, idt);
                    } else {
                        for (int k = 0; k < 32; ++k) {
                            tp = fma(w32[k], hthird_global<double>(hp, a.hm.n_in, j - 15 + k, inv12dt, idt), tp);
                            tc = fma(w32[k], hthird_global<double>(hc, a.hm.n_in, j - 15 + k, inv12dt, idt), tc);
                        }
                    }
                }
                dp = fma(kap, tp, dp);
                dc = fma(kap, tc, dc);
            }
            zval = -0.5 * Tl * (dp * (xp * c2 + xc * s2) + dc * (xc * c2 - xp * s2));
        }
        sm.zs[c][o] = zval;
    }
    __syncthreads();
}

// Next term of the Michelson expansions (kind NLO): about its centre the l =
// +-2 part of X1.5 is (1 + D_Tb)(1 - D_2Ta) y = 4 T_a [d/dt + (T_a^2/6 +
// T_b^2/8) d3/dt3] y, and of X2.0 (1 + D_Tb)(1 - D_2Ta)(1 - D_2(Ta+Tb)) y =
// 8 T_a (T_a + T_b) [d2/dt2 + (T_b^2/8 + T_a^2/6 + (T_a + T_b)^2/6) d4/dt4] y
// (D_x: delay by x; the l = +-3 part alike with a <-> b).  z[0..4] = z at
// i-2 .. i+2; third and fourth derivatives by 5-point stencils.
template <typename Real>
__device__ __forceinline__ Real lfa_nlo_channel15(Real Ta, Real Tb, const Real* za, const Real* zb, double dt)
{
    const Real k3 = Real(1) / (Real(2) * Real(dt) * Real(dt) * Real(dt));
    auto d3 = [&](const Real* z) { return ((z[4] - z[0]) - Real(2) * (z[3] - z[1])) * k3; };
    const Real ka = Ta * Ta / Real(6) + Tb * Tb / Real(8), kb = Tb * Tb / Real(6) + Ta * Ta / Real(8);
    return Real(4) * (Ta * ka * d3(za) - Tb * kb * d3(zb));
}

template <typename Real>
__device__ __forceinline__ Real lfa_nlo_channel20(Real Ta, Real Tb, const Real* za, const Real* zb, double dt)
{
    const Real k4 = Real(1) / (Real(dt) * Real(dt) * Real(dt) * Real(dt));
    auto d4 = [&](const Real* z) { return ((z[0] + z[4]) - Real(4) * (z[1] + z[3]) + Real(6) * z[2]) * k4; };
    const Real s = (Ta + Tb) * (Ta + Tb) / Real(6);
    const Real ka = Tb * Tb / Real(8) + Ta * Ta / Real(6) + s, kb = Ta * Ta / Real(8) + Tb * Tb / Real(6) + s;
    return Real(8) * (Ta + Tb) * (Ta * ka * d4(za) - Tb * kb * d4(zb));
}

// FP64 form: channels of sample i0 + t from the z values in shared memory (and
// z stored if requested).
__device__ inline void lfa_channels(const LfaArgs& a, int64_t i0, int64_t ic, const LfaSmem64& sm, double (&X)[3])
{
    const TileGeo& g = sm.g;
    const int t = threadIdx.x;
    const bool equal = (a.kind == LISA_LFA_EQUAL);
    const double half = 0.5 * a.tab.S;
    const int64_t i = i0 + t;
    if (a.z && i >= a.i_begin && i < a.i_end) {
        double* zo = (double*)a.z;
        for (int c = 0; c < 6; ++c) zo[(int64_t)c * a.nout + i] = sm.zs[c][t + 2];
    }
    const double k1 = 1.0 / (12.0 * a.dt_out);   // 1/(12 dt)
    const double k2 = k1 / a.dt_out;             // 1/(12 dt^2)
    const double u = (double)(i - ic) / half;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const double Ta = equal ? a.Lc : tg_eval(g, kQT + lfa_arm(ch, 0), u);
        const double Tb = equal ? a.Lc : tg_eval(g, kQT + lfa_arm(ch, 1), u);
        const double* za = sm.zs[2 * ch] + t;       // za[0..4] = z at i-2..i+2
        const double* zb = sm.zs[2 * ch + 1] + t;
        if (a.gen == LISA_TDI20) {
            // 5-point second derivative as (14 d2_0 - d2_-1 - d2_1)/12, d2 from first differences
            auto d2 = [&](const double* z) {
                const double e0 = z[1] - z[0], e1 = z[2] - z[1], e2 = z[3] - z[2], e3 = z[4] - z[3];
                const double m1 = e1 - e0, c0 = e2 - e1, p1 = e3 - e2;
                return (14.0 * c0 - m1 - p1) * k2;
            };
            X[ch] = 8.0 * (Ta + Tb) * (Ta * d2(za) - Tb * d2(zb));
            if (a.kind == LISA_LFA_NLO) X[ch] += lfa_nlo_channel20<double>(Ta, Tb, za, zb, a.dt_out);
        } else {
            auto d1 = [&](const double* z) { return ((z[3] - z[1]) * 8.0 - (z[4] - z[0])) * k1; };
            X[ch] = 4.0 * (Ta * d1(za) - Tb * d1(zb));
            if (a.kind == LISA_LFA_NLO) X[ch] += lfa_nlo_channel15<double>(Ta, Tb, za, zb, a.dt_out);
        }
    }
}

// FP64 form: one tile [i0, i0 + kTile) after lfa_tile_prologue at the centre
// ic: on return thread t holds X, Y, Z of sample i0 + t (before AET, blend
// and store) and z has been written if requested.  Every thread of the
// block must call it.
__device__ inline void lfa_tile_body(const LfaArgs& a, int64_t i0, int64_t ic, LfaSmem64& sm, double (&X)[3])
{
    __syncthreads();   // the previous tile's readers of the shared buffers are done
    lfa_window(a, i0, ic, sm);
    lfa_stage_hdot(a, sm);
    lfa_zvalues(a, i0, ic, sm);
    lfa_channels(a, i0, ic, sm, X);
}

// Tiles per CTA (mixed form): the FP64 prologue (segment polynomials shifted
// to the centre, the series' composed cubics) is shared by up to 8
// consecutive tiles, as many as keep the block's half-span within 1.1e4 s:
// the omitted quartic terms of the cubics (k.R/c: 500 s at the orbital
// frequency) then stay below 4e-10 s, a phase error under 1e-10 rad at
// 2e-2 Hz.
inline int lfa_group(double dt)
{
    int G = (int)floor(80.0 / dt);
    return G < 1 ? 1 : (G > 8 ? 8 : G);
}

// Tiles per CTA of the mixed LFA kernel in a single call: at most 6 (the
// last wave of CTAs ends sooner; on one year at 5 s the kernel took 0.513,
// 0.547 and 0.488 ms with groups of 8, 7 and 6 tiles).  The batched plan keeps
// lfa_group: its work items are autotuned runs of groups.
inline int lfa_group_mixed(double dt)
{
    const int G = lfa_group(dt);
    return G < 6 ? G : 6;
}

// Tiles per CTA of the double-float kernel: at most 6 (its groups take ~0.3 ms
// each, so smaller groups shorten the last wave of CTAs more than their
// prologues cost; on one year at 5 s, 24,644 tiles at 3 CTAs per SM, groups of
// 8, 7, 6 and 5 tiles gave 2.254, 2.174, 2.155 and 2.168 ms).
inline int lfa_group_df(double dt)
{
    const int G = lfa_group(dt);
    return G < 6 ? G : 6;
}

// ---------------------------------------------------------------------------
// Mixed form in sub-blocks of two tiles (the LFA kernel).
//
// A CTA's group of tiles shares one FP64 prologue; its tiles are processed two
// at a time, each thread computing the samples i0 + t and i0 + kTile + t.  The
// windows of every sub-block are located in the prologue, the h window of
// sub-block q + 1 is fetched by bulk copies while q is computed, and a
// sub-block costs three block barriers (copy landed, hdot formed, z formed)
// for 512 samples.
// ---------------------------------------------------------------------------
constexpr int kSub2 = 2 * kTile;          // samples per sub-block
constexpr int kWin2 = kSub2 + 384;        // hdot window of a sub-block
constexpr int kWinP2 = kWin2 + 16;        // planar h buffers: 4-sample margins and 16-byte alignment slack
constexpr int kZW2 = kSub2 + 4;           // z of a sub-block and its 2-sample halos
constexpr int kMaxSub2 = 4;               // sub-blocks per group (groups of up to 8 tiles)

struct Lfa2Smem {
    TileGeo g;
    alignas(16) float hb[2][2][kWinP2];   // h+ and hx windows, two buffers
    float2 dw[kWin2];                     // hdot window, or the differenced window S (interleaved pairs)
    float2 qw[kWin2];                     // differenced form: the B-term differences Q (interleaved pairs)
    union {
        float zs[6][kZW2];                // z values of a sub-block (z-series form)
        float4 d2[kWin2 + 8];             // second differences of h as (hi, lo) pairs (differenced form)
        float xacc[12][kTile];            // differenced form: channel sums of a thread's two samples (rows 0-5), the three arms' light times at them (rows 6-11)
    };
    LfaWin win[kMaxSub2];
    uint64_t bar[2];                      // completion barriers of the bulk copies
    int64_t jends[kMaxSub2][12];
    SerF32 ser[6];
    int64_t J[6];
    double comp[6][6][4];
    float c0[kRows];
    Cubic cu[kRows];
    float inv_half, inv_dt;
    float barg_c, barg_d;
    unsigned int smooth[3];               // differenced form: window maxima of |D3 h|, |D7 h|, |h| (float bits)
};

// Windows of the nsb sub-blocks starting at tile t0 (after the prologue at
// the group centre ic).  Every thread must call it (it synchronises twice).
static __device__ void lfa2_windows(const LfaArgs& a, int64_t t0, int nsb, int64_t ic, Lfa2Smem& sm)
{
    const int t = threadIdx.x;
    if (t < 12 * nsb) {
        const int sb = t / 12, k = t % 12, c = k % 6;
        const int64_t i0 = (t0 + 2 * sb) * (int64_t)kTile;
        const int64_t m = (k < 6) ? i0 - 2 : i0 + kSub2 + 1;
        int jr;
        float eps, u;
        lfa_ser_locate(a, sm.ser[c], sm.inv_half, sm.inv_dt, (int)(m - ic), jr, eps, u);
        sm.jends[sb][k] = sm.J[c] + jr;
    }
    __syncthreads();
    if (t < nsb) {
        int64_t lo = sm.jends[t][0], hi = sm.jends[t][0];
        for (int k = 1; k < 12; ++k) {
            lo = sm.jends[t][k] < lo ? sm.jends[t][k] : lo;
            hi = sm.jends[t][k] > hi ? sm.jends[t][k] : hi;
        }
        LfaWin& w = sm.win[t];
        w.wlo = lo - 15 - 3;
        const int64_t len = (hi + 16 + 3) - w.wlo + 1;
        w.wlen = (len + 4 <= kWin2) ? (int)len : 0;
        // h on [wlo - 4, wlo + wlen + 4): the 5-point hdot needs 2 samples each
        // side, the differenced window (9-point composite stencils) 4
        const int64_t s0 = w.wlo - 4, s1 = w.wlo + w.wlen + 4;
        const int64_t a0 = s0 - (((s0 % 4) + 4) % 4);
        const int64_t a1 = s1 + (((4 - s1 % 4) % 4 + 4) % 4);
        const bool bulk = a.h_aligned && w.wlen > 0 && a0 >= 0 && a1 <= a.hm.n_in && a1 - a0 <= kWinP2;
        w.bulk = bulk ? 1 : 0;
        w.a0 = bulk ? a0 : s0;
        w.nh = bulk ? (int)(a1 - a0) : (w.wlen > 0 ? w.wlen + 8 : 0);
        // differenced form: the composite stencils and B-term differences of
        // every staged element stay inside the h grid (no zero padding)
        w.diff = a.hm.unit_rho && a.gen != kLfaOwnTime && a.kind != LISA_LFA_NLO && !a.z && w.wlen > 0 && s0 >= 0 &&
                 s1 <= a.hm.n_in;
        for (int c = 0; c < 6; ++c) w.jrel[c] = w.wlen ? (int)(sm.J[c] - w.wlo) - 15 : 0;
    }
    __syncthreads();
}

// Stage the h window of sub-block sb into buffer b: bulk copies issued by
// thread 0 (completing on sm.bar[b]) or plain loads by every thread.
static __device__ void lfa2_stage(const LfaArgs& a, Lfa2Smem& sm, int sb, int b)
{
    const LfaWin& w = sm.win[sb];
    const float* __restrict__ hp = (const float*)a.hp;
    const float* __restrict__ hc = (const float*)a.hc;
    if (w.bulk) {
        if (threadIdx.x == 0) {
            const uint32_t bytes = (uint32_t)w.nh * (uint32_t)sizeof(float);
            mbar_arrive_expect_tx(&sm.bar[b], 2u * bytes);
            bulk_copy_g2s(sm.hb[b][0], hp + w.a0, bytes, &sm.bar[b]);
            bulk_copy_g2s(sm.hb[b][1], hc + w.a0, bytes, &sm.bar[b]);
        }
    } else {
        for (int k = threadIdx.x; k < w.nh; k += blockDim.x) {
            const int64_t idx = w.a0 + k;
            const bool in = idx >= 0 && idx < a.hm.n_in;
            sm.hb[b][0][k] = in ? hp[idx] : 0.f;
            sm.hb[b][1][k] = in ? hc[idx] : 0.f;
        }
    }
}

// ---------------------------------------------------------------------------
// Differenced form of the mixed LFA channels (unit grid ratio, interior
// sub-blocks).
//
// The TDI 2.0 channel takes the 5-point second difference of each z series
// on the output grid, sum_k c_k z(t_{i+k}) with c = (-1, 16, -30, 16, -1)
// (TDI 1.5: the first difference, d = (1, -8, 0, 8, -1)), and that difference
// cancels to O((omega dt)^2) of z.  Formed from FP32-rounded z values, FP32
// rounding is amplified by 1/(omega dt)^2.  Here the cancellation happens on
// the exact FP32 inputs instead.  With z_i = F(t_i) I(x_i), I the 32-point
// interpolant of hdot and x_i the retarded position of sample i on the h grid
// (x_{i+k} = x_i + k (1 + a1) + a2 k^2 + O(k^3), a1, a2 from the series'
// delay cubic), Taylor expansion in the small drift a1 ~ v/c and in the
// orbital variation of F gives, for TDI 2.0,
//   sum_k c_k z_{i+k} = (1 + a1)^2 F_i sum_p w_p(eps_i) S[J_i + p]
//                       + 24 (F1 + F a2) I'(x_i) + R,
//   S[m] = sum_k c_k hdot[m + k]   (a fixed 9-point stencil of h),
// with F1 = dF/di and I' = dI/dx.  The dropped terms R are O(a1 (omega dt)^4)
// ~ 1e-8, O(F'' ) ~ 1e-12 and O(a2 / (omega dt)) ~ 3e-8 of the first term
// (the second is itself below 1e-3 of it).  For TDI 1.5:
//   sum_k d_k z_{i+k} = (1 + a1) F_i sum_p w_p S1[J_i + p] + 12 F1 I(x_i) + R.
// S is formed on the staged window from third (TDI 1.5: second) differences
// of h with their rounding errors carried (two-sum): it is then exact to
// FP32 rounding of itself, so the interpolated sum keeps FP32 relative
// accuracy however small S is next to h.  The B-term (24 (F1 + F a2) I') needs
// ~1e-3 relative accuracy only (it is at most ~1e-3 of the first term for f
// >= 1e-4 Hz): I' is taken from the centred second difference Q of h at the
// two nodes around x (I' ~ Q / dt; TDI 1.5: I ~ Q1 / dt with Q1 the half
// central difference), interpolated linearly.
// ---------------------------------------------------------------------------

// |Seventh difference of h| from six consecutive second differences v[0..5]
// (their fifth difference), the larger of the two polarisations (value parts
// .x, .z).
__device__ __forceinline__ float lfa_d7_first(const float4 (&v)[7])
{
    const float p = (v[5].x - v[0].x) - 5.f * (v[4].x - v[1].x) + 10.f * (v[3].x - v[2].x);
    const float c = (v[5].z - v[0].z) - 5.f * (v[4].z - v[1].z) + 10.f * (v[3].z - v[2].z);
    return fmaxf(fabsf(p), fabsf(c));
}

// a - b split into its rounded value and exact error (two-sum).
__device__ __forceinline__ float2 two_diff(float a, float b)
{
    const float s = __fsub_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(-b, bb));
    return make_float2(s, e);
}

// Second difference h[n+2] - 2 h[n+1] + h[n] as (value, error) pairs whose
// sum is exact but for the final addition of the error parts.
__device__ __forceinline__ float2 second_diff_pair(const float* P, int n)
{
    const float2 d0 = two_diff(P[n + 1], P[n]);
    const float2 d1 = two_diff(P[n + 2], P[n + 1]);
    const float2 dd = two_diff(d1.x, d0.x);
    return make_float2(dd.x, __fadd_rn(dd.y, __fsub_rn(d1.y, d0.y)));
}

// Differenced window of a sub-block: S (TDI 2.0: sum_k c_k hdot[m+k]; TDI
// 1.5: sum_k d_k hdot[m+k]) as interleaved pairs in sm.dw and the B-term
// differences Q in sm.qw, for the window samples m = wlo .. wlo + wlen - 1
// (P, C: h+, hx with P[q] at sample wlo - 4 + q).  With hdot = D1 h / (12 dt),
// S = C(z) D(z) h / (12 dt): the composite polynomial is
//   z^-4 (z - 1)^3 G(z),   G = (z + 1)(z^2 - 14 z + 1)(z^2 - 8 z + 1)
//                            = 1 - 21 z + 92 z^2 + 92 z^3 - 21 z^4 + z^5
// for TDI 2.0, and z^-4 (z - 1)^2 G1(z), G1 = (z + 1)^2 (z^2 - 8 z + 1)^2 =
// 1 - 14 z + 35 z^2 + 100 z^3 + 35 z^4 - 14 z^5 + z^6 for TDI 1.5.
// Synchronises twice.
static __device__ bool lfa2_diff_window(const LfaArgs& a, Lfa2Smem& sm, const LfaWin& w, const float* P,
                                        const float* C)
{
    const int wlen = w.wlen;
    if (threadIdx.x < 3) sm.smooth[threadIdx.x] = 0u;
    // pass 1: second differences with their errors, d2[n] for the samples
    // wlo - 4 + n .. wlo - 2 + n, n = 0 .. wlen + 5
    for (int n = threadIdx.x; n < wlen + 6; n += blockDim.x) {
        const float2 p = second_diff_pair(P, n), c = second_diff_pair(C, n);
        sm.d2[n] = make_float4(p.x, p.y, c.x, c.y);
    }
    __syncthreads();
    float m3 = 0.f, m7 = 0.f, mh = 0.f;   // smoothness indicator of the window (below)
    const float inv12dt = a.inv12dtf;
    const bool tdi20 = a.gen == LISA_TDI20;
    for (int k = threadIdx.x; k < wlen; k += blockDim.x) {
        float4 v[7];
#pragma unroll
        for (int j = 0; j < 7; ++j) v[j] = sm.d2[k + j];
        float2 S;
        if (tdi20) {
            // third differences (of the value and the error parts separately:
            // adjacent second differences are within a factor two of each other
            // away from their zeros, so the value difference is exact there)
            constexpr float g[6] = {1.f, -21.f, 92.f, 92.f, -21.f, 1.f};
            float sp = 0.f, ep = 0.f, sc = 0.f, ec = 0.f;
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                sp = fmaf(g[j], __fsub_rn(v[j + 1].x, v[j].x), sp);
                ep = fmaf(g[j], __fsub_rn(v[j + 1].y, v[j].y), ep);
                sc = fmaf(g[j], __fsub_rn(v[j + 1].z, v[j].z), sc);
                ec = fmaf(g[j], __fsub_rn(v[j + 1].w, v[j].w), ec);
            }
            S = make_float2((sp + ep) * inv12dt, (sc + ec) * inv12dt);
            // Q: centred second difference at m = d2[k + 3]
            sm.qw[k] = make_float2(v[3].x + v[3].y, v[3].z + v[3].w);
            // third and seventh differences of h starting at the element's first
            // second difference (value parts): over the window's elements they
            // cover every start once
            m3 = fmaxf(m3, fmaxf(fabsf(v[1].x - v[0].x), fabsf(v[1].z - v[0].z)));
            m7 = fmaxf(m7, lfa_d7_first(v));
            mh = fmaxf(mh, fmaxf(fabsf(P[k + 4]), fabsf(C[k + 4])));
        } else {
            constexpr float g1[7] = {1.f, -14.f, 35.f, 100.f, 35.f, -14.f, 1.f};
            float sp = 0.f, ep = 0.f, sc = 0.f, ec = 0.f;
#pragma unroll
            for (int j = 0; j < 7; ++j) {
                sp = fmaf(g1[j], v[j].x, sp);
                ep = fmaf(g1[j], v[j].y, ep);
                sc = fmaf(g1[j], v[j].z, sc);
                ec = fmaf(g1[j], v[j].w, ec);
            }
            S = make_float2((sp + ep) * inv12dt, (sc + ec) * inv12dt);
            // Q1: half central difference at m
            sm.qw[k] = make_float2(0.5f * (P[k + 5] - P[k + 3]), 0.5f * (C[k + 5] - C[k + 3]));
            m3 = fmaxf(m3, fmaxf(fabsf(v[1].x - v[0].x), fabsf(v[1].z - v[0].z)));
            m7 = fmaxf(m7, lfa_d7_first(v));
            mh = fmaxf(mh, fmaxf(fabsf(P[k + 4]), fabsf(C[k + 4])));
        }
        sm.dw[k] = S;
    }
    // Smoothness test.  The drift terms of the expansion are exact for h
    // smooth on the stencil scale; their error is ~ a1 times a functional
    // of the interpolant that vanishes on quintics, which the seventh
    // difference of h bounds.  Measured on chirps, ringdowns and an h with a
    // jump in its derivative (FP64 emulation): error / output ~ 1e-10 at
    // D7/D3 ~ 1e-6 (inspiral), 1e-8 at 2e-3 (ringdown at 0.2 rad per
    // sample), 4e-5 at 9 (the derivative jump).  The form is kept where
    // |a1| D7 <= 2.5e-6 D3 (D7/D3 <= 0.025 at a1 = 1e-4), plus the FP32
    // rounding of h itself, which the seventh difference amplifies
    // ~60-fold (allowance 300 ulp of the window's largest |h|: the drift
    // terms carry it at a1 times the noise, as the exact form does).
    // Otherwise the sub-block falls back to the z-series form.
    const unsigned int lane = threadIdx.x & 31u;
    const unsigned int b3 = __reduce_max_sync(0xffffffffu, __float_as_uint(m3));
    const unsigned int b7 = __reduce_max_sync(0xffffffffu, __float_as_uint(m7));
    const unsigned int bh = __reduce_max_sync(0xffffffffu, __float_as_uint(mh));
    if (lane == 0) {
        atomicMax(&sm.smooth[0], b3);
        atomicMax(&sm.smooth[1], b7);
        atomicMax(&sm.smooth[2], bh);
    }
    __syncthreads();
    float a1max = 0.f;
    for (int c = 0; c < 6; ++c) {
        const SerF32& R = sm.ser[c];
        a1max = fmaxf(a1max, fabsf(R.d1) + 2.f * fabsf(R.d2) + 3.f * fabsf(R.d3));
    }
    a1max *= sm.inv_half * sm.inv_dt;   // |u| <= 1 over a group
    const float M3 = __uint_as_float(sm.smooth[0]), M7 = __uint_as_float(sm.smooth[1]);
    const float H = __uint_as_float(sm.smooth[2]);
    return a1max * M7 <= 2.5e-6f * M3 + a1max * 300.f * 5.9604645e-8f * H;
}

// Wait for buffer b (bounded for bulk copies), then form the window of
// sub-block sb: with dpath, the differenced window (lfa2_diff_window), kept
// if the window passes its smoothness test (returns 1); otherwise hdot in
// sm.dw for the z-series form (returns 0).  Synchronises two to four times.
// Returns -1 (for every thread) if a wait timed out: the status word is
// flagged after a second bounded wait for the copy to land, and the block
// must stop.
static __device__ int lfa2_wait_hdot(const LfaArgs& a, Lfa2Smem& sm, int sb, int b, uint32_t parity, bool dpath)
{
    const LfaWin& w = sm.win[sb];
    bool ok = true;
    if (w.bulk) ok = mbar_wait_bounded(&sm.bar[b], parity);
    if (__syncthreads_or(ok ? 0 : 1)) {
        if (threadIdx.x == 0) flag_timeout(a.status);
        if (w.bulk) mbar_wait_bounded(&sm.bar[b], parity);
        return -1;
    }
    const int off = (int)(w.wlo - 4 - w.a0);
    const float* P = sm.hb[b][0] + off;   // P[q] = h+ at sample wlo - 4 + q
    const float* C = sm.hb[b][1] + off;
    const float inv12dt = a.inv12dtf;
    if (dpath && lfa2_diff_window(a, sm, w, P, C)) return 1;   // (the decision is uniform over the block)
    for (int k = threadIdx.x; k < w.wlen; k += blockDim.x) {
        const int64_t idx = w.wlo + k;
        const bool in = (idx >= 0 && idx < a.hm.n_in);
        float2 d;
        d.x = in ? ((P[k + 5] - P[k + 3]) * 8.f - (P[k + 6] - P[k + 2])) * inv12dt : 0.f;
        d.y = in ? ((C[k + 5] - C[k + 3]) * 8.f - (C[k + 6] - C[k + 2])) * inv12dt : 0.f;
        sm.dw[k] = d;
    }
    __syncthreads();
    return 0;
}

// z of sub-block sb starting at sample i0: the 2 x kTile new values per
// series (offsets 4 + t and 4 + kTile + t), and on the group's first
// sub-block also the leading halo (offsets 0..3); later sub-blocks take it
// from the previous one (copied by the caller).  Synchronises at the end.
static __device__ void lfa2_zvalues(const LfaArgs& a, int64_t i0, int64_t ic, Lfa2Smem& sm, int sb, bool first)
{
    const LfaWin& W = sm.win[sb];
    const int t = threadIdx.x;
    const int dmt = (int)(i0 - ic);
    const bool interior = i0 - 2 >= 0 && i0 + kSub2 + 2 <= a.nout;
    if (first && t < 24) {
        const int c = t >> 2, o = t & 3;
        const int64_t m = i0 - 2 + o;
        float u, fp;
        int jp;
        lfa_sample_pos(a, sm.inv_half, dmt - 2 + o, u, jp, fp);
        const float z = lfa_z_mixed(a, sm, W, c, u, jp, fp);
        sm.zs[c][o] = (interior || (m >= 0 && m < a.nout)) ? z : 0.f;
    }
#if LISA_LFA_PAIR
    if (W.wlen > 0) {
        // window staged: the thread's two samples together
        // LISA_LFA_PAIR 2: adjacent samples 2t, 2t + 1; 1: samples t, kTile + t
        const int o0 = LISA_LFA_PAIR == 2 ? 4 + 2 * t : 4 + t;
        const int o1 = LISA_LFA_PAIR == 2 ? o0 + 1 : 4 + kTile + t;
        const bool v0 = interior || (i0 - 2 + o0 >= 0 && i0 - 2 + o0 < a.nout);
        const bool v1 = interior || (i0 - 2 + o1 >= 0 && i0 - 2 + o1 < a.nout);
        float2 u, fp;
        int2 jp;
        lfa_sample_pos(a, sm.inv_half, dmt - 2 + o0, u.x, jp.x, fp.x);
        lfa_sample_pos(a, sm.inv_half, dmt - 2 + o1, u.y, jp.y, fp.y);
#pragma unroll kLfaUnroll
        for (int c = 0; c < 6; ++c) {
            const float2 z = lfa_z_mixed_pair<LISA_LFA_PAIR == 2>(sm, W, c, u, jp, fp);
            sm.zs[c][o0] = v0 ? z.x : 0.f;
            sm.zs[c][o1] = v1 ? z.y : 0.f;
        }
        __syncthreads();
        return;
    }
#endif
    // the staged / global choice is uniform over the block: one loop each
    auto run = [&](auto staged) {
        constexpr int S = decltype(staged)::value;
#pragma unroll 1
        for (int r = 0; r < 2; ++r) {
            const int o = 4 + r * kTile + t;
            const int64_t m = i0 - 2 + o;
            const bool valid = interior || (m >= 0 && m < a.nout);
            float u, fp;
            int jp;
            lfa_sample_pos(a, sm.inv_half, dmt - 2 + o, u, jp, fp);
#pragma unroll kLfaUnroll
            for (int c = 0; c < 6; ++c) {
                const float z = lfa_z_mixed<S>(a, sm, W, c, u, jp, fp);
                sm.zs[c][o] = valid ? z : 0.f;
            }
        }
    };
    if (W.wlen > 0) run(std::integral_constant<int, 1>{});
    else run(std::integral_constant<int, 0>{});
    __syncthreads();
}

// Channels of sample i0 + r kTile + t from the z values of its sub-block.
__device__ __forceinline__ void lfa2_channels(const LfaArgs& a, int64_t i0, int64_t ic, const Lfa2Smem& sm, int r,
                                              float (&X)[3])
{
    const int t = threadIdx.x;
    const bool equal = (a.kind == LISA_LFA_EQUAL);
    const int o = r * kTile + t;               // zs[c][o .. o + 4] = z at i - 2 .. i + 2
    const int64_t i = i0 + o;
    if (a.z && i >= a.i_begin && i < a.i_end) {
        float* zo = (float*)a.z;
        for (int c = 0; c < 6; ++c) zo[(int64_t)c * a.nout + i] = sm.zs[c][o + 2];
    }
    const float k1 = a.c1f, k2 = a.c2f;
    const float u = (float)(int)(i - ic) * sm.inv_half;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const float Ta = equal ? a.Lcf : sm.c0[kQT + lfa_arm(ch, 0)] + sm.cu[kQT + lfa_arm(ch, 0)](u);
        const float Tb = equal ? a.Lcf : sm.c0[kQT + lfa_arm(ch, 1)] + sm.cu[kQT + lfa_arm(ch, 1)](u);
        const float* za = sm.zs[2 * ch] + o;
        const float* zb = sm.zs[2 * ch + 1] + o;
        if (a.gen == LISA_TDI20) {
            auto d2 = [&](const float* z) {
                const float e0 = z[1] - z[0], e1 = z[2] - z[1], e2 = z[3] - z[2], e3 = z[4] - z[3];
                const float m1 = e1 - e0, c0 = e2 - e1, p1 = e3 - e2;
                return (14.f * c0 - m1 - p1) * k2;
            };
            X[ch] = 8.f * (Ta + Tb) * (Ta * d2(za) - Tb * d2(zb));
        } else {
            auto d1 = [&](const float* z) { return ((z[3] - z[1]) * 8.f - (z[4] - z[0])) * k1; };
            X[ch] = 4.f * (Ta * d1(za) - Tb * d1(zb));
        }
    }
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
        if constexpr (sizeof(Real) == 4) {
            // below -17.5 the weight 1 / (1 + e^arg) rounds to 1 in FP32 (e^arg < 2^-24):
            // skipped, bit for bit the same
            const float ar = fmaf((float)di, barg_d, barg_c);
            if (ar > -17.5f) {
                const float wgt = 1.f / (1.f + expf(ar));
                o0 *= wgt;
                o1 *= wgt;
                o2 *= wgt;
            }
        } else {
            const Real wgt = 1.0 / (1.0 + exp(arg));
            o0 *= wgt;
            o1 *= wgt;
            o2 *= wgt;
        }
    }
    out[i] = o0;
    out[a.nout + i] = o1;
    out[2 * a.nout + i] = o2;
}

// Differenced form: channels of the samples i0 + t and i0 + kTile + t of
// sub-block sb (after lfa2_diff_window), stored with the blend.  Per series,
// the first term interpolates S with the 32-point weights of the sample's own
// retarded position (both samples' weights formed together in packed pair
// instructions, as in lfa_z_mixed_pair); the B-term uses the two Q values
// around it.  Each series adds its link's term straight into its channel:
// X = 8 (T_a + T_b) [T_a R_a - T_b R_b] / (12 dt^2) (TDI 2.0) or
// X = 4 [T_a R_a - T_b R_b] / (12 dt) (TDI 1.5), R the stencil sums above.
static __device__ void lfa2_dvalues(const LfaArgs& a, int64_t i0, int64_t ic, Lfa2Smem& sm, int sb, int nr)
{
    const LfaWin& W = sm.win[sb];
    const int t = threadIdx.x;
    const int dm0 = (int)(i0 - ic) + t;
    const bool tdi20 = a.gen == LISA_TDI20;
    const bool equal = a.kind == LISA_LFA_EQUAL;
    // channel sums of the thread's two samples live in shared memory (the
    // pair weights need the registers); sm.xacc[2 ch + r][t].  So do the
    // three arms' light times at the two samples, sm.xacc[6 + 3 r + q][t]
    // (arm q: link 2q), each used by two series and two channels.
#pragma unroll
    for (int q = 0; q < 6; ++q) sm.xacc[q][t] = 0.f;
    if (!equal) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const float ur = (float)(dm0 + r * kTile) * sm.inv_half;
#pragma unroll
            for (int q = 0; q < 3; ++q) sm.xacc[6 + 3 * r + q][t] = sm.c0[kQT + 2 * q] + sm.cu[kQT + 2 * q](ur);
        }
    }
#pragma unroll kLfaDUnroll
    for (int c = 0; c < 6; ++c) {
        const float ih = sm.inv_half, idt = sm.inv_dt;
        const float2 u = make_float2((float)dm0 * ih, (float)(dm0 + kTile) * ih);
        const float4* rp = reinterpret_cast<const float4*>(&sm.ser[c]);
        float2 e;
        int ba, bb;
        {
            const float4 r0 = rp[0];   // f, d1, d2, d3
            const float Da = u.x * fmaf(u.x, fmaf(u.x, r0.w, r0.z), r0.y);
            const float Db = u.y * fmaf(u.y, fmaf(u.y, r0.w, r0.z), r0.y);
            const float va = fmaf(-Da, idt, r0.x);
            const float vb = fmaf(-Db, idt, r0.x);
            const float fa = floorf(va), fb = floorf(vb);
            e = make_float2(va - fa, vb - fb);
            ba = min(max(W.jrel[c] + dm0 + (int)fa, 0), W.wlen - 32);
            bb = min(max(W.jrel[c] + dm0 + kTile + (int)fb, 0), W.wlen - 32);
        }
        float2 sv[2];
        lagrange32_dot2_pair(e, sm.dw + ba, sm.dw + bb, sv[0], sv[1]);
        const int ch = c >> 1, arm = lfa_arm(ch, c & 1);
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const float uu = r ? u.y : u.x;
            const float ee = r ? e.y : e.x;
            const int base = r ? bb : ba;
            const float4 r0 = rp[0], rp1 = rp[1], rp2 = rp[2];
            const float Fp = fmaf(uu, fmaf(uu, fmaf(uu, rp1.w, rp1.z), rp1.y), rp1.x);
            const float Fc = fmaf(uu, fmaf(uu, fmaf(uu, rp2.w, rp2.z), rp2.y), rp2.x);
            // dF/di, and a1 = dx/di - 1 = -D'(u) ih / dt
            const float Fp1 = fmaf(uu, fmaf(uu, 3.f * rp1.w, 2.f * rp1.z), rp1.y) * ih;
            const float Fc1 = fmaf(uu, fmaf(uu, 3.f * rp2.w, 2.f * rp2.z), rp2.y) * ih;
            const float a1 = -fmaf(uu, fmaf(uu, 3.f * r0.w, 2.f * r0.z), r0.y) * ih * idt;
            const float2 q0 = sm.qw[base + 15], q1 = sm.qw[base + 16];
            const float qp = fmaf(ee, q1.x - q0.x, q0.x), qc = fmaf(ee, q1.y - q0.y, q0.y);
            const float m = fmaf(Fp, sv[r].x, Fc * sv[r].y);
            float R;
            if (tdi20) {
                // a2 = x''/2 = -(d2 + 3 d3 u) ih^2 / dt; B-term 24 (F1 + F a2) I', I' ~ Q / dt
                const float a2 = -fmaf(uu, 3.f * r0.w, r0.z) * ih * ih * idt;
                const float g = (1.f + a1) * (1.f + a1);
                R = fmaf(g, m, (24.f * idt) * fmaf(fmaf(Fp, a2, Fp1), qp, fmaf(Fc, a2, Fc1) * qc));
            } else {
                // B-term 12 F1 I, I ~ Q1 / dt
                R = fmaf(1.f + a1, m, (12.f * idt) * fmaf(Fp1, qp, Fc1 * qc));
            }
            // this series' arm factor: +T_a for link a, -T_b for link b
            const float T = equal ? a.Lcf : sm.xacc[6 + 3 * r + (arm >> 1)][t];
            sm.xacc[2 * ch + r][t] = fmaf((c & 1) ? -T : T, R, sm.xacc[2 * ch + r][t]);
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        if (r >= nr) break;
        float X[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const float Ta = equal ? a.Lcf : sm.xacc[6 + 3 * r + (lfa_arm(ch, 0) >> 1)][t];
            const float Tb = equal ? a.Lcf : sm.xacc[6 + 3 * r + (lfa_arm(ch, 1) >> 1)][t];
            const float pref = tdi20 ? 8.f * (Ta + Tb) * a.c2f : 4.f * a.c1f;
            X[ch] = pref * sm.xacc[2 * ch + r][t];
        }
        const int64_t i = i0 + r * kTile + t;
        if (a.xyz && i >= a.i_begin && i < a.i_end) lfa_store<float>(a, i, X, sm.barg_c, sm.barg_d, (int)(i - ic));
    }
}

// One group of nt tiles from tile t0 (centre ic = t0 kTile + G kTile / 2)
// in sub-blocks of two tiles, stored with the blend of the arguments.  The
// caller initialised sm.bar[0..1]; ph0, ph1 carry their phase parities from
// call to call.  Every thread must call it.  False if a bounded wait timed
// out (the status word is flagged; the block must stop).
static __device__ bool lfa2_group(const LfaArgs& a, int64_t t0, int nt, int G, Lfa2Smem& sm, uint32_t& ph0, uint32_t& ph1)
{
    const int64_t ic = t0 * kTile + (int64_t)G * kTile / 2;
    const int nsb = (nt + 1) / 2;
    lfa_tile_prologue<true>(a, ic, sm);   // ends with a block barrier
    lfa2_windows(a, t0, nsb, ic, sm);
    lfa2_stage(a, sm, 0, 0);
    bool prev_z = false;   // the previous sub-block left its z values in sm.zs
    for (int sb = 0; sb < nsb; ++sb) {
        const int b = sb & 1;
        const int64_t i0 = (t0 + 2 * sb) * (int64_t)kTile;
        // differenced form where the sub-block and its 2-sample z halos are
        // inside the output grid and its window inside the h grid (a choice
        // uniform over the block); the z-series form elsewhere
        const bool dwant = sm.win[sb].diff && i0 - 2 >= 0 && i0 + kSub2 + 2 <= a.nout;
        if (sb + 1 < nsb) lfa2_stage(a, sm, sb + 1, b ^ 1);
        const int wr = lfa2_wait_hdot(a, sm, sb, b, b ? ph1 : ph0, dwant);
        if (wr < 0) return false;
        if (sm.win[sb].bulk) {
            if (b) ph1 ^= 1u;
            else ph0 ^= 1u;
        }
        if (wr == 1) {
            lfa2_dvalues(a, i0, ic, sm, sb, nt - 2 * sb < 2 ? nt - 2 * sb : 2);
            prev_z = false;
            continue;
        }
        // z at samples i0-2 .. i0+1: the previous sub-block's last four values
        // (the previous channels were read before the barriers just passed),
        // unless they were overwritten by an attempted differenced window
        // (which shares the memory): then they are computed again
        const bool keep_halo = prev_z && !dwant;
        if (keep_halo && threadIdx.x < 24) {
            const int c = threadIdx.x >> 2, o = threadIdx.x & 3;
            sm.zs[c][o] = sm.zs[c][kSub2 + o];
        }
        lfa2_zvalues(a, i0, ic, sm, sb, !keep_halo);
        prev_z = true;
        for (int r = 0; r < 2; ++r) {
            if (2 * sb + r >= nt) break;
            float X[3];
            lfa2_channels(a, i0, ic, sm, r, X);
            const int64_t i = i0 + r * kTile + threadIdx.x;
            if (a.xyz && i >= a.i_begin && i < a.i_end) lfa_store<float>(a, i, X, sm.barg_c, sm.barg_d, (int)(i - ic));
        }
    }
    return true;
}

}  // namespace lisa
