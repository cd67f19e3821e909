// Per-tile prologue and per-sample body of the full single-link response,
// shared by the links kernel and the fused full-response tile of the batched
// kernel.  See links_full.cu for the formulas.
#pragma once

#include <type_traits>

#include "lisa_common.cuh"
#include "lisa_internal.cuh"
#include "tile_geo.cuh"

namespace lisa {

constexpr int kWinMax = kTile + 768;

template <typename Real>
struct Pair;
template <>
struct Pair<double> { using T = double2; };
template <>
struct Pair<float> { using T = float2; };

struct LinksArgs {
    SegTable tab;
    SkyDev sky;
    GridMap hm;
    const void* hp;
    const void* hc;
    void* y;
    int64_t ny;
    int64_t y0;      // sample index held by y[0] (grouped links: stores go to y[li ny + i - y0])
    int64_t i_begin, i_end;
    int64_t tile0;
};

// Shared memory of one links tile: the staged h window and, for the mixed
// form, the tile-centre delay splits and in-tile cubics (12 link-times:
// li*2 + {0: sender, 1: receiver}) and the centre n_l - k with its cubic.
template <bool MIXED>
struct LinksTile {
    using Real = typename std::conditional<MIXED, float, double>::type;
    typename Pair<Real>::T win[kWinMax];
    int64_t jends[24];
    int64_t wlo;
    int wlen;
    int64_t J[12];
    float f[12];
    Cubic dd[12];
    float dk[6][3];
    Cubic dn[6][3];
    float inv_half, inv_dt;   // FP32 constants (no per-sample FP64 work)
};

// Interpolate both polarisations at (j, eps) from the staged window, or from
// global memory when the stencil is not inside the window.
template <typename Real>
__device__ __forceinline__ void interp_pair(const typename Pair<Real>::T* win, int64_t wlo, int wlen,
                                            const Real* __restrict__ hp, const Real* __restrict__ hc, int64_t nh,
                                            int64_t j, Real eps, Real& op, Real& oc)
{
    const int64_t base = j - 15 - wlo;
    if (eps == Real(0)) {
        const int64_t o = j - wlo;
        if (o >= 0 && o < wlen) {
            op = win[o].x;
            oc = win[o].y;
        } else {
            op = (j >= 0 && j < nh) ? hp[j] : Real(0);
            oc = (j >= 0 && j < nh) ? hc[j] : Real(0);
        }
        return;
    }
    Real w[32];
    lagrange32_weights(eps, w);
    Real ap = Real(0), ac = Real(0);
    if (base >= 0 && base + 32 <= wlen) {
        const typename Pair<Real>::T* p = win + base;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const typename Pair<Real>::T v = p[k];
            ap = fma(w[k], v.x, ap);
            ac = fma(w[k], v.y, ac);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const int64_t idx = j - 15 + k;
            if (idx >= 0 && idx < nh) {
                ap = fma(w[k], hp[idx], ap);
                ac = fma(w[k], hc[idx], ac);
            }
        }
    }
    op = ap;
    oc = ac;
}

// Both polarisations interpolated straight from global memory (zero outside
// the grid): stencils that the staged window does not hold.  Out of line.
static __device__ __noinline__ float2 links_interp_global_f32(const float* __restrict__ hp, const float* __restrict__ hc,
                                                              int64_t n, int64_t j, float eps)
{
    float ap = 0.f, ac = 0.f;
    lagrange32_paired_f32(eps, [&](int p, float w) {
        const int64_t idx = j - 15 + p;
        if (idx >= 0 && idx < n) {
            ap = fmaf(w, hp[idx], ap);
            ac = fmaf(w, hc[idx], ac);
        }
    });
    return make_float2(ap, ac);
}

// Stage the h window reachable from samples m_lo..m_hi (tile centre ic) and
// the mixed-precision per-tile data.  Every thread must call it (it
// synchronises); g must already hold the tile geometry around ic.
template <bool MIXED>
__device__ void links_tile_prologue(const LinksArgs& a, const TileGeo& g, int64_t ic, int64_t m_lo, int64_t m_hi,
                                    LinksTile<MIXED>& s)
{
    using Real = typename std::conditional<MIXED, float, double>::type;
    using Real2 = typename Pair<Real>::T;
    const double half = 0.5 * a.tab.S;
    const int t = threadIdx.x;
    if (t < 24) {
        const int end = t / 12, lt = t % 12, li = lt >> 1;
        const int64_t ie = end ? m_hi : m_lo;
        const double u = (double)(ie - ic) / half;
        const double d = (lt & 1) ? tg_eval(g, kRowKR + link_receiver(li), u)
                                  : tg_eval(g, kQT + li, u) + tg_eval(g, kRowKR + link_sender(li), u);
        int64_t j;
        double eps;
        split_f64(a.hm, ie, d, j, eps);
        s.jends[t] = j;
    }
    if constexpr (MIXED) {
        if (t == 45) {
            s.inv_half = (float)(2.0 / a.tab.S);
            s.inv_dt = (float)(1.0 / a.hm.dt_in);
        }
        if (t >= 32 && t < 44) {
            const int lt = t - 32, li = lt >> 1;
            const int rs = (lt & 1) ? kRowKR + link_receiver(li) : kRowKR + link_sender(li);
            double dc = g.b[rs][0];
            Cubic cv = tg_cubic(g, rs);
            if (!(lt & 1)) {
                dc += g.b[kQT + li][0];
                const Cubic ct = tg_cubic(g, kQT + li);
                cv.c1 += ct.c1; cv.c2 += ct.c2; cv.c3 += ct.c3;
            }
            int64_t j;
            double eps;
            split_f64(a.hm, ic, dc, j, eps);
            s.J[lt] = j;
            s.f[lt] = (float)eps;
            s.dd[lt] = cv;
        }
        if (t >= 64 && t < 82) {
            const int q = t - 64, li = q / 3, c = q % 3;
            s.dk[li][c] = (float)(g.b[kQN + 3 * li + c][0] - a.sky.k[c]);
            s.dn[li][c] = tg_cubic(g, kQN + 3 * li + c);
        }
    }
    __syncthreads();
    if (t == 0) {
        int64_t lo = s.jends[0], hi = s.jends[0];
        for (int k = 1; k < 24; ++k) {
            lo = s.jends[k] < lo ? s.jends[k] : lo;
            hi = s.jends[k] > hi ? s.jends[k] : hi;
        }
        s.wlo = lo - 15 - 3;
        const int64_t len = (hi + 16 + 3) - s.wlo + 1;
        s.wlen = len <= kWinMax ? (int)len : 0;
    }
    __syncthreads();
    const int64_t wlo = s.wlo;
    const int wlen = s.wlen;
    const Real* __restrict__ hp = (const Real*)a.hp;
    const Real* __restrict__ hc = (const Real*)a.hc;
    for (int k = t; k < wlen; k += blockDim.x) {
        const int64_t idx = wlo + k;
        Real2 v;
        v.x = (idx >= 0 && idx < a.hm.n_in) ? hp[idx] : Real(0);
        v.y = (idx >= 0 && idx < a.hm.n_in) ? hc[idx] : Real(0);
        s.win[k] = v;
    }
    __syncthreads();
}

// FP64 link li at sample m (block coordinate u, k.R/c of the three
// spacecraft kR): the projection of the polarisation tensors on n_l - k
// over |n_l - k|^2, times the difference of h at the sender and receiver ends.
__device__ __forceinline__ double link_value_f64(const LinksArgs& a, const TileGeo& g, double u, int64_t m,
                                                 const LinksTile<false>& s, int li, const double* kR)
{
    const double* __restrict__ hp = (const double*)a.hp;
    const double* __restrict__ hc = (const double*)a.hc;
    double d[3], dd = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        d[c] = tg_eval(g, kQN + 3 * li + c, u) - a.sky.k[c];
        dd = fma(d[c], d[c], dd);
    }
    if (!(dd >= 2e-12)) return 0.0;
    const double* ku = a.sky.u;
    const double* kv = a.sky.v;
    const double c2 = a.sky.c2p, s2 = a.sky.s2p;
    const double un = ku[0] * d[0] + ku[1] * d[1] + ku[2] * d[2];
    const double vn = kv[0] * d[0] + kv[1] * d[1] + kv[2] * d[2];
    const double xp = un * un - vn * vn, xc = 2.0 * un * vn;
    const double Fp = (xp * c2 + xc * s2) / dd, Fc = (xc * c2 - xp * s2) / dd;
    const double ds = tg_eval(g, kQT + li, u) + kR[link_sender(li)];
    const double dr = kR[link_receiver(li)];
    int64_t js, jr;
    double es, er;
    split_f64(a.hm, m, ds, js, es);
    split_f64(a.hm, m, dr, jr, er);
    double ps, cs, pr, cr;
    interp_pair<double>(s.win, s.wlo, s.wlen, hp, hc, a.hm.n_in, js, es, ps, cs);
    interp_pair<double>(s.win, s.wlo, s.wlen, hp, hc, a.hm.n_in, jr, er, pr, cr);
    return Fp * (ps - pr) + Fc * (cs - cr);
}

// The six links at sample m of the link grid, stored to out[li * stride].
template <bool MIXED>
__device__ __forceinline__ void links_sample(const LinksArgs& a, const TileGeo& g, int64_t ic, int64_t m,
                                             const LinksTile<MIXED>& s,
                                             typename std::conditional<MIXED, float, double>::type* out,
                                             int64_t stride)
{
    using Real = typename std::conditional<MIXED, float, double>::type;
    const Real* __restrict__ hp = (const Real*)a.hp;
    const Real* __restrict__ hc = (const Real*)a.hc;
    const double half = 0.5 * a.tab.S;
    const int64_t wlo = s.wlo;
    const int wlen = s.wlen;
    Real c2, s2, ku[3], kv[3];
    if constexpr (MIXED) {
        c2 = a.sky.c2f; s2 = a.sky.s2f;
        for (int q = 0; q < 3; ++q) { ku[q] = a.sky.uf[q]; kv[q] = a.sky.vf[q]; }
    } else {
        c2 = a.sky.c2p; s2 = a.sky.s2p;
        for (int q = 0; q < 3; ++q) { ku[q] = a.sky.u[q]; kv[q] = a.sky.v[q]; }
    }

    if constexpr (!MIXED) {
        const double u = (double)(m - ic) / half;
        double kR[3];
#pragma unroll
        for (int sc = 0; sc < 3; ++sc) kR[sc] = tg_eval(g, kRowKR + sc, u);
#pragma unroll 1
        for (int li = 0; li < 6; ++li) out[li * stride] = link_value_f64(a, g, u, m, s, li, kR);
    } else {
        // in-tile offsets are 32-bit: no 64-bit conversions (FP64 pipe) per sample
        const float u = (float)(int)(m - ic) * s.inv_half;
        // integer / fractional split of (m - ic) * rho, shared by all link-times
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
        const float inv_dt = s.inv_dt;
        // stencil position of link-time lt (even: sender end, odd: receiver end)
        auto interp_lt = [&](int lt, float& op, float& oc) {
            const float v = (fp + s.f[lt]) - s.dd[lt](u) * inv_dt;
            const float fv = floorf(v);
            const float eps = v - fv;
            if (wlen > 0) {
                // every stencil of the tile lies in the staged window (the
                // window spans the tile's end points plus margins and the
                // retarded index is monotonic); the clamp keeps reads in bounds
                const int base = min(max((int)(s.J[lt] - wlo) + (int)jp + (int)fv - 15, 0), wlen - 32);
                lagrange32_dot2(eps, reinterpret_cast<const float2*>(s.win) + base, op, oc);
            } else {
                const float2 r = links_interp_global_f32(hp, hc, a.hm.n_in, s.J[lt] + jp + (int)fv, eps);
                op = r.x;
                oc = r.y;
            }
        };
        // receiver ends: k.R_r/c depends on the receiving spacecraft only, so
        // the two links into a spacecraft share it (links 3, 0, 1 carry the
        // receivers 0, 1, 2)
        float rp[3], rc[3];
        interp_lt(2 * 3 + 1, rp[0], rc[0]);
        interp_lt(2 * 0 + 1, rp[1], rc[1]);
        interp_lt(2 * 1 + 1, rp[2], rc[2]);
#pragma unroll
        for (int li = 0; li < 6; ++li) {
            float d[3], dd = 0.f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                d[c] = s.dk[li][c] + s.dn[li][c](u);
                dd = fmaf(d[c], d[c], dd);
            }
            const float un = ku[0] * d[0] + ku[1] * d[1] + ku[2] * d[2];
            const float vn = kv[0] * d[0] + kv[1] * d[1] + kv[2] * d[2];
            const float xp = un * un - vn * vn, xc = 2.f * un * vn;
            const float rdd = 1.f / dd;
            const float Fp = (xp * c2 + xc * s2) * rdd, Fc = (xc * c2 - xp * s2) * rdd;
            float ps, cs;
            interp_lt(2 * li, ps, cs);
            const int r = link_receiver(li);
            const float y = Fp * (ps - rp[r]) + Fc * (cs - rc[r]);
            out[li * stride] = dd >= 2e-12f ? y : 0.f;
        }
    }
}

}  // namespace lisa
