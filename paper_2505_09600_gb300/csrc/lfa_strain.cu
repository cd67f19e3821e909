// Strain-derivative form of the LFA channels with the constellation centre
// (Sec. III, Eqs. X15_with_strain_derivatives, X20_with_strain_derivatives):
// equal constant arms T = L/c, and the mid-link positions k.(R_s + R_r)/2c of
// the equal-arm LFA replaced by k.R0/c, R0 the centre of the constellation
// (the mean of the three spacecraft positions):
//   X1.5(t) = 2 T^2 [(xi+_3 - xi+_2) d2h+SSB/dt2 + (xix_3 - xix_2) d2hxSSB/dt2](t - 2T - k.R0/c),
//   X2.0(t) = 8 T^3 [(xi+_3 - xi+_2) d3h+SSB/dt3 + (xix_3 - xix_2) d3hxSSB/dt3](t - 4T - k.R0/c),
// xi_2, xi_3 of the links +2 (y_123) and +3 (y_231) at t, Y and Z cyclic.
// All three channels share one retarded time, so a sample costs one 32-point
// interpolation of the two polarisations' strain derivative.
//
// One CTA per tile of kTile output samples:
//   1. the tile's retarded window: k.R0/c from the orbit polynomials (the mean
//      of the three k.R_s/c rows), the delay at the tile ends in FP64;
//   2. h staged on the window with a 4-sample margin, zero off the h grid;
//   3. the strain derivative S on the window: hdot (5-point first
//      derivative, zero off the grid), then the first (TDI 1.5) or second
//      (TDI 2.0) 5-point derivative of hdot, zero off the grid.  FP64 form:
//      literally.  Mixed form: inside the grid the 9-point composite of the
//      two stencils from second differences of h carried with their two-sum
//      errors (as the differenced LFA window), so S keeps FP32 relative
//      accuracy although it is ~(omega dt)^2..3 of h;
//   4. per sample the retarded position (mixed: the FP64 tile-centre split
//      plus an FP32 cubic of the in-tile variation), the 32-point weights,
//      xi of the links +1, +2, +3 from the link vectors, the three channels,
//      A/E/T, the blend and the store.
#include "lfa_tile.cuh"

namespace lisa {

constexpr int kStWin = kTile + 64;      // window: tile + 32-point stencil + drift margin
constexpr int kStWinP = kStWin + 16;    // staged h: 4-sample margins

struct StrainArgs {
    LfaArgs b;        // grids, sky, outputs, blend (the store of lfa_store)
    double T;         // L / c
    float Tf;
};

template <typename Real>
struct StrainSmem {
    using Pair = typename PairT<Real>::T;
    TileGeo g;
    Real hb[2][kStWinP];
    Pair sw[kStWin];
    float4 d2[kStWin + 8];
    int64_t jend[2];
    int64_t wlo;
    int wlen;
    int64_t J0;          // mixed: tile-centre split of the delay
    float f0;
    Cubic dvar;          // mixed: in-tile variation of the delay (s)
    float c0[kRows];
    Cubic cu[kRows];
    float inv_half, inv_dt, barg_c, barg_d;
};

// Delay of the shared retarded time at block coordinate u: shift + k.R0/c.
__device__ __forceinline__ double strain_delay(const TileGeo& g, double shift, double u)
{
    return shift + (tg_eval(g, kRowKR + 0, u) + tg_eval(g, kRowKR + 1, u) + tg_eval(g, kRowKR + 2, u)) / 3.0;
}

template <bool MIXED>
__global__ void __launch_bounds__(kTile) lfa_strain_kernel(StrainArgs sa)
{
    using Real = typename std::conditional<MIXED, float, double>::type;
    using Pair = typename PairT<Real>::T;
    __shared__ StrainSmem<Real> sm;
    const LfaArgs& a = sa.b;
    const int t = threadIdx.x;
    const int64_t i0 = (a.tile0 + blockIdx.x) * (int64_t)kTile;
    const int64_t ic = i0 + kTile / 2;
    const double half = 0.5 * a.tab.S;
    const bool tdi20 = a.gen == LISA_TDI20;
    const double shift = (tdi20 ? 4.0 : 2.0) * sa.T;
    tile_geo_load(sm.g, a.tab, ic, a.sky);
    const TileGeo& g = sm.g;
    if (t < 2) {
        const int64_t m = t ? i0 + kTile - 1 : i0;
        int64_t j;
        double eps;
        split_f64(a.hm, m, strain_delay(g, shift, (double)(m - ic) / half), j, eps);
        sm.jend[t] = j;
    }
    if (MIXED && t == 2) {
        int64_t j;
        double eps;
        split_f64(a.hm, ic, strain_delay(g, shift, 0.0), j, eps);
        sm.J0 = j;
        sm.f0 = (float)eps;
        sm.dvar = Cubic{(float)((g.b[kRowKR][1] + g.b[kRowKR + 1][1] + g.b[kRowKR + 2][1]) / 3.0),
                        (float)((g.b[kRowKR][2] + g.b[kRowKR + 1][2] + g.b[kRowKR + 2][2]) / 3.0),
                        (float)((g.b[kRowKR][3] + g.b[kRowKR + 1][3] + g.b[kRowKR + 2][3]) / 3.0)};
        sm.inv_half = (float)(1.0 / half);
        sm.inv_dt = (float)(1.0 / a.hm.dt_in);
        const double tc = a.t0_out + (double)ic * a.dt_out;
        sm.barg_c = (float)(a.bl.enabled ? a.bl.eps * (tc - a.bl.t_hyb) / a.bl.sigma : 0.0);
        sm.barg_d = (float)(a.bl.enabled ? a.bl.eps * a.dt_out / a.bl.sigma : 0.0);
    }
    if (MIXED && t >= 64 && t < 64 + kRows) {
        sm.c0[t - 64] = (float)g.b[t - 64][0];
        sm.cu[t - 64] = tg_cubic(g, t - 64);
    }
    __syncthreads();
    if (t == 0) {
        const int64_t lo = sm.jend[0] < sm.jend[1] ? sm.jend[0] : sm.jend[1];
        const int64_t hi = sm.jend[0] < sm.jend[1] ? sm.jend[1] : sm.jend[0];
        sm.wlo = lo - 15 - 2;
        const int64_t len = (hi + 16 + 2) - sm.wlo + 1;
        sm.wlen = len <= kStWin ? (int)len : 0;
    }
    __syncthreads();
    const int64_t wlo = sm.wlo;
    const int wlen = sm.wlen;
    const int64_t n_in = a.hm.n_in;
    const Real* __restrict__ hp = (const Real*)a.hp;
    const Real* __restrict__ hc = (const Real*)a.hc;
    // strain derivative at h-grid sample m from global memory (zero padding),
    // for windows that do not fit (not on the grids this library is used with)
    auto s_global = [&](const Real* h, int64_t m) -> Real {
        if (m < 0 || m >= n_in) return Real(0);
        auto hd = [&](int64_t q) -> Real {
            if (q < 0 || q >= n_in) return Real(0);
            auto at = [&](int64_t k) { return (k >= 0 && k < n_in) ? h[k] : Real(0); };
            return ((at(q + 1) - at(q - 1)) * Real(8) - (at(q + 2) - at(q - 2))) * Real(a.inv12dtf);
        };
        if constexpr (!MIXED) {
            const double i12 = 1.0 / (12.0 * a.hm.dt_in);
            auto hd64 = [&](int64_t q) -> double {
                if (q < 0 || q >= n_in) return 0.0;
                auto at = [&](int64_t k) { return (k >= 0 && k < n_in) ? h[k] : 0.0; };
                return ((at(q + 1) - at(q - 1)) * 8.0 - (at(q + 2) - at(q - 2))) * i12;
            };
            return tdi20 ? (-hd64(m - 2) + 16.0 * hd64(m - 1) - 30.0 * hd64(m) + 16.0 * hd64(m + 1) - hd64(m + 2))
                               * (i12 / a.hm.dt_in)
                         : ((hd64(m + 1) - hd64(m - 1)) * 8.0 - (hd64(m + 2) - hd64(m - 2))) * i12;
        } else {
            const float i12 = a.inv12dtf;
            return tdi20 ? (-hd(m - 2) + 16.f * hd(m - 1) - 30.f * hd(m) + 16.f * hd(m + 1) - hd(m + 2)) * i12 * sm.inv_dt
                         : ((hd(m + 1) - hd(m - 1)) * 8.f - (hd(m + 2) - hd(m - 2))) * i12;
        }
    };
    if (wlen > 0) {
        // h on [wlo - 4, wlo + wlen + 4), zero off the grid
        for (int k = t; k < wlen + 8; k += blockDim.x) {
            const int64_t idx = wlo - 4 + k;
            const bool in = idx >= 0 && idx < n_in;
            sm.hb[0][k] = in ? hp[idx] : Real(0);
            sm.hb[1][k] = in ? hc[idx] : Real(0);
        }
        __syncthreads();
        const Real* P = sm.hb[0];
        const Real* C = sm.hb[1];
        const bool interior = wlo - 4 >= 0 && wlo + wlen + 4 <= n_in;
        if constexpr (MIXED) {
            if (interior) {
                for (int n = t; n < wlen + 6; n += blockDim.x) {
                    const float2 p = second_diff_pair(P, n), c = second_diff_pair(C, n);
                    sm.d2[n] = make_float4(p.x, p.y, c.x, c.y);
                }
                __syncthreads();
                // composite stencils as in lfa2_diff_window, scaled by one more 1/(12 dt)
                const float sc = a.inv12dtf * a.inv12dtf * (tdi20 ? sm.inv_dt : 1.f);
                for (int k = t; k < wlen; k += blockDim.x) {
                    float4 v[7];
#pragma unroll
                    for (int j = 0; j < 7; ++j) v[j] = sm.d2[k + j];
                    float sp = 0.f, ep = 0.f, scx = 0.f, ec = 0.f;
                    if (tdi20) {
                        constexpr float gg[6] = {1.f, -21.f, 92.f, 92.f, -21.f, 1.f};
#pragma unroll
                        for (int j = 0; j < 6; ++j) {
                            sp = fmaf(gg[j], __fsub_rn(v[j + 1].x, v[j].x), sp);
                            ep = fmaf(gg[j], __fsub_rn(v[j + 1].y, v[j].y), ep);
                            scx = fmaf(gg[j], __fsub_rn(v[j + 1].z, v[j].z), scx);
                            ec = fmaf(gg[j], __fsub_rn(v[j + 1].w, v[j].w), ec);
                        }
                    } else {
                        constexpr float g1[7] = {1.f, -14.f, 35.f, 100.f, 35.f, -14.f, 1.f};
#pragma unroll
                        for (int j = 0; j < 7; ++j) {
                            sp = fmaf(g1[j], v[j].x, sp);
                            ep = fmaf(g1[j], v[j].y, ep);
                            scx = fmaf(g1[j], v[j].z, scx);
                            ec = fmaf(g1[j], v[j].w, ec);
                        }
                    }
                    sm.sw[k] = make_float2((sp + ep) * sc, (scx + ec) * sc);
                }
            } else {
                for (int k = t; k < wlen; k += blockDim.x) {
                    const int64_t m = wlo + k;
                    sm.sw[k] = make_float2(s_global(hp, m), s_global(hc, m));
                }
            }
        } else {
            // FP64: hdot on [wlo - 2, wlo + wlen + 2) from the staged h, then the stencil
            const double i12 = 1.0 / (12.0 * a.hm.dt_in);
            auto hd = [&](const double* X, int q) -> double {   // q: offset from wlo - 4
                const int64_t idx = wlo - 4 + q;
                if (idx < 0 || idx >= n_in) return 0.0;
                return ((X[q + 1] - X[q - 1]) * 8.0 - (X[q + 2] - X[q - 2])) * i12;
            };
            for (int k = t; k < wlen; k += blockDim.x) {
                const int64_t m = wlo + k;
                double2 v;
                if (m < 0 || m >= n_in) {
                    v = make_double2(0.0, 0.0);
                } else if (tdi20) {
                    const double s2 = i12 / a.hm.dt_in;
                    v.x = (-hd(P, k + 2) + 16.0 * hd(P, k + 3) - 30.0 * hd(P, k + 4) + 16.0 * hd(P, k + 5) - hd(P, k + 6)) * s2;
                    v.y = (-hd(C, k + 2) + 16.0 * hd(C, k + 3) - 30.0 * hd(C, k + 4) + 16.0 * hd(C, k + 5) - hd(C, k + 6)) * s2;
                } else {
                    v.x = ((hd(P, k + 5) - hd(P, k + 3)) * 8.0 - (hd(P, k + 6) - hd(P, k + 2))) * i12;
                    v.y = ((hd(C, k + 5) - hd(C, k + 3)) * 8.0 - (hd(C, k + 6) - hd(C, k + 2))) * i12;
                }
                sm.sw[k] = v;
            }
        }
        __syncthreads();
    }
    const int64_t i = i0 + t;
    if (i < a.i_begin || i >= a.i_end) return;
    // the shared retarded time: position, weights, the two strain derivatives
    Real Sp, Sc;
    Real up;   // block coordinate
    if constexpr (MIXED) {
        const int dm = (int)(i - ic);
        const float u = (float)dm * sm.inv_half;
        up = u;
        int jp;
        float fp;
        if (a.hm.unit_rho) {
            jp = dm;
            fp = 0.f;
        } else {
            const double Pp = (double)dm * a.hm.rho;
            const double fl = floor(Pp);
            jp = (int)fl;
            fp = (float)(Pp - fl);
        }
        const float v = fmaf(-sm.dvar(u), sm.inv_dt, fp + sm.f0);
        const float fv = floorf(v);
        const int64_t j = sm.J0 + jp + (int)fv;
        const float eps = v - fv;
        const int64_t base = j - 15 - wlo;
        if (wlen > 0 && base >= 0 && base + 32 <= wlen) {
            lagrange32_dot2(eps, sm.sw + base, Sp, Sc);
        } else {
            float w[32];
            lagrange32_weights(eps, w);
            Sp = Sc = 0.f;
            for (int k = 0; k < 32; ++k) {
                Sp = fmaf(w[k], s_global(hp, j - 15 + k), Sp);
                Sc = fmaf(w[k], s_global(hc, j - 15 + k), Sc);
            }
        }
    } else {
        const double u = (double)(i - ic) / half;
        up = u;
        int64_t j;
        double eps;
        split_f64(a.hm, i, strain_delay(g, shift, u), j, eps);
        double w[32];
        lagrange32_weights(eps, w);
        const int64_t base = j - 15 - wlo;
        Sp = Sc = 0.0;
        if (eps == 0.0) {
            const int64_t o = j - wlo;
            if (wlen > 0 && o >= 0 && o < wlen) {
                Sp = sm.sw[o].x;
                Sc = sm.sw[o].y;
            } else {
                Sp = s_global(hp, j);
                Sc = s_global(hc, j);
            }
        } else if (wlen > 0 && base >= 0 && base + 32 <= wlen) {
            for (int k = 0; k < 32; ++k) {
                Sp = fma(w[k], sm.sw[base + k].x, Sp);
                Sc = fma(w[k], sm.sw[base + k].y, Sc);
            }
        } else {
            for (int k = 0; k < 32; ++k) {
                Sp = fma(w[k], s_global(hp, j - 15 + k), Sp);
                Sc = fma(w[k], s_global(hc, j - 15 + k), Sc);
            }
        }
    }
    // xi of the links +1, +2, +3 at t, folded with the polarisation rotation:
    // G+ = xi+ cos 2psi + xix sin 2psi, Gx = xix cos 2psi - xi+ sin 2psi
    Real Gp[3], Gc[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int li = 2 * q;
        Real n3[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if constexpr (MIXED) n3[d] = sm.c0[kQN + 3 * li + d] + sm.cu[kQN + 3 * li + d](up);
            else n3[d] = tg_eval(g, kQN + 3 * li + d, up);
        }
        Real un, vn;
        if constexpr (MIXED) {
            un = a.sky.uf[0] * n3[0] + a.sky.uf[1] * n3[1] + a.sky.uf[2] * n3[2];
            vn = a.sky.vf[0] * n3[0] + a.sky.vf[1] * n3[1] + a.sky.vf[2] * n3[2];
        } else {
            un = a.sky.u[0] * n3[0] + a.sky.u[1] * n3[1] + a.sky.u[2] * n3[2];
            vn = a.sky.v[0] * n3[0] + a.sky.v[1] * n3[1] + a.sky.v[2] * n3[2];
        }
        const Real xp = un * un - vn * vn, xc = Real(2) * un * vn;
        const Real c2 = MIXED ? (Real)a.sky.c2f : (Real)a.sky.c2p, s2 = MIXED ? (Real)a.sky.s2f : (Real)a.sky.s2p;
        Gp[q] = xp * c2 + xc * s2;
        Gc[q] = xc * c2 - xp * s2;
    }
    const Real T = MIXED ? (Real)sa.Tf : (Real)sa.T;
    const Real pref = tdi20 ? Real(8) * T * T * T : Real(2) * T * T;
    Real X[3];
    // X: xi_3 - xi_2 (q = 2, 1); Y: xi_1 - xi_3 (0, 2); Z: xi_2 - xi_1 (1, 0)
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        const int q3 = (ch + 2) % 3, q2 = (ch + 1) % 3;
        X[ch] = pref * ((Gp[q3] - Gp[q2]) * Sp + (Gc[q3] - Gc[q2]) * Sc);
    }
    if constexpr (MIXED) lfa_store<float>(a, i, X, sm.barg_c, sm.barg_d, (int)(i - ic));
    else lfa_store<double>(a, i, X);
}

int launch_lfa_strain(const LfaArgs& a, double L_nominal, int precision, cudaStream_t st)
{
    StrainArgs sa;
    sa.b = a;
    sa.T = L_nominal / kC;
    sa.Tf = (float)sa.T;
    const int64_t tiles = (a.i_end - 1) / kTile - a.tile0 + 1;
    if (precision == LISA_MIXED) lfa_strain_kernel<true><<<(unsigned)tiles, kTile, 0, st>>>(sa);
    else lfa_strain_kernel<false><<<(unsigned)tiles, kTile, 0, st>>>(sa);
    return cuda_status(cudaGetLastError(), "lfa_strain_kernel launch");
}

}  // namespace lisa
