// Low-frequency approximation (Sec. III, App. B; Eqs. yslr_strain_derivatives,
// X15_nonequal, X20_nonequal, X15_equal, X20_equal).
//
// Per tile of kTile output samples one CTA
//   1. stages h+/hx over the window its retarded times reach and forms the
//      5-point central derivative hdot in shared memory,
//   2. computes the six TDI-shifted link series z (X_a, X_b, Y_a, Y_b, Z_a,
//      Z_b) on the tile plus a 2-sample halo each side:
//        z_a(t) = y_a(t - s_a),  y_l(t') = -(T_l/2)[xi+ hdot+SSB(tau) + xix hdotxSSB(tau)],
//        tau = t' - T_l/2 - k.(R_s + R_r)/(2c), geometry at t',
//      so z never goes to HBM unless the caller asks for it,
//   3. applies the 5-point first (TDI 1.5) or second (TDI 2.0) derivative to
//      z and the arm prefactors: X = 4[T_a z_a' - T_b z_b'] or
//      X = 8(T_a+T_b)[T_a z_a'' - T_b z_b''].
// The derivative stencils are evaluated as differences of differences, which
// keeps FP32 rounding from being amplified by the cancellation.
#include "lfa_tile.cuh"

namespace lisa {

#ifndef LISA_LFA_MINB
#define LISA_LFA_MINB 4
#endif
// FP64 form: one tile after another around the group's prologue.
__global__ void __launch_bounds__(kTile, 1) lfa_kernel_f64(LfaArgs a, int64_t tile_end, int G)
{
    __shared__ LfaSmem64 sm;
    const int64_t t0 = a.tile0 + (int64_t)blockIdx.x * G;
    const int64_t ic = t0 * kTile + (int64_t)G * kTile / 2;
    const int nt = (int)(tile_end - t0 < G ? tile_end - t0 : G);
    lfa_tile_prologue<false>(a, ic, sm);   // ends with a block barrier
    for (int q = 0; q < nt; ++q) {
        const int64_t i0 = (t0 + q) * (int64_t)kTile;
        double X[3];
        lfa_tile_body(a, i0, ic, sm, X);
        const int64_t i = i0 + threadIdx.x;
        if (a.xyz && i >= a.i_begin && i < a.i_end) lfa_store<double>(a, i, X);
    }
}

// Mixed form: the group's tiles share one prologue and run in sub-blocks of
// two tiles; the h window of the next sub-block is fetched with bulk copies
// (two buffers) while the current one is computed.
__global__ void __launch_bounds__(kTile, LISA_LFA_MINB) lfa_kernel_mixed(LfaArgs a, int64_t tile_end, int G)
{
    __shared__ Lfa2Smem sm;
    const int64_t t0 = a.tile0 + (int64_t)blockIdx.x * G;
    const int nt = (int)(tile_end - t0 < G ? tile_end - t0 : G);
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        mbar_init_fence();
    }
    uint32_t ph0 = 0u, ph1 = 0u;
    lfa2_group(a, t0, nt, G, sm, ph0, ph1);
}

int lfa_group_host(double dt) { return lfa_group(dt); }
int lfa_group_host(double dt, int precision)
{
    return precision == LISA_DF ? lfa_group_df(dt) : precision == LISA_MIXED ? lfa_group_mixed(dt) : lfa_group(dt);
}

int launch_lfa_strain(const LfaArgs& a, double L_nominal, int precision, cudaStream_t st);
int launch_lfa_df(const LfaArgs& a, cudaStream_t st);

int launch_lfa(const SegTable& tab, const SkyDev& sky, double L_nominal, const lisa_grid& hg, const void* hp,
               const void* hc, int precision, int gen, int kind, int channels, const lisa_grid& og, void* z,
               void* xyz, int64_t i_begin, int64_t i_end, const BlendSpec& bl, cudaStream_t st, int group)
{
    if (kind == LISA_LFA_NLO && precision == LISA_MIXED) {
        set_error("the next-to-leading-order LFA is an FP64 form: its third- and fourth-derivative stencils "
                  "amplify FP32 rounding beyond the terms they add at low frequency");
        return LISA_EINVAL;
    }
    if (i_end <= i_begin) return LISA_OK;
    LfaArgs a;
    a.tab = tab;
    a.sky = sky;
    a.hm = make_grid_map(og, hg);
    a.Lc = L_nominal / kC;
    a.gen = gen;
    a.kind = kind;
    a.channels = channels;
    a.hp = hp;
    a.hc = hc;
    a.z = z;
    a.xyz = xyz;
    a.nout = og.n;
    a.t0_out = og.t0;
    a.dt_out = og.dt;
    a.i_begin = i_begin;
    a.i_end = i_end;
    a.tile0 = i_begin / kTile;
    a.bl = bl;
    lfa_args_f32(a);
    a.h_aligned = ((uintptr_t)hp % 16 == 0) && ((uintptr_t)hc % 16 == 0);
    a.status = device_status_ptr();
    if (kind == LISA_LFA_STRAIN) {
        if (z || gen == kLfaOwnTime) {
            set_error("the strain-derivative form has no link series");
            return LISA_EINVAL;
        }
        prof_before(precision == LISA_MIXED ? "lfa_strain_mixed" : "lfa_strain_f64", st);
        const int rc = launch_lfa_strain(a, L_nominal, precision, st);
        prof_after(st);
        return rc;
    }
    if (precision == LISA_DF && a.hm.unit_rho && !z && gen != kLfaOwnTime && xyz &&
        (kind == LISA_LFA_UNEQUAL || kind == LISA_LFA_EQUAL || kind == LISA_LFA_BACKWARD ||
         kind == LISA_LFA_FORWARD)) {
        prof_before("lfa_df", st);
        const int rc = launch_lfa_df(a, st);
        prof_after(st);
        return rc;
    }
    const int64_t tiles = (i_end - 1) / kTile - a.tile0 + 1;
    const int64_t tile_end = a.tile0 + tiles;
    prof_before(gen == kLfaOwnTime ? (precision == LISA_MIXED ? "lfa_own_mixed" : "lfa_own_f64")
                                   : (precision == LISA_MIXED ? "lfa_mixed" : "lfa_f64"), st);
    if (precision == LISA_MIXED) {
        const int G0 = lfa_group_mixed(og.dt);
        int G = group > 0 && group < G0 ? group : G0;
        if (gen == kLfaOwnTime && group == 0) {
            // link series at their own time: groups narrowed on short ranges so
            // that the CTAs fill the SMs (2 tiles at least: one sub-block)
            static int sms = 0;
            if (sms == 0) {
                int dev = 0;
                cudaGetDevice(&dev);
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
                if (sms <= 0) sms = 1;
            }
            const int64_t per_sm = tiles / sms;
            const int Gs = per_sm < 2 ? 2 : (per_sm > 8 ? 8 : (int)per_sm);
            if (Gs < G) G = Gs;
        }
        lfa_kernel_mixed<<<(unsigned)((tiles + G - 1) / G), kTile, 0, st>>>(a, tile_end, G);
    } else {
        lfa_kernel_f64<<<(unsigned)tiles, kTile, 0, st>>>(a, tile_end, 1);
    }
    prof_after(st);
    return cuda_status(cudaGetLastError(), "lfa_kernel launch");
}

// ---------------------------------------------------------------------------
// lisa_tdi_lfa: channels from caller-provided z series
// ---------------------------------------------------------------------------
struct TdiLfaArgs {
    SegTable tab;
    double Lc, dt;
    int gen, kind, channels;
    const void* z;
    void* xyz;
    int64_t n;
};

template <typename Real>
__global__ void __launch_bounds__(kTile) tdi_lfa_kernel(TdiLfaArgs a)
{
    __shared__ TileGeo g;
    const int64_t i0 = (int64_t)blockIdx.x * kTile;
    const int64_t ic = i0 + kTile / 2;
    const double half = 0.5 * a.tab.S;
    tile_geo_load(g, a.tab, ic, SkyDev{});
    const int64_t i = i0 + threadIdx.x;
    if (i >= a.n) return;
    const Real* z = (const Real*)a.z;
    auto at = [&](int c, int64_t k) { return (k >= 0 && k < a.n) ? z[(int64_t)c * a.n + k] : Real(0); };
    const double u = (double)(i - ic) / half;
    const bool equal = (a.kind == LISA_LFA_EQUAL);
    const Real dt = (Real)a.dt;
    Real X[3];
    for (int ch = 0; ch < 3; ++ch) {
        const Real Ta = (Real)(equal ? a.Lc : tg_eval(g, kQT + lfa_arm(ch, 0), u));
        const Real Tb = (Real)(equal ? a.Lc : tg_eval(g, kQT + lfa_arm(ch, 1), u));
        Real za[5], zb[5];
        for (int k = 0; k < 5; ++k) {
            za[k] = at(2 * ch, i - 2 + k);
            zb[k] = at(2 * ch + 1, i - 2 + k);
        }
        if (a.gen == LISA_TDI20) {
            auto d2 = [&](const Real* zz) {
                const Real e0 = zz[1] - zz[0], e1 = zz[2] - zz[1], e2 = zz[3] - zz[2], e3 = zz[4] - zz[3];
                return (Real(14) * (e2 - e1) - (e1 - e0) - (e3 - e2)) / (Real(12) * dt * dt);
            };
            X[ch] = Real(8) * (Ta + Tb) * (Ta * d2(za) - Tb * d2(zb));
            if (a.kind == LISA_LFA_NLO) X[ch] += lfa_nlo_channel20<Real>(Ta, Tb, za, zb, a.dt);
        } else {
            auto d1 = [&](const Real* zz) { return ((zz[3] - zz[1]) * Real(8) - (zz[4] - zz[0])) / (Real(12) * dt); };
            X[ch] = Real(4) * (Ta * d1(za) - Tb * d1(zb));
            if (a.kind == LISA_LFA_NLO) X[ch] += lfa_nlo_channel15<Real>(Ta, Tb, za, zb, a.dt);
        }
    }
    Real* out = (Real*)a.xyz;
    if (a.channels == LISA_AET) {
        out[i] = (X[2] - X[0]) * Real(0.70710678118654752440);
        out[a.n + i] = (X[0] - Real(2) * X[1] + X[2]) * Real(0.40824829046386301637);
        out[2 * a.n + i] = (X[0] + X[1] + X[2]) * Real(0.57735026918962576451);
    } else {
        out[i] = X[0];
        out[a.n + i] = X[1];
        out[2 * a.n + i] = X[2];
    }
}

int launch_tdi_lfa(const SegTable& tab, double L_nominal, const lisa_grid& zg, const void* z, int precision, int gen,
                   int kind, int channels, void* xyz, cudaStream_t st)
{
    if (kind == LISA_LFA_NLO && precision == LISA_MIXED) {
        set_error("the next-to-leading-order LFA is an FP64 form");
        return LISA_EINVAL;
    }
    if (zg.n <= 0) return LISA_OK;
    TdiLfaArgs a{tab, L_nominal / kC, zg.dt, gen, kind, channels, z, xyz, zg.n};
    const int64_t tiles = (zg.n + kTile - 1) / kTile;
    prof_before(precision == LISA_MIXED ? "tdi_lfa_mixed" : "tdi_lfa_f64", st);
    if (precision == LISA_MIXED) tdi_lfa_kernel<float><<<(unsigned)tiles, kTile, 0, st>>>(a);
    else tdi_lfa_kernel<double><<<(unsigned)tiles, kTile, 0, st>>>(a);
    prof_after(st);
    return cuda_status(cudaGetLastError(), "tdi_lfa_kernel launch");
}

}  // namespace lisa
