// LFA channels in double-float arithmetic (precision LISA_DF): FP64 inputs
// and outputs, the per-sample arithmetic on the FP32 pipe in pairs of FP32
// numbers (dfloat.cuh), with FP64 only in the per-group set-up and at the two
// ends (staging of hdot, the store).  The method is the z-series form of the
// LFA kernel (Sec. III, Eqs. yslr_strain_derivatives, X15_nonequal,
// X20_nonequal; App. B for the expansion points):
//   z_c(t) = F+_c(t) hdot+(x_c(t)) + Fx_c(t) hdotx(x_c(t)),
//   X = 4 [T_a dz_a/dt - T_b dz_b/dt]  or  8 (T_a + T_b) [T_a d2z_a/dt2 - T_b d2z_b/dt2],
// with F+-, Fx the link's projection factors (-T_l/2 times the rotated
// antenna patterns), x_c the retarded position of series c on the h grid,
// 32-point Lagrange interpolation and 5-point stencils.
//
// Layout: one CTA of kTile threads per group of up to G tiles sharing one
// FP64 set-up at the group centre ic.  The set-up composes, for each of the
// six series, the light time, the two end projections k.R/c and the link
// vector with the series' retarded coordinate (TDI shift and light time) to
// degree 5 in the block coordinate u = (m - ic) / (S/2), exactly in FP64
// (Taylor shift of the orbit polynomials, then the composition with the
// powers of the retarded offset), and from them the delay variation d(u) -
// d(0) (degree 5) and the projection factors F+(u), Fx(u) (degree 4).  Over a
// group |u| <= 0.0625 and the orbital phase moves by < 1e-3 rad, so the
// dropped terms are below 1e-18 s in the delay and 1e-17 of the factors.  The
// centre delay is split once into (J, f) in FP64.  Per sample, u is exact in
// FP32 (S is a power of two), and every polynomial, the position, the 32
// weights (the paired mirrored-node scheme of the FP32 weights, with
// compensated products), the tap sums (two-sum accumulation of exact
// products, both polarisations per packed FP32 pair instruction) and the
// channel stencils run in double-float; the polynomials' tails (the terms
// from u^3 on) run in FP32: over a group of half-span <= 1.1e4 s they are
// below 1e-6 s in the delay (FP32 rounding < 1e-13 s, < 2e-14 of a sample at
// dt >= 5 s, an interpolation error at the level of the taps' own rounding)
// and below 2e-9 of the projection factors and light times.
#include "dfloat.cuh"
#include "lfa_tile.cuh"

namespace lisa {

#ifndef LISA_DF_MINB
#define LISA_DF_MINB 3   // resident CTAs per SM the register budget is set for (fastest of 2, 3, 4)
#endif

constexpr int kDfD = 6;   // delay polynomial coefficients (degree 5)
constexpr int kDfF = 5;   // projection factor coefficients (degree 4)

struct DfSer {
    df d[kDfD];          // delay variation d(u) - d(0) (s), d[0] = 0
    df fp[kDfF], fc[kDfF];
    df f0;               // fraction of the centre delay's split
};

constexpr int kDfGmax = 8;   // tiles per group (lfa_group)

struct DfWin {
    int64_t wlo;                  // first h sample of the tile's hdot window
    int wlen;                     // its length (0: read h from global memory)
};

struct DfSmem {
    TileGeo g;
    float4 dw[2][kWinH];          // hdot windows as double-floats (h+ hi, hx hi, h+ lo, hx lo), two buffers
    float2 wmax[2][kTile / 32];   // per warp: largest |h+ hi|, |hx hi| it staged into buffer 0 / 1
    df zs[2][6][kZW];             // z of a tile and its 2-sample halos, two buffers (tiles q, q - 1)
    df halo[2][6][4];             // z at the next tile's left halo and first two samples, two buffers
    DfSer ser[6];
    int64_t J[6];
    df arm[3][kDfF];              // light times of the links +1, +2, +3 (s), degree 4
    double dp64[6][kDfD];         // FP64 delay polynomial of each series (window location)
    double comp[6][6][kDfD];      // set-up scratch: composed quantities
    DfWin win[kDfGmax];
    int64_t jends[kDfGmax][12];
    float inv_half;
    df inv_dt;                    // 1 / dt (double-float)
    df k1, k2;                    // 1 / (12 dt), 1 / (12 dt^2) of the output grid (stencils)
    int blend;                    // the sigmoid weight differs from 1 somewhere in the group
};

// Truncated product of two degree-N-1 polynomials.
template <int N>
__device__ __forceinline__ void poly_mul(const double* a, const double* b, double* c)
{
#pragma unroll
    for (int k = 0; k < N; ++k) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j <= k; ++j) s = fma(a[j], b[k - j], s);
        c[k] = s;
    }
}

__device__ __forceinline__ df df_of(double d) { return df_from_double(d); }

// Set-up of the group of nt tiles from tile t0, centred at ic, and the hdot
// windows of its tiles (every thread; synchronises).
static __device__ void df_prologue(const LfaArgs& a, int64_t t0, int nt, int64_t ic, DfSmem& sm)
{
    TileGeo& g = sm.g;
    const int t = threadIdx.x;
    tile_geo_load(g, a.tab, ic, a.sky);
    const bool equal = (a.kind == LISA_LFA_EQUAL);
    const double u_per_s = 1.0 / (a.dt_out * 0.5 * a.tab.S);
    if (t < 36) {
        // series c, quantity r: 0 T_l, 1 k.R_s/c, 2 k.R_r/c, 3..5 n_l, composed
        // with the retarded coordinate up(u) = u - sh(u) u_per_s
        const int c = t / 6, r = t % 6;
        const int ch = c >> 1, which = c & 1;
        const int l = a.gen == kLfaOwnTime ? c : lfa_link(ch, which);
        double sh[kDfD] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        if (a.gen != kLfaOwnTime) {
            const double al = which ? (a.gen == LISA_TDI20 ? 1.5 : 0.5) : (a.gen == LISA_TDI20 ? 2.0 : 1.0);
            const double be = which ? (a.gen == LISA_TDI20 ? 2.0 : 1.0) : (a.gen == LISA_TDI20 ? 1.5 : 0.5);
            const int ra = kQT + lfa_arm(ch, 0), rb = kQT + lfa_arm(ch, 1);
            for (int k = 0; k < kDfD; ++k)
                sh[k] = equal ? (k == 0 ? (al + be) * a.Lc : 0.0) : al * g.b[ra][k] + be * g.b[rb][k];
        }
        // delta(u) = up(u) - up(0) and its powers
        double dl[kDfD];
        dl[0] = 0.0;
        for (int k = 1; k < kDfD; ++k) dl[k] = (k == 1 ? 1.0 : 0.0) - sh[k] * u_per_s;
        double out[kDfD];
        if (r == 0 && equal) {
            for (int k = 0; k < kDfD; ++k) out[k] = k == 0 ? a.Lc : 0.0;
        } else {
            const int row = r == 0 ? kQT + l : r == 1 ? kRowKR + link_sender(l)
                          : r == 2 ? kRowKR + link_receiver(l) : kQN + 3 * l + (r - 3);
            double b[7];
            taylor_shift7(g.b[row], -sh[0] * u_per_s, b);
            double pw[kDfD] = {1.0, 0.0, 0.0, 0.0, 0.0, 0.0};
            for (int k = 0; k < kDfD; ++k) out[k] = 0.0;
            for (int p = 0; p < kDfD; ++p) {
                for (int k = 0; k < kDfD; ++k) out[k] = fma(b[p], pw[k], out[k]);
                double nx[kDfD];
                poly_mul<kDfD>(pw, dl, nx);
                for (int k = 0; k < kDfD; ++k) pw[k] = nx[k];
            }
        }
        for (int k = 0; k < kDfD; ++k) sm.comp[c][r][k] = out[k];
        // the TDI shift itself goes with the delay (r == 0 thread keeps it)
        if (r == 0)
            for (int k = 0; k < kDfD; ++k) sm.dp64[c][k] = sh[k];
    }
    if (t >= 64 && t < 64 + 15) {
        const int q = (t - 64) / kDfF, k = (t - 64) % kDfF;
        sm.arm[q][k] = df_of(equal ? (k == 0 ? a.Lc : 0.0) : g.b[kQT + 2 * q][k]);
    }
    if (t == 96) {
        sm.inv_half = (float)(2.0 / a.tab.S);
        sm.inv_dt = df_of(1.0 / a.hm.dt_in);
        sm.k1 = df_of(1.0 / (12.0 * a.dt_out));
        sm.k2 = df_of(1.0 / (12.0 * a.dt_out * a.dt_out));
    }
    __syncthreads();
    if (t < 6) {
        const int c = t;
        double d[kDfD];
        for (int k = 0; k < kDfD; ++k) {
            const double Tl = sm.comp[c][0][k], ks = sm.comp[c][1][k], kr = sm.comp[c][2][k];
            d[k] = sm.dp64[c][k] + (a.kind == LISA_LFA_BACKWARD ? Tl + ks
                                    : a.kind == LISA_LFA_FORWARD ? kr : 0.5 * (Tl + ks + kr));
        }
        for (int k = 0; k < kDfD; ++k) sm.dp64[c][k] = d[k];
        int64_t j;
        double eps;
        split_f64(a.hm, ic, d[0], j, eps);
        sm.J[c] = j;
        DfSer& R = sm.ser[c];
        R.f0 = df_of(eps);
        R.d[0] = df{0.f, 0.f};
        for (int k = 1; k < kDfD; ++k) R.d[k] = df_of(d[k]);
        // projection factors: (u.n), (v.n), xi+, xix, rotated, times -T_l/2
        double un[kDfF], vn[kDfF], T[kDfF];
        for (int k = 0; k < kDfF; ++k) {
            un[k] = a.sky.u[0] * sm.comp[c][3][k] + a.sky.u[1] * sm.comp[c][4][k] + a.sky.u[2] * sm.comp[c][5][k];
            vn[k] = a.sky.v[0] * sm.comp[c][3][k] + a.sky.v[1] * sm.comp[c][4][k] + a.sky.v[2] * sm.comp[c][5][k];
            T[k] = -0.5 * sm.comp[c][0][k];
        }
        double uu[kDfF], vv[kDfF], uv[kDfF], gp[kDfF], gc[kDfF], Fp[kDfF], Fc[kDfF];
        poly_mul<kDfF>(un, un, uu);
        poly_mul<kDfF>(vn, vn, vv);
        poly_mul<kDfF>(un, vn, uv);
        for (int k = 0; k < kDfF; ++k) {
            const double xp = uu[k] - vv[k], xc = 2.0 * uv[k];
            gp[k] = xp * a.sky.c2p + xc * a.sky.s2p;
            gc[k] = xc * a.sky.c2p - xp * a.sky.s2p;
        }
        poly_mul<kDfF>(T, gp, Fp);
        poly_mul<kDfF>(T, gc, Fc);
        for (int k = 0; k < kDfF; ++k) {
            R.fp[k] = df_of(Fp[k]);
            R.fc[k] = df_of(Fc[k]);
        }
    }
    __syncthreads();
    // retarded samples of the six series at each tile's two ends (2-sample
    // halos included), FP64
    if (t < 12 * nt) {
        const int q = t / 12, e = t % 12, c = e % 6;
        const int64_t i0 = (t0 + q) * (int64_t)kTile;
        const int64_t m = (e < 6) ? i0 - 2 : i0 + kTile + 1;
        const double u = (double)(m - ic) * (2.0 / a.tab.S);
        const double d = horner_d<kDfD>(sm.dp64[c], u);
        int64_t j;
        double eps;
        split_f64(a.hm, m, d, j, eps);
        sm.jends[q][e] = j;
    }
    if (t == 128) {
        // the weight 1 / (1 + e^arg) is 1 to FP64 precision for arg <= -40;
        // arg is monotonic in the sample index: its two ends decide
        int on = 0;
        if (a.bl.enabled) {
            const int64_t i_a = t0 * (int64_t)kTile, i_b = (t0 + nt) * (int64_t)kTile - 1;
            const double ta = a.t0_out + (double)i_a * a.dt_out, tb = a.t0_out + (double)i_b * a.dt_out;
            const double ga = a.bl.eps * (ta - a.bl.t_hyb) / a.bl.sigma, gb = a.bl.eps * (tb - a.bl.t_hyb) / a.bl.sigma;
            on = (ga > -41.0 || gb > -41.0) ? 1 : 0;
        }
        sm.blend = on;
    }
    __syncthreads();
    if (t < nt) {
        int64_t lo = sm.jends[t][0], hi = sm.jends[t][0];
        for (int k = 1; k < 12; ++k) {
            lo = sm.jends[t][k] < lo ? sm.jends[t][k] : lo;
            hi = sm.jends[t][k] > hi ? sm.jends[t][k] : hi;
        }
        DfWin& w = sm.win[t];
        w.wlo = lo - 15 - 3;
        const int64_t len = (hi + 16 + 3) - w.wlo + 1;
        w.wlen = (len <= kWinH) ? (int)len : 0;
    }
    __syncthreads();
}

// hdot at h-grid sample idx in FP64 from global memory (zero off the grid).
__device__ __forceinline__ double df_hdot_global(const double* __restrict__ h, int64_t n, int64_t idx, double i12)
{
    if (idx < 0 || idx >= n) return 0.0;
    auto at = [&](int64_t k) { return (k >= 0 && k < n) ? h[k] : 0.0; };
    return ((at(idx + 1) - at(idx - 1)) * 8.0 - (at(idx + 2) - at(idx - 2))) * i12;
}

// (h+ hi, hx hi, h+ lo, hx lo): the two polarisations' high parts, then
// their low parts, as the register pairs of the packed tap arithmetic.
__device__ __forceinline__ float4 df_pack(double p, double c)
{
    const df a = df_of(p), b = df_of(c);
    return make_float4(a.hi, b.hi, a.lo, b.lo);
}

// hdot on the window of one tile (FP64 from h in global memory, kept as
// double-floats) into buffer dw, and each warp's largest |high part| of either
// polarisation into wm[warp].  No synchronisation.
static __device__ void df_stage(const LfaArgs& a, const DfWin& w, float4* __restrict__ dw, float2* __restrict__ wm)
{
    const double* __restrict__ hp = (const double*)a.hp;
    const double* __restrict__ hc = (const double*)a.hc;
    const double i12 = 1.0 / (12.0 * a.hm.dt_in);
    const int64_t n = a.hm.n_in;
    float mp = 0.f, mc = 0.f;
    for (int k = threadIdx.x; k < w.wlen; k += blockDim.x) {
        const int64_t idx = w.wlo + k;
        const float4 v = df_pack(df_hdot_global(hp, n, idx, i12), df_hdot_global(hc, n, idx, i12));
        dw[k] = v;
        mp = fmaxf(mp, fabsf(v.x));
        mc = fmaxf(mc, fabsf(v.y));
    }
    // non-negative floats order as their bit patterns
    const unsigned int bp = __reduce_max_sync(0xffffffffu, __float_as_uint(mp));
    const unsigned int bc = __reduce_max_sync(0xffffffffu, __float_as_uint(mc));
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = make_float2(__uint_as_float(bp), __uint_as_float(bc));
}

// The splitting constant of one polarisation's outer taps (below) over a
// window whose largest |node| is M, 2^e <= M < 2^(e+1): sigma = 2^(e-2)
// (1 for an all-zero window).
__device__ __forceinline__ float df_split_sigma(float M)
{
    const int e = (int)((__float_as_uint(M) >> 23) & 0xffu);
    if (M == 0.f) return 1.f;
    const int es = e < 3 ? 1 : e - 2;
    return __uint_as_float((unsigned int)(es < 254 ? es : 254) << 23);
}

// 32-point Lagrange interpolation of both polarisations at a double-float
// fraction eps (the paired mirrored-node scheme of lagrange32_paired_f32:
// s = eps - 1/2, e_k = s^2 - (k + 1/2)^2, e_0 = eps (eps - 1), Q_k =
// K_{15-k} prod_{j != k} e_j, w_{15-k} = (s - k - 1/2) Q_k, w_{16+k} =
// -(s + k + 1/2) Q_k), with compensated products.  node(p) gives node p's
// (h+ hi, hx hi, h+ lo, hx lo).  Both polarisations run in packed FP32 pair
// instructions, and the taps are summed exactly in one of two ways:
//  - two-sum of the exact products (Ogita, Rump and Oishi's Dot2), twelve
//    pair instructions a tap: every tap when kSplit is false (any node
//    values), else the eight central ones (pairs k = 0..3, nodes -3..4);
//  - with kSplit, the 24 outer taps (pairs k = 4..15, |w| <= 0.0197 and
//    sum |w| <= 0.0656 for eps in [0, 1], from the Lagrange basis of the 32
//    equispaced nodes): each product w h of the high parts is split against
//    the power of two sigma = 2^(e-2), 2^e <= max|h| over the window < 2^(e+1)
//    (Rump, Ogita and Oishi's ExtractScalar, with the product fused into the
//    split): u = fl(w h + sigma), q = u - sigma exactly (|w h| < sigma / 2,
//    Sterbenz's lemma), the q, multiples of 2^-24 sigma whose partial sums
//    stay below sigma, are summed exactly, and the remainders fl(w h - q) go
//    to the correction sum; seven pair instructions a tap.  The remainders
//    are bounded by 2^-26 max|h|, below the two-sum errors of the central
//    taps, so the correction's rounding stays at the level of Dot2's.  The
//    four outermost of them (pairs 14, 15, |w| <= 2.3e-9) take FP32 weights
//    and plain multiply-adds into the correction sum.
template <bool kSplit, class Node>
__device__ __forceinline__ void lagrange32_df(df eps, Node&& node, float2 sigma, df& op, df& oc)
{
    df s = two_sum(eps.hi, -0.5f);
    s.lo = __fadd_rn(s.lo, eps.lo);
    const df sig = df_mul(s, s);
    auto ek = [&](int k) -> df {   // s^2 - (k + 1/2)^2, k >= 1: |(k + 1/2)^2| > |sig|
        const float c2 = float((k + 0.5) * (k + 0.5));
        const df x = fast_two_sum(-c2, sig.hi);
        return df{x.hi, __fadd_rn(x.lo, sig.lo)};
    };
    df em1 = fast_two_sum(-1.f, eps.hi);   // eps - 1, |1| > |eps|
    em1.lo = __fadd_rn(em1.lo, eps.lo);
    const df e0 = df_mul(eps, em1);
    df S[16];   // S[k] = prod_{j>k} e_j
    S[15] = df{1.f, 0.f};
#pragma unroll
    for (int k = 14; k >= 0; --k) S[k] = df_mul(S[k + 1], ek(k + 1));
    df P = df{1.f, 0.f};   // prod_{j<k} e_j
    // both polarisations at once in packed FP32 pair instructions (one issue
    // slot for two operations): sums (S+, Sx) and corrections (C+, Cx)
    float2 S2 = make_float2(0.f, 0.f), C2 = make_float2(0.f, 0.f);
    const float2 M1 = make_float2(-1.f, -1.f);
    // the outer taps' exact sum, negated (kSplit)
    float2 NS2 = make_float2(0.f, 0.f);
    auto tap = [&](df w, float4 h, bool split) {
        const float2 W = make_float2(w.hi, w.hi), WL = make_float2(w.lo, w.lo);
        const float2 Hh = make_float2(h.x, h.y), Hl = make_float2(h.z, h.w);
        if (split) {
            const float2 U = __ffma2_rn(W, Hh, sigma);        // fl(w h + sigma)
            const float2 NQ = __ffma2_rn(U, M1, sigma);       // sigma - u = -q, exact
            NS2 = __fadd2_rn(NS2, NQ);                         // exact
            C2 = __fadd2_rn(C2, __ffma2_rn(W, Hh, NQ));        // w h - q
        } else {
            const float2 NW = make_float2(-w.hi, -w.hi);
            // exact product: P rounded, Pn = P - w h (minus its rounding error)
            const float2 P = __fmul2_rn(W, Hh);
            const float2 Pn = __ffma2_rn(NW, Hh, P);
            // two-sum of (S, P); x - y as fma(y, -1, x) (exact negation, one rounding)
            const float2 s = __fadd2_rn(S2, P);
            const float2 bb = __ffma2_rn(S2, M1, s);
            const float2 e = __fadd2_rn(__ffma2_rn(__ffma2_rn(bb, M1, s), M1, S2), __ffma2_rn(bb, M1, P));
            S2 = s;
            // corrections: the two-sum error, the product error
            C2 = __fadd2_rn(C2, __ffma2_rn(Pn, M1, e));
        }
        // the cross terms
        C2 = __ffma2_rn(W, Hl, C2);
        C2 = __ffma2_rn(WL, Hh, C2);
    };
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const double Kd = lagrange32_k(15 - k);
        const float Kh = float(Kd), Kl = float(Kd - double(float(Kd)));
        if (kSplit && k >= 14) {
            // the four outermost nodes: |w| <= 2.3e-9, so FP32 weights (a
            // few units of 2^-24 off) move the sum by < 2^-49 max|h|, and the
            // taps go straight into the correction sum
            const float Q = __fmul_rn(__fmul_rn(P.hi, S[k].hi), Kh);
            const float c = float(k + 0.5);
            const float2 W = make_float2(__fmul_rn(__fadd_rn(s.hi, -c), Q), __fmul_rn(__fadd_rn(s.hi, -c), Q));
            const float2 NWr = make_float2(__fmul_rn(__fadd_rn(s.hi, c), Q), __fmul_rn(__fadd_rn(s.hi, c), Q));
            const float4 hl = node(15 - k), hr = node(16 + k);
            C2 = __ffma2_rn(W, make_float2(hl.x, hl.y), C2);
            C2 = __ffma2_rn(NWr, make_float2(-hr.x, -hr.y), C2);
            if (k < 15) P.hi = __fmul_rn(P.hi, ek(k).hi);
            continue;
        }
        const df Q = df_mul(df_mul(P, S[k]), df{Kh, Kl});
        const float c = float(k + 0.5);
        df am = fast_two_sum(-c, s.hi);   // s - c, |c| >= 1/2 >= |s|
        am.lo = __fadd_rn(am.lo, s.lo);
        df ap = fast_two_sum(c, s.hi);    // s + c
        ap.lo = __fadd_rn(ap.lo, s.lo);
        const df wl = df_mul(am, Q);       // w_{15-k}
        df wr = df_mul(ap, Q);             // -w_{16+k}
        wr.hi = -wr.hi;
        wr.lo = -wr.lo;
        tap(wl, node(15 - k), kSplit && k >= 4);
        tap(wr, node(16 + k), kSplit && k >= 4);
        if (k < 15) P = df_mul(P, k == 0 ? e0 : ek(k));
    }
    if (kSplit) {
        const df ap = two_sum(S2.x, -NS2.x), ac = two_sum(S2.y, -NS2.y);
        op = two_sum(ap.hi, __fadd_rn(ap.lo, C2.x));
        oc = two_sum(ac.hi, __fadd_rn(ac.lo, C2.y));
    } else {
        op = fast_two_sum(S2.x, C2.x);
        oc = fast_two_sum(S2.y, C2.y);
    }
}

// z of tile q of the group (first sample i0) and its 2-sample halos: all of
// them on the group's first tile, else those at i0 + 2 .. i0 + kTile + 1 (one
// per thread), the first four coming from the previous tile through halo[q & 1];
// the last four go to halo[(q + 1) & 1] for the next tile.  hdot is read from
// buffer dw (window win).  No synchronisation.
static __device__ void df_zvalues(const LfaArgs& a, int64_t i0, int64_t ic, DfSmem& sm, const DfWin& win,
                                  const float4* __restrict__ dw, int q, bool first)
{
    const int t = threadIdx.x;
    if (!first && t >= 32 && t < 32 + 24) {
        const int c = (t - 32) >> 2, k = (t - 32) & 3;
        sm.zs[q & 1][c][k] = sm.halo[q & 1][c][k];
    }
    const int64_t wlo = win.wlo;
    const int wlen = win.wlen;
    // splitting constants of the staged window's outer taps (from its largest
    // |high part|, the maximum over the warps' maxima)
    float2 sigma;
    {
        float mp = 0.f, mc = 0.f;
#pragma unroll
        for (int k = 0; k < kTile / 32; ++k) {
            const float2 m = sm.wmax[q & 1][k];
            mp = fmaxf(mp, m.x);
            mc = fmaxf(mc, m.y);
        }
        sigma = make_float2(df_split_sigma(mp), df_split_sigma(mc));
    }
    const double* __restrict__ hp = (const double*)a.hp;
    const double* __restrict__ hc = (const double*)a.hc;
    const double i12 = 1.0 / (12.0 * a.hm.dt_in);
    const bool interior = i0 - 2 >= 0 && i0 + kTile + 2 <= a.nout;
    // (series, sample) items, series-major so that a warp's items share a
    // series: the group's first tile has 260 samples, so its items spread
    // 6 or 7 to a thread (one sample per thread with its 6 series would leave
    // 4 threads with 12 evaluations while the block waits for them)
    const int w0 = first ? 0 : 4, nw = kZW - w0;
#pragma unroll 1
    for (int item = threadIdx.x; item < 6 * nw; item += blockDim.x) {
        const int c = item / nw;
        const int w = w0 + item - c * nw;
        const int64_t m = i0 - 2 + w;
        const bool valid = interior || (m >= 0 && m < a.nout);
        const int dm = (int)(m - ic);
        const float u = (float)dm * sm.inv_half;   // exact: S is a power of two
        {
            df z = df{0.f, 0.f};
            if (valid) {
                const DfSer& R = sm.ser[c];
                // position on the h grid: J + dm + f0 - (d(u) - d(0)) / dt
                // d(u) - d(0): d_1, d_2 in double-float, the tail from d_3 in FP32
                const df dv = df_renorm(df_mul_f(df_horner_tail<kDfD - 1, 2>(R.d + 1, u), u));
                const df v = df_sub(R.f0, df_renorm(df_mul(dv, sm.inv_dt)));
                // fraction: v.hi - floor(v.hi) is not exact for negative v.hi
                // (its ulp is finer than that of the fraction), so it is taken
                // by two-sum, with v.lo added to the error term
                float fl = floorf(v.hi);
                const df fr = two_sum(v.hi, -fl);
                df e = two_sum(fr.hi, __fadd_rn(fr.lo, v.lo));
                if (e.hi < 0.f) {
                    fl -= 1.f;
                    e = df_add(e, df{1.f, 0.f});
                } else if (e.hi >= 1.f) {
                    fl += 1.f;
                    e = df_add(e, df{-1.f, 0.f});
                }
                const int64_t j = sm.J[c] + dm + (int64_t)fl;
                const int64_t base = j - 15 - wlo;
                df ip, ic2;
                if (wlen > 0 && base >= 0 && base + 32 <= wlen) {
                    const float4* nb = dw + base;
                    lagrange32_df<true>(e, [&](int p) { return nb[p]; }, sigma, ip, ic2);
                } else {
                    lagrange32_df<false>(e, [&](int p) {
                        const int64_t q = j - 15 + p;
                        return df_pack(df_hdot_global(hp, a.hm.n_in, q, i12), df_hdot_global(hc, a.hm.n_in, q, i12));
                    }, sigma, ip, ic2);
                }
                // factors: F_0..F_2 in double-float, the tail from F_3 in FP32
                const df Fp = df_horner_tail<kDfF, 3>(R.fp, u), Fc = df_horner_tail<kDfF, 3>(R.fc, u);
                z = df_add(df_renorm(df_mul(Fp, ip)), df_renorm(df_mul(Fc, ic2)));
            }
            sm.zs[q & 1][c][w] = z;
            if (w >= kTile) sm.halo[(q + 1) & 1][c][w - kTile] = z;
        }
    }
}

// Channels of sample i0 + t from the tile's z buffer zs, stored with AET and
// the blend (FP64).
static __device__ void df_channels(const LfaArgs& a, int64_t i0, int64_t ic, const DfSmem& sm,
                                   const df (*__restrict__ zs)[kZW])
{
    const int t = threadIdx.x;
    const int64_t i = i0 + t;
    if (!a.xyz || i < a.i_begin || i >= a.i_end) return;
    const float u = (float)(int)(i - ic) * sm.inv_half;
    const bool tdi20 = a.gen == LISA_TDI20;
    const df k1 = sm.k1, k2 = sm.k2;
    // the three light times, each entering two channels (once each: 2.12 ->
    // 2.09 ms on one year at 5 s against one evaluation per channel and arm)
    const df T0 = df_horner_tail<kDfF, 3>(sm.arm[0], u), T1 = df_horner_tail<kDfF, 3>(sm.arm[1], u),
             T2 = df_horner_tail<kDfF, 3>(sm.arm[2], u);
    auto arm_T = [&](int k) { return k == 0 ? T0 : (k == 1 ? T1 : T2); };
    df X[3];
#pragma unroll 1
    for (int ch = 0; ch < 3; ++ch) {
        const df Ta = arm_T(lfa_arm(ch, 0) >> 1);
        const df Tb = arm_T(lfa_arm(ch, 1) >> 1);
        df R[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const df* z = zs[2 * ch + q] + t;   // z[0..4] = z at i-2 .. i+2
            if (tdi20) {
                // 5-point second derivative as (14 d2_0 - d2_-1 - d2_1)/12, d2 from first differences
                const df e0 = df_sub(z[1], z[0]), e1 = df_sub(z[2], z[1]), e2 = df_sub(z[3], z[2]), e3 = df_sub(z[4], z[3]);
                const df m1 = df_sub(e1, e0), c0 = df_sub(e2, e1), p1 = df_sub(e3, e2);
                R[q] = df_renorm(df_mul(df_sub(df_renorm(df_mul_f(c0, 14.f)), df_add(m1, p1)), k2));
            } else {
                const df d31 = df_sub(z[3], z[1]), d40 = df_sub(z[4], z[0]);
                R[q] = df_renorm(df_mul(df_sub(df_renorm(df_mul_f(d31, 8.f)), d40), k1));
            }
        }
        const df diff = df_sub(df_renorm(df_mul(Ta, R[0])), df_renorm(df_mul(Tb, R[1])));
        X[ch] = tdi20 ? df_renorm(df_mul(df_renorm(df_mul_f(df_add(Ta, Tb), 8.f)), diff))
                      : df_renorm(df_mul_f(diff, 4.f));
    }
    double o[3];
    if (a.channels == LISA_AET) {
        const df r2 = df_of(0.70710678118654752440), r6 = df_of(0.40824829046386301637),
                 r3 = df_of(0.57735026918962576451);
        o[0] = df_to_double(df_renorm(df_mul(df_sub(X[2], X[0]), r2)));
        o[1] = df_to_double(df_renorm(df_mul(df_add(df_sub(X[0], df_renorm(df_mul_f(X[1], 2.f))), X[2]), r6)));
        o[2] = df_to_double(df_renorm(df_mul(df_add(df_add(X[0], X[1]), X[2]), r3)));
    } else {
        for (int ch = 0; ch < 3; ++ch) o[ch] = df_to_double(X[ch]);
    }
    if (sm.blend) {
        const double ti = a.t0_out + (double)i * a.dt_out;
        const double arg = a.bl.eps * (ti - a.bl.t_hyb) / a.bl.sigma;
        if (arg > -40.0) {   // below, 1 / (1 + e^arg) is 1 to FP64 precision
            const double wgt = 1.0 / (1.0 + exp(arg));
            for (int ch = 0; ch < 3; ++ch) o[ch] *= wgt;
        }
    }
    double* out = (double*)a.xyz;
    out[i] = o[0];
    out[a.nout + i] = o[1];
    out[2 * a.nout + i] = o[2];
}

// One barrier per tile: iteration q forms the channels of tile q - 1 (buffer
// (q - 1) & 1), the z of tile q (buffer q & 1) and stages the hdot window of
// tile q + 1 (buffer (q + 1) & 1, last read by the z of tile q - 1), so a warp
// goes from one part to the next instead of waiting at a barrier between
// them.  In this order (channels, z, staging) the LFA call on one year at
// 5 s took 2.122 ms against 2.152 ms for z, channels, staging and 2.146 ms
// for staging first.
__global__ void __launch_bounds__(kTile, LISA_DF_MINB) lfa_kernel_df(LfaArgs a, int64_t tile_end, int G)
{
    extern __shared__ __align__(16) unsigned char df_raw[];
    DfSmem& sm = *reinterpret_cast<DfSmem*>(df_raw);
    const int64_t t0 = a.tile0 + (int64_t)blockIdx.x * G;
    const int64_t ic = t0 * kTile + (int64_t)G * kTile / 2;
    const int nt = (int)(tile_end - t0 < G ? tile_end - t0 : G);
    df_prologue(a, t0, nt, ic, sm);
    df_stage(a, sm.win[0], sm.dw[0], sm.wmax[0]);
    __syncthreads();
    for (int q = 0; q < nt; ++q) {
        const int64_t i0 = (t0 + q) * (int64_t)kTile;
        if (q > 0) df_channels(a, i0 - kTile, ic, sm, sm.zs[(q - 1) & 1]);
        df_zvalues(a, i0, ic, sm, sm.win[q], sm.dw[q & 1], q, q == 0);
        if (q + 1 < nt) df_stage(a, sm.win[q + 1], sm.dw[(q + 1) & 1], sm.wmax[(q + 1) & 1]);
        __syncthreads();   // z of tile q complete, channels of q - 1 read, window of q + 1 staged
    }
    df_channels(a, (t0 + nt - 1) * (int64_t)kTile, ic, sm, sm.zs[(nt - 1) & 1]);
}

int launch_lfa_df(const LfaArgs& a, cudaStream_t st)
{
    static bool attr[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    const int d = dev < 64 ? dev : 63;
    if (!attr[d]) {
        const cudaError_t e = cudaFuncSetAttribute(lfa_kernel_df, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)sizeof(DfSmem));
        if (e != cudaSuccess) return cuda_status(e, "lfa_kernel_df shared memory");
        attr[d] = true;
    }
    const int64_t tiles = (a.i_end - 1) / kTile - a.tile0 + 1;
    const int64_t tile_end = a.tile0 + tiles;
    const int G = lfa_group_df(a.dt_out);
    lfa_kernel_df<<<(unsigned)((tiles + G - 1) / G), kTile, sizeof(DfSmem), st>>>(a, tile_end, G);
    return cuda_status(cudaGetLastError(), "lfa_kernel_df launch");
}

}  // namespace lisa
