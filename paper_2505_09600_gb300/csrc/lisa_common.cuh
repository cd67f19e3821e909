// Shared device code of liblisa: orbit model, per-segment orbit polynomials,
// tile-local geometry, 32-point Lagrange weights and retarded-time splitting.
//
// Design (GB300, sm_103a):
//  * The orbit quantities R_s(t), T_l(t) = L_l(t)/c and n_l(t) vary on the
//    orbital time scale (1 yr).  They are evaluated exactly (FP64) only at 7
//    Chebyshev nodes per segment of S output samples, by a separate kernel,
//    and stored as degree-6 monomial coefficients in the segment coordinate
//    x in [-1, 1].  Every response kernel re-expands its segment's polynomial
//    around its tile centre and evaluates it per sample (Horner), so per
//    sample there is no trigonometry, no Kepler solve and no light-time
//    iteration.  The truncation error of the degree-6 fit over a segment of
//    up to 330,000 s is ~1e-16 s, below FP64 rounding of the delays.
//  * LISA_F64 kernels keep every step in FP64.  LISA_MIXED kernels keep the
//    tile-centre values of delays in FP64, split once per tile into an
//    integer sample and a fraction, and evaluate the in-tile variation
//    (|dt| < ~0.5 s) and everything downstream in FP32.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lisa.h"

namespace lisa {

constexpr double kC = 299792458.0;
constexpr double kAU = 1.495978707e11;
constexpr double kYear = 31557600.0;  // 365.25 d
constexpr double kPi = 3.14159265358979323846;

// Orbit table quantities: R (3 spacecraft x 3), T (6 links), n (6 links x 3).
constexpr int kNQ = 33;
constexpr int kQR = 0;
constexpr int kQT = 9;
constexpr int kQN = 15;
constexpr int kDeg = 6;      // polynomial degree per segment
constexpr int kNodes = 7;    // Chebyshev nodes per segment
constexpr int kNC = 8;       // stored coefficients per quantity (7 used)
constexpr int kSegSamples = 512;  // smallest segment
// Samples per segment for a grid step dt: the largest power of two <= 65536
// with S*dt <= 330,000 s (at least 512).  Over 330,000 s the orbital phase
// moves by 0.066 rad and the degree-6 Chebyshev fit's truncation
// ~ (Omega W/2)^7 / (2^6 7!) is ~1e-16 of the orbit radius (~1e-5 m, 1e-16 s
// in the light times), below the FP64 evaluation of the exact geometry
// itself; a longer segment only saves table work (7 exact FP64 evaluations
// per segment).
__host__ __device__ inline int seg_samples(double dt)
{
    int S = kSegSamples;
    while (S < 65536 && 2.0 * S * dt <= 330000.0) S *= 2;
    return S;
}

// Link index li = 0..5 <-> l = +1,-1,+2,-2,+3,-3 (y_312, y_2-13, y_123, y_3-21,
// y_231, y_1-32); 0-based spacecraft of sender and receiver.
__host__ __device__ constexpr int link_sender(int li) { return li == 0 ? 2 : li == 1 ? 1 : li == 2 ? 0 : li == 3 ? 2 : li == 4 ? 1 : 0; }
__host__ __device__ constexpr int link_receiver(int li) { return li == 0 ? 1 : li == 1 ? 2 : li == 2 ? 2 : li == 3 ? 0 : li == 4 ? 0 : 1; }
// Cyclic relabelling |l| -> |l| mod 3 + 1 applied `times` (>= 0) times (Y, Z
// from X): the arm index li >> 1 advances by `times` modulo 3, the direction
// bit li & 1 is kept.  Closed form, so that it inlines (a recursive form is
// compiled as an out-of-line call).
__host__ __device__ constexpr int link_cycle(int li, int times)
{
    return (((li >> 1) + times) % 3) * 2 + (li & 1);
}

// Orbit parameters as the kernels use them (derived constants included).
struct OrbitDev {
    int kind, delay;
    double L, kappa0, lambda0, tilt, t_static, xi0, delta[3], flex, t_ref, T0[6], Tdot[6];
    double e, omega, sin_inc, cos_inc, sqrt1me2;
};

OrbitDev make_orbit_dev(const lisa_orbit& o);

// Source geometry on the host, copied by value into kernel arguments.
struct SkyDev {
    double k[3], u[3], v[3];
    double c2p, s2p;
    // FP32 copies for the mixed-precision kernels: converting FP64 values in
    // device code runs on the FP64 pipe (2 per clock per SM on GB300)
    float kf[3], uf[3], vf[3];
    float c2f, s2f;
};
SkyDev make_sky_dev(const lisa_sky& s);

// Polynomial segments of the orbit quantities on an output grid: segment s
// covers samples [s*S, (s+1)*S) of the grid, coordinate x = (q - mid)/half
// with q the (fractional) sample index, mid = s*S + S/2, half = S/2.
struct SegTable {
    const double* coef;  // [nseg][kNQ][kNC]
    int64_t nseg;
    int S;
    double t0, dt;
};

// Position of the time t_i - d of grid `out` on grid `in`, split into an
// integer sample j and a fraction eps in [0, 1):  x = i*rho + b0 - d/dt_in.
struct GridMap {
    double rho;      // dt_out / dt_in
    int64_t jb;      // floor(b0), b0 = (t0_out - t0_in) / dt_in
    double fb;       // b0 - jb
    double dt_in;
    int64_t n_in;
    int unit_rho;    // rho == 1 exactly
};
GridMap make_grid_map(const lisa_grid& out, const lisa_grid& in);

__device__ __forceinline__ void split_f64(const GridMap& m, int64_t i, double d, int64_t& j, double& eps)
{
    double A = (double)i * m.rho;
    double jA = floor(A);
    double fA = __dsub_rn(A, jA);
    double u = __dsub_rn(__dadd_rn(fA, m.fb), __ddiv_rn(d, m.dt_in));
    double fu = floor(u);
    j = (int64_t)jA + m.jb + (int64_t)fu;
    eps = __dsub_rn(u, fu);
}

// 32-point Lagrange weights, stencil k = -15..16 (index p = k + 15):
//   w_p = prod_{m != k}(eps - m)/(k - m) = K_p prod_{m != p} d_m,
//   d_m = eps - (m - 15).  The FP64 form builds A_p = prod_{m<p} d_m / p! and
// B_p = prod_{m>p} (-d_m) / (31 - p)! by a backward then a forward running
// product; the FP32 form pairs mirrored nodes (below).
// K_p = 1 / prod_{m != p} (p - m) = (-1)^(31-p) / (p! (31-p)!), p = 0..31.
__host__ __device__ constexpr double lagrange32_k(int p)
{
    double f = 1.0;
    for (int m = 2; m <= p; ++m) f *= m;
    for (int m = 2; m <= 31 - p; ++m) f *= m;
    return ((31 - p) & 1 ? -1.0 : 1.0) / f;
}

// FP32 form, pairing the nodes that mirror each other about eps = 1/2.  With
// s = eps - 1/2, the nodes 15 - k and 16 + k (k = 0..15) sit at s = -(k + 1/2)
// and s = k + 1/2, so their two differences multiply to
//   e_k = (s + k + 1/2)(s - k - 1/2) = s^2 - (k + 1/2)^2
// (e_0 = eps (eps - 1) directly: no cancellation near eps = 0 or 1), and with
// Q_k = K_{15-k} prod_{j != k} e_j (leave-one-out products by a suffix then a
// prefix pass) and K_{16+k} = -K_{15-k}:
//   w_{15-k} = (s - k - 1/2) Q_k,   w_{16+k} = (-s - k - 1/2) Q_k.
// Every instruction takes at most one constant operand (a factor (c - eps)/n
// would need two, hence a register move each).  About 141 operations for the
// 32 weights; the products stay inside the FP32 range (|e_j| <= 241,
// |Q_k| <= 1).  tap(p, w_p) receives the weights in pairs.
template <class Tap>
__device__ __forceinline__ void lagrange32_paired_f32(float eps, Tap&& tap)
{
    const float s = eps - 0.5f;
    const float sig = s * s;
    float e[16];
    e[0] = eps * (eps - 1.f);
#pragma unroll
    for (int k = 1; k < 16; ++k) e[k] = sig - float((k + 0.5) * (k + 0.5));
    float S[16];   // S[k] = prod_{j>k} e_j
    S[15] = 1.f;
#pragma unroll
    for (int k = 14; k >= 0; --k) S[k] = S[k + 1] * e[k + 1];
    float P = 1.f;   // prod_{j<k} e_j
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const float Q = (P * S[k]) * float(lagrange32_k(15 - k));
        tap(15 - k, (s - float(k + 0.5)) * Q);
        tap(16 + k, (-s - float(k + 0.5)) * Q);
        P *= e[k];
    }
}

template <typename Real>
__device__ __forceinline__ void lagrange32_weights(Real eps, Real (&w)[32])
{
    if constexpr (sizeof(Real) == 4) {
        lagrange32_paired_f32(eps, [&](int p, float v) { w[p] = v; });
    } else {
        // Fully unrolled.  Each factor (c - eps)/n is one fused multiply-add
        // with the compile-time constants -1/n and c/n (instead of a
        // subtraction and a multiplication): the same factor up to the
        // rounding of c/n.
        w[31] = Real(1);
#pragma unroll
        for (int p = 31; p >= 1; --p)
            w[p - 1] = w[p] * fma(eps, Real(-1) / Real(32 - p), Real(p - 15) / Real(32 - p));
        Real A = Real(1);
#pragma unroll
        for (int p = 0; p < 32; ++p) {
            w[p] *= A;
            A *= fma(eps, Real(1) / Real(p + 1), Real(15 - p) / Real(p + 1));
        }
    }
}

// FP32 interpolation of an interleaved pair series: sum_p w_p(eps) v[p] for
// both components, each weight used as soon as it is formed.
__device__ __forceinline__ void lagrange32_dot2(float eps, const float2* __restrict__ v, float& ox, float& oy)
{
    float ax = 0.f, ay = 0.f;
    lagrange32_paired_f32(eps, [&](int p, float w) {
        const float2 hv = v[p];
        ax = fmaf(w, hv.x, ax);
        ay = fmaf(w, hv.y, ay);
    });
    ox = ax;
    oy = ay;
}

// Two samples at once: the weights of eps.x and eps.y are formed as in
// lagrange32_paired_f32 with packed FP32 pair instructions (one instruction
// for both samples, each lane rounded as the scalar operation), and each
// sample's weights are applied to its own interleaved pair series (va for
// eps.x, vb for eps.y).  The mirrored factor -s - k - 1/2 enters as
// -(s + k + 1/2), its sign taken by the tap's fused multiply-add.
__device__ __forceinline__ void lagrange32_dot2_pair(float2 eps, const float2* __restrict__ va,
                                                     const float2* __restrict__ vb, float2& oa, float2& ob)
{
    const float2 s = __fadd2_rn(eps, make_float2(-0.5f, -0.5f));
    const float2 sig = __fmul2_rn(s, s);
    // e_k = s^2 - (k + 1/2)^2 (k >= 1) is one addition: it is formed again in
    // the prefix pass instead of being held in registers between the passes
    auto ek = [&](int k) {
        const float c2 = float((k + 0.5) * (k + 0.5));
        return __fadd2_rn(sig, make_float2(-c2, -c2));
    };
    const float2 e0 = __fmul2_rn(eps, __fadd2_rn(eps, make_float2(-1.f, -1.f)));
    float2 S[16];   // S[k] = prod_{j>k} e_j
    S[15] = make_float2(1.f, 1.f);
#pragma unroll
    for (int k = 14; k >= 0; --k) S[k] = __fmul2_rn(S[k + 1], ek(k + 1));
    float2 P = make_float2(1.f, 1.f);   // prod_{j<k} e_j
    float ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const float K = float(lagrange32_k(15 - k));
        const float c = float(k + 0.5);
        const float2 Q = __fmul2_rn(__fmul2_rn(P, S[k]), make_float2(K, K));
        const float2 wl = __fmul2_rn(__fadd2_rn(s, make_float2(-c, -c)), Q);   // w_{15-k}
        const float2 wr = __fmul2_rn(__fadd2_rn(s, make_float2(c, c)), Q);     // -w_{16+k}
        const float2 al = va[15 - k], ar = va[16 + k];
        const float2 bl = vb[15 - k], br = vb[16 + k];
        ax = fmaf(wl.x, al.x, ax);
        ay = fmaf(wl.x, al.y, ay);
        ax = fmaf(-wr.x, ar.x, ax);
        ay = fmaf(-wr.x, ar.y, ay);
        bx = fmaf(wl.y, bl.x, bx);
        by = fmaf(wl.y, bl.y, by);
        bx = fmaf(-wr.y, br.x, bx);
        by = fmaf(-wr.y, br.y, by);
        if (k < 15) P = __fmul2_rn(P, k == 0 ? e0 : ek(k));
    }
    oa = make_float2(ax, ay);
    ob = make_float2(bx, by);
}

// Two adjacent samples whose stencils start one node apart (sample b's node p
// is sample a's node p + 1): weights as in lagrange32_dot2_pair, and the 33
// distinct values of v[0..32] are read once, each feeding both sums.
__device__ __forceinline__ void lagrange32_dot2_adjacent(float2 eps, const float2* __restrict__ v, float2& oa,
                                                         float2& ob)
{
    const float2 s = __fadd2_rn(eps, make_float2(-0.5f, -0.5f));
    const float2 sig = __fmul2_rn(s, s);
    float2 e[16];
    e[0] = __fmul2_rn(eps, __fadd2_rn(eps, make_float2(-1.f, -1.f)));
#pragma unroll
    for (int k = 1; k < 16; ++k) {
        const float c2 = float((k + 0.5) * (k + 0.5));
        e[k] = __fadd2_rn(sig, make_float2(-c2, -c2));
    }
    float2 S[16];
    S[15] = make_float2(1.f, 1.f);
#pragma unroll
    for (int k = 14; k >= 0; --k) S[k] = __fmul2_rn(S[k + 1], e[k + 1]);
    float2 P = make_float2(1.f, 1.f);
    float ax = 0.f, ay = 0.f, bx = 0.f, by = 0.f;
    float2 pl = v[16], pr = pl;   // v[16 - k] and v[16 + k] of the step before
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const float K = float(lagrange32_k(15 - k));
        const float c = float(k + 0.5);
        const float2 Q = __fmul2_rn(__fmul2_rn(P, S[k]), make_float2(K, K));
        const float2 wl = __fmul2_rn(__fadd2_rn(s, make_float2(-c, -c)), Q);   // w_{15-k}
        const float2 wr = __fmul2_rn(__fadd2_rn(s, make_float2(c, c)), Q);     // -w_{16+k}
        const float2 l = v[15 - k], r = v[17 + k];
        // sample a: nodes 15 - k, 16 + k = v[15 - k], v[16 + k]
        ax = fmaf(wl.x, l.x, ax);
        ay = fmaf(wl.x, l.y, ay);
        ax = fmaf(-wr.x, pr.x, ax);
        ay = fmaf(-wr.x, pr.y, ay);
        // sample b: nodes 15 - k, 16 + k = v[16 - k], v[17 + k]
        bx = fmaf(wl.y, pl.x, bx);
        by = fmaf(wl.y, pl.y, by);
        bx = fmaf(-wr.y, r.x, bx);
        by = fmaf(-wr.y, r.y, by);
        pl = l;
        pr = r;
        if (k < 15) P = __fmul2_rn(P, e[k]);
    }
    oa = make_float2(ax, ay);
    ob = make_float2(bx, by);
}

// Monomial -> re-expansion around xc: b_m = sum_{p>=m} C(p,m) a_p xc^(p-m).
__device__ __forceinline__ void taylor_shift7(const double* a, double xc, double* b)
{
    double t[7];
#pragma unroll
    for (int p = 0; p < 7; ++p) t[p] = a[p];
    // repeated synthetic division by (x - xc)
#pragma unroll
    for (int m = 0; m < 7; ++m) {
#pragma unroll
        for (int p = 5; p >= m; --p) t[p] = fma(t[p + 1], xc, t[p]);
        b[m] = t[m];
    }
}

template <int N>
__device__ __forceinline__ double horner_d(const double* b, double u)
{
    double r = b[N - 1];
#pragma unroll
    for (int p = N - 2; p >= 0; --p) r = fma(r, u, b[p]);
    return r;
}

// Orbit state of spacecraft sc at time t: position, velocity, acceleration.
__device__ void sc_state(const OrbitDev& o, int sc, double t, double R[3], double V[3], double A[3]);
// Exact geometry at time t: 33 quantities (R, T, n) in table order.
__device__ void geometry_exact(const OrbitDev& o, double t, double* q);

// Host-side helpers ----------------------------------------------------------
int build_seg_table(const OrbitDev& orb, const lisa_grid& g, int S, double* coef_dev, int64_t nseg, cudaStream_t st);
int build_seg_table_pair(const OrbitDev& orb, const lisa_grid& g1, int S1, double* c1, int64_t n1,
                         const lisa_grid& g2, int S2, double* c2, int64_t n2, cudaStream_t st);
int64_t seg_count(int64_t n, int S);

// Error plumbing.
void set_error(const char* fmt, ...);
int cuda_status(cudaError_t e, const char* what);

}  // namespace lisa
