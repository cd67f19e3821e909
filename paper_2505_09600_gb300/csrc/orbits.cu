// Orbit model on the device and the per-segment orbit polynomial table.
//
// Sec. II B of the paper takes spacecraft positions from an analytic
// equal-arm orbit (LDC AnalyticOrbit, not printed).  The Keplerian
// constellation stands in: first order in e (KEPLER1) or exact ellipses
// (KEPLER2).  Light times follow one of four models (see lisa.h).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "lisa_common.cuh"
#include "lisa_internal.cuh"

namespace lisa {

// ---------------------------------------------------------------------------
// error plumbing (per host thread)
// ---------------------------------------------------------------------------
static thread_local char g_err[512];

void set_error(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

const char* last_error() { return g_err; }

int cuda_status(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return LISA_OK;
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LISA_ENOMEM : LISA_ECUDA;
}

// ---------------------------------------------------------------------------
// host-side parameter preparation
// ---------------------------------------------------------------------------
OrbitDev make_orbit_dev(const lisa_orbit& o)
{
    OrbitDev d;
    memset(&d, 0, sizeof(d));
    d.kind = o.kind;
    d.delay = o.delay;
    d.L = o.L_m;
    d.kappa0 = o.kappa0;
    d.lambda0 = o.lambda0;
    d.tilt = o.kepler_tilt;
    d.t_static = o.t_static;
    d.xi0 = o.xi0;
    for (int q = 0; q < 3; ++q) d.delta[q] = o.delta_l[q];
    d.flex = o.flex_scale;
    d.t_ref = o.t_ref;
    for (int q = 0; q < 6; ++q) {
        d.T0[q] = o.lin_T0[q];
        d.Tdot[q] = o.lin_Tdot[q];
    }
    d.e = o.L_m / (2.0 * sqrt(3.0) * kAU);
    d.omega = 2.0 * kPi / kYear;
    d.sin_inc = sqrt(3.0) * d.e * o.kepler_tilt;
    d.cos_inc = sqrt(1.0 - d.sin_inc * d.sin_inc);
    d.sqrt1me2 = sqrt(1.0 - d.e * d.e);
    return d;
}

// Propagation triad k = -e_r, u = -e_phi, v = -e_theta (Sec. II A).  The
// printed components of k and u have sign slips (the printed k is not
// orthogonal to v, the printed u not to k); the stated definitions are used.
SkyDev make_sky_dev(const lisa_sky& s)
{
    SkyDev d;
    const double cb = cos(s.beta), sb = sin(s.beta), cl = cos(s.lambda), sl = sin(s.lambda);
    d.k[0] = -cb * cl; d.k[1] = -cb * sl; d.k[2] = -sb;
    d.u[0] = sl;       d.u[1] = -cl;      d.u[2] = 0.0;
    d.v[0] = -sb * cl; d.v[1] = -sb * sl; d.v[2] = cb;
    d.c2p = cos(2.0 * s.psi);
    d.s2p = sin(2.0 * s.psi);
    for (int c = 0; c < 3; ++c) {
        d.kf[c] = (float)d.k[c];
        d.uf[c] = (float)d.u[c];
        d.vf[c] = (float)d.v[c];
    }
    d.c2f = (float)d.c2p;
    d.s2f = (float)d.s2p;
    return d;
}

GridMap make_grid_map(const lisa_grid& out, const lisa_grid& in)
{
    GridMap m;
    m.rho = out.dt / in.dt;
    const double b0 = (out.t0 - in.t0) / in.dt;
    const double jb = floor(b0);
    m.jb = (int64_t)jb;
    m.fb = b0 - jb;
    m.dt_in = in.dt;
    m.n_in = in.n;
    m.unit_rho = (m.rho == 1.0);
    return m;
}

int64_t seg_count(int64_t n, int S) { return (n + S - 1) / S; }

// ---------------------------------------------------------------------------
// device orbit model
// ---------------------------------------------------------------------------
__device__ void sc_state(const OrbitDev& o, int sc, double t, double R[3], double V[3], double A[3])
{
    const double Rau = kAU, e = o.e, W = o.omega;
    const double b = 2.0 * kPi * sc / 3.0 + o.lambda0;
    double sb, cb;
    sincos(b, &sb, &cb);
    if (o.kind == LISA_ORB_KEPLER2) {
        // exact ellipse: E - e sin E = M, position in the orbital plane,
        // tilted about its minor axis, rotated by b about the ecliptic pole
        const double M = W * t + o.kappa0 - b;
        double sM, cM;
        sincos(M, &sM, &cM);
        // start at O(e^2) ~ 2.5e-5; Newton squares the error: three steps
        // reach FP64 resolution
        double E = M + e * sM;
        double sE, cE;
#pragma unroll 1
        for (int it = 0; it < 3; ++it) {
            sincos(E, &sE, &cE);
            E -= (E - e * sE - M) / (1.0 - e * cE);
        }
        sincos(E, &sE, &cE);
        const double D = 1.0 - e * cE;
        const double Ed = W / D;
        const double Edd = -e * sE * Ed * Ed / D;
        const double X = Rau * (cE - e), Y = Rau * o.sqrt1me2 * sE;
        const double Xd = -Rau * sE * Ed, Yd = Rau * o.sqrt1me2 * cE * Ed;
        const double Xdd = -Rau * (cE * Ed * Ed + sE * Edd);
        const double Ydd = Rau * o.sqrt1me2 * (-sE * Ed * Ed + cE * Edd);
        const double P[3][3] = {{X, Y, 0}, {Xd, Yd, 0}, {Xdd, Ydd, 0}};
        double* out[3] = {R, V, A};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double xp = P[k][0] * o.cos_inc, yp = P[k][1], zp = -P[k][0] * o.sin_inc;
            out[k][0] = xp * cb - yp * sb;
            out[k][1] = xp * sb + yp * cb;
            out[k][2] = zp;
        }
        return;
    }
    const double tt = (o.kind == LISA_ORB_STATIC) ? o.t_static : t;
    const double a = W * tt + o.kappa0;
    double sa, ca, s2, c2, s1, c1;
    sincos(a, &sa, &ca);
    sincos(2.0 * a - b, &s2, &c2);
    sincos(a - b, &s1, &c1);
    const double r3 = sqrt(3.0) * e * Rau;
    R[0] = Rau * ca + 0.5 * e * Rau * (c2 - 3.0 * cb);
    R[1] = Rau * sa + 0.5 * e * Rau * (s2 - 3.0 * sb);
    R[2] = -r3 * c1;
    if (o.kind == LISA_ORB_STATIC) {
        V[0] = V[1] = V[2] = 0.0;
        A[0] = A[1] = A[2] = 0.0;
        return;
    }
    V[0] = W * (-Rau * sa - e * Rau * s2);
    V[1] = W * (Rau * ca + e * Rau * c2);
    V[2] = W * r3 * s1;
    A[0] = W * W * (-Rau * ca - 2.0 * e * Rau * c2);
    A[1] = W * W * (-Rau * sa - 2.0 * e * Rau * s2);
    A[2] = W * W * r3 * c1;
}

// Light time and unit vector of link li at time t from the receiver's
// position and the sender's position, velocity and acceleration at t.  The
// sender's emission position R_s(t - T) comes from a second-order Taylor
// expansion about t (the dropped third-order term is ~1e-7 m, i.e. ~3e-16 s
// of light time).
__device__ void link_geometry(const OrbitDev& o, int li, double t, const double* Rr, const double* Rs,
                              const double* Vs, const double* As, double* T_out, double* n_out)
{
    double T;
    if (o.delay == LISA_DELAY_EQUAL) {
        T = o.L / kC;
    } else if (o.delay == LISA_DELAY_LINEAR) {
        T = o.T0[li] + o.Tdot[li] * (t - o.t_ref);
    } else if (o.delay == LISA_DELAY_ANALYTIC) {
        const double sg = (li & 1) ? -1.0 : 1.0;
        const double L = o.L, e = o.e, W = o.omega;
        const double Lt = L + (1.0 / 32.0) * e * L * o.flex * sin(3.0 * W * t - 3.0 * o.xi0)
                        + ((kAU * W * L / kC) * sg - (15.0 / 32.0) * e * L * o.flex) * sin(W * t - o.delta[li >> 1]);
        T = Lt / kC;
    } else {
        double d0 = Rr[0] - Rs[0], d1 = Rr[1] - Rs[1], d2 = Rr[2] - Rs[2];
        T = sqrt(d0 * d0 + d1 * d1 + d2 * d2) / kC;
#pragma unroll 1
        for (int it = 0; it < 4; ++it) {
            d0 = Rr[0] - (Rs[0] - T * Vs[0] + 0.5 * T * T * As[0]);
            d1 = Rr[1] - (Rs[1] - T * Vs[1] + 0.5 * T * T * As[1]);
            d2 = Rr[2] - (Rs[2] - T * Vs[2] + 0.5 * T * T * As[2]);
            T = sqrt(d0 * d0 + d1 * d1 + d2 * d2) / kC;
        }
    }
    *T_out = T;
    double d[3];
    for (int c = 0; c < 3; ++c) d[c] = Rr[c] - (Rs[c] - T * Vs[c] + 0.5 * T * T * As[c]);
    const double nrm = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int c = 0; c < 3; ++c) n_out[c] = d[c] / nrm;
}

// Geometry at time t: R_s (9), T_l (6), n_l (18).
__device__ void geometry_exact(const OrbitDev& o, double t, double* q)
{
    double R[3][3], V[3][3], A[3][3];
#pragma unroll 1
    for (int s = 0; s < 3; ++s) {
        sc_state(o, s, t, R[s], V[s], A[s]);
        for (int c = 0; c < 3; ++c) q[kQR + 3 * s + c] = R[s][c];
    }
#pragma unroll 1
    for (int li = 0; li < 6; ++li) {
        const int s = link_sender(li), r = link_receiver(li);
        link_geometry(o, li, t, R[r], R[s], V[s], A[s], &q[kQT + li], &q[kQN + 3 * li]);
    }
}

// Chebyshev fit of one quantity from its values at the 7 first-kind nodes,
// stored as degree-6 monomial coefficients in x in [-1, 1]; cs[j][k] =
// cos(pi j (k + 1/2) / 7).
__device__ void cheb_fit_store(const double* v, const double (*cs)[kNodes], double* dst)
{
    double c[kNodes];
    for (int j = 0; j < kNodes; ++j) {
        double acc = 0.0;
        for (int k = 0; k < kNodes; ++k) acc = fma(v[k], cs[j][k], acc);
        c[j] = (2.0 / kNodes) * acc;
    }
    c[0] *= 0.5;
    dst[0] = c[0] - c[2] + c[4] - c[6];
    dst[1] = c[1] - 3.0 * c[3] + 5.0 * c[5];
    dst[2] = 2.0 * c[2] - 8.0 * c[4] + 18.0 * c[6];
    dst[3] = 4.0 * c[3] - 20.0 * c[5];
    dst[4] = 8.0 * c[4] - 48.0 * c[6];
    dst[5] = 16.0 * c[5];
    dst[6] = 32.0 * c[6];
    dst[7] = 0.0;
}

// One segment per block of 64 threads: spacecraft states at the 7 nodes (21
// threads), light times and link vectors (42 threads), then the 33 fits.
// Returns after writing coef[0 .. kNQ*kNC) of this segment.
__device__ void seg_fit_block(const OrbitDev& o, double t0, double dt, int S, int64_t s, double* coef)
{
    __shared__ double st[kNodes][3][9];       // R, V, A per node and spacecraft
    __shared__ double vals[kNQ][kNodes];
    __shared__ double cb[8];                  // cos(pi m / 14), m = 0..7
    __shared__ double cs[kNodes][kNodes];     // cos(pi j (2k + 1) / 14)
    const int t = threadIdx.x;
    // The 49 cosines of the fit are +-cos(pi m / 14) for m = 0..7: eight FP64
    // cosines per block (each FP64 instruction of a warp takes 16 cycles of
    // the SM's FP64 pipe, so they are not recomputed per quantity).
    if (t < 8) cb[t] = (t == 7) ? 0.0 : cospi(t / 14.0);
    __syncthreads();
    if (t < kNodes * kNodes) {
        const int j = t / kNodes, k = t % kNodes;
        int m = (j * (2 * k + 1)) % 28;
        if (m > 14) m = 28 - m;
        cs[j][k] = m <= 7 ? cb[m] : -cb[14 - m];
    }
    __syncthreads();
    auto node_time = [&](int node) {
        const double xk = cs[1][node];
        return t0 + ((double)(s * S) + 0.5 * S + xk * (0.5 * S)) * dt;
    };
    if (t < 3 * kNodes) {
        const int node = t / 3, sc = t % 3;
        double R[3], V[3], A[3];
        sc_state(o, sc, node_time(node), R, V, A);
        for (int c = 0; c < 3; ++c) {
            st[node][sc][c] = R[c];
            st[node][sc][3 + c] = V[c];
            st[node][sc][6 + c] = A[c];
            vals[kQR + 3 * sc + c][node] = R[c];
        }
    }
    __syncthreads();
    if (t < 6 * kNodes) {
        const int node = t / 6, li = t % 6;
        const int sd = link_sender(li), rc = link_receiver(li);
        double T, n[3];
        link_geometry(o, li, node_time(node), &st[node][rc][0], &st[node][sd][0], &st[node][sd][3], &st[node][sd][6],
                      &T, n);
        vals[kQT + li][node] = T;
        for (int c = 0; c < 3; ++c) vals[kQN + 3 * li + c][node] = n[c];
    }
    __syncthreads();
    if (t < kNQ) cheb_fit_store(vals[t], cs, coef + (int64_t)t * kNC);
    __syncthreads();
}

// ---------------------------------------------------------------------------
// segment table: one block (64 threads) per segment
// ---------------------------------------------------------------------------
constexpr int kSegThreads = 64;

__global__ void __launch_bounds__(kSegThreads)
seg_table_kernel(OrbitDev o, double t0, double dt, int S, int64_t nseg, double* __restrict__ coef)
{
    const int64_t s = blockIdx.x;
    if (s >= nseg) return;
    seg_fit_block(o, t0, dt, S, s, coef + s * kNQ * kNC);
}

// The tables of two grids in one launch: blocks [0, n1) fit the segments of
// grid 1, the next n2 blocks those of grid 2 (a block's fit is a chain of
// FP64 latencies, so two short tables cost about one).
__global__ void __launch_bounds__(kSegThreads)
seg_table_pair_kernel(OrbitDev o, double t01, double dt1, int S1, int64_t n1, double* __restrict__ c1, double t02,
                      double dt2, int S2, int64_t n2, double* __restrict__ c2)
{
    const int64_t s = blockIdx.x;
    if (s < n1) seg_fit_block(o, t01, dt1, S1, s, c1 + s * kNQ * kNC);
    else if (s - n1 < n2) seg_fit_block(o, t02, dt2, S2, s - n1, c2 + (s - n1) * kNQ * kNC);
}

int build_seg_table_pair(const OrbitDev& orb, const lisa_grid& g1, int S1, double* c1, int64_t n1,
                         const lisa_grid& g2, int S2, double* c2, int64_t n2, cudaStream_t st)
{
    if (n1 + n2 <= 0) return LISA_OK;
    prof_before("seg_table", st);
    seg_table_pair_kernel<<<(unsigned)(n1 + n2), kSegThreads, 0, st>>>(orb, g1.t0, g1.dt, S1, n1, c1, g2.t0, g2.dt,
                                                                      S2, n2, c2);
    prof_after(st);
    return cuda_status(cudaGetLastError(), "seg_table_pair_kernel launch");
}

int build_seg_table(const OrbitDev& orb, const lisa_grid& g, int S, double* coef_dev, int64_t nseg, cudaStream_t st)
{
    if (nseg <= 0) return LISA_OK;
    prof_before("seg_table", st);
    seg_table_kernel<<<(unsigned)nseg, kSegThreads, 0, st>>>(orb, g.t0, g.dt, S, nseg, coef_dev);
    prof_after(st);
    return cuda_status(cudaGetLastError(), "seg_table_kernel launch");
}

// ---------------------------------------------------------------------------
// batched segment tables: every segment of every source in one launch
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSegThreads)
seg_table_batched_kernel(OrbitDev o, const SegSource* __restrict__ srcs, int nsrc, int64_t total,
                         double* __restrict__ coef)
{
    const int64_t gs = blockIdx.x;
    if (gs >= total) return;
    int lo = 0, hi = nsrc - 1;
    while (lo < hi) {  // last source whose first segment is <= gs
        const int mid = (lo + hi + 1) >> 1;
        if (srcs[mid].seg_begin <= gs) lo = mid; else hi = mid - 1;
    }
    const SegSource& src = srcs[lo];
    seg_fit_block(o, src.t0, src.dt, src.S, gs - src.seg_begin, coef + gs * kNQ * kNC);
}

int build_seg_tables_batched(const OrbitDev& orb, const SegSource* srcs_dev, int nsrc, int64_t total_segs,
                             double* coef_dev, cudaStream_t st)
{
    if (total_segs <= 0) return LISA_OK;
    prof_before("seg_table_batched", st);
    seg_table_batched_kernel<<<(unsigned)total_segs, kSegThreads, 0, st>>>(orb, srcs_dev, nsrc, total_segs, coef_dev);
    prof_after(st);
    return cuda_status(cudaGetLastError(), "seg_table_batched_kernel launch");
}

// ---------------------------------------------------------------------------
// lisa_orbits: materialise R, T, n at every sample (from the table)
// ---------------------------------------------------------------------------
__global__ void orbits_eval_kernel(SegTable tab, int64_t n, double* __restrict__ R, double* __restrict__ T,
                                   double* __restrict__ nh)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t s = i / tab.S;
    const double half = 0.5 * tab.S;
    const double x = ((double)(i - s * tab.S) - half) / half;
    const double* cf = tab.coef + s * kNQ * kNC;
    for (int q = 0; q < kNQ; ++q) {
        const double v = horner_d<7>(cf + q * kNC, x);
        if (q < kQT) { if (R) R[(int64_t)q * n + i] = v; }
        else if (q < kQN) { if (T) T[(int64_t)(q - kQT) * n + i] = v; }
        else if (nh) nh[(int64_t)(q - kQN) * n + i] = v;
    }
}

int run_orbits(const lisa_orbit* orbit, lisa_grid g, double* R, double* T, double* nh, cudaStream_t st)
{
    const OrbitDev od = make_orbit_dev(*orbit);
    const int S = seg_samples(g.dt);
    const int64_t nseg = seg_count(g.n, S);
    Scratch sc(st);
    double* coef = (double*)sc.alloc(sizeof(double) * nseg * kNQ * kNC);
    if (!coef) return sc.status();
    int rc = build_seg_table(od, g, S, coef, nseg, st);
    if (rc) return rc;
    SegTable tab{coef, nseg, S, g.t0, g.dt};
    const int64_t blocks = (g.n + 255) / 256;
    prof_before("orbits_eval", st);
    orbits_eval_kernel<<<(unsigned)blocks, 256, 0, st>>>(tab, g.n, R, T, nh);
    prof_after(st);
    return cuda_status(cudaGetLastError(), "orbits_eval_kernel launch");
}

}  // namespace lisa
