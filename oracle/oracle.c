/*
 * Plain FP64 CPU oracle of the time-domain LISA response
 * (Valencia & Husa, arXiv:2505.09600).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this code; the library under test never
 * does, and the two share no source, header, table or helper.
 *
 * Every function restates one definition of the paper in the paper's order
 * and notation, written for clarity rather than speed:
 *   - no blocking, no fusion, no reordering beyond the definitions;
 *   - Lagrange weights by the direct product formula (O(32^2) per point);
 *   - spacecraft positions evaluated exactly at every time they are needed
 *     (Kepler's equation solved by Newton iteration to convergence);
 *   - light times by fixed-point iteration to convergence.
 * Compiled with -O2 -ffp-contract=off (no FMA contraction); OpenMP only
 * parallelises independent output samples.
 *
 * Readings where the paper is silent or garbled are stated beside the code
 * (triad signs, orbit model, stencil placement, boundaries, degenerate links).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

#define OG_C 299792458.0
#define OG_AU 1.495978707e11
#define OG_YEAR 31557600.0 /* 365.25 days */
#define OG_PI 3.14159265358979323846

static double og_omega(void) { return 2.0 * OG_PI / OG_YEAR; }

/* Orbital eccentricity that makes the first-order constellation arms equal to
 * L: e = L / (2 sqrt(3) R).  The paper prints e = 0.004811 (Eq. L_of_t); with
 * L = 2.5e9 m this gives 0.004825.  The derived value is used. */
double og_eccentricity(double L_m) { return L_m / (2.0 * sqrt(3.0) * OG_AU); }

/* Link index li = 0..5 <-> l = +1,-1,+2,-2,+3,-3.  sgn(l) = eps_{s|l|r}
 * (Sec. II A): y_312, y_2-13, y_123, y_3-21, y_231, y_1-32.
 * Spacecraft indices are 0-based here (S/C 1 -> 0). */
static const int og_sender[6] = {2, 1, 0, 2, 1, 0};
static const int og_receiver[6] = {1, 2, 2, 0, 0, 1};

int og_link_sender(int li) { return og_sender[li]; }
int og_link_receiver(int li) { return og_receiver[li]; }

/* Cyclic permutation 1->2->3->1 on |l|, sign kept (Y, Z from X, Sec. II B). */
static int og_perm(int li, int times)
{
    for (int k = 0; k < times; ++k) li = (((li / 2) + 1) % 3) * 2 + (li % 2);
    return li;
}

static double og_dot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ---------------------------------------------------------------------------
 * Orbits (Sec. II B: equal-arm analytic orbits).  The paper uses LDC
 * AnalyticOrbit without printing it; the published Keplerian constellation is
 * used instead:
 *   KEPLER1: first order in e,
 *     x = R cos a + e R/2 [cos(2a - b) - 3 cos b]
 *     y = R sin a + e R/2 [sin(2a - b) - 3 sin b]
 *     z = -sqrt(3) e R cos(a - b),   a = Omega t + kappa0, b = 2 pi n/3 + lambda0
 *   KEPLER2: exact Keplerian ellipses (semi-major axis R, eccentricity e,
 *     inclination asin(sqrt(3) e * tilt)), which reduce to KEPLER1 at first
 *     order; tilt != 1 breaks the equilateral design and makes the arms flex.
 *   STATIC: the KEPLER1 positions frozen at t_static (tests only).
 * ------------------------------------------------------------------------- */
static void og_pos_kepler1(const og_orbit* o, int sc, double t, double out[3])
{
    const double R = OG_AU, e = og_eccentricity(o->L_m);
    const double a = og_omega() * t + o->kappa0;
    const double b = 2.0 * OG_PI * sc / 3.0 + o->lambda0;
    out[0] = R * cos(a) + 0.5 * e * R * (cos(2.0 * a - b) - 3.0 * cos(b));
    out[1] = R * sin(a) + 0.5 * e * R * (sin(2.0 * a - b) - 3.0 * sin(b));
    out[2] = -sqrt(3.0) * e * R * cos(a - b);
}

static double og_kepler_solve(double M, double e)
{
    double E = M + e * sin(M);
    for (int it = 0; it < 60; ++it) {
        double dE = (E - e * sin(E) - M) / (1.0 - e * cos(E));
        E -= dE;
        if (fabs(dE) < 1e-16) break;
    }
    return E;
}

static void og_pos_kepler2(const og_orbit* o, int sc, double t, double out[3])
{
    const double R = OG_AU, e = og_eccentricity(o->L_m);
    const double b = 2.0 * OG_PI * sc / 3.0 + o->lambda0;
    const double M = og_omega() * t + o->kappa0 - b;
    const double E = og_kepler_solve(M, e);
    const double X = R * (cos(E) - e);
    const double Y = R * sqrt(1.0 - e * e) * sin(E);
    const double inc = asin(sqrt(3.0) * e * o->kepler_tilt);
    const double xp = X * cos(inc), yp = Y, zp = -X * sin(inc);
    out[0] = xp * cos(b) - yp * sin(b);
    out[1] = xp * sin(b) + yp * cos(b);
    out[2] = zp;
}

void og_position(const og_orbit* o, int sc, double t, double out[3])
{
    switch (o->kind) {
    case OG_KEPLER2: og_pos_kepler2(o, sc, t, out); break;
    case OG_STATIC: og_pos_kepler1(o, sc, o->t_static, out); break;
    default: og_pos_kepler1(o, sc, t, out); break;
    }
}

/* Light time T_l(t) = L_l(t)/c in seconds (Sec. II B, "optical path along
 * link l").  LIGHTTIME solves T = |R_r(t) - R_s(t - T)| / c by fixed-point
 * iteration, which makes L_l != L_-l (Sagnac).  ANALYTIC is the paper's
 * O(e^2) formula Eq. (L_of_t) with xi0, delta_|l| as parameters and the
 * e-terms scaled by flex_scale.  EQUAL is L/c.  LINEAR is a test model
 * T0 + Tdot (t - t_ref). */
double og_light_time(const og_orbit* o, int li, double t)
{
    const int s = og_sender[li], r = og_receiver[li];
    const int absl = li / 2 + 1;
    const double sgn = (li % 2 == 0) ? 1.0 : -1.0;
    switch (o->delay) {
    case OG_DELAY_EQUAL: return o->L_m / OG_C;
    case OG_DELAY_LINEAR: return o->lin_T0[li] + o->lin_Tdot[li] * (t - o->t_ref);
    case OG_DELAY_ANALYTIC: {
        const double L = o->L_m, e = og_eccentricity(L), W = og_omega();
        const double fs = o->flex_scale;
        double Lt = L + (1.0 / 32.0) * e * L * fs * sin(3.0 * W * t - 3.0 * o->xi0)
                  + ((OG_AU * W * L / OG_C) * sgn - (15.0 / 32.0) * e * L * fs) * sin(W * t - o->delta_l[absl - 1]);
        return Lt / OG_C;
    }
    default: {
        double Rr[3], Rs[3], d[3];
        og_position(o, r, t, Rr);
        og_position(o, s, t, Rs);
        for (int c = 0; c < 3; ++c) d[c] = Rr[c] - Rs[c];
        double T = sqrt(og_dot(d, d)) / OG_C;
        for (int it = 0; it < 50; ++it) {
            og_position(o, s, t - T, Rs);
            for (int c = 0; c < 3; ++c) d[c] = Rr[c] - Rs[c];
            double Tn = sqrt(og_dot(d, d)) / OG_C;
            double dT = Tn - T;
            T = Tn;
            if (fabs(dT) <= 1e-16 * T) break;
        }
        return T;
    }
    }
}

/* Link unit vector n_l(t): from the sender's emission position to the
 * receiver's position, n = (R_r(t) - R_s(t - T_l)) / |...|. */
void og_link_vector(const og_orbit* o, int li, double t, double T, double n[3])
{
    double Rr[3], Rs[3];
    og_position(o, og_receiver[li], t, Rr);
    og_position(o, og_sender[li], t - T, Rs);
    double d[3] = {Rr[0] - Rs[0], Rr[1] - Rs[1], Rr[2] - Rs[2]};
    double norm = sqrt(og_dot(d, d));
    for (int c = 0; c < 3; ++c) n[c] = d[c] / norm;
}

void og_geometry(const og_orbit* o, double t, double* R9, double* T6, double* n18)
{
    for (int s = 0; s < 3; ++s) og_position(o, s, t, R9 + 3 * s);
    for (int li = 0; li < 6; ++li) {
        T6[li] = og_light_time(o, li, t);
        og_link_vector(o, li, t, T6[li], n18 + 3 * li);
    }
}

void og_orbits(const og_orbit* o, og_grid g, double* R, double* T, double* nh)
{
    int64_t n = g.n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double t = g.t0 + (double)i * g.dt;
        double R9[9], T6[6], n18[18];
        og_geometry(o, t, R9, T6, n18);
        for (int q = 0; q < 9; ++q) R[q * n + i] = R9[q];
        for (int q = 0; q < 6; ++q) T[q * n + i] = T6[q];
        for (int q = 0; q < 18; ++q) nh[q * n + i] = n18[q];
    }
}

/* ---------------------------------------------------------------------------
 * Propagation triad (Sec. II A, Eq. 1).  The printed components contradict the
 * stated k = -e_r, u = -e_phi (the printed k has +sin(beta) and the printed u
 * has +cos(lambda) in y, neither orthogonal to the rest).  The definitions in
 * terms of the spherical basis are followed:
 *   k = (-cos b cos l, -cos b sin l, -sin b)
 *   u = ( sin l,       -cos l,        0    )
 *   v = (-sin b cos l, -sin b sin l,  cos b)
 * ------------------------------------------------------------------------- */
void og_sky_basis(double beta, double lam, double* k, double* u, double* v)
{
    k[0] = -cos(beta) * cos(lam); k[1] = -cos(beta) * sin(lam); k[2] = -sin(beta);
    u[0] = sin(lam);              u[1] = -cos(lam);             u[2] = 0.0;
    v[0] = -sin(beta) * cos(lam); v[1] = -sin(beta) * sin(lam); v[2] = cos(beta);
}

/* Antenna patterns (Sec. II A, Eqs. xi_plus, xi_cross). */
void og_antenna(const double* u, const double* v, const double* n, double* xp, double* xc)
{
    double un = og_dot(u, n), vn = og_dot(v, n);
    *xp = un * un - vn * vn;
    *xc = 2.0 * un * vn;
}

/* ---------------------------------------------------------------------------
 * 32-point Lagrange interpolation (the 31st-order interpolator named in
 * Sec. IV A as the accurate reference).  Stencil k = -15..16 around
 * j = floor(x), weights w_k = prod_{m != k} (eps - m)/(k - m), evaluated as a
 * direct product.  eps == 0 returns the sample itself.  Samples outside
 * [0, n) are zero (the paper is silent on boundaries).
 * ------------------------------------------------------------------------- */
static double og_at(const double* h, int64_t n, int64_t k) { return (k >= 0 && k < n) ? h[k] : 0.0; }

void og_weights32(double eps, double* w)
{
    for (int k = -15; k <= 16; ++k) {
        double num = 1.0, den = 1.0;
        for (int m = -15; m <= 16; ++m) {
            if (m == k) continue;
            num *= (eps - (double)m);
            den *= (double)(k - m);
        }
        w[k + 15] = num / den;
    }
}

static double og_apply32(const double* h, int64_t n, int64_t j, double eps, const double* w)
{
    if (eps == 0.0) return og_at(h, n, j);
    double s = 0.0;
    for (int k = -15; k <= 16; ++k) s += w[k + 15] * og_at(h, n, j + k);
    return s;
}

double og_lagrange32(const double* h, int64_t n, int64_t j, double eps)
{
    double w[32];
    og_weights32(eps, w);
    return og_apply32(h, n, j, eps, w);
}

/* Position of the time (t0_out + i dt_out) - d on the grid gin, split into an
 * integer sample j and a fraction eps in [0,1) without ever forming the large
 * absolute time: x = i*rho + b0 - d/dt_in with rho = dt_out/dt_in and
 * b0 = (t0_out - t0_in)/dt_in. */
void og_locate(og_grid gout, int64_t i, double d, og_grid gin, int64_t* j, double* eps)
{
    double A = (double)i * (gout.dt / gin.dt);
    double jA = floor(A);
    double fA = A - jA;
    double b0 = (gout.t0 - gin.t0) / gin.dt;
    double jb = floor(b0);
    double fb = b0 - jb;
    double u = (fA + fb) - d / gin.dt;
    double fu = floor(u);
    *j = (int64_t)jA + (int64_t)jb + (int64_t)fu;
    *eps = u - fu;
}

static double og_interp_at(const double* h, og_grid gin, og_grid gout, int64_t i, double d)
{
    int64_t j; double eps;
    og_locate(gout, i, d, gin, &j, &eps);
    return og_lagrange32(h, gin.n, j, eps);
}

/* ---------------------------------------------------------------------------
 * Full single-link response (Sec. II B, Eqs. H, yslr, delta_s, delta_r):
 *   h+SSB = h+ cos 2psi - hx sin 2psi,  hxSSB = h+ sin 2psi + hx cos 2psi
 *   H_l(t) = xi+_l h+SSB(t) + xix_l hxSSB(t)
 *   delta_s = L_l/c + k.R_s/c,  delta_r = k.R_r/c
 *   y_slr(t) = [H_l(t - delta_s) - H_l(t - delta_r)] / (2 (1 - k.n_l))
 * Geometry (R, L_l, n_l, hence xi) is evaluated at the reception time t; the
 * polarisations are interpolated at the two retarded times, then rotated.
 * A link with 1 - k.n_l < 1e-12 (source within ~1.4e-6 rad of the link
 * direction) returns 0; the paper is silent on that case.
 * ------------------------------------------------------------------------- */
typedef struct {
    const og_orbit* orb;
    double k[3], u[3], v[3], c2p, s2p;
    og_grid gh;
    const double *hp, *hc;
    const double *h3p, *h3c;   /* LFA next-to-leading order: third derivatives of h on gh */
} og_src;

static void og_src_init(og_src* S, const og_orbit* o, const og_sky* sky, og_grid gh, const double* hp, const double* hc)
{
    S->orb = o;
    og_sky_basis(sky->beta, sky->lambda, S->k, S->u, S->v);
    S->c2p = cos(2.0 * sky->psi);
    S->s2p = sin(2.0 * sky->psi);
    S->gh = gh;
    S->hp = hp;
    S->hc = hc;
    S->h3p = NULL;
    S->h3c = NULL;
}

static double og_link_full_at(const og_src* S, og_grid gy, int64_t i, int li)
{
    const double t = gy.t0 + (double)i * gy.dt;
    double Rs[3], Rr[3], n[3];
    og_position(S->orb, og_sender[li], t, Rs);
    og_position(S->orb, og_receiver[li], t, Rr);
    const double T = og_light_time(S->orb, li, t);
    og_link_vector(S->orb, li, t, T, n);
    const double delta_s = T + og_dot(S->k, Rs) / OG_C;
    const double delta_r = og_dot(S->k, Rr) / OG_C;
    const double kn = og_dot(S->k, n);
    if (1.0 - kn < 1e-12) return 0.0;
    double xp, xc;
    og_antenna(S->u, S->v, n, &xp, &xc);

    const double hp_s = og_interp_at(S->hp, S->gh, gy, i, delta_s);
    const double hc_s = og_interp_at(S->hc, S->gh, gy, i, delta_s);
    const double hp_r = og_interp_at(S->hp, S->gh, gy, i, delta_r);
    const double hc_r = og_interp_at(S->hc, S->gh, gy, i, delta_r);

    const double Hs = xp * (hp_s * S->c2p - hc_s * S->s2p) + xc * (hp_s * S->s2p + hc_s * S->c2p);
    const double Hr = xp * (hp_r * S->c2p - hc_r * S->s2p) + xc * (hp_r * S->s2p + hc_r * S->c2p);
    return (Hs - Hr) / (2.0 * (1.0 - kn));
}

void og_links_full(const og_orbit* o, const og_sky* sky, og_grid gh, const double* hp, const double* hc,
                   og_grid gy, double* y, const int64_t* idx, int64_t nidx)
{
    og_src S;
    og_src_init(&S, o, sky, gh, hp, hc);
    const int64_t m = idx ? nidx : gy.n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < m; ++q) {
        const int64_t i = idx ? idx[q] : q;
        for (int li = 0; li < 6; ++li) y[li * m + q] = og_link_full_at(&S, gy, i, li);
    }
}

/* ---------------------------------------------------------------------------
 * Michelson TDI (Sec. II B, Eqs. X1.5 and X2.0).  Each term is a signed link
 * series delayed by an ordered list of link delays.  The lists follow the
 * operator form X1.5 = (A-1)a + (1-B)b, X2.0 = (A-1+AB-BAA)a + (1-B-BA+ABB)b
 * with A = D_-2 D_2, B = D_3 D_-3, a = y_231 + D_3 y_1-32,
 * b = y_3-21 + D_-2 y_123, whose expansion reproduces every delay sum and sign
 * of Eqs. X1.5 and X2.0.
 *   FROZEN (the paper's choice): every L_l is evaluated at the output time t,
 *     so the order does not matter.
 *   NESTED: D_a D_b x(t) = x(t - T_a(t) - T_b(t - T_a(t))), the first listed
 *     delay evaluated at t.  Used for the laser-noise checks only.
 * Link indices: 0:+1 1:-1 2:+2 3:-2 4:+3 5:-3.
 * ------------------------------------------------------------------------- */
typedef struct { int sign, link, nd; int d[8]; } og_term;

static const og_term og_terms[16] = {
    {+1, 5, 3, {3, 2, 4}},                /* + y1-32(t - L-2 - L2 - L3)      */
    {-1, 5, 1, {4}},                      /* - y1-32(t - L3)                 */
    {+1, 4, 2, {3, 2}},                   /* + y231(t - L2 - L-2)            */
    {-1, 4, 0, {0}},                      /* - y231(t)                       */
    {+1, 2, 1, {3}},                      /* + y123(t - L-2)                 */
    {-1, 2, 3, {4, 5, 3}},                /* - y123(t - L-2 - L-3 - L3)      */
    {+1, 3, 0, {0}},                      /* + y3-21(t)                      */
    {-1, 3, 2, {4, 5}},                   /* - y3-21(t - L-3 - L3)           */
    {+1, 5, 5, {3, 2, 4, 5, 4}},          /* + y1-32(t - L-2 - L2 - 2L3 - L-3)          */
    {-1, 5, 7, {4, 5, 3, 2, 3, 2, 4}},    /* - y1-32(t - 2L3 - L-3 - 2L-2 - 2L2)        */
    {+1, 4, 4, {3, 2, 4, 5}},             /* + y231(t - L-2 - L2 - L3 - L-3)            */
    {-1, 4, 6, {4, 5, 3, 2, 3, 2}},       /* - y231(t - L3 - L-3 - 2L-2 - 2L2)          */
    {+1, 2, 7, {3, 2, 4, 5, 4, 5, 3}},    /* + y123(t - 2L-2 - L2 - 2L3 - 2L-3)         */
    {-1, 2, 5, {4, 5, 3, 2, 3}},          /* - y123(t - L3 - L-3 - 2L-2 - L2)           */
    {+1, 3, 6, {3, 2, 4, 5, 4, 5}},       /* + y3-21(t - L-2 - L2 - 2L3 - 2L-3)         */
    {-1, 3, 4, {4, 5, 3, 2}},             /* - y3-21(t - L3 - L-3 - L-2 - L2)           */
};

/* Total delay of term `tm` for channel `ch` at output time t. */
static double og_term_delay(const og_orbit* o, const og_term* tm, int ch, double t, int mode, const double* Tfrozen)
{
    double D = 0.0;
    for (int q = 0; q < tm->nd; ++q) {
        const int li = og_perm(tm->d[q], ch);
        if (mode == OG_NESTED) D += og_light_time(o, li, t - D);
        else D += Tfrozen[li];
    }
    return D;
}

typedef double (*og_yfun)(const void* ctx, int li, int64_t j);

typedef struct { const double* y; int64_t n; } og_yarr;
static double og_yfun_array(const void* ctx, int li, int64_t j)
{
    const og_yarr* A = (const og_yarr*)ctx;
    return (j >= 0 && j < A->n) ? A->y[li * A->n + j] : 0.0;
}

typedef struct { const og_src* S; og_grid gy; } og_ydirect;
static double og_yfun_direct(const void* ctx, int li, int64_t j)
{
    const og_ydirect* D = (const og_ydirect*)ctx;
    if (j < 0 || j >= D->gy.n) return 0.0;
    return og_link_full_at(D->S, D->gy, j, li);
}

/* Interpolate link li (given sample by sample through f) at (t_i - d). */
static double og_interp_y(og_yfun f, const void* ctx, int li, og_grid gy, og_grid gout, int64_t i, double d)
{
    int64_t j; double eps;
    og_locate(gout, i, d, gy, &j, &eps);
    if (eps == 0.0) return f(ctx, li, j);
    double w[32];
    og_weights32(eps, w);
    double s = 0.0;
    for (int k = -15; k <= 16; ++k) s += w[k + 15] * f(ctx, li, j + k);
    return s;
}

static void og_tdi_sample(const og_orbit* o, og_yfun f, const void* ctx, og_grid gy, int gen, int mode,
                          og_grid gout, int64_t i, double* xyz)
{
    const double t = gout.t0 + (double)i * gout.dt;
    double T[6];
    for (int li = 0; li < 6; ++li) T[li] = og_light_time(o, li, t);
    const int nterm = (gen == 20) ? 16 : 8;
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.0;
        for (int q = 0; q < nterm; ++q) {
            const og_term* tm = &og_terms[q];
            const int li = og_perm(tm->link, ch);
            const double D = og_term_delay(o, tm, ch, t, mode, T);
            acc += (double)tm->sign * og_interp_y(f, ctx, li, gy, gout, i, D);
        }
        xyz[ch] = acc;
    }
}

void og_tdi_from_y(const og_orbit* o, og_grid gy, const double* y, int gen, int mode,
                   og_grid gout, double* xyz, const int64_t* idx, int64_t nidx)
{
    og_yarr A = {y, gy.n};
    const int64_t m = idx ? nidx : gout.n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < m; ++q) {
        double v[3];
        og_tdi_sample(o, og_yfun_array, &A, gy, gen, mode, gout, idx ? idx[q] : q, v);
        for (int ch = 0; ch < 3; ++ch) xyz[ch * m + q] = v[ch];
    }
}

/* Same as og_tdi_from_y with every needed link sample recomputed from h
 * (for sampled checks of long series without materialising y). */
void og_tdi_full_direct(const og_orbit* o, const og_sky* sky, og_grid gh, const double* hp, const double* hc,
                        og_grid gy, int gen, int mode, og_grid gout, double* xyz, const int64_t* idx, int64_t nidx)
{
    og_src S;
    og_src_init(&S, o, sky, gh, hp, hc);
    og_ydirect D = {&S, gy};
    const int64_t m = idx ? nidx : gout.n;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < m; ++q) {
        double v[3];
        og_tdi_sample(o, og_yfun_direct, &D, gy, gen, mode, gout, idx ? idx[q] : q, v);
        for (int ch = 0; ch < 3; ++ch) xyz[ch * m + q] = v[ch];
    }
}

/* A, E, T (Sec. II B). */
void og_aet(const double* xyz, double* aet, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) {
        const double X = xyz[i], Y = xyz[n + i], Z = xyz[2 * n + i];
        aet[i] = (Z - X) / sqrt(2.0);
        aet[n + i] = (X - 2.0 * Y + Z) / sqrt(6.0);
        aet[2 * n + i] = (X + Y + Z) / sqrt(3.0);
    }
}

/* ---------------------------------------------------------------------------
 * Low-frequency approximation (Sec. III; App. B).
 *
 * Strain derivative: 5-point central difference on the h grid,
 *   hdot_i = (h_{i-2} - 8 h_{i-1} + 8 h_{i+1} - h_{i+2}) / (12 dt),
 * zero outside the grid (the paper uses numpy.gradient).
 *
 * Link at leading order (Eq. yslr_strain_derivatives):
 *   y_l(t') = -(T_l/2) [xi+_l hdot+SSB(tau) + xix_l hdotxSSB(tau)],
 *   tau = t' - T_l/2 - k.(R_s + R_r)/(2c),
 * with T_l, R, xi evaluated at t' itself.
 *
 * Michelson variables with L_l ~ L_-l (Eqs. X15_nonequal, X20_nonequal), per
 * channel with its two links a, b (X: a = y_123, b = y_231, T_a = T_3,
 * T_b = T_2, all evaluated at the output time t; Y, Z cyclic):
 *   1.5: z_a(t) = y_a(t - T_a - T_b/2), z_b(t) = y_b(t - T_b - T_a/2),
 *        X = 4 [T_a dz_a/dt - T_b dz_b/dt]
 *   2.0: z_a(t) = y_a(t - 2T_a - 3T_b/2), z_b(t) = y_b(t - 2T_b - 3T_a/2),
 *        X = 8 (T_a + T_b) [T_a d2z_a/dt2 - T_b d2z_b/dt2]
 * (the paper's intermediate Eq. with L_-3+L_-2+L_2 is a typo for the tau_2
 * definition; these equations follow tau_2 and Eq. X15_nonequal).  The
 * derivatives of z are 5-point central differences on the output grid, zero
 * outside.  L_{+|l|} stands for the arm.  EQUAL (Eqs. X15_equal, X20_equal)
 * replaces every T_l, including those inside y_l, by the nominal L/c.
 * ------------------------------------------------------------------------- */
void og_hdot(og_grid g, const double* h, double* hd)
{
    for (int64_t i = 0; i < g.n; ++i) {
        hd[i] = (og_at(h, g.n, i - 2) - 8.0 * og_at(h, g.n, i - 1) + 8.0 * og_at(h, g.n, i + 1)
                 - og_at(h, g.n, i + 2)) / (12.0 * g.dt);
    }
}

/* 5-point central second derivative on the grid (the stencil of the TDI 2.0
 * channels), zero outside the grid:
 *   x''_i = (-x_{i-2} + 16 x_{i-1} - 30 x_i + 16 x_{i+1} - x_{i+2}) / (12 dt^2).
 * Applied to hdot it gives the third derivative of h that the next-to-leading
 * terms need; hdot once more gives the second derivative. */
void og_d2(og_grid g, const double* x, double* out)
{
    for (int64_t i = 0; i < g.n; ++i) {
        out[i] = (-og_at(x, g.n, i - 2) + 16.0 * og_at(x, g.n, i - 1) - 30.0 * og_at(x, g.n, i)
                  + 16.0 * og_at(x, g.n, i + 1) - og_at(x, g.n, i + 2)) / (12.0 * g.dt * g.dt);
    }
}

static double og_arm(const og_orbit* o, int li, double t, int kind)
{
    return (kind == OG_LFA_EQUAL) ? o->L_m / OG_C : og_light_time(o, li, t);
}

/* y^LFA_l at time t' = t_i - a (S holds hdot as its series): the leading
 * term -(T_l/2) [xi+ hdot+ + xix hdotx] (Eq. yslr_strain_derivatives) at the
 * expansion point tau_eps = t' - delta_s + eps (delta_s - delta_r), with
 * delta_s = T_l + k.R_s/c and delta_r = k.R_r/c (App. B): eps = 1/2 for the
 * central kinds (Eq. tau_t_dependence), 0 for backward, 1 for forward. */
static double og_link_lfa_at(const og_src* S, og_grid gout, int64_t i, double a, int li, int kind, int pair_mean)
{
    const double tp = (gout.t0 + (double)i * gout.dt) - a;
    double Rs[3], Rr[3], n[3];
    og_position(S->orb, og_sender[li], tp, Rs);
    og_position(S->orb, og_receiver[li], tp, Rr);
    const double Tgeo = og_light_time(S->orb, li, tp);
    og_link_vector(S->orb, li, tp, Tgeo, n);
    const double T = og_arm(S->orb, li, tp, kind);
    double xp, xc;
    og_antenna(S->u, S->v, n, &xp, &xc);
    const double delta_s = T + og_dot(S->k, Rs) / OG_C, delta_r = og_dot(S->k, Rr) / OG_C;
    double d_tau;
    if (kind == OG_LFA_BACKWARD) d_tau = a + delta_s;
    else if (kind == OG_LFA_FORWARD) d_tau = a + delta_r;
    else d_tau = a + 0.5 * T + 0.5 * (og_dot(S->k, Rs) + og_dot(S->k, Rr)) / OG_C;
    double dp = og_interp_at(S->hp, S->gh, gout, i, d_tau);
    double dc = og_interp_at(S->hc, S->gh, gout, i, d_tau);
    if (kind == OG_LFA_NLO) {
        /* m = 1 term of the central series (App. B, Eq. yslr_with_tau_derivatives):
         * -(T/2) (1/3!) [(T/2)(1 - k.n)]^2 d3H/dtau3, with xi at t' as in the
         * leading term and d/dtau read as d/dt.  In the TDI-shifted series the
         * link stands for itself and its reverse (y_123 for y_123 and y_3-21:
         * the channels of Eqs. X15_nonequal and X20_nonequal rest on link
         * reversal), whose leading terms coincide but whose m = 1 terms carry
         * (1 - k.n) and (1 + k.n): the channels take their mean,
         * (T/2)^2 (1 + (k.n)^2) / 6 (pair_mean).  A link at its own time
         * (og_links_lfa_own) keeps its own (1 - k.n). */
        const double kn = og_dot(S->k, n);
        const double kap = pair_mean ? 0.25 * T * T * (1.0 + kn * kn) / 6.0
                                     : 0.25 * T * T * (1.0 - kn) * (1.0 - kn) / 6.0;
        dp += kap * og_interp_at(S->h3p, S->gh, gout, i, d_tau);
        dc += kap * og_interp_at(S->h3c, S->gh, gout, i, d_tau);
    }
    return -0.5 * T * (xp * (dp * S->c2p - dc * S->s2p) + xc * (dp * S->s2p + dc * S->c2p));
}

/* The two links (a, b) and arm indices (T_a, T_b) of channel ch. */
static void og_lfa_channel(int ch, int* la, int* lb, int* ia, int* ib)
{
    *la = og_perm(2, ch);  /* y_123 for X */
    *lb = og_perm(4, ch);  /* y_231 for X */
    *ia = og_perm(4, ch);  /* T_3 for X   */
    *ib = og_perm(2, ch);  /* T_2 for X   */
}

static void og_z_sample(const og_src* S, int gen, int kind, og_grid gout, int64_t i, double* z6)
{
    const double t = gout.t0 + (double)i * gout.dt;
    for (int ch = 0; ch < 3; ++ch) {
        int la, lb, ia, ib;
        og_lfa_channel(ch, &la, &lb, &ia, &ib);
        const double Ta = og_arm(S->orb, ia, t, kind), Tb = og_arm(S->orb, ib, t, kind);
        double sa, sb;
        if (gen == 20) { sa = 2.0 * Ta + 1.5 * Tb; sb = 2.0 * Tb + 1.5 * Ta; }
        else { sa = Ta + 0.5 * Tb; sb = Tb + 0.5 * Ta; }
        z6[2 * ch] = og_link_lfa_at(S, gout, i, sa, la, kind, 1);
        z6[2 * ch + 1] = og_link_lfa_at(S, gout, i, sb, lb, kind, 1);
    }
}

void og_z_lfa(const og_orbit* o, const og_sky* sky, og_grid gh, const double* hdp, const double* hdc,
              int gen, int kind, og_grid gout, double* z, const int64_t* idx, int64_t nidx)
{
    og_src S;
    og_src_init(&S, o, sky, gh, hdp, hdc);
    const int64_t m = idx ? nidx : gout.n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < m; ++q) {
        double z6[6];
        og_z_sample(&S, gen, kind, gout, idx ? idx[q] : q, z6);
        for (int c = 0; c < 6; ++c) z[c * m + q] = z6[c];
    }
}

static void og_tdi_lfa_sample(const og_orbit* o, const double* zwin /*[6][5], i-2..i+2*/, int gen, int kind,
                              og_grid gout, int64_t i, double* xyz)
{
    const double t = gout.t0 + (double)i * gout.dt;
    const double dt = gout.dt;
    for (int ch = 0; ch < 3; ++ch) {
        int la, lb, ia, ib;
        og_lfa_channel(ch, &la, &lb, &ia, &ib);
        const double Ta = og_arm(o, ia, t, kind), Tb = og_arm(o, ib, t, kind);
        const double* za = zwin + (2 * ch) * 5;
        const double* zb = zwin + (2 * ch + 1) * 5;
        if (gen == 20) {
            const double d2a = (-za[0] + 16.0 * za[1] - 30.0 * za[2] + 16.0 * za[3] - za[4]) / (12.0 * dt * dt);
            const double d2b = (-zb[0] + 16.0 * zb[1] - 30.0 * zb[2] + 16.0 * zb[3] - zb[4]) / (12.0 * dt * dt);
            xyz[ch] = 8.0 * (Ta + Tb) * (Ta * d2a - Tb * d2b);
            if (kind == OG_LFA_NLO) {
                /* next term of the TDI 2.0 expansion: the l = +-2 terms of X are
                 * (1 + D_Tb)(1 - D_2Ta)(1 - D_2(Ta+Tb)) y, i.e. around their centre
                 * 2cosh(s Tb/2) 2sinh(s Ta) 2sinh(s (Ta+Tb)) in the derivative s:
                 * 8 Ta (Ta+Tb) [s^2 + s^4 (Tb^2/8 + Ta^2/6 + (Ta+Tb)^2/6)]; l = +-3
                 * alike with Ta <-> Tb.  Fourth derivative: 5-point stencil. */
                const double d4a = (za[0] - 4.0 * za[1] + 6.0 * za[2] - 4.0 * za[3] + za[4]) / (dt * dt * dt * dt);
                const double d4b = (zb[0] - 4.0 * zb[1] + 6.0 * zb[2] - 4.0 * zb[3] + zb[4]) / (dt * dt * dt * dt);
                const double ka = Tb * Tb / 8.0 + Ta * Ta / 6.0 + (Ta + Tb) * (Ta + Tb) / 6.0;
                const double kb = Ta * Ta / 8.0 + Tb * Tb / 6.0 + (Ta + Tb) * (Ta + Tb) / 6.0;
                xyz[ch] += 8.0 * (Ta + Tb) * (Ta * ka * d4a - Tb * kb * d4b);
            }
        } else {
            const double d1a = (za[0] - 8.0 * za[1] + 8.0 * za[3] - za[4]) / (12.0 * dt);
            const double d1b = (zb[0] - 8.0 * zb[1] + 8.0 * zb[3] - zb[4]) / (12.0 * dt);
            xyz[ch] = 4.0 * (Ta * d1a - Tb * d1b);
            if (kind == OG_LFA_NLO) {
                /* TDI 1.5: (1 + D_Tb)(1 - D_2Ta) y around its centre is
                 * 2cosh(s Tb/2) 2sinh(s Ta) = 4 Ta [s + s^3 (Ta^2/6 + Tb^2/8)];
                 * third derivative: 5-point stencil */
                const double d3a = (-za[0] + 2.0 * za[1] - 2.0 * za[3] + za[4]) / (2.0 * dt * dt * dt);
                const double d3b = (-zb[0] + 2.0 * zb[1] - 2.0 * zb[3] + zb[4]) / (2.0 * dt * dt * dt);
                xyz[ch] += 4.0 * (Ta * (Ta * Ta / 6.0 + Tb * Tb / 8.0) * d3a - Tb * (Tb * Tb / 6.0 + Ta * Ta / 8.0) * d3b);
            }
        }
    }
}

void og_tdi_lfa_from_z(const og_orbit* o, og_grid gz, const double* z, int gen, int kind,
                       double* xyz, const int64_t* idx, int64_t nidx)
{
    const int64_t m = idx ? nidx : gz.n;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < m; ++q) {
        const int64_t i = idx ? idx[q] : q;
        double zw[30], v[3];
        for (int c = 0; c < 6; ++c)
            for (int s = 0; s < 5; ++s) zw[c * 5 + s] = og_at(z + c * gz.n, gz.n, i - 2 + s);
        og_tdi_lfa_sample(o, zw, gen, kind, gz, i, v);
        for (int ch = 0; ch < 3; ++ch) xyz[ch * m + q] = v[ch];
    }
}

/* Sampled LFA channels straight from hdot (z recomputed around each sample). */
void og_tdi_lfa_direct(const og_orbit* o, const og_sky* sky, og_grid gh, const double* hdp, const double* hdc,
                       int gen, int kind, og_grid gout, double* xyz, const int64_t* idx, int64_t nidx)
{
    og_src S;
    og_src_init(&S, o, sky, gh, hdp, hdc);
    const int64_t m = idx ? nidx : gout.n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < m; ++q) {
        const int64_t i = idx ? idx[q] : q;
        double zw[30], z6[6], v[3];
        for (int s = 0; s < 5; ++s) {
            const int64_t ii = i - 2 + s;
            if (ii < 0 || ii >= gout.n) { for (int c = 0; c < 6; ++c) zw[c * 5 + s] = 0.0; continue; }
            og_z_sample(&S, gen, kind, gout, ii, z6);
            for (int c = 0; c < 6; ++c) zw[c * 5 + s] = z6[c];
        }
        og_tdi_lfa_sample(o, zw, gen, kind, gout, i, v);
        for (int ch = 0; ch < 3; ++ch) xyz[ch * m + q] = v[ch];
    }
}

/* Next-to-leading order (kind OG_LFA_NLO): the z series with the m = 1 link
 * term (h3: third derivative of h on the h grid, og_d2 of hdot), and sampled
 * channels straight from hdot and h3.  The channel NLO terms are applied by
 * og_tdi_lfa_from_z / og_tdi_lfa_sample for this kind. */
void og_z_lfa_nlo(const og_orbit* o, const og_sky* sky, og_grid gh, const double* hdp, const double* hdc,
                  const double* h3p, const double* h3c, int gen, og_grid gout, double* z, const int64_t* idx,
                  int64_t nidx)
{
    og_src S;
    og_src_init(&S, o, sky, gh, hdp, hdc);
    S.h3p = h3p;
    S.h3c = h3c;
    const int64_t m = idx ? nidx : gout.n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < m; ++q) {
        double z6[6];
        og_z_sample(&S, gen, OG_LFA_NLO, gout, idx ? idx[q] : q, z6);
        for (int c = 0; c < 6; ++c) z[c * m + q] = z6[c];
    }
}

void og_tdi_lfa_direct_nlo(const og_orbit* o, const og_sky* sky, og_grid gh, const double* hdp, const double* hdc,
                           const double* h3p, const double* h3c, int gen, og_grid gout, double* xyz,
                           const int64_t* idx, int64_t nidx)
{
    og_src S;
    og_src_init(&S, o, sky, gh, hdp, hdc);
    S.h3p = h3p;
    S.h3c = h3c;
    const int64_t m = idx ? nidx : gout.n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < m; ++q) {
        const int64_t i = idx ? idx[q] : q;
        double zw[30], z6[6], v[3];
        for (int s5 = 0; s5 < 5; ++s5) {
            const int64_t ii = i - 2 + s5;
            if (ii < 0 || ii >= gout.n) { for (int c = 0; c < 6; ++c) zw[c * 5 + s5] = 0.0; continue; }
            og_z_sample(&S, gen, OG_LFA_NLO, gout, ii, z6);
            for (int c = 0; c < 6; ++c) zw[c * 5 + s5] = z6[c];
        }
        og_tdi_lfa_sample(o, zw, gen, OG_LFA_NLO, gout, i, v);
        for (int ch = 0; ch < 3; ++ch) xyz[ch * m + q] = v[ch];
    }
}

/* Links at their own time with the next-to-leading term (kind OG_LFA_NLO),
 * each with its own (1 - k.n_l). */
void og_links_lfa_own_nlo(const og_orbit* o, const og_sky* sky, og_grid gh, const double* hdp, const double* hdc,
                          const double* h3p, const double* h3c, og_grid gy, double* y, const int64_t* idx,
                          int64_t nidx)
{
    og_src S;
    og_src_init(&S, o, sky, gh, hdp, hdc);
    S.h3p = h3p;
    S.h3c = h3c;
    const int64_t m = idx ? nidx : gy.n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < m; ++q) {
        const int64_t i = idx ? idx[q] : q;
        for (int li = 0; li < 6; ++li) y[li * m + q] = og_link_lfa_at(&S, gy, i, 0.0, li, OG_LFA_NLO, 0);
    }
}

/* Strain-derivative form with the constellation centre (Sec. III, Eqs.
 * X15_with_strain_derivatives, X20_with_strain_derivatives): equal constant
 * arms T = L/c, k.(R_s + R_r)/2c replaced by k.R0/c with R0 the centre of the
 * constellation (the mean of the three spacecraft positions), antenna
 * patterns at t:
 *   X1.5(t) = 2 T^2 [(xi+_3 - xi+_2) d2h+SSB/dt2 + (xix_3 - xix_2) d2hxSSB/dt2](t - 2T - k.R0/c)
 *   X2.0(t) = 8 T^3 [(xi+_3 - xi+_2) d3h+SSB/dt3 + (xix_3 - xix_2) d3hxSSB/dt3](t - 4T - k.R0/c)
 * xi_2, xi_3 of the links +2 (y_123) and +3 (y_231); Y, Z cyclic.  sp, sc
 * hold the derivative of h on the h grid (the 5-point first derivative
 * applied twice for TDI 1.5; the second-derivative stencil applied to hdot
 * for TDI 2.0), interpolated with the 32-point Lagrange weights. */
void og_tdi_strain(const og_orbit* o, const og_sky* sky, og_grid gh, const double* sp, const double* sc, int gen,
                   og_grid gout, double* xyz, const int64_t* idx, int64_t nidx)
{
    og_src S;
    og_src_init(&S, o, sky, gh, sp, sc);
    const double T = o->L_m / OG_C;
    const int64_t m = idx ? nidx : gout.n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < m; ++q) {
        const int64_t i = idx ? idx[q] : q;
        const double t = gout.t0 + (double)i * gout.dt;
        double R0[3] = {0.0, 0.0, 0.0};
        for (int sc3 = 0; sc3 < 3; ++sc3) {
            double R[3];
            og_position(o, sc3, t, R);
            for (int d = 0; d < 3; ++d) R0[d] += R[d] / 3.0;
        }
        const double shift = (gen == 20 ? 4.0 : 2.0) * T + og_dot(S.k, R0) / OG_C;
        const double dp = og_interp_at(sp, gh, gout, i, shift);
        const double dc = og_interp_at(sc, gh, gout, i, shift);
        const double Hp = dp * S.c2p - dc * S.s2p, Hc = dp * S.s2p + dc * S.c2p;   /* SSB frame */
        double xp[6], xc[6];
        for (int li = 0; li < 6; li += 2) {
            double n[3];
            og_link_vector(o, li, t, og_light_time(o, li, t), n);
            og_antenna(S.u, S.v, n, &xp[li], &xc[li]);
        }
        const double pref = gen == 20 ? 8.0 * T * T * T : 2.0 * T * T;
        for (int ch = 0; ch < 3; ++ch) {
            const int l3 = og_perm(4, ch), l2 = og_perm(2, ch);
            xyz[ch * m + q] = pref * ((xp[l3] - xp[l2]) * Hp + (xc[l3] - xc[l2]) * Hc);
        }
    }
}

/* LFA links at their own time t (no TDI shift) from the LFA link formula
 * (Sec. III, Eq. yslr_strain_derivatives) applied to each of the six links
 * with its own T_l, n_l and end positions.  (The paper's LFA channels only
 * need y_+1, y_+2, y_+3; the formula itself holds for every link.) */
void og_links_lfa_own(const og_orbit* o, const og_sky* sky, og_grid gh, const double* hdp, const double* hdc,
                      int kind, og_grid gy, double* y, const int64_t* idx, int64_t nidx)
{
    og_src S;
    og_src_init(&S, o, sky, gh, hdp, hdc);
    const int64_t m = idx ? nidx : gy.n;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < m; ++q) {
        const int64_t i = idx ? idx[q] : q;
        for (int li = 0; li < 6; ++li)
            y[li * m + q] = og_link_lfa_at(&S, gy, i, 0.0, li, kind, 0);
    }
}

/* ---------------------------------------------------------------------------
 * Hybrid (Sec. IV, Eqs. sigmoid, thyb, hybridized_yslr, hybridized_xs):
 *   Sigma(t; tH, sigma, eps) = 1 / (1 + exp(eps (t - tH)/sigma))
 *   X(t) = Sigma(t;+1) X_LFA(t) [t <= tH + T/2] + Sigma(t;-1) X_Full(t) [t >= tH - T/2]
 * taken literally: outside the window the surviving weight is Sigma, not 1.
 * ------------------------------------------------------------------------- */
double og_sigmoid(double t, double tH, double sigma, double eps)
{
    return 1.0 / (1.0 + exp(eps * (t - tH) / sigma));
}

double og_t_hyb(double f_hyb, double mc_s, double tc)
{
    return tc - pow(f_hyb, -8.0 / 3.0) * 5.0 / pow(8.0 * OG_PI, 8.0 / 3.0) * pow(mc_s, -5.0 / 3.0);
}

void og_hybrid_blend(og_grid g, double tH, double Tw, double sigma, int nch,
                     const double* lfa, const double* full, double* out, const int64_t* idx, int64_t nidx)
{
    const int64_t m = idx ? nidx : g.n;
    for (int64_t q = 0; q < m; ++q) {
        const int64_t i = idx ? idx[q] : q;
        const double t = g.t0 + (double)i * g.dt;
        const double wl = (t <= tH + 0.5 * Tw) ? og_sigmoid(t, tH, sigma, +1.0) : 0.0;
        const double wf = (t >= tH - 0.5 * Tw) ? og_sigmoid(t, tH, sigma, -1.0) : 0.0;
        for (int c = 0; c < nch; ++c) {
            double v = 0.0;
            if (wl != 0.0) v += wl * lfa[c * m + q];
            if (wf != 0.0) v += wf * full[c * m + q];
            out[c * m + q] = v;
        }
    }
}
