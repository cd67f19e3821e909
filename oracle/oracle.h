/*
 * Declarations of the FP64 CPU oracle (test infrastructure only; see oracle.c).
 * This header belongs to the oracle alone; the CUDA library has its own.
 */
#ifndef LISA_ORACLE_H
#define LISA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double t0, dt; int64_t n; } og_grid;

enum { OG_KEPLER1 = 0, OG_KEPLER2 = 1, OG_STATIC = 2 };
enum { OG_DELAY_LIGHTTIME = 0, OG_DELAY_ANALYTIC = 1, OG_DELAY_EQUAL = 2, OG_DELAY_LINEAR = 3 };
enum { OG_FROZEN = 0, OG_NESTED = 1 };
/* LFA kinds: central expansion point (unequal or equal arms), and the
 * non-central variants of App. B ("Other finite differences"): backward
 * (epsilon = 0, tau_0 = t - delta_s) and forward (epsilon = 1, tau_1 = t - delta_r). */
enum { OG_LFA_UNEQUAL = 0, OG_LFA_EQUAL = 1, OG_LFA_BACKWARD = 2, OG_LFA_FORWARD = 3,
       /* App. B next-to-leading order of the central expansion (link and channel terms) */
       OG_LFA_NLO = 4,
       /* Sec. III strain-derivative form with the constellation centre R0 (Eqs.
        * X15_with_strain_derivatives, X20_with_strain_derivatives) */
       OG_LFA_STRAIN = 5 };

typedef struct {
    int32_t kind, delay;
    double L_m;
    double kappa0, lambda0;
    double kepler_tilt;
    double t_static;
    double xi0, delta_l[3], flex_scale;
    double t_ref, lin_T0[6], lin_Tdot[6];
} og_orbit;

typedef struct { double beta, lambda, psi; } og_sky;

double og_eccentricity(double L_m);
int og_link_sender(int li);
int og_link_receiver(int li);
void og_position(const og_orbit* o, int sc, double t, double out[3]);
double og_light_time(const og_orbit* o, int li, double t);
void og_link_vector(const og_orbit* o, int li, double t, double T, double n[3]);
void og_geometry(const og_orbit* o, double t, double* R9, double* T6, double* n18);
void og_orbits(const og_orbit* o, og_grid g, double* R, double* T, double* nh);
void og_sky_basis(double beta, double lam, double* k, double* u, double* v);
void og_antenna(const double* u, const double* v, const double* n, double* xp, double* xc);
void og_weights32(double eps, double* w);
double og_lagrange32(const double* h, int64_t n, int64_t j, double eps);
void og_locate(og_grid gout, int64_t i, double d, og_grid gin, int64_t* j, double* eps);
void og_links_full(const og_orbit* o, const og_sky* sky, og_grid gh, const double* hp, const double* hc,
                   og_grid gy, double* y, const int64_t* idx, int64_t nidx);
void og_tdi_from_y(const og_orbit* o, og_grid gy, const double* y, int gen, int mode,
                   og_grid gout, double* xyz, const int64_t* idx, int64_t nidx);
void og_tdi_full_direct(const og_orbit* o, const og_sky* sky, og_grid gh, const double* hp, const double* hc,
                        og_grid gy, int gen, int mode, og_grid gout, double* xyz, const int64_t* idx, int64_t nidx);
void og_aet(const double* xyz, double* aet, int64_t n);
void og_hdot(og_grid g, const double* h, double* hd);
void og_d2(og_grid g, const double* x, double* out);
void og_z_lfa_nlo(const og_orbit* o, const og_sky* sky, og_grid gh, const double* hdp, const double* hdc,
                  const double* h3p, const double* h3c, int gen, og_grid gout, double* z, const int64_t* idx,
                  int64_t nidx);
void og_tdi_lfa_direct_nlo(const og_orbit* o, const og_sky* sky, og_grid gh, const double* hdp, const double* hdc,
                           const double* h3p, const double* h3c, int gen, og_grid gout, double* xyz,
                           const int64_t* idx, int64_t nidx);
void og_links_lfa_own_nlo(const og_orbit* o, const og_sky* sky, og_grid gh, const double* hdp, const double* hdc,
                          const double* h3p, const double* h3c, og_grid gy, double* y, const int64_t* idx,
                          int64_t nidx);
void og_tdi_strain(const og_orbit* o, const og_sky* sky, og_grid gh, const double* sp, const double* sc, int gen,
                   og_grid gout, double* xyz, const int64_t* idx, int64_t nidx);
void og_z_lfa(const og_orbit* o, const og_sky* sky, og_grid gh, const double* hdp, const double* hdc,
              int gen, int kind, og_grid gout, double* z, const int64_t* idx, int64_t nidx);
void og_tdi_lfa_from_z(const og_orbit* o, og_grid gz, const double* z, int gen, int kind,
                       double* xyz, const int64_t* idx, int64_t nidx);
void og_tdi_lfa_direct(const og_orbit* o, const og_sky* sky, og_grid gh, const double* hdp, const double* hdc,
                       int gen, int kind, og_grid gout, double* xyz, const int64_t* idx, int64_t nidx);
void og_links_lfa_own(const og_orbit* o, const og_sky* sky, og_grid gh, const double* hdp, const double* hdc,
                      int kind, og_grid gy, double* y, const int64_t* idx, int64_t nidx);
double og_sigmoid(double t, double tH, double sigma, double eps);
double og_t_hyb(double f_hyb, double mc_s, double tc);
void og_hybrid_blend(og_grid g, double tH, double Tw, double sigma, int nch,
                     const double* lfa, const double* full, double* out, const int64_t* idx, int64_t nidx);

#ifdef __cplusplus
}
#endif
#endif
