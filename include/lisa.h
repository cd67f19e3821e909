/*
 * lisa.h -- C ABI of the GB300 (sm_103a) time-domain LISA response library
 * (liblisa.so), after Valencia & Husa, "Accelerating the time-domain LISA
 * response model with central finite differences and hybridization
 * techniques", arXiv:2505.09600.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Pointers to series are DEVICE pointers owned by the caller, unless a
 *    parameter says "host".  The library never frees them.
 *  - Every call is asynchronous on `stream` (a cudaStream_t passed as void*;
 *    NULL = legacy default stream) and returns an int status:
 *      LISA_OK (0), LISA_EINVAL (-1, bad argument or shape), LISA_ERANGE (-2),
 *      LISA_ECUDA (-3, a CUDA call failed; see lisa_last_error_message),
 *      LISA_ETIMEOUT (-4, a bounded device-side wait gave up),
 *      LISA_ENOMEM (-5), LISA_ECORRECTOR (-6, corrector fallback used).
 *    Arguments are validated on the host before anything is launched; on an
 *    error nothing is written.  The library never aborts and never prints.
 *  - Time grids: sample i of grid g is at g.t0 + i*g.dt (absolute SSB
 *    seconds, FP64).  Output times are never accumulated.
 *  - Series of several components are stored component-major ("SoA"):
 *    y[c*n + i].  Link order is l = +1,-1,+2,-2,+3,-3, i.e. y_312, y_2-13,
 *    y_123, y_3-21, y_231, y_1-32 (sgn(l) = eps_{s|l|r}, Sec. II A).
 *  - Precision: LISA_F64 = every step in FP64, series are double*.
 *    LISA_MIXED = interpolation, projection, TDI sums and LFA stencils in
 *    FP32 with absolute times, orbit phase and delays kept in FP64 (per tile)
 *    plus an FP32 in-tile offset; series are float*.
 *    LISA_DF = FP64-accurate with series as double*, like LISA_F64: the LFA
 *    channels (lisa_response_lfa, lisa_response_hybrid, lisa_response_hybrid_host,
 *    leading-order kinds on a unit-ratio grid) run in double-float arithmetic
 *    (pairs of FP32 numbers, ~48 significant bits, on the FP32 pipe, with an
 *    FP64 set-up per group of tiles); every other step, and the LFA outside
 *    those cases, runs in FP64 as LISA_F64 does.  Results stay within the FP64
 *    tolerance of the oracle.
 *  - Samples outside an input grid are zero (the paper is silent on
 *    boundaries); every output sample is defined.
 *  - Scratch memory needed inside a call (orbit coefficient table, link or z
 *    series) is taken from the device's stream-ordered pool
 *    (cudaMallocAsync/cudaFreeAsync on `stream`).
 */
#ifndef LISA_H
#define LISA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LISA_OK 0
#define LISA_EINVAL (-1)
#define LISA_ERANGE (-2)
#define LISA_ECUDA (-3)
#define LISA_ETIMEOUT (-4)
#define LISA_ENOMEM (-5)
#define LISA_ECORRECTOR (-6)

/* Uniform time grid: n samples at t0 + i*dt (seconds). */
typedef struct { double t0, dt; int64_t n; } lisa_grid;

/* Orbit models (Sec. II B uses the LDC AnalyticOrbit, whose formula the paper
 * does not print; the published Keplerian constellation stands in):
 *   LISA_ORB_KEPLER1  first order in the eccentricity e = L/(2 sqrt3 AU),
 *   LISA_ORB_KEPLER2  exact Keplerian ellipses, inclination
 *                     asin(sqrt3 e kepler_tilt); kepler_tilt = 1.01 gives
 *                     1% peak-to-peak arm flexing,
 *   LISA_ORB_STATIC   KEPLER1 positions frozen at t_static (tests). */
enum { LISA_ORB_KEPLER1 = 0, LISA_ORB_KEPLER2 = 1, LISA_ORB_STATIC = 2 };
/* Light-time models T_l(t) = L_l(t)/c:
 *   LISA_DELAY_LIGHTTIME  T = |R_r(t) - R_s(t - T)|/c (L_l != L_-l, Sec. II B),
 *   LISA_DELAY_ANALYTIC   the paper's O(e^2) Eq. (L_of_t), e-terms scaled by
 *                         flex_scale, phases xi0 and delta_l[|l|-1],
 *   LISA_DELAY_EQUAL      T = L/c,
 *   LISA_DELAY_LINEAR     T = lin_T0[l] + lin_Tdot[l] (t - t_ref) (tests). */
enum { LISA_DELAY_LIGHTTIME = 0, LISA_DELAY_ANALYTIC = 1, LISA_DELAY_EQUAL = 2, LISA_DELAY_LINEAR = 3 };

typedef struct {
    int32_t kind, delay;
    double L_m;                 /* nominal arm length, metres (2.5e9)          */
    double kappa0, lambda0;     /* orbital and constellation phases, rad       */
    double kepler_tilt;         /* KEPLER2 inclination multiplier (1 = design) */
    double t_static;            /* STATIC freeze time, s                       */
    double xi0, delta_l[3], flex_scale;         /* ANALYTIC only               */
    double t_ref, lin_T0[6], lin_Tdot[6];       /* LINEAR only (s, s/s)        */
} lisa_orbit;

/* Ecliptic latitude beta, longitude lambda, polarisation angle psi (rad). */
typedef struct { double beta, lambda, psi; } lisa_sky;

enum { LISA_F64 = 0, LISA_MIXED = 1, LISA_DF = 2 };
enum { LISA_TDI15 = 15, LISA_TDI20 = 20 };
enum { LISA_XYZ = 0, LISA_AET = 1 };
enum { LISA_FROZEN = 0, LISA_NESTED = 1 };
/* LFA kind.  UNEQUAL and EQUAL expand the link around the central point
 * tau = t - T_l/2 - k.(R_s + R_r)/(2c) (Sec. III, Eq. tau_t_dependence; EQUAL
 * with every T_l = L/c).  BACKWARD and FORWARD are the non-central variants of
 * App. B ("Other finite differences", Eqs. yslr_backward, yslr_forward), with
 * unequal arms: the link's leading term -(T_l/2) Hdot is evaluated at the
 * sender end tau_0 = t - T_l - k.R_s/c (backward, epsilon = 0) or at the
 * receiver end tau_1 = t - k.R_r/c (forward, epsilon = 1); their truncation
 * error is one order lower than the central point's. */
/* NLO (unequal arms, central point) adds the next-to-leading order of both
 * expansions of App. B: the m = 1 term of the central series of the link
 * (Eq. yslr_with_tau_derivatives),
 *   y_l = -(T_l/2) [Hdot + kappa_l d3H/dt3](tau),
 * kappa_l = [T_l (1 - k.n_l)/2]^2 / 6 for a link at its own time and, in the
 * TDI-shifted series, the mean over the link and its reverse,
 * (T_l/2)^2 (1 + (k.n_l)^2) / 6 (the channels rest on link reversal), and the
 * next term of the Michelson expansions:
 *   1.5: X += 4 [T_a (T_a^2/6 + T_b^2/8) d3z_a/dt3 - T_b (T_b^2/6 + T_a^2/8) d3z_b/dt3],
 *   2.0: X += 8 (T_a + T_b) [T_a k_a d4z_a/dt4 - T_b k_b d4z_b/dt4],
 *        k_a = T_b^2/8 + T_a^2/6 + (T_a + T_b)^2/6 (k_b: a <-> b),
 * from expanding the channels' delay operators about their centre.  d3h/dt3
 * is the 5-point second-derivative stencil applied to hdot; d3z/dt3 and
 * d4z/dt4 are 5-point stencils on the output grid.  NLO is an FP64 form:
 * LISA_MIXED returns LISA_EINVAL (the higher stencils amplify FP32 rounding of
 * z beyond the terms they add at low frequency).
 * STRAIN is the strain-derivative form with the constellation centre
 * (Sec. III, Eqs. X15_with_strain_derivatives, X20_with_strain_derivatives):
 * equal constant arms T = L/c and k.(R_s + R_r)/2c replaced by k.R0/c, R0 the
 * mean of the three spacecraft positions:
 *   X1.5 = 2 T^2 [(xi_3 - xi_2) . d2h/dt2](t - 2T - k.R0/c),
 *   X2.0 = 8 T^3 [(xi_3 - xi_2) . d3h/dt3](t - 4T - k.R0/c),
 * (xi_2, xi_3: the links +2, +3 at t; "." the sum over + and x of the SSB
 * polarisations), Y and Z cyclic: one interpolation per sample serves all
 * three channels.  d2h/dt2 is the 5-point first-derivative stencil applied to
 * hdot, d3h/dt3 the second-derivative stencil applied to hdot.  STRAIN has no
 * link series: lisa_links_lfa, lisa_links_lfa_own and lisa_tdi_lfa reject it
 * with LISA_EINVAL. */
enum { LISA_LFA_UNEQUAL = 0, LISA_LFA_EQUAL = 1, LISA_LFA_BACKWARD = 2, LISA_LFA_FORWARD = 3,
       LISA_LFA_NLO = 4, LISA_LFA_STRAIN = 5 };

/* Synthetic source family generated on the device, ahead of the response (the
 * paper's IMRPhenomTHM/TEHM waveforms are not available; this family has their
 * time-domain structure).  A Newtonian (0PN) chirp, masses in seconds
 * (G M / c^3), tau = tc - t:
 *   f = (1/pi)(5/256)^(3/8) Mc^(-5/8) tau^(-3/8),  phi = phi_c - 2 (tau/(5 Mc))^(5/8),
 *   A = 4 c Mc^(5/3) (pi f)^(2/3) / D,  Phi = phi + 4 e_t sin(phi/2),
 *   e_t = e0 (f/f0)^(-19/18) with f0 the frequency at the grid's first sample,
 *   h+ = A (1 + cos^2 iota)/2 cos Phi,  hx = A cos iota sin Phi,
 * up to t_join = tc - tau(f_join), f_join = min(f_ISCO, f_cut) with
 * f_ISCO = 1/(6^(3/2) pi M), M = Mc eta^(-3/5); after it a (2,2,0) damped
 * sinusoid of the remnant (m_final_frac M, spin a_final; Berti-Cardoso-Will
 * fits, frequency capped at f_cut) continuing amplitude and phase. */
typedef struct {
    double mc_s;          /* chirp mass G Mc / c^3 (s), > 0 */
    double q;             /* mass ratio m1 / m2 >= 1 */
    double dist_m;        /* luminosity distance (m), > 0 */
    double iota;          /* inclination (rad) */
    double phi_c;         /* coalescence phase (rad) */
    double tc;            /* coalescence time (s) */
    double e0;            /* eccentricity at the grid's first sample, in [0, 1) (0: circular) */
    double f_cut;         /* cap on the join and ringdown frequencies (Hz); <= 0: none */
    double m_final_frac;  /* remnant mass / total mass, in (0, 1] */
    double a_final;       /* remnant dimensionless spin, in [0, 1) */
} lisa_chirp;

/* Version of this ABI (major*10000 + minor*100 + patch). */
int lisa_version(void);
/* Static message for a status code. */
const char* lisa_strerror(int status);
/* Detail of the last error raised by a call on this host thread (static buffer). */
const char* lisa_last_error_message(void);

/* a1. Spacecraft positions, light times and link unit vectors at every sample
 * of grid g (Sec. II B: R_s(t), L_l(t)/c, n_l(t) with
 * n_l = (R_r(t) - R_s(t - T_l)) / |...|).
 * Output (device, caller-allocated, FP64): R[3][3][n] (spacecraft, xyz, i),
 * T[6][n] light times in seconds, nhat[6][3][n].  Any output may be NULL. */
int lisa_orbits(const lisa_orbit* orbit, lisa_grid g, double* R, double* T, double* nhat, void* stream);

/* a2-a5. Full single-link response (Sec. II A-B, Eqs. H, yslr, delta_s,
 * delta_r): y_l(t) = [H_l(t - delta_s) - H_l(t - delta_r)] / (2 (1 - k.n_l))
 * with h+/hx interpolated by 32-point Lagrange (stencil j-15..j+16 around
 * j = floor of the retarded sample position), geometry at reception time t.
 * hp, hc: device series on h_grid (double* for F64, float* for MIXED).
 * y: device output [6][y_grid.n] of the same type. */
int lisa_links_full(const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid h_grid,
                    const void* hp, const void* hc, int precision,
                    lisa_grid y_grid, void* y, void* stream);

/* a6-a7. Michelson TDI from the six links (Sec. II B, Eqs. X1.5, X2.0; Y, Z
 * by cyclic permutation; A, E, T).  FROZEN evaluates every L_l at the output
 * time (the paper's choice); NESTED applies the delays one after the other,
 * each at its own retarded time.  y: device [6][y_grid.n]; xyz: device
 * [3][out.n] (X,Y,Z or A,E,T). */
int lisa_tdi(const lisa_orbit* orbit, lisa_grid y_grid, const void* y, int precision,
             int tdi_gen, int delay_mode, int channels, lisa_grid out, void* xyz, void* stream);

/* a1-a7 in one call: links on the output grid, then TDI (FROZEN). */
int lisa_response_full(const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid h_grid,
                       const void* hp, const void* hc, int precision, int tdi_gen, int channels,
                       lisa_grid out, void* xyz, void* stream);

/* a8-a9. LFA link series shifted to the TDI retarded times (Sec. III, App. B,
 * Eqs. yslr_strain_derivatives, X15_nonequal, X20_nonequal): per channel
 * c = X,Y,Z and its links a, b (X: y_123, y_231),
 *   z_a(t) = y_a(t - s_a(t)),  y_l(t') = -(T_l/2)[xi+ hdot+SSB(tau) + xix hdotxSSB(tau)],
 *   tau = t' - T_l/2 - k.(R_s + R_r)/(2c),
 * hdot from the 5-point central difference of h on h_grid, interpolated by
 * 32-point Lagrange; s_a = T_a + T_b/2 (1.5) or 2T_a + 3T_b/2 (2.0).
 * EQUAL replaces every T_l by L/c.  z: device [6][out.n] ordered
 * X_a, X_b, Y_a, Y_b, Z_a, Z_b. */
int lisa_links_lfa(const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid h_grid,
                   const void* hp, const void* hc, int precision, int tdi_gen, int lfa_kind,
                   lisa_grid out, void* z, void* stream);

/* The LFA single links at their own reception time t (Sec. III, the LFA
 * link formula applied to each of the six links:
 * y_l(t) = -(T_l/2) [xi+_l hdot+ + xix_l hdotx](tau_l),
 * tau_l = t - T_l/2 - k.(R_s + R_r)/(2c), hdot from the 5-point central
 * stencil of h; the paper's LFA channels need only l = +1, +2, +3).
 * y: device [6][out.n] in link order.  lfa_kind EQUAL uses L/c for T_l. */
int lisa_links_lfa_own(const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid h_grid, const void* hp, const void* hc,
                       int precision, int lfa_kind, lisa_grid out, void* y, void* stream);

/* a10. LFA Michelson variables from z (same passages):
 *   1.5: X = 4 [T_a dz_a/dt - T_b dz_b/dt],
 *   2.0: X = 8 (T_a + T_b) [T_a d2z_a/dt2 - T_b d2z_b/dt2],
 * 5-point central differences on z_grid, arms at the output time. */
int lisa_tdi_lfa(const lisa_orbit* orbit, lisa_grid z_grid, const void* z, int precision,
                 int tdi_gen, int lfa_kind, int channels, void* xyz, void* stream);

/* h+, hx of nsrc draws (host array src[nsrc], nsrc <= 65535) on one grid,
 * into device hp, hc laid out [nsrc][grid.n] (double for LISA_F64, float for
 * LISA_MIXED: FP32 output continuing an FP64 phase anchor per 32 samples).
 * One launch; asynchronous on stream (the parameters are staged before the
 * call returns). */
int lisa_chirp_ringdown(const lisa_chirp* src, int nsrc, lisa_grid grid, int precision, void* hp, void* hc,
                        void* stream);

/* a8-a10 in one call (z kept on chip). */
int lisa_response_lfa(const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid h_grid,
                      const void* hp, const void* hc, int precision, int tdi_gen, int lfa_kind,
                      int channels, lisa_grid out, void* xyz, void* stream);

/* a11. Hybrid response (Sec. IV, Eqs. sigmoid, hybridized_xs):
 *   X(t) = S(t;+1) X_LFA(t) [t <= t_hyb + T_win/2] + S(t;-1) X_Full(t) [t >= t_hyb - T_win/2],
 *   S(t; eps) = 1 / (1 + exp(eps (t - t_hyb)/sigma)),
 * computing the LFA only where its indicator is set and the full response
 * (links and TDI) only where its own is.  T_win <= 0 selects the paper's
 * default 800 out.dt, sigma <= 0 selects T_win/40.  xyz: device [3][out.n].
 * When both parts are present, the full part's links run on a second stream
 * of the library's, forked from `stream` after the orbit table and joined
 * back into `stream` before the TDI: all of the call's work is still ordered
 * on `stream` (event fork and join, so the call can be captured in a graph).
 * That stream and its two events are created by the first such call on a
 * device (and reused); make one call before capturing any in a graph. */
int lisa_response_hybrid(const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid h_grid,
                         const void* hp, const void* hc, int precision, int tdi_gen, int lfa_kind,
                         int channels, double t_hyb, double T_win, double sigma,
                         lisa_grid out, void* xyz, void* stream);

/* No-allocation variant of lisa_response_hybrid (the paper has no
 * counterpart; this is an integration aid).  Some callers may not allocate
 * device memory while they run: an application that gives all device memory
 * to its own pool at start-up and forbids later driver allocations, a
 * latency-bound loop that must not wait on an allocator, or a platform
 * without the stream-ordered allocator.  This call computes exactly what
 * lisa_response_hybrid computes, with the same arguments, but takes its
 * scratch (orbit tables and link series) from one fixed device array of
 * LISA_STATIC_SCRATCH_BYTES inside the library and calls no cudaMalloc,
 * cudaFree or allocating routine.  It builds the same orbit table and the
 * same link range as lisa_response_hybrid and launches the same kernels, so
 * the two give identical outputs.
 *  - The array is resident on every GPU that loads the library until exit.
 *  - A call whose scratch does not fit returns LISA_EINVAL and says how many
 *    bytes it needed (the orbit table, 2.1 KB per segment of up to 65,536
 *    samples, and 6 links over the full part and its TDI reach: a one-year
 *    series at 5 s switched in its last hours needs under 0.5 MB).
 *  - The first call on a device looks up the array's device address (once
 *    per device, with that device current); make that first call before any
 *    stream capture on the device.
 *  - All calls share the array and leave the last call's contents in it:
 *    calls that overlap on the GPU (other streams, other host threads) race
 *    and must be serialised by the caller.  Nothing in it needs clearing;
 *    every call writes all it reads. */
#define LISA_STATIC_SCRATCH_BYTES (16u * 1024u * 1024u)
int lisa_response_hybrid_static(const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid h_grid,
                                const void* hp, const void* hc, int precision, int tdi_gen, int lfa_kind,
                                int channels, double t_hyb, double T_win, double sigma,
                                lisa_grid out, void* xyz, void* stream);

/* lisa_response_hybrid on series in host memory (the paper has no
 * counterpart; an integration aid).  grid is both the h grid and the output
 * grid.  hp, hc: host [grid.n]; xyz: host [3][grid.n] (float for LISA_MIXED,
 * double for LISA_F64).  The grid is cut into up to 8 chunks on the LFA tile
 * groups; the copy of chunk c+1 to the device and the copy of chunk c-1 back
 * run on two internal streams while chunk c is computed on `stream`, so with
 * page-locked host buffers the copies overlap the kernels.  Device buffers
 * come from the stream-ordered allocator on `stream`.  The call returns after
 * queuing; the results are in xyz once `stream` has completed the work
 * queued up to the return.  The values equal lisa_response_hybrid's up to
 * FP32 rounding in the TDI (its blocks follow the chunks). */
int lisa_response_hybrid_host(const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid grid,
                              const void* hp, const void* hc, int precision, int tdi_gen, int lfa_kind,
                              int channels, double t_hyb, double T_win, double sigma, void* xyz, void* stream);

/* ------------------------------------------------------------------------
 * Likelihood tail (Sec. IV steps iv-v; Sec. II C noise model): the Fourier
 * transform of A, E, T and the noise-weighted inner product
 *   <x|y> = 4 Re int_{f_min}^{f_max} df x~*(f) y~(f) / S_n(f)   (Eq. scalar_product),
 * with x~(f) = int dt e^{-2 pi i f t} x(t) (App. A) taken as dt times the
 * discrete transform on the bins f_k = k / (n dt), and the integral as the sum
 * over the bins in [f_min, f_max] times df = 1/(n dt).  The overlap
 * O = <x|y> / sqrt(<x|x><y|y>) and mismatch 1 - |O| (Eq. normalized_overlap)
 * and ln L = -<d - h|d - h>/2 follow from the three products.
 * ------------------------------------------------------------------------ */

/* Noise PSDs of A/E and T (Eqs. SnAE, SnT) from the proof-mass, optical-path
 * and galactic-foreground noises (Sec. II C, Eq. sgal; T_obs in years enters
 * the foreground knees), Lambda = 4 sin^2(2x) for TDI 2.0 and 1 for 1.5,
 * x = 2 pi f L / c.  psd: device double [2][nf] (S^{A,E}, then S^T) at
 * f0 + k df, f0 > 0.  galaxy = 0 drops the foreground. */
int lisa_psd_aet(double f0, double df, int64_t nf, int tdi_gen, double L_m, double t_obs_years, int galaxy,
                 double* psd, void* stream);

/* Smallest 2^a 3^b 5^c 7^d >= n: a transform length that keeps cuFFT on its
 * fast radices (one year at 5 s, 6,311,520 = 2^5 3^3 5 487 samples, pads to
 * 6,322,176 = 2^11 3^2 7^3). */
int64_t lisa_fft_length(int64_t n);

/* Weights of the inner product on the rfft bins of `grid` zero-padded to
 * nfft >= grid.n samples (0: grid.n), nf = nfft/2 + 1, f_k = k / (nfft dt):
 * w[0][k] = 4 df / S^{A,E}(f_k), w[1][k] = 4 df / S^T(f_k) for f_k in
 * [f_min, f_max] and k > 0, else 0.  w: device double [2][nf] for both
 * precisions (S_n ~ 1e-44 puts 4 df / S_n beyond the FP32 range).  Compute
 * once per grid and PSD. */
int lisa_noise_weights_aet(lisa_grid grid, int64_t nfft, int tdi_gen, double L_m, double t_obs_years, int galaxy,
                           double f_min, double f_max, double* w, void* stream);

/* <x|y>, <x|x>, <y|y> for A, E and T: out (device double[9]) =
 * {A: xy, xx, yy; E: ...; T: ...}.  x, y: device [3][grid.n] in the
 * precision's type (y may equal x), zero-padded to nfft >= grid.n samples
 * (0: none) in scratch; w from lisa_noise_weights_aet with the same nfft.
 * Zero padding samples the same continuous transform more finely (on a flat
 * PSD the products are unchanged, by Parseval).  Real FFTs by cuFFT (plans
 * cached per device, length and precision), then one pass over the bins and a
 * fixed-order reduction (run to run identical).  LISA_F64: products and sums
 * in FP64.  LISA_MIXED: a bin's products and weighting in FP32 (spectra
 * scaled by 2^64, weights by 2^-128, both exact), FP32 running sums added to
 * FP64 ones every 16 bins; a bin whose spectrum components leave
 * [2^-92, 2^-1) or whose scaled weight leaves [2^-60, 2^61) is formed in FP64;
 * a thread whose FP32 sums of squares of x (or of y) reach 2^120 recomputes
 * those sums and the cross sums over its bins in FP64, keeping the other
 * operand's (so <x|x> does not depend on y).  Any finite input is accepted.
 * Device scratch from the stream-ordered
 * allocator on `stream`. */
int lisa_inner_aet(lisa_grid grid, int64_t nfft, const void* x, const void* y, int precision, const double* w,
                   double* out, void* stream);

/* Hybridisation time at leading PN order (Sec. IV, Eq. thyb):
 * t_hyb = tc - f^(-8/3) * 5/(8 pi)^(8/3) * (G Mc/c^3)^(-5/3); mc_s = G Mc/c^3 in s. */
double lisa_t_hyb_from_f(double f_hyb, double mc_s, double tc);


/* ------------------------------------------------------------------------
 * Batched hybrid plans: many sources of uneven duration and sampling in one
 * persistent launch (mixed precision), capturable in a CUDA graph, with a
 * launch-shape autotuner.  The paper evaluates one source at a time; this is
 * the same hybrid response (Sec. IV) applied to a batch.
 * ------------------------------------------------------------------------ */
typedef struct {
    lisa_grid grid;              /* h grid, also the output grid (dt >= 0.5 s)          */
    const void* hp;              /* device float[grid.n]                                */
    const void* hc;              /* device float[grid.n]                                */
    lisa_sky sky;
    double t_hyb, T_win, sigma;  /* s; T_win <= 0: 800 dt, sigma <= 0: T_win/40         */
    void* out;                   /* device float[3][grid.n]: X,Y,Z or A,E,T             */
} lisa_source;

typedef struct lisa_plan lisa_plan;
typedef struct { int ctas_per_sm, tiles_per_item; float ms; } lisa_tune_result;

/* Create a plan over `nsrc` sources (host array, copied).  The plan owns its
 * device memory (cudaMalloc at creation: orbit tables of every source, source
 * descriptors, a work counter) until lisa_plan_destroy.  precision must be
 * LISA_MIXED.  Series pointers are borrowed: they must stay valid while the
 * plan executes. */
int lisa_plan_create(lisa_plan** plan, const lisa_orbit* orbit, int precision, int tdi_gen, int lfa_kind,
                     int channels, const lisa_source* sources, int nsrc);
int lisa_plan_destroy(lisa_plan* plan);
/* Enqueue one execution: counter reset, orbit tables, persistent kernel. */
int lisa_plan_execute(lisa_plan* plan, void* stream);
/* Capture one execution on `stream` (non-default) into a CUDA graph;
 * lisa_plan_replay launches it. */
int lisa_plan_capture_graph(lisa_plan* plan, void* stream);
int lisa_plan_replay(lisa_plan* plan, void* stream);
/* Launch shape: CTAs per SM of the persistent kernel (clamped to what fits)
 * and output tiles (256 samples) per work item.  A source's tiles form fixed
 * groups of up to 8 from its start; an item holds tiles_per_item / (group
 * size) whole groups (at least one), so the results do not depend on the
 * launch shape.  Drops a captured graph. */
int lisa_plan_set_launch(lisa_plan* plan, int ctas_per_sm, int tiles_per_item);
/* Time every (CTAs per SM in 1..4) x (tiles per item in 8,16,32,64: 1 to 8 groups) on this
 * plan's own data (synchronising), keep the fastest, report it. */
int lisa_plan_autotune(lisa_plan* plan, void* stream, lisa_tune_result* best);
int lisa_plan_info(const lisa_plan* plan, int64_t* total_samples, int64_t* total_tiles, int* ctas_per_sm,
                   int* tiles_per_item);

/* ------------------------------------------------------------------------
 * Learned corrector of the LFA links (no counterpart in the paper).
 *
 * An MLP 47 -> 64 -> 64 -> 64 -> 6 (GELU, tanh form; BF16 weights and
 * activations on the tensor cores, FP32 accumulation and FP32 master weights)
 * predicts the residuals between the six full single links (Sec. II) and the
 * base links z_l (1 + eps_l) at each output sample, where z_l are the LFA
 * links at their own time (lisa_links_lfa_own) and
 * eps_l = k.v_s / (c (1 - k.n_l)) is the O(v/c) term by which the full
 * formula (positions at the reception time) differs from T_l (1 - k.n_l)
 * (v_s: sender velocity).  Features per sample (47, stored as rows of 48
 * floats, the last one zero):
 *   [ 0,30) q_k,l / M_k: the 5-point stencil of z_l re-based as
 *           q_k = Tbar^k d^k z_l/dt^k, k = 0..4 (feature k*6 + l),
 *           M_k = max_l |q_k,l|;
 *   [30,34) clamp(log10(M_{k+1}/M_k), -8, 8) / 4;
 *   [34,40) (T_l/Tbar - 1) * 100;   [40,46) 1 - k.n_l;   46: dt/Tbar;
 *   Tbar = L/c.
 * Scale s = M_2 / 8; corrected link l = z_l (1 + eps_l) + s * MLP_l.  Local
 * frequency f = sqrt(M_2/M_0) / (2 pi Tbar): below the band [f_lo, f_hi] the
 * base link is used (s = 0), above it the full link (per 256-sample tile).
 * Parameters: a flat FP32 vector, per layer W [n_out][n_in] row-major then b.
 * ---------------------------------------------------------------------- */
typedef struct lisa_corrector lisa_corrector;

int64_t lisa_corrector_num_params(void);     /* 11782 */
int lisa_corrector_num_features(void);       /* 47 */
/* Create on the current device (cudaMalloc of its parameters, Adam state and
 * counters; synchronising).  host_params: n_params FP32 values, or NULL for
 * W ~ U(-1/sqrt(n_in), 1/sqrt(n_in)) drawn from SplitMix64(seed), b = 0.
 * Defaults: band [1e-4, 2e-2] Hz, a spot check every 64th tile (from the
 * first tile whose retarded times stay on the h grid, so that every call
 * checks at least one tile), tolerance 0.05. */
int lisa_corrector_create(lisa_corrector** c, const float* host_params, int64_t n_params, uint64_t seed);
int lisa_corrector_destroy(lisa_corrector* c);
/* Trained band (Hz), spot-check period in tiles (0 = none) and tolerance
 * (max |full - corrected| / max |full| over a tile). */
int lisa_corrector_configure(lisa_corrector* c, double f_lo, double f_hi, int spot_every, double spot_tol);
/* Checkpoint/resume: parameters, Adam moments and step count (host buffers of
 * n_params floats; any pointer may be NULL).  Synchronising. */
int lisa_corrector_get_state(const lisa_corrector* c, float* params, float* adam_m, float* adam_v, int64_t* step,
                             int64_t n_params);
int lisa_corrector_set_state(lisa_corrector* c, const float* params, const float* adam_m, const float* adam_v,
                             int64_t step, int64_t n_params);
/* Features, scale, base links and training targets on grid g from the LFA
 * links z (FP32, [6][g.n], lisa_links_lfa_own with LISA_MIXED).
 * feats: [g.n][48] (16-byte aligned), scale: [g.n], ybase ([6][g.n] or
 * NULL): z_l (1 + eps_l).  If target ([g.n][6]) is given, y_full ([6][g.n]
 * FP64 full links, required) and z_ref ([6][g.n] FP64 LFA links; NULL = z)
 * give target_l = (y_full_l - z_ref_l (1 + eps_l)) / s (0 where s = 0).
 * f_lo/f_hi: band for s (pass 0 and INFINITY for no band). */
int lisa_corrector_features(const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid g, const float* z,
                            const double* y_full, const double* z_ref, double f_lo, double f_hi, float* feats,
                            float* scale, float* ybase, float* target, void* stream);
/* out[r][6] = MLP(feats[r]) for r < M. */
int lisa_corrector_forward(const lisa_corrector* c, const float* feats, int64_t M, float* out, void* stream);
/* grad (device, n_params floats, overwritten) and loss (device float or
 * NULL) of L = mean_r sum_l (MLP(x_r)_l - target_r,l)^2 over either all
 * n_data rows (batch = 0) or `batch` rows drawn as SplitMix64(seed + r) mod n_data. */
int lisa_corrector_gradient(lisa_corrector* c, const float* feats, const float* target, int64_t n_data,
                            int64_t batch, uint64_t seed, float* grad, float* loss, void* stream);
/* One Adam step (beta 0.9/0.999, eps 1e-8, bias-corrected) with rate lr. */
int lisa_corrector_adam_step(lisa_corrector* c, const float* grad, float lr, void* stream);
/* `steps` minibatch Adam steps, rate cosine-decayed from lr_max to lr_min;
 * losses (device, `steps` floats, or NULL) receives each step's loss. */
int lisa_corrector_train(lisa_corrector* c, const float* feats, const float* target, int64_t n_data, int64_t steps,
                         int64_t batch, float lr_max, float lr_min, uint64_t seed, float* losses, void* stream);
/* Corrected links (FP32, [6][out.n]) on every sample of `out`: LFA links,
 * features, network, then full links on tiles above the band and on the
 * spot-checked tiles that fail the check; if one fails, on every tile
 * (decided on the device).  hp/hc are FP32 (LISA_MIXED). */
int lisa_corrector_links(lisa_corrector* c, const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid h_grid,
                         const void* hp, const void* hc, lisa_grid out, void* y, void* stream);
/* Hybrid with the corrector (LISA_MIXED, frozen TDI), in three zones joined by
 * the sigmoid of Sec. IV (Eqs. sigmoid, hybridized_xs) with window T_win and
 * width sigma at each seam:
 *   t <= t_lo + T/2            plain LFA channels (as lisa_response_hybrid),
 *   t_lo - T/2 .. t_hyb + T/2  the full TDI combine of the corrected links,
 *   t >= t_hyb - T/2           the full response.
 * Weights: LFA S_lo(t) S_hi(t), corrected (1 - S_lo(t)) S_hi(t), full
 * 1 - S_hi(t), with S(t; t_s) = 1 / (1 + exp((t - t_s) / sigma)); they sum to
 * one at every sample.  The costly corrected zone is then only as long as
 * the time the source spends between the two switch frequencies.
 * t_lo = -INFINITY: no plain zone (corrected links up to t_hyb).
 * LISA_EINVAL if t_lo is NaN, +INFINITY or later than t_hyb.  The full zone's
 * links run on the library's second stream as in lisa_response_hybrid
 * (forked from and joined back into `stream`). */
int lisa_response_hybrid_corrected(lisa_corrector* c, const lisa_orbit* orbit, const lisa_sky* sky, lisa_grid h_grid,
                                   const void* hp, const void* hc, int tdi_gen, int channels, double t_lo,
                                   double t_hyb, double T_win, double sigma, lisa_grid out, void* xyz, void* stream);
/* Counters since the last reset (synchronises the device): spot-checked
 * tiles, failed spot checks, tiles above the band, tiles recomputed after a
 * failure, largest spot-check error.  Returns LISA_ECORRECTOR if any spot
 * check failed (the outputs were still computed from full links there). */
int lisa_corrector_report(lisa_corrector* c, int64_t* spot_tiles, int64_t* spot_failed, int64_t* band_tiles,
                          int64_t* fallback_tiles, float* max_spot_err, int reset);

/* Device status (no counterpart in the paper).  Kernels that wait on
 * asynchronous copies bound every wait (about a second); a wait that gives up
 * sets bit 0 of a per-device status word and its block stops.  This call
 * synchronises the device, returns the word in *status (may be NULL), clears
 * it if reset != 0, and returns LISA_ETIMEOUT if bit 0 was set. */
int lisa_device_status(unsigned int* status, int reset);
/* Test of the bounded-wait path: one CTA waits on an mbarrier that nothing
 * arrives on; the wait gives up after its bound (about a second), sets the
 * status word and the kernel returns, leaving the context usable.  A later
 * lisa_device_status returns LISA_ETIMEOUT. */
int lisa_selftest_wait_timeout(void* stream);

/* Instrumentation (no counterpart in the paper).
 * lisa_profile_enable(1) clears the record and makes every kernel launch of
 * this library on this process record a CUDA event pair on its own stream;
 * lisa_profile_enable(0) stops recording.  lisa_profile_query synchronises
 * the recorded events and returns, for kernels whose name contains `name`
 * (NULL = all), the summed device time in ms and the number of launches.
 * lisa_launch_count returns the number of kernels this library has launched
 * since the process started (always counted). */
int lisa_profile_enable(int enable);
int lisa_profile_query(const char* name, double* total_ms, int64_t* launches);
int64_t lisa_launch_count(void);

/* Arithmetic peak microbenchmark (no counterpart in the paper; it gives the
 * rooflines a measured denominator).  One launch of blocks_per_sm CTAs of 256
 * threads on every SM; each thread runs 8 independent fused multiply-add
 * recurrences for `iters` steps.  kind 0: FP64 (sink: device double
 * [blocks x 256]); 1: FP32; 2: FP32 as packed pairs (__ffma2_rn) (sink:
 * device float [blocks x 256]).  *flop receives the launch's flop count (2 per
 * multiply-add); the caller times the launch on `stream`.
 * lisa_peak_fma_blocks gives the CTA count (SMs x blocks_per_sm) to size the
 * sink.  LISA_EINVAL on a bad kind, iters < 1, blocks_per_sm outside 1..64
 * or a NULL pointer. */
int lisa_peak_fma_blocks(int blocks_per_sm, int64_t* blocks);
int lisa_peak_fma(int kind, int64_t iters, int blocks_per_sm, void* sink, double* flop, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LISA_H */
