// Synthetic source family generated on the device, ahead of the response:
// a Newtonian (0PN, quadrupole) chirp with an optional eccentric phase
// modulation, joined at f_join = min(f_ISCO, f_cut) to a (2,2,0) damped
// sinusoid.  The paper's waveforms (IMRPhenomTHM/TEHM) are not available; this
// family has their time-domain structure (a long inspiral, then
// merger-ringdown).  Masses in seconds (G M / c^3), tau = t_c - t:
//   f(tau)   = (1/pi) (5/256)^(3/8) Mc^(-5/8) tau^(-3/8)
//   phi(tau) = phi_c - 2 (tau / (5 Mc))^(5/8)          (d phi / dt = 2 pi f)
//   A(f)     = 4 c Mc^(5/3) (pi f)^(2/3) / D
//   Phi      = phi + 4 e_t sin(phi / 2),  e_t = e0 (f / f0)^(-19/18),
//              f0 = f at the grid's first sample
//   h+ = A (1 + cos^2 i)/2 cos Phi,  hx = A cos i sin Phi   (t <= t_join)
//   ringdown: A(f_join) exp(-(t - t_join)/tau_rd) with phase
//             Phi(t_join) + 2 pi f_rd (t - t_join); f_rd, tau_rd from the
//             Berti-Cardoso-Will (2006) fits for the remnant (capped at f_cut).
//
// FP64 form: every sample evaluates these formulas in FP64.
// Mixed form (FP32 output): the absolute phase of a long chirp reaches 1e4 rad,
// so every 32 samples take an anchor at their middle sample: tau_a and the
// absolute phase phi_a in FP64 (x^(5/8) by square roots, Cody-Waite reduction
// of phi_a and phi_a/2), cos/sin of the reduced angles, the amplitude and the
// eccentricity there in FP32.  Each lane of a warp forms one sub-block's
// anchor, so the FP64 work runs on all lanes (an FP64 instruction holds the
// SM's FP64 pipe 16 cycles on GB300 whether one lane or 32 are active), and
// every sample continues its anchor in FP32 through small quantities only:
//   r = (tau - tau_a) / tau_a,  l = log1p(r),
//   phi - phi_a = -2 (tau_a / (5 Mc))^(5/8) expm1(5/8 l),
//   A = A_a exp(-l/4),  e_t = e_a exp(19/48 l),
// and the phase enters as rotations of the anchor's cos/sin by the small
// increments.  Samples after the join (the ringdown, ~1e4 s of a year) are
// evaluated in FP64.
#include <math.h>

#include "lisa_common.cuh"
#include "lisa_internal.cuh"

namespace lisa {
namespace {

constexpr int kWaveThreads = 256;

struct ChirpDev {
    double mc_s, phi_c, tc, e0, f0;
    double inv5mc;    // 1 / (5 Mc)
    double kf;        // f = kf tau^(-3/8)
    double ka;        // A = ka f^(2/3)
    double kp, kc;    // (1 + cos^2 i)/2, cos i
    double tau_join, t_join, a_join, ph_join, f_rd, tau_rd;
    int64_t i_join;   // last grid sample with t <= t_join (-1: none)
    // FP32 copies for the mixed form (a double -> float conversion in device
    // code runs on the FP64 pipe)
    float kpf, kcf, kff, kaf, f0f, e0f;
};

// Chirp phase (with the eccentric modulation) and amplitude at tau > 0, FP64.
__device__ __forceinline__ void chirp_f64(const ChirpDev& p, double tau, double& ph, double& amp)
{
    const double f = p.kf * pow(tau, -0.375);
    ph = p.phi_c - 2.0 * pow(tau / (5.0 * p.mc_s), 0.625);
    if (p.e0 != 0.0) ph += 4.0 * p.e0 * pow(f / p.f0, -19.0 / 18.0) * sin(0.5 * ph);
    amp = p.ka * pow(f, 2.0 / 3.0);
}

__device__ __forceinline__ void ringdown_f64(const ChirpDev& p, double t, double& ph, double& amp)
{
    const double d = t - p.t_join;
    amp = p.a_join * exp(-d / p.tau_rd);
    ph = p.ph_join + 2.0 * kPi * p.f_rd * d;
}

// One draw per blockIdx.y; outputs [nsrc][n].
__global__ void __launch_bounds__(kWaveThreads) chirp_kernel_f64(const ChirpDev* __restrict__ P, double t0, double dt,
                                                                 int64_t n, double* __restrict__ hp,
                                                                 double* __restrict__ hc)
{
    const ChirpDev& p = P[blockIdx.y];
    const int64_t i = (int64_t)blockIdx.x * kWaveThreads + threadIdx.x;
    if (i >= n) return;
    const double t = t0 + (double)i * dt;
    double ph, amp;
    if (i <= p.i_join) chirp_f64(p, p.tc - t, ph, amp);
    else ringdown_f64(p, t, ph, amp);
    double s, c;
    sincos(ph, &s, &c);
    const int64_t o = (int64_t)blockIdx.y * n + i;
    hp[o] = amp * p.kp * c;
    hc[o] = amp * p.kc * s;
}

// (tau / (5 Mc))^(5/8) in FP64 as x^(1/2) x^(1/8): four correctly rounded
// square roots and a product (a few ulp).
__device__ __forceinline__ double pow58(double x)
{
    const double r2 = sqrt(x);
    const double r8 = sqrt(sqrt(r2));
    return r2 * r8;
}

// x - 2 pi k, k = rint(x / 2pi), for |x| up to ~1e9: Cody-Waite reduction with
// 2 pi split into a double and its rounding error.
__device__ __forceinline__ double reduce_2pi(double x)
{
    const double hi = 6.283185307179586, lo = 2.4492935982947064e-16;
    const double k = rint(x * (1.0 / 6.283185307179586));
    return fma(-k, lo, fma(-k, hi, x));
}

// Samples per sub-block (one FP64 anchor each) and sub-blocks per warp: a
// warp covers 32 x 32 samples, lane k computing the anchor of sub-block k (so
// the FP64 work runs on all lanes), then the warp walks the sub-blocks with
// the anchor broadcast from lane k.
constexpr int kSub = 32;
constexpr int kWarpSpan = 32 * kSub;

__global__ void __launch_bounds__(kWaveThreads) chirp_kernel_f32(const ChirpDev* __restrict__ P, double t0, double dt,
                                                                 float dtf, int64_t n, float* __restrict__ hp,
                                                                 float* __restrict__ hc)
{
    const ChirpDev& p = P[blockIdx.y];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t wbase = ((int64_t)blockIdx.x * (kWaveThreads / 32) + warp) * kWarpSpan;
    if (wbase >= n) return;   // uniform over the warp
    // ---- anchor of sub-block `lane` at its middle sample, clamped to the
    // chirp (tau_a >= tau_join).  FP64 only for the absolute phase; the
    // relative quantities are FP32.
    const int64_t ia = wbase + (int64_t)lane * kSub + kSub / 2;
    float a_inv, a_A, a_off, a_c, a_s, a_ch, a_sh, a_amp, a_e;
    {
        const double tau_s = p.tc - (t0 + (double)ia * dt);
        const double tau_a = tau_s > p.tau_join ? tau_s : p.tau_join;
        const double Aa = 2.0 * pow58(tau_a * p.inv5mc);
        const double pha = p.phi_c - Aa;
        sincosf((float)reduce_2pi(pha), &a_s, &a_c);
        sincosf((float)reduce_2pi(0.5 * pha), &a_sh, &a_ch);
        const float taf = (float)tau_a;
        a_inv = 1.f / taf;
        a_A = (float)Aa;
        a_off = (float)(tau_s - tau_a);   // tau = tau_a + a_off - (i - ia) dt
        const float fa = p.kff * powf(taf, -0.375f);
        a_amp = p.kaf * powf(fa, 2.f / 3.f);
        a_e = p.e0f != 0.f ? p.e0f * powf(fa / p.f0f, -19.f / 18.f) : 0.f;
    }
    const float kp = p.kpf, kc = p.kcf;
    const int64_t o0 = (int64_t)blockIdx.y * n;
    for (int k = 0; k < 32; ++k) {
        const int64_t b0 = wbase + (int64_t)k * kSub;
        if (b0 >= n) break;   // uniform
        const float inv = __shfl_sync(0xffffffffu, a_inv, k);
        const float A = __shfl_sync(0xffffffffu, a_A, k);
        const float off = __shfl_sync(0xffffffffu, a_off, k);
        const float ac = __shfl_sync(0xffffffffu, a_c, k), as = __shfl_sync(0xffffffffu, a_s, k);
        const float ach = __shfl_sync(0xffffffffu, a_ch, k), ash = __shfl_sync(0xffffffffu, a_sh, k);
        const float amp_a = __shfl_sync(0xffffffffu, a_amp, k), e_a = __shfl_sync(0xffffffffu, a_e, k);
        const int64_t i = b0 + lane;
        if (i >= n) continue;
        float vp, vc;
        if (i <= p.i_join) {
            const float dtau = off - (float)(lane - kSub / 2) * dtf;   // dtf: dt in FP32
            const float l = log1pf(dtau * inv);
            const float dph = -A * expm1f(0.625f * l);
            float sd, cd;
            sincosf(dph, &sd, &cd);
            float c = ac * cd - as * sd;
            float s = as * cd + ac * sd;
            if (e_a != 0.f) {
                // Phi = phi + 4 e_t sin(phi/2), sin(phi/2) from the anchor's half angle
                float sh2, ch2;
                sincosf(0.5f * dph, &sh2, &ch2);
                const float shalf = ash * ch2 + ach * sh2;
                const float m = 4.f * e_a * expf((19.f / 48.f) * l) * shalf;
                float sm, cm;
                sincosf(m, &sm, &cm);
                const float c2 = c * cm - s * sm;
                s = s * cm + c * sm;
                c = c2;
            }
            const float amp = amp_a * expf(-0.25f * l);
            vp = amp * kp * c;
            vc = amp * kc * s;
        } else {
            double ph, amp;
            ringdown_f64(p, t0 + (double)i * dt, ph, amp);
            double sn, cs;
            sincos(ph, &sn, &cs);
            vp = (float)(amp * p.kp * cs);
            vc = (float)(amp * p.kc * sn);
        }
        hp[o0 + i] = vp;
        hc[o0 + i] = vc;
    }
}

// Host set-up of one draw, FP64.
int make_chirp(const lisa_chirp& c, const lisa_grid& g, ChirpDev& p)
{
    const double vals[] = {c.mc_s, c.q, c.dist_m, c.iota, c.phi_c, c.tc, c.e0, c.f_cut, c.m_final_frac, c.a_final};
    for (double v : vals)
        if (!isfinite(v)) { set_error("lisa_chirp_ringdown: non-finite parameter"); return LISA_EINVAL; }
    if (!(c.mc_s > 0.0) || !(c.q >= 1.0) || !(c.dist_m > 0.0) || !(c.e0 >= 0.0 && c.e0 < 1.0) ||
        !(c.m_final_frac > 0.0 && c.m_final_frac <= 1.0) || !(c.a_final >= 0.0 && c.a_final < 1.0)) {
        set_error("lisa_chirp_ringdown: need mc_s > 0, q >= 1, dist_m > 0, 0 <= e0 < 1, 0 < m_final_frac <= 1, "
                  "0 <= a_final < 1");
        return LISA_EINVAL;
    }
    const double eta = c.q / ((1.0 + c.q) * (1.0 + c.q));
    const double m_tot = c.mc_s * pow(eta, -0.6);
    const double f_isco = 1.0 / (pow(6.0, 1.5) * kPi * m_tot);
    const double f_join = c.f_cut > 0.0 ? fmin(f_isco, c.f_cut) : f_isco;
    p.mc_s = c.mc_s;
    p.inv5mc = 1.0 / (5.0 * c.mc_s);
    p.phi_c = c.phi_c;
    p.tc = c.tc;
    p.e0 = c.e0;
    p.kf = (1.0 / kPi) * pow(5.0 / 256.0, 0.375) * pow(c.mc_s, -0.625);
    p.ka = 4.0 * kC * pow(c.mc_s, 5.0 / 3.0) * pow(kPi, 2.0 / 3.0) / c.dist_m;
    const double ci = cos(c.iota);
    p.kp = 0.5 * (1.0 + ci * ci);
    p.kc = ci;
    p.tau_join = pow(p.kf / f_join, 8.0 / 3.0);
    p.t_join = c.tc - p.tau_join;
    p.f0 = c.tc - g.t0 > 0.0 ? p.kf * pow(c.tc - g.t0, -0.375) : f_join;
    // (2,2,0) remnant mode (Berti-Cardoso-Will fits)
    const double mf = c.m_final_frac * m_tot;
    const double mw = 1.5251 - 1.1568 * pow(1.0 - c.a_final, 0.1292);
    const double qf = 0.7000 + 1.4187 * pow(1.0 - c.a_final, -0.4990);
    double f_rd = mw / (2.0 * kPi * mf);
    p.tau_rd = qf / (kPi * f_rd);
    if (c.f_cut > 0.0) f_rd = fmin(f_rd, c.f_cut);
    p.f_rd = f_rd;
    // phase and amplitude at the join
    double ph = c.phi_c - 2.0 * pow(p.tau_join / (5.0 * c.mc_s), 0.625);
    if (c.e0 != 0.0) ph += 4.0 * c.e0 * pow(f_join / p.f0, -19.0 / 18.0) * sin(0.5 * ph);
    p.ph_join = ph;
    p.a_join = p.ka * pow(f_join, 2.0 / 3.0);
    // last sample with t0 + i dt <= t_join, by the same FP64 comparison as the definition
    int64_t ij = (int64_t)floor((p.t_join - g.t0) / g.dt);
    if (ij < -1) ij = -1;
    if (ij > g.n - 1) ij = g.n - 1;
    while (ij + 1 <= g.n - 1 && g.t0 + (double)(ij + 1) * g.dt <= p.t_join) ++ij;
    while (ij >= 0 && !(g.t0 + (double)ij * g.dt <= p.t_join)) --ij;
    p.i_join = ij;
    p.kpf = (float)p.kp;
    p.kcf = (float)p.kc;
    p.kff = (float)p.kf;
    p.kaf = (float)p.ka;
    p.f0f = (float)p.f0;
    p.e0f = (float)p.e0;
    return LISA_OK;
}

}  // namespace
}  // namespace lisa

using namespace lisa;

extern "C" int lisa_chirp_ringdown(const lisa_chirp* src, int nsrc, lisa_grid grid, int precision, void* hp, void* hc,
                                   void* stream)
{
    LISA_TRY(check_grid(grid, "grid"));
    if (precision != LISA_F64 && precision != LISA_MIXED) { set_error("precision %d unknown", precision); return LISA_EINVAL; }
    if (nsrc < 0 || nsrc > 65535) { set_error("nsrc must be in [0, 65535]"); return LISA_EINVAL; }
    if (nsrc == 0 || grid.n == 0) return LISA_OK;
    if (!src || !hp || !hc) { set_error("NULL pointer"); return LISA_EINVAL; }
    ChirpDev* host = new ChirpDev[nsrc];
    for (int k = 0; k < nsrc; ++k) {
        const int rc = make_chirp(src[k], grid, host[k]);
        if (rc) {
            delete[] host;
            return rc;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    Scratch sc(st);
    ChirpDev* dev = (ChirpDev*)sc.alloc(sizeof(ChirpDev) * (size_t)nsrc);
    if (!dev) {
        delete[] host;
        return sc.status();
    }
    // from pageable memory the copy has been staged when the call returns, so
    // the host array can go
    const int rc = cuda_status(cudaMemcpyAsync(dev, host, sizeof(ChirpDev) * (size_t)nsrc, cudaMemcpyHostToDevice, st),
                               "cudaMemcpyAsync(chirp params)");
    delete[] host;
    if (rc) return rc;
    if (precision == LISA_F64) {
        const dim3 blocks((unsigned)((grid.n + kWaveThreads - 1) / kWaveThreads), (unsigned)nsrc);
        prof_before("chirp_f64", st);
        chirp_kernel_f64<<<blocks, kWaveThreads, 0, st>>>(dev, grid.t0, grid.dt, grid.n, (double*)hp, (double*)hc);
    } else {
        const int64_t per_block = (int64_t)(kWaveThreads / 32) * kWarpSpan;
        const dim3 blocks((unsigned)((grid.n + per_block - 1) / per_block), (unsigned)nsrc);
        prof_before("chirp_mixed", st);
        chirp_kernel_f32<<<blocks, kWaveThreads, 0, st>>>(dev, grid.t0, grid.dt, (float)grid.dt, grid.n, (float*)hp,
                                                          (float*)hc);
    }
    prof_after(st);
    return cuda_status(cudaGetLastError(), "chirp_kernel");
}
