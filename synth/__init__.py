"""Seeded synthetic inputs for the LISA time-domain response.

This module is shared by the CPU oracle's tests, the CUDA parity tests and the
benchmark.  It holds none of the response method's arithmetic: it only draws
source parameters and samples the GW polarisations h+(t), hx(t) on uniform time
grids.  The waveform families stand in for the IMRPhenomTHM polarisations that
the paper feeds to its response (Sec. IV, "Response model validation"); none of
that model is reproduced here.

Waveform families (all FP64, numpy):

* ``chirp_0pn``: Newtonian quadrupole chirp.  With M = G*Mc/c^3 (seconds) and
  tau = tc - t,
  f(t)   = (1/pi) (5/256)^(3/8) M^(-5/8) tau^(-3/8),
  Phi(t) = Phi_c - 2 (tau / (5 M))^(5/8),
  A(t)   = 4 c M^(5/3) (pi f)^(2/3) / D,
  h+ = A (1 + cos^2 iota)/2 cos Phi,  hx = A cos iota sin Phi.
* ``chirp_ringdown``: the chirp up to f_isco = 1/(6^(3/2) pi M_tot), then a
  damped sinusoid at the (2,2,0) quasi-normal mode (Berti, Cardoso & Will 2006
  fits, remnant mass and spin stated in the call), joined with continuous
  amplitude and phase.
* eccentric chirp: Phi_ecc = Phi_circ + 4 e(t) sin(Phi_circ/2) with
  e(t) = e0 (f/f0)^(-19/18) (leading-order equation of the centre).

The grid of a source is (t0, dt, n) in absolute SSB seconds; sample i sits at
t0 + i*dt.  Seeds: configuration k uses seed 2505096000 + k.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 299792458.0
T_SUN = 4.925490947641267e-6          # G*Msun/c^3 in seconds
GPC = 3.0856775814913673e25           # metres
SEED_BASE = 2505096000
DAY = 86400.0
YEAR = 365.25 * DAY


@dataclass
class Source:
    """One synthetic source: grid, polarisations and its extrinsic parameters."""
    t0: float
    dt: float
    n: int
    hp: np.ndarray
    hc: np.ndarray
    beta: float
    lam: float
    psi: float
    tc: float
    mc_s: float                 # G*Mc/c^3 in seconds
    meta: dict = field(default_factory=dict)

    @property
    def grid(self):
        return (self.t0, self.dt, self.n)

    def times(self):
        return self.t0 + np.arange(self.n, dtype=np.float64) * self.dt


def draw_sky(rng: np.random.Generator):
    """Isotropic sky position and uniform polarisation angle."""
    beta = math.asin(rng.uniform(-1.0, 1.0))
    lam = rng.uniform(0.0, 2.0 * math.pi)
    psi = rng.uniform(0.0, math.pi)
    return beta, lam, psi


def chirp_frequency(tau, mc_s):
    """0PN GW frequency at time-to-coalescence tau (seconds)."""
    tau = np.asarray(tau, dtype=np.float64)
    return (1.0 / math.pi) * (5.0 / 256.0) ** 0.375 * mc_s ** -0.625 * tau ** -0.375


def chirp_tau_of_f(f, mc_s):
    """Inverse of chirp_frequency: time to coalescence at GW frequency f."""
    return ((1.0 / math.pi) * (5.0 / 256.0) ** 0.375 * mc_s ** -0.625 / f) ** (8.0 / 3.0)


def chirp_phase(tau, mc_s, phi_c):
    tau = np.asarray(tau, dtype=np.float64)
    return phi_c - 2.0 * (tau / (5.0 * mc_s)) ** 0.625


def chirp_amplitude(f, mc_s, dist_m):
    return 4.0 * C_LIGHT * mc_s ** (5.0 / 3.0) * (math.pi * np.asarray(f)) ** (2.0 / 3.0) / dist_m


def chirp_0pn(t, tc, mc_s, dist_m, iota, phi_c, ecc0=0.0, f_ecc_ref=None):
    """h+, hx of the Newtonian chirp at times t < tc (zero at and after tc)."""
    t = np.asarray(t, dtype=np.float64)
    tau = tc - t
    ok = tau > 0
    taus = np.where(ok, tau, 1.0)
    f = chirp_frequency(taus, mc_s)
    phi = chirp_phase(taus, mc_s, phi_c)
    if ecc0 != 0.0:
        f0 = f_ecc_ref if f_ecc_ref is not None else float(np.min(f))
        e_t = ecc0 * (f / f0) ** (-19.0 / 18.0)
        phi = phi + 4.0 * e_t * np.sin(0.5 * phi)
    amp = chirp_amplitude(f, mc_s, dist_m)
    ci = math.cos(iota)
    hp = np.where(ok, amp * 0.5 * (1.0 + ci * ci) * np.cos(phi), 0.0)
    hc = np.where(ok, amp * ci * np.sin(phi), 0.0)
    return hp, hc


def qnm_220(m_final_s, a_final):
    """(2,2,0) ringdown frequency (Hz) and damping time (s), BCW-2006 fits."""
    mw = 1.5251 - 1.1568 * (1.0 - a_final) ** 0.1292
    q = 0.7000 + 1.4187 * (1.0 - a_final) ** (-0.4990)
    f = mw / (2.0 * math.pi * m_final_s)
    return f, q / (math.pi * f)


def total_mass_s(mc_s, q):
    eta = q / (1.0 + q) ** 2
    return mc_s * eta ** -0.6


def chirp_ringdown(t, tc, mc_s, q, dist_m, iota, phi_c, f_cut=None,
                   m_final_frac=0.95, a_final=0.7, ecc0=0.0):
    """Chirp up to min(f_isco, f_cut), then a (2,2,0)-like damped sinusoid.

    Returns (hp, hc, info) with the join time and the ringdown parameters.
    """
    t = np.asarray(t, dtype=np.float64)
    m_tot = total_mass_s(mc_s, q)
    f_isco = 1.0 / (6.0 ** 1.5 * math.pi * m_tot)
    f_join = f_isco if f_cut is None else min(f_isco, f_cut)
    tau_join = chirp_tau_of_f(f_join, mc_s)
    t_join = tc - tau_join
    f_rd, tau_rd = qnm_220(m_final_frac * m_tot, a_final)
    if f_cut is not None:
        f_rd = min(f_rd, f_cut)
    ci = math.cos(iota)
    f0 = None
    if ecc0 != 0.0:
        f0 = float(chirp_frequency(tc - t[0], mc_s)) if tc - t[0] > 0 else f_join
    hp, hc = chirp_0pn(np.minimum(t, t_join), tc, mc_s, dist_m, iota, phi_c, ecc0, f0)
    phi_j = float(chirp_phase(tau_join, mc_s, phi_c))
    if ecc0 != 0.0:
        e_j = ecc0 * (f_join / f0) ** (-19.0 / 18.0)
        phi_j += 4.0 * e_j * math.sin(0.5 * phi_j)
    amp_j = float(chirp_amplitude(f_join, mc_s, dist_m))
    after = t > t_join
    dtr = np.where(after, t - t_join, 0.0)
    env = amp_j * np.exp(-dtr / tau_rd)
    ph = phi_j + 2.0 * math.pi * f_rd * dtr
    hp = np.where(after, env * 0.5 * (1.0 + ci * ci) * np.cos(ph), hp)
    hc = np.where(after, env * ci * np.sin(ph), hc)
    return hp, hc, dict(t_join=t_join, f_join=f_join, f_rd=f_rd, tau_rd=tau_rd,
                        m_tot_s=m_tot)


# ---------------------------------------------------------------------------
# configurations
# ---------------------------------------------------------------------------

def cfg1_source(seed_offset=0, n=8640, dt=10.0, tc=4.0e7):
    """Plain chirp, Mc=1e5 Msun, q=1, D=10 Gpc, iota=0.5; 1 day at 10 s ending at tc-dt."""
    rng = np.random.default_rng(SEED_BASE + 1 + seed_offset)
    beta, lam, psi = draw_sky(rng)
    phi_c = rng.uniform(0.0, 2.0 * math.pi)
    mc_s = 1.0e5 * T_SUN
    t0 = tc - n * dt
    t = t0 + np.arange(n) * dt
    hp, hc = chirp_0pn(t, tc, mc_s, 10.0 * GPC, 0.5, phi_c)
    return Source(t0, dt, n, hp, hc, beta, lam, psi, tc, mc_s,
                  dict(name="chirp Mc=1e5 q=1 1d@10s", phi_c=phi_c))


def cfg2_source(n=6311520, dt=5.0, t0=2.0e7, seed_offset=0, post_merger=1.0e4):
    """Chirp + ringdown, Mc=1e6 Msun, q=3; one year at 5 s (6,311,520 samples)."""
    rng = np.random.default_rng(SEED_BASE + 2 + seed_offset)
    beta, lam, psi = draw_sky(rng)
    phi_c = rng.uniform(0.0, 2.0 * math.pi)
    mc_s = 1.0e6 * T_SUN
    t_end = t0 + n * dt
    tc = t_end - post_merger
    t = t0 + np.arange(n) * dt
    hp, hc, info = chirp_ringdown(t, tc, mc_s, 3.0, 10.0 * GPC, 0.5, phi_c)
    info.update(name="chirp+ringdown Mc=1e6 q=3 1yr@5s", phi_c=phi_c)
    return Source(t0, dt, n, hp, hc, beta, lam, psi, tc, mc_s, info)


def cfg2_small(n=20000, dt=5.0, seed_offset=0):
    """cfg2-shaped source on a short grid that ends past the merger (parity size)."""
    return cfg2_source(n=n, dt=dt, t0=2.0e7, seed_offset=seed_offset, post_merger=min(1.0e4, 0.2 * n * dt))


def batch_params(nsrc=1024, seed=SEED_BASE + 3):
    """Parameters of the batched workload: Mc log-U[1e4,1e7], q U[1,10],
    duration log-U[1 d, 90 d], dt in {5,10} s, isotropic sky."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nsrc):
        mc = 10.0 ** rng.uniform(4.0, 7.0)
        q = rng.uniform(1.0, 10.0)
        dur = math.exp(rng.uniform(math.log(DAY), math.log(90.0 * DAY)))
        dt = 5.0 if rng.uniform() < 0.5 else 10.0
        beta, lam, psi = draw_sky(rng)
        phi_c = rng.uniform(0.0, 2.0 * math.pi)
        t0 = rng.uniform(1.0e7, 5.0e7)
        out.append(dict(mc=mc, q=q, dur=dur, dt=dt, beta=beta, lam=lam, psi=psi,
                        phi_c=phi_c, t0=t0))
    return out


def batch_source(p, dist_gpc=10.0, iota=0.5):
    """Materialise one batched source from its parameters (chirp truncated at
    min(f_isco, 0.8 Nyquist), then ringdown)."""
    dt = p["dt"]
    n = int(p["dur"] // dt)
    mc_s = p["mc"] * T_SUN
    m_tot = total_mass_s(mc_s, p["q"])
    f_nyq = 0.5 / dt
    f_cut = 0.8 * f_nyq
    _, tau_rd = qnm_220(0.95 * m_tot, 0.7)
    t0 = p["t0"]
    t_end = t0 + n * dt
    tc = t_end - max(12.0 * tau_rd, 40.0 * dt)
    t = t0 + np.arange(n) * dt
    hp, hc, info = chirp_ringdown(t, tc, mc_s, p["q"], dist_gpc * GPC, iota, p["phi_c"], f_cut=f_cut)
    info.update(p)
    return Source(t0, dt, n, hp, hc, p["beta"], p["lam"], p["psi"], tc, mc_s, info)


def pe_params(ndraw=4096, seed=SEED_BASE + 5):
    """Draws around Mc=5e5 Msun, q=2: 1e-3 relative spread on the masses, 1e-2 rad
    on the angles, e0 ~ U[0, 0.3]."""
    rng = np.random.default_rng(seed)
    rng0 = np.random.default_rng(seed + 1000)
    beta0, lam0, psi0 = draw_sky(rng0)
    out = []
    for _ in range(ndraw):
        out.append(dict(mc=5.0e5 * (1.0 + 1e-3 * rng.standard_normal()),
                        q=2.0 * (1.0 + 1e-3 * rng.standard_normal()),
                        beta=float(np.clip(beta0 + 1e-2 * rng.standard_normal(), -1.5, 1.5)),
                        lam=lam0 + 1e-2 * rng.standard_normal(),
                        psi=psi0 + 1e-2 * rng.standard_normal(),
                        phi_c=rng.uniform(0.0, 2.0 * math.pi),
                        e0=rng.uniform(0.0, 0.3)))
    return out


def pe_source(p, n=3155760, dt=10.0, t0=2.0e7):
    """One year at 10 s of an eccentric chirp + ringdown for one PE draw."""
    mc_s = p["mc"] * T_SUN
    t_end = t0 + n * dt
    tc = t_end - 1.0e4
    t = t0 + np.arange(n) * dt
    hp, hc, info = chirp_ringdown(t, tc, mc_s, p["q"], 10.0 * GPC, 0.5, p["phi_c"],
                                  f_cut=0.8 * 0.5 / dt, ecc0=p["e0"])
    info.update(p)
    return Source(t0, dt, n, hp, hc, p["beta"], p["lam"], p["psi"], tc, mc_s, info)



def corrector_params(nsrc=4096, seed=SEED_BASE + 4, n=4883, fmin=1e-4, fmax=2e-2, ecc_frac=0.5, e0_max=0.3):
    """Sources of the corrector's training and held-out sets: chirps whose GW
    frequency stays inside [fmin, fmax] over their grid.  Start frequency
    log-U[fmin, fmax/1.02], sweep ratio f_end/f_start log-U[1.001, min(3,
    fmax/f_start)], dt in {5, 10} s, n samples, isotropic sky, cos(iota)
    U[-1, 1], t0 U[1e7, 4e7] s (orbit phase), distance 10 Gpc; a fraction
    ecc_frac of them eccentric, e0 U[0, e0_max] at the start frequency (the
    leading-order phase modulation of chirp_0pn)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nsrc):
        f0 = math.exp(rng.uniform(math.log(fmin), math.log(fmax / 1.02)))
        rmax = min(3.0, fmax / f0)
        r = math.exp(rng.uniform(math.log(1.001), math.log(rmax)))
        dt = 5.0 if rng.uniform() < 0.5 else 10.0
        beta, lam, psi = draw_sky(rng)
        iota = math.acos(rng.uniform(-1.0, 1.0))
        phi_c = rng.uniform(0.0, 2.0 * math.pi)
        t0 = rng.uniform(1.0e7, 4.0e7)
        e0 = rng.uniform(0.0, e0_max) if rng.uniform() < ecc_frac else 0.0
        out.append(dict(f0=f0, ratio=r, dt=dt, n=n, beta=beta, lam=lam, psi=psi, iota=iota, phi_c=phi_c, t0=t0,
                        e0=e0))
    return out


def corrector_source(p, dist_gpc=10.0):
    """Materialise a corrector source: the 0PN chirp whose frequency goes from
    f0 at the first sample to f0*ratio at the end of the grid (chirp mass and
    coalescence time solved from the two frequencies)."""
    n, dt = p["n"], p["dt"]
    dur = n * dt
    f_end = p["f0"] * p["ratio"]
    tau_end = dur / (p["ratio"] ** (8.0 / 3.0) - 1.0)
    # f = (1/pi)(5/256)^(3/8) M^(-5/8) tau^(-3/8)  ->  M from (f_end, tau_end)
    mc_s = (math.pi * f_end * tau_end ** 0.375 / (5.0 / 256.0) ** 0.375) ** -1.6
    t0 = p["t0"]
    tc = t0 + dur + tau_end
    t = t0 + np.arange(n) * dt
    hp, hc = chirp_0pn(t, tc, mc_s, dist_gpc * GPC, p["iota"], p["phi_c"], ecc0=p.get("e0", 0.0), f_ecc_ref=p["f0"])
    return Source(t0, dt, n, hp, hc, p["beta"], p["lam"], p["psi"], tc, mc_s, dict(p))



def sweep_params(nsrc=256, seed=SEED_BASE + 40, f_start=5e-4, f_end=2e-2, dt=5.0):
    """Held-out chirps of the corrector's hybrid test: Newtonian chirps that
    sweep from f_start to f_end over their grid (Mc log-U[3e5, 1e6] Msun,
    tc U[2e7, 5e7] s, isotropic sky, cos(iota) U[-1, 1])."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(nsrc):
        mc = 10.0 ** rng.uniform(math.log10(3e5), 6.0)
        beta, lam, psi = draw_sky(rng)
        iota = math.acos(rng.uniform(-1.0, 1.0))
        out.append(dict(mc=mc, tc=rng.uniform(2.0e7, 5.0e7), beta=beta, lam=lam, psi=psi, iota=iota,
                        phi_c=rng.uniform(0.0, 2.0 * math.pi), f_start=f_start, f_end=f_end, dt=dt))
    return out


def sweep_source(p, dist_gpc=10.0):
    mc_s = p["mc"] * T_SUN
    tau0 = chirp_tau_of_f(p["f_start"], mc_s)
    tau1 = chirp_tau_of_f(p["f_end"], mc_s)
    dt = p["dt"]
    n = int((tau0 - tau1) // dt)
    t0 = p["tc"] - tau0
    t = t0 + np.arange(n) * dt
    hp, hc = chirp_0pn(t, p["tc"], mc_s, dist_gpc * GPC, p["iota"], p["phi_c"])
    return Source(t0, dt, n, hp, hc, p["beta"], p["lam"], p["psi"], p["tc"], mc_s, dict(p))


def monochromatic(t0, dt, n, f, amp_p=1.0, amp_c=1.0, phase=0.0):
    """h+ = amp_p cos(2 pi f t + phase), hx = amp_c sin(2 pi f t + phase)."""
    t = t0 + np.arange(n) * dt
    ph = 2.0 * math.pi * f * (t - t0) + phase
    return amp_p * np.cos(ph), amp_c * np.sin(ph)


def laser_noise_tones(seed, ntone=6, fmin=2e-3, fmax=1.5e-2):
    """Three smooth band-limited 'laser noise' signals p_s(t) as sums of tones.

    Returns a list (one per spacecraft) of (freqs, amps, phases) arrays."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(3):
        out.append((rng.uniform(fmin, fmax, ntone), rng.uniform(0.5, 1.0, ntone),
                    rng.uniform(0.0, 2.0 * math.pi, ntone)))
    return out


def eval_tones(tones, t):
    f, a, p = tones
    t = np.asarray(t, dtype=np.float64)[..., None]
    return np.sum(a * np.cos(2.0 * math.pi * f * t + p), axis=-1)


def host_cores():
    import os
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1
