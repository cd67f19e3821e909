"""FP64 oracle of the synthetic source family generated on the device: a
Newtonian (0PN, quadrupole) inspiral chirp with an optional eccentric phase
modulation, joined at f_join = min(f_ISCO, f_cut) to a (2,2,0) damped
sinusoid.  The paper's waveforms (IMRPhenomTHM/TEHM) are not available here;
this family stands in for them with the same time-domain structure (a long
chirp, then merger-ringdown), as the synthetic inputs of the benchmarks do.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): imported by tests/ and
bench.py's baseline legs, never by the library.

Definitions (masses in seconds, M = G M / c^3; tau = t_c - t):
  f(tau)    = (1/pi) (5/256)^(3/8) Mc^(-5/8) tau^(-3/8)
  phi(tau)  = phi_c - 2 (tau / (5 Mc))^(5/8)             (d phi / dt = 2 pi f)
  A(f)      = 4 c Mc^(5/3) (pi f)^(2/3) / D
  e_t(f)    = e0 (f / f0)^(-19/18),  f0 = f at the grid's first sample
  Phi       = phi + 4 e_t sin(phi / 2)                    (eccentric modulation)
  h+ = A (1 + cos^2 i)/2 cos Phi,   hx = A cos i sin Phi  (t <= t_join)
  M = Mc eta^(-3/5), eta = q / (1 + q)^2,  f_ISCO = 1 / (6^(3/2) pi M)
  ringdown (t > t_join): M_f = m_final_frac M, spin a_f, Berti-Cardoso-Will
  (2006) fits  M_f omega = 1.5251 - 1.1568 (1 - a_f)^0.1292,
               Q = 0.7000 + 1.4187 (1 - a_f)^(-0.4990),
  f_rd = omega / (2 pi) (capped at f_cut), tau_rd = Q / (pi f_rd),
  h = A(f_join) exp(-(t - t_join)/tau_rd) x [(1 + cos^2 i)/2 cos, cos i sin]
      (Phi(t_join) + 2 pi f_rd (t - t_join)).
"""
from __future__ import annotations

import math

import numpy as np

C_LIGHT = 299792458.0


def chirp_f(tau, mc_s):
    """0PN gravitational-wave frequency at time to coalescence tau."""
    return (1.0 / math.pi) * (5.0 / 256.0) ** 0.375 * mc_s ** -0.625 * np.asarray(tau, dtype=np.float64) ** -0.375


def chirp_tau(f, mc_s):
    """Time to coalescence at frequency f (inverse of chirp_f)."""
    return ((1.0 / math.pi) * (5.0 / 256.0) ** 0.375 * mc_s ** -0.625 / f) ** (8.0 / 3.0)


def chirp_phi(tau, mc_s, phi_c):
    return phi_c - 2.0 * (np.asarray(tau, dtype=np.float64) / (5.0 * mc_s)) ** 0.625


def chirp_amp(f, mc_s, dist_m):
    return 4.0 * C_LIGHT * mc_s ** (5.0 / 3.0) * (math.pi * np.asarray(f, dtype=np.float64)) ** (2.0 / 3.0) / dist_m


def join_point(mc_s, q, f_cut=0.0):
    """(f_join, tau_join, M) of the chirp-ringdown join."""
    eta = q / (1.0 + q) ** 2
    m_tot = mc_s * eta ** -0.6
    f_isco = 1.0 / (6.0 ** 1.5 * math.pi * m_tot)
    f_join = min(f_isco, f_cut) if f_cut > 0.0 else f_isco
    return f_join, chirp_tau(f_join, mc_s), m_tot


def qnm_220(m_final_s, a_final):
    mw = 1.5251 - 1.1568 * (1.0 - a_final) ** 0.1292
    qf = 0.7000 + 1.4187 * (1.0 - a_final) ** -0.4990
    f = mw / (2.0 * math.pi * m_final_s)
    return f, qf / (math.pi * f)


def chirp_ringdown(grid, mc_s, q, dist_m, iota, phi_c, tc, e0=0.0, f_cut=0.0, m_final_frac=0.95, a_final=0.7,
                   idx=None):
    """(h+, hx) on grid = (t0, dt, n) (or at its samples idx), one sample at a time."""
    t0, dt, n = float(grid[0]), float(grid[1]), int(grid[2])
    f_join, tau_join, m_tot = join_point(mc_s, q, f_cut)
    t_join = tc - tau_join
    f_rd, tau_rd = qnm_220(m_final_frac * m_tot, a_final)
    if f_cut > 0.0:
        f_rd = min(f_rd, f_cut)
    ci = math.cos(iota)
    kp, kc = 0.5 * (1.0 + ci * ci), ci
    f0 = float(chirp_f(tc - t0, mc_s)) if tc - t0 > 0.0 else f_join

    def phase(tau):
        f = float(chirp_f(tau, mc_s))
        ph = float(chirp_phi(tau, mc_s, phi_c))
        if e0 != 0.0:
            ph += 4.0 * e0 * (f / f0) ** (-19.0 / 18.0) * math.sin(0.5 * ph)
        return f, ph

    _, ph_join = phase(tau_join)
    a_join = float(chirp_amp(f_join, mc_s, dist_m))
    idx = np.arange(n) if idx is None else np.asarray(idx, dtype=np.int64)
    hp = np.zeros(idx.size)
    hc = np.zeros(idx.size)
    for k, i in enumerate(idx):
        t = t0 + float(i) * dt
        if t <= t_join:
            f, ph = phase(tc - t)
            a = float(chirp_amp(f, mc_s, dist_m))
        else:
            a = a_join * math.exp(-(t - t_join) / tau_rd)
            ph = ph_join + 2.0 * math.pi * f_rd * (t - t_join)
        hp[k] = a * kp * math.cos(ph)
        hc[k] = a * kc * math.sin(ph)
    return hp, hc
