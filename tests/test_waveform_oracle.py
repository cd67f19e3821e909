"""Pins of the FP64 oracle of the synthetic source family (oracle/waveform.py):
the 0PN chirp's frequency-phase relation and inversion, the amplitude law, the
join to the ringdown, the (2,2,0) fits against tabulated Kerr quasinormal
modes, the ISCO frequency, the eccentric modulation's bounds, and agreement
with the benchmarks' input generator (an independent implementation of the
same family)."""
import math

import numpy as np

import synth
from oracle import waveform as W

T_SUN = 4.925490947641267e-06   # G Msun / c^3 (s)


def test_phase_derivative_is_two_pi_f():
    mc = 1e6 * T_SUN
    for tau in (3e7, 1e6, 1e4, 300.0):
        h = 1e-3 * min(tau, 1e3)
        dphi_dt = (W.chirp_phi(tau - h, mc, 0.0) - W.chirp_phi(tau + h, mc, 0.0)) / (2.0 * h)
        assert abs(dphi_dt / (2.0 * math.pi * W.chirp_f(tau, mc)) - 1.0) < 1e-7


def test_tau_inverts_frequency():
    mc = 5e5 * T_SUN
    for tau in (3e7, 5e5, 123.0):
        assert abs(W.chirp_tau(float(W.chirp_f(tau, mc)), mc) / tau - 1.0) < 1e-13


def test_face_on_amplitude_and_polarisations():
    # iota = 0: h+ = A cos Phi, hx = A sin Phi, so h+^2 + hx^2 = A(f)^2 on the chirp
    mc, q, D, tc = 1e6 * T_SUN, 3.0, 3.0857e25, 2.0e7 + 4e5
    g = (2.0e7, 5.0, 3000)
    hp, hc = W.chirp_ringdown(g, mc, q, D, 0.0, 0.3, tc)
    t = g[0] + np.arange(g[2]) * g[1]
    a = W.chirp_amp(W.chirp_f(tc - t, mc), mc, D)
    assert np.allclose(hp ** 2 + hc ** 2, a ** 2, rtol=1e-12)
    # amplitude grows as f^(2/3) = tau^(-1/4)
    assert abs(a[-1] / a[0] - ((tc - t[-1]) / (tc - t[0])) ** -0.25) < 1e-12


def test_isco_frequency():
    # f_ISCO = 1 / (6^(3/2) pi M) = 4397 Hz for one solar mass
    for q in (1.0, 4.0):
        eta = q / (1.0 + q) ** 2
        mc = T_SUN * eta ** 0.6          # total mass one solar mass
        f_join, _, m_tot = W.join_point(mc, q)
        assert abs(m_tot / T_SUN - 1.0) < 1e-12
        assert abs(f_join / 4397.0 - 1.0) < 1e-3


def test_ringdown_fits_match_kerr_modes():
    # Berti-Cardoso-Will fits against tabulated (2,2,0) Kerr modes, to the
    # few per cent the fits are good for:
    # a = 0: M omega = 0.37367, M omega_I = 0.08896; a = 0.7: 0.5326, 0.0808
    for a, w_r, w_i in ((0.0, 0.37367, 0.08896), (0.7, 0.5326, 0.0808)):
        f, tau = W.qnm_220(1.0, a)
        assert abs(2.0 * math.pi * f / w_r - 1.0) < 0.03
        assert abs((1.0 / tau) / w_i - 1.0) < 0.03


def test_join_is_continuous_and_ringdown_decays():
    mc, q, D, tc, iota, phic = 1e6 * T_SUN, 3.0, 3.0857e25, 2.0e7 + 4e5, 0.5, 1.1
    f_join, tau_join, m_tot = W.join_point(mc, q)
    t_join = tc - tau_join
    a = W.chirp_ringdown((t_join, 1.0, 1), mc, q, D, iota, phic, tc)
    b = W.chirp_ringdown((t_join + 1e-6, 1.0, 1), mc, q, D, iota, phic, tc)
    amp = W.chirp_amp(f_join, mc, D)
    assert abs(a[0][0] - b[0][0]) < 1e-7 * amp and abs(a[1][0] - b[1][0]) < 1e-7 * amp
    # the envelope after the join decays with the fitted damping time
    f_rd, tau_rd = W.qnm_220(0.95 * m_tot, 0.7)
    g = (t_join + 0.5, 1.0, 400)
    hp, hc = W.chirp_ringdown(g, mc, q, D, iota, phic, tc)
    ci = math.cos(iota)
    env = np.sqrt((hp / (0.5 * (1 + ci * ci))) ** 2 + (hc / ci) ** 2)
    slope = np.polyfit(np.arange(g[2]) * g[1], np.log(env), 1)[0]
    assert abs(slope * tau_rd + 1.0) < 1e-9


def test_eccentric_modulation_bounds():
    mc, q, D, tc = 5e5 * T_SUN, 2.0, 3.0857e26, 2.0e7 + 3e5
    g = (2.0e7, 10.0, 2000)
    hp0, hc0 = W.chirp_ringdown(g, mc, q, D, 0.0, 0.4, tc, e0=0.0)
    hp1, hc1 = W.chirp_ringdown(g, mc, q, D, 0.0, 0.4, tc, e0=0.2)
    ph0 = np.unwrap(np.arctan2(hc0, hp0))
    ph1 = np.unwrap(np.arctan2(hc1, hp1))
    t = g[0] + np.arange(g[2]) * g[1]
    f = W.chirp_f(tc - t, mc)
    e_t = 0.2 * (f / f[0]) ** (-19.0 / 18.0)
    d = ph1 - ph0
    d -= 2 * np.pi * np.round((d[0]) / (2 * np.pi))
    assert np.all(np.abs(d) <= 4.0 * e_t + 1e-9)
    assert np.abs(d).max() > 2.0 * e_t.min()
    # circular face-on: the same amplitude
    assert np.allclose(hp1 ** 2 + hc1 ** 2, hp0 ** 2 + hc0 ** 2, rtol=1e-12)


def test_matches_input_generator():
    for p in synth.pe_params(ndraw=3)[:3]:
        s = synth.pe_source(p, n=20000, dt=10.0)
        hp, hc = W.chirp_ringdown(s.grid, p["mc"] * synth.T_SUN, p["q"], 10.0 * synth.GPC, 0.5, p["phi_c"], s.tc,
                                  e0=p["e0"], f_cut=0.8 * 0.5 / 10.0)
        scale = np.abs(s.hp).max()
        assert np.abs(hp - s.hp).max() < 1e-12 * scale and np.abs(hc - s.hc).max() < 1e-12 * scale
