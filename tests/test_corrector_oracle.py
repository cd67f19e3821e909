"""Pins of the corrector's FP64 reference (oracle/corrector.py): the stencils,
the local frequency, the scale conventions and the residual law that the
network is trained on, each checked against mathematics or the paper's
formulas rather than against the code itself."""
import math

import numpy as np
import pytest

import synth
from gpu_util import ORBITS
from oracle import corrector as OC

L_M = 2.5e9
TBAR = L_M / OC.C_LIGHT


def test_stencils_exact_for_quartics():
    # 5-point central stencils are exact for polynomials of degree <= 4
    rng = np.random.default_rng(7)
    dt = 5.0
    c = rng.normal(size=5)
    t = (np.arange(11) - 5) * dt / 100.0
    p = np.polynomial.Polynomial(c)
    z = p(t)
    # derivatives with respect to the sample time (t is in units of dt/100)
    q = OC.stencils(z, 5, dt / 100.0, TBAR)
    for k in range(5):
        want = TBAR ** k * p.deriv(k)(0.0) if k else p(0.0)
        assert q[k] == pytest.approx(want, rel=1e-9, abs=1e-9 * TBAR ** k * np.abs(c).max() * 1e4 ** k)


def test_local_frequency_of_a_sinusoid():
    # For z_l = A_l cos(w t + phi_l) the 5-point second difference has the
    # symbol -(32 cos th - 2 cos 2th - 30)/(12 dt^2) (th = w dt), so
    # M_2 / M_0 = Tbar^2 (30 - 32 cos th + 2 cos 2th)/(12 dt^2) exactly.
    rng = np.random.default_rng(11)
    dt = 10.0
    for f in (1e-4, 1e-3, 1.5e-2):
        w = 2 * math.pi * f
        n = 64
        t = np.arange(n) * dt
        A = rng.uniform(0.5, 2.0, 6)
        ph = rng.uniform(0, 2 * math.pi, 6)
        z = A[:, None] * np.cos(w * t[None, :] + ph[:, None])
        T = np.full((6, n), TBAR)
        kn = np.zeros((6, n))
        feats, scale, above, _ = OC.features(z, T, kn, L_M, dt)
        th = w * dt
        sym = TBAR ** 2 * (30 - 32 * math.cos(th) + 2 * math.cos(2 * th)) / (12 * dt ** 2)
        i = n // 2
        M0 = np.abs(z[:, i]).max()
        assert scale[i] * 8 / M0 == pytest.approx(sym, rel=1e-9)
        # the band decision uses the same ratio
        fl = math.sqrt(sym) / (2 * math.pi * TBAR)
        _, s_lo, _, _ = OC.features(z, T, kn, L_M, dt, f_lo=1.01 * fl)
        _, s_in, ab_in, _ = OC.features(z, T, kn, L_M, dt, f_lo=0.99 * fl, f_hi=1.01 * fl)
        _, _, ab_hi, _ = OC.features(z, T, kn, L_M, dt, f_lo=0.0, f_hi=0.99 * fl)
        assert s_lo[i] == 0.0 and s_in[i] > 0 and not ab_in[i] and ab_hi[i]


def test_scale_invariance():
    rng = np.random.default_rng(3)
    n, dt = 40, 5.0
    z = rng.normal(size=(6, n)).cumsum(axis=1) * 1e-21
    y = z * (1 + 1e-3 * rng.normal(size=(6, n)))
    T = TBAR * (1 + 1e-3 * rng.normal(size=(6, n)))
    kn = rng.uniform(-0.9, 0.9, (6, n))
    f1, s1, _, t1 = OC.features(z, T, kn, L_M, dt, y_full=y)
    f2, s2, _, t2 = OC.features(7.5 * z, T, kn, L_M, dt, y_full=7.5 * y)
    assert np.allclose(f1, f2, rtol=1e-12, atol=1e-12)
    assert np.allclose(s2, 7.5 * s1, rtol=1e-12)
    assert np.allclose(t1, t2, rtol=1e-9, atol=1e-9)
    # padding column is zero; geometry columns are the stated maps
    assert np.all(f1[:, 47] == 0) and np.all(f1[:, 46] == dt / TBAR)
    assert np.allclose(f1[:, 40:46].T, 1 - kn)
    assert np.allclose(f1[:, 34:40].T, (T / TBAR - 1) * 100)


def _monochromatic_case(orbit_mod, name, f, n=1000, dt=5.0, t0=2.0e7, sky=(0.3, 1.1, 0.4)):
    orb = orbit_mod.Orbit(**ORBITS[name])
    s = synth.monochromatic(t0, dt, n, f)
    g = (t0, dt, n)
    z = orbit_mod.links_lfa_own(orb, sky, g, s[0], s[1], orbit_mod.LFA_UNEQUAL, g)
    yf = orbit_mod.links_full(orb, sky, g, s[0], s[1], g)
    T, kn = OC.link_geometry(orbit_mod, orb, g, sky[0], sky[1])
    eps = OC.link_eps(orbit_mod, orb, g, sky[0], sky[1])
    return orb, z, yf, T, kn, eps


def test_reversed_lfa_links_coincide_for_a_rigid_static_triangle(oracle_mod):
    # static, equal arms: T_-l = T_+l and n_-l = -n_+l, and the LFA link
    # (Sec. III) is even in n and symmetric in sender/receiver
    orb, z, _, T, kn, eps = _monochromatic_case(oracle_mod, "static", 2e-3, n=300)
    for m in range(3):
        assert np.allclose(z[2 * m], z[2 * m + 1], rtol=0, atol=1e-12 * np.abs(z).max())
    assert np.all(eps == 0.0)


def test_velocity_term_is_the_low_frequency_residual(oracle_mod):
    # At 1e-4 Hz the truncation term ((omega T)^2 (1-k.n)^2/24 < 5e-6) is
    # below the O(v/c) term eps_l ~ 2e-5..4e-5 of moving orbits; the base link
    # z (1 + eps) removes it.
    _, z, yf, _, _, eps = _monochromatic_case(oracle_mod, "kepler2_flex", 1e-4)
    sl = slice(250, 750)
    scale = np.abs(yf[:, sl]).max()
    plain = np.abs(yf[:, sl] - z[:, sl]).max() / scale
    base = np.abs(yf[:, sl] - (z * (1 + eps))[:, sl]).max() / scale
    assert plain > 1e-5
    assert base < 5e-6


@pytest.mark.parametrize("f,tol", [(1e-3, 1e-3), (3e-3, 1e-2)])
def test_leading_order_residual_law(oracle_mod, f, tol):
    # y_l - z_l (1 + eps_l) = (1 - k.n_l)^2 T_l^2/24 z_l'' + O((omega T)^4):
    # in the training target's units, target_l = f[40+l]^2/3 (T_l/Tbar)^2 f[12+l]
    orb, z, yf, T, kn, eps = _monochromatic_case(oracle_mod, "kepler2_flex", f)
    feats, scale, _, target = OC.features(z, T, kn, orb.L_m, 5.0, y_full=yf, eps=eps)
    Tbar = orb.L_m / OC.C_LIGHT
    sl = slice(250, 750)
    pred = np.stack([feats[:, 40 + l] ** 2 / 3 * (T[l] / Tbar) ** 2 * feats[:, 12 + l] for l in range(6)], 1)
    dev = np.abs(pred[sl] - target[sl]).max() / np.abs(target[sl]).max()
    assert dev < tol
    assert 0.1 < np.abs(target[sl]).max() < 1.4
