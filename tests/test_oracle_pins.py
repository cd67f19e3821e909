"""Pins of the FP64 oracle against what the paper and mathematics fix.

None of these re-calls the oracle to check itself: each compares it with a
closed form, an identity the paper states, a textbook bound, or an
independently written high-precision brute force (test_oracle_bruteforce.py).
"""
import math

import numpy as np
import pytest

import synth

C = 299792458.0
AU = 1.495978707e11
YEAR = 31557600.0
OMEGA = 2 * math.pi / YEAR


# ---------------------------------------------------------------------------
# G1/G2: propagation triad and antenna patterns (Sec. II A)
# ---------------------------------------------------------------------------

def test_triad_orthonormal_right_handed(oracle_mod):
    rng = np.random.default_rng(1)
    for _ in range(50):
        beta, lam = math.asin(rng.uniform(-1, 1)), rng.uniform(0, 2 * math.pi)
        k, u, v = oracle_mod.sky_basis(beta, lam)
        M = np.stack([u, v, k])
        assert np.allclose(M @ M.T, np.eye(3), atol=1e-15)
        assert np.allclose(np.cross(u, v), k, atol=1e-15)
        # k points away from the source: k = -e_r with e_r toward (beta, lam)
        e_r = np.array([math.cos(beta) * math.cos(lam), math.cos(beta) * math.sin(lam), math.sin(beta)])
        assert np.allclose(k, -e_r, atol=1e-15)


def test_antenna_pattern_identity(oracle_mod):
    # xi+^2 + xix^2 = ((u.n)^2 + (v.n)^2)^2 = (1 - (k.n)^2)^2 for unit n
    rng = np.random.default_rng(2)
    for _ in range(50):
        k, u, v = oracle_mod.sky_basis(math.asin(rng.uniform(-1, 1)), rng.uniform(0, 2 * math.pi))
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        xp, xc = oracle_mod.antenna(u, v, n)
        assert abs(xp * xp + xc * xc - (1 - np.dot(k, n) ** 2) ** 2) < 1e-14


def test_polarisation_angle_symmetry(oracle_mod):
    # psi -> psi + pi leaves h^SSB unchanged, psi -> psi + pi/2 negates it (Eqs. hplus_ssb, hcross_ssb)
    s = synth.cfg1_source()
    g = s.grid
    o = oracle_mod.Orbit()
    idx = np.arange(200, 8600, 97)
    y0 = oracle_mod.links_full(o, (s.beta, s.lam, s.psi), g, s.hp, s.hc, g, idx)
    y1 = oracle_mod.links_full(o, (s.beta, s.lam, s.psi + math.pi), g, s.hp, s.hc, g, idx)
    y2 = oracle_mod.links_full(o, (s.beta, s.lam, s.psi + 0.5 * math.pi), g, s.hp, s.hc, g, idx)
    scale = np.abs(y0).max()
    assert np.abs(y1 - y0).max() <= 1e-13 * scale
    assert np.abs(y2 + y0).max() <= 1e-13 * scale


# ---------------------------------------------------------------------------
# I1: 32-point Lagrange interpolation
# ---------------------------------------------------------------------------

def test_lagrange_reproduces_polynomials(oracle_mod):
    rng = np.random.default_rng(3)
    x = np.arange(80, dtype=np.float64)
    for deg in (0, 1, 5, 17, 31):
        roots = rng.uniform(20, 60, deg)
        p = lambda xx: np.prod([(xx - r) / 20.0 for r in roots], axis=0) if deg else np.ones_like(xx)
        h = p(x)
        for _ in range(20):
            j = int(rng.integers(16, 63))
            eps = rng.uniform(0, 1)
            got = oracle_mod.lagrange32(h, j, eps)
            want = p(np.array([j + eps]))[0]
            assert abs(got - want) <= 1e-9 * max(1.0, np.abs(h[j - 15:j + 17]).max()), (deg, got, want)


def test_lagrange_sample_points_and_centering(oracle_mod):
    rng = np.random.default_rng(4)
    h = rng.standard_normal(100)
    for j in (20, 50, 77):
        assert oracle_mod.lagrange32(h, j, 0.0) == h[j]
    # stencil j-15..j+16 is symmetric about j + 1/2: interpolating the mirrored
    # series at 1 - eps gives the same value (a shifted stencil breaks this).
    hm = h[::-1].copy()
    for _ in range(30):
        j = int(rng.integers(20, 78))
        eps = rng.uniform(0.01, 0.99)
        a = oracle_mod.lagrange32(h, j, eps)
        jm = 100 - 2 - j
        b = oracle_mod.lagrange32(hm, jm, 1 - eps)
        assert abs(a - b) < 1e-12


def test_lagrange_sinusoid_error_bound(oracle_mod):
    # |f - p| <= prod|eps - m| * w^32 / 32!  for f = cos(w x)
    rng = np.random.default_rng(5)
    for w in (0.6, 1.0, 1.4):
        x = np.arange(100, dtype=np.float64)
        h = np.cos(w * x + 0.3)
        for _ in range(20):
            j = int(rng.integers(20, 78))
            eps = rng.uniform(0, 1)
            err = abs(oracle_mod.lagrange32(h, j, eps) - math.cos(w * (j + eps) + 0.3))
            bound = np.prod([abs(eps - m) for m in range(-15, 17)]) * w ** 32 / math.factorial(32)
            assert err <= bound * 1.0001 + 1e-14


def test_lagrange_zero_padding(oracle_mod):
    rng = np.random.default_rng(6)
    h = rng.standard_normal(40)
    hp = np.concatenate([np.zeros(20), h, np.zeros(20)])
    for j in (-10, -1, 0, 3, 30, 39, 45):
        eps = rng.uniform(0, 1)
        assert abs(oracle_mod.lagrange32(h, j, eps) - oracle_mod.lagrange32(hp, j + 20, eps)) < 1e-13


def test_locate_splits_time_exactly(oracle_mod):
    g = (4.0e7, 10.0, 100000)
    for i, d in [(0, 0.0), (5, 10.0), (99999, 483.25), (12345, -3.75), (7, 0.1)]:
        j, e = oracle_mod.locate(g, i, d, g)
        assert 0.0 <= e < 1.0
        assert abs((j + e) - (i - d / 10.0)) < 1e-12


# ---------------------------------------------------------------------------
# R1: orbits and light times
# ---------------------------------------------------------------------------

def _arms(o, oracle_mod, t):
    R = np.stack([oracle_mod.position(o, s, t) for s in range(3)])
    return R, [np.linalg.norm(R[a] - R[b]) for a, b in ((0, 1), (1, 2), (2, 0))]


def test_orbit_geometry_kepler1(oracle_mod):
    o = oracle_mod.Orbit()
    ts = np.linspace(0, YEAR, 40)
    for t in ts:
        R, arms = _arms(o, oracle_mod, t)
        assert np.all(np.abs(np.array(arms) / 2.5e9 - 1) < 5e-3)
        c = R.mean(axis=0)
        assert abs(np.linalg.norm(c) / AU - 1) < 1e-4
        nrm = np.cross(R[1] - R[0], R[2] - R[0])
        nrm /= np.linalg.norm(nrm)
        # constellation plane inclined 60 degrees to the ecliptic
        assert abs(math.degrees(math.acos(abs(nrm[2]))) - 60.0) < 0.5


def test_kepler2_is_exact_ellipse_and_first_order_kepler1(oracle_mod):
    o1 = oracle_mod.Orbit(kind=oracle_mod.KEPLER1)
    o2 = oracle_mod.Orbit(kind=oracle_mod.KEPLER2)
    e = oracle_mod.eccentricity(2.5e9)
    mu = OMEGA ** 2 * AU ** 3
    for t in np.linspace(1e6, YEAR, 25):
        for s in range(3):
            r1 = oracle_mod.position(o1, s, t)
            r2 = oracle_mod.position(o2, s, t)
            assert np.linalg.norm(r1 - r2) < 5 * e * e * AU  # second order in e; a first-order slip is ~e R
            h = 1.0
            v = (oracle_mod.position(o2, s, t + h) - oracle_mod.position(o2, s, t - h)) / (2 * h)
            energy = 0.5 * v @ v - mu / np.linalg.norm(r2)
            assert abs(energy / (-mu / (2 * AU)) - 1) < 1e-8


def test_light_time_solves_its_equation(oracle_mod):
    for kind in (oracle_mod.KEPLER1, oracle_mod.KEPLER2):
        o = oracle_mod.Orbit(kind=kind)
        for t in (1e6, 4e7, 9.1e7):
            for li in range(6):
                T = oracle_mod.light_time(o, li, t)
                s, r = [(2, 1), (1, 2), (0, 2), (2, 0), (1, 0), (0, 1)][li]
                d = oracle_mod.position(o, r, t) - oracle_mod.position(o, s, t - T)
                assert abs(np.linalg.norm(d) - C * T) < 1e-5


def test_sagnac_amplitude_matches_paper_formula(oracle_mod):
    # Eq. (L_of_t): L_l - L_-l = 2 (R Omega L / c) sin(Omega t - delta)  ->  amplitude 2 R Omega L / c^2 in time
    o = oracle_mod.Orbit()
    ts = np.linspace(0, YEAR, 200)
    amp_expect = 2 * AU * OMEGA * 2.5e9 / C / C
    for pair in ((0, 1), (2, 3), (4, 5)):
        diff = np.array([oracle_mod.light_time(o, pair[0], t) - oracle_mod.light_time(o, pair[1], t) for t in ts])
        amp = 0.5 * (diff.max() - diff.min())
        assert abs(amp / amp_expect - 1) < 0.1, (pair, amp, amp_expect)


# ---------------------------------------------------------------------------
# C1: static constellation, monochromatic wave: sinc closed form (App. C)
# ---------------------------------------------------------------------------

def _static_setup(oracle_mod, f, n=2000, dt=5.0, t0=3.0e7):
    o = oracle_mod.Orbit(kind=oracle_mod.STATIC, t_static=2.2e7)
    beta, lam, psi = 0.41, 2.3, 0.77
    hp, hc = synth.monochromatic(t0, dt, n, f, 1.3, 0.7, 0.4)
    return o, (beta, lam, psi), (t0, dt, n), hp, hc


def _closed_form_links(oracle_mod, o, sky, grid, f, idx):
    """y_l(t) = Re[-i w T/2 sinc(w T (1-k.n)/2) H^ e^{i(theta - w (ds+dr)/2)}]."""
    beta, lam, psi = sky
    k = np.array([-math.cos(beta) * math.cos(lam), -math.cos(beta) * math.sin(lam), -math.sin(beta)])
    u = np.array([math.sin(lam), -math.cos(lam), 0.0])
    v = np.array([-math.sin(beta) * math.cos(lam), -math.sin(beta) * math.sin(lam), math.cos(beta)])
    c2, s2 = math.cos(2 * psi), math.sin(2 * psi)
    w = 2 * math.pi * f
    t0, dt, n = grid
    R = np.stack([oracle_mod.position(o, s, 0.0) for s in range(3)])
    out = np.zeros((6, len(idx)))
    for li, (s, r) in enumerate([(2, 1), (1, 2), (0, 2), (2, 0), (1, 0), (0, 1)]):
        d = R[r] - R[s]
        T = np.linalg.norm(d) / C
        nl = d / np.linalg.norm(d)
        un, vn, kn = u @ nl, v @ nl, k @ nl
        xp, xc = un * un - vn * vn, 2 * un * vn
        Hh = xp * (1.3 * c2 + 1j * 0.7 * s2) + xc * (1.3 * s2 - 1j * 0.7 * c2)
        ds = T + k @ R[s] / C
        dr = k @ R[r] / C
        tt = np.asarray(idx) * dt
        theta = w * tt + 0.4
        x = w * T * (1 - kn) / 2
        out[li] = np.real(-1j * w * T / 2 * (np.sin(x) / x) * Hh * np.exp(1j * (theta - w * (ds + dr) / 2)))
    return out


@pytest.mark.parametrize("f", [1e-3, 1e-2])
def test_static_monochromatic_links_closed_form(oracle_mod, f):
    o, sky, grid, hp, hc = _static_setup(oracle_mod, f)
    idx = np.arange(300, 1700, 37)
    y = oracle_mod.links_full(o, sky, grid, hp, hc, grid, idx)
    yc = _closed_form_links(oracle_mod, o, sky, grid, f, idx)
    assert np.abs(y - yc).max() <= 1e-12 * np.abs(yc).max()


@pytest.mark.parametrize("gen", [15, 20])
def test_static_monochromatic_tdi_closed_form(oracle_mod, gen):
    # X written out from Eqs. (X1.5), (X2.0) with exact phasors (no interpolation)
    f = 4e-3
    o, sky, grid, hp, hc = _static_setup(oracle_mod, f)
    idx = np.arange(400, 1600, 53)
    y = oracle_mod.links_full(o, sky, grid, hp, hc, grid)
    X = oracle_mod.tdi_from_y(o, grid, y, gen, oracle_mod.FROZEN, grid, idx)
    w = 2 * math.pi * f
    R = np.stack([oracle_mod.position(o, s, 0.0) for s in range(3)])
    T = {}
    for li, (s, r) in enumerate([(2, 1), (1, 2), (0, 2), (2, 0), (1, 0), (0, 1)]):
        T[[1, -1, 2, -2, 3, -3][li]] = np.linalg.norm(R[r] - R[s]) / C
    # complex amplitude of each link so that y_l(t) = Re[Y_l e^{i w t}]
    lab = [1, -1, 2, -2, 3, -3]
    Yc = {}
    tt = np.array([400.0, 401.0])
    yy = _closed_form_links(oracle_mod, o, sky, grid, f, tt)
    for li, l in enumerate(lab):
        # solve a cos(th) - b sin(th) for Y = a + i b
        th = w * tt * grid[1]
        A = np.array([[math.cos(th[0]), -math.sin(th[0])], [math.cos(th[1]), -math.sin(th[1])]])
        a, b = np.linalg.solve(A, yy[li])
        Yc[l] = a + 1j * b

    def ydel(l, D):
        return Yc[l] * np.exp(-1j * w * D)

    L = T
    X15 = (ydel(-3, L[-2] + L[2] + L[3]) - ydel(-3, L[3]) + ydel(3, L[2] + L[-2]) - ydel(3, 0)
           + ydel(2, L[-2]) - ydel(2, L[-2] + L[-3] + L[3]) + ydel(-2, 0) - ydel(-2, L[-3] + L[3]))
    Xc = X15
    if gen == 20:
        Xc = X15 + (ydel(-3, L[-2] + L[2] + 2 * L[3] + L[-3]) - ydel(-3, 2 * L[3] + L[-3] + 2 * L[-2] + 2 * L[2])
                    + ydel(3, L[-2] + L[2] + L[3] + L[-3]) - ydel(3, L[3] + L[-3] + 2 * L[-2] + 2 * L[2])
                    + ydel(2, 2 * L[-2] + L[2] + 2 * L[3] + 2 * L[-3]) - ydel(2, L[3] + L[-3] + 2 * L[-2] + L[2])
                    + ydel(-2, L[-2] + L[2] + 2 * L[3] + 2 * L[-3]) - ydel(-2, L[3] + L[-3] + L[-2] + L[2]))
    want = np.real(Xc * np.exp(1j * w * idx * grid[1]))
    assert np.abs(X[0] - want).max() <= 1e-11 * np.abs(want).max()


# ---------------------------------------------------------------------------
# T1: X2.0(t) = X1.5(t) - X1.5(t - 4L/c) for equal constant arms
# ---------------------------------------------------------------------------

def test_tdi20_equal_arm_identity(oracle_mod):
    L = 8.0 * C   # L/c = 8 s, an integer number of 2 s samples: no interpolation
    o = oracle_mod.Orbit(delay=oracle_mod.DELAY_EQUAL, L_m=L)
    rng = np.random.default_rng(7)
    g = (1.0e7, 2.0, 600)
    y = rng.standard_normal((6, 600))
    x15 = oracle_mod.tdi_from_y(o, g, y, 15)
    x20 = oracle_mod.tdi_from_y(o, g, y, 20)
    sh = 16  # 4 L/c / dt
    lhs = x20[:, sh:]
    rhs = x15[:, sh:] - x15[:, :-sh]
    assert np.abs(lhs - rhs).max() < 1e-12


# ---------------------------------------------------------------------------
# T2: laser-noise cancellation
# ---------------------------------------------------------------------------

_SR = [(2, 1), (1, 2), (0, 2), (2, 0), (1, 0), (0, 1)]


def _laser_links(o, oracle_mod, tones, grid):
    # tones are evaluated in time relative to t0 so that t - T keeps full precision
    t0, dt, n = grid
    trel = np.arange(n) * dt
    y = np.zeros((6, n))
    for li, (s, r) in enumerate(_SR):
        T = np.array([oracle_mod.light_time(o, li, t0 + ti) for ti in trel])
        y[li] = synth.eval_tones(tones[s], trel - T) - synth.eval_tones(tones[r], trel)
    return y


def test_laser_noise_static_unequal_arms_cancels(oracle_mod):
    T0 = (8.1, 8.1, 8.5, 8.5, 8.25, 8.25)
    o = oracle_mod.Orbit(delay=oracle_mod.DELAY_LINEAR, lin_T0=T0, lin_Tdot=(0.0,) * 6, t_ref=1.0e7)
    tones = synth.laser_noise_tones(11)
    g = (1.0e7, 1.0, 600)
    y = _laser_links(o, oracle_mod, tones, g)
    for gen in (15, 20):
        for mode in (oracle_mod.FROZEN, oracle_mod.NESTED):
            X = oracle_mod.tdi_from_y(o, g, y, gen, mode)
            inner = X[:, 120:580]
            assert np.abs(inner).max() < 1e-11 * np.abs(y).max(), (gen, mode, np.abs(inner).max())
    # a broken term (wrong sign) would not cancel: sanity of the check itself
    X = oracle_mod.tdi_from_y(o, g, y, 15)
    assert np.abs(y).max() > 0.5


def test_laser_noise_flexing_orders(oracle_mod):
    T0 = (8.1, 8.12, 8.5, 8.47, 8.25, 8.27)
    tones = synth.laser_noise_tones(12)
    g = (1.0e7, 1.0, 700)

    def resid(scale, gen):
        Td = tuple(scale * x for x in (1.5e-4, -1e-4, 2e-4, 0.5e-4, -1.5e-4, 1e-4))
        o = oracle_mod.Orbit(delay=oracle_mod.DELAY_LINEAR, lin_T0=T0, lin_Tdot=Td, t_ref=1.0e7 + 350.0)
        y = _laser_links(o, oracle_mod, tones, g)
        X = oracle_mod.tdi_from_y(o, g, y, gen, oracle_mod.NESTED)
        return np.abs(X[:, 150:650]).max()

    r15a, r15b = resid(1.0, 15), resid(0.5, 15)
    r20a, r20b = resid(1.0, 20), resid(0.5, 20)
    assert 1.8 < r15a / r15b < 2.2
    assert 3.5 < r20a / r20b < 4.5
    assert r20a < 0.05 * r15a


# ---------------------------------------------------------------------------
# L1-L3: low-frequency approximation
# ---------------------------------------------------------------------------

def _lfa_vs_full(oracle_mod, o, f, gen, kind, n=3000, dt=5.0, t0=3.0e7):
    sky = (0.41, 2.3, 0.77)
    hp, hc = synth.monochromatic(t0, dt, n, f, 1.0, 0.8, 0.2)
    g = (t0, dt, n)
    full = oracle_mod.response_full(o, sky, g, hp, hc, gen)
    lfa = oracle_mod.response_lfa(o, sky, g, hp, hc, gen, kind)
    sl = slice(400, n - 400)
    return np.abs(lfa[:, sl] - full[:, sl]).max() / np.abs(full[:, sl]).max()


@pytest.mark.parametrize("gen", [15, 20])
def test_lfa_converges_as_f_squared(oracle_mod, gen):
    o = oracle_mod.Orbit(kind=oracle_mod.STATIC, t_static=2.2e7)
    fs = np.array([2e-4, 5e-4, 1e-3, 2e-3, 5e-3])
    errs = np.array([_lfa_vs_full(oracle_mod, o, f, gen, oracle_mod.LFA_UNEQUAL) for f in fs])
    slope = np.polyfit(np.log(fs), np.log(errs), 1)[0]
    assert 1.8 < slope < 2.2, (slope, errs)


def _link_lfa_err(oracle_mod, o, f, kind, n=3000, dt=5.0, t0=3.0e7):
    sky = (0.41, 2.3, 0.77)
    hp, hc = synth.monochromatic(t0, dt, n, f, 1.0, 0.8, 0.2)
    g = (t0, dt, n)
    yf = oracle_mod.links_full(o, sky, g, hp, hc, g)
    yl = oracle_mod.links_lfa_own(o, sky, g, hp, hc, kind, g)
    sl = slice(400, n - 400)
    return yl[:, sl] - yf[:, sl], np.abs(yf[:, sl]).max()


def test_lfa_expansion_point_orders(oracle_mod):
    # App. B, "Other finite differences": expanding the link around
    # tau_eps = t - delta_s + eps (delta_s - delta_r), the m = 2 term of the
    # series has the coefficient (1 - 2 eps)/2, zero only at the central
    # point.  So on a rigid static constellation the leading-term link error
    # falls as f^2 (relative) at eps = 1/2 and as f at eps = 0 (backward) and
    # eps = 1 (forward), and the backward and forward errors are opposite at
    # leading order: their mean falls as f^2 again.
    o = oracle_mod.Orbit(kind=oracle_mod.STATIC, t_static=2.2e7)
    fs = np.array([2e-4, 5e-4, 1e-3, 2e-3])
    slope = lambda e: np.polyfit(np.log(fs), np.log(e), 1)[0]
    ec, eb, ef, em = [], [], [], []
    for f in fs:
        dc, sc = _link_lfa_err(oracle_mod, o, f, oracle_mod.LFA_UNEQUAL)
        db, _ = _link_lfa_err(oracle_mod, o, f, oracle_mod.LFA_BACKWARD)
        df, _ = _link_lfa_err(oracle_mod, o, f, oracle_mod.LFA_FORWARD)
        ec.append(np.abs(dc).max() / sc)
        eb.append(np.abs(db).max() / sc)
        ef.append(np.abs(df).max() / sc)
        em.append(np.abs(0.5 * (db + df)).max() / sc)
    assert 1.9 < slope(ec) < 2.1, ec
    assert 0.9 < slope(eb) < 1.1, eb
    assert 0.9 < slope(ef) < 1.1, ef
    assert 1.8 < slope(em) < 2.2, em
    # at 1 mHz the non-central errors are ~100x the central one
    assert eb[2] > 50 * ec[2] and ef[2] > 50 * ec[2]
    # the backward point is the sender end: at f -> 0 all three agree with the full link
    assert max(eb[0], ef[0]) < 1e-2


def test_lfa_noncentral_leading_error_term(oracle_mod):
    # Which end is which: on a static constellation the full link is
    # y = -[H(t - delta_s) - H(t - delta_r)] / (2 (1 - k.n)); expanding about the
    # sender end (backward) leaves y_back - y = -(Delta/2) dy/dt and about the
    # receiver end (forward) +(Delta/2) dy/dt at leading order, with
    # Delta = delta_s - delta_r = T_l (1 - k.n_l) from the constellation's
    # positions (y_slr: sender s, receiver r; links +1,-1,+2,-2,+3,-3).
    sender, receiver = (2, 1, 0, 2, 1, 0), (1, 2, 2, 0, 0, 1)
    t_st = 2.2e7
    o = oracle_mod.Orbit(kind=oracle_mod.STATIC, t_static=t_st)
    sky = (0.41, 2.3, 0.77)
    k, _, _ = oracle_mod.sky_basis(sky[0], sky[1])
    t0, dt, n, f = 3.0e7, 5.0, 3000, 5e-4
    g = (t0, dt, n)
    hp, hc = synth.monochromatic(t0, dt, n, f, 1.0, 0.8, 0.2)
    yf = oracle_mod.links_full(o, sky, g, hp, hc, g)
    sl = slice(400, n - 400)
    for kind, sign in ((oracle_mod.LFA_BACKWARD, -1.0), (oracle_mod.LFA_FORWARD, +1.0)):
        e = oracle_mod.links_lfa_own(o, sky, g, hp, hc, kind, g) - yf
        for li in range(6):
            Rs = oracle_mod.position(o, sender[li], t_st)
            Rr = oracle_mod.position(o, receiver[li], t_st)
            delta = (np.linalg.norm(Rr - Rs) + k @ (Rs - Rr)) / C
            yd = oracle_mod.hdot(g, yf[li])[sl]
            coef = (e[li, sl] @ yd) / (yd @ yd)
            assert abs(coef - sign * 0.5 * delta) < 0.05 * 0.5 * delta, (kind, li, coef, delta)


def test_lfa_error_floors_moving_orbits(oracle_mod):
    # Sec. III / App. B: with moving arms the unequal-delay LFA is limited at
    # O(R Omega / c) ~ 1e-4 and the equal-delay one at O(e) ~ 1e-3.
    # Flexing Keplerian orbits (1% peak-to-peak arm variation).
    o = oracle_mod.Orbit(kind=oracle_mod.KEPLER2, kepler_tilt=1.01)
    for gen in (15, 20):
        e_uneq = _lfa_vs_full(oracle_mod, o, 1e-4, gen, oracle_mod.LFA_UNEQUAL, n=4000, dt=10.0)
        e_eq = _lfa_vs_full(oracle_mod, o, 1e-4, gen, oracle_mod.LFA_EQUAL, n=4000, dt=10.0)
        assert 3e-5 < e_uneq < 6e-4, e_uneq
        assert 1e-3 < e_eq < 3e-2, e_eq


def test_lfa_generation_relation_equal_arms(oracle_mod):
    # X2.0(t) = (4L/c) dX1.5/dt (t - 2L/c) in the equal-arm LFA
    o = oracle_mod.Orbit(kind=oracle_mod.KEPLER1)
    Tl = 2.5e9 / C
    s = synth.cfg1_source()
    g = s.grid
    sky = (s.beta, s.lam, s.psi)
    x15 = oracle_mod.response_lfa(o, sky, g, s.hp, s.hc, 15, oracle_mod.LFA_EQUAL)
    x20 = oracle_mod.response_lfa(o, sky, g, s.hp, s.hc, 20, oracle_mod.LFA_EQUAL)
    dx15 = np.stack([oracle_mod.hdot(g, x15[c]) for c in range(3)])
    idx = np.arange(200, 7000)
    shifted = np.stack([[oracle_mod.lagrange32(dx15[c], *oracle_mod.locate(g, i, 2 * Tl, g)) for i in idx]
                        for c in range(3)])
    want = 4 * Tl * shifted
    got = x20[:, idx]
    assert np.abs(got - want).max() < 1e-4 * np.abs(want).max()


def test_lfa_equal_arms_T_channel_vanishes(oracle_mod):
    o = oracle_mod.Orbit(kind=oracle_mod.KEPLER1)
    s = synth.cfg1_source()
    aet = oracle_mod.response_lfa(o, (s.beta, s.lam, s.psi), s.grid, s.hp, s.hc, 20, oracle_mod.LFA_EQUAL, "aet")
    assert np.abs(aet[2]).max() < 1e-12 * np.abs(aet[:2]).max()


# ---------------------------------------------------------------------------
# AET, hybrid, generators
# ---------------------------------------------------------------------------

def test_aet_is_orthonormal(oracle_mod):
    rng = np.random.default_rng(9)
    xyz = rng.standard_normal((3, 50))
    aet = oracle_mod.aet(xyz)
    assert np.allclose((aet ** 2).sum(0), (xyz ** 2).sum(0), rtol=1e-14)
    assert np.allclose(aet[2], xyz.sum(0) / math.sqrt(3), rtol=1e-14)


def test_hybrid_window_structure(oracle_mod):
    s = synth.cfg1_source()
    g = s.grid
    o = oracle_mod.Orbit()
    sky = (s.beta, s.lam, s.psi)
    tH = s.t0 + 0.5 * s.n * s.dt
    Tw, sig = 800 * s.dt, 20 * s.dt
    lfa = oracle_mod.response_lfa(o, sky, g, s.hp, s.hc, 20)
    full = oracle_mod.response_full(o, sky, g, s.hp, s.hc, 20)
    hyb = oracle_mod.response_hybrid(o, sky, g, s.hp, s.hc, 20, t_h=tH, Tw=Tw, sigma=sig)
    t = s.times()
    for ti in t[::50]:
        assert abs(oracle_mod.sigmoid(ti, tH, sig, 1) + oracle_mod.sigmoid(ti, tH, sig, -1) - 1) < 1e-15
    pre = t < tH - Tw / 2
    post = t > tH + Tw / 2
    wl = 1 / (1 + np.exp((t - tH) / sig))
    wf = 1 / (1 + np.exp(-(t - tH) / sig))
    assert np.array_equal(hyb[:, pre], wl[pre] * lfa[:, pre]) or np.allclose(hyb[:, pre], wl[pre] * lfa[:, pre], rtol=1e-15, atol=0)
    assert np.allclose(hyb[:, post], wf[post] * full[:, post], rtol=1e-15, atol=0)


def test_t_hyb_is_chirp_time_of_f_hyb(oracle_mod):
    for mc in (1e5, 1e6, 5e6):
        mc_s = mc * synth.T_SUN
        for fh in (3e-4, 1e-3):
            tH = oracle_mod.t_hyb(fh, mc_s, 5e7)
            tau = synth.chirp_tau_of_f(fh, mc_s)
            assert abs((5e7 - tH) / tau - 1) < 1e-10  # 5e7 - tH cancels ~7 digits
            assert abs(float(synth.chirp_frequency(5e7 - tH, mc_s)) / fh - 1) < 1e-10


def test_generators_phase_derivative_is_frequency():
    mc_s = 1e6 * synth.T_SUN
    tau = np.linspace(5e3, 3e7, 50)
    h = 1e-3 * tau
    dphi = (synth.chirp_phase(tau - h, mc_s, 0.3) - synth.chirp_phase(tau + h, mc_s, 0.3)) / (2 * h)
    f = synth.chirp_frequency(tau, mc_s)
    assert np.allclose(dphi, 2 * math.pi * f, rtol=1e-5)


# ---------------------------------------------------------------------------
# Higher-order LFA (App. B): next-to-leading order of the central series and
# of the Michelson expansions; the strain-derivative form with the
# constellation centre (Sec. III)
# ---------------------------------------------------------------------------

def _normal_sky(oracle_mod, t_st, psi=0.77):
    """Sky position whose propagation direction is the normal of the static
    constellation's plane (k.n_l = 0 for every link)."""
    o = oracle_mod.Orbit(kind=oracle_mod.STATIC, t_static=t_st)
    R = [oracle_mod.position(o, s, t_st) for s in range(3)]
    nrm = np.cross(R[1] - R[0], R[2] - R[0])
    nrm /= np.linalg.norm(nrm)
    e_r = -nrm   # k = -e_r
    sky = (math.asin(e_r[2]), math.atan2(e_r[1], e_r[0]), psi)
    k, _, _ = oracle_mod.sky_basis(sky[0], sky[1])
    assert abs(k @ nrm - 1.0) < 1e-12
    return o, sky


def _lfa_err(oracle_mod, o, sky, f, gen, kind, n=3000, dt=5.0, t0=3.0e7):
    hp, hc = synth.monochromatic(t0, dt, n, f, 1.0, 0.8, 0.2)
    g = (t0, dt, n)
    full = oracle_mod.response_full(o, sky, g, hp, hc, gen)
    lfa = oracle_mod.response_lfa(o, sky, g, hp, hc, gen, kind)
    sl = slice(400, n - 400)
    return np.abs(lfa[:, sl] - full[:, sl]).max() / np.abs(full[:, sl]).max()


@pytest.mark.parametrize("gen", [15, 20])
def test_lfa_nlo_error_order_normal_incidence(oracle_mod, gen):
    # With the source on the normal of a rigid constellation every link has
    # k.n = 0, so a link and its reverse carry the same m = 1 term: the
    # next-to-leading link term of Eq. yslr_with_tau_derivatives and the next
    # term of the Michelson expansion leave an error of relative order
    # (omega L)^4, against (omega L)^2 at leading order.
    o, sky = _normal_sky(oracle_mod, 2.2e7)
    fs = np.array([5e-4, 1e-3, 2e-3, 5e-3])
    lo = np.array([_lfa_err(oracle_mod, o, sky, f, gen, oracle_mod.LFA_UNEQUAL) for f in fs])
    nlo = np.array([_lfa_err(oracle_mod, o, sky, f, gen, oracle_mod.LFA_NLO) for f in fs])
    slope = lambda e: np.polyfit(np.log(fs), np.log(e), 1)[0]
    assert 1.9 < slope(lo) < 2.1, lo
    assert 3.7 < slope(nlo) < 4.3, nlo
    assert np.all(nlo < 3e-2 * lo), (nlo, lo)
    assert nlo[1] < 1e-3 * lo[1], (nlo, lo)      # at 1 mHz


@pytest.mark.parametrize("gen", [15, 20])
def test_lfa_nlo_error_order_general_direction(oracle_mod, gen):
    # For a general direction a link and its reverse carry m = 1 terms with
    # (1 - k.n) and (1 + k.n); the channels take their mean, which leaves the
    # difference: an error of relative order (omega L)^3, still one order
    # below the leading-order error (omega L)^2.
    o = oracle_mod.Orbit(kind=oracle_mod.STATIC, t_static=2.2e7)
    sky = (0.41, 2.3, 0.77)
    fs = np.array([5e-4, 1e-3, 2e-3, 5e-3])
    lo = np.array([_lfa_err(oracle_mod, o, sky, f, gen, oracle_mod.LFA_UNEQUAL) for f in fs])
    nlo = np.array([_lfa_err(oracle_mod, o, sky, f, gen, oracle_mod.LFA_NLO) for f in fs])
    slope = lambda e: np.polyfit(np.log(fs), np.log(e), 1)[0]
    assert 1.9 < slope(lo) < 2.1, lo
    assert 2.7 < slope(nlo) < 3.6, nlo
    assert np.all(nlo < 2.5e-2 * lo), (nlo, lo)


def test_lfa_nlo_link_error_order(oracle_mod):
    # The link alone (at its own time, its own (1 - k.n)): the central series
    # has odd powers only, so after the m = 1 term the error is O(f^4).
    o = oracle_mod.Orbit(kind=oracle_mod.STATIC, t_static=2.2e7)
    fs = np.array([2e-4, 5e-4, 1e-3, 2e-3, 5e-3])
    e_lo, e_nlo = [], []
    for f in fs:
        d, sc = _link_lfa_err(oracle_mod, o, f, oracle_mod.LFA_UNEQUAL)
        d2, _ = _link_lfa_err(oracle_mod, o, f, oracle_mod.LFA_NLO)
        e_lo.append(np.abs(d).max() / sc)
        e_nlo.append(np.abs(d2).max() / sc)
    slope = lambda e: np.polyfit(np.log(fs), np.log(e), 1)[0]
    assert 1.9 < slope(e_lo) < 2.1, e_lo
    assert 3.8 < slope(e_nlo) < 4.2, e_nlo


@pytest.mark.parametrize("gen", [15, 20])
def test_strain_form_equals_equal_arm_lfa_at_normal_incidence(oracle_mod, gen):
    # Eqs. X15_with_strain_derivatives, X20_with_strain_derivatives replace
    # k.(R_s + R_r)/2c by k.R0/c in the equal-arm LFA (Eqs. X15_equal,
    # X20_equal).  With k normal to the constellation's plane the two are the
    # same number for every link, and for a rigid constellation the strain
    # form is then the equal-arm LFA itself: the derivative stencil applied
    # on the h grid before interpolation equals the one applied to the
    # interpolated z series on the output grid (unit ratio).
    t0, dt, n, f = 3.0e7, 5.0, 3000, 1e-3
    o, sky = _normal_sky(oracle_mod, 2.2e7)
    hp, hc = synth.monochromatic(t0, dt, n, f, 1.0, 0.8, 0.2)
    g = (t0, dt, n)
    eq = oracle_mod.response_lfa(o, sky, g, hp, hc, gen, oracle_mod.LFA_EQUAL)
    st = oracle_mod.response_lfa(o, sky, g, hp, hc, gen, oracle_mod.LFA_STRAIN)
    sl = slice(400, n - 400)
    assert np.abs(st[:, sl] - eq[:, sl]).max() <= 1e-11 * np.abs(eq[:, sl]).max()


def test_strain_form_leading_difference_and_T(oracle_mod):
    # General direction, rigid constellation: the equal-arm LFA's link y_l is
    # the strain form's shifted by delta_l = k.((R_s + R_r)/2 - R0)/c, so at
    # leading order X_equal - X_strain = -2 T^2 [G_3 delta_3 - G_2 delta_2]
    # d3h/dt3 (TDI 1.5), G_l the link's projection of h^SSB (xi from Eqs.
    # xi_plus, xi_cross).  And X + Y + Z = 0 identically in the strain form
    # (the xi differences are cyclic), so T vanishes.
    t_st, t0, dt, n, f = 2.2e7, 3.0e7, 5.0, 3000, 1e-3
    o = oracle_mod.Orbit(kind=oracle_mod.STATIC, t_static=t_st)
    beta, lam, psi = 0.41, 2.3, 0.77
    k, u, v = oracle_mod.sky_basis(beta, lam)
    A, B, ph0 = 1.0, 0.8, 0.2
    hp, hc = synth.monochromatic(t0, dt, n, f, A, B, ph0)
    g = (t0, dt, n)
    eq = oracle_mod.response_lfa(o, (beta, lam, psi), g, hp, hc, 15, oracle_mod.LFA_EQUAL)
    st = oracle_mod.response_lfa(o, (beta, lam, psi), g, hp, hc, 15, oracle_mod.LFA_STRAIN)
    T = 2.5e9 / C
    R = [oracle_mod.position(o, s, t_st) for s in range(3)]
    R0 = (R[0] + R[1] + R[2]) / 3.0
    t = t0 + np.arange(n) * dt
    tau0 = t - 2 * T - (k @ R0) / C
    w = 2 * math.pi * f
    # third derivatives of h+ = A cos(w (t - t0) + ph0), hx = B sin(...), rotated by psi
    d3p = A * w ** 3 * np.sin(w * (tau0 - t0) + ph0)
    d3c = -B * w ** 3 * np.cos(w * (tau0 - t0) + ph0)
    c2, s2 = math.cos(2 * psi), math.sin(2 * psi)
    Hp, Hc = d3p * c2 - d3c * s2, d3p * s2 + d3c * c2

    def proj(sender, receiver):
        nl = R[receiver] - R[sender]
        nl = nl / np.linalg.norm(nl)
        xp, xc = oracle_mod.antenna(u, v, nl)
        delta = (k @ (0.5 * (R[sender] + R[receiver]) - R0)) / C
        return xp * Hp + xc * Hc, delta

    G2, d2 = proj(0, 2)    # link +2: y_123 (1 -> 3)
    G3, d3 = proj(1, 0)    # link +3: y_231 (2 -> 1)
    pred = -2 * T * T * (G3 * d3 - G2 * d2)
    sl = slice(400, n - 400)
    got = (eq - st)[0, sl]
    assert abs(d2) > 0.3 and abs(d3) > 0.3      # the shifts are not small here
    assert np.abs(got - pred[sl]).max() <= 0.02 * np.abs(pred[sl]).max()
    aet = oracle_mod.aet(st)
    assert np.abs(aet[2]).max() <= 1e-14 * np.abs(aet[:2]).max()
