"""Pins of the likelihood-tail oracle (oracle/noise.py) against what the paper
and the mathematics fix, independently of its own formulas:

  * structural zeros: every A/E/T PSD term carries sin^2(x), x = 2 pi f L/c,
    so the PSDs vanish at f = c/(2L); TDI 2.0 adds Lam = 4 sin^2(2x), zero at
    f = c/(4L) (Sec. II C, Eqs. SnAE, SnT);
  * the TDI 2.0 / 1.5 ratio is 4 sin^2(2x) at every frequency;
  * power laws of the instrument noises (log-log slopes): S_pm ~ f^-4 well
    below 0.4 mHz, f^-2 between 0.4 and 8 mHz, f^2 well above; S_op ~ f^-2
    well below 2 mHz, f^2 well above;
  * the foreground knees for T_obs = 1 yr are 10^b1 and 10^bk;
  * low-frequency T suppression: S^T / S^{A,E} -> 2 (x^2/2 S_op + x^4/2 S_pm) /
    (12 S_pm + 3 S_op) (the 16/8 prefactors and the x -> 0 expansion of the
    cosines) without the galaxy;
  * inner product closed forms: a bin-centred sinusoid A cos(2 pi f_k t) on a
    flat PSD gives <x|x> = A^2 N dt / S (Parseval); sinusoids on different
    bins are orthogonal; <x|y> is symmetric and bilinear;
  * overlap(x, a x) = sign(a) and mismatch(x, x) = 0; an overall time shift
    by a whole number of samples on a periodic signal leaves <x|x> unchanged;
  * zero padding: on a flat PSD covering every bin, <x|y> equals Parseval's
    2 dt sum x y for any transform length, up to the DC and Nyquist bins;
  * fft_length: the smallest 7-smooth number >= n.
"""
import numpy as np
import pytest

from oracle import noise as N

L = 2.5e9
C = 299792458.0


def slope(fun, f0, f1):
    f = np.array([f0, f1])
    v = fun(f)
    return np.log(v[1] / v[0]) / np.log(f1 / f0)


def test_psd_structural_zeros():
    f_pi = C / (2 * L)            # x = pi
    f_half = C / (4 * L)          # x = pi/2, where Lam(2.0) = 4 sin^2(pi) = 0
    for gen in (15, 20):
        sae, st = N.psd_aet(np.array([f_pi]), gen, L)
        ref = N.psd_aet(np.array([0.9 * f_pi]), gen, L)
        assert sae[0] < 1e-12 * ref[0][0] and st[0] < 1e-12 * ref[1][0]
    sae, st = N.psd_aet(np.array([f_half]), 20, L)
    ref = N.psd_aet(np.array([0.9 * f_half]), 20, L)
    assert sae[0] < 1e-12 * ref[0][0] and st[0] < 1e-12 * ref[1][0]
    sae15, _ = N.psd_aet(np.array([f_half]), 15, L)
    assert sae15[0] > 0


def test_tdi20_over_tdi15_ratio():
    f = np.logspace(-4.5, -1.2, 200)
    x = 2 * np.pi * f * L / C
    for gal in (True, False):
        a20, t20 = N.psd_aet(f, 20, L, 1.0, gal)
        a15, t15 = N.psd_aet(f, 15, L, 1.0, gal)
        lam = 4 * np.sin(2 * x) ** 2
        np.testing.assert_allclose(a20, lam * a15, rtol=1e-12)
        np.testing.assert_allclose(t20, lam * t15, rtol=1e-12, atol=1e-300)


def test_instrument_power_laws():
    assert abs(slope(N.s_pm, 1e-6, 2e-6) + 4.0) < 1e-3
    assert abs(slope(N.s_pm, 2.5e-3, 2.6e-3) + 2.0) < 0.05
    assert abs(slope(N.s_pm, 10.0, 11.0) - 2.0) < 1e-3
    assert abs(slope(N.s_op, 1e-6, 2e-6) + 2.0) < 1e-3
    assert abs(slope(N.s_op, 10.0, 11.0) - 2.0) < 1e-3


def test_instrument_amplitudes():
    # S_pm at 1 mHz: S_acc / (2 pi f c)^2 times the two corrections
    f = 1e-3
    want = 2.4e-15 ** 2 / (2 * np.pi * f * C) ** 2 * (1 + 0.4 ** 2) * (1 + (1 / 8) ** 4)
    assert N.s_pm(f) == pytest.approx(want, rel=1e-14)
    want = 7.9e-12 ** 2 * (2 * np.pi * f / C) ** 2 * (1 + 2.0 ** 4)
    assert N.s_op(f) == pytest.approx(want, rel=1e-14)


def test_galaxy_knees_one_year():
    f1, fk = N.gal_knees(1.0)
    assert f1 == pytest.approx(10 ** -2.70408439, rel=1e-14)
    assert fk == pytest.approx(10 ** -2.37822436, rel=1e-14)
    # the foreground is switched off well above the knee and vanishes at x = pi
    assert N.s_gal(np.array([3e-2]), L)[0] < 1e-6 * N.s_gal(np.array([1e-3]), L)[0]


def test_low_frequency_t_suppression():
    f = np.array([2e-5, 5e-5])
    x = 2 * np.pi * f * L / C
    a, t = N.psd_aet(f, 15, L, 1.0, galaxy=False)
    pm, op = N.s_pm(f), N.s_op(f)
    want = 2.0 * (x ** 2 / 2 * op + x ** 4 / 2 * pm) / (12 * pm + 3 * op)
    np.testing.assert_allclose(t / a, want, rtol=5e-3)


def test_inner_product_parseval_sinusoid():
    n, dt = 4096, 5.0
    k = 300
    fk = k / (n * dt)
    t = np.arange(n) * dt
    A = 3.0
    x = np.zeros((3, n))
    x[0] = A * np.cos(2 * np.pi * fk * t)
    x[1] = A * np.sin(2 * np.pi * fk * t)
    x[2] = 0.5 * A * np.cos(2 * np.pi * fk * t + 0.3)
    ip = N.inner_aet(x, x, dt, 1e-5, 5e-2, 15, L)
    sae, st = N.psd_aet(np.array([fk]), 15, L)
    assert ip[0, 1] == pytest.approx(A ** 2 * n * dt / sae[0], rel=1e-12)
    assert ip[1, 1] == pytest.approx(A ** 2 * n * dt / sae[0], rel=1e-12)
    assert ip[2, 1] == pytest.approx(0.25 * A ** 2 * n * dt / st[0], rel=1e-12)


def test_inner_product_orthogonality_symmetry_bilinearity():
    rng = np.random.default_rng(7)
    n, dt = 2048, 10.0
    t = np.arange(n) * dt
    x = np.zeros((3, n))
    y = np.zeros((3, n))
    for c in range(3):
        x[c] = np.cos(2 * np.pi * 100 / (n * dt) * t)
        y[c] = np.cos(2 * np.pi * 140 / (n * dt) * t)
    ip = N.inner_aet(x, y, dt, 1e-5, 4e-2, 20, L)
    assert np.all(np.abs(ip[:, 0]) < 1e-10 * np.sqrt(ip[:, 1] * ip[:, 2]))
    a = rng.standard_normal((3, n))
    b = rng.standard_normal((3, n))
    c = rng.standard_normal((3, n))
    ab = N.inner_aet(a, b, dt, 1e-4, 4e-2, 20, L)
    ba = N.inner_aet(b, a, dt, 1e-4, 4e-2, 20, L)
    np.testing.assert_allclose(ab[:, 0], ba[:, 0], rtol=1e-12)
    a_bc = N.inner_aet(a, 2.0 * b - 3.0 * c, dt, 1e-4, 4e-2, 20, L)[:, 0]
    lin = 2.0 * ab[:, 0] - 3.0 * N.inner_aet(a, c, dt, 1e-4, 4e-2, 20, L)[:, 0]
    np.testing.assert_allclose(a_bc, lin, rtol=1e-9, atol=1e-9 * np.abs(lin).max())


def test_overlap_and_mismatch():
    rng = np.random.default_rng(3)
    n, dt = 1024, 5.0
    x = rng.standard_normal((3, n))
    ip = N.inner_aet(x, -2.5 * x, dt, 1e-4, 8e-2, 20, L)
    np.testing.assert_allclose(N.overlap(ip), -1.0, rtol=1e-12)
    np.testing.assert_allclose(N.mismatch(ip), 0.0, atol=1e-12)
    ip2 = N.inner_aet(x, np.roll(x, 17, axis=-1), dt, 1e-4, 8e-2, 20, L)
    np.testing.assert_allclose(ip2[:, 2], ip[:, 1], rtol=1e-12)   # |x~| unchanged by a cyclic shift


def test_fft_length():
    assert N.fft_length(1) == 1
    assert N.fft_length(6311520) == 6322176   # 2^11 3^2 7^3
    for n in (17, 487, 1000, 4099, 6311520):
        m = N.fft_length(n)
        assert m >= n
        r = m
        for p in (2, 3, 5, 7):
            while r % p == 0:
                r //= p
        assert r == 1
        assert all(not _smooth(k) for k in range(n, m))


def _smooth(k):
    for p in (2, 3, 5, 7):
        while k % p == 0:
            k //= p
    return k == 1


def test_zero_padding_invariance_flat_psd(monkeypatch):
    rng = np.random.default_rng(11)
    n, dt = 1000, 5.0
    x = rng.standard_normal((3, n))
    y = rng.standard_normal((3, n))
    # flat PSD S = 1 and a band covering every bin but DC
    monkeypatch.setattr(N, "psd_aet", lambda f, *a, **k: (np.ones_like(f), np.ones_like(f)))
    ref = None
    for m in (n, 1024, 1536, 4000):
        ip = N.inner_aet(x, y, dt, 1e-12, 1e9, nfft=m)
        # 4 Re sum_{k>=1} X_k^* Y_k df = 2 dt sum x y - 2 X_0 Y_0 df (+ 2 X_{M/2} Y_{M/2} df if M is even:
        # Parseval's two-sided sum holds the Nyquist bin once, the one-sided sum counts it once)
        X = dt * np.fft.rfft(x, n=m)
        Y = dt * np.fft.rfft(y, n=m)
        df = 1.0 / (m * dt)
        want = 2 * dt * np.sum(x * y, axis=1) - 2 * np.real(np.conj(X[:, 0]) * Y[:, 0]) * df
        if m % 2 == 0:
            want += 2 * np.real(np.conj(X[:, -1]) * Y[:, -1]) * df
        np.testing.assert_allclose(ip[:, 0], want, rtol=1e-10)
