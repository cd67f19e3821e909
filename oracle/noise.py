"""FP64 oracle of the likelihood tail: A/E/T noise PSDs, the noise-weighted
inner product, overlap and mismatch (arXiv:2505.09600, Sec. II C "Noise
model" and Sec. IV, Eqs. scalar_product and normalized_overlap; App. A for the
Fourier convention).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): imported by tests/ and
bench.py's baseline legs, never by the library.

Plain numpy, written from the equations:
  S_pm(f)  = S_acc (2 pi f c)^-2 [1 + (0.4 mHz/f)^2] [1 + (f/8 mHz)^4]
  S_op(f)  = S_oms (2 pi f / c)^2 [1 + (2 mHz/f)^4]
  S_gal(f) = 2 x^2 sin^2 x  A f^(-7/3) exp[-(f/f1)^alpha] {1 + tanh[(f_knee - f)/f2]},
             x = 2 pi f L / c,  log10 f1 = a1 log10 T_obs + b1,
             log10 f_knee = ak log10 T_obs + bk  (T_obs in years)
  S^{A,E}  = 8 Lam sin^2 x {2 [3 + 2 cos x + cos 2x] S_pm + [2 + cos x] S_op} + (3/2) Lam S_gal
  S^T      = 16 Lam sin^2 x {[1 - cos x] S_op + 8 sin^4(x/2) S_pm} + Lam S_gal
  Lam = 4 sin^2(2x) for TDI 2.0, 1 for TDI 1.5.
The continuous transform x~(f) = int dt e^{-2 pi i f t} x(t) is taken as
dt times the discrete transform on the rfft bins f_k = k / (N dt) (the phase
of the grid start cancels in x~* y~), and
  <x|y> = 4 Re sum_{f_min <= f_k <= f_max} x~_k^* y~_k / S(f_k) df,  df = 1/(N dt),
the rectangle rule for Eq. scalar_product on those bins.
"""
from __future__ import annotations

import numpy as np

C_LIGHT = 299792458.0
S_ACC = (2.4e-15) ** 2          # m^2 s^-4 Hz^-1
S_OMS = (7.9e-12) ** 2          # m^2 Hz^-1
GAL_A = 1.28265531e-44
GAL_ALPHA = 1.62966700
GAL_F2 = 4.81078093e-4
GAL_A1, GAL_B1 = -0.223499956, -2.70408439
GAL_AK, GAL_BK = -0.360976122, -2.37822436


def s_pm(f):
    """Proof-mass noise (Sec. II C)."""
    f = np.asarray(f, dtype=np.float64)
    return S_ACC * (2.0 * np.pi * f * C_LIGHT) ** -2 * (1.0 + (4e-4 / f) ** 2) * (1.0 + (f / 8e-3) ** 4)


def s_op(f):
    """Optical-path noise (Sec. II C)."""
    f = np.asarray(f, dtype=np.float64)
    return S_OMS * (2.0 * np.pi * f / C_LIGHT) ** 2 * (1.0 + (2e-3 / f) ** 4)


def gal_knees(t_obs_years):
    """(f1, f_knee) of the galactic foreground for an observation of t_obs years."""
    lt = np.log10(t_obs_years)
    return 10.0 ** (GAL_A1 * lt + GAL_B1), 10.0 ** (GAL_AK * lt + GAL_BK)


def s_gal(f, L_m=2.5e9, t_obs_years=1.0):
    """Galactic confusion foreground (Eq. sgal)."""
    f = np.asarray(f, dtype=np.float64)
    x = 2.0 * np.pi * f * L_m / C_LIGHT
    f1, fk = gal_knees(t_obs_years)
    return (2.0 * x ** 2 * np.sin(x) ** 2 * GAL_A * f ** (-7.0 / 3.0) * np.exp(-(f / f1) ** GAL_ALPHA)
            * (1.0 + np.tanh((fk - f) / GAL_F2)))


def psd_aet(f, tdi_gen=20, L_m=2.5e9, t_obs_years=1.0, galaxy=True):
    """(S^{A,E}, S^T) at frequencies f (Eqs. SnAE, SnT)."""
    f = np.asarray(f, dtype=np.float64)
    x = 2.0 * np.pi * f * L_m / C_LIGHT
    lam = 4.0 * np.sin(2.0 * x) ** 2 if tdi_gen == 20 else np.ones_like(f)
    pm, op = s_pm(f), s_op(f)
    gal = s_gal(f, L_m, t_obs_years) if galaxy else np.zeros_like(f)
    s2 = np.sin(x) ** 2
    sae = 8.0 * lam * s2 * (2.0 * (3.0 + 2.0 * np.cos(x) + np.cos(2.0 * x)) * pm + (2.0 + np.cos(x)) * op) \
        + 1.5 * lam * gal
    st = 16.0 * lam * s2 * ((1.0 - np.cos(x)) * op + 8.0 * np.sin(0.5 * x) ** 4 * pm) + lam * gal
    return sae, st


def fft_length(n):
    """Smallest 2^a 3^b 5^c 7^d >= n (the transform length of a zero-padded row)."""
    best = None
    p2 = 1
    while p2 < 2 * n:
        p3 = p2
        while p3 < 2 * n:
            p5 = p3
            while p5 < 2 * n:
                p7 = p5
                while p7 < 2 * n:
                    if p7 >= n and (best is None or p7 < best):
                        best = p7
                    p7 *= 7
                p5 *= 5
            p3 *= 3
        p2 *= 2
    return best


def spectrum(x, dt, nfft=None):
    """x~(f_k) = dt * sum_n x_n e^{-2 pi i k n / M} on the rfft bins of the row
    zero-padded to M = nfft samples (M = N without padding)."""
    return dt * np.fft.rfft(np.asarray(x, dtype=np.float64), n=nfft, axis=-1)


def inner_aet(x, y, dt, f_min, f_max, tdi_gen=20, L_m=2.5e9, t_obs_years=1.0, galaxy=True, nfft=None):
    """<x|y>, <x|x>, <y|y> for each of A, E, T (rows of x, y: [3][N]), Eq.
    scalar_product with the A/E PSD for A and E and the T PSD for T, on the
    bins f_k = k / (M dt) of the rows zero-padded to M = nfft >= N samples
    (zero padding samples the same continuous transform more finely)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = x.shape[-1] if nfft is None else int(nfft)
    f = np.arange(n // 2 + 1) / (n * dt)
    df = 1.0 / (n * dt)
    sel = (f >= f_min) & (f <= f_max) & (f > 0)
    sae, st = psd_aet(np.where(sel, f, 1.0), tdi_gen, L_m, t_obs_years, galaxy)
    X, Y = spectrum(x, dt, n), spectrum(y, dt, n)
    out = np.zeros((3, 3))
    for c in range(3):
        s = sae if c < 2 else st
        w = np.where(sel, 4.0 * df / s, 0.0)
        out[c, 0] = np.sum(w * np.real(np.conj(X[c]) * Y[c]))
        out[c, 1] = np.sum(w * np.abs(X[c]) ** 2)
        out[c, 2] = np.sum(w * np.abs(Y[c]) ** 2)
    return out


def overlap(ip):
    """O = <x|y> / sqrt(<x|x><y|y>) per channel (Eq. normalized_overlap), from inner_aet's output."""
    ip = np.asarray(ip, dtype=np.float64)
    return ip[:, 0] / np.sqrt(ip[:, 1] * ip[:, 2])


def mismatch(ip):
    """M = 1 - |O| per channel."""
    return 1.0 - np.abs(overlap(ip))
