"""Evidence for the precision split of the mixed form (CPU only)."""
import numpy as np

import synth


def test_fp32_absolute_time_is_not_enough(oracle_mod):
    """Absolute times near 2e7 s rounded to FP32 (ulp 2 s) move the retarded
    times by up to a second, which changes the links by far more than the
    mixed-precision tolerance (~1e-5); the kernels therefore keep tile-centre
    times and delays in FP64 and only the in-tile offsets in FP32."""
    s = synth.cfg2_small(n=20000)
    oo = oracle_mod.Orbit(kind=oracle_mod.KEPLER2, kepler_tilt=1.01)
    sky = (s.beta, s.lam, s.psi)
    idx = np.arange(15000, 19000, 97)
    exact = oracle_mod.links_full(oo, sky, s.grid, s.hp, s.hc, s.grid, idx)
    t32 = np.float32(s.t0 + idx * s.dt).astype(np.float64)
    shifted = np.stack([oracle_mod.links_full(oo, sky, s.grid, s.hp, s.hc, (t32[k], s.dt, 1))[:, 0]
                        for k in range(idx.size)], axis=1)
    err = np.abs(shifted - exact).max() / np.abs(exact).max()
    assert err > 1e-3, err


def test_split_accumulation_bounds_of_the_outer_taps():
    """The double-float LFA sums its 24 outer taps (nodes -15..-4 and 5..16 of
    the 32-point stencil) exactly by splitting each product against
    sigma = 2^(e-2), where 2^e <= M < 2^(e+1) bounds the window's nodes.  That
    is exact when every outer |w_k| M stays below sigma / 2 and their sum below
    sigma, i.e. max |w_k| < 1/16 and sum |w_k| < 1/8 for every fraction in
    [0, 1].  The Lagrange basis, evaluated here in exact rational arithmetic
    at 257 fractions (the extremes sit at 0.5 and near the ends), gives
    max |w_k| = 0.0197 and sum |w_k| = 0.0656: margins of 3.2 and 1.9."""
    from fractions import Fraction
    nodes = list(range(-15, 17))
    outer = [k for k in nodes if k <= -4 or k >= 5]
    worst_max, worst_sum = Fraction(0), Fraction(0)
    for i in range(257):
        e = Fraction(i, 256)
        ws = []
        for k in outer:
            w = Fraction(1)
            for m in nodes:
                if m != k:
                    w *= (e - m) / Fraction(k - m)
            ws.append(abs(w))
        worst_max = max(worst_max, max(ws))
        worst_sum = max(worst_sum, sum(ws))
    assert worst_max < Fraction(1, 16) / 3, float(worst_max)
    assert worst_sum < Fraction(1, 8) / Fraction(3, 2), float(worst_sum)
