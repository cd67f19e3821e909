"""The oracle's sampled paths against its array forms.

The full-size and parameter-estimation GPU tests, and the benchmark's error
fields, check outputs at sampled indices with ``tdi_full_direct`` and
``tdi_lfa_direct``.  These recompute every link or z value that a sampled
output needs, one output at a time.  They need no link or z series in memory.
The array forms (``response_full`` = links on the grid then TDI;
``response_lfa`` = z series on the grid then the channel stencils) are the
ones pinned against the paper in test_oracle_pins.py and
test_oracle_bruteforce.py.

Both forms evaluate the same definitions: the links of Eq. yslr, the TDI sums
of Eqs. X1.5 and X2.0, the LFA links of Eq. yslr_strain_derivatives, the
channels of Eqs. X15_nonequal and X20_nonequal, and zero padding outside
every grid.  So the sampled outputs must equal the array outputs exactly.
They are checked on a grid of 1,800 samples at the first and last samples,
across a hybrid window, and at spread interior points.
"""
import numpy as np
import pytest

import synth

N = 1800


def _case():
    src = synth.cfg2_small(n=N)
    return src, (src.beta, src.lam, src.psi)


def _indices(n):
    rng = np.random.default_rng(17)
    ends = np.r_[np.arange(0, 40), np.arange(n - 40, n)]
    window = np.arange(int(0.55 * n), int(0.55 * n) + 60)
    spread = rng.choice(np.arange(40, n - 40), 60, replace=False)
    return np.unique(np.concatenate([ends, window, spread]))


@pytest.mark.parametrize("gen,mode", [(15, 0), (20, 0), (20, 1)])
def test_tdi_full_direct_equals_array_form(oracle_mod, gen, mode):
    src, sky = _case()
    o = oracle_mod.Orbit(kind=1, delay=0, kepler_tilt=1.01)
    g = src.grid
    want = oracle_mod.response_full(o, sky, g, src.hp, src.hc, gen, mode, "xyz", g)
    idx = _indices(src.n)
    got = oracle_mod.tdi_full_direct(o, sky, g, src.hp, src.hc, g, gen, mode, g, idx)
    assert np.abs(want[:, idx]).max() > 0
    assert np.array_equal(got, want[:, idx]), np.abs(got - want[:, idx]).max()


@pytest.mark.parametrize("gen", [15, 20])
@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_tdi_lfa_direct_equals_array_form(oracle_mod, gen, kind):
    src, sky = _case()
    o = oracle_mod.Orbit(kind=1, delay=0, kepler_tilt=1.01)
    g = src.grid
    want = oracle_mod.response_lfa(o, sky, g, src.hp, src.hc, gen, kind, "xyz", g)
    idx = _indices(src.n)
    got = oracle_mod.tdi_lfa_direct(o, sky, g, src.hp, src.hc, gen, kind, g, idx)
    assert np.abs(want[:, idx]).max() > 0
    assert np.array_equal(got, want[:, idx]), np.abs(got - want[:, idx]).max()


def test_sampled_hybrid_equals_array_hybrid(oracle_mod):
    # the benchmark's checker: sampled LFA and full parts blended at sampled indices
    src, sky = _case()
    o = oracle_mod.Orbit(kind=1, delay=0, kepler_tilt=1.01)
    g = src.grid
    tH = src.t0 + 0.55 * src.n * src.dt
    Tw, sig = 200 * src.dt, 5 * src.dt
    want = oracle_mod.response_hybrid(o, sky, g, src.hp, src.hc, 20, 0, "aet", tH, Tw, sig)
    idx = _indices(src.n)
    lf = oracle_mod.tdi_lfa_direct(o, sky, g, src.hp, src.hc, 20, 0, g, idx)
    fu = oracle_mod.tdi_full_direct(o, sky, g, src.hp, src.hc, g, 20, 0, g, idx)
    got = oracle_mod.aet(oracle_mod.hybrid_blend(g, tH, Tw, sig, lf, fu, idx))
    assert np.array_equal(got, want[:, idx]), np.abs(got - want[:, idx]).max()
