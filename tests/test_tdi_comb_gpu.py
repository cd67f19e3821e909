"""Mixed-precision TDI (frozen delays) from given link series against the FP64
oracle on the same FP32 link values, element by element.

On a common grid the kernel combines the terms of each link into one filter
whose weights are linearised in the block offset; blocks outside the
linearisation bounds (fast-changing arms, filters longer than 96 taps at small
dt) and other grids take per-sample weights.  The cases below reach each of
these branches:
  * kepler2_flex, static, analytic orbits at dt = 5 s: combined filters;
  * linear arms with |dT/dt| up to 3e-7: drift above the bound, per-sample path;
  * dt = 0.5 s: filters longer than 96 taps, per-sample path;
  * an output grid at twice the link step: the per-tile kernel.
The error scale is the link amplitude: the TDI sums cancel strongly at low
frequency, so max |X| is not the scale of the rounding (FP32 weights and
delays give a few 1e-7 of max |y| per term).
"""
import numpy as np
import pytest

import synth
from gpu_util import empty, host_inputs, orbit_pair, sky_of, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_OF_Y = 1e-5   # max |X - X_oracle| / max |y| over the six links


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_09600_gb300 import build
    build.build()
    import paper_2505_09600_gb300 as L
    L.load()
    return L


def _links(oracle_mod, oo, s):
    hp, hc = host_inputs(s, 1)
    y = oracle_mod.links_full(oo, sky_of(s), s.grid, hp, hc, s.grid)
    return np.asarray(y, dtype=np.float32).astype(np.float64)


def _run(L, oracle_mod, orbit, s, gen, out_grid=None):
    oo, lo = orbit_pair(orbit)
    y = _links(oracle_mod, oo, s)
    og = out_grid or s.grid
    want = np.asarray(oracle_mod.tdi_from_y(oo, s.grid, y, gen, 0, og))
    out = empty((3, og[2]), 1)
    L.lisa_tdi(lo, s.grid, to_dev(y, 1), L.MIXED, gen, L.FROZEN, 0, og, out)
    got = out.cpu().numpy().astype(np.float64)
    err = np.abs(got - want).max() / np.abs(y).max()
    assert np.isfinite(got).all()
    assert err <= TOL_OF_Y, (orbit, gen, err)
    return err


@pytest.mark.parametrize("orbit", ["kepler2_flex", "static", "analytic", "linear"])
@pytest.mark.parametrize("gen", [15, 20])
def test_tdi_mixed_orbits(L, oracle_mod, orbit, gen):
    s = synth.cfg2_small(n=6000)
    _run(L, oracle_mod, orbit, s, gen)


@pytest.mark.parametrize("gen", [15, 20])
def test_tdi_mixed_small_dt(L, oracle_mod, gen):
    s = synth.cfg2_source(n=12000, dt=0.5, t0=2.0e7, post_merger=2000.0)
    _run(L, oracle_mod, "kepler2_flex", s, gen)


def test_tdi_mixed_other_grid(L, oracle_mod):
    s = synth.cfg2_small(n=6000)
    t0, dt, n = s.grid
    og = (t0 + 40.0, 2 * dt, n // 2 - 40)
    _run(L, oracle_mod, "kepler2_flex", s, 20, out_grid=og)


def test_tdi_mixed_ragged_range(L, oracle_mod):
    # a length that leaves a partial group and a lone last tile
    s = synth.cfg2_small(n=256 * 8 * 3 + 256 + 77)
    _run(L, oracle_mod, "kepler2_flex", s, 20)
