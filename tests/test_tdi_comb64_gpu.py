"""FP64 frozen TDI on per-link combined filters (tdi_comb64.cu) against the
oracle: long ranges (512-sample blocks, one slice of taps per thread), coarse
grids (shorter blocks), short ranges (small blocks, taps split over slices)
and the per-sample path that blocks outside the expansion's bounds take."""
import os

import numpy as np
import pytest

import synth
from gpu_util import F64_TOL, empty, host_inputs, orbit_pair, rel_err, sky_of, to_dev
from tolerances import T_OWN_TOL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_09600_gb300 import build
    build.build()
    import paper_2505_09600_gb300 as L
    L.load()
    return L


def _full_sampled(L, oracle_mod, s, gen, channels, idx, exact=False):
    oo, lo = orbit_pair("kepler2_flex")
    hp, hc = host_inputs(s, 0)
    out = empty((3, s.n), 0)
    if exact:
        os.environ["LISA_TDI64_EXACT"] = "1"
    try:
        L.lisa_response_full(lo, sky_of(s), s.grid, to_dev(hp, 0), to_dev(hc, 0), L.F64, gen, channels, s.grid, out)
        torch.cuda.synchronize()
    finally:
        os.environ.pop("LISA_TDI64_EXACT", None)
    got = out.cpu().numpy()
    want = oracle_mod.tdi_full_direct(oo, sky_of(s), s.grid, hp, hc, s.grid, gen, 0, s.grid, idx)
    if channels == L.AET:
        want = oracle_mod.aet(want)
    return got, want


@pytest.mark.parametrize("gen,channels", [(20, "aet"), (15, "xyz")])
def test_full_f64_long_range_sampled(L, oracle_mod, gen, channels):
    """One million samples at 5 s: 512-sample blocks, every tap slice in one
    thread; sampled outputs across blocks, block edges and the grid end."""
    ch = L.AET if channels == "aet" else L.XYZ
    s = synth.cfg2_source(n=1000000, dt=5.0)
    rng = np.random.default_rng(64)
    edges = np.arange(512, s.n, 512 * 97)
    idx = np.unique(np.concatenate([rng.integers(0, s.n, 300), edges - 1, edges, edges + 255,
                                    np.arange(s.n - 1500, s.n, 3), np.arange(0, 40)]))
    got, want = _full_sampled(L, oracle_mod, s, gen, ch, idx)
    scale = np.abs(got).max(axis=1)
    if channels == "aet":
        err = np.abs(got[:, idx] - want).max(axis=1) / scale.max()
    else:
        err = np.abs(got[:, idx] - want).max(axis=1) / scale
    assert np.all(err <= F64_TOL), err


@pytest.mark.parametrize("dt", [20.0, 60.0])
def test_full_f64_coarse_grid(L, oracle_mod, dt):
    """Coarse grids shorten the blocks (the delay's curvature term grows as
    dt h^2): TDI 2.0 A/E/T over 200,000 samples, every output checked
    against the oracle's array form where it is cheap (the grid's last 6,000
    samples) and sampled elsewhere."""
    s = synth.cfg2_source(n=200000, dt=dt)
    rng = np.random.default_rng(int(dt))
    idx = np.unique(np.concatenate([rng.integers(0, s.n, 400), np.arange(s.n - 6000, s.n)]))
    got, want = _full_sampled(L, oracle_mod, s, 20, L.AET, idx)
    err = np.abs(got[:, idx] - want).max(axis=1) / np.abs(got).max()
    assert np.all(err <= F64_TOL), err


@pytest.mark.parametrize("n", [33, 700, 5000, 40000])
def test_full_f64_short_ranges(L, oracle_mod, n):
    """Short ranges: blocks of 32..512 samples whose taps are split over up to
    16 slices, a ragged last block; element by element against the oracle."""
    oo, lo = orbit_pair("kepler2_flex")
    s = synth.cfg2_small(n=n)
    want = oracle_mod.response_full(oo, sky_of(s), s.grid, s.hp, s.hc, 20, channels="aet")
    out = empty((3, s.n), 0)
    L.lisa_response_full(lo, sky_of(s), s.grid, to_dev(s.hp, 0), to_dev(s.hc, 0), L.F64, 20, L.AET, s.grid, out)
    got = out.cpu().numpy()
    err = rel_err(got, want, signal=True)
    assert err.max() <= F64_TOL, err
    own = rel_err(got, want)
    assert own[:2].max() <= F64_TOL and own[2] <= T_OWN_TOL["f64"], own


def test_full_f64_per_sample_path(L, oracle_mod):
    """Every block through the per-sample FP64 path (exact delay and own
    weights per term), as blocks outside the expansion's bounds take it: the
    same outputs within the FP64 tolerance, and equal to the filter path to
    well within it."""
    s = synth.cfg2_source(n=60000, dt=5.0)
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([rng.integers(0, s.n, 200), np.arange(s.n - 700, s.n)]))
    got_x, want = _full_sampled(L, oracle_mod, s, 20, L.AET, idx, exact=True)
    got_c, _ = _full_sampled(L, oracle_mod, s, 20, L.AET, idx, exact=False)
    scale = np.abs(got_c).max()
    assert np.abs(got_x[:, idx] - want).max() / scale <= F64_TOL
    assert np.abs(got_c - got_x).max() / scale <= F64_TOL
