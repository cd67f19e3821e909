"""Mixed-precision forms (FP32 arithmetic, FP64 tile-centre times) against the
FP64 oracle, element by element, at the frozen per-channel tolerances of
tolerances.py.  The oracle is fed exactly the FP32 values the kernels read."""
import math

import numpy as np
import pytest

import synth
from gpu_util import check_aet, empty, host_inputs, orbit_pair, rel_err, sky_of, to_dev
from tolerances import MIXED_TOL, T_OWN_TOL

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


@pytest.fixture(scope="module")
def case():
    s = synth.cfg2_small(n=20000)
    hp, hc = host_inputs(s, 1)
    return s, hp, hc


def _check(got, want, tol, aet=False, form=None, equal_arms=False):
    if aet:
        # every channel on the largest channel's scale and on its own (T at its
        # own frozen tolerance)
        return check_aet(got, want, tol, T_OWN_TOL["mixed"][form], equal_arms=equal_arms)[1]
    err = rel_err(got, want)
    assert np.all(err <= np.asarray(tol)), (err, tol)
    return err


def test_links_mixed(L, oracle_mod, case):
    s, hp, hc = case
    oo, lo = orbit_pair("kepler2_flex")
    want = oracle_mod.links_full(oo, sky_of(s), s.grid, hp, hc, s.grid)
    y = empty((6, s.n), 1)
    L.lisa_links_full(lo, sky_of(s), s.grid, to_dev(hp, 1), to_dev(hc, 1), L.MIXED, s.grid, y)
    _check(y.cpu().numpy(), want, MIXED_TOL["links"])


@pytest.mark.parametrize("gen", [15, 20])
@pytest.mark.parametrize("channels", [0, 1])
def test_full_mixed(L, oracle_mod, case, gen, channels):
    s, hp, hc = case
    oo, lo = orbit_pair("kepler2_flex")
    want = oracle_mod.response_full(oo, sky_of(s), s.grid, hp, hc, gen, 0, "aet" if channels else "xyz")
    out = empty((3, s.n), 1)
    L.lisa_response_full(lo, sky_of(s), s.grid, to_dev(hp, 1), to_dev(hc, 1), L.MIXED, gen, channels, s.grid, out)
    _check(out.cpu().numpy(), want, MIXED_TOL["full%d" % gen]["aet" if channels else "xyz"], aet=channels == 1,
           form="full")


@pytest.mark.parametrize("gen", [15, 20])
@pytest.mark.parametrize("kind", [0, 1, 2, 3])   # central unequal / equal, backward, forward
def test_lfa_mixed(L, oracle_mod, case, gen, kind):
    s, hp, hc = case
    oo, lo = orbit_pair("kepler2_flex")
    z_want = oracle_mod.z_lfa(oo, sky_of(s), s.grid, hp, hc, gen, kind, s.grid)
    x_want = oracle_mod.tdi_lfa_from_z(oo, s.grid, z_want, gen, kind)
    hpd, hcd = to_dev(hp, 1), to_dev(hc, 1)
    z = empty((6, s.n), 1)
    L.lisa_links_lfa(lo, sky_of(s), s.grid, hpd, hcd, L.MIXED, gen, kind, s.grid, z)
    _check(z.cpu().numpy(), z_want, MIXED_TOL["z"])
    for channels in (0, 1):
        out = empty((3, s.n), 1)
        L.lisa_response_lfa(lo, sky_of(s), s.grid, hpd, hcd, L.MIXED, gen, kind, channels, s.grid, out)
        want = oracle_mod.aet(x_want) if channels else x_want
        _check(out.cpu().numpy(), want, MIXED_TOL["lfa%d" % gen]["aet" if channels else "xyz"], aet=channels == 1,
               form="lfa", equal_arms=kind == 1)


@pytest.mark.parametrize("gen", [15, 20])
@pytest.mark.parametrize("channels", [0, 1])
def test_hybrid_mixed(L, oracle_mod, case, gen, channels):
    s, hp, hc = case
    oo, lo = orbit_pair("kepler2_flex")
    tH = oracle_mod.t_hyb(1e-3, s.mc_s, s.tc)
    Tw, sig = 800 * s.dt, 20 * s.dt
    want = oracle_mod.response_hybrid(oo, sky_of(s), s.grid, hp, hc, gen, 0, "aet" if channels else "xyz",
                                      tH, Tw, sig)
    out = empty((3, s.n), 1)
    L.lisa_response_hybrid(lo, sky_of(s), s.grid, to_dev(hp, 1), to_dev(hc, 1), L.MIXED, gen, 0, channels,
                           tH, Tw, sig, s.grid, out)
    _check(out.cpu().numpy(), want, MIXED_TOL["hybrid%d" % gen]["aet" if channels else "xyz"], aet=channels == 1,
           form="hybrid")


@pytest.mark.parametrize("shift,ratio", [(0.0, 1), (2.5, 1), (0.0, 2), (1.7, 3)])
def test_mixed_input_grid_differs_from_output(L, oracle_mod, shift, ratio):
    """Mixed forms with h on one grid and the outputs on another (offset start,
    other step): the grouped links and the LFA take the non-unit-ratio path
    of the sample position (FP64 split of the offset times the ratio)."""
    oo, lo = orbit_pair("kepler2_flex")
    s = synth.cfg2_small(n=12000)
    hp, hc = host_inputs(s, 1)
    # the window holds the merger (h peaks at sample ~9,600): errors are scaled by each
    # link's largest value, as in the other parity tests
    og = (s.t0 + shift + 600.0, s.dt * ratio, int(10400 / ratio))
    y_want = oracle_mod.links_full(oo, sky_of(s), s.grid, hp, hc, og)
    y = empty((6, og[2]), 1)
    L.lisa_links_full(lo, sky_of(s), s.grid, to_dev(hp, 1), to_dev(hc, 1), L.MIXED, og, y)
    _check(y.cpu().numpy(), y_want, MIXED_TOL["links"])
    x_want = oracle_mod.response_lfa(oo, sky_of(s), s.grid, hp, hc, 20, 0, "xyz", og)
    x = empty((3, og[2]), 1)
    L.lisa_response_lfa(lo, sky_of(s), s.grid, to_dev(hp, 1), to_dev(hc, 1), L.MIXED, 20, 0, L.XYZ, og, x)
    _check(x.cpu().numpy(), x_want, MIXED_TOL["lfa20"]["xyz"])


def test_links_mixed_grouped_large(L, oracle_mod):
    """Links over a range long enough for groups of 8 tiles (one FP64 set-up per
    2,048 samples) and a last group of 3 tiles, on sampled outputs: the group
    boundaries, the last group, and points spread over the series."""
    oo, lo = orbit_pair("kepler2_flex")
    s = synth.cfg2_source(n=1000000, dt=5.0)
    hp, hc = host_inputs(s, 1)
    y = empty((6, s.n), 1)
    L.lisa_links_full(lo, sky_of(s), s.grid, to_dev(hp, 1), to_dev(hc, 1), L.MIXED, s.grid, y)
    got = y.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(21)
    g = 8 * 256
    edges = np.arange(g, s.n, g)
    idx = np.unique(np.concatenate([rng.integers(0, s.n, 1200), edges[::20] - 1, edges[::20],
                                    np.arange(s.n - 3 * 256 - 300, s.n)]))
    want = oracle_mod.links_full(oo, sky_of(s), s.grid, hp, hc, s.grid, idx=idx)
    scale = np.abs(got).max(axis=1)
    err = np.abs(got[:, idx] - want).max(axis=1) / scale
    assert np.all(err <= np.asarray(MIXED_TOL["links"])), err


def test_full_mixed_large_sampled(L, oracle_mod):
    """Full TDI 2.0 A/E/T over one million samples (grouped links, combined
    filters in large groups) against the oracle on sampled outputs."""
    oo, lo = orbit_pair("kepler2_flex")
    s = synth.cfg2_source(n=1000000, dt=5.0)
    hp, hc = host_inputs(s, 1)
    out = empty((3, s.n), 1)
    L.lisa_response_full(lo, sky_of(s), s.grid, to_dev(hp, 1), to_dev(hc, 1), L.MIXED, 20, L.AET, s.grid, out)
    got = out.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(22)
    idx = np.unique(np.concatenate([rng.integers(200, s.n, 300), np.arange(s.n - 4000, s.n, 8)]))
    want = oracle_mod.aet(oracle_mod.tdi_full_direct(oo, sky_of(s), s.grid, hp, hc, s.grid, 20, 0, s.grid, idx))
    err = np.abs(got[:, idx] - want).max(axis=1) / np.abs(got).max()
    assert np.all(err <= np.asarray(MIXED_TOL["full20"]["aet"])), err
