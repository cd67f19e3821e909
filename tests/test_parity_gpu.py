"""GPU (liblisa, sm_103a) against the FP64 CPU oracle, element by element.

All-FP64 forms must agree within F64_TOL (5e-12) of each channel's largest
value (A, E, T: of the largest channel's).  Mixed-precision tolerances are in
tolerances.py and test_parity_mixed_gpu.py.
"""
import math

import numpy as np
import pytest

import synth
from gpu_util import F64_TOL, check_aet, empty, host_inputs, orbit_pair, rel_err, sky_of, to_dev
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


@pytest.fixture(scope="module")
def cfg1():
    return synth.cfg1_source()


@pytest.fixture(scope="module")
def cfg2s():
    return synth.cfg2_small(n=20000)


@pytest.mark.parametrize("orb", ["kepler1", "kepler2_flex", "analytic", "equal", "linear", "static"])
def test_orbits(L, oracle_mod, orb):
    oo, lo = orbit_pair(orb)
    g = (2.0e7 + 123.0, 10.0, 3000)
    R, T, nh = (torch.empty(s, device="cuda", dtype=torch.float64) for s in ((3, 3, 3000), (6, 3000), (6, 3, 3000)))
    L.lisa_orbits(lo, g, R, T, nh)
    torch.cuda.synchronize()
    Ro, To, no = oracle_mod.orbits(oo, g)
    assert np.abs(R.cpu().numpy() - Ro).max() < 2e-4          # metres (R ~ 1.5e11 m)
    # The oracle evaluates R_s at the absolute time t - T, whose FP64 rounding
    # (ulp(2e7 s) = 3.7e-9 s) moves the sender by |V| * 3.7e-9 s ~ 1e-4 m, i.e.
    # ~4e-13 s of light time; the kernels expand R_s(t - T) about t instead.
    assert np.abs(T.cpu().numpy() - To).max() < 1.5e-12       # seconds
    assert np.abs(nh.cpu().numpy() - no).max() < 2e-13


@pytest.mark.parametrize("orb", ["kepler1", "kepler2_flex"])
def test_links_full_f64(L, oracle_mod, cfg1, orb):
    oo, lo = orbit_pair(orb)
    s = cfg1
    want = oracle_mod.links_full(oo, sky_of(s), s.grid, s.hp, s.hc, s.grid)
    y = empty((6, s.n), 0)
    L.lisa_links_full(lo, sky_of(s), s.grid, to_dev(s.hp, 0), to_dev(s.hc, 0), L.F64, s.grid, y)
    err = rel_err(y.cpu().numpy(), want)
    assert err.max() <= F64_TOL, err


@pytest.mark.parametrize("gen", [15, 20])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("channels", [0, 1])
def test_tdi_f64_from_links(L, oracle_mod, gen, mode, channels):
    rng = np.random.default_rng(100 + gen + mode)
    g = (3.0e7, 5.0, 1500)
    oo, lo = orbit_pair("kepler2_flex")
    tt = np.arange(1500) * 5.0
    y = np.stack([np.sin(2 * math.pi * f * tt + p) for f, p in zip(rng.uniform(1e-3, 2e-2, 6), rng.uniform(0, 6, 6))])
    want = oracle_mod.tdi_from_y(oo, g, y, gen, mode, g)
    if channels == 1:
        want = oracle_mod.aet(want)
    out = empty((3, 1500), 0)
    L.lisa_tdi(lo, g, to_dev(y, 0), L.F64, gen, mode, channels, g, out)
    if channels == 1:
        check_aet(out.cpu().numpy(), want, F64_TOL, T_OWN_TOL["f64"])
    else:
        err = rel_err(out.cpu().numpy(), want)
        assert err.max() <= F64_TOL, err


def test_response_full_f64_config1(L, oracle_mod, cfg1):
    """Config 1: chirp Mc=1e5, 8640 samples at 10 s, first-order Kepler, TDI 1.5 XYZ."""
    oo, lo = orbit_pair("kepler1")
    s = cfg1
    want = oracle_mod.response_full(oo, sky_of(s), s.grid, s.hp, s.hc, 15)
    out = empty((3, s.n), 0)
    L.lisa_response_full(lo, sky_of(s), s.grid, to_dev(s.hp, 0), to_dev(s.hc, 0), L.F64, 15, L.XYZ, s.grid, out)
    err = rel_err(out.cpu().numpy(), want)
    assert err.max() <= F64_TOL, err


@pytest.mark.parametrize("gen", [15, 20])
@pytest.mark.parametrize("kind", [0, 1, 2, 3])   # central unequal / equal, backward, forward
def test_lfa_f64(L, oracle_mod, cfg2s, gen, kind):
    oo, lo = orbit_pair("kepler2_flex")
    s = cfg2s
    z_want = oracle_mod.z_lfa(oo, sky_of(s), s.grid, s.hp, s.hc, gen, kind, s.grid)
    x_want = oracle_mod.tdi_lfa_from_z(oo, s.grid, z_want, gen, kind)
    hp, hc = to_dev(s.hp, 0), to_dev(s.hc, 0)
    z = empty((6, s.n), 0)
    L.lisa_links_lfa(lo, sky_of(s), s.grid, hp, hc, L.F64, gen, kind, s.grid, z)
    assert rel_err(z.cpu().numpy(), z_want).max() <= F64_TOL
    x = empty((3, s.n), 0)
    L.lisa_response_lfa(lo, sky_of(s), s.grid, hp, hc, L.F64, gen, kind, L.XYZ, s.grid, x)
    assert rel_err(x.cpu().numpy(), x_want).max() <= F64_TOL
    # channels from caller-held z
    x2 = empty((3, s.n), 0)
    L.lisa_tdi_lfa(lo, s.grid, z, L.F64, gen, kind, L.AET, x2)
    check_aet(x2.cpu().numpy(), oracle_mod.aet(x_want), F64_TOL, T_OWN_TOL["f64"], equal_arms=kind == 1)
    # the same channels from the fused call
    x3 = empty((3, s.n), 0)
    L.lisa_response_lfa(lo, sky_of(s), s.grid, hp, hc, L.F64, gen, kind, L.AET, s.grid, x3)
    check_aet(x3.cpu().numpy(), oracle_mod.aet(x_want), F64_TOL, T_OWN_TOL["f64"], equal_arms=kind == 1)


@pytest.mark.parametrize("where", ["middle", "before_start", "after_end", "near_end"])
def test_hybrid_f64(L, oracle_mod, cfg2s, where):
    oo, lo = orbit_pair("kepler2_flex")
    s = cfg2s
    t_end = s.t0 + s.n * s.dt
    tH = {"middle": oracle_mod.t_hyb(1e-3, s.mc_s, s.tc), "before_start": s.t0 - 1e5,
          "after_end": t_end + 1e5, "near_end": t_end - 300 * s.dt}[where]
    Tw, sig = 800 * s.dt, 20 * s.dt
    want = oracle_mod.response_hybrid(oo, sky_of(s), s.grid, s.hp, s.hc, 20, 0, "aet", tH, Tw, sig)
    out = empty((3, s.n), 0)
    L.lisa_response_hybrid(lo, sky_of(s), s.grid, to_dev(s.hp, 0), to_dev(s.hc, 0), L.F64, 20, 0, L.AET,
                           tH, Tw, sig, s.grid, out)
    check_aet(out.cpu().numpy(), want, F64_TOL, T_OWN_TOL["f64"])


@pytest.mark.parametrize("n", [1, 7, 255, 257, 513, 1031])
def test_ragged_and_tiny_sizes(L, oracle_mod, n):
    oo, lo = orbit_pair("kepler1")
    s = synth.cfg1_source()
    hp, hc = s.hp[-n:], s.hc[-n:]
    g = (s.t0 + (s.n - n) * s.dt, s.dt, n)
    want = oracle_mod.response_full(oo, sky_of(s), g, hp, hc, 20)
    out = empty((3, n), 0)
    L.lisa_response_full(lo, sky_of(s), g, to_dev(hp, 0), to_dev(hc, 0), L.F64, 20, L.XYZ, g, out)
    assert np.isfinite(out.cpu().numpy()).all()
    assert rel_err(out.cpu().numpy(), want).max() <= F64_TOL
    wl = oracle_mod.response_lfa(oo, sky_of(s), g, hp, hc, 15)
    xl = empty((3, n), 0)
    L.lisa_response_lfa(lo, sky_of(s), g, to_dev(hp, 0), to_dev(hc, 0), L.F64, 15, 0, L.XYZ, g, xl)
    assert rel_err(xl.cpu().numpy(), wl).max() <= F64_TOL


@pytest.mark.parametrize("shift,ratio", [(37.5, 1.0), (-1234.0, 1.0), (5.0, 2.0), (0.0, 0.5)])
def test_input_grid_differs_from_output(L, oracle_mod, shift, ratio):
    """h on one grid, links/channels on another (offset start, other step)."""
    oo, lo = orbit_pair("kepler2_flex")
    s = synth.cfg2_small(n=6000)
    og = (s.t0 + shift + 600.0, s.dt * ratio, int(4000 / ratio))
    y_want = oracle_mod.links_full(oo, sky_of(s), s.grid, s.hp, s.hc, og)
    y = empty((6, og[2]), 0)
    L.lisa_links_full(lo, sky_of(s), s.grid, to_dev(s.hp, 0), to_dev(s.hc, 0), L.F64, og, y)
    assert rel_err(y.cpu().numpy(), y_want).max() <= F64_TOL
    x_want = oracle_mod.response_lfa(oo, sky_of(s), s.grid, s.hp, s.hc, 20, 0, "xyz", og)
    x = empty((3, og[2]), 0)
    L.lisa_response_lfa(lo, sky_of(s), s.grid, to_dev(s.hp, 0), to_dev(s.hc, 0), L.F64, 20, 0, L.XYZ, og, x)
    assert rel_err(x.cpu().numpy(), x_want).max() <= F64_TOL


def test_zero_input_gives_zero(L):
    lo = L.Orbit()
    g = (2e7, 5.0, 3000)
    z = torch.zeros(3000, device="cuda", dtype=torch.float64)
    out = empty((3, 3000), 0)
    L.lisa_response_hybrid(lo, (0.3, 1.0, 0.2), g, z, z, L.F64, 20, 0, L.XYZ, 2e7 + 7000.0, 0.0, 0.0, g, out)
    assert torch.count_nonzero(out).item() == 0


def test_stream_argument_and_async(L, oracle_mod, cfg1):
    oo, lo = orbit_pair("kepler1")
    s = cfg1
    st = torch.cuda.Stream()
    hp, hc = to_dev(s.hp, 0), to_dev(s.hc, 0)
    out = empty((3, s.n), 0)
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        L.lisa_response_full(lo, sky_of(s), s.grid, hp, hc, L.F64, 15, L.XYZ, s.grid, out, stream=st.cuda_stream)
    st.synchronize()
    want = oracle_mod.response_full(oo, sky_of(s), s.grid, s.hp, s.hc, 15)
    assert rel_err(out.cpu().numpy(), want).max() <= F64_TOL


def test_errors_raise(L):
    lo = L.Orbit(L_m=-5.0)
    g = (2e7, 5.0, 10)
    z = torch.zeros(10, device="cuda", dtype=torch.float64)
    with pytest.raises(L.LisaError) as e:
        L.lisa_links_full(lo, (0.1, 0.2, 0.3), g, z, z, L.F64, g, torch.zeros(60, device="cuda", dtype=torch.float64))
    assert e.value.status == -1
    with pytest.raises(TypeError):
        L.lisa_links_full(L.Orbit(), (0.1, 0.2, 0.3), g, z.float(), z.float(), L.F64, g,
                          torch.zeros(60, device="cuda", dtype=torch.float64))
