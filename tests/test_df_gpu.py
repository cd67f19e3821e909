"""The double-float LFA form (precision LISA_DF: FP64 inputs and outputs, the
LFA channels in pairs of FP32 numbers) against the FP64 oracle at the FP64
tolerance, element by element on the config-2-shaped source and at sampled
outputs of the full-year workload, and against the all-FP64 GPU form."""
import numpy as np
import pytest

import synth
from gpu_util import F64_TOL, check_aet, empty, orbit_pair, rel_err, sky_of, to_dev
from tolerances import T_OWN_TOL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DF = 2


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
def src():
    return synth.cfg2_small(n=20000)


@pytest.mark.parametrize("gen", [15, 20])
@pytest.mark.parametrize("kind", [0, 1, 2, 3])
def test_df_lfa(L, oracle_mod, src, gen, kind):
    s = src
    oo, lo = orbit_pair("kepler2_flex")
    hp, hc = to_dev(s.hp, 0), to_dev(s.hc, 0)
    want = oracle_mod.response_lfa(oo, sky_of(s), s.grid, s.hp, s.hc, gen, kind, "xyz")
    x = empty((3, s.n), 0)
    L.lisa_response_lfa(lo, sky_of(s), s.grid, hp, hc, DF, gen, kind, L.XYZ, s.grid, x)
    assert rel_err(x.cpu().numpy(), want).max() <= F64_TOL, rel_err(x.cpu().numpy(), want)
    a = empty((3, s.n), 0)
    L.lisa_response_lfa(lo, sky_of(s), s.grid, hp, hc, DF, gen, kind, L.AET, s.grid, a)
    check_aet(a.cpu().numpy(), oracle_mod.aet(want), F64_TOL, T_OWN_TOL["f64"], equal_arms=kind == 1)


@pytest.mark.parametrize("where", ["middle", "before_start", "after_end"])
def test_df_hybrid(L, oracle_mod, src, where):
    s = src
    oo, lo = orbit_pair("kepler2_flex")
    t_end = s.t0 + s.n * s.dt
    tH = {"middle": oracle_mod.t_hyb(1e-3, s.mc_s, s.tc), "before_start": s.t0 - 1e5, "after_end": t_end + 1e5}[where]
    Tw, sig = 800 * s.dt, 20 * s.dt
    want = oracle_mod.response_hybrid(oo, sky_of(s), s.grid, s.hp, s.hc, 20, 0, "aet", tH, Tw, sig)
    out = empty((3, s.n), 0)
    L.lisa_response_hybrid(lo, sky_of(s), s.grid, to_dev(s.hp, 0), to_dev(s.hc, 0), DF, 20, 0, L.AET, tH, Tw, sig,
                           s.grid, out)
    check_aet(out.cpu().numpy(), want, F64_TOL, T_OWN_TOL["f64"])


def test_df_other_grid_falls_back_to_f64(L, oracle_mod):
    # other grid ratios run the FP64 kernels: same results as LISA_F64, bit for bit
    oo, lo = orbit_pair("kepler2_flex")
    s = synth.cfg2_small(n=12000)
    og = (s.t0 + 1.7 + 600.0, s.dt * 3, 3466)
    outs = []
    for prec in (0, DF):
        x = empty((3, og[2]), 0)
        L.lisa_response_lfa(lo, sky_of(s), s.grid, to_dev(s.hp, 0), to_dev(s.hc, 0), prec, 20, 0, L.XYZ, og, x)
        outs.append(x.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_df_fullsize_sampled_and_local(L, oracle_mod):
    """The full-year workload as bench.py times it (its line of record): the
    global measure at the FP64 tolerance on sampled outputs, and the local
    error per frequency decade at the FP64 form's bound."""
    s = synth.cfg2_source()
    oo, lo = orbit_pair("kepler2_flex")
    tH = oracle_mod.t_hyb(1e-3, s.mc_s, s.tc)
    Tw, sig = 800 * s.dt, 20 * s.dt
    out = torch.empty((3, s.n), device="cuda", dtype=torch.float64)
    L.lisa_response_hybrid(lo, sky_of(s), s.grid, to_dev(s.hp, 0), to_dev(s.hc, 0), DF, 20, 0, L.AET, tH, Tw, sig,
                           s.grid, out)
    got = out.cpu().numpy()
    n = s.n
    rng = np.random.default_rng(5)
    iH = int((tH - s.t0) / s.dt)
    idx = np.unique(np.concatenate([rng.integers(0, n, 40), np.arange(iH - 420, iH + 420, 7), [0, 1, n - 2, n - 1],
                                    (n - 1 - np.geomspace(1, n - 1, 400).astype(np.int64))]))
    hd = (oracle_mod.hdot(s.grid, s.hp), oracle_mod.hdot(s.grid, s.hc))
    lf = oracle_mod.tdi_lfa_direct(oo, sky_of(s), s.grid, s.hp, s.hc, 20, 0, s.grid, idx, hd=hd)
    fu = np.zeros_like(lf)
    need = s.t0 + idx * s.dt >= tH - 0.5 * Tw
    fu[:, need] = oracle_mod.tdi_full_direct(oo, sky_of(s), s.grid, s.hp, s.hc, s.grid, 20, 0, s.grid, idx[need])
    want = oracle_mod.aet(oracle_mod.hybrid_blend(s.grid, tH, Tw, sig, lf, fu, idx))
    err = np.abs(got[:, idx] - want).max(axis=1) / np.abs(got).max()
    assert np.all(err <= F64_TOL), err
    t = s.t0 + idx * s.dt
    t_join = s.meta.get("t_join", s.tc)
    f = np.where(t <= t_join, synth.chirp_frequency(np.maximum(s.tc - t, 1e-9), s.mc_s), s.meta.get("f_rd", 1e-2))
    for k in (-4, -3):
        sel = (f >= 10.0 ** k) & (f < 10.0 ** (k + 1))
        assert sel.sum() >= 20, k
        e = np.abs(got[:, idx[sel]] - want[:, sel]).max(axis=1) / np.abs(want[:, sel]).max()
        assert np.all(e <= 2e-9), (k, e)
