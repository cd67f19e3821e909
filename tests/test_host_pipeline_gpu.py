"""lisa_response_hybrid_host (series in host memory, copies overlapped with the
kernels in up to 8 chunks) against lisa_response_hybrid on device copies of
the same series, and against the oracle.

Chunk boundaries fall on the LFA tile groups, so the LFA-only samples are
bit-identical; the TDI blocks (and, on short ranges, the split of the FP64
links and TDI over more CTAs) follow the chunks, so the full-response samples
agree to FP32 rounding (mixed) and to FP64 rounding (FP64)."""
import numpy as np
import pytest

import synth
from gpu_util import host_inputs, orbit_pair, rel_err, sky_of, to_dev
from tolerances import MIXED_TOL

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


def _pair(L, s, precision, gen, channels, pinned=True):
    oo, lo = orbit_pair("kepler2_flex")
    hp, hc = host_inputs(s, precision)
    tH = L.lisa_t_hyb_from_f(1e-3, s.mc_s, s.tc)
    Tw, sig = 800 * s.dt, 20 * s.dt
    dt = torch.float32 if precision == L.MIXED else torch.float64
    dev = torch.empty((3, s.n), device="cuda", dtype=dt)
    L.lisa_response_hybrid(lo, sky_of(s), s.grid, to_dev(hp, precision), to_dev(hc, precision), precision, gen, 0,
                           channels, tH, Tw, sig, s.grid, dev)
    hp_h = torch.as_tensor(np.ascontiguousarray(hp)).to(dt)
    hc_h = torch.as_tensor(np.ascontiguousarray(hc)).to(dt)
    out_h = torch.full((3, s.n), float("nan"), dtype=dt)
    if pinned:
        hp_h, hc_h, out_h = hp_h.pin_memory(), hc_h.pin_memory(), out_h.pin_memory()
    st = torch.cuda.Stream()
    L.lisa_response_hybrid_host(lo, sky_of(s), s.grid, hp_h, hc_h, precision, gen, 0, channels, tH, Tw, sig, out_h,
                                stream=st.cuda_stream)
    st.synchronize()
    return dev.cpu().numpy().astype(np.float64), out_h.numpy().astype(np.float64), (oo, hp, hc, tH, Tw, sig)


def _split(s, tH, Tw):
    t = s.t0 + np.arange(s.n) * s.dt
    return int(np.searchsorted(t, tH - 0.5 * Tw, side="left"))   # first full-response sample


@pytest.mark.parametrize("gen", [15, 20])
def test_host_pipeline_mixed_matches_device(L, gen):
    s = synth.cfg2_small(n=40000)
    dev, host, (_, _, _, tH, Tw, _) = _pair(L, s, L.MIXED, gen, 1)
    assert np.isfinite(host).all()
    iF = _split(s, tH, Tw)
    assert 0 < iF < s.n
    assert np.array_equal(host[:, :iF], dev[:, :iF])          # LFA only: same tiles, same groups
    assert np.abs(host - dev).max() <= 2e-6 * np.abs(dev).max()


def test_host_pipeline_f64(L):
    s = synth.cfg2_small(n=20000)
    dev, host, (_, _, _, tH, Tw, _) = _pair(L, s, L.F64, 20, 0)
    iF = _split(s, tH, Tw)
    assert 0 < iF < s.n
    assert np.array_equal(host[:, :iF], dev[:, :iF])          # LFA only: same tiles, same groups
    # full part: the same FP64 arithmetic over other block boundaries
    assert np.abs(host - dev).max() <= 1e-13 * np.abs(dev).max()


def test_host_pipeline_double_float(L):
    # chunks on the double-float kernel's own tile groups: LFA samples
    # bit-identical; n spans several groups of 6 tiles and ends in a ragged one
    s = synth.cfg2_small(n=40000)
    dev, host, (_, _, _, tH, Tw, _) = _pair(L, s, L.DF, 20, 1)
    iF = _split(s, tH, Tw)
    assert 0 < iF < s.n
    assert np.array_equal(host[:, :iF], dev[:, :iF])
    assert np.abs(host - dev).max() <= 1e-13 * np.abs(dev).max()


def test_host_pipeline_pageable_and_oracle(L, oracle_mod):
    s = synth.cfg2_small(n=20000)
    dev, host, (oo, hp, hc, tH, Tw, sig) = _pair(L, s, L.MIXED, 20, 1, pinned=False)
    assert np.abs(host - dev).max() <= 2e-6 * np.abs(dev).max()
    want = oracle_mod.response_hybrid(oo, sky_of(s), s.grid, hp, hc, 20, 0, "aet", tH, Tw, sig)
    err = rel_err(host, want, signal=True)
    assert np.all(err <= np.asarray(MIXED_TOL["hybrid20"]["aet"])), err


def test_host_pipeline_tiny_grid(L):
    # fewer samples than one tile group: a single chunk
    s = synth.cfg2_small(n=1500)
    dev, host, _ = _pair(L, s, L.MIXED, 20, 0)
    assert np.abs(host - dev).max() <= 2e-6 * np.abs(dev).max()
