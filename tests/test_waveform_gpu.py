"""On-device generation of the synthetic source family (lisa_chirp_ringdown)
against the FP64 oracle (oracle/waveform.py): FP64 and mixed forms, single
and batched draws, full-length config-5 draws on sampled outputs, ragged and
degenerate grids, and argument errors."""
import math

import numpy as np
import pytest

import synth
from oracle import waveform as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

T_SUN = synth.T_SUN
F64_TOL = 1e-11      # relative to the draw's max |h|
MIXED_TOL = 2e-6     # FP32 output continuing an FP64 phase anchor per 32 samples


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_09600_gb300 import build
    build.build()
    import paper_2505_09600_gb300 as L
    L.load()
    return L


def _draw(mc=1e6, q=3.0, e0=0.0, tc=2.0e7 + 1.4e5, iota=0.5, phi_c=1.3, f_cut=0.0, dist=10.0 * synth.GPC):
    return dict(mc_s=mc * T_SUN, q=q, dist_m=dist, iota=iota, phi_c=phi_c, tc=tc, e0=e0, f_cut=f_cut)


def _oracle(d, grid, idx=None):
    return W.chirp_ringdown(grid, d["mc_s"], d["q"], d["dist_m"], d["iota"], d["phi_c"], d["tc"], e0=d.get("e0", 0.0),
                            f_cut=d.get("f_cut", 0.0), m_final_frac=d.get("m_final_frac", 0.95),
                            a_final=d.get("a_final", 0.7), idx=idx)


def _gen(L, draws, grid, precision):
    dt = torch.float64 if precision == 0 else torch.float32
    hp = torch.full((len(draws), grid[2]), float("nan"), device="cuda", dtype=dt)
    hc = torch.full_like(hp, float("nan"))
    L.lisa_chirp_ringdown(draws, grid, precision, hp, hc)
    torch.cuda.synchronize()
    return hp.double().cpu().numpy(), hc.double().cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("e0", [0.0, 0.25])
def test_matches_oracle_through_merger(L, precision, e0):
    # 30,001 samples at 5 s: inspiral, the join and the ringdown (ragged tail)
    d = _draw(e0=e0)
    grid = (2.0e7, 5.0, 30001)
    hp, hc = _gen(L, [d], grid, precision)
    wp, wc = _oracle(d, grid)
    scale = max(np.abs(wp).max(), np.abs(wc).max())
    tol = F64_TOL if precision == 0 else MIXED_TOL
    assert np.abs(hp[0] - wp).max() <= tol * scale
    assert np.abs(hc[0] - wc).max() <= tol * scale


@pytest.mark.parametrize("precision", [0, 1])
def test_full_year_draws_sampled(L, precision):
    # config 5: one year at 10 s (3,155,760 samples) per draw, eccentric, batched;
    # sampled outputs: spread over the year, dense around the join and the end
    ps = synth.pe_params(ndraw=3)
    n, dt, t0 = 3155760, 10.0, 2.0e7
    tc = t0 + n * dt - 1.0e4
    draws = [dict(mc_s=p["mc"] * T_SUN, q=p["q"], dist_m=10.0 * synth.GPC, iota=0.5, phi_c=p["phi_c"], tc=tc,
                  e0=p["e0"], f_cut=0.8 * 0.5 / dt) for p in ps]
    grid = (t0, dt, n)
    hp, hc = _gen(L, draws, grid, precision)
    rng = np.random.default_rng(11)
    tol = F64_TOL if precision == 0 else MIXED_TOL
    for k, d in enumerate(draws):
        _, tau_join, _ = W.join_point(d["mc_s"], d["q"], d["f_cut"])
        i_j = int((tc - tau_join - t0) / dt)
        idx = np.unique(np.concatenate([rng.integers(0, n, 300), np.arange(i_j - 300, i_j + 300),
                                        np.arange(n - 1000, n, 5), [0, n - 1]]))
        wp, wc = _oracle(d, grid, idx)
        scale = max(np.abs(hp[k]).max(), np.abs(hc[k]).max())
        assert np.abs(hp[k, idx] - wp).max() <= tol * scale, k
        assert np.abs(hc[k, idx] - wc).max() <= tol * scale, k
    # a batched row is what the single-draw call returns
    one_p, one_c = _gen(L, [draws[1]], grid, precision)
    assert np.array_equal(one_p[0], hp[1]) and np.array_equal(one_c[0], hc[1])
    # and the mixed form is the benchmarks' input generator to FP32 accuracy
    if precision == 1:
        s = synth.pe_source(ps[0], n=n, dt=dt, t0=t0)
        assert np.abs(hp[0] - s.hp).max() <= MIXED_TOL * np.abs(s.hp).max()


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", ["one", "ragged", "after_tc", "face_on", "cut"])
def test_edges(L, precision, case):
    d = _draw()
    grid = (2.0e7 + 1.2e5, 5.0, 4099)
    if case == "one":
        grid = (2.0e7 + 1.39e5, 5.0, 1)
    elif case == "ragged":
        grid = (2.0e7, 7.0, 33)
    elif case == "after_tc":
        grid = (d["tc"] + 10.0, 5.0, 3000)        # ringdown only, decaying
    elif case == "face_on":
        d = _draw(iota=0.0, e0=0.1)
    elif case == "cut":
        d = _draw(f_cut=5e-4)                     # join and ringdown capped below f_ISCO
        _, tau_join, _ = W.join_point(d["mc_s"], d["q"], d["f_cut"])
        grid = (d["tc"] - tau_join - 1.0e4, 5.0, 4099)   # around the (earlier) join
    hp, hc = _gen(L, [d], grid, precision)
    wp, wc = _oracle(d, grid)
    scale = max(np.abs(wp).max(), np.abs(wc).max(), 1e-300)
    tol = F64_TOL if precision == 0 else MIXED_TOL
    assert np.isfinite(hp).all() and np.isfinite(hc).all()
    assert np.abs(hp[0] - wp).max() <= tol * scale
    assert np.abs(hc[0] - wc).max() <= tol * scale


def test_arguments(L):
    grid = (2.0e7, 5.0, 100)
    hp = torch.zeros((1, 100), device="cuda")
    hc = torch.zeros_like(hp)
    for bad in (dict(q=0.5), dict(e0=1.0), dict(mc=-1.0), dict(dist=0.0)):
        kw = dict(mc=1e6, q=3.0, e0=0.0, dist=1e25)
        kw.update(bad)
        with pytest.raises(L.LisaError):
            L.lisa_chirp_ringdown([_draw(**kw)], grid, L.MIXED, hp, hc)
    # no draws: nothing to do
    L.lisa_chirp_ringdown([], grid, L.MIXED, torch.zeros((0, 100), device="cuda"), torch.zeros((0, 100), device="cuda"))
