"""Config 5 (parameter-estimation draws): eccentric chirp + ringdown around
Mc = 5e5 Msun, q = 2, one year at 10 s (3,155,760 samples per draw).

The mixed hybrid response of whole draws, through the host-buffer call and
through one batched plan, against the FP64 oracle on sampled outputs (the
oracle evaluates chosen samples directly: the LFA from the grid derivative
of h, the full response from the links at the TDI delays, then the blend),
at the frozen hybrid tolerance.  The batched plan must return what the
single-draw call returns (same groups, same kernels; the TDI blocks follow
the plan's groups, so FP32 rounding)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import orbit_pair
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


@pytest.fixture(scope="module")
def draws():
    ps = synth.pe_params(ndraw=3)
    return [synth.pe_source(p) for p in ps[:2]]


def _sampled_oracle(oo, s, hp, hc, tH, Tw, sig, idx):
    sky = (s.beta, s.lam, s.psi)
    hd = (oracle.hdot(s.grid, hp), oracle.hdot(s.grid, hc))
    lf = oracle.tdi_lfa_direct(oo, sky, s.grid, hp, hc, 20, 0, s.grid, idx, hd=hd)
    fu = np.zeros_like(lf)
    need = s.t0 + idx * s.dt >= tH - 0.5 * Tw
    if need.any():
        fu[:, need] = oracle.tdi_full_direct(oo, sky, s.grid, hp, hc, s.grid, 20, 0, s.grid, idx[need])
    return oracle.aet(oracle.hybrid_blend(s.grid, tH, Tw, sig, lf, fu, idx))


def test_pe_draws_hybrid_against_oracle(L, draws):
    oo, lo = orbit_pair("kepler2_flex")
    rng = np.random.default_rng(5)
    for s in draws:
        hp = s.hp.astype(np.float32)
        hc = s.hc.astype(np.float32)
        tH = L.lisa_t_hyb_from_f(1e-3, s.mc_s, s.tc)
        Tw, sig = 800 * s.dt, 20 * s.dt
        out = torch.empty((3, s.n), dtype=torch.float32).pin_memory()
        st = torch.cuda.Stream()
        L.lisa_response_hybrid_host(lo, (s.beta, s.lam, s.psi), s.grid, torch.from_numpy(hp).pin_memory(),
                                    torch.from_numpy(hc).pin_memory(), L.MIXED, 20, 0, L.AET, tH, Tw, sig, out,
                                    stream=st.cuda_stream)
        st.synchronize()
        got = out.numpy().astype(np.float64)
        assert np.isfinite(got).all()
        # samples: spread over the year, dense around the switch and the merger
        i_h = int((tH - s.t0) / s.dt)
        idx = np.unique(np.concatenate([rng.integers(0, s.n, 120), np.arange(i_h - 500, i_h + 500, 25),
                                        np.arange(s.n - 1400, s.n, 20)]))
        idx = idx[(idx >= 0) & (idx < s.n)]
        want = _sampled_oracle(oo, s, hp.astype(np.float64), hc.astype(np.float64), tH, Tw, sig, idx)
        err = np.abs(got[:, idx] - want).max(axis=1) / np.abs(got).max()
        assert np.all(err <= np.asarray(MIXED_TOL["hybrid20"]["aet"])), err


def test_pe_draws_batched_plan_matches_single(L, draws):
    oo, lo = orbit_pair("kepler2_flex")
    srcs, singles = [], []
    keep = []
    for s in draws:
        hp = torch.as_tensor(s.hp.astype(np.float32), device="cuda")
        hc = torch.as_tensor(s.hc.astype(np.float32), device="cuda")
        tH = L.lisa_t_hyb_from_f(1e-3, s.mc_s, s.tc)
        one = torch.empty((3, s.n), device="cuda")
        L.lisa_response_hybrid(lo, (s.beta, s.lam, s.psi), s.grid, hp, hc, L.MIXED, 20, 0, L.AET, tH, 0.0, 0.0,
                               s.grid, one)
        out = torch.full((3, s.n), float("nan"), device="cuda")
        keep += [hp, hc, out]
        srcs.append(dict(grid=s.grid, hp=hp, hc=hc, sky=(s.beta, s.lam, s.psi), t_hyb=tH, T_win=0.0, sigma=0.0,
                         out=out))
        singles.append(one)
    plan = L.LisaPlan(lo, srcs, precision=L.MIXED, tdi_gen=20, lfa_kind=0, channels=L.AET)
    plan.execute()
    torch.cuda.synchronize()
    for d, one in zip(srcs, singles):
        got, ref = d["out"], one
        assert torch.isfinite(got).all()
        assert float((got - ref).abs().max() / ref.abs().max()) <= 2e-6
