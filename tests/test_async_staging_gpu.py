"""The mixed LFA kernel stages each tile's h window with bulk asynchronous
copies (cp.async.bulk) when h starts on a 16-byte boundary, and with plain
loads otherwise: both must give bit-identical results, and no bounded device
wait may time out."""
import numpy as np
import pytest

import synth
from gpu_util import orbit_pair, sky_of

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


@pytest.mark.parametrize("n,dt", [(200000, 5.0), (50000, 10.0), (20000, 30.0)])
def test_bulk_and_plain_staging_agree(L, n, dt):
    s = synth.cfg2_small(n=n, dt=dt)
    _, lo = orbit_pair("kepler2_flex")
    hp32, hc32 = s.hp.astype(np.float32), s.hc.astype(np.float32)
    # aligned (bulk copies) and shifted by one float (plain loads)
    hp_a = torch.as_tensor(hp32, device="cuda")
    hc_a = torch.as_tensor(hc32, device="cuda")
    bp = torch.zeros(n + 1, device="cuda")
    bc = torch.zeros(n + 1, device="cuda")
    bp[1:] = hp_a
    bc[1:] = hc_a
    hp_u, hc_u = bp[1:], bc[1:]
    assert hp_u.data_ptr() % 16 != 0 and hp_a.data_ptr() % 16 == 0
    out_a = torch.full((3, n), float("nan"), device="cuda")
    out_u = torch.full((3, n), float("nan"), device="cuda")
    z_a = torch.full((6, n), float("nan"), device="cuda")
    z_u = torch.full((6, n), float("nan"), device="cuda")
    for gen in (L.TDI15, L.TDI20):
        L.lisa_response_lfa(lo, sky_of(s), s.grid, hp_a, hc_a, L.MIXED, gen, L.LFA_UNEQUAL, L.AET, s.grid, out_a)
        L.lisa_response_lfa(lo, sky_of(s), s.grid, hp_u, hc_u, L.MIXED, gen, L.LFA_UNEQUAL, L.AET, s.grid, out_u)
        L.lisa_links_lfa(lo, sky_of(s), s.grid, hp_a, hc_a, L.MIXED, gen, L.LFA_UNEQUAL, s.grid, z_a)
        L.lisa_links_lfa(lo, sky_of(s), s.grid, hp_u, hc_u, L.MIXED, gen, L.LFA_UNEQUAL, s.grid, z_u)
        torch.cuda.synchronize()
        assert torch.isfinite(out_a).all()
        assert torch.equal(out_a, out_u)
        assert torch.equal(z_a, z_u)
    assert L.lisa_device_status() == 0


def test_bounded_wait_times_out_and_context_survives(L):
    # a wait on an mbarrier that nothing arrives on gives up after its bound,
    # flags the status word and returns; the host reads LISA_ETIMEOUT once,
    # the word is cleared, and the context keeps working
    assert L.lisa_device_status() == 0
    L.lisa_selftest_wait_timeout()
    with pytest.raises(L.LisaError) as e:
        L.lisa_device_status()
    assert e.value.status == -4          # LISA_ETIMEOUT
    assert L.lisa_device_status() == 0   # cleared by the read
    s = synth.cfg2_small(n=3000)
    _, lo = orbit_pair("kepler2_flex")
    out = torch.full((3, s.n), float("nan"), device="cuda")
    L.lisa_response_lfa(lo, sky_of(s), s.grid, torch.as_tensor(s.hp.astype(np.float32), device="cuda"),
                        torch.as_tensor(s.hc.astype(np.float32), device="cuda"), L.MIXED, L.TDI20, L.LFA_UNEQUAL,
                        L.AET, s.grid, out)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
