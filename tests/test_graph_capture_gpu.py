"""The hybrid call's second stream (the full part's links run on it beside the
LFA kernel): captured in a CUDA graph (its stream-ordered scratch, the side
stream and the kernels become graph nodes) and replayed, bit-identical to the
direct call, replay after replay, including after the inputs in the captured
buffers change; and two calls in flight on two streams at once."""
import numpy as np
import pytest

import synth
from gpu_util import orbit_pair, sky_of, to_dev

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


@pytest.mark.parametrize("precision", [1, 2])
def test_hybrid_graph_replay_matches_call(L, precision):
    s = synth.cfg2_small(n=30000)
    s2 = synth.cfg2_small(n=30000, seed_offset=3)
    _, lo = orbit_pair("kepler2_flex")
    tH = L.lisa_t_hyb_from_f(1e-3, s.mc_s, s.tc)
    Tw, sig = 800 * s.dt, 20 * s.dt
    hp, hc = to_dev(s.hp, precision), to_dev(s.hc, precision)
    dt = torch.float32 if precision == 1 else torch.float64
    out = torch.empty((3, s.n), device="cuda", dtype=dt)

    def call(o):
        L.lisa_response_hybrid(lo, sky_of(s), s.grid, hp, hc, precision, 20, 0, L.AET, tH, Tw, sig, s.grid, o)

    want = torch.empty_like(out)
    call(want)                               # also creates the side stream before the capture
    torch.cuda.synchronize()
    gs = torch.cuda.Stream()
    gs.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=gs):
        call(out)
    for _ in range(2):
        out.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, want)
    # new inputs in the captured buffers: the replay follows them
    hp.copy_(to_dev(s2.hp, precision))
    hc.copy_(to_dev(s2.hc, precision))
    g.replay()
    want2 = torch.empty_like(out)
    call(want2)
    torch.cuda.synchronize()
    assert torch.equal(out, want2)
    assert not torch.equal(want2, want)


def test_hybrid_calls_in_flight_on_two_streams(L):
    """Two hybrid calls queued back to back on two streams (each call forks
    its own side stream from the library's pool) give the results of the
    same calls run one after the other."""
    _, lo = orbit_pair("kepler2_flex")
    srcs = [synth.cfg2_small(n=30000), synth.cfg2_small(n=30000, seed_offset=5)]
    args = []
    for s in srcs:
        tH = L.lisa_t_hyb_from_f(1e-3, s.mc_s, s.tc)
        args.append((s, to_dev(s.hp, 2), to_dev(s.hc, 2), tH))

    def call(k, o, stream=None):
        s, hp, hc, tH = args[k]
        L.lisa_response_hybrid(lo, sky_of(s), s.grid, hp, hc, 2, 20, 0, L.AET, tH, 800 * s.dt, 20 * s.dt, s.grid,
                               o, stream=stream)

    want = [torch.empty((3, s.n), device="cuda", dtype=torch.float64) for s in srcs]
    for k in range(2):
        call(k, want[k])
    torch.cuda.synchronize()
    got = [torch.full_like(w, float("nan")) for w in want]
    st = [torch.cuda.Stream(), torch.cuda.Stream()]
    for k in range(2):
        st[k].wait_stream(torch.cuda.current_stream())
        call(k, got[k], stream=st[k].cuda_stream)
    torch.cuda.synchronize()
    for k in range(2):
        assert torch.equal(got[k], want[k]), k
