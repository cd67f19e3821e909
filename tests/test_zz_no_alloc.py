"""The no-allocation hybrid call (lisa_response_hybrid_static) against the
regular one, bit for bit.

It serves callers that may not allocate device memory while running (their
own pool owns the GPU, or an allocator wait is not acceptable, or the
stream-ordered allocator is missing): same arguments and results, scratch in
a fixed array inside the library.  Both calls build the same orbit table
and the same link range and launch the same kernels, so their outputs must
be identical, bit for bit.  Called through the C ABI twice in a row,
on two different sources, so that leftovers of the first call in the shared
array would show up in the second.  This file is collected last so that a
run stopping at the first failure has already run every other test; it also
passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

import synth
from gpu_util import host_inputs, orbit_pair, sky_of, to_dev

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


def _call(L, fn, src, precision, tH, orbit):
    import paper_2505_09600_gb300.native as N
    hp, hc = host_inputs(src, precision)
    hpd, hcd = to_dev(hp, precision), to_dev(hc, precision)
    out = torch.full((3, src.n), float("nan"), device="cuda",
                     dtype=torch.float32 if precision == 1 else torch.float64)
    o = orbit.c()
    sky = N.lisa_sky(*sky_of(src))
    g = N.lisa_grid(src.t0, src.dt, src.n)
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(C.byref(o), C.byref(sky), g, C.c_void_p(hpd.data_ptr()), C.c_void_p(hcd.data_ptr()), precision, 20, 0,
            L.AET, tH, 800 * src.dt, 20 * src.dt, g, C.c_void_p(out.data_ptr()), st)
    assert rc == 0, L.load().lisa_last_error_message()
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_static_scratch_matches_allocating_call(L, precision):
    lib = L.load()
    _, lo = orbit_pair("kepler2_flex")
    for k, src in enumerate((synth.cfg2_small(n=20000), synth.cfg2_small(n=12000, seed_offset=7))):
        tH = src.t0 + (0.55 + 0.1 * k) * src.n * src.dt
        want = _call(L, lib.lisa_response_hybrid, src, precision, tH, lo)
        got = _call(L, lib.lisa_response_hybrid_static, src, precision, tH, lo)
        assert np.isfinite(got).all()
        assert np.array_equal(got, want), (k, np.abs(got - want).max())


def test_static_scratch_rejects_oversize(L):
    lib = L.load()
    import paper_2505_09600_gb300.native as N
    o = L.Orbit().c()
    sky = N.lisa_sky(0.2, 0.4, 0.6)
    g = N.lisa_grid(2e7, 0.5, 200_000_000)     # table alone would exceed the array
    x = torch.zeros(8, device="cuda")
    rc = lib.lisa_response_hybrid_static(C.byref(o), C.byref(sky), g, C.c_void_p(x.data_ptr()),
                                         C.c_void_p(x.data_ptr()), 1, 20, 0, 1, 2e7 + 1e6, 0.0, 0.0, g,
                                         C.c_void_p(x.data_ptr()), None)
    assert rc == -1
    assert b"static scratch" in lib.lisa_last_error_message()
