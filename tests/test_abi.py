"""The C ABI library builds, loads and exports every symbol include/lisa.h
declares; argument validation answers on the host before anything launches
(no GPU needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_09600_gb300 import build, native
    build.build()
    return native.load()


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(lisa_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_2505_09600_gb300 import native
    assert set(native.exported_symbols()) <= set(_declared())


def test_strerror_and_version(lib):
    from paper_2505_09600_gb300 import native
    assert native.lisa_version() >= 10000
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert lib.lisa_strerror(code)
    assert lib.lisa_strerror(-99) == b"unknown status"


def test_t_hyb_matches_oracle(oracle_mod):
    from paper_2505_09600_gb300 import native
    for f, m, tc in ((3e-4, 4.9, 5e7), (1e-3, 0.49, 4e7)):
        assert native.lisa_t_hyb_from_f(f, m, tc) == pytest.approx(oracle_mod.t_hyb(f, m, tc), rel=0, abs=1e-6)


def test_validation_rejects_bad_arguments_without_launching(lib):
    from paper_2505_09600_gb300 import native as N
    o = N.Orbit().c()
    s = N.lisa_sky(0.1, 0.2, 0.3)
    g = N.lisa_grid(0.0, 5.0, 100)
    bad_dt = N.lisa_grid(0.0, 0.0, 100)
    neg_n = N.lisa_grid(0.0, 5.0, -1)
    nul = C.c_void_p(0)
    # NULL orbit / sky, bad grids, bad enums and NULL series are rejected on the host
    assert lib.lisa_links_full(None, C.byref(s), g, nul, nul, 0, g, nul, nul) == N.LISA_EINVAL
    assert lib.lisa_links_full(C.byref(o), None, g, nul, nul, 0, g, nul, nul) == N.LISA_EINVAL
    assert lib.lisa_links_full(C.byref(o), C.byref(s), bad_dt, nul, nul, 0, g, nul, nul) == N.LISA_EINVAL
    assert lib.lisa_links_full(C.byref(o), C.byref(s), g, nul, nul, 0, neg_n, nul, nul) == N.LISA_EINVAL
    assert lib.lisa_links_full(C.byref(o), C.byref(s), g, nul, nul, 7, g, nul, nul) == N.LISA_EINVAL
    assert lib.lisa_links_full(C.byref(o), C.byref(s), g, nul, nul, 0, g, nul, nul) == N.LISA_EINVAL
    assert lib.lisa_tdi(C.byref(o), g, nul, 0, 16, 0, 0, g, nul, nul) == N.LISA_EINVAL
    assert lib.lisa_tdi(C.byref(o), g, nul, 0, 20, 5, 0, g, nul, nul) == N.LISA_EINVAL
    assert lib.lisa_response_lfa(C.byref(o), C.byref(s), g, nul, nul, 0, 20, 3, 0, g, nul, nul) == N.LISA_EINVAL
    assert lib.lisa_response_hybrid(C.byref(o), C.byref(s), g, nul, nul, 0, 20, 0, 0, float("nan"), 0.0, 0.0, g,
                                    nul, nul) == N.LISA_EINVAL
    ob = N.Orbit(kind=9).c()
    assert lib.lisa_orbits(C.byref(ob), g, nul, nul, nul, nul) == N.LISA_EINVAL
    ob = N.Orbit(L_m=-1.0).c()
    assert lib.lisa_orbits(C.byref(ob), g, nul, nul, nul, nul) == N.LISA_EINVAL
    assert b"L_m" in lib.lisa_last_error_message()
    # empty outputs are a no-op
    e = N.lisa_grid(0.0, 5.0, 0)
    assert lib.lisa_orbits(C.byref(o), e, nul, nul, nul, nul) == N.LISA_OK
    assert lib.lisa_response_full(C.byref(o), C.byref(s), g, nul, nul, 0, 20, 0, e, nul, nul) == N.LISA_OK
