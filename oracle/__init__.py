"""FP64 CPU oracle of the time-domain LISA response (arXiv:2505.09600).

TEST INFRASTRUCTURE ONLY.  This package may be imported by the test suite,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``, and by
nothing else.  The CUDA library never imports, links or calls it, and shares
no code with it.  The arithmetic lives in ``oracle.c`` (plain C, FP64, no FMA
contraction); this module only builds it and marshals numpy arrays.

Functions and the paper passages they follow are documented in oracle.c.
Parity pins that check this oracle against what the paper and mathematics fix
live in tests/test_oracle_pins.py.  Submodules in plain numpy: ``noise`` (the
likelihood tail), ``mlp`` and ``corrector`` (the learned corrector),
``waveform`` (the synthetic source family generated on the device; pins in
tests/test_waveform_oracle.py).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

KEPLER1, KEPLER2, STATIC = 0, 1, 2
DELAY_LIGHTTIME, DELAY_ANALYTIC, DELAY_EQUAL, DELAY_LINEAR = 0, 1, 2, 3
FROZEN, NESTED = 0, 1
LFA_UNEQUAL, LFA_EQUAL, LFA_BACKWARD, LFA_FORWARD = 0, 1, 2, 3   # central (2 kinds); App. B non-central
LFA_NLO = 4       # central, next-to-leading order (App. B series and Michelson expansions)
LFA_STRAIN = 5    # strain-derivative form with the constellation centre (Sec. III)
C_LIGHT = 299792458.0
AU = 1.495978707e11
YEAR = 31557600.0


def build(force=False):
    """Compile oracle.c into _liboracle.so (gcc, -O2 -ffp-contract=off, OpenMP)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Grid(C.Structure):
    _fields_ = [("t0", C.c_double), ("dt", C.c_double), ("n", C.c_int64)]


class _Orbit(C.Structure):
    _fields_ = [("kind", C.c_int32), ("delay", C.c_int32), ("L_m", C.c_double),
                ("kappa0", C.c_double), ("lambda0", C.c_double), ("kepler_tilt", C.c_double),
                ("t_static", C.c_double), ("xi0", C.c_double), ("delta_l", C.c_double * 3),
                ("flex_scale", C.c_double), ("t_ref", C.c_double), ("lin_T0", C.c_double * 6),
                ("lin_Tdot", C.c_double * 6)]


class _Sky(C.Structure):
    _fields_ = [("beta", C.c_double), ("lam", C.c_double), ("psi", C.c_double)]


@dataclass
class Orbit:
    """Orbit and delay model (see oracle.c for the formulas)."""
    kind: int = KEPLER1
    delay: int = DELAY_LIGHTTIME
    L_m: float = 2.5e9
    kappa0: float = 0.0
    lambda0: float = 0.0
    kepler_tilt: float = 1.0
    t_static: float = 0.0
    xi0: float = 0.0
    delta_l: tuple = (0.0, 2.0943951023931953, 4.1887902047863905)
    flex_scale: float = 1.0
    t_ref: float = 0.0
    lin_T0: tuple = (0.0,) * 6
    lin_Tdot: tuple = (0.0,) * 6

    def c(self):
        o = _Orbit()
        o.kind, o.delay, o.L_m = self.kind, self.delay, self.L_m
        o.kappa0, o.lambda0, o.kepler_tilt, o.t_static = self.kappa0, self.lambda0, self.kepler_tilt, self.t_static
        o.xi0, o.flex_scale, o.t_ref = self.xi0, self.flex_scale, self.t_ref
        for q in range(3):
            o.delta_l[q] = self.delta_l[q]
        for q in range(6):
            o.lin_T0[q] = self.lin_T0[q]
            o.lin_Tdot[q] = self.lin_Tdot[q]
        return o


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_SO)
            P = C.POINTER
            d, i64, i32 = C.c_double, C.c_int64, C.c_int
            pd, pi64 = P(d), P(i64)
            po, ps = P(_Orbit), P(_Sky)
            sig = {
                "og_eccentricity": (d, [d]),
                "og_position": (None, [po, i32, d, pd]),
                "og_light_time": (d, [po, i32, d]),
                "og_link_vector": (None, [po, i32, d, d, pd]),
                "og_geometry": (None, [po, d, pd, pd, pd]),
                "og_orbits": (None, [po, Grid, pd, pd, pd]),
                "og_sky_basis": (None, [d, d, pd, pd, pd]),
                "og_antenna": (None, [pd, pd, pd, pd, pd]),
                "og_weights32": (None, [d, pd]),
                "og_lagrange32": (d, [pd, i64, i64, d]),
                "og_locate": (None, [Grid, i64, d, Grid, pi64, pd]),
                "og_links_full": (None, [po, ps, Grid, pd, pd, Grid, pd, pi64, i64]),
                "og_tdi_from_y": (None, [po, Grid, pd, i32, i32, Grid, pd, pi64, i64]),
                "og_tdi_full_direct": (None, [po, ps, Grid, pd, pd, Grid, i32, i32, Grid, pd, pi64, i64]),
                "og_aet": (None, [pd, pd, i64]),
                "og_hdot": (None, [Grid, pd, pd]),
                "og_d2": (None, [Grid, pd, pd]),
                "og_z_lfa_nlo": (None, [po, ps, Grid, pd, pd, pd, pd, i32, Grid, pd, pi64, i64]),
                "og_tdi_lfa_direct_nlo": (None, [po, ps, Grid, pd, pd, pd, pd, i32, Grid, pd, pi64, i64]),
                "og_tdi_strain": (None, [po, ps, Grid, pd, pd, i32, Grid, pd, pi64, i64]),
                "og_links_lfa_own_nlo": (None, [po, ps, Grid, pd, pd, pd, pd, Grid, pd, pi64, i64]),
                "og_z_lfa": (None, [po, ps, Grid, pd, pd, i32, i32, Grid, pd, pi64, i64]),
                "og_tdi_lfa_from_z": (None, [po, Grid, pd, i32, i32, pd, pi64, i64]),
                "og_tdi_lfa_direct": (None, [po, ps, Grid, pd, pd, i32, i32, Grid, pd, pi64, i64]),
                "og_links_lfa_own": (None, [po, ps, Grid, pd, pd, i32, Grid, pd, pi64, i64]),
                "og_sigmoid": (d, [d, d, d, d]),
                "og_t_hyb": (d, [d, d, d]),
                "og_hybrid_blend": (None, [Grid, d, d, d, i32, pd, pd, pd, pi64, i64]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _g(grid):
    if isinstance(grid, Grid):
        return grid
    t0, dt, n = grid
    return Grid(float(t0), float(dt), int(n))


def _pd(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _arr(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _idx(idx):
    if idx is None:
        return None, None, 0
    ix = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    return ix, ix.ctypes.data_as(C.POINTER(C.c_int64)), ix.size


def _sky(beta, lam, psi):
    return _Sky(float(beta), float(lam), float(psi))


# ---------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------

def eccentricity(L_m=2.5e9):
    return _load().og_eccentricity(L_m)


def position(orbit, sc, t):
    out = np.zeros(3)
    _load().og_position(C.byref(orbit.c()), sc, float(t), _pd(out))
    return out


def light_time(orbit, li, t):
    return _load().og_light_time(C.byref(orbit.c()), li, float(t))


def geometry(orbit, t):
    R, T, n = np.zeros(9), np.zeros(6), np.zeros(18)
    _load().og_geometry(C.byref(orbit.c()), float(t), _pd(R), _pd(T), _pd(n))
    return R.reshape(3, 3), T, n.reshape(6, 3)


def orbits(orbit, grid):
    g = _g(grid)
    R = np.zeros((3, 3, g.n)); T = np.zeros((6, g.n)); nh = np.zeros((6, 3, g.n))
    _load().og_orbits(C.byref(orbit.c()), g, _pd(R), _pd(T), _pd(nh))
    return R, T, nh


def sky_basis(beta, lam):
    k, u, v = np.zeros(3), np.zeros(3), np.zeros(3)
    _load().og_sky_basis(beta, lam, _pd(k), _pd(u), _pd(v))
    return k, u, v


def antenna(u, v, n):
    xp, xc = C.c_double(), C.c_double()
    _load().og_antenna(_pd(_arr(u)), _pd(_arr(v)), _pd(_arr(n)), C.byref(xp), C.byref(xc))
    return xp.value, xc.value


def weights32(eps):
    w = np.zeros(32)
    _load().og_weights32(float(eps), _pd(w))
    return w


def lagrange32(h, j, eps):
    h = _arr(h)
    return _load().og_lagrange32(_pd(h), h.size, int(j), float(eps))


def locate(gout, i, d, gin):
    j, e = C.c_int64(), C.c_double()
    _load().og_locate(_g(gout), int(i), float(d), _g(gin), C.byref(j), C.byref(e))
    return j.value, e.value


# ---------------------------------------------------------------------------
# full response
# ---------------------------------------------------------------------------

def links_full(orbit, sky, hgrid, hp, hc, ygrid, idx=None):
    """Six links y[6, m] (order l = +1,-1,+2,-2,+3,-3) on ygrid (or its samples idx)."""
    hp, hc = _arr(hp), _arr(hc)
    g = _g(ygrid)
    ix, pix, nix = _idx(idx)
    m = nix if ix is not None else g.n
    y = np.zeros((6, m))
    _load().og_links_full(C.byref(orbit.c()), C.byref(_sky(*sky)), _g(hgrid), _pd(hp), _pd(hc), g,
                          _pd(y), pix, nix)
    return y


def tdi_from_y(orbit, ygrid, y, gen=15, mode=FROZEN, outgrid=None, idx=None):
    y = _arr(y)
    gy = _g(ygrid)
    go = _g(outgrid) if outgrid is not None else gy
    ix, pix, nix = _idx(idx)
    m = nix if ix is not None else go.n
    xyz = np.zeros((3, m))
    _load().og_tdi_from_y(C.byref(orbit.c()), gy, _pd(y), gen, mode, go, _pd(xyz), pix, nix)
    return xyz


def tdi_full_direct(orbit, sky, hgrid, hp, hc, ygrid, gen, mode, outgrid, idx):
    hp, hc = _arr(hp), _arr(hc)
    ix, pix, nix = _idx(idx)
    xyz = np.zeros((3, nix))
    _load().og_tdi_full_direct(C.byref(orbit.c()), C.byref(_sky(*sky)), _g(hgrid), _pd(hp), _pd(hc),
                               _g(ygrid), gen, mode, _g(outgrid), _pd(xyz), pix, nix)
    return xyz


def aet(xyz):
    xyz = _arr(xyz)
    n = xyz.shape[1]
    out = np.zeros_like(xyz)
    _load().og_aet(_pd(xyz), _pd(out), n)
    return out


def response_full(orbit, sky, hgrid, hp, hc, gen=20, mode=FROZEN, channels="xyz", outgrid=None):
    """Full response: links on the output grid, then TDI, then optionally AET."""
    go = _g(outgrid) if outgrid is not None else _g(hgrid)
    y = links_full(orbit, sky, hgrid, hp, hc, go)
    xyz = tdi_from_y(orbit, go, y, gen, mode, go)
    return aet(xyz) if channels == "aet" else xyz


# ---------------------------------------------------------------------------
# LFA and hybrid
# ---------------------------------------------------------------------------

def hdot(grid, h):
    h = _arr(h)
    out = np.zeros_like(h)
    _load().og_hdot(_g(grid), _pd(h), _pd(out))
    return out


def d2(grid, x):
    """5-point second derivative on the grid, zero outside (og_d2)."""
    x = _arr(x)
    out = np.zeros_like(x)
    _load().og_d2(_g(grid), _pd(x), _pd(out))
    return out


def z_lfa(orbit, sky, hgrid, hp, hc, gen, kind, outgrid, idx=None, hd=None):
    """TDI-shifted LFA link series z[6, m] (X_a, X_b, Y_a, Y_b, Z_a, Z_b).
    kind LFA_NLO adds the next-to-leading link term (third derivative of h
    = og_d2 of hdot); LFA_STRAIN has no z series."""
    if kind == LFA_STRAIN:
        raise ValueError("the strain-derivative form has no z series")
    hdp, hdc = (hdot(hgrid, hp), hdot(hgrid, hc)) if hd is None else hd
    go = _g(outgrid)
    ix, pix, nix = _idx(idx)
    m = nix if ix is not None else go.n
    z = np.zeros((6, m))
    if kind == LFA_NLO:
        h3p, h3c = d2(hgrid, hdp), d2(hgrid, hdc)
        _load().og_z_lfa_nlo(C.byref(orbit.c()), C.byref(_sky(*sky)), _g(hgrid), _pd(hdp), _pd(hdc), _pd(h3p),
                             _pd(h3c), gen, go, _pd(z), pix, nix)
        return z
    _load().og_z_lfa(C.byref(orbit.c()), C.byref(_sky(*sky)), _g(hgrid), _pd(hdp), _pd(hdc),
                     gen, kind, go, _pd(z), pix, nix)
    return z


def strain_series(hgrid, h, gen, hd=None):
    """The strain derivative the strain-derivative form interpolates:
    d2h/dt2 = hdot of hdot (TDI 1.5), d3h/dt3 = og_d2 of hdot (TDI 2.0)."""
    hd = hdot(hgrid, h) if hd is None else hd
    return hdot(hgrid, hd) if gen == 15 else d2(hgrid, hd)


def tdi_strain(orbit, sky, hgrid, hp, hc, gen, outgrid, idx=None, hd=None):
    """X, Y, Z of the strain-derivative form (og_tdi_strain)."""
    hdp, hdc = (None, None) if hd is None else hd
    sp, sc = strain_series(hgrid, hp, gen, hdp), strain_series(hgrid, hc, gen, hdc)
    go = _g(outgrid)
    ix, pix, nix = _idx(idx)
    m = nix if ix is not None else go.n
    xyz = np.zeros((3, m))
    _load().og_tdi_strain(C.byref(orbit.c()), C.byref(_sky(*sky)), _g(hgrid), _pd(sp), _pd(sc), gen, go,
                          _pd(xyz), pix, nix)
    return xyz


def tdi_lfa_from_z(orbit, zgrid, z, gen, kind, idx=None):
    z = _arr(z)
    g = _g(zgrid)
    ix, pix, nix = _idx(idx)
    m = nix if ix is not None else g.n
    xyz = np.zeros((3, m))
    _load().og_tdi_lfa_from_z(C.byref(orbit.c()), g, _pd(z), gen, kind, _pd(xyz), pix, nix)
    return xyz


def tdi_lfa_direct(orbit, sky, hgrid, hp, hc, gen, kind, outgrid, idx, hd=None):
    if hd is None:
        hdp, hdc = hdot(hgrid, hp), hdot(hgrid, hc)
    else:
        hdp, hdc = hd
    if kind == LFA_STRAIN:
        return tdi_strain(orbit, sky, hgrid, hp, hc, gen, outgrid, idx, hd=(hdp, hdc))
    ix, pix, nix = _idx(idx)
    xyz = np.zeros((3, nix))
    if kind == LFA_NLO:
        h3p, h3c = d2(hgrid, hdp), d2(hgrid, hdc)
        _load().og_tdi_lfa_direct_nlo(C.byref(orbit.c()), C.byref(_sky(*sky)), _g(hgrid), _pd(hdp), _pd(hdc),
                                      _pd(h3p), _pd(h3c), gen, _g(outgrid), _pd(xyz), pix, nix)
        return xyz
    _load().og_tdi_lfa_direct(C.byref(orbit.c()), C.byref(_sky(*sky)), _g(hgrid), _pd(hdp), _pd(hdc),
                              gen, kind, _g(outgrid), _pd(xyz), pix, nix)
    return xyz


def response_lfa(orbit, sky, hgrid, hp, hc, gen=20, kind=LFA_UNEQUAL, channels="xyz", outgrid=None):
    go = _g(outgrid) if outgrid is not None else _g(hgrid)
    if kind == LFA_STRAIN:
        xyz = tdi_strain(orbit, sky, hgrid, hp, hc, gen, go)
        return aet(xyz) if channels == "aet" else xyz
    z = z_lfa(orbit, sky, hgrid, hp, hc, gen, kind, go)
    xyz = tdi_lfa_from_z(orbit, go, z, gen, kind)
    return aet(xyz) if channels == "aet" else xyz


def links_lfa_own(orbit, sky, hgrid, hp, hc, kind, ygrid, idx=None):
    if kind == LFA_STRAIN:
        raise ValueError("the strain-derivative form has no link series")
    hdp, hdc = hdot(hgrid, hp), hdot(hgrid, hc)
    g = _g(ygrid)
    ix, pix, nix = _idx(idx)
    m = nix if ix is not None else g.n
    y = np.zeros((6, m))
    if kind == LFA_NLO:
        h3p, h3c = d2(hgrid, hdp), d2(hgrid, hdc)
        _load().og_links_lfa_own_nlo(C.byref(orbit.c()), C.byref(_sky(*sky)), _g(hgrid), _pd(hdp), _pd(hdc),
                                     _pd(h3p), _pd(h3c), g, _pd(y), pix, nix)
        return y
    _load().og_links_lfa_own(C.byref(orbit.c()), C.byref(_sky(*sky)), _g(hgrid), _pd(hdp), _pd(hdc),
                             kind, g, _pd(y), pix, nix)
    return y


def sigmoid(t, tH, sigma, eps):
    return _load().og_sigmoid(float(t), float(tH), float(sigma), float(eps))


def t_hyb(f_hyb, mc_s, tc):
    return _load().og_t_hyb(float(f_hyb), float(mc_s), float(tc))


def hybrid_blend(grid, tH, Tw, sigma, lfa, full, idx=None):
    lfa, full = _arr(lfa), _arr(full)
    nch = lfa.shape[0]
    ix, pix, nix = _idx(idx)
    out = np.zeros_like(lfa)
    _load().og_hybrid_blend(_g(grid), float(tH), float(Tw), float(sigma), nch, _pd(lfa), _pd(full),
                            _pd(out), pix, nix)
    return out


def response_hybrid(orbit, sky, hgrid, hp, hc, gen=20, kind=LFA_UNEQUAL, channels="xyz",
                    t_h=None, Tw=None, sigma=None, outgrid=None):
    """Hybrid: blend of the whole-grid LFA and full Michelson variables."""
    go = _g(outgrid) if outgrid is not None else _g(hgrid)
    Tw = 800.0 * go.dt if Tw is None else Tw
    sigma = Tw / 40.0 if sigma is None else sigma
    lfa = response_lfa(orbit, sky, hgrid, hp, hc, gen, kind, "xyz", go)
    full = response_full(orbit, sky, hgrid, hp, hc, gen, FROZEN, "xyz", go)
    xyz = hybrid_blend(go, t_h, Tw, sigma, lfa, full)
    return aet(xyz) if channels == "aet" else xyz
