"""ctypes binding of liblisa.so (include/lisa.h).

Argument marshalling only: every step of the response runs in the CUDA
library.  Series are torch CUDA tensors (device memory owned by the caller);
calls are asynchronous on the current torch stream unless `stream` is given.
If the library is missing or cannot be loaded, every call raises: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading
from dataclasses import dataclass

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblisa.so")

LISA_OK, LISA_EINVAL, LISA_ERANGE, LISA_ECUDA, LISA_ETIMEOUT, LISA_ENOMEM, LISA_ECORRECTOR = 0, -1, -2, -3, -4, -5, -6
ORB_KEPLER1, ORB_KEPLER2, ORB_STATIC = 0, 1, 2
DELAY_LIGHTTIME, DELAY_ANALYTIC, DELAY_EQUAL, DELAY_LINEAR = 0, 1, 2, 3
F64, MIXED, DF = 0, 1, 2
TDI15, TDI20 = 15, 20
XYZ, AET = 0, 1
FROZEN, NESTED = 0, 1
LFA_UNEQUAL, LFA_EQUAL, LFA_BACKWARD, LFA_FORWARD, LFA_NLO, LFA_STRAIN = 0, 1, 2, 3, 4, 5


class LisaError(RuntimeError):
    def __init__(self, status, where, detail):
        super().__init__("%s failed with status %d: %s" % (where, status, detail))
        self.status = status


class lisa_grid(C.Structure):
    _fields_ = [("t0", C.c_double), ("dt", C.c_double), ("n", C.c_int64)]


class lisa_orbit(C.Structure):
    _fields_ = [("kind", C.c_int32), ("delay", C.c_int32), ("L_m", C.c_double),
                ("kappa0", C.c_double), ("lambda0", C.c_double), ("kepler_tilt", C.c_double),
                ("t_static", C.c_double), ("xi0", C.c_double), ("delta_l", C.c_double * 3),
                ("flex_scale", C.c_double), ("t_ref", C.c_double), ("lin_T0", C.c_double * 6),
                ("lin_Tdot", C.c_double * 6)]


class lisa_sky(C.Structure):
    _fields_ = [("beta", C.c_double), ("lam", C.c_double), ("psi", C.c_double)]


class lisa_source(C.Structure):
    _fields_ = [("grid", lisa_grid), ("hp", C.c_void_p), ("hc", C.c_void_p), ("sky", lisa_sky),
                ("t_hyb", C.c_double), ("T_win", C.c_double), ("sigma", C.c_double), ("out", C.c_void_p)]


class lisa_chirp(C.Structure):
    _fields_ = [("mc_s", C.c_double), ("q", C.c_double), ("dist_m", C.c_double), ("iota", C.c_double),
                ("phi_c", C.c_double), ("tc", C.c_double), ("e0", C.c_double), ("f_cut", C.c_double),
                ("m_final_frac", C.c_double), ("a_final", C.c_double)]


class lisa_tune_result(C.Structure):
    _fields_ = [("ctas_per_sm", C.c_int), ("tiles_per_item", C.c_int), ("ms", C.c_float)]


@dataclass
class Orbit:
    """Orbit and light-time model (fields of lisa_orbit)."""
    kind: int = ORB_KEPLER1
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
        o = lisa_orbit()
        o.kind, o.delay, o.L_m = self.kind, self.delay, self.L_m
        o.kappa0, o.lambda0, o.kepler_tilt, o.t_static = self.kappa0, self.lambda0, self.kepler_tilt, self.t_static
        o.xi0, o.flex_scale, o.t_ref = self.xi0, self.flex_scale, self.t_ref
        for q in range(3):
            o.delta_l[q] = self.delta_l[q]
        for q in range(6):
            o.lin_T0[q] = self.lin_T0[q]
            o.lin_Tdot[q] = self.lin_Tdot[q]
        return o


_lock = threading.Lock()
_lib = None

_P = C.c_void_p
_SIGS = {
    "lisa_version": (C.c_int, []),
    "lisa_strerror": (C.c_char_p, [C.c_int]),
    "lisa_last_error_message": (C.c_char_p, []),
    "lisa_t_hyb_from_f": (C.c_double, [C.c_double, C.c_double, C.c_double]),
    "lisa_orbits": (C.c_int, [C.POINTER(lisa_orbit), lisa_grid, _P, _P, _P, _P]),
    "lisa_links_full": (C.c_int, [C.POINTER(lisa_orbit), C.POINTER(lisa_sky), lisa_grid, _P, _P, C.c_int,
                                  lisa_grid, _P, _P]),
    "lisa_tdi": (C.c_int, [C.POINTER(lisa_orbit), lisa_grid, _P, C.c_int, C.c_int, C.c_int, C.c_int,
                           lisa_grid, _P, _P]),
    "lisa_response_full": (C.c_int, [C.POINTER(lisa_orbit), C.POINTER(lisa_sky), lisa_grid, _P, _P, C.c_int,
                                     C.c_int, C.c_int, lisa_grid, _P, _P]),
    "lisa_links_lfa": (C.c_int, [C.POINTER(lisa_orbit), C.POINTER(lisa_sky), lisa_grid, _P, _P, C.c_int,
                                 C.c_int, C.c_int, lisa_grid, _P, _P]),
    "lisa_tdi_lfa": (C.c_int, [C.POINTER(lisa_orbit), lisa_grid, _P, C.c_int, C.c_int, C.c_int, C.c_int,
                               _P, _P]),
    "lisa_response_lfa": (C.c_int, [C.POINTER(lisa_orbit), C.POINTER(lisa_sky), lisa_grid, _P, _P, C.c_int,
                                    C.c_int, C.c_int, C.c_int, lisa_grid, _P, _P]),
    "lisa_response_hybrid_static": (C.c_int, [C.POINTER(lisa_orbit), C.POINTER(lisa_sky), lisa_grid, _P, _P, C.c_int,
                                              C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                              lisa_grid, _P, _P]),
    "lisa_plan_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(lisa_orbit), C.c_int, C.c_int, C.c_int, C.c_int,
                                   C.POINTER(lisa_source), C.c_int]),
    "lisa_plan_destroy": (C.c_int, [C.c_void_p]),
    "lisa_plan_execute": (C.c_int, [C.c_void_p, _P]),
    "lisa_plan_capture_graph": (C.c_int, [C.c_void_p, _P]),
    "lisa_plan_replay": (C.c_int, [C.c_void_p, _P]),
    "lisa_plan_set_launch": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "lisa_plan_autotune": (C.c_int, [C.c_void_p, _P, C.POINTER(lisa_tune_result)]),
    "lisa_plan_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int),
                                 C.POINTER(C.c_int)]),
    "lisa_profile_enable": (C.c_int, [C.c_int]),
    "lisa_profile_query": (C.c_int, [C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "lisa_launch_count": (C.c_int64, []),
    "lisa_peak_fma_blocks": (C.c_int, [C.c_int, C.POINTER(C.c_int64)]),
    "lisa_peak_fma": (C.c_int, [C.c_int, C.c_int64, C.c_int, _P, C.POINTER(C.c_double), _P]),
    "lisa_device_status": (C.c_int, [C.POINTER(C.c_uint), C.c_int]),
    "lisa_selftest_wait_timeout": (C.c_int, [_P]),
    "lisa_response_hybrid": (C.c_int, [C.POINTER(lisa_orbit), C.POINTER(lisa_sky), lisa_grid, _P, _P, C.c_int,
                                       C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                       lisa_grid, _P, _P]),
    "lisa_response_hybrid_host": (C.c_int, [C.POINTER(lisa_orbit), C.POINTER(lisa_sky), lisa_grid, _P, _P, C.c_int,
                                            C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, _P, _P]),
    "lisa_psd_aet": (C.c_int, [C.c_double, C.c_double, C.c_int64, C.c_int, C.c_double, C.c_double, C.c_int, _P,
                               _P]),
    "lisa_fft_length": (C.c_int64, [C.c_int64]),
    "lisa_chirp_ringdown": (C.c_int, [C.POINTER(lisa_chirp), C.c_int, lisa_grid, C.c_int, _P, _P, _P]),
    "lisa_noise_weights_aet": (C.c_int, [lisa_grid, C.c_int64, C.c_int, C.c_double, C.c_double, C.c_int, C.c_double,
                                         C.c_double, _P, _P]),
    "lisa_inner_aet": (C.c_int, [lisa_grid, C.c_int64, _P, _P, C.c_int, _P, _P, _P]),
    "lisa_corrector_num_params": (C.c_int64, []),
    "lisa_corrector_num_features": (C.c_int, []),
    "lisa_corrector_create": (C.c_int, [C.POINTER(C.c_void_p), _P, C.c_int64, C.c_uint64]),
    "lisa_corrector_destroy": (C.c_int, [C.c_void_p]),
    "lisa_corrector_configure": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_double]),
    "lisa_corrector_get_state": (C.c_int, [C.c_void_p, _P, _P, _P, C.POINTER(C.c_int64), C.c_int64]),
    "lisa_corrector_set_state": (C.c_int, [C.c_void_p, _P, _P, _P, C.c_int64, C.c_int64]),
    "lisa_corrector_features": (C.c_int, [C.POINTER(lisa_orbit), C.POINTER(lisa_sky), lisa_grid, _P, _P, _P,
                                          C.c_double, C.c_double, _P, _P, _P, _P, _P]),
    "lisa_corrector_forward": (C.c_int, [C.c_void_p, _P, C.c_int64, _P, _P]),
    "lisa_corrector_gradient": (C.c_int, [C.c_void_p, _P, _P, C.c_int64, C.c_int64, C.c_uint64, _P, _P, _P]),
    "lisa_corrector_adam_step": (C.c_int, [C.c_void_p, _P, C.c_float, _P]),
    "lisa_corrector_train": (C.c_int, [C.c_void_p, _P, _P, C.c_int64, C.c_int64, C.c_int64, C.c_float, C.c_float,
                                       C.c_uint64, _P, _P]),
    "lisa_corrector_links": (C.c_int, [C.c_void_p, C.POINTER(lisa_orbit), C.POINTER(lisa_sky), lisa_grid, _P, _P,
                                       lisa_grid, _P, _P]),
    "lisa_links_lfa_own": (C.c_int, [C.POINTER(lisa_orbit), C.POINTER(lisa_sky), lisa_grid, _P, _P, C.c_int, C.c_int,
                                     lisa_grid, _P, _P]),
    "lisa_response_hybrid_corrected": (C.c_int, [C.c_void_p, C.POINTER(lisa_orbit), C.POINTER(lisa_sky), lisa_grid,
                                                 _P, _P, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                                 C.c_double, lisa_grid, _P, _P]),
    "lisa_corrector_report": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                        C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_float), C.c_int]),
}


def exported_symbols():
    """Names this binding expects the library to export."""
    return list(_SIGS)


def load(path=None):
    """Load liblisa.so (build it first with paper_2505_09600_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError("liblisa.so not found at %s: run paper_2505_09600_gb300.build.build() "
                                   "(there is no CPU fallback)" % p)
            lib = C.CDLL(p)
            for name, (res, args) in _SIGS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _check(rc, where):
    if rc != LISA_OK:
        lib = load()
        raise LisaError(rc, where, lib.lisa_last_error_message().decode(errors="replace"))


def _grid(g):
    if isinstance(g, lisa_grid):
        return g
    t0, dt, n = g
    return lisa_grid(float(t0), float(dt), int(n))


def _sky(s):
    return lisa_sky(float(s[0]), float(s[1]), float(s[2]))


def _orb(o):
    return (o if isinstance(o, Orbit) else Orbit()).c()


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, dtype=None, numel=None, name="tensor"):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s (got %s)" % (name, dtype, t.dtype))
    if numel is not None and t.numel() != numel:
        raise ValueError("%s must have %d elements (got %d)" % (name, numel, t.numel()))
    return C.c_void_p(t.data_ptr())


def _host_ptr(t, dtype=None, numel=None, name="tensor"):
    """Host memory: a contiguous CPU tensor (page-locked for overlapped copies)."""
    import torch
    if not isinstance(t, torch.Tensor) or t.is_cuda:
        raise TypeError("%s must be a CPU tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if dtype is not None and t.dtype != dtype:
        raise TypeError("%s must be %s (got %s)" % (name, dtype, t.dtype))
    if numel is not None and t.numel() != numel:
        raise ValueError("%s must have %d elements (got %d)" % (name, numel, t.numel()))
    return C.c_void_p(t.data_ptr())


def _rdtype(precision):
    import torch
    return torch.float32 if precision == MIXED else torch.float64


# ---------------------------------------------------------------------------
# calls (same names as the C ABI)
# ---------------------------------------------------------------------------

def lisa_version():
    return load().lisa_version()


def lisa_t_hyb_from_f(f_hyb, mc_s, tc):
    return load().lisa_t_hyb_from_f(float(f_hyb), float(mc_s), float(tc))


def lisa_orbits(orbit, grid, R=None, T=None, nhat=None, stream=None):
    import torch
    g = _grid(grid)
    o = _orb(orbit)
    rc = load().lisa_orbits(C.byref(o), g, _ptr(R, torch.float64, 9 * g.n, "R"), _ptr(T, torch.float64, 6 * g.n, "T"),
                            _ptr(nhat, torch.float64, 18 * g.n, "nhat"), _stream(stream))
    _check(rc, "lisa_orbits")


def lisa_links_full(orbit, sky, h_grid, hp, hc, precision, y_grid, y, stream=None):
    hg, yg = _grid(h_grid), _grid(y_grid)
    dt = _rdtype(precision)
    o, s = _orb(orbit), _sky(sky)
    rc = load().lisa_links_full(C.byref(o), C.byref(s), hg, _ptr(hp, dt, hg.n, "hp"), _ptr(hc, dt, hg.n, "hc"),
                                precision, yg, _ptr(y, dt, 6 * yg.n, "y"), _stream(stream))
    _check(rc, "lisa_links_full")


def lisa_tdi(orbit, y_grid, y, precision, tdi_gen, delay_mode, channels, out_grid, xyz, stream=None):
    yg, og = _grid(y_grid), _grid(out_grid)
    dt = _rdtype(precision)
    o = _orb(orbit)
    rc = load().lisa_tdi(C.byref(o), yg, _ptr(y, dt, 6 * yg.n, "y"), precision, tdi_gen, delay_mode, channels, og,
                         _ptr(xyz, dt, 3 * og.n, "xyz"), _stream(stream))
    _check(rc, "lisa_tdi")


def lisa_response_full(orbit, sky, h_grid, hp, hc, precision, tdi_gen, channels, out_grid, xyz, stream=None):
    hg, og = _grid(h_grid), _grid(out_grid)
    dt = _rdtype(precision)
    o, s = _orb(orbit), _sky(sky)
    rc = load().lisa_response_full(C.byref(o), C.byref(s), hg, _ptr(hp, dt, hg.n, "hp"), _ptr(hc, dt, hg.n, "hc"),
                                   precision, tdi_gen, channels, og, _ptr(xyz, dt, 3 * og.n, "xyz"), _stream(stream))
    _check(rc, "lisa_response_full")


def lisa_links_lfa(orbit, sky, h_grid, hp, hc, precision, tdi_gen, lfa_kind, out_grid, z, stream=None):
    hg, og = _grid(h_grid), _grid(out_grid)
    dt = _rdtype(precision)
    o, s = _orb(orbit), _sky(sky)
    rc = load().lisa_links_lfa(C.byref(o), C.byref(s), hg, _ptr(hp, dt, hg.n, "hp"), _ptr(hc, dt, hg.n, "hc"),
                               precision, tdi_gen, lfa_kind, og, _ptr(z, dt, 6 * og.n, "z"), _stream(stream))
    _check(rc, "lisa_links_lfa")


def lisa_links_lfa_own(orbit, sky, h_grid, hp, hc, precision, lfa_kind, out_grid, y, stream=None):
    hg, og = _grid(h_grid), _grid(out_grid)
    dt = _rdtype(precision)
    o, s = _orb(orbit), _sky(sky)
    rc = load().lisa_links_lfa_own(C.byref(o), C.byref(s), hg, _ptr(hp, dt, hg.n, "hp"), _ptr(hc, dt, hg.n, "hc"),
                                   precision, lfa_kind, og, _ptr(y, dt, 6 * og.n, "y"), _stream(stream))
    _check(rc, "lisa_links_lfa_own")


def lisa_tdi_lfa(orbit, z_grid, z, precision, tdi_gen, lfa_kind, channels, xyz, stream=None):
    zg = _grid(z_grid)
    dt = _rdtype(precision)
    o = _orb(orbit)
    rc = load().lisa_tdi_lfa(C.byref(o), zg, _ptr(z, dt, 6 * zg.n, "z"), precision, tdi_gen, lfa_kind, channels,
                             _ptr(xyz, dt, 3 * zg.n, "xyz"), _stream(stream))
    _check(rc, "lisa_tdi_lfa")


def lisa_response_lfa(orbit, sky, h_grid, hp, hc, precision, tdi_gen, lfa_kind, channels, out_grid, xyz, stream=None):
    hg, og = _grid(h_grid), _grid(out_grid)
    dt = _rdtype(precision)
    o, s = _orb(orbit), _sky(sky)
    rc = load().lisa_response_lfa(C.byref(o), C.byref(s), hg, _ptr(hp, dt, hg.n, "hp"), _ptr(hc, dt, hg.n, "hc"),
                                  precision, tdi_gen, lfa_kind, channels, og, _ptr(xyz, dt, 3 * og.n, "xyz"),
                                  _stream(stream))
    _check(rc, "lisa_response_lfa")


def lisa_response_hybrid(orbit, sky, h_grid, hp, hc, precision, tdi_gen, lfa_kind, channels, t_hyb, T_win, sigma,
                         out_grid, xyz, stream=None):
    hg, og = _grid(h_grid), _grid(out_grid)
    dt = _rdtype(precision)
    o, s = _orb(orbit), _sky(sky)
    rc = load().lisa_response_hybrid(C.byref(o), C.byref(s), hg, _ptr(hp, dt, hg.n, "hp"), _ptr(hc, dt, hg.n, "hc"),
                                     precision, tdi_gen, lfa_kind, channels, float(t_hyb), float(T_win), float(sigma),
                                     og, _ptr(xyz, dt, 3 * og.n, "xyz"), _stream(stream))
    _check(rc, "lisa_response_hybrid")


def lisa_response_hybrid_host(orbit, sky, grid, hp, hc, precision, tdi_gen, lfa_kind, channels, t_hyb, T_win, sigma,
                              xyz, stream=None):
    """Hybrid response of host series (CPU tensors, page-locked for overlap);
    the results are in xyz once `stream` has completed."""
    g = _grid(grid)
    dt = _rdtype(precision)
    o, s = _orb(orbit), _sky(sky)
    rc = load().lisa_response_hybrid_host(C.byref(o), C.byref(s), g, _host_ptr(hp, dt, g.n, "hp"),
                                          _host_ptr(hc, dt, g.n, "hc"), precision, tdi_gen, lfa_kind, channels,
                                          float(t_hyb), float(T_win), float(sigma), _host_ptr(xyz, dt, 3 * g.n, "xyz"),
                                          _stream(stream))
    _check(rc, "lisa_response_hybrid_host")


def lisa_psd_aet(f0, df, nf, tdi_gen, L_m, t_obs_years, galaxy, psd, stream=None):
    """S^{A,E} and S^T at f0 + k df into psd (CUDA float64 [2][nf])."""
    import torch
    rc = load().lisa_psd_aet(float(f0), float(df), int(nf), tdi_gen, float(L_m), float(t_obs_years), int(galaxy),
                             _ptr(psd, torch.float64, 2 * int(nf), "psd"), _stream(stream))
    _check(rc, "lisa_psd_aet")


def lisa_chirp_ringdown(draws, grid, precision, hp, hc, stream=None):
    """Synthetic chirp + ringdown of each draw (dicts with keys mc_s, q, dist_m,
    iota, phi_c, tc and optionally e0, f_cut, m_final_frac, a_final) on grid,
    into CUDA tensors hp, hc of shape [len(draws)][n] (float64 for F64, float32
    for MIXED)."""
    arr = (lisa_chirp * max(len(draws), 1))()
    for k, d in enumerate(draws):
        arr[k] = lisa_chirp(float(d["mc_s"]), float(d["q"]), float(d["dist_m"]), float(d["iota"]),
                            float(d["phi_c"]), float(d["tc"]), float(d.get("e0", 0.0)), float(d.get("f_cut", 0.0)),
                            float(d.get("m_final_frac", 0.95)), float(d.get("a_final", 0.7)))
    g = _grid(grid)
    dt = _rdtype(precision)
    rc = load().lisa_chirp_ringdown(arr, len(draws), g, precision, _ptr(hp, dt, len(draws) * g.n, "hp"),
                                    _ptr(hc, dt, len(draws) * g.n, "hc"), _stream(stream))
    _check(rc, "lisa_chirp_ringdown")


def lisa_fft_length(n):
    return int(load().lisa_fft_length(int(n)))


def lisa_noise_weights_aet(grid, nfft, tdi_gen, L_m, t_obs_years, galaxy, f_min, f_max, w, stream=None):
    """Inner-product weights 4 df / S on the rfft bins of grid zero-padded to
    nfft samples (0: none) into w (CUDA float64 [2][nfft/2+1])."""
    import torch
    g = _grid(grid)
    m = int(nfft) or g.n
    rc = load().lisa_noise_weights_aet(g, m, tdi_gen, float(L_m), float(t_obs_years), int(galaxy), float(f_min),
                                       float(f_max), _ptr(w, torch.float64, 2 * (m // 2 + 1), "w"), _stream(stream))
    _check(rc, "lisa_noise_weights_aet")


def lisa_inner_aet(grid, nfft, x, y, precision, w, out, stream=None):
    """<x|y>, <x|x>, <y|y> per channel into out (CUDA float64 [9] or [3][3])."""
    import torch
    g = _grid(grid)
    m = int(nfft) or g.n
    dt = _rdtype(precision)
    rc = load().lisa_inner_aet(g, m, _ptr(x, dt, 3 * g.n, "x"), _ptr(y, dt, 3 * g.n, "y"), precision,
                               _ptr(w, torch.float64, 2 * (m // 2 + 1), "w"), _ptr(out, torch.float64, 9, "out"),
                               _stream(stream))
    _check(rc, "lisa_inner_aet")


def lisa_profile_enable(enable=True):
    _check(load().lisa_profile_enable(1 if enable else 0), "lisa_profile_enable")


def lisa_profile_query(name=None):
    """(total device ms, launches) of recorded launches whose kernel name contains `name`."""
    ms, cnt = C.c_double(), C.c_int64()
    _check(load().lisa_profile_query(name.encode() if name else None, C.byref(ms), C.byref(cnt)),
           "lisa_profile_query")
    return ms.value, cnt.value


def lisa_launch_count():
    return load().lisa_launch_count()


def lisa_peak_fma(kind, iters, blocks_per_sm=8, stream=None, reps=5):
    """Measured fused multiply-add throughput (TFLOP/s) of the FP64 (kind 0),
    FP32 (kind 1) or packed-pair FP32 (kind 2) pipe: the best of `reps`
    launches after one warm-up, each timed with CUDA events on `stream`."""
    import torch
    nb = C.c_int64()
    _check(load().lisa_peak_fma_blocks(int(blocks_per_sm), C.byref(nb)), "lisa_peak_fma_blocks")
    sink = torch.empty(nb.value * 256, device="cuda", dtype=torch.float64 if kind == 0 else torch.float32)
    st = torch.cuda.current_stream() if stream is None else stream
    flop = C.c_double()
    best = None
    for r in range(reps + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        _check(load().lisa_peak_fma(int(kind), int(iters), int(blocks_per_sm), C.c_void_p(sink.data_ptr()),
                                    C.byref(flop), C.c_void_p(st.cuda_stream)), "lisa_peak_fma")
        b.record(st)
        b.synchronize()
        if r > 0:
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
    return flop.value / (best / 1e3) / 1e12, best


def lisa_device_status(reset=True):
    """Device status word (bit 0: a bounded device wait timed out); raises
    LisaError(LISA_ETIMEOUT) if it was set."""
    st = C.c_uint()
    _check(load().lisa_device_status(C.byref(st), 1 if reset else 0), "lisa_device_status")
    return st.value


def lisa_selftest_wait_timeout(stream=None):
    """Launch the bounded-wait self-test (a wait that times out after about a
    second and flags the device status word)."""
    _check(load().lisa_selftest_wait_timeout(_stream(stream)), "lisa_selftest_wait_timeout")


def lisa_response_hybrid_static(orbit, sky, h_grid, hp, hc, precision, tdi_gen, lfa_kind, channels, t_hyb, T_win,
                                sigma, out_grid, xyz, stream=None):
    """lisa_response_hybrid with its scratch in the library's fixed device
    array instead of allocated memory (see include/lisa.h)."""
    hg, og = _grid(h_grid), _grid(out_grid)
    dt = _rdtype(precision)
    o, s = _orb(orbit), _sky(sky)
    rc = load().lisa_response_hybrid_static(C.byref(o), C.byref(s), hg, _ptr(hp, dt, hg.n, "hp"),
                                            _ptr(hc, dt, hg.n, "hc"), precision, tdi_gen, lfa_kind, channels,
                                            float(t_hyb), float(T_win), float(sigma), og,
                                            _ptr(xyz, dt, 3 * og.n, "xyz"), _stream(stream))
    _check(rc, "lisa_response_hybrid_static")


class LisaPlan:
    """Batched hybrid plan (lisa_plan_*).  `sources` is a list of dicts with
    keys grid, hp, hc, sky, t_hyb, out (and optionally T_win, sigma); the
    tensors are kept alive for the plan's lifetime."""

    def __init__(self, orbit, sources, precision=MIXED, tdi_gen=TDI20, lfa_kind=LFA_UNEQUAL, channels=AET):
        import torch
        self._keep = []
        arr = (lisa_source * len(sources))()
        for k, s in enumerate(sources):
            g = _grid(s["grid"])
            dt = _rdtype(precision)
            arr[k].grid = g
            arr[k].hp = _ptr(s["hp"], dt, g.n, "hp")
            arr[k].hc = _ptr(s["hc"], dt, g.n, "hc")
            arr[k].sky = _sky(s["sky"])
            arr[k].t_hyb = float(s["t_hyb"])
            arr[k].T_win = float(s.get("T_win", 0.0))
            arr[k].sigma = float(s.get("sigma", 0.0))
            arr[k].out = _ptr(s["out"], dt, 3 * g.n, "out")
            self._keep += [s["hp"], s["hc"], s["out"]]
        self._orbit = _orb(orbit)
        h = C.c_void_p()
        _check(load().lisa_plan_create(C.byref(h), C.byref(self._orbit), precision, tdi_gen, lfa_kind, channels, arr,
                                       len(sources)), "lisa_plan_create")
        self.handle = h

    def execute(self, stream=None):
        _check(load().lisa_plan_execute(self.handle, _stream(stream)), "lisa_plan_execute")

    def capture_graph(self, stream):
        _check(load().lisa_plan_capture_graph(self.handle, _stream(stream)), "lisa_plan_capture_graph")

    def replay(self, stream=None):
        _check(load().lisa_plan_replay(self.handle, _stream(stream)), "lisa_plan_replay")

    def set_launch(self, ctas_per_sm, tiles_per_item):
        _check(load().lisa_plan_set_launch(self.handle, ctas_per_sm, tiles_per_item), "lisa_plan_set_launch")

    def autotune(self, stream=None):
        r = lisa_tune_result()
        _check(load().lisa_plan_autotune(self.handle, _stream(stream), C.byref(r)), "lisa_plan_autotune")
        return {"ctas_per_sm": r.ctas_per_sm, "tiles_per_item": r.tiles_per_item, "ms": r.ms}

    def info(self):
        a, b, c, d = C.c_int64(), C.c_int64(), C.c_int(), C.c_int()
        _check(load().lisa_plan_info(self.handle, C.byref(a), C.byref(b), C.byref(c), C.byref(d)), "lisa_plan_info")
        return {"total_samples": a.value, "total_tiles": b.value, "ctas_per_sm": c.value, "tiles_per_item": d.value}

    def close(self):
        if getattr(self, "handle", None):
            load().lisa_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LisaCorrector:
    """The learned LFA-link corrector (lisa_corrector_*).  `params` is a flat
    FP32 vector (numpy) or None for the library's seeded initialisation."""

    def __init__(self, params=None, seed=0):
        import numpy as np
        lib = load()
        self.n_params = lib.lisa_corrector_num_params()
        self.n_features = lib.lisa_corrector_num_features()
        h = C.c_void_p()
        if params is None:
            rc = lib.lisa_corrector_create(C.byref(h), None, self.n_params, int(seed))
        else:
            p = np.ascontiguousarray(params, dtype=np.float32)
            if p.size != self.n_params:
                raise ValueError("need %d parameters (got %d)" % (self.n_params, p.size))
            rc = lib.lisa_corrector_create(C.byref(h), p.ctypes.data_as(C.c_void_p), self.n_params, int(seed))
        _check(rc, "lisa_corrector_create")
        self.handle = h

    def configure(self, f_lo=1e-4, f_hi=2e-2, spot_every=64, spot_tol=0.05):
        _check(load().lisa_corrector_configure(self.handle, float(f_lo), float(f_hi), int(spot_every),
                                               float(spot_tol)), "lisa_corrector_configure")

    def get_state(self):
        import numpy as np
        p, m, v = (np.empty(self.n_params, dtype=np.float32) for _ in range(3))
        step = C.c_int64()
        _check(load().lisa_corrector_get_state(self.handle, p.ctypes.data_as(C.c_void_p), m.ctypes.data_as(C.c_void_p),
                                               v.ctypes.data_as(C.c_void_p), C.byref(step), self.n_params),
               "lisa_corrector_get_state")
        return {"params": p, "adam_m": m, "adam_v": v, "step": step.value}

    def set_state(self, state):
        import numpy as np
        arrs = [np.ascontiguousarray(state[k], dtype=np.float32) if state.get(k) is not None else None
                for k in ("params", "adam_m", "adam_v")]
        ptrs = [a.ctypes.data_as(C.c_void_p) if a is not None else None for a in arrs]
        _check(load().lisa_corrector_set_state(self.handle, ptrs[0], ptrs[1], ptrs[2], int(state.get("step", 0)),
                                               self.n_params), "lisa_corrector_set_state")

    def save(self, path):
        """Checkpoint (parameters, Adam moments, step) as .npz."""
        import numpy as np
        st = self.get_state()
        np.savez(path, params=st["params"], adam_m=st["adam_m"], adam_v=st["adam_v"], step=np.int64(st["step"]))

    def load_checkpoint(self, path):
        import numpy as np
        with np.load(path) as d:
            self.set_state({"params": d["params"], "adam_m": d["adam_m"], "adam_v": d["adam_v"],
                            "step": int(d["step"])})

    def forward(self, feats, out, stream=None):
        import torch
        M = feats.shape[0]
        _check(load().lisa_corrector_forward(self.handle, _ptr(feats, torch.float32, M * 48, "feats"), M,
                                             _ptr(out, torch.float32, M * 6, "out"), _stream(stream)),
               "lisa_corrector_forward")

    def gradient(self, feats, target, grad, loss=None, batch=0, seed=0, stream=None):
        import torch
        n = feats.shape[0]
        _check(load().lisa_corrector_gradient(self.handle, _ptr(feats, torch.float32, n * 48, "feats"),
                                              _ptr(target, torch.float32, n * 6, "target"), n, int(batch), int(seed),
                                              _ptr(grad, torch.float32, self.n_params, "grad"),
                                              _ptr(loss, torch.float32, 1, "loss"), _stream(stream)),
               "lisa_corrector_gradient")

    def adam_step(self, grad, lr, stream=None):
        import torch
        _check(load().lisa_corrector_adam_step(self.handle, _ptr(grad, torch.float32, self.n_params, "grad"),
                                               float(lr), _stream(stream)), "lisa_corrector_adam_step")

    def train(self, feats, target, steps, batch, lr_max=3e-3, lr_min=3e-5, seed=0, losses=None, stream=None):
        import torch
        n = feats.shape[0]
        _check(load().lisa_corrector_train(self.handle, _ptr(feats, torch.float32, n * 48, "feats"),
                                           _ptr(target, torch.float32, n * 6, "target"), n, int(steps), int(batch),
                                           float(lr_max), float(lr_min), int(seed),
                                           _ptr(losses, torch.float32, int(steps), "losses"), _stream(stream)),
               "lisa_corrector_train")

    def links(self, orbit, sky, h_grid, hp, hc, out_grid, y, stream=None):
        import torch
        hg, og = _grid(h_grid), _grid(out_grid)
        o, s = _orb(orbit), _sky(sky)
        _check(load().lisa_corrector_links(self.handle, C.byref(o), C.byref(s), hg,
                                           _ptr(hp, torch.float32, hg.n, "hp"), _ptr(hc, torch.float32, hg.n, "hc"),
                                           og, _ptr(y, torch.float32, 6 * og.n, "y"), _stream(stream)),
               "lisa_corrector_links")

    def hybrid(self, orbit, sky, h_grid, hp, hc, tdi_gen, channels, t_hyb, T_win, sigma, out_grid, xyz, stream=None,
               t_lo=-math.inf):
        """Corrected hybrid: plain LFA for t <= t_lo, corrected links and the
        full TDI combine between t_lo and t_hyb, full response after t_hyb
        (t_lo = -inf: no plain-LFA zone)."""
        import torch
        hg, og = _grid(h_grid), _grid(out_grid)
        o, s = _orb(orbit), _sky(sky)
        _check(load().lisa_response_hybrid_corrected(self.handle, C.byref(o), C.byref(s), hg,
                                                     _ptr(hp, torch.float32, hg.n, "hp"),
                                                     _ptr(hc, torch.float32, hg.n, "hc"), tdi_gen, channels,
                                                     float(t_lo), float(t_hyb), float(T_win), float(sigma), og,
                                                     _ptr(xyz, torch.float32, 3 * og.n, "xyz"), _stream(stream)),
               "lisa_response_hybrid_corrected")

    def report(self, reset=True):
        """Counters and status (LISA_ECORRECTOR if a spot check failed since the last reset)."""
        a, b, c, d = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
        e = C.c_float()
        rc = load().lisa_corrector_report(self.handle, C.byref(a), C.byref(b), C.byref(c), C.byref(d), C.byref(e),
                                          1 if reset else 0)
        out = {"spot_tiles": a.value, "spot_failed": b.value, "band_tiles": c.value, "fallback_tiles": d.value,
               "max_spot_err": e.value, "status": rc}
        if rc not in (LISA_OK, LISA_ECORRECTOR):
            _check(rc, "lisa_corrector_report")
        return out

    def close(self):
        if getattr(self, "handle", None):
            load().lisa_corrector_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lisa_corrector_features(orbit, sky, grid, z, y_full, z_ref, f_lo, f_hi, feats, scale, ybase=None, target=None,
                            stream=None):
    import torch
    g = _grid(grid)
    o, s = _orb(orbit), _sky(sky)
    _check(load().lisa_corrector_features(C.byref(o), C.byref(s), g, _ptr(z, torch.float32, 6 * g.n, "z"),
                                          _ptr(y_full, torch.float64, 6 * g.n, "y_full"),
                                          _ptr(z_ref, torch.float64, 6 * g.n, "z_ref"), float(f_lo), float(f_hi),
                                          _ptr(feats, torch.float32, 48 * g.n, "feats"),
                                          _ptr(scale, torch.float32, g.n, "scale"),
                                          _ptr(ybase, torch.float32, 6 * g.n, "ybase"),
                                          _ptr(target, torch.float32, 6 * g.n, "target"), _stream(stream)),
           "lisa_corrector_features")
