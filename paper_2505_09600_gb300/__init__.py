"""GB300 (sm_103a) time-domain LISA response: full response, low-frequency
approximation and their hybrid (arXiv:2505.09600), as hand-written CUDA
kernels behind a C ABI (include/lisa.h, liblisa.so).

The Python side only marshals arguments (``native``); build the library with
``paper_2505_09600_gb300.build.build()``.
"""
from .native import *  # noqa: F401,F403
from .native import Orbit, LisaError, LisaPlan, LisaCorrector, load, exported_symbols  # noqa: F401

__all__ = [n for n in dir() if n.startswith("lisa_")] + [
    "Orbit", "LisaError", "LisaPlan", "LisaCorrector", "load", "exported_symbols",
    "ORB_KEPLER1", "ORB_KEPLER2", "ORB_STATIC", "DELAY_LIGHTTIME", "DELAY_ANALYTIC", "DELAY_EQUAL",
    "DELAY_LINEAR", "F64", "MIXED", "DF", "TDI15", "TDI20", "XYZ", "AET", "FROZEN", "NESTED", "LFA_UNEQUAL",
    "LFA_EQUAL", "LFA_BACKWARD", "LFA_FORWARD", "LFA_NLO", "LFA_STRAIN"]
