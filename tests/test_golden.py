"""Numbers the paper prints, reproduced through the oracle (fixtures in tests/golden/)."""
import math
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    out = {}
    with open(os.path.join(HERE, "golden", "paper_numbers.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, val, tol = line.split()[:3]
                out[name] = (float(val), float(tol))
    return out


def _lfa_fraction(oracle_mod, f_hyb, f_min, f_max=0.05, mc_s=1e6 * 4.925490947641267e-6, tc=5e7):
    # fraction of the time between f_min and f_max spent below f_hyb, from t_Hyb(f) (Eq. thyb)
    t = lambda f: oracle_mod.t_hyb(f, mc_s, tc)
    return (t(f_hyb) - t(f_min)) / (t(f_max) - t(f_min))


def test_lfa_fraction_values(oracle_mod):
    g = _golden()
    for name, (fh, fmin) in {"R_fhyb_3e-4_fmin_1e-4": (3e-4, 1e-4), "R_fhyb_3e-4_fmin_0.8e-4": (3e-4, 0.8e-4),
                             "R_fhyb_8e-4_fmin_0.8e-4": (8e-4, 0.8e-4)}.items():
        want, tol = g[name]
        got = _lfa_fraction(oracle_mod, fh, fmin)
        assert abs(got / want - 1) < tol, (name, got)


def test_reference_frequencies_and_omega(oracle_mod):
    g = _golden()
    c = oracle_mod.C_LIGHT
    assert abs(c / (2 * math.pi * 2.5e9) / g["f_c_over_2piL"][0] - 1) < g["f_c_over_2piL"][1]
    assert abs(c / (2 * math.pi * oracle_mod.AU) / g["f_c_over_2piR"][0] - 1) < g["f_c_over_2piR"][1]
    # Omega from the oracle's orbit: the constellation centre advances by 2 pi per year
    import numpy as np
    o = oracle_mod.Orbit()
    p0 = sum(oracle_mod.position(o, s, 0.0) for s in range(3))
    p1 = sum(oracle_mod.position(o, s, 1000.0) for s in range(3))
    w = math.atan2(p1[1], p1[0]) - math.atan2(p0[1], p0[0])
    assert abs(w / 1000.0 / g["omega"][0] - 1) < g["omega"][1]
