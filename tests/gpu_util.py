"""Helpers shared by the GPU parity tests (no arithmetic of the method here)."""
import math

import numpy as np

import synth

# All-FP64 GPU against the FP64 oracle.  The two use different but equivalent
# operation orders (FMA contraction, Lagrange weights as running products,
# orbit geometry from per-segment polynomials instead of exact evaluation at
# rounded absolute times); the LFA's 5-point second differences amplify the
# resulting rounding by up to 64/(omega dt)^2 at the lowest frequencies.
F64_TOL = 5e-12

# Orbits used by the parity cases: first-order Kepler (config 1) and exact
# Keplerian ellipses with 1% peak-to-peak arm flexing (config 2).
ORBITS = {
    "kepler1": dict(kind=0, delay=0),
    "kepler2_flex": dict(kind=1, delay=0, kepler_tilt=1.01),
    "analytic": dict(kind=0, delay=1, flex_scale=2.0, xi0=0.3),
    "equal": dict(kind=0, delay=2),
    "linear": dict(kind=0, delay=3, t_ref=2.0e7, lin_T0=(8.3, 8.31, 8.35, 8.33, 8.29, 8.30),
                   lin_Tdot=(1e-7, -2e-7, 3e-7, 1e-7, -1e-7, 2e-7)),
    "static": dict(kind=2, delay=0, t_static=2.2e7),
}


def orbit_pair(name):
    import oracle
    import paper_2505_09600_gb300 as L
    kw = ORBITS[name]
    return oracle.Orbit(**kw), L.Orbit(**kw)


def rel_err(got, want, signal=False):
    """Per channel: max |got - want| / max |want|.

    With signal=True (used for A, E, T) every channel is divided by the largest
    channel maximum instead: T is a near-cancelling sum of X, Y, Z (and is
    identically zero for equal arms in the LFA), so its own maximum is not a
    meaningful scale for errors inherited from X, Y, Z."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    scale = np.abs(want).max(axis=-1)
    if signal:
        scale = np.full_like(scale, scale.max())
    scale = np.where(scale > 0, scale, 1.0)
    return np.abs(got - want).max(axis=-1) / scale


def rel_err_own(got, want):
    """Per channel on its own scale (the error measure per channel):
    max |got - want| / max |want| of that channel."""
    return rel_err(got, want, signal=False)


def check_aet(got, want, tol_big, tol_T_own, equal_arms=False):
    """A, E, T against the oracle: every channel within tol_big of the
    largest channel maximum, A and E within tol_big of their own maxima, and
    T within tol_T_own of its own maximum (for equal-arm LFA outputs, where T
    vanishes identically, T is judged on the largest channel only).  Returns
    (largest-channel errors, own-scale errors)."""
    big = rel_err(got, want, signal=True)
    own = rel_err_own(got, want)
    tb = np.broadcast_to(np.asarray(tol_big, dtype=np.float64), (3,))
    assert np.all(big <= tb), ("largest-channel scale", big, tb)
    assert np.all(own[:2] <= tb[:2]), ("own scale A, E", own, tb)
    if not equal_arms:
        assert own[2] <= tol_T_own, ("own scale T", own, tol_T_own)
    return big, own


def to_dev(a, precision):
    import torch
    dt = torch.float32 if precision == 1 else torch.float64
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda").to(dt).contiguous()


def empty(shape, precision):
    import torch
    dt = torch.float32 if precision == 1 else torch.float64
    return torch.full(shape, float("nan"), device="cuda", dtype=dt)


def host_inputs(src, precision):
    """h as the GPU sees it, returned as FP64 for the oracle (the oracle is fed
    exactly the values the kernel reads)."""
    if precision == 1:
        return src.hp.astype(np.float32).astype(np.float64), src.hc.astype(np.float32).astype(np.float64)
    return src.hp, src.hc


def sky_of(src):
    return (src.beta, src.lam, src.psi)
