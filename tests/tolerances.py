"""Per-channel tolerances of the mixed-precision forms (FP32 arithmetic,
FP64 tile-centre times) against the FP64 oracle fed the same FP32 inputs.

Error measure: max |gpu - oracle| / max |oracle| per channel for links, z and
X, Y, Z; for A, E, T the divisor is the largest of the three channel maxima
(see gpu_util.rel_err).

FROZEN values: three times the largest error measured on the first run of
every mixed form on the config-2-shaped source (chirp + ringdown Mc=1e6 q=3,
20,000 samples at 5 s ending after the merger, flexing Kepler orbits), taken
before any performance tuning, rounded up.  Measured then (per channel, own
maximum): links <= 2.0e-5; full X,Y,Z <= 5.7e-5 (the weakest channel), A,E
<= 1.3e-5; LFA X,Y,Z <= 4.8e-6, A,E <= 2.1e-6; hybrid X,Y,Z <= 5.7e-5, A,E
<= 9.1e-6.  The limiting error is FP32 rounding of the Lagrange weights
(~60 chained products, ~5e-7 relative per interpolated value) divided by the
cancellation of the two retarded samples in a link (omega (delta_s - delta_r)).
"""
MIXED_TOL = {
    "links": [6e-5] * 6,
    "z": [2e-5] * 6,
    "full15": {"xyz": [2e-4] * 3, "aet": [4e-5] * 3},
    "full20": {"xyz": [2e-4] * 3, "aet": [4e-5] * 3},
    "lfa15": {"xyz": [1.5e-5] * 3, "aet": [1e-5] * 3},
    "lfa20": {"xyz": [1.5e-5] * 3, "aet": [1e-5] * 3},
    "hybrid15": {"xyz": [2e-4] * 3, "aet": [3e-5] * 3},
    "hybrid20": {"xyz": [2e-4] * 3, "aet": [3e-5] * 3},
}

# Own-scale tolerances of the T channel (err_T = max |T_gpu - T_oracle| /
# max |T_oracle|, the definition of the error per channel), FROZEN at three
# times the largest error measured on the kernels as they stood before the
# differenced LFA form was written (same config-2-shaped source, flexing
# orbits, all unequal-arm LFA kinds and both TDI generations), rounded up.
# A and E keep the tolerances above on their own scale too (their own maxima
# are within a factor two of the largest channel's).  T is a near-cancelling
# sum of X, Y, Z: its own maximum is ~1e-2 of A's here, so its own-scale
# error is larger by that factor.  Measured (own scale): full T <= 2.1e-4,
# LFA T <= 2.0e-4, hybrid T <= 1.6e-4 (mixed); FP64 T <= 2.7e-11 (the FP64
# A and E stay within F64_TOL on their own scale, <= 7.9e-13).  For the
# equal-arm LFA, T vanishes identically (pin L3) and has no scale of its own:
# it is judged on the largest channel as before.
T_OWN_TOL = {
    "mixed": {"full": 7e-4, "lfa": 7e-4, "hybrid": 5e-4},
    "f64": 1e-10,
}

