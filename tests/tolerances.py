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
