"""Per-channel tolerances of the mixed-precision (FP32 arithmetic, FP64 times)
forms against the FP64 oracle: max |gpu - oracle| / max |oracle| per channel.

PROVISIONAL: proposed values, to be replaced by the frozen ones after the
first measurement on the config-2 workload and before any tuning.
"""
MIXED_TOL = {
    "links": [1e-5] * 6,
    "full15": {"xyz": [1e-5] * 3, "aet": [1e-5, 1e-5, 1e-4]},
    "full20": {"xyz": [1e-5] * 3, "aet": [1e-5, 1e-5, 1e-4]},
    "lfa15": {"xyz": [1e-5] * 3, "aet": [1e-5, 1e-5, 1e-4]},
    "lfa20": {"xyz": [1e-5] * 3, "aet": [1e-5, 1e-5, 1e-4]},
    "hybrid20": {"xyz": [1e-5] * 3, "aet": [1e-5, 1e-5, 1e-4]},
}
