"""Evidence for the precision split of the mixed form (CPU only)."""
import numpy as np

import synth


def test_fp32_absolute_time_is_not_enough(oracle_mod):
    """Absolute times near 2e7 s rounded to FP32 (ulp 2 s) move the retarded
    times by up to a second, which changes the links by far more than the
    mixed-precision tolerance (~1e-5); the kernels therefore keep tile-centre
    times and delays in FP64 and only the in-tile offsets in FP32."""
    s = synth.cfg2_small(n=20000)
    oo = oracle_mod.Orbit(kind=oracle_mod.KEPLER2, kepler_tilt=1.01)
    sky = (s.beta, s.lam, s.psi)
    idx = np.arange(15000, 19000, 97)
    exact = oracle_mod.links_full(oo, sky, s.grid, s.hp, s.hc, s.grid, idx)
    t32 = np.float32(s.t0 + idx * s.dt).astype(np.float64)
    shifted = np.stack([oracle_mod.links_full(oo, sky, s.grid, s.hp, s.hc, (t32[k], s.dt, 1))[:, 0]
                        for k in range(idx.size)], axis=1)
    err = np.abs(shifted - exact).max() / np.abs(exact).max()
    assert err > 1e-3, err
