"""Training-set assembly for the LFA-link corrector: calls of the C ABI only
(the full links, the LFA links and the features all run in liblisa's
kernels; torch provides the device buffers).

Each source contributes the samples that are at least `edge_margin` samples
away from both ends of its grid: nearer the ends the retarded times
t - k.R/c (|k.R/c| <= 1 AU/c ~ 500 s) and their 32-point stencils reach
outside the sampled waveform, where h is zero by convention and neither link
form is meaningful.  The library itself takes the full links there (at most
1 AU/c + 2 T_max + 20 dt from either end, T_max < 50 s for the orbits here).
"""
from __future__ import annotations

import math

from . import native as N


AU_LIGHT_S = 1.495978707e11 / 299792458.0


def edge_margin(dt):
    """Samples near either grid end excluded from training and from errors."""
    return int(math.ceil((AU_LIGHT_S + 100.0 + 20.0 * dt) / dt)) + 4


def training_rows(sources):
    return sum(max(0, s["grid"][2] - 2 * edge_margin(s["grid"][1])) for s in sources)


def training_set(orbit, sources, stream=None):
    """Features [N][48] and targets [N][6] (device, FP32) of the corrector.

    `sources`: dicts with grid (t0, dt, n), sky (beta, lambda, psi) and the
    polarisations as device tensors hp32/hc32 (FP32, what the mixed-precision
    response reads) and hp64/hc64 (FP64).  Features come from the mixed LFA
    links (as at inference); targets from the FP64 full and LFA links."""
    import torch
    rows = training_rows(sources)
    feats = torch.empty((rows, 48), dtype=torch.float32, device="cuda")
    target = torch.empty((rows, 6), dtype=torch.float32, device="cuda")
    r = 0
    for s in sources:
        g = s["grid"]
        n = int(g[2])
        m = edge_margin(g[1])
        k = n - 2 * m
        if k <= 0:
            continue
        z = torch.empty((6, n), dtype=torch.float32, device="cuda")
        zr = torch.empty((6, n), dtype=torch.float64, device="cuda")
        y = torch.empty((6, n), dtype=torch.float64, device="cuda")
        N.lisa_links_lfa_own(orbit, s["sky"], g, s["hp32"], s["hc32"], N.MIXED, N.LFA_UNEQUAL, g, z, stream)
        N.lisa_links_lfa_own(orbit, s["sky"], g, s["hp64"], s["hc64"], N.F64, N.LFA_UNEQUAL, g, zr, stream)
        N.lisa_links_full(orbit, s["sky"], g, s["hp64"], s["hc64"], N.F64, g, y, stream)
        f = torch.empty((n, 48), dtype=torch.float32, device="cuda")
        sc = torch.empty(n, dtype=torch.float32, device="cuda")
        tg = torch.empty((n, 6), dtype=torch.float32, device="cuda")
        N.lisa_corrector_features(orbit, s["sky"], g, z, y, zr, 0.0, math.inf, f, sc, None, tg, stream)
        feats[r:r + k].copy_(f[m:n - m])
        target[r:r + k].copy_(tg[m:n - m])
        r += k
    return feats, target
