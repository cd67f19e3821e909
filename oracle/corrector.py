"""FP64 CPU reference of the corrector's inputs and targets (test
infrastructure only: imported by tests/ and nothing in the library).

The corrector is not part of the paper.  What it is fed follows from the
paper's LFA single link (Sec. III): the LFA link at its own time,
    z_l(t) = -(T_l/2) [xi+ hdot+ + xix hdotx](tau_l),
    tau_l = t - T_l/2 - k.(R_s + R_r)/(2c),
is the central (midpoint) expansion of the full link (Sec. II)
    y_l(t) = [H(t - delta_s) - H(t - delta_r)] / (2 (1 - k.n_l)),
whose expansion gives
    y_l - z_l = eps_l z_l + (1 - k.n_l)^2 T_l^2/24 z_l'' + O(T^4),
    eps_l = k.(R_s(t) - R_s(t - T_l)) / (c T_l (1 - k.n_l)):
with the positions of the full formula taken at the reception time t,
delta_s - delta_r = T_l (1 - k.n_l) (1 + eps_l) exactly (n_l is the
light-time link vector), a frequency-independent O(v/c) term.  The base link
is z_l (1 + eps_l).

Features of sample i (written out plainly, one sample at a time):
  q_k,l = Tbar^k * D_k z_l(i), with the textbook 5-point central stencils
      D_1 z = (z[i-2] - 8 z[i-1] + 8 z[i+1] - z[i+2]) / (12 dt)
      D_2 z = (-z[i-2] + 16 z[i-1] - 30 z[i] + 16 z[i+1] - z[i+2]) / (12 dt^2)
      D_3 z = (-z[i-2] + 2 z[i-1] - 2 z[i+1] + z[i+2]) / (2 dt^3)
      D_4 z = (z[i-2] - 4 z[i-1] + 6 z[i] - 4 z[i+1] + z[i+2]) / dt^4
  (z = 0 outside the grid); M_k = max_l |q_k,l|;
  f[k*6 + l] = q_k,l / M_k (0 if M_k = 0), k = 0..4, l = 0..5;
  f[30 + k] = clamp(log10(M_{k+1}/M_k), -8, 8) / 4 (-2 if either is 0);
  f[34 + l] = (T_l/Tbar - 1) * 100,  f[40 + l] = 1 - k.n_l;
  f[46] = dt/Tbar, f[47] = 0;  Tbar = L/c.
Scale s = M_2 / 8, set to 0 below the band, i.e. where M_2/M_0 < (2 pi f_lo
Tbar)^2 (M_0 = 0 counts as below); above the band: M_2/M_0 > (2 pi f_hi
Tbar)^2.  Target of link l: (y_full_l - z_l (1 + eps_l)) / s (0 where s = 0).
"""
from __future__ import annotations

import math

import numpy as np

N_FEAT = 47
ROW = 48
C_LIGHT = 299792458.0


def stencils(z, i, dt, Tbar):
    """q_k (k = 0..4) of one series z at sample i (zero outside the grid)."""
    n = len(z)
    v = [float(z[i + d]) if 0 <= i + d < n else 0.0 for d in (-2, -1, 0, 1, 2)]
    zm2, zm1, z0, zp1, zp2 = v
    d1 = (zm2 - 8.0 * zm1 + 8.0 * zp1 - zp2) / (12.0 * dt)
    d2 = (-zm2 + 16.0 * zm1 - 30.0 * z0 + 16.0 * zp1 - zp2) / (12.0 * dt ** 2)
    d3 = (-zm2 + 2.0 * zm1 - 2.0 * zp1 + zp2) / (2.0 * dt ** 3)
    d4 = (zm2 - 4.0 * zm1 + 6.0 * z0 - 4.0 * zp1 + zp2) / dt ** 4
    return [z0, Tbar * d1, Tbar ** 2 * d2, Tbar ** 3 * d3, Tbar ** 4 * d4]


def features(z, T, kn, L_m, dt, f_lo=0.0, f_hi=math.inf, y_full=None, eps=None):
    """z: [6][n] LFA links at their own time, T: [6][n] light times and
    kn: [6][n] k.n_l of the six links (link order +1,-1,+2,-2,+3,-3).
    eps: [6][n] (link_eps) or None for 0.  Returns (feats [n][48], scale [n],
    above_band [n] bool, target [n][6] or None)."""
    z = np.asarray(z, dtype=np.float64)
    n = z.shape[1]
    Tbar = L_m / C_LIGHT
    w_lo = (2.0 * math.pi * f_lo * Tbar) ** 2
    w_hi = (2.0 * math.pi * f_hi * Tbar) ** 2 if math.isfinite(f_hi) else math.inf
    feats = np.zeros((n, ROW))
    scale = np.zeros(n)
    above = np.zeros(n, dtype=bool)
    target = np.zeros((n, 6)) if y_full is not None else None
    eps = np.zeros((6, n)) if eps is None else np.asarray(eps)
    for i in range(n):
        q = np.array([stencils(z[l], i, dt, Tbar) for l in range(6)]).T     # q[k][l]
        M = np.abs(q).max(axis=1)
        for k in range(5):
            if M[k] > 0:
                feats[i, 6 * k:6 * k + 6] = q[k] / M[k]
        for k in range(4):
            r = math.log10(M[k + 1] / M[k]) if (M[k] > 0 and M[k + 1] > 0) else -8.0
            feats[i, 30 + k] = min(max(r, -8.0), 8.0) / 4.0
        feats[i, 34:40] = (T[:, i] / Tbar - 1.0) * 100.0
        feats[i, 40:46] = 1.0 - kn[:, i]
        feats[i, 46] = dt / Tbar
        w2 = M[2] / M[0] if M[0] > 0 else 0.0
        s = M[2] / 8.0 if w2 >= w_lo else 0.0
        above[i] = w2 > w_hi
        scale[i] = s
        if target is not None and s > 0:
            for l in range(6):
                target[i, l] = (y_full[l, i] - z[l, i] * (1.0 + eps[l, i])) / s
    return feats, scale, above, target


def link_geometry(orbit_mod, orbit, grid, beta, lam):
    """T [6][n] and k.n [6][n] from the oracle's orbit geometry."""
    _, T, nh = orbit_mod.orbits(orbit, grid)
    k, _, _ = orbit_mod.sky_basis(beta, lam)
    kn = np.einsum("c,lcn->ln", k, nh)
    return T, kn


SENDER = (2, 1, 0, 2, 1, 0)     # sender spacecraft of links +1,-1,+2,-2,+3,-3


def link_eps(orbit_mod, orbit, grid, beta, lam):
    """eps_l(t_i) = k.(R_s(t) - R_s(t - T_l)) / (c T_l (1 - k.n_l)) [6][n]."""
    t0, dt, n = grid
    k, _, _ = orbit_mod.sky_basis(beta, lam)
    out = np.zeros((6, n))
    for i in range(n):
        t = t0 + i * dt
        _, T, nh = orbit_mod.geometry(orbit, t)
        for l in range(6):
            kn = float(k @ nh[l])
            if 1.0 - kn < 1e-12:
                continue
            d = orbit_mod.position(orbit, SENDER[l], t) - orbit_mod.position(orbit, SENDER[l], t - T[l])
            out[l, i] = float(k @ d) / (C_LIGHT * T[l] * (1.0 - kn))
    return out
