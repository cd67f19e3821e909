"""B1: brute-force pin of the oracle on tiny inputs.

An independent implementation at 30 significant digits (mpmath): its own
orbit and light-time code, the barycentric form of the Lagrange interpolant
instead of the product form, the TDI sums written term by term from the
printed Eqs. (X1.5) and (X2.0), and the LFA from Eqs. (yslr_strain_derivatives),
(X15_nonequal), (X20_nonequal).  The oracle must agree to ~1e-12 of the
channel's largest value.
"""
import math

import numpy as np
import pytest

import synth

mpmath = pytest.importorskip("mpmath")
mp = mpmath.mp

N = 40
DT = 10.0
T0 = 4.0e7 - 2000.0


def _setup():
    rng = np.random.default_rng(77)
    t = T0 + np.arange(N) * DT
    # smooth but non-trivial input: two tones with random phases
    hp = np.cos(2 * math.pi * 7e-3 * (t - T0) + 0.3) + 0.4 * np.sin(2 * math.pi * 1.9e-2 * (t - T0))
    hc = 0.8 * np.sin(2 * math.pi * 7e-3 * (t - T0) + 0.3) + 0.1 * rng.standard_normal(N)
    return hp, hc, (0.37, 4.1, 1.13)


class BF:
    """High-precision restatement of the response definitions."""

    def __init__(self, hp, hc, sky, L=2.5e9, kappa0=0.0, lambda0=0.0):
        mp.dps = 30
        self.c = mp.mpf(299792458)
        self.R = mp.mpf("1.495978707e11")
        self.W = 2 * mp.pi / mp.mpf(31557600)
        self.L = mp.mpf(L)
        self.e = self.L / (2 * mp.sqrt(3) * self.R)
        self.k0, self.l0 = mp.mpf(kappa0), mp.mpf(lambda0)
        self.hp = [mp.mpf(float(x)) for x in hp]
        self.hc = [mp.mpf(float(x)) for x in hc]
        beta, lam, psi = [mp.mpf(x) for x in sky]
        self.k = [-mp.cos(beta) * mp.cos(lam), -mp.cos(beta) * mp.sin(lam), -mp.sin(beta)]
        self.u = [mp.sin(lam), -mp.cos(lam), mp.mpf(0)]
        self.v = [-mp.sin(beta) * mp.cos(lam), -mp.sin(beta) * mp.sin(lam), mp.cos(beta)]
        self.c2, self.s2 = mp.cos(2 * psi), mp.sin(2 * psi)
        self.t0, self.dt = mp.mpf(T0), mp.mpf(DT)
        # barycentric weights of nodes -15..16
        self.bw = []
        for kk in range(-15, 17):
            p = mp.mpf(1)
            for m in range(-15, 17):
                if m != kk:
                    p *= (kk - m)
            self.bw.append(1 / p)

    def pos(self, s, t):
        a = self.W * t + self.k0
        b = 2 * mp.pi * s / 3 + self.l0
        R, e = self.R, self.e
        return [R * mp.cos(a) + e * R / 2 * (mp.cos(2 * a - b) - 3 * mp.cos(b)),
                R * mp.sin(a) + e * R / 2 * (mp.sin(2 * a - b) - 3 * mp.sin(b)),
                -mp.sqrt(3) * e * R * mp.cos(a - b)]

    SR = {1: (3, 2), -1: (2, 3), 2: (1, 3), -2: (3, 1), 3: (2, 1), -3: (1, 2)}

    def light(self, l, t):
        s, r = self.SR[l]
        Rr = self.pos(r - 1, t)
        T = mp.mpf(8)
        for _ in range(12):
            Rs = self.pos(s - 1, t - T)
            T = mp.sqrt(sum((Rr[q] - Rs[q]) ** 2 for q in range(3))) / self.c
        Rs = self.pos(s - 1, t - T)
        d = [Rr[q] - Rs[q] for q in range(3)]
        nrm = mp.sqrt(sum(x * x for x in d))
        return T, [x / nrm for x in d]

    def interp(self, h, tq):
        x = (tq - self.t0) / self.dt
        j = int(mp.floor(x))
        eps = x - j
        if eps == 0:
            return h[j] if 0 <= j < len(h) else mp.mpf(0)
        num = den = mp.mpf(0)
        for idx, kk in enumerate(range(-15, 17)):
            c = self.bw[idx] / (eps - kk)
            v = h[j + kk] if 0 <= j + kk < len(h) else mp.mpf(0)
            num += c * v
            den += c
        return num / den

    def dot(self, a, b):
        return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]

    def H(self, hp, hc, xp, xc):
        return xp * (hp * self.c2 - hc * self.s2) + xc * (hp * self.s2 + hc * self.c2)

    def link(self, l, t):
        s, r = self.SR[l]
        T, n = self.light(l, t)
        Rs, Rr = self.pos(s - 1, t), self.pos(r - 1, t)
        ds = T + self.dot(self.k, Rs) / self.c
        dr = self.dot(self.k, Rr) / self.c
        un, vn = self.dot(self.u, n), self.dot(self.v, n)
        xp, xc = un * un - vn * vn, 2 * un * vn
        Hs = self.H(self.interp(self.hp, t - ds), self.interp(self.hc, t - ds), xp, xc)
        Hr = self.H(self.interp(self.hp, t - dr), self.interp(self.hc, t - dr), xp, xc)
        return (Hs - Hr) / (2 * (1 - self.dot(self.k, n)))

    def links_grid(self):
        return {l: [self.link(l, self.t0 + i * self.dt) for i in range(N)] for l in (1, -1, 2, -2, 3, -3)}

    @staticmethod
    def cyc(l, times):
        for _ in range(times):
            l = (1 if l > 0 else -1) * (abs(l) % 3 + 1)
        return l

    def X(self, y, t, gen, ch):
        Lr = {l: self.light(self.cyc(l, ch), t)[0] for l in (1, -1, 2, -2, 3, -3)}
        Y = lambda l, D: self.interp(y[self.cyc(l, ch)], t - D)
        L = Lr
        x = (Y(-3, L[-2] + L[2] + L[3]) - Y(-3, L[3]) + Y(3, L[2] + L[-2]) - Y(3, 0)
             + Y(2, L[-2]) - Y(2, L[-2] + L[-3] + L[3]) + Y(-2, 0) - Y(-2, L[-3] + L[3]))
        if gen == 20:
            x += (Y(-3, L[-2] + L[2] + 2 * L[3] + L[-3]) - Y(-3, 2 * L[3] + L[-3] + 2 * L[-2] + 2 * L[2])
                  + Y(3, L[-2] + L[2] + L[3] + L[-3]) - Y(3, L[3] + L[-3] + 2 * L[-2] + 2 * L[2])
                  + Y(2, 2 * L[-2] + L[2] + 2 * L[3] + 2 * L[-3]) - Y(2, L[3] + L[-3] + 2 * L[-2] + L[2])
                  + Y(-2, L[-2] + L[2] + 2 * L[3] + 2 * L[-3]) - Y(-2, L[3] + L[-3] + L[-2] + L[2]))
        return x

    # --- LFA ---
    def hdot(self, h):
        g = lambda i: h[i] if 0 <= i < len(h) else mp.mpf(0)
        return [(g(i - 2) - 8 * g(i - 1) + 8 * g(i + 1) - g(i + 2)) / (12 * self.dt) for i in range(len(h))]

    def ylfa(self, l, tp, hdp, hdc):
        s, r = self.SR[l]
        T, n = self.light(l, tp)
        tau = tp - T / 2 - (self.dot(self.k, self.pos(s - 1, tp)) + self.dot(self.k, self.pos(r - 1, tp))) / (2 * self.c)
        un, vn = self.dot(self.u, n), self.dot(self.v, n)
        xp, xc = un * un - vn * vn, 2 * un * vn
        return -T / 2 * self.H(self.interp(hdp, tau), self.interp(hdc, tau), xp, xc)

    def X_lfa(self, gen, ch):
        hdp, hdc = self.hdot(self.hp), self.hdot(self.hc)
        la, lb = self.cyc(2, ch), self.cyc(3, ch)        # X: y123, y231
        out = []
        za, zb, Ta, Tb = [], [], [], []
        for i in range(N):
            t = self.t0 + i * self.dt
            L3 = self.light(self.cyc(3, ch), t)[0]
            L2 = self.light(self.cyc(2, ch), t)[0]
            if gen == 15:
                za.append(self.ylfa(la, t - L3 - L2 / 2, hdp, hdc))
                zb.append(self.ylfa(lb, t - L2 - L3 / 2, hdp, hdc))
            else:
                za.append(self.ylfa(la, t - 2 * L3 - 3 * L2 / 2, hdp, hdc))
                zb.append(self.ylfa(lb, t - 2 * L2 - 3 * L3 / 2, hdp, hdc))
            Ta.append(L3)
            Tb.append(L2)
        g = lambda z, i: z[i] if 0 <= i < N else mp.mpf(0)
        for i in range(N):
            if gen == 15:
                d = lambda z: (g(z, i - 2) - 8 * g(z, i - 1) + 8 * g(z, i + 1) - g(z, i + 2)) / (12 * self.dt)
                out.append(4 * (Ta[i] * d(za) - Tb[i] * d(zb)))
            else:
                d = lambda z: (-g(z, i - 2) + 16 * g(z, i - 1) - 30 * g(z, i) + 16 * g(z, i + 1) - g(z, i + 2)) / (12 * self.dt ** 2)
                out.append(8 * (Ta[i] + Tb[i]) * (Ta[i] * d(za) - Tb[i] * d(zb)))
        return out


@pytest.fixture(scope="module")
def bf_case():
    hp, hc, sky = _setup()
    bf = BF(hp, hc, sky)
    return hp, hc, sky, bf, bf.links_grid()


def test_bruteforce_links(oracle_mod, bf_case):
    hp, hc, sky, bf, ybf = bf_case
    g = (T0, DT, N)
    y = oracle_mod.links_full(oracle_mod.Orbit(), sky, g, hp, hc, g)
    ref = np.array([[float(v) for v in ybf[l]] for l in (1, -1, 2, -2, 3, -3)])
    assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("gen", [15, 20])
def test_bruteforce_tdi(oracle_mod, bf_case, gen):
    hp, hc, sky, bf, ybf = bf_case
    g = (T0, DT, N)
    o = oracle_mod.Orbit()
    y = oracle_mod.links_full(o, sky, g, hp, hc, g)
    X = oracle_mod.tdi_from_y(o, g, y, gen)
    for ch in range(3):
        ref = np.array([float(bf.X(ybf, bf.t0 + i * bf.dt, gen, ch)) for i in range(N)])
        assert np.abs(X[ch] - ref).max() <= 1e-12 * np.abs(ref).max(), ch


@pytest.mark.parametrize("gen", [15, 20])
def test_bruteforce_lfa(oracle_mod, bf_case, gen):
    hp, hc, sky, bf, _ = bf_case
    g = (T0, DT, N)
    o = oracle_mod.Orbit()
    X = oracle_mod.response_lfa(o, sky, g, hp, hc, gen, oracle_mod.LFA_UNEQUAL)
    for ch in range(3):
        ref = np.array([float(v) for v in bf.X_lfa(gen, ch)])
        assert np.abs(X[ch] - ref).max() <= 1e-12 * np.abs(ref).max(), ch
