"""The learned LFA-link corrector on the GPU, through the C ABI.

* own-time LFA links, features, forward pass and gradients against the FP64
  references (oracle/__init__.links_lfa_own, oracle/corrector.py,
  oracle/mlp.py);
* Adam against its textbook definition; checkpoint round trip;
* the full-link fallbacks (above the band, failed spot check) and the
  below-band base link;
* training on the GPU and what the trained network gains over the plain LFA,
  per link and in the hybrid (the error of the three-zone corrected hybrid
  against the plain hybrid's at the same switch frequency, and its cost on
  the one-year workload).

BF16-scaled tolerances: the network runs with BF16 weights and activations
(unit roundoff u = 2^-8) and FP32 accumulation; a forward pass rounds four
times and a backward pass four more, so errors of a few u, i.e. ~1e-2 of the
output scale, are the expected size.  Relative L2 errors per parameter block
are held to 5e-2 (~13 u) and the loss to 1e-2.
"""
import math

import numpy as np
import pytest

import synth
from gpu_util import F64_TOL, ORBITS, orbit_pair, rel_err, to_dev
from tolerances import MIXED_TOL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_09600_gb300 import build
    build.build()
    import paper_2505_09600_gb300 as L
    L.load()
    return L


def _dev_source(s):
    return dict(grid=s.grid, sky=(s.beta, s.lam, s.psi), hp32=to_dev(s.hp, 1), hc32=to_dev(s.hc, 1),
                hp64=to_dev(s.hp, 0), hc64=to_dev(s.hc, 0))


def _small_source(n=900, f0=3e-3, ratio=1.5, dt=5.0, seed=1):
    p = synth.corrector_params(nsrc=1, seed=synth.SEED_BASE + 400 + seed, n=n)[0]
    p.update(f0=f0, ratio=ratio, dt=dt, e0=0.0)
    return synth.corrector_source(p)


# ---------------------------------------------------------------------------
# parity of the building blocks
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kind", [0, 2, 3])   # central, backward, forward expansion point
def test_links_lfa_own(L, oracle_mod, precision, kind):
    s = _small_source(n=1300)
    oo, lo = orbit_pair("kepler2_flex")
    sky = (s.beta, s.lam, s.psi)
    hp = s.hp.astype(np.float32).astype(np.float64) if precision == 1 else s.hp
    hc = s.hc.astype(np.float32).astype(np.float64) if precision == 1 else s.hc
    z = torch.full((6, s.n), float("nan"), device="cuda", dtype=torch.float64 if precision == 0 else torch.float32)
    L.lisa_links_lfa_own(lo, sky, s.grid, to_dev(hp, precision), to_dev(hc, precision), precision, kind, s.grid, z)
    want = oracle_mod.links_lfa_own(oo, sky, s.grid, hp, hc, kind, s.grid)
    got = z.cpu().numpy().astype(np.float64)
    tol = np.full(6, F64_TOL) if precision == 0 else np.array(MIXED_TOL["z"])
    assert np.all(rel_err(got, want) <= tol), rel_err(got, want)


def test_features_match_oracle(L, oracle_mod):
    from oracle import corrector as OC
    s = _small_source(n=700, f0=4e-3)
    oo, lo = orbit_pair("kepler2_flex")
    d = _dev_source(s)
    n = s.n
    z = torch.empty((6, n), device="cuda", dtype=torch.float32)
    L.lisa_links_lfa_own(lo, d["sky"], s.grid, d["hp32"], d["hc32"], L.MIXED, L.LFA_UNEQUAL, s.grid, z)
    y = torch.empty((6, n), device="cuda", dtype=torch.float64)
    L.lisa_links_full(lo, d["sky"], s.grid, d["hp64"], d["hc64"], L.F64, s.grid, y)
    feats = torch.full((n, 48), float("nan"), device="cuda")
    scale = torch.empty(n, device="cuda")
    ybase = torch.empty((6, n), device="cuda")
    target = torch.empty((n, 6), device="cuda")
    f_lo, f_hi = 1e-4, 2e-2
    L.lisa_corrector_features(lo, d["sky"], s.grid, z, y, None, f_lo, f_hi, feats, scale, ybase, target)
    zh = z.cpu().numpy().astype(np.float64)
    yh = y.cpu().numpy()
    T, kn = OC.link_geometry(oracle_mod, oo, s.grid, s.beta, s.lam)
    eps = OC.link_eps(oracle_mod, oo, s.grid, s.beta, s.lam)
    wf, ws, _, wt = OC.features(zh, T, kn, oo.L_m, s.dt, f_lo=f_lo, f_hi=f_hi, y_full=yh, eps=eps)
    gf = feats.cpu().numpy().astype(np.float64)
    assert np.isfinite(gf).all()
    # Interior samples (away from the ends, where h switches on abruptly and
    # the stencils of z are ill-conditioned in FP32): FP32 stencils of the
    # same FP32 series (differences first), FP32 evaluation of the orbit
    # polynomial for the geometry columns.
    from paper_2505_09600_gb300.corrector import edge_margin
    m = edge_margin(s.dt)
    sl = slice(m, n - m)
    # Stencil columns: each FP32 operation rounds by u = 2^-24 relative to
    # operands of size |z| (T/dt)^k S_k (S_k = sum of the stencil's |weights|:
    # 1, 1.5, 16/3, 3, 16), so the normalised q_k,l may differ by
    # 4 u (T/dt)^k S_k max|z| / M_k (ill-conditioned only where the z series
    # cross zero); the ratio columns by that over ln 10 / 4 per order.
    u = 2.0 ** -24
    r1 = (oo.L_m / OC.C_LIGHT) / s.dt
    S = [1.0, 1.5, 16.0 / 3.0, 3.0, 16.0]
    zpad = np.pad(zh, ((0, 0), (2, 2)))
    zmax = np.max([np.abs(zpad[:, j:j + n]).max(axis=0) for j in range(5)], axis=0)
    q = np.stack([np.array([OC.stencils(zh[l], i, s.dt, oo.L_m / OC.C_LIGHT)
                            for i in range(n)]) for l in range(6)], 0)                   # [6][n][5]
    Mk = np.abs(q).max(axis=0)                                                           # [n][5]
    tol = np.zeros((n, 34))
    for k in range(5):
        tk = 4 * u * r1 ** k * S[k] * zmax / np.where(Mk[:, k] > 0, Mk[:, k], np.inf) + 1e-6
        tol[:, 6 * k:6 * k + 6] = tk[:, None]
    for k in range(4):
        tol[:, 30 + k] = (tol[:, 6 * k] + tol[:, 6 * (k + 1)]) / math.log(10) / 4 + 1e-6
    d = np.abs(gf[:, :34] - wf[:, :34])
    bad = d[sl] > tol[sl]
    assert not bad.any(), (d[sl][bad][:5], tol[sl][bad][:5], np.argwhere(bad)[:5] + [m, 0])
    assert np.median(d[sl, :30]) < 1e-6
    assert np.abs(gf[sl, 34:40] - wf[sl, 34:40]).max() < 2e-4
    assert np.abs(gf[:, 40:46] - wf[:, 40:46]).max() < 2e-6
    assert np.allclose(gf[:, 46], wf[:, 46], rtol=1e-6) and np.all(gf[:, 47] == 0)
    gs = scale.cpu().numpy()
    assert np.allclose(gs[sl], ws[sl], rtol=2e-5, atol=0)
    gb = ybase.cpu().numpy().astype(np.float64)
    assert np.abs(gb - zh * (1 + eps)).max() <= 1e-7 * np.abs(zh).max()
    gt = target.cpu().numpy()[sl]
    assert np.abs(gt - wt[sl]).max() < 2e-3 * max(1.0, np.abs(wt[sl]).max())


def _params(seed):
    from oracle import mlp
    return mlp.init_params(mlp.layer_shapes(), seed).astype(np.float32)


def test_forward_matches_fp64_mlp(L):
    from oracle import mlp
    rng = np.random.default_rng(5)
    p = _params(21)
    x = np.zeros((1000, 48), dtype=np.float32)
    x[:, :47] = rng.normal(size=(1000, 47))
    c = L.LisaCorrector(p)
    out = torch.empty((1000, 6), device="cuda")
    c.forward(torch.as_tensor(x, device="cuda"), out)
    got = out.cpu().numpy().astype(np.float64)
    want, _, _ = mlp.forward(p.astype(np.float64), x[:, :47].astype(np.float64), mlp.layer_shapes())
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert err < 3e-2, err
    c.close()


def test_gradient_matches_fp64_backprop(L):
    from oracle import mlp
    rng = np.random.default_rng(9)
    shapes = mlp.layer_shapes()
    p = _params(33)
    M = 2000
    x = np.zeros((M, 48), dtype=np.float32)
    x[:, :47] = rng.normal(size=(M, 47))
    want_out, _, _ = mlp.forward(p.astype(np.float64), x[:, :47].astype(np.float64), shapes)
    t = (want_out + 0.5 * rng.normal(size=want_out.shape)).astype(np.float32)
    c = L.LisaCorrector(p)
    grad = torch.empty(c.n_params, device="cuda")
    loss = torch.empty(1, device="cuda")
    c.gradient(torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda"), grad, loss)
    g = grad.cpu().numpy().astype(np.float64)
    ref = mlp.backward(p.astype(np.float64), x[:, :47].astype(np.float64), t.astype(np.float64), shapes)
    lref = mlp.loss(p.astype(np.float64), x[:, :47].astype(np.float64), t.astype(np.float64), shapes)
    assert loss.item() == pytest.approx(lref, rel=1e-2)
    off = 0
    for o, i in shapes:
        for size in (o * i, o):
            a, b = g[off:off + size], ref[off:off + size]
            off += size
            assert np.linalg.norm(a - b) <= 5e-2 * np.linalg.norm(b), (o, i, size)
            assert a @ b >= 0.998 * np.linalg.norm(a) * np.linalg.norm(b)
    assert off == c.n_params
    # a minibatch of the whole set (all rows drawn with replacement) has the
    # same expected gradient; check only that it is finite and runs
    c.gradient(torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda"), grad, loss, batch=512, seed=3)
    assert torch.isfinite(grad).all()
    c.close()


def test_adam_step_is_textbook(L):
    rng = np.random.default_rng(2)
    p = _params(4)
    c = L.LisaCorrector(p)
    m = np.zeros_like(p, dtype=np.float64)
    v = np.zeros_like(p, dtype=np.float64)
    w = p.astype(np.float64)
    for step in range(1, 4):
        g = rng.normal(size=p.size).astype(np.float32)
        c.adam_step(torch.as_tensor(g, device="cuda"), 1e-2)
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g.astype(np.float64) ** 2
        w = w - 1e-2 * (m / (1 - 0.9 ** step)) / (np.sqrt(v / (1 - 0.999 ** step)) + 1e-8)
    st = c.get_state()
    assert st["step"] == 3
    assert np.abs(st["params"] - w).max() < 1e-5
    c.close()


def test_checkpoint_round_trip(L, tmp_path):
    rng = np.random.default_rng(8)
    x = torch.as_tensor(rng.normal(size=(300, 48)).astype(np.float32), device="cuda")
    x[:, 47:] = 0
    c = L.LisaCorrector(None, seed=77)
    g = torch.as_tensor(rng.normal(size=c.n_params).astype(np.float32), device="cuda")
    c.adam_step(g, 1e-3)
    path = str(tmp_path / "corr.npz")
    c.save(path)
    a = torch.empty((300, 6), device="cuda")
    c.forward(x, a)
    d = L.LisaCorrector(None, seed=1)
    d.load_checkpoint(path)
    b = torch.empty((300, 6), device="cuda")
    d.forward(x, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert d.get_state()["step"] == 1
    # the library's own initialisation is seeded and bounded by 1/sqrt(n_in)
    p = L.LisaCorrector(None, seed=77).get_state()["params"]
    q = L.LisaCorrector(None, seed=77).get_state()["params"]
    assert np.array_equal(p, q)
    assert np.abs(p[:64 * 47]).max() <= 1 / math.sqrt(47) + 1e-7
    c.close()
    d.close()


# ---------------------------------------------------------------------------
# fallbacks
# ---------------------------------------------------------------------------

def _same_links(y, full):
    # the corrector's full-link tiles and lisa_links_full evaluate the same
    # formulas in FP32 from their own kernels: equal to FP32 rounding
    return float((y - full).abs().max()) <= 2e-6 * float(full.abs().max())


def _fallback_case(L):
    s = _small_source(n=3000, f0=3e-3)
    _, lo = orbit_pair("kepler2_flex")
    d = _dev_source(s)
    full = torch.empty((6, s.n), device="cuda")
    L.lisa_links_full(lo, d["sky"], s.grid, d["hp32"], d["hc32"], L.MIXED, s.grid, full)
    return s, lo, d, full


def test_above_band_tiles_use_full_links(L):
    s, lo, d, full = _fallback_case(L)
    c = L.LisaCorrector(None, seed=5)
    c.configure(f_lo=0.0, f_hi=1e-5, spot_every=0)
    y = torch.full((6, s.n), float("nan"), device="cuda")
    c.links(lo, d["sky"], s.grid, d["hp32"], d["hc32"], s.grid, y)
    r = c.report()
    assert _same_links(y, full)
    assert r["band_tiles"] == (s.n + 255) // 256 and r["status"] == 0
    c.close()


def test_below_band_uses_base_links(L):
    s, lo, d, _ = _fallback_case(L)
    c = L.LisaCorrector(None, seed=5)
    c.configure(f_lo=1.0, f_hi=2.0, spot_every=0)
    y = torch.full((6, s.n), float("nan"), device="cuda")
    c.links(lo, d["sky"], s.grid, d["hp32"], d["hc32"], s.grid, y)
    z = torch.empty((6, s.n), device="cuda")
    L.lisa_links_lfa_own(lo, d["sky"], s.grid, d["hp32"], d["hc32"], L.MIXED, L.LFA_UNEQUAL, s.grid, z)
    feats = torch.empty((s.n, 48), device="cuda")
    scale = torch.empty(s.n, device="cuda")
    ybase = torch.empty((6, s.n), device="cuda")
    L.lisa_corrector_features(lo, d["sky"], s.grid, z, None, None, 1.0, 2.0, feats, scale, ybase)
    full = torch.empty((6, s.n), device="cuda")
    L.lisa_links_full(lo, d["sky"], s.grid, d["hp32"], d["hc32"], L.MIXED, s.grid, full)
    torch.cuda.synchronize()
    # interior: the base links; within ~670 s of either end (retarded times
    # off the h grid): the full links
    from paper_2505_09600_gb300.corrector import edge_margin
    m = edge_margin(s.dt)
    assert torch.equal(y[:, m:s.n - m], ybase[:, m:s.n - m])
    assert _same_links(y[:, :120], full[:, :120]) and _same_links(y[:, s.n - 120:], full[:, s.n - 120:])
    assert float(scale.abs().max()) == 0.0
    c.close()


def test_failed_spot_check_recomputes_every_tile(L):
    s, lo, d, full = _fallback_case(L)
    c = L.LisaCorrector(None, seed=5)          # untrained network
    c.configure(f_lo=0.0, f_hi=1.0, spot_every=4, spot_tol=1e-9)
    y = torch.full((6, s.n), float("nan"), device="cuda")
    c.links(lo, d["sky"], s.grid, d["hp32"], d["hc32"], s.grid, y)
    r = c.report()
    ntile = (s.n + 255) // 256
    # spot checks only on tiles whose retarded times stay on the h grid (about
    # 670 s = 134 samples lost at each end: tiles 1..10 of 12), every 4th from
    # the first of them: tiles 1, 5 and 9
    assert r["status"] == L.LISA_ECORRECTOR
    assert r["spot_tiles"] == 3 and r["spot_failed"] == r["spot_tiles"]
    assert r["fallback_tiles"] == ntile - r["spot_tiles"]
    assert _same_links(y, full)
    # counters were reset by the report; a lenient tolerance passes
    c.configure(f_lo=0.0, f_hi=1.0, spot_every=1, spot_tol=10.0)
    c.links(lo, d["sky"], s.grid, d["hp32"], d["hc32"], s.grid, y)
    r = c.report()
    assert r["status"] == 0 and r["spot_tiles"] == ntile - 2 and r["spot_failed"] == 0
    c.close()


# ---------------------------------------------------------------------------
# training and gain
# ---------------------------------------------------------------------------

N_TRAIN, N_HELD = 128, 24


@pytest.fixture(scope="module")
def trained(L):
    from paper_2505_09600_gb300 import corrector as CT
    _, lo = orbit_pair("kepler2_flex")
    params = synth.corrector_params(nsrc=N_TRAIN + N_HELD, seed=synth.SEED_BASE + 4, n=4096)
    srcs = [synth.corrector_source(p) for p in params]
    feats, target = CT.training_set(lo, [_dev_source(s) for s in srcs[:N_TRAIN]])
    c = L.LisaCorrector(None, seed=2505)
    steps = 6000
    losses = torch.empty(steps, device="cuda")
    c.train(feats, target, steps=steps, batch=8192, lr_max=2e-3, lr_min=2e-5, seed=11, losses=losses)
    torch.cuda.synchronize()
    return c, lo, srcs[N_TRAIN:], losses.cpu().numpy(), float(target.square().sum(1).mean())


def test_training_reduces_the_loss(trained):
    _, _, _, losses, var = trained
    assert np.isfinite(losses).all()
    first, last = losses[:50].mean(), losses[-200:].mean()
    print("corrector loss: first %.4g last %.4g (target mean square %.4g)" % (first, last, var))
    assert last < 0.02 * var


def test_link_gain_on_held_out_sources(L, trained):
    from paper_2505_09600_gb300 import corrector as CT
    c, lo, held, _, _ = trained
    c.configure(f_lo=1e-4, f_hi=2e-2, spot_every=64, spot_tol=0.05)
    rows = []
    for s in held:
        d = _dev_source(s)
        n, m = s.n, CT.edge_margin(s.dt)
        yref = torch.empty((6, n), device="cuda", dtype=torch.float64)
        L.lisa_links_full(lo, d["sky"], s.grid, d["hp64"], d["hc64"], L.F64, s.grid, yref)
        z = torch.empty((6, n), device="cuda")
        L.lisa_links_lfa_own(lo, d["sky"], s.grid, d["hp32"], d["hc32"], L.MIXED, L.LFA_UNEQUAL, s.grid, z)
        y = torch.empty((6, n), device="cuda")
        c.links(lo, d["sky"], s.grid, d["hp32"], d["hc32"], s.grid, y)
        ref = yref.cpu().numpy()[:, m:n - m]
        scale = np.abs(ref).max()
        e_lfa = np.abs(z.cpu().numpy()[:, m:n - m] - ref).max() / scale
        e_cor = np.abs(y.cpu().numpy()[:, m:n - m] - ref).max() / scale
        r = c.report()
        rows.append((s.meta["f0"], s.meta["f0"] * s.meta["ratio"], e_lfa, e_cor, r["status"], r["max_spot_err"],
                     r["band_tiles"]))
    rows = np.array(rows)
    for f0, f1, a, b, st, se, bt in rows:
        print("held-out f %.2e..%.2e  LFA %.2e  corrected %.2e  gain %.1f  (spot err %.1e%s, %d tiles above band)"
              % (f0, f1, a, b, a / b, se, " FAILED" if st else "", bt))
    assert np.all(rows[:, 4] == 0)
    # where the LFA error is well above the FP32 floor of the mixed links
    sel = rows[:, 2] > 2e-4
    assert sel.sum() >= 8
    gains = rows[sel, 2] / rows[sel, 3]
    assert np.median(gains) >= 10.0, gains
    assert np.all(rows[:, 3] <= np.maximum(rows[:, 2], 2e-5))


def _side_error(got, ref, i_end, m):
    g, r = got[:, m:i_end], ref[:, m:i_end]
    return np.abs(g - r).max() / np.abs(r).max()


def _sigmoid_keep(t, ts, sigma):
    """S(t; t_s) = 1 / (1 + exp((t - t_s) / sigma)) (Sec. IV, Eq. sigmoid)."""
    return 1.0 / (1.0 + np.exp(np.clip((t - ts) / sigma, -700.0, 700.0)))


def test_three_zone_hybrid_blend(L, trained):
    """The corrected hybrid is plain LFA below t_lo, corrected links with the
    full TDI combine between t_lo and t_hyb and the full response above,
    joined by the paper's sigmoid at both seams: it equals
    S_lo S_hi X_LFA + (1 - S_lo) S_hi X_corr + (1 - S_hi) X_full formed here
    from the separate calls (each zone's weights summing to one)."""
    c, lo, _, _, _ = trained
    c.configure(f_lo=1e-4, f_hi=2e-2, spot_every=64, spot_tol=0.05)
    p = synth.sweep_params(nsrc=1, seed=synth.SEED_BASE + 41)[0]
    s = synth.sweep_source(p)
    d = _dev_source(s)
    n = s.n
    Tw, sig = 800 * s.dt, 20 * s.dt
    t_hi = L.lisa_t_hyb_from_f(2e-3, s.mc_s, s.tc)
    t_lo = L.lisa_t_hyb_from_f(1e-3, s.mc_s, s.tc)
    x_lfa = torch.empty((3, n), device="cuda")
    L.lisa_response_lfa(lo, d["sky"], s.grid, d["hp32"], d["hc32"], L.MIXED, L.TDI20, L.LFA_UNEQUAL, L.AET, s.grid,
                        x_lfa)
    y = torch.empty((6, n), device="cuda")
    c.links(lo, d["sky"], s.grid, d["hp32"], d["hc32"], s.grid, y)
    x_cor = torch.empty((3, n), device="cuda")
    L.lisa_tdi(lo, s.grid, y, L.MIXED, L.TDI20, L.FROZEN, L.AET, s.grid, x_cor)
    x_full = torch.empty((3, n), device="cuda")
    L.lisa_response_full(lo, d["sky"], s.grid, d["hp32"], d["hc32"], L.MIXED, L.TDI20, L.AET, s.grid, x_full)
    got = torch.full((3, n), float("nan"), device="cuda")
    c.hybrid(lo, d["sky"], s.grid, d["hp32"], d["hc32"], L.TDI20, L.AET, t_hi, Tw, sig, s.grid, got, t_lo=t_lo)
    assert c.report()["status"] == 0
    t = s.t0 + np.arange(n) * s.dt
    s_lo, s_hi = _sigmoid_keep(t, t_lo, sig), _sigmoid_keep(t, t_hi, sig)
    want = (s_lo * s_hi * x_lfa.cpu().numpy().astype(np.float64)
            + (1.0 - s_lo) * s_hi * x_cor.cpu().numpy().astype(np.float64)
            + (1.0 - s_hi) * x_full.cpu().numpy().astype(np.float64))
    g = got.cpu().numpy().astype(np.float64)
    assert np.isfinite(g).all()
    # zones: both seams and all three parts are present on this grid
    i_lo, i_hi = np.searchsorted(t, t_lo), np.searchsorted(t, t_hi)
    assert 1000 < i_lo < i_hi - 1000 and i_hi < n - 500
    err = np.abs(g - want).max(axis=1) / np.abs(want).max()
    print("three-zone blend vs separate calls: A/E/T", err)
    assert np.all(err < MIXED_TOL["hybrid20"]["aet"][0]), err


F_H_EVAL = (1e-3, 2e-3)


def test_hybrid_error_gain_at_fixed_switch(L, trained):
    """What the trained network gains in the hybrid: at the same switch
    frequency f_H, the error of the corrected hybrid (plain LFA below f_H/2,
    corrected links up to f_H) against the plain hybrid's, both against the
    FP64 full response on the approximate side (no ceiling on the measure)."""
    from paper_2505_09600_gb300 import corrector as CT
    c, lo, _, _, _ = trained
    c.configure(f_lo=1e-4, f_hi=2e-2, spot_every=64, spot_tol=0.05)
    ratios = {fH: [] for fH in F_H_EVAL}
    for p in synth.sweep_params(nsrc=6, seed=synth.SEED_BASE + 41):
        s = synth.sweep_source(p)
        d = _dev_source(s)
        n, m = s.n, CT.edge_margin(s.dt)
        ref = torch.empty((3, n), device="cuda", dtype=torch.float64)
        L.lisa_response_full(lo, d["sky"], s.grid, d["hp64"], d["hc64"], L.F64, L.TDI20, L.AET, s.grid, ref)
        ref = ref.cpu().numpy()
        Tw = 800 * s.dt
        out = torch.empty((3, n), device="cuda")
        for fH in F_H_EVAL:
            tH = L.lisa_t_hyb_from_f(fH, s.mc_s, s.tc)
            tL = L.lisa_t_hyb_from_f(0.5 * fH, s.mc_s, s.tc)
            i_end = int(min(n, max(0, math.floor((tH + Tw / 2 - s.t0) / s.dt) + 1)))
            L.lisa_response_hybrid(lo, d["sky"], s.grid, d["hp32"], d["hc32"], L.MIXED, L.TDI20, L.LFA_UNEQUAL,
                                   L.AET, tH, 0.0, 0.0, s.grid, out)
            ep = _side_error(out.cpu().numpy(), ref, i_end, m)
            c.hybrid(lo, d["sky"], s.grid, d["hp32"], d["hc32"], L.TDI20, L.AET, tH, 0.0, 0.0, s.grid, out, t_lo=tL)
            ec = _side_error(out.cpu().numpy(), ref, i_end, m)
            print("Mc %.3g f_H %.0e: plain %.2e corrected %.2e ratio %.1f" % (p["mc"], fH, ep, ec, ep / ec))
            ratios[fH].append(ep / ec)
    assert c.report()["status"] == 0
    for fH, r in ratios.items():
        r = np.asarray(r)
        assert np.all(r > 2.0), (fH, r)
        assert np.median(r) >= 5.0, (fH, r)


def test_corrected_hybrid_cost(L, trained):
    """On the one-year workload (6.3M samples at 5 s, switch at 1e-3 Hz) the
    corrected hybrid, whose corrected zone spans f_H/2..f_H, costs at most
    1.2 times the plain mixed hybrid."""
    c, lo, _, _, _ = trained
    c.configure(f_lo=1e-4, f_hi=2e-2, spot_every=64, spot_tol=0.05)
    s = synth.cfg2_source()
    hp, hc = to_dev(s.hp, 1), to_dev(s.hc, 1)
    sky = (s.beta, s.lam, s.psi)
    out = torch.empty((3, s.n), device="cuda")
    tH = L.lisa_t_hyb_from_f(1e-3, s.mc_s, s.tc)
    tL = L.lisa_t_hyb_from_f(5e-4, s.mc_s, s.tc)
    Tw, sig = 800 * s.dt, 20 * s.dt

    def timed(fn, reps=7):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return float(np.median(ms))

    mp = timed(lambda: L.lisa_response_hybrid(lo, sky, s.grid, hp, hc, L.MIXED, L.TDI20, L.LFA_UNEQUAL, L.AET, tH,
                                              Tw, sig, s.grid, out))
    mc = timed(lambda: c.hybrid(lo, sky, s.grid, hp, hc, L.TDI20, L.AET, tH, Tw, sig, s.grid, out, t_lo=tL))
    print("config-2 year: plain hybrid %.3f ms, corrected hybrid %.3f ms (ratio %.2f)" % (mp, mc, mc / mp))
    assert c.report()["status"] == 0
    assert mc <= 1.2 * mp, (mp, mc)
