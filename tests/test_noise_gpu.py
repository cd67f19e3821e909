"""Likelihood tail on the GPU (PSDs, inner-product weights, FFT + inner
products) against the FP64 oracle (oracle/noise.py)."""
import numpy as np
import pytest

import synth
from gpu_util import host_inputs, orbit_pair, sky_of, to_dev
from oracle import noise as ON

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
L_M = 2.5e9


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_09600_gb300 import build
    build.build()
    import paper_2505_09600_gb300 as L
    L.load()
    return L


@pytest.mark.parametrize("gen", [15, 20])
@pytest.mark.parametrize("galaxy", [0, 1])
def test_psd_matches_oracle(L, gen, galaxy):
    f0, df, nf = 1e-5, 1.3e-5, 4000
    psd = torch.empty((2, nf), device="cuda", dtype=torch.float64)
    L.lisa_psd_aet(f0, df, nf, gen, L_M, 1.0, galaxy, psd)
    f = f0 + np.arange(nf) * df
    sae, st = ON.psd_aet(f, gen, L_M, 1.0, bool(galaxy))
    got = psd.cpu().numpy()
    for g, w in ((got[0], sae), (got[1], st)):
        assert np.all(np.abs(g - w) <= 1e-12 * np.abs(w) + 1e-14 * np.abs(w).max())


def test_weights_match_oracle(L):
    grid = (2.0e7, 5.0, 30001)
    f_min, f_max = 1e-4, 2.5e-2
    nf = grid[2] // 2 + 1
    w = torch.empty((2, nf), device="cuda", dtype=torch.float64)
    L.lisa_noise_weights_aet(grid, 0, 20, L_M, 1.0, 1, f_min, f_max, w)
    f = np.arange(nf) / (grid[2] * grid[1])
    df = 1.0 / (grid[2] * grid[1])
    sel = (f >= f_min) & (f <= f_max) & (f > 0)
    sae, st = ON.psd_aet(np.where(sel, f, 1.0), 20, L_M, 1.0, True)
    got = w.cpu().numpy()
    tol = 1e-12
    for row, s in ((0, sae), (1, st)):
        want = np.where(sel, 4 * df / s, 0.0)
        assert np.all((got[row] == 0) == (want == 0))
        assert np.allclose(got[row], want, rtol=tol, atol=0)


def _hybrid(L, s, precision):
    oo, lo = orbit_pair("kepler2_flex")
    hp, hc = host_inputs(s, precision)
    tH = L.lisa_t_hyb_from_f(1e-3, s.mc_s, s.tc)
    dt = torch.float32 if precision == 1 else torch.float64
    out = torch.empty((3, s.n), device="cuda", dtype=dt)
    L.lisa_response_hybrid(lo, sky_of(s), s.grid, to_dev(hp, precision), to_dev(hc, precision), precision, 20, 0, 1,
                           tH, 800 * s.dt, 20 * s.dt, s.grid, out)
    return out


def test_fft_length(L):
    for n in (1, 2, 17, 487, 30001, 6311520):
        assert L.lisa_fft_length(n) == ON.fft_length(n)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("pad", [False, True])
def test_inner_products_match_oracle(L, precision, pad):
    s = synth.cfg2_small(n=30001)
    x = _hybrid(L, s, precision)
    # y: the same signal with a small phase-like distortion (a shifted copy plus x)
    y = (0.8 * x + 0.2 * torch.roll(x, 3, dims=1)).contiguous()
    # band below the TDI 2.0 PSD zero at c/(4L) = 0.02998 Hz, where 4 df / S blows up
    f_min, f_max = 1e-4, 2.5e-2
    m = ON.fft_length(s.n) if pad else s.n
    nf = m // 2 + 1
    w = torch.empty((2, nf), device="cuda", dtype=torch.float64)
    L.lisa_noise_weights_aet(s.grid, m, 20, L_M, 1.0, 1, f_min, f_max, w)
    out = torch.empty(9, device="cuda", dtype=torch.float64)
    L.lisa_inner_aet(s.grid, m, x, y, precision, w, out)
    got = out.cpu().numpy().reshape(3, 3)
    want = ON.inner_aet(x.double().cpu().numpy(), y.double().cpu().numpy(), s.dt, f_min, f_max, 20, L_M, 1.0, True,
                        nfft=m)
    # mixed: FP32 transforms, products and partial sums (measured against the
    # FP64 products of the same FP32 series: 1.4e-7 for A and E, 6.5e-7 for T)
    tol = 1e-11 if precision == 0 else 2e-6
    np.testing.assert_allclose(got, want, rtol=tol)
    np.testing.assert_allclose(ON.overlap(got), ON.overlap(want), rtol=tol, atol=tol)
    # <x|x> with y = x (one transform) equals the xx product of the pair call
    out2 = torch.empty(9, device="cuda", dtype=torch.float64)
    L.lisa_inner_aet(s.grid, m, x, x, precision, w, out2)
    g2 = out2.cpu().numpy().reshape(3, 3)
    np.testing.assert_allclose(g2[:, 0], got[:, 1], rtol=1e-12)
    np.testing.assert_allclose(g2[:, 2], got[:, 1], rtol=1e-12)
    # run to run identical (fixed-order reduction)
    out3 = torch.empty(9, device="cuda", dtype=torch.float64)
    L.lisa_inner_aet(s.grid, m, x, y, precision, w, out3)
    assert torch.equal(out, out3)


@pytest.mark.parametrize("peak_exp", [4, -80, -96])
def test_inner_products_extreme_scales(L, peak_exp):
    """FP32 spectra far from the usual fractional-frequency scale: the response
    scaled so that its loudest bin sits at 2^peak_exp. At 2^4 the loud bins
    exceed the mixed kernel's scaled FP32 window [2^-92, 2^-1), at 2^-80 the
    quiet bins fall below it, at 2^-96 every bin does; those bins' products are
    formed in FP64. (All three rows take one scale: a batched FP32 transform
    of rows of very different size lets the rounding of the large row leak
    into the small ones, which no inner-product kernel can undo.)"""
    s = synth.cfg2_small(n=30001)
    x = _hybrid(L, s, 1)
    peak = torch.fft.rfft(x.double(), dim=1).abs().max().item()
    x = (x * float(2.0 ** peak_exp / peak)).contiguous()
    y = (0.8 * x + 0.2 * torch.roll(x, 3, dims=1)).contiguous()
    xs = torch.fft.rfft(x.double(), dim=1)
    comp = torch.maximum(xs.real.abs(), xs.imag.abs())
    if peak_exp == 4:
        assert comp.max().item() >= 0.5 and (comp < 0.5).any().item()
    elif peak_exp == -80:
        assert (comp >= 2.0 ** -92).any().item() and (comp[:, 1:] < 2.0 ** -92).any().item()
    else:
        assert comp.max().item() < 2.0 ** -92
    f_min, f_max = 1e-4, 2.5e-2
    nf = s.n // 2 + 1
    w = torch.empty((2, nf), device="cuda", dtype=torch.float64)
    L.lisa_noise_weights_aet(s.grid, 0, 20, L_M, 1.0, 1, f_min, f_max, w)
    out = torch.empty(9, device="cuda", dtype=torch.float64)
    L.lisa_inner_aet(s.grid, 0, x, y, 1, w, out)
    got = out.cpu().numpy().reshape(3, 3)
    want = ON.inner_aet(x.double().cpu().numpy(), y.double().cpu().numpy(), s.dt, f_min, f_max, 20, L_M, 1.0, True)
    assert np.isfinite(got).all()
    np.testing.assert_allclose(got, want, rtol=2e-5)


def test_mismatch_of_response_forms(L):
    """Mismatch between the mixed and FP64 hybrid responses: small, as the
    per-sample errors (~1e-6 of the peak) predict."""
    s = synth.cfg2_small(n=30000)
    x64 = _hybrid(L, s, 0)
    x32 = _hybrid(L, s, 1).double()
    nf = s.n // 2 + 1
    w = torch.empty((2, nf), device="cuda", dtype=torch.float64)
    L.lisa_noise_weights_aet(s.grid, 0, 20, L_M, 1.0, 1, 1e-4, 2.5e-2, w)
    out = torch.empty(9, device="cuda", dtype=torch.float64)
    L.lisa_inner_aet(s.grid, 0, x64, x32.contiguous(), 0, w, out)
    ip = out.cpu().numpy().reshape(3, 3)
    mm = ON.mismatch(ip)
    assert np.all(mm[:2] < 1e-8), mm


def test_inner_products_overflow_recompute(L):
    """A thread whose FP32 sums of weighted scaled squares overflow recomputes
    them in FP64: spectra whose loudest component is 2^-1.5 (inside the
    scaled FP32 window) with weights raised by 2^40 (their scaled values still
    inside [2^-60, 2^61)) push a single bin's scaled product past 2^128.
    Checked against the oracle (weights x 2^40: an exact power-of-two
    scaling), and the sums of squares of a quiet operand are kept from its
    FP32 path: <q|q> of the pair call (q, loud) equals that of (q, q)."""
    s = synth.cfg2_small(n=30001)
    x = _hybrid(L, s, 1)
    peak = torch.fft.rfft(x.double(), dim=1).abs().max().item()
    loud = (x * float(2.0 ** -1.5 / peak)).contiguous()
    quiet = (x * float(2.0 ** -40 / peak)).contiguous()
    f_min, f_max = 1e-4, 2.5e-2
    nf = s.n // 2 + 1
    w = torch.empty((2, nf), device="cuda", dtype=torch.float64)
    L.lisa_noise_weights_aet(s.grid, 0, 20, L_M, 1.0, 1, f_min, f_max, w)
    w = (w * 2.0 ** 40).contiguous()
    # the FP32 path is taken for bins whose scaled weight and components lie in
    # their windows; some of those bins alone overflow FP32 for the loud operand
    ws = w.cpu().numpy() * 2.0 ** -128
    X = np.fft.rfft(loud.double().cpu().numpy(), axis=1)
    comp = np.maximum(np.abs(X.real), np.abs(X.imag))
    w_in = (ws >= 2.0 ** -60) & (ws < 2.0 ** 61)
    rows = np.stack([ws[0], ws[0], ws[1]])
    win = np.stack([w_in[0], w_in[0], w_in[1]]) & (comp >= 2.0 ** -92) & (comp < 0.5)
    prod = rows * (np.abs(X) * 2.0 ** 64) ** 2
    assert (win & (prod >= 2.0 ** 128)).any()
    Q = np.fft.rfft(quiet.double().cpu().numpy(), axis=1)
    assert (rows * (np.abs(Q) * 2.0 ** 64) ** 2).max() < 2.0 ** 110

    def ip(a, b):
        out = torch.empty(9, device="cuda", dtype=torch.float64)
        L.lisa_inner_aet(s.grid, 0, a, b, 1, w, out)
        return out.cpu().numpy().reshape(3, 3)

    def want(a, b):
        return ON.inner_aet(a.double().cpu().numpy(), b.double().cpu().numpy(), s.dt, f_min, f_max, 20, L_M, 1.0,
                            True) * 2.0 ** 40

    got = {}
    for key, (a, b) in {"ll": (loud, loud), "ql": (quiet, loud), "lq": (loud, quiet), "qq": (quiet, quiet)}.items():
        got[key] = ip(a, b)
        assert np.isfinite(got[key]).all(), key
        np.testing.assert_allclose(got[key], want(a, b), rtol=2e-5, err_msg=key)
    np.testing.assert_allclose(got["ql"][:, 1], got["qq"][:, 1], rtol=1e-12)
    np.testing.assert_allclose(got["lq"][:, 2], got["qq"][:, 2], rtol=1e-12)
    np.testing.assert_allclose(got["ql"][:, 2], got["ll"][:, 2], rtol=1e-12)


def test_mixed_inner_products_against_f64(L):
    """The mixed inner products (FP32 transforms, FP32 products and partial
    sums) against the FP64 ones of the same FP32 series, and the mismatch
    they give at the scale of the paper's criterion (Sec. V A: 1e-5)."""
    s = synth.cfg2_small(n=30001)
    x = _hybrid(L, s, 1)
    f_min, f_max = 1e-4, 2.5e-2
    nf = s.n // 2 + 1
    w = torch.empty((2, nf), device="cuda", dtype=torch.float64)
    L.lisa_noise_weights_aet(s.grid, 0, 20, L_M, 1.0, 1, f_min, f_max, w)
    # y: x with a small admixture of a shifted copy, mismatch of order 1e-5
    y = (x + 2e-2 * torch.roll(x, 1, dims=1)).contiguous()

    def ip(a, b, precision):
        out = torch.empty(9, device="cuda", dtype=torch.float64)
        L.lisa_inner_aet(s.grid, 0, a, b, precision, w, out)
        return out.cpu().numpy().reshape(3, 3)

    m32 = ip(x, y, 1)
    m64 = ip(x.double().contiguous(), y.double().contiguous(), 0)
    rel = np.abs(m32 - m64) / np.abs(m64)
    mm32, mm64 = ON.mismatch(m32), ON.mismatch(m64)
    print("mixed vs FP64 inner products, relative:", rel.max(axis=1), "mismatch mixed", mm32, "FP64", mm64)
    assert np.all(rel < 2e-6), rel
    assert np.all(mm64[:2] > 1e-6) and np.all(mm64[:2] < 1e-4), mm64
    assert np.all(np.abs(mm32 - mm64)[:2] < 2e-7), (mm32, mm64)
