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
    tol = 1e-11 if precision == 0 else 2e-5
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
