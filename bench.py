#!/usr/bin/env python
"""Benchmark of the GB300 time-domain LISA response (arXiv:2505.09600).

Workload (one step): the hybrid TDI 2.0 A/E/T response of one synthetic
source -- one year at 5 s (6,311,520 samples), Newtonian chirp (Mc=1e6 Msun,
q=3) to f_isco joined to a ringdown, exact Keplerian orbits with 1% arm
flexing, 32-point Lagrange interpolation, LFA with 5-point central differences,
switch at f_Hyb = 1e-3 Hz (T = 800 dt, sigma = T/40) -- computed in the
FP64-accurate line-of-record form (REC_PRECISION: FP64 inputs and outputs,
the LFA channels in double-float arithmetic on the FP32 pipe, the full part
in FP64; results within the FP64 tolerance of the oracle).  One step runs every stage:
orbit table, LFA z-series and channels, full links, TDI, A/E/T, sigmoid blend.

Metric: TDI samples/s (one sample = one output time, all three channels).
Other forms (mixed FP32 arithmetic, full, LFA, higher-order LFA kinds) are
timed and reported under "forms", with their errors and rooflines.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TDI samples/s (full, LFA, hybrid) at fixed max rel err vs FP64 oracle"
UNIT = "samples/s"
F_HYB = 1e-3
ORBIT_KW = dict(kind=1, delay=0, kepler_tilt=1.01)
L2_BYTES = 129 * 2 ** 20
FP32_PEAK_TFLOPS_FALLBACK = None

# Algorithmic work per output sample (flop) used for the roofline: Lagrange
# taps only, 2 flop per tap per interpolated series (weights and orbit work
# not counted), plus the finite-difference stencils: 6 z-series x 2
# polarisations x 32 taps x 2 flop = 768, stencils ~60 -> 830 for the LFA
# (unequal arms).  The count that includes the weights (4 flop per weight)
# is reported beside it.
LFA_TAPS_FLOP = 6 * 2 * 32 * 2 + 62
# The full response TDI 2.0 on the same view: links 6 x 2 retarded times x 2
# polarisations x 32 taps x 2 flop = 1,536, TDI 48 interpolations x 32 taps x
# 2 flop = 3,072.
FULL20_TAPS_FLOP = 6 * 2 * 2 * 32 * 2 + 48 * 32 * 2
W32 = 4 * 32
TAP = 2 * 32
FLOP_PER_SAMPLE = {
    # 6 z-series x (weights + 2 series of taps) + hdot (2 x 5) + 3 channels x
    # (2 five-point second differences + prefactors) + AET
    "lfa20": 6 * (W32 + 2 * TAP) + 10 + 3 * (2 * 9 + 6) + 8,
    "lfa15": 6 * (W32 + 2 * TAP) + 10 + 3 * (2 * 6 + 4) + 8,
    # links: 12 retarded times x (weights + 2 series) + projection; TDI 2.0:
    # 42 non-trivial interpolations of one series + 48 signed sums; AET
    "full20": 12 * (W32 + 2 * TAP) + 6 * 6 + 42 * (W32 + TAP) + 48 + 8,
    "full15": 12 * (W32 + 2 * TAP) + 6 * 6 + 18 * (W32 + TAP) + 24 + 8,
}


WORKLOAD_BASE = ("hybrid TDI2.0 AET, chirp+ringdown Mc=1e6 q=3, 1 yr @ 5 s (6311520 samples), "
                 "Kepler ellipses 1% flex, f_hyb=1e-3 Hz")

# Precision of the line of record: 2 = double-float (FP64 inputs and outputs,
# the LFA channels in pairs of FP32 numbers, the full part in FP64; results
# within the FP64 tolerance of the oracle); 0 = FP64 throughout.
REC_PRECISION = 2
REC_DTYPE = {0: "f64", 2: "df64"}
REC_KERNEL = {0: "lfa_f64", 2: "lfa_df"}

# FP32 operations (add, multiply or fused multiply-add: one each; a packed
# pair instruction counts as two) of the double-float LFA per output sample
# (TDI 2.0, A/E/T), counted from the algorithm's operations:
#   per z-series sample: 32 Lagrange weights and taps 1052 (weights 552: the
#   running products, the mirrored-node factors and the pair products in
#   double-float, the four outermost weights in FP32; taps of both
#   polarisations 480: the eight central taps by two-sum accumulation of
#   exact products, 24 each, twenty outer taps split against a power of two,
#   14 each, the four outermost as plain multiply-adds, 2 each; joining the
#   exact sums and the correction 20), position (delay polynomial with its
#   FP32 tail, scale, fraction) 69, projection factors (FP32 tails from u^3)
#   and z 119 -> 1240, x 6 series;
#   channels: the three light-time polynomials 3 x 47 (each arm enters two
#   channels), two 5-point second differences and the prefactors 273 per
#   channel x 3, A/E/T 82.
DF_OPS_PER_SAMPLE = {"lfa20": 6 * 1240 + 3 * 47 + 3 * 273 + 82}


def measured_fma_peaks(L):
    """FMA throughput of the FP64 and FP32 pipes on this GPU, measured in this
    run by the project's microbenchmark (lisa_peak_fma: 8 independent
    multiply-add chains per thread, 8 CTAs of 256 threads per SM; best of 5
    launches).  TFLOP/s, 2 flop per multiply-add."""
    f64, _ = L.lisa_peak_fma(0, 20000)
    f32a, _ = L.lisa_peak_fma(1, 200000)
    f32b, _ = L.lisa_peak_fma(2, 100000)
    return {"fp64_tflops": f64, "fp32_tflops": max(f32a, f32b), "fp32_scalar_tflops": f32a, "fp32_pair_tflops": f32b,
            "how": "lisa_peak_fma in this run: 8 independent FMA chains per thread, SMs x 8 CTAs of 256 threads, best of 5"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    d = {}
    if os.path.exists(p):
        try:
            d = json.load(open(p))
        except Exception:
            d = {}
    return d


# Sources each profiled kernel is built from: a committed DRAM-traffic figure
# counts only while these files are unchanged since the capture.
KERNEL_SOURCES = {
    "lfa_mixed": ("lfa.cu", "lfa_tile.cuh", "async_copy.cuh", "lisa_common.cuh", "tile_geo.cuh"),
    "lfa_df": ("lfa_df.cu", "dfloat.cuh", "lfa_tile.cuh", "lisa_common.cuh", "tile_geo.cuh"),
}


def kernel_src_hash(kernel):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(ROOT, "paper_2505_09600_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def committed_traffic(kernel):
    """DRAM bytes per launch of the dominant kernel from a committed ncu
    capture, if it was taken on this kernel and its current source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p) or kernel not in KERNEL_SOURCES:
        return None
    try:
        d = json.load(open(p)).get(kernel)
    except Exception:
        return None
    if not d or d.get("src_hash") != kernel_src_hash(kernel):
        return None
    return d.get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        self.path = None

    def start(self):
        try:
            # the raw samples go to LISA_BENCH_OUT (default: the system temporary directory)
            out_dir = os.environ.get("LISA_BENCH_OUT") or tempfile.gettempdir()
            os.makedirs(out_dir, exist_ok=True)
            self.path = os.path.join(out_dir, "clocks_rank%d.csv" % self.index)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms, world, device):
    """Slowest rank's time: replicas run independently, so the job ends when
    the last one does (one scalar all_reduce, outside the timed region)."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, n_per_rank, steps, total_ms):
    """Samples of all ranks per second of the slowest rank (weak scaling)."""
    return world * n_per_rank * steps / (total_ms / 1e3)


def make_source(rank):
    import synth
    return synth.cfg2_source(seed_offset=rank)


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, on a bounded sample of the workload
# ---------------------------------------------------------------------------

def oracle_hybrid_rate(src, budget_s=12.0, one_core=False, fp32_inputs=False):
    """Oracle samples/s for the hybrid workload on the host cores.

    The oracle computes the LFA on every sample and the full response on the
    samples from t_hyb - T/2 on.  Both parts are timed on bounded contiguous
    chunks (LFA chunk grown until ~budget/2 s; full part on its first samples)
    and extrapolated linearly to the whole series.  Returns the line's dict.
    """
    import oracle
    import synth  # noqa: F401
    oracle.build()
    s = src
    oo = oracle.Orbit(**ORBIT_KW)
    sky = (s.beta, s.lam, s.psi)
    hp, hc = _oracle_inputs(s, fp32_inputs)
    tH = oracle.t_hyb(F_HYB, s.mc_s, s.tc)
    Tw = 800 * s.dt
    i_full = max(0, int(math.ceil((tH - 0.5 * Tw - s.t0) / s.dt)))
    n_full = s.n - i_full
    t0 = time.perf_counter()
    hd = (oracle.hdot(s.grid, hp), oracle.hdot(s.grid, hc))
    t_hdot = time.perf_counter() - t0
    # LFA on a contiguous chunk of the inspiral: z on the chunk and its
    # 2-sample halo, then the channels
    chunk = 20000
    while True:
        i0 = s.n // 3
        zg = (s.t0 + (i0 - 2) * s.dt, s.dt, chunk + 4)
        t0 = time.perf_counter()
        z = oracle.z_lfa(oo, sky, s.grid, hp, hc, 20, 0, zg, hd=hd)
        oracle.tdi_lfa_from_z(oo, zg, z, 20, 0, idx=np.arange(2, chunk + 2))
        t_lfa = time.perf_counter() - t0
        if t_lfa > 0.4 * budget_s or chunk >= s.n // 4:
            break
        chunk = int(chunk * min(8.0, 0.5 * budget_s / max(t_lfa, 1e-3)))
    # full response on its whole region: links on the grid from 60 s before
    # the first full sample (the TDI delays never exceed that), then TDI
    marg = int(math.ceil(60.0 / s.dt)) + 20
    j0 = max(0, i_full - marg)
    ygrid = (s.t0 + j0 * s.dt, s.dt, s.n - j0)
    ogrid = (s.t0 + i_full * s.dt, s.dt, n_full)
    t0 = time.perf_counter()
    y = oracle.links_full(oo, sky, s.grid, hp, hc, ygrid)
    oracle.tdi_from_y(oo, ygrid, y, 20, oracle.FROZEN, ogrid)
    t_full = time.perf_counter() - t0
    total = t_hdot + t_lfa * s.n / chunk + t_full
    out = {"value": s.n / total, "unit": UNIT, "kind": "oracle",
           "sample": ("LFA (z series then channels) on %d contiguous samples, extrapolated to all %d; "
                      "full response (links then TDI) on its whole region of %d samples"
                      % (chunk, s.n, n_full)),
           "seconds": round(t_hdot + t_lfa + t_full, 3), "chunk": [int(i0), int(chunk)]}
    try:
        import synth as _s
        out["cores"] = int(os.environ.get("OMP_NUM_THREADS", 0)) or _s.host_cores()
    except Exception:
        out["cores"] = os.cpu_count()
    # the same legs on one core (a fresh process with OMP_NUM_THREADS=1), to set beside
    # single-core CPU figures; its LFA chunk is 20,000 samples
    if one_core:
        try:
            env = dict(os.environ, OMP_NUM_THREADS="1")
            r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-one-core"], env=env,
                               capture_output=True, text=True, timeout=300)
            out["one_core"] = json.loads(r.stdout.strip().splitlines()[-1])
        except Exception as e:   # reported, not fatal: the main figure stands
            out["one_core"] = {"unavailable": str(e)[:200]}
    return out


def _oracle_inputs(s, fp32_inputs):
    """h as the GPU form reads it, as FP64 for the oracle."""
    if fp32_inputs:
        return s.hp.astype(np.float32).astype(np.float64), s.hc.astype(np.float32).astype(np.float64)
    return s.hp, s.hc


def sampled_errors(src, gpu_out, fp32_inputs, chunk=None):
    """The timed GPU output against the oracle on sampled outputs (the oracle
    evaluates them one by one): an inspiral chunk, the full-response region and
    400 points log-spaced in time before the end.  Returns the global measure
    (largest channel maximum), the own-scale measure (each channel on its own
    maximum) and the local diagnostic per frequency decade."""
    import oracle
    import synth
    oracle.build()
    s = src
    oo = oracle.Orbit(**ORBIT_KW)
    sky = (s.beta, s.lam, s.psi)
    hp, hc = _oracle_inputs(s, fp32_inputs)
    hd = (oracle.hdot(s.grid, hp), oracle.hdot(s.grid, hc))
    tH = oracle.t_hyb(F_HYB, s.mc_s, s.tc)
    Tw, sig = 800 * s.dt, 20 * s.dt
    i_full = max(0, int(math.ceil((tH - 0.5 * Tw - s.t0) / s.dt)))
    i0, ch = chunk if chunk else (s.n // 3, 20000)
    idx = np.arange(i0, i0 + ch)
    idxf = np.arange(i_full, s.n)
    spread = (s.n - 1 - np.unique(np.geomspace(1, s.n - 1, 400).astype(np.int64))).astype(np.int64)
    blend_idx = np.unique(np.concatenate([idx[:: max(1, ch // 200)], idxf[::10], spread]))
    lf = oracle.tdi_lfa_direct(oo, sky, s.grid, hp, hc, 20, 0, s.grid, blend_idx, hd=hd)
    fu = np.zeros_like(lf)
    need = s.t0 + blend_idx * s.dt >= tH - 0.5 * Tw
    if need.any():
        fu[:, need] = oracle.tdi_full_direct(oo, sky, s.grid, hp, hc, s.grid, 20, 0, s.grid, blend_idx[need])
    want = oracle.aet(oracle.hybrid_blend(s.grid, tH, Tw, sig, lf, fu, blend_idx))
    d = np.abs(gpu_out[:, blend_idx] - want).max(axis=1)
    own = np.abs(want).max(axis=1)
    res = {"points": int(blend_idx.size),
           "max_rel_err": (d / np.abs(gpu_out).max()).tolist(),
           "max_rel_err_own": (d / np.where(own > 0, own, 1.0)).tolist()}
    # local diagnostic: per decade of the source's instantaneous frequency (0PN chirp
    # before the ringdown join, the ringdown frequency after), the error scaled by
    # the largest sampled |A, E, T| in that decade (and each channel by its own)
    tt = s.t0 + blend_idx * s.dt
    t_join = s.meta.get("t_join", s.tc)
    f_inst = np.where(tt <= t_join, synth.chirp_frequency(np.maximum(s.tc - tt, 1e-9), s.mc_s),
                      s.meta.get("f_rd", 1e-2))
    local = {}
    for k in range(-6, -1):
        sel = (f_inst >= 10.0 ** k) & (f_inst < 10.0 ** (k + 1))
        if sel.sum() < 3:
            continue
        sc_d = np.abs(want[:, sel]).max()
        if sc_d > 0:
            dd = np.abs(gpu_out[:, blend_idx[sel]] - want[:, sel]).max(axis=1)
            own_d = np.abs(want[:, sel]).max(axis=1)
            local["1e%d-1e%d Hz" % (k, k + 1)] = {
                "points": int(sel.sum()), "err": (dd / sc_d).tolist(),
                "err_own": (dd / np.where(own_d > 0, own_d, 1.0)).tolist()}
    res["local_per_decade"] = local
    return res


# ---------------------------------------------------------------------------
# learned corrector and batched plan (reported next to the headline)
# ---------------------------------------------------------------------------

def _timed(torch, stream, flush, fn, reps=3):
    fn()
    torch.cuda.synchronize()
    ms = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return float(np.median(ms))


def kernel_breakdown(L, torch, fn):
    """Device ms per kernel name of one call (lisa_profile event pairs)."""
    names = ("seg_table", "lfa_own_mixed", "lfa_mixed", "corr_features", "corr_fused_tc", "mlp_forward", "corr_fallback_all",
             "corr_fallback", "links_full_mixed", "tdi_mixed", "batch")
    L.lisa_profile_enable(True)
    fn()
    torch.cuda.synchronize()
    out = {}
    total, _ = L.lisa_profile_query(None)
    for nm in names:
        ms, cnt = L.lisa_profile_query(nm)
        if cnt:
            out[nm] = round(ms, 4)
    # fallback names overlap ("corr_fallback" also matches "corr_fallback_all")
    if "corr_fallback" in out and "corr_fallback_all" in out:
        out["corr_fallback"] = round(out["corr_fallback"] - out["corr_fallback_all"], 4)
    if "lfa_mixed" in out and "lfa_own_mixed" in out:
        pass
    out["all"] = round(total, 4)
    L.lisa_profile_enable(False)
    return out


# switch frequencies at which the corrected hybrid is compared with the plain
# one (same f_H); its lower seam (plain LFA below) sits at F_LO_RATIO * f_H
F_H_EVAL = (1e-3, 2e-3, 4e-3)
F_LO_RATIO = 0.5


def _quantiles(v):
    v = np.asarray(v, dtype=np.float64)
    return {"min": float(v.min()), "p10": float(np.quantile(v, 0.1)), "median": float(np.median(v)),
            "p90": float(np.quantile(v, 0.9)), "max": float(v.max())}


def _side_errors(got, ref, i_end, m):
    """Error on the approximate side t <= t_H + T/2 (ends of the grid
    excluded): max over A, E, T of |X - X_ref| / max |X_ref| (largest
    channel), and each channel on its own maximum."""
    g, r = got[:, m:i_end], ref[:, m:i_end]
    d = np.abs(g - r).max(axis=1)
    own = np.abs(r).max(axis=1)
    return float(d.max() / own.max()), (d / np.maximum(own, 1e-300)).tolist()


def bench_corrector(L, torch, dev, src, orbit, sky, hp32, hc32, out32, flush, stream, tH, Tw, sig,
                    n_sources=4096, n_per_source=5100, n_held=256, steps=8000, batch=8192, n_sweep=256):
    """Config 4: train the LFA-link corrector on the GPU on 4,096 seeded
    sources of the band 1e-4..2e-2 Hz (about 2e7 rows); judge it on 256
    held-out sources of the same distribution (link error against the FP64
    full links) and on 256 held-out chirps sweeping 5e-4..2e-2 Hz (hybrid
    error against the FP64 full response, corrected and plain at the same
    switch frequency); time both hybrids on the headline workload."""
    import synth
    from paper_2505_09600_gb300 import corrector as CT
    t0 = time.perf_counter()
    params = synth.corrector_params(nsrc=n_sources + n_held, seed=synth.SEED_BASE + 4, n=n_per_source)

    def dev_source(p):
        s = synth.corrector_source(p)
        return s, dict(grid=s.grid, sky=(s.beta, s.lam, s.psi),
                       hp32=torch.as_tensor(s.hp.astype(np.float32), device=dev),
                       hc32=torch.as_tensor(s.hc.astype(np.float32), device=dev),
                       hp64=torch.as_tensor(s.hp, device=dev), hc64=torch.as_tensor(s.hc, device=dev))
    devsrc = [dev_source(p)[1] for p in params[:n_sources]]
    t_gen = time.perf_counter() - t0
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    feats, target = CT.training_set(orbit, devsrc)
    b.record(stream)
    b.synchronize()
    t_set = a.elapsed_time(b)
    del devsrc
    c = L.LisaCorrector(None, seed=2505)
    losses = torch.empty(steps, device=dev)
    a.record(stream)
    c.train(feats, target, steps=steps, batch=batch, lr_max=2e-3, lr_min=2e-5, seed=11, losses=losses)
    b.record(stream)
    b.synchronize()
    t_train = a.elapsed_time(b)
    ls = losses.cpu().numpy()
    res = {"train_sources": n_sources, "train_rows": int(feats.shape[0]), "train_steps": steps, "batch": batch,
           "train_ms": round(t_train, 1), "train_rows_per_s": steps * batch / (t_train / 1e3),
           "training_set_ms": round(t_set, 1), "source_generation_s": round(t_gen, 2),
           "loss_first": float(ls[:50].mean()), "loss_last": float(ls[-200:].mean()),
           "target_mean_square": float(target.square().sum(1).mean())}
    del feats, target
    c.configure(f_lo=1e-4, f_hi=2e-2, spot_every=64, spot_tol=0.05)
    c.report()
    # link gain on the held-out sources of the training distribution
    g_rows = []
    for p in params[n_sources:]:
        s, d = dev_source(p)
        n, m = s.n, CT.edge_margin(s.dt)
        yref = torch.empty((6, n), device=dev, dtype=torch.float64)
        L.lisa_links_full(orbit, d["sky"], s.grid, d["hp64"], d["hc64"], L.F64, s.grid, yref)
        z = torch.empty((6, n), device=dev)
        L.lisa_links_lfa_own(orbit, d["sky"], s.grid, d["hp32"], d["hc32"], L.MIXED, L.LFA_UNEQUAL, s.grid, z)
        y = torch.empty((6, n), device=dev)
        c.links(orbit, d["sky"], s.grid, d["hp32"], d["hc32"], s.grid, y)
        ref = yref[:, m:n - m]
        scale = float(ref.abs().max())
        e_lfa = float((z[:, m:n - m].double() - ref).abs().max()) / scale
        e_cor = float((y[:, m:n - m].double() - ref).abs().max()) / scale
        g_rows.append((p["f0"], p["f0"] * p["ratio"], e_lfa, e_cor))
    g_rows = np.array(g_rows)
    sel = g_rows[:, 2] > 2e-4     # LFA error well above the FP32 floor of the mixed links
    rep = c.report()
    res["link_gain_held_out"] = {
        "sources": n_held, "sources_above_fp32_floor": int(sel.sum()),
        "gain_lfa_over_corrected": _quantiles(g_rows[sel, 2] / g_rows[sel, 3]) if sel.any() else None,
        "corrected_err": _quantiles(g_rows[:, 3]), "lfa_err": _quantiles(g_rows[:, 2]),
        "corrected_worse_than_lfa": int(np.sum(g_rows[:, 3] > np.maximum(g_rows[:, 2], 2e-5))),
        "spot_failed": rep["spot_failed"], "band_tiles": rep["band_tiles"],
        "error_measure": "max over the six links and samples (grid ends excluded) of |y - y_FP64full| / max |y_FP64full|"}
    # hybrid error, corrected vs plain at the same f_H, on held-out sweeping chirps
    per_f = {fH: {"ratio": [], "plain": [], "corrected": [], "ratio_own": []} for fH in F_H_EVAL}
    for p in synth.sweep_params(nsrc=n_sweep, seed=synth.SEED_BASE + 41):
        s = synth.sweep_source(p)
        n, m = s.n, CT.edge_margin(s.dt)
        sk = (s.beta, s.lam, s.psi)
        h32 = (torch.as_tensor(s.hp.astype(np.float32), device=dev), torch.as_tensor(s.hc.astype(np.float32), device=dev))
        h64 = (torch.as_tensor(s.hp, device=dev), torch.as_tensor(s.hc, device=dev))
        ref = torch.empty((3, n), device=dev, dtype=torch.float64)
        L.lisa_response_full(orbit, sk, s.grid, h64[0], h64[1], L.F64, 20, L.AET, s.grid, ref)
        refh = ref.cpu().numpy()
        o = torch.empty((3, n), device=dev)
        Tws = 800 * s.dt
        for fH in F_H_EVAL:
            tHx = L.lisa_t_hyb_from_f(fH, s.mc_s, s.tc)
            tLx = L.lisa_t_hyb_from_f(F_LO_RATIO * fH, s.mc_s, s.tc)
            i_end = int(min(n, max(0, math.floor((tHx + Tws / 2 - s.t0) / s.dt) + 1)))
            L.lisa_response_hybrid(orbit, sk, s.grid, h32[0], h32[1], L.MIXED, 20, 0, L.AET, tHx, 0.0, 0.0, s.grid, o)
            ep, ep_own = _side_errors(o.cpu().numpy().astype(np.float64), refh, i_end, m)
            c.hybrid(orbit, sk, s.grid, h32[0], h32[1], 20, L.AET, tHx, 0.0, 0.0, s.grid, o, t_lo=tLx)
            ec, ec_own = _side_errors(o.cpu().numpy().astype(np.float64), refh, i_end, m)
            per_f[fH]["plain"].append(ep)
            per_f[fH]["corrected"].append(ec)
            per_f[fH]["ratio"].append(ep / ec)
            per_f[fH]["ratio_own"].append(max(ep_own[:2]) / max(ec_own[:2]))
    rep = c.report()
    res["hybrid_error_gain"] = {
        "held_out_sources": n_sweep, "f_lo_over_f_H": F_LO_RATIO,
        "per_f_H": {"%g" % fH: {"plain_over_corrected": _quantiles(v["ratio"]),
                               "plain_over_corrected_AE_own_scale": _quantiles(v["ratio_own"]),
                               "sources_improved": int(np.sum(np.asarray(v["ratio"]) > 1.0)),
                               "plain_err": _quantiles(v["plain"]), "corrected_err": _quantiles(v["corrected"])}
                    for fH, v in per_f.items()},
        "spot_failed": rep["spot_failed"],
        "error_measure": "max |X - X_FP64full| / max |X_FP64full| over A, E, T on t <= t_H + T/2 (grid ends "
                         "excluded); own scale: A and E each on its own maximum; plain = lisa_response_hybrid "
                         "(mixed) at f_H, corrected = plain LFA below f_lo = f_H/2, corrected links to f_H, full after"}
    # cost on the headline workload: corrected (f_H/2, f_H) against plain at f_H
    n = src.n
    cost = {}
    for fH in F_H_EVAL:
        tHx = L.lisa_t_hyb_from_f(fH, src.mc_s, src.tc)
        tLx = L.lisa_t_hyb_from_f(F_LO_RATIO * fH, src.mc_s, src.tc)
        fp = lambda: L.lisa_response_hybrid(orbit, sky, src.grid, hp32, hc32, L.MIXED, 20, 0, L.AET, tHx, Tw, sig,   # noqa: E731
                                            src.grid, out32)
        fc = lambda: c.hybrid(orbit, sky, src.grid, hp32, hc32, 20, L.AET, tHx, Tw, sig, src.grid, out32,   # noqa: E731
                              t_lo=tLx)
        mp = _timed(torch, stream, flush, fp)
        torch.cuda.nvtx.range_push("corrected_hybrid_headline")   # range for targeted profiler captures
        mc = _timed(torch, stream, flush, fc)
        torch.cuda.nvtx.range_pop()
        cost["%g" % fH] = {"plain_ms": round(mp, 4), "corrected_ms": round(mc, 4), "cost_ratio": round(mc / mp, 3),
                           "corrected_samples_per_s": n / (mc / 1e3),
                           "corrected_zone_samples": int(max(0, min(n, math.floor((tHx - src.t0) / src.dt))
                                                            - max(0, math.ceil((tLx - src.t0) / src.dt))))}
        if fH == F_H_EVAL[0]:
            cost["%g" % fH]["kernels_ms"] = kernel_breakdown(L, torch, fc)
    res["headline_workload_cost"] = cost
    # the previous single-zone form (corrected links over the whole LFA side) for reference
    fo = lambda: c.hybrid(orbit, sky, src.grid, hp32, hc32, 20, L.AET, tH, Tw, sig, src.grid, out32)   # noqa: E731
    torch.cuda.nvtx.range_push("corrected_links_whole_lfa_side")   # range for targeted profiler captures
    res["corrected_links_whole_lfa_side_ms"] = round(_timed(torch, stream, flush, fo), 4)
    torch.cuda.nvtx.range_pop()
    # the fused tensor-core corrector over the whole LFA side: its MMA work
    # (padded shapes 48 -> 64 -> 64 -> 64 -> 16 per row) against the measured
    # bf16 GEMM rate
    kb = kernel_breakdown(L, torch, fo)
    res["corrected_links_whole_lfa_side_kernels_ms"] = kb
    if kb.get("corr_fused_tc"):
        rows = int(math.floor((tH + 0.5 * Tw - src.t0) / src.dt)) + 1
        rows = max(1, min(n, rows))
        flop = 2.0 * (48 * 64 + 2 * 64 * 64 + 64 * 16) * rows
        ach = flop / (kb["corr_fused_tc"] / 1e3) / 1e12
        pk = float(peaks().get("bf16_tflops", 1886.2))
        res["corr_fused_tc_roofline"] = {"bound": "tensor", "rows": rows, "flop_per_row": flop / rows,
                                         "achieved": round(ach, 2), "peak": pk, "unit": "TFLOP/s",
                                         "frac": round(ach / pk, 4),
                                         "peak_note": "bf16 GEMM burst rate, MEASURED_PEAKS.json; of measured"}
    rep = c.report()
    res["spot_checks"] = {k: rep[k] for k in ("spot_tiles", "spot_failed", "band_tiles", "fallback_tiles",
                                             "max_spot_err", "status")}
    return res, c


def mismatches(L, torch, dev, src, orbit, sky, hp64, hc64, hp32, hc32, gens=(20, 15), f_hybs=(3e-4, 1e-3),
               with_nlo=True):
    """The paper's accuracy criteria (Sec. V A) on this workload: mismatch
    1 - |O| of A, E, T (Eq. normalized_overlap; noise-weighted inner products
    of Eq. scalar_product with the analytic PSDs, band 1e-4 Hz to 0.02 Hz for
    TDI 2.0 and 0.05 Hz for TDI 1.5) of the hybrid (double-float, f_H = 3e-4
    and 1e-3 Hz), the LFA (double-float; next-to-leading order in FP64) and
    the mixed hybrid, each against the FP64 full response; and the mixed
    hybrid against the double-float hybrid."""
    n = src.n
    nfft = L.lisa_fft_length(n)
    nf = nfft // 2 + 1
    Tw, sig = 800 * src.dt, 20 * src.dt
    res = {}
    w = torch.empty((2, nf), device=dev, dtype=torch.float64)
    full = torch.empty((3, n), device=dev, dtype=torch.float64)
    x = torch.empty((3, n), device=dev, dtype=torch.float64)
    x32 = torch.empty((3, n), device=dev, dtype=torch.float32)
    ip = torch.empty(9, device=dev, dtype=torch.float64)

    def mm(a, b):
        L.lisa_inner_aet(src.grid, nfft, a, b, L.F64, w, ip)
        v = ip.cpu().numpy().reshape(3, 3)
        return [float(1.0 - abs(v[c, 0] / math.sqrt(v[c, 1] * v[c, 2]))) for c in range(3)]

    for gen in gens:
        f_max = 0.02 if gen == 20 else 0.05
        L.lisa_noise_weights_aet(src.grid, nfft, gen, ORBIT_KW.get("L_m", 2.5e9), 1.0, 1, 1e-4, f_max, w)
        L.lisa_response_full(orbit, sky, src.grid, hp64, hc64, L.F64, gen, L.AET, src.grid, full)
        r = {"band_hz": [1e-4, f_max]}
        for fh in f_hybs:
            tH = L.lisa_t_hyb_from_f(fh, src.mc_s, src.tc)
            L.lisa_response_hybrid(orbit, sky, src.grid, hp64, hc64, L.DF, gen, L.LFA_UNEQUAL, L.AET, tH, Tw, sig,
                                   src.grid, x)
            r["hybrid_df_fH_%g" % fh] = mm(full, x)
            if fh == f_hybs[-1]:
                L.lisa_response_hybrid(orbit, sky, src.grid, hp32, hc32, L.MIXED, gen, L.LFA_UNEQUAL, L.AET, tH, Tw,
                                       sig, src.grid, x32)
                xm = x32.double()
                r["hybrid_mixed_fH_%g" % fh] = mm(full, xm)
                r["hybrid_mixed_vs_hybrid_df_fH_%g" % fh] = mm(x, xm)
                del xm
        L.lisa_response_lfa(orbit, sky, src.grid, hp64, hc64, L.DF, gen, L.LFA_UNEQUAL, L.AET, src.grid, x)
        r["lfa_df"] = mm(full, x)
        if with_nlo and gen == 20:
            L.lisa_response_lfa(orbit, sky, src.grid, hp64, hc64, L.F64, gen, L.LFA_NLO, L.AET, src.grid, x)
            r["lfa_nlo_f64"] = mm(full, x)
        res["tdi%d" % gen] = r
    res["channels"] = "A, E, T"
    res["targets"] = ("Sec. V A: hybrid A,E < 1e-5 (1.5 and 2.0); LFA A,E < 1e-3 (1.5), < 1e-1 (2.0); "
                      "T: LFA 10-100 %, hybrid < 10 %")
    del w, full, x, x32, ip
    return res


def bench_loglike(L, torch, dev, src, orbit, sky, hp32, hc32, out32, flush, stream, tH, Tw, sig):
    """Log-likelihood evaluation as the paper times it (Sec. IV, steps ii-v
    on given polarisations): hybrid response -> A, E, T -> real FFTs ->
    noise-weighted inner products with fixed data d (here the response
    itself), ln L = -(<d|d> + <h|h> - 2<d|h>)/2, read back to the host."""
    n = src.n
    nfft = L.lisa_fft_length(n)          # zero padding to a 7-smooth length (fast transform)
    nf = nfft // 2 + 1
    f_min, f_max = 1e-4, 2.5e-2         # below the TDI 2.0 PSD zero at c/(4L) = 0.02998 Hz
    w = torch.empty((2, nf), device=dev, dtype=torch.float64)
    L.lisa_noise_weights_aet(src.grid, nfft, 20, ORBIT_KW.get("L_m", 2.5e9), 1.0, 1, f_min, f_max, w)
    d = torch.empty((3, n), device=dev, dtype=torch.float32)
    L.lisa_response_hybrid(orbit, sky, src.grid, hp32, hc32, L.MIXED, 20, L.LFA_UNEQUAL, L.AET, tH, Tw, sig,
                           src.grid, d)
    ip = torch.empty(9, device=dev, dtype=torch.float64)
    ip_h = torch.empty(9, dtype=torch.float64).pin_memory()

    def loglike():
        L.lisa_response_hybrid(orbit, sky, src.grid, hp32, hc32, L.MIXED, 20, L.LFA_UNEQUAL, L.AET, tH, Tw, sig,
                               src.grid, out32)
        L.lisa_inner_aet(src.grid, nfft, d, out32, L.MIXED, w, ip)
        ip_h.copy_(ip, non_blocking=True)

    for _ in range(3):
        loglike()
    torch.cuda.synchronize()
    L.lisa_profile_enable(False)
    L.lisa_profile_enable(True)
    ms = []
    for _ in range(10):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        loglike()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    inner_ms, inner_n = L.lisa_profile_query("inner_aet")
    L.lisa_profile_enable(False)
    v = ip_h.numpy().reshape(3, 3)
    lnl = [float(-0.5 * (v[c, 1] + v[c, 2] - 2.0 * v[c, 0])) for c in range(3)]
    snr = [float(np.sqrt(max(v[c, 1], 0.0))) for c in range(3)]
    best = float(np.median(ms))
    return {"ms": round(best, 4), "evaluations_per_s": round(1e3 / best, 1),
            "inner_ms": round(inner_ms / max(inner_n, 1), 4),
            "steps": "hybrid response (A, E, T) + 2 x 3 real FFTs (cuFFT, rows zero-padded to %d) + weighted inner "
                     "products + 9-value read-back" % nfft,
            "band_hz": [f_min, f_max], "ln_L_per_channel": lnl, "snr_per_channel_of_d": snr,
            "note": "d = the same response, so ln L = 0 up to FP32 rounding of the repeated evaluation"}


def bench_batch(L, torch, dev, orbit, flush, stream, args, fma_peaks=None):
    """Batched hybrid plan over the seeded config-3 population (Mc log-U
    [1e4, 1e7], q U[1, 10], 1 day to 3 months at 5 or 10 s): one persistent
    launch, autotuned tiles, captured graph."""
    import synth
    params = synth.batch_params(nsrc=args.batch_sources, seed=synth.SEED_BASE + 3)
    t0 = time.perf_counter()
    descs = []
    total = 0
    n_lfa = n_full = 0   # samples each part computes (the blend window's in both)
    for p in params:
        s = synth.batch_source(p)
        tHs = L.lisa_t_hyb_from_f(F_HYB, s.mc_s, s.tc)
        descs.append(dict(grid=s.grid, hp=torch.as_tensor(s.hp.astype(np.float32), device=dev),
                          hc=torch.as_tensor(s.hc.astype(np.float32), device=dev),
                          sky=(s.beta, s.lam, s.psi), t_hyb=tHs, out=torch.empty((3, s.n), device=dev)))
        total += s.n
        half_w = 400 * s.dt      # the plan's default window, 800 samples
        i_l = int(math.floor((tHs + half_w - s.t0) / s.dt))
        i_f = int(math.ceil((tHs - half_w - s.t0) / s.dt))
        n_lfa += min(s.n, max(0, i_l + 1))
        n_full += min(s.n, max(0, s.n - max(0, i_f)))
    t_gen = time.perf_counter() - t0
    plan = L.LisaPlan(orbit, descs)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        tune = plan.autotune(stream=st.cuda_stream)
        plan.capture_graph(st.cuda_stream)
        fn = lambda: plan.replay(stream=st.cuda_stream)   # noqa: E731
        torch.cuda.nvtx.range_push("batched_replay")       # range for targeted profiler captures
        ms = _timed(torch, st, flush, fn, reps=5)
        torch.cuda.nvtx.range_pop()
    plan.close()
    res = {"sources": len(descs), "samples": total, "ms": round(ms, 3), "samples_per_s": total / (ms / 1e3),
           "autotune": tune, "source_generation_s": round(t_gen, 1),
           "workload": "hybrid TDI2.0 AET, f_hyb=1e-3 Hz, mixed precision, one persistent launch (graph replay)"}
    res["lfa_samples"], res["full_samples"] = n_lfa, n_full
    if fma_peaks:
        # the hybrid's taps-and-stencils work: LFA samples at the LFA's flop,
        # full-response samples at the full TDI 2.0's (the blend window's samples
        # in both, as computed)
        flop = LFA_TAPS_FLOP * n_lfa + FULL20_TAPS_FLOP * n_full
        ach = flop / (ms / 1e3) / 1e12
        res["roofline"] = {"bound": "alu", "achieved": round(ach, 3), "peak": round(fma_peaks["fp32_tflops"], 2),
                           "unit": "TFLOP/s", "frac": round(ach / fma_peaks["fp32_tflops"], 4),
                           "flop_per_sample": round(flop / max(total, 1), 1),
                           "flop_note": "%d flop per LFA sample, %d per full-response sample (taps and stencils)"
                                        % (LFA_TAPS_FLOP, FULL20_TAPS_FLOP),
                           "peak_note": "FP32 FMA, measured in this run (lisa_peak_fma); of measured"}
    return res


def bench_pe_draws(L, torch, dev, orbit, stream, args, corr=None):
    """Config 5: PE draws around Mc = 5e5 Msun, q = 2 (eccentric), one year at
    10 s each, generated on the device (lisa_chirp_ringdown) and put through the
    hybrid response, a chunk of draws at a time (generation into one buffer,
    then one batched persistent plan per chunk).  Plans are built before the
    timed region; the timed region covers generation and response of every
    draw."""
    import synth
    ndraw, chunk = args.pe_draws, min(args.pe_chunk, args.pe_draws)
    n, dt, t0 = 3155760, 10.0, 2.0e7
    tc = t0 + n * dt - 1.0e4
    ps = synth.pe_params(ndraw=ndraw)
    draws = [dict(mc_s=p["mc"] * synth.T_SUN, q=p["q"], dist_m=10.0 * synth.GPC, iota=0.5, phi_c=p["phi_c"], tc=tc,
                  e0=p["e0"], f_cut=0.8 * 0.5 / dt) for p in ps]
    hp = torch.empty((chunk, n), device=dev)
    hc = torch.empty((chunk, n), device=dev)
    out = torch.empty((chunk, 3, n), device=dev)
    t_setup = time.perf_counter()
    plans = []
    for c0 in range(0, ndraw, chunk):
        descs = []
        for k, d in enumerate(draws[c0:c0 + chunk]):
            p = ps[c0 + k]
            descs.append(dict(grid=(t0, dt, n), hp=hp[k], hc=hc[k], sky=(p["beta"], p["lam"], p["psi"]),
                              t_hyb=L.lisa_t_hyb_from_f(F_HYB, d["mc_s"], tc), out=out[k]))
        plans.append((c0, L.LisaPlan(orbit, descs)))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup

    def run_all():
        for c0, plan in plans:
            part = draws[c0:c0 + chunk]
            L.lisa_chirp_ringdown(part, (t0, dt, n), L.MIXED, hp[:len(part)], hc[:len(part)],
                                  stream=stream.cuda_stream)
            plan.execute(stream=stream.cuda_stream)

    def gen_only():
        for c0, _ in plans:
            part = draws[c0:c0 + chunk]
            L.lisa_chirp_ringdown(part, (t0, dt, n), L.MIXED, hp[:len(part)], hc[:len(part)],
                                  stream=stream.cuda_stream)

    with torch.cuda.stream(stream):
        run_all()
        torch.cuda.synchronize()
        ms = []
        for _ in range(2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            run_all()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        gen_only()
        b.record(stream)
        b.synchronize()
        gen_ms = a.elapsed_time(b)
    best = float(np.median(ms))
    finite = bool(torch.isfinite(out).all().item())
    for _, plan in plans:
        plan.close()
    total = ndraw * n
    res = {"draws": ndraw, "samples_per_draw": n, "samples": total,
           "plain_batched": {"ms": round(best, 2), "draws_per_s": ndraw / (best / 1e3),
                             "samples_per_s": total / (best / 1e3), "generation_ms": round(gen_ms, 2),
                             "generation_share": round(gen_ms / best, 4), "chunk": chunk,
                             "plan_setup_s": round(t_setup, 2), "outputs_finite": finite,
                             "form": "plain hybrid TDI 2.0 A/E/T (f_H = 1e-3 Hz), one batched persistent plan per chunk"}}
    if corr is not None:
        res["corrected"] = pe_corrected(L, torch, dev, orbit, stream, ps, draws, (t0, dt, n), chunk, hp, hc, out, corr)
    del hp, hc, out
    res["workload"] = ("config 5: eccentric chirp + ringdown draws (Mc 5e5 Msun, q 2, e0 U[0, 0.3]), 1 yr at 10 s, "
                       "generated on the device (mixed) + hybrid TDI 2.0 A/E/T")
    return res


def pe_corrected(L, torch, dev, orbit, stream, ps, draws, grid, chunk, hp, hc, out, corr, n_check=16):
    """Config 5 with the learned corrector: every draw generated on the device
    and put through the corrected hybrid (plain LFA below f_H/2, corrected
    links to f_H = 1e-3 Hz, full response after), timed over all draws; on
    n_check draws spread over the set, the corrected and the plain hybrid
    against the FP64 full response of the same waveform on the same GPU
    (sample errors on the approximate side and A/E/T mismatches)."""
    t0, dt, n = grid
    ndraw = len(draws)
    Tw, sig = 800 * dt, 20 * dt
    zones = [(L.lisa_t_hyb_from_f(F_LO_RATIO * F_HYB, d["mc_s"], d["tc"]), L.lisa_t_hyb_from_f(F_HYB, d["mc_s"], d["tc"]))
             for d in draws]
    skies = [(p["beta"], p["lam"], p["psi"]) for p in ps]
    st = stream.cuda_stream

    def run_all():
        for c0 in range(0, ndraw, chunk):
            part = draws[c0:c0 + chunk]
            L.lisa_chirp_ringdown(part, grid, L.MIXED, hp[:len(part)], hc[:len(part)], stream=st)
            for k in range(len(part)):
                tl, th = zones[c0 + k]
                corr.hybrid(orbit, skies[c0 + k], grid, hp[k], hc[k], 20, L.AET, th, Tw, sig, grid, out[k], stream=st,
                            t_lo=tl)

    corr.report()
    with torch.cuda.stream(stream):
        run_all()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run_all()
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
    rep = corr.report()
    finite = bool(torch.isfinite(out).all().item())
    # accuracy on a spread of draws against the FP64 full response
    nfft = L.lisa_fft_length(n)
    w = torch.empty((2, nfft // 2 + 1), device=dev, dtype=torch.float64)
    L.lisa_noise_weights_aet(grid, nfft, 20, 2.5e9, 1.0, 1, 1e-4, 2e-2, w)
    ip = torch.empty(9, device=dev, dtype=torch.float64)
    full = torch.empty((3, n), device=dev, dtype=torch.float64)
    hyb = torch.empty((3, n), device=dev)
    m0 = int(math.ceil((1.01 * 499.0048 + 100.0 + 20.0 * dt) / dt)) + 4

    def errs(x, i_end):
        d = (x[:, m0:i_end].double() - full[:, m0:i_end]).abs().amax(dim=1)
        own = full[:, m0:i_end].abs().amax(dim=1)
        return (d / own.max()).max().item(), (d / own).tolist()

    def mism(x):
        L.lisa_inner_aet(grid, nfft, full, x.double().contiguous(), L.F64, w, ip)
        v = ip.cpu().numpy().reshape(3, 3)
        return [float(1.0 - abs(v[c, 0] / math.sqrt(v[c, 1] * v[c, 2]))) for c in range(3)]

    picks = sorted(set(int(round(x)) for x in np.linspace(0, ndraw - 1, n_check)))
    rows = []
    for j in picks:
        d = draws[j]
        h1 = torch.empty((1, n), device=dev)
        h2 = torch.empty((1, n), device=dev)
        L.lisa_chirp_ringdown([d], grid, L.MIXED, h1, h2)
        H1, H2 = h1[0].double().contiguous(), h2[0].double().contiguous()
        L.lisa_response_full(orbit, skies[j], grid, H1, H2, L.F64, 20, L.AET, grid, full)
        tl, th = zones[j]
        i_end = int(min(n, max(0, math.floor((th + Tw / 2 - t0) / dt) + 1)))
        corr.hybrid(orbit, skies[j], grid, h1[0], h2[0], 20, L.AET, th, Tw, sig, grid, hyb, t_lo=tl)
        ec, ec_own = errs(hyb, i_end)
        mc = mism(hyb)
        L.lisa_response_hybrid(orbit, skies[j], grid, h1[0], h2[0], L.MIXED, 20, 0, L.AET, th, Tw, sig, grid, hyb)
        ep, ep_own = errs(hyb, i_end)
        mp = mism(hyb)
        rows.append(dict(draw=j, e0=d["e0"], corrected_err=ec, plain_err=ep, corrected_err_own_AET=ec_own,
                         plain_err_own_AET=ep_own, corrected_mismatch_AET=mc, plain_mismatch_AET=mp))
    rep2 = corr.report()
    ratio = [r["plain_err"] / r["corrected_err"] for r in rows]
    return {"ms": round(ms, 2), "draws_per_s": ndraw / (ms / 1e3), "samples_per_s": ndraw * n / (ms / 1e3),
            "outputs_finite": finite, "f_H": F_HYB, "f_lo": F_LO_RATIO * F_HYB,
            "spot_checks": {k: rep[k] for k in ("spot_tiles", "spot_failed", "band_tiles", "fallback_tiles",
                                               "max_spot_err", "status")},
            "vs_fp64_full": {"draws_checked": len(rows), "plain_over_corrected_err": _quantiles(ratio),
                             "corrected_err": _quantiles([r["corrected_err"] for r in rows]),
                             "plain_err": _quantiles([r["plain_err"] for r in rows]),
                             "corrected_mismatch_AE_max": max(max(r["corrected_mismatch_AET"][:2]) for r in rows),
                             "plain_mismatch_AE_max": max(max(r["plain_mismatch_AET"][:2]) for r in rows),
                             "spot_failed": rep2["spot_failed"], "per_draw": rows,
                             "measure": "FP64 full response of the same (device-generated FP32) waveform; errors: "
                                        "max |X - X_full| / max |X_full| on t <= t_H + T/2 (grid start excluded), "
                                        "largest channel and each channel on its own maximum; mismatch 1 - |O| "
                                        "with the TDI 2.0 PSDs over 1e-4..2e-2 Hz (Sec. V A)"}}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2505_09600_gb300 as L
    from paper_2505_09600_gb300 import build as B

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    L.load()
    dev = torch.device("cuda", torch.cuda.current_device())

    src = make_source(rank)
    n = src.n
    sky = (src.beta, src.lam, src.psi)
    orbit = L.Orbit(**ORBIT_KW)
    tH = L.lisa_t_hyb_from_f(F_HYB, src.mc_s, src.tc)
    Tw, sig = 800 * src.dt, 20 * src.dt
    hp32 = torch.as_tensor(src.hp.astype(np.float32), device=dev)
    hc32 = torch.as_tensor(src.hc.astype(np.float32), device=dev)
    out32 = torch.empty((3, n), device=dev, dtype=torch.float32)
    hp64 = torch.as_tensor(src.hp, device=dev)
    hc64 = torch.as_tensor(src.hc, device=dev)
    out64 = torch.empty((3, n), device=dev, dtype=torch.float64)
    flush = torch.empty(2 * L2_BYTES // 4, device=dev, dtype=torch.float32)
    stream = torch.cuda.current_stream()
    fma_peaks = measured_fma_peaks(L)
    prec = REC_PRECISION

    def step():
        # the line of record: FP64 inputs and outputs, FP64-accurate arithmetic
        L.lisa_response_hybrid(orbit, sky, src.grid, hp64, hc64, prec, 20, L.LFA_UNEQUAL, L.AET, tH, Tw, sig,
                               src.grid, out64)

    def step_mixed():
        L.lisa_response_hybrid(orbit, sky, src.grid, hp32, hc32, L.MIXED, 20, L.LFA_UNEQUAL, L.AET, tH, Tw, sig,
                               src.grid, out32)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(dev.index)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    L.lisa_profile_enable(True)
    launches0 = L.lisa_launch_count()
    for k in range(args.steps):
        flush.zero_()                      # evict L2 between steps (outside the timed events)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    launches = L.lisa_launch_count() - launches0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    lfa_ms, lfa_launches = L.lisa_profile_query(REC_KERNEL[prec])
    L.lisa_profile_enable(False)

    # The same call captured once in a CUDA graph (its stream-ordered
    # allocations, side-stream fork and join and kernels as graph nodes) and
    # replayed K times: reported beside the line, which times the calls.
    graph_ms = None
    try:
        gs = torch.cuda.Stream()
        gs.wait_stream(stream)
        with torch.cuda.stream(gs):
            step()
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=gs):
            step()
        torch.cuda.synchronize()
        for _ in range(args.warmup):
            graph.replay()
        gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()
            gev[k][0].record(stream)
            graph.replay()
            gev[k][1].record(stream)
        torch.cuda.synchronize()
        graph_ms = round(float(np.median([a.elapsed_time(b) for a, b in gev])), 5)
        del graph
    except Exception as e:   # capture refused: reported as such
        graph_ms = "capture failed: %s" % type(e).__name__
        torch.cuda.synchronize()
    total_ms = max_over_ranks(float(sum(step_ms)), world, dev)
    value = whole_job_rate(world, n, args.steps, total_ms)

    # end to end through the public call on host buffers (page-locked): the
    # host->device copies of h and the device->host copy of A, E, T are inside
    # the timed region (the library overlaps them with its kernels in chunks)
    hp_h = torch.as_tensor(src.hp).pin_memory()
    hc_h = torch.as_tensor(src.hc).pin_memory()
    out_h = torch.empty((3, n), dtype=torch.float64).pin_memory()
    e2e_ms = []
    for k in range(args.warmup + args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        L.lisa_response_hybrid_host(orbit, sky, src.grid, hp_h, hc_h, prec, 20, L.LFA_UNEQUAL, L.AET, tH, Tw, sig,
                                    out_h, stream=stream.cuda_stream)
        b.record(stream)
        b.synchronize()
        if k >= args.warmup:
            e2e_ms.append(a.elapsed_time(b))
    # the host-buffer call returns what the device call returns (the TDI blocks
    # follow its chunks: FP32 rounding)
    ref = out64.cpu()
    e2e_diff = float((out_h - ref).abs().max() / ref.abs().max().clamp_min(1e-300))
    e2e_total = max_over_ranks(float(sum(e2e_ms)), world, dev)
    e2e_value = whole_job_rate(world, n, len(e2e_ms), e2e_total)

    # other forms (same source), fewer steps
    forms = {}
    if not args.no_forms:
        cases = {
            "hybrid20_mixed": lambda: step_mixed(),
            "lfa20_mixed": lambda: L.lisa_response_lfa(orbit, sky, src.grid, hp32, hc32, L.MIXED, 20, 0, L.AET,
                                                       src.grid, out32),
            "full20_mixed": lambda: L.lisa_response_full(orbit, sky, src.grid, hp32, hc32, L.MIXED, 20, L.AET,
                                                         src.grid, out32),
            "hybrid20_f64": lambda: L.lisa_response_hybrid(orbit, sky, src.grid, hp64, hc64, L.F64, 20, 0, L.AET, tH,
                                                           Tw, sig, src.grid, out64),
            "lfa20_df": lambda: L.lisa_response_lfa(orbit, sky, src.grid, hp64, hc64, L.DF, 20, 0, L.AET,
                                                    src.grid, out64),
            "lfa20_f64": lambda: L.lisa_response_lfa(orbit, sky, src.grid, hp64, hc64, L.F64, 20, 0, L.AET,
                                                     src.grid, out64),
            "full20_f64": lambda: L.lisa_response_full(orbit, sky, src.grid, hp64, hc64, L.F64, 20, L.AET,
                                                       src.grid, out64),
        }
        if args.forms:
            keep = args.forms.split(",")
            cases = {k: v for k, v in cases.items() if k in keep}
        # per-kernel rooflines of the forms: algorithmic flop per sample (Lagrange
        # taps, 2 flop each, and stencils; weights not counted) against the
        # measured FMA peak of the pipe the kernel runs on
        kern_flop = {"lfa_mixed": LFA_TAPS_FLOP, "lfa_f64": LFA_TAPS_FLOP,
                     "links_full_mixed": 12 * 2 * TAP, "links_full_f64": 12 * 2 * TAP,
                     "tdi_mixed": 48 * TAP, "tdi_f64": 48 * TAP, "lfa_df": LFA_TAPS_FLOP}
        # the TDI kernels run combined per-link filters: per sample, 6 links x
        # 44 taps (a link's terms span up to 7 light times, 12 samples at 5 s,
        # plus the 32-point stencil, rounded up to 4) x 4 multiply-adds (value
        # and drift of two channels; the FP64 form's FP32 di^2, di^3 sums not
        # counted); this executed count is reported beside the definition's
        kern_exec_flop = {"tdi_mixed": 6 * 44 * 8, "tdi_f64": 6 * 44 * 8}
        for name, fn in cases.items():
            torch.cuda.nvtx.range_push("form_" + name)   # range for targeted profiler captures
            fn()
            torch.cuda.synchronize()
            reps = 3
            ms = []
            L.lisa_profile_enable(True)
            for _ in range(reps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            torch.cuda.nvtx.range_pop()
            best = float(np.median(ms))
            forms[name] = {"ms": round(best, 4), "samples_per_s": n / (best / 1e3)}
            roofs = {}
            for kn, fl in kern_flop.items():
                kms, kcnt = L.lisa_profile_query(kn)
                if not kcnt:
                    continue
                avg = kms / kcnt
                pk64 = kn.endswith("_f64")
                if name.startswith(("lfa", "full")):
                    units = n
                elif kn.startswith("lfa"):
                    # the hybrid's LFA part: samples t <= t_H + T/2
                    units = int(math.floor((tH + 0.5 * Tw - src.t0) / src.dt)) + 1
                else:
                    # the hybrid's full part: TDI on t >= t_H - T/2, links from
                    # 8 light times (+40 samples) earlier, as the library holds them
                    i_f = max(0, int(math.ceil((tH - 0.5 * Tw - src.t0) / src.dt)))
                    lo = max(0, i_f - int(math.ceil(8.0 * 1.01 * 2.5e9 / 299792458.0 / src.dt)) - 40)
                    units = n - (lo if kn.startswith("links") else i_f)
                ach = fl * units / (avg / 1e3) / 1e12
                pk = fma_peaks["fp64_tflops"] if pk64 else fma_peaks["fp32_tflops"]
                roofs[kn] = {"avg_launch_ms": round(avg, 5), "achieved_tflops": round(ach, 4),
                             "peak_tflops": round(pk, 3), "frac": round(ach / pk, 4),
                             "peak": ("FP64" if pk64 else "FP32") + " FMA, measured (lisa_peak_fma)",
                             "flop_per_sample": fl, "samples_per_launch": units}
                if kn in kern_exec_flop:
                    ex = kern_exec_flop[kn] * units / (avg / 1e3) / 1e12
                    roofs[kn].update({"flop_note": "flop_per_sample: the definition (48 interpolations of 32 "
                                      "taps); executed: the combined filters", "executed_flop_per_sample":
                                      kern_exec_flop[kn], "executed_tflops": round(ex, 4),
                                      "executed_frac": round(ex / pk, 4)})
            L.lisa_profile_enable(False)
            if roofs:
                forms[name]["roofline"] = roofs
        if "full20_f64" in cases:
            # expansion point of the LFA link (App. B): the central point against
            # the non-central backward / forward variants, mixed A/E/T, error
            # against the FP64 full response on the LFA side of the switch (t <= t_H)
            ref_aet = out64   # the full20_f64 case ran last: FP64 full response, A/E/T
            i_h = int(math.floor((tH - src.t0) / src.dt)) + 1
            # the first samples see the step of h at the grid start through delays of up to
            # |k.R|/c: excluded, as in the corrector's error measure
            m0 = int(math.ceil((1.01 * 499.0048 + 100.0 + 20.0 * src.dt) / src.dt)) + 4
            ref_aet = ref_aet[:, m0:]
            i_h -= m0
            scale = ref_aet[:, :i_h].abs().max().item()
            points = {}
            out64b = torch.empty_like(out64)
            kinds = (("central", L.LFA_UNEQUAL, L.MIXED), ("backward", L.LFA_BACKWARD, L.MIXED),
                     ("forward", L.LFA_FORWARD, L.MIXED), ("strain_R0", L.LFA_STRAIN, L.MIXED),
                     ("central_f64", L.LFA_UNEQUAL, L.F64), ("nlo_f64", L.LFA_NLO, L.F64),
                     ("strain_R0_f64", L.LFA_STRAIN, L.F64))
            for pname, kind, pr in kinds:
                o_ = out32 if pr == L.MIXED else out64b
                h_ = (hp32, hc32) if pr == L.MIXED else (hp64, hc64)
                fn = lambda: L.lisa_response_lfa(orbit, sky, src.grid, h_[0], h_[1], pr, 20, kind, L.AET, src.grid, o_)
                best = _timed(torch, stream, flush, fn)
                d = (o_[:, m0:m0 + i_h].double() - ref_aet[:, :i_h]).abs().amax(dim=1)
                own = ref_aet[:, :i_h].abs().amax(dim=1).clamp_min(1e-300)
                points[pname] = {"ms": round(best, 4), "samples_per_s": n / (best / 1e3),
                                 "err_aet_vs_full_f64": (d / scale).tolist(), "err_aet_vs_full_f64_own": (d / own).tolist()}
            del out64b
            forms["lfa20_kinds_vs_full"] = {
                "points": points, "range": "t <= t_H (LFA side), grid start excluded (%d samples); errors / max |A,E,T| of the FP64 full response there (own: each channel on its own maximum)" % m0,
                "note": "central: Eq. tau_t_dependence; backward / forward: App. B non-central variants; nlo: App. B next-to-leading order (link m = 1 term and next Michelson term); strain_R0: Sec. III strain-derivative form with the constellation centre (Eqs. X15/X20_with_strain_derivatives)"}

    # the headline step's output, for the oracle comparison below, and the mixed form's
    step()
    torch.cuda.synchronize()
    keep_out = rank == 0 and world == 1 and not args.no_cpu
    gpu_out = out64.cpu().numpy() if keep_out else None
    step_mixed()
    torch.cuda.synchronize()
    gpu_out_mixed = out32.float().cpu().numpy().astype(np.float64) if keep_out else None

    corrector, corr_obj = None, None
    if not args.no_corrector and rank == 0:
        corrector, corr_obj = bench_corrector(L, torch, dev, src, orbit, sky, hp32, hc32, out32, flush, stream, tH, Tw,
                                              sig)
    mism = None
    if not args.no_mismatch and rank == 0:
        mism = mismatches(L, torch, dev, src, orbit, sky, hp64, hc64, hp32, hc32)
    loglike = None
    if not args.no_loglike and rank == 0:
        loglike = bench_loglike(L, torch, dev, src, orbit, sky, hp32, hc32, out32, flush, stream, tH, Tw, sig)
    batched = None
    if not args.no_batch and rank == 0:
        batched = bench_batch(L, torch, dev, orbit, flush, stream, args, fma_peaks)
    pe_draws = None
    if not args.no_pe and rank == 0:
        pe_draws = bench_pe_draws(L, torch, dev, orbit, stream, args, corr=corr_obj)
    if corr_obj is not None:
        corr_obj.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    pk = peaks()
    flop = LFA_TAPS_FLOP
    lfa_avg_ms = lfa_ms / max(lfa_launches, 1)
    # samples the LFA kernel covers per launch: t <= t_hyb + T/2
    i_l = int(math.floor((tH + 0.5 * Tw - src.t0) / src.dt)) + 1
    if prec == 2:
        # double-float: FP32 operations per sample against the FP32 pipe's
        # measured operation rate (one FMA per lane per cycle = flop / 2)
        ops = DF_OPS_PER_SAMPLE["lfa20"]
        achieved = ops * i_l / (lfa_avg_ms / 1e3) / 1e12
        peak = fma_peaks["fp32_tflops"] / 2.0
        roof = {"bound": "alu", "kernel": "lfa_df (FP32 pipe, double-float arithmetic)",
                "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "T FP32 op/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "peak_note": "FP32 FMA instruction rate measured in this run by lisa_peak_fma (TFLOP/s / 2); "
                             "of measured",
                "ops_per_sample": ops, "ops_note": "FP32 add/mul/fma of the double-float algorithm, one each "
                "(weights, taps, positions, projection factors, stencils); FP64 set-up and hdot staging not counted",
                "taps_flop_view": {"flop_per_sample": flop, "achieved_tflops":
                                   round(flop * i_l / (lfa_avg_ms / 1e3) / 1e12, 4)}}
    else:
        achieved = flop * i_l / (lfa_avg_ms / 1e3) / 1e12
        peak = fma_peaks["fp64_tflops"]
        roof = {"bound": "alu", "kernel": "%s (FP64 pipe)" % REC_KERNEL[prec],
                "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "peak_note": "FP64 FMA throughput measured in this run by lisa_peak_fma (project microbenchmark); "
                             "of measured",
                "flop_per_sample": flop, "flop_note": "Lagrange taps (2 flop/tap) + stencils; weights not counted"}
    roof.update({"samples_per_launch": i_l, "avg_launch_ms": round(lfa_avg_ms, 5),
            "share_of_step": round(lfa_ms / max(float(sum(step_ms)), 1e-9), 4),
            "hbm_gbs": round(40 * i_l / (lfa_avg_ms / 1e3) / 1e9, 1),
            "hbm_frac_of_measured": round(40 * i_l / (lfa_avg_ms / 1e3) / 1e9 / float(pk.get("hbm_gbs", 6800.0)), 4)})
    tr = committed_traffic(REC_KERNEL[prec])
    if tr is not None:
        roof["traffic"] = tr
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": REC_DTYPE[prec], "data": "synthetic",
        "config": {"workload": WORKLOAD_BASE + ", FP64 inputs and outputs, " + (
                               "double-float LFA (FP32 pairs), FP64 full part" if prec == 2 else "FP64 arithmetic"),
                   "precision_of_record": REC_DTYPE[prec],
                   "n_samples": n, "dt": src.dt, "sources_per_gpu": 1, "l2": "flushed between steps "
                   "(256 MiB write outside the timed events)", "parallelism": "replicas" if world > 1 else "single",
                   "timing": "library call per step",
                   "graph_replay_ms_per_step_median": graph_ms},
        "roofline": roof,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * n * 8, "d2h_bytes_per_step": 3 * n * 8,
                "call": "lisa_response_hybrid_host (page-locked host buffers, copies overlapped in chunks)",
                "max_rel_diff_vs_device_call": e2e_diff},
        "gpu_launches": int(launches),
        "clocks": clk,
        "forms": forms,
        "fma_peaks_measured": fma_peaks,
        "gpu_name": torch.cuda.get_device_name(dev),
    }
    if corrector is not None:
        line["corrector"] = corrector
    if batched is not None:
        line["batched"] = batched
    if pe_draws is not None:
        line["pe_draws"] = pe_draws
    if loglike is not None:
        line["loglike"] = loglike
    if mism is not None:
        line["mismatch"] = mism
    if not args.no_cpu and world == 1:
        cb = oracle_hybrid_rate(src, budget_s=args.cpu_budget, one_core=True)
        er = sampled_errors(src, gpu_out, fp32_inputs=False, chunk=cb.get("chunk"))
        er["tolerance"] = "A,E,T <= 5e-12 of the largest channel and A,E on their own scale; T on its own <= 1e-10"
        cb["gpu_err_sampled"] = er
        line["cpu_baseline"] = cb
        em = sampled_errors(src, gpu_out_mixed, fp32_inputs=True, chunk=cb.get("chunk"))
        em["tolerance"] = ("A,E,T <= 3e-5 of the largest channel and A,E on their own scale; T on its own <= 5e-4 "
                           "(tests/tolerances.py, hybrid20)")
        forms.setdefault("hybrid20_mixed", {})["err_sampled"] = em
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_reference(args):
    """The oracle (the only reference implementation of this method) on the
    host cores.  Each step times a bounded sample of the same workload (the
    oracle LFA on a contiguous chunk grown to about budget/2 s, and the full
    response on its whole region); the step's rate is the workload's samples
    over the time extrapolated from that sample, and ms_per_step is the
    measured time of the sample itself.  Warm-up steps run a small sample
    untimed."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    src = make_source(0)
    for _ in range(args.warmup):
        oracle_hybrid_rate(src, budget_s=0.0)
    rates, secs = [], []
    cb = None
    for k in range(max(1, args.steps)):
        cb = oracle_hybrid_rate(src, budget_s=args.cpu_budget / max(1, args.steps) + 2.0)
        rates.append(cb["value"])
        secs.append(cb["seconds"])
    value = float(np.median(rates))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.median(secs)) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_BASE + ", FP64 CPU oracle", "n_samples": src.n,
                       "step": "a bounded sample of the workload (" + cb["sample"] + "); value = the workload's "
                               "samples over the time extrapolated from the sample; ms_per_step = the sample's "
                               "measured time"},
            "cpu_baseline": dict(cb, value=value),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--forms", default="", help="comma-separated subset of the forms section (profiling aid)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-corrector", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-loglike", action="store_true")
    ap.add_argument("--no-mismatch", action="store_true")
    ap.add_argument("--batch-sources", type=int, default=1024)
    ap.add_argument("--no-pe", action="store_true")
    ap.add_argument("--pe-draws", type=int, default=4096)
    ap.add_argument("--pe-chunk", type=int, default=256)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


def oracle_one_core():
    """The oracle legs of oracle_hybrid_rate on one core: the LFA on a
    20,000-sample chunk, extrapolated, plus the full response on its whole
    region.  Must run in a process started with OMP_NUM_THREADS=1."""
    if os.environ.get("OMP_NUM_THREADS") != "1":
        raise SystemExit("--oracle-one-core needs OMP_NUM_THREADS=1 in the environment")
    src = make_source(0)
    r = oracle_hybrid_rate(src, budget_s=0.0)
    print(json.dumps({"value": r["value"], "unit": r["unit"], "cores": 1, "sample": r["sample"]}))


if __name__ == "__main__":
    if "--oracle-one-core" in sys.argv:
        oracle_one_core()
        sys.exit(0)
    main()
