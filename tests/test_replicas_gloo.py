"""Multi-rank host logic of the benchmark, on CPU with the gloo backend.

Sources are independent, so N GPUs run N replicas with no exchange on the data
path; the only collective is the max over ranks of the timed region.  These
tests run that logic as two gloo processes (world size 2) and check:
  * the reduced time is the slowest rank's and every rank sees it;
  * the whole-job rate counts every rank's samples against that time;
  * each rank draws its own source (different sky and phase, same grid);
  * the reference arm runs on rank 0 only.
"""
import io
import os
import socket
import sys
import types
from contextlib import redirect_stdout

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    import synth

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, loc = bench.dist_env()
        ms = 10.0 + 7.5 * rank
        total = bench.max_over_ranks(ms, w, torch.device("cpu"))
        rate = bench.whole_job_rate(w, 1000, 4, total)
        src = synth.cfg2_small(n=4096, seed_offset=r)
        geo = [None] * w
        dist.all_gather_object(geo, (src.n, src.dt, src.t0, src.beta, src.lam, src.psi, float(src.hp[100])))
        q.put((r, w, loc, total, rate, geo))
    finally:
        dist.destroy_process_group()


def test_two_replicas_timing_and_sources():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for r, (rank, world, loc, total, rate, geo) in enumerate(res):
        assert (rank, world, loc) == (r, 2, r)
        assert total == pytest.approx(17.5)                   # the slower rank
        assert rate == pytest.approx(2 * 1000 * 4 / 17.5e-3)  # both ranks' samples
        assert geo == res[0][5]                               # every rank saw the same gather
    g0, g1 = res[0][5]
    assert g0[:3] == g1[:3]                                   # same grid
    assert g0[3:] != g1[3:]                                   # own sky, phase and waveform


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25, 1, None) == 3.25
    assert bench.whole_job_rate(1, 6311520, 20, 16.0) == pytest.approx(6311520 * 20 / 0.016)


def test_reference_arm_only_on_rank0(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    called = []
    monkeypatch.setattr(bench, "make_source", lambda rank: called.append(rank))
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(types.SimpleNamespace(steps=2, warmup=3, cpu_budget=1.0))
    assert buf.getvalue() == "" and called == []
