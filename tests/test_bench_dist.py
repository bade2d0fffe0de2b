"""The multi-rank path of bench.py (replicas, barrier, max of the step time
over ranks) on CPU with the gloo backend, world size 2."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    bench.barrier(w)
    m = bench.reduce_max(10.0 + 5.0 * rank, w)
    out[rank] = (r, w, m)
    dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == (0, 2, 15.0)
    assert out[1] == (1, 2, 15.0)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    bench.barrier(1)


def test_reference_arm_line_shape(monkeypatch):
    """The reference arm (the FP64 oracle on the host) prints the same metric."""
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, gpus = 1, 0, 1
    line = bench.run_reference(A, 0, 1)
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["e2e"]["h2d_bytes_per_step"] == 0
    assert bench.run_reference(A, 1, 2) is None


def test_serve_trace_from_timestamps():
    """The serving record's trace: admission spacing, batches grouped by launch
    time, and the part of the span with a batch in flight (a union of the
    batches' intervals, overlapping ones counted once)."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    # (submitted, admitted, launched, completed) in seconds; three batches:
    # launched at 2 ms (two requests, done by 6 ms), at 4 ms (overlapping the
    # first, done at 8 ms) and at 9 ms (done at 10 ms)
    t = np.array([[0.000, 0.001, 0.002, 0.005],
                  [0.000, 0.0015, 0.002, 0.006],
                  [0.000, 0.003, 0.004, 0.008],
                  [0.001, 0.004, 0.009, 0.010]])
    tr = bench.serve_trace(t, 0.010)
    assert tr["batches"] == 3 and tr["largest_batch"] == 2
    assert abs(tr["mean_batch"] - 4 / 3) < 1e-12
    assert abs(tr["first_launch_ms"] - 2.0) < 1e-9
    assert abs(tr["admission_span_ms"] - 3.0) < 1e-9
    assert abs(tr["admit_us_per_request"] - 1000.0) < 1e-6  # median of 0.5, 1.5, 1 ms gaps
    # in flight: [2, 8] ms and [9, 10] ms -> 7 ms of the 10 ms span
    assert abs(tr["batch_in_flight_frac"] - 0.7) < 1e-12
    # per batch, launch to last completion: 4, 4 and 1 ms
    assert abs(tr["mean_batch_ms"] - 3.0) < 1e-9
    assert bench.serve_trace(t[:0], 0.0) is None


def test_roofline_records_follow_the_scope_counts(monkeypatch):
    """Sweep: half-shell stencil candidates x 8 + pair-images x 26 FLOP per
    launch over the CUDA-event time, against 152 SMs x 128 lanes x 2 x 2.07
    GHz; binning: 44 B per particle + 8 B per cell over the measured copy
    bandwidth. Figures of the 1M lattice step."""
    sys.path.insert(0, ROOT)
    import bench
    peak = 152 * 128 * 2 * 2070e6 / 1e12
    monkeypatch.setattr(bench, "fp32_peak", lambda dev, clocks: (peak, "test"))
    cand, pairs, kms = 1_457_508_307, 361_637_312, 1.2142307305335998
    r = bench.sweep_roofline(None, None, cand, pairs, kms, 911_427_599, "k", True)
    flop = cand * 8 + pairs * 26
    assert r["flop_per_launch"] == flop == 21_062_636_568
    assert abs(r["achieved"] - flop / (kms * 1e-3) / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / 80.54784) < 1e-12 and 0.21 < r["frac"] < 0.22
    assert r["evaluated"]["flop"] == 911_427_599 * 8 + pairs * 22
    b = bench.binning_record(1_000_000, 42_875, 0.05, {"hbm_gbs": 6782.8}, "test")
    assert b["bytes"] == 44 * 1_000_000 + 8 * 42_875
    assert abs(b["achieved"] - b["bytes"] / 0.05e-3 / 1e9) < 1e-9
    assert abs(b["frac"] - b["achieved"] / 6782.8) < 1e-12
