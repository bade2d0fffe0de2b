"""Benchmark of the cell-list pair map on GB300: in-cutoff pairs per second at
1M particles.

One step is one pass of the whole hot path over the 1M jittered-lattice
workload (3D, 100^3 sites at density 0.1, box 215.44, rc 12), the forward
and backward of a differentiable energy:
  cell binning (FP64 wrap, fractional cell, counting sort, prefix sum, scatter)
  -> neighbourhood sweep: shifted-force energy, dE/dx (forces) and dE/dH
     (virial) fused in one pass (cl_energy_grad)
  -> fixed-order FP64 reduction of the per-CTA partials
  -> chain rule by the upstream gradient (cl_scale) for positions and box.
value = pairs within the cutoff per step * ranks / time per step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload w1_lattice_1m|w4_clustered_16m|w2_triclinic_1m]
The default workload is the 1M lattice the metric is quoted on; the 16M
clustered set (box 600, rc 8, 2,000 Gaussian clusters + 20 % background) runs
the same step for the strongly inhomogeneous case. w2_triclinic_1m (rows
(220,0,0), (30,215,0), (20,25,210), rc 10) runs binning + the sorted i<j pair
list + a 200-bin histogram per step instead (GPU arm only, no e2e or serving
legs).
N > 1 runs under torchrun, one rank per GPU; each rank runs its own replica
of the workload (the path has no exchange step: replicas only), and the step
time is the maximum over ranks.
"""
import argparse
import json
import numpy as np
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pairs-within-cutoff/sec at 1M particles"
UNIT = "pairs/s"
WORKLOAD = "w1_lattice_1m"
LCELL = 2
# cells per cutoff length by workload: two on the homogeneous sets; one on the
# clustered set, where larger cells keep fewer particles in sparse cells and
# fewer cells over the staging limits (measured: fused sweep 37 ms at 1, 57 ms at 2)
LCELL_BY_WORKLOAD = {"w1_lattice_1m": 2, "w2_triclinic_1m": 2, "w4_clustered_16m": 1}
# Algorithmic FP32 work of the sweep (FMA = 2 FLOP, 1/r = 1), counted on the
# method's own work, not on what a kernel happens to evaluate:
#   per candidate pair of the half-shell cell stencil (each unordered pair-image
#   tested once): 3 sub + 1 mul + 2 fma for |x_j + S_o - x_i|^2 = 8 FLOP;
#   per pair-image within the cutoff, shifted-force energy + forces + virial:
#   1/r, u, u'/r, 3 force FMAs for i and 3 for j, 6 virial FMAs = 26 FLOP.
FLOP_PER_CANDIDATE = 8
FLOP_PER_PAIR = 26
# What the sweep itself evaluates, reported beside the algorithmic figure: 8 FLOP
# per staged candidate, and per pair-image within the cutoff either 16 FLOP from
# each end (full-shell kernels: 1/r, fsn, 3 force FMAs, energy term) or, on the
# half-shell path (each pair-image once), the force on both particles as well
# (1/r, fsn, 6 force FMAs, energy term: 22 FLOP).
FLOP_PER_HIT_FUSED = 16
FLOP_PER_HIT_HALF = 22
# Algorithmic bytes of binning per particle: FP64 position read (24 B), FP32
# cell-centred coordinate + index written (16 B), cell-sorted position of the
# original index (4 B); the per-cell counts and offsets add 8 B per cell.
BIN_BYTES_PER_PARTICLE = 44
BIN_BYTES_PER_CELL = 8
# DRAM bytes per launch of the dominant kernel (k_hood_half<3, 0> on the 1M
# lattice) from one ncu capture of its current version (dram__bytes_read.sum +
# dram__bytes_write.sum = 36.40 + 0.00 MB), or None when the kernel has changed
# since the counters were taken.
SWEEP_DRAM_BYTES = 36_400_384
FP32_LANES_PER_SM = 128
# kernels of one headline step: bin, 2 scan, scatter, packed cells (binning);
# cell list, octant order of the windowed cells, half-shell sweep of the
# fast-path cells, of the windowed cells (both exit at once when there are
# none), per-particle finish, final reduction (cl_energy_grad); 2 scale
# (chain rule for positions and box)
STEP_LAUNCHES = 13


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-extra", action="store_true", help="skip the CPU baseline, precision and other workloads")
    p.add_argument("--workload", choices=["w1_lattice_1m", "w4_clustered_16m", "w2_triclinic_1m"],
                   default=WORKLOAD)
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(value, world, device=None):
    """Maximum of a float over the ranks (identity when world == 1)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world, device=None):
    if world <= 1:
        return
    import torch.distributed as dist
    if device is not None and device.type == "cuda":
        dist.barrier(device_ids=[device.index])
    else:
        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def gpu_id(dev):
    """nvidia-smi -i accepts the UUID, which survives CUDA_VISIBLE_DEVICES renumbering."""
    import torch
    uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    if uuid is None:
        return str(dev.index)
    s = str(uuid)
    return s if s.startswith("GPU-") else "GPU-" + s


def load_workload(name):
    import synth
    make = {"w0_small_10k": synth.w0_small, "w1_lattice_1m": synth.w1_lattice,
            "w2_triclinic_1m": synth.w2_triclinic, "w4_clustered_16m": synth.w4_clustered}
    return make[name]()


def _oracle_part(job):
    """One worker of the host-core pool: the oracle, as it stands, on the pairs
    whose smaller index lies in [lo, hi) (positions from a memory-mapped file)."""
    import oracle
    if job is None:  # warm-up: the import alone
        return None
    path, h, rc, nbins, forces, lo, hi = job
    x = np.load(path, mmap_mode="r")
    t0 = time.perf_counter()
    r = oracle.pair_map(x, h, rc, nbins=nbins, forces=forces, i_range=(lo, hi))
    r["seconds"] = time.perf_counter() - t0
    return r


class OraclePool:
    """The single-threaded FP64 oracle run on all host cores: one spawned
    process per core, each on a range of the smaller pair index; partial sums
    are added in a fixed order. Started with spawn, so that it is safe after
    the first CUDA call."""

    def __init__(self, x, nproc=None):
        import multiprocessing as mp
        import tempfile
        self.nproc = nproc or os.cpu_count() or 1
        self.tmp = tempfile.TemporaryDirectory()
        self.path = os.path.join(self.tmp.name, "x.npy")
        np.save(self.path, np.ascontiguousarray(x, dtype=np.float64))
        self.n = x.shape[0]
        self.pool = mp.get_context("spawn").Pool(self.nproc)
        self.pool.map(_oracle_part, [None] * self.nproc)  # workers import the oracle once

    def load(self, x):
        """Positions for the following runs (a new memory-mapped file)."""
        self.path = os.path.join(self.tmp.name, "x%d.npy" % id(x))
        np.save(self.path, np.ascontiguousarray(x, dtype=np.float64))
        self.n = x.shape[0]

    def run(self, h, rc, lo=0, hi=None, nbins=0, forces=True):
        hi = self.n if hi is None else hi
        cuts = np.unique(np.linspace(lo, hi, 4 * self.nproc + 1).astype(np.int64))
        jobs = [(self.path, h, rc, nbins, forces, int(a), int(b)) for a, b in zip(cuts[:-1], cuts[1:])]
        t0 = time.perf_counter()
        parts = self.pool.map(_oracle_part, jobs, chunksize=1)
        wall = time.perf_counter() - t0
        out = {k: sum(p[k] for p in parts) for k in ("count", "band_in", "band_out", "suminvr", "energy")}
        out["virial"] = sum(p["virial"] for p in parts)
        out["dedh"] = sum(p["dedh"] for p in parts)
        if forces:
            out["forces"] = sum(p["forces"] for p in parts)
        if nbins:
            out["hist_core"] = sum(p["hist_core"] for p in parts)
            out["hist_maybe"] = sum(p["hist_maybe"] for p in parts)
        out["wall_s"] = wall
        return out

    def close(self):
        self.pool.close()
        self.pool.join()
        self.tmp.cleanup()


def cpu_baseline(w, pool, budget_s=15.0):
    """The FP64 oracle as it stands on the host: all cores on the whole
    workload (energy, forces, virial), and one core on a bounded sample (pairs
    whose smaller index is below k). Returns the record and the all-core result,
    which the precision record compares the GPU against."""
    import oracle
    x, h, rc = w["x"], w["h"], w["rc"]
    full = pool.run(h, rc, forces=True)
    k = 20_000
    t0 = time.perf_counter()
    r = oracle.pair_map(x, h, rc, forces=True, i_range=(0, k))
    dt = time.perf_counter() - t0
    if dt < budget_s / 4:
        k = min(x.shape[0], int(k * budget_s / max(dt, 1e-3) * 0.8))
        t0 = time.perf_counter()
        r = oracle.pair_map(x, h, rc, forces=True, i_range=(0, k))
        dt = time.perf_counter() - t0
    rec = {"value": full["count"] / full["wall_s"], "unit": UNIT, "cores": pool.nproc, "kind": "oracle",
           "sample": "whole workload (%d particles, %d pairs): FP64 energy, forces, virial, box gradient; "
                     "one process per core over ranges of the smaller index; %.2f s wall"
                     % (x.shape[0], full["count"], full["wall_s"]),
           "single_core": {"value": r["count"] / dt, "unit": UNIT, "cores": 1,
                           "sample": "pairs (i<j) with i < %d: %.1f s, %d pairs" % (k, dt, r["count"])}}
    return rec, full


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle, as it stands, on all host cores (one
    process per core over ranges of the smaller pair index), same metric and
    workload. Each step maps the pairs whose smaller index is below k, with k
    chosen so that the whole run stays within about two minutes."""
    if rank != 0:
        return None
    w = load_workload(getattr(args, "workload", WORKLOAD))
    x, h, rc = w["x"], w["h"], w["rc"]
    n = x.shape[0]
    pool = OraclePool(x)
    try:
        probe = pool.run(h, rc, 0, min(n, 64 * pool.nproc), forces=True)
        per_row = probe["wall_s"] / min(n, 64 * pool.nproc)
        budget = 120.0 / max(1, args.steps + min(args.warmup, 3))
        k = int(min(n, max(pool.nproc * 16, budget / max(per_row, 1e-9))))
        for _ in range(min(args.warmup, 3)):
            pool.run(h, rc, 0, k, forces=True)
        times, pairs = [], 0
        for _ in range(args.steps):
            r = pool.run(h, rc, 0, k, forces=True)
            times.append(r["wall_s"])
            pairs = r["count"]
    finally:
        pool.close()
    ms = 1e3 * sum(times) / len(times)
    value = pairs / (ms / 1e3)
    sample = ("each step: pairs (i<j) with i < %d of the %d-particle workload (%d pairs), FP64 energy, forces, "
              "virial, box gradient; %d processes" % (k, n, pairs, pool.nproc))
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": getattr(args, "workload", WORKLOAD), "n": n, "cutoff": rc, "sample": sample,
                       "same_config": k == n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.nproc, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured (MEASURED_PEAKS.json)"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0}, "fallback (6.8 TB/s copy bandwidth; no MEASURED_PEAKS.json on this machine)"


def fp32_peak(dev, clocks):
    """FP32 peak of the ALUs: SMs x 128 lanes x 2 FLOP (FMA) x SM clock. The
    clock is the highest sampled during the timed region (the sweep runs at the
    maximum clock), else the 2,070 MHz maximum of the part."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, \
        "%d SMs x 128 FP32 lanes x 2 FLOP x %.0f MHz (derived from unit counts and the maximum clock)" % (sms, mhz)


def sweep_roofline(dev, clocks, cand_half, pairs, kms, cand_eval, kernel, half_path):
    """Roofline record of the sweep: algorithmic FP32 work (half-shell stencil
    candidates x 8 + pair-images x 26) / the sweep's CUDA-event time, against
    the FP32 peak. The work the kernels themselves evaluated is reported beside
    it (half_path: each pair-image once)."""
    peak, basis = fp32_peak(dev, clocks)
    flop = cand_half * FLOP_PER_CANDIDATE + pairs * FLOP_PER_PAIR
    achieved = flop / (kms / 1e3) / 1e12
    if half_path:
        flop_eval = cand_eval * FLOP_PER_CANDIDATE + pairs * FLOP_PER_HIT_HALF
        ebasis = "staged half-shell candidates x 8 + pair-images x 22 (each once, forces on both particles)"
    else:
        flop_eval = cand_eval * FLOP_PER_CANDIDATE + 2 * pairs * FLOP_PER_HIT_FUSED
        ebasis = "staged full-shell candidates x 8 + ordered pair-images x 16"
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": kernel, "kernel_ms": kms, "flop_per_launch": flop,
            "flop_basis": "half-shell stencil candidates x %d + pair-images x %d (energy, forces, virial)"
                          % (FLOP_PER_CANDIDATE, FLOP_PER_PAIR),
            "candidates_half_shell_stencil": cand_half,
            "evaluated": {"candidates": cand_eval, "flop": flop_eval, "tflops": flop_eval / (kms / 1e3) / 1e12,
                          "frac": flop_eval / (kms / 1e3) / 1e12 / peak, "half_shell": bool(half_path),
                          "basis": ebasis},
            "peak_basis": basis}


def binning_record(n, ncells, ms, peaks, basis):
    nbytes = BIN_BYTES_PER_PARTICLE * n + BIN_BYTES_PER_CELL * ncells
    gbs = nbytes / (ms / 1e3) / 1e9
    return {"bound": "hbm", "ms": ms, "bytes": nbytes, "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": gbs / peaks["hbm_gbs"], "peak_basis": basis,
            "bytes_basis": "%d B per particle + %d B per cell (algorithmic)" % (BIN_BYTES_PER_PARTICLE,
                                                                                 BIN_BYTES_PER_CELL)}


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = float(np.abs(b).max()) if b.size else 0.0
    return float(np.abs(a - b).max() / scale) if scale > 0 else float(np.abs(a - b).max())


def count_record(gpu, ref):
    return {"gpu": int(gpu), "oracle": int(ref["count"]), "diff": int(gpu) - int(ref["count"]),
            "band_in": int(ref["band_in"]), "band_out": int(ref["band_out"]),
            "within_band": bool(ref["count"] - ref["band_in"] <= gpu <= ref["count"] + ref["band_out"])}


def hist_record(gpu, ref):
    gpu = np.asarray(gpu, dtype=np.int64)
    core, maybe = ref["hist_core"], ref["hist_maybe"]
    outside = int(np.sum((gpu < core) | (gpu > core + maybe)))
    return {"bins": int(gpu.size), "bins_outside_band": outside, "band_pairs": int(maybe.sum()),
            "off_core": int(np.sum(gpu - core))}


def pairlist_leg(dev, steps, warmup, pool=None):
    """The triclinic 1M workload (rows (220,0,0), (30,215,0), (20,25,210), rc 10):
    binning, the sorted i<j pair list (count pass, 64-bit scan, one
    synchronisation for the total, fill pass) and the 200-bin histogram. With a
    pool, the histogram and the pair count are checked against the oracle."""
    import torch
    import paper_2202_06427_gb300 as P
    w = load_workload("w2_triclinic_1m")
    x = torch.from_numpy(w["x"]).to(dev)
    h, rc, nbins = w["h"], w["rc"], w["nbins"]
    n = x.shape[0]
    stream = torch.cuda.current_stream(dev)
    cl = P.cl_build(x, h, rc, LCELL)
    pairs = P.cl_map(cl, "pairlist")["npairs"]
    bufs = (torch.empty(pairs, dtype=torch.int32, device=dev), torch.empty(pairs, dtype=torch.int32, device=dev),
            torch.empty(pairs, dtype=torch.float32, device=dev))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]

    def step(e=None):
        if e is not None:
            e[0].record(stream)
        P.cl_update(cl, x)
        if e is not None:
            e[1].record(stream)
        got = P.cl_map(cl, "pairlist", out=bufs)["npairs"]
        if e is not None:
            e[2].record(stream)
        hist = P.cl_map(cl, "hist", nbins=nbins)["hist"]
        if e is not None:
            e[3].record(stream)
        return got, hist

    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    for k in range(steps):
        flush.fill_(float(k))
        got, hist = step(ev[k])
        assert got == pairs
    torch.cuda.synchronize(dev)
    avg = lambda a, b: sum(e[a].elapsed_time(e[b]) for e in ev) / steps
    ms, bms, lms, hms = avg(0, 3), avg(0, 1), avg(1, 2), avg(2, 3)
    peaks, basis = load_peaks()
    # algorithmic bytes of the list passes: 12 B written per pair, the sorted
    # float4 particles read once per pass
    nbytes = 12 * pairs + 2 * 16 * n
    gbs = nbytes / (lms / 1e3) / 1e9
    out = {"workload": "w2_triclinic_1m", "n": n, "cutoff": rc, "lcell": LCELL, "pairs_per_step": pairs,
           "steps": steps, "ms_per_step": ms, "pairs_per_s": pairs / (ms / 1e3),
           "step": "binning + sorted i<j pair list (count, 64-bit scan, fill) + 200-bin histogram",
           "binning_ms": bms, "pairlist_ms": lms, "hist_ms": hms,
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": gbs / peaks["hbm_gbs"], "traffic": None, "kernel": "pair-list passes",
                        "kernel_ms": lms, "bytes_per_launch": nbytes,
                        "bytes_basis": "12 B per pair written + 16 B per particle read per pass", "peak_basis": basis},
           "binning": binning_record(n, P.cl_query(cl, "ncells"), bms, peaks, basis),
           "gpu_launches_per_step": 15}
    if pool is not None:
        pool.load(w["x"])
        ref = pool.run(h, rc, nbins=nbins, forces=False)
        out["precision"] = {"pairs": count_record(pairs, ref), "histogram": hist_record(hist.cpu().numpy(), ref),
                            "oracle_wall_s": ref["wall_s"]}
    return out


def run_pairlist(args, rank, world, local):
    """--workload w2_triclinic_1m: the pair-list step as the bench line."""
    import torch
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    sampler = ClockSampler(gpu_id(dev))
    sampler.start()
    barrier(world, dev)
    leg = pairlist_leg(dev, args.steps, args.warmup)
    barrier(world, dev)
    sampler.stop()
    ms = reduce_max(leg["ms_per_step"], world, dev)
    return {"metric": METRIC, "value": leg["pairs_per_step"] * world / (ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "w2_triclinic_1m", "n": leg["n"], "cutoff": leg["cutoff"], "lcell": LCELL,
                       "pairs_per_step": leg["pairs_per_step"], "step": leg["step"],
                       "l2": "flushed between steps by a 256 MB write outside the timed events",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "gpu_launches": leg["gpu_launches_per_step"] * args.steps, "clocks": sampler.summary(),
            "roofline": leg["roofline"], "binning": leg["binning"]}


def energy_grad_step(P, cl, out, g, grad_x, grad_h, stream, e=None):
    """One step of the hot path: binning, the fused energy/forces/box-gradient
    sweep, chain rule. e: four events (start, after binning, after sweep, end)."""
    if e is not None:
        e[0].record(stream)
    P.cl_update(cl, out[4])
    if e is not None:
        e[1].record(stream)
    P.cl_energy_grad(cl, out=out[:4])  # forward: energy, dE/dx, dE/dH in one sweep
    if e is not None:
        e[2].record(stream)
    P.cl_scale(g, out[1], grad_x)  # backward: dL/dx = dL/dE dE/dx
    P.cl_scale(g, out[2], grad_h)
    if e is not None:
        e[3].record(stream)


def clustered_leg(dev, steps, warmup):
    """The 16M clustered set (box 600, rc 8): the same step as the headline."""
    import torch
    import paper_2202_06427_gb300 as P
    w = load_workload("w4_clustered_16m")
    x = torch.from_numpy(w["x"]).to(dev)
    h, rc = w["h"], w["rc"]
    n = x.shape[0]
    lcell = LCELL_BY_WORKLOAD["w4_clustered_16m"]
    stream = torch.cuda.current_stream(dev)
    cl = P.cl_build(x, h, rc, lcell)
    pairs = int(P.cl_map(cl, "count")["count"].item())
    cand_half = P.cl_query(cl, "candidates")
    g = torch.ones(1, dtype=torch.float64, device=dev)
    out = (torch.empty(1, dtype=torch.float64, device=dev), torch.empty((n, 3), dtype=torch.float64, device=dev),
           torch.empty((3, 3), dtype=torch.float64, device=dev), None, x)
    grad_x = torch.empty((n, 3), dtype=torch.float64, device=dev)
    grad_h = torch.empty((3, 3), dtype=torch.float64, device=dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    for _ in range(warmup):
        energy_grad_step(P, cl, out, g, grad_x, grad_h, stream)
    cand = P.cl_query(cl, "sweep_candidates")
    half_path = P.cl_query(cl, "sweep_half")
    torch.cuda.synchronize(dev)
    for k in range(steps):
        energy_grad_step(P, cl, out, g, grad_x, grad_h, stream, ev[k])
    torch.cuda.synchronize(dev)
    avg = lambda a, b: sum(e[a].elapsed_time(e[b]) for e in ev) / steps
    ms, bms, kms = avg(0, 3), avg(0, 1), avg(1, 2)
    peaks, basis = load_peaks()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    red = reduction_times(P, cl, dev, flush, reps=5)
    del flush
    return {"workload": "w4_clustered_16m", "n": n, "cutoff": rc, "lcell": lcell, "pairs_per_step": pairs,
            "reductions": red,
            "steps": steps, "ms_per_step": ms, "pairs_per_s": pairs / (ms / 1e3),
            "step": "binning + fused energy/forces/box-gradient sweep + chain rule",
            "l2": "inputs (384 MB positions) larger than L2",
            "roofline": sweep_roofline(dev, None, cand_half, pairs, kms, cand, "cl_energy_grad sweep kernels",
                                       half_path),
            "binning": binning_record(n, P.cl_query(cl, "ncells"), bms, peaks, basis)}


def precision_small(P, dev, pool):
    """Every output of the library on the 10k workload (3D, box 46.416, rc 12)
    against the oracle: count (with the band), sum 1/r, energy, forces, virial,
    dE/dH, a 100-bin histogram."""
    import torch
    w = load_workload("w0_small_10k")
    x, h, rc = w["x"], w["h"], w["rc"]
    pool.load(x)
    ref = pool.run(h, rc, nbins=100, forces=True)
    pos = torch.from_numpy(x).to(dev)
    cl = P.cl_build(pos, h, rc, LCELL)
    cnt = int(P.cl_map(cl, "count")["count"].item())
    s1 = P.cl_map(cl, "sum_inv_r")["sum_inv_r"].item()
    hist = P.cl_map(cl, "hist", nbins=100)["hist"].cpu().numpy()
    e, dedx, dedh, vir = P.cl_energy_grad(cl, want_virial=True)
    return {"count": count_record(cnt, ref), "sum_inv_r_rel": abs(s1 - ref["suminvr"]) / abs(ref["suminvr"]),
            "energy_rel": abs(e.item() - ref["energy"]) / abs(ref["energy"]),
            "forces_maxnorm_rel": rel_err(-dedx.cpu().numpy(), ref["forces"]),
            "virial_rel": rel_err(vir.cpu().numpy(), ref["virial"]),
            "dedh_rel": rel_err(dedh.cpu().numpy(), ref["dedh"]),
            "histogram": hist_record(hist, ref)}


def run_ours(args, rank, world, local):
    if getattr(args, "workload", WORKLOAD) == "w2_triclinic_1m":
        return run_pairlist(args, rank, world, local)
    import torch
    import paper_2202_06427_gb300 as P

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    workload = getattr(args, "workload", WORKLOAD)
    w = load_workload(workload)
    x = torch.from_numpy(w["x"]).to(dev)
    h, rc = w["h"], w["rc"]
    n = x.shape[0]
    stream = torch.cuda.current_stream(dev)
    lcell = LCELL_BY_WORKLOAD.get(workload, LCELL)
    cl = P.cl_build(x, h, rc, lcell)
    pairs = int(P.cl_map(cl, "count")["count"].item())
    cand_half = P.cl_query(cl, "candidates")
    ncells = P.cl_query(cl, "ncells")
    g = torch.ones(1, dtype=torch.float64, device=dev)
    out = (torch.empty(1, dtype=torch.float64, device=dev), torch.empty((n, 3), dtype=torch.float64, device=dev),
           torch.empty((3, 3), dtype=torch.float64, device=dev), None, x)
    grad_x = torch.empty((n, 3), dtype=torch.float64, device=dev)
    grad_h = torch.empty((3, 3), dtype=torch.float64, device=dev)
    P.cl_energy_grad(cl, out=out[:4])
    cand = P.cl_query(cl, "sweep_candidates")  # candidate pairs the fused sweep evaluates
    half_path = P.cl_query(cl, "sweep_half")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2

    for _ in range(args.warmup):
        energy_grad_step(P, cl, out, g, grad_x, grad_h, stream)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(gpu_id(dev))
    sampler.start()
    time.sleep(0.3)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    barrier(world, dev)
    torch.cuda.synchronize(dev)
    for k in range(args.steps):
        flush.fill_(float(k))  # evict the inputs from L2 between steps (outside the timed events)
        energy_grad_step(P, cl, out, g, grad_x, grad_h, stream, ev[k])
    torch.cuda.synchronize(dev)
    barrier(world, dev)
    sampler.stop()
    avg = lambda a, b: sum(e[a].elapsed_time(e[b]) for e in ev) / args.steps
    ms = reduce_max(avg(0, 3), world, dev)
    bms, kms = avg(0, 1), avg(1, 2)
    value = pairs * world / (ms / 1e3)
    clocks = sampler.summary()
    peaks, basis = load_peaks()
    roofline = sweep_roofline(dev, clocks, cand_half, pairs, kms, cand,
                              "cl_energy_grad sweep kernels (neighbourhood sweep: energy + forces + box gradient)",
                              half_path)
    roofline["traffic"] = SWEEP_DRAM_BYTES if workload == WORKLOAD and half_path else None
    if roofline["traffic"] is not None:
        roofline["traffic_basis"] = "k_hood_half<3> (the dominant kernel of the sweep), one ncu capture"

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload, "n": n, "box": float(h[0][0]), "cutoff": rc, "lcell": lcell,
                       "pairs_per_step": pairs, "candidates_sweep": cand, "candidates_half_shell_stencil": cand_half,
                       "step": "binning + fused energy/forces/box-gradient sweep (forward) + chain rule (backward)",
                       "l2": "flushed between steps by a 256 MB write outside the timed events",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "gpu_launches": STEP_LAUNCHES * args.steps,
            "clocks": clocks, "roofline": roofline,
            "binning": binning_record(n, ncells, bms, peaks, basis),
            "sweep_pairs_per_s": pairs / (kms / 1e3)}
    if not args.no_extra:
        line["reductions"] = reduction_times(P, cl, dev, flush)

    if not args.no_e2e:
        line["e2e"] = e2e(P, cl, w, dev, stream, pairs, args, world)
    if not args.no_serve:
        line["serve"] = serve_leg(dev)
    if rank == 0 and world == 1 and not args.no_extra:
        line["workloads"] = {"w2_triclinic_1m": None, "w4_clustered_16m": None}
        pool = OraclePool(w["x"]) if not args.no_cpu_baseline else None
        try:
            if pool is not None:
                line["cpu_baseline"], full = cpu_baseline(w, pool)
                e, dedx, dedh, vir = P.cl_energy_grad(cl, want_virial=True)
                line["precision"] = {
                    workload: {"count": count_record(pairs, full),
                               "energy_rel": abs(e.item() - full["energy"]) / abs(full["energy"]),
                               "forces_maxnorm_rel": rel_err(-dedx.cpu().numpy(), full["forces"]),
                               "virial_rel": rel_err(vir.cpu().numpy(), full["virial"]),
                               "dedh_rel": rel_err(dedh.cpu().numpy(), full["dedh"])},
                    "w0_small_10k": precision_small(P, dev, pool)}
            line["workloads"]["w2_triclinic_1m"] = pairlist_leg(dev, 20, 3, pool)
            if pool is not None:
                line["precision"]["w2_triclinic_1m"] = line["workloads"]["w2_triclinic_1m"].pop("precision")
        finally:
            if pool is not None:
                pool.close()
        del out, grad_x, flush
        P.cl_free(cl)
        torch.cuda.empty_cache()
        line["workloads"]["w4_clustered_16m"] = clustered_leg(dev, 10, 3)
    return line


def reduction_times(P, cl, dev, flush, reps=20):
    """Device time of each built-in reduction on the built list (one cl_map
    call, output allocation included; L2 flushed before each call)."""
    import torch
    calls = {"count": lambda: P.cl_map(cl, "count"),
             "sum_inv_r": lambda: P.cl_map(cl, "sum_inv_r"),
             "energy": lambda: P.cl_map(cl, "energy"),
             "hist_100_bins": lambda: P.cl_map(cl, "hist", nbins=100),
             "energy_forces_virial": lambda: P.cl_map(cl, "energy_forces_virial")}
    out = {}
    for name, f in calls.items():
        for _ in range(2):
            f()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for k in range(reps):
            flush.fill_(float(k))
            ev[k][0].record()
            f()
            ev[k][1].record()
        torch.cuda.synchronize(dev)
        out[name + "_ms"] = sum(a.elapsed_time(b) for a, b in ev) / reps
    return out


def serve_trace(times, span):
    """Where a served stream's time goes, from the server's own host
    timestamps (submitted, admitted, batch launched, completed): the host
    time between consecutive admissions, the batches (grouped by launch time)
    and the part of the span with at least one batch in flight."""
    if len(times) == 0:
        return None
    t0 = times[:, 0].min()
    t1 = np.sort(times[:, 1])
    launch, inv = np.unique(times[:, 2], return_inverse=True)
    sizes = np.bincount(inv)
    end = np.array([times[inv == k, 3].max() for k in range(len(launch))])
    busy, cur0, cur1 = 0.0, None, None  # union of the batches' [launch, last completion] intervals
    for a, b in sorted(zip(launch, end)):
        if cur1 is None or a > cur1:
            if cur1 is not None:
                busy += cur1 - cur0
            cur0, cur1 = a, b
        else:
            cur1 = max(cur1, b)
    busy += cur1 - cur0
    gaps = np.diff(t1)
    return {"admit_us_per_request": float(np.median(gaps)) * 1e6 if len(gaps) else 0.0,
            "admission_span_ms": float(t1[-1] - t1[0]) * 1e3,
            "first_launch_ms": float(launch[0] - t0) * 1e3,
            "batches": int(len(sizes)), "mean_batch": float(sizes.mean()), "largest_batch": int(sizes.max()),
            "mean_batch_ms": float(np.mean(end - launch)) * 1e3,
            "batch_in_flight_frac": float(busy / span) if span > 0 else 0.0}


def serve_leg(dev):
    """Serving stream (512 seeded requests, Poisson arrivals with 2 ms mean
    gap, 2D/3D, 1e3..2e5 particles, ortho/triclinic, energy/forces/histogram)
    through the continuous-batching server, against one-request-at-a-time
    serving with the same kernels (a server admitting one request at a time)
    and against plain per-request launches through the public API."""
    import torch
    import paper_2202_06427_gb300 as P
    from paper_2202_06427_gb300 import serve as S
    import synth
    specs = synth.serve_stream()
    reqs = [S.Request(synth.request_positions(s), s["h"], s["rc"], s["task"], lcell=2, nbins=s["nbins"])
            for s in specs]
    warm = [S.Request(synth.request_positions(s), s["h"], s["rc"], s["task"], lcell=2, nbins=s["nbins"])
            for s in synth.serve_stream(n_requests=16, seed=7, n_max=20_000)]

    def run(max_inflight, realtime):
        srv = S.Server(arena_bytes=8 << 30, max_inflight=max_inflight, device=dev.index)
        try:
            for r in warm:
                srv.submit(r)
            for r in warm:
                srv.wait(r.ticket, 120.0)
            b0 = srv.stats()["batches"]
            wall0 = time.perf_counter()
            for spec, r in zip(specs, reqs):
                if realtime:
                    target = wall0 + spec["arrival_s"]
                    while True:
                        left = target - time.perf_counter()
                        if left <= 0:
                            break
                        time.sleep(left - 2e-4 if left > 5e-4 else 0)
                srv.submit(r)
            status = [srv.wait(r.ticket, 300.0) for r in reqs]
            times = np.array([srv.times(r.ticket) for r in reqs])
            st = srv.stats()
        finally:
            srv.close()
        lat = (times[:, 3] - times[:, 0]) * 1e3
        span = times[:, 3].max() - times[:, 0].min()
        return {"req_per_s": len(reqs) / span, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "batches": st["batches"] - b0,
                "largest_batch": st["largest_batch"], "failed": int(sum(1 for x in status if x != 0)),
                "trace": serve_trace(times[np.array(status) == 0], span)}

    def plain(k_max=None):
        """one request at a time through cl_build + cl_map, H2D and D2H included"""
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for spec, r in zip(specs, reqs):
            x = r.pos.to(dev, non_blocking=True)
            cl = P.cl_build(x, spec["h"], spec["rc"], 2)
            if spec["task"] == "energy":
                r.energy.copy_(P.cl_map(cl, "energy")["energy"], non_blocking=True)
            elif spec["task"] == "forces":
                o = P.cl_map(cl, "energy_forces_virial")
                r.energy.copy_(o["energy"], non_blocking=True)
                r.forces.copy_(o["forces"], non_blocking=True)
            else:
                r.hist.copy_(P.cl_map(cl, "hist", nbins=spec["nbins"])["hist"], non_blocking=True)
            torch.cuda.synchronize(dev)
            P.cl_free(cl)
        return {"req_per_s": len(reqs) / (time.perf_counter() - t0)}

    out = {"workload": "w3_serve_stream: 512 requests, Poisson arrivals (mean gap 2 ms), 2D rho 0.7 rc 2.5 / "
                       "3D rho 0.1 rc 12, N log-uniform 1e3..2e5, ortho/triclinic, energy/forces/100-bin hist",
           "offered_req_per_s": len(specs) / max(s["arrival_s"] for s in specs),
           "total_particles": int(sum(s["n"] for s in specs))}
    sat = run(256, False)
    poi = run(256, True)
    one_sat = run(1, False)
    one_poi = run(1, True)
    out.update({"req_per_s": sat["req_per_s"], "p50_ms": poi["p50_ms"], "p99_ms": poi["p99_ms"],
                "batched_saturation": sat, "batched_poisson": poi,
                "one_at_a_time": {"saturation": one_sat, "poisson": one_poi},
                "plain_api_one_at_a_time": plain()})
    return out


def e2e(P, cl, w, dev, stream, pairs, args, world):
    """Same step through the public API with host buffers: every step copies
    its positions in from pinned host memory and its energy and gradients out
    to pinned host memory. The copies run on a second stream with two device
    buffer sets, so step k+1's upload and step k's download overlap step k's
    and k+1's kernels (the pipelining a throughput deployment uses); the timed
    region ends when the last download has landed."""
    import torch
    host_x = torch.from_numpy(w["x"]).pin_memory()
    out_g = torch.empty(host_x.shape, dtype=torch.float64).pin_memory()
    out_e = torch.empty(1, dtype=torch.float64).pin_memory()
    out_b = torch.empty((3, 3), dtype=torch.float64).pin_memory()
    g = torch.ones(1, dtype=torch.float64, device=dev)
    steps = max(3, min(args.steps, 50))
    cs = torch.cuda.Stream(dev)
    f64 = dict(dtype=torch.float64, device=dev)
    xb = [torch.empty(host_x.shape, **f64) for _ in range(2)]
    outs = [(torch.empty(1, **f64), torch.empty(host_x.shape, **f64), torch.empty((3, 3), **f64), None)
            for _ in range(2)]
    gxb = [torch.empty(host_x.shape, **f64) for _ in range(2)]
    ghb = [torch.empty((3, 3), **f64) for _ in range(2)]
    up = [torch.cuda.Event() for _ in range(2)]      # inputs of buffer set b on the device
    comp = [torch.cuda.Event() for _ in range(2)]    # kernels of buffer set b done
    down = [torch.cuda.Event() for _ in range(2)]    # results of buffer set b copied out
    for b in range(2):
        comp[b].record(stream)
        down[b].record(cs)

    def upload(k):
        b = k % 2
        with torch.cuda.stream(cs):
            cs.wait_event(comp[b])        # step k - 2 no longer reads xb[b]
            xb[b].copy_(host_x, non_blocking=True)
            up[b].record(cs)

    def compute_and_download(k):
        b = k % 2
        stream.wait_event(up[b])
        stream.wait_event(down[b])        # step k - 2's results have left gxb[b]
        P.cl_update(cl, xb[b])
        P.cl_energy_grad(cl, out=outs[b])
        P.cl_scale(g, outs[b][1], gxb[b])
        P.cl_scale(g, outs[b][2], ghb[b])
        comp[b].record(stream)
        with torch.cuda.stream(cs):
            cs.wait_event(comp[b])
            out_e.copy_(outs[b][0], non_blocking=True)
            out_g.copy_(gxb[b], non_blocking=True)
            out_b.copy_(ghb[b], non_blocking=True)
            down[b].record(cs)

    def run(n):
        upload(0)
        for k in range(n):
            if k + 1 < n:
                upload(k + 1)
            compute_and_download(k)

    def serial():  # the same step with the copies in line on one stream
        xb[0].copy_(host_x, non_blocking=True)
        P.cl_update(cl, xb[0])
        P.cl_energy_grad(cl, out=outs[0])
        P.cl_scale(g, outs[0][1], gxb[0])
        P.cl_scale(g, outs[0][2], ghb[0])
        out_e.copy_(outs[0][0], non_blocking=True)
        out_g.copy_(gxb[0], non_blocking=True)
        out_b.copy_(ghb[0], non_blocking=True)

    run(3)
    torch.cuda.synchronize(dev)
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    cs.wait_event(a)
    run(steps)
    stream.wait_stream(cs)
    e.record(stream)
    torch.cuda.synchronize(dev)
    ms = reduce_max(a.elapsed_time(e) / steps, world, dev)
    for _ in range(3):
        serial()
    torch.cuda.synchronize(dev)
    a.record(stream)
    for _ in range(steps):
        serial()
    e.record(stream)
    torch.cuda.synchronize(dev)
    ms_serial = reduce_max(a.elapsed_time(e) / steps, world, dev)
    return {"value": pairs * world / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
            "h2d_bytes_per_step": host_x.numel() * 8,
            "d2h_bytes_per_step": out_g.numel() * 8 + 8 + 72,
            "pipelining": "copies on a second stream, two device buffer sets: uploads and downloads overlap "
                          "the neighbouring steps' kernels",
            "serial": {"value": pairs * world / (ms_serial / 1e3), "ms_per_step": ms_serial,
                       "note": "copies in line with the kernels on one stream"}}


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if args.impl == "ours":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        line = run_ours(args, rank, world, local)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
