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
# FP32 arithmetic per candidate pair and per ordered pair-image within the cutoff
# (FMA = 2 FLOP, 1/r = 1) of the fused energy-and-gradient sweep:
FLOP_PER_CANDIDATE = 8      # 3 sub + 1 mul + 2 fma for |x_j' - x_i|^2
FLOP_PER_HIT_FUSED = 16     # 1/r (1); fsn = y (y^2 - 1/rc^2) (3); force 3 fma (6); r = d2 y (1),
                            # t = 1 - r/rc (2), t^2 (1), e += t^2 y (2)
# DRAM bytes per launch of the fused sweep (k_hood<3>, 1M lattice, lcell 2), from
# ncu --set full: dram__bytes_read.sum + dram__bytes_write.sum = 40.71 MB + 1.21 MB.
SWEEP_DRAM_BYTES = 41.93e6
SM_COUNT_GB300 = 152
FP32_LANES_PER_SM = 128


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-serve", action="store_true")
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
    if name == "w2_triclinic_1m":
        return synth.w2_triclinic()
    return synth.w1_lattice() if name == "w1_lattice_1m" else synth.w4_clustered()


def cpu_baseline(w, budget_s=15.0):
    """The FP64 oracle as it stands, single-threaded on the host, on a bounded
    sample: pairs whose smaller index is below k (energy, forces, virial)."""
    import oracle
    x, h, rc = w["x"], w["h"], w["rc"]
    k = 20_000
    t0 = time.perf_counter()
    r = oracle.pair_map(x, h, rc, forces=True, i_range=(0, k))
    dt = time.perf_counter() - t0
    if dt < budget_s / 4:
        k = min(x.shape[0], int(k * budget_s / max(dt, 1e-3) * 0.8))
        t0 = time.perf_counter()
        r = oracle.pair_map(x, h, rc, forces=True, i_range=(0, k))
        dt = time.perf_counter() - t0
    return {"value": r["count"] / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "pairs (i<j) with i < %d of the %d-particle workload: energy, forces, virial in FP64; "
                      "%.1f s, %d pairs" % (k, x.shape[0], dt, r["count"]), "seconds": dt, "pairs": r["count"]}


def run_reference(args, rank, world):
    """Reference arm: the FP64 oracle on the host cores, same metric and workload."""
    if rank != 0:
        return None
    import synth
    w = load_workload(getattr(args, "workload", WORKLOAD))
    import oracle
    x, h, rc = w["x"], w["h"], w["rc"]
    k = 2000
    for _ in range(min(args.warmup, 2)):
        oracle.pair_map(x, h, rc, forces=True, i_range=(0, k))
    times, pairs = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.pair_map(x, h, rc, forces=True, i_range=(0, k))
        times.append(time.perf_counter() - t0)
        pairs = r["count"]
    ms = 1e3 * sum(times) / len(times)
    value = pairs / (ms / 1e3)
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": getattr(args, "workload", WORKLOAD), "n": x.shape[0], "cutoff": rc,
                       "sample": "each step: pairs (i<j) with i < %d" % k},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "pairs (i<j) with i < %d of the 1M lattice per step, FP64 energy, "
                                       "forces, virial, single thread" % k},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_pairlist(args, rank, world, local):
    """w2_triclinic_1m: binning, the sorted i<j pair list (count pass, one
    synchronisation for the total, fill pass) and the 200-bin histogram."""
    import torch
    import paper_2202_06427_gb300 as P

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
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

    def step(ev=None):
        P.cl_update(cl, x)
        if ev is not None:
            ev[0].record(stream)
        got = P.cl_map(cl, "pairlist", out=bufs)["npairs"]
        if ev is not None:
            ev[1].record(stream)
        P.cl_map(cl, "hist", nbins=nbins)
        return got

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(gpu_id(dev))
    sampler.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world, dev)
    torch.cuda.synchronize(dev)
    for k in range(args.steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        assert step(kev[k]) == pairs
        ends[k].record(stream)
    torch.cuda.synchronize(dev)
    barrier(world, dev)
    sampler.stop()
    ms = reduce_max(sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / args.steps, world, dev)
    kms = sum(a.elapsed_time(b) for a, b in kev) / args.steps
    peaks, basis = {"hbm_gbs": 6800.0}, "fallback copy bandwidth (6.8 TB/s, no measured peaks on this machine)"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks, basis = json.load(f), "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError):
        pass
    # algorithmic bytes of the list passes: 12 B written per pair, the sorted float4
    # particles and cell offsets read once per pass
    nbytes = 12 * pairs + 2 * 16 * n
    achieved = nbytes / (kms / 1e3) / 1e9
    return {"metric": METRIC, "value": pairs * world / (ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "w2_triclinic_1m", "n": n, "cutoff": rc, "lcell": LCELL, "pairs_per_step": pairs,
                       "step": "binning + sorted i<j pair list (count, scan, fill) + 200-bin histogram",
                       "l2": "flushed between steps by a 256 MB write outside the timed events",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            # bin, 3 scan, scatter, pair pack; cell count, listed-cell count, 3 scan, cell fill,
            # listed-cell fill, long-segment sort; histogram sweep
            "gpu_launches": 15 * args.steps,
            "clocks": sampler.summary(),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                         "kernel": "pair-list passes (k_pairs_cell count and fill, scan, per-particle paths)",
                         "kernel_ms": kms, "bytes_per_launch": nbytes,
                         "peak_basis": basis}}


def run_ours(args, rank, world, local):
    if getattr(args, "workload", WORKLOAD) == "w2_triclinic_1m":
        return run_pairlist(args, rank, world, local)
    import torch
    import paper_2202_06427_gb300 as P
    import synth

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w = load_workload(getattr(args, "workload", WORKLOAD))
    x = torch.from_numpy(w["x"]).to(dev)
    h, rc = w["h"], w["rc"]
    n = x.shape[0]
    stream = torch.cuda.current_stream(dev)
    lcell = LCELL_BY_WORKLOAD.get(getattr(args, "workload", WORKLOAD), LCELL)
    cl = P.cl_build(x, h, rc, lcell)
    pairs = int(P.cl_map(cl, "count")["count"].item())
    cand_half = P.cl_query(cl, "candidates")
    g = torch.ones(1, dtype=torch.float64, device=dev)
    out = (torch.empty(1, dtype=torch.float64, device=dev), torch.empty((n, 3), dtype=torch.float64, device=dev),
           torch.empty((3, 3), dtype=torch.float64, device=dev), None)
    grad_x = torch.empty((n, 3), dtype=torch.float64, device=dev)
    grad_h = torch.empty((3, 3), dtype=torch.float64, device=dev)
    P.cl_energy_grad(cl, out=out)
    cand = P.cl_query(cl, "sweep_candidates")  # candidate pairs the fused sweep evaluates
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2

    def step(ev=None):
        P.cl_update(cl, x)
        if ev is not None:
            ev[0].record(stream)
        P.cl_energy_grad(cl, out=out)  # forward: energy, dE/dx, dE/dH in one sweep
        if ev is not None:
            ev[1].record(stream)
        P.cl_scale(g, out[1], grad_x)  # backward: dL/dx = dL/dE dE/dx
        P.cl_scale(g, out[2], grad_h)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(gpu_id(dev))
    sampler.start()
    time.sleep(0.3)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world, dev)
    torch.cuda.synchronize(dev)
    for k in range(args.steps):
        flush.fill_(float(k))  # evict the inputs from L2 between steps (outside the timed events)
        starts[k].record(stream)
        step(kev[k])
        ends[k].record(stream)
    torch.cuda.synchronize(dev)
    barrier(world, dev)
    sampler.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    kern_ms = [a.elapsed_time(b) for a, b in kev]
    ms = reduce_max(sum(step_ms) / len(step_ms), world, dev)
    kms = sum(kern_ms) / len(kern_ms)
    value = pairs * world / (ms / 1e3)

    # roofline of the dominant kernel (the fused energy-and-gradient sweep)
    clocks = sampler.summary()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    max_mhz = clocks["sm_max_mhz"] or 2070.0
    peak_tflops = sms * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12
    flop = cand * FLOP_PER_CANDIDATE + 2 * pairs * FLOP_PER_HIT_FUSED
    achieved = flop / (kms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops,
                "traffic": SWEEP_DRAM_BYTES if getattr(args, "workload", WORKLOAD) == WORKLOAD else None,
                "kernel": "k_hood<3> (cl_energy_grad: neighbourhood sweep, energy + forces + box gradient)",
                "kernel_ms": kms, "flop_per_launch": flop, "candidates_per_launch": cand,
                "peak_basis": "%d SMs x 128 FP32 lanes x 2 x %.0f MHz (of max clock, not measured)" % (sms, max_mhz)}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": getattr(args, "workload", WORKLOAD), "n": n, "box": float(h[0][0]), "cutoff": rc, "lcell": lcell,
                       "pairs_per_step": pairs, "candidates_sweep": cand, "candidates_half_shell_stencil": cand_half,
                       "step": "binning + fused energy/forces/box-gradient sweep (forward) + chain rule (backward)",
                       "l2": "flushed between steps by a 256 MB write outside the timed events",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            # bin, 3 scan, scatter, pair pack; cell list, sweep, per-particle companion, dense-cell sweep,
            # 2 reduce; 2 scale
            "gpu_launches": 14 * args.steps,
            "clocks": clocks, "roofline": roofline}

    if not args.no_e2e:
        line["e2e"] = e2e(P, cl, w, dev, stream, pairs, args, world)
    if not args.no_serve:
        line["serve"] = serve_leg(dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w)
    return line


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
                "largest_batch": st["largest_batch"], "failed": int(sum(1 for x in status if x != 0))}

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
