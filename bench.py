"""Benchmark: long-range energy + potentials + forces, particles/s, on GB300.

Workload (the metric's configuration): N = 1e6 charges +-1 uniform in a
400 x 400 x 50 slab, alpha = 0.1, random batch P = 200 k-vectors per call
drawn on the device, M = 16 SOE terms (conditioned table), compensated FP32.
One step = one qslab_compute() call: input checks, z-sort, gather, k-sampler
and mode table, k-space chunk aggregates, carries, bidirectional recurrences
with the fused gather, the k = 0 term, the combine and the energy reduction.
The same step in FP64 is reported beside it, and so is the 512-replica
batched workload (one CUDA-graph-replayed batched call per step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica (the path is
not sharded across GPUs: replicas only); value = particles of all ranks / the
slowest rank's time. The reference arm (--impl reference) times the FP64 CPU
oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "long-range energy+force particles/s at N=1e6 on 1 GB300 (FP32 vs FP64); % roofline"
FP32_LANES_PER_SM = 128
L2_BYTES = 129 * 1024 * 1024


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


def algorithmic_instr(K, N, M):
    """FP32 arithmetic instructions the recurrences + gather must execute per
    call: per (k, beta, particle) a forward step, a backward step and the
    gather (~24), per (k, particle) the phase and the combination (~20)."""
    return float(K) * N * (24 * (M + 1) + 20)


def kernel_sources_sha256(names):
    """sha256 over the listed CUDA source files (in order): the traffic figure
    recorded in profiles/traffic.json holds only while they are unchanged."""
    import hashlib

    from paper_2403_01521_gb300 import build as _b
    if not names:
        return None
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(_b.CSRC, n), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        """Start polling every 50 ms and wait (up to 3 s) for the first
        sample, so that the samples cover the timed region that follows."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t0 = time.time()
        while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
            time.sleep(0.01)
        self.first = len(self.lines)   # samples before the timed region are not counted

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        during = self.lines[getattr(self, "first", 0):] or self.lines[-1:]
        for ln in during:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_max(x, device=None):
    """Maximum of x over all ranks (x itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, ms_slowest):
    """Whole-job rate: the units every rank processed over the slowest rank's time."""
    return world * units_per_rank / (ms_slowest * 1e-3)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _omp_threads():
    """OpenMP threads the oracle's k-space loop runs on (its default is every
    core this process may use)."""
    env = os.environ.get("OMP_NUM_THREADS")
    if env and env.strip().isdigit():
        return int(env)
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_oracle_call(sl, soe, P, seed, modes=None):
    """Time the FP64 oracle on one random-batch call of the workload: the
    k-space recursion over `modes` of the P sampled modes (all of them by
    default; OpenMP over the modes), then the whole k = 0 term (serial).
    Returns (seconds per full call, description, threads), where a partial
    mode sample is scaled to the P modes and says so."""
    from oracle import lattice, soe_ewald2d
    Lx, Ly, _ = sl.box
    mx, my = lattice.sample_modes(P, seed, 0, sl.alpha, Lx, Ly)
    H = lattice.H_direct(sl.alpha, Lx, Ly)
    gam = soe_ewald2d.rbe_prefactor(sl.alpha, Lx, Ly, mx, my, H, P)
    soe_ewald2d._load()
    m = P if modes is None else min(int(modes), P)
    t0 = time.perf_counter()
    soe_ewald2d.kspace_pairs(sl.pos, sl.q, sl.box, sl.alpha, *soe, mx[:m], my[:m], gam[:m])
    t1 = time.perf_counter()
    soe_ewald2d.kzero_pairs(sl.pos, sl.q, sl.box, sl.alpha, *soe)
    t2 = time.perf_counter()
    threads = min(_omp_threads(), m)
    if m == P:
        desc = (f"oracle (C FP64 recursion) on one full call: N={sl.N}, all {P} sampled k "
                f"(OpenMP over the modes, {threads} threads) and the k=0 term (serial); "
                f"k-space {t1 - t0:.2f} s, k=0 {t2 - t1:.2f} s")
        return (t2 - t0), desc, threads
    desc = (f"oracle (C FP64 recursion) on N={sl.N} with {m} of the {P} sampled k "
            f"({threads} threads) and the whole k=0 term (serial); the k-space time "
            f"({t1 - t0:.2f} s) scaled by {P}/{m}, k=0 {t2 - t1:.2f} s")
    return (t1 - t0) * P / m + (t2 - t1), desc, threads


def cpu_oracle_single_core(P, seed, modes=16):
    """The same oracle call on one core (OMP_NUM_THREADS=1, in a child
    process so that the OpenMP runtime starts with one thread), on a stated
    sample: `modes` of the P sampled k, scaled to P, plus the whole k = 0
    term. Returns (seconds per full call, description), or (None, reason)."""
    code = ("import sys, json; sys.path.insert(0, %r); import bench, workloads;"
            "from paper_2403_01521_gb300.soe import load_soe;"
            "t, d, n = bench.cpu_oracle_call(workloads.rbe_large(), load_soe(16), %d, %d, %d);"
            "print(json.dumps([t, d]))") % (ROOT, P, seed, modes)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True,
                           env=env, timeout=600)
        t, d = json.loads(r.stdout.strip().splitlines()[-1])
        return float(t), "single core: " + d
    except Exception as exc:  # noqa: BLE001 - reported, not fatal
        return None, f"single-core run failed: {exc}"


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, timed on the
    headline workload. Each step is one full random-batch call (all 200
    sampled modes) when the run has at most 20 steps, else a stated sample
    of 200 * 20 / steps modes (at least 16) scaled to 200, so that the whole
    run stays within a few minutes."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import workloads
    from paper_2403_01521_gb300.soe import load_soe
    sl = workloads.rbe_large()
    soe = load_soe(16)
    P = 200
    modes = P if args.steps <= 20 else max(16, (P * 20) // max(args.steps, 1))
    for _ in range(min(args.warmup, 1)):
        cpu_oracle_call(sl, soe, P, 11, modes=16)
    times = []
    desc = cores = None
    for _ in range(args.steps):
        t, desc, cores = cpu_oracle_call(sl, soe, P, 11, modes=modes)
        times.append(t)
    sec = float(np.mean(times))
    value = sl.N / sec
    line = {"metric": METRIC, "impl": "reference", "value": value, "unit": "particles/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "rbe_large: N=1e6 charges +-1 uniform in 400x400x50, "
                                   "alpha=0.1, P=200 random-batch k per call, M=16 SOE",
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "particles/s", "cores": cores,
                             "kind": "oracle", "sample": f"each of the {args.steps} steps: " + desc},
            "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    import paper_2403_01521_gb300 as qslab
    import workloads
    from paper_2403_01521_gb300.soe import load_soe

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    peaks, peak_kind = _peaks()
    M = 16
    P = 200
    soe = load_soe(M)
    sl = workloads.rbe_large(seed=3 + rank)
    N = sl.N

    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count

    def make(prec):
        return qslab.QSlab(local, prec).configure(sl.box, sl.alpha, soe, rbe=(P, 1000 + rank))

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(slab, dtype, steps, warmup, sampler=None, phase_steps=0):
        """Time `steps` calls with the library's per-phase events off and
        nothing read back between calls; then, if phase_steps > 0, as many
        more calls with the per-phase events on (read after each call) for
        the phase breakdown and the recurrence kernel's duration."""
        pos = torch.tensor(sl.pos, device=dev, dtype=dtype)
        q = torch.tensor(sl.q, device=dev, dtype=dtype)
        e = torch.empty(1, dtype=torch.float64, device=dev)
        phi = torch.empty(N, dtype=dtype, device=dev)
        F = torch.empty((N, 3), dtype=dtype, device=dev)
        qslab.qslab_set_timing(slab.h, False)
        for _ in range(warmup):
            slab.compute(pos, q, e, phi, F)
        slab.check()
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        if sampler:
            sampler.start()
        for i in range(steps):
            flush.zero_()                       # evict L2 between steps (not timed)
            ev0[i].record(stream)
            slab.compute(pos, q, e, phi, F)
            ev1[i].record(stream)
        torch.cuda.synchronize(dev)
        clocks = sampler.stop() if sampler else None
        if ws > 1:
            torch.distributed.barrier()
        slab.check()
        ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
        phases, launches = [], 0
        if phase_steps:
            qslab.qslab_set_timing(slab.h, True)
            for i in range(phase_steps):
                flush.zero_()
                slab.compute(pos, q, e, phi, F)
                ph, nl = qslab.qslab_get_timings(slab.h)
                phases.append(ph)
                launches = nl
            qslab.qslab_set_timing(slab.h, False)
            slab.check()
        return float(np.mean(ms)), phases, launches, clocks, float(e.item())

    # ---- FP32C (headline)
    s32 = make("fp32c")
    ms32, ph32, nl32, clocks, E32 = timed(s32, torch.float32, args.steps, args.warmup,
                                          ClockSampler(local), phase_steps=min(args.steps, 20))
    # ---- FP64 (reported beside it)
    s64 = make("fp64")
    st64 = max(1, min(args.steps, 3))
    ms64, ph64, _, _, E64 = timed(s64, torch.float64, st64, 1, phase_steps=1)
    s64.close()

    # slowest rank decides
    ms32_max = reduce_max(ms32, dev)
    ms64_max = reduce_max(ms64, dev)
    value = job_throughput(N, ws, ms32_max)

    # ---- end to end through the C ABI with pinned host buffers
    pos_h = torch.tensor(sl.pos, dtype=torch.float32).pin_memory()
    q_h = torch.tensor(sl.q, dtype=torch.float32).pin_memory()
    e_h = torch.zeros(1, dtype=torch.float64).pin_memory()
    phi_h = torch.zeros(N, dtype=torch.float32).pin_memory()
    F_h = torch.zeros((N, 3), dtype=torch.float32).pin_memory()
    for _ in range(2):
        qslab.qslab_compute_host(s32.h, N, pos_h.data_ptr(), q_h.data_ptr(), e_h.data_ptr(),
                                 phi_h.data_ptr(), F_h.data_ptr(), stream.cuda_stream)
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        qslab.qslab_compute_host(s32.h, N, pos_h.data_ptr(), q_h.data_ptr(), e_h.data_ptr(),
                                 phi_h.data_ptr(), F_h.data_ptr(), stream.cuda_stream)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = reduce_max(float(np.mean(e2e_ms)), dev)
    s32.close()

    # ---- roofline of the dominant kernel (the recurrences + gather)
    rec_ms = float(np.mean([p["recurrence"] for p in ph32]))
    work = algorithmic_instr(P, N, M)
    achieved = work / (rec_ms * 1e-3) / 1e12
    smax = float(peaks.get("sm_max_mhz", 2070.0))
    peak = sm_count * FP32_LANES_PER_SM * smax * 1e6 / 1e12
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        try:
            with open(tpath) as fh:
                tj = json.load(fh)
            if tj.get("sources_sha256") == kernel_sources_sha256(tj.get("sources", [])):
                traffic = tj.get("recurrence_bytes_per_launch")
        except (OSError, ValueError):
            traffic = None

    phases = {k: float(np.mean([p[k] for p in ph32])) for k in qslab.TIMING_PHASES}
    # measured arithmetic rates of this GPU (project microbenchmark), beside
    # the peak derived from unit counts and the clock
    mp = qslab.qslab_measure_peaks(local, stream.cuda_stream)
    line = {
        "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms32_max,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "rbe_large: N=1e6 charges +-1 uniform in 400x400x50, alpha=0.1, "
                               "P=200 random-batch k per call (sampled on the device), "
                               "M=16 SOE (conditioned table), compensated FP32 "
                               "(FP32 phases and in-chunk scans, chunk aggregates as split-TF32 "
                               "tensor-core products with FP32 accumulation, double-float chunk "
                               "carries, k=0 prefix sums and per-particle reductions)",
                   "N": N, "P": P, "M": M, "per_rank": "independent replica",
                   "l2": "flushed between steps (256 MB write, untimed)"},
        "fp64": {"value": job_throughput(N, ws, ms64_max), "unit": "particles/s", "ms_per_step": ms64_max,
                 "steps": st64, "energy": E64,
                 "roofline": {"bound": "fp64", "kernel": "kspace_final_kernel<double> (recurrences "
                                                       "+ gather, FP64)",
                              "achieved": work / (ph64[0]["recurrence"] * 1e-3) / 1e12,
                              "peak": mp["fp64_fma"] / 1e12, "unit": "Tinstr/s",
                              "frac": work / (ph64[0]["recurrence"] * 1e-3) / mp["fp64_fma"],
                              "kernel_ms": ph64[0]["recurrence"],
                              "peak_basis": "measured FP64 FMA rate (qslab_measure_peaks)",
                              "work": "the same K*N*(24*(M+1)+20) count, in FP64 instructions"}},
        "energy_fp32c": E32,
        "phases_ms": phases,
        "roofline": {"bound": "alu", "kernel": "kspace_final_f2_kernel (recurrences + gather)",
                     "achieved": achieved, "peak": peak, "unit": "Tinstr/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel_ms": rec_ms,
                     "timing": f"CUDA events around the kernel on its stream, mean of "
                               f"{len(ph32)} calls after the timed loop (same inputs, L2 "
                               f"flushed)",
                     "peak_basis": f"{sm_count} SMs (device query) x {FP32_LANES_PER_SM} FP32 "
                                   f"lanes x {smax:.0f} MHz ({peak_kind} max SM clock)",
                     "work": "K*N*(24*(M+1)+20) FP32 instructions per launch",
                     "measured_tops": {k: v / 1e12 for k, v in mp.items()},
                     "frac_of_measured_fp32_fma": achieved / (mp["fp32_fma"] / 1e12)},
        "e2e": {"value": job_throughput(N, ws, e2e_ms), "unit": "particles/s",
                "h2d_bytes_per_step": int(N * 3 * 4 + N * 4),
                "d2h_bytes_per_step": int(8 + N * 4 + N * 12)},
        "clocks": clocks,
        "gpu_launches": int(nl32) * args.steps,
        "gpu_launches_per_step": int(nl32),
    }
    if not args.no_batched:
        line["batched"] = run_batched(args, qslab, soe, dev, ws, rank, local, peak, smax)
    line["realspace"] = run_realspace(args, qslab, soe, dev, ws)
    line["virial"] = run_virial(args, qslab, soe, dev, ws, sl, P, ms32_max)
    line["energy_only"] = run_energy_only(args, qslab, soe, dev, ws, sl, P, ms32_max)
    line["md"] = run_md(args, qslab, soe, dev, ws)
    line["configs"] = run_configs(args, qslab, dev, ws, smax, sm_count)
    if rank == 0 and not args.no_cpu_baseline and ws == 1:
        t, desc, cores = cpu_oracle_call(sl, soe, P, 1000)
        t1, desc1 = cpu_oracle_single_core(P, 1000)
        line["cpu_baseline"] = {"value": N / t, "unit": "particles/s", "cores": cores,
                                "kind": "oracle", "sample": desc,
                                "single_core_value": (N / t1) if t1 else None,
                                "single_core_sample": desc1}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_batched(args, qslab, soe, dev, ws, rank, local, peak, smax):
    """The 512-replica workload (N per replica uniform in [500, 50000], number
    density 0.05, Lz uniform in [5, 40], charges +-1, random batch P = 200,
    M = 16, alpha = 0.25), FP32C, as one qslab_compute_batched() call
    captured in a CUDA graph after the autotuner picked the launch shape;
    the timed steps are graph replays (each draws a fresh sample). The
    inputs (206 MB) and the workspace exceed L2, so no flush is needed. The
    FP64 form of the same call is timed beside it (no graph)."""
    import torch

    import workloads
    reps = workloads.replicas(seed=4 + rank)
    sizes = [r.N for r in reps]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    boxes = np.array([r.box for r in reps])
    pos = np.concatenate([r.pos for r in reps])
    q = np.concatenate([r.q for r in reps])
    Ntot = int(off[-1])
    P, M = 200, 16
    stream = torch.cuda.current_stream(dev)
    out = {"workload": "512 independent neutral slabs, N per slab uniform in [500, 50000], "
                       "Lx=Ly from number density 0.05, Lz uniform in [5, 40], charges +-1, "
                       "alpha=0.25, random batch P=200 per slab, M=16, compensated FP32, "
                       "one batched call replayed from a CUDA graph",
           "replicas": len(reps), "N_total": Ntot, "unit": "particles/s",
           "l2": "inputs and workspace larger than L2 (no flush)"}
    s = qslab.QSlab(local, "fp32c").configure(reps[0].box, 0.25, soe, rbe=(P, 7000 + rank))
    tpos = torch.tensor(pos, device=dev, dtype=torch.float32)
    tq = torch.tensor(q, device=dev, dtype=torch.float32)
    t0 = time.perf_counter()
    out["tuning"] = list(s.autotune(tpos, tq, off, boxes, reps=2))
    out["autotune_s"] = time.perf_counter() - t0
    # one timed call outside the graph for the per-phase breakdown
    qslab.qslab_set_timing(s.h, True)
    s.compute_batched(tpos, tq, off, boxes)
    ph, nl = qslab.qslab_get_timings(s.h)
    qslab.qslab_set_timing(s.h, False)
    g = qslab.GraphedBatch(s, tpos, tq, off, boxes)
    for _ in range(args.warmup):
        g.replay()
    s.check()
    steps = args.steps
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    for i in range(steps):
        ev0[i].record(stream)
        g.replay()
        ev1[i].record(stream)
    torch.cuda.synchronize(dev)
    if ws > 1:
        torch.distributed.barrier()
    s.check()
    ms = reduce_max(float(np.mean([a.elapsed_time(b) for a, b in zip(ev0, ev1)])), dev)
    out.update({"value": job_throughput(Ntot, ws, ms), "ms_per_step": ms, "steps": steps,
                "warmup": args.warmup, "graph": True, "gpu_launches_per_step": nl,
                "phases_ms": dict(ph)})
    rec_ms = ph["recurrence"]
    achieved = algorithmic_instr(P, Ntot, M) / (rec_ms * 1e-3) / 1e12
    out["roofline"] = {"bound": "alu", "kernel": "kspace_final_kernel (recurrences + gather)",
                       "achieved": achieved, "peak": peak, "unit": "Tinstr/s",
                       "frac": achieved / peak, "traffic": None,
                       "note": "recurrence phase of one timed call outside the graph"}
    del g
    s.close()
    # FP64 form of the same batched call
    s64 = qslab.QSlab(local, "fp64").configure(reps[0].box, 0.25, soe, rbe=(P, 7000 + rank))
    tpos = torch.tensor(pos, device=dev, dtype=torch.float64)
    tq = torch.tensor(q, device=dev, dtype=torch.float64)
    outs = s64.compute_batched(tpos, tq, off, boxes)
    s64.check()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n64 = 2
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(n64):
        s64.compute_batched(tpos, tq, off, boxes, *outs)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    s64.check()
    ms64 = reduce_max(e0.elapsed_time(e1) / n64, dev)
    out["fp64"] = {"value": job_throughput(Ntot, ws, ms64), "unit": "particles/s",
                   "ms_per_step": ms64, "steps": n64}
    s64.close()
    return out


def run_md(args, qslab, soe, dev, ws):
    """Langevin steps of Section 5.2's cation-only system (436 cations in
    100 x 100 x 30 between an uncharged wall and one at -0.0436, LJ
    particles and walls, alpha = 0.3, rc = 4/alpha), FP32C, random batch
    P = 100 with the Metropolis sampler, 100 steps per CUDA-graph replay.
    Each step: one long-range call, one real-space call, two MD kernels."""
    import torch

    import workloads
    sl = workloads.cations_walls()
    rng = np.random.default_rng(1)
    g = (np.arange(8) + 0.5) * 12.5
    gx, gy, gz = np.meshgrid(g, g, 2.0 + np.arange(7) * 4.3, indexing="ij")
    pos0 = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], 1)[:sl.N] + rng.uniform(-1, 1, (sl.N, 3))
    s = qslab.QSlab(dev.index or 0, "fp32c").configure(sl.box, 0.3, soe, rbe=(100, 7), rcut=4 / 0.3)
    s.sampler("metropolis", 1)
    s.set_walls(*sl.walls)
    s.md_configure(0.005, 1.0, 1.0, 1.0, (1.0, 1.0), (1.0, 0.5), 3)
    pos = torch.tensor(pos0, device=dev, dtype=torch.float32)
    vel = torch.tensor(rng.normal(size=(sl.N, 3)), device=dev, dtype=torch.float32)
    q = torch.tensor(sl.q, device=dev, dtype=torch.float32)
    F, _ = s.md_forces(pos, q, vel)
    chunk = 100
    gr = qslab.GraphedMD(s, pos, vel, q, F, chunk)
    for _ in range(3):
        gr.replay()
    reps = max(5, args.steps // 5)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(reps):
        gr.replay()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    s.check()
    ms = reduce_max(e0.elapsed_time(e1) / (reps * chunk), dev)
    s.close()
    return {"workload": "436 cations in 100x100x30, top wall -0.0436, LJ, alpha=0.3, rc=4/alpha, "
                        "RBE P=100 (Metropolis), BAOAB dt=0.005, FP32C",
            "us_per_step": 1e3 * ms, "steps_per_s": ws / (ms * 1e-3), "steps": reps * chunk}


def run_configs(args, qslab, dev, ws, smax, sm_count):
    """The other workloads of the paper's shape, full k-sum, one call per
    step (median of CUDA-event timings after warm-up, L2 flushed): the
    1000-particle parity slab, the N = 1e5 slab (FP32 vs FP64) and the
    strongly confined N = 2e5 slab with M = 24, whose differentiable form
    (energy-only forward, adjoint backward) is timed too. Particles/s per
    precision and the recurrence kernel's share of the FP32 peak."""
    import torch

    import workloads
    from paper_2403_01521_gb300.soe import load_soe
    peak = sm_count * FP32_LANES_PER_SM * smax * 1e6
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    cases = [("small_full N=1000 30x30x10 alpha=0.3 M=16 full-k", workloads.small_full(), 16),
             ("fp32_full N=1e5 100x100x20 alpha=0.25 M=16 full-k", workloads.fp32_full(), 16),
             ("confined N=2e5 200x200x2 alpha=0.2 M=24 full-k", workloads.confined(), 24)]
    out = []
    for name, sl, M in cases:
        soe = load_soe(M)
        kc = qslab.kcut_for_tail(sl.alpha, sl.tail)
        row = {"workload": name, "N": sl.N}
        for prec in ("fp32c", "fp64"):
            dt = torch.float32 if prec == "fp32c" else torch.float64
            s = qslab.QSlab(dev.index or 0, prec).configure(sl.box, sl.alpha, soe, kcut=kc)
            qslab.qslab_set_timing(s.h, True)
            pos = torch.tensor(sl.pos, device=dev, dtype=dt)
            q = torch.tensor(sl.q, device=dev, dtype=dt)
            outs = s.compute(pos, q)
            steps = 5 if prec == "fp32c" else 2
            ms, rec = [], []
            for _ in range(steps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                s.compute(pos, q, *outs)
                b.record()
                torch.cuda.synchronize(dev)
                ms.append(a.elapsed_time(b))
                rec.append(qslab.qslab_get_timings(s.h)[0]["recurrence"])
            s.check()
            K = s.num_modes()
            t = float(np.median(ms))
            row[prec] = {"particles_per_s": sl.N / (t * 1e-3), "ms_per_call": t, "modes": K}
            if prec == "fp32c":
                work = algorithmic_instr(K, sl.N, M)
                row[prec]["recurrence_frac"] = work / (float(np.median(rec)) * 1e-3) / peak
            if prec == "fp32c" and M == 24:
                # differentiable form: energy-only forward, adjoint backward
                p_ = pos.clone().requires_grad_(True)
                q_ = q.clone().requires_grad_(True)
                for _ in range(2):
                    qslab.slab_energy(p_, q_, s, adjoint=True).backward()
                ts = []
                for _ in range(3):
                    flush.zero_()
                    p_.grad = None
                    q_.grad = None
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record()
                    qslab.slab_energy(p_, q_, s, adjoint=True).backward()
                    b.record()
                    torch.cuda.synchronize(dev)
                    ts.append(a.elapsed_time(b))
                row["autograd_adjoint_ms"] = float(np.median(ts))
            s.close()
        row["fp32c_vs_fp64"] = row["fp32c"]["particles_per_s"] / row["fp64"]["particles_per_s"]
        out.append(row)
    return out


def run_energy_only(args, qslab, soe, dev, ws, sl, P, ms_plain):
    """The energy-only call (qslab_compute_energy: forward sums, no gather)
    and its adjoint (qslab_compute_adjoint: the gradient from the stored
    sorted order and carries) on the headline workload, L2 flushed between
    calls."""
    import torch
    N = sl.N
    s = qslab.QSlab(dev.index or 0, "fp32c").configure(sl.box, sl.alpha, soe, rbe=(P, 78))
    pos = torch.tensor(sl.pos, device=dev, dtype=torch.float32)
    q = torch.tensor(sl.q, device=dev, dtype=torch.float32)
    e = torch.empty(1, dtype=torch.float64, device=dev)
    phi = torch.empty(N, dtype=torch.float32, device=dev)
    F = torch.empty((N, 3), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def energy():
        qslab.qslab_compute_energy(s.h, N, pos.data_ptr(), q.data_ptr(), e.data_ptr(),
                                   stream.cuda_stream)

    def adjoint():
        qslab.qslab_compute_adjoint(s.h, phi.data_ptr(), F.data_ptr(), stream.cuda_stream)
    for _ in range(max(args.warmup, 3)):
        energy()
        adjoint()
    s.check()
    steps = max(args.steps, 5)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    torch.cuda.synchronize(dev)
    for a, b, c in ev:
        flush.zero_()
        a.record(stream)
        energy()
        b.record(stream)
        adjoint()
        c.record(stream)
    torch.cuda.synchronize(dev)
    s.check()
    ms_e = reduce_max(float(np.mean([a.elapsed_time(b) for a, b, _ in ev])), dev)
    ms_a = reduce_max(float(np.mean([b.elapsed_time(c) for _, b, c in ev])), dev)
    s.close()
    return {"workload": "energy only (qslab_compute_energy), then its adjoint "
                        "(qslab_compute_adjoint), same workload as the headline",
            "energy_ms_per_call": ms_e, "energy_particles_per_s": job_throughput(N, ws, ms_e),
            "adjoint_ms_per_call": ms_a, "energy_vs_full_call": ms_e / ms_plain,
            "steps": steps}


def run_virial(args, qslab, soe, dev, ws, sl, P, ms_plain):
    """The long-range call with the virial tensor (qslab_compute_virial) on
    the headline workload (N = 1e6, P = 200, FP32C), L2 flushed between calls
    as for the headline; and the real-space pair virial on the N = 1e5 case."""
    import torch

    import workloads
    N = sl.N
    s = qslab.QSlab(dev.index or 0, "fp32c").configure(sl.box, sl.alpha, soe, rbe=(P, 77))
    pos = torch.tensor(sl.pos, device=dev, dtype=torch.float32)
    q = torch.tensor(sl.q, device=dev, dtype=torch.float32)
    e = torch.empty(1, dtype=torch.float64, device=dev)
    phi = torch.empty(N, dtype=torch.float32, device=dev)
    F = torch.empty((N, 3), dtype=torch.float32, device=dev)
    W = torch.empty(6, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def call():
        qslab.qslab_compute_virial(s.h, N, pos.data_ptr(), q.data_ptr(), e.data_ptr(),
                                   phi.data_ptr(), F.data_ptr(), W.data_ptr(), stream.cuda_stream)
    for _ in range(max(args.warmup, 3)):
        call()
    s.check()
    steps = max(args.steps, 5)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    torch.cuda.synchronize(dev)
    for a, b in ev:
        flush.zero_()
        a.record(stream)
        call()
        b.record(stream)
    torch.cuda.synchronize(dev)
    s.check()
    ms = reduce_max(float(np.mean([a.elapsed_time(b) for a, b in ev])), dev)
    s.close()
    # real-space pair virial, N = 1e5 case of run_realspace
    rs = workloads.fp32_full()
    t = qslab.QSlab(dev.index or 0, "fp32c").configure(rs.box, 0.25, soe, kcut=1.0, rcut=10.0)
    rpos = torch.tensor(rs.pos, device=dev, dtype=torch.float32)
    rq = torch.tensor(rs.q, device=dev, dtype=torch.float32)
    for _ in range(3):
        t.compute_realspace_virial(rpos, rq)
    t.check()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(steps):
        t.compute_realspace_virial(rpos, rq)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t.check()
    rs_ms = reduce_max(e0.elapsed_time(e1) / steps, dev)
    t.close()
    return {"workload": "long-range energy, forces and virial tensor (qslab_compute_virial), "
                        "same workload as the headline (N=1e6, P=200, FP32C)",
            "ms_per_call": ms, "particles_per_s": job_throughput(N, ws, ms),
            "overhead_vs_plain": ms / ms_plain - 1.0, "steps": steps,
            "realspace_virial_ms_per_call": rs_ms,
            "realspace_workload": "N=1e5, 100x100x20, alpha=0.25, rc=10, FP32C, pair virial"}


def run_realspace(args, qslab, soe, dev, ws):
    """The real-space part (Eq. 2.10) on the N = 1e5 workload of the FP32
    full-k configuration (100 x 100 x 20, alpha = 0.25, rc = 10), FP32C:
    cell list, every pair from both ends. Pairs per second counts the pairs
    inside rc (each once per direction)."""
    import torch

    import workloads
    sl = workloads.fp32_full()
    s = qslab.QSlab(dev.index or 0, "fp32c").configure(sl.box, 0.25, soe, kcut=1.0, rcut=10.0)
    pos = torch.tensor(sl.pos, device=dev, dtype=torch.float32)
    q = torch.tensor(sl.q, device=dev, dtype=torch.float32)
    outs = s.compute_realspace(pos, q)
    for _ in range(max(args.warmup, 3)):
        s.compute_realspace(pos, q, *outs)
    s.check()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(args.steps, 5)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(steps):
        s.compute_realspace(pos, q, *outs)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    s.check()
    ms = reduce_max(e0.elapsed_time(e1) / steps, dev)
    s.close()
    # pairs inside rc: density x sphere volume, cut by the walls (estimate
    # from the uniform density over the slab thickness)
    Lx, Ly, Lz = sl.box
    rho = sl.N / (Lx * Ly * Lz)
    rc = 10.0
    # mean volume of the sphere of radius rc inside the slab, for uniform z
    zs = np.linspace(0.0, Lz, 401)
    def cap(h):   # volume of a sphere cap of height h
        h = np.clip(h, 0.0, 2 * rc)
        return np.pi * h * h * (3 * rc - h) / 3.0
    vol = 4.0 / 3.0 * np.pi * rc ** 3 - cap(rc - zs) - cap(rc - (Lz - zs))
    pairs = sl.N * rho * float(vol.mean())
    return {"workload": "N=1e5 charges +-1 uniform in 100x100x20, alpha=0.25, rc=10 (real-space "
                        "part of the FP32 full-k configuration), FP32C",
            "ms_per_call": ms, "particles_per_s": job_throughput(sl.N, ws, ms),
            "pairs_in_rc_per_s": pairs * ws / (ms * 1e-3), "steps": steps}


def profile_case(kind="single"):
    """Two FP32 calls for profilers: 'single' = the random-batch benchmark
    workload (N = 1e6); 'batched' = the first 128 slabs of the replica
    workload (about 3.3e6 particles) as one batched call, launch shape fixed
    at 512-particle chunks; 'realspace' = the real-space part on the N = 1e5
    FP32 full-k workload (rc = 10); 'single+realspace' = both, one after
    the other; 'virial' = two qslab_compute_virial calls on the benchmark
    workload (N = 1e6); 'virial-small' = the same on N = 2.5e5 at the same
    density (200 x 200 x 50), small enough for a full ncu capture; 'md' =
    four Langevin steps of the 436-cation system of run_md (no graph)."""
    import torch

    import paper_2403_01521_gb300 as qslab
    import workloads
    soe = qslab.load_soe(16)
    if kind == "single+realspace":
        profile_case("single")
        return profile_case("realspace")
    if kind == "realspace":
        sl = workloads.fp32_full()
        slab = qslab.QSlab(0, "fp32c").configure(sl.box, 0.25, soe, kcut=1.0, rcut=10.0)
        pos = torch.tensor(sl.pos, device="cuda", dtype=torch.float32)
        q = torch.tensor(sl.q, device="cuda", dtype=torch.float32)
        for _ in range(2):
            e, _, _ = slab.compute_realspace(pos, q)
        slab.check()
        torch.cuda.synchronize()
        print("profile case realspace done, E =", float(e.item()))
        return 0
    if kind == "md":
        sl = workloads.cations_walls()
        rng = np.random.default_rng(1)
        g = (np.arange(8) + 0.5) * 12.5
        gx, gy, gz = np.meshgrid(g, g, 2.0 + np.arange(7) * 4.3, indexing="ij")
        pos0 = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], 1)[:sl.N] + rng.uniform(-1, 1, (sl.N, 3))
        s = qslab.QSlab(0, "fp32c").configure(sl.box, 0.3, soe, rbe=(100, 7), rcut=4 / 0.3)
        s.sampler("metropolis", 1)
        s.set_walls(*sl.walls)
        s.md_configure(0.005, 1.0, 1.0, 1.0, (1.0, 1.0), (1.0, 0.5), 3)
        pos = torch.tensor(pos0, device="cuda", dtype=torch.float32)
        vel = torch.tensor(rng.normal(size=(sl.N, 3)), device="cuda", dtype=torch.float32)
        q = torch.tensor(sl.q, device="cuda", dtype=torch.float32)
        F, _ = s.md_forces(pos, q, vel)
        s.md_step(pos, vel, q, F, 4)
        s.check()
        torch.cuda.synchronize()
        print("profile case md done")
        return 0
    if kind in ("virial", "virial-small"):
        n = 1_000_000 if kind == "virial" else 250_000
        L = 400.0 * (n / 1e6) ** 0.5
        sl = workloads.uniform_slab(n, (L, L, 50.0), 3, alpha=0.1, P=200)
        slab = qslab.QSlab(0, "fp32c").configure(sl.box, sl.alpha, soe, rbe=(200, 5))
        pos = torch.tensor(sl.pos, device="cuda", dtype=torch.float32)
        q = torch.tensor(sl.q, device="cuda", dtype=torch.float32)
        for _ in range(2):
            e, _, _, W = slab.compute_virial(pos, q)
        slab.check()
        torch.cuda.synchronize()
        print("profile case", kind, "done, E =", float(e.item()), "W =", W.cpu().numpy().tolist())
        return 0
    if kind == "batched":
        reps = workloads.replicas()[:128]
        off = np.concatenate([[0], np.cumsum([r.N for r in reps])]).astype(np.int64)
        boxes = np.array([r.box for r in reps])
        pos = torch.tensor(np.concatenate([r.pos for r in reps]), device="cuda", dtype=torch.float32)
        q = torch.tensor(np.concatenate([r.q for r in reps]), device="cuda", dtype=torch.float32)
        slab = qslab.QSlab(0, "fp32c").configure(reps[0].box, 0.25, soe, rbe=(200, 5)).tuning(512, 0)
        for _ in range(2):
            e, _, _ = slab.compute_batched(pos, q, off, boxes)
        E = float(e.sum().item())
    else:
        sl = workloads.rbe_large()
        slab = qslab.QSlab(0, "fp32c").configure(sl.box, sl.alpha, soe, rbe=(200, 5))
        pos = torch.tensor(sl.pos, device="cuda", dtype=torch.float32)
        q = torch.tensor(sl.q, device="cuda", dtype=torch.float32)
        for _ in range(2):
            e, _, _ = slab.compute(pos, q)
        E = float(e.item())
    slab.check()
    torch.cuda.synchronize()
    print("profile case", kind, "done, E =", E)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 512-replica batched measurement")
    ap.add_argument("--profile-case", nargs="?", const="single",
                    choices=["single", "batched", "realspace", "single+realspace", "virial",
                             "virial-small", "md"],
                    help="only run two FP32 random-batch calls (for profilers)")
    args = ap.parse_args()
    if args.profile_case:
        return profile_case(args.profile_case)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
