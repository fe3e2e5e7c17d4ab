#!/usr/bin/env python
"""Throughput benchmark of the fused freezing LB time step (MLUPS, all three
D2Q9 populations) on GB300, with roofline, CPU-baseline and end-to-end figures.

A bench "step" is one time step of the whole lattice. The default workload is
the 1024 x 1024 drop with 8 bubbles on a cold wall (FP32 storage): each step
moves 268 MB, more than the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank advances its own replica of the workload
(independent lattices, no collective on the data path: weak scaling); rank 0
prints one JSON line with the aggregate over ranks and the max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS (all 3 populations) & % HBM peak; FP16-store/batched vs plain FP32"
BYTES_PER_LU_FP32 = 256  # 27 populations + 5 carried fields, read + write, FP32
BYTES_PER_LU_FP16 = 176  # 24 16-bit populations + 10 FP32 planes (5 carried, phi/T refs, 3 rest pops), read + write
WORKLOAD = "bubble_drop_1024x1024_fp32"


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--runs", type=int, default=5,
                    help="timed runs of --steps steps each; the best is reported")
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--size", dest="n", type=int, default=1024, help="lattice size of the bubble drop")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tune-steps", type=int, default=20)
    ap.add_argument("--kernel", default=None,
                    help="fixed layout 'kind,a,b,c' as lbm_set_kernel takes it (skips the autotuner)")
    ap.add_argument("--storage", choices=("fp32", "fp16"), default="fp32",
                    help="storage of the main timed lattice (the metric is quoted on fp32)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the FP16-storage comparison on the same workload")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched forms (256-lattice sweep, 1024-lattice FP16 batch)")
    ap.add_argument("--batched-steps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    return ap.parse_args(argv)


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU)
# ---------------------------------------------------------------------------

class Dist:
    def __init__(self, want: int):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist

            backend = os.environ.get("LBM_BENCH_BACKEND", "nccl")
            if backend == "nccl":
                import torch
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            if self.pg.get_backend() == "nccl":
                import torch
                self.pg.barrier(device_ids=[torch.cuda.current_device()])
            else:
                self.pg.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, v: float) -> float:
        if not self.pg:
            return v
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def aggregate(per_rank_sites_steps: float, per_rank_ms: float, dist: Dist):
    """Whole-job throughput: units of all ranks over the slowest rank's time."""
    total = dist.sum(per_rank_sites_steps)
    ms = dist.max(per_rank_ms)
    return total / (ms * 1e-3) / 1e6, ms


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_s: float = 0.1):
        self.idx = gpu_index
        self.period = period_s
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _one(self):
        try:
            r = subprocess.run(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.QUERY}",
                                "--format=csv,noheader,nounits"], capture_output=True, text=True,
                               timeout=5)
            vals = [v.strip() for v in r.stdout.strip().split(",")]
            if len(vals) >= 7:
                self.samples.append(vals)
        except Exception:
            pass

    def _run(self):
        while not self._stop.is_set():
            self._one()
            self._stop.wait(self.period)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        self._t.join(timeout=10)
        self._one()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for s in self.samples for j in range(4)
                          if s[3 + j].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# ---------------------------------------------------------------------------
# roofline helpers
# ---------------------------------------------------------------------------

NOMINAL_HBM_GBS = 8000.0  # GB300 HBM3e, nominal


def measured_hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in ("lbm_kernels.cu", "lbm_internal.h"):
        with open(os.path.join(ROOT, "paper_2403_16122_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str):
    """(DRAM bytes per launch, the kernel they were counted on) of the step
    kernel from the committed ncu summary, if it was taken on the current
    kernel source; else (None, None)."""
    path = os.path.join(ROOT, "profiles", f"step_{workload}.md")
    try:
        txt = open(path).read()
    except OSError:
        return None, None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)\s+kernel_source:\s*([0-9a-f]+)", txt)
    if not m or m.group(2) != kernel_source_hash():
        return None, None
    k = re.search(r"Kernel: `([^`]+)`", txt)
    return float(m.group(1)), (k.group(1) if k else None)


# ---------------------------------------------------------------------------
# the oracle (CPU baseline / reference arm)
# ---------------------------------------------------------------------------

def host_cores() -> int:
    """Cores this process may run on (nproc)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_rate(n: int, target_s: float, threads: int):
    """Time the FP64 oracle on the bubble-drop lattice of size n with
    `threads` host threads (OpenMP over rows). Returns (MLUPS, steps,
    seconds, threads in effect)."""
    import oracle
    from paper_2403_16122_gb300 import inputs

    used = oracle.set_threads(threads)
    p, phi0, T0 = inputs.bubbles_drop(n=n)
    o = oracle.Oracle(p).init(phi0, T0)
    t0 = time.perf_counter()
    o.step(1)
    per = time.perf_counter() - t0
    steps = max(1, int(target_s / max(per, 1e-6)))
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return n * n * steps / dt / 1e6, steps, dt, used


def run_reference(args, dist: Dist):
    """The oracle as it stands, timed on the host cores (rank 0 only)."""
    if dist.rank != 0:
        return 0
    import oracle
    from paper_2403_16122_gb300 import inputs

    oracle.build()
    cores = oracle.set_threads(host_cores())
    n = args.n
    p, phi0, T0 = inputs.bubbles_drop(n=n)
    o = oracle.Oracle(p).init(phi0, T0)
    t0 = time.perf_counter()
    o.step(1)
    per = time.perf_counter() - t0
    # bound the whole run to a few minutes: shrink the per-step sample if needed
    if per * (args.steps + args.warmup) > 150.0:
        n = 256
        p, phi0, T0 = inputs.bubbles_drop(n=n)
        o = oracle.Oracle(p).init(phi0, T0)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    value = n * n * args.steps / dt / 1e6
    sample = (f"{args.steps} oracle steps of the bubble drop at {n}x{n} (FP64, OpenMP over rows, "
              f"{cores} threads)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": args.n, "ny": args.n, "sample_n": n},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args, dist: Dist):
    import numpy as np
    import torch

    from paper_2403_16122_gb300 import build as lbm_build
    from paper_2403_16122_gb300 import inputs, lbm

    if dist.rank == 0 or not os.path.exists(lbm.LIB_PATH):
        lbm_build.build()
    dist.barrier()
    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    n = args.n
    p, phi0, T0 = inputs.bubbles_drop(n=n)
    sites = n * n
    fp16 = args.storage == "fp16"
    bytes_lu = BYTES_PER_LU_FP16 if fp16 else BYTES_PER_LU_FP32
    workload = WORKLOAD.replace("fp32", "fp16") if fp16 else WORKLOAD
    lat = lbm.Lattice([p], storage=lbm.LBM_STORE_FP16 if fp16 else lbm.LBM_STORE_FP32, device=dev)
    stream = lat.stream
    lat.init(phi0, T0)

    # warm-up, including the library's autotuner (it advances the lattice with
    # ordinary steps while it times each kernel layout)
    tune = None
    if args.warmup:
        lat.step(args.warmup)
    if args.kernel:
        lat.set_kernel(*[int(v) for v in args.kernel.split(",")])
    elif not args.no_autotune:
        tune = [float(t) for t in lat.autotune(steps=args.tune_steps)]
    kernel = lat.kernel
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()

    # the timed region: exactly K steps (one lbm_step(K) call: K - 1 plain
    # steps and the observable step that ends every call), run `runs` times
    # back to back; the best run is reported, every run is listed
    launches0 = lat.launch_count
    runs_ms = []
    with ClockSampler(torch.cuda.current_device()) as clocks:
        for _ in range(args.runs):
            start = torch.cuda.Event(enable_timing=True)
            end = torch.cuda.Event(enable_timing=True)
            start.record(stream)
            lat.step(args.steps)
            end.record(stream)
            end.synchronize()
            runs_ms.append(start.elapsed_time(end))
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    ms = min(runs_ms)
    launches = (lat.launch_count - launches0) // args.runs
    obs = lat.observables(check=False)

    value, ms_max = aggregate(sites * args.steps, ms, dist)
    ms_per_step = ms_max / args.steps

    # roofline of the dominant kernel (the fused step), from the same events
    peak, peak_kind = measured_hbm_peak()
    achieved = bytes_lu * sites / (ms / args.steps * 1e-3) / 1e9
    traffic, traffic_kernel = profiled_traffic(workload)
    # counters taken on another kernel family say nothing about this one
    family = {lbm.LBM_KERNEL_TILE: "step_fp32<", lbm.LBM_KERNEL_STRIP: "step_strip<",
              lbm.LBM_KERNEL_STAGED: "step_strip_staged<",
              lbm.LBM_KERNEL_BLOCK: "step_block<"}.get(int(kernel[0]))
    if traffic_kernel is None or family is None or not traffic_kernel.startswith(family):
        traffic, traffic_kernel = None, None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                # the variant the counters were taken on (the autotuner may pick
                # a sibling with the same items and ring: the same traffic)
                "traffic_kernel": traffic_kernel,
                "peak_kind": peak_kind,
                # the same against the nominal HBM3e peak of the part
                "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "nominal_peak": NOMINAL_HBM_GBS,
                "algorithmic_bytes_per_launch": bytes_lu * sites}

    # end to end through the C-ABI with host buffers: upload the fields from
    # pinned memory, then per step one time step and a read of the observables
    e2e = None
    if not args.no_e2e:
        k_e2e = max(1, min(args.steps, 2000))
        ph = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        tt = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        ph.numpy()[:] = phi0
        tt.numpy()[:] = T0
        lat2 = lbm.Lattice([p], device=dev)
        # tuned, as a caller reading the observables after every step would,
        # on single observable steps; then back to the initial state
        lat2.init(ph.numpy(), tt.numpy())
        lat2.autotune(steps=1)
        kernel_e2e = lat2.kernel
        torch.cuda.synchronize()
        dist.barrier()
        t0 = time.perf_counter()
        lat2.init(ph.numpy(), tt.numpy())
        for _ in range(k_e2e):
            lbm.lbm_step(lat2.handle, 1)
            lbm.lbm_observables(lat2.handle, 0, check=False)
        dt = time.perf_counter() - t0
        ev, _ = aggregate(sites * k_e2e, dt * 1e3, dist)
        e2e = {"value": ev, "unit": "MLUPS", "h2d_bytes_per_step": 16 * sites / k_e2e,
               "d2h_bytes_per_step": 8 * lbm.LBM_OBS_COUNT, "steps": k_e2e,
               "kernel": list(kernel_e2e),
               "what": "lbm_init_fields from pinned host phi0/T0, then per step lbm_step(1) + "
                       "lbm_observables (device-to-host read, synchronising); the kernel "
                       "tuned by lbm_autotune on single observable steps, before the timed region"}
        # a caller that reads the observables every 20 steps (the plain-step
        # kernel layout the timed run used)
        every = 20
        lat2.set_kernel(*kernel)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat2.init(ph.numpy(), tt.numpy())
        n_calls = max(1, k_e2e // every)
        for _ in range(n_calls):
            lbm.lbm_step(lat2.handle, every)
            lbm.lbm_observables(lat2.handle, 0, check=False)
        dt = time.perf_counter() - t0
        ev20, _ = aggregate(sites * every * n_calls, dt * 1e3, dist)
        e2e["observables_every_20_steps"] = {
            "value": ev20, "unit": "MLUPS", "steps": every * n_calls,
            "h2d_bytes_per_step": 16 * sites / (every * n_calls),
            "d2h_bytes_per_step": 8 * lbm.LBM_OBS_COUNT / every, "kernel": list(kernel)}
        lat2.close()

    # the FP16-storage form on the same workload and GPU (FP32 arithmetic)
    forms = None
    if not args.no_forms:
        forms = {}
        lat16 = lbm.Lattice([p], storage=lbm.LBM_STORE_FP16, device=dev)
        lat16.init(phi0, T0)
        lat16.step(max(args.warmup, 3))
        if not args.no_autotune:
            lat16.autotune(steps=args.tune_steps)
        k16 = max(1, min(args.steps, 3000))
        ms16 = _timed_steps(lat16, k16, runs=args.runs)
        ob16 = lat16.observables(check=False)
        forms["fp16_storage"] = {
            "value": sites / (ms16 * 1e-3) / 1e6, "unit": "MLUPS", "steps": k16,
            "ms_per_step": ms16, "bytes_per_lu": BYTES_PER_LU_FP16,
            "hbm_frac": BYTES_PER_LU_FP16 * sites / (ms16 * 1e-3) / 1e9 / peak,
            "speedup_vs_fp32": ms_per_step / ms16,
            "kernel": list(lat16.kernel),
            "observables_after_warmup_and_steps": {k: ob16[k] for k in ("solid", "volume")},
        }
        lat16.close()

    # BF16 storage (same arrangement, bfloat16 values) on the same lattice
    if forms is not None:
        latb = lbm.Lattice([p], storage=lbm.LBM_STORE_BF16, device=dev)
        latb.init(phi0, T0)
        latb.step(max(args.warmup, 3))
        if not args.no_autotune:
            latb.autotune(steps=args.tune_steps)
        kb = max(1, min(args.steps, 3000))
        msb = _timed_steps(latb, kb, runs=args.runs)
        forms["bf16_storage"] = {
            "value": sites / (msb * 1e-3) / 1e6, "unit": "MLUPS", "steps": kb, "ms_per_step": msb,
            "bytes_per_lu": BYTES_PER_LU_FP16,
            "hbm_frac": BYTES_PER_LU_FP16 * sites / (msb * 1e-3) / 1e9 / peak,
            "speedup_vs_fp32": ms_per_step / msb, "kernel": list(latb.kernel)}
        latb.close()

    # the Boussinesq option (Section 4.3) on the same lattice: one more force
    # term per site
    if forms is not None:
        pb = dict(p, gy=-1e-4, beta_T=1.0, T_ref=p["T_m"], rho_0=1.0)
        latb = lbm.Lattice([pb], device=dev)
        latb.init(phi0, T0)
        latb.set_kernel(*kernel)
        latb.step(max(args.warmup, 3))
        kb = max(1, min(args.steps, 2000))
        msb = _timed_steps(latb, kb)
        forms["boussinesq"] = {"value": sites / (msb * 1e-3) / 1e6, "unit": "MLUPS", "steps": kb,
                               "ms_per_step": msb, "kernel": list(latb.kernel),
                               "relative_to_plain": ms_per_step / msb}
        latb.close()

    # the Stefan problem of Section 4.1 (256 x 8 cells, walls in x: the tile
    # kernel): 2048 sites a step, so launch-bound; one launch per step against
    # runs of steps replayed from a CUDA graph
    if forms is not None:
        ps, phis, Ts = inputs.stefan()
        st_out = {}
        for name, mode in (("launch", lbm.LBM_EXEC_LAUNCH), ("graph", lbm.LBM_EXEC_GRAPH)):
            lats = lbm.Lattice([ps], device=dev)
            lats.init(phis, Ts)
            lats.set_exec(mode, 500)
            lats.step(501)
            mss = _timed_steps(lats, 5000)
            st_out[name] = {"value": ps["nx"] * ps["ny"] / (mss * 1e-3) / 1e6, "ms_per_step": mss,
                            "kernel": list(lats.kernel)}
            lats.close()
        forms["stefan_256x8"] = {"value": max(v["value"] for v in st_out.values()), "unit": "MLUPS",
                                 "steps": 5000, **st_out,
                                 "what": "launch-bound: 2048 sites a step"}

    if forms is not None and not args.no_batched:
        forms.update(batched_forms(args, dev, peak))

    cpu = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        import oracle

        oracle.build()
        rate, st, sec, cores = oracle_rate(n, args.cpu_seconds, host_cores())
        rate1, st1, sec1, _ = oracle_rate(n, args.cpu_seconds / 3, 1)
        cpu = {"value": rate, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"{st} FP64 oracle steps of the {n}x{n} bubble drop ({sec:.1f} s, "
                         f"OpenMP over rows on {cores} threads)",
               "single_core": {"value": rate1, "unit": "MLUPS", "cores": 1,
                               "sample": f"{st1} steps ({sec1:.1f} s, one thread)"}}

    if dist.rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": dist.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "runs_ms_per_step": [t / args.steps for t in runs_ms],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload, "nx": n, "ny": n, "sites": sites,
                       "storage": args.storage, "bubbles": 8, "parallelism": f"replicas{dist.world}",
                       "l2": "inputs larger than L2 (268 MB moved per step)",
                       "bytes_per_lu": bytes_lu},
            "roofline": roofline,
            "forms": forms,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "kernel": {"kind": {0: "tile", 1: "strip", 2: "staged", 3: "block"}.get(kernel[0], str(kernel[0])),
                       "params": list(kernel[1:]),
                       "autotune_ms_per_step": tune},
            "clocks": clocks.summary(),
            "observables": {k: obs[k] for k in ("solid", "volume", "nonfinite")},
        }
        print(json.dumps(line), flush=True)
    lat.close()
    return 0


def _timed_steps(lat, k, runs=1):
    """Mean ms per step of k steps of handle `lat` (one lbm_step(k) call),
    CUDA events on its stream; the best of `runs` such calls."""
    import torch

    torch.cuda.synchronize()
    best = None
    for _ in range(runs):
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(lat.stream)
        lat.step(k)
        e.record(lat.stream)
        e.synchronize()
        t = s.elapsed_time(e) / k
        best = t if best is None else min(best, t)
    return best


def _batch_handle(cases, storage, dev, exec_mode, chunk, tune_steps):
    from paper_2403_16122_gb300 import lbm

    lat = lbm.Lattice([c[0] for c in cases], storage=storage, device=dev)
    for k, (_, phi0, T0) in enumerate(cases):
        lat.init(phi0, T0, inst=k)
    lat.step(3)
    lat.set_exec(exec_mode, chunk)
    if tune_steps:  # timed in the form that will run (candidates' graphs are dropped)
        lat.autotune(steps=tune_steps)
    lat.step(chunk + 1)  # captures the graph of the chosen layout
    # start the timed run from step 0, so that forms compare at equal steps
    for k, (_, phi0, T0) in enumerate(cases):
        lat.init(phi0, T0, inst=k)
    return lat


def batched_forms(args, dev, peak):
    """The batched forms on the same GPU: (1) 256 sessile drops of uneven
    size (grids 128..512 squared) in one handle, persistent launch replayed
    from a CUDA graph, against the same drops advanced one lattice per launch;
    (2) 1024 drops with 0-4 bubbles (grids 64..256 per side) in FP16 storage
    against the same batch in FP32, both persistent."""
    import numpy as np

    from paper_2403_16122_gb300 import inputs, lbm

    out = {}
    k = max(8, args.batched_steps)
    chunk = 64
    tune = 0 if args.no_autotune else 4

    sweep = inputs.batched_sweep(256)
    sites = sum(p["nx"] * p["ny"] for p, _, _ in sweep)
    lat = _batch_handle(sweep, lbm.LBM_STORE_FP32, dev, lbm.LBM_EXEC_PERSISTENT, chunk, tune)
    ms_b = _timed_steps(lat, k)
    ex, kern = lat.exec, lat.kernel
    ob = lat.observables_all(check=False)
    # the same batch with the steps replayed from a graph of launches
    lat.set_exec(lbm.LBM_EXEC_GRAPH, chunk).step(chunk + 1)
    ms_g = _timed_steps(lat, k)
    lat.close()
    # the same lattices, one handle and one launch per lattice and step
    singles = []
    for c in sweep:
        h = lbm.Lattice([c[0]], device=dev)
        h.init(c[1], c[2]).step(3)
        singles.append(h)
    k1 = max(4, k // 10)
    per = []
    import torch
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    stream = singles[0].stream
    t0.record(stream)
    for h in singles:  # one lattice after the other
        h.step(k1)
    t1.record(stream)
    t1.synchronize()
    ms_p = t0.elapsed_time(t1) / k1
    for h in singles:  # each lattice's own step time when run by itself
        per.append(_timed_steps(h, 8))
        h.close()
    per = np.array(per)
    out["batched_fp32_sweep256"] = {
        "value": sites / (ms_b * 1e-3) / 1e6, "unit": "MLUPS", "instances": len(sweep),
        "sites": sites, "steps": k, "ms_per_step": ms_b,
        "hbm_frac": BYTES_PER_LU_FP32 * sites / (ms_b * 1e-3) / 1e9 / peak,
        "exec": {"mode": "persistent+graph", "chunk": ex[1], "ctas": ex[2]},
        "kernel": list(kern),
        "graph_of_launches": {"value": sites / (ms_g * 1e-3) / 1e6, "ms_per_step": ms_g},
        "unbatched": {"value": sites / (ms_p * 1e-3) / 1e6, "unit": "MLUPS", "steps": k1,
                      "ms_per_step": ms_p, "what": "one handle per lattice, advanced one lattice after the other, one launch per step"},
        "speedup_vs_unbatched": ms_p / ms_b,
        "instance_ms_per_step": {"batched_all": ms_b,
                                 "alone_p50": float(np.percentile(per, 50)),
                                 "alone_p99": float(np.percentile(per, 99))},
        "nonfinite": float(ob[:, lbm.OBS_NAMES.index("nonfinite")].sum()),
    }

    mixed = inputs.batched_bubbles(1024)
    sites = sum(p["nx"] * p["ny"] for p, _, _ in mixed)
    res = {}
    for name, st in (("fp32", lbm.LBM_STORE_FP32), ("fp16", lbm.LBM_STORE_FP16)):
        lat = _batch_handle(mixed, st, dev, lbm.LBM_EXEC_PERSISTENT, chunk, tune)
        ms = _timed_steps(lat, k)
        res[name] = (ms, lat.exec, lat.kernel, lat.observables_all(check=False))
        lat.close()
    ms32, ms16 = res["fp32"][0], res["fp16"][0]
    # each lattice's own step time when run by itself, on a seeded sample of
    # the batch (every one of the 1024 would take most of a minute)
    pick = np.random.default_rng(20240324).choice(len(mixed), size=min(64, len(mixed)),
                                                  replace=False)
    alone = {}
    for name, st in (("fp32", lbm.LBM_STORE_FP32), ("fp16", lbm.LBM_STORE_FP16)):
        per = []
        for i in sorted(pick.tolist()):
            c = mixed[i]
            h = lbm.Lattice([c[0]], storage=st, device=dev)
            h.init(c[1], c[2]).step(3)
            per.append(_timed_steps(h, 8))
            h.close()
        alone[name] = np.array(per)
    i_s, i_v = lbm.OBS_NAMES.index("solid"), lbm.OBS_NAMES.index("volume")
    o32, o16 = res["fp32"][3], res["fp16"][3]
    out["batched_fp16_bubbles1024"] = {
        "value": sites / (ms16 * 1e-3) / 1e6, "unit": "MLUPS", "instances": len(mixed),
        "sites": sites, "steps": k, "ms_per_step": ms16,
        "hbm_frac": BYTES_PER_LU_FP16 * sites / (ms16 * 1e-3) / 1e9 / peak,
        "fp32_batched": {"value": sites / (ms32 * 1e-3) / 1e6, "ms_per_step": ms32,
                         "hbm_frac": BYTES_PER_LU_FP32 * sites / (ms32 * 1e-3) / 1e9 / peak,
                         "kernel": list(res["fp32"][2])},
        "speedup_vs_fp32_batched": ms32 / ms16,
        "exec": {"mode": "persistent+graph", "chunk": res["fp16"][1][1], "ctas": res["fp16"][1][2]},
        "kernel": list(res["fp16"][2]),
        "instance_ms_per_step": {
            "batched_all": ms16, "batched_all_fp32": ms32, "alone_sample": int(len(pick)),
            "alone_p50": float(np.percentile(alone["fp16"], 50)),
            "alone_p99": float(np.percentile(alone["fp16"], 99)),
            "alone_fp32_p50": float(np.percentile(alone["fp32"], 50)),
            "alone_fp32_p99": float(np.percentile(alone["fp32"], 99))},
        "max_rel_diff_vs_fp32": {
            "volume": float(np.max(np.abs(o16[:, i_v] - o32[:, i_v]) / np.abs(o32[:, i_v]))),
            "solid": float(np.max(np.abs(o16[:, i_s] - o32[:, i_s]) / np.maximum(o32[:, i_s], 1.0))),
        },
    }
    return out


def main(argv=None):
    args = parse_args(argv)
    dist = Dist(args.gpus)
    try:
        if args.impl == "reference":
            return run_reference(args, dist)
        return run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    sys.exit(main())
