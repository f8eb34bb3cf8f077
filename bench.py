#!/usr/bin/env python3
"""Benchmark of the D1Q3 Monte Carlo Lattice Gas step on GB300.

One "step" is one MCLG time step (pull streaming + C = 10 exact random
sub-collisions per node) of the whole workload.  Default workload: one
periodic lattice of 2^24 nodes, rho = 100 (1 + 0.01 sin(2 pi 4 x / L)), u = 0,
Poisson(f^eq) initial state (the paper-shaped single-lattice run), 10^4 steps
timed after the warm-up.  The state (192 MiB double-buffered) is larger than
L2, so no flush is needed between steps.

Metric: GSUPS = node updates per second / 1e9, whole job (all ranks).
Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the CPU oracle on the same workload
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1706_01094_gb300 import workloads  # noqa: E402



def metric(C: int = 10) -> str:
    return f"MCLG site updates/sec (GSUPS), D1Q3 C={C} lambda=1, bit-exact vs CPU oracle"


BYTES_PER_NODE_STEP = 12        # 3 uint16 read + 3 uint16 written


def int_ops_per_node_step(C: int) -> int:
    """Algorithmic integer operations of the sequential sampler per node-step: one
    Philox4x32-10 block per 10 decisions = 10 rounds x (2 mul-hi + 2 mul-lo + 4 xor)
    + 9 x 2 key adds = 98; each sub-collision = 3 mul (a c, b (b-1), q D) + 2 shifts
    + 1 add (thresholds) + 4 compares + 3 adds (state update) = 13."""
    return 98 * max(1, -(-C // 10)) + 13 * C


INT32_LANES_PER_SM_CLK = 64     # integer pipe lanes per SM and clock (unit count of the ALU pipe)


def sm_count(index: int = 0) -> int:
    """Streaming multiprocessors of the GPU, from the device attribute."""
    import torch
    return int(torch.cuda.get_device_properties(index).multi_processor_count)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10_000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="single",
                    choices=["single", "batched", "uneven", "small", "fluct", "d2q9"])
    ap.add_argument("--u", type=float, default=0.2, help="velocity of the fluct workload")
    ap.add_argument("--C", type=int, default=10,
                    help="sub-collisions per node and step (the paper's runs: 10)")
    ap.add_argument("--sampler", default="auto", choices=["auto", "slice", "sequential"],
                    help="slice: the C sub-collisions of a node drawn at once from exact "
                         "cumulative-law tables; sequential: one sub-collision at a time "
                         "(the persistent batched kernel); auto: slice (tables to mass 512 for "
                         "the batches)")
    ap.add_argument("--mode", default="auto", choices=["auto", "plain", "persistent", "batched"])
    ap.add_argument("--slice-n-max", type=int, default=0,
                    help="slice sampler: largest node mass the tables cover (0: the library's "
                         "256; 512 for the batches, whose densities reach 500 and 1000)")
    ap.add_argument("--kernel-variant", type=int, default=None,
                    help="fix the per-step kernel's launch variant (default: autotuned)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched and statistics workloads that the default "
                         "single-lattice run reports beside its headline")
    return ap.parse_args()


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def committed_figure(kernel: str, workload: str, key: str = "dram_bytes_per_launch",
                     variant=None):
    """A figure (per-launch DRAM bytes by default) of `kernel` from the committed ncu
    summary of that kernel on that workload, if there is one.  A summary that names
    the launch variant it captured gives its figures for that variant only: with
    `variant` set to another one the figure is None."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    for line in lines:
        if variant is not None and line.startswith("variant:"):
            if int(line.split(":", 1)[1].split()[0]) != int(variant):
                return None
    for line in lines:
        if line.startswith(key + ":"):
            v = (line.split(":", 1)[1].split() or ["null"])[0]
            return None if v == "null" else float(v)
    return None


def pick_sampler(args) -> str:
    if args.sampler != "auto":
        return args.sampler
    return "slice" if args.workload in ("single", "fluct", "batched", "uneven") else "sequential"


class NvmlClocks:
    """SM clock and clock-event (throttle) reasons read through NVML (libnvidia-ml,
    read-only queries) from a thread that polls every 0.2 ms, so that even a
    timed region of a few milliseconds gets samples; one sample is also taken
    right at its start and right at its end."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, cuda_index: int):
        import ctypes
        self.samples, self.reasons = [], set()
        self.max_mhz = None
        self.ok = False
        try:
            self.nvml = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nvml.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            bus = None
            try:
                import torch
                pr = torch.cuda.get_device_properties(cuda_index)
                bus = "%08x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
            except Exception:
                bus = None
            rc = 1
            if bus is not None:
                rc = self.nvml.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(self.h))
            if rc != 0:
                rc = self.nvml.nvmlDeviceGetHandleByIndex_v2(cuda_index, ctypes.byref(self.h))
            if rc != 0:
                return
            mx = ctypes.c_uint(0)
            if self.nvml.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0:  # 1: SM
                self.max_mhz = float(mx.value)
            # the reasons query under its current name, or its older one
            self.why = getattr(self.nvml, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(self.nvml, "nvmlDeviceGetCurrentClocksThrottleReasons", None)
            self.ok = True
        except (OSError, AttributeError):
            self.ok = False

    def sample(self):
        import ctypes
        if not self.ok:
            return
        clk, why = ctypes.c_uint(0), ctypes.c_ulonglong(0)
        if self.nvml.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(clk)) == 0:
            self.samples.append(float(clk.value))
        if self.why is not None and self.why(self.h, ctypes.byref(why)) == 0:
            for bit, name in self.REASONS.items():
                if why.value & bit:
                    self.reasons.add(name)

    def __enter__(self):
        self._stop = threading.Event()
        self.sample()
        self._thread = threading.Thread(target=self._poll, daemon=True)
        self._thread.start()
        return self

    def _poll(self):
        while not self._stop.wait(0.0002):
            self.sample()

    def __exit__(self, *exc):
        self._stop.set()
        self._thread.join()
        self.sample()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": sorted(self.reasons),
                    "samples": 0, "source": "nvml"}
        return {"sm_mhz": statistics.median(self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(self.reasons), "samples": len(self.samples),
                "min_mhz": min(self.samples), "source": "nvml"}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region
    (used when NVML cannot be loaded)."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_workload(name: str, args=None):
    from dataclasses import replace
    wl = workloads.fluct(u=args.u if args is not None else 0.2) if name == "fluct" \
        else workloads.BY_NAME[name]()
    return replace(wl, C=args.C) if args is not None and getattr(args, "C", None) else wl


def sample_workload(wl, nodes: int):
    """A bounded sample of the workload: its first replicas (whole) up to about
    `nodes` nodes, or for a single lattice a periodic window of `nodes` nodes
    with the same density and velocity profile values."""
    from dataclasses import replace
    if wl.replicas == 1:
        m = max(8, min(int(nodes), wl.nodes))
        return replace(wl, L=np.array([m], dtype=np.uint32), rho=wl.rho[:m], u=wl.u[:m])
    cum = np.cumsum(wl.L.astype(np.int64))
    k = int(max(1, np.searchsorted(cum, nodes, side="right")))
    m = int(cum[k - 1])
    return replace(wl, L=wl.L[:k].copy(), rho=wl.rho[:m], u=wl.u[:m])


def oracle_stepper(sampler: str):
    import oracle
    oracle.build()
    return oracle.slice_step if sampler == "slice" else oracle.step


def oracle_rate(wl, seconds: float, sampler: str, threads: int = 0):
    """Time the CPU oracle (as it stands, its node loops on `threads` host cores,
    0 = all) for about `seconds` on a bounded sample of the workload; returns
    (GSUPS, sample description, threads used)."""
    import oracle
    ostep = oracle_stepper(sampler)
    used = oracle.set_threads(threads)
    probe = sample_workload(wl, 1 << 16)
    n, err = oracle.init(probe.L, probe.seed, probe.rho, probe.u)
    for k in range(2):  # the second pass times the oracle with the laws it remembers
        t0 = time.perf_counter()
        ostep(probe.L, probe.seed, n, k, 1, C=probe.C, lam=probe.lam)
        rate = probe.nodes / max(time.perf_counter() - t0, 1e-9)
    sw = sample_workload(wl, min(wl.nodes, max(1 << 14, int(rate * seconds / 4))))
    steps = max(1, int(rate * seconds / sw.nodes))
    n, err = oracle.init(sw.L, sw.seed, sw.rho, sw.u)
    assert err == 0
    t0 = time.perf_counter()
    n, err = ostep(sw.L, sw.seed, n, 0, steps, C=sw.C, lam=sw.lam)
    dt = time.perf_counter() - t0
    oracle.set_threads(0)
    sample = (f"{steps} time step(s) of a {sw.nodes}-node, {sw.replicas}-replica sample of the "
              f"workload (same profile values), {dt:.1f} s on {used} thread(s)")
    return sw.nodes * steps / dt / 1e9, sample, used


def cpu_baseline(wl, seconds: float, sampler: str) -> dict:
    """The oracle on every host core (the baseline) and on one core beside it."""
    v, sample, used = oracle_rate(wl, seconds * 2 / 3, sampler, 0)
    v1, sample1, _ = oracle_rate(wl, seconds / 3, sampler, 1)
    return {"value": v, "unit": "GSUPS", "cores": used, "kind": "oracle", "sample": sample,
            "nproc": os.cpu_count(), "single_thread": {"value": v1, "cores": 1, "sample": sample1}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    wl = make_workload(args.workload, args)
    import oracle
    sampler_name = pick_sampler(args)
    ostep = oracle_stepper(sampler_name)
    cores = oracle.set_threads(0)  # the oracle's node loops on every host core
    # size the per-step sample so that warm-up + timed steps take about two minutes
    probe = sample_workload(wl, 1 << 14)
    n, err = oracle.init(probe.L, probe.seed, probe.rho, probe.u)
    for k in range(2):  # the second pass times the oracle with the laws it remembers
        t0 = time.perf_counter()
        ostep(probe.L, probe.seed, n, k, 1, C=probe.C, lam=probe.lam)
        rate = probe.nodes / max(time.perf_counter() - t0, 1e-9)
    per_step = 120.0 / max(1, args.steps + args.warmup)
    sw = sample_workload(wl, max(8, int(rate * per_step)))  # one 8-node chunk at least
    n, err = oracle.init(sw.L, sw.seed, sw.rho, sw.u)
    assert err == 0
    t = 0
    for _ in range(args.warmup):
        n, err = ostep(sw.L, sw.seed, n, t, 1, C=sw.C, lam=sw.lam)
        t += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        n, err = ostep(sw.L, sw.seed, n, t, 1, C=sw.C, lam=sw.lam)
        t += 1
    dt = time.perf_counter() - t0
    value = sw.nodes * args.steps / dt / 1e9
    sample = (f"each step: one time step of a {sw.nodes}-node, {sw.replicas}-replica sample of "
              f"the workload (same profile values)")
    line = {"impl": "reference", "metric": metric(wl.C), "value": value, "unit": "GSUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak" if wl.replicas == 1 else "strong",
            "vs_baseline": None, "dtype": "u16", "data": "synthetic",
            "config": {**config_dict(wl, args, world), "sampler": sampler_name},
            "cpu_baseline": {"value": value, "unit": "GSUPS", "cores": cores, "kind": "oracle",
                             "sample": sample, "nproc": os.cpu_count()},
            "e2e": {"value": value, "unit": "GSUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(wl, args, world):
    """Workload description; a single lattice is replicated per rank (independent
    lattices), a batch is split over the ranks."""
    single = wl.replicas == 1
    per_gpu = wl.nodes if single else -(-wl.nodes // world)
    return {"workload": f"{wl.name}: {wl.replicas} replica(s), {wl.nodes} nodes, C={wl.C}, "
                        f"lambda={wl.lam[0]}/{wl.lam[1]}",
            "replicas": wl.replicas * (world if single else 1),
            "nodes_per_gpu": per_gpu,
            "global_nodes": wl.nodes * world if single else wl.nodes,
            "C": wl.C, "seed": wl.seed,
            "parallelism": (f"independent lattices x{world}" if single
                            else f"replica batch split over {world} rank(s)"),
            "l2": ("state (12 B/node double-buffered) larger than L2: every launch reads one "
                   "buffer and writes the other, so no flush"
                   if per_gpu * 12 > 129e6 else "state L2-resident")}


GRAPH_STEPS = 32  # steps per CUDA graph the library replays


def graph_launches(steps: int, per_step: int) -> int:
    """Kernels of `steps` steps replayed from 32-step graphs: per_step kernels per
    step, one time-advance kernel per graph and one time-set kernel per call."""
    groups = steps // GRAPH_STEPS
    return steps * per_step + groups + (1 if groups else 0)


# steps per launch of the slice sampler's temporally blocked variants (14 .. 19);
# every other variant takes one step per launch
SLICE_BLOCKED_SPAN = {14: 16, 15: 8, 16: 4, 17: 8, 18: 16, 19: 16}


def blocked_span(tuning, wl, stats_on) -> int:
    if stats_on or wl.replicas != 1:
        return 1
    return SLICE_BLOCKED_SPAN.get(int(tuning.get("plain_variant", 0)), 1)


def count_launches(steps, wl, mode, persistent, stats_on, mclg, slice_sampler=False, span=1):
    """Our kernels launched by one mclg_step(steps) call, as the library issues them."""
    groups = steps // GRAPH_STEPS
    rest = steps - groups * GRAPH_STEPS
    if slice_sampler and stats_on:
        # the statistics form: per step the step kernel and the heavy-node pass;
        # per 32-step graph a merge and a time advance; per call the threshold
        # set, the time set (with graphs), the call's last field's partial pass
        # and the final merge
        return 2 * steps + 2 * groups + (1 if groups else 0) + 3
    if persistent:
        long_replicas = int((((wl.L.astype(np.int64) + 7) // 8) * 8 > 4096).sum())
        # one persistent launch per 65536 steps, plus the long replicas' batched per-step
        # launches (with the slice sampler each followed by its heavy-node pass)
        return -(-steps // 65536) + (graph_launches(steps, 2 if slice_sampler else 1)
                                     if long_replicas else 0)
    if slice_sampler and span > 1:
        # temporally blocked: one kernel per `span` steps (heavy nodes collided in
        # place); per 32-step graph one time-advance kernel, one time-set per call
        return (groups * (GRAPH_STEPS // span) + groups + (1 if groups else 0)
                + -(-rest // span))
    if slice_sampler:
        # per step: the table kernel and the sequential pass over heavy nodes
        if mode == mclg.MODE_PLAIN and wl.replicas > 1 and not stats_on:
            return steps * wl.replicas * 2
        return graph_launches(steps, 2)
    if mode == mclg.MODE_PLAIN and wl.replicas > 1 and not stats_on:
        return steps * wl.replicas  # the per-replica baseline, launched directly
    if stats_on:  # step and partial pass per step, a merge per graph and one per call
        return graph_launches(steps, 2) + groups + 1
    return graph_launches(steps, 1)


def stats_report(lat, wl) -> dict:
    """FP32-vs-FP64 error of the statistics and their Poisson check (Eqs. poisson,
    corr): pooled mean and variance over f^eq of Eq. D1Q3equil."""
    import math
    st = lat.stats_read()
    rho, u = float(wl.rho[0]), float(wl.u[0])
    sq = math.sqrt(1.0 + 3.0 * u * u) - 1.0
    feq = np.array([rho * w * (1 + 3 * v * u + (3 * v * v - 1) * sq)
                    for w, v in ((1 / 6, -1), (2 / 3, 0), (1 / 6, 1))])
    var32 = st["cov32"][:, [0, 3, 5]].astype(np.float64)
    var64 = st["cov64"][:, [0, 3, 5]]
    scale = np.sqrt(var64[:, [0, 0, 1]] * var64[:, [1, 2, 2]])
    cnt = st["count"]
    mean = st["s1"].sum(axis=0) / (float(cnt) * float(wl.L[0]))  # no uint32 product
    return {
        "samples_per_position": cnt,
        "fp32_var_max_rel_err_vs_fp64": float((np.abs(var32 - var64) / var64).max()),
        "fp32_cov_max_err_rel_sqrt_var": float((np.abs(st["cov32"][:, [1, 2, 4]]
                                                       - st["cov64"][:, [1, 2, 4]]) / scale).max()),
        "target_rel_err": 1e-6,
        "mean_over_feq": (mean / feq).tolist(),
        "var_over_feq_pooled": (var64.mean(axis=0) / feq).tolist(),
        "feq": feq.tolist(),
    }


def timed_steps(lat, stream, steps: int) -> float:
    """Milliseconds of one mclg_step(steps) call, CUDA events on the handle's stream."""
    import torch
    lat.sync()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lat.step(steps)
    e1.record(stream)
    e1.synchronize()
    lat.sync()
    return e0.elapsed_time(e1)


BATCHED_SLICE_N_MAX = 512  # the batch's densities reach 500: tables to mass 512 cover nearly all nodes


def batched_extra(mclg, persistent_steps: int = 2000, plain_steps: int = 10) -> dict:
    """The 4096 x 1024 batch (rho ~ U[5, 500], u ~ U[-0.3, 0.3]) with the slice
    sampler (tables to mass 512): one persistent launch for all its steps against
    per-replica launches of the per-step kernel (the baseline, timed on fewer
    steps: it is launch-bound), and the per-step kernel over the whole batch
    (one launch per step, graph replays) beside them."""
    import torch
    wl = workloads.batched()
    out = {"workload": f"batched: {wl.replicas} replicas x {int(wl.L[0])} nodes, C={wl.C}, "
                       "rho ~ U[5,500], u ~ U[-0.3,0.3]", "sampler": "slice",
           "slice_n_max": BATCHED_SLICE_N_MAX}
    stream = torch.cuda.Stream()
    for name, mode, steps in (("persistent", mclg.MODE_PERSISTENT, persistent_steps),
                              ("per_replica_plain", mclg.MODE_PLAIN, plain_steps),
                              ("batched_per_step", mclg.MODE_BATCHED, persistent_steps)):
        with mclg.Lattice(wl.L, seed=wl.seed, C=wl.C, lam=wl.lam, mode=mode, stream=stream,
                          sampler=mclg.SAMPLER_SLICE, slice_n_max=BATCHED_SLICE_N_MAX) as lat:
            lat.init(wl.rho, wl.u)
            tot0 = lat.totals()
            lat.step(2)  # tables, autotuning and warm-up
            ms = timed_steps(lat, stream, steps)
            assert np.array_equal(lat.totals(), tot0), "mass/momentum not conserved"
            out[name] = {"gsups": wl.nodes * steps / (ms / 1e3) / 1e9, "steps": steps,
                         "ms_per_step": ms / steps,
                         "launches_per_step": (1.0 / steps if mode == mclg.MODE_PERSISTENT
                                               else 2 * wl.replicas if mode == mclg.MODE_PLAIN
                                               else 2.0)}
            if mode == mclg.MODE_PERSISTENT:
                out["tuning"] = lat.tuning()
    out["speedup"] = out["persistent"]["gsups"] / out["per_replica_plain"]["gsups"]
    return out


def stats_extra(mclg, burn_in: int = 1000, steps: int = 10_000) -> list:
    """The fluctuation workload (512 x 4096, rho = 50, u in {0, 0.2}): 10^4 steps of
    statistics after 10^3 burn-in, slice sampler; GSUPS and the FP32 error."""
    import torch
    out = []
    stream = torch.cuda.Stream()
    for u in (0.0, 0.2):
        wl = workloads.fluct(u=u)
        with mclg.Lattice(wl.L, seed=wl.seed, C=wl.C, lam=wl.lam, flags=mclg.STATS,
                          sampler=mclg.SAMPLER_SLICE, stream=stream) as lat:
            lat.init(wl.rho, wl.u)
            lat.step(burn_in)
            lat.stats_reset()
            ms = timed_steps(lat, stream, steps)
            rep = stats_report(lat, wl)
        out.append({"u": u, "gsups": wl.nodes * steps / (ms / 1e3) / 1e9, "steps": steps,
                    "burn_in": burn_in, **rep})
    return out


def run_gb300(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_1706_01094_gb300 import build, mclg, sharding
    build.build()
    wl_full = make_workload(args.workload, args)
    stats_on = wl_full.name == "fluct"
    if wl_full.replicas == 1:
        # independent lattices: rank k runs replica k of an N-lattice ensemble
        wl, first = wl_full, rank
    else:
        # a batch: rank k runs its contiguous share of the replicas
        wl, first = sharding.local_workload(wl_full, rank, world)
    mode = {"auto": mclg.MODE_AUTO, "plain": mclg.MODE_PLAIN, "persistent": mclg.MODE_PERSISTENT,
            "batched": mclg.MODE_BATCHED}[args.mode]
    if args.mode == "auto" and wl_full.name == "uneven":
        mode = mclg.MODE_PERSISTENT  # the uneven batch's configuration: the persistent kernel
    stream = torch.cuda.Stream()
    sampler_name = pick_sampler(args)
    sampler = mclg.SAMPLER_SLICE if sampler_name == "slice" else mclg.SAMPLER_SEQUENTIAL
    lat = mclg.Lattice(wl.L, seed=wl.seed, C=wl.C, lam=wl.lam, mode=mode, stream=stream,
                       first_replica=first, flags=mclg.STATS if stats_on else 0,
                       sampler=sampler, kernel_variant=args.kernel_variant,
                       slice_n_max=args.slice_n_max or (
                           BATCHED_SLICE_N_MAX if wl_full.name in ("batched", "uneven") else 0))
    lat.init(wl.rho, wl.u)
    tot0 = lat.totals()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # warm-up (also runs the persistent autotuner when it applies); the
    # statistics workload also burns in before its sums start
    lat.step(args.warmup + (wl.burn_in if stats_on else 0))
    lat.sync()
    if stats_on:
        lat.stats_reset()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = NvmlClocks(local)
    if not clocks.ok:
        clocks = ClockSampler(local)
    with clocks:
        ev0.record(stream)
        persistent = (mode == mclg.MODE_PERSISTENT or (mode == mclg.MODE_AUTO and wl.replicas > 1
                                                       and sampler != mclg.SAMPLER_SLICE)) \
            and not stats_on
        lat.step(args.steps)  # the library loops over the steps (CUDA graphs where it can)
        ev1.record(stream)
        ev1.synchronize()
    lat.sync()
    torch.cuda.synchronize()
    barrier()
    tuning = lat.tuning()
    ms = ev0.elapsed_time(ev1)
    t_max = ms
    if world > 1:
        tt = torch.tensor([ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_max = float(tt.item())
    # correctness guard on the timed run: exact conservation of mass and momentum
    assert np.array_equal(lat.totals(), tot0), "mass/momentum not conserved"
    nodes_all = wl.nodes * world if wl_full.replicas == 1 else wl_full.nodes
    value = nodes_all * args.steps / (t_max / 1e3) / 1e9
    span = blocked_span(tuning, wl, stats_on) if sampler == mclg.SAMPLER_SLICE else 1
    launches = count_launches(args.steps, wl, mode, persistent, stats_on, mclg,
                              sampler == mclg.SAMPLER_SLICE, span)
    stats_summary = stats_report(lat, wl) if stats_on else None

    # end to end through the C ABI with pinned host buffers: every step uploads
    # the state, advances one step and reads the new state back
    host_in = torch.empty((3, wl.nodes), dtype=torch.int16).pin_memory()
    host_out = torch.empty((3, wl.nodes), dtype=torch.int16).pin_memory()
    st, _ = lat.get_state()
    host_in.copy_(torch.from_numpy(st.view(np.int16)))
    e2e_steps = max(1, args.e2e_steps)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tcur = lat.t
    for k in range(e2e_steps):
        lat.set_state(host_in, t=tcur + k)
        lat.step(1)
        lat.get_state(host_out)
    e2e_dt = time.perf_counter() - t0
    e2e_dt_max = e2e_dt
    if world > 1:
        tt = torch.tensor([e2e_dt], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        e2e_dt_max = float(tt.item())
    e2e_value = nodes_all * e2e_steps / e2e_dt_max / 1e9
    lat.close()

    if rank == 0:
        pk = peaks()
        hbm_peak = pk.get("hbm_gbs", 6800.0)
        sm_max = pk.get("sm_max_mhz", 2070.0)
        clk = clocks.summary()
        ms_launch = ms / max(1, launches) if launches else ms
        per_launch_nodes = wl.nodes if args.mode != "plain" or wl.replicas == 1 else None
        sms = sm_count(local)
        alu_peak = INT32_LANES_PER_SM_CLK * sms * sm_max * 1e6 / 1e9  # Gop/s
        achieved_gbs = BYTES_PER_NODE_STEP * wl.nodes * args.steps / (ms / 1e3) / 1e9
        hbm = {"achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
               "frac": achieved_gbs / hbm_peak, "bytes_per_node_step": BYTES_PER_NODE_STEP,
               "peak_basis": "of measured copy bandwidth"}
        if sampler == mclg.SAMPLER_SLICE:
            # a table lookup per node: against the state's HBM traffic of a step
            # (12 B per node-step, the streaming bound of the method); the
            # temporally blocked kernel moves the state through HBM once per
            # launch of `span` steps, so its DRAM traffic per launch (committed
            # profile) is far below the algorithmic bytes of its steps
            # (the persistent form's slice path has no committed profile: its figures stay null)
            kernel = ("k_step_persistent_slice" if persistent else
                      "k_step_slice_tb" if span > 1 else "k_step_slice")
            # (the blocked kernel's summary holds for the launch variant it captured)
            pv = tuning.get("plain_variant")
            roofline = {"bound": "hbm", **hbm,
                        "traffic": committed_figure(kernel, wl.name, variant=pv),
                        "kernel": kernel, "launch_variant": pv, "steps_per_launch": span,
                        "algorithmic_bytes_per_launch": BYTES_PER_NODE_STEP * wl.nodes * span,
                        "alu_pipe_pct_ncu": committed_figure(kernel, wl.name, "alu_pipe_pct",
                                                             variant=pv),
                        "issue_active_pct_ncu": committed_figure(kernel, wl.name,
                                                                 "issue_active_pct", variant=pv),
                        "time_basis": ("whole step: temporally blocked launches of "
                                       f"{span} steps, heavy nodes collided in place"
                                       if span > 1 else
                                       "whole step (table kernel + heavy-node pass) per step")}
        else:
            # integer-bound: the fraction is ncu's ALU-pipe utilisation of the kernel on
            # this workload (committed profile); the hand tally of integer operations
            # against the unit-count peak is kept beside it
            achieved_ops = int_ops_per_node_step(wl.C) * wl.nodes * args.steps / (ms / 1e3) / 1e9
            kernel = ("k_step_plain" if (wl.replicas == 1 or args.mode in ("plain", "batched"))
                      else "k_step_persistent")
            alu_pct = committed_figure(kernel, wl.name, "alu_pipe_pct")
            roofline = {"bound": "alu", "achieved": alu_pct, "peak": 100.0,
                        "unit": "% of ALU-pipe issue (ncu sm__inst_executed_pipe_alu)",
                        "frac": None if alu_pct is None else alu_pct / 100.0,
                        "issue_active_pct_ncu": committed_figure(kernel, wl.name,
                                                                 "issue_active_pct"),
                        "traffic": committed_figure(kernel, wl.name), "kernel": kernel,
                        "op_tally": {"ops_per_node_step": int_ops_per_node_step(wl.C),
                                     "achieved_gops": achieved_ops, "peak_gops": alu_peak,
                                     "frac": achieved_ops / alu_peak,
                                     "peak_basis": (f"{INT32_LANES_PER_SM_CLK} int32 lanes x "
                                                    f"{sms} SMs (device attribute) x "
                                                    f"{sm_max:.0f} MHz")},
                        "hbm": hbm}
        line = {
            "metric": metric(wl.C), "value": value, "unit": "GSUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True,
            "scaling": "weak" if wl_full.replicas == 1 else "strong",
            "vs_baseline": None, "dtype": "u16",
            "data": "synthetic: Poisson(f^eq) initial state of the paper-shaped workload",
            "config": {**config_dict(wl_full, args, world), "sampler": sampler_name,
                       "tuning": tuning},
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": "GSUPS",
                    "h2d_bytes_per_step": 6 * wl.nodes, "d2h_bytes_per_step": 6 * wl.nodes,
                    "steps": e2e_steps,
                    "path": "mclg_set_state(pinned host) + mclg_step(1) + mclg_get_state(pinned host)"},
            "gpu_launches": launches,
            **({"stats": stats_summary} if stats_summary else {}),
            "ms_per_launch": ms_launch,
            "clocks": clk,
        }
        line["config"]["sms"] = sms
        if world == 1 and args.workload == "single" and not args.no_extras:
            line["batched"] = batched_extra(mclg)
            line["stats"] = stats_extra(mclg)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds, sampler_name)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# D2Q9 workload (Sec. II.B, III.B): one 4096 x 4096 periodic lattice at rho = 36, u = 0, with
# Poisson(f^eq) occupations, C = 10 and the paper's rates; 9 x uint16 read and written per node-step
D2Q9_SIDE = 4096
D2Q9_RHO = 36.0
D2Q9_BYTES_PER_NODE_STEP = 36


def d2q9_metric() -> str:
    return "D2Q9 site updates per second (10^9, C = 10 particle-pick sub-collisions per node)"


def d2q9_oracle_rate(seconds: float, threads: int = 0) -> tuple:
    """The oracle's D2Q9 steps on a square lattice sized for about `seconds` of host
    time; returns (GSUPS, nodes, steps, elapsed, threads)."""
    import oracle
    oracle.build()
    oracle.set_threads(threads)
    used = oracle.threads()
    side = 128
    while True:
        S = side * side
        n0, err = oracle.d2q9_init(side, side, 1, 1, np.full(S, D2Q9_RHO), np.zeros(S), np.zeros(S))
        t0 = time.perf_counter()
        n, err = oracle.d2q9_step(side, side, 1, 1, n0, 0, 2)
        dt = time.perf_counter() - t0
        if dt > seconds / 8 or side >= 2048:
            break
        side *= 2
    steps = max(2, int(2 * seconds / max(dt, 1e-3)))
    t0 = time.perf_counter()
    n, err = oracle.d2q9_step(side, side, 1, 1, n0, 0, steps)
    dt = time.perf_counter() - t0
    return side * side * steps / dt / 1e9, side * side, steps, dt, used


def run_d2q9(args, reference: bool = False):
    """The D2Q9 line: the GPU kernel (or, with reference, the CPU oracle) on the
    4096^2 lattice; the same JSON keys as the D1Q3 line."""
    if reference:
        gs, nodes, steps, dt, used = d2q9_oracle_rate(args.cpu_seconds)
        print(json.dumps({"impl": "reference", "metric": d2q9_metric(), "value": gs, "unit": "GSUPS",
                          "n_gpus": 0, "steps": steps, "warmup": 0,
                          "ms_per_step": dt / steps * 1e3, "higher_is_better": True,
                          "vs_baseline": None, "dtype": "u16", "data": "synthetic",
                          "config": {"workload": f"d2q9: {int(nodes ** 0.5)}^2 sample of the "
                                                 f"{D2Q9_SIDE}^2 lattice, rho = {D2Q9_RHO}, u = 0"},
                          "cpu_baseline": {"value": gs, "unit": "GSUPS", "cores": used,
                                           "kind": "oracle",
                                           "sample": f"{steps} steps of a {nodes}-node square lattice"},
                          "e2e": {"value": gs, "unit": "GSUPS", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    from paper_1706_01094_gb300 import build, mclg
    build.build()
    side, S = D2Q9_SIDE, D2Q9_SIDE * D2Q9_SIDE
    stream = torch.cuda.Stream()
    lat = mclg.Lattice2D(side, side, 1, seed=1 + rank, C=10, lam=mclg.D2Q9_PAPER_LAMBDA,
                         stream=stream)
    lat.init(np.full(S, D2Q9_RHO), np.zeros(S), np.zeros(S))
    tot0 = lat.moments()
    lat.step(args.warmup)
    lat.sync()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = NvmlClocks(local)
    if not clocks.ok:
        clocks = ClockSampler(local)
    with clocks:
        ev0.record(stream)
        lat.step(args.steps)  # one kernel per step
        ev1.record(stream)
        ev1.synchronize()
    lat.sync()
    ms = ev0.elapsed_time(ev1)
    tot1 = lat.moments()
    assert np.array_equal(tot0, tot1), "mass/momentum not conserved"
    value = S * args.steps / (ms / 1e3) / 1e9
    # end to end through the C ABI with pinned host buffers
    host_in = torch.empty((9, S), dtype=torch.int16).pin_memory()
    host_out = torch.empty((9, S), dtype=torch.int16).pin_memory()
    st, tcur = lat.get_state()
    host_in.copy_(torch.from_numpy(st.view(np.int16)))
    e2e_steps = max(1, args.e2e_steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        lat.set_state(host_in, t=tcur + k)
        lat.step(1)
        lat.get_state(host_out)
    e2e = S * e2e_steps / (time.perf_counter() - t0) / 1e9
    lat.close()
    if rank != 0:
        return
    pk = peaks()
    hbm_gbs = D2Q9_BYTES_PER_NODE_STEP * S * args.steps / (ms / 1e3) / 1e9
    alu_pct = committed_figure("k_step_d2q9", "d2q9", "alu_pipe_pct")
    line = {"metric": d2q9_metric(), "value": value, "unit": "GSUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16",
            "data": "synthetic: Poisson(f^eq) initial state, rho = 36, u = 0",
            "config": {"workload": f"d2q9: {side} x {side} periodic lattice, rho = {D2Q9_RHO}, "
                                   "u = 0, C = 10, the paper's rates (Sec. IV.B)",
                       "l2": "state (36 B/node double-buffered, 1.2 GB) larger than L2; no flush",
                       "sms": sm_count(local)},
            "roofline": {"bound": "alu", "achieved": alu_pct, "peak": 100.0,
                         "unit": "% of ALU-pipe issue (ncu sm__inst_executed_pipe_alu)",
                         "frac": None if alu_pct is None else alu_pct / 100.0,
                         "kernel": "k_step_d2q9",
                         "issue_active_pct_ncu": committed_figure("k_step_d2q9", "d2q9",
                                                                  "issue_active_pct"),
                         "traffic": committed_figure("k_step_d2q9", "d2q9"),
                         "hbm_equivalent": {"achieved": hbm_gbs, "peak": pk.get("hbm_gbs", 6800.0),
                                            "unit": "GB/s",
                                            "frac": hbm_gbs / pk.get("hbm_gbs", 6800.0),
                                            "bytes_per_node_step": D2Q9_BYTES_PER_NODE_STEP}},
            "e2e": {"value": e2e, "unit": "GSUPS", "h2d_bytes_per_step": 18 * S,
                    "d2h_bytes_per_step": 18 * S, "steps": e2e_steps,
                    "path": "mclg2d_set_state(pinned host) + mclg2d_step(1) + "
                            "mclg2d_get_state(pinned host)"},
            "gpu_launches": args.steps,
            "clocks": clocks.summary()}
    if not args.no_cpu_baseline:
        gs, nodes, steps, dt, used = d2q9_oracle_rate(args.cpu_seconds)
        line["cpu_baseline"] = {"value": gs, "unit": "GSUPS", "cores": used, "kind": "oracle",
                                "sample": f"{steps} steps of a {nodes}-node square lattice, "
                                          f"{dt:.1f} s on {used} thread(s)"}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload == "d2q9":
        run_d2q9(args, reference=args.impl == "reference")
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
