#!/usr/bin/env python3
"""Benchmark of the LCO contraction hot path on one GB300 per rank.

Workload (the metric's configuration): the 3D 7-point Dirichlet Laplacian on
a 64^3 grid (6th-order tensor, 1,810,432 non-zeros) composed with a seeded
U(-1,1) first derivative in x (Eq. 1 pattern, 532,480 non-zeros), followed by
the stand-alone radix permutation of the product (3,382,784 non-zeros) to
mode order (k,l,m,i,j,n).  One step = the whole path: re-linearise/permute
operands when needed, build B's CSR, scan the work, multiply (Table-4 branch:
CSR), then permute C.  Inputs are synthetic (seeded generators in synth/).

Timing: W warm-up steps, then K steps replayed from a CUDA graph, each
bracketed by CUDA events on the launching stream, with L2 flushed (a 256 MiB
memset) before every step, outside the events.  value = (nnz_A + nnz_B +
nnz_C) / mean step time, summed over ranks (replicas: each rank runs its own
copy, no collective in the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lco|reference]
"""
from __future__ import annotations

import argparse
import gc
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

# The batch and the server run work on 16 and 64 streams; by default CUDA
# maps all streams of a process onto 8 hardware work queues, so kernels of
# unrelated streams wait on each other.  32 queues (read when the CUDA
# context is created, so before torch touches the GPU) let them overlap.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import numpy as np  # noqa: E402

METRIC = "contraction GNNZ/s"
UNIT = "GNNZ/s"
WORKLOAD = "fd3d_laplacian7_64^3_x_dx_uniform + permute_to_klmijn"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "roofline_traffic.md")
KERNEL_SOURCES = {
    "k_rows": "paper_1802_02619_gb300/csrc/lco_contract.cu",
    "k_heavy": "paper_1802_02619_gb300/csrc/lco_contract.cu",
    "k_row_table": "paper_1802_02619_gb300/csrc/lco_contract.cu",
    "k_row_heavy": "paper_1802_02619_gb300/csrc/lco_contract.cu",
    "k_copy_rows": "paper_1802_02619_gb300/csrc/lco_contract.cu",
    "k_dcsr_build": "paper_1802_02619_gb300/csrc/lco_contract.cu",
    "k_work_scan": "paper_1802_02619_gb300/csrc/lco_contract.cu",
    "k_csr_rowptr": "paper_1802_02619_gb300/csrc/lco_contract.cu",
    "k_radix_scatter": "paper_1802_02619_gb300/csrc/lco_radix.cu",
    "k_radix_upsweep": "paper_1802_02619_gb300/csrc/lco_radix.cu",
    "k_radix_local": "paper_1802_02619_gb300/csrc/lco_radix.cu",
    "k_compact": "paper_1802_02619_gb300/csrc/lco_contract.cu",
    "k_entry_lookup": "paper_1802_02619_gb300/csrc/lco_contract.cu",
}
# headers every kernel source includes: a change there changes the kernels too
KERNEL_HEADERS = ["paper_1802_02619_gb300/csrc/lco_internal.cuh", "paper_1802_02619_gb300/csrc/lco_radix.cuh"]


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["lco", "reference"], default="lco")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--soak-s", type=float, default=1.5,
                    help="seconds of clock-sampled graph replays before the timed region (0 = none, e.g. under ncu)")
    ap.add_argument("--no-extras", action="store_true",
                    help="--case step: skip the C3, C3b, batch and serve measurements after the headline")
    ap.add_argument("--case", choices=["step", "permute", "batch", "serve", "permsweep", "permute_wide"],
                    default="step",
                    help="step: the benchmark workload; permute: a stand-alone radix permutation "
                         "of a random 6th-order 64^6 tensor (profiling aid); batch / serve: C4 / C5; "
                         "permsweep: the Eq. 4 operator into all 23 other orders; permute_wide: a "
                         "wide-LIV (128-bit) permutation")
    ap.add_argument("--nnz", type=int, default=16 << 20, help="non-zeros for --case permute / permute_wide")
    ap.add_argument("--config", choices=sorted(CONFIGS), default="C2",
                    help="--case step: C1 fd2d 16^2 L^2, C2 fd3d 64^3 L.Dx + permute (the metric's), "
                         "C3 R-MAT 1e7 DCSR, C3b R-MAT 2^18 CSRNA, E17 the Sec. 6 product at N = 2047")
    ap.add_argument("--count", type=int, default=4096, help="problems for --case batch")
    ap.add_argument("--max-digit-bits", type=int, default=0,
                    help="cap on the radix digit width of the operand permutations (0: library default)")
    ap.add_argument("--streams", type=int, default=16, help="stream pool for --case batch")
    ap.add_argument("--per-kind", action="store_true", help="--case batch: also time each kind alone")
    ap.add_argument("--tune", action="store_true", help="--case batch: also run the autotuned batch")
    ap.add_argument("--requests", type=int, default=10000, help="--case serve: requests per run")
    ap.add_argument("--N", type=int, default=2895, help="--case permsweep: image side of the Eq. 4 operator")
    ap.add_argument("--slots", type=int, default=64, help="--case serve: requests in flight")
    ap.add_argument("--workers", type=int, default=8, help="--case serve: host worker threads")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only; NCCL is used for the barrier and the
# max-over-ranks timing, never in the data path)
# ---------------------------------------------------------------------------

def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(x, world):
    """Maximum of x over the ranks (NCCL on GPUs, gloo on the CPU)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, flag in zip(names, parts[5:9]):
                if flag.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline helpers
# ---------------------------------------------------------------------------

def measured_peak_hbm():
    try:
        with open(PEAKS_FILE) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def source_digest(kernel):
    """sha256 (16 hex digits) of the kernel's source file and the shared
    device headers, in that order."""
    if kernel not in KERNEL_SOURCES:
        return None
    h = hashlib.sha256()
    try:
        for rel in [KERNEL_SOURCES[kernel]] + KERNEL_HEADERS:
            with open(os.path.join(ROOT, rel), "rb") as fh:
                h.update(fh.read())
    except OSError:
        return None
    return h.hexdigest()[:16]


def profiled_traffic(kernel, config="C2"):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of the kernel (matching digest) and on this
    configuration (the summary covers C2 only); else None."""
    if config != "C2":
        return None
    try:
        text = open(PROFILE_SUMMARY).read()
    except OSError:
        return None
    for line in text.splitlines():
        m = re.match(r"\|\s*(k_\w+)\s*\|\s*([0-9a-f]{16})\s*\|\s*([0-9.eE+]+)\s*\|", line)
        if m and m.group(1) == kernel:
            if m.group(2) != source_digest(kernel):
                return None
            return float(m.group(3))
    return None


# ---------------------------------------------------------------------------
# the step
# ---------------------------------------------------------------------------

CONFIGS = {
    # name: (synth constructor, workload label)
    "C1": ("config_fd2d", "fd2d_laplacian5_16^2_squared"),
    "C2": ("config_fd3d", WORKLOAD),
    "C3": ("config_rmat_dcsr", "rmat_2^20x2^20x2^12_1e7_each_a_ijk_b_ljk"),
    "C3b": ("config_rmat_na", "rmat_2^14x2^14x2^12_2^18_each_mode2_x_mode0"),
    "E17": ("config_eq17", "eq17_b_ii'jl_d_i'k_N2047 (Sec. 6; paper: 2.0 s on an E8400)"),
}


def c_dims_of(cfg):
    """Dims of the product: A's free modes in order, then B's."""
    A, B = cfg["A"], cfg["B"]
    fa = [d for t, d in enumerate(A["dims"]) if t not in cfg["modes_a"]]
    fb = [d for t, d in enumerate(B["dims"]) if t not in cfg["modes_b"]]
    return fa + fb


class ConfigStep:
    """One pass of the hot path on a configuration: contract (with whatever
    operand permutations and conversions its plan needs) and, when the
    configuration asks for it, permute the product."""

    def __init__(self, cfg, device, max_digit_bits=0):
        import torch
        import paper_1802_02619_gb300 as lco
        self.torch, self.lco = torch, lco
        self.cfg = cfg
        self.A = lco.LcoTensor.from_host(cfg["A"], device)
        self.B = lco.LcoTensor.from_host(cfg["B"], device)
        self.plan = lco.ContractPlan(self.A.dims, self.A.sig, self.A.nnz, self.B.dims, self.B.sig, self.B.nnz,
                                     cfg["modes_a"], cfg["modes_b"], max_digit_bits=max_digit_bits)
        # first run sizes the output by the product count f
        self.plan.ensure_workspace(0, device)
        self.plan.symbolic(self.A, self.B)
        r = self.plan.result()
        assert r["status"] == 0, r
        self.f = r["f"]
        self.plan.ensure_workspace(self.f, device)
        self.c_liv = torch.empty(max(self.f, 1), dtype=torch.int64, device=device)
        self.c_val = torch.empty(max(self.f, 1), dtype=torch.float64, device=device)
        self.plan.run(self.A, self.B, self.c_liv, self.c_val)
        r = self.plan.result()
        assert r["status"] == 0, r
        self.nnz_c = r["nnz_c"]
        self.nzr_b = r["nzr_b"]
        self.alg = r["alg"]
        self.perm = None
        if "permute_sig" in cfg:
            self.perm = lco.Permuter(self.plan.c_dims, self.plan.c_sig, cfg["permute_sig"], self.nnz_c, device)
            self.p_liv = torch.empty(self.nnz_c, dtype=torch.int64, device=device)
            self.p_val = torch.empty(self.nnz_c, dtype=torch.float64, device=device)
        self.out_liv = self.p_liv if self.perm else self.c_liv[:self.nnz_c]
        self.out_val = self.p_val if self.perm else self.c_val[:self.nnz_c]
        self.units = self.A.nnz + self.B.nnz + self.nnz_c
        # tensors the radix engine permutes in one step
        info = self.plan.info
        self.permuted = ([self.A.nnz] if info["permute_a"] else []) + \
            ([self.B.nnz] if info["permute_b"] else []) + ([self.nnz_c] if self.perm else [])

    def contract(self):
        self.plan.run(self.A, self.B, self.c_liv, self.c_val)

    def permute(self):
        if self.perm:
            self.perm(self.c_liv[:self.nnz_c], self.c_val[:self.nnz_c], self.p_liv, self.p_val)

    def __call__(self):
        self.contract()
        self.permute()


def load_config(name):
    import synth
    ctor, label = CONFIGS[name]
    cfg = getattr(synth, ctor)()
    return cfg, label


def measure_config(name, device, K, warmup, world=1, local=0, max_digit_bits=0, soak_s=0.0):
    """Device timing of one configuration's step: the step captured in a CUDA
    graph, K replays each bracketed by events with L2 flushed before it, then
    a per-kernel timing pass (direct launches, L2 flushed) and a warm-L2
    replay.  With soak_s > 0 the graph is first replayed for that long under
    the clock sampler, so that the clock record covers a loaded GPU.  Returns
    (record, step)."""
    import torch
    import paper_1802_02619_gb300 as lco
    lib = lco.load()
    cfg, workload = load_config(name)
    step = ConfigStep(cfg, device, max_digit_bits)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)

    # sanity: the output is strictly ascending
    step()
    torch.cuda.synchronize()
    assert bool((step.out_liv[1:] > step.out_liv[:-1]).all()), "output LIVs not ascending"

    # ---- warm-up and graph capture ----
    for _ in range(max(warmup, 3)):
        step()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        step()                       # warm the side stream
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=side):
            step()
    stream.wait_stream(side)
    for _ in range(warmup):
        flush.zero_()
        graph.replay()
    torch.cuda.synchronize()

    # ---- clock soak and timed region ----
    clocks = ClockSampler(local) if soak_s > 0 else None
    soak = None
    if clocks:
        clocks.start()
        t0 = time.perf_counter()
        nsoak = 0
        while time.perf_counter() - t0 < soak_s:
            for _ in range(64):
                flush.zero_()
                graph.replay()
            nsoak += 64
            torch.cuda.synchronize()
        soak = {"s": round(time.perf_counter() - t0, 3), "steps": nsoak}
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(K):
        flush.zero_()
        evs[i][0].record(stream)
        graph.replay()
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - t0
    clk = clocks.stop() if clocks else None
    if clk is not None:
        clk["soak"] = soak
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    step_sorted = sorted(step_ms)
    total_ms_max = reduce_max(total_ms, world)
    ms_per_step = total_ms_max / K
    value = world * step.units * K / (total_ms_max * 1e-3) / 1e9

    # ---- per-kernel timing pass (same step, launched directly, L2 flushed) ----
    n_prof = min(K, 50)
    lib.lco_timing_enable(1)
    phase_c, phase_p = [], []
    for _ in range(n_prof):
        flush.zero_()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        step.contract()
        e1.record(stream)
        step.permute()
        e2.record(stream)
        torch.cuda.synchronize()
        phase_c.append(e0.elapsed_time(e1))
        phase_p.append(e1.elapsed_time(e2))
    # ---- warm-L2 variant (reported beside the cold number): the same graph
    # replayed back to back without the flush ----
    n_warm = min(K, 200)
    wev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_warm)]
    for i in range(n_warm):
        wev[i][0].record(stream)
        graph.replay()
        wev[i][1].record(stream)
    torch.cuda.synchronize()
    warm_ms = statistics.median([a.elapsed_time(b) for a, b in wev])
    recs = (lco.TimingRecord * 4096)()
    import ctypes
    cnt = ctypes.c_int32()
    lib.lco_timing_read(recs, 4096, ctypes.byref(cnt))
    lib.lco_timing_enable(0)
    per = {}
    for i in range(cnt.value):
        nm = recs[i].name.decode()
        per.setdefault(nm, []).append(recs[i].ms)
    launches_per_step = cnt.value / n_prof
    # A kernel may be launched for work that the device then finds it need
    # not do (a radix pass whose digit is constant, the scatter pass that a
    # high-digit-first sort leaves out): such launches return at once.  A
    # kernel's launches within a step that take under a quarter of its
    # longest one in that step are counted as such and left out of its
    # per-launch time (the step time keeps them).
    per_step = len(recs[:cnt.value]) // max(n_prof, 1)
    work = {}
    for st in range(n_prof):
        by = {}
        for i in range(st * per_step, (st + 1) * per_step):
            by.setdefault(recs[i].name.decode(), []).append(recs[i].ms)
        for nm, v in by.items():
            mx = max(v)
            work.setdefault(nm, []).extend(x for x in v if x >= 0.25 * mx)
    kern_total = sum(sum(v) for v in per.values())
    kernels = {nm: {"launches_per_step": len(v) / n_prof, "avg_ms": sum(v) / len(v),
                    "work_launches_per_step": len(work.get(nm, v)) / n_prof,
                    "work_avg_ms": sum(work.get(nm, v)) / max(len(work.get(nm, v)), 1),
                    "share": sum(v) / kern_total if kern_total else 0.0} for nm, v in per.items()}
    dominant = max(per, key=lambda nm: sum(per[nm]))
    peak, peak_kind = measured_peak_hbm()
    alg_bytes = algorithmic_bytes(dominant, step)
    avg_s = kernels[dominant]["work_avg_ms"] * 1e-3
    achieved = alg_bytes / avg_s / 1e9 if avg_s > 0 else 0.0
    traffic = profiled_traffic(dominant, name)
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": round(achieved, 1), "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": traffic, "algorithmic_bytes": alg_bytes}
    del graph
    rec = {
        "value": round(value, 4), "ms_per_step": round(ms_per_step, 5), "steps": K,
        "config": {"workload": workload, "name": name, "nnz_a": step.A.nnz, "nnz_b": step.B.nnz,
                   "nnz_c": step.nnz_c, "f": step.f, "alg": step.alg, "permuted_keys": step.permuted,
                   "l2": "flushed before every step (256 MiB memset, outside the step events)",
                   "graph": "each step replayed from one CUDA graph", "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "gpu_launches": int(round(launches_per_step * K)),
        "clocks": clk,
        "warm_l2": {"ms_per_step": round(warm_ms, 5), "value": round(step.units / (warm_ms * 1e-3) / 1e9, 4),
                    "steps": n_warm, "note": "median step of the same graph replayed back to back, no L2 flush"},
        "latency_ms": {"p50": round(step_sorted[len(step_sorted) // 2], 5),
                       "p99": round(step_sorted[min(len(step_sorted) - 1, int(0.99 * len(step_sorted)))], 5)},
        "breakdown": {"contract_ms": round(statistics.median(phase_c), 5),
                      "permute_ms": round(statistics.median(phase_p), 5),
                      "contract_gnnz_s": round(step.units / (statistics.median(phase_c) * 1e-3) / 1e9, 3),
                      "permute_gkeys_s": (round(step.nnz_c / (statistics.median(phase_p) * 1e-3) / 1e9, 3)
                                          if step.perm else None),
                      "kernels": {k: {kk: round(vv, 5) for kk, vv in v.items()} for k, v in kernels.items()},
                      "wall_s_timed_region": round(wall, 4)},
    }
    return rec, step, cfg


def run_lco(args):
    import torch
    rank, world, local = dist_setup()
    device = f"cuda:{local}"
    # the clock record covers at least 1.5 s of replays just before the timed region
    rec, step, cfg = measure_config(args.config, device, args.steps, args.warmup, world, local,
                                    args.max_digit_bits, soak_s=args.soak_s)
    out = {"metric": METRIC, "value": rec["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic"}
    out.update({k: v for k, v in rec.items() if k not in ("value", "ms_per_step", "steps")})
    if not args.no_e2e:
        out["e2e"] = run_e2e(step, device, min(args.steps, 200), world)
    del step
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(cfg, budget_s=12.0)
    del cfg
    if rank == 0 and world == 1 and not args.no_extras:
        out["extras"] = run_extras(args, device)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_extras(args, device):
    """The other configurations, measured in the same run on the same GPU:
    C3 (R-MAT 1e7 per operand, DCSR) and C3b (R-MAT 2^18, CSRNA) as device-
    timed steps with their dominant kernel's roofline and the oracle beside
    them; C4 (the 4096-problem batch) and C5 (served requests) against their
    plain per-call paths.  Each is skipped with its error recorded rather
    than failing the headline line."""
    import torch
    extras = {}
    K = max(3, min(args.steps, 20))
    for name in ("C3", "C3b"):
        try:
            rec, step, cfg = measure_config(name, device, K, max(args.warmup, 3), max_digit_bits=args.max_digit_bits)
            del step
            torch.cuda.empty_cache()
            if not args.no_cpu_baseline:
                rec["cpu_baseline"] = cpu_baseline(cfg, budget_s=6.0, all_cores=False)
            extras[name] = rec
        except Exception as e:    # recorded, not fatal for the headline
            extras[name] = {"error": repr(e)[:300]}
        torch.cuda.empty_cache()
    try:
        extras["batch"] = measure_batch(args.count, K, max(args.warmup, 3), args.streams,
                                        cpu_budget_s=0.0 if args.no_cpu_baseline else 6.0)
    except Exception as e:
        extras["batch"] = {"error": repr(e)[:300]}
    torch.cuda.empty_cache()
    try:
        extras["serve"] = measure_serve(min(args.requests, 4000), args.slots, args.workers)
    except Exception as e:
        extras["serve"] = {"error": repr(e)[:300]}
    torch.cuda.empty_cache()
    return extras


def algorithmic_bytes(kernel, step):
    """Bytes the method must move per launch of `kernel` (lower bound).
    Radix kernels are charged per element of the tensor they permute (the
    mean over the step's permuted tensors, exact when there is one)."""
    nA, nB, nC = step.A.nnz, step.B.nnz, step.nnz_c
    nperm = statistics.mean(step.permuted) if step.permuted else 0
    if kernel == "k_rows":
        return 16 * (nA + nB + nC)            # read L and R once, write C
    if kernel in ("k_row_table", "k_row_heavy"):
        return 8 * nA                         # row work offsets (upper bound: one row per entry)
    if kernel in ("k_radix_scatter", "k_radix_local"):
        return int(32 * nperm)                # read key+value, write key+value
    if kernel == "k_radix_upsweep":
        return int(8 * nperm)                 # read keys
    if kernel == "k_work_scan":
        return 16 * nA                        # read L's LIVs, write the work prefix
    if kernel == "k_csr_rowptr":
        return 8 * nB + 8 * (step.plan.info["k"] + 1)
    if kernel == "k_dcsr_build":
        return 8 * nB + 16 * step.nzr_b       # read R's LIVs, write row ids and pointers
    return 0


def run_e2e(step, device, K, world):
    """Same metric through the public API with host buffers: every step copies
    A and B in from pinned host memory, contracts, permutes and copies the
    permuted product back to pinned host memory, all inside the timed region.
    Steps are pipelined as a user streaming contractions would run them: the
    inputs of step i+1 go in and the result of step i-1 comes out while step i
    computes (copy-in, compute and copy-out streams; two sets of device input
    and output buffers, two pinned result buffers).  Each buffer set's compute
    -- the same public calls, plan.run and the permutation -- is captured
    once into a CUDA graph and replayed, so that the host enqueues one graph
    per step instead of a dozen library calls."""
    import torch
    import paper_1802_02619_gb300 as lco
    ins_d = [(step.A.liv, step.A.val, step.B.liv, step.B.val)]
    ins_d.append(tuple(torch.empty_like(t) for t in ins_d[0]))
    ins_h = [t.cpu().pin_memory() for t in ins_d[0]]
    outs_d = [(step.out_liv, step.out_val), (torch.empty_like(step.out_liv), torch.empty_like(step.out_val))]
    outs_h = [(torch.empty(step.nnz_c, dtype=torch.int64).pin_memory(),
               torch.empty(step.nnz_c, dtype=torch.float64).pin_memory()) for _ in range(2)]
    tens = [(lco.LcoTensor(step.A.dims, step.A.sig, a_l, a_v), lco.LcoTensor(step.B.dims, step.B.sig, b_l, b_v))
            for a_l, a_v, b_l, b_v in ins_d]
    h2d = sum(t.numel() * t.element_size() for t in ins_h)
    d2h = step.nnz_c * 16
    s_in, s_c, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()

    def compute(b):
        A, B = tens[b]
        step.plan.run(A, B, step.c_liv, step.c_val)
        if step.perm:
            step.perm(step.c_liv[:step.nnz_c], step.c_val[:step.nnz_c], outs_d[b][0], outs_d[b][1])

    graphs = []
    for b in range(2):
        with torch.cuda.stream(s_c):
            compute(b)                       # warm (allocations, attributes) outside capture
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s_c):
            compute(b)
        graphs.append(g)
    torch.cuda.synchronize()

    def run(n):
        ev_c = [None] * n
        ev_out = [None] * n
        for i in range(n):
            b = i % 2
            # copy-in: the buffer set was last read by step i - 2
            if i >= 2:
                s_in.wait_event(ev_c[i - 2])
            with torch.cuda.stream(s_in):
                for h, d in zip(ins_h, ins_d[b]):
                    d.copy_(h, non_blocking=True)
            ev_in = torch.cuda.Event()
            ev_in.record(s_in)
            # compute: its outputs were last read by step i - 2's copy-out (by
            # step i - 1's when the result is the contraction buffer itself)
            s_c.wait_event(ev_in)
            if step.perm and i >= 2:
                s_c.wait_event(ev_out[i - 2])
            elif not step.perm and i >= 1:
                s_c.wait_event(ev_out[i - 1])
            with torch.cuda.stream(s_c):
                graphs[b].replay()
            ev_c[i] = torch.cuda.Event()
            ev_c[i].record(s_c)
            # copy-out of the step's result
            s_out.wait_event(ev_c[i])
            with torch.cuda.stream(s_out):
                src_l, src_v = outs_d[b] if step.perm else (step.c_liv[:step.nnz_c], step.c_val[:step.nnz_c])
                outs_h[b][0].copy_(src_l, non_blocking=True)
                outs_h[b][1].copy_(src_v, non_blocking=True)
            ev_out[i] = torch.cuda.Event()
            ev_out[i].record(s_out)
        torch.cuda.synchronize()

    run(4)
    barrier(world)
    t0 = time.perf_counter()
    run(K)
    dt = time.perf_counter() - t0
    dt = reduce_max(dt, world)
    # the last result read back equals the device-timed step's output
    last = outs_h[(K - 1) % 2]
    assert torch.equal(last[0], step.out_liv.cpu()), "e2e result LIVs differ"
    assert torch.equal(last[1].view(torch.int64), step.out_val.cpu().view(torch.int64)), "e2e result values differ"
    return {"value": round(world * step.units * K / dt / 1e9, 4), "unit": UNIT, "steps": K,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": round(dt / K * 1e3, 4),
            "pipelined": "copy-in of step i+1 and copy-out of step i-1 overlap step i's compute",
            "compute": "each buffer set's public calls (plan.run, permutation) replayed from a CUDA graph"}


def _rows_sample(A, frac):
    """The leading rows of A (A is stored with its row modes most
    significant, so a prefix of its index space is a set of leading rows)."""
    if frac >= 1.0:
        return A
    total = int(np.prod(np.asarray(A["dims"], dtype=np.float64)))
    keep = A["liv"] < int(frac * total)
    return {"dims": A["dims"], "sig": A["sig"], "liv": A["liv"][keep], "val": A["val"][keep]}


def _oracle_step(cfg):
    """One step of the oracle (contraction, then the product's permutation
    when the configuration has one) on a given A; returns (seconds, units)."""
    import oracle
    B = cfg["B"]

    def one(As):
        t0 = time.perf_counter()
        liv, val, _ = oracle.contract(As, B, cfg["modes_a"], cfg["modes_b"])
        if "permute_sig" in cfg:
            cd = c_dims_of(cfg)
            oracle.permute(cd, list(range(len(cd) - 1, -1, -1)), cfg["permute_sig"], liv, val)
        return time.perf_counter() - t0, len(As["liv"]) + len(B["liv"]) + len(liv)
    return one


def cpu_baseline(cfg, budget_s=12.0, all_cores=True):
    """The oracle as it stands (single-threaded C) on this host, on a
    bounded sample of the workload: whole steps when one takes at most a
    third of the budget, else the leading rows of A sized from two probes
    (1% and 4% of the rows) so that a step takes about a third of it.
    With all_cores, also `cores` copies of the same step run at once (one
    host thread each; the C oracle runs outside the interpreter lock): the
    host's aggregate oracle throughput."""
    one = _oracle_step(cfg)
    A = cfg["A"]
    # step time ~ fixed (B's bucketing) + frac * per-row part: two probes
    t1, _ = one(_rows_sample(A, 0.01))
    t4, _ = one(_rows_sample(A, 0.04))
    t_var = max((t4 - t1) / 0.03, 1e-6)
    t_fix = max(t1 - 0.01 * t_var, 0.0)
    est_full = t_fix + t_var
    frac = 1.0 if est_full <= budget_s / 3 else max(0.01, (budget_s / 3 - t_fix) / t_var)
    As = _rows_sample(A, frac)
    times, units = [], None
    t_start = time.perf_counter()
    while True:
        t, units = one(As)
        times.append(t)
        if time.perf_counter() - t_start > budget_s or len(times) >= 5:
            break
    t = statistics.median(times)
    what = "full workload" if frac >= 1.0 else f"leading {frac:.3f} of A's rows (B whole)"
    out = {"value": round(units / t / 1e9, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{len(times)} step(s) of the {what}, median {t:.3f} s"}
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    out["host_cores"] = cores
    if all_cores and cores > 1:
        import concurrent.futures as cf
        with cf.ThreadPoolExecutor(max_workers=cores) as ex:
            t0 = time.perf_counter()
            res = list(ex.map(lambda _i: one(As), range(cores)))
            wall = time.perf_counter() - t0
        u = sum(r[1] for r in res)
        out["all_cores"] = {"value": round(u / wall / 1e9, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{cores} concurrent copies of one step of the {what}, wall {wall:.3f} s"}
    return out


# ---------------------------------------------------------------------------
# reference arm: the oracle, timed on the host cores
# ---------------------------------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    cfg, workload = load_config(args.config)
    A, B = cfg["A"], cfg["B"]
    nA, nB = len(A["liv"]), len(B["liv"])
    total_a = int(np.prod(np.asarray(A["dims"], dtype=np.float64)))

    # bounded sample: the leading rows of A (A is row-major, so a LIV prefix)
    def sample(frac):
        keep = A["liv"] < int(frac * total_a)
        return {"dims": A["dims"], "sig": A["sig"], "liv": A["liv"][keep], "val": A["val"][keep]}

    def one(As):
        t0 = time.perf_counter()
        liv, val, _ = oracle.contract(As, B, cfg["modes_a"], cfg["modes_b"])
        if "permute_sig" in cfg:
            cd = c_dims_of(cfg)
            oracle.permute(cd, list(range(len(cd) - 1, -1, -1)), cfg["permute_sig"], liv, val)
        return time.perf_counter() - t0, len(As["liv"]) + nB + len(liv)

    t_full, _ = one(A)
    total_steps = args.steps + args.warmup
    frac = min(1.0, 150.0 / max(total_steps * t_full, 1e-9))
    As = A if frac >= 1.0 else sample(frac)
    for _ in range(args.warmup):
        one(As)
    times, units = [], 0
    for _ in range(args.steps):
        t, u = one(As)
        times.append(t)
        units = u
    total = sum(times)
    value = units * args.steps / total / 1e9
    desc = ("full workload" if frac >= 1.0 else f"leading {frac:.3f} of A's rows") + \
        f" per step, {args.steps} steps"
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
           "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(total / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload, "name": args.config, "nnz_a": nA, "nnz_b": nB},
           "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
           "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_permute_case(args):
    """Stand-alone permutation (k,l,m,i,j,n) of a random 64^6 tensor with
    --nnz non-zeros; prints per-kernel times.  Not the benchmark line."""
    import torch
    import paper_1802_02619_gb300 as lco
    rng = np.random.default_rng(7)
    liv = np.unique(rng.integers(0, 1 << 36, size=int(args.nnz * 1.02) + 16))[:args.nnz].astype(np.int64)
    val = rng.standard_normal(liv.shape[0])
    t = lco.LcoTensor([64] * 6, [5, 4, 3, 2, 1, 0], torch.tensor(liv, device="cuda"),
                      torch.tensor(val, device="cuda"))
    new_sig = [5, 1, 0, 4, 3, 2]
    perm = lco.Permuter(t.dims, t.sig, new_sig, t.nnz)
    out_l, out_v = torch.empty_like(t.liv), torch.empty_like(t.val)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        perm(t.liv, t.val, out_l, out_v)
    torch.cuda.synchronize()
    lco.timing_enable(True)
    for _ in range(args.steps):
        flush.zero_()
        perm(t.liv, t.val, out_l, out_v)
    recs = lco.timing_read()
    lco.timing_enable(False)
    per = {}
    for nm, ms in recs:
        per.setdefault(nm, []).append(ms)
    n = t.nnz
    out = {"case": "permute", "nnz": n, "kernels": {k: round(sum(v) / len(v), 5) for k, v in per.items()}}
    if "k_radix_scatter" in per:
        ms = sum(per["k_radix_scatter"]) / len(per["k_radix_scatter"])
        out["scatter_gbs"] = round(32 * n / (ms * 1e-3) / 1e9, 1)
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# batched workload: thousands of small contractions
# ---------------------------------------------------------------------------

def _lco_tensor(T, device):
    import torch
    import paper_1802_02619_gb300 as lco
    if isinstance(T["liv"], torch.Tensor):
        return lco.LcoTensor(list(T["dims"]), list(T["sig"]), T["liv"].to(device), T["val"].to(device))
    return lco.LcoTensor.from_host(T, device)


def batch_workload(count, seed, device):
    """The batch mix with its admission rule: a drawn item is kept only if
    its product count f is at most 16 (nnz_A + nnz_B) (f from the library's
    symbolic phase); rejected items are redrawn from the next seed."""
    import paper_1802_02619_gb300 as lco
    import synth

    def admit(A, B, ma, mb):
        At, Bt = _lco_tensor(A, device), _lco_tensor(B, device)
        p = lco.ContractPlan(At.dims, At.sig, At.nnz, Bt.dims, Bt.sig, Bt.nnz, ma, mb)
        p.ensure_workspace(0, device)
        p.symbolic(At, Bt)
        return p.result()["f"] <= 16 * (At.nnz + Bt.nnz)

    probs = synth.batch_problems(count=count, seed=seed, admit=admit, device=device)
    items = [(_lco_tensor(A, device), _lco_tensor(B, device), ma, mb) for A, B, ma, mb, _ in probs]
    return probs, items


def run_batch_case(args):
    """C4 on its own (--case batch): the measure_batch record, printed."""
    out = measure_batch(args.count, args.steps, args.warmup, args.streams,
                        cpu_budget_s=0.0 if args.no_cpu_baseline else 12.0, tune=args.tune,
                        per_kind=args.per_kind)
    print(json.dumps(out), flush=True)


def measure_batch(count, K, warmup, streams, cpu_budget_s=12.0, tune=False, per_kind=False):
    """C4: `count` problems (1/4 2D FD, 1/4 3D FD, 1/2 R-MAT) contracted
    as one batch replayed from a CUDA graph, against the plain loop of one
    contraction call per problem with a stream synchronisation after each
    (plans and workspaces prepared in advance for both)."""
    import torch
    import paper_1802_02619_gb300 as lco
    device = "cuda"
    t_gen = time.perf_counter()
    probs, items = batch_workload(count, 100, device)
    t_gen = time.perf_counter() - t_gen
    kinds = {}
    for *_x, kind in probs:
        kinds[kind] = kinds.get(kind, 0) + 1
    batch = lco.Batch(items, nstreams=streams)
    batch.run()
    outs = batch.results()
    nnz_in = sum(A.nnz + B.nnz for A, B, _a, _b in items)
    nnz_c = sum(C.nnz for C in outs)
    units = nnz_in + nnz_c
    algs = {}
    for inf in batch.info:
        algs[inf["alg"]] = algs.get(inf["alg"], 0) + 1
    stream = torch.cuda.current_stream()

    # ---- batched: one graph replay per step ----
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    t_cap = time.perf_counter()
    with torch.cuda.stream(side):
        batch.run()
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=side):
            batch.run()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    t_cap = time.perf_counter() - t_cap
    n0 = lco.launch_count()
    batch.run()
    torch.cuda.synchronize()
    launches_per_step = lco.launch_count() - n0
    for _ in range(max(warmup, 3)):
        graph.replay()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(K):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_batch = e0.elapsed_time(e1) / K
    for C, C2 in zip(outs, batch.results()):
        assert torch.equal(C.liv, C2.liv), "graph replay changed a result"
    # per-kernel times of one stacked run (direct launches, kernel events)
    lco.timing_enable(True)
    batch.run()
    torch.cuda.synchronize()
    recs = lco.timing_read()
    lco.timing_enable(False)
    per_kernel = {}
    for nm, ms in recs:
        t = per_kernel.setdefault(nm, [0, 0.0])
        t[0] += 1
        t[1] += ms
    top = sorted(per_kernel.items(), key=lambda kv: -kv[1][1])[:12]
    kernels = {nm: {"launches": c, "ms": round(ms, 3)} for nm, (c, ms) in top}
    # the per-problem path (every problem's phases on the stream pool), same graph form
    gpp = torch.cuda.CUDAGraph()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        batch.run_per_problem()
        torch.cuda.synchronize()
        with torch.cuda.graph(gpp, stream=side):
            batch.run_per_problem()
    stream.wait_stream(side)
    for _ in range(3):
        gpp.replay()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(K):
        gpp.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_pp = e0.elapsed_time(e1) / K
    for C, C2 in zip(outs, batch.results()):
        assert torch.equal(C.liv, C2.liv), "per-problem path differs from the stacked one"
    del gpp

    # ---- plain loop: one call per problem, stream sync after each ----
    plans = []
    for (A, B, ma, mb), f in zip(items, batch.f):
        p = lco.ContractPlan(A.dims, A.sig, A.nnz, B.dims, B.sig, B.nnz, ma, mb)
        p.ensure_workspace(f, device)
        plans.append(p)
    c_liv = [batch.c_liv_all[o:o + f] for o, f in zip(batch.c_off, batch.f)]
    c_val = [batch.c_val_all[o:o + f] for o, f in zip(batch.c_off, batch.f)]

    def plain():
        for p, (A, B, _a, _b), cl, cv in zip(plans, items, c_liv, c_val):
            p.run(A, B, cl, cv)
            stream.synchronize()

    plain()
    Kp = max(1, min(K, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(Kp):
        plain()
    ms_plain = (time.perf_counter() - t0) * 1e3 / Kp
    del plans, c_liv, c_val                 # the plain loop's workspaces
    torch.cuda.empty_cache()

    out = {
        "metric": "batched contraction GNNZ/s", "value": round(units / (ms_batch * 1e-3) / 1e9, 4),
        "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": warmup, "ms_per_step": round(ms_batch, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"batch of {count}: fd2d/fd3d self-compositions + R-MAT Eq.14/Eq.16/SOP",
                   "kinds": kinds, "algs": algs, "nnz_in": nnz_in, "nnz_c": nnz_c, "f": sum(batch.f),
                   "streams": streams, "l2": "inputs larger than L2 (no flush)",
                   "graph": "whole batch replayed from one CUDA graph",
                   "gen_s": round(t_gen, 2), "capture_s": round(t_cap, 2)},
        "plain_loop": {"value": round(units / (ms_plain * 1e-3) / 1e9, 4), "unit": UNIT,
                       "ms_per_step": round(ms_plain, 3), "steps": Kp,
                       "what": "one contraction call per problem + stream sync, plans/workspaces prepared"},
        "speedup_vs_plain_loop": round(ms_plain / ms_batch, 3),
        "per_problem_graph": {"value": round(units / (ms_pp * 1e-3) / 1e9, 4), "ms_per_step": round(ms_pp, 4),
                              "what": "every problem's two phases on the stream pool, one graph replay"},
        "kernels_stacked_run": kernels,
        "roofline": {"bound": "hbm", "kernel": "whole batch (all kernels)",
                     "achieved": round(16 * units / (ms_batch * 1e-3) / 1e9, 1),
                     "peak": measured_peak_hbm()[0], "unit": "GB/s",
                     "frac": round(16 * units / (ms_batch * 1e-3) / 1e9 / measured_peak_hbm()[0], 4),
                     "traffic": None, "algorithmic_bytes": 16 * units,
                     "note": "16 B per input and output entry over the batch time (operand permutation "
                             "passes not counted)"},
        "gpu_launches": int(launches_per_step * K),
        "clocks": clk,
    }
    if tune:
        # the autotuner's per-signature choices (one sample per group), then
        # the same batch rebuilt with them and replayed the same way
        from paper_1802_02619_gb300.tune import Tuner
        t_tune = time.perf_counter()
        tuner = Tuner(cache_path=None, reps=2)
        choice = tuner.tune_batch(items, per_class=1)
        t_tune = time.perf_counter() - t_tune
        infos = [dict(x) for x in batch.info]
        # the untuned batch's graph and workspaces go first: a tuned choice
        # (SOP, wide digits) can need far larger workspaces
        del graph, batch
        gc.collect()
        torch.cuda.empty_cache()
        bt = lco.Batch([it + tuple(c) for it, c in zip(items, choice)], nstreams=streams)
        bt.run()
        gt = torch.cuda.CUDAGraph()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            with torch.cuda.graph(gt, stream=side):
                bt.run()
        stream.wait_stream(side)
        for _ in range(3):
            gt.replay()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(K):
            gt.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_t = e0.elapsed_time(e1) / K
        changed = sum(1 for inf, (alg, bits, order) in zip(infos, choice)
                      if inf["alg"] != alg or bits != 0 or order != 0)
        out["tuned"] = {"value": round(units / (ms_t * 1e-3) / 1e9, 4), "ms_per_step": round(ms_t, 4),
                        "groups": len(tuner.cache), "problems_changed": changed, "tune_s": round(t_tune, 1)}
        del gt, bt
    if per_kind:
        # each kind of problem as a batch of its own (same graph replay)
        per = {}
        for kind in sorted(kinds):
            sel = [it for it, pr in zip(items, probs) if pr[4] == kind]
            bk = lco.Batch(sel, nstreams=streams)
            bk.run()
            u = sum(A.nnz + B.nnz for A, B, _a, _b in sel) + sum(C.nnz for C in bk.results())
            g = torch.cuda.CUDAGraph()
            side.wait_stream(stream)
            with torch.cuda.stream(side):
                with torch.cuda.graph(g, stream=side):
                    bk.run()
            stream.wait_stream(side)
            for _ in range(3):
                g.replay()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(K):
                g.replay()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / K
            per[kind] = {"problems": len(sel), "units": u, "ms": round(ms, 3),
                         "gnnz_s": round(u / (ms * 1e-3) / 1e9, 3)}
            del g, bk
        out["per_kind"] = per
    if cpu_budget_s > 0:
        import oracle
        t_start, done_units, done_t = time.perf_counter(), 0, 0.0
        order = np.random.default_rng(1).permutation(len(probs))
        nprob = 0
        for i in order:
            A, B, ma, mb, _k = probs[i]
            Ah = {kk: (v.cpu().numpy() if hasattr(v, "cpu") else v) for kk, v in A.items()}
            Bh = {kk: (v.cpu().numpy() if hasattr(v, "cpu") else v) for kk, v in B.items()}
            t1 = time.perf_counter()
            liv, _v, _ = oracle.contract(Ah, Bh, ma, mb)
            done_t += time.perf_counter() - t1
            done_units += len(Ah["liv"]) + len(Bh["liv"]) + len(liv)
            nprob += 1
            if time.perf_counter() - t_start > cpu_budget_s:
                break
        out["cpu_baseline"] = {"value": round(done_units / done_t / 1e9, 6), "unit": UNIT, "cores": 1,
                               "kind": "oracle", "sample": f"{nprob} random problems of the batch"}
    return out


# ---------------------------------------------------------------------------
# served workload: Poisson arrivals against the server
# ---------------------------------------------------------------------------

def _percentiles(xs):
    xs = sorted(xs)
    if not xs:
        return {"p50": None, "p99": None}
    return {"p50": round(xs[len(xs) // 2], 1), "p99": round(xs[min(len(xs) - 1, int(0.99 * len(xs)))], 1),
            "max": round(xs[-1], 1)}


def run_serve_case(args):
    """C5 on its own (--case serve): the measure_serve record, printed."""
    print(json.dumps(measure_serve(args.requests, args.slots, args.workers)), flush=True)


def measure_serve(N, slots, workers):
    """C5: 128 resident problems (32 2D FD 16^2..256^2, 32 3D FD, 64 R-MAT
    pairs of 1e3..1e6 non-zeros in the batch forms); requests pick a problem
    uniformly (seed 200).  Saturation throughput from a burst of all
    requests; then Poisson arrivals at 0.5x and 0.8x that rate, latency =
    completion - arrival.  The plain path serves the same arrivals with one
    contraction call and one stream synchronisation per request, in order."""
    import threading as th
    import torch
    import paper_1802_02619_gb300 as lco
    device = "cuda"
    probs, items = batch_workload(128, 300, device)
    rng = np.random.default_rng(200)
    pick = rng.integers(0, len(items), size=N)
    srv = lco.Server(pool_bytes=64 << 30, nslots=slots, nworkers=workers)
    handles = [(srv.put(A), srv.put(B)) for A, B, _a, _b in items]
    # units of each problem (nnz_A + nnz_B + nnz_C), from one served run
    units = []
    for (ha, hb), (A, B, ma, mb) in zip(handles, items):
        r = srv.wait(srv.submit(ha, hb, ma, mb))
        assert r["status"] == 0, r
        units.append(A.nnz + B.nnz + r["C"].nnz)
    for rid in range(1, len(items) + 1):
        srv.release(rid)

    def serve_run(arrivals):
        """Submit request k at arrivals[k] (seconds from start; None: all at
        once); a collector thread waits and releases in submission order."""
        rids = [0] * N
        ready = [th.Event() for _ in range(N)]
        lat, done_t = [0.0] * N, [0.0] * N

        def collect():
            for k in range(N):
                ready[k].wait()
                r = srv.wait(rids[k])
                assert r["status"] == 0, r
                lat[k] = r["done_us"] - r["submit_us"]
                done_t[k] = r["done_us"]
                srv.release(rids[k])

        t = th.Thread(target=collect)
        t.start()
        t0 = time.perf_counter()
        for k in range(N):
            if arrivals is not None:
                while time.perf_counter() - t0 < arrivals[k]:
                    pass
            ha, hb = handles[pick[k]]
            A, B, ma, mb = items[pick[k]]
            rids[k] = srv.submit(ha, hb, ma, mb)
            ready[k].set()
        t.join()
        wall = time.perf_counter() - t0
        u = sum(units[i] for i in pick)
        return {"requests_per_s": round(N / wall, 1), "gnnz_s": round(u / wall / 1e9, 4),
                "latency_us": _percentiles(lat), "wall_s": round(wall, 3)}

    serve_run(None)                                        # warm-up
    sat = serve_run(None)
    lam = sat["requests_per_s"]

    # plain path: plans and workspaces made in advance, one call + sync per request
    plans, outs = [], []
    for A, B, ma, mb in items:
        p = lco.ContractPlan(A.dims, A.sig, A.nnz, B.dims, B.sig, B.nnz, ma, mb)
        p.ensure_workspace(0, device)
        p.symbolic(A, B)
        f = p.result()["f"]
        p.ensure_workspace(f, device)
        plans.append(p)
        outs.append((torch.empty(max(f, 1), dtype=torch.int64, device=device),
                     torch.empty(max(f, 1), dtype=torch.float64, device=device)))
    stream = torch.cuda.current_stream()

    def plain_run(arrivals):
        lat = []
        t0 = time.perf_counter()
        for k in range(N):
            i = pick[k]
            if arrivals is not None:
                while time.perf_counter() - t0 < arrivals[k]:
                    pass
            A, B, _a, _b = items[i]
            plans[i].run(A, B, outs[i][0], outs[i][1])
            stream.synchronize()
            lat.append((time.perf_counter() - t0 - (arrivals[k] if arrivals is not None else 0.0)) * 1e6)
        wall = time.perf_counter() - t0
        u = sum(units[i] for i in pick)
        return {"requests_per_s": round(N / wall, 1), "gnnz_s": round(u / wall / 1e9, 4),
                "latency_us": _percentiles(lat), "wall_s": round(wall, 3)}

    plain_run(None)
    plain_sat = plain_run(None)

    def api_run(n_req):
        """The public one-call API per request (plan, workspace, two
        synchronisations), back to back: its saturation throughput."""
        t0 = time.perf_counter()
        for k in range(n_req):
            A, B, ma, mb = items[pick[k]]
            lco.contract(A, B, ma, mb)
        wall = time.perf_counter() - t0
        u = sum(units[pick[k]] for k in range(n_req))
        return {"requests_per_s": round(n_req / wall, 1), "gnnz_s": round(u / wall / 1e9, 4),
                "requests": n_req, "wall_s": round(wall, 3)}

    api_run(min(N, 200))
    api_sat = api_run(min(N, 2000))
    rates = {}
    for frac in (0.5, 0.8):
        arr = np.cumsum(rng.exponential(1.0 / (frac * lam), size=N))
        rates[str(frac)] = {"rate_per_s": round(frac * lam, 1), "served": serve_run(arr), "plain": plain_run(arr)}
    st = srv.stats()
    srv.close()
    out = {"metric": "served contraction GNNZ/s", "value": rates["0.8"]["served"]["gnnz_s"], "unit": UNIT,
           "n_gpus": 1, "higher_is_better": True, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "128 resident problems (fd2d, fd3d, R-MAT Eq.14/Eq.16/SOP), uniform picks",
                      "requests": N, "slots": slots, "workers": workers, "pool_gb": 64},
           "saturation": {"served": sat, "plain": plain_sat, "plain_api": api_sat,
                          "served_vs_plain": round(sat["requests_per_s"] / plain_sat["requests_per_s"], 2),
                          "served_vs_plain_api": round(sat["requests_per_s"] / api_sat["requests_per_s"], 2)},
           "poisson": rates, "pool_peak_gb": round(st["pool_peak"] / 2**30, 2)}
    return out


# ---------------------------------------------------------------------------
# permutation sweep: every order of the Eq. 4 operator (Table 2's setting)
# ---------------------------------------------------------------------------

def run_permsweep_case(args):
    """The combinatorial Laplacian of Eq. 4 (N x N image: N^4 index space,
    ~5 N^2 entries) permuted from its row-major order into each of the 23
    other orders of its four modes with the radix permutation (Sec. 4.1).
    Per order: median time over the timed repetitions (L2 flushed before
    each), keys/s, and the sort key's width and passes after the resting
    digits are skipped."""
    import itertools
    import torch
    import paper_1802_02619_gb300 as lco
    import synth
    from paper_1802_02619_gb300.laplacian import combinatorial_laplacian
    N = args.N
    a = combinatorial_laplacian(lco.LcoTensor.from_host(synth.fd_matrix(N), "cuda"),
                                lco.LcoTensor.from_host(synth.kronecker_delta(N), "cuda"))
    n = a.nnz
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out_l, out_v = torch.empty_like(a.liv), torch.empty_like(a.val)
    stream = torch.cuda.current_stream()
    rows = []
    for perm in itertools.permutations(range(4)):
        sig = list(perm)
        if sig == list(a.sig):
            continue
        info = lco.radix_permute_info(a.dims, a.sig, sig, n)
        p = lco.Permuter(a.dims, a.sig, sig, n)
        for _ in range(max(args.warmup, 2)):
            p(a.liv, a.val, out_l, out_v)
        ts = []
        for _ in range(max(args.steps, 3)):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            p(a.liv, a.val, out_l, out_v)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        assert p.device_status() == 0
        ms = statistics.median(ts)
        rows.append({"sig": sig, "ms": round(ms, 4), "gkeys_s": round(n / (ms * 1e-3) / 1e9, 3),
                     "key_bits": info["key_bits"], "passes": info["passes"], "n_rearr": info["n_rearr"]})
    ms_all = sorted(r["ms"] for r in rows)
    out = {"case": "permsweep", "metric": "permutation Gkeys/s", "N": N, "nnz": n, "orders": len(rows),
           "summary_ms": {"max": ms_all[-1], "median": ms_all[len(ms_all) // 2], "min": ms_all[0]},
           "paper_context": "RP on an E8400 at N ~ 2896 (Table 2): max 3.54 s, median 3.45 s, min 1.38 s",
           "rows": rows}
    print(json.dumps(out), flush=True)


def run_permute_wide_case(args):
    """Radix permutation of a tensor with wide (128-bit) LIVs: order 4,
    dims 2^40 x (2^40 - 3) x (2^30 + 3) x 1000 (~2^120 index space), 16M
    non-zeros drawn uniformly, row-major -> fully reversed order (an 80-bit
    sort key in two 54-bit chunks).  Inputs resident on the device; L2
    flushed before every step.  Algorithmic bytes per non-zero: 48 (read and
    write a 16-byte LIV and an 8-byte value)."""
    import torch
    import paper_1802_02619_gb300 as lco
    import synth
    dims, sig, new_sig = [1 << 40, (1 << 40) - 3, (1 << 30) + 3, 1000], [3, 2, 1, 0], [0, 1, 2, 3]
    nnz = args.nnz or 16_000_000
    T = synth.wide_tensor(dims, sig, nnz, seed=21)
    n = T["liv"].shape[0]
    liv = torch.from_numpy(T["liv"].view(np.int64)).cuda()
    val = torch.as_tensor(T["val"]).cuda()
    p = lco.WidePermuter(dims, sig, new_sig, n)
    out_l, out_v = torch.empty_like(liv), torch.empty_like(val)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        p(liv, val, out_l, out_v)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    ts = []
    steps = max(min(args.steps, 50), 5)
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p(liv, val, out_l, out_v)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    assert p.device_status() == 0
    # output LIVs strictly ascending as unsigned 128-bit numbers (the low word
    # compared unsigned by flipping its sign bit)
    hi, lo = out_l[:, 1], out_l[:, 0] ^ torch.iinfo(torch.int64).min
    assert bool(((hi[1:] > hi[:-1]) | ((hi[1:] == hi[:-1]) & (lo[1:] > lo[:-1]))).all()), "output not ascending"
    ms = statistics.median(ts)
    info = lco.radix_permute_wide_info(dims, sig, new_sig, n)
    peak, kind = measured_peak_hbm()
    achieved = 48.0 * n / (ms * 1e-3) / 1e9
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        m = min(n, 1_000_000)
        t0 = time.perf_counter()
        oracle.permute_wide(dims, sig, new_sig, T["liv"][:m], T["val"][:m])
        dt = time.perf_counter() - t0
        cpu = {"value": round(m / dt / 1e9, 5), "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
               "sample": f"the first {m} non-zeros of the same tensor, one run, {dt:.2f} s"}
    out = {"case": "permute_wide", "metric": "wide-LIV permutation Gkeys/s", "value": round(n / (ms * 1e-3) / 1e9, 4),
           "unit": "Gkeys/s", "ms_per_step": round(ms, 4), "steps": steps, "nnz": n, "dtype": "u128+f64",
           "config": {"workload": "order-4 wide tensor 2^40 x (2^40-3) x (2^30+3) x 1000, uniform LIVs, "
                                  "row-major -> reversed", "l2": "flushed before every step"},
           "key": info, "clocks": clk,
           "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "peak_kind": kind,
                        "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                        "algorithmic_bytes": 48 * n},
           "cpu_baseline": cpu}
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.case == "permute":
        run_permute_case(args)
        return
    if args.case == "batch":
        run_batch_case(args)
        return
    if args.case == "serve":
        run_serve_case(args)
        return
    if args.case == "permute_wide":
        run_permute_wide_case(args)
        return
    if args.case == "permsweep":
        run_permsweep_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_lco(args)


if __name__ == "__main__":
    main()
