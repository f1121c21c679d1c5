#!/usr/bin/env python
"""Benchmark: Bellman transitions/s of the GB300 engine.

Default workload: the largest configuration that fits one GPU, the 6-D linear
traffic ring -- 21^6 = 85.8 M states, 4 inputs (two binary on-ramp lights),
sigma 0.5, explicit 5^6 windows (15,625 slots), safety [0,18]^6, horizon 8,
FP32 with Kahan-compensated window sums, per-dimension tables.  The other
workloads (unicycle 51x51x30, robot 41x41, rooms 9^7, the served stream) run
with --workload.

One step = one pass of the whole hot path over the workload: the tables are
rebuilt on the GPU (amy_rebuild), the spec mask and V_N are formed, and
`horizon` fused backups + max/argmax run, every pi_k written.  Transitions
per step = n_states * n_inputs * prod(W) * horizon (every allocated window
slot).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl amy|reference] [--workload ...]

N > 1 runs one independent replica per GPU (weak scaling, no collective).
--impl reference times the FP64 CPU oracle on the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

WORKLOAD_NAME = ("unicycle 51x51x30 states (theta periodic), 45 inputs, sigma 0.05, gamma 1e-6 "
                 "(3x3x3 window), reach [8,10]^2, horizon 32")
TRAFFIC_NAME = ("6-D traffic ring 21^6 states (85.8 M), 4 inputs, sigma 0.5, window 5^6, safety [0,18]^6, "
                "horizon 8, FP32 + Kahan")
DEFAULT_WORKLOAD = "traffic6"
METRIC = "Bellman transitions/s (x*u*x' window slots * horizon)"
UNIT = "transitions/s"


# DRAM traffic of the dominant kernel per backup, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of the launch, divided by the
# backups that launch performed).  A figure holds only for the kernel sources
# it was captured on: each entry carries the digest of the kernel's header and
# the headers it includes, and is reported as null once they change.  A
# capture on a reduced grid is scaled to the full launch by the number of
# states (the traffic is V in/out, pi and the mask per state; the tables are a
# few hundred KB at most).
# (workload, tmode, prec, v_store) -> (digest, DRAM bytes per backup, states
# of the measured case, profile summary, kernel header)
MEASURED_TRAFFIC = {
    # k_synth_runs<float,3,3,0>, launch shape 1,288,1,0,3, grid barrier: 710,656 B read +
    # 65,024 B written per launch of 32 backups
    ("unicycle", "stored_separable", "fp32", "native"):
        ("a0f7d4cc08dc1935", 24240, 78030, "profiles/k_synth_runs_unicycle_51x51x30.md", "amy_runs.cuh"),
    # k_backup_tile<float,5> at 18^6 (34,012,224 states): 597,405,440 B read + 563,790,848 B
    # written per backup, scaled to the workload's states (V in and out and their re-fetches)
    ("traffic6", "stored_separable", "fp32_kahan", "native"):
        ("1048333ee2290287", 1161196288, 34012224, "profiles/k_backup_tile_traffic6.md", "amy_tile.cuh"),
}


def csrc_digest(root: str = None) -> str:
    """Digest of device code: the header `root` (in csrc/) and every header it
    includes from there, recursively; without `root`, every .cuh header."""
    import hashlib
    import re
    d = os.path.join(ROOT, "paper_2005_06191_gb300", "csrc")
    if root is None:
        files = sorted(f for f in os.listdir(d) if f.endswith(".cuh"))
    else:
        files, todo = set(), [root]
        while todo:
            f = todo.pop()
            if f in files or not os.path.exists(os.path.join(d, f)):
                continue
            files.add(f)
            todo += re.findall(r'#include "([^"/]+)"', open(os.path.join(d, f)).read())
        files = sorted(files)
    h = hashlib.sha256()
    for f in files:
        h.update(f.encode())
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(args, n_states: int):
    e = MEASURED_TRAFFIC.get((args.workload, args.tmode, args.prec, args.v_store))
    if e is None or e[0] != csrc_digest(e[4]):
        return None, None
    return int(round(e[1] * n_states / e[2])), e[3]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)),
                "source": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clock/throttle samples taken while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"amy_clocks_gpu{gpu_index}_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus: int):
    rank, world = 0, 1
    if n_gpus > 1 or "WORLD_SIZE" in os.environ:
        import torch.distributed as dist
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        if world > 1:
            import torch
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(backend=backend)
    return rank, world


def barrier_max(value: float, world: int) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


WORKLOADS = {
    # name: (constructor(size or None), default T mode, default precision, description)
    "unicycle": (lambda s: W.unicycle(nxy=s or 51), "stored_separable", "fp32", WORKLOAD_NAME),
    "robot": (lambda s: W.robot_lin(n_per_dim=s or 41), "stored_full", "fp64",
              "2-D linear robot 41x41 states, 25 inputs, sigma 0.2, dense rows, reach-avoid, horizon 8"),
    "rooms7": (lambda s: W.rooms7(n_per_dim=s or 9), "stored_separable", "fp32_kahan",
               "7-room temperature ring 9^7 states, 5 inputs, sigma 0.02, window 3^7, safety, horizon 10"),
    "traffic6": (lambda s: W.traffic6(n_per_dim=s or 21), "stored_separable", "fp32_kahan", TRAFFIC_NAME),
    "robot_dist": (lambda s: W.robot_dist(n_per_dim=s or 41), "stored_separable", "fp32",
                   "2-D robot of Sec. 7 with its disturbance: 41^2 states, 121 inputs, 11 disturbance points, "
                   "Sigma = 0.75 I, gamma 1e-3 (13x13 window), safety in X, horizon 8 (203401 state-input pairs)"),
}


def workload(args):
    w = WORKLOADS[args.workload][0](args.size)
    w.tmode, w.precision = args.tmode, args.prec
    if args.horizon is not None:
        w.horizon = args.horizon
    return w


def workload_name(args) -> str:
    name = WORKLOADS[args.workload][3]
    if args.size is not None or args.horizon is not None:
        name += f" [reduced: size {args.size}, horizon {args.horizon}]"
    return name


def transitions_per_step(w, window_slots: int) -> int:
    p = w.problem
    return p.n_states * p.n_inputs * p.n_disturbances * window_slots * w.horizon


# ---------------------------------------------------------------------------
# the engine arm
# ---------------------------------------------------------------------------
def run_amy(args, rank, world):
    import torch
    import paper_2005_06191_gb300 as amy
    from paper_2005_06191_gb300 import build as engine_build

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if rank == 0 or not engine_build.up_to_date():
        engine_build.build()
    barrier(world)
    w = workload(args)
    p, spec, N = w.problem, w.spec, w.horizon
    stream = torch.cuda.current_stream()
    shape = [int(v) for v in args.shape.split(",")] if args.shape else None
    h = amy.amy_build(p, tmode=args.tmode, prec=args.prec, v_store=args.v_store, autotune=shape is None,
                      launch_shape=shape)
    if args.step_wait is not None:
        amy.amy_set_step_wait(h, args.step_wait)
    if args.plane is not None or args.plane_smem:
        amy.amy_set_plane(h, args.plane if args.plane is not None else 1, args.plane_smem)
    info = amy.amy_info(h)
    trans = transitions_per_step(w, info["window_slots"])
    V = torch.empty(p.n_states, dtype=torch.float64 if args.prec == "fp64" else torch.float32, device="cuda")
    PI = torch.empty((N, p.n_states), dtype=torch.int16, device="cuda")
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)

    def step():
        amy.amy_rebuild(h)
        amy.amy_synthesize(h, spec, N, V_out=V, policy_out=PI, policy_all_steps=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    lane_peaks = amy.amy_measure_lane_loads()  # roofline denominators (outside the timed region)
    plane_family = info["backup_kernel"] in (7, 8)
    lane_peaks.update({"fma_" + k: v for k, v in amy.amy_measure_fma().items()})
    if args.tmode == "otf":
        lane_peaks.update({"erfc_" + k: v for k, v in amy.amy_measure_erfc().items()})
    if plane_family:
        lane_peaks["l2_bytes"] = amy.amy_measure_l2()
    # the plane kernel's own work in one backup (counted in an untimed run)
    work = amy.amy_backup_work(h, spec) if plane_family else None
    barrier(world)
    amy.amy_kernel_times(h)  # reset
    amy.amy_set_profiling(h, True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()  # evict L2 between timed iterations (outside the timed interval)
            starts[i].record(stream)
            step()
            ends[i].record(stream)
        torch.cuda.synchronize()
    amy.amy_set_profiling(h, False)
    kt = amy.amy_kernel_times(h)
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    ms_max = barrier_max(ms, world)
    value = trans * args.steps * world / (ms_max / 1e3)
    # kernel-level roofline of the dominant kernel (the fused backup)
    # kernels per timed step: the backups, one spec-mask kernel, and the build
    # (for the per-dimension tables: bounds reset + tables [+ shifted inner table])
    launches = (info["backup_launch_kernels"] * kt["backup_launches"] + info["build_kernels"] * kt["build_launches"]
                + args.steps)
    if plane_family:
        launches += args.steps  # the padded copy of V_N the plane kernel reads, once per synthesis
    # per backup: the persistent kernel performs the whole horizon in one launch
    bk_ms = kt["backup_ms"] / max(kt["backup_steps"], 1)
    launch_ms = kt["backup_ms"] / max(kt["backup_launches"], 1)
    build_ms = kt["build_ms"] / max(kt["build_launches"], 1)
    V_host = V.cpu().numpy()
    # states whose value the spec fixes carry policy 0xFFFF and cost no backup work
    free = int((PI[0] != -1).sum().item())
    roof = roofline(args, w, info, bk_ms, free, lane_peaks, work)
    roof["backups_per_launch"] = kt["backup_steps"] / max(kt["backup_launches"], 1)
    roof["launch_ms"] = launch_ms

    # end to end through the C ABI with host buffers, per step: the system
    # parameters from pinned host memory (amy_rebuild: H2D + table build),
    # then amy_synthesize with host outputs (D2H of V_0 and every pi_k into
    # pinned host memory).  The handle (its device buffers and launch shape)
    # is set up once, as a caller solving a stream of problems of one shape
    # would.  e2e_cold adds amy_build and amy_destroy to every step.
    heavy = trans > 1e12   # e.g. the 21^6 traffic ring: about a second per step
    e2e_steps = 0 if args.no_e2e else (min(3, max(args.steps, 1)) if heavy else max(3, min(args.steps, 50)))
    pin_params = torch.from_numpy(np.asarray(p.params, dtype=np.float64)).pin_memory().numpy()
    h2d = pin_params.nbytes
    d2h = p.n_states * 4 + N * p.n_states * 2
    Ve, e2e, e2e_cold = None, None, None
    if e2e_steps:
        Vh = torch.empty(p.n_states, dtype=torch.float64 if args.prec == "fp64" else torch.float32,
                         pin_memory=True).numpy()
        PIh = torch.empty((N, p.n_states), dtype=torch.int16, pin_memory=True).numpy()
        for _ in range(3):
            amy.amy_rebuild(h, pin_params)
            amy.amy_synthesize(h, spec, N, V_out=Vh, policy_out=PIh, policy_all_steps=True)
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            amy.amy_rebuild(h, pin_params)
            amy.amy_synthesize(h, spec, N, V_out=Vh, policy_out=PIh, policy_all_steps=True)
        e2e_s = barrier_max(time.perf_counter() - t0, world)
        Ve = Vh.copy()
        e2e = {"value": trans * e2e_steps * world / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "per_step": "amy_rebuild(params from pinned host memory) + amy_synthesize(host outputs, pinned)"}
        cold_steps = 1 if heavy else max(1, min(e2e_steps, 5))
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(cold_steps):
            with amy.amy_build(p, tmode=args.tmode, prec=args.prec, v_store=args.v_store) as he:
                amy.amy_synthesize(he, spec, N, V_out=Vh, policy_out=PIh, policy_all_steps=True)
        cold_s = barrier_max(time.perf_counter() - t0, world)
        e2e_cold = {"value": trans * cold_steps * world / cold_s, "unit": UNIT,
                    "per_step": "amy_build + amy_synthesize(host outputs, pinned) + amy_destroy"}
    amy.amy_destroy(h)
    clocks = clk.summary()
    return {
        "value": value, "ms_per_step": ms_max / args.steps, "trans": trans, "info": info,
        "backup_ms": bk_ms, "build_ms": build_ms, "launches": launches, "roofline": roof,
        "e2e": e2e, "e2e_cold": e2e_cold,
        "clocks": clocks, "V": V_host, "V_e2e": Ve,
        "synth_only_value": trans * args.steps * world / ((ms_max - build_ms * args.steps) / 1e3),
    }


def roofline_plane(args, w, info, backup_ms, work, lane_peaks):
    """Roofline of the plane kernel (backup kernel 7, or its tiled form 8) from the work it counts
    in one backup (amy_backup_work): stage 1 streams V_{k+1} through L2 (each
    staged row reads K values, coalesced across a plane), stage 2 reads the
    partial box from shared memory, and both issue FP32 fused multiply-adds
    (one per value read, plus W[n-2] + 1 per second-stage row).  Three
    ceilings, each measured on this GPU (amy_measure_l2,
    amy_measure_lane_loads, amy_measure_fma); the closest one is reported as
    the bound and the others beside it."""
    bk_s = backup_ms / 1e3
    vbytes = 2 if args.v_store != "native" else 4
    l2_bytes = work["v_loads"] * vbytes
    fmas = work["v_loads"] + work["box_loads"] + work["box_rows"] * (info["window"][-2] + 1)
    c_l2 = {"bound": "l2", "achieved": l2_bytes / bk_s / 1e9, "peak": lane_peaks["l2_bytes"] / 1e9,
            "unit": "GB/s", "peak_source": "measured on this GPU by amy_measure_l2 (32 MiB L2-resident read)",
            "algorithmic_bytes_per_backup": int(l2_bytes)}
    c_sh = {"bound": "alu", "achieved": work["box_loads"] / bk_s / 1e9, "peak": lane_peaks["shared"] / 1e9,
            "unit": "G shared lane-loads/s",
            "peak_source": "measured on this GPU by amy_measure_lane_loads (shared path)",
            "algorithmic_lane_loads_per_backup": int(work["box_loads"])}
    c_fma = {"bound": "alu", "achieved": fmas / bk_s / 1e12, "peak": lane_peaks["fma_fp32"] / 1e12,
             "unit": "T FMA/s (FP32)", "peak_source": "measured on this GPU by amy_measure_fma (FP32)",
             "algorithmic_fmas_per_backup": int(fmas)}
    cs = [c_l2, c_sh, c_fma]
    for c in cs:
        c["frac"] = c["achieved"] / c["peak"]
    cs.sort(key=lambda c: -c["frac"])
    first = dict(cs[0])
    first["other_ceilings"] = [{k: c[k] for k in ("bound", "achieved", "peak", "unit", "frac")} for c in cs[1:]]
    traffic, src = measured_traffic(args, w.problem.n_states)
    nominal = int(w.problem.n_states * w.problem.n_inputs * info["window_slots"])
    first.update({"traffic": traffic, "traffic_source": src, "backup_kernel": info["backup_kernel"],
                  "work_per_backup": work,
                  "nominal_window_slots_per_backup": nominal,
                  # one FMA per window slot is the per-transition work of a
                  # kernel that sums every slot; the plane kernels reassociate
                  # the sum and perform fewer (work_per_backup)
                  "nominal_slot_rate_vs_fma_peak": nominal / bk_s / lane_peaks["fma_fp32"]})
    return first


def with_erfc_ceiling(first, args, w, info, backup_ms, free, nu, lane_peaks):
    """On-the-fly rows under Gaussian noise form every pair's masses from
    erfc: sum_i (W_i + 1) edge values per (free state, input) pair, against
    the erfc rate measured by amy_measure_erfc in the arithmetic's precision.
    The closest ceiling is the bound; the others are listed, closest first."""
    key = "erfc_fp64" if args.prec == "fp64" else "erfc_fp32"
    if args.tmode != "otf" or key not in lane_peaks or getattr(w.problem, "noise", "gaussian") != "gaussian":
        return first
    evals = free * nu * (info["window_sum"] + info["n"])
    ach = evals / (backup_ms / 1e3) / 1e9
    pk = lane_peaks[key] / 1e9
    width = "FP64" if args.prec == "fp64" else "FP32"
    erfc = {"bound": "alu", "achieved": ach, "peak": pk, "unit": f"G erfc/s ({width})", "frac": ach / pk,
            "traffic": first.get("traffic"), "peak_source": f"measured on this GPU by amy_measure_erfc ({width})",
            "algorithmic_erfc_per_backup": int(evals), "backup_kernel": first.get("backup_kernel")}

    def summary(c):
        return {k: c[k] for k in ("bound", "achieved", "peak", "unit", "frac")}

    rest = [first["other_ceiling"]] if "other_ceiling" in first else []
    if erfc["frac"] > first["frac"]:
        out = erfc
        rest = [summary(first)] + rest
    else:
        out = dict(first)
        rest = rest + [summary(erfc)]
    rest.sort(key=lambda c: -c["frac"])
    out["other_ceiling"] = rest[0]
    out["other_ceilings"] = rest
    return out


def roofline(args, w, info, backup_ms, free, lane_peaks, work=None):
    """Roofline of the fused backup kernel.

    Stored full / factored rows are streamed from HBM: bound = hbm,
    algorithmic bytes = rows + V in/out + pi + mask.  With per-dimension
    tables or rows on the fly T stays out of HBM and V_{k+1} is L2-resident
    (or streamed once); the kernel is then bound by the rate at which lanes
    receive their operands: the shared-memory path for the staged kernels,
    the L1 path of global loads for the register-resident ones.  Both
    ceilings are measured on the device (amy_measure_lane_loads).
    Algorithmic lane-loads per backup: one V value per (free state, input,
    window slot) for the gather kernels; for the per-run kernels, the outer
    contraction's K x W^(n-1) V values per (free state, input run) plus the
    W innermost-dim masses per (free state, input) that each input's sum
    applies to it.  The persistent kernel performs all backups of the horizon
    in one launch; the figures are per backup (the same ratio per launch)."""
    if work is not None:
        return roofline_plane(args, w, info, backup_ms, work, lane_peaks)
    pk = peaks()
    p = w.problem
    # the kernels' pairs: (input, disturbance point) pairs with a disturbance grid
    nx, nu = p.n_states, p.n_inputs * p.n_disturbances
    slots = info["window_slots"]
    esz = 8 if args.prec == "fp64" else 4  # stored masses and V in the arithmetic's width
    vbytes = 2 if args.v_store != "native" else esz
    per_state = vbytes + vbytes + 2 + 1  # V_{k+1} read once, V_k write, pi write, mask read
    if args.tmode in ("stored_full", "stored_factored"):
        per_pair = esz * (slots if args.tmode == "stored_full" else info["window_sum"]) + 2 * info["n"]
        algo = free * nu * per_pair + nx * per_state
        achieved = algo / (backup_ms / 1e3) / 1e9
        hbm = {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
               "frac": achieved / pk["hbm_gbs"], "traffic": measured_traffic(args, nx)[0],
               "peak_source": pk["source"], "algorithmic_bytes_per_launch": int(algo),
               "backup_kernel": info["backup_kernel"]}
        if args.prec != "fp64" or "fma_fp64" not in lane_peaks:
            return hbm
        # FP64: one fused multiply-add per (free state, input, slot) against the
        # measured FP64 FMA rate; the closer of the two ceilings is the bound
        fmas = free * nu * slots
        ach = fmas / (backup_ms / 1e3) / 1e12
        peak = lane_peaks["fma_fp64"] / 1e12
        alu = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "T FMA/s (FP64)", "frac": ach / peak,
               "traffic": hbm["traffic"], "peak_source": "measured on this GPU by amy_measure_fma (FP64)",
               "algorithmic_fmas_per_backup": int(fmas), "backup_kernel": info["backup_kernel"]}
        first, other = (alu, hbm) if alu["frac"] > hbm["frac"] else (hbm, alu)
        first["other_ceiling"] = {k: other[k] for k in ("bound", "achieved", "peak", "unit", "frac")}
        return first
    traffic, src = measured_traffic(args, nx)
    kern = info["backup_kernel"]
    gather = free * nu * slots
    if kern in (3, 4, 5):
        wm = max(info["window"])
        loads = (free * info["input_runs"] * info["inner_span"] * wm ** (info["n"] - 1)
                 + free * nu * info["window"][-1])
        path, what = ("shared", "K x W^(n-1) V values per (free state, input run) + the W innermost-dim "
                      "masses per (free state, input), read from shared memory")
    elif kern == 2:
        loads, path, what = gather, "shared", "one shared-memory load per (free state, input, slot)"
    elif kern == 9:
        loads, path, what = gather, "shared", ("one shared-memory load per (free state, input-disturbance "
                                               "pair, slot) from the block's bordered copy of V")
    else:
        loads, path, what = gather, "global_l1", "one global (L1) load per (free state, input, slot)"
    peak = lane_peaks[path] / 1e9
    achieved = loads / (backup_ms / 1e3) / 1e9
    lanes = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G lane-loads/s",
             "frac": achieved / peak, "traffic": traffic, "traffic_source": src,
             "peak_source": f"measured on this GPU by amy_measure_lane_loads ({path} path)",
             "algorithmic_lane_loads_per_backup": int(loads), "algorithmic_unit": what,
             "backup_kernel": kern,
             "window_slot_rate_vs_gather_ceiling": (gather / (backup_ms / 1e3) / 1e9) / peak}
    if args.prec != "fp64":
        # FP32: one fused multiply-add per (free state, input, slot) -- the
        # per-transition work of a kernel that sums every slot -- against the
        # measured FP32 FMA rate, reported beside the lane-load ceiling
        if "fma_fp32" in lane_peaks:
            ach = gather / (backup_ms / 1e3) / 1e12
            fpk = lane_peaks["fma_fp32"] / 1e12
            lanes["other_ceiling"] = {"bound": "alu", "achieved": ach, "peak": fpk, "unit": "T FMA/s (FP32)",
                                      "frac": ach / fpk}
        return with_erfc_ceiling(lanes, args, w, info, backup_ms, free, nu, lane_peaks)
    # FP64 on the fly: one FP64 fused multiply-add per (free state, input,
    # slot) against the measured FP64 FMA rate; the closer ceiling is the bound
    ach = gather / (backup_ms / 1e3) / 1e12
    fpk = lane_peaks["fma_fp64"] / 1e12
    alu = {"bound": "alu", "achieved": ach, "peak": fpk, "unit": "T FMA/s (FP64)", "frac": ach / fpk,
           "traffic": traffic, "peak_source": "measured on this GPU by amy_measure_fma (FP64)",
           "algorithmic_fmas_per_backup": int(gather), "backup_kernel": kern}
    first, other = (alu, lanes) if alu["frac"] > lanes["frac"] else (lanes, alu)
    first["other_ceiling"] = {k: other[k] for k in ("bound", "achieved", "peak", "unit", "frac")}
    return with_erfc_ceiling(first, args, w, info, backup_ms, free, nu, lane_peaks)


# ---------------------------------------------------------------------------
# the CPU oracle (baseline / reference arm)
# ---------------------------------------------------------------------------
def time_oracle(w, horizon: int):
    import oracle
    oracle.build_oracle()
    t0 = time.perf_counter()
    r = oracle.synthesize(w.problem, w.spec, horizon)
    return time.perf_counter() - t0, r


def time_oracle_sample(w, n_states: int, seed: int = W.SEED, nthreads: int = 0):
    """One backup of the oracle at n_states seeded states (rows computed in
    full) on nthreads host threads (0: all cores); returns (seconds,
    transitions)."""
    import oracle
    oracle.build_oracle()
    rng = np.random.default_rng(seed)
    st = rng.choice(w.problem.n_states, size=min(n_states, w.problem.n_states), replace=False)
    Vn = rng.uniform(0.0, 1.0, size=w.problem.n_states)
    t0 = time.perf_counter()
    oracle.backup_states(w.problem, w.spec, Vn, st, nthreads=nthreads)
    return time.perf_counter() - t0, len(st) * w.problem.n_inputs * w.problem.n_disturbances * window_slots_of(w)


# seeded states per oracle backup sample (full rows): all cores for the CPU
# baseline (about 10 s), one thread (a few seconds), one step of the
# reference arm (a few seconds, so that its warm-up and timed steps end
# within a few minutes)
ORACLE_SAMPLE = {"rooms7": 2000, "traffic6": 200_000}
ONE_CORE_SAMPLE = {"unicycle": 20000, "robot": 400, "rooms7": 200, "traffic6": 2000}
REFERENCE_SAMPLE = {"rooms7": 2000, "traffic6": 50_000}


def one_core_oracle(w, workload: str) -> dict:
    """The oracle on one host thread: one backup at a bounded sample of seeded
    states (a few seconds of work)."""
    n_s = ONE_CORE_SAMPLE.get(workload, 10)
    dt, tr = time_oracle_sample(w, n_s, nthreads=1)
    return {"value": tr / dt, "unit": UNIT, "cores": 1,
            "sample": f"one backup at {n_s} seeded states (full rows), FP64, one thread"}


def window_slots_of(w) -> int:
    import oracle
    Wd, _ = oracle.window_shape(w.problem)
    return int(np.prod(Wd))


def oracle_step(args, w):
    """One timed step of the oracle and its description: the whole workload
    where the oracle finishes it in seconds (robot, unicycle), else one
    backup at a bounded set of seeded states with full rows."""
    if args.workload in ("unicycle", "robot", "robot_dist"):
        slots = window_slots_of(w)
        trans = w.problem.n_states * w.problem.n_inputs * w.problem.n_disturbances * slots * w.horizon
        return (lambda: time_oracle(w, w.horizon)[0], trans,
                f"the whole workload per step (full grid, {w.horizon} backups), FP64")
    n_s = REFERENCE_SAMPLE.get(args.workload, 100)

    def run():
        return time_oracle_sample(w, n_s)[0]
    trans = min(n_s, w.problem.n_states) * w.problem.n_inputs * w.problem.n_disturbances * window_slots_of(w)
    return run, trans, f"one backup at {n_s} seeded states (full rows) per step, FP64"


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = workload(args)
    run, trans, sample = oracle_step(args, w)
    for _ in range(args.warmup):
        run()
    tot = sum(run() for _ in range(args.steps))
    value = trans * args.steps / tot
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload_name(args), "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# served stream: continuous batching vs the plain per-problem form
# ---------------------------------------------------------------------------
def run_served(args, rank, world):
    import threading

    import torch
    import paper_2005_06191_gb300 as amy
    from paper_2005_06191_gb300 import build as engine_build

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    engine_build.build()
    reqs = W.served_stream(args.served_n)
    trans = []
    for w in reqs:
        with amy.amy_build(w.problem, tmode="otf", prec="fp32") as h:
            trans.append(w.problem.n_states * w.problem.n_inputs * amy.amy_info(h)["window_slots"] * w.horizon)
    total_trans = float(sum(trans))

    def plain_one(w):
        # the plain form: build and synthesize one problem at a time (host outputs)
        with amy.amy_build(w.problem, tmode="auto", prec="fp32", device_mem_budget=4 << 30) as h:
            amy.amy_synthesize(h, w.spec, w.horizon)

    # closed loop: service rate of the plain form (warm)
    for w in reqs[:8]:
        plain_one(w)
    t0 = time.perf_counter()
    for w in reqs:
        plain_one(w)
    t_plain = time.perf_counter() - t0
    rate = len(reqs) / t_plain

    # closed loop with directly launched ticks, for comparison with the graphs
    srv_direct = amy.amy_server_create(batched=True, max_slots=64, use_graphs=False)
    tk = [amy.amy_submit(srv_direct, w) for w in reqs[:32]]
    for t in tk:
        amy.amy_wait(srv_direct, t)
    t0 = time.perf_counter()
    tk = [amy.amy_submit(srv_direct, w) for w in reqs]
    for t in tk:
        amy.amy_wait(srv_direct, t)
    t_direct = time.perf_counter() - t0
    srv_direct.close()

    srv = amy.amy_server_create(batched=True, max_slots=64)
    tk = [amy.amy_submit(srv, w) for w in reqs[:32]]  # warm: autotune the shape classes
    for t in tk:
        amy.amy_wait(srv, t)
    t0 = time.perf_counter()
    tk = [amy.amy_submit(srv, w) for w in reqs]
    res = [amy.amy_wait(srv, t) for t in tk]
    t_batched = time.perf_counter() - t0

    out = {}
    for mult in (0.5, 1.0, 2.0):
        arr = W.poisson_arrivals(len(reqs), rate * mult)
        # plain form, open loop
        lat = []
        base = time.perf_counter() + 0.01
        for i, w in enumerate(reqs):
            while time.perf_counter() < base + arr[i]:
                pass
            plain_one(w)
            lat.append(time.perf_counter() - (base + arr[i]))
        span_p = (base + arr[-1] + lat[-1]) - base
        # batched server, open loop: a submitter thread at the arrival times
        tickets = [None] * len(reqs)
        base = time.perf_counter() + 0.01

        def submitter():
            for i, w in enumerate(reqs):
                while time.perf_counter() < base + arr[i]:
                    pass
                tickets[i] = amy.amy_submit(srv, w)

        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        lat_b = []
        last = 0.0
        for i, t in enumerate(tickets):
            r = amy.amy_wait(srv, t)
            fin = r["finish_us"] * 1e-6
            lat_b.append(fin - (base + arr[i]))
            last = max(last, fin)
        span_b = last - base

        def pct(x, q):
            return float(np.percentile(np.asarray(x) * 1e3, q))

        out[f"{mult}x"] = {
            "arrival_rate_per_s": rate * mult,
            "batched": {"p50_ms": pct(lat_b, 50), "p99_ms": pct(lat_b, 99), "throughput": total_trans / span_b},
            "plain": {"p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "throughput": total_trans / span_p},
        }
    stats = amy.amy_server_stats(srv)
    stats.update(amy.amy_server_graph_stats(srv))
    srv.close()
    if rank != 0:
        return
    line = {
        "metric": "served p99 synthesis latency (ms), arrivals at the plain form's service rate",
        "value": out["1.0x"]["batched"]["p99_ms"], "unit": "ms", "n_gpus": world, "steps": 1,
        "warmup": 1, "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"served stream: {len(reqs)} seeded random linear problems (2-4 dims, "
                               "20^2-15^4 states, 4-16 inputs, gamma 1e-3, horizons 5-50), Poisson arrivals"},
        "closed_loop": {"plain_s": t_plain, "batched_s": t_batched, "batched_direct_ticks_s": t_direct,
                        "plain_throughput": total_trans / t_plain, "batched_throughput": total_trans / t_batched,
                        "batched_direct_ticks_throughput": total_trans / t_direct},
        "open_loop": out, "server_stats": stats, "transitions_total": total_trans,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 10 for the traffic ring, 400 for the unicycle, 50 otherwise)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="amy", choices=["amy", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=list(WORKLOADS) + ["served"])
    ap.add_argument("--tmode", default=None, choices=["otf", "stored_full", "stored_factored", "stored_separable"])
    ap.add_argument("--prec", default=None, choices=["fp64", "fp32", "fp32_kahan"])
    ap.add_argument("--served-n", dest="served_n", type=int, default=256)
    ap.add_argument("--v-store", dest="v_store", default="native", choices=["native", "u16", "bf16"])
    ap.add_argument("--step-wait", dest="step_wait", type=int, default=None, choices=[0, 1],
                    help="persistent kernel between backups: 0 = neighbour tiles, 1 = grid barrier "
                         "(default: the handle's choice, autotuned)")
    ap.add_argument("--plane", type=int, default=None, choices=[0, 1, 2],
                    help="banded problems with tables: 1 = the plane kernel (default where it applies), "
                         "2 = its tiled form where that applies, 0 = the per-state kernel")
    ap.add_argument("--plane-smem", dest="plane_smem", type=int, default=0,
                    help="shared memory per block of the plane kernel in bytes (0 = default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", dest="no_e2e", action="store_true",
                    help="skip the end-to-end (host buffer) measurement, e.g. under a profiler")
    ap.add_argument("--size", type=int, default=None,
                    help="grid points per dimension (x/y for the unicycle) instead of the workload's own")
    ap.add_argument("--horizon", type=int, default=None, help="horizon instead of the workload's own")
    ap.add_argument("--shape", default=None,
                    help="fixed backup launch shape 'lanes,states_per_block,rows(1)|consecutive(2),box_floats' "
                         "(0 = automatic) instead of the build-time autotuner")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.steps is None:
        args.steps = {"traffic6": 10, "unicycle": 400}.get(args.workload, 50)
    if args.workload != "served":
        args.tmode = args.tmode or WORKLOADS[args.workload][1]
        args.prec = args.prec or WORKLOADS[args.workload][2]
    rank, world = dist_setup(args.gpus)
    if args.workload == "served":
        run_served(args, rank, world)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    r = run_amy(args, rank, world)
    if rank != 0:
        return
    w = workload(args)
    cpu = None
    max_dv = None
    if not args.no_cpu_baseline:
        if args.workload in ("unicycle", "robot", "robot_dist"):
            dt, ref = time_oracle(w, w.horizon)
            cpu = {"value": r["trans"] / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"the whole workload once (full grid, {w.horizon} backups), FP64"}
            max_dv = float(np.max(np.abs(r["V"].astype(np.float64) - ref["V"])))
        else:
            n_s = ORACLE_SAMPLE.get(args.workload, 100)
            dt, tr = time_oracle_sample(w, n_s)
            cpu = {"value": tr / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"one backup at {n_s} seeded states (full rows), FP64"}
        cpu["one_core"] = one_core_oracle(w, args.workload)
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.prec == "fp64" else "f32",
        "data": "synthetic",
        "config": {"workload": workload_name(args), "tmode": args.tmode, "prec": args.prec,
                   "v_store": args.v_store,
                   "launch_shape": {"input_lanes": r["info"]["input_lanes"], "states_per_block": r["info"]["block_states"],
                                    "row_tiles": r["info"]["row_tiles"], "grouped_inputs": r["info"]["grouped_inputs"],
                                    "chosen_by": ("fixed: " + args.shape) if args.shape else
                                    "amy_build autotune (timed at build, outside the timed region)"},
                   "step_wait": ("grid barrier" if r["info"]["step_wait"] else "neighbour tiles")
                   if r["info"]["backup_kernel"] == 5 else None,
                   "l2": "flushed (256 MB write) between timed iterations",
                   "step": f"rebuild stored rows + spec mask + {w.horizon} fused backups (all pi_k written)"},
        "roofline": r["roofline"],
        "cpu_baseline": cpu,
        "e2e": r["e2e"],
        "e2e_cold": r["e2e_cold"],
        "gpu_launches": int(r["launches"]),
        "clocks": r["clocks"],
        "backup_kernel_ms": r["backup_ms"], "build_kernel_ms": r["build_ms"],
        "synth_only_value": r["synth_only_value"],
        "max_abs_dV_vs_oracle": max_dv,
        "e2e_V_equals_device_V": (None if r["V_e2e"] is None else bool(np.array_equal(r["V_e2e"], r["V"]))),
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
