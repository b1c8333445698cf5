#!/usr/bin/env python3
"""Benchmark of the difference-free conservative phase-field LBM step on GB300.

Prints ONE JSON line (rank 0). A "step" is one lattice update of the whole grid: one launch
of the fused difference-free kernel (the finite-difference variant, timed beside it, takes two
launches). The workload is the 3D static droplet: D3Q19, 128^3 periodic, R = 24, xi = 4,
sigma = 1e-3, density and viscosity ratio 1, tau_f = 0.8, M = 0.02, FP32 populations.

  value        MLUPS = cells x steps / (seconds x 1e6) over exactly --steps steps after --warmup
               untimed ones, populations resident in HBM, CUDA events on the stream the kernel
               runs on; whole-job aggregate over ranks
  roofline     algorithmic bytes per launch (2 x 2 x 19 x 4 B = 304 B per cell) / mean launch time,
               against the measured HBM copy bandwidth
  e2e          the same metric through the C ABI with host buffers: init from a pinned host phi0,
               the steps, and the result back to the host (the static-droplet diagnostics reduced
               on the device, and the mass), all inside the timed region; `fields` beside it reads
               the full FP64 fields back instead
  cpu_baseline the FP64 oracle on the host cores, all of them and one (bounded samples)
  detail       the other workloads (2D droplet, Rayleigh-Taylor, Taylor-Green, surrogate) and the
               GPU's errors against the oracle
  summary      last, so that it ends the line: the rest of the metric. The same step timed for
               at least a quarter second; the finite-difference variant and the ratio; 16-bit
               storage with its error against the oracle; the batched cases; spurious currents and
               the Laplace jump of both schemes after 5000 steps; the Rayleigh-Taylor tips. Every
               leg there is timed over at least a quarter second of device time.

--impl reference times the oracle alone (the reference arm of this metric). With --gpus N > 1
(launched by torchrun) every rank advances its own replica of the workload (the method needs no
exchange between independent replicas); rank 0 prints the aggregate over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import platform
import re
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

from paper_2407_12263_gb300 import inputs as I  # noqa: E402

METRIC = "MLUPS and % of HBM roofline, 1 GB300, vs same-GPU FD variant & FP32 at stated error"
WORKLOAD = "droplet3d_128"
# bytes per cell and step: the difference-free step reads and writes 19 (f, g) pairs; the
# finite-difference step adds a phi pass that reads the 19 pairs (f and g are interleaved, so g
# alone cannot be read for less) and writes phi, and reads phi in the step
BYTES_PER_CELL = {"df": 2 * 2 * 19 * 4, "fd": 2 * 2 * 19 * 4 + 2 * 19 * 4 + 4 + 4}
FD_METHOD_BYTES = 2 * 2 * 19 * 4 + 19 * 4 + 4 + 4  # the FD method's minimum with g readable alone
# 16-bit storage: the 8-byte zeroth-moment pair (FP32 sum f, fixed-point phi) plus 18 moving pairs
# of 2 x 16 bits, read and written
BYTES_PER_CELL_16 = 2 * (8 + 18 * 4)
PROFILE = ROOT / "profiles" / "step_kernel_droplet3d_128.md"
KERNEL_SOURCES = ["paper_2407_12263_gb300/csrc/cell.cuh", "paper_2407_12263_gb300/csrc/lattice.cuh",
                  "paper_2407_12263_gb300/csrc/step_kernels.cu", "paper_2407_12263_gb300/csrc/lbm_internal.h",
                  "paper_2407_12263_gb300/csrc/storage.cuh"]


# ---------------------------------------------------------------- multi-rank helpers (host logic)
def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(value: float, world: int) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate_mlups(cells: int, steps: int, seconds_max: float, world: int) -> float:
    """Whole-job MLUPS: every rank advanced its own `cells` for `steps`; time is the slowest rank's."""
    return cells * steps * world / (seconds_max * 1e6)


# ---------------------------------------------------------------- clocks
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.path = Path(tempfile.mkstemp(suffix=".csv")[1])
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        rows = [r.split(",") for r in self.path.read_text().strip().splitlines() if r.strip()]
        self.path.unlink(missing_ok=True)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, name in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- profile summary (traffic)
def strip_comments(src: str) -> str:
    """C/C++/CUDA source without its comments, whitespace runs collapsed to one space; string
    and character literals are kept as written."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            out.append(" ")
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_source_hash() -> str:
    """SHA-256 (first 16 hex digits) of the step kernel's sources with their comments removed:
    a change of code invalidates a profile taken before it, a change of comments does not."""
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        h.update(strip_comments((ROOT / rel).read_text()).encode())
        h.update(b"\0")
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the step kernel from the committed ncu summary, or None when the
    kernel sources changed since that capture."""
    if not PROFILE.exists():
        return None
    text = PROFILE.read_text()
    m_hash = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    m_traffic = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_traffic or m_hash.group(1) != kernel_source_hash():
        return None
    return float(m_traffic.group(1))


def measured_peak_hbm():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        return float(json.loads(p.read_text())["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def sig(x, n=4):
    """x rounded to n significant digits (None stays None)."""
    if x is None or not math.isfinite(x) or x == 0:
        return x
    return round(x, n - 1 - int(math.floor(math.log10(abs(x)))))


def hold_stream(torch, stream):
    """Keep `stream` busy for about half a millisecond (a bounded spin of torch's), so that the
    host has queued the timed launches before the start event is reached: the timed region then
    holds the steps, not the host's latency in issuing the first of them."""
    with torch.cuda.stream(stream):
        torch.cuda._sleep(1_000_000)


def time_region(torch, stream, step_fn, world):
    """Device seconds of step_fn on `stream` (CUDA events), barrier and synchronize on both
    sides, max over ranks."""
    torch.cuda.synchronize()
    barrier(world)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hold_stream(torch, stream)
    ev0.record(stream)
    step_fn()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    return max_over_ranks(ev0.elapsed_time(ev1) / 1e3, world)


LEGS = ("small2d", "rt", "batch", "tgv", "surrogate", "laplace", "accuracy")


def leg_warmup(warmup, graph_steps=32):
    """Warm-up steps of a leg other than the headline: at least --warmup, even, and at least one
    whole graph of the library's default graph_steps, so that the leg's timed region (an even
    count) starts from a buffer whose step graph is already captured."""
    return max(warmup + warmup % 2, graph_steps)


def long_steps(torch, stream, step, world, min_steps=2, target_s=0.25, cap=20000):
    """A step count whose timed region takes about target_s of device time (from 8 probe steps),
    at least min_steps, even, the same on every rank."""
    secs = time_region(torch, stream, lambda: step(8), world)
    n = int(math.ceil(target_s / max(secs / 8, 1e-7)))
    n = max(min_steps, min(cap, n))
    n += n % 2
    return int(max_over_ranks(float(n), world))


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl")
    torch.cuda.set_device(local)
    from paper_2407_12263_gb300 import build as cuda_build
    from paper_2407_12263_gb300 import lbm
    cuda_build.build()
    lbm.load()

    w = I.WORKLOADS[args.workload]
    grid = w["grid"]
    cells = grid[0] * grid[1] * grid[2]
    phi0 = I.droplet_phi(grid, w["R"], w["xi"])
    params = dict(tau_f=w["tau_f"], tau_g=w["tau_g"], M=w["M"], xi=w["xi"], sigma=w["sigma"],
                  rho_ratio=w["rho_ratio"], mu_ratio=w["mu_ratio"], body_force=w["body_force"])
    stream = torch.cuda.Stream()
    peak, peak_kind = measured_peak_hbm()

    def handle(scheme=0, storage=0, graph_steps=None):
        g = lbm.Lattice(grid, w["Q"], scheme=scheme, stream=stream.cuda_stream, storage=storage,
                        graph_steps=graph_steps, **params)
        g.init_phi(phi0)
        return g

    def long_leg(scheme, storage, bpc):
        """The step timed over at least a quarter second after --warmup steps."""
        g = handle(scheme, storage)
        m0 = g.mass()[0]
        g.step(leg_warmup(args.warmup))
        n = long_steps(torch, stream, g.step, world, min_steps=args.steps)
        n0 = g.launch_count
        secs = time_region(torch, stream, lambda: g.step(n), world)
        launches = g.launch_count - n0
        drift = g.mass()[0] - m0
        g.close()
        v = aggregate_mlups(cells, n, secs, world)
        return {"value": round(v, 1), "steps": n, "ms_per_step": round(secs / n * 1e3, 5), "launches": launches,
                "bytes_per_cell": bpc, "hbm_frac": round(bpc * cells / (secs / n) / 1e9 / peak, 4),
                "sum_phi_change": drift}

    # The finite-difference variant first: it also brings the GPU to its running clocks before the
    # headline's own timed region.
    fd = long_leg(1, 0, BYTES_PER_CELL["fd"])

    # the headline: exactly --warmup untimed steps, then exactly --steps timed steps, replayed
    # from a CUDA graph of gs steps captured and uploaded after the warm-up without running it
    gs = headline_graph_steps(args.steps)
    g = handle(graph_steps=gs)
    m0 = g.mass()[0]
    g.step(args.warmup)
    if gs:
        g.graph_prepare()      # the graph from the buffer the timed steps start from
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    n0 = g.launch_count
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hold_stream(torch, stream)
    ev0.record(stream)
    g.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = g.launch_count - n0
    t_df = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, world)
    clk = clocks.stop()
    drift = g.mass()[0] - m0
    g.close()
    value = aggregate_mlups(cells, args.steps, t_df, world)
    launch_s = t_df / args.steps  # one fused kernel per step
    achieved = BYTES_PER_CELL["df"] * cells / launch_s / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": profiled_traffic(),
                "peak_kind": peak_kind, "bytes_per_cell": BYTES_PER_CELL["df"],
                "kernel": "step_kernel<19, difference-free>"}

    df_long = long_leg(0, 0, BYTES_PER_CELL["df"])
    sixteen = {name: long_leg(0, st, BYTES_PER_CELL_16)
               for name, st in (("fp16", lbm.LBM_STORAGE_FP16), ("bf16", lbm.LBM_STORAGE_BF16))}

    e2e = run_e2e(lbm, torch, grid, w, params, phi0, cells, args, world)
    legs = set(args.legs.split(",")) if args.legs else set(LEGS)
    if args.no_surrogate:
        legs.discard("surrogate")
    small = run_small_2d(lbm, torch, stream, args, world) if "small2d" in legs else None
    rt = run_rayleigh_taylor(lbm, torch, stream, args, world) if "rt" in legs else None
    bubbles = run_batched_bubbles(lbm, torch, stream, args, world) if "batch" in legs else None
    tgv = run_taylor_green(lbm, torch, stream, args, world) if "tgv" in legs else None
    sg = run_surrogate(lbm, torch, stream, args, world) if "surrogate" in legs else None
    laplace = run_laplace(lbm, torch, stream, w, params, phi0) if "laplace" in legs else None

    out = {"metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(t_df / args.steps * 1e3, 5), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"{args.workload}: D3Q19 {grid[0]}x{grid[1]}x{grid[2]} periodic static droplet "
                                  f"R={w['R']:g} xi={w['xi']:g} sigma={w['sigma']:g}, density/viscosity ratio 1, "
                                  f"tau_f={w['tau_f']}, M={w['M']} (tau_phi=0.06), Courant 0.997",
                      "lattice": "D3Q19", "scheme": "difference-free", "storage": "fp32",
                      "l2": "working set 638 MB > 129 MB L2: no flush needed",
                      "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
           "gpu_launches": launches, "clocks": clk, "roofline": roofline, "e2e": e2e}
    detail = {"sum_phi_change": {"df": drift, "df_long": df_long["sum_phi_change"], "fd": fd["sum_phi_change"]},
              "droplet2d_64": small, "rayleigh_taylor_128x128x512": rt, "taylor_green_256": tgv,
              "batched_rising_bubbles": bubbles, "surrogate_taylor_green": sg}
    acc16 = rt_acc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and "accuracy" in legs:
        out["cpu_baseline"], detail["accuracy"] = run_cpu_baseline(lbm, grid, w, params, phi0, cells, args)
        rt_acc = run_rt_accuracy(lbm)
        detail["accuracy"]["rayleigh_taylor_32x32x128"] = rt_acc
        detail["accuracy"]["taylor_green_64"] = run_tgv_accuracy(lbm)
        acc16 = detail["accuracy"]
    out["detail"] = detail
    out["summary"] = summary(value, df_long, fd, sixteen, bubbles, laplace, acc16, rt_acc, tgv, rt, sg)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def headline_graph_steps(steps):
    """Steps per CUDA graph of the headline handle: the whole timed region when --steps is even
    and at most 64, else the largest even count up to 32 that divides --steps; 0 (direct
    launches) when there is none. The graph is captured and uploaded after the warm-up without
    running (lbm_graph_prepare), so the timed region replays it and nothing else."""
    if steps % 2 == 0 and 2 <= steps <= 64:
        return steps
    for gs in range(32, 1, -2):
        if steps % gs == 0:
            return gs
    return 0


def summary(value, df_long, fd, sixteen, bubbles, laplace, acc, rt_acc, tgv, rt, sg):
    """The rest of the metric, compact, to end the line: rates in MLUPS, fractions of the
    measured HBM copy bandwidth at each variant's own bytes per cell."""
    fd_method = fd["value"] * BYTES_PER_CELL["fd"] / FD_METHOD_BYTES  # FD at its method's 388 B, same efficiency
    s = {"df": {"value": sig(df_long["value"]), "steps": df_long["steps"], "hbm_frac": df_long["hbm_frac"]},
         "fd": {"value": sig(fd["value"]), "steps": fd["steps"], "hbm_frac": fd["hbm_frac"], "bytes": BYTES_PER_CELL["fd"]},
         "df_vs_fd": sig(df_long["value"] / fd["value"]),
         "df_vs_fd_if_fd_moved_388B": sig(df_long["value"] / fd_method),
         "headline_vs_long": sig(value / df_long["value"])}
    for name, leg in sixteen.items():
        e = {"value": sig(leg["value"]), "hbm_frac": leg["hbm_frac"], "vs_fp32": sig(leg["value"] / df_long["value"])}
        if acc:  # max |dphi| and rel-L2(du) against the oracle after acc[...]["steps"] steps
            e["err"] = [sig(acc[name]["max_abs_phi"], 2), sig(acc[name]["rel_l2_u"], 2)]
        s[name] = e
    if tgv:
        s["tgv256_fp16_vs_fp32"] = tgv["fp16_speedup_vs_fp32"]
    if rt:
        s["rt512_fp16_vs_fp32"] = rt["fp16"]["speedup_vs_fp32"]
    b = bubbles
    if b:
        s["batch"] = {"one_per_launch": sig(b["one_case_per_launch_fp32"]),
                      "group_only": sig(b["batched_fp32_group_launches_only"]["value"]),
                      "group_only_hbm_frac": b["batched_fp32_group_launches_only"]["hbm_frac"],
                      "fp32": sig(b["batched_fp32_default_tiles"]["value"]),
                      "fp32_tuned": sig(b["batched_fp32_tuned"]["value"]),
                      "auto_tuned": sig(b["batched_auto_tuned"]["value"]),
                      "x": [b[k]["speedup_vs_one_case_per_launch"] for k in
                            ("batched_fp32_default_tiles", "batched_fp32_tuned", "batched_auto_tuned")]}
    if laplace:
        s["droplet128_5000"] = laplace
    if rt_acc:
        s["rt_tips_2400"] = {k: sig(rt_acc[k]["tip_error_cells"], 2) for k in ("fp32", "fp16", "bf16")}
        s["rt_field_2400"] = {"fp32": [sig(rt_acc["fp32"]["max_abs_phi"], 2), sig(rt_acc["fp32"]["rel_l2_u"], 2)],
                              "fp64_twin": [sig(rt_acc["fp64_twin"]["max_abs_phi"], 2),
                                            sig(rt_acc["fp64_twin"]["rel_l2_u"], 2)]}
    if sg:
        a = sg["apply"]
        s["surrogate"] = {"accepted": a["accepted"], "x": a["speedup"], "shift": sig(a["interface_shift"], 3),
                          "limit": sig(a["interface_limit"], 3), "relax": sig(a["relax_ratio"], 3),
                          "relax_tol": sig(a["relax_tol"], 3), "projected": a["velocity_projected"],
                          "phi_err": [a["phi_l1_error"]["surrogate"], a["phi_l1_error"]["persistence"]],
                          "chain": {"accepted": [j["accepted"] for j in sg["chain"]["jumps"]],
                                    "x": sg["chain"]["speedup"],
                                    "phi_err": [sg["chain"]["phi_l1_error_end"], sg["chain"]["phi_l1_change_of_the_lbm"]]}}
    return s


def run_laplace(lbm, torch, stream, w, params, phi0):
    """The 3D droplet workload after 5000 steps in both schemes: the spurious currents (max |u|)
    and the Laplace jump (mean p inside r < R - 2 xi minus mean p outside r > R + 2 xi) against
    2 sigma / R_eff, R_eff from the volume of the phi = 0 phase."""
    grid, R, xi = w["grid"], w["R"], w["xi"]
    centre = tuple((n - 1) / 2 for n in grid)
    cells = grid[0] * grid[1] * grid[2]
    out = {"steps": w["steps"], "reduced_on": "device (lbm_diagnostics, lbm_mass)"}
    for name, scheme in (("df", 0), ("fd", 1)):
        g = lbm.Lattice(grid, w["Q"], scheme=scheme, stream=stream.cuda_stream, **params)
        g.init_phi(phi0)
        g.step(w["steps"])
        d = g.diagnostics(centre, R - 2 * xi, R + 2 * xi)
        sum_phi = g.mass()[0]
        g.close()
        jump = d["p_in"] - d["p_out"]
        r_eff = float(((cells - sum_phi) * 3 / (4 * np.pi)) ** (1 / 3))  # the volume of the phi = 0 phase
        want = 2 * w["sigma"] / r_eff
        out[name] = {"max_u": sig(d["max_speed"], 3), "jump": sig(jump), "2s_R": sig(want),
                     "rel": sig(jump / want - 1, 2)}
    return out


def run_small_2d(lbm, torch, stream, args, world):
    """The 2D droplet (D2Q9, 64^2, 4096 cells): 0.6 MB of state that stays in L2, so each step is
    a few microseconds of launch overhead and kernel; timed with CUDA graph replay (the default,
    32 steps per graph) and with one launch per step."""
    w = I.WORKLOADS["droplet2d_64"]
    phi0 = I.droplet_phi(w["grid"], w["R"], w["xi"])
    params = dict(tau_f=w["tau_f"], tau_g=w["tau_g"], M=w["M"], xi=w["xi"], sigma=w["sigma"])
    cells = w["grid"][0] * w["grid"][1]
    out = {"unit": "MLUPS", "steps": args.steps, "note": "L2-resident and launch-bound: no roofline claim"}
    for name, gsteps in (("graphs", 32), ("direct", 0)):
        g = lbm.Lattice(w["grid"], w["Q"], stream=stream.cuda_stream, graph_steps=gsteps, **params)
        g.init_phi(phi0)
        g.step(max(args.warmup, 64))
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        g.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        secs = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, world)
        out[name] = round(aggregate_mlups(cells, args.steps, secs, world), 1)
        out[name + "_us_per_step"] = round(secs / args.steps * 1e6, 3)
        g.close()
    return out


def rt_params(w):
    return dict(tau_f=w["tau_f"], tau_g=w["tau_g"], M=w["M"], xi=w["xi"], sigma=w["sigma"],
                rho_ratio=w["rho_ratio"], mu_ratio=w["mu_ratio"], body_force=w["body_force"])


def run_rayleigh_taylor(lbm, torch, stream, args, world):
    """The Rayleigh-Taylor workload at full size (D3Q19, 128 x 128 x 512, walls in z, density
    ratio 3, gravity): the general step kernel (body force, density ratio, walls) in FP32, FP16
    and BF16 storage, device-timed over at least a quarter second from the initial interface."""
    w = I.WORKLOADS["rayleigh_taylor_128x128x512"]
    grid = w["grid"]
    cells = grid[0] * grid[1] * grid[2]
    phi0 = I.rayleigh_taylor_phi(grid, w["amplitude"], w["xi"])
    peak = measured_peak_hbm()[0]
    out = {"unit": "MLUPS", "warmup": leg_warmup(args.warmup),
           "config": f"D3Q19 {grid[0]}x{grid[1]}x{grid[2]}, walls in z, At=0.5 (rho1/rho2=3), Re=256, "
                     f"U=sqrt(gW)=0.04, Ca=1, cosine perturbation 0.05W, xi={w['xi']:g}"}
    fp32 = None
    for name, storage, bpc in (("fp32", 0, BYTES_PER_CELL["df"]), ("fp16", lbm.LBM_STORAGE_FP16, BYTES_PER_CELL_16),
                               ("bf16", lbm.LBM_STORAGE_BF16, BYTES_PER_CELL_16)):
        g = lbm.Lattice(grid, 19, stream=stream.cuda_stream, storage=storage, walls=w["walls"], **rt_params(w))
        g.init_phi(phi0)
        m0 = g.mass()[0]
        g.step(leg_warmup(args.warmup))
        steps = long_steps(torch, stream, g.step, world)
        secs = time_region(torch, stream, lambda: g.step(steps), world)
        m1 = g.mass()[0]
        g.close()
        v = aggregate_mlups(cells, steps, secs, world)
        fp32 = fp32 or v
        out[name] = {"value": round(v, 1), "steps": steps, "ms_per_step": round(secs / steps * 1e3, 5),
                     "bytes_per_cell": bpc, "hbm_frac": round(bpc * cells / (secs / steps) / 1e9 / peak, 4),
                     "speedup_vs_fp32": round(v / fp32, 4), "sum_phi_change": m1 - m0}
    return out


def tgv_fields(w):
    grid = w["grid"]
    return (I.droplet_phi(grid, w["R"], w["xi"]), I.taylor_green_velocity(grid, w["u0"]),
            I.taylor_green_pressure(grid, w["u0"]))


def run_taylor_green(lbm, torch, stream, args, world):
    """Droplet breakup in a Taylor-Green vortex at 256^3 (periodic, u0 = 0.04, Re = 1000, We = 20,
    R = 32, initial pressure field): the difference-free step in FP16 storage (the workload's)
    and FP32, device-timed over at least a quarter second."""
    w = I.WORKLOADS["taylor_green_256"]
    grid = w["grid"]
    cells = grid[0] * grid[1] * grid[2]
    phi0, u0, p = tgv_fields(w)
    peak = measured_peak_hbm()[0]
    out = {"unit": "MLUPS", "warmup": leg_warmup(args.warmup),
           "config": "D3Q19 256^3 periodic, u0=0.04, Re=1000, We=20, droplet R=32 at the centre, xi=4, "
                     "Taylor-Green pressure field, arguments 2 pi x / 256"}
    for name, storage, bpc in (("fp16", lbm.LBM_STORAGE_FP16, BYTES_PER_CELL_16), ("fp32", 0, BYTES_PER_CELL["df"])):
        g = lbm.Lattice(grid, 19, stream=stream.cuda_stream, storage=storage, tau_f=w["tau_f"], tau_g=w["tau_g"],
                        M=w["M"], xi=w["xi"], sigma=w["sigma"])
        g.init_phi(phi0, u0, p=p)
        m0 = g.mass()[0]
        g.step(leg_warmup(args.warmup))
        steps = long_steps(torch, stream, g.step, world)
        secs = time_region(torch, stream, lambda: g.step(steps), world)
        m1 = g.mass()[0]
        g.close()
        v = aggregate_mlups(cells, steps, secs, world)
        out[name] = {"value": round(v, 1), "steps": steps, "ms_per_step": round(secs / steps * 1e3, 5),
                     "bytes_per_cell": bpc, "hbm_frac": round(bpc * cells / (secs / steps) / 1e9 / peak, 4),
                     "sum_phi_change": m1 - m0}
    out["fp16_speedup_vs_fp32"] = round(out["fp16"]["value"] / out["fp32"]["value"], 4)
    return out


def tgv_case(n, u0, R, We, Re=1000.0, xi=4.0, M=0.02):
    eta = u0 * n / Re
    return dict(grid=(n, n, n), u0=u0, R=R, xi=xi, sigma=u0 * u0 * 2 * R / We, tau_f=3 * eta, tau_g=0.8, M=M)


def tgv_lattice(lbm, c, stream, storage):
    g = lbm.Lattice(c["grid"], 19, tau_f=c["tau_f"], tau_g=c["tau_g"], M=c["M"], xi=c["xi"], sigma=c["sigma"],
                    stream=stream.cuda_stream, storage=storage)
    g.init_phi(I.droplet_phi(c["grid"], c["R"], c["xi"]), I.taylor_green_velocity(c["grid"], c["u0"]),
               p=I.taylor_green_pressure(c["grid"], c["u0"]))
    return g


def run_surrogate(lbm, torch, stream, args, world):
    """run_surrogate_on_stream on a torch stream of its own, which the network shares with the
    torch kernels that build its inputs (torch's default stream has the handle 0, which the
    network would read as "make a stream of your own")."""
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        out = run_surrogate_on_stream(lbm, torch, stream, args, world)
    s.synchronize()
    return out


def run_surrogate_on_stream(lbm, torch, stream, args, world):
    """The convolutional surrogate on the Taylor-Green breakup case: trained on 128^3 trajectories
    of this solver (FP16 storage, Re = 1000, seeded u0 in [0.03, 0.05], We in [10, 30], R in
    [12, 20]; pairs 100 steps apart coarsened 2x to 64^3), then applied to the 256^3 workload
    (coarsened 4x to 64^3; k = 200 steps, the same jump in units of L0 / u0) with the LBM as judge.
    The jump replaces the predicted velocity by its divergence-free part before the restart.
    Reported beside 200 LBM steps: wall time, and the coarse phi and u errors against the LBM's
    own state, with persistence (the starting state) as the reference."""
    # training trajectories on the workload's own grid (f = 4, k = 200) or on a 128^3 copy (f = 2,
    # k = 100, the same jump in units of L0 / u0 and the same coarse grid)
    n_train = args.surrogate_train_grid
    f_train, k_train = (4, 200) if n_train == 256 else (2, 100)
    rng = np.random.default_rng(12263)
    coarse = lambda g, f: _coarse_fields(lbm, torch, g, f)
    t0 = time.perf_counter()
    xs, ys = [], []
    for s in range(6):
        c = tgv_case(n_train, rng.uniform(0.03, 0.05), rng.uniform(12.0, 20.0) * n_train / 128, rng.uniform(10.0, 30.0))
        g = tgv_lattice(lbm, c, stream, lbm.LBM_STORAGE_FP16)
        prev = coarse(g, f_train)
        for _ in range(30):
            g.step(k_train)
            cur = coarse(g, f_train)
            xs.append(prev)
            ys.append(cur)
            prev = cur
        g.close()
    X, Y = torch.stack(xs), torch.stack(ys)
    mean = X.mean(dim=(0, 2, 3, 4))
    std = X.std(dim=(0, 2, 3, 4)) + 1e-12
    norm = lambda a: ((a - mean[:, None, None, None]) / std[:, None, None, None]).contiguous()
    Xn, Yn = norm(X), norm(Y)
    t_data = time.perf_counter() - t0
    # the network runs on torch's current stream, which also builds its input batches
    net = lbm.Net(fp16=True, seed=7, stream=torch.cuda.current_stream().cuda_stream)
    grid_c = tuple(int(v) for v in X.shape[2:][::-1])
    gen = torch.Generator(device="cpu").manual_seed(0)
    iters, batch = args.surrogate_iters, 4
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    first = last = None
    for it in range(iters):
        idx = torch.randint(0, X.shape[0], (batch,), generator=gen)
        xb, yb = Xn[idx].contiguous(), Yn[idx].contiguous()
        last = net.gradients(xb.data_ptr(), yb.data_ptr(), batch, grid_c)
        first = last if first is None else first
        net.adam(1e-3 if it < (2 * iters) // 3 else 3e-4)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del X, Y, Xn, Yn
    # the 256^3 workload
    w = I.WORKLOADS["taylor_green_256"]
    c = tgv_case(256, w["u0"], w["R"], 20.0)
    k, f, judge_steps = 200, 4, 8
    truth = tgv_lattice(lbm, c, stream, lbm.LBM_STORAGE_FP16)
    jumper = tgv_lattice(lbm, c, stream, lbm.LBM_STORAGE_FP16)
    for h in (truth, jumper):
        h.step(1600)
    t0 = time.perf_counter()
    lbm.lbm_surrogate_reserve(jumper.h, f)  # the jump's workspace, allocated once per handle
    t_reserve = time.perf_counter() - t0
    x0 = coarse(jumper, f)
    s0 = jumper.mass()[0]
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    truth.step(k)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_lbm = ev0.elapsed_time(ev1) / 1e3
    xt = coarse(truth, f)
    # the LBM's own interface displacement over the k steps, measured as the judge measures it
    gphi = torch.stack([0.5 * (torch.roll(x0[0], -1, a) - torch.roll(x0[0], 1, a)) for a in range(3)])
    shift_true = f * float((xt[0] - x0[0]).abs().sum()) / float(gphi.pow(2).sum(0).sqrt().sum())
    ms = torch.cat([mean, std]).cpu().numpy().tolist()
    # judge: mass within 1%; the kinematic interface bound (interface_tol = 1); and phi may move
    # at most twice as fast after the restart from the prediction as after the same restart from
    # the starting state (relax_tol = 2)
    relax_tol = 2.0
    rep = lbm.lbm_surrogate_jump(jumper.h, net, f, ms, k, judge_steps, 1e-2, relax_tol, 1.0)
    t_jump = rep["seconds"]
    # the prediction itself, for its error (the jumper now holds it advanced by the judge's steps)
    xin = norm(x0)[None].contiguous()
    y = torch.empty_like(xin)
    net.forward(xin.data_ptr(), y.data_ptr(), 1, tuple(int(v) for v in x0.shape[1:][::-1]))
    pred = y[0] * std[:, None, None, None] + mean[:, None, None, None]
    # the velocity the lattice restarts from: the prediction's divergence-free part
    pred_p = pred.clone().contiguous()
    grid_c = tuple(int(v) for v in x0.shape[1:][::-1])
    wb = lbm.lbm_project_workspace_bytes(grid_c)
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    if lbm.lbm_project_solenoidal(pred_p.data_ptr() + pred_p[0].numel() * 4, grid_c, work.data_ptr(), wb,
                                  torch.cuda.current_stream().cuda_stream) != lbm.LBM_OK:
        raise RuntimeError("lbm_project_solenoidal failed")
    torch.cuda.synchronize()
    err = lambda a, chans: float(sum((a[ch] - xt[ch]).abs().mean() for ch in chans))
    out = {"train": {"grid": [n_train] * 3, "trajectories": 6, "pairs": len(xs), "k": k_train, "factor": f_train,
                     "iterations": iters, "batch": batch, "loss_first": sig(first), "loss_last": sig(last),
                     "seconds_data": round(t_data, 2), "seconds_train": round(t_train, 2)},
           "apply": {"grid": [256] * 3, "storage": "fp16", "start_step": 1600, "k": k, "factor": f,
                     "judge_steps": judge_steps, "accepted": rep["accepted"],
                     "velocity_projected": rep["projected"],
                     "mass_error_of_prediction": sig(rep["mass_error"], 3),
                     "interface_shift": rep["interface_shift"], "interface_limit": rep["interface_limit"],
                     "interface_shift_of_the_lbm": sig(shift_true, 3),
                     "relax_ratio": rep["relax_ratio"], "relax_tol": relax_tol, "seconds_jump": round(t_jump, 5),
                     "seconds_workspace_reserve": round(t_reserve, 5),
                     "seconds_lbm_k_steps": round(t_lbm, 5), "speedup": round(t_lbm / t_jump, 3),
                     "phi_l1_error": {"surrogate": sig(err(pred, [0]), 3), "persistence": sig(err(x0, [0]), 3)},
                     "u_l1_error": {"surrogate": sig(err(pred_p, [1, 2, 3]), 3),
                                    "surrogate_unprojected": sig(err(pred, [1, 2, 3]), 3),
                                    "persistence": sig(err(x0, [1, 2, 3]), 3)},
                     "sum_phi_change": jumper.mass()[0] - s0}}
    # a chain: two more judged jumps of k steps from where the first one left the lattice, the
    # LBM's own trajectory advanced to the same times beside it
    t_now = 1600 + k + (judge_steps if rep["accepted"] else 0)
    truth.step(t_now - (1600 + k))
    jumps, secs_jumps, secs_lbm = [dict(accepted=rep["accepted"], relax=sig(rep["relax_ratio"], 3))], t_jump, 0.0
    secs_lbm += t_lbm * (t_now - 1600) / k
    for _ in range(2):
        r = lbm.lbm_surrogate_jump(jumper.h, net, f, ms, k, judge_steps, 1e-2, relax_tol, 1.0)
        dt = k + (judge_steps if r["accepted"] else 0)
        ev0.record(stream)
        truth.step(dt)
        ev1.record(stream)
        torch.cuda.synchronize()
        secs_lbm += ev0.elapsed_time(ev1) / 1e3
        secs_jumps += r["seconds"]
        t_now += dt
        jumps.append(dict(accepted=r["accepted"], relax=sig(r["relax_ratio"], 3),
                          shift=sig(r["interface_shift"], 3)))
    xe, xt_end = coarse(jumper, f), coarse(truth, f)
    out["chain"] = {"jumps": jumps, "start_step": 1600, "end_step": t_now,
                    "seconds_jumps": round(secs_jumps, 5), "seconds_lbm_same_steps": round(secs_lbm, 5),
                    "speedup": round(secs_lbm / secs_jumps, 3),
                    "phi_l1_error_end": sig(float((xe[0] - xt_end[0]).abs().mean()), 3),
                    "phi_l1_change_of_the_lbm": sig(float((xt_end[0] - x0[0]).abs().mean()), 3),
                    "sum_phi_change": jumper.mass()[0] - s0}
    truth.close()
    jumper.close()
    net.close()
    return out


def _coarse_fields(lbm, torch, g, f):
    n = g.grid
    out = torch.empty((5, n[2] // f, n[1] // f, n[0] // f), device="cuda")
    torch.cuda.synchronize()
    lbm.lbm_coarse_fields(g.h, f, out.data_ptr())
    torch.cuda.synchronize()  # the lattice's stream wrote it; torch reads it on its own
    return out


def run_tgv_accuracy(lbm):
    """The 64^3 copy of the Taylor-Green breakup case after 200 steps against the FP64 oracle."""
    import oracle
    w = I.WORKLOADS["taylor_green_64"]
    phi0, u0, p = tgv_fields(w)
    params = dict(tau_f=w["tau_f"], tau_g=w["tau_g"], M=w["M"], xi=w["xi"], sigma=w["sigma"])
    ref = oracle.Oracle(19, w["grid"], **params)
    ref.init_phi(phi0, u0, p=p)
    ref.step(200)
    phi_o, p_o, u_o = ref.moments()
    out = {"steps": 200}
    for name, storage in (("fp32", 0), ("fp16", lbm.LBM_STORAGE_FP16), ("bf16", lbm.LBM_STORAGE_BF16)):
        g = lbm.Lattice(w["grid"], 19, storage=storage, **params)
        g.init_phi(phi0, u0, p=p)
        g.step(200)
        phi_g, p_g, u_g = g.moments()
        g.close()
        out[name] = {"max_abs_phi": float(np.abs(phi_g - phi_o).max()),
                     "rel_l2_u": float(np.linalg.norm(u_g - u_o) / np.linalg.norm(u_o)),
                     "max_abs_p": float(np.abs(p_g - p_o).max())}
    return out


CASE_KEYS = ("grid", "lattice", "tau_f", "tau_g", "M", "xi", "sigma", "rho_ratio", "mu_ratio", "body_force", "walls")


def run_batched_bubbles(lbm, torch, stream, args, world):
    """256 seeded rising-bubble boxes of uneven size (D3Q19, walls on every side, density ratio
    2-10, viscosity ratio 1-10, Eo 1-50, Mo 1e-5..1e-1): aggregate MLUPS of one handle per case
    (FP32, each case's steps launched on its own, graph-replayed, one stream) against the batch
    (group launches per size class and dedicated launches on concurrent branches, graph-replayed)
    untuned, tuned in form and tile, and tuned in form, tile and storage. Every arm is timed over
    the same step count, chosen so that the slowest arm takes at least a quarter second."""
    cases = I.rising_bubble_cases()[:args.batch_cases]
    cells = sum(int(np.prod(c["grid"])) for c in cases)
    out = {"cases": len(cases), "cells": cells, "warmup": leg_warmup(args.warmup), "unit": "MLUPS",
           "config": f"rising_bubble_cases(n=256, seed=12263)[:{len(cases)}]: widths {{32,48,64,96}} x height "
                     "{1,2}, R = width/8, walls on all sides, gravity -z"}

    # one handle per case, FP32
    singles = []
    for c in cases:
        h = lbm.Lattice(c["grid"], 19, **{k: c[k] for k in CASE_KEYS[2:]}, stream=stream.cuda_stream)
        h.init_phi(I.bubble_phi(c))
        singles.append(h)
    for h in singles:
        h.step(leg_warmup(args.warmup))
    steps = long_steps(torch, stream, lambda n: [h.step(n) for h in singles], world)
    out["steps"] = steps
    secs = time_region(torch, stream, lambda: [h.step(steps) for h in singles], world)
    out["one_case_per_launch_fp32"] = round(aggregate_mlups(cells, steps, secs, world), 1)
    out["one_case_per_launch_launches_per_step"] = len(cases)
    for h in singles:
        h.close()
    del singles

    def batched(storage, tune, group_only=False):
        structs = [lbm.make_case(**{k: c[k] for k in CASE_KEYS}, storage=storage) for c in cases]
        b = lbm.Batch(structs, stream=stream.cuda_stream)
        if tune:
            b.tune(trial_steps=5)
        if group_only:  # every case in group launches of its default tile
            for k in range(len(cases)):
                b.set_config(k, b.config(k)[0], dedicated=False)
        for k, c in enumerate(cases):
            b.case(k).init_phi(I.bubble_phi(c))
        m0 = [b.case(k).mass()[0] for k in range(len(cases))]
        b.step(leg_warmup(args.warmup))
        n0 = b.launch_count
        secs = time_region(torch, stream, lambda: b.step(steps), world)
        launches = b.launch_count - n0
        nonfinite, changed = 0, 0
        for k in range(len(cases)):
            try:
                if b.case(k).mass()[0] != m0[k]:
                    changed += 1
            except lbm.LBMError:
                nonfinite += 1
        forms = {}
        for k, c in enumerate(cases):
            tile, st, ded = b.config(k)
            key = ("dedicated" if ded else "group") + "_" + ["fp32", "fp16", "bf16"][st]
            forms[key] = forms.get(key, 0) + 1
        b.close()
        return {"value": round(aggregate_mlups(cells, steps, secs, world), 1), "launches_per_step": launches / steps,
                "cases_by_form": forms, "nonfinite_cases": nonfinite, "sum_phi_changed_cases": changed}

    out["batched_fp32_group_launches_only"] = batched(lbm.LBM_STORAGE_FP32, False, group_only=True)
    out["batched_fp32_default_tiles"] = batched(lbm.LBM_STORAGE_FP32, False)
    out["batched_fp32_tuned"] = batched(lbm.LBM_STORAGE_FP32, True)
    out["batched_auto_tuned"] = batched(lbm.LBM_STORAGE_AUTO, True)
    base = out["one_case_per_launch_fp32"]
    peak = measured_peak_hbm()[0]
    out["one_case_per_launch_hbm_frac"] = round(base * 1e6 * BYTES_PER_CELL["df"] / 1e9 / peak, 4)
    for key in ("batched_fp32_group_launches_only", "batched_fp32_default_tiles", "batched_fp32_tuned",
                "batched_auto_tuned"):
        out[key]["speedup_vs_one_case_per_launch"] = round(out[key]["value"] / base, 4)
    for key in ("batched_fp32_group_launches_only", "batched_fp32_default_tiles", "batched_fp32_tuned"):
        out[key]["hbm_frac"] = round(out[key]["value"] * 1e6 * BYTES_PER_CELL["df"] / 1e9 / peak, 4)
    return out


def run_rt_accuracy(lbm):
    """Interface tips of the 32 x 32 x 128 copy of the Rayleigh-Taylor workload after 2400 steps
    (3 time units W/U) against the FP64 oracle: bubble tip (column x = y = 0) and spike tip
    (x = W/2, y = 0), and the field errors."""
    import oracle
    w = I.WORKLOADS["rayleigh_taylor_32x32x128"]
    grid, steps = w["grid"], 2400
    phi0 = I.rayleigh_taylor_phi(grid, w["amplitude"], w["xi"])
    tips = lambda phi: [I.interface_height(phi[:, 0, 0]), I.interface_height(phi[:, 0, grid[0] // 2])]
    ref = oracle.Oracle(19, grid, walls=w["walls"], **rt_params(w))
    ref.init_phi(phi0)
    # the oracle's own sensitivity: an FP64 twin started from the same state perturbed by
    # FP32-sized relative noise (3e-8)
    twin = oracle.Oracle(19, grid, walls=w["walls"], **rt_params(w))
    f, g = ref.get_pops()
    rng = np.random.default_rng(2400)
    twin.set_pops(f * (1 + 3e-8 * rng.standard_normal(f.shape)), g * (1 + 3e-8 * rng.standard_normal(g.shape)))
    t0 = time.perf_counter()
    ref.step(steps)
    secs = time.perf_counter() - t0
    twin.step(steps)
    phi_o, p_o, u_o = ref.moments()
    phi_t, _, u_t = twin.moments()
    out = {"steps": steps, "initial_tips": tips(phi0), "oracle_tips": tips(phi_o),
           "oracle_seconds": round(secs, 1),
           "fp64_twin": {"max_abs_phi": float(np.abs(phi_t - phi_o).max()),
                         "rel_l2_u": float(np.linalg.norm(u_t - u_o) / np.linalg.norm(u_o)),
                         "tip_error_cells": float(np.abs(np.subtract(tips(phi_t), tips(phi_o))).max())}}
    for name, storage in (("fp32", 0), ("fp16", lbm.LBM_STORAGE_FP16), ("bf16", lbm.LBM_STORAGE_BF16)):
        g = lbm.Lattice(grid, 19, storage=storage, walls=w["walls"], **rt_params(w))
        g.init_phi(phi0)
        g.step(steps)
        phi_g, p_g, u_g = g.moments()
        g.close()
        out[name] = {"tip_error_cells": float(np.abs(np.subtract(tips(phi_g), tips(phi_o))).max()),
                     "max_abs_phi": float(np.abs(phi_g - phi_o).max()),
                     "rel_l2_u": float(np.linalg.norm(u_g - u_o) / np.linalg.norm(u_o))}
    return out


def run_e2e(lbm, torch, grid, w, params, phi0, cells, args, world):
    """Through the C ABI with host buffers, each region: pinned phi0 in, the steps, the result out.
    The result is the workload's metric, the static-droplet checks of Sec. 3.1 as lbm_diagnostics
    reduces them on the device (largest |u|, the mean pressure inside r < R - 2 xi and outside
    r > R + 2 xi, the kinetic energy) and sum phi and sum rho phi from lbm_mass: 80 bytes. The
    same region reading the full fields back (phi, p, u as FP64 through lbm_moments, 84 MB at
    128^3) is reported beside it as `fields`."""
    shape = phi0.shape
    pin = lambda n: torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    phi_h = pin(phi0.size).reshape(shape)
    phi_h[...] = phi0
    phi_o, p_o, u_o = pin(phi0.size).reshape(shape), pin(phi0.size).reshape(shape), pin(3 * phi0.size).reshape((3,) + shape)
    centre = tuple((n - 1) / 2 for n in grid)
    r_in, r_out = w["R"] - 2 * w["xi"], w["R"] + 2 * w["xi"]
    g = lbm.Lattice(grid, w["Q"], **params)
    g.init_phi(phi_h)                 # warm the handle (staging allocation, module load)
    g.step(args.warmup)
    lbm.lbm_moments(g.h, phi_o, p_o, u_o)
    g.diagnostics(centre, r_in, r_out)

    def region(read_fields):
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.init_phi(phi_h)
        g.step(args.steps)
        if read_fields:
            lbm.lbm_moments(g.h, phi_o, p_o, u_o)
            d = None
        else:
            d = g.diagnostics(centre, r_in, r_out)
        s = g.mass()
        t1 = time.perf_counter()
        return max_over_ranks(t1 - t0, world), d, s

    secs, d, s = region(False)
    secs_f, _, _ = region(True)
    g.close()
    h2d = phi0.size * 8
    d2h_metric = 7 * 8 + 3 * 8          # lbm_diag's seven 8-byte members, lbm_mass's three doubles
    d2h_fields = 5 * phi0.size * 8 + 3 * 8
    return {"value": round(aggregate_mlups(cells, args.steps, secs, world), 1), "unit": "MLUPS",
            "h2d_bytes_per_step": round(h2d / args.steps, 1), "d2h_bytes_per_step": round(d2h_metric / args.steps, 1),
            "seconds": round(secs, 4), "result": "lbm_diagnostics + lbm_mass",
            "max_u": sig(d["max_speed"], 3), "laplace_jump": sig(d["p_in"] - d["p_out"]), "sum_phi": s[0],
            "fields": {"value": round(aggregate_mlups(cells, args.steps, secs_f, world), 1), "unit": "MLUPS",
                       "h2d_bytes_per_step": round(h2d / args.steps, 1),
                       "d2h_bytes_per_step": round(d2h_fields / args.steps, 1), "seconds": round(secs_f, 4),
                       "result": "lbm_moments (phi, p, u as FP64) + lbm_mass"}}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


def run_cpu_baseline(lbm, grid, w, params, phi0, cells, args):
    """The FP64 oracle on the host cores over full-grid steps of the workload: all cores (bounded
    to about args.cpu_seconds) and one thread (one step); and the GPU's error against it after
    the same steps."""
    import oracle
    oracle.build()
    cores = oracle.num_threads()
    ref = oracle.Oracle(w["Q"], grid, **params)
    ref.init_phi(phi0)
    t0 = time.perf_counter()
    ref.step(1)
    one = time.perf_counter() - t0
    oracle.set_num_threads(1)
    t0 = time.perf_counter()
    ref.step(1)
    single = time.perf_counter() - t0
    oracle.set_num_threads(cores)
    k = max(1, min(50, int(args.cpu_seconds / max(one, 1e-3)) - 2))
    t0 = time.perf_counter()
    ref.step(k)
    secs = time.perf_counter() - t0
    n = k + 2
    cpu = {"value": round(cells * k / secs / 1e6, 3), "unit": "MLUPS", "cores": cores,
           "kind": "oracle", "sample": f"{k} full-grid steps of {WORKLOAD} (FP64 C, OpenMP over rows), "
                                       f"{secs:.1f} s; one thread: 1 step, {single:.1f} s",
           "one_thread": round(cells / single / 1e6, 4), "cpu_model": cpu_model(), "nproc": os.cpu_count()}
    phi_o, p_o, u_o = ref.moments()
    acc = {}
    bounds = {"fp32": {"max_abs_phi": 1e-4, "rel_l2_u": 1e-3, "sum_phi_drift": 0.0},
              "fp16": {"max_abs_phi": 1e-3, "rel_l2_u": 1e-2, "sum_phi_drift": 0.0},
              "bf16": {"max_abs_phi": 1e-2, "rel_l2_u": 3e-2, "sum_phi_drift": 0.0}}
    for name, storage in (("fp32", 0), ("fp16", lbm.LBM_STORAGE_FP16), ("bf16", lbm.LBM_STORAGE_BF16)):
        g = lbm.Lattice(grid, w["Q"], storage=storage, **params)
        g.init_phi(phi0)
        g.step(n)
        phi_g, p_g, u_g = g.moments()
        g.close()
        acc[name] = {"steps": n, "max_abs_phi": float(np.abs(phi_g - phi_o).max()),
                     "rel_l2_u": float(np.linalg.norm(u_g - u_o) / np.linalg.norm(u_o)),
                     "max_abs_u": float(np.abs(u_g - u_o).max()),
                     "max_abs_p": float(np.abs(p_g - p_o).max()), "bounds": bounds[name]}
    cpu["droplet2d_64"] = run_cpu_droplet2d(oracle, cores)
    return cpu, acc


def run_cpu_droplet2d(oracle, cores):
    """The 2D static droplet (D2Q9, 64^2, R = 16, 5000 steps) on the FP64 oracle, all steps on
    the host cores: its time, and Laplace's law (mean p over r < R - 2 xi minus mean p over
    r > R + 2 xi against sigma / R_eff, R_eff from the area of the phi = 0 phase) and the drift
    of sum phi at the end."""
    w = I.WORKLOADS["droplet2d_64"]
    grid = w["grid"]
    ref = oracle.Oracle(9, grid, w["tau_f"], w["tau_g"], w["M"], w["xi"], w["sigma"])
    phi0 = I.droplet_phi(grid, w["R"], w["xi"])
    ref.init_phi(phi0)
    s0 = math.fsum(ref.moments()[0].ravel())  # correctly rounded sums: the drift is the scheme's own
    t0 = time.perf_counter()
    ref.step(w["steps"])
    secs = time.perf_counter() - t0
    phi, p, u = ref.moments()
    r = I.periodic_distance(grid, tuple((n - 1) / 2 for n in grid))
    jump = float(p[r < w["R"] - 2 * w["xi"]].mean() - p[r > w["R"] + 2 * w["xi"]].mean())
    r_eff = float(np.sqrt((1 - phi).sum() / np.pi))
    want = w["sigma"] / r_eff
    cells = grid[0] * grid[1] * grid[2]
    return {"steps": w["steps"], "seconds": round(secs, 3), "mlups": round(cells * w["steps"] / secs / 1e6, 3),
            "cores": cores, "laplace_jump": sig(jump), "sigma_over_R": sig(want), "rel": sig(jump / want - 1, 2),
            "max_u": sig(float(np.sqrt((u ** 2).sum(0)).max()), 3),
            "sum_phi_drift_rel": sig((math.fsum(phi.ravel()) - s0) / s0, 2)}


# ---------------------------------------------------------------- reference arm: the oracle
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = I.WORKLOADS[args.workload]
    grid = w["grid"]
    params = dict(tau_f=w["tau_f"], tau_g=w["tau_g"], M=w["M"], xi=w["xi"], sigma=w["sigma"],
                  rho_ratio=w["rho_ratio"], mu_ratio=w["mu_ratio"], body_force=w["body_force"])
    full = I.droplet_phi(grid, w["R"], w["xi"])
    # each step: one update of a periodic slab cut through the droplet centre, sized so that the
    # whole --warmup + --steps run takes about args.ref_seconds
    def slab(nz):
        z0 = grid[2] // 2 - nz // 2
        return np.ascontiguousarray(full[z0:z0 + nz])

    probe = oracle.Oracle(w["Q"], (grid[0], grid[1], 3), **params)
    probe.init_phi(slab(3))
    t0 = time.perf_counter()
    probe.step(2)
    per_cell = (time.perf_counter() - t0) / (2 * grid[0] * grid[1] * 3)
    budget = args.ref_seconds / max(1, args.steps + args.warmup)
    nz = int(max(3, min(grid[2], budget / (per_cell * grid[0] * grid[1]))))
    sub = (grid[0], grid[1], nz)
    o = oracle.Oracle(w["Q"], sub, **params)
    o.init_phi(slab(nz))
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    secs = time.perf_counter() - t0
    cells = sub[0] * sub[1] * sub[2]
    value = cells * args.steps / secs / 1e6
    sample = f"each step updates a {sub[0]}x{sub[1]}x{sub[2]} periodic slab cut through the droplet centre"
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "MLUPS", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{args.workload} (oracle sample: {sample})", "lattice": "D3Q19",
                      "scheme": "difference-free"},
           "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": oracle.num_threads(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(I.WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate leg")
    ap.add_argument("--legs", default="",
                    help="comma-separated subset of the legs beside the headline, the FD and 16-bit steps and "
                         "e2e (default all: " + ",".join(LEGS) + "); for short profiling runs")
    ap.add_argument("--batch-cases", type=int, default=256,
                    help="rising-bubble cases of the batched leg (the first N of the seeded 256)")
    ap.add_argument("--surrogate-iters", type=int, default=1500, help="training iterations of the surrogate leg")
    ap.add_argument("--surrogate-train-grid", type=int, default=128, choices=[128, 256],
                    help="grid of the surrogate's training trajectories")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=90.0)
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    unknown = [l for l in args.legs.split(",") if l] if args.legs else []
    unknown = [l for l in unknown if l not in LEGS]
    if unknown:
        ap.error(f"unknown legs {unknown}; choose from {','.join(LEGS)}")
    if args.workload != WORKLOAD:
        ap.error("the benchmark line is defined on droplet3d_128 only")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
