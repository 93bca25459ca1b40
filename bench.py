#!/usr/bin/env python3
"""Throughput of the forward FDTD hot path (Gcell-updates/s).

A step is one whole run of the path on the config-2 workload: a 2000 x 12500
synthetic dicot cross-section (dx = 20 nm, S = 0.5), 30 000 leapfrog steps
with CPML, TF/SF source, running-DFT monitors, the empty-domain reference run
and the flux reduction to R and T. Steps cycle through the five wavelengths
450, 550, 662, 800 and 1450 nm. Under torchrun every rank runs its own steps
(independent runs, weak scaling, no collective on the data path).

`--impl reference` times the FP64 oracle on the host cores instead, on a
bounded sample of the same workload (100 leapfrog steps per bench step of
its C time loop on all cores). The default line also carries one config-5
gradient pass (the adjoint's Gcell-updates/s), the oracle on the host cores
and the R/T error of the timed runs against stored full-length oracle runs.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gcell-updates/s (fwd, adjoint), % of HBM roofline, at R/T error ≤2e-3"
UNIT = "Gcell-updates/s"
BYTES_PER_CELL_UPDATE = 25          # read+write Ez, Hx, Hy (FP32) + 1 label byte
WAVELENGTHS = (450e-9, 550e-9, 662e-9, 800e-9, 1450e-9)
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", default="c2", choices=["c1", "c2", "c3", "c4", "c5", "campaign"])
    p.add_argument("--fdtd-steps", type=int, default=0,
                   help="leapfrog steps per run (default: the config's own count)")
    p.add_argument("--kernel", type=int, default=0)
    p.add_argument("--block-steps", type=int, default=0)
    p.add_argument("--seg-rows", type=int, default=0)
    p.add_argument("--variant", type=int, default=-1,
                   help="blocked-kernel code shape (default: the library's choice)")
    p.add_argument("--plan-weight", type=float, default=0.0,
                   help="segment planner weight of a general-path iteration (0: default)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-adjoint", action="store_true",
                   help="skip the config-5 adjoint pass of the default line")
    p.add_argument("--adj-block", type=int, default=-1,
                   help="reverse steps per adjoint launch (0: one per step; default: the "
                        "library's)")
    p.add_argument("--pol", default="s", choices=["s", "p"],
                   help="polarisation of the runs: s (TMz, the default) or p (TEz)")
    return p.parse_args()


def workload(args, lam):
    import fdtd_inputs as fi
    if args.config == "c1":
        spec = fi.config_c1b()
        spec = spec.with_(lambda0=lam, materials=spec.materials)
    elif args.config == "c3":
        spec = fi.config_c3(lambda0=lam, labels=_labels_cache("c3"))
    else:
        spec = fi.config_c2(lambda0=lam, labels=_labels_cache("c2"))
    if args.fdtd_steps:
        spec = spec.with_(steps=args.fdtd_steps)
    if getattr(args, "pol", "s") == "p":
        spec = spec.with_(polarization=fi.POL_P)
    return spec


def _oracle_class(spec):
    if getattr(spec, "polarization", 0):
        from oracle.fdtd_tez import TEzOracle
        return TEzOracle
    from oracle import TMzOracle
    return TMzOracle


_LABELS = {}


def _labels_cache(name):
    import fdtd_inputs as fi
    if name not in _LABELS:
        _LABELS[name] = (fi.config_c2().labels if name == "c2"
                         else fi.config_c3(diseased=True).labels)
    return _LABELS[name]


def describe(spec, args):
    names = {"c1": "config 1b slab with cylinders",
             "c2": "config 2 dicot cross-section",
             "c3": "config 3 monocot cross-section with hyphae"}
    return {
        "workload": f"{names[args.config]} {spec.nx}x{spec.ny} cells, dx={spec.dx * 1e9:.0f} nm, "
                    f"{'P (TEz)' if getattr(spec, 'polarization', 0) else 'S (TMz)'} polarisation, "
                    f"S={spec.courant:.2f}, {spec.steps} leapfrog steps per run, "
                    f"wavelengths 450/550/662/800/1450 nm cycled",
        "nx": spec.nx, "ny": spec.ny, "fdtd_steps_per_run": spec.steps,
        "cell_updates_per_step": spec.nx * spec.ny * spec.steps,
        "l2": "inputs larger than L2: two 3-field FP32 ping-pong sets of "
              f"{spec.nx * spec.ny * 12 / 1e6:.0f} MB each vs 129 MB of L2",
    }


# -- clocks ------------------------------------------------------------------

class ClockSampler:
    def __init__(self, device_id):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={CLOCK_QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(device_id)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s, p in zip(sm, power) if p >= 0.5 * max(power)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power)}


def _device_id():
    import torch
    try:
        u = torch.cuda.get_device_properties(torch.cuda.current_device()).uuid
        return "GPU-" + str(u)
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]
        return vis or "0"


# -- distributed helpers --------------------------------------------------------------------

def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(world, v):
    """The largest value over the ranks (the slowest rank sets the job time);
    a CUDA tensor under NCCL, a host tensor under gloo."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_order(rank, steps, warmup):
    """Wavelengths of a rank's warm-up and timed runs: each rank starts at its
    own place in the cycle, so the ranks' runs are independent problems
    (weak scaling, no data exchanged)."""
    return [WAVELENGTHS[(rank * (steps + warmup) + i) % len(WAVELENGTHS)]
            for i in range(warmup + steps)]


def aggregate_rate(world, steps, cells_per_run, elapsed_max):
    """Whole-job throughput in Gcell-updates/s: all ranks' runs over the
    slowest rank's time."""
    return world * steps * cells_per_run / elapsed_max / 1e9


# -- CPU baseline (the FP64 oracle) -------------------------------------------

def oracle_rate(spec, budget_s=12.0, min_steps=2):
    """Times the oracle as it stands on a bounded number of leapfrog steps of
    the same grid; returns (Gcell-updates/s, steps, seconds)."""
    sim = _oracle_class(spec)(spec)
    sim.step()                                   # first step outside the clock
    steps, t0 = 0, time.perf_counter()
    while steps < min_steps or time.perf_counter() - t0 < budget_s:
        sim.step()
        steps += 1
    dt = time.perf_counter() - t0
    return spec.nx * spec.ny * steps / dt / 1e9, steps, dt


def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    spec = workload(args, WAVELENGTHS[1])
    cores = os.cpu_count() or 1
    if getattr(spec, "polarization", 0):
        # P polarisation: the numpy TEz oracle (one core)
        sim, cores = _oracle_class(spec)(spec), 1
        advance = lambda n: [sim.step() for _ in range(n)]
        how = "numpy FP64 TEz oracle, single-threaded elementwise"
    else:
        from oracle.fdtd_tmz_c import TMzOracleC
        sim = TMzOracleC(spec)
        advance = lambda n: sim.run(n, cores)
        how = "the oracle's C time loop, FP64, OpenMP over rows on all cores"
    sample_steps = 100 if args.config != "c1" else 4000
    if cores == 1 and args.config != "c1":
        sample_steps = 2
    for _ in range(args.warmup):
        advance(sample_steps)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        advance(sample_steps)
    dt = time.perf_counter() - t0
    cells = spec.nx * spec.ny
    value = cells * sample_steps * args.steps / dt / 1e9
    sample = (f"{sample_steps} leapfrog steps of the {spec.nx}x{spec.ny} grid per bench step "
              f"({how})")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": describe(spec, args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample, "cpu_model": cpu_model(), "nproc": os.cpu_count()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# -- our arm --------------------------------------------------------------------------------

def event_seconds(ev0, ev1, wall):
    """Seconds between two CUDA events recorded on the handles' stream, and
    how the time was taken; the synchronised wall clock when the events
    could not be read or do not span the work (under half the wall time)."""
    try:
        dev = ev0.elapsed_time(ev1) / 1e3
    except RuntimeError:
        dev = 0.0
    if dev >= 0.5 * wall:
        return dev, "CUDA events on the handles' stream"
    return wall, "CUDA-synchronised wall clock (events did not span the work)"


def finite_or_none(x):
    """x as a float, or None where it is not finite (R and T of a run too
    short for the pulse to reach the monitors), so that the line stays
    strict JSON."""
    x = float(x)
    return x if math.isfinite(x) else None


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("blocked_impl.cuh", "blocked_s.cu", "fdtd_device.cuh"):
        with open(os.path.join(ROOT, "paper_2512_17132_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def plan_hash(fdtd, spec, seg_rows, block_steps):
    """Hash and segment count of the blocked kernel's segment plan for this
    grid (the library's host-only plan query, default planner weight)."""
    pol = int(getattr(spec, "polarization", 0))
    b = fdtd.fdtd_plan_segments(fdtd.make_grid(spec), seg_rows, block_steps, pol)
    return hashlib.sha256(b.tobytes()).hexdigest()[:16], int(len(b) - 1)


def measured_counters(spec, block_steps, variant, plan_sha):
    """DRAM bytes and warp instructions per launch of the blocked kernel from
    the committed ncu record, or None when the kernel source, the depth, the
    code shape or the segment plan differ from those the counters were
    taken with."""
    path = os.path.join(ROOT, "profiles", "blocked_stencil_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    if (d.get("kernel_src_sha") != kernel_source_hash() or d.get("block_steps") != block_steps
            or d.get("variant") != variant or d.get("plan_sha") != plan_sha
            or d.get("cells") != spec.nx * spec.ny):
        return None
    return d


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def roofline_record(achieved, peak, peak_kind, algo_bytes, avg_launch_s, traffic, inst, clk):
    """Roofline of the blocked stencil. frac is the effective HBM fraction
    (algorithmic bytes of the launch's K steps over its event-timed
    duration): temporal blocking moves about 1/K of those bytes, so it can
    exceed 1. What binds is instruction issue: issue_frac = ncu warp
    instructions per launch / (launch time x SMs x 4 schedulers x the
    sampled SM clock); dram_frac is the real DRAM traffic (ncu bytes per
    launch over the same duration) against the measured copy bandwidth."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = (clk or {}).get("sm_mhz") or None
    ok = avg_launch_s and avg_launch_s > 0
    issue_peak = sms * 4 * mhz * 1e6 if mhz else None
    return {
        "bound": "issue", "achieved": achieved, "peak": peak, "unit": "GB/s",
        "frac": (achieved / peak) if achieved else None, "frac_kind": "effective",
        "traffic": traffic, "peak_kind": f"{peak_kind} copy bandwidth",
        "algorithmic_bytes_per_launch": algo_bytes, "avg_launch_ms": avg_launch_s * 1e3,
        "dram_gbs": (traffic / avg_launch_s / 1e9) if traffic and ok else None,
        "dram_frac": (traffic / avg_launch_s / 1e9 / peak) if traffic and ok and peak else None,
        "warp_inst_per_launch": inst,
        "issue_rate_ginst_s": (inst / avg_launch_s / 1e9) if inst and ok else None,
        "issue_peak_ginst_s": issue_peak / 1e9 if issue_peak else None,
        "issue_frac": (inst / avg_launch_s / issue_peak) if inst and ok and issue_peak else None,
        "note": "frac = 25 B x cells x steps per launch / event-timed launch duration / measured "
                "copy bandwidth (effective: temporal blocking moves fewer DRAM bytes); "
                "dram_frac and issue_frac use the ncu counters of the same kernel, plan and "
                "depth (null when the source, shape or plan changed since they were taken); "
                "issue peak = SMs x 4 schedulers x 1 warp instruction per clock x sampled SM clock"}


def golden_rt_check(results, steps, pol):
    """R and T of the timed runs against the FP64 oracle's values for the
    same full-length config-2 runs (tests/golden), where they exist: same
    step count and the same polarisation ("s" or "p")."""
    errs = []
    for lam, (R, T) in results:
        stem = "oracle_c2p" if pol == "p" else "oracle_c2"
        path = os.path.join(ROOT, "tests", "golden", f"{stem}_{lam * 1e9:g}nm.json")
        try:
            with open(path) as f:
                g = json.load(f)
        except Exception:
            continue
        if (g.get("steps") != steps or g.get("R") is None
                or not str(g.get("polarization", "")).lower().startswith(pol)):
            continue
        errs.append((lam, abs(R - g["R"]), abs(T - g["T"])))
    if not errs:
        return None
    return {"max_abs_err_R": max(e[1] for e in errs), "max_abs_err_T": max(e[2] for e in errs),
            "runs_checked": len(errs),
            "wavelengths_nm": sorted({round(e[0] * 1e9) for e in errs}),
            "vs": ("FP64 oracle, same full-length runs (tests/golden/"
                   + ("oracle_c2p_*.json)" if pol == "p" else "oracle_c2_*.json)")),
            "bound": 2e-3}


def adjoint_pass(fdtd, torch, adj_block=-1):
    """One config-5 gradient pass (1000 x 6000 cells, 30 000 steps,
    checkpoints every 500): the checkpointed forward and the discrete
    adjoint of R(550 nm), each timed with the CUDA-synchronised wall clock
    (the handle runs on the library's own streams). The adjoint's roofline
    is 90 algorithmic bytes per reverse cell-update."""
    import fdtd_inputs as fi
    spec = fi.config_c5()
    cells = spec.nx * spec.ny * spec.steps
    with fdtd.Simulation(spec) as sim:
        if adj_block >= 0:
            fdtd.fdtd_set_option(sim.h, fdtd.FDTD_OPT_ADJ_BLOCK, adj_block)
        # warm-up at the timed length, so that the 60 checkpoint buffers are
        # allocated before the timed pass
        fdtd.fdtd_forward_checkpointed(sim.h, spec.steps, 500)
        fdtd.fdtd_backward(sim.h, 1.0, 0.0, spec.ny, spec.nx, len(spec.materials))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fdtd.fdtd_forward_checkpointed(sim.h, spec.steps, 500)
        R, T = sim.flux()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        fdtd.fdtd_backward(sim.h, 1.0, 0.0, spec.ny, spec.nx, len(spec.materials))
        torch.cuda.synchronize()
        t2 = time.perf_counter()
    peak, kind = peaks()
    adj = cells / (t2 - t1) / 1e9
    return {"value": adj, "unit": UNIT, "ms": (t2 - t1) * 1e3,
            "roofline_frac": adj / (peak / 90.0),
            "roofline": f"{peak / 90.0:.1f} Gcell-updates/s = {kind} copy bandwidth / 90 B",
            "forward_checkpointed": {"value": cells / (t1 - t0) / 1e9, "unit": UNIT,
                                     "ms": (t1 - t0) * 1e3},
            "workload": f"config 5: {spec.nx}x{spec.ny} cells, {spec.steps} steps, dR(550 nm)/d"
                        "(eps_r, sigma, n, k), checkpoints every 500 steps",
            "timing": "CUDA-synchronised wall clock", "R": R}


def cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(spec, budget_s=8.0):
    """The oracle timed on this machine's host cores on a bounded sample of
    the same grid: its C time loop on all cores (OpenMP over rows) and the
    numpy loop on one core."""
    from oracle.fdtd_tmz_c import TMzOracleC
    cores = os.cpu_count() or 1
    sim = TMzOracleC(spec)
    sim.run(2, cores)
    n, t0 = 0, time.perf_counter()
    while n < 4 or time.perf_counter() - t0 < budget_s:
        sim.run(8, cores)
        n += 8
    dt = time.perf_counter() - t0
    rate = spec.nx * spec.ny * n / dt / 1e9
    r1, n1, s1 = oracle_rate(spec, budget_s=budget_s)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} leapfrog steps of the {spec.nx}x{spec.ny} grid in {dt:.1f} s "
                      f"(the oracle's C time loop, FP64, OpenMP over rows on all cores)",
            "cpu_model": cpu_model(), "nproc": cores,
            "single_core": {"value": r1, "unit": UNIT, "cores": 1,
                            "sample": f"{n1} leapfrog steps in {s1:.1f} s (numpy oracle, "
                                      "single-threaded elementwise)"}}


def run_c4(args):
    """Config 4: 64 dicot simulations of uneven height, batched (one launch
    per K steps over all of them, graph-captured chunks, autotuned launch
    shape) against the same 64 handles run one after another (each
    autotuned). One bench step = one pass of the whole batch."""
    import torch
    import fdtd_inputs as fi
    torch.cuda.set_device(0)
    from paper_2512_17132_gb300 import build as b
    b.build()
    from paper_2512_17132_gb300 import fdtd
    steps = args.fdtd_steps or 30000
    specs = fi.config_c4(steps=steps, workers=os.cpu_count())
    cells = sum(sp.nx * sp.ny for sp in specs) * steps
    sims = [fdtd.Simulation(sp, timing=True) for sp in specs]
    batch = fdtd.Batch(sims, timing=True)
    batch.autotune(3)
    warm = min(1024, steps)
    batch.run(warm)
    for s in sims:
        s.reset()
    torch.cuda.synchronize()
    clocks = ClockSampler(_device_id())
    times = []
    for _ in range(args.steps):
        for s in sims:
            s.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        batch.run(steps)
        rt_b = [s.flux() for s in sims]
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    clk = clocks.stop()
    bst = batch.stats()
    t_batch = statistics.median(times)
    for s in sims:                                  # each sequential run tuned for its grid
        fdtd.fdtd_autotune(s.h, 3)
        s.reset()
        s.run(warm)
        s.reset()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in sims:
        s.run(steps)
        s.flux()
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    rt_s = [s.flux() for s in sims]
    same = all(a == c or (math.isnan(a[0]) and math.isnan(c[0])) for a, c in zip(rt_b, rt_s))
    batch.close()
    for s in sims:
        s.close()
    line = {
        "metric": METRIC, "value": cells / t_batch / 1e9, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": 1, "ms_per_step": t_batch * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"config 4: 64 dicot simulations, width 2000, heights "
                               f"{min(sp.ny for sp in specs)}-{max(sp.ny for sp in specs)}, "
                               f"{steps} leapfrog steps each, wavelengths 400-2500 nm",
                   "total_cells": sum(sp.nx * sp.ny for sp in specs),
                   "batched_block_steps": bst["block_steps"], "batched_seg_rows": bst["seg_rows"],
                   "cuda_graph": bst["graph"]},
        "sequential": {"value": cells / t_seq / 1e9, "unit": UNIT, "ms": t_seq * 1e3,
                       "note": "the same 64 handles run one after another, each autotuned"},
        "batched_over_sequential": t_seq / t_batch,
        "rt_identical": bool(same),
        "clocks": clk, "gpu_launches": int(bst["total_launches"]),
    }
    print(json.dumps(line))
    return 0


def run_campaign_bench(args):
    """Spectrum/slice campaign (Sec. 4) on the config-2 cross-section: the
    2000-column section cut into five 400-column slices, the five config-2
    wavelengths, both polarisations (50 independent runs), slice- and
    polarisation-averaged. One bench step = one whole campaign on resident
    handles (one tuned batch per polarisation); e2e repeats it through
    run_campaign from the host label map (handles created and destroyed)."""
    import torch
    import fdtd_inputs as fi
    torch.cuda.set_device(0)
    from paper_2512_17132_gb300 import build as b
    b.build()
    from paper_2512_17132_gb300 import fdtd
    from paper_2512_17132_gb300.campaign import Campaign, run_campaign
    steps = args.fdtd_steps or 30000
    labels = _labels_cache("c2")

    def make(lam):
        return fi.config_c2(lambda0=lam, labels=labels, steps=steps)

    wl = list(fi.C2_WAVELENGTHS)
    camp = Campaign(make, wl, n_slices=5, timing=True)
    cells = camp.cell_updates_per_step * steps
    for _ in range(args.warmup):
        camp.run(steps)
    torch.cuda.synchronize()
    before = camp.stats()
    clocks = ClockSampler(_device_id())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        res = camp.run(steps)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    clk = clocks.stop()
    after = camp.stats()
    launches = sum(a["total_launches"] - b_["total_launches"] for a, b_ in zip(after, before))
    camp.close()
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(args.steps):
            run_campaign(make, wl, n_slices=5, steps=steps)
        torch.cuda.synchronize()
        e_el = time.perf_counter() - t1
        h2d = 2 * labels.nbytes + 50 * steps * (4 + 4 + 16 + 16)
        e2e = {"value": args.steps * cells / e_el / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 50 * 3 * 8,
               "ms_per_step": e_el / args.steps * 1e3,
               "note": "per step: run_campaign from the host label map (50 handles created, "
                       "batched, autotuned, run, flux read, destroyed)"}
    line = {
        "metric": METRIC, "value": args.steps * cells / el / 1e9, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"campaign: config-2 dicot 2000x12500 cut into 5 slices of 400 "
                               f"columns x 5 wavelengths (450-1450 nm) x 2 polarisations, "
                               f"{steps} leapfrog steps per run, averaged (Sec. 4)",
                   "runs_per_step": len(camp.specs), "cell_updates_per_step": cells,
                   "l2": "inputs larger than L2 (50 runs x 2 x 60 MB of fields)"},
        "spectrum": {"lambda_nm": [round(x * 1e9) for x in wl], "R": list(map(float, res["R"])),
                     "T": list(map(float, res["T"])), "A": list(map(float, res["A"]))},
        "e2e": e2e, "clocks": clk, "gpu_launches": int(launches),
    }
    print(json.dumps(line))
    return 0


def run_c5(args):
    """Config 5: gradient of R(550 nm) on the config-1 stack at 1000 x 6000
    cells, 30 000 steps, checkpoints every 500 steps: the checkpointed forward
    and the discrete adjoint (segment recompute + reverse steps) timed
    separately, as Gcell-updates/s of forward and of reverse steps."""
    import torch
    import fdtd_inputs as fi
    torch.cuda.set_device(0)
    from paper_2512_17132_gb300 import build as b
    b.build()
    from paper_2512_17132_gb300 import fdtd
    spec = fi.config_c5(steps=args.fdtd_steps or 30000)
    cells = spec.nx * spec.ny * spec.steps
    sim = fdtd.Simulation(spec)
    if args.adj_block >= 0:
        fdtd.fdtd_set_option(sim.h, fdtd.FDTD_OPT_ADJ_BLOCK, args.adj_block)
    if args.plan_weight > 0:
        fdtd.fdtd_set_option(sim.h, fdtd.FDTD_OPT_PLAN_WEIGHT, round(args.plan_weight * 1000))
    fdtd.fdtd_forward_checkpointed(sim.h, spec.steps, 500)   # warm-up: checkpoints allocated
    fdtd.fdtd_backward(sim.h, 1.0, 0.0, spec.ny, spec.nx, len(spec.materials))
    clocks = ClockSampler(_device_id())
    t_f, t_b = [], []
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fdtd.fdtd_forward_checkpointed(sim.h, spec.steps, 500)
        R, T = sim.flux()
        t1 = time.perf_counter()
        g = fdtd.fdtd_backward(sim.h, 1.0, 0.0, spec.ny, spec.nx, len(spec.materials))
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        t_f.append(t1 - t0)
        t_b.append(t2 - t1)
    clk = clocks.stop()
    st = sim.stats()
    sim.close()
    tf, tb = statistics.median(t_f), statistics.median(t_b)
    line = {
        "metric": METRIC, "value": cells / tb / 1e9, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": 1, "ms_per_step": (tf + tb) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"config 5: config-1 stack at {spec.nx}x{spec.ny}, "
                               f"{spec.steps} steps, dR(550 nm)/d(eps_r, sigma, n, k), "
                               "checkpoints every 500 steps",
                   "value_is": "adjoint (backward) Gcell-updates/s: reverse steps incl. the "
                               "segment recompute"},
        "forward": {"value": cells / tf / 1e9, "unit": UNIT, "ms": tf * 1e3,
                    "note": "checkpointed forward (blocked kernel + state copies)"},
        "adjoint": {"value": cells / tb / 1e9, "unit": UNIT, "ms": tb * 1e3},
        "R": R, "T": T, "dR_dn": list(g["g_n"]), "dR_dk": list(g["g_k"]),
        "clocks": clk, "gpu_launches": int(st["total_launches"]),
    }
    print(json.dumps(line))
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "c4":
        return run_c4(args)
    if args.config == "c5":
        return run_c5(args)
    if args.config == "campaign":
        return run_campaign_bench(args)
    world, rank, local = dist_setup(args)
    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        from paper_2512_17132_gb300 import build as b
        b.build()
    _barrier(world)
    from paper_2512_17132_gb300 import fdtd
    fdtd.load_library()

    K, W = args.steps, args.warmup
    order = rank_order(rank, K, W)
    specs = {lam: workload(args, lam) for lam in set(order)}
    spec0 = specs[order[-1]]
    cells_per_run = spec0.nx * spec0.ny * spec0.steps
    # every handle works on one stream of ours, so that CUDA events on it
    # bracket the timed region
    stream = torch.cuda.Stream()
    sims = {}
    for lam, sp in specs.items():
        s = fdtd.Simulation(sp, stream=stream, kernel=args.kernel,
                            block_steps=args.block_steps or None,
                            seg_rows=args.seg_rows or None, timing=True)
        if args.variant >= 0:
            fdtd.fdtd_set_option(s.h, fdtd.FDTD_OPT_VARIANT, args.variant)
        if args.plan_weight > 0:
            fdtd.fdtd_set_option(s.h, fdtd.FDTD_OPT_PLAN_WEIGHT, round(args.plan_weight * 1000))
        sims[lam] = s
    results = []

    def one(lam):
        s = sims[lam]
        s.reset()
        s.run(specs[lam].steps)
        results.append((lam, s.flux()))

    for lam in order[:W]:
        one(lam)
    torch.cuda.synchronize()
    before = {lam: s.stats() for lam, s in sims.items()}
    clocks = ClockSampler(_device_id()) if rank == 0 else None
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    _barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev0.record(stream)
    for lam in order[W:]:
        one(lam)
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    elapsed, timing = event_seconds(ev0, ev1, wall)
    _barrier(world)
    clk = clocks.stop() if clocks else None
    after = {lam: s.stats() for lam, s in sims.items()}
    elapsed = _max_over_ranks(world, elapsed)
    value = aggregate_rate(world, K, cells_per_run, elapsed)

    st_ms = sum(after[l]["stencil_ms"] - before[l]["stencil_ms"] for l in sims)
    st_n = sum(after[l]["stencil_launches"] - before[l]["stencil_launches"] for l in sims)
    launches = sum(after[l]["total_launches"] - before[l]["total_launches"] for l in sims)
    st = after[order[-1]]
    kern = st["kernel"]
    steps_per_launch = st["block_steps"] if kern == 2 else 1
    avg_launch_s = st_ms / 1e3 / max(st_n, 1)
    algo_bytes = BYTES_PER_CELL_UPDATE * spec0.nx * spec0.ny * steps_per_launch
    peak, peak_kind = peaks()
    achieved = algo_bytes / avg_launch_s / 1e9 if avg_launch_s > 0 else None
    # the stored counters were captured on the S kernel with the default plan
    counters = None
    if kern == 2 and args.pol == "s" and args.plan_weight <= 0:
        p_sha, n_segs = plan_hash(fdtd, spec0, st["seg_rows"], steps_per_launch)
        counters = measured_counters(spec0, steps_per_launch, st["variant"], p_sha)
    traffic = counters["dram_bytes_per_launch"] if counters else None
    inst = counters.get("warp_inst_per_launch") if counters else None
    rt_check = golden_rt_check([(lam, rt) for lam, rt in results[W:]], spec0.steps, args.pol)
    for s in sims.values():
        s.close()

    e2e = None
    if not args.no_e2e:
        # end to end through the C ABI from host buffers: create (label map and
        # material table copied from the host), run, flux (R, T read back), destroy
        import numpy as np
        h2d = 0
        # the step's inputs wait in pinned host memory
        pinned = {lam: torch.from_numpy(np.ascontiguousarray(specs[lam].labels)).pin_memory()
                  for lam in set(order[W:])}
        torch.cuda.synchronize()
        _barrier(world)
        t1 = time.perf_counter()
        for lam in order[W:]:
            sp = specs[lam]
            with fdtd.Simulation(sp, labels=pinned[lam]) as s:
                s.run(sp.steps)
                s.flux()
            h2d = (sp.labels.nbytes + sp.materials.size * 8
                   + sp.steps * (4 + 4 + 16 + 16))
        torch.cuda.synchronize()
        e_el = _max_over_ranks(world, time.perf_counter() - t1)
        _barrier(world)
        e2e = {"value": world * K * cells_per_run / e_el / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 3 * 8,
               "ms_per_step": e_el / K * 1e3,
               "note": "per step: fdtd_create from a pinned host label map + fdtd_run + "
                       "fdtd_flux + fdtd_destroy; h2d = label map, material table, "
                       "incident/phase tables"}

    adjoint = None
    if rank == 0 and world == 1 and not args.no_adjoint and args.pol == "s":
        adjoint = adjoint_pass(fdtd, torch, args.adj_block)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(specs[order[-1]])

    if rank == 0:
        cfg = describe(spec0, args)
        cfg.update({"kernel": "temporally blocked" if kern == 2 else "per-half-step",
                    "steps_per_launch": steps_per_launch, "seg_rows": st["seg_rows"],
                    "code_shape": st["variant"],
                    "parallelism": f"{world} independent run stream(s), one per GPU"})
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": elapsed / K * 1e3, "timing": timing,
            "wall_ms_per_step": wall / K * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": cfg,
            "roofline": roofline_record(achieved, peak, peak_kind, algo_bytes, avg_launch_s,
                                        traffic, inst, clk),
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": int(launches),
            "rt_last": {"lambda_nm": results[-1][0] * 1e9, "R": finite_or_none(results[-1][1][0]),
                        "T": finite_or_none(results[-1][1][1])},
            "rt_check": rt_check,
            "adjoint": adjoint,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
