#!/usr/bin/env python
"""Throughput of the ternary phase-field lattice Boltzmann update on GB300.

One bench step = one time step of the whole hot path (fused interior kernel +
near-wall kernel) over the 2048x2048 tiled-drops lattice (binary drops on a
wetting bottom wall, neutral top wall, periodic in x, free compound drops in
the bulk).  The state (FP64: 1.8 GB double-buffered) is far larger than the
129 MB L2, so no explicit flush is needed between steps.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the host cores instead, on a bounded sample of the same workload.
Multi-GPU (torchrun): independent replicas, one lattice per rank, no
collective on the data path (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & % of HBM roofline, batched/served vs plain; p50/p99 solve latency"


def bytes_per_node(precision):
    """Algorithmic bytes per node update: the state the method must carry from
    one step to the next, read once and written once -- the 27 distributions
    f^1, f^2, g (Eqs. 1a, 1b) and the 4 c_i u values of Eq. 19 (62 values):
    496 B in FP64, 248 B in FP32, 140 B with 16-bit distributions and FP32
    c_i u.  Storage-layout extras (the lo halves that keep the rest
    populations mass-conserving) are not the method's work and are reported
    apart (storage_bytes_per_node)."""
    if precision == "fp64":
        return 2 * (27 + 4) * 8
    if precision == "fp32":
        return 2 * (27 + 4) * 4
    return 2 * (27 * 2 + 4 * 4)


def storage_bytes_per_node(precision):
    """Bytes per node update that this library's storage layout moves: FP32
    keeps the two rest populations as float pairs (two extra planes); 16-bit
    storage keeps the 25 moving populations in 16 bits and the two rest
    populations as FP32 pairs (16 bytes)."""
    if precision == "fp64":
        return 2 * (27 + 4) * 8
    if precision == "fp32":
        return 2 * (29 + 4) * 4
    return 2 * (25 * 2 + 4 * 4 + 4 * 4)


KERNEL = {"fp64": "k_step_interior<double>", "fp32": "k_step_interior<float>",
          "fp16": "k_step_interior<__half>", "bf16": "k_step_interior<__nv_bfloat16>"}


# FP64 arithmetic per node update of the fused interior kernel as counted by
# ncu on the 2048^2 lattice: (DADD + DMUL + DFMA instructions, flops with an
# FMA as 2).  "uniform": the update taken when all three fluids share density
# and viscosity (the tiled-drops workload); "general": any densities and
# viscosities (the same lattice with rho_2 = 3).
FP64_DP = {"uniform": (216.9, 312.9), "general": (281.1, 407.4)}
# The same counts for the D3Q19 update kernel k3_update (ncu, 128x64x128
# drops on a wetting wall, uniform properties: 150.0 DFMA + 149.0 DADD + 53.0
# DMUL per node).
FP64_DP3 = {"uniform": (352.0, 502.0)}
# FP64 vector unit: 152 SMs x 2 DP instructions/clk x 2.07 GHz (an FMA is 2 flops)
FP64_DP_INST_PEAK = 152 * 2 * 2.07e9
FP64_PEAK_TFLOPS = 2 * FP64_DP_INST_PEAK / 1e12
SAMPLE_ROWS = 256


def whole_job_mlups(nodes_per_rank, steps, world, ms_max):
    """Aggregate throughput: every rank's node updates over the slowest rank's time."""
    return nodes_per_rank * steps * world / (ms_max / 1e3) / 1e6


def max_over_ranks(D, ms, device="cpu"):
    """Max of a per-rank time over the process group (identity without one)."""
    if D is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    D.all_reduce(t, op=D.ReduceOp.MAX)
    return float(t.item())


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "fp16", "bf16"])
    ap.add_argument("--inplace", action="store_true",
                    help="step the main lattice with in-place (AA-pattern) streaming; the interior time then "
                         "includes the order-parameter pass")
    ap.add_argument("--rho2", type=float, default=None,
                    help="density of fluid 2 on the main lattice (default: the workload's 1.0; another value "
                         "times the general, density-contrast update)")
    ap.add_argument("--nx", type=int, default=2048)
    ap.add_argument("--ny", type=int, default=2048)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--variants", default="fp32,fp16,bf16",
                    help="comma list of extra precisions to time; 'none' also skips the density-contrast, MRT and in-place variants")
    ap.add_argument("--impact-steps", type=int, default=2000,
                    help="least steps of the 1024x2048 cylinder-impact workload per precision and Weber number (0: skip)")
    ap.add_argument("--impact-max-steps", type=int, default=9000,
                    help="a Weber number whose drop reaches the cylinder within this many steps runs until 1500 "
                         "steps after contact, so that a film forms")
    ap.add_argument("--shear-steps", type=int, default=20000,
                    help="steps of the 512x256 sheared compound drop, FP64 and FP32 (0: skip)")
    ap.add_argument("--batch-count", type=int, default=256, help="lattices in the batched workload (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=5000, help="steps of every lattice in one batch")
    ap.add_argument("--batch-plain-steps", type=int, default=500,
                    help="steps timed on the plain path (one tlb_step per lattice), whose rate does not "
                         "depend on the step count")
    ap.add_argument("--d3-steps", type=int, default=100,
                    help="steps of the D3Q19 drops-on-wall lattice (0: skip)")
    ap.add_argument("--d3-size", default="192,96,192", help="nx,ny,nz of the D3Q19 lattice")
    ap.add_argument("--serve-count", type=int, default=200, help="requests in the served workload (0: skip)")
    ap.add_argument("--serve-budget-gb", type=float, default=40.0)
    ap.add_argument("--serve-hi", type=int, default=2048, help="largest side of a served lattice")
    ap.add_argument("--serve-steps-lo", type=int, default=1000)
    ap.add_argument("--serve-steps-hi", type=int, default=20000)
    return ap.parse_args()


# the sources that define the two-buffer interior kernel and its launch
INTERIOR_SOURCES = ("tlbm_device.cuh", "tlbm_kernels.cuh", "tlbm_ops.h", "tlbm_ops_impl.cuh",
                    "tlbm_f64.cu", "tlbm_f32.cu", "tlbm_f16.cu", "tlbm_bf16.cu")


def kernel_source_hash():
    """SHA-256 over the sources of the interior kernel, to tell whether a
    stored ncu capture still describes the kernel being timed."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1710_09534_gb300", "csrc")
    for f in INTERIOR_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    from paper_1710_09534_gb300 import build
    fl = build._flags()
    # the compiler flags shape the code too (the include paths, which depend on
    # where the checkout lives, do not)
    fl = [f for i, f in enumerate(fl) if f != "-I" and (i == 0 or fl[i - 1] != "-I")]
    h.update(" ".join(fl).encode())
    return h.hexdigest()


def measured_traffic(precision, units):
    """DRAM bytes per launch of the interior kernel from the committed ncu
    capture (profiles/interior_traffic.json), scaled to `units` interior
    nodes; None when the capture predates the current kernel sources."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "interior_traffic.json")))
    except Exception:
        return None
    if d.get("csrc_sha256") != kernel_source_hash() or precision not in d:
        return None
    e = d[precision]
    return round(e["dram_bytes"] / e["interior_nodes"] * units)


def measured_fp64_peak(T):
    """FP64 fused-multiply-add rate measured on this device just before the
    timed region (tlb_fma_peak: independent FMA chains on every SM, fastest of
    five launches); the nominal figure if the measurement fails."""
    try:
        r = T.fma_peak("fp64")
        return r["tflops"], (f"measured in this run: tlb_fma_peak FP64 FMA chains on every SM, "
                             f"{r['ms']:.3f} ms per launch, fastest of 5")
    except Exception as e:  # the kernel roofline still needs a denominator
        return FP64_PEAK_TFLOPS, f"nominal (FMA measurement failed: {e})"


def peaks():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except Exception:
            self.p.kill()
        self.f.seek(0)
        sms, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sms) if sms else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sms)}


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as D
        backend = os.environ.get("TLB_BENCH_BACKEND", "nccl")
        D.init_process_group(backend)
        return D, D.get_rank(), ws, int(os.environ.get("LOCAL_RANK", "0"))
    return None, 0, 1, 0


def sample_workload(w, rows=SAMPLE_ROWS):
    """Bottom `rows` rows of a workload (same edges, physics and drops)."""
    import copy
    s = copy.copy(w)
    s.ny = rows
    for k in ("mask", "c1", "c2", "ux", "uy"):
        setattr(s, k, np.ascontiguousarray(getattr(w, k)[:rows]))
    s.name = f"{w.name}[rows 0..{rows - 1}]"
    return s


def oracle_run(w, steps, warmup=0):
    """Time the FP64 oracle on workload w (host cores); returns (MLUPS, seconds, threads)."""
    import oracle
    O = oracle.OracleLattice(w.nx, w.ny, w.edges, w.mask, w.params)
    O.set_fields(w.c1, w.c2, w.ux, w.uy)
    if warmup:
        O.step(warmup)
    t0 = time.perf_counter()
    O.step(steps)
    dt = time.perf_counter() - t0
    return w.nx * w.ny * steps / dt / 1e6, dt, oracle.threads()


def cpu_model():
    """The host CPU as lscpu names it (machine type if lscpu is missing)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                name = line.split(":", 1)[1].strip()
                if name and not name.isdigit():
                    return f"{name} ({platform.machine()})"
    except Exception:
        pass
    return platform.machine() or "unknown"


def cpu_baseline(w, budget_s=12.0, single_s=5.0):
    """The oracle on a bounded sample (~budget_s seconds of host work on all
    cores), and the same sample on one core (~single_s seconds) beside it."""
    import oracle
    s = sample_workload(w)
    _, t1, _ = oracle_run(s, 2)
    steps = max(1, min(5000, int(budget_s / max(t1 / 2, 1e-3))))
    mlups, dt, thr = oracle_run(s, steps)
    out = {"value": round(mlups, 3), "unit": "MLUPS", "cores": thr, "kind": "oracle",
           "cpu": cpu_model(), "nproc": os.cpu_count(),
           "sample": f"{s.nx}x{s.ny} bottom strip of the {w.nx}x{w.ny} lattice, {steps} steps, "
                     f"{dt:.1f} s, FP64 C oracle with OpenMP over nodes"}
    oracle.set_threads(1)
    try:
        _, t1, _ = oracle_run(s, 1)
        steps1 = max(1, int(single_s / max(t1, 1e-3)))
        m1, dt1, _ = oracle_run(s, steps1)
    finally:
        oracle.set_threads(thr)
    out["single_core"] = {"value": round(m1, 3), "unit": "MLUPS", "cores": 1,
                          "sample": f"the same strip, {steps1} steps, {dt1:.1f} s"}
    # the 128x64 two-drop wetting case, its full 2000 steps, on all cores
    import workloads as W
    c1 = W.binary_drops_on_wall()
    mc, dtc, _ = oracle_run(c1, 2000)
    out["binary_drops_128x64"] = {"value": round(mc, 3), "unit": "MLUPS", "cores": thr,
                                  "sample": f"{c1.name}, 2000 steps, {dtc:.1f} s"}
    return out


def run_reference(args):
    D, rank, ws, _ = dist()
    if rank != 0:
        return
    import workloads as W
    full = W.tiled_drops(args.nx, args.ny)
    w = sample_workload(full)
    import oracle
    O = oracle.OracleLattice(w.nx, w.ny, w.edges, w.mask, w.params)
    O.set_fields(w.c1, w.c2, w.ux, w.uy)
    O.step(args.warmup)
    t0 = time.perf_counter()
    O.step(args.steps)
    dt = time.perf_counter() - t0
    mlups = w.nx * w.ny * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": round(mlups, 3), "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            # the workload of the GPU arm; each step runs on a bounded sample of it
            "config": {"workload": full.name, "nx": full.nx, "ny": full.ny, "precision": "fp64",
                       "storage": "f64", "parallelism": "host cores (OpenMP)",
                       "sample": f"bottom {w.ny} rows ({w.nx}x{w.ny}) per step"},
            "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": oracle.threads(),
                             "kind": "oracle", "cpu": cpu_model(), "nproc": os.cpu_count(),
                             "sample": f"{w.name}, {args.steps} steps per run"},
            "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_steps(L, steps, torch, stream):
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    L.step(steps)
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end)


def run_ours(args):
    import torch
    D, rank, ws, local = dist()
    torch.cuda.set_device(local)
    import paper_1710_09534_gb300 as T
    import workloads as W
    stream = torch.cuda.current_stream()
    w = W.tiled_drops(args.nx, args.ny)
    if args.rho2 is not None:
        w.params.update(rho2=args.rho2)
    L = T.lattice_from_workload(w, args.precision, inplace=args.inplace)
    n_nodes = w.nx * w.ny
    L.step(args.warmup)
    L.sync()
    fp64_peak = measured_fp64_peak(T) if args.precision == "fp64" else None
    # timed region: K steps, barrier + synchronize on both sides
    if D:
        D.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local) if rank == 0 else None
    L.profile(True)
    ms = time_steps(L, args.steps, torch, stream)
    k1_ms, k2_ms, k1_n, k2_n = L.profile_read()
    L.profile(False)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    ms = max_over_ranks(D, ms, "cuda")
    if D:
        D.barrier()
    mlups = whole_job_mlups(n_nodes, args.steps, ws, ms)
    hbm_gbs, peak_kind = peaks()
    bytes_node = bytes_per_node(args.precision)
    k1_avg = k1_ms / max(k1_n, 1)
    # the fused interior kernel dominates; its algorithmic units are the
    # interior nodes it updates per launch
    interior_nodes = n_nodes - L.wall_nodes()
    ach_gbs = interior_nodes * bytes_node / (k1_avg / 1e3) / 1e9
    hbm_frac = ach_gbs / hbm_gbs
    # stored DRAM traffic describes the two-buffer interior kernel only
    traffic = None if args.inplace else measured_traffic(args.precision, interior_nodes)
    prm = w.params
    path = "uniform" if (prm["rho1"] == prm["rho3"] == prm["rho2"] and prm["nu1"] == prm["nu3"] == prm["nu2"]) else "general"
    if args.precision == "fp64":
        dp_inst, dp_flops = FP64_DP[path]
        ach_tf = interior_nodes * dp_flops / (k1_avg / 1e3) / 1e12
        dp_issue = interior_nodes * dp_inst / (k1_avg / 1e3) / FP64_DP_INST_PEAK
        peak_tf, peak_src = fp64_peak
        roof = {"bound": "alu", "achieved": round(ach_tf, 4), "peak": round(peak_tf, 4),
                "unit": "TFLOP/s", "frac": round(ach_tf / peak_tf, 4), "traffic": traffic,
                "peak_source": peak_src,
                "peak_nominal": round(FP64_PEAK_TFLOPS, 4),
                "peak_nominal_source": "152 SMs x 2 DP inst/clk x 2 flop x 2.07 GHz",
                "kernel": "k_step_interior<double>", "update": path,
                "dp_inst_per_node": dp_inst, "flops_per_node": dp_flops,
                "dp_issue_frac": round(dp_issue, 4),
                "hbm_achieved_gbs": round(ach_gbs, 1), "hbm_peak_gbs": hbm_gbs, "hbm_frac": round(hbm_frac, 4)}
    else:
        roof = {"bound": "hbm", "achieved": round(ach_gbs, 1), "peak": hbm_gbs, "unit": "GB/s",
                "frac": round(hbm_frac, 4), "traffic": traffic,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                "kernel": ("k_csum + k_step_interior_ip" if args.inplace else KERNEL[args.precision]),
                "algorithmic_bytes_per_node": bytes_node,
                "storage_bytes_per_node": storage_bytes_per_node(args.precision)}
    result = {
        "metric": METRIC, "value": round(mlups, 2), "unit": "MLUPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
        "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "precision": args.precision,
                   "streaming": "in-place (AA pattern)" if args.inplace else "two buffers",
                   "storage": {"fp64": "f64", "fp32": "f32", "fp16": "f16 (shifted, x2^12) + f32 rest pairs",
                               "bf16": "bf16 (shifted) + f32 rest pairs"}[args.precision],
                   "l2": f"state {bytes_node * n_nodes / 1e9:.2f} GB moved per step > 129 MB L2 (no flush needed)",
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "wall_nodes": int(L.wall_nodes())},
        "hbm_roofline_pct": round(100 * mlups / ws * 1e6 * bytes_node / (hbm_gbs * 1e9), 2),
        "roofline": roof,
        "kernel_ms": {"interior_avg": round(k1_avg, 4), "wall_avg": round(k2_ms / max(k2_n, 1), 4),
                      "wall_note": "the near-wall kernel runs on a side stream concurrently with the interior "
                                   "kernel; its time spans launch to end, mostly waiting for SMs"},
        # two buffers: interior + near-wall kernel per step; in place: the
        # order-parameter pass, the interior, the lid row (if any) and the
        # near-wall kernel, plus the streaming swap after an odd step count
        "gpu_launches": int(k1_n + k2_n) if not args.inplace else
        int(args.steps * (3 + (w.edges[3] == 3)) + args.steps % 2),
        "clocks": clk,
    }
    if rank == 0 and not args.no_e2e:
        result["e2e"] = e2e(L, w, args, torch, T)
    if rank == 0:
        variants = {}
        extras = args.variants != "none"  # "none": no variant of any kind (short profiling runs)
        for prec in [v for v in args.variants.split(",") if v and v not in ("none", args.precision)]:
            V = T.lattice_from_workload(w, prec)
            V.step(args.warmup)
            V.sync()
            vms = time_steps(V, args.steps, torch, stream)
            v_mlups = n_nodes * args.steps / (vms / 1e3) / 1e6
            variants[prec] = {"value": round(v_mlups, 2), "unit": "MLUPS",
                              "hbm_roofline_pct": round(100 * v_mlups * 1e6 * bytes_per_node(prec) / (hbm_gbs * 1e9), 2),
                              "algorithmic_bytes_per_node": bytes_per_node(prec),
                              "storage_bytes_per_node": storage_bytes_per_node(prec)}
            del V
        # the general (per-node density and viscosity) update: fluid 2 three times denser
        for prec in ("fp64", "fp32") if extras else ():
            wd = W.tiled_drops(args.nx, args.ny)
            wd.params.update(rho2=3.0)
            V = T.lattice_from_workload(wd, prec)
            V.step(args.warmup)
            V.sync()
            n_d = max(10, args.steps // (4 if prec == "fp64" else 1))
            vms = time_steps(V, n_d, torch, stream)
            variants[prec + "_density_contrast"] = {
                "value": round(n_nodes * n_d / (vms / 1e3) / 1e6, 2), "unit": "MLUPS", "steps": n_d,
                "update": "general (rho = 1, 3, 1)"}
            del V
        # the MRT collision option on the same lattice (FP64 and FP32 storage)
        for prec in ("fp64", "fp32") if extras else ():
            wm = W.tiled_drops(args.nx, args.ny)
            wm.params.update(collision=1.0, mrt_s_f=1.2, mrt_s_g=1.2)
            V = T.lattice_from_workload(wm, prec)
            V.step(args.warmup)
            V.sync()
            n_mrt = max(10, args.steps // (4 if prec == "fp64" else 1))
            vms = time_steps(V, n_mrt, torch, stream)
            v_mlups = n_nodes * n_mrt / (vms / 1e3) / 1e6
            variants[prec + "_mrt"] = {"value": round(v_mlups, 2), "unit": "MLUPS", "steps": n_mrt,
                                       "collision": "MRT (s_f = s_g = 1.2)"}
            del V
        # in-place (AA-pattern) streaming: one distribution buffer plus the
        # order-parameter planes, the extra order-parameter pass in every step
        for prec in ("fp64", "fp32", "fp16") if extras else ():
            V = T.lattice_from_workload(w, prec, inplace=True)
            V.step(args.warmup)
            V.sync()
            n_ip = max(10, args.steps // (4 if prec == "fp64" else 1)) // 2 * 2
            vms = time_steps(V, n_ip, torch, stream)
            v_mlups = n_nodes * n_ip / (vms / 1e3) / 1e6
            variants[prec + "_inplace"] = {
                "value": round(v_mlups, 2), "unit": "MLUPS", "steps": n_ip,
                "hbm_roofline_pct": round(100 * v_mlups * 1e6 * bytes_per_node(prec) / (hbm_gbs * 1e9), 2),
                "workspace_bytes": int(V.workspace.numel()),
                "two_buffer_workspace_bytes": int(T.load_library().tlb_workspace_bytes(w.nx, w.ny, T.PRECISIONS[prec]))}
            del V
        result["variants"] = variants
        if args.impact_steps > 0:
            result["impact"] = impact(args, torch, T)
        if args.shear_steps > 0:
            result["shear"] = shear(args, torch, T)
        if args.batch_count > 0:
            result["batched"] = batched(args, torch, T)
        if args.serve_count > 0:
            result["served"] = served(args, torch, T)
        if args.d3_steps > 0:
            result["d3q19"] = d3q19(args, torch, T, fp64_peak)
        if not args.no_cpu_baseline:
            result["cpu_baseline"] = cpu_baseline(w)
        print(json.dumps(result), flush=True)
    if D:
        D.barrier()
        D.destroy_process_group()


def batched(args, torch, T):
    """The batched workload: `batch_count` lattices with sides log-uniform in
    [64, 512] (drops on a wetting wall, random tensions and angles), in FP32
    and in shifted-FP16 storage.  Aggregate MLUPS of (a) the plain path, one
    tlb_step call per lattice, and (b) one batch (persistent tile-queue
    kernel, graph-captured), after the batch tuner picked its tile shape."""
    import workloads as W
    ws = W.batch_population(args.batch_count, seed=1710)
    nodes = sum(w.nodes for w in ws)
    k = args.batch_steps
    kp = min(args.batch_plain_steps, k)
    out = {"workload": f"{len(ws)} lattices, sides log-uniform 64..512 (seed 1710), drops on a wetting wall",
           "nodes": nodes, "steps": k, "plain_steps": kp}
    for prec in ("fp32", "fp16"):
        plain = [T.lattice_from_workload(w, prec) for w in ws]
        for L in plain:
            L.step(2)
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        for L in plain:
            L.step(kp)
        s1.record()
        s1.synchronize()
        plain_ms = s0.elapsed_time(s1)
        del plain
        mem = [T.lattice_from_workload(w, prec) for w in ws]
        B = T.Batch(prec, max_lattices=len(mem), max_tiles=sum(T.Batch.tiles_needed(w.nx, w.ny) for w in ws),
                    max_wall_nodes=sum(L.wall_nodes() for L in mem))
        for L in mem:
            B.add(L)
        cfg = B.tune(trial_steps=3)
        B.step(2)
        B.synchronize()
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(B.stream)
        B.step(k)
        b1.record(B.stream)
        b1.synchronize()
        batch_ms = b0.elapsed_time(b1)
        r = {"plain_mlups": round(nodes * kp / (plain_ms / 1e3) / 1e6, 1),
             "batched_mlups": round(nodes * k / (batch_ms / 1e3) / 1e6, 1), "tuned": cfg,
             "batched_s": round(batch_ms / 1e3, 3)}
        r["speedup"] = round(r["batched_mlups"] / r["plain_mlups"], 2)
        B.close()
        del mem
        if prec == "fp32":
            out.update(r)  # the FP32 figures at the top level
        else:
            out[prec] = r
    return out


def cushion_gap(f, col, y_top):
    """Thickness of the layer of fluid 3 between the cylinder top and the drop
    on column `col`: distance from the half-way wall above solid row y_top to
    the first crossing of c1 + c2 = 1/2 (linear interpolation); NaN if the
    column holds no drop.  0 once the drop touches the wall (the film
    thickness of `tlb_film_thickness` then measures the drop's own layer)."""
    s = f["c1"][:, col] + f["c2"][:, col]
    above = s[y_top + 1:]
    if above[0] >= 0.5:
        return 0.0
    idx = np.nonzero(above >= 0.5)[0]
    if not len(idx):
        return float("nan")
    j = int(idx[0])
    t = (0.5 - above[j - 1]) / (above[j] - above[j - 1])
    return float(j - 1 + t + 0.5)


def impact(args, torch, T):
    """Compound drop falling onto a wetting cylinder at full size (1024 x 2048,
    R_cyl = 120, core R = 60, shell R = 100, fully periodic), for We = 1, 10,
    50 with cylinder angles 90 deg: `impact_steps` steps each in FP64, FP32 and
    shifted-FP16 storage.  MLUPS of each; the FP32 and FP16 results' errors
    against the FP64 one (which equals the oracle to 1e-12): order-parameter
    max error, u and p max error relative to their scale, mass drift of fluids
    1 and 2, the film thickness on the cylinder top (0 before the drop
    touches it) and the thickness of the fluid-3 cushion between drop and
    cylinder top (`cushion_gap`).  Then an angle sweep (30..150 deg, We = 10, FP32 storage)
    timed over the same steps."""
    import workloads as W
    n0 = args.impact_steps
    out = {"workload": "compound_drop_on_cylinder_1024x2048, periodic, cylinder R = 120 (curved wetting wall), "
                       "core R = 60, shell R = 100, 48 lattice units between shell and cylinder at the start",
           "We": {}}
    for We in (1.0, 10.0, 50.0):
        w = W.compound_drop_on_cylinder(1024, 2048, We=We)
        col = w.nx // 2
        y_top = int(max(y for y in range(w.ny) if w.mask[y, col]))
        contact = int(48.0 / w.meta["U"])  # steps until the falling shell reaches the cylinder top
        n = max(n0, contact + 1500) if contact + 1500 <= args.impact_max_steps else n0
        fields = {}
        fluid = float((w.mask == 0).sum()) / (w.nx * w.ny)
        res = {"U": round(w.meta["U"], 5), "Re": round(w.meta["Re"], 1), "steps": n,
               "contact_step_estimate": contact, "fluid_fraction": round(fluid, 5)}
        for prec in ("fp64", "fp32", "fp16"):
            L = T.lattice_from_workload(w, prec)
            m0 = np.array(L.diagnostics()["mass"])
            L.step(3)
            L.sync()
            ms = time_steps(L, n, torch, torch.cuda.current_stream())
            res[prec + "_mlups"] = round(w.nx * w.ny * n / (ms / 1e3) / 1e6, 1)
            res[prec + "_fluid_mlups"] = round(fluid * w.nx * w.ny * n / (ms / 1e3) / 1e6, 1)
            fields[prec] = L.fields(("c1", "c2", "ux", "uy", "p"))
            res[prec + "_gap"] = round(cushion_gap(fields[prec], col, y_top), 4)
            m1 = np.array(L.diagnostics()["mass"])
            res[prec + "_mass_drift"] = [float(f"{v:.3g}") for v in np.abs(m1[:2] - m0[:2]) / np.abs(m0[:2])]
            res[prec + "_film_h"] = round(L.film_thickness(col, y_top, 3), 6)
            L.close()
        ref = fields["fp64"]
        for prec in ("fp32", "fp16"):
            a = fields[prec]
            err = {"c_abs": float(max(np.abs(a[k] - ref[k]).max() for k in ("c1", "c2")))}
            for k in ("ux", "uy", "p"):
                err[k + "_rel"] = float(np.abs(a[k] - ref[k]).max() / max(float(np.abs(ref[k]).max()), 1e-12))
            err["film_h_abs"] = abs(res[prec + "_film_h"] - res["fp64_film_h"])
            err["gap_abs"] = abs(res[prec + "_gap"] - res["fp64_gap"])
            res[prec + "_vs_fp64"] = {k: float(f"{v:.3g}") for k, v in err.items()}
        out["We"][f"{We:g}"] = res
    sweep = {}
    n = n0
    out["angle_sweep_steps"] = n
    for th in (30.0, 60.0, 90.0, 120.0, 150.0):
        w = W.compound_drop_on_cylinder(1024, 2048, We=10.0, theta=th)
        L = T.lattice_from_workload(w, "fp32")
        L.step(3)
        L.sync()
        ms = time_steps(L, n, torch, torch.cuda.current_stream())
        sweep[f"{th:g}"] = round(w.nx * w.ny * n / (ms / 1e3) / 1e6, 1)
        L.close()
    out["angle_sweep_fp32_mlups"] = sweep
    return out


def shear(args, torch, T):
    """Compound drop on a wetting wall sheared by the velocity lid (512 x 256,
    the full 20000 steps), FP64 and FP32 storage: MLUPS of each, and the FP32
    result's error against the FP64 one (which equals the oracle to 1e-12) and
    the FP32 mass drift of fluids 1 and 2 (the lid row holds fluid 3 only)."""
    import workloads as W
    w = W.compound_drop_shear()
    n = args.shear_steps
    out = {"workload": f"{w.name}, lid U0 = 0.01, densities 1:2:1", "steps": n}
    fields = {}
    for prec in ("fp64", "fp32"):
        L = T.lattice_from_workload(w, prec)
        m0 = np.array(L.diagnostics()["mass"])
        ms = time_steps(L, n, torch, torch.cuda.current_stream())
        out[prec + "_mlups"] = round(w.nx * w.ny * n / (ms / 1e3) / 1e6, 1)
        fields[prec] = L.fields()
        if prec == "fp32":
            m1 = np.array(L.diagnostics()["mass"])
            out["fp32_mass_drift"] = [float(f"{v:.3g}") for v in np.abs(m1[:2] - m0[:2]) / np.abs(m0[:2])]
        L.close()
    a, b = fields["fp32"], fields["fp64"]
    err = {k: float(np.abs(a[k] - b[k]).max()) for k in ("c1", "c2", "c3")}
    for k in ("ux", "uy", "p"):
        err[k + "_rel"] = float(np.abs(a[k] - b[k]).max() / max(float(np.abs(b[k]).max()), 1e-12))
    out["fp32_vs_fp64"] = {k: float(f"{v:.3g}") for k, v in err.items()}
    return out


def served(args, torch, T):
    """The served workload: Poisson arrivals (20 requests/s, seed 1710) of
    drop-on-wall and drop-on-cylinder jobs, sides log-uniform 128..serve_hi,
    steps log-uniform serve_steps_lo..serve_steps_hi (defaults: the full
    configuration, 200 requests, 128..2048, 1000..20000 steps), FP32 and
    shifted-FP16 storage alternating, admitted by device footprint against an
    HBM budget; time to result (p50, p99), aggregate MLUPS over the whole run,
    the GPU's busy share of it and the tile shapes the tuner picked."""
    import workloads as W
    from paper_1710_09534_gb300.serve import Request, Server, poisson_arrivals
    hi, slo, shi = args.serve_hi, args.serve_steps_lo, args.serve_steps_hi
    jobs = W.served_requests(args.serve_count, seed=1710, lo=128, hi=hi, steps_lo=slo, steps_hi=shi)
    t_arr = poisson_arrivals(len(jobs), 20.0, seed=1710)
    # every other request asks for shifted-FP16 storage; the server keeps one batch per precision
    reqs = [Request(i, w, s, "fp16" if i % 2 else "fp32", float(t)) for i, ((w, s), t) in enumerate(zip(jobs, t_arr))]
    srv = Server(int(args.serve_budget_gb * 1e9), max_lattices=256, chunk=200)
    stats = srv.run(reqs)
    srv.close()
    out = stats.summary()
    out["workload"] = (f"{len(reqs)} requests, Poisson 20/s (seed 1710), sides 128..{hi}, steps {slo}..{shi}, "
                       f"FP32 and shifted-FP16 alternating, HBM budget {args.serve_budget_gb} GB")
    return out


def d3q19(args, torch, T, fp64_peak=None):
    """The D3Q19 form: tiled hemispherical drops of fluids 1 and 2 on a
    wetting wall, periodic in x and z; whole steps (three launches each)
    timed with CUDA events on the lattice's stream, each launch timed apart
    (tlb3_profile) for the roofline of the update kernel (FP64: bound by the
    FP64 unit; FP32 storage: by HBM, on 2 (57 + 6) 4 B per node); and the
    c_1, c_2 mass drift over the timed steps."""
    import workloads as W
    nx, ny, nz = (int(v) for v in args.d3_size.split(","))
    w = W.drops3d_on_wall(nx, ny, nz)
    L = T.lattice3_from_workload(w)
    stream = torch.cuda.current_stream()
    L.step(max(args.warmup, 3))
    L.sync()
    m0 = np.array(L.diagnostics()["mass"])
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    L.step(args.d3_steps)
    ev[1].record(stream)
    ev[1].synchronize()
    ms = ev[0].elapsed_time(ev[1])
    m1 = np.array(L.diagnostics()["mass"])
    # the same number of steps again with each launch bracketed by events
    L.profile(True)
    L.step(args.d3_steps)
    kms, kn = L.profile_read()
    L.profile(False)
    n = nx * ny * nz
    fluid = n  # drops3d_on_wall has no solid nodes (the wall is an edge)
    L.close()
    # the general update (per-node density and viscosity): fluid 2 three times denser
    wg = W.drops3d_on_wall(nx, ny, nz)
    wg.params.update(rho2=3.0, nu1=0.08, nu2=0.12)
    G = T.lattice3_from_workload(wg)
    G.step(3)
    G.sync()
    ng = max(10, args.d3_steps // 4)
    ev[0].record(stream)
    G.step(ng)
    ev[1].record(stream)
    ev[1].synchronize()
    gms = ev[0].elapsed_time(ev[1])
    G.close()
    # FP32 storage and arithmetic (rest populations as float pairs), the same lattice
    F = T.lattice3_from_workload(w, precision="fp32")
    F.step(3)
    F.sync()
    fm0 = np.array(F.diagnostics()["mass"])
    F.profile(True)
    ev[0].record(stream)
    F.step(args.d3_steps)
    ev[1].record(stream)
    ev[1].synchronize()
    fms = ev[0].elapsed_time(ev[1])
    fk, fn = F.profile_read()
    F.profile(False)
    fm1 = np.array(F.diagnostics()["mass"])
    F.close()
    fupd = fk[2] / max(fn[2], 1)
    f32_bytes = 2 * (57 + 6) * 4
    upd_ms = kms[2] / max(kn[2], 1)
    dp_inst, flops = FP64_DP3["uniform"]
    ach = fluid * flops / (upd_ms / 1e3) / 1e12
    peak, src = fp64_peak if fp64_peak else measured_fp64_peak(T)
    return {"workload": w.name, "nx": nx, "ny": ny, "nz": nz, "precision": "fp64", "steps": args.d3_steps,
            "value": round(n * args.d3_steps / (ms / 1e3) / 1e6, 2), "unit": "MLUPS",
            "ms_per_step": round(ms / args.d3_steps, 4),
            "kernel_ms": {"k3_csum": round(kms[0] / max(kn[0], 1), 4), "k3_mu": round(kms[1] / max(kn[1], 1), 4),
                          "k3_update": round(upd_ms, 4)},
            "roofline": {"bound": "alu", "kernel": "k3_update<uniform>", "achieved": round(ach, 4),
                         "peak": round(peak, 4), "unit": "TFLOP/s", "frac": round(ach / peak, 4),
                         "peak_source": src, "dp_inst_per_node": dp_inst, "flops_per_node": flops,
                         "dp_issue_frac": round(fluid * dp_inst / (upd_ms / 1e3) / FP64_DP_INST_PEAK, 4),
                         "algorithmic_bytes_per_node": 2 * (57 + 6) * 8,
                         "hbm_achieved_gbs": round(fluid * 2 * (57 + 6) * 8 / (upd_ms / 1e3) / 1e9, 1)},
            "gpu_launches": 3 * args.d3_steps,
            "mass_drift": [float(f"{v:.3g}") for v in np.abs(m1[:2] - m0[:2]) / np.abs(m0[:2])],
            "general": {"value": round(n * ng / (gms / 1e3) / 1e6, 2), "unit": "MLUPS", "steps": ng,
                        "update": "general (rho = 1, 3, 1; nu = 0.08, 0.12, 0.1)"},
            "fp32": {"value": round(n * args.d3_steps / (fms / 1e3) / 1e6, 2), "unit": "MLUPS",
                     "steps": args.d3_steps, "ms_per_step": round(fms / args.d3_steps, 4),
                     "kernel_ms": {"k3_csum": round(fk[0] / max(fn[0], 1), 4),
                                   "k3_mu": round(fk[1] / max(fn[1], 1), 4), "k3_update": round(fupd, 4)},
                     "roofline": {"bound": "hbm", "kernel": "k3_update<float, uniform>",
                                  "algorithmic_bytes_per_node": f32_bytes,
                                  "achieved": round(fluid * f32_bytes / (fupd / 1e3) / 1e9, 1),
                                  "peak": peaks()[0], "unit": "GB/s",
                                  "frac": round(fluid * f32_bytes / (fupd / 1e3) / 1e9 / peaks()[0], 4)},
                     "hbm_roofline_pct_whole_step": round(100 * n * args.d3_steps / (fms / 1e3) * f32_bytes
                                                          / (peaks()[0] * 1e9), 2),
                     "mass_drift": [float(f"{v:.3g}") for v in np.abs(fm1[:2] - fm0[:2]) / np.abs(fm0[:2])]}}


def e2e(L, w, args, torch, T):
    """Whole jobs through the C ABI with host buffers: each job sets the
    fields from pinned host arrays (tlb_set_fields copies them to the
    device), runs K steps and reads all 10 fields back into pinned host
    memory (tlb_read_fields); the copies are inside the timed region.
    Reported: six jobs over two lattices on two streams, one host thread per
    lattice (the C calls release the interpreter lock), so that one job's
    copies overlap the other's steps; beside it, two jobs one after the
    other on one lattice."""
    import threading
    n = w.nx * w.ny
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float64)).pin_memory()
    ins = [pin(a) for a in (w.c1, w.c2, w.ux, w.uy)]
    h2d = int(4 * n * 8 / args.steps)
    d2h = int(10 * n * 8 / args.steps)
    # one after the other
    out = torch.empty((10, w.ny, w.nx), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(2):
        L.set_fields(*(t.numpy() for t in ins))
        L.step(args.steps)
        L.fields(out=out.numpy())
    torch.cuda.synchronize()
    seq = n * args.steps * 2 / (time.perf_counter() - t0) / 1e6
    ref = out.clone()
    # two lattices, two streams, one host thread each
    dev = torch.device("cuda", torch.cuda.current_device())
    lats = [T.lattice_from_workload(w, args.precision, stream=torch.cuda.Stream(dev)) for _ in range(2)]
    outs = [torch.empty((10, w.ny, w.nx), dtype=torch.float64).pin_memory() for _ in lats]
    per = 3
    errors = []

    def worker(Lx, ox):
        try:
            for _ in range(per):
                Lx.set_fields(*(t.numpy() for t in ins))
                Lx.step(args.steps)
                Lx.fields(out=ox.numpy())
        except Exception as e:  # reported below, after the timing
            errors.append(repr(e))

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    threads = [threading.Thread(target=worker, args=(Lx, ox)) for Lx, ox in zip(lats, outs)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    dt = time.perf_counter() - t0
    if errors:
        raise RuntimeError(f"e2e worker failed: {errors[0]}")
    same = all(bool(torch.equal(o, ref)) for o in outs)
    for Lx in lats:
        Lx.close()
    jobs = per * len(lats)
    return {"value": round(n * args.steps * jobs / dt / 1e6, 2), "unit": "MLUPS",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "job": f"tlb_set_fields (4 FP64 planes from pinned host memory) + {args.steps} steps + tlb_read_fields "
                   f"(10 FP64 planes into pinned host memory); {jobs} jobs over 2 lattices on 2 streams, "
                   f"one host thread each",
            "results_equal_sequential": same,
            "sequential": {"value": round(seq, 2), "unit": "MLUPS", "job": "2 jobs one after the other, one lattice"}}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
