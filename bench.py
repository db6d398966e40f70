#!/usr/bin/env python
"""Benchmark of the hydrothermal time step on one GB300.

Workload (default, city_q1): the city-scale workload, 10 km x 10 km x 200 m,
512 x 512 x 96 Q1 cells (25,527,393 nodes per field), layered + Gaussian
random lnK (the Table 3 soils), 20,000 energy piles and 50 basement / subway
heat sources, dt = 1 day, both linear systems solved to relative residual
1e-10.  A "step" is one backward-Euler step: loads, head CG solve, heat
BiCGStab solve.  Other workloads: pile_q1 (256 x 256 x 64 Q1, 1000 piles),
ates_q2 (128 x 128 x 32 Q2, well pair), plain_q1 (16^3 Q1), ates_table1 (the
hot-water injection benchmark of Section 2 on a graded quarter mesh,
266 x 266 x 90 Q1, wellbore flux and temperature).

Printed metric: simulated years per hour of the FP32-inner / FP64-outer form
(value), with the plain FP64 form beside it and the relative L2 difference
of the two forms' fields, operator GDoF/s and the roofline of the dominant
kernel (the head CG iteration).

--impl reference times the CPU FP64 oracle (the plain assembled-matrix
reference) on bounded samples of the same workload.
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

if "--impl" in sys.argv and "reference" in sys.argv:
    # the oracle arm runs single-threaded; say so truthfully in "cores"
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import scenarios as S  # noqa: E402

YEAR = 365.0 * 86400.0
METRIC = "simulated-years/hour at 1e-10 residual (FP32-inner/FP64-outer; plain FP64 beside it)"
UNIT = "sim-years/h"


WORKLOADS = {"city_q1": S.config5, "pile_q1": S.config3, "ates_q2": S.config2, "plain_q1": S.config1,
             "ates_table1": S.ates_table1}


def workload(name):
    if name in WORKLOADS:
        return WORKLOADS[name]()
    if name.startswith("ates_q2_"):          # e.g. ates_q2_32 -> 32x32x8 cells
        n = int(name.split("_")[-1])
        return S.config2(nx=n, ny=n, nz=max(2, n // 4))
    if name.startswith("city_q1_"):          # e.g. city_q1_128 -> 128x128x24 cells
        n = int(name.split("_")[-1])
        return S.config5(nx=n, ny=n, nz=max(2, (3 * n) // 16))
    if name.startswith("pile_q1_"):          # e.g. pile_q1_64 -> 64x64x16 cells
        n = int(name.split("_")[-1])
        return S.config3(nx=n, ny=n, nz=max(2, n // 4))
    raise SystemExit(f"unknown workload {name}")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    out = {"hbm_gbs": 6800.0, "source": "fallback", "sm_max_mhz": 2070.0}
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        out.update(hbm_gbs=float(d["hbm_gbs"]), source="measured",
                   sm_max_mhz=float(d.get("sm_max_mhz", 2070.0)))
    # ALU peaks derived from unit counts and the maximum SM clock:
    # FP32: 152 SMs x 128 lanes x 2 flop/FMA; FP64: GB300 nominal 1.25 TFLOP/s.
    out["fp32_tflops"] = 152 * 128 * 2 * out["sm_max_mhz"] * 1e6 / 1e12
    out["fp64_tflops"] = 1.25
    return out


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 7:
                    continue
                try:
                    sm.append(float(parts[0]))
                    mx.append(float(parts[1]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[3:7]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        except Exception:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def apply_flops_per_node(order):
    """Algorithmic FLOPs of one head-operator apply per node: per cell, the
    six one-dimensional sweeps of the fast diagonalisation (12 n^4 flops,
    n = p + 1) plus the scaling and accumulation of the n^3 local values,
    spread over the nodes of a cell (one per Q1 cell, eight per Q2 cell)."""
    if order == 1:
        return 242.0
    return 143.0


def apply_bytes_per_node(order, fp32):
    w = 4 if fp32 else 8
    cells_per_node = 1.0 if order == 1 else 1.0 / 8.0
    return 2 * w + w * cells_per_node


def heat_apply_bytes(order, nn, nc):
    """Algorithmic DRAM bytes of one FP64 heat-operator apply: x read and y
    written (16 bytes per node) and the Darcy velocity at the (p+1)^3 Gauss
    points of every cell (three FP64 components each); the uniform c_T and
    lambda are scalars."""
    return 16.0 * nn + 24.0 * (order + 1) ** 3 * nc


def cg_bytes(order, nn, nc, graded=False):
    """Algorithmic DRAM bytes of one FP32 head CG iteration of the kernel
    the library runs for this order.

    Q1, the single-pass iteration of the single-reduction CG: it reads x, r,
    p and the cell conductivity K and writes x, r, p; the Jacobi diagonal is
    formed from K and A p from p on chip, so nothing else is stored:
    4 (6 nn + nc) bytes.

    Q2, the fused two-pass iteration: the operator apply (x in, y out, K per
    cell: 4 (2 nn + nc)) plus the CG vector work of three vectors read and
    three written (24 bytes per node); the element buffer between the passes
    is the split's own intermediate, not the method's, and is not counted.

    A graded mesh runs the fused two-pass iteration for either order and
    reads each cell's geometry besides (volume and 1/h per axis: 16 bytes
    per cell)."""
    if graded:
        return 4.0 * (2 * nn + nc) + 24.0 * nn + 16.0 * nc
    if order == 1:
        return 4.0 * (6 * nn + nc)
    return 4.0 * (2 * nn + nc) + 24.0 * nn


def cg_kernel_source(order):
    return "ht_q1.cu" if order == 1 else "ht_ops.cu"


def measured_traffic(workload, order):
    """DRAM bytes per CG iteration from the committed ncu summary, if it was
    taken on this workload and the kernel source has not changed since
    (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "cg_iteration_traffic.json")
    src = os.path.join(ROOT, "paper_2103_00081_gb300", "csrc", cg_kernel_source(order))
    try:
        with open(path) as f:
            recs = json.load(f)
        with open(src, "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except (OSError, ValueError):
        return None
    for d in recs if isinstance(recs, list) else [recs]:
        if d.get("source_sha256") == sha and d.get("workload") == workload:
            return d.get("dram_bytes_per_iteration")
    return None


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def arm_config(sc, world):
    """The workload description shared by both arms of the benchmark."""
    return {"workload": f"{sc.name} {sc.nx}x{sc.ny}x{sc.nz} Q{sc.order}, {sc.n_nodes} nodes/field, "
                        f"dt={sc.dt / 86400:g} d, tol 1e-10",
            "nodes_per_field": sc.n_nodes, "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "working set per step > L2 (no flush needed)"}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    import torch.distributed as dist
    backend = "nccl"
    dist.init_process_group(backend=backend)
    return dist.get_rank(), ws, dist


def run_ours(args):
    import torch
    from paper_2103_00081_gb300 import build as B
    B.build()
    from paper_2103_00081_gb300 import hydro
    from paper_2103_00081_gb300 import _lib as L
    from paper_2103_00081_gb300 import replicas as R

    rank, world, dist = dist_init()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    sc = workload(args.workload)
    dt = sc.dt
    nn, nc = sc.n_nodes, sc.n_cells
    stream = torch.cuda.Stream(device=local)
    pk = peaks()
    lib = L.lib()
    fp64_peak = ctypes_peak(lib, local, fp64=True)
    fp32_peak = ctypes_peak(lib, local, fp64=False)

    def barrier():
        if dist:
            dist.barrier()

    # the choice the autotuner makes on these workloads; used as is with --no-autotune
    tuned = dict(apply_variant=L.HT_APPLY_AUTO, krylov=L.HT_KRYLOV_BICGSTAB, precond=L.HT_PREC_JACOBI)
    if sc.spacing is not None:
        # the graded ATES mesh: FP32 BiCGStab breaks down next to the wellbore
        # (non-finite iterates); GMRES(100) converges
        tuned["krylov"] = L.HT_KRYLOV_GMRES
    tune_table = []
    if not args.no_autotune:
        from paper_2103_00081_gb300 import autotune as AT

        def factory(opts):
            return hydro.Simulator.from_scenario(sc, device=local, stream=stream.cuda_stream, tol=1e-10,
                                                 precision=L.HT_MIXED, inner_tol=args.inner_tol,
                                                 inner_tol_heat=args.inner_tol_heat,
                                                 max_iter=200000, **opts)
        tuned, tune_table = AT.tune(factory, dt, AT.signature(sc.nx, sc.ny, sc.nz, sc.order, L.HT_MIXED),
                                    candidates=AT.default_candidates(L.HT_MIXED, sc.order), force=args.retune)

    def timed_run(precision):
        extra = tuned if precision == L.HT_MIXED else {}
        sim = hydro.Simulator.from_scenario(sc, device=local, stream=stream.cuda_stream,
                                            tol=1e-10, precision=precision, inner_tol=args.inner_tol,
                                            inner_tol_heat=args.inner_tol_heat,
                                            max_iter=200000, **extra)
        for _ in range(args.warmup):
            sim.step(dt)
        torch.cuda.synchronize()
        sim.profile(True)
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stats = []
        with Clocks(local) as clk:
            e0.record(stream)
            for _ in range(args.steps):
                stats.append(sim.step(dt))
            e1.record(stream)
            torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        barrier()
        prof = sim.profile_read()
        sim.profile(False)
        fields = (sim.get_field(S.HEAD), sim.get_field(S.TEMP))
        return sim, ms, stats, prof, clk.summary(), fields

    # --- mixed precision (the headline form) --------------------------------
    sim, ms_mixed, st_mixed, prof_mixed, clk, f_mixed = timed_run(L.HT_MIXED)
    # --- end to end through the C ABI with host buffers ---------------------
    h_host = np.ascontiguousarray(f_mixed[0])
    T_host = np.ascontiguousarray(f_mixed[1])
    torch.cuda.synchronize()
    t_now = sim.time
    w0 = time.perf_counter()
    for _ in range(args.steps):
        sim.set_state(h_host, T_host, t_now)
        sim.step(dt)
        h_host = sim.get_field(S.HEAD)
        T_host = sim.get_field(S.TEMP)
        t_now += dt
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - w0
    sim.close()
    # --- mixed precision with the learned initial guess ---------------------
    learned = None
    if not args.no_learned and sc.order == 1:
        learned = learned_leg(args, sc, tuned, stream, local, st_mixed)
    # --- plain FP64 over the same steps --------------------------------------
    ms_fp64 = None
    if not args.no_fp64:
        sim64, ms_fp64, st_fp64, prof_fp64, clk64, f_fp64 = timed_run(L.HT_FP64)
        sim64.close()

    # max over ranks of the timed duration; each rank stepped its own replica
    vals = [ms_mixed, e2e_s] + ([ms_fp64] if ms_fp64 is not None else [])
    vals = R.max_over_ranks(vals, dist, f"cuda:{local}")
    ms_mixed, e2e_s = vals[0], vals[1]
    if ms_fp64 is not None:
        ms_fp64 = vals[2]
    if rank != 0:
        return
    years_all = args.steps * dt / YEAR * world
    rate_mixed = R.job_rate(years_all, ms_mixed / 1000.0 / 3600.0)
    rate_e2e = R.job_rate(years_all, e2e_s / 3600.0)

    order = sc.order
    # dominant kernel: the FP32 head CG iteration, bracketed by CUDA events on
    # the library's stream over its check intervals
    n_cg = prof_mixed["cg_iters"]
    avg_cg = prof_mixed["cg_iter_ms"] / max(n_cg, 1)
    n_bi = prof_mixed["bicgstab_iters"]
    avg_bi = prof_mixed["bicgstab_iter_ms"] / max(n_bi, 1)
    graded = sc.spacing is not None
    bytes_cg = cg_bytes(order, nn, nc, graded)
    wl_name = f"{sc.name} {sc.nx}x{sc.ny}x{sc.nz} Q{order}"
    kname = ("fused Jacobi-CG iteration on a graded mesh, FP32 (fcg_cell_kernel + fcg_node_kernel)" if graded else
             "single-pass Jacobi-CG iteration, FP32 (q1_cg_kernel, one launch)" if order == 1 else
             "fused Jacobi-CG iteration, FP32 (fcg_cell_kernel + fcg_node_kernel)")
    achieved = bytes_cg / (avg_cg / 1e3) / 1e9 if n_cg and avg_cg > 0 else None
    roof = {
        "kernel": kname,
        "bound": "hbm",
        "achieved": achieved,
        "peak": pk["hbm_gbs"],
        "unit": "GB/s",
        "frac": achieved / pk["hbm_gbs"] if achieved else None,
        "traffic": None if graded else measured_traffic(wl_name, order),
        "algorithmic_bytes": bytes_cg,
        "avg_launch_us": avg_cg * 1e3 if n_cg else None,
        "launches": n_cg,
        "peak_source": f"HBM {pk['hbm_gbs']:.0f} GB/s ({pk['source']}, burst copy)",
    }
    # None when no check interval of the heat solves was all working iterations
    heat_iter = {"kernel": "fused Jacobi-BiCGStab iteration, FP32 (2 heat applies)",
                 "avg_us": avg_bi * 1e3 if n_bi else None, "iterations": n_bi}
    its_h = [s["iters_head"] for s in st_mixed]
    its_T = [s["iters_heat"] for s in st_mixed]
    line = {
        "metric": METRIC,
        "value": rate_mixed,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_mixed / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32-inner/f64-outer",
        "data": "synthetic (seeded layered + Gaussian lnK, piles, heat sources)",
        "config": arm_config(sc, world),
        "iters_head": its_h, "iters_heat": its_T,
        "initial_guess": {f: {"extrapolated": sum(s[f"guess_{f}"] == 2 for s in st_mixed),
                              "previous": sum(s[f"guess_{f}"] == 0 for s in st_mixed)} for f in ("head", "heat")},
        "outer_head": [s["outer_head"] for s in st_mixed],
        "res_head": max(s["res_head"] for s in st_mixed), "res_heat": max(s["res_heat"] for s in st_mixed),
        "ms_split": {k: sum(s[k] for s in st_mixed) / args.steps for k in ("ms_loads", "ms_head", "ms_heat")},
        "operator_gdofs": {"fp32_cg_iteration": nn / (avg_cg / 1e3) / 1e9 if n_cg and avg_cg > 0 else None},
        "roofline": roof,
        "heat_iteration": heat_iter,
        "e2e": {"value": rate_e2e, "unit": UNIT, "h2d_bytes_per_step": 2 * nn * 8,
                "d2h_bytes_per_step": 2 * nn * 8},
        "gpu_launches": prof_mixed["launches"],
        "autotuned": {"opts": tuned, "candidates": [[o, t, st] for o, t, st in tune_table]},
        "measured_alu_peaks_tflops": {"fp64": fp64_peak, "fp32": fp32_peak},
        "clocks": clk,
    }
    if ms_fp64 is not None:
        rate_fp64 = R.job_rate(years_all, ms_fp64 / 1000.0 / 3600.0)
        n64 = prof_fp64["head_applies"]
        avg64 = prof_fp64["head_apply_ms"] / max(n64, 1)
        flops = apply_flops_per_node(order) * nn
        bytes64 = apply_bytes_per_node(order, False) * nn
        line["plain_fp64"] = {
            "value": rate_fp64, "unit": UNIT, "ms_per_step": ms_fp64 / args.steps,
            "iters_head": [s["iters_head"] for s in st_fp64], "iters_heat": [s["iters_heat"] for s in st_fp64],
            "roofline": {"kernel": "head operator apply (FP64, tiled)", "bound": "alu",
                         "achieved": flops / (avg64 / 1e3) / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                         "frac": flops / (avg64 / 1e3) / 1e12 / fp64_peak if fp64_peak else None,
                         "peak_source": "FP64 FMA chains on this GPU (ht_fma_peak, measured in this run)",
                         "avg_launch_us": avg64 * 1e3, "launches": n64,
                         "hbm_achieved_gbs": bytes64 / (avg64 / 1e3) / 1e9,
                         "hbm_frac": bytes64 / (avg64 / 1e3) / 1e9 / pk["hbm_gbs"]},
            "clocks": clk64}
        nh = prof_fp64["heat_applies"]
        if nh > 0 and prof_fp64["heat_apply_ms"] > 0:
            avgh = prof_fp64["heat_apply_ms"] / nh
            bh = heat_apply_bytes(order, nn, nc)
            # no flop count is derived for the Gauss-point advection, so only
            # the bandwidth side of this apply is reported
            line["plain_fp64"]["heat_apply"] = {
                "kernel": "heat operator apply (FP64, Darcy velocity at the Gauss points)",
                "avg_launch_us": avgh * 1e3, "launches": nh, "gdofs": nn / (avgh / 1e3) / 1e9,
                "algorithmic_bytes": bh, "hbm_achieved_gbs": bh / (avgh / 1e3) / 1e9,
                "hbm_frac": bh / (avgh / 1e3) / 1e9 / pk["hbm_gbs"]}
        line["speedup_vs_fp64"] = rate_mixed / rate_fp64 if rate_fp64 > 0 else None
        # the two forms from the same initial state after the same steps
        line["mixed_vs_fp64_rel_l2"] = {"head": rel_l2(f_mixed[0], f_fp64[0]),
                                        "temperature": rel_l2(f_mixed[1], f_fp64[1]),
                                        "temperature_change": rel_l2(f_mixed[1] - sc.T0, f_fp64[1] - sc.T0)}
        line["operator_gdofs"]["fp64_head_apply"] = nn / (avg64 / 1e3) / 1e9
    if learned is not None:
        line["learned"] = learned
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sc, args.workload)
    if args.workload == "city_q1" and world == 1 and not args.no_batch:
        line["batch64"] = batch_subrun()
    print(json.dumps(line))


def batch_subrun(timeout_s=300):
    """The batched workload (64 uneven Q1 problems, `--workload batch64`) run
    in a child process after the timed region, so that its figures travel
    with the default line; a failure of the child is recorded, not raised."""
    cmd = [sys.executable, os.path.abspath(__file__), "--workload", "batch64", "--steps", "3", "--warmup", "3"]
    try:
        p = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s, cwd=ROOT)
    except subprocess.TimeoutExpired:
        return {"error": f"timed out after {timeout_s} s", "command": " ".join(["bench.py"] + cmd[2:])}
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    if p.returncode != 0 or not lines:
        tail = (p.stderr or p.stdout).strip().splitlines()[-1:] or [""]
        return {"error": f"exit {p.returncode}: {tail[0][:200]}", "command": " ".join(["bench.py"] + cmd[2:])}
    d = json.loads(lines[-1])
    keep = ("metric", "value", "unit", "mode", "ms_per_step", "steps", "warmup", "config", "sequential",
            "concurrent", "shared_launches", "speedup_vs_sequential", "gpu_launches")
    out = {k: d[k] for k in keep if k in d}
    out["command"] = " ".join(["bench.py"] + cmd[2:])
    return out


def learned_leg(args, sc, tuned, stream, local, st_plain):
    """The learned initial guess (spec addition): the U-Net is trained
    with the library's kernels on trajectories of the pile-field workload
    (256 x 256 x 64 Q1, a different generator and mesh), then attached to the
    workload being measured; the same timed steps as the mixed leg, with the
    gate choosing per field and step between the prediction and the guess the
    step takes without it (the extrapolated field, or the field at t^n).
    Training is not part of the timed region."""
    import torch
    from paper_2103_00081_gb300 import hydro, learned as LG
    from paper_2103_00081_gb300 import _lib as L
    opts = dict(tol=1e-10, precision=L.HT_MIXED, inner_tol=args.inner_tol, inner_tol_heat=args.inner_tol_heat,
                max_iter=200000, **tuned)
    t0 = time.perf_counter()
    train_sc = S.config3()
    tsim = hydro.Simulator.from_scenario(train_sc, device=local, stream=stream.cuda_stream, **opts)
    samples = LG.collect_samples(tsim, train_sc.dt, args.learn_steps)
    tsim.close()
    t1 = time.perf_counter()
    net = LG.UNet(device=local, seed=0)
    losses = LG.train(net, samples, epochs=args.learn_epochs, lr=1e-3)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    del samples
    sim = hydro.Simulator.from_scenario(sc, device=local, stream=stream.cuda_stream, **opts)
    LG.attach(sim, net)
    for _ in range(max(args.warmup, 3)):
        sim.step(sc.dt)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stats = [sim.step(sc.dt) for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # the network's forward pass alone, on this workload's padded grid
    D, H, W = ((sim.dims[2] + 7) // 8 * 8, (sim.dims[1] + 7) // 8 * 8, (sim.dims[0] + 7) // 8 * 8)
    x = torch.zeros((LG.FEATURES, D, H, W), dtype=torch.float32, device=f"cuda:{local}")
    y = torch.empty((2, D, H, W), dtype=torch.float32, device=f"cuda:{local}")
    import ctypes
    lib = L.lib()
    ustream = torch.cuda.current_stream(local)
    for _ in range(2):
        lib.ht_unet_forward(net._h, ctypes.c_void_p(x.data_ptr()), D, H, W, ctypes.c_void_p(y.data_ptr()))
    torch.cuda.synchronize()
    f0 = time.perf_counter()
    for _ in range(3):
        lib.ht_unet_forward(net._h, ctypes.c_void_p(x.data_ptr()), D, H, W, ctypes.c_void_p(y.data_ptr()))
    torch.cuda.synchronize()
    fwd_ms = (time.perf_counter() - f0) / 3 * 1e3
    del ustream
    sim.close()
    net.close()
    flops = unet_forward_flops(D * H * W)
    return {"value": (args.steps * sc.dt / YEAR) / (ms / 1000.0 / 3600.0), "unit": UNIT,
            "ms_per_step": ms / args.steps,
            "iters_head": [s["iters_head"] for s in stats], "iters_heat": [s["iters_heat"] for s in stats],
            "iters_head_without": [s["iters_head"] for s in st_plain],
            "iters_heat_without": [s["iters_heat"] for s in st_plain],
            "gate_wins": {"head": sum(s["guess_head"] == 1 for s in stats),
                          "heat": sum(s["guess_heat"] == 1 for s in stats)},
            "unet_forward_ms": fwd_ms, "unet_forward_tflops": flops / (fwd_ms * 1e-3) / 1e12,
            "unet_grid": [D, H, W],
            "training": {"workload": f"{train_sc.name} {train_sc.nx}x{train_sc.ny}x{train_sc.nz} Q1",
                         "samples": args.learn_steps - 2, "epochs": args.learn_epochs,
                         "loss_first_last": [losses[0], losses[-1]], "sampling_s": t1 - t0, "training_s": t2 - t1}}


def unet_forward_flops(voxels):
    """Multiply-add FLOPs (2 per MAC) of one forward pass of the library's
    U-Net on a grid of `voxels` voxels: the 3x3x3 layers at their levels plus
    the 1x1 output layer."""
    c1, c2, c3, c4 = 16, 32, 48, 64
    lv = [(16, c1), (c1, c1), (c2 + c1, c1), (c1, c1)]                  # level 1 (input padded to 16)
    l2 = [(c1, c2), (c2, c2), (c3 + c2, c2), (c2, c2)]
    l3 = [(c2, c3), (c3, c3), (c4 + c3, c3), (c3, c3)]
    l4 = [(c3, c4), (c4, c4)]
    f = 0.0
    for lay, div in ((lv, 1), (l2, 8), (l3, 64), (l4, 512)):
        f += sum(2.0 * 27 * ci * co for ci, co in lay) * voxels / div
    return f + 2.0 * c1 * 2 * voxels


def ctypes_peak(lib, device, fp64):
    import ctypes
    v = ctypes.c_double()
    return v.value if lib.ht_fma_peak(int(device), int(bool(fp64)), ctypes.byref(v)) == 0 else None


def oracle_samples(wl, sc_full):
    """Bounded samples of the workload for the CPU oracle: the same domain,
    physics and sources on coarser meshes."""
    if sc_full.order == 2:
        return [S.config2(nx=n, ny=n, nz=max(2, n // 4)) for n in (24, 40)]
    if sc_full.name.startswith("city"):
        return [S.config5(nx=n, ny=n, nz=(3 * n) // 16) for n in (48, 80)]
    if sc_full.name.startswith("pile"):
        return [S.config3(nx=n, ny=n, nz=n // 4) for n in (48, 80)]
    if sc_full.name.startswith("ates_table1"):
        return [S.ates_table1(n_bore=nb, n_out=no, nz_aquifer=na, nz_confining=nc)
                for nb, no, na, nc in ((4, 20, 6, 4), (6, 34, 10, 6))]
    return [S.config1(nx=n) for n in (8, 16)]


def oracle_solver(sc):
    """The oracle's solver for the samples of a workload: Jacobi-PCG /
    BiCGStab to 1e-10, except on the graded ATES benchmark, whose
    advection-dominated heat system breaks scipy's BiCGStab down; its
    samples (below 40k nodes) take the oracle's direct sparse solve."""
    return "direct" if sc.name.startswith("ates_table1") else "iterative"


def cpu_info():
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "hardware") and model is None:
                    model = line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    # Arm CPUs report a part number instead of a model name
    parts = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1"}
    if model in parts:
        model = f"{parts[model]} (CPU part {model})"
    return {"nproc": os.cpu_count(), "model": model, "machine": platform.machine()}


def time_oracle_sample(sc, steps):
    """Seconds per step of the oracle (assembled CSR, Jacobi-PCG / BiCGStab
    to 1e-10) on scenario sc after one untimed step."""
    from oracle import fem
    o = fem.OracleSim(sc, solver=oracle_solver(sc), tol=1e-10)
    o.step(sc.dt)
    t0 = time.perf_counter()
    for _ in range(steps):
        o.step(sc.dt)
    return (time.perf_counter() - t0) / steps, o


THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _oracle_replica(payload):
    """One oracle replica (a child process): seconds of its second step on
    the sample scenario."""
    sc, solver = payload
    from oracle import fem
    o = fem.OracleSim(sc, solver=solver, tol=1e-10)
    o.step(sc.dt)
    t0 = time.perf_counter()
    o.step(sc.dt)
    return time.perf_counter() - t0


def oracle_all_cores(sc, n_procs=None, timeout_s=240.0):
    """The oracle on every host core at once: one independent single-threaded
    replica of the sample per core (spawned processes), each timing one step
    while all run.  Returns (cores, slowest replica's seconds per step);
    raises on a failure or after timeout_s (the pool is then terminated)."""
    import multiprocessing as mp
    n = n_procs or os.cpu_count() or 1
    saved = {k: os.environ.get(k) for k in THREAD_VARS}
    for k in THREAD_VARS:
        os.environ[k] = "1"
    # by module name, so that the children find it also when this file runs as __main__
    import importlib
    fn = importlib.import_module("bench")._oracle_replica
    try:
        with mp.get_context("spawn").Pool(n) as pool:
            times = pool.map_async(fn, [(sc, oracle_solver(sc))] * n).get(timeout_s)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return n, max(times)


def cpu_baseline(sc_full, wl, steps=1):
    """The oracle timed on two coarser samples of the workload; the cost per
    step is extrapolated to the full mesh with the power law in node count
    fitted through the two samples (it carries the growth of the iteration
    counts along with the matrix size)."""
    samples = oracle_samples(wl, sc_full)
    t, n = [], []
    o = None
    for sc in samples:
        ts, o = time_oracle_sample(sc, steps)
        t.append(ts)
        n.append(sc.n_nodes)
    k = float(np.log(t[1] / t[0]) / np.log(n[1] / n[0])) if t[1] > 0 and t[0] > 0 else 1.0
    k = max(k, 1.0)                     # never below linear growth
    s_full = t[1] * (sc_full.n_nodes / n[1]) ** k
    rate = (sc_full.dt / YEAR) / (s_full / 3600.0)
    return {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"{steps} step(s) each of {', '.join(f'{sc.nx}x{sc.ny}x{sc.nz} Q{sc.order} ({sc.n_nodes} nodes)' for sc in samples)}"
                       f" of {sc_full.name}, "
                       + ("direct sparse LU" if oracle_solver(sc_full) == "direct" else "Jacobi-PCG/BiCGStab to 1e-10")
                       + " on assembled CSR (scipy, one thread); "
                       f"extrapolated to {sc_full.n_nodes} nodes by the fitted law s/step ~ nodes^{k:.2f}"),
            "s_per_step_samples": t, "nodes_samples": n, "exponent": k, "s_per_step_full_extrapolated": s_full,
            "host": cpu_info(), "spmv": oracle_spmv_rate(o, samples[-1]),
            "all_cores": all_cores_figure(sc_full, samples[-1], k)}


def all_cores_figure(sc_full, sample, k):
    """Aggregate oracle throughput with every host core busy: independent
    replicas (the oracle does not parallelise one run), each extrapolated to
    the full mesh by the single-core law; a failure is recorded, not raised."""
    try:
        cores, s_rep = oracle_all_cores(sample)
    except Exception as e:   # noqa: BLE001 -- the baseline must not stop the benchmark
        return {"error": f"{type(e).__name__}: {str(e)[:160]}"}
    s_full = s_rep * (sc_full.n_nodes / sample.n_nodes) ** k
    return {"value": cores * (sc_full.dt / YEAR) / (s_full / 3600.0), "unit": UNIT, "cores": cores,
            "kind": "oracle replicas, one per core (aggregate throughput; one run is no faster)",
            "s_per_step_sample_under_load": s_rep}


def oracle_spmv_rate(o, sc, reps=5):
    """The oracle's assembled head-operator SpMV on the sample: GB/s counted
    as CSR values and column indices (12 B per nonzero) plus x read and y
    written (16 B per row), best of `reps`."""
    from oracle import fem
    A = fem.constrain(o.head_matrix(sc.dt), o.dmask[fem.HEAD])
    x = np.random.default_rng(0).standard_normal(A.shape[0])
    best = float("inf")
    for _ in range(reps):
        t0 = time.perf_counter()
        A @ x
        best = min(best, time.perf_counter() - t0)
    nbytes = 12.0 * A.nnz + 16.0 * A.shape[0]
    return {"gbs": nbytes / best / 1e9, "nnz": int(A.nnz), "rows": int(A.shape[0]), "seconds": best}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sc_full = workload(args.workload)
    samples = oracle_samples(args.workload, sc_full)
    # each reference step: one oracle step on each sample, the full-size cost
    # extrapolated as in the cpu_baseline; warm-up steps untimed
    t, n = [], []
    o = None
    for sc in samples:
        from oracle import fem
        o = fem.OracleSim(sc, solver=oracle_solver(sc), tol=1e-10)
        for _ in range(args.warmup):
            o.step(sc.dt)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            o.step(sc.dt)
        t.append((time.perf_counter() - t0) / args.steps)
        n.append(sc.n_nodes)
    k = max(float(np.log(t[1] / t[0]) / np.log(n[1] / n[0])), 1.0)
    s_full = t[1] * (sc_full.n_nodes / n[1]) ** k
    rate = (sc_full.dt / YEAR) / (s_full / 3600.0)
    cb = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
          "sample": (f"{args.steps} step(s) each of {', '.join(f'{sc.nx}x{sc.ny}x{sc.nz}' for sc in samples)} "
                     f"of {sc_full.name}; extrapolated to {sc_full.n_nodes} nodes by s/step ~ nodes^{k:.2f}"),
          "s_per_step_samples": t, "nodes_samples": n, "host": cpu_info(), "spmv": oracle_spmv_rate(o, samples[-1])}
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": s_full * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded layered + Gaussian lnK, piles, heat sources)",
        "config": arm_config(sc_full, args.gpus), "cpu_baseline": cb,
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_batch(args):
    """Batched workload: 64 independent Q1 problems (32x32x16 .. 96x96x48)
    advanced together by ht_batch_step, against the same problems stepped one
    after another; value = simulated years per hour summed over problems.
    With N ranks the problems are dealt round-robin over the GPUs (no
    data-path collective) and the slowest rank's time is the job's."""
    import torch
    from paper_2103_00081_gb300 import build as B
    B.build()
    from paper_2103_00081_gb300 import hydro
    from paper_2103_00081_gb300 import _lib as L
    from paper_2103_00081_gb300 import replicas as R
    rank, world, dist = dist_init()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    scs_all = S.config4(n_problems=args.batch_size)
    if len(scs_all) < world:
        raise SystemExit(f"--batch-size {len(scs_all)} is smaller than the {world} ranks")
    scs = [scs_all[i] for i in R.shard(len(scs_all), rank, world)]
    opts = dict(tol=1e-10, precision=L.HT_MIXED, inner_tol=1e-4, krylov=L.HT_KRYLOV_BICGSTAB)
    sims = [hydro.Simulator.from_scenario(sc, device=local, **opts) for sc in scs]
    dt = scs[0].dt

    def barrier():
        if dist:
            dist.barrier()

    def timed_batch(mode):
        batch = hydro.Batch(sims, mode=mode)
        for _ in range(args.warmup):
            batch.step(dt)
        for sm in sims:
            sm.profile(True)
        torch.cuda.synchronize()
        barrier()
        w0 = time.perf_counter()
        for _ in range(args.steps):
            stats = batch.step(dt)
        torch.cuda.synchronize()
        t = time.perf_counter() - w0
        barrier()
        launches = sum(sm.profile_read()["launches"] for sm in sims)
        for sm in sims:
            sm.profile(False)
        batch.close()
        return t, stats, launches

    # concurrent per-problem steps (the default), then the shared-launch head CG
    t_batch, stats, _ = timed_batch(L.HT_BATCH_CONCURRENT)
    t_shared, _, _ = timed_batch(L.HT_BATCH_SHARED_LAUNCHES)
    t_pers, stats_p, launches = timed_batch(L.HT_BATCH_PERSISTENT)
    # the same problems stepped one by one through ht_step
    barrier()
    w0 = time.perf_counter()
    for _ in range(args.steps):
        for sm in sims:
            sm.step(dt)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - w0
    dev = f"cuda:{local}"
    t_batch, t_shared, t_pers, t_seq = R.max_over_ranks([t_batch, t_shared, t_pers, t_seq], dist, dev)
    (launches,) = R.sum_over_ranks([launches], dist, dev)
    if rank != 0:
        return
    years = args.steps * dt / YEAR * len(scs_all)
    nodes = sum(sc.n_nodes for sc in scs_all)
    # the headline is the persistent mode (one cooperative launch per outer
    # pass for the inner head CG of all problems); the other modes beside it
    print(json.dumps({
        "metric": "simulated-years/hour summed over the batch at 1e-10 residual",
        "value": R.job_rate(years, t_pers / 3600), "mode": "persistent",
        "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_pers / args.steps * 1e3, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "f32-inner/f64-outer", "data": "synthetic (seeded GRF lnK, piles)",
        "config": {"workload": f"{len(scs_all)} Q1 problems, {nodes} nodes in total, dt=1 d, tol 1e-10",
                   "sizes": sorted(set(f"{sc.nx}x{sc.ny}x{sc.nz}" for sc in scs_all))[:8],
                   "parallelism": "problems dealt round-robin over ranks" if world > 1 else "single GPU"},
        "sequential": {"value": R.job_rate(years, t_seq / 3600), "ms_per_step": t_seq / args.steps * 1e3},
        "shared_launches": {"value": R.job_rate(years, t_shared / 3600),
                            "ms_per_step": t_shared / args.steps * 1e3},
        "concurrent": {"value": R.job_rate(years, t_batch / 3600), "ms_per_step": t_batch / args.steps * 1e3,
                       "iters_head": [st["iters_head"] for st in stats][:8]},
        "speedup_vs_sequential": t_seq / t_pers,
        "iters_head": [st["iters_head"] for st in stats_p][:8], "gpu_launches": int(launches),
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="city_q1")
    ap.add_argument("--inner-tol", dest="inner_tol", type=float, default=1e-5,
                    help="FP32 inner-solve reduction floor, head system")
    ap.add_argument("--inner-tol-heat", dest="inner_tol_heat", type=float, default=1e-4,
                    help="FP32 inner-solve reduction floor, heat system")
    ap.add_argument("--no-fp64", dest="no_fp64", action="store_true", help="skip the plain FP64 leg")
    ap.add_argument("--no-learned", dest="no_learned", action="store_true", help="skip the learned-guess leg")
    ap.add_argument("--learn-steps", dest="learn_steps", type=int, default=14,
                    help="steps of the pile-field trajectory that give training samples (two fewer samples)")
    ap.add_argument("--learn-epochs", dest="learn_epochs", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", dest="no_cpu_baseline", action="store_true")
    ap.add_argument("--no-autotune", dest="no_autotune", action="store_true")
    ap.add_argument("--no-batch", dest="no_batch", action="store_true",
                    help="skip the batched workload that the default run adds after its own line's legs")
    ap.add_argument("--retune", action="store_true", help="ignore the autotuning cache")
    ap.add_argument("--batch-size", dest="batch_size", type=int, default=64)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
