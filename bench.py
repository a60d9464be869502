"""Benchmark: PCG solves/sec to relative residual 1e-8 on one GB300.

One step = one pass of the whole path on one synthetic cell configuration:
collision graph -> per-contact friction coefficients -> friction blocks ->
maximum spanning forest -> tree factor -> PCG solve of Gamma v = F.
Inputs are resident in HBM when the timed region starts (``value``); the
``e2e`` figure repeats the step through the public API from pinned host
buffers, with the host<->device copies inside the timed region.

Default workload: a spheroid of 1,000,000 cells (centres uniform in a ball
at packing fraction 0.6, radii U[0.45, 0.55]), per-pair gamma_par and
gamma_perp log-uniform in [0.1, 10], gamma0 = 1e-3, F ~ N(0, 1), solved to
relative residual 1e-8 with the spanning-forest preconditioner.  The timed
form (``value``) is the mixed-precision one (FP32 inner PCG inside FP64
iterative refinement); the same line reports plain FP64 PCG and FP64
block-Jacobi PCG on the same workload (``forms``), timed after the main
region.

``--impl reference`` times the CPU oracle instead (host cores, a bounded
sample of the same workload).  Under torchrun each rank solves its own
independent replica (weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "PCG solves/sec to rel-res 1e-8 (% HBM roofline); chosen form vs plain FP64, 1 GB300"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (non-tensor) nominal rate


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
WORKLOADS = {
    "ball1m": dict(desc="spheroid of 1,000,000 cells, ball at packing 0.6, radii U[0.45,0.55], "
                        "gamma log-uniform [0.1,10] per pair, gamma0=1e-3, F~N(0,1)",
                   make=lambda seed: workloads.ball(n=1_000_000, seed=seed, gamma0=1e-3)),
    "cube1k": dict(desc="1,000 cells uniform in a cube of side 8.886, radii U[0.45,0.55], "
                        "gamma log-uniform [0.1,10], gamma0=1e-2",
                   make=lambda seed: workloads.cube(n=1000, side=8.886, seed=seed)),
    "hex4m": dict(desc="monolayer of 4,000,000 cells, 2000x2000 jittered hexagonal lattice a=0.9, "
                       "radii U[0.48,0.52], gamma log-uniform [0.01,100], gamma0=1e-4",
                  make=lambda seed: workloads.hex_sheet(nx=2000, ny=2000, seed=seed)),
}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# replicas: one independent system per rank, no data-path collective
# ---------------------------------------------------------------------------
def replica_seed(rank: int) -> int:
    """Seed of rank `rank`'s replica of the workload (rank 0: the default)."""
    return 2000 + rank


def max_over_ranks(x: float, device=None) -> float:
    """MAX of a per-rank value over the default process group (the slowest
    rank's time); the value itself without a group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world: int, steps: int, max_elapsed_s: float) -> float:
    """Whole-job solves per second: every rank solved `steps` systems, the job
    took as long as its slowest rank."""
    return world * steps / max_elapsed_s


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def tree_bytes(n: int, npairs: int, nrecv: int, fp: int) -> int:
    """Algorithmic bytes of one tree solve (forward + backward, all levels).
    Forward: per L block its contributor id, the block and the contributor's
    w; per receiver entry its id, its contributor range and w read+write.
    Backward: per vertex its id, pair range, D^-1 and w read+write; per L
    block the receiver id, the block and the receiver's z."""
    wb, lb, db = 3 * fp, 9 * fp, 6 * fp
    fwd = npairs * (4 + lb + wb) + nrecv * (8 + 2 * wb)
    bwd = n * (8 + db + 2 * wb) + npairs * (4 + lb + wb)
    return fwd + bwd


def binned_bytes(n: int, npairs: int, nrecv: int, nleak: int, ntop: int, fp: int) -> int:
    """Algorithmic bytes of one fused step around the binned tree solve
    (its forward, leak-sum, top and backward launches).  Vectors: the
    forward launch reads r and q and writes r and the forward values, the
    backward launch reads them and r (for r^T z) and writes z; the top reads
    r, q and its leak sums, writes r and z.  Blocks: every L block once in
    each pass, D^-1 once.  Leaks: each product written and read, each top
    sum written and read.  Indices: per forward entry its receiver and
    contributor start, per pair its contributor / receiver reference, per
    leak its source and slot, per cell its pair start."""
    w = 3 * fp
    vec = 7 * w * (n - ntop) + 5 * w * ntop
    blocks = 2 * 9 * fp * npairs + 6 * fp * n
    leaks = 2 * w * nleak + 2 * w * ntop
    idx = 8 * nrecv + 8 * npairs + 8 * nleak + 4 * n
    return vec + blocks + leaks + idx


def update_bytes(n: int, fp: int) -> int:
    """Bytes of the fused step's last launch: x += alpha p, p = z + beta p
    (reads x, p, z, writes x, p)."""
    return 5 * 3 * fp * n


def vector_bytes(n: int, fp: int, precond: str) -> int:
    """Algorithmic bytes of the vector kernels of one PCG iteration (3n
    entries each): the update reads p, q, r, x and writes x, r and the
    preconditioner's input w; the tree form adds r^T z (reads r, w) and the
    direction update p = z + beta p (reads z, p, writes p)."""
    e = 3 * n * fp
    return 7 * e + (2 * e + 3 * e if precond == "tree" else 3 * e)


def outer_bytes(n: int, m: int) -> int:
    """Algorithmic bytes of one FP64 refinement step of the mixed solve: the
    FP64 residual (blocks and columns, row pointer, v, F, r) and the FP32
    scaling and accumulation of the inner correction."""
    return 2 * m * 52 + n * (4 + 4 * 24) + n * (24 + 12 + 12) + n * (12 + 24 + 24)


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
# the current kernels on the default workload and form, one kernel per ncu
# capture, one launch each (profiles/dram_fused_step_ball1m.md): the tree
# step is its four launches (k_bin_fwd 87.77 MB, k_leaksum 0.17 MB, k_top
# 0.22 MB, k_bin_bwd 107.91 MB); other workloads and forms report null.
FP64_TFLOPS = 1.25   # FP64 FMA rate of the GB300 (no FP64 tensor path is used)

MEASURED_TRAFFIC = {
    ("ball1m", "mixed", "tree"): {"spmv": 136916992, "tree": 196094464, "vector": 36145920},
}


def spmv_bytes(n: int, m: int, fp: int) -> int:
    """Algorithmic bytes of one product q = Gamma p with p^T q: per directed
    slot the symmetric block (6 words) and the column in FP64, or the eq. (1)
    form (g_perp, g_par - g_perp, u: 5 floats) and the column in FP32 (24
    bytes); per row the row pointer, p_i and q_i."""
    slot = 6 * fp + 4 if fp == 8 else 24
    return 2 * m * slot + n * (4 + 3 * fp + 3 * fp)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    import paper_2410_04512_gb300 as sgp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks, peaks_src = load_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))

    wl = WORKLOADS[args.workload]
    cells = wl["make"](replica_seed(rank))   # each rank: its own independent replica
    n = cells.n
    F_host = cells.forces()
    tp, tq = cells.tables()
    pos = torch.from_numpy(cells.pos).to(dev)
    radii = torch.from_numpy(cells.radii).to(dev)
    F = torch.from_numpy(F_host).to(dev)
    tpd, tqd = torch.from_numpy(tp).to(dev), torch.from_numpy(tq).to(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = sgp.Context(local, stream)
    PREC = {"f64": sgp.PREC_F64, "mixed": sgp.PREC_MIXED}
    PRECOND = {"tree": sgp.PRECOND_TREE, "jacobi": sgp.PRECOND_BLOCK_JACOBI, "none": sgp.PRECOND_NONE}

    class Form:
        """One solver form with its own reusable handles."""

        def __init__(self, precision: str, precond: str):
            self.precision, self.precond = PREC[precision], PRECOND[precond]
            self.H = {"g": None, "M": None, "T": None, "Fh": None}
            self.last = None

        def step(self, pos_d, radii_d, F_d, out_v):
            H = self.H
            H["g"] = ctx.collision_graph(pos_d, radii_d, H["g"])
            ij = H["g"].edges()
            gp, gq = workloads.pair_gamma_torch(cells.seed, ij, tpd, tqd)
            H["M"] = ctx.friction_assemble(H["g"], pos_d, gp.contiguous(), gq.contiguous(), cells.gamma0,
                                           self.precision, H["M"])
            if self.precond == sgp.PRECOND_TREE:
                H["T"] = ctx.max_spanning_tree(H["M"], H["T"])
                H["Fh"] = ctx.tree_factor(H["M"], H["T"], H["Fh"])
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            _, info = ctx.pcg_solve(H["M"], H["Fh"], F_d, out_v, tol=args.tol, precond=self.precond,
                                    precision=self.precision)
            ev1.record(stream)
            self.last = (info, ev0, ev1)
            return info

        def timed(self, steps: int, warmup: int, kernel_timing: bool):
            v = torch.zeros_like(F)
            for _ in range(warmup):
                self.step(pos, radii, F, v)
            torch.cuda.synchronize()
            if world > 1:
                dist.barrier()
            ctx.set_kernel_timing(kernel_timing)
            for k in (sgp.KT_SPMV, sgp.KT_TREE_SOLVE, sgp.KT_PCG_VECTOR):
                ctx.kernel_time(k, reset=True)
            ctx.launch_count(reset=True)
            solve_ms, iters = [], []
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(steps):
                info = self.step(pos, radii, F, v)
                _, a, b = self.last
                b.synchronize()
                solve_ms.append(a.elapsed_time(b))
                iters.append(info.iterations)
            t1.record(stream)
            torch.cuda.synchronize()
            elapsed = t0.elapsed_time(t1) / 1e3
            kt = {k: ctx.kernel_time(k) for k in (sgp.KT_SPMV, sgp.KT_TREE_SOLVE, sgp.KT_PCG_VECTOR)}
            launches = ctx.launch_count()
            ctx.set_kernel_timing(False)
            elapsed = max_over_ranks(elapsed, dev)
            return dict(elapsed=elapsed, solve_ms=float(np.median(solve_ms)), iters=float(np.mean(iters)),
                        iters_total=int(np.sum(iters)), steps=steps, info=self.last[0], kt=kt,
                        launches=launches, v=v)

    # ---- timed region: the chosen form, device-resident inputs ------------
    chosen = Form(args.precision, args.precond)
    tuning = None
    if args.autotune:
        # launch shapes picked by the library's autotuner on this workload
        # (outside the timed region; the factor is rebuilt every step anyway)
        chosen.step(pos, radii, F, torch.zeros_like(F))
        tuning = ctx.autotune(chosen.H["M"], chosen.H["T"], chosen.H["Fh"], F, precond=chosen.precond,
                              precision=chosen.precision, iterations=0, tol=args.tol)
    with ClockSampler(local) as clk:
        # `value`: the timed steps with nothing inside them but the step.
        # Per-kernel CUDA events (event nodes in the captured iteration
        # graphs) cut the programmatic-dependent-launch overlap between
        # kernels, so the kernel averages of the rooflines come from the same
        # number of steps repeated right after with the events switched on.
        res = chosen.timed(args.steps, args.warmup, kernel_timing=False)
        kres = chosen.timed(args.steps, 0, kernel_timing=True)
    elapsed = res["elapsed"]
    value = replica_throughput(world, args.steps, elapsed)
    info = res["info"]

    # ---- end to end through the public API from pinned host buffers -------
    pos_h = torch.from_numpy(cells.pos).pin_memory()
    rad_h = torch.from_numpy(cells.radii).pin_memory()
    F_h = torch.from_numpy(F_host).pin_memory()
    v_h = torch.empty_like(F_h).pin_memory()
    pos_e, rad_e, F_e, v_e = torch.empty_like(pos), torch.empty_like(radii), torch.empty_like(F), torch.empty_like(F)
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        pos_e.copy_(pos_h, non_blocking=True)
        rad_e.copy_(rad_h, non_blocking=True)
        F_e.copy_(F_h, non_blocking=True)
        chosen.step(pos_e, rad_e, F_e, v_e)
        v_h.copy_(v_e, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_s = e0.elapsed_time(e1) / 1e3
    e2e_s = max_over_ranks(e2e_s, dev)
    e2e_value = replica_throughput(world, e2e_steps, e2e_s)

    # ---- rooflines of the per-iteration kernels ----------------------------
    M = chosen.H["M"]
    m = M.m
    fp = 4 if chosen.precision == sgp.PREC_MIXED else 8

    def roof(name, bytes_per, total_ms, launches, unit_note, traffic_bytes=None):
        avg_s = (total_ms / max(launches, 1)) / 1e3
        gbs = bytes_per / avg_s / 1e9 if avg_s > 0 else 0.0
        return {"kernel": name, "bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(gbs / hbm_peak, 4), "traffic": traffic_bytes,
                "peak_source": ("measured (MEASURED_PEAKS.json hbm_gbs)" if peaks_src == "measured"
                                else "fallback"),
                "algorithmic_bytes_per_launch": int(bytes_per), "avg_launch_us": round(avg_s * 1e6, 2),
                "launches": launches, "unit_of_work": unit_note}

    def form_rooflines(form, kres, label=""):
        """Rooflines of a form's kernel classes from its timed repeat: the
        product, the tree step (fused binned solve, or the level kernels),
        and the vector updates (per iteration)."""
        H = form.H
        fpx = 4 if form.precision == sgp.PREC_MIXED else 8
        tn = "float" if fpx == 4 else "double"
        mm = H["M"].m
        traffic = MEASURED_TRAFFIC.get((args.workload, "mixed" if fpx == 4 else "f64", "tree"), {})
        spmv_ms, spmv_n = kres["kt"][sgp.KT_SPMV]
        tree_ms, tree_n = kres["kt"][sgp.KT_TREE_SOLVE]
        vec_ms, _ = kres["kt"][sgp.KT_PCG_VECTOR]
        its = max(int(kres["iters_total"]), 1)   # iterations of every timed step
        out = {"spmv": roof(label + "k_spmv_pq<%s>" % tn, spmv_bytes(n, mm, fpx), spmv_ms, spmv_n,
                            "one product Gamma p + p^T q over all rows", traffic.get("spmv"))}
        if fpx == 8:
            # FP64 is issue-bound on this GPU: the product against the FP64
            # rate too (per slot 9 FMA + 3 subtractions, per row 3 FMA for
            # gamma0 and 3 for p^T q)
            flops = 2 * mm * (2 * 9 + 3) + n * (2 * 3 + 2 * 3)
            avg_s = (spmv_ms / max(spmv_n, 1)) / 1e3
            tf = flops / avg_s / 1e12 if avg_s > 0 else 0.0
            out["spmv_alu"] = {"kernel": label + "k_spmv_pq<double> (FP64 arithmetic)", "bound": "alu",
                               "achieved": round(tf, 4), "peak": FP64_TFLOPS, "unit": "TFLOP/s",
                               "frac": round(tf / FP64_TFLOPS, 4), "traffic": None,
                               "peak_source": "nominal FP64 rate (152 SMs x 2 FMA/clock x 2070 MHz; an FMA loop "
                                              "measured 1.20 TFLOP/s)",
                               "algorithmic_flops_per_launch": int(flops), "avg_launch_us": round(avg_s * 1e6, 2),
                               "launches": spmv_n}
        it_bytes = spmv_bytes(n, mm, fpx)
        if form.precond == sgp.PRECOND_TREE:
            _, levels, npairs, nrecv = H["Fh"].stats()
            lay = H["Fh"].layout()
            if lay["fp32" if fpx == 4 else "fp64"]:
                tb = binned_bytes(n, npairs, nrecv, lay["leaks"], lay["top"], fpx)
                out["tree"] = roof(label + "fused tree step (k_bin_fwd, k_leaksum, k_top, k_bin_bwd <%s>; %d bins, "
                                   "top %d)" % (tn, lay["bins"], lay["top"]), tb, tree_ms, tree_n,
                                   "one application of P^-1 with r -= alpha q, |r|^2 and r^T z (four launches)",
                                   traffic.get("tree"))
                vb = update_bytes(n, fpx)
                out["vector"] = roof(label + "k_pupd_x<%s> (class time also holds the solve's start and the "
                                     "refinement's residual kernels)" % tn, vb, vec_ms, its,
                                     "x += alpha p, p = z + beta p, per iteration", traffic.get("vector"))
            else:
                tb = tree_bytes(n, npairs, nrecv, fpx)
                out["tree"] = roof(label + "tree solve (level kernels <%s>, %d levels)" % (tn, levels), tb,
                                   tree_ms, tree_n, "one application of P^-1 (all levels)")
                vb = vector_bytes(n, fpx, "tree")
                out["vector"] = roof(label + "PCG vector kernels <%s>" % tn, vb, vec_ms, its,
                                     "update, r^T z and direction kernels, per iteration")
            it_bytes += tb + vb
        else:
            vb = vector_bytes(n, fpx, "jacobi")
            out["vector"] = roof(label + "PCG vector kernels <%s>" % tn, vb, vec_ms, its,
                                 "update with the block-Jacobi product, per iteration")
            it_bytes += vb
        return out, it_bytes

    roofmap, it_bytes = form_rooflines(chosen, kres)
    names = list(roofmap)
    dominant = max(names, key=lambda k: roofmap[k]["avg_launch_us"] * roofmap[k]["launches"])
    # the solve against the bandwidth roofline: algorithmic bytes of all its
    # iterations (product + tree step + vector updates) and refinement steps
    solve_bytes = res["iters"] * it_bytes + (info.outer_iterations + 1) * outer_bytes(n, m) * (fp == 4)
    roof_ms = solve_bytes / (hbm_peak * 1e9) * 1e3
    solve_roof = {"bytes": int(solve_bytes), "bytes_per_inner_iteration": int(it_bytes),
                  "roof_ms": round(roof_ms, 3), "measured_ms": round(res["solve_ms"], 3),
                  "frac": round(roof_ms / res["solve_ms"], 4), "peak_gbs": hbm_peak}
    roof_other = [roofmap[k] for k in names if k != dominant]
    tree_layout = chosen.H["Fh"].layout() if chosen.precond == sgp.PRECOND_TREE else None

    # ---- the other forms on the same workload (outside the timed region) --
    forms = {}
    if rank == 0 and args.compare:
        ctx.set_tuning()      # the other forms run with the built-in launch shapes
        for label, prec, pc, steps in (("plain_fp64_mst", "f64", "tree", 2), ("fp64_block_jacobi", "f64", "jacobi", 1)):
            if (prec, pc) == (args.precision, args.precond):
                continue
            f = Form(prec, pc)
            r = f.timed(steps, 1, kernel_timing=False)
            forms[label] = {"solves_per_s": round(steps / r["elapsed"], 4),
                            "solve_only_per_s": round(1e3 / r["solve_ms"], 4),
                            "iterations": int(round(r["iters"])),
                            "true_rel_residual": r["info"].true_rel_residual}
            if label == "plain_fp64_mst":
                kr = f.timed(1, 0, kernel_timing=True)
                rm, _ = form_rooflines(f, kr, "plain FP64 form: ")
                roof_other += list(rm.values())
        if "plain_fp64_mst" in forms:
            forms["chosen_vs_plain_fp64"] = round(value / forms["plain_fp64_mst"]["solves_per_s"], 3)

    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(elapsed / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if fp == 8 else "f32+f64",
        "data": "synthetic",
        "config": {"workload": wl["desc"], "n_cells": n, "edges": int(m), "mean_degree": round(2.0 * m / n, 3),
                   "form": "%s precision, %s preconditioner" % (args.precision, args.precond),
                   "tol": args.tol,
                   "step": "collision graph + friction blocks + spanning forest + tree factor + PCG solve",
                   "l2": "working set > L2 (friction blocks alone %.0f MB: FP64 %s)"
                         % (2 * m * (52 + (24 if fp == 4 else 0)) / 1e6, "and FP32 records" if fp == 4 else "only"),
                   "parallelism": "replicas" if world > 1 else "single"},
        "iterations": int(round(res["iters"])), "true_rel_residual": info.true_rel_residual,
        "outer_iterations": info.outer_iterations,
        "solve_only": {"value": round(1e3 / res["solve_ms"], 4), "unit": "solves/s",
                       "ms_median": round(res["solve_ms"], 3)},
        "e2e": {"value": round(e2e_value, 4), "unit": "solves/s", "h2d_bytes_per_step": h2d_bytes(pos, radii, F),
                "d2h_bytes_per_step": F.numel() * 8, "steps": e2e_steps},
        "gpu_launches": int(res["launches"]),
        "roofline": roofmap[dominant], "roofline_other": roof_other,
        "solve_roofline": solve_roof, "tree_layout": tree_layout,
        "time_share_ms": {"spmv": round(kres["kt"][sgp.KT_SPMV][0], 2),
                          "tree_solve": round(kres["kt"][sgp.KT_TREE_SOLVE][0], 2),
                          "vector": round(kres["kt"][sgp.KT_PCG_VECTOR][0], 2),
                          "timed": round(kres["elapsed"] * 1e3, 2),
                          "note": "kernel events over a repeat of the timed steps (%d steps, %.2f solves/s "
                                  "with the events on)" % (args.steps, args.steps / kres["elapsed"])},
        "forms": forms,
        "tuning": tuning if tuning is not None else ctx.get_tuning(),
        "clocks": clk.summary(),
    }
    if rank == 0 and args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, forms.get("plain_fp64_mst", {}).get("iterations"))
    if rank == 0 and world == 1 and args.configs and args.workload == "ball1m":
        line["configs"] = other_configs(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def other_configs(args):
    """The other configurations of the benchmark's set, each run as its own
    bench.py process with short step counts (built-in launch shapes): the
    1000-cell cube, the 4e6-cell sheet against plain FP64, the 512-spheroid
    batch against looped solves, the learned warm start.  A compact record
    of each goes into the main line."""
    runs = [("cube1k", ["--workload", "cube1k", "--steps", "20", "--compare", "1"]),
            ("hex4m", ["--workload", "hex4m", "--steps", "2", "--compare", "1"]),
            ("batch512", ["--workload", "batch512", "--steps", "2"]),
            ("warm200k", ["--workload", "warm200k"]),
            ("aug1m", ["--workload", "aug1m", "--steps", "2"]),
            ("local1m", ["--workload", "local1m", "--steps", "3"]),
            ("paper", ["--workload", "paper", "--paper-reps", "3"])]
    out = {}
    for name, extra in runs:
        cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--warmup", "3", "--autotune", "0",
               "--cpu-baseline", "0", "--configs", "0"] + extra
        t0 = time.perf_counter()
        try:
            p = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
            rec = None
            for ln in p.stdout.splitlines():
                if ln.startswith("{"):
                    rec = json.loads(ln)
            if rec is None:
                out[name] = {"error": (p.stderr or p.stdout)[-400:]}
                continue
        except subprocess.TimeoutExpired:
            out[name] = {"error": "timed out"}
            continue
        keep = {k: rec[k] for k in ("value", "unit", "ms_per_step", "iterations", "true_rel_residual",
                                    "outer_iterations", "true_rel_residual_max", "solve_only", "forms",
                                    "latency_ms", "looped_plain_fp64", "looped_mixed", "learned", "zero_guess",
                                    "previous_v", "solve_only_ms_mean", "tree_layout", "clocks", "augmented",
                                    "plain_fp64", "outer_vs_plain_iterations", "augmented_sweep",
                                    "error_bound_stopping", "paper_workloads", "hex_scaling", "global_forest",
                                    "local_forests", "best_local_vs_global_step", "paper_hex_1e5_tol_1e-5")
                if k in rec}
        keep["workload"] = rec.get("config", {}).get("workload")
        if "roofline" in rec:
            keep["roofline"] = {k: rec["roofline"][k] for k in ("kernel", "achieved", "frac", "avg_launch_us")}
            keep["roofline_other"] = [{k: r[k] for k in ("kernel", "achieved", "frac", "avg_launch_us")}
                                      for r in rec.get("roofline_other", [])]
        if "solve_roofline" in rec:
            keep["solve_roofline_frac"] = rec["solve_roofline"]["frac"]
        keep["run_s"] = round(time.perf_counter() - t0, 1)
        out[name] = keep
    return out


def h2d_bytes(*ts) -> int:
    return int(sum(t.numel() * t.element_size() for t in ts))


def run_batch(args):
    """The batched workload: 512 independent spheroids with N log-uniform in
    [1e3, 1e5] (the cube workload's density and law), solved together per
    step (batched graph, assembly, spanning forest, factor, batched PCG),
    against a loop of single plain-FP64 solves of the same instances."""
    import torch

    import paper_2410_04512_gb300 as sgp

    dev = torch.device("cuda", 0)
    sizes = workloads.batch_sizes(args.batch, seed=4000)
    off = workloads.sphere_offsets(sizes)
    cells = [workloads.batch_instance(int(n), s) for s, n in enumerate(sizes)]
    pos_h = np.ascontiguousarray(np.concatenate([c.pos for c in cells]))
    rad_h = np.ascontiguousarray(np.concatenate([c.radii for c in cells]))
    n = int(off[-1])
    F_h = np.random.Generator(np.random.PCG64([4000, 7919])).standard_normal((n, 3))
    pos, radii, F = (torch.from_numpy(a).to(dev) for a in (pos_h, rad_h, F_h))
    t = torch.from_numpy(workloads.gamma_table(0.1, 10.0)).to(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = sgp.Context(0, stream)
    prec = sgp.PREC_MIXED if args.precision == "mixed" else sgp.PREC_F64
    H = {"g": None, "M": None, "T": None, "Fh": None}

    def step(v):
        H["g"] = ctx.collision_graph_batched(off, pos, radii, H["g"])
        ij = H["g"].edges()
        gp, gq = workloads.pair_gamma_torch(4000, ij, t, t)
        H["M"] = ctx.friction_assemble(H["g"], pos, gp.contiguous(), gq.contiguous(), 1e-2, prec, H["M"])
        H["T"] = ctx.max_spanning_tree(H["M"], H["T"])
        H["Fh"] = ctx.tree_factor(H["M"], H["T"], H["Fh"])
        return ctx.pcg_solve_batched(H["M"], H["Fh"], off, F, v, tol=args.tol, precision=prec)[1]

    v = torch.zeros_like(F)
    tuning = None
    if args.autotune:
        step(v)
        tuning = ctx.autotune(H["M"], H["T"], H["Fh"], F, offsets=off, precision=prec, iterations=0, tol=args.tol)
    for _ in range(args.warmup):
        step(v)
    torch.cuda.synchronize()
    ctx.launch_count(reset=True)
    with ClockSampler(0) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            infos = step(v)
        e1.record(stream)
        torch.cuda.synchronize()
    elapsed = e0.elapsed_time(e1) / 1e3
    launches = ctx.launch_count()
    step_s = elapsed / args.steps
    its = np.array([i.iterations for i in infos])
    res = np.array([i.true_rel_residual for i in infos])

    # the single-system solver looped over the same instances, one at a
    # time (built-in launch shapes): plain FP64, and the batch's own
    # precision (isolating what batching gains)
    ctx.set_tuning()

    def looped(pr):
        lat = []
        Hs = {"g": None, "M": None, "T": None, "Fh": None}
        for s in range(len(cells)):
            lo, hi = int(off[s]), int(off[s + 1])
            p_s, r_s, F_s = pos[lo:hi].contiguous(), radii[lo:hi].contiguous(), F[lo:hi].contiguous()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            Hs["g"] = ctx.collision_graph(p_s, r_s, Hs["g"])
            ij = Hs["g"].edges().to(torch.int64) + lo
            gp, gq = workloads.pair_gamma_torch(4000, ij, t, t)
            Hs["M"] = ctx.friction_assemble(Hs["g"], p_s, gp.contiguous(), gq.contiguous(), 1e-2, pr, Hs["M"])
            Hs["T"] = ctx.max_spanning_tree(Hs["M"], Hs["T"])
            Hs["Fh"] = ctx.tree_factor(Hs["M"], Hs["T"], Hs["Fh"])
            ctx.pcg_solve(Hs["M"], Hs["Fh"], F_s, tol=args.tol, precision=pr)
            b.record(stream)
            b.synchronize()
            lat.append(a.elapsed_time(b))
        return np.array(lat)

    lat = looped(sgp.PREC_F64)
    lat_m = looped(prec) if prec != sgp.PREC_F64 else lat
    line = {
        "metric": METRIC, "value": round(len(cells) / step_s, 3), "unit": "instance solves/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_s * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec == sgp.PREC_MIXED else "f64", "data": "synthetic",
        "config": {"workload": "%d independent spheroids, N log-uniform in [1e3, 1e5] (total %d cells), "
                               "cube-workload density and law, gamma0=1e-2, tol %g" % (len(cells), n, args.tol),
                   "form": "batched, %s precision, tree preconditioner" % args.precision,
                   "step": "batched graph + friction blocks + spanning forest + tree factor + batched PCG"},
        "iterations": {"p50": float(np.percentile(its, 50)), "max": int(its.max())},
        "true_rel_residual_max": float(res.max()),
        "latency_ms": {"batched_p50": round(step_s * 1e3, 3), "batched_p99": round(step_s * 1e3, 3),
                       "looped_plain_fp64_p50": round(float(np.percentile(lat, 50)), 3),
                       "looped_plain_fp64_p99": round(float(np.percentile(lat, 99)), 3)},
        "looped_plain_fp64": {"value": round(len(cells) / (lat.sum() / 1e3), 3), "unit": "instance solves/s"},
        "looped_mixed": {"value": round(len(cells) / (lat_m.sum() / 1e3), 3), "unit": "instance solves/s",
                         "p50_ms": round(float(np.percentile(lat_m, 50)), 3),
                         "p99_ms": round(float(np.percentile(lat_m, 99)), 3),
                         "note": "the same precision as the batch, one instance per solve: the batching gain "
                                 "is value / this"},
        "gpu_launches": int(launches), "tuning": tuning, "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_augmented(args):
    """The augmented spanning-forest preconditioner (Section 3.1) with the
    nested flexible CG of Section 5 against the plain spanning-forest PCG on
    the 1e6-cell spheroid, FP64 both (the nested solve is FP64): setup of
    graph, blocks, forest and factor once, then per step the augmentation
    (partition + added edges + P') and one flexible solve, and separately
    one plain solve; iteration counts and solves/s of each.  Also one solve
    each of two other settings (1000 pieces; inner tolerance 1e-3) and the
    plain PCG stopped on the Gauss-Radau error bound (Sections 4-5) next to
    residual stopping at this tolerance and at the paper's 1e-5."""
    import torch

    import paper_2410_04512_gb300 as sgp

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = sgp.Context(0, stream)
    c = WORKLOADS["ball1m"]["make"](replica_seed(0))
    n = c.n
    pos = torch.from_numpy(c.pos).to(dev)
    radii = torch.from_numpy(c.radii).to(dev)
    tp, tq = (torch.from_numpy(t).to(dev) for t in c.tables())
    F = torch.from_numpy(c.forces()).to(dev)
    g = ctx.collision_graph(pos, radii)
    ij = g.edges()
    gp, gq = workloads.pair_gamma_torch(c.seed, ij, tp, tq)
    M = ctx.friction_assemble(g, pos, gp.contiguous(), gq.contiguous(), c.gamma0, sgp.PREC_F64)
    T = ctx.max_spanning_tree(M)
    Fh = ctx.tree_factor(M, T)
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(fn):
        a, b = ev(), ev()
        a.record(stream)
        out = fn()
        b.record(stream)
        b.synchronize()
        return out, a.elapsed_time(b)

    A = None
    plain, aug = [], []
    for step in range(args.warmup + args.steps):
        (_, ip), pms = timed(lambda: ctx.pcg_solve(M, Fh, F, tol=args.tol))
        A, ams = timed(lambda: ctx.augment_tree(M, T, args.aug_t, A))
        (_, ia), fms = timed(lambda: ctx.fcg_solve(M, A, Fh, F, tol=args.tol, inner_tol=args.aug_delta))
        if step >= args.warmup:
            plain.append((pms, ip))
            aug.append((ams, fms, ia))
    info = A.info()
    p_ms = float(np.median([x[0] for x in plain]))
    a_ms = float(np.median([x[0] + x[1] for x in aug]))
    ia = aug[-1][2]
    ip = plain[-1][1]
    # one solve each of other piece counts and inner tolerances
    sweep = []
    for t, delta in ((1000, args.aug_delta), (0, 1e-3)):
        At, ams2 = timed(lambda: ctx.augment_tree(M, T, t))
        (_, it2), fms2 = timed(lambda: ctx.fcg_solve(M, At, Fh, F, tol=args.tol, inner_tol=delta))
        i2 = At.info()
        sweep.append({"t": i2["t"], "pieces": i2["pieces"], "added_edges": i2["added"], "inner_tol": delta,
                      "outer_iterations": it2.outer_iterations, "inner_iterations": it2.iterations,
                      "solve_ms": round(fms2, 3), "true_rel_residual": it2.true_rel_residual})
    # Gauss-Radau error-bound stopping (mu = 1) against residual stopping,
    # plain forest PCG, at this tolerance and at the paper's 1e-5
    estop = []
    for tol in (args.tol, 1e-5):
        (_, ir), rms = timed(lambda: ctx.pcg_solve(M, Fh, F, tol=tol))
        (_, ie), ems = timed(lambda: ctx.pcg_solve(M, Fh, F, tol=tol, stop=sgp.STOP_ERROR))
        estop.append({"tol": tol, "residual_stop": {"iterations": ir.iterations, "solve_ms": round(rms, 3),
                                                     "err_bound": ir.err_bound,
                                                     "true_rel_residual": ir.true_rel_residual},
                      "error_stop": {"iterations": ie.iterations, "solve_ms": round(ems, 3),
                                     "err_bound": ie.err_bound, "true_rel_residual": ie.true_rel_residual}})
    line = {
        "metric": METRIC, "value": round(1e3 / a_ms, 4), "unit": "solves/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(a_ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS["ball1m"]["desc"] + "; augmented spanning forest (t=%d pieces of at "
                               "most %d cells, %d edges added) + flexible CG, inner PCG to delta=%g"
                               % (info["t"], info["piece_cap"], info["added"], args.aug_delta),
                   "n_cells": n, "tol": args.tol,
                   "step": "augmentation (partition, added edges, P') + flexible CG solve; graph, blocks, "
                           "forest and factor built once"},
        "augmented": {"t": info["t"], "pieces": info["pieces"], "added_edges": info["added"],
                      "outer_iterations": ia.outer_iterations, "inner_iterations": ia.iterations,
                      "true_rel_residual": ia.true_rel_residual,
                      "augment_ms": round(float(np.median([x[0] for x in aug])), 3),
                      "solve_ms": round(float(np.median([x[1] for x in aug])), 3),
                      "solves_per_s": round(1e3 / a_ms, 4)},
        "plain_fp64": {"iterations": ip.iterations, "true_rel_residual": ip.true_rel_residual,
                       "solve_ms": round(p_ms, 3), "solves_per_s": round(1e3 / p_ms, 4)},
        "outer_vs_plain_iterations": round(ia.outer_iterations / max(ip.iterations, 1), 3),
        "augmented_sweep": sweep,
        "error_bound_stopping": estop,
    }
    print(json.dumps(line), flush=True)


def run_local(args):
    """The partitioned spanning-forest preconditioner (Section 6) on the
    1e6-cell spheroid, mixed precision (the chosen form): per step the
    leaves of a uniform grid, the union of the leaves' forests, its factor
    and one solve, against the same step with the global forest, for leaf
    sides giving about 190, 510 and 1000 cells per leaf (grid, blocks and
    the contact graph built once)."""
    import torch

    import paper_2410_04512_gb300 as sgp

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = sgp.Context(0, stream)
    c = WORKLOADS["ball1m"]["make"](replica_seed(0))
    n = c.n
    pos = torch.from_numpy(c.pos).to(dev)
    radii = torch.from_numpy(c.radii).to(dev)
    tp, tq = (torch.from_numpy(t).to(dev) for t in c.tables())
    F = torch.from_numpy(c.forces()).to(dev)
    g = ctx.collision_graph(pos, radii)
    ij = g.edges()
    gp, gq = workloads.pair_gamma_torch(c.seed, ij, tp, tq)
    prec = sgp.PREC_MIXED
    M = ctx.friction_assemble(g, pos, gp.contiguous(), gq.contiguous(), c.gamma0, prec)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    density = n / (4.0 / 3.0 * np.pi * c.meta["radius"] ** 3) if "radius" in c.meta else None

    def run(h):
        H = {"leaf": None, "T": None, "Fh": None}
        rows = []
        for step in range(args.warmup + args.steps):
            a, b, m = ev(), ev(), ev()
            a.record(stream)
            if h is None:
                H["T"] = ctx.max_spanning_tree(M, H["T"])
            else:
                H["leaf"] = ctx.grid_leaves(pos, h, H["leaf"])
                H["T"] = ctx.local_spanning_forest(M, H["leaf"], H["T"])
            H["Fh"] = ctx.tree_factor(M, H["T"], H["Fh"])
            m.record(stream)
            _, info = ctx.pcg_solve(M, H["Fh"], F, tol=args.tol, precision=prec)
            b.record(stream)
            b.synchronize()
            if step >= args.warmup:
                rows.append((a.elapsed_time(b), m.elapsed_time(b), info))
        info = rows[-1][2]
        step_ms = float(np.median([r[0] for r in rows]))
        lay = H["Fh"].layout()
        out = {"step_ms": round(step_ms, 3), "solve_ms": round(float(np.median([r[1] for r in rows])), 3),
               "solves_per_s": round(1e3 / step_ms, 4), "inner_iterations": info.iterations,
               "outer_iterations": info.outer_iterations, "true_rel_residual": info.true_rel_residual,
               "forest_edges": H["T"].info()[0], "components": H["T"].info()[1],
               "bins": lay["bins"], "top": lay["top"]}
        if h is not None:
            out["leaf_side"] = h
            out["leaves"] = int(torch.unique(H["leaf"]).numel())
            out["cells_per_leaf_mean"] = round(n / out["leaves"], 1)
        return out

    glob = run(None)
    # sides for about 190, 510 and 1000 cells per leaf at the spheroid's density
    rho = density if density else n / (8.0 * float(pos.abs().max()) ** 3)
    sides = [round((k / rho) ** (1.0 / 3.0), 3) for k in (190, 510, 1000)]
    local = [run(h) for h in sides]
    best = max(local, key=lambda r: r["solves_per_s"])
    # the paper's noisy hexagonal packing (1e5 cells, gamma_med 3e4, Hertz
    # areas, tol 1e-5 as in its Section 5), global against local forests
    hx = workloads.paper_hex(n=100_000, seed=6400)
    pos, radii = torch.from_numpy(hx.pos).to(dev), torch.from_numpy(hx.radii).to(dev)
    g = ctx.collision_graph(pos, radii)
    gp, gq = hx.gammas_torch(g.edges(), pos, radii)
    M = ctx.friction_assemble(g, pos, gp.contiguous(), gq.contiguous(), hx.gamma0, prec)
    F = torch.from_numpy(np.random.Generator(np.random.PCG64([6400, 1])).standard_normal((hx.n, 3))).to(dev)
    n = hx.n
    tol_saved, args.tol = args.tol, 1e-5
    hex_rows = {"global": run(None)}
    for k in (190, 510, 1000):
        hex_rows["cells_%d" % k] = run(round((k / 1.4142) ** (1.0 / 3.0), 3))   # 1.414 cells per unit volume
    args.tol = tol_saved
    line = {
        "metric": METRIC, "value": best["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": best["step_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "mixed f32/f64", "data": "synthetic",
        "config": {"workload": WORKLOADS["ball1m"]["desc"] + "; partitioned spanning forest: uniform-grid "
                               "leaves, each leaf's own maximum spanning forest, contacts between leaves dropped",
                   "n_cells": n, "tol": args.tol,
                   "step": "leaves + local forest + factor + mixed solve (graph and blocks built once)"},
        "global_forest": glob, "local_forests": local,
        "best_local_vs_global_step": round(glob["step_ms"] / best["step_ms"], 3),
        "paper_hex_1e5_tol_1e-5": hex_rows,
    }
    print(json.dumps(line), flush=True)


def run_paper(args):
    """The paper's own experiments re-created (Section 5): noisy hexagonal
    close packing at gamma_med 3e4 and 3e3, a rejection-sampled spheroid and
    a dumbbell, n = 50,000 equal cells with Hertz contact areas, a known
    solution x* (F = Gamma x*), tolerance 1e-5; iterations of no
    preconditioner, block Jacobi, the spanning forest and the augmented
    forest (flexible CG), averaged over independent realizations, and their
    ratios next to the ones the paper prints.  Three stopping readings:
    the true relative error |x_k - x*| <= 1e-5 |x*| (the count found by runs
    of fixed length), the Gauss-Radau bound of the Gamma-norm error, and the
    relative residual.  Also the hexagonal lattice from 1e2 to 1e5 cells:
    wall clock of assembly, preconditioner construction and factorization
    and CG, the forest against no preconditioner.  FP64."""
    import torch

    import paper_2410_04512_gb300 as sgp

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = sgp.Context(0, stream)
    reps = args.paper_reps
    n = args.paper_n
    tol = 1e-5
    paper_ratio = {"hex": {"none_over_tree": 4.9, "none_over_jacobi": 1.2},
                   "hex_high_kappa": {"none_over_tree": 9.2},
                   "random": {"none_over_tree": 3.8}, "dumbbell": {"none_over_tree": 8.5}}
    makers = {"hex": lambda s: workloads.paper_hex(n=n, seed=6000 + s),
              "hex_high_kappa": lambda s: workloads.paper_hex(n=n, seed=6100 + s, gamma_med=3.0e3),
              "random": lambda s: workloads.paper_random(n=n, seed=7000 + s),
              "dumbbell": lambda s: workloads.paper_dumbbell(n=n, seed=8000 + s)}
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def system(c):
        pos = torch.from_numpy(c.pos).to(dev)
        radii = torch.from_numpy(c.radii).to(dev)
        g = ctx.collision_graph(pos, radii)
        ij = g.edges()
        gp, gq = c.gammas_torch(ij, pos, radii)
        M = ctx.friction_assemble(g, pos, gp.contiguous(), gq.contiguous(), c.gamma0, sgp.PREC_F64)
        T = ctx.max_spanning_tree(M)
        Fh = ctx.tree_factor(M, T)
        return pos, radii, g, M, T, Fh

    def rel(v, xs):
        return float(torch.linalg.norm(v - xs) / torch.linalg.norm(xs))

    def to_true_error(M, Fh, F, xs, pc, start):
        """Fewest iterations whose iterate has |x_k - x*| <= tol |x*|: runs of
        a fixed count (maxit, no other stop) doubled, then bisected."""
        def err(k):
            v, _ = ctx.pcg_solve(M, Fh, F, tol=1e-300, maxit=k, precond=pc, raise_on_error=False)
            return rel(v, xs)
        lo, hi = 0, max(1, start)
        while err(hi) > tol:
            lo, hi = hi, 2 * hi
            if hi > 200_000:
                return -1
        while hi - lo > 1:
            mid = (lo + hi) // 2
            lo, hi = (lo, mid) if err(mid) <= tol else (mid, hi)
        return hi

    out = {}
    for name, make in makers.items():
        rows = []
        for rep in range(reps):
            c = make(rep)
            pos, radii, g, M, T, Fh = system(c)
            xs = torch.from_numpy(np.random.Generator(np.random.PCG64([9100, rep])).standard_normal((c.n, 3))).to(dev)
            F = ctx.spmv(M, xs)
            row = {}
            for label, kw in (("none", dict(precond=sgp.PRECOND_NONE)),
                              ("jacobi", dict(precond=sgp.PRECOND_BLOCK_JACOBI)),
                              ("tree", dict(precond=sgp.PRECOND_TREE)),
                              ("tree_error_bound", dict(precond=sgp.PRECOND_TREE, stop=sgp.STOP_ERROR)),
                              ("none_error_bound", dict(precond=sgp.PRECOND_NONE, stop=sgp.STOP_ERROR))):
                a, b = ev(), ev()
                a.record(stream)
                v, info = ctx.pcg_solve(M, Fh, F, tol=tol, **kw)
                b.record(stream)
                b.synchronize()
                row[label] = (info.iterations, a.elapsed_time(b), rel(v, xs))
            for label, pc in (("none", sgp.PRECOND_NONE), ("jacobi", sgp.PRECOND_BLOCK_JACOBI),
                              ("tree", sgp.PRECOND_TREE)):
                row[label + "_to_true_error"] = (to_true_error(M, Fh, F, xs, pc, row[label][0]), 0.0, tol)
            A = ctx.augment_tree(M, T, 0)
            a, b = ev(), ev()
            a.record(stream)
            v, info = ctx.fcg_solve(M, A, Fh, F, tol=tol, inner_tol=0.1)
            b.record(stream)
            b.synchronize()
            row["augmented"] = (info.outer_iterations, a.elapsed_time(b), rel(v, xs))
            rows.append(row)
        mean = {k: float(np.mean([r[k][0] for r in rows])) for k in rows[0]}
        out[name] = {"iterations_mean": {k: round(v, 1) for k, v in mean.items()},
                     "solve_ms_mean": {k: round(float(np.mean([r[k][1] for r in rows])), 3) for k in rows[0]
                                       if not k.endswith("_to_true_error")},
                     "true_rel_error_max": {k: float(np.max([r[k][2] for r in rows])) for k in rows[0]
                                            if not k.endswith("_to_true_error")},
                     "none_over_tree_true_error": round(mean["none_to_true_error"] / mean["tree_to_true_error"], 2),
                     "none_over_jacobi_true_error": round(mean["none_to_true_error"] /
                                                          mean["jacobi_to_true_error"], 2),
                     "none_over_tree_residual": round(mean["none"] / mean["tree"], 2),
                     "none_over_tree_error_bound": round(mean["none_error_bound"] / mean["tree_error_bound"], 2),
                     "tree_over_augmented": round(mean["tree"] / mean["augmented"], 3),
                     "paper": paper_ratio[name], "cells": n, "realizations": reps}
    # wall-clock scaling on the hexagonal lattice: what the paper's scaling
    # figure times (assembly, preconditioner construction and factorization,
    # CG), with the contact graph and the Hertz coefficients given
    scaling = []
    for ns in (100, 1000, 10_000, 100_000):
        c = workloads.paper_hex(n=ns, seed=6200)
        pos = torch.from_numpy(c.pos).to(dev)
        radii = torch.from_numpy(c.radii).to(dev)
        g = ctx.collision_graph(pos, radii)
        gp, gq = (t.contiguous() for t in c.gammas_torch(g.edges(), pos, radii))
        xs = torch.from_numpy(np.random.Generator(np.random.PCG64([9200, ns])).standard_normal((ns, 3))).to(dev)
        F = ctx.spmv(ctx.friction_assemble(g, pos, gp, gq, c.gamma0, sgp.PREC_F64), xs)
        entry = {"cells": ns}
        for pname, prec in (("f64", sgp.PREC_F64), ("mixed", sgp.PREC_MIXED)):
            res = {}
            for label, pc in (("tree", sgp.PRECOND_TREE), ("none", sgp.PRECOND_NONE),
                              ("jacobi", sgp.PRECOND_BLOCK_JACOBI)):
                times = []
                for rep in range(4):
                    a, b = ev(), ev()
                    a.record(stream)
                    M = ctx.friction_assemble(g, pos, gp, gq, c.gamma0, prec)
                    Fh = ctx.tree_factor(M, ctx.max_spanning_tree(M)) if pc == sgp.PRECOND_TREE else None
                    v, info = ctx.pcg_solve(M, Fh, F, tol=tol, precond=pc, precision=prec)
                    b.record(stream)
                    b.synchronize()
                    times.append(a.elapsed_time(b))
                res[label] = {"step_ms": round(float(np.median(times[1:])), 3), "iterations": info.iterations,
                              "true_rel_error": float(torch.linalg.norm(v - xs) / torch.linalg.norm(xs))}
            res["none_over_tree_time"] = round(res["none"]["step_ms"] / res["tree"]["step_ms"], 2)
            entry[pname] = res
        scaling.append(entry)
    line = {
        "metric": METRIC, "value": None, "unit": "iterations", "n_gpus": 1, "steps": reps, "warmup": 0,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "the paper's Section 5 geometries re-created: noisy hexagonal close packing "
                               "(spacing 2r, noise N(0,(0.3 r)^2)), rejection-sampled spheroid and dumbbell "
                               "(minimum distance 0.7, density 1.6), r = 0.5, Hertz contact areas, gamma_par 2e6, "
                               "gamma_perp 8e7, gamma_med 3e4 (3e3 for high kappa), known solution, tol 1e-5",
                   "cells": n},
        "paper_workloads": out, "hex_scaling": scaling,
    }
    print(json.dumps(line), flush=True)


def run_warm(args):
    """The learned-warm-start workload: a 200,000-cell spheroid advanced by
    x <- x + v dt (dt = 0.01) for ``--warm-steps`` steps under overlap springs
    (k = 1) plus fresh active noise N(0, 0.1^2); graph, friction blocks,
    spanning forest and factor are rebuilt every step.  The network is
    trained (energy-norm loss, Adam) on the solver's solutions of the first
    ``--warm-train`` steps and predicts v0 afterwards; each predicted step is
    solved to the same tolerance from the learned v0, from zero and from the
    previous step's v."""
    import torch

    import paper_2410_04512_gb300 as sgp

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    ctx = sgp.Context(0, stream)
    peaks, peaks_src = load_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]))
    c = workloads.spheroid_200k()
    n = c.n
    pos = torch.from_numpy(c.pos).to(dev)
    radii = torch.from_numpy(c.radii).to(dev)
    tp, tq = (torch.from_numpy(t).to(dev) for t in c.tables())
    prec = sgp.PREC_MIXED if args.precision == "mixed" else sgp.PREC_F64
    net = ctx.mpnn_create(workloads.mpnn_init(5000))
    H = {"g": None, "M": None, "T": None, "Fh": None}
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def build(step):
        H["g"] = ctx.collision_graph(pos, radii, H["g"])
        ij = H["g"].edges()
        gp, gq = workloads.pair_gamma_torch(c.seed, ij, tp, tq)
        H["M"] = ctx.friction_assemble(H["g"], pos, gp.contiguous(), gq.contiguous(), c.gamma0, prec, H["M"])
        H["T"] = ctx.max_spanning_tree(H["M"], H["T"])
        H["Fh"] = ctx.tree_factor(H["M"], H["T"], H["Fh"])
        noise = torch.from_numpy(workloads.active_noise(c.seed, step, n)).to(dev)
        return (workloads.spring_forces_torch(pos, radii, ij) + noise).contiguous()

    def timed(fn):
        a, b = ev(), ev()
        a.record(stream)
        out = fn()
        b.record(stream)
        b.synchronize()
        return out, a.elapsed_time(b)

    def solve(F, x0):
        v = torch.zeros_like(F) if x0 is None else x0.clone()
        _, inf = ctx.pcg_solve(H["M"], H["Fh"], F, v, tol=args.tol, precision=prec, x0_given=x0 is not None)
        return v, inf

    vprev = None
    train_ms, rows = [], []
    ctx.launch_count(reset=True)
    with ClockSampler(0) as clk:
        for step in range(1, args.warm_steps + 1):
            F, build_ms = timed(lambda: build(step))
            (vstar, inf0), zero_ms = timed(lambda: solve(F, None))
            if step <= args.warm_train:
                def train():
                    L = 0.0
                    for _ in range(args.warm_epochs):
                        ctx.mpnn_forward(net, H["M"], H["Fh"], F, vprev)
                        L = ctx.mpnn_backward(net, vstar, sgp.MPNN_LOSS_ENERGY)
                        ctx.mpnn_step(net, args.warm_lr)
                    return L
                L, ms = timed(train)
                train_ms.append(ms)
                v_next = vstar
            else:
                (v0, used), inf_ms = timed(lambda: ctx.warm_start(net, H["M"], H["Fh"], F, vprev, mr_scale=True))
                (vw, infw), warm_ms = timed(lambda: solve(F, v0))
                (vp, infp), prev_ms = timed(lambda: solve(F, vprev))
                e = (v0 - vstar).contiguous()
                E = float(torch.sum(e * ctx.spmv(H["M"], e)) / torch.sum(vstar * F))
                rows.append(dict(build=build_ms, zero=zero_ms, infer=inf_ms, warm=warm_ms, prev=prev_ms,
                                 it0=inf0.iterations, itw=infw.iterations, itp=infp.iterations, used=used, E=E,
                                 res=max(inf0.true_rel_residual, infw.true_rel_residual)))
                v_next = vw
            vprev = v_next
            pos = (pos + 0.01 * v_next).contiguous()
    launches = ctx.launch_count()
    # inference broken into its stages (per-stage CUDA events, repeated on
    # the last step's system after the timed sequence)
    KW = (sgp.KT_WARM_BASIS, sgp.KT_WARM_LAYERS, sgp.KT_WARM_CHECK)
    ctx.set_kernel_timing(True)
    for k in KW:
        ctx.kernel_time(k, reset=True)
    reps = 10
    for _ in range(reps):
        ctx.warm_start(net, H["M"], H["Fh"], F, vprev, mr_scale=True)
    torch.cuda.synchronize()
    stage = {name: round(ctx.kernel_time(k)[0] / reps, 4)
             for name, k in zip(("basis_and_features", "layers_and_output", "scaling_and_check"), KW)}
    ctx.set_kernel_timing(False)
    R = {k: np.array([r[k] for r in rows], dtype=np.float64) for k in rows[0]}
    # what the guess's error should save: CG shrinks the Gamma-norm error by
    # about rho = tol^(1 / iterations) per iteration (from the zero-guess
    # solves); a start with relative Gamma-norm error sqrt(E) (E is the
    # squared ratio) is ln sqrt(E) / ln rho iterations ahead
    rho_it = args.tol ** (1.0 / float(R["it0"].mean()))
    expect = float(np.log(np.sqrt(np.median(R["E"]))) / np.log(rho_it))
    per_learned = R["build"] + R["infer"] + R["warm"]
    per_zero = R["build"] + R["zero"]
    per_prev = R["build"] + R["prev"]
    value = len(rows) / (per_learned.sum() / 1e3)
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "solves/s", "n_gpus": 1,
        "steps": len(rows), "warmup": args.warm_train, "ms_per_step": round(float(per_learned.mean()), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec == sgp.PREC_MIXED else "f64", "data": "synthetic",
        "config": {"workload": "learned warm start: %d-cell spheroid (ball at packing 0.6), %d time steps "
                               "x <- x + v dt, dt 0.01, overlap springs k=1 + active noise N(0,0.1^2), gamma "
                               "log-uniform [0.1,10], gamma0 1e-3; trained on steps 1-%d (%d Adam steps per "
                               "step, lr %g, energy-norm loss), predicting steps %d-%d"
                               % (n, args.warm_steps, args.warm_train, args.warm_epochs, args.warm_lr,
                                  args.warm_train + 1, args.warm_steps),
                   "form": "%s precision, tree preconditioner, v0 from the network (minimal-residual "
                           "scaled, residual-checked)" % args.precision,
                   "tol": args.tol,
                   "step": "collision graph + friction blocks + spanning forest + tree factor + network "
                           "inference + PCG from v0"},
        "learned": {"solves_per_s": round(value, 4), "iterations_mean": float(R["itw"].mean()),
                    "inference_ms_mean": round(float(R["infer"].mean()), 3),
                    "inference_stages_ms": stage,
                    "iterations_saved_mean": round(float((R["it0"] - R["itw"]).mean()), 2),
                    "iterations_saved_expected_from_error": round(expect, 2),
                    "break_even_inference_ms": round(float((R["it0"] - R["itw"]).mean()
                                                           * (R["zero"] / R["it0"]).mean()), 3),
                    "accepted": int(R["used"].sum()), "energy_error_median": float(np.median(R["E"]))},
        "zero_guess": {"solves_per_s": round(len(rows) / (per_zero.sum() / 1e3), 4),
                       "iterations_mean": float(R["it0"].mean())},
        "previous_v": {"solves_per_s": round(len(rows) / (per_prev.sum() / 1e3), 4),
                       "iterations_mean": float(R["itp"].mean())},
        "solve_only_ms_mean": {"learned": round(float((R["infer"] + R["warm"]).mean()), 3),
                               "zero": round(float(R["zero"].mean()), 3), "prev": round(float(R["prev"].mean()), 3)},
        "build_ms_mean": round(float(R["build"].mean()), 3),
        "training": {"steps": args.warm_train, "ms_per_step_mean": round(float(np.mean(train_ms)), 3)},
        "true_rel_residual_max": float(R["res"].max()),
        "gpu_launches": int(launches), "clocks": clk.summary(),
        "peak_hbm_gbs": hbm_peak, "peak_source": peaks_src,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the CPU oracle: cpu_baseline leg and the reference arm
# ---------------------------------------------------------------------------
def oracle_iterations(workload: str, fallback=None):
    """The oracle's own PCG iteration count to the tolerance on a benchmark
    workload (oracle/calibration.json, written by ``python -m
    oracle.calibrate``), else `fallback` (the FP64 GPU solve's count of the
    same system, which the parity tests keep within 2 of the oracle's)."""
    p = os.path.join(ROOT, "oracle", "calibration.json")
    if os.path.exists(p):
        with open(p) as f:
            cal = json.load(f)
        if workload in cal:
            return int(cal[workload]["iterations"]), "the oracle's own count, oracle/calibration.json"
    if fallback is not None:
        return int(fallback), "FP64 GPU solve of the same system"
    return None, None


class OracleSystem:
    """The full workload of rank 0's replica on the CPU: k-d tree contact
    search (the oracle's contact rule), eq. (1) blocks; then the solve
    phase the paper times (Section 5): Prim, TreeLDLT, PCG."""

    def __init__(self, workload: str):
        import oracle
        self.oracle = oracle
        self.cells = WORKLOADS[workload]["make"](replica_seed(0))
        c = self.cells
        self.F = c.forces()
        t = time.perf_counter()
        ij = oracle.contacts_kdtree(c.pos, c.radii)
        self.contacts_s = time.perf_counter() - t
        t = time.perf_counter()
        self.sys = oracle.build_system(c.pos, c.radii, c.gammas_np, c.gamma0, ij=ij)
        self.blocks_s = time.perf_counter() - t

    def factor(self):
        o, s = self.oracle, self.sys
        t = time.perf_counter()
        forest = o.prim_msf(s.n, s.ij, s.w)
        t1 = time.perf_counter()
        fac = o.tree_ldlt(forest, s.blocks, s.gamma0)
        t2 = time.perf_counter()
        return fac, t1 - t, t2 - t1

    def pcg_iter_s(self, fac, k: int, parallel: bool) -> float:
        """Seconds per PCG iteration at full size, from k timed iterations."""
        o, s = self.oracle, self.sys
        t = time.perf_counter()
        if parallel:
            o.pcg_parallel(s.n, s.ij, s.blocks, s.gamma0, self.F, fac, tol=1e-300, maxit=k)
        else:
            o.pcg(s.n, s.ij, s.blocks, s.gamma0, self.F, o.PRECOND_TREE, fac, fixed_iters=k)
        return (time.perf_counter() - t) / k

    def contact_scan(self, n_sample: int = 20000):
        """The oracle's brute-force contact test over all pairs of a sample
        of cells: pair tests per second, and the full scan's time at that
        rate (extrapolated)."""
        c = self.cells
        ns = min(n_sample, c.n)
        t = time.perf_counter()
        self.oracle.contacts(c.pos[:ns], c.radii[:ns])
        dt = time.perf_counter() - t
        rate = ns * (ns - 1) / 2 / dt
        return {"sample_cells": ns, "pair_tests_per_s": round(rate, 1),
                "full_scan_s": round(c.n * (c.n - 1) / 2 / rate, 1), "extrapolated": True}


def cpu_baseline(args, gpu_fp64_iters=None, k_iters: int = 20):
    """The oracle on the host cores, on the full workload: Prim and TreeLDLT
    timed in full, PCG timed for k_iters iterations at full size (one core,
    as the oracle stands; and all cores: the same PCG with the product and
    the vector operations over OpenMP threads, the tree solve sequential),
    each scaled to the oracle's own iteration count to the tolerance."""
    osys = OracleSystem(args.workload)
    iters, src = oracle_iterations(args.workload, gpu_fp64_iters)
    if iters is None:
        return {"unavailable": "no oracle iteration count for this workload (python -m oracle.calibrate)"}
    fac, prim_s, ldlt_s = osys.factor()
    it1 = osys.pcg_iter_s(fac, k_iters, parallel=False)
    itn = osys.pcg_iter_s(fac, k_iters, parallel=True)
    threads = osys.oracle.parallel_threads()
    one = prim_s + ldlt_s + it1 * iters
    alln = prim_s + ldlt_s + itn * iters
    n = osys.cells.n
    return {"value": round(1.0 / one, 6), "unit": "solves/s", "cores": 1, "kind": "oracle", "extrapolated": True,
            "sample": f"full {n}-cell workload: Prim {prim_s:.2f} s and TreeLDLT {ldlt_s:.2f} s timed in full, "
                      f"PCG timed for {k_iters} iterations at full size ({it1 * 1e3:.1f} ms each) and scaled "
                      f"to {iters} iterations to {args.tol:g} ({src})",
            "solve_s": round(one, 3),
            "all_cores": {"value": round(1.0 / alln, 6), "unit": "solves/s", "cores": threads,
                          "nproc": os.cpu_count(), "solve_s": round(alln, 3),
                          "pcg_iteration_ms": round(itn * 1e3, 2),
                          "note": "product and vector operations over OpenMP threads, tree solve sequential"},
            "setup_not_in_value": {"contacts_kdtree_s": round(osys.contacts_s, 3),
                                   "friction_blocks_s": round(osys.blocks_s, 3)},
            "contact_scan_bruteforce": osys.contact_scan()}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload not in WORKLOADS:
        print(json.dumps({"impl": "reference", "unavailable": f"no CPU reference for workload {args.workload}"}))
        return
    iters, src = oracle_iterations(args.workload)
    if iters is None:
        print(json.dumps({"impl": "reference",
                          "unavailable": "no oracle iteration count for this workload (python -m oracle.calibrate)"}))
        return
    osys = OracleSystem(args.workload)
    k_iters = 10

    def step():
        fac, prim_s, ldlt_s = osys.factor()
        return prim_s + ldlt_s + osys.pcg_iter_s(fac, k_iters, parallel=False) * iters

    for _ in range(args.warmup):
        step()
    times = [step() for _ in range(args.steps)]
    total = float(np.sum(times))
    value = args.steps / total
    n = osys.cells.n
    sample = (f"each step: Prim and TreeLDLT on the full {n}-cell workload timed in full, PCG timed for "
              f"{k_iters} iterations at full size and scaled to {iters} iterations to {args.tol:g} ({src})")
    line = {"metric": METRIC, "value": round(value, 6), "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total / args.steps * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOADS[args.workload]["desc"], "n_cells": n, "tol": args.tol,
                       "precond": "tree", "precision": "fp64"},
            "cpu_baseline": {"value": round(value, 6), "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "extrapolated": True, "sample": sample},
            "e2e": {"value": round(value, 6), "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="sgp", choices=["sgp", "reference"])
    ap.add_argument("--workload", default="ball1m",
                    choices=sorted(WORKLOADS) + ["batch512", "warm200k", "aug1m", "paper", "local1m"])
    ap.add_argument("--paper-reps", dest="paper_reps", type=int, default=5,
                    help="paper: independent realizations per geometry")
    ap.add_argument("--paper-n", dest="paper_n", type=int, default=50_000, help="paper: cells per geometry")
    ap.add_argument("--aug-t", dest="aug_t", type=int, default=0,
                    help="aug1m: pieces of the augmented forest (0: round(n^(1/4)))")
    ap.add_argument("--aug-delta", dest="aug_delta", type=float, default=0.1,
                    help="aug1m: relative tolerance of the inner PCG")
    ap.add_argument("--batch", type=int, default=512, help="instances of the batch512 workload")
    ap.add_argument("--precision", default="mixed", choices=["f64", "mixed"])
    ap.add_argument("--precond", default="tree", choices=["tree", "jacobi", "none"])
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--cpu-baseline", dest="cpu_baseline", type=int, default=1)
    ap.add_argument("--compare", type=int, default=1, help="also time plain FP64 and block-Jacobi")
    ap.add_argument("--configs", type=int, default=1,
                    help="1: also run the other configurations (cube, sheet, batch, warm start) and record them")
    ap.add_argument("--autotune", type=int, default=1,
                    help="1: pick the launch shapes with the library's autotuner before timing "
                         "(whole solves plus factor builds per candidate); 0: built-in defaults")
    ap.add_argument("--warm-steps", dest="warm_steps", type=int, default=200)
    ap.add_argument("--warm-train", dest="warm_train", type=int, default=50)
    ap.add_argument("--warm-epochs", dest="warm_epochs", type=int, default=8)
    ap.add_argument("--warm-lr", dest="warm_lr", type=float, default=2e-3)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "sgp":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch512":
        run_batch(args)
    elif args.workload == "warm200k":
        run_warm(args)
    elif args.workload == "aug1m":
        run_augmented(args)
    elif args.workload == "paper":
        run_paper(args)
    elif args.workload == "local1m":
        run_local(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
