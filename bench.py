"""Benchmark: cell integration + global CSR assembly on one GB300 (per rank).

One step = one fe_assemble call (geometry, gradients, cell-matrix contraction,
cell vectors, deterministic scatter into CSR + RHS). The default workload is the
largest single-GPU configuration, Q1 linear elasticity on 128^3 cells of the
unit cube (2,097,152 cells, 6,440,067 DOFs, 513,599,625 nonzeros), mixed FP32
contraction with FP64 geometry and FP64 CSR accumulation;
``--workload elasticity_q2_beam`` times the 32x32x32 Q2 beam (32,768 cells,
152,771,337 nonzeros) instead. Inputs are seeded synthetic meshes; the working
set (cell matrices and CSR values, gigabytes) is far larger than L2, so no
flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp32|bf16|fp64] [--workload NAME]
  python bench.py --impl reference     # the FP64 CPU oracle on the host cores

Prints one JSON line (rank 0). Under torchrun every rank assembles its own
replica (weak scaling, no collective on the data path); the barrier and the
max over ranks are for timing only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRICS = {
    "elasticity_q1_128": "cells/s integrate+assemble (elasticity Q1 128^3 unit cube), mixed-prec vs FP64 at <=1e-6 "
                         "rel err",
    "elasticity_q2_beam": "cells/s integrate+assemble (elasticity Q2 32^3 beam), mixed-prec vs FP64 at <=1e-6 rel err",
}
UNIT = "cells/s"
WORKLOAD = "elasticity_q1_128"


def metric_of(workload: str) -> str:
    return METRICS.get(workload, f"cells/s integrate+assemble ({workload}), mixed-prec vs FP64 at <=1e-6 rel err")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="fp32", choices=["fp32", "bf16", "fp64"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--kernel", default="auto", choices=["auto", "cuda_core", "tensor_core"],
                    help="cell-integration kernel selection (fe_space_set_kernel)")
    ap.add_argument("--reorder", action="store_true",
                    help="give the cells in the locality order of fe_mesh_locality_order (Morton order of "
                         "the cell centroids) before creating the space")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-comparators", action="store_true")
    ap.add_argument("--extras", action="store_true",
                    help="also time the 128^3 Q1 elasticity assembly and the 64^3 cantilever adjoint")
    ap.add_argument("--batched", action="store_true",
                    help="also time the 64-mesh batched assembly (host setup takes minutes)")
    ap.add_argument("--extra", action="append", default=None,
                    help="time only this secondary workload (repeatable): elasticity_q2_beam_clamped, "
                         "cantilever_q1_64_compliance, stokes_q2q1_32, dg_q2_32, elasticity_q1_128, "
                         "cantilever_q1_64_adjoint")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ----------------------------------------------------------------------------- helpers
def max_over_ranks(x: float, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (timing only; no data path)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t)


def whole_job_rate(units_per_rank: int, world_size: int, steps: int, ms_total: float) -> float:
    """Units per second over all ranks: every rank processes its own replica."""
    return world_size * units_per_rank * steps / (ms_total / 1e3)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("bf16_tflops", 1900.0)), "measured"
    return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.1)
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
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def source_sha(files) -> str:
    """Short hash of the kernel's source files (csrc/), to tell stale counters."""
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_1708_01773_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def kernel_traffic(workload: str, kernel: str, cells: int):
    """DRAM traffic per launch from a committed ncu summary of this workload's
    kernel, if the kernel sources are unchanged since the counters were taken
    (else None). A capture taken on a smaller mesh of the same kernels is scaled
    by the number of cells (the traffic of these kernels grows in proportion)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f).get(f"{workload}:{kernel}")
    if not d or source_sha(d["sources"]) != d["sources_sha"]:
        return None
    return int(round(d["bytes_per_launch"] * cells / d.get("cells", cells)))


def on_tensor_cores(prob, prec: str, kernel: str) -> bool:
    """Whether fe_assemble's cell integration runs on tcgen05 for this workload
    under the kernel selection `kernel` (auto, cuda_core, tensor_core)."""
    from paper_1708_01773_gb300 import inputs
    if prec == "fp64" or kernel == "cuda_core" or prob.quad_1d != prob.order + 1:
        return False
    if prob.problem == inputs.ELASTICITY and prob.order == 2:
        return True
    if prob.problem == inputs.ELASTICITY and prob.order == 3:
        return kernel == "tensor_core" or (kernel == "auto" and prec == "bf16")
    if prob.problem != inputs.POISSON or prob.order not in (2, 3):
        return False
    return kernel == "tensor_core" or (kernel == "auto" and prob.order == 3 and prec == "bf16")


def kernel_names(prob, prec: str, kernel: str = "auto"):
    """Names of the cell and scatter kernels fe_assemble launches for a workload
    under the kernel selection `kernel`."""
    from paper_1708_01773_gb300 import inputs
    el = prob.problem == inputs.ELASTICITY
    nl = prob.ncomp * (prob.order + 1) ** 3
    scat = f"k_scatter_slots<{nl},{3 if el and nl <= 32 else 1}>"
    if prec == "fp64":
        return f"k_cell<{prob.order},{3 if el else 1},0>", "k_scatter_rows<double>"
    if on_tensor_cores(prob, prec, kernel):
        if el:
            return ("tc::k_cell_tc" if prob.order == 2 else "tce::k_cell_tce"), scat
        return f"tcp::k_cell_tcp<{prob.order}>", scat
    if el and prob.order == 1 and prob.quad_1d == 2 and kernel == "auto":
        return "q1e::k_cell_q1e", scat
    return f"k_cell<{prob.order},{3 if el else 1},{1 if prec == 'fp32' else 2}>", scat


def scatter_bytes(sp, prec: str) -> int:
    """Algorithmic bytes of one scatter launch: every cell-matrix entry read once
    (FP32, or FP64 for the FP64 form), the FP64 values written, the row
    descriptors (row, slot and code pointers), cell vectors and slot lists read,
    the RHS written, and the permutation: for the FP32/BF16 forms one 16-bit
    slot-major position per contribution, shared by the three rows of a node
    where they are scattered together (3-component Q1 rows); for the FP64 form
    one 16-bit destination-sorted code per contribution plus one count byte per
    nonzero."""
    nl = sp.nl
    rows_per_item = 3 if (prec != "fp64" and sp.prob.ncomp == 3 and sp.prob.problem != 2 and nl <= 32) else 1
    common = sp.nnz * 8 + sp.n_cells * nl * 8 + (sp.n_dofs + 1) * 8 * 3 + sp.n_dofs * 8
    if prec == "fp64":
        return int(sp.n_cells * nl * nl * 8 + sp.n_contrib * 2 + sp.nnz + sp.n_cells * nl * 4 + common)
    return int(sp.n_cells * nl * nl * 4 + (sp.n_contrib * 2 + sp.n_cells * nl * 4) // rows_per_item + common)


def cell_bytes(sp, prec: str) -> int:
    """Algorithmic bytes of one cell-integration launch: vertex coordinates and the
    coefficient read, cell matrices and cell vectors written."""
    ke = 8 if prec == "fp64" else 4
    nl = sp.nl
    return int(sp.n_cells * (24 * 8 + 8) + sp.n_cells * nl * nl * ke + sp.n_cells * nl * 8)


# ----------------------------------------------------------------------------- CPU oracle
def oracle_rate(prob, target_s: float, max_cells: int | None = None):
    """Times the FP64 CPU oracle (numbering + cell loop + COO compress) on the first
    cells of the workload, sized to take about target_s seconds. Returns
    (cells/s, cells in the sample, seconds)."""
    import oracle
    from paper_1708_01773_gb300 import inputs

    def sample(n):
        cv = prob.mesh.cell_vertices[:n]
        sub = inputs.Problem(prob.name, inputs.Mesh(prob.mesh.coords, cv), prob.order, prob.quad_1d,
                             prob.problem, prob.coef[:n], prob.force, prob.nu)
        t = time.perf_counter()
        oracle.assemble_csr(sub)
        return time.perf_counter() - t

    n = 4
    dt = sample(n)
    while dt < 0.5 and n < prob.mesh.n_cells:
        n = min(prob.mesh.n_cells, n * 4)
        dt = sample(n)
    n_target = int(min(prob.mesh.n_cells, max(1, n * target_s / max(dt, 1e-6))))
    if max_cells:
        n_target = min(n_target, max_cells)
    dt = sample(n_target)
    return n_target / dt, n_target, dt


def _oracle_worker(workload, lo, hi, barrier, results):
    """One host core's share of the all-cores oracle timing: the same oracle call
    as oracle_rate on cells [lo, hi) of the workload, started together with the
    other workers."""
    import oracle
    from paper_1708_01773_gb300 import inputs
    prob = inputs.WORKLOADS[workload]()
    sub = inputs.Problem(prob.name, inputs.Mesh(prob.mesh.coords, prob.mesh.cell_vertices[lo:hi]), prob.order,
                         prob.quad_1d, prob.problem, prob.coef[lo:hi], prob.force, prob.nu)
    barrier.wait()
    t = time.perf_counter()
    oracle.assemble_csr(sub)
    results.put((hi - lo, time.perf_counter() - t))


def oracle_rate_all_cores(workload: str, n_cells: int, cells_per_core: int):
    """The single-threaded oracle run as one process per host core (spawned, so
    that no CUDA state is inherited), each on its own range of cells_per_core
    cells, all released together. Returns (cells/s over the slowest worker,
    cores, seconds)."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0))
    ctx = mp.get_context("spawn")
    barrier, results = ctx.Barrier(cores), ctx.Queue()
    span = max(1, n_cells - cells_per_core)
    procs = []
    for i in range(cores):
        lo = (i * cells_per_core) % span
        procs.append(ctx.Process(target=_oracle_worker,
                                 args=(workload, lo, min(n_cells, lo + cells_per_core), barrier, results)))
    for pr in procs:
        pr.start()
    got = [results.get(timeout=600) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
    cells = sum(c for c, _ in got)
    wall = max(dt for _, dt in got)
    return cells / wall, cores, wall


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1708_01773_gb300 import inputs
    import oracle
    oracle.build()
    prob = inputs.WORKLOADS[args.workload]()
    # size one step so that warmup + steps take about two minutes in total
    per_step = max(0.5, min(20.0, 120.0 / max(1, args.steps + args.warmup)))
    rate, n, _ = oracle_rate(prob, per_step)
    import oracle as _o  # noqa: F401
    times = []
    from paper_1708_01773_gb300 import inputs as _i
    cv = prob.mesh.cell_vertices[:n]
    sub = _i.Problem(prob.name, _i.Mesh(prob.mesh.coords, cv), prob.order, prob.quad_1d, prob.problem,
                     prob.coef[:n], prob.force, prob.nu)
    for s in range(args.warmup + args.steps):
        t = time.perf_counter()
        oracle.assemble_csr(sub)
        if s >= args.warmup:
            times.append(time.perf_counter() - t)
    step = float(np.mean(times))
    value = n / step
    out = {
        "impl": "reference", "metric": metric_of(args.workload), "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "cells": int(prob.mesh.n_cells), "sample_cells": int(n),
                   "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"first {n} cells of {args.workload}, single-threaded C oracle, "
                                   f"numbering + cell loop + COO compress per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(out), flush=True)
    return 0


# ----------------------------------------------------------------------------- extra workloads
def time_events(fn, n, stream):
    import torch
    for _ in range(3):
        fn()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(n):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / n


def split_kernels(sp, coef, force, vals, rhs, prec, stream, n=5):
    """Cell-kernel and scatter times (ms) of one assembly, from an event recorded between them."""
    import torch
    from paper_1708_01773_gb300 import feasm
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(n)] for _ in range(3)]
    for e in evs[1]:
        e.record(stream)
    torch.cuda.synchronize()
    for k in range(n):
        evs[0][k].record(stream)
        feasm.fe_assemble_ex(sp.handle, coef, force, vals, rhs, feasm.PRECISIONS[prec], stream, evs[1][k].cuda_event)
        evs[2][k].record(stream)
    torch.cuda.synchronize()
    cell = float(np.mean([evs[0][k].elapsed_time(evs[1][k]) for k in range(n)]))
    scat = float(np.mean([evs[1][k].elapsed_time(evs[2][k]) for k in range(n)]))
    return {"cell_ms": cell, "scatter_ms": scat}


def clamped_beam(dev, stream):
    """The Q2 beam with its x = 0 face clamped to a prescribed linear displacement
    (strong Dirichlet conditions): fe_assemble_dirichlet against fe_assemble on the
    same space, and the algorithmic bytes of the constrained scatter."""
    import torch
    from paper_1708_01773_gb300 import feasm, inputs
    prob = inputs.elasticity_q2_beam()
    sp = feasm.FESpace(prob)
    pos = sp.dof_points()
    fixed = np.abs(pos[:, 0]) < 1e-12
    comp = np.arange(sp.n_dofs) % 3
    disp = np.stack([0.01 * pos[:, 1], -0.02 * pos[:, 2], 0.03 * (pos[:, 1] - 0.5)], axis=1)
    dsys = sp.dirichlet(fixed)
    coef = torch.tensor(prob.coef, device=dev)
    uD = torch.tensor(disp[fixed, comp[fixed]], device=dev)
    vals = torch.empty(dsys.nnz, dtype=torch.float64, device=dev)
    rhs = torch.empty(dsys.n_free, dtype=torch.float64, device=dev)
    vals_u = torch.empty(sp.nnz, dtype=torch.float64, device=dev)
    rhs_u = torch.empty(sp.n_dofs, dtype=torch.float64, device=dev)
    cd = sp.cell_dofs()
    free_inc = int((~fixed[cd]).sum())          # (cell, local DOF) incidences of free rows
    rec = {}
    for prec in ("fp32", "fp64"):
        pr = feasm.PRECISIONS[prec]
        ms = time_events(lambda: feasm.fe_assemble_dirichlet(dsys.handle, coef, prob.force, uD, vals, rhs, pr,
                                                             stream), 20, stream)
        ms_u = time_events(lambda: feasm.fe_assemble(sp.handle, coef, prob.force, vals_u, rhs_u, pr, stream),
                           20, stream)
        split = split_kernels(sp, coef, prob.force, vals_u, rhs_u, prec, stream)
        tk = 8 if prec == "fp64" else 4
        sbytes = (free_inc * sp.nl * (tk + 2) + dsys.nnz * 8 + free_inc * (4 + 8) + (dsys.n_free + 1) * 24
                  + dsys.n_free * 8)
        rec[prec] = {"ms_per_step": ms, "cells_per_s": sp.n_cells / (ms / 1e3), "nnz_per_s": dsys.nnz / (ms / 1e3),
                     "unconstrained_ms_per_step": ms_u, "cell_ms": split["cell_ms"],
                     "lift_and_scatter_ms": ms - split["cell_ms"], "scatter_algorithmic_bytes": int(sbytes)}
    torch.cuda.synchronize()
    out = {"cells": sp.n_cells, "n_free": dsys.n_free, "n_fixed": dsys.n_fixed, "nnz": dsys.nnz, **rec}
    dsys.close()
    sp.close()
    return out


def cantilever_compliance(dev, stream):
    """The 64^3 Q1 cantilever clamped at x = 0 under its body force: fe_compliance
    (assembly of the constrained system, Jacobi PCG in FP64 to ||r|| <= 1e-8 ||f||,
    c and dc/dE). Per-iteration time = (call - assembly - gradient) / iterations,
    against the algorithmic bytes of one iteration (compulsory traffic, below)."""
    import torch
    from paper_1708_01773_gb300 import feasm, inputs
    prob = inputs.cantilever_q1_64()
    sp = feasm.FESpace(prob)
    fixed = np.abs(sp.dof_points()[:, 0]) < 1e-12
    dsys = sp.dirichlet(fixed)
    coef = torch.tensor(prob.coef, device=dev)
    work = torch.empty(feasm.fe_compliance_work_size(dsys.handle), dtype=torch.float64, device=dev)
    u = torch.empty(sp.n_dofs, dtype=torch.float64, device=dev)
    c = torch.empty(1, dtype=torch.float64, device=dev)
    g = torch.empty(sp.n_cells, dtype=torch.float64, device=dev)
    vals = torch.empty(dsys.nnz, dtype=torch.float64, device=dev)
    rhs = torch.empty(dsys.n_free, dtype=torch.float64, device=dev)
    n, nnz = dsys.n_free, dsys.nnz
    # compulsory bytes: SpMV values + columns, row pointers, p read, q written (p's
    # gathers hit the L2: 6.5 MB); update reads x, p, q, r, D^-1 and writes x, r, z;
    # the p update reads z, p and writes p
    iter_bytes = nnz * (8 + 4) + n * 8 * (3 + 8 + 3)
    rec = {}
    for prec in ("fp32", "fp64"):
        pr = feasm.PRECISIONS[prec]
        it_rel = [None]

        def call():
            it_rel[0] = feasm.fe_compliance(dsys.handle, coef, prob.force, pr, 1e-8, 100000, work, u, c, g, stream)
        t_call = time_events(call, 3, stream)
        t_asm = time_events(lambda: feasm.fe_assemble_dirichlet(dsys.handle, coef, prob.force, None, vals, rhs, pr,
                                                                stream), 10, stream)
        pa = feasm.PRECISIONS["fp64" if prec == "fp64" else "fp32"]
        t_adj = time_events(lambda: feasm.fe_assemble_adjoint(sp.handle, u, coef, -1.0, g, None, pa, stream), 10,
                            stream)
        it, rel = it_rel[0]
        t_it = (t_call - t_asm - t_adj) / it
        rec[prec] = {"ms_per_call": t_call, "cells_per_s": sp.n_cells / (t_call / 1e3), "iterations": it,
                     "rel_residual": rel, "assembly_ms": t_asm, "gradient_ms": t_adj, "ms_per_iteration": t_it,
                     "iteration_algorithmic_bytes": int(iter_bytes),
                     "iteration_gbs": iter_bytes / (t_it / 1e3) / 1e9, "compliance": float(c)}
    out = {"cells": sp.n_cells, "n_free": n, "nnz": nnz, **rec}
    dsys.close()
    sp.close()
    return out


def extra_workloads(args, dev, stream):
    """Secondary measurements (all, or those named by --extra): the clamped Q2 beam
    (strong Dirichlet conditions), the clamped cantilever's self-adjoint compliance
    solve, the Stokes Taylor-Hood assembly, the interior penalty DG assembly, the
    scatter-bound 128^3 Q1 elasticity assembly, the 64^3 Q1 cantilever
    compliance adjoint and (with --batched) the batched assembly."""
    want = (lambda name: args.extra is None or name in args.extra)
    out = {}
    if want("elasticity_q2_beam_clamped"):
        out["elasticity_q2_beam_clamped"] = clamped_beam(dev, stream)
    if want("cantilever_q1_64_compliance"):
        out["cantilever_q1_64_compliance"] = cantilever_compliance(dev, stream)
    if want("stokes_q2q1_32"):
        out["stokes_q2q1_32"] = stokes_32(dev, stream)
    if want("dg_q2_32"):
        out["dg_q2_32"] = dg_32(dev, stream)
    if want("elasticity_q1_128"):
        out["elasticity_q1_128"] = q1_128(dev, stream)
    if want("cantilever_q1_64_adjoint"):
        out["cantilever_q1_64_adjoint"] = adjoint_64(dev, stream)
    if args.batched:
        out["batched64"] = batched(dev, stream)
    return out


def stokes_32(dev, stream):
    """Stokes, Taylor-Hood Q2/Q1 on 32^3 cells (the paper's driver workload),
    FP32 and FP64 forms: step time, cell and scatter kernels, their algorithmic
    bytes."""
    import torch
    from paper_1708_01773_gb300 import feasm, inputs
    prob = inputs.stokes_q2q1_32()
    sp = feasm.FESpace(prob)
    coef = torch.tensor(prob.coef, device=dev)
    vals = torch.empty(sp.nnz, dtype=torch.float64, device=dev)
    rhs = torch.empty(sp.n_dofs, dtype=torch.float64, device=dev)
    rec = {}
    for prec in ("fp32", "fp64"):
        ms = time_events(lambda: feasm.fe_assemble(sp.handle, coef, prob.force, vals, rhs, feasm.PRECISIONS[prec],
                                                   stream), 10, stream)
        split = split_kernels(sp, coef, prob.force, vals, rhs, prec, stream)
        sb, cb = scatter_bytes(sp, prec), cell_bytes(sp, prec)
        rec[prec] = {"ms_per_step": ms, "cells_per_s": sp.n_cells / (ms / 1e3), "nnz_per_s": sp.nnz / (ms / 1e3),
                     **split, "scatter_gbs": sb / (split["scatter_ms"] / 1e3) / 1e9,
                     "cell_gbs": cb / (split["cell_ms"] / 1e3) / 1e9, "scatter_algorithmic_bytes": sb,
                     "cell_algorithmic_bytes": cb}
    sp.close()
    return {"cells": sp.n_cells, "dofs": sp.n_dofs, "velocity_dofs": sp.n_first, "nnz": sp.nnz, **rec}


def dg_32(dev, stream):
    """Interior penalty DG (Poisson, discontinuous Q2) on 32^3 cells, tau = 1,
    gamma = 10, f = 1: assembly time per call (cell integrals, facet blocks, block
    rows), and the algorithmic bytes of the facet and row kernels."""
    import torch
    from paper_1708_01773_gb300 import feasm, inputs
    mesh = inputs.dg_q2_32()
    g = feasm.DGSpace(mesh, 2)
    vals = torch.empty(g.nnz, dtype=torch.float64, device=dev)
    rhs = torch.empty(g.n_dofs, dtype=torch.float64, device=dev)
    nb2 = 27 * 27
    facet_bytes = (4 * g.n_interior + g.n_boundary) * nb2 * 8 + mesh.n_cells * 24 * 8
    rec = {}
    for prec in ("fp32", "fp64"):
        tk = 8 if prec == "fp64" else 4
        ms = time_events(lambda: g.assemble(1.0, 10.0, 1.0, vals, rhs, prec=prec, stream=stream), 10, stream)
        row_bytes = (mesh.n_cells * nb2 * tk + (4 * g.n_interior + g.n_boundary) * nb2 * 8 + g.nnz * 8
                     + (g.n_dofs + 1) * 8 + g.n_dofs * 16)
        rec[prec] = {"ms_per_step": ms, "cells_per_s": mesh.n_cells / (ms / 1e3), "nnz_per_s": g.nnz / (ms / 1e3),
                     "facet_algorithmic_bytes": int(facet_bytes), "row_algorithmic_bytes": int(row_bytes)}
    out = {"cells": mesh.n_cells, "dofs": g.n_dofs, "nnz": g.nnz, "interior_facets": g.n_interior,
           "boundary_facets": g.n_boundary, **rec}
    g.close()
    return out


def q1_128(dev, stream):
    """The scatter-bound 128^3 Q1 elasticity assembly, FP32 and FP64 forms."""
    import torch
    from paper_1708_01773_gb300 import feasm, inputs
    prob = inputs.elasticity_q1_128()
    sp = feasm.FESpace(prob)
    coef = torch.tensor(prob.coef, device=dev)
    vals = torch.empty(sp.nnz, dtype=torch.float64, device=dev)
    rhs = torch.empty(sp.n_dofs, dtype=torch.float64, device=dev)
    rec = {}
    for prec in ("fp32", "fp64"):
        ms = time_events(lambda: feasm.fe_assemble(sp.handle, coef, prob.force, vals, rhs, feasm.PRECISIONS[prec],
                                                   stream), 10, stream)
        rec[prec] = {"ms_per_step": ms, "cells_per_s": sp.n_cells / (ms / 1e3), "nnz_per_s": sp.nnz / (ms / 1e3),
                     **split_kernels(sp, coef, prob.force, vals, rhs, prec, stream)}
    sp.close()
    return {"cells": sp.n_cells, "nnz": sp.nnz, **rec}


def adjoint_64(dev, stream):
    """The compliance adjoint on the 64^3 Q1 cantilever for a fixed seeded u."""
    import torch
    from paper_1708_01773_gb300 import feasm, inputs
    prob = inputs.cantilever_q1_64()
    sp = feasm.FESpace(prob)
    u = torch.tensor(inputs.unit_rms_field(sp.n_dofs, inputs.SEED_BASE + 5), device=dev)
    E = torch.tensor(prob.coef, device=dev)
    g = torch.empty(sp.n_cells, dtype=torch.float64, device=dev)
    c = torch.empty(1, dtype=torch.float64, device=dev)
    rec = {}
    for prec in ("fp64", "fp32"):
        ms = time_events(lambda: feasm.fe_assemble_adjoint(sp.handle, u, E, 1.0, g, c, feasm.PRECISIONS[prec],
                                                           stream), 20, stream)
        rec[prec] = {"ms_per_call": ms, "cells_per_s": sp.n_cells / (ms / 1e3)}
    sp.close()
    return {"cells": sp.n_cells, **rec}


def batched(dev, stream):
    """The 64-mesh batched assembly (one persistent launch in a CUDA graph)."""
    import torch
    from paper_1708_01773_gb300 import feasm, inputs
    probs = inputs.batched64()
    t0 = time.perf_counter()
    spaces = [feasm.FESpace(p) for p in probs]
    setup = time.perf_counter() - t0
    coefs = [torch.tensor(p.coef, device=dev) for p in probs]
    vals = [torch.empty(s.nnz, dtype=torch.float64, device=dev) for s in spaces]
    rhss = [torch.empty(s.n_dofs, dtype=torch.float64, device=dev) for s in spaces]
    cells = sum(s.n_cells for s in spaces)
    nnz = sum(s.nnz for s in spaces)
    rec = {}
    for prec in ("fp32", "bf16", "fp64"):
        b = feasm.fe_batch_create([s.handle for s in spaces])
        ms = time_events(lambda: feasm.fe_batch_assemble(b, coefs, [p.force for p in probs], vals, rhss,
                                                         feasm.PRECISIONS[prec], stream), 3, stream)
        rec[prec] = {"ms_per_step": ms, "cells_per_s": cells / (ms / 1e3), "nnz_per_s": nnz / (ms / 1e3)}
        feasm.fe_batch_destroy(b)
    for s in spaces:
        s.close()
    return {"meshes": len(probs), "cells": cells, "nnz": nnz, "setup_s": setup,
            "redraw_attempt": probs[0].extra.get("attempt"), **rec}


# ----------------------------------------------------------------------------- GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_1708_01773_gb300 import build, feasm, inputs
    build.build()

    prob = inputs.WORKLOADS[args.workload]()
    t0 = time.perf_counter()
    if args.reorder:
        prob = inputs.reordered(prob, feasm.fe_mesh_locality_order(prob.mesh.coords, prob.mesh.cell_vertices))
    sp = feasm.FESpace(prob)
    setup_s = time.perf_counter() - t0
    sp.set_kernel(args.kernel)
    prec = feasm.PRECISIONS[args.prec]
    dev = torch.device("cuda", local)
    coef = torch.tensor(prob.coef, device=dev)
    vals = torch.empty(sp.nnz, dtype=torch.float64, device=dev)
    rhs = torch.empty(sp.n_dofs, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def step(ev_mid=None):
        if ev_mid is None:
            feasm.fe_assemble(sp.handle, coef, prob.force, vals, rhs, prec, stream)
        else:
            feasm.fe_assemble_ex(sp.handle, coef, prob.force, vals, rhs, prec, stream, ev_mid.cuda_event)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if sp.status() != 0:
        raise RuntimeError("device error during warm-up")

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(K)] for _ in range(3)]
    for e in ev[1]:
        e.record(stream)  # materialise the event handles before handing them to the library
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for k in range(K):
            ev[0][k].record(stream)
            step(ev[1][k])
            ev[2][k].record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if sp.status() != 0:
        raise RuntimeError("device error in the timed region")
    total_ms = ev[0][0].elapsed_time(ev[2][K - 1])
    cell_ms = [ev[0][k].elapsed_time(ev[1][k]) for k in range(K)]
    scat_ms = [ev[1][k].elapsed_time(ev[2][k]) for k in range(K)]
    total_ms = max_over_ranks(total_ms, dev)
    ms_per_step = total_ms / K
    value = whole_job_rate(sp.n_cells, ws, K, total_ms)

    # end to end through the host-buffer entry point (pinned memory, copies timed)
    Ke2e = max(3, min(K, 20))
    hc = torch.tensor(prob.coef).pin_memory()
    hv = torch.empty(sp.nnz, dtype=torch.float64).pin_memory()
    hr = torch.empty(sp.n_dofs, dtype=torch.float64).pin_memory()
    feasm.fe_assemble_host(sp.handle, hc, prob.force, hv, hr, prec, stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(Ke2e):
        feasm.fe_assemble_host(sp.handle, hc, prob.force, hv, hr, prec, stream)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / Ke2e
    e2e_s = max_over_ranks(e2e_s, dev)

    # same-GPU comparators (plain FP64 assembler, BF16 form)
    comparators = {}
    if not args.no_comparators:
        for name in ("fp64", "fp32", "bf16"):
            if name == args.prec:
                continue
            p2 = feasm.PRECISIONS[name]
            sp.set_kernel("auto" if name == "fp64" else args.kernel)  # FP64 has CUDA-core kernels only
            for _ in range(3):
                feasm.fe_assemble(sp.handle, coef, prob.force, vals, rhs, p2, stream)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            n2 = 20
            a.record(stream)
            for _ in range(n2):
                feasm.fe_assemble(sp.handle, coef, prob.force, vals, rhs, p2, stream)
            b.record(stream)
            torch.cuda.synchronize()
            comparators[name] = {"cells_per_s": sp.n_cells * n2 / (a.elapsed_time(b) / 1e3),
                                 "ms_per_step": a.elapsed_time(b) / n2}

    hbm, bf16_tf, peak_src = measured_peaks()
    cell_avg, scat_avg = float(np.mean(cell_ms)), float(np.mean(scat_ms))
    cell_name, scat_name = kernel_names(prob, args.prec, args.kernel)
    kernels = {
        "k_scatter": {"ms": scat_avg, "bytes": scatter_bytes(sp, args.prec), "name": scat_name},
        "k_cell": {"ms": cell_avg, "bytes": cell_bytes(sp, args.prec), "name": cell_name},
    }
    for k in kernels.values():
        k["gbs"] = k["bytes"] / (k["ms"] / 1e3) / 1e9
        k["frac"] = k["gbs"] / hbm
    if on_tensor_cores(prob, args.prec, args.kernel):
        # the contraction runs on tcgen05 (3xTF32 for the FP32 form, BF16): its
        # algorithmic flops per cell, 2 nl^2 K for the Gram of nl rows over K
        # columns (elasticity: 3 nb rows, nq columns; Poisson: nb rows, 3 nq
        # columns), times the passes of the split, against the dtype's peak (TF32:
        # the measured BF16 burst x 1.1 / 2.25)
        passes, peak_tf = (3, bf16_tf * 1.1 / 2.25) if args.prec == "fp32" else (1, bf16_tf)
        kdim = prob.quad_1d ** 3 * (1 if prob.problem == inputs.ELASTICITY else 3)
        flops = sp.n_cells * sp.nl * sp.nl * kdim * 2
        tflops = passes * flops / (cell_avg / 1e3) / 1e12
        kernels["k_cell"].update({"contraction_flops": int(flops), "tensor_passes": passes,
                                  "tensor_tflops": tflops, "tensor_peak_tflops": peak_tf,
                                  "tensor_frac": tflops / peak_tf,
                                  "tensor_dtype": "tf32 (3xTF32)" if args.prec == "fp32" else "bf16"})
    dom = max(kernels, key=lambda k: kernels[k]["ms"])
    roof = {"kernel": kernels[dom]["name"], "bound": "hbm", "achieved": kernels[dom]["gbs"], "peak": hbm,
            "unit": "GB/s", "frac": kernels[dom]["frac"], "traffic": kernel_traffic(args.workload, dom, sp.n_cells),
            "algorithmic_bytes": kernels[dom]["bytes"], "peak_source": peak_src + " (burst copy)"}

    extras = extra_workloads(args, dev, stream) if (args.extras or args.batched or args.extra) else None

    cpu = cpu_all = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, n, dt = oracle_rate(prob, 12.0)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {n} cells of {args.workload} ({dt:.1f} s), single-threaded C oracle: "
                         f"numbering + cell loop + COO compress"}
        # the same oracle on every host core: one process per core, each on its own cell range
        per_core = max(1, int(rate * 6.0))
        rate_all, cores, wall = oracle_rate_all_cores(args.workload, int(prob.mesh.n_cells), per_core)
        cpu_all = {"value": rate_all, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"{cores} processes x {per_core} cells of {args.workload} ({wall:.1f} s), "
                             f"the single-threaded C oracle per process on its own cell range"}

    if rank == 0:
        out = {
            "metric": metric_of(args.workload), "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16": "bf16", "fp64": "f64"}[args.prec], "data": "synthetic",
            "config": {"workload": args.workload, "cells": int(sp.n_cells), "dofs": int(sp.n_dofs),
                       "nnz": int(sp.nnz), "contributions": int(sp.n_contrib), "order": prob.order,
                       "precision": f"{args.prec} contraction, fp64 geometry + fp64 CSR accumulation",
                       "l2": "working set > L2 (no flush)", "parallelism": f"replicas x{ws}",
                       "kernel": args.kernel, "setup_s": setup_s,
                       "cell_order": "morton (fe_mesh_locality_order)" if args.reorder else "as generated"},
            "nnz_per_s": value / sp.n_cells * sp.nnz,
            "e2e": {"value": ws * sp.n_cells / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(sp.n_cells * 8),
                    "d2h_bytes_per_step": int((sp.nnz + sp.n_dofs) * 8)},
            "gpu_launches": 2 * K,
            "roofline": roof,
            "kernels": kernels,
            "comparators": comparators,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
            "cpu_baseline_all_cores": cpu_all,
        }
        if extras:
            out["extra_workloads"] = extras
        print(json.dumps(out), flush=True)
    sp.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
