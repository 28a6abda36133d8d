#!/usr/bin/env python
"""Throughput of the batched npFEM step on B300 (one JSON line on stdout).

A step is one npfem_step over the whole batch: every cell runs the full quasi-Newton
solve (prediction, local projections, global FP64 solves, L-BFGS, line search,
write-back).  Metric: RBC-equivalent cell-steps per second, one RBC-equivalent being
(n_vertices/642)*(iterations/5).  Default workload: the heterogeneous 10^4-cell batch
(4500 642-vertex RBCs, 4500 2562-vertex RBCs, 1000 162-vertex platelets, 3..8 iterations
per cell), FP32 form (FP32 local work, FP64 factor/solves/reductions), followed by a
short pass of the same batch in the plain FP64 form for the FP32-form speed-up.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload hetero10k|homog4096|...]
                  [--precision fp32form|fp64] [--impl ours|reference] [--tune]

`--impl reference` times the CPU FP64 oracle (the only other implementation of the
method) on a bounded sample of the same workload.  Under torchrun every rank steps its
own batch (cells are independent: no collective); rank 0 prints the line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "RBC-equivalent cell-steps/sec on 1 B300 at stated residual"
UNIT = "RBC-equivalent cell-steps/s"


# Rayleigh damping (c_alpha 1/us, c_beta us) given to every cell type (--damping)
DAMPING = (0.0, 0.0)
# strain limits (s_min, s_max) given to every cell type (--strain-limits); (0, 0): none
STRAIN_LIMITS = (0.0, 0.0)


def _mat(spec):
    """Material tuple of a cell-type spec, with the benchmark's damping and strain limits
    appended (the limits only when set)."""
    m = spec.material.as_tuple() + DAMPING
    return m + STRAIN_LIMITS if any(STRAIN_LIMITS) else m


# ------------------------------------------------------------------ workloads
# collision parameters (search radius um, contact thickness um, weight nN/um) per workload
# (and whether the packing box's walls act: a box 1 um outside the initial cells)
COLLISIONS = {"pack4096": (0.5, 0.05, 60.0, False), "packbox4096": (0.5, 0.05, 60.0, True)}


def _box(b, coll):
    """The wall box of a collision workload (lo[3], hi[3]), or None."""
    if coll is None or not coll[3]:
        return None
    return (b.x.min(axis=1) - 1.0, b.x.max(axis=1) + 1.0)


def make_workload(name: str, rank: int = 0):
    from paper_2011_04332_b300 import inputs as I
    if name == "homog4096":
        b = I.homogeneous_rbc_batch(ncells=4096, seed=1001 + 100 * rank)
        desc = "homogeneous 4096 RBC (642 vertices, Evans-Fung), 5 iterations, random placement in a 200 um box"
    elif name == "hetero10k":
        b = I.heterogeneous_batch(4500, 4500, 1000, seed=1002 + 100 * rank)
        desc = ("heterogeneous 10^4 cells: 4500 RBC 642v + 4500 RBC 2562v + 1000 PLT 162v, "
                "3..8 iterations per cell, seeded random order")
    elif name == "homog1776":
        b = I.homogeneous_rbc_batch(ncells=1776, seed=1001 + 100 * rank)
        desc = "homogeneous 1776 RBC (642 vertices; one cell per warp slot of 148 SMs x 12 warps), 5 iterations"
    elif name == "stress20k":
        b = I.stress_mix_batch(ncells=20000, seed=1005 + 100 * rank)
        desc = ("serving-shaped mix: 20000 cells (70 % RBC 642v, 10 % RBC 2562v, 20 % PLT 162v), "
                "5 iterations, force field re-drawn every 10 steps")
    elif name == "homog2562":
        b = I.homogeneous_rbc_batch(ncells=1184, seed=1001 + 100 * rank, subdiv=4)
        desc = "homogeneous 1184 RBC (2562 vertices, Evans-Fung), 5 iterations"
    elif name in ("pack4096", "packbox4096"):
        b = I.packing_batch(4096, 0, hematocrit=0.35, seed=1006 + 100 * rank)
        r, d, w, walls = COLLISIONS[name]
        desc = ("cell packing: 4096 RBC (642 vertices) at rest with random positions and orientations in a "
                f"cube at 35 % volume fraction (overlapping), 5 iterations, collisions radius {r} um, "
                f"delta {d} um, weight {w} nN/um, contact detection inside every step"
                + ("; box walls 1 um outside the initial cells" if walls else ""))
    elif name == "plt1776":
        b = I.placed_cells([I.CellTypeSpec(I.platelet_mesh(2), I.PLT_MATERIAL)], [0] * 1776, 1007 + 100 * rank, 5)
        desc = "homogeneous 1776 platelets (162 vertices, oblate ellipsoid), 5 iterations"
    elif name == "small":
        b = I.homogeneous_rbc_batch(ncells=64, seed=1001 + 100 * rank)
        desc = "64 RBC (642 vertices), 5 iterations"
    else:
        raise SystemExit(f"unknown workload {name}")
    return b, desc


def residual_mode(b, desc: str, tol: float, budget: int):
    """Converged-residual mode (tol > 0): every cell's count becomes the budget and the
    step ends per cell at |g|/|g0| < tol."""
    if tol > 0:
        b.iters = np.full(b.ncells, budget, dtype=np.int32)
        desc += (f"; converged-residual mode in place of the fixed counts: each cell stops at |g|/|g0| < {tol:g} "
                 f"(budget {budget} iterations)")
    return b, desc


# ------------------------------------------------------------------ oracle baseline
def _oracle_worker(args):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import npfem_oracle as O
    mesh_v, mesh_t, mat, dt, cells, tol = args
    ct = O.CellType(mesh_v, mesh_t, mat, dt)
    t0 = time.perf_counter()
    for (x, v, f, it, con, wl) in cells:
        O.step(ct.rest, ct.solver, x, v, f, int(it), tol=tol, contact=con, walls=wl)
    return time.perf_counter() - t0, len(cells)


def step_units(b, sel=None, tol: float = 0.0) -> float:
    """RBC-equivalent cell-steps of one step over the cells `sel` (default all): a cell
    of n vertices counts n/642; with fixed counts it is also weighted by iterations/5
    (five iterations of a 642-vertex RBC = 1), in the converged-residual mode (tol > 0)
    every cell-step is delivered at the stated residual and counts n/642."""
    sel = np.arange(b.ncells) if sel is None else np.asarray(sel)
    n = np.array([b.types[int(b.type_of_cell[c])].mesh.n for c in sel], dtype=np.float64)
    if tol > 0:
        return float(np.sum(n / 642.0))
    return float(np.sum(n / 642.0 * b.iters[sel] / 5.0))


def oracle_baseline(b, sample_cells: int, workers: int, tol: float = 0.0, collisions=None):
    """Time the oracle on the first `sample_cells` cells, one step each, spread over
    `workers` single-threaded processes (spawn).  Returns (rbc_eq per s, cores, desc)."""
    import multiprocessing as mp
    sel = list(range(min(sample_cells, b.ncells)))
    contacts, t_detect = {}, 0.0
    if collisions is not None:
        # the sampled cells' contact detection (over the whole batch) is part of their step
        from oracle import npfem_oracle as O
        radius, delta, weight = collisions[:3]
        ots = [O.CellType(t.mesh.verts, t.mesh.tris, _mat(t), b.dt) for t in b.types]
        verts = [i for c in sel for i in range(int(b.offsets[c]), int(b.offsets[c + 1]))]
        t0 = time.perf_counter()
        con = O.detect_contacts(ots, b.type_of_cell, b.offsets, b.x, radius, vertices=verts)
        for c in sel:
            contacts[c] = (*O.cell_contacts(con, int(b.offsets[c]), int(b.offsets[c + 1])), delta, weight)
        t_detect = time.perf_counter() - t0
    box = _box(b, collisions)
    walls = None if box is None else (box[0], box[1], collisions[1], collisions[2])
    by_type = {}
    for c in sel:
        by_type.setdefault(int(b.type_of_cell[c]), []).append(c)
    jobs = []
    for t, cells in by_type.items():
        ty = b.types[t]
        chunks = [cells[i::workers] for i in range(workers)]
        for ch in chunks:
            if ch:
                jobs.append((ty.mesh.verts, ty.mesh.tris, _mat(ty), b.dt,
                             [(*b.cell_state(c), b.iters[c], contacts.get(c), walls) for c in ch], tol))
    ctx = mp.get_context("spawn")
    env_backup = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_backup:
        os.environ[k] = "1"
    try:
        t0 = time.perf_counter()
        with ctx.Pool(workers) as pool:
            res = pool.map(_oracle_worker, jobs)
        wall = time.perf_counter() - t0
    finally:
        for k, v in env_backup.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    busy = max(r[0] for r in res)  # the slowest worker's stepping time (setup excluded)
    rbc_eq = step_units(b, sel, tol)
    desc = (f"{len(sel)} cells x 1 step of the same workload (first cells in batch order), "
            f"{workers} single-threaded processes; type setup excluded; wall incl. setup {wall:.1f}s")
    if collisions is not None:
        busy += t_detect
        desc += f"; contact detection of the sampled cells (one process) {t_detect:.2f}s included"
    return rbc_eq / busy, workers, desc


# ------------------------------------------------------------------ parity sample
def sample_cells(b, per_type: int = 3):
    """The cells the parity check compares with the oracle: for every cell type the
    first, middle and last cell of that type in batch order (all, if it has fewer)."""
    out = []
    for t in sorted({int(q) for q in b.type_of_cell}):
        idx = np.flatnonzero(b.type_of_cell == t)
        pos = np.unique(np.linspace(0, len(idx) - 1, per_type).round().astype(int))
        out += [int(idx[i]) for i in pos]
    return sorted(out)


def oracle_parity(b, x0, v0, f, xs, cells, bar, tol, coll, done_gpu, ocache):
    """Per-cell relative position error (max |x - x_oracle| over the cell radius) of the
    GPU step xs taken from (x0, v0, f) against the oracle's step of the same inputs, for
    the sampled cells; reported per cell type.  FP32-form runs give the oracle the
    FP32-rounded inputs (x0, v0, f as stored)."""
    from oracle import npfem_oracle as O
    xin, vin, fin = (t.double().cpu().numpy() for t in (x0, v0, f))
    scon = None
    if coll is not None:
        allt = [O.CellType(t.mesh.verts, t.mesh.tris, _mat(t), b.dt) for t in b.types]
        scon = O.detect_contacts(allt, b.type_of_cell, b.offsets, xin, coll[0],
                                 vertices=[i for c in cells for i in range(int(b.offsets[c]), int(b.offsets[c + 1]))])
    bx = _box(b, coll)
    wl = None if bx is None else (bx[0], bx[1], coll[1], coll[2])
    xg = xs.double().cpu().numpy()
    per_type, counts = {}, []
    for c in cells:
        t = int(b.type_of_cell[c])
        if t not in ocache:
            ty = b.types[t]
            ocache[t] = O.CellType(ty.mesh.verts, ty.mesh.tris, _mat(ty), b.dt)
        s = b.cell_slice(c)
        con = None if scon is None else (*O.cell_contacts(scon, s.start, s.stop), coll[1], coll[2])
        r = O.step(ocache[t].rest, ocache[t].solver, xin[:, s].T, vin[:, s].T, fin[:, s].T, int(b.iters[c]), tol=tol,
                   contact=con, walls=wl)
        rad = np.max(np.linalg.norm(r.x - r.x.mean(axis=0), axis=1))
        e = float(np.max(np.abs(xg[:, s].T - r.x)) / rad)
        key = f"{t}:{b.types[t].mesh.n}v"
        per_type[key] = max(per_type.get(key, 0.0), e)
        if done_gpu is not None:
            counts.append((int(done_gpu[c]), len(r.alphas)))
    worst = max(per_type.values())
    out = {"cells": cells, "per_type_max_rel_position_error": per_type, "max_rel_position_error": worst,
           "bar": bar, "pass": bool(worst <= bar),
           "definition": "max over the cell's vertices of |x - x_oracle|_inf / cell radius, one step from the "
                         "same inputs; per cell type the max over its sampled cells (first, middle, last)"}
    if done_gpu is not None:
        out["iterations_gpu_oracle"] = counts
    return out


# ------------------------------------------------------------------ clocks
class ClockSampler:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            p = [q.strip() for q in line.split(",")]
            if len(p) < 7:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for nm, val in zip(names, p[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ multi-rank aggregation
def max_over_ranks(value: float, world: int, device=None) -> float:
    """Max of a per-rank float over all ranks (identity when world == 1)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, steps: int, max_total_ms: float) -> float:
    """Units all ranks processed (each rank steps its own batch) over the slowest rank's time."""
    return units_per_rank * world * steps / (max_total_ms / 1e3)


# ------------------------------------------------------------------ GPU arm
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2011_04332_b300 import build as B
    from paper_2011_04332_b300 import native
    B.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    b, desc = make_workload(args.workload, rank)
    b, desc = residual_mode(b, desc, args.tol, args.budget)
    tol = args.tol
    # oracle baseline first (spawned processes, before heavy GPU work), rank 0 only
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        # with collisions the oracle's brute-force detection dominates: a smaller sample
        nsample = args.cpu_sample if args.workload not in COLLISIONS else min(args.cpu_sample, 16)
        v, cores, sdesc = oracle_baseline(b, nsample, args.cpu_workers, tol, COLLISIONS.get(args.workload))
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sdesc}

    prec = native.FP32FORM if args.precision == "fp32form" else native.FP64
    tdt = torch.float32 if prec == native.FP32FORM else torch.float64
    types = [native.CellType(t.mesh.verts, t.mesh.tris, _mat(t), b.dt) for t in b.types]
    infos = [t.info() for t in types]
    batch = native.Batch(types, b.type_of_cell, prec)
    coll = COLLISIONS.get(args.workload)
    if coll is not None:
        batch.set_collisions(coll[0], coll[1], coll[2], box=_box(b, coll))
    x0 = torch.tensor(b.x, dtype=tdt, device=dev)
    v0 = torch.tensor(b.v, dtype=tdt, device=dev)
    f = torch.tensor(b.f, dtype=tdt, device=dev)
    fpool = None
    if args.workload == "stress20k":
        # coupling-force updates: the step's force buffer takes a re-drawn field every 10 steps
        from paper_2011_04332_b300 import inputs as I
        fpool = [f.clone()] + [torch.tensor(I.redrawn_forces(b, b.x, 1005 + 100 * rank, k), dtype=tdt, device=dev)
                               for k in (1, 2)]
    iters = torch.tensor(b.iters, device=dev)
    res = torch.zeros(b.ncells, dtype=torch.float64, device=dev)
    st = torch.zeros(b.ncells, dtype=torch.int32, device=dev)
    done = torch.zeros(b.ncells, dtype=torch.int32, device=dev) if tol > 0 else None
    done_sum = torch.zeros(b.ncells, dtype=torch.int64, device=dev) if tol > 0 else None
    x, v = x0.clone(), v0.clone()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 126 MB L2
    stream = torch.cuda.current_stream(dev)

    # sampled parity against the oracle on the first step (rank 0): every cell type
    sample = sample_cells(b)
    err = None
    ocache = {}
    if rank == 0 and not args.no_check:
        xs, vs_ = x0.clone(), v0.clone()
        batch.step(xs, vs_, f, iters=iters, residual=res, status=st, tol=tol, iters_done=done)
        torch.cuda.synchronize()
        err = oracle_parity(b, x0, v0, f, xs, sample, 1e-5 if prec == native.FP32FORM else 1e-10, tol, coll,
                            done.cpu().numpy() if done is not None else None, ocache)

    tuned = None
    if not args.tune and args.groups > 0:
        for t in sorted({int(q) for q in b.type_of_cell}):
            batch.set_groups(t, args.groups)
    if args.tune:
        # launch-shape autotuning on copies of the state (outside the timed region)
        from paper_2011_04332_b300 import tuning
        t0 = time.perf_counter()
        tuned = tuning.autotune_split(batch, x0, v0, f, iters=iters, tol=tol)
        tuned = {"seconds": round(time.perf_counter() - t0, 1),
                 "shapes": {str(t): list(r["split_shape"]) for t, r in tuned.items()},
                 "groups": {str(t): r["groups"] for t, r in tuned.items()}}
    batch.set_kernel_timing(True)       # CUDA events around every launch (also inside the graph)
    for _ in range(args.warmup):
        batch.step(x, v, f, iters=iters, residual=res, status=st, tol=tol, iters_done=done)
    torch.cuda.synchronize()
    graph = None
    if not args.no_graph:
        # one step = one CUDA-graph launch (queue-counter memset + one kernel per cell type)
        graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            with torch.cuda.graph(graph, stream=side):
                batch.step(x, v, f, iters=iters, residual=res, status=st, tol=tol, iters_done=done)
        stream.wait_stream(side)
        torch.cuda.synchronize()
        graph.replay()          # the capture does not execute; replay once as warm-up
        torch.cuda.synchronize()

    def one_step():
        if graph is not None:
            graph.replay()
        else:
            batch.step(x, v, f, iters=iters, residual=res, status=st, tol=tol, iters_done=done)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    present = sorted({int(t) for t in b.type_of_cell})
    ktime = {t: {k: [0.0, 0] for k in native.Batch.KERNELS} for t in present}
    kspan = {k: 0.0 for k in native.Batch.KERNELS}      # union of concurrent launches, all types
    detect_ms = 0.0                                      # contact detection (collisions on)
    t_wall = 0.0                                         # host time of the timed replays only
    with ClockSampler(local_rank) as clk:
        for k in range(args.steps):
            flush.zero_()
            if fpool is not None and k % 10 == 0:
                f.copy_(fpool[(k // 10) % len(fpool)])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ev[k][0].record(stream)
            one_step()
            ev[k][1].record(stream)
            ev[k][1].synchronize()
            t_wall += time.perf_counter() - t0
            # outside the timed interval: iterations each cell ran, and the per-kernel
            # durations of this step (events on the kernels' own streams, re-recorded by
            # every replay, so they are read before the next one)
            if done_sum is not None:
                done_sum += done
            for t in present:
                for name, (kms, kn) in batch.kernel_times(t).items():
                    ktime[t][name][0] += kms
                    ktime[t][name][1] += kn
            for name, sms in batch.kernel_spans(-1).items():
                kspan[name] += sms
            if coll is not None:
                detect_ms += batch.contact_time()
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = [a.elapsed_time(bq) for a, bq in ev]
    total_ms = max_over_ranks(float(sum(ms)), world, dev)
    rbc_eq_per_rank = step_units(b, None, tol)
    value = whole_job_rate(rbc_eq_per_rank, world, args.steps, total_ms)
    ms_per_step = total_ms / args.steps
    resid = res.cpu().numpy()
    status = st.cpu().numpy()

    # roofline of the dominant kernel, npfem_k_solve (the FP64 triangular solves; ALU
    # bound on the FP64 pipe): its algorithmic flops over the time its launches run (the
    # union of their intervals: the chains of a step run concurrently)
    nnz = np.array([infos[t]["nnz_factor"] for t in b.type_of_cell], dtype=np.float64)
    nv = np.array([infos[t]["n_verts"] for t in b.type_of_cell], dtype=np.float64)
    # iterations per cell and step: the fixed counts, or the mean of those run under tol
    its = b.iters.astype(np.float64) if done_sum is None else done_sum.cpu().numpy() / args.steps
    solve_flops = its * (12.0 * nnz + 3.0 * nv)          # per cell and step
    flops_per_step = float(np.sum(solve_flops))
    fp64_peak, fp32_peak = probe_peaks()
    kernels = {}
    for t in present:
        kt = ktime[t]
        step_ms = {name: kt[name][0] / args.steps for name in kt}
        ft = float(np.sum(solve_flops[b.type_of_cell == t]))
        launches = kt["k_solve"][1] / args.steps
        kernels[str(t)] = {"ms_per_step": step_ms, "launches_per_step": {n: kt[n][1] / args.steps for n in kt},
                           "k_solve_flops_per_launch": ft / launches if launches else None,
                           "k_solve_tflops": ft / (step_ms["k_solve"] / 1e3) / 1e12 if step_ms["k_solve"] else None}
    solve_ms_total = sum(ktime[t]["k_solve"][0] for t in present) / args.steps
    solve_launches = sum(ktime[t]["k_solve"][1] for t in present) / args.steps
    solve_span = kspan["k_solve"] / args.steps
    achieved = flops_per_step / (solve_span / 1e3) / 1e12 if solve_span > 0 else None
    # DRAM bytes of an average solve launch: per cell size, the captured bytes per
    # cell-solve times the cell-solves of a step, over the step's solve launches
    traffic_cell, traffic_how = measured_traffic(nv, args.precision)
    traffic = None
    if traffic_cell and solve_launches:
        traffic = float(sum(traffic_cell[int(n)] * i for n, i in zip(nv, its))) / solve_launches
    roofline = {"bound": "alu", "pipe": "fp64", "kernel": "npfem_k_solve", "achieved": achieved, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": achieved / fp64_peak if fp64_peak and achieved else None, "traffic": traffic,
                "traffic_note": traffic_how,
                "peak_source": "measured live: FP64 FMA probe (8 chains/thread, 4 CTAs/SM)",
                "algorithmic": "FP64 flops of the triangular solves: iters*(12*nnz(L)+3n) per cell and step, "
                               f"{flops_per_step / max(solve_launches, 1):.4g} per launch on average",
                "kernel_time": ("CUDA events around each npfem_k_solve launch on its own stream, recorded by the "
                                "timed graph replays; the step's solve launches (%d per step, %.3f ms summed) overlap "
                                "across concurrent chains, so the time is the union of their intervals, %.3f ms per "
                                "step" % (round(solve_launches), solve_ms_total, solve_span)),
                "kernel_share_of_step": solve_span / ms_per_step if ms_per_step else None,
                # the same flops over the summed durations of the solve launches (average launch
                # duration x launches): each launch shares the GPU with the other chains' kernels
                # while it runs, so this reads lower than the union-of-intervals figure
                "achieved_per_launch": (flops_per_step / (solve_ms_total / 1e3) / 1e12) if solve_ms_total > 0 else None,
                "frac_per_launch": (flops_per_step / (solve_ms_total / 1e3) / 1e12 / fp64_peak)
                if solve_ms_total > 0 and fp64_peak else None,
                "step_frac": flops_per_step / (ms_per_step / 1e3) / 1e12 / fp64_peak if fp64_peak else None}

    # HBM: the method's algorithmic I/O (read x, v, f and write x, v: 15 scalars per vertex
    # and step) over the step time, against the measured copy bandwidth
    ssz_ = 4 if prec == native.FP32FORM else 8
    io_bytes = 15.0 * ssz_ * b.n_total
    hbm_peak, hbm_src = measured_hbm_peak()
    hbm = {"algorithmic_bytes_per_step": io_bytes, "achieved_gbs": io_bytes / (ms_per_step / 1e3) / 1e9,
           "peak_gbs": hbm_peak, "peak_source": hbm_src,
           "frac": io_bytes / (ms_per_step / 1e3) / 1e9 / hbm_peak if hbm_peak else None,
           "note": "the step's algorithmic HBM traffic; per-type constants stay L2-resident, and the per-cell "
                   "workspace traffic of the iteration kernels is not algorithmic (see the kernels' DRAM bytes in "
                   "the ncu summaries)"}
    # the whole step's DRAM traffic and FP32 / FP64 flops from the per-kernel ncu records,
    # over the measured step time: HBM bandwidth and the two pipes' fractions
    recs, recs_how = kernel_records(nv, args.precision)
    pipes = None
    if recs:
        cnt = step_counters(recs, nv, its)
        sec = ms_per_step / 1e3
        hbm["dram_bytes_per_step"] = cnt["dram_bytes"]
        hbm["measured_gbs"] = cnt["dram_bytes"] / sec / 1e9
        hbm["measured_frac"] = hbm["measured_gbs"] / hbm_peak if hbm_peak else None
        hbm["measured_how"] = ("DRAM bytes per cell, cell-solve and cell-iteration of k_begin, k_solve and k_iter "
                               "(ncu, profiles/traffic.json) times the step's cells and iterations, over the "
                               "CUDA-event step time")
        pipes = {"fp32_flops_per_step": cnt["fp32_flops"], "fp64_flops_per_step": cnt["fp64_flops"],
                 "fp32_tflops": cnt["fp32_flops"] / sec / 1e12, "fp64_tflops": cnt["fp64_flops"] / sec / 1e12,
                 "fp32_frac": cnt["fp32_flops"] / sec / 1e12 / fp32_peak if fp32_peak else None,
                 "fp64_frac": cnt["fp64_flops"] / sec / 1e12 / fp64_peak if fp64_peak else None,
                 "peaks": "FP32 and FP64 FMA rates measured live by the probe",
                 "how": "executed FP32 / FP64 add, multiply (1 flop) and fused multiply-add (2 flops) thread "
                        "instructions of every kernel of the step (ncu, profiles/traffic.json: " + recs_how + ")"}
    else:
        hbm["measured_how"] = recs_how

    # end-to-end through the C ABI with host (pinned) buffers
    e2e = None
    if rank == 0 and not args.no_e2e:
        ssz = 4 if prec == native.FP32FORM else 8
        hx = torch.empty((3, b.n_total), dtype=tdt, pin_memory=True)
        hv = torch.empty_like(hx, pin_memory=True)
        hf = torch.empty_like(hx, pin_memory=True)
        hx.copy_(x0.cpu())
        hv.copy_(v0.cpu())
        hf.copy_(f.cpu())
        hit = torch.tensor(b.iters, dtype=torch.int32).pin_memory()
        hres = torch.zeros(b.ncells, dtype=torch.float64).pin_memory()
        hst = torch.zeros(b.ncells, dtype=torch.int32).pin_memory()
        hdn = torch.zeros(b.ncells, dtype=torch.int32).pin_memory() if tol > 0 else None
        nx, nv_, nf, ni, nr, ns = (hx.numpy(), hv.numpy(), hf.numpy(), hit.numpy(), hres.numpy(), hst.numpy())
        nd = hdn.numpy() if hdn is not None else None
        for _ in range(max(1, args.warmup)):
            batch.step_host(nx, nv_, nf, iters=ni, residual=nr, status=ns, stream=stream.cuda_stream,
                            tol=tol, iters_done=nd)
        times = []
        for _ in range(args.steps):
            flush.zero_()                       # L2 flushed between steps, as in the device-timed leg
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            batch.step_host(nx, nv_, nf, iters=ni, residual=nr, status=ns, stream=stream.cuda_stream,
                            tol=tol, iters_done=nd)
            times.append(time.perf_counter() - t0)
        h2d = 3 * 3 * b.n_total * ssz + 4 * b.ncells
        d2h = 2 * 3 * b.n_total * ssz + 12 * b.ncells + (4 * b.ncells if nd is not None else 0)
        e2e = {"value": rbc_eq_per_rank / statistics.mean(times), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "api": "npfem_step_host (pinned host buffers, copies + step + copies, synchronous)",
               "l2": "flushed before each step (untimed)"}

    # the same batch in the plain FP64 form: its throughput and its parity at the FP64 bar,
    # for the FP32-form speed-up at stated accuracy
    fp64 = None
    if rank == 0 and prec == native.FP32FORM and not args.no_fp64:
        fp64 = fp64_pass(args, b, types, iters, tol, coll, sample, ocache, dev, flush, rbc_eq_per_rank)
        if fp64.get("value"):
            fp64["speedup_fp32form_over_fp64"] = value / fp64["value"]

    adjoint = None
    if rank == 0 and not args.no_adjoint:
        adjoint = measure_adjoint(dev)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if prec == native.FP32FORM else "f64", "data": "synthetic",
        "config": {"workload": desc, "cells": b.ncells, "rbc_equivalents_per_step": rbc_eq_per_rank,
                   "precision": args.precision, "l2": "flushed between steps (256 MB write, untimed)",
                   "damping": ({"c_alpha_per_us": DAMPING[0], "c_beta_us": DAMPING[1]} if any(DAMPING) else None),
                   "strain_limits": ({"s_min": STRAIN_LIMITS[0], "s_max": STRAIN_LIMITS[1]}
                                     if any(STRAIN_LIMITS) else None),
                   "launch": "one CUDA graph per step" if graph is not None else "direct npfem_step call",
                   "mode": "split kernels (k_begin, then k_solve + k_iter per iteration and cell type)",
                   "split_shapes": {str(t): list(batch.get_split_launch(t)[0]) for t in sorted(set(int(q) for q in b.type_of_cell))},
                   "groups": {str(t): batch.get_groups(t) for t in sorted(set(int(q) for q in b.type_of_cell))},
                   "autotune": tuned,
                   "collisions": ({"radius_um": coll[0], "delta_um": coll[1], "weight_nN_per_um": coll[2],
                                   "walls": bool(coll[3]),
                                   "detection": "normals, spatial hash, scan, scatter, query kernels inside the step",
                                   "detection_ms_per_step": detect_ms / args.steps}
                                  if coll is not None else None),
                   "parallelism": "cells sharded across ranks, no collective" if world > 1 else "1 GPU"},
        "residual": {"median": float(np.median(resid)), "max": float(np.max(resid)),
                     "definition": "|grad f(x_final)| / |grad f(x_0)| per cell after the step"},
        "residual_mode": ({"tol": tol, "budget": args.budget, "mean_iterations": float(np.mean(its)),
                           "cells_at_budget_last_step": int(np.sum(done.cpu().numpy() >= args.budget)),
                           "unit_rule": "each cell-step at the stated residual counts n/642"}
                          if tol > 0 else {"fixed_iterations": True,
                                           "unit_rule": "each cell-step counts (n/642)*(iterations/5)"}),
        "status_nonzero_cells": int(np.count_nonzero(status)),
        "parity_sample": err,
        "roofline": roofline,
        "hbm": hbm,
        "pipes": pipes,
        "fp32_peak_tflops": fp32_peak,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "fp64_form": fp64,
        "adjoint": adjoint,
        "kernels": kernels,
        "gpu_launches": args.steps * (sum(min(batch.get_groups(t), int(np.sum(b.type_of_cell == t)))
                                          for t in set(int(q) for q in b.type_of_cell)) * (1 + 2 * int(np.max(b.iters)))
                                      + (len(set(int(q) for q in b.type_of_cell)) + 6 if coll is not None else 0)),
        "clocks": clk.summary(),
        "wall_s_timed_region": t_wall,
    }
    return out


def fp64_pass(args, b, types, iters, tol, coll, sample, ocache, dev, flush, units):
    """The workload's batch in the plain FP64 form (FP64 everywhere): parity of its first
    step against the oracle on the sampled cells at the FP64 bar, then `args.fp64_steps`
    CUDA-graph replays timed with events (L2 flushed between them, library default
    shapes)."""
    import torch
    from paper_2011_04332_b300 import native
    batch = native.Batch(types, b.type_of_cell, native.FP64)
    if coll is not None:
        batch.set_collisions(coll[0], coll[1], coll[2], box=_box(b, coll))
    x0 = torch.tensor(b.x, dtype=torch.float64, device=dev)
    v0 = torch.tensor(b.v, dtype=torch.float64, device=dev)
    f = torch.tensor(b.f, dtype=torch.float64, device=dev)
    it = iters.clone()
    res = torch.zeros(b.ncells, dtype=torch.float64, device=dev)
    st = torch.zeros(b.ncells, dtype=torch.int32, device=dev)
    done = torch.zeros(b.ncells, dtype=torch.int32, device=dev) if tol > 0 else None
    x, v = x0.clone(), v0.clone()
    batch.step(x, v, f, iters=it, residual=res, status=st, tol=tol, iters_done=done)
    torch.cuda.synchronize()
    err = None
    if not args.no_check:
        err = oracle_parity(b, x0, v0, f, x, sample, 1e-10, tol, coll,
                            done.cpu().numpy() if done is not None else None, ocache)
    stream = torch.cuda.current_stream(dev)
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            batch.step(x, v, f, iters=it, residual=res, status=st, tol=tol, iters_done=done)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.fp64_steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    mean = statistics.mean(ms)
    del graph
    return {"value": units / (mean / 1e3), "unit": UNIT, "ms_per_step": mean, "steps": args.fp64_steps,
            "warmup": 2, "parity_sample": err,
            "residual": {"median": float(res.median()), "max": float(res.max())},
            "how": "same batch and inputs in the plain FP64 form (FP64 local work, two-loop and solves), "
                   "one CUDA graph per step, L2 flushed between steps, library default launch shapes"}


def measure_adjoint(dev, nsteps: int = 200, ckpt_every: int = 20, ncells: int = 256):
    """Adjoint throughput on the calibration workload: ncells placed 642-vertex RBCs,
    FP64, loss = squared distance of axial/transverse diameters to seeded targets after
    an nsteps rollout with checkpoints every ckpt_every steps (forward + backward)."""
    import torch
    from paper_2011_04332_b300 import autograd as AG
    from paper_2011_04332_b300 import inputs as I
    b = I.homogeneous_rbc_batch(ncells=ncells, seed=1003)
    targets = torch.tensor(np.random.default_rng(1003).uniform(6, 12, size=(ncells, 2)), device=dev)
    cal = AG.Calibration(b.types[0].mesh, b.types[0].material.as_tuple(), b.dt, ncells)
    x0 = torch.tensor(b.x, device=dev)
    v0 = torch.tensor(b.v, device=dev)
    f = torch.tensor(b.f, device=dev, requires_grad=True)
    iters = torch.tensor(b.iters, device=dev)
    loss, w = cal.loss(x0, v0, f, targets, iters, 2, 1)       # warm-up (allocates the workspace)
    loss.backward()
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    f.grad = None
    e[0].record()
    loss, w = cal.loss(x0, v0, f, targets, iters, nsteps, ckpt_every)
    e[1].record()
    loss.backward()
    e[2].record()
    torch.cuda.synchronize()
    t_fwd, t_bwd = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
    return {"workload": f"calibration: {ncells} RBC (642 vertices) FP64, {nsteps}-step rollout, "
                        f"checkpoints every {ckpt_every} steps, diameter loss",
            "adjoint_cell_steps_per_s": ncells * nsteps / (t_bwd / 1e3),
            "ms_per_adjoint_step": t_bwd / nsteps,
            "ms_per_forward_step": t_fwd / nsteps,
            "backward_includes": "npfem_rollout_adjoint: a checkpointed forward rollout, segment recomputation "
                                 "and the step adjoints (the library recomputes the forward from (x0, v0))",
            "loss": float(loss.detach()), "grad_w": [float(g) for g in w.grad[0].tolist()],
            "implicit": measure_adjoint_implicit(dev, b)}


def measure_adjoint_implicit(dev, b, reps: int = 5, fwd_tol: float = 1e-10, budget: int = 100,
                             cg_tol: float = 1e-10):
    """Implicit-function adjoint on the same cells: one call = the forward step run to
    |g|/|g0| < fwd_tol (fused kernel, budget iterations) + CG on the Hessian per cell."""
    import torch
    from paper_2011_04332_b300 import native
    t = b.types[0]
    ct = native.CellType(t.mesh.verts, t.mesh.tris, t.material.as_tuple(), b.dt)
    batch = native.Batch([ct], b.type_of_cell, native.FP64)
    batch.set_mode(False)
    x, v, f = (torch.tensor(a, device=dev) for a in (b.x, b.v, b.f))
    gxn = torch.tensor(np.random.default_rng(1004).standard_normal(b.x.shape), device=dev)
    gx, gv, gf = (torch.zeros_like(x) for _ in range(3))
    gw = torch.zeros((b.ncells, 4), dtype=torch.float64, device=dev)
    st = torch.zeros(b.ncells, dtype=torch.int32, device=dev)
    it = torch.full((b.ncells,), budget, dtype=torch.int32, device=dev)
    dn = torch.zeros(b.ncells, dtype=torch.int32, device=dev)

    def call():
        batch.step_adjoint_implicit(x, v, f, gxn, None, gx, gv, gf, gw, iters=it, tol=fwd_tol, cg_tol=cg_tol,
                                    cg_max_iters=500, status=st)
    call()
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    xs, vs = x.clone(), v.clone()
    e0.record()
    batch.step(xs, vs, f, iters=it, tol=fwd_tol, iters_done=dn)
    e1.record()
    for _ in range(reps):
        call()
    e2.record()
    torch.cuda.synchronize()
    ms_fwd, ms_call = e0.elapsed_time(e1), e1.elapsed_time(e2) / reps
    return {"workload": f"{b.ncells} RBC (642 vertices) FP64, forward to |g|/|g0| < {fwd_tol:g} "
                        f"(budget {budget}), CG to {cg_tol:g}",
            "adjoint_cell_steps_per_s": b.ncells / (ms_call / 1e3), "ms_per_call": ms_call,
            "ms_forward_alone": ms_fwd, "forward_iterations_mean": float(dn.double().mean()),
            "cg_status_bits_set": int(((st & 16) != 0).sum())}


# Sources that define what the step kernels execute: the device code and the host
# packer that lays out the factor they stream (launch plumbing is excluded).
# The sources a step's kernels are compiled from; the adjoint kernels (adjoint.cuh) take
# no part in a step, so an edit there leaves the captured solve traffic valid.
KERNEL_SOURCES = ("npfem_internal.h", "step_kernel.cuh", "split_kernels.cuh", "iter_cta.cuh", "host_setup.cpp",
                  "contact_kernels.cuh")


def kernel_source_hash() -> str:
    """SHA-256 over the kernel sources (detects a changed kernel)."""
    import hashlib
    d = os.path.join(ROOT, "paper_2011_04332_b300", "csrc")
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        h.update(name.encode())
        h.update(open(os.path.join(d, name), "rb").read())
    return h.hexdigest()


def measured_traffic(sizes, precision: str):
    """DRAM bytes per cell-solve of the solve kernel for each cell size (vertices) from
    profiles/traffic.json, only if captured for the current kernel sources, this
    precision and every size; else None and the reason."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(p))
    except (OSError, ValueError):
        return None, "no traffic record"
    if rec.get("kernel_src_sha256") != kernel_source_hash():
        return None, "kernel changed since the ncu capture"
    out, how = {}, []
    for n in sorted(set(int(s) for s in sizes)):
        ent = rec.get("entries", {}).get(f"n{n}/{precision}")
        if not ent:
            return None, f"no capture for {n}-vertex cells"
        out[n] = ent["dram_bytes_per_cell_solve"]
        how.append(f"{n} vertices: {ent['how']}")
    return out, "; ".join(how)


def kernel_records(sizes, precision: str):
    """Per-kernel DRAM bytes and FP32 / FP64 flops of the step's kernels for each cell
    size, from profiles/traffic.json ("kernels": ncu counters of every launch of one step
    of a homogeneous batch, divided by the cells (k_begin), cell-solves (k_solve) or
    cell-iterations (k_iter) of the launch), only if captured for the current kernel
    sources, this precision and every size; else None and the reason."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(p))
    except (OSError, ValueError):
        return None, "no traffic record"
    if rec.get("kernel_src_sha256") != kernel_source_hash():
        return None, "kernel changed since the ncu capture"
    out = {}
    for n in sorted(set(int(s) for s in sizes)):
        ent = rec.get("kernels", {}).get(f"n{n}/{precision}")
        if not ent:
            return None, f"no kernel record for {n}-vertex cells"
        out[n] = ent
    return out, rec.get("kernels_how", "")


def step_counters(recs, nv, its):
    """DRAM bytes, FP32 flops and FP64 flops of one step from the per-unit kernel records:
    per cell k_begin once, k_solve and k_iter once per iteration."""
    tot = {"dram_bytes": 0.0, "fp32_flops": 0.0, "fp64_flops": 0.0}
    for n, i in zip(nv, its):
        r = recs[int(n)]
        for key in tot:
            tot[key] += r["k_begin"][key] + i * (r["k_solve"][key] + r["k_iter"][key])
    return tot


def measured_hbm_peak():
    """Copy bandwidth measured on the B300s (MEASURED_PEAKS.json), else the
    profiling recipe's fallback figure."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured (copy)"
    except (OSError, ValueError, KeyError):
        return 6400.0, "fallback"


def probe_peaks():
    import ctypes
    from paper_2011_04332_b300 import build as B
    try:
        lib = ctypes.CDLL(B.build_probe())
        fn = lib.npfem_probe_fma_peaks
        fn.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        a, c = ctypes.c_double(), ctypes.c_double()
        if fn(ctypes.byref(a), ctypes.byref(c)) == 0:
            return a.value, c.value
    except OSError:
        pass
    return None, None


def run_reference(args, rank, world):
    if rank != 0:
        return None
    b, desc = make_workload(args.workload, 0)
    b, desc = residual_mode(b, desc, args.tol, args.budget)
    per_step = []
    cores = args.cpu_workers
    sdesc = ""
    for _ in range(args.warmup + args.steps):
        nsample = args.ref_sample if args.workload not in COLLISIONS else min(args.ref_sample, 4)
        v, cores, sdesc = oracle_baseline(b, nsample, args.cpu_workers, args.tol, COLLISIONS.get(args.workload))
        per_step.append(v)
    vals = per_step[args.warmup:]
    value = float(statistics.mean(vals))
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "precision": "fp64 (CPU oracle)",
                       "damping": ({"c_alpha_per_us": DAMPING[0], "c_beta_us": DAMPING[1]} if any(DAMPING) else None),
                       "strain_limits": ({"s_min": STRAIN_LIMITS[0], "s_max": STRAIN_LIMITS[1]}
                                         if any(STRAIN_LIMITS) else None)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sdesc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="hetero10k", choices=["homog4096", "hetero10k", "stress20k", "homog1776", "homog2562", "plt1776",
                                                            "pack4096", "packbox4096", "small"])
    ap.add_argument("--precision", default="fp32form", choices=["fp32form", "fp64"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=128)
    ap.add_argument("--ref-sample", type=int, default=32)
    ap.add_argument("--cpu-workers", type=int, default=max(1, os.cpu_count() or 1))
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-check", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain-FP64 pass of an FP32-form run")
    ap.add_argument("--fp64-steps", type=int, default=5, help="timed steps of the plain-FP64 pass")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--tune", action="store_true",
                    help="autotune the split launch shapes and groups first (default: the library's per-size-class "
                         "defaults, which measured as fast as the tuner's choice on the 10^4-cell batch)")
    ap.add_argument("--no-tune", action="store_true", help="(the default; kept for older command lines)")
    ap.add_argument("--tol", type=float, default=0.0,
                    help="converged-residual mode: per-cell stop at |g|/|g0| < tol (0: fixed iteration counts)")
    ap.add_argument("--budget", type=int, default=16, help="with --tol: iteration budget per cell")
    ap.add_argument("--damping", default="0,0",
                    help="Rayleigh damping c_alpha,c_beta (1/us, us) for every cell type")
    ap.add_argument("--strain-limits", default="0,0",
                    help="strain limits s_min,s_max for every cell type (0,0: the rotations)")
    ap.add_argument("--groups", type=int, default=0,
                    help="without --tune: phase-offset chains per cell type (0: library default)")
    args = ap.parse_args()
    global DAMPING, STRAIN_LIMITS
    DAMPING = tuple(float(q) for q in args.damping.split(","))
    STRAIN_LIMITS = tuple(float(q) for q in args.strain_limits.split(","))
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    out = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
