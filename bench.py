#!/usr/bin/env python3
"""Benchmark of the batched hydro RHS / SSP-RK3 step on GB300.

One step = one full SSP-RK3 step (three RHS evaluations, the CFL dt
reduction, three combines with floors and dual-energy re-synchronisation,
three ghost fills) over the 256^3 binary-star box (32768 subgrids of 8^3
cells, 3 ghost layers, 5 species, outflow edges), in FP64, replayed from the
library's CUDA graph.  Inputs are resident in HBM before the timed region
(the 7.9 GB state is larger than L2, and L2 is flushed by a 256 MiB write
before each timed step as well), each step timed by its own CUDA events on
the launching stream.  The mixed form and the RHS alone are measured the
same way and reported beside the headline; the FP64 and FP32 FMA peaks the
roofline divides by are measured in the same process.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME]
  python bench.py --profile rhs|step|gravity [--workload NAME] [--precision 0|1] [--reps R]

--impl reference times the FP64 CPU oracle (the reference arm) on the host
cores for the same metric.  --profile only runs R launches of one path on the
workload (the RHS or the graph-replayed SSP-RK3 step of one form, after one
autotuning pass unless --no-autotune, or the monopole gravity kernel), for
captures under a profiler; it prints no benchmark line.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "hydro cell-updates/s (FP64 vs mixed) and % of HBM roofline on 1 GB300"
WORKLOADS = {
    # name: (description, generator of the full workload, generator of the oracle's CPU sample)
    "periodic_box_64": ("512 subgrids of 8^3 cells (64^3 periodic box), 3 ghost layers, 5 species (11 fields), "
                        "log-normal density, seed 1002", lambda inp: inp.periodic_box(seed=1002),
                        lambda inp: inp.periodic_box(seed=1002)),
    "mixed_levels": ("4096 subgrids of edge 8/12/16 on 3 levels (dx halving), ghosts given, 5 species, seed 1003",
                     lambda inp: inp.mixed_levels(), lambda inp: inp.mixed_levels(n=96)),
    "binary_star_128": ("4096 subgrids of 8^3 (128^3 outflow box), two n=1.5 polytropes (mass ratio 0.7) in a "
                        "1e-10 atmosphere, Keplerian rotation, 5 species", lambda inp: inp.binary_star(16),
                        lambda inp: inp.binary_star(4)),
    "binary_star_256": ("32768 subgrids of 8^3 (256^3 outflow box), the binary-star law, 5 species",
                        lambda inp: inp.binary_star(32), lambda inp: inp.binary_star(4)),
    "sedov_64": ("512 subgrids of 8^3 (64^3 outflow box), Sedov-Taylor point explosion (E = 1 in the cells within "
                 "2 cells of the centre, rho = 1, p = 1e-5 elsewhere), 1 species",
                 lambda inp: inp.sedov_blast(nsub=8), lambda inp: inp.sedov_blast(nsub=2)),
    "amr_box_64": ("568 subgrids of 8^3 on 2 levels: a periodic 64^3 box of level-0 subgrids whose central 16^3 "
                   "cells are refined into 64 level-1 subgrids; ghost fill across levels and flux correction at "
                   "coarse-fine faces; the periodic_box law, 5 species, seed 1006",
                   lambda inp: inp.amr_box(n_coarse=8), lambda inp: inp.amr_box(n_coarse=4)),
}
# per workload: (edges of its subgrids, species) -- the shape without the data
SHAPES = {
    "periodic_box_64": (lambda: [8] * 512, 5),
    "mixed_levels": (lambda: [(8, 12, 16)[i % 3] for i in range(4096)], 5),
    "binary_star_128": (lambda: [8] * 4096, 5),
    "binary_star_256": (lambda: [8] * 32768, 5),
    "sedov_64": (lambda: [8] * 512, 1),
    "amr_box_64": (lambda: [8] * 568, 5),
}
UNIT = "cell-updates/s"
STEP = ("one step = one SSP-RK3 step (3 RHS + dt + 3 combine/floor + 3 ghost fill), FP64, each timed step from "
        "the initial state")

# ---------------------------------------------------------------------------
# Work and byte counts per cell: the floating-point arithmetic of the
# method's formulas as the oracle writes them (+, -, *, /, sqrt; compares,
# min and max are not counted), every PPM line of a needed cell once, both
# sides' primitives at every face point.
# ---------------------------------------------------------------------------
OPS_PPM = 38          # 3 MC slopes (6 each), 2 interface values (5 each), CW84 constraint terms (10)
OPS_PRIM = 17         # v (3), kinetic energy (7), e_int and its switch (2), p (2), c^2 and sqrt (3)
OPS_KT_FIELD = 8      # two physical fluxes and the KT combination per field
OPS_KT_POINT = 2 + 4  # signal speeds (2) and the pressure terms (4)
OPS_SIMPSON_FIELD = 11
OPS_DIV_FIELD = 6


def rhs_counts(E: int, nf: int):
    """(FP64 ops, algorithmic HBM bytes) per interior cell of an edge-E
    subgrid with nf fields for one RHS evaluation."""
    cells = E ** 3
    ring = 6 * E * E  # cells just outside each face
    line_cells = cells * 13 + ring * 9  # each ring cell needs the 9 lines that cross its face
    faces = 3 * (E + 1) * E * E
    ops = (line_cells * nf * OPS_PPM
           + faces * 9 * (2 * OPS_PRIM + OPS_KT_POINT + nf * OPS_KT_FIELD)
           + faces * nf * OPS_SIMPSON_FIELD
           + cells * nf * OPS_DIV_FIELD)
    B = E + 6
    bytes_ = (B ** 3 + E ** 3) * nf * 8
    return ops / cells, bytes_ / cells


def problem_counts(prob):
    """(FP64 ops, algorithmic bytes) per interior cell of one RHS over a batch."""
    ops = byt = 0.0
    for E in prob.edge:
        o, b = rhs_counts(int(E), prob.nf)
        ops += o * int(E) ** 3
        byt += b * int(E) ** 3
    return ops / prob.n_cells, byt / prob.n_cells


def step_bytes(E: int, nf: int):
    """Algorithmic HBM bytes per interior cell of one RK3 step in the launch
    split used (3 RHS reads of the ghosted state + RHS writes, 3 combines,
    3 ghost fills)."""
    B = E + 6
    cells = E ** 3
    ghosts = B ** 3 - cells
    rhs = 3 * (B ** 3 + cells) * nf * 8
    comb = (3 * cells * nf * 8            # stage 1: read U, L; write W
            + 2 * 4 * cells * nf * 8)     # stages 2, 3: read U0, X, L; write out
    gfill = 3 * 2 * ghosts * nf * 8
    return (rhs + comb + gfill) / cells


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# DRAM bytes (read + write) of one FP64 RHS call per workload: the uniform
# test, the work list and the RHS kernel, from ncu captures of the three
# kernels (dram__bytes_read.sum + dram__bytes_write.sum) as they are now.
# binary_star_128: measured (uniform test 990.9 MB read + 147.0 MB written,
# work list 0.04 MB, RHS kernel 57.6 MB). binary_star_256: the 128^3 capture
# scaled per kind of subgrid -- the uniform test reads every subgrid's whole
# block and writes the RHS of the uniform ones, the RHS kernel reads the block
# of a subgrid left, and each kind grows with its own count (4096 -> 32768
# blocks, 3796 -> 31512 uniform, 300 -> 1256 left).  A workload without an
# entry reports null.
RHS_FP64_TRAFFIC = {"binary_star_128": 1.195e9, "binary_star_256": 9.39e9}

# The 13 PPM lines (canonical directions).
LINES = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1), (0, 1, 1), (0, 1, -1),
         (1, 1, 1), (1, -1, -1), (1, -1, 1), (1, 1, -1)]


def skipped_work(U, prob):
    """What the RHS kernels leave out on the state U (a CUDA tensor in the
    ghosted layout; uniform edge only, else None), as (uniform subgrids,
    PPM line evaluations counted by rhs_counts in the other subgrids, how many
    of those have a 5-cell stencil of one value).
      - A subgrid whose whole ghosted block holds one value per field: every
        face flux is the same, its RHS is zero and a_max follows from the one
        state; the kernels write both without reconstruction or fluxes (the
        8x8 tiles of edge 8 are whole subgrids).
      - Elsewhere the FP64 kernel returns a stencil of one value as its own
        reconstruction without slope arithmetic.
    Counted cells as in rhs_counts: all 13 lines of every interior cell, the
    9 lines with a step across a face for each cell just outside it."""
    import torch
    if len(set(int(e) for e in prob.edge)) != 1:
        return None
    E, n, nf = int(prob.edge[0]), prob.n_sub, prob.nf
    B = E + 6
    stride = int(prob.off[1] - prob.off[0]) if n > 1 else nf * B ** 3
    if any(int(prob.off[s]) != s * stride for s in (0, n - 1)):
        return None
    V = U[: n * stride].view(n, stride)[:, : nf * B ** 3].view(n, nf, B, B, B)
    uniform = torch.ones(n, dtype=torch.bool, device=U.device)
    for f in range(nf):
        X = V[:, f]
        uniform &= (X == X[:, :1, :1, :1]).flatten(1).all(dim=1)
    live = (~uniform)[:, None, None, None]
    R = E + 2  # cells -1 .. E per axis
    r = torch.arange(R, device=U.device)
    inner = (r >= 1) & (r <= E)
    ring = ~inner
    total = nconst = 0
    n_live = int((~uniform).sum().item())
    for d in LINES:
        dx, dy, dz = d
        m = inner[:, None, None] & inner[None, :, None] & inner[None, None, :]
        if dx:
            m = m | (inner[:, None, None] & inner[None, :, None] & ring[None, None, :])
        if dy:
            m = m | (inner[:, None, None] & ring[None, :, None] & inner[None, None, :])
        if dz:
            m = m | (ring[:, None, None] & inner[None, :, None] & inner[None, None, :])
        total += int(m.sum().item()) * n_live * nf
        for f in range(nf):
            X = V[:, f]
            c0 = X[:, 2:2 + R, 2:2 + R, 2:2 + R]
            const = None
            for k in (-2, -1, 1, 2):
                sl = X[:, 2 + k * dz:2 + k * dz + R, 2 + k * dy:2 + k * dy + R, 2 + k * dx:2 + k * dx + R]
                eq = sl == c0
                const = eq if const is None else const & eq
            nconst += int((const & m & live).sum().item())
    return n - n_live, total, nconst


GRAV_RS = 2.0 / 0.34  # same-level interaction radius (cell widths) for the paper's opening angle


def grav_pairs(r_s):
    """Cells j != i of a cell's stencil: integer offsets with |d|^2 <= r_s^2."""
    R = int(math.floor(r_s))
    return sum(1 for dz in range(-R, R + 1) for dy in range(-R, R + 1) for dx in range(-R, R + 1)
               if 0 < dx * dx + dy * dy + dz * dz <= r_s * r_s)


def bound_of(alu_frac, hbm_frac):
    """The roof a kernel is closest to, or issue/latency when it is far below
    both (under half of each)."""
    if max(alu_frac, hbm_frac) < 0.5:
        return "issue/latency"
    return "alu" if alu_frac >= hbm_frac else "hbm"


def make_config(args, world):
    """The benchmark line's config: the workload and its shape (the same for
    both arms)."""
    import numpy as np
    from paper_2210_06439_gb300 import inputs
    edges_fn, ns = SHAPES[args.workload]
    edge = np.array(edges_fn(), np.int32)
    _, state_len = inputs.layout_offsets(edge, 6 + ns)
    state_bytes = 8 * state_len
    return {"workload": f"{args.workload}: {WORKLOADS[args.workload][0]}; {STEP}"
                        + ("; primitive reconstruction" if args.recon else ""), "subgrids": int(edge.size),
            "edges": sorted(set(int(e) for e in edge)), "ghost": 3, "n_species": ns,
            "interior_cells": int(np.sum(edge.astype(np.int64) ** 3)), "parallelism": f"replicas x{world}",
            "l2": (f"inputs larger than L2 ({state_bytes / 1e9:.2f} GB state); " if state_bytes > 129e6 else "")
                  + "flushed (256 MiB write) before each timed step"}


def reduce_max(v: float, world: int, device="cuda") -> float:
    """Max of a per-rank scalar over all ranks (identity on one rank)."""
    if world == 1:
        return float(v)
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def aggregate(cells_per_rank: int, world: int, ms_total_max: float, steps: int):
    """Whole-job throughput: every rank's cells over the slowest rank's time."""
    ms_step = ms_total_max / steps
    return world * cells_per_rank / (ms_step * 1e-3), ms_step


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------
def run_ours(args, rank, world):
    import numpy as np
    import torch
    from paper_2210_06439_gb300 import binding, inputs

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream()
    prob = WORKLOADS[args.workload][1](inputs)
    nf, n_cells = prob.nf, prob.n_cells
    flush = torch.empty(256 * 2 ** 20 // 4, dtype=torch.float32, device="cuda")

    def make(precision):
        H = binding.Hydro.from_problem(prob, precision=precision, recon=args.recon)
        U = torch.from_numpy(prob.U).cuda()
        with torch.cuda.stream(stream):
            H.fill_ghosts(U, stream=stream)
        dU = torch.zeros(H.rhs_len, dtype=torch.float64, device="cuda")
        return H, U, dU

    def timed(fn, k, w, reset=None):
        """Runs fn w times untimed, then k times each between its own events
        (L2 flushed before each, and reset() run before that, outside the
        events, when given).  Returns per-iteration ms."""
        for _ in range(w):
            with torch.cuda.stream(stream):
                if reset is not None:
                    reset()
                fn()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for a, b in evs:
            with torch.cuda.stream(stream):
                if reset is not None:
                    reset()
                flush.fill_(1.0)
                a.record(stream)
                fn()
                b.record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in evs]

    results = {}
    sampler = ClockSampler(dev)
    for prec in (binding.OCT_FP64, binding.OCT_MIXED):
        H, U, dU = make(prec)
        H.autotune(U, stream=stream)
        U0 = U.clone()
        # full RK3 step (graph replay) -- the timed step; every timed step
        # starts from the workload's initial state, restored before the L2
        # flush outside the timed region, so that each measures the same work
        # (the state evolves within a step and the cost of later steps
        # depends on how many came before: reported apart as "evolving")
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        if prec == binding.OCT_FP64:
            sampler.start()
        step_ms = timed(lambda: H.rk_step(U, want_dt=False, stream=stream), args.steps, args.warmup,
                        reset=lambda: U.copy_(U0))
        if prec == binding.OCT_FP64:
            clocks = sampler.stop()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        # K consecutive steps from the initial state, each timed
        U.copy_(U0)
        torch.cuda.synchronize()
        evolve_ms = timed(lambda: H.rk_step(U, want_dt=False, stream=stream), args.steps, 0)
        # the RHS kernel alone (dominant kernel), same stream
        U.copy_(U0)
        rhs_ms = timed(lambda: H.rhs(U, dU, stream=stream), args.steps, args.warmup)
        flags = H.error_flags()
        results[prec] = dict(step_ms=step_ms, rhs_ms=rhs_ms, flags=flags, H=H, U=U, dU=dU, U0=U0,
                             launch=H.launch_info(), evolve_ms=evolve_ms)

    # same-level monopole gravity (a separate solver step, not part of the
    # hydro RK3 step): its kernel alone, on the FP64 handle's state
    grav = None
    if prob.bc in (1, 2):
        H64g, U64g = results[binding.OCT_FP64]["H"], results[binding.OCT_FP64]["U0"]
        E3 = int(prob.edge[0]) ** 3
        phi = torch.empty(prob.n_sub * E3, dtype=torch.float64, device="cuda")
        gacc = torch.empty(3 * prob.n_sub * E3, dtype=torch.float64, device="cuda")
        grav_ms = timed(lambda: H64g.gravity_monopole(U64g, phi, gacc, G=1.0, r_s=GRAV_RS, stream=stream),
                        max(3, min(args.steps, 5)), args.warmup)
        grav = reduce_max(statistics.mean(grav_ms), world)
        del phi, gacc

    # end to end through the host-buffer ABI call (pinned host state)
    H64 = results[binding.OCT_FP64]["H"]
    Uh = torch.from_numpy(prob.U.copy()).pin_memory()
    H64.fill_ghosts(results[binding.OCT_FP64]["U"], stream=stream)
    torch.cuda.synchronize()
    Uh.copy_(results[binding.OCT_FP64]["U"].cpu())
    Uh0 = Uh.clone()  # each timed call starts from the initial state, like the device-timed steps
    H64.rk_steps_host(Uh, 1, stream=stream)
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(max(3, min(args.steps, 5))):
        Uh.copy_(Uh0)
        t0 = time.perf_counter()
        H64.rk_steps_host(Uh, 1, stream=stream)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    del Uh0

    e2e_in, e2e_out = H64.host_copy_bytes()
    # reduce over ranks: max time
    s64 = results[binding.OCT_FP64]
    smx = results[binding.OCT_MIXED]
    tot64 = reduce_max(sum(s64["step_ms"]), world)
    totmx = reduce_max(sum(smx["step_ms"]), world)
    rhs64 = reduce_max(statistics.mean(s64["rhs_ms"]), world)
    rhsmx = reduce_max(statistics.mean(smx["rhs_ms"]), world)
    e2e = reduce_max(statistics.median(e2e_ms), world)
    mixed_err = None
    if args.cpu_baseline and rank == 0 and prob.n_cells <= 2 ** 21:
        mixed_err = mixed_error_table(prob, results, stream)
    # the RHS was timed on U0: the work its kernels skip there
    skip = skipped_work(s64["U0"], prob) if rank == 0 else None
    # measured FMA peaks of this GPU (one launch of >= 200 ms each, as long as
    # the FP64 RHS launch of the largest workloads)
    with torch.cuda.stream(stream):
        f64_peak, f32_peak = binding.pipe_peaks(200.0, stream=stream)
    torch.cuda.synchronize()
    if rank != 0:
        return None
    K = args.steps
    config = make_config(args, world)
    assert config["interior_cells"] == n_cells and config["subgrids"] == prob.n_sub
    value, ms_step = aggregate(n_cells, world, tot64, K)
    ops_cell, bytes_cell = problem_counts(prob)
    ops_eff = ops_mx = ops_cell
    if skip is not None:
        live = 1.0 - skip[0] * int(prob.edge[0]) ** 3 / n_cells  # cells outside uniform subgrids
        ops_mx = ops_cell * live
        ops_eff = ops_mx - skip[2] * OPS_PPM / n_cells
    hbm_peak, hbm_src = _peaks()
    rhs_tflops = ops_eff * n_cells / (rhs64 * 1e-3) / 1e12
    rhs_gbs = bytes_cell * n_cells / (rhs64 * 1e-3) / 1e9
    mx_tflops = ops_mx * n_cells / (rhsmx * 1e-3) / 1e12
    mx_gbs = bytes_cell * n_cells / (rhsmx * 1e-3) / 1e9
    state_bytes = prob.U.nbytes
    out = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded generators of paper_2210_06439_gb300.inputs)",
        "config": config,
        "rhs": {"value": world * n_cells / (rhs64 * 1e-3), "unit": "RHS cell-updates/s", "ms": rhs64},
        # K consecutive steps from the initial state: where the state has
        # regions of one value (the binary star's atmosphere) later steps cost
        # more, as disturbances spread through it
        "evolving": {k: {"steps": K, "ms_per_step": statistics.mean(r["evolve_ms"]), "first_ms": r["evolve_ms"][0],
                         "last_ms": r["evolve_ms"][-1],
                         "value": world * n_cells / (statistics.mean(r["evolve_ms"]) * 1e-3)}
                     for k, r in (("fp64", s64), ("mixed", smx))},
        "mixed": {"value": world * n_cells / (totmx / K * 1e-3), "unit": UNIT, "ms_per_step": totmx / K,
                  "rhs_value": world * n_cells / (rhsmx * 1e-3), "rhs_ms": rhsmx,
                  "speedup_vs_fp64_step": ms_step / (totmx / K), "speedup_vs_fp64_rhs": rhs64 / rhsmx,
                  "rhs_roofline": {"ops_per_cell": ops_mx,
                                   "bound": bound_of(mx_tflops / f32_peak, mx_gbs / hbm_peak),
                                   "achieved": mx_tflops, "peak": f32_peak, "unit": "TFLOP/s",
                                   "frac": mx_tflops / f32_peak, "peak_source": "measured (FFMA loop, this process)",
                                   "hbm_gbs": mx_gbs, "hbm_frac": mx_gbs / hbm_peak}},
        "roofline": {"bound": "alu", "achieved": rhs_tflops, "peak": f64_peak, "unit": "TFLOP/s",
                     "frac": rhs_tflops / f64_peak,
                     # which roof the kernel is nearest on this workload: on the binary
                     # star most subgrids take the uniform-column path, and the rest
                     # runs below both roofs (barriers and memory latency)
                     "limiter": bound_of(rhs_tflops / f64_peak, rhs_gbs / hbm_peak),
                     "traffic": RHS_FP64_TRAFFIC.get(args.workload) if args.recon == 0 else None,
                     "traffic_unit": "bytes per launch (ncu dram read + write)",
                     "kernel": "FP64 RHS call: uniform_subgrid_kernel + live_items_kernel + rhs_kernel<double>",
                     "ops_per_cell": ops_eff, "method_ops_per_cell": ops_cell,
                     "ops_note": "FP64 flops of the method's formulas per interior cell, less the work the kernel "
                                 "leaves out: subgrids whose ghosted block holds one value per field (RHS zero, "
                                 "written directly) and, elsewhere, the PPM lines whose 5-cell stencil holds one "
                                 "value" + (f": {skip[0]} of {prob.n_sub} subgrids uniform, {skip[2]} of {skip[1]} "
                                            "line evaluations in the others constant" if skip else ""),
                     "peak_source": "measured (DFMA loop, this process)",
                     "fp64_peak_tflops": f64_peak, "fp32_peak_tflops": f32_peak,
                     "hbm": {"achieved": rhs_gbs, "peak": hbm_peak, "unit": "GB/s", "frac": rhs_gbs / hbm_peak,
                             "bytes_per_cell": bytes_cell, "peak_source": hbm_src,
                             # each field of a cell read once and written once (no ghosts): the
                             # lower bound of any layout, as a secondary figure
                             "compact_bytes_per_cell": 16 * nf,
                             "compact_achieved": 16 * nf * n_cells / (rhs64 * 1e-3) / 1e9}},
        "e2e": {"value": world * n_cells / (e2e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": e2e_in,
                "d2h_bytes_per_step": e2e_out + 8,
                "how": "oct_hydro_rk_steps_host on pinned host state: H2D copy (on a uniform level the interior "
                       "z-planes of each field block, the ghosts then filled on the device), RK3 step, D2H copy "
                       "of the whole state, per step"},
        # the library's own count of the kernels one step launches (RHS,
        # dt, combines, and ghost fills unless the combines do them)
        "gpu_launches": s64["H"].step_launches() * K,
        "clocks": clocks,
        "error_flags": {"fp64": s64["flags"], "mixed": smx["flags"]},
        "launch": {k: {"tile_mode": r["launch"][0], "ctas_per_sm": r["launch"][1], "work_items": r["launch"][2]}
                   for k, r in (("fp64", s64), ("mixed", smx))},
    }
    if grav is not None:
        pairs = grav_pairs(GRAV_RS)
        gt = 8.0 * pairs * n_cells / (grav * 1e-3) / 1e12
        out["gravity_monopole"] = {
            "ms": grav, "unit": "ms per launch", "r_s": GRAV_RS, "pairs_per_cell": pairs,
            "roofline": {"bound": "alu", "achieved": gt, "peak": f64_peak, "unit": "TFLOP/s", "frac": gt / f64_peak,
                         "work": "4 FP64 FMAs (8 flops) per interacting pair: the potential and three field "
                                 "components from one mass and the stencil's 1/|d|, d/|d|^3"}}
    if mixed_err is not None:
        out["mixed"]["max_rel_err_per_field_vs_oracle"] = mixed_err
    if args.cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload, reps=2)
    return out


# ---------------------------------------------------------------------------
# The oracle (CPU) as the reference arm and the CPU baseline
# ---------------------------------------------------------------------------
def mixed_error_table(prob, results, stream):
    """Per-field max relative error of the mixed-form RHS against the FP64
    oracle on the benchmark's own state (the CPU leg runs the oracle)."""
    import numpy as np
    import oracle
    import torch
    from paper_2210_06439_gb300 import binding
    ref = prob.copy()
    if ref.bc == 3:
        m = ref.meta
        amr = (m["level"], m["origin"], m["n0"], m["periodic"])
        oracle.amr_ghost_fill(int(ref.edge[0]), ref.off, ref.nf, *amr, ref.U)
        d_o, _, F, _ = oracle.rhs_faces(ref.edge, ref.off, ref.dx, ref.nf, ref.U, gamma=ref.gamma)
        oracle.amr_reflux(int(ref.edge[0]), ref.dx, ref.nf, *amr, F, d_o)
    else:
        if ref.bc != 0:
            oracle.ghost_fill(int(ref.edge[0]), ref.off, ref.nf, ref.nbr, ref.U)
        d_o, _, _ = oracle.rhs(ref.edge, ref.off, ref.dx, ref.nf, ref.U, gamma=ref.gamma)
    r = results[binding.OCT_MIXED]
    r["U"].copy_(r["U0"])
    r["H"].rhs(r["U"], r["dU"], stream=stream)
    torch.cuda.synchronize()
    g = r["dU"].cpu().numpy()
    names = ["rho", "s_x", "s_y", "s_z", "E", "tau"] + [f"rho_{i + 1}" for i in range(prob.nf - 6)]
    out = {}
    for f in range(prob.nf):
        idx, o = [], 0
        for E in prob.edge:
            E3 = int(E) ** 3
            idx.append(np.arange(o + f * E3, o + (f + 1) * E3))
            o += prob.nf * E3
        idx = np.concatenate(idx)
        m = np.max(np.abs(d_o[idx]))
        out[names[f]] = float(np.max(np.abs(g[idx] - d_o[idx])) / m) if m > 0 else 0.0
    return out


def _oracle_step_time(workload):
    import oracle
    from paper_2210_06439_gb300 import inputs
    p = WORKLOADS[workload][2](inputs)
    if p.bc == 3:
        m = p.meta
        amr = (m["level"], m["origin"], m["n0"], m["periodic"])
        oracle.amr_ghost_fill(int(p.edge[0]), p.off, p.nf, *amr, p.U)
        t0 = time.perf_counter()
        oracle.rk3_step_amr(p.edge, p.off, p.dx, p.nf, p.U, *amr, gamma=p.gamma, nthreads=0)
        return time.perf_counter() - t0, p.n_cells, p.n_sub
    if p.bc != 0:
        oracle.ghost_fill(int(p.edge[0]), p.off, p.nf, p.nbr, p.U)
    t0 = time.perf_counter()
    dt, fired, st = oracle.rk3_step(p.edge, p.off, p.dx, p.nf, p.U, bc=p.bc, nbr=p.nbr, gamma=p.gamma, nthreads=0)
    t = time.perf_counter() - t0
    return t, p.n_cells, p.n_sub


def cpu_baseline(workload, reps=1):
    import oracle
    ts = []
    for _ in range(reps):
        t, cells, nsub = _oracle_step_time(workload)
        ts.append(t)
    t = min(ts)
    return {"value": cells / t, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"one SSP-RK3 step of {nsub} subgrids ({cells} cells) of the {workload} law, best of {reps}, "
                      "FP64 C oracle (gcc -O2, OpenMP over subgrids)",
            "single_thread": _oracle_rhs_single_thread(workload)}


def _oracle_rhs_single_thread(workload, n_sub=32):
    """The oracle's RHS on one host thread, on the first n_sub subgrids of the
    workload's oracle sample with their ghosts filled (a bounded sample)."""
    import oracle
    from paper_2210_06439_gb300 import inputs
    p = WORKLOADS[workload][2](inputs)
    if p.bc == 3:
        m = p.meta
        oracle.amr_ghost_fill(int(p.edge[0]), p.off, p.nf, m["level"], m["origin"], m["n0"], m["periodic"], p.U)
    elif p.bc != 0:
        oracle.ghost_fill(int(p.edge[0]), p.off, p.nf, p.nbr, p.U)
    k = min(n_sub, p.n_sub)
    cells = int(sum(int(E) ** 3 for E in p.edge[:k]))
    n_threads = oracle.max_threads()
    t0 = time.perf_counter()
    oracle.rhs(p.edge[:k], p.off[:k], p.dx[:k], p.nf, p.U, gamma=p.gamma, nthreads=1)
    t = time.perf_counter() - t0
    oracle.rhs(p.edge[:0], p.off[:0], p.dx[:0], p.nf, p.U, nthreads=n_threads)  # restore the thread count
    return {"value": cells / t, "unit": "RHS cell-updates/s", "cores": 1,
            "sample": f"one RHS of the first {k} subgrids ({cells} cells) of the {workload} law, one thread"}


def run_reference(args):
    import oracle
    oracle.build_oracle()
    for _ in range(args.warmup):
        _oracle_step_time(args.workload)
    ts = []
    cells = nsub = 0
    for _ in range(args.steps):
        t, cells, nsub = _oracle_step_time(args.workload)
        ts.append(t)
    ms = 1e3 * sum(ts) / len(ts)
    value = cells / (ms * 1e-3)
    cb = {"value": value, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
          "sample": f"one SSP-RK3 step of {nsub} subgrids ({cells} cells) of the {args.workload} law per step"}
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generators of paper_2210_06439_gb300.inputs)",
            "config": make_config(args, 1),
            "cpu_baseline": cb, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}


def profile_run(args):
    """args.reps launches of one kernel path on the workload, for a profiler:
    the RHS of one form, a graph-replayed SSP-RK3 step of one form, or the
    monopole gravity kernel (on the FP64 handle)."""
    import torch
    from paper_2210_06439_gb300 import binding, inputs
    prob = WORKLOADS[args.workload][1](inputs)
    H = binding.Hydro.from_problem(prob, precision=args.precision, recon=args.recon)
    U = torch.from_numpy(prob.U).cuda()
    H.fill_ghosts(U)
    if args.autotune and args.profile != "gravity":
        H.autotune(U)
    stream = torch.cuda.Stream()
    if args.profile == "gravity":
        E3 = int(prob.edge[0]) ** 3
        out = (torch.empty(prob.n_sub * E3, dtype=torch.float64, device="cuda"),
               torch.empty(3 * prob.n_sub * E3, dtype=torch.float64, device="cuda"))
    else:
        out = torch.zeros(H.rhs_len, dtype=torch.float64, device="cuda")
    for _ in range(args.reps):
        with torch.cuda.stream(stream):
            if args.profile == "step":
                H.rk_step(U, want_dt=False, stream=stream)
            elif args.profile == "rhs":
                H.rhs(U, out, stream=stream)
            else:
                H.gravity_monopole(U, *out, G=1.0, r_s=GRAV_RS, stream=stream)
    torch.cuda.synchronize()
    flags = H.error_flags()
    # floors may fire inside a step; nothing else may be flagged
    assert flags & ~binding.OCT_FLAG_FLOOR == 0 and (args.profile == "step" or flags == 0), flags
    print("profile", args.profile, "ok:", args.workload, "precision", args.precision, "launch", H.launch_info(),
          "flags", flags)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="binary_star_256", choices=sorted(WORKLOADS))
    ap.add_argument("--recon", type=int, default=0, choices=(0, 1),
                    help="reconstructed variables: 0 the conserved fields (the method's default), 1 primitive")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--profile", choices=("rhs", "step", "gravity"),
                    help="only run --reps launches of the RHS, the graph-replayed RK3 step or the monopole "
                         "gravity kernel (for profiler captures); no benchmark line")
    ap.add_argument("--precision", type=int, default=0, choices=(0, 1), help="form for --profile rhs|step")
    ap.add_argument("--reps", type=int, default=3, help="launches for --profile")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false", help="--profile without autotuning")
    args = ap.parse_args()
    if args.profile:
        import __graft_entry__
        __graft_entry__.build()
        profile_run(args)
        return
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)))
        return
    if world > 1:
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.distributed.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build() if rank == 0 else None
    if world > 1:
        import torch
        torch.distributed.barrier()
    args.cpu_baseline = args.cpu_baseline and rank == 0 and world == 1
    out = run_ours(args, rank, world)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
