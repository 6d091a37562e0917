#!/usr/bin/env python
"""Throughput benchmark of the P-ERK step on one or more GB300s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl perk|reference]
                    [--workload kh|kh_shock|vortex|vortex_large|shear|ensemble|adjoint|spectrum|tgv]

Prints one JSON line (rank 0).  Metric: P-ERK DoF-stage updates per second,
i.e. the active DoF (nodes) summed over the stages of a step, divided by the
step's device time; the same job also reports the wall time to t_end against
the full-RHS S-stage method (every element evaluated at every stage, same S
and dt) on the same GPU, the accuracy of both against a reference solution,
the roofline of the dominant kernel against the measured FP64 rate, the
end-to-end rate through the public API with host buffers, and the CPU oracle
on a bounded sample.  Workloads: kh (default: Kelvin-Helmholtz with dynamic
AMR), kh_shock (the same with HLLE and subcell shock capturing), vortex (static
two-level isentropic vortex, 448 cells), vortex_large (the same
pattern at 114,688 cells, the roofline case), shear (Navier-Stokes shear
layer, third order, dynamic AMR), ensemble (64 KH members in one context),
adjoint (discrete-adjoint gradient over 200 steps), spectrum (spectrum-optimised
stability polynomials against the disk polynomials), tgv (3D Taylor-Green vortex,
Navier-Stokes at Re 1600, on an octree adapted by the enstrophy indicator, levels 4-6,
P-ERK3 {3,4,6}, N = 2).

Multi-GPU: the step does not shard across GPUs here; N ranks run N
independent replicas of the workload (weak scaling, no collective on the
data path).  ``--impl reference`` times the CPU oracle on the same workload,
one stage evaluation per step (rank 0 only).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from perk_inputs import (isentropic_vortex, kelvin_helmholtz, nodal_state, shear_layer, uniform_cells,
                         vortex_two_level_cells)

METRIC = "P-ERK DoF-stage updates/s and wall time to t_end vs full-RK on same GB300"
UNIT = "DoF-stage updates/s"

# Algorithmic FP64 operations of one element-stage of the volume term (Euler, N = 3), counted
# by the oracle's operation counter (oracle/opcount.py; add/mul 1, divide and logarithm 1 each;
# tests/test_oracle_opcount.py checks that this constant is its result): stage state 256, node
# quantities 192 (48 divides, 32 logarithms), the 48 symmetric pair fluxes 1,392 (144 divides),
# flux differencing 640, surface lifting and Jacobian 192.  The roofline's `achieved` is this
# count times the element-stages of the profiled volume launches over their CUDA-event time.
VOL_ALG_FLOPS_PER_ELEM = 2672
# The same counter on the numerical surface flux at one face node (subsonic case) and on one
# mortar's interpolation and L2 projection: the face work of a stage, which the fused stage
# kernel performs beside the volume work (per stage: 4 face nodes per active interface, 8 per
# active mortar, and one mortar's operators per active mortar).
FACE_ALG_FLOPS_PER_NODE = {"hll": 70, "hllc": 69, "ec": 53, "hlle": 93}
MORTAR_ALG_FLOPS = 380
# FP64 issue slots of one element-stage of the volume kernel (flux
# differencing + surface lifting + stage combination) in the library's
# formulation (add, mul, FMA, compare = 1 slot; reciprocal = 4 FMA after the
# approximate seed; table logarithm = 15 slots), reported beside the roofline as
# how busy the kernel keeps the FP64 issue slots:
#   16 nodes x 60   (combination 10, pressure 5, reciprocal 5, primitives 10, two logarithms 30)
# + 48 pairs x 44   (means' branches 9, reciprocal 5, quotients 3, two log-mean series 15, flux 12)
# + 16 nodes x 6 pairs x 4 variables (accumulation) + 128 (lifting, Jacobian)
VOL_SLOTS_PER_ELEM = 16 * 60 + 48 * 44 + 16 * 6 * 4 + 128
# DRAM bytes per element-stage of the same kernel (two elements per block, stage state formed from
# U_n, K_1, K_{i-1}), measured by ncu on the current kernel (dram__bytes_read.sum +
# dram__bytes_write.sum = 8.08 MB for a launch over all 3,904 elements of the KH mesh); the
# algorithmic minimum is the 4 x 512 B read of U_n, K_1, K_{i-1} and the face fluxes (K_i stays in
# L2 within the launch)
VOL_DRAM_BYTES_PER_ELEM = 8.077312e6 / 3904
# DRAM bytes per element-stage of the one-launch stage kernel (face and volume work), measured by
# ncu on the current kernel: the 16 stage launches of one step of the 3,904-cell KH mesh read
# 86.87 MB for 55,936 element-stages (profiles/k_stage_kelvin_helmholtz_amr_3904cells.md)
STAGE_DRAM_BYTES_PER_ELEM = 86.868736e6 / 55936


AMR_KH = dict(level_min=4, level_max=7, refine_above=0.1, coarsen_below=0.02)
AMR_SHEAR = dict(level_min=6, level_max=8, refine_above=0.1, coarsen_below=0.02, indicator="lohner_vx")
SHEAR_CFL = 0.7


def workload(name: str) -> dict:
    if name == "kh":
        # Kelvin-Helmholtz on [-1, 1]^2: base level 4, dynamic AMR up to level 7 every 5 steps
        # (density-gradient indicator), P-ERK2 {4, 6, 10, 16}, HLLC, N = 3, t_end = 3
        return dict(name="kelvin_helmholtz_amr_levels4-7", cells=uniform_cells(4), x0=-1.0, L=2.0,
                    ic=kelvin_helmholtz, E=[4, 6, 10, 16], flux="hllc", cfl=0.7, t_end=3.0, amr=AMR_KH, n_amr=5,
                    init_cycles=3)
    if name == "kh_shock":
        # the Kelvin-Helmholtz run with the paper's spatial scheme of Sec. 7.2.1: HLLE surface flux and
        # subcell shock capturing with the density as indicator variable (alpha_max 0.5)
        return dict(workload("kh"), name="kelvin_helmholtz_amr_levels4-7_hlle_shock_capturing", flux="hlle",
                    shock="density")
    if name == "shear":
        # doubly periodic shear layer on [0, 1]^2 (Sec. 7.1.1 set-up at Mach 0.3, Re 2500, Pr 0.72):
        # Navier-Stokes with BR1, P-ERK3 {4, 8, 16}, HLL, N = 3, base level 6, dynamic AMR between
        # levels 6 and 8 every 20 steps driven by Loehner's indicator of v_x, t_end = 1.2
        return dict(name="shear_layer_navier_stokes_amr_levels6-8", cells=uniform_cells(6), x0=0.0, L=1.0,
                    ic=shear_layer, E=[4, 8, 16], order=3, flux="hll", cfl=SHEAR_CFL, t_end=1.2,
                    equations="navier_stokes", mu=1.0 / 2500.0, prandtl=0.72, amr=AMR_SHEAR, n_amr=20,
                    init_cycles=2)
    if name == "vortex_large":
        # the same two-level pattern scaled up to saturate the GPU: base 256 x 256 with the central
        # 128 x 128 block refined once (114,688 cells, 1.8M DoF), P-ERK2 {4, 8}, HLL
        return dict(name="isentropic_vortex_256x256_center128x128_refined",
                    cells=vortex_two_level_cells(base_level=8, lo=64, hi=192), x0=-10.0, L=20.0,
                    ic=isentropic_vortex, E=[4, 8], flux="hll", cfl=0.5, t_end=20.0, amr=None, n_amr=0,
                    init_cycles=0)
    if name == "vortex":
        # isentropic vortex, 16x16 base with the central 8x8 block refined (static), P-ERK2 {4, 8}, HLL
        return dict(name="isentropic_vortex_16x16_center8x8_refined", cells=vortex_two_level_cells(), x0=-10.0,
                    L=20.0, ic=isentropic_vortex, E=[4, 8], flux="hll", cfl=0.5, t_end=20.0, amr=None, n_amr=0,
                    init_cycles=0)
    raise SystemExit(f"unknown workload {name}")


class Run:
    """One simulation through the library: mesh, P-ERK family, state, AMR every n_amr steps."""

    def __init__(self, torch, wl: dict, E, use_graph: bool = True):
        from paper_2403_05144_gb300 import PerkSolver, perk2_disk_tableau, perk3_disk_tableau, reference_nodes

        self.torch = torch
        self.wl = wl
        self.solver = PerkSolver(surface_flux=wl["flux"], use_graph=use_graph,
                                 equations=wl.get("equations", "euler"), mu=wl.get("mu", 0.0),
                                 prandtl=wl.get("prandtl", 0.72), shock_capturing=wl.get("shock"))
        self.solver.upload_mesh(wl["cells"], wl["x0"], wl["L"])
        if wl.get("order", 2) == 3:
            c, a = perk3_disk_tableau(E)
            self.solver.set_tableau(3, E, c, a)
        elif wl.get("pattern", "classic") != "classic":
            self.solver.set_perk2_pattern(E, wl["pattern"], max(wl["E"]))
        else:
            b_S = wl.get("b_S", 1.0)
            c, a = perk2_disk_tableau(E, max(wl["E"]), b_S)
            self.solver.set_tableau(2, E, c, a)
            if b_S != 1.0:
                self.solver.set_weights(1.0 - b_S, b_S)
        self.x, _ = reference_nodes(3)
        self.U = self._sample()
        for _ in range(wl["init_cycles"]):          # initial adaptation on the initial condition itself
            self.solver.adapt(self.U, **wl["amr"])
            self.U = self._sample()
        self.k = 0
        self.t = 0.0
        self.amr_cycles = 0
        self._refresh()

    def _sample(self):
        return self.torch.from_numpy(nodal_state(self.wl["ic"], self.solver.cells, self.wl["x0"], self.wl["L"],
                                                 self.x)).cuda()

    def _refresh(self):
        self.dt = self.solver.compute_dt(self.U, self.wl["cfl"])
        self.dof = self.solver.info()["dof_stage_updates"]

    def step(self):
        """One step (preceded by an AMR cycle every n_amr steps); returns its DoF-stage updates."""
        if self.wl["amr"] and self.k > 0 and self.k % self.wl["n_amr"] == 0:
            # the new state's step size comes back with the partition's counts (one wait)
            self.U = self.solver.adapt(self.U, cfl=self.wl["cfl"], **self.wl["amr"])
            self.amr_cycles += 1
            self.dt = self.solver.last_dt
            self.dof = self.solver.info()["dof_stage_updates"]
        self.solver.step(self.U, self.dt)
        self.k += 1
        self.t += self.dt
        return self.dof


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def max_over_ranks(vals, world: int, device: str):
    """Element-wise maximum of a list of timings over the ranks (identity for one rank)."""
    if world == 1:
        return [float(v) for v in vals]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def replica_rate(units_per_rank: float, ms_max: float, world: int) -> float:
    """Whole-job rate of N independent replicas: every rank processes the same units, the job
    takes the slowest rank's time."""
    return world * units_per_rank / (ms_max * 1e-3)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def time_steps(torch, run: Run, K: int, flush):
    """Device time (CUDA events on the launching stream) of K steps of ``run``, each
    including its AMR cycle when one falls due; the L2 flush before every step is
    outside the events.  Returns (total ms, DoF-stage updates)."""
    st = torch.cuda.current_stream()
    evs, units = [], 0
    for _ in range(K):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        units += run.step()
        b.record(st)
        evs.append((a, b))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs), units


def run_to_t_end(torch, wl: dict, E, budget_s: float) -> dict:
    """Wall time of a whole run from t = 0 to t_end (or to a rejected step, or the budget)."""
    from paper_2403_05144_gb300 import PerkError

    run = Run(torch, wl, E)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    status = "reached t_end"
    units = 0
    try:
        while run.t < wl["t_end"] - 1e-12:
            units += run.step()
            if run.k % 25 == 0:
                run.solver.check()
                if time.perf_counter() - t0 > budget_s:
                    status = "wall budget exhausted"
                    break
        run.solver.check()
    except PerkError as e:
        status = f"step rejected ({e.status})"
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    return {"status": status, "t": run.t, "steps": run.k, "wall_s": wall, "n_elem_final": run.solver.n_elem,
            "dof_stage_updates": units}


def density_errors(torch, solver, U, exact: np.ndarray, x0: float, L: float) -> dict:
    """(1/|Omega|) ||e_rho||_L1 by the LGL quadrature of every cell, and max |e_rho| over the nodes."""
    from paper_2403_05144_gb300 import reference_nodes
    _, w = reference_nodes(3)
    e = np.abs(U[:, 0].cpu().numpy() - exact[:, 0])
    h = L / 2.0 ** solver.cells[:, 0]
    l1 = float(np.sum((0.5 * h) ** 2 * np.einsum("eji,j,i->e", e, w, w))) / (L * L)
    return {"l1": l1, "linf": float(e.max())}


def equal_error_vortex(torch) -> dict:
    """Density errors at t = 20 (one period of the periodic vortex) against the exact
    translated vortex, for the P-ERK2 {4, 8} family and the standalone 8-stage member at the
    same dt (the accuracy comparison of Sec. 5)."""
    from paper_2403_05144_gb300 import reference_nodes
    wl = workload("vortex")
    x, _ = reference_nodes(3)
    t_end = wl["t_end"]
    out = {}
    for name, E in (("perk", wl["E"]), ("full_rk", [max(wl["E"])])):
        run = Run(torch, wl, E)
        n = math.ceil(t_end / run.dt)
        run.dt = t_end / n
        for _ in range(n):
            run.step()
        run.solver.check()
        exact = nodal_state(lambda X, Y: isentropic_vortex(X, Y, t_end), run.solver.cells, wl["x0"], wl["L"], x)
        out[name] = {**density_errors(torch, run.solver, run.U, exact, wl["x0"], wl["L"]), "steps": n, "dt": run.dt}
    out["ratio_l1"] = out["perk"]["l1"] / out["full_rk"]["l1"]
    out["ratio_linf"] = out["perk"]["linf"] / out["full_rk"]["linf"]
    out["t_end"] = t_end
    out["mesh"] = wl["name"]
    return out


def equal_error_kh(torch, t_end: float = 0.5) -> dict:
    """Density errors at t = 0.5 of the P-ERK2 family (weights b = e_S, the Heun and Ralston
    variants of Sec. 3.1, and the early-shared stage pattern of Sec. 3.2.4) and of the full-RK
    method (same dt) against the full-RK method at dt/4,
    all on the frozen initially adapted KH mesh (the flow is chaotic later, so only this early
    window is compared)."""
    wl = dict(workload("kh"))
    runs = {}
    base = Run(torch, wl, wl["E"])
    cells, U0 = base.solver.cells.copy(), base.U.clone()
    dt0 = base.dt
    frozen = dict(wl, amr=None, cells=cells, init_cycles=0)
    cases = (("perk", wl["E"], 1, 1.0, "classic"), ("perk_heun_weights", wl["E"], 1, 0.5, "classic"),
             ("perk_ralston_weights", wl["E"], 1, 0.75, "classic"),
             ("perk_early_pattern", wl["E"], 1, 1.0, "early"), ("full_rk", [max(wl["E"])], 1, 1.0, "classic"),
             ("reference", [max(wl["E"])], 4, 1.0, "classic"))
    for name, E, div, b_S, pattern in cases:
        run = Run(torch, dict(frozen, b_S=b_S, pattern=pattern), E)
        run.U = U0.clone()
        n = div * math.ceil(t_end / dt0)
        run.dt = t_end / n
        for _ in range(n):
            run.step()
        run.solver.check()
        runs[name] = run
    ref = runs["reference"].U.cpu().numpy()
    out = {k: {**density_errors(torch, runs[k].solver, runs[k].U, ref, wl["x0"], wl["L"]), "dt": runs[k].dt}
           for k in ("perk", "perk_heun_weights", "perk_ralston_weights", "perk_early_pattern", "full_rk")}
    out["ratio_l1"] = out["perk"]["l1"] / out["full_rk"]["l1"]
    out["ratio_linf"] = out["perk"]["linf"] / out["full_rk"]["linf"]
    out["t_end"] = t_end
    out["mesh"] = f"kelvin_helmholtz initially adapted, frozen, {len(cells)} cells"
    out["reference"] = "full-RK S=16 at dt/4"
    return out


def state_l1(torch, solver, U, ref: np.ndarray, L: float, variables=(0,), by_level: bool = False):
    """(1/|Omega|) sum over the given conserved variables of ||U_v - ref_v||_L1 (LGL quadrature);
    with by_level also the contributions of the cells of each refinement level."""
    from paper_2403_05144_gb300 import reference_nodes
    _, w = reference_nodes(3)
    lev = solver.cells[:, 0]
    h = L / 2.0 ** lev
    e = np.abs(U.cpu().numpy()[:, list(variables)] - ref[:, list(variables)])
    per_cell = (0.5 * h) ** 2 * np.einsum("evji,j,i->e", e, w, w) / (L * L)
    total = float(np.sum(per_cell))
    if not by_level:
        return total
    return total, {int(l): float(np.sum(per_cell[lev == l])) for l in sorted(set(lev.tolist()))}


def equal_error_cfl(torch, wl: dict, t_window: float, variables=(0,), cfl0: float | None = None) -> dict:
    """Step sizes at equal temporal error (the comparison of Sec. 5 at matched accuracy).

    On the frozen initially adapted mesh of the workload, from its initial state over
    [0, t_window]: the error of a run at CFL c is measured against the full-RK method (the
    standalone largest member, every element every stage) at a quarter of the step of CFL cfl0.
    The target is the full-RK error at cfl0; the P-ERK family's CFL for that error is found from
    its errors at cfl0 and cfl0/2 (the measured order p: c* = cfl0 (target / e(cfl0))^(1/p)),
    refined once by the local slope, and its error there is measured."""
    cfl0 = wl["cfl"] if cfl0 is None else cfl0
    base = Run(torch, wl, wl["E"])
    cells, U0 = base.solver.cells.copy(), base.U.clone()
    frozen = dict(wl, amr=None, cells=cells, init_cycles=0)
    S = max(wl["E"])

    def run_at(E, cfl, div=1):
        run = Run(torch, frozen, E)
        run.U = U0.clone()
        dt = run.solver.compute_dt(U0, cfl) / div
        n = math.ceil(t_window / dt)
        run.dt = t_window / n
        for _ in range(n):
            run.step()
        run.solver.check()
        return run, n

    ref_run, _ = run_at([S], cfl0, 4)
    ref = ref_run.U.cpu().numpy()

    def err(E, cfl, by_level=False):
        run, n = run_at(E, cfl)
        r = state_l1(torch, run.solver, run.U, ref, wl["L"], variables, by_level)
        return (r[0], n, r[1]) if by_level else (r, n)

    e_full, n_full, lev_full = err([S], cfl0, True)
    e0, n0, lev_perk = err(wl["E"], cfl0, True)
    e1, _ = err(wl["E"], 0.5 * cfl0)
    p = math.log(e0 / e1) / math.log(2.0)
    c1 = cfl0 * (e_full / e0) ** (1.0 / p)
    ec1, _ = err(wl["E"], c1)
    p_loc = math.log(e0 / ec1) / math.log(cfl0 / c1) if abs(c1 - cfl0) > 1e-3 * cfl0 else p
    c2 = c1 * (e_full / ec1) ** (1.0 / p_loc)
    ec2, n2 = err(wl["E"], c2)
    return {"window": [0.0, t_window], "mesh": f"{wl['name']}: initially adapted, frozen, {len(cells)} cells",
            "error": "L1 of conserved variables %s against full-RK (S=%d) at a quarter of the CFL-%g step"
                     % (list(variables), S, cfl0),
            "full_rk": {"cfl": cfl0, "error": e_full, "steps": n_full, "error_by_level": lev_full},
            "perk_same_cfl": {"cfl": cfl0, "error": e0, "steps": n0, "ratio_to_full_rk": e0 / e_full,
                              "error_by_level": lev_perk,
                              "member_E_by_level": dict(zip(sorted(lev_perk), sorted(wl["E"])[-len(lev_perk):]))},
            "perk_half_cfl_error": e1, "perk_measured_order": p,
            "perk_equal_error": {"cfl": c2, "error": ec2, "steps": n2, "ratio_to_full_rk": ec2 / e_full}}


def cell_means(U: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Cell averages [n, 4] of a nodal DGSEM state by the LGL quadrature."""
    return 0.25 * np.einsum("evji,j,i->ev", U, w, w)


def l1_against_fine(cells, means: np.ndarray, ref_grid: np.ndarray, ref_level: int) -> float:
    """L1 difference (as a fraction of the domain's area) between the cell averages `means` of the
    leaves `cells` (level, ix, iy) and the averages over the same squares of `ref_grid`, the cell
    averages of the uniform level-ref_level mesh indexed [iy, ix]."""
    err = 0.0
    for (l, ix, iy), m in zip(np.asarray(cells).tolist(), means):
        k = 1 << (ref_level - l)
        err += abs(m - ref_grid[iy * k:(iy + 1) * k, ix * k:(ix + 1) * k].mean()) / (1 << (2 * l))
    return err


def total_error_kh(torch, t_window: float = 0.5, ref_level: int = 8) -> dict:
    """Total (spatial + temporal) density error of the P-ERK family and of full-RK at the
    workload's CFL on the frozen initially adapted KH mesh at t_window, against full-RK on the
    uniformly refined level-ref_level mesh from the same initial state (cell averages of the
    reference aggregated onto the coarse cells; L1 over the domain)."""
    from paper_2403_05144_gb300 import reference_nodes
    wl = workload("kh")
    _, w = reference_nodes(3)
    base = Run(torch, wl, wl["E"])
    cells, U0 = base.solver.cells.copy(), base.U.clone()
    frozen = dict(wl, amr=None, cells=cells, init_cycles=0)
    S = max(wl["E"])

    def run(wl_, E, U_init):
        r = Run(torch, wl_, E)
        if U_init is not None:
            r.U = U_init.clone()
        n = math.ceil(t_window / r.solver.compute_dt(r.U, wl_["cfl"]))
        r.dt = t_window / n
        for _ in range(n):
            r.step()
        r.solver.check()
        return r, n

    fine = dict(wl, amr=None, cells=uniform_cells(ref_level), init_cycles=0)
    ref_run, n_ref = run(fine, [S], None)
    ref_means = cell_means(ref_run.U.cpu().numpy(), w)[:, 0]
    side = 1 << ref_level
    ref_grid = np.zeros((side, side))
    for (l, ix, iy), m in zip(ref_run.solver.cells.tolist(), ref_means):
        ref_grid[iy, ix] = m
    out = {"reference": f"full-RK S={S} on the uniform level-{ref_level} mesh ({side * side} cells), "
                        f"{n_ref} steps", "window": [0.0, t_window]}
    for name, E in (("perk", wl["E"]), ("full_rk", [S])):
        r, n = run(frozen, E, U0)
        means = cell_means(r.U.cpu().numpy(), w)[:, 0]
        err = l1_against_fine(r.solver.cells, means, ref_grid, ref_level)
        out[name] = {"l1_cell_average_density_error": err, "steps": n, "cfl": wl["cfl"]}
    out["ratio_perk_over_full_rk"] = out["perk"]["l1_cell_average_density_error"] / \
        out["full_rk"]["l1_cell_average_density_error"]
    return out


def oracle_problem(wl: dict, cells):
    """The oracle's mesh, P-ERK family, member of each cell and RHS for a workload."""
    from oracle.br1 import NavierStokesDGSEM
    from oracle.dgsem import DGSEM
    from oracle.perk import element_methods, perk2_family, perk3_family
    from oracle.treemesh import TreeMesh

    mesh = TreeMesh(cells, wl["x0"], wl["L"])
    fam = (perk3_family if wl.get("order", 2) == 3 else perk2_family)(wl["E"])
    meth = element_methods(mesh.cells[:, 0], fam.R)
    if wl.get("equations", "euler") == "navier_stokes":
        dg = NavierStokesDGSEM(mesh, 3, wl["flux"], mu=wl["mu"], prandtl=wl["prandtl"])
    elif wl.get("shock"):
        from oracle.shock import ShockCapturingDGSEM
        dg = ShockCapturingDGSEM(mesh, 3, wl["flux"], variable=wl["shock"])
    else:
        dg = DGSEM(mesh, 3, wl["flux"])
    return mesh, fam, meth, dg


def oracle_stage_sample(wl: dict, cells, U: np.ndarray, n_stages: int = 0, budget_s: float = 10.0):
    """Times the oracle's partitioned RHS I^(act(i)) F(U) for stages i = 0, 1, ... (cycling over
    the S stages): n_stages evaluations, or as many as fit in budget_s (at least one).
    Returns (DoF-stage updates, seconds, evaluations, S)."""
    mesh, fam, meth, dg = oracle_problem(wl, cells)
    act = [np.array([fam.active(int(r), i) for r in meth]) for i in range(fam.S)]
    units, k = 0, 0
    t0 = time.perf_counter()
    while True:
        dg.rhs_masked(U, act[k % fam.S])
        units += 16 * int(act[k % fam.S].sum())
        k += 1
        sec = time.perf_counter() - t0
        if (n_stages and k >= n_stages) or (not n_stages and sec >= budget_s):
            break
    return units, sec, k, fam.S


def host_cpu() -> dict:
    """The host's logical core count and CPU model (lscpu, else /proc/cpuinfo)."""
    import platform
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        try:
            for line in open("/proc/cpuinfo"):
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "model": model, "machine": platform.machine()}


def _oracle_worker(job):
    """One host process timing the oracle's partitioned stage evaluations (cpu_baseline)."""
    wl_name, cells, U, budget_s = job
    units, sec, k, _ = oracle_stage_sample(workload(wl_name), cells, U, budget_s=budget_s)
    return units, sec, k


def cpu_baseline(wl_name: str, wl: dict, cells, U0: np.ndarray, budget_s: float = 10.0) -> dict:
    """The oracle as it stands, on a bounded sample of the same workload: partitioned stage
    evaluations of the workload's current mesh for about ten seconds, in one host process (one
    thread), then in one process per host core at once (spawned, each single-threaded)."""
    import multiprocessing as mp
    cells = [tuple(int(v) for v in c) for c in cells]
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_keep:
        os.environ[k] = "1"                      # inherited by the spawned workers
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(1) as pool:
            units, sec, k = pool.map(_oracle_worker, [(wl_name, cells, U0, budget_s)])[0]
        n = os.cpu_count() or 1
        with ctx.Pool(n) as pool:
            res = pool.map(_oracle_worker, [(wl_name, cells, U0, budget_s)] * n)
    finally:
        for k_, v in env_keep.items():
            if v is None:
                os.environ.pop(k_, None)
            else:
                os.environ[k_] = v
    all_units = sum(r[0] for r in res)
    all_sec = max(r[1] for r in res)
    S = max(wl["E"])
    return {"value": all_units / all_sec, "unit": UNIT, "cores": n, "kind": "oracle", "host": host_cpu(),
            "sample": f"{n} processes (one per host core, each single-threaded) evaluating the oracle's partitioned "
                      f"stages (stages 0.. of S={S}, cycling) of the workload's current mesh ({len(cells)} cells) "
                      f"for about {budget_s:.0f} s each: {sum(r[2] for r in res)} evaluations",
            "single_core": {"value": units / sec, "unit": UNIT, "cores": 1,
                            "sample": f"{k} partitioned stage evaluations in one single-threaded process, "
                                      f"{sec:.1f} s"}}


_REF = {}


def _ref_init(wl_name: str, cells, U: np.ndarray) -> None:
    """Reference-arm worker: the oracle's problem for the workload's mesh, built once."""
    mesh, fam, meth, dg = oracle_problem(workload(wl_name), cells)
    _REF.update(dg=dg, U=U, S=fam.S, act=[np.array([fam.active(int(r), i) for r in meth]) for i in range(fam.S)])


def _ref_stage(k: int) -> int:
    """Reference-arm worker: the oracle's partitioned RHS of stage k % S; its DoF-stage updates."""
    act = _REF["act"][k % _REF["S"]]
    _REF["dg"].rhs_masked(_REF["U"], act)
    return 16 * int(act.sum())


def run_reference(args) -> None:
    rank, _, world = dist_info()
    if rank != 0:
        return
    from oracle.amr import desired_levels, indicator, new_cells
    from oracle.lgl import lgl_nodes_weights
    from oracle.treemesh import TreeMesh

    if args.workload not in ("kh", "kh_shock", "vortex", "vortex_large", "shear"):
        raise SystemExit("--impl reference times the oracle on the kh, kh_shock, vortex, vortex_large or shear "
                         "workload")
    wl = workload(args.workload)
    x, _ = lgl_nodes_weights(3)
    cells = wl["cells"]
    amr = dict(wl["amr"] or {})
    kind = amr.pop("indicator", "density")
    for _ in range(wl["init_cycles"]):          # the same initial adaptation as the library run
        m0 = TreeMesh(cells, wl["x0"], wl["L"])
        U0 = nodal_state(wl["ic"], cells, wl["x0"], wl["L"], x)
        cells = new_cells(m0, desired_levels(m0, indicator(U0, kind=kind), **amr))
    U = nodal_state(wl["ic"], cells, wl["x0"], wl["L"], x)
    # on every host core: one single-threaded process per core, each evaluating one partitioned
    # stage per step (stage k of the S stages at step k), the step timed until all are done
    import multiprocessing as mp
    cells = [tuple(int(v) for v in c) for c in cells]
    n = os.cpu_count() or 1
    S = max(wl["E"])
    env_keep = {k_: os.environ.get(k_) for k_ in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k_ in env_keep:
        os.environ[k_] = "1"                     # inherited by the spawned workers
    try:
        with mp.get_context("spawn").Pool(n, initializer=_ref_init, initargs=(args.workload, cells, U)) as pool:
            for w in range(args.warmup):
                pool.map(_ref_stage, [w] * n, chunksize=1)
            units = 0
            t0 = time.perf_counter()
            for k in range(args.steps):
                units += sum(pool.map(_ref_stage, [k] * n, chunksize=1))
            sec = time.perf_counter() - t0
    finally:
        for k_, v in env_keep.items():
            if v is None:
                os.environ.pop(k_, None)
            else:
                os.environ[k_] = v
    value = units / sec
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": wl["name"], "n_elem": len(cells), "family": wl["E"],
                       "surface_flux": wl["flux"],
                       "step": f"one partitioned stage evaluation of the oracle on the initially adapted mesh in "
                               f"each of {n} processes (one per host core) at once"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": n, "kind": "oracle", "host": host_cpu(),
                             "sample": f"{args.steps} steps of {n} concurrent single-threaded stage evaluations "
                                       f"(stage k of the S={S} stages at step k) of the {len(cells)}-cell initially "
                                       f"adapted mesh"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_perk(args) -> None:
    import torch

    rank, local_rank, world = dist_info()
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2403_05144_gb300 import measure_fp64
    from paper_2403_05144_gb300.build import build

    build()
    wl = workload(args.workload)
    S = max(wl["E"])
    perk = Run(torch, wl, wl["E"])
    full = Run(torch, wl, [S])
    # the launch structure of each method's step, chosen by the library's autotuner on this mesh
    modes = {"perk": perk.solver.autotune_step(perk.U, perk.dt), "full_rk": full.solver.autotune_step(full.U, full.dt)}
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    for _ in range(args.warmup):
        perk.step()
        full.step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    cycles0 = perk.amr_cycles
    with ClockSampler(local_rank) as clk:
        barrier()
        ms, units = time_steps(torch, perk, args.steps, flush)
        timed_cycles = perk.amr_cycles - cycles0
        barrier()
        ms_full, units_full = time_steps(torch, full, args.steps, flush)
        barrier()
    # the same steps without AMR cycles (graph replays only, on the mesh the timed steps ended on):
    # the difference is the cost of the AMR cycles inside the timed region
    ms_no_amr = None
    if wl["amr"] and timed_cycles:
        Ukeep, wl_keep = perk.U.clone(), perk.wl
        perk.wl = dict(wl, amr=None)
        for _ in range(2):
            perk.step()
        ms_no_amr, _ = time_steps(torch, perk, args.steps, flush)
        perk.wl, perk.U = wl_keep, Ukeep
        (ms_no_amr,) = max_over_ranks([ms_no_amr], world, "cuda")
    perk.solver.check()
    full.solver.check()
    ms, ms_full = max_over_ranks([ms, ms_full], world, "cuda")
    value = replica_rate(units, ms, world)
    value_full = replica_rate(units_full, ms_full, world)
    info = perk.solver.info()

    # roofline of the volume kernel: CUDA events around every launch of K profiled steps
    fma_flops, div_s, log_s = measure_fp64()
    Up = perk.U.clone()
    acc = None
    for _ in range(args.steps):
        acc = perk.solver.step_profiled(Up, perk.dt, acc)
    vol_ms, vol_launches = acc.ms[1], acc.launches[1]
    fused = acc.launches[0] == 0            # one launch per stage: the face work is in kind 1 too
    face_nodes = args.steps * sum(4 * a + 8 * b for a, b in zip(info["active_interfaces"], info["active_mortars"]))
    mortars = args.steps * sum(info["active_mortars"])
    alg_flops = VOL_ALG_FLOPS_PER_ELEM * acc.element_stages
    if fused:
        alg_flops += FACE_ALG_FLOPS_PER_NODE[wl["flux"]] * face_nodes + MORTAR_ALG_FLOPS * mortars
    achieved = alg_flops / (vol_ms * 1e-3)
    slot_rate = 2.0 * VOL_SLOTS_PER_ELEM * acc.element_stages / (vol_ms * 1e-3)   # FMA-equivalent slots
    kernel_ms_total = sum(acc.ms[k] for k in range(4))

    # end to end through the public API: the state lives in pinned host memory;
    # every step copies it in, steps (adapting when due) and copies it back
    st = torch.cuda.current_stream()
    Uh = perk.U.cpu().pin_memory()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    h2d = d2h = 0
    units_e2e = 0
    barrier()
    e0.record(st)
    for _ in range(args.steps):
        perk.U = Uh.to("cuda", non_blocking=True)
        h2d += Uh.numel() * 8
        units_e2e += perk.step()
        if perk.U.shape != Uh.shape:
            Uh = torch.empty(perk.U.shape, dtype=torch.float64).pin_memory()
        Uh.copy_(perk.U, non_blocking=True)
        d2h += Uh.numel() * 8
    e1.record(st)
    torch.cuda.synchronize()
    (ms_e2e,) = max_over_ranks([e0.elapsed_time(e1)], world, "cuda")

    # wall time to t_end, P-ERK family against the full-RHS method (same S, same dt rule)
    tend = {"perk": run_to_t_end(torch, wl, wl["E"], args.t_end_budget),
            "full_rk": run_to_t_end(torch, wl, [S], args.t_end_budget)}
    if wl.get("order", 2) == 3:
        # the Shu-Osher scheme (the third-order member with E = S = 3) as a standalone comparator, at
        # the step its disk radius allows relative to the family's largest member, with the AMR
        # interval scaled so that the mesh adapts at about the same physical times
        from paper_2403_05144_gb300 import perk3_disk_alpha
        ratio = perk3_disk_alpha(3)[1] / perk3_disk_alpha(S)[1]
        tend["ssp33"] = run_to_t_end(torch, dict(wl, cfl=wl["cfl"] * ratio,
                                                 n_amr=max(1, int(round(wl["n_amr"] / ratio)))), [3],
                                     args.t_end_budget)
        tend["ssp33"]["cfl"] = wl["cfl"] * ratio
    for k in ("perk", "full_rk", "ssp33"):
        if k in tend:
            tend[k]["sim_time_per_wall_s"] = tend[k]["t"] / tend[k]["wall_s"]
    tend["t_end"] = wl["t_end"]
    if tend["perk"]["status"] == tend["full_rk"]["status"] == "reached t_end":
        # both at the workload's CFL (the same dt rule), not at equal error: see t_end.equal_error
        tend["wall_ratio_full_over_perk_same_cfl"] = tend["full_rk"]["wall_s"] / tend["perk"]["wall_s"]
    equal_error = None
    if args.workload in ("kh", "vortex"):
        equal_error = {"vortex": equal_error_vortex(torch)}
    if args.workload == "kh":
        equal_error["kelvin_helmholtz"] = equal_error_kh(torch)
        equal_error["kelvin_helmholtz_total_error"] = total_error_kh(torch)
    if args.workload in ("kh", "shear"):
        # both methods to t_end at equal temporal error: the family at the CFL where its error on the
        # frozen window equals the full-RK error at the workload's CFL (AMR interval scaled with the
        # step, so that the mesh adapts at about the same physical times)
        ee = equal_error_cfl(torch, wl, 0.5 if args.workload == "kh" else 0.1,
                             variables=(0,) if args.workload == "kh" else (0, 1, 2, 3))
        c_eq = ee["perk_equal_error"]["cfl"]
        wl_eq = dict(wl, cfl=c_eq, n_amr=max(1, int(round(wl["n_amr"] * wl["cfl"] / c_eq))))
        run_eq = run_to_t_end(torch, wl_eq, wl["E"], args.t_end_budget)
        run_eq["sim_time_per_wall_s"] = run_eq["t"] / run_eq["wall_s"]
        ee["t_end"] = {"perk_at_equal_error": {**run_eq, "cfl": c_eq, "n_amr": wl_eq["n_amr"]},
                       "full_rk": {k: tend["full_rk"][k] for k in ("status", "t", "steps", "wall_s")}}
        if run_eq["status"] == tend["full_rk"]["status"] == "reached t_end":
            ee["t_end"]["wall_ratio_full_over_perk_at_equal_error"] = tend["full_rk"]["wall_s"] / run_eq["wall_s"]
        else:   # compare simulated time per wall second when a budget ends a run
            ee["t_end"]["sim_rate_ratio_perk_over_full_at_equal_error"] = (
                run_eq["sim_time_per_wall_s"] / tend["full_rk"]["sim_time_per_wall_s"])
        equal_error = dict(equal_error or {}, **{"equal_error_" + wl["name"]: ee})
        tend["equal_error"] = ee["t_end"]

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["name"], "n_elem": info["n_elem"], "levels": [info["level_min"], info["level_max"]],
                   "family": wl["E"], "stages": S, "surface_flux": wl["flux"], "cfl": wl["cfl"], "dt": perk.dt,
                   "amr": ({**wl["amr"], "every_steps": wl["n_amr"], "in_timed_region": True} if wl["amr"] else None),
                   "dof_stage_updates_per_step": units / args.steps,
                   "amr_cycles_in_timed_region": timed_cycles,
                   "ms_per_step_without_amr": None if ms_no_amr is None else ms_no_amr / args.steps,
                   "amr_ms_per_cycle": (None if ms_no_amr is None
                                        else (ms - ms_no_amr) / timed_cycles),
                   "amr_share_of_step_time": None if ms_no_amr is None else (ms - ms_no_amr) / ms,
                   "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": f"{world} independent replica(s)", "graph": True,
                   "launch_structure_autotuned": dict(modes, meaning="perk_set_stage_fusion mode: 0 two launches "
                                                      "per stage, 1 one per stage, 2 one per step")},
        "full_rk": {"value": value_full, "ms_per_step": ms_full / args.steps,
                    "dof_stage_updates_per_step": units_full / args.steps,
                    "ratio_ms_per_step_full_over_perk": ms_full / ms},
        "t_end": tend,
        "equal_error": equal_error,
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": fma_flops / 1e12, "unit": "TFLOP/s",
                     "frac": achieved / fma_flops,
                     "traffic": ((STAGE_DRAM_BYTES_PER_ELEM if fused else VOL_DRAM_BYTES_PER_ELEM)
                                 * acc.element_stages / max(vol_launches, 1)),
                     "traffic_note": "DRAM bytes per launch: ncu bytes per element-stage x element-stages "
                                     "per launch",
                     "kernel": "k_stage (face fluxes and volume terms of a stage in one launch)" if fused
                               else "k_volume",
                     "launches": vol_launches, "avg_launch_ms": vol_ms / max(vol_launches, 1),
                     "share_of_kernel_time": vol_ms / kernel_ms_total,
                     "peak_source": "FP64 FMA microbenchmark measured live on this GPU (perk_measure_fp64)",
                     "work": {"volume_flops_per_element_stage": VOL_ALG_FLOPS_PER_ELEM,
                              "face_flops_per_face_node": FACE_ALG_FLOPS_PER_NODE[wl["flux"]] if fused else 0,
                              "mortar_operator_flops": MORTAR_ALG_FLOPS if fused else 0,
                              "element_stages": acc.element_stages, "face_node_fluxes": face_nodes if fused else 0,
                              "mortars": mortars if fused else 0, "algorithmic_flops": alg_flops,
                              "source": "oracle operation counter (add/mul 1, divide, square root and logarithm "
                                        "1 each; 48 symmetric pairs; subsonic face fluxes)"},
                     "issue_slot_frac": None if fused else slot_rate / fma_flops,
                     "issue_slot_note": f"{VOL_SLOTS_PER_ELEM} FP64 issue slots per element-stage in the "
                                        "kernel's own formulation, each counted as an FMA (2 flops), "
                                        "over the measured FMA peak: how busy the FP64 issue slots are",
                     "fp64_pipe_active_source": "ncu sm__pipe_fp64_cycles_active in "
                                                "profiles/k_stage_kelvin_helmholtz_amr_3904cells.md",
                     "cuda_fp64_rates": {"div_per_s": div_s, "log_per_s": log_s}},
        "e2e": {"value": replica_rate(units_e2e, ms_e2e, world), "unit": UNIT,
                "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps},
        # per step 2 launches per stage (6 with the four BR1 kernels of Navier-Stokes) + the
        # commit; per AMR cycle: indicator, transfer, partition, two step-size reductions and the
        # step-size store
        "gpu_launches": args.steps * ((6 if wl.get("equations") == "navier_stokes" else 2) * S + 1) + 6 * timed_cycles,
        "clocks": clk.summary(),
    }
    if rank == 0:
        if world == 1:
            line["cpu_baseline"] = cpu_baseline(args.workload, wl, perk.solver.cells, perk.U.cpu().numpy())
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_ensemble(args) -> None:
    """64 Kelvin-Helmholtz members (seeded amplitude U(0.05, 0.15), wavenumber 2 or 4, finest
    level 6 or 7), each on its own adaptively refined mesh, advanced by one context: one
    launch per kernel and P-ERK stage for all members, per-member dt, AMR every 5 steps."""
    import torch

    from paper_2403_05144_gb300 import PerkSolver, reference_nodes
    from paper_2403_05144_gb300.build import build

    build()
    torch.cuda.set_device(0)
    rng = np.random.default_rng(20240308 + 4)
    n = 64
    amps = rng.uniform(0.05, 0.15, n)
    ks = rng.choice([2, 4], n)
    lmaxs = rng.choice([6, 7], n)
    x, _ = reference_nodes(3)
    # initial meshes: three adaptation cycles of every member on its own initial state
    meshes = []
    for m in range(n):
        s = PerkSolver(surface_flux="hllc", use_graph=False)
        s.upload_mesh(uniform_cells(4), -1.0, 2.0)
        amr = dict(AMR_KH, level_max=int(lmaxs[m]))
        for _ in range(3):
            U = torch.from_numpy(nodal_state(kelvin_helmholtz, s.cells, -1.0, 2.0, x, amplitude=float(amps[m]),
                                             wavenumber=int(ks[m]))).cuda()
            s.adapt(U, **amr)
        meshes.append(s.cells.copy())
        del s
    ens = PerkSolver(surface_flux="hllc", use_graph=True)
    ens.upload_ensemble(meshes, -1.0, 2.0)
    ens.set_perk2_disk([4, 6, 10, 16])
    U = torch.from_numpy(np.concatenate([nodal_state(kelvin_helmholtz, c, -1.0, 2.0, x, amplitude=float(a),
                                                     wavenumber=int(k)) for c, a, k in zip(meshes, amps, ks)])).cuda()
    amr = dict(AMR_KH, level_max=7)
    dts = ens.compute_dt_members(U, 0.7)
    dof_member = [16 * len(c) for c in meshes]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    k = 0

    def step():
        nonlocal U, dts, k
        if k > 0 and k % 5 == 0:
            U = ens.adapt(U, **amr)
            dts = ens.compute_dt_members(U, 0.7)
        ens.step(U, dts)
        k += 1
        return ens.info()["dof_stage_updates"]

    epb = ens.autotune(U)          # elements per block of the volume kernel, timed on this mesh
    mode = ens.autotune_step(U, dts)   # launch structure of the step, timed on this mesh
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs, units = [], 0
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            units += step()
            b.record(st)
            evs.append((a, b))
        torch.cuda.synchronize()
    ens.check()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    info = ens.info()
    line = {"metric": METRIC, "value": units / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "kelvin_helmholtz_ensemble_64_members", "members": n,
                       "member_dof_initial_min_max": [min(dof_member), max(dof_member)],
                       "n_elem_total": info["n_elem"], "family": [4, 6, 10, 16], "amr_every_steps": 5,
                       "graph": True, "launch_structure_autotuned": mode,
                       "launch_structure_meaning": "perk_set_stage_fusion mode: 0 two launches per stage, 1 one "
                                                   "per stage, 2 one per step",
                       "volume_elems_per_block_autotuned": epb,
                       "l2": "flushed (256 MB write) before every timed step"},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_adjoint(args) -> None:
    """Discrete adjoint: gradient of the end-time kinetic energy with respect to the initial
    state over 200 P-ERK2 {6, 10, 16} steps of the Kelvin-Helmholtz problem on a frozen
    three-level mesh (the adapted mesh at t = 1, levels 6-8, about 180k DoF), checkpoints every
    20 steps, checked against central differences along 16 seeded directions."""
    import torch

    from paper_2403_05144_gb300 import PerkSolver, perk2_disk_tableau
    from paper_2403_05144_gb300.adjoint import gradient, kinetic_energy
    from paper_2403_05144_gb300.build import build

    build()
    torch.cuda.set_device(0)
    # the Kelvin-Helmholtz run on base level 6 with AMR between levels 6 and 8, to t = 1: the
    # adapted mesh (three levels, about 11k cells) is then frozen
    wl = dict(workload("kh"), cells=uniform_cells(6), amr=dict(AMR_KH, level_min=6, level_max=8), E=[4, 6, 10, 16])
    run = Run(torch, wl, wl["E"])
    while run.t < 1.0:
        run.step()
    run.solver.check()
    cells, U0 = run.solver.cells.copy(), run.U.clone()
    mesh_name = "kelvin_helmholtz_t1_frozen_levels%d-%d" % (cells[:, 0].min(), cells[:, 0].max())
    s = PerkSolver(surface_flux="hllc", use_graph=True)
    s.upload_mesh(cells, -1.0, 2.0)
    c, a = perk2_disk_tableau([6, 10, 16])
    s.set_tableau(2, [6, 10, 16], c, a)
    dt = s.compute_dt(U0, 0.7)
    x, w = lgl_weights_of(s)
    h = torch.tensor(2.0 / 2.0 ** cells[:, 0], dtype=torch.float64, device="cuda")
    J = lambda U: kinetic_energy(U, h, w)
    n_steps = 200
    st = torch.cuda.current_stream()

    def timed(fn, reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    Uw = U0.clone()
    lam = torch.ones_like(U0)
    lam_out = torch.empty_like(U0)
    K = torch.empty((s.S,) + tuple(U0.shape), dtype=U0.dtype, device=U0.device)
    ms_fwd = timed(lambda: s.step(Uw, dt), 20)
    ms_store = timed(lambda: s.step_store(Uw, dt, stages=K), 20)
    ms_rev = timed(lambda: s.step_vjp(U0, dt, lam, out=lam_out, stages=K), 20)
    ms_adj = timed(lambda: s.step_vjp(U0, dt, lam, out=lam_out), 20)
    # one short gradient first: the functional's autograd and reductions initialise on first use
    gradient(s, U0, dt, 2, J, checkpoint_every=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Jv, grad = gradient(s, U0, dt, n_steps, J, checkpoint_every=20)
    torch.cuda.synchronize()
    wall_grad = time.perf_counter() - t0
    t0 = time.perf_counter()
    Uf = U0.clone()
    for _ in range(n_steps):
        s.step(Uf, dt)
    torch.cuda.synchronize()
    wall_fwd = time.perf_counter() - t0

    def J_of(U):
        U = U.clone()
        for _ in range(n_steps):
            s.step(U, dt)
        s.check()
        return float(J(U))

    rng = np.random.default_rng(20240308 + 5)
    errs = []
    for _ in range(16):
        d = torch.from_numpy(rng.normal(size=U0.shape)).cuda() * U0.abs()
        d = d / torch.linalg.vector_norm(d)
        eps = 1e-6 * float(torch.linalg.vector_norm(U0))
        fd = (J_of(U0 + eps * d) - J_of(U0 - eps * d)) / (2 * eps)
        ad = float(torch.sum(grad * d))
        errs.append(abs(fd - ad) / max(abs(fd), 1e-300))
    line = {"metric": "discrete-adjoint gradient over 200 P-ERK steps (checkpoints every 20, stages stored while "
                      "a window is recomputed): wall time relative to the 200 forward steps",
            "value": wall_grad / wall_fwd, "unit": "x forward run", "n_gpus": 1, "steps": n_steps,
            "warmup": 1, "ms_per_step": 1e3 * wall_grad / n_steps, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": mesh_name, "n_elem": len(cells), "dof": 16 * len(cells),
                       "levels": sorted(set(int(v) for v in cells[:, 0])), "family": [6, 10, 16], "dt": dt,
                       "checkpoint_every": 20},
            "gradient_wall_s": wall_grad, "forward_wall_s": wall_fwd,
            "forward_ms_per_step": ms_fwd, "store_ms_per_step": ms_store, "reverse_from_stored_ms_per_step": ms_rev,
            "reverse_recomputing_ms_per_step": ms_adj,
            "reverse_over_forward": ms_rev / ms_fwd, "reverse_recomputing_over_forward": ms_adj / ms_fwd,
            "J": float(Jv), "fd_directions": 16, "fd_max_rel_err": max(errs), "fd_median_rel_err": float(np.median(errs))}
    print(json.dumps(line), flush=True)


def run_spectrum(args) -> None:
    """Spectrum-optimised second-order members (Sec. 4) against the disk polynomials on the
    initially adapted Kelvin-Helmholtz mesh (3,904 cells, levels 4-7), for a smooth seeded state
    without physical instability (background (1, 0.3, -0.2, 1) plus low Fourier modes of
    amplitude 0.05).  Spectrum: the reduced system (uniform level 3, 4,096 unknowns) from the
    Jacobian assembled by the JVP kernels and its eigendecomposition, scaled to the finest cells,
    joined with the Ritz values of 500 Arnoldi steps on the full mesh.  Members {4, 6, 10, 16}
    optimised for it.  Stability by experiment: a step size is stable when a seeded 1e-8 nodal
    perturbation of the state does not grow more than tenfold in 1,000 steps (a growth factor
    per step below 1.0023); the largest stable step of each family is found by bisection."""
    import torch

    from paper_2403_05144_gb300 import PerkError, PerkSolver, perk2_disk_tableau, reference_nodes
    from paper_2403_05144_gb300.build import build
    from paper_2403_05144_gb300.spectrum import (boundary, jacobian_dense, max_stable_dt,
                                                 perk2_family_from_spectrum, ritz_values)
    from perk_inputs import smooth_random_state

    build()
    torch.cuda.set_device(0)
    x, _ = reference_nodes(3)
    wl = workload("kh")
    E = wl["E"]
    times = {}
    cells = Run(torch, wl, E).solver.cells.copy()       # the initially adapted mesh
    lmax = int(cells[:, 0].max())
    red_level = 3
    red = uniform_cells(red_level)
    s = PerkSolver(surface_flux="hllc")
    s.upload_mesh(red, wl["x0"], wl["L"])
    Ur = torch.from_numpy(smooth_random_state(red, wl["x0"], wl["L"], x)).cuda()
    t0 = time.perf_counter()
    J = jacobian_dense(s, Ur)
    torch.cuda.synchronize()
    times["reduced_jacobian_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    ev = np.linalg.eigvals(J)
    times["reduced_eig_s"] = time.perf_counter() - t0
    sf = PerkSolver(surface_flux="hllc")
    sf.upload_mesh(cells, wl["x0"], wl["L"])
    sf.set_perk2_disk(E)
    U0 = torch.from_numpy(smooth_random_state(cells, wl["x0"], wl["L"], x)).cuda()
    t0 = time.perf_counter()
    rv = ritz_values(sf, U0, m=500)
    torch.cuda.synchronize()
    times["arnoldi_500_s"] = time.perf_counter() - t0
    scale = 2.0 ** (lmax - red_level)               # h_reduced / h_finest
    sigma = boundary(np.concatenate([ev * scale, rv]))
    t0 = time.perf_counter()
    c, a_opt, dt_opt, dt_fam_opt = perk2_family_from_spectrum(sigma, E)
    times["optimisation_s"] = time.perf_counter() - t0
    R = len(E)
    dt_disk = []
    for r, e in enumerate(E):
        al = [((e - 1) / e) * math.comb(e, k) / (e - 1) ** k for k in range(e + 1)]
        al[0] += 1.0 / e
        dt_disk.append(max_stable_dt(al, sigma / 2.0 ** (R - 1 - r)))
    dt_fam_disk = min(dt_disk)
    dt_rule = sf.compute_dt(U0, wl["cfl"])
    noise = 1e-8 * torch.from_numpy(np.random.default_rng(20240308 + 6).normal(size=U0.shape)).cuda()

    def stable(cc, aa, dt, n=1000):
        runs = []
        for U in (U0.clone(), U0 + noise):
            sv = PerkSolver(surface_flux="hllc")
            sv.upload_mesh(cells, wl["x0"], wl["L"])
            sv.set_tableau(2, E, cc, aa)
            for _ in range(n):
                sv.step(U, dt)
            try:
                sv.check()
            except PerkError:
                return False
            runs.append(U)
        growth = float((runs[1] - runs[0]).abs().max()) / float(noise.abs().max())
        return bool(np.isfinite(growth) and growth <= 10.0)

    def largest_stable(cc, aa, guess):
        lo, hi = 0.0, guess
        for _ in range(8):                     # grow while stable
            if not stable(cc, aa, hi):
                break
            lo, hi = hi, 2.0 * hi
        for _ in range(20):                    # shrink until stable
            if lo > 0.0:
                break
            hi *= 0.5
            if stable(cc, aa, hi):
                lo, hi = hi, 2.0 * hi
        for _ in range(7):
            mid = 0.5 * (lo + hi)
            lo, hi = (mid, hi) if stable(cc, aa, mid) else (lo, mid)
        return lo

    t0 = time.perf_counter()
    emp_opt = largest_stable(c, a_opt, dt_fam_opt)
    emp_disk = largest_stable(*perk2_disk_tableau(E), dt_fam_disk)
    times["stability_search_s"] = time.perf_counter() - t0
    line = {"metric": "spectrum-optimised P-ERK2 family: largest stable step relative to the disk polynomials",
            "value": emp_opt / emp_disk, "unit": "x disk-family dt", "n_gpus": 1, "steps": 1000,
            "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "kelvin_helmholtz_initially_adapted_mesh_smooth_state", "n_elem": len(cells),
                       "family": E, "reduced_mesh": f"uniform level {red_level} ({len(red)} cells, {J.shape[0]} unknowns)",
                       "arnoldi_steps": 500, "boundary_points": len(sigma),
                       "stable": "a 1e-8 nodal perturbation grows at most 10x in 1000 steps, no rejected step"},
            "predicted": {"dt_member_optimised": list(map(float, dt_opt)), "dt_member_disk": dt_disk,
                          "dt_family_optimised": dt_fam_opt, "dt_family_disk": dt_fam_disk,
                          "ratio": dt_fam_opt / dt_fam_disk},
            "empirical": {"dt_family_optimised": emp_opt, "dt_family_disk": emp_disk,
                          "cfl_family_optimised": wl["cfl"] * emp_opt / dt_rule,
                          "cfl_family_disk": wl["cfl"] * emp_disk / dt_rule},
            "dt_cfl_rule": dt_rule, "spectral_radius_finest": float(np.abs(sigma).max()), "times": times}
    print(json.dumps(line), flush=True)


# FP64 issue slots of one element-stage of the 3D volume kernel at N = 2 (27 nodes, 81 symmetric
# pairs), counted as for the 2D kernel:
#   27 nodes x 64   (combination 15, pressure 6, reciprocal 5, primitives 8, two logarithms 30)
# + 81 pairs x 50   (the 2D pair's 44 plus the third velocity's mean, product and flux component)
# + 27 nodes x 6 partners x 5 variables (accumulation) + 270 (lifting on up to three faces, Jacobian)
VOL3_SLOTS_PER_ELEM = 27 * 64 + 81 * 50 + 27 * 6 * 5 + 270
TGV = dict(name="taylor_green_3d_navier_stokes_re1600_octree_enstrophy_amr_levels4-6_n2_hlle", N=2, flux="hlle",
           E=[3, 4, 6], cfl=0.5, equations="navier_stokes", mu=1.0 / 1600.0, prandtl=0.72,
           base_level=4, amr=dict(level_min=4, level_max=6, refine_above=1.2, coarsen_below=0.3), n_amr=5,
           init_cycles=2, x0=0.0, L=2.0 * math.pi, mach=0.1, t_end=20.0)


def tgv_initial():
    from perk_inputs.octree import nodal_state3, taylor_green, uniform_cells3
    from paper_2403_05144_gb300 import reference_nodes

    cells = uniform_cells3(TGV["base_level"])
    x, _ = reference_nodes(TGV["N"])
    return cells, nodal_state3(taylor_green, cells, TGV["x0"], TGV["L"], x, mach=TGV["mach"])


class Run3:
    """One 3D run: the Taylor-Green state on 16^3 cells adapted by the enstrophy indicator
    (init_cycles cycles), then P-ERK steps with an AMR cycle every n_amr steps (the step size
    recomputed after each), all through the library."""

    def __init__(self, torch, E):
        from paper_2403_05144_gb300.perk3d import Perk3DSolver

        cells, U0 = tgv_initial()
        self.s = Perk3DSolver(N=TGV["N"], surface_flux=TGV["flux"], use_graph=True, equations=TGV["equations"],
                              mu=TGV["mu"], prandtl=TGV["prandtl"])
        self.s.upload_mesh(cells, TGV["x0"], TGV["L"])
        self.s.set_perk3_disk(E)
        self.U = torch.from_numpy(U0).cuda()
        self.k = 0
        self.t = 0.0
        self.cycles = 0
        for _ in range(TGV["init_cycles"]):
            self.adapt()
        self.cycles = 0

    def adapt(self):
        self.U = self.s.adapt(self.U, **TGV["amr"])
        self.dt = self.s.compute_dt(self.U, TGV["cfl"])
        self.units = self.s.info()["dof_stage_updates"]
        self.cycles += 1

    def step(self) -> int:
        if self.k > 0 and self.k % TGV["n_amr"] == 0:
            self.adapt()
        self.s.step(self.U, self.dt)
        self.k += 1
        self.t += self.dt
        return self.units


def tgv_oracle_sample(cells, U, n_stages: int = 0, budget_s: float = 10.0):
    """The 3D oracle's partitioned RHS I^(act(i)) F(U) for stages i = 0, 1, ... (cycling): n_stages
    evaluations or as many as fit in budget_s.  Returns (DoF-stage updates, seconds, evaluations, S)."""
    from oracle.br1_3d import NavierStokesDGSEM3D
    from oracle.octree import OctreeMesh
    from oracle.perk import element_methods, perk3_family

    mesh = OctreeMesh(np.asarray(cells), TGV["x0"], TGV["L"])
    fam = perk3_family(TGV["E"])
    meth = element_methods(mesh.cells[:, 0], fam.R)
    dg = NavierStokesDGSEM3D(mesh, TGV["N"], TGV["flux"], mu=TGV["mu"], prandtl=TGV["prandtl"])
    nodes = (TGV["N"] + 1) ** 3
    act = [np.array([fam.active(int(r), i) for r in meth]) for i in range(fam.S)]
    units, k = 0, 0
    t0 = time.perf_counter()
    while True:
        dg.rhs_masked(U, act[k % fam.S])
        units += nodes * int(act[k % fam.S].sum())
        k += 1
        sec = time.perf_counter() - t0
        if (n_stages and k >= n_stages) or (not n_stages and sec >= budget_s):
            break
    return units, sec, k, fam.S


def run_tgv(args) -> None:
    """3D Taylor-Green vortex (the paper's Sec. 7.1.3: Navier-Stokes at Re 1600, Pr 0.72, Mach 0.1
    initial state of Eq. IC_TaylorGreen): 16^3 cells adapted
    twice by the enstrophy indicator (levels 4-6), N = 2, HLLE, an AMR cycle every five steps
    inside the timed region; P-ERK3 {3, 4, 6} against the standalone six-stage member (full RHS
    every stage, same AMR)."""
    import torch

    rank, local_rank, world = dist_info()
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2403_05144_gb300 import PerkError, measure_fp64
    from paper_2403_05144_gb300.build import build

    build()
    S = max(TGV["E"])
    perk, full = Run3(torch, TGV["E"]), Run3(torch, [S])
    info0 = perk.s.info()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    for _ in range(args.warmup):
        perk.step()
        full.step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def timed(run):
        st = torch.cuda.current_stream()
        evs, units = [], 0
        c0 = run.cycles
        for _ in range(args.steps):
            flush.fill_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            units += run.step()
            b.record(st)
            evs.append((a, b))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs), units, run.cycles - c0

    with ClockSampler(local_rank) as clk:
        barrier()
        ms, units, cycles = timed(perk)
        barrier()
        ms_full, units_full, _ = timed(full)
        barrier()
    perk.s.check()
    full.s.check()
    ms, ms_full = max_over_ranks([ms, ms_full], world, "cuda")
    value = replica_rate(units, ms, world)
    value_full = replica_rate(units_full, ms_full, world)
    info = perk.s.info()

    fma_flops, _, _ = measure_fp64()
    Upr = perk.U.clone()
    acc = None
    for _ in range(args.steps):
        acc = perk.s.step_profiled(Upr, perk.dt, acc)
    vol_ms, vol_launches = acc.ms[1], acc.launches[1]
    achieved = 2.0 * VOL3_SLOTS_PER_ELEM * acc.element_stages / (vol_ms * 1e-3)
    kernel_ms_total = sum(acc.ms[k] for k in range(4))

    # end to end through the public API with the state in pinned host memory (AMR included)
    st = torch.cuda.current_stream()
    Uh = perk.U.cpu().pin_memory()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    h2d = d2h = units_e2e = 0
    barrier()
    e0.record(st)
    for _ in range(args.steps):
        perk.U = Uh.to("cuda", non_blocking=True)
        h2d += Uh.numel() * 8
        units_e2e += perk.step()
        if perk.U.shape != Uh.shape:
            Uh = torch.empty(perk.U.shape, dtype=torch.float64).pin_memory()
        Uh.copy_(perk.U, non_blocking=True)
        d2h += Uh.numel() * 8
    e1.record(st)
    torch.cuda.synchronize()
    (ms_e2e,) = max_over_ranks([e0.elapsed_time(e1)], world, "cuda")

    # simulated time per wall second over a fixed wall budget (t_end = 20 is out of its reach)
    tend = {"t_end": TGV["t_end"]}
    for key, E in (("perk", TGV["E"]), ("full_rk", [S])):
        run = Run3(torch, E)
        torch.cuda.synchronize()
        status = "budget"
        t0 = time.perf_counter()
        try:
            while run.t < TGV["t_end"] - 1e-12 and time.perf_counter() - t0 < args.t_end_budget:
                for _ in range(TGV["n_amr"] * 10):
                    run.step()
                run.s.check()
            if run.t >= TGV["t_end"] - 1e-12:
                status = "reached t_end"
        except PerkError:
            status = "rejected step"
        wall = time.perf_counter() - t0
        tend[key] = {"t": run.t, "steps": run.k, "amr_cycles": run.cycles, "wall_s": wall, "status": status,
                     "sim_time_per_wall_s": run.t / wall, "n_elem_end": run.s.n_elem}
    tend["sim_time_ratio_perk_over_full_rk"] = (tend["perk"]["sim_time_per_wall_s"]
                                               / tend["full_rk"]["sim_time_per_wall_s"])

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": TGV["name"], "n_elem": info["n_elem"], "n_elem_initial": info0["n_elem"],
                   "levels": [info["level_min"], info["level_max"]], "N": TGV["N"], "family": TGV["E"],
                   "stages": S, "surface_flux": TGV["flux"], "cfl": TGV["cfl"], "dt": perk.dt, "mach": TGV["mach"],
                   "equations": TGV["equations"], "reynolds": 1.0 / TGV["mu"], "prandtl": TGV["prandtl"],
                   "amr": {**TGV["amr"], "indicator": "enstrophy", "every_steps": TGV["n_amr"],
                           "in_timed_region": True, "cycles_timed": cycles},
                   "dof_stage_updates_per_step": units / args.steps,
                   "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": f"{world} independent replica(s)", "graph": True},
        "full_rk": {"value": value_full, "ms_per_step": ms_full / args.steps,
                    "dof_stage_updates_per_step": units_full / args.steps,
                    "ratio_ms_per_step_full_over_perk": ms_full / ms},
        "t_end": tend,
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": fma_flops / 1e12, "unit": "TFLOP/s",
                     "frac": achieved / fma_flops, "traffic": None, "kernel": "k3_volume",
                     "launches": vol_launches, "avg_launch_ms": vol_ms / max(vol_launches, 1),
                     "share_of_kernel_time": vol_ms / kernel_ms_total,
                     "kernel_ms_by_kind": {"faces": acc.ms[0], "volume": acc.ms[1], "commit": acc.ms[2],
                                           "viscous_br1": acc.ms[3]},
                     "peak_source": "FP64 FMA microbenchmark measured live on this GPU (perk_measure_fp64)",
                     "work_per_element_stage": {"fp64_slots": VOL3_SLOTS_PER_ELEM, "flops": 2 * VOL3_SLOTS_PER_ELEM}},
        "e2e": {"value": replica_rate(units_e2e, ms_e2e, world), "unit": UNIT,
                "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps},
        # per step 6 launches per stage (faces, volume, the four BR1 kernels) + the commit; per AMR
        # cycle: indicator, transfer, partition, the step-size reset and reduction
        "gpu_launches": args.steps * (6 * S + 1) + 5 * cycles,
        "clocks": clk.summary(),
    }
    if rank == 0:
        if world == 1:
            u, sec, k, SS = tgv_oracle_sample(perk.s.cells, perk.U.cpu().numpy())
            line["cpu_baseline"] = {"value": u / sec, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
                                    "sample": f"{k} partitioned stage evaluations (cycling over S={SS}) of the "
                                              f"{perk.s.n_elem}-cell adapted octree, {sec:.1f} s, numpy float64, "
                                              f"one thread"}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_reference_tgv(args) -> None:
    rank, _, world = dist_info()
    if rank != 0:
        return
    from oracle.amr3d import adapt3
    from oracle.lgl import lgl_nodes_weights
    from oracle.octree import OctreeMesh
    from perk_inputs.octree import nodal_state3, taylor_green, uniform_cells3

    cells = uniform_cells3(TGV["base_level"])
    x, _ = lgl_nodes_weights(TGV["N"])
    U = nodal_state3(taylor_green, cells, TGV["x0"], TGV["L"], x, mach=TGV["mach"])
    mesh = OctreeMesh(np.asarray(cells), TGV["x0"], TGV["L"])
    for _ in range(TGV["init_cycles"]):          # the same initial adaptation as the library run
        mesh, U, _ = adapt3(mesh, U, **TGV["amr"], N=TGV["N"])
    cells = [tuple(c) for c in mesh.cells.tolist()]
    tgv_oracle_sample(cells, U, n_stages=args.warmup)
    units, sec, k, S = tgv_oracle_sample(cells, U, n_stages=args.steps)
    value = units / sec
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": TGV["name"], "n_elem": len(cells), "family": TGV["E"], "surface_flux": TGV["flux"],
                       "step": "one partitioned stage evaluation of the 3D oracle on the initially adapted octree"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
                             "sample": f"{args.steps} stage evaluations (cycling over the S={S} stages) of the "
                                       f"{len(cells)}-cell initially adapted octree"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def lgl_weights_of(solver):
    import torch

    from paper_2403_05144_gb300 import reference_nodes
    x, w = reference_nodes(3)
    return x, torch.tensor(w, dtype=torch.float64, device="cuda")


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="perk", choices=["perk", "reference"])
    p.add_argument("--workload", default="kh",
                   choices=["kh", "kh_shock", "vortex", "vortex_large", "shear", "ensemble", "adjoint", "spectrum",
                            "tgv"])
    p.add_argument("--t-end-budget", type=float, default=60.0, help="wall seconds per run to t_end")
    args = p.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference_tgv(args) if args.workload == "tgv" else run_reference(args)
    elif args.workload == "tgv":
        run_tgv(args)
    elif args.workload == "ensemble":
        run_ensemble(args)
    elif args.workload == "adjoint":
        run_adjoint(args)
    elif args.workload == "spectrum":
        run_spectrum(args)
    else:
        run_perk(args)


if __name__ == "__main__":
    main()
