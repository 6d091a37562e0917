#!/usr/bin/env python
"""Throughput benchmark of the P-ERK step on one or more GB300s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl perk|reference] [--workload kh|vortex]

Prints one JSON line (rank 0).  Metric: P-ERK DoF-stage updates per second,
i.e. the active DoF (nodes) summed over the stages of a step, divided by the
step's device time; the same job also reports the wall time to t_end against
the full-RHS S-stage method (every element evaluated at every stage, same S
and dt) on the same GPU, the roofline of the dominant kernel against the
measured FP64 rate, the end-to-end rate through the public API with host
buffers, and the CPU oracle on a bounded sample.

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

from perk_inputs import isentropic_vortex, kelvin_helmholtz, kh_band_cells, nodal_state, vortex_two_level_cells

METRIC = "P-ERK DoF-stage updates/s and wall time to t_end vs full-RK on same GB300"
UNIT = "DoF-stage updates/s"

# FP64 issue slots of one element-stage of the volume kernel (flux
# differencing + surface lifting + stage combination) in the library's
# formulation (add, mul, FMA, compare = 1 slot; reciprocal = 4 FMA after the
# approximate seed; table logarithm = 15 slots):
#   16 nodes x 60   (combination 10, pressure 5, reciprocal 5, primitives 10, two logarithms 30)
# + 48 pairs x 44   (means' branches 9, reciprocal 5, quotients 3, two log-mean series 15, flux 12)
# + 16 nodes x 6 pairs x 4 variables (accumulation) + 128 (lifting, Jacobian)
VOL_SLOTS_PER_ELEM = 16 * 60 + 48 * 44 + 16 * 6 * 4 + 128


def workload(name: str) -> dict:
    if name == "kh":
        # Kelvin-Helmholtz on [-1, 1]^2, levels 4..7 graded towards the shear lines,
        # P-ERK2 {4, 6, 10, 16}, HLLC, N = 3
        return dict(name="kelvin_helmholtz_levels4-7_static_band", cells=kh_band_cells(4, 7, 0.06), x0=-1.0,
                    L=2.0, ic=kelvin_helmholtz, E=[4, 6, 10, 16], flux="hllc", cfl=0.7, t_end=3.0)
    if name == "vortex":
        return dict(name="isentropic_vortex_16x16_center8x8_refined", cells=vortex_two_level_cells(), x0=-10.0,
                    L=20.0, ic=isentropic_vortex, E=[4, 8], flux="hll", cfl=0.5, t_end=20.0)
    raise SystemExit(f"unknown workload {name}")


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


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


def time_steps(torch, solver, U, dt, K, flush):
    """Device time of K steps, L2 flushed (untimed) before each; returns total ms."""
    st = torch.cuda.current_stream()
    total = 0.0
    evs = []
    for _ in range(K):
        flush.fill_(1.0)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(st)
        solver.step(U, dt)
        b.record(st)
        evs.append((a, b))
    torch.cuda.synchronize()
    for a, b in evs:
        total += a.elapsed_time(b)
    return total


def cpu_baseline(wl: dict, U0: np.ndarray, dt: float) -> dict:
    """The oracle as it stands on one dense P-ERK step of the same workload."""
    from oracle.dgsem import DGSEM
    from oracle.perk import element_methods, perk2_family, prkm_step
    from oracle.treemesh import TreeMesh

    mesh = TreeMesh(wl["cells"], wl["x0"], wl["L"])
    fam = perk2_family(wl["E"])
    meth = element_methods(mesh.cells[:, 0], fam.R)
    dg = DGSEM(mesh, 3, wl["flux"])
    t0 = time.perf_counter()
    prkm_step(dg.rhs, U0, dt, fam, meth)
    sec = time.perf_counter() - t0
    units = sum(16 * int(sum(1 for r in meth if fam.active(int(r), i))) for i in range(fam.S))
    return {"value": units / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one dense P-ERK step of the same mesh ({len(wl['cells'])} cells, S={fam.S}), "
                      f"{sec:.1f} s, numpy float64 on one host thread"}


def run_reference(args) -> None:
    rank, _, world = dist_info()
    if rank != 0:
        return
    from oracle.dgsem import DGSEM
    from oracle.lgl import lgl_nodes_weights
    from oracle.perk import element_methods, perk2_family
    from oracle.treemesh import TreeMesh

    wl = workload(args.workload)
    x, _ = lgl_nodes_weights(3)
    U = nodal_state(wl["ic"], wl["cells"], wl["x0"], wl["L"], x)
    mesh = TreeMesh(wl["cells"], wl["x0"], wl["L"])
    fam = perk2_family(wl["E"])
    meth = element_methods(mesh.cells[:, 0], fam.R)
    dg = DGSEM(mesh, 3, wl["flux"])
    act = [16 * int(sum(1 for r in meth if fam.active(int(r), i))) for i in range(fam.S)]
    for w in range(args.warmup):
        dg.rhs(U)
    units = 0
    t0 = time.perf_counter()
    for k in range(args.steps):
        dg.rhs_masked(U, np.array([fam.active(int(r), k % fam.S) for r in meth]))
        units += act[k % fam.S]
    sec = time.perf_counter() - t0
    value = units / sec
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": wl["name"], "n_elem": len(wl["cells"]), "family": wl["E"],
                       "surface_flux": wl["flux"], "step": "one partitioned RHS stage of the dense oracle step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} stage evaluations (cycling over the S={fam.S} stages) "
                                       f"of the {len(wl['cells'])}-cell mesh"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_perk(args) -> None:
    import torch

    rank, local_rank, world = dist_info()
    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2403_05144_gb300 import PerkSolver, measure_fp64, perk2_disk_tableau, reference_nodes
    from paper_2403_05144_gb300.build import build

    build()
    wl = workload(args.workload)
    x, _ = reference_nodes(3)
    U0 = nodal_state(wl["ic"], wl["cells"], wl["x0"], wl["L"], x)
    S = max(wl["E"])

    solver = PerkSolver(surface_flux=wl["flux"], use_graph=True)
    solver.upload_mesh(wl["cells"], wl["x0"], wl["L"])
    solver.set_perk2_disk(wl["E"])
    full = PerkSolver(surface_flux=wl["flux"], use_graph=True)
    full.upload_mesh(wl["cells"], wl["x0"], wl["L"])
    c, a = perk2_disk_tableau([S])
    full.set_tableau(2, [S], c, a)

    Ud = torch.from_numpy(U0).cuda()
    dt = solver.compute_dt(Ud, wl["cfl"])
    info = solver.info()
    finfo = full.info()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2

    U = Ud.clone()
    Uf = Ud.clone()
    for _ in range(args.warmup):
        solver.step(U, dt)
        full.step(Uf, dt)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    with ClockSampler(local_rank) as clk:
        barrier()
        ms = time_steps(torch, solver, U, dt, args.steps, flush)
        barrier()
        ms_full = time_steps(torch, full, Uf, dt, args.steps, flush)
        barrier()
    solver.check()
    full.check()
    if world > 1:
        t = torch.tensor([ms, ms_full], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms, ms_full = float(t[0]), float(t[1])
    dof_step = info["dof_stage_updates"]
    value = world * dof_step * args.steps / (ms * 1e-3)
    value_full = world * finfo["dof_stage_updates"] * args.steps / (ms_full * 1e-3)

    # roofline of the volume kernel: per-launch CUDA events over K profiled steps
    fma_flops, div_s, log_s = measure_fp64()
    slot_rate = fma_flops / 2.0
    slots_per_elem = VOL_SLOTS_PER_ELEM
    Up = Ud.clone()
    acc = None
    for _ in range(args.steps):
        acc = solver.step_profiled(Up, dt, acc)
    vol_ms = acc.ms[1]
    vol_launches = acc.launches[1]
    achieved = 2.0 * slots_per_elem * acc.element_stages / (vol_ms * 1e-3)
    kernel_ms_total = sum(acc.ms[k] for k in range(3))

    # end to end through the public API: pinned host U, H2D + step + D2H every step
    Uh = torch.from_numpy(U0.copy()).pin_memory()
    Ue = torch.empty_like(Ud)
    st = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(st)
    for _ in range(args.steps):
        Ue.copy_(Uh, non_blocking=True)
        solver.step(Ue, dt)
        Uh.copy_(Ue, non_blocking=True)
    e1.record(st)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms_e2e], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_e2e = float(t[0])
    nbytes = int(U0.nbytes)

    steps_to_end = math.ceil(wl["t_end"] / dt)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["name"], "n_elem": info["n_elem"], "levels": [info["level_min"], info["level_max"]],
                   "family": wl["E"], "stages": S, "surface_flux": wl["flux"], "cfl": wl["cfl"], "dt": dt,
                   "dof_stage_updates_per_step": dof_step, "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": f"{world} independent replica(s)", "graph": True},
        "full_rk": {"value": value_full, "ms_per_step": ms_full / args.steps,
                    "dof_stage_updates_per_step": finfo["dof_stage_updates"],
                    "t_end": wl["t_end"], "steps_to_t_end": steps_to_end,
                    "perk_wall_s_to_t_end": steps_to_end * ms / args.steps * 1e-3,
                    "full_rk_wall_s_to_t_end": steps_to_end * ms_full / args.steps * 1e-3,
                    "wall_ratio_full_over_perk": ms_full / ms,
                    "note": "projected from the measured per-step device time at the fixed initial dt"},
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": fma_flops / 1e12, "unit": "TFLOP/s",
                     "frac": achieved / fma_flops, "traffic": None, "kernel": "k_volume",
                     "launches": vol_launches, "avg_launch_ms": vol_ms / max(vol_launches, 1),
                     "share_of_kernel_time": vol_ms / kernel_ms_total,
                     "peak_source": "FP64 FMA microbenchmark measured live on this GPU (perk_measure_fp64)",
                     "work_per_element_stage": {"fp64_slots": VOL_SLOTS_PER_ELEM,
                                                "flops": 2 * VOL_SLOTS_PER_ELEM,
                                                "note": "FMA-equivalent: every FP64 issue slot counted as 2 flops"},
                     "cuda_fp64_rates": {"div_per_s": div_s, "log_per_s": log_s}},
        "e2e": {"value": world * dof_step * args.steps / (ms_e2e * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
        "gpu_launches": args.steps * (2 * S + 1),
        "clocks": clk.summary(),
    }
    if rank == 0:
        line["cpu_baseline"] = cpu_baseline(wl, U0, dt) if world == 1 else None
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="perk", choices=["perk", "reference"])
    p.add_argument("--workload", default="kh", choices=["kh", "vortex"])
    args = p.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_perk(args)


if __name__ == "__main__":
    main()
