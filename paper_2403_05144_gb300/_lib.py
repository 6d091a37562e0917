"""ctypes declarations of libperk's C ABI (include/perk.h).

Argument marshalling only: every computation runs inside libperk.so.  Loading
fails loudly when the library has not been built; there is no fallback.
"""

from __future__ import annotations

import ctypes as C
import os

from .build import LIB

PERK_OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "NONFINITE", 4: "TIMEOUT", 5: "NOT_READY", 6: "OOM"}
SURFACE = {"hll": 0, "hllc": 1, "ec": 2, "hlle": 3}
SHOCK = {None: 0, "density_pressure": 1, "density": 2}


class PerkProblem(C.Structure):
    _fields_ = [("N", C.c_int), ("gamma", C.c_double), ("surface_flux", C.c_int), ("use_graph", C.c_int),
                ("equations", C.c_int), ("mu", C.c_double), ("prandtl", C.c_double), ("shock_capturing", C.c_int),
                ("alpha_max", C.c_double)]


class PerkMeshInfo(C.Structure):
    _fields_ = [("n_elem", C.c_int64), ("n_interfaces", C.c_int64), ("n_mortars", C.c_int64),
                ("level_min", C.c_int32), ("level_max", C.c_int32), ("S", C.c_int32),
                ("dof_stage_updates", C.c_int64), ("active_elements", C.c_int64 * 64),
                ("active_interfaces", C.c_int64 * 64), ("active_mortars", C.c_int64 * 64),
                ("index_bytes", C.c_int64)]


class PerkCounters(C.Structure):
    _fields_ = [("steps", C.c_int64), ("element_stage_evaluations", C.c_int64), ("dof_stage_updates", C.c_int64),
                ("rejected_steps_checked", C.c_int64), ("device_allocations", C.c_int64)]


class PerkAmrParams(C.Structure):
    _fields_ = [("level_min", C.c_int32), ("level_max", C.c_int32), ("refine_above", C.c_double),
                ("coarsen_below", C.c_double), ("indicator", C.c_int32)]


class PerkKernelTimes(C.Structure):
    _fields_ = [("ms", C.c_double * 4), ("launches", C.c_int64 * 4), ("element_stages", C.c_int64)]


# (name, restype, argtypes) for every entry point of include/perk.h
SIGNATURES = [
    ("perk_create", C.c_int, [C.POINTER(PerkProblem), C.POINTER(C.c_void_p)]),
    ("perk_destroy", None, [C.c_void_p]),
    ("perk_last_error", C.c_char_p, [C.c_void_p]),
    ("perk_set_stream", C.c_int, [C.c_void_p, C.c_void_p]),
    ("perk_mesh_upload", C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_int32), C.c_double, C.c_double]),
    ("perk_mesh_faces", C.c_int, [C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                  C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.c_int64]),
    ("perk_mesh_query", C.c_int, [C.c_void_p, C.POINTER(PerkMeshInfo)]),
    ("perk_ensemble_upload", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.c_double,
                                       C.c_double]),
    ("perk_get_members", C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int64]),
    ("perk_step_dts", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    ("perk_compute_dt_members", C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.POINTER(C.c_double)]),
    ("perk_set_tableau", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int32),
                                   C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("perk_perk2_disk_tableau", C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                          C.POINTER(C.c_double)]),
    ("perk_perk2_disk_tableau_weights", C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_int32), C.c_double,
                                                  C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("perk_perk2_member", C.c_int, [C.c_int, C.c_int, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("perk_set_weights", C.c_int, [C.c_void_p, C.c_double, C.c_double]),
    ("perk_set_tableau_pattern", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int32),
                                           C.POINTER(C.c_uint8), C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                           C.POINTER(C.c_double)]),
    ("perk_perk2_pattern_tableau", C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_int32), C.c_int, C.POINTER(C.c_double),
                                             C.POINTER(C.c_uint8), C.POINTER(C.c_int32), C.POINTER(C.c_double)]),
    ("perk_partition", C.c_int, [C.c_void_p]),
    ("perk_perk3_disk_alpha", C.c_int, [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("perk_perk3_member", C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("perk_perk3_disk_tableau", C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                          C.POINTER(C.c_double)]),
    ("perk_reference_nodes", C.c_int, [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("perk_rhs_full", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("perk_rhs_active", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    ("perk_step", C.c_int, [C.c_void_p, C.c_void_p, C.c_double]),
    ("perk_check", C.c_int, [C.c_void_p]),
    ("perk_compute_dt", C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.POINTER(C.c_double)]),
    ("perk_get_counters", C.c_int, [C.c_void_p, C.POINTER(PerkCounters)]),
    ("perk_rhs_jvp", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("perk_rhs_vjp", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("perk_step_vjp", C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]),
    ("perk_step_store", C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]),
    ("perk_step_vjp_stored", C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("perk_autotune_volume", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int32)]),
    ("perk_autotune_step", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
    ("perk_set_volume_blocks", C.c_int, [C.c_void_p, C.c_int32]),
    ("perk_amr_indicator", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    ("perk_adapt_plan", C.c_int, [C.c_void_p, C.POINTER(PerkAmrParams), C.POINTER(C.c_int32), C.c_void_p,
                                  C.POINTER(C.c_int64)]),
    ("perk_adapt_commit", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("perk_adapt_commit_dt", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.POINTER(C.c_double)]),
    ("perk_get_cells", C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int64]),
    ("perk_amr_balance", C.c_int, [C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    ("perk_selftest_math", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    ("perk_step_profiled", C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.POINTER(PerkKernelTimes)]),
    ("perk_measure_fp64", C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("perk_set_stage_fusion", C.c_int, [C.c_void_p, C.c_int]),
    ("perk_workspace_bytes", C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_size_t)]),
    ("perk_bind_workspace", C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    ("perk_compute_dt_noalloc", C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_double, C.c_double,
                                          C.c_void_p, C.POINTER(C.c_double)]),
]


class Perk3DProblem(C.Structure):
    _fields_ = [("N", C.c_int), ("gamma", C.c_double), ("surface_flux", C.c_int), ("use_graph", C.c_int),
                ("equations", C.c_int), ("mu", C.c_double), ("prandtl", C.c_double)]


class Perk3DAmrParams(C.Structure):
    _fields_ = [("level_min", C.c_int32), ("level_max", C.c_int32), ("refine_above", C.c_double),
                ("coarsen_below", C.c_double)]


# the entry points of include/perk3d.h
SIGNATURES_3D = [
    ("perk3d_create", C.c_int, [C.POINTER(Perk3DProblem), C.POINTER(C.c_void_p)]),
    ("perk3d_destroy", None, [C.c_void_p]),
    ("perk3d_last_error", C.c_char_p, [C.c_void_p]),
    ("perk3d_set_stream", C.c_int, [C.c_void_p, C.c_void_p]),
    ("perk3d_mesh_upload", C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_int32), C.c_double, C.c_double]),
    ("perk3d_mesh_faces", C.c_int, [C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                    C.c_int64, C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.c_int64]),
    ("perk3d_mesh_query", C.c_int, [C.c_void_p, C.POINTER(PerkMeshInfo)]),
    ("perk3d_set_tableau", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int32),
                                     C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("perk3d_rhs_full", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("perk3d_rhs_active", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    ("perk3d_step", C.c_int, [C.c_void_p, C.c_void_p, C.c_double]),
    ("perk3d_check", C.c_int, [C.c_void_p]),
    ("perk3d_compute_dt", C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.POINTER(C.c_double)]),
    ("perk3d_step_profiled", C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.POINTER(PerkKernelTimes)]),
    ("perk3d_get_counters", C.c_int, [C.c_void_p, C.POINTER(PerkCounters)]),
    ("perk3d_amr_indicator", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("perk3d_adapt_plan", C.c_int, [C.c_void_p, C.POINTER(Perk3DAmrParams), C.POINTER(C.c_int32), C.c_void_p,
                                    C.POINTER(C.c_int64)]),
    ("perk3d_adapt_commit", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("perk3d_get_cells", C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_int64]),
    ("perk3d_amr_plan_cells", C.c_int, [C.c_int64, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                        C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_int64]),
]
SIGNATURES = SIGNATURES + SIGNATURES_3D

_lib = None


def load(path: str = LIB) -> C.CDLL:
    """Load libperk.so (built by ``__graft_entry__.build()`` or ``paper_2403_05144_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libperk is not built ({path} missing): run __graft_entry__.build() first")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class PerkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libperk {STATUS.get(status, status)}: {msg}")
        self.status = status
