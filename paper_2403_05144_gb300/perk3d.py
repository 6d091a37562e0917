"""Python layer of the 3D path (include/perk3d.h): P-ERK steps of an octree DGSEM.

``Perk3DSolver`` marshals arguments to libperk's 3D entry points; PyTorch
supplies device memory and the stream, every step runs in the library's sm_103a
kernels.  There is no CPU path: without the built library or a CUDA device the
calls raise.
"""

from __future__ import annotations

import ctypes as C
from typing import Sequence

import numpy as np

from . import _lib
from ._lib import PerkError

__all__ = ["Perk3DSolver", "mesh_faces3", "amr_plan_cells"]


def _check(lib, ctx, status: int):
    if status != _lib.PERK_OK:
        raise PerkError(status, lib.perk3d_last_error(ctx).decode())


def mesh_faces3(cells):
    """(interfaces [n_if, 4], mortars [n_mort, 6]) the library builds for an octree leaf list
    (host only): interface (left, right, dir, 0); mortar (large, s0, s1, s2, s3,
    dir | large_side << 2) with the small cells by quadrant q1 + 2 q2."""
    lib = _lib.load()
    arr = np.ascontiguousarray(np.asarray(cells, dtype=np.int32).reshape(-1, 4))
    ni, nm = C.c_int64(), C.c_int64()
    cp = arr.ctypes.data_as(C.POINTER(C.c_int32))
    _check(lib, None, lib.perk3d_mesh_faces(len(arr), cp, C.byref(ni), None, 0, C.byref(nm), None, 0))
    ifs = np.zeros((ni.value, 4), dtype=np.int32)
    ms = np.zeros((nm.value, 6), dtype=np.int32)
    _check(lib, None, lib.perk3d_mesh_faces(len(arr), cp, C.byref(ni), ifs.ctypes.data_as(C.POINTER(C.c_int32)),
                                            ni.value, C.byref(nm), ms.ctypes.data_as(C.POINTER(C.c_int32)), nm.value))
    return ifs, ms


def amr_plan_cells(cells, desired):
    """(balanced levels [n], new leaves [m, 4], transfer records [m, 9]) of one AMR cycle with the
    given desired levels (host only; the plan perk3d_adapt_plan makes)."""
    lib = _lib.load()
    arr = np.ascontiguousarray(np.asarray(cells, dtype=np.int32).reshape(-1, 4))
    d = np.ascontiguousarray(np.asarray(desired, dtype=np.int32).reshape(-1))
    if len(d) != len(arr):
        raise ValueError("desired needs one level per cell")
    levels = np.zeros(len(arr), dtype=np.int32)
    m = C.c_int64()
    P = C.POINTER(C.c_int32)
    _check(lib, None, lib.perk3d_amr_plan_cells(len(arr), arr.ctypes.data_as(P), d.ctypes.data_as(P),
                                                levels.ctypes.data_as(P), C.byref(m), None, None, 0))
    new = np.zeros((m.value, 4), dtype=np.int32)
    mp = np.zeros((m.value, 9), dtype=np.int32)
    _check(lib, None, lib.perk3d_amr_plan_cells(len(arr), arr.ctypes.data_as(P), d.ctypes.data_as(P),
                                                levels.ctypes.data_as(P), C.byref(m), new.ctypes.data_as(P),
                                                mp.ctypes.data_as(P), m.value))
    return levels, new, mp


class Perk3DSolver:
    """One 3D libperk context: octree mesh, level partition, coefficient table, stage buffers."""

    def __init__(self, N: int = 2, gamma: float = 1.4, surface_flux: str = "hlle", use_graph: bool = True,
                 equations: str = "euler", mu: float = 0.0, prandtl: float = 0.72):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("Perk3DSolver needs a CUDA device")
        self.torch = torch
        self.lib = _lib.load()
        eq = {"euler": 0, "navier_stokes": 1}[equations]
        prob = _lib.Perk3DProblem(int(N), float(gamma), _lib.SURFACE[surface_flux], 1 if use_graph else 0, eq,
                                  float(mu), float(prandtl))
        h = C.c_void_p()
        torch.cuda.init()
        _check(self.lib, None, self.lib.perk3d_create(C.byref(prob), C.byref(h)))
        self.ctx = h
        self.N = int(N)
        self.n = self.N + 1
        self.gamma = gamma
        self.n_elem = 0
        self.S = 0

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx:
            self.lib.perk3d_destroy(ctx)
            self.ctx = None

    def _call(self, fn, *args):
        s = self.torch.cuda.current_stream().cuda_stream
        _check(self.lib, self.ctx, self.lib.perk3d_set_stream(self.ctx, C.c_void_p(s)))
        _check(self.lib, self.ctx, fn(self.ctx, *args))

    # ------------------------------------------------------------------ setup
    def upload_mesh(self, cells, x0: float, length: float):
        arr = np.ascontiguousarray(np.asarray(cells, dtype=np.int32).reshape(-1, 4))
        self._call(self.lib.perk3d_mesh_upload, C.c_int64(len(arr)), arr.ctypes.data_as(C.POINTER(C.c_int32)),
                   C.c_double(x0), C.c_double(length))
        self.n_elem = len(arr)
        self.x0, self.length = float(x0), float(length)
        self.cells = arr

    def set_tableau(self, order: int, E: Sequence[int], c, a):
        E = [int(e) for e in E]
        c = np.ascontiguousarray(c, dtype=np.float64)
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(len(E), len(c))
        Ea = (C.c_int32 * len(E))(*E)
        self._call(self.lib.perk3d_set_tableau, int(order), len(c), len(E), Ea,
                   c.ctypes.data_as(C.POINTER(C.c_double)), a.ctypes.data_as(C.POINTER(C.c_double)))
        self.S = len(c)
        self.E = E

    def set_perk2_disk(self, E: Sequence[int], S: int | None = None):
        from . import perk2_disk_tableau

        c, a = perk2_disk_tableau(E, S)
        self.set_tableau(2, E, c, a)
        return c, a

    def set_perk3_disk(self, E: Sequence[int], S: int | None = None):
        from . import perk3_disk_tableau

        c, a = perk3_disk_tableau(E, S)
        self.set_tableau(3, E, c, a)
        return c, a

    def info(self) -> dict:
        inf = _lib.PerkMeshInfo()
        _check(self.lib, self.ctx, self.lib.perk3d_mesh_query(self.ctx, C.byref(inf)))
        S = inf.S
        return {"n_elem": inf.n_elem, "n_interfaces": inf.n_interfaces, "n_mortars": inf.n_mortars,
                "level_min": inf.level_min, "level_max": inf.level_max, "S": S,
                "dof_stage_updates": inf.dof_stage_updates, "active_elements": list(inf.active_elements[:S]),
                "active_interfaces": list(inf.active_interfaces[:S]), "active_mortars": list(inf.active_mortars[:S]),
                "index_bytes": inf.index_bytes}

    def counters(self) -> dict:
        c = _lib.PerkCounters()
        _check(self.lib, self.ctx, self.lib.perk3d_get_counters(self.ctx, C.byref(c)))
        return {f: getattr(c, f) for f, _ in c._fields_}

    # -------------------------------------------------------------- compute
    def _shape(self):
        return (self.n_elem, 5, self.n, self.n, self.n)

    def _state(self, t):
        torch = self.torch
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError("expected a contiguous float64 CUDA tensor")
        if tuple(t.shape) != self._shape():
            raise ValueError(f"expected shape {self._shape()}, got {tuple(t.shape)}")
        return t

    def empty_state(self):
        return self.torch.empty(self._shape(), dtype=self.torch.float64, device="cuda")

    def rhs_full(self, Y, out=None):
        Y = self._state(Y)
        K = self.empty_state() if out is None else self._state(out)
        self._call(self.lib.perk3d_rhs_full, C.c_void_p(Y.data_ptr()), C.c_void_p(K.data_ptr()))
        return K

    def rhs_active(self, stage: int, Y, out=None):
        Y = self._state(Y)
        K = self.torch.zeros_like(Y) if out is None else self._state(out)
        self._call(self.lib.perk3d_rhs_active, int(stage), C.c_void_p(Y.data_ptr()), C.c_void_p(K.data_ptr()))
        return K

    def step(self, U, dt: float):
        U = self._state(U)
        self._call(self.lib.perk3d_step, C.c_void_p(U.data_ptr()), C.c_double(float(dt)))
        return U

    def step_profiled(self, U, dt: float, acc=None):
        U = self._state(U)
        acc = acc if acc is not None else _lib.PerkKernelTimes()
        self._call(self.lib.perk3d_step_profiled, C.c_void_p(U.data_ptr()), C.c_double(dt), C.byref(acc))
        return acc

    def check(self):
        self._call(self.lib.perk3d_check)

    def compute_dt(self, U, cfl: float) -> float:
        U = self._state(U)
        out = C.c_double()
        self._call(self.lib.perk3d_compute_dt, C.c_void_p(U.data_ptr()), C.c_double(cfl), C.byref(out))
        return out.value

    # ------------------------------------------------------------------- AMR
    def amr_indicator(self, U):
        """Per-element enstrophy indicator (max over nodes of rho |curl v|^2 / 2), on the device."""
        U = self._state(U)
        eta = self.torch.empty(self.n_elem, dtype=self.torch.float64, device="cuda")
        self._call(self.lib.perk3d_amr_indicator, C.c_void_p(U.data_ptr()), C.c_void_p(eta.data_ptr()))
        return eta

    def get_cells(self):
        out = np.zeros((self.n_elem, 4), dtype=np.int32)
        self._call(self.lib.perk3d_get_cells, out.ctypes.data_as(C.POINTER(C.c_int32)), C.c_int64(self.n_elem))
        return out

    def adapt(self, U, level_min: int = 0, level_max: int = 19, refine_above: float = float("inf"),
              coarsen_below: float = 0.0, desired=None):
        """One AMR cycle: returns the transferred state on the new mesh (a new tensor; U is left
        as it was).  ``desired`` (levels per cell) replaces the indicator's decisions."""
        U = self._state(U)
        n_new = C.c_int64()
        if desired is not None:
            d = np.ascontiguousarray(desired, dtype=np.int32)
            if d.shape != (self.n_elem,):
                raise ValueError("desired needs one level per cell")
            self._call(self.lib.perk3d_adapt_plan, None, d.ctypes.data_as(C.POINTER(C.c_int32)), None,
                       C.byref(n_new))
        else:
            prm = _lib.Perk3DAmrParams(int(level_min), int(level_max), float(refine_above), float(coarsen_below))
            self._call(self.lib.perk3d_adapt_plan, C.byref(prm), None, C.c_void_p(U.data_ptr()), C.byref(n_new))
        Unew = self.torch.empty((n_new.value, 5, self.n, self.n, self.n), dtype=self.torch.float64, device="cuda")
        self._call(self.lib.perk3d_adapt_commit, C.c_void_p(U.data_ptr()), C.c_void_p(Unew.data_ptr()))
        self.n_elem = n_new.value
        self.cells = self.get_cells()
        return Unew

