"""GB300-native P-ERK multirate time stepping of a quadtree DGSEM (Python layer).

``PerkSolver`` is a thin wrapper over libperk's C ABI (include/perk.h):
PyTorch provides device memory and the stream, every step of the method runs
in the library's sm_103a kernels.  There is no CPU path: without the built
library or a CUDA device the calls raise.
"""

from __future__ import annotations

import ctypes as C
from typing import Sequence

import numpy as np

from . import _lib
from ._lib import PerkError

__all__ = ["PerkSolver", "PerkError", "reference_nodes", "perk2_disk_tableau", "mesh_faces", "measure_fp64"]


def _check(lib, ctx, status: int):
    if status != _lib.PERK_OK:
        msg = lib.perk_last_error(ctx).decode()
        raise PerkError(status, msg)


def reference_nodes(N: int = 3):
    """Gauss-Lobatto nodes and weights the library collocates on."""
    lib = _lib.load()
    x = (C.c_double * (N + 1))()
    w = (C.c_double * (N + 1))()
    _check(lib, None, lib.perk_reference_nodes(N, x, w))
    return np.array(x[:]), np.array(w[:])


def perk2_disk_tableau(E: Sequence[int], S: int | None = None, b_S: float = 1.0):
    """(c[S], a[R, S]) of the second-order family with disk-optimal members E (ascending) and
    weights b_1 = 1 - b_S, b_S (1: the classic b = e_S; 1/2: Heun; 3/4: Ralston)."""
    lib = _lib.load()
    E = [int(e) for e in E]
    S = int(S or max(E))
    R = len(E)
    Ea = (C.c_int32 * R)(*E)
    c = (C.c_double * S)()
    a = (C.c_double * (R * S))()
    if b_S == 1.0:
        _check(lib, None, lib.perk_perk2_disk_tableau(S, R, Ea, c, a))
    else:
        _check(lib, None, lib.perk_perk2_disk_tableau_weights(S, R, Ea, C.c_double(b_S), c, a))
    return np.array(c[:]), np.array(a[:]).reshape(R, S)


PATTERNS = {"classic": 0, "alternating": 1, "early": 2}


def perk2_pattern_tableau(E: Sequence[int], pattern: str, S: int | None = None):
    """(c[S], eval[R, S], src[R, S], a[R, S]) of the disk-polynomial family with a stage pattern
    (classic, alternating or early)."""
    lib = _lib.load()
    E = [int(e) for e in E]
    S = int(S or max(E))
    R = len(E)
    Ea = (C.c_int32 * R)(*E)
    c = (C.c_double * S)()
    ev = (C.c_uint8 * (R * S))()
    src = (C.c_int32 * (R * S))()
    a = (C.c_double * (R * S))()
    _check(lib, None, lib.perk_perk2_pattern_tableau(S, R, Ea, PATTERNS[pattern], c, ev, src, a))
    return (np.array(c[:]), np.array(ev[:], dtype=np.uint8).reshape(R, S),
            np.array(src[:], dtype=np.int32).reshape(R, S), np.array(a[:]).reshape(R, S))


def perk2_member(S: int, E: int, alpha, b_S: float = 1.0) -> np.ndarray:
    """a[S] (one row of a tableau) of the second-order member with E evaluations whose stability
    polynomial has the monomial coefficients alpha[0..E] (alpha[0..2] = 1, 1, 1/2)."""
    lib = _lib.load()
    al = np.ascontiguousarray(alpha, dtype=np.float64)
    if al.shape != (E + 1,):
        raise ValueError(f"alpha must have E + 1 = {E + 1} coefficients")
    a = (C.c_double * S)()
    _check(lib, None, lib.perk_perk2_member(int(S), int(E), C.c_double(b_S),
                                            al.ctypes.data_as(C.POINTER(C.c_double)), a))
    return np.array(a[:])


def perk3_disk_alpha(E: int):
    """(alpha[0..E], r) of the library's third-order disk polynomial."""
    lib = _lib.load()
    al = (C.c_double * (E + 1))()
    r = C.c_double()
    _check(lib, None, lib.perk_perk3_disk_alpha(E, al, C.byref(r)))
    return np.array(al[:]), r.value


def perk3_member(S: int, E: int, alpha):
    lib = _lib.load()
    al = np.ascontiguousarray(alpha, dtype=np.float64)
    out = (C.c_double * S)()
    _check(lib, None, lib.perk_perk3_member(S, E, al.ctypes.data_as(C.POINTER(C.c_double)), out))
    return np.array(out[:])


def perk3_disk_tableau(E: Sequence[int], S: int | None = None):
    """(c[S], a[R, S]) of the library's third-order family with members E (ascending)."""
    lib = _lib.load()
    E = [int(e) for e in E]
    S = int(S or max(E))
    R = len(E)
    Ea = (C.c_int32 * R)(*E)
    c = (C.c_double * S)()
    a = (C.c_double * (R * S))()
    _check(lib, None, lib.perk_perk3_disk_tableau(S, R, Ea, c, a))
    return np.array(c[:]), np.array(a[:]).reshape(R, S)


def mesh_faces(cells):
    """(interfaces [n_if, 4], mortars [n_mort, 4]) the library builds for a leaf list (host only)."""
    lib = _lib.load()
    arr = np.ascontiguousarray(np.asarray(cells, dtype=np.int32).reshape(-1, 3))
    ni, nm = C.c_int64(), C.c_int64()
    cp = arr.ctypes.data_as(C.POINTER(C.c_int32))
    _check(lib, None, lib.perk_mesh_faces(len(arr), cp, C.byref(ni), None, 0, C.byref(nm), None, 0))
    ifs = np.zeros((ni.value, 4), dtype=np.int32)
    ms = np.zeros((nm.value, 4), dtype=np.int32)
    _check(lib, None, lib.perk_mesh_faces(len(arr), cp, C.byref(ni), ifs.ctypes.data_as(C.POINTER(C.c_int32)),
                                          ni.value, C.byref(nm), ms.ctypes.data_as(C.POINTER(C.c_int32)), nm.value))
    return ifs, ms


def amr_balance(cells, desired):
    """Balanced levels of one AMR cycle for desired levels (host only; what perk_adapt_plan applies)."""
    lib = _lib.load()
    arr = np.ascontiguousarray(np.asarray(cells, dtype=np.int32).reshape(-1, 3))
    d = np.ascontiguousarray(np.asarray(desired, dtype=np.int32).reshape(-1))
    if len(d) != len(arr):
        raise ValueError("desired needs one level per cell")
    out = np.zeros(len(arr), dtype=np.int32)
    P = C.POINTER(C.c_int32)
    _check(lib, None, lib.perk_amr_balance(len(arr), arr.ctypes.data_as(P), d.ctypes.data_as(P),
                                           out.ctypes.data_as(P)))
    return out


def measure_fp64():
    """Measured FP64 rates of the current device: (FMA flop/s, divisions/s, logarithms/s)."""
    lib = _lib.load()
    f, d, l = C.c_double(), C.c_double(), C.c_double()
    _check(lib, None, lib.perk_measure_fp64(C.byref(f), C.byref(d), C.byref(l)))
    return f.value, d.value, l.value


def _ptr(t) -> int:
    return t.data_ptr()


class PerkSolver:
    """One libperk context: mesh, partition, coefficient table and stage buffers."""

    def __init__(self, gamma: float = 1.4, surface_flux: str = "hll", use_graph: bool = True, N: int = 3,
                 equations: str = "euler", mu: float = 0.0, prandtl: float = 0.72, shock_capturing=None,
                 alpha_max: float = 0.5):
        """shock_capturing: None, "density_pressure" or "density" (the indicator variable of the
        subcell blending of the volume term)."""
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("PerkSolver needs a CUDA device")
        self.torch = torch
        self.lib = _lib.load()
        eq = {"euler": 0, "navier_stokes": 1}[equations]
        prob = _lib.PerkProblem(N, gamma, _lib.SURFACE[surface_flux], 1 if use_graph else 0, eq, mu, prandtl,
                                _lib.SHOCK[shock_capturing], alpha_max)
        h = C.c_void_p()
        torch.cuda.init()
        _check(self.lib, None, self.lib.perk_create(C.byref(prob), C.byref(h)))
        self.ctx = h
        self.gamma = gamma
        self._cells = None
        self.n_elem = 0
        self.S = 0

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx:
            self.lib.perk_destroy(ctx)
            self.ctx = None

    def _stream(self):
        s = self.torch.cuda.current_stream().cuda_stream
        _check(self.lib, self.ctx, self.lib.perk_set_stream(self.ctx, C.c_void_p(s)))

    def _call(self, fn, *args):
        self._stream()
        _check(self.lib, self.ctx, fn(self.ctx, *args))

    # ------------------------------------------------------------------ setup
    def upload_mesh(self, cells, x0: float, length: float):
        arr = np.ascontiguousarray(np.asarray(cells, dtype=np.int32).reshape(-1, 3))
        self._call(self.lib.perk_mesh_upload, C.c_int64(len(arr)), arr.ctypes.data_as(C.POINTER(C.c_int32)),
                   C.c_double(x0), C.c_double(length))
        self.n_elem = len(arr)
        self.x0, self.length = float(x0), float(length)
        self.cells = arr
        self.n_members = 1

    def upload_ensemble(self, members, x0: float, length: float):
        """Independent meshes (a list of leaf lists) advanced together by one context."""
        arrs = [np.asarray(c, dtype=np.int32).reshape(-1, 3) for c in members]
        counts = (C.c_int64 * len(arrs))(*[len(a) for a in arrs])
        cat = np.ascontiguousarray(np.concatenate(arrs))
        self._call(self.lib.perk_ensemble_upload, len(arrs), counts, cat.ctypes.data_as(C.POINTER(C.c_int32)),
                   C.c_double(x0), C.c_double(length))
        self.n_elem = len(cat)
        self.x0, self.length = float(x0), float(length)
        self.cells = cat
        self.n_members = len(arrs)

    def members(self):
        m = np.zeros(self.n_elem, dtype=np.int32)
        self._call(self.lib.perk_get_members, m.ctypes.data_as(C.POINTER(C.c_int32)), C.c_int64(self.n_elem))
        return m

    def set_tableau(self, order: int, E: Sequence[int], c, a):
        E = [int(e) for e in E]
        c = np.ascontiguousarray(c, dtype=np.float64)
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(len(E), len(c))
        Ea = (C.c_int32 * len(E))(*E)
        self._call(self.lib.perk_set_tableau, int(order), len(c), len(E), Ea, c.ctypes.data_as(C.POINTER(C.c_double)),
                   a.ctypes.data_as(C.POINTER(C.c_double)))
        self.S = len(c)
        self.E = E

    def set_perk2_disk(self, E: Sequence[int], S: int | None = None, b_S: float = 1.0):
        c, a = perk2_disk_tableau(E, S, b_S)
        self.set_tableau(2, E, c, a)
        if b_S != 1.0:
            self.set_weights(1.0 - b_S, b_S)
        return c, a

    def set_tableau_pattern(self, E: Sequence[int], c, evaluated, src, a):
        E = [int(e) for e in E]
        c = np.ascontiguousarray(c, dtype=np.float64)
        S, R = len(c), len(E)
        ev = np.ascontiguousarray(evaluated, dtype=np.uint8).reshape(R, S)
        sr = np.ascontiguousarray(src, dtype=np.int32).reshape(R, S)
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(R, S)
        Ea = (C.c_int32 * R)(*E)
        self._call(self.lib.perk_set_tableau_pattern, 2, S, R, Ea, ev.ctypes.data_as(C.POINTER(C.c_uint8)),
                   sr.ctypes.data_as(C.POINTER(C.c_int32)), c.ctypes.data_as(C.POINTER(C.c_double)),
                   a.ctypes.data_as(C.POINTER(C.c_double)))
        self.S = S
        self.E = E

    def set_perk2_pattern(self, E: Sequence[int], pattern: str, S: int | None = None):
        c, ev, src, a = perk2_pattern_tableau(E, pattern, S)
        self.set_tableau_pattern(E, c, ev, src, a)
        return c, ev, src, a

    def set_weights(self, b1: float, bS: float):
        self._call(self.lib.perk_set_weights, C.c_double(b1), C.c_double(bS))

    def info(self) -> dict:
        inf = _lib.PerkMeshInfo()
        _check(self.lib, self.ctx, self.lib.perk_mesh_query(self.ctx, C.byref(inf)))
        S = inf.S
        return {"n_elem": inf.n_elem, "n_interfaces": inf.n_interfaces, "n_mortars": inf.n_mortars,
                "level_min": inf.level_min, "level_max": inf.level_max, "S": S,
                "dof_stage_updates": inf.dof_stage_updates, "active_elements": list(inf.active_elements[:S]),
                "active_interfaces": list(inf.active_interfaces[:S]), "active_mortars": list(inf.active_mortars[:S]),
                "index_bytes": inf.index_bytes}

    def set_stage_fusion(self, mode):
        """0 / False: two launches per stage; 1 / True: one launch per stage (faces and volume
        together); 2: one launch per step (all stages' items in order)."""
        self._call(self.lib.perk_set_stage_fusion, C.c_int(int(mode)))

    def workspace_bytes(self, n_cells: int = 0) -> int:
        """Bytes of a caller-owned workspace serving meshes of up to n_cells cells (0: the current mesh)."""
        out = C.c_size_t()
        _check(self.lib, self.ctx, self.lib.perk_workspace_bytes(self.ctx, C.c_int64(n_cells), C.byref(out)))
        return out.value

    def bind_workspace(self, ws):
        """Binds a caller-owned device block (a CUDA tensor of at least workspace_bytes() bytes, 256-byte
        aligned) as the context's device memory; None returns to the library's own allocations.  The
        tensor is kept referenced while bound."""
        if ws is None:
            self._call(self.lib.perk_bind_workspace, None, C.c_size_t(0))
            self._ws = None
            return
        if not ws.is_cuda or not ws.is_contiguous():
            raise ValueError("the workspace must be a contiguous CUDA tensor")
        self._call(self.lib.perk_bind_workspace, C.c_void_p(ws.data_ptr()),
                   C.c_size_t(ws.numel() * ws.element_size()))
        self._ws = ws

    def counters(self) -> dict:
        c = _lib.PerkCounters()
        _check(self.lib, self.ctx, self.lib.perk_get_counters(self.ctx, C.byref(c)))
        return {f: getattr(c, f) for f, _ in c._fields_}

    # -------------------------------------------------------------- compute
    def _state(self, t):
        torch = self.torch
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError("expected a contiguous float64 CUDA tensor")
        if tuple(t.shape) != (self.n_elem, 4, 4, 4):
            raise ValueError(f"expected shape {(self.n_elem, 4, 4, 4)}, got {tuple(t.shape)}")
        return t

    def empty_state(self):
        return self.torch.empty((self.n_elem, 4, 4, 4), dtype=self.torch.float64, device="cuda")

    def rhs_full(self, Y, out=None):
        Y = self._state(Y)
        K = self.empty_state() if out is None else self._state(out)
        self._call(self.lib.perk_rhs_full, C.c_void_p(_ptr(Y)), C.c_void_p(_ptr(K)))
        return K

    def rhs_active(self, stage: int, Y, out=None):
        Y = self._state(Y)
        K = self.torch.zeros_like(Y) if out is None else self._state(out)
        self._call(self.lib.perk_rhs_active, int(stage), C.c_void_p(_ptr(Y)), C.c_void_p(_ptr(K)))
        return K

    def step(self, U, dt):
        """One step; dt is a number, or one number per ensemble member."""
        U = self._state(U)
        if np.ndim(dt) == 0:
            self._call(self.lib.perk_step, C.c_void_p(_ptr(U)), C.c_double(float(dt)))
        else:
            d = np.ascontiguousarray(dt, dtype=np.float64)
            self._call(self.lib.perk_step_dts, C.c_void_p(_ptr(U)), d.ctypes.data_as(C.POINTER(C.c_double)))
        return U

    def compute_dt_members(self, U, cfl: float):
        U = self._state(U)
        out = np.zeros(getattr(self, "n_members", 1))
        self._call(self.lib.perk_compute_dt_members, C.c_void_p(_ptr(U)), C.c_double(cfl),
                   out.ctypes.data_as(C.POINTER(C.c_double)))
        return out

    def step_profiled(self, U, dt: float, acc=None):
        """One step with per-kernel CUDA-event timing; returns the accumulated times."""
        U = self._state(U)
        acc = acc if acc is not None else _lib.PerkKernelTimes()
        self._call(self.lib.perk_step_profiled, C.c_void_p(_ptr(U)), C.c_double(dt), C.byref(acc))
        return acc

    # ----------------------------------------------------------- derivatives
    def rhs_jvp(self, Y, V, stage: int = -1, out=None):
        Y, V = self._state(Y), self._state(V)
        Kd = self.torch.zeros_like(Y) if out is None else self._state(out)
        self._call(self.lib.perk_rhs_jvp, int(stage), C.c_void_p(_ptr(Y)), C.c_void_p(_ptr(V)), C.c_void_p(_ptr(Kd)))
        return Kd

    def rhs_vjp(self, Y, lam, stage: int = -1, out=None):
        Y, lam = self._state(Y), self._state(lam)
        g = self.empty_state() if out is None else self._state(out)
        self._call(self.lib.perk_rhs_vjp, int(stage), C.c_void_p(_ptr(Y)), C.c_void_p(_ptr(lam)), C.c_void_p(_ptr(g)))
        return g

    def step_vjp(self, Un, dt: float, lam_np1, out=None, stages=None):
        """lam_n = (dU_{n+1}/dU_n)^T lam_np1; with ``stages`` (from ``step_store`` on Un) the
        forward stages are not recomputed."""
        Un, lam_np1 = self._state(Un), self._state(lam_np1)
        lam_n = self.empty_state() if out is None else self._state(out)
        if stages is None:
            self._call(self.lib.perk_step_vjp, C.c_void_p(_ptr(Un)), C.c_double(dt), C.c_void_p(_ptr(lam_np1)),
                       C.c_void_p(_ptr(lam_n)))
        else:
            self._call(self.lib.perk_step_vjp_stored, C.c_void_p(_ptr(Un)), C.c_double(dt),
                       C.c_void_p(_ptr(self._stages(stages))), C.c_void_p(_ptr(lam_np1)), C.c_void_p(_ptr(lam_n)))
        return lam_n

    def step_store(self, U, dt: float, stages=None):
        """One step of U in place (as ``step``) that also returns its S stages [S, n_elem, 4, 4, 4]."""
        U = self._state(U)
        if stages is None:
            stages = self.torch.empty((self.S, self.n_elem, 4, 4, 4), dtype=self.torch.float64, device="cuda")
        self._call(self.lib.perk_step_store, C.c_void_p(_ptr(U)), C.c_double(dt), C.c_void_p(_ptr(self._stages(stages))))
        return stages

    def _stages(self, K):
        torch = self.torch
        if not (K.is_cuda and K.dtype == torch.float64 and K.is_contiguous()):
            raise ValueError("expected a contiguous float64 CUDA tensor of stages")
        if tuple(K.shape) != (self.S, self.n_elem, 4, 4, 4):
            raise ValueError(f"expected stages of shape {(self.S, self.n_elem, 4, 4, 4)}, got {tuple(K.shape)}")
        return K

    # ------------------------------------------------------------------ AMR
    def autotune(self, U) -> int:
        """Times the volume kernel with 2, 4 and 8 elements per block on the current mesh and keeps
        the fastest; returns the choice."""
        U = self._state(U)
        out = C.c_int32()
        self._call(self.lib.perk_autotune_volume, C.c_void_p(_ptr(U)), C.byref(out))
        return out.value

    def autotune_step(self, U, dt) -> int:
        """Times whole steps from U (left unchanged) with one launch per stage (1), one launch per
        step (2) and two launches per stage (0), keeps the fastest and returns it; dt: a step size,
        or one per ensemble member."""
        U = self._state(U)
        dts = np.ascontiguousarray(np.atleast_1d(np.asarray(dt, dtype=np.float64)))
        out = C.c_int32()
        self._call(self.lib.perk_autotune_step, C.c_void_p(_ptr(U)), dts.ctypes.data_as(C.POINTER(C.c_double)),
                   C.byref(out))
        return out.value

    def set_volume_blocks(self, elems_per_block: int):
        self._call(self.lib.perk_set_volume_blocks, C.c_int32(elems_per_block))

    INDICATORS = {"density": 0, "lohner_vx": 1}

    def amr_indicator(self, U, indicator: str = "density"):
        U = self._state(U)
        eta = self.torch.empty(self.n_elem, dtype=self.torch.float64, device="cuda")
        self._call(self.lib.perk_amr_indicator, C.c_int32(self.INDICATORS[indicator]), C.c_void_p(_ptr(U)),
                   C.c_void_p(_ptr(eta)))
        return eta

    def adapt(self, U, level_min: int = 4, level_max: int = 7, refine_above: float = 0.1,
              coarsen_below: float = 0.02, desired=None, indicator: str = "density", cfl: float | None = None):
        """One AMR cycle: returns the solution on the new mesh (a new tensor).  With cfl, the step
        size of the new state (as compute_dt) is computed in the same call and left in
        ``last_dt``."""
        U = self._state(U)
        prm = _lib.PerkAmrParams(level_min, level_max, refine_above, coarsen_below, self.INDICATORS[indicator])
        n_new = C.c_int64()
        if desired is not None:
            d = np.ascontiguousarray(np.asarray(desired, dtype=np.int32))
            self._call(self.lib.perk_adapt_plan, C.byref(prm), d.ctypes.data_as(C.POINTER(C.c_int32)),
                       C.c_void_p(_ptr(U)), C.byref(n_new))
        else:
            self._call(self.lib.perk_adapt_plan, C.byref(prm), None, C.c_void_p(_ptr(U)), C.byref(n_new))
        Unew = self.torch.empty((n_new.value, 4, 4, 4), dtype=self.torch.float64, device="cuda")
        if cfl is None:
            self._call(self.lib.perk_adapt_commit, C.c_void_p(_ptr(U)), C.c_void_p(_ptr(Unew)))
        else:
            dt = C.c_double()
            self._call(self.lib.perk_adapt_commit_dt, C.c_void_p(_ptr(U)), C.c_void_p(_ptr(Unew)), C.c_double(cfl),
                       C.byref(dt))
            self.last_dt = dt.value
        self.n_elem = n_new.value
        self.n_members = getattr(self, "n_members", 1)
        self._cells = None                  # read back from the library when first asked for
        return Unew

    @property
    def cells(self):
        """The current leaves (n_elem x 3 int32: level, ix, iy)."""
        if self._cells is None:
            cells = np.zeros((self.n_elem, 3), dtype=np.int32)
            self._call(self.lib.perk_get_cells, cells.ctypes.data_as(C.POINTER(C.c_int32)), C.c_int64(self.n_elem))
            self._cells = cells
        return self._cells

    @cells.setter
    def cells(self, value):
        self._cells = value

    def check(self):
        self._call(self.lib.perk_check)

    def compute_dt(self, U, cfl: float) -> float:
        U = self._state(U)
        out = C.c_double()
        self._call(self.lib.perk_compute_dt, C.c_void_p(_ptr(U)), C.c_double(cfl), C.byref(out))
        return out.value
