"""Floating-point operation counts of the stage work of the DGSEM (measurement aid).

Test and measurement infrastructure only (like the rest of ``oracle/``): the roofline
figure of the stage kernels divides an algorithmic operation count by the kernels' time,
and this module fixes that count from the oracle's own formulas instead of from the
kernels' instruction mix.

``OpCount`` is a float that records, for every arithmetic operation applied to it, a node
of an expression graph.  The count of a computation is the number of operation nodes its
outputs depend on, by kind: add (and subtract) and multiply 1 flop each (a fused
multiply-add would be 2), divide, square root and logarithm 1 each and tallied apart.
Counting what the outputs depend on keeps the count to the method's work rather than to
how an expression is spelled:

* a branch not taken (``np.where`` on a decided condition) is not counted, but every
  value a decision compares is (``np.minimum`` needs both of its arguments);
* an operation on the same operands is one node (common subexpressions: a node's
  primitive variables are formed once per node, not once per pair that reads them);
* operations with the identity constants (x + 0, x - 0, x * 1), products with zero, sign
  flips (-x, x * -1, |x|, folded into the consuming add) and operations on constants alone
  (such as gamma - 1) make no node.

Counted computations (N = 3, Euler; Sec. 6.1 with Eq. PartitionedRKSystem):

``volume_element_stage``: one stage of one element of the flux-differencing volume term:

* the stage state Y = U + dt (alpha K_1 + beta K_{i-1}) at the 16 nodes;
* per node the primitive variables (``euler.primitives``), rho / p and the logarithms of
  rho and rho / p;
* the 48 symmetric pairs of the 2 x 4 grid lines (6 pairs per line), each a call of
  ``euler.ec_flux`` with the logarithmic mean taken from its definition
  (b - a) / (ln b - ln a) on the node logarithms;
* the flux-differencing sum sum_m 2 D_im f#(u_i, u_m) over the three off-diagonal
  partners per direction (the diagonal terms cancel against the physical flux of the
  strong-form surface term, 2 D_00 + 1/w_0 = 0);
* the surface lifting (one multiply-add per variable at each of the 16 face-node slots)
  and the Jacobian factor -(2/h).

``face_node_flux``: the numerical surface flux (the oracle's ``hll_flux``, ``hllc_flux``,
``ec_flux`` or ``hlle_flux``) at one face node from the two traces, in the subsonic case
S_L < 0 < S_R of the workloads (HLLC: the left star state).

``mortar_operators``: per 2:1 mortar, the interpolation of the large trace to the 2 x 4
half-face nodes and the exact L2 projection of the two half-face fluxes back onto the
large face (the operators as matrices; their 8 flux evaluations are counted by
``face_node_flux``).
"""

from __future__ import annotations

import math

import numpy as np

from . import euler
from .lgl import derivative_matrix, l2_project_two_halves, lagrange_basis, lgl_nodes_weights

_SEEN = None       # the common-subexpression table of the current count, if any
_COMPARED = None   # values compared by decisions in the current count

KINDS = ("add", "mul", "div", "sqrt", "log")


class OpCount:
    """A float recording the operations applied to it (see the module docstring)."""

    __slots__ = ("v", "kind", "args")

    def __init__(self, v: float, kind: str = "input", args=()):
        self.v = float(v)
        self.kind = kind
        self.args = args

    def __repr__(self) -> str:
        return f"OpCount({self.v!r}, {self.kind})"

    def __float__(self) -> float:
        return self.v

    # ---- arithmetic
    def __add__(self, o):
        if isinstance(o, np.ndarray) and o.ndim > 0:
            return NotImplemented      # numpy applies the operation element by element
        if _is_const(o) and _val(o) == 0.0:
            return self
        return _op("add", "add", self, o, self.v + _val(o))

    __radd__ = __add__

    def __sub__(self, o):
        if isinstance(o, np.ndarray) and o.ndim > 0:
            return NotImplemented      # numpy applies the operation element by element
        if _is_const(o) and _val(o) == 0.0:
            return self
        return _op("add", "sub", self, o, self.v - _val(o))

    def __rsub__(self, o):
        if isinstance(o, np.ndarray) and o.ndim > 0:
            return NotImplemented      # numpy applies the operation element by element
        return _op("add", "sub", o, self, _val(o) - self.v)

    def __mul__(self, o):
        if isinstance(o, np.ndarray) and o.ndim > 0:
            return NotImplemented      # numpy applies the operation element by element
        if _is_const(o) and _val(o) == 1.0:
            return self
        if _is_const(o) and _val(o) == -1.0:
            return -self
        if _is_const(o) and _val(o) == 0.0:
            return 0.0
        return _op("mul", "mul", self, o, self.v * _val(o))

    __rmul__ = __mul__

    def __truediv__(self, o):
        if isinstance(o, np.ndarray) and o.ndim > 0:
            return NotImplemented      # numpy applies the operation element by element
        if _is_const(o) and _val(o) == 1.0:
            return self
        return _op("div", "div", self, o, self.v / _val(o))

    def __rtruediv__(self, o):
        if isinstance(o, np.ndarray) and o.ndim > 0:
            return NotImplemented      # numpy applies the operation element by element
        return _op("div", "div", o, self, _val(o) / self.v)

    def __neg__(self):
        return OpCount(-self.v, "sign", (self,))

    def __abs__(self):
        return OpCount(abs(self.v), "sign", (self,))

    # ---- comparisons decide branches: plain booleans; both compared values are needed
    def _cmp(self, o):
        if _COMPARED is not None:
            _COMPARED.append(self)
            if isinstance(_unwrap(o), OpCount):
                _COMPARED.append(_unwrap(o))
        return _val(o)

    def __lt__(self, o):
        return self.v < self._cmp(o)

    def __le__(self, o):
        return self.v <= self._cmp(o)

    def __gt__(self, o):
        return self.v > self._cmp(o)

    def __ge__(self, o):
        return self.v >= self._cmp(o)

    # ---- numpy's object-dtype ufuncs call these methods
    def sqrt(self):
        return _op("sqrt", "sqrt", self, None, math.sqrt(self.v))

    def log(self):
        return _op("log", "log", self, None, math.log(self.v))

    def log1p(self):
        return _op("log", "log1p", self, None, math.log1p(self.v))


def _unwrap(x):
    if isinstance(x, np.ndarray) and x.ndim == 0:
        return x.item()
    return x


def _is_const(x) -> bool:
    return not isinstance(_unwrap(x), OpCount)


def _val(x) -> float:
    x = _unwrap(x)
    return x.v if isinstance(x, OpCount) else float(x)


def _key(x):
    x = _unwrap(x)
    return ("n", id(x)) if isinstance(x, OpCount) else ("c", float(x))


def _op(kind: str, name: str, a, b, value: float):
    a, b = _unwrap(a), _unwrap(b)
    ka, kb = _key(a), (None if b is None else _key(b))
    if name in ("add", "mul") and repr(kb) < repr(ka):
        ka, kb = kb, ka                       # commutative
    key = (name, ka, kb)
    if _SEEN is not None:
        hit = _SEEN.get(key)
        if hit is not None:
            return hit[0]
    r = OpCount(value, kind, tuple(x for x in (a, b) if isinstance(x, OpCount)))
    if _SEEN is not None:
        _SEEN[key] = (r, a, b)                # the operands stay alive, so their ids stay unique
    return r


class Counting:
    """Context of one counted computation (common subexpressions shared inside it)."""

    def __enter__(self):
        global _SEEN, _COMPARED
        self._prev = (_SEEN, _COMPARED)
        _SEEN, _COMPARED = {}, []
        return self

    def __exit__(self, *exc):
        global _SEEN, _COMPARED
        _SEEN, _COMPARED = self._prev


def _leaves(x):
    x = _unwrap(x)
    if isinstance(x, OpCount):
        yield x
    elif isinstance(x, (list, tuple, np.ndarray)):
        for y in (x.flat if isinstance(x, np.ndarray) else x):
            yield from _leaves(y)


def tally(outputs) -> dict:
    """Counts by kind of the operations the outputs depend on, the values that decisions of
    the current count compared included; 'flops' is their sum."""
    counts = {k: 0 for k in KINDS}
    seen, stack = set(), list(_leaves(outputs)) + list(_COMPARED or [])
    while stack:
        n = stack.pop()
        if id(n) in seen:
            continue
        seen.add(id(n))
        if n.kind in KINDS:
            counts[n.kind] += 1
        stack.extend(n.args)
    counts["flops"] = sum(counts[k] for k in KINDS)
    return counts


def _diff(a: dict, b: dict) -> dict:
    return {k: a[k] - b[k] for k in a}


def _log_mean_definition(a, b):
    """(b - a) / (ln b - ln a), the logarithmic mean by its definition."""
    return (b - a) / (np.log(b) - np.log(a))


def _node_arrays(U: np.ndarray):
    """OpCount inputs of one element's nodes: node[j][i] is a length-4 object array."""
    n = U.shape[-1]
    return [[np.array([OpCount(U[v, j, i]) for v in range(4)], dtype=object) for i in range(n)]
            for j in range(n)]


def _state(rng, gamma, shape):
    rho = 1.0 + 0.1 * rng.uniform(-1, 1, shape)
    v1 = 0.3 + 0.1 * rng.uniform(-1, 1, shape)
    v2 = -0.2 + 0.1 * rng.uniform(-1, 1, shape)
    p = 1.0 + 0.1 * rng.uniform(-1, 1, shape)
    return np.stack([rho, rho * v1, rho * v2, p / (gamma - 1.0) + 0.5 * rho * (v1 * v1 + v2 * v2)])


def volume_element_stage(seed: int = 7, N: int = 3, gamma: float = euler.GAMMA,
                         alpha: float = 0.3, beta: float = 0.45, dt: float = 1e-3, h: float = 0.125) -> dict:
    """Operation counts of one element-stage of the volume term (see the module docstring).

    Returns the counts per part and in total, and the values of the counted computation
    (the element's volume-term contribution with given face fluxes) for checking against
    the oracle's own evaluation."""
    n = N + 1
    rng = np.random.default_rng(seed)
    U = _state(rng, gamma, (n, n))
    K1 = rng.standard_normal((4, n, n))
    Kp = rng.standard_normal((4, n, n))
    x, w = lgl_nodes_weights(N)
    D = derivative_matrix(x)
    da, db = dt * alpha, dt * beta           # per stage and element: constants
    parts = {}
    old = euler.log_mean
    euler.log_mean = _log_mean_definition
    try:
        with Counting():
            u, k1, kp = _node_arrays(U), _node_arrays(K1), _node_arrays(Kp)
            Y = [[u[j][i] + da * k1[j][i] + db * kp[j][i] for i in range(n)] for j in range(n)]
            done = tally(Y)
            parts["stage_state"] = done
            nodeq = []
            for j in range(n):
                for i in range(n):
                    r, v1, v2, pp = euler.primitives(Y[j][i], gamma)
                    b = r / pp
                    nodeq += [r, v1, v2, pp, b, np.log(r), np.log(b)]
            now = tally([Y, nodeq])
            parts["node_quantities"] = _diff(now, done)
            done = now
            F = {}
            for j in range(n):                  # x lines
                for i in range(n):
                    for m in range(i + 1, n):
                        F[(0, j, i, m)] = euler.ec_flux(Y[j][i], Y[j][m], 0, gamma)
            for i in range(n):                  # y lines
                for j in range(n):
                    for m in range(j + 1, n):
                        F[(1, i, j, m)] = euler.ec_flux(Y[j][i], Y[m][i], 1, gamma)
            now = tally([Y, nodeq, list(F.values())])
            parts["pair_fluxes"] = _diff(now, done)
            done = now
            acc = [[None] * n for _ in range(n)]
            for j in range(n):
                for i in range(n):
                    terms = [(2.0 * D[i, m]) * F[(0, j, min(i, m), max(i, m))] for m in range(n) if m != i]
                    terms += [(2.0 * D[j, m]) * F[(1, i, min(j, m), max(j, m))] for m in range(n) if m != j]
                    a = terms[0]
                    for t in terms[1:]:
                        a = a + t
                    acc[j][i] = a
            now = tally([Y, nodeq, list(F.values()), acc])
            parts["flux_differencing"] = _diff(now, done)
            done = now
            fstar = {(face, k): np.array([OpCount(0.1 * (face + 1) + 0.01 * k + 0.001 * v) for v in range(4)],
                                         dtype=object) for face in range(4) for k in range(n)}
            K = [[None] * n for _ in range(n)]
            for j in range(n):
                for i in range(n):
                    a = acc[j][i]
                    if i == 0:
                        a = a - (1.0 / w[0]) * fstar[(0, j)]
                    if i == N:
                        a = a + (1.0 / w[N]) * fstar[(1, j)]
                    if j == 0:
                        a = a - (1.0 / w[0]) * fstar[(2, i)]
                    if j == N:
                        a = a + (1.0 / w[N]) * fstar[(3, i)]
                    K[j][i] = (-2.0 / h) * a
            total = tally([Y, nodeq, list(F.values()), K])
            parts["lifting_jacobian"] = _diff(total, done)
    finally:
        euler.log_mean = old
    vol = np.array([[[float(K[j][i][v]) for i in range(n)] for j in range(n)] for v in range(4)])
    Yv = np.array([[[float(Y[j][i][v]) for i in range(n)] for j in range(n)] for v in range(4)])
    return {"parts": parts, "total": total,
            "values": {"Y": Yv, "K": vol, "fstar": {k: [float(q) for q in v] for k, v in fstar.items()},
                       "w": w, "D": D, "h": h}}


SURFACE = {"hll": euler.hll_flux, "hllc": euler.hllc_flux, "ec": euler.ec_flux, "hlle": euler.hlle_flux}


def face_node_flux(flux: str = "hllc", seed: int = 11, gamma: float = euler.GAMMA, direction: int = 0) -> dict:
    """Operation count of the numerical flux at one face node from its two traces (a subsonic
    state pair, S_L < 0 < S_R), with the counted and the plain-float flux values."""
    rng = np.random.default_rng(seed)
    uL, uR = _state(rng, gamma, ()), _state(rng, gamma, ())
    old = euler.log_mean
    euler.log_mean = _log_mean_definition
    try:
        with Counting():
            a = np.array([OpCount(v) for v in uL], dtype=object)
            b = np.array([OpCount(v) for v in uR], dtype=object)
            f = SURFACE[flux](a, b, direction, gamma)
            counts = tally(f)
    finally:
        euler.log_mean = old
    return {"counts": counts, "value": np.array([_val(q) for q in np.asarray(f, dtype=object).ravel()]),
            "plain": np.asarray(SURFACE[flux](uL, uR, direction, gamma), dtype=np.float64),
            "speeds": euler.davis_speeds(uL, uR, direction, gamma)}


def mortar_operators(N: int = 3, seed: int = 3) -> dict:
    """Operation counts of one mortar's operators: the large trace (4 variables at N + 1 nodes)
    interpolated to both half faces, and the two half-face fluxes projected back by the exact
    L2 projection (its matrix from ``l2_project_two_halves`` applied to unit vectors); also the
    counted values and their plain-float evaluation."""
    n = N + 1
    x, _ = lgl_nodes_weights(N)
    P = [lagrange_basis(x, 0.5 * (x - 1.0)), lagrange_basis(x, 0.5 * (x + 1.0))]   # [half][node, l]
    R = np.zeros((n, 2 * n))                                                       # projection matrix
    for c in range(2 * n):
        e = np.zeros(2 * n)
        e[c] = 1.0
        R[:, c] = l2_project_two_halves(x, e[:n], e[n:])
    rng = np.random.default_rng(seed)
    trace = rng.standard_normal((4, n))
    halves = rng.standard_normal((2, 4, n))
    with Counting():
        t = np.array([[OpCount(v) for v in row] for row in trace], dtype=object)
        fh = np.array([[[OpCount(v) for v in row] for row in hv] for hv in halves], dtype=object)
        interp = np.empty((2, 4, n), dtype=object)
        for hf in range(2):
            for k in range(n):
                for v in range(4):
                    terms = [P[hf][k, l] * t[v, l] for l in range(n)]
                    acc = terms[0]
                    for term in terms[1:]:
                        acc = acc + term
                    interp[hf, v, k] = acc
        proj = np.empty((4, n), dtype=object)
        for k in range(n):
            for v in range(4):
                terms = [R[k, c] * fh[c // n, v, c % n] for c in range(2 * n)]
                acc = terms[0]
                for term in terms[1:]:
                    acc = acc + term
                proj[v, k] = acc
        counts = {"interpolation": tally(interp), "projection": tally(proj), "total": tally([interp, proj])}
    plain_interp = np.stack([trace @ P[hf].T for hf in range(2)])
    plain_proj = l2_project_two_halves(x, halves[0], halves[1])
    return {**counts, "values": {"interpolation": np.vectorize(_val)(interp), "projection": np.vectorize(_val)(proj),
                                 "plain_interpolation": plain_interp, "plain_projection": plain_proj}}


def stage_counts(flux: str = "hllc") -> dict:
    """Algorithmic flops of one element-stage of the volume term, of one face-node flux and of
    one mortar's operators."""
    return {"volume_element_stage": volume_element_stage()["total"]["flops"],
            "face_node_flux": face_node_flux(flux)["counts"]["flops"],
            "mortar_operators": mortar_operators()["total"]["flops"]}


if __name__ == "__main__":
    import json
    r = volume_element_stage()
    print(json.dumps({"volume_parts": r["parts"], "volume_total": r["total"],
                      "faces": {f: face_node_flux(f)["counts"] for f in SURFACE},
                      "mortar": {k: mortar_operators()[k] for k in ("interpolation", "projection", "total")}},
                     indent=1))
