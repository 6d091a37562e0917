"""Floating-point operation counts of one element-stage of the DGSEM volume term.

Test and measurement infrastructure only (like the rest of ``oracle/``): the
roofline figure of the volume kernel divides an algorithmic operation count by
the kernel's time, and this module fixes that count from the oracle's own
formulas instead of from the kernel's instruction mix.

``OpCount`` is a float that records every arithmetic operation applied to it.
The convention (add, subtract, multiply = 1; a fused multiply-add would be 2;
divide, square root and logarithm 1 each and tallied separately; comparisons
tallied but not counted as flops) is applied to the oracle's expressions as
written.  Two rules keep the count to the method's work rather than to how an
expression happens to be spelled:

* operations with the identity constants (x + 0, x - 0, x * 1), sign flips
  (-x, x * -1, |x|: folded into the consuming add) and operations on
  constants alone (such as gamma - 1) cost nothing;
* within one ``Tally`` an operation on the same operands is counted once
  (common subexpressions: a node's primitive variables are formed once per
  node, not once per pair that reads them).

``volume_element_stage`` counts one stage of one element (N = 3, Euler) of the
flux-differencing volume term with the work the method needs (Sec. 6.1 with
Eq. PartitionedRKSystem):

* the stage state Y = U + dt (alpha K_1 + beta K_{i-1}) at the 16 nodes;
* per node the primitive variables (``euler.primitives``), rho / p and the
  logarithms of rho and rho / p;
* the 48 symmetric pairs of the 2 x 4 grid lines (6 pairs per line), each a
  call of ``euler.ec_flux`` with the logarithmic mean taken from its definition
  (b - a) / (ln b - ln a) on the node logarithms;
* the flux-differencing sum sum_m 2 D_im f#(u_i, u_m) over the three
  off-diagonal partners per direction (the diagonal terms cancel against the
  physical flux of the strong-form surface term, 2 D_00 + 1/w_0 = 0);
* the surface lifting (one multiply-add per variable at each of the 16
  face-node slots) and the Jacobian factor -(2/h).
"""

from __future__ import annotations

import contextlib
import math
from dataclasses import dataclass, field

import numpy as np

from . import euler
from .lgl import derivative_matrix, lgl_nodes_weights

_ACTIVE = None   # the Tally collecting counts, if any


@dataclass
class Tally:
    add: int = 0
    mul: int = 0
    div: int = 0
    sqrt: int = 0
    log: int = 0
    cmp: int = 0
    _seen: dict = field(default_factory=dict, repr=False)

    @property
    def flops(self) -> int:
        """add/mul = 1 each, divide, square root and logarithm 1 each."""
        return self.add + self.mul + self.div + self.sqrt + self.log

    def as_dict(self) -> dict:
        return {"add": self.add, "mul": self.mul, "div": self.div, "sqrt": self.sqrt, "log": self.log,
                "cmp": self.cmp, "flops": self.flops}


@contextlib.contextmanager
def tally():
    """Collects the operations of OpCount values inside the block."""
    global _ACTIVE
    prev, _ACTIVE = _ACTIVE, Tally()
    try:
        yield _ACTIVE
    finally:
        _ACTIVE = prev


def _is_const(x) -> bool:
    return not isinstance(x, OpCount)


def _val(x) -> float:
    return x.v if isinstance(x, OpCount) else float(x)


def _op(kind: str, key, value: float, operands=()):
    """Result of an operation; counted unless the same operation was counted before."""
    t = _ACTIVE
    if t is None:
        return OpCount(value)
    hit = t._seen.get(key)
    if hit is not None:
        return hit[0]
    setattr(t, kind, getattr(t, kind) + 1)
    r = OpCount(value)
    t._seen[key] = (r, operands)   # the operands stay alive, so their ids stay unique
    return r


def _key(name, a, b=None):
    ka = id(a) if isinstance(a, OpCount) else ("c", _val(a))
    kb = None if b is None else (id(b) if isinstance(b, OpCount) else ("c", _val(b)))
    if name in ("add", "mul") and kb is not None and repr(kb) < repr(ka):
        ka, kb = kb, ka                      # commutative
    return (name, ka, kb)


class OpCount:
    """A float that counts the operations applied to it (see the module docstring)."""

    __slots__ = ("v", "__weakref__")

    def __init__(self, v: float):
        self.v = float(v)

    def __repr__(self) -> str:
        return f"OpCount({self.v!r})"

    def __float__(self) -> float:
        return self.v

    # ---- arithmetic
    def __add__(self, o):
        if _is_const(o) and _val(o) == 0.0:
            return self
        return _op("add", _key("add", self, o), self.v + _val(o), (self, o))

    __radd__ = __add__

    def __sub__(self, o):
        if _is_const(o) and _val(o) == 0.0:
            return self
        return _op("add", _key("sub", self, o), self.v - _val(o), (self, o))

    def __rsub__(self, o):
        return _op("add", _key("sub", o, self), _val(o) - self.v, (self, o))

    def __mul__(self, o):
        if _is_const(o) and _val(o) == 1.0:
            return self
        if _is_const(o) and _val(o) == -1.0:
            return -self
        return _op("mul", _key("mul", self, o), self.v * _val(o), (self, o))

    __rmul__ = __mul__

    def __truediv__(self, o):
        if _is_const(o) and _val(o) == 1.0:
            return self
        return _op("div", _key("div", self, o), self.v / _val(o), (self, o))

    def __rtruediv__(self, o):
        return _op("div", _key("div", o, self), _val(o) / self.v, (self, o))

    def __neg__(self):
        return OpCount(-self.v)            # a sign flip, folded into the consumer

    def __abs__(self):
        return OpCount(abs(self.v))        # clears the sign bit

    # ---- comparisons (tallied, not flops)
    def _cmp(self, o, f):
        if _ACTIVE is not None:
            _ACTIVE.cmp += 1
        return f(self.v, _val(o))

    def __lt__(self, o):
        return self._cmp(o, lambda a, b: a < b)

    def __le__(self, o):
        return self._cmp(o, lambda a, b: a <= b)

    def __gt__(self, o):
        return self._cmp(o, lambda a, b: a > b)

    def __ge__(self, o):
        return self._cmp(o, lambda a, b: a >= b)

    # ---- numpy's object-dtype ufuncs call these methods
    def sqrt(self):
        return _op("sqrt", _key("sqrt", self), math.sqrt(self.v), (self,))

    def log(self):
        return _op("log", _key("log", self), math.log(self.v), (self,))

    def log1p(self):
        return _op("log", _key("log1p", self), math.log1p(self.v), (self,))


def _log_mean_definition(a, b):
    """(b - a) / (ln b - ln a), the logarithmic mean by its definition."""
    return (b - a) / (np.log(b) - np.log(a))


def _node_arrays(U: np.ndarray):
    """OpCount values of one element's nodes: node[j][i] is a length-4 object array."""
    return [[np.array([OpCount(U[v, j, i]) for v in range(4)], dtype=object) for i in range(4)]
            for j in range(4)]


def volume_element_stage(seed: int = 7, N: int = 3, gamma: float = euler.GAMMA,
                         alpha: float = 0.3, beta: float = 0.45, dt: float = 1e-3, h: float = 0.125) -> dict:
    """Operation counts of one element-stage of the volume term (see the module docstring).

    Returns the tally per part and in total, and the values of the counted
    computation (the element's volume-term contribution, without the surface
    fluxes) for checking against the oracle's own evaluation."""
    n = N + 1
    rng = np.random.default_rng(seed)
    # a smooth admissible element state and two stage derivatives
    rho = 1.0 + 0.1 * rng.uniform(-1, 1, (n, n))
    v1 = 0.3 + 0.1 * rng.uniform(-1, 1, (n, n))
    v2 = -0.2 + 0.1 * rng.uniform(-1, 1, (n, n))
    p = 1.0 + 0.1 * rng.uniform(-1, 1, (n, n))
    U = np.stack([rho, rho * v1, rho * v2, p / (gamma - 1.0) + 0.5 * rho * (v1 * v1 + v2 * v2)])
    K1 = rng.standard_normal((4, n, n))
    Kp = rng.standard_normal((4, n, n))
    x, w = lgl_nodes_weights(N)
    D = derivative_matrix(x)
    da, db = dt * alpha, dt * beta           # per stage and element: constants
    parts = {}
    old = (euler.log_mean,)
    euler.log_mean = _log_mean_definition
    try:
        with tally() as t:
            u, k1, kp = _node_arrays(U), _node_arrays(K1), _node_arrays(Kp)
            # stage state
            Y = [[u[j][i] + da * k1[j][i] + db * kp[j][i] for i in range(n)] for j in range(n)]
            parts["stage_state"] = t.as_dict()
            # node quantities: primitives, rho / p and the two logarithms (formed once per node)
            for j in range(n):
                for i in range(n):
                    r, _, _, pp = euler.primitives(Y[j][i], gamma)
                    b = r / pp
                    np.log(r)
                    np.log(b)
            parts["node_quantities"] = _diff(t.as_dict(), parts["stage_state"])
            # the symmetric pairs of every grid line
            F = {}
            before = t.as_dict()
            for j in range(n):                  # x lines
                for i in range(n):
                    for m in range(i + 1, n):
                        F[(0, j, i, m)] = euler.ec_flux(Y[j][i], Y[j][m], 0, gamma)
            for i in range(n):                  # y lines
                for j in range(n):
                    for m in range(j + 1, n):
                        F[(1, i, j, m)] = euler.ec_flux(Y[j][i], Y[m][i], 1, gamma)
            parts["pair_fluxes"] = _diff(t.as_dict(), before)
            # flux differencing: sum over the off-diagonal partners of 2 D_im f#
            before = t.as_dict()
            acc = [[None] * n for _ in range(n)]
            for j in range(n):
                for i in range(n):
                    a = np.array([OpCount(0.0)] * 4, dtype=object)
                    first = True
                    for m in range(n):
                        if m == i:
                            continue
                        f = F[(0, j, min(i, m), max(i, m))]
                        term = (2.0 * D[i, m]) * f
                        a = term if first else a + term
                        first = False
                    for m in range(n):
                        if m == j:
                            continue
                        f = F[(1, i, min(j, m), max(j, m))]
                        a = a + (2.0 * D[j, m]) * f
                    acc[j][i] = a
            parts["flux_differencing"] = _diff(t.as_dict(), before)
            # surface lifting (the numerical face fluxes come from the face kernel) and Jacobian
            before = t.as_dict()
            fstar = {(face, k): np.array([OpCount(0.1 * (face + 1) + 0.01 * k + 0.001 * v) for v in range(4)],
                                         dtype=object) for face in range(4) for k in range(n)}
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
                    acc[j][i] = (-2.0 / h) * a
            parts["lifting_jacobian"] = _diff(t.as_dict(), before)
            total = t.as_dict()
    finally:
        (euler.log_mean,) = old
    vol = np.array([[[float(acc[j][i][v]) for i in range(n)] for j in range(n)] for v in range(4)])
    Yv = np.array([[[float(Y[j][i][v]) for i in range(n)] for j in range(n)] for v in range(4)])
    return {"parts": parts, "total": total, "values": {"Y": Yv, "K": vol, "fstar": {k: [float(q) for q in v]
                                                                                     for k, v in fstar.items()},
                                                        "w": w, "D": D, "h": h}}


def _diff(a: dict, b: dict) -> dict:
    return {k: a[k] - b[k] for k in a}


if __name__ == "__main__":
    import json
    r = volume_element_stage()
    print(json.dumps({"parts": r["parts"], "total": r["total"]}, indent=1))
