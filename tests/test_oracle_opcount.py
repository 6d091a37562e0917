"""Pins of the operation counter (oracle/opcount.py) behind the volume kernel's roofline figure.

The counter must (1) compute the same values as plain floats, (2) count by the stated rules, and
(3) count a computation that really is the volume term: the counted element-stage is compared
with the oracle's own DGSEM volume and surface terms on the same element."""
import math

import numpy as np
import pytest

from oracle import euler
from oracle.dgsem import DGSEM
from oracle.opcount import OpCount, tally, volume_element_stage
from oracle.treemesh import TreeMesh


def test_values_are_plain_float_arithmetic():
    a, b, c = 1.25, -0.375, 3.0
    A, B, Cc = OpCount(a), OpCount(b), OpCount(c)
    got = (A * B + Cc) / (A - 2.0) - np.sqrt(Cc) + np.log(A) * (1.0 - B)
    want = (a * b + c) / (a - 2.0) - math.sqrt(c) + math.log(a) * (1.0 - b)
    assert float(got) == want


def test_counting_rules():
    with tally() as t:
        x, y, z = OpCount(2.0), OpCount(3.0), OpCount(5.0)
        r = x * y + z                    # one multiply, one add
        r2 = y * x + z                   # the same operations again (commutative): free
        assert r2 is r
        x + 0.0, x * 1.0, x * -1.0, -x, abs(x)    # identities and sign flips: free
        q = x / y                        # a divide
        np.sqrt(z), np.log(z), np.log(z)  # square root once, logarithm once (repeated: free)
        bool(x < y)                      # a comparison, not a flop
        x - y, y - x                     # subtraction is not commutative: two adds
    assert (t.add, t.mul, t.div, t.sqrt, t.log, t.cmp) == (3, 1, 1, 1, 1, 1)
    assert t.flops == 3 + 1 + 1 + 1 + 1
    assert float(q) == 2.0 / 3.0


def test_pair_flux_count_by_hand():
    # Ranocha's flux on node quantities already formed: the two logarithmic means
    # (b - a)/(ln b - ln a): 2 adds + 1 divide each; the arithmetic means of v1, v2, p: add + multiply
    # each; f_rho: multiply; f_m (normal direction): multiply + add, tangential: multiply;
    # f_E: v_L.v_R/2 (2 multiplies, add, multiply), 1/((gamma-1) beta_ln) (multiply, divide), their
    # sum (add) times f_rho (multiply), (p_L v_n,R + p_R v_n,L)/2 (2 multiplies, add, multiply), sum
    # (add).  12 adds, 14 multiplies, 3 divides (the third is 1/((gamma-1) beta_ln)).
    r = volume_element_stage()
    pairs = r["parts"]["pair_fluxes"]
    assert (pairs["add"], pairs["mul"], pairs["div"], pairs["log"]) == (48 * 12, 48 * 14, 48 * 3, 0)
    nodes = r["parts"]["node_quantities"]
    # per node: v1, v2, rho/p (3 divides); p = (gamma-1)(E - rho/2 (v1^2 + v2^2)): 5 multiplies,
    # 2 adds; the logarithms of rho and rho/p
    assert (nodes["add"], nodes["mul"], nodes["div"], nodes["log"]) == (16 * 2, 16 * 5, 16 * 3, 16 * 2)
    st = r["parts"]["stage_state"]
    assert (st["add"], st["mul"]) == (64 * 2, 64 * 2)
    fd = r["parts"]["flux_differencing"]
    # 6 off-diagonal partners per node and variable, 5 adds; the coefficients 2 D_03 = 1 and
    # 2 D_30 = -1 of every grid line need no multiply (16 per variable)
    assert (fd["add"], fd["mul"]) == (16 * 4 * 5, 16 * 4 * 6 - 4 * 16)
    lj = r["parts"]["lifting_jacobian"]
    assert (lj["add"], lj["mul"]) == (16 * 4, 16 * 4 + 64)
    assert r["total"]["flops"] == 256 + 192 + 48 * 29 + 640 + 192 == 2672


def test_counted_element_stage_is_the_oracle_volume_term():
    r = volume_element_stage()
    v = r["values"]
    Y = v["Y"]                                            # [4, j, i]
    cells = [(0, 0, 0)]
    dg = DGSEM(TreeMesh(cells, 0.0, v["h"]), 3, "hll")
    V = Y[:, None]                                        # [4, e, j, i]
    vol = dg._volume(V)[:, 0]
    # the strong-form surface term with the counted face fluxes (faces 0..3 = -x, +x, -y, +y)
    fs = {k: np.array(q) for k, q in v["fstar"].items()}
    w = v["w"]
    S = np.zeros_like(Y)
    for j in range(4):
        S[:, j, 0] -= (fs[(0, j)] - euler.physical_flux(Y[:, j, 0], 0)) / w[0]
        S[:, j, 3] += (fs[(1, j)] - euler.physical_flux(Y[:, j, 3], 0)) / w[3]
    for i in range(4):
        S[:, 0, i] -= (fs[(2, i)] - euler.physical_flux(Y[:, 0, i], 1)) / w[0]
        S[:, 3, i] += (fs[(3, i)] - euler.physical_flux(Y[:, 3, i], 1)) / w[3]
    want = -(2.0 / v["h"]) * (vol + S)
    # the counted form takes the logarithmic mean from its definition (no series near equal
    # arguments), so it agrees with the oracle's stable form to a few hundred ulps of the RHS
    assert np.max(np.abs(v["K"] - want)) / np.max(np.abs(want)) < 1e-10


def test_bench_constant_is_the_counted_number():
    bench = pytest.importorskip("bench")
    assert bench.VOL_ALG_FLOPS_PER_ELEM == volume_element_stage()["total"]["flops"]
