"""Pins of the operation counter (oracle/opcount.py) behind the stage kernels' roofline figure.

The counter must (1) compute the same values as plain floats, (2) count by the stated rules,
and (3) count computations that really are the method's: the counted element-stage is compared
with the oracle's own DGSEM volume and surface terms on the same element, the counted face
fluxes and mortar operators with their plain-float evaluations, and the flux counts with hand
counts from the formulas."""
import math

import numpy as np
import pytest

from oracle import euler
from oracle.dgsem import DGSEM
from oracle.opcount import Counting, OpCount, face_node_flux, mortar_operators, tally, volume_element_stage
from oracle.treemesh import TreeMesh


def test_values_are_plain_float_arithmetic():
    a, b, c = 1.25, -0.375, 3.0
    A, B, Cc = OpCount(a), OpCount(b), OpCount(c)
    got = (A * B + Cc) / (A - 2.0) - np.sqrt(Cc) + np.log(A) * (1.0 - B)
    want = (a * b + c) / (a - 2.0) - math.sqrt(c) + math.log(a) * (1.0 - b)
    assert float(got) == want


def test_counting_rules():
    with Counting():
        x, y, z = OpCount(2.0), OpCount(3.0), OpCount(5.0)
        r = x * y + z                        # one multiply, one add
        assert (y * x + z) is r              # the same operations again (commutative): one node each
        assert tally(r) == {"add": 1, "mul": 1, "div": 0, "sqrt": 0, "log": 0, "flops": 2}
        # identities, zero products and sign flips make no node
        assert tally([x + 0.0, x * 1.0, x * -1.0, -x, abs(x), x * 0.0])["flops"] == 0
        q = x / y
        s = np.sqrt(z) + np.log(z) + np.log(z)                   # the repeated logarithm is one node
        assert tally(s) == {"add": 2, "mul": 0, "div": 0, "sqrt": 1, "log": 1, "flops": 4}
        assert tally([x - y, y - x])["add"] == 2                  # subtraction is not commutative
        # a branch not taken is not counted
        picked = np.where(x < y, q, x * y * z)
        assert float(picked) == 2.0 / 3.0
    with Counting():
        x, y = OpCount(2.0), OpCount(3.0)
        t = tally(np.where(x < y, x / y, (x * y) * (x * y)))
        assert (t["div"], t["mul"]) == (1, 0)
    with Counting():
        # a decision needs both compared values: min(x - 1, y - 1) costs both subtractions
        x, y = OpCount(2.0), OpCount(3.0)
        m = np.minimum(x - 1.0, y - 1.0)
        assert tally(m)["add"] == 2


def test_volume_count_by_hand():
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
    dg = DGSEM(TreeMesh([(0, 0, 0)], 0.0, v["h"]), 3, "hll")
    vol = dg._volume(Y[:, None])[:, 0]
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


@pytest.mark.parametrize("flux", ["hll", "hllc", "ec", "hlle"])
def test_face_flux_counts_evaluate_the_flux(flux):
    r = face_node_flux(flux)
    SL, SR = r["speeds"]
    assert SL < 0.0 < SR                                   # the subsonic case is the one counted
    scale = np.max(np.abs(r["plain"]))
    tol = 1e-12 if flux == "ec" else 1e-15                 # ec: definition form of the log mean
    assert np.max(np.abs(r["value"] - r["plain"])) <= tol * scale


def test_hll_count_by_hand():
    # per side: v1, v2 (2 divides), p (5 multiplies, 2 adds), c = sqrt(gamma p / rho) (multiply,
    # divide, square root), f(u) (4 multiplies, 2 adds); the speeds v -/+ c (4 adds); the flux
    # (S_R f_L - S_L f_R + S_L S_R (u_R - u_L)) / (S_R - S_L): 8 + 1 + 4 multiplies, 4 + 4 + 4 + 1
    # adds, 4 divides
    c = face_node_flux("hll")["counts"]
    assert (c["add"], c["mul"], c["div"], c["sqrt"]) == (2 * 4 + 4 + 13, 2 * 10 + 13, 2 * 3 + 4, 2)


def test_mortar_operators_are_interpolation_and_projection():
    r = mortar_operators()
    v = r["values"]
    np.testing.assert_allclose(v["interpolation"], v["plain_interpolation"], rtol=0, atol=1e-14)
    np.testing.assert_allclose(v["projection"], v["plain_projection"], rtol=0, atol=1e-14)
    # projection: 4 outputs x 4 variables from 8 half-face values: 8 multiplies (no zero or unit
    # weights), 7 adds each
    assert (r["projection"]["mul"], r["projection"]["add"]) == (16 * 8, 16 * 7)
    assert r["total"]["flops"] == r["interpolation"]["flops"] + r["projection"]["flops"]


def test_bench_constants_are_the_counted_numbers():
    bench = pytest.importorskip("bench")
    assert bench.VOL_ALG_FLOPS_PER_ELEM == volume_element_stage()["total"]["flops"]
    for flux, n in bench.FACE_ALG_FLOPS_PER_NODE.items():
        assert n == face_node_flux(flux)["counts"]["flops"], flux
    assert bench.MORTAR_ALG_FLOPS == mortar_operators()["total"]["flops"]
