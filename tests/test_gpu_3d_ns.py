"""GPU parity of the 3D Navier-Stokes path (BR1 viscous terms, the paper's viscous Taylor-Green
run of Sec. 7.1.3) with the 3D BR1 oracle: full and stage-wise right-hand sides for both built
degrees, P-ERK3 {3,4,6} steps, and the admissibility check on the viscous kernel's last stage."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.br1_3d import NavierStokesDGSEM3D
from oracle.dgsem3d import max_wave_speed_dt3
from oracle.lgl import lgl_nodes_weights
from oracle.octree import OctreeMesh
from oracle.perk import element_methods, perk3_family, prkm_step
from perk_inputs.octree import (block_refined_cells3, nodal_state3, refine_cells3, smooth_random_state3,
                                taylor_green, uniform_cells3)

pytestmark = pytest.mark.gpu

L = 2.0 * math.pi
MU = 1.0 / 1600.0


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_05144_gb300.build import build
    build()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def three_level_cells():
    c = refine_cells3(uniform_cells3(2), lambda l, ix, iy, iz: 1 <= ix < 3 and 0 <= iy < 2 and 1 <= iz < 4)
    return refine_cells3(c, lambda l, ix, iy, iz: l == 3 and 3 <= ix < 5 and 1 <= iy < 3 and 3 <= iz < 5)


def solver(cells, N=2, flux="hlle", mu=MU):
    from paper_2403_05144_gb300.perk3d import Perk3DSolver
    s = Perk3DSolver(N=N, surface_flux=flux, equations="navier_stokes", mu=mu, prandtl=0.72)
    s.upload_mesh(cells, 0.0, L)
    return s


def state(cells, N, seed=17):
    x, _ = lgl_nodes_weights(N)
    U = smooth_random_state3(cells, 0.0, L, x, seed=seed, amplitude=0.2)
    return U * (1.0 + 0.05 * np.random.default_rng(seed + 1).uniform(-1, 1, size=U.shape))


def rel_err(got, want):
    return max(np.max(np.abs(got[:, v] - want[:, v])) / max(np.max(np.abs(want[:, v])), 1e-300) for v in range(5))


def oracle_tableau_into(s, fam):
    a = np.zeros((fam.R, fam.S))
    for r in range(fam.R):
        for i in range(2, fam.S):
            a[r, i] = fam.A[r][i, i - 1]
    s.set_tableau(fam.order, fam.E, fam.c, a)


@pytest.mark.parametrize("N", [2, 3])
@pytest.mark.parametrize("mesh", ["block", "three_level"])
def test_rhs_full(N, mesh):
    cells = block_refined_cells3(2, 1, 3) if mesh == "block" else three_level_cells()
    U = state(cells, N)
    mu = 0.05            # large enough that the viscous part is a visible share of the RHS
    got = solver(cells, N, "hllc", mu).rhs_full(cuda(U)).cpu().numpy()
    op = NavierStokesDGSEM3D(OctreeMesh(np.asarray(cells), 0.0, L), N, "hllc", mu=mu, prandtl=0.72)
    assert rel_err(got, op.rhs(U)) < 1e-12
    visc = op.viscous_rhs(U)
    assert np.max(np.abs(visc)) > 1e-3 * np.max(np.abs(op.rhs(U)))


def test_rhs_active_every_stage():
    cells = three_level_cells()
    mesh = OctreeMesh(np.asarray(cells), 0.0, L)
    fam = perk3_family([3, 4, 6])
    s = solver(cells, 2, "hlle", 0.05)
    oracle_tableau_into(s, fam)
    U = state(cells, 2)
    full = NavierStokesDGSEM3D(mesh, 2, "hlle", mu=0.05, prandtl=0.72).rhs(U)
    meth = element_methods(mesh.cells[:, 0], fam.R)
    for i in range(fam.S):
        active = np.array([fam.active(int(m), i) for m in meth])
        got = s.rhs_active(i, cuda(U)).cpu().numpy()
        assert rel_err(got[active], full[active]) < 1e-12
        assert np.all(got[~active] == 0.0)


def test_perk3_steps_match_oracle():
    """Three P-ERK3 {3,4,6} steps of the viscous Taylor-Green state (Re 1600, Pr 0.72), N = 2."""
    cells = three_level_cells()
    mesh = OctreeMesh(np.asarray(cells), 0.0, L)
    x, _ = lgl_nodes_weights(2)
    U0 = nodal_state3(taylor_green, cells, 0.0, L, x)
    fam = perk3_family([3, 4, 6])
    dt = max_wave_speed_dt3(U0, mesh.h, 2, 0.5)
    s = solver(cells)
    oracle_tableau_into(s, fam)
    U = cuda(U0.copy())
    for _ in range(3):
        s.step(U, dt)
    s.check()
    rhs = NavierStokesDGSEM3D(mesh, 2, "hlle", mu=MU, prandtl=0.72).rhs
    want = U0
    meth = element_methods(mesh.cells[:, 0], fam.R)
    for _ in range(3):
        want = prkm_step(rhs, want, dt, fam, meth)
    got = U.cpu().numpy()
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_rejected_viscous_step_leaves_state_unchanged():
    cells = block_refined_cells3(2, 1, 3)
    U0 = state(cells, 2)
    s = solver(cells)
    s.set_perk3_disk([3, 4, 6])
    U = cuda(U0.copy())
    s.step(U, 50.0)
    from paper_2403_05144_gb300._lib import PerkError
    with pytest.raises(PerkError, match="NONFINITE"):
        s.check()
    assert np.array_equal(U.cpu().numpy(), U0)
