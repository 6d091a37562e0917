"""One launch per step (k_step: all stages' items dealt in order, mode 2) and one launch per stage
(k_stage: face fluxes and volume terms together, mode 1) against two launches per stage (mode 0):
the same arithmetic on the same data, so the steps must agree bit for bit; the fused steps are also
checked against the oracle here and by the parity tests, which run in the default mode."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.dgsem import DGSEM
from oracle.perk import element_methods, max_wave_speed_dt, perk2_family, prkm_step
from oracle.treemesh import TreeMesh
from perk_inputs import kelvin_helmholtz, kh_band_cells, nested_band_cells, nodal_state, uniform_cells
from tests.gpu_common import X3

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_05144_gb300.build import build
    build()


def solver(cells, fused, use_graph=True, flux="hllc", E=(4, 6, 10, 16)):
    from paper_2403_05144_gb300 import PerkSolver
    s = PerkSolver(surface_flux=flux, use_graph=use_graph)
    s.set_stage_fusion(fused)
    s.upload_mesh(cells, -1.0, 2.0)
    s.set_perk2_disk(list(E))
    return s


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("flux", ["hllc", "hll", "ec"])
def test_fused_steps_bitwise_equal_to_two_launches(use_graph, flux):
    cells = kh_band_cells(4, 7, 0.03)
    U0 = torch.from_numpy(nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)).cuda()
    out = []
    for mode in (2, 1, 0):
        s = solver(cells, mode, use_graph, flux)
        U = U0.clone()
        dt = s.compute_dt(U, 0.7)
        for _ in range(5):
            s.step(U, dt)
        s.check()
        out.append(U)
    assert torch.equal(out[0], out[2]) and torch.equal(out[1], out[2])


def test_fused_steps_with_amr_and_ensembles():
    # dynamic AMR (device-built meshes) and a two-member ensemble with per-member dt
    amr = dict(level_min=3, level_max=6, refine_above=0.1, coarsen_below=0.02)
    out = []
    for fused in (2, 1, 0):
        s = solver(uniform_cells(3), fused)
        U = torch.from_numpy(nodal_state(kelvin_helmholtz, uniform_cells(3), -1.0, 2.0, X3)).cuda()
        for _ in range(4):
            U = s.adapt(U, **amr)
            dt = s.compute_dt(U, 0.7)
            for _ in range(3):
                s.step(U, dt)
        s.check()
        out.append(U)
    assert torch.equal(out[0], out[2]) and torch.equal(out[1], out[2])
    from paper_2403_05144_gb300 import PerkSolver
    meshes = [kh_band_cells(4, 6, 0.05), nested_band_cells(2, 5)]
    res = []
    for fused in (2, 1, 0):
        e = PerkSolver(surface_flux="hllc")
        e.set_stage_fusion(fused)
        e.upload_ensemble(meshes, -1.0, 2.0)
        e.set_perk2_disk([4, 6, 10, 16])
        U = torch.from_numpy(np.concatenate([nodal_state(kelvin_helmholtz, c, -1.0, 2.0, X3) for c in meshes])).cuda()
        dts = e.compute_dt_members(U, 0.7)
        for _ in range(3):
            e.step(U, dts)
        e.check()
        res.append(U)
    assert torch.equal(res[0], res[2]) and torch.equal(res[1], res[2])


def test_fused_pattern_steps_and_profile():
    cells = nested_band_cells(2, 5)
    U0 = torch.from_numpy(nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)).cuda()
    out = []
    for fused in (2, True, False):   # stage patterns keep one launch per stage in mode 2
        s = solver(cells, fused, E=(4, 8))
        s.set_perk2_pattern([4, 8], "early")
        U = U0.clone()
        for _ in range(3):
            s.step(U, 2e-3)
        s.check()
        out.append(U)
    assert torch.equal(out[0], out[2]) and torch.equal(out[1], out[2])
    s = solver(cells, True)
    U = U0.clone()
    acc = s.step_profiled(U, 2e-3)
    assert acc.launches[0] == 0 and acc.launches[1] == 16 and acc.launches[2] == 1


@pytest.mark.parametrize("mode", [1, 2])
def test_fused_step_matches_oracle_on_four_levels(mode):
    cells = nested_band_cells(2, 5)
    U0 = nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)
    m = TreeMesh(cells, -1.0, 2.0)
    fam = perk2_family([4, 6, 10, 16])
    dt = max_wave_speed_dt(U0, m.h, 3, 0.7)
    s = solver(cells, mode)
    U = torch.from_numpy(U0.copy()).cuda()
    want = U0
    dg = DGSEM(m, 3, "hllc")
    for _ in range(3):
        s.step(U, dt)
        want = prkm_step(dg.rhs, want, dt, fam, element_methods(m.cells[:, 0], fam.R))
    s.check()
    assert np.max(np.abs(U.cpu().numpy() - want)) / np.max(np.abs(want)) < 1e-12


@pytest.mark.parametrize("flux", ["hllc", "hll", "ec"])
@pytest.mark.parametrize("stored", [True, False])
def test_fused_reverse_stages_bitwise_equal_to_two_launches(flux, stored):
    # the reverse sweep of the step: face and volume adjoints of a stage in one launch (items dealt
    # from a counter) against two launches on two streams; disjoint outputs, so bit for bit
    cells = nested_band_cells()
    U0 = torch.from_numpy(nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)).cuda()
    lam = torch.from_numpy(np.random.default_rng(41).normal(size=tuple(U0.shape))).cuda()
    out = []
    for fused in (True, False):
        s = solver(cells, fused, flux=flux)
        dt = s.compute_dt(U0, 0.7)
        if stored:
            K = torch.empty((s.S,) + tuple(U0.shape), dtype=U0.dtype, device=U0.device)
            U1 = U0.clone()
            s.step_store(U1, dt, stages=K)
            r = s.step_vjp(U0, dt, lam, stages=K)
        else:
            r = s.step_vjp(U0, dt, lam)
        s.check()
        out.append(r)
    assert torch.isfinite(out[0]).all()
    assert torch.equal(out[0], out[1])


def test_step_autotuner_keeps_state_and_results():
    # the tuner times whole steps from U without changing it; the mode it keeps gives the same
    # bits as any other mode
    cells = kh_band_cells(4, 7, 0.03)
    U0 = torch.from_numpy(nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)).cuda()
    s = solver(cells, 1)
    dt = s.compute_dt(U0, 0.7)
    U = U0.clone()
    mode = s.autotune_step(U, dt)
    assert mode in (0, 1, 2)
    assert torch.equal(U, U0)
    for _ in range(3):
        s.step(U, dt)
    s.check()
    ref = solver(cells, 0)
    V = U0.clone()
    for _ in range(3):
        ref.step(V, dt)
    ref.check()
    assert torch.equal(U, V)
