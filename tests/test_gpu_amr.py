"""GPU parity of the AMR path (indicator, planned mesh, transfer, dynamic run) with the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.amr import adapt as oracle_adapt
from oracle.amr import balance, indicator, new_cells, transfer
from oracle.dgsem import DGSEM
from oracle.perk import element_methods, max_wave_speed_dt, perk2_family, prkm_step
from oracle.treemesh import TreeMesh
from perk_inputs import kelvin_helmholtz, kh_band_cells, nodal_state, uniform_cells
from tests.gpu_common import X3, discontinuous_state, solver_for

pytestmark = pytest.mark.gpu
AMR = dict(level_min=4, level_max=7, refine_above=0.1, coarsen_below=0.02)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_05144_gb300.build import build
    build()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_indicator_parity():
    cells = kh_band_cells(4, 6, 0.05)
    U = discontinuous_state(cells, -1.0, 2.0)
    s = solver_for(cells, -1.0, 2.0, "hllc")
    got = s.amr_indicator(cuda(U)).cpu().numpy()
    np.testing.assert_allclose(got, indicator(U), rtol=1e-12)


def test_lohner_indicator_parity_bitwise():
    # the kernel evaluates the estimator in the oracle's operation order with
    # round-to-nearest operations, so the values agree bit for bit
    cells = kh_band_cells(4, 6, 0.05)
    U = discontinuous_state(cells, -1.0, 2.0)
    s = solver_for(cells, -1.0, 2.0, "hllc")
    got = s.amr_indicator(cuda(U), indicator="lohner_vx").cpu().numpy()
    want = indicator(U, kind="lohner_vx")
    assert np.array_equal(got, want)
    assert want.max() > 0.1


def test_lohner_driven_cycles_on_the_shear_layer_match_oracle():
    from perk_inputs import shear_layer
    cells = uniform_cells(4)
    U = nodal_state(shear_layer, cells, 0.0, 1.0, X3)
    s = solver_for(cells, 0.0, 1.0, "hll")
    m = TreeMesh(cells, 0.0, 1.0)
    Ug = cuda(U)
    prm = dict(level_min=4, level_max=6, refine_above=0.3, coarsen_below=0.05)
    for _ in range(3):
        m, U, _ = oracle_adapt(m, U, **prm, kind="lohner_vx")
        Ug = s.adapt(Ug, **prm, indicator="lohner_vx")
        assert [tuple(c) for c in s.cells.tolist()] == [tuple(c) for c in m.cells.tolist()]
        np.testing.assert_allclose(Ug.cpu().numpy(), U, rtol=0, atol=1e-13 * np.max(np.abs(U)))
    assert m.cells[:, 0].max() == 6


def test_plan_and_transfer_match_oracle_with_given_levels():
    cells = kh_band_cells(4, 6, 0.05)
    m = TreeMesh(cells, -1.0, 2.0)
    U = discontinuous_state(cells, -1.0, 2.0)
    rng = np.random.default_rng(4)
    lev = m.cells[:, 0]
    raw = np.clip(lev + rng.integers(-1, 2, size=len(lev)), 4, 7)
    want_d = balance(m, raw)
    want_cells = new_cells(m, want_d)
    want_U = transfer([tuple(c) for c in cells], U, want_cells)
    s = solver_for(cells, -1.0, 2.0, "hllc", [4, 6, 10, 16])
    Unew = s.adapt(cuda(U), desired=raw).cpu().numpy()
    assert [tuple(c) for c in s.cells.tolist()] == want_cells
    np.testing.assert_allclose(Unew, want_U, rtol=0, atol=1e-13 * np.max(np.abs(want_U)))
    info = s.info()
    assert info["n_elem"] == len(want_cells)


def test_indicator_driven_cycle_matches_oracle():
    cells = uniform_cells(4)
    U = nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)
    s = solver_for(cells, -1.0, 2.0, "hllc", [4, 6, 10, 16])
    m = TreeMesh(cells, -1.0, 2.0)
    Ug = cuda(U)
    for _ in range(3):
        m, U, _ = oracle_adapt(m, U, **AMR)
        Ug = s.adapt(Ug, **AMR)
        assert [tuple(c) for c in s.cells.tolist()] == [tuple(c) for c in m.cells.tolist()]
        np.testing.assert_allclose(Ug.cpu().numpy(), U, rtol=0, atol=1e-13 * np.max(np.abs(U)))


def test_dynamic_kh_run_with_replayed_decisions():
    # 15 P-ERK2 {4,6,10,16} steps with an AMR cycle every 5 steps; the GPU takes
    # the oracle's raw desired levels so both meshes stay identical
    cells = kh_band_cells(4, 6, 0.05)
    m = TreeMesh(cells, -1.0, 2.0)
    U = nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)
    fam = perk2_family([4, 6, 10, 16])
    dt = max_wave_speed_dt(U, m.h, 3, 0.7)
    s = solver_for(cells, -1.0, 2.0, "hllc", [4, 6, 10, 16])
    Ug = cuda(U)
    for k in range(15):
        if k > 0 and k % 5 == 0:
            eta = indicator(U)
            lev = m.cells[:, 0]
            raw = lev.copy()
            raw[(eta > AMR["refine_above"]) & (lev < 7)] += 1
            raw[(eta < AMR["coarsen_below"]) & (lev > 4)] -= 1
            m, U, _ = oracle_adapt(m, U, **AMR, desired=balance(m, raw))
            Ug = s.adapt(Ug, desired=raw)
        dg = DGSEM(m, 3, "hllc")
        U = prkm_step(dg.rhs, U, dt, fam, element_methods(m.cells[:, 0], fam.R))
        s.step(Ug, dt)
    s.check()
    got = Ug.cpu().numpy()
    assert np.max(np.abs(got - U)) / np.max(np.abs(U)) < 1e-10


def test_device_built_mesh_equals_a_fresh_upload():
    # after each indicator-driven cycle (plan, balance, new leaves, connectivity and partition on
    # the device) the context must hold exactly what uploading the same leaves builds on the host:
    # the same counts per stage and bitwise the same right-hand side (a wrong neighbour or mortar
    # would change it)
    from paper_2403_05144_gb300 import _lib
    cells = uniform_cells(4)
    U = cuda(nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3))
    s = solver_for(cells, -1.0, 2.0, "hllc", [4, 6, 10, 16])
    for cycle in range(4):
        U = s.adapt(U, **AMR)
        fresh = solver_for(s.cells, -1.0, 2.0, "hllc", [4, 6, 10, 16])
        a, b = s.info(), fresh.info()
        for k in ("n_elem", "n_interfaces", "n_mortars", "level_min", "level_max", "active_elements",
                  "active_interfaces", "active_mortars", "dof_stage_updates"):
            assert a[k] == b[k], (cycle, k)
        assert torch.equal(s.rhs_full(U), fresh.rhs_full(U))
        for i in (0, 7, 15):
            assert torch.equal(s.rhs_active(i, U, out=torch.zeros_like(U)), fresh.rhs_active(i, U, out=torch.zeros_like(U)))
    assert s.info()["level_max"] == 7 and s.info()["n_mortars"] > 0


def test_unsorted_upload_is_planned_on_the_host_then_matches_oracle():
    # a leaf list not in Morton order takes the host plan (its result is in Morton order, after
    # which plans run on the device); both cycles match the oracle's meshes and transfer
    cells = kh_band_cells(4, 6, 0.05)
    perm = np.random.default_rng(9).permutation(len(cells))
    shuffled = [cells[k] for k in perm]
    U = discontinuous_state(shuffled, -1.0, 2.0)
    m = TreeMesh(shuffled, -1.0, 2.0)
    s = solver_for(shuffled, -1.0, 2.0, "hllc", [4, 6, 10, 16])
    Ug = cuda(U)
    rng = np.random.default_rng(5)
    for _ in range(2):
        lev = m.cells[:, 0]
        raw = np.clip(lev + rng.integers(-1, 2, size=len(lev)), 4, 7)
        want_cells = new_cells(m, balance(m, raw))
        U = transfer([tuple(c) for c in m.cells.tolist()], U, want_cells)
        m = TreeMesh(want_cells, -1.0, 2.0)
        Ug = s.adapt(Ug, desired=raw)
        assert [tuple(c) for c in s.cells.tolist()] == want_cells
        np.testing.assert_allclose(Ug.cpu().numpy(), U, rtol=0, atol=1e-13 * np.max(np.abs(U)))


def test_step_size_read_back_with_the_partition():
    # adapt(..., cfl) computes the new state's step size with the partition's readback: the same
    # value as compute_dt on the new state, also on a cycle that changes nothing
    cells = uniform_cells(4)
    U = cuda(nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3))
    s = solver_for(cells, -1.0, 2.0, "hllc", [4, 6, 10, 16])
    for cycle in range(3):
        U = s.adapt(U, cfl=0.7, **AMR)
        assert s.last_dt == s.compute_dt(U, 0.7), cycle
    frozen = dict(AMR, refine_above=1e30, coarsen_below=-1.0)   # no cell changes level
    n = s.info()["n_elem"]
    U = s.adapt(U, cfl=0.7, **frozen)
    assert s.info()["n_elem"] == n and s.last_dt == s.compute_dt(U, 0.7)
