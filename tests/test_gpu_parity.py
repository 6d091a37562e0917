"""GPU parity of libperk's kernels (through the C ABI) with the CPU oracle.

Tolerances: per right-hand-side call 1e-12 relative per conserved variable,
after many steps 1e-10 relative (infinity norms), bit-exact for the integer
partition counts."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.dgsem import DGSEM
from oracle.perk import element_methods, max_wave_speed_dt, perk2_family, prkm_step
from oracle.treemesh import TreeMesh
from perk_inputs import (isentropic_vortex, kelvin_helmholtz, kh_band_cells, nested_band_cells, nodal_state,
                         uniform_cells, vortex_two_level_cells)
from tests.gpu_common import X3, discontinuous_state, rel_err_per_var, solver_for

pytestmark = pytest.mark.gpu

VORTEX = dict(x0=-10.0, L=20.0)
KH = dict(x0=-1.0, L=2.0)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_05144_gb300.build import build
    build()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


MESHES = {
    "vortex448": (lambda: vortex_two_level_cells(), VORTEX),
    "ragged76": (lambda: vortex_two_level_cells(3, 3, 5), VORTEX),
    "kh4lev": (lambda: kh_band_cells(4, 6, 0.05), KH),
    "uniform16": (lambda: uniform_cells(2), KH),
    "single": (lambda: [(0, 0, 0)], KH),
}


@pytest.mark.parametrize("flux", ["hll", "hllc", "ec"])
@pytest.mark.parametrize("mesh", list(MESHES))
def test_rhs_full(flux, mesh):
    cells_fn, dom = MESHES[mesh]
    cells = cells_fn()
    U = discontinuous_state(cells, dom["x0"], dom["L"])
    s = solver_for(cells, dom["x0"], dom["L"], flux)
    got = s.rhs_full(cuda(U)).cpu().numpy()
    want = DGSEM(TreeMesh(cells, dom["x0"], dom["L"]), 3, flux).rhs(U)
    assert rel_err_per_var(got, want) < 1e-12


@pytest.mark.parametrize("E", [[4, 8], [4, 6, 10, 16]])
def test_rhs_active_every_stage(E):
    cells = kh_band_cells(4, 6, 0.05)
    dom = KH
    U = discontinuous_state(cells, dom["x0"], dom["L"])
    s = solver_for(cells, dom["x0"], dom["L"], "hllc", E)
    mesh = TreeMesh(cells, dom["x0"], dom["L"])
    fam = perk2_family(E)
    meth = element_methods(mesh.cells[:, 0], fam.R)
    full = DGSEM(mesh, 3, "hllc").rhs(U)
    info = s.info()
    for i in range(fam.S):
        active = np.array([fam.active(int(r), i) for r in meth])
        assert info["active_elements"][i] == int(active.sum())
        sentinel = np.full_like(U, 7.0)
        got = s.rhs_active(i, cuda(U), out=cuda(sentinel)).cpu().numpy()
        assert np.all(got[~active] == 7.0)
        assert rel_err_per_var(got[active], full[active]) < 1e-12


def oracle_steps(cells, dom, E, U0, dt, n, flux="hll"):
    mesh = TreeMesh(cells, dom["x0"], dom["L"])
    fam = perk2_family(E)
    rhs = DGSEM(mesh, 3, flux).rhs
    meth = element_methods(mesh.cells[:, 0], fam.R)
    U = U0
    for _ in range(n):
        U = prkm_step(rhs, U, dt, fam, meth)
    return U


def gpu_steps(cells, dom, E, U0, dt, n, flux="hll", use_graph=True):
    s = solver_for(cells, dom["x0"], dom["L"], flux, E, use_graph)
    U = cuda(U0.copy())
    for _ in range(n):
        s.step(U, dt)
    s.check()
    return U.cpu().numpy(), s


def test_one_step_vortex448():
    cells = vortex_two_level_cells()
    U0 = nodal_state(isentropic_vortex, cells, -10.0, 20.0, X3)
    dt = max_wave_speed_dt(U0, TreeMesh(cells, -10.0, 20.0).h, 3, 0.5 * 7)
    got, _ = gpu_steps(cells, VORTEX, [4, 8], U0, dt, 1)
    want = oracle_steps(cells, VORTEX, [4, 8], U0, dt, 1)
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 1e-12


def test_twenty_steps_vortex448():
    # the two-level vortex workload: 448 cells, P-ERK2 {4, 8}, HLL, fixed CFL step, 20 steps
    cells = vortex_two_level_cells()
    U0 = nodal_state(isentropic_vortex, cells, -10.0, 20.0, X3)
    dt = max_wave_speed_dt(U0, TreeMesh(cells, -10.0, 20.0).h, 3, 0.5 * 7)
    got, s = gpu_steps(cells, VORTEX, [4, 8], U0, dt, 20)
    want = oracle_steps(cells, VORTEX, [4, 8], U0, dt, 20)
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 1e-10
    c = s.counters()
    assert c["steps"] == 20 and c["rejected_steps_checked"] == 0


def test_hundred_steps_vortex448():
    # the two-level vortex workload itself (448 cells, 32 mortars, P-ERK2 {4, 8}, HLL) for 100
    # steps against the oracle's dense partitioned step: 1e-10 relative after 100 steps
    cells = vortex_two_level_cells()
    U0 = nodal_state(isentropic_vortex, cells, -10.0, 20.0, X3)
    dt = max_wave_speed_dt(U0, TreeMesh(cells, -10.0, 20.0).h, 3, 0.5 * 7)
    got, s = gpu_steps(cells, VORTEX, [4, 8], U0, dt, 100)
    want = oracle_steps(cells, VORTEX, [4, 8], U0, dt, 100)
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 1e-10
    assert s.counters()["steps"] == 100


def test_hundred_steps_kh_four_levels():
    # Kelvin-Helmholtz state on a four-level mesh (levels 2-5, 184 cells) so that every member of
    # the P-ERK2 {4, 6, 10, 16} family (HLLC) owns cells: 100 steps at CFL 0.7 in the bench's
    # launch configuration (graph replay) against the oracle's dense step
    cells = nested_band_cells(2, 5)
    assert sorted({c[0] for c in cells}) == [2, 3, 4, 5]
    E = [4, 6, 10, 16]
    U0 = nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)
    dt = max_wave_speed_dt(U0, TreeMesh(cells, -1.0, 2.0).h, 3, 0.7)
    got, s = gpu_steps(cells, KH, E, U0, dt, 100, "hllc")
    info = s.info()
    assert info["active_elements"][0] == len(cells) and info["active_elements"][15] == len(cells)
    assert min(info["active_elements"][:16]) == sum(1 for c in cells if c[0] == 5)
    want = oracle_steps(cells, KH, E, U0, dt, 100, "hllc")
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 1e-10


def test_hundred_steps_small_mesh():
    cells = vortex_two_level_cells(3, 2, 6)
    U0 = nodal_state(isentropic_vortex, cells, -10.0, 20.0, X3)
    dt = max_wave_speed_dt(U0, TreeMesh(cells, -10.0, 20.0).h, 3, 0.5 * 7)
    got, _ = gpu_steps(cells, VORTEX, [4, 8], U0, dt, 100)
    want = oracle_steps(cells, VORTEX, [4, 8], U0, dt, 100)
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 1e-10


@pytest.mark.parametrize("E,flux", [([4, 6, 10, 16], "hllc"), ([4, 8], "hll"), ([8], "hll")])
def test_kh_step_four_levels(E, flux):
    # four levels; with two members the coarse levels clamp onto member 0
    cells = kh_band_cells(4, 7, 0.03)
    U0 = nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)
    dt = max_wave_speed_dt(U0, TreeMesh(cells, -1.0, 2.0).h, 3, 0.5 * (max(E) - 1))
    got, _ = gpu_steps(cells, KH, E, U0, dt, 2, flux)
    want = oracle_steps(cells, KH, E, U0, dt, 2, flux)
    # per-RHS differences of ~1e-12 pass through up to 16 stages per step with
    # |dt lambda| ~ 30, which amplifies them (observed 2.6e-12 after 2 steps):
    # few-step comparisons use 1e-11, the 100-step runs the 1e-10 bound
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 1e-11


def test_graph_replay_bitwise_equal_to_direct_launches():
    cells = vortex_two_level_cells()
    U0 = nodal_state(isentropic_vortex, cells, -10.0, 20.0, X3)
    dt = max_wave_speed_dt(U0, TreeMesh(cells, -10.0, 20.0).h, 3, 0.5)
    a, _ = gpu_steps(cells, VORTEX, [4, 8], U0, dt, 5, use_graph=True)
    b, _ = gpu_steps(cells, VORTEX, [4, 8], U0, dt, 5, use_graph=False)
    assert np.array_equal(a, b)


def test_nonadmissible_step_is_not_committed():
    from paper_2403_05144_gb300 import PerkError
    cells = vortex_two_level_cells(3, 2, 6)
    U0 = nodal_state(isentropic_vortex, cells, -10.0, 20.0, X3)
    U0[5, 3] = -1.0                        # negative energy: pressure < 0 after the step
    s = solver_for(cells, VORTEX["x0"], VORTEX["L"], "hll", [4, 8])
    U = cuda(U0.copy())
    s.step(U, 0.05)
    with pytest.raises(PerkError) as ei:
        s.check()
    assert ei.value.status == 3
    assert np.array_equal(U.cpu().numpy(), U0)
    s.check()                              # flag cleared


def test_dt_matches_oracle():
    cells = kh_band_cells(4, 6, 0.05)
    U0 = nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)
    s = solver_for(cells, KH["x0"], KH["L"], "hllc")
    want = max_wave_speed_dt(U0, TreeMesh(cells, -1.0, 2.0).h, 3, 0.7)
    assert s.compute_dt(cuda(U0), 0.7) == pytest.approx(want, rel=1e-14)


@pytest.mark.parametrize("bad", ["negative_density", "negative_pressure", "nan"])
def test_dt_refuses_inadmissible_states(bad):
    # the oracle's step size is NaN when a node has rho <= 0, p <= 0 or a NaN entry; the library
    # reports NONFINITE instead of a step size taken from the other nodes
    from paper_2403_05144_gb300 import PerkError
    cells = vortex_two_level_cells(3, 2, 6)
    U0 = nodal_state(isentropic_vortex, cells, -10.0, 20.0, X3)
    if bad == "negative_density":
        U0[5, 0, 1, 2] = -0.5
    elif bad == "negative_pressure":
        U0[7, 3, 3, 0] = -1.0
    else:
        U0[9, 2, 0, 3] = np.nan
    assert np.isnan(max_wave_speed_dt(U0, TreeMesh(cells, -10.0, 20.0).h, 3, 0.5))
    s = solver_for(cells, VORTEX["x0"], VORTEX["L"], "hll")
    with pytest.raises(PerkError) as ei:
        s.compute_dt(cuda(U0), 0.5)
    assert ei.value.status == 3
    with pytest.raises(PerkError) as ei:
        s.compute_dt_members(cuda(U0), 0.5)
    assert ei.value.status == 3
    good = nodal_state(isentropic_vortex, cells, -10.0, 20.0, X3)
    assert s.compute_dt(cuda(good), 0.5) == pytest.approx(
        max_wave_speed_dt(good, TreeMesh(cells, -10.0, 20.0).h, 3, 0.5), rel=1e-14)


def test_partition_counts_match_oracle():
    cells = kh_band_cells(4, 7, 0.06)
    s = solver_for(cells, KH["x0"], KH["L"], "hllc", [4, 6, 10, 16])
    info = s.info()
    mesh = TreeMesh(cells, -1.0, 2.0)
    fam = perk2_family([4, 6, 10, 16])
    meth = element_methods(mesh.cells[:, 0], fam.R)
    for i in range(fam.S):
        want = sum(1 for r in meth if fam.active(int(r), i))
        assert info["active_elements"][i] == want
        # interfaces take their elements' member; mortars their fine side's
        wi = sum(1 for (A, B, d) in mesh.conforming if fam.active(int(meth[A]), i))
        assert info["active_interfaces"][i] == wi
        fine = {}
        for (A, B, d, large, half) in mesh.hanging:
            small = B if large == A else A
            fine[(large, d, large == A)] = meth[small]
        assert info["active_mortars"][i] == sum(1 for r in fine.values() if fam.active(int(r), i))
    assert info["dof_stage_updates"] == 16 * sum(info["active_elements"])


def test_volume_block_sizes_give_identical_steps():
    # the elements per block of the volume kernel change only the launch shape
    from paper_2403_05144_gb300 import PerkSolver
    cells = kh_band_cells(4, 6, 0.05)
    U0 = torch.from_numpy(nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)).cuda()
    outs = []
    for epb in (2, 4, 8):
        s = PerkSolver(surface_flux="hllc")
        s.upload_mesh(cells, -1.0, 2.0)
        s.set_perk2_disk([4, 6, 10, 16])
        s.set_volume_blocks(epb)
        U = U0.clone()
        dt = s.compute_dt(U, 0.5)
        for _ in range(3):
            s.step(U, dt)
        outs.append(U)
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    s = PerkSolver(surface_flux="hllc")
    s.upload_mesh(cells, -1.0, 2.0)
    s.set_perk2_disk([4, 6, 10, 16])
    assert s.autotune(U0) in (2, 4, 8)
    U = U0.clone()
    dt = s.compute_dt(U, 0.5)
    for _ in range(3):
        s.step(U, dt)
    assert torch.equal(U, outs[0])
    with pytest.raises(Exception):
        s.set_volume_blocks(3)


@pytest.mark.parametrize("b_S", [0.5, 0.75])
def test_heun_and_ralston_weighted_steps(b_S):
    # the weight variants of Sec. 3.1 (b_1 = 1 - b_S) against the oracle's dense step
    cells = vortex_two_level_cells()
    m = TreeMesh(cells, -10.0, 20.0)
    U0 = nodal_state(isentropic_vortex, cells, -10.0, 20.0, X3)
    fam = perk2_family([4, 8], b_S=b_S)
    meth = element_methods(m.cells[:, 0], fam.R)
    dt = max_wave_speed_dt(U0, m.h, 3, 0.4)
    s = solver_for(cells, -10.0, 20.0, "hll")
    s.set_perk2_disk([4, 8], b_S=b_S)
    U = torch.from_numpy(U0.copy()).cuda()
    want = U0
    dg = DGSEM(m, 3, "hll")
    for _ in range(3):
        s.step(U, dt)
        want = prkm_step(dg.rhs, want, dt, fam, meth)
    s.check()
    assert np.max(np.abs(U.cpu().numpy() - want)) / np.max(np.abs(want)) < 1e-12
