"""Caller-owned workspace (perk_workspace_bytes / perk_bind_workspace) on the GPU.

A context bound to a torch tensor must compute exactly what an unbound context computes (same
kernels on the same data: bitwise equal), and must make no device allocation of its own after
the bind while it uploads meshes, partitions, steps, computes step sizes, tunes and adapts."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from perk_inputs import kelvin_helmholtz, nodal_state, shear_layer, uniform_cells
from tests.gpu_common import X3

pytestmark = pytest.mark.gpu

AMR = dict(level_min=3, level_max=5, refine_above=0.1, coarsen_below=0.02)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_05144_gb300.build import build
    build()


def kh_run(solver, cycles=3, steps_per_cycle=4):
    """A short dynamic Kelvin-Helmholtz run: AMR, step size, steps; returns the final state."""
    solver.upload_mesh(uniform_cells(3), -1.0, 2.0)
    solver.set_perk2_disk([4, 6, 10, 16])
    U = torch.from_numpy(nodal_state(kelvin_helmholtz, uniform_cells(3), -1.0, 2.0, X3)).cuda()
    for _ in range(cycles):
        U = solver.adapt(U, **AMR)
        dt = solver.compute_dt(U, 0.7)
        for _ in range(steps_per_cycle):
            solver.step(U, dt)
    solver.check()
    return U, solver.cells.copy()


def test_bound_workspace_matches_unbound_and_allocates_nothing():
    from paper_2403_05144_gb300 import PerkSolver
    ref = PerkSolver(surface_flux="hllc", use_graph=True)
    U_ref, cells_ref = kh_run(ref)

    s = PerkSolver(surface_flux="hllc", use_graph=True)
    s.upload_mesh(uniform_cells(3), -1.0, 2.0)
    s.set_perk2_disk([4, 6, 10, 16])
    need = s.workspace_bytes(4 ** 5)            # every cell of level 5 at most
    assert need >= s.workspace_bytes() > 0
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    s.bind_workspace(ws)
    before = s.counters()["device_allocations"]
    U, cells = kh_run(s)
    s.autotune(U)
    s.compute_dt_members(U, 0.7)
    assert s.counters()["device_allocations"] == before
    assert np.array_equal(cells, cells_ref)
    assert torch.equal(U, U_ref)
    # back to the library's own memory: the same results again
    s.bind_workspace(None)
    U2, _ = kh_run(s)
    assert torch.equal(U2, U_ref)


def test_workspace_too_small_is_refused_before_any_work():
    from paper_2403_05144_gb300 import PerkError, PerkSolver
    s = PerkSolver(surface_flux="hllc")
    cells = uniform_cells(3)
    s.upload_mesh(cells, -1.0, 2.0)
    s.set_perk2_disk([4, 8])
    with pytest.raises(PerkError) as ei:                       # smaller than the current mesh needs
        s.bind_workspace(torch.empty(s.workspace_bytes() - 4096, dtype=torch.uint8, device="cuda"))
    assert ei.value.status == 1
    ws = torch.empty(s.workspace_bytes(len(cells)), dtype=torch.uint8, device="cuda")
    s.bind_workspace(ws)
    U = torch.from_numpy(nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)).cuda()
    with pytest.raises(PerkError) as ei:                       # a finer mesh does not fit
        s.upload_mesh(uniform_cells(4), -1.0, 2.0)
    assert ei.value.status == 6
    # the context still holds its mesh and steps as before
    ref = PerkSolver(surface_flux="hllc")
    ref.upload_mesh(cells, -1.0, 2.0)
    ref.set_perk2_disk([4, 8])
    V = U.clone()
    dt = ref.compute_dt(U, 0.5)
    s.step(U, dt)
    ref.step(V, dt)
    s.check()
    assert torch.equal(U, V)


def test_workspace_for_navier_stokes_and_stage_patterns():
    from paper_2403_05144_gb300 import PerkSolver, perk3_disk_tableau
    cells = uniform_cells(4)
    out = []
    for bind in (False, True):
        s = PerkSolver(surface_flux="hll", equations="navier_stokes", mu=1.0 / 2500.0, prandtl=0.72)
        s.upload_mesh(cells, 0.0, 1.0)
        c, a = perk3_disk_tableau([4, 8, 16])
        s.set_tableau(3, [4, 8, 16], c, a)
        if bind:
            ws = torch.empty(s.workspace_bytes(), dtype=torch.uint8, device="cuda")
            s.bind_workspace(ws)
            n0 = s.counters()["device_allocations"]
        U = torch.from_numpy(nodal_state(shear_layer, cells, 0.0, 1.0, X3)).cuda()
        dt = s.compute_dt(U, 0.5)
        for _ in range(3):
            s.step(U, dt)
        s.check()
        if bind:
            assert s.counters()["device_allocations"] == n0
        out.append(U)
    assert torch.equal(out[0], out[1])
    # a stage pattern keeps every stage: the layout grows, and an older binding is refused
    s = PerkSolver(surface_flux="hllc")
    s.upload_mesh(cells, -1.0, 2.0)
    s.set_perk2_disk([4, 8])
    small = s.workspace_bytes()
    ws = torch.empty(small, dtype=torch.uint8, device="cuda")
    s.bind_workspace(ws)
    s.set_perk2_pattern([4, 8], "early")
    assert s.workspace_bytes() > small
    U = torch.from_numpy(nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)).cuda()
    from paper_2403_05144_gb300 import PerkError
    with pytest.raises(PerkError) as ei:
        s.step(U, 1e-3)
    assert ei.value.status == 6
    ws2 = torch.empty(s.workspace_bytes(), dtype=torch.uint8, device="cuda")
    s.bind_workspace(ws2)
    n0 = s.counters()["device_allocations"]
    s.step(U, 1e-3)
    s.check()
    assert s.counters()["device_allocations"] == n0
