"""Ensembles: independent meshes advanced by one context (one launch per kernel
and stage for all members) agree bit for bit with each member run alone, for
steps with per-member step sizes and for AMR cycles."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from perk_inputs import kelvin_helmholtz, kh_band_cells, nodal_state, uniform_cells, vortex_two_level_cells
from tests.gpu_common import X3

pytestmark = pytest.mark.gpu

E = [4, 6, 10, 16]
AMR = dict(level_min=3, level_max=6, refine_above=0.1, coarsen_below=0.02)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_05144_gb300.build import build
    build()


def members():
    meshes = [kh_band_cells(3, 6, 0.05), vortex_two_level_cells(3, 2, 6), uniform_cells(3), kh_band_cells(4, 5, 0.1)]
    params = [(0.1, 2), (0.05, 4), (0.15, 2), (0.08, 4)]
    states = [nodal_state(kelvin_helmholtz, c, -1.0, 2.0, X3, amplitude=a, wavenumber=k) for c, (a, k) in zip(meshes, params)]
    return meshes, states


def single(cells, U0):
    from paper_2403_05144_gb300 import PerkSolver
    s = PerkSolver(surface_flux="hllc", use_graph=True)
    s.upload_mesh(cells, -1.0, 2.0)
    s.set_perk2_disk(E)
    return s, torch.from_numpy(U0.copy()).cuda()


def test_ensemble_steps_equal_single_runs():
    from paper_2403_05144_gb300 import PerkSolver
    meshes, states = members()
    ens = PerkSolver(surface_flux="hllc", use_graph=True)
    ens.upload_ensemble(meshes, -1.0, 2.0)
    ens.set_perk2_disk(E)
    Ue = torch.from_numpy(np.concatenate(states)).cuda()
    dts = ens.compute_dt_members(Ue, 0.7)
    solo = [single(c, U) for c, U in zip(meshes, states)]
    for (s, U), dt in zip(solo, dts):
        assert s.compute_dt(U, 0.7) == dt
    info = ens.info()
    assert info["n_elem"] == sum(len(c) for c in meshes)
    assert info["dof_stage_updates"] == sum(s.info()["dof_stage_updates"] for s, _ in solo)
    for _ in range(6):
        ens.step(Ue, dts)
        for (s, U), dt in zip(solo, dts):
            s.step(U, dt)
    ens.check()
    want = torch.cat([U for _, U in solo]).cpu().numpy()
    assert np.array_equal(Ue.cpu().numpy(), want)


def test_ensemble_amr_equals_single_amr():
    from paper_2403_05144_gb300 import PerkSolver
    meshes, states = members()
    ens = PerkSolver(surface_flux="hllc", use_graph=True)
    ens.upload_ensemble(meshes, -1.0, 2.0)
    ens.set_perk2_disk(E)
    Ue = torch.from_numpy(np.concatenate(states)).cuda()
    solo = [single(c, U) for c, U in zip(meshes, states)]
    for cycle in range(2):
        Ue = ens.adapt(Ue, **AMR)
        dts = ens.compute_dt_members(Ue, 0.7)
        new = []
        for (s, U), dt in zip(solo, dts):
            U = s.adapt(U, **AMR)
            assert s.compute_dt(U, 0.7) == dt
            new.append((s, U))
        solo = new
        mem = ens.members()
        for m, (s, U) in enumerate(solo):
            assert np.array_equal(ens.cells[mem == m], s.cells)
        for _ in range(3):
            ens.step(Ue, dts)
            for (s, U), dt in zip(solo, dts):
                s.step(U, dt)
    want = torch.cat([U for _, U in solo]).cpu().numpy()
    assert np.array_equal(Ue.cpu().numpy(), want)
