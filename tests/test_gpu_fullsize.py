"""Parity at the benchmark's full sizes, in the launch configuration bench.py times (CUDA-graph
replay, default launch shapes):

* one P-ERK2 {4,6,10,16} step on the initially adapted Kelvin-Helmholtz mesh (3,904 cells,
  levels 4-7) against the oracle's dense step, every output;
* the Navier-Stokes shear layer on its initially adapted three-level mesh (6,400 cells), the
  partitioned right-hand side of three stages against the oracle's masked full one, for the
  low-Mach initial state (measured against the scale of its cancelling derivative terms) and for
  a seeded state without cancellation (1e-12 relative per conserved variable);
* the 64-member Kelvin-Helmholtz ensemble (autotuned volume blocks, per-member dt, an AMR cycle):
  sampled members against the oracle's dense steps and, after the AMR cycle, bit for bit
  against the same members run alone;
* the discrete adjoint over 200 steps on the frozen three-level Kelvin-Helmholtz mesh at t = 1
  (about 219k DoF, checkpoints every 20 steps) against central differences along 16 seeded
  directions (a property that holds at any size; the adjoint itself is checked against the
  oracle's reverse sweep on small meshes).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.amr import desired_levels, indicator, new_cells
from oracle.br1 import NavierStokesDGSEM
from oracle.dgsem import DGSEM
from oracle.perk import element_methods, perk2_family, prkm_step
from oracle.lgl import lgl_nodes_weights
from oracle.treemesh import TreeMesh
from perk_inputs import kelvin_helmholtz, nodal_state, shear_layer, uniform_cells
from tests.gpu_common import X3, discontinuous_state, rel_err_per_var

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_05144_gb300.build import build
    build()


def initially_adapted(ic, base, x0, L, amr, kind, cycles):
    """The benchmark's initial mesh: adaptation cycles on the initial state itself."""
    cells = uniform_cells(base)
    for _ in range(cycles):
        m = TreeMesh(cells, x0, L)
        U = nodal_state(ic, cells, x0, L, X3)
        cells = new_cells(m, desired_levels(m, indicator(U, kind=kind), **amr))
    return cells


def test_kelvin_helmholtz_step_at_bench_size():
    from paper_2403_05144_gb300 import PerkSolver
    cells = initially_adapted(kelvin_helmholtz, 4, -1.0, 2.0,
                              dict(level_min=4, level_max=7, refine_above=0.1, coarsen_below=0.02), "density", 3)
    assert len(cells) == 3904
    U0 = nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)
    E = [4, 6, 10, 16]
    s = PerkSolver(surface_flux="hllc", use_graph=True)
    s.upload_mesh(cells, -1.0, 2.0)
    s.set_perk2_disk(E)
    U = torch.from_numpy(U0.copy()).cuda()
    dt = s.compute_dt(U, 0.7)
    s.step(U, dt)
    s.check()
    m = TreeMesh(cells, -1.0, 2.0)
    fam = perk2_family(E)
    want = prkm_step(DGSEM(m, 3, "hllc").rhs, U0, dt, fam, element_methods(m.cells[:, 0], fam.R))
    got = U.cpu().numpy()
    # per-RHS differences of ~1e-13 pass through 16 stages (|dt lambda| up to ~30)
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 1e-11


def test_shear_layer_partitioned_rhs_at_bench_size():
    from paper_2403_05144_gb300 import PerkSolver, perk3_disk_tableau
    cells = initially_adapted(shear_layer, 6, 0.0, 1.0,
                              dict(level_min=6, level_max=8, refine_above=0.1, coarsen_below=0.02), "lohner_vx", 2)
    assert len(cells) == 6400
    U = nodal_state(shear_layer, cells, 0.0, 1.0, X3)
    E = [4, 8, 16]
    s = PerkSolver(surface_flux="hll", equations="navier_stokes", mu=1.0 / 2500.0, prandtl=0.72)
    s.upload_mesh(cells, 0.0, 1.0)
    c, a = perk3_disk_tableau(E)
    s.set_tableau(3, E, c, a)
    m = TreeMesh(cells, 0.0, 1.0)
    fam = perk2_family(E)                    # the members' activity pattern is the same at third order
    meth = element_methods(m.cells[:, 0], fam.R)
    full = NavierStokesDGSEM(m, 3, "hll", mu=1.0 / 2500.0, prandtl=0.72).rhs(U)
    # The right-hand side is a sum of derivative terms of size up to (2/h) |f(u)|.  In this
    # low-Mach state they cancel almost completely: the pressure (~7.9) has no gradient at t = 0
    # and the density RHS vanishes analytically (rho = 1, v_x depends on y only, v_y on x only),
    # so what remains (momentum RHS <= 5, density RHS ~1e-13) is far below the terms whose
    # rounding it carries (~1e-11 absolute).  Errors are therefore measured against the scale of
    # the derivative terms, (2/h_min) max |u|; a wrong term would be 1e-3 of that, not 1e-12.
    scale = (2.0 / m.h.min()) * np.max(np.abs(U))
    for i in (0, 9, 15):
        active = np.array([fam.active(int(r), i) for r in meth])
        got = s.rhs_active(i, torch.from_numpy(U).cuda(),
                           out=torch.from_numpy(np.full_like(U, 7.0)).cuda()).cpu().numpy()
        assert np.all(got[~active] == 7.0)
        assert np.max(np.abs(got[active] - full[active])) / scale < 1e-12, i
        # and against the RHS itself where it is not a cancellation remainder (energy)
        assert np.max(np.abs(got[active][:, 3] - full[active][:, 3])) / np.max(np.abs(full[:, 3])) < 1e-10
    # A seeded state without that cancellation on the same mesh, viscosity and tableau: here every
    # variable's RHS is of the size of its derivative terms, and the parity bound is the plain one,
    # 1e-12 relative per conserved variable on the active elements of each stage.
    V = discontinuous_state(cells, 0.0, 1.0, seed=23)
    fullV = NavierStokesDGSEM(m, 3, "hll", mu=1.0 / 2500.0, prandtl=0.72).rhs(V)
    for i in (0, 9, 15):
        active = np.array([fam.active(int(r), i) for r in meth])
        got = s.rhs_active(i, torch.from_numpy(V).cuda(),
                           out=torch.from_numpy(np.full_like(V, 7.0)).cuda()).cpu().numpy()
        assert np.all(got[~active] == 7.0)
        assert rel_err_per_var(got[active], fullV[active]) < 1e-12, i


KH_AMR = dict(refine_above=0.1, coarsen_below=0.02)


def ensemble_members(n=64, seed=20240308 + 4):
    """The benchmark's ensemble: seeded amplitude U(0.05, 0.15), wavenumber 2 or 4, finest level 6
    or 7; each member's mesh from three adaptation cycles (oracle) on its own initial state."""
    import functools
    rng = np.random.default_rng(seed)
    amps = rng.uniform(0.05, 0.15, n)
    ks = rng.choice([2, 4], n)
    lmaxs = rng.choice([6, 7], n)
    ics = [functools.partial(kelvin_helmholtz, amplitude=float(a), wavenumber=int(k)) for a, k in zip(amps, ks)]
    cache = {}
    meshes = []
    for ic, lm, k in zip(ics, lmaxs, ks):
        key = (int(lm), int(k))
        if key not in cache:
            cache[key] = initially_adapted(ic, 4, -1.0, 2.0, dict(KH_AMR, level_min=4, level_max=int(lm)), "density", 3)
        meshes.append(cache[key])
    states = [nodal_state(ic, c, -1.0, 2.0, X3) for ic, c in zip(ics, meshes)]
    return meshes, states


def test_ensemble_at_bench_size():
    from paper_2403_05144_gb300 import PerkSolver
    E = [4, 6, 10, 16]
    meshes, states = ensemble_members()
    sizes = [len(c) for c in meshes]
    assert len(meshes) == 64 and min(sizes) < max(sizes)
    ens = PerkSolver(surface_flux="hllc", use_graph=True)
    ens.upload_ensemble(meshes, -1.0, 2.0)
    ens.set_perk2_disk(E)
    Ue = torch.from_numpy(np.concatenate(states)).cuda()
    ens.autotune(Ue)
    dts = ens.compute_dt_members(Ue, 0.7)
    # sampled members: the first of the smallest and of the largest meshes
    sample = [int(np.argmin(sizes)), int(np.argmax(sizes))]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    solo = {}
    for m in sample:
        s = PerkSolver(surface_flux="hllc", use_graph=True)
        s.upload_mesh(meshes[m], -1.0, 2.0)
        s.set_perk2_disk(E)
        solo[m] = (s, torch.from_numpy(states[m].copy()).cuda())
    fam = perk2_family(E)
    for _ in range(2):
        ens.step(Ue, dts)
        for m, (s, U) in solo.items():
            s.step(U, dts[m])
    ens.check()
    got = Ue.cpu().numpy()
    for m in sample:
        mesh = TreeMesh(meshes[m], -1.0, 2.0)
        meth = element_methods(mesh.cells[:, 0], fam.R)
        rhs = DGSEM(mesh, 3, "hllc").rhs
        want = states[m]
        for _ in range(2):
            want = prkm_step(rhs, want, dts[m], fam, meth)
        part = got[offs[m]:offs[m + 1]]
        assert np.max(np.abs(part - want)) / np.max(np.abs(want)) < 1e-11, m
    # an AMR cycle of the whole ensemble, then two more steps: equal to the members run alone
    amr = dict(KH_AMR, level_min=4, level_max=7)
    Ue = ens.adapt(Ue, **amr)
    dts = ens.compute_dt_members(Ue, 0.7)
    mem = ens.members()
    for m in sample:
        s, U = solo[m]
        U = s.adapt(U, **amr)
        assert s.compute_dt(U, 0.7) == dts[m]
        assert np.array_equal(ens.cells[mem == m], s.cells)
        solo[m] = (s, U)
    for _ in range(2):
        ens.step(Ue, dts)
        for m, (s, U) in solo.items():
            s.step(U, dts[m])
    ens.check()
    got = Ue.cpu().numpy()
    for m, (s, U) in solo.items():
        assert np.array_equal(got[mem == m], U.cpu().numpy()), m


def test_adjoint_at_bench_size():
    from paper_2403_05144_gb300 import PerkSolver, perk2_disk_tableau
    from paper_2403_05144_gb300.adjoint import gradient, kinetic_energy
    # the Kelvin-Helmholtz run on base level 6 with AMR between levels 6 and 8 every 5 steps, to t = 1
    amr = dict(KH_AMR, level_min=6, level_max=8)
    run = PerkSolver(surface_flux="hllc", use_graph=True)
    run.upload_mesh(uniform_cells(6), -1.0, 2.0)
    run.set_perk2_disk([4, 6, 10, 16])
    U = torch.from_numpy(nodal_state(kelvin_helmholtz, run.cells, -1.0, 2.0, X3)).cuda()
    for _ in range(3):
        run.adapt(U, **amr)
        U = torch.from_numpy(nodal_state(kelvin_helmholtz, run.cells, -1.0, 2.0, X3)).cuda()
    t, k = 0.0, 0
    dt = run.compute_dt(U, 0.7)
    while t < 1.0:
        if k > 0 and k % 5 == 0:
            U = run.adapt(U, **amr)
            dt = run.compute_dt(U, 0.7)
        run.step(U, dt)
        t += dt
        k += 1
    run.check()
    cells, U0 = run.cells.copy(), U.clone()
    assert len(set(cells[:, 0].tolist())) == 3 and 150_000 < 16 * len(cells) < 300_000
    s = PerkSolver(surface_flux="hllc", use_graph=True)
    s.upload_mesh(cells, -1.0, 2.0)
    c, a = perk2_disk_tableau([6, 10, 16])
    s.set_tableau(2, [6, 10, 16], c, a)
    dt = s.compute_dt(U0, 0.7)
    h = torch.tensor(2.0 / 2.0 ** cells[:, 0], dtype=torch.float64, device="cuda")
    w = torch.tensor(lgl_nodes_weights(3)[1], device="cuda")
    J = lambda V: kinetic_energy(V, h, w)
    n = 200
    _, grad = gradient(s, U0, dt, n, J, checkpoint_every=20)

    def J_of(V):
        V = V.clone()
        for _ in range(n):
            s.step(V, dt)
        s.check()
        return float(J(V))

    rng = np.random.default_rng(20240308 + 5)
    for q in range(16):
        d = torch.from_numpy(rng.normal(size=U0.shape)).cuda() * U0.abs()
        d = d / torch.linalg.vector_norm(d)
        eps = 1e-6 * float(torch.linalg.vector_norm(U0))
        fd = (J_of(U0 + eps * d) - J_of(U0 - eps * d)) / (2 * eps)
        ad = float(torch.sum(grad * d))
        assert abs(fd - ad) <= 1e-6 * abs(fd), (q, fd, ad)
