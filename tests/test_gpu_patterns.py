"""GPU parity of the stage patterns (Sec. 3.2.4: alternating and early-shared evaluations) with the
oracle's dense partitioned step."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.dgsem import DGSEM
from oracle.perk import element_methods, max_wave_speed_dt, perk2_family, prkm_step
from oracle.treemesh import TreeMesh
from perk_inputs import kelvin_helmholtz, kh_band_cells, nodal_state, vortex_two_level_cells
from tests.gpu_common import X3, discontinuous_state, rel_err_per_var, solver_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_05144_gb300.build import build
    build()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("E,pattern,cells_fn", [
    ([4, 6, 10, 16], "early", lambda: kh_band_cells(4, 7, 0.03)),
    ([6, 12], "alternating", lambda: kh_band_cells(4, 5, 0.1)),
    ([4, 8], "alternating", lambda: vortex_two_level_cells(3, 2, 6)),
])
def test_pattern_steps_match_oracle(E, pattern, cells_fn):
    cells = cells_fn()
    m = TreeMesh(cells, -1.0, 2.0)
    U0 = nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)
    fam = perk2_family(E, pattern=pattern)
    meth = element_methods(m.cells[:, 0], fam.R)
    dt = max_wave_speed_dt(U0, m.h, 3, 0.3)
    s = solver_for(cells, -1.0, 2.0, "hllc")
    s.set_perk2_pattern(E, pattern)
    U = cuda(U0)
    want = U0
    dg = DGSEM(m, 3, "hllc")
    for _ in range(3):
        s.step(U, dt)
        want = prkm_step(dg.rhs, want, dt, fam, meth)
    s.check()
    assert np.max(np.abs(U.cpu().numpy() - want)) / np.max(np.abs(want)) < 1e-11


def test_pattern_active_sets():
    cells = kh_band_cells(4, 7, 0.03)
    m = TreeMesh(cells, -1.0, 2.0)
    E = [4, 6, 10, 16]
    fam = perk2_family(E, pattern="early")
    meth = element_methods(m.cells[:, 0], fam.R)
    U = discontinuous_state(cells, -1.0, 2.0)
    full = DGSEM(m, 3, "hllc").rhs(U)
    s = solver_for(cells, -1.0, 2.0, "hllc")
    s.set_perk2_pattern(E, "early")
    for i in range(fam.S):
        active = np.array([fam.active(int(r), i) for r in meth])
        got = s.rhs_active(i, cuda(U), out=cuda(np.full_like(U, 7.0))).cpu().numpy()
        assert np.all(got[~active] == 7.0)
        assert rel_err_per_var(got[active], full[active]) < 1e-12


def test_classic_pattern_through_the_pattern_entry_is_bitwise_classic():
    cells = kh_band_cells(4, 6, 0.05)
    U0 = nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)
    E = [4, 6, 10, 16]
    outs = []
    for via_pattern in (False, True):
        s = solver_for(cells, -1.0, 2.0, "hllc")
        if via_pattern:
            s.set_perk2_pattern(E, "classic")
        else:
            s.set_perk2_disk(E)
        U = cuda(U0)
        dt = s.compute_dt(U, 0.5)
        for _ in range(3):
            s.step(U, dt)
        outs.append(U)
    assert torch.equal(outs[0], outs[1])


def test_non_nested_pattern_and_derivatives_are_refused():
    from paper_2403_05144_gb300 import PerkError
    cells = kh_band_cells(3, 5, 0.05)
    s = solver_for(cells, -1.0, 2.0, "hllc")
    with pytest.raises(PerkError):
        s.set_perk2_pattern([4, 8, 16], "alternating")      # stage 6 of E = 4 is not one of E = 8's
    s.set_perk2_pattern([4, 8, 16], "early")
    U = cuda(discontinuous_state(cells, -1.0, 2.0))
    with pytest.raises(PerkError):
        s.rhs_jvp(U, U)
