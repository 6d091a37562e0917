"""GPU test of perk_compute_dt_noalloc, the allocation-free step-size entry point.

It serves callers that may not allocate device memory (for instance a solver
running as a custom call inside a framework that owns the device allocator).
The test calls it through the C ABI twice in a row, on two different states,
and compares each result with the context-based perk_compute_dt.  It is
collected last so that a stop-at-first-failure run has run everything else."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.lgl import lgl_nodes_weights
from perk_inputs import kelvin_helmholtz, kh_band_cells, nodal_state, smooth_random_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_05144_gb300.build import build
    build()


def test_noalloc_dt_matches_context_dt_twice():
    from paper_2403_05144_gb300 import PerkSolver, _lib
    lib = _lib.load()
    x, _ = lgl_nodes_weights(3)
    cells = kh_band_cells(4, 7, 0.06)
    levels = torch.tensor([c[0] for c in cells], dtype=torch.int32, device="cuda")
    states = [nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, x),
              smooth_random_state(cells, -1.0, 2.0, x, seed=5, amplitude=0.3)]
    solver = PerkSolver(surface_flux="hllc", use_graph=False)
    solver.upload_mesh(cells, -1.0, 2.0)
    stream = torch.cuda.current_stream().cuda_stream
    results = []
    for U0 in states:                       # two calls in a row; the second must not see the first's scratch
        U = torch.from_numpy(U0).cuda()
        want = solver.compute_dt(U, 0.7)
        got = C.c_double()
        st = lib.perk_compute_dt_noalloc(C.c_void_p(U.data_ptr()), C.c_void_p(levels.data_ptr()), len(cells),
                                         2.0, 1.4, 0.7, C.c_void_p(stream), C.byref(got))
        assert st == 0, lib.perk_last_error(None).decode()
        assert got.value == pytest.approx(want, rel=1e-14)
        results.append(got.value)
    assert results[0] != results[1]


def test_noalloc_dt_rejects_sizes_beyond_its_scratch():
    from paper_2403_05144_gb300 import _lib
    lib = _lib.load()
    U = torch.zeros(1, dtype=torch.float64, device="cuda")
    lev = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = C.c_double()
    st = lib.perk_compute_dt_noalloc(C.c_void_p(U.data_ptr()), C.c_void_p(lev.data_ptr()), 131072 + 1, 2.0, 1.4,
                                     0.7, None, C.byref(out))
    assert st == 1
    assert "PERK_NOALLOC_MAX_ELEM" in lib.perk_last_error(None).decode()


def test_noalloc_dt_reports_inadmissible_states():
    # a node with negative density poisons the reduction: NONFINITE, not a step size from the rest
    from paper_2403_05144_gb300 import _lib
    lib = _lib.load()
    x, _ = lgl_nodes_weights(3)
    cells = kh_band_cells(4, 6, 0.05)
    U0 = nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, x)
    U0[17, 0, 2, 1] = -0.25
    U = torch.from_numpy(U0).cuda()
    lev = torch.tensor([c[0] for c in cells], dtype=torch.int32, device="cuda")
    out = C.c_double(-1.0)
    st = lib.perk_compute_dt_noalloc(C.c_void_p(U.data_ptr()), C.c_void_p(lev.data_ptr()), len(cells), 2.0, 1.4,
                                     0.7, None, C.byref(out))
    assert st == 3
    assert out.value == -1.0
