"""Error of the volume kernel's own FP64 logarithm (table-driven, Tang 1990) and
Newton-Raphson reciprocal against float64 reference values (numpy/libm)."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_05144_gb300.build import build
    build()
    from paper_2403_05144_gb300 import PerkSolver
    return PerkSolver()


def run(solver, x):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = torch.empty(2 * len(x), dtype=torch.float64, device="cuda")
    assert solver.lib.perk_selftest_math(solver.ctx, len(x), C.c_void_p(xd.data_ptr()), C.c_void_p(out.data_ptr())) == 0
    o = out.cpu().numpy()
    return o[0::2], o[1::2]


def test_log_and_reciprocal_accuracy(solver):
    rng = np.random.default_rng(3)
    x = np.exp(rng.uniform(np.log(1e-6), np.log(1e6), 200000))
    x = np.concatenate([x, 1.0 + np.linspace(-1e-3, 1e-3, 2001), 2.0 ** np.arange(-40, 41),
                        np.nextafter(1.0, 2.0) * np.ones(3), [np.finfo(float).tiny * 4, 1e300]])
    lg, rc = run(solver, x)
    ref_log = np.log(x)
    err = np.abs(lg - ref_log) / np.maximum(1.0, np.abs(ref_log))
    assert err.max() < 3.5e-16, err.max()
    rel = np.abs(rc * x - 1.0)
    assert rel.max() < 4.5e-16, rel.max()


def test_log_of_nonpositive_is_nan(solver):
    lg, _ = run(solver, np.array([-1.0, 0.0, -0.0, np.nan]))
    assert np.all(np.isnan(lg))
