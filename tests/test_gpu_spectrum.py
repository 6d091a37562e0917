"""The spectrum pipeline on the GPU: the Jacobian assembled from the library's JVP kernels
against the oracle's autograd Jacobian, and Arnoldi Ritz values against its eigenvalues."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.autodiff import TorchDGSEM
from oracle.spectrum import dense_jacobian as oracle_jacobian
from oracle.treemesh import TreeMesh
from perk_inputs import kelvin_helmholtz, nodal_state, uniform_cells
from tests.gpu_common import X3, solver_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_05144_gb300.build import build
    build()


@pytest.fixture(scope="module")
def case():
    cells = uniform_cells(1)
    U = nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)
    J_ref = oracle_jacobian(lambda V: TorchDGSEM(TreeMesh(cells, -1.0, 2.0), 3, "hllc").rhs(V), U)
    return cells, U, J_ref


def test_jacobian_from_jvp_kernels_matches_autograd(case):
    from paper_2403_05144_gb300.spectrum import jacobian_dense
    cells, U, J_ref = case
    s = solver_for(cells, -1.0, 2.0, "hllc")
    J = jacobian_dense(s, torch.from_numpy(U).cuda())
    assert np.max(np.abs(J - J_ref)) <= 1e-11 * np.max(np.abs(J_ref))


def test_full_arnoldi_recovers_the_spectrum(case):
    from paper_2403_05144_gb300.spectrum import ritz_values
    cells, U, J_ref = case
    s = solver_for(cells, -1.0, 2.0, "hllc")
    ev = np.linalg.eigvals(J_ref)
    rv = ritz_values(s, torch.from_numpy(U).cuda(), m=U.size)
    rho = np.abs(ev).max()
    assert abs(np.abs(rv).max() - rho) < 1e-6 * rho
    # the outer eigenvalues (largest moduli, which bound the stable time step) all have a
    # Ritz value next to them
    for z in ev[np.argsort(-np.abs(ev))[:16]]:
        assert np.min(np.abs(rv - z)) < 1e-6 * rho
