"""GPU derivatives against the oracle's automatic differentiation: JVP, VJP
(full and partitioned), the dot-product identity, the adjoint of one P-ERK
step, the autograd.Function, and a checkpointed multi-step gradient against
central finite differences along seeded directions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.autodiff import TorchDGSEM, jvp_rhs, vjp_rhs, vjp_steps
from oracle.lgl import lgl_nodes_weights
from oracle.perk import element_methods, max_wave_speed_dt, perk2_family
from oracle.treemesh import TreeMesh
from perk_inputs import kelvin_helmholtz, kh_band_cells, nodal_state, vortex_two_level_cells
from tests.gpu_common import X3, discontinuous_state, solver_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_05144_gb300.build import build
    build()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


SMALL = vortex_two_level_cells(3, 2, 6)


@pytest.mark.parametrize("flux", ["hll", "hllc", "ec"])
def test_jvp_and_vjp_match_autodiff(flux):
    U = discontinuous_state(SMALL, -1.0, 2.0)
    rng = np.random.default_rng(8)
    v = rng.normal(size=U.shape)
    lam = rng.normal(size=U.shape)
    dg = TorchDGSEM(TreeMesh(SMALL, -1.0, 2.0), 3, flux)
    s = solver_for(SMALL, -1.0, 2.0, flux)
    # derivatives amplify the ~1e-15 differences between the library's logarithmic
    # mean (node logarithms, series branch) and the oracle's (log1p): the EC
    # surface flux shows 1.3e-11, hence 5e-11 for the derivative parity
    jv = s.rhs_jvp(cuda(U), cuda(v)).cpu().numpy()
    assert rel(jv, jvp_rhs(dg, U, v)) < 5e-11
    jt = s.rhs_vjp(cuda(U), cuda(lam)).cpu().numpy()
    assert rel(jt, vjp_rhs(dg, U, lam)) < 5e-11
    # dot-product identity on the GPU itself
    assert abs(np.sum(jv * lam) - np.sum(v * jt)) < 1e-12 * np.sum(np.abs(jv * lam))


def test_partitioned_vjp_every_stage():
    cells = kh_band_cells(4, 6, 0.05)
    U = discontinuous_state(cells, -1.0, 2.0)
    lam = np.random.default_rng(9).normal(size=U.shape)
    m = TreeMesh(cells, -1.0, 2.0)
    fam = perk2_family([4, 6, 10, 16])
    meth = element_methods(m.cells[:, 0], fam.R)
    s = solver_for(cells, -1.0, 2.0, "hllc", [4, 6, 10, 16])
    dg = TorchDGSEM(m, 3, "hllc")
    for i in (0, 3, 7, 12, 15):
        active = np.array([fam.active(int(r), i) for r in meth])
        got = s.rhs_vjp(cuda(U), cuda(lam), stage=i).cpu().numpy()
        assert rel(got, vjp_rhs(dg, U, lam, active)) < 5e-11


@pytest.mark.parametrize("E,cells_fn", [([4, 8], lambda: SMALL), ([4, 6, 10, 16], lambda: kh_band_cells(3, 5, 0.05))])
def test_step_vjp_matches_autodiff(E, cells_fn):
    cells = cells_fn()
    m = TreeMesh(cells, -1.0, 2.0)
    U = nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)
    dt = max_wave_speed_dt(U, m.h, 3, 0.5)
    lam = np.random.default_rng(10).normal(size=U.shape)
    fam = perk2_family(E)
    meth = element_methods(m.cells[:, 0], fam.R)
    want = vjp_steps(TorchDGSEM(m, 3, "hllc"), U, lam, dt, fam, meth, 1)
    s = solver_for(cells, -1.0, 2.0, "hllc", E)
    got = s.step_vjp(cuda(U), dt, cuda(lam)).cpu().numpy()
    assert rel(got, want) < 1e-10


def test_autograd_function_two_steps():
    from paper_2403_05144_gb300.adjoint import PerkStep
    cells = SMALL
    U = nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)
    m = TreeMesh(cells, -1.0, 2.0)
    dt = max_wave_speed_dt(U, m.h, 3, 0.5)
    s = solver_for(cells, -1.0, 2.0, "hllc", [4, 8])
    w = cuda(np.random.default_rng(11).normal(size=U.shape))
    U0 = cuda(U).requires_grad_(True)
    U2 = PerkStep.apply(PerkStep.apply(U0, s, dt), s, dt)
    (g,) = torch.autograd.grad(torch.sum(w * U2), U0)
    fam = perk2_family([4, 8])
    want = vjp_steps(TorchDGSEM(m, 3, "hllc"), U, w.cpu().numpy(), dt, fam, element_methods(m.cells[:, 0], 2), 2)
    assert rel(g.cpu().numpy(), want) < 1e-10


def test_checkpointed_gradient_vs_central_differences():
    # kinetic energy after 40 steps on a frozen three-level KH mesh, checkpoints every 20 steps
    from paper_2403_05144_gb300.adjoint import gradient, kinetic_energy
    cells = kh_band_cells(4, 6, 0.05)
    m = TreeMesh(cells, -1.0, 2.0)
    U0 = cuda(nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3))
    s = solver_for(cells, -1.0, 2.0, "hllc", [4, 6, 10, 16])
    dt = s.compute_dt(U0, 0.5)
    h = torch.tensor(m.h, device="cuda")
    w = torch.tensor(lgl_nodes_weights(3)[1], device="cuda")
    J = lambda U: kinetic_energy(U, h, w)
    n = 40
    _, grad = gradient(s, U0, dt, n, J, checkpoint_every=20)

    def J_of(U):
        U = U.clone()
        for _ in range(n):
            s.step(U, dt)
        s.check()
        return float(J(U))

    rng = np.random.default_rng(12)
    for k in range(4):
        d = cuda(rng.normal(size=U0.shape)) * U0.abs()
        d = d / torch.linalg.vector_norm(d)
        eps = 1e-6 * float(torch.linalg.vector_norm(U0))
        fd = (J_of(U0 + eps * d) - J_of(U0 - eps * d)) / (2 * eps)
        ad = float(torch.sum(grad * d))
        assert abs(fd - ad) <= 1e-6 * max(abs(ad), 1e-12) + 1e-9 * float(torch.linalg.vector_norm(grad)), (k, fd, ad)


@pytest.mark.parametrize("order", [2, 3])
def test_stored_stages_match_recomputation(order):
    # perk_step_store is perk_step bit for bit, and the reverse sweep from the stored
    # stages is the recomputing reverse sweep bit for bit (same kernels, same inputs)
    cells = kh_band_cells(3, 5, 0.05)
    m = TreeMesh(cells, -1.0, 2.0)
    U = cuda(nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3))
    if order == 2:
        s = solver_for(cells, -1.0, 2.0, "hllc", [4, 6, 10, 16])
    else:
        from paper_2403_05144_gb300 import perk3_disk_tableau
        s = solver_for(cells, -1.0, 2.0, "hllc")
        c, a = perk3_disk_tableau([4, 8, 16])
        s.set_tableau(3, [4, 8, 16], c, a)
    dt = s.compute_dt(U, 0.5)
    lam = cuda(np.random.default_rng(13).normal(size=U.shape))
    Ua, Ub = U.clone(), U.clone()
    s.step(Ua, dt)
    K = s.step_store(Ub, dt)
    assert torch.equal(Ua, Ub)
    assert K.shape == (s.S, len(cells), 4, 4, 4)
    got = s.step_vjp(U, dt, lam, stages=K)
    want = s.step_vjp(U, dt, lam)
    assert torch.equal(got, want)
    s.check()


def test_gradient_with_and_without_stored_stages():
    from paper_2403_05144_gb300.adjoint import gradient, kinetic_energy
    cells = kh_band_cells(3, 5, 0.05)
    m = TreeMesh(cells, -1.0, 2.0)
    U0 = cuda(nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3))
    s = solver_for(cells, -1.0, 2.0, "hllc", [4, 6, 10, 16])
    dt = s.compute_dt(U0, 0.5)
    h = torch.tensor(m.h, device="cuda")
    w = torch.tensor(lgl_nodes_weights(3)[1], device="cuda")
    J = lambda U: kinetic_energy(U, h, w)
    Ja, ga = gradient(s, U0, dt, 13, J, checkpoint_every=5, store_stages=True)
    Jb, gb = gradient(s, U0, dt, 13, J, checkpoint_every=5, store_stages=False)
    assert float(Ja) == float(Jb)
    assert torch.equal(ga, gb)


def test_step_vjp_with_heun_weights_matches_autodiff():
    from oracle.perk import perk2_family as fam_of
    cells = SMALL
    m = TreeMesh(cells, -1.0, 2.0)
    U = nodal_state(kelvin_helmholtz, cells, -1.0, 2.0, X3)
    dt = max_wave_speed_dt(U, m.h, 3, 0.4)
    lam = np.random.default_rng(14).normal(size=U.shape)
    fam = fam_of([4, 8], b_S=0.5)
    meth = element_methods(m.cells[:, 0], fam.R)
    want = vjp_steps(TorchDGSEM(m, 3, "hllc"), U, lam, dt, fam, meth, 1)
    s = solver_for(cells, -1.0, 2.0, "hllc")
    s.set_perk2_disk([4, 8], b_S=0.5)
    got = s.step_vjp(cuda(U), dt, cuda(lam)).cpu().numpy()
    assert rel(got, want) < 1e-10
