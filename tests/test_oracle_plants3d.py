"""Planted mistakes in the 3D oracle (on the CPU, in a patched copy of its functions) are caught
by its pins: a transposed mortar quadrant, a wrong energy term of the two-point flux along z, and
a dropped cross term of the 3D viscous stress.  This checks that the pins of
test_oracle_dgsem3d.py and test_oracle_br1_3d.py constrain what they are meant to."""
import numpy as np

import oracle.br1_3d as br1_3d
import oracle.dgsem3d as dgsem3d
import oracle.euler3d as euler3d
import oracle.octree as octree


def _run(test_fn, *args):
    try:
        test_fn(*args)
    except AssertionError:
        return False
    return True


def test_transposed_quadrant_is_caught(monkeypatch):
    from tests import test_oracle_dgsem3d as pins
    assert _run(pins.test_reduces_to_the_2d_oracle_on_an_extruded_mesh, "hll")
    orig = octree.match_faces3

    def swapped(lo, size, D):
        c, h = orig(lo, size, D)
        return c, [(A, B, d, lg, q2, q1) for (A, B, d, lg, q1, q2) in h]

    monkeypatch.setattr(octree, "match_faces3", swapped)
    assert not _run(pins.test_reduces_to_the_2d_oracle_on_an_extruded_mesh, "hll")


def test_wrong_z_energy_flux_is_caught(monkeypatch):
    from tests import test_oracle_dgsem3d as pins
    orig = euler3d.ec_flux

    def bad(uL, uR, d, gamma=1.4):
        f = orig(uL, uR, d, gamma)
        if d == 2:
            f = f.copy()
            f[4] = f[4] * (1.0 + 1e-7)
        return f

    assert _run(pins.test_axis_permutation_symmetry)
    monkeypatch.setattr(euler3d, "ec_flux", bad)
    assert not _run(pins.test_axis_permutation_symmetry)


def test_dropped_stress_cross_term_is_caught(monkeypatch):
    from tests import test_oracle_br1_3d as pins
    assert _run(pins.test_axis_relabelling)

    def bad_fluxes(self, V, q):
        rho = V[0]
        v = [V[1 + d] / rho for d in range(3)]
        mu, k = self.mu, self.kappa
        dv = [[q[b][a] for b in range(3)] for a in range(3)]
        div = dv[0][0] + dv[1][1] + dv[2][2]
        # the transposed gradient of the stress is left out along z
        tau = [[mu * (dv[a][b] + (dv[b][a] if b < 2 else 0.0) - (2.0 / 3.0 if a == b else 0.0) * div)
                for b in range(3)] for a in range(3)]
        z = np.zeros_like(rho)
        return [np.stack([z, tau[0][d], tau[1][d], tau[2][d],
                          v[0] * tau[0][d] + v[1] * tau[1][d] + v[2] * tau[2][d] + k * q[d][3]]) for d in range(3)]

    monkeypatch.setattr(br1_3d.NavierStokesDGSEM3D, "viscous_fluxes", bad_fluxes)
    assert not _run(pins.test_axis_relabelling)
