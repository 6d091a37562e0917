"""3D compressible Euler fluxes (oracle; test infrastructure only).

Conserved variables u = (rho, rho v1, rho v2, rho v3, E), ideal gas
p = (gamma - 1) (E - rho |v|^2 / 2).  The paper's three-dimensional run
(Sec. 7.1.3, the Taylor-Green vortex, Eq. IC_TaylorGreen) uses an
entropy-conservative volume flux (Ranocha's two-point flux) and the HLLE
surface flux (Einfeldt 1988); HLL and HLLC are the surface fluxes of the 2D
runs, written here for three components of velocity.  All functions are
vectorised over trailing axes; the variable axis is axis 0 of every state.
"""

from __future__ import annotations

import numpy as np

from .euler import log_mean

GAMMA = 1.4


def primitives(u, gamma=GAMMA):
    rho = u[0]
    v1 = u[1] / rho
    v2 = u[2] / rho
    v3 = u[3] / rho
    p = (gamma - 1.0) * (u[4] - 0.5 * rho * (v1 * v1 + v2 * v2 + v3 * v3))
    return rho, v1, v2, v3, p


def physical_flux(u, direction: int, gamma=GAMMA):
    """f(u) along axis ``direction`` (0 = x, 1 = y, 2 = z)."""
    rho, v1, v2, v3, p = primitives(u, gamma)
    vn = (v1, v2, v3)[direction]
    f = [rho * vn]
    for d in range(3):
        f.append(u[1 + d] * vn + (p if d == direction else 0.0 * p))
    f.append((u[4] + p) * vn)
    return np.stack(f)


def ec_flux(uL, uR, direction: int, gamma=GAMMA):
    """Ranocha's entropy-conservative, kinetic-energy-preserving two-point flux
    in three dimensions: with log means {{.}}_ln and arithmetic means {{.}},
      f_rho = {{rho}}_ln {{v_n}},   f_m = f_rho {{v}} + {{p}} n,
      f_E   = f_rho ( v_L . v_R / 2 + 1 / ((gamma - 1) {{rho/p}}_ln) ) + (p_L v_n,R + p_R v_n,L) / 2
    (H. Ranocha, J. Sci. Comput. 2018)."""
    rL, *vL, pL = primitives(uL, gamma)
    rR, *vR, pR = primitives(uR, gamma)
    rho_ln = log_mean(rL, rR)
    beta_ln = log_mean(rL / pL, rR / pR)
    vm = [0.5 * (a + b) for a, b in zip(vL, vR)]
    pm = 0.5 * (pL + pR)
    f_rho = rho_ln * vm[direction]
    f = [f_rho]
    for d in range(3):
        f.append(f_rho * vm[d] + (pm if d == direction else 0.0))
    dot = vL[0] * vR[0] + vL[1] * vR[1] + vL[2] * vR[2]
    f.append(f_rho * (0.5 * dot + 1.0 / ((gamma - 1.0) * beta_ln)) + 0.5 * (pL * vR[direction] + pR * vL[direction]))
    return np.stack(f)


def _hll_mid(uL, uR, fL, fR, SL, SR):
    mid = (SR * fL - SL * fR + SL * SR * (uR - uL)) / (SR - SL)
    return np.where(SL >= 0.0, fL, np.where(SR <= 0.0, fR, mid))


def davis_speeds(uL, uR, direction: int, gamma=GAMMA):
    """S_L = min(v_L - c_L, v_R - c_R), S_R = max(v_L + c_L, v_R + c_R) of the normal velocity."""
    rL, *vL, pL = primitives(uL, gamma)
    rR, *vR, pR = primitives(uR, gamma)
    cL = np.sqrt(gamma * pL / rL)
    cR = np.sqrt(gamma * pR / rR)
    return np.minimum(vL[direction] - cL, vR[direction] - cR), np.maximum(vL[direction] + cL, vR[direction] + cR)


def hll_flux(uL, uR, direction: int, gamma=GAMMA):
    """HLL flux (Harten, Lax, van Leer 1983) with Davis wave-speed estimates."""
    SL, SR = davis_speeds(uL, uR, direction, gamma)
    return _hll_mid(uL, uR, physical_flux(uL, direction, gamma), physical_flux(uR, direction, gamma), SL, SR)


def einfeldt_speeds(uL, uR, direction: int, gamma=GAMMA):
    """Einfeldt's bounds: S_L = min(v_L - c_L, v~ - c~), S_R = max(v_R + c_R, v~ + c~) with Roe
    averages (weights sqrt(rho)) of all three velocity components and of H = (E + p)/rho,
    c~^2 = (gamma - 1)(H~ - |v~|^2 / 2)."""
    rL, *vL, pL = primitives(uL, gamma)
    rR, *vR, pR = primitives(uR, gamma)
    sL, sR = np.sqrt(rL), np.sqrt(rR)
    wL, wR = sL / (sL + sR), sR / (sL + sR)
    vt = [wL * a + wR * b for a, b in zip(vL, vR)]
    H = wL * (uL[4] + pL) / rL + wR * (uR[4] + pR) / rR
    c = np.sqrt((gamma - 1.0) * (H - 0.5 * (vt[0] ** 2 + vt[1] ** 2 + vt[2] ** 2)))
    cL = np.sqrt(gamma * pL / rL)
    cR = np.sqrt(gamma * pR / rR)
    d = direction
    return np.minimum(vL[d] - cL, vt[d] - c), np.maximum(vR[d] + cR, vt[d] + c)


def hlle_flux(uL, uR, direction: int, gamma=GAMMA):
    """HLL flux with Einfeldt's wave-speed bounds (the paper's surface flux of Sec. 7.1.3)."""
    SL, SR = einfeldt_speeds(uL, uR, direction, gamma)
    return _hll_mid(uL, uR, physical_flux(uL, direction, gamma), physical_flux(uR, direction, gamma), SL, SR)


def hllc_flux(uL, uR, direction: int, gamma=GAMMA):
    """HLLC flux (Toro, Spruce, Speares 1994) with the Davis speeds and the contact speed
    S* = (p_R - p_L + rho_L v_L (S_L - v_L) - rho_R v_R (S_R - v_R)) / (rho_L (S_L - v_L) - rho_R (S_R - v_R));
    the star states keep both tangential velocities."""
    SL, SR = davis_speeds(uL, uR, direction, gamma)
    rL, *vL, pL = primitives(uL, gamma)
    rR, *vR, pR = primitives(uR, gamma)
    d = direction
    nL, nR = vL[d], vR[d]
    Sstar = (pR - pL + rL * nL * (SL - nL) - rR * nR * (SR - nR)) / (rL * (SL - nL) - rR * (SR - nR))
    fL = physical_flux(uL, d, gamma)
    fR = physical_flux(uR, d, gamma)

    def star_state(r, v, p, E, S):
        fac = r * (S - v[d]) / (S - Sstar)
        m = [fac * (Sstar if k == d else v[k]) for k in range(3)]
        Es = fac * (E / r + (Sstar - v[d]) * (Sstar + p / (r * (S - v[d]))))
        return np.stack([fac, *m, Es])

    fLs = fL + SL * (star_state(rL, vL, pL, uL[4], SL) - uL)
    fRs = fR + SR * (star_state(rR, vR, pR, uR[4], SR) - uR)
    return np.where(SL >= 0.0, fL, np.where(Sstar >= 0.0, fLs, np.where(SR > 0.0, fRs, fR)))


def entropy_variables(u, gamma=GAMMA):
    """w = dU/du for the entropy U = -rho s / (gamma - 1), s = ln(p rho^-gamma)."""
    rho, v1, v2, v3, p = primitives(u, gamma)
    s = np.log(p) - gamma * np.log(rho)
    b = rho / p
    return np.stack([(gamma - s) / (gamma - 1.0) - 0.5 * b * (v1 * v1 + v2 * v2 + v3 * v3), b * v1, b * v2, b * v3,
                     -b])


def entropy_flux_potential(u, direction: int, gamma=GAMMA):
    """psi = w . f - F_entropy = rho v_n for the Euler equations."""
    rho, v1, v2, v3, p = primitives(u, gamma)
    return rho * (v1, v2, v3)[direction]
