"""2D compressible Euler fluxes (oracle; test infrastructure only).

Conserved variables u = (rho, rho v1, rho v2, E), ideal gas
p = (gamma - 1) (E - rho |v|^2 / 2).  The paper discretises the Euler and
Navier-Stokes equations with an entropy-conservative flux-differencing volume
integral (Ranocha's two-point flux, cited in Secs. 6.1 and 7.1) and HLL/HLLC
surface fluxes (Secs. 5, 7.2).  All functions are vectorised over leading axes:
the variable axis is axis 0 of every state array.
"""

from __future__ import annotations

import numpy as np

GAMMA = 1.4


def primitives(u, gamma=GAMMA):
    rho = u[0]
    v1 = u[1] / rho
    v2 = u[2] / rho
    p = (gamma - 1.0) * (u[3] - 0.5 * rho * (v1 * v1 + v2 * v2))
    return rho, v1, v2, p


def physical_flux(u, direction: int, gamma=GAMMA):
    """f(u) in x (direction 0) or y (direction 1)."""
    rho, v1, v2, p = primitives(u, gamma)
    vn = v1 if direction == 0 else v2
    return np.stack([rho * vn,
                     u[1] * vn + (p if direction == 0 else 0.0 * p),
                     u[2] * vn + (p if direction == 1 else 0.0 * p),
                     (u[3] + p) * vn])


def log_mean(a, b):
    """Logarithmic mean (b - a) / (ln b - ln a), equal to a when a == b.

    With f = (b - a)/(b + a) and u = f^2:  ln(b/a) = 2 artanh f = 2 f sum_k u^k/(2k+1),
    so the mean is (a + b) / (2 sum_k u^k/(2k+1)).  For |f| < 1e-2 this series
    (to u^3; remainder below 1e-17 relative) is used, as in the stable
    evaluation of Ismail and Roe (J. Comput. Phys. 228, 2009); it is smooth
    across a == b.  Otherwise (b - a) / log1p((b - a)/a), where log1p keeps full
    relative accuracy.
    """
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = b - a
    s = a + b
    f = d / s
    u = f * f
    small = np.abs(f) < 1e-2
    series = s / (2.0 * (1.0 + u / 3.0 + u * u / 5.0 + u * u * u / 7.0))
    safe = np.where(small, 1.0, d)
    return np.where(small, series, safe / np.log1p(safe / a))


def ec_flux(uL, uR, direction: int, gamma=GAMMA):
    """Ranocha's entropy-conservative, kinetic-energy-preserving two-point flux.

    With log means {{.}}_ln, arithmetic means {{.}} and normal velocity v_n:
      f_rho = {{rho}}_ln {{v_n}}
      f_m   = f_rho {{v}} + {{p}} n
      f_E   = f_rho ( v_L . v_R / 2 + 1 / ((gamma - 1) {{rho/p}}_ln) )
              + (p_L v_n,R + p_R v_n,L) / 2
    (H. Ranocha, J. Sci. Comput. 2018, and his 2018 thesis).
    """
    rL, v1L, v2L, pL = primitives(uL, gamma)
    rR, v1R, v2R, pR = primitives(uR, gamma)
    rho_ln = log_mean(rL, rR)
    beta_ln = log_mean(rL / pL, rR / pR)
    v1m = 0.5 * (v1L + v1R)
    v2m = 0.5 * (v2L + v2R)
    pm = 0.5 * (pL + pR)
    vnL, vnR = (v1L, v1R) if direction == 0 else (v2L, v2R)
    vnm = 0.5 * (vnL + vnR)
    f_rho = rho_ln * vnm
    f_m1 = f_rho * v1m + (pm if direction == 0 else 0.0)
    f_m2 = f_rho * v2m + (pm if direction == 1 else 0.0)
    f_E = f_rho * (0.5 * (v1L * v1R + v2L * v2R) + 1.0 / ((gamma - 1.0) * beta_ln)) \
        + 0.5 * (pL * vnR + pR * vnL)
    return np.stack([f_rho, f_m1, f_m2, f_E])


def davis_speeds(uL, uR, direction: int, gamma=GAMMA):
    """S_L = min(v_L - c_L, v_R - c_R), S_R = max(v_L + c_L, v_R + c_R)."""
    rL, v1L, v2L, pL = primitives(uL, gamma)
    rR, v1R, v2R, pR = primitives(uR, gamma)
    vL = v1L if direction == 0 else v2L
    vR = v1R if direction == 0 else v2R
    cL = np.sqrt(gamma * pL / rL)
    cR = np.sqrt(gamma * pR / rR)
    return np.minimum(vL - cL, vR - cR), np.maximum(vL + cL, vR + cR)


def hll_flux(uL, uR, direction: int, gamma=GAMMA):
    """HLL flux (Harten, Lax, van Leer 1983) with Davis wave-speed estimates."""
    SL, SR = davis_speeds(uL, uR, direction, gamma)
    fL = physical_flux(uL, direction, gamma)
    fR = physical_flux(uR, direction, gamma)
    mid = (SR * fL - SL * fR + SL * SR * (uR - uL)) / (SR - SL)
    return np.where(SL >= 0.0, fL, np.where(SR <= 0.0, fR, mid))


def einfeldt_speeds(uL, uR, direction: int, gamma=GAMMA):
    """Einfeldt's bounds (1988): S_L = min(v_L - c_L, v~ - c~), S_R = max(v_R + c_R, v~ + c~), with
    the Roe averages v~ = (sqrt(rho_L) v_L + sqrt(rho_R) v_R)/(sqrt(rho_L) + sqrt(rho_R)) (both
    components), H~ likewise for the enthalpy H = (E + p)/rho, c~^2 = (gamma - 1)(H~ - |v~|^2/2)."""
    rL, v1L, v2L, pL = primitives(uL, gamma)
    rR, v1R, v2R, pR = primitives(uR, gamma)
    sL, sR = np.sqrt(rL), np.sqrt(rR)
    wL, wR = sL / (sL + sR), sR / (sL + sR)
    v1 = wL * v1L + wR * v1R
    v2 = wL * v2L + wR * v2R
    H = wL * (uL[3] + pL) / rL + wR * (uR[3] + pR) / rR
    c = np.sqrt((gamma - 1.0) * (H - 0.5 * (v1 * v1 + v2 * v2)))
    vL, vR, vm = (v1L, v1R, v1) if direction == 0 else (v2L, v2R, v2)
    cL = np.sqrt(gamma * pL / rL)
    cR = np.sqrt(gamma * pR / rR)
    return np.minimum(vL - cL, vm - c), np.maximum(vR + cR, vm + c)


def hlle_flux(uL, uR, direction: int, gamma=GAMMA):
    """HLL flux with Einfeldt's wave-speed bounds (HLLE, the surface flux of the paper's
    shock-capturing runs, Sec. 7.2)."""
    SL, SR = einfeldt_speeds(uL, uR, direction, gamma)
    fL = physical_flux(uL, direction, gamma)
    fR = physical_flux(uR, direction, gamma)
    mid = (SR * fL - SL * fR + SL * SR * (uR - uL)) / (SR - SL)
    return np.where(SL >= 0.0, fL, np.where(SR <= 0.0, fR, mid))


def hllc_flux(uL, uR, direction: int, gamma=GAMMA):
    """HLLC flux (Toro, Spruce, Speares 1994; Toro's textbook, Sec. 10.4) with
    the Davis speeds S_L, S_R and the contact speed
    S* = (p_R - p_L + rho_L v_L (S_L - v_L) - rho_R v_R (S_R - v_R))
         / (rho_L (S_L - v_L) - rho_R (S_R - v_R))."""
    SL, SR = davis_speeds(uL, uR, direction, gamma)
    rL, v1L, v2L, pL = primitives(uL, gamma)
    rR, v1R, v2R, pR = primitives(uR, gamma)
    vL, tL = (v1L, v2L) if direction == 0 else (v2L, v1L)
    vR, tR = (v1R, v2R) if direction == 0 else (v2R, v1R)
    Sstar = (pR - pL + rL * vL * (SL - vL) - rR * vR * (SR - vR)) / (rL * (SL - vL) - rR * (SR - vR))
    fL = physical_flux(uL, direction, gamma)
    fR = physical_flux(uR, direction, gamma)

    def star_state(r, v, t, p, E, S):
        fac = r * (S - v) / (S - Sstar)
        mn = fac * Sstar
        mt = fac * t
        Es = fac * (E / r + (Sstar - v) * (Sstar + p / (r * (S - v))))
        if direction == 0:
            return np.stack([fac, mn, mt, Es])
        return np.stack([fac, mt, mn, Es])

    uLs = star_state(rL, vL, tL, pL, uL[3], SL)
    uRs = star_state(rR, vR, tR, pR, uR[3], SR)
    fLs = fL + SL * (uLs - uL)
    fRs = fR + SR * (uRs - uR)
    return np.where(SL >= 0.0, fL, np.where(Sstar >= 0.0, fLs, np.where(SR > 0.0, fRs, fR)))


def entropy_variables(u, gamma=GAMMA):
    """w = dU/du for the entropy U = -rho s / (gamma - 1), s = ln(p rho^-gamma)."""
    rho, v1, v2, p = primitives(u, gamma)
    s = np.log(p) - gamma * np.log(rho)
    b = rho / p
    return np.stack([(gamma - s) / (gamma - 1.0) - 0.5 * b * (v1 * v1 + v2 * v2), b * v1, b * v2, -b])


def entropy_flux_potential(u, direction: int, gamma=GAMMA):
    """psi = w . f - F_entropy = rho v_n for the Euler equations."""
    rho, v1, v2, p = primitives(u, gamma)
    return rho * (v1 if direction == 0 else v2)
