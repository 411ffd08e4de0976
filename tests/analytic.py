"""Reference solutions that pin the oracle to the paper's closed forms.

Channel coordinates: halfway bounce-back walls sit half a spacing outside the
first and last node layer, so node row y lies at distance eta = y + 1/2 from the
lower wall and the channel height is H = ny.
"""
from __future__ import annotations

import numpy as np


def free_poiseuille(eta, H, b, nu):
    """epsilon = 1 limit of Eq. (Poiseuille_v_BVP): v = b eta (H - eta) / (2 nu)."""
    return b * eta * (H - eta) / (2.0 * nu)


def brinkman_channel(eta, H, eps, b, mu_D, nu_eff):
    """Eq. (Poiseuille_v_Darcy_analyt): homogeneous porous channel, mu_F = 0."""
    r = np.sqrt(mu_D / nu_eff)
    return eps * b / mu_D * (1.0 - np.cosh(r * (eta - H / 2.0)) / np.cosh(r * H / 2.0))


def layered_channel(eta, H, h, eps, kappa, b, nu_f, nu_eff):
    """Porous layer 0 < eta < h (porosity eps, permeability kappa, F = 0) under a
    free layer h < eta < H, both governed by Eq. (Poiseuille_v_BVP):
      porous: nu v'' + eps b - mu_D v = 0,  v(0) = 0
      free:   nu v'' + b = 0,               v(H) = 0
    with v and v' continuous at eta = h (the stress of Eq. (visc_stress_target)
    acts on the superficial velocity with one nu_eff)."""
    mu_D = eps * nu_f / kappa
    r = np.sqrt(mu_D / nu_eff)
    vD = eps * b / mu_D
    L = H - h
    sh, ch = np.sinh(r * h), np.cosh(r * h)
    B = ((b / (2 * nu_eff)) * L * L + L * vD * r * sh - vD * (1.0 - ch)) / (L * r * ch + sh)
    E = vD * (1.0 - ch) + B * sh
    C = -vD * r * sh + B * r * ch
    eta = np.asarray(eta, dtype=np.float64)
    vp = vD * (1.0 - np.cosh(r * eta)) + B * np.sinh(r * eta)
    vf = -(b / (2 * nu_eff)) * (eta - h) ** 2 + C * (eta - h) + E
    return np.where(eta < h, vp, vf)


def uniform_darcy_forchheimer(eps, b, mu_D, mu_F):
    """Steady uniform flow: a = 0 in Eq. (accel) gives eps b = mu_D v + mu_F v^2."""
    if mu_F == 0.0:
        return eps * b / mu_D
    return (-mu_D + np.sqrt(mu_D * mu_D + 4.0 * mu_F * eps * b)) / (2.0 * mu_F)


def smoothstep(psi):
    """Eq. (s_cinf), the C-infinity smoothstep."""
    psi = np.asarray(psi, dtype=np.float64)
    out = np.where(psi <= 0.0, 0.0, 1.0)
    inside = (psi > 0.0) & (psi < 1.0)
    p = np.where(inside, psi, 0.5)
    a = np.exp(-1.0 / p)
    c = np.exp(-1.0 / (1.0 - p))
    return np.where(inside, a / (a + c), out)


def setup_I_porosity(eta, H, eps_bot, eps_top, phi_bot, phi_top):
    """Eq. (Hetero_Channel_Setup_I_Profile)."""
    return eps_bot + (eps_top - eps_bot) * smoothstep(((eta / H) - phi_bot) / (1.0 - phi_top - phi_bot))


def channel_bvp(H, eps_fn, muD_fn, muF_fn, b, nu_eff, M=20001, intrinsic_stress=False, tol=1e-14, maxit=100):
    """Fine-grid Newton solution of the steady channel problem (second-order
    finite differences, tridiagonal Newton steps).

    intrinsic_stress=False: Eq. (Poiseuille_v_BVP)
        v'' + (eps b - mu_D v - mu_F |v| v) / nu = 0
    intrinsic_stress=True: Eq. (Poiseuille_u_BVP_wrong_visc_stress) for u = v / eps
        u'' + (eps'/eps) u' + (b - mu_D u - eps mu_F |u| u) / nu = 0
    Both with zero velocity at eta = 0 and eta = H.  Returns (eta grid, v)."""
    from scipy.linalg import solve_banded

    eta = np.linspace(0.0, H, M)
    h = eta[1] - eta[0]
    e = eps_fn(eta) * np.ones_like(eta)
    mD = muD_fn(eta) * np.ones_like(eta)
    mF = muF_fn(eta) * np.ones_like(eta)
    de = np.gradient(e, h)
    ee, md, mf = e[1:-1], mD[1:-1], mF[1:-1]
    g = de[1:-1] / ee if intrinsic_stress else np.zeros_like(ee)
    w = np.zeros(M - 2)
    for _ in range(maxit):
        full = np.concatenate([[0.0], w, [0.0]])
        lap = (full[2:] - 2 * full[1:-1] + full[:-2]) / h**2
        d1 = (full[2:] - full[:-2]) / (2 * h)
        ab = np.zeros((3, M - 2))
        ab[0, 1:] = 1.0 / h**2 + g[:-1] / (2 * h)   # super-diagonal
        ab[2, :-1] = 1.0 / h**2 - g[1:] / (2 * h)   # sub-diagonal
        if not intrinsic_stress:
            F = lap + (ee * b - md * w - mf * np.abs(w) * w) / nu_eff
            ab[1] = -2.0 / h**2 + (-md - 2.0 * mf * np.abs(w)) / nu_eff
        else:
            F = lap + g * d1 + (b - md * w - ee * mf * np.abs(w) * w) / nu_eff
            ab[1] = -2.0 / h**2 + (-md - 2.0 * ee * mf * np.abs(w)) / nu_eff
        dw = solve_banded((1, 1), ab, -F)
        w += dw
        if np.max(np.abs(dw)) <= tol * max(1e-300, np.max(np.abs(w))):
            break
    sol = np.concatenate([[0.0], w, [0.0]])
    if intrinsic_stress:
        sol = sol * e
    return eta, sol


# --------------------------------------------------------------- Couette flow (Sec. 5.1)
# Wet-node walls sit on the first and last node row: row y lies at distance y
# from the lower wall and the channel height is H = ny - 1.

def couette_density(y, H, rho0, g, RT):
    """Eq. (Couette_rho_analyt): rho(y) = rho0 G exp(-G y / H) / (1 - exp(-G)),
    G = g H / RT, with rho0 the mean of rho over [0, H]."""
    if g == 0.0:
        return np.full_like(np.asarray(y, dtype=float), rho0)
    G = g * H / RT
    return rho0 * G * np.exp(-g * np.asarray(y) / RT) / (1.0 - np.exp(-G))


def couette_darcy(y, H, v_bot, v_top, g, RT, mu_D, nu_eff):
    """Eq. (Couette_v_Darcy_analyt): the mu_F = 0 solution of Eq.
    (Couette_v_ODE), v'' - (g / RT) v' - (mu_D / nu_eff) v = 0, v(0) = v_bot,
    v(H) = v_top, with r+- = (g/RT +- sqrt((g/RT)^2 + 4 mu_D / nu_eff)) / 2."""
    y = np.asarray(y, dtype=float)
    k = g / RT
    disc = np.sqrt(k * k + 4.0 * mu_D / nu_eff)
    rp, rm = (k + disc) / 2.0, (k - disc) / 2.0
    if mu_D == 0.0 and k == 0.0:
        return v_bot + (v_top - v_bot) * y / H
    num = (v_top - v_bot * np.exp(rm * H)) * np.exp(rp * y) + (v_bot * np.exp(rp * H) - v_top) * np.exp(rm * y)
    return num / (np.exp(rp * H) - np.exp(rm * H))
