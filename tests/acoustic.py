"""Travelling acoustic wave of Sec. 4.1 (test infrastructure).

A single normal mode (k = 2 pi / L along x) on a homogeneous porous medium,
advected across the wave at Ma0 (along y) by the acceleration that balances
the drag.  The density mode rho_hat = DFT_(1,0)[rho - rho0] (Eq. (2D-DFT))
rotates at the acoustic frequency and decays at chi:

  omega = sqrt(RT k^2 - chi^2)                               Eq. (omega_analyt)
  chi   = [(nu_L + eta_eff) k^2 + mu_D + mu_F eps Ma0 sqrt(RT)] / 2
                                                             Eq. (chi_perp)

with nu_L the longitudinal shear coefficient of the viscous stress, nu_eff in
two dimensions and 4 nu_eff / 3 in three (the paper states the 2D form).
The frequency is the slope of the unwrapped phase of rho_hat, the decay rate
the slope of log |rho_hat|, both least-squares fits over every step.

Parameter sets: the viscous-drag balance of Eq. (VDB_params) (mu_D = nu k^2,
mu_F = nu k^2 / (eps sqrt(RT))), or the closures with a fixed Darcy number
Da = kappa / L^2 (Eqs. (F_eps_Ergun), (mu_D_Ergun_perm), (mu_F_Ergun_perm)).
"""
from __future__ import annotations

import numpy as np


def wave_setup(D, *, L=48, eps=0.5, nu=0.01, JT=1.0, Jeta=1.0, Ma0=0.0, params="VDB", Da=1e-4, a0=1e-4):
    RT = JT / 3.0
    k = 2 * np.pi / L
    if params == "VDB":
        muD = nu * k * k
        muF = nu * k * k / (eps * np.sqrt(RT))
        kappa = eps * nu / muD
        F = muF * np.sqrt(kappa) / eps
    else:
        kappa = Da * L * L
        F = 1.75 / np.sqrt(150 * eps**3)
        muD = eps * nu / kappa
        muF = eps * F / np.sqrt(kappa)
    nz = 1 if D == 2 else 3
    shape = (nz, L, L)
    X = np.broadcast_to(np.arange(L)[None, None, :], shape).astype(float)
    nuL = (1.0 if D == 2 else 4.0 / 3.0) * nu
    chi = 0.5 * ((nuL + Jeta * nu) * k * k + muD + muF * eps * Ma0 * np.sqrt(RT))
    omega = np.sqrt(RT * k * k - chi * chi)
    # initial state of Sec. 4.1: the velocity leads the density by arg(omega - i chi)
    Av = eps * a0 * np.sqrt(RT)
    theta = np.angle(-1j * chi + omega)
    rho0 = 1.0 + a0 * np.cos(k * X)
    v0 = np.stack([Av * np.cos(k * X + theta), eps * Ma0 * np.sqrt(RT) + 0 * X, 0 * X])
    b = (0.0, muD * Ma0 * np.sqrt(RT) + muF * eps * Ma0**2 * RT, 0.0)
    return dict(eps=np.full(shape, eps), kappa=np.full(shape, kappa), F=F, nu=nu, b=b, RT=RT, J_eta=Jeta,
                rho0=rho0, v0=v0, omega=omega, chi=chi, L=L)


def mode(rho, L):
    """rho_hat of Eq. (2D-DFT) at (1, 0) on the first plane."""
    return np.fft.fft2(rho[0] - 1.0)[0, 1] / L**2


def fit(samples, floor=1e-3):
    """(omega, decay rate) from the per-step rho_hat samples, up to the first
    one whose magnitude fell below floor times the initial one (below that,
    storage rounding decides the phase)."""
    z = np.asarray(samples)
    low = np.nonzero(np.abs(z) < floor * abs(z[0]))[0]
    if len(low):
        z = z[: low[0]]
    t = np.arange(len(z))
    omega = -np.polyfit(t, np.unwrap(np.angle(z)), 1)[0]
    rate = -np.polyfit(t, np.log(np.abs(z)), 1)[0]
    return omega, rate
