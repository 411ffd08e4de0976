"""Dynamic pins of the correction terms Phi_ext and Phi_eta (Sec. 4.2).

Small plane-wave disturbances on a homogeneous advected porous medium decay at
the rates the normal-mode analysis of the target equations predicts
(Eqs. for r_ac in setups II and IV).  With the correction terms the measured
rate matches; with the term switched off it visibly does not.  Runs use the
viscous-drag-balance parameters of Eq. (VDB_params) on a smaller box (L = 48).
"""
import numpy as np
import pytest

import oracle

FULL = oracle.CORR_FULL


def acoustic_decay_ratio(setup, lattice=oracle.D2Q9, Ma0=0.1, JT=1.0, Jeta=1.0, corr=FULL, L=48,
                         nsteps=3000, eps=0.5, nu=0.01, a0=1e-5):
    RT = JT / 3.0
    k = 2 * np.pi / L
    muD = nu * k * k
    muF = nu * k * k / (eps * np.sqrt(RT))
    kappa = eps * nu / muD
    F = muF * np.sqrt(kappa) / eps
    nz = 1 if lattice == oracle.D2Q9 else 3
    e = np.full((nz, L, L), eps)
    kap = np.full_like(e, kappa)
    bb = muD * Ma0 * np.sqrt(RT) + muF * eps * Ma0**2 * RT
    X = np.broadcast_to(np.arange(L)[None, None, :], (nz, L, L)).astype(float)
    # longitudinal stress coefficient: nu (2 - 2/D) + eta
    visc = (1.0 if lattice == oracle.D2Q9 else 4.0 / 3.0) + Jeta
    if setup == "II":
        b = (bb, 0, 0)
        vx = eps * Ma0 * np.sqrt(RT) + a0 * np.sin(k * X)
        vy = 0 * X
        r_an = 2 * np.pi**2 * nu / L**2 * (visc + 1 + 2 * Ma0)
    else:
        b = (0, bb, 0)
        vx = a0 * np.sin(k * X)
        vy = eps * Ma0 * np.sqrt(RT) + 0 * X
        r_an = 2 * np.pi**2 * nu / L**2 * (visc + 1 + Ma0)
    o = oracle.Oracle(lattice, e, kap, nu_f=nu, b=b, forch=F, RT=RT, J_eta=Jeta, corr=corr)
    o.init(None, np.stack([vx, vy, 0 * X]))
    amps = []
    for _ in range(nsteps):
        _, v = o.moments()
        vx_, vy_ = v[0, 0], v[1, 0]
        div = (np.roll(vx_, -1, 1) - np.roll(vx_, 1, 1)) / 2 + (np.roll(vy_, -1, 0) - np.roll(vy_, 1, 0)) / 2
        amps.append(abs(np.fft.fft2(div)[0, 1]) / L**2)
        o.step(1)
    A = np.array(amps)
    t = np.arange(nsteps)
    pk = [i for i in range(int(0.1 * nsteps), nsteps - 1) if A[i] >= A[i - 1] and A[i] > A[i + 1]]
    slope = np.polyfit(t[pk], np.log(A[pk]), 1)[0]
    return -slope / r_an


def test_phi_ext_restores_galilean_invariance():
    """Setup II at Ma0 = 0.3: acoustic decay matches with Phi_ext, not without."""
    assert acoustic_decay_ratio("II", Ma0=0.3) == pytest.approx(1.0, abs=0.01)
    assert abs(acoustic_decay_ratio("II", Ma0=0.3, corr=FULL & ~oracle.CORR_PHI_EXT) - 1.0) > 0.05


def test_phi_ext_temperature_independence():
    """Setup IV at J_T = 0.5 (RT = 1/6): the (1 - 3RT) part of Phi_ext."""
    assert acoustic_decay_ratio("IV", JT=0.5) == pytest.approx(1.0, abs=0.01)
    assert abs(acoustic_decay_ratio("IV", JT=0.5, corr=FULL & ~oracle.CORR_PHI_EXT) - 1.0) > 0.3


@pytest.mark.parametrize("lattice", [oracle.D2Q9, oracle.D3Q27])
def test_phi_eta_sets_bulk_viscosity(lattice):
    """Setup IV with eta_eff = 2 nu_f: Phi_eta makes the bulk viscosity independent."""
    steps = 3000 if lattice == oracle.D2Q9 else 2000
    assert acoustic_decay_ratio("IV", lattice=lattice, Jeta=2.0, nsteps=steps) == pytest.approx(1.0, abs=0.015)
    assert abs(acoustic_decay_ratio("IV", lattice=lattice, Jeta=2.0, nsteps=steps,
                                    corr=FULL & ~oracle.CORR_PHI_ETA) - 1.0) > 0.1


def _travelling_wave(lattice, nsteps, corr=FULL, **kw):
    from acoustic import fit, mode, wave_setup

    D = 2 if lattice == oracle.D2Q9 else 3
    w = wave_setup(D, **kw)
    o = oracle.Oracle(lattice, w["eps"], w["kappa"], nu_f=w["nu"], b=w["b"], forch=w["F"], RT=w["RT"],
                      J_eta=w["J_eta"], corr=corr).init(w["rho0"], w["v0"])
    z = []
    for _ in range(nsteps):
        z.append(mode(o.moments()[0], w["L"]))
        o.step(1)
    omega, rate = fit(z)
    return omega / w["omega"], rate / w["chi"]


@pytest.mark.parametrize("JT", [0.2, 1.0, 2.0])
def test_acoustic_phase_speed_temperature(JT):
    """Sec. 4.1 at Ma0 = 0 (VDB parameters): the density mode rotates at
    Eq. (omega_analyt) and decays at chi, Eq. (chi_perp)."""
    w_ratio, r_ratio = _travelling_wave(oracle.D2Q9, 800, JT=JT)
    assert w_ratio == pytest.approx(1.0, abs=2e-3)
    assert r_ratio == pytest.approx(1.0, abs=0.03)


@pytest.mark.parametrize("Ma0", [0.0, 0.5])
def test_acoustic_phase_speed_closure(Ma0):
    """Sec. 4.1 with the closures at Da = 1e-4: the Forchheimer drag of the
    base flow enters chi and slows the wave (Fig. cs_eff_plots (b))."""
    w_ratio, r_ratio = _travelling_wave(oracle.D2Q9, 250, params="closure", Ma0=Ma0)
    assert w_ratio == pytest.approx(1.0, abs=2e-3)
    assert r_ratio == pytest.approx(1.0, abs=0.03)


@pytest.mark.parametrize("lattice", [oracle.D2Q9, oracle.D3Q27])
def test_bulk_viscosity_without_phi_eta_is_tied(lattice):
    """Without Phi_eta the bulk viscosity is eta_0 = 2 nu / D (Eq.
    (eta_0_no_corr)) whatever J_eta asks for; with it, eta = J_eta nu."""
    from acoustic import wave_setup

    D = 2 if lattice == oracle.D2Q9 else 3
    _, r = _travelling_wave(lattice, 800, Jeta=4.0, Ma0=0.1)
    assert r == pytest.approx(1.0, abs=0.015)
    _, r0 = _travelling_wave(lattice, 800, corr=FULL & ~oracle.CORR_PHI_ETA, Jeta=4.0, Ma0=0.1)
    chi4 = wave_setup(D, Jeta=4.0, Ma0=0.1)["chi"]
    chi0 = wave_setup(D, Jeta=2.0 / D, Ma0=0.1)["chi"]
    assert r0 * chi4 / chi0 == pytest.approx(1.0, abs=0.015)
