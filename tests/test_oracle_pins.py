"""Pins of the FP64 oracle against what the paper and mathematics fix.

None of these tests re-types the oracle's formulas: each compares it with a
textbook value, a closed form, an invariant, or an independently derived
quantity (sympy differentiation of the divergence forms).
"""
import numpy as np
import pytest
import sympy as sp

import analytic
import oracle
from paper_2606_29619_b300 import workloads

INF = np.inf


def _box(shape, eps, kappa=INF):
    e = np.full(shape, float(eps))
    k = np.full(shape, float(kappa))
    return e, k


# --------------------------------------------------------------- lattice / equilibrium

def test_weights_textbook_values():
    """Eq. (eq_weights) at RT = 1/3 gives the standard D2Q9 / D3Q27 weights."""
    e, k = _box((1, 4, 4), 1.0)
    w, c = oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.1).lattice()
    for wi, ci in zip(w, c):
        nnz = int(np.count_nonzero(ci))
        assert wi == pytest.approx({0: 4 / 9, 1: 1 / 9, 2: 1 / 36}[nnz], rel=1e-15)
    e, k = _box((4, 4, 4), 1.0)
    w, c = oracle.Oracle(oracle.D3Q27, e, k, nu_f=0.1).lattice()
    for wi, ci in zip(w, c):
        nnz = int(np.count_nonzero(ci))
        assert wi == pytest.approx({0: 8 / 27, 1: 2 / 27, 2: 1 / 54, 3: 1 / 216}[nnz], rel=1e-15)
    # velocity order: i = ix + 3 iy + 9 iz with c = digit - 1, opposite is Q-1-i
    for i in range(27):
        assert tuple(c[i]) == (i % 3 - 1, (i // 3) % 3 - 1, i // 9 - 1)
        assert tuple(c[26 - i]) == tuple(-c[i])


@pytest.mark.parametrize("RT", [0.2, 1.0 / 3.0, 0.45])
def test_weights_general_temperature(RT):
    """Second form of Eq. (eq_weights): prod over axes of 1 - c^2 + (3c^2/2 - 1) RT."""
    e, k = _box((3, 3, 3), 1.0)
    w, c = oracle.Oracle(oracle.D3Q27, e, k, nu_f=0.1, RT=RT).lattice()
    for wi, ci in zip(w, c):
        ref = np.prod([(1 - RT) if cc == 0 else RT / 2 for cc in ci])
        assert wi == pytest.approx(ref, rel=1e-14)
    assert w.sum() == pytest.approx(1.0, rel=1e-15)


@pytest.mark.parametrize("lattice", [oracle.D2Q9, oracle.D3Q27])
def test_product_form_moments(lattice):
    """Scaled moments of the product form, Eqs. (Pi_1_prod_general)-(Pi_3_prod_general)
    and the diagonal third-moment anomaly of Eq. (prod_deviation)."""
    shape = (1, 4, 4) if lattice == oracle.D2Q9 else (3, 3, 3)
    e, k = _box(shape, 1.0)
    o = oracle.Oracle(lattice, e, k, nu_f=0.1)
    w, c = o.lattice()
    D = o.D
    rng = np.random.default_rng(7)
    for _ in range(5):
        xi = rng.uniform(-0.2, 0.2, D)
        P = xi**2 + rng.uniform(0.2, 0.45, D)
        er = rng.uniform(0.3, 1.2)
        f = o.product_form(er, xi, P)
        cc = c[:, :D].astype(float)
        assert f.sum() == pytest.approx(er, rel=1e-14)
        np.testing.assert_allclose(cc.T @ f, er * xi, rtol=1e-13, atol=1e-15)
        M2 = np.einsum("ia,ib,i->ab", cc, cc, f)
        ref2 = er * np.outer(xi, xi)
        ref2[np.diag_indices(D)] = er * P
        np.testing.assert_allclose(M2, ref2, rtol=1e-13, atol=1e-15)
        M3 = np.einsum("ia,ib,ig,i->abg", cc, cc, cc, f)
        for a in range(D):
            assert M3[a, a, a] == pytest.approx(er * xi[a], rel=1e-12, abs=1e-15)
            for b in range(D):
                if b != a:
                    assert M3[a, a, b] == pytest.approx(er * P[a] * xi[b], rel=1e-12, abs=1e-15)
        # at P = xi^2 + RT the deviation from the target third moment is
        # eps rho [(1 - 3RT) xi_a - xi_a^3] on the diagonal only
        RT = 1.0 / 3.0
        f = o.product_form(er, xi, xi**2 + RT)
        M3 = np.einsum("ia,ib,ig,i->abg", cc, cc, cc, f)
        I = np.eye(D)
        tgt = er * (np.einsum("a,b,g->abg", xi, xi, xi) + RT * (np.einsum("a,bg->abg", xi, I)
                                                                + np.einsum("b,ag->abg", xi, I)
                                                                + np.einsum("g,ab->abg", xi, I)))
        dev = M3 - tgt
        ref = np.zeros_like(dev)
        for a in range(D):
            ref[a, a, a] = er * ((1 - 3 * RT) * xi[a] - xi[a] ** 3)
        np.testing.assert_allclose(dev, ref, atol=1e-15)


# --------------------------------------------------------------- uniform box

@pytest.mark.parametrize("lattice", [oracle.D2Q9, oracle.D3Q27])
def test_uniform_box_momentum_gain_and_steady_state(lattice):
    """Homogeneous periodic box: every node evolves alike, the momentum moment
    gains exactly rho a per step (Appendix D), and the steady state solves
    eps b = mu_D v + mu_F |v| v (Eq. (accel) with a = 0)."""
    shape = (1, 4, 4) if lattice == oracle.D2Q9 else (3, 3, 3)
    eps, kappa, F, nu = 0.4, 0.5, 0.55, 0.05
    e, k = _box(shape, eps, kappa)
    b = np.array([2e-3, -1e-3, 5e-4])
    o = oracle.Oracle(lattice, e, k, nu_f=nu, b=b, forch=F).init()
    w, c = o.lattice()
    D = o.D
    for _ in range(20):
        rho, v = o.moments()
        a, _, _ = o.forces()
        P1 = np.einsum("ia,i...->a...", c[:, :D].astype(float), o.get_f())
        o.step(1)
        P1n = np.einsum("ia,i...->a...", c[:, :D].astype(float), o.get_f())
        np.testing.assert_allclose(P1n - P1, rho[None] * a[:D], rtol=1e-10, atol=1e-17)
    o.step(3000)
    rho, v = o.moments()
    muD, muF = eps * nu / kappa, eps * F / np.sqrt(kappa)
    vmag = np.sqrt((v**2).sum(axis=0))
    bmag = np.linalg.norm(b[:D])
    ref = analytic.uniform_darcy_forchheimer(eps, bmag, muD, muF)
    np.testing.assert_allclose(vmag, ref, rtol=1e-10)
    np.testing.assert_allclose(v[:D, 0, 0, 0] / vmag.flat[0], b[:D] / bmag, rtol=1e-10)
    np.testing.assert_allclose(rho, 1.0, rtol=1e-12)


def test_uniform_box_ergun_mode():
    """forch < 0 selects F_eps = 1.75 / sqrt(150 eps^3), Eq. (F_eps_Ergun)."""
    eps, kappa, nu = 0.5, 0.2, 0.05
    e, k = _box((1, 4, 4), eps, kappa)
    o = oracle.Oracle(oracle.D2Q9, e, k, nu_f=nu, b=(1e-3, 0, 0), forch=-1.0)
    muD, muF, _, _ = o.static()
    assert muD.flat[0] == pytest.approx(eps * nu / kappa, rel=1e-15)
    assert muF.flat[0] == pytest.approx(eps * 1.75 / np.sqrt(150 * eps**3) / np.sqrt(kappa), rel=1e-15)


# --------------------------------------------------------------- conservation

@pytest.mark.parametrize("lattice,walls", [(oracle.D2Q9, (0, 1, 0)), (oracle.D3Q27, (0, 1, 1)),
                                           (oracle.D3Q27, (0, 0, 0))])
def test_mass_conservation(lattice, walls):
    """Collision conserves sum_i f (Eq. (transformed_density_moment_2)); periodic
    wrap and halfway bounce-back move populations without loss."""
    shape = (1, 12, 10) if lattice == oracle.D2Q9 else (8, 7, 6)
    e = workloads.random_smooth_porosity(shape, seed=3)
    k = workloads.carman_kappa(e, 2.0)
    o = oracle.Oracle(lattice, e, k, nu_f=0.05, b=(1e-3, 5e-4, 2e-4), forch=-1, wall=walls).init()
    m0 = o.mass()
    o.step(200)
    assert abs(o.mass() - m0) / m0 < 1e-13


# --------------------------------------------------------------- channels

def _channel(lattice, ny, eps_y, kappa_y, nx=4, nz=3):
    if lattice == oracle.D2Q9:
        e = np.broadcast_to(eps_y[None, :, None], (1, ny, nx)).copy()
        k = np.broadcast_to(kappa_y[None, :, None], (1, ny, nx)).copy()
    else:
        e = np.broadcast_to(eps_y[None, :, None], (nz, ny, nx)).copy()
        k = np.broadcast_to(kappa_y[None, :, None], (nz, ny, nx)).copy()
    return e, k


def _steady(o, check_every=2000, tol=1e-11, max_steps=200000):
    _, vprev = o.moments()
    while o.steps < max_steps:
        o.step(check_every)
        _, v = o.moments()
        r = np.sqrt(((v - vprev) ** 2).sum() / max(1e-300, (vprev**2).sum()))
        vprev = v
        if r < tol:
            break
    return o.moments()


@pytest.mark.parametrize("lattice", [oracle.D2Q9, oracle.D3Q27])
def test_free_poiseuille(lattice):
    """eps = 1 reduces the model to plain LBM: v = b eta (H - eta) / (2 nu)."""
    ny, nu, b = 24, 1.0 / 6.0, 1e-6
    e, k = _channel(lattice, ny, np.ones(ny), np.full(ny, INF))
    o = oracle.Oracle(lattice, e, k, nu_f=nu, b=(b, 0, 0), wall=(0, 1, 0)).init()
    _, v = _steady(o)
    eta = np.arange(ny) + 0.5
    ref = analytic.free_poiseuille(eta, ny, b, nu)
    prof = v[0, 0, :, 0]
    assert np.max(np.abs(prof - ref)) / ref.max() < 2e-3
    assert np.max(np.abs(v[1:])) < 1e-12 * ref.max()


def test_brinkman_channel():
    """Homogeneous porous channel against Eq. (Poiseuille_v_Darcy_analyt)."""
    ny, nu, b, eps = 40, 0.1, 1e-5, 0.3
    kappa = 4.0  # r H = sqrt(eps/kappa) H ~ 11
    e, k = _channel(oracle.D2Q9, ny, np.full(ny, eps), np.full(ny, kappa))
    o = oracle.Oracle(oracle.D2Q9, e, k, nu_f=nu, b=(b, 0, 0), wall=(0, 1, 0)).init()
    _, v = _steady(o)
    eta = np.arange(ny) + 0.5
    ref = analytic.brinkman_channel(eta, ny, eps, b, eps * nu / kappa, nu)
    prof = v[0, 0, :, 0]
    assert np.max(np.abs(prof - ref)) / ref.max() < 1e-2


def test_layered_reference_solutions_agree():
    """The coupled porous/free closed form and the fine-grid BVP solver give the
    same profile for the sharp two-layer channel (pins the BVP solver)."""
    H, nu, b, eps, kappa = 64.0, 1.0 / 6.0, 1e-6, 0.5, 4.096
    eta = np.arange(64) + 0.5
    ref = analytic.layered_channel(eta, H, H / 2, eps, kappa, b, nu, nu)
    ef = lambda x: np.where(x < H / 2, eps, 1.0)
    mD = lambda x: np.where(x < H / 2, eps * nu / kappa, 0.0)
    g, v = analytic.channel_bvp(H, ef, mD, lambda x: 0.0 * x, b, nu, M=64001)
    np.testing.assert_allclose(np.interp(eta, g, v), ref, rtol=0, atol=2e-4 * ref.max())


@pytest.mark.parametrize("F", [0.0, 0.1])
def test_layered_channel_smoothed_interface(F):
    """Two-layer channel (porous half eps = 0.5, Da = 1e-3, nu = 1/6) with the
    porosity step smoothed over 4 nodes by Eq. (s_cinf), as the method requires
    a C2 porosity field (Sec. 3.5): the steady profile solves Eq.
    (Poiseuille_v_BVP), Forchheimer drag included."""
    ny, nu, b = 64, 1.0 / 6.0, 1e-6
    H, kap, w = float(ny), 1e-3 * ny * ny, 4.0
    ef = lambda x: 0.5 + 0.5 * analytic.smoothstep((x - (H / 2 - w / 2)) / w)
    mD = lambda x: np.where(ef(x) >= 1.0, 0.0, ef(x) * nu / kap)
    mF = lambda x: np.where(ef(x) >= 1.0, 0.0, ef(x) * F / np.sqrt(kap))
    eta = np.arange(ny) + 0.5
    e, k = _channel(oracle.D2Q9, ny, ef(eta), np.where(ef(eta) >= 1.0, INF, kap))
    o = oracle.Oracle(oracle.D2Q9, e, k, nu_f=nu, b=(b, 0, 0), forch=F, wall=(0, 1, 0)).init()
    _, v = _steady(o, check_every=5000)
    g, vb = analytic.channel_bvp(H, ef, mD, mF, b, nu)
    ref = np.interp(eta, g, vb)
    assert np.max(np.abs(v[0, 0, :, 0] - ref)) / ref.max() < 1e-2


def test_heterogeneous_channel_delta_nu():
    """Setup I porosity (Eq. (Hetero_Channel_Setup_I_Profile)) with fixed Da:
    with the porosity correction Delta_nu the steady profile solves
    Eq. (Poiseuille_v_BVP); without it the profile solves
    Eq. (Poiseuille_u_BVP_wrong_visc_stress).  Each model must sit much closer
    to its own BVP than to the other one."""
    ny, nu, Hg, Da = 48, 0.1, 1000.0, 1e-2
    H = float(ny)
    b = Hg * nu * nu / H**3
    kappa = Da * H * H
    eps_fn = lambda eta: analytic.setup_I_porosity(eta, H, 1.0, 0.5, 0.1, 0.1)
    eta = np.arange(ny) + 0.5
    e, k = _channel(oracle.D2Q9, ny, eps_fn(eta), np.full(ny, kappa))
    muD_fn = lambda x: eps_fn(x) * nu / kappa
    zero = lambda x: 0.0 * x
    _, v_sup = analytic.channel_bvp(H, eps_fn, muD_fn, zero, b, nu, intrinsic_stress=False)
    eta_f, v_int = analytic.channel_bvp(H, eps_fn, muD_fn, zero, b, nu, intrinsic_stress=True)
    ref_sup = np.interp(eta, eta_f, v_sup)
    ref_int = np.interp(eta, eta_f, v_int)
    gap = np.max(np.abs(ref_sup - ref_int)) / ref_sup.max()
    assert gap > 0.05  # the two targets differ
    full = oracle.Oracle(oracle.D2Q9, e, k, nu_f=nu, b=(b, 0, 0), wall=(0, 1, 0)).init()
    _, v = _steady(full)
    err_sup = np.max(np.abs(v[0, 0, :, 0] - ref_sup)) / ref_sup.max()
    assert err_sup < 0.15 * gap
    nodn = oracle.Oracle(oracle.D2Q9, e, k, nu_f=nu, b=(b, 0, 0), wall=(0, 1, 0),
                         corr=oracle.CORR_PHI_EXT | oracle.CORR_PHI_ETA).init()
    _, v = _steady(nodn)
    err_int = np.max(np.abs(v[0, 0, :, 0] - ref_int)) / ref_int.max()
    assert err_int < 0.15 * gap


# --------------------------------------------------------------- differential operators

def _manufactured(L, walls, seed=0):
    """Symbolic smooth fields on an L^3 grid; along wall axes they are not periodic."""
    x, y, z = sp.symbols("x y z", real=True)
    X = (x, y, z)
    kx = [2 * sp.pi / L if not walls[a] else sp.Rational(37, 10) / L for a in range(3)]
    eps = (sp.Rational(7, 10) + sp.Rational(1, 10) * sp.sin(kx[0] * x + sp.Rational(1, 5)) * sp.cos(kx[1] * y)
           + sp.Rational(1, 20) * sp.sin(kx[2] * z + sp.Rational(3, 10)))
    m = [sp.Rational(1, 50) * sp.cos(kx[0] * x + sp.Rational(1, 10)) * sp.sin(kx[1] * y + sp.Rational(1, 7))
         + sp.Rational(1, 100) * sp.sin(kx[2] * z),
         sp.Rational(3, 200) * sp.sin(kx[0] * x) * sp.cos(kx[2] * z + sp.Rational(1, 3)),
         sp.Rational(1, 100) * sp.cos(kx[1] * y + kx[2] * z)]
    rho = 1 + sp.Rational(1, 20) * sp.sin(kx[0] * x + kx[1] * y + sp.Rational(2, 5))
    return X, eps, m, rho


def _grid(L):
    g = np.arange(L, dtype=np.float64)
    Z, Y, Xg = np.meshgrid(g, g, g, indexing="ij")
    return Xg, Y, Z


@pytest.mark.parametrize("walls", [(0, 0, 0), (0, 1, 1)])
def test_delta_nu_operator_converges_to_divergence_form(walls):
    """The expanded Delta_nu (Eq. (porosity_correction_expanded)) evaluated by the
    oracle's finite differences converges at second order to the divergence
    form of Eq. (porosity_correction), differentiated symbolically."""
    nu_eff = 0.07
    errs = []
    for L in (16, 32):
        X, eps, m, _ = _manufactured(L, walls)
        ge = [sp.diff(eps, xx) for xx in X]
        ref_sym = [sum(sp.diff(nu_eff * (m[a] * ge[b] + ge[a] * m[b]), X[b]) for b in range(3)) for a in range(3)]
        Xg, Y, Z = _grid(L)
        f = lambda ex: sp.lambdify(X, ex, "numpy")(Xg, Y, Z) * np.ones_like(Xg)
        e = f(eps)
        o = oracle.Oracle(oracle.D3Q27, e, np.full_like(e, INF), nu_f=nu_eff, wall=walls)
        out = o.delta_nu(np.stack([f(mm) for mm in m]))
        ref = np.stack([f(r) for r in ref_sym])
        errs.append(np.max(np.abs(out - ref)) / np.max(np.abs(ref)))
    assert errs[1] < 2e-2
    assert 3.0 < errs[0] / errs[1] < 5.5


@pytest.mark.parametrize("walls", [(0, 0, 0), (1, 0, 1)])
def test_corrections_converge_to_definitions(walls):
    """Phi_ext (Eq. (ex_corr)) and Phi_eta (Eq. (eta_corr)) by the oracle's finite
    differences converge at second order to the symbolic derivatives, away from
    RT = 1/3 and with eta_eff != nu_eff so that every term is active."""
    RT, J_eta, nu = 0.25, 1.7, 0.05
    errs_x, errs_e = [], []
    for L in (16, 32):
        X, eps, m, rho = _manufactured(L, walls)
        v = [mm * 5 for mm in m]
        phx_sym = [sp.diff(rho * v[a] * (1 - 3 * RT) - rho * v[a] ** 3 / eps**2, X[a]) for a in range(3)]
        phe_sym = rho * RT * (sp.Rational(2, 3) - J_eta) * sum(sp.diff(v[a], X[a]) for a in range(3))
        Xg, Y, Z = _grid(L)
        f = lambda ex: sp.lambdify(X, ex, "numpy")(Xg, Y, Z) * np.ones_like(Xg)
        e = f(eps)
        o = oracle.Oracle(oracle.D3Q27, e, np.full_like(e, INF), nu_f=nu, RT=RT, J_eta=J_eta, wall=walls)
        phx, phe = o.corrections(f(rho), np.stack([f(vv) for vv in v]))
        ref_x = np.stack([f(r) for r in phx_sym])
        ref_e = f(phe_sym)
        errs_x.append(np.max(np.abs(phx - ref_x)) / np.max(np.abs(ref_x)))
        errs_e.append(np.max(np.abs(phe - ref_e)) / np.max(np.abs(ref_e)))
    for errs in (errs_x, errs_e):
        assert errs[1] < 2e-2
        assert 3.0 < errs[0] / errs[1] < 5.5


# --------------------------------------------------------------- cross-lattice

def test_z_invariant_d3q27_equals_d2q9():
    """For z-invariant inputs the z-sums of D3Q27 populations evolve exactly as
    D2Q9 ones, because sum_c Psi(c; xi, P) = 1 for any P (Eq. (1d_scaled_eq)),
    provided Phi_eta vanishes on both lattices (eta_eff / nu_eff = 2 / D)."""
    ny, nx, nz = 10, 9, 3
    e2 = workloads.random_smooth_porosity((1, ny, nx), seed=11)
    k2 = workloads.carman_kappa(e2, 2.0)
    kw = dict(nu_f=0.04, b=(2e-4, 1e-4, 0.0), forch=-1, wall=(0, 1, 0))
    o2 = oracle.Oracle(oracle.D2Q9, e2, k2, J_eta=1.0, **kw).init()
    e3 = np.broadcast_to(e2, (nz, ny, nx)).copy()
    k3 = np.broadcast_to(k2, (nz, ny, nx)).copy()
    o3 = oracle.Oracle(oracle.D3Q27, e3, k3, J_eta=2.0 / 3.0, **kw).init()
    o2.step(150)
    o3.step(150)
    r2, v2 = o2.moments()
    r3, v3 = o3.moments()
    for zz in range(nz):
        np.testing.assert_allclose(r3[zz], r2[0], rtol=1e-13)
        np.testing.assert_allclose(v3[:2, zz], v2[:2, 0], rtol=1e-9, atol=1e-16)
    assert np.max(np.abs(v3[2])) < 1e-15


# --------------------------------------------------------------- inlet / outlet planes

PLANE_SCHEMES = [oracle.PLANES_NEEM, oracle.PLANES_EQUILIBRIUM, oracle.PLANES_TMS]


@pytest.mark.parametrize("scheme", PLANE_SCHEMES)
def test_inlet_outlet_channel_develops_plane_poiseuille(scheme):
    """Velocity inlet (uniform U) and pressure outlet (rho = 1) planes, rebuilt by
    the boundary density of Eq. (bc_density_impermWall) and each reconstruction
    of Sec. 3.4 (non-equilibrium extrapolation Eq. (NEEM_bc_f_bar), the
    equilibrium scheme Eq. (eq_bc_f_bar), Tamm--Mott-Smith Eq. (f_i_neq_TMS)), on
    a free channel between halfway bounce-back walls: near steady state the node
    mass flux is the same through every cross-section of the upstream half (the
    outlet carries a thin boundary layer of ~0.3 % in the node flux), the
    developed profile is plane Poiseuille flow with the local mean velocity, the
    inlet nodes carry the prescribed velocity and the outlet holds its
    prescribed density."""
    ny, nx, U, nu = 16, 80, 0.02, 0.1
    e = np.ones((1, ny, nx))
    k = np.full_like(e, INF)
    o = oracle.Oracle(oracle.D2Q9, e, k, nu_f=nu, wall=(2, 1, 0), v_in=(U, 0, 0), rho_out=1.0,
                      plane_scheme=scheme).init()
    rho, v = _steady(o, check_every=2000, tol=1e-7, max_steps=20000)
    flux = (rho * v[0])[0].sum(axis=0)
    assert np.max(np.abs(flux[: nx // 2] - flux[0])) / flux[0] < 1e-4
    assert flux[0] / (ny * U) == pytest.approx(rho[0, :, 0].mean(), rel=1e-6)
    eta = np.arange(ny) + 0.5
    for x in (30, 50):
        prof = v[0, 0, :, x]
        ref = 6 * prof.mean() * eta * (ny - eta) / ny**2
        assert np.max(np.abs(prof - ref)) / ref.max() < 5e-3
    np.testing.assert_allclose(v[0, 0, :, 0], U, rtol=1e-2)
    np.testing.assert_allclose(rho[0, :, nx - 1], 1.0, atol=1e-3)


@pytest.mark.parametrize("scheme", PLANE_SCHEMES)
def test_plane_schemes_enforce_the_boundary_targets(scheme):
    """Every reconstruction gives the boundary node the zeroth and first moments
    of 1.5 f_tgt - 0.5 f_*: the non-equilibrium parts it adds carry no mass and
    no momentum (for TMS by construction, Sec. 3.4).  Read back through the
    moments of Eqs. (density_moment), (v_(0))-(v_final) -- the drag solve of
    Eq. (v_(1)) inverts the half-step shift exactly, and the porosity is uniform
    at the planes -- the inlet nodes carry exactly the prescribed velocity and
    the outlet nodes exactly the prescribed density, in any transient state:
    a free D2Q9 channel and a D3Q27 channel with a porous inlet section, an
    oblique inlet velocity, Forchheimer drag and a body force."""
    ny, nx, U = 16, 40, 0.02
    e = np.ones((1, ny, nx))
    k = np.full_like(e, INF)
    o = oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.1, wall=(2, 1, 0), v_in=(U, 0, 0), rho_out=1.0,
                      plane_scheme=scheme).init()
    o.step(300)
    rho, v = o.moments()
    assert np.max(np.abs(v[0, 0, :, 0] - U)) < 1e-14
    assert np.max(np.abs(v[1, 0, :, 0])) < 1e-14
    assert np.max(np.abs(rho[0, :, nx - 1] - 1.0)) < 1e-14
    e3 = np.full((6, 10, 24), 0.7)
    k3 = np.full_like(e3, 0.5)
    e3[:, :, -4:] = 1.0
    k3[:, :, -4:] = INF
    vin = (0.01, 0.002, 0.0)
    o3 = oracle.Oracle(oracle.D3Q27, e3, k3, nu_f=0.05, wall=(2, 1, 0), v_in=vin, rho_out=1.0, forch=0.3,
                       b=(1e-4, 0, 0), plane_scheme=scheme).init()
    o3.step(60)
    r3, v3 = o3.moments()
    for a in range(3):
        assert np.max(np.abs(v3[a, :, :, 0] - vin[a])) < 1e-14
    assert np.max(np.abs(r3[:, :, -1] - 1.0)) < 1e-14


@pytest.mark.parametrize("scheme", PLANE_SCHEMES)
def test_plane_schemes_keep_uniform_flow(scheme):
    """Uniform free flow at the inlet velocity and outlet density is an exact
    steady state (all populations at the equilibrium): every reconstruction
    must leave it unchanged."""
    e = np.ones((1, 8, 20))
    k = np.full_like(e, INF)
    o = oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.1, wall=(2, 0, 0), v_in=(0.03, 0, 0), rho_out=1.0,
                      plane_scheme=scheme).init(v0=(0.03, 0, 0))
    f0 = o.get_f()
    o.step(50)
    assert np.max(np.abs(o.get_f() - f0)) < 1e-15


def test_plane_schemes_differ_off_equilibrium():
    """In a developing flow the three reconstructions give different boundary
    populations (each scheme's own code runs)."""
    ny, nx = 12, 30
    e = np.ones((1, ny, nx))
    k = np.full_like(e, INF)
    fs = []
    for scheme in PLANE_SCHEMES:
        o = oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.1, wall=(2, 1, 0), v_in=(0.02, 0, 0), rho_out=1.0,
                          plane_scheme=scheme).init()
        o.step(100)
        fs.append(o.get_f()[:, 0, :, 0])
    for a in range(3):
        for b in range(a + 1, 3):
            assert np.max(np.abs(fs[a] - fs[b])) > 1e-6


def test_inlet_outlet_requires_uniform_plane_layers():
    ny, nx = 8, 12
    e = np.ones((1, ny, nx))
    k = np.full_like(e, INF)
    e[0, 3, 1] = 0.9
    k[0, 3, 1] = 1.0
    with pytest.raises(ValueError):
        oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.1, wall=(2, 1, 0), v_in=(0.01, 0, 0))


# --------------------------------------------------------------- moving wet-node walls: Couette flow (Sec. 5.1)

def test_couette_free_fluid_is_linear():
    """eps = 1, no force: wet-node walls at y = 0 and y = ny-1 moving with -V0
    and +V0 (density by continuity, Eq. (bc_density_impermWall), populations by
    Eq. (NEEM_bc_f_bar)) hold the linear Couette profile, which the lattice
    represents exactly, at steady state."""
    ny, V0 = 17, 0.01
    e = np.ones((1, ny, 4))
    k = np.full_like(e, INF)
    o = oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.1, wall=(0, 3, 0), wall_v=((-V0, 0, 0), (V0, 0, 0))).init()
    rho, v = _steady(o, check_every=2000, tol=1e-12)
    y = np.arange(ny)
    ref = np.broadcast_to((-V0 + 2 * V0 * y / (ny - 1))[:, None], v[0, 0].shape)
    np.testing.assert_allclose(v[0, 0], ref, rtol=0, atol=1e-12 * V0)
    assert np.max(np.abs(v[1])) < 1e-14
    np.testing.assert_allclose(rho, 1.0, atol=1e-13)


@pytest.mark.parametrize("g", [0.0, 1e-3])
def test_couette_darcy_limit_with_gravity(g):
    """Homogeneous porous Couette channel (eps = 0.5, Da = 1e-2, Forchheimer
    off) under gravity b = (0, -g): at steady state the velocity follows the
    Darcy-limit closed form Eq. (Couette_v_Darcy_analyt) of Eq.
    (Couette_v_ODE) and the density the exponential profile Eq.
    (Couette_rho_analyt) with the computed mean density.  H = 64 resolves the
    Brinkman layer (decay length sqrt(nu_eff / mu_D) = 9 nodes) to 0.2 %."""
    H, V0, eps, nu, RT = 64, 0.01, 0.5, 0.1, 1.0 / 3.0
    ny = H + 1
    kap = 1e-2 * H * H
    e = np.full((1, ny, 4), eps)
    k = np.full_like(e, kap)
    y = np.arange(ny)
    rho_init = np.broadcast_to(analytic.couette_density(y, H, 1.0, g, RT)[None, :, None], e.shape)
    o = oracle.Oracle(oracle.D2Q9, e, k, nu_f=nu, wall=(0, 3, 0), b=(0, -g, 0),
                      wall_v=((-V0, 0, 0), (V0, 0, 0)), forch=0.0).init(rho0=rho_init)
    rho, v = _steady(o, check_every=2000, tol=1e-12)
    vref = analytic.couette_darcy(y, H, -V0, V0, g, RT, eps * nu / kap, nu)
    assert np.max(np.abs(v[0, 0, :, 1] - vref)) / V0 < 3e-3
    r = rho[0, :, 1]
    rref = analytic.couette_density(y, H, np.trapezoid(r, y) / H, g, RT)
    assert np.max(np.abs(r - rref)) < 2e-6


def test_bounce_back_density_conserves_mass_exactly():
    """Eq. (bc_density_BounceBack): at a wall node the density of the known
    post-advection populations plus the reflected post-collision outgoing ones
    is exactly the mass bounce-back would leave there, and every reconstruction
    keeps the node's zeroth moment, so the total mass of a channel between
    moving porous walls (Forchheimer drag, gravity, a body force along x)
    stays constant to round-off; the density by mass continuity, Eq.
    (bc_density_impermWall), does not (1e-7 drift here)."""
    e = np.full((1, 20, 6), 0.6)
    k = np.full_like(e, 3.0)
    drift = {}
    for dens in (oracle.DENSITY_BOUNCE_BACK, oracle.DENSITY_CONTINUITY):
        o = oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.05, wall=(0, 3, 0), b=(1e-4, -1e-4, 0), forch=0.3,
                          wall_v=((0.01, 0, 0), (-0.02, 0, 0)), plane_density=dens).init()
        m0 = o.get_f().sum()
        o.step(800)
        drift[dens] = abs(o.get_f().sum() - m0) / m0
    assert drift[oracle.DENSITY_BOUNCE_BACK] < 1e-13
    assert drift[oracle.DENSITY_CONTINUITY] > 1e-10


@pytest.mark.parametrize("dens", [oracle.DENSITY_CONTINUITY, oracle.DENSITY_BOUNCE_BACK])
def test_poiseuille_between_wet_walls_at_rest(dens):
    """Free fluid driven by b along x between wet-node walls at rest on the node
    rows y = 0 and y = H: plane Poiseuille flow b y (H - y) / (2 nu) to the
    lattice's O(1/H^2) accuracy (0.6 % at H = 16, 0.16 % at H = 32), uniform
    density, with either boundary density."""
    for H, tol in ((16, 7e-3), (32, 1.8e-3)):
        ny, b, nu = H + 1, 1e-5, 0.1
        e = np.ones((1, ny, 4))
        k = np.full_like(e, INF)
        o = oracle.Oracle(oracle.D2Q9, e, k, nu_f=nu, wall=(0, 3, 0), b=(b, 0, 0), plane_density=dens).init()
        rho, v = _steady(o, check_every=2000, tol=1e-12)
        y = np.arange(ny)
        ref = b * y * (H - y) / (2 * nu)
        assert np.max(np.abs(v[0, 0, :, 0] - ref)) / ref.max() < tol
        np.testing.assert_allclose(rho, 1.0, atol=1e-11)


def test_moving_walls_need_periodic_sides_and_tangential_motion():
    e = np.ones((1, 12, 8))
    k = np.full_like(e, INF)
    with pytest.raises(ValueError):
        oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.1, wall=(1, 3, 0), wall_v=((0.01, 0, 0), (0, 0, 0)))
    with pytest.raises(ValueError):
        oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.1, wall=(0, 3, 0), wall_v=((0.0, 0.01, 0), (0, 0, 0)))


# --------------------------------------------------------------- channel past a porous cylinder (Sec. 6.1)

def _poiseuille_inlet(ny, V0):
    """Eq. (cylinder_inlet_BC) on the node rows between wet-node walls at y = 0, ny - 1."""
    eta = np.arange(ny) / (ny - 1)
    return 6.0 * V0 * eta * (1.0 - eta)


@pytest.mark.parametrize("outlet", [oracle.OUTLET_PRESSURE, oracle.OUTLET_ZERO_GRADIENT])
@pytest.mark.parametrize("scheme", PLANE_SCHEMES)
def test_poiseuille_inlet_walls_and_corners_hold_targets(scheme, outlet):
    """Inlet/outlet planes meeting wet-node walls at rest (Sec. 6.1): in any
    transient the inlet nodes carry exactly the Poiseuille profile of Eq.
    (cylinder_inlet_BC), the wall rows -- corners included -- exactly zero
    velocity, and each corner the density of its diagonal bulk neighbour (the
    corner density extrapolated from neighbouring bulk fluid nodes); the
    non-equilibrium parts the reconstructions add carry no mass or momentum.  A
    porous section with Forchheimer drag sits in the middle of the channel."""
    ny, nx, V0 = 14, 36, 0.03
    e = np.ones((1, ny, nx))
    k = np.full_like(e, INF)
    e[0, 4:10, 14:22] = 0.6
    k[0, 4:10, 14:22] = 0.8
    o = oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.08, wall=(2, 3, 0), forch=0.3, plane_scheme=scheme,
                      v_in=(V0, 0, 0), rho_out=1.0, inlet_profile=oracle.INLET_POISEUILLE, outlet=outlet).init()
    o.step(150)
    rho, v = o.moments()
    prof = _poiseuille_inlet(ny, V0)
    assert np.max(np.abs(v[0, 0, 1:-1, 0] - prof[1:-1])) < 1e-14
    assert np.max(np.abs(v[1, 0, :, 0])) < 1e-14
    for y, yi in ((0, 1), (ny - 1, ny - 2)):
        assert np.max(np.abs(v[:, 0, y, :])) < 1e-14
        assert abs(rho[0, y, 0] - rho[0, yi, 1]) < 1e-14
        assert abs(rho[0, y, nx - 1] - rho[0, yi, nx - 2]) < 1e-14
    if outlet == oracle.OUTLET_PRESSURE:
        assert np.max(np.abs(rho[0, 1:-1, nx - 1] - 1.0)) < 1e-14
    # the entering populations of the zero-gradient outlet are its neighbour's
    if outlet == oracle.OUTLET_ZERO_GRADIENT:
        o2 = oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.08, wall=(2, 3, 0), forch=0.3, plane_scheme=scheme,
                           v_in=(V0, 0, 0), inlet_profile=oracle.INLET_POISEUILLE, outlet=outlet).init()
        o2.step(150)
        f = o2.get_f()
        w, c = o2.lattice()
        for i in range(9):
            if c[i][0] < 0:
                np.testing.assert_array_equal(f[i, 0, 1:-1, nx - 1], f[i, 0, 1:-1, nx - 2])


@pytest.mark.parametrize("scheme", PLANE_SCHEMES)
def test_zero_gradient_outflow_keeps_uniform_flow(scheme):
    """Uniform free flow at the inlet velocity is an exact steady state of the
    zero-gradient outflow, Eq. (f_bar_outflow_BC): every population of the
    outlet's neighbour is already the outlet's."""
    e = np.ones((1, 8, 20))
    k = np.full_like(e, INF)
    o = oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.1, wall=(2, 0, 0), v_in=(0.03, 0, 0), plane_scheme=scheme,
                      outlet=oracle.OUTLET_ZERO_GRADIENT).init(v0=(0.03, 0, 0))
    f0 = o.get_f()
    o.step(50)
    assert np.max(np.abs(o.get_f() - f0)) < 1e-15


def test_porous_cylinder_channel_conserves_section_flux():
    """The confined channel past a porous cylinder (Sec. 6.1) at D = 6, Re = 10,
    eps_core = 0.5, with the pressure outlet (rho = 1): at steady state the mass
    flux sum_y rho v_x through a cross-section far downstream equals the
    inlet's to 1e-5 -- the mass that passes through the porous cylinder
    (superficial velocity) is not lost -- and differs from it by less than
    2e-3 anywhere (the moments omit the link flux of the rebuilt wall rows where
    the near-wall flow varies along x: 1.7e-3 beside the cylinder, decaying
    downstream); the velocity is zero on the wall rows and the flow through the
    cylinder is slowed."""
    D, V0, Re = 6, 0.05, 10.0
    e, k = workloads.porous_cylinder(D=D, eps_core=0.5)
    ny, nx = e.shape[1:]
    o = oracle.Oracle(oracle.D2Q9, e, k, nu_f=V0 * D / Re, wall=(2, 3, 0), forch=-1.0, v_in=(V0, 0, 0),
                      rho_out=1.0, inlet_profile=oracle.INLET_POISEUILLE).init()
    rho, v = _steady(o, check_every=2000, tol=1e-10, max_steps=60000)
    flux = (rho[0] * v[0, 0]).sum(axis=0)
    dev = np.abs(flux - flux[0]) / flux[0]
    assert np.max(dev[100:-1]) < 1e-5
    assert np.max(dev) < 2e-3
    assert flux[0] == pytest.approx((rho[0, :, 0] * _poiseuille_inlet(ny, V0)).sum(), rel=1e-14)
    assert np.max(np.abs(v[:, 0, [0, ny - 1], :])) < 1e-14
    xc, yc = 2 * D, 2 * D
    assert v[0, 0, yc, xc] < 0.5 * _poiseuille_inlet(ny, V0)[yc]


def test_zero_gradient_outflow_has_no_mass_anchor():
    """Eq. (f_bar_outflow_BC) with a velocity inlet fixes no density level, and
    every boundary rule is homogeneous in rho: with periodic y the mean density
    of a developing channel settles, but between walls the flow needs a density
    drop along x against the wall friction, the inlet brings rho_in v_in in,
    the copied outlet lets less out, and the density grows by a fixed factor
    per step (the velocity field is unchanged) -- about 11 % per 4000 steps at
    H = 25, nu = 0.03; the pressure outlet anchors it."""
    def mean_rho_ratio(walls, outlet):
        e = np.ones((1, 26, 60))
        k = np.full_like(e, INF)
        o = oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.03, wall=walls, v_in=(0.05, 0, 0), rho_out=1.0,
                          outlet=outlet).init()
        o.step(6000)
        r1, v1 = o.moments()
        o.step(4000)
        r2, v2 = o.moments()
        return r2.mean() / r1.mean(), np.max(np.abs(v2 - v1))
    ratio, dv = mean_rho_ratio((2, 0, 0), oracle.OUTLET_ZERO_GRADIENT)
    assert abs(ratio - 1.0) < 1e-9
    ratio, dv = mean_rho_ratio((2, 3, 0), oracle.OUTLET_ZERO_GRADIENT)
    assert 1.05 < ratio < 1.2 and dv < 1e-6
    ratio, dv = mean_rho_ratio((2, 3, 0), oracle.OUTLET_PRESSURE)
    assert abs(ratio - 1.0) < 2e-3  # still relaxing, but bounded


def test_porous_cylinder_profile():
    """Eqs. (s_cylinder_circle)-(b_cinf): eps_core at the centre, eps = 1 where
    s >= 1, and the eps_50 = (1 + eps_core)/2 isocontour has the diameter
    D_50 ~= 0.64 D that the paper prints; permeability from Eq. (kappa_Ergun)
    with d_p = D/5, infinite in the free fluid."""
    D, core = 40, 0.3
    e, k = workloads.porous_cylinder(D=D, eps_core=core)
    assert e.shape == (1, 165, 881)
    assert e[0, 2 * D, 2 * D] == pytest.approx(core, abs=1e-15)
    y, x = np.meshgrid(np.arange(165), np.arange(881), indexing="ij")
    s = (2 * (x - 2 * D) / D) ** 2 + (2 * (y - 2 * D) / D) ** 2
    assert np.all(e[0][s >= 1] == 1.0) and np.all(np.isinf(k[0][s >= 1]))
    assert np.all(e[0] <= 1.0) and np.all(e[0][s < 0.9] < 1.0)  # the bump is flat to round-off as s -> 1
    row = e[0, 2 * D]
    e50 = 0.5 * (1 + core)
    i = np.where(row < e50)[0]
    lo, hi = i.min(), i.max()
    xl = lo - 1 + (row[lo - 1] - e50) / (row[lo - 1] - row[lo])
    xr = hi + (row[hi] - e50) / (row[hi] - row[hi + 1])
    assert (xr - xl) / D == pytest.approx(0.64, abs=0.005)
    dp = D / 5
    inside = e[0] < 1.0
    np.testing.assert_allclose(k[0][inside], dp**2 * e[0][inside] ** 3 / (150 * (1 - e[0][inside]) ** 2), rtol=1e-14)


def test_inlet_profile_and_outlet_kind_validation():
    e = np.ones((1, 12, 16))
    k = np.full_like(e, INF)
    with pytest.raises(ValueError):  # the Poiseuille profile spans walls on y
        oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.1, wall=(2, 0, 0), v_in=(0.01, 0, 0),
                      inlet_profile=oracle.INLET_POISEUILLE)
    with pytest.raises(ValueError):  # outlet kinds belong to inlet/outlet planes
        oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.1, wall=(0, 3, 0), outlet=oracle.OUTLET_ZERO_GRADIENT)
    with pytest.raises(ValueError):
        oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.1, wall=(2, 1, 0), outlet=2)
    oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.1, wall=(2, 1, 0), v_in=(0.01, 0, 0),
                  inlet_profile=oracle.INLET_POISEUILLE)
    oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.1, wall=(2, 3, 0), v_in=(0.01, 0, 0),
                  inlet_profile=oracle.INLET_POISEUILLE, outlet=oracle.OUTLET_ZERO_GRADIENT)


# --------------------------------------------------------------- lid-driven cavity with a porous obstacle (Sec. 6.2)

def _smoothstep(psi):
    """Eq. (s_cinf)."""
    psi = np.asarray(psi, dtype=np.float64)
    out = np.where(psi >= 1.0, 1.0, 0.0)
    mid = (psi > 0) & (psi < 1)
    a = np.exp(-1.0 / psi[mid])
    b = np.exp(-1.0 / (1.0 - psi[mid]))
    out[mid] = a / (a + b)
    return out


def _cavity(L, V0, nu, eps_core=1.0, scheme=0, density=oracle.DENSITY_BOUNCE_BACK, D=None, forch=-1.0):
    e, k = workloads.porous_cavity(L=L, D=D if D else 0.55 * L, eps_core=eps_core)
    return oracle.Oracle(oracle.D2Q9, e, k, nu_f=nu, wall=(3, 3, 0), forch=forch, plane_scheme=scheme,
                         plane_density=density, wall_v=((0, 0, 0), (V0, 0, 0)),
                         lid_profile=oracle.LID_REGULARISED, lid_delta=0.1).init()


@pytest.mark.parametrize("density", [oracle.DENSITY_BOUNCE_BACK, oracle.DENSITY_CONTINUITY])
@pytest.mark.parametrize("scheme", PLANE_SCHEMES)
def test_cavity_walls_and_regularised_lid_hold_targets(scheme, density):
    """Wet-node walls on all four sides (Eq. (cavity_BC)): in any transient the
    side walls and the bottom carry exactly zero velocity and the lid exactly
    V0 S(min(x, L - x) / (delta L)), Eq. (cavity_velocity_profile), corners
    included; the profile is V0 over the central 80 % of the lid (delta = 0.1),
    vanishes at both corners and is mirror-symmetric."""
    L, V0 = 30, 0.05
    o = _cavity(L, V0, 0.1, eps_core=0.6, scheme=scheme, density=density)
    o.step(200)
    rho, v = o.moments()
    x = np.arange(L + 1)
    lid = V0 * _smoothstep(np.minimum(x, L - x) / (0.1 * L))
    assert np.max(np.abs(v[0, 0, L, :] - lid)) < 1e-14
    assert np.max(np.abs(v[1, 0, L, :])) < 1e-14
    assert np.max(np.abs(v[:, 0, 0, :])) < 1e-14
    assert np.max(np.abs(v[:, 0, :L, 0])) < 1e-14 and np.max(np.abs(v[:, 0, :L, L])) < 1e-14
    plateau = (x >= 3) & (x <= L - 3)
    assert np.max(np.abs(v[0, 0, L, plateau] - V0)) < 1e-14
    assert abs(v[0, 0, L, 0]) < 1e-14 and abs(v[0, 0, L, L]) < 1e-14
    np.testing.assert_allclose(v[0, 0, L, :], v[0, 0, L, ::-1], rtol=0, atol=1e-15)
    assert _smoothstep(np.array([0.5]))[0] == pytest.approx(0.5, abs=1e-15)


def test_cavity_bounce_back_density_conserves_mass():
    """A closed cavity with a porous core (eps_core = 0.5, Ergun drag) whose four
    wet-node walls take the bounce-back density, Eq. (bc_density_BounceBack) --
    the set-up of Sec. 6.2 --, including its corners: the total mass stays
    constant to round-off; with the density by mass continuity it drifts."""
    drift = {}
    for dens in (oracle.DENSITY_BOUNCE_BACK, oracle.DENSITY_CONTINUITY):
        o = _cavity(30, 0.05, 0.05, eps_core=0.5, density=dens)
        m0 = o.get_f().sum()
        o.step(1500)
        drift[dens] = abs(o.get_f().sum() - m0) / m0
    assert drift[oracle.DENSITY_BOUNCE_BACK] < 1e-13
    assert drift[oracle.DENSITY_CONTINUITY] > 1e-10


def test_cavity_stokes_flow_is_mirror_symmetric():
    """Creeping flow (Re = 0.1): the steady Stokes problem with the symmetric
    regularised lid is reversible under x -> L - x (v_x even, v_y odd), and the
    mirror asymmetry of the lattice solution is the inertial part, O(Re): ten
    times smaller at Re = 0.1 than at Re = 1."""
    L, nu = 24, 0.1
    asym = {}
    for Re in (0.1, 1.0):
        o = _cavity(L, Re * nu / L, nu)
        rho, v = _steady(o, check_every=2000, tol=1e-11, max_steps=60000)
        vx, vy = v[0, 0], v[1, 0]
        scale = np.max(np.abs(vx))
        asym[Re] = max(np.max(np.abs(vx - vx[:, ::-1])), np.max(np.abs(vy + vy[:, ::-1]))) / scale
    assert asym[0.1] < 0.15 * asym[1.0]
    assert asym[0.1] < 1e-2


def test_porous_core_weakens_the_flow_through_the_obstacle():
    """At Re = 10 the superficial speed at the cavity centre drops as the core
    porosity (and with it the Ergun permeability) decreases (Sec. 6.2)."""
    L = 24
    nu = workloads.cavity_viscosity(L, 10.0)
    speed = []
    for core in (1.0, 0.8, 0.5):
        o = _cavity(L, 10.0 * nu / L, nu, eps_core=core)
        rho, v = _steady(o, check_every=2000, tol=1e-9, max_steps=40000)
        speed.append(np.hypot(v[0, 0, L // 2, L // 2], v[1, 0, L // 2, L // 2]))
    assert speed[0] > speed[1] > speed[2]


def test_porous_cavity_profile():
    """Eq. (Cavity_Porosity_Profile): eps_core at the centre, eps = 1 outside the
    superellipse s_se >= 1, and the eps_50 isocontour has the diameter
    D_50 ~= 0.8 D that the paper prints; Ergun permeability with d_p = D/5."""
    L, D, core = 300, 165, 0.4
    e, k = workloads.porous_cavity(L=L, D=D, eps_core=core)
    assert e.shape == (1, L + 1, L + 1)
    assert e[0, L // 2, L // 2] == pytest.approx(core, abs=1e-15)
    row = e[0, L // 2]
    e50 = 0.5 * (1 + core)
    i = np.where(row < e50)[0]
    lo, hi = i.min(), i.max()
    xl = lo - 1 + (row[lo - 1] - e50) / (row[lo - 1] - row[lo])
    xr = hi + (row[hi] - e50) / (row[hi] - row[hi + 1])
    assert (xr - xl) / D == pytest.approx(0.8, abs=0.005)
    assert np.all(e[0, :, 0] == 1.0) and np.all(np.isinf(k[0, :, 0]))
    inside = e[0] < 1.0
    dp = D / 5
    np.testing.assert_allclose(k[0][inside], dp**2 * e[0][inside] ** 3 / (150 * (1 - e[0][inside]) ** 2), rtol=1e-14)
    assert workloads.cavity_viscosity(300, 100.0) == 0.1
    assert workloads.cavity_viscosity(300, 1000.0) == pytest.approx(300 * np.sqrt(1 / 3) / 4000)


@pytest.mark.parametrize("dens", [oracle.DENSITY_CONTINUITY, oracle.DENSITY_BOUNCE_BACK])
def test_poiseuille_between_wet_side_walls(dens):
    """Free fluid driven by b along y between wet-node walls at rest on the node
    columns x = 0 and x = H (y periodic): plane Poiseuille flow b x (H - x) /
    (2 nu), to the lattice's O(1/H^2) accuracy (0.6 % at H = 16), and the same
    profile as between wet walls on y -- the x-wall rule is the y-wall rule
    turned by a quarter."""
    H, b, nu = 16, 1e-5, 0.1
    e = np.ones((1, 4, H + 1))
    k = np.full_like(e, INF)
    o = oracle.Oracle(oracle.D2Q9, e, k, nu_f=nu, wall=(3, 0, 0), b=(0, b, 0), plane_density=dens).init()
    rho, v = _steady(o, check_every=2000, tol=1e-12)
    x = np.arange(H + 1)
    ref = b * x * (H - x) / (2 * nu)
    assert np.max(np.abs(v[1, 0, 1, :] - ref)) / ref.max() < 7e-3
    et = np.ones((1, H + 1, 4))
    kt = np.full_like(et, INF)
    ot = oracle.Oracle(oracle.D2Q9, et, kt, nu_f=nu, wall=(0, 3, 0), b=(b, 0, 0), plane_density=dens).init()
    rt, vt = _steady(ot, check_every=2000, tol=1e-12)
    np.testing.assert_allclose(v[1, 0, 1, :], vt[0, 0, :, 1], rtol=1e-9, atol=1e-15)
    assert np.max(np.abs(v[0])) < 1e-15


def test_oracle_result_does_not_depend_on_threads():
    """The oracle's node loops are independent per node: one thread and all
    threads give the same populations bit for bit."""
    eps = workloads.random_smooth_porosity((6, 10, 12), seed=7, lo=0.5, hi=0.95)
    kap = workloads.carman_kappa(eps, 2.0)
    n0 = oracle.threads()
    out = []
    for n in (1, max(n0, 2)):
        oracle.set_threads(n)
        o = oracle.Oracle(oracle.D3Q27, eps, kap, nu_f=0.05, b=(1e-4, 0, 0), forch=0.3, wall=(0, 1, 1)).init()
        o.step(20)
        out.append(o.get_f())
    oracle.set_threads(n0)
    np.testing.assert_array_equal(out[0], out[1])


def test_cavity_validation():
    e = np.ones((1, 12, 12))
    k = np.full_like(e, INF)
    with pytest.raises(ValueError):  # the regularised lid needs wet side walls
        oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.1, wall=(0, 3, 0), lid_profile=oracle.LID_REGULARISED)
    with pytest.raises(ValueError):
        oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.1, wall=(3, 3, 0), lid_profile=oracle.LID_REGULARISED,
                      lid_delta=0.0)
    with pytest.raises(ValueError):  # wet side walls with bounce-back y walls
        oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.1, wall=(3, 1, 0))
    oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.1, wall=(3, 0, 0))
    oracle.Oracle(oracle.D2Q9, e, k, nu_f=0.1, wall=(3, 3, 0), lid_profile=oracle.LID_REGULARISED)


# --------------------------------------------------------------- Picard iteration (Appendix F)

def _implicit_velocity_residual(o, eps, b, muD, muF, geps, v, RT=1.0 / 3.0):
    """c1 v + c2 |v| v - v(0) - Delta_nu(rho v / eps) / (2 rho), from the populations."""
    w, c = o.lattice()
    f = o.get_f()
    rho = f.sum(axis=0) / eps
    P1 = np.einsum("ia,i...->a...", c.astype(float), f)
    v0 = P1 / rho + 0.5 * (eps * np.asarray(b)[:, None, None, None] + RT * geps)
    dnu = o.delta_nu(rho * v / eps)
    nv = np.sqrt((v**2).sum(axis=0))
    c1, c2 = 1 + 0.5 * muD, 0.5 * muF
    return c1 * v + c2 * nv * v - v0 - dnu / (2 * rho)


def test_picard_iteration_solves_the_implicit_velocity_equation():
    """With enough Picard iterations the velocity solves the implicit equation of
    Appendix F (checked with Delta_nu applied to the returned velocity); the
    one-shot velocity of Eq. (v_final) does not, and for uniform porosity both
    coincide."""
    shape = (10, 12, 14)
    eps = workloads.random_smooth_porosity(shape, seed=17, lo=0.4, hi=0.95, ell=2.0)
    kap = workloads.carman_kappa(eps, 2.0)
    b = (3e-4, -1e-4, 2e-4)
    kw = dict(nu_f=0.05, b=b, forch=-1.0)
    base = oracle.Oracle(oracle.D3Q27, eps, kap, **kw).init()
    base.step(40)
    f = base.get_f()
    muD, muF, geps, _ = base.static()
    _, v_one = base.moments()
    pic = oracle.Oracle(oracle.D3Q27, eps, kap, picard_iters=40, **kw)
    pic.set_f(f)
    _, v_pic = pic.moments()
    r_one = _implicit_velocity_residual(base, eps, b, muD, muF, geps, v_one)
    r_pic = _implicit_velocity_residual(pic, eps, b, muD, muF, geps, v_pic)
    scale = np.abs(v_pic).max()
    assert np.abs(r_pic).max() < 1e-10 * scale
    assert np.abs(r_one).max() > 1e-5 * scale
    # under-relaxed iteration reaches the same fixed point
    half = oracle.Oracle(oracle.D3Q27, eps, kap, picard_iters=120, picard_omega=0.5, **kw)
    half.set_f(f)
    _, v_half = half.moments()
    np.testing.assert_allclose(v_half, v_pic, rtol=0, atol=1e-9 * scale)
    # uniform porosity: Delta_nu vanishes and the iteration changes nothing
    e1, k1 = np.full(shape, 0.6), np.full(shape, 0.3)
    u1 = oracle.Oracle(oracle.D3Q27, e1, k1, **kw).init().step(10)
    u2 = oracle.Oracle(oracle.D3Q27, e1, k1, picard_iters=5, **kw)
    u2.set_f(u1.get_f())
    np.testing.assert_array_equal(u2.moments()[1], u1.moments()[1])
