"""Pins of the oracle's whole step, its initial state and its RT grad(eps) term.

* The whole step against a second statement of the method written
  independently in NumPy (``np_lbm.py``, from Sec. 3 and the flowchart of
  Sec. 3.5): initial populations and three steps on tiny random grids with
  walls, D2Q9 and D3Q27, every correction on, Ergun and scalar Forchheimer
  drag, free-fluid nodes, RT != 1/3, J_nu, J_eta != 1.  An error in the order
  of the sweeps, a stencil, a bounce-back slot or a sign in either statement
  shows up as an O(1e-3) difference; the two agree to rounding.
* The initial state, Eq. (eq_bc_f_bar) with lambda = 1: its moments are the
  closed forms of Eqs. (transformed_density_moment) and
  (transformed_momentum_moment), eps rho0 and rho0 v0 - rho0 a0 / 2, with a0
  of Eq. (accel) on the initial fields (computed by the NumPy statement).
* The RT grad(eps) term of Eqs. (v_(0)) and (accel): a force-free box with a
  smooth heterogeneous porosity must come to rest with a uniform density (the
  continuum balance is -RT eps grad rho = 0).  The discrete rest state keeps an
  O(h^2) density non-uniformity; the pin asserts second-order convergence of
  it.  With the term's sign flipped the density would settle near eps^-2, and
  with the term dropped near 1/eps: an O(1) spread that does not converge
  (measured on mutated copies of the oracle: spread 1.17 and 0.58 at L = 16,
  against 0.030 for the correct term).
"""
import numpy as np
import pytest

import oracle
from np_lbm import NpLBM

CASES = [
    # lattice, shape (nz, ny, nx), walls (x, y, z), forchheimer
    (2, (1, 4, 3), (0, 1, 0), -1.0),
    (2, (1, 4, 5), (1, 1, 0), 0.3),
    (3, (4, 4, 4), (1, 0, 1), -1.0),
    (3, (4, 5, 3), (0, 1, 0), 0.2),
]


def _random_case(D, shape, wall, forch, seed):
    rng = np.random.default_rng(seed)
    eps = rng.uniform(0.4, 1.0, shape)
    kap = rng.uniform(0.5, 5.0, shape)
    kap[rng.random(shape) < 0.3] = np.inf
    kw = dict(nu_f=0.07, b=(2e-3, -1e-3, 1.5e-3), forch=forch, RT=0.3, J_nu=1.3, J_eta=0.7, wall=wall)
    rho0 = rng.uniform(0.9, 1.1, shape)
    v0 = rng.uniform(-0.02, 0.02, (3,) + shape)
    if D == 2:
        v0[2] = 0.0
    return eps, kap, kw, rho0, v0


@pytest.mark.parametrize("case", range(len(CASES)))
def test_whole_step_matches_independent_numpy_statement(case):
    D, shape, wall, forch = CASES[case]
    eps, kap, kw, rho0, v0 = _random_case(D, shape, wall, forch, seed=10 + case)
    lat = oracle.D2Q9 if D == 2 else oracle.D3Q27
    o = oracle.Oracle(lat, eps, kap, **kw).init(rho0, v0[:D])
    n = NpLBM(D, eps, kap, **kw).init(rho0, v0[:D])
    for k in range(4):
        fo, fn = o.get_f(), n.f
        err = np.abs(fo - fn).max() / np.abs(fo).max()
        assert err < 1e-14, f"after {k} steps: relative difference {err:.2e}"
        # the populations moved: the comparison is not of a fixed point
        if k:
            assert np.abs(fo - prev).max() > 1e-4 * np.abs(fo).max()
        prev = fo
        o.step(1)
        n.step(1)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_initial_state_moments(case):
    """Eq. (eq_bc_f_bar): sum f0 = eps rho0 and sum c f0 = rho0 v0 - rho0 a0 / 2."""
    D, shape, wall, forch = CASES[case]
    eps, kap, kw, rho0, v0 = _random_case(D, shape, wall, forch, seed=20 + case)
    lat = oracle.D2Q9 if D == 2 else oracle.D3Q27
    o = oracle.Oracle(lat, eps, kap, **kw).init(rho0, v0[:D])
    f = o.get_f()
    _, c = o.lattice()
    a0 = NpLBM(D, eps, kap, **kw).init(rho0, v0[:D]).a0
    np.testing.assert_allclose(f.sum(axis=0), eps * rho0, rtol=1e-14, atol=0)
    for a in range(D):
        mom = np.tensordot(c[:, a].astype(float), f, axes=(0, 0))
        ref = rho0 * v0[a] - 0.5 * rho0 * a0[a]
        assert np.abs(mom - ref).max() < 1e-15 + 1e-13 * np.abs(ref).max()
        # the acceleration term is not negligible in the comparison
        assert np.abs(0.5 * rho0 * a0[a]).max() > 1e-4


def _rest_box(L, D):
    x = (np.arange(L) + 0.5) / L
    if D == 2:
        X, Y = np.meshgrid(x, x, indexing="xy")
        eps = (0.7 + 0.2 * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y))[None]
    else:
        Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
        eps = 0.7 + 0.2 * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y) * np.sin(2 * np.pi * Z)
    o = oracle.Oracle(oracle.D2Q9 if D == 2 else oracle.D3Q27, eps, np.full_like(eps, 2.0), nu_f=0.1,
                      forch=-1.0).init()
    o.step(1000 if D == 2 else 500)
    rho, v = o.moments()
    return (rho.max() - rho.min()) / rho.mean(), np.abs(v).max()


@pytest.mark.parametrize("D,sizes", [(2, (16, 32, 64)), (3, (12, 24))])
def test_force_free_heterogeneous_box_comes_to_rest_with_uniform_density(D, sizes):
    spread, vmax = zip(*[_rest_box(L, D) for L in sizes])
    for k in range(1, len(sizes)):
        # second order: the spread falls ~4x per halving of the spacing
        assert spread[k - 1] / spread[k] > 3.4, spread
        assert vmax[k - 1] / vmax[k] > 8.0, vmax
    # an O(1) spread (flipped or dropped RT grad eps) is far above these
    assert spread[0] < 0.07 and spread[-1] < 0.02
    assert vmax[-1] < 1e-5
