"""Seeded synthetic inputs: porosity and permeability fields.

This module holds input generation only (random fields, geometry, the packed-bed
permeability correlation used to turn a porosity field into a permeability
field).  It contains none of the lattice Boltzmann arithmetic, so both the CUDA
path and the test oracle may draw their inputs from it.  All fields are numpy
arrays of shape (nz, ny, nx), x fastest; permeability +inf marks free fluid.
"""
from __future__ import annotations

import numpy as np


def gaussian_random_field(shape, ell, seed):
    """Periodic, zero-mean, unit-variance Gaussian field with covariance
    exp(-r^2 / (2 ell^2)): white noise filtered in Fourier space by
    exp(-k^2 ell^2 / 4), then standardised."""
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal(shape)
    ks = [np.fft.fftfreq(n) * 2.0 * np.pi for n in shape[:-1]] + [np.fft.rfftfreq(shape[-1]) * 2.0 * np.pi]
    k2 = np.zeros([len(k) for k in ks])
    for ax, k in enumerate(ks):
        sh = [1] * len(ks)
        sh[ax] = len(k)
        k2 = k2 + (k.reshape(sh)) ** 2
    axes = list(range(len(shape)))
    g = np.fft.irfftn(np.fft.rfftn(noise, axes=axes) * np.exp(-k2 * ell * ell / 4.0), s=shape, axes=axes)
    g -= g.mean()
    g /= g.std()
    return g


def _normal_cdf(g):
    from scipy.special import ndtr
    return ndtr(g)


def carman_kappa(eps, d, c=180.0):
    """Packed-bed permeability kappa = d^2 eps^3 / (c (1 - eps)^2); eps = 1 gives +inf
    (free fluid).  c = 150 is Ergun's constant, c = 180 the Carman-Kozeny one."""
    eps = np.asarray(eps, dtype=np.float64)
    with np.errstate(divide="ignore"):
        k = d * d * eps**3 / (c * (1.0 - eps) ** 2)
    return np.where(eps >= 1.0, np.inf, k)


def grf_porosity(shape, ell, seed, lo=0.35, free_above=0.99):
    """Porosity in [lo, 1] from a Gaussian random field through the normal CDF:
    eps = lo + (1 - lo) Phi(g).  Nodes with eps >= free_above become free fluid
    (eps = 1)."""
    g = gaussian_random_field(shape, ell, seed)
    eps = lo + (1.0 - lo) * _normal_cdf(g)
    return np.where(eps >= free_above, 1.0, eps)


def porous_box(shape, ell=16.0, seed=2, d=2.0):
    """Periodic box with Gaussian-random-field porosity in [0.35, 1] and
    Carman-Kozeny permeability with grain size d."""
    eps = grf_porosity(shape, ell, seed)
    return eps, carman_kappa(eps, d)


def layered_channel(nx=128, ny=64, eps_porous=0.5, Da=1e-3):
    """Two-layer channel: rows y < ny/2 porous (eps, kappa = Da H^2 with H = ny),
    rows above free fluid."""
    eps = np.ones((1, ny, nx))
    kappa = np.full((1, ny, nx), np.inf)
    eps[:, : ny // 2, :] = eps_porous
    kappa[:, : ny // 2, :] = Da * ny * ny
    return eps, kappa


def smoothstep(psi):
    """C-infinity step from 0 (psi <= 0) to 1 (psi >= 1): exp(-1/psi) / (exp(-1/psi) + exp(-1/(1-psi)))."""
    psi = np.asarray(psi, dtype=np.float64)
    inside = (psi > 0.0) & (psi < 1.0)
    p = np.where(inside, psi, 0.5)
    a = np.exp(-1.0 / p)
    b = np.exp(-1.0 / (1.0 - p))
    return np.where(inside, a / (a + b), np.where(psi <= 0.0, 0.0, 1.0))


def cube_channel(nx=512, ny=256, nz=256, side=128, eps_cube=0.4, Da=1e-4, smooth=0):
    """Free channel with a centred porous cube (kappa = Da side^2).  smooth > 0
    blends the porosity from the cube value to 1 over `smooth` nodes outside
    each face with the C-infinity smoothstep (a product over the three axes);
    the blended shell keeps the cube's permeability."""
    eps = np.ones((nz, ny, nx))
    kappa = np.full((nz, ny, nx), np.inf)
    x0, y0, z0 = (nx - side) // 2, (ny - side) // 2, (nz - side) // 2
    if smooth <= 0:
        sl = (slice(z0, z0 + side), slice(y0, y0 + side), slice(x0, x0 + side))
        eps[sl] = eps_cube
        kappa[sl] = Da * side * side
        return eps, kappa
    inside = np.ones((nz, ny, nx))
    for ax, (n, lo) in enumerate(((nz, z0), (ny, y0), (nx, x0))):
        c = np.arange(n) + 0.5
        dist = np.maximum(lo - c, c - (lo + side))  # > 0 outside the face pair
        w = 1.0 - smoothstep(dist / smooth)
        shape = [1, 1, 1]
        shape[ax] = n
        inside = inside * w.reshape(shape)
    eps = 1.0 - (1.0 - eps_cube) * inside
    kappa = np.where(inside > 0.0, Da * side * side, np.inf)
    eps = np.where(inside > 0.0, eps, 1.0)
    return eps, kappa


def slot_box(n=640, ell=16.0, seed=5, d=2.0, slot=64):
    """Porous box as porous_box, cut by a free slot of width `slot` in y that spans
    x and z at the y-centre."""
    eps = grf_porosity((n, n, n), ell, seed)
    y0 = (n - slot) // 2
    eps[:, y0:y0 + slot, :] = 1.0
    return eps, carman_kappa(eps, d)


def bump(s, m=1):
    """Localized generalized bump function B_m(s) of Eq. (b_cinf): exp(1 - 1/(1 - s^m))
    for s < 1, 0 for s >= 1 (all derivatives vanish at s = 1)."""
    s = np.asarray(s, dtype=np.float64)
    out = np.zeros_like(s)
    inside = s < 1.0
    out[inside] = np.exp(1.0 - 1.0 / (1.0 - s[inside] ** m))
    return out


def porous_cylinder(D=40, eps_core=0.5, H_over_D=4.1, L_over_D=22.0, centre=(2.0, 2.0), dp_over_D=0.2):
    """Confined channel past a porous cylinder (Sec. 6.1, after Schaefer et al.):
    the channel spans y in [0, H], H = 4.1 D, between wet-node walls on the node
    rows y = 0 and y = ny - 1, and x in [0, L], L = 22 D, between the inlet (x = 0)
    and outlet (x = nx - 1) planes.  Porosity eps = 1 - (1 - eps_core) B_1(s) with
    the normalized radius s = (2(x - xc)/D)^2 + (2(y - yc)/D)^2, Eqs.
    (s_cylinder_circle), (Porous_Cylinder_Profile), centre (xc, yc) = (2D, 2D);
    permeability from the Ergun correlation, Eq. (kappa_Ergun), with the particle
    diameter d_p = D / 5.  Returns (eps, kappa) of shape (1, ny, nx) (a 2D field)."""
    ny = int(round(H_over_D * D)) + 1
    nx = int(round(L_over_D * D)) + 1
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    xc, yc = centre[0] * D, centre[1] * D
    s = (2.0 * (x - xc) / D) ** 2 + (2.0 * (y - yc) / D) ** 2
    eps = 1.0 - (1.0 - eps_core) * bump(s, 1)
    kappa = carman_kappa(eps, dp_over_D * D, c=150.0)
    return eps[None], kappa[None]


def porous_cavity(L=300, D=165, eps_core=0.5, dp_over_D=0.2):
    """Lid-driven cavity with a porous obstacle (Sec. 6.2): wet-node walls on the
    node rows and columns 0 and L (L + 1 nodes a side), porosity
    eps = 1 + (eps_core - 1) B_1(s_se) with the superelliptic radius
    s_se = ((2x - L)/D)^4 + ((2y - L)/D)^4, Eq. (Cavity_Porosity_Profile), and the
    Ergun permeability of Eq. (kappa_Ergun) with d_p = D / 5.  Returns
    (eps, kappa) of shape (1, L + 1, L + 1)."""
    n = L + 1
    y, x = np.meshgrid(np.arange(n, dtype=np.float64), np.arange(n, dtype=np.float64), indexing="ij")
    s = ((2.0 * x - L) / D) ** 4 + ((2.0 * y - L) / D) ** 4
    eps = 1.0 + (eps_core - 1.0) * bump(s, 1)
    kappa = carman_kappa(eps, dp_over_D * D, c=150.0)
    return eps[None], kappa[None]


def cavity_viscosity(L, Re, RT=1.0 / 3.0):
    """Eq. (Cavity_nu): nu_f = min(0.1, L sqrt(RT) / (4 Re)); the lid speed is then
    V0 = Re nu_f / L."""
    return min(0.1, L * np.sqrt(RT) / (4.0 * Re))


def serving_request(k, sides=(32, 48, 64, 96, 128, 192)):
    """Request k of the serving stream: a periodic cube with side drawn from
    `sides`, mean porosity target m in U[0.4, 0.9], correlation length in
    U[4, 24].  eps = clip(m + 0.1 g, 0.1, 1)."""
    rng = np.random.default_rng(1000 + k)
    side = int(rng.choice(sides))
    m = float(rng.uniform(0.4, 0.9))
    ell = float(rng.uniform(4.0, 24.0))
    g = gaussian_random_field((side, side, side), ell, 1000 + k)
    eps = np.clip(m + 0.1 * g, 0.1, 1.0)
    return {"side": side, "mean_target": m, "ell": ell, "eps": eps, "kappa": carman_kappa(eps, 2.0)}


def random_smooth_porosity(shape, seed, lo=0.4, hi=0.95, ell=3.0):
    """Small smooth random porosity in [lo, hi] for parity cases."""
    g = gaussian_random_field(shape, ell, seed)
    g = (g - g.min()) / max(1e-300, g.max() - g.min())
    return lo + (hi - lo) * g
