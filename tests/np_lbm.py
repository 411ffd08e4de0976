"""A second, independent statement of the porous-media LBM step in NumPy.

Test infrastructure only.  It is written from the paper (Gusev & Karlin,
Sec. 3 and the flowchart of Sec. 3.5), not from the C oracle, and exists to pin
the oracle on tiny grids: the two must agree to rounding after initialisation
and after whole steps.  Whole-array operations replace the oracle's node loops;
the readings of the paper are the same ones (expanded Delta_nu with constant
nu_eff, lagged Delta_nu, final v in the drag and the corrections, halfway
bounce-back at walls, one-sided second-order stencils at wall ends).

Arrays are (nz, ny, nx); lattice axis a (x, y, z) is NumPy axis 2 - a.
"""
from __future__ import annotations

import itertools

import numpy as np


def _shift(f, ax, k):
    """g[j] = f[j + k] along lattice axis ax, periodic."""
    return np.roll(f, -k, axis=2 - ax)


def d1(f, ax, wall):
    """First derivative, Sec. 3.5: central; one-sided second order at the
    first and last node of a wall axis."""
    g = 0.5 * (_shift(f, ax, 1) - _shift(f, ax, -1))
    if wall:
        g = np.moveaxis(g, 2 - ax, 0)
        h = np.moveaxis(f, 2 - ax, 0)
        g[0] = 0.5 * (-3.0 * h[0] + 4.0 * h[1] - h[2])
        g[-1] = 0.5 * (3.0 * h[-1] - 4.0 * h[-2] + h[-3])
        g = np.moveaxis(g, 0, 2 - ax)
    return g


def d2(f, ax, wall):
    """Second derivative: three-point; four-point one-sided at wall ends."""
    g = _shift(f, ax, 1) - 2.0 * f + _shift(f, ax, -1)
    if wall:
        g = np.moveaxis(g, 2 - ax, 0)
        h = np.moveaxis(f, 2 - ax, 0)
        g[0] = 2.0 * h[0] - 5.0 * h[1] + 4.0 * h[2] - h[3]
        g[-1] = 2.0 * h[-1] - 5.0 * h[-2] + 4.0 * h[-3] - h[-4]
        g = np.moveaxis(g, 0, 2 - ax)
    return g


class NpLBM:
    def __init__(self, D, eps, kappa, *, nu_f, b=(0.0, 0.0, 0.0), forch=0.0, RT=1.0 / 3.0, J_nu=1.0, J_eta=1.0,
                 wall=(0, 0, 0), corr=7):
        self.D = D
        self.eps = np.array(eps, dtype=np.float64).reshape(np.shape(eps) if np.ndim(eps) == 3 else (1,) + np.shape(eps))
        kap = np.array(kappa, dtype=np.float64).reshape(self.eps.shape)
        self.shape = self.eps.shape
        self.RT, self.nu_f, self.J_nu, self.J_eta, self.corr = RT, nu_f, J_nu, J_eta, corr
        self.wall = [bool(wall[a]) if a < D else False for a in range(3)]
        self.b = np.array([b[a] if a < D else 0.0 for a in range(3)], dtype=np.float64)
        # lattice: i = ix + 3 iy (+ 9 iz), c = digit - 1
        self.c = np.array([[(i // 3 ** a) % 3 - 1 if a < D else 0 for a in range(3)] for i in range(3 ** D)])
        self.Q = len(self.c)
        # Eq. (eq_weights): the product form at xi = 0, P = RT
        self.w = np.array([np.prod([self.psi(ci[a], 0.0, RT) for a in range(D)]) for ci in self.c])
        # Eqs. (mu_D_Ergun_perm), (mu_F_Ergun_perm), (F_eps_Ergun); kappa = inf is free fluid
        e = self.eps
        F = 1.75 / np.sqrt(150.0 * e**3) if forch < 0 else np.full(self.shape, float(forch))
        free = np.isinf(kap)
        ks = np.where(free, 1.0, kap)
        self.muD = np.where(free, 0.0, e * nu_f / ks)
        self.muF = np.where(free, 0.0, e * F / np.sqrt(ks))
        # beta from Eq. (nu_eff_def) with delta t = 1 and nu_eff = J_nu nu_f
        self.nu_eff = J_nu * nu_f
        self.beta = 1.0 / (2.0 * self.nu_eff / RT + 1.0)
        # porosity gradient and Hessian by finite differences of the node field
        self.ge = [d1(e, a, self.wall[a]) if a < D else np.zeros(self.shape) for a in range(3)]
        H = [[np.zeros(self.shape) for _ in range(3)] for _ in range(3)]
        for a in range(D):
            H[a][a] = d2(e, a, self.wall[a])
            for bb in range(a + 1, D):
                H[a][bb] = H[bb][a] = d1(d1(e, bb, self.wall[bb]), a, self.wall[a])
        self.H = H
        self.f = None

    @staticmethod
    def psi(c, xi, P):
        """Eq. (1d_scaled_eq)."""
        return 1.0 - c * c + ((3.0 * c * c - 2.0) * P + c * xi) / 2.0

    def d1(self, f, a):
        return d1(f, a, self.wall[a])

    # ---------------------------------------------------------------- macroscopic
    def delta_nu(self, m):
        """Eq. (porosity_correction_expanded) with nu_eff constant: the divergence
        of nu (m (x) grad eps + grad eps (x) m), expanded term by term."""
        D = self.D
        trH = sum(self.H[a][a] for a in range(D))
        divm = sum(self.d1(m[a], a) for a in range(D))
        out = []
        for a in range(3):
            if a >= D:
                out.append(np.zeros(self.shape))
                continue
            r = trH * m[a] + divm * self.ge[a]
            for bb in range(D):
                r = r + self.H[a][bb] * m[bb] + self.d1(m[a], bb) * self.ge[bb]
            out.append(self.nu_eff * r)
        return out

    def acceleration(self, rho, v, dnu):
        """Eq. (accel); dnu = Delta_nu(rho u) (the lagged one of Eq. (v_final))."""
        nv = np.sqrt(sum(x * x for x in v))
        return [self.eps * self.b[a] - self.muD * v[a] - self.muF * nv * v[a] + self.RT * self.ge[a] + dnu[a] / rho
                for a in range(3)]

    def velocity(self, rho, P1):
        """Eqs. (v_(0)), (v_(1)), (velocity_coefficients), (v_final) and (accel)."""
        e = self.eps
        v0 = [P1[a] / rho + 0.5 * (e * self.b[a] + self.RT * self.ge[a]) for a in range(3)]
        n0 = np.sqrt(sum(x * x for x in v0))
        c1 = 1.0 + 0.5 * self.muD
        c2 = 0.5 * self.muF
        v1 = [2.0 * x / (c1 + np.sqrt(c1 * c1 + 4.0 * c2 * n0)) for x in v0]
        dnu = self.delta_nu([rho * x / e for x in v1]) if self.corr & 1 else [np.zeros(self.shape)] * 3
        v = [v1[a] + dnu[a] / (2.0 * rho) for a in range(3)]
        return v, self.acceleration(rho, v, dnu)

    def corrections(self, rho, v):
        """Eqs. (ex_corr), (eta_corr)."""
        D, RT, e = self.D, self.RT, self.eps
        phx = [np.zeros(self.shape) for _ in range(3)]
        if self.corr & 2:
            for a in range(D):
                phx[a] = self.d1(rho * v[a] * (1.0 - 3.0 * RT) - rho * v[a] ** 3 / e**2, a)
        phe = np.zeros(self.shape)
        if self.corr & 4:
            phe = rho * RT * (2.0 / D - self.J_eta / self.J_nu) * sum(self.d1(v[a], a) for a in range(D))
        return phx, phe

    def product(self, rho, xi, P):
        """Eq. (prod_form): eps rho prod_a Psi(c_ia; xi_a, P_aa), for every i."""
        out = np.empty((self.Q,) + self.shape)
        for i, ci in enumerate(self.c):
            g = self.eps * rho
            for a in range(self.D):
                g = g * self.psi(ci[a], xi[a], P[a])
            out[i] = g
        return out

    def equilibria(self, rho, v, a, phx, phe):
        """f_eq (Eqs. (xi_alpha_eq), (P_alpha_alpha_eq)) and f_* (Eqs.
        (xi_alpha_*), (P_aa_*), lambda = 1)."""
        e = self.eps
        xe = [v[k] / e for k in range(3)]
        Pe = [xe[k] ** 2 + self.RT for k in range(3)]
        xs = [(v[k] + a[k]) / e for k in range(3)]
        Ps = [xs[k] ** 2 + self.RT + (phx[k] + phe) / (e * rho) for k in range(3)]
        return self.product(rho, xe, Pe), self.product(rho, xs, Ps)

    def moments(self, f=None):
        f = self.f if f is None else f
        er = f.sum(axis=0)
        rho = er / self.eps
        P1 = [np.tensordot(self.c[:, a].astype(float), f, axes=(0, 0)) for a in range(3)]
        v, a = self.velocity(rho, P1)
        return rho, v, a

    # ---------------------------------------------------------------- populations
    def init(self, rho0, v0):
        """Eq. (eq_bc_f_bar) with lambda = 1 on the initial fields: a_0 by Eq.
        (accel) with Delta_nu(rho0 v0 / eps), Phi_0 from rho0, v0 (flowchart)."""
        rho0 = np.broadcast_to(np.asarray(rho0, np.float64), self.shape).copy()
        v0 = [np.broadcast_to(np.asarray(v0[k], np.float64), self.shape).copy() if k < len(v0) else np.zeros(self.shape)
              for k in range(3)]
        dnu = self.delta_nu([rho0 * x / self.eps for x in v0]) if self.corr & 1 else [np.zeros(self.shape)] * 3
        a0 = self.acceleration(rho0, v0, dnu)
        phx, phe = self.corrections(rho0, v0)
        feq, fst = self.equilibria(rho0, v0, a0, phx, phe)
        self.f = 1.5 * feq - 0.5 * fst
        self.a0 = a0
        return self

    def step(self, n=1):
        for _ in range(n):
            rho, v, a = self.moments()
            phx, phe = self.corrections(rho, v)
            feq, fst = self.equilibria(rho, v, a, phx, phe)
            f = self.f
            # Eqs. (dicrete_scheme), (momentum_rate) with lambda = delta t = 1
            fpc = f + 2.0 * self.beta * (feq - f) + (1.0 - self.beta) * (fst - feq)
            self.f = self.stream(fpc)
        return self

    def stream(self, fpc):
        """f(x + c_i) <- f_pc(x), periodic wrap; a population whose target lies
        beyond a wall face is reflected into the opposite slot of x."""
        out = np.empty_like(fpc)
        nz, ny, nx = self.shape
        n = (nx, ny, nz)
        for i, ci in enumerate(self.c):
            opp = self.Q - 1 - i
            for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
                t = [x + ci[0], y + ci[1], z + ci[2]]
                out_of = any(self.wall[a] and not (0 <= t[a] < n[a]) for a in range(3))
                if out_of:
                    out[opp, z, y, x] = fpc[i, z, y, x]
                else:
                    out[i, t[2] % nz, t[1] % ny, t[0] % nx] = fpc[i, z, y, x]
        return out
