"""Host reference of the slab decomposition along z (test infrastructure).

One rank owns the planes [z0, z1) of a D3Q27 domain that is periodic in z
(x and y: periodic or walls, whole planes per rank).  A step is the split
step with three halo exchanges between neighbouring ranks, the pattern the
device kernels follow (moments -> exchange -> velocity -> exchange -> collide
and stream -> exchange):

  1. after the moments: m = rho v1 / eps of the first and last owned plane
     (3 values per node), which Delta_nu's z-derivatives at the neighbour's
     edge plane need (Eq. (porosity_correction_expanded));
  2. after the velocity: rho and v_z of the edge planes (2 values per node),
     which the z-derivatives of Phi_ext_zz and of div v need (Eqs. (ex_corr),
     (eta_corr));
  3. after collide and stream: the 9 populations with c_z = -1 pushed out of
     the first plane and the 9 with c_z = +1 pushed out of the last plane,
     which stream into the neighbour's edge plane.

The arithmetic is that of the independent NumPy statement (np_lbm.NpLBM).
Static fields (porosity, its gradient and Hessian, mu_D, mu_F) come from
the global porosity, so a rank holds them for its planes exactly.
"""
from __future__ import annotations

import itertools

import numpy as np

from np_lbm import NpLBM


class Slab:
    """The state of one rank.  glob: an NpLBM of the global domain (its
    static fields and lattice; its populations are not used); f_init: the
    global initial populations (Q, nz, ny, nx)."""

    def __init__(self, glob: NpLBM, f_init, z0, z1):
        assert glob.D == 3 and not glob.wall[2]
        self.g, self.z0, self.z1 = glob, z0, z1
        self.n = z1 - z0
        sl = slice(z0, z1)
        self.eps = glob.eps[sl]
        self.muD, self.muF = glob.muD[sl], glob.muF[sl]
        self.ge = [x[sl] for x in glob.ge]
        self.H = [[x[sl] for x in row] for row in glob.H]
        self.f = np.array(f_init[:, sl])
        nz = glob.shape[0]
        # porosity of the planes next to the slab (static: no exchange)
        self.eps_lo = glob.eps[(z0 - 1) % nz]
        self.eps_hi = glob.eps[z1 % nz]

    # ------------------------------------------------------------ z stencils with halo planes
    @staticmethod
    def dz(f, lo, hi):
        """Central z-derivative on the owned planes, with the neighbours' planes."""
        ext = np.concatenate([lo[None], f, hi[None]], axis=0)
        return 0.5 * (ext[2:] - ext[:-2])

    def d(self, f, a, lo=None, hi=None):
        """First derivative on the owned planes; z needs the halo planes."""
        if a == 2:
            return self.dz(f, lo, hi)
        return self.g.d1(f, a)

    # ------------------------------------------------------------ phases
    def moments(self):
        g = self.g
        f = self.f
        rho = f.sum(axis=0) / self.eps
        P1 = [np.tensordot(g.c[:, a].astype(float), f, axes=(0, 0)) for a in range(3)]
        v0 = [P1[a] / rho + 0.5 * (self.eps * g.b[a] + g.RT * self.ge[a]) for a in range(3)]
        n0 = np.sqrt(sum(x * x for x in v0))
        c1 = 1.0 + 0.5 * self.muD
        c2 = 0.5 * self.muF
        self.v1 = [2.0 * x / (c1 + np.sqrt(c1 * c1 + 4.0 * c2 * n0)) for x in v0]
        self.rho = rho
        self.m = [rho * x / self.eps for x in self.v1]
        # halo 1: m of the edge planes
        return np.stack([x[0] for x in self.m]), np.stack([x[-1] for x in self.m])

    def velocity(self, m_lo, m_hi):
        """m_lo / m_hi: m (3, ny, nx) of the neighbours' planes below and above."""
        g = self.g
        rho, m = self.rho, self.m
        dnu = [np.zeros_like(rho) for _ in range(3)]
        if g.corr & 1:
            trH = self.H[0][0] + self.H[1][1] + self.H[2][2]
            dm = [[self.d(m[c], a, m_lo[c], m_hi[c]) for a in range(3)] for c in range(3)]
            divm = dm[0][0] + dm[1][1] + dm[2][2]
            for a in range(3):
                r = trH * m[a] + divm * self.ge[a]
                for b in range(3):
                    r = r + self.H[a][b] * m[b] + dm[a][b] * self.ge[b]
                dnu[a] = g.nu_eff * r
        self.v = [self.v1[a] + dnu[a] / (2.0 * rho) for a in range(3)]
        nv = np.sqrt(sum(x * x for x in self.v))
        self.a = [self.eps * g.b[a] - self.muD * self.v[a] - self.muF * nv * self.v[a] + g.RT * self.ge[a]
                  + dnu[a] / rho for a in range(3)]
        # halo 2: rho and v_z of the edge planes
        return (np.stack([rho[0], self.v[2][0]]), np.stack([rho[-1], self.v[2][-1]]))

    def collide_stream(self, rv_lo, rv_hi):
        """rv_lo / rv_hi: (rho, v_z) of the neighbours' planes; returns the
        populations pushed across the lower and the upper cut: (9, ny, nx)
        each, in the order of the populations with c_z = -1 and c_z = +1."""
        g = self.g
        rho, v, e = self.rho, self.v, self.eps
        RT = g.RT
        phx = [np.zeros_like(rho) for _ in range(3)]
        if g.corr & 2:
            for a in range(2):
                phx[a] = g.d1(rho * v[a] * (1.0 - 3.0 * RT) - rho * v[a] ** 3 / e**2, a)
            q = rho * v[2] * (1.0 - 3.0 * RT) - rho * v[2] ** 3 / e**2
            q_lo = rv_lo[0] * rv_lo[1] * (1.0 - 3.0 * RT) - rv_lo[0] * rv_lo[1] ** 3 / self.eps_lo**2
            q_hi = rv_hi[0] * rv_hi[1] * (1.0 - 3.0 * RT) - rv_hi[0] * rv_hi[1] ** 3 / self.eps_hi**2
            phx[2] = self.dz(q, q_lo, q_hi)
        phe = np.zeros_like(rho)
        if g.corr & 4:
            divv = g.d1(v[0], 0) + g.d1(v[1], 1) + self.dz(v[2], rv_lo[1], rv_hi[1])
            phe = rho * RT * (2.0 / 3.0 - g.J_eta / g.J_nu) * divv
        xe = [v[k] / e for k in range(3)]
        Pe = [xe[k] ** 2 + RT for k in range(3)]
        xs = [(v[k] + self.a[k]) / e for k in range(3)]
        Ps = [xs[k] ** 2 + RT + (phx[k] + phe) / (e * rho) for k in range(3)]
        feq = self._product(rho, xe, Pe)
        fst = self._product(rho, xs, Ps)
        f = self.f
        fpc = f + 2.0 * g.beta * (feq - f) + (1.0 - g.beta) * (fst - feq)
        # stream (np_lbm.NpLBM.stream within the slab): a population whose target
        # lies beyond an x / y wall is reflected into the opposite slot of its
        # node; one that leaves through a cut goes to the neighbouring rank
        out = np.zeros_like(fpc)
        up_ids = [i for i, ci in enumerate(g.c) if ci[2] == 1]
        down_ids = [i for i, ci in enumerate(g.c) if ci[2] == -1]
        ny, nx = e.shape[1], e.shape[2]
        # entries no population reaches (its source would lie beyond an x / y
        # wall: the slot holds a reflection instead) stay NaN and are not written
        up = np.full((9, ny, nx), np.nan)
        down = np.full((9, ny, nx), np.nan)
        for i, ci in enumerate(g.c):
            for z, y, x in itertools.product(range(self.n), range(ny), range(nx)):
                tx, ty, tz = x + ci[0], y + ci[1], z + ci[2]
                if (g.wall[0] and not 0 <= tx < nx) or (g.wall[1] and not 0 <= ty < ny):
                    out[g.Q - 1 - i, z, y, x] = fpc[i, z, y, x]
                    continue
                tx, ty = tx % nx, ty % ny
                if tz >= self.n:
                    up[up_ids.index(i), ty, tx] = fpc[i, z, y, x]
                elif tz < 0:
                    down[down_ids.index(i), ty, tx] = fpc[i, z, y, x]
                else:
                    out[i, tz, ty, tx] = fpc[i, z, y, x]
        self.f = out
        return down, up

    def receive(self, from_below, from_above):
        """The populations that crossed into this slab: from the rank below
        (c_z = +1) into the first plane, from the rank above (c_z = -1) into
        the last plane."""
        g = self.g
        up_ids = [i for i, ci in enumerate(g.c) if ci[2] == 1]
        down_ids = [i for i, ci in enumerate(g.c) if ci[2] == -1]
        for k, i in enumerate(up_ids):
            self.f[i, 0] = np.where(np.isnan(from_below[k]), self.f[i, 0], from_below[k])
        for k, i in enumerate(down_ids):
            self.f[i, -1] = np.where(np.isnan(from_above[k]), self.f[i, -1], from_above[k])

    def _product(self, rho, xi, P):
        g = self.g
        out = np.empty((g.Q,) + rho.shape)
        for i, ci in enumerate(g.c):
            t = self.eps * rho
            for a in range(3):
                t = t * g.psi(ci[a], xi[a], P[a])
            out[i] = t
        return out


def slab_bounds(nz, ranks):
    """Contiguous z ranges, as even as possible (at least 2 planes each)."""
    cuts = [round(k * nz / ranks) for k in range(ranks + 1)]
    assert all(b - a >= 2 for a, b in zip(cuts, cuts[1:]))
    return list(zip(cuts, cuts[1:]))


def step_slab(slab: Slab, swap):
    """One step of one rank.  swap(kind, to_below, to_above) sends the two
    payloads to the ranks below and above (periodic) and returns what arrives
    (from_below, from_above)."""
    m_lo_edge, m_hi_edge = slab.moments()
    m_below, m_above = swap("m", m_lo_edge, m_hi_edge)
    rv_lo_edge, rv_hi_edge = slab.velocity(m_below, m_above)
    rv_below, rv_above = swap("rv", rv_lo_edge, rv_hi_edge)
    down, up = slab.collide_stream(rv_below, rv_above)
    from_below, from_above = swap("f", down, up)
    slab.receive(from_below, from_above)


def run_local(glob: NpLBM, f_init, ranks, steps):
    """All ranks in one process, the exchange done by copying (the host
    reference of the exchange); returns the assembled populations."""
    slabs = [Slab(glob, f_init, a, b) for a, b in slab_bounds(glob.shape[0], ranks)]
    R = len(slabs)
    for _ in range(steps):
        # the phases run rank by rank; each exchange waits for all ranks
        outs = [s.moments() for s in slabs]
        ins = [(outs[(r - 1) % R][1], outs[(r + 1) % R][0]) for r in range(R)]
        outs = [s.velocity(*ins[r]) for r, s in enumerate(slabs)]
        ins = [(outs[(r - 1) % R][1], outs[(r + 1) % R][0]) for r in range(R)]
        outs = [s.collide_stream(*ins[r]) for r, s in enumerate(slabs)]
        for r, s in enumerate(slabs):
            s.receive(outs[(r - 1) % R][1], outs[(r + 1) % R][0])
    return np.concatenate([s.f for s in slabs], axis=1)
