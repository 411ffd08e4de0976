/*
 * Oracle for the porous-media lattice Boltzmann step of Gusev & Karlin,
 * "Monolithic kinetic algorithm for heterogeneous porous media systems using a
 * continuous one-domain approach".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, FP64 CPU statement of
 * the method, written to be checked against the paper by eye.  It shares no
 * code, header, table or helper with the CUDA library; only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It must
 * be compiled with -ffp-contract=off so that every operation rounds as written.
 *
 * Conventions (an interface shared with the CUDA library by documentation
 * only; each side writes its own tables):
 *   node index        n = x + nx*(y + ny*z)
 *   populations       SoA, f[i*N + n]
 *   velocity index    D2Q9:  i = ix + 3*iy,          c = (ix-1, iy-1)
 *                     D3Q27: i = ix + 3*iy + 9*iz,   c = (ix-1, iy-1, iz-1)
 *                     so the opposite direction is Q-1-i.
 *   delta t = delta x = 1, lambda = delta t (Sec. 3.3).
 *
 * Per step, each sweep finishes over all nodes before the next starts
 * (flowchart of Sec. 3.5):
 *   S1  rho, v(0), v(1), m = rho v(1)/eps                    Eqs. (v_(0)), (v_(1))
 *   S2  Delta_nu(m) (expanded form), v, a                    Eqs. (porosity_correction_expanded), (v_final), (accel)
 *   S3  Phi_ext, Phi_eta from the final rho, v               Eqs. (ex_corr), (eta_corr)
 *   S4  f_eq, f_star (product form), collision               Eqs. (1d_scaled_eq)-(P_aa_*), (dicrete_scheme)
 *   S5  streaming, periodic wrap or halfway bounce-back      Eq. (dicrete_scheme)
 * Readings where the paper leaves a choice (each is listed in the design notes):
 *   - the acceleration a reuses Delta_nu(rho v(1)/eps) computed for v (the
 *     lagged treatment of Sec. 3.3); its drag terms use the final v;
 *   - Phi_ext and Phi_eta use the final v of S2;
 *   - derivatives: second-order central differences; on a wall axis the first
 *     and last node use second-order one-sided stencils (Sec. 3.5); diagonal
 *     Hessian entries use the three-point (four-point one-sided) second
 *     difference, off-diagonal entries nest two first differences;
 *   - nu_eff is constant in space, so nu_eff'(eps) = 0;
 *   - walls are link-wise halfway bounce-back, half a spacing outside the
 *     first and last node layer;
 *   - inlet / outlet planes (S6) are wet nodes at x = 0 and x = nx-1 whose
 *     populations are rebuilt after streaming; the porosity and permeability
 *     must be uniform over the three node layers next to each plane (and the
 *     outlet layers free fluid), where Eq. (accel) is explicit (Sec. 3.4.1);
 *     the outlet either prescribes the density or copies the entering
 *     populations from its neighbour (zero-gradient outflow, Sec. 6.1);
 *   - where inlet/outlet planes meet wet-node walls (Sec. 6.1), a corner node
 *     takes the wall velocity and the density of its diagonal bulk neighbour
 *     (zeroth-order extrapolation from the neighbouring bulk node);
 *   - the bounce-back density, stated for solid boundaries, applies to
 *     wet-node walls; an inlet takes the density by mass continuity; with it
 *     a corner takes its own bounce-back density;
 *   - the regularised lid of a cavity (Sec. 6.2) tapers the wall velocity
 *     over L = nx - 1, the distance between the wet side walls.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_CORR_DELTA_NU 1
#define OR_CORR_PHI_EXT 2
#define OR_CORR_PHI_ETA 4

typedef struct {
    int lattice;      /* 0: D2Q9, 1: D3Q27 */
    int nx, ny, nz;   /* nz = 1 for D2Q9 */
    int wall[3];      /* per axis: 0 periodic, 1 halfway bounce-back walls on both faces,
                         2 (x only) velocity inlet at x = 0 and outlet at x = nx-1,
                         3 on y (x periodic, 2 or 3; z periodic): wet-node walls at y = 0 and
                           y = ny-1 moving with the velocities wall_v[0] and wall_v[1];
                         3 on x (y periodic or 3; z periodic): wet-node walls at rest at x = 0
                           and x = nx-1 (the side walls of a cavity) */
    double RT;        /* lattice temperature, default 1/3 */
    double nu_f;      /* fluid kinematic viscosity, enters mu_D */
    double J_nu;      /* nu_eff / nu_f */
    double J_eta;     /* eta_eff / nu_f */
    double forch;     /* F_eps >= 0, or < 0 for the Ergun correlation Eq. (F_eps_Ergun) */
    double b[3];      /* body acceleration */
    int corr;         /* bit mask of OR_CORR_* terms that are switched on */
    double v_in[3];   /* superficial inlet velocity (wall[0] == 2) */
    double rho_out;   /* outlet intrinsic density (wall[0] == 2) */
    int picard_iters; /* 0: one-shot velocity (Eq. (v_final)); k > 0: k Picard iterations (Appendix F) */
    double picard_omega; /* under-relaxation of the Picard iteration, (0, 1] */
    int plane_scheme; /* wet-node planes: 0 non-equilibrium extrapolation, Eq. (NEEM_bc_f_bar);
                         1 equilibrium scheme, Eq. (eq_bc_f_bar); 2 Tamm--Mott-Smith, Eq. (f_i_neq_TMS) */
    double wall_v[2][3]; /* superficial velocities of the wet-node walls at y = 0 and y = ny-1 (wall[1] == 3) */
    int plane_density;   /* density of a velocity boundary node: 0 mass continuity, Eq. (bc_density_impermWall);
                            1 bounce-back, Eq. (bc_density_BounceBack) */
    int outlet;          /* wall[0] == 2: 0 pressure outlet (rho_out); 1 zero-gradient outflow,
                            Eq. (f_bar_outflow_BC) */
    int inlet_profile;   /* wall[0] == 2: 0 uniform v_in; 1 Poiseuille profile across y with mean v_in[0],
                            Eq. (cylinder_inlet_BC) (needs walls on y) */
    int lid_profile;     /* wall[1] == 3: 0 uniform wall velocities; 1 regularised, Eq.
                            (cavity_velocity_profile): the x velocity of each wall times
                            S(min(x, L - x) / (lid_delta L)), L = nx - 1 (needs wall[0] == 3) */
    double lid_delta;    /* relative width of each taper, (0, 0.5] */
} or_params;

typedef struct {
    or_params p;
    int D, Q;
    long N;
    int dims[3];
    int c[27][3];
    double w[27];
    double beta, nu_eff, eta_eff;
    double *eps, *muD, *muF;   /* N */
    double *geps;              /* 3*N, gradient of eps */
    double *heps;              /* 9*N, Hessian of eps, row-major 3x3 */
    double *f;                 /* Q*N, post-stream state */
    double *fpc;               /* Q*N, post-collision scratch */
    double *rho, *v1, *m, *v, *a, *dnu; /* N and 3*N work fields */
    double *v0b;               /* 3*N, v(0) of Eq. (v_(0)) */
    double *phx, *phe;         /* 3*N Phi_ext diagonal, N Phi_eta */
    double *tmp;               /* 3*N scratch for derivative fields */
    long steps;
} or_state;

/* ---------------------------------------------------------------- lattice */

/* Eq. (1d_scaled_eq): Psi(c; xi, P) = 1 - c^2 + ((3c^2 - 2) P + c xi) / 2 */
static double psi(int c, double xi, double P)
{
    double c2 = (double)(c * c);
    return 1.0 - c2 + ((3.0 * c2 - 2.0) * P + c * xi) / 2.0;
}

static void setup_lattice(or_state* s)
{
    s->D = s->p.lattice == 0 ? 2 : 3;
    s->Q = s->p.lattice == 0 ? 9 : 27;
    for (int i = 0; i < s->Q; ++i) {
        s->c[i][0] = i % 3 - 1;
        s->c[i][1] = (i / 3) % 3 - 1;
        s->c[i][2] = s->D == 3 ? i / 9 - 1 : 0;
        /* Eq. (eq_weights): w_i = prod_alpha Psi(c_i alpha; 0, RT) */
        double w = 1.0;
        for (int al = 0; al < s->D; ++al) w *= psi(s->c[i][al], 0.0, s->p.RT);
        s->w[i] = w;
    }
}

/* Eq. (prod_form): f_i = eps rho prod_alpha Psi(c_i alpha; xi_alpha, P_alpha alpha) */
static void product_form(const or_state* s, double eps_rho, const double* xi, const double* P, double* out)
{
    for (int i = 0; i < s->Q; ++i) {
        double prod = 1.0;
        for (int al = 0; al < s->D; ++al) prod *= psi(s->c[i][al], xi[al], P[al]);
        out[i] = eps_rho * prod;
    }
}

/* ------------------------------------------------------------ grid helpers */

static long node(const or_state* s, int x, int y, int z) { return x + (long)s->p.nx * (y + (long)s->p.ny * z); }

static void coords(const or_state* s, long n, int* x)
{
    x[0] = (int)(n % s->p.nx);
    x[1] = (int)((n / s->p.nx) % s->p.ny);
    x[2] = (int)(n / ((long)s->p.nx * s->p.ny));
}

/* value of field g at the node displaced by d along axis ax (periodic wrap) */
static double at(const or_state* s, const double* g, const int* x, int ax, int d)
{
    int y[3] = {x[0], x[1], x[2]};
    int n = s->dims[ax];
    y[ax] = ((y[ax] + d) % n + n) % n;
    return g[node(s, y[0], y[1], y[2])];
}

/* first derivative of g along ax at x: second-order central differences, and
   second-order one-sided differences at the first and last node of a wall axis */
static double d1(const or_state* s, const double* g, const int* x, int ax)
{
    int n = s->dims[ax], k = x[ax];
    if (s->p.wall[ax]) {
        if (k == 0) return (-3.0 * at(s, g, x, ax, 0) + 4.0 * at(s, g, x, ax, 1) - at(s, g, x, ax, 2)) / 2.0;
        if (k == n - 1) return (3.0 * at(s, g, x, ax, 0) - 4.0 * at(s, g, x, ax, -1) + at(s, g, x, ax, -2)) / 2.0;
    }
    return (at(s, g, x, ax, 1) - at(s, g, x, ax, -1)) / 2.0;
}

/* second derivative of g along ax at x, same boundary rule */
static double d2(const or_state* s, const double* g, const int* x, int ax)
{
    int n = s->dims[ax], k = x[ax];
    if (s->p.wall[ax]) {
        if (k == 0)
            return 2.0 * at(s, g, x, ax, 0) - 5.0 * at(s, g, x, ax, 1) + 4.0 * at(s, g, x, ax, 2) - at(s, g, x, ax, 3);
        if (k == n - 1)
            return 2.0 * at(s, g, x, ax, 0) - 5.0 * at(s, g, x, ax, -1) + 4.0 * at(s, g, x, ax, -2) - at(s, g, x, ax, -3);
    }
    return at(s, g, x, ax, 1) - 2.0 * at(s, g, x, ax, 0) + at(s, g, x, ax, -1);
}

/* ---------------------------------------------------------- static fields */

/* Eqs. (mu_D_Ergun_perm), (mu_F_Ergun_perm), (F_eps_Ergun); kappa = +inf is free fluid */
static void static_fields(or_state* s, const double* kappa)
{
    long N = s->N;
    for (long n = 0; n < N; ++n) {
        double e = s->eps[n], k = kappa[n];
        if (isinf(k)) {
            s->muD[n] = 0.0;
            s->muF[n] = 0.0;
        } else {
            double F = s->p.forch >= 0.0 ? s->p.forch : 1.75 / sqrt(150.0 * e * e * e);
            s->muD[n] = e * s->p.nu_f / k;
            s->muF[n] = e * F / sqrt(k);
        }
    }
    /* gradient and Hessian of eps by finite differences (Sec. 3.5) */
    for (long n = 0; n < N; ++n) {
        int x[3];
        coords(s, n, x);
        for (int al = 0; al < 3; ++al) s->geps[3 * n + al] = al < s->D ? d1(s, s->eps, x, al) : 0.0;
    }
    for (int be = 0; be < 3; ++be) {
        for (long n = 0; n < N; ++n) s->tmp[n] = s->geps[3 * n + be];
        for (long n = 0; n < N; ++n) {
            int x[3];
            coords(s, n, x);
            for (int al = 0; al < 3; ++al) {
                double h = 0.0;
                if (al < s->D && be < s->D) h = (al == be) ? d2(s, s->eps, x, al) : d1(s, s->tmp, x, al);
                s->heps[9 * n + 3 * al + be] = h;
            }
        }
    }
}

/* ------------------------------------------------------------ the sweeps */

/* S1: Eqs. (transformed_density_moment), (transformed_momentum_moment), (v_(0)),
   (v_(1)), (velocity_coefficients); m = rho v(1) / eps is the argument of Delta_nu
   in Eq. (v_final). */
static void sweep_moments(or_state* s, const double* f)
{
    long N = s->N;
    int D = s->D, Q = s->Q;
    double RT = s->p.RT;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        double e = s->eps[n];
        double sum = 0.0, P1[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q; ++i) {
            double fi = f[(long)i * N + n];
            sum += fi;
            for (int al = 0; al < D; ++al) P1[al] += s->c[i][al] * fi;
        }
        double rho = sum / e;
        double v0[3] = {0.0, 0.0, 0.0}, nv0 = 0.0;
        for (int al = 0; al < D; ++al) {
            v0[al] = P1[al] / rho + 0.5 * (e * s->p.b[al] + RT * s->geps[3 * n + al]);
            nv0 += v0[al] * v0[al];
        }
        nv0 = sqrt(nv0);
        double c1 = 1.0 + 0.5 * s->muD[n];
        double c2 = 0.5 * s->muF[n];
        double den = c1 + sqrt(c1 * c1 + 4.0 * c2 * nv0);
        s->rho[n] = rho;
        for (int al = 0; al < 3; ++al) s->v0b[3 * n + al] = v0[al];
        for (int al = 0; al < 3; ++al) {
            double v1 = al < D ? 2.0 * v0[al] / den : 0.0;
            s->v1[3 * n + al] = v1;
            s->m[3 * n + al] = rho * v1 / e;
        }
    }
}

/* Eq. (porosity_correction_expanded) with constant nu_eff:
   Delta_nu(m)_a = nu_eff [ sum_b H_ab m_b + tr(H) m_a + (div m) d_a eps + sum_b (d_b m_a)(d_b eps) ] */
static void delta_nu(or_state* s, const double* m, double* out)
{
    long N = s->N;
    int D = s->D;
    /* component fields of m for the finite differences */
    double* mc[3] = {s->tmp, s->tmp + N, s->tmp + 2 * N};
    for (long n = 0; n < N; ++n)
        for (int al = 0; al < 3; ++al) mc[al][n] = m[3 * n + al];
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        int x[3];
        coords(s, n, x);
        double dm[3][3] = {{0}};
        for (int al = 0; al < D; ++al)
            for (int be = 0; be < D; ++be) dm[al][be] = d1(s, mc[al], x, be);
        const double* H = s->heps + 9 * n;
        const double* ge = s->geps + 3 * n;
        double trH = 0.0, divm = 0.0;
        for (int al = 0; al < D; ++al) {
            trH += H[3 * al + al];
            divm += dm[al][al];
        }
        for (int al = 0; al < 3; ++al) {
            double r = 0.0;
            if (al < D) {
                for (int be = 0; be < D; ++be) r += H[3 * al + be] * m[3 * n + be];
                r += trH * m[3 * n + al];
                r += divm * ge[al];
                for (int be = 0; be < D; ++be) r += dm[al][be] * ge[be];
                r *= s->nu_eff;
            }
            out[3 * n + al] = r;
        }
    }
}

/* Eq. (accel): a = eps b - mu_D v - mu_F |v| v + RT grad eps + Delta_nu / rho,
   from the fields s->v and s->dnu */
static void acceleration(or_state* s)
{
    long N = s->N;
    int D = s->D;
    for (long n = 0; n < N; ++n) {
        double rho = s->rho[n], e = s->eps[n];
        double nv = 0.0;
        for (int al = 0; al < 3; ++al) nv += s->v[3 * n + al] * s->v[3 * n + al];
        nv = sqrt(nv);
        for (int al = 0; al < 3; ++al) {
            double va = s->v[3 * n + al];
            s->a[3 * n + al] = al < D ? e * s->p.b[al] - s->muD[n] * va - s->muF[n] * nv * va
                                            + s->p.RT * s->geps[3 * n + al] + s->dnu[3 * n + al] / rho
                                      : 0.0;
        }
    }
}

/* Appendix F: Picard (fixed-point) iteration of the implicit velocity equation
     c1 v + c2 |v| v = v(0) + Delta_nu(rho v / eps) / (2 rho),
   started from the one-shot v of Eq. (v_final):
     s = v(0) + Delta_nu(rho v(k) / eps) / (2 rho),
     v(k+1) = 2 s / (c1 + sqrt(c1^2 + 4 c2 |s|)),
     v(k+1) <- (1 - omega) v(k) + omega v(k+1).
   dnu keeps the correction of the last iteration, which the acceleration of
   Eq. (accel) then uses, so that (with omega = 1) Pi_1 = rho v - rho a / 2 holds. */
static void picard(or_state* s)
{
    long N = s->N;
    int D = s->D;
    double w = s->p.picard_omega;
    for (int k = 0; k < s->p.picard_iters; ++k) {
        for (long n = 0; n < N; ++n)
            for (int al = 0; al < 3; ++al) s->m[3 * n + al] = s->rho[n] * s->v[3 * n + al] / s->eps[n];
        delta_nu(s, s->m, s->dnu);
        for (long n = 0; n < N; ++n) {
            double sv[3] = {0, 0, 0}, ns = 0.0;
            for (int al = 0; al < D; ++al) {
                sv[al] = s->v0b[3 * n + al] + s->dnu[3 * n + al] / (2.0 * s->rho[n]);
                ns += sv[al] * sv[al];
            }
            ns = sqrt(ns);
            double c1 = 1.0 + 0.5 * s->muD[n], c2 = 0.5 * s->muF[n];
            double den = c1 + sqrt(c1 * c1 + 4.0 * c2 * ns);
            for (int al = 0; al < D; ++al)
                s->v[3 * n + al] = (1.0 - w) * s->v[3 * n + al] + w * (2.0 * sv[al] / den);
        }
    }
}

/* S2: Eq. (v_final) v = v(1) + Delta_nu(m) / (2 rho), optionally refined by
   the Picard iteration of Appendix F, then the acceleration */
static void sweep_velocity(or_state* s)
{
    long N = s->N;
    if (s->p.corr & OR_CORR_DELTA_NU)
        delta_nu(s, s->m, s->dnu);
    else
        memset(s->dnu, 0, sizeof(double) * 3 * N);
    for (long n = 0; n < N; ++n)
        for (int al = 0; al < 3; ++al) s->v[3 * n + al] = s->v1[3 * n + al] + s->dnu[3 * n + al] / (2.0 * s->rho[n]);
    if (s->p.picard_iters > 0 && (s->p.corr & OR_CORR_DELTA_NU)) picard(s);
    acceleration(s);
}

/* S3: Eq. (ex_corr) Phi_ext_aa = d_a [ rho v_a (1 - 3RT) - rho v_a^3 / eps^2 ],
   Eq. (eta_corr) Phi_eta = rho RT (2/D - eta_eff/nu_eff) div v */
static void sweep_corrections(or_state* s)
{
    long N = s->N;
    int D = s->D;
    double RT = s->p.RT;
    double* q = s->tmp;          /* N */
    double* vc = s->tmp + N;     /* N */
    for (long n = 0; n < N; ++n) s->phe[n] = 0.0;
    for (int al = 0; al < 3; ++al) {
        for (long n = 0; n < N; ++n) {
            double va = s->v[3 * n + al], r = s->rho[n], e = s->eps[n];
            q[n] = r * va * (1.0 - 3.0 * RT) - r * va * va * va / (e * e);
            vc[n] = va;
        }
        for (long n = 0; n < N; ++n) {
            int x[3];
            coords(s, n, x);
            double ph = 0.0, dv = 0.0;
            if (al < D) {
                ph = d1(s, q, x, al);
                dv = d1(s, vc, x, al);
            }
            s->phx[3 * n + al] = (s->p.corr & OR_CORR_PHI_EXT) ? ph : 0.0;
            s->phe[n] += dv; /* accumulates div v */
        }
    }
    for (long n = 0; n < N; ++n) {
        double coef = 2.0 / D - s->eta_eff / s->nu_eff;
        s->phe[n] = (s->p.corr & OR_CORR_PHI_ETA) ? s->rho[n] * RT * coef * s->phe[n] : 0.0;
    }
}

/* equilibrium and shifted equilibrium at node n from the S1-S3 fields,
   Eqs. (xi_alpha_eq), (P_alpha_alpha_eq), (xi_alpha_*), (P_aa_*) with lambda = 1 */
static void equilibria(const or_state* s, long n, double* feq, double* fst)
{
    double e = s->eps[n], rho = s->rho[n], RT = s->p.RT;
    double xe[3], Pe[3], xs[3], Ps[3];
    for (int al = 0; al < s->D; ++al) {
        xe[al] = s->v[3 * n + al] / e;
        Pe[al] = xe[al] * xe[al] + RT;
        xs[al] = s->v[3 * n + al] / e + s->a[3 * n + al] / e;
        Ps[al] = xs[al] * xs[al] + RT + (s->phx[3 * n + al] + s->phe[n]) / (e * rho);
    }
    product_form(s, e * rho, xe, Pe, feq);
    product_form(s, e * rho, xs, Ps, fst);
}

/* S4: Eqs. (dicrete_scheme), (momentum_rate) with lambda = delta t = 1:
   f_pc = f + 2 beta (f_eq - f) + (1 - beta)(f_star - f_eq) */
static void sweep_collide(or_state* s)
{
    long N = s->N;
    int Q = s->Q;
    double beta = s->beta;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        double feq[27], fst[27];
        equilibria(s, n, feq, fst);
        for (int i = 0; i < Q; ++i) {
            double fi = s->f[(long)i * N + n];
            s->fpc[(long)i * N + n] = fi + 2.0 * beta * (feq[i] - fi) + (1.0 - beta) * (fst[i] - feq[i]);
        }
    }
}

/* S5: f_i(x + c_i) <- f_pc_i(x).  Written as a pull: the population arriving at
   x along c_i comes from x - c_i; if x - c_i lies beyond a wall, the population
   is the one that left x towards the wall, reflected: f_i(x) <- f_pc_opp(i)(x).
   A population arriving through an inlet or outlet plane or a wet-node wall
   is unknown; it is given the same reflected value (the bounce-back of Eq.
   (bc_density_BounceBack), which the bounce-back density reads) and rebuilt
   by S6. */
static void sweep_stream(or_state* s)
{
    long N = s->N;
    int Q = s->Q;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        int x[3];
        coords(s, n, x);
        for (int i = 0; i < Q; ++i) {
            int src[3], out = 0, open = 0;
            for (int al = 0; al < 3; ++al) {
                int k = x[al] - s->c[i][al], d = s->dims[al];
                if (k < 0 || k >= d) {
                    if (s->p.wall[al] == 1) out = 1;
                    if (s->p.wall[al] == 2 || s->p.wall[al] == 3) open = 1;
                    k = (k % d + d) % d;
                }
                src[al] = k;
            }
            if (out || open)
                s->f[(long)i * N + n] = s->fpc[(long)(Q - 1 - i) * N + n];
            else
                s->f[(long)i * N + n] = s->fpc[(long)i * N + node(s, src[0], src[1], src[2])];
        }
    }
}

/* f_eq(eps, rho, v) of Eqs. (prod_form), (xi_alpha_eq), (P_alpha_alpha_eq) */
static void feq_of(const or_state* s, double e, double rho, const double* v, double* out)
{
    double xi[3], P[3];
    for (int al = 0; al < s->D; ++al) {
        xi[al] = v[al] / e;
        P[al] = xi[al] * xi[al] + s->p.RT;
    }
    product_form(s, e * rho, xi, P, out);
}

/* Eq. (accel) where the porosity is locally uniform (grad eps = 0, Delta_nu = 0) */
static void accel_uniform(const or_state* s, long n, const double* v, double* a)
{
    double nv = 0.0;
    for (int al = 0; al < s->D; ++al) nv += v[al] * v[al];
    nv = sqrt(nv);
    for (int al = 0; al < 3; ++al)
        a[al] = al < s->D ? s->eps[n] * s->p.b[al] - s->muD[n] * v[al] - s->muF[n] * nv * v[al] : 0.0;
}

/* S6: inlet (x = 0, prescribed v_b) and outlet (x = nx-1, prescribed rho_b)
   wet-node planes, and the wet-node walls at y = 0 and y = ny-1 moving with
   prescribed velocities (the Couette walls of Sec. 5.1), rebuilt after
   streaming (flowchart of Sec. 3.5):
   - the boundary density by mass continuity, Eqs. (boundary_density_split),
     (bc_rho_components_def), (bc_density_impermWall); at the outlet the same
     relation is solved for the normal velocity, the tangential velocity is
     taken from the interior neighbour;
   - every population by one of the reconstructions of Sec. 3.4, with
     lambda = dt = 1 and the targets (rho_b, v_b), f_tgt = f_eq(eps_b, rho_b, v_b),
     f_* = f_eq(eps_b, rho_b, v_b + a_b):
     plane_scheme 0, non-equilibrium extrapolation from the interior
       neighbour x_f along the normal, Eqs. (NEEM_bc_f_bar), (zeta_beta_NEEM)
       with zeta = 1 (beta is uniform);
     plane_scheme 1, the equilibrium scheme, Eq. (eq_bc_f_bar):
       f_bar = 1.5 f_tgt - 0.5 f_*;
     plane_scheme 2, Tamm--Mott-Smith, Eq. (f_i_neq_TMS) in the three steps
       of Sec. 3.4: (rho_loc, v_loc) from the known post-advection
       populations (those not in P-, the set of populations entering from
       outside, c_i . n_out < 0), f_loc = f_eq(eps_b, rho_loc, v_loc), then
       f_bar = (f_tgt - f_loc) / (1 - beta) + 1.5 f_tgt - 0.5 f_*   (i in P-),
       f_bar = (f_tgt - f_loc) / (1 - beta) + f_bar_pa              (otherwise). */
/* Density of a velocity boundary node b (wall normal ax, outward nout,
   prescribed velocity vb) from its post-stream populations: mass continuity,
   Eq. (bc_density_impermWall) with rho^0, rho^+ of Eqs. (boundary_density_split),
   (bc_rho_components_def); at a wet-node wall (not an inlet) optionally the
   bounce-back density, Eq. (bc_density_BounceBack), which the paper states for
   solid boundaries (an inlet always takes continuity). */
static double velocity_node_density(const or_state* s, long b, int ax, double nout, const double* vb)
{
    int Q = s->Q;
    long N = s->N;
    double eb = s->eps[b];
    if (s->p.plane_density == 1 && (ax == 1 || s->p.wall[0] == 3)) {
        /* the unknown slots hold the reflected post-collision outgoing populations after S5 */
        double sum = 0.0;
        for (int i = 0; i < Q; ++i) sum += s->f[(long)i * N + b];
        return sum / eb;
    }
    double r0 = 0.0, rp = 0.0, ab[3];
    for (int i = 0; i < Q; ++i) {
        double cn = s->c[i][ax] * nout;
        double fi = s->f[(long)i * N + b];
        if (cn == 0.0) r0 += fi / eb;
        if (cn > 0.0) rp += fi / eb;
    }
    accel_uniform(s, b, vb, ab);
    return eb * (r0 + 2.0 * rp) / (eb + vb[ax] * nout - 0.5 * ab[ax] * nout);
}

/* One wet node x_b of a plane normal to axis ax (outward normal nout = -1 at
   the low face, +1 at the high face) with interior neighbour x_f = x_b - nout
   along the axis.  kind 0: prescribed velocity vt (inlet, moving wall), density
   by velocity_node_density; kind 1: prescribed density rho_t (outlet; normal
   velocity by continuity, tangential velocity from x_f); kind 2: prescribed
   velocity vt and density rho_t (a corner of an inlet/outlet plane and a wall). */
static void rebuild_node(or_state* s, long b, long f, int ax, double nout, int kind, const double* vt, double rho_t)
{
    int Q = s->Q, D = s->D;
    long N = s->N;
    double eb = s->eps[b], ef = s->eps[f];
    /* interior neighbour: moments and velocity (S1 with Delta_nu = 0) */
    double sum = 0.0, P1[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
        double fi = s->f[(long)i * N + f];
        sum += fi;
        for (int al = 0; al < D; ++al) P1[al] += s->c[i][al] * fi;
    }
    double rf = sum / ef, v0[3] = {0, 0, 0}, nv0 = 0.0;
    for (int al = 0; al < D; ++al) {
        v0[al] = P1[al] / rf + 0.5 * ef * s->p.b[al];
        nv0 += v0[al] * v0[al];
    }
    nv0 = sqrt(nv0);
    double c1 = 1.0 + 0.5 * s->muD[f], c2 = 0.5 * s->muF[f];
    double vf[3] = {0, 0, 0}, af[3];
    for (int al = 0; al < D; ++al) vf[al] = 2.0 * v0[al] / (c1 + sqrt(c1 * c1 + 4.0 * c2 * nv0));
    accel_uniform(s, f, vf, af);
    /* boundary node: rho^0 and rho^+ from the known populations */
    double r0 = 0.0, rp = 0.0;
    for (int i = 0; i < Q; ++i) {
        double cn = s->c[i][ax] * nout;
        double fi = s->f[(long)i * N + b];
        if (cn == 0.0) r0 += fi / eb;
        if (cn > 0.0) rp += fi / eb;
    }
    double vb[3] = {0, 0, 0}, ab[3], rb;
    if (kind == 0 || kind == 2) {
        for (int al = 0; al < D; ++al) vb[al] = vt[al];
        accel_uniform(s, b, vb, ab);
        rb = kind == 2 ? rho_t : velocity_node_density(s, b, ax, nout, vb);
    } else {
        rb = rho_t;
        double aperp = eb * s->p.b[ax] * nout; /* free-fluid outlet: no drag */
        double vperp = eb * (r0 + 2.0 * rp) / rb - eb + 0.5 * aperp;
        for (int al = 0; al < D; ++al) vb[al] = vf[al];
        vb[ax] = vperp * nout;
        accel_uniform(s, b, vb, ab);
    }
    double feb[27], fef[27], fsb[27], fsf[27], vsb[3], vsf[3];
    for (int al = 0; al < 3; ++al) {
        vsb[al] = vb[al] + ab[al];
        vsf[al] = vf[al] + af[al];
    }
    feq_of(s, eb, rb, vb, feb);
    feq_of(s, ef, rf, vf, fef);
    feq_of(s, eb, rb, vsb, fsb);
    feq_of(s, ef, rf, vsf, fsf);
    if (s->p.plane_scheme == 1) {
        for (int i = 0; i < Q; ++i) s->f[(long)i * N + b] = 1.5 * feb[i] - 0.5 * fsb[i];
    } else if (s->p.plane_scheme == 2) {
        /* step 1: local density and momentum from the known populations */
        double omb = 1.0 - s->beta, dr = 0.0, dj[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q; ++i) {
            if (s->c[i][ax] * nout < 0.0) continue; /* i in P- */
            double d = s->f[(long)i * N + b] - 1.5 * feb[i] + 0.5 * fsb[i];
            dr += d;
            for (int al = 0; al < D; ++al) dj[al] += s->c[i][al] * d;
        }
        double rloc = (eb * rb + omb * dr) / eb, vloc[3] = {0.0, 0.0, 0.0}, floc[27];
        for (int al = 0; al < D; ++al) vloc[al] = (rb * vb[al] + omb * dj[al]) / rloc;
        /* step 2: local equilibrium */
        feq_of(s, eb, rloc, vloc, floc);
        /* step 3: every boundary population */
        for (int i = 0; i < Q; ++i) {
            double corr = (feb[i] - floc[i]) / omb;
            if (s->c[i][ax] * nout < 0.0)
                s->f[(long)i * N + b] = corr + 1.5 * feb[i] - 0.5 * fsb[i];
            else
                s->f[(long)i * N + b] = corr + s->f[(long)i * N + b];
        }
    } else {
        double zeta = 1.0;
        for (int i = 0; i < Q; ++i)
            s->f[(long)i * N + b] = zeta * s->f[(long)i * N + f] + 1.5 * (feb[i] - zeta * fef[i])
                                    + 0.5 * (zeta * fsf[i] - fsb[i]);
    }
}

/* Eq. (f_bar_outflow_BC): zero-gradient outflow at x_b = (nx-1, y, z); the
   populations entering from outside (c_x < 0) are copied from x_f = x_b - 1. */
static void outflow_node(or_state* s, long b, long f)
{
    for (int i = 0; i < s->Q; ++i)
        if (s->c[i][0] < 0) s->f[(long)i * s->N + b] = s->f[(long)i * s->N + f];
}

/* Inlet velocity at row y, Eq. (cylinder_inlet_BC) for the Poiseuille profile:
   v_x = 6 V0 eta (1 - eta) with the walls at eta = 0, 1 (wet-node walls on the
   rows y = 0 and ny-1; halfway bounce-back walls half a spacing outside them). */
static void inlet_velocity(const or_state* s, int y, double* vt)
{
    for (int al = 0; al < 3; ++al) vt[al] = s->p.v_in[al];
    if (s->p.inlet_profile == 1) {
        int ny = s->p.ny;
        double eta = s->p.wall[1] == 3 ? (double)y / (ny - 1) : (y + 0.5) / ny;
        vt[0] = 6.0 * s->p.v_in[0] * eta * (1.0 - eta);
        vt[1] = vt[2] = 0.0;
    }
}

/* Intrinsic density of an interior node from its post-stream populations (S1) */
static double node_density(const or_state* s, long n)
{
    double sum = 0.0;
    for (int i = 0; i < s->Q; ++i) sum += s->f[(long)i * s->N + n];
    return sum / s->eps[n];
}

/* Eq. (s_cinf): the smoothstep S(psi), 0 for psi <= 0, 1 for psi >= 1 */
static double smoothstep(double psi)
{
    if (psi <= 0.0) return 0.0;
    if (psi >= 1.0) return 1.0;
    double a = exp(-1.0 / psi), b = exp(-1.0 / (1.0 - psi));
    return a / (a + b);
}

/* Velocity of the wet-node wall on row y = 0 (side 0) or ny-1 (side 1) at
   column x: wall_v[side], its x component tapered by Eq.
   (cavity_velocity_profile) when lid_profile is set. */
static void wall_velocity(const or_state* s, int side, int x, double* vt)
{
    for (int al = 0; al < 3; ++al) vt[al] = s->p.wall_v[side][al];
    if (s->p.lid_profile == 1) {
        double L = s->p.nx - 1.0, d = x < L - x ? x : L - x;
        vt[0] *= smoothstep(d / (s->p.lid_delta * L));
    }
}

/* S6 in the order: (A) the x sides -- inlet and outlet planes, or wet-node
   walls at rest --, (B) the corner columns where they meet wet-node walls on
   y, (C) the wall rows.  A corner takes the velocity of the y wall there and,
   for its density, the bounce-back density of the corner node itself when the
   walls take it (the bounce-back operation, the paper's second remedy where
   boundaries meet), else the density of its diagonal bulk neighbour (the
   paper extrapolates the corner density from neighbouring bulk fluid nodes;
   this is the zeroth-order extrapolation); its populations come from the
   wall rule with x_f on the x side, rebuilt in (A). */
static void sweep_planes(or_state* s)
{
    int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
    int xw = s->p.wall[0] == 2, xs = s->p.wall[0] == 3, yw = s->p.wall[1] == 3;
    if (xw || xs)
        for (int side = 0; side < 2; ++side) {
            int xb = side == 0 ? 0 : nx - 1, xf = side == 0 ? 1 : nx - 2;
            for (int z = 0; z < nz; ++z)
                for (int y = yw ? 1 : 0; y < (yw ? ny - 1 : ny); ++y) {
                    long b = node(s, xb, y, z), f = node(s, xf, y, z);
                    if (xs) {
                        const double rest[3] = {0.0, 0.0, 0.0};
                        rebuild_node(s, b, f, 0, side == 0 ? -1.0 : 1.0, 0, rest, 0.0);
                    } else if (side == 0) {
                        double vt[3];
                        inlet_velocity(s, y, vt);
                        rebuild_node(s, b, f, 0, -1.0, 0, vt, 0.0);
                    } else if (s->p.outlet == 1) {
                        outflow_node(s, b, f);
                    } else {
                        rebuild_node(s, b, f, 0, 1.0, 1, NULL, s->p.rho_out);
                    }
                }
        }
    if ((xw || xs) && yw)
        for (int sy = 0; sy < 2; ++sy)
            for (int sx = 0; sx < 2; ++sx) {
                int yb = sy == 0 ? 0 : ny - 1, yf = sy == 0 ? 1 : ny - 2;
                int xb = sx == 0 ? 0 : nx - 1, xa = sx == 0 ? 1 : nx - 2;
                double nout = sy == 0 ? -1.0 : 1.0, vt[3];
                wall_velocity(s, sy, xb, vt);
                for (int z = 0; z < nz; ++z) {
                    long b = node(s, xb, yb, z);
                    double rho = s->p.plane_density == 1 ? node_density(s, b) : node_density(s, node(s, xa, yf, z));
                    rebuild_node(s, b, node(s, xb, yf, z), 1, nout, 2, vt, rho);
                }
            }
    if (yw)
        for (int side = 0; side < 2; ++side) {
            int yb = side == 0 ? 0 : ny - 1, yf = side == 0 ? 1 : ny - 2;
            for (int z = 0; z < nz; ++z)
                for (int x = (xw || xs) ? 1 : 0; x < ((xw || xs) ? nx - 1 : nx); ++x) {
                    double vt[3];
                    wall_velocity(s, side, x, vt);
                    rebuild_node(s, node(s, x, yb, z), node(s, x, yf, z), 1, side == 0 ? -1.0 : 1.0, 0, vt, 0.0);
                }
        }
}

/* ------------------------------------------------------------- public API */

/* Threads the node loops run on (1 without OpenMP), and a way to set them; the
   loops are independent per node, so the result does not depend on it. */
int or_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

void or_free(or_state* s)
{
    if (!s) return;
    double* ptrs[] = {s->eps, s->muD, s->muF, s->geps, s->heps, s->f, s->fpc, s->rho, s->v1,
                      s->m, s->v, s->a, s->dnu, s->phx, s->phe, s->tmp, s->v0b};
    for (unsigned k = 0; k < sizeof(ptrs) / sizeof(ptrs[0]); ++k) free(ptrs[k]);
    free(s);
}

/* Creates the oracle state; eps and kappa are N-node fields (copied).  Returns
   NULL on invalid input. */
or_state* or_create(const or_params* p, const double* eps, const double* kappa)
{
    if (p->lattice != 0 && p->lattice != 1) return NULL;
    if (p->lattice == 0 && p->nz != 1) return NULL;
    if (p->picard_iters < 0 || (p->picard_iters > 0 && !(p->picard_omega > 0.0 && p->picard_omega <= 1.0))) return NULL;
    if (p->plane_scheme < 0 || p->plane_scheme > 2) return NULL;
    if (p->plane_density < 0 || p->plane_density > 1) return NULL;
    or_state* s = (or_state*)calloc(1, sizeof(or_state));
    s->p = *p;
    setup_lattice(s);
    s->dims[0] = p->nx;
    s->dims[1] = p->ny;
    s->dims[2] = p->nz;
    if (s->D == 2) s->p.wall[2] = 0;
    for (int al = 0; al < s->D; ++al)
        if (s->dims[al] < (s->p.wall[al] ? 4 : 3)) {
            free(s);
            return NULL;
        }
    for (int al = 1; al < 3; ++al)
        if (s->p.wall[al] == 2) {
            free(s);
            return NULL;
        }
    /* wet-node walls: moving ones on y, with x periodic, inlet/outlet planes
       (corners, Sec. 6.1) or wet-node walls at rest (a cavity, Sec. 6.2); wet
       walls at rest on x with y periodic or wet walls; z periodic (no edges) */
    if (s->p.wall[2] == 3 || (s->p.wall[0] == 3 && s->p.wall[1] != 0 && s->p.wall[1] != 3) ||
        ((s->p.wall[0] == 3 || s->p.wall[1] == 3) && s->p.wall[2] != 0) ||
        (s->p.wall[1] == 3 && (s->p.wall[0] == 1 || s->p.wall_v[0][1] != 0.0 || s->p.wall_v[1][1] != 0.0))) {
        free(s);
        return NULL;
    }
    /* the regularised lid tapers into wet side walls */
    if (p->lid_profile < 0 || p->lid_profile > 1 ||
        (p->lid_profile == 1 && (s->p.wall[0] != 3 || s->p.wall[1] != 3 || !(p->lid_delta > 0.0 && p->lid_delta <= 0.5)))) {
        free(s);
        return NULL;
    }
    /* the outlet kind and the inlet profile belong to inlet/outlet planes; the
       Poiseuille profile spans walls on y */
    if (p->outlet < 0 || p->outlet > 1 || p->inlet_profile < 0 || p->inlet_profile > 1 ||
        ((p->outlet != 0 || p->inlet_profile != 0) && s->p.wall[0] != 2) ||
        (p->inlet_profile == 1 && s->p.wall[1] != 1 && s->p.wall[1] != 3)) {
        free(s);
        return NULL;
    }
    long N = (long)p->nx * p->ny * p->nz;
    s->N = N;
    s->nu_eff = p->J_nu * p->nu_f;
    s->eta_eff = p->J_eta * p->nu_f;
    /* Eq. (nu_eff_def) solved for beta: beta = 1 / (2 nu_eff / RT + 1) */
    s->beta = 1.0 / (2.0 * s->nu_eff / p->RT + 1.0);
    s->eps = malloc(sizeof(double) * N);
    s->muD = malloc(sizeof(double) * N);
    s->muF = malloc(sizeof(double) * N);
    s->geps = calloc(3 * N, sizeof(double));
    s->heps = calloc(9 * N, sizeof(double));
    s->f = calloc((size_t)s->Q * N, sizeof(double));
    s->fpc = calloc((size_t)s->Q * N, sizeof(double));
    s->rho = calloc(N, sizeof(double));
    s->v1 = calloc(3 * N, sizeof(double));
    s->v0b = calloc(3 * N, sizeof(double));
    s->m = calloc(3 * N, sizeof(double));
    s->v = calloc(3 * N, sizeof(double));
    s->a = calloc(3 * N, sizeof(double));
    s->dnu = calloc(3 * N, sizeof(double));
    s->phx = calloc(3 * N, sizeof(double));
    s->phe = calloc(N, sizeof(double));
    s->tmp = calloc(3 * N, sizeof(double));
    memcpy(s->eps, eps, sizeof(double) * N);
    static_fields(s, kappa);
    if (s->p.wall[0] == 2) {
        /* inlet/outlet planes need uniform porosity and permeability over their
           three node layers, and free fluid at the outlet */
        int ok = p->nx >= 6;
        for (long n = 0; n < N && ok; ++n) {
            int x[3];
            coords(s, n, x);
            int side = x[0] <= 2 ? 0 : (x[0] >= p->nx - 3 ? 1 : -1);
            if (side < 0) continue;
            long r = node(s, side == 0 ? 0 : p->nx - 1, 0, 0);
            if (eps[n] != eps[r] || kappa[n] != kappa[r]) ok = 0;
            if (side == 1 && !isinf(kappa[n])) ok = 0;
        }
        if (!ok) {
            or_free(s);
            return NULL;
        }
    }
    if (s->p.wall[0] == 3) {
        /* wet side walls: uniform porosity and permeability over three layers */
        int ok = p->nx >= 6;
        for (long n = 0; n < N && ok; ++n) {
            int x[3];
            coords(s, n, x);
            int side = x[0] <= 2 ? 0 : (x[0] >= p->nx - 3 ? 1 : -1);
            if (side < 0) continue;
            long r = node(s, side == 0 ? 0 : p->nx - 1, 0, 0);
            if (eps[n] != eps[r] || kappa[n] != kappa[r]) ok = 0;
        }
        if (!ok) {
            or_free(s);
            return NULL;
        }
    }
    if (s->p.wall[1] == 3) {
        /* moving walls need uniform porosity and permeability over their three
           node layers (there Eq. (accel) is explicit and Delta_nu vanishes) */
        int ok = p->ny >= 6;
        for (long n = 0; n < N && ok; ++n) {
            int x[3];
            coords(s, n, x);
            int side = x[1] <= 2 ? 0 : (x[1] >= p->ny - 3 ? 1 : -1);
            if (side < 0) continue;
            long r = node(s, 0, side == 0 ? 0 : p->ny - 1, 0);
            if (eps[n] != eps[r] || kappa[n] != kappa[r]) ok = 0;
        }
        if (!ok) {
            or_free(s);
            return NULL;
        }
    }
    return s;
}

/* Initial state, flowchart of Sec. 3.5: a_0 from the initial fields by
   Eqs. (accel), (porosity_correction_expanded) with m = rho_0 v_0 / eps, Phi_0
   by Eqs. (ex_corr), (eta_corr), then Eq. (eq_bc_f_bar) with lambda = 1:
   f_bar = (1 + 1/2) f_eq - (1/2) f_star.  rho0 is N, v0 is 3*N (superficial). */
void or_init(or_state* s, const double* rho0, const double* v0)
{
    long N = s->N;
    int D = s->D, Q = s->Q;
    for (long n = 0; n < N; ++n) {
        s->rho[n] = rho0[n];
        for (int al = 0; al < 3; ++al) {
            double v = al < D ? v0[3 * n + al] : 0.0;
            s->v[3 * n + al] = v;
            s->m[3 * n + al] = rho0[n] * v / s->eps[n];
        }
    }
    if (s->p.corr & OR_CORR_DELTA_NU)
        delta_nu(s, s->m, s->dnu);
    else
        memset(s->dnu, 0, sizeof(double) * 3 * N);
    acceleration(s);
    sweep_corrections(s);
    for (long n = 0; n < N; ++n) {
        double feq[27], fst[27];
        equilibria(s, n, feq, fst);
        for (int i = 0; i < Q; ++i) s->f[(long)i * N + n] = 1.5 * feq[i] - 0.5 * fst[i];
    }
    s->steps = 0;
}

void or_step(or_state* s, long nsteps)
{
    for (long k = 0; k < nsteps; ++k) {
        sweep_moments(s, s->f);
        sweep_velocity(s);
        sweep_corrections(s);
        sweep_collide(s);
        sweep_stream(s);
        sweep_planes(s);
        s->steps++;
    }
}

/* rho (N) and superficial v (3*N, components 2 of D2Q9 zero) of the current
   post-stream state, from S1 and S2. */
void or_moments(or_state* s, double* rho, double* v)
{
    sweep_moments(s, s->f);
    sweep_velocity(s);
    long N = s->N;
    if (rho) memcpy(rho, s->rho, sizeof(double) * N);
    if (v) memcpy(v, s->v, sizeof(double) * 3 * N);
}

/* acceleration a (3*N) and Phi_ext (3*N), Phi_eta (N) of the current state */
void or_forces(or_state* s, double* a, double* phx, double* phe)
{
    sweep_moments(s, s->f);
    sweep_velocity(s);
    sweep_corrections(s);
    long N = s->N;
    if (a) memcpy(a, s->a, sizeof(double) * 3 * N);
    if (phx) memcpy(phx, s->phx, sizeof(double) * 3 * N);
    if (phe) memcpy(phe, s->phe, sizeof(double) * N);
}

void or_get_f(const or_state* s, double* f) { memcpy(f, s->f, sizeof(double) * s->Q * s->N); }
void or_set_f(or_state* s, const double* f) { memcpy(s->f, f, sizeof(double) * s->Q * s->N); }
long or_num_steps(const or_state* s) { return s->steps; }
double or_beta(const or_state* s) { return s->beta; }
void or_weights(const or_state* s, double* w, int* c)
{
    for (int i = 0; i < s->Q; ++i) {
        w[i] = s->w[i];
        for (int al = 0; al < 3; ++al) c[3 * i + al] = s->c[i][al];
    }
}

/* static fields: mu_D, mu_F (N each), grad eps (3*N), Hessian (9*N) */
void or_static(const or_state* s, double* muD, double* muF, double* geps, double* heps)
{
    long N = s->N;
    if (muD) memcpy(muD, s->muD, sizeof(double) * N);
    if (muF) memcpy(muF, s->muF, sizeof(double) * N);
    if (geps) memcpy(geps, s->geps, sizeof(double) * 3 * N);
    if (heps) memcpy(heps, s->heps, sizeof(double) * 9 * N);
}

/* Delta_nu of an arbitrary field m (3*N) with this state's eps derivatives */
void or_delta_nu(or_state* s, const double* m, double* out) { delta_nu(s, m, out); }

/* Phi_ext (3*N) and Phi_eta (N) of arbitrary rho (N), v (3*N) */
void or_corrections(or_state* s, const double* rho, const double* v, double* phx, double* phe)
{
    long N = s->N;
    memcpy(s->rho, rho, sizeof(double) * N);
    memcpy(s->v, v, sizeof(double) * 3 * N);
    sweep_corrections(s);
    memcpy(phx, s->phx, sizeof(double) * 3 * N);
    memcpy(phe, s->phe, sizeof(double) * N);
}

/* Eq. (prod_form) on its own, for the moment identities of Appendix C */
void or_product_form(const or_state* s, double eps_rho, const double* xi, const double* P, double* out)
{
    product_form(s, eps_rho, xi, P, out);
}
