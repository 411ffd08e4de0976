// Sweep kernels: one step of the porous-media LBM as three grid-wide passes
// through device scratch fields (moments -> velocity/acceleration -> collide
// and stream).  They run every lattice, storage and boundary combination and
// are the FP64 reference path on the device; the fused kernel replaces them on
// the D3Q27 performance path.  Equation names refer to Gusev & Karlin, Sec. 3.
#pragma once

#include "lbm_common.cuh"

namespace lbm {

// Device arrays of one context, compute type T (component-major vectors).
template <typename T>
struct Fields {
    const T* eps;  // N
    const T* kap;  // N, +inf = free fluid
    T* muD;        // N
    T* muF;        // N
    T* ge;         // 3N, gradient of eps
    T* H;          // 6N, Hessian of eps: xx yy zz xy xz yz
    T* rho;        // N
    T* v1;         // 3N, Eq. (v_(1))
    T* m;          // 3N, rho v1 / eps
    T* v;          // 3N, Eq. (v_final)
    T* a;          // 3N, Eq. (accel)
    unsigned* err; // sticky error flag
};

__device__ __forceinline__ int hidx(int a, int b)
{
    if (a == b) return a;
    int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo == 0 ? (hi == 1 ? 3 : 4) : 5;
}

// a-1: drag coefficients and the gradient of eps
template <int D, typename T>
__global__ void k_static_grad(Params<T> p, Fields<T> F)
{
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    Coord c = coord_of(n, p.nx, p.ny);
    T muD, muF;
    drag_coefficients(p, F.eps[n], F.kap[n], muD, muF);
    F.muD[n] = muD;
    F.muF[n] = muF;
    for (int a = 0; a < 3; ++a) {
        T g = T(0);
        if (a < D) g = fd1(p, c, a, [&](int k) { return F.eps[shifted(p, c, a, k)]; });
        F.ge[a * p.N + n] = g;
    }
}

// a-1: Hessian of eps; diagonal by the second difference, off-diagonal by
// differencing the gradient
template <int D, typename T>
__global__ void k_static_hess(Params<T> p, Fields<T> F)
{
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    Coord c = coord_of(n, p.nx, p.ny);
    for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b) {
            T h = T(0);
            if (a < D && b < D) {
                if (a == b)
                    h = fd2(p, c, a, [&](int k) { return F.eps[shifted(p, c, a, k)]; });
                else
                    h = fd1(p, c, a, [&](int k) { return F.ge[b * p.N + shifted(p, c, a, k)]; });
            }
            F.H[hidx(a, b) * p.N + n] = h;
        }
}

// S1: Eqs. (transformed_density_moment), (transformed_momentum_moment),
// (v_(0)), (v_(1)); m = rho v1 / eps
template <int D, typename S>
__global__ void k_moments(Params<typename Codec<S>::T> p, Fields<typename Codec<S>::T> F, const S* __restrict__ f)
{
    using T = typename Codec<S>::T;
    constexpr int Q = Lattice<D>::Q;
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    T e = F.eps[n];
    T dm = T(0), P1[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        T g = Codec<S>::load(f + aa_slot<D>(p, i, n), p.w[i], p.inv_w[i]);
        dm += g;
#pragma unroll
        for (int a = 0; a < D; ++a)
            if (Lattice<D>::c(i, a) != 0) P1[a] += Lattice<D>::c(i, a) > 0 ? g : -g;
    }
    T rho = p.rho0 + dm / e;
    T v0[3] = {T(0), T(0), T(0)}, nv = T(0);
    for (int a = 0; a < D; ++a) {
        v0[a] = P1[a] / rho + T(0.5) * (e * p.b[a] + p.RT * F.ge[a * p.N + n]);
        nv += v0[a] * v0[a];
    }
    nv = sqrt(nv);
    T fac = drag_solve_factor(F.muD[n], F.muF[n], nv);
    F.rho[n] = rho;
    for (int a = 0; a < 3; ++a) {
        T v1 = v0[a] * fac;
        F.v1[a * p.N + n] = v1;
        F.m[a * p.N + n] = rho * v1 / e;
    }
    if (!(rho > T(0)) || !isfinite(rho) || !(nv * fac <= T(0.5) * e)) atomicOr(F.err, ERR_DIVERGED);
}

// S2: Delta_nu(m) by Eq. (porosity_correction_expanded) with constant nu_eff,
// v = v1 + Delta_nu / (2 rho) (Eq. (v_final)) and the acceleration Eq. (accel)
// whose drag uses the final v.  With keep_v1 (initialisation) v stays v1.
template <int D, typename T>
__global__ void k_velocity(Params<T> p, Fields<T> F, int keep_v1)
{
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    Coord c = coord_of(n, p.nx, p.ny);
    T rho = F.rho[n], e = F.eps[n];
    T dnu[3] = {T(0), T(0), T(0)};
    if (p.corr & 1) {
        T m[3], ge[3], dm[3][3];
        for (int a = 0; a < D; ++a) {
            m[a] = F.m[a * p.N + n];
            ge[a] = F.ge[a * p.N + n];
        }
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b)
                dm[a][b] = fd1(p, c, b, [&](int k) { return F.m[a * p.N + shifted(p, c, b, k)]; });
        T trH = T(0), divm = T(0);
        for (int a = 0; a < D; ++a) {
            trH += F.H[a * p.N + n];
            divm += dm[a][a];
        }
        for (int a = 0; a < D; ++a) {
            T r = trH * m[a] + divm * ge[a];
            for (int b = 0; b < D; ++b) r += F.H[hidx(a, b) * p.N + n] * m[b] + dm[a][b] * ge[b];
            dnu[a] = p.nu_eff * r;
        }
    }
    T v[3] = {T(0), T(0), T(0)}, nv = T(0);
    for (int a = 0; a < D; ++a) {
        v[a] = F.v1[a * p.N + n] + (keep_v1 ? T(0) : dnu[a] / (T(2) * rho));
        nv += v[a] * v[a];
    }
    nv = sqrt(nv);
    T muD = F.muD[n], muF = F.muF[n];
    for (int a = 0; a < 3; ++a) {
        T acc = T(0);
        if (a < D) acc = e * p.b[a] - muD * v[a] - muF * nv * v[a] + p.RT * F.ge[a * p.N + n] + dnu[a] / rho;
        F.v[a * p.N + n] = v[a];
        F.a[a * p.N + n] = acc;
    }
}

// Appendix F: one Picard iteration of the implicit velocity equation
//   c1 v + c2 |v| v = v(0) + Delta_nu(rho v / eps) / (2 rho)
// from the iterate vin (3N) into vout (3N), under-relaxed by omega; v(0) is
// recovered from v1 (c1 v1 + c2 |v1| v1 = v(0), Eq. (v_(1))).  On the last
// iteration the acceleration of Eq. (accel) is formed with this iteration's
// Delta_nu.
template <int D, typename T>
__global__ void k_picard(Params<T> p, Fields<T> F, const T* __restrict__ vin, T* __restrict__ vout, int last)
{
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    Coord c = coord_of(n, p.nx, p.ny);
    T rho = F.rho[n], e = F.eps[n];
    auto mfield = [&](int a, long long j) { return F.rho[j] * vin[a * p.N + j] / F.eps[j]; };
    T m[3], ge[3], dm[3][3];
    for (int a = 0; a < D; ++a) {
        m[a] = mfield(a, n);
        ge[a] = F.ge[a * p.N + n];
    }
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) dm[a][b] = fd1(p, c, b, [&](int k) { return mfield(a, shifted(p, c, b, k)); });
    T trH = T(0), divm = T(0);
    for (int a = 0; a < D; ++a) {
        trH += F.H[a * p.N + n];
        divm += dm[a][a];
    }
    T dnu[3] = {T(0), T(0), T(0)};
    for (int a = 0; a < D; ++a) {
        T r = trH * m[a] + divm * ge[a];
        for (int b = 0; b < D; ++b) r += F.H[hidx(a, b) * p.N + n] * m[b] + dm[a][b] * ge[b];
        dnu[a] = p.nu_eff * r;
    }
    T muD = F.muD[n], muF = F.muF[n];
    T v1[3] = {T(0), T(0), T(0)}, nv1 = T(0);
    for (int a = 0; a < D; ++a) {
        v1[a] = F.v1[a * p.N + n];
        nv1 += v1[a] * v1[a];
    }
    nv1 = sqrt(nv1);
    T c1 = T(1) + T(0.5) * muD, c2 = T(0.5) * muF;
    T sv[3] = {T(0), T(0), T(0)}, ns = T(0);
    for (int a = 0; a < D; ++a) {
        sv[a] = (c1 * v1[a] + c2 * nv1 * v1[a]) + dnu[a] / (T(2) * rho);
        ns += sv[a] * sv[a];
    }
    ns = sqrt(ns);
    T fac = drag_solve_factor(muD, muF, ns);
    T w = p.picard_omega;
    T v[3] = {T(0), T(0), T(0)}, nv = T(0);
    for (int a = 0; a < D; ++a) {
        v[a] = (T(1) - w) * vin[a * p.N + n] + w * (sv[a] * fac);
        nv += v[a] * v[a];
    }
    nv = sqrt(nv);
    for (int a = 0; a < 3; ++a) vout[a * p.N + n] = v[a];
    if (last)
        for (int a = 0; a < 3; ++a)
            F.a[a * p.N + n] = a < D ? e * p.b[a] - muD * v[a] - muF * nv * v[a] + p.RT * F.ge[a * p.N + n] + dnu[a] / rho
                                     : T(0);
}

// S3 + S4 at node n: Phi_ext, Phi_eta from neighbouring rho, v (Eqs. (ex_corr),
// (eta_corr)), then the equilibrium parameters Eqs. (xi_alpha_eq),
// (P_alpha_alpha_eq), (xi_alpha_*), (P_aa_*) with lambda = 1, as deviations.
template <int D, typename T>
__device__ __forceinline__ void node_equilibria(const Params<T>& p, const Fields<T>& F, long long n,
                                                ProductDev<D, T>& Peq, ProductDev<D, T>& Pst, T& rho, T& e)
{
    Coord c = coord_of(n, p.nx, p.ny);
    rho = F.rho[n];
    e = F.eps[n];
    T phx[3] = {T(0), T(0), T(0)}, divv = T(0);
    for (int a = 0; a < D; ++a) {
        if (p.corr & 2)
            phx[a] = fd1(p, c, a, [&](int k) {
                long long j = shifted(p, c, a, k);
                T r = F.rho[j], va = F.v[a * p.N + j], ej = F.eps[j];
                return r * va * p.one_m_3RT - r * va * va * va / (ej * ej);
            });
        if (p.corr & 4) divv += fd1(p, c, a, [&](int k) { return F.v[a * p.N + shifted(p, c, a, k)]; });
    }
    T phe = (p.corr & 4) ? rho * p.eta_coef * divv : T(0);
    T xe[3], qe[3], xs[3], qs[3];
    for (int a = 0; a < D; ++a) {
        T va = F.v[a * p.N + n], aa = F.a[a * p.N + n];
        xe[a] = va / e;
        qe[a] = xe[a] * xe[a];
        xs[a] = (va + aa) / e;
        qs[a] = xs[a] * xs[a] + (phx[a] + phe) / (e * rho);
    }
    Peq.set(xe, qe, p.RT);
    Pst.set(xs, qs, p.RT);
}

// S4 + S5: collide (Eqs. (dicrete_scheme), (momentum_rate), lambda = 1) and push
// each post-collision population to x + c_i, or reflect it into the opposite
// slot of x when x + c_i lies beyond a non-periodic face (a wall; at an inlet /
// outlet plane or a moving wall the reflected value serves the bounce-back
// density, Eq. (bc_density_BounceBack), and the plane rebuild replaces it).
// The stored deviation is rebased on the destination's porosity.
template <int D, typename S>
__global__ void k_collide_stream(Params<typename Codec<S>::T> p, Fields<typename Codec<S>::T> F,
                                 const S* __restrict__ fin, S* __restrict__ fout)
{
    using T = typename Codec<S>::T;
    constexpr int Q = Lattice<D>::Q;
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    ProductDev<D, T> Peq, Pst;
    T rho, e;
    node_equilibria<D, T>(p, F, n, Peq, Pst, rho, e);
    Coord c = coord_of(n, p.nx, p.ny);
    T drho = rho - p.rho0;
    T beta = p.beta;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        T fe, fs;
        T de = Peq.dev(i, fe), ds = Pst.dev(i, fs);
        T geq = e * (drho * fe + p.rho0 * de);
        T gst = e * (drho * fs + p.rho0 * ds);
        T g = Codec<S>::load(fin + i * p.NS + n, p.w[i], p.inv_w[i]);
        T gpc = g + T(2) * beta * (geq - g) + (T(1) - beta) * (gst - geq);
        int d[3], out = 0;
        for (int a = 0; a < 3; ++a) {
            int k = c.x[a] + Lattice<D>::c(i, a), nn = dim_of(a, p.nx, p.ny, p.nz);
            if (k < 0 || k >= nn) {
                if (p.wall[a]) out = 1;
                k = wrap(k, nn);
            }
            d[a] = k;
        }
        if (out) {
            int o = Lattice<D>::opp(i);
            Codec<S>::store(fout + o * p.NS + n, gpc, p.w[o], p.inv_w[o]);
        } else {
            long long j = d[0] + (long long)p.nx * (d[1] + (long long)p.ny * d[2]);
            T shift = (e - F.eps[j]) * p.w[i] * p.rho0;
            Codec<S>::store(fout + i * p.NS + j, gpc + shift, p.w[i], p.inv_w[i]);
        }
    }
}

// Initial populations, Eq. (eq_bc_f_bar) with lambda = 1: f = 1.5 f_eq - 0.5 f_star
template <int D, typename S>
__global__ void k_init_populations(Params<typename Codec<S>::T> p, Fields<typename Codec<S>::T> F, S* __restrict__ f)
{
    using T = typename Codec<S>::T;
    constexpr int Q = Lattice<D>::Q;
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    ProductDev<D, T> Peq, Pst;
    T rho, e;
    node_equilibria<D, T>(p, F, n, Peq, Pst, rho, e);
    T drho = rho - p.rho0;
    for (int i = 0; i < Q; ++i) {
        T fe, fs;
        T de = Peq.dev(i, fe), ds = Pst.dev(i, fs);
        T geq = e * (drho * fe + p.rho0 * de);
        T gst = e * (drho * fs + p.rho0 * ds);
        Codec<S>::store(f + i * p.NS + n, T(1.5) * geq - T(0.5) * gst, p.w[i], p.inv_w[i]);
    }
}

// set rho and v1 from initial fields (FP64 input), m = rho v1 / eps
template <typename T>
__global__ void k_set_initial(Params<T> p, Fields<T> F, const double* rho0, const double* v0)
{
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    T r = rho0 ? T(rho0[n]) : p.rho0;
    F.rho[n] = r;
    for (int a = 0; a < 3; ++a) {
        T va = v0 ? T(v0[a * p.N + n]) : T(0);
        F.v1[a * p.N + n] = va;
        F.m[a * p.N + n] = r * va / F.eps[n];
    }
}

template <typename T>
__global__ void k_fill_v0(Params<T> p, double* v0, double vx, double vy, double vz)
{
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    v0[n] = vx;
    v0[p.N + n] = vy;
    v0[2 * p.N + n] = vz;
}

// macroscopic output in FP64
template <typename T>
__global__ void k_export_moments(Params<T> p, Fields<T> F, double* rho, double* v)
{
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    if (rho) rho[n] = (double)F.rho[n];
    if (v)
        for (int a = 0; a < 3; ++a) v[a * p.N + n] = (double)F.v[a * p.N + n];
}

// populations f_bar = g + eps w_i rho0 in FP64, and back
template <int D, typename S>
__global__ void k_decode(Params<typename Codec<S>::T> p, Fields<typename Codec<S>::T> F, const S* f, double* out)
{
    constexpr int Q = Lattice<D>::Q;
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    double e = (double)F.eps[n];
    for (int i = 0; i < Q; ++i)
        out[i * p.N + n] = (double)Codec<S>::load(f + aa_slot<D>(p, i, n), p.w[i], p.inv_w[i]) + e * (double)p.w[i] * (double)p.rho0;
}

template <int D, typename S>
__global__ void k_encode(Params<typename Codec<S>::T> p, Fields<typename Codec<S>::T> F, const double* in, S* f)
{
    using T = typename Codec<S>::T;
    constexpr int Q = Lattice<D>::Q;
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    double e = (double)F.eps[n];
    for (int i = 0; i < Q; ++i)
        Codec<S>::store(f + aa_slot<D>(p, i, n), T(in[i * p.N + n] - e * (double)p.w[i] * (double)p.rho0), p.w[i], p.inv_w[i]);
}


// S6: inlet (x = 0, prescribed v_b) and outlet (x = nx-1, prescribed rho_b)
// wet-node planes, rebuilt after streaming from the post-stream populations f:
// the boundary density by mass continuity (Eqs. (boundary_density_split),
// (bc_rho_components_def), (bc_density_impermWall); at the outlet the relation
// is solved for the normal velocity and the tangential velocity comes from the
// interior neighbour), then every population by non-equilibrium extrapolation
// from the interior neighbour x_f (Eqs. (NEEM_bc_f_bar), (zeta_beta_NEEM),
// zeta = 1 since beta is uniform, lambda = 1).  The porosity is uniform near
// the planes (checked at creation), so Eq. (accel) has no gradient terms there.
template <int D, typename T>
__device__ __forceinline__ void feq_full(const Params<T>& p, T e, T rho, const T* v, T* out)
{
    constexpr int Q = Lattice<D>::Q;
    T xi[3], q[3];
    for (int a = 0; a < D; ++a) {
        xi[a] = v[a] / e;
        q[a] = xi[a] * xi[a];
    }
    ProductDev<D, T> P;
    P.set(xi, q, p.RT);
    for (int i = 0; i < Q; ++i) {
        T full;
        T dev = P.dev(i, full);
        out[i] = e * ((rho - p.rho0) * full + p.rho0 * dev);  // f_eq - eps w_i rho0
    }
}

template <int D, typename T>
__device__ __forceinline__ void accel_uniform(const Params<T>& p, T e, T muD, T muF, const T* v, T* a)
{
    T nv = T(0);
    for (int b = 0; b < D; ++b) nv += v[b] * v[b];
    nv = sqrt(nv);
    for (int b = 0; b < 3; ++b) a[b] = b < D ? e * p.b[b] - muD * v[b] - muF * nv * v[b] : T(0);
}

// Rebuild of one wet node b whose interior neighbour along the normal axis ax
// is fn (side 0: the low face, outward normal -1; side 1: the high face, +1):
//   mode 0: prescribed velocity vt (an inlet); the density by mass continuity;
//   mode 1: prescribed density rho_t (pressure outlet): the normal velocity by
//           continuity, the tangential velocity from the interior neighbour;
//   mode 2: prescribed velocity vt and density rho_t (a corner column);
//   mode 3: a wet-node wall with velocity vt; the density by mass continuity,
//           or the bounce-back density if plane_density asks for it (the
//           paper states it for solid boundaries);
// then every population by the reconstruction that plane_scheme selects.
template <int D, typename S>
__device__ void rebuild_wet_node(const Params<typename Codec<S>::T>& p, const Fields<typename Codec<S>::T>& F,
                                 S* __restrict__ f, long long b, long long fn, int ax, int side, int mode,
                                 const typename Codec<S>::T* vt, typename Codec<S>::T rho_t)
{
    using T = typename Codec<S>::T;
    constexpr int Q = Lattice<D>::Q;
    T nout = side == 0 ? T(-1) : T(1);
    T eb = F.eps[b], ef = F.eps[fn];
    // interior neighbour: moments, velocity (Delta_nu = 0, grad eps = 0), acceleration
    T gf[Q];
    T dm = T(0), P1[3] = {T(0), T(0), T(0)};
    for (int i = 0; i < Q; ++i) {
        gf[i] = Codec<S>::load(f + aa_slot<D>(p, i, fn), p.w[i], p.inv_w[i]);
        dm += gf[i];
        for (int a = 0; a < D; ++a) P1[a] += T(Lattice<D>::c(i, a)) * gf[i];
    }
    T rf = p.rho0 + dm / ef;
    T v0[3] = {T(0), T(0), T(0)}, nv0 = T(0);
    for (int a = 0; a < D; ++a) {
        v0[a] = P1[a] / rf + T(0.5) * ef * p.b[a];
        nv0 += v0[a] * v0[a];
    }
    nv0 = sqrt(nv0);
    T fac = drag_solve_factor(F.muD[fn], F.muF[fn], nv0);
    T vf[3] = {T(0), T(0), T(0)}, af[3];
    for (int a = 0; a < D; ++a) vf[a] = v0[a] * fac;
    accel_uniform<D, T>(p, ef, F.muD[fn], F.muF[fn], vf, af);
    // boundary node: rho^0 and rho^+ from the known populations
    T r0 = T(0), rp = T(0);
    for (int i = 0; i < Q; ++i) {
        int cn = Lattice<D>::c(i, ax) * (side == 0 ? -1 : 1);
        if (cn < 0) continue;
        T fi = Codec<S>::load(f + aa_slot<D>(p, i, b), p.w[i], p.inv_w[i]) + eb * p.w[i] * p.rho0;
        if (cn == 0) r0 += fi;
        else rp += fi;
    }
    r0 /= eb;
    rp /= eb;
    T vb[3] = {T(0), T(0), T(0)}, ab[3], rb;
    if (mode != 1) {
        for (int a = 0; a < D; ++a) vb[a] = vt[a];
        accel_uniform<D, T>(p, eb, F.muD[b], F.muF[b], vb, ab);
        if (mode == 2) {
            rb = rho_t;
        } else if (p.plane_density == 1 && mode == 3) {
            // Eq. (bc_density_BounceBack): the unknown slots hold the reflected
            // post-collision outgoing populations after the push
            T dsum = T(0);
            for (int i = 0; i < Q; ++i) dsum += Codec<S>::load(f + aa_slot<D>(p, i, b), p.w[i], p.inv_w[i]);
            rb = p.rho0 + dsum / eb;
        } else {
            rb = eb * (r0 + T(2) * rp) / (eb + vb[ax] * nout - T(0.5) * ab[ax] * nout);
        }
    } else {
        rb = rho_t;
        T vperp = eb * (r0 + T(2) * rp) / rb - eb + T(0.5) * eb * p.b[ax] * nout;
        for (int a = 0; a < D; ++a) vb[a] = vf[a];
        vb[ax] = vperp * nout;
        accel_uniform<D, T>(p, eb, F.muD[b], F.muF[b], vb, ab);
    }
    T vsb[3], vsf[3];
    for (int a = 0; a < 3; ++a) {
        vsb[a] = vb[a] + ab[a];
        vsf[a] = vf[a] + af[a];
    }
    T feb[Q], fef[Q], fsb[Q], fsf[Q];
    feq_full<D, T>(p, eb, rb, vb, feb);
    feq_full<D, T>(p, ef, rf, vf, fef);
    feq_full<D, T>(p, eb, rb, vsb, fsb);
    feq_full<D, T>(p, ef, rf, vsf, fsf);
    // In deviations from eps w_i rho0 (feq_full returns f_eq - eps w_i rho0): the
    // eps w_i rho0 parts of the populations and equilibria cancel in every scheme.
    if (p.plane_scheme == 1) {
        // equilibrium scheme, Eq. (eq_bc_f_bar): f_bar = 1.5 f_tgt - 0.5 f_*
        for (int i = 0; i < Q; ++i) Codec<S>::store(f + aa_slot<D>(p, i, b), T(1.5) * feb[i] - T(0.5) * fsb[i], p.w[i], p.inv_w[i]);
    } else if (p.plane_scheme == 2) {
        // Tamm--Mott-Smith, Eq. (f_i_neq_TMS) in the three steps of Sec. 3.4;
        // P- = populations entering from outside (c_i . n_out < 0)
        const T omb = T(1) - p.beta;
        T dr = T(0), dj[3] = {T(0), T(0), T(0)};
        for (int i = 0; i < Q; ++i) {
            if (Lattice<D>::c(i, ax) * (side == 0 ? -1 : 1) < 0) continue;
            const T d = Codec<S>::load(f + aa_slot<D>(p, i, b), p.w[i], p.inv_w[i]) - T(1.5) * feb[i] + T(0.5) * fsb[i];
            dr += d;
            for (int a = 0; a < D; ++a) dj[a] += T(Lattice<D>::c(i, a)) * d;
        }
        const T rloc = (eb * rb + omb * dr) / eb;
        T vloc[3] = {T(0), T(0), T(0)};
        for (int a = 0; a < D; ++a) vloc[a] = (rb * vb[a] + omb * dj[a]) / rloc;
        T floc[Q];
        feq_full<D, T>(p, eb, rloc, vloc, floc);
        for (int i = 0; i < Q; ++i) {
            const T corr = (feb[i] - floc[i]) / omb;
            const bool unknown = Lattice<D>::c(i, ax) * (side == 0 ? -1 : 1) < 0;
            const T g = unknown ? corr + T(1.5) * feb[i] - T(0.5) * fsb[i]
                                : corr + Codec<S>::load(f + aa_slot<D>(p, i, b), p.w[i], p.inv_w[i]);
            Codec<S>::store(f + aa_slot<D>(p, i, b), g, p.w[i], p.inv_w[i]);
        }
    } else {
        // Eq. (NEEM_bc_f_bar) with zeta = 1
        for (int i = 0; i < Q; ++i) {
            T g = gf[i] + T(1.5) * (feb[i] - fef[i]) + T(0.5) * (fsf[i] - fsb[i]);
            Codec<S>::store(f + aa_slot<D>(p, i, b), g, p.w[i], p.inv_w[i]);
        }
    }
}

// Eq. (s_cinf): the smoothstep S(psi), 0 for psi <= 0, 1 for psi >= 1
template <typename T>
__device__ __forceinline__ T smoothstep(T psi)
{
    if (psi <= T(0)) return T(0);
    if (psi >= T(1)) return T(1);
    const T a = exp(T(-1) / psi), b = exp(T(-1) / (T(1) - psi));
    return a / (a + b);
}

// Velocity of the moving wall on row y = 0 (side 0) or ny-1 (side 1) at column
// x: wall_v[side], its x component tapered by Eq. (cavity_velocity_profile)
// with the regularised lid.
template <typename T>
__device__ __forceinline__ void wall_velocity(const Params<T>& p, int side, long long x, T* vt)
{
    for (int a = 0; a < 3; ++a) vt[a] = p.wall_v[side][a];
    if (p.lid_profile == 1) {
        const T L = T(p.nx - 1), xd = T(x), d = xd < L - xd ? xd : L - xd;
        vt[0] *= smoothstep(d / (p.lid_delta * L));
    }
}

// One thread per wet node of the two planes normal to axis ax.  ax = 0: the
// inlet (x = 0; inlet_v, or the Poiseuille profile of Eq. (cylinder_inlet_BC))
// and the outlet (x = nx-1; prescribed density, or the zero-gradient outflow
// of Eq. (f_bar_outflow_BC), which copies the populations entering from
// outside from the interior neighbour), or wet-node side walls at rest; with
// moving walls on y the corner columns are left to k_plane_corners.  ax = 1:
// the moving walls at y = 0 and y = ny-1 (wall_v[0], [1], optionally the
// regularised lid); with x sides their end columns are the corners.
template <int D, typename S>
__global__ void k_planes(Params<typename Codec<S>::T> p, Fields<typename Codec<S>::T> F, S* __restrict__ f, int ax)
{
    using T = typename Codec<S>::T;
    constexpr int Q = Lattice<D>::Q;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int nb = ax == 0 ? p.nx : p.ny;  // nodes along the normal
    long long plane = ax == 0 ? (long long)p.ny * p.nz : (long long)p.nx * p.nz;
    if (t >= 2 * plane) return;
    int side = t >= plane ? 1 : 0;
    long long r = t - side * plane;  // ax 0: y + ny z; ax 1: x + nx z
    const int kb = side == 0 ? 0 : nb - 1, kf = side == 0 ? 1 : nb - 2;
    long long b, fn;
    if (ax == 0) {
        const int y = (int)(r % p.ny);
        if (p.yplanes && (y == 0 || y == p.ny - 1)) return;  // a corner column
        b = kb + (long long)p.nx * r;
        fn = kf + (long long)p.nx * r;
        if (p.xwalls) {
            const T rest[3] = {T(0), T(0), T(0)};
            rebuild_wet_node<D, S>(p, F, f, b, fn, 0, side, 3, rest, T(0));
            return;
        }
        if (side == 1 && p.outlet == 1) {
            for (int i = 0; i < Q; ++i)
                if (Lattice<D>::c(i, 0) < 0) f[aa_slot<D>(p, i, b)] = f[aa_slot<D>(p, i, fn)];
            return;
        }
        if (side == 0) {
            T vt[3] = {p.v_in[0], p.v_in[1], p.v_in[2]};
            if (p.inlet_profile == 1) {
                const T eta = p.yplanes ? T(y) / T(p.ny - 1) : (T(y) + T(0.5)) / T(p.ny);
                vt[0] = T(6) * p.v_in[0] * eta * (T(1) - eta);
                vt[1] = vt[2] = T(0);
            }
            rebuild_wet_node<D, S>(p, F, f, b, fn, 0, 0, 0, vt, T(0));
        } else {
            rebuild_wet_node<D, S>(p, F, f, b, fn, 0, 1, 1, nullptr, p.rho_out);
        }
    } else {
        const long long x = r % p.nx, z = r / p.nx;
        if ((p.planes || p.xwalls) && (x == 0 || x == p.nx - 1)) return;  // a corner column
        b = x + (long long)p.nx * (kb + (long long)p.ny * z);
        fn = x + (long long)p.nx * (kf + (long long)p.ny * z);
        T vt[3];
        wall_velocity(p, side, x, vt);
        rebuild_wet_node<D, S>(p, F, f, b, fn, 1, side, 3, vt, T(0));
    }
}

// The x planes of a D3Q27 grid with reduced storage in the common case --
// velocity inlet at x = 0 (uniform or Poiseuille), pressure outlet at
// x = nx-1, non-equilibrium extrapolation (zeta = 1, lambda = 1), density by
// mass continuity: rebuild_wet_node's modes 0 and 1, one warp per plane node
// and one lane per population.  The plane's nodes lie nx apart, so a thread per
// node walks 27 scattered populations one after another; here a warp issues
// them together, and the sums over populations (the neighbour's moments, the
// known populations' rho^0 and rho^+) are warp reductions (their order of
// summation differs from rebuild_wet_node's).
template <typename S>
__global__ void __launch_bounds__(256) k_planes_x_warp(Params<float> p, Fields<float> F, S* __restrict__ f)
{
    const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const long long plane = (long long)p.ny * p.nz;
    if (wid >= 2 * plane) return;  // whole warps
    const int side = wid >= plane ? 1 : 0;
    const long long r = wid - side * plane;  // y + ny z
    const int y = (int)(r % p.ny);
    if (p.yplanes && (y == 0 || y == p.ny - 1)) return;  // a corner column
    const long long b = (side == 0 ? 0 : p.nx - 1) + (long long)p.nx * r;
    const long long fn = (side == 0 ? 1 : p.nx - 2) + (long long)p.nx * r;
    const float nout = side == 0 ? -1.f : 1.f;
    const bool act = lane < 27;
    const int i = act ? lane : 0;
    const float c[3] = {float(i % 3 - 1), float((i / 3) % 3 - 1), float(i / 9 - 1)};
    const float eb = F.eps[b], ef = F.eps[fn];
    const float wi = p.w[i], iwi = p.inv_w[i];
    // interior neighbour's population i; known population i of the plane node
    // (c_x . n_out >= 0)
    const float cn = c[0] * nout;
    const float gf = act ? Codec<S>::load(f + aa_slot<3>(p, i, fn), wi, iwi) : 0.f;
    const float fb = act && cn >= 0.f ? Codec<S>::load(f + aa_slot<3>(p, i, b), wi, iwi) + eb * wi * p.rho0 : 0.f;
    float sm[6] = {gf, c[0] * gf, c[1] * gf, c[2] * gf, cn == 0.f ? fb : 0.f, cn > 0.f ? fb : 0.f};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 6; ++k) sm[k] += __shfl_xor_sync(0xffffffffu, sm[k], o);
    // neighbour: rho, v (Delta_nu = 0, grad eps = 0 near the plane), a
    const float rf = p.rho0 + sm[0] / ef;
    float v0[3], nv0 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        v0[a] = sm[1 + a] / rf + 0.5f * ef * p.b[a];
        nv0 += v0[a] * v0[a];
    }
    nv0 = sqrtf(nv0);
    const float muDf = F.muD[fn], muFf = F.muF[fn], muDb = F.muD[b], muFb = F.muF[b];
    const float fac = drag_solve_factor(muDf, muFf, nv0);
    float vf[3], af[3], vb[3], ab[3];
    auto accel = [&](float e, float muD, float muF, const float* v, float* acc) {
        const float nv = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[a] = e * p.b[a] - muD * v[a] - muF * nv * v[a];
    };
#pragma unroll
    for (int a = 0; a < 3; ++a) vf[a] = v0[a] * fac;
    accel(ef, muDf, muFf, vf, af);
    const float r0 = sm[4] / eb, rp = sm[5] / eb;
    float rb;
    if (side == 0) {
        vb[0] = p.v_in[0];
        vb[1] = p.v_in[1];
        vb[2] = p.v_in[2];
        if (p.inlet_profile == 1) {
            const float eta = p.yplanes ? float(y) / float(p.ny - 1) : (float(y) + 0.5f) / float(p.ny);
            vb[0] = 6.f * p.v_in[0] * eta * (1.f - eta);
            vb[1] = vb[2] = 0.f;
        }
        accel(eb, muDb, muFb, vb, ab);
        rb = eb * (r0 + 2.f * rp) / (eb + vb[0] * nout - 0.5f * ab[0] * nout);
    } else {
        rb = p.rho_out;
        const float vperp = eb * (r0 + 2.f * rp) / rb - eb + 0.5f * eb * p.b[0] * nout;
        vb[0] = vperp * nout;
        vb[1] = vf[1];
        vb[2] = vf[2];
        accel(eb, muDb, muFb, vb, ab);
    }
    // the four equilibria of population i (deviations from eps w_i rho0): the
    // product form of ProductDev with the lane's own digits picked by selects,
    // so that no table is indexed by the lane (same operations, same results)
    const int dg[3] = {i % 3, (i / 3) % 3, i / 9};
    auto feq = [&](float e, float rho, const float* v) {
        float a0[3], dp[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float xi = v[a] / e, q = xi * xi;
            a0[a] = dg[a] == 1 ? 1.f - p.RT : p.RT * 0.5f;
            dp[a] = dg[a] == 0 ? (q - xi) * 0.5f : dg[a] == 1 ? -q : (q + xi) * 0.5f;
        }
        const float px = a0[0] + dp[0], py = a0[1] + dp[1], pz = a0[2] + dp[2];
        const float full = px * py * pz;
        const float dev = dp[0] * (py * pz) + a0[0] * (dp[1] * pz + a0[1] * dp[2]);
        return e * ((rho - p.rho0) * full + p.rho0 * dev);
    };
    float vsb[3], vsf[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        vsb[a] = vb[a] + ab[a];
        vsf[a] = vf[a] + af[a];
    }
    // Eq. (NEEM_bc_f_bar) with zeta = 1
    const float g = gf + 1.5f * (feq(eb, rb, vb) - feq(ef, rf, vf)) + 0.5f * (feq(ef, rf, vsf) - feq(eb, rb, vsb));
    if (act) Codec<S>::store(f + aa_slot<3>(p, i, b), g, wi, iwi);
}

// The four corner columns where the x sides (inlet / outlet planes or wet side
// walls) meet moving walls, one thread per corner node, after the x sides and
// before the wall rows: the y wall's velocity there, and for the density the
// node's own bounce-back density when the walls take it (the bounce-back
// operation, the paper's second remedy where boundaries meet), else the density
// of the diagonal bulk neighbour (the paper extrapolates the corner density
// from neighbouring bulk fluid nodes; this is the zeroth-order extrapolation);
// then the wall's reconstruction with the interior neighbour on the x side.
template <int D, typename S>
__global__ void k_plane_corners(Params<typename Codec<S>::T> p, Fields<typename Codec<S>::T> F, S* __restrict__ f)
{
    using T = typename Codec<S>::T;
    constexpr int Q = Lattice<D>::Q;
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= 4LL * p.nz) return;
    const int sx = (int)(t & 1), sy = (int)((t >> 1) & 1);
    const long long z = t >> 2;
    const int xb = sx ? p.nx - 1 : 0, xa = sx ? p.nx - 2 : 1;
    const int yb = sy ? p.ny - 1 : 0, yf = sy ? p.ny - 2 : 1;
    auto node = [&](int x, int y) { return x + (long long)p.nx * (y + (long long)p.ny * z); };
    const long long b = node(xb, yb), fn = node(xb, yf);
    const long long d = p.plane_density == 1 ? b : node(xa, yf);
    T dsum = T(0);
    for (int i = 0; i < Q; ++i) dsum += Codec<S>::load(f + aa_slot<D>(p, i, d), p.w[i], p.inv_w[i]);
    const T rho_d = p.rho0 + dsum / F.eps[d];
    T vt[3];
    wall_velocity(p, sy, xb, vt);
    rebuild_wet_node<D, S>(p, F, f, b, fn, 1, sy, 2, vt, rho_d);
}

}  // namespace lbm
