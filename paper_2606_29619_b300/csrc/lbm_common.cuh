// Shared device-side definitions of the porous-media LBM library: lattice
// tables, run parameters, the population storage codec and the finite-
// difference stencils.  Equation names refer to Gusev & Karlin, Sec. 3.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// D2Q9 / D3Q27 (Sec. 3.1): i = ix + 3 iy (+ 9 iz), c = digit - 1, opposite Q-1-i.
template <int D>
struct Lattice {
    static constexpr int Q = D == 2 ? 9 : 27;
    __host__ __device__ static constexpr int c(int i, int a)
    {
        return a == 0 ? i % 3 - 1 : a == 1 ? (i / 3) % 3 - 1 : (D == 3 ? i / 9 - 1 : 0);
    }
    __host__ __device__ static constexpr int opp(int i) { return Q - 1 - i; }
};

// Error bits of the sticky device flag.  ERR_WAIT_TIMEOUT: a kernel gave up
// waiting for its copies into shared memory (bounded wait) and skipped its work.
enum : unsigned { ERR_DIVERGED = 1u, ERR_WAIT_TIMEOUT = 2u };

// Everything a step needs besides the arrays, in the compute type T.
template <typename T>
struct Params {
    int nx, ny, nz;
    long long N;
    long long NS;    // stride of the population planes (elements), pop_stride(N)
    int wall[3];     // non-periodic axis: one-sided stencils at its first / last node, and populations
                     // leaving through its faces are reflected (halfway bounce-back at a wall; at an
                     // inlet / outlet plane or moving wall they hold the bounce-back density's
                     // post-collision values until the plane rebuild)
    int planes;      // inlet (x = 0) and outlet (x = nx-1) planes
    int yplanes;     // moving wet-node walls at y = 0 and y = ny-1
    int plane_scheme; // their reconstruction: LBM_PLANES_NEEM / _EQUILIBRIUM / _TMS
    int plane_density; // density of wet-node walls: LBM_DENSITY_CONTINUITY / _BOUNCE_BACK
    int outlet;      // LBM_OUTLET_PRESSURE / _ZERO_GRADIENT
    int inlet_profile; // LBM_INLET_UNIFORM / _POISEUILLE
    int xwalls;      // wet-node walls at rest at x = 0 and x = nx-1
    int lid_profile; // LBM_LID_UNIFORM / _REGULARISED
    T lid_delta;     // relative width of each lid taper
    int corr;        // LBM_CORR_* mask
    int ergun;       // Forchheimer coefficient from the Ergun correlation
    T RT;            // lattice temperature
    T one_m_3RT;     // 1 - 3 RT (Eq. (ex_corr))
    T rho0;          // deviation reference density
    T b[3];          // body acceleration
    T beta;          // Eq. (beta_def) from Eq. (nu_eff_def)
    T nu_eff;        // effective shear viscosity
    T nu_f;          // fluid viscosity (Darcy coefficient)
    T forch;         // F_eps when not Ergun
    T eta_coef;      // RT (2/D - eta_eff/nu_eff), Eq. (eta_corr)
    int picard_iters; // Picard iterations of the velocity (sweep path), 0 = one-shot
    T picard_omega;   // their under-relaxation
    T v_in[3];       // inlet superficial velocity
    T wall_v[2][3];  // superficial velocities of the moving walls (y = 0, y = ny-1)
    T rho_out;       // outlet density
    T w[27];         // lattice weights, Eq. (eq_weights)
    T inv_w[27];
    int aa_parity;   // layout of the stored state (aa_slot): 0 natural, 1 after an even in-place step
};

// Stride of the population planes: N rounded up to a multiple of 128 bytes,
// so that every plane starts on a cache-line boundary and the paired (8- or
// 4-byte) accesses of two x-adjacent nodes stay aligned in every plane.
inline long long pop_stride(long long N, int bytes)
{
    const long long line = 128 / bytes;
    return (N + line - 1) / line * line;
}

// Optional event marks around the kernels of a step (measurement only): mark()
// records the next event of a host-owned array on the launch stream.
struct KernelClock {
    cudaEvent_t* ev = nullptr;
    int n = 0, cap = 0;
    void mark(cudaStream_t st)
    {
        if (ev && n < cap) cudaEventRecord(ev[n++], st);
    }
};
inline void clock_mark(KernelClock* kc, cudaStream_t st)
{
    if (kc) kc->mark(st);
}

// In-place (AA) streaming keeps one population array.  A step of parity 0
// reads f_bar_i of node x from slot i of x and writes the post-collision
// population back into slot opp(i) of x; a step of parity 1 reads f_bar_i of x
// from slot opp(i) of x - c_i and writes the post-collision population to
// slot i of x + c_i.  A population that would cross a non-periodic face stays
// at its node (halfway bounce-back), in slot i of x.  Between steps the state
// therefore has one of two layouts; aa_slot gives the storage index of the
// post-stream f_bar_i of node n in the layout p.aa_parity (double-buffered
// paths keep layout 0, the natural one).
template <int D, typename T>
__device__ __forceinline__ long long aa_slot(const Params<T>& p, int i, long long n)
{
    if (p.aa_parity == 0) return i * p.NS + n;
    const int dim[3] = {p.nx, p.ny, p.nz};
    int g[3];
    long long r = n;
    g[0] = (int)(r % p.nx);
    r /= p.nx;
    g[1] = (int)(r % p.ny);
    g[2] = (int)(r / p.ny);
    for (int a = 0; a < D; ++a) {
        g[a] -= Lattice<D>::c(i, a);
        if (g[a] < 0 || g[a] >= dim[a]) {
            if (p.wall[a]) return i * p.NS + n;  // arrived by reflection at a non-periodic face
            g[a] = g[a] < 0 ? g[a] + dim[a] : g[a] - dim[a];
        }
    }
    return (long long)(Lattice<D>::Q - 1 - i) * p.NS + g[0] + (long long)p.nx * (g[1] + (long long)p.ny * g[2]);
}

// ---------------------------------------------------------------- storage codec
// Stored value: deviation g_i = f_bar_i - eps w_i rho0; FP16/BF16 store g_i / w_i.
template <typename S>
struct Codec;

template <>
struct Codec<double> {
    using T = double;
    static constexpr int bytes = 8;
    __device__ static double load(const double* p, double, double) { return *p; }
    __device__ static void store(double* p, double g, double, double) { *p = g; }
};
template <>
struct Codec<float> {
    using T = float;
    static constexpr int bytes = 4;
    __device__ static float load(const float* p, float, float) { return *p; }
    __device__ static void store(float* p, float g, float, float) { *p = g; }
};
template <>
struct Codec<__half> {
    using T = float;
    static constexpr int bytes = 2;
    __device__ static float load(const __half* p, float w, float) { return __half2float(*p) * w; }
    __device__ static void store(__half* p, float g, float, float inv_w) { *p = __float2half_rn(g * inv_w); }
};
template <>
struct Codec<__nv_bfloat16> {
    using T = float;
    static constexpr int bytes = 2;
    __device__ static float load(const __nv_bfloat16* p, float w, float) { return __bfloat162float(*p) * w; }
    __device__ static void store(__nv_bfloat16* p, float g, float, float inv_w) { *p = __float2bfloat16_rn(g * inv_w); }
};

// ---------------------------------------------------------------- grid helpers
struct Coord {
    int x[3];
};

__device__ __forceinline__ Coord coord_of(long long n, int nx, int ny)
{
    Coord c;
    c.x[0] = (int)(n % nx);
    long long r = n / nx;
    c.x[1] = (int)(r % ny);
    c.x[2] = (int)(r / ny);
    return c;
}

__device__ __forceinline__ int wrap(int k, int n) { return k < 0 ? k + n : (k >= n ? k - n : k); }

// index of the node displaced by d (|d| <= 3) along axis a, periodic wrap
template <typename T>
__device__ __forceinline__ long long shifted(const Params<T>& p, const Coord& c, int a, int d)
{
    int x = c.x[0], y = c.x[1], z = c.x[2];
    if (a == 0) x = wrap(x + d, p.nx);
    else if (a == 1) y = wrap(y + d, p.ny);
    else z = wrap(z + d, p.nz);
    return x + (long long)p.nx * (y + (long long)p.ny * z);
}

__device__ __forceinline__ int dim_of(int a, int nx, int ny, int nz) { return a == 0 ? nx : a == 1 ? ny : nz; }

// First derivative (Sec. 3.5): central differences; second-order one-sided
// at the first (k == 0) / last (k == n-1) node of a wall axis.  `get(j)`
// returns the field at offset j along the axis.
template <typename T, typename Get>
__device__ __forceinline__ T fd1w(bool wall, int k, int n, Get get)
{
    if (wall) {
        if (k == 0) return (T(-3) * get(0) + T(4) * get(1) - get(2)) * T(0.5);
        if (k == n - 1) return (T(3) * get(0) - T(4) * get(-1) + get(-2)) * T(0.5);
    }
    return (get(1) - get(-1)) * T(0.5);
}

// Second derivative: three-point; four-point one-sided at wall ends.
template <typename T, typename Get>
__device__ __forceinline__ T fd2w(bool wall, int k, int n, Get get)
{
    if (wall) {
        if (k == 0) return T(2) * get(0) - T(5) * get(1) + T(4) * get(2) - get(3);
        if (k == n - 1) return T(2) * get(0) - T(5) * get(-1) + T(4) * get(-2) - get(-3);
    }
    return get(1) - T(2) * get(0) + get(-1);
}

template <typename T, typename Get>
__device__ __forceinline__ T fd1(const Params<T>& p, const Coord& c, int a, Get get)
{
    return fd1w<T>(p.wall[a] != 0, c.x[a], dim_of(a, p.nx, p.ny, p.nz), get);
}

template <typename T, typename Get>
__device__ __forceinline__ T fd2(const Params<T>& p, const Coord& c, int a, Get get)
{
    return fd2w<T>(p.wall[a] != 0, c.x[a], dim_of(a, p.nx, p.ny, p.nz), get);
}

// mu_D and mu_F of Eqs. (mu_D_Ergun_perm), (mu_F_Ergun_perm), (F_eps_Ergun)
template <typename T>
__device__ __forceinline__ void drag_coefficients(const Params<T>& p, T eps, T kappa, T& muD, T& muF)
{
    if (isinf(kappa)) {
        muD = T(0);
        muF = T(0);
        return;
    }
    T F = p.ergun ? T(1.75) / sqrt(T(150) * eps * eps * eps) : p.forch;
    muD = eps * p.nu_f / kappa;
    muF = eps * F / sqrt(kappa);
}

// Eq. (v_(1)): v1 = 2 v0 / (c1 + sqrt(c1^2 + 4 c2 |v0|)), c1 = 1 + mu_D/2, c2 = mu_F/2
template <typename T>
__device__ __forceinline__ T drag_solve_factor(T muD, T muF, T v0norm)
{
    T c1 = T(1) + T(0.5) * muD;
    T c2 = T(0.5) * muF;
    return T(2) / (c1 + sqrt(c1 * c1 + T(4) * c2 * v0norm));
}

// asynchronous global -> shared copy of BYTES (4, 8 or 16) bytes
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
// wait until at most N of this thread's committed copy groups are pending
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// brings the 128-byte line holding p into L2 (no register, no wait)
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p)); }

// ---------------------------------------------------------------- bulk copies
// One-phase mbarriers in shared memory that count the bytes of bulk
// (untiled TMA) global -> shared copies.  Addresses and sizes of a bulk copy
// are multiples of 16 bytes; the callers check this on the host.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned arrivals)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(arrivals) : "memory");
}
// makes initialised barriers visible to the copy engine; a __syncthreads()
// must follow before other threads use them
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// one arrival that also announces `bytes` more bytes of copies to come
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* smem, const void* gmem, unsigned bytes, unsigned long long* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(smem)),
                 "l"(gmem), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// Tiled (tensor) TMA loads: the box at the given element coordinates (x
// first) lands in shared memory as a dense array, x fastest; elements outside
// the tensor read as zero.  The map is a __grid_constant__ kernel parameter.
__device__ __forceinline__ void tma_load_3d(void* smem, const void* map, int c0, int c1, int c2,
                                            unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_u32(smem)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* smem, const void* map, int c0, int c1, int c2, int c3,
                                            unsigned long long* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(smem_u32(smem)),
        "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}
// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Every wait of the library's kernels gives up after a bounded time and
// reports it (ERR_WAIT_TIMEOUT); no wait is unbounded.
constexpr unsigned long long kWaitBudgetNs = 1000000000ull;  // 1 s

// Waits for phase `parity` of the barrier to complete; gives up after
// budget_ns nanoseconds of the global timer and returns false.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity,
                                          unsigned long long budget_ns = kWaitBudgetNs)
{
    const unsigned a = smem_u32(bar);
    unsigned long long t0 = 0;
    for (unsigned k = 0;; ++k) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if ((k & 15) == 0) {
            const unsigned long long t = globaltimer_ns();
            if (k == 0) t0 = t;
            else if (t - t0 > budget_ns) return false;
        }
    }
}

// Finite differences by boundary code: 0 central, 1 first node of a
// non-periodic axis (forward one-sided), 2 last node (backward one-sided).
template <typename Get>
__device__ __forceinline__ float fd1c(int code, Get get)
{
    if (code == 1) return (-3.f * get(0) + 4.f * get(1) - get(2)) * 0.5f;
    if (code == 2) return (3.f * get(0) - 4.f * get(-1) + get(-2)) * 0.5f;
    return (get(1) - get(-1)) * 0.5f;
}
template <typename Get>
__device__ __forceinline__ float fd2c(int code, Get get)
{
    if (code == 1) return 2.f * get(0) - 5.f * get(1) + 4.f * get(2) - get(3);
    if (code == 2) return 2.f * get(0) - 5.f * get(-1) + 4.f * get(-2) - get(-3);
    return get(1) - 2.f * get(0) + get(-1);
}

__device__ __forceinline__ int axis_code(bool nonper, int g, int n)
{
    return (nonper && g == 0) ? 1 : (nonper && g == n - 1) ? 2 : 0;
}

// Deviation of the product-form populations, split per axis (see ProductDev):
// for each (y, z) digit pair the partial products YZ = Psi_y Psi_z and
// dYZ = dPsi_y Psi_z + Psi0_y dPsi_z are formed once, then for each x digit
// prod Psi - w_i = dPsi_x YZ + Psi0_x dYZ.
struct AxisFactors {
    float d[3][3];  // dPsi[axis][digit]
};

__device__ __forceinline__ void axis_factors(AxisFactors& F, const float* xi, const float* q)
{
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        F.d[a][0] = (q[a] - xi[a]) * 0.5f;
        F.d[a][1] = -q[a];
        F.d[a][2] = (q[a] + xi[a]) * 0.5f;
    }
}

// Deviation of the product-form populations from eps w_i rho0 (Eqs.
// (1d_scaled_eq), (prod_form)):
//   f_i - eps w_i rho0 = eps [ (rho - rho0) prod Psi + rho0 (prod Psi - w_i) ]
// Per axis Psi = Psi0 + dPsi with Psi0 = (1 - RT, RT/2) and, for q = P - RT,
//   dPsi(0) = -q,  dPsi(+-1) = (q +- xi) / 2,
// so every term is small and FP32 keeps its relative precision.  The
// difference of products is expanded by telescoping over the axes.
template <int D, typename T>
struct ProductDev {
    T psi0[3];    // Psi0(c) per digit (c+1)
    T dpsi[3][3]; // dPsi[axis][digit]
    __device__ __forceinline__ void set(const T* xi, const T* q, T RT)
    {
        psi0[0] = RT * T(0.5);
        psi0[1] = T(1) - RT;
        psi0[2] = RT * T(0.5);
        for (int a = 0; a < D; ++a) {
            dpsi[a][0] = (q[a] - xi[a]) * T(0.5);
            dpsi[a][1] = -q[a];
            dpsi[a][2] = (q[a] + xi[a]) * T(0.5);
        }
    }
    // returns prod Psi - w_i for population i, and prod Psi in `full`
    __device__ __forceinline__ T dev(int i, T& full) const
    {
        int dx = i % 3, dy = (i / 3) % 3;
        if (D == 2) {
            T ax = psi0[dx], ay = psi0[dy];
            T px = ax + dpsi[0][dx], py = ay + dpsi[1][dy];
            full = px * py;
            return dpsi[0][dx] * py + ax * dpsi[1][dy];
        } else {
            int dz = i / 9;
            T ax = psi0[dx], ay = psi0[dy], az = psi0[dz];
            T px = ax + dpsi[0][dx], py = ay + dpsi[1][dy], pz = az + dpsi[2][dz];
            full = px * py * pz;
            return dpsi[0][dx] * (py * pz) + ax * (dpsi[1][dy] * pz + ay * dpsi[2][dz]);
        }
    }
};

}  // namespace lbm
