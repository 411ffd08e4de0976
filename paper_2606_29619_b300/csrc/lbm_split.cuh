// Split D3Q27 step: three streaming kernels per time step, one node (or one
// pair of x-adjacent nodes) per thread, with the intermediate fields of the
// step in device scratch arrays.
//
//   K1 k_split_moments   populations -> rho, m = rho v1 / eps       (Eqs. (v_(0)), (v_(1)))
//   K2 k_split_velocity  rho, m on the 1-ring -> v, a               (Eqs. (porosity_correction_expanded),
//                                                                     (v_final), (accel))
//   K3 k_split_collide   populations, rho and v on the 1-ring -> collide, push-stream
//                                                                    (Eqs. (ex_corr), (eta_corr), (prod_form),
//                                                                     the collision)
//
// The non-local parts of the step (Delta_nu needs m on the 1-ring of a node,
// Phi_ext / Phi_eta need rho and v on the 1-ring) are read back from the
// scratch arrays, whose halo rows sit in L2 when a neighbouring block wants
// them.  Compared with the z-marching fused kernel this moves 16 + 24 bytes
// per node through HBM twice more and reads the populations twice, but every
// kernel is a plain stream with no barriers between planes, so the warps of
// many blocks keep loads in flight instead of waiting at each plane of a
// pipeline.
//
// Arithmetic is the fused kernel's: same moment summation order, the same
// finite-difference codes at non-periodic axes (Sec. 3.5), the same
// collision in deviations and the same rebase of pushed populations.
#pragma once

#include <cuda.h>  // CUtensorMap; the encoder is looked up in the driver at run time

#include <type_traits>

#include "lbm_common.cuh"
#include "lbm_sweep.cuh"

namespace lbm {

constexpr int kSplitBX = 32, kSplitBY = 4;  // a warp is one x row of 32 nodes
constexpr int kSplitThreads = kSplitBX * kSplitBY;
// Tile heights (rows of node pairs per block) of the all-periodic pair
// kernels that the autotuner chooses from; the other split kernels keep
// kSplitBY.  The collide kernels keep about 100 registers a thread for
// every height (minimum resident blocks 20 / BY).
constexpr int kSplitMaxThreads = kSplitBX * 8;
__host__ __device__ constexpr int collide_min_blocks(int by) { return by >= 8 ? 2 : 20 / by; }
inline bool tile_height_ok(int by) { return by == 2 || by == 4 || by == 8; }

// Padded porosity for the collide kernel's tiled copies: (nx + 2 kPadX) x
// (ny + 2) x (nz + 2) values, grid node (x, y, z) at (x + kPadX, y + 1, z + 1).
// The margins hold the periodic images, or 1 past a non-periodic face (the
// value the kernels give porosity outside the grid), so that one box of the
// padded array is a block's whole neighbourhood, wrap and walls included.
constexpr int kPadX = 4;  // 16 bytes: the box's x coordinate stays 16-byte aligned

static __global__ void k_pad_eps(Params<float> p, const float* __restrict__ eps, float* __restrict__ pad)
{
    const long long X = p.nx + 2 * kPadX, Y = p.ny + 2, Z = p.nz + 2, M = X * Y * Z;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < M; k += (long long)gridDim.x * blockDim.x) {
        const int xp = (int)(k % X), yp = (int)((k / X) % Y), zp = (int)(k / (X * Y));
        int g[3] = {xp - kPadX, yp - 1, zp - 1};
        const int nn[3] = {p.nx, p.ny, p.nz};
        bool in = true;
        for (int a = 0; a < 3; ++a) {
            if (g[a] >= 0 && g[a] < nn[a]) continue;
            if (p.wall[a]) in = false;
            g[a] = g[a] < 0 ? g[a] + nn[a] : g[a] - nn[a];
        }
        pad[k] = in ? eps[g[0] + (long long)p.nx * (g[1] + (long long)p.ny * g[2])] : 1.f;
    }
}

// Tensor maps of the collide kernel: the two population buffers (x, y, z,
// population; box 64 x 4 x 1 x 9) and the padded porosity (box 72 x 6 x 3).
struct SplitTma {
    CUtensorMap f[2];
    CUtensorMap eps;
    const void* fbase[2] = {nullptr, nullptr};
    int by = kSplitBY;  // tile height the maps were built for
    bool ok = false;
};

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn tensor_map_encoder()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
    }
    return fn;
}

// Builds the maps for tiles of `by` rows; false (and the cp.async path) when
// nx is not a multiple of 8 (rows of 16-byte multiples), an address is not
// 16-byte aligned or the driver has no encoder.
template <typename S>
bool split_tma_setup(SplitTma& t, const Params<float>& p, void* f0, void* f1, float* eps_pad, int by = kSplitBY)
{
    t.ok = false;
    const EncodeTiledFn enc = tensor_map_encoder();
    if (!enc || p.nx % 8 != 0 || !eps_pad) return false;
    if (((uintptr_t)f0 | (uintptr_t)f1 | (uintptr_t)eps_pad) % 16 != 0) return false;
    const cuuint64_t sb = sizeof(S);
    const CUtensorMapDataType dt = sizeof(S) == 4                          ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : std::is_same<S, __half>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                                    : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const cuuint64_t nx = p.nx, ny = p.ny, nz = p.nz;
    const cuuint64_t fdim[4] = {nx, ny, nz, 27};
    const cuuint64_t fstride[3] = {nx * sb, nx * ny * sb, (cuuint64_t)p.NS * sb};
    const cuuint32_t fbox[4] = {2 * kSplitBX, (cuuint32_t)by, 1, 9};
    const cuuint32_t one[4] = {1, 1, 1, 1};
    void* fb[2] = {f0, f1};
    for (int b = 0; b < 2; ++b)
        if (enc(&t.f[b], dt, 4, fb[b], fdim, fstride, fbox, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    const cuuint64_t X = nx + 2 * kPadX, Y = ny + 2, Z = nz + 2;
    const cuuint64_t edim[3] = {X, Y, Z};
    const cuuint64_t estride[2] = {X * 4, X * Y * 4};
    const cuuint32_t ebox[3] = {2 * kSplitBX + 2 * kPadX, (cuuint32_t)by + 2, 3};
    if (enc(&t.eps, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, eps_pad, edim, estride, ebox, one,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    t.fbase[0] = f0;
    t.fbase[1] = f1;
    t.by = by;
    t.ok = true;
    return true;
}

// This thread's node, from a (x tiles, y tiles, z) grid of (32, 4) blocks.
// Indices are 32-bit: the split path is planned only for N < 2^31.
struct SplitGeo {
    int x, y, z, n, nx, ny, nz, nxy;
    __device__ __forceinline__ bool init(const Params<float>& p)
    {
        nx = p.nx;
        ny = p.ny;
        nz = p.nz;
        nxy = nx * ny;
        x = blockIdx.x * kSplitBX + threadIdx.x;
        y = blockIdx.y * kSplitBY + threadIdx.y;
        z = blockIdx.z;
        n = x + nx * y + nxy * z;
        return x < nx && y < ny;
    }
    // the node (x_, y_, z_) itself
    __device__ __forceinline__ void at(const Params<float>& p, int x_, int y_, int z_)
    {
        nx = p.nx;
        ny = p.ny;
        nz = p.nz;
        nxy = nx * ny;
        x = x_;
        y = y_;
        z = z_;
        n = x + nx * y + nxy * z;
    }
    // offset of the node displaced by d (|d| <= 3) along an axis, periodic wrap
    __device__ __forceinline__ int ox(int d) const
    {
        int g = x + d;
        return (g < 0 ? g + nx : g >= nx ? g - nx : g) - x;
    }
    __device__ __forceinline__ int oy(int d) const
    {
        int g = y + d;
        return nx * ((g < 0 ? g + ny : g >= ny ? g - ny : g) - y);
    }
    __device__ __forceinline__ int oz(int d) const
    {
        int g = z + d;
        return nxy * ((g < 0 ? g + nz : g >= nz ? g - nz : g) - z);
    }
};

// The argument of Phi_ext along one axis, Eq. (ex_corr): q = rho v (1 - 3RT) - rho v^3 / eps^2
__device__ __forceinline__ float qflux(const Params<float>& p, float rho, float v, float e)
{
    const float rho_ie2 = rho / (e * e);
    return rho * v * p.one_m_3RT - rho_ie2 * v * v * v;
}

// Shared-memory copy of NF fields over the block's neighbourhood: planes
// z-1..z+1, rows y0-1..y0+4, columns x0-1..x0+32 (halo 1 around the 32 x 4
// block).  One warp per (z, y) row; lanes 0 and 1 also take its last two
// columns.  Wrapped positions take the periodic image; positions outside a
// non-periodic axis get `fill`, and columns or rows past a ragged grid end
// are left unset: no thread of the block reads either.
constexpr int kHoodX = kSplitBX + 2, kHoodY = kSplitBY + 2;
template <bool WALL, int NF>
__device__ __forceinline__ void stage_hood(const Params<float>& p, const SplitGeo& G, const float* __restrict__ src,
                                           long long stride, float (*dst)[3][kHoodY][kHoodX], float fill)
{
    const int x0 = blockIdx.x * kSplitBX - 1;
    for (int row = threadIdx.y; row < 3 * kHoodY; row += kSplitBY) {
        const int dz = row / kHoodY, dy = row - dz * kHoodY;
        int gy = blockIdx.y * kSplitBY - 1 + dy, gz = blockIdx.z - 1 + dz;
        const bool in_yz = !WALL || ((!p.wall[1] || (gy >= 0 && gy < G.ny)) && (!p.wall[2] || (gz >= 0 && gz < G.nz)));
        gy = gy < 0 ? gy + G.ny : gy >= G.ny ? gy - G.ny : gy;
        gz = gz < 0 ? gz + G.nz : gz >= G.nz ? gz - G.nz : gz;
        if (gy >= G.ny) continue;  // past a ragged y end
        const float* r = src + G.nx * gy + G.nxy * gz;
        for (int dx = threadIdx.x; dx < kHoodX; dx += kSplitBX) {
            int gx = x0 + dx;
            if (gx > G.nx) continue;  // past a ragged x end
            const bool in = in_yz && (!WALL || !p.wall[0] || (gx >= 0 && gx < G.nx));
            gx = gx < 0 ? gx + G.nx : gx >= G.nx ? gx - G.nx : gx;
#pragma unroll
            for (int f = 0; f < NF; ++f) dst[f][dz][dy][dx] = in ? __ldg(r + f * stride + gx) : fill;
        }
    }
}

// K1: moments and the drag-corrected velocity v1, stored as rho and m.
template <typename S, bool WALL>
__global__ void __launch_bounds__(kSplitThreads) k_split_moments(Params<float> p, const float* __restrict__ eps,
                                                                 const float* __restrict__ kap,
                                                                 const S* __restrict__ f, float* __restrict__ rho_out,
                                                                 float* __restrict__ m_out, unsigned* __restrict__ err)
{
    SplitGeo G;
    if (!G.init(p)) return;
    const int n = G.n;
    const long long NS = p.NS, N = p.N;
    float g[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) g[i] = Codec<S>::load(f + i * NS + n, p.w[i], p.inv_w[i]);
    float r[9], rx[9];
#pragma unroll
    for (int yz = 0; yz < 9; ++yz) {
        r[yz] = g[3 * yz] + g[3 * yz + 1] + g[3 * yz + 2];
        rx[yz] = g[3 * yz + 2] - g[3 * yz];
    }
    float dm = 0.f, P1x = 0.f;
#pragma unroll
    for (int yz = 0; yz < 9; ++yz) {
        dm += r[yz];
        P1x += rx[yz];
    }
    const float P1y = (r[2] - r[0]) + (r[5] - r[3]) + (r[8] - r[6]);
    const float P1z = (r[6] - r[0]) + (r[7] - r[1]) + (r[8] - r[2]);
    const int xc = WALL ? axis_code(p.wall[0], G.x, G.nx) : 0;
    const int yc = WALL ? axis_code(p.wall[1], G.y, G.ny) : 0;
    const int zc = WALL ? axis_code(p.wall[2], G.z, G.nz) : 0;
    const float e = __ldg(eps + n);
    const float gex = fd1c(xc, [&](int j) { return __ldg(eps + n + G.ox(j)); });
    const float gey = fd1c(yc, [&](int j) { return __ldg(eps + n + G.oy(j)); });
    const float gez = fd1c(zc, [&](int j) { return __ldg(eps + n + G.oz(j)); });
    const float rho = p.rho0 + dm / e;
    const float inv_rho = 1.f / rho;
    const float RT = p.RT;
    const float v0x = P1x * inv_rho + 0.5f * (e * p.b[0] + RT * gex);
    const float v0y = P1y * inv_rho + 0.5f * (e * p.b[1] + RT * gey);
    const float v0z = P1z * inv_rho + 0.5f * (e * p.b[2] + RT * gez);
    const float nv = sqrtf(v0x * v0x + v0y * v0y + v0z * v0z);
    float muD, muF;
    drag_coefficients<float>(p, e, __ldg(kap + n), muD, muF);
    const float fac = drag_solve_factor<float>(muD, muF, nv);
    const float s = rho * fac / e;
    rho_out[n] = rho;
    m_out[n] = v0x * s;
    m_out[N + n] = v0y * s;
    m_out[2 * N + n] = v0z * s;
    if (!(rho > 0.f) || !isfinite(rho) || !(nv * fac <= 0.5f * e)) atomicOr(err, ERR_DIVERGED);
}

// K2 of one node: Delta_nu(m), the final velocity v and the acceleration a.
template <bool WALL>
__device__ __forceinline__ void split_velocity_node(const Params<float>& p, const SplitGeo& G,
                                                    const float* __restrict__ eps, const float* __restrict__ kap,
                                                    const float* __restrict__ rho_in, const float* __restrict__ m_in,
                                                    float* __restrict__ v_out, float* __restrict__ a_out)
{
    const int n = G.n;
    const long long N = p.N;
    const int xc = WALL ? axis_code(p.wall[0], G.x, G.nx) : 0;
    const int yc = WALL ? axis_code(p.wall[1], G.y, G.ny) : 0;
    const int zc = WALL ? axis_code(p.wall[2], G.z, G.nz) : 0;
    auto E = [&](int dx, int dy, int dz) { return __ldg(eps + n + G.ox(dx) + G.oy(dy) + G.oz(dz)); };
    const float rho = __ldg(rho_in + n);
    const float m[3] = {__ldg(m_in + n), __ldg(m_in + N + n), __ldg(m_in + 2 * N + n)};
    const float e = E(0, 0, 0);
    const float ge[3] = {fd1c(xc, [&](int j) { return E(j, 0, 0); }), fd1c(yc, [&](int j) { return E(0, j, 0); }),
                         fd1c(zc, [&](int j) { return E(0, 0, j); })};
    float dnu[3] = {0.f, 0.f, 0.f};
    if (p.corr & 1) {
        // Hessian of eps: diagonal by the second difference, off-diagonal by
        // differencing the first derivative
        float H[3][3];
        H[0][0] = fd2c(xc, [&](int j) { return E(j, 0, 0); });
        H[1][1] = fd2c(yc, [&](int j) { return E(0, j, 0); });
        H[2][2] = fd2c(zc, [&](int j) { return E(0, 0, j); });
        H[0][1] = H[1][0] = fd1c(xc, [&](int j) { return fd1c(yc, [&](int k) { return E(j, k, 0); }); });
        H[0][2] = H[2][0] = fd1c(xc, [&](int j) { return fd1c(zc, [&](int k) { return E(j, 0, k); }); });
        H[1][2] = H[2][1] = fd1c(yc, [&](int j) { return fd1c(zc, [&](int k) { return E(0, j, k); }); });
        float dmm[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float* mc = m_in + c * N + n;
            dmm[c][0] = fd1c(xc, [&](int j) { return __ldg(mc + G.ox(j)); });
            dmm[c][1] = fd1c(yc, [&](int j) { return __ldg(mc + G.oy(j)); });
            dmm[c][2] = fd1c(zc, [&](int j) { return __ldg(mc + G.oz(j)); });
        }
        const float trH = H[0][0] + H[1][1] + H[2][2];
        const float divm = dmm[0][0] + dmm[1][1] + dmm[2][2];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float r = trH * m[a] + divm * ge[a];
#pragma unroll
            for (int b = 0; b < 3; ++b) r += H[a][b] * m[b] + dmm[a][b] * ge[b];
            dnu[a] = p.nu_eff * r;
        }
    }
    const float inv_rho = 1.f / rho;
    float vv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) vv[a] = m[a] * e * inv_rho + dnu[a] * (0.5f * inv_rho);
    const float nv = sqrtf(vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2]);
    float muD, muF;
    drag_coefficients<float>(p, e, __ldg(kap + n), muD, muF);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        v_out[a * N + n] = vv[a];
        a_out[a * N + n] = e * p.b[a] - muD * vv[a] - muF * nv * vv[a] + p.RT * ge[a] + dnu[a] * inv_rho;
    }
}

// K2: one node per thread (odd nx)
template <bool WALL>
__global__ void __launch_bounds__(kSplitThreads) k_split_velocity(Params<float> p, const float* __restrict__ eps,
                                                                  const float* __restrict__ kap,
                                                                  const float* __restrict__ rho_in,
                                                                  const float* __restrict__ m_in,
                                                                  float* __restrict__ v_out, float* __restrict__ a_out)
{
    SplitGeo G;
    if (!G.init(p)) return;
    split_velocity_node<WALL>(p, G, eps, kap, rho_in, m_in, v_out, a_out);
}

// Appendix F on the split path: one Picard iteration of the implicit
// velocity equation  c1 v + c2 |v| v = v(0) + Delta_nu(rho v / eps) / (2 rho)
// from the iterate vin (3N) into vout (3N), under-relaxed by picard_omega.
// v(0) = c1 v1 + c2 |v1| v1 is recovered from m = rho v1 / eps (Eq. (v_(1))),
// the drag coefficients come from eps and kappa as in K1 / K2, and on the last
// iteration the acceleration of Eq. (accel) takes this iteration's Delta_nu
// (the arithmetic of the sweep path's k_picard).
template <bool WALL>
__global__ void __launch_bounds__(kSplitThreads) k_split_picard(Params<float> p, const float* __restrict__ eps,
                                                                const float* __restrict__ kap,
                                                                const float* __restrict__ rho_in,
                                                                const float* __restrict__ m_in,
                                                                const float* __restrict__ vin, float* __restrict__ vout,
                                                                float* __restrict__ a_out, int last)
{
    SplitGeo G;
    if (!G.init(p)) return;
    const int n = G.n;
    const long long N = p.N;
    const int xc = WALL ? axis_code(p.wall[0], G.x, G.nx) : 0;
    const int yc = WALL ? axis_code(p.wall[1], G.y, G.ny) : 0;
    const int zc = WALL ? axis_code(p.wall[2], G.z, G.nz) : 0;
    auto E = [&](int dx, int dy, int dz) { return __ldg(eps + n + G.ox(dx) + G.oy(dy) + G.oz(dz)); };
    // the iterate's momentum field rho v / eps at an offset node
    auto M = [&](int c, int o) { return __ldg(rho_in + n + o) * __ldg(vin + c * N + n + o) / __ldg(eps + n + o); };
    const float rho = __ldg(rho_in + n);
    const float e = E(0, 0, 0);
    const float ge[3] = {fd1c(xc, [&](int j) { return E(j, 0, 0); }), fd1c(yc, [&](int j) { return E(0, j, 0); }),
                         fd1c(zc, [&](int j) { return E(0, 0, j); })};
    float H[3][3];
    H[0][0] = fd2c(xc, [&](int j) { return E(j, 0, 0); });
    H[1][1] = fd2c(yc, [&](int j) { return E(0, j, 0); });
    H[2][2] = fd2c(zc, [&](int j) { return E(0, 0, j); });
    H[0][1] = H[1][0] = fd1c(xc, [&](int j) { return fd1c(yc, [&](int k) { return E(j, k, 0); }); });
    H[0][2] = H[2][0] = fd1c(xc, [&](int j) { return fd1c(zc, [&](int k) { return E(j, 0, k); }); });
    H[1][2] = H[2][1] = fd1c(yc, [&](int j) { return fd1c(zc, [&](int k) { return E(0, j, k); }); });
    float m[3], dmm[3][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        m[c] = M(c, 0);
        dmm[c][0] = fd1c(xc, [&](int j) { return M(c, G.ox(j)); });
        dmm[c][1] = fd1c(yc, [&](int j) { return M(c, G.oy(j)); });
        dmm[c][2] = fd1c(zc, [&](int j) { return M(c, G.oz(j)); });
    }
    const float trH = H[0][0] + H[1][1] + H[2][2];
    const float divm = dmm[0][0] + dmm[1][1] + dmm[2][2];
    float dnu[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float r = trH * m[a] + divm * ge[a];
#pragma unroll
        for (int b = 0; b < 3; ++b) r += H[a][b] * m[b] + dmm[a][b] * ge[b];
        dnu[a] = p.nu_eff * r;
    }
    float muD, muF;
    drag_coefficients<float>(p, e, __ldg(kap + n), muD, muF);
    float v1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) v1[a] = __ldg(m_in + a * N + n) * e / rho;
    const float nv1 = sqrtf(v1[0] * v1[0] + v1[1] * v1[1] + v1[2] * v1[2]);
    const float c1 = 1.f + 0.5f * muD, c2 = 0.5f * muF;
    float sv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) sv[a] = (c1 * v1[a] + c2 * nv1 * v1[a]) + dnu[a] / (2.f * rho);
    const float ns = sqrtf(sv[0] * sv[0] + sv[1] * sv[1] + sv[2] * sv[2]);
    const float fac = drag_solve_factor<float>(muD, muF, ns);
    const float w = p.picard_omega;
    float v[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] = (1.f - w) * __ldg(vin + a * N + n) + w * (sv[a] * fac);
    const float nv = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        vout[a * N + n] = v[a];
        if (last) a_out[a * N + n] = e * p.b[a] - muD * v[a] - muF * nv * v[a] + p.RT * ge[a] + dnu[a] / rho;
    }
}

// The Picard iterations after K2 (picard_iters of them, ping-pong between
// F.v and the spare F.v1); returns the array that holds the final velocity.
inline float* split_picard(const Params<float>& p, const Fields<float>& F, cudaStream_t st)
{
    const int K = p.picard_iters;
    const bool wall = p.wall[0] || p.wall[1] || p.wall[2];
    const dim3 blk(kSplitBX, kSplitBY), grd((p.nx + kSplitBX - 1) / kSplitBX, (p.ny + kSplitBY - 1) / kSplitBY, p.nz);
    float* cur = F.v;
    for (int k = 0; k < K; ++k) {
        float* nxt = cur == F.v ? F.v1 : F.v;
        if (wall)
            k_split_picard<true><<<grd, blk, 0, st>>>(p, F.eps, F.kap, F.rho, F.m, cur, nxt, F.a, k == K - 1);
        else
            k_split_picard<false><<<grd, blk, 0, st>>>(p, F.eps, F.kap, F.rho, F.m, cur, nxt, F.a, k == K - 1);
        cur = nxt;
    }
    return cur;
}

// K3: Phi_ext and Phi_eta from q and v on the 1-ring, the two product-form
// equilibria, the collision and the push to the neighbours (reflected at a
// non-periodic face, rebased on the destination's eps).
// The porosity of the block's neighbourhood is staged in shared memory once,
// so that the 27 rebases read it there.  I: index type of the
// population arrays (int when 27 planes fit 2^31 elements).
template <typename S, bool WALL, typename I>
__global__ void __launch_bounds__(kSplitThreads) k_split_collide(Params<float> p, const float* __restrict__ eps,
                                                                 const float* __restrict__ rho_in,
                                                                 const float* __restrict__ v_in,
                                                                 const float* __restrict__ a_in,
                                                                 const S* __restrict__ fin, S* __restrict__ fout)
{
    __shared__ float se[1][3][kHoodY][kHoodX];
    SplitGeo G;
    const bool on = G.init(p);
    stage_hood<WALL, 1>(p, G, eps, 0, se, 1.f);
    __syncthreads();
    if (!on) return;
    const int n = G.n;
    const I N = (I)p.N, NS = (I)p.NS;
    const int xc = WALL ? axis_code(p.wall[0], G.x, G.nx) : 0;
    const int yc = WALL ? axis_code(p.wall[1], G.y, G.ny) : 0;
    const int zc = WALL ? axis_code(p.wall[2], G.z, G.nz) : 0;
    const int tx = threadIdx.x + 1, ty = threadIdx.y + 1;
    const float RT = p.RT;
    const float rho = __ldg(rho_in + n);
    const float v[3] = {__ldg(v_in + n), __ldg(v_in + N + n), __ldg(v_in + 2 * N + n)};
    const float acc[3] = {__ldg(a_in + n), __ldg(a_in + N + n), __ldg(a_in + 2 * N + n)};
    const float e = se[0][1][ty][tx];
    // destinations: per axis the wrapped offset; bit (axis*3 + digit) marks a
    // population leaving through a non-periodic face: it is reflected (a wall;
    // at an inlet / outlet plane or a moving wall the plane rebuild overwrites
    // it, after the bounce-back density has read it)
    int off[3][3];
    unsigned bbm = 0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        off[0][d] = G.ox(d - 1);
        off[1][d] = G.oy(d - 1);
        off[2][d] = G.oz(d - 1);
        if (WALL) {
            const int gg[3] = {G.x + d - 1, G.y + d - 1, G.z + d - 1};
            const int nn[3] = {G.nx, G.ny, G.nz};
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if (p.wall[a] && (gg[a] < 0 || gg[a] >= nn[a])) bbm |= 1u << (3 * a + d);
        }
    }
    // neighbour offsets for the finite differences: the destination offsets
    // where the stencil stays within the 1-ring
    auto OX = [&](int j) { return (j >= -1 && j <= 1) ? off[0][j + 1] : G.ox(j); };
    auto OY = [&](int j) { return (j >= -1 && j <= 1) ? off[1][j + 1] : G.oy(j); };
    auto OZ = [&](int j) { return (j >= -1 && j <= 1) ? off[2][j + 1] : G.oz(j); };
    float phx[3] = {0.f, 0.f, 0.f}, divv = 0.f;
    if (p.corr & 2) {
        // q of Eq. (ex_corr) at the stencil points, from rho, v and eps there
        auto Q = [&](const float* vc, int o) { return qflux(p, __ldg(rho_in + n + o), __ldg(vc + n + o), __ldg(eps + n + o)); };
        phx[0] = fd1c(xc, [&](int j) { return Q(v_in, OX(j)); });
        phx[1] = fd1c(yc, [&](int j) { return Q(v_in + N, OY(j)); });
        phx[2] = fd1c(zc, [&](int j) { return Q(v_in + 2 * N, OZ(j)); });
    }
    if (p.corr & 4) {
        divv = fd1c(xc, [&](int j) { return __ldg(v_in + n + OX(j)); }) +
               fd1c(yc, [&](int j) { return __ldg(v_in + N + n + OY(j)); }) +
               fd1c(zc, [&](int j) { return __ldg(v_in + 2 * N + n + OZ(j)); });
    }
    const float phe = (p.corr & 4) ? rho * p.eta_coef * divv : 0.f;
    const float inv_e = 1.f / e;
    const float inv_erho = inv_e / rho;
    float xe[3], qe[3], xs[3], qs[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        xe[a] = v[a] * inv_e;
        qe[a] = xe[a] * xe[a];
        xs[a] = (v[a] + acc[a]) * inv_e;
        qs[a] = xs[a] * xs[a] + (phx[a] + phe) * inv_erho;
    }
    AxisFactors Fe, Fs;
    axis_factors(Fe, xe, qe);
    axis_factors(Fs, xs, qs);
    const float psi0[3] = {0.5f * RT, 1.f - RT, 0.5f * RT};
    // collision in deviations with the equilibrium weights folded into the z
    // factors (see fused_segment, stage C)
    const float erho = e * rho;
    const float c_eq = erho * (3.f * p.beta - 1.f), c_st = erho * (1.f - p.beta);
    const float omb = 1.f - 2.f * p.beta, c_w = 2.f * p.beta * e * (rho - p.rho0);
#pragma unroll
    for (int dz = 0; dz < 3; ++dz) {
        const float dZe = c_eq * Fe.d[2][dz], dZs = c_st * Fs.d[2][dz];
        const float Ze = c_eq * psi0[dz] + dZe, Zs = c_st * psi0[dz] + dZs;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            const float YZe = (psi0[dy] + Fe.d[1][dy]) * Ze, dYZe = Fe.d[1][dy] * Ze + psi0[dy] * dZe;
            const float YZs = (psi0[dy] + Fs.d[1][dy]) * Zs, dYZs = Fs.d[1][dy] * Zs + psi0[dy] * dZs;
            const float Bsum = dYZe + dYZs;
            const float Bx[2] = {psi0[0] * Bsum, psi0[1] * Bsum};
            const int row = n + off[1][dy] + off[2][dz];
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const int i = dx + 3 * dy + 9 * dz;
                const float comb = Fe.d[0][dx] * YZe + (Fs.d[0][dx] * YZs + Bx[dx & 1]);
                const float gpc = omb * Codec<S>::load(fin + (i * NS + n), p.w[i], p.inv_w[i]) + comb;
                const unsigned bit = (1u << dx) | (1u << (3 + dy)) | (1u << (6 + dz));
                if (WALL && (bbm & bit)) {
                    Codec<S>::store(fout + ((26 - i) * NS + n), gpc + c_w * p.w[i], p.w[26 - i], p.inv_w[26 - i]);
                } else {
                    const int dst = row + off[0][dx];
                    const float de = e - se[0][dz][ty + dy - 1][tx + dx - 1];
                    Codec<S>::store(fout + (i * NS + dst), gpc + p.w[i] * (c_w + p.rho0 * de), p.w[i], p.inv_w[i]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------- node pairs
// K3 for grids with an even nx: each thread takes two x-adjacent nodes, so
// that a population moves as one 8-byte (FP32) or 4-byte (FP16/BF16) access
// per pair and the arithmetic, identical for the two nodes, runs as packed
// FP32x2 operations (FFMA2 / FADD2 / FMUL2 of sm_100 and later).  The
// results equal the one-node kernel's operation by operation.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f), a); }  // exact a - b

template <typename S>
struct Codec2;
template <>
struct Codec2<float> {
    __device__ static float2 load(const float* p, float) { return *reinterpret_cast<const float2*>(p); }
    __device__ static void store(float* p, float2 g, float) { *reinterpret_cast<float2*>(p) = g; }
};
template <>
struct Codec2<__half> {
    // the stored value g / w_i itself (no scaling)
    __device__ static float2 load_raw(const __half* p) { return __half22float2(*reinterpret_cast<const __half2*>(p)); }
    __device__ static void store_raw(__half* p, float2 g) { *reinterpret_cast<__half2*>(p) = __float22half2_rn(g); }
    __device__ static void store_raw1(__half* p, float g) { *p = __float2half_rn(g); }
    __device__ static float2 load(const __half* p, float w)
    {
        return mul2(__half22float2(*reinterpret_cast<const __half2*>(p)), f2(w));
    }
    __device__ static void store(__half* p, float2 g, float inv_w)
    {
        *reinterpret_cast<__half2*>(p) = __float22half2_rn(mul2(g, f2(inv_w)));
    }
};
template <>
struct Codec2<__nv_bfloat16> {
    // a bfloat16 is the upper half of a binary32: widening is a shift
    __device__ static float2 load_raw(const __nv_bfloat16* p)
    {
        const unsigned u = *reinterpret_cast<const unsigned*>(p);
        return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
    }
    __device__ static void store_raw(__nv_bfloat16* p, float2 g)
    {
        *reinterpret_cast<__nv_bfloat162*>(p) = __float22bfloat162_rn(g);
    }
    __device__ static void store_raw1(__nv_bfloat16* p, float g) { *p = __float2bfloat16_rn(g); }
    __device__ static float2 load(const __nv_bfloat16* p, float w) { return mul2(load_raw(p), f2(w)); }
    __device__ static void store(__nv_bfloat16* p, float2 g, float inv_w)
    {
        *reinterpret_cast<__nv_bfloat162*>(p) = __float22bfloat162_rn(mul2(g, f2(inv_w)));
    }
};

__device__ __forceinline__ float2 ld2(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }

// boundary-coded first difference of a pair of nodes on the y or z axis
template <typename Get>
__device__ __forceinline__ float2 fd1c_pair(int code, Get get)
{
    const float2 r = {fd1c(code, [&](int j) { return get(j).x; }), fd1c(code, [&](int j) { return get(j).y; })};
    return r;
}

// TMA (nx a multiple of 8, tensor maps built for the context): one thread
// loads the block's populations, a z digit (9 populations x 4 rows x 64
// nodes) per tiled copy, and its porosity neighbourhood, one 72 x 6 x 3 box of
// the padded porosity, counted on four mbarriers; otherwise each thread copies
// its own populations with cp.async and the block stages the neighbourhood
// with plain loads.
// shared-memory tile of the collide kernel
template <typename S, bool TMA, int BY>
struct CollideSmem {
    static constexpr int PX = 2 * kSplitBX;     // nodes per block row
    static constexpr int HO = TMA ? kPadX : 2;  // porosity column of node x0 (TMA: the padded grid's margin)
    static constexpr int HX = PX + 2 * HO;      // porosity columns x0-HO .. x0+PX+HO-1 (pairs stay 8-byte aligned)
    static constexpr int HY = BY + 2;           // porosity rows y0-1 .. y0+BY
    __align__(128) float se[3][HY][HX];
    __align__(128) S sg[27][BY][PX];            // the block's populations
    __align__(8) unsigned long long bar[4];     // TMA: populations by z digit, porosity
};

template <typename S, bool WALL, typename I, bool TMA, int BY>
__device__ __forceinline__ void split_collide_tile(const Params<float>& p, const float* __restrict__ eps,
                                                   const float* __restrict__ rho_in, const float* __restrict__ v_in,
                                                   const float* __restrict__ a_in, const S* __restrict__ fin,
                                                   S* __restrict__ fout, unsigned* __restrict__ err,
                                                   const CUtensorMap& tm_f, const CUtensorMap& tm_eps,
                                                   CollideSmem<S, TMA, BY>& sm)
{
    using SM = CollideSmem<S, TMA, BY>;
    constexpr int PX = SM::PX, HO = SM::HO, HX = SM::HX, HY = SM::HY;
    auto& se = sm.se;
    auto& sg = sm.sg;
    auto& bar = sm.bar;
    (void)HX;
    const int nx = p.nx, ny = p.ny, nz = p.nz, nxy = nx * ny;
    const int x0 = blockIdx.x * PX, y0 = blockIdx.y * BY;
    const int x = x0 + 2 * threadIdx.x, y = y0 + threadIdx.y, z = blockIdx.z;
    const bool on = x < nx && y < ny;
    const int n = x + nx * y + nxy * z;
    const I N = (I)p.N, NS = (I)p.NS;
    if constexpr (TMA) {
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            for (int b = 0; b < 4; ++b) mbar_init(&bar[b], 1);
            mbar_fence_init();
            // padded porosity rows y0-1 .. y0+BY of planes z-1 .. z+1, columns x0-4 .. x0+67
            mbar_arrive_tx(&bar[3], (unsigned)sizeof(se));
            tma_load_3d(&se[0][0][0], &tm_eps, x0, y0, z, &bar[3]);
            for (int g = 0; g < 3; ++g) {
                mbar_arrive_tx(&bar[g], 9u * BY * PX * (unsigned)sizeof(S));
                tma_load_4d(&sg[9 * g][0][0], &tm_f, x0, y0, z, 9 * g, &bar[g]);
            }
        }
    } else {
        // the 27 population pairs are copied to shared memory asynchronously,
        // in three groups by z digit, so that their loads are all in flight
        // while the porosity neighbourhood is staged and the first groups can
        // be collided while the last are still arriving.  Each thread reads
        // back only its own copies.
#pragma unroll
        for (int dz = 0; dz < 3; ++dz) {
            if (on) {
#pragma unroll
                for (int i = 9 * dz; i < 9 * dz + 9; ++i)
                    cp_async<2 * sizeof(S)>(&sg[i][threadIdx.y][2 * threadIdx.x], fin + (i * NS + n));
            }
            cp_async_commit();
        }
    }
    auto wrapx = [&](int g) { return g < 0 ? g + nx : g >= nx ? g - nx : g; };
    // x offset of node x + k displaced by d; y and z offsets shared by the pair
    auto OXk = [&](int k, int d) { return wrapx(x + k + d) - (x + k); };
    auto OY = [&](int d) {
        const int g = y + d;
        return nx * ((g < 0 ? g + ny : g >= ny ? g - ny : g) - y);
    };
    auto OZ = [&](int d) {
        const int g = z + d;
        return nxy * ((g < 0 ? g + nz : g >= nz ? g - nz : g) - z);
    };
    const int xc0 = WALL ? axis_code(p.wall[0], x, nx) : 0, xc1 = WALL ? axis_code(p.wall[0], x + 1, nx) : 0;
    const int yc = WALL ? axis_code(p.wall[1], y, ny) : 0;
    const int zc = WALL ? axis_code(p.wall[2], z, nz) : 0;
    const float RT = p.RT;
    // this pair's moments and the neighbour values of the corrections, loaded
    // before the barrier so that they too are in flight during the staging
    float2 rho = f2(1.f), v[3] = {f2(0.f), f2(0.f), f2(0.f)}, acc[3] = {f2(0.f), f2(0.f), f2(0.f)};
    float2 phx[3] = {f2(0.f), f2(0.f), f2(0.f)}, divv = f2(0.f);
    if (on) {
        rho = ld2(rho_in + n);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            v[a] = ld2(v_in + a * N + n);
            acc[a] = ld2(a_in + a * N + n);
        }
        if (p.corr & 2) {
            // q of Eq. (ex_corr) at the stencil points, from rho, v and eps there
            auto Qx = [&](int xo) {
                const int o = OXk(0, xo);
                return qflux(p, __ldg(rho_in + n + o), __ldg(v_in + n + o), __ldg(eps + n + o));
            };
            auto Q2 = [&](const float* vc, int o) {
                const float2 r = ld2(rho_in + n + o), vv = ld2(vc + n + o), ee = ld2(eps + n + o);
                return make_float2(qflux(p, r.x, vv.x, ee.x), qflux(p, r.y, vv.y, ee.y));
            };
            phx[0] = make_float2(fd1c(xc0, [&](int j) { return Qx(j); }), fd1c(xc1, [&](int j) { return Qx(1 + j); }));
            phx[1] = fd1c_pair(yc, [&](int j) { return Q2(v_in + N, OY(j)); });
            phx[2] = fd1c_pair(zc, [&](int j) { return Q2(v_in + 2 * N, OZ(j)); });
        }
        if (p.corr & 4) {
            const float2 dvx = make_float2(fd1c(xc0, [&](int j) { return __ldg(v_in + n + OXk(0, j)); }),
                                           fd1c(xc1, [&](int j) { return __ldg(v_in + n + 1 + OXk(1, j)); }));
            const float2 dvy = fd1c_pair(yc, [&](int j) { return ld2(v_in + N + n + OY(j)); });
            const float2 dvz = fd1c_pair(zc, [&](int j) { return ld2(v_in + 2 * N + n + OZ(j)); });
            divv = add2(add2(dvx, dvy), dvz);
        }
    }
    if constexpr (!TMA) {
        // porosity of the neighbourhood, as column pairs (nx is even, so a
        // pair never straddles the periodic seam)
        for (int row = threadIdx.y; row < 3 * HY; row += BY) {
            const int dz = row / HY, dy = row - dz * HY;
            int gy = y0 - 1 + dy, gz = z - 1 + dz;
            const bool in_yz = !WALL || ((!p.wall[1] || (gy >= 0 && gy < ny)) && (!p.wall[2] || (gz >= 0 && gz < nz)));
            gy = gy < 0 ? gy + ny : gy >= ny ? gy - ny : gy;
            gz = gz < 0 ? gz + nz : gz >= nz ? gz - nz : gz;
            if (gy >= ny) continue;  // past a ragged y end
            const float* r = eps + nx * gy + nxy * gz;
            for (int j = threadIdx.x; j < HX / 2; j += kSplitBX) {
                int gx = x0 - 2 + 2 * j;
                if (gx > nx) continue;  // past a ragged x end
                const bool in = in_yz && (!WALL || !p.wall[0] || (gx >= 0 && gx < nx));
                gx = gx < 0 ? gx + nx : gx >= nx ? gx - nx : gx;
                *reinterpret_cast<float2*>(&se[dz][dy][2 * j]) = in ? ld2(r + gx) : f2(1.f);
            }
        }
    }
    __syncthreads();  // TMA: also publishes the initialised barriers
    if (!on) return;
    // TMA: a wait that runs out flags the error, waits (bounded) for the
    // block's remaining copies and abandons the block
    auto landed = [&](int b) {
        if (mbar_wait(&bar[b], 0u)) return true;
        atomicOr(err, ERR_WAIT_TIMEOUT);
        for (int k = 0; k < 4; ++k) mbar_wait(&bar[k], 0u);
        return false;
    };
    if constexpr (TMA)
        if (!landed(3)) return;
    const int tx = 2 * threadIdx.x + HO, ty = threadIdx.y + 1;  // porosity column of node x
    const float2 e = *reinterpret_cast<const float2*>(&se[1][ty][tx]);
    const float2 phe = (p.corr & 4) ? mul2(mul2(rho, f2(p.eta_coef)), divv) : f2(0.f);
    const float2 inv_e = make_float2(1.f / e.x, 1.f / e.y);
    const float2 inv_erho = make_float2(inv_e.x / rho.x, inv_e.y / rho.y);
    // per axis: dPsi(-1), dPsi(0), dPsi(+1) of the equilibrium (e) and of f* (s)
    float2 Fe[3][3], Fs[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float2 xe = mul2(v[a], inv_e);
        const float2 qe = mul2(xe, xe);
        const float2 xs = mul2(add2(v[a], acc[a]), inv_e);
        const float2 qs = fma2(xs, xs, mul2(add2(phx[a], phe), inv_erho));
        Fe[a][0] = mul2(sub2(qe, xe), f2(0.5f));
        Fe[a][1] = mul2(qe, f2(-1.f));
        Fe[a][2] = mul2(add2(qe, xe), f2(0.5f));
        Fs[a][0] = mul2(sub2(qs, xs), f2(0.5f));
        Fs[a][1] = mul2(qs, f2(-1.f));
        Fs[a][2] = mul2(add2(qs, xs), f2(0.5f));
    }
    const float psi0[3] = {0.5f * RT, 1.f - RT, 0.5f * RT};
    // FP16/BF16 store g_i / w_i.  With every dPsi divided by its Psi0 the
    // collision yields g_pc / w_i directly, w_i = Psi0_x Psi0_y Psi0_z, so the
    // stored value is decoded and encoded without the w_i factors.
    constexpr bool SC = sizeof(S) == 2;
    if constexpr (SC) {
        const float ipsi[3] = {2.f / RT, 1.f / (1.f - RT), 2.f / RT};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                Fe[a][d] = mul2(Fe[a][d], f2(ipsi[d]));
                Fs[a][d] = mul2(Fs[a][d], f2(ipsi[d]));
            }
    }
    const float2 erho = mul2(e, rho);
    const float2 c_eq = mul2(erho, f2(3.f * p.beta - 1.f)), c_st = mul2(erho, f2(1.f - p.beta));
    const float2 omb = f2(1.f - 2.f * p.beta);
    const float2 c_w = mul2(mul2(f2(2.f * p.beta), e), sub2(rho, f2(p.rho0)));
    // A pushed population gains w_i (c_w + rho0 (e - e_dest)), the density
    // term and the rebase onto its destination's porosity.  w_i c_w is folded
    // into the row factors below; rho0 (e - e_dest) is formed from the small
    // difference e - e_dest (exact for nearby porosities), not from rho0 e and
    // rho0 e_dest, whose rounding would swamp the deviation.  A reflected
    // population stays at the node (e_dest = e).
    // bit (axis*3 + digit): the population leaves through a non-periodic face
    // and is reflected; x bits per node of the pair
    unsigned bbm[2] = {0u, 0u};
    if (WALL) {
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int gg[3] = {x + k + d - 1, y + d - 1, z + d - 1};
                const int nn[3] = {nx, ny, nz};
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    if (p.wall[a] && (gg[a] < 0 || gg[a] >= nn[a])) bbm[k] |= 1u << (3 * a + d);
            }
    }
    const int ox[2][2] = {{OXk(0, -1), OXk(0, 1)}, {OXk(1, -1), OXk(1, 1)}};  // [node][dx = 0, 2]
    auto st2 = [&](S* d, float2 g) {
        if constexpr (SC) Codec2<S>::store_raw(d, g);
        else *reinterpret_cast<float2*>(d) = g;
    };
    auto st1 = [&](S* d, float g) {
        if constexpr (SC) Codec2<S>::store_raw1(d, g);
        else *d = g;
    };
#pragma unroll
    for (int dz = 0; dz < 3; ++dz) {
        // this z digit's copies have landed
        if constexpr (TMA) {
            if (!landed(dz)) return;
        } else if (dz == 0) {
            cp_async_wait_group<2>();
        } else if (dz == 1) {
            cp_async_wait_group<1>();
        } else {
            cp_async_wait_group<0>();
        }
        const float2 dZe = mul2(c_eq, Fe[2][dz]), dZs = mul2(c_st, Fs[2][dz]);
        const float2 Ze = SC ? add2(c_eq, dZe) : fma2(c_eq, f2(psi0[dz]), dZe);
        const float2 Zs = SC ? add2(c_st, dZs) : fma2(c_st, f2(psi0[dz]), dZs);
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            const float py = SC ? 1.f : psi0[dy];
            const float2 YZe = mul2(add2(f2(py), Fe[1][dy]), Ze);
            const float2 dYZe = SC ? fma2(Fe[1][dy], Ze, dZe) : fma2(Fe[1][dy], Ze, mul2(f2(psi0[dy]), dZe));
            const float2 YZs = mul2(add2(f2(py), Fs[1][dy]), Zs);
            const float2 dYZs = SC ? fma2(Fs[1][dy], Zs, dZs) : fma2(Fs[1][dy], Zs, mul2(f2(psi0[dy]), dZs));
            // + w_i / Psi0_x c_w
            const float2 Bsum = SC ? add2(add2(dYZe, dYZs), c_w) : fma2(f2(psi0[dy] * psi0[dz]), c_w, add2(dYZe, dYZs));
            const float2 Bx[2] = {SC ? Bsum : mul2(f2(psi0[0]), Bsum), SC ? Bsum : mul2(f2(psi0[1]), Bsum)};
            const int row = n + OY(dy - 1) + OZ(dz - 1);
            const float* er = &se[dz][ty + dy - 1][tx];  // destination porosity, this pair's columns
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const int i = dx + 3 * dy + 9 * dz;
                const float rw = SC ? p.rho0 : p.rho0 * p.w[i];  // coefficient of e - e_dest
                const float2 comb = fma2(Fe[0][dx], YZe, fma2(Fs[0][dx], YZs, Bx[dx & 1]));
                const S* gi = &sg[i][threadIdx.y][2 * threadIdx.x];
                float2 gin;
                if constexpr (SC) gin = Codec2<S>::load_raw(gi);
                else gin = Codec2<S>::load(gi, 1.f);
                const float2 gpc = fma2(omb, gin, comb);  // includes w_i c_w
                const unsigned byz = (1u << (3 + dy)) | (1u << (6 + dz));
                if (dx == 1) {
                    // no x displacement: both nodes go the same way, as a pair
                    if (WALL && (bbm[0] & (byz | 2u)))
                        st2(fout + ((26 - i) * NS + n), gpc);
                    else
                        st2(fout + (i * NS + row), fma2(f2(rw), sub2(e, *reinterpret_cast<const float2*>(er)), gpc));
                } else {
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const float g = k ? gpc.y : gpc.x, ek = k ? e.y : e.x;
                        const unsigned bit = byz | (1u << dx);
                        if (WALL && (bbm[k] & bit))
                            st1(fout + ((26 - i) * NS + n + k), g);
                        else
                            st1(fout + (i * NS + row + k + ox[k][dx >> 1]), fmaf(rw, ek - er[k + dx - 1], g));
                    }
                }
            }
        }
    }
}

// K3.  With walls, a block whose tile has no node on the first or last layer
// of a non-periodic axis runs the all-periodic form: its stencils and pushes
// stay inside the grid, where the two forms take the same arithmetic.
template <typename S, bool WALL, typename I, bool TMA, int BY = kSplitBY>
__global__ void __launch_bounds__(kSplitBX * BY, collide_min_blocks(BY))
    k_split_collide2(Params<float> p, const float* __restrict__ eps, const float* __restrict__ rho_in,
                     const float* __restrict__ v_in, const float* __restrict__ a_in, const S* __restrict__ fin,
                     S* __restrict__ fout, unsigned* __restrict__ err, const __grid_constant__ CUtensorMap tm_f,
                     const __grid_constant__ CUtensorMap tm_eps)
{
    __shared__ CollideSmem<S, TMA, BY> sm;
    if constexpr (WALL) {
        const int x0 = blockIdx.x * 2 * kSplitBX, y0 = blockIdx.y * BY, z = blockIdx.z;
        const bool inside = (!p.wall[0] || (x0 > 0 && x0 + 2 * kSplitBX < p.nx)) &&
                            (!p.wall[1] || (y0 > 0 && y0 + BY < p.ny)) && (!p.wall[2] || (z > 0 && z + 1 < p.nz));
        if (inside) {
            split_collide_tile<S, false, I, TMA, BY>(p, eps, rho_in, v_in, a_in, fin, fout, err, tm_f, tm_eps, sm);
            return;
        }
    }
    split_collide_tile<S, WALL, I, TMA, BY>(p, eps, rho_in, v_in, a_in, fin, fout, err, tm_f, tm_eps, sm);
}

// Pair versions of K1 and K2 for an all-periodic grid with an even nx: two
// x-adjacent nodes per thread, packed FP32x2 arithmetic, and the x
// neighbours of a row taken as one aligned pair plus the two outer scalars.
struct PairGeo {
    int x, y, z, n, nx, ny, nz, nxy;
    int xl, xr;  // offsets of x-1 from x and of x+2 from x+1 (periodic)
    __device__ __forceinline__ bool init(const Params<float>& p) { return init(p, blockIdx.x, blockIdx.y, blockIdx.z); }
    // the block's tile given explicitly (batched launches over many cases)
    __device__ __forceinline__ bool init(const Params<float>& p, int bx, int by, int bz)
    {
        nx = p.nx;
        ny = p.ny;
        nz = p.nz;
        nxy = nx * ny;
        x = 2 * (bx * kSplitBX + threadIdx.x);
        y = by * blockDim.y + threadIdx.y;
        z = bz;
        n = x + nx * y + nxy * z;
        xl = x == 0 ? nx - 1 : -1;
        xr = x + 2 == nx ? 1 - nx : 1;
        return x < nx && y < ny;
    }
    __device__ __forceinline__ int oy(int d) const
    {
        const int g = y + d;
        return nx * ((g < 0 ? g + ny : g >= ny ? g - ny : g) - y);
    }
    __device__ __forceinline__ int oz(int d) const
    {
        const int g = z + d;
        return nxy * ((g < 0 ? g + nz : g >= nz ? g - nz : g) - z);
    }
};

// one row of a field around the pair: values at x-1, x, x+1, x+2
struct Row4 {
    float l, c0, c1, r;
    __device__ __forceinline__ float2 L() const { return make_float2(l, c0); }   // (x-1, x)
    __device__ __forceinline__ float2 C() const { return make_float2(c0, c1); }  // (x, x+1)
    __device__ __forceinline__ float2 R() const { return make_float2(c1, r); }   // (x+1, x+2)
};
__device__ __forceinline__ Row4 row4(const float* __restrict__ b, const PairGeo& G)
{
    const float2 c = ld2(b);
    return {__ldg(b + G.xl), c.x, c.y, __ldg(b + 1 + G.xr)};
}
__device__ __forceinline__ float2 cdiff(float2 a, float2 b) { return mul2(sub2(a, b), f2(0.5f)); }  // (a - b) / 2

template <typename S>
__global__ void __launch_bounds__(kSplitMaxThreads) k_split_moments2(Params<float> p, const float* __restrict__ eps,
                                                                  const float* __restrict__ kap,
                                                                  const S* __restrict__ f, float* __restrict__ rho_out,
                                                                  float* __restrict__ m_out, unsigned* __restrict__ err)
{
    PairGeo G;
    if (!G.init(p)) return;
    const int n = G.n;
    const long long NS = p.NS, N = p.N;
    float2 g[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) g[i] = Codec2<S>::load(f + i * NS + n, p.w[i]);
    float2 r[9], rx[9];
#pragma unroll
    for (int yz = 0; yz < 9; ++yz) {
        r[yz] = add2(add2(g[3 * yz], g[3 * yz + 1]), g[3 * yz + 2]);
        rx[yz] = sub2(g[3 * yz + 2], g[3 * yz]);
    }
    float2 dm = f2(0.f), P1x = f2(0.f);
#pragma unroll
    for (int yz = 0; yz < 9; ++yz) {
        dm = add2(dm, r[yz]);
        P1x = add2(P1x, rx[yz]);
    }
    const float2 P1y = add2(add2(sub2(r[2], r[0]), sub2(r[5], r[3])), sub2(r[8], r[6]));
    const float2 P1z = add2(add2(sub2(r[6], r[0]), sub2(r[7], r[1])), sub2(r[8], r[2]));
    const Row4 E = row4(eps + n, G);
    const float2 e = E.C();
    const float2 gex = cdiff(E.R(), E.L());
    const float2 gey = cdiff(ld2(eps + n + G.oy(1)), ld2(eps + n + G.oy(-1)));
    const float2 gez = cdiff(ld2(eps + n + G.oz(1)), ld2(eps + n + G.oz(-1)));
    const float2 kp = ld2(kap + n);
    const float RT = p.RT;
    float2 rho, inv_rho;
    rho.x = p.rho0 + dm.x / e.x;
    rho.y = p.rho0 + dm.y / e.y;
    inv_rho = make_float2(1.f / rho.x, 1.f / rho.y);
    const float2 v0x = fma2(P1x, inv_rho, mul2(f2(0.5f), fma2(e, f2(p.b[0]), mul2(f2(RT), gex))));
    const float2 v0y = fma2(P1y, inv_rho, mul2(f2(0.5f), fma2(e, f2(p.b[1]), mul2(f2(RT), gey))));
    const float2 v0z = fma2(P1z, inv_rho, mul2(f2(0.5f), fma2(e, f2(p.b[2]), mul2(f2(RT), gez))));
    const float2 n2 = fma2(v0z, v0z, fma2(v0y, v0y, mul2(v0x, v0x)));
    const float2 nv = make_float2(sqrtf(n2.x), sqrtf(n2.y));
    float2 s, fac;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float ek = k ? e.y : e.x, rk = k ? rho.y : rho.x, nk = k ? nv.y : nv.x;
        float muD, muF;
        drag_coefficients<float>(p, ek, k ? kp.y : kp.x, muD, muF);
        const float fk = drag_solve_factor<float>(muD, muF, nk);
        (k ? fac.y : fac.x) = fk;
        (k ? s.y : s.x) = rk * fk / ek;
        bad |= !(rk > 0.f) || !isfinite(rk) || !(nk * fk <= 0.5f * ek);
    }
    *reinterpret_cast<float2*>(rho_out + n) = rho;
    *reinterpret_cast<float2*>(m_out + n) = mul2(v0x, s);
    *reinterpret_cast<float2*>(m_out + N + n) = mul2(v0y, s);
    *reinterpret_cast<float2*>(m_out + 2 * N + n) = mul2(v0z, s);
    if (bad) atomicOr(err, ERR_DIVERGED);
}

// nodes ahead: about one wave of resident blocks (148 SMs x 8 blocks x 256
// nodes = 303K); at 256^3, 2^17 .. 2^19 measured within 1 %
constexpr int kSplitPrefetch = 1 << 18;
__device__ __forceinline__ void split_velocity_pair(const Params<float>& p, const PairGeo& G,
                                                    const float* __restrict__ eps, const float* __restrict__ kap,
                                                    const float* __restrict__ rho_in, const float* __restrict__ m_in,
                                                    float* __restrict__ v_out, float* __restrict__ a_out);

// K2 for node pairs.  With walls, a pair with a node on the first or last
// layer of a non-periodic axis is left to k_split_velocity_faces (the one-node
// form with its one-sided stencils); every other pair's stencils stay inside
// the grid, where the pair form's central differences are the ones the
// one-node form takes there.
template <bool WALL>
static __global__ void __launch_bounds__(kSplitMaxThreads, 4) k_split_velocity2(Params<float> p, const float* __restrict__ eps,
                                                                   const float* __restrict__ kap,
                                                                   const float* __restrict__ rho_in,
                                                                   const float* __restrict__ m_in,
                                                                   float* __restrict__ v_out, float* __restrict__ a_out)
{
    PairGeo G;
    if (!G.init(p)) return;
    if (WALL && ((p.wall[0] && (G.x == 0 || G.x + 2 >= G.nx)) || (p.wall[1] && (G.y == 0 || G.y == G.ny - 1)) ||
                 (p.wall[2] && (G.z == 0 || G.z == G.nz - 1))))
        return;
    split_velocity_pair(p, G, eps, kap, rho_in, m_in, v_out, a_out);
}

// The nodes k_split_velocity2 leaves out on a walled grid, one per thread: the
// x columns 0, 1, nx-2, nx-1 of a non-periodic x axis, then the first and last
// y rows (other columns), then the first and last z planes (other columns and
// rows).  threads: velocity_face_threads(p).
inline long long velocity_face_threads(const Params<float>& p)
{
    return (p.wall[0] ? 4LL * p.ny * p.nz : 0) + (p.wall[1] ? 2LL * p.nx * p.nz : 0) +
           (p.wall[2] ? 2LL * p.nx * p.ny : 0);
}
static __global__ void __launch_bounds__(256) k_split_velocity_faces(Params<float> p, const float* __restrict__ eps,
                                                                      const float* __restrict__ kap,
                                                                      const float* __restrict__ rho_in,
                                                                      const float* __restrict__ m_in,
                                                                      float* __restrict__ v_out,
                                                                      float* __restrict__ a_out)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    auto xface = [&](int x) { return p.wall[0] && (x <= 1 || x >= nx - 2); };
    int x, y, z;
    const long long sx = p.wall[0] ? 4LL * ny * nz : 0, sy = p.wall[1] ? 2LL * nx * nz : 0;
    if (t < sx) {
        const int c = (int)(t % 4);
        const long long r = t / 4;
        x = c < 2 ? c : nx - 4 + c;
        y = (int)(r % ny);
        z = (int)(r / ny);
    } else if ((t -= sx) < sy) {
        x = (int)(t % nx);
        const long long r = t / nx;
        y = (r & 1) ? ny - 1 : 0;
        z = (int)(r >> 1);
        if (xface(x)) return;
    } else {
        t -= sy;
        if (!p.wall[2] || t >= 2LL * nx * ny) return;
        x = (int)(t % nx);
        const long long r = t / nx;
        y = (int)(r % ny);
        z = (r / ny) ? nz - 1 : 0;
        if (xface(x) || (p.wall[1] && (y == 0 || y == ny - 1))) return;
    }
    SplitGeo g;
    g.at(p, x, y, z);
    split_velocity_node<true>(p, g, eps, kap, rho_in, m_in, v_out, a_out);
}

// K2 over the grid: node pairs, then the face nodes of a walled grid
template <bool WALL>
inline void split_velocity_launch(const Params<float>& p, const Fields<float>& F, dim3 grd, dim3 blk, cudaStream_t st)
{
    k_split_velocity2<WALL><<<grd, blk, 0, st>>>(p, F.eps, F.kap, F.rho, F.m, F.v, F.a);
    if (WALL) {
        const long long m = velocity_face_threads(p);
        if (m > 0)
            k_split_velocity_faces<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(p, F.eps, F.kap, F.rho, F.m, F.v, F.a);
    }
}

// K2 for one node pair of an all-periodic grid
__device__ __forceinline__ void split_velocity_pair(const Params<float>& p, const PairGeo& G,
                                                    const float* __restrict__ eps, const float* __restrict__ kap,
                                                    const float* __restrict__ rho_in, const float* __restrict__ m_in,
                                                    float* __restrict__ v_out, float* __restrict__ a_out)
{
    const int n = G.n;
    const long long N = p.N;
    // The register budget lets a thread keep only part of its ~45 loads in
    // flight, so the first touches of a row (DRAM misses) would wait behind
    // L2 hits.  Each thread therefore asks L2 for the inputs of the node
    // kSplitPrefetch nodes ahead, holding no registers; the blocks that run
    // about one wave later find them in L2.
    if (n + kSplitPrefetch < N) {
        const int o = n + kSplitPrefetch;
        prefetch_l2(rho_in + o);
        prefetch_l2(eps + o);
        prefetch_l2(kap + o);
#pragma unroll
        for (int c = 0; c < 3; ++c) prefetch_l2(m_in + c * N + o);
    }
    const int ym = G.oy(-1), yp = G.oy(1), zm = G.oz(-1), zp = G.oz(1);
    const Row4 E0 = row4(eps + n, G);
    const float2 e = E0.C();
    const float2 rho = ld2(rho_in + n);
    Row4 Mr[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) Mr[c] = row4(m_in + c * N + n, G);
    const float2 m[3] = {Mr[0].C(), Mr[1].C(), Mr[2].C()};
    const float2 Eyp = ld2(eps + n + yp), Eym = ld2(eps + n + ym), Ezp = ld2(eps + n + zp), Ezm = ld2(eps + n + zm);
    const float2 ge[3] = {cdiff(E0.R(), E0.L()), cdiff(Eyp, Eym), cdiff(Ezp, Ezm)};
    float2 dnu[3] = {f2(0.f), f2(0.f), f2(0.f)};
    if (p.corr & 1) {
        const Row4 Ey1 = row4(eps + n + yp, G), Ey0 = row4(eps + n + ym, G);
        const Row4 Ez1 = row4(eps + n + zp, G), Ez0 = row4(eps + n + zm, G);
        float2 H[3][3];
        H[0][0] = add2(fma2(f2(-2.f), e, E0.R()), E0.L());
        H[1][1] = add2(fma2(f2(-2.f), e, Eyp), Eym);
        H[2][2] = add2(fma2(f2(-2.f), e, Ezp), Ezm);
        H[0][1] = H[1][0] = cdiff(cdiff(Ey1.R(), Ey0.R()), cdiff(Ey1.L(), Ey0.L()));
        H[0][2] = H[2][0] = cdiff(cdiff(Ez1.R(), Ez0.R()), cdiff(Ez1.L(), Ez0.L()));
        H[1][2] = H[2][1] = cdiff(cdiff(ld2(eps + n + yp + zp), ld2(eps + n + yp + zm)),
                                  cdiff(ld2(eps + n + ym + zp), ld2(eps + n + ym + zm)));
        float2 dmm[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float* mc = m_in + c * N + n;
            dmm[c][0] = cdiff(Mr[c].R(), Mr[c].L());
            dmm[c][1] = cdiff(ld2(mc + yp), ld2(mc + ym));
            dmm[c][2] = cdiff(ld2(mc + zp), ld2(mc + zm));
        }
        const float2 trH = add2(add2(H[0][0], H[1][1]), H[2][2]);
        const float2 divm = add2(add2(dmm[0][0], dmm[1][1]), dmm[2][2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float2 r = fma2(trH, m[a], mul2(divm, ge[a]));
#pragma unroll
            for (int b = 0; b < 3; ++b) r = add2(r, fma2(H[a][b], m[b], mul2(dmm[a][b], ge[b])));
            dnu[a] = mul2(f2(p.nu_eff), r);
        }
    }
    const float2 inv_rho = make_float2(1.f / rho.x, 1.f / rho.y);
    const float2 hinv = mul2(f2(0.5f), inv_rho);
    float2 vv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) vv[a] = fma2(mul2(m[a], e), inv_rho, mul2(dnu[a], hinv));
    const float2 n2 = fma2(vv[2], vv[2], fma2(vv[1], vv[1], mul2(vv[0], vv[0])));
    const float2 nv = make_float2(sqrtf(n2.x), sqrtf(n2.y));
    const float2 kp = ld2(kap + n);
    float2 muD, muF;
    drag_coefficients<float>(p, e.x, kp.x, muD.x, muF.x);
    drag_coefficients<float>(p, e.y, kp.y, muD.y, muF.y);
    const float2 muFn = mul2(muF, nv);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        *reinterpret_cast<float2*>(v_out + a * N + n) = vv[a];
        // e b - muD v - muF |v| v + RT ge + dnu / rho
        float2 acc = fma2(e, f2(p.b[a]), mul2(mul2(muD, vv[a]), f2(-1.f)));
        acc = fma2(mul2(muFn, vv[a]), f2(-1.f), acc);
        acc = fma2(f2(p.RT), ge[a], acc);
        *reinterpret_cast<float2*>(a_out + a * N + n) = fma2(dnu[a], inv_rho, acc);
    }
}

inline bool split_supported(int lattice, int storage, int nx, int ny, int nz)
{
    const long long N = (long long)nx * ny * nz;
    return lattice == 1 && storage >= 1 && storage <= 3 && N < (1LL << 31) && nz <= 65535;
}

// Tile height of the all-periodic pair kernels: the tensor maps' height where
// they serve the collide kernel with 32-bit indices, else kSplitBY.
inline int split_tile_height(const Params<float>& p, const SplitTma* tma, bool wall)
{
    const bool i32 = 27 * p.NS < (1LL << 31);
    return !wall && p.nx % 2 == 0 && i32 && tma && tma->ok ? tma->by : kSplitBY;
}

}  // namespace lbm
