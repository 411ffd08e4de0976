// Fused D3Q27 step: one kernel per time step that marches each CTA through z
// over an (x, y) tile and keeps every intermediate field in shared memory.
//
// The step is not local: the velocity of Eq. (v_final) needs Delta_nu
// (Eq. (porosity_correction_expanded)) and hence m = rho v1 / eps on the
// neighbours, and Phi_ext / Phi_eta (Eqs. (ex_corr), (eta_corr)) need the final
// v on the neighbours, so a node depends on the moments of a halo of 2.  Each
// CTA therefore runs a three-stage pipeline per z plane:
//   A  (halo 2)  load f, moments, v0, v1, m                 -> MOM ring
//   B  (halo 1)  Delta_nu, v, a, q = rho v (1-3RT) - rho v^3/eps^2 -> VEL ring
//   C  (tile)    Phi, equilibria, collide, push-stream        -> global
// B runs two planes behind A and C two planes behind B, so that one-sided
// wall stencils (Sec. 3.5) always find their inward neighbours.  Halo nodes
// are recomputed by neighbouring CTAs (their populations are read again from
// L2); HBM sees each population about once.  Two population buffers
// alternate between steps (a halo read must not see the neighbour's update).
#pragma once

#include <algorithm>
#include <type_traits>

#include "lbm_common.cuh"
#include "lbm_sweep.cuh"

namespace lbm {

struct FusedPlan {
    int tx = 0, ty = 0, zc = 0;  // tile and z chunk
    int tiles_x = 0, tiles_y = 0, chunks = 0;
    int variant = 0;             // index of the compiled tile configuration
    size_t smem = 0;
    int threads = 0;
};

template <int TX_, int TY_, int NT_>
struct FusedShape {
    static constexpr int TX = TX_, TY = TY_, NT = NT_;
    static constexpr int EX = TX + 6, EY = TY + 6;  // porosity region, origin -3
    static constexpr int MX = TX + 4, MY = TY + 4;  // moments region,  origin -2
    static constexpr int VX = TX + 2, VY = TY + 2;  // velocity region, origin -1
    static constexpr int ER = 8, MR = 5, VR = 5, RR = 3;
    static constexpr int EPS_OFF = 0;
    static constexpr int MOM_OFF = EPS_OFF + ER * EX * EY;        // [MR][4][MY*MX]: rho, m
    static constexpr int VEL_OFF = MOM_OFF + MR * 4 * MX * MY;    // [VR][6][VY*VX]: v, q
    static constexpr int RA_OFF = VEL_OFF + VR * 6 * VX * VY;     // [RR][4][TY*TX]: rho, a
    static constexpr int FLOATS = RA_OFF + RR * 4 * TX * TY;
    static constexpr size_t SMEM = sizeof(float) * FLOATS;
};

__device__ __forceinline__ int ring(int z, int r) { return ((z % r) + r) % r; }
__device__ __forceinline__ int wrapn(int k, int n) { return ((k % n) + n) % n; }

template <typename S, typename Sh>
__global__ void __launch_bounds__(Sh::NT) k_fused_d3q27(Params<float> p, const float* __restrict__ eps_g,
                                                       const float* __restrict__ kap_g, const S* __restrict__ fin,
                                                       S* __restrict__ fout, unsigned* __restrict__ err, int tiles_x,
                                                       int zc)
{
    constexpr int TX = Sh::TX, TY = Sh::TY, NT = Sh::NT;
    constexpr int EX = Sh::EX, EY = Sh::EY, MX = Sh::MX, MY = Sh::MY, VX = Sh::VX, VY = Sh::VY;
    extern __shared__ float sm[];
    float* E = sm + Sh::EPS_OFF;
    float* M = sm + Sh::MOM_OFF;
    float* V = sm + Sh::VEL_OFF;
    float* RA = sm + Sh::RA_OFF;

    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const long long N = p.N;
    const bool wx = p.wall[0], wy = p.wall[1], wz = p.wall[2];
    int x0 = (blockIdx.x % tiles_x) * TX;
    int y0 = (blockIdx.x / tiles_x) * TY;
    int z0 = blockIdx.y * zc;
    // on a wall axis the last tile is shifted back to full size so that the
    // one-sided stencils of its last node find their inward neighbours
    if (wx && x0 + TX > nx) x0 = nx > TX ? nx - TX : 0;
    if (wy && y0 + TY > ny) y0 = ny > TY ? ny - TY : 0;
    if (wz && z0 + zc > nz) z0 = nz > zc ? nz - zc : 0;
    const int z1 = min(z0 + zc, nz);

    auto valid = [&](int g, int n, bool w) { return !w || (g >= 0 && g < n); };
    auto gidx = [&](int gx, int gy, int gz) -> long long {
        return wrapn(gx, nx) + (long long)nx * (wrapn(gy, ny) + (long long)ny * wrapn(gz, nz));
    };
    // porosity in shared memory at region-E coordinates (ex, ey) of plane z
    auto Eat = [&](int z, int ey, int ex) -> float { return E[(ring(z, Sh::ER) * EY + ey) * EX + ex]; };

    auto load_eps_plane = [&](int z) {
        if (!valid(z, nz, wz)) return;
        float* dst = E + ring(z, Sh::ER) * EY * EX;
        for (int t = threadIdx.x; t < EX * EY; t += NT) {
            int ex = t % EX, ey = t / EX;
            int gx = x0 - 3 + ex, gy = y0 - 3 + ey;
            float e = 1.0f;
            if (valid(gx, nx, wx) && valid(gy, ny, wy)) e = __ldg(eps_g + gidx(gx, gy, z));
            dst[t] = e;
        }
    };

    // first derivative of eps along axis a at region-E position (ex, ey, z)
    auto deps = [&](int a, int ex, int ey, int z) -> float {
        if (a == 0) return fd1w<float>(wx, x0 - 3 + ex, nx, [&](int j) { return Eat(z, ey, ex + j); });
        if (a == 1) return fd1w<float>(wy, y0 - 3 + ey, ny, [&](int j) { return Eat(z, ey + j, ex); });
        return fd1w<float>(wz, z, nz, [&](int j) { return Eat(z + j, ey, ex); });
    };

    for (int z = z0 - 4; z <= z0 - 1; ++z) load_eps_plane(z);

    const float RT = p.RT;
    for (int za = z0 - 2; za <= z1 + 3; ++za) {
        __syncthreads();
        load_eps_plane(za + 2);
        __syncthreads();

        // ------------------------------------------------ stage A: moments (halo 2)
        if (za <= z1 + 1 && valid(za, nz, wz)) {
            float* Mz = M + ring(za, Sh::MR) * 4 * MX * MY;
            for (int t = threadIdx.x; t < MX * MY; t += NT) {
                int mx = t % MX, my = t / MX;
                int gx = x0 - 2 + mx, gy = y0 - 2 + my;
                if (!valid(gx, nx, wx) || !valid(gy, ny, wy)) continue;
                long long n = gidx(gx, gy, za);
                int ex = mx + 1, ey = my + 1;
                float e = Eat(za, ey, ex);
                float g[27];
#pragma unroll
                for (int i = 0; i < 27; ++i) g[i] = Codec<S>::load(fin + i * N + n, p.w[i], p.inv_w[i]);
                float dm = 0.f, P1x = 0.f, P1y = 0.f, P1z = 0.f;
#pragma unroll
                for (int i = 0; i < 27; ++i) {
                    dm += g[i];
                    if (i % 3 == 2) P1x += g[i];
                    if (i % 3 == 0) P1x -= g[i];
                    if ((i / 3) % 3 == 2) P1y += g[i];
                    if ((i / 3) % 3 == 0) P1y -= g[i];
                    if (i / 9 == 2) P1z += g[i];
                    if (i / 9 == 0) P1z -= g[i];
                }
                float rho = p.rho0 + dm / e;
                float ge[3] = {deps(0, ex, ey, za), deps(1, ex, ey, za), deps(2, ex, ey, za)};
                float v0[3] = {P1x / rho + 0.5f * (e * p.b[0] + RT * ge[0]), P1y / rho + 0.5f * (e * p.b[1] + RT * ge[1]),
                               P1z / rho + 0.5f * (e * p.b[2] + RT * ge[2])};
                float nv = sqrtf(v0[0] * v0[0] + v0[1] * v0[1] + v0[2] * v0[2]);
                float muD, muF;
                drag_coefficients<float>(p, e, __ldg(kap_g + n), muD, muF);
                float fac = drag_solve_factor<float>(muD, muF, nv);
                float s = rho * fac / e;
                Mz[0 * MX * MY + t] = rho;
                Mz[1 * MX * MY + t] = v0[0] * s;
                Mz[2 * MX * MY + t] = v0[1] * s;
                Mz[3 * MX * MY + t] = v0[2] * s;
                if (!(rho > 0.f) || !isfinite(rho) || !(nv * fac <= 0.5f * e)) atomicOr(err, ERR_DIVERGED);
            }
        }
        __syncthreads();

        // ------------------------------------------------ stage B: velocity, acceleration (halo 1)
        const int zb = za - 2;
        if (zb >= z0 - 1 && zb <= z1 && valid(zb, nz, wz)) {
            float* Vz = V + ring(zb, Sh::VR) * 6 * VX * VY;
            float* Rz = RA + ring(zb, Sh::RR) * 4 * TX * TY;
            const int gzb = wz ? zb : wrapn(zb, nz);
            for (int t = threadIdx.x; t < VX * VY; t += NT) {
                int vx = t % VX, vy = t / VX;
                int gx = x0 - 1 + vx, gy = y0 - 1 + vy;
                if (!valid(gx, nx, wx) || !valid(gy, ny, wy)) continue;
                int mx = vx + 1, my = vy + 1, ex = vx + 2, ey = vy + 2;
                const int gxx = wx ? gx : wrapn(gx, nx), gyy = wy ? gy : wrapn(gy, ny);
                auto Mat = [&](int z, int c, int yy, int xx) -> float {
                    return M[(ring(z, Sh::MR) * 4 + c) * MX * MY + yy * MX + xx];
                };
                float rho = Mat(zb, 0, my, mx);
                float m[3] = {Mat(zb, 1, my, mx), Mat(zb, 2, my, mx), Mat(zb, 3, my, mx)};
                float e = Eat(zb, ey, ex);
                float ge[3] = {deps(0, ex, ey, zb), deps(1, ex, ey, zb), deps(2, ex, ey, zb)};
                float dnu[3] = {0.f, 0.f, 0.f};
                if (p.corr & 1) {
                    // Hessian of eps: diagonal by the second difference, off-diagonal
                    // by differencing the first derivative
                    float H[3][3];
                    H[0][0] = fd2w<float>(wx, gxx, nx, [&](int j) { return Eat(zb, ey, ex + j); });
                    H[1][1] = fd2w<float>(wy, gyy, ny, [&](int j) { return Eat(zb, ey + j, ex); });
                    H[2][2] = fd2w<float>(wz, gzb, nz, [&](int j) { return Eat(zb + j, ey, ex); });
                    H[0][1] = H[1][0] = fd1w<float>(wx, gxx, nx, [&](int j) { return deps(1, ex + j, ey, zb); });
                    H[0][2] = H[2][0] = fd1w<float>(wx, gxx, nx, [&](int j) { return deps(2, ex + j, ey, zb); });
                    H[1][2] = H[2][1] = fd1w<float>(wy, gyy, ny, [&](int j) { return deps(2, ex, ey + j, zb); });
                    float dmm[3][3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        dmm[c][0] = fd1w<float>(wx, gxx, nx, [&](int j) { return Mat(zb, 1 + c, my, mx + j); });
                        dmm[c][1] = fd1w<float>(wy, gyy, ny, [&](int j) { return Mat(zb, 1 + c, my + j, mx); });
                        dmm[c][2] = fd1w<float>(wz, gzb, nz, [&](int j) { return Mat(zb + j, 1 + c, my, mx); });
                    }
                    float trH = H[0][0] + H[1][1] + H[2][2];
                    float divm = dmm[0][0] + dmm[1][1] + dmm[2][2];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        float r = trH * m[a] + divm * ge[a];
#pragma unroll
                        for (int b = 0; b < 3; ++b) r += H[a][b] * m[b] + dmm[a][b] * ge[b];
                        dnu[a] = p.nu_eff * r;
                    }
                }
                float muD, muF;
                long long n = gidx(gx, gy, zb);
                drag_coefficients<float>(p, e, __ldg(kap_g + n), muD, muF);
                float vv[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) vv[a] = m[a] * e / rho + dnu[a] / (2.f * rho);
                float nv = sqrtf(vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2]);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    Vz[a * VX * VY + t] = vv[a];
                    Vz[(3 + a) * VX * VY + t] = rho * vv[a] * p.one_m_3RT - rho * vv[a] * vv[a] * vv[a] / (e * e);
                }
                int cx = vx - 1, cy = vy - 1;
                if (cx >= 0 && cx < TX && cy >= 0 && cy < TY) {
                    int c = cy * TX + cx;
                    Rz[c] = rho;
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        Rz[(1 + a) * TX * TY + c] =
                            e * p.b[a] - muD * vv[a] - muF * nv * vv[a] + RT * ge[a] + dnu[a] / rho;
                }
            }
        }
        __syncthreads();

        // ------------------------------------------------ stage C: collide and stream (tile)
        const int zcur = za - 4;
        if (zcur >= z0 && zcur < z1) {
            const int gzc = zcur;  // inside [0, nz)
            const float beta = p.beta;
            for (int t = threadIdx.x; t < TX * TY; t += NT) {
                int cx = t % TX, cy = t / TX;
                int gx = x0 + cx, gy = y0 + cy;
                if (gx >= nx || gy >= ny) continue;
                int vx = cx + 1, vy = cy + 1, ex = cx + 3, ey = cy + 3;
                auto Vat = [&](int z, int c, int yy, int xx) -> float {
                    return V[(ring(z, Sh::VR) * 6 + c) * VX * VY + yy * VX + xx];
                };
                const float* Rz = RA + ring(zcur, Sh::RR) * 4 * TX * TY;
                float rho = Rz[t];
                float acc[3] = {Rz[TX * TY + t], Rz[2 * TX * TY + t], Rz[3 * TX * TY + t]};
                float v[3] = {Vat(zcur, 0, vy, vx), Vat(zcur, 1, vy, vx), Vat(zcur, 2, vy, vx)};
                float e = Eat(zcur, ey, ex);
                float phx[3] = {0.f, 0.f, 0.f}, divv = 0.f;
                if (p.corr & 2) {
                    phx[0] = fd1w<float>(wx, gx, nx, [&](int j) { return Vat(zcur, 3, vy, vx + j); });
                    phx[1] = fd1w<float>(wy, gy, ny, [&](int j) { return Vat(zcur, 4, vy + j, vx); });
                    phx[2] = fd1w<float>(wz, gzc, nz, [&](int j) { return Vat(zcur + j, 5, vy, vx); });
                }
                if (p.corr & 4) {
                    divv = fd1w<float>(wx, gx, nx, [&](int j) { return Vat(zcur, 0, vy, vx + j); }) +
                           fd1w<float>(wy, gy, ny, [&](int j) { return Vat(zcur, 1, vy + j, vx); }) +
                           fd1w<float>(wz, gzc, nz, [&](int j) { return Vat(zcur + j, 2, vy, vx); });
                }
                float phe = (p.corr & 4) ? rho * p.eta_coef * divv : 0.f;
                float xe[3], qe[3], xs[3], qs[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    xe[a] = v[a] / e;
                    qe[a] = xe[a] * xe[a];
                    xs[a] = (v[a] + acc[a]) / e;
                    qs[a] = xs[a] * xs[a] + (phx[a] + phe) / (e * rho);
                }
                ProductDev<3, float> Peq, Pst;
                Peq.set(xe, qe, RT);
                Pst.set(xs, qs, RT);
                const float drho = rho - p.rho0;
                const long long n = gidx(gx, gy, gzc);
#pragma unroll
                for (int i = 0; i < 27; ++i) {
                    const int ci0 = i % 3 - 1, ci1 = (i / 3) % 3 - 1, ci2 = i / 9 - 1;
                    float fe, fs;
                    float de = Peq.dev(i, fe), ds = Pst.dev(i, fs);
                    float geq = e * (drho * fe + p.rho0 * de);
                    float gst = e * (drho * fs + p.rho0 * ds);
                    float g = Codec<S>::load(fin + i * N + n, p.w[i], p.inv_w[i]);
                    float gpc = g + 2.f * beta * (geq - g) + (1.f - beta) * (gst - geq);
                    int dx = gx + ci0, dy = gy + ci1, dz = gzc + ci2;
                    bool out = (wx && (dx < 0 || dx >= nx)) || (wy && (dy < 0 || dy >= ny)) ||
                               (wz && (dz < 0 || dz >= nz));
                    if (out) {
                        Codec<S>::store(fout + (26 - i) * N + n, gpc, p.w[26 - i], p.inv_w[26 - i]);
                    } else {
                        float shift = (e - Eat(zcur + ci2, ey + ci1, ex + ci0)) * p.w[i] * p.rho0;
                        Codec<S>::store(fout + i * N + gidx(dx, dy, dz), gpc + shift, p.w[i], p.inv_w[i]);
                    }
                }
            }
        }
    }
}

// ------------------------------------------------------------------ host side
using ShapeA = FusedShape<28, 8, 256>;

inline bool fused_supported(int lattice, int storage) { return lattice == 1 && storage >= 1 && storage <= 3; }

inline int fused_plan(FusedPlan& pl, int lattice, int nx, int ny, int nz, int storage, const int* wall)
{
    (void)wall;
    if (!fused_supported(lattice, storage)) return 1;
    pl.tx = ShapeA::TX;
    pl.ty = ShapeA::TY;
    pl.threads = ShapeA::NT;
    pl.smem = ShapeA::SMEM;
    pl.tiles_x = (nx + pl.tx - 1) / pl.tx;
    pl.tiles_y = (ny + pl.ty - 1) / pl.ty;
    // enough CTAs for a few waves of two CTAs per SM, chunks of at least 16 planes
    long long tiles = (long long)pl.tiles_x * pl.tiles_y;
    int chunks = (int)std::max<long long>(1, (4 * 148 * 2 + tiles - 1) / tiles);
    int zc = (nz + chunks - 1) / chunks;
    if (zc < 16) zc = std::min(16, nz);
    pl.zc = zc;
    pl.chunks = (nz + zc - 1) / zc;
    return 0;
}

template <typename S>
int fused_launch(const FusedPlan& pl, const Params<float>& p, const Fields<float>& F, const S* fin, S* fout,
                 cudaStream_t st)
{
    auto kern = k_fused_d3q27<S, ShapeA>;
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ShapeA::SMEM) != cudaSuccess)
            return 1;
        attr_set = true;
    }
    dim3 grid(pl.tiles_x * pl.tiles_y, pl.chunks);
    kern<<<grid, ShapeA::NT, ShapeA::SMEM, st>>>(p, F.eps, F.kap, fin, fout, F.err, pl.tiles_x, pl.zc);
    return cudaGetLastError() != cudaSuccess;
}

template <int D, typename S>
int fused_step(const FusedPlan& pl, const Params<typename Codec<S>::T>& p, const Fields<typename Codec<S>::T>& F,
               void* f[2], int& cur, long n, cudaStream_t st)
{
    if constexpr (D == 3 && !std::is_same<S, double>::value) {
        for (long k = 0; k < n; ++k) {
            if (fused_launch<S>(pl, p, F, (const S*)f[cur], (S*)f[cur ^ 1], st)) return 1;
            cur ^= 1;
        }
        return 0;
    } else {
        (void)pl; (void)p; (void)F; (void)f; (void)cur; (void)n; (void)st;
        return 1;
    }
}

}  // namespace lbm
