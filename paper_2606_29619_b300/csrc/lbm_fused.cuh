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
// (a population leaving through a wall is reflected, one leaving through an
// inlet / outlet plane is dropped; the planes are rebuilt by k_planes).
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

template <typename S, typename Sh>
__global__ void __launch_bounds__(Sh::NT, 2) k_fused_d3q27(Params<float> p, const float* __restrict__ eps_g,
                                                       const float* __restrict__ kap_g, const S* __restrict__ fin,
                                                       S* __restrict__ fout, unsigned* __restrict__ err, int tiles_x,
                                                       int zc)
{
    constexpr int TX = Sh::TX, TY = Sh::TY, NT = Sh::NT;
    constexpr int EX = Sh::EX, EY = Sh::EY, MX = Sh::MX, MY = Sh::MY, VX = Sh::VX, VY = Sh::VY;
    constexpr int EP = EX * EY, MP = MX * MY, VP = VX * VY, CP = TX * TY;
    constexpr int APASS = (MP + NT - 1) / NT, BPASS = (VP + NT - 1) / NT;
    extern __shared__ float sm[];
    float* E = sm + Sh::EPS_OFF;
    float* M = sm + Sh::MOM_OFF;
    float* V = sm + Sh::VEL_OFF;
    float* RA = sm + Sh::RA_OFF;

    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const long long N = p.N;
    const long long NXY = (long long)nx * ny;
    const bool wx = p.wall[0], wy = p.wall[1], wz = p.wall[2];
    int x0 = (blockIdx.x % tiles_x) * TX;
    int y0 = (blockIdx.x / tiles_x) * TY;
    int z0 = blockIdx.y * zc;
    // on a non-periodic axis the last tile is shifted back to full size so that
    // the one-sided stencils of its last node find their inward neighbours
    if (wx && x0 + TX > nx) x0 = nx > TX ? nx - TX : 0;
    if (wy && y0 + TY > ny) y0 = ny > TY ? ny - TY : 0;
    if (wz && z0 + zc > nz) z0 = nz > zc ? nz - zc : 0;
    const int z1 = min(z0 + zc, nz);
    auto ok = [&](int g, int n, bool w) { return !w || (g >= 0 && g < n); };
    auto eplane = [&](int z) { return E + ((z + 64) & (Sh::ER - 1)) * EP; };
    auto mplane = [&](int z) { return M + ((z + 100) % Sh::MR) * 4 * MP; };
    auto vplane = [&](int z) { return V + ((z + 100) % Sh::VR) * 6 * VP; };
    auto rplane = [&](int z) { return RA + ((z + 99) % Sh::RR) * 4 * CP; };
    auto zcode = [&](int z) { return axis_code(wz, z, nz); };

    // ---- per-thread node descriptors, fixed for the whole z march
    int a_xy[APASS];  // wrapped in-plane global offset, -1 if outside a wall
    int a_xc[APASS], a_yc[APASS];
    for (int k = 0; k < APASS; ++k) {
        int t = threadIdx.x + k * NT;
        a_xy[k] = -1;
        a_xc[k] = a_yc[k] = 0;
        if (t < MP) {
            int gx = x0 - 2 + t % MX, gy = y0 - 2 + t / MX;
            if (ok(gx, nx, wx) && ok(gy, ny, wy)) {
                a_xy[k] = wrapn(gx, nx) + nx * wrapn(gy, ny);
                a_xc[k] = axis_code(wx, gx, nx);
                a_yc[k] = axis_code(wy, gy, ny);
            }
        }
    }
    int b_xy[BPASS];
    int b_xc[BPASS], b_yc[BPASS];
    for (int k = 0; k < BPASS; ++k) {
        int t = threadIdx.x + k * NT;
        b_xy[k] = -1;
        b_xc[k] = b_yc[k] = 0;
        if (t < VP) {
            int gx = x0 - 1 + t % VX, gy = y0 - 1 + t / VX;
            if (ok(gx, nx, wx) && ok(gy, ny, wy)) {
                b_xy[k] = wrapn(gx, nx) + nx * wrapn(gy, ny);
                b_xc[k] = axis_code(wx, gx, nx);
                b_yc[k] = axis_code(wy, gy, ny);
            }
        }
    }
    // stage C: one tile node per thread (TX*TY <= NT)
    const int tc = threadIdx.x;
    const int ccx = tc % TX, ccy = tc / TX;
    const int cgx = x0 + ccx, cgy = y0 + ccy;
    const bool c_on = tc < CP && cgx < nx && cgy < ny;
    int c_xy = 0;
    int c_xc = 0, c_yc = 0;
    int offx[3] = {0, 0, 0}, offy[3] = {0, 0, 0};
    // per direction: leaves through a bounce-back wall / through an open plane
    bool bbx[3] = {false, false, false}, bby[3] = {false, false, false};
    bool opx[3] = {false, false, false}, opy[3] = {false, false, false};
    if (c_on) {
        c_xy = cgx + nx * cgy;
        c_xc = axis_code(wx, cgx, nx);
        c_yc = axis_code(wy, cgy, ny);
        for (int d = -1; d <= 1; ++d) {
            int gx = cgx + d, gy = cgy + d;
            bool ox = wx && (gx < 0 || gx >= nx), oy = wy && (gy < 0 || gy >= ny);
            bbx[d + 1] = ox && p.bb[0];
            opx[d + 1] = ox && !p.bb[0];
            bby[d + 1] = oy && p.bb[1];
            opy[d + 1] = oy && !p.bb[1];
            offx[d + 1] = wrapn(gx, nx) - cgx;
            offy[d + 1] = nx * (wrapn(gy, ny) - cgy);
        }
    }

    auto load_eps_plane = [&](int z) {
        if (!ok(z, nz, wz)) return;
        float* dst = eplane(z);
        const long long zoff = NXY * wrapn(z, nz);
        for (int t = threadIdx.x; t < EP; t += NT) {
            int gx = x0 - 3 + t % EX, gy = y0 - 3 + t / EX;
            float e = 1.0f;
            if (ok(gx, nx, wx) && ok(gy, ny, wy)) e = __ldg(eps_g + zoff + wrapn(gx, nx) + (long long)nx * wrapn(gy, ny));
            dst[t] = e;
        }
    };

    for (int z = z0 - 4; z <= z0 - 1; ++z) load_eps_plane(z);

    const float RT = p.RT;
    for (int za = z0 - 2; za <= z1 + 3; ++za) {
        __syncthreads();
        load_eps_plane(za + 2);
        __syncthreads();

        // ------------------------------------------------ stage A: moments (halo 2)
        if (za <= z1 + 1 && ok(za, nz, wz)) {
            const float* Ez[5] = {eplane(za - 2), eplane(za - 1), eplane(za), eplane(za + 1), eplane(za + 2)};
            float* Mz = mplane(za);
            const long long zoff = NXY * wrapn(za, nz);
            const int zcd = zcode(za);
#pragma unroll
            for (int k = 0; k < APASS; ++k) {
                const int t = threadIdx.x + k * NT;
                if (a_xy[k] < 0) continue;
                const long long n = zoff + a_xy[k];
                const int ie = (t / MX + 1) * EX + (t % MX) + 1;
                float g[27];
#pragma unroll
                for (int i = 0; i < 27; ++i) g[i] = Codec<S>::load(fin + i * N + n, p.w[i], p.inv_w[i]);
                const float kap = __ldg(kap_g + n);
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
                const float e = Ez[2][ie];
                const float rho = p.rho0 + dm / e;
                const float gex = fd1c(a_xc[k], [&](int j) { return Ez[2][ie + j]; });
                const float gey = fd1c(a_yc[k], [&](int j) { return Ez[2][ie + j * EX]; });
                const float gez = fd1c(zcd, [&](int j) { return Ez[2 + j][ie]; });
                float v0x = P1x / rho + 0.5f * (e * p.b[0] + RT * gex);
                float v0y = P1y / rho + 0.5f * (e * p.b[1] + RT * gey);
                float v0z = P1z / rho + 0.5f * (e * p.b[2] + RT * gez);
                const float nv = sqrtf(v0x * v0x + v0y * v0y + v0z * v0z);
                float muD, muF;
                drag_coefficients<float>(p, e, kap, muD, muF);
                const float fac = drag_solve_factor<float>(muD, muF, nv);
                const float s = rho * fac / e;
                Mz[t] = rho;
                Mz[MP + t] = v0x * s;
                Mz[2 * MP + t] = v0y * s;
                Mz[3 * MP + t] = v0z * s;
                if (!(rho > 0.f) || !isfinite(rho) || !(nv * fac <= 0.5f * e)) atomicOr(err, ERR_DIVERGED);
            }
        }
        __syncthreads();

        // ------------------------------------------------ stage B: velocity, acceleration (halo 1)
        const int zb = za - 2;
        if (zb >= z0 - 1 && zb <= z1 && ok(zb, nz, wz)) {
            const float* Ez[7] = {eplane(zb - 3), eplane(zb - 2), eplane(zb - 1), eplane(zb),
                                  eplane(zb + 1), eplane(zb + 2), eplane(zb + 3)};
            const float* Mz[5] = {mplane(zb - 2), mplane(zb - 1), mplane(zb), mplane(zb + 1), mplane(zb + 2)};
            float* Vz = vplane(zb);
            float* Rz = rplane(zb);
            const long long zoff = NXY * wrapn(zb, nz);
            const int zcd = zcode(zb);
#pragma unroll
            for (int k = 0; k < BPASS; ++k) {
                const int t = threadIdx.x + k * NT;
                if (b_xy[k] < 0) continue;
                const int vx = t % VX, vy = t / VX;
                const int im = (vy + 1) * MX + vx + 1;
                const int ie = (vy + 2) * EX + vx + 2;
                const int xc = b_xc[k], yc = b_yc[k];
                const float kap = __ldg(kap_g + zoff + b_xy[k]);
                const float rho = Mz[2][im];
                const float m[3] = {Mz[2][MP + im], Mz[2][2 * MP + im], Mz[2][3 * MP + im]};
                const float e = Ez[3][ie];
                // first derivatives of eps at an in-plane E position of plane Ez[3 + dz]
                auto dex = [&](int dz, int pos) { return fd1c(xc, [&](int j) { return Ez[3 + dz][pos + j]; }); };
                auto dey = [&](int dz, int pos) { return fd1c(yc, [&](int j) { return Ez[3 + dz][pos + j * EX]; }); };
                auto dez = [&](int pos) { return fd1c(zcd, [&](int j) { return Ez[3 + j][pos]; }); };
                const float ge[3] = {dex(0, ie), dey(0, ie), dez(ie)};
                float dnu[3] = {0.f, 0.f, 0.f};
                if (p.corr & 1) {
                    // Hessian of eps: diagonal by the second difference, off-diagonal
                    // by differencing the first derivative
                    float H[3][3];
                    H[0][0] = fd2c(xc, [&](int j) { return Ez[3][ie + j]; });
                    H[1][1] = fd2c(yc, [&](int j) { return Ez[3][ie + j * EX]; });
                    H[2][2] = fd2c(zcd, [&](int j) { return Ez[3 + j][ie]; });
                    H[0][1] = H[1][0] = fd1c(xc, [&](int j) { return dey(0, ie + j); });
                    H[0][2] = H[2][0] = fd1c(xc, [&](int j) { return dez(ie + j); });
                    H[1][2] = H[2][1] = fd1c(yc, [&](int j) { return dez(ie + j * EX); });
                    float dmm[3][3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const int co = (1 + c) * MP + im;
                        dmm[c][0] = fd1c(xc, [&](int j) { return Mz[2][co + j]; });
                        dmm[c][1] = fd1c(yc, [&](int j) { return Mz[2][co + j * MX]; });
                        dmm[c][2] = fd1c(zcd, [&](int j) { return Mz[2 + j][co]; });
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
                float muD, muF;
                drag_coefficients<float>(p, e, kap, muD, muF);
                const float inv_rho = 1.f / rho;
                float vv[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) vv[a] = m[a] * e * inv_rho + dnu[a] * (0.5f * inv_rho);
                const float nv = sqrtf(vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2]);
                const float inv_e2 = 1.f / (e * e);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    Vz[a * VP + t] = vv[a];
                    Vz[(3 + a) * VP + t] = rho * vv[a] * p.one_m_3RT - rho * vv[a] * vv[a] * vv[a] * inv_e2;
                }
                const int cx = vx - 1, cy = vy - 1;
                if (cx >= 0 && cx < TX && cy >= 0 && cy < TY) {
                    const int c = cy * TX + cx;
                    Rz[c] = rho;
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        Rz[(1 + a) * CP + c] = e * p.b[a] - muD * vv[a] - muF * nv * vv[a] + RT * ge[a] + dnu[a] * inv_rho;
                }
            }
        }
        __syncthreads();

        // ------------------------------------------------ stage C: collide and stream (tile)
        const int zq = za - 4;
        if (zq >= z0 && zq < z1 && c_on) {
            const float* Vz[5] = {vplane(zq - 2), vplane(zq - 1), vplane(zq), vplane(zq + 1), vplane(zq + 2)};
            const float* Ez[3] = {eplane(zq - 1), eplane(zq), eplane(zq + 1)};
            const float* Rz = rplane(zq);
            const int zcd = zcode(zq);
            const int iv = (ccy + 1) * VX + ccx + 1;
            const int ie = (ccy + 3) * EX + ccx + 3;
            const float rho = Rz[tc];
            const float acc[3] = {Rz[CP + tc], Rz[2 * CP + tc], Rz[3 * CP + tc]};
            const float v[3] = {Vz[2][iv], Vz[2][VP + iv], Vz[2][2 * VP + iv]};
            const float e = Ez[1][ie];
            float phx[3] = {0.f, 0.f, 0.f}, divv = 0.f;
            if (p.corr & 2) {
                phx[0] = fd1c(c_xc, [&](int j) { return Vz[2][3 * VP + iv + j]; });
                phx[1] = fd1c(c_yc, [&](int j) { return Vz[2][4 * VP + iv + j * VX]; });
                phx[2] = fd1c(zcd, [&](int j) { return Vz[2 + j][5 * VP + iv]; });
            }
            if (p.corr & 4) {
                divv = fd1c(c_xc, [&](int j) { return Vz[2][iv + j]; }) +
                       fd1c(c_yc, [&](int j) { return Vz[2][VP + iv + j * VX]; }) +
                       fd1c(zcd, [&](int j) { return Vz[2 + j][2 * VP + iv]; });
            }
            const float phe = (p.corr & 4) ? rho * p.eta_coef * divv : 0.f;
            const float inv_e = 1.f / e;
            const float inv_erho = 1.f / (e * rho);
            float xe[3], qe[3], xs[3], qs[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                xe[a] = v[a] * inv_e;
                qe[a] = xe[a] * xe[a];
                xs[a] = (v[a] + acc[a]) * inv_e;
                qs[a] = xs[a] * xs[a] + (phx[a] + phe) * inv_erho;
            }
            ProductDev<3, float> Peq, Pst;
            Peq.set(xe, qe, RT);
            Pst.set(xs, qs, RT);
            const float drho = rho - p.rho0;
            const float beta = p.beta;
            const long long n = NXY * zq + c_xy;
            long long offz[3];
            bool bbz[3], opz[3];
#pragma unroll
            for (int d = -1; d <= 1; ++d) {
                int gz = zq + d;
                bool oz = wz && (gz < 0 || gz >= nz);
                bbz[d + 1] = oz && p.bb[2];
                opz[d + 1] = oz && !p.bb[2];
                offz[d + 1] = NXY * (wrapn(gz, nz) - zq);
            }
#pragma unroll
            for (int i = 0; i < 27; ++i) {
                const int dx = i % 3, dy = (i / 3) % 3, dz = i / 9;
                float fe, fs;
                const float de = Peq.dev(i, fe), ds = Pst.dev(i, fs);
                const float geq = e * (drho * fe + p.rho0 * de);
                const float gst = e * (drho * fs + p.rho0 * ds);
                const float g = Codec<S>::load(fin + i * N + n, p.w[i], p.inv_w[i]);
                const float gpc = g + 2.f * beta * (geq - g) + (1.f - beta) * (gst - geq);
                if (bbx[dx] || bby[dy] || bbz[dz]) {
                    Codec<S>::store(fout + (26 - i) * N + n, gpc, p.w[26 - i], p.inv_w[26 - i]);
                } else if (!(opx[dx] || opy[dy] || opz[dz])) {
                    const float shift = (e - Ez[dz][ie + (dx - 1) + (dy - 1) * EX]) * p.w[i] * p.rho0;
                    Codec<S>::store(fout + i * N + n + offx[dx] + offy[dy] + offz[dz], gpc + shift, p.w[i], p.inv_w[i]);
                }
            }
        }
    }
}

// ------------------------------------------------------------------ host side
using ShapeA = FusedShape<28, 8, 256>;
static_assert(ShapeA::TX * ShapeA::TY <= ShapeA::NT, "stage C maps one tile node per thread");

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
