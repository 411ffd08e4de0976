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
// (a population leaving through a non-periodic face is reflected; inlet /
// outlet planes and moving walls are then rebuilt by k_planes).
// B runs two planes behind A and C two planes behind B, so that one-sided
// wall stencils (Sec. 3.5) always find their inward neighbours.  The grid is
// persistent: each CTA takes an equal share of the (tile column, z) work and
// restarts the pipeline where its share moves to the next column.  Halo nodes
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
    int tx = 0, ty = 0, zc = 0;  // tile; zc unused (the z range is split by work share)
    int tiles_x = 0, tiles_y = 0, chunks = 0;  // chunks: CTAs in the persistent grid
    int variant = 0;             // 0: periodic z (lag 1), 1: z walls (lag 2)
    int items = 0;               // work items: tile columns * z chunks
    size_t smem = 0;
    int threads = 0;
};

// LAG: planes stage B runs behind A and C behind B.  1 suffices for a
// periodic z axis (central stencils only); 2 lets the one-sided stencils at
// z walls find their inward neighbours.
// WALL: false compiles the all-periodic kernel (no one-sided stencils, no
// bounce-back or open-plane checks); true handles every boundary.
// MINB: CTAs per SM the register budget is sized for (3 fits the
// all-periodic kernel in 80 registers without spills; the wall kernels need 2).
// STG: stage the tile's populations for stage C into shared memory with
// cp.async while stage B computes, instead of loading them in stage C.
template <int TX_, int TY_, int NT_, int LAG_, bool WALL_, int MINB_, bool STG_ = false>
struct FusedShape {
    static constexpr int TX = TX_, TY = TY_, NT = NT_, LAG = LAG_, MINB = MINB_;
    static constexpr bool WALL = WALL_, STG = STG_;
    static constexpr int EX = TX + 6, EY = TY + 6;  // porosity region, origin -3
    static constexpr int MX = TX + 4, MY = TY + 4;  // moments region,  origin -2
    static constexpr int VX = TX + 2, VY = TY + 2;  // velocity region, origin -1
    // porosity ring: planes are loaded LAG + 2 ahead of stage A (two barriers
    // before their first use) and stage B's one-sided stencils reach 3 behind
    static constexpr int ER = LAG == 1 ? 8 : 16, MR = 2 * LAG + 1, VR = 2 * LAG + 1, RR = LAG + 1;
    static constexpr int EPS_OFF = 0;
    static constexpr int MF = 6;                                  // rho, m, mu_D, mu_F
    static constexpr int MOM_OFF = EPS_OFF + ER * EX * EY;        // [MR][MF][MY*MX]
    static constexpr int VEL_OFF = MOM_OFF + MR * MF * MX * MY;   // [VR][6][VY*VX]: v, q
    static constexpr int RA_OFF = VEL_OFF + VR * 6 * VX * VY;     // [RR][4][TY*TX]: rho, a
    static constexpr int FLOATS = RA_OFF + RR * 4 * TX * TY;
    static constexpr size_t SMEM = sizeof(float) * FLOATS;
    static_assert(FLOATS % 4 == 0, "the staging buffer must start 16-byte aligned");
    static_assert(TX % 4 == 0, "staging copies chunks of 4 nodes");
};

// dynamic shared memory of one CTA: the rings, plus the staging buffer
template <typename S, typename Sh>
constexpr size_t fused_smem()
{
    return Sh::SMEM + (Sh::STG ? 27 * Sh::TX * Sh::TY * sizeof(S) : 0);
}


__device__ __forceinline__ int ring(int z, int r) { return ((z % r) + r) % r; }
__device__ __forceinline__ int wrapn(int k, int n) { return ((k % n) + n) % n; }

// Per-thread view of one (x, y) tile column being marched through z.
template <typename Sh>
struct ColumnDesc {
    static constexpr int APASS = (Sh::MX * Sh::MY + Sh::NT - 1) / Sh::NT;
    static constexpr int BPASS = (Sh::VX * Sh::VY + Sh::NT - 1) / Sh::NT;
    static constexpr int EPASS = (Sh::EX * Sh::EY + Sh::NT - 1) / Sh::NT;
    int x0, y0;
    int e_xy[EPASS];            // porosity-region node: in-plane offset, -1 outside a wall
    int a_xy[APASS], a_code[APASS];  // moments-region node; code = xcode + 3 ycode
    int b_xy[BPASS], b_code[BPASS];  // velocity-region node
};

// One tile column, planes [z0, z1), of one case: the three-stage pipeline.
template <typename S, typename Sh>
__device__ __forceinline__ void fused_segment(const Params<float>& p, const float* __restrict__ eps_g,
                                              const float* __restrict__ kap_g, const S* __restrict__ fin,
                                              S* __restrict__ fout, unsigned* __restrict__ err, int tiles_x, int col,
                                              int z0, int z1, float* sm)
{
    constexpr int TX = Sh::TX, TY = Sh::TY, NT = Sh::NT;
    constexpr int EX = Sh::EX, EY = Sh::EY, MX = Sh::MX, MY = Sh::MY, VX = Sh::VX, VY = Sh::VY;
    constexpr int EP = EX * EY, MP = MX * MY, VP = VX * VY, CP = TX * TY;
    using CD = ColumnDesc<Sh>;
    float* E = sm + Sh::EPS_OFF;
    float* M = sm + Sh::MOM_OFF;
    float* V = sm + Sh::VEL_OFF;
    float* RA = sm + Sh::RA_OFF;
    S* stg = reinterpret_cast<S*>(sm + Sh::FLOATS);  // [27][TY*TX] when Sh::STG

    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const long long NS = p.NS;  // population plane stride
    const long long NXY = (long long)nx * ny;
    const bool wx = Sh::WALL && p.wall[0], wy = Sh::WALL && p.wall[1], wz = Sh::WALL && p.wall[2];
    const int xm = wz ? 1 : 0;  // extra halo planes a non-periodic z axis needs
    const float RT = p.RT;
    const float omb = 1.f - 2.f * p.beta;
    const float c3b = 3.f * p.beta - 1.f, c1b = 1.f - p.beta, c2b = 2.f * p.beta;
    auto ok = [&](int g, int n, bool w) { return !w || (g >= 0 && g < n); };
    auto eplane = [&](int z) { return E + ((z + 256) & (Sh::ER - 1)) * EP; };
    auto mplane = [&](int z) { return M + ((z + 120) % Sh::MR) * Sh::MF * MP; };
    auto vplane = [&](int z) { return V + ((z + 120) % Sh::VR) * 6 * VP; };
    auto rplane = [&](int z) { return RA + ((z + 120) % Sh::RR) * 4 * CP; };
    auto zcode = [&](int z) { return axis_code(wz, z, nz); };

    CD cd;
    // ---- column descriptors
    int x0 = (col % tiles_x) * TX, y0 = (col / tiles_x) * TY;
    // on a non-periodic axis the last tile is shifted back to full size so
    // that the one-sided stencils of its last node find their inward neighbours
    if (wx && x0 + TX > nx) x0 = nx > TX ? nx - TX : 0;
    if (wy && y0 + TY > ny) y0 = ny > TY ? ny - TY : 0;
    cd.x0 = x0;
    cd.y0 = y0;
#pragma unroll
    for (int k = 0; k < CD::EPASS; ++k) {
        int t = threadIdx.x + k * NT, gx = x0 - 3 + t % EX, gy = y0 - 3 + t / EX;
        cd.e_xy[k] = (t < EP && ok(gx, nx, wx) && ok(gy, ny, wy)) ? wrapn(gx, nx) + nx * wrapn(gy, ny) : -1;
    }
#pragma unroll
    for (int k = 0; k < CD::APASS; ++k) {
        int t = threadIdx.x + k * NT, gx = x0 - 2 + t % MX, gy = y0 - 2 + t / MX;
        bool on = t < MP && ok(gx, nx, wx) && ok(gy, ny, wy);
        cd.a_xy[k] = on ? wrapn(gx, nx) + nx * wrapn(gy, ny) : -1;
        cd.a_code[k] = on ? axis_code(wx, gx, nx) + 3 * axis_code(wy, gy, ny) : 0;
    }
#pragma unroll
    for (int k = 0; k < CD::BPASS; ++k) {
        int t = threadIdx.x + k * NT, gx = x0 - 1 + t % VX, gy = y0 - 1 + t / VX;
        bool on = t < VP && ok(gx, nx, wx) && ok(gy, ny, wy);
        cd.b_xy[k] = on ? wrapn(gx, nx) + nx * wrapn(gy, ny) : -1;
        cd.b_code[k] = on ? axis_code(wx, gx, nx) + 3 * axis_code(wy, gy, ny) : 0;
    }
    // stage C: one tile node per thread
    const int tc = threadIdx.x;
    const int ccx = tc % TX, ccy = tc / TX;
    const int cgx = x0 + ccx, cgy = y0 + ccy;
    const bool c_on = tc < CP && cgx < nx && cgy < ny;
    int c_xy = 0, c_xc = 0, c_yc = 0;
    int offx[3] = {0, 0, 0}, offy[3] = {0, 0, 0};
    unsigned bbm = 0;  // bit (axis*3 + digit): leaves through a non-periodic face (reflected)
    if (c_on) {
        c_xy = cgx + nx * cgy;
        c_xc = axis_code(wx, cgx, nx);
        c_yc = axis_code(wy, cgy, ny);
        for (int d = 0; d < 3; ++d) {
            int gx = cgx + d - 1, gy = cgy + d - 1;
            bool ox = wx && (gx < 0 || gx >= nx), oy = wy && (gy < 0 || gy >= ny);
            if (ox) bbm |= 1u << d;
            if (oy) bbm |= 1u << (3 + d);
            offx[d] = wrapn(gx, nx) - cgx;
            offy[d] = nx * (wrapn(gy, ny) - cgy);
        }
    }

    auto load_eps_plane = [&](int z) {
        if (!ok(z, nz, wz)) return;
        float* dst = eplane(z);
        const long long zoff = NXY * wrapn(z, nz);
#pragma unroll
        for (int k = 0; k < CD::EPASS; ++k) {
            int t = threadIdx.x + k * NT;
            if (t < EP) {
                if (cd.e_xy[k] >= 0) cp_async<4>(dst + t, eps_g + zoff + cd.e_xy[k]);
                else dst[t] = 1.0f;
            }
        }
        cp_async_commit();
    };

    constexpr int LAG = Sh::LAG;
    const int Alo = z0 - 2 - xm, Ahi = z1 + 1 + xm, Blo = z0 - 1 - xm, Bhi = z1 + xm;
    // Two barriers per plane: A | B | C.  The porosity plane za + LAG + 2 is
    // copied asynchronously after stage C of iteration za; iteration za + 1
    // waits for the copy before its second barrier, which orders it before
    // its first use by stage A of iteration za + 2.  The slot it overwrites is
    // older than any plane still read.
    __syncthreads();
    for (int z = Alo - LAG; z <= Alo + LAG + 1; ++z) load_eps_plane(z);
    cp_async_wait_all();
    __syncthreads();

    for (int za = Alo; za <= z1 - 1 + 2 * LAG; ++za) {

        // -------------------------------------------- stage A: moments (halo 2)
        if (za <= Ahi && ok(za, nz, wz)) {
            const float* Ez[5] = {eplane(za - 2), eplane(za - 1), eplane(za), eplane(za + 1), eplane(za + 2)};
            float* Mz = mplane(za);
            const long long zoff = NXY * wrapn(za, nz);
            const int zcd = zcode(za);
#pragma unroll
            for (int k = 0; k < CD::APASS; ++k) {
                const int t = threadIdx.x + k * NT;
                if (cd.a_xy[k] < 0) continue;
                const long long n = zoff + cd.a_xy[k];
                const int ie = (t / MX + 1) * EX + (t % MX) + 1;
                const int xc = cd.a_code[k] % 3, yc = cd.a_code[k] / 3;
                float g[27];
#pragma unroll
                for (int i = 0; i < 27; ++i) g[i] = Codec<S>::load(fin + i * NS + n, p.w[i], p.inv_w[i]);
                const float kap = __ldg(kap_g + n);
                // row sums over the x digit first: r = sum over dx, rx = (dx=+1) - (dx=-1)
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
                const float e = Ez[2][ie];
                const float rho = p.rho0 + dm / e;
                const float inv_rho = 1.f / rho;
                const float gex = fd1c(xc, [&](int j) { return Ez[2][ie + j]; });
                const float gey = fd1c(yc, [&](int j) { return Ez[2][ie + j * EX]; });
                const float gez = fd1c(zcd, [&](int j) { return Ez[2 + j][ie]; });
                const float v0x = P1x * inv_rho + 0.5f * (e * p.b[0] + RT * gex);
                const float v0y = P1y * inv_rho + 0.5f * (e * p.b[1] + RT * gey);
                const float v0z = P1z * inv_rho + 0.5f * (e * p.b[2] + RT * gez);
                const float nv = sqrtf(v0x * v0x + v0y * v0y + v0z * v0z);
                float muD, muF;
                drag_coefficients<float>(p, e, kap, muD, muF);
                const float fac = drag_solve_factor<float>(muD, muF, nv);
                const float s = rho * fac / e;
                Mz[t] = rho;
                Mz[MP + t] = v0x * s;
                Mz[2 * MP + t] = v0y * s;
                Mz[3 * MP + t] = v0z * s;
                Mz[4 * MP + t] = muD;
                Mz[5 * MP + t] = muF;
                if (!(rho > 0.f) || !isfinite(rho) || !(nv * fac <= 0.5f * e)) atomicOr(err, ERR_DIVERGED);
            }
        }
        __syncthreads();

        // -------------------------------------------- stage B: velocity, acceleration (halo 1)
        // stage C's populations of this iteration: copied while stage B runs
        if constexpr (Sh::STG) {
            const int zs = za - 2 * LAG;
            if (zs >= z0 && zs < z1) {
                constexpr int CH = TX / 4;
                const long long zoff = NXY * zs;
                const bool vec = (nx % 4 == 0) && (x0 % 4 == 0);
                for (int t = threadIdx.x; t < 27 * TY * CH; t += NT) {
                    const int i = t / (TY * CH), r = t - i * (TY * CH), cy = r / CH, k = r - cy * CH;
                    const int gx = x0 + 4 * k, gy = y0 + cy;
                    if (gy >= ny) continue;
                    S* dst = stg + i * CP + cy * TX + 4 * k;
                    const S* src = fin + i * NS + zoff + (long long)nx * gy + gx;
                    if (vec && gx + 3 < nx) {
                        cp_async<4 * sizeof(S)>(dst, src);
                    } else {
                        for (int e = 0; e < 4; ++e)
                            if (gx + e < nx) dst[e] = src[e];
                    }
                }
                cp_async_commit();
            }
        }
        const int zb = za - LAG;
        if (zb >= Blo && zb <= Bhi && ok(zb, nz, wz)) {
            const float* Ez[7] = {eplane(zb - 3), eplane(zb - 2), eplane(zb - 1), eplane(zb),
                                  eplane(zb + 1), eplane(zb + 2), eplane(zb + 3)};
            const float* Mz[5] = {mplane(zb - 2), mplane(zb - 1), mplane(zb), mplane(zb + 1), mplane(zb + 2)};
            float* Vz = vplane(zb);
            float* Rz = rplane(zb);
            const long long zoff = NXY * wrapn(zb, nz);
            const int zcd = zcode(zb);
#pragma unroll
            for (int k = 0; k < CD::BPASS; ++k) {
                const int t = threadIdx.x + k * NT;
                if (cd.b_xy[k] < 0) continue;
                const int vx = t % VX, vy = t / VX;
                const int im = (vy + 1) * MX + vx + 1;
                const int ie = (vy + 2) * EX + vx + 2;
                const int xc = cd.b_code[k] % 3, yc = cd.b_code[k] / 3;
                const float rho = Mz[2][im];
                const float m[3] = {Mz[2][MP + im], Mz[2][2 * MP + im], Mz[2][3 * MP + im]};
                const float e = Ez[3][ie];
                auto dex = [&](int pos) { return fd1c(xc, [&](int j) { return Ez[3][pos + j]; }); };
                auto dey = [&](int pos) { return fd1c(yc, [&](int j) { return Ez[3][pos + j * EX]; }); };
                auto dez = [&](int pos) { return fd1c(zcd, [&](int j) { return Ez[3 + j][pos]; }); };
                const float ge[3] = {dex(ie), dey(ie), dez(ie)};
                float dnu[3] = {0.f, 0.f, 0.f};
                if (p.corr & 1) {
                    // Hessian of eps: diagonal by the second difference, off-diagonal
                    // by differencing the first derivative
                    float H[3][3];
                    H[0][0] = fd2c(xc, [&](int j) { return Ez[3][ie + j]; });
                    H[1][1] = fd2c(yc, [&](int j) { return Ez[3][ie + j * EX]; });
                    H[2][2] = fd2c(zcd, [&](int j) { return Ez[3 + j][ie]; });
                    H[0][1] = H[1][0] = fd1c(xc, [&](int j) { return dey(ie + j); });
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
                const float inv_rho = 1.f / rho;
                float vv[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) vv[a] = m[a] * e * inv_rho + dnu[a] * (0.5f * inv_rho);
                const float nv = sqrtf(vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2]);
                const float rho_ie2 = rho / (e * e);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    Vz[a * VP + t] = vv[a];
                    Vz[(3 + a) * VP + t] = rho * vv[a] * p.one_m_3RT - rho_ie2 * vv[a] * vv[a] * vv[a];
                }
                const int cx = vx - 1, cy = vy - 1;
                if (cx >= 0 && cx < TX && cy >= 0 && cy < TY) {
                    const int c = cy * TX + cx;
                    const float muD = Mz[2][4 * MP + im], muF = Mz[2][5 * MP + im];
                    Rz[c] = rho;
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        Rz[(1 + a) * CP + c] = e * p.b[a] - muD * vv[a] - muF * nv * vv[a] + RT * ge[a] + dnu[a] * inv_rho;
                }
            }
        }
        // the porosity plane copied during the previous iteration's stage C
        // (and the staged populations) land before this barrier
        cp_async_wait_all();
        __syncthreads();

        // -------------------------------------------- stage C: collide and stream (tile)
        const int zq = za - 2 * LAG;
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
            // collision with lambda = 1 in deviations:
            //   g_pc = (1 - 2 beta) g + (3 beta - 1) g_eq + (1 - beta) g_star,
            //   g_eq = eps (drho w_i + rho dev_eq_i), g_star likewise, so
            //   g_pc = (1 - 2 beta) g + c_eq dev_eq + c_st dev_st + 2 beta eps drho w_i.
            // c_eq and c_st are folded into the z factors, so that per (y, z)
            // digit pair YZ = Psi_y (c Psi_z), dYZ = dPsi_y (c Psi_z) + Psi0_y (c dPsi_z)
            // and per population c dev = dPsi_x YZ + Psi0_x dYZ.
            const float erho = e * rho;
            const float c_eq = erho * c3b, c_st = erho * c1b, c_w = c2b * e * (rho - p.rho0);
            const long long n = NXY * zq + c_xy;
            long long offz[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                int gz = zq + d - 1;
                bool oz = wz && (gz < 0 || gz >= nz);
                if (oz) bbm |= 1u << (6 + d);
                else bbm &= ~(1u << (6 + d));
                offz[d] = NXY * (wrapn(gz, nz) - zq);
            }
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
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
                        const int i = dx + 3 * dy + 9 * dz;
                        const float comb = Fe.d[0][dx] * YZe + (Fs.d[0][dx] * YZs + Bx[dx & 1]);
                        const float g = Sh::STG ? Codec<S>::load(stg + i * CP + tc, p.w[i], p.inv_w[i])
                                                : Codec<S>::load(fin + i * NS + n, p.w[i], p.inv_w[i]);
                        const float gpc = omb * g + comb;
                        const unsigned bit = (1u << dx) | (1u << (3 + dy)) | (1u << (6 + dz));
                        if (Sh::WALL && (bbm & bit)) {
                            Codec<S>::store(fout + (26 - i) * NS + n, gpc + c_w * p.w[i], p.w[26 - i], p.inv_w[26 - i]);
                        } else {
                            // rebased on the destination's eps: + (eps - eps_dst) w_i rho0
                            const float de = e - Ez[dz][ie + (dx - 1) + (dy - 1) * EX];
                            Codec<S>::store(fout + i * NS + n + offx[dx] + offy[dy] + offz[dz],
                                            gpc + p.w[i] * (c_w + p.rho0 * de), p.w[i], p.inv_w[i]);
                        }
                    }
                }
            }
        }
        load_eps_plane(za + LAG + 2);
    }
    __syncthreads();
}

// One step of one case.  Persistent grid fed by a work queue: an item is one
// tile column over one z chunk, items are handed out chunk by chunk with the
// columns fastest, so the CTAs running at any moment work on neighbouring
// columns of the same planes and find each other's halo populations in L2.
template <typename S, typename Sh>
__global__ void __launch_bounds__(Sh::NT, Sh::MINB) k_fused_d3q27(Params<float> p, const float* __restrict__ eps_g,
                                                          const float* __restrict__ kap_g, const S* __restrict__ fin,
                                                          S* __restrict__ fout, unsigned* __restrict__ err,
                                                          int tiles_x, int ncols, int zc, int nitems,
                                                          int* __restrict__ counter)
{
    extern __shared__ float sm[];
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= nitems) break;
        const int chunk = item / ncols, col = item - chunk * ncols;
        const int z0 = chunk * zc, z1 = min(p.nz, z0 + zc);
        fused_segment<S, Sh>(p, eps_g, kap_g, fin, fout, err, tiles_x, col, z0, z1, sm);
    }
}

// ------------------------------------------------------------------ host side
// The all-periodic tile is one warp wide (stage C: a warp stores one row of
// 32 nodes); the wall shapes keep a 28-wide tile so that their larger rings
// (lag 2 in z) still fit two CTAs per SM.
using ShapeP = FusedShape<32, 8, 256, 1, false, 3>;  // periodic on every axis
using ShapeX = FusedShape<28, 8, 256, 1, true, 2>;   // walls or planes in x / y, periodic z
using ShapeW = FusedShape<28, 8, 256, 2, true, 2>;   // walls in z
static_assert(ShapeP::TX * ShapeP::TY <= ShapeP::NT && ShapeX::TX * ShapeX::TY <= ShapeX::NT &&
                  ShapeW::TX * ShapeW::TY <= ShapeW::NT,
              "stage C maps one tile node per thread");

inline bool fused_supported(int lattice, int storage) { return lattice == 1 && storage >= 1 && storage <= 3; }

template <typename K>
inline int fused_attr(K kern, size_t smem)
{
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess;
}

template <typename S, typename Sh>
inline int fused_occupancy(int* per_sm)
{
    if (fused_attr(k_fused_d3q27<S, Sh>, fused_smem<S, Sh>())) return 1;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_fused_d3q27<S, Sh>, Sh::NT, fused_smem<S, Sh>()) !=
           cudaSuccess;
}

constexpr int kFusedChunk = 32;  // z planes per work item

// Grid: as many CTAs as fit on the device at once (persistent), fed by the
// work queue; tiny grids get fewer CTAs.
inline int fused_plan(FusedPlan& pl, int lattice, int nx, int ny, int nz, int storage, const int* wall)
{
    if (!fused_supported(lattice, storage)) return 1;
    const bool zw = wall[2] != 0, anyw = wall[0] || wall[1] || wall[2];
    pl.variant = zw ? 2 : anyw ? 1 : 0;
    pl.tx = zw ? ShapeW::TX : anyw ? ShapeX::TX : ShapeP::TX;
    pl.ty = zw ? ShapeW::TY : anyw ? ShapeX::TY : ShapeP::TY;
    pl.threads = zw ? ShapeW::NT : anyw ? ShapeX::NT : ShapeP::NT;
    pl.smem = zw ? ShapeW::SMEM : anyw ? ShapeX::SMEM : ShapeP::SMEM;
    pl.tiles_x = (nx + pl.tx - 1) / pl.tx;
    pl.tiles_y = (ny + pl.ty - 1) / pl.ty;
    pl.zc = std::min(nz, kFusedChunk);
    int dev = 0, sms = 148, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int r;
    auto occ = [&](auto tag) {
        using S = decltype(tag);
        return pl.variant == 2 ? fused_occupancy<S, ShapeW>(&per_sm)
               : pl.variant == 1 ? fused_occupancy<S, ShapeX>(&per_sm)
                                 : fused_occupancy<S, ShapeP>(&per_sm);
    };
    if (storage == 1) r = occ(float());
    else if (storage == 2) r = occ(__half());
    else r = occ(__nv_bfloat16());
    if (r || per_sm < 1) return 1;
    long long items = (long long)pl.tiles_x * pl.tiles_y * ((nz + pl.zc - 1) / pl.zc);
    if (items >= (1LL << 31)) return 1;
    pl.chunks = (int)std::min<long long>((long long)sms * per_sm, items);  // CTAs in the grid
    pl.items = (int)items;
    return 0;
}

template <typename S, typename Sh>
int fused_launch(const FusedPlan& pl, const Params<float>& p, const Fields<float>& F, const S* fin, S* fout,
                 int* counter, cudaStream_t st, KernelClock* kc)
{
    if (cudaMemsetAsync(counter, 0, sizeof(int), st) != cudaSuccess) return 1;
    clock_mark(kc, st);
    k_fused_d3q27<S, Sh><<<pl.chunks, Sh::NT, fused_smem<S, Sh>(), st>>>(p, F.eps, F.kap, fin, fout, F.err, pl.tiles_x,
                                                              pl.tiles_x * pl.tiles_y, pl.zc, pl.items, counter);
    clock_mark(kc, st);
    return cudaGetLastError() != cudaSuccess;
}

template <int D, typename S>
int fused_step(const FusedPlan& pl, const Params<typename Codec<S>::T>& p, const Fields<typename Codec<S>::T>& F,
               void* f[2], int& cur, long n, int* counter, cudaStream_t st, KernelClock* kc = nullptr)
{
    if constexpr (D == 3 && !std::is_same<S, double>::value) {
        for (long k = 0; k < n; ++k) {
            int r = pl.variant == 2
                        ? fused_launch<S, ShapeW>(pl, p, F, (const S*)f[cur], (S*)f[cur ^ 1], counter, st, kc)
                    : pl.variant == 1
                        ? fused_launch<S, ShapeX>(pl, p, F, (const S*)f[cur], (S*)f[cur ^ 1], counter, st, kc)
                        : fused_launch<S, ShapeP>(pl, p, F, (const S*)f[cur], (S*)f[cur ^ 1], counter, st, kc);
            if (r) return 1;
            cur ^= 1;
        }
        return 0;
    } else {
        (void)pl; (void)p; (void)F; (void)f; (void)cur; (void)n; (void)counter; (void)st; (void)kc;
        return 1;
    }
}

}  // namespace lbm
