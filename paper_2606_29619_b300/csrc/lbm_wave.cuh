// One D3Q27 step as a single persistent launch that sweeps a wavefront through
// z, with the populations streamed in place (AA pattern, see aa_slot): one
// population array instead of two.
//
// A step has three kinds of work per plane z, each split into tiles of
// 64 x 4 nodes (one node pair per thread, the arithmetic of the split kernels):
//   M(z)  moments: post-stream populations -> rho, m = rho v1 / eps   (Eqs. (v_(0)), (v_(1)))
//   V(z)  velocity: rho, m on the 1-ring -> v, a                       (Eqs. (porosity_correction_expanded),
//                                                                        (v_final), (accel))
//   C(z)  collide: populations, rho and v on the 1-ring -> collide and stream in place
//                                                                       (Eqs. (ex_corr), (eta_corr), (prod_form),
//                                                                        (dicrete_scheme))
// V(z) needs M on the planes its stencils touch, C(z) needs V on its planes.
// A host-built schedule lists the plane items in wavefront order -- M(z)
// leads, V(z - lag_v) and C(z - lag_c) follow -- with the schedule indices of
// the plane items each one waits for.  Every CTA of a co-resident grid takes
// the tiles j, j + grid, j + 2 grid, ... of the flattened schedule; before a V
// or C tile it waits (bounded in time) until the counters of its dependencies
// show all their tiles finished.  Every dependency points to an earlier item,
// so the earliest unfinished item can always run: the sweep cannot deadlock.
//
// Why: a split step (separate moments, velocity and collide launches) reads
// every population twice from HBM and moves its scratch fields through HBM.
// In the wavefront, C(z) runs a few planes after M(z), so its second read of
// the populations and its reads of rho, m, v and a come from L2; what reaches
// HBM is close to the populations read once and written once.  In-place
// streaming is race-free here because only C writes populations, and C(z)
// writes exactly the slots that the nodes of plane z read (in M(z), which it
// waits for, and in C(z) itself, before it writes them).
#pragma once

#include <algorithm>
#include <utility>
#include <vector>

#include "lbm_split.cuh"

namespace lbm {

enum : int { WAVE_M = 0, WAVE_V = 1, WAVE_C = 2 };

// One plane of one kind of work (all its tiles); dep: schedule indices of the
// plane items whose tiles must all have finished first (-1: none).
struct WaveItem {
    int phase, z;
    int dep[3];
};

struct WaveCtl {
    const WaveItem* items;        // the schedule, P plane items
    unsigned* cnt;                // finished work items per plane item; cnt[P] counts finished CTAs,
                                  // cnt[P + 1] hands out work items in schedule order
    int P;                        // plane items (3 nz)
    int T;                        // tiles per plane
    int tiles_x;                  // tiles along x
    int tpi;                      // tiles per work item (consecutive tiles of one plane)
    int Gp;                       // work items per plane item, ceil(T / tpi)
    unsigned long long budget_ns; // limit of every wait
    int probe;                    // test only: CTA 0 first waits on a barrier that no copy completes
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* q)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(q) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_volatile_u32(const unsigned* q) { return *(const volatile unsigned*)q; }

// fields written earlier in the same launch: read through L2 (no stale L1 line)
__device__ __forceinline__ float ldc(const float* q) { return __ldcg(q); }
__device__ __forceinline__ float2 ldc2(const float* q) { return __ldcg(reinterpret_cast<const float2*>(q)); }

// L2 eviction priorities.  The moments work reads the populations of a plane
// first and the collide work reads them again a few planes later: those
// lines are kept (evict_last).  The collide work's stores are the step's
// output, read only by the next launch: they leave L2 first (evict_first),
// so that they do not push the populations still to be re-read out of it.
__device__ __forceinline__ unsigned long long l2_evict_last()
{
    unsigned long long q;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(q));
    return q;
}
__device__ __forceinline__ unsigned long long l2_evict_first()
{
    unsigned long long q;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(q));
    return q;
}
__device__ __forceinline__ unsigned ldh_b32(const void* a, unsigned long long q)
{
    unsigned v;
    asm volatile("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;\n" : "=r"(v) : "l"(a), "l"(q));
    return v;
}
__device__ __forceinline__ unsigned short ldh_b16(const void* a, unsigned long long q)
{
    unsigned short v;
    asm volatile("ld.global.nc.L2::cache_hint.b16 %0, [%1], %2;\n" : "=h"(v) : "l"(a), "l"(q));
    return v;
}
__device__ __forceinline__ uint2 ldh_b64(const void* a, unsigned long long q)
{
    uint2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.b32 {%0, %1}, [%2], %3;\n" : "=r"(v.x), "=r"(v.y) : "l"(a), "l"(q));
    return v;
}
__device__ __forceinline__ void sth_b16(void* a, unsigned short v, unsigned long long q)
{
    asm volatile("st.global.L2::cache_hint.b16 [%0], %1, %2;\n" ::"l"(a), "h"(v), "l"(q) : "memory");
}
__device__ __forceinline__ void sth_b32(void* a, unsigned v, unsigned long long q)
{
    asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;\n" ::"l"(a), "r"(v), "l"(q) : "memory");
}
__device__ __forceinline__ void sth_b64(void* a, uint2 v, unsigned long long q)
{
    asm volatile("st.global.L2::cache_hint.v2.b32 [%0], {%1, %2}, %3;\n" ::"l"(a), "r"(v.x), "r"(v.y), "l"(q) : "memory");
}

// stored values widened to FP32 without the 1/w_i scale of FP16/BF16 storage
template <typename S>
struct Raw;
template <>
struct Raw<float> {
    __device__ static float one(const float* q) { return __ldg(q); }
    __device__ static float2 two(const float* q) { return __ldg(reinterpret_cast<const float2*>(q)); }
};
template <>
struct Raw<__half> {
    __device__ static float one(const __half* q) { return __half2float(__ldg(q)); }
    __device__ static float2 two(const __half* q) { return __half22float2(__ldg(reinterpret_cast<const __half2*>(q))); }
};
template <>
struct Raw<__nv_bfloat16> {
    __device__ static float one(const __nv_bfloat16* q)
    {
        return __uint_as_float((unsigned)__ldg(reinterpret_cast<const unsigned short*>(q)) << 16);
    }
    __device__ static float2 two(const __nv_bfloat16* q)
    {
        const unsigned u = __ldg(reinterpret_cast<const unsigned*>(q));
        return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
    }
};
// the same, read with an L2 eviction priority
template <typename S>
struct RawH;
template <>
struct RawH<float> {
    __device__ static float one(const float* a, unsigned long long q) { return __uint_as_float(ldh_b32(a, q)); }
    __device__ static float2 two(const float* a, unsigned long long q)
    {
        const uint2 u = ldh_b64(a, q);
        return make_float2(__uint_as_float(u.x), __uint_as_float(u.y));
    }
};
template <>
struct RawH<__half> {
    __device__ static float one(const __half* a, unsigned long long q)
    {
        return __half2float(__ushort_as_half(ldh_b16(a, q)));
    }
    __device__ static float2 two(const __half* a, unsigned long long q)
    {
        const unsigned u = ldh_b32(a, q);
        return __half22float2(*reinterpret_cast<const __half2*>(&u));
    }
};
template <>
struct RawH<__nv_bfloat16> {
    __device__ static float one(const __nv_bfloat16* a, unsigned long long q)
    {
        return __uint_as_float((unsigned)ldh_b16(a, q) << 16);
    }
    __device__ static float2 two(const __nv_bfloat16* a, unsigned long long q)
    {
        const unsigned u = ldh_b32(a, q);
        return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
    }
};

// the raw bits of one stored value (staging copies)
template <typename S>
using Bits = typename std::conditional<sizeof(S) == 4, unsigned, unsigned short>::type;

// A tile's thread: the node pair (x, x+1) of row y in plane z.
struct WGeo {
    int x, y, z, n, nx, ny, nz, nxy;
    int x0, y0;
    bool on;
    int xl, xr;  // offsets of x-1 from x and of x+2 from x+1 (periodic wrap)
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
    // x offset of node x + k displaced by d, periodic wrap
    __device__ __forceinline__ int oxk(int k, int d) const
    {
        const int g = x + k + d;
        return (g < 0 ? g + nx : g >= nx ? g - nx : g) - (x + k);
    }
};

__device__ __forceinline__ WGeo wave_geo(const Params<float>& p, int tile, int tiles_x, int z)
{
    WGeo G;
    G.nx = p.nx;
    G.ny = p.ny;
    G.nz = p.nz;
    G.nxy = p.nx * p.ny;
    const int bx = tile % tiles_x, by = tile / tiles_x;
    G.x0 = bx * 2 * kSplitBX;
    G.y0 = by * kSplitBY;
    G.x = G.x0 + 2 * threadIdx.x;
    G.y = G.y0 + threadIdx.y;
    G.z = z;
    G.on = G.x < G.nx && G.y < G.ny;
    G.n = G.x + G.nx * G.y + G.nxy * z;
    G.xl = G.x == 0 ? G.nx - 1 : -1;
    G.xr = G.x + 2 == G.nx ? 1 - G.nx : 1;
    return G;
}

// Element indices of the stored post-stream f_bar_i of the pair's two nodes
// in layout 1 (a step of parity 1 reads them): slot opp(i) of x - c_i, or
// slot i of the node itself when x - c_i lies beyond a non-periodic face.
template <bool WALL, typename I>
__device__ __forceinline__ void aa_src_pair(const Params<float>& p, const WGeo& G, int i, I NS, I& s0, I& s1)
{
    const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
    const I base = (I)(26 - i) * NS + (I)(G.n + G.oy(-cy) + G.oz(-cz));
    if (!WALL) {
        if (cx == 0) {
            s0 = base;
            s1 = base + 1;
        } else if (cx == 1) {
            s0 = base + G.xl;
            s1 = base;
        } else {
            s0 = base + 1;
            s1 = base + 1 + G.xr;
        }
        return;
    }
    const int ys = G.y - cy, zs = G.z - cz;
    const bool ryz = (p.wall[1] && (ys < 0 || ys >= G.ny)) || (p.wall[2] && (zs < 0 || zs >= G.nz));
    const I own = (I)i * NS + (I)G.n;
    I s[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int xs = G.x + k - cx;
        const bool r = ryz || (p.wall[0] && (xs < 0 || xs >= G.nx));
        s[k] = r ? own + k : base + k + G.oxk(k, -cx);
    }
    s0 = s[0];
    s1 = s[1];
}

// ---------------------------------------------------------------- M: moments
template <typename S, bool WALL, int PAR, typename I>
__device__ __forceinline__ void wave_moments(const Params<float>& p, const Fields<float>& F,
                                             const S* __restrict__ f, const WGeo& G)
{
    if (!G.on) return;
    const int n = G.n;
    const I NS = (I)p.NS;
    const long long N = p.N;
    float2 g[27];
    const unsigned long long keep = l2_evict_last();  // the collide work reads them again
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        float2 r;
        if (PAR == 0) {
            r = RawH<S>::two(f + ((I)i * NS + n), keep);
        } else {
            I s0, s1;
            aa_src_pair<WALL, I>(p, G, i, NS, s0, s1);
            if (!WALL && i % 3 == 1) r = RawH<S>::two(f + s0, keep);  // no x displacement: an aligned pair
            else r = make_float2(RawH<S>::one(f + s0, keep), RawH<S>::one(f + s1, keep));
        }
        g[i] = sizeof(S) == 2 ? mul2(r, f2(p.w[i])) : r;
    }
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
    const float2 e = ld2(F.eps + n);
    float2 gex, gey, gez;
    if (WALL) {
        const int xc0 = axis_code(p.wall[0], G.x, G.nx), xc1 = axis_code(p.wall[0], G.x + 1, G.nx);
        const int yc = axis_code(p.wall[1], G.y, G.ny), zc = axis_code(p.wall[2], G.z, G.nz);
        gex = make_float2(fd1c(xc0, [&](int j) { return __ldg(F.eps + n + G.oxk(0, j)); }),
                          fd1c(xc1, [&](int j) { return __ldg(F.eps + n + 1 + G.oxk(1, j)); }));
        gey = fd1c_pair(yc, [&](int j) { return ld2(F.eps + n + G.oy(j)); });
        gez = fd1c_pair(zc, [&](int j) { return ld2(F.eps + n + G.oz(j)); });
    } else {
        const float el = __ldg(F.eps + n + G.xl), er = __ldg(F.eps + n + 1 + G.xr);
        gex = cdiff(make_float2(e.y, er), make_float2(el, e.x));
        gey = cdiff(ld2(F.eps + n + G.oy(1)), ld2(F.eps + n + G.oy(-1)));
        gez = cdiff(ld2(F.eps + n + G.oz(1)), ld2(F.eps + n + G.oz(-1)));
    }
    const float2 kp = ld2(F.kap + n);
    const float RT = p.RT;
    float2 rho;
    rho.x = p.rho0 + dm.x / e.x;
    rho.y = p.rho0 + dm.y / e.y;
    const float2 inv_rho = make_float2(1.f / rho.x, 1.f / rho.y);
    const float2 v0x = fma2(P1x, inv_rho, mul2(f2(0.5f), fma2(e, f2(p.b[0]), mul2(f2(RT), gex))));
    const float2 v0y = fma2(P1y, inv_rho, mul2(f2(0.5f), fma2(e, f2(p.b[1]), mul2(f2(RT), gey))));
    const float2 v0z = fma2(P1z, inv_rho, mul2(f2(0.5f), fma2(e, f2(p.b[2]), mul2(f2(RT), gez))));
    const float2 n2 = fma2(v0z, v0z, fma2(v0y, v0y, mul2(v0x, v0x)));
    const float2 nv = make_float2(sqrtf(n2.x), sqrtf(n2.y));
    float2 s;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float ek = k ? e.y : e.x, rk = k ? rho.y : rho.x, nk = k ? nv.y : nv.x;
        float muD, muF;
        drag_coefficients<float>(p, ek, k ? kp.y : kp.x, muD, muF);
        const float fk = drag_solve_factor<float>(muD, muF, nk);
        (k ? s.y : s.x) = rk * fk / ek;
        bad |= !(rk > 0.f) || !isfinite(rk) || !(nk * fk <= 0.5f * ek);
    }
    *reinterpret_cast<float2*>(F.rho + n) = rho;
    *reinterpret_cast<float2*>(F.m + n) = mul2(v0x, s);
    *reinterpret_cast<float2*>(F.m + N + n) = mul2(v0y, s);
    *reinterpret_cast<float2*>(F.m + 2 * N + n) = mul2(v0z, s);
    if (bad) atomicOr(F.err, ERR_DIVERGED);
}

// ---------------------------------------------------------------- V: velocity
// one row of a field written in this launch around the pair: x-1, x, x+1, x+2
__device__ __forceinline__ Row4 row4c(const float* __restrict__ b, const WGeo& G)
{
    const float2 c = ldc2(b);
    return {ldc(b + G.xl), c.x, c.y, ldc(b + 1 + G.xr)};
}
__device__ __forceinline__ Row4 row4g(const float* __restrict__ b, const WGeo& G)
{
    const float2 c = ld2(b);
    return {__ldg(b + G.xl), c.x, c.y, __ldg(b + 1 + G.xr)};
}

// all-periodic grids: the pair arithmetic of k_split_velocity2
__device__ __forceinline__ void wave_velocity_pair(const Params<float>& p, const Fields<float>& F, const WGeo& G)
{
    if (!G.on) return;
    const int n = G.n;
    const long long N = p.N;
    const int ym = G.oy(-1), yp = G.oy(1), zm = G.oz(-1), zp = G.oz(1);
    const Row4 E0 = row4g(F.eps + n, G);
    const float2 e = E0.C();
    const float2 rho = ldc2(F.rho + n);
    Row4 Mr[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) Mr[c] = row4c(F.m + c * N + n, G);
    const float2 m[3] = {Mr[0].C(), Mr[1].C(), Mr[2].C()};
    const float2 Eyp = ld2(F.eps + n + yp), Eym = ld2(F.eps + n + ym), Ezp = ld2(F.eps + n + zp),
                 Ezm = ld2(F.eps + n + zm);
    const float2 ge[3] = {cdiff(E0.R(), E0.L()), cdiff(Eyp, Eym), cdiff(Ezp, Ezm)};
    float2 dnu[3] = {f2(0.f), f2(0.f), f2(0.f)};
    if (p.corr & 1) {
        const Row4 Ey1 = row4g(F.eps + n + yp, G), Ey0 = row4g(F.eps + n + ym, G);
        const Row4 Ez1 = row4g(F.eps + n + zp, G), Ez0 = row4g(F.eps + n + zm, G);
        float2 H[3][3];
        H[0][0] = add2(fma2(f2(-2.f), e, E0.R()), E0.L());
        H[1][1] = add2(fma2(f2(-2.f), e, Eyp), Eym);
        H[2][2] = add2(fma2(f2(-2.f), e, Ezp), Ezm);
        H[0][1] = H[1][0] = cdiff(cdiff(Ey1.R(), Ey0.R()), cdiff(Ey1.L(), Ey0.L()));
        H[0][2] = H[2][0] = cdiff(cdiff(Ez1.R(), Ez0.R()), cdiff(Ez1.L(), Ez0.L()));
        H[1][2] = H[2][1] = cdiff(cdiff(ld2(F.eps + n + yp + zp), ld2(F.eps + n + yp + zm)),
                                  cdiff(ld2(F.eps + n + ym + zp), ld2(F.eps + n + ym + zm)));
        float2 dmm[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float* mc = F.m + c * N + n;
            dmm[c][0] = cdiff(Mr[c].R(), Mr[c].L());
            dmm[c][1] = cdiff(ldc2(mc + yp), ldc2(mc + ym));
            dmm[c][2] = cdiff(ldc2(mc + zp), ldc2(mc + zm));
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
    const float2 kp = ld2(F.kap + n);
    float2 muD, muF;
    drag_coefficients<float>(p, e.x, kp.x, muD.x, muF.x);
    drag_coefficients<float>(p, e.y, kp.y, muD.y, muF.y);
    const float2 muFn = mul2(muF, nv);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        *reinterpret_cast<float2*>(F.v + a * N + n) = vv[a];
        float2 acc = fma2(e, f2(p.b[a]), mul2(mul2(muD, vv[a]), f2(-1.f)));
        acc = fma2(mul2(muFn, vv[a]), f2(-1.f), acc);
        acc = fma2(f2(p.RT), ge[a], acc);
        *reinterpret_cast<float2*>(F.a + a * N + n) = fma2(dnu[a], inv_rho, acc);
    }
}

// grids with a non-periodic axis: the one-node arithmetic of k_split_velocity
// (boundary-coded stencils) for each node of the pair
__device__ __forceinline__ void wave_velocity_walls(const Params<float>& p, const Fields<float>& F, const WGeo& G)
{
    if (!G.on) return;
    const long long N = p.N;
#pragma unroll 1
    for (int k = 0; k < 2; ++k) {
        const int n = G.n + k, xk = G.x + k;
        const int xc = axis_code(p.wall[0], xk, G.nx);
        const int yc = axis_code(p.wall[1], G.y, G.ny);
        const int zc = axis_code(p.wall[2], G.z, G.nz);
        auto OX = [&](int d) { return G.oxk(k, d); };
        auto E = [&](int dx, int dy, int dz) { return __ldg(F.eps + n + OX(dx) + G.oy(dy) + G.oz(dz)); };
        const float rho = ldc(F.rho + n);
        const float m[3] = {ldc(F.m + n), ldc(F.m + N + n), ldc(F.m + 2 * N + n)};
        const float e = E(0, 0, 0);
        const float ge[3] = {fd1c(xc, [&](int j) { return E(j, 0, 0); }), fd1c(yc, [&](int j) { return E(0, j, 0); }),
                             fd1c(zc, [&](int j) { return E(0, 0, j); })};
        float dnu[3] = {0.f, 0.f, 0.f};
        if (p.corr & 1) {
            float H[3][3];
            H[0][0] = fd2c(xc, [&](int j) { return E(j, 0, 0); });
            H[1][1] = fd2c(yc, [&](int j) { return E(0, j, 0); });
            H[2][2] = fd2c(zc, [&](int j) { return E(0, 0, j); });
            H[0][1] = H[1][0] = fd1c(xc, [&](int j) { return fd1c(yc, [&](int q) { return E(j, q, 0); }); });
            H[0][2] = H[2][0] = fd1c(xc, [&](int j) { return fd1c(zc, [&](int q) { return E(j, 0, q); }); });
            H[1][2] = H[2][1] = fd1c(yc, [&](int j) { return fd1c(zc, [&](int q) { return E(0, j, q); }); });
            float dmm[3][3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float* mc = F.m + c * N + n;
                dmm[c][0] = fd1c(xc, [&](int j) { return ldc(mc + OX(j)); });
                dmm[c][1] = fd1c(yc, [&](int j) { return ldc(mc + G.oy(j)); });
                dmm[c][2] = fd1c(zc, [&](int j) { return ldc(mc + G.oz(j)); });
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
        drag_coefficients<float>(p, e, __ldg(F.kap + n), muD, muF);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            F.v[a * N + n] = vv[a];
            F.a[a * N + n] = e * p.b[a] - muD * vv[a] - muF * nv * vv[a] + p.RT * ge[a] + dnu[a] * inv_rho;
        }
    }
}

// ---------------------------------------------------------------- C: collide and stream in place
// The pair's collision (the split collide kernel's arithmetic) once its
// copies have landed: porosity neighbourhood in se, stored populations in sg.
// Parity 0 writes the post-collision population i of each node into slot
// opp(i) of the node itself (both nodes as one aligned pair); parity 1 pushes
// it to slot i of x + c_i (slot opp(i) of x where that crosses a
// non-periodic face).  The stored value is rebased on the porosity of the node
// that will read it (x + c_i, or x itself when reflected).  False when a
// bounded wait for the copies ran out.
template <typename S, bool WALL, int PAR, typename I, int HO, int HX>
__device__ __forceinline__ bool wave_collide_pair(const Params<float>& p, const Fields<float>& F, S* __restrict__ f,
                                                  const WGeo& G, const float (&se)[3][kHoodY][HX],
                                                  const S (&sg)[27][kSplitBY][2 * kSplitBX], unsigned long long* bar,
                                                  unsigned cph)
{
    const int n = G.n, x = G.x, y = G.y, z = G.z, nx = G.nx, ny = G.ny, nz = G.nz;
    const I N = (I)p.N, NS = (I)p.NS;
    auto OY = [&](int d) { return G.oy(d); };
    auto OZ = [&](int d) { return G.oz(d); };
    const int xc0 = WALL ? axis_code(p.wall[0], x, nx) : 0, xc1 = WALL ? axis_code(p.wall[0], x + 1, nx) : 0;
    const int yc = WALL ? axis_code(p.wall[1], y, ny) : 0;
    const int zc = WALL ? axis_code(p.wall[2], z, nz) : 0;
    const float RT = p.RT;
    // this pair's moments and the neighbour values of the corrections (written in this launch)
    const float2 rho = ldc2(F.rho + n);
    float2 v[3], acc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        v[a] = ldc2(F.v + a * N + n);
        acc[a] = ldc2(F.a + a * N + n);
    }
    float2 phx[3] = {f2(0.f), f2(0.f), f2(0.f)}, divv = f2(0.f);
    if (p.corr & 2) {
        // q of Eq. (ex_corr) at the stencil points, from rho, v and eps there
        auto Qx = [&](int xo) {
            const int o = G.oxk(0, xo);
            return qflux(p, ldc(F.rho + n + o), ldc(F.v + n + o), __ldg(F.eps + n + o));
        };
        auto Q2 = [&](const float* vc, int o) {
            const float2 r = ldc2(F.rho + n + o), vv = ldc2(vc + n + o), ee = ld2(F.eps + n + o);
            return make_float2(qflux(p, r.x, vv.x, ee.x), qflux(p, r.y, vv.y, ee.y));
        };
        phx[0] = make_float2(fd1c(xc0, [&](int j) { return Qx(j); }), fd1c(xc1, [&](int j) { return Qx(1 + j); }));
        phx[1] = fd1c_pair(yc, [&](int j) { return Q2(F.v + N, OY(j)); });
        phx[2] = fd1c_pair(zc, [&](int j) { return Q2(F.v + 2 * N, OZ(j)); });
    }
    if (p.corr & 4) {
        const float2 dvx = make_float2(fd1c(xc0, [&](int j) { return ldc(F.v + n + G.oxk(0, j)); }),
                                       fd1c(xc1, [&](int j) { return ldc(F.v + n + 1 + G.oxk(1, j)); }));
        const float2 dvy = fd1c_pair(yc, [&](int j) { return ldc2(F.v + N + n + OY(j)); });
        const float2 dvz = fd1c_pair(zc, [&](int j) { return ldc2(F.v + 2 * N + n + OZ(j)); });
        divv = add2(add2(dvx, dvy), dvz);
    }
    if (!mbar_wait(&bar[3], cph)) return false;
    const int tx = 2 * threadIdx.x + HO, ty = threadIdx.y + 1;  // porosity column of node x
    const float2 e = *reinterpret_cast<const float2*>(&se[1][ty][tx]);
    const float2 phe = (p.corr & 4) ? mul2(mul2(rho, f2(p.eta_coef)), divv) : f2(0.f);
    const float2 inv_e = make_float2(1.f / e.x, 1.f / e.y);
    const float2 inv_erho = make_float2(inv_e.x / rho.x, inv_e.y / rho.y);
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
    constexpr bool SC = sizeof(S) == 2;
    if constexpr (SC) {
        // collide in units of the stored value g / w_i (see k_split_collide2)
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
    const int ox[2][2] = {{G.oxk(0, -1), G.oxk(0, 1)}, {G.oxk(1, -1), G.oxk(1, 1)}};  // [node][dx = 0, 2]
    // the step's output: stored with L2 priority evict_first (see l2_evict_first)
    const unsigned long long out = l2_evict_first();
    auto st2 = [&](S* d, float2 g) {
        if constexpr (std::is_same<S, __half>::value) {
            const __half2 h = __float22half2_rn(g);
            sth_b32(d, *reinterpret_cast<const unsigned*>(&h), out);
        } else if constexpr (SC) {
            const __nv_bfloat162 h = __float22bfloat162_rn(g);
            sth_b32(d, *reinterpret_cast<const unsigned*>(&h), out);
        } else {
            sth_b64(d, make_uint2(__float_as_uint(g.x), __float_as_uint(g.y)), out);
        }
    };
    auto st1 = [&](S* d, float g) {
        if constexpr (std::is_same<S, __half>::value) sth_b16(d, __half_as_ushort(__float2half_rn(g)), out);
        else if constexpr (SC) sth_b16(d, __bfloat16_as_ushort(__float2bfloat16_rn(g)), out);
        else sth_b32(d, __float_as_uint(g), out);
    };
#pragma unroll
    for (int dz = 0; dz < 3; ++dz) {
        if (PAR == 0 && !mbar_wait(&bar[dz], cph)) return false;
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
                if (PAR == 0) {
                    // both nodes keep the population in their own slot opp(i): one aligned pair
                    float2 val;
                    if (dx == 1) {
                        val = (WALL && (bbm[0] & (byz | 2u))) ? gpc
                                                               : fma2(f2(rw), sub2(e, *reinterpret_cast<const float2*>(er)), gpc);
                    } else {
                        const unsigned bit = byz | (1u << dx);
                        val.x = (WALL && (bbm[0] & bit)) ? gpc.x : fmaf(rw, e.x - er[dx - 1], gpc.x);
                        val.y = (WALL && (bbm[1] & bit)) ? gpc.y : fmaf(rw, e.y - er[dx], gpc.y);
                    }
                    st2(f + ((I)(26 - i) * NS + n), val);
                } else if (dx == 1) {
                    // no x displacement: both nodes go the same way, as a pair
                    if (WALL && (bbm[0] & (byz | 2u)))
                        st2(f + ((I)(26 - i) * NS + n), gpc);
                    else
                        st2(f + ((I)i * NS + row), fma2(f2(rw), sub2(e, *reinterpret_cast<const float2*>(er)), gpc));
                } else {
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const float g = k ? gpc.y : gpc.x, ek = k ? e.y : e.x;
                        const unsigned bit = byz | (1u << dx);
                        if (WALL && (bbm[k] & bit))
                            st1(f + ((I)(26 - i) * NS + n + k), g);
                        else
                            st1(f + ((I)i * NS + row + k + ox[k][dx >> 1]), fmaf(rw, ek - er[k + dx - 1], g));
                    }
                }
            }
        }
    }
    return true;
}

// ---------------------------------------------------------------- the sweep
// Waits (thread 0) until every dependency of `it` has all its tiles finished;
// false when the wait ran out (ERR_WAIT_TIMEOUT is set) or another CTA gave up.
static __device__ __noinline__ bool wave_wait_deps(const WaveCtl& ctl, const WaveItem& it, unsigned* err)
{
    const unsigned long long t0 = globaltimer_ns();
#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
        const int q = it.dep[d];
        if (q < 0) continue;
        unsigned k = 0;
        while (ld_acquire_u32(ctl.cnt + q) < (unsigned)ctl.Gp) {
            if ((++k & 7) == 0) {
                if (ld_volatile_u32(err) & ERR_WAIT_TIMEOUT) return false;
                if (globaltimer_ns() - t0 > ctl.budget_ns) {
                    atomicOr(err, ERR_WAIT_TIMEOUT);
                    return false;
                }
            }
            __nanosleep(100);
        }
    }
    __threadfence();
    return true;
}

template <typename S, bool WALL, int PAR, typename I>
__global__ void __launch_bounds__(kSplitThreads, 5) k_wave(Params<float> p, Fields<float> F, S* __restrict__ f,
                                                         WaveCtl ctl, const __grid_constant__ CUtensorMap tm_f,
                                                         const __grid_constant__ CUtensorMap tm_eps)
{
    constexpr int PX = 2 * kSplitBX;  // nodes per tile row
    constexpr int HO = kPadX;         // porosity column of node x0 in se (the padded grid's margin)
    constexpr int HX = PX + 2 * HO;
    __shared__ __align__(128) float se[3][kHoodY][HX];
    __shared__ __align__(128) S sg[27][kSplitBY][PX];
    __shared__ __align__(8) unsigned long long bar[5];  // populations by z digit, porosity; [4]: probe
    __shared__ int s_go, s_last;
    const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
    const int tid = threadIdx.x + kSplitBX * threadIdx.y;
    const I NS = (I)p.NS;
    if (lead) {
        for (int b = 0; b < 5; ++b) mbar_init(&bar[b], 1);
        mbar_fence_init();
    }
    __syncthreads();
    bool alive = true;
    if (ctl.probe && blockIdx.x == 0) {
        // test only: 16 bytes are announced on a barrier and no copy brings
        // them, so the bounded wait runs out (no copy is in flight)
        if (lead) {
            mbar_arrive_tx(&bar[4], 16u);
            s_go = mbar_wait(&bar[4], 0u, 20000ull);
            if (!s_go) atomicOr(F.err, ERR_WAIT_TIMEOUT);
        }
        __syncthreads();
        alive = s_go != 0;
    }
    unsigned cph = 0;  // phase of the copy barriers: one completion per collide tile
    // One work item: a group of ctl.tpi consecutive tiles of one plane item.
    // CTAs take work items in schedule order from a shared ticket counter, the
    // next ticket fetched while the current item runs.  Every dependency of an
    // item belongs to an earlier ticket, already taken by a running CTA, so
    // the waits always end.
    const unsigned total = (unsigned)ctl.P * (unsigned)ctl.Gp;
    __shared__ unsigned s_item;
    if (lead) s_item = atomicAdd(ctl.cnt + ctl.P + 1, 1u);
    __syncthreads();
#pragma unroll 1
    for (unsigned j = s_item; alive && j < total; j = s_item) {
        unsigned next = 0;
        if (lead) next = atomicAdd(ctl.cnt + ctl.P + 1, 1u);
        const int pi = (int)(j / (unsigned)ctl.Gp), grp = (int)(j - (unsigned)pi * (unsigned)ctl.Gp);
        const WaveItem it = ctl.items[pi];
        const int t0 = grp * ctl.tpi, t1 = min(ctl.T, t0 + ctl.tpi);
        if (it.phase == WAVE_M) {
#pragma unroll 1
            for (int t = t0; t < t1; ++t) wave_moments<S, WALL, PAR, I>(p, F, f, wave_geo(p, t, ctl.tiles_x, it.z));
        } else if (it.phase == WAVE_V) {
            if (lead) s_go = wave_wait_deps(ctl, it, F.err);
            __syncthreads();
            if (!s_go) break;
#pragma unroll 1
            for (int t = t0; t < t1; ++t) {
                const WGeo G = wave_geo(p, t, ctl.tiles_x, it.z);
                if (WALL) wave_velocity_walls(p, F, G);
                else wave_velocity_pair(p, F, G);
            }
        } else {
            // ---- C, tile by tile.  The copies of a tile that depend on nothing
            // of this launch go first: the porosity neighbourhood (one box of
            // the padded porosity) and, at parity 0, the tile's populations
            // (three boxes by z digit); the first tile's are in flight while
            // the dependencies are awaited.
            constexpr bool tma_pop = PAR == 0;
            auto issue = [&](int x0, int y0) {
                mbar_arrive_tx(&bar[3], (unsigned)sizeof(se));
                tma_load_3d(&se[0][0][0], &tm_eps, x0, y0, it.z, &bar[3]);
                if (tma_pop)
                    for (int q = 0; q < 3; ++q) {
                        mbar_arrive_tx(&bar[q], 9u * kSplitBY * PX * (unsigned)sizeof(S));
                        tma_load_4d(&sg[9 * q][0][0], &tm_f, x0, y0, it.z, 9 * q, &bar[q]);
                    }
            };
            auto drain = [&]() {
                // a wait ran out: let the copies already issued land before leaving
                if (lead) {
                    mbar_wait(&bar[3], cph);
                    if (tma_pop)
                        for (int q = 0; q < 3; ++q) mbar_wait(&bar[q], cph);
                }
            };
            bool failed = false;
#pragma unroll 1
            for (int t = t0; t < t1; ++t) {
                const WGeo G = wave_geo(p, t, ctl.tiles_x, it.z);
                if (lead) issue(G.x0, G.y0);
                if (!tma_pop && G.on) {
                    // this pair's stored populations into the tile copy (read back by this thread only)
                    using B = Bits<S>;
                    const B* fb = reinterpret_cast<const B*>(f);
#pragma unroll
                    for (int i = 0; i < 27; ++i) {
                        B* d = reinterpret_cast<B*>(&sg[i][threadIdx.y][2 * threadIdx.x]);
                        I s0, s1;
                        aa_src_pair<WALL, I>(p, G, i, NS, s0, s1);
                        d[0] = __ldg(fb + s0);
                        d[1] = __ldg(fb + s1);
                    }
                }
                if (t == t0) {
                    if (lead) s_go = wave_wait_deps(ctl, it, F.err);
                    __syncthreads();
                    if (!s_go) {
                        drain();
                        failed = true;
                        break;
                    }
                }
                bool ok = true;
                if (G.on) ok = wave_collide_pair<S, WALL, PAR, I, HO, HX>(p, F, f, G, se, sg, bar, cph);
                // (also: every thread is done with se / sg before the next tile's copies)
                if (!__syncthreads_and(ok)) {
                    drain();
                    atomicOr(F.err, ERR_WAIT_TIMEOUT);
                    failed = true;
                    break;
                }
                cph ^= 1u;
            }
            if (failed) break;
        }
        __syncthreads();
        if (lead) {
            __threadfence();
            atomicAdd(ctl.cnt + pi, 1u);
            s_item = next;
        }
        __syncthreads();
    }
    // every CTA counts itself out; the last one clears the counters for the next launch
    __syncthreads();
    if (lead) {
        __threadfence();
        s_last = atomicAdd(ctl.cnt + ctl.P, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int k = tid; k <= ctl.P + 1; k += kSplitThreads) ctl.cnt[k] = 0u;
    }
}

// ---------------------------------------------------------------- host side
// Planes whose M (or V) values the stencils of plane z read: z and its two
// neighbours (periodic wrap), or the three planes of the one-sided stencils at
// the ends of a non-periodic z axis (Sec. 3.5).
inline void wave_stencil_planes(int z, int nz, bool zwall, int* q)
{
    if (zwall) {
        const int lo = z == 0 ? 0 : z == nz - 1 ? nz - 3 : z - 1;
        for (int k = 0; k < 3; ++k) q[k] = lo + k;
    } else {
        q[0] = (z - 1 + nz) % nz;
        q[1] = z;
        q[2] = (z + 1) % nz;
    }
}

// The wavefront: round r offers M(r), V(r - lag_v) and C(r - lag_c); an item
// whose dependencies have not all been listed yet waits in a pending list
// (the planes next to a periodic seam) and is listed as soon as they are.
// Every item therefore depends only on items listed before it.
inline std::vector<WaveItem> wave_schedule(int nz, bool zwall, int lag_v, int lag_c)
{
    std::vector<WaveItem> items;
    std::vector<int> idx(3 * (size_t)nz, -1);
    std::vector<std::pair<int, int>> pending;
    auto ready = [&](int ph, int z) {
        if (ph == WAVE_M) return true;
        int q[3];
        wave_stencil_planes(z, nz, zwall, q);
        for (int k = 0; k < 3; ++k)
            if (idx[(size_t)(ph - 1) * nz + q[k]] < 0) return false;
        return true;
    };
    auto emit = [&](int ph, int z) {
        WaveItem it;
        it.phase = ph;
        it.z = z;
        int q[3];
        wave_stencil_planes(z, nz, zwall, q);
        for (int k = 0; k < 3; ++k) it.dep[k] = ph == WAVE_M ? -1 : idx[(size_t)(ph - 1) * nz + q[k]];
        idx[(size_t)ph * nz + z] = (int)items.size();
        items.push_back(it);
    };
    auto flush = [&]() {
        for (bool moved = true; moved;) {
            moved = false;
            for (size_t k = 0; k < pending.size();) {
                if (ready(pending[k].first, pending[k].second)) {
                    emit(pending[k].first, pending[k].second);
                    pending.erase(pending.begin() + (long)k);
                    moved = true;
                } else {
                    ++k;
                }
            }
        }
    };
    for (int r = 0; r < nz + lag_c + 1; ++r) {
        if (r < nz) pending.push_back({WAVE_M, r});
        if (r - lag_v >= 0 && r - lag_v < nz) pending.push_back({WAVE_V, r - lag_v});
        if (r - lag_c >= 0 && r - lag_c < nz) pending.push_back({WAVE_C, r - lag_c});
        flush();
    }
    flush();
    return items;  // 3 nz items when every plane was listed
}

inline bool wave_supported(int lattice, int storage, int nx, int ny, int nz)
{
    const long long N = (long long)nx * ny * nz;
    return lattice == 1 && storage >= 1 && storage <= 3 && nx % 8 == 0 && N < (1LL << 31) &&
           tensor_map_encoder() != nullptr;
}

// CTAs of one instance that fit on the device at once (the grid of the
// cooperative launch: every CTA resident, so that the waits always end)
template <typename S, bool WALL, int PAR, typename I>
int wave_grid_limit()
{
    static int limit = 0;
    if (!limit) {
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wave<S, WALL, PAR, I>, kSplitThreads, 0) !=
                cudaSuccess)
            return 0;
        limit = per_sm * sms;
    }
    return limit;
}

template <typename S, bool WALL, int PAR, typename I>
int wave_launch_one(const Params<float>& p, const Fields<float>& F, S* f, const WaveCtl& ctl, const SplitTma& tma,
                    int ctas, cudaStream_t st)
{
    const int lim = wave_grid_limit<S, WALL, PAR, I>();
    if (lim <= 0) return 1;
    const long long total = (long long)ctl.P * ctl.Gp;
    const int grid = (int)std::min<long long>(std::min<long long>(lim, total), ctas > 0 ? ctas : lim);
    Params<float> pp = p;
    Fields<float> FF = F;
    S* ff = f;
    WaveCtl cc = ctl;
    CUtensorMap tf = tma.f[0], te = tma.eps;
    void* args[] = {&pp, &FF, &ff, &cc, &tf, &te};
    return cudaLaunchCooperativeKernel((const void*)k_wave<S, WALL, PAR, I>, dim3(grid), dim3(kSplitBX, kSplitBY),
                                       args, 0, st) != cudaSuccess;
}

// One step of parity `parity` (0 or 1); the caller flips the parity after it.
// ctas: grid size (0: as many CTAs as fit on the device at once; never more).
template <typename S>
int wave_launch(const Params<float>& p, const Fields<float>& F, S* f, int parity, const WaveCtl& ctl,
                const SplitTma& tma, int ctas, cudaStream_t st)
{
    const bool wall = p.wall[0] || p.wall[1] || p.wall[2];
    const bool i32 = 27 * p.NS < (1LL << 31);
    if (wall) {
        if (parity == 0)
            return i32 ? wave_launch_one<S, true, 0, int>(p, F, f, ctl, tma, ctas, st)
                       : wave_launch_one<S, true, 0, long long>(p, F, f, ctl, tma, ctas, st);
        return i32 ? wave_launch_one<S, true, 1, int>(p, F, f, ctl, tma, ctas, st)
                   : wave_launch_one<S, true, 1, long long>(p, F, f, ctl, tma, ctas, st);
    }
    if (parity == 0)
        return i32 ? wave_launch_one<S, false, 0, int>(p, F, f, ctl, tma, ctas, st)
                   : wave_launch_one<S, false, 0, long long>(p, F, f, ctl, tma, ctas, st);
    return i32 ? wave_launch_one<S, false, 1, int>(p, F, f, ctl, tma, ctas, st)
               : wave_launch_one<S, false, 1, long long>(p, F, f, ctl, tma, ctas, st);
}

}  // namespace lbm
