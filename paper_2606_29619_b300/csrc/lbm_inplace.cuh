// The split D3Q27 step with in-place (AA-pattern) streaming: one population
// array instead of two.  The three kernels of the split step (moments,
// velocity, collide) keep their arithmetic; the moments and collide kernels
// read and write the populations in the layout of the step's parity (see
// aa_slot).  In place is race-free here: only the collide kernel writes
// populations, it reads no population of another node, and each node writes
// exactly the slots it read -- so no node can overwrite a value another node
// has yet to read.  A parity-0 step keeps every population at its node (slot
// opp(i), stored as aligned node pairs); a parity-1 step reads from and
// writes to the neighbours' slots (the pushes of the double-buffered step).
#pragma once

#include "lbm_split.cuh"

namespace lbm {

// ---------------------------------------------------------------- helpers
// L2 eviction priority for streams that are not read again in the same pass:
// the moments kernel's population reads and the collide kernel's population
// stores (the step's output, read by the next step's moments kernel only
// after the whole grid has been swept).
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

// This thread's node pair (x, x+1) of row y in plane z, from a (x tiles of
// 64 nodes, y tiles of 4 rows, z) grid of 32 x 4 blocks.
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

__device__ __forceinline__ WGeo ip_geo(const Params<float>& p, int bx, int by, int bz)
{
    WGeo G;
    G.nx = p.nx;
    G.ny = p.ny;
    G.nz = p.nz;
    G.nxy = p.nx * p.ny;
    G.x0 = bx * 2 * kSplitBX;
    G.y0 = by * blockDim.y;
    G.x = G.x0 + 2 * threadIdx.x;
    G.y = G.y0 + threadIdx.y;
    G.z = bz;
    G.on = G.x < G.nx && G.y < G.ny;
    G.n = G.x + G.nx * G.y + G.nxy * G.z;
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

__device__ __forceinline__ WGeo ip_geo(const Params<float>& p) { return ip_geo(p, blockIdx.x, blockIdx.y, blockIdx.z); }

// ---------------------------------------------------------------- moments
template <typename S, bool WALL, int PAR, typename I>
__device__ __forceinline__ void ip_moments_pair(const Params<float>& p, const Fields<float>& F,
                                             const S* __restrict__ f, const WGeo& G)
{
    if (!G.on) return;
    const int n = G.n;
    const I NS = (I)p.NS;
    const long long N = p.N;
    float2 g[27];
    const unsigned long long once = l2_evict_first();
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        float2 r;
        if (PAR == 0) {
            r = RawH<S>::two(f + ((I)i * NS + n), once);
        } else {
            I s0, s1;
            aa_src_pair<WALL, I>(p, G, i, NS, s0, s1);
            if (!WALL && i % 3 == 1) r = RawH<S>::two(f + s0, once);  // no x displacement: an aligned pair
            else r = make_float2(RawH<S>::one(f + s0, once), RawH<S>::one(f + s1, once));
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

// ---------------------------------------------------------------- collide and stream in place
// The pair's collision (the arithmetic of k_split_collide2) once its copies
// have landed: porosity neighbourhood in se, stored populations in sg.
// Parity 0 writes the post-collision population i of each node into slot
// opp(i) of the node itself (both nodes as one aligned pair); parity 1 pushes
// it to slot i of x + c_i (slot opp(i) of x where that crosses a
// non-periodic face).  The stored value is rebased on the porosity of the node
// that will read it (x + c_i, or x itself when reflected).  False when a
// bounded wait for the copies ran out.
template <typename S, bool WALL, int PAR, typename I, bool TMA, int HO, int HX, int BY>
__device__ __forceinline__ bool ip_collide_pair(const Params<float>& p, const Fields<float>& F, S* __restrict__ f,
                                                  const WGeo& G, const float (&se)[3][BY + 2][HX],
                                                  const S (&sg)[27][BY][2 * kSplitBX], unsigned long long* bar,
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
    // this pair's moments and the neighbour values of the corrections
    const float2 rho = ld2(F.rho + n);
    float2 v[3], acc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        v[a] = ld2(F.v + a * N + n);
        acc[a] = ld2(F.a + a * N + n);
    }
    float2 phx[3] = {f2(0.f), f2(0.f), f2(0.f)}, divv = f2(0.f);
    if (p.corr & 2) {
        // q of Eq. (ex_corr) at the stencil points, from rho, v and eps there
        auto Qx = [&](int xo) {
            const int o = G.oxk(0, xo);
            return qflux(p, __ldg(F.rho + n + o), __ldg(F.v + n + o), __ldg(F.eps + n + o));
        };
        auto Q2 = [&](const float* vc, int o) {
            const float2 r = ld2(F.rho + n + o), vv = ld2(vc + n + o), ee = ld2(F.eps + n + o);
            return make_float2(qflux(p, r.x, vv.x, ee.x), qflux(p, r.y, vv.y, ee.y));
        };
        phx[0] = make_float2(fd1c(xc0, [&](int j) { return Qx(j); }), fd1c(xc1, [&](int j) { return Qx(1 + j); }));
        phx[1] = fd1c_pair(yc, [&](int j) { return Q2(F.v + N, OY(j)); });
        phx[2] = fd1c_pair(zc, [&](int j) { return Q2(F.v + 2 * N, OZ(j)); });
    }
    if (p.corr & 4) {
        const float2 dvx = make_float2(fd1c(xc0, [&](int j) { return __ldg(F.v + n + G.oxk(0, j)); }),
                                       fd1c(xc1, [&](int j) { return __ldg(F.v + n + 1 + G.oxk(1, j)); }));
        const float2 dvy = fd1c_pair(yc, [&](int j) { return ld2(F.v + N + n + OY(j)); });
        const float2 dvz = fd1c_pair(zc, [&](int j) { return ld2(F.v + 2 * N + n + OZ(j)); });
        divv = add2(add2(dvx, dvy), dvz);
    }
    if (TMA && !mbar_wait(&bar[3], cph)) return false;
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
    // the step's output: stored with L2 priority evict_first
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
        if (TMA && PAR == 0 && !mbar_wait(&bar[dz], cph)) return false;
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
                float2 gin;
                const S* gi = &sg[i][threadIdx.y][2 * threadIdx.x];
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

// ---------------------------------------------------------------- kernels
// no node of the pair on the first or last layer of a non-periodic axis: its
// sources x - c_i and its stencils stay inside the grid, where the
// all-periodic form takes the same values and arithmetic
__device__ __forceinline__ bool ip_pair_inside(const Params<float>& p, const WGeo& G)
{
    return (!p.wall[0] || (G.x > 0 && G.x + 2 < G.nx)) && (!p.wall[1] || (G.y > 0 && G.y + 1 < G.ny)) &&
           (!p.wall[2] || (G.z > 0 && G.z + 1 < G.nz));
}

template <typename S, bool WALL, int PAR, typename I>
__global__ void __launch_bounds__(kSplitMaxThreads) k_ip_moments(Params<float> p, Fields<float> F,
                                                              const S* __restrict__ f)
{
    const WGeo G = ip_geo(p);
    // parity 1 only: there the wall form checks every source slot for a
    // reflection; at parity 0 it differs in the one-sided stencils alone
    if (WALL && PAR == 1 && ip_pair_inside(p, G)) {
        ip_moments_pair<S, false, PAR, I>(p, F, f, G);
        return;
    }
    ip_moments_pair<S, WALL, PAR, I>(p, F, f, G);
}

// One block collides the 64 x 4 node tile of one plane.  The porosity
// neighbourhood arrives by one tiled copy of the padded porosity and, at
// parity 0, the populations (the nodes' own slots) by three tiled copies, one
// per z digit.  At parity 1 each population sits in slots shifted by its own
// -c_i, which tiled copies serve poorly (measured: nine boxes per tile, 16
// bytes wider on each side, were no faster than plain loads): each thread
// stages its pair's values with plain loads.  Without tensor maps (nx not a
// multiple of 8) the porosity neighbourhood is staged with plain loads too.  probe (test only): block 0
// first waits on a barrier that no copy completes, so that its bounded wait
// runs out with nothing in flight; the kernel then reports ERR_WAIT_TIMEOUT.
// shared-memory tile of the in-place collide kernels
template <typename S, bool TMA, int BY>
struct IpSmem {
    static constexpr int PX = 2 * kSplitBX;     // nodes per tile row
    static constexpr int HO = TMA ? kPadX : 2;  // porosity column of node x0 in se
    static constexpr int HX = PX + 2 * HO;
    static constexpr int HY = BY + 2;           // porosity rows y0-1 .. y0+BY
    __align__(128) float se[3][HY][HX];
    __align__(128) S sg[27][BY][PX];
    __align__(8) unsigned long long bar[5];     // populations by z digit, porosity; [4]: probe
    int s_ok;
};

template <typename S, bool WALL, int PAR, typename I, bool TMA, int BY = kSplitBY>
__device__ __forceinline__ void ip_collide_tile(const Params<float>& p, const Fields<float>& F, S* __restrict__ f,
                                                int probe, const CUtensorMap* tm_f, const CUtensorMap* tm_eps, int bx,
                                                int by, int bz, IpSmem<S, TMA, BY>& sm)
{
    using SM = IpSmem<S, TMA, BY>;
    constexpr int PX = SM::PX, HO = SM::HO, HX = SM::HX, HY = SM::HY;
    constexpr bool tma_pop = TMA && PAR == 0;
    auto& se = sm.se;
    auto& sg = sm.sg;
    auto& bar = sm.bar;
    int& s_ok = sm.s_ok;
    const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
    const WGeo G = ip_geo(p, bx, by, bz);
    const I NS = (I)p.NS;
    if (lead) {
        for (int b = 0; b < 5; ++b) mbar_init(&bar[b], 1);
        mbar_fence_init();
        s_ok = 1;
        if (probe && bx == 0 && by == 0 && bz == 0) {
            mbar_arrive_tx(&bar[4], 16u);  // 16 bytes announced, no copy brings them
            if (!mbar_wait(&bar[4], 0u, 20000ull)) {
                atomicOr(F.err, ERR_WAIT_TIMEOUT);
                s_ok = 0;
            }
        }
        if (s_ok && TMA) {
            mbar_arrive_tx(&bar[3], (unsigned)sizeof(se));
            tma_load_3d(&se[0][0][0], tm_eps, G.x0, G.y0, G.z, &bar[3]);
            if (tma_pop)
                for (int q = 0; q < 3; ++q) {
                    mbar_arrive_tx(&bar[q], 9u * BY * PX * (unsigned)sizeof(S));
                    tma_load_4d(&sg[9 * q][0][0], tm_f, G.x0, G.y0, G.z, 9 * q, &bar[q]);
                }
        }
    }
    if (!TMA) {
        // porosity of the neighbourhood, as column pairs (nx is even, so a
        // pair never straddles the periodic seam)
        for (int row = threadIdx.y; row < 3 * HY; row += BY) {
            const int dz = row / HY, dy = row - dz * HY;
            int gy = G.y0 - 1 + dy, gz = G.z - 1 + dz;
            const bool in_yz =
                !WALL || ((!p.wall[1] || (gy >= 0 && gy < G.ny)) && (!p.wall[2] || (gz >= 0 && gz < G.nz)));
            gy = gy < 0 ? gy + G.ny : gy >= G.ny ? gy - G.ny : gy;
            gz = gz < 0 ? gz + G.nz : gz >= G.nz ? gz - G.nz : gz;
            if (gy >= G.ny) continue;  // past a ragged y end
            const float* rr = F.eps + G.nx * gy + G.nxy * gz;
            for (int q = threadIdx.x; q < HX / 2; q += kSplitBX) {
                int gx = G.x0 - 2 + 2 * q;
                if (gx > G.nx) continue;  // past a ragged x end
                const bool in = in_yz && (!WALL || !p.wall[0] || (gx >= 0 && gx < G.nx));
                gx = gx < 0 ? gx + G.nx : gx >= G.nx ? gx - G.nx : gx;
                *reinterpret_cast<float2*>(&se[dz][dy][2 * q]) = in ? ld2(rr + gx) : f2(1.f);
            }
        }
    }
    if (!tma_pop && G.on) {
        // this pair's stored populations into the tile copy (read back by this thread only)
        using B = Bits<S>;
        const B* fb = reinterpret_cast<const B*>(f);
#pragma unroll
        for (int i = 0; i < 27; ++i) {
            B* d = reinterpret_cast<B*>(&sg[i][threadIdx.y][2 * threadIdx.x]);
            I s0, s1;
            if (PAR == 0) {
                s0 = (I)i * NS + G.n;
                s1 = s0 + 1;
            } else {
                aa_src_pair<WALL, I>(p, G, i, NS, s0, s1);
            }
            d[0] = __ldg(fb + s0);
            d[1] = __ldg(fb + s1);
        }
    }
    __syncthreads();  // also publishes the initialised barriers
    if (!s_ok) return;
    bool ok = true;
    if (G.on) ok = ip_collide_pair<S, WALL, PAR, I, TMA, HO, HX, BY>(p, F, f, G, se, sg, bar, 0u);
    if (!__syncthreads_and(ok)) {
        // a wait ran out: flag it and let the copies already issued land before leaving
        if (lead && TMA) {
            atomicOr(F.err, ERR_WAIT_TIMEOUT);
            mbar_wait(&bar[3], 0u);
            if (tma_pop)
                for (int q = 0; q < 3; ++q) mbar_wait(&bar[q], 0u);
        }
    }
}

// With walls, a block whose tile has no node on the first or last layer of a
// non-periodic axis runs the all-periodic form (same arithmetic there).
template <typename S, bool WALL, int PAR, typename I, bool TMA, int BY = kSplitBY>
__global__ void __launch_bounds__(kSplitBX * BY, collide_min_blocks(BY))
    k_ip_collide(Params<float> p, Fields<float> F, S* __restrict__ f, int probe,
                 const __grid_constant__ CUtensorMap tm_f, const __grid_constant__ CUtensorMap tm_eps)
{
    __shared__ IpSmem<S, TMA, BY> sm;
    if constexpr (WALL) {
        const int x0 = blockIdx.x * 2 * kSplitBX, y0 = blockIdx.y * BY, z = blockIdx.z;
        const bool inside = (!p.wall[0] || (x0 > 0 && x0 + 2 * kSplitBX < p.nx)) &&
                            (!p.wall[1] || (y0 > 0 && y0 + BY < p.ny)) && (!p.wall[2] || (z > 0 && z + 1 < p.nz));
        if (inside) {
            ip_collide_tile<S, false, PAR, I, TMA, BY>(p, F, f, probe, &tm_f, &tm_eps, blockIdx.x, blockIdx.y,
                                                       blockIdx.z, sm);
            return;
        }
    }
    ip_collide_tile<S, WALL, PAR, I, TMA, BY>(p, F, f, probe, &tm_f, &tm_eps, blockIdx.x, blockIdx.y, blockIdx.z, sm);
}

// ---------------------------------------------------------------- host side
inline bool inplace_supported(int lattice, int storage, int nx, int ny, int nz)
{
    return split_supported(lattice, storage, nx, ny, nz) && nx % 2 == 0;
}

template <typename S, int PAR, int BY>
void ip_collide_tiled(const Params<float>& p, const Fields<float>& F, S* f, const SplitTma& tma, int probe,
                      cudaStream_t st)
{
    const dim3 blk(kSplitBX, BY), grd((p.nx + 2 * kSplitBX - 1) / (2 * kSplitBX), (p.ny + BY - 1) / BY, p.nz);
    k_ip_collide<S, false, PAR, int, true, BY><<<grd, blk, 0, st>>>(p, F, f, probe, tma.f[0], tma.eps);
}

template <typename S, bool WALL, int PAR, typename I>
int ip_launch_par(const Params<float>& p, const Fields<float>& F, S* f, const SplitTma& tma, int probe,
                  cudaStream_t st, KernelClock* kc)
{
    const int by = split_tile_height(p, &tma, WALL);
    const dim3 blk(kSplitBX, by);
    const dim3 grd((p.nx + 2 * kSplitBX - 1) / (2 * kSplitBX), (p.ny + by - 1) / by, p.nz);
    clock_mark(kc, st);
    k_ip_moments<S, WALL, PAR, I><<<grd, blk, 0, st>>>(p, F, f);
    clock_mark(kc, st);
    split_velocity_launch<WALL>(p, F, grd, blk, st);
    Fields<float> FC = F;  // the collide kernel's view: the final velocity of the Picard iterations
    if (p.picard_iters > 0) FC.v = split_picard(p, F, st);
    clock_mark(kc, st);
    static const CUtensorMap none{};
    if (by == 2)
        ip_collide_tiled<S, PAR, 2>(p, FC, f, tma, probe, st);
    else if (by == 8)
        ip_collide_tiled<S, PAR, 8>(p, FC, f, tma, probe, st);
    else if (tma.ok)
        k_ip_collide<S, WALL, PAR, I, true><<<grd, blk, 0, st>>>(p, FC, f, probe, tma.f[0], tma.eps);
    else
        k_ip_collide<S, WALL, PAR, I, false><<<grd, blk, 0, st>>>(p, FC, f, probe, none, none);
    clock_mark(kc, st);
    return cudaGetLastError() != cudaSuccess;
}

// One in-place step of parity `parity`; the caller flips the parity after it.
template <typename S>
int inplace_step(const Params<float>& p, const Fields<float>& F, S* f, int parity, const SplitTma& tma, int probe,
                 cudaStream_t st, KernelClock* kc)
{
    const bool wall = p.wall[0] || p.wall[1] || p.wall[2];
    const bool i32 = 27 * p.NS < (1LL << 31);
if (wall) {
        if (parity == 0)
            return i32 ? ip_launch_par<S, true, 0, int>(p, F, f, tma, probe, st, kc)
                       : ip_launch_par<S, true, 0, long long>(p, F, f, tma, probe, st, kc);
        return i32 ? ip_launch_par<S, true, 1, int>(p, F, f, tma, probe, st, kc)
                   : ip_launch_par<S, true, 1, long long>(p, F, f, tma, probe, st, kc);
    }
    if (parity == 0)
        return i32 ? ip_launch_par<S, false, 0, int>(p, F, f, tma, probe, st, kc)
                   : ip_launch_par<S, false, 0, long long>(p, F, f, tma, probe, st, kc);
    return i32 ? ip_launch_par<S, false, 1, int>(p, F, f, tma, probe, st, kc)
               : ip_launch_par<S, false, 1, long long>(p, F, f, tma, probe, st, kc);
}

// ---------------------------------------------------------------- the two-array split step
// (here, after the in-place kernels: with walls its moments kernel is theirs)
template <typename S, int BY>
void split_collide_tiled(const Params<float>& p, const Fields<float>& F, const S* fin, S* fout, cudaStream_t st,
                         const CUtensorMap& tmf, const CUtensorMap& tme)
{
    const dim3 blk(kSplitBX, BY), grd((p.nx + 2 * kSplitBX - 1) / (2 * kSplitBX), (p.ny + BY - 1) / BY, p.nz);
    k_split_collide2<S, false, int, true, BY><<<grd, blk, 0, st>>>(p, F.eps, F.rho, F.v, F.a, fin, fout, F.err, tmf, tme);
}

template <typename S, bool WALL>
int split_launch(const Params<float>& p, const Fields<float>& F, const S* fin, S* fout, cudaStream_t st,
                 KernelClock* kc, const SplitTma* tma)
{
    clock_mark(kc, st);
    const dim3 blk(kSplitBX, kSplitBY), grd((p.nx + kSplitBX - 1) / kSplitBX, (p.ny + kSplitBY - 1) / kSplitBY, p.nz);
    // node pairs (even nx): half as many blocks along x
    const dim3 grd2((p.nx + 2 * kSplitBX - 1) / (2 * kSplitBX), grd.y, grd.z);
    const int by = split_tile_height(p, tma, WALL);
    if (!WALL && p.nx % 2 == 0) {
        const dim3 blkh(kSplitBX, by), grdh(grd2.x, (p.ny + by - 1) / by, p.nz);
        k_split_moments2<S><<<grdh, blkh, 0, st>>>(p, F.eps, F.kap, fin, F.rho, F.m, F.err);
        clock_mark(kc, st);
        k_split_velocity2<false><<<grdh, blkh, 0, st>>>(p, F.eps, F.kap, F.rho, F.m, F.v, F.a);
    } else if (p.nx % 2 == 0) {
        // walls: the node-pair moments of the in-place kernels, which read the
        // natural layout (that of a step of parity 0)
        Fields<float> FM = F;
        if (27 * p.NS < (1LL << 31))
            k_ip_moments<S, WALL, 0, int><<<grd2, blk, 0, st>>>(p, FM, fin);
        else
            k_ip_moments<S, WALL, 0, long long><<<grd2, blk, 0, st>>>(p, FM, fin);
        clock_mark(kc, st);
        split_velocity_launch<WALL>(p, F, grd2, blk, st);
    } else {
        k_split_moments<S, WALL><<<grd, blk, 0, st>>>(p, F.eps, F.kap, fin, F.rho, F.m, F.err);
        clock_mark(kc, st);
        k_split_velocity<WALL><<<grd, blk, 0, st>>>(p, F.eps, F.kap, F.rho, F.m, F.v, F.a);
    }
    Fields<float> FC = F;  // K3's view: the final velocity of the Picard iterations
    if (p.picard_iters > 0) FC.v = split_picard(p, F, st);
    clock_mark(kc, st);
    const bool i32 = 27 * p.NS < (1LL << 31);
    const CUtensorMap* tmf = nullptr;
    if (tma && tma->ok) tmf = fin == tma->fbase[0] ? &tma->f[0] : fin == tma->fbase[1] ? &tma->f[1] : nullptr;
    if (!WALL && tmf && by != kSplitBY) {
        if (by == 2)
            split_collide_tiled<S, 2>(p, FC, fin, fout, st, *tmf, tma->eps);
        else
            split_collide_tiled<S, 8>(p, FC, fin, fout, st, *tmf, tma->eps);
    } else if (p.nx % 2 == 0) {
        static const CUtensorMap none{};
        if (tmf) {
            if (i32)
                k_split_collide2<S, WALL, int, true>
                    <<<grd2, blk, 0, st>>>(p, FC.eps, FC.rho, FC.v, FC.a, fin, fout, FC.err, *tmf, tma->eps);
            else
                k_split_collide2<S, WALL, long long, true>
                    <<<grd2, blk, 0, st>>>(p, FC.eps, FC.rho, FC.v, FC.a, fin, fout, FC.err, *tmf, tma->eps);
        } else {
            if (i32)
                k_split_collide2<S, WALL, int, false>
                    <<<grd2, blk, 0, st>>>(p, FC.eps, FC.rho, FC.v, FC.a, fin, fout, FC.err, none, none);
            else
                k_split_collide2<S, WALL, long long, false>
                    <<<grd2, blk, 0, st>>>(p, FC.eps, FC.rho, FC.v, FC.a, fin, fout, FC.err, none, none);
        }
    } else if (i32) {
        k_split_collide<S, WALL, int><<<grd, blk, 0, st>>>(p, FC.eps, FC.rho, FC.v, FC.a, fin, fout);
    } else {
        k_split_collide<S, WALL, long long><<<grd, blk, 0, st>>>(p, FC.eps, FC.rho, FC.v, FC.a, fin, fout);
    }
    clock_mark(kc, st);
    return cudaGetLastError() != cudaSuccess;
}

template <int D, typename S>
int split_step(const Params<typename Codec<S>::T>& p, const Fields<typename Codec<S>::T>& F, void* f[2], int& cur,
               cudaStream_t st, KernelClock* kc, const SplitTma* tma)
{
    if constexpr (D == 3 && !std::is_same<S, double>::value) {
        const bool wall = p.wall[0] || p.wall[1] || p.wall[2];
        const int r = wall ? split_launch<S, true>(p, F, (const S*)f[cur], (S*)f[cur ^ 1], st, kc, tma)
                           : split_launch<S, false>(p, F, (const S*)f[cur], (S*)f[cur ^ 1], st, kc, tma);
        if (r) return 1;
        cur ^= 1;
        return 0;
    } else {
        (void)p; (void)F; (void)f; (void)cur; (void)st; (void)kc; (void)tma;
        return 1;
    }
}

}  // namespace lbm
