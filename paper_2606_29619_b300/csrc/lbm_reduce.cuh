// Domain-wide FP64 reductions (mass, mean velocity, steady-state residual,
// drag) in two deterministic passes: per-block partial sums with warp
// shuffles, then one block that adds the partials in a fixed order.
#pragma once

#include "lbm_common.cuh"
#include "lbm_sweep.cuh"

namespace lbm {

constexpr int RED_N = 12;  // mass, sum v (3), sum |v|^2, sum |v-vref|^2, drag (3), sum |vref|^2, 2 spare
constexpr int RED_THREADS = 256;

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Block-reduces acc[RED_N] and writes the block's sums to out[RED_N].
__device__ __forceinline__ void block_store(double* acc, double* out)
{
    __shared__ double sh[RED_THREADS / 32][RED_N];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < RED_N; ++k) {
        double s = warp_sum(acc[k]);
        if (lane == 0) sh[wid][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < RED_N) {
        double s = 0.0;
        for (int w = 0; w < RED_THREADS / 32; ++w) s += sh[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// Pass 1 over the current state; rho and v are the fields of the last moments
// pass.  vref may be null (no residual).
template <int D, typename S>
__global__ void __launch_bounds__(RED_THREADS) k_reduce_partial(Params<typename Codec<S>::T> p, Fields<typename Codec<S>::T> F,
                                                                const S* __restrict__ f,
                                                                const typename Codec<S>::T* __restrict__ vref,
                                                                double* __restrict__ partial)
{
    constexpr int Q = Lattice<D>::Q;
    double acc[RED_N];
    for (int k = 0; k < RED_N; ++k) acc[k] = 0.0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < p.N; n += (long long)gridDim.x * blockDim.x) {
        double e = (double)F.eps[n];
        double mass = e * (double)p.rho0;
        for (int i = 0; i < Q; ++i) mass += (double)Codec<S>::load(f + aa_slot<D>(p, i, n), p.w[i], p.inv_w[i]);
        acc[0] += mass;
        double rho = (double)F.rho[n];
        double v[3], nv2 = 0.0, d2 = 0.0, r2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            v[a] = (double)F.v[a * p.N + n];
            nv2 += v[a] * v[a];
            if (vref) {
                double r = (double)vref[a * p.N + n];
                d2 += (v[a] - r) * (v[a] - r);
                r2 += r * r;
            }
        }
        double nv = sqrt(nv2);
        double sink = rho * ((double)F.muD[n] + (double)F.muF[n] * nv);
        for (int a = 0; a < 3; ++a) {
            acc[1 + a] += v[a];
            acc[6 + a] += sink * v[a];
        }
        acc[4] += nv2;
        acc[5] += d2;
        acc[9] += r2;
    }
    block_store(acc, partial + (long long)blockIdx.x * RED_N);
}

// Pass 2: one block of RED_THREADS threads sums nblocks partials.
static __global__ void __launch_bounds__(RED_THREADS) k_reduce_final(const double* __restrict__ partial, int nblocks, double* __restrict__ out)
{
    double acc[RED_N];
    for (int k = 0; k < RED_N; ++k) acc[k] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int k = 0; k < RED_N; ++k) acc[k] += partial[(long long)b * RED_N + k];
    block_store(acc, out);
}

template <typename T>
__global__ void k_copy_v(Params<T> p, const T* v, T* vref)
{
    long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= 3 * p.N) return;
    vref[n] = v[n];
}

}  // namespace lbm
