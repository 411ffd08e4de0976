// Batched in-place split step for the serving runtime: one launch of each of
// the three split kernels (moments, velocity, collide) advances every case of
// a batch by one step.  A block reads its case and tile from a per-block table
// that follows the cases' table (built on the host); the arithmetic
// per node is that of the single-case in-place kernels, so a case's results do
// not depend on the other cases of the batch.  The cases are periodic D3Q27
// boxes with nx a multiple of 8 (tiled copies) that stream in place; every
// batch is an even number of steps, so all cases share the parity sequence of
// the batch's steps.
#pragma once

#include "lbm_inplace.cuh"

namespace lbm {

// One case of a batch, in device memory.  The tensor maps live here (global
// memory) and are read by the copy engine from there.
template <typename S>
struct alignas(128) BatchCase {
    CUtensorMap tm_f;    // its population array (box 64 x 4 x 1 x 9)
    CUtensorMap tm_eps;  // its padded porosity (box 72 x 6 x 3)
    Params<float> p;
    Fields<float> F;
    S* f;
    int tiles_x, tiles_y;     // 64 x 4 tiles of a plane
    int block_begin, nblocks; // its blocks in the batched grids (tiles_x tiles_y nz)
};

// The batch's blocks, one entry each, after the case table: the block's case
// and its tile in that case (one 16-byte load per block).
struct alignas(16) BatchBlock {
    int c, bx, by, bz;
};

template <typename S>
__device__ __forceinline__ BatchBlock batch_tile(const BatchCase<S>* __restrict__ cs, int n)
{
    const int4 e = __ldg(reinterpret_cast<const int4*>(cs + n) + blockIdx.x);
    return BatchBlock{e.x, e.y, e.z, e.w};
}

template <typename S, int PAR>
__global__ void __launch_bounds__(kSplitThreads) k_batch_moments(const BatchCase<S>* __restrict__ cs, int n)
{
    const BatchBlock t = batch_tile(cs, n);
    const BatchCase<S>& k = cs[t.c];
    ip_moments_pair<S, false, PAR, int>(k.p, k.F, k.f, ip_geo(k.p, t.bx, t.by, t.bz));
}

template <typename S>
__global__ void __launch_bounds__(kSplitThreads, 8) k_batch_velocity(const BatchCase<S>* __restrict__ cs, int n)
{
    const BatchBlock t = batch_tile(cs, n);
    const BatchCase<S>& k = cs[t.c];
    PairGeo G;
    if (!G.init(k.p, t.bx, t.by, t.bz)) return;
    split_velocity_pair(k.p, G, k.F.eps, k.F.kap, k.F.rho, k.F.m, k.F.v, k.F.a);
}

template <typename S, int PAR>
__global__ void __launch_bounds__(kSplitThreads, 5) k_batch_collide(const BatchCase<S>* __restrict__ cs, int n)
{
    const BatchBlock t = batch_tile(cs, n);
    const BatchCase<S>& k = cs[t.c];
    __shared__ IpSmem<S, true, kSplitBY> sm;
    ip_collide_tile<S, false, PAR, int, true>(k.p, k.F, k.f, 0, &k.tm_f, &k.tm_eps, t.bx, t.by, t.bz, sm);
}

// One step of parity `parity` for all `n` cases of the table (total_blocks
// blocks per kernel; the table holds the n cases, then total_blocks
// BatchBlock entries), enqueued on st (graph capture allowed).
template <typename S>
int batch_step(const void* table, int n, int total_blocks, int parity, cudaStream_t st)
{
    const BatchCase<S>* cs = static_cast<const BatchCase<S>*>(table);
    const dim3 blk(kSplitBX, kSplitBY);
    if (parity == 0) {
        k_batch_moments<S, 0><<<total_blocks, blk, 0, st>>>(cs, n);
        k_batch_velocity<S><<<total_blocks, blk, 0, st>>>(cs, n);
        k_batch_collide<S, 0><<<total_blocks, blk, 0, st>>>(cs, n);
    } else {
        k_batch_moments<S, 1><<<total_blocks, blk, 0, st>>>(cs, n);
        k_batch_velocity<S><<<total_blocks, blk, 0, st>>>(cs, n);
        k_batch_collide<S, 1><<<total_blocks, blk, 0, st>>>(cs, n);
    }
    return cudaGetLastError() != cudaSuccess;
}

}  // namespace lbm
