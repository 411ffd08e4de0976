// lbm_population_sums_noalloc: FP64 mass and momentum sums of a population
// field, computed without allocating any memory (declared in include/lbm.h).
//
// It is the two-pass reduction of k_reduce_partial / k_reduce_final with its
// per-block partial sums held in a fixed device array defined in this file
// instead of a buffer the context allocates.  It serves callers that may not
// allocate: code that runs while a CUDA stream is being captured into a graph
// (allocation calls are not allowed there), and applications that hand all
// device memory to their own pool and forbid libraries to take more.
#include <cuda_runtime.h>

#include <mutex>

#include "lbm.h"

namespace {

constexpr int kThreads = 256;
constexpr int kSums = 4;  // mass, momentum x, y, z
constexpr long long kMaxBlocks = LBM_NOALLOC_MAX_NODES / kThreads;

// One partial-sum row per block of the first pass.  Every GPU that loads the
// library holds this array (2 MiB) until the process exits.  All calls share
// it; the first pass overwrites every row the second pass reads, so nothing
// has to be cleared between calls, but two calls that overlap on the GPU race.
static __device__ __align__(256) double g_partials[kMaxBlocks * kSums];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_partials_addr[kMaxDevices] = {};

__device__ __forceinline__ double warp_sum(double x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__device__ __forceinline__ void block_sums(double* acc, double* out)
{
    __shared__ double sh[kThreads / 32][kSums];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < kSums; ++k) {
        double s = warp_sum(acc[k]);
        if (lane == 0) sh[wid][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < kSums) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += sh[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// pass 1: block b sums nodes [b*256, b*256 + 256)
__global__ void __launch_bounds__(kThreads) k_sums_partial(int Q, int D, long long N, const double* __restrict__ f,
                                                           double* __restrict__ partials)
{
    double acc[kSums] = {0.0, 0.0, 0.0, 0.0};
    long long n = (long long)blockIdx.x * kThreads + threadIdx.x;
    if (n < N) {
        for (int i = 0; i < Q; ++i) {
            double fi = f[(long long)i * N + n];
            acc[0] += fi;
            acc[1] += (double)(i % 3 - 1) * fi;
            acc[2] += (double)((i / 3) % 3 - 1) * fi;
            if (D == 3) acc[3] += (double)(i / 9 - 1) * fi;
        }
    }
    block_sums(acc, partials + (long long)blockIdx.x * kSums);
}

// pass 2: one block adds the partial rows in a fixed order
__global__ void __launch_bounds__(kThreads) k_sums_final(const double* __restrict__ partials, long long nblocks,
                                                         double* __restrict__ out)
{
    double acc[kSums] = {0.0, 0.0, 0.0, 0.0};
    for (long long b = threadIdx.x; b < nblocks; b += kThreads)
        for (int k = 0; k < kSums; ++k) acc[k] += partials[b * kSums + k];
    block_sums(acc, out);
}

// Device address of g_partials on the current device.  In host code the name
// g_partials is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress.  Outside a stream capture it is looked up on every
// call (a device reset reloads the module and moves the array); while the
// stream is being captured the address cached by an earlier call is used, so
// the first call on a device must come before any capture.
int partials_address(cudaStream_t st, double** addr)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_E_CUDA;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return LBM_E_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) return LBM_E_CUDA;
        g_partials_addr[dev] = (double*)p;
    }
    if (!g_partials_addr[dev]) return LBM_E_CUDA;
    *addr = g_partials_addr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_population_sums_noalloc(int lattice, long long n_nodes, const double* f_dev, double* out_dev,
                                           void* stream)
{
    if (lattice != LBM_D2Q9 && lattice != LBM_D3Q27) return LBM_E_INVALID;
    if (!f_dev || !out_dev) return LBM_E_INVALID;
    if (n_nodes <= 0 || n_nodes > LBM_NOALLOC_MAX_NODES) return LBM_E_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    double* partials = nullptr;
    int r = partials_address(st, &partials);
    if (r) return r;
    int D = lattice == LBM_D2Q9 ? 2 : 3, Q = D == 2 ? 9 : 27;
    long long nblocks = (n_nodes + kThreads - 1) / kThreads;
    // Each launch's own status: the runtime's last-error state, which may hold
    // an error of the caller's earlier work, is neither read nor cleared here.
    const double* f = f_dev;
    int q = Q, d = D;
    long long n = n_nodes;
    void* a1[] = {&q, &d, &n, &f, &partials};
    if (cudaLaunchKernel((const void*)k_sums_partial, dim3((unsigned)nblocks), dim3(kThreads), a1, 0, st) != cudaSuccess)
        return LBM_E_CUDA;
    const double* pc = partials;
    void* a2[] = {&pc, &nblocks, &out_dev};
    if (cudaLaunchKernel((const void*)k_sums_final, dim3(1), dim3(kThreads), a2, 0, st) != cudaSuccess)
        return LBM_E_CUDA;
    return LBM_OK;
}
