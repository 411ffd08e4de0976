// C ABI of liblbm.so (declared in include/lbm.h): context lifetime, input
// validation, device memory, stream handling and dispatch to the sweep and
// fused kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_common.cuh"
#include "lbm_fused.cuh"
#include "lbm_split.cuh"
#include "lbm_batch.cuh"

// the in-place step's and the batched step's instances live in lbm_inplace.cu
namespace lbm {
extern template int batch_step<float>(const void*, int, int, int, cudaStream_t);
extern template int batch_step<__half>(const void*, int, int, int, cudaStream_t);
extern template int batch_step<__nv_bfloat16>(const void*, int, int, int, cudaStream_t);
extern template int inplace_step<float>(const Params<float>&, const Fields<float>&, float*, int, const SplitTma&, int,
                                        cudaStream_t, KernelClock*);
extern template int inplace_step<__half>(const Params<float>&, const Fields<float>&, __half*, int, const SplitTma&,
                                         int, cudaStream_t, KernelClock*);
extern template int inplace_step<__nv_bfloat16>(const Params<float>&, const Fields<float>&, __nv_bfloat16*, int,
                                                const SplitTma&, int, cudaStream_t, KernelClock*);
}  // namespace lbm
#include "lbm_reduce.cuh"
#include "lbm_sweep.cuh"

#include <chrono>
#include <deque>

using namespace lbm;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

#define CK(call)                                                                                       \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return fail(LBM_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_));      \
    } while (0)

constexpr int TPB = 256;

inline unsigned nblocks(long long n, int tpb = TPB) { return (unsigned)((n + tpb - 1) / tpb); }

}  // namespace

struct lbm_ctx {
    int lattice = 0, D = 2, Q = 9;
    int nx = 0, ny = 0, nz = 0;
    long long N = 0;
    long long NS = 0;  // population plane stride (elements)
    lbm_params prm{};
    double forch = 0, nu_f = 0, b[3] = {0, 0, 0};
    int kernel = LBM_KERNEL_SWEEP;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<void*> allocs;
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    void* vref = nullptr;
    double* red_partial = nullptr;
    double* red_out = nullptr;
    int red_blocks = 0;
    unsigned* err_dev = nullptr;
    unsigned* err_host = nullptr;  // pinned
    int* queue_counter = nullptr;  // work-queue counter of the fused kernel
    KernelClock* kclock = nullptr; // event marks around kernels (lbm_time_kernels only)
    bool have_ref = false;
    long long steps = 0;
    Params<double> pd{};
    Params<float> pf{};
    Fields<double> Fd{};
    Fields<float> Ff{};
    FusedPlan plan{};
    float* eps_pad = nullptr;  // padded porosity of the split collide kernel's tiled copies
    SplitTma tma{};            // its tensor maps (tma.ok false: cp.async path)
    bool inplace = false;      // split kernels streaming in place (one population array)
    int parity = 0;            // layout of the stored populations (aa_slot); in-place steps flip it
    int wait_probe = 0;        // test only: the next in-place step's bounded wait must run out
    int tune_source = 0;       // tile height: 0 default or forced, 1 timed at creation, 2 from the cache
    std::vector<int> tune_tiles;      // the autotuner's candidates ...
    std::vector<double> tune_ms;      // ... and their ms per step
    void set_parity(int q)
    {
        parity = q;
        pd.aa_parity = q;
        pf.aa_parity = q;
    }

    void* dalloc(size_t bytes)
    {
        void* p = nullptr;
        if (bytes == 0) bytes = 16;
        if (prm.alloc)
            p = prm.alloc(bytes, prm.alloc_user);
        else if (cudaMalloc(&p, bytes) != cudaSuccess)
            p = nullptr;
        if (p) allocs.push_back(p);
        return p;
    }
    void release()
    {
        for (void* p : allocs) {
            if (prm.free)
                prm.free(p, prm.alloc_user);
            else
                cudaFree(p);
        }
        allocs.clear();
        if (err_host) cudaFreeHost(err_host);
        err_host = nullptr;
        if (own_stream && stream) cudaStreamDestroy(stream);
        stream = nullptr;
    }
};

namespace {

template <typename T>
Params<T>& params_of(lbm_ctx* c);
template <>
Params<double>& params_of<double>(lbm_ctx* c) { return c->pd; }
template <>
Params<float>& params_of<float>(lbm_ctx* c) { return c->pf; }
template <typename T>
Fields<T>& fields_of(lbm_ctx* c);
template <>
Fields<double>& fields_of<double>(lbm_ctx* c) { return c->Fd; }
template <>
Fields<float>& fields_of<float>(lbm_ctx* c) { return c->Ff; }

template <typename T>
void fill_params(lbm_ctx* c, Params<T>& p)
{
    const lbm_params& o = c->prm;
    p.nx = c->nx;
    p.ny = c->ny;
    p.nz = c->nz;
    p.N = c->N;
    p.NS = c->NS;
    for (int a = 0; a < 3; ++a) {
        p.wall[a] = (a < c->D) ? (o.bc[a] != LBM_BC_PERIODIC) : 0;
    }
    p.planes = o.bc[0] == LBM_BC_INFLOW_OUTFLOW;
    p.yplanes = c->D >= 2 && o.bc[1] == LBM_BC_MOVING_WALLS;
    for (int a = 0; a < 3; ++a) {
        p.wall_v[0][a] = (T)(a < c->D ? o.wall_v_low[a] : 0.0);
        p.wall_v[1][a] = (T)(a < c->D ? o.wall_v_high[a] : 0.0);
    }
    p.plane_scheme = o.plane_scheme;
    p.plane_density = o.plane_density;
    p.outlet = o.outlet;
    p.inlet_profile = o.inlet_profile;
    p.xwalls = o.bc[0] == LBM_BC_MOVING_WALLS;
    p.lid_profile = o.lid_profile;
    p.lid_delta = (T)o.lid_delta;
    p.picard_iters = (o.corrections & LBM_CORR_DELTA_NU) ? o.picard_iters : 0;
    p.picard_omega = (T)o.picard_omega;
    for (int a = 0; a < 3; ++a) p.v_in[a] = (T)(a < c->D ? o.inlet_v[a] : 0.0);
    p.rho_out = (T)o.outlet_rho;
    p.corr = o.corrections;
    p.ergun = c->forch < 0.0;
    p.RT = (T)o.RT;
    p.one_m_3RT = (T)(1.0 - 3.0 * o.RT);
    p.rho0 = (T)o.rho0;
    for (int a = 0; a < 3; ++a) p.b[a] = (T)(a < c->D ? c->b[a] : 0.0);
    double nu_eff = o.J_nu * c->nu_f;
    p.beta = (T)(1.0 / (2.0 * nu_eff / o.RT + 1.0));  // Eq. (nu_eff_def) solved for beta
    p.nu_eff = (T)nu_eff;
    p.nu_f = (T)c->nu_f;
    p.forch = (T)(c->forch < 0 ? 0.0 : c->forch);
    p.eta_coef = (T)(o.RT * (2.0 / c->D - o.J_eta / o.J_nu));
    for (int i = 0; i < 27; ++i) {
        double w = 0.0;
        if (i < c->Q) {
            // Eq. (eq_weights): w_i = prod_a Psi(c_ia; 0, RT)
            w = 1.0;
            for (int a = 0; a < c->D; ++a) {
                int ci = a == 0 ? i % 3 - 1 : a == 1 ? (i / 3) % 3 - 1 : i / 9 - 1;
                w *= ci == 0 ? 1.0 - o.RT : 0.5 * o.RT;
            }
        }
        p.w[i] = (T)w;
        p.inv_w[i] = (T)(w > 0 ? 1.0 / w : 0.0);
    }
}

// -------------------------------------------------------------- dispatch
template <int D, typename S>
struct Impl {
    using T = typename Codec<S>::T;

    static int alloc(lbm_ctx* c)
    {
        size_t N = (size_t)c->N, tb = sizeof(T);
        Fields<T>& F = fields_of<T>(c);
        T* eps = (T*)c->dalloc(N * tb);
        T* kap = (T*)c->dalloc(N * tb);
        F.eps = eps;
        F.kap = kap;
        F.muD = (T*)c->dalloc(N * tb);
        F.muF = (T*)c->dalloc(N * tb);
        F.ge = (T*)c->dalloc(3 * N * tb);
        F.H = (T*)c->dalloc(6 * N * tb);
        F.rho = (T*)c->dalloc(N * tb);
        F.v1 = (T*)c->dalloc(3 * N * tb);
        F.m = (T*)c->dalloc(3 * N * tb);
        F.v = (T*)c->dalloc(3 * N * tb);
        F.a = (T*)c->dalloc(3 * N * tb);
        c->err_dev = (unsigned*)c->dalloc(sizeof(unsigned) * 4);
        F.err = c->err_dev;
        c->queue_counter = (int*)(c->err_dev + 2);
        c->f[0] = c->dalloc((size_t)c->Q * (size_t)c->NS * sizeof(S));
        // in-place streaming keeps one population array
        c->f[1] = c->inplace ? c->f[0] : c->dalloc((size_t)c->Q * (size_t)c->NS * sizeof(S));
        c->red_blocks = (int)std::min<long long>(1024, (c->N + RED_THREADS - 1) / RED_THREADS);
        c->red_partial = (double*)c->dalloc((size_t)c->red_blocks * RED_N * sizeof(double));
        c->red_out = (double*)c->dalloc(RED_N * sizeof(double));
        for (void* p : c->allocs)
            if (!p) return fail(LBM_E_NOMEM, "device allocation failed");
        if (!eps || !kap || !F.muD || !F.muF || !F.ge || !F.H || !F.rho || !F.v1 || !F.m || !F.v || !F.a ||
            !c->err_dev || !c->f[0] || !c->f[1] || !c->red_partial || !c->red_out)
            return fail(LBM_E_NOMEM, "device allocation of %.3f GB failed",
                        (double)((c->Q * 2 * sizeof(S) + 22 * tb) * N) / 1e9);
        return LBM_OK;
    }

    static int upload_static(lbm_ctx* c, const double* eps, const double* kap)
    {
        size_t N = (size_t)c->N;
        Fields<T>& F = fields_of<T>(c);
        std::vector<T> tmp(N);
        for (size_t n = 0; n < N; ++n) tmp[n] = (T)eps[n];
        CK(cudaMemcpyAsync((void*)F.eps, tmp.data(), N * sizeof(T), cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (size_t n = 0; n < N; ++n) tmp[n] = std::isinf(kap[n]) ? (T)INFINITY : (T)kap[n];
        CK(cudaMemcpyAsync((void*)F.kap, tmp.data(), N * sizeof(T), cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemsetAsync(c->err_dev, 0, sizeof(unsigned) * 4, c->stream));
        Params<T>& p = params_of<T>(c);
        k_static_grad<D, T><<<nblocks(c->N), TPB, 0, c->stream>>>(p, F);
        k_static_hess<D, T><<<nblocks(c->N), TPB, 0, c->stream>>>(p, F);
        CK(cudaGetLastError());
        if constexpr (D == 3 && !std::is_same<S, double>::value) {
            // the split collide kernel's padded porosity and tensor maps
            if (c->kernel == LBM_KERNEL_SPLIT && c->nx % 8 == 0) {
                const long long M = (long long)(c->nx + 2 * kPadX) * (c->ny + 2) * (c->nz + 2);
                c->eps_pad = (float*)c->dalloc((size_t)M * sizeof(float));
                if (!c->eps_pad) return fail(LBM_E_NOMEM, "padded porosity allocation failed");
                k_pad_eps<<<(unsigned)std::min<long long>((M + TPB - 1) / TPB, 65535), TPB, 0, c->stream>>>(
                    c->pf, c->Ff.eps, c->eps_pad);
                CK(cudaGetLastError());
                split_tma_setup<S>(c->tma, c->pf, c->f[0], c->f[1], c->eps_pad);
            }

        }
        CK(cudaStreamSynchronize(c->stream));
        return LBM_OK;
    }

    // tensor maps of the split collide kernels for tiles of `by` rows
    static int retile(lbm_ctx* c, int by)
    {
        if constexpr (D == 3 && !std::is_same<S, double>::value) {
            if (!c->eps_pad || !split_tma_setup<S>(c->tma, c->pf, c->f[0], c->f[1], c->eps_pad, by))
                return fail(LBM_E_UNSUPPORTED, "no tensor maps for tiles of %d rows", by);
            return LBM_OK;
        } else {
            (void)c;
            (void)by;
            return fail(LBM_E_UNSUPPORTED, "tile heights apply to the D3Q27 split kernels");
        }
    }

    // initial populations from per-node (or uniform) rho0, v0 (device FP64 arrays or null)
    static int init(lbm_ctx* c, const double* rho0_dev, const double* v0_dev)
    {
        c->set_parity(0);
        Params<T>& p = params_of<T>(c);
        Fields<T>& F = fields_of<T>(c);
        k_set_initial<T><<<nblocks(c->N), TPB, 0, c->stream>>>(p, F, rho0_dev, v0_dev);
        k_velocity<D, T><<<nblocks(c->N), TPB, 0, c->stream>>>(p, F, 1);
        k_init_populations<D, S><<<nblocks(c->N), TPB, 0, c->stream>>>(p, F, (S*)c->f[c->cur]);
        CK(cudaGetLastError());
        c->set_parity(0);
        c->steps = 0;
        c->have_ref = false;
        return LBM_OK;
    }

    // S2: one-shot velocity, then the Picard iterations of Appendix F if asked
    // for (ping-pong between F.v and F.m, which is free after k_velocity)
    static void velocity(lbm_ctx* c)
    {
        Params<T>& p = params_of<T>(c);
        Fields<T>& F = fields_of<T>(c);
        k_velocity<D, T><<<nblocks(c->N), TPB, 0, c->stream>>>(p, F, 0);
        const int K = p.picard_iters;
        for (int k = 0; k < K; ++k) {
            const T* src = (k & 1) ? F.m : F.v;
            T* dst = (k & 1) ? F.v : F.m;
            k_picard<D, T><<<nblocks(c->N), TPB, 0, c->stream>>>(p, F, src, dst, k == K - 1);
        }
        if (K & 1) k_copy_v<T><<<nblocks(3 * c->N), TPB, 0, c->stream>>>(p, F.m, F.v);
    }

    static int moments(lbm_ctx* c)
    {
        Params<T>& p = params_of<T>(c);
        Fields<T>& F = fields_of<T>(c);
        k_moments<D, S><<<nblocks(c->N), TPB, 0, c->stream>>>(p, F, (const S*)c->f[c->cur]);
        velocity(c);
        CK(cudaGetLastError());
        return LBM_OK;
    }

    static int step_sweep(lbm_ctx* c, long n)
    {
        Params<T>& p = params_of<T>(c);
        Fields<T>& F = fields_of<T>(c);
        for (long k = 0; k < n; ++k) {
            k_moments<D, S><<<nblocks(c->N), TPB, 0, c->stream>>>(p, F, (const S*)c->f[c->cur]);
            velocity(c);
            k_collide_stream<D, S><<<nblocks(c->N), TPB, 0, c->stream>>>(p, F, (const S*)c->f[c->cur],
                                                                         (S*)c->f[c->cur ^ 1]);
            c->cur ^= 1;
            if (p.planes || p.yplanes || p.xwalls) planes(c);
        }
        CK(cudaGetLastError());
        return LBM_OK;
    }

    // inlet / outlet planes (x), then the corner columns where they meet
    // moving walls, then the walls (y), in stream order
    static void planes(lbm_ctx* c)
    {
        const Params<T>& p = params_of<T>(c);
        S* f = (S*)c->f[c->cur];
        if (p.planes || p.xwalls) {
            long long m = 2LL * c->ny * c->nz;
            bool done = false;
            if constexpr (D == 3 && !std::is_same<S, double>::value) {
                // the common case, one warp per plane node
                if (p.planes && !p.xwalls && p.plane_scheme == LBM_PLANES_NEEM && p.outlet == LBM_OUTLET_PRESSURE) {
                    k_planes_x_warp<S><<<(unsigned)((32 * m + 255) / 256), 256, 0, c->stream>>>(p, fields_of<T>(c), f);
                    done = true;
                }
            }
            if (!done) k_planes<D, S><<<nblocks(m), TPB, 0, c->stream>>>(p, fields_of<T>(c), f, 0);
        }
        if ((p.planes || p.xwalls) && p.yplanes)
            k_plane_corners<D, S><<<nblocks(4LL * c->nz), TPB, 0, c->stream>>>(p, fields_of<T>(c), f);
        if (p.yplanes) {
            long long m = 2LL * c->nx * c->nz;
            k_planes<D, S><<<nblocks(m), TPB, 0, c->stream>>>(p, fields_of<T>(c), f, 1);
        }
    }

    static int step(lbm_ctx* c, long n)
    {
        if (c->kernel == LBM_KERNEL_SPLIT) {
            Params<T>& p = params_of<T>(c);
            for (long k = 0; k < n; ++k) {
                if (c->inplace) {
                    if constexpr (D == 3 && !std::is_same<S, double>::value) {
                        const int probe = c->wait_probe;
                        c->wait_probe = 0;
                        if (inplace_step<S>(c->pf, c->Ff, (S*)c->f[0], c->parity, c->tma, probe, c->stream, c->kclock))
                            return fail(LBM_E_CUDA, "in-place split step: %s", cudaGetErrorString(cudaGetLastError()));
                        c->set_parity(c->parity ^ 1);
                    }
                } else if (split_step<D, S>(p, fields_of<T>(c), c->f, c->cur, c->stream, c->kclock, &c->tma))
                    return fail(LBM_E_CUDA, "split step: %s", cudaGetErrorString(cudaGetLastError()));
                if (p.planes || p.yplanes || p.xwalls) {
                    planes(c);
                    clock_mark(c->kclock, c->stream);
                }
            }
            CK(cudaGetLastError());
            return LBM_OK;
        }
        if (c->kernel == LBM_KERNEL_FUSED) {
            Params<T>& p = params_of<T>(c);
            for (long k = 0; k < n; ++k) {
                int r = fused_step<D, S>(c->plan, p, fields_of<T>(c), c->f, c->cur, 1, c->queue_counter, c->stream,
                                         c->kclock);
                if (r) return fail(LBM_E_CUDA, "fused step: %s", cudaGetErrorString(cudaGetLastError()));
                if (p.planes || p.yplanes || p.xwalls) {
                    planes(c);
                    clock_mark(c->kclock, c->stream);
                }
            }
            CK(cudaGetLastError());
            return LBM_OK;
        }
        return step_sweep(c, n);
    }

    static int export_moments(lbm_ctx* c, double* rho_dev, double* v_dev)
    {
        int r = moments(c);
        if (r) return r;
        k_export_moments<T><<<nblocks(c->N), TPB, 0, c->stream>>>(params_of<T>(c), fields_of<T>(c), rho_dev, v_dev);
        CK(cudaGetLastError());
        return LBM_OK;
    }

    static int decode(lbm_ctx* c, double* out_dev)
    {
        k_decode<D, S><<<nblocks(c->N), TPB, 0, c->stream>>>(params_of<T>(c), fields_of<T>(c), (const S*)c->f[c->cur], out_dev);
        CK(cudaGetLastError());
        return LBM_OK;
    }

    static int encode(lbm_ctx* c, const double* in_dev)
    {
        k_encode<D, S><<<nblocks(c->N), TPB, 0, c->stream>>>(params_of<T>(c), fields_of<T>(c), in_dev, (S*)c->f[c->cur]);
        CK(cudaGetLastError());
        return LBM_OK;
    }

    // porosity and permeability back to host doubles (exact: the device holds T values)
    static int read_static(lbm_ctx* c, double* eps, double* kap)
    {
        size_t N = (size_t)c->N;
        std::vector<T> tmp(N);
        Fields<T>& F = fields_of<T>(c);
        CK(cudaMemcpyAsync(tmp.data(), F.eps, N * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (size_t n = 0; n < N; ++n) eps[n] = (double)tmp[n];
        CK(cudaMemcpyAsync(tmp.data(), F.kap, N * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (size_t n = 0; n < N; ++n) kap[n] = (double)tmp[n];
        return LBM_OK;
    }

    static int reduce(lbm_ctx* c, double* host_out, int snapshot)
    {
        int r = reduce_enqueue(c, host_out, snapshot);
        if (r) return r;
        CK(cudaStreamSynchronize(c->stream));
        return LBM_OK;
    }

    // enqueues the reductions; host_out (RED_N doubles) is valid after the stream syncs
    static int reduce_enqueue(lbm_ctx* c, double* host_out, int snapshot)
    {
        int r = moments(c);
        if (r) return r;
        Params<T>& p = params_of<T>(c);
        Fields<T>& F = fields_of<T>(c);
        if (snapshot && !c->vref) {
            c->vref = c->dalloc(3 * (size_t)c->N * sizeof(T));
            if (!c->vref) return fail(LBM_E_NOMEM, "residual snapshot allocation failed");
        }
        const T* vref = c->have_ref ? (const T*)c->vref : nullptr;
        k_reduce_partial<D, S><<<c->red_blocks, RED_THREADS, 0, c->stream>>>(p, F, (const S*)c->f[c->cur], vref,
                                                                             c->red_partial);
        k_reduce_final<<<1, RED_THREADS, 0, c->stream>>>(c->red_partial, c->red_blocks, c->red_out);
        if (snapshot) {
            k_copy_v<T><<<nblocks(3 * c->N), TPB, 0, c->stream>>>(p, F.v, (T*)c->vref);
            c->have_ref = true;
        }
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(host_out, c->red_out, RED_N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        return LBM_OK;
    }
};

#define LBM_DISPATCH(c, FN, ...)                                                                  \
    ((c)->lattice == LBM_D2Q9                                                                     \
         ? ((c)->prm.storage == LBM_STORE_FP64   ? Impl<2, double>::FN(__VA_ARGS__)               \
            : (c)->prm.storage == LBM_STORE_FP32 ? Impl<2, float>::FN(__VA_ARGS__)                \
            : (c)->prm.storage == LBM_STORE_FP16 ? Impl<2, __half>::FN(__VA_ARGS__)               \
                                                 : Impl<2, __nv_bfloat16>::FN(__VA_ARGS__))       \
         : ((c)->prm.storage == LBM_STORE_FP64   ? Impl<3, double>::FN(__VA_ARGS__)               \
            : (c)->prm.storage == LBM_STORE_FP32 ? Impl<3, float>::FN(__VA_ARGS__)                \
            : (c)->prm.storage == LBM_STORE_FP16 ? Impl<3, __half>::FN(__VA_ARGS__)               \
                                                 : Impl<3, __nv_bfloat16>::FN(__VA_ARGS__)))

// ------------------------------------------------------------------ autotuner
// Tile height of the split kernels on all-periodic grids (a launch shape: the
// arithmetic of every node is the same for every height).
bool tile_tunable(const lbm_ctx* c)
{
    return c->kernel == LBM_KERNEL_SPLIT && c->lattice == LBM_D3Q27 && c->tma.ok && !c->pf.wall[0] &&
           !c->pf.wall[1] && !c->pf.wall[2] && !c->pf.planes && !c->pf.yplanes && !c->pf.xwalls && c->nx % 2 == 0 &&
           27 * c->NS < (1LL << 31);
}

// cache key: lattice, storage, streaming form, size class (ceil log2 N) and device
std::string tune_key(const lbm_ctx* c)
{
    static const char* st[] = {"fp64", "fp32", "fp16", "bf16"};
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop{};
    std::string name = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? prop.name : "unknown";
    for (char& ch : name)
        if (ch == '"' || ch == '\\' || (unsigned char)ch < 32) ch = '_';
    int cls = 0;
    while ((1LL << cls) < c->N) ++cls;
    char buf[256];
    snprintf(buf, sizeof buf, "D3Q27/%s/%s/2^%d/%s", st[c->prm.storage], c->inplace ? "in_place" : "two_arrays", cls,
             name.c_str());
    return buf;
}

// mean ms per step at tile height `by`: two steps of warm-up, then k timed
int time_tile_height(lbm_ctx* c, int by, long k, double* ms)
{
    int r = LBM_DISPATCH(c, retile, c, by);
    if (r) return r;
    r = LBM_DISPATCH(c, step, c, 2);
    if (r) return r;
    cudaEvent_t e[2];
    if (cudaEventCreate(&e[0]) != cudaSuccess) return fail(LBM_E_CUDA, "event creation failed");
    if (cudaEventCreate(&e[1]) != cudaSuccess) {
        cudaEventDestroy(e[0]);
        return fail(LBM_E_CUDA, "event creation failed");
    }
    cudaEventRecord(e[0], c->stream);
    r = LBM_DISPATCH(c, step, c, k);
    cudaEventRecord(e[1], c->stream);
    float t = 0.f;
    if (!r && (cudaEventSynchronize(e[1]) != cudaSuccess || cudaEventElapsedTime(&t, e[0], e[1]) != cudaSuccess))
        r = fail(LBM_E_CUDA, "tuning step failed: %s", cudaGetErrorString(cudaGetLastError()));
    cudaEventDestroy(e[0]);
    cudaEventDestroy(e[1]);
    *ms = t / (double)k;
    return r;
}

int choose_tile_height(lbm_ctx* c, const lbm_params& prm)
{
    c->tune_source = 0;
    if (!tile_tunable(c)) {
        if (prm.tile_y != 0 && prm.tile_y != kSplitBY)
            return fail(LBM_E_UNSUPPORTED, "tile_y applies to the split kernels on all-periodic grids with even nx");
        return LBM_OK;
    }
    if (prm.tile_y != 0) return prm.tile_y == kSplitBY ? LBM_OK : LBM_DISPATCH(c, retile, c, prm.tile_y);
    if (!prm.autotune) return LBM_OK;
    const std::string key = tune_key(c);
    if (prm.tune_cache) {
        int t = 0;
        if (lbm_tune_cache_lookup(prm.tune_cache, key.c_str(), &t) == LBM_OK && t != 0 && t <= c->ny) {
            c->tune_source = 2;
            return t == kSplitBY ? LBM_OK : LBM_DISPATCH(c, retile, c, t);
        }
    }
    // enough steps for about 4e7 node updates per candidate, an even count
    // (both layouts of in-place streaming)
    long k = (long)std::min<long long>(400, std::max<long long>(4, 40000000LL / c->N));
    k += k & 1;
    int best = kSplitBY;
    double best_ms = 0.0;
    for (int by : {2, 4, 8}) {
        if (by > c->ny) continue;
        double ms = 0.0;
        int r = time_tile_height(c, by, k, &ms);
        if (r) return r;
        c->tune_tiles.push_back(by);
        c->tune_ms.push_back(ms);
    }
    // the default height unless another is faster by more than 1 % (the spread
    // of repeated timings): a tie keeps the shape the kernels were tuned around
    for (size_t j = 0; j < c->tune_tiles.size(); ++j)
        if (c->tune_tiles[j] == kSplitBY) best_ms = c->tune_ms[j];
    for (size_t j = 0; j < c->tune_tiles.size(); ++j)
        if (best_ms == 0.0 || c->tune_ms[j] < 0.99 * best_ms) {
            best = c->tune_tiles[j];
            best_ms = c->tune_ms[j];
        }
    int r = LBM_DISPATCH(c, retile, c, best);
    if (r) return r;
    c->tune_source = 1;
    if (prm.tune_cache)
        lbm_tune_cache_store(prm.tune_cache, key.c_str(), best, (int)c->tune_tiles.size(), c->tune_tiles.data(),
                             c->tune_ms.data());
    // the timed steps moved the state: back to the initial one
    if (cudaMemsetAsync(c->err_dev, 0, sizeof(unsigned), c->stream) != cudaSuccess)
        return fail(LBM_E_CUDA, "error flag reset failed");
    *c->err_host = 0;
    return lbm_init_fields(c, nullptr, nullptr);
}

int check_error_flag(lbm_ctx* c)
{
    CK(cudaMemcpyAsync(c->err_host, c->err_dev, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (*c->err_host & ERR_DIVERGED)
        return fail(LBM_E_DIVERGED, "the simulation diverged (rho <= 0, non-finite value or |v|/eps > 0.5)");
    if (*c->err_host & ERR_WAIT_TIMEOUT)
        return fail(LBM_E_TIMEOUT, "a kernel gave up waiting for its copies into shared memory; its step is invalid");
    return LBM_OK;
}

int storage_bytes(int storage) { return storage == LBM_STORE_FP64 ? 8 : storage == LBM_STORE_FP32 ? 4 : 2; }

}  // namespace

extern "C" {

void lbm_default_params(lbm_params* p)
{
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->storage = LBM_STORE_FP32;
    p->RT = 1.0 / 3.0;
    p->J_nu = 1.0;
    p->J_eta = 1.0;
    p->corrections = LBM_CORR_FULL;
    p->rho0 = 1.0;
    p->kernel = LBM_KERNEL_AUTO;
    p->outlet_rho = 1.0;
    p->picard_omega = 1.0;
    p->plane_scheme = LBM_PLANES_NEEM;
    p->plane_density = LBM_DENSITY_CONTINUITY;
    p->outlet = LBM_OUTLET_PRESSURE;
    p->inlet_profile = LBM_INLET_UNIFORM;
    p->lid_profile = LBM_LID_UNIFORM;
    p->lid_delta = 0.1;
}

const char* lbm_last_error(void) { return g_last_error.c_str(); }

int lbm_create(lbm_ctx** out, int lattice, int nx, int ny, int nz, const double* porosity, const double* permeability,
               double forchheimer, double viscosity, const double force[3], const lbm_params* opt)
{
    g_last_error.clear();
    if (!out) return fail(LBM_E_INVALID, "out is NULL");
    *out = nullptr;
    if (lattice != LBM_D2Q9 && lattice != LBM_D3Q27) return fail(LBM_E_INVALID, "unknown lattice %d", lattice);
    if (!porosity || !permeability || !force) return fail(LBM_E_INVALID, "NULL input array");
    lbm_params prm;
    lbm_default_params(&prm);
    if (opt) prm = *opt;
    if (prm.storage < LBM_STORE_FP64 || prm.storage > LBM_STORE_BF16)
        return fail(LBM_E_INVALID, "unknown storage %d", prm.storage);
    if (!(prm.RT > 0.0 && prm.RT < 1.0)) return fail(LBM_E_INVALID, "RT must lie in (0, 1)");
    if (!(prm.J_nu > 0.0) || !(prm.J_eta >= 0.0)) return fail(LBM_E_INVALID, "J_nu must be > 0 and J_eta >= 0");
    if (!(viscosity > 0.0) || !std::isfinite(viscosity)) return fail(LBM_E_INVALID, "viscosity must be > 0");
    if (std::isnan(forchheimer)) return fail(LBM_E_INVALID, "forchheimer is NaN");
    if (!(prm.rho0 > 0.0)) return fail(LBM_E_INVALID, "rho0 must be > 0");
    if ((prm.alloc == nullptr) != (prm.free == nullptr)) return fail(LBM_E_INVALID, "alloc and free must be set together");
    if (prm.corrections < 0 || prm.corrections > LBM_CORR_FULL) return fail(LBM_E_INVALID, "bad corrections mask");
    if (prm.tile_y != 0 && !tile_height_ok(prm.tile_y)) return fail(LBM_E_INVALID, "tile_y must be 0, 2, 4 or 8");
    int D = lattice == LBM_D2Q9 ? 2 : 3;
    if (D == 2 && nz != 1) return fail(LBM_E_INVALID, "D2Q9 needs nz = 1");
    int dims[3] = {nx, ny, nz};
    for (int a = 0; a < D; ++a) {
        if (prm.bc[a] != LBM_BC_PERIODIC && prm.bc[a] != LBM_BC_WALL && !(a == 0 && prm.bc[a] == LBM_BC_INFLOW_OUTFLOW) &&
            !(a <= 1 && prm.bc[a] == LBM_BC_MOVING_WALLS))
            return fail(LBM_E_INVALID, "unknown boundary %d on axis %d", prm.bc[a], a);
        int need = prm.bc[a] == LBM_BC_PERIODIC ? 3 : prm.bc[a] == LBM_BC_WALL ? 4 : 6;
        if (dims[a] < need) return fail(LBM_E_INVALID, "axis %d has %d nodes, needs >= %d", a, dims[a], need);
    }
    long long N = (long long)nx * ny * nz;
    if (N > (1LL << 40)) return fail(LBM_E_INVALID, "grid too large");
    if ((long long)nx * ny >= (1LL << 31)) return fail(LBM_E_INVALID, "an x-y plane must hold fewer than 2^31 nodes");
    for (long long n = 0; n < N; ++n) {
        double e = porosity[n], k = permeability[n];
        if (!(e > 0.0 && e <= 1.0)) return fail(LBM_E_INVALID, "porosity[%lld] = %g outside (0, 1]", n, e);
        if (!(k > 0.0)) return fail(LBM_E_INVALID, "permeability[%lld] = %g must be > 0 or +inf", n, k);
    }
    if (prm.bc[0] == LBM_BC_INFLOW_OUTFLOW) {
        if (!(prm.outlet_rho > 0.0)) return fail(LBM_E_INVALID, "outlet_rho must be > 0");
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(prm.inlet_v[a])) return fail(LBM_E_INVALID, "inlet_v is not finite");
        // uniform porosity / permeability over three layers at each plane, free fluid at the outlet
        for (long long n = 0; n < N; ++n) {
            int x = (int)(n % nx);
            int side = x <= 2 ? 0 : (x >= nx - 3 ? 1 : -1);
            if (side < 0) continue;
            long long r = side == 0 ? 0 : nx - 1;
            if (porosity[n] != porosity[r] || permeability[n] != permeability[r])
                return fail(LBM_E_UNSUPPORTED, "inlet/outlet planes need uniform porosity and permeability over 3 layers");
            if (side == 1 && !std::isinf(permeability[n]))
                return fail(LBM_E_UNSUPPORTED, "the outlet layers must be free fluid (permeability +inf)");
        }
    }
    if (prm.outlet != LBM_OUTLET_PRESSURE && prm.outlet != LBM_OUTLET_ZERO_GRADIENT)
        return fail(LBM_E_INVALID, "unknown outlet %d", prm.outlet);
    if (prm.inlet_profile != LBM_INLET_UNIFORM && prm.inlet_profile != LBM_INLET_POISEUILLE)
        return fail(LBM_E_INVALID, "unknown inlet profile %d", prm.inlet_profile);
    if ((prm.outlet != LBM_OUTLET_PRESSURE || prm.inlet_profile != LBM_INLET_UNIFORM) &&
        prm.bc[0] != LBM_BC_INFLOW_OUTFLOW)
        return fail(LBM_E_INVALID, "outlet and inlet_profile belong to LBM_BC_INFLOW_OUTFLOW");
    if (prm.inlet_profile == LBM_INLET_POISEUILLE && prm.bc[1] != LBM_BC_WALL && prm.bc[1] != LBM_BC_MOVING_WALLS)
        return fail(LBM_E_INVALID, "the Poiseuille inlet profile spans walls on y");
    if (prm.lid_profile != LBM_LID_UNIFORM && prm.lid_profile != LBM_LID_REGULARISED)
        return fail(LBM_E_INVALID, "unknown lid profile %d", prm.lid_profile);
    if (prm.lid_profile == LBM_LID_REGULARISED &&
        (prm.bc[0] != LBM_BC_MOVING_WALLS || prm.bc[1] != LBM_BC_MOVING_WALLS || !(prm.lid_delta > 0.0 && prm.lid_delta <= 0.5)))
        return fail(LBM_E_INVALID, "the regularised lid needs wet walls on x and y and lid_delta in (0, 0.5]");
    if (prm.bc[0] == LBM_BC_MOVING_WALLS) {
        if ((prm.bc[1] != LBM_BC_PERIODIC && prm.bc[1] != LBM_BC_MOVING_WALLS) || (D == 3 && prm.bc[2] != LBM_BC_PERIODIC))
            return fail(LBM_E_UNSUPPORTED, "wet side walls on x need y periodic or wet walls and z periodic");
        for (long long n = 0; n < N; ++n) {
            int x = (int)(n % nx);
            int side = x <= 2 ? 0 : (x >= nx - 3 ? 1 : -1);
            if (side < 0) continue;
            long long r = side == 0 ? 0 : nx - 1;
            if (porosity[n] != porosity[r] || permeability[n] != permeability[r])
                return fail(LBM_E_UNSUPPORTED, "wet side walls need uniform porosity and permeability over 3 layers");
        }
    }
    if (prm.bc[1] == LBM_BC_MOVING_WALLS) {
        if (prm.bc[0] == LBM_BC_WALL || (D == 3 && prm.bc[2] != LBM_BC_PERIODIC))
            return fail(LBM_E_UNSUPPORTED, "moving walls need a periodic z axis and a periodic, inflow/outflow or "
                                           "wet-wall x axis");
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(prm.wall_v_low[a]) || !std::isfinite(prm.wall_v_high[a]))
                return fail(LBM_E_INVALID, "wall velocities must be finite");
        if (prm.wall_v_low[1] != 0.0 || prm.wall_v_high[1] != 0.0)
            return fail(LBM_E_INVALID, "moving walls move tangentially (normal velocity 0)");
        // uniform porosity / permeability over three layers at each wall
        for (long long n = 0; n < N; ++n) {
            int y = (int)((n / nx) % ny);
            int side = y <= 2 ? 0 : (y >= ny - 3 ? 1 : -1);
            if (side < 0) continue;
            long long r = side == 0 ? 0 : (long long)nx * (ny - 1);
            if (porosity[n] != porosity[r] || permeability[n] != permeability[r])
                return fail(LBM_E_UNSUPPORTED, "moving walls need uniform porosity and permeability over 3 layers");
        }
    }
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(force[a])) return fail(LBM_E_INVALID, "force is not finite");
    if (prm.picard_iters < 0 || prm.picard_iters > 1000) return fail(LBM_E_INVALID, "picard_iters must be in [0, 1000]");
    if (prm.picard_iters > 0 && !(prm.picard_omega > 0.0 && prm.picard_omega <= 1.0))
        return fail(LBM_E_INVALID, "picard_omega must be in (0, 1]");
    if (prm.plane_scheme < LBM_PLANES_NEEM || prm.plane_scheme > LBM_PLANES_TMS)
        return fail(LBM_E_INVALID, "unknown plane scheme %d", prm.plane_scheme);
    if (prm.plane_density != LBM_DENSITY_CONTINUITY && prm.plane_density != LBM_DENSITY_BOUNCE_BACK)
        return fail(LBM_E_INVALID, "unknown plane density %d", prm.plane_density);
    if (prm.streaming < LBM_STREAM_AUTO || prm.streaming > LBM_STREAM_IN_PLACE)
        return fail(LBM_E_INVALID, "unknown streaming %d", prm.streaming);
    int kernel = prm.kernel;
    bool fused_ok = fused_supported(lattice, prm.storage) && prm.picard_iters == 0;
    if (kernel == LBM_KERNEL_FUSED && !fused_ok)
        return fail(LBM_E_UNSUPPORTED,
                    "the fused kernel is built for D3Q27 with FP32/FP16/BF16 storage and the one-shot velocity");
    bool split_ok = split_supported(lattice, prm.storage, nx, ny, nz);
    if (kernel == LBM_KERNEL_SPLIT && !split_ok)
        return fail(LBM_E_UNSUPPORTED, "the split kernels are built for D3Q27 with FP32/FP16/BF16 storage, fewer "
                                       "than 2^31 nodes and nz <= 65535");
    if (kernel == LBM_KERNEL_AUTO)
        kernel = split_ok ? LBM_KERNEL_SPLIT : fused_ok ? LBM_KERNEL_FUSED : LBM_KERNEL_SWEEP;
    if (kernel != LBM_KERNEL_SWEEP && kernel != LBM_KERNEL_FUSED && kernel != LBM_KERNEL_SPLIT)
        return fail(LBM_E_INVALID, "unknown kernel %d", kernel);

    lbm_ctx* c = new lbm_ctx();
    c->lattice = lattice;
    c->D = D;
    c->Q = D == 2 ? 9 : 27;
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->N = N;
    c->NS = pop_stride(N, storage_bytes(prm.storage));
    c->prm = prm;
    c->forch = forchheimer;
    c->nu_f = viscosity;
    for (int a = 0; a < 3; ++a) c->b[a] = force[a];
    c->kernel = kernel;
    c->wait_probe = prm.wait_probe != 0;
    auto bail = [&](int r) {
        c->release();
        delete c;
        return r;
    };
    if (cudaSetDevice(prm.device) != cudaSuccess) return bail(fail(LBM_E_CUDA, "cudaSetDevice(%d) failed", prm.device));
    {
        const bool ip_ok = kernel == LBM_KERNEL_SPLIT && inplace_supported(lattice, prm.storage, nx, ny, nz);
        if (prm.streaming == LBM_STREAM_IN_PLACE && !ip_ok)
            return bail(fail(LBM_E_UNSUPPORTED, "in-place streaming is built for the split kernels with nx even"));
        if (prm.streaming == LBM_STREAM_IN_PLACE) {
            c->inplace = true;
        } else if (prm.streaming == LBM_STREAM_AUTO && ip_ok) {
            size_t free_b = 0, total_b = 0;
            if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return bail(fail(LBM_E_CUDA, "cudaMemGetInfo failed"));
            const double two = 2.0 * c->Q * (double)c->NS * storage_bytes(prm.storage);
            c->inplace = two > 0.5 * (double)free_b;
        }
    }
    if (prm.stream) {
        c->stream = (cudaStream_t)prm.stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(fail(LBM_E_CUDA, "stream creation failed"));
        c->own_stream = true;
    }
    if (cudaMallocHost((void**)&c->err_host, sizeof(unsigned)) != cudaSuccess)
        return bail(fail(LBM_E_CUDA, "pinned allocation failed"));
    *c->err_host = 0;  // pinned memory is not zeroed by the allocator
    fill_params(c, c->pd);
    fill_params(c, c->pf);
    int r = LBM_DISPATCH(c, alloc, c);
    if (r) return bail(r);
    r = LBM_DISPATCH(c, upload_static, c, porosity, permeability);
    if (r) return bail(r);
    if (kernel == LBM_KERNEL_FUSED) {
        r = fused_plan(c->plan, lattice, nx, ny, nz, prm.storage, c->pf.wall);
        if (r) return bail(fail(LBM_E_UNSUPPORTED, "no fused launch plan for this grid"));
    }
    r = lbm_init_fields(c, nullptr, nullptr);
    if (r) return bail(r);
    r = choose_tile_height(c, prm);
    if (r) return bail(r);
    c->prm.tune_cache = nullptr;  // the caller's string; read during creation only
    *out = c;
    return LBM_OK;
}

int lbm_init_fields(lbm_ctx* c, const double* rho0, const double* v0)
{
    if (!c) return fail(LBM_E_INVALID, "ctx is NULL");
    size_t N = (size_t)c->N;
    double* buf = nullptr;
    if (cudaMalloc((void**)&buf, 4 * N * sizeof(double)) != cudaSuccess)
        return fail(LBM_E_NOMEM, "initial-field staging allocation failed");
    double* rdev = buf;
    double* vdev = buf + N;
    int r = LBM_OK;
    do {
        if (rho0) {
            if (cudaMemcpyAsync(rdev, rho0, N * sizeof(double), cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
                r = fail(LBM_E_CUDA, "copy of rho0 failed");
                break;
            }
        }
        if (v0) {
            if (cudaMemcpyAsync(vdev, v0, 3 * N * sizeof(double), cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
                r = fail(LBM_E_CUDA, "copy of v0 failed");
                break;
            }
        } else {
            k_fill_v0<double><<<nblocks(c->N), TPB, 0, c->stream>>>(c->pd, vdev, c->prm.v0[0], c->prm.v0[1],
                                                                     c->D == 3 ? c->prm.v0[2] : 0.0);
        }
        r = LBM_DISPATCH(c, init, c, rho0 ? rdev : nullptr, vdev);
        if (r) break;
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) r = fail(LBM_E_CUDA, "initialisation failed");
    } while (0);
    cudaFree(buf);
    return r;
}

int lbm_step(lbm_ctx* c, long n)
{
    if (!c) return fail(LBM_E_INVALID, "ctx is NULL");
    if (n < 0) return fail(LBM_E_INVALID, "negative step count");
    if (*c->err_host & ERR_DIVERGED) return fail(LBM_E_DIVERGED, "the simulation diverged earlier");
    if (*c->err_host & ERR_WAIT_TIMEOUT) return fail(LBM_E_TIMEOUT, "a kernel timed out earlier; the state is invalid");
    if (n == 0) return LBM_OK;
    int r = LBM_DISPATCH(c, step, c, n);
    if (r) return r;
    c->steps += n;
    return LBM_OK;
}

int lbm_sync(lbm_ctx* c)
{
    if (!c) return fail(LBM_E_INVALID, "ctx is NULL");
    return check_error_flag(c);
}

int lbm_moments_device(lbm_ctx* c, double* rho_dev, double* v_dev)
{
    if (!c) return fail(LBM_E_INVALID, "ctx is NULL");
    return LBM_DISPATCH(c, export_moments, c, rho_dev, v_dev);
}

int lbm_moments(lbm_ctx* c, double* rho, double* v)
{
    if (!c) return fail(LBM_E_INVALID, "ctx is NULL");
    size_t N = (size_t)c->N;
    double* buf = nullptr;
    if (cudaMalloc((void**)&buf, 4 * N * sizeof(double)) != cudaSuccess) return fail(LBM_E_NOMEM, "staging allocation failed");
    int r = LBM_DISPATCH(c, export_moments, c, buf, buf + N);
    if (!r && rho && cudaMemcpyAsync(rho, buf, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        r = fail(LBM_E_CUDA, "copy of rho failed");
    if (!r && v && cudaMemcpyAsync(v, buf + N, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        r = fail(LBM_E_CUDA, "copy of v failed");
    if (!r && cudaStreamSynchronize(c->stream) != cudaSuccess) r = fail(LBM_E_CUDA, "moments failed");
    cudaFree(buf);
    if (!r) r = check_error_flag(c);
    return r;
}

int lbm_get_populations(lbm_ctx* c, double* f)
{
    if (!c || !f) return fail(LBM_E_INVALID, "NULL argument");
    size_t bytes = (size_t)c->Q * c->N * sizeof(double);
    double* buf = nullptr;
    if (cudaMalloc((void**)&buf, bytes) != cudaSuccess) return fail(LBM_E_NOMEM, "staging allocation failed");
    int r = LBM_DISPATCH(c, decode, c, buf);
    if (!r && cudaMemcpyAsync(f, buf, bytes, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
        r = fail(LBM_E_CUDA, "copy failed");
    if (!r && cudaStreamSynchronize(c->stream) != cudaSuccess) r = fail(LBM_E_CUDA, "decode failed");
    cudaFree(buf);
    return r;
}

int lbm_set_populations(lbm_ctx* c, const double* f)
{
    if (!c || !f) return fail(LBM_E_INVALID, "NULL argument");
    size_t bytes = (size_t)c->Q * c->N * sizeof(double);
    double* buf = nullptr;
    if (cudaMalloc((void**)&buf, bytes) != cudaSuccess) return fail(LBM_E_NOMEM, "staging allocation failed");
    int r = LBM_OK;
    if (cudaMemcpyAsync(buf, f, bytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) r = fail(LBM_E_CUDA, "copy failed");
    if (!r) r = LBM_DISPATCH(c, encode, c, buf);
    if (!r && cudaStreamSynchronize(c->stream) != cudaSuccess) r = fail(LBM_E_CUDA, "encode failed");
    cudaFree(buf);
    c->have_ref = false;
    return r;
}

int lbm_reduce(lbm_ctx* c, lbm_stats* st, int snapshot)
{
    if (!c || !st) return fail(LBM_E_INVALID, "NULL argument");
    double q[RED_N];
    bool had_ref = c->have_ref;
    int r = LBM_DISPATCH(c, reduce, c, q, snapshot);
    if (r) return r;
    double N = (double)c->N;
    memset(st, 0, sizeof *st);
    st->mass = q[0];
    for (int a = 0; a < 3; ++a) {
        st->mean_v[a] = q[1 + a] / N;
        st->drag[a] = q[6 + a];
        st->k_app[a] = c->b[a] != 0.0 ? c->nu_f * st->mean_v[a] / c->b[a] : 0.0;
    }
    st->v2_sum = q[4];
    st->dv2_sum = had_ref ? q[5] : 0.0;
    st->residual = had_ref && q[9] > 0 ? std::sqrt(q[5] / q[9]) : (had_ref ? 0.0 : INFINITY);
    st->steps = c->steps;
    return check_error_flag(c);
}

int lbm_time_kernels(lbm_ctx* c, long n, double* ms_per_launch, int max_kernels, int* kernels)
{
    if (!c || !ms_per_launch || !kernels || max_kernels < 1) return fail(LBM_E_INVALID, "NULL argument");
    if (n < 1 || n > 100000) return fail(LBM_E_INVALID, "n must be in [1, 100000]");
    if (c->kernel != LBM_KERNEL_SPLIT && c->kernel != LBM_KERNEL_FUSED)
        return fail(LBM_E_UNSUPPORTED, "kernel timing covers the fused and split kernels only");
    const int per_step = (c->kernel == LBM_KERNEL_SPLIT ? 3 : 1) + (c->pf.planes || c->pf.yplanes || c->pf.xwalls ? 1 : 0);
    const int marks = per_step + 1;
    std::vector<cudaEvent_t> ev((size_t)n * marks);
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            e = nullptr;
            for (auto& x : ev)
                if (x) cudaEventDestroy(x);
            return fail(LBM_E_CUDA, "event creation failed");
        }
    KernelClock kc;
    kc.ev = ev.data();
    kc.cap = (int)ev.size();
    c->kclock = &kc;
    int r = lbm_step(c, n);
    c->kclock = nullptr;
    if (!r && (kc.n != (int)ev.size() || cudaStreamSynchronize(c->stream) != cudaSuccess))
        r = fail(LBM_E_CUDA, "kernel timing: %d of %zu events recorded", kc.n, ev.size());
    if (!r) {
        for (int k = 0; k < per_step && k < max_kernels; ++k) {
            double sum = 0.0;
            for (long s = 0; s < n; ++s) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, ev[(size_t)s * marks + k], ev[(size_t)s * marks + k + 1]);
                sum += ms;
            }
            ms_per_launch[k] = sum / (double)n;
        }
        *kernels = per_step;
    }
    for (auto& e : ev) cudaEventDestroy(e);
    return r;
}

int lbm_info(const lbm_ctx* c, double* bytes_per_node_update, int* launches_per_step, int* kernel_in_use,
             int* in_place)
{
    if (!c) return fail(LBM_E_INVALID, "ctx is NULL");
    int sb = storage_bytes(c->prm.storage);
    int tb = c->prm.storage == LBM_STORE_FP64 ? 8 : 4;
    if (bytes_per_node_update) *bytes_per_node_update = 2.0 * c->Q * sb + 2.0 * tb;
    if (launches_per_step) {
        // the step's kernels, then the wet-node rebuilds after it
        const Params<float>& pf = c->pf;
        const bool wall = pf.wall[0] || pf.wall[1] || pf.wall[2];
        int k = c->kernel == LBM_KERNEL_FUSED ? 1 : 3 + pf.picard_iters;
        // the face nodes of the split velocity kernel
        if (c->kernel == LBM_KERNEL_SPLIT && c->D == 3 && c->prm.storage != LBM_STORE_FP64 && wall && c->nx % 2 == 0)
            k += 1;
        const bool xside = pf.planes || pf.xwalls;
        k += (xside ? 1 : 0) + (xside && pf.yplanes ? 1 : 0) + (pf.yplanes ? 1 : 0);
        *launches_per_step = k;
    }
    if (kernel_in_use) *kernel_in_use = c->kernel;
    if (in_place) *in_place = c->inplace ? 1 : 0;
    return LBM_OK;
}

int lbm_tuning(const lbm_ctx* c, int* tile_y, int* n, int* tiles, double* ms, int* source)
{
    if (!c) return fail(LBM_E_INVALID, "ctx is NULL");
    if (tile_y) *tile_y = split_tile_height(c->pf, &c->tma, !tile_tunable(c));
    const int k = (int)std::min<size_t>(8, c->tune_tiles.size());
    if (n) *n = k;
    for (int j = 0; j < k; ++j) {
        if (tiles) tiles[j] = c->tune_tiles[j];
        if (ms) ms[j] = c->tune_ms[j];
    }
    if (source) *source = c->tune_source;
    return LBM_OK;
}

namespace {
bool tune_key_ok(const char* key)
{
    if (!key || !*key) return false;
    for (const char* q = key; *q; ++q)
        if (*q == '"' || *q == '\\' || (unsigned char)*q < 32) return false;
    return true;
}
}  // namespace

int lbm_tune_cache_lookup(const char* path, const char* key, int* tile_y)
{
    if (!path || !tile_y || !tune_key_ok(key)) return fail(LBM_E_INVALID, "bad cache lookup arguments");
    *tile_y = 0;
    FILE* fp = fopen(path, "r");
    if (!fp) return LBM_OK;
    const std::string want = std::string("\"key\": \"") + key + "\"";
    std::string line;
    int ch;
    auto take = [&]() {
        const size_t k = line.find(want);
        const size_t t = line.find("\"tile_y\":");
        int v = 0;
        if (k != std::string::npos && t != std::string::npos && sscanf(line.c_str() + t + 9, " %d", &v) == 1 &&
            tile_height_ok(v))
            *tile_y = v;
        line.clear();
    };
    while ((ch = fgetc(fp)) != EOF) {
        if (ch == '\n')
            take();
        else
            line.push_back((char)ch);
    }
    take();
    fclose(fp);
    return LBM_OK;
}

int lbm_tune_cache_store(const char* path, const char* key, int tile_y, int n, const int* tiles, const double* ms)
{
    if (!path || !tune_key_ok(key) || !tile_height_ok(tile_y) || n < 0 || n > 8 || (n > 0 && (!tiles || !ms)))
        return fail(LBM_E_INVALID, "bad cache store arguments");
    FILE* fp = fopen(path, "a");
    if (!fp) return fail(LBM_E_INVALID, "cannot append to %s", path);
    fprintf(fp, "{\"key\": \"%s\", \"tile_y\": %d, \"candidates\": [", key, tile_y);
    for (int j = 0; j < n; ++j) fprintf(fp, "%s%d", j ? ", " : "", tiles[j]);
    fprintf(fp, "], \"ms_per_step\": [");
    for (int j = 0; j < n; ++j) fprintf(fp, "%s%.6g", j ? ", " : "", ms[j]);
    fprintf(fp, "]}\n");
    fclose(fp);
    return LBM_OK;
}

// ------------------------------------------------------------------ checkpoint
namespace {
const char kMagic[8] = {'P', 'L', 'B', 'M', 'C', 'K', '0', '6'};
struct CkptHeader {
    char magic[8];
    int lattice, nx, ny, nz, storage, kernel, corrections, bc[3];
    double RT, J_nu, J_eta, rho0, v0[3], inlet_v[3], outlet_rho, forch, nu_f, b[3];
    long long steps;
    long long pop_bytes;
    int picard_iters;
    double picard_omega;
    int plane_scheme;
    double wall_v_low[3], wall_v_high[3];
    int plane_density;
    int outlet, inlet_profile;
    int lid_profile;
    double lid_delta;
    int aa_parity;  // layout of the raw populations (in-place streaming)
    int in_place;   // the context streamed in place
};

// Copies the current population buffer to or from a dense host image of
// Q planes of N values (one copy per plane: the device planes are NS apart).
int copy_planes(lbm_ctx* c, void* host, cudaMemcpyKind kind)
{
    const size_t sb = (size_t)storage_bytes(c->prm.storage), plane = (size_t)c->N * sb;
    char* dev = (char*)c->f[c->cur];
    char* h = (char*)host;
    for (int i = 0; i < c->Q; ++i) {
        char* d = dev + (size_t)i * (size_t)c->NS * sb;
        cudaError_t e = kind == cudaMemcpyDeviceToHost
                            ? cudaMemcpyAsync(h + i * plane, d, plane, kind, c->stream)
                            : cudaMemcpyAsync(d, h + i * plane, plane, kind, c->stream);
        if (e != cudaSuccess) return 1;
    }
    return cudaStreamSynchronize(c->stream) != cudaSuccess;
}
}  // namespace

int lbm_save(const lbm_ctx* cc, const char* path)
{
    lbm_ctx* c = const_cast<lbm_ctx*>(cc);
    if (!c || !path) return fail(LBM_E_INVALID, "NULL argument");
    CkptHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, kMagic, 8);
    h.lattice = c->lattice;
    h.nx = c->nx;
    h.ny = c->ny;
    h.nz = c->nz;
    h.storage = c->prm.storage;
    h.kernel = c->kernel;
    h.corrections = c->prm.corrections;
    for (int a = 0; a < 3; ++a) {
        h.bc[a] = c->prm.bc[a];
        h.v0[a] = c->prm.v0[a];
        h.inlet_v[a] = c->prm.inlet_v[a];
        h.b[a] = c->b[a];
    }
    h.RT = c->prm.RT;
    h.J_nu = c->prm.J_nu;
    h.J_eta = c->prm.J_eta;
    h.rho0 = c->prm.rho0;
    h.outlet_rho = c->prm.outlet_rho;
    h.forch = c->forch;
    h.nu_f = c->nu_f;
    h.steps = c->steps;
    h.picard_iters = c->prm.picard_iters;
    h.picard_omega = c->prm.picard_omega;
    h.plane_scheme = c->prm.plane_scheme;
    h.plane_density = c->prm.plane_density;
    h.outlet = c->prm.outlet;
    h.inlet_profile = c->prm.inlet_profile;
    h.lid_profile = c->prm.lid_profile;
    h.lid_delta = c->prm.lid_delta;
    h.aa_parity = c->parity;
    h.in_place = c->inplace ? 1 : 0;
    for (int a = 0; a < 3; ++a) {
        h.wall_v_low[a] = c->prm.wall_v_low[a];
        h.wall_v_high[a] = c->prm.wall_v_high[a];
    }
    h.pop_bytes = (long long)c->Q * c->N * storage_bytes(c->prm.storage);
    size_t N = (size_t)c->N;
    std::vector<double> eps(N), kap(N);
    int r = LBM_DISPATCH(c, read_static, c, eps.data(), kap.data());
    if (r) return r;
    std::vector<char> pop((size_t)h.pop_bytes);
    if (copy_planes(c, pop.data(), cudaMemcpyDeviceToHost)) return fail(LBM_E_CUDA, "population copy failed");
    FILE* fp = fopen(path, "wb");
    if (!fp) return fail(LBM_E_INVALID, "cannot open %s for writing", path);
    bool ok = fwrite(&h, sizeof h, 1, fp) == 1 && fwrite(eps.data(), sizeof(double), N, fp) == N &&
              fwrite(kap.data(), sizeof(double), N, fp) == N && fwrite(pop.data(), 1, pop.size(), fp) == pop.size();
    ok = (fclose(fp) == 0) && ok;
    return ok ? LBM_OK : fail(LBM_E_INVALID, "write to %s failed", path);
}

int lbm_load(lbm_ctx** out, const char* path, const lbm_params* runtime)
{
    if (!out || !path) return fail(LBM_E_INVALID, "NULL argument");
    *out = nullptr;
    FILE* fp = fopen(path, "rb");
    if (!fp) return fail(LBM_E_INVALID, "cannot open %s", path);
    CkptHeader h;
    bool ok = fread(&h, sizeof h, 1, fp) == 1 && memcmp(h.magic, kMagic, 8) == 0;
    long long N = ok ? (long long)h.nx * h.ny * h.nz : 0;
    ok = ok && N > 0 && h.pop_bytes == (long long)(h.lattice == LBM_D2Q9 ? 9 : 27) * N * storage_bytes(h.storage);
    std::vector<double> eps, kap;
    std::vector<char> pop;
    if (ok) {
        eps.resize((size_t)N);
        kap.resize((size_t)N);
        pop.resize((size_t)h.pop_bytes);
        ok = fread(eps.data(), sizeof(double), (size_t)N, fp) == (size_t)N &&
             fread(kap.data(), sizeof(double), (size_t)N, fp) == (size_t)N &&
             fread(pop.data(), 1, pop.size(), fp) == pop.size();
    }
    fclose(fp);
    if (!ok) return fail(LBM_E_INVALID, "%s is not a valid checkpoint", path);
    lbm_params prm;
    lbm_default_params(&prm);
    if (runtime) {
        prm.stream = runtime->stream;
        prm.device = runtime->device;
        prm.alloc = runtime->alloc;
        prm.free = runtime->free;
        prm.alloc_user = runtime->alloc_user;
    }
    prm.storage = h.storage;
    prm.kernel = h.kernel;
    prm.corrections = h.corrections;
    for (int a = 0; a < 3; ++a) {
        prm.bc[a] = h.bc[a];
        prm.v0[a] = h.v0[a];
        prm.inlet_v[a] = h.inlet_v[a];
    }
    prm.RT = h.RT;
    prm.J_nu = h.J_nu;
    prm.J_eta = h.J_eta;
    prm.rho0 = h.rho0;
    prm.outlet_rho = h.outlet_rho;
    prm.picard_iters = h.picard_iters;
    prm.picard_omega = h.picard_omega;
    prm.plane_scheme = h.plane_scheme;
    prm.plane_density = h.plane_density;
    prm.outlet = h.outlet;
    prm.inlet_profile = h.inlet_profile;
    prm.lid_profile = h.lid_profile;
    prm.lid_delta = h.lid_delta;
    prm.streaming = h.in_place ? LBM_STREAM_IN_PLACE : LBM_STREAM_TWO_ARRAYS;
    for (int a = 0; a < 3; ++a) {
        prm.wall_v_low[a] = h.wall_v_low[a];
        prm.wall_v_high[a] = h.wall_v_high[a];
    }
    lbm_ctx* c = nullptr;
    int r = lbm_create(&c, h.lattice, h.nx, h.ny, h.nz, eps.data(), kap.data(), h.forch, h.nu_f, h.b, &prm);
    if (r) return r;
    if (copy_planes(c, pop.data(), cudaMemcpyHostToDevice)) {
        lbm_destroy(c);
        return fail(LBM_E_CUDA, "population upload failed");
    }
    c->steps = h.steps;
    if (h.aa_parity != 0 && !c->inplace) {
        lbm_destroy(c);
        return fail(LBM_E_INVALID, "%s holds in-place populations that only the in-place split kernels read", path);
    }
    c->set_parity(h.aa_parity);
    *out = c;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx* c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    c->release();
    delete c;
}

}  // extern "C"

// ==================================================================== serving
// Continuous-batching server: requests (independent D3Q27 cases of any size)
// are queued on submission, admitted in arrival order while their device
// footprint fits under the HBM cap, advanced together by one launch of each
// of the three in-place split kernels per step over all admitted cases (the
// steps of a batch captured in one CUDA graph), checked for steady state
// after every batch and retired as soon as they converge, which frees memory
// for the next queued requests.

namespace {

struct PendingCase {
    long long id;
    int nx, ny, nz;
    std::vector<double> eps, kap;
    double forch, visc, b[3], tol;
    long max_steps;
    double submit_time;
};

struct ActiveCase {
    long long id;
    lbm_ctx* ctx;
    double bytes;
    double tol, b[3];
    long max_steps;
    double submit_time;
    double* red;  // pinned: RED_N doubles of reductions, then the error flag
    std::vector<double> history;  // residual after each batch
    std::vector<double> mean_along_b;  // mean superficial velocity along the force after each batch
};

}  // namespace

struct lbm_server {
    int storage = LBM_STORE_FP16;
    double cap = 0, used = 0;
    int check_every = 100;
    lbm_params defaults{};
    cudaStream_t stream = nullptr;
    std::deque<PendingCase> queue;
    std::vector<ActiveCase> active;
    long long next_id = 1;
    std::chrono::steady_clock::time_point t0;
    void* table_dev = nullptr;
    size_t table_cap = 0;
    void* table_host = nullptr;  // pinned
    cudaGraphExec_t graph = nullptr;
    bool graph_valid = false;
    int total_blocks = 0;  // blocks of one batched launch
    long long launches = 0, node_updates = 0;
    long long launches_per_batch = 0;  // kernel launches of the captured batch graph
    double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

namespace {

// Device bytes of one case: one population array (in-place streaming),
// porosity, permeability and the scratch fields (22 FP32 values), the
// residual snapshot (3), the padded porosity of the tiled copies, and 4 MiB
// for the reductions, flags and allocator rounding.
double case_bytes(int storage, int nx, int ny, int nz)
{
    const double N = (double)nx * ny * nz;
    const double pad = (double)(nx + 8) * (ny + 2) * (nz + 2) * 4.0;
    return N * (27.0 * storage_bytes(storage) + 25.0 * 4.0) + pad + 4.0 * 1024 * 1024;
}

// cases of at least this many nodes run the single-case kernels in a batch
// (at 2^20 nodes and above one case keeps the GPU busy: measured 16.7 GLUPS for
// one 128^3 FP16 case on its own kernels against 14.4 in the shared launch)
constexpr long long kServerOwnNodes = 1LL << 20;

template <typename S>
int server_batch(lbm_server* sv)
{
    size_t n = sv->active.size();
    if (n == 0) return LBM_OK;
    // Cases of at least kServerOwnNodes nodes fill the GPU on their own and run
    // the single-case kernels (whose parameters are kernel arguments); the
    // smaller cases share one launch of each batch kernel per step.  Both take
    // the same arithmetic per node.
    std::vector<size_t> shared, own;
    for (size_t k = 0; k < n; ++k) (sv->active[k].ctx->N >= kServerOwnNodes ? own : shared).push_back(k);
    const size_t nb = shared.size();
    if (!sv->graph_valid) {
        // the table: nb cases, then one entry per block of the batched grids
        // (its case and tile), read with one load by each block
        long long total = 0;
        for (size_t j = 0; j < nb; ++j) {
            lbm_ctx* c = sv->active[shared[j]].ctx;
            const long long tx = (c->nx + 2 * kSplitBX - 1) / (2 * kSplitBX), ty = (c->ny + kSplitBY - 1) / kSplitBY;
            total += tx * ty * c->nz;
        }
        if (total >= (1LL << 31)) return fail(LBM_E_INVALID, "too many blocks in one batch");
        const size_t need = std::max<size_t>(1, nb * sizeof(BatchCase<S>) + (size_t)total * sizeof(BatchBlock));
        if (need > sv->table_cap) {
            if (sv->table_dev) cudaFree(sv->table_dev);
            if (sv->table_host) cudaFreeHost(sv->table_host);
            sv->table_cap = std::max(need, 2 * sv->table_cap);
            if (cudaMalloc(&sv->table_dev, sv->table_cap) != cudaSuccess ||
                cudaMallocHost(&sv->table_host, sv->table_cap) != cudaSuccess) {
                sv->table_dev = sv->table_host = nullptr;
                sv->table_cap = 0;
                return fail(LBM_E_NOMEM, "case table allocation failed");
            }
        }
        BatchCase<S>* tab = (BatchCase<S>*)sv->table_host;
        BatchBlock* blocks = (BatchBlock*)(tab + nb);
        long long at = 0;
        for (size_t j = 0; j < nb; ++j) {
            lbm_ctx* c = sv->active[shared[j]].ctx;
            BatchCase<S>& e = tab[j];
            memset((void*)&e, 0, sizeof e);
            e.tm_f = c->tma.f[0];
            e.tm_eps = c->tma.eps;
            e.p = c->pf;
            e.F = c->Ff;
            e.f = (S*)c->f[0];
            e.tiles_x = (c->nx + 2 * kSplitBX - 1) / (2 * kSplitBX);
            e.tiles_y = (c->ny + kSplitBY - 1) / kSplitBY;
            e.nblocks = e.tiles_x * e.tiles_y * c->nz;
            e.block_begin = (int)at;
            for (int q = 0; q < e.nblocks; ++q)
                blocks[at + q] = BatchBlock{(int)j, q % e.tiles_x, (q / e.tiles_x) % e.tiles_y, q / (e.tiles_x * e.tiles_y)};
            at += e.nblocks;
        }
        sv->total_blocks = (int)total;
        if (nb) CK(cudaMemcpyAsync(sv->table_dev, sv->table_host, need, cudaMemcpyHostToDevice, sv->stream));
        if (sv->graph) cudaGraphExecDestroy(sv->graph);
        sv->graph = nullptr;
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(sv->stream, cudaStreamCaptureModeThreadLocal));
        int bad = 0;
        for (int k = 0; k < sv->check_every; ++k) {
            if (nb) bad |= batch_step<S>(sv->table_dev, (int)nb, sv->total_blocks, k & 1, sv->stream);
            for (size_t j : own) {
                lbm_ctx* c = sv->active[j].ctx;
                bad |= inplace_step<S>(c->pf, c->Ff, (S*)c->f[0], k & 1, c->tma, 0, sv->stream, nullptr);
            }
        }
        CK(cudaStreamEndCapture(sv->stream, &g));
        if (bad) {
            cudaGraphDestroy(g);
            return fail(LBM_E_CUDA, "batched launch capture failed");
        }
        cudaError_t e = cudaGraphInstantiate(&sv->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(LBM_E_CUDA, "graph instantiation: %s", cudaGetErrorString(e));
        sv->graph_valid = true;
        sv->launches_per_batch = 3LL * sv->check_every * ((nb ? 1 : 0) + (long long)own.size());
    }
    CK(cudaGraphLaunch(sv->graph, sv->stream));
    sv->launches += sv->launches_per_batch;
    for (auto& a : sv->active) {
        a.ctx->steps += sv->check_every;  // an even count: the in-place layout is back to parity 0
        sv->node_updates += (long long)sv->check_every * a.ctx->N;
    }
    return LBM_OK;
}

int server_admit(lbm_server* sv, std::vector<lbm_case_result>& done)
{
    while (!sv->queue.empty()) {
        PendingCase& pc = sv->queue.front();
        double bytes = case_bytes(sv->storage, pc.nx, pc.ny, pc.nz);
        if (bytes > sv->cap) {  // can never fit
            lbm_case_result r{};
            r.id = pc.id;
            r.status = LBM_E_NOMEM;
            r.submit_time = pc.submit_time;
            r.finish_time = sv->now();
            done.push_back(r);
            sv->queue.pop_front();
            continue;
        }
        if (sv->used + bytes > sv->cap) break;
        lbm_params prm = sv->defaults;
        prm.storage = sv->storage;
        prm.kernel = LBM_KERNEL_SPLIT;
        prm.streaming = LBM_STREAM_IN_PLACE;
        prm.stream = sv->stream;
        lbm_ctx* c = nullptr;
        int rc = lbm_create(&c, LBM_D3Q27, pc.nx, pc.ny, pc.nz, pc.eps.data(), pc.kap.data(), pc.forch, pc.visc, pc.b, &prm);
        if (rc) {
            lbm_case_result r{};
            r.id = pc.id;
            r.status = rc;
            r.submit_time = pc.submit_time;
            r.finish_time = sv->now();
            done.push_back(r);
            sv->queue.pop_front();
            continue;
        }
        if (!c->tma.ok) {
            lbm_destroy(c);
            return fail(LBM_E_UNSUPPORTED, "the batched kernels need the tiled copies of a case");
        }
        ActiveCase a{};
        a.id = pc.id;
        a.ctx = c;
        a.bytes = bytes;
        a.tol = pc.tol;
        for (int k = 0; k < 3; ++k) a.b[k] = pc.b[k];
        a.max_steps = pc.max_steps;
        a.submit_time = pc.submit_time;
        if (cudaMallocHost((void**)&a.red, (RED_N + 1) * sizeof(double)) != cudaSuccess) {
            lbm_destroy(c);
            return fail(LBM_E_CUDA, "pinned allocation failed");
        }
        sv->used += bytes;
        sv->active.push_back(a);
        sv->graph_valid = false;
        sv->queue.pop_front();
    }
    return LBM_OK;
}

template <typename S>
int server_check(lbm_server* sv, std::vector<lbm_case_result>& done)
{
    // residual snapshot of every active case, one synchronisation
    for (auto& a : sv->active) {
        int r = Impl<3, S>::reduce_enqueue(a.ctx, a.red, 1);
        if (r) return r;
        CK(cudaMemcpyAsync(a.red + RED_N, a.ctx->err_dev, sizeof(unsigned), cudaMemcpyDeviceToHost, sv->stream));
    }
    CK(cudaStreamSynchronize(sv->stream));
    std::vector<ActiveCase> keep;
    for (auto& a : sv->active) {
        lbm_ctx* c = a.ctx;
        const double res = (c->steps > sv->check_every && a.red[9] > 0) ? std::sqrt(a.red[5] / a.red[9]) : INFINITY;
        unsigned flag = 0;
        memcpy(&flag, a.red + RED_N, sizeof flag);
        if (std::isfinite(res)) a.history.push_back(res);
        {
            double bm = 0, vb = 0;
            for (int k = 0; k < 3; ++k) {
                bm += a.b[k] * a.b[k];
                vb += a.red[1 + k] / (double)c->N * a.b[k];
            }
            a.mean_along_b.push_back(bm > 0 ? vb / std::sqrt(bm) : 0.0);
        }
        // the mean flow (hence K_app) has settled: its relative change over the
        // last batch is at most 10 tol
        const size_t M = a.mean_along_b.size();
        const bool mean_settled = M >= 2 && std::fabs(a.mean_along_b[M - 1] - a.mean_along_b[M - 2]) <=
                                                10.0 * a.tol * std::fabs(a.mean_along_b[M - 1]);
        int status = LBM_OK;
        bool finish = false;
        const size_t H = a.history.size(), W = 5;
        // noise floor: the smallest residual of the last W batches is no better
        // than 0.9x the smallest of the W batches before
        bool floor = false;
        if (H >= 2 * W) {
            double recent = INFINITY, before = INFINITY;
            for (size_t k = H - W; k < H; ++k) recent = std::min(recent, a.history[k]);
            for (size_t k = H - 2 * W; k < H - W; ++k) before = std::min(before, a.history[k]);
            floor = recent > 0.9 * before;
        }
        if (flag & ERR_DIVERGED) {
            status = LBM_E_DIVERGED;
            finish = true;
        } else if (res < a.tol) {
            finish = true;
        } else if (floor && mean_settled) {
            status = LBM_RETIRED_AT_FLOOR;
            finish = true;
        } else if (c->steps >= a.max_steps) {
            status = LBM_E_INVALID;
            finish = true;
        }
        if (!finish) {
            keep.push_back(a);
            continue;
        }
        lbm_case_result r{};
        r.id = a.id;
        r.status = status;
        r.steps = c->steps;
        r.residual = res;
        double Nn = (double)c->N;
        double bmag = 0, vb = 0;
        for (int k = 0; k < 3; ++k) {
            r.mean_v[k] = a.red[1 + k] / Nn;
            bmag += a.b[k] * a.b[k];
            vb += r.mean_v[k] * a.b[k];
        }
        bmag = std::sqrt(bmag);
        r.k_app = bmag > 0 ? c->nu_f * (vb / bmag) / bmag : 0.0;
        r.submit_time = a.submit_time;
        r.finish_time = sv->now();
        done.push_back(r);
        sv->used -= a.bytes;
        cudaFreeHost(a.red);
        lbm_destroy(c);
        sv->graph_valid = false;
    }
    sv->active.swap(keep);
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_server_create(lbm_server** out, int storage, double hbm_cap_bytes, int check_every, const lbm_params* defaults)
{
    if (!out) return fail(LBM_E_INVALID, "out is NULL");
    *out = nullptr;
    if (storage < LBM_STORE_FP32 || storage > LBM_STORE_BF16)
        return fail(LBM_E_UNSUPPORTED, "the server runs the split kernels: FP32, FP16 or BF16 storage");
    if (!(hbm_cap_bytes > 0)) return fail(LBM_E_INVALID, "hbm_cap_bytes must be > 0");
    if (check_every < 2 || (check_every & 1)) return fail(LBM_E_INVALID, "check_every must be even and >= 2");
    lbm_server* sv = new lbm_server();
    sv->storage = storage;
    sv->cap = hbm_cap_bytes;
    sv->check_every = check_every;
    lbm_default_params(&sv->defaults);
    if (defaults) sv->defaults = *defaults;
    for (int a = 0; a < 3; ++a) sv->defaults.bc[a] = LBM_BC_PERIODIC;
    if (cudaSetDevice(sv->defaults.device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete sv;
        return fail(LBM_E_CUDA, "server stream creation failed");
    }
    sv->defaults.stream = sv->stream;
    sv->t0 = std::chrono::steady_clock::now();
    *out = sv;
    return LBM_OK;
}

double lbm_server_clock(const lbm_server* sv) { return sv ? sv->now() : 0.0; }

int lbm_server_submit(lbm_server* sv, int nx, int ny, int nz, const double* porosity, const double* permeability,
                      double forchheimer, double viscosity, const double force[3], double tol, long max_steps,
                      long long* ticket)
{
    if (!sv || !porosity || !permeability || !force) return fail(LBM_E_INVALID, "NULL argument");
    if (nx < 3 || ny < 3 || nz < 3) return fail(LBM_E_INVALID, "each axis needs >= 3 nodes");
    if (nx % 8 != 0) return fail(LBM_E_UNSUPPORTED, "served cases need nx a multiple of 8 (tiled copies)");
    if (!(tol > 0) || max_steps <= 0) return fail(LBM_E_INVALID, "tol and max_steps must be > 0");
    PendingCase pc;
    pc.id = sv->next_id++;
    pc.nx = nx;
    pc.ny = ny;
    pc.nz = nz;
    size_t N = (size_t)nx * ny * nz;
    pc.eps.assign(porosity, porosity + N);
    pc.kap.assign(permeability, permeability + N);
    pc.forch = forchheimer;
    pc.visc = viscosity;
    for (int a = 0; a < 3; ++a) pc.b[a] = force[a];
    pc.tol = tol;
    pc.max_steps = max_steps;
    pc.submit_time = sv->now();
    if (ticket) *ticket = pc.id;
    sv->queue.push_back(std::move(pc));
    return LBM_OK;
}

int lbm_server_run(lbm_server* sv, int batches, lbm_case_result* results, int max_results, int* n_results,
                   int* n_active, int* n_queued)
{
    if (!sv || batches < 0 || (max_results > 0 && !results)) return fail(LBM_E_INVALID, "bad argument");
    std::vector<lbm_case_result> done;
    int r = LBM_OK;
    for (int k = 0; k < batches && !r; ++k) {
        r = server_admit(sv, done);
        if (r || sv->active.empty()) break;
        r = sv->storage == LBM_STORE_FP32   ? server_batch<float>(sv)
            : sv->storage == LBM_STORE_FP16 ? server_batch<__half>(sv)
                                            : server_batch<__nv_bfloat16>(sv);
        if (r) break;
        r = sv->storage == LBM_STORE_FP32   ? server_check<float>(sv, done)
            : sv->storage == LBM_STORE_FP16 ? server_check<__half>(sv, done)
                                            : server_check<__nv_bfloat16>(sv, done);
    }
    if (!r) r = server_admit(sv, done);
    int m = (int)std::min<size_t>(done.size(), (size_t)std::max(0, max_results));
    for (int k = 0; k < m; ++k) results[k] = done[k];
    if (done.size() > (size_t)m && !r) r = fail(LBM_E_INVALID, "results buffer too small: %zu finished", done.size());
    if (n_results) *n_results = m;
    if (n_active) *n_active = (int)sv->active.size();
    if (n_queued) *n_queued = (int)sv->queue.size();
    return r;
}

int lbm_server_stats(const lbm_server* sv, double* used_bytes, long long* kernel_launches, long long* node_updates)
{
    if (!sv) return fail(LBM_E_INVALID, "server is NULL");
    if (used_bytes) *used_bytes = sv->used;
    if (kernel_launches) *kernel_launches = sv->launches;
    if (node_updates) *node_updates = sv->node_updates;
    return LBM_OK;
}

void lbm_server_destroy(lbm_server* sv)
{
    if (!sv) return;
    cudaStreamSynchronize(sv->stream);
    for (auto& a : sv->active) {
        cudaFreeHost(a.red);
        lbm_destroy(a.ctx);
    }
    if (sv->graph) cudaGraphExecDestroy(sv->graph);
    if (sv->table_dev) cudaFree(sv->table_dev);
    if (sv->table_host) cudaFreeHost(sv->table_host);
    cudaStreamDestroy(sv->stream);
    delete sv;
}

}  // extern "C"
