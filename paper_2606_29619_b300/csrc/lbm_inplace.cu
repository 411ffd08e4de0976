// Instances of the in-place split step (lbm_inplace.cuh) and of its batched
// form for the serving runtime (lbm_batch.cuh), compiled in a
// translation unit of their own so that the library's units build in parallel.
#include "lbm_batch.cuh"

namespace lbm {
template int inplace_step<float>(const Params<float>&, const Fields<float>&, float*, int, const SplitTma&, int,
                                 cudaStream_t, KernelClock*);
template int inplace_step<__half>(const Params<float>&, const Fields<float>&, __half*, int, const SplitTma&, int,
                                  cudaStream_t, KernelClock*);
template int inplace_step<__nv_bfloat16>(const Params<float>&, const Fields<float>&, __nv_bfloat16*, int,
                                         const SplitTma&, int, cudaStream_t, KernelClock*);
template int batch_step<float>(const void*, int, int, int, cudaStream_t);
template int batch_step<__half>(const void*, int, int, int, cudaStream_t);
template int batch_step<__nv_bfloat16>(const void*, int, int, int, cudaStream_t);
}  // namespace lbm
