// Instances of the wavefront step (lbm_wave.cuh), compiled in a translation
// unit of their own so that the library's units build in parallel.
#include "lbm_wave.cuh"

namespace lbm {
template int wave_launch<float>(const Params<float>&, const Fields<float>&, float*, int, const WaveCtl&,
                                const SplitTma&, int, cudaStream_t);
template int wave_launch<__half>(const Params<float>&, const Fields<float>&, __half*, int, const WaveCtl&,
                                 const SplitTma&, int, cudaStream_t);
template int wave_launch<__nv_bfloat16>(const Params<float>&, const Fields<float>&, __nv_bfloat16*, int,
                                        const WaveCtl&, const SplitTma&, int, cudaStream_t);
}  // namespace lbm
