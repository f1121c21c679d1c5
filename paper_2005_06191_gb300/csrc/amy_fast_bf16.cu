// amy_fast_bf16.cu -- register-resident backup kernels (single problem and
// grouped persistent batch) with V stored as __nv_bfloat16.
#include "amy_batch.cuh"
#include "amy_fast_launch.cuh"

namespace amy {
template amy_status launch_fast_vt<__nv_bfloat16>(const Geom &, int, int, int, const FastCall &, int, cudaStream_t);
template amy_status launch_synth_vt<__nv_bfloat16>(const Geom &, int, int, int, const FastCall &, const SynthCall &, int,
                                          cudaStream_t, bool);
template amy_status launch_group_vt<__nv_bfloat16>(int, int, int, const BatchEntry *, int32_t, int64_t, int32_t *, int, int,
                                         cudaStream_t);
}  // namespace amy
