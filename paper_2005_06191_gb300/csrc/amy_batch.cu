// amy_batch.cu -- dispatch of the grouped persistent step kernels
// (amy_batch.cuh) over the V storage type; the kernel variants themselves are
// instantiated in the per-storage-type translation units.
#include "amy_batch.cuh"

namespace amy {

template <class VT>
amy_status launch_group_vt(int wm, int tm, int var, const BatchEntry *d, int32_t n, int64_t tiles,
                           int32_t *counter, int max_n, int sm, cudaStream_t st);
extern template amy_status launch_group_vt<float>(int, int, int, const BatchEntry *, int32_t, int64_t, int32_t *,
                                                  int, int, cudaStream_t);
extern template amy_status launch_group_vt<unorm16>(int, int, int, const BatchEntry *, int32_t, int64_t, int32_t *,
                                                    int, int, cudaStream_t);
extern template amy_status launch_group_vt<__nv_bfloat16>(int, int, int, const BatchEntry *, int32_t, int64_t,
                                                          int32_t *, int, int, cudaStream_t);

size_t batched_smem_bytes(int n, int wm) { return kGeomSmemBytes + fast_smem_bytes(n, wm); }

amy_status launch_step_group(int vt, int wm, int tm, int var, const BatchEntry *d_entries, int32_t n_entries,
                             int64_t total_tiles, int32_t *d_counter, int max_n, int sm_count, cudaStream_t st) {
    if (vt == AMY_V_BF16)
        return launch_group_vt<__nv_bfloat16>(wm, tm, var, d_entries, n_entries, total_tiles, d_counter, max_n,
                                              sm_count, st);
    if (vt == AMY_V_UNORM16)
        return launch_group_vt<unorm16>(wm, tm, var, d_entries, n_entries, total_tiles, d_counter, max_n, sm_count,
                                        st);
    return launch_group_vt<float>(wm, tm, var, d_entries, n_entries, total_tiles, d_counter, max_n, sm_count, st);
}

}  // namespace amy
