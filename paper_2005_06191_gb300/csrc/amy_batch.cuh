// amy_batch.cuh -- persistent step kernel over a group of problems that share
// one kernel variant (V storage type, width bound, row mode, exact widths):
// one launch per group advances every problem of the group by one backup of
// Algorithm 4 (continuous batching).
//
// Each problem is cut into tiles of tileX consecutive states (its tuned
// input-lane count decides tileX); a global atomic counter hands tiles to
// persistent CTAs in order.  A CTA copies the tile's problem geometry into
// shared memory when the problem changes and runs the same per-tile body as
// the single-problem register-resident kernel.
#pragma once

#include <atomic>

#include <climits>

#include <algorithm>

#include "amy_fast.cuh"
#include "amy_internal.h"

namespace amy {

constexpr size_t kGeomSmemBytes = (sizeof(Geom) + 15) / 16 * 16;

template <class VT, int WM, int TM, int VAR>
__global__ void __launch_bounds__(FAST_THREADS) k_step_group(const BatchEntry *__restrict__ entries, int32_t n_entries,
                                                             int64_t total_tiles, int32_t *__restrict__ counter) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Geom &sg = *reinterpret_cast<Geom *>(smem_raw);
    unsigned char *work = smem_raw + kGeomSmemBytes;
    __shared__ int64_t s_tile;
    __shared__ int32_t s_prob;
    int32_t cur = -1;
    while (true) {
        if (threadIdx.x == 0) {
            const int64_t t = atomicAdd(counter, 1);
            int32_t p = 0;
            if (t < total_tiles) {
                int32_t lo = 0, hi = n_entries - 1;  // last entry with tile_begin <= t
                while (lo < hi) {
                    const int32_t mid = (lo + hi + 1) >> 1;
                    if (entries[mid].tile_begin <= t)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
                p = lo;
            }
            s_tile = t;
            s_prob = p;
        }
        __syncwarp();  // lane 0 searched alone: reconverge warp 0 before the block barrier
        __syncthreads();
        const int64_t t = s_tile;
        if (t >= total_tiles) break;
        const int32_t p = s_prob;
        if (p != cur) {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(entries[p].g);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&sg);
            for (int i = threadIdx.x; i < (int)(sizeof(Geom) / 4); i += blockDim.x) dst[i] = src[i];
            cur = p;
            __syncthreads();
        }
        const BatchEntry &e = entries[p];
        FastArgs<VT> a;
        a.Vn = (const VT *)e.Vn;
        a.Vo = (VT *)e.Vo;
        a.Vfinal = e.Vfinal;
        a.pi = e.pi;
        a.mask = e.mask;
        a.spec_kind = e.spec_kind;
        a.tileX = e.tileX;
        a.ulanes = e.ulanes;
        a.kahan = e.kahan;
        a.T = e.T;
        a.O = e.O;
        a.npairs = e.npairs;
        a.tab = e.tab;
        a.rowtile = 0;
        a.grouped = 0;
        a.box_floats = 0;
        a.stage_tab = 0;
        a.stage_recs = 0;
        a.runs_planes = 0;
        a.tx_magic = 0;
        a.chu_shift = 0;
        a.outer = 1;
        a.bnd_known = 0;
        a.nrs = 0;
        a.in_stride_b = INT_MIN;
        const int64_t x = (t - e.tile_begin) * e.tileX + threadIdx.x % e.tileX;
        backup_tile<VT, WM, TM, VAR>(sg, a, (int32_t)min(x, (int64_t)INT_MAX), work);
        __syncthreads();
    }
}

template <class VT, int WM, int TM, int VAR>
amy_status launch_group_t(const BatchEntry *d_entries, int32_t n, int64_t tiles, int32_t *counter, int max_n,
                          int sm_count, cudaStream_t st) {
    const size_t smem = kGeomSmemBytes + fast_smem_bytes(max_n, WM);
    auto kern = k_step_group<VT, WM, TM, VAR>;
    if (smem > 48 * 1024) {
        static std::atomic<uint64_t> raised{0};
        const amy_status r = smem_optin((const void *)kern, 200 * 1024, raised, "batched smem attribute");
        if (r != AMY_OK) return r;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, FAST_THREADS, smem);
    if (e != cudaSuccess) return cuda_error(e, "batched occupancy");
    per_sm = std::max(per_sm, 1);
    const int64_t grid = std::min<int64_t>(tiles, (int64_t)per_sm * sm_count);
    e = cudaMemsetAsync(counter, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return cuda_error(e, "batched counter reset");
    kern<<<(unsigned)grid, FAST_THREADS, smem, st>>>(d_entries, n, tiles, counter);
    e = cudaGetLastError();
    return e == cudaSuccess ? AMY_OK : cuda_error(e, "batched step launch");
}

template <class VT, int WM, int TM>
amy_status launch_group_var(int var, const BatchEntry *d, int32_t n, int64_t tiles, int32_t *counter, int max_n,
                            int sm, cudaStream_t st) {
    if (var == VAR_EXACT_CONTIG) return launch_group_t<VT, WM, TM, VAR_EXACT_CONTIG>(d, n, tiles, counter, max_n, sm, st);
    if (var == VAR_EXACT) return launch_group_t<VT, WM, TM, VAR_EXACT>(d, n, tiles, counter, max_n, sm, st);
    return launch_group_t<VT, WM, TM, VAR_GENERAL>(d, n, tiles, counter, max_n, sm, st);
}

template <class VT, int WM>
amy_status launch_group_tm(int tm, int var, const BatchEntry *d, int32_t n, int64_t tiles, int32_t *counter,
                           int max_n, int sm, cudaStream_t st) {
    if (tm == TM_OTF) return launch_group_var<VT, WM, TM_OTF>(var, d, n, tiles, counter, max_n, sm, st);
    if (tm == TM_FACTORED)
        return launch_group_t<VT, WM, TM_FACTORED, VAR_GENERAL>(d, n, tiles, counter, max_n, sm, st);
    return launch_group_var<VT, WM, TM_SEPARABLE>(var, d, n, tiles, counter, max_n, sm, st);
}

template <class VT>
amy_status launch_group_vt(int wm, int tm, int var, const BatchEntry *d, int32_t n, int64_t tiles,
                           int32_t *counter, int max_n, int sm, cudaStream_t st) {
    if (n <= 0 || tiles <= 0) return AMY_OK;
    if (wm == 3) return launch_group_tm<VT, 3>(tm, var, d, n, tiles, counter, max_n, sm, st);
    if (wm == 5) return launch_group_tm<VT, 5>(tm, var, d, n, tiles, counter, max_n, sm, st);
    return launch_group_tm<VT, 8>(tm, var, d, n, tiles, counter, max_n, sm, st);
}

}  // namespace amy
