// amy_fast_launch.cuh -- launcher of the register-resident backup for one V
// storage type; instantiated once per storage type in its own translation
// unit (amy_fast_f32.cu, amy_fast_u16.cu, amy_fast_bf16.cu) so the variants
// compile in parallel.
#pragma once

#include <algorithm>

#include "amy_fast.cuh"
#include "amy_internal.h"
#include "amy_staged.cuh"

namespace amy {

template <class VT>
amy_status launch_fast_vt(const Geom &g, int wm, int var, int tmode, const FastCall &c, int sm_count,
                          cudaStream_t st);

namespace fastimpl {

template <class VT, int WM, int TM, int VAR>
amy_status launch_t(const Geom &g, const FastCall &c, int sm_count, cudaStream_t st) {
    FastArgs<VT> a;
    a.Vn = (const VT *)c.Vn;
    a.Vo = (VT *)c.Vo;
    a.Vfinal = c.Vfinal;
    a.pi = c.pi;
    a.mask = c.mask;
    a.spec_kind = c.spec_kind;
    a.kahan = c.kahan;
    a.T = c.T;
    a.O = c.O;
    a.npairs = c.npairs;
    a.tab = c.tab;
    a.rowtile = 0;
    a.grouped = 0;
    a.box_floats = 0;
    a.stage_tab = 0;
    // Input lanes per state: one when the grid alone fills the GPU several
    // times over, otherwise up to 8 (power of two) to expose parallelism.
    a.ulanes = (c.ulanes > 0 && FAST_THREADS % c.ulanes == 0) ? c.ulanes : fast_default_ulanes(g, sm_count);
    a.tileX = FAST_THREADS / a.ulanes;
    const size_t smem = fast_smem_bytes(g.n, WM);
    auto kern = k_backup_fast<VT, WM, TM, VAR>;
    if (smem > 48 * 1024) {
        static bool raised = false;
        if (!raised) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            if (e != cudaSuccess) return cuda_error(e, "fast backup smem attribute");
            raised = true;
        }
    }
    const int64_t blocks = ((int64_t)g.nx + a.tileX - 1) / a.tileX;
    kern<<<(unsigned)blocks, FAST_THREADS, smem, st>>>(g, a);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AMY_OK : cuda_error(e, "fast backup launch");
}

// Staged variant (low-dimensional problems, exact widths): window boxes in
// shared memory.
template <class VT, int WM, int TM, int NS>
amy_status launch_staged_ns(const Geom &g, const FastCall &c, int sm_count, cudaStream_t st) {
    FastArgs<VT> a;
    a.Vn = (const VT *)c.Vn;
    a.Vo = (VT *)c.Vo;
    a.Vfinal = c.Vfinal;
    a.pi = c.pi;
    a.mask = c.mask;
    a.spec_kind = c.spec_kind;
    a.kahan = c.kahan;
    a.T = c.T;
    a.O = c.O;
    a.npairs = c.npairs;
    a.tab = c.tab;
    int ul = 0, tx = 0;
    staged_default_shape(g, c, sm_count, ul, tx);
    if (ul < 1 || tx < 32 || tx % 32 != 0 || tx * ul > STAGE_MAX_THREADS)
        return set_error(AMY_E_INVALID_ARG, "staged backup shape %d x %d", tx, ul);
    a.ulanes = ul;
    a.tileX = tx;
    a.rowtile = staged_rowtile(g, a.tileX, c.rows);
    a.grouped = c.grouped;
    a.box_floats = c.box_floats > 0 ? std::min(std::max(c.box_floats, 256), STAGE_BOX_FLOATS) : STAGE_BOX_FLOATS;
    const int64_t tabw = (int64_t)g.tent[g.n - 1] * g.trw[g.n - 1];
    a.stage_tab = (c.grouped && tabw <= STAGE_TAB_WORDS) ? (int32_t)tabw : 0;
    const int64_t blocks = staged_blocks(g, a.tileX, a.rowtile);
    const size_t smem = staged_smem_bytes(g.n, WM, a.box_floats, g.nu, a.stage_tab, a.tileX * a.ulanes);
    auto kern = k_backup_staged<VT, WM, TM, NS>;
    static bool raised = false;
    if (!raised) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return cuda_error(e, "staged backup smem attribute");
        raised = true;
    }
    kern<<<(unsigned)blocks, (unsigned)(a.tileX * a.ulanes), smem, st>>>(g, a);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AMY_OK : cuda_error(e, "staged backup launch");
}

template <class VT, int WM, int TM>
amy_status launch_var(const Geom &g, int var, const FastCall &c, int sm, cudaStream_t st) {
    if constexpr (WM <= 5 && TM == TM_SEPARABLE) {
        if (var >= VAR_EXACT && g.n <= 3 && !c.no_stage) {
            if (g.n == 1) return launch_staged_ns<VT, WM, TM, 1>(g, c, sm, st);
            if (g.n == 2) return launch_staged_ns<VT, WM, TM, 2>(g, c, sm, st);
            return launch_staged_ns<VT, WM, TM, 3>(g, c, sm, st);
        }
    }
    if (var == VAR_EXACT_CONTIG) return launch_t<VT, WM, TM, VAR_EXACT_CONTIG>(g, c, sm, st);
    if (var == VAR_EXACT) return launch_t<VT, WM, TM, VAR_EXACT>(g, c, sm, st);
    return launch_t<VT, WM, TM, VAR_GENERAL>(g, c, sm, st);
}

template <class VT, int WM>
amy_status launch_tm(const Geom &g, int var, int tmode, const FastCall &c, int sm, cudaStream_t st) {
    switch (tmode) {
        case TM_OTF: return launch_var<VT, WM, TM_OTF>(g, var, c, sm, st);
        case TM_FACTORED: return launch_t<VT, WM, TM_FACTORED, VAR_GENERAL>(g, c, sm, st);
        default: return launch_var<VT, WM, TM_SEPARABLE>(g, var, c, sm, st);
    }
}

}  // namespace fastimpl

template <class VT>
amy_status launch_fast_vt(const Geom &g, int wm, int var, int tmode, const FastCall &c, int sm_count,
                          cudaStream_t st) {
    if (wm == 3) return fastimpl::launch_tm<VT, 3>(g, var, tmode, c, sm_count, st);
    if (wm == 5) return fastimpl::launch_tm<VT, 5>(g, var, tmode, c, sm_count, st);
    return fastimpl::launch_tm<VT, 8>(g, var, tmode, c, sm_count, st);
}

}  // namespace amy
