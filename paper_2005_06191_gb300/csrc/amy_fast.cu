// amy_fast.cu -- dispatch of the register-resident fused backup
// (amy_fast.cuh) and launch of the per-dimension table build.
#include <algorithm>

#include "amy_fast.cuh"
#include "amy_internal.h"

namespace amy {

template <class VT>
amy_status launch_fast_vt(const Geom &g, int wm, int var, int tmode, const FastCall &c, int sm_count,
                          cudaStream_t st);
extern template amy_status launch_fast_vt<float>(const Geom &, int, int, int, const FastCall &, int, cudaStream_t);
extern template amy_status launch_fast_vt<unorm16>(const Geom &, int, int, int, const FastCall &, int,
                                                   cudaStream_t);
extern template amy_status launch_fast_vt<__nv_bfloat16>(const Geom &, int, int, int, const FastCall &, int,
                                                         cudaStream_t);
template <class VT>
amy_status launch_synth_vt(const Geom &g, int wm, int var, int tmode, const FastCall &c, const SynthCall &sc,
                           int sm_count, cudaStream_t st, bool dry_run);
extern template amy_status launch_synth_vt<float>(const Geom &, int, int, int, const FastCall &, const SynthCall &,
                                                  int, cudaStream_t, bool);
extern template amy_status launch_synth_vt<unorm16>(const Geom &, int, int, int, const FastCall &,
                                                    const SynthCall &, int, cudaStream_t, bool);
extern template amy_status launch_synth_vt<__nv_bfloat16>(const Geom &, int, int, int, const FastCall &,
                                                          const SynthCall &, int, cudaStream_t, bool);

int fast_wm(const Geom &g, int prec) {
    if (prec == AMY_PREC_FP64) return 0;
    int wmax = 0;
    for (int d = 0; d < g.n; ++d) wmax = std::max(wmax, g.W[d]);
    const int wm = wmax <= 3 ? 3 : (wmax <= 5 ? 5 : (wmax <= 8 ? 8 : 0));
    if (wm == 0) return 0;
    if (fast_smem_bytes(g.n, wm) > 200 * 1024) return 0;
    return wm;
}

int fast_variant(const Geom &g, int wm, int tmode) {
    if (tmode == TM_FACTORED) return VAR_GENERAL;
    bool exact = true;
    for (int d = 0; d < g.n; ++d) exact = exact && g.W[d] == wm;
    if (!exact) return VAR_GENERAL;
    return ((g.periodic >> (g.n - 1)) & 1u) ? VAR_EXACT : VAR_EXACT_CONTIG;
}

FastShape fast_shape(const Geom &g, int tmode, const FastCall &c, int sm_count) {
    FastShape sh;
    const int wm = fast_wm(g, AMY_PREC_FP32);
    const int var = wm ? fast_variant(g, wm, tmode) : VAR_GENERAL;
    sh.staged = wm > 0 && wm <= 5 && tmode == TM_SEPARABLE && var >= VAR_EXACT && g.n <= 3 && !c.no_stage;
    if (sh.staged) {
        staged_default_shape(g, c, sm_count, sh.ulanes, sh.tilex);
    } else {
        sh.ulanes = (c.ulanes > 0 && FAST_THREADS % c.ulanes == 0) ? c.ulanes : fast_default_ulanes(g, sm_count);
        sh.tilex = FAST_THREADS / sh.ulanes;
    }
    sh.rowtile = sh.staged ? staged_rowtile(g, sh.tilex, c.rows) : 0;
    int rt = 0, outer = 1;
    sh.runs = sh.staged && c.grouped && sh.rowtile > 0 && g.n >= 2 && runs_kernel_applies(g, wm) &&
              runs_tile_split(g, sh.rowtile, c.outer, rt, outer);
    sh.outer = sh.runs ? outer : 1;
    return sh;
}

amy_status launch_backup_fast(const Geom &g, int tmode, int v_store, const FastCall &c, int sm_count,
                              cudaStream_t st) {
    const int wm = fast_wm(g, AMY_PREC_FP32);
    if (wm == 0 || tmode == TM_FULL) return set_error(AMY_E_UNSUPPORTED, "fast backup not applicable");
    const int var = fast_variant(g, wm, tmode);
    if (v_store == AMY_V_BF16) return launch_fast_vt<__nv_bfloat16>(g, wm, var, tmode, c, sm_count, st);
    if (v_store == AMY_V_UNORM16) return launch_fast_vt<unorm16>(g, wm, var, tmode, c, sm_count, st);
    return launch_fast_vt<float>(g, wm, var, tmode, c, sm_count, st);
}

amy_status launch_synth_fast(const Geom &g, int tmode, int v_store, const FastCall &c, const SynthCall &sc,
                             int sm_count, cudaStream_t st, bool dry_run) {
    const int wm = fast_wm(g, AMY_PREC_FP32);
    if (wm == 0 || tmode == TM_FULL) return AMY_E_UNSUPPORTED;
    const int var = fast_variant(g, wm, tmode);
    if (v_store == AMY_V_BF16) return launch_synth_vt<__nv_bfloat16>(g, wm, var, tmode, c, sc, sm_count, st, dry_run);
    if (v_store == AMY_V_UNORM16) return launch_synth_vt<unorm16>(g, wm, var, tmode, c, sc, sm_count, st, dry_run);
    return launch_synth_vt<float>(g, wm, var, tmode, c, sc, sm_count, st, dry_run);
}

amy_status launch_build_sep(const Geom &g, uint32_t *tab, int sm_count, cudaStream_t st) {
    int64_t total = 0;
    for (int d = 0; d < g.n; ++d) total += g.tent[d];
    const int blocks = (int)std::min<int64_t>((total + 127) / 128, (int64_t)sm_count * 16);
    k_build_sep_bounds_init<<<1, 32, 0, st>>>(g, tab);
    k_build_sep<<<std::max(blocks, 1), 128, 0, st>>>(g, tab, total);
    if (g.shoff > 0 && g.tsx[g.n - 1][g.n - 1] != 0)
        k_build_shift<<<(g.tent[g.n - 1] + 127) / 128, 128, 0, st>>>(g, tab);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AMY_OK : cuda_error(e, "table build launch");
}

}  // namespace amy
