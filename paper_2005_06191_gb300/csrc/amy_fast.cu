// amy_fast.cu -- dispatch of the register-resident fused backup
// (amy_fast.cuh) and launch of the per-dimension table build.
#include <algorithm>

#include "amy_fast.cuh"
#include "amy_plane.cuh"
#include "amy_tile.cuh"
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

bool plane_structure(const Geom &g, int tmode, int prec, int64_t &rows, int32_t &Ppad) {
    const int n = g.n;
    if (tmode != TM_SEPARABLE || prec == AMY_PREC_FP64 || n < 4 || g.periodic != 0 || g.nw != 1) return false;
    if (fast_wm(g, AMY_PREC_FP32) == 0) return false;
    const int64_t P = (int64_t)g.N[n - 2] * g.N[n - 1];
    if (P > PLANE_MAX_THREADS) return false;
    bool shared = false;
    for (int d = 0; d < n - 2; ++d) shared = shared || (g.tsx[d][n - 2] == 0 && g.tsx[d][n - 1] == 0);
    if (!shared) return false;
    rows = (int64_t)g.nx / P;
    Ppad = (int32_t)((P + 3) / 4 * 4);
    return rows * Ppad + 64 < 2147483647LL;
}

amy_status launch_plane_repack(int v_store, const void *V, void *Vp, int64_t rows, int32_t P, int32_t Ppad,
                               cudaStream_t st) {
    const int blocks = (int)std::min<int64_t>((rows * Ppad + 255) / 256, 16384);
    if (v_store == AMY_V_BF16)
        k_plane_repack<__nv_bfloat16><<<blocks, 256, 0, st>>>((const __nv_bfloat16 *)V, (__nv_bfloat16 *)Vp, rows, P,
                                                              Ppad);
    else if (v_store == AMY_V_UNORM16)
        k_plane_repack<unorm16><<<blocks, 256, 0, st>>>((const unorm16 *)V, (unorm16 *)Vp, rows, P, Ppad);
    else
        k_plane_repack<float><<<blocks, 256, 0, st>>>((const float *)V, (float *)Vp, rows, P, Ppad);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AMY_OK : cuda_error(e, "plane repack launch");
}

// The tile kernel's part of a plane plan (pl.ok already set): tile dim a =
// the first B dim, which no other B dim's component may read; the S dims
// whose components do not read x_a are shared by the tile, at most one other
// S dim's window moves with it.  smem_budget > 0 caps one block's shared
// memory; 0 prefers two blocks per SM holding two values of dim a each.
static void plan_tile(const Geom &g, PlanePlan &pl, int smem_budget) {
    pl.tile = 0;
    if (pl.nB < 1) return;
    const int a = pl.bdim[0];
    for (int b = 1; b < pl.nB; ++b)
        if (g.tsx[pl.bdim[b]][a] != 0) return;
    int nSh = 0, ow = -1;
    int64_t Ksh = 1;
    for (int s = 0; s < pl.nS; ++s) {
        const int d = pl.sdim[s];
        if (g.tsx[d][a] == 0) {
            pl.tshdim[nSh++] = d;
            Ksh *= g.W[d];
        } else {
            if (ow >= 0) return;  // two S dims move with x_a
            ow = d;
        }
    }
    if (nSh == 0 || Ksh > 4096) return;
    if (ow >= 0 && g.W[ow] > 16) return;
    if ((pl.P + 31) / 32 * 32 > TILE_MAX_THREADS) return;
    // threads of a block holding t groups: one per state where they fit
    // (small planes), else one per plane position (each thread then holds
    // up to t states in stage 2)
    auto threads_for = [&](int t) {
        return std::min(TILE_MAX_THREADS, std::max(128, (t * pl.P + 31) / 32 * 32));
    };
    // groups per tile and chunk (values of the first B dim staged at once):
    // the largest tile whose block, holding TILE_WANT0 of those values, fits
    // TILE_BUDGET0 (two blocks per SM by default), else the largest tile
    // holding one value at one block per SM
    const int Na = g.N[a];
    int T = 0, threads = 0;
    int64_t chunk = 0;
    for (int pass = smem_budget > 0 ? 1 : 0; pass < 2 && T == 0; ++pass) {
        const int64_t budget = pass == 0 ? TILE_BUDGET0 : (smem_budget > 0 ? smem_budget : 200 * 1024);
        const int64_t want = pass == 0 ? TILE_WANT0 : 1;
        for (int t = std::min(TILE_MAXT, Na); t >= 2 && T == 0; --t) {
            const int th = threads_for(t);
            int64_t ch = 0;
            while ((int64_t)tile_smem_bytes((int)Ksh, th, t, (int)((ch + 1) * pl.rs0), pl.Ppad) <= budget &&
                   ch < 64)
                ++ch;
            if (ch >= want) {
                T = t;
                chunk = ch;
                threads = th;
            }
        }
    }
    if (T < 2) return;
    pl.tT = T;
    pl.tnSh = nSh;
    pl.tKsh = (int32_t)Ksh;
    pl.tow = ow;
    pl.tchunk = (int32_t)chunk;
    pl.trent = (int32_t)(chunk * pl.rs0);
    pl.tthreads = threads;
    pl.tsmem = (int64_t)tile_smem_bytes((int)Ksh, threads, T, pl.trent, pl.Ppad);
    pl.tile = 1;
}

void plan_plane(const Geom &g, int tmode, int prec, const int32_t *spread, int smem_budget, PlanePlan &pl) {
    pl = PlanePlan();
    const int n = g.n;
    int64_t rows = 0;
    int32_t Ppad = 0;
    if (!spread || !plane_structure(g, tmode, prec, rows, Ppad)) return;
    const int64_t P = (int64_t)g.N[n - 2] * g.N[n - 1];
    int64_t ngroups = 1;
    for (int d = 0; d < n - 2; ++d) {
        ngroups *= g.N[d];
        const bool dep = g.tsx[d][n - 2] != 0 || g.tsx[d][n - 1] != 0;
        if (dep) {
            if (pl.nB == PLANE_MAXB || spread[d] < 0) return;
            pl.bdim[pl.nB] = d;
            pl.brange[pl.nB] = spread[d] + g.W[d];
            pl.bstrideF[pl.nB] = (int32_t)(g.stride[d] / P);
            ++pl.nB;
        } else {
            if (pl.nS == PLANE_MAXS) return;
            pl.sdim[pl.nS++] = d;
        }
    }
    if (pl.nS == 0) return;  // nothing is shared by a plane: the per-state kernels do as well
    int64_t K = 1;
    for (int s = 0; s < pl.nS; ++s) K *= g.W[pl.sdim[s]];
    if (K > 4096) return;
    pl.K = (int32_t)K;
    pl.P = (int32_t)P;
    int64_t rs0 = 1;
    for (int b = 1; b < pl.nB; ++b) rs0 *= pl.brange[b];
    pl.rs0 = (int32_t)rs0;
    const int64_t budget = smem_budget > 0 ? smem_budget : kPlaneSmemDefault;
    const int64_t span0 = pl.nB > 0 ? pl.brange[0] : 1;
    // the most groups per block that hold their whole staged union, else one
    // group with the union staged in chunks of the first B dim
    int64_t G = std::min<int64_t>(std::max<int64_t>(PLANE_MAX_THREADS / P, 1), ngroups);
    int64_t chunk = span0;
    while (G > 1 && (int64_t)plane_smem_bytes((int)G, pl.K, (int)(span0 * rs0), Ppad) > budget) --G;
    if ((int64_t)plane_smem_bytes((int)G, pl.K, (int)(span0 * rs0), Ppad) > budget) {
        G = 1;
        chunk = 0;
        while (chunk < span0 && (int64_t)plane_smem_bytes(1, pl.K, (int)((chunk + 1) * rs0), Ppad) <= budget)
            ++chunk;
        if (chunk < 1) return;
    }
    pl.G = (int32_t)G;
    pl.chunk = (int32_t)chunk;
    pl.rent = (int32_t)(chunk * rs0);
    pl.threads = (int32_t)((G * P + 31) / 32 * 32);
    pl.Ppad = Ppad;
    pl.Q = Ppad / 4;
    pl.teams = std::max(1, pl.threads / (pl.G * pl.Q));
    pl.smem = (int64_t)plane_smem_bytes(pl.G, pl.K, pl.rent, Ppad);
    if (pl.smem > 200 * 1024) return;
    pl.ok = 1;
    plan_tile(g, pl, smem_budget);
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
    sh.staged = wm > 0 && wm <= 5 && tmode == TM_SEPARABLE && var >= VAR_EXACT && g.n <= 3 && !c.no_stage &&
                g.nw == 1;
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
    if (g.n >= 4) {
        int64_t tmax = 1;
        for (int d = 0; d < g.n - 2; ++d) tmax = std::max<int64_t>(tmax, g.tent[d]);
        const int sb = (int)std::min<int64_t>((tmax + 127) / 128, (int64_t)sm_count * 8);
        k_plane_spread<<<std::max(sb, 1), 128, 0, st>>>(g, tab);
    }
    if (g.shoff > 0 && g.tsx[g.n - 1][g.n - 1] != 0)
        k_build_shift<<<(g.tent[g.n - 1] + 127) / 128, 128, 0, st>>>(g, tab);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AMY_OK : cuda_error(e, "table build launch");
}

}  // namespace amy
