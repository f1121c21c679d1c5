// amy_fast_launch.cuh -- launcher of the register-resident backup for one V
// storage type; instantiated once per storage type in its own translation
// unit (amy_fast_f32.cu, amy_fast_u16.cu, amy_fast_bf16.cu) so the variants
// compile in parallel.
#pragma once

#include <algorithm>
#include <atomic>

#include "amy_fast.cuh"
#include "amy_internal.h"
#include "amy_plane.cuh"
#include "amy_tile.cuh"
#include "amy_runs.cuh"
#include "amy_staged.cuh"

namespace amy {

template <class VT>
amy_status launch_fast_vt(const Geom &g, int wm, int var, int tmode, const FastCall &c, int sm_count,
                          cudaStream_t st);
template <class VT>
amy_status launch_synth_vt(const Geom &g, int wm, int var, int tmode, const FastCall &c, const SynthCall &sc,
                           int sm_count, cudaStream_t st, bool dry_run);

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
    a.stage_recs = 0;
    a.runs_planes = 0;
    a.tx_magic = 0;
    a.chu_shift = 0;
    a.outer = 1;
    a.bnd_known = 0;
    a.nrs = 0;
    a.in_stride_b = INT_MIN;
    // Input lanes per state: one when the grid alone fills the GPU several
    // times over, otherwise up to 8 (power of two) to expose parallelism.
    a.ulanes = (c.ulanes > 0 && FAST_THREADS % c.ulanes == 0) ? c.ulanes : fast_default_ulanes(g, sm_count);
    a.tileX = FAST_THREADS / a.ulanes;
    const size_t smem = fast_smem_bytes(g.n, WM);
    auto kern = k_backup_fast<VT, WM, TM, VAR>;
    if (smem > 48 * 1024) {
        static std::atomic<uint64_t> raised{0};
        const amy_status r = smem_optin((const void *)kern, 200 * 1024, raised, "fast backup smem attribute");
        if (r != AMY_OK) return r;
    }
    const int64_t blocks = ((int64_t)g.nx + a.tileX - 1) / a.tileX;
    kern<<<(unsigned)blocks, FAST_THREADS, smem, st>>>(g, a);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AMY_OK : cuda_error(e, "fast backup launch");
}

// Per-run variant (row tiles, inputs in runs sharing their outer records,
// innermost dim's table staged in shared memory as shifted weights).  The
// box budget is the tile's exact sliding box when the tables' origin bounds
// are known on the host (c.bounds_known), else a default; a caller-given
// budget (c.box_floats) caps it.
// rowtile: rows of dim n-2 per tile; outer: values of dim 0 per tile (3-D, else 1)
template <class VT, int WM, int NS>
void fill_runs_args(const Geom &g, const FastCall &c, int ul, int tx, int rowtile, int outer, bool kahan,
                    FastArgs<VT> &a) {
    a.Vn = (const VT *)c.Vn;
    a.Vo = (VT *)c.Vo;
    a.Vfinal = c.Vfinal;
    a.pi = c.pi;
    a.mask = c.mask;
    a.spec_kind = c.spec_kind;
    a.kahan = kahan ? 1 : 0;
    a.T = c.T;
    a.O = c.O;
    a.npairs = c.npairs;
    a.tab = c.tab;
    a.ulanes = ul;
    a.tileX = tx;
    a.rowtile = rowtile;
    a.grouped = 1;
    a.stage_tab = 0;
    a.stage_recs = g.tent[g.n - 1];
    const int L = g.n - 1;
    int box;
    if (c.bounds_known) {
        const int K = WM + (c.bnd_hi[L] - c.bnd_lo[L]);
        a.runs_planes = runs_planes(std::min(std::max(K, WM), WM + 3));
        int64_t nrows = (int64_t)rowtile - 1 + (c.bnd_hi[L - 1] - c.bnd_lo[L - 1]) + WM;
        if (NS == 3) nrows *= (int64_t)outer - 1 + (c.bnd_hi[0] - c.bnd_lo[0]) + WM;
        box = (int)std::min<int64_t>(runs_box_floats(nrows, g.N[L], K), 48 * 1024);
    } else {
        a.runs_planes = runs_planes(WM + 3);
        box = RUNS_BOX_DEFAULT;
    }
    if (c.box_floats > 0) box = std::min(box, c.box_floats);
    a.box_floats = (std::max(box, 4) + 3) & ~3;
    a.bnd_known = c.bounds_known;
    for (int d = 0; d < 3; ++d) {
        a.bnd_lo[d] = c.bnd_lo[d];
        a.bnd_hi[d] = c.bnd_hi[d];
    }
    a.nrs = (c.run_starts && c.n_runs >= 1 && c.n_runs <= 64) ? c.n_runs : 0;
    for (int i = 0; i <= a.nrs && a.nrs > 0; ++i) a.rs[i] = (uint16_t)c.run_starts[i];
    a.in_stride_b = a.nrs > 0 ? c.in_stride_b : INT_MIN;
    a.tx_magic = (uint32_t)(((1ULL << 32) + (uint64_t)tx - 1) / (uint64_t)tx);
    int chu = tx / (32 * rowtile * outer), sh = 0;
    while ((1 << sh) < chu) ++sh;
    a.chu_shift = sh;
    a.outer = outer;
}

// grid of the per-run kernels: (row tiles of dim n-2, dim 0) for 3-D problems,
// row tiles of dim 0 for 2-D
// Neighbour radius (in tiles) of the persistent kernel's wait along one grid
// extent of G tiles of S points of a dim with N points.  The box of the tile
// [t, t + S) spans the cells [t + lo, t + S - 1 + hi + wm - 1] (lo, hi: the
// bounds of origin minus own coordinate), so the tiles it reads lie within
// max(ceil(-lo / S), ceil((hi + wm - 1) / S)) of it, and by the same bound
// every tile that reads it lies within that radius too.  A periodic dim wraps
// by whole tiles when S divides N (sets `bit` in wrap); otherwise it waits for
// the whole extent.
inline int nbr_radius(int lo, int hi, int wm, int S, int N, int G, bool periodic, uint32_t &wrap, uint32_t bit) {
    const int below = std::max(0, -lo), above = std::max(0, hi + wm - 1);
    int r = std::max((below + S - 1) / S, (above + S - 1) / S);
    if (periodic) {
        if (N % S == 0)
            wrap |= bit;
        else
            r = G;
    }
    return std::min(r, G);
}

inline dim3 runs_grid(const Geom &g, int rowtile, int outer) {
    return g.n == 3 ? dim3((unsigned)((g.N[1] + rowtile - 1) / rowtile), (unsigned)((g.N[0] + outer - 1) / outer))
                    : dim3((unsigned)((g.N[0] + rowtile - 1) / rowtile));
}


// Per-run variant (row tiles, inputs in runs sharing their outer records,
// innermost dim's table staged in shared memory as shifted weights).  The
// box budget is the tile's exact sliding box when the tables' origin bounds
// are known on the host (c.bounds_known), else a default; a caller-given
// budget (c.box_floats) caps it.
template <class VT, int WM, int NS, bool KAHAN>
amy_status launch_runs_k(const Geom &g, const FastCall &c, int ul, int tx, int rowtile, int outer, cudaStream_t st) {
    FastArgs<VT> a;
    fill_runs_args<VT, WM, NS>(g, c, ul, tx, rowtile, outer, KAHAN, a);
    const dim3 grid = runs_grid(g, rowtile, outer);
    if (grid.y > 65535) return set_error(AMY_E_UNSUPPORTED, "per-run backup: dim 0 above 65535 tiles");
    const size_t smem = runs_smem_bytes(NS, WM, a.box_floats, g.nu, a.stage_recs, a.runs_planes, a.tileX * a.ulanes);
    auto kern = k_backup_runs<VT, WM, NS, KAHAN>;
    static std::atomic<uint64_t> raised{0};
    {
        const amy_status r = smem_optin((const void *)kern, 200 * 1024, raised, "per-run backup smem attribute");
        if (r != AMY_OK) return r;
    }
    if (smem > 200 * 1024) return set_error(AMY_E_UNSUPPORTED, "per-run backup needs %zu bytes of shared memory", smem);
    kern<<<grid, (unsigned)(a.tileX * a.ulanes), smem, st>>>(g, a);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AMY_OK : cuda_error(e, "per-run backup launch");
}

// The persistent horizon kernel: needs the host copies of the bounds (and an
// inner span of at most WM + 3 slots), at most 64 runs, a box that fits, and
// every block of the grid resident at once.
template <class VT, int WM, int NS, bool KAHAN>
amy_status launch_synth_k(const Geom &g, const FastCall &c, const SynthCall &sc, int ul, int tx, int rowtile,
                          int outer, int sm_count, cudaStream_t st, bool dry_run) {
    if (!c.bounds_known || !c.run_starts || c.n_runs < 1 || c.n_runs > 64 || g.shoff == 0)
        return AMY_E_UNSUPPORTED;
    const int L = g.n - 1;
    const int KX = c.bnd_hi[L] - c.bnd_lo[L];
    if (KX < 0 || KX > 3 || WM + KX > g.N[L]) return AMY_E_UNSUPPORTED;
    FastArgs<VT> a;
    fill_runs_args<VT, WM, NS>(g, c, ul, tx, rowtile, outer, KAHAN, a);
    int64_t nrows = (int64_t)rowtile - 1 + (c.bnd_hi[L - 1] - c.bnd_lo[L - 1]) + WM;
    if (NS == 3) nrows *= (int64_t)outer - 1 + (c.bnd_hi[0] - c.bnd_lo[0]) + WM;
    if (runs_box_floats(nrows, g.N[L], WM + KX) > a.box_floats) return AMY_E_UNSUPPORTED;
    const dim3 grid = runs_grid(g, rowtile, outer);
    if (grid.y > 65535) return AMY_E_UNSUPPORTED;
    const int threads = a.tileX * a.ulanes;
    const size_t smem = runs_smem_bytes(NS, WM, a.box_floats, g.nu, a.stage_recs, a.runs_planes, threads);
    if (smem > 200 * 1024) return AMY_E_UNSUPPORTED;
    auto kern = k_synth_runs<VT, WM, NS, KAHAN>;
    static std::atomic<uint64_t> raised{0};
    {
        const amy_status r = smem_optin((const void *)kern, 200 * 1024, raised, "persistent backup smem attribute");
        if (r != AMY_OK) return r;
    }
    // the occupancy query does not reject a block above the kernel's launch
    // bound (the launch would fail): check it first
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return cuda_error(e, "persistent backup attributes");
    if (threads > fa.maxThreadsPerBlock) return AMY_E_UNSUPPORTED;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return cuda_error(e, "persistent backup occupancy");
    if ((int64_t)per_sm * sm_count < (int64_t)grid.x * grid.y) return AMY_E_UNSUPPORTED;
    if (dry_run) return AMY_OK;
    RunsHorizon hz;
    hz.V0 = sc.V0;
    hz.V1 = sc.V1;
    hz.Vfinal = sc.Vfinal;
    hz.pi = sc.pi;
    hz.all_steps = sc.all_steps;
    hz.horizon = sc.horizon;
    hz.bar = sc.bar;
    hz.err = sc.err;
    hz.spin_limit = sc.spin_limit;
    hz.flags = nullptr;
    hz.nr_y = hz.nr_x = 0;
    hz.wrap = 0;
    if (!sc.grid_barrier && (int64_t)grid.x * grid.y <= kBarTiles) {
        // neighbour radius per grid extent: blockIdx.x tiles dim n-2 by
        // rowtile points, blockIdx.y (3-D) tiles dim 0 by outer points
        const int dx = g.n - 2;
        hz.nr_x = nbr_radius(c.bnd_lo[dx], c.bnd_hi[dx], WM, rowtile, g.N[dx], (int)grid.x,
                             (g.periodic >> dx) & 1u, hz.wrap, 2u);
        if (NS == 3)
            hz.nr_y = nbr_radius(c.bnd_lo[0], c.bnd_hi[0], WM, outer, g.N[0], (int)grid.y, g.periodic & 1u,
                                 hz.wrap, 1u);
        hz.flags = sc.bar + 2;
    }
    Geom gg = g;
    void *args[] = {(void *)&gg, (void *)&a, (void *)&hz};
    e = cudaLaunchCooperativeKernel((const void *)kern, grid, dim3((unsigned)threads), args, smem, st);
    return e == cudaSuccess ? AMY_OK : cuda_error(e, "persistent backup launch");
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
    if constexpr (NS >= 2 && TM == TM_SEPARABLE) {
        int rt = 0, outer = 1;
        if (c.grouped && a.rowtile > 0 && runs_kernel_applies(g, WM) && runs_tile_split(g, a.rowtile, c.outer, rt, outer)) {
            if (c.kahan) return launch_runs_k<VT, WM, NS, true>(g, c, ul, tx, rt, outer, st);
            return launch_runs_k<VT, WM, NS, false>(g, c, ul, tx, rt, outer, st);
        }
    }
    a.grouped = c.grouped;
    a.box_floats = c.box_floats > 0 ? std::min(std::max(c.box_floats, 256), STAGE_BOX_FLOATS) : STAGE_BOX_FLOATS;
    const int64_t tabw = (int64_t)g.tent[g.n - 1] * g.trw[g.n - 1];
    a.stage_tab = (c.grouped && tabw <= STAGE_TAB_WORDS) ? (int32_t)tabw : 0;
    a.stage_recs = 0;
    a.runs_planes = 0;
    a.tx_magic = 0;
    a.chu_shift = 0;
    a.outer = 1;
    a.bnd_known = 0;
    a.nrs = 0;
    a.in_stride_b = INT_MIN;
    const int64_t blocks = staged_blocks(g, a.tileX, a.rowtile);
    const size_t smem = staged_smem_bytes(g.n, WM, a.box_floats, g.nu, a.stage_tab, a.tileX * a.ulanes);
    auto kern = k_backup_staged<VT, WM, TM, NS>;
    static std::atomic<uint64_t> raised{0};
    {
        const amy_status r = smem_optin((const void *)kern, 200 * 1024, raised, "staged backup smem attribute");
        if (r != AMY_OK) return r;
    }
    kern<<<(unsigned)blocks, (unsigned)(a.tileX * a.ulanes), smem, st>>>(g, a);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AMY_OK : cuda_error(e, "staged backup launch");
}

template <class VT, int WM, int TM>
amy_status launch_var(const Geom &g, int var, const FastCall &c, int sm, cudaStream_t st) {
    if constexpr (WM <= 5 && TM == TM_SEPARABLE) {
        if (var >= VAR_EXACT && g.n <= 3 && !c.no_stage && g.nw == 1) {
            if (g.n == 1) return launch_staged_ns<VT, WM, TM, 1>(g, c, sm, st);
            if (g.n == 2) return launch_staged_ns<VT, WM, TM, 2>(g, c, sm, st);
            return launch_staged_ns<VT, WM, TM, 3>(g, c, sm, st);
        }
    }
    if (var == VAR_EXACT_CONTIG) return launch_t<VT, WM, TM, VAR_EXACT_CONTIG>(g, c, sm, st);
    if (var == VAR_EXACT) return launch_t<VT, WM, TM, VAR_EXACT>(g, c, sm, st);
    return launch_t<VT, WM, TM, VAR_GENERAL>(g, c, sm, st);
}

// The plane kernel (amy_plane.cuh) with the handle's plan.
template <class VT, int WM>
amy_status launch_plane_t(const Geom &g, const FastCall &c, cudaStream_t st) {
    const PlanePlan &pl = *c.plane;
    PlaneArgs<VT> a;
    a.Vn = (const VT *)c.Vn;
    a.Vo = (VT *)c.Vo;
    a.Vfinal = c.Vfinal;
    a.pi = c.pi;
    a.mask = c.mask;
    a.tab = c.tab;
    a.spec_kind = c.spec_kind;
    a.kahan = c.kahan;
    a.P = pl.P;
    a.N1 = g.N[g.n - 1];
    a.G = pl.G;
    int64_t ngroups = 1;
    for (int d = 0; d < g.n - 2; ++d) ngroups *= g.N[d];
    a.ngroups = (int32_t)ngroups;
    a.nS = pl.nS;
    a.nB = pl.nB;
    for (int i = 0; i < PLANE_MAXS; ++i) a.sdim[i] = pl.sdim[i];
    for (int i = 0; i < PLANE_MAXB; ++i) {
        a.bdim[i] = pl.bdim[i];
        a.brange[i] = pl.brange[i];
    }
    a.chunk = pl.chunk;
    a.rs0 = pl.rs0;
    a.rent = pl.rent;
    a.K = pl.K;
    a.work = c.work;
    a.Vpn = (const VT *)c.Vpn;
    a.Vpo = (VT *)c.Vpo;
    a.Ppad = pl.Ppad;
    a.Q = pl.Q;
    a.teams = pl.teams;
    for (int i = 0; i < PLANE_MAXB; ++i) a.bstrideF[i] = pl.bstrideF[i];
    if (!a.Vpn || !a.Vpo) return set_error(AMY_E_INVALID_ARG, "plane backup without its padded V copies");
    auto kern = k_backup_plane<VT, WM>;
    static std::atomic<uint64_t> raised{0};
    {
        const amy_status r = smem_optin((const void *)kern, 200 * 1024, raised, "plane backup smem attribute");
        if (r != AMY_OK) return r;
    }
    const int64_t blocks = (ngroups + pl.G - 1) / pl.G;
    kern<<<(unsigned)blocks, (unsigned)pl.threads, (size_t)pl.smem, st>>>(g, a);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AMY_OK : cuda_error(e, "plane backup launch");
}

// The tile kernel (amy_tile.cuh) with the plan's tile part.
template <class VT, int WM>
amy_status launch_tile_t(const Geom &g, const FastCall &c, cudaStream_t st) {
    const PlanePlan &pl = *c.plane;
    TileArgs<VT> a;
    a.Vo = (VT *)c.Vo;
    a.Vpn = (const VT *)c.Vpn;
    a.Vpo = (VT *)c.Vpo;
    a.Vfinal = c.Vfinal;
    a.pi = c.pi;
    a.mask = c.mask;
    a.tab = c.tab;
    a.spec_kind = c.spec_kind;
    a.kahan = c.kahan;
    a.P = pl.P;
    a.N1 = g.N[g.n - 1];
    a.Ppad = pl.Ppad;
    a.Q = pl.Ppad / 4;
    a.adim = pl.bdim[0];
    a.T = pl.tT;
    a.Na = g.N[a.adim];
    a.ntiles_a = (a.Na + a.T - 1) / a.T;
    int64_t ngroups = 1;
    for (int d = 0; d < g.n - 2; ++d) ngroups *= g.N[d];
    a.nrest = ngroups / a.Na;
    a.nB = pl.nB;
    for (int i = 0; i < PLANE_MAXB; ++i) {
        a.bdim[i] = pl.bdim[i];
        a.brange[i] = pl.brange[i];
        a.bstrideF[i] = pl.bstrideF[i];
    }
    a.rs0 = pl.rs0;
    a.chunk = pl.tchunk;
    a.rent = pl.trent;
    a.nSh = pl.tnSh;
    for (int i = 0; i < PLANE_MAXS; ++i) a.shdim[i] = pl.tshdim[i];
    a.Ksh = pl.tKsh;
    a.ow = pl.tow;
    a.owstrideF = pl.tow >= 0 ? (int32_t)(g.stride[pl.tow] / pl.P) : 0;
    a.work = c.work;
    if (!a.Vpn || !a.Vpo) return set_error(AMY_E_INVALID_ARG, "tile backup without its padded V copies");
    auto kern = k_backup_tile<VT, WM>;
    static std::atomic<uint64_t> raised{0};
    {
        const amy_status r = smem_optin((const void *)kern, 200 * 1024 + 4096, raised, "tile backup smem attribute");
        if (r != AMY_OK) return r;
    }
    const int64_t blocks = a.nrest * a.ntiles_a;
    kern<<<(unsigned)blocks, (unsigned)pl.tthreads, (size_t)pl.tsmem, st>>>(g, a);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AMY_OK : cuda_error(e, "tile backup launch");
}

template <class VT, int WM>
amy_status launch_tm(const Geom &g, int var, int tmode, const FastCall &c, int sm, cudaStream_t st) {
    if (tmode == TM_SEPARABLE && c.plane && c.plane->ok && c.tile && c.plane->tile)
        return launch_tile_t<VT, WM>(g, c, st);
    if (tmode == TM_SEPARABLE && c.plane && c.plane->ok) return launch_plane_t<VT, WM>(g, c, st);
    switch (tmode) {
        case TM_OTF: return launch_var<VT, WM, TM_OTF>(g, var, c, sm, st);
        case TM_FACTORED: return launch_t<VT, WM, TM_FACTORED, VAR_GENERAL>(g, c, sm, st);
        default: return launch_var<VT, WM, TM_SEPARABLE>(g, var, c, sm, st);
    }
}

}  // namespace fastimpl

template <class VT>
amy_status launch_synth_vt(const Geom &g, int wm, int var, int tmode, const FastCall &c, const SynthCall &sc,
                           int sm_count, cudaStream_t st, bool dry_run) {
    if (tmode != TM_SEPARABLE || var < VAR_EXACT || (wm != 3 && wm != 5) || g.n < 2 || g.n > 3 || c.no_stage ||
        !c.grouped || !runs_kernel_applies(g, wm))
        return AMY_E_UNSUPPORTED;
    int ul = 0, tx = 0;
    staged_default_shape(g, c, sm_count, ul, tx);
    if (ul < 1 || tx < 32 || tx % 32 != 0 || tx * ul > STAGE_MAX_THREADS) return AMY_E_UNSUPPORTED;
    int rowtile = 0, outer = 1;
    if (!runs_tile_split(g, staged_rowtile(g, tx, c.rows), c.outer, rowtile, outer)) return AMY_E_UNSUPPORTED;
#define AMY_SYNTH_DISPATCH(WMV, NSV)                                                                               \
    return c.kahan ? fastimpl::launch_synth_k<VT, WMV, NSV, true>(g, c, sc, ul, tx, rowtile, outer, sm_count, st,  \
                                                                  dry_run)                                         \
                   : fastimpl::launch_synth_k<VT, WMV, NSV, false>(g, c, sc, ul, tx, rowtile, outer, sm_count, st, \
                                                                   dry_run);
    if (wm == 3 && g.n == 3) AMY_SYNTH_DISPATCH(3, 3)
    if (wm == 3) AMY_SYNTH_DISPATCH(3, 2)
    if (g.n == 3) AMY_SYNTH_DISPATCH(5, 3)
    AMY_SYNTH_DISPATCH(5, 2)
#undef AMY_SYNTH_DISPATCH
}

template <class VT>
amy_status launch_fast_vt(const Geom &g, int wm, int var, int tmode, const FastCall &c, int sm_count,
                          cudaStream_t st) {
    if (wm == 3) return fastimpl::launch_tm<VT, 3>(g, var, tmode, c, sm_count, st);
    if (wm == 5) return fastimpl::launch_tm<VT, 5>(g, var, tmode, c, sm_count, st);
    return fastimpl::launch_tm<VT, 8>(g, var, tmode, c, sm_count, st);
}

}  // namespace amy
