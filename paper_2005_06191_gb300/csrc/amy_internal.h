// amy_internal.h -- declarations shared by the translation units of the
// engine (error reporting, problem validation, small conversion kernels).
#pragma once

#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/amy.h"
#include "amy_core.cuh"

namespace amy {

amy_status set_error(amy_status st, const char *fmt, ...);
amy_status cuda_error(cudaError_t e, const char *what);
int64_t grid_count(double lb, double ub, double eta);
// Validation, grid and window geometry of a problem (no heap use).
amy_status fill_geom(const amy_system *sys, const amy_grid *st, const amy_grid *in, const double *sigma,
                     const amy_cut *cut, Geom &g);
// fill_geom plus a host copy of the system parameters.
amy_status make_geom(const amy_system *sys, const amy_grid *st, const amy_grid *in, const double *sigma,
                     const amy_cut *cut, Geom &g, std::vector<double> &params);
amy_status make_spec(const Geom &g, const amy_spec *spec, SpecDev &s);
int choose_tile(int32_t nx, int32_t nu, int sm_count);
// Raises a kernel's dynamic shared-memory limit to `bytes` on the current
// device the first time it is needed there.  The attribute belongs to the
// device, so `done` keeps one bit per device ordinal (0..63; higher ordinals
// set the attribute on every call).
amy_status smem_optin(const void *func, int bytes, std::atomic<uint64_t> &done, const char *what);
// Plan of the plane kernel (amy_plane.cuh, backup kernel 7): the F dims
// contracted first (S: mean component free of the two innermost coordinates)
// and those staged as ranges (B), the largest range of a group's windows per
// B dim, and the launch shape (G groups of P states per block, R staged in
// chunks of `chunk` values of the first B dim).
struct PlanePlan {
    int32_t ok = 0;
    int32_t nS = 0, nB = 0;
    int32_t sdim[6] = {0, 0, 0, 0, 0, 0};
    int32_t bdim[3] = {0, 0, 0};
    int32_t brange[3] = {1, 1, 1};
    int32_t K = 0, G = 0, chunk = 1, rs0 = 1, rent = 1, threads = 0, P = 0;
    int32_t Ppad = 0, Q = 0, teams = 0;  // padded plane, stage-1 team size, teams per group
    int32_t bstrideF[3] = {0, 0, 0};     // plane-index strides of the B dims
    int64_t smem = 0;
    // The tile kernel (amy_tile.cuh, backup kernel 8): tiles of tT groups
    // along the first B dim a, whose first stage is shared by the tile; the
    // S dims split into tnSh shared ones (windows free of x_a) and at most one
    // (tow) whose window moves with x_a.  tile = 0 when it does not apply.
    int32_t tile = 0, tT = 0, tnSh = 0, tKsh = 0, tow = -1, tchunk = 0, trent = 0, tthreads = 0;
    int32_t tshdim[6] = {0, 0, 0, 0, 0, 0};
    int64_t tsmem = 0;
};
// Whether a problem has the plane kernel's structure (independent of the
// tables' origin spreads): tables, FP32, four or more dims, no periodic dim,
// planes of at most 448 states, some F dim shared by a plane.  Its padded V
// copies then take rows * Ppad values each (rows = nx / P).
bool plane_structure(const Geom &g, int tmode, int prec, int64_t &rows, int32_t &Ppad);
// Padded copy of V for the plane kernel (k_plane_repack), on `st`.
amy_status launch_plane_repack(int v_store, const void *V, void *Vp, int64_t rows, int32_t P, int32_t Ppad,
                               cudaStream_t st);
// Default shared memory of one plane-kernel block: two blocks per SM.
constexpr int kPlaneSmemDefault = 100 * 1024;
// The plan for a problem with per-dimension tables; spread[d] is the tables'
// largest spread (max - min) of dim d's window origin over one plane of
// states, read back after the table build (negative: unknown).  smem_budget
// 0 takes kPlaneSmemDefault.  pl.ok = 0 when the kernel does not apply.
void plan_plane(const Geom &g, int tmode, int prec, const int32_t *spread, int smem_budget, PlanePlan &pl);

// Text systems (amy_expr.cu): the parsed mean expressions as the CUDA source
// of their table kernel, and the variables each component reads (input bit i
// < m for u_i, bit m + k for the disturbance w_k).
struct ExprProgram {
    std::string source;
    uint32_t dep_x[MAXD];
    uint32_t dep_u[MAXD];
};
amy_status expr_compile(const char *const *text, int n, int m_ctrl, int p_dist, int64_t n_params, ExprProgram &out);
// Fills g.mtab (device, sum_d tent[d] doubles at moff[d]) on `st`: compiles
// the kernel with NVRTC on first use per source, then launches it.
amy_status expr_fill_means(const ExprProgram &prog, const Geom &g, double *d_mtab, cudaStream_t st);

// User noise densities (amy_expr.cu): compiles the n density texts (the
// variable t) and fills g.n tables of 2 (USER_KNOTS + 1) doubles at d_tab
// (the normalised CDF at the knots of the box, then the density there);
// INVALID_ARG for bad text or a table that is not a density.  Synchronous.
amy_status user_tables(const char *const *pdf, const Geom &g, double *d_tab, cudaStream_t st);

// Closed-loop Monte-Carlo runs (amy_simulate.cu): n_x0 * runs runs of
// `horizon` steps under pi[horizon][nx], successes counted per initial state
// into succ[n_x0] (zeroed by the caller); err bits: 1 an initial state out of
// range, 2 the policy names an input out of range at a live state.
amy_status launch_simulate(const Geom &g, int spec_kind, const uint8_t *mask, const uint16_t *pi, int32_t horizon,
                           const int64_t *x0, int64_t n_x0, int64_t runs, uint64_t seed, unsigned long long *succ,
                           unsigned int *err, int sm_count, cudaStream_t st);

// Type-erased arguments of the register-resident backup kernel.
struct FastCall {
    const void *Vn;
    void *Vo;
    float *Vfinal;
    uint16_t *pi;
    const uint8_t *mask;
    int32_t spec_kind;
    int32_t kahan;
    const float *T;
    const int16_t *O;
    int64_t npairs;
    const uint32_t *tab;
    int32_t ulanes;   // input lanes per state (1, 2, 4, 8); 0 = heuristic
    int32_t no_stage = 0;  // 1: never use the shared-memory staged variant
    int32_t rows = 1;      // staged variant: 1 = tiles of whole innermost-dim rows
                           // (when most lanes stay busy), 0 = consecutive states
    int32_t grouped = 0;   // staged variant: inputs come in runs that share every
                           // outer dim's table record (see input_runs_share_outer)
    int32_t runs = 0;      // number of such runs (0 = not grouped)
    const int32_t *run_starts = nullptr;  // host copy of the input runs' starts (n_runs + 1
    int32_t n_runs = 0;                   // entries, the last = inputs), or null
    int32_t in_stride_b = INT_MIN;        // constant byte step of the inner records within a run
    int32_t bounds_known = 0;  // 1: bnd_lo / bnd_hi hold the tables' bounds on (window
    int32_t bnd_lo[3] = {0, 0, 0};  // origin - own coordinate) per dim (n <= 3), read
    int32_t bnd_hi[3] = {0, 0, 0};  // back after the table build; sizes the per-run box
    int32_t tilex = 0;     // staged variant: lane columns (states) per block, a
                           // multiple of 32 with tilex * ulanes <= 512; 0 = default
    int32_t box_floats = 0;  // staged variant: box budget in floats (0 = 6144)
    int32_t outer = 0;       // per-run kernels, 3-D: values of dim 0 per row tile (0 = 1)
    const PlanePlan *plane = nullptr;  // tables mode: the plane kernel's plan when it runs
    int32_t tile = 0;                  // 1: the tile kernel (8) where the plan has it, else the plane kernel
    unsigned long long *work = nullptr;  // plane kernel: work counters (3 words), or null
    const void *Vpn = nullptr;  // plane kernel: padded copy of V_{k+1}
    void *Vpo = nullptr;        // plane kernel: padded copy of V_k (written)
};

// Whether consecutive inputs form runs (at least two inputs per run on
// average) whose table records agree on every dim but the innermost one, so
// that the staged backup may contract the outer dims once per run.  upart
// holds each input's table-index part per dim (urw words per input).
bool input_runs_share_outer(const Geom &g, const std::vector<int32_t> &upart);
// Starts of the runs of consecutive inputs sharing their outer records
// (with the input count appended), and the byte step between the 16-byte
// shifted inner records of consecutive inputs of a run when it is the same
// everywhere (else INT_MIN).
void input_run_layout(const Geom &g, const std::vector<int32_t> &upart, std::vector<int32_t> &starts,
                      int32_t &stride_b);
// Number of runs of consecutive inputs with equal outer-dim table records.
int32_t input_outer_runs(const Geom &g, const std::vector<int32_t> &upart);


// Input lanes per state: one when the grid alone fills the GPU several times
// over, otherwise up to 8 (power of two) to expose parallelism.
inline int fast_default_ulanes(const Geom &g, int sm_count) {
    int ul = 1;
    const int64_t want = (int64_t)sm_count * 2048 * 4;
    while (ul < 8 && ul < g.nu && (int64_t)g.nx * ul < want) ul <<= 1;
    return ul;
}

// Rows per tile of the staged backup's row-aligned mapping for tileX lane
// columns: each warp takes up to 32 consecutive states of one innermost-dim
// row (chunks of 32 when the row is longer), so the lanes of a warp differ in
// the innermost coordinate only and their reads of the staged window box fall
// in distinct banks.  0 (consecutive states instead) when the mapping is off,
// n < 2, or fewer than three quarters of the lanes would stay busy.
inline int staged_rowtile(const Geom &g, int tileX, int rows) {
    if (!rows || g.n < 2 || g.n > 3) return 0;
    const int R = g.N[g.n - 1];
    int ch = 1;
    while (ch * 32 < R) ch <<= 1;
    const int rw = tileX / (32 * ch);
    return (rw >= 1 && 4 * R >= 3 * 32 * ch) ? rw : 0;
}
// Rows of dim n-2 and values of dim 0 per tile of the per-run kernels from
// the staged row tiling (rows per tile, all dims): the tile's rows split as
// outer x rows when `outer` divides them (3-D), else false.
inline bool runs_tile_split(const Geom &g, int rows_total, int want_outer, int &rowtile, int &outer) {
    outer = (g.n == 3 && want_outer > 1) ? want_outer : 1;
    if (rows_total < 1 || rows_total % outer != 0) return false;
    rowtile = rows_total / outer;
    return true;
}
// Grid of the staged backup: row tiles (within one outermost index when n = 3)
// or tiles of tileX consecutive states.
inline int64_t staged_blocks(const Geom &g, int tileX, int rowtile) {
    if (rowtile == 0) return ((int64_t)g.nx + tileX - 1) / tileX;
    if (g.n == 3) return (int64_t)g.N[0] * ((g.N[1] + rowtile - 1) / rowtile);
    return ((int64_t)g.N[0] + rowtile - 1) / rowtile;
}
// Launch shape the register-resident backup takes for these arguments.
struct FastShape {
    int ulanes;   // input lanes per state
    int tilex;    // lane columns (states) per block
    int rowtile;  // staged variant's rows per tile (0 = consecutive states)
    int staged;   // 1 = shared-memory staged variant
    int runs;     // 1 = its per-run kernel (grouped inputs on row tiles)
    int outer;    // the per-run kernel's values of dim 0 per tile
};
// Default input lanes and lane columns of the staged variant: with input runs
// (grouped), one lane per run when there are at most 8 runs, so that every
// lane contracts the outer dims once; otherwise the register-resident default.
inline void staged_default_shape(const Geom &g, const FastCall &c, int sm_count, int &ulanes, int &tilex) {
    if (c.ulanes > 0)
        ulanes = c.ulanes;
    else if (c.grouped && c.runs >= 1 && c.runs <= 8)
        ulanes = c.runs;
    else
        ulanes = fast_default_ulanes(g, sm_count);
    if (c.tilex > 0)
        tilex = c.tilex;
    else
        tilex = std::min(256, 32 * std::max(1, 16 / ulanes));
}
FastShape fast_shape(const Geom &g, int tmode, const FastCall &c, int sm_count);
// Whether the per-run kernel (amy_runs.cuh) serves a grouped staged launch
// with row tiles: 2-D or 3-D, at most 512 inputs, every mean component
// depending on its own coordinate (so each dim has origin bounds), 4-word
// input parts and records, and an innermost-dim table of at most 4096 records.
inline bool runs_kernel_applies(const Geom &g, int wm) {
    if (g.n < 2 || g.n > 3 || g.nu > 512 || g.urw != 4 || g.nw != 1) return false;
    for (int d = 0; d < g.n; ++d)
        if (g.tsx[d][d] == 0 || g.trw[d] != 4 * ((wm + 1 + 3) / 4)) return false;
    return g.tent[g.n - 1] <= 4096 && g.shoff > 0;
}

// Width bound (3, 5, 8) of the fast backup for this geometry, 0 if it does not apply.
int fast_wm(const Geom &g, int prec);
// Kernel variant of the fast backup (general, exact widths, exact widths with
// a contiguous bounded innermost row).
int fast_variant(const Geom &g, int wm, int tmode);
// Finite guard cells on each side of every V buffer the fast kernels read:
// the contiguous-row variant reads a bounded innermost row unclamped (the
// off-grid slots have zero mass; origins are clamped to [-(W+1), N+1], so a
// row reaches at most W + 1 <= 9 cells past either end of the buffer).
constexpr int64_t kVGuard = 32;
amy_status launch_backup_fast(const Geom &g, int tmode, int v_store, const FastCall &c, int sm_count,
                              cudaStream_t st);
// The whole horizon in one cooperative launch of the per-run kernel
// (k_synth_runs): V0 holds V_N, V1 is the other resident vector; policies and
// the FP32 copy of V_0 as in the per-step path.  bar is the handle's barrier
// block (kBarWords words): the grid barrier's arrival count and a spare word,
// one backup counter per tile for the neighbour wait, then the error flag
// *err.  The caller zeroes its first kBarResetBytes before each launch.
constexpr int kBarTiles = 4096;
constexpr int kBarErrWord = 2 + kBarTiles;
constexpr int kBarWords = kBarErrWord + 2;
constexpr size_t kBarResetBytes = (size_t)kBarErrWord * sizeof(unsigned);
struct SynthCall {
    const void *V0;
    void *V1;
    float *Vfinal;
    uint16_t *pi;
    int32_t all_steps;
    int32_t horizon;
    unsigned *bar;
    int32_t *err;
    int32_t spin_limit;
    int32_t grid_barrier;  // 1: wait for every block between backups (no neighbour wait)
};
// Launches it, or with dry_run only checks that it applies to this problem and
// launch shape and that every block can be resident at once.  Returns
// AMY_E_UNSUPPORTED (and launches nothing) when it does not apply.
amy_status launch_synth_fast(const Geom &g, int tmode, int v_store, const FastCall &c, const SynthCall &sc,
                             int sm_count, cudaStream_t st, bool dry_run);
amy_status launch_build_sep(const Geom &g, uint32_t *tab, int sm_count, cudaStream_t st);
// Fills the separable-table fields of g (dependency sets, strides, offsets);
// returns the table size in 32-bit words.
amy_status plan_sep_tables(Geom &g, const std::vector<double> &params, int64_t &words,
                           std::vector<int32_t> *upart);

// One problem's share of a batched step: its device geometry, this step's
// V in/out and outputs, and its tile range in the launch.
struct BatchEntry {
    const Geom *g;        // device copy of the problem geometry
    const void *Vn;       // V_{k+1}
    void *Vo;             // V_k
    float *Vfinal;        // V_0 output (last step) or null
    uint16_t *pi;         // pi_0 output (last step) or null
    const uint8_t *mask;
    const uint32_t *tab;  // per-dimension tables (separable rows)
    const float *T;       // per-pair masses (factored rows)
    const int16_t *O;     // per-pair origins (factored rows)
    int64_t npairs;
    int64_t tile_begin;   // first tile of this problem within its group's launch
    int32_t tm;           // TM_SEPARABLE or TM_OTF
    int32_t spec_kind;
    int32_t kahan;
    int32_t vt;           // amy_vstore
    int32_t wm;           // window-width bound 3, 5 or 8
    int32_t tileX;
    int32_t ulanes;
};

size_t batched_smem_bytes(int n, int wm);
// One persistent launch over problems sharing a kernel variant (storage type,
// width bound, row mode, exact widths); max_n = largest state dimension.
amy_status launch_step_group(int vt, int wm, int tm, int var, const BatchEntry *d_entries, int32_t n_entries,
                             int64_t total_tiles, int32_t *d_counter, int max_n, int sm_count, cudaStream_t st);
// Row mode picked automatically: separable tables when they stay small,
// per-pair factored rows when they fit the budget, otherwise on the fly.
int choose_tmode(const Geom &g, const std::vector<double> &params, int prec, int64_t budget);
constexpr int64_t kAutoTableBytes = 8LL << 20;
constexpr int64_t kAutoFactoredBytes = 1LL << 30;
amy_status launch_build_factored(const Geom &g, float *T, int16_t *O, int64_t npairs, int sm_count, cudaStream_t st);
// Generic (any window width) FP32 backup of a separable-table (TM_SEPARABLE)
// or on-the-fly (TM_OTF) problem.
amy_status launch_backup_generic_fp32(const Geom &g, int tm, const FastCall &c, int v_store, int sm_count,
                                      cudaStream_t st);
amy_status launch_spec_mask(const Geom &g, const SpecDev &s, uint8_t *mask, void *VN, int v_store, cudaStream_t st);

amy_status launch_v16_to_f32(const void *src, int32_t v_store, float *dst, int64_t n, cudaStream_t s);
amy_status launch_f32_to_v16(const float *src, void *dst, int32_t v_store, int64_t n, cudaStream_t s);

}  // namespace amy
