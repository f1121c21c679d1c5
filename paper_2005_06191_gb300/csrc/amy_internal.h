// amy_internal.h -- declarations shared by the translation units of the
// engine (error reporting, problem validation, small conversion kernels).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/amy.h"
#include "amy_core.cuh"

namespace amy {

amy_status set_error(amy_status st, const char *fmt, ...);
amy_status cuda_error(cudaError_t e, const char *what);
int64_t grid_count(double lb, double ub, double eta);
amy_status make_geom(const amy_system *sys, const amy_grid *st, const amy_grid *in, const double *sigma,
                     const amy_cut *cut, Geom &g, std::vector<double> &params);
amy_status make_spec(const Geom &g, const amy_spec *spec, SpecDev &s);
int choose_tile(int32_t nx, int32_t nu, int sm_count);
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
};

// Input lanes per state: one when the grid alone fills the GPU several times
// over, otherwise up to 8 (power of two) to expose parallelism.
inline int fast_default_ulanes(const Geom &g, int sm_count) {
    int ul = 1;
    const int64_t want = (int64_t)sm_count * 2048 * 4;
    while (ul < 8 && ul < g.nu && (int64_t)g.nx * ul < want) ul <<= 1;
    return ul;
}

// Width bound (3, 5, 8) of the fast backup for this geometry, 0 if it does not apply.
int fast_wm(const Geom &g, int prec);
// Kernel variant of the fast backup (general, exact widths, exact widths with
// a contiguous bounded innermost row).
int fast_variant(const Geom &g, int wm, int tmode);
// Finite guard cells on each side of every V buffer the fast kernels read:
// the contiguous-row variant reads a bounded innermost row unclamped (the
// off-grid slots have zero mass), up to kVGuard cells past either end.
constexpr int64_t kVGuard = 16;
amy_status launch_backup_fast(const Geom &g, int tmode, int v_store, const FastCall &c, int sm_count,
                              cudaStream_t st);
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
