// amy_kernels.cuh -- kernels of the single-problem path: spec mask + V_N,
// stored-T construction (Algorithm 2), the fused backup + max/argmax
// (Algorithm 4, stored or on-the-fly per Sec. 6.1) and a row query used to
// check rows against an independent implementation.
#pragma once

#include "amy_core.cuh"

namespace amy {

// Storage types of V between backups: native FP32/FP64, bfloat16, or a
// 16-bit fixed-point code round(V * 65535) (V is a probability in [0, 1]).
//
// The bfloat16 form is folded about 1/2: V < 1/2 is stored as bf16(V) and
// V >= 1/2 as -bf16(1 - V), the sign bit (unused by a probability) marking
// the fold.  Both 1 - V (V in [1/2, 1]) and the decode 1 + b (b in
// [-1/2, -0]) are exact in FP32, so the only rounding is bf16's, relative to
// min(V, 1 - V): at most 2^-10 absolute instead of 2^-9, and exact at 0 and
// 1, where reach and safety values collect.
__device__ __forceinline__ __nv_bfloat16 bf16_fold(float v) {
    v = fminf(fmaxf(v, 0.0f), 1.0f);
    return v < 0.5f ? __float2bfloat16_rn(v) : __float2bfloat16_rn(-(1.0f - v));
}
__device__ __forceinline__ float bf16_unfold(__nv_bfloat16 b) {
    const float f = __bfloat162float(b);
    return signbit(f) ? 1.0f + f : f;
}
template <class R, class VT> __device__ __forceinline__ R vload(const VT *p);
template <> __device__ __forceinline__ double vload<double, double>(const double *p) { return __ldg(p); }
template <> __device__ __forceinline__ float vload<float, float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ float vload<float, __nv_bfloat16>(const __nv_bfloat16 *p) {
    return bf16_unfold(__ldg(p));
}
template <> __device__ __forceinline__ float vload<float, unorm16>(const unorm16 *p) {
    return (float)__ldg(&p->bits) * (1.0f / 65535.0f);
}

template <class VT, class R> __device__ __forceinline__ VT vstore_cast(R v);
template <> __device__ __forceinline__ double vstore_cast<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float vstore_cast<float, float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 vstore_cast<__nv_bfloat16, float>(float v) {
    return bf16_fold(v);
}
template <> __device__ __forceinline__ unorm16 vstore_cast<unorm16, float>(float v) {
    unorm16 r;
    r.bits = (uint16_t)__float2uint_rn(fminf(fmaxf(v, 0.0f), 1.0f) * 65535.0f);
    return r;
}

__device__ __forceinline__ float min_r(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double min_r(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float fma_r(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_r(double a, double b, double c) { return fma(a, b, c); }

// Compensated (Kahan) or plain accumulation of one term.
template <class R, bool KAHAN>
__device__ __forceinline__ void accum(R &acc, R &comp, R term) {
    if (KAHAN) {
        const R y = term - comp;
        const R t = acc + y;
        comp = (t - acc) - y;
        acc = t;
    } else {
        acc += term;
    }
}

// ---------------------------------------------------------------------------
// Spec sets (Algorithm 3, initial value function) on representative points.
// ---------------------------------------------------------------------------
template <class R, class VT>
__global__ void k_spec_mask(const __grid_constant__ Geom g, const __grid_constant__ SpecDev s,
                            uint8_t *__restrict__ mask, VT *__restrict__ VN) {
    for (int64_t xl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; xl < g.nx;
         xl += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = (int32_t)xl;
        int32_t xi[MAXD];
        decode_state(g, x, xi);
        double c[MAXD];
        for (int d = 0; d < g.n; ++d) c[d] = state_centre(g, d, xi[d]);
        uint8_t f = 0;
        for (int b = 0; b < s.n_target; ++b) {
            bool in = true;
            for (int d = 0; d < g.n; ++d) in = in && (s.t_lb[b][d] <= c[d] && c[d] <= s.t_ub[b][d]);
            if (in) f |= F_TARGET;
        }
        for (int b = 0; b < s.n_avoid; ++b) {
            bool in = true;
            for (int d = 0; d < g.n; ++d) in = in && (s.a_lb[b][d] <= c[d] && c[d] <= s.a_ub[b][d]);
            if (in) f |= F_AVOID;
        }
        if (s.kind == SPEC_SAFETY) {
            bool in = true;
            if (s.has_safe)
                for (int d = 0; d < g.n; ++d) in = in && (s.safe_lb[d] <= c[d] && c[d] <= s.safe_ub[d]);
            if (in) f |= F_SAFE;
        } else {
            f |= F_SAFE;
        }
        mask[x] = f;
        R v;
        if (s.kind == SPEC_SAFETY)
            v = (f & F_SAFE) ? R(1) : R(0);
        else
            v = (f & F_TARGET) ? R(1) : R(0);
        VN[x] = vstore_cast<VT, R>(v);
    }
}

// ---------------------------------------------------------------------------
// Row setup for one (x, u) pair: per-dim masses `fac` and cell offsets `off`
// (each dim d occupies W[d] consecutive entries).
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void row_setup_otf(const Geom &g, int32_t x, int32_t u, R *fac,
                                              int32_t *off, int32_t *origin) {
    double mu[MAXD];
    mean_of(g, x, u, mu);
    int b = 0;
    for (int d = 0; d < g.n; ++d) {
        const int32_t o = origin_of(g, d, mu[d]);
        if (origin) origin[d] = o;
        dim_masses<R>(g, d, mu[d], o, noise_centre(g, x, d), fac + b, off + b);
        b += g.W[d];
    }
}

template <class R>
__device__ __forceinline__ void row_setup_stored(const Geom &g, const R *__restrict__ T,
                                                 const int16_t *__restrict__ O, int64_t npairs,
                                                 int64_t pair, bool factored, R *fac, int32_t *off,
                                                 int32_t *origin) {
    int b = 0;
    for (int d = 0; d < g.n; ++d) {
        const int32_t o = __ldg(O + d * npairs + pair);
        if (origin) origin[d] = o;
        dim_offsets(g, d, o, off + b);
        if (factored)
            for (int k = 0; k < g.W[d]; ++k) fac[b + k] = __ldg(T + (int64_t)(b + k) * npairs + pair);
        b += g.W[d];
    }
}

// Row setup from the per-dimension tables of the separable stored mode.
__device__ __forceinline__ void row_setup_sep(const Geom &g, const uint32_t *__restrict__ tab, int32_t x,
                                              int32_t u, float *fac, int32_t *off, int32_t *origin) {
    int32_t xi[MAXD], ui[MAXD];
    decode_state(g, x, xi);
    uint32_t r = (uint32_t)u;
    for (int i = g.m - 1; i >= 0; --i) {
        ui[i] = (int32_t)(r % (uint32_t)g.ucount[i]);
        r /= (uint32_t)g.ucount[i];
    }
    int b = 0;
    for (int d = 0; d < g.n; ++d) {
        int64_t e = 0;
        for (int j = 0; j < g.n; ++j) e += (int64_t)xi[j] * g.tsx[d][j];
        for (int i = 0; i < g.m; ++i) e += (int64_t)ui[i] * g.tsu[d][i];
        const uint32_t *rec = tab + g.toff[d] + e * g.trw[d];
        const int32_t o = (int32_t)__ldg(rec);
        if (origin) origin[d] = o;
        dim_offsets(g, d, o, off + b);
        for (int k = 0; k < g.W[d]; ++k) fac[b + k] = __uint_as_float(__ldg(rec + 1 + k));
        b += g.W[d];
    }
}

// Window sum of a factored row: sum over the window box (C order) of
// prod_d fac_d[k_d] * V[sum_d off_d[k_d]].  The last dimension is the inner
// run; the outer dims carry prefix products and prefix offsets.
template <class R, class VT, bool KAHAN>
__device__ __forceinline__ R window_sum_factored(const Geom &g, const R *fac, const int32_t *off,
                                                 const VT *__restrict__ V) {
    const int n = g.n;
    const int WL = g.W[n - 1];
    const int bL = g.wsum - WL;
    int k[MAXD], fb[MAXD];
    R pp[MAXD];
    int32_t po[MAXD];
    int acc_fb = 0;
    for (int d = 0; d < n; ++d) {
        fb[d] = acc_fb;
        acc_fb += g.W[d];
        k[d] = 0;
    }
    R p = R(1);
    int32_t q = 0;
    for (int d = 0; d < n - 1; ++d) {
        p *= fac[fb[d]];
        q += off[fb[d]];
        pp[d] = p;
        po[d] = q;
    }
    R acc = R(0), comp = R(0);
    const int rows = g.wtot / WL;
    for (int r = 0; r < rows; ++r) {
        const R w = (n > 1) ? pp[n - 2] : R(1);
        const int32_t base = (n > 1) ? po[n - 2] : 0;
        if (w != R(0)) {
            R inner = R(0);
            for (int j = 0; j < WL; ++j) inner = fma_r(fac[bL + j], vload<R, VT>(V + base + off[bL + j]), inner);
            accum<R, KAHAN>(acc, comp, w * inner);
        }
        int d = n - 2;
        while (d >= 0) {
            if (++k[d] < g.W[d]) break;
            k[d] = 0;
            --d;
        }
        if (d < 0) break;
        for (int e = d; e < n - 1; ++e) {
            pp[e] = (e > 0 ? pp[e - 1] : R(1)) * fac[fb[e] + k[e]];
            po[e] = (e > 0 ? po[e - 1] : 0) + off[fb[e] + k[e]];
        }
    }
    return acc;
}

// Window sum of a stored full row T[slot][pair] (slot in C order).
template <class R, class VT, bool KAHAN>
__device__ __forceinline__ R window_sum_full(const Geom &g, const R *__restrict__ Trow, int64_t npairs,
                                             const int32_t *off, const VT *__restrict__ V) {
    const int n = g.n;
    const int WL = g.W[n - 1];
    const int bL = g.wsum - WL;
    int k[MAXD], fb[MAXD];
    int32_t po[MAXD];
    int acc_fb = 0;
    for (int d = 0; d < n; ++d) {
        fb[d] = acc_fb;
        acc_fb += g.W[d];
        k[d] = 0;
    }
    int32_t q = 0;
    for (int d = 0; d < n - 1; ++d) {
        q += off[fb[d]];
        po[d] = q;
    }
    R acc = R(0), comp = R(0);
    const int rows = g.wtot / WL;
    int64_t t = 0;
    for (int r = 0; r < rows; ++r) {
        const int32_t base = (n > 1) ? po[n - 2] : 0;
        R inner = R(0);
        for (int j = 0; j < WL; ++j, ++t)
            inner = fma_r(__ldg(Trow + t * npairs), vload<R, VT>(V + base + off[bL + j]), inner);
        accum<R, KAHAN>(acc, comp, inner);
        int d = n - 2;
        while (d >= 0) {
            if (++k[d] < g.W[d]) break;
            k[d] = 0;
            --d;
        }
        if (d < 0) break;
        for (int e = d; e < n - 1; ++e) po[e] = (e > 0 ? po[e - 1] : 0) + off[fb[e] + k[e]];
    }
    return acc;
}

template <class R, class VT> struct BackupArgs {
    const VT *Vn;       // V_{k+1}
    VT *Vo;             // V_k
    R *Vfinal;          // optional unrounded copy of V_k (output precision)
    uint16_t *pi;       // optional policy of this step
    const uint8_t *mask;
    int32_t spec_kind;
    int32_t tileX;      // states per block
    const R *T;         // stored rows (full or factored)
    const int16_t *O;   // stored origins [n][pairs]
    int64_t npairs;
    const uint32_t *tab;  // per-dimension tables (separable stored mode)
};

__device__ __forceinline__ bool state_masked(int32_t spec_kind, uint8_t f) {
    return (spec_kind == SPEC_SAFETY) ? !(f & F_SAFE) : ((f & (F_TARGET | F_AVOID)) != 0);
}

// Fused backup + max/argmax (Algorithm 4, collect step included).  A block
// owns tileX consecutive states and all their inputs: items q = u*tileX + xl
// (consecutive lanes -> consecutive states of one input, so stored rows and V
// windows are read coalesced).  Window sums land in shared memory, then one
// thread per state takes the max and the lowest maximising input.
template <class R, class VT, int TM, bool KAHAN>
__global__ void __launch_bounds__(256) k_backup(const __grid_constant__ Geom g, const BackupArgs<R, VT> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *sbuf = reinterpret_cast<R *>(smem_raw);
    const int TX = a.tileX;
    const int32_t x0 = (int32_t)blockIdx.x * TX;
    const int nitems = TX * g.nu;
    R fac[MAXWS];
    int32_t off[MAXWS];
    for (int q = threadIdx.x; q < nitems; q += blockDim.x) {
        const int u = q / TX;
        const int xl = q - u * TX;
        const int32_t x = x0 + xl;
        R s = R(-1);
        if (x < g.nx && !state_masked(a.spec_kind, a.mask[x])) {
            const int64_t pair = (int64_t)u * g.nx + x;
            if constexpr (TM == TM_OTF) {
                row_setup_otf<R>(g, x, u, fac, off, nullptr);
                s = window_sum_factored<R, VT, KAHAN>(g, fac, off, a.Vn);
            } else if constexpr (TM == TM_FACTORED) {
                row_setup_stored<R>(g, a.T, a.O, a.npairs, pair, true, fac, off, nullptr);
                s = window_sum_factored<R, VT, KAHAN>(g, fac, off, a.Vn);
            } else if constexpr (TM == TM_SEPARABLE) {
                if constexpr (sizeof(R) == 4) {
                    row_setup_sep(g, a.tab, x, u, fac, off, nullptr);
                    s = window_sum_factored<R, VT, KAHAN>(g, fac, off, a.Vn);
                }
            } else {
                row_setup_stored<R>(g, a.T, a.O, a.npairs, pair, false, fac, off, nullptr);
                s = window_sum_full<R, VT, KAHAN>(g, a.T + pair, a.npairs, off, a.Vn);
            }
        }
        sbuf[q] = s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < TX; t += blockDim.x) {
        const int32_t x = x0 + t;
        if (x >= g.nx) continue;
        const uint8_t f = a.mask[x];
        R best;
        uint16_t arg;
        if (state_masked(a.spec_kind, f)) {
            best = (a.spec_kind != SPEC_SAFETY && (f & F_TARGET)) ? R(1) : R(0);
            arg = 0xFFFF;
        } else {
            best = R(-1);
            arg = 0;
            // each input's value: min over its disturbance block (nw = 1: none)
            for (int u = 0; u < g.nu / g.nw; ++u) {
                R s = sbuf[(u * g.nw) * TX + t];
                for (int w = 1; w < g.nw; ++w) s = min_r(s, sbuf[(u * g.nw + w) * TX + t]);
                if (s > best) {
                    best = s;
                    arg = (uint16_t)u;
                }
            }
        }
        a.Vo[x] = vstore_cast<VT, R>(best);
        if (a.Vfinal) a.Vfinal[x] = best;
        if (a.pi) a.pi[x] = arg;
    }
}

// ---------------------------------------------------------------------------
// Stored-row backup split over window rows (dense or wide windows with few
// pairs: one thread per pair leaves the GPU short of loads in flight).  A
// block takes 32 consecutive states of one input (T read coalesced across
// the 32 pairs) and blockDim.y groups; group q sums the window rows (runs of
// the innermost dim, C order) [q*rows/G, (q+1)*rows/G) with the same per-row
// arithmetic as window_sum_full / window_sum_factored, the group partials are
// added in group order, and the pair's sum s(x, u) goes to S[u][x] (-1 for
// masked states).
// k_argmax_rows then takes the max over u and the lowest maximiser.
// ---------------------------------------------------------------------------
template <class R, class VT, bool KAHAN>
__device__ __forceinline__ R window_rows_full(const Geom &g, const R *__restrict__ Trow, int64_t npairs,
                                              const int32_t *off, const VT *__restrict__ V, int r0, int r1) {
    const int n = g.n;
    const int WL = g.W[n - 1];
    const int bL = g.wsum - WL;
    int k[MAXD], fb[MAXD];
    int acc_fb = 0;
    for (int d = 0; d < n; ++d) {
        fb[d] = acc_fb;
        acc_fb += g.W[d];
        k[d] = 0;
    }
    // multi-index of row r0 over dims 0..n-2 (C order)
    int rem = r0;
    for (int d = n - 2; d >= 0; --d) {
        k[d] = rem % g.W[d];
        rem /= g.W[d];
    }
    R acc = R(0), comp = R(0);
    for (int r = r0; r < r1; ++r) {
        int32_t base = 0;
        for (int d = 0; d < n - 1; ++d) base += off[fb[d] + k[d]];
        const R *Tr = Trow + (int64_t)r * WL * npairs;
        R inner = R(0);
        for (int j = 0; j < WL; ++j)
            inner = fma_r(__ldg(Tr + (int64_t)j * npairs), vload<R, VT>(V + base + off[bL + j]), inner);
        accum<R, KAHAN>(acc, comp, inner);
        for (int d = n - 2; d >= 0; --d) {
            if (++k[d] < g.W[d]) break;
            k[d] = 0;
        }
    }
    return acc;
}

// The same for a factored row: row r's weight is the product of its outer
// dims' masses taken left to right (the prefix product window_sum_factored
// carries), rows of weight zero are skipped.
template <class R, class VT, bool KAHAN, int ST = 1>
__device__ __forceinline__ R window_rows_factored(const Geom &g, const R *fac, const int32_t *off,
                                                  const VT *__restrict__ V, int r0, int r1) {
    const int n = g.n;
    const int WL = g.W[n - 1];
    const int bL = g.wsum - WL;
    int k[MAXD], fb[MAXD];
    int acc_fb = 0;
    for (int d = 0; d < n; ++d) {
        fb[d] = acc_fb;
        acc_fb += g.W[d];
        k[d] = 0;
    }
    int rem = r0;
    for (int d = n - 2; d >= 0; --d) {
        k[d] = rem % g.W[d];
        rem /= g.W[d];
    }
    R acc = R(0), comp = R(0);
    for (int r = r0; r < r1; ++r) {
        R w = R(1);
        int32_t base = 0;
        for (int d = 0; d < n - 1; ++d) {
            w *= fac[(fb[d] + k[d]) * ST];
            base += off[(fb[d] + k[d]) * ST];
        }
        if (w != R(0)) {
            R inner = R(0);
            for (int j = 0; j < WL; ++j)
                inner = fma_r(fac[(bL + j) * ST], vload<R, VT>(V + base + off[(bL + j) * ST]), inner);
            accum<R, KAHAN>(acc, comp, w * inner);
        }
        for (int d = n - 2; d >= 0; --d) {
            if (++k[d] < g.W[d]) break;
            k[d] = 0;
        }
    }
    return acc;
}

constexpr int ROWS_MAX_GROUPS = 8;

template <class R, class VT, int TM, bool KAHAN>
__global__ void __launch_bounds__(32 * ROWS_MAX_GROUPS) k_backup_rows(const __grid_constant__ Geom g,
                                                                      const BackupArgs<R, VT> a,
                                                                      R *__restrict__ S) {
    static_assert(TM == TM_FULL || TM == TM_FACTORED, "stored rows");
    __shared__ R part[ROWS_MAX_GROUPS][32];
    const int lane = threadIdx.x, q = threadIdx.y, G = blockDim.y;
    const int32_t x = (int32_t)blockIdx.x * 32 + lane;
    const int32_t u = (int32_t)blockIdx.y;
    const bool live = x < g.nx && !state_masked(a.spec_kind, a.mask[x]);
    R s = R(0);
    if (live) {
        const int rows = g.wtot / g.W[g.n - 1];
        const int r0 = (int)((int64_t)rows * q / G), r1 = (int)((int64_t)rows * (q + 1) / G);
        const int64_t pair = (int64_t)u * g.nx + x;
        int32_t off[MAXWS];
        if constexpr (TM == TM_FULL) {
            row_setup_stored<R>(g, a.T, a.O, a.npairs, pair, false, nullptr, off, nullptr);
            s = window_rows_full<R, VT, KAHAN>(g, a.T + pair, a.npairs, off, a.Vn, r0, r1);
        } else {
            R fac[MAXWS];
            row_setup_stored<R>(g, a.T, a.O, a.npairs, pair, true, fac, off, nullptr);
            s = window_rows_factored<R, VT, KAHAN>(g, fac, off, a.Vn, r0, r1);
        }
    }
    part[q][lane] = s;
    __syncthreads();
    if (q == 0 && x < g.nx) {
        R acc = R(0), comp = R(0);
        for (int i = 0; i < G; ++i) accum<R, KAHAN>(acc, comp, part[i][lane]);
        S[(int64_t)u * g.nx + x] = live ? acc : R(-1);
    }
}

// The same split for rows on the fly.  The pair's masses are computed once
// per block and shared: the pair's mean, origins and kept widths are formed
// once per dim (FP64, which this part issues at 1/64 of the FP32 rate), then
// group q evaluates a contiguous share of the slots of the concatenated
// per-dim windows (each slot's mass as dim_masses computes it) into shared
// memory, laid out [slot][lane]
// so that the row sums read them without bank conflicts; then every group
// sums its window rows from there.
template <class R, class VT, bool KAHAN>
__global__ void __launch_bounds__(32 * ROWS_MAX_GROUPS) k_backup_rows_otf(const __grid_constant__ Geom g,
                                                                          const BackupArgs<R, VT> a,
                                                                          R *__restrict__ S) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *sfac = reinterpret_cast<R *>(smem_raw);                            // [wsum][32]
    int32_t *soff = reinterpret_cast<int32_t *>(sfac + (size_t)g.wsum * 32);  // [wsum][32]
    __shared__ R part[ROWS_MAX_GROUPS][32];
    __shared__ double s_mu[MAXD][32];
    __shared__ int32_t s_o[MAXD][32], s_kmax[MAXD][32];
    const int lane = threadIdx.x, q = threadIdx.y, G = blockDim.y;
    const int32_t x = (int32_t)blockIdx.x * 32 + lane;
    const int32_t u = (int32_t)blockIdx.y;
    const bool live = x < g.nx && !state_masked(a.spec_kind, a.mask[x]);
    if (live && q < g.n) {
        // the pair's mean, window origins and kept widths (FP64), once per
        // dim: group q takes dims q, q + G, ...
        double mu[MAXD];
        mean_of(g, x, u, mu);
        for (int d = q; d < g.n; d += G) {
            const int32_t o = origin_of(g, d, mu[d]);
            s_mu[d][lane] = mu[d];
            s_o[d][lane] = o;
            s_kmax[d][lane] = kept_upper(g, d, mu[d], o);
        }
    }
    __syncthreads();
    if (live) {
        // group q takes a contiguous share of the concatenated slots, so that
        // neighbouring slots of a dim share their edge evaluations
        const int s0 = (int)((int64_t)g.wsum * q / G), s1 = (int)((int64_t)g.wsum * (q + 1) / G);
        int b = 0;
        for (int d = 0; d < g.n && b < s1; b += g.W[d], ++d) {
            const int k0 = max(s0 - b, 0), k1 = min(s1 - b, g.W[d]);
            if (k0 >= k1) continue;
            slot_run(g, d, s_mu[d][lane], s_o[d][lane], s_kmax[d][lane], k0, k1, noise_centre(g, x, d),
                     [&](int k, R m, int32_t f) {
                         sfac[(b + k) * 32 + lane] = m;
                         soff[(b + k) * 32 + lane] = f;
                     },
                     R(0));
        }
    }
    __syncthreads();
    R s = R(0);
    if (live) {
        const int rows = g.wtot / g.W[g.n - 1];
        const int r0 = (int)((int64_t)rows * q / G), r1 = (int)((int64_t)rows * (q + 1) / G);
        s = window_rows_factored<R, VT, KAHAN, 32>(g, sfac + lane, soff + lane, a.Vn, r0, r1);
    }
    part[q][lane] = s;
    __syncthreads();
    if (q == 0 && x < g.nx) {
        R acc = R(0), comp = R(0);
        for (int i = 0; i < G; ++i) accum<R, KAHAN>(acc, comp, part[i][lane]);
        S[(int64_t)u * g.nx + x] = live ? acc : R(-1);
    }
}

// Backup of 2-D problems with per-dimension tables whose windows are too wide
// for the register-resident kernels (the disturbed robot of Sec. 7: 13 x 13
// windows, 121 inputs x 11 disturbance points), in two kernels.
// k_sums_sep2: one thread per (control input, state), states fastest, so that
// a warp's lanes read neighbouring cells of V (L1).  For each disturbance
// point of the input the two dims' table records give the window origins and
// masses; the window sum runs over the rows of dim 0, each row's inner sum in
// slot order, the rows added in order (Kahan-compensated when asked);
// off-grid slots have zero mass and read a clamped cell.  The input's value
// is the min over its disturbance points (Algorithm 4's inner min), and
// max_key[x] keeps the largest (value, -input) key by atomic max: the max
// over inputs with the lowest maximiser, whatever the order of the atomics.
// k_collect_keys then writes V_k and pi_k (spec values on masked states) and
// clears the keys for the next backup.
constexpr int SEP2_WMAX = 16;
// disturbance points of one input whose window sums are unrolled together
#ifndef AMY_SEP2_WUNROLL
#define AMY_SEP2_WUNROLL 1
#endif
constexpr int SEP2_WUNROLL = AMY_SEP2_WUNROLL;
__device__ __forceinline__ unsigned long long sep2_key(float v, int u) {
    // order-preserving map of the float onto 32 bits (negative values below
    // positive ones), then the input complemented: ties favour the lowest input
    uint32_t b = __float_as_uint(v);
    b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    return ((unsigned long long)b << 32) | (unsigned long long)(0xFFFFu - (uint32_t)u);
}
__device__ __forceinline__ float sep2_key_value(unsigned long long k) {
    uint32_t b = (uint32_t)(k >> 32);
    b = (b & 0x80000000u) ? (b & 0x7fffffffu) : ~b;
    return __uint_as_float(b);
}

// Shared-memory form (both dims non-periodic): V_{k+1} staged once per block
// with a zero border of W + 1 cells on each side, so that every window slot
// -- window origins are clamped to [-W - 1, N + 1] -- reads a staged cell and
// the slots of a row are consecutive: one shared load per transition.
__host__ __device__ inline size_t sep2_smem_bytes(int N0, int W0, int N1, int W1) {
    // plus SEP2_WMAX floats of slack after the last row
    return ((size_t)(N0 + 2 * (W0 + 1)) * (size_t)(N1 + 2 * (W1 + 1)) + SEP2_WMAX) * sizeof(float);
}

template <class VT, bool KAHAN, bool SMEM>
__global__ void __launch_bounds__(256) k_sums_sep2(const __grid_constant__ Geom g, const uint32_t *__restrict__ tab,
                                                   const VT *__restrict__ Vn, const uint8_t *__restrict__ mask,
                                                   int32_t spec_kind, unsigned long long *__restrict__ max_key) {
    extern __shared__ float vs[];
    const int nuc = g.nu / g.nw;
    const int64_t total = (int64_t)g.nx * nuc;
    const int32_t N0 = g.N[0], N1 = g.N[1];
    const int W0 = g.W[0], W1 = g.W[1];
    const bool per0 = (g.periodic & 1u) != 0, per1 = (g.periodic & 2u) != 0;
    const int32_t B0 = W0 + 1, B1 = W1 + 1, P1 = N1 + 2 * B1;  // border, padded row
    if (SMEM) {
        const int32_t P0 = N0 + 2 * B0;
        for (int32_t k = threadIdx.x; k < P0 * P1; k += blockDim.x) {
            const int32_t r = k / P1 - B0, c = k - (k / P1) * P1 - B1;
            vs[k] = (r >= 0 && r < N0 && c >= 0 && c < N1) ? vload<float, VT>(Vn + (int64_t)r * N1 + c) : 0.0f;
        }
        __syncthreads();
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t uc = (int32_t)(i / g.nx), x = (int32_t)(i - (int64_t)uc * g.nx);
        if (state_masked(spec_kind, mask[x])) continue;
        const int32_t x0 = x / N1, x1 = x - (x / N1) * N1;
        const int32_t e0 = x0 * g.tsx[0][0] + x1 * g.tsx[0][1], e1 = x0 * g.tsx[1][0] + x1 * g.tsx[1][1];
        float vmin = 0.0f;
#pragma unroll SEP2_WUNROLL
        for (int w = 0; w < g.nw; ++w) {
            const int32_t u = uc * g.nw + w;
            const int32_t *up = reinterpret_cast<const int32_t *>(tab + g.uoff + (int64_t)u * g.urw);
            const uint32_t *r0 = tab + g.toff[0] + (int64_t)(e0 + __ldg(up + 0)) * g.trw[0];
            const uint32_t *r1 = tab + g.toff[1] + (int64_t)(e1 + __ldg(up + 1)) * g.trw[1];
            const int32_t o0 = (int32_t)__ldg(r0);
            // dim 1's record (origin, then W1 masses; 16-byte aligned, padded to
            // 4 words) in 16-byte loads: the lanes of a warp read neighbouring records
            uint32_t rw[SEP2_WMAX + 4];
#pragma unroll
            for (int q = 0; q < (SEP2_WMAX + 4) / 4; ++q) {
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (q * 4 < W1 + 1) v = __ldg(reinterpret_cast<const uint4 *>(r1) + q);
                rw[q * 4 + 0] = v.x;
                rw[q * 4 + 1] = v.y;
                rw[q * 4 + 2] = v.z;
                rw[q * 4 + 3] = v.w;
            }
            const int32_t o1 = (int32_t)rw[0];
            float t1[SEP2_WMAX];
#pragma unroll
            for (int b = 0; b < SEP2_WMAX; ++b) t1[b] = b < W1 ? __uint_as_float(rw[1 + b]) : 0.0f;
            float acc = 0.0f, comp = 0.0f;
            if (SMEM) {
                const float *base = vs + (o0 + B0) * P1 + (o1 + B1);
                for (int a = 0; a < W0; ++a) {
                    const float w0 = __uint_as_float(__ldg(r0 + 1 + a));
                    if (w0 == 0.0f) continue;
                    const float *row = base + a * P1;
                    float r = 0.0f;
#pragma unroll
                    for (int b = 0; b < SEP2_WMAX; ++b)
                        if (b < W1) r = fmaf(t1[b], row[b], r);
                    accum<float, KAHAN>(acc, comp, __fmul_rn(w0, r));
                }
            } else {
                // cells of the window's slots: wrapped (periodic dim) or clamped
                // (off-grid slots have zero mass); the two loops stay apart so
                // that the division is taken only for a periodic dim
                int32_t c1[SEP2_WMAX];
                if (per1) {
                    int32_t c = o1 % N1;
                    if (c < 0) c += N1;
#pragma unroll
                    for (int b = 0; b < SEP2_WMAX; ++b) {
                        c1[b] = c;
                        c = c + 1 == N1 ? 0 : c + 1;
                    }
                } else {
#pragma unroll
                    for (int b = 0; b < SEP2_WMAX; ++b) c1[b] = min(max(o1 + b, 0), N1 - 1);
                }
                int32_t c0w = 0;  // dim 0's first cell, wrapped (periodic dim only)
                if (per0) {
                    c0w = o0 % N0;
                    if (c0w < 0) c0w += N0;
                }
                for (int a = 0; a < W0; ++a) {
                    const float w0 = __uint_as_float(__ldg(r0 + 1 + a));
                    const int32_t c0 = per0 ? c0w : min(max(o0 + a, 0), N0 - 1);
                    c0w = c0w + 1 == N0 ? 0 : c0w + 1;
                    if (w0 == 0.0f) continue;
                    const VT *row = Vn + (int64_t)c0 * N1;
                    float r = 0.0f;
#pragma unroll
                    for (int b = 0; b < SEP2_WMAX; ++b)
                        if (b < W1) r = fmaf(t1[b], vload<float, VT>(row + c1[b]), r);
                    accum<float, KAHAN>(acc, comp, __fmul_rn(w0, r));
                }
            }
            vmin = (w == 0 || acc < vmin) ? acc : vmin;
        }
        atomicMax(max_key + x, sep2_key(vmin, uc));
    }
}

template <class VT>
__global__ void __launch_bounds__(256) k_collect_keys(const __grid_constant__ Geom g, const uint8_t *__restrict__ mask,
                                                      int32_t spec_kind, unsigned long long *__restrict__ max_key,
                                                      VT *__restrict__ Vo, float *__restrict__ Vfinal,
                                                      uint16_t *__restrict__ pi) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.nx; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = (int32_t)i;
        const uint8_t f = mask[x];
        float best;
        uint16_t arg;
        if (state_masked(spec_kind, f)) {
            best = (spec_kind != SPEC_SAFETY && (f & F_TARGET)) ? 1.0f : 0.0f;
            arg = 0xFFFF;
        } else {
            const unsigned long long k = max_key[x];
            best = sep2_key_value(k);
            arg = (uint16_t)(0xFFFFu - (uint32_t)(k & 0xFFFFu));
        }
        max_key[x] = 0ull;
        Vo[x] = vstore_cast<VT, float>(best);
        if (Vfinal) Vfinal[x] = best;
        if (pi) pi[x] = arg;
    }
}

// Max over inputs of S[u][x] per state, lowest maximiser, spec values on
// masked states (the collect step of k_backup).
template <class R, class VT>
__global__ void __launch_bounds__(256) k_argmax_rows(const __grid_constant__ Geom g, const BackupArgs<R, VT> a,
                                                     const R *__restrict__ S) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.nx; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = (int32_t)i;
        const uint8_t f = a.mask[x];
        R best;
        uint16_t arg;
        if (state_masked(a.spec_kind, f)) {
            best = (a.spec_kind != SPEC_SAFETY && (f & F_TARGET)) ? R(1) : R(0);
            arg = 0xFFFF;
        } else {
            best = R(-1);
            arg = 0;
            // each input's value: min over its disturbance block (nw = 1: none)
            for (int u = 0; u < g.nu / g.nw; ++u) {
                R s = S[(int64_t)(u * g.nw) * g.nx + x];
                for (int w = 1; w < g.nw; ++w) s = min_r(s, S[(int64_t)(u * g.nw + w) * g.nx + x]);
                if (s > best) {
                    best = s;
                    arg = (uint16_t)u;
                }
            }
        }
        a.Vo[x] = vstore_cast<VT, R>(best);
        if (a.Vfinal) a.Vfinal[x] = best;
        if (a.pi) a.pi[x] = arg;
    }
}

// ---------------------------------------------------------------------------
// Stored T construction (Algorithm 2): one thread per (x, u) pair.
// ---------------------------------------------------------------------------
template <class R, int TM>
__global__ void __launch_bounds__(128) k_build(const __grid_constant__ Geom g, R *__restrict__ T,
                                               int16_t *__restrict__ O, int64_t npairs) {
    R fac[MAXWS];
    int32_t off[MAXWS];
    int32_t org[MAXD];
    for (int64_t pair = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pair < npairs;
         pair += (int64_t)gridDim.x * blockDim.x) {
        const int32_t u = (int32_t)(pair / g.nx);
        const int32_t x = (int32_t)(pair - (int64_t)u * g.nx);
        row_setup_otf<R>(g, x, u, fac, off, org);
        for (int d = 0; d < g.n; ++d) O[d * npairs + pair] = (int16_t)org[d];
        if (TM == TM_FACTORED) {
            for (int j = 0; j < g.wsum; ++j) T[(int64_t)j * npairs + pair] = fac[j];
        } else {
            int k[MAXD], fb[MAXD];
            int acc = 0;
            for (int d = 0; d < g.n; ++d) {
                fb[d] = acc;
                acc += g.W[d];
                k[d] = 0;
            }
            for (int t = 0; t < g.wtot; ++t) {
                R v = R(1);
                for (int d = 0; d < g.n; ++d) v = v * fac[fb[d] + k[d]];
                T[(int64_t)t * npairs + pair] = v;
                for (int d = g.n - 1; d >= 0; --d) {
                    if (++k[d] < g.W[d]) break;
                    k[d] = 0;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Row query: origin and window probabilities (double) of listed pairs.
// ---------------------------------------------------------------------------
template <class R>
__global__ void k_query_rows(const __grid_constant__ Geom g, int32_t tmode, const R *__restrict__ T,
                             const int16_t *__restrict__ O, int64_t npairs, const uint32_t *__restrict__ tab,
                             const int64_t *__restrict__ qx,
                             const int64_t *__restrict__ qu, int64_t count, int32_t *__restrict__ origin_out,
                             double *__restrict__ probs_out) {
    R fac[MAXWS];
    int32_t off[MAXWS];
    int32_t org[MAXD];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = (int32_t)qx[i], u = (int32_t)qu[i];
        const int64_t pair = (int64_t)u * g.nx + x;
        if (tmode == TM_OTF)
            row_setup_otf<R>(g, x, u, fac, off, org);
        else if (tmode == TM_SEPARABLE) {
            if constexpr (sizeof(R) == 4) row_setup_sep(g, tab, x, u, fac, off, org);
        } else
            row_setup_stored<R>(g, T, O, npairs, pair, tmode == TM_FACTORED, fac, off, org);
        for (int d = 0; d < g.n; ++d) origin_out[i * g.n + d] = org[d];
        int k[MAXD], fb[MAXD];
        int acc = 0;
        for (int d = 0; d < g.n; ++d) {
            fb[d] = acc;
            acc += g.W[d];
            k[d] = 0;
        }
        for (int t = 0; t < g.wtot; ++t) {
            double v;
            if (tmode == TM_FULL) {
                v = (double)T[(int64_t)t * npairs + pair];
            } else {
                R pr = R(1);
                for (int d = 0; d < g.n; ++d) pr = pr * fac[fb[d] + k[d]];
                v = (double)pr;
            }
            probs_out[i * (int64_t)g.wtot + t] = v;
            for (int d = g.n - 1; d >= 0; --d) {
                if (++k[d] < g.W[d]) break;
                k[d] = 0;
            }
        }
    }
}

}  // namespace amy
