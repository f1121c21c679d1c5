// amy_staged.cuh -- fused backup + max/argmax (Algorithm 4) for low-dimensional
// problems (n <= 3) whose windows all have width WM: the union of the
// successor windows of a block's tile is staged once in shared memory and
// every window gather reads it with 32-bit shared-memory addresses.
//
// A block owns tileX consecutive states and all their inputs (same thread
// mapping as amy_fast.cuh).  Pass 1 collects, per dim, the smallest and
// largest window origin over the tile's (state, input) items; the box
// [lo, hi + WM) is loaded from V_{k+1} (periodic dims wrap, off-grid cells
// hold 0 -- their mass is zero); pass 2 forms each item's window sum from the
// box.  A block whose box exceeds the shared-memory budget runs the
// register-resident body of amy_fast.cuh instead.  The arithmetic (masses,
// products and summation order) is that of amy_fast.cuh, so both give
// bit-identical values.
#pragma once

#include <climits>
#include <type_traits>

#include "amy_fast.cuh"

namespace amy {

constexpr int STAGE_BOX_FLOATS = 6144;  // default staging box per block (24 KiB)
constexpr int STAGE_UP_MAX = 512;       // inputs whose table-index parts are staged too
constexpr int STAGE_TAB_WORDS = 4096;   // inner-dim table staged when at most this many words
constexpr int STAGE_MAX_THREADS = 512;  // threads per block of the staged kernel

// The register-resident body's area (its odometer arrays, laid out for
// FAST_THREADS, and the lane-merge arrays, one entry per thread).
__host__ __device__ inline size_t staged_work_bytes(int n, int WM, int threads) {
    const size_t a = fast_smem_bytes(n, WM), b = (size_t)threads * 8;
    return a > b ? a : b;
}

// Shared memory of one block: the staging box, the work area, the inputs'
// table-index parts and, for the per-run pass, the innermost dim's table
// (tab_words, 0 = not staged).
__host__ __device__ inline size_t staged_smem_bytes(int n, int WM, int box_floats, int nu, int tab_words,
                                                    int threads) {
    return (size_t)box_floats * 4 + staged_work_bytes(n, WM, threads) +
           (nu <= STAGE_UP_MAX ? (size_t)nu * 16 : 0) + (size_t)tab_words * 4;
}

// Mean of one (state, input) pair from the state's precomputed FP64 centres
// (same operation order as mean_of).
__device__ __forceinline__ void item_mean(const Geom &g, int32_t u, const double *xc, double cth, double sth,
                                          double *mu) {
    const int n = g.n;
    if (g.sys == SYS_AFFINE) {
        const double *A = g.params + (int64_t)u * (n * n + n);
        const double *cc = A + n * n;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            mu[i] = 0.0;
            if (i < n) {
                double acc = 0.0;
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    if (j < n) acc = dadd(acc, dmul(__ldg(A + i * n + j), xc[j]));
                mu[i] = dadd(acc, __ldg(cc + i));
            }
        }
    } else {
        const int32_t uw = u % g.ucount[1];
        const int32_t uv = u / g.ucount[1];
        const double v = dadd(g.ulb[0], dmul((double)uv, g.ueta[0]));
        const double w = dadd(g.ulb[1], dmul((double)uw, g.ueta[1]));
        const double tau = __ldg(g.params);
        const double tv = dmul(tau, v);
        mu[0] = dadd(xc[0], dmul(tv, cth));
        mu[1] = dadd(xc[1], dmul(tv, sth));
        mu[2] = dadd(xc[2], dmul(tau, w));
    }
}

// Asynchronous global -> shared copy of one 4-byte word (cp.async, cached in
// L1) and the wait for all of this thread's outstanding copies.
__device__ __forceinline__ void cp_async4(float *smem_dst, const float *gmem_src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    const size_t gsrc = __cvta_generic_to_global(gmem_src);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Extra inner-dim slots, beyond the window width, that one cached outer
// contraction may span (inputs whose inner windows start up to this many
// cells apart share it).
constexpr int STAGE_KX = 3;

// Window sums of one state for the inputs [u0, u1) when inputs come in runs
// that share every outer dim's record (same masses and origins; e.g. the
// unicycle's speed fixes the x and y rows and only the turn rate moves the
// heading window).  For a run, the outer dims are contracted once over the K
// inner slots [r0, r0 + K) that any input's inner window can reach,
//   R[k] = sum_i t0_i * (sum_j t1_j * V[o0 + i, o1 + j, r0 + k])   (NS = 3),
// and each input then needs only its inner row: s = sum_k tL_k * R[oL - r0 + k].
// R depends only on the state and the run's records, so the result does not
// depend on how inputs are split over threads.  BOX: V from the staged
// shared-memory box; otherwise from global memory with clamped / wrapped
// cells (off-grid cells carry zero mass either way, so both give the same
// bits).
template <class VT, int WM, int NS, bool BOX>
__device__ __forceinline__ void grouped_items(const Geom &g, const FastArgs<VT> &a, const int4 *up,
                                              const uint4 *tabL, const int32_t (&xi)[MAXD], const int32_t (&es)[3], int32_t u0,
                                              int32_t u1, int32_t dminL, int32_t K, const float *sbox,
                                              const int32_t (&blo)[3], const int32_t (&bs)[3], float &best,
                                              int32_t &arg) {
    constexpr int L = NS - 1;
    constexpr int KM = WM + STAGE_KX;
    constexpr int NQ = (WM + 1 + 3) / 4;  // uint4 words of one record (origin + WM masses)
    if (u0 >= u1) return;
    float R[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) R[k] = 0.0f;
    int32_t key0 = INT_MIN, key1 = INT_MIN;
    const int32_t r0 = xi[L] + dminL;  // first inner slot of R (unwrapped)
    // this state's records of the inner dim: record es[L] + ui[L] of table L
    const uint4 *recL = tabL + (int64_t)es[L] * NQ;
    // one input ahead: its table-index parts and its inner record are loaded
    // while the current input is summed
    int4 uv_n = up[u0];
    uint4 rq_n[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) rq_n[q] = recL[(int64_t)(NS == 3 ? uv_n.z : uv_n.y) * NQ + q];
    for (int32_t u = u0; u < u1; ++u) {
        const int4 uv = uv_n;
        uint4 rq[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) rq[q] = rq_n[q];
        if (u + 1 < u1) {
            uv_n = up[u + 1];
#pragma unroll
            for (int q = 0; q < NQ; ++q) rq_n[q] = recL[(int64_t)(NS == 3 ? uv_n.z : uv_n.y) * NQ + q];
        }
        const int32_t k0 = es[0] + uv.x;
        const int32_t k1 = NS == 3 ? es[1] + uv.y : 0;
        if (k0 != key0 || k1 != key1) {
            key0 = k0;
            key1 = k1;
            int32_t o[2] = {0, 0};
            float t[2][WM];
#pragma unroll
            for (int d = 0; d < L; ++d) {
                const uint4 *rec = reinterpret_cast<const uint4 *>(a.tab + g.toff[d]) + (int64_t)(d == 0 ? k0 : k1) * NQ;
                uint32_t wds[NQ * 4];
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const uint4 v = __ldg(rec + q);
                    wds[q * 4 + 0] = v.x;
                    wds[q * 4 + 1] = v.y;
                    wds[q * 4 + 2] = v.z;
                    wds[q * 4 + 3] = v.w;
                }
                o[d] = (int32_t)wds[0];
#pragma unroll
                for (int k = 0; k < WM; ++k) t[d][k] = __uint_as_float(wds[1 + k]);
            }
            if (BOX) {
                int32_t base = r0 - blo[L];
#pragma unroll
                for (int d = 0; d < L; ++d) base += (o[d] - blo[d]) * bs[d];
#pragma unroll
                for (int kk = 0; kk < KM; ++kk) {
                    if (kk < K) {
                        float acc = 0.0f, comp = 0.0f;
#pragma unroll
                        for (int i = 0; i < WM; ++i) {
                            const float *pr = sbox + base + i * bs[0] + kk;
                            float inner;
                            if (NS == 3) {
                                inner = 0.0f;
#pragma unroll
                                for (int j = 0; j < WM; ++j) inner = fmaf(t[1][j], pr[j * bs[1]], inner);
                            } else {
                                inner = pr[0];
                            }
                            accum_row(acc, comp, __fmul_rn(t[0][i], inner), a.kahan);
                        }
                        R[kk] = acc;
                    }
                }
            } else {
                int32_t of0[WM], of1[WM], ofL[KM];
                dim_offsets_reg<WM>(g, 0, o[0], WM, of0);
                if (NS == 3) dim_offsets_reg<WM>(g, 1, o[1], WM, of1);
                dim_offsets_reg<KM>(g, L, r0, K, ofL);
#pragma unroll
                for (int kk = 0; kk < KM; ++kk) {
                    if (kk < K) {
                        float acc = 0.0f, comp = 0.0f;
#pragma unroll
                        for (int i = 0; i < WM; ++i) {
                            float inner;
                            if (NS == 3) {
                                inner = 0.0f;
#pragma unroll
                                for (int j = 0; j < WM; ++j)
                                    inner = fmaf(t[1][j], vload<float, VT>(a.Vn + (of0[i] + of1[j] + ofL[kk])), inner);
                            } else {
                                inner = vload<float, VT>(a.Vn + (of0[i] + ofL[kk]));
                            }
                            accum_row(acc, comp, __fmul_rn(t[0][i], inner), a.kahan);
                        }
                        R[kk] = acc;
                    }
                }
            }
        }
        // the input's own inner row: s = sum_k tL_k * R[sh + k], sh = oL - r0 in [0, K - WM]
        uint32_t wds[NQ * 4];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            wds[q * 4 + 0] = rq[q].x;
            wds[q * 4 + 1] = rq[q].y;
            wds[q * 4 + 2] = rq[q].z;
            wds[q * 4 + 3] = rq[q].w;
        }
        const int32_t sh = (int32_t)wds[0] - r0;
        float w[WM];
#pragma unroll
        for (int k = 0; k < WM; ++k) w[k] = R[k];
#pragma unroll
        for (int q = 1; q <= STAGE_KX; ++q) {
            if (sh >= q) {
#pragma unroll
                for (int k = 0; k < WM; ++k) w[k] = R[q + k];
            }
        }
        float sum = 0.0f;
#pragma unroll
        for (int k = 0; k < WM; ++k) sum = fmaf(__uint_as_float(wds[1 + k]), w[k], sum);
        if (sum > best) {
            best = sum;
            arg = u;
        }
    }
}

template <class VT, int WM, int TM, int NS>
__global__ void __launch_bounds__(STAGE_MAX_THREADS) k_backup_staged(const __grid_constant__ Geom g,
                                                                const FastArgs<VT> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int BT = blockDim.x;
    float *sbox = reinterpret_cast<float *>(smem_raw);
    unsigned char *work = smem_raw + (size_t)a.box_floats * 4;  // also the fallback's area
    int4 *s_up = reinterpret_cast<int4 *>(work + staged_work_bytes(NS, WM, BT));
    uint4 *s_tabL = reinterpret_cast<uint4 *>(s_up + (g.nu <= STAGE_UP_MAX ? g.nu : 0));
    float *cBest = reinterpret_cast<float *>(work);
    int32_t *cArg = reinterpret_cast<int32_t *>(cBest + BT);
    __shared__ int32_t s_lo[3], s_hi[3];

    const int tid = threadIdx.x;
    const int TX = a.tileX, UL = a.ulanes;
    const int xl = tid % TX;
    const int c = tid / TX;
    int32_t x;
    if (NS >= 2 && a.rowtile > 0) {
        // row-aligned tile: lane column xl = (row r, chunk ch, lane) of rowtile
        // consecutive innermost-dim rows (within one outermost index when NS = 3)
        const int RW = a.rowtile;
        const int CHU = TX / (32 * RW);
        const int32_t R = g.N[NS - 1];
        const int r = (xl >> 5) / CHU;
        const int32_t k_in = ((xl >> 5) % CHU) * 32 + (xl & 31);
        int32_t row;
        bool ok;
        if (NS == 3) {
            const int32_t t1 = (g.N[1] + RW - 1) / RW;
            const int32_t i1 = (int32_t)(blockIdx.x % t1) * RW + r;
            row = (int32_t)(blockIdx.x / t1) * g.N[1] + i1;
            ok = i1 < g.N[1];
        } else {
            row = (int32_t)blockIdx.x * RW + r;
            ok = row < g.N[0];
        }
        x = (ok && k_in < R) ? row * R + k_in : INT_MAX;
    } else {
        x = (int32_t)blockIdx.x * TX + xl;
    }
    if (tid < 3) {
        s_lo[tid] = INT_MAX;
        s_hi[tid] = INT_MIN;
    }
    const bool active = x >= 0 && x < g.nx;
    const uint8_t f = active ? a.mask[x] : (uint8_t)0;
    const bool masked = active && state_masked(a.spec_kind, f);
    const bool work_items = active && !masked;

    int32_t xi[MAXD];
    double xc[3] = {0.0, 0.0, 0.0};
    int32_t es[3] = {0, 0, 0};
    double cth = 0.0, sth = 0.0;
    if (work_items) {
        decode_state(g, x, xi);
#pragma unroll
        for (int d = 0; d < NS; ++d) {
            if (TM == TM_OTF) xc[d] = state_centre(g, d, xi[d]);
            if (TM == TM_SEPARABLE) {
                int32_t e = 0;
#pragma unroll
                for (int j = 0; j < NS; ++j) e += xi[j] * g.tsx[d][j];
                es[d] = e;
            }
        }
        if (TM == TM_OTF && g.sys == SYS_UNICYCLE) {
            cth = cos(xc[2]);
            sth = sin(xc[2]);
        }
    }
    // per-item origins (and masses in pass 2) of every dim
    auto item = [&](int32_t u, int32_t (&o)[3], float (&t)[3][WM], bool want_masses) {
        if (TM == TM_OTF) {
            double mu[3];
            item_mean(g, u, xc, cth, sth, mu);
#pragma unroll
            for (int d = 0; d < NS; ++d) {
                o[d] = origin_of(g, d, mu[d]);
                if (want_masses) {
                    int32_t ok[WM];
                    dim_masses_reg<WM>(g, d, mu[d], o[d], WM, xc[d], t[d], ok);
                }
            }
        } else {  // TM_SEPARABLE
            const int4 *up = reinterpret_cast<const int4 *>(a.tab + g.uoff + (int64_t)u * g.urw);
            const int4 uv = __ldg(up);
            const int32_t ui[3] = {uv.x, uv.y, uv.z};
#pragma unroll
            for (int d = 0; d < NS; ++d) {
                const uint4 *rec = reinterpret_cast<const uint4 *>(a.tab + g.toff[d] + (int64_t)(es[d] + ui[d]) * g.trw[d]);
                constexpr int NQ = (WM + 1 + 3) / 4;
                uint32_t wds[NQ * 4];
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    uint4 v = make_uint4(0u, 0u, 0u, 0u);
                    if (q == 0 || want_masses) v = __ldg(rec + q);
                    wds[q * 4 + 0] = v.x;
                    wds[q * 4 + 1] = v.y;
                    wds[q * 4 + 2] = v.z;
                    wds[q * 4 + 3] = v.w;
                }
                o[d] = (int32_t)wds[0];
                if (want_masses) {
#pragma unroll
                    for (int k = 0; k < WM; ++k) t[d][k] = __uint_as_float(wds[1 + k]);
                }
            }
        }
    };

    // pass 1: the tile's window box -- from the tables' bounds on (origin -
    // own coordinate) when every dim has one, else from the items' origins
    const int32_t *rb = TM == TM_SEPARABLE ? reinterpret_cast<const int32_t *>(a.tab + g.boff) : nullptr;
    const bool analytic = rb && ((__ldg(rb + 2 * MAXD) & ((1 << NS) - 1)) == ((1 << NS) - 1));
    int32_t lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    if (work_items) {
        if (analytic) {
#pragma unroll
            for (int d = 0; d < NS; ++d) {
                lo[d] = xi[d] + __ldg(rb + d);
                hi[d] = xi[d] + __ldg(rb + MAXD + d);
            }
        } else {
            for (int32_t u = c; u < g.nu; u += UL) {
                int32_t o[3];
                float t[3][WM];
                item(u, o, t, false);
#pragma unroll
                for (int d = 0; d < NS; ++d) {
                    lo[d] = min(lo[d], o[d]);
                    hi[d] = max(hi[d], o[d]);
                }
            }
        }
    }
    __syncthreads();
    {
        // one shared atomic per warp and dim (with table bounds, the first
        // input lane of each state speaks for all of them)
        const bool contrib = work_items && (!analytic || c == 0);
#pragma unroll
        for (int d = 0; d < NS; ++d) {
            const int32_t l = __reduce_min_sync(0xffffffffu, contrib ? lo[d] : INT_MAX);
            const int32_t h = __reduce_max_sync(0xffffffffu, contrib ? hi[d] : INT_MIN);
            if ((tid & 31) == 0 && l != INT_MAX) {
                atomicMin(&s_lo[d], l);
                atomicMax(&s_hi[d], h);
            }
        }
    }
    __syncthreads();
    int32_t blo[3] = {0, 0, 0}, bn[3] = {1, 1, 1}, bs[3] = {0, 0, 0};
    int64_t vol = 1;
    const bool any = s_lo[0] != INT_MAX;
#pragma unroll
    for (int d = 0; d < NS; ++d) {
        blo[d] = any ? s_lo[d] : 0;
        bn[d] = any ? (s_hi[d] - s_lo[d] + WM) : 1;
        vol *= bn[d];
    }
    // inputs in runs sharing their outer records: contract the outer dims
    // once per run (decided per launch from the tables, the same in every block)
    constexpr int L = NS - 1;
    int32_t dminL = 0, KL = 0;
    bool grouped = false;
    if (TM == TM_SEPARABLE && NS >= 2 && a.grouped && analytic) {
        dminL = __ldg(rb + L);
        KL = __ldg(rb + MAXD + L) - dminL + WM;
        // (K <= N keeps a wrapped row of K cells to one lap of a periodic dim)
        // (records of 4*NQ words and 4-word table-index parts are assumed)
        bool strides = g.urw == 4;
#pragma unroll
        for (int d = 0; d < NS; ++d) strides = strides && g.trw[d] == 4 * ((WM + 1 + 3) / 4);
        grouped = strides && KL >= WM && KL <= WM + STAGE_KX && KL <= g.N[L];
    }
    const bool fits = vol <= a.box_floats;
    if (!fits && !grouped) {
        // this tile's windows spread too far: the register-resident body
        backup_tile<VT, WM, TM, VAR_EXACT>(g, a, x, work);
        return;
    }
    if (fits) {
        // row stride padded to a multiple of 32 floats when it fits: lanes whose
        // windows differ by whole rows then still hit distinct banks
        int32_t inner = bn[NS - 1];
        const int32_t padded = (inner + 31) / 32 * 32;
        if (NS > 1 && (vol / inner) * padded <= a.box_floats) inner = padded;
        int32_t s = 1;
#pragma unroll
        for (int d = NS - 1; d >= 0; --d) {
            bs[d] = s;
            s *= (d == NS - 1) ? inner : bn[d];
        }
    }
    // stage the box: periodic dims wrap, off-grid cells hold 0 (zero mass
    // there).  A warp takes one box row (outer coordinates decoded once per
    // row) and its lanes walk the innermost extent; the innermost cell wraps
    // or clips with a compare per element.
    if (any && fits) {
        const int32_t inner = bn[NS - 1];
        const int32_t nrows = (int32_t)(vol / inner);
        const int d_in = NS - 1;
        const int32_t Nin = g.N[d_in], st_in = g.stride[d_in];
        const bool per_in = (g.periodic >> d_in) & 1u;
        const int lane = tid & 31;
        for (int32_t rr = tid >> 5; rr < nrows; rr += (int32_t)(blockDim.x >> 5)) {
            int64_t lin = 0;
            int32_t sidx = 0;
            bool on = true;
            int32_t q = rr;
#pragma unroll
            for (int d = NS - 2; d >= 0; --d) {
                const int32_t kd = q % bn[d];
                q /= bn[d];
                bool ond;
                const int32_t cell = cell_of(g, d, blo[d] + kd, ond);
                on = on && ond;
                lin += (int64_t)cell * g.stride[d];
                sidx += kd * bs[d];
            }
            for (int32_t k = lane; k < inner; k += 32) {
                int32_t cin = blo[d_in] + k;
                bool onk = on;
                if ((uint32_t)cin >= (uint32_t)Nin) {
                    if (per_in) {
                        cin %= Nin;
                        cin = cin < 0 ? cin + Nin : cin;
                    } else {
                        onk = false;
                        cin = 0;
                    }
                }
                if constexpr (std::is_same<VT, float>::value) {
                    // FP32 V: asynchronous 4-byte copies, all of this thread's
                    // cells in flight at once (completed before the barrier)
                    if (onk)
                        cp_async4(sbox + sidx + k, a.Vn + lin + (int64_t)cin * st_in);
                    else
                        sbox[sidx + k] = 0.0f;
                } else {
                    sbox[sidx + k] = onk ? vload<float, VT>(a.Vn + lin + (int64_t)cin * st_in) : 0.0f;
                }
            }
        }
        if constexpr (std::is_same<VT, float>::value) cp_async_wait_all();
    }
    // the inputs' table-index parts and the innermost dim's table, for the
    // per-run pass (read through generic pointers: shared or global)
    const int4 *up = reinterpret_cast<const int4 *>(a.tab + g.uoff);
    const uint4 *tabL = reinterpret_cast<const uint4 *>(a.tab + g.toff[L]);
    if (TM == TM_SEPARABLE && grouped) {
        if (g.nu <= STAGE_UP_MAX) {
            for (int32_t u = tid; u < g.nu; u += (int32_t)blockDim.x) s_up[u] = __ldg(up + u);
            up = s_up;
        }
        if (a.stage_tab > 0) {
            for (int32_t i = tid; i < a.stage_tab / 4; i += (int32_t)blockDim.x) s_tabL[i] = __ldg(tabL + i);
            tabL = s_tabL;
        }
    }
    __syncthreads();

    // pass 2: window sums from the box (summation order of amy_fast.cuh), or
    // per run of inputs sharing their outer records
    float best = -1.0f;
    int32_t arg = 0x7fffffff;
    if (work_items && grouped) {
        if constexpr (TM == TM_SEPARABLE && NS >= 2) {
            // a run belongs to the lane whose share [c*chunk, (c+1)*chunk) holds
            // its first input, so no lane repeats another's outer contraction
            const int32_t chunk = (g.nu + UL - 1) / UL;
            auto run_start = [&](int32_t u) {
                if (u <= 0 || u >= g.nu) return true;
                const int4 p = up[u - 1], q = up[u];
                return p.x != q.x || (NS == 3 && p.y != q.y);
            };
            int32_t u0 = min(g.nu, c * chunk), u1 = min(g.nu, u0 + chunk);
            while (!run_start(u0)) ++u0;
            while (!run_start(u1)) ++u1;
            if (fits)
                grouped_items<VT, WM, NS, true>(g, a, up, tabL, xi, es, u0, u1, dminL, KL, sbox, blo, bs, best,
                                                arg);
            else
                grouped_items<VT, WM, NS, false>(g, a, up, tabL, xi, es, u0, u1, dminL, KL, sbox, blo, bs, best,
                                                 arg);
        }
    } else if (work_items) {
        for (int32_t u = c; u < g.nu; u += UL) {
            int32_t o[3];
            float t[3][WM];
            item(u, o, t, true);
            int32_t base = 0;
#pragma unroll
            for (int d = 0; d < NS; ++d) base += (o[d] - blo[d]) * bs[d];
            const float *pb = sbox + base;
            float s;
            if (NS == 1) {
                float r = 0.0f;
#pragma unroll
                for (int k = 0; k < WM; ++k) r = fmaf(t[0][k], pb[k], r);
                s = r;
            } else if (NS == 2) {
                s = 0.0f;
#pragma unroll
                for (int j = 0; j < WM; ++j) {
                    const float *pr = pb + j * bs[0];
                    float r = 0.0f;
#pragma unroll
                    for (int k = 0; k < WM; ++k) r = fmaf(t[1][k], pr[k], r);
                    s = fmaf(t[0][j], r, s);
                }
            } else {
                float acc = 0.0f, comp = 0.0f;
#pragma unroll
                for (int i = 0; i < WM; ++i) {
                    const float *pi = pb + i * bs[0];
                    float inner = 0.0f;
#pragma unroll
                    for (int j = 0; j < WM; ++j) {
                        const float *pr = pi + j * bs[1];
                        float r = 0.0f;
#pragma unroll
                        for (int k = 0; k < WM; ++k) r = fmaf(t[2][k], pr[k], r);
                        inner = fmaf(t[1][j], r, inner);
                    }
                    const float term = __fmul_rn(__fmul_rn(1.0f, t[0][i]), inner);
                    accum_row(acc, comp, term, a.kahan);
                }
                s = acc;
            }
            if (s > best) {
                best = s;
                arg = u;
            }
        }
    }
    cBest[tid] = best;
    cArg[tid] = arg;
    __syncthreads();
    if (c == 0 && active) {
        for (int l = 1; l < UL; ++l) {
            const float b2 = cBest[l * TX + xl];
            const int32_t a2 = cArg[l * TX + xl];
            if (b2 > best || (b2 == best && a2 < arg)) {
                best = b2;
                arg = a2;
            }
        }
        uint16_t pol;
        if (masked) {
            best = (a.spec_kind != SPEC_SAFETY && (f & F_TARGET)) ? 1.0f : 0.0f;
            pol = 0xFFFF;
        } else {
            pol = (uint16_t)arg;
        }
        a.Vo[x] = vstore_cast<VT, float>(best);
        if (a.Vfinal) a.Vfinal[x] = best;
        if (a.pi) a.pi[x] = pol;
    }
}

}  // namespace amy
