// amy_runs.cuh -- fused backup + max/argmax (Algorithm 4) with one outer
// contraction per run of inputs, for 2-D and 3-D problems with per-dimension
// tables whose consecutive inputs come in runs that share every outer dim's
// table record (the unicycle: a speed fixes the x and y rows of the window,
// the turn rates of that speed move only the heading row).
//
// A block owns a tile of whole innermost-dim rows (for 3-D problems, `outer`
// values of dim 0 by RW rows of dim 1; for 2-D, RW rows) and all inputs; lane p of a warp
// holds innermost coordinate p (plus 32 per chunk of longer rows), and lane
// group c of a state takes the runs c, c + UL, c + 2 UL, ...  The state's
// coordinates come from the tile mapping, without divisions.  Per (state,
// run) the outer dims are contracted over the K inner slots r0 + k,
// r0 = own inner coordinate + the smallest inner origin offset, that any
// input of the run reaches,
//   R[k] = sum_i t0_i * (sum_j t1_j * V[o0 + i, o1 + j, r0 + k]),
// and each input of the run then needs only its own inner row,
//   s(x, u) = sum_k tL_k * R[oL - r0 + k].
// This is the window sum of Algorithm 4 reassociated: the same terms, with the
// outer factors shared by the run.
//
// Shared memory holds:
//  * the tile's window box in a sliding layout: entry (o0, o1, p) of plane q
//    is the float4 V[o0, o1, r0(p) + 4q .. r0(p) + 4q + 3] of the state at
//    inner coordinate p, so one 16-byte load per plane gives all K inner
//    slots of one outer cell (periodic dims wrap, off-grid cells hold 0 --
//    their mass is zero);
//  * the innermost dim's table as shifted weights: record (own inner
//    coordinate p, input part) holds tL at positions sh .. sh + W - 1 of K,
//    sh = oL - r0(p), zeros elsewhere;
//  * the inputs' table-index parts and the run starts.
// Each input's sum is then the chain of fused multiply-adds
// sum_{k < K} w_k * R[k] from 0, which is the same chain as
// sum_k tL_k * R[sh + k]: the leading zero weights leave +0 (R >= 0) and the
// trailing ones add +0.  The arithmetic (products, summation order, Kahan
// compensation) is that of the staged kernel's per-run pass, so both give
// the same bits.  K = W + KX (KX = 0..3) and the compensation are
// compile-time constants; a tile whose box exceeds its shared-memory budget
// reads V from global memory with the same arithmetic.
#pragma once

#include <climits>
#include <type_traits>

#include "amy_staged.cuh"

namespace amy {

constexpr int RUNS_MAX_THREADS = 512;
constexpr int RUNS_MAX_INPUTS = 512;     // inputs whose table-index parts and run starts are staged
constexpr int RUNS_BOX_DEFAULT = 16384;  // box budget (floats) when the table bounds are not known on the host

// 16-byte planes of one sliding entry for inner span K.
__host__ __device__ constexpr int runs_planes(int K) { return (K + 3) / 4; }

// Sliding-box floats of one tile: rows x entries per row (the inner extent
// padded to 8 entries) x planes x 4.
__host__ __device__ inline int64_t runs_box_floats(int64_t nrows, int32_t inner_n, int K) {
    return nrows * (int64_t)((inner_n + 7) & ~7) * runs_planes(K) * 4;
}

// Shared memory of one block: the sliding box, the work area (lane merge, or
// the register-resident fallback), the inputs' table-index parts, the run
// starts, each input's inner-record byte offset and the shifted inner table
// (planes float4s per record).
__host__ __device__ inline size_t runs_smem_bytes(int n, int WM, int box_floats, int nu, int tab_records, int planes,
                                                  int threads) {
    return (size_t)box_floats * 4 + staged_work_bytes(n, WM, threads) + (size_t)nu * 16 +
           (size_t)((nu + 1 + 3) / 4) * 16 + (size_t)((nu + 3) / 4) * 16 + (size_t)tab_records * planes * 16;
}

// Asynchronous 4-byte global -> shared copy that writes zero instead when
// bytes == 0 (src must still be a valid address).
__device__ __forceinline__ void cp_async4_zfill(float *smem_dst, const float *gmem_src, unsigned bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    const size_t gsrc = __cvta_generic_to_global(gmem_src);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gsrc), "r"(bytes) : "memory");
}

// The outer records (window origin + WM masses) of one run: table d at
// record es[d] + the run's input part for d.
template <int WM, int NS>
struct RunRecs {
    uint4 q[2][(WM + 1 + 3) / 4];
};
template <int WM, int NS>
__device__ __forceinline__ void run_records(const Geom &g, const uint32_t *tab, int4 uv, const int32_t (&es)[3],
                                            RunRecs<WM, NS> &rr) {
    constexpr int NQ = (WM + 1 + 3) / 4;
#pragma unroll
    for (int d = 0; d < NS - 1; ++d) {
        const uint4 *rec =
            reinterpret_cast<const uint4 *>(tab + g.toff[d]) + (int64_t)(es[d] + (d == 0 ? uv.x : uv.y)) * NQ;
#pragma unroll
        for (int q = 0; q < NQ; ++q) rr.q[d][q] = __ldg(rec + q);
    }
}

// 16- and 4-byte shared-memory loads at a 32-bit shared address.
__device__ __forceinline__ float4 lds_f4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr));
    return v;
}
__device__ __forceinline__ int32_t lds_i32(uint32_t addr) {
    int32_t v;
    asm volatile("ld.shared.b32 %0, [%1];\n" : "=r"(v) : "r"(addr));
    return v;
}

// Loads of V at L2 (not cached in L1), widened to FP32.
__device__ __forceinline__ float ld_cg(const float *p) {
    float v;
    asm volatile("ld.global.cg.f32 %0, [%1];\n" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_cg(const __nv_bfloat16 *p) {
    unsigned short b;
    asm volatile("ld.global.cg.u16 %0, [%1];\n" : "=h"(b) : "l"(p));
    return bf16_unfold(__ushort_as_bfloat16(b));
}
__device__ __forceinline__ float ld_cg(const unorm16 *p) {
    unsigned short b;
    asm volatile("ld.global.cg.u16 %0, [%1];\n" : "=h"(b) : "l"(p));
    return (float)b * (1.0f / 65535.0f);
}

// Outer contraction of one run: R[k], k < K, for the state whose sliding
// entries start at box entry `ebase` (BOX) or from global memory.
template <class VT, int WM, int NS, int K, bool KAHAN, bool BOX>
__device__ __forceinline__ void run_contract(const Geom &g, const FastArgs<VT> &a, const RunRecs<WM, NS> &rr,
                                             int32_t r0, uint32_t sbase, const int32_t (&offij)[WM * WM],
                                             int32_t bs0b, int32_t bs1b, int32_t planeb, float (&R)[K]) {
    constexpr int L = NS - 1;
    constexpr int NQ = (WM + 1 + 3) / 4;
    constexpr int NP = runs_planes(K);
    int32_t o[2] = {0, 0};
    float t[2][WM];
#pragma unroll
    for (int d = 0; d < L; ++d) {
        uint32_t wds[NQ * 4];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            wds[q * 4 + 0] = rr.q[d][q].x;
            wds[q * 4 + 1] = rr.q[d][q].y;
            wds[q * 4 + 2] = rr.q[d][q].z;
            wds[q * 4 + 3] = rr.q[d][q].w;
        }
        o[d] = (int32_t)wds[0];
#pragma unroll
        for (int k = 0; k < WM; ++k) t[d][k] = __uint_as_float(wds[1 + k]);
    }
    float acc[K], comp[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        acc[k] = 0.0f;
        comp[k] = 0.0f;
    }
    if (BOX) {
        const uint32_t pb = sbase + (uint32_t)(o[0] * bs0b + (NS == 3 ? o[1] * bs1b : 0));
#pragma unroll
        for (int i = 0; i < WM; ++i) {
            float inner[K];
#pragma unroll
            for (int k = 0; k < K; ++k) inner[k] = 0.0f;
#pragma unroll
            for (int j = 0; j < (NS == 3 ? WM : 1); ++j) {
                const uint32_t pe = pb + (uint32_t)offij[i * WM + j];
                float v[NP * 4];
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    const float4 e = lds_f4(pe + (uint32_t)(q * planeb));
                    v[4 * q + 0] = e.x;
                    v[4 * q + 1] = e.y;
                    v[4 * q + 2] = e.z;
                    v[4 * q + 3] = e.w;
                }
#pragma unroll
                for (int k = 0; k < K; ++k) inner[k] = NS == 3 ? fmaf(t[1][j], v[k], inner[k]) : v[k];
            }
#pragma unroll
            for (int k = 0; k < K; ++k) accum_row(acc[k], comp[k], __fmul_rn(t[0][i], inner[k]), KAHAN ? 1 : 0);
        }
    } else {
        int32_t of0[WM], of1[WM], ofL[K];
        dim_offsets_reg<WM>(g, 0, o[0], WM, of0);
        if (NS == 3) dim_offsets_reg<WM>(g, 1, o[1], WM, of1);
        dim_offsets_reg<K>(g, L, r0, K, ofL);
#pragma unroll
        for (int i = 0; i < WM; ++i) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                float inner;
                if (NS == 3) {
                    inner = 0.0f;
#pragma unroll
                    for (int j = 0; j < WM; ++j)
                        inner = fmaf(t[1][j], vload<float, VT>(a.Vn + (of0[i] + of1[j] + ofL[k])), inner);
                } else {
                    inner = vload<float, VT>(a.Vn + (of0[i] + ofL[k]));
                }
                accum_row(acc[k], comp[k], __fmul_rn(t[0][i], inner), KAHAN ? 1 : 0);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) R[k] = acc[k];
}

// One input's window sum from its shifted inner weights at shared address pw
// and the run's outer contraction R; keeps the max and the lowest maximiser.
template <int K, int NP>
__device__ __forceinline__ void input_sum(uint32_t pw, int32_t tt_planeb, const float (&R)[K], int32_t u, float &best,
                                          int32_t &arg) {
    float w[NP * 4];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const float4 e = lds_f4(pw + (uint32_t)(p * tt_planeb));
        w[4 * p + 0] = e.x;
        w[4 * p + 1] = e.y;
        w[4 * p + 2] = e.z;
        w[4 * p + 3] = e.w;
    }
    float sum = 0.0f;
#pragma unroll
    for (int k = 0; k < K; ++k) sum = fmaf(w[k], R[k], sum);
    const bool gt = sum > best;
    best = gt ? sum : best;
    arg = gt ? u : arg;
}

// Window sums of one state for its runs rr = c, c + UL, ... (inputs
// [rs[rr], rs[rr + 1])); max and lowest maximiser kept in (best, arg).  The
// next run's outer records are loaded while the current run is summed.
template <class VT, int WM, int NS, int KX, bool KAHAN, bool BOX>
__device__ __forceinline__ void runs_sums(const Geom &g, const FastArgs<VT> &a, const int4 *s_up, const int32_t *s_rs,
                                          uint32_t s_in, int32_t stride, int32_t nruns, uint32_t ttL,
                                          int32_t tt_planeb,
                                          const int32_t (&es)[3], int32_t r0, int c, int UL, uint32_t sbase,
                                          int32_t bs0b, int32_t bs1b, int32_t planeb, float &best, int32_t &arg) {
    constexpr int K = WM + KX;
    constexpr int NP = runs_planes(K);
    if (c >= nruns) return;
    // byte offsets of the outer cells (i, j) from cell (0, 0), the same for every run
    int32_t offij[WM * WM];
#pragma unroll
    for (int i = 0; i < WM; ++i)
#pragma unroll
        for (int j = 0; j < WM; ++j) offij[i * WM + j] = i * bs0b + (NS == 3 ? j * bs1b : 0);
    RunRecs<WM, NS> nxt;
    run_records<WM, NS>(g, a.tab, s_up[s_rs[c]], es, nxt);
    for (int32_t rr = c; rr < nruns; rr += UL) {
        const int32_t u0 = s_rs[rr], u1 = s_rs[rr + 1];
        const RunRecs<WM, NS> cur = nxt;
        if (rr + UL < nruns) run_records<WM, NS>(g, a.tab, s_up[s_rs[rr + UL]], es, nxt);
        float R[K];
        run_contract<VT, WM, NS, K, KAHAN, BOX>(g, a, cur, r0, sbase, offij, bs0b, bs1b, planeb, R);
        // each input's shifted inner weights: s_in[u] holds its record's byte
        // offset; within a run they advance by `stride` bytes when
        // stride != INT_MIN (a uniform choice, made outside the loop)
        if (stride != INT_MIN) {
            uint32_t pw = ttL + (uint32_t)lds_i32(s_in + 4u * (uint32_t)u0);
#pragma unroll 3
            for (int32_t u = u0; u < u1; ++u) {
                input_sum<K, NP>(pw, tt_planeb, R, u, best, arg);
                pw += (uint32_t)stride;
            }
        } else {
#pragma unroll 3
            for (int32_t u = u0; u < u1; ++u)
                input_sum<K, NP>(ttL + (uint32_t)lds_i32(s_in + 4u * (uint32_t)u), tt_planeb, R, u, best, arg);
        }
    }
}

// Stages the tile's sliding box.  Warp w takes box rows w, w + NW, ...:
// lane l first decodes the outer cells of the warp's row jb + l (offset of
// the row in V, -1 when off the grid, and its first box entry); then the warp
// walks its rows, taking each row's decode by a shuffle.  Lane p fills the
// entries of inner coordinate p (+ 32 per chunk): slot r0(p) + k comes from
// inner cell dmin + p + k, wrapped when periodic, zero beyond a bounded edge
// (those slots carry zero mass).  Source offsets and copy sizes are set once
// per lane; a row off the grid is written as zeros.
// Inner cell c of a box row: wrapped into [0, Rn) when the dim is periodic,
// else flagged off (ok = false: its slots carry zero mass and hold 0).
__device__ __forceinline__ void inner_cell(int32_t &c, bool &ok, int32_t Rn, bool periodic) {
    if ((uint32_t)c < (uint32_t)Rn) return;
    if (periodic) {
        c %= Rn;
        c = c < 0 ? c + Rn : c;
    } else {
        ok = false;
        c = 0;
    }
}

template <class VT, int NS, int NP, bool L2ONLY>
__device__ __forceinline__ void stage_box(const Geom &g, const VT *Vn, float4 *sbox4, int32_t nrows,
                                          const int32_t (&bn)[2], const int32_t (&blo)[2], int32_t bs0, int32_t bs1,
                                          int32_t plane, int32_t dminL, int32_t Rn) {
    constexpr int L = NS - 1;
    constexpr int NC = 4 * NP;  // slots per entry
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NW = blockDim.x >> 5;
    const bool per_in = (g.periodic >> L) & 1u;
    const uint32_t sb = (uint32_t)__cvta_generic_to_shared(sbox4);
    const int32_t my_rows = warp < nrows ? (nrows - 1 - warp) / NW + 1 : 0;
    for (int32_t jb = 0; jb < my_rows; jb += 32) {
        const int32_t rr = warp + (jb + lane) * NW;
        int32_t mlin = -1, msidx = 0;
        if (jb + lane < my_rows) {
            bool on;
            if (NS == 3) {
                const int32_t k1 = rr % bn[1], k0 = rr / bn[1];
                bool o0, o1;
                const int32_t c0 = cell_of(g, 0, blo[0] + k0, o0);
                const int32_t c1 = cell_of(g, 1, blo[1] + k1, o1);
                on = o0 && o1;
                mlin = c0 * g.stride[0] + c1 * g.stride[1];
                msidx = k0 * bs0 + k1 * bs1;
            } else {
                bool o0;
                const int32_t c0 = cell_of(g, 0, blo[0] + rr, o0);
                on = o0;
                mlin = c0 * g.stride[0];
                msidx = rr * bs0;
            }
            if (!on) mlin = -1;
        }
        const int32_t cnt = min(32, my_rows - jb);
        for (int32_t p0 = 0; p0 < Rn; p0 += 32) {
            const int32_t p = p0 + lane;
            // source inner cell of each slot of this lane's entry
            int32_t srcb[NC];
            uint32_t nb[NC];
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                int32_t cc = dminL + p + k;
                bool okc = true;
                if ((uint32_t)cc >= (uint32_t)Rn) {
                    if (per_in) {
                        cc = cc < 0 ? cc + Rn : cc - Rn;
                        if ((uint32_t)cc >= (uint32_t)Rn) {  // more than one lap away
                            cc %= Rn;
                            cc = cc < 0 ? cc + Rn : cc;
                        }
                    } else {
                        okc = false;
                    }
                }
                srcb[k] = okc ? cc : 0;
                nb[k] = okc ? 4u : 0u;
            }
            if constexpr (L2ONLY) {
                // Loads that bypass L1 (V was written by other SMs since this
                // SM last read it).  Slot k of entry p is inner cell
                // dminL + p + k, so a row needs only the cells dminL + p0 + 0
                // ... + 31 + NC - 1: lane l loads cells l and 32 + l (l < NC - 1)
                // of that range, and slot k of lane l's entry is taken by a
                // shuffle from lane (l + k) mod 32, which offers its first
                // cell when l + k < 32, i.e. when its own lane index is >= k,
                // else its second.  RB rows at a time: their loads are all
                // issued before the first store, sharing one L2 round trip.
                int32_t ca = dminL + p0 + lane, cb = ca + 32;
                bool oka = true, okb = lane < NC - 1;
                inner_cell(ca, oka, Rn, per_in);
                inner_cell(cb, okb, Rn, per_in);
                constexpr int RB = 4;
                for (int32_t j0 = 0; j0 < cnt; j0 += RB) {
                    int32_t lin[RB], sidx[RB];
                    float va[RB], vb[RB];
#pragma unroll
                    for (int r = 0; r < RB; ++r) {
                        const int32_t jj = min(j0 + r, cnt - 1);
                        lin[r] = __shfl_sync(0xffffffffu, mlin, jj);
                        sidx[r] = __shfl_sync(0xffffffffu, msidx, jj);
                        if (j0 + r >= cnt) lin[r] = -1;
                    }
#pragma unroll
                    for (int r = 0; r < RB; ++r) {
                        va[r] = (lin[r] >= 0 && oka) ? ld_cg(Vn + lin[r] + ca) : 0.0f;
                        vb[r] = (lin[r] >= 0 && okb) ? ld_cg(Vn + lin[r] + cb) : 0.0f;
                    }
#pragma unroll
                    for (int r = 0; r < RB; ++r) {
                        if (j0 + r < cnt) {
                            float v[NC];
#pragma unroll
                            for (int k = 0; k < NC; ++k)
                                v[k] = __shfl_sync(0xffffffffu, lane >= k ? va[r] : vb[r], (lane + k) & 31);
                            if (p < Rn) {
                                const uint32_t dst = sb + 16u * (uint32_t)(sidx[r] + p);
#pragma unroll
                                for (int q = 0; q < NP; ++q)
                                    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(
                                                     dst + 16u * (uint32_t)(q * plane)),
                                                 "f"(v[4 * q]), "f"(v[4 * q + 1]), "f"(v[4 * q + 2]), "f"(v[4 * q + 3])
                                                 : "memory");
                            }
                        }
                    }
                }
                continue;
            }
            for (int32_t j = 0; j < cnt; ++j) {
                const int32_t lin = __shfl_sync(0xffffffffu, mlin, j);
                const int32_t sidx = __shfl_sync(0xffffffffu, msidx, j);
                if (p < Rn) {
                    const uint32_t dst = sb + 16u * (uint32_t)(sidx + p);
                    if (lin < 0) {
#pragma unroll
                        for (int q = 0; q < NP; ++q)
                            asm volatile("st.shared.v4.f32 [%0], {%1, %1, %1, %1};\n" ::"r"(dst + 16u * (uint32_t)(q * plane)),
                                         "f"(0.0f)
                                         : "memory");
                    } else if constexpr (std::is_same<VT, float>::value) {
                        const float *row = Vn + lin;
#pragma unroll
                        for (int k = 0; k < NC; ++k) {
                            const size_t gsrc = __cvta_generic_to_global(row + srcb[k]);
                            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(
                                             dst + 16u * (uint32_t)((k >> 2) * plane) + 4u * (uint32_t)(k & 3)),
                                         "l"(gsrc), "r"(nb[k])
                                         : "memory");
                        }
                    } else {
                        float *d = reinterpret_cast<float *>(sbox4 + (sidx + p));
#pragma unroll
                        for (int k = 0; k < NC; ++k)
                            d[(k >> 2) * 4 * plane + (k & 3)] = nb[k] ? vload<float, VT>(Vn + (lin + srcb[k])) : 0.0f;
                    }
                }
            }
        }
    }
}

template <class VT, int WM, int NS, bool KAHAN>
__global__ void __launch_bounds__(RUNS_MAX_THREADS) k_backup_runs(const __grid_constant__ Geom g,
                                                                 const FastArgs<VT> a) {
    static_assert(NS == 2 || NS == 3, "row tiles of 2-D or 3-D problems");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int L = NS - 1;
    const int BT = blockDim.x;
    float4 *sbox4 = reinterpret_cast<float4 *>(smem_raw);
    unsigned char *work = smem_raw + (size_t)a.box_floats * 4;
    int4 *s_up = reinterpret_cast<int4 *>(work + staged_work_bytes(NS, WM, BT));
    int32_t *s_rs = reinterpret_cast<int32_t *>(s_up + g.nu);
    int32_t *s_inb = s_rs + ((g.nu + 1 + 3) / 4) * 4;  // per input: byte offset of its inner record
    float4 *s_tt = reinterpret_cast<float4 *>(s_inb + ((g.nu + 3) / 4) * 4);
    float *cBest = reinterpret_cast<float *>(work);
    int32_t *cArg = reinterpret_cast<int32_t *>(cBest + BT);
    __shared__ int32_t s_nruns, s_stride;

    const int tid = threadIdx.x;
    const int TX = a.tileX, UL = a.ulanes, RW = a.rowtile;
    const int c = (int)__umulhi((uint32_t)tid, a.tx_magic);  // tid / TX (tid, TX <= 512)
    const int xl = tid - c * TX;
    // lane column xl = (row r of the tile, chunk of 32 cells of that row, lane)
    const int32_t Rn = g.N[L];
    const int r = (xl >> 5) >> a.chu_shift;
    const int32_t k_in = (((xl >> 5) & ((1 << a.chu_shift) - 1)) << 5) + (xl & 31);
    int32_t xi[3] = {0, 0, 0};
    int32_t rowlo, rowhi;  // first and last row index (dim L - 1) of the tile
    int32_t x0lo = 0, x0hi = 0;  // first and last value of dim 0 (3-D)
    bool ok;
    if (NS == 3) {
        // grid (row tiles of dim 1, tiles of `outer` values of dim 0); tile
        // row r = (value r / RW of dim 0, row r % RW of dim 1)
        const int rx = r / RW, ry = r - rx * RW;
        x0lo = (int32_t)blockIdx.y * a.outer;
        x0hi = min(x0lo + a.outer, g.N[0]) - 1;
        xi[0] = x0lo + rx;
        rowlo = (int32_t)blockIdx.x * RW;
        rowhi = min(rowlo + RW, g.N[1]) - 1;
        xi[1] = rowlo + ry;
        ok = xi[0] < g.N[0] && xi[1] < g.N[1];
    } else {
        rowlo = (int32_t)blockIdx.x * RW;
        rowhi = min(rowlo + RW, g.N[0]) - 1;
        xi[0] = rowlo + r;
        ok = xi[0] < g.N[0];
    }
    xi[L] = k_in;
    ok = ok && k_in < Rn;
    const int32_t x = ok ? (NS == 3 ? (xi[0] * g.N[1] + xi[1]) * Rn + k_in : xi[0] * Rn + k_in) : INT_MAX;
    const uint8_t f = ok ? a.mask[x] : (uint8_t)0;
    const bool masked = ok && state_masked(a.spec_kind, f);
    const bool work_items = ok && !masked;

    // per dim, the range of (window origin - own coordinate) over the tables:
    // launch parameters when the host holds them, else from the bounds block
    int32_t dmin[3] = {0, 0, 0}, dmax[3] = {0, 0, 0};
    bool analytic = true;
    if (a.bnd_known) {
#pragma unroll
        for (int d = 0; d < NS; ++d) {
            dmin[d] = a.bnd_lo[d];
            dmax[d] = a.bnd_hi[d];
        }
    } else {
        const int32_t *rb = reinterpret_cast<const int32_t *>(a.tab + g.boff);
#pragma unroll
        for (int d = 0; d < NS; ++d) {
            dmin[d] = __ldg(rb + d);
            dmax[d] = __ldg(rb + MAXD + d);
        }
        analytic = (__ldg(rb + 2 * MAXD) & ((1 << NS) - 1)) == ((1 << NS) - 1);
    }
    const int32_t KX = dmax[L] - dmin[L];
    if (!analytic || g.shoff == 0 || KX < 0 || KX > 3 || WM + KX > Rn || runs_planes(WM + KX) > a.runs_planes) {
        // inner windows spread too far for one shared contraction: the
        // register-resident body (uniform over the block)
        backup_tile<VT, WM, TM_SEPARABLE, VAR_EXACT>(g, a, x, work);
        return;
    }
    const int NPK = runs_planes(WM + KX);
    // the tile's outer box [blo, blo + bn) per outer dim; entries per row:
    // the inner coordinates 0 .. Rn - 1 (padded to 8)
    int32_t blo[2] = {0, 0}, bn[2] = {1, 1};
    if (NS == 3) {
        blo[0] = x0lo + dmin[0];
        bn[0] = x0hi - x0lo + dmax[0] - dmin[0] + WM;
        blo[1] = rowlo + dmin[1];
        bn[1] = rowhi - rowlo + dmax[1] - dmin[1] + WM;
    } else {
        blo[0] = rowlo + dmin[0];
        bn[0] = rowhi - rowlo + dmax[0] - dmin[0] + WM;
    }
    const int32_t nrows = NS == 3 ? bn[0] * bn[1] : bn[0];
    const int32_t E = (Rn + 7) & ~7;
    const int32_t plane = nrows * E;  // float4 entries of one plane
    const bool fits = (int64_t)plane * NPK * 4 <= a.box_floats;
    const int32_t bs1 = E;
    const int32_t bs0 = NS == 3 ? bn[1] * E : E;
    const int lane = tid & 31, warp = tid >> 5, NW = BT >> 5;
    if (fits) {
        if (NPK == 1)
            stage_box<VT, NS, 1, false>(g, a.Vn, sbox4, nrows, bn, blo, bs0, bs1, plane, dmin[L], Rn);
        else
            stage_box<VT, NS, 2, false>(g, a.Vn, sbox4, nrows, bn, blo, bs0, bs1, plane, dmin[L], Rn);
    }
    // the inputs' table-index parts and the innermost dim's table as shifted
    // weights (built with the tables at word shoff: plane p of record e at
    // float4 p * records + e)
    {
        const int4 *up = reinterpret_cast<const int4 *>(a.tab + g.uoff);
        for (int32_t u = tid; u < g.nu; u += BT) {
            const int4 v = __ldg(up + u);
            s_up[u] = v;
            s_inb[u] = (NS == 3 ? v.z : v.y) * 16;
        }
        const float4 *sh = reinterpret_cast<const float4 *>(a.tab + g.shoff);
        const int32_t nrec = a.stage_recs;
        for (int32_t i = tid; i < NPK * nrec; i += BT) {
            const unsigned sdst = (unsigned)__cvta_generic_to_shared(s_tt + i);
            const size_t gsrc = __cvta_generic_to_global(sh + i);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sdst), "l"(gsrc) : "memory");
        }
    }
    // run starts: inputs whose outer table-index parts differ from the
    // previous input's -- from the launch parameters when the host gave them,
    // else found by warp 0 after the barrier below
    if (a.nrs > 0) {
        for (int32_t i = tid; i <= a.nrs; i += BT) s_rs[i] = a.rs[i];
        if (tid == 0) {
            s_nruns = a.nrs;
            s_stride = a.in_stride_b;
        }
    }
    cp_async_wait_all();
    __syncthreads();
    if (a.nrs == 0 && tid < 32) {
        int32_t cnt = 0;
        // byte step between the inner records of consecutive inputs of a run
        // (inputs 0 and 1 when they share a run; any value when no run has two inputs)
        const int32_t stride = g.nu > 1 ? s_inb[1] - s_inb[0] : 0;
        bool affine = true;
        for (int32_t base = 0; base < g.nu; base += 32) {
            const int32_t u = base + tid;
            bool st = false;
            if (u < g.nu) {
                if (u == 0) {
                    st = true;
                } else {
                    const int4 p = s_up[u - 1], q = s_up[u];
                    st = p.x != q.x || (NS == 3 && p.y != q.y);
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, st);
            if (st) s_rs[cnt + __popc(bal & ((1u << tid) - 1u))] = u;
            cnt += __popc(bal);
            // inner records a constant stride apart within every run?
            const bool same = st || u >= g.nu || s_inb[u] - s_inb[u - 1] == stride;
            affine = affine && __all_sync(0xffffffffu, same);
        }
        if (tid == 0) {
            s_rs[cnt] = g.nu;
            s_nruns = cnt;
            s_stride = affine ? stride : INT_MIN;
        }
    }
    if (a.nrs == 0) __syncthreads();

    float best = -1.0f;
    int32_t arg = 0x7fffffff;
    if (work_items) {
        int32_t es[3] = {0, 0, 0};
#pragma unroll
        for (int d = 0; d < NS; ++d) {
            int32_t e = 0;
#pragma unroll
            for (int j = 0; j < NS; ++j) e += xi[j] * g.tsx[d][j];
            es[d] = e;
        }
        const int32_t r0 = xi[L] + dmin[L];
        // shared byte address of the sliding entry of outer cell (o0, o1) for
        // this state: sbase + 16 * (o0 * bs0 + o1 * bs1), with
        // sbase = box + 16 * (own inner coordinate - blo0 * bs0 - blo1 * bs1)
        const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sbox4) +
                               16u * (uint32_t)(xi[L] - (blo[0] * bs0 + (NS == 3 ? blo[1] * bs1 : 0)));
        const uint32_t ttL = (uint32_t)__cvta_generic_to_shared(s_tt) + 16u * (uint32_t)es[L];
        const uint32_t s_in = (uint32_t)__cvta_generic_to_shared(s_inb);
        const int32_t nruns = s_nruns;
        const int32_t stride = s_stride;
#define AMY_RUNS_CASE(KXV)                                                                                         \
    case KXV:                                                                                                      \
        if (fits)                                                                                                  \
            runs_sums<VT, WM, NS, KXV, KAHAN, true>(g, a, s_up, s_rs, s_in, stride, nruns, ttL, 16 * a.stage_recs, es, r0, \
                                                    c, UL, sbase, 16 * bs0, 16 * bs1, 16 * plane, best, arg);      \
        else                                                                                                       \
            runs_sums<VT, WM, NS, KXV, KAHAN, false>(g, a, s_up, s_rs, s_in, stride, nruns, ttL, 16 * a.stage_recs, es,    \
                                                     r0, c, UL, sbase, 16 * bs0, 16 * bs1, 16 * plane, best, arg); \
        break;
        switch (KX) {
            AMY_RUNS_CASE(0)
            AMY_RUNS_CASE(1)
            AMY_RUNS_CASE(2)
            AMY_RUNS_CASE(3)
            default: break;
        }
#undef AMY_RUNS_CASE
    }
    if (UL > 1) {
        cBest[tid] = best;
        cArg[tid] = arg;
        __syncwarp();
        __syncthreads();
    }
    if (c == 0 && ok) {
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

// ---------------------------------------------------------------------------
// The whole horizon in one launch (Algorithm 4's N backups): every block owns
// one row tile for all steps, stages its tables, run starts and per-state
// data once, and per step stages only its window box from V_{k+1}.  Between
// backups a block waits only for the tiles its box reads and the tiles whose
// boxes read it (a neighbour wait on per-tile backup counters), or, when the
// host asks for it, for every block (grid barrier).  All blocks must be
// resident at once (a cooperative launch checks this).  Values and policies
// are those of N launches of k_backup_runs with the same shape.
// ---------------------------------------------------------------------------
struct RunsHorizon {
    const void *V0;      // V_N (read by the first backup)
    void *V1;            // the other resident V vector
    float *Vfinal;       // FP32 copy of V_0, or null
    uint16_t *pi;        // policies: [horizon][n_x] when all_steps, else pi_0 only; or null
    int32_t all_steps;
    int32_t horizon;
    unsigned *bar;       // grid barrier: monotonic arrival count (zero at launch)
    unsigned *flags;     // per-tile backup counters (zero at launch), or null: grid barrier
    int32_t *err;        // set to 1 when a wait gives up, 2 on a bad launch shape
    int32_t spin_limit;  // polls before a wait gives up (0: every wait gives up at once)
    // neighbour radius in tiles along blockIdx.y and blockIdx.x (a radius
    // with 2r + 1 >= the grid's extent means the whole extent), and bit 0 / 1:
    // that extent wraps (a periodic dim whose points fill whole tiles)
    int32_t nr_y, nr_x;
    uint32_t wrap;
};

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;\n" : : "l"(p), "r"(v) : "memory");
}

// Tile index along one grid extent for neighbour i of 2r + 1 (or of the
// whole extent), or -1 when that neighbour lies off a non-wrapping edge.
__device__ __forceinline__ int nbr_tile(int self, int i, int r, int G, bool wrap) {
    if (2 * r + 1 >= G) return i;
    int t = self - r + i;
    if (wrap) {
        t = t < 0 ? t + G : (t >= G ? t - G : t);
    } else if (t < 0 || t >= G) {
        return -1;
    }
    return t;
}

// Neighbour wait after backup number `done` (1-based) of this launch: the
// block publishes its counter (after all of its V and policy writes), then
// the lanes of warp 0 poll the counters of the neighbour tiles until each
// reaches `done`.  The neighbours are the tiles within the host's radius: they
// include every tile whose V cells this block's next box reads (read after
// write) and every tile whose box reads this block's cells (their reads of
// the buffer this block overwrites next must be over: write after read).
// Each poll loop stops after spin_limit polls, or sooner once another block
// reported an error; a block that gives up sets the error flag.  Returns
// false when the kernel has to stop.
__device__ __forceinline__ bool neighbour_wait(const RunsHorizon &hz, unsigned done) {
    __shared__ int s_ok;
    __syncwarp();
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const int Gx = (int)gridDim.x, Gy = (int)gridDim.y;
        const int bx = (int)blockIdx.x, by = (int)blockIdx.y;
        // the block's V and policy writes (ordered before this lane by the
        // block barrier) before its counter: a release store
        if (lane == 0) st_release_gpu(hz.flags + by * Gx + bx, done);
        __syncwarp();
        const int cy = min(2 * hz.nr_y + 1, Gy), cx = min(2 * hz.nr_x + 1, Gx);
        int ok = hz.spin_limit > 0;
        for (int i = lane; ok && i < cy * cx; i += 32) {
            const int iy = i / cx, ix = i - iy * cx;
            const int ty = nbr_tile(by, iy, hz.nr_y, Gy, hz.wrap & 1u);
            const int tx = nbr_tile(bx, ix, hz.nr_x, Gx, hz.wrap & 2u);
            if (ty < 0 || tx < 0 || (ty == by && tx == bx)) continue;
            const unsigned *fl = hz.flags + ty * Gx + tx;
            int32_t it = 0;
            while (ld_acquire_gpu(fl) < done) {
                if (++it > hz.spin_limit ||
                    ((it & 31) == 0 && ld_acquire_gpu(reinterpret_cast<const unsigned *>(hz.err)) != 0)) {
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        ok = __all_sync(0xffffffffu, ok);
        if (lane == 0) {
            if (!ok) atomicExch(hz.err, 1);
            s_ok = ok;
        }
    }
    // warp 0 polled alone: reconverge it before the block barrier
    __syncwarp();
    __syncthreads();
    return s_ok != 0;
}

// Grid-wide barrier number `done` (1-based) of this launch on a monotonic
// arrival count (zero at launch): after the block's V and policy writes,
// thread 0 adds one with release semantics (a fence, then a reduction that
// returns nothing) and polls the count with acquire loads until every block
// has arrived `done` times.  No block resets anything, so no arrival waits on
// another block's second round trip.  Each wait stops after spin_limit polls
// (0: at once), or sooner once another block reported an error; a block that
// gives up sets the error flag.  Returns false when the kernel has to stop.
__device__ __forceinline__ bool grid_barrier(unsigned *count, int32_t *err, unsigned nblocks, unsigned done,
                                             int32_t spin_limit) {
    __shared__ int s_ok;
    __syncwarp();
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("fence.acq_rel.gpu;\n"
                     "red.relaxed.gpu.global.add.u32 [%0], 1;\n" ::"l"(count)
                     : "memory");
        // modulo 2^32: the count stays within nblocks of the target, so the
        // signed difference decides even after the product wraps (long horizons)
        const unsigned target = nblocks * done;
        int ok = spin_limit > 0;
        int32_t it = 0;
        while (ok && (int32_t)(ld_acquire_gpu(count) - target) < 0) {
            if (++it > spin_limit ||
                ((it & 31) == 0 && ld_acquire_gpu(reinterpret_cast<const unsigned *>(err)) != 0)) {
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        if (!ok) atomicExch(err, 1);
        s_ok = ok;
    }
    // lane 0 spun alone: reconverge warp 0 before the block barrier (an
    // aligned barrier must be reached by whole warps)
    __syncwarp();
    __syncthreads();
    return s_ok != 0;
}

template <class VT, int WM, int NS, bool KAHAN>
__global__ void __launch_bounds__(RUNS_MAX_THREADS, 2) k_synth_runs(const __grid_constant__ Geom g,
                                                                const __grid_constant__ FastArgs<VT> a,
                                                                const RunsHorizon hz) {
    static_assert(NS == 2 || NS == 3, "row tiles of 2-D or 3-D problems");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int L = NS - 1;
    const int BT = blockDim.x;
    float4 *sbox4 = reinterpret_cast<float4 *>(smem_raw);
    unsigned char *work = smem_raw + (size_t)a.box_floats * 4;
    int4 *s_up = reinterpret_cast<int4 *>(work + staged_work_bytes(NS, WM, BT));
    int32_t *s_rs = reinterpret_cast<int32_t *>(s_up + g.nu);
    int32_t *s_inb = s_rs + ((g.nu + 1 + 3) / 4) * 4;
    float4 *s_tt = reinterpret_cast<float4 *>(s_inb + ((g.nu + 3) / 4) * 4);
    float *cBest = reinterpret_cast<float *>(work);
    int32_t *cArg = reinterpret_cast<int32_t *>(cBest + BT);

    const int tid = threadIdx.x;
    const int TX = a.tileX, UL = a.ulanes, RW = a.rowtile;
    const int c = (int)__umulhi((uint32_t)tid, a.tx_magic);
    const int xl = tid - c * TX;
    const int32_t Rn = g.N[L];
    const int r = (xl >> 5) >> a.chu_shift;
    const int32_t k_in = (((xl >> 5) & ((1 << a.chu_shift) - 1)) << 5) + (xl & 31);
    int32_t xi[3] = {0, 0, 0};
    int32_t rowlo, rowhi;
    int32_t x0lo = 0, x0hi = 0;
    bool ok;
    if (NS == 3) {
        const int rx = r / RW, ry = r - rx * RW;
        x0lo = (int32_t)blockIdx.y * a.outer;
        x0hi = min(x0lo + a.outer, g.N[0]) - 1;
        xi[0] = x0lo + rx;
        rowlo = (int32_t)blockIdx.x * RW;
        rowhi = min(rowlo + RW, g.N[1]) - 1;
        xi[1] = rowlo + ry;
        ok = xi[0] < g.N[0] && xi[1] < g.N[1];
    } else {
        rowlo = (int32_t)blockIdx.x * RW;
        rowhi = min(rowlo + RW, g.N[0]) - 1;
        xi[0] = rowlo + r;
        ok = xi[0] < g.N[0];
    }
    xi[L] = k_in;
    ok = ok && k_in < Rn;
    const int32_t x = ok ? (NS == 3 ? (xi[0] * g.N[1] + xi[1]) * Rn + k_in : xi[0] * Rn + k_in) : INT_MAX;
    const uint8_t f = ok ? a.mask[x] : (uint8_t)0;
    const bool masked = ok && state_masked(a.spec_kind, f);
    const bool work_items = ok && !masked;

    int32_t dmin[3] = {0, 0, 0}, dmax[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < NS; ++d) {
        dmin[d] = a.bnd_lo[d];
        dmax[d] = a.bnd_hi[d];
    }
    const int32_t KX = dmax[L] - dmin[L];
    const int NPK = runs_planes(WM + KX);
    int32_t blo[2] = {0, 0}, bn[2] = {1, 1};
    if (NS == 3) {
        blo[0] = x0lo + dmin[0];
        bn[0] = x0hi - x0lo + dmax[0] - dmin[0] + WM;
        blo[1] = rowlo + dmin[1];
        bn[1] = rowhi - rowlo + dmax[1] - dmin[1] + WM;
    } else {
        blo[0] = rowlo + dmin[0];
        bn[0] = rowhi - rowlo + dmax[0] - dmin[0] + WM;
    }
    const int32_t nrows = NS == 3 ? bn[0] * bn[1] : bn[0];
    const int32_t E = (Rn + 7) & ~7;
    const int32_t plane = nrows * E;
    const bool fits = (int64_t)plane * NPK * 4 <= a.box_floats;
    // the host launches this kernel only with the bounds, run starts and a
    // box that fits; anything else is reported (uniformly, no block waits)
    if (!a.bnd_known || a.nrs <= 0 || g.shoff == 0 || KX < 0 || KX > 3 || WM + KX > Rn ||
        NPK > a.runs_planes || !fits) {
        if (blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) atomicExch(hz.err, 2);
        return;
    }
    const int32_t bs1 = E;
    const int32_t bs0 = NS == 3 ? bn[1] * E : E;
    // constant for the whole horizon: input parts, inner weights, run starts
    {
        const int4 *up = reinterpret_cast<const int4 *>(a.tab + g.uoff);
        for (int32_t u = tid; u < g.nu; u += BT) {
            const int4 v = __ldg(up + u);
            s_up[u] = v;
            s_inb[u] = (NS == 3 ? v.z : v.y) * 16;
        }
        const float4 *sh = reinterpret_cast<const float4 *>(a.tab + g.shoff);
        for (int32_t i = tid; i < NPK * a.stage_recs; i += BT) s_tt[i] = __ldg(sh + i);
        for (int32_t i = tid; i <= a.nrs; i += BT) s_rs[i] = a.rs[i];
    }
    __syncthreads();
    int32_t es[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < NS; ++d) {
        int32_t e = 0;
#pragma unroll
        for (int j = 0; j < NS; ++j) e += xi[j] * g.tsx[d][j];
        es[d] = e;
    }
    const int32_t r0 = xi[L] + dmin[L];
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(sbox4) +
                           16u * (uint32_t)(xi[L] - (blo[0] * bs0 + (NS == 3 ? blo[1] * bs1 : 0)));
    const uint32_t ttL = (uint32_t)__cvta_generic_to_shared(s_tt) + 16u * (uint32_t)es[L];
    const uint32_t s_in = (uint32_t)__cvta_generic_to_shared(s_inb);
    const unsigned nblocks = gridDim.x * gridDim.y;
    const int64_t nx = g.nx;
    const VT *Vn = reinterpret_cast<const VT *>(hz.V0);
    VT *Vo = reinterpret_cast<VT *>(hz.V1);
    for (int32_t j = 0; j < hz.horizon; ++j) {
        const int32_t k = hz.horizon - 1 - j;
        if (NPK == 1)
            stage_box<VT, NS, 1, true>(g, Vn, sbox4, nrows, bn, blo, bs0, bs1, plane, dmin[L], Rn);
        else
            stage_box<VT, NS, 2, true>(g, Vn, sbox4, nrows, bn, blo, bs0, bs1, plane, dmin[L], Rn);
        __syncwarp();
        __syncthreads();
        float best = -1.0f;
        int32_t arg = 0x7fffffff;
        if (work_items) {
#define AMY_SYNTH_CASE(KXV)                                                                                        \
    case KXV:                                                                                                      \
        runs_sums<VT, WM, NS, KXV, KAHAN, true>(g, a, s_up, s_rs, s_in, a.in_stride_b, a.nrs, ttL,                 \
                                                16 * a.stage_recs, es, r0, c, UL, sbase, 16 * bs0, 16 * bs1,       \
                                                16 * plane, best, arg);                                            \
        break;
            switch (KX) {
                AMY_SYNTH_CASE(0)
                AMY_SYNTH_CASE(1)
                AMY_SYNTH_CASE(2)
                AMY_SYNTH_CASE(3)
                default: break;
            }
#undef AMY_SYNTH_CASE
        }
        if (UL > 1) {
            cBest[tid] = best;
            cArg[tid] = arg;
            __syncwarp();
            __syncthreads();
        }
        if (c == 0 && ok) {
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
            Vo[x] = vstore_cast<VT, float>(best);
            if (k == 0 && hz.Vfinal) hz.Vfinal[x] = best;
            if (hz.pi && (hz.all_steps || k == 0)) hz.pi[(hz.all_steps ? (int64_t)k * nx : 0) + x] = pol;
        }
        if (j + 1 < hz.horizon) {
            const bool go = hz.flags ? neighbour_wait(hz, (unsigned)(j + 1))
                                     : grid_barrier(hz.bar, hz.err, nblocks, (unsigned)(j + 1), hz.spin_limit);
            if (!go) return;
        }
        const VT *t = Vn;
        Vn = Vo;
        Vo = const_cast<VT *>(t);
    }
}

}  // namespace amy
