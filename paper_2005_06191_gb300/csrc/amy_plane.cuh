// amy_plane.cuh -- fused backup + max/argmax (Algorithm 4) for problems whose
// mean components each depend on a few state coordinates (banded coupling:
// rings of rooms or of road cells, Sec. 8.2 / 8.3), with the window sum
// reassociated so that the dimensions whose masses a whole plane of states
// shares are contracted once per plane instead of once per state.
//
// Notation.  Z = the two innermost dims: a "plane" of P = N[n-2] * N[n-1]
// states, contiguous in V.  F = the other dims; a group is the plane of
// states sharing their F coordinates.  S = the F dims whose mean component
// depends on F coordinates only (the per-dimension tables say which): within
// a group and an input their window origin and masses are the same for every
// state.  B = F minus S: their windows move across the plane (through the
// coupling), so the union of the group's windows in those dims is staged.
//
// For one group and input u the window sum s(x,u) = sum_j prod_d t_d[j_d]
// V[o + j] (Algorithm 4, a product of per-dimension masses for diagonal
// noise) is formed in two stages:
//   stage 1: R[y_B][p] = sum_{j_S} (prod_{d in S} t_d[j_d]) V[y_B, o_S + j_S, p]
//            for every plane position p and every y_B of the staged union;
//            each term reads a whole plane of V, coalesced across threads;
//   stage 2: s(x,u) = sum_{j_B} (prod_{d in B} t_d[j_d])
//                       sum_{j_Z} (prod_{d in Z} t_d[j_d]) R[o_B + j_B][o_Z + j_Z]
//            per state, from R in shared memory (Kahan-compensated over the
//            j_B rows when asked).
// Every term of the window sum appears exactly once (an exact
// reassociation); only the FP32 rounding order differs from the per-state
// kernels.  The max over inputs keeps the lowest maximising input.
//
// R is staged in chunks of `chunk` values of the first B dim (the j_B rows
// are summed in the same order whatever the chunk size, so the result does
// not depend on it).  A block holds G groups (G * P threads, one state each).
//
// Stage 1 reads V_{k+1} from a padded copy: every plane is stored in Ppad =
// P rounded up to 4 values (the pad holds zeros), so that each plane starts
// on a 16-byte boundary and is read with 16-byte loads, four plane positions
// per load.  For stage 1 the block's threads form teams of Q = Ppad / 4
// threads (one per group of four positions); the teams of a group share
// its staged rows.  Each kernel writes V_k twice: in the standard layout
// (what every other kernel and the caller read) and padded (what the next
// backup's stage 1 reads); k_plane_repack makes the padded copy of any other
// V (V_N, a caller's V_{k+1}).
#pragma once

#include <climits>

#include "amy_fast.cuh"

namespace amy {

constexpr int PLANE_MAXB = 3;   // B dims (windows staged as ranges)
constexpr int PLANE_MAXS = 6;   // S dims (contracted in stage 1)
constexpr int PLANE_MAX_THREADS = 448;  // two blocks per SM at up to 72 registers
// Stage-1 loads in flight per thread: PLANE_EB rows x PLANE_KU S combinations.
#ifndef AMY_PLANE_EB
#define AMY_PLANE_EB 2
#endif
#ifndef AMY_PLANE_KU
#define AMY_PLANE_KU 4
#endif
constexpr int PLANE_EB = AMY_PLANE_EB;  // R rows per stage-1 batch
constexpr int PLANE_KU = AMY_PLANE_KU;  // S combinations per step of a batch
// Stage-2 rows of the second staged dim whose window sums are formed together
#ifndef AMY_PLANE_S2ROWS
#define AMY_PLANE_S2ROWS 2
#endif
constexpr int PLANE_S2ROWS = AMY_PLANE_S2ROWS;
// Paired FP32 FMAs (two lanes per instruction, each lane rounded as one
// fmaf): the same values with half the FMA instructions.  Switched per site:
// kernel 7's stage 1 (windows of at most 3 slots), kernel 8's stage 1, the
// Z sums of stage 2 two rows at a time, stage 2's single rows (pairs of Z
// rows).
#ifndef AMY_FFMA2_P1
#define AMY_FFMA2_P1 1
#endif
#ifndef AMY_FFMA2_T1
#define AMY_FFMA2_T1 0
#endif
#ifndef AMY_FFMA2_S2
#define AMY_FFMA2_S2 1
#endif
#ifndef AMY_FFMA2_S2T
#define AMY_FFMA2_S2T 0
#endif

// acc += w * v, lane by lane
template <bool PAIRED>
__device__ __forceinline__ void fma4(float w, const float4 &v, float4 &acc) {
    if constexpr (PAIRED) {
        const float2 ww = make_float2(w, w);
        const float2 lo = __ffma2_rn(ww, make_float2(v.x, v.y), make_float2(acc.x, acc.y));
        const float2 hi = __ffma2_rn(ww, make_float2(v.z, v.w), make_float2(acc.z, acc.w));
        acc = make_float4(lo.x, lo.y, hi.x, hi.y);
    } else {
        acc.x = fmaf(w, v.x, acc.x);
        acc.y = fmaf(w, v.y, acc.y);
        acc.z = fmaf(w, v.z, acc.z);
        acc.w = fmaf(w, v.w, acc.w);
    }
}

template <class VT> struct PlaneArgs {
    const VT *Vn;          // V_{k+1} (unused: stage 1 reads the padded copy)
    VT *Vo;                // V_k
    const VT *Vpn;         // V_{k+1}, planes padded to Ppad values
    VT *Vpo;               // V_k, planes padded to Ppad values (pads left untouched)
    float *Vfinal;         // optional FP32 copy of V_k
    uint16_t *pi;          // optional policy of this step
    const uint8_t *mask;
    const uint32_t *tab;   // per-dimension tables (origin + masses per record)
    int32_t spec_kind;
    int32_t kahan;
    int32_t P;             // plane positions (states per group)
    int32_t N1;            // points of the innermost dim
    int32_t G;             // groups per block
    int32_t ngroups;       // groups of the grid: prod_{d < n-2} N[d]
    int32_t nS, nB;
    int32_t sdim[PLANE_MAXS];
    int32_t bdim[PLANE_MAXB];
    int32_t brange[PLANE_MAXB];  // largest union of one group's windows per B dim
    int32_t chunk;         // values of the first B dim per staged chunk
    int32_t rs0;           // R rows per value of the first B dim: prod_{b > 0} brange[b]
    int32_t rent;          // R rows per group and chunk: chunk * rs0 (at least 1)
    int32_t K;             // S-window combinations: prod_{d in S} W[d]
    int32_t Ppad;          // padded plane: P rounded up to a multiple of 4
    int32_t Q;             // Ppad / 4: threads of one stage-1 team
    int32_t teams;         // stage-1 teams per group
    int32_t bstrideF[PLANE_MAXB];  // plane-index strides of the B dims: stride[bdim] / P
    // optional work counters (null in timed runs): [0] V values read in
    // stage 1, [1] R values read in stage 2, [2] stage-2 rows summed (B
    // combinations with non-zero weight)
    unsigned long long *work;
};

// Dynamic shared memory of one block: per group the B origin bounds and the
// S dims' table indices, the S combinations' weights and offsets, and one
// chunk of R.
__host__ __device__ inline size_t plane_smem_head(int G, int K) {
    return ((size_t)G * ((2 * PLANE_MAXB + PLANE_MAXS + 1) * 4 + (size_t)K * 8) + 15) / 16 * 16;
}
__host__ __device__ inline size_t plane_smem_bytes(int G, int K, int rent, int Ppad) {
    return plane_smem_head(G, K) + (size_t)G * rent * Ppad * 4;
}

// Four consecutive values of V (16-byte aligned; 8 bytes for 16-bit storage).
template <class VT> __device__ __forceinline__ float4 vload4(const VT *p);
template <> __device__ __forceinline__ float4 vload4<float>(const float *p) {
    return __ldg(reinterpret_cast<const float4 *>(p));
}
template <> __device__ __forceinline__ float4 vload4<__nv_bfloat16>(const __nv_bfloat16 *p) {
    const uint2 r = __ldg(reinterpret_cast<const uint2 *>(p));
    return make_float4(bf16_unfold(__ushort_as_bfloat16((unsigned short)(r.x & 0xffffu))),
                       bf16_unfold(__ushort_as_bfloat16((unsigned short)(r.x >> 16))),
                       bf16_unfold(__ushort_as_bfloat16((unsigned short)(r.y & 0xffffu))),
                       bf16_unfold(__ushort_as_bfloat16((unsigned short)(r.y >> 16))));
}
template <> __device__ __forceinline__ float4 vload4<unorm16>(const unorm16 *p) {
    const uint2 r = __ldg(reinterpret_cast<const uint2 *>(p));
    const float s = 1.0f / 65535.0f;
    return make_float4((float)(r.x & 0xffffu) * s, (float)(r.x >> 16) * s, (float)(r.y & 0xffffu) * s,
                       (float)(r.y >> 16) * s);
}

// Origin and WM masses of record e of dim d's table (origin at word 0,
// masses at words 1..W, padded to a multiple of 4 words).
template <int WM>
__device__ __forceinline__ int32_t plane_record(const Geom &g, const uint32_t *tab, int d, int64_t e,
                                                float (&t)[WM]) {
    constexpr int NQ = (WM + 1 + 3) / 4;
    const uint4 *rec = reinterpret_cast<const uint4 *>(tab + g.toff[d] + e * g.trw[d]);
    uint32_t w[NQ * 4];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const uint4 v = __ldg(rec + q);
        w[q * 4 + 0] = v.x;
        w[q * 4 + 1] = v.y;
        w[q * 4 + 2] = v.z;
        w[q * 4 + 3] = v.w;
    }
    const int Wd = g.W[d];
#pragma unroll
    for (int k = 0; k < WM; ++k) t[k] = (k < Wd) ? __uint_as_float(w[1 + k]) : 0.0f;
    return (int32_t)w[0];
}

// A Z window moved onto the grid: with W == WM slots and N >= W cells, the
// window [o, o + W) is shifted to start s = clamp(o, 0, N - W) and its masses
// re-indexed (slots that leave the grid carried zero mass, the cells that
// enter it get zero mass), so that every slot addresses an on-grid cell and
// the slot addresses are affine.  The nonzero terms keep their order, so the
// sum is the same bit for bit.
template <int WM>
__device__ __forceinline__ int32_t plane_rebase(int32_t o, int32_t N, float (&t)[WM]) {
    const int32_t s = min(max(o, 0), N - WM);
    const int shift = s - o;
    if (shift != 0) {
        float u[WM];
#pragma unroll
        for (int k = 0; k < WM; ++k) {
            const int m = k + shift;
            u[k] = (m >= 0 && m < WM) ? sel_reg<WM>(t, m) : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < WM; ++k) t[k] = u[k];
    }
    return s;
}

// Stage 2 of the plane kernels for one state and one staged chunk: the sum
// over the state's B rows in the chunk (rows whose first-B-dim value falls
// in [c * chunk, (c + 1) * chunk)) of the product of its B masses and the
// row's sum over the Z window, accumulated row by row into (acc, comp).
// eB[b], eZ0, eZ1: the state part of the tables' indices; lo[b]: the low
// end of the staged range of B dim b; Rg: the group's staged rows.  The
// windows' masses are read from the tables (L1) here, so that nothing per
// state stays live across stage 1.
template <int WM>
__device__ __forceinline__ void plane_stage2(const Geom &g, const uint32_t *__restrict__ tab, const int32_t *up,
                                             int nB, const int32_t *bdim, const int32_t *eB, int32_t eZ0,
                                             int32_t eZ1, const int32_t *lo, const float *Rg, int rs0, int rs1,
                                             int chunk, int c, int Ppad, int kahan, float &acc, float &comp,
                                             uint32_t &n_rld, uint32_t &n_rows, bool count) {
    const int n = g.n;
    const int32_t Nz0 = g.N[n - 2], Nz1 = g.N[n - 1];
    // B windows: origin rows in the staged ranges, masses read where used
    const uint32_t *rb[PLANE_MAXB];
    int32_t ys[PLANE_MAXB];
    int Wb[PLANE_MAXB];
#pragma unroll
    for (int b = 0; b < PLANE_MAXB; ++b) {
        rb[b] = nullptr;
        ys[b] = 0;
        Wb[b] = 1;
        if (b < nB) {
            const int d = bdim[b];
            rb[b] = tab + g.toff[d] + (int64_t)(eB[b] + __ldg(up + d)) * g.trw[d];
            ys[b] = (int32_t)__ldg(rb[b]) - lo[b];
            Wb[b] = g.W[d];
        }
    }
    const int32_t y0s = ys[0] - c * chunk;
    const int j0lo = max(0, -y0s), j0hi = min(Wb[0], chunk - y0s);
    if (j0lo >= j0hi) return;  // no row of this chunk
    float tz0[WM], tz1[WM];
    const int32_t oz0 = plane_record<WM>(g, tab, n - 2, eZ0 + __ldg(up + n - 2), tz0);
    const int32_t oz1 = plane_record<WM>(g, tab, n - 1, eZ1 + __ldg(up + n - 1), tz1);
    const bool affine = g.W[n - 2] == WM && g.W[n - 1] == WM && Nz0 >= WM && Nz1 >= WM;
    int32_t zb = 0;  // affine: offset of the window's first cell in a row
    if (affine) zb = plane_rebase<WM>(oz0, Nz0, tz0) * Nz1 + plane_rebase<WM>(oz1, Nz1, tz1);
    // Z-window sum of one staged row
    auto zsum = [&](const float *row) {
        float in = 0.0f;
        if (affine) {
            const float *rz = row + zb;
#pragma unroll
            for (int k0 = 0; k0 < WM; ++k0) {
                const float *rr = rz + k0 * Nz1;
                float q = 0.0f;
#pragma unroll
                for (int k1 = 0; k1 < WM; ++k1) q = fmaf(tz1[k1], rr[k1], q);
                in = fmaf(tz0[k0], q, in);
            }
        } else {
            // clamped cells: off-grid slots carry zero mass and read a valid R entry
#pragma unroll
            for (int k0 = 0; k0 < WM; ++k0) {
                const float *rr = row + min(max(oz0 + k0, 0), Nz0 - 1) * Nz1;
                float q = 0.0f;
#pragma unroll
                for (int k1 = 0; k1 < WM; ++k1) q = fmaf(tz1[k1], rr[min(max(oz1 + k1, 0), Nz1 - 1)], q);
                in = fmaf(tz0[k0], q, in);
            }
        }
        return in;
    };
#if AMY_FFMA2_S2
    // affine windows: the Z sums of two staged rows at once, each row's terms
    // in the order zsum takes them
    auto zsum2 = [&](const float *ra, const float *rc) {
        float2 in = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int k0 = 0; k0 < WM; ++k0) {
            const float *pa = ra + zb + k0 * Nz1, *pc = rc + zb + k0 * Nz1;
            float2 q = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int k1 = 0; k1 < WM; ++k1)
                q = __ffma2_rn(make_float2(tz1[k1], tz1[k1]), make_float2(pa[k1], pc[k1]), q);
            in = __ffma2_rn(make_float2(tz0[k0], tz0[k0]), q, in);
        }
        return in;
    };
#endif
    // one row's Z sum with its Z rows taken in pairs (the same chains as zsum)
    auto zsum_row = [&](const float *row) {
#if AMY_FFMA2_S2T
        if (affine) {
            const float *rz = row + zb;
            float q[WM];
#pragma unroll
            for (int k0 = 0; k0 + 1 < WM; k0 += 2) {
                float2 qq = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int k1 = 0; k1 < WM; ++k1)
                    qq = __ffma2_rn(make_float2(tz1[k1], tz1[k1]),
                                    make_float2(rz[k0 * Nz1 + k1], rz[(k0 + 1) * Nz1 + k1]), qq);
                q[k0] = qq.x;
                q[k0 + 1] = qq.y;
            }
            if (WM % 2) {
                float qq = 0.0f;
#pragma unroll
                for (int k1 = 0; k1 < WM; ++k1) qq = fmaf(tz1[k1], rz[(WM - 1) * Nz1 + k1], qq);
                q[WM - 1] = qq;
            }
            float in = 0.0f;
#pragma unroll
            for (int k0 = 0; k0 < WM; ++k0) in = fmaf(tz0[k0], q[k0], in);
            return in;
        }
#endif
        return zsum(row);
    };
    auto add_row = [&](float w, float in) {
        accum_row(acc, comp, __fmul_rn(w, in), kahan);
        if (count) {
            n_rld += (uint32_t)(g.W[n - 2] * g.W[n - 1]);
            ++n_rows;
        }
    };
    // the row loops stay rolled (one copy of the Z contraction per batch in
    // the code); rows of the second B dim go PLANE_S2ROWS at a time, each
    // batch's sums formed together and added in row order
#pragma unroll 1
    for (int j0 = j0lo; j0 < j0hi; ++j0) {
        const int32_t y0 = y0s + j0;
        const float w0 = nB > 0 ? __uint_as_float(__ldg(rb[0] + 1 + j0)) : 1.0f;
        if (w0 == 0.0f) continue;
        if (nB == 2) {
            const float *r0 = Rg + (int64_t)(y0 * rs0 + ys[1]) * Ppad;
            int j1 = 0;
#pragma unroll 1
            for (; j1 + PLANE_S2ROWS <= Wb[1]; j1 += PLANE_S2ROWS) {
                float wr[PLANE_S2ROWS], in[PLANE_S2ROWS];
                bool any = false;
#pragma unroll
                for (int q = 0; q < PLANE_S2ROWS; ++q) {
                    wr[q] = __fmul_rn(w0, __uint_as_float(__ldg(rb[1] + 1 + j1 + q)));
                    any = any || wr[q] != 0.0f;
                }
                if (!any) continue;
#if AMY_FFMA2_S2
                if (affine) {
#pragma unroll
                    for (int q = 0; q + 1 < PLANE_S2ROWS; q += 2) {
                        const float2 s2 = zsum2(r0 + (int64_t)(j1 + q) * rs1 * Ppad,
                                                r0 + (int64_t)(j1 + q + 1) * rs1 * Ppad);
                        in[q] = s2.x;
                        in[q + 1] = s2.y;
                    }
                    if (PLANE_S2ROWS % 2)
                        in[PLANE_S2ROWS - 1] = zsum_row(r0 + (int64_t)(j1 + PLANE_S2ROWS - 1) * rs1 * Ppad);
                } else
#endif
                {
#pragma unroll
                    for (int q = 0; q < PLANE_S2ROWS; ++q) in[q] = zsum(r0 + (int64_t)(j1 + q) * rs1 * Ppad);
                }
#pragma unroll
                for (int q = 0; q < PLANE_S2ROWS; ++q)
                    if (wr[q] != 0.0f) add_row(wr[q], in[q]);
            }
#pragma unroll 1
            for (; j1 < Wb[1]; ++j1) {
                const float wa = __fmul_rn(w0, __uint_as_float(__ldg(rb[1] + 1 + j1)));
                if (wa != 0.0f) add_row(wa, zsum_row(r0 + (int64_t)j1 * rs1 * Ppad));
            }
            continue;
        }
#pragma unroll 1
        for (int j1 = 0; j1 < Wb[1]; ++j1) {
            const float w1 = nB > 1 ? __fmul_rn(w0, __uint_as_float(__ldg(rb[1] + 1 + j1))) : w0;
            if (w1 == 0.0f) continue;
            for (int j2 = 0; j2 < Wb[2]; ++j2) {
                const float w = nB > 2 ? __fmul_rn(w1, __uint_as_float(__ldg(rb[2] + 1 + j2))) : w1;
                if (w == 0.0f) continue;
                add_row(w, zsum_row(Rg + (int64_t)(y0 * rs0 + (ys[1] + j1) * rs1 + (ys[2] + j2)) * Ppad));
            }
        }
    }
}

template <class VT, int WM>
__global__ void __launch_bounds__(PLANE_MAX_THREADS, 2) k_backup_plane(const __grid_constant__ Geom g,
                                                                   const __grid_constant__ PlaneArgs<VT> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = a.G, P = a.P, K = a.K, nB = a.nB;
    int32_t *s_lo = reinterpret_cast<int32_t *>(smem_raw);     // [G][PLANE_MAXB]
    int32_t *s_hi = s_lo + G * PLANE_MAXB;                      // [G][PLANE_MAXB]
    int32_t *s_eS = s_hi + G * PLANE_MAXB;                      // [G][PLANE_MAXS]
    int32_t *s_any = s_eS + G * PLANE_MAXS;                     // [G]: a free state in the group
    float *s_w = reinterpret_cast<float *>(s_any + G);              // [G][K]
    int32_t *s_off = reinterpret_cast<int32_t *>(s_w + G * K);      // [G][K], padded-V offsets
    float *s_R = reinterpret_cast<float *>(smem_raw + plane_smem_head(G, K));  // [G][rent][Ppad]
    const int Ppad = a.Ppad;

    const int n = g.n;
    const int tid = threadIdx.x;
    const int gl = tid / P;                     // group within the block
    const int p = tid - gl * P;                 // plane position
    const int64_t gi = (int64_t)blockIdx.x * G + gl;
    const bool gvalid = gl < G && gi < a.ngroups;
    const int64_t x64 = gi * P + p;
    const int32_t x = gvalid ? (int32_t)x64 : 0;
    const uint8_t f = gvalid ? a.mask[x] : (uint8_t)0;
    const bool masked = gvalid && state_masked(a.spec_kind, f);
    const bool fr = gvalid && !masked;

    // coordinates: F from the group index, Z from the plane position
    int32_t xi[MAXD];
    {
        int64_t r = gvalid ? gi : 0;
        const int32_t pr = p / a.N1;
#pragma unroll
        for (int d = MAXD - 1; d >= 0; --d) {
            xi[d] = 0;
            if (d < n - 2) {
                xi[d] = (int32_t)(r % g.N[d]);
                r /= g.N[d];
            } else if (d == n - 2) {
                xi[d] = pr;
            } else if (d == n - 1) {
                xi[d] = p - pr * a.N1;
            }
        }
    }
    // state part of every dim's table index (tables hold fewer than 2^31 records)
    auto tab_index = [&](int d) {
        int32_t e = 0;
#pragma unroll
        for (int j = 0; j < MAXD; ++j)
            if (j < n) e += xi[j] * g.tsx[d][j];
        return e;
    };
    int32_t eB[PLANE_MAXB];
#pragma unroll
    for (int b = 0; b < PLANE_MAXB; ++b) eB[b] = b < nB ? tab_index(a.bdim[b]) : 0;
    const int32_t eZ0 = tab_index(n - 2), eZ1 = tab_index(n - 1);
    // S dims depend on F coordinates only: one table index per group
    if (gvalid)
        for (int q = p; q < a.nS; q += P) s_eS[gl * PLANE_MAXS + q] = tab_index(a.sdim[q]);

    const int bd0 = nB > 0 ? a.bdim[0] : 0;
    const int32_t Nz0 = g.N[n - 2], Nz1 = g.N[n - 1];
    float best = -1.0f;
    int32_t arg = 0x7fffffff;
    uint32_t n_vld = 0, n_rld = 0, n_rows = 0;  // work counters (used when a.work is set)

    for (int i = tid; i < G * PLANE_MAXB; i += blockDim.x) {
        s_lo[i] = INT_MAX;
        s_hi[i] = INT_MIN;
    }
    for (int i = tid; i < G; i += blockDim.x) s_any[i] = 0;
    __syncthreads();
    // stage-1 role of this thread: group, team and four-position column
    const int s1g = tid / (a.teams * a.Q);
    const int s1r = (tid / a.Q) - s1g * a.teams;
    const int s1q = tid - (tid / a.Q) * a.Q;
    const bool s1valid = s1g < G && (int64_t)blockIdx.x * G + s1g < a.ngroups;
    for (int u = 0; u < g.nu; ++u) {
        const int32_t *up = reinterpret_cast<const int32_t *>(a.tab + g.uoff + (int64_t)u * g.urw);
        // ---- A: this state's B origins into its group's bounds; the group's
        // S combinations (weight and cell offset each)
        if (fr) {
            s_any[gl] = 1;
#pragma unroll
            for (int b = 0; b < PLANE_MAXB; ++b) {
                if (b < nB) {
                    const int d = a.bdim[b];
                    const int32_t o =
                        (int32_t)__ldg(a.tab + g.toff[d] + (int64_t)(eB[b] + __ldg(up + d)) * g.trw[d]);
                    atomicMin(&s_lo[gl * PLANE_MAXB + b], o);
                    atomicMax(&s_hi[gl * PLANE_MAXB + b], o);
                }
            }
        }
        if (gvalid) {
            for (int k = p; k < K; k += P) {
                // S combination k (last S dim fastest): product of its masses in
                // dim order, offset of its cells; off-grid slots weigh zero
                int32_t r = k, off = 0;
                int32_t js[PLANE_MAXS];
#pragma unroll
                for (int s = PLANE_MAXS - 1; s >= 0; --s) {
                    js[s] = 0;
                    if (s < a.nS) {
                        const int Wd = g.W[a.sdim[s]];
                        js[s] = r % Wd;
                        r /= Wd;
                    }
                }
                float w = 1.0f;
#pragma unroll
                for (int s = 0; s < PLANE_MAXS; ++s) {
                    if (s < a.nS) {
                        const int d = a.sdim[s];
                        // S dims depend on F coordinates only: the same record for the group
                        const uint32_t *rec =
                            a.tab + g.toff[d] + (int64_t)(s_eS[gl * PLANE_MAXS + s] + __ldg(up + d)) * g.trw[d];
                        const int32_t cell = (int32_t)__ldg(rec) + js[s];
                        const bool on = cell >= 0 && cell < g.N[d];
                        w = __fmul_rn(w, on ? __uint_as_float(__ldg(rec + 1 + js[s])) : 0.0f);
                        off += (on ? cell : 0) * (g.stride[d] / P);
                    }
                }
                s_w[gl * K + k] = w;
                s_off[gl * K + k] = off * Ppad;
            }
        }
        __syncthreads();
        // ---- B: the groups' staged ranges, then stage 1 / stage 2 per chunk
        // (stage 2 reads its own group's ranges, stage 1 those of the group
        // its team works for)
        // (both are read from shared memory where they are used, so that no
        // register holds them across the other stage)
        const bool s1free = s1valid && s_any[s1g] != 0;
        float acc = 0.0f, comp = 0.0f;
        const int nch = nB > 0 ? (a.brange[0] + a.chunk - 1) / a.chunk : 1;
        const float *Rg = s_R + (int64_t)gl * a.rent * Ppad;
        const int rs1 = nB > 2 ? a.brange[2] : 1;
        for (int c = 0; c < nch; ++c) {
            // stage 1: this chunk's rows of the team's group, four positions per
            // thread.  The used rows (first B value in the chunk and below the
            // group's range, the other B values below theirs) are dealt to the
            // teams in turn, PLANE_EB at a time; each row sums its S
            // combinations in order, PLANE_KU of them per step.
            if (s1free) {
                int32_t lob1[PLANE_MAXB], rng1[PLANE_MAXB];
#pragma unroll
                for (int b = 0; b < PLANE_MAXB; ++b) {
                    lob1[b] = 0;
                    rng1[b] = 1;
                    if (b < nB) {
                        lob1[b] = s_lo[s1g * PLANE_MAXB + b];
                        rng1[b] = s_hi[s1g * PLANE_MAXB + b] - lob1[b] + g.W[a.bdim[b]];
                    }
                }
                const int n0 = nB > 0 ? min(a.chunk, rng1[0] - c * a.chunk) : 1;
                const int nr1 = nB > 1 ? rng1[1] : 1, nr2 = nB > 2 ? rng1[2] : 1;
                const int nr = n0 > 0 ? n0 * nr1 * nr2 : 0;
                float *Rw = s_R + (int64_t)s1g * a.rent * Ppad + 4 * s1q;
                const float *ws = s_w + s1g * K;
                const int32_t *os = s_off + s1g * K;
                const VT *vq = a.Vpn + 4 * s1q;
                for (int f0 = s1r; f0 < nr; f0 += a.teams * PLANE_EB) {
                    const VT *pr[PLANE_EB];
                    int32_t er[PLANE_EB];
                    bool live[PLANE_EB], on[PLANE_EB];
#pragma unroll
                    for (int i = 0; i < PLANE_EB; ++i) {
                        const int f = f0 + i * a.teams;
                        live[i] = f < nr;
                        const int ff = live[i] ? f : 0;
                        const int y2 = ff % nr2, y1 = (ff / nr2) % nr1, y0 = ff / (nr2 * nr1) + c * a.chunk;
                        er[i] = (y0 - c * a.chunk) * a.rs0 + y1 * rs1 + y2;
                        int32_t y[PLANE_MAXB] = {y0, y1, y2};
                        bool ok = true;
                        int32_t bF = 0;  // plane index of the row's B cells
#pragma unroll
                        for (int b = 0; b < PLANE_MAXB; ++b) {
                            if (b < nB) {
                                const int32_t cell = lob1[b] + y[b];
                                ok = ok && cell >= 0 && cell < g.N[a.bdim[b]];
                                bF += (ok ? cell : 0) * a.bstrideF[b];
                            }
                        }
                        on[i] = live[i] && ok;
                        pr[i] = vq + (on[i] ? bF : 0) * Ppad;  // off-grid rows read a valid plane, then weigh 0
                    }
                    float4 r[PLANE_EB];
#pragma unroll
                    for (int i = 0; i < PLANE_EB; ++i) r[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    int k = 0;
                    for (; k + PLANE_KU <= K; k += PLANE_KU) {
                        float4 v[PLANE_KU][PLANE_EB];
#pragma unroll
                        for (int q = 0; q < PLANE_KU; ++q) {
                            const int32_t o = os[k + q];
#pragma unroll
                            for (int i = 0; i < PLANE_EB; ++i) v[q][i] = vload4<VT>(pr[i] + o);
                        }
#pragma unroll
                        for (int q = 0; q < PLANE_KU; ++q) {
                            const float w = ws[k + q];
#pragma unroll
                            for (int i = 0; i < PLANE_EB; ++i) fma4<AMY_FFMA2_P1 != 0 && WM <= 3>(w, v[q][i], r[i]);
                        }
                    }
                    for (; k < K; ++k) {
                        const float w = ws[k];
                        const int32_t o = os[k];
#pragma unroll
                        for (int i = 0; i < PLANE_EB; ++i) {
                            fma4<AMY_FFMA2_P1 != 0 && WM <= 3>(w, vload4<VT>(pr[i] + o), r[i]);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < PLANE_EB; ++i) {
                        if (live[i])
                            *reinterpret_cast<float4 *>(Rw + (int64_t)er[i] * Ppad) =
                                on[i] ? r[i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        if (a.work && on[i]) n_vld += 4u * (uint32_t)K;
                    }
                }
            }
            __syncthreads();
            // stage 2: this state's B rows that fall in the chunk
            if (fr)
                plane_stage2<WM>(g, a.tab, up, nB, a.bdim, eB, eZ0, eZ1, s_lo + gl * PLANE_MAXB, Rg, a.rs0, rs1,
                                 a.chunk, c, Ppad, a.kahan, acc, comp, n_rld, n_rows, a.work != nullptr);
            __syncthreads();
        }
        if (fr && acc > best) {
            best = acc;
            arg = u;
        }
        for (int i = tid; i < G * PLANE_MAXB; i += blockDim.x) {
            s_lo[i] = INT_MAX;
            s_hi[i] = INT_MIN;
        }
        for (int i = tid; i < G; i += blockDim.x) s_any[i] = 0;
        __syncthreads();
    }
    if (a.work) {
        unsigned long long c0 = n_vld, c1 = n_rld, c2 = n_rows;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c0 += __shfl_down_sync(0xffffffffu, c0, o);
            c1 += __shfl_down_sync(0xffffffffu, c1, o);
            c2 += __shfl_down_sync(0xffffffffu, c2, o);
        }
        if ((tid & 31) == 0) {
            atomicAdd(a.work + 0, c0);
            atomicAdd(a.work + 1, c1);
            atomicAdd(a.work + 2, c2);
        }
    }
    if (gvalid) {
        uint16_t pol;
        if (masked) {
            best = (a.spec_kind != SPEC_SAFETY && (f & F_TARGET)) ? 1.0f : 0.0f;
            pol = 0xFFFF;
        } else {
            pol = (uint16_t)arg;
        }
        const VT vb = vstore_cast<VT, float>(best);
        a.Vo[x] = vb;
        a.Vpo[gi * Ppad + p] = vb;
        if (a.Vfinal) a.Vfinal[x] = best;
        if (a.pi) a.pi[x] = pol;
    }
}

// Padded copy of a V vector for the plane kernel: plane r's P values at
// Vp[r * Ppad ...], zeros in the Ppad - P pad entries.
template <class VT>
__global__ void k_plane_repack(const VT *__restrict__ V, VT *__restrict__ Vp, int64_t rows, int32_t P, int32_t Ppad) {
    const int64_t total = rows * Ppad;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / Ppad;
        const int32_t q = (int32_t)(i - r * Ppad);
        VT z;
        memset(&z, 0, sizeof z);
        Vp[i] = q < P ? V[r * P + q] : z;
    }
}

// Largest spread (max - min) of dim d's window origin over one plane of
// states, for every F dim whose mean component depends on a plane
// coordinate, written to the bounds block (word boff + 2 * MAXD + 4 + d).
// One thread per table record whose plane coordinates are zero; it walks
// the records of the plane coordinates the component depends on.
static __global__ void k_plane_spread(const __grid_constant__ Geom g, uint32_t *__restrict__ tab) {
    const int n = g.n;
    if (n < 3) return;
    int32_t *spread = reinterpret_cast<int32_t *>(tab + g.boff) + 2 * MAXD + 4;
    for (int d = 0; d < n - 2; ++d) {
        const int32_t s0 = g.tsx[d][n - 2], s1 = g.tsx[d][n - 1];
        if (s0 == 0 && s1 == 0) continue;
        const int32_t m0 = s0 ? g.N[n - 2] : 1, m1 = s1 ? g.N[n - 1] : 1;
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < g.tent[d];
             e += (int64_t)gridDim.x * blockDim.x) {
            if ((s0 && (e / s0) % g.N[n - 2] != 0) || (s1 && (e / s1) % g.N[n - 1] != 0)) continue;
            int32_t lo = INT_MAX, hi = INT_MIN;
            for (int32_t i0 = 0; i0 < m0; ++i0)
                for (int32_t i1 = 0; i1 < m1; ++i1) {
                    const int64_t r = e + (int64_t)i0 * s0 + (int64_t)i1 * s1;
                    const int32_t o = (int32_t)tab[g.toff[d] + r * g.trw[d]];
                    lo = min(lo, o);
                    hi = max(hi, o);
                }
            atomicMax(spread + d, hi - lo);
        }
    }
}

}  // namespace amy
