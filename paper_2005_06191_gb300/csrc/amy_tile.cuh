// amy_tile.cuh -- the plane kernel's window sum with its first stage shared
// by a tile of neighbouring groups (backup kernel 8).
//
// Notation as in amy_plane.cuh: Z = the two innermost dims (a plane of P
// states), F = the others, a group = the states sharing their F
// coordinates, S = the F dims whose windows a whole group shares, B = F
// minus S (windows moving across the plane, staged as ranges).
//
// A tile is T groups that differ only in one F coordinate x_a, where a is
// the first B dim and no other B dim's component reads x_a.  The S dims split
// into Sh, whose components do not read x_a either -- their window origins
// and masses are the same for every group of the tile -- and at most one
// dim o (Ow) whose window moves with x_a.  For one input and one staged row
// y_B, with the Ow window's union over the tile [lo_o, lo_o + n_o):
//   stage 1a: A[c][p] = sum_{j in Sh} (prod_{d in Sh} t_d[j_d]) V[y_B, lo_o + c, o_Sh + j, p]
//             for every c < n_o, once for the whole tile;
//   stage 1b: R_g[y_B][p] = sum_{j < W_o} t_{o,g}[j] A[o_{o,g} - lo_o + j][p]  for each group g;
//   stage 2:  as in the plane kernel, per state from its group's R_g.
// Stage 1 thus reads n_o * K_Sh planes of V per staged row for the whole
// tile, where the plane kernel reads K = W_o * K_Sh planes per row and group.
// Every term of the window sum appears once (an exact reassociation); the
// FP32 rounding order differs from the plane kernel's (the Ow masses are
// applied after the Sh sums instead of inside the product of weights).
#pragma once

#include "amy_plane.cuh"

namespace amy {

#ifndef AMY_TILE_MAXT
#define AMY_TILE_MAXT 4
#endif
constexpr int TILE_MAXT = AMY_TILE_MAXT;  // groups per tile (at most)
#ifndef AMY_TILE_KU
#define AMY_TILE_KU 2
#endif
// Sh combinations per step (two Ow cells at a time: 2 * TILE_KU loads in flight)
constexpr int TILE_KU = AMY_TILE_KU;
// Blocks per SM the kernel is compiled for (its register cap), and the
// planner's first choice: the shared memory of one block and the values of
// the first staged dim it must hold at once for that many blocks per SM
#ifndef AMY_TILE_MINB
#define AMY_TILE_MINB 2
#endif
constexpr int TILE_MINB = AMY_TILE_MINB;
#ifndef AMY_TILE_BUDGET0
#define AMY_TILE_BUDGET0 (112 * 1024)
#endif
#ifndef AMY_TILE_WANT0
#define AMY_TILE_WANT0 2
#endif
constexpr int TILE_BUDGET0 = AMY_TILE_BUDGET0;
constexpr int TILE_WANT0 = AMY_TILE_WANT0;
constexpr int TILE_MAX_THREADS = 448;
// Extra floats between consecutive staged rows of R (a multiple of 4): the row
// pitch Ppad + AMY_TILE_RPAD moves rows onto other shared-memory banks.
#ifndef AMY_TILE_RPAD
#define AMY_TILE_RPAD 0
#endif
constexpr int TILE_RPAD = AMY_TILE_RPAD;

template <class VT> struct TileArgs {
    VT *Vo;                // V_k
    const VT *Vpn;         // V_{k+1}, planes padded to Ppad values
    VT *Vpo;               // V_k, padded
    float *Vfinal;         // optional FP32 copy of V_k
    uint16_t *pi;          // optional policy of this step
    const uint8_t *mask;
    const uint32_t *tab;
    int32_t spec_kind;
    int32_t kahan;
    int32_t P, N1, Ppad, Q;
    int32_t adim;          // tile dim a (= the first B dim)
    int32_t T;             // groups per tile
    int32_t Na;            // points of dim a
    int32_t ntiles_a;      // tiles along dim a: ceil(Na / T)
    int64_t nrest;         // groups per value of dim a
    int32_t nB;
    int32_t bdim[PLANE_MAXB];
    int32_t brange[PLANE_MAXB];   // bound of the staged range per B dim (the first: unused)
    int32_t bstrideF[PLANE_MAXB];
    int32_t rs0;           // R rows per value of the first B dim
    int32_t chunk;         // values of the first B dim per chunk
    int32_t rent;          // R rows per group and chunk: chunk * rs0
    int32_t nSh;
    int32_t shdim[PLANE_MAXS];
    int32_t Ksh;           // Sh combinations: prod_{d in Sh} W[d]
    int32_t ow;            // the Ow dim, or -1 (every S dim shared)
    int32_t owstrideF;     // plane-index stride of the Ow dim
    unsigned long long *work;  // optional counters, as the plane kernel's
};

// Shared memory: tile bounds and flags, the tile's table-index bases, the
// Sh combinations' weights and offsets, each group's Ow origin and masses,
// every state's running sum, compensation, best value and input, then R for
// the T groups.
__host__ __device__ inline size_t tile_smem_head(int Ksh, int threads, int T) {
    return ((size_t)(2 * PLANE_MAXB + 4 + MAXD) * 4 + (size_t)Ksh * 8 + (size_t)TILE_MAXT * 4 +
            (size_t)TILE_MAXT * 16 * 4 + (size_t)4 * T * threads * 4 + 15) / 16 * 16;
}
__host__ __device__ inline size_t tile_smem_bytes(int Ksh, int threads, int T, int rent, int Ppad) {
    return tile_smem_head(Ksh, threads, T) + (size_t)T * rent * (Ppad + TILE_RPAD) * 4;
}

template <class VT, int WM>
__global__ void __launch_bounds__(TILE_MAX_THREADS, TILE_MINB) k_backup_tile(const __grid_constant__ Geom g,
                                                                 const __grid_constant__ TileArgs<VT> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int32_t *s_lo = reinterpret_cast<int32_t *>(smem_raw);                // [PLANE_MAXB] tile bounds
    int32_t *s_hi = s_lo + PLANE_MAXB;                                    // [PLANE_MAXB]
    int32_t *s_any = s_hi + PLANE_MAXB;                                   // a free state in the tile
    int32_t *s_base = s_lo + 2 * PLANE_MAXB + 4;                          // [MAXD] tile table-index parts
    float *s_shw = reinterpret_cast<float *>(s_base + MAXD);              // [Ksh] Sh weights
    int32_t *s_sho = reinterpret_cast<int32_t *>(s_shw + a.Ksh);          // [Ksh] padded-V offsets
    int32_t *s_owo = s_sho + a.Ksh;                                       // [TILE_MAXT] Ow origins
    float *s_oww = reinterpret_cast<float *>(s_owo + TILE_MAXT);          // [TILE_MAXT][16] Ow masses
    // per state i of this thread (i < T: a thread holds at most T states)
    float *s_acc = s_oww + TILE_MAXT * 16;                                // [T][threads] sums
    float *s_cmp = s_acc + a.T * blockDim.x;                              // [T][threads] compensations
    float *s_best = s_cmp + a.T * blockDim.x;                             // [T][threads] best value
    int32_t *s_arg = reinterpret_cast<int32_t *>(s_best + a.T * blockDim.x);  // its input
    float *s_R = reinterpret_cast<float *>(smem_raw + tile_smem_head(a.Ksh, blockDim.x, a.T));  // [T][rent][Rp]

    const int n = g.n;
    const int tid = threadIdx.x, NT = blockDim.x;
    const int P = a.P, Ppad = a.Ppad, Q = a.Q;
    const int Rp = Ppad + TILE_RPAD;  // row pitch of R
    const int ad = a.adim;
    const int64_t rest = (int64_t)blockIdx.x % a.nrest;
    const int32_t a0 = (int32_t)((int64_t)blockIdx.x / a.nrest) * a.T;
    const int Tt = min(a.T, a.Na - a0);
    // F coordinates of the tile's first group (dim a at a0): its plane index,
    // and per dim the F part of the table index (in shared memory)
    int64_t gplane0 = 0;
    {
        int32_t fc[MAXD];
        int64_t r = rest;
#pragma unroll
        for (int d = MAXD - 1; d >= 0; --d) {
            fc[d] = 0;
            if (d < n - 2 && d != ad) {
                fc[d] = (int32_t)(r % g.N[d]);
                r /= g.N[d];
            }
        }
        fc[ad] = a0;
#pragma unroll
        for (int d = 0; d < MAXD; ++d)
            if (d < n - 2) gplane0 += (int64_t)fc[d] * (g.stride[d] / P);
        if (tid < n) {
            int32_t e = 0;
#pragma unroll
            for (int j = 0; j < MAXD; ++j)
                if (j < n - 2) e += fc[j] * g.tsx[tid][j];
            s_base[tid] = e;
        }
    }
    const int64_t astrideF = g.stride[ad] / P;
    // table index of dim d at group gg, plane position p
    auto tab_index = [&](int d, int gg, int p) {
        const int32_t z0 = p / a.N1, z1 = p - (p / a.N1) * a.N1;
        return s_base[d] + gg * g.tsx[d][ad] + z0 * g.tsx[d][n - 2] + z1 * g.tsx[d][n - 1];
    };
    const int32_t Nz0 = g.N[n - 2], Nz1 = g.N[n - 1];
    const int nB = a.nB;
    const int bd0 = a.bdim[0];
    const int rs1 = nB > 2 ? a.brange[2] : 1;
    const int Wow = a.ow >= 0 ? g.W[a.ow] : 1;

    for (int i = 0; i < a.T; ++i) {
        s_best[i * NT + tid] = -1.0f;
        s_arg[i * NT + tid] = 0x7fffffff;
    }
    // this thread's states: s = tid + i * NT, group s / P, position s % P
    uint32_t freebits = 0, livebits = 0;
#pragma unroll
    for (int i = 0; i < TILE_MAXT; ++i) {
        const int s = tid + i * NT;
        const int gg = s / P, p = s - gg * P;
        if (gg < Tt) {
            livebits |= 1u << i;
            const int64_t x = (gplane0 + gg * astrideF) * P + p;
            if (!state_masked(a.spec_kind, a.mask[x])) freebits |= 1u << i;
        }
    }
    uint32_t n_vld = 0, n_rld = 0, n_rows = 0;
    // stage-1 role: team of Q threads and four-position column
    const int s1teams = NT / Q, s1team = tid / Q, s1q = tid - (tid / Q) * Q;
    if (tid < PLANE_MAXB) {
        s_lo[tid] = INT_MAX;
        s_hi[tid] = INT_MIN;
    }
    if (tid == 0) s_any[0] = 0;
    __syncthreads();
    for (int u = 0; u < g.nu; ++u) {
        const int32_t *up = reinterpret_cast<const int32_t *>(a.tab + g.uoff + (int64_t)u * g.urw);
        // ---- A: the tile's B bounds from its free states; each group's Ow
        // window; the Sh combinations (the same for every group of the tile)
#pragma unroll
        for (int i = 0; i < TILE_MAXT; ++i) {
            if (freebits & (1u << i)) {
                const int s = tid + i * NT;
                const int gg = s / P, p = s - gg * P;
                s_any[0] = 1;
#pragma unroll
                for (int b = 0; b < PLANE_MAXB; ++b) {
                    if (b < nB) {
                        const int d = a.bdim[b];
                        const int32_t o = (int32_t)__ldg(a.tab + g.toff[d] +
                                                         (int64_t)(tab_index(d, gg, p) + __ldg(up + d)) * g.trw[d]);
                        atomicMin(&s_lo[b], o);
                        atomicMax(&s_hi[b], o);
                    }
                }
            }
        }
        if (tid < TILE_MAXT) {
            const int gg = tid;
            if (a.ow >= 0 && gg < Tt) {
                const int d = a.ow;
                const uint32_t *rec = a.tab + g.toff[d] + (int64_t)(tab_index(d, gg, 0) + __ldg(up + d)) * g.trw[d];
                const int32_t o = (int32_t)__ldg(rec);
                s_owo[gg] = o;
                for (int j = 0; j < 16; ++j) {
                    const int32_t cell = o + j;
                    s_oww[gg * 16 + j] =
                        (j < Wow && cell >= 0 && cell < g.N[d]) ? __uint_as_float(__ldg(rec + 1 + j)) : 0.0f;
                }
            } else {
                s_owo[gg] = 0;
                for (int j = 0; j < 16; ++j) s_oww[gg * 16 + j] = (j == 0) ? 1.0f : 0.0f;
            }
        }
        for (int k = tid; k < a.Ksh; k += NT) {
            // Sh combination k (last Sh dim fastest): product of its masses in
            // dim order, offset of its cells; off-grid slots weigh zero
            int32_t r = k, off = 0;
            int32_t js[PLANE_MAXS];
#pragma unroll
            for (int q = PLANE_MAXS - 1; q >= 0; --q) {
                js[q] = 0;
                if (q < a.nSh) {
                    const int Wd = g.W[a.shdim[q]];
                    js[q] = r % Wd;
                    r /= Wd;
                }
            }
            float w = 1.0f;
#pragma unroll
            for (int q = 0; q < PLANE_MAXS; ++q) {
                if (q < a.nSh) {
                    const int d = a.shdim[q];
                    const uint32_t *rec = a.tab + g.toff[d] + (int64_t)(tab_index(d, 0, 0) + __ldg(up + d)) * g.trw[d];
                    const int32_t cell = (int32_t)__ldg(rec) + js[q];
                    const bool on = cell >= 0 && cell < g.N[d];
                    w = __fmul_rn(w, on ? __uint_as_float(__ldg(rec + 1 + js[q])) : 0.0f);
                    off += (on ? cell : 0) * (g.stride[d] / P);
                }
            }
            s_shw[k] = w;
            s_sho[k] = off * Ppad;
        }
        __syncthreads();
        if (s_any[0] != 0) {  // block-uniform
            int32_t owlo = INT_MAX, owhi = INT_MIN;
            for (int gg = 0; gg < Tt; ++gg) {
                owlo = min(owlo, s_owo[gg]);
                owhi = max(owhi, s_owo[gg]);
            }
            const int own = owhi - owlo + Wow;
            const int n0 = s_hi[0] - s_lo[0] + g.W[bd0];
            const int nr1 = nB > 1 ? s_hi[1] - s_lo[1] + g.W[a.bdim[1]] : 1;
            const int nr2 = nB > 2 ? s_hi[2] - s_lo[2] + g.W[a.bdim[2]] : 1;
            for (int i = 0; i < a.T; ++i) {
                s_acc[i * NT + tid] = 0.0f;
                s_cmp[i * NT + tid] = 0.0f;
            }
            const int nch = (n0 + a.chunk - 1) / a.chunk;
            for (int c = 0; c < nch; ++c) {
                // ---- stage 1: this chunk's rows, dealt to the teams of Q threads
                // (four plane positions per thread) in turn; per row each Ow cell
                // of the union sums its Sh combinations in order (stage 1a),
                // then every group adds it with its own Ow mass (stage 1b)
                const int n0c = min(a.chunk, n0 - c * a.chunk);
                const int nrows = n0c * nr1 * nr2;
                for (int f = s1team; s1team < s1teams && f < nrows; f += s1teams) {
                    int y2 = 0, y1 = 0, y0l = f;
                    if (nB > 2) {
                        y2 = y0l % nr2;
                        y0l /= nr2;
                    }
                    if (nB > 1) {
                        y1 = y0l % nr1;
                        y0l /= nr1;
                    }
                    const int er = y0l * a.rs0 + y1 * rs1 + y2;
                    const int32_t yy[PLANE_MAXB] = {c * a.chunk + y0l, y1, y2};
                    bool on = true;
                    int32_t bF = 0;
#pragma unroll
                    for (int b = 0; b < PLANE_MAXB; ++b) {
                        if (b < nB) {
                            const int32_t cell = s_lo[b] + yy[b];
                            on = on && cell >= 0 && cell < g.N[a.bdim[b]];
                            bF += (on ? cell : 0) * a.bstrideF[b];
                        }
                    }
                    float4 r[TILE_MAXT];
#pragma unroll
                    for (int gg = 0; gg < TILE_MAXT; ++gg) r[gg] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    auto apply = [&](int ii, const float4 &pa) {
#pragma unroll
                        for (int gg = 0; gg < TILE_MAXT; ++gg) {
                            const int j = ii - (s_owo[gg] - owlo);
                            if (gg < Tt && j >= 0 && j < Wow) {
                                const float w = s_oww[gg * 16 + j];
                                fma4<AMY_FFMA2_T1 != 0>(w, pa, r[gg]);
                            }
                        }
                    };
                    auto cell_off = [&](int ii) {
                        int32_t cc = owlo + ii;
                        if (a.ow < 0) return 0;
                        cc = min(max(cc, 0), g.N[a.ow] - 1);
                        return cc * a.owstrideF * Ppad;
                    };
                    if (on) {
                        const VT *vb = a.Vpn + (int64_t)bF * Ppad + 4 * s1q;
                        int ii = 0;
                        for (; ii + 2 <= own; ii += 2) {
                            const VT *v0 = vb + cell_off(ii), *v1 = vb + cell_off(ii + 1);
                            float4 p0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), p1 = p0;
                            int k = 0;
                            for (; k + TILE_KU <= a.Ksh; k += TILE_KU) {
                                float4 va[TILE_KU], vc[TILE_KU];
#pragma unroll
                                for (int kk = 0; kk < TILE_KU; ++kk) {
                                    const int32_t o = s_sho[k + kk];
                                    va[kk] = vload4<VT>(v0 + o);
                                    vc[kk] = vload4<VT>(v1 + o);
                                }
#pragma unroll
                                for (int kk = 0; kk < TILE_KU; ++kk) {
                                    const float w = s_shw[k + kk];
                                    fma4<AMY_FFMA2_T1 != 0>(w, va[kk], p0);
                                    fma4<AMY_FFMA2_T1 != 0>(w, vc[kk], p1);
                                }
                            }
                            for (; k < a.Ksh; ++k) {
                                const int32_t o = s_sho[k];
                                const float w = s_shw[k];
                                const float4 va = vload4<VT>(v0 + o), vc = vload4<VT>(v1 + o);
                                fma4<AMY_FFMA2_T1 != 0>(w, va, p0);
                                fma4<AMY_FFMA2_T1 != 0>(w, vc, p1);
                            }
                            apply(ii, p0);
                            apply(ii + 1, p1);
                        }
                        if (ii < own) {
                            const VT *v0 = vb + cell_off(ii);
                            float4 p0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                            int k = 0;
                            for (; k + TILE_KU <= a.Ksh; k += TILE_KU) {
                                float4 va[TILE_KU];
#pragma unroll
                                for (int kk = 0; kk < TILE_KU; ++kk) va[kk] = vload4<VT>(v0 + s_sho[k + kk]);
#pragma unroll
                                for (int kk = 0; kk < TILE_KU; ++kk) {
                                    const float w = s_shw[k + kk];
                                    fma4<AMY_FFMA2_T1 != 0>(w, va[kk], p0);
                                }
                            }
                            for (; k < a.Ksh; ++k) {
                                const float w = s_shw[k];
                                fma4<AMY_FFMA2_T1 != 0>(w, vload4<VT>(v0 + s_sho[k]), p0);
                            }
                            apply(ii, p0);
                        }
                        if (a.work) n_vld += 4u * (uint32_t)a.Ksh * (uint32_t)own;
                    }
#pragma unroll
                    for (int gg = 0; gg < TILE_MAXT; ++gg)
                        if (gg < Tt)
                            *reinterpret_cast<float4 *>(s_R + ((int64_t)gg * a.rent + er) * Rp + 4 * s1q) = r[gg];
                }
                __syncthreads();
                // ---- stage 2: every free state's B rows that fall in the chunk
#pragma unroll 1
                for (int i = 0; i < TILE_MAXT; ++i) {
                    if (!(freebits & (1u << i))) continue;
                    const int s = tid + i * NT;
                    const int gg = s / P, p = s - gg * P;
                    int32_t eB[PLANE_MAXB];
#pragma unroll
                    for (int b = 0; b < PLANE_MAXB; ++b) eB[b] = b < nB ? tab_index(a.bdim[b], gg, p) : 0;
                    float acc = s_acc[i * NT + tid], comp = s_cmp[i * NT + tid];
                    plane_stage2<WM>(g, a.tab, up, nB, a.bdim, eB, tab_index(n - 2, gg, p), tab_index(n - 1, gg, p),
                                     s_lo, s_R + (int64_t)gg * a.rent * Rp, a.rs0, rs1, a.chunk, c, Rp, a.kahan,
                                     acc, comp, n_rld, n_rows, a.work != nullptr);
                    s_acc[i * NT + tid] = acc;
                    s_cmp[i * NT + tid] = comp;
                }
                __syncthreads();
            }
#pragma unroll
            for (int i = 0; i < TILE_MAXT; ++i) {
                if ((freebits & (1u << i)) && s_acc[i * NT + tid] > s_best[i * NT + tid]) {
                    s_best[i * NT + tid] = s_acc[i * NT + tid];
                    s_arg[i * NT + tid] = u;
                }
            }
        }
        if (tid < PLANE_MAXB) {
            s_lo[tid] = INT_MAX;
            s_hi[tid] = INT_MIN;
        }
        if (tid == 0) s_any[0] = 0;
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
#pragma unroll
    for (int i = 0; i < TILE_MAXT; ++i) {
        if (!(livebits & (1u << i))) continue;
        const int s = tid + i * NT;
        const int gg = s / P, p = s - gg * P;
        const int64_t gp = gplane0 + gg * astrideF;
        const int64_t x = gp * P + p;
        float v = s_best[i * NT + tid];
        uint16_t pol = (uint16_t)s_arg[i * NT + tid];
        if (!(freebits & (1u << i))) {
            const uint8_t f = a.mask[x];
            v = (a.spec_kind != SPEC_SAFETY && (f & F_TARGET)) ? 1.0f : 0.0f;
            pol = 0xFFFF;
        }
        const VT vb = vstore_cast<VT, float>(v);
        a.Vo[x] = vb;
        a.Vpo[gp * Ppad + p] = vb;
        if (a.Vfinal) a.Vfinal[x] = v;
        if (a.pi) a.pi[x] = pol;
    }
}

}  // namespace amy
