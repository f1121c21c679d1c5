// amy_fast.cuh -- register-resident fused backup + max/argmax (Algorithm 4)
// for windows whose per-dimension width is at most WM (3, 5 or 8), FP32
// arithmetic, rows on the fly (Sec. 6.1), stored per pair, or tabulated per
// dimension over the coordinates each mean component depends on.
//
// Thread mapping: a block owns TX consecutive states; thread tid handles
// state xl = tid % TX and the inputs u = c, c + UL, ... with c = tid / TX
// (UL = 256 / TX input lanes).  Lanes of a warp are consecutive states, so V
// windows and stored rows are read coalesced.  Each thread keeps the two
// innermost window dims (masses and cell offsets) in registers and walks the
// outer dims with an odometer whose per-thread state lives in shared memory
// ([slot][thread] layout, conflict free).  The max and the lowest maximising
// input are kept in registers per lane and merged across lanes at the end.
#pragma once

#include <climits>

#include "amy_kernels.cuh"

namespace amy {

constexpr int FAST_THREADS = 256;
enum FastVariant : int { VAR_GENERAL = 0, VAR_EXACT = 1, VAR_EXACT_CONTIG = 2 };

template <class VT> struct FastArgs {
    const VT *Vn;        // V_{k+1}
    VT *Vo;              // V_k
    float *Vfinal;       // optional FP32 copy of V_k
    uint16_t *pi;        // optional policy of this step
    const uint8_t *mask;
    int32_t spec_kind;
    int32_t tileX;       // states per block
    int32_t ulanes;      // input lanes per state (tileX * ulanes == 256)
    int32_t rowtile;     // staged kernel: innermost-dim rows per tile (0 = consecutive states)
    int32_t grouped;     // staged kernel: inputs come in runs sharing their outer-dim records
    int32_t box_floats;  // staged kernel: shared-memory box budget (floats)
    int32_t stage_tab;   // staged kernel: words of the innermost dim's table to stage (0 = none)
    int32_t stage_recs;  // per-run kernel: records of the innermost dim's table (staged as weights)
    int32_t runs_planes; // per-run kernel: 16-byte planes allocated per sliding entry (1 or 2)
    uint32_t tx_magic;   // per-run kernel: ceil(2^32 / tileX), so tid / tileX = umulhi(tid, tx_magic)
    int32_t chu_shift;   // per-run kernel: log2 of the 32-lane chunks per innermost row
    int32_t outer;       // per-run kernel, 3-D: values of dim 0 per row tile (rowtile rows of dim 1 each)
    // per-run kernel, from the host when known (else read or derived on the device):
    int32_t bnd_known;   // 1: bnd_lo / bnd_hi hold the tables' (origin - own coordinate) bounds
    int32_t bnd_lo[3], bnd_hi[3];
    int32_t nrs;         // > 0: the input runs (at most 64) start at rs[0 .. nrs - 1], rs[nrs] = inputs
    int32_t in_stride_b; // byte step between the inner records of consecutive inputs of a run
                         // (INT_MIN: not constant)
    uint16_t rs[66];
    int32_t kahan;       // compensated accumulation over window rows
    const float *T;      // per-pair masses [sum W][pairs] (stored factored)
    const int16_t *O;    // per-pair origins [n][pairs]
    int64_t npairs;
    const uint32_t *tab; // per-dimension tables (separable)
};

// Shared-memory bytes of one block for n state dims and width bound WM.
__host__ __device__ inline size_t fast_smem_bytes(int n, int WM) {
    const int DO = n > 2 ? n - 2 : 0;
    const int DH = DO > 1 ? DO - 1 : 0;
    return (size_t)(2 * DH * WM + 3 * DH + 2) * FAST_THREADS * 4;
}

// Masses and offsets of one dim into fixed-size register arrays (FP32 path;
// same arithmetic as dim_masses_f32; xd: the state's centre in dim d, used by
// multiplicative noise).
template <int WM>
__device__ __forceinline__ void dim_masses_reg(const Geom &g, int d, double mu, int32_t o, int W, double xd,
                                               float (&fac)[WM], int32_t (&off)[WM]) {
    // W: this dim's window width (a compile-time constant when all widths equal WM)
    const int kmax = kept_upper(g, d, mu, o);
    const double c0 = state_centre(g, d, o);
    const float e0 = (float)dsub(dsub(c0, dmul(0.5, g.eta[d])), mu);
    const float etaf = (float)g.eta[d];
    const bool gauss = g.noise == NOISE_GAUSSIAN || g.noise == NOISE_MULT_GAUSSIAN;
    const float r = gauss_r_f32(g, d, xd);
    float dlo = e0;
    float tlo = gauss ? 0.5f * erfcf(fabsf(dlo) * r) : 0.0f;
#pragma unroll
    for (int k = 0; k < WM; ++k) {
        if (k < W) {
            const float dhi = fmaf((float)(k + 1), etaf, e0);
            const float thi = gauss ? 0.5f * erfcf(fabsf(dhi) * r) : 0.0f;
            const float mass = gauss ? gauss_cell_f32(dlo, dhi, tlo, thi, r) : noise_mass<float>(g, d, dlo, dhi);
            bool on;
            const int32_t cell = cell_of(g, d, o + k, on);
            fac[k] = (on && k < kmax) ? fmaxf(mass, 0.0f) : 0.0f;
            off[k] = cell * g.stride[d];
            dlo = dhi;
            tlo = thi;
        } else {
            fac[k] = 0.0f;
            off[k] = 0;
        }
    }
}

// Cell offsets of a window starting at slot o: clamped on a bounded dim
// (the clamped slots carry zero mass), wrapped on a periodic one (a single
// modulo per dim, then at most one subtraction per slot since W <= N).
template <int WM>
__device__ __forceinline__ void dim_offsets_reg(const Geom &g, int d, int32_t o, int W, int32_t (&off)[WM]) {
    const int32_t N = g.N[d], st = g.stride[d];
    if ((g.periodic >> d) & 1u) {
        int32_t w = o % N;
        w = w < 0 ? w + N : w;
#pragma unroll
        for (int k = 0; k < WM; ++k) {
            int32_t c = w + k;
            c = c >= N ? c - N : c;
            off[k] = (k < W) ? c * st : 0;
        }
    } else {
#pragma unroll
        for (int k = 0; k < WM; ++k) {
            const int32_t c = min(max(o + k, 0), N - 1);
            off[k] = (k < W) ? c * st : 0;
        }
    }
}

// Adds one window row's contribution with explicit rounding (no contraction
// into a fused multiply-add), plainly or Kahan-compensated, so that every
// kernel variant sums in exactly the same arithmetic.
__device__ __forceinline__ void accum_row(float &acc, float &comp, float term, int kahan) {
    if (kahan) {
        const float y = __fsub_rn(term, comp);
        const float t = __fadd_rn(acc, y);
        comp = __fsub_rn(__fsub_rn(t, acc), y);
        acc = t;
    } else {
        acc = __fadd_rn(acc, term);
    }
}

// Entry k of a register array (k runtime): a select chain, no local memory.
template <int WM, class T>
__device__ __forceinline__ T sel_reg(const T (&arr)[WM], int k) {
    T v = arr[0];
#pragma unroll
    for (int j = 1; j < WM; ++j)
        if (k == j) v = arr[j];
    return v;
}

// Sum over the two innermost window dims: sum_j tA[j] * sum_k tB[k] * V[b + oA[j] + oB[k]].
template <class VT, int WM>
__device__ __forceinline__ float inner_block(const VT *__restrict__ V, int32_t b, const float (&tA)[WM],
                                             const int32_t (&oA)[WM], int WA, const float (&tB)[WM],
                                             const int32_t (&oB)[WM], int WB) {
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < WM; ++j) {
        if (j < WA) {
            const VT *p = V + (b + oA[j]);
            float r = 0.0f;
#pragma unroll
            for (int k = 0; k < WM; ++k)
                if (k < WB) r = fmaf(tB[k], vload<float, VT>(p + oB[k]), r);
            s = fmaf(tA[j], r, s);
        }
    }
    return s;
}

// One tile (tileX states, all inputs) of the fused backup; x is the state of
// this thread's lane column (xl = tid % tileX), any value >= nx when the
// column is idle.
// Kernel variants: VAR_GENERAL (widths up to WM), VAR_EXACT (every width
// equals WM, so all width guards fold away), VAR_EXACT_CONTIG (also a bounded
// innermost dim: its window row is read unclamped -- off-grid slots have zero
// mass and the V buffers carry kVGuard finite guard cells on each side -- so
// one base address plus immediate offsets reads the whole row).
// g may live in kernel parameters or in shared memory (batched kernel).
template <class VT, int WM, int TM, int VAR>
__device__ __forceinline__ void backup_tile(const Geom &g, const FastArgs<VT> &a, int32_t x,
                                            unsigned char *smem_raw) {
    constexpr bool EXACT = VAR >= VAR_EXACT;
    constexpr bool CONTIG = VAR == VAR_EXACT_CONTIG;
    constexpr int BT = FAST_THREADS;
    const int tid = threadIdx.x;
    const int TX = a.tileX, UL = a.ulanes;
    const int xl = tid % TX;
    const int c = tid / TX;
    const int n = g.n;
    const int DO = n > 2 ? n - 2 : 0;   // outer dims walked by the odometer
    const int DH = DO > 1 ? DO - 1 : 0; // outer dims above the last outer one
    float *sF = reinterpret_cast<float *>(smem_raw);
    int32_t *sO = reinterpret_cast<int32_t *>(sF + DH * WM * BT);
    int32_t *sK = sO + DH * WM * BT;
    float *sP = reinterpret_cast<float *>(sK + DH * BT);
    int32_t *sB = reinterpret_cast<int32_t *>(sP + DH * BT);
    float *cBest = reinterpret_cast<float *>(sB + DH * BT);
    int32_t *cArg = reinterpret_cast<int32_t *>(cBest + blockDim.x);  // one entry per thread

    float best = -1.0f;
    int32_t arg = 0x7fffffff;
    const bool active = x >= 0 && x < g.nx;
    const uint8_t f = active ? a.mask[x] : (uint8_t)0;
    const bool masked = active && state_masked(a.spec_kind, f);
    if (active && !masked) {
        int32_t xi[MAXD];
        decode_state(g, x, xi);
        double xc[MAXD];
        int32_t es[MAXD];
#pragma unroll
        for (int d = 0; d < MAXD; ++d) {
            xc[d] = 0.0;
            es[d] = 0;
            if (d < n) {
                if (TM == TM_OTF) xc[d] = state_centre(g, d, xi[d]);
                if (TM == TM_SEPARABLE) {
                    int32_t e = 0;
#pragma unroll
                    for (int j = 0; j < MAXD; ++j)
                        if (j < n) e += xi[j] * g.tsx[d][j];
                    es[d] = e;
                }
            }
        }
        double cth = 0.0, sth = 0.0;
        if (TM == TM_OTF && g.sys == SYS_UNICYCLE) {
            cth = cos(xc[2]);
            sth = sin(xc[2]);
        }
        // Inputs of this lane: u = c, c + UL, ...; with a disturbance grid
        // (nw points per input, pair index u * nw + w) the lane takes whole
        // blocks of nw pairs and keeps the min over each block (the
        // adversary's move of the max-min game) before the max over inputs.
        const int NW = g.nw;
        int wk = 0;
        float mn = 0.0f;
        for (int u = c * NW; u < g.nu; ++u) {
            float tA[WM], tB[WM], tL[WM];
            int32_t oA[WM], oB[WM], oL[WM];
#pragma unroll
            for (int k = 0; k < WM; ++k) {
                tA[k] = (k == 0) ? 1.0f : 0.0f;
                oA[k] = 0;
                tB[k] = 0.0f;
                oB[k] = 0;
                tL[k] = 0.0f;
                oL[k] = 0;
            }
            int WA = EXACT ? WM : 1, WB = EXACT ? WM : 1;
            double mu[MAXD];
            int32_t ui[MAXD];
            if (TM == TM_OTF) {
                if (g.sys == SYS_AFFINE) {
                    const double *A = g.params + (int64_t)u * (n * n + n);
                    const double *cc = A + n * n;
#pragma unroll
                    for (int i = 0; i < MAXD; ++i) {
                        mu[i] = 0.0;
                        if (i < n) {
                            double acc = 0.0;
#pragma unroll
                            for (int j = 0; j < MAXD; ++j)
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
#pragma unroll
                    for (int i = 3; i < MAXD; ++i) mu[i] = 0.0;
                }
            }
            if (TM == TM_SEPARABLE) {
                // input part of every dim's table index (precomputed per input)
                const int4 *up = reinterpret_cast<const int4 *>(a.tab + g.uoff + (int64_t)u * g.urw);
#pragma unroll
                for (int q = 0; q < MAXD / 4; ++q) {
                    int4 v = make_int4(0, 0, 0, 0);
                    if (q * 4 < n) v = __ldg(up + q);
                    ui[q * 4 + 0] = v.x;
                    ui[q * 4 + 1] = v.y;
                    ui[q * 4 + 2] = v.z;
                    ui[q * 4 + 3] = v.w;
                }
            }
            const int64_t pair = (int64_t)u * g.nx + x;
            int fb = 0;
#pragma unroll
            for (int d = 0; d < MAXD; ++d) {
                if (d < n) {
                    const int Wd = EXACT ? WM : g.W[d];
                    float fk[WM];
                    int32_t ok[WM];
                    int32_t od = 0;  // window origin of this dim
                    if (TM == TM_OTF) {
                        od = origin_of(g, d, mu[d]);
                        dim_masses_reg<WM>(g, d, mu[d], od, Wd, xc[d], fk, ok);
                    } else if (TM == TM_SEPARABLE) {
                        const int32_t e = es[d] + ui[d];
                        const uint4 *rec = reinterpret_cast<const uint4 *>(a.tab + g.toff[d] + (int64_t)e * g.trw[d]);
                        constexpr int NQ = (WM + 1 + 3) / 4;
                        uint32_t wds[NQ * 4];
#pragma unroll
                        for (int q = 0; q < NQ; ++q) {
                            uint4 v = make_uint4(0u, 0u, 0u, 0u);
                            if (q * 4 < Wd + 1) v = __ldg(rec + q);
                            wds[q * 4 + 0] = v.x;
                            wds[q * 4 + 1] = v.y;
                            wds[q * 4 + 2] = v.z;
                            wds[q * 4 + 3] = v.w;
                        }
                        // origin at word 0, masses at words 1..Wd
#pragma unroll
                        for (int k = 0; k < WM; ++k) fk[k] = (k < Wd) ? __uint_as_float(wds[1 + k]) : 0.0f;
                        od = (int32_t)wds[0];
                        dim_offsets_reg<WM>(g, d, od, Wd, ok);
                    } else {  // TM_FACTORED
                        od = __ldg(a.O + d * a.npairs + pair);
#pragma unroll
                        for (int k = 0; k < WM; ++k)
                            fk[k] = (k < Wd) ? __ldg(a.T + (int64_t)(fb + k) * a.npairs + pair) : 0.0f;
                        dim_offsets_reg<WM>(g, d, od, Wd, ok);
                    }
                    if (CONTIG && d == n - 1) {
                        // bounded innermost dim (stride 1): unclamped, contiguous row
#pragma unroll
                        for (int k = 0; k < WM; ++k) ok[k] = od + k;
                    }
                    fb += Wd;
                    if (d < n - 3) {
#pragma unroll
                        for (int k = 0; k < WM; ++k) {
                            if (k < Wd) {
                                sF[(d * WM + k) * BT + tid] = fk[k];
                                sO[(d * WM + k) * BT + tid] = ok[k];
                            }
                        }
                    } else if (d == n - 3) {
#pragma unroll
                        for (int k = 0; k < WM; ++k) {
                            tL[k] = fk[k];
                            oL[k] = ok[k];
                        }
                    } else if (d == n - 2) {
#pragma unroll
                        for (int k = 0; k < WM; ++k) {
                            tA[k] = fk[k];
                            oA[k] = ok[k];
                        }
                        if (!EXACT) WA = Wd;
                    } else {
#pragma unroll
                        for (int k = 0; k < WM; ++k) {
                            tB[k] = fk[k];
                            oB[k] = ok[k];
                        }
                        if (!EXACT) WB = Wd;
                    }
                }
            }
            // window sum: odometer over the outer dims, inner 2-D block in registers
            float s;
            if (DO == 0) {
                s = inner_block<VT, WM>(a.Vn, 0, tA, oA, WA, tB, oB, WB);
            } else {
                float acc = 0.0f, comp = 0.0f;
                // higher levels 0..DO-2 keep (k, prefix product, prefix offset) in shared memory
                for (int e = 0; e < DH; ++e) {
                    sK[e * BT + tid] = 0;
                    const float pe = __fmul_rn(e > 0 ? sP[(e - 1) * BT + tid] : 1.0f, sF[(e * WM) * BT + tid]);
                    const int32_t be = (e > 0 ? sB[(e - 1) * BT + tid] : 0) + sO[(e * WM) * BT + tid];
                    sP[e * BT + tid] = pe;
                    sB[e * BT + tid] = be;
                }
                const int L = DO - 1;  // last outer level, looped in registers
                const int WL = EXACT ? WM : g.W[L];
                while (true) {
                    const float pw = DH > 0 ? sP[(DH - 1) * BT + tid] : 1.0f;
                    const int32_t pb = DH > 0 ? sB[(DH - 1) * BT + tid] : 0;
                    if (pw != 0.0f) {
                        if constexpr (WM <= 5) {
                            // last outer level unrolled without branches so that all
                            // WM^3 window loads of this row group can be in flight
                            // (dropped slots have zero mass and a valid offset)
#pragma unroll
                            for (int k = 0; k < WM; ++k) {
                                if (k < WL) {
                                    const float w = __fmul_rn(pw, tL[k]);
                                    const float term = __fmul_rn(w, inner_block<VT, WM>(
                                                                          a.Vn, pb + oL[k], tA, oA, WA, tB, oB, WB));
                                    accum_row(acc, comp, term, a.kahan);
                                }
                            }
                        } else {
                            for (int k = 0; k < WL; ++k) {
                                const float w = __fmul_rn(pw, sel_reg<WM>(tL, k));
                                if (w != 0.0f) {
                                    const float term = __fmul_rn(w, inner_block<VT, WM>(
                                                                          a.Vn, pb + sel_reg<WM>(oL, k), tA, oA, WA, tB, oB, WB));
                                    accum_row(acc, comp, term, a.kahan);
                                }
                            }
                        }
                    }
                    int e = DH - 1;
                    while (e >= 0) {
                        const int ke = sK[e * BT + tid] + 1;
                        if (ke < (EXACT ? WM : g.W[e])) {
                            sK[e * BT + tid] = ke;
                            break;
                        }
                        sK[e * BT + tid] = 0;
                        --e;
                    }
                    if (e < 0) break;
                    for (int q = e; q < DH; ++q) {
                        const int kq = sK[q * BT + tid];
                        sP[q * BT + tid] = __fmul_rn(q > 0 ? sP[(q - 1) * BT + tid] : 1.0f, sF[(q * WM + kq) * BT + tid]);
                        sB[q * BT + tid] = (q > 0 ? sB[(q - 1) * BT + tid] : 0) + sO[(q * WM + kq) * BT + tid];
                    }
                }
                s = acc;
            }
            if (NW == 1) {
                if (s > best) {
                    best = s;
                    arg = u;
                }
                u += UL - 1;
            } else {
                mn = wk == 0 ? s : fminf(mn, s);
                if (wk == NW - 1) {
                    if (mn > best) {
                        best = mn;
                        arg = u / NW;
                    }
                    wk = 0;
                    u += (UL - 1) * NW;
                } else {
                    ++wk;
                }
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

template <class VT, int WM, int TM, int VAR>
__global__ void __launch_bounds__(FAST_THREADS) k_backup_fast(const __grid_constant__ Geom g,
                                                              const FastArgs<VT> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int64_t x = (int64_t)blockIdx.x * a.tileX + threadIdx.x % a.tileX;
    backup_tile<VT, WM, TM, VAR>(g, a, (int32_t)min(x, (int64_t)INT_MAX), smem_raw);
}

// Per-dimension table construction (separable stored mode): record e of
// table d holds the window origin and masses of mean component d evaluated at
// the state/input coordinates encoded in e (all other coordinates 0, which
// mean component d does not depend on).
static __global__ void k_build_sep(const __grid_constant__ Geom g, uint32_t *__restrict__ tab, int64_t total) {
    float fac[MAXWS];
    int32_t off[MAXWS];
    // origin bounds gathered per block in shared memory, then one global
    // atomic per dim and block
    __shared__ int32_t s_lo[MAXD], s_hi[MAXD];
    if (threadIdx.x < MAXD) {
        s_lo[threadIdx.x] = INT_MAX;
        s_hi[threadIdx.x] = INT_MIN;
    }
    __syncthreads();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int d = 0;
        int64_t e = t;
        while (d < g.n - 1 && e >= g.tent[d]) {
            e -= g.tent[d];
            ++d;
        }
        // decode e into state and input coordinates (strides of table d)
        int32_t x = 0, u = 0;
        int64_t r = e;
        // input coordinates are the fastest in the table index
        for (int i = g.m - 1; i >= 0; --i) {
            if (g.tsu[d][i] == 0) continue;
            const int32_t U = g.ucount[i];
            const int32_t ui = (int32_t)((r / g.tsu[d][i]) % U);
            int32_t s = 1;
            for (int q = i + 1; q < g.m; ++q) s *= g.ucount[q];
            u += ui * s;
        }
        for (int j = 0; j < g.n; ++j) {
            if (g.tsx[d][j] == 0) continue;
            const int32_t xj = (int32_t)((r / g.tsx[d][j]) % g.N[j]);
            x += xj * g.stride[j];
        }
        const double mud = mean_component(g, x, u, d);
        const int32_t o = origin_of(g, d, mud);
        dim_masses_f32(g, d, mud, o, noise_centre(g, x, d), fac, off);
        uint32_t *rec = tab + g.toff[d] + e * g.trw[d];
        const int Wd = g.W[d];
        rec[0] = (uint32_t)o;
        for (int k = 0; k < Wd; ++k) rec[1 + k] = __float_as_uint(fac[k]);
        for (int k = 1 + Wd; k < g.trw[d]; ++k) rec[k] = 0u;
        // origin bounds relative to the state's own coordinate d
        if (g.tsx[d][d] != 0) {
            const int32_t xd = (int32_t)((e / g.tsx[d][d]) % g.N[d]);
            atomicMin(&s_lo[d], o - xd);
            atomicMax(&s_hi[d], o - xd);
        }
    }
    __syncthreads();
    if (threadIdx.x < MAXD && s_lo[threadIdx.x] != INT_MAX) {
        int32_t *b = reinterpret_cast<int32_t *>(tab + g.boff);
        atomicMin(b + threadIdx.x, s_lo[threadIdx.x]);
        atomicMax(b + MAXD + threadIdx.x, s_hi[threadIdx.x]);
    }
}

// Shifted-weight copy of the innermost dim's table (Geom::shoff), once the
// table and its bounds are built: record e gets its masses at the slots they
// occupy among the K = W + (largest - smallest origin offset) slots that
// start at own coordinate + smallest offset.
static __global__ void k_build_shift(const __grid_constant__ Geom g, uint32_t *__restrict__ tab) {
    const int L = g.n - 1;
    const int32_t e = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (e >= g.tent[L]) return;
    const int32_t *b = reinterpret_cast<const int32_t *>(tab + g.boff);
    const uint32_t *rec = tab + g.toff[L] + (int64_t)e * g.trw[L];
    const int32_t own = (e / g.tsx[L][L]) % g.N[L];
    const int32_t sh = (int32_t)rec[0] - own - b[L];
    const int Wd = g.W[L];
    float w[8];
    for (int k = 0; k < 8; ++k) {
        const int32_t j = k - sh;
        w[k] = (sh >= 0 && sh + Wd <= 8 && j >= 0 && j < Wd) ? __uint_as_float(rec[1 + j]) : 0.0f;
    }
    float4 *out = reinterpret_cast<float4 *>(tab + g.shoff);
    out[e] = make_float4(w[0], w[1], w[2], w[3]);
    out[g.tent[L] + e] = make_float4(w[4], w[5], w[6], w[7]);
}

static __global__ void k_build_sep_bounds_init(const __grid_constant__ Geom g, uint32_t *__restrict__ tab) {
    int32_t *b = reinterpret_cast<int32_t *>(tab + g.boff);
    const int d = threadIdx.x;
    if (d < MAXD) {
        b[d] = INT_MAX;
        b[MAXD + d] = INT_MIN;
        b[2 * MAXD + 4 + d] = 0;  // plane spreads (k_plane_spread)
    }
    if (d == 0) {
        int32_t m = 0;
        for (int q = 0; q < g.n; ++q)
            if (g.tsx[q][q] != 0) m |= 1 << q;
        b[2 * MAXD] = m;
    }
}

}  // namespace amy
