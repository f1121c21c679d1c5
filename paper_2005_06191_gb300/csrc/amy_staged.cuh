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

#include "amy_fast.cuh"

namespace amy {

constexpr int STAGE_BOX_FLOATS = 6144;  // 24 KiB staging box per block

__host__ __device__ inline size_t staged_smem_bytes(int n, int WM) {
    return (size_t)STAGE_BOX_FLOATS * 4 + fast_smem_bytes(n, WM);
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

template <class VT, int WM, int TM, int NS>
__global__ void __launch_bounds__(FAST_THREADS) k_backup_staged(const __grid_constant__ Geom g,
                                                                const FastArgs<VT> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int BT = FAST_THREADS;
    float *sbox = reinterpret_cast<float *>(smem_raw);
    unsigned char *work = smem_raw + (size_t)STAGE_BOX_FLOATS * 4;  // also the fallback's area
    float *cBest = reinterpret_cast<float *>(work);
    int32_t *cArg = reinterpret_cast<int32_t *>(cBest + BT);
    __shared__ int32_t s_lo[3], s_hi[3];

    const int tid = threadIdx.x;
    const int TX = a.tileX, UL = a.ulanes;
    const int xl = tid % TX;
    const int c = tid / TX;
    const int32_t x = (int32_t)blockIdx.x * TX + xl;
    if (tid < 3) {
        s_lo[tid] = INT_MAX;
        s_hi[tid] = INT_MIN;
    }
    const bool active = x < g.nx;
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
                    dim_masses_reg<WM>(g, d, mu[d], o[d], WM, t[d], ok);
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
    if (work_items) {
#pragma unroll
        for (int d = 0; d < NS; ++d) {
            atomicMin(&s_lo[d], lo[d]);
            atomicMax(&s_hi[d], hi[d]);
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
    if (vol > STAGE_BOX_FLOATS) {
        // this tile's windows spread too far: the register-resident body
        backup_tile<VT, WM, TM, VAR_EXACT>(g, a, blockIdx.x, work);
        return;
    }
    {
        // row stride padded to a multiple of 32 floats when it fits: lanes whose
        // windows differ by whole rows then still hit distinct banks
        int32_t inner = bn[NS - 1];
        const int32_t padded = (inner + 31) / 32 * 32;
        if (NS > 1 && (vol / inner) * padded <= STAGE_BOX_FLOATS) inner = padded;
        int32_t s = 1;
#pragma unroll
        for (int d = NS - 1; d >= 0; --d) {
            bs[d] = s;
            s *= (d == NS - 1) ? inner : bn[d];
        }
    }
    // stage the box: periodic dims wrap, off-grid cells hold 0 (zero mass there)
    if (any) {
        for (int32_t i = tid; i < (int32_t)vol; i += BT) {
            int64_t lin = 0;
            int32_t sidx = 0;
            bool on = true;
            int32_t r = i;
#pragma unroll
            for (int d = NS - 1; d >= 0; --d) {
                const int32_t kd = r % bn[d];
                r /= bn[d];
                bool ond;
                const int32_t cell = cell_of(g, d, blo[d] + kd, ond);
                on = on && ond;
                lin += (int64_t)cell * g.stride[d];
                sidx += kd * bs[d];
            }
            sbox[sidx] = on ? vload<float, VT>(a.Vn + lin) : 0.0f;
        }
    }
    __syncthreads();

    // pass 2: window sums from the box (summation order of amy_fast.cuh)
    float best = -1.0f;
    int32_t arg = 0x7fffffff;
    if (work_items) {
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
