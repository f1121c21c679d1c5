// amy_core.cuh -- device-side problem geometry and the per-(x,u) row setup of
// the AMYTISS abstraction (arxiv 2005.06191), shared by every kernel of the
// engine.  Host code fills a Geom once per problem; kernels take it by value.
//
// What a row is (Algorithm 1 / Algorithm 2): for a state x and an input u the
// mean mu = f(centre(x), centre(u)) (Eq. 4), the cutting window of Sec. 5.2
// (Remark on constructing the cutting region) and, per dimension, the Gaussian
// mass of each window cell; for a diagonal covariance the row entry is the
// product of the per-dimension masses.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace amy {

constexpr int MAXD = 8;
constexpr int MAX_BOXES = 16;
constexpr int MAXWS = 160;  // largest sum of window widths a kernel keeps per row

enum WindowMode : int32_t { WM_DENSE = 0, WM_GAMMA = 1, WM_EXPLICIT = 2 };
enum SysKind : int32_t { SYS_AFFINE = 0, SYS_UNICYCLE = 1 };
enum SpecKind : int32_t { SPEC_SAFETY = 0, SPEC_REACH = 1, SPEC_REACH_AVOID = 2 };
enum TMode : int32_t { TM_OTF = 0, TM_FULL = 1, TM_FACTORED = 2, TM_SEPARABLE = 3 };

// 16-bit fixed-point storage of a probability: value = bits / 65535.
struct unorm16 {
    uint16_t bits;
};

// Per-state flag bits written by the spec-mask kernel.
constexpr uint8_t F_TARGET = 1, F_AVOID = 2, F_SAFE = 4;

struct Geom {
    int32_t n, m;
    int32_t nx, nu;              // states (< 2^31) and inputs: (input, disturbance) pairs
    int32_t nw;                  // disturbance points per input (1: no disturbance); the
                                 // pair index is u * nw + w, so nu / nw control inputs
    int32_t N[MAXD];             // points per state dim
    int32_t stride[MAXD];        // C-order strides of the state index
    double lb[MAXD], eta[MAXD];
    uint32_t periodic;           // bit d set: dim d wraps
    int32_t W[MAXD];             // window width per dim
    int32_t wsum, wtot;          // sum and product of W
    int32_t wmode;               // WindowMode
    double xs[MAXD];             // gamma-mode cut half width
    double k2[MAXD];             // sigma*sqrt(2)
    float rk2f[MAXD];            // 1/(sigma*sqrt(2)) in FP32
    int32_t sys;                 // SysKind
    int32_t ucount[MAXD];
    double ulb[MAXD], ueta[MAXD];
    const double *params;        // device copy of the system parameters
    // Dependency-compressed per-dimension tables (separable stored mode):
    // mean component d depends only on the state dims j with tsx[d][j] != 0
    // and the input dims i with tsu[d][i] != 0, so its window origin and
    // masses are tabulated over those coordinates.  Record e of table d sits
    // at word toff[d] + e*trw[d]: the window origin (int32) then the W[d]
    // masses (FP32), padded to a multiple of 4 words.
    // The input part of every table index, sum_i u_i * tsu[d][i], is stored
    // per input u at word uoff + u*urw (one int32 per dim).
    int32_t tsx[MAXD][MAXD];
    int32_t tsu[MAXD][MAXD];
    int64_t toff[MAXD];
    int32_t trw[MAXD];
    int32_t tent[MAXD];
    int64_t uoff;
    int32_t urw;
    // After the index parts, at word boff: per dim d the smallest and largest
    // window origin minus the state's own coordinate d over the table
    // (words boff + d and boff + MAXD + d), then a bit mask of the dims for
    // which that bound exists (component d depends on coordinate d), three
    // spare words, and per dim d < n - 2 the largest spread (max - min) of
    // its window origin over one plane of the two innermost dims (words
    // boff + 2 * MAXD + 4 + d; 0 when component d ignores those coordinates).
    int64_t boff;
    // After the bounds block, at word shoff (0 = absent; 2-D and 3-D problems
    // whose innermost table has at most 4096 records): that table as shifted
    // weights, 8 floats per record (two planes of 4 at shoff and
    // shoff + 4 * tent[n - 1]): record e holds its W masses at positions
    // sh .. sh + W - 1, sh = origin - own coordinate - the smallest such
    // offset over the table, and zeros elsewhere (all zeros when sh > 7 - W + 1).
    int64_t shoff;
};

struct SpecDev {
    int32_t kind;
    int32_t n_target, n_avoid, has_safe;
    double safe_lb[MAXD], safe_ub[MAXD];
    double t_lb[MAX_BOXES][MAXD], t_ub[MAX_BOXES][MAXD];
    double a_lb[MAX_BOXES][MAXD], a_ub[MAX_BOXES][MAXD];
};

// FP64 helpers with explicit rounding: no multiply-add is ever fused, so the
// mean and the window origin reproduce the documented FP64 expression order.
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }

__device__ __forceinline__ void decode_state(const Geom &g, int32_t x, int32_t *idx) {
    uint32_t r = (uint32_t)x;
#pragma unroll
    for (int d = MAXD - 1; d >= 0; --d) {
        if (d < g.n) {
            uint32_t N = (uint32_t)g.N[d];
            idx[d] = (int32_t)(r % N);
            r /= N;
        }
    }
}

__device__ __forceinline__ double state_centre(const Geom &g, int d, int32_t j) {
    return dadd(g.lb[d], dmul((double)j, g.eta[d]));
}

// Mean of the post state, Algorithm 2 "Set mu = f(x, nu, w)" for the
// disturbance-free system of Eq. 4.
__device__ __forceinline__ void mean_of(const Geom &g, int32_t x, int32_t u, double *mu) {
    int32_t xi[MAXD];
    double xc[MAXD];
    decode_state(g, x, xi);
#pragma unroll
    for (int d = 0; d < MAXD; ++d)
        if (d < g.n) xc[d] = state_centre(g, d, xi[d]);
    if (g.sys == SYS_AFFINE) {
        const int n = g.n;
        const double *A = g.params + (int64_t)u * (n * n + n);
        const double *c = A + n * n;
#pragma unroll
        for (int i = 0; i < MAXD; ++i) {
            if (i < n) {
                double acc = 0.0;
#pragma unroll
                for (int j = 0; j < MAXD; ++j)
                    if (j < n) acc = dadd(acc, dmul(__ldg(A + i * n + j), xc[j]));
                mu[i] = dadd(acc, __ldg(c + i));
            }
        }
    } else {
        // unicycle: input (v, w) in C order over a 2-D input grid
        const int32_t uw = u % g.ucount[1];
        const int32_t uv = u / g.ucount[1];
        const double v = dadd(g.ulb[0], dmul((double)uv, g.ueta[0]));
        const double w = dadd(g.ulb[1], dmul((double)uw, g.ueta[1]));
        const double tau = __ldg(g.params);
        const double tv = dmul(tau, v);
        mu[0] = dadd(xc[0], dmul(tv, cos(xc[2])));
        mu[1] = dadd(xc[1], dmul(tv, sin(xc[2])));
        mu[2] = dadd(xc[2], dmul(tau, w));
    }
}

// Component d of the mean, with the same FP64 operations in the same order
// as mean_of (for the per-dimension tables, which need one component).
__device__ __forceinline__ double mean_component(const Geom &g, int32_t x, int32_t u, int d) {
    int32_t xi[MAXD];
    decode_state(g, x, xi);
    if (g.sys == SYS_AFFINE) {
        const int n = g.n;
        const double *A = g.params + (int64_t)u * (n * n + n);
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < MAXD; ++j)
            if (j < n) acc = dadd(acc, dmul(__ldg(A + d * n + j), state_centre(g, j, xi[j])));
        return dadd(acc, __ldg(A + n * n + d));
    }
    const int32_t uw = u % g.ucount[1];
    const int32_t uv = u / g.ucount[1];
    const double v = dadd(g.ulb[0], dmul((double)uv, g.ueta[0]));
    const double w = dadd(g.ulb[1], dmul((double)uw, g.ueta[1]));
    const double tau = __ldg(g.params);
    const double th = state_centre(g, 2, xi[2]);
    if (d == 2) return dadd(th, dmul(tau, w));
    const double tv = dmul(tau, v);
    if (d == 0) return dadd(state_centre(g, 0, xi[0]), dmul(tv, cos(th)));
    return dadd(state_centre(g, 1, xi[1]), dmul(tv, sin(th)));
}

// Window origin of one dimension (first slot index, unwrapped), in the FP64
// expression order fixed by the ABI.  Far-away origins are clamped where every
// slot is off the grid anyway.
__device__ __forceinline__ int32_t origin_of(const Geom &g, int d, double mu) {
    double od;
    if (g.wmode == WM_EXPLICIT)
        od = dsub(floor(dadd(ddiv(dsub(mu, g.lb[d]), g.eta[d]), 0.5)), (double)((g.W[d] - 1) / 2));
    else if (g.wmode == WM_DENSE)
        od = 0.0;
    else
        od = ceil(ddiv(dsub(dsub(mu, g.xs[d]), g.lb[d]), g.eta[d]));
    if (!((g.periodic >> d) & 1u)) {
        const double lo = -(double)(g.W[d] + 1), hi = (double)(g.N[d] + 1);
        if (!(od >= lo)) od = lo;
        if (!(od <= hi)) od = hi;
    } else {
        if (!(od >= -1073741824.0)) od = -1073741824.0;
        if (!(od <= 1073741824.0)) od = 1073741824.0;
    }
    return (int32_t)od;
}

// Number of leading slots of the window that pass the gamma-mode upper test
// centre <= mu + xs (centres grow with the slot, so test from the top).
__device__ __forceinline__ int kept_upper(const Geom &g, int d, double mu, int32_t o) {
    int kmax = g.W[d];
    if (g.wmode == WM_GAMMA) {
        const double hi = dadd(mu, g.xs[d]);
        while (kmax > 0) {
            const double c = state_centre(g, d, o + kmax - 1);
            if (c <= hi) break;
            --kmax;
        }
    }
    return kmax;
}

__device__ __forceinline__ int32_t cell_of(const Geom &g, int d, int32_t s, bool &on_grid) {
    const int32_t N = g.N[d];
    if ((g.periodic >> d) & 1u) {
        on_grid = true;
        int32_t r = s % N;
        return r < 0 ? r + N : r;
    }
    on_grid = (s >= 0 && s < N);
    return s < 0 ? 0 : (s >= N ? N - 1 : s);
}

// Per-dimension cell masses of one window (FP32 path).  Each edge's tail
// beyond it (away from mu) is evaluated once with erfcf; a cell's mass is the
// difference of its edge tails on the same side of mu, or one minus both tails
// when it contains mu -- no probability close to one is subtracted.
__device__ __forceinline__ void dim_masses_f32(const Geom &g, int d, double mu, int32_t o,
                                               float *fac, int32_t *off) {
    const int W = g.W[d];
    const int kmax = kept_upper(g, d, mu, o);
    const double c0 = state_centre(g, d, o);
    const float e0 = (float)dsub(dsub(c0, dmul(0.5, g.eta[d])), mu);  // first edge - mu
    const float etaf = (float)g.eta[d];
    const float r = g.rk2f[d];
    float dlo = e0;
    float tlo = 0.5f * erfcf(fabsf(dlo) * r);
    for (int k = 0; k < W; ++k) {
        const float dhi = fmaf((float)(k + 1), etaf, e0);
        const float thi = 0.5f * erfcf(fabsf(dhi) * r);
        float mass;
        if (dlo >= 0.0f)
            mass = tlo - thi;
        else if (dhi <= 0.0f)
            mass = thi - tlo;
        else
            mass = 1.0f - tlo - thi;
        bool on;
        const int32_t cell = cell_of(g, d, o + k, on);
        fac[k] = (on && k < kmax) ? fmaxf(mass, 0.0f) : 0.0f;
        off[k] = cell * g.stride[d];
        dlo = dhi;
        tlo = thi;
    }
}

// FP64 path: each cell's mass from its own two edges, as in Algorithm 1.
// Slot k of dim d's window (origin o, kmax slots kept): its mass and V offset.
__device__ __forceinline__ void slot_mass_f64(const Geom &g, int d, double mu, int32_t o, int kmax, int k,
                                              double &fac, int32_t &off) {
    const double k2 = g.k2[d];
    const double h = dmul(0.5, g.eta[d]);
    const double c = state_centre(g, d, o + k);
    const double elo = dsub(c, h), ehi = dadd(c, h);
    double mass;
    if (elo >= mu)
        mass = 0.5 * erfc(ddiv(dsub(elo, mu), k2)) - 0.5 * erfc(ddiv(dsub(ehi, mu), k2));
    else if (ehi <= mu)
        mass = 0.5 * erfc(ddiv(dsub(mu, ehi), k2)) - 0.5 * erfc(ddiv(dsub(mu, elo), k2));
    else
        mass = 1.0 - 0.5 * erfc(ddiv(dsub(mu, elo), k2)) - 0.5 * erfc(ddiv(dsub(ehi, mu), k2));
    bool on;
    const int32_t cell = cell_of(g, d, o + k, on);
    fac = (on && k < kmax) ? mass : 0.0;
    off = cell * g.stride[d];
}

__device__ __forceinline__ void dim_masses_f64(const Geom &g, int d, double mu, int32_t o,
                                               double *fac, int32_t *off) {
    const int W = g.W[d];
    const int kmax = kept_upper(g, d, mu, o);
    for (int k = 0; k < W; ++k) slot_mass_f64(g, d, mu, o, kmax, k, fac[k], off[k]);
}

// One slot of dim_masses_f32 on its own: the same edge values (edge k is
// fmaf(k, eta, e0), edge 0 is e0) and the same arithmetic, so the mass is
// bit for bit the one the incremental loop gives.
__device__ __forceinline__ void slot_mass_f32(const Geom &g, int d, double mu, int32_t o, int kmax, int k,
                                              float &fac, int32_t &off) {
    const double c0 = state_centre(g, d, o);
    const float e0 = (float)dsub(dsub(c0, dmul(0.5, g.eta[d])), mu);
    const float etaf = (float)g.eta[d];
    const float r = g.rk2f[d];
    const float dlo = k == 0 ? e0 : fmaf((float)k, etaf, e0);
    const float dhi = fmaf((float)(k + 1), etaf, e0);
    const float tlo = 0.5f * erfcf(fabsf(dlo) * r);
    const float thi = 0.5f * erfcf(fabsf(dhi) * r);
    float mass;
    if (dlo >= 0.0f)
        mass = tlo - thi;
    else if (dhi <= 0.0f)
        mass = thi - tlo;
    else
        mass = 1.0f - tlo - thi;
    bool on;
    const int32_t cell = cell_of(g, d, o + k, on);
    fac = (on && k < kmax) ? fmaxf(mass, 0.0f) : 0.0f;
    off = cell * g.stride[d];
}

__device__ __forceinline__ void slot_mass(const Geom &g, int d, double mu, int32_t o, int kmax, int k, double &fac,
                                          int32_t &off) {
    slot_mass_f64(g, d, mu, o, kmax, k, fac, off);
}
__device__ __forceinline__ void slot_mass(const Geom &g, int d, double mu, int32_t o, int kmax, int k, float &fac,
                                          int32_t &off) {
    slot_mass_f32(g, d, mu, o, kmax, k, fac, off);
}

template <class R>
__device__ __forceinline__ void dim_masses(const Geom &g, int d, double mu, int32_t o, R *fac,
                                           int32_t *off);
template <>
__device__ __forceinline__ void dim_masses<float>(const Geom &g, int d, double mu, int32_t o,
                                                  float *fac, int32_t *off) {
    dim_masses_f32(g, d, mu, o, fac, off);
}
template <>
__device__ __forceinline__ void dim_masses<double>(const Geom &g, int d, double mu, int32_t o,
                                                   double *fac, int32_t *off) {
    dim_masses_f64(g, d, mu, o, fac, off);
}

// Offsets of a stored row's slots from its stored origin (dropped slots keep a
// valid clamped offset; their stored mass is zero).
__device__ __forceinline__ void dim_offsets(const Geom &g, int d, int32_t o, int32_t *off) {
    const int W = g.W[d];
    for (int k = 0; k < W; ++k) {
        bool on;
        off[k] = cell_of(g, d, o + k, on) * g.stride[d];
    }
}

}  // namespace amy
