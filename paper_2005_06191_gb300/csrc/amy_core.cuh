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
enum SysKind : int32_t { SYS_AFFINE = 0, SYS_UNICYCLE = 1, SYS_EXPR = 2 };
enum SpecKind : int32_t { SPEC_SAFETY = 0, SPEC_REACH = 1, SPEC_REACH_AVOID = 2 };
enum TMode : int32_t { TM_OTF = 0, TM_FULL = 1, TM_FACTORED = 2, TM_SEPARABLE = 3 };
// Noise distribution per dimension (Sec. 6.2; multiplicative noise as in Eq. (1a)).
enum NoiseKind : int32_t { NOISE_GAUSSIAN = 0, NOISE_UNIFORM = 1, NOISE_EXPONENTIAL = 2, NOISE_BETA = 3,
                           NOISE_MULT_GAUSSIAN = 4, NOISE_USER = 5 };
// Knot intervals of a user density's CDF table (the knots t_i = lo + i h).
constexpr int USER_KNOTS = 1024;

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
    double xs[MAXD];             // gamma-mode cut half width (Gaussian noise)
    double clo[MAXD], chi[MAXD]; // gamma-mode cut interval of the noise: [mu + clo, mu + chi]
    double k2[MAXD];             // sigma*sqrt(2) (Gaussian noise)
    float rk2f[MAXD];            // 1/(sigma*sqrt(2)) in FP32 (Gaussian noise)
    int32_t noise;               // NoiseKind
    double np[4][MAXD];          // its parameters: uniform a; exponential rate; beta alpha, beta,
                                 // lo, hi (integer shapes); multiplicative Gaussian s (std s*|x_d|)
    int32_t sys;                 // SysKind
    int32_t ucount[MAXD];
    double ulb[MAXD], ueta[MAXD];
    const double *params;        // device copy of the system parameters
    // Text systems (SYS_EXPR): component d of the mean, tabulated over the
    // coordinates it reads -- record e = sum_j xi_j * tsx[d][j] + sum_i ui_i *
    // tsu[d][i], the index of the per-dimension tables -- at mtab[moff[d] + e].
    const double *mtab;
    int64_t moff[MAXD];
    // User densities (NOISE_USER): per dim the normalised CDF at the
    // USER_KNOTS + 1 knots of the support box [np[0][d], np[1][d]], then the
    // normalised density there (2 (USER_KNOTS + 1) doubles per dim)
    const double *ucdf;
    uint32_t xdep[MAXD], udep[MAXD];  // the coordinates each component's text reads (host planning)
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

// The centre in dim d of state x where the noise depends on it
// (multiplicative noise), else 0 (unused).
__device__ __forceinline__ double noise_centre(const Geom &g, int32_t x, int d) {
    if (g.noise != NOISE_MULT_GAUSSIAN) return 0.0;
    const int32_t j = (int32_t)(((uint32_t)x / (uint32_t)g.stride[d]) % (uint32_t)g.N[d]);
    return state_centre(g, d, j);
}

// Component d of a text system's mean at state coordinates xi and (input,
// disturbance) pair u: its tabulated value.
__device__ __forceinline__ double expr_mean(const Geom &g, const int32_t *xi, int32_t u, int d) {
    int64_t e = 0;
    uint32_t r = (uint32_t)u;
#pragma unroll
    for (int i = MAXD - 1; i >= 0; --i) {
        if (i < g.m) {
            const uint32_t U = (uint32_t)g.ucount[i];
            e += (int64_t)(r % U) * g.tsu[d][i];
            r /= U;
        }
    }
#pragma unroll
    for (int j = 0; j < MAXD; ++j)
        if (j < g.n) e += (int64_t)xi[j] * g.tsx[d][j];
    return __ldg(g.mtab + g.moff[d] + e);
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
    if (g.sys == SYS_EXPR) {
#pragma unroll
        for (int d = 0; d < MAXD; ++d)
            if (d < g.n) mu[d] = expr_mean(g, xi, u, d);
        return;
    }
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
    if (g.sys == SYS_EXPR) return expr_mean(g, xi, u, d);
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
// expression order fixed by the ABI: ceil(((mu + clo) - lb) / eta) in gamma
// mode (for the Gaussian clo = -xs, and mu + (-xs) is mu - xs exactly).
// Far-away origins are clamped where every slot is off the grid anyway.
__device__ __forceinline__ int32_t origin_of(const Geom &g, int d, double mu) {
    double od;
    if (g.wmode == WM_EXPLICIT)
        od = dsub(floor(dadd(ddiv(dsub(mu, g.lb[d]), g.eta[d]), 0.5)), (double)((g.W[d] - 1) / 2));
    else if (g.wmode == WM_DENSE)
        od = 0.0;
    else
        od = ceil(ddiv(dsub(dadd(mu, g.clo[d]), g.lb[d]), g.eta[d]));
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
// centre <= mu + chi (centres grow with the slot, so test from the top).
__device__ __forceinline__ int kept_upper(const Geom &g, int d, double mu, int32_t o) {
    int kmax = g.W[d];
    if (g.wmode == WM_GAMMA) {
        const double hi = dadd(mu, g.chi[d]);
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

// Regularised incomplete beta I_z(a, b) for integer a, b >= 1 (a + b <= 64):
// the probability that at least a of a + b - 1 trials with success
// probability z succeed, a binomial tail summed term by term.
template <class R>
__device__ __noinline__ R inc_beta_int(int a, int b, R z) {
    if (z <= R(0)) return R(0);
    if (z >= R(1)) return R(1);
    const int n = a + b - 1;
    R sum = R(0);
    for (int j = a; j <= n; ++j) {
        R c = R(1);  // C(n, j)
        for (int i = 1; i <= j; ++i) c = c * (R)(n - j + i) / (R)i;
        sum += c * pow(z, (R)j) * pow(R(1) - z, (R)(n - j));
    }
    return sum;
}

// Cell mass for the noise kinds other than the (additive or multiplicative)
// Gaussian, Algorithm 1's cell integral for the distributions of Sec. 6.2;
// tlo < thi are the cell's edges minus the mean.  Uniform on [-a, a]: the
// overlap; exponential: the difference of the survival function at the two
// edges; beta (noise = lo + (hi - lo) B, integer shapes): incomplete-beta
// differences, from the upper tail in the upper half.  Kept out of line:
// the Gaussian is the common case, and the unrolled kernels would otherwise
// inline this code into every slot.
// CDF of dim d's user density at t (t relative to the mean): 0 below the
// box, 1 above, between knots the cubic Hermite interpolant of the tabulated
// CDF values and densities, in FP64 with every operation rounded as written.
__device__ __forceinline__ double user_cdf(const Geom &g, int d, double t) {
    const double lo = g.np[0][d], hi = g.np[1][d];
    if (t <= lo) return 0.0;
    if (t >= hi) return 1.0;
    const double h = ddiv(dsub(hi, lo), (double)USER_KNOTS);
    const double s = ddiv(dsub(t, lo), h);
    int i = (int)floor(s);
    if (i > USER_KNOTS - 1) i = USER_KNOTS - 1;
    const double tau = dsub(s, (double)i), tau2 = dmul(tau, tau), tau3 = dmul(tau2, tau);
    const double h00 = dadd(dsub(dmul(2.0, tau3), dmul(3.0, tau2)), 1.0);
    const double h10 = dadd(dsub(tau3, dmul(2.0, tau2)), tau);
    const double h01 = dadd(dmul(-2.0, tau3), dmul(3.0, tau2));
    const double h11 = dsub(tau3, tau2);
    const double *F = g.ucdf + (int64_t)d * 2 * (USER_KNOTS + 1), *f = F + (USER_KNOTS + 1);
    return dadd(dadd(dadd(dmul(h00, __ldg(F + i)), dmul(dmul(h10, h), __ldg(f + i))), dmul(h01, __ldg(F + i + 1))),
                dmul(dmul(h11, h), __ldg(f + i + 1)));
}

template <class R>
__device__ __noinline__ R noise_mass(const Geom &g, int d, R tlo, R thi) {
    if (g.noise == NOISE_USER) {
        const double m = dsub(user_cdf(g, d, (double)thi), user_cdf(g, d, (double)tlo));
        return (R)(m > 0.0 ? m : 0.0);
    }
    if (g.noise == NOISE_UNIFORM) {
        const R a = (R)g.np[0][d];
        const R lo = tlo > -a ? tlo : -a, hi = thi < a ? thi : a;
        return hi > lo ? (hi - lo) / (R(2) * a) : R(0);
    }
    if (g.noise == NOISE_EXPONENTIAL) {
        const R rate = (R)g.np[0][d];
        const R slo = tlo > R(0) ? exp(-rate * tlo) : R(1);
        const R shi = thi > R(0) ? exp(-rate * thi) : R(1);
        return slo - shi;
    }
    // NOISE_BETA
    const int a = (int)g.np[0][d], b = (int)g.np[1][d];
    const R lo = (R)g.np[2][d], span = (R)(g.np[3][d] - g.np[2][d]);
    const R zlo = (tlo - lo) / span, zhi = (thi - lo) / span;
    if (zlo >= R(0.5)) return inc_beta_int<R>(b, a, R(1) - zlo) - inc_beta_int<R>(b, a, R(1) - zhi);
    return inc_beta_int<R>(a, b, zhi) - inc_beta_int<R>(a, b, zlo);
}

// 1/(sigma*sqrt(2)) of dim d's Gaussian noise at a state whose centre in dim
// d is xd: the fixed sigma, or s*|xd| for multiplicative noise (0 when that
// std is 0: no noise, the whole mass in the cell holding the mean).
__device__ __forceinline__ float gauss_r_f32(const Geom &g, int d, double xd) {
    if (g.noise != NOISE_MULT_GAUSSIAN) return g.rk2f[d];
    const double s = g.np[0][d] * fabs(xd);
    return s > 0.0 ? (float)(1.0 / (s * 1.4142135623730951)) : 0.0f;
}

// FP32 mass of one cell with edges dlo < dhi (minus the mean) from the
// Gaussian tails tlo = Q(|dlo|), thi = Q(|dhi|) taken on the far side of the
// mean; r = 0 is the noiseless case of multiplicative noise.
__device__ __forceinline__ float gauss_cell_f32(float dlo, float dhi, float tlo, float thi, float r) {
    if (r == 0.0f) return (dlo <= 0.0f && 0.0f < dhi) ? 1.0f : 0.0f;
    if (dlo >= 0.0f) return tlo - thi;
    if (dhi <= 0.0f) return thi - tlo;
    return 1.0f - tlo - thi;
}

// Per-dimension cell masses of one window (FP32 path).  Gaussian noise: each
// edge's tail beyond it (away from mu) is evaluated once with erfcf; a cell's
// mass is the difference of its edge tails on the same side of mu, or one
// minus both tails when it contains mu -- no probability close to one is
// subtracted.  The other kinds take each cell from its two edges.  xd: the
// state's centre in dim d (multiplicative noise scales with it).
__device__ __forceinline__ void dim_masses_f32(const Geom &g, int d, double mu, int32_t o, double xd,
                                               float *fac, int32_t *off) {
    const int W = g.W[d];
    const int kmax = kept_upper(g, d, mu, o);
    const double c0 = state_centre(g, d, o);
    const float e0 = (float)dsub(dsub(c0, dmul(0.5, g.eta[d])), mu);  // first edge - mu
    const float etaf = (float)g.eta[d];
    const bool gauss = g.noise == NOISE_GAUSSIAN || g.noise == NOISE_MULT_GAUSSIAN;
    const float r = gauss_r_f32(g, d, xd);
    float dlo = e0;
    float tlo = gauss ? 0.5f * erfcf(fabsf(dlo) * r) : 0.0f;
    for (int k = 0; k < W; ++k) {
        const float dhi = fmaf((float)(k + 1), etaf, e0);
        const float thi = gauss ? 0.5f * erfcf(fabsf(dhi) * r) : 0.0f;
        const float mass = gauss ? gauss_cell_f32(dlo, dhi, tlo, thi, r) : noise_mass<float>(g, d, dlo, dhi);
        bool on;
        const int32_t cell = cell_of(g, d, o + k, on);
        fac[k] = (on && k < kmax) ? fmaxf(mass, 0.0f) : 0.0f;
        off[k] = cell * g.stride[d];
        dlo = dhi;
        tlo = thi;
    }
}

// FP64 path, Algorithm 1's cell integral.  Edge k of dim d's window (origin
// o) lies at c(o + k) - eta/2, so that a cell's upper edge is the next cell's
// lower edge (c(o + k) + eta/2 up to rounding) and a run of cells evaluates
// each edge's tail once.  Edges are kept relative to the mean: t = edge - mu.
__device__ __forceinline__ double edge_rel_f64(const Geom &g, int d, double mu, int32_t o, int k) {
    return dsub(dsub(state_centre(g, d, o + k), dmul(0.5, g.eta[d])), mu);
}

// sigma * sqrt(2) of dim d's Gaussian noise at a state whose centre in dim d
// is xd (0 for multiplicative noise at xd = 0: no noise)
__device__ __forceinline__ double gauss_k2_f64(const Geom &g, int d, double xd) {
    return g.noise == NOISE_GAUSSIAN ? g.k2[d] : dmul(dmul(g.np[0][d], fabs(xd)), 1.4142135623730951);
}

// Gaussian tail beyond edge t, away from the mean: erfc(|t| / k2) / 2
__device__ __forceinline__ double gauss_tail_f64(double t, double k2) {
    return k2 == 0.0 ? 0.0 : 0.5 * erfc(ddiv(fabs(t), k2));
}

// Mass of the cell with edges tlo < thi (minus the mean) from their tails:
// the difference of the tails on the same side of the mean, or one minus
// both tails when the cell holds the mean
__device__ __forceinline__ double gauss_cell_f64(double tlo, double thi, double qlo, double qhi, double k2) {
    if (k2 == 0.0) return (tlo <= 0.0 && 0.0 < thi) ? 1.0 : 0.0;
    if (tlo >= 0.0) return qlo - qhi;
    if (thi <= 0.0) return qhi - qlo;
    return 1.0 - qlo - qhi;
}

// Slots [k0, k1) of dim d's window (origin o, kmax slots kept): put(k, mass,
// V offset) for each, every edge evaluated once.  A slot's values do not
// depend on the run it is evaluated in.
template <class Put>
__device__ __forceinline__ void slot_run_f64(const Geom &g, int d, double mu, int32_t o, int kmax, int k0, int k1,
                                             double xd, Put &&put) {
    const bool gauss = g.noise == NOISE_GAUSSIAN || g.noise == NOISE_MULT_GAUSSIAN;
    const double k2 = gauss ? gauss_k2_f64(g, d, xd) : 0.0;
    double tlo = edge_rel_f64(g, d, mu, o, k0);
    double qlo = gauss ? gauss_tail_f64(tlo, k2) : 0.0;
    for (int k = k0; k < k1; ++k) {
        const double thi = edge_rel_f64(g, d, mu, o, k + 1);
        const double qhi = gauss ? gauss_tail_f64(thi, k2) : 0.0;
        const double mass = gauss ? gauss_cell_f64(tlo, thi, qlo, qhi, k2) : noise_mass<double>(g, d, tlo, thi);
        bool on;
        const int32_t cell = cell_of(g, d, o + k, on);
        put(k, (on && k < kmax) ? mass : 0.0, cell * g.stride[d]);
        tlo = thi;
        qlo = qhi;
    }
}

__device__ __forceinline__ void dim_masses_f64(const Geom &g, int d, double mu, int32_t o, double xd,
                                               double *fac, int32_t *off) {
    slot_run_f64(g, d, mu, o, kept_upper(g, d, mu, o), 0, g.W[d], xd, [&](int k, double m, int32_t f) {
        fac[k] = m;
        off[k] = f;
    });
}

// Slots [k0, k1) of dim d's window in FP32, each edge's tail evaluated once:
// the values dim_masses_f32 gives (edge k is fmaf(k, eta, e0), edge 0 is e0),
// whichever run a slot is evaluated in.
template <class Put>
__device__ __forceinline__ void slot_run_f32(const Geom &g, int d, double mu, int32_t o, int kmax, int k0, int k1,
                                             double xd, Put &&put) {
    const double c0 = state_centre(g, d, o);
    const float e0 = (float)dsub(dsub(c0, dmul(0.5, g.eta[d])), mu);
    const float etaf = (float)g.eta[d];
    const bool gauss = g.noise == NOISE_GAUSSIAN || g.noise == NOISE_MULT_GAUSSIAN;
    const float r = gauss ? gauss_r_f32(g, d, xd) : 0.0f;
    float dlo = k0 == 0 ? e0 : fmaf((float)k0, etaf, e0);
    float tlo = gauss ? 0.5f * erfcf(fabsf(dlo) * r) : 0.0f;
    for (int k = k0; k < k1; ++k) {
        const float dhi = fmaf((float)(k + 1), etaf, e0);
        const float thi = gauss ? 0.5f * erfcf(fabsf(dhi) * r) : 0.0f;
        const float mass = gauss ? gauss_cell_f32(dlo, dhi, tlo, thi, r) : noise_mass<float>(g, d, dlo, dhi);
        bool on;
        const int32_t cell = cell_of(g, d, o + k, on);
        put(k, (on && k < kmax) ? fmaxf(mass, 0.0f) : 0.0f, cell * g.stride[d]);
        dlo = dhi;
        tlo = thi;
    }
}

template <class Put>
__device__ __forceinline__ void slot_run(const Geom &g, int d, double mu, int32_t o, int kmax, int k0, int k1,
                                         double xd, Put &&put, double) {
    slot_run_f64(g, d, mu, o, kmax, k0, k1, xd, put);
}
template <class Put>
__device__ __forceinline__ void slot_run(const Geom &g, int d, double mu, int32_t o, int kmax, int k0, int k1,
                                         double xd, Put &&put, float) {
    slot_run_f32(g, d, mu, o, kmax, k0, k1, xd, put);
}

template <class R>
__device__ __forceinline__ void dim_masses(const Geom &g, int d, double mu, int32_t o, double xd, R *fac,
                                           int32_t *off);
template <>
__device__ __forceinline__ void dim_masses<float>(const Geom &g, int d, double mu, int32_t o, double xd,
                                                  float *fac, int32_t *off) {
    dim_masses_f32(g, d, mu, o, xd, fac, off);
}
template <>
__device__ __forceinline__ void dim_masses<double>(const Geom &g, int d, double mu, int32_t o, double xd,
                                                   double *fac, int32_t *off) {
    dim_masses_f64(g, d, mu, o, xd, fac, off);
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
