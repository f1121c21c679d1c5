/*
 * amy_oracle.h -- plain FP64 CPU oracle for the finite-MDP abstraction and the
 * finite-horizon Bellman backup of the AMYTISS method (arxiv 2005.06191).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library; both are written from the
 * paper independently.
 *
 * What it computes (paper sections cited per function in amy_oracle.c):
 *   - grid quantiser (Sec. 4, Eq. 7): centres lb + j*eta, j < N,
 *     N = floor((ub-lb)/eta + 1e-9) + 1;
 *   - cutting region (Sec. 5.2, Remark "constructing the cutting region"):
 *     per-dimension 1-D density cut, window widths and origins;
 *   - transition probabilities (Algorithm 1 / Algorithm 2): Gaussian mass of
 *     each post-state cell, a product of per-dimension masses for diagonal
 *     covariance;
 *   - Bellman synthesis (Algorithm 3 / Algorithm 4, OFA semantics of Sec. 6.1):
 *     safety, reachability and reach-avoid value functions with the
 *     lowest-index argmax policy; with a disturbance grid the max over inputs
 *     of the min over disturbances (the two-and-a-half player game of the
 *     Remark in Sec. 3, Algorithm 4's collect step).
 *
 * Everything is IEEE FP64; compile with -ffp-contract=off so that no multiply
 * and add are fused (the exact operation order is part of the definition of
 * the window origin, see amy_oracle.c).
 */
#ifndef AMY_ORACLE_H
#define AMY_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAXD 8

enum { ORC_SYS_AFFINE_PER_INPUT = 0, ORC_SYS_UNICYCLE = 1, ORC_SYS_EXPR = 2 };

/* A system given as text (Sec. 3: the right-hand side of the difference
 * equation written in a configuration file): one C-syntax arithmetic
 * expression per mean component over x0.., u0.., w0.. (the representative
 * points of the state, input and disturbance) and p0.. (the parameters);
 * grammar and functions in amy_oracle_expr.c.  Compiled once, evaluated in
 * FP64 with the C library's functions. */
typedef struct orc_expr orc_expr;
/* NULL on a syntax error or an unknown name, with a message in err. */
orc_expr *orc_expr_compile(const char *const *text, int n, int m, int p, int64_t n_params, char *err, int errlen);
void orc_expr_free(orc_expr *e);
double orc_expr_eval(const orc_expr *e, int d, const double *x, const double *u, const double *w,
                     const double *params);

/* User densities (Sec. 6.2): one expression per dim in the variable t (the
 * noise value), with a box [lo, hi] enclosing its support.  The table of a
 * dim holds 2 (ORC_USER_KNOTS + 1) doubles: the normalised CDF at the knots,
 * then the normalised density there (amy_oracle_expr.c). */
#define ORC_USER_KNOTS 1024
orc_expr *orc_expr_compile_pdf(const char *const *text, int n, char *err, int errlen);
double orc_gauss_legendre8(const orc_expr *pdf, int d, double a, double b);
int orc_user_table(const orc_expr *pdf, int d, double lo, double hi, double *table);
double orc_user_cdf(const double *table, double lo, double hi, double t);
enum { ORC_SAFETY = 0, ORC_REACH = 1, ORC_REACH_AVOID = 2 };

typedef struct {
    int32_t n;                 /* state dimension, 1..8 */
    int32_t m;                 /* input dimension, 1..8 */
    const double *x_lb;        /* [n] first state centre per dim */
    const double *x_eta;       /* [n] state quantisation step */
    const int32_t *x_count;    /* [n] points per dim */
    const uint8_t *x_periodic; /* [n] 1 = index wraps modulo count (may be NULL) */
    const double *u_lb;        /* [m] */
    const double *u_eta;       /* [m] */
    const int32_t *u_count;    /* [m] */
    int32_t sys_kind;          /* ORC_SYS_* */
    const double *params;      /* affine: per input u (C-order) A_u[n*n] row-major then c_u[n];
                                  unicycle: {tau}; expressions: their parameters p0.. */
    int64_t n_params;
    const double *sigma;       /* [n] per-dim noise standard deviation */
    double gamma;              /* cutting threshold; 0 = dense */
    const int32_t *window;     /* [n] explicit odd window widths, or NULL */
    /* Disturbance grid W^ (Sec. 3, the dt-SCS with bounded disturbances; the
     * max-min game of its Remark): p dims, representative points
     * w_lb + j*w_eta, j < w_count.  p = 0: no disturbance (W^ a single point).
     * With p > 0 only the affine system applies and params holds one
     * (A, c) record per (input, disturbance) pair, disturbance fastest:
     * pair index u*n_w + w, n_w = prod(w_count). */
    int32_t p;
    const double *w_lb;        /* [p] */
    const double *w_eta;       /* [p] */
    const int32_t *w_count;    /* [p] */
    /* Noise distribution per dimension (Sec. 6.2: the tool supports other
     * distributions and multiplicative noise; Eq. (1a) for the latter).
     * ORC_NOISE_GAUSSIAN uses sigma; the others their own parameters:
     *   UNIFORM        noise ~ U[-a, a]                        p0 = a
     *   EXPONENTIAL    noise ~ Exp(rate), density rate*e^{-rate t}, t >= 0
     *                                                          p0 = rate
     *   BETA           noise = lo + (hi - lo) * B, B ~ Beta(alpha, beta),
     *                  integer alpha, beta >= 1                p0 = alpha, p1 = beta,
     *                                                          p2 = lo, p3 = hi
     *   MULT_GAUSSIAN  multiplicative: noise = s * x_d * Z, Z ~ N(0,1), x_d
     *                  the state's centre (std s*|x_d|); dense or explicit
     *                  windows only (the cut is disabled, Sec. 6.2)
     *                                                          p0 = s
     * Cutting region (gamma mode) of a bounded support: the support itself;
     * of the exponential: [0, log(rate/gamma)/rate]. */
    int32_t noise;
    const double *noise_p0, *noise_p1, *noise_p2, *noise_p3; /* [n] each (unused ones may be NULL) */
    /* ORC_SYS_EXPR: the compiled mean expressions (params are their p0..);
     * a disturbance grid is allowed, its point bound to w0.. */
    const orc_expr *expr;
    /* ORC_NOISE_USER: per dim the table of orc_user_table (n blocks of
     * 2 (ORC_USER_KNOTS + 1) doubles); noise_p0 / noise_p1 the support box */
    const double *noise_cdf;
} orc_problem;

enum { ORC_NOISE_GAUSSIAN = 0, ORC_NOISE_UNIFORM = 1, ORC_NOISE_EXPONENTIAL = 2, ORC_NOISE_BETA = 3,
       ORC_NOISE_MULT_GAUSSIAN = 4, ORC_NOISE_USER = 5 };

typedef struct {
    int32_t kind;              /* ORC_SAFETY / ORC_REACH / ORC_REACH_AVOID */
    const double *safe_lb;     /* [n] (safety only) */
    const double *safe_ub;
    int32_t n_target;
    const double *target_lb;   /* [n_target*n] */
    const double *target_ub;
    int32_t n_avoid;
    const double *avoid_lb;    /* [n_avoid*n] */
    const double *avoid_ub;
} orc_spec;

/* N = floor((ub - lb)/eta + 1e-9) + 1 */
int64_t orc_grid_count(double lb, double ub, double eta);

/* Window widths W[n] and cut offsets xstar[n]: the Gaussian cut half-width,
 * the upper end of the cut interval for the other distributions (INFINITY
 * when not in gamma mode).  Returns 0, or -1 when the cut is empty / invalid. */
int orc_window_shape(const orc_problem *p, int32_t *W, double *xstar);

/* Mean mu[n] = f(centre(x), centre(u), centre(w)) for linear state index x
 * and input index u -- with a disturbance grid, the pair index u*n_w + w. */
int orc_mean(const orc_problem *p, int64_t x, int64_t u, double *mu);

/* One transition row: origin[n] (first slot index per dim, unwrapped) and the
 * |W| window probabilities in C order over the window box (0 for dropped
 * slots); u as in orc_mean.  Returns 0 or -1. */
int orc_row(const orc_problem *p, int64_t x, int64_t u, int32_t *origin, double *probs);

/* Per-state flags: bit0 target, bit1 avoid, bit2 safe. */
int orc_spec_mask(const orc_problem *p, const orc_spec *s, uint8_t *mask);

/* One Bellman backup for a list of states given V_next[n_x].
 * V_out[i], pi_out[i] (0xFFFF on masked states) and gap_out[i] (top-1 minus
 * top-2 action value, +INF when n_u == 1 or masked) for states[i].
 * Any output pointer may be NULL.  nthreads <= 0: OpenMP default. */
int orc_backup_states(const orc_problem *p, const orc_spec *s, const double *V_next,
                      const int64_t *states, int64_t n_states,
                      double *V_out, uint16_t *pi_out, double *gap_out, int nthreads);

/* Action values at one (unmasked) state x for every input u: the window sum
 * s_{u,w} = sum over the window of T(x'|x,u,w) * V_next[x'], minimised over
 * the disturbances w (just s_u without a disturbance grid): out[n_u]. */
int orc_action_values(const orc_problem *p, const double *V_next, int64_t x, double *out);

/* Philox4x64-10 (the counter-based generator of Salmon et al., SC'11): ten
 * rounds of two 64x64->128-bit multiplies and a key schedule by the Weyl
 * constants; out = the four 64-bit words for counter ctr[4] and key key[2]. */
void orc_philox4x64(const uint64_t *ctr, const uint64_t *key, uint64_t *out);

/* Closed-loop simulation of the finite MDP (the validation of Sec. 7: runs of
 * the controlled system from chosen initial states) under a synthesized
 * policy: policy[horizon][n_x] holds pi_t for t = 0..horizon-1 (as
 * orc_synthesize writes it).  For each initial state x0[i], `runs` runs of
 * `horizon` steps: a run succeeds when it meets the spec (reaches a target
 * before any avoid state and before the horizon; stays in the safe set
 * through the horizon).  Each step draws, per state dim d, the next cell by
 * inverse CDF from that dim's window masses (a uniform draw beyond their sum
 * -- the truncated or off-grid mass -- loses the run), and with a
 * disturbance grid first draws its point uniformly.  Draw q of step t of
 * global run g = i*runs + r is word q%4 of Philox4x64-10 at counter
 * (g, t, q/4, 0), key (seed, 0), as a double (w >> 11) * 2^-53; draws
 * q = 0..n-1 pick the dims, q = n the disturbance.  successes[i] counts the
 * successful runs of x0[i]. */
int orc_simulate(const orc_problem *p, const orc_spec *s, int32_t horizon, const uint16_t *policy,
                 const int64_t *x0, int64_t n_x0, int64_t runs, uint64_t seed, int64_t *successes);

/* Full synthesis over `horizon` backups.  V_out[n_x] = V_0.
 * pi_out: [horizon][n_x] (pi_k for k = 0..horizon-1) or NULL.
 * gap_out: [horizon][n_x] or NULL.  V_all: [(horizon+1)][n_x] (V_k, k=0..horizon) or NULL. */
int orc_synthesize(const orc_problem *p, const orc_spec *s, int32_t horizon,
                   double *V_out, uint16_t *pi_out, double *gap_out, double *V_all,
                   int nthreads);

#ifdef __cplusplus
}
#endif
#endif
