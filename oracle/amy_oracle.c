/*
 * amy_oracle.c -- plain, slow, FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests, the smoke check and the benchmark's CPU-baseline leg load this.
 * It shares no code with the CUDA library.  Every step follows the paper
 * (arxiv 2005.06191, "AMYTISS") in its own order and notation:
 *
 *   Sec. 4 (finite MDP, Eq. 5):  T^(x'|x,u) = T(Xi(x')|x,u), the
 *       probability that f(x,u) + noise lands in the cell of x'.
 *   Algorithm 1:  T entry = integral of the Gaussian density over the cell;
 *       for a diagonal covariance this is a product of 1-D masses.
 *   Sec. 5.2 + Remark on constructing the cutting region:  per dimension the
 *       1-D density equals gamma at +-xs, and the kept post states are the
 *       grid centres inside [mu - xs, mu + xs]; the row has a fixed width.
 *   Algorithm 3 / Algorithm 4:  backward recursion over the horizon, V_in as
 *       the window sum of T * V_{k+1}, then max (and lowest argmax) over u.
 *   Sec. 6.1 (OFA):  rows are recomputed where needed; the oracle does so for
 *       every state and step, which is the same arithmetic as storing them.
 *
 * Readings of points the paper leaves open (kept identical in the CUDA path,
 * which implements them independently):
 *   - points per dim N = floor((ub-lb)/eta + 1e-9) + 1, centre_j = lb + j*eta;
 *   - cells tile [lb - eta/2, ub + eta/2]; mass leaving the grid is lost;
 *   - gamma mode: xs = sigma*sqrt(2*log(1/(gamma*sigma*sqrt(2*pi)))),
 *     W = floor(2*xs/eta) + 1, origin o = ceil(((mu - xs) - lb)/eta), slot
 *     o+k kept iff its centre lb + (o+k)*eta <= mu + xs and it is on the grid
 *     (or the dim is periodic, where the index wraps and the mass is that of
 *     the unwrapped cell);
 *   - explicit odd window W: o = floor((mu - lb)/eta + 0.5) - (W-1)/2;
 *   - gamma == 0: dense, W = N, o = 0;
 *   - reach-avoid via V masking (V = 1 on the target, 0 on the avoid set),
 *     safety as V_k = 1_S * max_u sum;
 *   - argmax ties: lowest input index; masked states carry policy 0xFFFF;
 *   - with a disturbance grid each input's value is the min over the grid
 *     (the adversary moves after the input, knowing it; Sec. 3 Remark);
 *   - other noise distributions (Sec. 6.2): cells are kept by their centres
 *     inside the cut interval [mu + clo, mu + chi] as in the Gaussian case;
 *     bounded supports are their own cut; multiplicative noise is uncut.
 * The target-jump vector of Algorithm 3 is not formed: with V fixed to 1 on
 * the target and 0 on the avoid set, sum_x' T V equals T0 + T_zeroed V exactly.
 */
#include "amy_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static int64_t prod_i32(const int32_t *a, int n) {
    int64_t p = 1;
    for (int i = 0; i < n; ++i) p *= a[i];
    return p;
}

/* C-order decode: last dimension fastest. */
static void decode(int64_t lin, const int32_t *count, int n, int32_t *idx) {
    for (int d = n - 1; d >= 0; --d) {
        idx[d] = (int32_t)(lin % count[d]);
        lin /= count[d];
    }
}

static int is_periodic(const orc_problem *p, int d) {
    return p->x_periodic != NULL && p->x_periodic[d] != 0;
}

/* Grid quantiser, Sec. 4 (map Pi_x and Eq. 7): points per dimension. */
int64_t orc_grid_count(double lb, double ub, double eta) {
    return (int64_t)floor((ub - lb) / eta + 1e-9) + 1;
}

/* Cutting region of one dimension in gamma mode (Sec. 5.2 and its Remark):
 * the noise values t with density >= gamma, as the interval [clo, chi]
 * around the mean.  Gaussian: the 1-D density equals gamma at +-xs.  For the
 * other distributions of Sec. 6.2 the region follows their support: the
 * support itself when it is bounded (uniform: where the flat density reaches
 * gamma at all; beta), [0, log(rate/gamma)/rate] for the exponential.
 * Multiplicative noise has no cut.  Returns 0, or -1 when the region is
 * empty or not defined. */
static int cut_interval(const orc_problem *p, int d, double *clo, double *chi) {
    const double g = p->gamma;
    switch (p->noise) {
        case ORC_NOISE_GAUSSIAN: {
            double s = p->sigma[d];
            double arg = 1.0 / (g * s * sqrt(2.0 * M_PI));
            if (!(arg > 1.0)) return -1; /* gamma at or above the peak density */
            double xs = s * sqrt(2.0 * log(arg));
            *clo = -xs;
            *chi = xs;
            return 0;
        }
        case ORC_NOISE_UNIFORM: {
            double a = p->noise_p0[d];
            if (!(g <= 1.0 / (2.0 * a))) return -1;
            *clo = -a;
            *chi = a;
            return 0;
        }
        case ORC_NOISE_EXPONENTIAL: {
            double rate = p->noise_p0[d];
            if (!(g < rate)) return -1;
            *clo = 0.0;
            *chi = log(rate / g) / rate;
            return 0;
        }
        case ORC_NOISE_BETA:
            *clo = p->noise_p2[d];
            *chi = p->noise_p3[d];
            return 0;
        case ORC_NOISE_USER: /* the user's box enclosing the support */
            *clo = p->noise_p0[d];
            *chi = p->noise_p1[d];
            return 0;
        default:
            return -1;
    }
}

static int noise_valid(const orc_problem *p) {
    for (int d = 0; d < p->n; ++d) {
        switch (p->noise) {
            case ORC_NOISE_GAUSSIAN:
                if (!(p->sigma[d] > 0.0)) return 0;
                break;
            case ORC_NOISE_UNIFORM:
            case ORC_NOISE_EXPONENTIAL:
            case ORC_NOISE_MULT_GAUSSIAN:
                if (!p->noise_p0 || !(p->noise_p0[d] > 0.0)) return 0;
                break;
            case ORC_NOISE_BETA: {
                if (!p->noise_p0 || !p->noise_p1 || !p->noise_p2 || !p->noise_p3) return 0;
                double a = p->noise_p0[d], b = p->noise_p1[d];
                if (!(a >= 1.0 && b >= 1.0 && a == floor(a) && b == floor(b) && a + b <= 64.0)) return 0;
                if (!(p->noise_p3[d] > p->noise_p2[d])) return 0;
                break;
            }
            case ORC_NOISE_USER:
                if (!p->noise_p0 || !p->noise_p1 || !p->noise_cdf) return 0;
                if (!(p->noise_p1[d] > p->noise_p0[d])) return 0;
                break;
            default:
                return 0;
        }
    }
    return 1;
}

/* Cutting region size, Sec. 5.2 and its Remark: the cut interval per
 * dimension, then the fixed number of slots per dimension. */
int orc_window_shape(const orc_problem *p, int32_t *W, double *xstar) {
    if (!noise_valid(p)) return -1;
    for (int d = 0; d < p->n; ++d) {
        if (p->window != NULL) {
            W[d] = p->window[d];
            if (W[d] < 1 || (W[d] % 2) == 0) return -1;
            if (is_periodic(p, d) && W[d] > p->x_count[d]) return -1;
            xstar[d] = INFINITY;
        } else if (p->gamma == 0.0) {
            if (is_periodic(p, d)) return -1;
            W[d] = p->x_count[d];
            xstar[d] = INFINITY;
        } else {
            double clo, chi;
            if (cut_interval(p, d, &clo, &chi) != 0) return -1;
            double w = floor((chi - clo) / p->x_eta[d]) + 1.0;
            if (!(w >= 1.0) || w > 1.0e6) return -1;
            W[d] = (int32_t)w;
            if (is_periodic(p, d) && W[d] > p->x_count[d]) return -1;
            xstar[d] = chi;
        }
    }
    return 0;
}

/* Mean of the post state, Algorithm 2 "Set mu = f(x, nu, w)": the system is
 * evaluated at the representative points of the state, input and (when
 * given) disturbance cells.  The affine system carries one (A, c) per
 * (input, disturbance) pair, so f(x, nu, w) = A x + c needs only the pair's
 * index; u is that index (u*n_w + w). */
int orc_mean(const orc_problem *p, int64_t x, int64_t u, double *mu) {
    const int n = p->n, m = p->m;
    int32_t xi[ORC_MAXD], ui[ORC_MAXD];
    double xc[ORC_MAXD], uc[ORC_MAXD];
    decode(x, p->x_count, n, xi);
    if (p->sys_kind == ORC_SYS_EXPR) {
        /* pair index u = input * n_w + disturbance, each in C order */
        int64_t nw = 1;
        for (int d = 0; d < p->p; ++d) nw *= p->w_count[d];
        int32_t wi[ORC_MAXD];
        double wc[ORC_MAXD];
        decode(u / nw, p->u_count, m, ui);
        decode(u % nw, p->w_count, p->p, wi);
        for (int d = 0; d < n; ++d) xc[d] = p->x_lb[d] + (double)xi[d] * p->x_eta[d];
        for (int d = 0; d < m; ++d) uc[d] = p->u_lb[d] + (double)ui[d] * p->u_eta[d];
        for (int d = 0; d < p->p; ++d) wc[d] = p->w_lb[d] + (double)wi[d] * p->w_eta[d];
        if (!p->expr) return -1;
        for (int d = 0; d < n; ++d) mu[d] = orc_expr_eval(p->expr, d, xc, uc, wc, p->params);
        return 0;
    }
    if (p->sys_kind == ORC_SYS_UNICYCLE) decode(u, p->u_count, m, ui);
    else for (int d = 0; d < m; ++d) ui[d] = 0;
    for (int d = 0; d < n; ++d) xc[d] = p->x_lb[d] + (double)xi[d] * p->x_eta[d];
    for (int d = 0; d < m; ++d) uc[d] = p->u_lb[d] + (double)ui[d] * p->u_eta[d];
    if (p->sys_kind == ORC_SYS_AFFINE_PER_INPUT) {
        const double *A = p->params + u * (int64_t)(n * n + n);
        const double *c = A + n * n;
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int j = 0; j < n; ++j) acc = acc + A[i * n + j] * xc[j];
            mu[i] = acc + c[i];
        }
        return 0;
    }
    if (p->sys_kind == ORC_SYS_UNICYCLE) {
        double tau = p->params[0];
        double v = uc[0], w = uc[1];
        mu[0] = xc[0] + tau * v * cos(xc[2]);
        mu[1] = xc[1] + tau * v * sin(xc[2]);
        mu[2] = xc[2] + tau * w;
        return 0;
    }
    return -1;
}

/* Gaussian mass of [elo, ehi) around mu, Algorithm 1's cell integral in one
 * dimension.  Each tail is taken from the side where it is small, so no
 * probability close to 1 is subtracted from another one. */
static double cell_mass(double elo, double ehi, double mu, double sigma) {
    const double k = sigma * sqrt(2.0);
    if (elo >= mu) return 0.5 * erfc((elo - mu) / k) - 0.5 * erfc((ehi - mu) / k);
    if (ehi <= mu) return 0.5 * erfc((mu - ehi) / k) - 0.5 * erfc((mu - elo) / k);
    return 1.0 - 0.5 * erfc((mu - elo) / k) - 0.5 * erfc((ehi - mu) / k);
}

/* Regularised incomplete beta I_z(a, b) for integer a, b >= 1: the
 * probability that at least a of a + b - 1 independent trials with success
 * probability z succeed, sum_{j=a}^{a+b-1} C(a+b-1, j) z^j (1-z)^{a+b-1-j}. */
static double inc_beta_int(int a, int b, double z) {
    if (z <= 0.0) return 0.0;
    if (z >= 1.0) return 1.0;
    const int n = a + b - 1;
    double sum = 0.0;
    for (int j = a; j <= n; ++j) {
        double c = 1.0; /* C(n, j) */
        for (int i = 1; i <= j; ++i) c = c * (double)(n - j + i) / (double)i;
        sum += c * pow(z, (double)j) * pow(1.0 - z, (double)(n - j));
    }
    return sum;
}

/* Mass of the cell [elo, ehi) for the noise of dimension d around the mean
 * mu (Algorithm 1's cell integral for the distributions of Sec. 6.2); xd is
 * the state's centre in dimension d (multiplicative noise scales with it). */
static double noise_mass(const orc_problem *p, int d, double elo, double ehi, double mu, double xd) {
    const double tlo = elo - mu, thi = ehi - mu;
    switch (p->noise) {
        case ORC_NOISE_UNIFORM: {
            const double a = p->noise_p0[d];
            const double lo = tlo > -a ? tlo : -a, hi = thi < a ? thi : a;
            return hi > lo ? (hi - lo) / (2.0 * a) : 0.0;
        }
        case ORC_NOISE_EXPONENTIAL: {
            /* difference of the survival function exp(-rate t) at the two edges */
            const double rate = p->noise_p0[d];
            const double slo = tlo > 0.0 ? exp(-rate * tlo) : 1.0;
            const double shi = thi > 0.0 ? exp(-rate * thi) : 1.0;
            return slo - shi;
        }
        case ORC_NOISE_BETA: {
            const int a = (int)p->noise_p0[d], b = (int)p->noise_p1[d];
            const double lo = p->noise_p2[d], hi = p->noise_p3[d];
            const double zlo = (tlo - lo) / (hi - lo), zhi = (thi - lo) / (hi - lo);
            /* upper half: differences of the upper tail I_{1-z}(b, a) */
            if (zlo >= 0.5) return inc_beta_int(b, a, 1.0 - zlo) - inc_beta_int(b, a, 1.0 - zhi);
            return inc_beta_int(a, b, zhi) - inc_beta_int(a, b, zlo);
        }
        case ORC_NOISE_USER: {
            /* the normalised CDF of the user's density at the two edges */
            const double *table = p->noise_cdf + (size_t)d * 2 * (ORC_USER_KNOTS + 1);
            const double lo = p->noise_p0[d], hi = p->noise_p1[d];
            const double m = orc_user_cdf(table, lo, hi, thi) - orc_user_cdf(table, lo, hi, tlo);
            return m > 0.0 ? m : 0.0;
        }
        case ORC_NOISE_MULT_GAUSSIAN: {
            const double s = p->noise_p0[d] * fabs(xd);
            if (s == 0.0) return (elo <= mu && mu < ehi) ? 1.0 : 0.0; /* no noise at x_d = 0 */
            return cell_mass(elo, ehi, mu, s);
        }
        default:
            return cell_mass(elo, ehi, mu, p->sigma[d]);
    }
}

/* Cutting window of one dimension, Remark on constructing the cutting region:
 * origin, per-slot mass and cell index (-1 for a dropped slot). */
static int32_t dim_window(const orc_problem *p, int d, int32_t W, double mu, double xd,
                          double *fac, int64_t *cell) {
    const int32_t N = p->x_count[d];
    const double lb = p->x_lb[d], eta = p->x_eta[d];
    const int per = is_periodic(p, d);
    const int gmode = (p->window == NULL && p->gamma != 0.0);
    double clo = 0.0, chi = 0.0;
    if (gmode) cut_interval(p, d, &clo, &chi);
    double od;
    if (p->window != NULL)
        od = floor((mu - lb) / eta + 0.5) - (double)((W - 1) / 2);
    else if (p->gamma == 0.0)
        od = 0.0;
    else
        od = ceil(((mu + clo) - lb) / eta);
    /* Clamp far-away origins: outside [-(W+1), N+1] every slot is off the grid
     * anyway (non-periodic); periodic origins are kept within +-2^30. */
    if (!per) {
        if (!(od >= -(double)(W + 1))) od = -(double)(W + 1);
        if (!(od <= (double)(N + 1))) od = (double)(N + 1);
    } else {
        if (!(od >= -1073741824.0)) od = -1073741824.0;
        if (!(od <= 1073741824.0)) od = 1073741824.0;
    }
    const int32_t o = (int32_t)od;
    for (int32_t k = 0; k < W; ++k) {
        int64_t s = (int64_t)o + k;
        double c = lb + (double)s * eta;
        int keep = per || (s >= 0 && s < N);
        if (gmode && !(c <= mu + chi)) keep = 0;
        if (!keep) {
            fac[k] = 0.0;
            cell[k] = -1;
            continue;
        }
        fac[k] = noise_mass(p, d, c - 0.5 * eta, c + 0.5 * eta, mu, xd);
        cell[k] = per ? (((s % N) + N) % N) : s;
    }
    return o;
}

typedef struct {
    int32_t W[ORC_MAXD];
    double xs[ORC_MAXD];
    int64_t wtot;
    int32_t wsum;
    int64_t stride[ORC_MAXD];
    int64_t nx, nu, nw; /* states, inputs, disturbance points (1 without a grid) */
} orc_shape;

static int shape_of(const orc_problem *p, orc_shape *sh) {
    if (p->n < 1 || p->n > ORC_MAXD || p->m < 1 || p->m > ORC_MAXD) return -1;
    if (p->p < 0 || p->p > ORC_MAXD) return -1;
    if (orc_window_shape(p, sh->W, sh->xs) != 0) return -1;
    sh->wtot = prod_i32(sh->W, p->n);
    sh->wsum = 0;
    for (int d = 0; d < p->n; ++d) sh->wsum += sh->W[d];
    sh->nx = prod_i32(p->x_count, p->n);
    sh->nu = prod_i32(p->u_count, p->m);
    sh->nw = p->p > 0 ? prod_i32(p->w_count, p->p) : 1;
    if (sh->nw < 1) return -1;
    int64_t st = 1;
    for (int d = p->n - 1; d >= 0; --d) {
        sh->stride[d] = st;
        st *= p->x_count[d];
    }
    if (p->sys_kind == ORC_SYS_AFFINE_PER_INPUT &&
        p->n_params != sh->nu * sh->nw * (int64_t)(p->n * p->n + p->n))
        return -1;
    if (p->sys_kind == ORC_SYS_UNICYCLE && (p->n != 3 || p->m != 2 || p->n_params < 1 || p->p != 0)) return -1;
    if (p->sys_kind == ORC_SYS_EXPR && !p->expr) return -1;
    if (p->noise == ORC_NOISE_MULT_GAUSSIAN && p->window == NULL && p->gamma != 0.0) return -1;
    return 0;
}

/* Per-dimension factors for one (x,u) pair; fac/cell hold sum_d W[d] entries. */
static int pair_factors(const orc_problem *p, const orc_shape *sh, int64_t x, int64_t u,
                        int32_t *origin, double *fac, int64_t *cell) {
    double mu[ORC_MAXD];
    if (orc_mean(p, x, u, mu) != 0) return -1;
    int32_t xi[ORC_MAXD];
    decode(x, p->x_count, p->n, xi);
    int off = 0;
    for (int d = 0; d < p->n; ++d) {
        const double xd = p->x_lb[d] + (double)xi[d] * p->x_eta[d];
        int32_t o = dim_window(p, d, sh->W[d], mu[d], xd, fac + off, cell + off);
        if (origin) origin[d] = o;
        off += sh->W[d];
    }
    return 0;
}

int orc_row(const orc_problem *p, int64_t x, int64_t u, int32_t *origin, double *probs) {
    orc_shape sh;
    if (shape_of(p, &sh) != 0) return -1;
    if (x < 0 || x >= sh.nx || u < 0 || u >= sh.nu * sh.nw) return -1;
    double *fac = (double *)malloc(sizeof(double) * sh.wsum);
    int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * sh.wsum);
    if (!fac || !cell || pair_factors(p, &sh, x, u, origin, fac, cell) != 0) {
        free(fac);
        free(cell);
        return -1;
    }
    int32_t k[ORC_MAXD] = {0};
    for (int64_t t = 0; t < sh.wtot; ++t) {
        double v = 1.0;
        int off = 0;
        for (int d = 0; d < p->n; ++d) {
            v = v * fac[off + k[d]];
            off += sh.W[d];
        }
        probs[t] = v;
        for (int d = p->n - 1; d >= 0; --d) {
            if (++k[d] < sh.W[d]) break;
            k[d] = 0;
        }
    }
    free(fac);
    free(cell);
    return 0;
}

static int in_box(const double *c, const double *lb, const double *ub, int n) {
    for (int d = 0; d < n; ++d)
        if (!(lb[d] <= c[d] && c[d] <= ub[d])) return 0;
    return 1;
}

/* Spec sets of Algorithm 3 evaluated on representative points (closed boxes). */
int orc_spec_mask(const orc_problem *p, const orc_spec *s, uint8_t *mask) {
    orc_shape sh;
    if (shape_of(p, &sh) != 0) return -1;
    const int n = p->n;
    for (int64_t x = 0; x < sh.nx; ++x) {
        int32_t xi[ORC_MAXD];
        double c[ORC_MAXD];
        decode(x, p->x_count, n, xi);
        for (int d = 0; d < n; ++d) c[d] = p->x_lb[d] + (double)xi[d] * p->x_eta[d];
        uint8_t f = 0;
        for (int b = 0; b < s->n_target; ++b)
            if (in_box(c, s->target_lb + b * n, s->target_ub + b * n, n)) f |= 1;
        for (int b = 0; b < s->n_avoid; ++b)
            if (in_box(c, s->avoid_lb + b * n, s->avoid_ub + b * n, n)) f |= 2;
        if (s->kind == ORC_SAFETY) {
            if (in_box(c, s->safe_lb, s->safe_ub, n)) f |= 4;
        } else {
            f |= 4;
        }
        if ((f & 3) == 3) return -1; /* target and avoid share a state */
        mask[x] = f;
    }
    return 0;
}

/* V_in of Algorithm 4 for one state and one (input, disturbance) pair index:
 * the sum over the cutting window of T(x'|x,u,w) * V_next[x'], in increasing
 * window (C) order. */
static double window_sum(const orc_problem *p, const orc_shape *sh, int64_t x, int64_t pair, const double *Vn,
                         double *fac, int64_t *cell) {
    const int n = p->n;
    pair_factors(p, sh, x, pair, NULL, fac, cell);
    int32_t k[ORC_MAXD] = {0};
    double acc = 0.0;
    for (int64_t t = 0; t < sh->wtot; ++t) {
        double w = 1.0;
        int64_t lin = 0;
        int off = 0, drop = 0;
        for (int d = 0; d < n; ++d) {
            int64_t cidx = cell[off + k[d]];
            if (cidx < 0) {
                drop = 1;
                break;
            }
            w = w * fac[off + k[d]];
            lin += cidx * sh->stride[d];
            off += sh->W[d];
        }
        if (!drop) acc += w * Vn[lin];
        for (int d = n - 1; d >= 0; --d) {
            if (++k[d] < sh->W[d]) break;
            k[d] = 0;
        }
    }
    return acc;
}

/* The value the input u secures at x: the worst case over the disturbance
 * grid, min_w V_in(x, u, w) (Algorithm 3's "minimize with respect to W",
 * Algorithm 4's inner min); V_in itself without a disturbance grid. */
static double input_value(const orc_problem *p, const orc_shape *sh, int64_t x, int64_t u, const double *Vn,
                          double *fac, int64_t *cell) {
    double mn = INFINITY;
    for (int64_t w = 0; w < sh->nw; ++w) {
        const double v = window_sum(p, sh, x, u * sh->nw + w, Vn, fac, cell);
        if (v < mn) mn = v;
    }
    return mn;
}

/* The collect step of Algorithm 4 for one state: the value of every input,
 * then the max over inputs with the lowest maximising index. */
static void backup_one(const orc_problem *p, const orc_shape *sh, const orc_spec *s,
                       uint8_t f, const double *Vn, int64_t x, double *fac, int64_t *cell,
                       double *V, uint16_t *pi, double *gap) {
    int masked;
    double mval;
    if (s->kind == ORC_SAFETY) {
        masked = !(f & 4);
        mval = 0.0;
    } else {
        masked = (f & 3) != 0;
        mval = (f & 1) ? 1.0 : 0.0;
    }
    if (masked) {
        *V = mval;
        *pi = 0xFFFF;
        *gap = INFINITY;
        return;
    }
    double best = -INFINITY, best2 = -INFINITY;
    int64_t arg = 0;
    for (int64_t u = 0; u < sh->nu; ++u) {
        const double acc = input_value(p, sh, x, u, Vn, fac, cell);
        if (acc > best) {
            best2 = best;
            best = acc;
            arg = u;
        } else if (acc > best2) {
            best2 = acc;
        }
    }
    *V = best;
    *pi = (uint16_t)arg;
    *gap = (sh->nu > 1) ? best - best2 : INFINITY;
}

/* The action values of Algorithm 4 at one state (every input's value). */
int orc_action_values(const orc_problem *p, const double *V_next, int64_t x, double *out) {
    orc_shape sh;
    if (shape_of(p, &sh) != 0 || x < 0 || x >= sh.nx) return -1;
    double *fac = (double *)malloc(sizeof(double) * sh.wsum);
    int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * sh.wsum);
    if (!fac || !cell) {
        free(fac);
        free(cell);
        return -1;
    }
    for (int64_t u = 0; u < sh.nu; ++u) out[u] = input_value(p, &sh, x, u, V_next, fac, cell);
    free(fac);
    free(cell);
    return 0;
}

int orc_backup_states(const orc_problem *p, const orc_spec *s, const double *V_next,
                      const int64_t *states, int64_t n_states, double *V_out,
                      uint16_t *pi_out, double *gap_out, int nthreads) {
    orc_shape sh;
    if (shape_of(p, &sh) != 0 || sh.nu > 65535) return -1;
    uint8_t *mask = (uint8_t *)malloc((size_t)sh.nx);
    if (!mask) return -1;
    if (orc_spec_mask(p, s, mask) != 0) {
        free(mask);
        return -1;
    }
    int err = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        double *fac = (double *)malloc(sizeof(double) * sh.wsum);
        int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * sh.wsum);
        if (!fac || !cell) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            err = 1;
        }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t i = 0; i < n_states; ++i) {
            if (!fac || !cell) continue;
            int64_t x = states[i];
            if (x < 0 || x >= sh.nx) continue;
            double V, gap;
            uint16_t pi;
            backup_one(p, &sh, s, mask[x], V_next, x, fac, cell, &V, &pi, &gap);
            if (V_out) V_out[i] = V;
            if (pi_out) pi_out[i] = pi;
            if (gap_out) gap_out[i] = gap;
        }
        free(fac);
        free(cell);
    }
    free(mask);
    return err ? -1 : 0;
}

int orc_synthesize(const orc_problem *p, const orc_spec *s, int32_t horizon, double *V_out,
                   uint16_t *pi_out, double *gap_out, double *V_all, int nthreads) {
    orc_shape sh;
    if (horizon < 0 || shape_of(p, &sh) != 0 || sh.nu > 65535) return -1;
    const int64_t nx = sh.nx;
    uint8_t *mask = (uint8_t *)malloc((size_t)nx);
    double *Va = (double *)malloc(sizeof(double) * nx);
    double *Vb = (double *)malloc(sizeof(double) * nx);
    if (!mask || !Va || !Vb || orc_spec_mask(p, s, mask) != 0) {
        free(mask);
        free(Va);
        free(Vb);
        return -1;
    }
    /* V_N: indicator of the safe set (safety) or of the target (reach). */
    for (int64_t x = 0; x < nx; ++x)
        Va[x] = (s->kind == ORC_SAFETY) ? ((mask[x] & 4) ? 1.0 : 0.0) : ((mask[x] & 1) ? 1.0 : 0.0);
    if (V_all) memcpy(V_all + (int64_t)horizon * nx, Va, sizeof(double) * nx);
    int err = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#endif
    for (int32_t k = horizon - 1; k >= 0; --k) {
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
        {
            double *fac = (double *)malloc(sizeof(double) * sh.wsum);
            int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * sh.wsum);
            if (!fac || !cell) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
                err = 1;
            }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
            for (int64_t x = 0; x < nx; ++x) {
                if (!fac || !cell) continue;
                double V, gap;
                uint16_t pi;
                backup_one(p, &sh, s, mask[x], Va, x, fac, cell, &V, &pi, &gap);
                Vb[x] = V;
                if (pi_out) pi_out[(int64_t)k * nx + x] = pi;
                if (gap_out) gap_out[(int64_t)k * nx + x] = gap;
            }
            free(fac);
            free(cell);
        }
        double *t = Va;
        Va = Vb;
        Vb = t;
        if (V_all) memcpy(V_all + (int64_t)k * nx, Va, sizeof(double) * nx);
    }
    memcpy(V_out, Va, sizeof(double) * nx);
    free(mask);
    free(Va);
    free(Vb);
    return err ? -1 : 0;
}

/* ---------------------------------------------------------------------------
 * Closed-loop simulation (Sec. 7: the controller is validated by simulating
 * the closed loop from initial states; here on the finite MDP itself, so the
 * success frequency estimates V_0 exactly in expectation).
 * ------------------------------------------------------------------------- */

static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
    const unsigned __int128 p = (unsigned __int128)a * b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64(const uint64_t *ctr, const uint64_t *key, uint64_t *out) {
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(0xD2E7470EE14C6C93ull, c0, &hi0, &lo0);
        mulhilo64(0xCA5A826395121157ull, c2, &hi1, &lo1);
        const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Uniform double in [0, 1) of draw q at step t of run g. */
static double sim_draw(uint64_t g, int32_t t, int q, uint64_t seed) {
    const uint64_t ctr[4] = {g, (uint64_t)t, (uint64_t)(q / 4), 0};
    const uint64_t key[2] = {seed, 0};
    uint64_t w[4];
    orc_philox4x64(ctr, key, w);
    return (double)(w[q % 4] >> 11) * (1.0 / 9007199254740992.0);
}

/* Spec status of a state: 1 = the run has succeeded, 0 = failed, -1 = goes on
 * (safety: success only at the horizon). */
static int sim_status(const orc_spec *s, uint8_t f) {
    if (s->kind == ORC_SAFETY) return (f & 4) ? -1 : 0;
    if (f & 1) return 1;
    if (f & 2) return 0;
    return -1;
}

int orc_simulate(const orc_problem *p, const orc_spec *s, int32_t horizon, const uint16_t *policy,
                 const int64_t *x0, int64_t n_x0, int64_t runs, uint64_t seed, int64_t *successes) {
    orc_shape sh;
    if (horizon < 0 || runs < 0 || shape_of(p, &sh) != 0) return -1;
    uint8_t *mask = (uint8_t *)malloc((size_t)sh.nx);
    if (!mask) return -1;
    if (orc_spec_mask(p, s, mask) != 0) {
        free(mask);
        return -1;
    }
    for (int64_t i = 0; i < n_x0; ++i)
        if (x0[i] < 0 || x0[i] >= sh.nx) {
            free(mask);
            return -1;
        }
    int rc = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n_x0; ++i) {
        double *fac = (double *)malloc(sizeof(double) * sh.wsum);
        int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * sh.wsum);
        int32_t origin[ORC_MAXD];
        int64_t wins = 0;
        if (!fac || !cell) {
#pragma omp atomic write
            rc = -1;
        } else {
            for (int64_t r = 0; r < runs; ++r) {
                const uint64_t g = (uint64_t)(i * runs + r);
                int64_t x = x0[i];
                int st = sim_status(s, mask[x]);
                for (int32_t t = 0; t < horizon && st < 0; ++t) {
                    const int64_t u = policy[(int64_t)t * sh.nx + x];
                    int64_t w = 0;
                    if (sh.nw > 1) {
                        w = (int64_t)(sim_draw(g, t, p->n, seed) * (double)sh.nw);
                        if (w >= sh.nw) w = sh.nw - 1;
                    }
                    pair_factors(p, &sh, x, u * sh.nw + w, origin, fac, cell);
                    int64_t nxt = 0;
                    int lost = 0, off = 0;
                    for (int d = 0; d < p->n && !lost; ++d) {
                        const double q = sim_draw(g, t, d, seed);
                        double cum = 0.0;
                        int64_t pick = -1;
                        for (int k = 0; k < sh.W[d]; ++k) {
                            cum += fac[off + k];
                            if (q < cum) {
                                pick = cell[off + k];
                                break;
                            }
                        }
                        if (pick < 0) lost = 1;
                        else nxt += pick * sh.stride[d];
                        off += sh.W[d];
                    }
                    if (lost) {
                        st = 0;
                        break;
                    }
                    x = nxt;
                    st = sim_status(s, mask[x]);
                }
                if (st < 0) st = (s->kind == ORC_SAFETY) ? 1 : 0;
                wins += st;
            }
        }
        successes[i] = wins;
        free(fac);
        free(cell);
    }
    free(mask);
    return rc;
}
