/*
 * amy_oracle_expr.c -- the oracle's reading of a system given as text
 * (TEST INFRASTRUCTURE ONLY; part of liboracle.so, shares nothing with the
 * CUDA library).
 *
 * Sec. 3 of the paper has the user supply the right-hand side of the
 * difference equation x(k+1) = f(x(k), nu(k), w(k)) + noise as text in a
 * configuration file.  Here each mean component f_d is one arithmetic
 * expression in C syntax over the FP64 variables
 *   x0 .. x{n-1}   the state's representative point (grid centre),
 *   u0 .. u{m-1}   the input's representative point,
 *   w0 .. w{p-1}   the disturbance's representative point,
 *   p0 .. p{k-1}   the system's parameters,
 * with numeric literals (always doubles), unary + and -, the binary + - * /
 * (left associative, * and / binding tighter), parentheses and the calls
 *   sin cos tan asin acos atan sinh cosh tanh exp log log10 sqrt fabs floor
 *   ceil (one argument), atan2 pow fmin fmax (two arguments).
 * The oracle parses each expression once into postfix form and evaluates it
 * with a value stack: every operation is one IEEE FP64 operation (the library
 * is built without fused multiply-add), the calls are the C library's.
 */
#include <ctype.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "amy_oracle.h"

enum {
    OP_CONST, OP_X, OP_U, OP_W, OP_P, OP_NEG, OP_ADD, OP_SUB, OP_MUL, OP_DIV, OP_CALL1, OP_CALL2
};

typedef struct {
    int op;
    int arg;
    double val;
} orc_op;

typedef struct {
    orc_op *ops;
    int len, cap;
} orc_prog;

struct orc_expr {
    int n;
    orc_prog prog[ORC_MAXD];
};

static const char *const kFun1[] = {"sin", "cos", "tan", "asin", "acos", "atan", "sinh", "cosh",
                                    "tanh", "exp", "log", "log10", "sqrt", "fabs", "floor", "ceil"};
static const char *const kFun2[] = {"atan2", "pow", "fmin", "fmax"};
#define N_FUN1 ((int)(sizeof kFun1 / sizeof kFun1[0]))
#define N_FUN2 ((int)(sizeof kFun2 / sizeof kFun2[0]))

static double call1(int f, double a) {
    switch (f) {
    case 0: return sin(a);
    case 1: return cos(a);
    case 2: return tan(a);
    case 3: return asin(a);
    case 4: return acos(a);
    case 5: return atan(a);
    case 6: return sinh(a);
    case 7: return cosh(a);
    case 8: return tanh(a);
    case 9: return exp(a);
    case 10: return log(a);
    case 11: return log10(a);
    case 12: return sqrt(a);
    case 13: return fabs(a);
    case 14: return floor(a);
    default: return ceil(a);
    }
}

static double call2(int f, double a, double b) {
    switch (f) {
    case 0: return atan2(a, b);
    case 1: return pow(a, b);
    case 2: return fmin(a, b);
    default: return fmax(a, b);
    }
}

/* ---- recursive-descent parser ------------------------------------------ */

typedef struct {
    const char *s;
    size_t pos;
    int pdf; /* a density: the one variable t (read as x0) */
    int m, p, depth;
    int64_t n_params;
    int n;
    orc_prog *out;
    char *err;
    int errlen;
    int failed;
} parser;

static void fail(parser *ps, const char *what) {
    if (!ps->failed && ps->err && ps->errlen > 0)
        snprintf(ps->err, (size_t)ps->errlen, "%s at offset %zu", what, ps->pos);
    ps->failed = 1;
}

static void emit(parser *ps, int op, int arg, double val) {
    if (ps->failed) return;
    orc_prog *pr = ps->out;
    if (pr->len == pr->cap) {
        int cap = pr->cap ? 2 * pr->cap : 16;
        orc_op *nops = (orc_op *)realloc(pr->ops, sizeof(orc_op) * (size_t)cap);
        if (!nops) {
            fail(ps, "out of memory");
            return;
        }
        pr->ops = nops;
        pr->cap = cap;
    }
    pr->ops[pr->len].op = op;
    pr->ops[pr->len].arg = arg;
    pr->ops[pr->len].val = val;
    pr->len++;
}

static void skip_ws(parser *ps) {
    while (isspace((unsigned char)ps->s[ps->pos])) ps->pos++;
}

static void parse_sum(parser *ps);

static void parse_primary(parser *ps) {
    skip_ws(ps);
    const char *s = ps->s;
    const char c = s[ps->pos];
    if (c == '(') {
        ps->pos++;
        parse_sum(ps);
        skip_ws(ps);
        if (s[ps->pos] != ')') {
            fail(ps, "expected ')'");
            return;
        }
        ps->pos++;
        return;
    }
    if (isdigit((unsigned char)c) || c == '.') {
        /* digits [. digits] [(e|E) [+-] digits], or . digits */
        size_t q = ps->pos;
        int mant = 0;
        while (isdigit((unsigned char)s[q])) q++, mant = 1;
        if (s[q] == '.') {
            q++;
            while (isdigit((unsigned char)s[q])) q++, mant = 1;
        }
        if (!mant) {
            fail(ps, "malformed number");
            return;
        }
        if (s[q] == 'e' || s[q] == 'E') {
            size_t r = q + 1;
            if (s[r] == '+' || s[r] == '-') r++;
            if (!isdigit((unsigned char)s[r])) {
                fail(ps, "malformed exponent");
                return;
            }
            while (isdigit((unsigned char)s[r])) r++;
            q = r;
        }
        if (isalpha((unsigned char)s[q]) || s[q] == '_') {
            fail(ps, "malformed number");
            return;
        }
        char buf[128];
        const size_t len = q - ps->pos;
        if (len >= sizeof buf) {
            fail(ps, "number too long");
            return;
        }
        memcpy(buf, s + ps->pos, len);
        buf[len] = '\0';
        emit(ps, OP_CONST, 0, strtod(buf, NULL));
        ps->pos = q;
        return;
    }
    if (isalpha((unsigned char)c) || c == '_') {
        size_t q = ps->pos;
        while (isalnum((unsigned char)s[q]) || s[q] == '_') q++;
        char name[32];
        const size_t len = q - ps->pos;
        if (len >= sizeof name) {
            fail(ps, "identifier too long");
            return;
        }
        memcpy(name, s + ps->pos, len);
        name[len] = '\0';
        ps->pos = q;
        skip_ws(ps);
        if (s[ps->pos] == '(') {
            ps->pos++;
            int f1 = -1, f2 = -1;
            for (int i = 0; i < N_FUN1; ++i)
                if (strcmp(name, kFun1[i]) == 0) f1 = i;
            for (int i = 0; i < N_FUN2; ++i)
                if (strcmp(name, kFun2[i]) == 0) f2 = i;
            if (f1 < 0 && f2 < 0) {
                fail(ps, "unknown function");
                return;
            }
            parse_sum(ps);
            skip_ws(ps);
            if (f2 >= 0) {
                if (s[ps->pos] != ',') {
                    fail(ps, "expected ',' (two-argument function)");
                    return;
                }
                ps->pos++;
                parse_sum(ps);
                skip_ws(ps);
            }
            if (s[ps->pos] != ')') {
                fail(ps, "expected ')' after the arguments");
                return;
            }
            ps->pos++;
            if (f2 >= 0) emit(ps, OP_CALL2, f2, 0.0);
            else emit(ps, OP_CALL1, f1, 0.0);
            return;
        }
        if (ps->pdf) {
            if (strcmp(name, "t") != 0) {
                fail(ps, "unknown identifier (a density reads t only)");
                return;
            }
            emit(ps, OP_X, 0, 0.0);
            return;
        }
        /* a variable: one letter then a decimal index without leading zeros */
        const char kind = name[0];
        const char *digits = name + 1;
        int ok = (kind == 'x' || kind == 'u' || kind == 'w' || kind == 'p') && digits[0] != '\0';
        for (const char *d = digits; ok && *d; ++d) ok = isdigit((unsigned char)*d);
        if (ok && digits[0] == '0' && digits[1] != '\0') ok = 0;
        if (!ok || strlen(digits) > 6) {
            fail(ps, "unknown identifier");
            return;
        }
        const long idx = strtol(digits, NULL, 10);
        const long lim = kind == 'x' ? ps->n : kind == 'u' ? ps->m : kind == 'w' ? ps->p : (long)ps->n_params;
        if (idx >= lim) {
            fail(ps, "variable index out of range");
            return;
        }
        emit(ps, kind == 'x' ? OP_X : kind == 'u' ? OP_U : kind == 'w' ? OP_W : OP_P, (int)idx, 0.0);
        return;
    }
    fail(ps, c ? "unexpected character" : "unexpected end of expression");
}

static void parse_unary(parser *ps) {
    if (++ps->depth > 256) {
        fail(ps, "expression nested too deeply");
        return;
    }
    skip_ws(ps);
    const char c = ps->s[ps->pos];
    if (c == '-') {
        ps->pos++;
        parse_unary(ps);
        emit(ps, OP_NEG, 0, 0.0);
    } else if (c == '+') {
        ps->pos++;
        parse_unary(ps);
    } else {
        parse_primary(ps);
    }
    ps->depth--;
}

static void parse_product(parser *ps) {
    parse_unary(ps);
    for (;;) {
        if (ps->failed) return;
        skip_ws(ps);
        const char c = ps->s[ps->pos];
        if (c != '*' && c != '/') return;
        ps->pos++;
        parse_unary(ps);
        emit(ps, c == '*' ? OP_MUL : OP_DIV, 0, 0.0);
    }
}

static void parse_sum(parser *ps) {
    if (++ps->depth > 256) {
        fail(ps, "expression nested too deeply");
        return;
    }
    parse_product(ps);
    for (;;) {
        if (ps->failed) break;
        skip_ws(ps);
        const char c = ps->s[ps->pos];
        if (c != '+' && c != '-') break;
        ps->pos++;
        parse_product(ps);
        emit(ps, c == '+' ? OP_ADD : OP_SUB, 0, 0.0);
    }
    ps->depth--;
}

void orc_expr_free(orc_expr *e) {
    if (!e) return;
    for (int d = 0; d < ORC_MAXD; ++d) free(e->prog[d].ops);
    free(e);
}

static orc_expr *compile_any(const char *const *text, int n, int m, int p, int64_t n_params, int pdf, char *err,
                             int errlen) {
    if (err && errlen > 0) err[0] = '\0';
    if (!text || n < 1 || n > ORC_MAXD || m < 0 || p < 0) {
        if (err && errlen > 0) snprintf(err, (size_t)errlen, "bad arguments");
        return NULL;
    }
    orc_expr *e = (orc_expr *)calloc(1, sizeof(orc_expr));
    if (!e) return NULL;
    e->n = n;
    for (int d = 0; d < n; ++d) {
        parser ps;
        memset(&ps, 0, sizeof ps);
        ps.s = text[d] ? text[d] : "";
        ps.n = n;
        ps.m = m;
        ps.p = p;
        ps.n_params = n_params;
        ps.pdf = pdf;
        ps.out = &e->prog[d];
        ps.err = err;
        ps.errlen = errlen;
        parse_sum(&ps);
        skip_ws(&ps);
        if (!ps.failed && ps.s[ps.pos] != '\0') fail(&ps, "trailing characters");
        if (ps.failed) {
            if (err && errlen > 0) {
                char tmp[256];
                snprintf(tmp, sizeof tmp, "component %d: %s", d, err);
                snprintf(err, (size_t)errlen, "%s", tmp);
            }
            orc_expr_free(e);
            return NULL;
        }
    }
    return e;
}

orc_expr *orc_expr_compile(const char *const *text, int n, int m, int p, int64_t n_params, char *err, int errlen) {
    return compile_any(text, n, m, p, n_params, 0, err, errlen);
}

orc_expr *orc_expr_compile_pdf(const char *const *text, int n, char *err, int errlen) {
    return compile_any(text, n, 0, 0, 0, 1, err, errlen);
}

double orc_expr_eval(const orc_expr *e, int d, const double *x, const double *u, const double *w,
                     const double *params) {
    const orc_prog *pr = &e->prog[d];
    double stackbuf[64];
    double *st = pr->len <= 64 ? stackbuf : (double *)malloc(sizeof(double) * (size_t)pr->len);
    if (!st) return NAN;
    int top = 0;
    for (int i = 0; i < pr->len; ++i) {
        const orc_op *o = &pr->ops[i];
        switch (o->op) {
        case OP_CONST: st[top++] = o->val; break;
        case OP_X: st[top++] = x[o->arg]; break;
        case OP_U: st[top++] = u[o->arg]; break;
        case OP_W: st[top++] = w[o->arg]; break;
        case OP_P: st[top++] = params[o->arg]; break;
        case OP_NEG: st[top - 1] = -st[top - 1]; break;
        case OP_ADD: top--; st[top - 1] = st[top - 1] + st[top]; break;
        case OP_SUB: top--; st[top - 1] = st[top - 1] - st[top]; break;
        case OP_MUL: top--; st[top - 1] = st[top - 1] * st[top]; break;
        case OP_DIV: top--; st[top - 1] = st[top - 1] / st[top]; break;
        case OP_CALL1: st[top - 1] = call1(o->arg, st[top - 1]); break;
        default: top--; st[top - 1] = call2(o->arg, st[top - 1], st[top]); break;
        }
    }
    const double r = top == 1 ? st[0] : NAN;
    if (st != stackbuf) free(st);
    return r;
}

/* ---- user densities (Sec. 6.2: the user gives the density and a box
 * enclosing its support) ----------------------------------------------------
 * The density of dim d is integrated over [lo, hi] once: at the M + 1 knots
 * t_i = lo + i h (h = (hi - lo) / M; t_M = hi) its values f_i, and per interval the
 * 8-point Gauss-Legendre rule, the interval sums added in order into the
 * cumulative C_i; F_i = C_i / C_M and f_i / C_M normalise the density to
 * one.  The CDF between knots is the cubic Hermite interpolant of (F_i, f_i),
 * exact for CDFs of degree 3 and of error O(h^4) otherwise. */
static const double kGLx[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
static const double kGLw[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};

double orc_gauss_legendre8(const orc_expr *pdf, int d, double a, double b) {
    const double c = 0.5 * (a + b), r = 0.5 * (b - a);
    double sum = 0.0;
    for (int q = 3; q >= 0; --q) {
        const double t = c - r * kGLx[q];
        sum = sum + kGLw[q] * orc_expr_eval(pdf, d, &t, NULL, NULL, NULL);
    }
    for (int q = 0; q < 4; ++q) {
        const double t = c + r * kGLx[q];
        sum = sum + kGLw[q] * orc_expr_eval(pdf, d, &t, NULL, NULL, NULL);
    }
    return r * sum;
}

int orc_user_table(const orc_expr *pdf, int d, double lo, double hi, double *table) {
    const int M = ORC_USER_KNOTS;
    if (!(hi > lo)) return -1;
    const double h = (hi - lo) / (double)M;
    double *F = table, *f = table + (M + 1);
    F[0] = 0.0;
    /* knot i at lo + i h, the last one at hi exactly */
    for (int i = 0; i < M; ++i) {
        const double a = lo + (double)i * h, b = i + 1 == M ? hi : lo + (double)(i + 1) * h;
        F[i + 1] = F[i] + orc_gauss_legendre8(pdf, d, a, b);
    }
    const double Z = F[M];
    if (!(Z > 0.0) || !isfinite(Z)) return -1;
    for (int i = 0; i <= M; ++i) {
        const double t = i == M ? hi : lo + (double)i * h;
        F[i] = F[i] / Z;
        f[i] = orc_expr_eval(pdf, d, &t, NULL, NULL, NULL) / Z;
        if (!(f[i] >= 0.0) || !isfinite(f[i])) return -1;
    }
    return 0;
}

double orc_user_cdf(const double *table, double lo, double hi, double t) {
    const int M = ORC_USER_KNOTS;
    if (t <= lo) return 0.0;
    if (t >= hi) return 1.0;
    const double h = (hi - lo) / (double)M;
    const double s = (t - lo) / h;
    int i = (int)floor(s);
    if (i > M - 1) i = M - 1;
    const double tau = s - (double)i, tau2 = tau * tau, tau3 = tau2 * tau;
    const double h00 = 2.0 * tau3 - 3.0 * tau2 + 1.0, h10 = tau3 - 2.0 * tau2 + tau;
    const double h01 = -2.0 * tau3 + 3.0 * tau2, h11 = tau3 - tau2;
    const double *F = table, *f = table + (M + 1);
    return h00 * F[i] + h10 * h * f[i] + h01 * F[i + 1] + h11 * h * f[i + 1];
}
