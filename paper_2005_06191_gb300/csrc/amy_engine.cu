// amy_engine.cu -- C ABI of the single-problem path (amy_build,
// amy_synthesize, amy_backup_step, amy_query_rows, amy_info, amy_destroy).
//
// Host side: validation, window shape (Sec. 5.2 Remark, scalars per dim),
// device allocation and kernel launches.  Every per-state and per-pair step
// runs in the kernels of amy_kernels.cuh.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/amy.h"
#include "amy_internal.h"
#include "amy_kernels.cuh"

using namespace amy;

namespace amy {

static thread_local std::string g_last_error;

amy_status set_error(amy_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

amy_status cuda_error(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_error(AMY_E_OUT_OF_MEMORY, "%s: %s", what, cudaGetErrorString(e));
    }
    return set_error(AMY_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

amy_status smem_optin(const void *func, int bytes, std::atomic<uint64_t> &done, const char *what) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, what);
    const uint64_t bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return AMY_OK;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return cuda_error(e, what);
    done.fetch_or(bit, std::memory_order_acq_rel);
    return AMY_OK;
}

int64_t grid_count(double lb, double ub, double eta) {
    return (int64_t)std::floor((ub - lb) / eta + 1e-9) + 1;
}

// Window shape per dim (Sec. 5.2 and the Remark on the cutting region): the
// 1-D density of N(0, sigma^2) equals gamma at +-xs; the row keeps
// floor(2 xs / eta) + 1 slots.  Same FP64 expression as documented in amy.h.
// Validation and geometry only, with no heap use (amy_synthesize_noalloc
// calls it directly; make_geom adds the host copy of the parameters).
amy_status fill_geom(const amy_system *sys, const amy_grid *st, const amy_grid *in, const double *sigma,
                     const amy_cut *cut, Geom &g) {
    if (!sys || !st || !in || !sigma || !cut) return set_error(AMY_E_INVALID_ARG, "null argument");
    const int n = st->n, m = in->n;
    if (n < 1 || n > MAXD || m < 1 || m > MAXD) return set_error(AMY_E_INVALID_ARG, "dims must be 1..8");
    if (sys->n != n || sys->m != m) return set_error(AMY_E_INVALID_ARG, "system dims differ from grids");
    if (!st->lb || !st->eta || !st->count || !in->lb || !in->eta || !in->count)
        return set_error(AMY_E_INVALID_ARG, "null grid array");
    memset(&g, 0, sizeof g);
    g.n = n;
    g.m = m;
    int64_t nx = 1, nu = 1;
    // noise distribution (Gaussian unless sys->noise says otherwise)
    const amy_noise *nz = sys->noise;
    g.noise = nz ? nz->kind : NOISE_GAUSSIAN;
    if (g.noise < NOISE_GAUSSIAN || g.noise > NOISE_USER)
        return set_error(AMY_E_INVALID_ARG, "unknown noise kind %d", g.noise);
    if (g.noise == NOISE_USER && !nz->pdf) return set_error(AMY_E_INVALID_ARG, "user noise needs its densities");
    for (int d = 0; d < n; ++d) {
        const double *pp[4] = {nz ? nz->p0 : nullptr, nz ? nz->p1 : nullptr, nz ? nz->p2 : nullptr,
                               nz ? nz->p3 : nullptr};
        const int need = g.noise == NOISE_GAUSSIAN ? 0 : g.noise == NOISE_BETA ? 4 : g.noise == NOISE_USER ? 2 : 1;
        for (int i = 0; i < 4; ++i) {
            if (i < need && !pp[i]) return set_error(AMY_E_INVALID_ARG, "noise kind %d needs %d parameter arrays", g.noise, need);
            g.np[i][d] = i < need ? pp[i][d] : 0.0;
            if (!std::isfinite(g.np[i][d])) return set_error(AMY_E_INVALID_ARG, "non-finite noise parameter");
        }
        if (g.noise == NOISE_UNIFORM || g.noise == NOISE_EXPONENTIAL || g.noise == NOISE_MULT_GAUSSIAN) {
            if (!(g.np[0][d] > 0.0)) return set_error(AMY_E_INVALID_ARG, "noise parameter p0[%d] must be positive", d);
        } else if (g.noise == NOISE_BETA) {
            const double a = g.np[0][d], b = g.np[1][d];
            if (!(a >= 1.0 && b >= 1.0 && a == std::floor(a) && b == std::floor(b) && a + b <= 64.0))
                return set_error(AMY_E_INVALID_ARG, "beta noise needs integer shapes >= 1 summing to at most 64 (dim %d)", d);
            if (!(g.np[3][d] > g.np[2][d])) return set_error(AMY_E_INVALID_ARG, "beta noise needs lo < hi (dim %d)", d);
        } else if (g.noise == NOISE_USER) {
            if (!(g.np[1][d] > g.np[0][d]))
                return set_error(AMY_E_INVALID_ARG, "user noise needs a support box lo < hi (dim %d)", d);
        }
    }
    for (int d = 0; d < n; ++d) {
        if (st->count[d] < 1 || !(st->eta[d] > 0.0) || !std::isfinite(st->lb[d]) || !std::isfinite(st->eta[d]))
            return set_error(AMY_E_INVALID_ARG, "bad state grid in dim %d", d);
        if (g.noise == NOISE_GAUSSIAN && (!(sigma[d] > 0.0) || !std::isfinite(sigma[d])))
            return set_error(AMY_E_INVALID_ARG, "sigma[%d] must be positive", d);
        g.N[d] = st->count[d];
        g.lb[d] = st->lb[d];
        g.eta[d] = st->eta[d];
        if (st->periodic && st->periodic[d]) g.periodic |= 1u << d;
        nx *= st->count[d];
        if (nx > 2147483647LL) return set_error(AMY_E_INVALID_ARG, "more than 2^31-1 states");
    }
    for (int d = 0; d < m; ++d) {
        if (in->count[d] < 1 || !(in->eta[d] > 0.0)) return set_error(AMY_E_INVALID_ARG, "bad input grid in dim %d", d);
        g.ucount[d] = in->count[d];
        g.ulb[d] = in->lb[d];
        g.ueta[d] = in->eta[d];
        nu *= in->count[d];
        if (nu > 65535) return set_error(AMY_E_INVALID_ARG, "more than 65535 inputs");
    }
    // disturbance grid (Sec. 3): its dims follow the input dims, so that the
    // (input, disturbance) pairs are enumerated in C order with the
    // disturbance fastest -- pair index u * nw + w
    int64_t nw = 1;
    const amy_grid *dg = sys->disturb;
    if (dg && dg->n > 0) {
        if (sys->kind != AMY_SYS_AFFINE_PER_INPUT && sys->kind != AMY_SYS_EXPR)
            return set_error(AMY_E_UNSUPPORTED, "a disturbance grid needs the affine or the text system kind");
        if (m + dg->n > MAXD) return set_error(AMY_E_INVALID_ARG, "input and disturbance dims must total at most 8");
        if (!dg->lb || !dg->eta || !dg->count) return set_error(AMY_E_INVALID_ARG, "null disturbance grid array");
        for (int d = 0; d < dg->n; ++d) {
            if (dg->count[d] < 1 || !(dg->eta[d] > 0.0) || !std::isfinite(dg->lb[d]))
                return set_error(AMY_E_INVALID_ARG, "bad disturbance grid in dim %d", d);
            g.ucount[m + d] = dg->count[d];
            g.ulb[m + d] = dg->lb[d];
            g.ueta[m + d] = dg->eta[d];
            nw *= dg->count[d];
            if (nu * nw > (1 << 24)) return set_error(AMY_E_INVALID_ARG, "more than 2^24 input-disturbance pairs");
        }
        g.m = m + dg->n;
    }
    g.nx = (int32_t)nx;
    g.nu = (int32_t)(nu * nw);
    g.nw = (int32_t)nw;
    int64_t s = 1;
    for (int d = n - 1; d >= 0; --d) {
        g.stride[d] = (int32_t)s;
        s *= g.N[d];
    }
    // system
    if (sys->kind == AMY_SYS_AFFINE_PER_INPUT) {
        if (!sys->params || sys->n_params != nu * nw * (int64_t)(n * n + n))
            return set_error(AMY_E_INVALID_ARG, "affine system needs n_u*n_w*(n*n+n) params");
        g.sys = SYS_AFFINE;
    } else if (sys->kind == AMY_SYS_UNICYCLE) {
        if (n != 3 || m != 2 || !sys->params || sys->n_params < 1)
            return set_error(AMY_E_INVALID_ARG, "unicycle needs n=3, m=2, params={tau}");
        g.sys = SYS_UNICYCLE;
    } else if (sys->kind == AMY_SYS_EXPR) {
        if (!sys->expr) return set_error(AMY_E_INVALID_ARG, "text system needs one expression per state dim");
        if (sys->n_params < 0 || (sys->n_params > 0 && !sys->params))
            return set_error(AMY_E_INVALID_ARG, "text system: bad parameter array");
        g.sys = SYS_EXPR;
    } else {
        return set_error(AMY_E_INVALID_ARG, "unknown system kind %d", sys->kind);
    }
    for (int64_t i = 0; i < sys->n_params; ++i)
        if (!std::isfinite(sys->params[i])) return set_error(AMY_E_INVALID_ARG, "non-finite system parameter");
    // window
    int64_t wtot = 1;
    int32_t wsum = 0;
    for (int d = 0; d < n; ++d) {
        const bool per = (g.periodic >> d) & 1u;
        if (g.noise == NOISE_GAUSSIAN) {
            g.k2[d] = sigma[d] * std::sqrt(2.0);
            g.rk2f[d] = (float)(1.0 / (sigma[d] * std::sqrt(2.0)));
        }
        if (cut->window) {
            g.wmode = WM_EXPLICIT;
            const int32_t W = cut->window[d];
            if (W < 1 || (W % 2) == 0) return set_error(AMY_E_INVALID_ARG, "explicit window must be odd (dim %d)", d);
            if (per && W > g.N[d]) return set_error(AMY_E_INVALID_ARG, "window wider than periodic dim %d", d);
            g.W[d] = W;
            g.xs[d] = INFINITY;
        } else if (cut->gamma == 0.0) {
            g.wmode = WM_DENSE;
            if (per) return set_error(AMY_E_INVALID_ARG, "dense rows need non-periodic dims");
            g.W[d] = g.N[d];
            g.xs[d] = INFINITY;
        } else {
            g.wmode = WM_GAMMA;
            if (!(cut->gamma > 0.0) || !std::isfinite(cut->gamma)) return set_error(AMY_E_INVALID_ARG, "bad gamma");
            // the cut interval [clo, chi] of the noise around the mean
            double clo = 0.0, chi = 0.0;
            if (g.noise == NOISE_GAUSSIAN) {
                const double arg = 1.0 / (cut->gamma * sigma[d] * std::sqrt(2.0 * M_PI));
                if (!(arg > 1.0)) return set_error(AMY_E_INVALID_ARG, "gamma at or above the peak density (dim %d)", d);
                const double xs = sigma[d] * std::sqrt(2.0 * std::log(arg));
                clo = -xs;
                chi = xs;
            } else if (g.noise == NOISE_UNIFORM) {
                const double a = g.np[0][d];
                if (!(cut->gamma <= 1.0 / (2.0 * a)))
                    return set_error(AMY_E_INVALID_ARG, "gamma above the uniform density (dim %d)", d);
                clo = -a;
                chi = a;
            } else if (g.noise == NOISE_EXPONENTIAL) {
                const double rate = g.np[0][d];
                if (!(cut->gamma < rate)) return set_error(AMY_E_INVALID_ARG, "gamma at or above the peak density (dim %d)", d);
                clo = 0.0;
                chi = std::log(rate / cut->gamma) / rate;
            } else if (g.noise == NOISE_BETA) {
                clo = g.np[2][d];
                chi = g.np[3][d];
            } else if (g.noise == NOISE_USER) {  // the box enclosing the density's support
                clo = g.np[0][d];
                chi = g.np[1][d];
            } else {
                return set_error(AMY_E_INVALID_ARG, "multiplicative noise has no cut: use gamma 0 or explicit windows");
            }
            const double w = std::floor((chi - clo) / g.eta[d]) + 1.0;
            if (!(w >= 1.0) || w > 1.0e6) return set_error(AMY_E_INVALID_ARG, "bad window width (dim %d)", d);
            g.W[d] = (int32_t)w;
            if (per && g.W[d] > g.N[d]) return set_error(AMY_E_INVALID_ARG, "window wider than periodic dim %d", d);
            g.clo[d] = clo;
            g.chi[d] = chi;
            g.xs[d] = chi;
        }
        wtot *= g.W[d];
        wsum += g.W[d];
        if (wtot > (1LL << 30)) return set_error(AMY_E_UNSUPPORTED, "window box too large");
    }
    if (wsum > MAXWS) return set_error(AMY_E_UNSUPPORTED, "sum of window widths %d exceeds %d", wsum, MAXWS);
    g.wtot = (int32_t)wtot;
    g.wsum = wsum;
    return AMY_OK;
}

amy_status make_geom(const amy_system *sys, const amy_grid *st, const amy_grid *in,
                     const double *sigma, const amy_cut *cut, Geom &g, std::vector<double> &params) {
    const amy_status r = fill_geom(sys, st, in, sigma, cut, g);
    if (r != AMY_OK) return r;
    params.assign(sys->params, sys->params + sys->n_params);
    return AMY_OK;
}

// Spec boxes -> device struct; checks that no grid state is both target and
// avoid (per dim: some centre inside the intersection of the two boxes).
amy_status make_spec(const Geom &g, const amy_spec *spec, SpecDev &s) {
    if (!spec) return set_error(AMY_E_INVALID_ARG, "null spec");
    memset(&s, 0, sizeof s);
    s.kind = spec->kind;
    if (spec->kind != AMY_SAFETY && spec->kind != AMY_REACH && spec->kind != AMY_REACH_AVOID)
        return set_error(AMY_E_INVALID_ARG, "unknown spec kind");
    if (spec->n_target < 0 || spec->n_target > MAX_BOXES || spec->n_avoid < 0 || spec->n_avoid > MAX_BOXES)
        return set_error(AMY_E_INVALID_ARG, "at most %d boxes of each kind", MAX_BOXES);
    if (spec->kind != AMY_SAFETY && spec->n_target < 1) return set_error(AMY_E_INVALID_ARG, "reach needs a target");
    if (spec->kind == AMY_REACH && spec->n_avoid != 0) return set_error(AMY_E_INVALID_ARG, "reach takes no avoid set");
    s.n_target = spec->n_target;
    s.n_avoid = spec->kind == AMY_REACH_AVOID ? spec->n_avoid : 0;
    for (int b = 0; b < s.n_target; ++b) {
        if (!spec->target || !spec->target[b].lb || !spec->target[b].ub) return set_error(AMY_E_INVALID_ARG, "null target box");
        for (int d = 0; d < g.n; ++d) {
            s.t_lb[b][d] = spec->target[b].lb[d];
            s.t_ub[b][d] = spec->target[b].ub[d];
        }
    }
    for (int b = 0; b < s.n_avoid; ++b) {
        if (!spec->avoid || !spec->avoid[b].lb || !spec->avoid[b].ub) return set_error(AMY_E_INVALID_ARG, "null avoid box");
        for (int d = 0; d < g.n; ++d) {
            s.a_lb[b][d] = spec->avoid[b].lb[d];
            s.a_ub[b][d] = spec->avoid[b].ub[d];
        }
    }
    if (spec->kind == AMY_SAFETY && spec->safe) {
        if (!spec->safe->lb || !spec->safe->ub) return set_error(AMY_E_INVALID_ARG, "null safe box");
        s.has_safe = 1;
        for (int d = 0; d < g.n; ++d) {
            s.safe_lb[d] = spec->safe->lb[d];
            s.safe_ub[d] = spec->safe->ub[d];
        }
    }
    for (int bt = 0; bt < s.n_target; ++bt)
        for (int ba = 0; ba < s.n_avoid; ++ba) {
            bool all = true;
            for (int d = 0; d < g.n && all; ++d) {
                const double lo = std::fmax(s.t_lb[bt][d], s.a_lb[ba][d]);
                const double hi = std::fmin(s.t_ub[bt][d], s.a_ub[ba][d]);
                bool any = false;
                for (int j = 0; j < g.N[d] && !any; ++j) {
                    const double c = g.lb[d] + (double)j * g.eta[d];
                    any = (lo <= c && c <= hi);
                }
                all = any;
            }
            if (all) return set_error(AMY_E_INVALID_ARG, "target box %d and avoid box %d share a grid state", bt, ba);
        }
    return AMY_OK;
}

// Separable stored mode: which state and input coordinates each mean
// component depends on.  Affine systems: state dim j matters for component d
// iff some A_u[d][j] is non-zero (a zero coefficient adds an exact zero in
// FP64); input dim i matters iff two inputs differing only in that coordinate
// have bitwise different rows (A_u[d][:], c_u[d]).  Unicycle: x on (x, th, v),
// y on (y, th, v), th on (th, w).
// Which state and input coordinates each mean component reads (bit j of
// Sx[d], bit i of Su[d]); the masses of dim d under multiplicative noise read
// x_d as well.
void system_deps(const Geom &g, const std::vector<double> &params, uint32_t *Sx, uint32_t *Su) {
    const int n = g.n, m = g.m;
    for (int d = 0; d < MAXD; ++d) Sx[d] = Su[d] = 0;
    if (g.sys == SYS_UNICYCLE) {
        Sx[0] = (1u << 0) | (1u << 2);
        Su[0] = 1u << 0;
        Sx[1] = (1u << 1) | (1u << 2);
        Su[1] = 1u << 0;
        Sx[2] = 1u << 2;
        Su[2] = 1u << 1;
    } else if (g.sys == SYS_EXPR) {
        for (int d = 0; d < n; ++d) {
            Sx[d] = g.xdep[d];
            Su[d] = g.udep[d];
        }
    } else {
        const int rec = n * n + n;
        int32_t ustr[MAXD];
        int32_t s = 1;
        for (int i = m - 1; i >= 0; --i) {
            ustr[i] = s;
            s *= g.ucount[i];
        }
        for (int u = 0; u < g.nu; ++u) {
            const double *A = params.data() + (size_t)u * rec;
            for (int d = 0; d < n; ++d)
                for (int j = 0; j < n; ++j)
                    if (A[d * n + j] != 0.0) Sx[d] |= 1u << j;
            int32_t r = u;
            for (int i = m - 1; i >= 0; --i) {
                const int32_t ui = r % g.ucount[i];
                r /= g.ucount[i];
                if (ui == 0) continue;
                const double *B = params.data() + (size_t)(u - ustr[i]) * rec;
                for (int d = 0; d < n; ++d) {
                    if (Su[d] & (1u << i)) continue;
                    bool same = memcmp(A + n * n + d, B + n * n + d, sizeof(double)) == 0;
                    for (int j = 0; j < n && same; ++j) same = memcmp(A + d * n + j, B + d * n + j, sizeof(double)) == 0;
                    if (!same) Su[d] |= 1u << i;
                }
            }
        }
    }
    if (g.noise == NOISE_MULT_GAUSSIAN)
        for (int d = 0; d < n; ++d) Sx[d] |= 1u << d;
}

// Strides of the dependency-compressed index of each dim's table: state
// coordinates fastest (lanes of a warp -- consecutive states, one input --
// then read consecutive records), then the input coordinates.
amy_status table_strides(Geom &g, const uint32_t *Sx, const uint32_t *Su) {
    for (int d = 0; d < g.n; ++d) {
        int64_t st = 1;
        for (int j = g.n - 1; j >= 0; --j) {
            g.tsx[d][j] = 0;
            if (Sx[d] & (1u << j)) {
                g.tsx[d][j] = (int32_t)st;
                st *= g.N[j];
                if (st > 2147483647LL) return set_error(AMY_E_UNSUPPORTED, "table of dim %d too large", d);
            }
        }
        for (int i = g.m - 1; i >= 0; --i) {
            g.tsu[d][i] = 0;
            if (Su[d] & (1u << i)) {
                if (st > 2147483647LL) return set_error(AMY_E_UNSUPPORTED, "table of dim %d too large", d);
                g.tsu[d][i] = (int32_t)st;
                st *= g.ucount[i];
            }
        }
        if (st > 2147483647LL) return set_error(AMY_E_UNSUPPORTED, "table of dim %d too large", d);
        g.tent[d] = (int32_t)st;
    }
    return AMY_OK;
}

amy_status plan_sep_tables(Geom &g, const std::vector<double> &params, int64_t &words,
                           std::vector<int32_t> *upart) {
    const int n = g.n, m = g.m;
    uint32_t Sx[MAXD], Su[MAXD];
    system_deps(g, params, Sx, Su);
    amy_status st0 = table_strides(g, Sx, Su);
    if (st0 != AMY_OK) return st0;
    int64_t off = 0;
    for (int d = 0; d < n; ++d) {
        g.trw[d] = ((1 + g.W[d]) + 3) / 4 * 4;
        g.toff[d] = off;
        off += (int64_t)g.tent[d] * g.trw[d];
    }
    // input part of each table index, one record of urw words per input
    g.uoff = off;
    g.urw = (n + 3) / 4 * 4;
    if (upart) {
        upart->assign((size_t)g.nu * g.urw, 0);
        for (int u = 0; u < g.nu; ++u) {
            int32_t ui[MAXD];
            int32_t r = u;
            for (int i = m - 1; i >= 0; --i) {
                ui[i] = r % g.ucount[i];
                r /= g.ucount[i];
            }
            for (int d = 0; d < n; ++d) {
                int64_t e = 0;
                for (int i = 0; i < m; ++i) e += (int64_t)ui[i] * g.tsu[d][i];
                (*upart)[(size_t)u * g.urw + d] = (int32_t)e;
            }
        }
    }
    g.boff = off + (int64_t)g.nu * g.urw;
    words = g.boff + 3 * MAXD + 4;
    g.shoff = 0;
    if (n >= 2 && n <= 3 && g.tent[n - 1] <= 4096) {
        g.shoff = (words + 3) / 4 * 4;
        words = g.shoff + 8 * (int64_t)g.tent[n - 1];
    }
    return AMY_OK;
}

int32_t input_outer_runs(const Geom &g, const std::vector<int32_t> &upart) {
    if (g.n < 2 || upart.size() < (size_t)g.nu * g.urw) return g.nu;
    int32_t runs = 0;
    for (int32_t u = 0; u < g.nu; ++u) {
        bool same = u > 0;
        for (int d = 0; d < g.n - 1 && same; ++d)
            same = upart[(size_t)u * g.urw + d] == upart[(size_t)(u - 1) * g.urw + d];
        if (!same) ++runs;
    }
    return runs;
}

void input_run_layout(const Geom &g, const std::vector<int32_t> &upart, std::vector<int32_t> &starts,
                      int32_t &stride_b) {
    starts.clear();
    stride_b = INT_MIN;
    if (g.n < 2 || upart.size() < (size_t)g.nu * g.urw) return;
    const int L = g.n - 1;
    bool have = false, same = true;
    int32_t step = 0;
    for (int32_t u = 0; u < g.nu; ++u) {
        bool start = u == 0;
        for (int d = 0; d < L && !start; ++d)
            start = upart[(size_t)u * g.urw + d] != upart[(size_t)(u - 1) * g.urw + d];
        if (start) {
            starts.push_back(u);
            continue;
        }
        const int32_t dd = upart[(size_t)u * g.urw + L] - upart[(size_t)(u - 1) * g.urw + L];
        if (!have) {
            step = dd;
            have = true;
        }
        same = same && dd == step;
    }
    starts.push_back(g.nu);
    if (same && (int64_t)step * 16 < INT32_MAX && (int64_t)step * 16 > INT32_MIN + 1) stride_b = step * 16;
}

bool input_runs_share_outer(const Geom &g, const std::vector<int32_t> &upart) {
    if (g.n < 2 || g.n > 3) return false;
    return 2 * (int64_t)input_outer_runs(g, upart) <= g.nu;
}

int choose_tile(int32_t nx, int32_t nu, int sm_count) {
    int tx = 256;
    while (tx > 1 && (int64_t)tx * nu > 4096) tx >>= 1;
    while (tx > 8 && ((int64_t)nx + tx - 1) / tx < 4LL * sm_count) tx >>= 1;
    return tx;
}

// ---------------------------------------------------------------------------
// Stored-row construction for wide windows with few pairs (where one thread
// per pair leaves the GPU idle): one thread per (run of BUILD_RUN window
// slots, pair) computes those slots' masses (the mean and origin in FP64, the
// masses as dim_masses does, each edge evaluated once) into F[slot][pair] --
// the factored layout -- and the run holding a dim's first slot writes the
// pair's origin; k_build_expand then forms each full-row entry as the product
// of its dims' masses in the order k_build multiplies them.
// ---------------------------------------------------------------------------
constexpr int BUILD_RUN = 8;
template <class R>
__global__ void __launch_bounds__(256) k_build_slots(const __grid_constant__ Geom g, R *__restrict__ F,
                                                     int16_t *__restrict__ O, int64_t npairs) {
    const int nruns = (g.wsum + BUILD_RUN - 1) / BUILD_RUN;
    const int64_t total = (int64_t)nruns * npairs;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = (int32_t)(i / npairs);
        const int64_t pair = i - (int64_t)r * npairs;
        const int32_t u = (int32_t)(pair / g.nx);
        const int32_t x = (int32_t)(pair - (int64_t)u * g.nx);
        double mu[MAXD];
        mean_of(g, x, u, mu);
        const int s0 = r * BUILD_RUN, s1 = min(g.wsum, s0 + BUILD_RUN);
        int b = 0;
        for (int d = 0; d < g.n && b < s1; b += g.W[d], ++d) {
            const int k0 = max(s0 - b, 0), k1 = min(s1 - b, g.W[d]);
            if (k0 >= k1) continue;
            const int32_t o = origin_of(g, d, mu[d]);
            slot_run(g, d, mu[d], o, kept_upper(g, d, mu[d], o), k0, k1, noise_centre(g, x, d),
                     [&](int k, R m, int32_t) { F[(int64_t)(b + k) * npairs + pair] = m; }, R(0));
            if (k0 == 0) O[(int64_t)d * npairs + pair] = (int16_t)o;
        }
    }
}

template <class R>
__global__ void __launch_bounds__(256) k_build_expand(const __grid_constant__ Geom g, const R *__restrict__ F,
                                                      R *__restrict__ T, int64_t npairs) {
    int fb[MAXD];
    int acc = 0;
    for (int d = 0; d < g.n; ++d) {
        fb[d] = acc;
        acc += g.W[d];
    }
    const int64_t total = (int64_t)g.wtot * npairs;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t t = (int32_t)(i / npairs);
        const int64_t pair = i - (int64_t)t * npairs;
        int k[MAXD];
        int32_t rem = t;
        for (int d = g.n - 1; d >= 0; --d) {
            k[d] = rem % g.W[d];
            rem /= g.W[d];
        }
        R v = R(1);
        for (int d = 0; d < g.n; ++d) v = v * F[(int64_t)(fb[d] + k[d]) * npairs + pair];
        T[i] = v;
    }
}

}  // namespace amy

struct amy_handle_s {
    Geom g;
    int32_t tmode, prec, v_store;
    cudaStream_t stream;
    bool own_stream;
    int device;
    int sm_count;
    int64_t budget;
    int64_t bytes;
    double *d_params;
    ExprProgram expr;     // text system: its parsed expressions and table kernel source
    double *d_mtab;       // and its mean tables (null for the built-in systems)
    double *d_ucdf;       // user noise densities: their CDF tables (null otherwise)
    void *d_T;
    int16_t *d_O;
    // stored rows (full or factored) with wide windows: the backup is split
    // over window rows (k_backup_rows), its pair sums S[u][x] kept here, or null
    void *d_split;
    int32_t split_groups;
    // 2-D tables with windows wider than the register-resident kernels take
    // (k_sums_sep2 + k_collect_keys, backup kernel 9): d_split holds the
    // per-state max keys
    int32_t sep_wide;
    // wide stored rows: the build runs one thread per (slot, pair)
    // (k_build_slots); stored full rows take their per-slot masses from
    // d_bfac (wsum x pairs) and expand them (k_build_expand)
    int32_t slot_build;
    void *d_bfac;
    int64_t npairs;
    void *d_V[2];         // V ping-pong (interior start)
    void *d_Vbase[2];     // allocations: kVGuard finite guard cells on each side
    uint8_t *d_mask;
    uint32_t *d_tab;      // per-dimension tables (separable stored mode)
    int64_t tab_words;
    int tileX;
    int fast_wm;          // width bound of the register-resident backup, 0 = generic kernel
    int ulanes;           // its input lanes per state (0 = heuristic)
    int rows;             // staged variant: row-aligned tiles allowed
    int grouped;          // staged variant: outer dims contracted once per input run
    int runs;             // number of those runs
    std::vector<int32_t> run_starts;  // input runs sharing their outer records (+ input count)
    int32_t in_stride_b;              // byte step of their shifted inner records (INT_MIN: varies)
    int bounds_known;     // tables' origin bounds read back after the last build
    int32_t bnd_lo[MAXD], bnd_hi[MAXD];
    int tilex;            // staged variant: lane columns per block (0 = default)
    int box_floats;       // staged variant: box budget (0 = default)
    int outer;            // per-run kernels: values of dim 0 per row tile (0 = 1)
    // plane kernel (banded problems with tables): its plan from the tables'
    // origin spreads, whether it is used where it applies, and its
    // shared-memory budget per block (0 = default)
    int32_t spread[MAXD];
    PlanePlan plane;
    int use_plane;
    int plane_smem;
    // its padded copies of the two V vectors (planes padded to Ppad values;
    // null when the problem lacks the plane structure) and which V vector
    // the padded copies currently mirror (null: none, repack first)
    void *d_Vp[2];
    int64_t vp_rows;
    int32_t vp_pad;
    const void *vp_src;
    std::vector<double> host_params;
    // kernel timing: CUDA events around every backup / build kernel when profiling
    bool profiling;
    // CUDA graph of the horizon loop (a spec-mask launch + `horizon` backups),
    // replayed while the spec, horizon and output pointers repeat
    int use_graphs;
    cudaStream_t cap_stream;
    cudaGraphExec_t graph_exec;
    bool graph_valid;
    SpecDev g_spec;
    int32_t g_horizon, g_all;
    void *g_vout;
    uint16_t *g_pi;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_backup, ev_build;
    std::vector<int32_t> ev_backup_steps;  // backups performed by each timed backup launch
    // persistent horizon kernel: applies to this handle's problem and shape
    // (checked after the shape is fixed), its barrier block (kBarWords:
    // grid-barrier words, per-tile backup counters, error flag), the polls a
    // wait makes before it gives up, and whether blocks wait for every block
    // (grid barrier) or only for their neighbour tiles between backups
    int synth_ok;
    unsigned *d_bar;
    int32_t spin_limit;
    int32_t grid_barrier;
    // host outputs: a device staging buffer kept across calls (grown on
    // demand; a per-call stream-ordered allocation went back to the driver at
    // every synchronisation and cost more than the synthesis), and a
    // page-locked word the barrier error flag is read into
    void *d_stage;
    size_t stage_cap;
    int32_t *h_err;
    amy_info_t info;
};

namespace {

size_t rsize(const amy_handle_s *h) { return h->prec == AMY_PREC_FP64 ? 8 : 4; }
size_t vsize(const amy_handle_s *h) { return h->prec == AMY_PREC_FP64 ? 8 : (h->v_store ? 2 : 4); }

amy_status dev_alloc(amy_handle_s *h, void **p, size_t bytes, const char *what) {
    if (h->budget > 0 && h->bytes + (int64_t)bytes > h->budget)
        return set_error(AMY_E_OUT_OF_MEMORY, "%s: %zu bytes exceed the device memory budget", what, bytes);
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) return cuda_error(e, what);
    h->bytes += (int64_t)bytes;
    return AMY_OK;
}

// Page-locked words the handles read their barrier error flag into, handed
// out from 4 KiB pages that stay allocated until the process exits: one
// page-locked allocation (and its release, which synchronises the device) per
// handle cost a large share of building and destroying a small problem.
struct PinnedWords {
    std::mutex mu;
    std::vector<int32_t *> free_words;
    int32_t *take() {
        std::lock_guard<std::mutex> lk(mu);
        if (free_words.empty()) {
            int32_t *page = nullptr;
            if (cudaHostAlloc((void **)&page, 4096, cudaHostAllocPortable) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
            for (int i = 0; i < 4096 / (int)sizeof(int32_t); ++i) free_words.push_back(page + i);
        }
        int32_t *w = free_words.back();
        free_words.pop_back();
        return w;
    }
    void give(int32_t *w) {
        std::lock_guard<std::mutex> lk(mu);
        free_words.push_back(w);
    }
};
PinnedWords &pinned_words() {
    static PinnedWords *p = new PinnedWords();  // never destroyed: handles may outlive static destructors
    return *p;
}

void free_handle(amy_handle_s *h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    cudaFree(h->d_params);
    cudaFree(h->d_mtab);
    cudaFree(h->d_ucdf);
    cudaFree(h->d_T);
    cudaFree(h->d_O);
    cudaFree(h->d_split);
    cudaFree(h->d_bfac);
    cudaFree(h->d_Vbase[0]);
    cudaFree(h->d_Vbase[1]);
    cudaFree(h->d_Vp[0]);
    cudaFree(h->d_Vp[1]);
    cudaFree(h->d_mask);
    cudaFree(h->d_tab);
    cudaFree(h->d_bar);
    cudaFree(h->d_stage);
    if (h->h_err) pinned_words().give(h->h_err);
    for (auto &p : h->ev_backup) h->ev_pool.push_back(p.first), h->ev_pool.push_back(p.second);
    for (auto &p : h->ev_build) h->ev_pool.push_back(p.first), h->ev_pool.push_back(p.second);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

// Whether splitting each pair's window rows over thread groups can help:
// only when one thread per pair leaves the GPU's thread slots (2048 per SM)
// unfilled; with more pairs than that the generic kernel already keeps every
// SM busy and the split would only add the pair sums' round trip.
bool split_pays(const amy_handle_s *h) { return h->npairs < (int64_t)h->sm_count * 2048; }

// The host-output staging buffer, at least `bytes` long.  Grown with the
// stream idle (the previous call's copies out of it have completed).  It is
// outside the device-memory budget (a call with host outputs must not fail
// where one with device outputs succeeds) and reported in device_bytes.
amy_status stage_buffer(amy_handle_s *h, size_t bytes, void **out) {
    if (bytes > h->stage_cap) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_error(e, "output staging");
        cudaFree(h->d_stage);
        h->d_stage = nullptr;
        h->stage_cap = 0;
        e = cudaMalloc(&h->d_stage, bytes);
        if (e != cudaSuccess) return cuda_error(e, "output staging");
        h->stage_cap = bytes;
    }
    *out = h->d_stage;
    return AMY_OK;
}

// The device address of page-locked host memory the device can write
// (cudaHostAlloc / cudaHostRegister'ed, mapped), or null for any other
// pointer (pageable memory goes through the staging buffer).
void *mapped_host(void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

#define AMY_CUDA(call, what)                          \
    do {                                              \
        cudaError_t e__ = (call);                     \
        if (e__ != cudaSuccess) return cuda_error(e__, what); \
    } while (0)

template <class R, class VT>
amy_status launch_mask(amy_handle_s *h, const SpecDev &s, VT *VN) {
    const int blocks = (int)std::min<int64_t>((h->g.nx + 255) / 256, 65535);
    k_spec_mask<R, VT><<<blocks, 256, 0, h->stream>>>(h->g, s, h->d_mask, VN);
    AMY_CUDA(cudaGetLastError(), "spec mask launch");
    return AMY_OK;
}

template <class R, class VT, int TM, bool KAHAN>
amy_status launch_backup_t(amy_handle_s *h, int spec_kind, const VT *Vn, VT *Vo, R *Vfinal, uint16_t *pi) {
    BackupArgs<R, VT> a;
    a.Vn = Vn;
    a.Vo = Vo;
    a.Vfinal = Vfinal;
    a.pi = pi;
    a.mask = h->d_mask;
    a.spec_kind = spec_kind;
    a.tileX = h->tileX;
    a.T = (const R *)h->d_T;
    a.O = h->d_O;
    a.npairs = h->npairs;
    a.tab = h->d_tab;
    if constexpr (TM == TM_SEPARABLE && sizeof(R) == 4) {
        if (h->sep_wide && h->d_split) {
            // 2-D tables with wide windows: each input's value into a per-state
            // max key, then V_k and pi_k from the keys (which are cleared)
            const int64_t items = (int64_t)h->g.nx * (h->g.nu / h->g.nw);
            const int blocks = (int)std::min<int64_t>((items + 255) / 256, (int64_t)h->sm_count * 64);
            unsigned long long *keys = (unsigned long long *)h->d_split;
            const Geom &g = h->g;
            const size_t vsm = sep2_smem_bytes(g.N[0], g.W[0], g.N[1], g.W[1]);
            if (g.periodic == 0 && vsm <= 48 * 1024)  // V staged in shared memory with a zero border
                k_sums_sep2<VT, KAHAN, true><<<blocks, 256, vsm, h->stream>>>(g, h->d_tab, Vn, h->d_mask, spec_kind,
                                                                              keys);
            else
                k_sums_sep2<VT, KAHAN, false><<<blocks, 256, 0, h->stream>>>(g, h->d_tab, Vn, h->d_mask, spec_kind,
                                                                             keys);
            AMY_CUDA(cudaGetLastError(), "input values launch");
            const int cb = (int)std::min<int64_t>((h->g.nx + 255) / 256, 65535);
            k_collect_keys<VT><<<cb, 256, 0, h->stream>>>(h->g, h->d_mask, spec_kind, keys, Vo, (float *)Vfinal, pi);
            AMY_CUDA(cudaGetLastError(), "collect launch");
            return AMY_OK;
        }
    }
    if constexpr (TM == TM_FULL || TM == TM_FACTORED || TM == TM_OTF) {
        if (h->d_split) {
            // split over window rows: pair sums, then max / argmax per state
            const dim3 grid((unsigned)((h->g.nx + 31) / 32), (unsigned)h->g.nu);
            const dim3 block(32, (unsigned)h->split_groups);
            if constexpr (TM == TM_OTF) {
                const size_t smem = (size_t)h->g.wsum * 32 * (sizeof(R) + sizeof(int32_t));
                auto kern = k_backup_rows_otf<R, VT, KAHAN>;
                // above the default 48 KiB the kernel needs the opt-in (set on
                // every such launch: the attribute is per device)
                if (smem > 48 * 1024)
                    AMY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                             "row-split smem attribute");
                kern<<<grid, block, smem, h->stream>>>(h->g, a, (R *)h->d_split);
            } else {
                k_backup_rows<R, VT, TM, KAHAN><<<grid, block, 0, h->stream>>>(h->g, a, (R *)h->d_split);
            }
            AMY_CUDA(cudaGetLastError(), "backup launch");
            const int blocks = (int)std::min<int64_t>((h->g.nx + 255) / 256, 65535);
            k_argmax_rows<R, VT><<<blocks, 256, 0, h->stream>>>(h->g, a, (const R *)h->d_split);
            AMY_CUDA(cudaGetLastError(), "argmax launch");
            return AMY_OK;
        }
    }
    const int blocks = (h->g.nx + h->tileX - 1) / h->tileX;
    const size_t smem = (size_t)h->tileX * h->g.nu * sizeof(R);
    k_backup<R, VT, TM, KAHAN><<<blocks, 256, smem, h->stream>>>(h->g, a);
    AMY_CUDA(cudaGetLastError(), "backup launch");
    return AMY_OK;
}

template <class R, class VT, bool KAHAN>
amy_status launch_backup_k(amy_handle_s *h, int spec_kind, const VT *Vn, VT *Vo, R *Vfinal, uint16_t *pi) {
    switch (h->tmode) {
        case AMY_T_ON_THE_FLY: return launch_backup_t<R, VT, TM_OTF, KAHAN>(h, spec_kind, Vn, Vo, Vfinal, pi);
        case AMY_T_STORED_FULL: return launch_backup_t<R, VT, TM_FULL, KAHAN>(h, spec_kind, Vn, Vo, Vfinal, pi);
        case AMY_T_STORED_SEPARABLE:
            return launch_backup_t<R, VT, TM_SEPARABLE, KAHAN>(h, spec_kind, Vn, Vo, Vfinal, pi);
        default: return launch_backup_t<R, VT, TM_FACTORED, KAHAN>(h, spec_kind, Vn, Vo, Vfinal, pi);
    }
}

cudaEvent_t pooled_event(amy_handle_s *h) {
    if (!h->ev_pool.empty()) {
        cudaEvent_t e = h->ev_pool.back();
        h->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Brackets one kernel launch with CUDA events on the handle's stream when
// profiling is on.
struct KernelTimer {
    amy_handle_s *h;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *list;
    int32_t steps;  // backups the bracketed launch performs (backup list only)
    cudaEvent_t a = nullptr, b = nullptr;
    KernelTimer(amy_handle_s *hh, std::vector<std::pair<cudaEvent_t, cudaEvent_t>> *l, int32_t n_steps = 1)
        : h(hh), list(l), steps(n_steps) {
        if (!h->profiling) return;
        a = pooled_event(h);
        b = pooled_event(h);
        if (a && b) cudaEventRecord(a, h->stream);
    }
    void done() {
        if (!h->profiling || !a || !b) return;
        cudaEventRecord(b, h->stream);
        list->push_back({a, b});
        if (list == &h->ev_backup) h->ev_backup_steps.push_back(steps);
    }
};

amy_status launch_backup_generic(amy_handle_s *h, int spec_kind, const void *Vn, void *Vo, void *Vfinal,
                                 uint16_t *pi);

// Reads and clears the persistent kernel's error flag (synchronises the
// handle's stream).
amy_status check_synth_error(amy_handle_s *h) {
    if (!h->d_bar || !h->h_err) return AMY_OK;
    *h->h_err = 0;
    AMY_CUDA(cudaMemcpyAsync(h->h_err, h->d_bar + kBarErrWord, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream),
             "barrier flag read");
    AMY_CUDA(cudaStreamSynchronize(h->stream), "barrier flag read");
    const int32_t err = *h->h_err;
    if (err == 0) return AMY_OK;
    AMY_CUDA(cudaMemsetAsync(h->d_bar + kBarErrWord, 0, sizeof(int32_t), h->stream), "barrier flag reset");
    if (err == 1) return set_error(AMY_E_TIMEOUT, "persistent backup: a grid barrier wait gave up");
    return set_error(AMY_E_CUDA, "persistent backup: launch shape rejected on the device");
}

int tm_kind_of(const amy_handle_s *h) {
    return h->tmode == AMY_T_ON_THE_FLY ? TM_OTF : h->tmode == AMY_T_STORED_FACTORED ? TM_FACTORED : TM_SEPARABLE;
}

bool fast_path(const amy_handle_s *h) { return h->fast_wm > 0 && h->tmode != AMY_T_STORED_FULL; }

// Whether the plane kernel runs in its tiled form (backup kernel 8): always
// where it applies in mode 2, never in mode 3, and in the default mode 1 for
// planes of at least kTileMinPlane states (on GB300 the tile kernel was faster
// on the 21^6 traffic ring's planes of 441 states and slower on the rooms'
// planes of 81, where the plane kernel packs five groups per block).
constexpr int kTileMinPlane = 256;
bool tile_on(const amy_handle_s *h) {
    if (!h->plane.tile) return false;
    return h->use_plane == 2 || (h->use_plane == 1 && h->plane.P >= kTileMinPlane);
}

// The tables' bounds on (window origin - own coordinate) as the launch sees them.
void set_bounds(const amy_handle_s *h, FastCall &c) {
    c.run_starts = h->run_starts.empty() ? nullptr : h->run_starts.data();
    c.n_runs = h->run_starts.empty() ? 0 : (int32_t)h->run_starts.size() - 1;
    c.in_stride_b = h->in_stride_b;
    c.bounds_known = h->bounds_known;
    for (int d = 0; d < 3; ++d) {
        c.bnd_lo[d] = d < h->g.n ? h->bnd_lo[d] : 0;
        c.bnd_hi[d] = d < h->g.n ? h->bnd_hi[d] : 0;
    }
}

// Reads the bounds block the table build leaves after the tables: the host
// copy sizes the per-run kernel's box and goes to it as launch parameters.
amy_status read_bounds(amy_handle_s *h) {
    h->bounds_known = 0;
    h->plane = PlanePlan();
    if (h->tmode != AMY_T_STORED_SEPARABLE) return AMY_OK;
    int32_t b[3 * MAXD + 4];
    AMY_CUDA(cudaMemcpyAsync(b, h->d_tab + h->g.boff, sizeof b, cudaMemcpyDeviceToHost, h->stream), "bounds read");
    AMY_CUDA(cudaStreamSynchronize(h->stream), "bounds read");
    for (int d = 0; d < MAXD; ++d) h->spread[d] = b[2 * MAXD + 4 + d];
    plan_plane(h->g, TM_SEPARABLE, h->prec, h->spread, h->plane_smem, h->plane);
    const int all = (1 << h->g.n) - 1;
    if ((b[2 * MAXD] & all) != all) return AMY_OK;
    for (int d = 0; d < h->g.n; ++d) {
        h->bnd_lo[d] = b[d];
        h->bnd_hi[d] = b[MAXD + d];
    }
    h->bounds_known = 1;
    return AMY_OK;
}

// One backup V_{k+1} (Vn) -> V_k (Vo) with the handle's precision: the
// register-resident kernel when the window fits it, the generic one otherwise.
// Arguments of the register-resident / staged backups for this handle's
// problem, tables and launch shape.
FastCall fast_call(const amy_handle_s *h, int spec_kind, const void *Vn, void *Vo, void *Vfinal, uint16_t *pi) {
    FastCall c;
    c.Vn = Vn;
    c.Vo = Vo;
    c.Vfinal = (float *)Vfinal;
    c.pi = pi;
    c.mask = h->d_mask;
    c.spec_kind = spec_kind;
    c.kahan = h->prec == AMY_PREC_FP32_KAHAN;
    c.T = (const float *)h->d_T;
    c.O = h->d_O;
    c.npairs = h->npairs;
    c.tab = h->d_tab;
    c.ulanes = h->ulanes;
    c.rows = h->rows;
    c.grouped = h->grouped;
    c.runs = h->runs;
    set_bounds(h, c);
    c.tilex = h->tilex;
    c.box_floats = h->box_floats;
    c.outer = h->outer;
    c.plane = (h->use_plane && h->plane.ok && h->d_Vp[0]) ? &h->plane : nullptr;
    c.tile = tile_on(h);
    return c;
}

// The persistent horizon kernel's arguments (V_N in d_V[0]).
SynthCall synth_call(amy_handle_s *h, int32_t horizon, void *d_Vout, uint16_t *d_pi, int32_t all_steps) {
    SynthCall sc;
    sc.V0 = h->d_V[0];
    sc.V1 = h->d_V[1];
    sc.Vfinal = (float *)d_Vout;
    sc.pi = d_pi;
    sc.all_steps = all_steps;
    sc.horizon = horizon;
    sc.bar = h->d_bar;
    sc.err = reinterpret_cast<int32_t *>(h->d_bar + kBarErrWord);
    sc.grid_barrier = h->grid_barrier;
    sc.spin_limit = h->spin_limit;
    return sc;
}

// Whether the persistent horizon kernel applies with the handle's current
// tables, bounds and launch shape (all blocks resident at once).
void update_synth_ok(amy_handle_s *h) {
    h->synth_ok = 0;
    if (!h->d_bar || !fast_path(h)) return;
    const FastCall c = fast_call(h, SPEC_SAFETY, h->d_V[0], h->d_V[1], nullptr, nullptr);
    const SynthCall sc = synth_call(h, 1, nullptr, nullptr, 0);
    h->synth_ok = launch_synth_fast(h->g, tm_kind_of(h), h->v_store, c, sc, h->sm_count, h->stream, true) == AMY_OK;
    cudaGetLastError();
}

amy_status launch_backup(amy_handle_s *h, int spec_kind, const void *Vn, void *Vo, void *Vfinal, uint16_t *pi,
                         unsigned long long *work = nullptr) {
    if (fast_path(h)) {
        FastCall c = fast_call(h, spec_kind, Vn, Vo, Vfinal, pi);
        c.work = work;
        if (c.plane) {
            // the plane kernel reads V_{k+1} from its padded copy: make it when
            // the copies do not mirror Vn (V_N, a caller's V_{k+1})
            if (Vn != h->d_V[0] && Vn != h->d_V[1])
                return set_error(AMY_E_INVALID_ARG, "plane backup: V_{k+1} is not one of the handle's vectors");
            const int in = Vn == h->d_V[1] ? 1 : 0;
            if (h->vp_src != Vn) {
                amy_status r = launch_plane_repack(h->v_store, Vn, h->d_Vp[in], h->vp_rows, h->plane.P, h->vp_pad,
                                                   h->stream);
                if (r != AMY_OK) return r;
            }
            c.Vpn = h->d_Vp[in];
            c.Vpo = h->d_Vp[in ^ 1];
        }
        KernelTimer tm(h, &h->ev_backup);
        const amy_status st = launch_backup_fast(h->g, tm_kind_of(h), h->v_store, c, h->sm_count, h->stream);
        tm.done();
        h->vp_src = (c.plane && st == AMY_OK) ? Vo : nullptr;
        return st;
    }
    KernelTimer tm(h, &h->ev_backup);
    const amy_status st = launch_backup_generic(h, spec_kind, Vn, Vo, Vfinal, pi);
    tm.done();
    return st;
}

amy_status launch_backup_generic(amy_handle_s *h, int spec_kind, const void *Vn, void *Vo, void *Vfinal,
                                 uint16_t *pi) {
    if (h->prec == AMY_PREC_FP64)
        return launch_backup_k<double, double, false>(h, spec_kind, (const double *)Vn, (double *)Vo,
                                                      (double *)Vfinal, pi);
    const bool kahan = h->prec == AMY_PREC_FP32_KAHAN;
    if (h->v_store == AMY_V_BF16) {
        if (kahan)
            return launch_backup_k<float, __nv_bfloat16, true>(h, spec_kind, (const __nv_bfloat16 *)Vn,
                                                               (__nv_bfloat16 *)Vo, (float *)Vfinal, pi);
        return launch_backup_k<float, __nv_bfloat16, false>(h, spec_kind, (const __nv_bfloat16 *)Vn,
                                                            (__nv_bfloat16 *)Vo, (float *)Vfinal, pi);
    }
    if (h->v_store == AMY_V_UNORM16) {
        if (kahan)
            return launch_backup_k<float, unorm16, true>(h, spec_kind, (const unorm16 *)Vn, (unorm16 *)Vo,
                                                         (float *)Vfinal, pi);
        return launch_backup_k<float, unorm16, false>(h, spec_kind, (const unorm16 *)Vn, (unorm16 *)Vo,
                                                      (float *)Vfinal, pi);
    }
    if (kahan)
        return launch_backup_k<float, float, true>(h, spec_kind, (const float *)Vn, (float *)Vo, (float *)Vfinal, pi);
    return launch_backup_k<float, float, false>(h, spec_kind, (const float *)Vn, (float *)Vo, (float *)Vfinal, pi);
}

amy_status launch_mask_any(amy_handle_s *h, const SpecDev &s, void *VN) {
    h->vp_src = nullptr;  // V is rewritten: the plane kernel's padded copies no longer mirror it
    if (h->prec == AMY_PREC_FP64) return launch_mask<double, double>(h, s, (double *)VN);
    if (h->v_store == AMY_V_BF16) return launch_mask<float, __nv_bfloat16>(h, s, (__nv_bfloat16 *)VN);
    if (h->v_store == AMY_V_UNORM16) return launch_mask<float, unorm16>(h, s, (unorm16 *)VN);
    return launch_mask<float, float>(h, s, (float *)VN);
}

template <class R>
amy_status launch_build(amy_handle_s *h) {
    KernelTimer tm(h, &h->ev_build);
    if (h->tmode == AMY_T_STORED_SEPARABLE) {
        amy_status st = launch_build_sep(h->g, h->d_tab, h->sm_count, h->stream);
        tm.done();
        return st;
    }
    if (h->slot_build) {
        const int64_t items = (int64_t)((h->g.wsum + BUILD_RUN - 1) / BUILD_RUN) * h->npairs;
        const int bs = (int)std::min<int64_t>((items + 255) / 256, (int64_t)h->sm_count * 64);
        R *F = h->tmode == AMY_T_STORED_FULL ? (R *)h->d_bfac : (R *)h->d_T;
        k_build_slots<R><<<bs, 256, 0, h->stream>>>(h->g, F, h->d_O, h->npairs);
        if (h->tmode == AMY_T_STORED_FULL) {
            const int64_t entries = (int64_t)h->g.wtot * h->npairs;
            const int be = (int)std::min<int64_t>((entries + 255) / 256, (int64_t)h->sm_count * 64);
            k_build_expand<R><<<be, 256, 0, h->stream>>>(h->g, F, (R *)h->d_T, h->npairs);
        }
        tm.done();
        AMY_CUDA(cudaGetLastError(), "build launch");
        return AMY_OK;
    }
    const int blocks = (int)std::min<int64_t>((h->npairs + 127) / 128, (int64_t)h->sm_count * 32);
    if (h->tmode == AMY_T_STORED_FULL)
        k_build<R, TM_FULL><<<blocks, 128, 0, h->stream>>>(h->g, (R *)h->d_T, h->d_O, h->npairs);
    else
        k_build<R, TM_FACTORED><<<blocks, 128, 0, h->stream>>>(h->g, (R *)h->d_T, h->d_O, h->npairs);
    tm.done();
    AMY_CUDA(cudaGetLastError(), "build launch");
    return AMY_OK;
}

}  // namespace

extern "C" {

const char *amy_last_error(void) { return amy::g_last_error.c_str(); }

int64_t amy_grid_count(double lb, double ub, double eta) { return amy::grid_count(lb, ub, eta); }

namespace {

// Launch-shape autotuner (amy_opts.autotune).  Times the register-resident
// backup for every input-lane count and, where the staged variant runs, both
// tile mappings, on the handle's own V buffers with every state free, and
// keeps the fastest.  The results do not depend on the shape: each (state,
// input) sum is formed by the same arithmetic whatever thread owns it, and
// the merge over input lanes keeps the lowest maximising input.
amy_status autotune_shape(amy_handle_s *h) {
    const double slots = (double)h->g.nx * (double)h->g.nu * (double)h->g.wtot;
    if (!fast_path(h) || slots > 4e9) return AMY_OK;
    AMY_CUDA(cudaMemsetAsync(h->d_mask, 0, (size_t)h->g.nx, h->stream), "autotune mask");
    cudaEvent_t ea = nullptr, eb = nullptr;
    AMY_CUDA(cudaEventCreate(&ea), "autotune event");
    if (cudaEventCreate(&eb) != cudaSuccess) {
        cudaEventDestroy(ea);
        return set_error(AMY_E_CUDA, "autotune event");
    }
    FastCall c;
    c.Vn = h->d_V[0];
    c.Vo = h->d_V[1];
    c.Vfinal = nullptr;
    c.pi = nullptr;
    c.mask = h->d_mask;
    c.spec_kind = SPEC_REACH;  // a zero mask leaves every state free
    c.kahan = h->prec == AMY_PREC_FP32_KAHAN;
    c.T = (const float *)h->d_T;
    c.O = h->d_O;
    c.npairs = h->npairs;
    c.tab = h->d_tab;
    c.grouped = h->grouped;
    c.runs = h->runs;
    set_bounds(h, c);
    const bool staged = fast_shape(h->g, tm_kind_of(h), c, h->sm_count).staged;
    // candidates: power-of-two input lanes, plus one lane per input run; the
    // staged variant also varies the states per block and the tile mapping
    std::vector<int> uls = {1, 2, 4, 8};
    if (staged && h->grouped && h->runs >= 2)  // lanes take whole runs: any count up to the runs
        for (int ul = 3; ul <= std::min(h->runs, 8); ++ul)
            if ((ul & (ul - 1)) != 0) uls.push_back(ul);
    // candidate shapes: (input lanes, states per block, row tiles, box budget,
    // dim-0 values per tile).  Staged: powers of two states per block with
    // either tile mapping and two box budgets; where the per-run kernels take
    // row tiles also any multiple of 32 states per block split over 1..4
    // values of dim 0 (exact boxes).  Register-resident: 256 threads.
    struct Cand {
        int ul, tx, rows, box, outer;
    };
    std::vector<Cand> cands;
    for (int ul : uls) {
        if (ul > 1 && ul > h->g.nu) continue;
        if (!staged) {
            if (256 % ul == 0) cands.push_back({ul, 0, 1, 0, 0});
            continue;
        }
        for (int tx = 32; tx * ul <= 512; tx <<= 1)
            for (int cand = 0; cand < 4; ++cand) cands.push_back({ul, tx, cand & 1, (cand >> 1) ? 3072 : 0, 0});
        FastCall q = c;
        q.ulanes = ul;
        q.rows = 1;
        for (int tx = 32; tx * ul <= 512; tx += 32) {
            q.tilex = tx;
            for (int outer = 1; outer <= (h->g.n == 3 ? 4 : 1); ++outer) {
                q.outer = outer;
                const FastShape sh = fast_shape(h->g, tm_kind_of(h), q, h->sm_count);
                if (!sh.runs || sh.outer != outer) continue;
                if ((tx & (tx - 1)) == 0 && outer == 1) continue;  // already listed
                cands.push_back({ul, tx, 1, 0, outer});
            }
        }
    }
    float best = 3.4e38f;
    int best_ul = h->ulanes, best_tx = h->tilex, best_rows = h->rows, best_box = h->box_floats,
        best_outer = h->outer, best_wait = h->grid_barrier;
    amy_status st = AMY_OK;
    for (const Cand &cd : cands) {
        if (st != AMY_OK) break;
        {
            {
                const int ul = cd.ul, rows = cd.rows;
                c.ulanes = ul;
                c.tilex = cd.tx;
                c.rows = rows;
                c.box_floats = cd.box;
                c.outer = cd.outer;
                if (rows == 1 && staged && fast_shape(h->g, tm_kind_of(h), c, h->sm_count).rowtile == 0) continue;
                // per backup: the persistent horizon kernel over 8 backups where
                // it applies with this shape (synthesis then uses it), else 3
                // launches of the per-step kernel after a warm-up launch
                const SynthCall sc = synth_call(h, 8, nullptr, nullptr, 0);
                const bool persist =
                    h->d_bar &&
                    launch_synth_fast(h->g, tm_kind_of(h), h->v_store, c, sc, h->sm_count, h->stream, true) == AMY_OK;
                cudaGetLastError();
                const int reps = persist ? 8 : 3;
                // the persistent kernel is timed with either wait between
                // backups (grid barrier first)
                for (int wait = 1; wait >= (persist ? 0 : 1) && st == AMY_OK; --wait) {
                    h->grid_barrier = wait;
                    const SynthCall scw = synth_call(h, 8, nullptr, nullptr, 0);
                    cudaError_t e = cudaSuccess;
                    float ms_first = 3.4e38f;
                    if (persist) {
                        // the better of two launches (the first one also warms up)
                        for (int t = 0; t < 2 && st == AMY_OK && e == cudaSuccess; ++t) {
                            e = cudaMemsetAsync(h->d_bar, 0, kBarResetBytes, h->stream);
                            if (e == cudaSuccess) e = cudaEventRecord(ea, h->stream);
                            if (e == cudaSuccess)
                                st = launch_synth_fast(h->g, tm_kind_of(h), h->v_store, c, scw, h->sm_count, h->stream,
                                                       false);
                            if (t == 0 && st == AMY_OK && e == cudaSuccess) {
                                e = cudaEventRecord(eb, h->stream);
                                if (e == cudaSuccess) e = cudaEventSynchronize(eb);
                                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_first, ea, eb);
                            }
                        }
                    } else {
                        st = launch_backup_fast(h->g, tm_kind_of(h), h->v_store, c, h->sm_count, h->stream);
                        if (st == AMY_OK) e = cudaEventRecord(ea, h->stream);
                        for (int rep = 0; rep < reps && st == AMY_OK && e == cudaSuccess; ++rep)
                            st = launch_backup_fast(h->g, tm_kind_of(h), h->v_store, c, h->sm_count, h->stream);
                    }
                    if (st == AMY_OK && e == cudaSuccess) e = cudaEventRecord(eb, h->stream);
                    if (st == AMY_OK && e == cudaSuccess) e = cudaEventSynchronize(eb);
                    float ms = 0.0f;
                    if (st == AMY_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, ea, eb);
                    if (st == AMY_OK && e != cudaSuccess) st = cuda_error(e, "autotune timing");
                    if (st == AMY_OK && persist) st = check_synth_error(h);
                    ms = std::min(ms, ms_first) / (float)reps;
                    if (st == AMY_OK && ms < best) {
                        best = ms;
                        best_ul = ul;
                        best_tx = c.tilex;
                        best_rows = rows;
                        best_box = c.box_floats;
                        best_outer = c.outer;
                        best_wait = wait;
                    }
                }
            }
        }
    }
    cudaEventDestroy(ea);
    cudaEventDestroy(eb);
    if (st != AMY_OK) return st;
    h->ulanes = best_ul;
    h->tilex = best_tx;
    h->rows = best_rows;
    h->box_floats = best_box;
    h->outer = best_outer;
    h->grid_barrier = best_wait;
    return AMY_OK;
}

}  // namespace

amy_status amy_build(const amy_system *sys, const amy_grid *states, const amy_grid *inputs,
                     const double *sigma, const amy_cut *cut, const amy_opts *opts, amy_handle *out) {
    if (!out || !opts) return set_error(AMY_E_INVALID_ARG, "null argument");
    *out = nullptr;
    Geom g;
    std::vector<double> params;
    amy_status st = make_geom(sys, states, inputs, sigma, cut, g, params);
    if (st != AMY_OK) return st;
    ExprProgram prog;
    if (g.sys == SYS_EXPR) {
        const int p_dist = (sys->disturb && sys->disturb->n > 0) ? sys->disturb->n : 0;
        st = expr_compile(sys->expr, g.n, g.m - p_dist, p_dist, sys->n_params, prog);
        if (st != AMY_OK) return st;
        for (int d = 0; d < MAXD; ++d) {
            g.xdep[d] = prog.dep_x[d];
            g.udep[d] = prog.dep_u[d];
        }
    }
    if (opts->tmode < AMY_T_ON_THE_FLY || opts->tmode > AMY_T_AUTO)
        return set_error(AMY_E_INVALID_ARG, "unknown tmode");
    if (opts->prec < AMY_PREC_FP64 || opts->prec > AMY_PREC_FP32_KAHAN)
        return set_error(AMY_E_INVALID_ARG, "unknown precision");
    const int32_t tmode =
        opts->tmode == AMY_T_AUTO ? choose_tmode(g, params, opts->prec, opts->device_mem_budget) : opts->tmode;
    if (tmode == AMY_T_STORED_SEPARABLE && opts->prec == AMY_PREC_FP64)
        return set_error(AMY_E_UNSUPPORTED, "separable tables hold FP32 masses");
    if (opts->prec < AMY_PREC_FP64 || opts->prec > AMY_PREC_FP32_KAHAN)
        return set_error(AMY_E_INVALID_ARG, "unknown precision");
    if (opts->v_store < AMY_V_NATIVE || opts->v_store > AMY_V_UNORM16)
        return set_error(AMY_E_INVALID_ARG, "unknown V storage");
    if (opts->v_store != AMY_V_NATIVE && opts->prec == AMY_PREC_FP64)
        return set_error(AMY_E_INVALID_ARG, "16-bit V storage needs an FP32 precision");
    if (tmode == AMY_T_STORED_FULL || tmode == AMY_T_STORED_FACTORED)
        for (int d = 0; d < g.n; ++d)
            if (g.N[d] + g.W[d] + 2 > 32767)
                return set_error(AMY_E_UNSUPPORTED, "stored origins are int16: dim %d too large", d);
    amy_handle_s *h = new (std::nothrow) amy_handle_s();
    if (!h) return set_error(AMY_E_OUT_OF_MEMORY, "host allocation");
    h->g = g;
    h->tmode = tmode;
    h->prec = opts->prec;
    h->v_store = opts->v_store;
    h->budget = opts->device_mem_budget;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_error(e, "device query");
    }
    if (opts->cuda_stream) {
        h->stream = (cudaStream_t)opts->cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete h;
            return cuda_error(e, "stream create");
        }
        h->own_stream = true;
    }
    h->tileX = choose_tile(g.nx, g.nu, h->sm_count);
    h->npairs = (int64_t)g.nx * g.nu;
    h->fast_wm = fast_wm(g, h->prec);
    // the register-resident kernels compute on-the-fly means inline for the
    // built-in systems only; a text system's on-the-fly rows take the generic
    // kernels, which read its mean tables
    if (g.sys == SYS_EXPR && tmode == AMY_T_ON_THE_FLY) h->fast_wm = 0;
    h->expr = prog;
    h->ulanes = 0;
    h->rows = 1;
    h->grouped = 0;
    h->runs = 0;
    h->bounds_known = 0;
    h->in_stride_b = INT_MIN;
    h->tilex = 0;
    h->box_floats = 0;
    h->use_plane = 1;
    h->plane_smem = 0;
    for (int d = 0; d < MAXD; ++d) h->spread[d] = -1;
    h->d_Vp[0] = h->d_Vp[1] = nullptr;
    h->vp_rows = 0;
    h->vp_pad = 0;
    h->vp_src = nullptr;
    {
        const int32_t *ls = opts->launch_shape;
        if (ls[0] < 0 || ls[0] > 8 || ls[1] < 0 || ls[1] > 512 || ls[1] % 32 != 0 ||
            (ls[0] > 0 && ls[1] > 0 && ls[0] * ls[1] > 512) || ls[2] < 0 || ls[2] > 2 ||
            (ls[3] != 0 && (ls[3] < 256 || ls[3] > 6144)) || ls[4] < 0 || ls[4] > 8) {
            free_handle(h);
            return set_error(AMY_E_INVALID_ARG, "bad launch shape");
        }
        h->ulanes = ls[0];
        h->tilex = ls[1];
        h->rows = ls[2] == 2 ? 0 : 1;
        h->box_floats = ls[3];
        h->outer = ls[4];
    }
    h->use_graphs = opts->use_graphs;
    h->host_params = params;
#define TRY(x)                 \
    do {                       \
        amy_status s__ = (x);  \
        if (s__ != AMY_OK) {   \
            free_handle(h);    \
            return s__;        \
        }                      \
    } while (0)
    TRY(dev_alloc(h, (void **)&h->d_params, params.size() * sizeof(double), "params"));
    h->g.params = h->d_params;
    for (int i = 0; i < 2; ++i) {
        const size_t vb = (size_t)(g.nx + 2 * kVGuard) * vsize(h);
        TRY(dev_alloc(h, &h->d_Vbase[i], vb, "V"));
        e = cudaMemsetAsync(h->d_Vbase[i], 0, vb, h->stream);
        if (e != cudaSuccess) {
            free_handle(h);
            return cuda_error(e, "V guard init");
        }
        h->d_V[i] = (char *)h->d_Vbase[i] + kVGuard * vsize(h);
    }
    TRY(dev_alloc(h, (void **)&h->d_mask, (size_t)g.nx, "mask"));
    if (h->tmode == AMY_T_STORED_SEPARABLE) {
        std::vector<int32_t> upart;
        TRY(plan_sep_tables(h->g, params, h->tab_words, &upart));
        h->grouped = input_runs_share_outer(h->g, upart);
        h->runs = input_outer_runs(h->g, upart);
        input_run_layout(h->g, upart, h->run_starts, h->in_stride_b);
        TRY(dev_alloc(h, (void **)&h->d_tab, (size_t)h->tab_words * 4, "separable tables"));
        if (h->fast_wm == 0 && g.n == 2 && std::max(g.W[0], g.W[1]) <= SEP2_WMAX) {
            // the per-state max keys of the wide 2-D kernel (zero between backups)
            const size_t kbytes = (size_t)g.nx * sizeof(unsigned long long);
            if (h->budget <= 0 || h->bytes + (int64_t)kbytes <= h->budget) {
                TRY(dev_alloc(h, &h->d_split, kbytes, "max keys"));
                e = cudaMemset(h->d_split, 0, kbytes);
                if (e != cudaSuccess) {
                    free_handle(h);
                    return cuda_error(e, "max keys init");
                }
                h->sep_wide = 1;
            }
        }
        e = cudaMemcpy(h->d_tab + h->g.uoff, upart.data(), upart.size() * 4, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            free_handle(h);
            return cuda_error(e, "table index upload");
        }
    } else if (h->tmode == AMY_T_ON_THE_FLY) {
        // wide windows on the fly: split each pair's window over up to 8
        // groups of rows, its masses shared in shared memory (at most 96 KiB)
        const int rows = g.wtot / g.W[g.n - 1];
        const size_t sbytes = (size_t)h->npairs * rsize(h);
        const size_t smem = (size_t)g.wsum * 32 * (rsize(h) + sizeof(int32_t));
        if (!fast_path(h) && g.wtot >= 256 && rows >= 2 && smem <= 96 * 1024 && split_pays(h) &&
            (h->budget <= 0 || h->bytes + (int64_t)sbytes <= h->budget)) {
            TRY(dev_alloc(h, &h->d_split, sbytes, "pair sums"));
            h->split_groups = std::min(rows, ROWS_MAX_GROUPS);
        }
    } else {
        const int64_t per_pair = (h->tmode == AMY_T_STORED_FULL) ? g.wtot : g.wsum;
        TRY(dev_alloc(h, &h->d_T, (size_t)(h->npairs * per_pair) * rsize(h), "stored T"));
        TRY(dev_alloc(h, (void **)&h->d_O, (size_t)(h->npairs * g.n) * sizeof(int16_t), "stored origins"));
        // wide stored rows with few pairs: the build runs per (slot, pair)
        // (full rows need the per-slot masses in a buffer of their own, when
        // it fits the budget), and the backup splits each pair's window over
        // up to 8 groups of rows when the pair sums fit (else one thread per
        // pair does each)
        const int rows = g.wtot / g.W[g.n - 1];
        if (g.wtot >= 256 && split_pays(h)) {
            if (h->tmode == AMY_T_STORED_FACTORED) {
                h->slot_build = 1;
            } else {
                const size_t fbytes = (size_t)h->npairs * g.wsum * rsize(h);
                if (h->budget <= 0 || h->bytes + (int64_t)fbytes <= h->budget) {
                    TRY(dev_alloc(h, &h->d_bfac, fbytes, "per-slot masses"));
                    h->slot_build = 1;
                }
            }
        }
        const size_t sbytes = (size_t)h->npairs * rsize(h);
        if (g.wtot >= 256 && rows >= 2 && split_pays(h) &&
            (h->budget <= 0 || h->bytes + (int64_t)sbytes <= h->budget)) {
            TRY(dev_alloc(h, &h->d_split, sbytes, "pair sums"));
            h->split_groups = std::min(rows, ROWS_MAX_GROUPS);
        }
    }
    e = cudaMemcpyAsync(h->d_params, params.data(), params.size() * sizeof(double), cudaMemcpyHostToDevice,
                        h->stream);
    if (e != cudaSuccess) {
        free_handle(h);
        return cuda_error(e, "params upload");
    }
    if (h->g.noise == NOISE_USER) {
        // the user densities' CDF tables, before anything computes a mass
        TRY(dev_alloc(h, (void **)&h->d_ucdf, (size_t)h->g.n * 2 * (USER_KNOTS + 1) * sizeof(double),
                      "user density tables"));
        h->g.ucdf = h->d_ucdf;
        TRY(user_tables(sys->noise->pdf, h->g, h->d_ucdf, h->stream));
    }
    if (h->g.sys == SYS_EXPR) {
        // mean tables of the text system, indexed like the per-dimension tables
        if (h->tmode != AMY_T_STORED_SEPARABLE) {
            uint32_t Sx[MAXD], Su[MAXD];
            system_deps(h->g, params, Sx, Su);
            TRY(table_strides(h->g, Sx, Su));
        }
        int64_t tot = 0;
        for (int d = 0; d < h->g.n; ++d) {
            h->g.moff[d] = tot;
            tot += h->g.tent[d];
        }
        TRY(dev_alloc(h, (void **)&h->d_mtab, (size_t)tot * sizeof(double), "mean tables"));
        h->g.mtab = h->d_mtab;
        TRY(expr_fill_means(h->expr, h->g, h->d_mtab, h->stream));
    }
    if (h->tmode != AMY_T_ON_THE_FLY) {
        if (h->prec == AMY_PREC_FP64)
            TRY(launch_build<double>(h));
        else
            TRY(launch_build<float>(h));
    }
    // The params upload reads pageable host memory owned by `params`: make
    // sure it has completed before that vector goes away.
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        free_handle(h);
        return cuda_error(e, "build");
    }
    {
        int64_t rows = 0;
        int32_t Ppad = 0;
        if (plane_structure(h->g, tm_kind_of(h), h->prec, rows, Ppad)) {
            // the plane kernel's padded V copies (pads stay zero)
            const size_t vb = (size_t)rows * Ppad * vsize(h);
            for (int i = 0; i < 2; ++i) {
                TRY(dev_alloc(h, &h->d_Vp[i], vb, "padded V"));
                e = cudaMemsetAsync(h->d_Vp[i], 0, vb, h->stream);
                if (e != cudaSuccess) {
                    free_handle(h);
                    return cuda_error(e, "padded V init");
                }
            }
            h->vp_rows = rows;
            h->vp_pad = Ppad;
        }
    }
    TRY(read_bounds(h));
    h->spin_limit = 1 << 20;
    h->grid_barrier = 1;
    h->synth_ok = 0;
    if (fast_path(h) && h->tmode == AMY_T_STORED_SEPARABLE && h->grouped) {
        TRY(dev_alloc(h, (void **)&h->d_bar, kBarWords * sizeof(unsigned), "barrier words"));
        h->h_err = pinned_words().take();
        if (!h->h_err) {
            free_handle(h);
            return set_error(AMY_E_CUDA, "barrier flag host word: page-locked allocation failed");
        }
        e = cudaMemsetAsync(h->d_bar, 0, kBarWords * sizeof(unsigned), h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) {
            free_handle(h);
            return cuda_error(e, "barrier words");
        }
    }
    if (opts->autotune) TRY(autotune_shape(h));
    h->vp_src = nullptr;
    update_synth_ok(h);
#undef TRY
    amy_info_t &inf = h->info;
    memset(&inf, 0, sizeof inf);
    inf.n_states = g.nx;
    inf.n_inputs = g.nu / g.nw;
    inf.n_disturbances = g.nw;
    inf.n = g.n;
    for (int d = 0; d < g.n; ++d) {
        inf.window[d] = g.W[d];
        inf.cut_half_width[d] = g.xs[d];
    }
    inf.window_slots = g.wtot;
    inf.window_sum = g.wsum;
    inf.tmode = h->tmode;
    inf.prec = h->prec;
    inf.v_store = h->v_store;
    if (fast_path(h)) {
        const FastCall c = fast_call(h, SPEC_SAFETY, nullptr, nullptr, nullptr, nullptr);
        const FastShape sh = fast_shape(h->g, tm_kind_of(h), c, h->sm_count);
        inf.input_lanes = sh.ulanes;
        inf.row_tiles = sh.rowtile > 0;
        inf.block_states = sh.tilex;
        inf.grouped_inputs = sh.staged && h->grouped;
        inf.tile_outer_rows = sh.runs ? sh.outer : 1;
    }
    *out = h;
    return AMY_OK;
}

amy_status amy_info(amy_handle h, amy_info_t *out) {
    if (!h || !out) return set_error(AMY_E_INVALID_ARG, "null argument");
    *out = h->info;
    out->device_bytes = h->bytes + (int64_t)h->stage_cap;
    out->step_wait = h->grid_barrier;
    out->backup_kernel = h->d_split ? (h->sep_wide ? 9 : 6) : 0;
    out->backup_launch_kernels = h->d_split ? 2 : 1;
    out->inner_span = 0;
    if (fast_path(h) && h->use_plane && h->plane.ok && h->tmode == AMY_T_STORED_SEPARABLE) {
        const bool tile = tile_on(h);
        out->backup_kernel = tile ? 8 : 7;
        out->input_lanes = 1;
        out->row_tiles = 0;
        out->block_states = tile ? h->plane.tT * h->plane.P : h->plane.G * h->plane.P;
        out->grouped_inputs = 0;
    } else if (fast_path(h)) {
        const FastCall c = fast_call(h, SPEC_SAFETY, nullptr, nullptr, nullptr, nullptr);
        const FastShape sh = fast_shape(h->g, tm_kind_of(h), c, h->sm_count);
        out->backup_kernel = sh.staged ? 2 : 1;
        if (sh.staged && h->grouped && h->tmode == AMY_T_STORED_SEPARABLE) {
            // the per-run pass runs when every dim has origin bounds and the
            // inner dim's bounds span at most WM + 3 slots (the kernel's test)
            int32_t b[2 * MAXD + 4];
            AMY_CUDA(cudaMemcpyAsync(b, h->d_tab + h->g.boff, sizeof b, cudaMemcpyDeviceToHost, h->stream),
                     "bounds read");
            AMY_CUDA(cudaStreamSynchronize(h->stream), "bounds read");
            const int L = h->g.n - 1, wm = h->fast_wm;
            const int32_t K = b[MAXD + L] - b[L] + wm;
            const bool all = (b[2 * MAXD] & ((1 << h->g.n) - 1)) == ((1 << h->g.n) - 1);
            if (all && K >= wm && K <= wm + 3 && K <= h->g.N[L]) {
                out->backup_kernel = h->synth_ok ? 5 : sh.runs ? 4 : 3;
                out->inner_span = K;
            }
        }
    }
    out->input_runs = h->runs;
    out->build_kernels = h->tmode == AMY_T_ON_THE_FLY ? 0
                         : h->tmode != AMY_T_STORED_SEPARABLE ? (h->slot_build && h->tmode == AMY_T_STORED_FULL ? 2 : 1)
                         : 2 + ((h->g.shoff > 0 && h->g.tsx[h->g.n - 1][h->g.n - 1] != 0) ? 1 : 0) +
                               (h->g.n >= 4 ? 1 : 0);
    return AMY_OK;
}

void amy_destroy(amy_handle h) { free_handle(h); }

amy_status amy_rebuild(amy_handle h, const double *params, int64_t n_params) {
    if (!h) return set_error(AMY_E_INVALID_ARG, "null handle");
    if (params) {
        if (n_params != (int64_t)h->host_params.size())
            return set_error(AMY_E_INVALID_ARG, "rebuild needs %lld parameters", (long long)h->host_params.size());
        for (int64_t i = 0; i < n_params; ++i)
            if (!std::isfinite(params[i])) return set_error(AMY_E_INVALID_ARG, "non-finite system parameter");
        if (h->tmode == AMY_T_STORED_SEPARABLE) {
            // the dependency sets (hence the table layout) must not change
            Geom g2 = h->g;
            std::vector<double> p2(params, params + n_params);
            int64_t words = 0;
            amy_status st = plan_sep_tables(g2, p2, words, nullptr);
            if (st != AMY_OK) return st;
            if (words != h->tab_words || memcmp(g2.tsx, h->g.tsx, sizeof g2.tsx) != 0 ||
                memcmp(g2.tsu, h->g.tsu, sizeof g2.tsu) != 0)
                return set_error(AMY_E_INVALID_ARG, "new parameters change the table layout; build a new handle");
        }
        h->host_params.assign(params, params + n_params);
        AMY_CUDA(cudaMemcpyAsync(h->d_params, h->host_params.data(), n_params * sizeof(double),
                                 cudaMemcpyHostToDevice, h->stream), "params upload");
        if (h->g.sys == SYS_EXPR) {
            const amy_status st = expr_fill_means(h->expr, h->g, h->d_mtab, h->stream);
            if (st != AMY_OK) return st;
            h->graph_valid = false;
        }
    }
    if (h->tmode == AMY_T_ON_THE_FLY) return AMY_OK;
    amy_status st = h->prec == AMY_PREC_FP64 ? launch_build<double>(h) : launch_build<float>(h);
    // new parameters may move the window origins: refresh the host copy of the bounds
    if (st == AMY_OK && params) {
        st = read_bounds(h);
        if (st == AMY_OK) update_synth_ok(h);
        h->graph_valid = false;
    }
    return st;
}

amy_status amy_set_wait_limit(amy_handle h, int32_t polls) {
    if (!h) return set_error(AMY_E_INVALID_ARG, "null handle");
    h->spin_limit = polls < 0 ? (1 << 20) : polls;
    h->graph_valid = false;
    return AMY_OK;
}

amy_status amy_set_step_wait(amy_handle h, int32_t mode) {
    if (!h) return set_error(AMY_E_INVALID_ARG, "null handle");
    if (mode != 0 && mode != 1) return set_error(AMY_E_INVALID_ARG, "step wait mode %d (0 or 1)", (int)mode);
    h->grid_barrier = mode;
    h->graph_valid = false;
    return AMY_OK;
}

amy_status amy_set_plane(amy_handle h, int32_t on, int32_t smem_bytes) {
    if (!h) return set_error(AMY_E_INVALID_ARG, "null handle");
    if (on < 0 || on > 3) return set_error(AMY_E_INVALID_ARG, "plane mode %d (0 .. 3)", (int)on);
    if (smem_bytes != 0 && (smem_bytes < 16 * 1024 || smem_bytes > 200 * 1024))
        return set_error(AMY_E_INVALID_ARG, "plane kernel shared memory %d bytes (0, or 16 KiB..200 KiB)",
                         (int)smem_bytes);
    h->use_plane = on;
    h->plane_smem = smem_bytes;
    if (h->tmode == AMY_T_STORED_SEPARABLE)
        plan_plane(h->g, TM_SEPARABLE, h->prec, h->spread, h->plane_smem, h->plane);
    h->graph_valid = false;
    return AMY_OK;
}

amy_status amy_backup_work(amy_handle h, const amy_spec *spec, int64_t *v_loads, int64_t *box_loads,
                           int64_t *box_rows) {
    if (!h || !spec || !v_loads || !box_loads || !box_rows) return set_error(AMY_E_INVALID_ARG, "null argument");
    if (!(fast_path(h) && h->use_plane && h->plane.ok && h->tmode == AMY_T_STORED_SEPARABLE))
        return set_error(AMY_E_UNSUPPORTED, "work counters exist for the plane kernel (backup kernel 7) only");
    SpecDev s;
    amy_status st = make_spec(h->g, spec, s);
    if (st != AMY_OK) return st;
    unsigned long long *d_work = nullptr;
    AMY_CUDA(cudaMallocAsync((void **)&d_work, 4 * sizeof(unsigned long long), h->stream), "work counters");
    cudaError_t e = cudaMemsetAsync(d_work, 0, 4 * sizeof(unsigned long long), h->stream);
    if (e == cudaSuccess) {
        st = launch_mask_any(h, s, h->d_V[0]);
        if (st == AMY_OK) st = launch_backup(h, s.kind, h->d_V[0], h->d_V[1], nullptr, nullptr, d_work);
    }
    unsigned long long w[4] = {0, 0, 0, 0};
    if (e == cudaSuccess && st == AMY_OK) e = cudaMemcpyAsync(w, d_work, sizeof w, cudaMemcpyDeviceToHost, h->stream);
    cudaFreeAsync(d_work, h->stream);
    const cudaError_t e2 = cudaStreamSynchronize(h->stream);
    if (st != AMY_OK) return st;
    if (e != cudaSuccess) return cuda_error(e, "work counters");
    if (e2 != cudaSuccess) return cuda_error(e2, "work counters");
    *v_loads = (int64_t)w[0];
    *box_loads = (int64_t)w[1];
    *box_rows = (int64_t)w[2];
    return AMY_OK;
}

amy_status amy_set_profiling(amy_handle h, int32_t on) {
    if (!h) return set_error(AMY_E_INVALID_ARG, "null handle");
    h->profiling = on != 0;
    return AMY_OK;
}

amy_status amy_kernel_times(amy_handle h, double *backup_ms, int64_t *backup_launches, int64_t *backup_steps,
                            double *build_ms, int64_t *build_launches) {
    if (!h) return set_error(AMY_E_INVALID_ARG, "null handle");
    if (backup_steps) {
        int64_t n = 0;
        for (int32_t k : h->ev_backup_steps) n += k;
        *backup_steps = n;
    }
    h->ev_backup_steps.clear();
    auto drain = [&](std::vector<std::pair<cudaEvent_t, cudaEvent_t>> &l, double *ms, int64_t *cnt) -> amy_status {
        double tot = 0.0;
        for (auto &p : l) {
            cudaError_t e = cudaEventSynchronize(p.second);
            float t = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, p.first, p.second);
            if (e != cudaSuccess) return cuda_error(e, "kernel timing");
            tot += t;
        }
        if (ms) *ms = tot;
        if (cnt) *cnt = (int64_t)l.size();
        for (auto &p : l) h->ev_pool.push_back(p.first), h->ev_pool.push_back(p.second);
        l.clear();
        return AMY_OK;
    };
    amy_status st = drain(h->ev_backup, backup_ms, backup_launches);
    if (st == AMY_OK) st = drain(h->ev_build, build_ms, build_launches);
    if (st == AMY_OK) st = check_synth_error(h);
    return st;
}

}  // extern "C"

namespace {

// The horizon loop of Algorithm 4 on the handle's stream: spec mask and V_N,
// then backups k = N-1..0 ping-ponging between the two resident V vectors;
// the last one writes V_0 into d_Vout.
amy_status enqueue_synthesis(amy_handle_s *h, const SpecDev &s, int32_t horizon, void *d_Vout, uint16_t *d_pi,
                             int32_t all_steps) {
    const int64_t nx = h->g.nx;
    amy_status st = launch_mask_any(h, s, h->d_V[0]);
    if (st != AMY_OK) return st;
    if (h->synth_ok && horizon > 0) {
        // the whole horizon in one persistent launch
        AMY_CUDA(cudaMemsetAsync(h->d_bar, 0, kBarResetBytes, h->stream), "barrier reset");
        const FastCall c = fast_call(h, s.kind, h->d_V[0], h->d_V[1], nullptr, nullptr);
        const SynthCall sc = synth_call(h, horizon, d_Vout, d_pi, all_steps);
        KernelTimer tm(h, &h->ev_backup, horizon);
        st = launch_synth_fast(h->g, tm_kind_of(h), h->v_store, c, sc, h->sm_count, h->stream, false);
        tm.done();
        return st;
    }
    int cur = 0;
    for (int32_t k = horizon - 1; k >= 0; --k) {
        uint16_t *pk = nullptr;
        if (d_pi) pk = all_steps ? d_pi + (int64_t)k * nx : (k == 0 ? d_pi : nullptr);
        void *vfinal = (k == 0) ? d_Vout : nullptr;
        st = launch_backup(h, s.kind, h->d_V[cur], h->d_V[cur ^ 1], vfinal, pk);
        if (st != AMY_OK) return st;
        cur ^= 1;
    }
    if (horizon == 0) {
        // V_0 = V_N: convert the initial vector into the output type.
        if (h->prec == AMY_PREC_FP64 || h->v_store == AMY_V_NATIVE) {
            AMY_CUDA(cudaMemcpyAsync(d_Vout, h->d_V[0], (size_t)nx * rsize(h), cudaMemcpyDeviceToDevice, h->stream),
                     "copy V_N");
        } else {
            st = launch_v16_to_f32(h->d_V[0], h->v_store, (float *)d_Vout, nx, h->stream);
            if (st != AMY_OK) return st;
        }
    }
    return AMY_OK;
}

// Replays the cached graph of the horizon loop when the call repeats the
// previous one (same spec, horizon, outputs); otherwise captures a new one on
// a private stream and instantiates it.
amy_status synthesize_graph(amy_handle_s *h, const SpecDev &s, int32_t horizon, void *d_Vout, uint16_t *d_pi,
                            int32_t all_steps) {
    const bool hit = h->graph_valid && memcmp(&h->g_spec, &s, sizeof s) == 0 && h->g_horizon == horizon &&
                     h->g_vout == d_Vout && h->g_pi == d_pi && h->g_all == all_steps;
    if (!hit) {
        if (!h->cap_stream) AMY_CUDA(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking), "capture stream");
        if (h->graph_exec) {
            cudaGraphExecDestroy(h->graph_exec);
            h->graph_exec = nullptr;
        }
        h->graph_valid = false;
        cudaStream_t user = h->stream;
        AMY_CUDA(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed), "begin capture");
        h->stream = h->cap_stream;
        amy_status st = enqueue_synthesis(h, s, horizon, d_Vout, d_pi, all_steps);
        h->stream = user;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
        if (st != AMY_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph_exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_error(e, "graph capture");
        h->graph_valid = true;
        h->g_spec = s;
        h->g_horizon = horizon;
        h->g_vout = d_Vout;
        h->g_pi = d_pi;
        h->g_all = all_steps;
    }
    AMY_CUDA(cudaGraphLaunch(h->graph_exec, h->stream), "graph launch");
    return AMY_OK;
}

// Rows of `count` device-given pairs (x[i], u[i]) as the handle's mode
// computes them (k_query_rows): window origins and prod-W FP64 masses.
cudaError_t enqueue_rows(amy_handle_s *h, const int64_t *dx, const int64_t *du, int64_t count, int32_t *dor,
                         double *dpr) {
    const Geom &g = h->g;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((count + 127) / 128, 4096));
    if (h->prec == AMY_PREC_FP64)
        k_query_rows<double><<<blocks, 128, 0, h->stream>>>(g, h->tmode, (const double *)h->d_T, h->d_O, h->npairs,
                                                            h->d_tab, dx, du, count, dor, dpr);
    else
        k_query_rows<float><<<blocks, 128, 0, h->stream>>>(g, h->tmode, (const float *)h->d_T, h->d_O, h->npairs,
                                                           h->d_tab, dx, du, count, dor, dpr);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

amy_status amy_synthesize(amy_handle h, const amy_spec *spec, int32_t horizon, void *V_out,
                          uint16_t *policy_out, int32_t policy_all_steps, int32_t outputs_on_device) {
    if (!h || !V_out) return set_error(AMY_E_INVALID_ARG, "null argument");
    if (horizon < 0) return set_error(AMY_E_INVALID_ARG, "negative horizon");
    SpecDev s;
    amy_status st = make_spec(h->g, spec, s);
    if (st != AMY_OK) return st;
    const int64_t nx = h->g.nx;
    const size_t osz = rsize(h);
    // Outputs: V_0 is written by the last backup straight into the output
    // buffer (device) or a staging buffer (host).
    void *d_Vout = nullptr;
    uint16_t *d_pi = nullptr;
    // host outputs the kernels write in place (page-locked, device-mapped):
    // their copy-out then overlaps the backups
    bool v_direct = false, pi_direct = false;
    if (outputs_on_device) {
        d_Vout = V_out;
        d_pi = policy_out;
    } else {
        if (horizon > 0) {
            d_Vout = mapped_host(V_out);
            v_direct = d_Vout != nullptr;
            if (policy_out) {
                d_pi = static_cast<uint16_t *>(mapped_host(policy_out));
                pi_direct = d_pi != nullptr;
            }
        }
        // the others in the handle's staging buffer: V_0, then the policies
        const size_t vbytes = v_direct ? 0 : ((size_t)nx * osz + 255) & ~(size_t)255;
        const size_t pbytes = policy_out && horizon > 0 && !pi_direct
                                  ? (size_t)nx * sizeof(uint16_t) * (policy_all_steps ? horizon : 1)
                                  : 0;
        if (vbytes + pbytes > 0) {
            void *buf = nullptr;
            st = stage_buffer(h, vbytes + pbytes, &buf);
            if (st != AMY_OK) return st;
            if (!v_direct) d_Vout = buf;
            if (pbytes) d_pi = reinterpret_cast<uint16_t *>(static_cast<unsigned char *>(buf) + vbytes);
        }
    }
    auto cleanup = [&]() {};
    if (outputs_on_device && h->use_graphs && !h->profiling && !(h->synth_ok && horizon > 0)) {
        st = synthesize_graph(h, s, horizon, d_Vout, d_pi, policy_all_steps);
    } else {
        st = enqueue_synthesis(h, s, horizon, d_Vout, d_pi, policy_all_steps);
    }
    if (st != AMY_OK) {
        cleanup();
        return st;
    }
    if (!outputs_on_device) {
        cudaError_t e = cudaSuccess;
        if (!v_direct) e = cudaMemcpyAsync(V_out, d_Vout, (size_t)nx * osz, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess && policy_out && horizon > 0 && !pi_direct)
            e = cudaMemcpyAsync(policy_out, d_pi, (size_t)nx * sizeof(uint16_t) * (policy_all_steps ? horizon : 1),
                                cudaMemcpyDeviceToHost, h->stream);
        // the persistent kernel's error flag rides on the same wait
        const bool persist = h->synth_ok && horizon > 0 && h->d_bar && h->h_err;
        if (persist) *h->h_err = 0;
        if (e == cudaSuccess && persist)
            e = cudaMemcpyAsync(h->h_err, h->d_bar + kBarErrWord, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                h->stream);
        cleanup();
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_error(e, "copy out");
        const int32_t err = persist ? *h->h_err : 0;
        if (err != 0) {
            AMY_CUDA(cudaMemsetAsync(h->d_bar + kBarErrWord, 0, sizeof(int32_t), h->stream), "barrier flag reset");
            if (err == 1) return set_error(AMY_E_TIMEOUT, "persistent backup: a grid barrier wait gave up");
            return set_error(AMY_E_CUDA, "persistent backup: launch shape rejected on the device");
        }
        if (policy_out && horizon == 0) {
            // no backup: no policy entries to report
        }
    } else {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_error(e, "synthesize");
    }
    return AMY_OK;
}

amy_status amy_backup_step(amy_handle h, const amy_spec *spec, const void *V_next, void *V_out,
                           uint16_t *policy_out, int32_t on_device) {
    if (!h || !V_next || !V_out) return set_error(AMY_E_INVALID_ARG, "null argument");
    SpecDev s;
    amy_status st = make_spec(h->g, spec, s);
    if (st != AMY_OK) return st;
    const int64_t nx = h->g.nx;
    const size_t osz = rsize(h);
    // The mask kernel also writes V_N into d_V[1]; the caller's V_next then
    // replaces it in d_V[0] (converted to the storage type).
    st = launch_mask_any(h, s, h->d_V[1]);
    if (st != AMY_OK) return st;
    const void *src = V_next;
    // host buffers: V_next, then V_k and pi_k, in the handle's staging buffer
    const size_t vbytes = ((size_t)nx * osz + 255) & ~(size_t)255;
    unsigned char *stage = nullptr;
    if (!on_device) {
        void *buf = nullptr;
        st = stage_buffer(h, 2 * vbytes + (size_t)nx * 2, &buf);
        if (st != AMY_OK) return st;
        stage = static_cast<unsigned char *>(buf);
        AMY_CUDA(cudaMemcpyAsync(stage, V_next, (size_t)nx * osz, cudaMemcpyHostToDevice, h->stream), "V_next upload");
        src = stage;
    }
    cudaError_t e = cudaSuccess;
    if (h->prec == AMY_PREC_FP64 || h->v_store == AMY_V_NATIVE)
        e = cudaMemcpyAsync(h->d_V[0], src, (size_t)nx * osz, cudaMemcpyDeviceToDevice, h->stream);
    else
        st = launch_f32_to_v16((const float *)src, h->d_V[0], h->v_store, nx, h->stream);
    if (e != cudaSuccess || st != AMY_OK) return e != cudaSuccess ? cuda_error(e, "V_next copy") : st;
    void *d_out = V_out;
    uint16_t *d_pi = policy_out;
    if (!on_device) {
        d_out = stage + vbytes;
        d_pi = policy_out ? reinterpret_cast<uint16_t *>(stage + 2 * vbytes) : nullptr;
    }
    st = launch_backup(h, s.kind, h->d_V[0], h->d_V[1], d_out, d_pi);
    if (st == AMY_OK && !on_device) {
        e = cudaMemcpyAsync(V_out, d_out, (size_t)nx * osz, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess && policy_out)
            e = cudaMemcpyAsync(policy_out, d_pi, (size_t)nx * 2, cudaMemcpyDeviceToHost, h->stream);
    }
    if (st != AMY_OK) return st;
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_error(e, "backup step");
    return AMY_OK;
}

amy_status amy_query_rows(amy_handle h, const int64_t *x, const int64_t *u, int64_t count,
                          int32_t *origin_out, double *probs_out) {
    if (!h || !x || !u || !origin_out || !probs_out || count < 0) return set_error(AMY_E_INVALID_ARG, "null argument");
    if (count == 0) return AMY_OK;
    for (int64_t i = 0; i < count; ++i)
        if (x[i] < 0 || x[i] >= h->g.nx || u[i] < 0 || u[i] >= h->g.nu)
            return set_error(AMY_E_INVALID_ARG, "pair %lld out of range", (long long)i);
    const Geom &g = h->g;
    int64_t *dx = nullptr, *du = nullptr;
    int32_t *dor = nullptr;
    double *dpr = nullptr;
    const size_t prb = (size_t)count * g.wtot * sizeof(double);
    cudaError_t e = cudaMallocAsync((void **)&dx, count * 8, h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&du, count * 8, h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&dor, count * g.n * 4, h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&dpr, prb, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dx, x, count * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(du, u, count * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = enqueue_rows(h, dx, du, count, dor, dpr);
    if (e == cudaSuccess) e = cudaMemcpyAsync(origin_out, dor, count * g.n * 4, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(probs_out, dpr, prb, cudaMemcpyDeviceToHost, h->stream);
    if (dx) cudaFreeAsync(dx, h->stream);
    if (du) cudaFreeAsync(du, h->stream);
    if (dor) cudaFreeAsync(dor, h->stream);
    if (dpr) cudaFreeAsync(dpr, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_error(e, "query rows");
    return AMY_OK;
}

amy_status amy_simulate(amy_handle h, const amy_spec *spec, int32_t horizon, const uint16_t *policy,
                        const int64_t *x0, int64_t n_x0, int64_t runs_per_x0, uint64_t seed,
                        int64_t *successes_out, int32_t on_device) {
    if (!h || !successes_out || (n_x0 > 0 && !x0) || (horizon > 0 && !policy))
        return set_error(AMY_E_INVALID_ARG, "null argument");
    if (horizon < 0 || n_x0 < 0 || runs_per_x0 < 0) return set_error(AMY_E_INVALID_ARG, "negative count");
    if (runs_per_x0 > 0 && n_x0 > ((int64_t)1 << 62) / runs_per_x0)
        return set_error(AMY_E_INVALID_ARG, "more than 2^62 runs");
    SpecDev s;
    amy_status st = make_spec(h->g, spec, s);
    if (st != AMY_OK) return st;
    if (n_x0 == 0) return AMY_OK;
    const Geom &g = h->g;
    if (!on_device)
        for (int64_t i = 0; i < n_x0; ++i)
            if (x0[i] < 0 || x0[i] >= g.nx)
                return set_error(AMY_E_INVALID_ARG, "initial state %lld out of range", (long long)i);
    const size_t pbytes = (size_t)horizon * (size_t)g.nx * sizeof(uint16_t);
    const uint16_t *d_pi = policy;
    const int64_t *d_x0 = x0;
    unsigned long long *d_succ = reinterpret_cast<unsigned long long *>(successes_out);
    uint16_t *own_pi = nullptr;
    int64_t *own_x0 = nullptr;
    unsigned long long *own_succ = nullptr;
    unsigned int *d_err = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&d_err, sizeof(unsigned int), h->stream);
    if (e == cudaSuccess && !on_device) {
        if (pbytes) e = cudaMallocAsync((void **)&own_pi, pbytes, h->stream);
        if (e == cudaSuccess) e = cudaMallocAsync((void **)&own_x0, (size_t)n_x0 * 8, h->stream);
        if (e == cudaSuccess) e = cudaMallocAsync((void **)&own_succ, (size_t)n_x0 * 8, h->stream);
        if (e == cudaSuccess && pbytes) e = cudaMemcpyAsync(own_pi, policy, pbytes, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(own_x0, x0, (size_t)n_x0 * 8, cudaMemcpyHostToDevice, h->stream);
        d_pi = own_pi;
        d_x0 = own_x0;
        d_succ = own_succ;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(unsigned int), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_succ, 0, (size_t)n_x0 * 8, h->stream);
    if (e == cudaSuccess) {
        st = launch_mask_any(h, s, h->d_V[0]);
        if (st == AMY_OK)
            st = launch_simulate(g, s.kind, h->d_mask, d_pi, horizon, d_x0, n_x0, runs_per_x0, seed, d_succ, d_err,
                                 h->sm_count, h->stream);
    }
    unsigned int err = 0;
    if (e == cudaSuccess && st == AMY_OK) e = cudaMemcpyAsync(&err, d_err, sizeof err, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && st == AMY_OK && !on_device)
        e = cudaMemcpyAsync(successes_out, own_succ, (size_t)n_x0 * 8, cudaMemcpyDeviceToHost, h->stream);
    if (d_err) cudaFreeAsync(d_err, h->stream);
    if (own_pi) cudaFreeAsync(own_pi, h->stream);
    if (own_x0) cudaFreeAsync(own_x0, h->stream);
    if (own_succ) cudaFreeAsync(own_succ, h->stream);
    const cudaError_t e2 = cudaStreamSynchronize(h->stream);
    if (st != AMY_OK) return st;
    if (e != cudaSuccess) return cuda_error(e, "simulate");
    if (e2 != cudaSuccess) return cuda_error(e2, "simulate");
    if (err & 1u) return set_error(AMY_E_INVALID_ARG, "an initial state is out of range");
    if (err & 2u) return set_error(AMY_E_INVALID_ARG, "the policy names an input >= %d at a live state", g.nu / g.nw);
    return AMY_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Export of the finite MDP in PRISM's explicit-model files (the tool's PRISM
// export of the abstraction, Sec. 2): .tra (transitions), .lab (labels),
// .sta (state coordinates) and .props (the bounded-horizon property whose
// maximal probability is V_0).
// ---------------------------------------------------------------------------
namespace {

struct FileCloser {
    std::FILE *f = nullptr;
    ~FileCloser() {
        if (f) std::fclose(f);
    }
};

amy_status open_out(const std::string &path, FileCloser &fc) {
    fc.f = std::fopen(path.c_str(), "wb");
    if (!fc.f) return set_error(AMY_E_INVALID_ARG, "cannot open %s for writing", path.c_str());
    return AMY_OK;
}

amy_status close_out(const std::string &path, FileCloser &fc) {
    const bool bad = std::ferror(fc.f) != 0;
    const int rc = std::fclose(fc.f);
    fc.f = nullptr;
    if (bad || rc != 0) return set_error(AMY_E_INVALID_ARG, "write to %s failed", path.c_str());
    return AMY_OK;
}

// Writes the .tra body for every (state, input) pair, rows from the handle's
// own abstraction computed on the device in batches; returns the number of
// transitions written.  A row's slots that land on one cell (a periodic
// window wider than its ring) are merged; the mass the cut or the grid's
// edge removes goes to the sink state nx.
amy_status write_transitions(amy_handle_s *h, std::FILE *f, int64_t &n_trans) {
    const Geom &g = h->g;
    const int64_t nx = g.nx, nu = g.nu, wt = g.wtot;
    const int64_t npair = nx * nu;
    const int64_t batch = std::max<int64_t>(1, std::min<int64_t>(npair, ((int64_t)32 << 20) / (wt * 8)));
    std::vector<int64_t> hx((size_t)batch), hu((size_t)batch);
    std::vector<int32_t> horg((size_t)(batch * g.n));
    std::vector<double> hpr((size_t)(batch * wt));
    int64_t *dx = nullptr, *du = nullptr;
    int32_t *dor = nullptr;
    double *dpr = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&dx, (size_t)batch * 8, h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&du, (size_t)batch * 8, h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&dor, (size_t)(batch * g.n) * 4, h->stream);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&dpr, (size_t)(batch * wt) * 8, h->stream);
    std::vector<std::pair<int64_t, double>> row((size_t)wt);
    n_trans = 0;
    for (int64_t p0 = 0; p0 < npair && e == cudaSuccess; p0 += batch) {
        const int64_t cnt = std::min(batch, npair - p0);
        for (int64_t i = 0; i < cnt; ++i) {
            hx[(size_t)i] = (p0 + i) / nu;
            hu[(size_t)i] = (p0 + i) % nu;
        }
        e = cudaMemcpyAsync(dx, hx.data(), (size_t)cnt * 8, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(du, hu.data(), (size_t)cnt * 8, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = enqueue_rows(h, dx, du, cnt, dor, dpr);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(horg.data(), dor, (size_t)(cnt * g.n) * 4, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(hpr.data(), dpr, (size_t)(cnt * wt) * 8, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) break;
        for (int64_t i = 0; i < cnt; ++i) {
            const int32_t *org = &horg[(size_t)(i * g.n)];
            const double *pr = &hpr[(size_t)(i * wt)];
            size_t nr = 0;
            double sum = 0.0;
            int32_t k[MAXD] = {0};
            for (int64_t t = 0; t < wt; ++t) {
                if (pr[t] > 0.0) {
                    int64_t tgt = 0;
                    bool on = true;
                    for (int d = 0; d < g.n; ++d) {
                        int32_t c = org[d] + k[d];
                        if ((g.periodic >> d) & 1u) c = ((c % g.N[d]) + g.N[d]) % g.N[d];
                        else if (c < 0 || c >= g.N[d]) on = false;
                        tgt += (int64_t)c * g.stride[d];
                    }
                    if (on) {
                        row[nr++] = {tgt, pr[t]};
                        sum += pr[t];
                    }
                }
                for (int d = g.n - 1; d >= 0; --d) {
                    if (++k[d] < g.W[d]) break;
                    k[d] = 0;
                }
            }
            std::sort(row.begin(), row.begin() + (std::ptrdiff_t)nr);
            const int64_t x = hx[(size_t)i], u = hu[(size_t)i];
            for (size_t j = 0; j < nr;) {
                const int64_t tgt = row[j].first;
                double v = 0.0;
                for (; j < nr && row[j].first == tgt; ++j) v += row[j].second;
                std::fprintf(f, "%lld %lld %lld %.17g\n", (long long)x, (long long)u, (long long)tgt, v);
                ++n_trans;
            }
            const double lost = 1.0 - sum;
            if (lost > 0.0) {
                std::fprintf(f, "%lld %lld %lld %.17g\n", (long long)x, (long long)u, (long long)nx, lost);
                ++n_trans;
            }
        }
    }
    if (dx) cudaFreeAsync(dx, h->stream);
    if (du) cudaFreeAsync(du, h->stream);
    if (dor) cudaFreeAsync(dor, h->stream);
    if (dpr) cudaFreeAsync(dpr, h->stream);
    const cudaError_t e2 = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_error(e, "export rows");
    if (e2 != cudaSuccess) return cuda_error(e2, "export rows");
    return AMY_OK;
}

}  // namespace

extern "C" {

amy_status amy_export_prism(amy_handle h, const amy_spec *spec, int32_t horizon, const char *path_prefix,
                            int64_t *n_transitions_out) {
    if (!h || !spec || !path_prefix || !*path_prefix) return set_error(AMY_E_INVALID_ARG, "null argument");
    if (horizon < 0) return set_error(AMY_E_INVALID_ARG, "negative horizon");
    const Geom &g = h->g;
    if (g.nw > 1)
        return set_error(AMY_E_UNSUPPORTED, "a disturbance grid makes the model a stochastic game, not an MDP");
    SpecDev s;
    amy_status st = make_spec(g, spec, s);
    if (st != AMY_OK) return st;
    const int64_t nx = g.nx, nu = g.nu;
    std::vector<uint8_t> mask((size_t)nx);
    st = launch_mask_any(h, s, h->d_V[0]);
    if (st != AMY_OK) return st;
    AMY_CUDA(cudaMemcpyAsync(mask.data(), h->d_mask, (size_t)nx, cudaMemcpyDeviceToHost, h->stream), "export mask");
    AMY_CUDA(cudaStreamSynchronize(h->stream), "export mask");
    const std::string pre(path_prefix);
    // transitions: body to a part file, then the header and the body
    const std::string tra = pre + ".tra", part = pre + ".tra.part";
    int64_t n_trans = 0;
    {
        FileCloser fc;
        if ((st = open_out(part, fc)) != AMY_OK) return st;
        st = write_transitions(h, fc.f, n_trans);
        if (st != AMY_OK) {
            std::fclose(fc.f);
            fc.f = nullptr;
            std::remove(part.c_str());
            return st;
        }
        std::fprintf(fc.f, "%lld 0 %lld 1\n", (long long)nx, (long long)nx);  // the sink: absorbing
        ++n_trans;
        if ((st = close_out(part, fc)) != AMY_OK) return st;
    }
    {
        FileCloser out, in;
        if ((st = open_out(tra, out)) != AMY_OK) return st;
        std::fprintf(out.f, "%lld %lld %lld\n", (long long)(nx + 1), (long long)(nx * nu + 1), (long long)n_trans);
        in.f = std::fopen(part.c_str(), "rb");
        if (!in.f) return set_error(AMY_E_INVALID_ARG, "cannot reopen %s", part.c_str());
        std::vector<char> buf(1 << 20);
        size_t got;
        while ((got = std::fread(buf.data(), 1, buf.size(), in.f)) > 0) std::fwrite(buf.data(), 1, got, out.f);
        std::fclose(in.f);
        in.f = nullptr;
        if ((st = close_out(tra, out)) != AMY_OK) return st;
        std::remove(part.c_str());
    }
    // labels: every grid state is initial; the sink carries only "sink"
    {
        const std::string lab = pre + ".lab";
        FileCloser fc;
        if ((st = open_out(lab, fc)) != AMY_OK) return st;
        std::fprintf(fc.f, "0=\"init\" 1=\"deadlock\" 2=\"target\" 3=\"avoid\" 4=\"safe\" 5=\"sink\"\n");
        for (int64_t x = 0; x < nx; ++x) {
            const uint8_t f = mask[(size_t)x];
            std::fprintf(fc.f, "%lld: 0%s%s%s\n", (long long)x, (f & F_TARGET) ? " 2" : "", (f & F_AVOID) ? " 3" : "",
                         (s.kind == SPEC_SAFETY && (f & F_SAFE)) ? " 4" : "");
        }
        std::fprintf(fc.f, "%lld: 5\n", (long long)nx);
        if ((st = close_out(lab, fc)) != AMY_OK) return st;
    }
    // state coordinates: grid indices per dim, the sink at -1
    {
        const std::string sta = pre + ".sta";
        FileCloser fc;
        if ((st = open_out(sta, fc)) != AMY_OK) return st;
        std::fprintf(fc.f, "(");
        for (int d = 0; d < g.n; ++d) std::fprintf(fc.f, d ? ",x%d" : "x%d", d);
        std::fprintf(fc.f, ")\n");
        for (int64_t x = 0; x <= nx; ++x) {
            std::fprintf(fc.f, "%lld:(", (long long)x);
            for (int d = 0; d < g.n; ++d) {
                const long long c = x < nx ? (long long)((x / g.stride[d]) % g.N[d]) : -1;
                std::fprintf(fc.f, d ? ",%lld" : "%lld", c);
            }
            std::fprintf(fc.f, ")\n");
        }
        if ((st = close_out(sta, fc)) != AMY_OK) return st;
    }
    // the property: V_0 is its maximal probability from every state
    {
        const std::string props = pre + ".props";
        FileCloser fc;
        if ((st = open_out(props, fc)) != AMY_OK) return st;
        if (s.kind == SPEC_SAFETY)
            std::fprintf(fc.f, "Pmax=? [ G<=%d \"safe\" ]\n", (int)horizon);
        else if (s.n_avoid > 0)
            std::fprintf(fc.f, "Pmax=? [ !\"avoid\" U<=%d \"target\" ]\n", (int)horizon);
        else
            std::fprintf(fc.f, "Pmax=? [ F<=%d \"target\" ]\n", (int)horizon);
        if ((st = close_out(props, fc)) != AMY_OK) return st;
    }
    if (n_transitions_out) *n_transitions_out = n_trans;
    return AMY_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// 16-bit V storage <-> float (used only at the boundary of a call: V_N output
// with horizon 0, caller-given V_next with 16-bit storage).
// ---------------------------------------------------------------------------
namespace amy {

template <class VT>
__global__ void k_v16_to_f32(const VT *__restrict__ s, float *__restrict__ d, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = vload<float, VT>(s + i);
}

template <class VT>
__global__ void k_f32_to_v16(const float *__restrict__ s, VT *__restrict__ d, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = vstore_cast<VT, float>(s[i]);
}

amy_status launch_v16_to_f32(const void *src, int32_t v_store, float *dst, int64_t n, cudaStream_t s) {
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 8192);
    if (v_store == AMY_V_BF16)
        k_v16_to_f32<__nv_bfloat16><<<blocks, 256, 0, s>>>((const __nv_bfloat16 *)src, dst, n);
    else
        k_v16_to_f32<unorm16><<<blocks, 256, 0, s>>>((const unorm16 *)src, dst, n);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AMY_OK : cuda_error(e, "16-bit V -> f32");
}

amy_status launch_f32_to_v16(const float *src, void *dst, int32_t v_store, int64_t n, cudaStream_t s) {
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 8192);
    if (v_store == AMY_V_BF16)
        k_f32_to_v16<__nv_bfloat16><<<blocks, 256, 0, s>>>(src, (__nv_bfloat16 *)dst, n);
    else
        k_f32_to_v16<unorm16><<<blocks, 256, 0, s>>>(src, (unorm16 *)dst, n);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AMY_OK : cuda_error(e, "f32 -> 16-bit V");
}

}  // namespace amy

// ---------------------------------------------------------------------------
// Launchers used by the serving scheduler (problems without a handle).
// ---------------------------------------------------------------------------
namespace amy {

amy_status launch_spec_mask(const Geom &g, const SpecDev &s, uint8_t *mask, void *VN, int v_store, cudaStream_t st) {
    const int blocks = (int)std::min<int64_t>((g.nx + 255) / 256, 65535);
    if (v_store == AMY_V_BF16)
        k_spec_mask<float, __nv_bfloat16><<<blocks, 256, 0, st>>>(g, s, mask, (__nv_bfloat16 *)VN);
    else if (v_store == AMY_V_UNORM16)
        k_spec_mask<float, unorm16><<<blocks, 256, 0, st>>>(g, s, mask, (unorm16 *)VN);
    else
        k_spec_mask<float, float><<<blocks, 256, 0, st>>>(g, s, mask, (float *)VN);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AMY_OK : cuda_error(e, "spec mask launch");
}

namespace {
template <class VT, int TM, bool KAHAN>
amy_status generic_fp32_t(const Geom &g, const FastCall &c, int sm_count, cudaStream_t st) {
    BackupArgs<float, VT> a;
    a.Vn = (const VT *)c.Vn;
    a.Vo = (VT *)c.Vo;
    a.Vfinal = c.Vfinal;
    a.pi = c.pi;
    a.mask = c.mask;
    a.spec_kind = c.spec_kind;
    a.tileX = choose_tile(g.nx, g.nu, sm_count);
    a.T = nullptr;
    a.O = nullptr;
    a.npairs = 0;
    a.tab = c.tab;
    const int blocks = (g.nx + a.tileX - 1) / a.tileX;
    const size_t smem = (size_t)a.tileX * g.nu * sizeof(float);
    k_backup<float, VT, TM, KAHAN><<<blocks, 256, smem, st>>>(g, a);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AMY_OK : cuda_error(e, "backup launch");
}

template <int TM>
amy_status generic_fp32_tm(const Geom &g, const FastCall &c, int v_store, int sm_count, cudaStream_t st) {
    if (v_store == AMY_V_BF16)
        return c.kahan ? generic_fp32_t<__nv_bfloat16, TM, true>(g, c, sm_count, st)
                       : generic_fp32_t<__nv_bfloat16, TM, false>(g, c, sm_count, st);
    if (v_store == AMY_V_UNORM16)
        return c.kahan ? generic_fp32_t<unorm16, TM, true>(g, c, sm_count, st)
                       : generic_fp32_t<unorm16, TM, false>(g, c, sm_count, st);
    return c.kahan ? generic_fp32_t<float, TM, true>(g, c, sm_count, st)
                   : generic_fp32_t<float, TM, false>(g, c, sm_count, st);
}
}  // namespace

amy_status launch_backup_generic_fp32(const Geom &g, int tm, const FastCall &c, int v_store, int sm_count,
                                      cudaStream_t st) {
    if (tm == TM_OTF) return generic_fp32_tm<TM_OTF>(g, c, v_store, sm_count, st);
    return generic_fp32_tm<TM_SEPARABLE>(g, c, v_store, sm_count, st);
}

}  // namespace amy

namespace amy {

int choose_tmode(const Geom &g, const std::vector<double> &params, int prec, int64_t budget) {
    const int64_t cap = budget > 0 ? budget / 4 : INT64_MAX;
    if (prec != AMY_PREC_FP64) {
        Geom g2 = g;
        int64_t words = 0;
        if (plan_sep_tables(g2, params, words, nullptr) == AMY_OK && words * 4 <= std::min(kAutoTableBytes, cap))
            return TM_SEPARABLE;
    }
    bool fits16 = true;
    for (int d = 0; d < g.n; ++d) fits16 = fits16 && (g.N[d] + g.W[d] + 2 <= 32767);
    const int64_t rsz = prec == AMY_PREC_FP64 ? 8 : 4;
    const int64_t fact = (int64_t)g.nx * g.nu * ((int64_t)g.wsum * rsz + 2 * g.n);
    if (fits16 && fact <= std::min(kAutoFactoredBytes, cap)) return TM_FACTORED;
    return TM_OTF;
}

amy_status launch_build_factored(const Geom &g, float *T, int16_t *O, int64_t npairs, int sm_count, cudaStream_t st) {
    const int blocks = (int)std::min<int64_t>((npairs + 127) / 128, (int64_t)sm_count * 32);
    k_build<float, TM_FACTORED><<<std::max(blocks, 1), 128, 0, st>>>(g, T, O, npairs);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? AMY_OK : cuda_error(e, "factored build launch");
}

}  // namespace amy
