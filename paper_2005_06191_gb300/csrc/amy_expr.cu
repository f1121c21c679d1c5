// amy_expr.cu -- systems given as text (Sec. 3: the user writes the
// right-hand side of x(k+1) = f(x(k), nu(k), w(k)) + noise in a
// configuration file).
//
// Each mean component f_d is one C-syntax arithmetic expression over the
// FP64 variables x0.. (state centre), u0.. (input point), w0.. (disturbance
// point) and p0.. (system parameters): numeric literals (doubles), unary + -,
// binary + - * / (left associative, * / binding tighter), parentheses and
// the calls sin cos tan asin acos atan sinh cosh tanh exp log log10 sqrt fabs
// floor ceil (one argument), atan2 pow fmin fmax (two).
//
// The host parses the text (precedence climbing), records which variables
// each component reads, and emits a CUDA kernel that evaluates every
// component once per record of its dependency-compressed mean table (the
// coordinates the component reads, as the per-dimension tables of the
// separable mode index them).  The kernel is compiled at run time with NVRTC
// (loaded with dlopen on first use, without fused multiply-add, so every
// operation is rounded as written) and kept per source text for the life of
// the process.  The backup, build and query kernels then read the means from
// the table (mean_of with SYS_EXPR).
#include <dlfcn.h>
#include <nvrtc.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "amy_internal.h"

namespace amy {

namespace {

// ---------------------------------------------------------------------------
// Parser: text -> fully parenthesised CUDA expression + dependency masks
// ---------------------------------------------------------------------------
struct Fn {
    const char *name;
    int arity;
};
constexpr Fn kFns[] = {{"sin", 1},  {"cos", 1},   {"tan", 1},  {"asin", 1},  {"acos", 1},  {"atan", 1},
                       {"sinh", 1}, {"cosh", 1},  {"tanh", 1}, {"exp", 1},   {"log", 1},   {"log10", 1},
                       {"sqrt", 1}, {"fabs", 1},  {"floor", 1}, {"ceil", 1}, {"atan2", 2}, {"pow", 2},
                       {"fmin", 2}, {"fmax", 2}};

class Parser {
  public:
    Parser(const char *text, int n, int m, int p, int64_t n_params, bool pdf = false)
        : s_(text), n_(n), m_(m), p_(p), np_(n_params), pdf_(pdf) {}

    // Whole expression; false with a message on error.
    bool run(std::string &code, uint32_t &dep_x, uint32_t &dep_u, std::string &err) {
        std::string out;
        const bool ok = expr(0, out) && (skip(), s_[i_] == '\0' ? true : fail("trailing characters"));
        if (!ok) {
            err = msg_;
            return false;
        }
        code = out;
        dep_x = dx_;
        dep_u = du_;
        return true;
    }

  private:
    const char *s_;
    size_t i_ = 0;
    int n_, m_, p_;
    int64_t np_;
    bool pdf_;  // a density: the one variable is t
    int depth_ = 0;
    uint32_t dx_ = 0, du_ = 0;
    std::string msg_;

    bool fail(const char *what) {
        if (msg_.empty()) {
            char buf[160];
            snprintf(buf, sizeof buf, "%s at offset %zu", what, i_);
            msg_ = buf;
        }
        return false;
    }
    void skip() {
        while (s_[i_] == ' ' || s_[i_] == '\t' || s_[i_] == '\n' || s_[i_] == '\r') ++i_;
    }
    static int prec(char c) { return (c == '+' || c == '-') ? 1 : (c == '*' || c == '/') ? 2 : 0; }

    // precedence climbing over the binary operators
    bool expr(int min_prec, std::string &out) {
        if (++depth_ > 200) return fail("expression nested too deeply");
        std::string lhs;
        if (!prefix(lhs)) return false;
        for (;;) {
            skip();
            const char op = s_[i_];
            const int pr = prec(op);
            if (pr == 0 || pr < min_prec) break;
            ++i_;
            std::string rhs;
            if (!expr(pr + 1, rhs)) return false;
            lhs = "(" + lhs + " " + op + " " + rhs + ")";
        }
        --depth_;
        out = lhs;
        return true;
    }

    // unary signs bind tighter than every binary operator
    bool prefix(std::string &out) {
        if (++depth_ > 200) return fail("expression nested too deeply");
        skip();
        const char c = s_[i_];
        bool ok;
        if (c == '-') {
            ++i_;
            std::string a;
            ok = prefix(a);
            out = "(-" + a + ")";
        } else if (c == '+') {
            ++i_;
            ok = prefix(out);
        } else {
            ok = atom(out);
        }
        --depth_;
        return ok;
    }

    bool atom(std::string &out) {
        skip();
        const char c = s_[i_];
        if (c == '(') {
            ++i_;
            std::string a;
            if (!expr(0, a)) return false;
            skip();
            if (s_[i_] != ')') return fail("expected ')'");
            ++i_;
            out = a;
            return true;
        }
        if ((c >= '0' && c <= '9') || c == '.') return number(out);
        if ((c >= 'a' && c <= 'z') || (c >= 'A' && c <= 'Z') || c == '_') return name(out);
        return fail(c ? "unexpected character" : "unexpected end of expression");
    }

    bool number(std::string &out) {
        const size_t b = i_;
        bool digits = false;
        while (s_[i_] >= '0' && s_[i_] <= '9') ++i_, digits = true;
        if (s_[i_] == '.') {
            ++i_;
            while (s_[i_] >= '0' && s_[i_] <= '9') ++i_, digits = true;
        }
        if (!digits) return fail("malformed number");
        if (s_[i_] == 'e' || s_[i_] == 'E') {
            ++i_;
            if (s_[i_] == '+' || s_[i_] == '-') ++i_;
            if (!(s_[i_] >= '0' && s_[i_] <= '9')) return fail("malformed exponent");
            while (s_[i_] >= '0' && s_[i_] <= '9') ++i_;
        }
        const char t = s_[i_];
        if ((t >= 'a' && t <= 'z') || (t >= 'A' && t <= 'Z') || t == '_') return fail("malformed number");
        const std::string lit(s_ + b, i_ - b);
        const double v = std::strtod(lit.c_str(), nullptr);
        if (!std::isfinite(v)) return fail("number out of range");
        char buf[64];
        snprintf(buf, sizeof buf, "%a", v);  // exact, and always a double literal
        out = buf;
        return true;
    }

    bool name(std::string &out) {
        const size_t b = i_;
        while ((s_[i_] >= 'a' && s_[i_] <= 'z') || (s_[i_] >= 'A' && s_[i_] <= 'Z') ||
               (s_[i_] >= '0' && s_[i_] <= '9') || s_[i_] == '_')
            ++i_;
        const std::string id(s_ + b, i_ - b);
        skip();
        if (s_[i_] == '(') {
            const Fn *fn = nullptr;
            for (const Fn &f : kFns)
                if (id == f.name) fn = &f;
            if (!fn) return fail("unknown function");
            ++i_;
            std::string a, bb;
            if (!expr(0, a)) return false;
            skip();
            if (fn->arity == 2) {
                if (s_[i_] != ',') return fail("expected ',' (two-argument function)");
                ++i_;
                if (!expr(0, bb)) return false;
                skip();
            }
            if (s_[i_] != ')') return fail("expected ')' after the arguments");
            ++i_;
            out = std::string(fn->name) + "(" + a + (fn->arity == 2 ? ", " + bb : std::string()) + ")";
            return true;
        }
        if (pdf_) {
            if (id != "t") return fail("unknown identifier (a density reads t only)");
            out = "t";
            return true;
        }
        // variable: a letter, then a decimal index without leading zeros
        const char k = id.empty() ? '\0' : id[0];
        const std::string num = id.size() > 1 ? id.substr(1) : std::string();
        bool ok = (k == 'x' || k == 'u' || k == 'w' || k == 'p') && !num.empty() && num.size() <= 6 &&
                  !(num.size() > 1 && num[0] == '0');
        for (char ch : num) ok = ok && ch >= '0' && ch <= '9';
        if (!ok) return fail("unknown identifier");
        const long idx = std::strtol(num.c_str(), nullptr, 10);
        const long lim = k == 'x' ? n_ : k == 'u' ? m_ : k == 'w' ? p_ : (long)np_;
        if (idx >= lim) return fail("variable index out of range");
        char buf[32];
        if (k == 'x') {
            dx_ |= 1u << idx;
            snprintf(buf, sizeof buf, "x[%ld]", idx);
        } else if (k == 'u') {
            du_ |= 1u << idx;
            snprintf(buf, sizeof buf, "u[%ld]", idx);
        } else if (k == 'w') {
            du_ |= 1u << (m_ + idx);  // the disturbance dims follow the input dims
            snprintf(buf, sizeof buf, "u[%ld]", (long)m_ + idx);
        } else {
            snprintf(buf, sizeof buf, "P[%ld]", idx);
        }
        out = buf;
        return true;
    }
};

// The kernel's view of the grid; the same declaration is emitted into the
// run-time source, so host and device agree on the layout.
#define AMY_EXPR_GRID_FIELDS                                  \
    double xlb[8], xeta[8], ulb[8], ueta[8];                  \
    int N[8], uc[8];                                          \
    int tsx[8][8], tsu[8][8];                                 \
    long long moff[8];                                        \
    int tent[8];                                              \
    int n, m;
#define AMY_STR2(...) #__VA_ARGS__
#define AMY_STR(...) AMY_STR2(__VA_ARGS__)

struct ExprGrid {
    AMY_EXPR_GRID_FIELDS
};

const char *kKernelHead =
    "struct ExprGrid { " AMY_STR(AMY_EXPR_GRID_FIELDS) " };\n"
    "extern \"C\" __global__ void amy_expr_means(const ExprGrid g, const double *__restrict__ P,\n"
    "                                            double *__restrict__ mt) {\n"
    "    const int d = blockIdx.y;\n"
    "    const long long cnt = g.tent[d];\n"
    "    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < cnt;\n"
    "         e += (long long)gridDim.x * blockDim.x) {\n"
    "        double x[8], u[8];\n"
    "        for (int j = 0; j < 8; ++j) {\n"
    "            x[j] = 0.0;\n"
    "            u[j] = 0.0;\n"
    "            if (j < g.n && g.tsx[d][j] != 0)\n"
    "                x[j] = g.xlb[j] + (double)(int)((e / g.tsx[d][j]) % g.N[j]) * g.xeta[j];\n"
    "            if (j < g.m && g.tsu[d][j] != 0)\n"
    "                u[j] = g.ulb[j] + (double)(int)((e / g.tsu[d][j]) % g.uc[j]) * g.ueta[j];\n"
    "        }\n"
    "        double r = 0.0;\n"
    "        switch (d) {\n";

// ---------------------------------------------------------------------------
// NVRTC, loaded on first use
// ---------------------------------------------------------------------------
struct Nvrtc {
    bool ok = false;
    std::string why;
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
};

Nvrtc load_nvrtc() {
    Nvrtc r;
    void *h = nullptr;
    std::vector<std::string> names = {"libnvrtc.so.13", "libnvrtc.so"};
    if (const char *home = std::getenv("CUDA_HOME")) names.push_back(std::string(home) + "/lib64/libnvrtc.so.13");
    names.push_back("/usr/local/cuda/lib64/libnvrtc.so.13");
    for (const std::string &nm : names)
        if ((h = dlopen(nm.c_str(), RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
    if (!h) {
        r.why = "NVRTC (libnvrtc.so.13) not found";
        return r;
    }
    r.create = reinterpret_cast<decltype(r.create)>(dlsym(h, "nvrtcCreateProgram"));
    r.compile = reinterpret_cast<decltype(r.compile)>(dlsym(h, "nvrtcCompileProgram"));
    r.log_size = reinterpret_cast<decltype(r.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
    r.log = reinterpret_cast<decltype(r.log)>(dlsym(h, "nvrtcGetProgramLog"));
    r.cubin_size = reinterpret_cast<decltype(r.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
    r.cubin = reinterpret_cast<decltype(r.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
    r.destroy = reinterpret_cast<decltype(r.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
    r.ok = r.create && r.compile && r.log_size && r.log && r.cubin_size && r.cubin && r.destroy;
    if (!r.ok) r.why = "NVRTC lacks an entry point";
    return r;
}

const Nvrtc &nvrtc() {
    static const Nvrtc n = load_nvrtc();
    return n;
}

// Compiled mean-table kernels per (device architecture, source).
std::mutex g_kernels_mu;
std::map<std::string, cudaKernel_t> g_kernels;

amy_status compile_kernel(const std::string &src, const char *name, cudaKernel_t &out) {
    int dev = 0, major = 0, minor = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (e != cudaSuccess) return cuda_error(e, "device query");
    char arch[48];
    snprintf(arch, sizeof arch, "--gpu-architecture=sm_%d%d", major, minor);
    const std::string key = std::string(arch) + "\n" + name + "\n" + src;
    std::lock_guard<std::mutex> lk(g_kernels_mu);
    auto it = g_kernels.find(key);
    if (it != g_kernels.end()) {
        out = it->second;
        return AMY_OK;
    }
    const Nvrtc &nv = nvrtc();
    if (!nv.ok) return set_error(AMY_E_UNSUPPORTED, "text systems need NVRTC: %s", nv.why.c_str());
    nvrtcProgram prog = nullptr;
    if (nv.create(&prog, src.c_str(), "amy_expr.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
        return set_error(AMY_E_CUDA, "NVRTC: program creation failed");
    const char *opts[] = {arch, "--fmad=false", "--std=c++17"};
    const nvrtcResult rc = nv.compile(prog, 3, opts);
    if (rc != NVRTC_SUCCESS) {
        size_t n = 0;
        nv.log_size(prog, &n);
        std::string log(n, '\0');
        if (n) nv.log(prog, &log[0]);
        nv.destroy(&prog);
        if (log.size() > 300) log.resize(300);
        return set_error(AMY_E_CUDA, "NVRTC compile of the mean expressions failed: %s", log.c_str());
    }
    size_t n = 0;
    nv.cubin_size(prog, &n);
    std::vector<char> bin(n);
    if (n) nv.cubin(prog, bin.data());
    nv.destroy(&prog);
    cudaLibrary_t lib = nullptr;
    e = cudaLibraryLoadData(&lib, bin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) return cuda_error(e, "mean expressions: library load");
    cudaKernel_t k = nullptr;
    e = cudaLibraryGetKernel(&k, lib, name);
    if (e != cudaSuccess) return cuda_error(e, "mean expressions: kernel lookup");
    g_kernels.emplace(key, k);  // kept (and its library loaded) for the life of the process
    out = k;
    return AMY_OK;
}

// The user densities' table kernel: per dim (one thread each) the density at
// the knots and its 8-point Gauss-Legendre integral over each knot interval
// (nodes and weights: the Legendre polynomial P8's roots and their weights),
// summed in order into the CDF, then both normalised by the total.
const char *kUserHead =
    "struct UserBox { double lo[8], hi[8]; int n; };\n"
    "__device__ double amy_pdf(int d, double t) {\n"
    "    switch (d) {\n";
const char *kUserTail =
    "    }\n"
    "    return 0.0;\n"
    "}\n"
    "extern \"C\" __global__ void amy_user_tables(const UserBox b, double *__restrict__ out) {\n"
    "    const int d = blockIdx.x * blockDim.x + threadIdx.x;\n"
    "    if (d >= b.n) return;\n"
    "    const int M = 1024;\n"
    "    const double X[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};\n"
    "    const double Wt[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};\n"
    "    const double lo = b.lo[d], hi = b.hi[d], h = (hi - lo) / (double)M;\n"
    "    double *F = out + (long long)d * 2 * (M + 1), *f = F + (M + 1);\n"
    "    F[0] = 0.0;\n"
    "    for (int i = 0; i < M; ++i) {\n"
    "        const double a = lo + (double)i * h, e = i + 1 == M ? hi : lo + (double)(i + 1) * h;\n"
    "        const double c = 0.5 * (a + e), r = 0.5 * (e - a);\n"
    "        double sum = 0.0;\n"
    "        for (int q = 3; q >= 0; --q) sum = sum + Wt[q] * amy_pdf(d, c - r * X[q]);\n"
    "        for (int q = 0; q < 4; ++q) sum = sum + Wt[q] * amy_pdf(d, c + r * X[q]);\n"
    "        F[i + 1] = F[i] + r * sum;\n"
    "    }\n"
    "    const double Z = F[M];\n"
    "    for (int i = 0; i <= M; ++i) {\n"
    "        const double t = i == M ? hi : lo + (double)i * h;\n"
    "        F[i] = F[i] / Z;\n"
    "        f[i] = amy_pdf(d, t) / Z;\n"
    "    }\n"
    "}\n";

amy_status compile_kernel(const std::string &src, const char *name, cudaKernel_t &out);

}  // namespace

amy_status expr_compile(const char *const *text, int n, int m_ctrl, int p_dist, int64_t n_params, ExprProgram &out) {
    if (!text) return set_error(AMY_E_INVALID_ARG, "text system: null expression list");
    std::string src = kKernelHead;
    for (int d = 0; d < MAXD; ++d) out.dep_x[d] = out.dep_u[d] = 0;
    for (int d = 0; d < n; ++d) {
        if (!text[d]) return set_error(AMY_E_INVALID_ARG, "text system: null expression for component %d", d);
        if (std::strlen(text[d]) > 65536) return set_error(AMY_E_INVALID_ARG, "text system: component %d too long", d);
        Parser ps(text[d], n, m_ctrl, p_dist, n_params);
        std::string code, err;
        if (!ps.run(code, out.dep_x[d], out.dep_u[d], err))
            return set_error(AMY_E_INVALID_ARG, "text system, component %d: %s", d, err.c_str());
        char head[48];
        snprintf(head, sizeof head, "        case %d: r = ", d);
        src += head + code + "; break;\n";
    }
    src += "        }\n        mt[g.moff[d] + e] = r;\n    }\n}\n";
    out.source = src;
    return AMY_OK;
}

amy_status expr_fill_means(const ExprProgram &prog, const Geom &g, double *d_mtab, cudaStream_t st) {
    cudaKernel_t k = nullptr;
    amy_status s = compile_kernel(prog.source, "amy_expr_means", k);
    if (s != AMY_OK) return s;
    ExprGrid eg;
    memset(&eg, 0, sizeof eg);
    int64_t most = 1;
    for (int d = 0; d < MAXD; ++d) {
        eg.xlb[d] = g.lb[d];
        eg.xeta[d] = g.eta[d];
        eg.ulb[d] = g.ulb[d];
        eg.ueta[d] = g.ueta[d];
        eg.N[d] = g.N[d];
        eg.uc[d] = g.ucount[d];
        for (int j = 0; j < MAXD; ++j) {
            eg.tsx[d][j] = g.tsx[d][j];
            eg.tsu[d][j] = g.tsu[d][j];
        }
        eg.moff[d] = g.moff[d];
        eg.tent[d] = d < g.n ? g.tent[d] : 0;
        most = std::max<int64_t>(most, eg.tent[d]);
    }
    eg.n = g.n;
    eg.m = g.m;
    const double *P = g.params;
    double *mt = d_mtab;
    void *args[] = {&eg, &P, &mt};
    const dim3 grid((unsigned)std::min<int64_t>((most + 255) / 256, 4096), (unsigned)g.n);
    const cudaError_t e = cudaLaunchKernel((const void *)k, grid, dim3(256), args, 0, st);
    if (e != cudaSuccess) return cuda_error(e, "mean expressions launch");
    return AMY_OK;
}

}  // namespace amy

namespace amy {

amy_status user_tables(const char *const *pdf, const Geom &g, double *d_tab, cudaStream_t st) {
    if (!pdf) return set_error(AMY_E_INVALID_ARG, "user noise: null density list");
    std::string src = kUserHead;
    for (int d = 0; d < g.n; ++d) {
        if (!pdf[d]) return set_error(AMY_E_INVALID_ARG, "user noise: null density for dim %d", d);
        if (std::strlen(pdf[d]) > 65536) return set_error(AMY_E_INVALID_ARG, "user noise: density %d too long", d);
        Parser ps(pdf[d], g.n, 0, 0, 0, true);
        std::string code, err;
        uint32_t dx = 0, du = 0;
        if (!ps.run(code, dx, du, err))
            return set_error(AMY_E_INVALID_ARG, "user noise, density %d: %s", d, err.c_str());
        char head[48];
        snprintf(head, sizeof head, "        case %d: return ", d);
        src += head + code + ";\n";
    }
    src += kUserTail;
    cudaKernel_t k = nullptr;
    amy_status s = compile_kernel(src, "amy_user_tables", k);
    if (s != AMY_OK) return s;
    struct UserBox {
        double lo[8], hi[8];
        int n;
    } b;
    memset(&b, 0, sizeof b);
    for (int d = 0; d < g.n; ++d) {
        b.lo[d] = g.np[0][d];
        b.hi[d] = g.np[1][d];
    }
    b.n = g.n;
    void *args[] = {&b, &d_tab};
    cudaError_t e = cudaLaunchKernel((const void *)k, dim3(1), dim3(32), args, 0, st);
    if (e != cudaSuccess) return cuda_error(e, "user densities launch");
    // the tables must describe densities: finite, non-negative, a positive total
    const size_t per = (size_t)2 * (USER_KNOTS + 1);
    std::vector<double> host((size_t)g.n * per);
    e = cudaMemcpyAsync(host.data(), d_tab, host.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "user densities");
    for (int d = 0; d < g.n; ++d) {
        const double *F = host.data() + d * per, *f = F + (USER_KNOTS + 1);
        bool ok = F[USER_KNOTS] == 1.0;
        for (int i = 0; i <= USER_KNOTS && ok; ++i) ok = std::isfinite(F[i]) && std::isfinite(f[i]) && f[i] >= 0.0;
        if (!ok) return set_error(AMY_E_INVALID_ARG, "user noise: density %d is not a density on its box", d);
    }
    return AMY_OK;
}

}  // namespace amy
