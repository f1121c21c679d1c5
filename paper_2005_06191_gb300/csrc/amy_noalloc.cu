// amy_noalloc.cu -- amy_synthesize_noalloc: finite-horizon synthesis with
// rows on the fly for callers that may not allocate memory.
//
// Who needs it: code that must not call cudaMalloc, cudaMallocAsync or any
// other allocator -- for example a caller whose device memory is entirely
// owned by its own pool or by another framework, or a latency-critical loop
// where an allocation could synchronise the device or fail.  Such a caller
// passes its problem and its own device output buffers; every piece of
// intermediate device memory the synthesis needs (the system parameters, the
// per-state spec flags and the two value vectors the backups ping-pong
// between) lives in one file-scope device array, `g_noalloc_scratch`, of
// AMY_NOALLOC_SCRATCH_BYTES.  Every GPU that loads the library holds that
// array until the process exits.
//
// The array is shared by all calls on a device and keeps the last call's
// contents.  Every entry a call reads is written earlier by that same call:
// the spec-mask kernel writes every flag and V_N, each backup writes every
// V_k, and the few guard cells around each value vector (read with zero
// mass by the contiguous-row kernels, so they must hold finite values) are
// cleared at the start of every call.  Calls whose work overlaps on the GPU
// (e.g. on two streams at once) race on the array; serialise them.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/amy.h"
#include "amy_internal.h"

namespace amy {

// Scratch for amy_synthesize_noalloc (see the file comment).
static __device__ __align__(256) unsigned char g_noalloc_scratch[AMY_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void *g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device: looked up once
// per device, with that device current, on the first call there.
amy_status scratch_address(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return set_error(AMY_E_UNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "scratch symbol address");
        g_scratch_addr[dev] = p;
    }
    *out = (unsigned char *)g_scratch_addr[dev];
    return AMY_OK;
}

size_t up256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace
}  // namespace amy

using namespace amy;

extern "C" amy_status amy_synthesize_noalloc(const amy_system *sys, const amy_grid *states, const amy_grid *inputs,
                                             const double *sigma, const amy_cut *cut, int32_t prec,
                                             const amy_spec *spec, int32_t horizon, float *V_out,
                                             uint16_t *policy_out, void *cuda_stream) {
    if (!V_out) return set_error(AMY_E_INVALID_ARG, "null V_out");
    if (horizon < 0) return set_error(AMY_E_INVALID_ARG, "negative horizon");
    if (prec != AMY_PREC_FP32 && prec != AMY_PREC_FP32_KAHAN)
        return set_error(AMY_E_UNSUPPORTED, "amy_synthesize_noalloc runs in FP32 or FP32_KAHAN");
    Geom g;
    amy_status st = fill_geom(sys, states, inputs, sigma, cut, g);
    if (st != AMY_OK) return st;
    if (g.sys == SYS_EXPR)
        return set_error(AMY_E_UNSUPPORTED, "text systems are built with amy_build (their mean tables need a handle)");
    if (g.noise == NOISE_USER)
        return set_error(AMY_E_UNSUPPORTED, "user noise densities are built with amy_build (their tables need a handle)");
    SpecDev sd;
    st = make_spec(g, spec, sd);
    if (st != AMY_OK) return st;
    // scratch layout: parameters | spec flags | V ping-pong (FP32)
    const size_t nx = (size_t)g.nx;
    const size_t pbytes = up256((size_t)sys->n_params * sizeof(double));
    const size_t mbytes = up256(nx);
    const size_t vbytes = up256((nx + 2 * kVGuard) * sizeof(float));
    const size_t need = pbytes + mbytes + 2 * vbytes;
    if (need > (size_t)AMY_NOALLOC_SCRATCH_BYTES)
        return set_error(AMY_E_INVALID_ARG,
                         "problem needs %zu bytes of scratch (parameters, flags, two value vectors); "
                         "amy_synthesize_noalloc holds at most %zu -- use amy_build/amy_synthesize",
                         need, (size_t)AMY_NOALLOC_SCRATCH_BYTES);
    int dev = 0, sm_count = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_error(e, "device query");
    unsigned char *base = nullptr;
    st = scratch_address(dev, &base);
    if (st != AMY_OK) return st;
    double *d_params = (double *)base;
    uint8_t *d_mask = base + pbytes;
    // each value vector carries kVGuard finite guard cells on both sides
    float *d_V[2] = {(float *)(base + pbytes + mbytes) + kVGuard, (float *)(base + pbytes + mbytes + vbytes) + kVGuard};
    cudaStream_t s = (cudaStream_t)cuda_stream;
    g.params = d_params;
    e = cudaMemcpyAsync(d_params, sys->params, (size_t)sys->n_params * sizeof(double), cudaMemcpyHostToDevice, s);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        // guard cells must hold finite values: cleared on every call
        e = cudaMemsetAsync(d_V[i] - kVGuard, 0, kVGuard * sizeof(float), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_V[i] + nx, 0, kVGuard * sizeof(float), s);
    }
    if (e != cudaSuccess) return cuda_error(e, "parameter upload");
    st = launch_spec_mask(g, sd, d_mask, d_V[0], AMY_V_NATIVE, s);
    if (st != AMY_OK) return st;
    const bool fast = fast_wm(g, prec) > 0;
    int cur = 0;
    for (int32_t k = horizon - 1; k >= 0; --k) {
        FastCall c;
        c.Vn = d_V[cur];
        c.Vo = d_V[cur ^ 1];
        c.Vfinal = (k == 0) ? V_out : nullptr;
        c.pi = (k == 0) ? policy_out : nullptr;
        c.mask = d_mask;
        c.spec_kind = sd.kind;
        c.kahan = prec == AMY_PREC_FP32_KAHAN;
        c.T = nullptr;
        c.O = nullptr;
        c.npairs = 0;
        c.tab = nullptr;
        c.ulanes = 0;
        st = fast ? launch_backup_fast(g, TM_OTF, AMY_V_NATIVE, c, sm_count, s)
                  : launch_backup_generic_fp32(g, TM_OTF, c, AMY_V_NATIVE, sm_count, s);
        if (st != AMY_OK) return st;
        cur ^= 1;
    }
    if (horizon == 0) {
        e = cudaMemcpyAsync(V_out, d_V[0], nx * sizeof(float), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_error(e, "V_N copy");
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? AMY_OK : cuda_error(e, "synthesize (no allocation)");
}
