// amy_calibrate.cu -- measured ceilings used as roofline denominators: the
// FP32 and FP64 fused multiply-add issue rates, the FP32 and FP64 erfc
// evaluation rates, the L2 read bandwidth, and the two load paths the
// fused backup kernels gather V through:
//   - shared memory: 32-bit loads, every warp reading 32 consecutive words
//     (one wavefront per instruction, no bank conflict);
//   - global memory hitting L1: 32-bit loads, every warp reading 32
//     consecutive words of a 16 KiB block-private slice that stays in L1.
// Each thread keeps four independent sums so that loads, not the adds, set
// the pace; the sums are written out so that nothing is optimised away.
// The rates count lane-loads (one 4-byte value delivered to one thread).
#include <cuda_runtime.h>

#include "../../include/amy.h"
#include "amy_internal.h"

namespace amy {
namespace {

constexpr int CAL_THREADS = 512;
constexpr int CAL_WORDS = 4096;  // per block: 16 KiB
constexpr int CAL_ITERS = 256;   // passes over the block's words

__global__ void __launch_bounds__(CAL_THREADS) k_cal_shared(const float *__restrict__ src, float *__restrict__ out) {
    __shared__ float buf[CAL_WORDS];
    for (int i = threadIdx.x; i < CAL_WORDS; i += blockDim.x) buf[i] = src[i];
    __syncthreads();
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int it = 0; it < CAL_ITERS; ++it) {
        const int b = ((warp + it) * 128) & (CAL_WORDS - 1);  // 4 rows of 32 words per step
        s0 += buf[b + lane];
        s1 += buf[b + 32 + lane];
        s2 += buf[b + 64 + lane];
        s3 += buf[b + 96 + lane];
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = (s0 + s1) + (s2 + s3);
}

__global__ void __launch_bounds__(CAL_THREADS) k_cal_global(const float *__restrict__ src, float *__restrict__ out) {
    const float *base = src + (size_t)(blockIdx.x % 1024) * CAL_WORDS;  // block-private, L1-resident slice
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int it = 0; it < CAL_ITERS; ++it) {
        const int b = ((warp + it) * 128) & (CAL_WORDS - 1);
        s0 += __ldg(base + b + lane);
        s1 += __ldg(base + b + 32 + lane);
        s2 += __ldg(base + b + 64 + lane);
        s3 += __ldg(base + b + 96 + lane);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = (s0 + s1) + (s2 + s3);
}

// Fused multiply-add issue: every thread runs FMA_CHAINS independent chains
// a = a * b + c (b, c runtime values, so nothing folds), FMA_ITERS steps
// each; the chains keep the pipe busy rather than waiting on one result.
constexpr int FMA_THREADS = 256;
constexpr int FMA_CHAINS = 8;

template <class R>
__global__ void __launch_bounds__(FMA_THREADS) k_cal_fma(R b, R c, int iters, R *__restrict__ out) {
    R acc[FMA_CHAINS];
#pragma unroll
    for (int i = 0; i < FMA_CHAINS; ++i) acc[i] = (R)(threadIdx.x + i);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < FMA_CHAINS; ++i) acc[i] = fma(acc[i], b, c);
    }
    R s = 0;
#pragma unroll
    for (int i = 0; i < FMA_CHAINS; ++i) s += acc[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Complementary error function throughput: every thread evaluates erfc at
// ERFC_CHAINS independent arguments per step, spread over [0, 4.1] (the
// tail-side arguments (edge - mu) / (sigma sqrt 2) the cell masses take),
// neighbouring lanes at different arguments as in the mass kernels; the
// arguments depend on runtime values only, and the sums are written out.
constexpr int ERFC_THREADS = 256;
constexpr int ERFC_CHAINS = 4;

template <class R>
__global__ void __launch_bounds__(ERFC_THREADS) k_cal_erfc(R dx, int iters, R *__restrict__ out) {
    R x[ERFC_CHAINS], s[ERFC_CHAINS];
#pragma unroll
    for (int i = 0; i < ERFC_CHAINS; ++i) {
        x[i] = (R)((threadIdx.x & 31) + 32 * i) * (R)(4.0 / 128.0);
        s[i] = (R)0;
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < ERFC_CHAINS; ++i) {
            s[i] += erfc(x[i]);
            x[i] += dx;
        }
    }
    R t = 0;
#pragma unroll
    for (int i = 0; i < ERFC_CHAINS; ++i) t += s[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = t;
}

// L2 read bandwidth: 16-byte loads at L2 (not cached in L1) over a buffer
// that fits in L2, every thread striding through it; four loads in flight per
// thread per step.
constexpr int L2_THREADS = 512;
__global__ void __launch_bounds__(L2_THREADS) k_cal_l2(const float4 *__restrict__ src, int64_t n4, int passes,
                                                      float *__restrict__ out) {
    float s = 0.0f;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    for (int ps = 0; ps < passes; ++ps) {
        const int64_t start = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x + (int64_t)ps * 4096) % step;
        for (int64_t i = start; i + 3 * step < n4; i += 4 * step) {
            float4 v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                asm volatile("ld.global.cg.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                             : "=f"(v[q].x), "=f"(v[q].y), "=f"(v[q].z), "=f"(v[q].w)
                             : "l"(src + i + q * step));
#pragma unroll
            for (int q = 0; q < 4; ++q) s += (v[q].x + v[q].y) + (v[q].z + v[q].w);
        }
    }
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace amy

using namespace amy;

extern "C" amy_status amy_measure_l2(double *bytes_per_s) {
    if (!bytes_per_s) return set_error(AMY_E_INVALID_ARG, "null argument");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_error(e, "device query");
    const int blocks = sms * 4;  // 2048 threads per SM
    const int64_t n4 = (int64_t)(32 << 20) / 16;
    const int passes = 64;
    float4 *src = nullptr;
    float *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&src, (size_t)n4 * 16, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&out, (size_t)blocks * L2_THREADS * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(src, 0, (size_t)n4 * 16, st);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    float best = 3.4e38f;
    for (int rep = 0; rep < 5 && e == cudaSuccess; ++rep) {  // first pass warms L2 up
        e = cudaEventRecord(a, st);
        if (e == cudaSuccess) k_cal_l2<<<blocks, L2_THREADS, 0, st>>>(src, n4, passes, out);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventRecord(b, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
    }
    // bytes actually read: each pass reads the whole groups of 4 * step vectors
    const int64_t step = (int64_t)blocks * L2_THREADS;
    const int64_t per_pass = (n4 / (4 * step)) * 4 * step * 16;
    if (src) cudaFreeAsync(src, st);
    if (out) cudaFreeAsync(out, st);
    if (st) cudaStreamSynchronize(st);
    if (st) cudaStreamDestroy(st);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_error(e, "L2 calibration");
    *bytes_per_s = (double)per_pass * passes / (best * 1e-3);
    return AMY_OK;
}

extern "C" amy_status amy_measure_fma(double *fp32_per_s, double *fp64_per_s) {
    if (!fp32_per_s || !fp64_per_s) return set_error(AMY_E_INVALID_ARG, "null argument");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_error(e, "device query");
    const int blocks = sms * 8;  // 2048 threads per SM
    double *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&out, (size_t)blocks * FMA_THREADS * sizeof(double), st);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    double rate[2] = {0.0, 0.0};
    for (int which = 0; which < 2 && e == cudaSuccess; ++which) {
        const int iters = which == 0 ? 4096 : 256;  // FP64 issues far slower on this part
        float best = 3.4e38f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // first pass warms up
            e = cudaEventRecord(a, st);
            if (which == 0)
                k_cal_fma<float><<<blocks, FMA_THREADS, 0, st>>>(0.999f, 1e-3f, iters, reinterpret_cast<float *>(out));
            else
                k_cal_fma<double><<<blocks, FMA_THREADS, 0, st>>>(0.999, 1e-3, iters, out);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(b, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(b);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
            if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
        }
        const double fmas = (double)blocks * FMA_THREADS * FMA_CHAINS * iters;
        rate[which] = fmas / (best * 1e-3);
    }
    if (out) cudaFreeAsync(out, st);
    if (st) cudaStreamSynchronize(st);
    if (st) cudaStreamDestroy(st);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_error(e, "FMA calibration");
    *fp32_per_s = rate[0];
    *fp64_per_s = rate[1];
    return AMY_OK;
}

extern "C" amy_status amy_measure_lane_loads(double *shared_per_s, double *global_per_s) {
    if (!shared_per_s || !global_per_s) return set_error(AMY_E_INVALID_ARG, "null argument");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_error(e, "device query");
    const int blocks = sms * 4 * 8;  // several waves of full blocks
    float *src = nullptr, *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    const size_t src_words = (size_t)1024 * CAL_WORDS;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&src, src_words * 4, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&out, (size_t)blocks * CAL_THREADS * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(src, 0, src_words * 4, st);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    double rate[2] = {0.0, 0.0};
    for (int which = 0; which < 2 && e == cudaSuccess; ++which) {
        float best = 3.4e38f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // first pass warms up
            e = cudaEventRecord(a, st);
            if (which == 0)
                k_cal_shared<<<blocks, CAL_THREADS, 0, st>>>(src, out);
            else
                k_cal_global<<<blocks, CAL_THREADS, 0, st>>>(src, out);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(b, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(b);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
            if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
        }
        const double loads = (double)blocks * CAL_THREADS * CAL_ITERS * 4.0;
        rate[which] = loads / (best * 1e-3);
    }
    if (src) cudaFreeAsync(src, st);
    if (out) cudaFreeAsync(out, st);
    if (st) cudaStreamSynchronize(st);
    if (st) cudaStreamDestroy(st);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_error(e, "lane-load calibration");
    *shared_per_s = rate[0];
    *global_per_s = rate[1];
    return AMY_OK;
}

extern "C" amy_status amy_measure_erfc(double *fp32_per_s, double *fp64_per_s) {
    if (!fp32_per_s || !fp64_per_s) return set_error(AMY_E_INVALID_ARG, "null argument");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_error(e, "device query");
    const int blocks = sms * 8;  // 2048 threads per SM
    double *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&out, (size_t)blocks * ERFC_THREADS * sizeof(double), st);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    double rate[2] = {0.0, 0.0};
    for (int which = 0; which < 2 && e == cudaSuccess; ++which) {
        const int iters = which == 0 ? 256 : 32;  // x stays below 4 + iters * dx
        float best = 3.4e38f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // first pass warms up
            e = cudaEventRecord(a, st);
            if (which == 0)
                k_cal_erfc<float><<<blocks, ERFC_THREADS, 0, st>>>(1e-4f, iters, reinterpret_cast<float *>(out));
            else
                k_cal_erfc<double><<<blocks, ERFC_THREADS, 0, st>>>(1e-4, iters, out);
            if (e == cudaSuccess) e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaEventRecord(b, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(b);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
            if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
        }
        const double evals = (double)blocks * ERFC_THREADS * ERFC_CHAINS * iters;
        rate[which] = evals / (best * 1e-3);
    }
    if (out) cudaFreeAsync(out, st);
    if (st) cudaStreamSynchronize(st);
    if (st) cudaStreamDestroy(st);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_error(e, "erfc calibration");
    *fp32_per_s = rate[0];
    *fp64_per_s = rate[1];
    return AMY_OK;
}
