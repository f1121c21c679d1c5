// amy_simulate.cu -- closed-loop Monte-Carlo simulation of the finite MDP
// under a synthesized policy (the validation of Sec. 7: the controller is run
// from initial states and the success frequency compared with V_0).
//
// One thread per run.  Each step draws, per state dim d, the next cell by
// inverse CDF over that dim's FP64 window masses (the row of Algorithm 1, in
// window order); a draw beyond their sum -- the mass the cut or the grid's
// edge removes -- ends the run as a failure, which is what V treats as 0.
// With a disturbance grid the disturbance point is drawn uniformly first.
// Draws come from Philox4x64-10 (Salmon, Moraes, Dror and Shaw, "Parallel
// random numbers: as easy as 1, 2, 3", SC'11): draw q of step t of global
// run g is word q % 4 of the block at counter (g, t, q / 4, 0) under key
// (seed, 0), taken as (w >> 11) * 2^-53; q = 0..n-1 picks the dims and q = n
// the disturbance.  Runs are independent streams, so the counts do not depend
// on the launch shape.
#include <cstring>

#include "amy_internal.h"

namespace amy {

namespace {

// Philox4x64 round constants: the multipliers and the Weyl key increments
// (golden ratio and sqrt(3) - 1 in 64-bit fixed point).
constexpr uint64_t kPhiloxM0 = 0xD2E7470EE14C6C93ull;
constexpr uint64_t kPhiloxM1 = 0xCA5A826395121157ull;
constexpr uint64_t kPhiloxW0 = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kPhiloxW1 = 0xBB67AE8584CAA73Bull;

__device__ __forceinline__ void philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0,
                                              uint64_t k1, uint64_t out[4]) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t lo0 = kPhiloxM0 * c0, hi0 = __umul64hi(kPhiloxM0, c0);
        const uint64_t lo1 = kPhiloxM1 * c2, hi1 = __umul64hi(kPhiloxM1, c2);
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

// The draws of one step: blocks of four words made when first needed.
struct StepDraws {
    uint64_t run, step, seed;
    int block = -1;
    uint64_t w[4];
    __device__ double operator()(int q) {
        if (q / 4 != block) {
            block = q / 4;
            philox4x64_10(run, step, (uint64_t)block, 0ull, seed, 0ull, w);
        }
        return (double)(w[q & 3] >> 11) * 0x1.0p-53;
    }
};

struct SimArgs {
    const uint16_t *pi;  // [horizon][nx]
    int32_t horizon;
    const int64_t *x0;
    int64_t n_x0, runs, total;
    uint64_t seed;
    const uint8_t *mask;
    int32_t spec_kind;
    unsigned long long *succ;  // [n_x0]
    unsigned int *err;         // bit 0: x0 out of range; bit 1: policy input out of range
};

// Spec status of a state: 1 success, 0 failure, -1 the run goes on (safety
// succeeds only at the horizon).
__device__ __forceinline__ int sim_status(int spec_kind, uint8_t f) {
    if (spec_kind == SPEC_SAFETY) return (f & F_SAFE) ? -1 : 0;
    if (f & F_TARGET) return 1;
    if (f & F_AVOID) return 0;
    return -1;
}

__global__ void __launch_bounds__(256) k_simulate(const __grid_constant__ Geom g, const SimArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t wstride = (int64_t)gridDim.x * blockDim.x;
    const int nin = g.nu / g.nw;
    // warp-uniform loop: all 32 lanes take the same iterations, so the
    // per-initial-state counts can be combined across the warp
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < a.total; base += wstride) {
        const int64_t gi = base + lane;
        const bool live = gi < a.total;
        int64_t i = -1;
        int win = 0;
        if (live) {
            i = gi / a.runs;
            const int64_t x0 = a.x0[i];
            if (x0 < 0 || x0 >= g.nx) {
                atomicOr(a.err, 1u);
            } else {
                int32_t x = (int32_t)x0;
                int st = sim_status(a.spec_kind, a.mask[x]);
                for (int32_t t = 0; t < a.horizon && st < 0; ++t) {
                    const int u = a.pi[(int64_t)t * g.nx + x];
                    if (u >= nin) {
                        atomicOr(a.err, 2u);
                        st = 0;
                        break;
                    }
                    StepDraws draw{(uint64_t)gi, (uint64_t)t, a.seed};
                    int w = 0;
                    if (g.nw > 1) w = min((int)(draw(g.n) * (double)g.nw), g.nw - 1);
                    double mu[MAXD];
                    mean_of(g, x, u * g.nw + w, mu);
                    int32_t nxt = 0;
                    bool lost = false;
                    for (int d = 0; d < g.n && !lost; ++d) {
                        const int32_t o = origin_of(g, d, mu[d]);
                        const int kmax = kept_upper(g, d, mu[d], o);
                        const double xd = noise_centre(g, x, d);
                        const double q = draw(d);
                        double cum = 0.0;
                        int32_t pick = -1;
                        // the window's cells in order, each edge's tail evaluated
                        // once (the masses slot_run_f64 gives), until the draw
                        // falls in the cumulative mass
                        const bool gauss = g.noise == NOISE_GAUSSIAN || g.noise == NOISE_MULT_GAUSSIAN;
                        const double k2 = gauss ? gauss_k2_f64(g, d, xd) : 0.0;
                        double tlo = edge_rel_f64(g, d, mu[d], o, 0);
                        double qlo = gauss ? gauss_tail_f64(tlo, k2) : 0.0;
                        for (int k = 0; k < g.W[d]; ++k) {
                            const double thi = edge_rel_f64(g, d, mu[d], o, k + 1);
                            const double qhi = gauss ? gauss_tail_f64(thi, k2) : 0.0;
                            const double mass =
                                gauss ? gauss_cell_f64(tlo, thi, qlo, qhi, k2) : noise_mass<double>(g, d, tlo, thi);
                            bool on;
                            const int32_t cell = cell_of(g, d, o + k, on);
                            cum += (on && k < kmax) ? mass : 0.0;
                            if (q < cum) {
                                pick = cell * g.stride[d];
                                break;
                            }
                            tlo = thi;
                            qlo = qhi;
                        }
                        if (pick < 0) lost = true;
                        else nxt += pick;
                    }
                    if (lost) {
                        st = 0;
                        break;
                    }
                    x = nxt;
                    st = sim_status(a.spec_kind, a.mask[x]);
                }
                if (st < 0) st = a.spec_kind == SPEC_SAFETY ? 1 : 0;
                win = st;
            }
        }
        __syncwarp();
        const unsigned same = __match_any_sync(0xffffffffu, (unsigned long long)i);
        const unsigned wins = __ballot_sync(0xffffffffu, win != 0) & same;
        if (live && lane == __ffs(same) - 1 && wins) atomicAdd(a.succ + i, (unsigned long long)__popc(wins));
    }
}

}  // namespace

amy_status launch_simulate(const Geom &g, int spec_kind, const uint8_t *mask, const uint16_t *pi, int32_t horizon,
                           const int64_t *x0, int64_t n_x0, int64_t runs, uint64_t seed, unsigned long long *succ,
                           unsigned int *err, int sm_count, cudaStream_t st) {
    SimArgs a;
    a.pi = pi;
    a.horizon = horizon;
    a.x0 = x0;
    a.n_x0 = n_x0;
    a.runs = runs;
    a.total = n_x0 * runs;
    a.seed = seed;
    a.mask = mask;
    a.spec_kind = spec_kind;
    a.succ = succ;
    a.err = err;
    if (a.total == 0) return AMY_OK;
    const int64_t want = (a.total + 255) / 256;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)std::max(sm_count, 1) * 8));
    k_simulate<<<blocks, 256, 0, st>>>(g, a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "simulate launch");
    return AMY_OK;
}

}  // namespace amy
