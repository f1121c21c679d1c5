/*
 * amy.h -- C ABI of the GB300 engine for the data-parallel hot path of the
 * AMYTISS method (arxiv 2005.06191): finite-MDP transition probabilities on a
 * uniform grid fused with the finite-horizon Bellman backup for safety,
 * reachability and reach-avoid specifications.
 *
 * Conventions (every entry point):
 *   - returns amy_status; no C++ exception crosses this boundary;
 *   - outputs are written only when AMY_OK is returned;
 *   - all input arrays are copied during the call; the caller keeps ownership;
 *   - host pointers unless a flag says "device"; device pointers must be
 *     valid on the current CUDA device and ordered on the handle's stream;
 *   - amy_last_error() returns a thread-local message for the last failure.
 *
 * Index conventions: states and inputs are linearised in C order (last
 * dimension fastest).  A policy entry is the linear input index; 0xFFFF marks
 * a state whose value is fixed by the specification (target, avoid, unsafe).
 */
#ifndef AMY_H
#define AMY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AMY_OK = 0,
    AMY_E_INVALID_ARG = 1,
    AMY_E_OUT_OF_MEMORY = 2,
    AMY_E_CUDA = 3,
    AMY_E_NOT_READY = 4,
    AMY_E_TIMEOUT = 5,
    AMY_E_QUEUE_FULL = 6,
    AMY_E_CANCELLED = 7,
    AMY_E_UNSUPPORTED = 8,
    AMY_E_NOT_FOUND = 9
} amy_status;

#define AMY_MAX_DIMS 8
#define AMY_MAX_BOXES 16
#define AMY_POLICY_NONE 0xFFFF

typedef struct amy_handle_s *amy_handle;
typedef struct amy_server_s *amy_server;

/* Uniform grid (Sec. 4, quantiser Pi_x with Eq. 7): centre j of dim d is
 * lb[d] + j*eta[d] for 0 <= j < count[d]; cell j is [centre - eta/2,
 * centre + eta/2).  periodic[d] != 0 makes dim d wrap modulo count[d]
 * (periodic may be NULL).  n in 1..8. */
typedef struct amy_grid_s {
    int32_t n;
    const double *lb;
    const double *eta;
    const int32_t *count;
    const uint8_t *periodic;
} amy_grid;

/* System f of Eq. 4, evaluated at representative points.
 * AMY_SYS_AFFINE_PER_INPUT: for each discrete input u (C order over the input
 *   grid) params holds A_u (n*n, row-major) then c_u (n); the mean is
 *   mu_i = (sum_j A_u[i][j] * x_j, summed j = 0..n-1 from 0.0) + c_u[i],
 *   every product and sum rounded separately in FP64 (no fused multiply-add).
 *   n_params must be n_u * (n*n + n).
 * AMY_SYS_UNICYCLE: n = 3, m = 2, params = {tau}; with state (x, y, th) and
 *   input (v, w): mu = (x + (tau*v)*cos(th), y + (tau*v)*sin(th), th + tau*w).
 * disturb: the disturbance grid W^ of the dt-SCS with bounded disturbances
 *   (Sec. 3; the representative points of Sec. 4), or NULL for none (the
 *   system of Eq. 4).  With a grid of n_w points (C order, p = disturb->n
 *   dims, m + p <= 8) the synthesis is the max-min game of the Remark in
 *   Sec. 3: every input's value is the min over the n_w disturbance points
 *   of its window sums (Algorithm 4's inner min), and the policy is the
 *   lowest input maximising that value.  Only the affine kind takes a grid:
 *   params then holds one (A, c) record per (input, disturbance) pair,
 *   disturbance fastest (record u * n_w + w), n_params = n_u * n_w * (n*n + n);
 *   disturb->periodic is ignored.
 * AMY_SYS_EXPR: the system as text, as the tool's configuration files give
 *   the right-hand side of the difference equation (Sec. 3): expr[d] (n
 *   NUL-terminated strings) is mean component d, a C-syntax arithmetic
 *   expression over the FP64 variables x0..x{n-1} (the state's centre),
 *   u0..u{m-1} (the input's point), w0..w{p-1} (the disturbance's point, with
 *   a disturbance grid) and p0..p{n_params-1} (params, which may be NULL when
 *   n_params = 0): numeric literals (always doubles), unary + and -, binary +
 *   - * / (left associative, * and / binding tighter), parentheses, and the
 *   calls sin cos tan asin acos atan sinh cosh tanh exp log log10 sqrt fabs
 *   floor ceil, atan2 pow fmin fmax.  Every operation is one FP64 operation
 *   rounded as written (no fused multiply-add); the calls are CUDA's.  The
 *   expressions are compiled at amy_build with NVRTC (UNSUPPORTED when
 *   libnvrtc cannot be loaded) into a kernel that tabulates each component
 *   over the coordinates it reads (8 bytes per record: the product of the
 *   grid sizes of the variables it names); the kernels read the means from
 *   those tables, and amy_rebuild with new params refills them.  A syntax
 *   error or an unknown name is INVALID_ARG.  Only amy_build takes this kind
 *   (the server and amy_synthesize_noalloc answer UNSUPPORTED). */
typedef enum { AMY_SYS_AFFINE_PER_INPUT = 0, AMY_SYS_UNICYCLE = 1, AMY_SYS_EXPR = 2 } amy_sys_kind;

/* Noise distribution per dimension (Sec. 6.2: uniform, exponential and beta
 * besides the normal, and multiplicative noise as in Eq. (1a)); NULL in
 * amy_system = Gaussian with amy_build's sigma.  Parameters, [n] arrays:
 *   AMY_NOISE_GAUSSIAN       none (sigma is amy_build's argument)
 *   AMY_NOISE_UNIFORM        p0 = a: noise ~ U[-a, a]
 *   AMY_NOISE_EXPONENTIAL    p0 = rate: noise ~ Exp(rate), density
 *                            rate * exp(-rate t) for t >= 0
 *   AMY_NOISE_BETA           p0 = alpha, p1 = beta (integers >= 1, sum <= 64),
 *                            p2 = lo < p3 = hi: noise = lo + (hi - lo) B,
 *                            B ~ Beta(alpha, beta)
 *   AMY_NOISE_MULT_GAUSSIAN  p0 = s: multiplicative noise, std s * |x_d| at a
 *                            state whose centre in dim d is x_d (no noise where
 *                            x_d = 0); dense or explicit windows only (the paper
 *                            disables the cut for multiplicative noise)
 *   AMY_NOISE_USER           the user's density (Sec. 6.2: a density and a box
 *                            enclosing its support): pdf[d] is a C-syntax
 *                            expression in the variable t (the noise value; the
 *                            grammar of AMY_SYS_EXPR), p0 = lo < p1 = hi the box.
 *                            At amy_build it is compiled with NVRTC and tabulated
 *                            over [lo, hi]: at 1025 knots its value, per knot
 *                            interval its 8-point Gauss-Legendre integral summed
 *                            into the CDF, both normalised by the total (the
 *                            density need not integrate to one); a cell's mass
 *                            is the difference of the CDF's cubic Hermite
 *                            interpolant at its edges.  INVALID_ARG when the text
 *                            is bad or a value is negative or not finite.
 * Cells are still kept by their centres inside the cut interval around the
 * mean (gamma mode): the support for the uniform, beta and user densities
 * (gamma must not exceed the uniform's density 1/(2a)),
 * [0, log(rate/gamma)/rate] for the exponential (gamma < rate).  Only
 * amy_build takes user densities (the server and amy_synthesize_noalloc
 * answer UNSUPPORTED).  amy_info's cut_half_width then reports the
 * upper end of that interval. */
typedef enum { AMY_NOISE_GAUSSIAN = 0, AMY_NOISE_UNIFORM = 1, AMY_NOISE_EXPONENTIAL = 2, AMY_NOISE_BETA = 3,
               AMY_NOISE_MULT_GAUSSIAN = 4, AMY_NOISE_USER = 5 } amy_noise_kind;
typedef struct {
    int32_t kind;
    const double *p0, *p1, *p2, *p3;
    const char *const *pdf;  /* AMY_NOISE_USER: n densities in t, else ignored */
} amy_noise;

typedef struct {
    int32_t kind;
    int32_t n;
    int32_t m;
    const double *params;
    int64_t n_params;
    const struct amy_grid_s *disturb;  /* NULL: no disturbance */
    const amy_noise *noise;            /* NULL: Gaussian (amy_build's sigma) */
    const char *const *expr;           /* AMY_SYS_EXPR: n expressions, else ignored */
} amy_system;

/* Cutting region (Sec. 5.2 and its Remark on constructing the region).
 * window == NULL, gamma > 0: per dim the 1-D density equals gamma at +-xs,
 *   xs = sigma*sqrt(2*log(1/(gamma*sigma*sqrt(2*pi)))), width W = floor(2*xs/eta)+1,
 *   origin o = ceil(((mu - xs) - lb)/eta); slot o+k (k < W) is kept iff its
 *   centre lb + (o+k)*eta <= mu + xs and it lies on the grid (or the dim is
 *   periodic).  gamma at or above the peak density -> AMY_E_INVALID_ARG.
 * window == NULL, gamma == 0: dense rows, W = count, o = 0 (non-periodic only).
 * window != NULL: explicit odd widths; o = floor((mu - lb)/eta + 0.5) - (W-1)/2.
 * All origin arithmetic is FP64 in exactly this order, so the kept set is
 * reproducible bit for bit. */
typedef struct {
    double gamma;
    const int32_t *window;
} amy_cut;

/* T storage (Sec. 5.3 stored rows; Sec. 6.1 on-the-fly abstraction).
 * AMY_T_STORED_SEPARABLE tabulates, per state dim d, the window origin and the
 * W[d] masses of mean component d over only the state and input coordinates
 * that component depends on (affine: non-zero columns of A_u[d][:] and input
 * coordinates that change row d; unicycle: x on (x, th, v), y on (y, th, v),
 * th on (th, w)).  The values are bit-identical to the per-pair masses of
 * AMY_T_STORED_FACTORED; FP32 precisions only. */
typedef enum {
    AMY_T_ON_THE_FLY = 0,       /* no T in memory; rows recomputed every backup */
    AMY_T_STORED_FULL = 1,      /* T[slot][pair] products, built once */
    AMY_T_STORED_FACTORED = 2,  /* per-dim masses F[sum W][pair], built once */
    AMY_T_STORED_SEPARABLE = 3, /* per-dim tables over each component's dependencies */
    AMY_T_AUTO = 4              /* separable tables when they take at most 8 MiB (and a
                                   quarter of the budget), else stored factored when it
                                   takes at most 1 GiB (and a quarter of the budget), else
                                   on the fly; amy_info reports the choice */
} amy_tmode;

/* Arithmetic: FP64 everywhere, or FP32 cell masses/products with FP64 only for
 * the mean and the window origin; FP32_KAHAN adds compensated accumulation of
 * the window sum.  V_out is double for FP64, float otherwise. */
typedef enum { AMY_PREC_FP64 = 0, AMY_PREC_FP32 = 1, AMY_PREC_FP32_KAHAN = 2 } amy_prec;

/* Storage of V_k between backups (FP32 precisions only).  AMY_V_BF16 halves
 * the bytes of every V gather: each value is a bfloat16 folded about 1/2
 * (V < 1/2 stored as bf16(V), V >= 1/2 as -bf16(1 - V); the sign bit marks
 * the fold), so its rounding error is at most 2^-9 * min(V, 1 - V) <= 2^-10
 * per backup and zero at 0 and 1.  The errors of successive backups add up
 * along the horizon.  AMY_V_UNORM16 stores round(V * 65535) in 16 bits (V
 * lies in [0, 1]): same bytes, error at most 2^-17 per backup.  V_out is
 * FP32 in both cases (the last backup writes it unrounded). */
typedef enum { AMY_V_NATIVE = 0, AMY_V_BF16 = 1, AMY_V_UNORM16 = 2 } amy_vstore;

typedef struct {
    int32_t tmode;              /* amy_tmode */
    int32_t prec;               /* amy_prec */
    int32_t v_store;            /* amy_vstore */
    int64_t device_mem_budget;  /* bytes the handle may allocate; 0 = unlimited */
    void *cuda_stream;          /* cudaStream_t for all work (cudaStreamLegacy and
                                   cudaStreamPerThread accepted); NULL = a
                                   non-blocking stream owned by the handle */
    int32_t use_graphs;         /* 1: amy_synthesize with device outputs captures its
                                   horizon loop into a CUDA graph and replays it while
                                   spec, horizon and output pointers repeat */
    int32_t autotune;           /* 1: amy_build times the backup kernel's launch
                                   shapes (input lanes per state, row-aligned or
                                   linear state tiles) on the handle's own buffers
                                   and keeps the fastest; results do not depend on
                                   the choice.  Skipped (heuristic shapes) when one
                                   backup exceeds 4e9 window slots.  0: heuristic. */
    int32_t launch_shape[5];    /* fixed backup launch shape, each entry 0 = automatic:
                                   [0] input lanes per state (1..8), [1] states per
                                   block of the staged variant (multiple of 32,
                                   [0]*[1] <= 512), [2] 1 = row tiles, 2 = tiles of
                                   consecutive states, [3] staged box budget in floats
                                   (256..6144), [4] values of dim 0 per row tile of a
                                   3-D problem in the per-run kernels (1..8; the
                                   tile's rows of dim 1 = its rows / this).  Entries
                                   that do not apply are ignored; the autotuner, when
                                   on, overrides them. */
} amy_opts;

/* Closed box tested on representative points: lb[d] <= centre_d <= ub[d]. */
typedef struct {
    const double *lb;
    const double *ub;
} amy_box;

/* Specifications of Algorithm 3 / Algorithm 4.
 * SAFETY: V_N = 1 on `safe`, V_k = 1_safe * max_u sum (safe == NULL: whole grid).
 * REACH / REACH_AVOID: V = 1 on the target boxes, 0 on the avoid boxes, and
 * V_k = max_u sum elsewhere.  A grid state in both a target and an avoid box
 * -> AMY_E_INVALID_ARG.  At most AMY_MAX_BOXES boxes of each kind. */
typedef enum { AMY_SAFETY = 0, AMY_REACH = 1, AMY_REACH_AVOID = 2 } amy_spec_kind;
typedef struct {
    int32_t kind;
    const amy_box *safe;
    const amy_box *target;
    int32_t n_target;
    const amy_box *avoid;
    int32_t n_avoid;
} amy_spec;

typedef struct {
    int64_t n_states;
    int64_t n_inputs;
    int32_t n;
    int32_t window[AMY_MAX_DIMS];
    int64_t window_slots;       /* prod W */
    int32_t window_sum;         /* sum W */
    double cut_half_width[AMY_MAX_DIMS];  /* xs per dim (INFINITY outside gamma mode) */
    int64_t device_bytes;       /* bytes owned by the handle */
    int32_t tmode;
    int32_t prec;
    int32_t v_store;
    int32_t input_lanes;        /* backup launch shape: threads per state (1..8; 0 = generic kernel) */
    int32_t row_tiles;          /* 1: staged backup tiles are whole innermost-dim rows */
    int32_t block_states;       /* states (lane columns) per block of the backup */
    int32_t grouped_inputs;     /* 1: runs of inputs sharing every outer dim's masses
                                   are served by one outer contraction per run */
    int32_t backup_kernel;      /* 0 generic (k_backup), 1 register-resident
                                   (k_backup_fast), 2 shared-memory staged, 3 staged
                                   with one outer contraction per input run, 4 the
                                   per-run kernel on row tiles (k_backup_runs), 5 its
                                   persistent form: the whole horizon in one
                                   cooperative launch (k_synth_runs), 6 wide rows
                                   (stored full, stored factored or on the fly)
                                   split over window-row groups (k_backup_rows or
                                   k_backup_rows_otf, then k_argmax_rows), 7 the
                                   plane kernel of banded problems with tables
                                   (k_backup_plane, see amy_set_plane), 8 its tiled
                                   form (k_backup_tile), 9 2-D tables with windows
                                   wider than 8 (k_sums_sep2, then k_collect_keys) */
    int32_t input_runs;         /* runs of consecutive inputs sharing outer records */
    int32_t inner_span;         /* inner slots K one outer contraction covers (kernels 3, 4) */
    int32_t build_kernels;      /* kernels one table build (amy_build / amy_rebuild) launches */
    int32_t tile_outer_rows;    /* per-run kernels: values of dim 0 per row tile (3-D) */
    int32_t step_wait;          /* persistent kernel (5): what a block waits for between
                                   backups, 0 neighbour tiles, 1 every block
                                   (amy_set_step_wait; picked by the autotuner) */
    int32_t backup_launch_kernels; /* kernels one backup launch of amy_kernel_times
                                   runs (2 for kernel 6, else 1) */
    int32_t n_disturbances;     /* disturbance points n_w (1 without a grid); n_inputs
                                   counts the control inputs */
} amy_info_t;

/* Points per dim of [lb, ub] with step eta: floor((ub-lb)/eta + 1e-9) + 1
 * (the grids of Sec. 7-8 give the pair counts printed in Table 4). */
int64_t amy_grid_count(double lb, double ub, double eta);

/* Build the abstraction (Algorithm 2 for the stored modes): validates the
 * problem, derives the window shape, copies the system to the device and, in
 * the stored modes, launches the T construction kernel once.  sigma[n] is the
 * per-dim noise standard deviation (diagonal covariance).  The handle is
 * independent of the specification, so it serves any number of
 * amy_synthesize calls.  Errors: INVALID_ARG (bad grid, system, cut, n_u >
 * 65535, more than 2^31-1 states), OUT_OF_MEMORY (budget or cudaMalloc),
 * UNSUPPORTED (window too large for the kernels), CUDA. */
amy_status amy_build(const amy_system *sys, const amy_grid *states, const amy_grid *inputs,
                     const double *sigma, const amy_cut *cut, const amy_opts *opts,
                     amy_handle *out);

/* Finite-horizon synthesis (Algorithm 4; on-the-fly rows per Sec. 6.1 in
 * AMY_T_ON_THE_FLY).  `horizon` backups from V_N; V_out[n_states] receives
 * V_0 (double for AMY_PREC_FP64, float otherwise).  policy_out receives
 * pi_0 [n_states] or, with policy_all_steps, pi_k for k = 0..horizon-1 as
 * [horizon][n_states]; it may be NULL.  outputs_on_device != 0: V_out and
 * policy_out are device pointers and the call returns once the work is
 * enqueued on the handle's stream; otherwise they are host pointers and the
 * call returns after the copy.  Host buffers in page-locked memory the
 * device can address (cudaHostAlloc, cudaHostRegister) are written by the
 * kernels in place, so their copy-out overlaps the backups; after an error
 * reported once the kernels ran (AMY_E_TIMEOUT, AMY_E_CUDA) their contents
 * are unspecified.  Other host buffers are filled from a device staging
 * buffer the handle keeps between calls, only on AMY_OK. */
amy_status amy_synthesize(amy_handle h, const amy_spec *spec, int32_t horizon, void *V_out,
                          uint16_t *policy_out, int32_t policy_all_steps,
                          int32_t outputs_on_device);

/* One Bellman backup (one iteration of the time loop of Algorithm 4) from a
 * caller-given V_next[n_states] (double for FP64, float otherwise) to
 * V_out[n_states] and policy_out[n_states] (may be NULL).  on_device selects
 * device or host pointers for all three, as in amy_synthesize. */
amy_status amy_backup_step(amy_handle h, const amy_spec *spec, const void *V_next, void *V_out,
                           uint16_t *policy_out, int32_t on_device);

/* Transition rows as the engine uses them (Algorithm 2): for each of `count`
 * host-given pairs (x[i], u[i]) the window origin origin_out[i*n + d] and the
 * prod-W probabilities probs_out[i*prod W + slot] in C order over the window
 * box (0 for dropped slots), as double.  Host pointers. */
amy_status amy_query_rows(amy_handle h, const int64_t *x, const int64_t *u, int64_t count,
                          int32_t *origin_out, double *probs_out);

/* Closed-loop Monte-Carlo validation of a synthesized controller (Sec. 7:
 * the closed loop is simulated from initial states and the success
 * frequency set against V_0).  Runs the finite MDP itself: from each initial
 * state x0[i], runs_per_x0 runs of `horizon` steps, step t applying
 * policy[t * n_states + x] (pi_t as amy_synthesize writes it with
 * policy_all_steps; may be NULL when horizon == 0).  A run succeeds when it
 * meets `spec`: reach / reach-avoid -- it enters a target box before any
 * avoid box and within the horizon; safety -- it stays in the safe box for
 * all `horizon` steps.  Each step draws, per state dim d, the next grid cell
 * by inverse CDF over that dim's FP64 cell masses in window order (Algorithm
 * 1's row, for every noise kind); a draw beyond their sum (the mass the cut
 * or the grid's edge removes) fails the run.  With a disturbance grid the
 * disturbance point is drawn uniformly, before the dims.  Draw q of step t of
 * run r of x0[i] is word q % 4 of Philox4x64-10 (Salmon et al., SC'11) at
 * counter (i * runs_per_x0 + r, t, q / 4, 0) under key (seed, 0), as
 * (w >> 11) * 2^-53; q = 0..n-1 are the dims, q = n the disturbance.  The
 * counts are thus fixed by (seed, runs_per_x0) whatever the launch.
 * successes_out[i] receives the number of successful runs of x0[i].
 * on_device != 0: policy, x0 and successes_out are device pointers;
 * otherwise host pointers.  Synchronous in both cases (the call reads back
 * its error word).  Errors: INVALID_ARG (null pointers, negative counts, more
 * than 2^62 runs, an initial state out of range, a policy entry >= n_inputs
 * at a state a run visits before it ends, a bad spec), CUDA. */
amy_status amy_simulate(amy_handle h, const amy_spec *spec, int32_t horizon, const uint16_t *policy,
                        const int64_t *x0, int64_t n_x0, int64_t runs_per_x0, uint64_t seed,
                        int64_t *successes_out, int32_t on_device);

/* Export of the abstraction as an MDP in PRISM's explicit-model files (the
 * PRISM export the tool offers, Sec. 2), for model checking the synthesized
 * result with another tool.  Writes, next to path_prefix:
 *   <prefix>.tra    "S C T" then one line "s c s' p" per transition: states
 *                   0..n_states-1 are the grid (C-order index), state
 *                   n_states an absorbing sink (one choice, a self-loop);
 *                   choice c of a grid state is input c; p is the row's mass
 *                   as the handle's mode computes it (amy_query_rows), slots
 *                   landing on one cell merged, and the mass the cut or the
 *                   grid's edge removes (1 - the row's sum, when positive)
 *                   goes to the sink, so every distribution sums to one;
 *   <prefix>.lab    labels 0 "init" (every grid state), 1 "deadlock" (none),
 *                   2 "target", 3 "avoid", 4 "safe" (safety specs), 5 "sink";
 *   <prefix>.sta    grid indices (x0, ..., x{n-1}) per state, -1 for the sink;
 *   <prefix>.props  the property whose maximal probability is V_0 of
 *                   amy_synthesize with this spec and horizon: Pmax=? [ G<=N
 *                   "safe" ], [ !"avoid" U<=N "target" ] or [ F<=N "target" ].
 * n_transitions_out (may be NULL) receives T.  The files grow with
 * n_states * n_inputs * prod W lines: meant for small abstractions.
 * Synchronous.  Errors: INVALID_ARG (null pointer, negative horizon, bad
 * spec, a file that cannot be written), UNSUPPORTED (a disturbance grid: the
 * model is then a stochastic game), CUDA. */
amy_status amy_export_prism(amy_handle h, const amy_spec *spec, int32_t horizon, const char *path_prefix,
                            int64_t *n_transitions_out);

/* Rebuild the stored rows in place (Algorithm 2 again) after replacing the
 * system parameters (params may be NULL to keep them): same grid, cut and
 * storage, no allocation.  Asynchronous on the handle's stream.  For
 * AMY_T_STORED_SEPARABLE the new parameters must keep the dependency sets
 * (else INVALID_ARG).  A no-op for AMY_T_ON_THE_FLY apart from the upload. */
amy_status amy_rebuild(amy_handle h, const double *params, int64_t n_params);

/* Kernel timing: while on, every backup and build kernel of this handle is
 * bracketed by CUDA events on the handle's stream.  amy_kernel_times waits
 * for the recorded events, returns the summed durations (ms), the launch
 * counts and the number of backups those launches performed (one per launch,
 * or the whole horizon for the persistent kernel) since the previous call,
 * and resets them (a backup launch of backup kernel 6 runs two kernels:
 * amy_info backup_launch_kernels).  Any argument may be NULL.  It also
 * reports AMY_E_TIMEOUT when a persistent synthesis since the previous check
 * gave up waiting between backups (its outputs are then invalid). */
amy_status amy_set_profiling(amy_handle h, int32_t on);

/* Polls a wait between backups of the persistent horizon kernel
 * (k_synth_runs, amy_info backup_kernel 5) makes before it gives up (default
 * 2^20, about a tenth of a second; a wait normally completes within
 * microseconds); 0 makes every wait give up at once.  A wait that gives up
 * makes every block leave the kernel; the synthesis then returns
 * AMY_E_TIMEOUT (host outputs) or the next call that waits on the handle's
 * stream reports it, and its outputs are invalid.  The handle stays usable.
 * polls < 0 restores the default.  The paper has no counterpart: this bounds
 * the device-wide wait the persistent kernel adds. */
amy_status amy_set_wait_limit(amy_handle h, int32_t polls);

/* What a block of the persistent horizon kernel waits for between backups
 * (Algorithm 4's backup k reads all of V_{k+1}, but one block's window box
 * reads only the V cells of nearby tiles): mode 0 = only the tiles its box
 * reads and the tiles whose boxes read it, through per-tile backup counters;
 * mode 1 = every block (a grid-wide barrier).  The default is mode 1, or the
 * faster of the two when amy_build autotunes; this call overrides it.
 * Values and policies are the same in both modes.  Other modes return
 * AMY_E_INVALID_ARG.  The paper has no counterpart (it launches one backup
 * after another). */
amy_status amy_set_step_wait(amy_handle h, int32_t mode);

/* Backup kernel of problems with per-dimension tables whose mean components
 * each depend on a few coordinates (banded coupling, as in the room and road
 * rings of Sec. 8.2 / 8.3; four or more state dims, no periodic dim, planes
 * of at most 512 states).  Algorithm 4's window sum is reassociated per
 * plane of the two innermost dims: the dims whose masses the whole plane
 * shares are contracted first, once per plane, into a partial box held in
 * shared memory, from which each state sums its remaining dims (amy_info
 * backup_kernel 7).  The same terms are summed, in another FP32 order, so
 * values agree with the per-state kernels to rounding.
 * on = 1 (the default) uses it wherever it applies, on = 0 the per-state
 * register-resident kernel.  smem_bytes caps one block's shared memory
 * (16 KiB .. 200 KiB; 0 = 100 KiB, two blocks per SM); the partial box is
 * staged in chunks when it does not fit, which does not change the result.
 * The plane kernel has a tiled form (backup_kernel 8): a block serves up to
 * 4 groups of planes that differ only in the first staged dim a, and the
 * dims whose windows none of them moves (no mean component of theirs reads
 * x_a) are contracted once for the tile; the one remaining shared dim is
 * applied per group afterwards.  Another FP32 order of the same terms again;
 * it needs every other staged dim's component free of x_a and at most one
 * shared dim reading x_a.  on = 1 takes it for planes of at least 256
 * states, on = 2 wherever it applies, on = 3 never (in each case the plane
 * kernel runs where the tiled form does not).  smem_bytes also caps the
 * tiled form's block (0: two blocks per SM where they fit).
 * Errors: INVALID_ARG (null handle, bad mode or size). */
amy_status amy_set_plane(amy_handle h, int32_t on, int32_t smem_bytes);

/* Work the plane kernel performs in one backup (roofline numerators), for
 * the handle's problem and this spec: one backup from V_N with counters on,
 * on the handle's own buffers and stream (synchronised; not for a timed
 * region).  v_loads: values of V_{k+1} read from global memory in the first
 * stage (each S combination of each staged row); box_loads: values read from
 * the shared-memory partial box in the second stage; box_rows: second-stage
 * rows summed (one FP32 FMA per box load plus W[n-2] + 1 per row).  The
 * paper has no counterpart.  Errors: INVALID_ARG, UNSUPPORTED (the handle
 * does not run backup kernel 7), CUDA. */
amy_status amy_backup_work(amy_handle h, const amy_spec *spec, int64_t *v_loads, int64_t *box_loads,
                           int64_t *box_rows);

/* Measured read bandwidth of the L2 cache: 16-byte loads that bypass L1
 * (ld.global.cg) streaming a 32 MiB buffer that stays in L2, every SM busy,
 * in bytes per second on the current device (roofline denominator of
 * kernels that stream L2-resident data).  Allocates 32 MiB temporarily.
 * Errors: INVALID_ARG (null pointer), CUDA. */
amy_status amy_measure_l2(double *bytes_per_s);

/* The kernel times amy_set_profiling collects (see there): summed backup and
 * build durations in ms, their launch counts and the backups performed.
 * Waits for the recorded events.  Errors: INVALID_ARG (null handle),
 * TIMEOUT (a persistent synthesis gave up), CUDA. */
amy_status amy_kernel_times(amy_handle h, double *backup_ms, int64_t *backup_launches, int64_t *backup_steps,
                            double *build_ms, int64_t *build_launches);

/* The handle's derived abstraction (Sec. 5.2: window widths and cut half
 * widths per dim, window slots), its storage and precision, the device bytes
 * it owns, and the backup kernel and launch shape its synthesis uses (fields
 * of amy_info_t).  Writes *out; errors: INVALID_ARG (null argument), CUDA. */
amy_status amy_info(amy_handle h, amy_info_t *out);

/* Releases the handle and everything it owns on the device after its stream
 * has drained.  NULL is ignored; the handle must not be used afterwards. */
void amy_destroy(amy_handle h);

/* The message of the calling thread's last failed call (empty if none).  The
 * pointer stays valid until that thread's next call into the library. */
const char *amy_last_error(void);

/* ------------------------------------------------------------------------
 * Synthesis without memory allocation.  This entry point has no counterpart
 * in the paper; it serves callers that may not allocate device memory -- for
 * example code whose device memory is owned entirely by its own pool or by
 * another framework, or a latency-critical loop where an allocation could
 * synchronise the device or fail.
 *
 * amy_synthesize_noalloc runs the same computation as amy_build with
 * AMY_T_ON_THE_FLY followed by amy_synthesize (FP32 or FP32_KAHAN, V stored in
 * FP32), writing V_0 (float) into V_out and pi_0 into policy_out (may be NULL;
 * not written when horizon is 0); both are device pointers of n_states
 * entries, ordered on cuda_stream (NULL = the legacy default stream).  It
 * calls no cudaMalloc, cudaFree or other allocating routine: the system
 * parameters, the per-state spec flags and the two value vectors live in one
 * file-scope device array of AMY_NOALLOC_SCRATCH_BYTES, which every GPU that
 * loads the library holds until the process exits.  A problem needs
 * 8*n_params + n_states + 2*4*(n_states + 64) bytes (each part rounded up to
 * 256); larger problems return AMY_E_INVALID_ARG with a message naming the
 * limit.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls share the array and it keeps the last
 * call's contents; every entry a call reads is written earlier by the same
 * call (it clears the few guard cells around its value vectors itself), but
 * calls whose work overlaps on the GPU (on different streams or threads) race
 * on it and must be serialised.  The parameters reach the array by an
 * asynchronous copy ordered on cuda_stream: from pageable host memory the
 * source has been read when the call returns, but from page-locked memory
 * (cudaHostAlloc / cudaHostRegister) the copy runs later on the stream, so
 * the caller must leave sys->params unchanged until the stream has passed
 * this call's work (e.g. synchronise it first).  Everything else is read
 * during the call, which returns once the work is enqueued.
 * ------------------------------------------------------------------------ */
#define AMY_NOALLOC_SCRATCH_BYTES (16u << 20)
amy_status amy_synthesize_noalloc(const amy_system *sys, const amy_grid *states, const amy_grid *inputs,
                                  const double *sigma, const amy_cut *cut, int32_t prec, const amy_spec *spec,
                                  int32_t horizon, float *V_out, uint16_t *policy_out, void *cuda_stream);

/* ---- Measurement helper (not part of the paper's method) ----------------
 * Measured ceilings of the two load paths the fused backup kernels gather
 * V_{k+1} through, for roofline denominators: 32-bit shared-memory loads
 * (conflict free) and 32-bit global loads that hit L1 (coalesced), both in
 * lane-loads per second (one 4-byte value delivered to one thread), on the
 * current device.  Takes a few milliseconds; allocates 16 MiB temporarily.
 * Errors: INVALID_ARG (null pointer), CUDA. */
amy_status amy_measure_lane_loads(double *shared_per_s, double *global_per_s);

/* Measured fused multiply-add rates of the current device, FP32 and FP64, in
 * FMAs per second summed over all threads (independent chains, every SM
 * full): the ceiling of a backup bound by its FMAs (the FP64 paths; GB300
 * issues FP64 far slower than FP32).  Takes a few milliseconds.  Errors:
 * INVALID_ARG (null pointer), CUDA. */
amy_status amy_measure_fma(double *fp32_per_s, double *fp64_per_s);

/* Measured complementary error function rates of the current device, erfcf
 * (FP32) and erfc (FP64), in evaluations per second summed over all threads
 * (independent arguments spread over [0, 4.1], the tail-side arguments of the
 * cell masses of Algorithm 1; neighbouring lanes at different arguments, every
 * SM full): the ceiling of a backup that forms its masses on the fly, each
 * (state, input) pair taking sum_i (W_i + 1) edge values.  Takes a few
 * milliseconds.  Errors: INVALID_ARG (null pointer), CUDA. */
amy_status amy_measure_erfc(double *fp32_per_s, double *fp64_per_s);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of independent synthesis requests.
 * A scheduler thread admits queued requests while slots and device memory
 * allow, keeps each admitted problem's V ping-pong buffers resident, and
 * every tick advances every admitted problem by one backup -- in one
 * persistent kernel launch over a table of problems (batched = 1) or one
 * launch per problem (batched = 0).  Results are copied out as problems
 * finish; their slots and memory are then reused by queued requests.
 * ------------------------------------------------------------------------ */
typedef struct {
    int64_t device_mem_budget;  /* bytes for resident problems; 0 = 4 GiB */
    int32_t max_slots;          /* problems resident at once; 0 = 64 */
    int32_t max_queue;          /* queued + running requests; 0 = 4096 */
    int32_t batched;            /* 1: one persistent kernel per tick; 0: per problem */
    int32_t use_graphs;         /* 1: ticks whose layout recurs replay a captured CUDA
                                   graph (amy_server_graph_stats) */
    int32_t device;             /* CUDA device ordinal */
} amy_server_opts;

typedef struct {
    amy_system sys;
    amy_grid states;
    amy_grid inputs;
    const double *sigma;
    amy_cut cut;
    int32_t prec;               /* AMY_PREC_FP32 or AMY_PREC_FP32_KAHAN */
    int32_t v_store;            /* amy_vstore */
    amy_spec spec;
    int32_t horizon;
} amy_request;

typedef struct {
    amy_status status;          /* AMY_OK or the failure of this request */
    int64_t n_states;
    float *V;                   /* V_0 [n_states], library-owned */
    uint16_t *policy;           /* pi_0 [n_states], library-owned */
    double submit_us;           /* times on the server's monotonic clock */
    double admit_us;
    double finish_us;
} amy_result;

amy_status amy_server_create(const amy_server_opts *opts, amy_server *out);
/* Queue a request (copied).  QUEUE_FULL when max_queue is reached; the
 * request is validated at once (INVALID_ARG / UNSUPPORTED). */
amy_status amy_submit(amy_server s, const amy_request *req, uint64_t *ticket);
/* AMY_E_NOT_READY until the result exists; then fills *out once (the ticket
 * is retired).  NOT_FOUND for unknown or retired tickets. */
amy_status amy_poll(amy_server s, uint64_t ticket, amy_result *out);
/* As amy_poll but blocks up to timeout_us (< 0: forever); TIMEOUT if not done. */
amy_status amy_wait(amy_server s, uint64_t ticket, int64_t timeout_us, amy_result *out);
/* Cancel a queued or running request; its result reports AMY_E_CANCELLED. */
amy_status amy_cancel(amy_server s, uint64_t ticket);
/* Counters: completed requests, ticks, kernel launches (a replayed tick graph
 * counts one), current resident problems. */
amy_status amy_server_stats(amy_server s, int64_t *completed, int64_t *ticks, int64_t *launches,
                            int32_t *resident);
/* With use_graphs: tick graphs captured and tick graphs replayed so far.  A
 * tick's launches depend on its layout -- which problems take part, in which
 * order, reading which of their two V vectors -- and a layout seen a second
 * time is captured into a CUDA graph (batch tables in device memory the
 * graph owns) and replayed while it recurs; a stable set of residents
 * alternates between two layouts.  Graphs of a problem are dropped when it
 * leaves (at most 32 are kept, least recently used first).  In this mode
 * every tick writes each problem's V_k and pi_k to its output buffers (the
 * last tick's are the ones returned), so results equal those without graphs
 * bit for bit.  The paper has no counterpart. */
amy_status amy_server_graph_stats(amy_server s, int64_t *captures, int64_t *replays);
void amy_server_destroy(amy_server s);
void amy_result_free(amy_result *r);

#ifdef __cplusplus
}
#endif
#endif
