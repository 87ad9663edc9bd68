/*
 * ht.h -- C ABI of the GB300 many-path polynomial homotopy tracker.
 *
 * The operations follow Verschelde & Yu, "Tracking Many Solution Paths of a
 * Polynomial Homotopy on a Graphics Processing Unit" (2015):
 *   - the homotopy gamma (1 - t) g(x) + t f(x) = 0 of Eq. (eqlinhom), Section 1;
 *   - evaluation and differentiation of all monomials at many points with the
 *     reverse mode of Table tabmoneval, Section 3;
 *   - the predictor-corrector loop over many paths, Section 2, with Newton's
 *     method solving each linear system in the least squares sense by modified
 *     Gram-Schmidt (Section 1), the status codes and the scan compaction of
 *     Table tabjobidx.
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int: HT_OK (0) on success, a negative HT_E*
 *     code on failure; ht_last_error() then holds a message for the calling
 *     thread.  No C++ exception crosses this interface.
 *   - Precision is given as the number of limbs L per real number: 1 complex
 *     double, 2 complex double double, 4 complex quad double (Section 1,
 *     Section 4.1).  A real number is the unevaluated sum of its L doubles,
 *     limb 0 the leading one.
 *   - Batches of points are stored "vertically" (Section 3, Table tabtranspose):
 *     a quantity with `count` complex entries over `n` points is the array
 *     [count][2][L][n] of doubles -- entry, real/imaginary part, limb, point --
 *     so all points' values of one limb of one entry are contiguous.
 *   - Buffers named "device" are caller-owned CUDA device memory on the current
 *     device, 8-byte aligned; the library neither frees nor keeps them.  Calls
 *     taking a `stream` enqueue work on that cudaStream_t (NULL = legacy default
 *     stream) and return before it finishes unless stated otherwise.
 *   - Invalid arguments are rejected with HT_EINVAL before any launch.
 *
 * Accuracy contract of the arithmetic: every computed value differs from the
 * exact value of the same formula by at most a small multiple of 2^(-53 L)
 * times the sum of the moduli of the terms that make it up.
 */
#ifndef HT_H
#define HT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { HT_D = 1, HT_DD = 2, HT_QD = 4 };

enum {
  HT_OK = 0,
  HT_EINVAL = -1,       /* invalid argument */
  HT_ENOMEM = -2,       /* device or host allocation failed */
  HT_ECUDA = -3,        /* a CUDA call failed (message in ht_last_error) */
  HT_ETIMEOUT = -4,     /* a bounded device-side wait expired */
  HT_EUNSUPPORTED = -5  /* valid but not supported (e.g. too many variables) */
};

/* Opaque, library-owned polynomial system ("instructions" of Table tabmemory:
 * the monomial supports (idx) and coefficients (cff), shared by all paths). */
typedef struct ht_system ht_system;

/* Message of the last failing call on this thread ("" if none). */
const char* ht_last_error(void);

/*
 * ht_create_system -- copy a polynomial system to the device (Table tabmemory).
 *   n_vars   number of variables, 1..255
 *   n_polys  number of polynomials, >= 1
 *   n_terms  host [n_polys]: monomials in each polynomial, each >= 1
 *   exps     host [M][n_vars] (M = sum of n_terms): exponents, 0..127,
 *            polynomial 0's monomials first
 *   coef     host [M][2][limbs]: complex coefficients (re limbs, im limbs)
 *   limbs    HT_D, HT_DD or HT_QD: the precision evaluations use
 *   out      receives the handle; release it with ht_destroy_system
 * Uses the current CUDA device.  Errors: HT_EINVAL for bad shapes or values,
 * HT_EUNSUPPORTED for a monomial with more than 64 variables, HT_ENOMEM,
 * HT_ECUDA.
 */
int ht_create_system(int n_vars, int n_polys, const int32_t* n_terms, const int8_t* exps,
                     const double* coef, int limbs, ht_system** out);

/* Release a system (NULL is accepted).  Waits for the device to finish. */
int ht_destroy_system(ht_system* sys);

/* Shape of a system: any output pointer may be NULL. */
int ht_system_info(const ht_system* sys, int* n_vars, int* n_polys, int* limbs, int64_t* n_monomials);

/*
 * ht_eval_diff -- evaluate every polynomial and its Jacobian at n_pts points
 * (Section 3, Table tabcpugpu: coefficient, monomial value and derivatives by
 * the reverse mode of Table tabmoneval, sums into the polynomial and the
 * Jacobian, here fused in one kernel).
 *   x    device [n_vars][2][L][n_pts]   points
 *   val  device [n_polys][2][L][n_pts]  receives f_j(x_p)
 *   jac  device [n_polys][n_vars][2][L][n_pts] receives df_j/dx_i (x_p)
 * L is the system's precision.  n_pts == 0 is a no-op.  x must not overlap val
 * or jac.  Asynchronous on `stream`.
 */
int ht_eval_diff(const ht_system* sys, int64_t n_pts, const double* x, double* val, double* jac,
                 void* stream);

/*
 * ht_eval_diff_host -- ht_eval_diff on HOST buffers of the same layouts: copies
 * x to the device, evaluates, copies val and jac back, and returns when the
 * results are in host memory.  The points go to the device in one copy (after
 * the work already queued on `stream`); the polynomials are then evaluated in
 * blocks of at least 8 (at most 8 blocks) on one internal stream into up to
 * three device slabs, and a second internal stream copies each finished
 * block's rows of val and jac -- contiguous in the point-fastest layouts --
 * back in one transfer while the next blocks are evaluated.  Uses a device
 * workspace and two streams owned by the system (grown on demand, freed with
 * the system).  Pinned host memory gives the fastest copies; pageable memory
 * works.
 */
int ht_eval_diff_host(ht_system* sys, int64_t n_pts, const double* x_host, double* val_host,
                      double* jac_host, void* stream);

/*
 * ht_eval_diff_unfused -- ht_eval_diff organised as the paper's three kernels
 * (Section 3, Tables tabcpugpu and tabmemory), kept as an ablation of the
 * fused kernel and for bandwidth measurements like Table tabbench:
 *   coeff  writes the coefficient of every monomial at every point to a
 *          workspace in device memory;
 *   mon    evaluates every monomial and its derivatives at every point by the
 *          reverse mode of Table tabmoneval and writes them to the workspace;
 *   sum    adds every polynomial's terms and every Jacobian entry's terms
 *          (in monomial order) into val and jac.
 * The workspace rows are vertical (point fastest), so every access is
 * coalesced.  The operations and their order are those of ht_eval_diff's
 * FP64 bodies (variants 0 and 1), so the results are bitwise identical to
 * theirs.  Points go in chunks whose workspace fits in 2 GiB; the workspace
 * and the sum kernel's term lists are built on first use and kept in the
 * system.  Up to 65,535 monomials and n_polys (n_vars + 1) <= 65,535.
 *   x, val, jac  device, as ht_eval_diff
 *   stats        host, or NULL; when given, each kernel is timed with CUDA
 *                events on `stream` (the call then blocks) and its
 *                algorithmic bytes (every workspace row written or read once,
 *                16 L bytes per complex entry) are summed over the chunks
 */
typedef struct ht_unfused_stats {
  double ms_coeff, ms_mon, ms_sum;          /* kernel times, summed over chunks */
  double bytes_coeff, bytes_mon, bytes_sum; /* algorithmic bytes moved by each kernel */
} ht_unfused_stats;

int ht_eval_diff_unfused(ht_system* sys, int64_t n_pts, const double* x, double* val, double* jac,
                         ht_unfused_stats* stats, void* stream);

/* ------------------------------------------------------------ tuning */

/*
 * ht_set_eval_config -- choose how ht_eval_diff runs on this system:
 *   variant  1 compact monomial bodies (one code path for every support size),
 *            0 unrolled bodies for supports of up to 8 variables,
 *            2 integer limbs: the complex products on the integer pipe in
 *              radix-2^29 limbs, sums in an exact fixed-point frame per
 *              output (systems with at most 64 variables; HT_EUNSUPPORTED
 *              otherwise),
 *            3 the three kernels of ht_eval_diff_unfused (coeff, mon, sum
 *              over a workspace): work spread over monomials and points,
 *              which suits few points; the first call allocates the
 *              workspace (grown on demand, kept in the system, so the call
 *              is not allocation-free), and results are bitwise those of
 *              variants 0 and 1 (at most 65,535 monomials and outputs;
 *              HT_EUNSUPPORTED otherwise),
 *           -1 default (1)
 *   threads  CTA size 64, 128 or 256, or 0 for the default (128); for
 *            variant 2, 128 (or 0, 64) runs one unit of 32 points and one
 *            polynomial per warp with the lane's point in local memory, and
 *            256 runs work items of 32 points and a group of polynomials per
 *            CTA (one polynomial per warp: 16-warp CTAs for systems of at
 *            least 16 polynomials, else 8) with the points in shared memory
 *            (the same bits either way)
 * Variants 0, 1 and 3 perform the same operations in the same order, so their
 * results are bitwise identical; variant 2 meets the same accuracy bound
 * (a small multiple of 2^(-53 L) times the sum of the moduli of the terms of
 * each output) with its own rounding.
 * The choice also applies inside ht_track_paths for DD and QD systems with
 * n <= 32: by default (and with variant 2) the tracker runs its Newton round
 * on the integer pipe: f and its Jacobian rows, the homotopy terms and the
 * least squares (the arithmetic of ht_mgs_solve_ex variant 2) in limb
 * strings; with variant 0 or 1 it uses the FP64 pipe throughout (variant 3
 * counts as FP64 there).  Double systems always track on the FP64 pipe.
 */
int ht_set_eval_config(ht_system* sys, int variant, int threads);

/*
 * ht_tune_eval -- autotuner for ht_eval_diff: times every (variant, threads)
 * configuration on the given device buffers (reps timed launches each, CUDA
 * events on `stream`), keeps the fastest in the system and reports it (any
 * output pointer may be NULL).  On return val and jac hold the chosen
 * configuration's results.  Blocks.
 */
int ht_tune_eval(ht_system* sys, int64_t n_pts, const double* x, double* val, double* jac, int reps, int* variant,
                 int* threads, float* best_ms, void* stream);

/* ------------------------------------------------------- learned step MLP */

/*
 * The learned step-size proposer (a workload addition on top of Section 2,
 * where the step-size rule is left open): a dense network
 * 16 -> 64 -> 64 -> 2 with ReLU after both hidden layers.  Inputs are the
 * per-path step features (ht_track_paths_ex documents them); outputs are
 * (rho, alpha): the log of the proposed step multiplier and a scale for the
 * predictor's displacement.  Products run on the tensor cores with BF16
 * operands and FP32 accumulation; parameters are FP32 masters.
 * Parameter vector (HT_MLP_NPARAM floats): W1[64][16] b1[64] W2[64][64] b2[64]
 * W3[2][64] b3[2], weights row-major [out][in].
 */
#define HT_MLP_IN 16
#define HT_MLP_OUT 2
#define HT_MLP_NPARAM 5378
typedef struct ht_mlp ht_mlp;

/* Create a network with all parameters zero (set them with ht_mlp_set_params). */
int ht_mlp_create(ht_mlp** out);
int ht_mlp_destroy(ht_mlp* net);
/* Copy parameters from / to host [HT_MLP_NPARAM] floats.  Setting them also
 * resets the optimiser state. */
int ht_mlp_set_params(ht_mlp* net, const float* params);
int ht_mlp_get_params(const ht_mlp* net, float* params);
/* y = network(x) for B samples: x device [B][16], y device [B][2].  Async. */
int ht_mlp_forward(const ht_mlp* net, int64_t B, const float* x, float* y, void* stream);
/* Mean squared error (1/B) sum_b sum_o (y_bo - target_bo)^2 over B samples and
 * its gradient with respect to the parameters: x device [B][16], target device
 * [B][2], grad device [HT_MLP_NPARAM] or NULL, loss device [1] or NULL.  Async. */
int ht_mlp_loss_grad(ht_mlp* net, int64_t B, const float* x, const float* target, float* grad, float* loss,
                     void* stream);
/* The gradient's products also run on the tensor cores (BF16 operands: the
 * loss derivative, the activation gradients and the activations; FP32
 * accumulation).  Per chunk of 64 samples the partial gradients are summed in
 * a fixed order, so the result depends only on B, x, target and the
 * parameters. */
/* Train on n samples (x, target as above, device) for `epochs` passes over
 * consecutive minibatches of `batch` samples (shuffle the data beforehand),
 * one Adam step (as ht_mlp_adam_step) per minibatch at rate lr.
 * epoch_loss: host [epochs] mean minibatch loss per epoch, or NULL.  Blocks. */
int ht_mlp_train(ht_mlp* net, int64_t n, const float* x, const float* target, int epochs, int64_t batch, float lr,
                 float* epoch_loss, void* stream);
/* One Adam step (Kingma & Ba 2015: beta1 0.9, beta2 0.999, eps 1e-8, bias
 * correction by the network's step count, which ht_mlp_set_params resets) on
 * the FP32 masters with the gradient grad (device [HT_MLP_NPARAM] floats),
 * then the BF16 copy.  Async. */
int ht_mlp_adam_step(ht_mlp* net, const float* grad, float lr, void* stream);
/* Adam's state: first and second moments (host [HT_MLP_NPARAM] floats each,
 * either may be NULL) and the step count (may be NULL).  Blocks. */
int ht_mlp_get_moments(const ht_mlp* net, float* m, float* v, int32_t* step);

/* ---------------------------------------------------------------- tracking */

/* Parameters of the predictor-corrector loop (Section 2 leaves every value
 * open; ht_default_params gives this library's defaults). */
typedef struct ht_params {
  double h0;          /* first step size in t */
  double h_min;       /* a path fails when a rejection takes the step below this */
  double h_max;       /* largest step size */
  double f_up;        /* step growth after an accepted step (>= 1) */
  double f_down;      /* step shrink after a rejected step (0 < f_down < 1) */
  double tol_dx;      /* corrector converged: |dx|_inf <= tol_dx max(1, |x|_inf) ... */
  double tol_res;     /* ... and |h|_inf <= tol_res max(1, |x|_inf)^deg (deg: largest degree) */
  double tol_polish;  /* Newton at t = 1 stops when |dx|_inf <= tol_polish max(1, |x|_inf) */
  double r_div;       /* an accepted point with |x|_inf > r_div ends the path as diverged */
  int32_t newton_max; /* evaluate-correct rounds per step (1..100) */
  int32_t polish_max; /* Newton steps at t = 1 (0..100) */
  int32_t max_steps;  /* steps (accepted + rejected) before a path fails */
  int32_t max_order;  /* predictor order: extrapolation through up to max_order + 1 points (0..7) */
  int32_t team_warps;       /* warps serving one group of 32 paths (1..8; 16 for D and DD);
                               0 = chosen per round: the tuned or built-in size, and 16 warps for D
                               and DD systems with n >= 8 while fewer groups than SMs are active */
  int32_t iters_per_launch; /* Newton steps per kernel launch; 0 = default (4) */
  int32_t rounds_per_sync;  /* launches between host reads of the active count, even; 0 = default (8) */
  int32_t predictor;        /* 0 extrapolation through up to max_order + 1 accepted points (default);
                               1 Euler and 2 cubic Hermite on the path's tangent v = dx/dt, which each
                               Newton round also solves from J v = -dh/dt with the same factorisation
                               (Euler: x + (t1 - t) v at the current point; Hermite: the cubic matching
                               the current and the previous accepted point and their tangents).  The
                               start point has no tangent: until one exists the step predicts x itself,
                               and Hermite uses Euler while only the current point has one */
} ht_params;

/* Counts of one ht_track_paths call. */
typedef struct ht_stats {
  int64_t converged, failed, diverged; /* final status 1, -1, -2 */
  int64_t steps, rejects, newton;      /* totals over all paths */
  int32_t launches;                    /* kernel launches (tracking + compaction) */
  int32_t syncs;                       /* host reads of the active count */
  double ms;                           /* wall time of the call */
} ht_stats;

/* Defaults for `limbs` (HT_D, HT_DD, HT_QD): h0 0.05, h_min 1e-5, h_max 0.1,
 * f_up 1.5, f_down 0.5, tol_dx 1e-6, tol_res 1e-4, tol_polish 1e-12 / 1e-24 /
 * 1e-48, r_div 1e8, newton_max 3, polish_max 4, max_steps 2000, max_order 4, predictor 0. */
int ht_default_params(int limbs, ht_params* p);

/*
 * ht_start_solutions -- start points of the total-degree start system
 * g_i = x_i^d_i - 1 (Eq. eqlinhom): path q gets x_i = exp(2 pi i k_i / d_i)
 * with (k_0, k_1, ...) the mixed-radix digits of first + q, k_0 fastest, so the
 * d_0 d_1 ... d_{n-1} paths (the Bezout number) are numbered 0.. without gaps.
 *   degrees host [n], each >= 1;  x0 device [n][2][limbs][count].
 * Blocks until the points are written.
 */
int ht_start_solutions(int n, const int32_t* degrees, int limbs, int64_t first, int64_t count, double* x0,
                       void* stream);

/*
 * ht_mgs_solve -- least squares min |A x - b| for n_sys independent complex
 * systems by modified Gram-Schmidt on the augmented matrix [A | b] followed by
 * back substitution (the corrector's linear solve, Section 1 and Table
 * tabmemory "correct").
 *   Ab  device [rows][cols + 1][2][limbs][n_sys]: A then b as the last column;
 *       overwritten with Q
 *   R   device [cols][cols + 1][2][limbs][n_sys]: workspace, receives R (its
 *       diagonal holds 1 / r_qq)
 *   x   device [cols][2][limbs][n_sys]
 * rows >= cols >= 1.  A rank-deficient system gives non-finite x.  Async.
 */
int ht_mgs_solve(int limbs, int rows, int cols, int64_t n_sys, double* Ab, double* R, double* x, void* stream);

/*
 * ht_mgs_solve_ex -- ht_mgs_solve with a choice of arithmetic:
 *   variant 0  error-free DD/QD arithmetic on the FP64 pipe (ht_mgs_solve);
 *   variant 2  integer limbs (limbs 2 or 4, rows <= 64): every entry is read
 *              as a radix-2^29 limb string, every dot product and norm is one
 *              exact fixed-point sum of its products rounded once, 1/r_qq
 *              comes from Newton's iteration for 1/sqrt; results are written
 *              back as doubles (the leading 53-bit pieces of each value).
 * The tracker uses variant 2 for QD systems unless ht_set_eval_config chose
 * an FP64 variant.  Errors as ht_mgs_solve; HT_EUNSUPPORTED for
 * variant 2 with limbs 1 or more than 64 rows.
 */
int ht_mgs_solve_ex(int limbs, int variant, int rows, int cols, int64_t n_sys, double* Ab, double* R, double* x,
                    void* stream);

/*
 * ht_compact -- the scan of Table tabjobidx: path_idx receives, in increasing
 * order, the indices i < m with status[i] == 0, and *count their number.
 *   status device [m] (int8), path_idx device [m] (int32), count device [1].
 * m < 2^31.  Blocks until done.
 */
int ht_compact(const int8_t* status, int64_t m, int32_t* path_idx, int32_t* count, void* stream);

/*
 * ht_track_paths -- track n_paths solution paths of
 *     gamma (1 - t) g(x) + t f(x) = 0,   g_i(x) = x_i^start_deg[i] - 1,
 * from t = 0 to t = 1 (Eq. eqlinhom, Section 2): per step an extrapolation
 * predictor through the current and up to max_order previous points, then up
 * to newton_max evaluate-correct rounds (Newton with least squares by modified
 * Gram-Schmidt), then step-size control; converged paths are refined by Newton
 * at t = 1.  Status per path (Section 2, plus a reason code for failures):
 * 1 success, -1 failure (step below h_min, too many steps, non-finite point),
 * -2 diverged (|x|_inf > r_div).
 *   f          square system (n_polys == n_vars == n) of the chosen precision;
 *              the call keeps a workspace and CUDA graphs in it
 *   start_deg  host [n], 1..64
 *   gamma      host [2]: the random complex constant (re, im), nonzero
 *   first_path paths first_path .. first_path + n_paths - 1 of the start
 *              system when x0 is NULL (see ht_start_solutions)
 *   x0         device [n][2][L][n_paths] start points, or NULL
 *   p          parameters, or NULL for ht_default_params(L)
 *   x_end      device [n][2][L][n_paths]: last accepted point of each path
 *   status     device [n_paths] (int8)
 *   t_end      device [n_paths]: t of the last accepted point
 *   steps      device [n_paths] (int32) steps per path, or NULL
 *   stats      host, or NULL
 * Launch shape: p->team_warps warps per group of 32 paths and
 * p->iters_per_launch Newton rounds per launch, or, where they are 0, the
 * system's tuned shape (ht_tune_track) or the built-in one.  Results do not
 * depend on the shape.
 * Blocks until every path has finished.  HT_ETIMEOUT if paths are still
 * active after the step limit allows (a bug guard).
 */
int ht_track_paths(ht_system* f, const int32_t* start_deg, const double* gamma, int64_t n_paths, int64_t first_path,
                   const double* x0, const ht_params* p, double* x_end, int8_t* status, double* t_end,
                   int32_t* steps, ht_stats* stats, void* stream);

/*
 * ht_track_paths_ex -- ht_track_paths with optional extras (io may be NULL,
 * which makes it ht_track_paths):
 *
 *   Restart from recorded states.  init_records (device [n_paths][R] doubles,
 *   R = ht_record_size(n, L, max_order)) gives every path its t, step size h,
 *   history of accepted points and last-step summary; x0 and first_path are
 *   then ignored.  Used to probe what step a state allows (labels for the
 *   learned step).
 *
 *   Step-start recording.  With trace != NULL, the state of each path at the
 *   start of every trace_stride-th step is written as one record to trace
 *   (device [trace_capacity][R]); *trace_count (device, zero it first) counts
 *   the records offered, and those beyond trace_capacity are dropped.
 *
 *   Learned step sizes.  With mlp != NULL, at the start of each step the
 *   network maps the step features (ht_step_features) to rho; the step tried
 *   is clamp(h exp(clamp(rho, rho_min, rho_max)), h_min, h_max) in place of
 *   the plain rule's h.  With alpha_max > 0 the second output is a tangent
 *   correction: the learned step's predicted point is x + (1 + alpha)(p - x)
 *   with p the extrapolation predictor's point, x the current point and
 *   alpha = clamp(output, -alpha_max, alpha_max).  The corrector still judges
 *   the step: a rejected learned step shrinks as usual and the next
 *   fallback_steps steps of that path use the plain rule.
 *
 *   Start points of another precision.  x0_limbs (1, 2 or 4, at most the
 *   system's L; 0 means L) is the number of limbs per component of x0, laid
 *   out [n][2][x0_limbs][n_paths]; the missing limbs are zero.  With fewer
 *   limbs than L, x0 must not overlap x_end.
 *
 *   Endpoint refinement.  With polish_only != 0 (x0 required, no
 *   init_records, polish_max >= 1) every path starts at t = 1 in the polish
 *   phase: Newton's method on the target system f alone, in the system's
 *   precision, until |dx|_inf <= tol_polish max(1, |x|_inf) or polish_max
 *   rounds; status 1 if the final point is finite, -1 otherwise.  Used to
 *   check endpoints of a lower-precision run in a higher precision.
 *
 *   Last norms.  last_dx_out / last_res_out (device [n_paths], optional)
 *   receive |dx|_inf and |h|_inf of each path's last Newton round (of its
 *   last step, or of its last polish round); newton_out (device [n_paths],
 *   optional) the number of Newton rounds each path took.
 *
 * Record layout: 16 header doubles [path index in this call, t, h, number of
 * history points nh, |dx|_inf and |h|_inf of the last Newton round, rounds of
 * the last step, last step rejected (0/1), 8 zeros], then the t of the
 * max_order + 1 history slots, then the history points
 * [max_order + 1][n][2][L] (oldest first; slots past nh are zero).
 */
typedef struct ht_track_io {
  const double* init_records;
  double* trace;
  int64_t trace_capacity;
  unsigned long long* trace_count;
  int32_t trace_stride;
  int32_t fallback_steps;
  const ht_mlp* mlp;
  double rho_min, rho_max;
  int32_t x0_limbs;      /* limbs per component in x0 (0: the system's L) */
  int32_t polish_only;   /* nonzero: Newton at t = 1 from x0 only */
  double* last_dx_out;   /* device [n_paths] or NULL */
  double* last_res_out;  /* device [n_paths] or NULL */
  int32_t* newton_out;   /* device [n_paths] or NULL */
  double alpha_max;      /* learned tangent correction clamp in [0, 1] (0: off) */
} ht_track_io;

int ht_track_paths_ex(ht_system* f, const int32_t* start_deg, const double* gamma, int64_t n_paths,
                      int64_t first_path, const double* x0, const ht_params* p, double* x_end, int8_t* status,
                      double* t_end, int32_t* steps, ht_stats* stats, const ht_track_io* io, void* stream);

/*
 * ht_track_refined -- mixed-precision tracking, the "quality up" of Sections 1
 * and 4.4 (the speed of the device spent on accuracy rather than on time):
 *   1. every path is tracked in the precision of `lo` (ht_track_paths);
 *   2. every endpoint is refined by Newton's method on f in the precision of
 *      `hi` (ht_track_paths_ex with polish_only, p_hi->polish_max rounds, x0
 *      the low-precision endpoints);
 *   3. every path that failed or diverged in step 1, or whose refinement
 *      ended non-finite or with its last update above
 *      p_hi->tol_polish max(1, |x|_inf), is tracked again from its start
 *      point in the precision of `hi`; its results replace step 2's.
 * A path tracked again is the high-precision run's path bit for bit; the
 * others end at the root the low-precision path reached, to the high
 * precision's accuracy.
 *   lo, hi     the same system (same monomials) created with fewer limbs
 *              (lo) and more limbs (hi); both keep workspaces
 *   start_deg, gamma, n_paths, first_path   as ht_track_paths
 *   p_lo, p_hi parameters of the two precisions (NULL: ht_default_params)
 *   x_end      device [n][2][L_hi][n_paths]; status, t_end as ht_track_paths
 *   rs         host, or NULL: final counts, step-1 converged count, paths
 *              tracked again, and the wall time of each step
 * Allocates (stream-ordered) workspaces for the low-precision run and the
 * selected paths.  Blocks until done.
 */
typedef struct ht_refine_stats {
  int64_t converged, failed, diverged; /* final status 1, -1, -2 */
  int64_t lo_converged;                /* converged in the low precision */
  int64_t retracked;                   /* paths tracked again in the high precision */
  double ms_lo, ms_refine, ms_retrack; /* wall time of steps 1, 2 (with the selection), 3 */
} ht_refine_stats;

int ht_track_refined(ht_system* lo, ht_system* hi, const int32_t* start_deg, const double* gamma, int64_t n_paths,
                     int64_t first_path, const ht_params* p_lo, const ht_params* p_hi, double* x_end, int8_t* status,
                     double* t_end, ht_refine_stats* rs, void* stream);

/*
 * ht_tune_track -- autotuner for ht_track_paths on this system: tracks the
 * first n_paths paths (from the start solutions) once per candidate launch
 * shape -- team_warps in {1, 2, 4, 8} (up to n; also 16 for D and DD with n >= 8) and iters_per_launch in
 * {2, 4, 8}, p's other settings unchanged (p may be NULL: defaults) -- keeps
 * the fastest (wall time of the call) in the system, where it replaces the
 * built-in choice whenever a call's params leave team_warps or
 * iters_per_launch at 0, and reports it (output pointers may be NULL).  The
 * launch shape changes the speed only: every team size and launch shape gives
 * the same results.  Allocates its own output buffers.  Blocks.
 */
int ht_tune_track(ht_system* f, const int32_t* start_deg, const double* gamma, int64_t n_paths, const ht_params* p,
                  int* team_warps, int* iters_per_launch, double* best_ms, void* stream);

/*
 * ht_step_labels -- training labels for the learned step: every record is
 * restarted once per multiplier mu_j (mults host [n_mult], n_mult <= 64) with
 * its step h scaled by mu_j, and takes one step of at most newton_max
 * evaluate-correct rounds (p's other settings apply; h_min is lifted).  Among
 * the accepted probes the label takes the one with the most progress per
 * round, mu_j / rounds_j (ties to the larger mu_j): rho = log mu_j (log of the
 * smallest mu_j if no probe was accepted); the second output is that probe's
 * tangent correction alpha = Re <p - x, x* - p> / |p - x|^2 (x the record's
 * point, p the extrapolation predictor's point at the probe's t1, x* the
 * probe's corrected point; leading limbs, clamped to [-1, 1]; 0 without an
 * accepted probe or when p = x).
 *   records device [n_rec][R]; labels device [n_rec][2] floats.  Blocks.
 */
int ht_step_labels(ht_system* f, const int32_t* start_deg, const double* gamma, const ht_params* p, int64_t n_rec,
                   const double* records, int n_mult, const double* mults, int newton_max, float* labels,
                   void* stream);

/* Doubles per step-start record for n variables, `limbs` limbs and predictor
 * order max_order (-1 for invalid arguments). */
int64_t ht_record_size(int n, int limbs, int max_order);

/*
 * ht_step_features -- the 16 inputs of the learned step for each record
 * (device [n_rec][R] -> device [n_rec][16] floats), computed by the same device
 * code the tracker uses, on the leading limbs: t, log10 h, log10 |dx/dt|_inf / 4
 * (from the last two accepted points), log10 of the last round's |dx|_inf and
 * |h|_inf / 16, last step's rounds / newton_max, last step rejected,
 * nh / (max_order + 1), log10(1 - t) / 16, log10 of the curvature estimate
 * 2 |second divided difference|_inf over the last three accepted points / 8
 * (0 with fewer than three), log10(h / last accepted step) / 2 (0 with fewer
 * than two), each clamped to [-4, 4], then zeros.  Async.
 */
int ht_step_features(int n, int limbs, int max_order, int newton_max, int64_t n_rec, const double* records,
                     float* features, void* stream);

/*
 * ht_compact_noalloc -- ht_compact for callers that cannot allocate device
 * memory.  The paper has no counterpart; this is an interface variant.
 *
 * Who needs it: code that runs where cudaMalloc and cudaFree are forbidden or
 * harmful.  Examples are a host thread inside another framework's allocator
 * (which must own every device allocation), a latency-critical loop that must
 * not synchronise the device the way cudaFree can, or a caller with a fixed
 * memory budget.  ht_compact allocates a temporary index list on every call;
 * this variant instead uses a fixed array of HT_NOALLOC_MAX_PATHS + 1 int32
 * (16 MiB) that the library declares at file scope.  Every GPU that loads the
 * library holds that array until the process exits.
 *
 * Same arguments, result and blocking behaviour as ht_compact, except:
 *   - m above HT_NOALLOC_MAX_PATHS is rejected with HT_EINVAL;
 *   - no cudaMalloc, cudaFree or other allocating routine is called;
 *   - every call looks up the array's device address in the current context
 *     (cudaGetSymbolAddress, which allocates nothing); the first call on a
 *     device also loads the library's module there, so make it before any
 *     stream capture;
 *   - all calls share the one array, which keeps the last call's contents.
 *     Each call rewrites all of it that it reads.  Calls whose work overlaps on
 *     the GPU (other streams, other host threads) race on it, so serialise them.
 */
#define HT_NOALLOC_MAX_PATHS (1 << 22)
int ht_compact_noalloc(const int8_t* status, int64_t m, int32_t* path_idx, int32_t* count, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HT_H */
