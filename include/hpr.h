/*
 * hpr.h -- C ABI of the B300 HPR-LP solver (CUDA, sm_103a).
 *
 * Solves the linear program of Section 1, eq. (1) of Chen, Sun, Yuan, Zhang & Zhao,
 * "HPR-LP: An implementation of an HPR method for solving linear programming"
 * (arXiv 2408.12179):
 *
 *     min <c, x>   s.t.   A1 x = b1,   A2 x >= b2,   l <= x <= u,
 *
 * and its dual eq. (2), with the Halpern Peaceman-Rachford method of Algorithm 2
 * (semi-proximal term T1 = lambda I - A A^*, Section 3.3), the restart criteria of
 * Section 3.1, the sigma update of Algorithm 3 / eq. (sigma_T1!=0), and the
 * preprocessing, power method and termination test of Section 4.1.
 *
 * Conventions for every entry point:
 *   - all array arguments are HOST pointers unless stated otherwise;
 *   - nothing is retained: hpr_create deep-copies its inputs to the GPU, the caller
 *     may free them on return; every device allocation belongs to the context and is
 *     released by hpr_destroy;
 *   - errors are returned as a status code (never thrown across the ABI); the detail
 *     of the last error of a context is in hpr_last_error();
 *   - a context is not thread-safe; separate contexts are independent.  A context
 *     uses the CUDA device that was current when it was created.
 *
 * Host-side fault injection, for testing the error paths without faulting a GPU (read
 * from the environment by hpr_create; unset or 0: off):
 *   HPR_FAULT_ALLOC=n      the n-th device or pinned host allocation that the context
 *                          makes (creation and solves counted together) reports
 *                          out-of-memory: the call returns HPR_ERR_NOMEM and a context
 *                          that exists stays valid for hpr_destroy;
 *   HPR_FAULT_NAN_CHECK=n  the check scalars of the n-th check period of the multi-CTA
 *                          path are replaced by NaN on the host after read-back: the solve
 *                          returns HPR_ERR_NUMERIC;
 *   HPR_FAULT_BARRIER=n    persistent grid path (persistent = 3): its last CTA skips its
 *                          arrival at grid barrier n-1; persistent cluster path: its last
 *                          CTA does not send its rows of x_hat in iteration n-1.  Every
 *                          wait's budget drops to 200 us: the solve returns
 *                          HPR_ERR_DEVICE_TIMEOUT.
 * and, for measurements, HPR_GRID_CTAS=G: the CTA count of the persistent grid path (at
 * most one per SM) and of the cluster path (at most 16; the largest resident cluster up to
 * G is taken); unset or 0: chosen from the FP64 work of an iteration.
 */
#ifndef HPR_H
#define HPR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
enum {
    HPR_OK = 0,              /* converged: KKT residual <= tol (Section 4.1) */
    HPR_MAX_ITER = 1,        /* iteration limit reached; the last w_bar is retrievable */
    HPR_TIME_LIMIT = 2,      /* time limit reached; the last w_bar is retrievable */
    HPR_ERR_ARG = -1,        /* NULL / inconsistent sizes, unsorted or duplicate column
                                indices, non-finite data, l > u, l = +inf or u = -inf */
    HPR_ERR_ZERO_MATRIX = -2,/* A has no nonzero entry (Section 1 assumes A != 0) */
    HPR_ERR_NOMEM = -3,      /* device or pinned host allocation failed */
    HPR_ERR_CUDA = -4,       /* any other CUDA runtime error */
    HPR_ERR_DEVICE_TIMEOUT = -5, /* a bounded device-side wait gave up */
    HPR_ERR_NUMERIC = -6,    /* a residual became NaN or infinite */
    HPR_ERR_STATE = -7,      /* call out of order (e.g. results requested before a solve) */
    HPR_ERR_NO_DEVICE = -8   /* no CUDA device or not an sm_103 device */
};

typedef struct hpr_ctx hpr_ctx;

/* A sparse block in CSR form (host arrays).  row_ptr[0] = 0, row_ptr[rows] = nnz,
 * non-decreasing; col_idx strictly increasing within a row and in [0, cols); val
 * finite.  A block with rows = 0 may pass NULL arrays; a NULL hpr_csr* means an
 * empty block. */
typedef struct {
    int64_t rows, cols, nnz;
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const double *val;
} hpr_csr;

/* Solver options.  hpr_default_options() fills the paper's settings (Section 4.1). */
typedef struct {
    double tol;               /* stopping tolerance eps of Section 4.1 (1e-8) */
    int64_t max_iter;         /* iteration limit (10,000,000) */
    double time_limit_s;      /* wall-clock limit of hpr_solve; <= 0: none */
    int64_t check_every;      /* termination / restart check period (150, Section 4.1) */
    double alpha1, alpha2, alpha3; /* restart parameters (0.2, 0.6, 0.2, Section 4.1) */
    double sigma0;            /* initial penalty parameter (1) */
    int64_t ruiz_iters;       /* Ruiz iterations (10) */
    double pc_alpha;          /* Pock-Chambolle alpha (1); negative disables that step */
    int64_t power_max_iter;   /* power-method iteration cap (5000) */
    double power_tol;         /* stop when |lambda_k - lambda_{k-1}| <= tol lambda_k (1e-10) */
    uint64_t seed;            /* SplitMix64 seed of the power-method start vector */
    double lambda_fixed;      /* > 0: use this lambda (T1 = lambda I - A A^*) and skip the
                                 power method; 0: power method (default) */
    int64_t restart;          /* 0 disables the restart criteria (ablation) */
    int64_t sigma_update;     /* 0 keeps sigma at restarts (ablation) */
    int64_t trace_iters;      /* record the scaled iterates of the first trace_iters
                                 iterations (for parity checks; slow) */
    int64_t use_graph;        /* 1: run each check period as one captured CUDA graph */
    int64_t verbose;          /* 1: print one line per check to stderr */
    void *cuda_stream;        /* cudaStream_t to order the work after; NULL: the
                                 context's own stream */
    int64_t precision;        /* 0: FP64 throughout (default).  1: FP32 form first -- FP32
                                 matrix values and FP32 iterates x, x_hat, y, row sums of
                                 FP32 products accumulated in double-float, FP64 anchors,
                                 data, epilogue arithmetic, checks and power method --
                                 then FP64 iterates from the first check with
                                 kkt < switch_tol */
    double switch_tol;        /* KKT level of the switch to FP64 iterates (1e-5) */
    int64_t halpern;          /* 1: Halpern step w = w0/(t+2) + (t+1)/(t+2) w_target of
                                 Algorithm 2 (default); 0: w = w_target (ablation) */
    int64_t reflect;          /* 1: w_target = w_hat = 2 w_bar - w, the relaxation step of
                                 Algorithm 2 (default); 0: w_target = w_bar (the DR and
                                 HDR variants of the Section 4.2 ablation).  The y step
                                 uses A(2 x_bar - x) either way (eq. update-y-2) */
    int64_t autotune;         /* 1: at hpr_create, time the phase kernels with candidate
                                 sliced-ELL layouts (lanes-per-row bound 16..128, work-unit
                                 size 32..256) for A and A^T and keep the fastest; 0 (default):
                                 the layouts given below */
    int64_t sell_steps_a, sell_steps_t;  /* lanes-per-row bound of A's / A^T's layout: a group
                                 of 32 rows uses the fewest lanes per row (1..32) that keep
                                 its longest row within this many steps; 0: 40, or 16 when
                                 the phase's algorithmic traffic is below 40 MB (the x phase:
                                 12 nnz + 60 n + 8 m bytes, the y phase: 12 nnz + 8 n + 36 m) */
    double unit_cost_a, unit_cost_t;     /* work-unit size of A's / A^T's layout (a group
                                 costlier than this is split into one unit per slice); 0: 64,
                                 or 32 below the same 40 MB */
    int64_t sigma_policy;     /* sigma at a restart where Algorithm 3 computes Delta_x / Delta_y:
                                 0 (default) that value; 1 (exploration, for training data)
                                 2^((a-2)/2) times it with a in 0..4 drawn by SplitMix64 from
                                 policy_seed and the restart count; 2 the same multiplier with
                                 a = the argmin of the policy network set by hpr_set_policy,
                                 except after a learned choice whose inner loop saw the KKT
                                 residual rise above its value at the decision: the next
                                 restart then keeps Algorithm 3's value (a fallback) */
    uint64_t policy_seed;
    double policy_margin;     /* sigma_policy 2: a multiplier other than 1 (a = 2) is taken only
                                 when its predicted outcome beats a = 2's by more than this
                                 (log10 KKT units; default 0) */
    int64_t persistent;       /* the persistent paths, which run the power method and all of
                                 Algorithm 2 in one launch (plain FP64 solves without tracing,
                                 time limit or policy only):
                                   single-CTA: one CTA of 1024 threads, iterates in shared memory
                                   (LPs with 48 n + 32 m bytes <= 200 KB);
                                   cluster: one thread-block cluster of up to 16 CTAs, y and
                                   x_hat replicated in every CTA's shared memory and filled by
                                   stores that count on a transaction barrier per replica, each
                                   wait bounded (HPR_ERR_DEVICE_TIMEOUT), the CTAs' slices of A
                                   and A^T and their rows in their own shared memory (LPs with
                                   8 (m + n) bytes plus a CTA's share of the matrices within one
                                   CTA's shared memory, ~227 KB);
                                   grid: one cooperative launch of up to one CTA per SM, software
                                   grid barriers with a bounded wait (HPR_ERR_DEVICE_TIMEOUT when
                                   a wait runs out), gathers through L2.
                                 0 never; 1 (default) the single-CTA path when the LP fits and
                                 one SM's share of FP64 work per iteration is small enough to
                                 beat the multi-CTA path (stored entries of A and A^T / 32 + 8 x
                                 their 32-row slices <= 600), else the cluster path when it fits
                                 and is expected to be faster, else the multi-CTA path;
                                 2 / 4 / 3: the single-CTA / cluster / grid path whenever it can
                                 run (HPR_ERR_ARG if it cannot) */
    int64_t pdl;              /* 1 (default): the two phases of a normal iteration are launched as
                                 programmatic dependents of the kernel before them, so that their
                                 set-up overlaps its tail; 0: plain stream order */
    int64_t gather_tiles;     /* the x phase of normal FP64 iterations on the multi-CTA path:
                                 0 (default): the sliced-ELL kernel, which gathers y from L2;
                                 1: gather-tiled when the x phase moves at least 40 MB (12 nnz +
                                 60 n + 8 m bytes) and y takes at most one block per 4 SMs;
                                 2: gather-tiled whenever y takes at most one block per SM and
                                 the layout's offsets fit in 32 bits (HPR_ERR_ARG at hpr_create
                                 otherwise).  Gather-tiled: y is
                                 cut into blocks of consecutive entries that fit one CTA's
                                 shared memory, each CTA (one per SM) stages one block and
                                 streams the entries of A^T whose columns lie in it, the
                                 per-block partial sums of each row go to a buffer and a second
                                 kernel adds them in block order before the x update.  Row
                                 sums are added in another order than on the sliced-ELL
                                 kernel (FP64 either way).  Decided at hpr_create (the layout
                                 is built there); set to 0 later, the solve takes the
                                 sliced-ELL kernel.  Check iterations, the FP32 form's normal
                                 iterations, the persistent paths and batched solves always
                                 take their own kernels.  On the medium planted LP (m = 200k,
                                 n = 500k) the tiled x phase is slower (41 against 35 us): the
                                 split adds FP64 work (per-block sums, a separate epilogue) on
                                 B300's scarce FP64 pipe */
    int64_t tile_len;         /* gather_tiles: most entries of y in one block, 0 (default: as
                                 many as one CTA's shared memory holds, 28,928 on B300) or in
                                 [2, 65,536]; odd values are taken one lower */
} hpr_options;

/* Result summary (original, unscaled problem). */
typedef struct {
    double primal_obj, dual_obj;  /* <c,x> and <b,y> - delta_C^*(-z) */
    double err_p, err_d, err_gap; /* relative residuals of Section 4.1 */
    double kkt;                   /* max(err_p, err_d, err_gap) */
    double sigma, lambda;         /* final penalty parameter; lambda of T1 */
    double solve_time_s;          /* power method + iterations (Section 4.1 timing) */
    double power_time_s;          /* power method alone */
    double time_to_1e4_s;         /* first check with kkt <= 1e-4 (-1 if none) */
    int64_t iters_to_1e4;         /* iterations at that check (-1 if none) */
    int64_t iters, restarts, power_iters, n_checks;
    int64_t launches;             /* kernels launched by the solve (graph nodes included) */
    int64_t status;               /* HPR_OK, HPR_MAX_ITER or HPR_TIME_LIMIT */
    int64_t iters_fp32;           /* iterations run in the FP32 form (precision 1) */
    int64_t policy_decisions;     /* restarts whose sigma the policy network chose */
    int64_t policy_fallbacks;     /* restarts that fell back to Algorithm 3 (sigma_policy 2) */
    double power_rel_change;      /* power method: |lambda_k - lambda_{k-1}| / lambda_k at its last
                                     step (above power_tol when it stopped at power_max_iter) */
    int64_t path;                 /* the path the solve took, in hpr_options.persistent's codes:
                                     0 multi-CTA (launches per iteration), 2 single-CTA, 3 grid,
                                     4 cluster */
    int64_t path_ctas;            /* CTAs of the persistent grid or cluster launch (else 0) */
    int64_t x_tiles;              /* blocks of y of the gather-tiled x phase that the multi-CTA
                                     path's normal FP64 iterations took (0: the sliced-ELL x
                                     phase; see hpr_options.gather_tiles) */
} hpr_info;

/* One evaluation of the restart / termination quantities.  kind: 1 = periodic check,
 * 2 = R~_{r,0} at the first iteration of an inner loop, 3 = both.  cause: 0 none,
 * 1..3 = restart criterion eq. (restart_1)..(restart_3), -1 = terminated. */
typedef struct {
    int64_t k, r, t, kind, cause;
    double sigma, err_p, err_d, err_gap, kkt, pobj, dobj;
    double Rt, R0, sigma_next, Dx, Dy, elapsed_s;
    int64_t action;               /* sigma multiplier index of a restart (-1: Algorithm 3's) */
    double sigma_rule;            /* Algorithm 3's sigma at that restart */
} hpr_check_record;

/* Fills *opt with the defaults above.  Returns HPR_OK or HPR_ERR_ARG (opt NULL). */
int hpr_default_options(hpr_options *opt);

/* Validates and uploads the LP of eq. (1), builds the explicit CSR of A^T, and runs the
 * preprocessing of Section 4.1 on the GPU (Ruiz, Pock-Chambolle, b/c normalisation).
 * A1 is m1 x n, A2 is m2 x n (either may be NULL or have rows = 0, not both empty);
 * b1 (m1), b2 (m2), c, l, u (n) are host arrays; l may hold -inf, u +inf.
 * opt may be NULL (defaults).  On success *out owns all device memory. */
int hpr_create(hpr_ctx **out, const hpr_csr *A1, const hpr_csr *A2, const double *b1,
               const double *b2, const double *c, const double *l, const double *u,
               const hpr_options *opt);

/* Replaces the context's options (the preprocessing already done is kept; ruiz_iters
 * and pc_alpha take effect only at creation). */
int hpr_set_options(hpr_ctx *ctx, const hpr_options *opt);

/* Runs the power method of Section 4.1 on the scaled A: lambda_1(A A^*).  Writes
 * lambda and the number of iterations (either pointer may be NULL). */
int hpr_power(hpr_ctx *ctx, double *lambda, int64_t *iters);

/* Runs Algorithm 2 from the origin with sigma_0 (Section 4.1) until the termination
 * test holds for tol (> 0; overrides opt.tol), max_iter or time_limit_s.  Returns
 * HPR_OK, HPR_MAX_ITER, HPR_TIME_LIMIT or an error. */
int hpr_solve(hpr_ctx *ctx, double tol);

/* Copies the last w_bar of hpr_solve, mapped back to the original LP (x projected
 * onto C), into caller-allocated host arrays x (n), y (m1+m2), z (n) and the summary
 * into *info; any pointer may be NULL.  HPR_ERR_STATE before the first solve. */
int hpr_get(const hpr_ctx *ctx, double *x, double *y, double *z, hpr_info *info);

/* ---- Checkpoint / resume (no counterpart in the paper; its natural checkpoint is the
 * restart state of Algorithm 2: the anchor w^{r,0} = w_bar^{r-1,tau}, sigma_r, the
 * counters r and k at the restart, with lambda and the scaling).
 * hpr_get_state writes the state of the last restart of the last hpr_solve (the origin
 * and sigma_0 if it made none) into a caller buffer: an opaque blob of
 * hpr_get_state(ctx, NULL, 0, &bytes) bytes, in the solver's internal (scaled, renumbered)
 * order, valid for a context of the same LP with the same options.  hpr_set_state loads
 * such a blob; the next hpr_solve of that context then starts from it -- no power method
 * (lambda is the blob's), the restart step of Algorithm 2 applied to the stored anchor,
 * the counters continued -- and runs on the multi-CTA path.  Since a solve stopped by
 * max_iter takes no restart decision at its last check, resuming from its state replays
 * the uninterrupted solve bit for bit (same iterations, same w_bar).
 *   hpr_get_state: HPR_ERR_STATE before a solve, or when the last solve ran on a
 *                  persistent path (persistent = 2, 3, 4, or 1 when it chose one: its
 *                  anchors live in shared memory; solve with persistent = 0 to checkpoint);
 *                  HPR_ERR_ARG when buf is non-NULL and bytes is smaller than needed.
 *   hpr_set_state: HPR_ERR_ARG when the blob is shorter than needed, or was taken from
 *                  another LP (sizes or scaling differ) or another build of the blob;
 *                  HPR_ERR_STATE for a context in a batch, with tracing or a sigma
 *                  policy (their history is not part of the state). */
int hpr_get_state(const hpr_ctx *ctx, void *buf, int64_t bytes, int64_t *needed);
int hpr_set_state(hpr_ctx *ctx, const void *buf, int64_t bytes);

/* Preprocessing results: D_r (m), D_c (n), the scaled values of A in the CSR order of
 * [A1; A2] (nnz), the scaled b (m), c, l, u (n) and beta = {||D_r b||+1, ||D_c c||+1}
 * (2).  Any pointer may be NULL. */
int hpr_get_scaling(const hpr_ctx *ctx, double *Dr, double *Dc, double *As_val,
                    double *bs, double *cs, double *ls, double *us, double *beta);

/* The check records of the last solve, in order: copies min(cap, count) records into
 * out (may be NULL with cap 0) and the count into *count. */
int hpr_get_checks(const hpr_ctx *ctx, hpr_check_record *out, int64_t cap, int64_t *count);

/* Scaled-space iterates of iteration k (0-based, k < trace_iters and < iterations
 * run) of the last solve: x_bar, x_hat (n), x after the Halpern / restart step (n),
 * y_bar (m) and y after the step (m).  Any pointer may be NULL. */
int hpr_get_trace(const hpr_ctx *ctx, int64_t k, double *xbar, double *xhat, double *x,
                  double *ybar, double *y);

/* Times `reps` plain HPR iterations (Section 3.3: the A^T phase with the x update,
 * then the A phase with the y update) of the form selected by opt.precision: reps + 2
 * iterations are enqueued back to back on the context's stream with a CUDA event between
 * every two kernels and one host synchronisation at the end; the first two iterations
 * are left out of the averages.  Starts from the current iterate and advances it (call
 * after hpr_solve).  Writes the average duration in milliseconds of the x phase (ms_x),
 * the y phase (ms_y) and of a whole iteration (ms_iter); any pointer may be NULL.
 * HPR_ERR_STATE before the first solve. */
int hpr_time_iteration(hpr_ctx *ctx, int64_t reps, double *ms_x, double *ms_y, double *ms_iter);

/* Allocation-free power method (the paper has no counterpart: it is an extra entry
 * point of this library).  For callers that are not allowed to allocate device memory
 * themselves -- code that runs under a memory budget or pool owned by someone else
 * (an inference server, a framework's caching allocator) or that must not call
 * cudaMalloc at that point -- and that already hold the LP matrix on the device.
 * Computes the same lambda_1(A A^*) as hpr_power on the given matrix (the largest
 * eigenvalue of A A^* by power iteration from a SplitMix64 start vector), but allocates
 * nothing: its per-CTA partial sums, reduced scalars and control block live in one
 * fixed array of 131,456 bytes in device global memory that is part of the library
 * and stays allocated on every device that loaded the library until the process exits.
 *   m, n            rows and columns of A; each in [1, 2^31 - 2] (otherwise HPR_ERR_ARG)
 *   A_*, At_*       DEVICE CSR arrays (32-bit) of A (m rows) and of its transpose
 *                   (n rows), column indices sorted within rows
 *   seed, max_iter, tol   as in hpr_options (power_max_iter, power_tol)
 *   u (m), s (n)    DEVICE output buffers: the final unit vector u and s = A^T u of
 *                   the last step (both are overwritten during the iteration)
 *   cuda_stream     cudaStream_t to run on (NULL: the legacy default stream)
 *   lambda, iters   HOST outputs (may be NULL)
 * The call copies a control block to the device and synchronises its stream every 16
 * power steps, so it must not be made while its stream is being captured into a CUDA
 * graph.  The first call on a device looks up the array's device address with that
 * device current.  All calls on a device share the array, so calls that
 * overlap on the GPU (other threads, other streams) race and must be serialised by the
 * caller.  Returns HPR_OK, HPR_ERR_ARG, HPR_ERR_NUMERIC or HPR_ERR_CUDA; the detail is
 * in hpr_last_error(NULL). */
int hpr_power_noalloc(int64_t m, int64_t n, const int32_t *A_row_ptr, const int32_t *A_col_idx,
                      const double *A_val, const int32_t *At_row_ptr, const int32_t *At_col_idx,
                      const double *At_val, uint64_t seed, int64_t max_iter, double tol,
                      double *u, double *s, void *cuda_stream, double *lambda, int64_t *iters);

/* Memory-system probe (no counterpart in the paper: a measurement helper for the roofline
 * of the phase kernels, which are bound by HBM bandwidth for their streamed arrays and by
 * the rate of random 8-byte gathers, each costing an L1 cache-tag lookup).  On the current
 * device and `cuda_stream` (NULL: the legacy default stream), timed with CUDA events, best of
 * five runs after one warm-up:
 *   *read_gbs    a read-only stream of read_bytes bytes (16-byte loads, integer consumer, no
 *                FP64 work) after L2 was filled with another buffer: GB/s;
 *   *gather_gps  random 8-byte gathers from an L2-resident array of gather_len doubles
 *                (indices hashed in registers, integer consumer): 1e9 gathers/s.
 * read_bytes in [2^20, 2^34]; gather_len a power of two in [2^10, 2^28].  Allocates and frees
 * its own device buffers (read_bytes + max(4 x L2 size, 256 MiB) + 8 gather_len bytes).
 * Returns HPR_OK, HPR_ERR_ARG, HPR_ERR_NO_DEVICE, HPR_ERR_NOMEM or HPR_ERR_CUDA; detail in
 * hpr_last_error(NULL). */
/* ---- Bounds-checking build (no counterpart in the paper; a test build standing in for a
 * memory checker).  Built with HPR_BOUNDS_CHECK, every gather's index -- the sliced-ELL
 * SpMVs of all paths, the allocation-free power method, the preprocessing's column scaling
 * and permutation gathers -- is checked against the length of the vector it reads; an index
 * out of range is counted and replaced by 0, so the load stays in bounds and no kernel
 * traps.  hpr_bounds_violations waits for the current device and returns the count since
 * the library was loaded in *count (-1 in the normal build, which checks nothing).  Returns
 * HPR_OK, HPR_ERR_ARG (count NULL) or HPR_ERR_CUDA. */
int hpr_bounds_violations(int64_t *count);

int hpr_memory_probe(int64_t read_bytes, int64_t gather_len, void *cuda_stream, double *read_gbs,
                     double *gather_gps);

/* ---- FP64 issue probe (no counterpart in the paper: a measurement aid for the benchmark's
 * roofline).  B300 issues FP64 at a small fraction of its FP32 rate, and every stored matrix
 * entry of an HPR phase costs one DFMA: the phases are bound by FP64 issue as well as by HBM.
 * Times a kernel of independent DFMA chains (eight per thread, 8 warps per CTA, 8 CTAs per
 * SM) on the current device and writes the whole GPU's rate of FP64 warp instructions, in
 * 1e9 per second, to *warp_ginst_per_s (best of three launches after a warm-up).
 *   cuda_stream   stream to run on (NULL: the legacy default stream); the call synchronises it.
 * Allocates and frees 64 bytes of device memory.  Returns HPR_OK, HPR_ERR_ARG (NULL output),
 * HPR_ERR_NO_DEVICE or HPR_ERR_NOMEM / HPR_ERR_CUDA (detail in hpr_last_error(NULL)). */
int hpr_fp64_probe(void *cuda_stream, double *warp_ginst_per_s);

/* Layout of the context's sliced-ELL copies (no counterpart in the paper: a storage choice
 * of this library), after autotuning if asked: for A (index 0) and A^T (index 1) the
 * lanes-per-row bound, the work-unit size and the number of work units; any pointer may
 * be NULL.  Returns HPR_OK or HPR_ERR_ARG (ctx NULL). */
int hpr_get_layout(const hpr_ctx *ctx, int64_t *sell_steps, double *unit_cost, int64_t *units);

/* Host only (no device work, no context; for tests and tools): the sliced-ELL layout that
 * hpr_create builds for the rows of the CSR matrix B, with B's own column numbering.  Rows
 * are taken in order of decreasing length (stable) in groups of 32; a group gives each row
 * L = 2^slg lanes, the fewest (L <= 32) that keep its longest row within steps_max steps,
 * and is stored as L slices of 32 / L rows, column-major: entry e of the q-th row of a slice
 * sits at sptr[s] + (e / L) * 32 + q * L + e % L.  Work units (one warp each) are a group
 * whole, or each of its slices when the group's cost (steps + 2 + log2 L + the epilogue's
 * share 8 * rows / 32, summed over its slices) exceeds unit_cost.
 *   steps_max in [1, 4096], unit_cost > 0: the layout parameters (hpr_options.sell_steps_*,
 *   unit_cost_*).  Sizes go to *nslices, *entries (stored entries, padding included) and
 *   *units (any may be NULL).  Each array may be NULL, else it must hold: row_order rows
 *   (row_order[new] = old), srow and sptr nslices + 1 (first row, first entry of slice s),
 *   slg nslices, col and src entries (src: the CSR position of each stored entry, -1 for
 *   padding, whose col is 0), wstart units + 1 (first slice of each unit).  Call once with
 *   NULL arrays for the sizes.  Returns HPR_OK, or HPR_ERR_ARG (bad matrix or parameters;
 *   detail in hpr_last_error(NULL)). */
int hpr_layout_plan(const hpr_csr *B, int64_t steps_max, double unit_cost, int64_t *nslices, int64_t *entries,
                    int64_t *units, int32_t *row_order, int32_t *srow, int32_t *sptr, uint8_t *slg, int32_t *col,
                    int32_t *src, int32_t *wstart);

/* Host only (no device work, no context; for tests): the gather-tiled layout that hpr_create
 * builds for the x phase when hpr_options.gather_tiles asks for it (no counterpart in the
 * paper), here for the rows of the CSR matrix B with B's own column numbering and rows in
 * order of decreasing length (stable, row_order).  The gathered vector (B's columns) is cut
 * into nblk blocks of consecutive entries, at most tile_len (taken even) each and starting
 * at even indices, balanced by stored entries (bstart, nblk + 1).  Each block gets CTAs of
 * a grid of `grid` in proportion to its entries, at least one each (cta_blk, grid).  The
 * entries of each block form a sub-matrix whose rows (sub-rows: the rows with an entry in
 * the block, in row_order) take hpr_layout_plan's sliced-ELL layout (40, 64) with column
 * offsets within the block; slices and sub-rows of block b follow those of block b - 1.
 * smeta (4 per slice): first sub-row, first stored entry, steps (32 entries each), log2
 * lanes per sub-row | sub-rows << 8.  Work units are runs of slices of one block (wstart,
 * units + 1); block b owns units ustart[b] .. ustart[b+1]-1.  Sub-row t's sum goes to slot
 * oslot[t]; row r (in row_order position r) owns slots slot_ptr[r] .. slot_ptr[r+1]-1, one per
 * block holding an entry of it, in block order.  col: the column offset within the block of
 * each stored entry (padding: 0); src: its position in B's CSR arrays (padding: -1).
 *   tile_len in [2, 65536], grid in [1, 65536].  Sizes go to sizes[0..5] = nblk, slices,
 *   stored entries, sub-rows (slots), units, grid (sizes may be NULL).  Each array may be
 *   NULL, else it must hold: row_order rows, bstart and ustart nblk + 1, cta_blk grid,
 *   wstart units + 1, smeta 4 x slices, oslot sub-rows, slot_ptr rows + 1, col and src
 *   entries.  Returns HPR_OK, or HPR_ERR_ARG (bad matrix or parameters, or a layout that
 *   would need more blocks than min(grid, 256) or offsets beyond 32 bits; detail in
 *   hpr_last_error(NULL)). */
int hpr_tile_plan(const hpr_csr *B, int64_t tile_len, int64_t grid, int64_t *sizes, int32_t *row_order,
                  int32_t *bstart, int32_t *ustart, int32_t *cta_blk, int32_t *wstart, int32_t *smeta,
                  int32_t *oslot, int32_t *slot_ptr, uint16_t *col, int32_t *src);

/* ---- Batched solve (no counterpart in the paper: many independent LPs in lock step).
 * A batch takes `count` contexts made by hpr_create (their LPs may differ in size and
 * structure) and solves them together: each check period's normal iterations of all
 * contexts run as fused sliced-ELL launches over one work list of every context's work
 * units (captured as one CUDA graph per period length), while each context keeps its
 * own power method (run on up to 8 host worker threads with their own streams), checks,
 * restart / sigma decisions (Algorithm 2 and 3), FP32 -> FP64 switch and termination.
 * Results are read per context with hpr_get.  Each context's options are those set when
 * hpr_batch_solve is called (reflect: when the batch was created); all contexts need the
 * same check_every and trace_iters = 0.
 *   ctxs         `count` distinct contexts on the same device, none in another batch;
 *                the batch does not own them: destroy the batch first, then the
 *                contexts.  While in the batch a context cannot be solved on its own
 *                (hpr_solve returns HPR_ERR_STATE) and runs on the batch's stream.
 *                When the contexts' x phases (12 nnz + 60 n + 8 m bytes each) or y phases
 *                (12 nnz + 8 n + 36 m) add up to 40 MB or more, the fused phase is
 *                bandwidth-bound and the contexts whose layout took the short-slice
 *                default for small phases (no layout options, no autotune) get the
 *                default layout (40, 64) instead, for good (hpr_get_layout shows it).
 *   cuda_stream  the batch's stream (NULL: a stream of its own).
 * When every context would take the persistent single-CTA path on its own (see
 * hpr_options.persistent), the batch runs them as one launch with one CTA per LP, each
 * result equal to the context's own single-CTA solve (hpr_batch_stats: 0 periods, 1 launch).
 * Otherwise, when every context would take the persistent cluster path on its own, the
 * batch runs one launch per cluster size among them, each on a stream of its own, with
 * one cluster per LP (costliest first), each result equal to the context's own cluster
 * solve (hpr_batch_stats: 0 periods, one launch per cluster size).
 * hpr_batch_solve returns HPR_OK when every context converged, else the status of a
 * context that did not (HPR_MAX_ITER / HPR_TIME_LIMIT), or an error code; detail in
 * hpr_last_error(NULL) or of the context. */
typedef struct hpr_batch hpr_batch;
int hpr_batch_create(hpr_batch **out, int64_t count, hpr_ctx *const *ctxs, void *cuda_stream);
int hpr_batch_solve(hpr_batch *batch, double tol);
/* Wall time of the last hpr_batch_solve (power methods included), its check periods and
 * the fused (or persistent) launches it made; any pointer may be NULL. */
int hpr_batch_stats(const hpr_batch *batch, double *solve_time_s, int64_t *periods, int64_t *fused_launches);
void hpr_batch_destroy(hpr_batch *batch);

/* ---- The sigma policy network (no counterpart in the paper).  An MLP with three hidden
 * layers of 64 ReLU units maps 64 features of the recent check history (for each of the
 * last 16 checks: log10 err_p, log10 err_d, log10 gap, log10 sigma, each over 8) to five
 * outputs, the predicted change of log10 KKT after choosing sigma = 2^((a-2)/2) times
 * Algorithm 3's sigma (a = 0..4) at a restart.  Weights: hpr_mlp_param_count() FP32
 * values, rows of W[out][in] then biases, layer by layer (W1 64x64, b1, W2 64x64, b2,
 * W3 64x64, b3, W4 5x64, b4); the kernels compute with their BF16 rounding and FP32
 * accumulation.  All arrays are HOST arrays owned by the caller; X is n x 64 row-major.
 * Each returns HPR_OK, HPR_ERR_ARG (NULL array, n outside [1, 2^26], action outside
 * [0, 5), non-finite input) or HPR_ERR_NOMEM / HPR_ERR_CUDA, detail in hpr_last_error(NULL). */
int hpr_mlp_param_count(void);
/* The policy a context uses with sigma_policy = 2: w (hpr_mlp_param_count() FP32 values,
 * host) is copied; NULL removes it (sigma_policy 2 then behaves as 0).  Returns HPR_OK,
 * HPR_ERR_ARG (ctx NULL or a non-finite weight), HPR_ERR_NOMEM or HPR_ERR_CUDA. */
int hpr_set_policy(hpr_ctx *ctx, const float *w);
/* The 64 features of check record `rec` of the last solve (as the policy sees them at a
 * restart decided at that check) into out (host, 64 floats).  HPR_ERR_ARG when rec is not
 * a record of the last solve. */
int hpr_policy_features(const hpr_ctx *ctx, int64_t rec, float *out);
/* Q (n x 5): the outputs for each row of X. */
int hpr_mlp_infer(const float *w, int64_t n, const float *X, float *Q);
/* Loss L = mean_i 1/2 (Q(x_i)[act_i] - y_i)^2 and dL/dw (P values, with respect to the
 * BF16 weights) into grad and *loss. */
int hpr_mlp_grad(const float *w, int64_t n, const float *X, const int32_t *act, const float *y, float *grad,
                 double *loss);
/* Adam (beta 0.9 / 0.999, eps 1e-8, step lr) over `epochs` passes in minibatches of
 * `batch` samples, the order of each pass drawn from SplitMix64(seed); w is updated in
 * place (FP32 masters); epoch_loss (epochs values, may be NULL) gets each pass's mean
 * minibatch loss. */
int hpr_mlp_train(float *w, int64_t n, const float *X, const int32_t *act, const float *y, int64_t epochs,
                  int64_t batch, double lr, uint64_t seed, double *epoch_loss);

/* Detail of the last error of ctx.  With ctx NULL: the detail of the last failing call
 * made without a context (hpr_create, hpr_power_noalloc, hpr_batch_*, hpr_mlp_*,
 * hpr_layout_plan) on the calling host thread; it stays valid until that thread's next
 * such failure. */
const char *hpr_last_error(const hpr_ctx *ctx);

/* Name of a status code. */
const char *hpr_status_str(int status);

/* Frees everything the context owns.  NULL is ignored. */
void hpr_destroy(hpr_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* HPR_H */
