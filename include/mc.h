/*
 * libmc -- motion-compensated SPDHG on one GPU (sm_103a), C ABI.
 *
 * Method: Delplancke, Thielemans, Ehrhardt, "Accelerated Convergent Motion
 * Compensated Image Reconstruction", arXiv 2410.10503.
 *
 * Model (Sec. II-A): N gates with data d_i = A_i x + eps_i, A_i = A D_i,
 * solved as  min_x  O(x) = alpha ||x||^2 + sum_i N^-1 ||A_i x - d_i||^2
 * by SPDHG (Algorithm 1, one gate drawn per iteration with p_i = 1/N) or by
 * PDHG (p_i = 1, all gates every iteration).  One epoch = N SPDHG iterations
 * = one PDHG iteration = N forward and N adjoint operator applications.
 *
 * Conventions shared by every entry point
 *  - Images are n x n float32, row-major [r*n + c].  Pixel (r, c) has centre
 *    (x, y) = (c - h, r - h), h = (n-1)/2, unit spacing.
 *  - Sinograms are n_angles x n_bins float32, row-major [k*n_bins + b].
 *    Angle k is phi_k = k*pi/n_angles; bin b has centre s_b = b - (n_bins-1)/2;
 *    ray (k, b) is the line {p : p . (cos phi_k, sin phi_k) = s_b}.
 *  - A is Joseph's ray-driven projector: rays with n_a <= 4k <= 3 n_a are
 *    sampled once per image column (step 1/|sin phi|), the others once per row
 *    (step 1/|cos phi|), linear interpolation, zero outside the image.
 *  - D_i is a bilinear pull-back warp, (D_i x)(p) = x(q_i(p)), zero outside;
 *    rigid: q = R(phi_i) p + t_i about the image centre; dense: q = p + u_i(p).
 *  - Gate indices are 0-based.
 *  - Array pointers may be HOST or DEVICE memory (detected per call); device
 *    arrays must belong to the context's device.  Arrays are contiguous and
 *    caller-owned; the library never keeps or frees them.  Host arrays are
 *    staged through the context's own device buffers; such calls return after
 *    the results have reached host memory.  Calls with device arrays are
 *    ordered on the context's stream and may return before the GPU finishes.
 *  - Every entry point validates its arguments on the host before any launch
 *    and returns a status; nothing throws or aborts across the ABI.  The
 *    message of the last failure is kept per context (mc_last_error).
 *  - A context is not thread-safe: one host thread at a time.
 */
#ifndef MC_H
#define MC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mc_ctx mc_ctx;

typedef enum {
    MC_OK = 0,
    MC_EINVAL = -1,    /* bad argument (null, out of range, wrong device ...) */
    MC_ENOMEM = -2,    /* device or pinned host allocation failed            */
    MC_ECUDA = -3,     /* a CUDA runtime call or kernel launch failed         */
    MC_ETIMEOUT = -4,  /* a bounded device-side wait ran out (error word set) */
    MC_ESTATE = -5,    /* call out of order (e.g. run before mc_set_data)     */
    MC_EDEVICE = -6    /* no usable CUDA device / wrong architecture          */
} mc_status;

typedef struct {
    int32_t n;         /* image side, 2 <= n <= 2048                           */
    int32_t n_angles;  /* angles over [0, pi), 1 <= n_angles <= 8192           */
    int32_t n_bins;    /* detector bins at unit spacing, 1 <= n_bins <= 8192   */
} mc_geometry;

enum { MC_MOTION_RIGID = 0, MC_MOTION_FIELD = 1 };

typedef struct {
    int32_t kind;          /* MC_MOTION_RIGID or MC_MOTION_FIELD               */
    const double* rigid;   /* RIGID: N x 3 {phi (rad), tx, ty (px)}, host;
                              q = R(phi) p + (tx, ty), R(phi) = [[c,-s],[s,c]] */
    const float* field;    /* FIELD: N x 2 x n x n {ux (column), uy (row)} in px,
                              host or device; q = p + u(p)                     */
} mc_motion;

/* Serial sampling of one gate per SPDHG iteration, P(i) = p_i (Algorithm 1
 * step (ii), Sec. II-A).  p == NULL: uniform, p_i = 1/N, gate =
 * floor(word0 N / 2^32).  Otherwise p (HOST, N doubles, each finite and > 0)
 * is normalised to sum 1 and the gate is the first i with
 * word0 < floor(2^32 (p_0 + ... + p_i)) (the running sum taken in gate order;
 * the last threshold is 2^32), word0 the first Philox4x32-10 output word of
 * the iteration's counter.  Step (iii) then weights the increment by theta/p_i,
 * and the step sizes follow the uniform rule (mc_get_steps) with n = 1/min_i p_i
 * in place of N, so that omega tau sigma ||A_i||^2 = min_j p_j <= p_i for every
 * gate (reduces to the uniform steps at p_i = 1/N).  Non-uniform p is defined
 * over gates only: with angle subsets (mc_set_subsets, S > 1) p must be NULL. */
typedef struct {
    uint64_t seed;         /* Philox4x32-10 key                                */
    uint32_t stream;       /* counter word 1; lets runs share a seed           */
    const double* p;       /* NULL (uniform) or N sampling probabilities, host */
} mc_sampling;

/* Options for mc_set_option. */
enum {
    MC_OPT_GRAPH = 1,            /* 1 (default): replay each epoch as a CUDA graph */
    MC_OPT_PROFILE = 2,          /* 1: time every launch with CUDA events (slower)  */
    MC_OPT_TRACE_OBJECTIVE = 3,  /* 1: trace also evaluates O(x) (N extra A_i x)    */
    MC_OPT_STORAGE = 4,          /* storage type of the data d and the dual y read and
                                    written by every iteration: MC_STORE_F32 (default),
                                    MC_STORE_F16 (IEEE binary16) or MC_STORE_BF16
                                    (bfloat16); arithmetic stays float32.  d is rounded
                                    once, each new y_i is rounded (to nearest even) when
                                    stored and y_i^{k+1} - y_i^k is taken from the stored
                                    values, so z = sum_i A_i^* y_i holds.  The iterates
                                    then settle near x* of the rounded data, within
                                    ||d_h - d|| / (2 sqrt(alpha N)) of x*: at 512^2
                                    (rbf512, alpha = 1e-3) 100 epochs ended 4.8e-5 (f16)
                                    and 3.9e-4 (bf16) from x* against 7.3e-6 in float32;
                                    small problems have higher floors (bf16 at 16^2:
                                    2e-3).  The float32 d
                                    is kept for mc_objective, mc_set_reference and
                                    mc_solve_normal.  Switching converts the current y. */
    MC_OPT_TEST_STALL = 5,       /* 1: for testing the failure path of the bounded
                                    device-side waits.  The next forward projection
                                    this context launches (runs then launch epochs
                                    directly instead of replaying a graph) gets a
                                    TMA producer that issues no copies and consumer
                                    waits limited to 2^12 polls: the waits run out,
                                    the consumers leave without touching y, the
                                    device error word is set (so a run reports
                                    MC_ETIMEOUT) and nothing is left in flight, so
                                    the context stays usable.  Cleared by that
                                    launch; 0 clears it before. */
    MC_OPT_SUBSET_BANDS = 6,     /* line bands of the angle-subset forward (0, default:
                                    min(8, max(1, S / 2)); 1..8): each subset launch's
                                    work items stream one band of the image's lines
                                    and a combine adds the bands' partial ray sums in
                                    band order.  With S > 1 the subset tables are
                                    rebuilt at once (norms and step sizes kept);
                                    results change within float32 rounding (the
                                    order of the ray sums).  mc_autotune picks it
                                    when S > 1. */
    MC_OPT_SUBSET_ROWS = 7,      /* rows per thread of the angle-subset backprojection
                                    tiles (0, default: those of the all-angle launches;
                                    4, 8, 14, 16 or 28); results change within float32
                                    rounding. */
    MC_OPT_FORWARD_LINES = 8,    /* lines per staged chunk of the forward projector
                                    (2, 4, 8 or 16): its ring, in the shared memory a
                                    block may use, holds 5 chunks, or 3 for 16-line
                                    chunks and for 8-line chunks of large images, and
                                    must fit (16-line chunks: images up to 528^2;
                                    MC_EINVAL otherwise); 16 also needs the image side
                                    rounded up to 8 to be a multiple of 16.  The
                                    forward's work items are cut again for it
                                    (mc_autotune also tries every size).  Results
                                    change within float32 rounding. */
    MC_OPT_BACKPROJECT_ROWS = 9  /* rows per thread of the backprojection tiles (4, 8,
                                    14, 16: four blocks of 8 warps per SM; 28: two),
                                    overriding the creation-time choice (the grid
                                    that fills whole waves at the least work per
                                    SM) or mc_autotune's.  Results change within
                                    float32 rounding. */
};

enum { MC_STORE_F32 = 0, MC_STORE_F16 = 1, MC_STORE_BF16 = 2 };

/* Create a context on the current CUDA device (Sec. II-A: geometry of A,
 * N gates, motion of D_i).  Builds the angle tables, uploads the motion and
 * builds each gate's transpose warp D_i^T as a CSR matrix (rows = source
 * pixels, entries sorted by destination pixel, bilinear weights identical to
 * those of D_i).  cuda_stream: a cudaStream_t to order all work on, or NULL
 * for a stream the context creates.  On success *out owns all device memory
 * of the context; release it with mc_destroy.  Errors: MC_EINVAL,
 * MC_ENOMEM, MC_ECUDA, MC_EDEVICE (message: mc_last_error(NULL)); a failed
 * create frees everything it allocated.  Fault injection for tests: with
 * the environment variable MC_FAIL_ALLOC_AFTER=k set at creation, the
 * context's (k+1)-th device allocation fails with MC_ENOMEM (at creation or
 * in a later call that allocates). */
mc_status mc_create(const mc_geometry* geom, int32_t n_gates, const mc_motion* motion,
                    void* cuda_stream, mc_ctx** out);

/* Free everything the context owns.  NULL is a no-op. */
void mc_destroy(mc_ctx* ctx);

/* Message of the last failed call on ctx (or of the last failed mc_create
 * when ctx is NULL); "" if none.  Valid until the next call on ctx. */
const char* mc_last_error(const mc_ctx* ctx);

/* Set the gated data d (N x n_angles x n_bins, copied) and alpha > 0 of
 * g(x) = alpha ||x||^2 (Sec. II-A).  Resets the solver state. */
mc_status mc_set_data(mc_ctx* ctx, const float* d, double alpha);

/* Double-buffered upload for callers that reconstruct one data set after
 * another (the gated data d of Sec. II-A).  mc_stage_data starts copying the
 * next d (N x n_angles x n_bins float32, HOST memory; pinned memory makes the
 * copy asynchronous) into a staging buffer of the context, on a copy stream
 * of the context's own, and returns without waiting: the upload overlaps
 * whatever the context runs meanwhile.  d must stay valid and unchanged until
 * the copy has landed, at the latest when mc_commit_data returns.  A second
 * mc_stage_data before the commit replaces the staged data.  The staging
 * buffer (one d) is allocated on the first call.  Errors: MC_EINVAL (NULL or
 * device d), MC_ENOMEM, MC_ECUDA.
 * mc_commit_data then makes the staged data current exactly as
 * mc_set_data(ctx, d, alpha) does (same solver-state reset, step sizes and
 * storage conversion): the context's stream waits for the upload and copies
 * it into place on the device; the call returns when that is done.  MC_ESTATE
 * when nothing is staged. */
mc_status mc_stage_data(mc_ctx* ctx, const float* d);
mc_status mc_commit_data(mc_ctx* ctx, double alpha);

/* out = A_i x = A D_i x (Sec. II-A).  x: n x n; out: n_angles x n_bins. */
mc_status mc_forward(mc_ctx* ctx, int32_t gate, const float* x, float* out);

/* out = A_i^* y = D_i^T A^T y, the exact transpose of mc_forward (the
 * operator SPDHG applies in step (iii) of Algorithm 1).  A^T is a pixel-
 * driven gather with the same interpolation weights as A; D_i^T gathers
 * through the gate's CSR.  y: n_angles x n_bins; out: n x n. */
mc_status mc_adjoint(mc_ctx* ctx, int32_t gate, const float* y, float* out);

/* out = A x (no motion) and out = A^T y: the ray transform alone. */
mc_status mc_project(mc_ctx* ctx, const float* x, float* out);
mc_status mc_backproject(mc_ctx* ctx, const float* y, float* out);

/* out = D_i x and out = D_i^T v: the warp of gate i alone. */
mc_status mc_warp(mc_ctx* ctx, int32_t gate, const float* x, float* out);
mc_status mc_warp_adjoint(mc_ctx* ctx, int32_t gate, const float* v, float* out);

/* Tune the launch shapes of the two projectors for this context's geometry
 * by timing them on the device (each candidate `reps` launches after one
 * warm-up, CUDA events on the context's stream): the forward's lines per
 * staged chunk (2, 4, 8, 16, as the layouts and shared memory allow), work
 * items per block and ray-group slots per warp, and the backprojector's rows
 * per thread (4, 8, 14, 16, 28).  The fastest setting is kept; results are
 * unchanged bit for bit by the item split and change within float32 rounding
 * with the chunk size and rows per thread.  out (nullable, host, 4 int32):
 * {lines per chunk, items per block, group slots per warp, rows per thread}.
 * Captured epoch graphs are dropped.  The creation-time choice is a
 * heuristic (the longest chunk whose ring fits, fewest items, and the tile
 * height whose grid fills every SM's resident blocks with the least work on
 * the busiest SM).  With angle
 * subsets (mc_set_subsets, S > 1) it also picks the subset forward's line
 * bands (MC_OPT_SUBSET_BANDS: 1, 2, 3, 4, 6 or 8, timed on the S blocks of
 * gate 0) and leaves the option at that value; norms, step sizes and
 * iterates are kept. */
mc_status mc_autotune(mc_ctx* ctx, int32_t reps, int32_t* out);

/* Sample gates and angle subsets together (the extension named in Sec. IV):
 * split the angles into `subsets` = S interleaved subsets (subset s holds
 * the angles k = s, s + S, s + 2S, ...; 1 <= S <= n_angles, S = 1 restores
 * gate sampling).  SPDHG then works on the N S blocks j = i S + s with
 * A_j = R_s A D_i (R_s keeps the rows of subset s) and data terms
 * N^-1 ||A_j x - d_{i,s}||^2, so the objective O is unchanged; each iteration
 * draws one block uniformly (p_j = 1/(N S), Philox as in mc_spdhg_run with
 * i replaced by j in [0, N S)) and an epoch is N S iterations, the same
 * operator work as N gate iterations.  After this call: mc_norms and
 * mc_set_norms use N S + 1 values {||A_0||^2 .. ||A_{N S - 1}||^2, stacked
 * norm}, SPDHG step sizes take kappa = max_j ||A_j||^2/(alpha N) and n = N S,
 * and mc_draw_gates returns block indices.  The norms and step sizes are
 * dropped (call mc_norms or mc_set_norms again); iterates are kept.  PDHG,
 * the operators (mc_forward ...) and mc_objective are unaffected. */
mc_status mc_set_subsets(mc_ctx* ctx, int32_t subsets);

/* Replace the dense displacement field of one gate (Sec. II-A: D_i is the
 * pull-back warp by u_i).  field: 2 x n x n {ux (column), uy (row)} in px,
 * host or device, copied; values must be finite with |u| <= 1e5.  Rebuilds
 * that gate's D_i^T CSR in place, without allocating (every gate owns a
 * fixed slice of 4 n^2 entries, the most its taps can need).  A_i changes,
 * so the squared norms, the step sizes and x* are dropped: call mc_norms or
 * mc_set_norms (and mc_set_reference) again before the next run.  The
 * iterates are kept (a warm start).  MC_ESTATE for rigid-motion contexts. */
mc_status mc_set_field(mc_ctx* ctx, int32_t gate, const float* field);

/* Vector-Jacobian product of (x, u_i) -> A D_{u_i} x at cotangent r
 * (n_angles x n_bins): with b = A^T r,
 *   grad_x     = D_i^T b = A_i^* r                      (n x n),
 *   grad_field = b(p) * d x(q)/dq at q = p + u_i(p)     (2 x n x n, {ux, uy}),
 * the second being the derivative of the bilinear sample inside the cell
 * that floor(q) selects (zero-padded like D_i).  The data term
 * N^-1 ||A_i x - d_i||^2 of Sec. II-A has gradient mc_vjp at
 * r = (2/N)(A_i x - d_i).  Either output may be NULL (not both); grad_field
 * needs a dense-field context (MC_ESTATE otherwise) and x, the image the
 * forward map was applied to.  One backprojection serves both outputs. */
mc_status mc_vjp(mc_ctx* ctx, int32_t gate, const float* x, const float* r, float* grad_x,
                 float* grad_field);

/* Power iteration (Theorem, Sec. II-B) with float32 operators and float64
 * reductions.  out (host or device, N+1 doubles): ||A_0||^2 .. ||A_{N-1}||^2,
 * then ||(A_0; ...; A_{N-1})||^2 = lambda_max(sum_i A_i^T A_i).  Stops per
 * norm after max_iter iterations or when the Rayleigh quotient changes by
 * less than tol (relative).  The result also sets the step sizes.  After
 * mc_set_subsets(S > 1) the first N S values are the block norms ||A_j||^2,
 * j = i S + s, and out holds N S + 1 doubles. */
mc_status mc_norms(mc_ctx* ctx, int32_t max_iter, double tol, double* out);

/* Use these squared norms (same layout as mc_norms: N+1 doubles, or N S + 1
 * with angle subsets) for the step sizes instead of running mc_norms. */
mc_status mc_set_norms(mc_ctx* ctx, const double* norms2);

/* Step sizes in use (host out, 5 doubles): {sigma, tau, theta, kappa, omega}
 * for SPDHG (pdhg = 0) or PDHG (pdhg = 1).  With mu_g = 2 alpha, mu_f = N/2,
 * kappa = ||A||^2/(mu_g mu_f) (||A||^2 = max_i ||A_i||^2 for SPDHG, the stacked
 * norm for PDHG), s = sqrt(1 + kappa), n = N (SPDHG) or 1 (PDHG):
 * omega = 1 - 2/(n (1 + s)), sigma_i = 1/(mu_f (s - 1)),
 * tau = (1 - omega)/(2 mu_g omega), theta = omega, so that the per-epoch rate
 * is omega^n = l(kappa, n) of Sec. II-B.  After an SPDHG run (or batch run)
 * with non-uniform sampling p, the SPDHG steps use n = 1/min_i p_i (see
 * mc_sampling) until a run with another p.  MC_ESTATE before norms and data. */
mc_status mc_get_steps(mc_ctx* ctx, int32_t pdhg, double* out);

/* Reference solution x* (n x n) for the trace; y_i* = (2/N)(A_i x* - d_i)
 * is derived from it.  Call after mc_set_data.  NULL clears it. */
mc_status mc_set_reference(mc_ctx* ctx, const float* x_star);

/* Reference solution by conjugate gradients on the optimality condition of
 * O (Sec. II-A): (alpha I + N^-1 sum_i A_i^T A_i) x = N^-1 sum_i A_i^T d_i, with
 * float32 operators (all gates per iteration) and float64 inner products.
 * Stops after max_iter iterations or once ||r|| <= tol ||b|| (checked every
 * 10 iterations).  x_out (n x n, host or device) receives x; info (nullable,
 * host, 2 doubles) receives {iterations, ||r||/||b||}.  Needs mc_set_data. */
mc_status mc_solve_normal(mc_ctx* ctx, int32_t max_iter, double tol, float* x_out, double* info);

/* Zero the solver state (x = z = zbar = 0, y = 0) and the iteration count. */
mc_status mc_reset(mc_ctx* ctx);

/* Run `epochs` epochs (N iterations each) of SPDHG, Algorithm 1, continuing
 * from the current state:
 *   (i)   x^{k+1} = prox_{tau g}(x^k - tau zbar^k) = (x^k - tau zbar^k)/(1 + 2 tau alpha)
 *   (ii)  draw i (Philox4x32-10 on the device, key = seed, counter =
 *         (k mod 2^32, stream, k >> 32, 0), i = floor(word0 * N / 2^32), or by
 *         the thresholds of sampling->p, see mc_sampling);
 *         y_i^{k+1} = prox_{sigma f_i^*}(y_i^k + sigma A_i x^{k+1})
 *                   = (y_i^k + sigma (A_i x^{k+1} - d_i)) / (1 + sigma N/2)
 *   (iii) z^{k+1} = z^k + A_i^* (y_i^{k+1} - y_i^k),
 *         zbar^{k+1} = z^{k+1} + (theta / p_i) A_i^* (y_i^{k+1} - y_i^k).
 * (Algorithm 1 as printed uses z^k in step (i) and accumulates zbar on
 * zbar^k; this is read as the standard SPDHG above.)
 * x_out (nullable, n x n): x^K after the K-th iteration of this context.
 * trace (nullable, epochs x 3 doubles): per epoch
 * {||x - x*||/||x*||, ||x - x*||^2 + sum_i ||y_i - y_i*||^2, O(x)}; NaN where the
 * reference is unset or MC_OPT_TRACE_OBJECTIVE is off.
 * With a host x_out or trace the call returns after they have reached host
 * memory and reports a device-side failure of the run (MC_ETIMEOUT).  With
 * device (or no) outputs it returns without waiting: the run's error word is
 * then checked by a later mc_spdhg_run / mc_pdhg_run (as soon as the run has
 * finished) or by mc_sync.
 * MC_ESTATE if data or step sizes are missing. */
mc_status mc_spdhg_run(mc_ctx* ctx, int32_t epochs, const mc_sampling* sampling,
                       float* x_out, double* trace);

/* Many independent slices (one context each, e.g. different sizes, gate
 * counts and motion kinds), without a batch object: run `epochs` SPDHG epochs
 * on every context, enqueuing epoch e of every slice (its own epoch graph)
 * before epoch e + 1 of any, each on its own context stream, so small slices'
 * launches overlap with large ones (mc_batch_run instead merges the slices'
 * launches).
 * Per context the result equals `epochs` calls of mc_spdhg_run with
 * sampling[i] (same gate draws, same iterates).  sampling: count entries.
 * All contexts must live on one device and have data and step sizes.
 * Returns after every slice has finished (its error word checked); on
 * failure *failed (nullable) receives the index of the context whose
 * mc_last_error holds the message. */
mc_status mc_batch_spdhg_run(mc_ctx* const* ctxs, int32_t count, int32_t epochs,
                             const mc_sampling* sampling, int32_t* failed);

/* Batched SPDHG over many independent slices in ONE launch per stage.
 *
 * SPDHG's cost per iteration does not grow with N (Sec. II-A), so a slice's
 * iteration is a few small launches; slices of uneven sizes and gate counts
 * (each its own context: geometry, gates, motion kind) are therefore advanced
 * together.  One batched iteration runs one SPDHG iteration (Algorithm 1) of
 * every slice still in flight as four stages, each ONE launch over the blocks
 * of all those slices: the warp D_i, the Joseph forward with the fused dual
 * update, the backprojection and the transpose warp with the fused
 * z / zbar / prox update, whose first block per slice also advances that
 * slice's position in its epoch and, at an epoch's end, draws the next
 * epoch's gates (Philox counter on the device, the one-slice draw's
 * sequence): four stages per batched iteration whatever the slices' launch
 * shapes (the forward is one launch per class of slices that share a chunk
 * size and ring, the classes run concurrently between a fork and a join; the
 * backprojection's blocks run with their slice's rows per thread, an instance
 * compiled for one height when all slices in flight share it).  Block lists
 * put the slices with the most work per block first.  Each batched iteration
 * is captured once as a CUDA graph per set of slices in flight and parity of
 * the iteration index, and replayed.
 *
 * mc_batch_create groups `count` contexts (same device, angle subsets = 1),
 * orders work on cuda_stream (NULL: a stream of the batch's own) and keeps
 * pointers to the contexts: destroy the batch before any of them.  It also
 * cuts each slice's forward work into its own coarser items where the
 * slice's share of a merged launch is small (a block then streams the
 * slice's image once for more ray groups); these serve while the slices in
 * flight give every SM at least four such blocks, the slices' own items
 * otherwise (results do not depend on the cut).  After a call that rebuilds
 * a slice's forward tables or sets its launch shapes (mc_autotune,
 * MC_OPT_FORWARD_LINES, MC_OPT_BACKPROJECT_ROWS), even to the values it had,
 * mc_batch_run returns MC_ESTATE: create the batch again.  Slices with angle
 * subsets (mc_set_subsets, S > 1) are refused too.
 * mc_batch_run runs `epochs` SPDHG epochs of every slice (slice i: epochs x
 * N_i iterations, sampling[i] as in mc_spdhg_run, p included); slices with
 * fewer gates finish first and leave the launches.  Per slice the result is
 * bit-identical to mc_spdhg_run(ctx_i, epochs, &sampling[i], ...) from the
 * same state (same draws, same arithmetic), and the contexts' iterates,
 * iteration counters and duals continue from there.  The call waits for each
 * context's pending work first and returns when the batch has finished (every
 * slice's error word checked).  On failure *failed (nullable) is the slice
 * index, mc_batch_last_error(b) holds the message.  Errors: MC_EINVAL,
 * MC_ESTATE (a slice without data or step sizes), MC_ENOMEM, MC_ECUDA,
 * MC_ETIMEOUT. */
typedef struct mc_batch mc_batch;
mc_status mc_batch_create(mc_ctx* const* ctxs, int32_t count, void* cuda_stream, mc_batch** out);
mc_status mc_batch_run(mc_batch* b, int32_t epochs, const mc_sampling* sampling, int32_t* failed);
const char* mc_batch_last_error(const mc_batch* b);
void mc_batch_destroy(mc_batch* b);

/* Run `epochs` iterations of PDHG (p_i = 1, every gate each iteration,
 * zbar^{k+1} = z^{k+1} + theta sum_i A_i^*(y_i^{k+1} - y_i^k)), continuing from
 * the current state.  Arguments as for mc_spdhg_run. */
mc_status mc_pdhg_run(mc_ctx* ctx, int32_t epochs, float* x_out, double* trace);

/* The device gate draw alone: out[j] = gate of iteration k0 + j (int32,
 * host or device, count >= 0).  Does not touch the solver state. */
mc_status mc_draw_gates(mc_ctx* ctx, const mc_sampling* sampling, uint64_t k0,
                        int32_t count, int32_t* out);

/* O(x) = alpha ||x||^2 + sum_i N^-1 ||A_i x - d_i||^2 in float64 (Sec. II-A). */
mc_status mc_objective(mc_ctx* ctx, const float* x, double* out);

/* Set an MC_OPT_* option. */
mc_status mc_set_option(mc_ctx* ctx, int32_t option, int64_t value);

/* With MC_OPT_PROFILE on: per kernel class, launches and summed device time
 * (ms) since the last mc_profile_reset.  names/counts/ms are host arrays of
 * capacity `cap`; *n_out receives the number of classes.  Classes: "warp",
 * "project", "backproject", "warp_adjoint_update", "gate_draw", "misc". */
mc_status mc_profile_read(mc_ctx* ctx, int32_t cap, const char** names, int64_t* counts,
                          double* ms, int32_t* n_out);
mc_status mc_profile_reset(mc_ctx* ctx);

/* Iteration counter k of the next SPDHG iteration (host out). */
mc_status mc_iteration(mc_ctx* ctx, uint64_t* out);

/* Wait for all work of the context and report a device-side failure of a
 * run that returned without waiting (MC_ETIMEOUT, MC_EDEVICE), or MC_OK. */
mc_status mc_sync(mc_ctx* ctx);

/* Checkpoint and resume of the solver state (x^K, x^{K+1}, z, every y_i in
 * the current storage type, and the iteration counter k that keys the
 * Philox draw).  mc_state_size gives the bytes; mc_save_state writes them to
 * a HOST buffer of capacity cap; mc_load_state restores them into a context
 * with the same geometry, gate count, storage type (MC_OPT_STORAGE) and
 * angle-subset count, after mc_set_data and the step sizes as at saving.  A
 * run continued from a loaded state with the same sampling seed and stream
 * is bit-identical to the uninterrupted run.  The data, the steps, the
 * motion and the reference are not part of the state.  Errors: MC_EINVAL
 * for a foreign, mismatched or truncated buffer. */
mc_status mc_state_size(mc_ctx* ctx, uint64_t* bytes);
mc_status mc_save_state(mc_ctx* ctx, void* buf, uint64_t cap);
mc_status mc_load_state(mc_ctx* ctx, const void* buf, uint64_t size);

/* Measured rate of conflict-free 64-bit shared-memory loads on the current
 * device (no context needed): the bound of both projectors, which gather
 * 8-byte pairs from shared memory (the roofline of the Joseph A and A^T of
 * Sec. II-A).  Two blocks of 1024 threads per SM stream ld.shared.b64 at
 * consecutive addresses, about reps x 5 GB in total after one warm-up
 * launch, timed by CUDA events on a stream of its own.  out (host, 3 doubles):
 * {bytes per second over the whole GPU, bytes per SM clock, the SM clock in
 * GHz seen by the kernel (clock64 span / event time)}.  Allocates two small
 * scratch buffers and frees them; changes no device setting.  The paper has
 * no counterpart; this is a measurement aid. */
mc_status mc_measure_shared_load_peak(int32_t reps, double* out);

/* Library version string. */
const char* mc_version(void);

/* The launch shapes and layouts mc_create would choose for this geometry on a
 * GPU with `sms` SMs, computed on the host (no device needed; mc_autotune and
 * the MC_OPT_* shape options may change them later).  out (host, 10 int32):
 * {guard: zero pairs around each line of the warped-image layouts (17, or 33
 * where 16-line chunks are sampled whole), line pitch P in pairs (>= n + 2
 * guard), layout lines (n rounded up to 8), forward lines per staged chunk,
 * lines per sampled part of a chunk (each part clamps its positions: the
 * guard must hold 2 x part + 1 pairs), ring stages (5, or 3), backprojection
 * rows per thread, zero bins Gb before each line of the dual increment and
 * its pitch Pb, forward consumer warps per block (15 where 16-line chunks are
 * sampled in two parts, whose state wants up to 128 registers a thread; 23
 * otherwise), each block one more warp for the copies}.  The paper has no
 * counterpart: these are this library's own layouts (Sec. II-A defines only
 * the operators).  MC_EINVAL for a geometry mc_create refuses. */
mc_status mc_plan_shapes(const mc_geometry* geom, int32_t sms, int32_t* out);

/* The launch shapes and layouts the context uses now, in mc_plan_shapes'
 * order (host, 10 int32): at creation they equal mc_plan_shapes for the
 * context's geometry and device; MC_OPT_FORWARD_LINES,
 * MC_OPT_BACKPROJECT_ROWS and mc_autotune change the chunk lines (with the
 * part lines, ring stages and consumer warps that follow from them) and the
 * rows per thread.  The subset launches' own options (MC_OPT_SUBSET_*) are not
 * reported.  Reads host state only.  MC_EINVAL for a NULL argument. */
mc_status mc_get_shapes(const mc_ctx* ctx, int32_t* out);

/* Allocation-free forward operator, for callers that must not allocate
 * device memory (code running inside an allocator hook, a plugin with a
 * fixed memory budget, or a host whose GPU memory is already owned by its
 * own pool).  The paper has no counterpart: this is a deployment variant of
 * mc_forward for a single motion state, with no context.
 *   out = A D x, where D is the rigid map rigid = {phi, tx, ty} (as in
 *   mc_motion) or the identity when rigid is NULL; geometry as mc_create.
 *   x (n x n) and out (n_angles x n_bins) are DEVICE arrays of the current
 *   device, owned by the caller; host arrays are rejected (MC_EINVAL).
 * All scratch (tables, the warped image's line layouts, an error word) lives
 * in one fixed 24 MiB device array built into the library, which every device
 * that loads the library holds until the process exits; the call makes no
 * cudaMalloc, cudaFree or other allocation.  Sizes whose scratch exceeds the
 * array (about n > 1220 at 720 angles) return MC_EINVAL.  The first call on
 * each device sets up (looks up the array's device address, sets kernel
 * attributes); make that first call before any stream capture (a first call
 * inside a capture returns MC_ESTATE).  Every later call made outside a
 * capture looks the address up again, so a device reset by the host
 * application leaves no stale pointer.  Every call shares the array: calls
 * that overlap on the GPU (different streams, or different host threads)
 * race and must be serialised by the caller.  Work
 * is ordered on cuda_stream (NULL = legacy default stream) and the call
 * returns before it completes.  err (nullable, err_cap bytes) receives a
 * message when the call itself fails (arguments, sizes, launches).  A
 * failure on the device while the work runs (a bounded wait that ran out) is
 * not known when the call returns: it is recorded in the array's error word
 * and reported by mc_forward_static_status.  Test hook: with the environment
 * variable MC_STATIC_TEST_STALL=1 (read at every call) the projection's TMA
 * producer issues no copies and its consumers' waits run out after 2^12
 * polls, leaving nothing in flight, so that the failure report can be tested. */
mc_status mc_forward_static(const mc_geometry* geom, const double* rigid, const float* x,
                            float* out, void* cuda_stream, char* err, int32_t err_cap);

/* Outcome on the device of the last mc_forward_static call on the current
 * device: waits for cuda_stream (the stream that call used, or one ordered
 * after it; not while it is being captured), reads the 4-byte error word of
 * the fixed array, and returns MC_OK, MC_ETIMEOUT (a bounded wait of the
 * projection ran out: out is incomplete) or MC_EDEVICE (a bounds check of a
 * checked build fired).  The word is cleared by the next mc_forward_static
 * call, not by this one.  Allocates nothing.  MC_ESTATE before the first
 * mc_forward_static call on the device; err as in mc_forward_static.  The
 * paper has no counterpart; this belongs to the allocation-free entry point. */
mc_status mc_forward_static_status(void* cuda_stream, char* err, int32_t err_cap);

#ifdef __cplusplus
}
#endif
#endif /* MC_H */
