/*
 * hc.h -- C ABI of the GB300 (sm_103a) implementation of one time step of the
 * Fourier spectral FFT+CG splitting scheme for the periodic Hu-Cai
 * network-formation system
 *
 *     -div((m (x) m + r I) grad p) = S                              (eq. 1.1a)
 *     d_t m - D^2 Lap m - c^2 (m . grad p) grad p + |m|^{2(gamma-1)} m = 0   (eq. 1.1b)
 *
 * of Aceves-Sanchez, Degond, Merino-Aceituno and Wytrzens (arXiv 2606.06720).
 * One step is the loop body of Algorithm 1: the FFT+CG pressure solve of
 * Section 2.4 (eq. p_discrete) from m^k with warm start p^k, then the split
 * m-update of Section 2.3 -- exact activation (eq. m_activation_discrete),
 * exact relaxation (eq. m_relaxation_discrete), exact Fourier diffusion
 * (eq. diffusion_space_discrete).
 *
 * Conventions shared by every entry point
 *   - Grid (Section 2.2): n[a] nodes per axis, periodic end point excluded,
 *     x_i = i L[a] / n[a].  dim = 2: n[0] = nx, n[1] = ny, powers of two in
 *     [8, 4096], n[2] = 1.  dim = 3 (the method's 3D case, Section 2.3):
 *     nx, ny, nz powers of two in [8, 1024], nx*ny*nz <= 2^28.
 *   - Field layout: row-major, x fastest.  A scalar field has npts = nx*ny*nz
 *     doubles (nz = 1 in 2D) at index (k*ny + j)*nx + i.  A vector field (m,
 *     the gradient) is component-major: component c of point q at c*npts + q,
 *     so count = dim*npts.
 *   - Every host pointer is FP64 whatever the internal precision; it is read
 *     or written completely before the call returns (the call waits for its
 *     own copies), so the caller may reuse the buffer right away.
 *   - Every call returns HC_OK (0) or a negative HC_E* code and never throws.
 *     A non-HC_OK return from a setter leaves the context's previous value.
 *   - A context is not thread-safe; calls on one context must not overlap.
 *   - Device work runs on params.stream (a cudaStream_t, NULL = legacy default
 *     stream).  Calls that return data to the host synchronise that stream.
 */
#ifndef HC_H
#define HC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HC_OK 0
#define HC_EINVAL (-1)     /* bad argument: null pointer, size mismatch, unsupported grid, r <= 0 ... */
#define HC_ENOMEM (-2)     /* device allocation failed or the workspace given is too small */
#define HC_ECUDA (-3)      /* a CUDA runtime call failed (the context should be destroyed) */
#define HC_ENOCONV (-4)    /* CG hit its iteration cap; the state was still advanced */
#define HC_ENONFINITE (-5) /* NaN/Inf in p or m, e.g. the activation exponential overflowed (Remark 2.1) */
#define HC_ETIMEOUT (-6)   /* a bounded device-side wait gave up */
#define HC_ENOTSUP (-7)    /* valid request that this build does not implement */
#define HC_EBOUNDS (-8)    /* bounds-checked build: a guard zone after a device buffer was written */

/* Why hc_run stopped (Algorithm 1's loop, Section 2.5). */
#define HC_STOP_NONE 0      /* max_steps reached */
#define HC_STOP_DELTA_M 1   /* Delta m <= eps */
#define HC_STOP_ENERGY 2    /* the discrete energy did not decrease */
#define HC_STOP_STATUS 3    /* a step failed (HC_ENONFINITE) */

/* Arithmetic of the path. */
#define HC_FP64_PLAIN 0   /* every kernel in IEEE FP64 */
#define HC_FP32_REFINED 1 /* FFTs, operator applies and split step in FP32; pressure solve wrapped in
                             FP64 iterative refinement (FP64 residual, FP64 correction accumulation,
                             FP64 dot products and null-space projection) */
#define HC_FP32_REFINED_DF 2 /* as HC_FP32_REFINED, with the refinement's FP64-class arithmetic
                                (residual, correction accumulation, state p and S) carried in
                                double-float pairs on the FP32 pipes: 48-bit significands instead
                                of 53, for GB300's low FP64 issue rate */

typedef struct hc_ctx hc_ctx; /* opaque; owns (or borrows) all device memory of one problem */

/* Supported grids.  2D: each axis 4 .. 4096 nodes with no prime factor above 5.
 * When both axes are powers of two in [8, 4096] the step runs the fused
 * radix-8 kernels in any precision; otherwise (e.g. the paper's N = 50 2^k
 * convergence grids, Section 4) it runs mixed-radix FP64 kernels, in
 * HC_FP64_PLAIN only (other precisions: HC_ENOTSUP), without the adjoint,
 * tuning or kernel timing (HC_ENOTSUP).  3D: each axis a power of two in
 * [8, 1024], at most 2^28 points. */
typedef struct {
  int dim;      /* 2 or 3 */
  int n[3];     /* nodes per axis (x, y, z) */
  double L[3];  /* domain lengths, > 0 */
} hc_grid;

typedef struct {
  double c, D, gamma, dt; /* activation c, diffusion D, metabolic exponent gamma, time step (Algorithm 1 inputs) */
  double cg_rtol;         /* stop when ||S - A p||_2 <= cg_rtol ||S||_2, S projected (Section 2.4; default 1e-7 if <= 0) */
  int cg_maxit;           /* CG iteration cap per solve; in refined mode per inner FP32 solve (default 1000 if <= 0) */
  int precision;          /* HC_FP64_PLAIN or HC_FP32_REFINED */
  double kappa;           /* > 0: preconditioner kappa (-Laplacian); <= 0: chosen by precond,
                             recomputed every step (the conclusion's constant-coefficient
                             preconditioner, reading R3) */
  double inner_rtol;      /* refined mode: inner FP32 CG stops at this reduction of its own residual (default 1e-4 if <= 0) */
  int max_sweeps;         /* refined mode: cap on FP64 refinement sweeps per solve (default 10 if <= 0) */
  int use_graph;          /* 1: each step runs as one CUDA graph with device-side loop control; 0: host loop */
  void* stream;           /* cudaStream_t the context launches on */
  int diagnostics;        /* 1: every step also computes the energy and Delta m of Section 2.5 (see hc_step_stats) */
  int fp64_first_residual; /* refined modes.  0 (default): when the warm start is off by more than
                              1e-5 ||S||, the first refinement sweep solves for S - A p^k evaluated
                              in FP32 (a low-precision first solve, as mixed-precision iterative
                              refinement starts); the FP64 residual after it removes that
                              evaluation's error.  1: every sweep starts from an FP64 residual.
                              Either way every convergence test uses an FP64 residual. */
  int fp64_mid_residual;   /* HC_FP32_REFINED.  0 (default): the residual that follows an FP32 first
                              sweep (it only supplies the second inner solve's right-hand side) is
                              evaluated in double-float on the FP32 pipes, with p += delta still
                              accumulated in FP64; the refinement loop after it is decided by FP64
                              residuals.  1: that residual is FP64 too. */
  int precond;             /* with kappa <= 0: HC_PRECOND_SCALAR (0, default) kappa (-Laplacian) with
                              kappa = mean(r) + mean(|m|^2)/dim; HC_PRECOND_KBAR (1) -div(Kbar grad)
                              with Kbar = mean(m m^T) + mean(r) I, the whole mean of the coefficient
                              tensor (fewer CG iterations when m is anisotropic on average) */
  int sync_cert;           /* 2D HC_FP32_REFINED steps in graph mode with diagnostics off.
                              0 (default): lagged certification.  A step's FP32 inner solves end
                              with the double-float residual's solve; the FP64 residual that
                              certifies its pressure (||S - A p|| <= cg_rtol ||S||, as always) runs
                              beside the next step's solve, on the spare FP64 pipes, and the last
                              step's after the loop.  If a certification fails (rare), hc_step
                              goes back to that step's start, redoes it with the refinement loop
                              and runs the call's remaining steps certifying each before the
                              next, so every step hc_step returns is certified.
                              When every certification passes, the results are bit-identical to
                              sync_cert = 1.  1: each step certifies (and, if needed, refines)
                              before the next one starts. */
} hc_params;

enum { HC_PRECOND_SCALAR = 0, HC_PRECOND_KBAR = 1 };

typedef struct {
  int cg_iters;        /* CG iterations of the last step's pressure solve (summed over sweeps) */
  int refine_sweeps;   /* refined mode: inner solves run; plain mode: 0 */
  double rel_residual; /* ||S - A p||_2 / ||S||_2 at exit: FP64-evaluated in refined mode, recursive in plain mode */
  double kappa;        /* trace(Kbar) / dim of the preconditioner used (the isotropic part) */
  int status;          /* HC_OK, HC_ENOCONV or HC_ENONFINITE for that step */
  long long total_cg_iters; /* CG iterations summed over all steps of the hc_step call */
  long long total_sweeps;   /* refinement sweeps summed likewise */
  /* With params.diagnostics (Section 2.5; discrete L2 norms with the cell volume as weight):
   *   energy  = E_h(m) for the m the step started from, with that m's own pressure (the p the
   *             step solved): D^2/2 ||grad m||^2 + c^2/2 ||r^(1/2) grad p||^2
   *             + c^2/2 ||m . grad p||^2 + 1/(2 gamma) || |m|^gamma ||^2, gradients by the
   *             spectral derivative of the scheme.  At gamma = 0 the last term is
   *             sum h ln|m|, its gradient-flow limit (the gamma = 0 relaxation term of
   *             eq. 1.1b is the m-gradient of ln|m|), and -inf when some |m| = 0; the
   *             energy rule then stops a run, as -inf < -inf is false;
   *   delta_m = ||m_new - m_old||_2 / (dt ||m_old||_2) of the step. */
  double energy;
  double delta_m;
  int energy_valid;    /* 0 when the energy of the starting m is not known (diagnostics were off when it was made or set) */
  int stop_reason;     /* hc_run: HC_STOP_*; hc_step: HC_STOP_NONE */
  long long energy_step; /* hc_run with HC_STOP_ENERGY: 0-based index, within the call, of the step whose result did not lower the energy; else -1 */
  int first_sweep_fp32;  /* refined modes: the step's first sweep started from the FP32 residual */
  long long total_first_fp32; /* such steps summed over the call */
  int mid_residual_df;   /* HC_FP32_REFINED: the step evaluated the double-float mid-step residual */
  long long total_mid_df;     /* such steps summed over the call */
  int refine_residuals;  /* refined modes: residuals evaluated in the mode's refinement arithmetic
                            (FP64; double-float in HC_FP32_REFINED_DF), the final one included */
  long long total_refine_residuals; /* summed over the call */
} hc_step_stats;

/* Bytes of device workspace hc_create needs for this grid and precision
 * (host arithmetic only, no GPU work).  Errors: HC_EINVAL for an unsupported
 * grid, invalid params or a NULL bytes; HC_ENOTSUP for a mixed-radix grid in a
 * precision other than HC_FP64_PLAIN. */
int hc_workspace_size(const hc_grid* grid, const hc_params* params, size_t* bytes);

/* Create a context.  If workspace is non-NULL it must be a device pointer to at
 * least hc_workspace_size() bytes, 256-byte aligned; the context borrows it
 * (the caller frees it after hc_destroy).  If NULL the context allocates its
 * own with cudaMalloc.  Initial state: r = 1, S = 0, m = 0, p = 0.
 * Errors: HC_EINVAL (grid/params), HC_ENOTSUP (as hc_workspace_size),
 * HC_ENOMEM, HC_ECUDA. */
int hc_create(hc_ctx** out, const hc_grid* grid, const hc_params* params, void* workspace,
              size_t workspace_bytes);

/* Replace the scalar parameters (c, D, gamma, dt, tolerances, kappa, use_graph,
 * diagnostics, precond ...; Algorithm 1 inputs); the grid, precision and stream
 * must match the ones given at creation.  The step graphs are rebuilt at the
 * next step.  Errors: HC_EINVAL (invalid params, or another precision or
 * stream), HC_ECUDA. */
int hc_set_params(hc_ctx* ctx, const hc_params* params);

/* Background permeability r(x) (eq. 1.1a); count = npts; requires r > 0
 * everywhere (the paper assumes r >= r0 > 0) and finite, else HC_EINVAL. */
int hc_set_r(hc_ctx* ctx, const double* r, size_t count);

/* Source/sink field S (eq. 1.1a); count = npts.  Stored after projection onto
 * the complement of the operator's null space (zero mean and no corner modes:
 * the solvability condition that the paper states as int S = 0).
 * Errors: HC_EINVAL (NULL, wrong count, a non-finite value), HC_ECUDA. */
int hc_set_source(hc_ctx* ctx, const double* S, size_t count);

/* Conductivity m (count = dim*npts, component-major; the initial m0 of
 * Algorithm 1).  With params.diagnostics it also computes the gradient norm
 * that the energy of this m needs; without, the first step's energy is
 * unknown (energy_valid = 0) unless hc_run, which computes it, takes the step.
 * The refined modes hold m in FP32.  Errors: HC_EINVAL (NULL, wrong count),
 * HC_ECUDA; non-finite values are not checked here (the next step reports
 * HC_ENONFINITE). */
int hc_set_m(hc_ctx* ctx, const double* m, size_t count);

/* Pressure p used as the CG initial guess of the next step (Section 2.4 uses
 * p^k; default 0).  Projected like S.  Errors: HC_EINVAL (NULL, wrong count),
 * HC_ECUDA. */
int hc_set_p(hc_ctx* ctx, const double* p, size_t count);

/* Run nsteps passes of the loop body of Algorithm 1.  `last` (may be NULL)
 * receives the stats of the final step.  Returns HC_OK, or the first non-OK
 * step status (HC_ENOCONV: the steps still ran; HC_ENONFINITE: stopped). */
int hc_step(hc_ctx* ctx, int nsteps, hc_step_stats* last);

/* Algorithm 1 with its stopping rules (Section 2.5): run loop bodies until
 * Delta m <= eps (eps <= 0: never), or, when stop_on_energy is set, until the
 * discrete energy does not decrease, or until max_steps.  Diagnostics are on
 * for the call whatever params.diagnostics says.  The energy of a state is
 * known once its pressure has been solved, i.e. during the next step, so an
 * energy stop comes one step after the step that raised the energy
 * (reported in last->energy_step).  In graph mode the loop runs as repeated
 * launches of a step graph gated on the device (steps after a stop are
 * skipped on the GPU); the host checks every few launches.
 * *steps_done (may be NULL) gets the number of steps run; `last` the stats of
 * the final step, with stop_reason.  Returns as hc_step. */
int hc_run(hc_ctx* ctx, int max_steps, double eps, int stop_on_energy, int* steps_done,
           hc_step_stats* last);

/* Copy the current p (count = npts) or m (count = dim*npts), the outputs of
 * Algorithm 1, to host memory in the field layout above; the call waits for
 * the copy.  Errors: HC_EINVAL (NULL, wrong count), HC_ECUDA. */
int hc_get_p(hc_ctx* ctx, double* out, size_t count);
int hc_get_m(hc_ctx* ctx, double* out, size_t count);

/* The whole state of Algorithm 1 in one call: m (m_count = dim*npts) and p
 * (p_count = npts), host FP64 in the layouts above, with the effect of
 * hc_set_m followed by hc_set_p (hc_set_state) or of hc_get_m and hc_get_p
 * (hc_get_state), bit for bit; both wait for their copies.  A caller that
 * hands the state over every step moves m and p (3 npts doubles each way)
 * across the host link per step, and p needs an FP64 2D transform each way.
 * In the 2D FP32-refined mode the copy of m runs on a second stream of the
 * context while p is transformed, and p is staged in the FP64 scratch of the
 * step's certification (free between hc_step calls); the other modes call the
 * single-field entry points in turn.  Page-locked host buffers give the full
 * link bandwidth.  Errors: HC_EINVAL (NULL, wrong counts), HC_ECUDA. */
int hc_set_state(hc_ctx* ctx, const double* m, size_t m_count, const double* p, size_t p_count);
int hc_get_state(hc_ctx* ctx, double* m_out, size_t m_count, double* p_out, size_t p_count);

/* --- Component entry points (each runs one part of the step on the GPU) --- */

/* Spectral gradient of the current p (Section 2.4 and Algorithm 1 "compute
 * gradient of p via FFT"): out = (d_x p, d_y p[, d_z p]), count = dim*npts,
 * component-major host memory.  Errors: HC_EINVAL (NULL, wrong count),
 * HC_ECUDA.  The same holds for the component calls below: they run on the
 * context's stream and wait for their own results. */
int hc_gradient(hc_ctx* ctx, double* out, size_t count);

/* Apply the discrete pressure operator of eq. (p_discrete) with the current m
 * and r: out = A f for the field f (count = npts; f is projected first). */
int hc_apply_operator(hc_ctx* ctx, const double* f, double* out, size_t count);

/* Only Step 2 of Algorithm 1 (activation, relaxation, diffusion) with the
 * current p and m; m is updated in place on the device. */
int hc_split_step(hc_ctx* ctx);

/* Forward DFT of a real field (count = npts) in the packed half-spectrum
 * layout: out has nz*ny*(nx/2) complex values (npts doubles, re/im
 * interleaved); entry (kz, ky, kx) for 1 <= kx < nx/2 is F[kz][ky][kx] and
 * entry (kz, ky, 0) is F[kz][ky][0] + i F[kz][ky][nx/2] (kz = 0 in 2D).
 * On a mixed-radix grid: the unpacked half spectrum, ny*(nx/2 + 1) complex
 * values, entry (ky, kx) = F[ky][kx] for kx = 0 .. nx/2. */
int hc_spectrum(hc_ctx* ctx, const double* f, double* out, size_t count);

/* Launch shapes of the FFT passes, per arithmetic precision ([0] FP32
 * kernels, [1] FP64 kernels).  col_tile: packed columns per column-pass CTA
 * (power of two, col_tile*ny/8 <= 1024 threads for [0] and <= 512 for [1],
 * col_tile <= nx/2, <= 32);
 * row_rows: rows per row-pass CTA (power of two, row_rows*nx/8 <= 512,
 * row_rows <= ny), col_pipe (see below).  Results do not depend on them
 * beyond the order of floating-point sums. */
typedef struct {
  int col_tile[2];
  int row_rows[2];
  int col_pipe[2]; /* 1: the CG/residual/heat column passes run persistent, prefetching the next
                      tile with cp.async while transforming the current one; needs
                      col_tile * (8 bytes FP32 | 16 bytes FP64) to be a multiple of 16, or
                      one FP32 column (8-byte copies) */
  int row_pipe[2]; /* [0] = 1: the FP32 operator-apply row pass runs persistent, one CTA per
                      resident slot, prefetching the next row block with cp.async while
                      transforming the current one (needs 48 row_rows nx bytes of shared
                      memory); [1] must be 0 */
} hc_tuning;

int hc_get_tuning(const hc_ctx* ctx, hc_tuning* out);
/* HC_EINVAL if a value breaks the limits above or needs more shared memory
 * than a CTA may have; HC_ENOTSUP on 3D grids (their launch shapes are fixed
 * when the context is created). */
int hc_set_tuning(hc_ctx* ctx, const hc_tuning* in);

/* Kernels of one step, as timed by hc_time_kernel.  The CG_* kernels are the
 * CG iteration (FP32 inner CG in refined mode, FP64 CG in plain mode); RES_*
 * the FP64 residual evaluation (refined: p64 += delta then S - A p64; plain:
 * the initial residual); SPLIT_* Step 2 of Algorithm 1.  On a 3D grid the
 * same ids time the 3D kernels: *_GRAD the z pass with the gradient
 * multipliers, *_APPLY the row-pair pass, *_DIV the z pass with the
 * divergence, *_YPASS the y pass between them, SPLIT_ROW the row pass with
 * activation, relaxation and diffusion along x, SPLIT_HEAT / SPLIT_C2R the
 * diffusion along y / along z. */
enum {
  HC_K_CG_GRAD = 0,    /* column pass: d-update, i xi d / n, inverse FFT_y */
  HC_K_CG_APPLY = 1,   /* row pass: C2R, (m m^T + r I) g, R2C */
  HC_K_CG_DIV = 2,     /* column pass: FFT_y, -i xi . q (alpha comes from the row pass) */
  HC_K_CG_UPDATE = 3,  /* x += alpha d, r -= alpha A d, <r, M^-1 r> */
  HC_K_RES_GRAD = 4,
  HC_K_RES_APPLY = 5,
  HC_K_RES_DIV = 6,
  HC_K_SPLIT_GRAD = 7, /* column pass: gradient of the new p */
  HC_K_SPLIT_ROW = 8,  /* row pass: C2R, activation, relaxation, R2C */
  HC_K_SPLIT_HEAT = 9, /* column pass: FFT_y, heat factor, IFFT_y */
  HC_K_SPLIT_C2R = 10, /* row pass: C2R to physical m, sum |m|^2 */
  HC_K_CG_YPASS = 11,  /* 3D only: y pass (FFT of 3 fields) of the inner CG */
  HC_K_RES_YPASS = 12, /* 3D only: y pass of the refinement residual */
  HC_K_FIRST_GRAD = 13,  /* refined: the FP32 first residual's gradient pass (from p64) */
  HC_K_FIRST_APPLY = 14, /* refined: its row pass (2D) / row-pair pass (3D) */
  HC_K_FIRST_DIV = 15,   /* refined: its divergence pass, r32 = b32 - q and the inner-CG start */
  HC_K_MID_GRAD = 16,    /* HC_FP32_REFINED: the double-float mid-step residual's gradient pass (from p64) */
  HC_K_MID_APPLY = 17,   /* its row pass (2D) / row-pair pass (3D) */
  HC_K_MID_DIV = 18,     /* its divergence pass */
  HC_K_MID_YPASS = 19,   /* 3D only: its y pass */
  HC_K_COUNT = 20
};

/* Launch one step kernel `reps` times back to back on the context's current
 * buffers, between two CUDA events on the context's stream, and return the
 * mean milliseconds per launch.  Outputs go to scratch buffers and a scratch
 * solve state, so the state of the problem (m, p, S, r) is left as it was;
 * the scratch contents are undefined afterwards.  For measurement only. */
int hc_time_kernel(hc_ctx* ctx, int kernel, int reps, double* ms_per_launch);

/* Number of this library's kernel launches issued by the context so far
 * (graph launches count every kernel node). */
int hc_launch_count(const hc_ctx* ctx, long long* count);

/* Measured FP64 FMA throughput of the current device in TFLOP/s (an FMA counts
 * two flops): the ALU roof against which the FP64 residual kernels are
 * reported.  Two warm-up launches, then `reps` launches of a kernel of
 * independent FMA chains filling every SM, each timed between CUDA events on
 * `stream` (NULL: legacy default stream); the fastest gives the figure.
 * Synchronises that stream.  No context needed; allocates nothing.
 * Errors: HC_EINVAL (reps < 1, NULL tflops), HC_ECUDA. */
int hc_fp64_fma_peak(int reps, void* stream, double* tflops);

/* --- Adjoint (gradients of a loss on m(T)) --- */

/* Bytes of device memory hc_adjoint needs for nsteps steps with a checkpoint
 * every `every` steps: ceil(nsteps/every) checkpoints of (m, p), one segment
 * of `every` states, and the reverse sweep's buffers.  HC_ENOTSUP in the
 * double-float precision mode and on 3D grids. */
int hc_adjoint_workspace_size(const hc_ctx* ctx, int nsteps, int every, size_t* bytes);

/* Discrete adjoint of nsteps loop bodies of Algorithm 1 started from the
 * context's current (m, p): runs the forward steps (storing a checkpoint every
 * `every` steps), then reverses them segment by segment, recomputing each
 * segment's states from its checkpoint.  The pressure solves are differentiated
 * as exact solves (the adjoint solve uses the same operator, which is
 * symmetric, and the context's tolerance).
 *   lamT: dL/dm(T), host, 2*nx*ny FP64 (component-major), for any loss L of
 *         the final conductivity.
 *   outputs (host FP64, each may be NULL): dL/d(c^2), dL/d(D^2) (scalars),
 *         dL/dr (nx*ny), dL/dS (nx*ny, orthogonal to the null space), dL/dm0
 *         (2*nx*ny); derivatives with respect to the grid values.
 *   workspace: device memory of hc_adjoint_workspace_size bytes (256-byte
 *         aligned) or NULL (the call allocates and frees its own).
 * On return the context holds the forward state at step nsteps, as after
 * hc_step(nsteps).  Returns HC_OK, HC_ENOCONV (some solve hit its cap; the
 * gradients are still computed), or an error. */
int hc_adjoint(hc_ctx* ctx, int nsteps, int every, const double* lamT, double* dL_dc2,
               double* dL_dD2, double* dL_dr, double* dL_dS, double* dL_dm0, void* workspace,
               size_t workspace_bytes);

/* --- Batched parameter sweeps --- */

typedef struct hc_batch hc_batch; /* opaque; refers to (does not own) its contexts */

/* Group `count` existing contexts (any mix of grids, parameters and precisions)
 * so that one CUDA graph launch on `stream` advances every one of them by a
 * step.  2D HC_FP32_REFINED contexts that share a grid size (with the default
 * residual switches) form a size class: the class's step is one chain of
 * batched launches, one launch per pass of the step over all its members
 * (each member with its own parameters, fields, tables and device-side CG and
 * refinement loops; a loop runs until its slowest member is done, finished
 * members skip).  The class runs the first member's launch shapes, without
 * the persistent passes.  Every other context (3D, FP64, double-float, a size
 * with a single context) keeps its own step chain.  All chains sit side by
 * side in one graph.  The contexts must stay alive and keep their grids until
 * hc_batch_destroy; changing a context's parameters or tuning afterwards
 * requires rebuilding the batch.  The batch allocates a little device memory
 * of its own (the members' records).
 * Errors: HC_EINVAL (null/duplicate contexts, count < 1), HC_ENOMEM, HC_ECUDA. */
int hc_batch_create(hc_batch** out, hc_ctx* const* ctxs, int count, void* stream);

/* How the batch runs: the number of size classes and of contexts in them
 * (the rest run their own chains).  Errors: HC_EINVAL. */
int hc_batch_classes(const hc_batch* batch, int* classes, int* batched_members);

/* nsteps batched steps.  stats (may be NULL) receives count entries, the last
 * step of each context.  Returns HC_OK or the first non-OK step status of any
 * context (as hc_step does).  A size class's kernel launches are added to the
 * launch count (hc_launch_count) of its first member. */
int hc_batch_step(hc_batch* batch, int nsteps, hc_step_stats* stats);

void hc_batch_destroy(hc_batch* batch);

/* --- Transform without device allocation (the paper has no counterpart) --- */

#define HC_NOALLOC_MAX_POINTS 65536 /* nx*ny limit of hc_spectrum_noalloc */

/* The forward 2D transform of hc_spectrum for callers that cannot allocate
 * device memory: for example a plugin inside a host framework that reserves the
 * whole GPU for its own pool allocator, or a loop where cudaMalloc's implicit
 * device synchronisation is not acceptable.  No context is needed.
 *   f:      device pointer, nx*ny FP64 values, row-major with x fastest.
 *   out:    device pointer receiving ny*(nx/2) complex FP64 values (re/im
 *           interleaved) in the packed layout of hc_spectrum.
 *   nx, ny: powers of two in [8, 4096] with nx*ny <= HC_NOALLOC_MAX_POINTS;
 *           anything else (or a null pointer) returns HC_EINVAL.
 *   stream: cudaStream_t (NULL: legacy default stream); the call only enqueues
 *           work on it and returns.  CUDA failures of its own launches return
 *           HC_ECUDA; a non-sticky error left pending on the calling thread by
 *           earlier work is cleared on entry (cudaGetLastError), not reported.
 * Scratch lives in one fixed 640 KiB static device array of the library
 * (present on every GPU the process uses, until the process exits); the call
 * allocates nothing and calls no allocating routine.  All calls share that
 * array; each call rewrites it completely before reading it, so nothing from
 * an earlier call is reused, but calls whose GPU work overlaps (other streams
 * or threads at the same time) race on it and must be serialised by the
 * caller.  The first call on each device does a one-time set-up (it looks up
 * the array's device address and raises the kernels' shared-memory limit):
 * make that first call before any stream capture. */
int hc_spectrum_noalloc(const double* f, double* out, int nx, int ny, void* stream);

/* --- Bounds-checked build (no counterpart in the paper) ---
 *
 * The library also builds as libhc_gb300_check.so, compiled with HC_CHECK=1.
 * Its kernels are the production kernels. Every device buffer carved from a
 * workspace (the context's, and the adjoint's) is followed by a guard zone of
 * HC_REDZONE_BYTES bytes plus the alignment gap before the next buffer, filled
 * with the byte 0xA5 when the workspace is set up. A kernel or copy that writes
 * past the end of a buffer by up to that much changes the zone. The checked
 * build stands in for a memory checker on machines where none may run.
 *
 * hc_check_redzones scans every guard zone of ctx: one kernel on the context's
 * stream, then a synchronisation. It returns HC_EBOUNDS if any byte changed,
 * with *zone = the first damaged zone in carve order and *owner_bytes = the size
 * of the buffer that zone follows; otherwise HC_OK with *zone = -1. *nzones gets
 * the number of zones checked (0 in the production build, where the call does
 * nothing and returns HC_OK). Any output pointer may be null. Scans from
 * several threads are serialised inside the library. hc_adjoint scans its own
 * workspace's zones before it returns, and reports damage as HC_EBOUNDS.
 *
 * hc_check_poke is a test hook of the checked build. It overwrites one byte of
 * zone `zone` with a host-issued cudaMemsetAsync (no kernel, inside the
 * workspace), so a test can see the scan report it. It returns HC_EINVAL for a
 * zone out of range, and HC_ENOTSUP in the production build. */
#define HC_REDZONE_BYTES 65536
int hc_check_redzones(hc_ctx* ctx, int* nzones, int* zone, size_t* owner_bytes);
int hc_check_poke(hc_ctx* ctx, int zone);

void hc_destroy(hc_ctx* ctx);
const char* hc_strerror(int code);

/* Description of the most recent CUDA failure behind an HC_ECUDA on the
 * calling thread (source line, call, CUDA error name and text); "" if none.
 * The string is owned by the library and overwritten by the next failure. */
const char* hc_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif
