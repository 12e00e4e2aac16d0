/*
 * sdf.h -- C ABI of the B300-native (sm_103a) spectral-deflation active-set
 * solver for state-constrained optimal control (arXiv 2606.17971).
 *
 * The method (paper references are sections / equations / algorithms):
 *   S = M + alpha K^T M^-1 K with M = mass*I, K = kscale*A_h      (Sec. 2.1.2 Eq. schur)
 *   primal active-set loop: A <- {i : y_i > psi_i - tau}            (App. B.1 Alg. pdas)
 *   restricted system S_II y_I = rhs_I - S_IA psi_A                  (Sec. 2.1.2 Eq. reduced)
 *   inner solve: A-DEF2 deflated Jacobi-PCG with Z = Phi|_I          (Sec. 2.2.1 Alg. adef2,
 *                (orthonormalised), E = Z^T S_II Z, guard             Sec. 2.2.2, Alg.
 *                cond(E) > tau_cond -> plain Jacobi-PCG               online_deflation l. 5-18)
 *   stop on the unprojected residual ||r|| <= rtol ||b||            (App. B.2 Eq. cg_stop)
 *   A_h: 5-point (2D) / 7-point (3D) -diff_scale div(kappa grad)     (App. A Eq. fd_lap,
 *        with harmonic face means, plus optional per-instance          Eq. harmonic)
 *        first-order upwind convection b . grad
 *
 * Conventions for every entry point:
 *   - Grids are interior nodes of the unit box, n_d per direction,
 *     h_d = 1/(n_d+1), node index i + n_x (j + n_y l) (x fastest).
 *   - "device" pointers are CUDA global-memory addresses on the current device;
 *     "host" pointers are ordinary CPU memory.  The library never allocates
 *     device memory: the caller passes every device buffer (problem buffer,
 *     workspace, inputs, outputs) and keeps it alive for the duration of the
 *     calls that use it.  All work is enqueued on the caller's stream
 *     (a cudaStream_t passed as void*, NULL = legacy default stream).
 *   - Every function returns an sdf_status; no exception or abort crosses the
 *     ABI.  On a non-OK status sdf_last_error(handle) holds a one-line reason.
 *     A sticky CUDA error is reported as SDF_ERR_CUDA with CUDA's text.
 *   - A handle is not thread-safe: calls on one handle must not run
 *     concurrently from several host threads.
 */
#ifndef SDF_H_
#define SDF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SDF_OK = 0,
  SDF_ERR_INVALID_ARG = 1, /* bad size, NULL pointer, misaligned buffer       */
  SDF_ERR_WORKSPACE = 2,   /* buffer smaller than the size query returned     */
  SDF_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed     */
  SDF_ERR_NOT_SPD = 4,     /* reserved: a coarse matrix was not SPD           */
  SDF_ERR_CG_MAXIT = 5,    /* CG hit max_cg without meeting rtol              */
  SDF_ERR_OUTER_MAXIT = 6, /* active set still changing after max_outer       */
  SDF_ERR_BREAKDOWN = 7,   /* CG breakdown: p^T S p <= 0                      */
  SDF_ERR_NONFINITE = 8,   /* NaN / Inf met in a reduction                    */
  SDF_ERR_TIMEOUT = 9,     /* host watchdog: solve exceeded its launch budget */
  SDF_ERR_UNSUPPORTED = 10 /* combination not built (e.g. k > SDF_MAX_K)      */
} sdf_status;

typedef enum { SDF_F64 = 0, SDF_F32 = 1, SDF_BF16 = 2 } sdf_dtype;

/* Arithmetic of the inner solve.
 *   SDF_PREC_F64    every vector, stencil and projection in FP64 (FP64 modes).
 *   SDF_PREC_MIXED  CG vectors, stencil and projections in FP32 with FP32 or
 *                   BF16 modes; the iterate x, the right-hand side, every dot
 *                   product and reduction, the k x k coarse operator and its
 *                   set-up stay FP64, and every `replace_every` iterations
 *                   the residual is recomputed as b - S_II x with the FP64
 *                   stencil and the coarse correction x += Q r is applied;
 *                   convergence is declared only on that FP64 residual:
 *                   ||b - S_II x|| <= max(rtol ||b||, floor_c u || |S_II||x| ||)
 *                   (the second term, the attainable accuracy of an FP64
 *                   residual, is evaluated once per solve, when the
 *                   recurrence has met rtol or the true residual has stopped
 *                   falling; see sdf_stats).
 *                   Not available with per-instance convection
 *                   (SDF_ERR_UNSUPPORTED). */
typedef enum { SDF_PREC_F64 = 0, SDF_PREC_MIXED = 1 } sdf_precision;

/* Maximum deflation rank and outer iterations recorded per instance. */
#define SDF_MAX_K 128
#define SDF_MAX_OUTER 32
/* Instance parameters: 7 doubles per instance, in this order. */
#define SDF_INSTANCE_DOUBLES 7 /* a, c_x, c_y, c_z, b_x, b_y, b_z */

typedef struct sdf_problem sdf_problem;

/* Problem description (host struct, copied by sdf_problem_create).
 *   dim          2 or 3
 *   n[3]         interior nodes per direction (n[2] ignored for dim 2)
 *   alpha        Tikhonov weight (> 0)
 *   mass         M = mass * I (> 0); the paper's form is mass = 1
 *   kscale       K = kscale * A_h; the paper's form is kscale = 1
 *   diff_scale   A_h = diff_scale * (-div(kappa grad)) + b . grad
 *   has_kappa    1: node diffusivity given to sdf_problem_create, 0: kappa = 1
 *   convection   1: each instance carries its upwind convection velocity b
 *   yd_sigma     width of the Gaussian desired state
 *                y_d(x) = a exp(-|x - c|^2 / (2 yd_sigma^2)), rhs = mass y_d
 *   time_axis    1: the all-at-once space-time problem (App. E.2) of the
 *                parabolic state equation y_t + A_x y = u, y(., 0) = 0, on
 *                (0, t_final] with implicit Euler.  Needs dim = 3: axes 0 and
 *                1 are space (unit square, n[0] x n[1] interior nodes),
 *                axis 2 is time with n[2] steps of dt = t_final / n[2].  The
 *                forward operator F (block lower bidiagonal: I/dt + A_x on
 *                the diagonal, -I/dt below) takes the place of A, so
 *                S = mass I + wgt F^T F; there is no diffusion along time
 *                (time faces of kappa are unused), and an instance's
 *                convection velocity, if any, acts in space only (b_z is
 *                ignored).  The desired state is ramped in time (App. F.5):
 *                y_d(x, t_l) = (1 - exp(-t_l / ramp_tau)) a exp(-|x - c|^2 /
 *                (2 yd_sigma^2)), x in space, t_l = (l + 1) dt.
 *                FP64 path only (SDF_PREC_MIXED is refused, as for
 *                convection).  0: the steady problem (t_final, ramp_tau
 *                unused).
 *   t_final, ramp_tau  (> 0 when time_axis = 1) */
typedef struct {
  int32_t dim;
  int32_t n[3];
  double alpha;
  double mass;
  double kscale;
  double diff_scale;
  int32_t has_kappa;
  int32_t convection;
  double yd_sigma;
  int32_t time_axis;
  double t_final;
  double ramp_tau;
} sdf_problem_desc;

/* Solve options (defaults from sdf_default_opts).
 *   rtol         CG tolerance on ||r||/||b|| (App. B.2)            [1e-8]
 *   tau          active-set tolerance (App. B.1)                  [1e-10]
 *   tau_cond     solve-time guard on cond(E) (Remark tau_cond)    [1e10]
 *   max_outer    maximum inner solves per instance (<= SDF_MAX_OUTER) [30]
 *   max_cg       CG iteration cap per inner solve                 [1000000]
 *   deflate      1: A-DEF2 with the reference modes, 0: plain Jacobi-PCG [1]
 *   check_every  CG iterations enqueued between two host polls of the
 *                per-instance convergence flags                   [64]
 *   profile      1: time the first CG iteration of every poll interval with
 *                CUDA events on the solve's stream (see sdf_get_profile) [0]
 *   max_blocks   cap on the blocks per instance of the grid-stride kernels
 *                (0 = automatic: about two blocks per SM in total)  [0]
 *   precision    sdf_precision of the inner solve                 [SDF_PREC_F64]
 *   replace_every mixed path: CG iterations between FP64 residual
 *                replacements (0 = 100)                           [100]
 *   max_launches host watchdog: total iteration launches per solve call
 *                before SDF_ERR_TIMEOUT (0 = 4 * max_cg)          [0]
 *   ritz_r       Ritz re-selection (Sec. 2.2.3): 0 < ritz_r < k deflates
 *                with the ritz_r Ritz vectors of S_II of smallest Ritz value
 *                in the restricted pool of the k registered modes; the
 *                guard then applies to their Galerkin matrix      [0: off]
 *   safe_r       conditioning-based safe merge (Sec. 2.2.5, Algorithm safe):
 *                0 < safe_r < k takes the first safe_r registered modes as
 *                the eigenmode part and the rest, in order, as POD
 *                candidates; each candidate is orthogonalised against the
 *                basis so far (skipped if its norm < tau_dep) and accepted
 *                while cond(Z^T S_II Z) <= tau_safe (the first violation ends
 *                the merge).  Takes precedence over ritz_r        [0: off]
 *   tau_safe, tau_dep  thresholds of the safe merge          [1e4, 1e-10]
 *   floor_c      constant of the attainable-accuracy floor (sdf_stats); the
 *                mixed path stops on max(rtol, floor); 0: rtol only  [10]
 *   column_depth mixed 3D path: z planes per column item of the stencil
 *                kernels, 8, 16, 32 or 64 (0: the depth sdf_autotune chose
 *                for this batch size, else 32 for batches of 8 or more) [0]
 *   column_pairs mixed 3D path: 1 runs the stencil kernels on instance pairs
 *                (two instances per block on the packed FP32 pipe), 2 one
 *                instance per block, 0 what sdf_autotune chose for this
 *                batch size (pairs for 2 or more instances when untuned) [0]
 *   graph        1: the launches between two host polls (check_every CG
 *                iterations on the FP64 path; replace_every iterations, the
 *                residual replacement and the correction pass on the mixed
 *                path) are captured once per call into a CUDA graph on a
 *                private stream and replayed on `stream`; 0: launched one by
 *                one.  Passes timed with profile = 1 are launched one by one.
 *                The call must not be made while `stream` is being captured
 *                (it synchronises `stream` between chunks)             [1] */
typedef struct {
  double rtol;
  double tau;
  double tau_cond;
  int32_t max_outer;
  int32_t max_cg;
  int32_t deflate;
  int32_t check_every;
  int32_t profile;
  int32_t max_blocks;
  int32_t precision;
  int32_t replace_every;
  int64_t max_launches;
  int32_t ritz_r;
  int32_t safe_r;
  double tau_safe;
  double tau_dep;
  double floor_c;
  int32_t column_depth;
  int32_t column_pairs;
  int32_t graph;
} sdf_opts;

/* Per-instance statistics (host struct filled at the end of a solve).
 * true_relres and relres_floor are taken in FP64 on each inner solve's final
 * iterate x_I (App. B.2: the stopping rule tests the recurrence residual,
 * which can drift from the true one):
 *   true_relres  = ||b_I - S_II x_I|| / ||b_I||,
 *   relres_floor = floor_c u || |S_II| |x_I| || / ||b_I||, u = 2^-53, the
 *                  attainable accuracy of an FP64 residual (|S_II| is the
 *                  entrywise absolute value; both are 0 when b_I = 0). */
typedef struct {
  int32_t status;                     /* sdf_status of this instance          */
  int32_t outer_iters;                /* inner solves performed               */
  int32_t cg_iters[SDF_MAX_OUTER];    /* CG iterations of each inner solve    */
  int32_t n_active[SDF_MAX_OUTER];    /* |A| in force during each solve       */
  int32_t fallback[SDF_MAX_OUTER];    /* 1: guard fired, plain PCG used       */
  int32_t floor_stop[SDF_MAX_OUTER];  /* mixed path: 1 when the solve was
                                         declared converged on the floor
                                         (rtol not attainable), 0 on rtol     */
  double cond_E[SDF_MAX_OUTER];       /* estimated cond(E) (0 if plain)       */
  double relres[SDF_MAX_OUTER];       /* recurrence ||r||/||b|| at exit       */
  double true_relres[SDF_MAX_OUTER];  /* FP64 ||b - S_II x||/||b|| at exit    */
  double relres_floor[SDF_MAX_OUTER]; /* attainable-accuracy floor (above)    */
} sdf_stats;

void sdf_default_opts(sdf_opts *o);

/* Create a host-side problem handle.
 *   kappa_host: N node diffusivities (host, copied) when desc->has_kappa, else
 *   ignored.  Errors: SDF_ERR_INVALID_ARG for a bad description. */
sdf_status sdf_problem_create(const sdf_problem_desc *desc, const double *kappa_host,
                              sdf_problem **out);

/* A problem given by its state operator K instead of a grid (the general
 * form of Sec. 2.1.2 Eq. schur): K is n x n CSR on the host (rowptr n+1,
 * col and val rowptr[n] entries, 0-based, FP64; copied), and the library
 * assembles S = mass I + (alpha kscale^2 / mass) K^T K on the host once
 * (Gustavson's row-merge product), with its inverse diagonal.  Bind it with
 * sdf_problem_device_bytes / sdf_problem_bind as any problem; S is then
 * applied row by row from the assembled CSR in every FP64-path kernel
 * (sdf_apply_S, the solve, the coarse set-up).  There is no grid: solve
 * with sdf_solve_batch_rhs; the mixed path, the closed-form modes and the
 * eigensolves of the grid's A return SDF_ERR_UNSUPPORTED.  n <= 2^30 and
 * nnz(S) <= INT_MAX; SDF_ERR_INVALID_ARG on a malformed CSR (decreasing
 * row pointers, a column outside [0, n), a non-finite value). */
sdf_status sdf_problem_create_csr(int64_t n, const int32_t *rowptr, const int32_t *col,
                                  const double *val, double mass, double alpha, double kscale,
                                  sdf_problem **out);

/* Bytes of device memory the problem's operator data needs (face
 * coefficients of A_h); may be 0 for constant kappa. */
sdf_status sdf_problem_device_bytes(const sdf_problem *p, size_t *bytes);

/* Bind a caller-owned device buffer of at least sdf_problem_device_bytes bytes
 * (256-byte aligned) and fill it: kappa is copied to it and the harmonic face
 * coefficients diff_scale * kappa_f / h_d^2 (App. A Eq. harmonic; a face
 * towards the Dirichlet boundary takes the node value) are computed on the
 * device.  Must precede every solve.  Enqueued on `stream`. */
sdf_status sdf_problem_bind(sdf_problem *p, void *dev_buf, size_t bytes, void *stream);

/* Register the reference modes Phi (Sec. 2.2.2 Eq. eig): device pointer to an
 * N x k column-major array (mode j at Phi + j*ld elements), ld >= N,
 * 1 <= k <= SDF_MAX_K, of type `dtype` (SDF_F64 for the FP64 path, SDF_F32 or
 * SDF_BF16 for the mixed path).  The
 * library keeps the pointer, not a copy; the caller keeps the memory alive and
 * unchanged while solves use it.  The base address must be 16-byte aligned. */
sdf_status sdf_set_reference_modes(sdf_problem *p, const void *phi_dev, int k, int64_t ld,
                                   sdf_dtype dtype);

/* Closed-form reference modes for a constant-coefficient diffusion reference
 * S_ref = mass I + w (diff_scale L_h)^2 (Sec. 2.2.8): the k smallest Kronecker
 * sine modes, ties broken lexicographically by (i_d, ..., i_1).  Writes
 * phi_dev (N x k column-major, ld, dtype) on the device and, if eigvals_host
 * is not NULL, the k eigenvalues of S_ref to host memory.  Does not register
 * the modes (call sdf_set_reference_modes). */
sdf_status sdf_analytic_modes(sdf_problem *p, int k, void *phi_dev, int64_t ld, sdf_dtype dtype,
                              double *eigvals_host, void *stream);

/* Space-time Kronecker deflation basis (App. E.2.1 Eq. kron_basis):
 * Phi_st = I_{n_t} (x) Z_s for a problem with time_axis = 1.  Z_s (device,
 * N_s = n[0] n[1] rows, r columns, leading dimension ldz, dtype) is a
 * spatial basis, e.g. sdf_analytic_modes of the 2D problem on the same
 * spatial grid.  phi_dev (device, N rows, r n_t columns, leading dimension
 * ld, the same dtype) receives column l r + j = Z_s[:, j] on time step l
 * and zero elsewhere.  r n_t <= SDF_MAX_K. */
sdf_status sdf_spacetime_kron_modes(sdf_problem *p, const void *zs_dev, int r, int64_t ldz,
                                    sdf_dtype dtype, void *phi_dev, int64_t ld, void *stream);

/* A general temporal factor (App. E.2.1): Phi_st = W_t (x) Z_s with W_t
 * (host, n_t x r_t, column-major, FP64) and Z_s as above; column a r + j is
 * spatial mode j scaled by W_t[l, a] on time step l (the product in FP64,
 * rounded once to dtype).  W_t = I gives the Kronecker basis, the DCT-II
 * columns of sdf_dct2_basis the paper's cosine basis.  n_t r_t <= 1024,
 * r r_t <= SDF_MAX_K. */
sdf_status sdf_spacetime_modes(sdf_problem *p, const double *wt_host, int rt, const void *zs_dev,
                               int r, int64_t ldz, sdf_dtype dtype, void *phi_dev, int64_t ld,
                               void *stream);

/* The first r orthonormal DCT-II basis vectors of length n as the columns
 * of w_host (n x r, column-major):
 * w[l, a] = sqrt((2 - [a = 0]) / n) cos(pi (l + 1/2) a / n).  1 <= r <= n;
 * other arguments leave w_host untouched.  Host only. */
void sdf_dct2_basis(int n, int r, double *w_host);

/* Workspace bytes for a batch of `batch` instances under `opts`. */
sdf_status sdf_workspace_size(const sdf_problem *p, int batch, const sdf_opts *opts,
                              size_t *bytes);

/* Solve `batch` instances (primal active-set loop around A-DEF2 or plain
 * Jacobi-PCG), all resident on the device:
 *   inst_dev    batch x SDF_INSTANCE_DOUBLES doubles (device)
 *   psi_dev     N doubles: the state bound, shared by the batch (device)
 *   ws, ws_bytes  workspace of at least sdf_workspace_size bytes (device,
 *                 256-byte aligned); contents on entry are ignored
 *   y_dev       batch x N doubles out: state, y_A = psi_A (device)
 *   lambda_dev  batch x N doubles out: multiplier rhs - S y, or NULL (device)
 *   active_dev  batch x N bytes out: 1 on the final active set (device)
 *   stats_host  batch sdf_stats out (host), or NULL
 * Returns the worst instance status (SDF_OK when every instance converged).
 * The call returns after the solve has finished on `stream` (it polls
 * convergence flags between launches). */
sdf_status sdf_solve_batch(sdf_problem *p, const double *inst_dev, int batch,
                           const double *psi_dev, const sdf_opts *opts, void *ws, size_t ws_bytes,
                           void *stream, double *y_dev, double *lambda_dev, uint8_t *active_dev,
                           sdf_stats *stats_host);

/* The same solve with a given start instead of zero: the first inner solve
 * (A = {}) starts from x0_dev (batch x N doubles, device) and every later one
 * from the previous outer iterate, each restricted to its inactive set.  The
 * active-set path is the cold one (A grows from {} by the same rule); only the
 * CG iterations change.  x0 is meant to approximate the solution of the
 * first (unconstrained) solve, e.g. the learned warm start below.  No
 * counterpart in the paper, whose inner solves start from zero. */
sdf_status sdf_solve_batch_x0(sdf_problem *p, const double *inst_dev, int batch,
                              const double *psi_dev, const double *x0_dev, const sdf_opts *opts,
                              void *ws, size_t ws_bytes, void *stream, double *y_dev,
                              double *lambda_dev, uint8_t *active_dev, sdf_stats *stats_host);

/* sdf_solve_batch with caller-given right-hand sides: rhs_dev (batch x N
 * FP64, device, instance-major) replaces mass y_d of every instance (Sec.
 * 2.1.2 Eq. reduced then uses rhs_I - S_IA psi_A).  inst_dev may be NULL
 * when the problem has no per-instance convection (it is read for nothing
 * else); a problem created by sdf_problem_create_csr must be solved this
 * way.  Everything else as sdf_solve_batch; lambda = rhs - S y. */
sdf_status sdf_solve_batch_rhs(sdf_problem *p, const double *inst_dev, const double *rhs_dev,
                               int batch, const double *psi_dev, const sdf_opts *opts, void *ws,
                               size_t ws_bytes, void *stream, double *y_dev, double *lambda_dev,
                               uint8_t *active_dev, sdf_stats *stats_host);

/* Autotuner of the batched mixed 3D path: for this batch size, time a short
 * capped solve (40 CG iterations) of these instances with each candidate
 * column depth of the stencil kernels (8, 16, 32, 64 planes per block), each
 * with instance pairs and with one instance per block, and keep the fastest
 * for later solves of this handle with the same batch size (*choice receives
 * the depth; 0 when nothing is tuned for this problem).  Outputs y_dev /
 * active_dev are scratch here.  sdf_autotune_choice returns the depth and the
 * pairing (1 pairs, 0 single, -1 not tuned) kept for a batch size.  No
 * counterpart in the paper. */
sdf_status sdf_autotune(sdf_problem *p, const double *inst_dev, int batch, const double *psi_dev,
                        const sdf_opts *opts, void *ws, size_t ws_bytes, void *stream,
                        double *y_dev, uint8_t *active_dev, int *choice);
sdf_status sdf_autotune_choice(const sdf_problem *p, int batch, int *depth, int *pairs);

/* The same solve with every input and output in HOST memory: the instance
 * array and psi are copied to the device inside the call and y, lambda (if not
 * NULL) and active are copied back; the workspace (device) must be at least
 * sdf_workspace_size(...) + sdf_host_io_bytes(p, batch) bytes. */
sdf_status sdf_host_io_bytes(const sdf_problem *p, int batch, size_t *bytes);
sdf_status sdf_solve_batch_host(sdf_problem *p, const double *inst_host, int batch,
                                const double *psi_host, const sdf_opts *opts, void *ws,
                                size_t ws_bytes, void *stream, double *y_host,
                                double *lambda_host, uint8_t *active_host,
                                sdf_stats *stats_host);

/* Building blocks, exposed for tests.
 * sdf_apply_S: out = S_II u on I and 0 on A (mode 0), or out = S u on the
 * whole grid (mode 1), for one instance `inst_dev` (7 doubles, device; its
 * convection velocity is used), `active_dev` N bytes (1 = active; ignored in
 * mode 1), u_dev and out_dev N doubles (device).  In mode 0 u must be zero on
 * A.  Sec. 2.1.2 Eq. schur / Eq. reduced, applied matrix-free in flux form. */
sdf_status sdf_apply_S(sdf_problem *p, const double *inst_dev, const uint8_t *active_dev,
                       const double *u_dev, double *out_dev, int mode, void *ws, size_t ws_bytes,
                       void *stream);

/* sdf_project: out_dev[j] = sum_{i in I} Phi_j(i) v_i for the registered modes
 * (the masked projection Phi_I^T v of Alg. adef2), k doubles (device).
 * `active_dev` N bytes (1 = active), v_dev N doubles (device). */
sdf_status sdf_project(sdf_problem *p, const uint8_t *active_dev, const double *v_dev,
                       double *out_dev, void *ws, size_t ws_bytes, void *stream);

/* sdf_project_noalloc: the same result as sdf_project, for callers that may
 * not allocate device memory at all -- for example code running inside a host
 * application that hands out all GPU memory itself, or a loop with hard
 * latency limits where an allocation (and the device synchronisation it can
 * cause) is not allowed.  Instead of a caller workspace it uses one fixed
 * scratch array built into the library: 512 x 128 doubles of partial sums plus
 * 64 words of counters (about 513 KB), held on every GPU that loads the
 * library until the process exits.  Limits: k <= SDF_MAX_K (128), otherwise
 * SDF_ERR_UNSUPPORTED with a message; FP64 modes only.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.  Later calls reuse the address.  The array's
 *     memory is reserved when CUDA loads the library's module on that device:
 *     at context creation, or with lazy module loading at the latest during
 *     that first call -- one more reason to make it before any capture.
 *   - Call it with the device current on which the problem was bound
 *     (sdf_problem_bind); another current device is refused with
 *     SDF_ERR_INVALID_ARG.
 *   - The array is shared by all calls in the process and keeps the last
 *     call's contents; the call clears the counters it needs, so results do
 *     not depend on earlier calls.  Calls that overlap on the GPU (different
 *     streams, or different handles at once) race on the array: serialise
 *     them.
 *   - Calls no device-memory allocator (cudaMalloc, cudaFree, or a library
 *     routine that allocates).
 * The paper has no counterpart to this entry point; it exists only for
 * callers that cannot allocate.  Arguments as for sdf_project. */
sdf_status sdf_project_noalloc(sdf_problem *p, const uint8_t *active_dev, const double *v_dev,
                               double *out_dev, void *stream);

/* Kernel timing and launch counts (tracing).  Kernel ids of sdf_profile:
 *   0 expand   p = P z + beta p             (coarse GEMV + Phi expansion)
 *   1 spmv     q = S_II p, (p, q)
 *   2 update   x, r update, S_II z, Phi_I^T S_II z, (r, z), ||r||
 *   3 setup    b = rhs_I - S_IA psi_A, Jacobi diagonal
 *   4 coarse   W = S_II Phi_I, Gram matrices, k x k factorisation
 *   5 active   active-set update
 *   6 lambda   multiplier
 *   7 resid    mixed path: FP64 residual replacement
 *   8 project  mixed path: projection GEMM Phi^T [v_1..v_B] and coarse GEMV
 * ms[i] / samples[i] is the mean duration of kernel i over the launches timed
 * with opts.profile = 1; launches counts every kernel the library enqueued
 * since the last reset (timed or not). */
#define SDF_NPROF 9
typedef struct {
  double ms[SDF_NPROF];
  int64_t samples[SDF_NPROF];
  int64_t launches;
} sdf_profile;
sdf_status sdf_get_profile(const sdf_problem *p, sdf_profile *out);
sdf_status sdf_reset_profile(sdf_problem *p);

/* One-line description of the last error on this handle ("" if none). */
const char *sdf_last_error(const sdf_problem *p);

/* Release the host handle (device buffers stay the caller's). */
void sdf_problem_destroy(sdf_problem *p);

/* Reference eigensolve (Sec. 2.2.2, where the paper uses ARPACK): the k
 * smallest eigenpairs of A (no convection: A symmetric), which are those of
 * S with lambda_S = mass + wgt lambda_A^2, by Chebyshev-filtered subspace
 * iteration (Zhou & Saad's scaled filter on [a, b], a = the largest Ritz
 * value of the block, b = a Gershgorin bound of A) with Cholesky-QR
 * orthonormalisation (twice) and Rayleigh-Ritz; all vector work in FP64 on
 * the GPU, the (k + guard)^2 factorisations on the host.  The start block is
 * SplitMix64 of (seed, index).
 *   tol       stop when every wanted pair has ||A phi - lambda phi|| <=
 *             tol |lambda|
 *   degree    Chebyshev degree per filter pass
 *   guard     extra block vectors (0: max(16, k / 2)); k + guard <= 320
 *   max_iter  filter passes
 * phi_dev: k orthonormal columns of N doubles with leading dimension ld
 * (device); lambda_S_host / lambda_A_host (k, ascending, may be NULL).
 * SDF_ERR_UNSUPPORTED with convection; SDF_ERR_CG_MAXIT if not converged (the
 * best block so far is written). */
typedef struct {
  double tol;
  int32_t degree;
  int32_t guard;
  int32_t max_iter;
  uint64_t seed;
} sdf_eig_opts;
typedef struct {
  int32_t iters;
  int32_t converged;
  double max_rel_resid;
  int64_t matvecs;
  double seconds;
} sdf_eig_stats;
void sdf_default_eig_opts(sdf_eig_opts *o);
sdf_status sdf_eig_workspace_size(const sdf_problem *p, int k, const sdf_eig_opts *o,
                                  size_t *bytes);
sdf_status sdf_reference_modes_eig(sdf_problem *p, int k, const sdf_eig_opts *o, double *phi_dev,
                                   int64_t ld, double *lambda_S_host, double *lambda_A_host,
                                   sdf_eig_stats *stats, void *ws, size_t ws_bytes, void *stream);

/* Coarse-grid reference basis (Sec. 2.2.7, Algorithm coarse): the r_pool
 * smallest eigenpairs of the same problem on a grid of n_d / c interior nodes
 * per direction (kappa injected at the fine node nearest to each coarse node;
 * sdf_reference_modes_eig with the options o), prolongated to the fine grid by
 * (bi/tri)linear interpolation with zero boundary values (Eq. prolong), then
 * orthonormalised by a QR that discards every column whose R_jj is below
 * tau_sv times the largest column norm.  phi_dev receives *r_out <= r_pool
 * orthonormal columns (N doubles, leading dimension ld, device);
 * lambda_c_host (r_pool, may be NULL) the coarse eigenvalues of S_c; stats
 * those of the coarse eigensolve.  c >= 2; SDF_ERR_UNSUPPORTED with
 * convection. */
sdf_status sdf_coarse_modes_workspace_size(const sdf_problem *p, int c, int r_pool,
                                           const sdf_eig_opts *o, size_t *bytes);
sdf_status sdf_reference_modes_coarse(sdf_problem *p, int c, int r_pool, const sdf_eig_opts *o,
                                      double tau_sv, double *phi_dev, int64_t ld, int *r_out,
                                      double *lambda_c_host, sdf_eig_stats *stats, void *ws,
                                      size_t ws_bytes, void *stream);

/* ==========================================================================
 * Spectral diagnostics (App. A.1 sources of spectral variation, Sec. 4.1 and
 * App. D spectral-coherence diagnostics).  Off the solve path: tooling that
 * explains iteration counts.  Each call synchronises its stream before it
 * returns, and results land in host memory.
 * ========================================================================== */

/* Active-set distances of B instances from one reference active set:
 *   sym_diff_host[b] = |A_ref sym-diff A_b|, delta_host[b] = sym_diff / N (Eq. delta),
 *   n_active_host[b] = |A_b|,               rho_host[b]   = n_active / N (Eq. rho),
 *   delta_w_host[b]  = sum_j w_j |A_ref(j) - A_b(j)| / sum_j w_j with
 *                      w_j = sum_{q<r} phi_q(j)^2 over the registered
 *                      reference modes (the eigenmode-weighted distance of
 *                      App. D.6); r = 0 skips it (delta_w_host may be NULL),
 *                      r > 0 needs registered modes with r <= k.
 * active_ref_dev: N bytes; active_dev: B x N bytes (1 = active), device.
 * The counts are exact.  delta_w is FP64 and summed in a fixed order, so it
 * is deterministic.  Any host output may be NULL.  ws: device, 256-byte
 * aligned, at least sdf_diag_sets_workspace_size bytes. */
sdf_status sdf_diag_sets_workspace_size(const sdf_problem *p, int B, size_t *bytes);
sdf_status sdf_diag_active_sets(sdf_problem *p, const uint8_t *active_ref_dev,
                                const uint8_t *active_dev, int B, int r, int64_t *sym_diff_host,
                                int64_t *n_active_host, double *delta_host, double *rho_host,
                                double *delta_w_host, void *ws, size_t ws_bytes, void *stream);

/* Operator drift (Eq. epsilon) of the full-domain Schur complements:
 *   eps_host[b] = ||S(ref) - S(b)||_2 / ||S(ref)||_2,
 * with S(ref) and S(b) the operators of the reference instance inst_ref_dev
 * (SDF_INSTANCE_DOUBLES, device) and of the B instances inst_dev
 * (B x SDF_INSTANCE_DOUBLES, device).  They differ through the per-instance
 * convection velocity, the only instance-dependent part of S.  Each 2-norm
 * is the largest |eigenvalue| of a symmetric operator.  It is computed by
 * `steps` Lanczos steps with full reorthogonalisation from a fixed
 * SplitMix64 start vector, each step applying S through sdf_apply_S.  The
 * result is a lower bound that becomes exact once steps reaches the
 * dimension, or earlier on an invariant subspace.  A zero difference gives
 * eps = 0 exactly.  norm_ref_host (may be NULL) receives ||S(ref)||_2.
 * 1 <= steps <= 1024.  ws: at least sdf_diag_drift_workspace_size bytes. */
sdf_status sdf_diag_drift_workspace_size(const sdf_problem *p, int steps, size_t *bytes);
sdf_status sdf_diag_drift(sdf_problem *p, const double *inst_ref_dev, const double *inst_dev,
                          int B, int steps, double *eps_host, double *norm_ref_host, void *ws,
                          size_t ws_bytes, void *stream);

/* The k smallest eigenpairs of the restricted operator S_II (App. A.2, whose
 * spectrum interlaces that of S).  S_II is taken on the inactive set of
 * active_dev (N bytes, device) for the instance inst_dev (device), as
 * sdf_apply_S mode 0 applies it; convection is allowed, because S is
 * symmetric either way.  Method: Chebyshev-filtered subspace iteration as in
 * sdf_reference_modes_eig, on S_II itself, with the spectrum bounded above by
 * mass + wgt (Gershgorin bound of A)^2.  The block stays zero on A.
 * phi_dev receives k orthonormal columns (N doubles, leading dimension ld,
 * zero on A), lambda_host (k) their eigenvalues in ascending order.  Needs
 * |I| >= k + guard; SDF_ERR_CG_MAXIT if not converged within o->max_iter.
 * o = NULL takes sdf_default_restricted_eig_opts: degree 200, guard
 * max(32, k/2), tol 1e-8 (the low spectrum of S_II is that of A squared, so
 * a filter degree gains about the square root of what it gains on A, and
 * the attainable relative residual is about 1e-16 ||S|| / lambda_1).
 * ws: at least sdf_restricted_eig_workspace_size bytes (o may be NULL). */
void sdf_default_restricted_eig_opts(int k, sdf_eig_opts *o);
sdf_status sdf_restricted_eig_workspace_size(const sdf_problem *p, int k, const sdf_eig_opts *o,
                                             size_t *bytes);
sdf_status sdf_restricted_modes_eig(sdf_problem *p, const double *inst_dev,
                                    const uint8_t *active_dev, int k, const sdf_eig_opts *o,
                                    double *phi_dev, int64_t ld, double *lambda_host,
                                    sdf_eig_stats *stats, void *ws, size_t ws_bytes,
                                    void *stream);

/* Principal angles between the restricted reference modes and V, in two
 * readings.  sorted_host[i] (k values, may be NULL): the principal angles in
 * radians between the k-dimensional spans of Phi_I[:, :k] and V[:, :k],
 * ascending; the paper's diagnostic theta_r (Sec. 4.1, App. D, "the
 * principal angle at the deflation cutoff") is sorted_host[r-1] and
 * theta_max the last.  theta_host[r-1], r = 1..k: the nested angle of
 * Prop. dk (App. A.3) with S = {1..r}, the largest principal angle between
 * span(Phi_I[:, :r]) and span(V[:, :r]).  Phi_I is the first
 * r registered reference modes with their rows on the active set of
 * active_dev zeroed.  V_dev is N x k FP64, column-major, leading dimension
 * ldv, device: for instance the eigenvectors of S_II from
 * sdf_restricted_modes_eig.  Both bases are orthonormalised by Cholesky-QR,
 * which keeps the nested spans.  cos theta_r is the smallest singular value
 * of the leading r x r block of Q_Phi^T Q_V.  Because the angle is taken
 * from its cosine, angles below about 1e-7 rad are resolved only to about
 * that.  SDF_ERR_NOT_SPD if either restricted basis is numerically rank
 * deficient.  k <= the number of registered modes.
 * ws: at least sdf_diag_angles_workspace_size bytes. */
sdf_status sdf_diag_angles_workspace_size(const sdf_problem *p, int k, size_t *bytes);

/* True relative residual of each instance's final inner solve, from the
 * outputs of a solve with lambda requested (App. B.2: the solve stops on the
 * recurrence residual, which can drift from the true one):
 *   relres_host[b] = ||r_I|| / ||b_I||, r_I = lambda_I (lambda = rhs - S y),
 *   b_I = rhs_I - S_IA psi_A = r_I + S_II y_I.
 * y_dev, lambda_dev: B x N FP64; active_dev: B x N bytes (the final active
 * sets); inst_dev: B x SDF_INSTANCE_DOUBLES, may be NULL without per-instance
 * convection; all device.  One S_II application per instance.  ws: at
 * least sdf_diag_relres_workspace_size bytes. */
sdf_status sdf_diag_relres_workspace_size(const sdf_problem *p, size_t *bytes);
sdf_status sdf_diag_relres(sdf_problem *p, const double *inst_dev, int B, const double *y_dev,
                           const double *lambda_dev, const uint8_t *active_dev,
                           double *relres_host, void *ws, size_t ws_bytes, void *stream);
sdf_status sdf_diag_angles(sdf_problem *p, const uint8_t *active_dev, const double *V_dev,
                           int64_t ldv, int k, double *theta_host, double *sorted_host, void *ws,
                           size_t ws_bytes, void *stream);

/* ==========================================================================
 * Learned warm start (no counterpart in the paper, which lists learned
 * initialisations only as related work).  A multilayer perceptron maps the
 * instance parameters to the coefficients of a POD basis of solved states
 * (the paper's POD, Sec. 2.2.4, mean-centred); the expansion
 * x0 = ybar + Psi c is the start of every inner solve (sdf_solve_batch_x0).
 * The MLP's products run on the tensor cores (tcgen05.mma, BF16 operands,
 * FP32 accumulation in tensor memory); everything else is FP32 (MLP) or FP64
 * (POD).  These entry points take no problem handle; their error text is
 * returned by sdf_aux_last_error() (per host thread).
 * ========================================================================== */

#define SDF_MLP_MAX_LAYERS 8
#define SDF_POD_MAX_R 64
#define SDF_POD_MAX_SNAPSHOTS 512
#define SDF_FIT_MAX_SNAPSHOTS 4096

/* width[0] inputs, width[1..n_layers-1] hidden (GELU), width[n_layers]
 * outputs (identity); every width in 1..256. */
typedef struct {
  int32_t n_layers;
  int32_t width[SDF_MLP_MAX_LAYERS + 1];
} sdf_mlp_desc;

/* Parameters (FP32, device): for each layer l = 1..n_layers, W_l
 * (width[l] x width[l-1], row-major) then b_l (width[l]).  Returns the count,
 * or -1 for a bad description. */
int64_t sdf_mlp_param_count(const sdf_mlp_desc *d);

/* Workspace (device, 256-byte aligned) of sdf_mlp_forward and
 * sdf_mlp_loss_grad for `batch` rows. */
sdf_status sdf_mlp_workspace_size(const sdf_mlp_desc *d, int batch, size_t *bytes);

/* y = f(x): x_dev batch x width[0] FP32 row-major, y_dev batch x
 * width[n_layers] FP32 (device).  Weights and layer inputs are rounded to
 * BF16 for the products; biases and GELU are FP32.  SDF_ERR_TIMEOUT if a
 * tensor-core completion wait gave up (the result is then undefined). */
sdf_status sdf_mlp_forward(const sdf_mlp_desc *d, const float *theta_dev, const float *x_dev,
                           int batch, float *y_dev, void *ws, size_t ws_bytes, void *stream);

/* Mean squared error L = mean((f(x) - t)^2) over the batch and the outputs,
 * written to *loss_dev (one double, device), and its gradient with respect to
 * theta (grad_dev, same layout as theta, FP32, device).  t_dev: batch x
 * width[n_layers] FP32.  The back-propagated errors are rounded to BF16 for
 * the products, as the layer inputs are. */
sdf_status sdf_mlp_loss_grad(const sdf_mlp_desc *d, const float *theta_dev, const float *x_dev,
                             const float *t_dev, int batch, float *grad_dev, double *loss_dev,
                             void *ws, size_t ws_bytes, void *stream);

/* One Adam step with bias correction (Kingma & Ba) on n FP32 parameters:
 * m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * theta -= lr (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps); step >= 1. */
sdf_status sdf_adam_step(float *theta_dev, const float *grad_dev, float *m_dev, float *v_dev,
                         int64_t n, int step, float lr, float beta1, float beta2, float eps,
                         void *stream);

/* POD of m solved states Y_dev (m x n FP64, one state per row, device):
 * ybar_dev (n FP64) the mean; the r leading left singular vectors of the
 * centred snapshots (method of snapshots: eigen-decomposition of the m x m
 * Gram matrix, FP64), each column's sign chosen so that its largest-magnitude
 * entry is positive, written node-major in BF16 (psi_rm_bf16_dev, n x r,
 * r contiguous) and column-major in FP64 (psi_cm_dev, n x r); the singular
 * values (sing_host, r) and the snapshots' coefficients (coef_host, m x r,
 * may be NULL).  2 <= m <= SDF_POD_MAX_SNAPSHOTS, 1 <= r <= min(m - 1,
 * SDF_POD_MAX_R), m * r <= 25600.  SDF_ERR_NOT_SPD if fewer than r singular
 * values are positive. */
sdf_status sdf_pod_workspace_size(int64_t n, int m, size_t *bytes);
sdf_status sdf_pod(const double *Y_dev, int m, int64_t n, int r, double *ybar_dev,
                   void *psi_rm_bf16_dev, double *psi_cm_dev, double *sing_host,
                   double *coef_host, void *ws, size_t ws_bytes, void *stream);

/* x0[b] = ybar + Psi (cstd[b] * cscale + cmean) for b < batch (<= 256):
 * psi_rm_bf16_dev n x r BF16 node-major (16-byte aligned, r a multiple of 16),
 * cstd_dev batch x r FP32 (standardised coefficients, e.g. the MLP output),
 * cmean_dev / cscale_dev r FP32, x0_dev batch x n FP64 (all device).  The
 * coefficients are rounded to BF16 for the tensor-core product. */
sdf_status sdf_warm_expand_workspace_size(int batch, int r, size_t *bytes);
sdf_status sdf_warm_expand(const void *psi_rm_bf16_dev, const double *ybar_dev, int64_t n, int r,
                           const float *cstd_dev, const float *cmean_dev, const float *cscale_dev,
                           int batch, double *x0_dev, void *ws, size_t ws_bytes, void *stream);

/* A warm-start model: every pointer is a caller-owned device buffer.
 *   mlp        width[0] = number of instance parameters used as inputs (the
 *              first width[0] of the SDF_INSTANCE_DOUBLES, e.g. a, c_x, c_y,
 *              c_z in 3D), width[n_layers] = r
 *   r          POD rank, a multiple of 16, <= SDF_POD_MAX_R
 *   n          state length N
 *   in_lo/hi   parameter box: inputs are scaled to [-1, 1] by min-max
 *   theta      sdf_mlp_param_count FP32 (initialised by the caller before
 *              sdf_warm_fit: the initial weights are an input)
 *   ybar       n FP64; psi n x r FP64 column-major (mode j at psi + j n)
 *   cmean, cscale  r FP32: the targets are (c_j - cmean_j) / cscale_j with
 *              cmean_j the mean of coefficient j over the training snapshots
 *              and one common scale cscale_j = max_j std(c_j), so that the
 *              loss weighs each coefficient by its share of the state */
typedef struct {
  sdf_mlp_desc mlp;
  int32_t r;
  int64_t n;
  double in_lo[8], in_hi[8];
  float *theta;
  double *ybar;
  double *psi;
  float *cmean, *cscale;
} sdf_warm_model;

/* Fit the model to m solved states Y_dev (m x n FP64, device) of the
 * instances inst_dev (m x SDF_INSTANCE_DOUBLES, device): POD (writes ybar,
 * psi), target scaling (cmean, cscale), then `epochs` full-batch Adam steps
 * (beta 0.9 / 0.999, eps 1e-8) with the learning rate decaying from lr0 to 0
 * on a cosine, starting from the caller's theta.  loss_host (epochs doubles,
 * may be NULL) receives the loss before each step.  2 <= m <=
 * SDF_FIT_MAX_SNAPSHOTS, epochs <= 4096.  The POD basis comes from the first
 * min(m, 384) states (the method of snapshots diagonalises their Gram matrix
 * on the host); the MLP is fit to the coefficients of all m states on that
 * basis, Psi^T (y_i - ybar) in FP64, so a large training set costs one
 * projection, not a larger eigenproblem. */
sdf_status sdf_warm_fit_workspace_size(const sdf_warm_model *M, int m, size_t *bytes);
sdf_status sdf_warm_fit(sdf_warm_model *M, const double *Y_dev, const double *inst_dev, int m,
                        int epochs, float lr0, double *loss_host, void *ws, size_t ws_bytes,
                        void *stream);

/* x0 (batch x n FP64, device) = ybar + psi (f(scaled inst) * cscale + cmean)
 * for the instances inst_dev (batch x SDF_INSTANCE_DOUBLES, device),
 * batch <= 256: the start for sdf_solve_batch_x0.  The MLP runs on the
 * tensor cores; the expansion is FP64, because BF16 rounding of psi (2^-9
 * relative, uncorrelated from node to node) would put high-frequency error
 * into x0 that the stiff S amplifies in the starting residual. */
sdf_status sdf_warm_predict_workspace_size(const sdf_warm_model *M, int batch, size_t *bytes);
sdf_status sdf_warm_predict(const sdf_warm_model *M, const double *inst_dev, int batch,
                            double *x0_dev, void *ws, size_t ws_bytes, void *stream);

/* Error text of the last failing call above on this host thread. */
const char *sdf_aux_last_error(void);

/* The learned pipeline end to end from HOST buffers (no counterpart in the
 * paper): the instances (batch x SDF_INSTANCE_DOUBLES) and psi (N) are copied
 * to the device inside the call, x0 is predicted by the model M
 * (sdf_warm_predict: MLP on the tensor cores, FP64 expansion), the batch is
 * solved from x0 (sdf_solve_batch_x0), and y, lambda (if not NULL) and the
 * active sets are copied back; every copy is on `stream`, and the call returns
 * after the last one.  batch <= 256.  ws (device, 256-byte aligned): at least
 * sdf_workspace_size(p, batch, opts) rounded up to 256 plus
 * sdf_learned_host_io_bytes(p, M, batch) bytes.  Returns the solve's status
 * (instance statuses in stats_host), or the prediction's error. */
sdf_status sdf_learned_host_io_bytes(const sdf_problem *p, const sdf_warm_model *M, int batch,
                                     size_t *bytes);
sdf_status sdf_solve_batch_learned_host(sdf_problem *p, const sdf_warm_model *M,
                                        const double *inst_host, int batch,
                                        const double *psi_host, const sdf_opts *opts, void *ws,
                                        size_t ws_bytes, void *stream, double *y_host,
                                        double *lambda_host, uint8_t *active_host,
                                        sdf_stats *stats_host);

#ifdef __cplusplus
}
#endif
#endif /* SDF_H_ */
