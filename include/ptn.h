/*
 * ptn.h -- C ABI of the GB300 (sm_103a) parallel-in-time Newton solver for
 * constrained nonlinear model predictive control (arXiv 2409.20027).
 *
 * Problem (Sec. II-A, eq. ocp): minimise
 *     l_{N+1}(x_{N+1}) + sum_{t=1..N} l_t(x_t, u_t)
 * subject to x_{t+1} = f(x_t, u_t), g(x_t) <= 0, h(u_t) <= 0, x_1 = x0.
 * Here N = T, l_t(x,u) = (x-xref)^T Q (x-xref) + (u-uref)^T R (u-uref) (no 1/2),
 * l_{N+1}(x) = (x-xref)^T Qf (x-xref), f is a built-in or user-registered model and g, h are
 * box bounds (each finite bound is one constraint row).
 *
 * Solvers: primal log-barrier interior point (Sec. II-B, eq. lb-min / lb-step-2) and
 * ADMM (Sec. II-C, eq. admm-min ... admm-step-5).  Every sub-problem is solved by the
 * parallel-in-time Newton method (Sec. III, Alg. 4): co-state scan (Alg. 1), value
 * function scan (Alg. 2), state propagation scan (Alg. 3), then a line search over
 * closed-loop nonlinear rollouts.  The whole solve of an instance runs on the GPU.
 *
 * Memory: all trajectory arguments are DEVICE pointers to float64 arrays, row-major and
 * time-major (x: (T+1) x nx, u: T x nu, lam: (T+1) x nx).  The caller owns them.  The
 * solver owns its device workspace (allocated by ptn_solver_create).  Problem data are
 * HOST pointers, copied at create.  `stream` is a cudaStream_t (NULL = legacy default);
 * calls are stream-ordered and return after the stream has reached the end of the
 * solve (they synchronise once to read the status).
 *
 * Errors: functions return a status code (0 = PTN_OK, negative = error); the message
 * of the last error is ptn_last_error().  A handle must not be used by two host threads
 * at once.  Device waits are bounded: a wait that expires returns PTN_ERR_TIMEOUT.
 */
#ifndef PTN_H
#define PTN_H

#ifdef __cplusplus
extern "C" {
#endif

#define PTN_OK 0
#define PTN_ERR_INVALID_ARG (-1)
#define PTN_ERR_INFEASIBLE_START (-2) /* IP start not strictly inside the constraints */
#define PTN_ERR_NOT_CONVERGED (-3)    /* outputs hold the last iterate */
#define PTN_ERR_NUMERICAL (-4)        /* non-finite values or regularisation exhausted */
#define PTN_ERR_TIMEOUT (-5)          /* a bounded device wait expired */
#define PTN_ERR_CUDA (-6)

enum { PTN_MODEL_PENDULUM = 0, PTN_MODEL_CARTPOLE = 1, PTN_MODEL_QUADROTOR = 2, PTN_MODEL_SYNTH_TANH = 3 };
enum { PTN_EULER = 0, PTN_RK4 = 1 };
/* Precision of the Newton step (trajectories, co-states, gradients and the final
 * convergence test are FP64 in every mode):
 *   PTN_FP64            all arithmetic in FP64
 *   PTN_FP32_FP64SOLVE  model increments, LQR elements, scans and feedback in FP32;
 *                       (I + C J)^{-1} and Cholesky solves in FP64
 *   PTN_FP32            as above with FP32 solves */
enum { PTN_FP64 = 0, PTN_FP32_FP64SOLVE = 1, PTN_FP32 = 2 };
enum { PTN_METHOD_IP = 0, PTN_METHOD_ADMM = 1 };

/* Problem description (Sec. II-A).  Model constants prm:
 *   pendulum  [g, l, m, b]                       x = (theta, omega), u = torque
 *   cart-pole [m_c, m_p, l, g]                   x = (p, theta, p', theta'), u = force
 *   quadrotor [mass, Ixx, Iyy, Izz, arm, k_m, g] x = (pos, ZYX angles, vel, rates),
 *                                                u = 4 rotor thrusts
 *   synthetic [c]  x+ = A x + B u + c tanh(W x)  (A, B, W host row-major)
 * Bounds: +-INFINITY (or |b| >= 1e300) means no bound.  Rows are ordered state rows
 * first (per component: upper, lower) then control rows; ADMM z, v use this order. */
typedef struct ptn_problem {
  int model, nx, nu, integrator;
  double dt;
  double prm[8];
  const double *A, *B, *W;
  const double *Q, *R, *Qf;
  const double *xref, *uref;
  const double *xlo, *xhi, *ulo, *uhi;
} ptn_problem;

/* Solver settings; ptn_default_options() fills the defaults:
 *   precision FP32_FP64SOLVE, mu 1e-1 -> 1e-6 (x0.1), tol_inner 1e-4, tol_final 1e-6,
 *   block_threads 128, grid_min_T 512, grid_steps_per_thread 2, polish 100, polish_after 50,
 *   cluster_max_blocks 16, sequential 0, costate_mode 0 (the co-state scan), update_mode 0,
 *   max_newton 500 per barrier level, ADMM rho 1, admm_tol 1e-2, max_outer 2000, fp64_finish 1,
 *   alpha0 1e-6 in [1e-10, 1e10], ten step sizes 1, 1/2, ..., Armijo c1 1e-4,
 *   rollout: at most 30 multiple-shooting Newton iterations to relative defect 1e-12. */
typedef struct ptn_options {
  int precision;        /* PTN_FP64, PTN_FP32_FP64SOLVE or PTN_FP32 */
  int max_newton;       /* Newton iterations per barrier level / ADMM sub-problem */
  int max_outer;        /* ADMM outer iterations */
  int ls_count;         /* candidate step sizes 1, beta, beta^2, ... */
  int admm_fixed_iters; /* > 0: run exactly this many ADMM iterations */
  int roll_max_iter;    /* multiple-shooting Newton iterations per rollout */
  int block_threads;    /* threads per CTA when one CTA solves one instance */
  int grid_min_T;       /* single solves with T >= grid_min_T use all SMs (0: never); with
                           grid_min_T > 0, batches of a model with nx >= 8 also use every
                           co-resident CTA of one cooperative launch, a contiguous CTA range
                           per instance sized by its horizon (when one CTA per instance
                           fits), else one CTA per instance */
  int grid_steps_per_thread;
  int polish_after;     /* FP32 modes: exact FP64 gradients after this many iterations of
                           the final barrier level or an ADMM sub-problem, and of an
                           intermediate level once max|d| <= polish * its tolerance */
  int cluster_max_blocks; /* single solves needing 2..cluster_max_blocks CTAs (block_threads
                             threads, grid_steps_per_thread steps each) run on one thread-block
                             cluster (at most 16; 0: never) before the cooperative grid is used */
  int sequential;       /* nonzero: the sequential-in-time baseline, one thread per instance
                           running the serial recursions (n < 8 only); for comparisons */
  int costate_mode;     /* 0: co-states by the suffix scan of Alg. 1 (the paper's method);
                           1: multiplier form, a variant: multipliers nu of the dynamics take
                           the duals of each Newton step's LQR (nu_t += S_t dx_t + s_t), the
                           Lagrangian's gradients d_t, q_t are local in t (no product of
                           F_t^T is formed), the LQR carries q_t as a linear state term, and
                           the stopping test is max(|d|, |q|) <= tol; lam_out returns nu.
                           Same KKT point as mode 0.
                           2: as 1, but every Newton sub-problem (barrier level, ADMM
                           iteration) restarts the multipliers from the co-states of the
                           scan; more robust than 1 far from the solution (where the
                           pure form can stall), still fewer Newton iterations than 0 on
                           long horizons. */
  int update_mode;      /* 0: a Newton step is taken on the closed-loop nonlinear rollout
                           (line search over step sizes; the default); 1: the update of
                           Alg. 4 as printed, x <- x + dx, u <- u + du, taken whenever its
                           cost is finite (for IP: strictly feasible), which leaves dynamics
                           defects of second order; for comparisons */
  double mu0, zeta, mu_final, tol_inner, tol_final, rho, admm_tol;
  double alpha0, alpha_min, alpha_max, ls_beta, armijo_c1, armijo_eps, roll_tol;
  double polish;        /* FP32 modes: exact FP64 gradients once max|d| <= polish * tol_final */
  double armijo_eps32;  /* FP32 modes: Armijo allowance, relative to |J_c|, for merits
                           accumulated as FP32 differences (their rounding floor) */
  int fp64_finish;      /* FP32 modes, single IP solves (ptn_solve_ip, ptn_solve_batch with
                           B = 1): when the solve stops without converging (line search
                           failure or iteration cap), finish it with FP64 LQR data from its
                           last iterate: a second launch of the FP64 kernels, warm-started
                           with the controls reached, starting at the barrier weight where
                           the first stopped; its Newton iterations are added to
                           newton_iters and reported in finish_iters.  With the finish on,
                           the mixed-precision launch also leaves a final barrier level on
                           which 20 iterations of the exact path have not halved max|d|.
                           0: off; default 1.  Not done by ptn_solve_batch_async (no host
                           step) or by ptn_solve_ip_static. */
  int pad_opt;
} ptn_options;

/* Per-solve report.  r_kkt = max(r_stat, r_dyn, r_feas, mu) for IP, where r_stat is
 * max_t |d_t|_inf (gradient of the augmented cost), r_dyn the largest dynamics defect and
 * r_feas the largest constraint violation.  cycles[] are SM clock cycles spent by the
 * group's first thread in the co-state pass, second-order expansion, value pass, state
 * pass, line search, initial rollout, and everything else.  finish_iters: Newton
 * iterations of the FP64 finish (ptn_options.fp64_finish), 0 when none ran; the cycle
 * counts and the other counters then add both launches. */
typedef struct ptn_info {
  int status, newton_iters, outer_iters, ls_rejects, factor_fails, roll_fails;
  int roll_iters, ls_evals, exact_passes, finish_iters;
  double mu, alpha, r_stat, r_dyn, r_feas, r_kkt, J, J_c, r_p, r_d;
  long long cycles[7];
} ptn_info;

typedef struct ptn_solver ptn_solver;

/* Dimensions of model id `model`: a built-in model (pendulum, cart-pole, quadrotor) or one
 * registered from a user unit linked into this library (ids >= 64, see
 * ptn_user_model.cuh).  Writes *nx, *nu and returns 0, or returns PTN_ERR_INVALID_ARG for
 * an id this library does not know.  Needs no GPU. */
int ptn_model_dims(int model, int* nx, int* nu);

/* Fill *opt with the defaults listed above. */
void ptn_default_options(ptn_options* opt);

/* Create a solver for `prob` (copied) able to run batches of up to max_batch instances
 * whose horizons sum to at most max_T * max_batch steps.  Allocates the device
 * workspace on the current device.  Returns PTN_OK and *out, or an error. */
int ptn_solver_create(const ptn_problem* prob, const ptn_options* opt, int max_T, int max_batch,
                      ptn_solver** out);

/* Free the workspace and the handle (NULL is ignored). */
void ptn_solver_destroy(ptn_solver* s);

/* Message of the last error on this handle ("" if none); s may be NULL. */
const char* ptn_last_error(const ptn_solver* s);

/* Replace the options of an existing handle (e.g. precision, tolerances). */
int ptn_set_options(ptn_solver* s, const ptn_options* opt);

/* Time-varying tracking targets for the solves and adjoints that follow (the stage cost
 * l_t of Sec. II-A, eq. ocp, with targets that change with t):
 *   l_t = (x_t - xr_t)^T Q (x_t - xr_t) + (u_t - ur_t)^T R (u_t - ur_t),
 *   terminal (x_T - xr_T)^T Qf (x_T - xr_T).
 * xref_traj: device, the instances' target states concatenated like the state outputs
 * (instance b: T_b + 1 rows of nx); uref_traj: device, like the control outputs (T_b rows
 * of nu).  Either may be NULL (the constant targets of the problem, or of xref per
 * instance, apply).  The handle keeps the pointers, not the data: the arrays must stay
 * valid and match the horizons of every solve until the next call (NULL, NULL restores
 * constant targets).  Not used by ptn_solve_ip_static.  Returns PTN_OK, or
 * PTN_ERR_INVALID_ARG for a NULL handle. */
int ptn_set_reference(ptn_solver* s, const double* xref_traj, const double* uref_traj);

/* Primal log-barrier IP solve of one instance (Sec. II-B with Alg. 4 sub-solves).
 *   x0      device, nx            initial state x_1
 *   u_init  device, T x nu        strictly feasible initial controls, or NULL (zeros)
 *   x_out   device, (T+1) x nx    optimal states (also used as iterate storage)
 *   u_out   device, T x nu        optimal controls
 *   lam_out device, (T+1) x nx    co-states at the solution, or NULL
 *   info    host                  status, iterations, KKT residuals, costs (may be NULL)
 * Returns info->status: PTN_OK, PTN_ERR_NOT_CONVERGED, PTN_ERR_INFEASIBLE_START, ... */
int ptn_solve_ip(ptn_solver* s, const double* x0, const double* u_init, int T, double* x_out,
                 double* u_out, double* lam_out, ptn_info* info, void* stream);

/* ADMM solve of one instance (Sec. II-C).  Arguments as ptn_solve_ip, plus the final
 * consensus variables z_out and multipliers v_out (device, T x nw each, may be NULL),
 * nw = number of finite bounds.  Options rho, admm_tol, max_outer, admm_fixed_iters. */
int ptn_solve_admm(ptn_solver* s, const double* x0, const double* u_init, int T, double* x_out,
                   double* u_out, double* lam_out, double* z_out, double* v_out, ptn_info* info,
                   void* stream);

/* Solve B independent instances of the same model with horizons T_b (host array) in one
 * launch, one CTA per instance (a batch of one runs like ptn_solve_ip).  dt_b (host, B, or NULL) gives each instance its own time
 * step: instance b integrates with dt_b[b] and its stage weights Q, R are multiplied by
 * dt_b[b] / prob.dt (the same continuous-time cost sampled at another rate; Qf is not
 * scaled) -- the fixed-time, varying-sampling-rate protocol of the paper's experiments
 * (Sec. IV).  x0 is device B x nx; xref is device B x nx (per-instance tracking target)
 * or NULL; u_init is device (sum T_b) x nu or NULL.  Outputs are concatenated in
 * instance order: x_out (sum (T_b+1)) x nx, u_out (sum T_b) x nu, lam_out like x_out or
 * NULL.  info_b is a host array of B records (may be NULL).  method is PTN_METHOD_IP or
 * PTN_METHOD_ADMM.  Returns PTN_OK when every instance converged, else the first
 * non-zero instance status (PTN_ERR_INVALID_ARG for a non-positive dt_b entry). */
int ptn_solve_batch(ptn_solver* s, int method, int B, const int* T_b, const double* dt_b,
                    const double* x0, const double* xref, const double* u_init, double* x_out,
                    double* u_out, double* lam_out, ptn_info* info_b, void* stream);

/* Graph-capturable batch solves.  ptn_batch_prepare validates a batch layout (method, B,
 * T_b, dt_b as in ptn_solve_batch), fixes the execution tier and launch shape from the
 * handle's current options, copies the instance table and the options to device buffers
 * reserved for it, and synchronises `stream`.  The layout stays in force until the next
 * ptn_batch_prepare on this handle; synchronous solves in between do not change it, and
 * later option changes reach it only through another prepare.  Returns PTN_OK or
 * PTN_ERR_INVALID_ARG / PTN_ERR_CUDA (with ptn_last_error). */
int ptn_batch_prepare(ptn_solver* s, int method, int B, const int* T_b, const double* dt_b,
                      void* stream);

/* Enqueue one solve of the prepared batch on `stream` and return without waiting: kernel
 * launches only (for a single instance on the cooperative grid tier, two memsets of its
 * barrier counters before the kernel), no host<->device copy, no allocation, no
 * synchronisation -- so the call can be recorded by CUDA stream capture and replayed as a
 * graph (the pointers are then fixed in the graph; update the inputs in place).  Device
 * arguments as in ptn_solve_batch.  info_dev: device array of B ptn_info records that the
 * kernel fills (status, iterations, residuals; read it after the stream has reached the
 * solve), or NULL to keep them in the handle.  ADMM's z, v stay in the handle's workspace.
 * Returns PTN_OK when the work was enqueued, PTN_ERR_INVALID_ARG without a prepared batch,
 * PTN_ERR_CUDA when a launch failed; the solve's own status is in info_dev. */
int ptn_solve_batch_async(ptn_solver* s, const double* x0, const double* xref, const double* u_init,
                          double* x_out, double* u_out, double* lam_out, ptn_info* info_dev,
                          void* stream);

/* Gradients of the scalar loss  gJ * J* + <gx, x*> + <gu, u*>  at B solutions of the
 * barrier problem (at the problem's own dt) with weight mu (J* = optimal barrier objective; x*, u* concatenated as
 * in ptn_solve_batch), with respect to x0 (B x nx), diag Q (B x nx), diag R (B x nu),
 * diag Qf (B x nx) and the model constants prm (B x 8).  The J* part follows the
 * envelope theorem on the Lagrangian eq. ocp-lagrangian (gradient in x0 = lam_1); the x*, u*
 * part solves the adjoint LQR (same Hessian as the Newton step, linear terms from
 * gx, gu) with the value and state scans, and its multipliers with the co-state scan.
 * The adjoint runs in FP64 in every precision mode (one CTA of block_threads threads per
 * instance; a single instance with T_b >= grid_min_T on the cooperative grid): at a solution
 * the reduced Hessian is ill-conditioned near active bounds.
 * All array arguments are device pointers; gx, gu may be NULL (J* part only); any output
 * may be NULL.  xref as in ptn_solve_batch.  Returns PTN_ERR_NUMERICAL when the Hessian
 * is not positive definite on the dynamics at some instance's solution, PTN_ERR_TIMEOUT
 * when a grid barrier wait expired, PTN_ERR_INVALID_ARG for the synthetic model (no
 * adjoint is built for it). */
int ptn_adjoint(ptn_solver* s, int B, const int* T_b, const double* x0, const double* xref,
                const double* x_star, const double* u_star, double mu, double gJ,
                const double* gx, const double* gu, double* g_x0, double* g_Qd, double* g_Rd,
                double* g_Qfd, double* g_prm, void* stream);

/* Checkpointed adjoint of ONE instance whose horizon T may exceed the handle's workspace
 * (Sec. III-A, eq. ocp-lagrangian: the same gradients as ptn_adjoint).  Only the
 * trajectory (x_star: (T+1) x nx, u_star: T x nu, device) is kept for the whole horizon;
 * the horizon is taken in segments of seg_len steps (1 <= seg_len <= max_T * max_batch of
 * the handle), and every segment's linearisations (Jacobians, Hessians, co-states) are
 * recomputed from the trajectory in each of three sweeps over the segments: co-states and
 * the adjoint LQR's value function backward, its states forward, its multipliers and the
 * gradient contributions backward; the sweeps pass boundary values between segments.
 * Segments use the CTA tier, or the cooperative grid from grid_min_T on.  Device memory
 * beyond the handle's workspace: about (T / seg_len) (nx^2 + 4 nx) doubles, allocated and
 * freed by the call.  gx, gu, outputs and errors as in ptn_adjoint; PTN_ERR_INVALID_ARG
 * for nx >= 8 (the wide tier has no segmented form). */
int ptn_adjoint_checkpointed(ptn_solver* s, int T, int seg_len, const double* x0, const double* xref,
                             const double* x_star, const double* u_star, double mu, double gJ,
                             const double* gx, const double* gu, double* g_x0, double* g_Qd,
                             double* g_Rd, double* g_Qfd, double* g_prm, void* stream);

/* Number of constraint rows nw of the handle's problem. */
int ptn_num_rows(const ptn_solver* s);

/* Allocation-free single interior-point solve.  The paper has no counterpart: this is
 * an integration entry point for callers that must not reach the device allocator while
 * solving (a fixed-rate MPC loop, where cudaMalloc/cudaFree can synchronise the device
 * and take unbounded time; a plug-in that keeps no handle between calls).
 *
 * Same problem, options and results as ptn_solver_create + ptn_solve_ip on a one-CTA
 * solve (block_threads threads; grid_min_T and cluster_max_blocks are ignored; option
 * sequential must be 0, else PTN_ERR_INVALID_ARG), but no handle: the problem record,
 * options, report and all workspace arrays live in one file-scope device array of 4 MiB
 * (the cart-pole model needs about 0.7 KB per step, so T up to about 5800; the pendulum
 * about 0.3 KB per step; the quadrotor about 5.7 KB per step, so T up to about 740).
 * A T that does not fit is rejected with PTN_ERR_INVALID_ARG and a message giving the
 * bytes needed.  No device or pinned memory is allocated and no allocating library call
 * is made.
 *
 * Set-up: the array's device address belongs to the CUDA context that loaded the module.
 * A call whose stream is not being captured looks it up in the calling thread's current
 * context (cudaGetSymbolAddress, which loads the module on first use and makes the
 * device's primary context current when the thread has none) and remembers it for that
 * context.  A call made while its stream is being captured uses the remembered address
 * and fails with PTN_ERR_INVALID_ARG when this context has none, so make the first call
 * in each context (the first on each device, and the first after cudaDeviceReset) before
 * any stream capture.
 *
 * Nothing in the array has to start at zero: each call copies the problem record,
 * options and instance entry into it in stream order, and the kernel writes every
 * workspace entry before it reads it.  All calls on one device share the array, so calls
 * whose executions can overlap (other host threads, or streams not ordered with each
 * other) race and corrupt each other's results; serialise them, e.g. on one stream.
 *
 * x0 (device, nx doubles), u_init (device, T*nu doubles, or NULL for zeros), x_out
 * ((T+1)*nx), u_out (T*nu) and lam_out ((T+1)*nx, or NULL) are device buffers owned by
 * the caller.  opt NULL means the defaults.  err (err_len bytes, may be NULL) receives
 * a message on failure, "" on success.  Returns PTN_OK or a status code; the call
 * returns after the solve has finished on `stream`. */
int ptn_solve_ip_static(const ptn_problem* prob, const ptn_options* opt, const double* x0,
                        const double* u_init, int T, double* x_out, double* u_out, double* lam_out,
                        ptn_info* info, char* err, int err_len, void* stream);

/* Library version string. */
const char* ptn_version(void);

/* Self-check of the arithmetic routines the kernels' FP64 solves use in place of a
 * division and of the FP32 <-> FP64 conversion instructions (no counterpart in the paper;
 * for tests).  For i < n: rcp_out[i] = the pivot reciprocal of p[i] (0 where p[i] counts
 * as a singular pivot: zero, not finite, or a binary exponent outside [-1000, 1000]),
 * f2d_out[i] = f[i] widened to FP64, d2f_out[i] = d[i] rounded to FP32 (nearest even),
 * each by the device routine the solver uses.  All pointers are device pointers to n
 * elements owned by the caller; an input and its output may both be NULL to skip that
 * routine.  Enqueued on `stream` (NULL: the legacy default stream); returns PTN_OK,
 * PTN_ERR_INVALID_ARG for n < 0 or an output without its input, or PTN_ERR_CUDA when the
 * launch fails. */
int ptn_arith_check(int n, const double* p, double* rcp_out, const float* f, double* f2d_out,
                    const double* d, float* d2f_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PTN_H */
