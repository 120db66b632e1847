// ptn_api.cu -- C ABI of the solver (declared in include/ptn.h): handle, workspace,
// option records, instance tables and the launches of the device-resident solver.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "../../include/ptn.h"
#include "ptn_launch.cuh"
#include "ptn_user_model.cuh"

using namespace ptn;

// per (model, precision) launchers, one translation unit each; weak references so a
// library built without some model units still links (those models report an error)
#define PTN_WEAK __attribute__((weak))
#define PTN_DECL(m)                                      \
  cudaError_t ptn_launch_##m##_f64(LaunchReq&) PTN_WEAK;  \
  cudaError_t ptn_launch_##m##_f32d(LaunchReq&) PTN_WEAK; \
  cudaError_t ptn_launch_##m##_f32(LaunchReq&) PTN_WEAK;
PTN_DECL(pendulum)
PTN_DECL(cartpole)
PTN_DECL(quadrotor)
PTN_DECL(synth)

namespace {

typedef cudaError_t (*launch_fn)(LaunchReq&);

#define PTN_PICK(m) \
  (precision == PTN_FP64 ? ptn_launch_##m##_f64 : precision == PTN_FP32_FP64SOLVE ? ptn_launch_##m##_f32d : ptn_launch_##m##_f32)

// models registered from outside the library (ptn_user_model.cuh); filled by static
// initialisers of the user units while the library loads, read-only afterwards
struct UserModel {
  int id, nx, nu, nrows;  // nrows: the model's own inequality rows (interior point only)
  launch_fn f64, f32d, f32;
};
constexpr int kMaxUserModels = 32;
UserModel g_user_models[kMaxUserModels];
int g_num_user_models = 0;

const UserModel* find_user_model(int id) {
  for (int i = 0; i < g_num_user_models; i++)
    if (g_user_models[i].id == id) return &g_user_models[i];
  return nullptr;
}

launch_fn pick_launcher(int model, int precision) {
  switch (model) {
    case PTN_MODEL_PENDULUM: return PTN_PICK(pendulum);
    case PTN_MODEL_CARTPOLE: return PTN_PICK(cartpole);
    case PTN_MODEL_QUADROTOR: return PTN_PICK(quadrotor);
    case PTN_MODEL_SYNTH_TANH: return PTN_PICK(synth);
    default: {
      const UserModel* um = find_user_model(model);
      if (!um) return nullptr;
      return precision == PTN_FP64 ? um->f64 : precision == PTN_FP32_FP64SOLVE ? um->f32d : um->f32;
    }
  }
}

int model_dims(int model, int* nx, int* nu) {
  switch (model) {
    case PTN_MODEL_PENDULUM: *nx = 2; *nu = 1; return 0;
    case PTN_MODEL_CARTPOLE: *nx = 4; *nu = 1; return 0;
    case PTN_MODEL_QUADROTOR: *nx = 12; *nu = 4; return 0;
    case PTN_MODEL_SYNTH_TANH: *nx = 32; *nu = 8; return 0;
    default: {
      const UserModel* um = find_user_model(model);
      if (!um) return -1;
      *nx = um->nx;
      *nu = um->nu;
      return 0;
    }
  }
}

bool has_bound(const double* b, int i) { return b && isfinite(b[i]) && fabs(b[i]) < 1e300; }

}  // namespace

namespace ptn {
int register_model(int id, int nx, int nu, user_launch_fn f64, user_launch_fn f32d, user_launch_fn f32,
                   int nrows) {
  if (id < PTN_USER_MODEL_MIN || nx < 1 || nx > PTN_MAXN || nu < 1 || nu > PTN_MAXM) return -1;
  if (find_user_model(id) || g_num_user_models >= kMaxUserModels) return -1;
  g_user_models[g_num_user_models++] = UserModel{id, nx, nu, nrows, f64, f32d, f32};
  return 0;
}
}  // namespace ptn

namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// Launch shape of one solve call, fixed on the host before anything is enqueued.
struct LaunchPlan {
  launch_fn fn = nullptr;
  int method = 0, precision = 0, B = 0, tier = 0, nblocks = 0, nthreads = 0;
  long long steps = 0;
};

struct ptn_solver {
  ptn_options opt;
  const double* xtraj = nullptr;  // time-varying targets of the solves (ptn_set_reference), device
  const double* utraj = nullptr;
  ProbDev hprob;
  ProbDev* dprob = nullptr;
  OptDev* dopt = nullptr;
  double* dsynth = nullptr;
  int n = 0, m = 0, nw = 0;
  long long cap_steps = 0;
  int cap_batch = 0;
  char* ws = nullptr;
  WorkRaw w{};
  InstDev* dinst = nullptr;
  InfoDev* dinfo = nullptr;
  InstDev* hinst = nullptr;  // pinned
  InfoDev* hinfo = nullptr;  // pinned
  OptDev* hopt = nullptr;    // pinned
  GridScratch gs{};
  // batch prepared for ptn_solve_batch_async: its own instance table and option record,
  // so that synchronous solves in between do not change what a captured graph reads
  InstDev* dinst_a = nullptr;
  OptDev* dopt_a = nullptr;
  LaunchPlan plan_a{};
  bool plan_a_ok = false;
  int grid_cap_blocks = 0;
  int num_sms = 0;
  char err[512];
};

static int fail(ptn_solver* s, int code, const char* fmt, ...) {
  if (s) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(s->err, sizeof(s->err), fmt, ap);
    va_end(ap);
  }
  return code;
}

#define CK(call)                                                                             \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return fail(s, PTN_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

extern "C" int ptn_model_dims(int model, int* nx, int* nu) {
  if (!nx || !nu) return PTN_ERR_INVALID_ARG;
  return model_dims(model, nx, nu) == 0 ? PTN_OK : PTN_ERR_INVALID_ARG;
}

extern "C" void ptn_default_options(ptn_options* o) {
  memset(o, 0, sizeof(*o));
  o->precision = PTN_FP32_FP64SOLVE;
  o->max_newton = 500;
  o->max_outer = 2000;
  o->ls_count = 10;
  o->admm_fixed_iters = 0;
  o->roll_max_iter = 30;
  o->block_threads = 128;
  o->grid_min_T = 512;
  o->grid_steps_per_thread = 2;
  o->mu0 = 1e-1;
  o->zeta = 0.1;
  o->mu_final = 1e-6;
  o->tol_inner = 1e-4;
  o->tol_final = 1e-6;
  o->rho = 1.0;
  o->admm_tol = 1e-2;
  o->alpha0 = 1e-6;
  o->alpha_min = 1e-10;
  o->alpha_max = 1e10;
  o->ls_beta = 0.5;
  o->armijo_c1 = 1e-4;
  o->armijo_eps = 1e-12;
  o->roll_tol = 1e-12;
  o->polish = 100.0;
  o->armijo_eps32 = 1e-9;
  o->polish_after = 50;
  o->cluster_max_blocks = 16;
  o->fp64_finish = 1;
}

extern "C" const char* ptn_version(void) { return "ptn 0.1 (sm_103a)"; }

// the solves' pivot reciprocal and conversions, element by element (ptn_arith_check)
__global__ void k_arith_check(int n, const double* p, double* rcp_out, const float* f, double* f2d_out,
                              const double* d, float* d2f_out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (p) rcp_out[i] = ptn::pivot_ok(p[i]) ? ptn::pivot_rcp(p[i]) : 0.0;
    if (f) f2d_out[i] = ptn::f32_to_f64(f[i]);
    if (d) d2f_out[i] = ptn::f64_to_f32(d[i]);
  }
}

extern "C" int ptn_arith_check(int n, const double* p, double* rcp_out, const float* f, double* f2d_out,
                               const double* d, float* d2f_out, void* stream) {
  if (n < 0 || (p && !rcp_out) || (f && !f2d_out) || (d && !d2f_out)) return PTN_ERR_INVALID_ARG;
  if (n == 0) return PTN_OK;
  const int blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
  k_arith_check<<<blocks, 256, 0, (cudaStream_t)stream>>>(n, p, rcp_out, f, f2d_out, d, d2f_out);
  return cudaGetLastError() == cudaSuccess ? PTN_OK : PTN_ERR_CUDA;
}

extern "C" const char* ptn_last_error(const ptn_solver* s) { return s ? s->err : ""; }

extern "C" int ptn_num_rows(const ptn_solver* s) { return s ? s->nw : 0; }

static int check_options(ptn_solver* s, const ptn_options* o) {
  if (o->precision != PTN_FP64 && o->precision != PTN_FP32_FP64SOLVE && o->precision != PTN_FP32)
    return fail(s, PTN_ERR_INVALID_ARG, "precision must be PTN_FP64, PTN_FP32_FP64SOLVE or PTN_FP32");
  if (o->block_threads < 32 || o->block_threads > 256 || (o->block_threads % 32))
    return fail(s, PTN_ERR_INVALID_ARG, "block_threads must be a multiple of 32 in [32, 256]");
  if (o->max_newton < 1 || o->ls_count < 1 || o->roll_max_iter < 1 || o->max_outer < 1)
    return fail(s, PTN_ERR_INVALID_ARG, "iteration limits must be positive");
  if (!(o->mu0 > 0) || !(o->zeta > 0 && o->zeta < 1) || !(o->mu_final > 0) || !(o->rho > 0) ||
      !(o->ls_beta > 0 && o->ls_beta < 1) || !(o->alpha_max >= o->alpha_min) || !(o->alpha_min >= 0))
    return fail(s, PTN_ERR_INVALID_ARG, "invalid continuation, penalty or regularisation parameter");
  if (o->grid_steps_per_thread < 1) return fail(s, PTN_ERR_INVALID_ARG, "grid_steps_per_thread must be >= 1");
  if (o->cluster_max_blocks < 0 || o->cluster_max_blocks > 16)
    return fail(s, PTN_ERR_INVALID_ARG, "cluster_max_blocks must be in [0, 16]");
  if (o->update_mode < 0 || o->update_mode > 1)
    return fail(s, PTN_ERR_INVALID_ARG, "update_mode must be 0 (rollout line search) or 1 (x += dx, u += du)");
  if (o->costate_mode < 0 || o->costate_mode > 2)
    return fail(s, PTN_ERR_INVALID_ARG,
                "costate_mode must be 0 (co-state scan), 1 (multiplier form) or 2 (multiplier form restarted "
                "from the co-states at each sub-problem)");
  return PTN_OK;
}

extern "C" int ptn_set_options(ptn_solver* s, const ptn_options* opt) {
  if (!s || !opt) return PTN_ERR_INVALID_ARG;
  int rc = check_options(s, opt);
  if (rc) return rc;
  s->opt = *opt;
  return PTN_OK;
}

extern "C" int ptn_set_reference(ptn_solver* s, const double* xref_traj, const double* uref_traj) {
  if (!s) return PTN_ERR_INVALID_ARG;
  s->err[0] = 0;
  s->xtraj = xref_traj;
  s->utraj = uref_traj;
  return PTN_OK;
}

extern "C" void ptn_solver_destroy(ptn_solver* s) {
  if (!s) return;
  cudaFree(s->dprob);
  cudaFree(s->dopt);
  cudaFree(s->dsynth);
  cudaFree(s->ws);
  cudaFree(s->dinst);
  cudaFree(s->dinfo);
  cudaFree(s->dinst_a);
  cudaFree(s->dopt_a);
  cudaFree(s->gs.bar);
  cudaFree(s->gs.err);
  cudaFree(s->gs.red);
  cudaFree(s->gs.xs);
  cudaFreeHost(s->hinst);
  cudaFreeHost(s->hinfo);
  cudaFreeHost(s->hopt);
  delete s;
}

extern "C" int ptn_solver_create(const ptn_problem* prob, const ptn_options* opt, int max_T, int max_batch,
                                 ptn_solver** out) {
  if (!out) return PTN_ERR_INVALID_ARG;
  *out = nullptr;
  ptn_solver* s = new ptn_solver();
  s->err[0] = 0;
  *out = s;  // on error the caller reads ptn_last_error() and destroys the handle
  int rc = PTN_OK;
  auto bad = [&](int code) { *out = s; return code; };
  if (!prob) return bad(fail(s, PTN_ERR_INVALID_ARG, "prob is NULL"));
  if (opt) {
    rc = check_options(s, opt);
    if (rc) return bad(rc);
    s->opt = *opt;
  } else {
    ptn_default_options(&s->opt);
  }
  int nx, nu;
  if (model_dims(prob->model, &nx, &nu))
    return bad(fail(s, PTN_ERR_INVALID_ARG, "unknown or unsupported model id %d", prob->model));
  if (prob->nx != nx || prob->nu != nu)
    return bad(fail(s, PTN_ERR_INVALID_ARG, "model %d has nx=%d nu=%d, got %d %d", prob->model, nx, nu, prob->nx,
                    prob->nu));
  if (prob->integrator != PTN_EULER && prob->integrator != PTN_RK4)
    return bad(fail(s, PTN_ERR_INVALID_ARG, "integrator must be PTN_EULER or PTN_RK4"));
  if (!(prob->dt > 0) || !isfinite(prob->dt)) return bad(fail(s, PTN_ERR_INVALID_ARG, "dt must be positive"));
  if (!prob->Q || !prob->R || !prob->Qf || !prob->xref || !prob->uref)
    return bad(fail(s, PTN_ERR_INVALID_ARG, "Q, R, Qf, xref, uref are required"));
  if (max_T < 1 || max_batch < 1) return bad(fail(s, PTN_ERR_INVALID_ARG, "max_T and max_batch must be >= 1"));
  s->n = nx;
  s->m = nu;
  ProbDev& P = s->hprob;
  memset(&P, 0, sizeof(P));
  P.model = prob->model;
  P.nx = nx;
  P.nu = nu;
  P.integrator = prob->integrator;
  P.dt = prob->dt;
  for (int i = 0; i < 8; i++) P.prm[i] = prob->prm[i];
  for (int i = 0; i < nx * nx; i++) {
    if (!isfinite(prob->Q[i]) || !isfinite(prob->Qf[i])) return bad(fail(s, PTN_ERR_INVALID_ARG, "Q/Qf not finite"));
    P.Q[i] = prob->Q[i];
    P.Qf[i] = prob->Qf[i];
  }
  for (int i = 0; i < nu * nu; i++) {
    if (!isfinite(prob->R[i])) return bad(fail(s, PTN_ERR_INVALID_ARG, "R not finite"));
    P.R[i] = prob->R[i];
  }
  for (int i = 0; i < nx; i++) P.xref[i] = prob->xref[i];
  for (int i = 0; i < nu; i++) P.uref[i] = prob->uref[i];
  int k = 0;
  for (int i = 0; i < nx; i++) {
    if (has_bound(prob->xhi, i)) { P.row_isx[k] = 1; P.row_idx[k] = i; P.row_sgn[k] = 1.0; P.row_bnd[k] = prob->xhi[i]; k++; }
    if (has_bound(prob->xlo, i)) { P.row_isx[k] = 1; P.row_idx[k] = i; P.row_sgn[k] = -1.0; P.row_bnd[k] = prob->xlo[i]; k++; }
  }
  for (int i = 0; i < nu; i++) {
    if (has_bound(prob->uhi, i)) { P.row_isx[k] = 0; P.row_idx[k] = i; P.row_sgn[k] = 1.0; P.row_bnd[k] = prob->uhi[i]; k++; }
    if (has_bound(prob->ulo, i)) { P.row_isx[k] = 0; P.row_idx[k] = i; P.row_sgn[k] = -1.0; P.row_bnd[k] = prob->ulo[i]; k++; }
  }
  P.nw = k;
  s->nw = k;
  cudaDeviceProp dp;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaGetDeviceProperties(&dp, dev));
  s->num_sms = dp.multiProcessorCount;
  if (prob->model == PTN_MODEL_SYNTH_TANH) {
    // the map's matrices A (nx x nx), B (nx x nu), W (nx x nx): FP64 and FP32 copies in
    // device memory owned by the handle
    if (!prob->A || !prob->B || !prob->W)
      return bad(fail(s, PTN_ERR_INVALID_ARG, "the synthetic model needs A, B and W"));
    const size_t na = (size_t)nx * nx, nb = (size_t)nx * nu, tot = 2 * na + nb;
    std::vector<double> h(tot);
    std::vector<float> hf(tot);
    for (size_t i = 0; i < na; i++) { h[i] = prob->A[i]; h[na + nb + i] = prob->W[i]; }
    for (size_t i = 0; i < nb; i++) h[na + i] = prob->B[i];
    for (size_t i = 0; i < tot; i++) {
      if (!isfinite(h[i])) return bad(fail(s, PTN_ERR_INVALID_ARG, "A, B, W not finite"));
      hf[i] = (float)h[i];
    }
    CK(cudaMalloc(&s->dsynth, tot * (sizeof(double) + sizeof(float))));
    CK(cudaMemcpy(s->dsynth, h.data(), tot * sizeof(double), cudaMemcpyHostToDevice));
    float* df = reinterpret_cast<float*>(s->dsynth + tot);
    CK(cudaMemcpy(df, hf.data(), tot * sizeof(float), cudaMemcpyHostToDevice));
    P.A = s->dsynth; P.B = s->dsynth + na; P.W = s->dsynth + na + nb;
    P.A32 = df; P.B32 = df + na; P.W32 = df + na + nb;
  }
  CK(cudaMalloc(&s->dprob, sizeof(ProbDev)));
  CK(cudaMemcpy(s->dprob, &P, sizeof(ProbDev), cudaMemcpyHostToDevice));
  CK(cudaMalloc(&s->dopt, sizeof(OptDev)));
  CK(cudaMalloc(&s->dinst, sizeof(InstDev) * max_batch));
  CK(cudaMalloc(&s->dinfo, sizeof(InfoDev) * max_batch));
  CK(cudaMalloc(&s->dinst_a, sizeof(InstDev) * max_batch));
  CK(cudaMalloc(&s->dopt_a, sizeof(OptDev)));
  CK(cudaMallocHost(&s->hinst, sizeof(InstDev) * max_batch));
  CK(cudaMallocHost(&s->hinfo, sizeof(InfoDev) * max_batch));
  CK(cudaMallocHost(&s->hopt, sizeof(OptDev)));
  // workspace
  const long long S = (long long)max_T * max_batch, SB = S + max_batch;
  s->cap_steps = S;
  s->cap_batch = max_batch;
  const int n = nx, m = nu, nw = k;
  size_t off = 0;
  size_t o_xB = off; off = align256(off + sizeof(double) * SB * n);
  size_t o_uB = off; off = align256(off + sizeof(double) * S * m);
  size_t o_lam = off; off = align256(off + sizeof(double) * SB * n);
  size_t o_d = off; off = align256(off + sizeof(double) * S * m);
  size_t o_F64 = off; off = align256(off + sizeof(double) * S * n * n);
  size_t o_G64 = off; off = align256(off + sizeof(double) * S * n * m);
  size_t o_E = off; off = align256(off + 8 * S * n * n);
  size_t o_Gm = off; off = align256(off + 8 * S * n * m);
  size_t o_Pm = off; off = align256(off + 8 * SB * n * n);
  size_t o_Mm = off; off = align256(off + 8 * S * n * m);
  size_t o_Rm = off; off = align256(off + 8 * S * m * m);
  size_t o_Gam = off; off = align256(off + 8 * S * m * n);
  size_t o_gam = off; off = align256(off + 8 * S * m);
  size_t o_dx = off; off = align256(off + 8 * SB * n);
  size_t o_du = off; off = align256(off + 8 * S * m);
  size_t o_z = off; off = align256(off + sizeof(double) * S * (nw > 0 ? nw : 1));
  size_t o_v = off; off = align256(off + sizeof(double) * S * (nw > 0 ? nw : 1));
  size_t o_q = off; off = align256(off + sizeof(double) * SB * n);
  size_t o_dnu = off; off = align256(off + sizeof(double) * SB * n);
  size_t o_Sv = off; off = align256(off + 8 * SB * n * n);
  size_t o_sv = off; off = align256(off + 8 * SB * n);
  CK(cudaMalloc(&s->ws, off));
  char* b = s->ws;
  s->w.xB = (double*)(b + o_xB); s->w.uB = (double*)(b + o_uB); s->w.lam = (double*)(b + o_lam);
  s->w.d = (double*)(b + o_d); s->w.F64 = (double*)(b + o_F64); s->w.G64 = (double*)(b + o_G64);
  s->w.E = b + o_E; s->w.Gm = b + o_Gm;
  s->w.Pm = b + o_Pm; s->w.Mm = b + o_Mm; s->w.Rm = b + o_Rm; s->w.Gam = b + o_Gam; s->w.gam = b + o_gam;
  s->w.dx = b + o_dx; s->w.du = b + o_du;
  s->w.z = (double*)(b + o_z); s->w.v = (double*)(b + o_v);
  s->w.q = (double*)(b + o_q); s->w.dnu = (double*)(b + o_dnu); s->w.Sv = b + o_Sv; s->w.sv = b + o_sv;
  // grid-tier scratch, sized for 4 co-resident blocks per SM
  s->grid_cap_blocks = 4 * s->num_sms;
  CK(cudaMalloc(&s->gs.bar, 2 * sizeof(unsigned) * max_batch));  // a counter pair per instance (wide batches)
  CK(cudaMalloc(&s->gs.err, sizeof(int)));
  CK(cudaMalloc(&s->gs.red, sizeof(double) * 2 * 8 * s->grid_cap_blocks));
  size_t eb = 0;
  {
    LaunchReq q{};
    q.tier = 0; q.precision = PTN_FP64; q.query = 1; q.nthreads = 128; q.elem_bytes = &eb;
    launch_fn fn = pick_launcher(P.model, PTN_FP64);
    if (!fn) fn = pick_launcher(P.model, PTN_FP32_FP64SOLVE);
    if (!fn) return fail(s, PTN_ERR_INVALID_ARG, "kernels for model %d are not built", P.model);
    CK(fn(q));
  }
  s->gs.elem_bytes = (int)((eb + 15) & ~size_t(15));
  CK(cudaMalloc(&s->gs.xs, (size_t)2 * s->gs.elem_bytes * s->grid_cap_blocks));
  s->gs.spin_limit = 1ll << 26;
  *out = s;
  return PTN_OK;
}

static void to_optdev(const ptn_options& o, int method, OptDev* d) {
  memset(d, 0, sizeof(*d));
  d->mu0 = o.mu0; d->zeta = o.zeta; d->mu_final = o.mu_final; d->tol_inner = o.tol_inner;
  d->tol_final = o.tol_final; d->rho = o.rho; d->admm_tol = o.admm_tol;
  d->alpha0 = o.alpha0; d->alpha_min = o.alpha_min; d->alpha_max = o.alpha_max; d->ls_beta = o.ls_beta;
  d->armijo_c1 = o.armijo_c1;
  d->armijo_eps = o.armijo_eps;
  d->roll_tol = o.roll_tol;
  d->polish = o.polish;
  d->armijo_eps32 = o.armijo_eps32;
  d->polish_after = o.polish_after;
  d->init_max_iter = 64;
  d->max_newton = o.max_newton; d->max_outer = o.max_outer; d->ls_count = o.ls_count;
  d->admm_fixed_iters = o.admm_fixed_iters; d->roll_max_iter = o.roll_max_iter; d->method = method;
  d->costate_mode = o.costate_mode;
  d->update_mode = o.update_mode;
  d->spin_limit = 1ll << 26;
}

static void from_info(const InfoDev& d, ptn_info* o) {
  o->status = d.status; o->newton_iters = d.newton_iters; o->outer_iters = d.outer_iters;
  o->ls_rejects = d.ls_rejects; o->factor_fails = d.factor_fails; o->roll_fails = d.roll_fails;
  o->roll_iters = d.roll_iters; o->ls_evals = d.ls_evals; o->exact_passes = d.exact_passes; o->finish_iters = 0;
  for (int k = 0; k < 7; k++) o->cycles[k] = d.cyc[k];
  o->mu = d.mu; o->alpha = d.alpha; o->r_stat = d.r_stat; o->r_dyn = d.r_dyn; o->r_feas = d.r_feas;
  o->r_kkt = d.r_kkt; o->J = d.J; o->J_c = d.J_c; o->r_p = d.r_p; o->r_d = d.r_d;
}

// Validate the horizons (and optional time steps) of a batch and fill the instance table
// hi: per-instance offsets into the concatenated time axis.  *steps = sum of T_b.
static int fill_instances(ptn_solver* s, int B, const int* T_b, const double* dt_b, InstDev* hi,
                          long long* steps_out) {
  if (B < 1 || B > s->cap_batch) return fail(s, PTN_ERR_INVALID_ARG, "B=%d outside [1, %d]", B, s->cap_batch);
  if (!T_b) return fail(s, PTN_ERR_INVALID_ARG, "NULL argument");
  long long steps = 0;
  for (int i = 0; i < B; i++) {
    if (T_b[i] < 1) return fail(s, PTN_ERR_INVALID_ARG, "horizon T_b[%d]=%d must be >= 1", i, T_b[i]);
    if (dt_b && !(dt_b[i] > 0 && isfinite(dt_b[i])))
      return fail(s, PTN_ERR_INVALID_ARG, "time step dt_b[%d] must be positive and finite", i);
    hi[i].T = T_b[i];
    hi[i].uoff = (int)steps;
    hi[i].xoff = (int)(steps + i);
    hi[i].pad = 0;
    hi[i].dt = dt_b ? dt_b[i] : 0.0;
    steps += T_b[i];
  }
  if (steps > s->cap_steps)
    return fail(s, PTN_ERR_INVALID_ARG, "total horizon %lld exceeds the workspace (%lld)", steps, s->cap_steps);
  *steps_out = steps;
  return PTN_OK;
}

// Choose the execution tier and launch shape of a solve of B instances (host-side
// occupancy queries only, no stream work) and set the kernel's function attributes for
// it, so that the launch itself needs no other runtime call.
// Wide batch on every co-resident CTA (tier 8): instance i gets a contiguous range of n_i
// CTAs, first CTA in hinst[i].pad, n_i >= 1 and grown one at a time for the instance with
// the most steps per warp (n_i warps no more than its steps).  Returns false (tier 4 is
// used) when the batch does not fit one CTA per instance in one cooperative launch.
static bool wide_batch_ranges(ptn_solver* s, launch_fn fn, int B, const int* T_b, int threads, LaunchPlan* p) {
  LaunchReq q{};
  int maxb = 0;
  q.tier = 8;
  q.precision = s->opt.precision;
  q.nthreads = threads;
  q.query = 1;
  q.max_blocks = &maxb;
  if (fn(q) != cudaSuccess) return false;
  if (maxb > s->grid_cap_blocks) maxb = s->grid_cap_blocks;
  if (B > maxb) return false;
  const int nw = threads / 32;
  std::vector<int> n(B, 1);
  for (int extra = maxb - B; extra > 0; extra--) {
    int best = -1;
    double key = 0.0;
    for (int i = 0; i < B; i++) {
      if ((long long)(n[i] + 1) * nw > T_b[i]) continue;  // every warp keeps a step
      const double k = (double)T_b[i] / n[i];
      if (k > key) { key = k; best = i; }
    }
    if (best < 0) break;
    n[best]++;
  }
  int c = 0;
  for (int i = 0; i < B; i++) {
    s->hinst[i].pad = c;
    c += n[i];
  }
  p->tier = 8;
  p->nthreads = threads;
  p->nblocks = c;
  return true;
}

static int plan_launch(ptn_solver* s, int method, int B, const int* T_b, long long steps, LaunchPlan* p) {
  if (method == PTN_METHOD_ADMM) {
    const UserModel* um = find_user_model(s->hprob.model);
    if (um && um->nrows > 0)
      return fail(s, PTN_ERR_INVALID_ARG, "model %d has its own constraint rows: interior point only", um->id);
  }
  launch_fn fn = pick_launcher(s->hprob.model, s->opt.precision);
  if (!fn) return fail(s, PTN_ERR_INVALID_ARG, "kernels for model %d, precision %d are not built", s->hprob.model, s->opt.precision);
  *p = LaunchPlan{};
  p->fn = fn;
  p->method = method;
  p->B = B;
  p->steps = steps;
  p->precision = s->opt.precision;
  LaunchReq q{};
  q.precision = s->opt.precision;
  // one instance: a thread-block cluster when the horizon needs 2..16 CTAs, else the
  // cooperative grid from grid_min_T on, else one CTA
  int cl_blocks = 0;
  // models with n >= 8 run the wide tier (one warp per chunk): one CTA per instance, or for
  // one instance from grid_min_T on the whole cooperative grid (tier 6); as many threads per
  // CTA as block_threads asks and shared memory allows
  const bool wide = s->n >= 8;
  int wide_threads = s->opt.block_threads;
  if (wide) {
    int fit = 0;
    q.query = 4;
    q.max_blocks = &fit;
    CK(fn(q));
    if (fit < 32) return fail(s, PTN_ERR_INVALID_ARG, "model %d: one warp's scratch does not fit in shared memory", s->hprob.model);
    if (wide_threads > fit) wide_threads = fit;
    q = LaunchReq{};
    q.precision = s->opt.precision;
  }
  if (!wide && !s->opt.sequential && B == 1 && s->opt.cluster_max_blocks >= 2) {
    const long long per = (long long)s->opt.block_threads * s->opt.grid_steps_per_thread;
    const long long need = (T_b[0] + per - 1) / per;
    if (need >= 2 && need <= s->opt.cluster_max_blocks) {
      int maxc = 0;
      q.tier = 2;
      q.nthreads = s->opt.block_threads;
      q.query = 1;
      q.max_blocks = &maxc;
      CK(fn(q));
      if (need <= maxc) cl_blocks = (int)need;
    }
  }
  const bool grid = !wide && !cl_blocks && B == 1 && s->opt.grid_min_T > 0 && T_b[0] >= s->opt.grid_min_T;
  const bool wide_grid = wide && B == 1 && s->opt.grid_min_T > 0 && T_b[0] >= s->opt.grid_min_T;
  if (s->opt.sequential && !wide) {
    p->tier = 5;
    p->nthreads = 32;
    p->nblocks = (B + 31) / 32;
  } else if (wide_grid) {
    p->tier = 6;
    p->nthreads = wide_threads;
    int maxb = 0;
    q.tier = 6;
    q.nthreads = wide_threads;
    q.query = 1;
    q.max_blocks = &maxb;
    CK(fn(q));
    const long long per = (long long)(wide_threads / 32) * s->opt.grid_steps_per_thread;
    long long want = (T_b[0] + per - 1) / per;
    int nb = want < maxb ? (int)want : maxb;
    if (nb > s->grid_cap_blocks) nb = s->grid_cap_blocks;
    if (nb < 1) return fail(s, PTN_ERR_INVALID_ARG, "no co-resident CTA for the wide grid tier");
    p->nblocks = nb;
  } else if (wide && B > 1 && s->opt.grid_min_T > 0 && wide_batch_ranges(s, fn, B, T_b, wide_threads, p)) {
    // tier 8 planned: CTA ranges per instance in hinst[].pad
  } else if (wide) {
    p->tier = 4;
    p->nthreads = wide_threads;
    p->nblocks = B;
  } else if (cl_blocks) {
    p->tier = 2;
    p->nthreads = s->opt.block_threads;
    p->nblocks = cl_blocks;
  } else if (grid) {
    p->tier = 1;
    p->nthreads = 128;
    int maxb = 0;
    q.tier = 1;
    q.nthreads = 128;
    q.query = 1;
    q.max_blocks = &maxb;
    CK(fn(q));
    int want = (int)((T_b[0] + (long long)p->nthreads * s->opt.grid_steps_per_thread - 1) /
                     ((long long)p->nthreads * s->opt.grid_steps_per_thread));
    int nb = want < maxb ? want : maxb;
    if (nb > s->grid_cap_blocks) nb = s->grid_cap_blocks;
    if (nb < 1) nb = 1;
    p->nblocks = nb;
  } else {
    p->tier = 0;
    p->nthreads = s->opt.block_threads;
    p->nblocks = B;
  }
  q = LaunchReq{};
  q.precision = p->precision;
  q.tier = p->tier;
  q.nthreads = p->nthreads;
  q.nblocks = p->nblocks;
  q.query = 2;
  CK(fn(q));
  return PTN_OK;
}

// Enqueue a planned solve on st: the kernel launch (preceded, for the cooperative grid
// tier, by the reset of its barrier counters).  No host<->device copy, no
// synchronisation, no allocation.
static int enqueue(ptn_solver* s, const LaunchPlan& p, const OptDev* dopt, const InstDev* dinst, const double* x0,
                   const double* xref, const double* u_init, double* x_out, double* u_out, double* lam_out,
                   InfoDev* dinfo, cudaStream_t st) {
  LaunchReq q{};
  q.precision = p.precision;
  q.stream = st;
  q.tier = p.tier;
  q.nthreads = p.nthreads;
  q.nblocks = p.nblocks;
  q.attrs_set = 1;
  q.w = s->w;
  q.w.xA = x_out;
  q.w.uA = u_out;
  if (lam_out) q.w.lam = lam_out;
  q.args.prob = s->dprob;
  q.args.opt = dopt;
  q.args.inst = dinst;
  q.args.x0 = x0;
  q.args.xref = xref;
  q.args.u_init = u_init;
  q.args.xtraj = s->xtraj;
  q.args.utraj = s->utraj;
  q.args.info = dinfo;
  q.args.B = p.B;
  if (p.tier == 1 || p.tier == 6 || p.tier == 8) {
    q.args.gs = s->gs;
    CK(cudaMemsetAsync(s->gs.bar, 0, 2 * sizeof(unsigned) * (p.tier == 8 ? p.B : 1), st));
    CK(cudaMemsetAsync(s->gs.err, 0, sizeof(int), st));
  }
  CK(p.fn(q));
  return PTN_OK;
}

// whether a solve of this shape gets the FP64 finish when it does not converge
static bool finish_applies(const ptn_solver* s, int method, int B) {
  return method == PTN_METHOD_IP && B == 1 && s->opt.fp64_finish && s->opt.precision != PTN_FP64 &&
         !s->opt.sequential && s->opt.update_mode == 0 && pick_launcher(s->hprob.model, PTN_FP64) != nullptr;
}

// FP64 finish of a single mixed-precision IP solve that stopped without converging (line
// search failure or iteration cap): the FP64 kernels relaunched on the same instance,
// warm-started with the controls reached (u_out serves as u_init: each thread reads its
// own steps before it writes them), from the barrier weight where the first launch
// stopped, with the initial nominal built in parallel.  On return s->hinfo[0] holds the
// finish's report and *first the first launch's; *finished tells whether it ran.
static int fp64_finish(ptn_solver* s, int method, int B, const int* T_b, long long steps, const double* x0,
                       const double* xref, double* x_out, double* u_out, double* lam_out, cudaStream_t st,
                       InfoDev* first, bool* finished) {
  *finished = false;
  const int st0 = s->hinfo[0].status;
  if (!finish_applies(s, method, B) || (st0 != ST_ENOTCONV && st0 != ST_ENUM)) return PTN_OK;
  *first = s->hinfo[0];
  const ptn_options keep = s->opt;
  s->opt.precision = PTN_FP64;
  s->opt.mu0 = first->mu > keep.mu_final ? first->mu : keep.mu_final;
  LaunchPlan p;
  int rc = plan_launch(s, method, B, T_b, steps, &p);
  if (rc == PTN_OK) {
    to_optdev(s->opt, method, s->hopt);
    s->hopt->init_parallel64 = 1;
    s->opt = keep;
    CK(cudaMemcpyAsync(s->dopt, s->hopt, sizeof(OptDev), cudaMemcpyHostToDevice, st));
    rc = enqueue(s, p, s->dopt, s->dinst, x0, xref, u_out, x_out, u_out, lam_out, s->dinfo, st);
    if (rc) return rc;
    CK(cudaMemcpyAsync(s->hinfo, s->dinfo, sizeof(InfoDev), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *finished = true;
  }
  s->opt = keep;
  return rc;
}

// adds the first launch's counters to the report of the FP64 finish
static void merge_first(const InfoDev& a, ptn_info* o) {
  o->finish_iters = o->newton_iters;
  o->newton_iters += a.newton_iters;
  o->outer_iters += a.outer_iters;
  o->ls_rejects += a.ls_rejects;
  o->factor_fails += a.factor_fails;
  o->roll_fails += a.roll_fails;
  o->roll_iters += a.roll_iters;
  o->ls_evals += a.ls_evals;
  o->exact_passes += a.exact_passes;
  for (int k = 0; k < 7; k++) o->cycles[k] += a.cyc[k];
}

static int solve_common(ptn_solver* s, int method, int B, const int* T_b, const double* x0, const double* xref,
                        const double* u_init, double* x_out, double* u_out, double* lam_out, double* z_out,
                        double* v_out, ptn_info* info, void* stream_, const double* dt_b = nullptr) {
  if (!s) return PTN_ERR_INVALID_ARG;
  s->err[0] = 0;
  cudaStream_t st = (cudaStream_t)stream_;
  if (method != PTN_METHOD_IP && method != PTN_METHOD_ADMM) return fail(s, PTN_ERR_INVALID_ARG, "bad method");
  if (!x0 || !x_out || !u_out) return fail(s, PTN_ERR_INVALID_ARG, "NULL argument");
  long long steps = 0;
  int rc = fill_instances(s, B, T_b, dt_b, s->hinst, &steps);
  if (rc) return rc;
  LaunchPlan p;
  rc = plan_launch(s, method, B, T_b, steps, &p);
  if (rc) return rc;
  to_optdev(s->opt, method, s->hopt);
  // a final barrier level that stalls on the mixed path hands over to the FP64 finish
  s->hopt->stall_exit = finish_applies(s, method, B) ? 20 : 0;
  CK(cudaMemcpyAsync(s->dinst, s->hinst, sizeof(InstDev) * B, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(s->dopt, s->hopt, sizeof(OptDev), cudaMemcpyHostToDevice, st));
  rc = enqueue(s, p, s->dopt, s->dinst, x0, xref, u_init, x_out, u_out, lam_out, s->dinfo, st);
  if (rc) return rc;
  CK(cudaMemcpyAsync(s->hinfo, s->dinfo, sizeof(InfoDev) * B, cudaMemcpyDeviceToHost, st));
  if (method == PTN_METHOD_ADMM && s->nw > 0) {
    if (z_out) CK(cudaMemcpyAsync(z_out, s->w.z, sizeof(double) * steps * s->nw, cudaMemcpyDeviceToDevice, st));
    if (v_out) CK(cudaMemcpyAsync(v_out, s->w.v, sizeof(double) * steps * s->nw, cudaMemcpyDeviceToDevice, st));
  }
  CK(cudaStreamSynchronize(st));
  InfoDev first{};
  bool finished = false;
  rc = fp64_finish(s, method, B, T_b, steps, x0, xref, x_out, u_out, lam_out, st, &first, &finished);
  if (rc) return rc;
  for (int i = 0; i < B; i++) {
    if (info) {
      from_info(s->hinfo[i], info + i);
      if (finished) merge_first(first, info + i);
    }
    if (rc == PTN_OK && s->hinfo[i].status != 0) rc = s->hinfo[i].status;
  }
  if (rc != PTN_OK && !s->err[0]) fail(s, rc, "solve finished with status %d", rc);
  return rc;
}

extern "C" int ptn_solve_ip(ptn_solver* s, const double* x0, const double* u_init, int T, double* x_out,
                            double* u_out, double* lam_out, ptn_info* info, void* stream) {
  return solve_common(s, PTN_METHOD_IP, 1, &T, x0, nullptr, u_init, x_out, u_out, lam_out, nullptr, nullptr, info,
                      stream);
}

extern "C" int ptn_solve_admm(ptn_solver* s, const double* x0, const double* u_init, int T, double* x_out,
                              double* u_out, double* lam_out, double* z_out, double* v_out, ptn_info* info,
                              void* stream) {
  return solve_common(s, PTN_METHOD_ADMM, 1, &T, x0, nullptr, u_init, x_out, u_out, lam_out, z_out, v_out, info,
                      stream);
}

extern "C" int ptn_solve_batch(ptn_solver* s, int method, int B, const int* T_b, const double* dt_b,
                               const double* x0, const double* xref, const double* u_init, double* x_out,
                               double* u_out, double* lam_out, ptn_info* info_b, void* stream) {
  return solve_common(s, method, B, T_b, x0, xref, u_init, x_out, u_out, lam_out, nullptr, nullptr, info_b,
                      stream, dt_b);
}

// The kernels write ptn_info records directly into ptn_solve_batch_async's info_dev.
static_assert(sizeof(InfoDev) == sizeof(ptn_info), "InfoDev must match ptn_info");
static_assert(offsetof(InfoDev, mu) == offsetof(ptn_info, mu), "InfoDev must match ptn_info");
static_assert(offsetof(InfoDev, r_d) == offsetof(ptn_info, r_d), "InfoDev must match ptn_info");
static_assert(offsetof(InfoDev, cyc) == offsetof(ptn_info, cycles), "InfoDev must match ptn_info");

extern "C" int ptn_batch_prepare(ptn_solver* s, int method, int B, const int* T_b, const double* dt_b,
                                 void* stream) {
  if (!s) return PTN_ERR_INVALID_ARG;
  s->err[0] = 0;
  s->plan_a_ok = false;
  cudaStream_t st = (cudaStream_t)stream;
  if (method != PTN_METHOD_IP && method != PTN_METHOD_ADMM) return fail(s, PTN_ERR_INVALID_ARG, "bad method");
  long long steps = 0;
  int rc = fill_instances(s, B, T_b, dt_b, s->hinst, &steps);
  if (rc) return rc;
  LaunchPlan p;
  rc = plan_launch(s, method, B, T_b, steps, &p);
  if (rc) return rc;
  to_optdev(s->opt, method, s->hopt);
  CK(cudaMemcpyAsync(s->dinst_a, s->hinst, sizeof(InstDev) * B, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(s->dopt_a, s->hopt, sizeof(OptDev), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  s->plan_a = p;
  s->plan_a_ok = true;
  return PTN_OK;
}

extern "C" int ptn_solve_batch_async(ptn_solver* s, const double* x0, const double* xref, const double* u_init,
                                     double* x_out, double* u_out, double* lam_out, ptn_info* info_dev,
                                     void* stream) {
  if (!s) return PTN_ERR_INVALID_ARG;
  if (!s->plan_a_ok) return fail(s, PTN_ERR_INVALID_ARG, "no batch prepared (ptn_batch_prepare)");
  if (!x0 || !x_out || !u_out) return fail(s, PTN_ERR_INVALID_ARG, "NULL argument");
  InfoDev* di = info_dev ? reinterpret_cast<InfoDev*>(info_dev) : s->dinfo;
  return enqueue(s, s->plan_a, s->dopt_a, s->dinst_a, x0, xref, u_init, x_out, u_out, lam_out, di,
                 (cudaStream_t)stream);
}

// one adjoint launch (FP64 kernels): the CTA tier, one CTA per instance, or for one long
// instance the cooperative grid, 128 threads per CTA, grid_steps_per_thread steps per
// thread as far as the co-resident CTAs allow.  T0: the horizon of the first instance.
static int launch_adjoint(ptn_solver* s, launch_fn fn, int B, int T0, const InstDev* dinst, const double* x0,
                          const double* xref, const double* x_star, const double* u_star, const AdjArgs& aa,
                          InfoDev* dinfo, cudaStream_t st, const double* xtr, const double* utr) {
  LaunchReq q{};
  q.tier = 3;
  q.precision = PTN_FP64;
  q.stream = st;
  q.w = s->w;
  q.w.xA = const_cast<double*>(x_star);  // read only: the adjoint writes no trajectory
  q.w.uA = const_cast<double*>(u_star);
  q.args.prob = s->dprob;
  q.args.opt = s->dopt;
  q.args.inst = dinst;
  q.args.x0 = x0;
  q.args.xref = xref;
  q.args.xtraj = xtr;
  q.args.utraj = utr;
  q.args.info = dinfo;
  q.args.B = B;
  q.adj = &aa;
  q.nthreads = s->opt.block_threads;
  q.nblocks = B;
  if (B == 1 && s->n < 8 && s->opt.grid_min_T > 0 && T0 >= s->opt.grid_min_T) {
    LaunchReq qq{};
    int maxb = 0;
    qq.tier = 7;
    qq.precision = PTN_FP64;
    qq.nthreads = 128;
    qq.query = 1;
    qq.max_blocks = &maxb;
    CK(fn(qq));
    const long long per = 128LL * s->opt.grid_steps_per_thread;
    long long want = (T0 + per - 1) / per;
    int nb = want < maxb ? (int)want : maxb;
    if (nb > s->grid_cap_blocks) nb = s->grid_cap_blocks;
    if (nb < 1) return fail(s, PTN_ERR_INVALID_ARG, "no co-resident CTA for the grid adjoint");
    q.tier = 7;
    q.nthreads = 128;
    q.nblocks = nb;
    q.args.gs = s->gs;
    CK(cudaMemsetAsync(s->gs.bar, 0, 2 * sizeof(unsigned), st));
    CK(cudaMemsetAsync(s->gs.err, 0, sizeof(int), st));
  }
  CK(fn(q));
  return PTN_OK;
}

extern "C" int ptn_adjoint(ptn_solver* s, int B, const int* T_b, const double* x0, const double* xref,
                           const double* x_star, const double* u_star, double mu, double gJ, const double* gx,
                           const double* gu, double* g_x0, double* g_Qd, double* g_Rd, double* g_Qfd,
                           double* g_prm, void* stream_) {
  if (!s) return PTN_ERR_INVALID_ARG;
  s->err[0] = 0;
  cudaStream_t st = (cudaStream_t)stream_;
  if (B < 1 || B > s->cap_batch) return fail(s, PTN_ERR_INVALID_ARG, "B=%d outside [1, %d]", B, s->cap_batch);
  if (!T_b || !x0 || !x_star || !u_star) return fail(s, PTN_ERR_INVALID_ARG, "NULL argument");
  if (!(mu > 0) || !isfinite(mu) || !isfinite(gJ)) return fail(s, PTN_ERR_INVALID_ARG, "mu must be positive, gJ finite");
  long long steps = 0;
  for (int i = 0; i < B; i++) {
    if (T_b[i] < 1) return fail(s, PTN_ERR_INVALID_ARG, "horizon T_b[%d]=%d must be >= 1", i, T_b[i]);
    s->hinst[i].T = T_b[i];
    s->hinst[i].uoff = (int)steps;
    s->hinst[i].xoff = (int)(steps + i);
    s->hinst[i].pad = 0;
    s->hinst[i].dt = 0.0;
    steps += T_b[i];
  }
  if (steps > s->cap_steps)
    return fail(s, PTN_ERR_INVALID_ARG, "total horizon %lld exceeds the workspace (%lld)", steps, s->cap_steps);
  if (s->hprob.model == PTN_MODEL_SYNTH_TANH)
    return fail(s, PTN_ERR_INVALID_ARG, "the adjoint is not built for the synthetic model");
  // the adjoint LQR runs in FP64 whatever the solver's precision
  launch_fn fn = pick_launcher(s->hprob.model, PTN_FP64);
  if (!fn) return fail(s, PTN_ERR_INVALID_ARG, "FP64 kernels for model %d are not built", s->hprob.model);
  CK(cudaMemcpyAsync(s->dinst, s->hinst, sizeof(InstDev) * B, cudaMemcpyHostToDevice, st));
  AdjArgs aa{};
  aa.gx = gx;
  aa.gu = gu;
  aa.qx = s->w.xB;  // the candidate-trajectory array is free outside a solve
  aa.mu = mu;
  aa.gJ = gJ;
  aa.g_x0 = g_x0; aa.g_Qd = g_Qd; aa.g_Rd = g_Rd; aa.g_Qfd = g_Qfd; aa.g_prm = g_prm;
  int rc = launch_adjoint(s, fn, B, T_b[0], s->dinst, x0, xref, x_star, u_star, aa, s->dinfo, st, s->xtraj,
                          s->utraj);
  if (rc) return rc;
  CK(cudaMemcpyAsync(s->hinfo, s->dinfo, sizeof(InfoDev) * B, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int i = 0; i < B; i++) {
    if (s->hinfo[i].status == ST_ETIMEOUT)
      return fail(s, PTN_ERR_TIMEOUT, "instance %d: a grid barrier wait expired", i);
    if (s->hinfo[i].status != 0)
      return fail(s, PTN_ERR_NUMERICAL, "instance %d: the Hessian is not positive definite on the dynamics", i);
  }
  return PTN_OK;
}

// Checkpointed adjoint of one long horizon: segments of seg_len steps, each segment's
// linearisations recomputed from the stored trajectory in each of the three sweeps of the
// AdjSeg form (co-states and value function backward, LQR states forward, multipliers and
// gradient shares backward); boundary values pass between segments in device buffers of
// (segments + 1) entries, the gradient shares are summed on the host.
extern "C" int ptn_adjoint_checkpointed(ptn_solver* s, int T, int seg_len, const double* x0, const double* xref,
                                        const double* x_star, const double* u_star, double mu, double gJ,
                                        const double* gx, const double* gu, double* g_x0, double* g_Qd,
                                        double* g_Rd, double* g_Qfd, double* g_prm, void* stream_) {
  if (!s) return PTN_ERR_INVALID_ARG;
  s->err[0] = 0;
  cudaStream_t st = (cudaStream_t)stream_;
  if (T < 1) return fail(s, PTN_ERR_INVALID_ARG, "horizon T=%d must be >= 1", T);
  if (seg_len < 1 || seg_len > s->cap_steps)
    return fail(s, PTN_ERR_INVALID_ARG, "segment length %d outside [1, %lld] (the workspace)", seg_len, s->cap_steps);
  if (!x0 || !x_star || !u_star) return fail(s, PTN_ERR_INVALID_ARG, "NULL argument");
  if (!(mu > 0) || !isfinite(mu) || !isfinite(gJ)) return fail(s, PTN_ERR_INVALID_ARG, "mu must be positive, gJ finite");
  if (s->n >= 8) return fail(s, PTN_ERR_INVALID_ARG, "the checkpointed adjoint is built for models with nx < 8");
  launch_fn fn = pick_launcher(s->hprob.model, PTN_FP64);
  if (!fn) return fail(s, PTN_ERR_INVALID_ARG, "FP64 kernels for model %d are not built", s->hprob.model);
  const int n = s->n, m = s->m;
  const int nseg = (int)(((long long)T + seg_len - 1) / seg_len);
  const int KO = 3 * n + m + PTN_MAXP;  // x0, Qd, Rd, Qfd, prm shares of one segment
  // device buffers: boundary values at the nseg + 1 segment ends, per-launch records and
  // reports, per-segment gradient shares
  const size_t nb = (size_t)nseg + 1;
  const size_t o_lam = 0, o_S = o_lam + nb * n, o_s = o_S + nb * n * n, o_dx = o_s + nb * n, o_nu = o_dx + nb * n;
  const size_t o_out = o_nu + nb * n, nd = o_out + (size_t)nseg * KO;
  const int nl = 3 * nseg;
  double* dbuf = nullptr;
  AdjSeg* dseg = nullptr;
  InstDev* dinst = nullptr;
  InfoDev* dinfo = nullptr;
  int rc = PTN_OK;
  std::vector<AdjSeg> hseg(nl);
  std::vector<InstDev> hinst(nseg);
  std::vector<InfoDev> hinfo(nl);
  std::vector<double> hout((size_t)nseg * KO), sum(KO, 0.0);
  auto cleanup = [&]() { cudaFree(dbuf); cudaFree(dseg); cudaFree(dinst); cudaFree(dinfo); };
  if (cudaMalloc(&dbuf, nd * sizeof(double)) != cudaSuccess || cudaMalloc(&dseg, nl * sizeof(AdjSeg)) != cudaSuccess ||
      cudaMalloc(&dinst, nseg * sizeof(InstDev)) != cudaSuccess ||
      cudaMalloc(&dinfo, nl * sizeof(InfoDev)) != cudaSuccess) {
    cleanup();
    return fail(s, PTN_ERR_CUDA, "device allocation for the checkpointed adjoint failed");
  }
  for (int k = 0; k < nseg; k++) {
    const long long t0 = (long long)k * seg_len, t1 = t0 + seg_len < T ? t0 + seg_len : T;
    hinst[k].T = (int)(t1 - t0);
    hinst[k].xoff = 0;
    hinst[k].uoff = 0;
    hinst[k].pad = 0;
    hinst[k].dt = 0.0;
    for (int stg = 1; stg <= 3; stg++) {
      AdjSeg& a = hseg[(size_t)(stg - 1) * nseg + k];
      a = AdjSeg{};
      a.stage = stg;
      a.first = k == 0;
      a.last = k == nseg - 1;
      a.lam_end = dbuf + o_lam + (size_t)(k + 1) * n;
      a.S_end = dbuf + o_S + (size_t)(k + 1) * n * n;
      a.s_end = dbuf + o_s + (size_t)(k + 1) * n;
      a.dx_start = dbuf + o_dx + (size_t)k * n;
      a.nu_end = dbuf + o_nu + (size_t)(k + 1) * n;
      a.lam_start = dbuf + o_lam + (size_t)k * n;
      a.S_start = dbuf + o_S + (size_t)k * n * n;
      a.s_start = dbuf + o_s + (size_t)k * n;
      a.dx_end = dbuf + o_dx + (size_t)(k + 1) * n;
      a.nu_start = dbuf + o_nu + (size_t)k * n;
    }
  }
  CK(cudaMemcpyAsync(dseg, hseg.data(), nl * sizeof(AdjSeg), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dinst, hinst.data(), nseg * sizeof(InstDev), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(dbuf, 0, nd * sizeof(double), st));
  // sweep 1 backward, sweep 2 forward, sweep 3 backward
  for (int stg = 1; stg <= 3 && rc == PTN_OK; stg++) {
    for (int j = 0; j < nseg && rc == PTN_OK; j++) {
      const int k = stg == 2 ? j : nseg - 1 - j;
      const size_t l = (size_t)(stg - 1) * nseg + k;
      const size_t xo = (size_t)k * seg_len * n, uo = (size_t)k * seg_len * m;
      AdjArgs aa{};
      aa.gx = gx ? gx + xo : nullptr;
      aa.gu = gu ? gu + uo : nullptr;
      aa.qx = s->w.xB;
      aa.mu = mu;
      aa.gJ = gJ;
      aa.seg = dseg + l;
      if (stg == 3) {
        double* o = dbuf + o_out + (size_t)k * KO;
        aa.g_x0 = o; aa.g_Qd = o + n; aa.g_Rd = o + 2 * n; aa.g_Qfd = o + 2 * n + m; aa.g_prm = o + 3 * n + m;
      }
      rc = launch_adjoint(s, fn, 1, hinst[k].T, dinst + k, x_star + xo, xref, x_star + xo, u_star + uo, aa,
                          dinfo + l, st, s->xtraj ? s->xtraj + xo : nullptr, s->utraj ? s->utraj + uo : nullptr);
    }
  }
  if (rc == PTN_OK) {
    CK(cudaMemcpyAsync(hinfo.data(), dinfo, nl * sizeof(InfoDev), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hout.data(), dbuf + o_out, (size_t)nseg * KO * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int l = 0; l < nl && rc == PTN_OK; l++) {
      if (hinfo[l].status == ST_ETIMEOUT) rc = fail(s, PTN_ERR_TIMEOUT, "a grid barrier wait expired");
      else if (hinfo[l].status != 0)
        rc = fail(s, PTN_ERR_NUMERICAL, "segment %d: the Hessian is not positive definite on the dynamics", l % nseg);
    }
  }
  if (rc == PTN_OK) {
    for (int k = 0; k < nseg; k++)
      for (int i = 0; i < KO; i++) sum[i] += hout[(size_t)k * KO + i];
    const double* h = sum.data();
    if (g_x0) CK(cudaMemcpyAsync(g_x0, h, n * sizeof(double), cudaMemcpyHostToDevice, st));
    if (g_Qd) CK(cudaMemcpyAsync(g_Qd, h + n, n * sizeof(double), cudaMemcpyHostToDevice, st));
    if (g_Rd) CK(cudaMemcpyAsync(g_Rd, h + 2 * n, m * sizeof(double), cudaMemcpyHostToDevice, st));
    if (g_Qfd) CK(cudaMemcpyAsync(g_Qfd, h + 2 * n + m, n * sizeof(double), cudaMemcpyHostToDevice, st));
    if (g_prm) CK(cudaMemcpyAsync(g_prm, h + 3 * n + m, PTN_MAXP * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  }
  cudaStreamSynchronize(st);
  cleanup();
  return rc;
}

// ---------------------------------------------------------------------------
// Allocation-free single solve.  Some callers must not reach the device allocator on
// their solve path: a fixed-rate MPC loop, where cudaMalloc / cudaFree may synchronise
// the whole device and take unbounded time, and hosts that keep no handle between calls
// (a plug-in called through a plain C function pointer).  For them the problem record,
// options, instance table, report and every workspace array of one CTA-tier solve live
// in one file-scope device array of fixed size instead of a handle's cudaMalloc'd
// workspace; everything else (kernels, launch, options) is the handle's code path.
namespace {

constexpr size_t kStaticScratchBytes = size_t(4) << 20;  // 4 MiB
constexpr int kStaticMaxContexts = 64;

struct StaticHead {
  ProbDev prob;
  OptDev opt;
  InstDev inst;
  InfoDev info;
};

// The device address of g_static_scratch belongs to the CUDA context that loaded the
// module: a non-primary context, or a primary context created again after
// cudaDeviceReset, has its own.  So the address is looked up again on every call whose
// stream is not being captured (cudaGetSymbolAddress is a host-side lookup: no stream
// work, no allocation once the module is loaded), and remembered per context for calls
// made while a capture is recording, when no module may be loaded.
struct StaticCtxAddr {
  void* ctx;
  char* base;
};
std::mutex g_static_mu;
StaticCtxAddr g_static_addr[kStaticMaxContexts];
int g_static_naddr = 0;

typedef int (*ctx_get_current_fn)(void**);  // cuCtxGetCurrent(CUcontext*)

// Current context of the calling thread (nullptr if none or the query is unavailable),
// through the driver entry point, so that the library does not link libcuda itself.
void* static_current_ctx() {
  static ctx_get_current_fn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<ctx_get_current_fn>(f);
  }();
  void* c = nullptr;
  if (!fn || fn(&c) != 0) return nullptr;
  return c;
}

int static_fail(char* err, int err_len, int code, const char* fmt, ...) {
  if (err && err_len > 0) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(err, (size_t)err_len, fmt, ap);
    va_end(ap);
  }
  return code;
}

}  // namespace

static __device__ __align__(256) char g_static_scratch[kStaticScratchBytes];

extern "C" int ptn_solve_ip_static(const ptn_problem* prob, const ptn_options* opt_in, const double* x0,
                                   const double* u_init, int T, double* x_out, double* u_out, double* lam_out,
                                   ptn_info* info, char* err, int err_len, void* stream_) {
  if (err && err_len > 0) err[0] = 0;
  if (!prob || !x0 || !x_out || !u_out) return static_fail(err, err_len, PTN_ERR_INVALID_ARG, "NULL argument");
  if (T < 1) return static_fail(err, err_len, PTN_ERR_INVALID_ARG, "horizon T=%d must be >= 1", T);
  ptn_options o;
  if (opt_in) o = *opt_in;
  else ptn_default_options(&o);
  {
    ptn_solver tmp;  // only for the option check's message; holds no device memory
    tmp.err[0] = 0;
    const int rc = check_options(&tmp, &o);
    if (rc) return static_fail(err, err_len, rc, "%s", tmp.err);
  }
  // problem record, as the handle builds it
  int nx, nu;
  if (model_dims(prob->model, &nx, &nu))
    return static_fail(err, err_len, PTN_ERR_INVALID_ARG, "unknown or unsupported model id %d", prob->model);
  if (prob->model == PTN_MODEL_SYNTH_TANH)
    return static_fail(err, err_len, PTN_ERR_INVALID_ARG,
                       "the synthetic model is not offered without a handle (its matrices live in a handle's "
                       "device memory)");
  if (o.sequential != 0)
    return static_fail(err, err_len, PTN_ERR_INVALID_ARG,
                       "the sequential-in-time baseline (option sequential) is not offered without a handle");
  if (prob->nx != nx || prob->nu != nu)
    return static_fail(err, err_len, PTN_ERR_INVALID_ARG, "model %d has nx=%d nu=%d, got %d %d", prob->model, nx, nu,
                       prob->nx, prob->nu);
  if (prob->integrator != PTN_EULER && prob->integrator != PTN_RK4)
    return static_fail(err, err_len, PTN_ERR_INVALID_ARG, "integrator must be PTN_EULER or PTN_RK4");
  if (!(prob->dt > 0) || !isfinite(prob->dt))
    return static_fail(err, err_len, PTN_ERR_INVALID_ARG, "dt must be positive");
  if (!prob->Q || !prob->R || !prob->Qf || !prob->xref || !prob->uref)
    return static_fail(err, err_len, PTN_ERR_INVALID_ARG, "Q, R, Qf, xref, uref are required");
  StaticHead h;
  memset(&h, 0, sizeof(h));
  ProbDev& P = h.prob;
  P.model = prob->model;
  P.nx = nx;
  P.nu = nu;
  P.integrator = prob->integrator;
  P.dt = prob->dt;
  for (int i = 0; i < 8; i++) P.prm[i] = prob->prm[i];
  for (int i = 0; i < nx * nx; i++) {
    if (!isfinite(prob->Q[i]) || !isfinite(prob->Qf[i]))
      return static_fail(err, err_len, PTN_ERR_INVALID_ARG, "Q/Qf not finite");
    P.Q[i] = prob->Q[i];
    P.Qf[i] = prob->Qf[i];
  }
  for (int i = 0; i < nu * nu; i++) {
    if (!isfinite(prob->R[i])) return static_fail(err, err_len, PTN_ERR_INVALID_ARG, "R not finite");
    P.R[i] = prob->R[i];
  }
  for (int i = 0; i < nx; i++) P.xref[i] = prob->xref[i];
  for (int i = 0; i < nu; i++) P.uref[i] = prob->uref[i];
  int k = 0;
  for (int i = 0; i < nx; i++) {
    if (has_bound(prob->xhi, i)) { P.row_isx[k] = 1; P.row_idx[k] = i; P.row_sgn[k] = 1.0; P.row_bnd[k] = prob->xhi[i]; k++; }
    if (has_bound(prob->xlo, i)) { P.row_isx[k] = 1; P.row_idx[k] = i; P.row_sgn[k] = -1.0; P.row_bnd[k] = prob->xlo[i]; k++; }
  }
  for (int i = 0; i < nu; i++) {
    if (has_bound(prob->uhi, i)) { P.row_isx[k] = 0; P.row_idx[k] = i; P.row_sgn[k] = 1.0; P.row_bnd[k] = prob->uhi[i]; k++; }
    if (has_bound(prob->ulo, i)) { P.row_isx[k] = 0; P.row_idx[k] = i; P.row_sgn[k] = -1.0; P.row_bnd[k] = prob->ulo[i]; k++; }
  }
  P.nw = k;
  launch_fn fn = pick_launcher(P.model, o.precision);
  if (!fn)
    return static_fail(err, err_len, PTN_ERR_INVALID_ARG, "kernels for model %d, precision %d are not built", P.model,
                       o.precision);
  // workspace layout of a one-instance handle with max_T = T, inside the static array
  const long long S = T, SB = T + 1;
  const int n = nx, m = nu, nw = k;
  size_t off = align256(sizeof(StaticHead));
  size_t o_xB = off; off = align256(off + sizeof(double) * SB * n);
  size_t o_uB = off; off = align256(off + sizeof(double) * S * m);
  size_t o_lam = off; off = align256(off + sizeof(double) * SB * n);
  size_t o_d = off; off = align256(off + sizeof(double) * S * m);
  size_t o_F64 = off; off = align256(off + sizeof(double) * S * n * n);
  size_t o_G64 = off; off = align256(off + sizeof(double) * S * n * m);
  size_t o_E = off; off = align256(off + 8 * S * n * n);
  size_t o_Gm = off; off = align256(off + 8 * S * n * m);
  size_t o_Pm = off; off = align256(off + 8 * SB * n * n);
  size_t o_Mm = off; off = align256(off + 8 * S * n * m);
  size_t o_Rm = off; off = align256(off + 8 * S * m * m);
  size_t o_Gam = off; off = align256(off + 8 * S * m * n);
  size_t o_gam = off; off = align256(off + 8 * S * m);
  size_t o_dx = off; off = align256(off + 8 * SB * n);
  size_t o_du = off; off = align256(off + 8 * S * m);
  size_t o_z = off; off = align256(off + sizeof(double) * S * (nw > 0 ? nw : 1));
  size_t o_v = off; off = align256(off + sizeof(double) * S * (nw > 0 ? nw : 1));
  // the multiplier form's arrays only when it is selected
  const bool mult = o.costate_mode != 0;
  size_t o_q = off; off = align256(off + (mult ? sizeof(double) * SB * n : 0));
  size_t o_dnu = off; off = align256(off + (mult ? sizeof(double) * SB * n : 0));
  size_t o_Sv = off; off = align256(off + (mult ? 8 * SB * n * n : 0));
  size_t o_sv = off; off = align256(off + (mult ? 8 * SB * n : 0));
  if (off > kStaticScratchBytes)
    return static_fail(err, err_len, PTN_ERR_INVALID_ARG,
                       "T=%d needs %zu bytes of static scratch for model %d; the array holds %zu bytes", T, off,
                       P.model, kStaticScratchBytes);
  // the array's address in the calling thread's current context (see g_static_addr)
  cudaStream_t st = (cudaStream_t)stream_;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t ce = cudaStreamIsCapturing(st, &cap);
  const bool capturing = ce != cudaSuccess || cap != cudaStreamCaptureStatusNone;
  if (ce != cudaSuccess) (void)cudaGetLastError();  // e.g. the legacy stream during a global capture
  char* b = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    void* a = nullptr;
    if (!capturing) {
      // also makes the device's primary context current when the thread has none
      ce = cudaGetSymbolAddress(&a, g_static_scratch);
      if (ce != cudaSuccess)
        return static_fail(err, err_len, PTN_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(ce));
    }
    void* ctx = static_current_ctx();
    int slot = -1;
    for (int i = 0; i < g_static_naddr; i++)
      if (g_static_addr[i].ctx == ctx) slot = i;
    if (!capturing) {
      if (slot < 0) {
        slot = g_static_naddr < kStaticMaxContexts ? g_static_naddr++ : kStaticMaxContexts - 1;
        g_static_addr[slot].ctx = ctx;
      }
      g_static_addr[slot].base = static_cast<char*>(a);
    } else if (slot < 0) {
      return static_fail(err, err_len, PTN_ERR_INVALID_ARG,
                         "no earlier call in this CUDA context: make one call before capturing the stream");
    }
    b = g_static_addr[slot].base;
  }
  StaticHead* dh = reinterpret_cast<StaticHead*>(b);
  to_optdev(o, PTN_METHOD_IP, &h.opt);
  h.inst.T = T;
  h.inst.xoff = 0;
  h.inst.uoff = 0;
  h.inst.pad = 0;
  // the head is copied from this stack frame in stream order; nothing else needs to be
  // initialised, because the kernel writes every workspace entry before reading it
  ce = cudaMemcpyAsync(dh, &h, offsetof(StaticHead, info), cudaMemcpyHostToDevice, st);
  if (ce != cudaSuccess) return static_fail(err, err_len, PTN_ERR_CUDA, "cudaMemcpyAsync: %s", cudaGetErrorString(ce));
  LaunchReq q{};
  q.tier = 0;
  q.precision = o.precision;
  q.nthreads = o.block_threads;
  q.nblocks = 1;
  q.stream = st;
  q.w.xA = x_out;
  q.w.uA = u_out;
  q.w.xB = (double*)(b + o_xB); q.w.uB = (double*)(b + o_uB);
  q.w.lam = lam_out ? lam_out : (double*)(b + o_lam);
  q.w.d = (double*)(b + o_d); q.w.F64 = (double*)(b + o_F64); q.w.G64 = (double*)(b + o_G64);
  q.w.E = b + o_E; q.w.Gm = b + o_Gm; q.w.Pm = b + o_Pm; q.w.Mm = b + o_Mm; q.w.Rm = b + o_Rm;
  q.w.Gam = b + o_Gam; q.w.gam = b + o_gam; q.w.dx = b + o_dx; q.w.du = b + o_du;
  q.w.z = (double*)(b + o_z); q.w.v = (double*)(b + o_v);
  if (mult) {
    q.w.q = (double*)(b + o_q); q.w.dnu = (double*)(b + o_dnu); q.w.Sv = b + o_Sv; q.w.sv = b + o_sv;
  }
  q.args.prob = &dh->prob;
  q.args.opt = &dh->opt;
  q.args.inst = &dh->inst;
  q.args.x0 = x0;
  q.args.xref = nullptr;
  q.args.u_init = u_init;
  q.args.info = &dh->info;
  q.args.B = 1;
  ce = fn(q);
  if (ce != cudaSuccess) return static_fail(err, err_len, PTN_ERR_CUDA, "launch: %s", cudaGetErrorString(ce));
  InfoDev hi;
  ce = cudaMemcpyAsync(&hi, &dh->info, sizeof(InfoDev), cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return static_fail(err, err_len, PTN_ERR_CUDA, "solve: %s", cudaGetErrorString(ce));
  if (info) from_info(hi, info);
  if (hi.status != 0) return static_fail(err, err_len, hi.status, "solve finished with status %d", hi.status);
  return PTN_OK;
}
