// ptn_solver.cuh -- the device-resident solver for one OCP instance (arXiv 2409.20027).
//
// A group of threads (one CTA, or the whole cooperative grid) runs the complete
// interior-point (Sec. II-B) or ADMM (Sec. II-C) solve.  Every Newton iteration
// (Alg. 4) is three associative scans plus a line search:
//
//   1. co-state pass (Alg. 1): FP64 Jacobians F, G and gradients at every step, suffix
//      scan of (g, F^T) elements -> lam_t, d_t (eq. co-state-eq), max |d| for the test
//   2. second-order expansion P, M, R (Sec. III-C) with lam_{t+1} . f_zz
//   3. value pass (Alg. 2): element init (eq. value-fun-elem-init), suffix scan with the
//      operator eq. value-fun-param, Bellman/feedback sweep (eq. value-fun-feedback)
//   4. state pass (Alg. 3): prefix scan of closed-loop affine maps -> dx, du, and the
//      model terms G1 = sum d^T du, G2 = 1/2 du^T H du
//   5. step acceptance: closed-loop nonlinear rollouts (multiple shooting solved by
//      Newton with the same affine prefix scan), Armijo test, Marquardt alpha update
//
// Each thread owns the steps [a, b) of a balanced partition of 0..T-1 (the last thread
// also owns the terminal state T).  Inside a chunk the thread runs the recursion
// sequentially; across chunks the group scans combine the chunk aggregates.
//
// Precision (GB300 issues FP64 at a small fraction of the FP32 rate, so FP64 is kept
// off the critical path): states, controls, co-states and gradients are stored in
// FP64.  In the mixed modes (L = float) the model is evaluated on increments
// x+ = x + dx(x, u) with dx and its Jacobian E = d dx/dx (F = I + E) in FP32 and the
// state accumulated in FP64; line-search merits are accumulated as FP32 differences
// to the nominal; the co-state scan uses an element with an FP64 vector and an FP32
// matrix increment.  Near the final convergence test the gradient is recomputed
// exactly (FP64 Jacobians).  Solves (Cholesky, (I + C J)^{-1}) run in SV.
#pragma once
#include "ptn_group.cuh"
#include "ptn_models.cuh"

namespace ptn {

// per-instance problem data copied to shared memory at kernel start
template <int N, int U>
struct ProbS {
  static constexpr int NW = 2 * (N + U);
  double Q[N * N], R[U * U], Qf[N * N], xref[N], uref[U];
  float Qs[N * N], Rs[U * U], Qfs[N * N];  // symmetrised FP32 copies Q + Q^T etc.
  double prm[PTN_MAXP];
  double sgn[NW], bnd[NW];
  int isx[NW], idx[NW];
  int nw, integ, model, Tr;  // Tr: the instance's horizon (index of the terminal target)
  double dt;
  const double *A, *B, *W;
  const float *A32, *B32, *W32;
  const double *xtr, *utr;  // time-varying targets of the instance ((Tr+1) x N, Tr x U) or null
};

// the tracking targets of step t: the instance's target trajectories when given, else the
// constant targets (the stage cost l_t of Sec. II-A may vary with t)
template <int N, int U>
__device__ __forceinline__ const double* xref_at(const ProbS<N, U>& P, int t) {
  return P.xtr ? P.xtr + (size_t)t * N : P.xref;
}
template <int N, int U>
__device__ __forceinline__ const double* uref_at(const ProbS<N, U>& P, int t) {
  return P.utr ? P.utr + (size_t)t * U : P.uref;
}

template <int N, int U>
// dt_inst > 0: the instance's own time step; the stage weights Q, R are scaled by
// dt_inst / P.dt (the same continuous-time cost at another sampling rate), Qf is not.
// xtr, utr (optional): the instance's target trajectories; T: its horizon.
__device__ void load_prob(ProbS<N, U>& S, const ProbDev& P, const double* xref_override, double dt_inst = 0.0,
                          const double* xtr = nullptr, const double* utr = nullptr, int T = 0) {
  const double sc = dt_inst > 0.0 ? dt_inst / P.dt : 1.0;
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
    S.Q[i] = sc * P.Q[i];
    S.Qf[i] = P.Qf[i];
    S.Qs[i] = float(sc * (P.Q[i] + P.Q[(i % N) * N + i / N]));
    S.Qfs[i] = float(P.Qf[i] + P.Qf[(i % N) * N + i / N]);
  }
  for (int i = threadIdx.x; i < U * U; i += blockDim.x) {
    S.R[i] = sc * P.R[i];
    S.Rs[i] = float(sc * (P.R[i] + P.R[(i % U) * U + i / U]));
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) S.xref[i] = xref_override ? xref_override[i] : P.xref[i];
  for (int i = threadIdx.x; i < U; i += blockDim.x) S.uref[i] = P.uref[i];
  for (int i = threadIdx.x; i < PTN_MAXP; i += blockDim.x) S.prm[i] = P.prm[i];
  for (int i = threadIdx.x; i < P.nw; i += blockDim.x) {
    S.sgn[i] = P.row_sgn[i]; S.bnd[i] = P.row_bnd[i]; S.isx[i] = P.row_isx[i]; S.idx[i] = P.row_idx[i];
  }
  if (threadIdx.x == 0) {
    S.nw = P.nw; S.integ = P.integrator; S.model = P.model; S.dt = dt_inst > 0.0 ? dt_inst : P.dt;
    S.A = P.A; S.B = P.B; S.W = P.W;
    S.A32 = P.A32; S.B32 = P.B32; S.W32 = P.W32;
    S.xtr = xtr; S.utr = utr; S.Tr = T;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// For large state dimensions (N >= 8) the per-element routines are called through
// out-of-line wrappers: their operands live in local memory anyway, and compiling
// them once instead of at every call site keeps build times bounded.
template <int N>
struct Big {
  static constexpr bool value = N >= 8;
};

template <class SV, int N, class L>
__device__ __noinline__ bool value_combine_ni(const Val<N, L>& a, const Val<N, L>& b, Val<N, L>& o) {
  return ValueOp<SV>()(a, b, o);
}
template <class SV>
struct ValueOpSel {
  template <int N, class L>
  __device__ __forceinline__ bool operator()(const Val<N, L>& a, const Val<N, L>& b, Val<N, L>& o) const {
    if constexpr (Big<N>::value) return value_combine_ni<SV, N, L>(a, b, o);
    else return ValueOp<SV>()(a, b, o);
  }
};
// value elements of the narrow tiers combine in row-parallel form across lane groups of
// G >= N lanes where few combinations are on the critical path (ptn_group.cuh)
template <class SV, int N, class L>
struct GroupOp<ValueOpSel<SV>, Val<N, L>> {
  static constexpr int G = N <= 2 ? 2 : (N <= 4 ? 4 : (N <= 8 ? 8 : 1));
  __device__ static bool run(const ValueOpSel<SV>& op, const Val<N, L>& a, const Val<N, L>& b, Val<N, L>& o) {
    if constexpr (G > 1) return value_combine_rows<SV, G, N, L>(a, b, o);
    else return op(a, b, o);
  }
};

template <int N, int U, class L, class SV>
__device__ __noinline__ bool value_fold_ni(const L* F, const L* G, const L* Pm, const L* Mm, const L* Rm,
                                           const double* d, double alpha, Val<N, L>& e) {
  return value_fold_step<N, U, L, SV>(F, G, Pm, Mm, Rm, d, alpha, e);
}
template <int N, int U, class L, class SV>
__device__ __forceinline__ bool value_fold_sel(const L* F, const L* G, const L* Pm, const L* Mm, const L* Rm,
                                               const double* d, double alpha, Val<N, L>& e) {
  if constexpr (Big<N>::value) return value_fold_ni<N, U, L, SV>(F, G, Pm, Mm, Rm, d, alpha, e);
  else return value_fold_step<N, U, L, SV>(F, G, Pm, Mm, Rm, d, alpha, e);
}
template <int N, int U, class L, class SV>
__device__ __noinline__ bool riccati_step_ni(const L* F, const L* G, const L* Pm, const L* Mm, const L* Rm,
                                             const double* d, double alpha, L* S, L* s, L* Gam, L* gam) {
  return riccati_step<N, U, L, SV>(F, G, Pm, Mm, Rm, d, alpha, S, s, Gam, gam);
}
template <int N, int U, class L, class SV>
__device__ __forceinline__ bool riccati_step_sel(const L* F, const L* G, const L* Pm, const L* Mm, const L* Rm,
                                                 const double* d, double alpha, L* S, L* s, L* Gam, L* gam) {
  if constexpr (Big<N>::value) return riccati_step_ni<N, U, L, SV>(F, G, Pm, Mm, Rm, d, alpha, S, s, Gam, gam);
  else return riccati_step<N, U, L, SV>(F, G, Pm, Mm, Rm, d, alpha, S, s, Gam, gam);
}
template <class M, class S>
__device__ __noinline__ void step_hess_ni(int integ, double dt, const double* p, const double* x, const double* u,
                                          const double* lam, S* Hxx, S* Hxu, S* Huu) {
  step_hess<M, S>(integ, dt, p, x, u, lam, Hxx, Hxu, Huu);
}
template <class M, class S>
__device__ __noinline__ void inc_jac_ni(int integ, double dt, const double* p, const double* x, const double* u,
                                        S* dv, S* E, S* G) {
  inc_jac<M, S>(integ, dt, p, x, u, dv, E, G);
}
template <class M, class S>
__device__ __noinline__ void step_cl_jac_ni(int integ, double dt, const double* p, const double* x,
                                            const double* u, const S* Gam, S* Fcl) {
  step_cl_jac<M, S>(integ, dt, p, x, u, Gam, Fcl);
}

// ---------------------------------------------------------------------------
// model hooks: generic models use the templated right-hand side and AD scalars;
// the synthetic model has closed-form derivatives.
template <class M>
struct MOps {
  static constexpr int N = M::NX, U = M::NU;
  template <class PS>
  __device__ static void f(const PS& P, const double* x, const double* u, double* xn) {
    step<M>(P.integ, P.dt, P.prm, x, u, xn);
  }
  template <class PS>
  __device__ static void jac(const PS& P, const double* x, const double* u, double* F, double* G) {
    step_jac<M, double>(P.integ, P.dt, P.prm, x, u, (double*)nullptr, F, G);
  }
  template <class PS, class L>
  __device__ static void hess(const PS& P, const double* x, const double* u, const double* lam, L* Hxx,
                              L* Hxu, L* Huu) {
    if constexpr (Big<N>::value) step_hess_ni<M, L>(P.integ, P.dt, P.prm, x, u, lam, Hxx, Hxu, Huu);
    else step_hess<M, L>(P.integ, P.dt, P.prm, x, u, lam, Hxx, Hxu, Huu);
  }
  template <class PS, class L>
  __device__ static void cl(const PS& P, const double* x, const double* u, const L* Gam, double* xn, L* Fcl) {
    if constexpr (Big<N>::value) step_cl_jac_ni<M, L>(P.integ, P.dt, P.prm, x, u, Gam, Fcl);
    else step_cl_jac<M, L>(P.integ, P.dt, P.prm, x, u, Gam, Fcl);
    step<M>(P.integ, P.dt, P.prm, x, u, xn);
  }
  // increment Jacobians E = d(f - x)/dx, G = df/du in scalar S (and the increment)
  template <class PS, class S>
  __device__ static void ijac(const PS& P, const double* x, const double* u, S* E, S* G, S* dv = nullptr) {
    if constexpr (Big<N>::value) inc_jac_ni<M, S>(P.integ, P.dt, P.prm, x, u, dv, E, G);
    else inc_jac<M, S>(P.integ, P.dt, P.prm, x, u, dv, E, G);
  }
  // closed-loop increment and its Jacobian in FP32
  template <class PS>
  __device__ static void icl(const PS& P, const float* x, const float* u, const float* Gam, float* dv, float* Ecl) {
    inc_cl<M, float>(P.integ, P.dt, P.prm, x, u, Gam, dv, Ecl);
  }
  template <class PS>
  __device__ static void inc32(const PS& P, const float* x, const float* u, float* dv) {
    step_inc<M, float>(P.integ, P.dt, P.prm, x, u, dv);
  }
};

// ---------------------------------------------------------------------------
// stage costs l_t + c_t (Sec. III-A) and their derivatives
struct Aug {
  int kind;       // AUG_BARRIER or AUG_ADMM
  double mu, rho;
  const double* z;  // ADMM, T x nw
  const double* v;
};

// FP32 copies of the augmentation weights for the FP32 paths
struct AugF {
  float mu, rho, irho;
  __device__ AugF(const Aug& A) : mu(float(A.mu)), rho(float(A.rho)), irho(float(1.0 / A.rho)) {}
};

// quadratic tracking term of l_t
template <int N, int U>
__device__ double track_cost(const ProbS<N, U>& P, int t, const double* x, const double* u) {
  const double *xr = xref_at(P, t), *ur = uref_at(P, t);
  double l = 0.0, e[N];
#pragma unroll
  for (int i = 0; i < N; i++) e[i] = x[i] - xr[i];
#pragma unroll
  for (int i = 0; i < N; i++) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < N; j++) s += P.Q[i * N + j] * e[j];
    l += e[i] * s;
  }
  double eu[U];
#pragma unroll
  for (int i = 0; i < U; i++) eu[i] = u[i] - ur[i];
#pragma unroll
  for (int i = 0; i < U; i++) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < U; j++) s += P.R[i * U + j] * eu[j];
    l += eu[i] * s;
  }
  return l;
}

// barrier / penalty terms c_t of the box rows; infeas set when a barrier row is not
// strictly inside
template <int N, int U>
__device__ double rows_cost(const ProbS<N, U>& P, const Aug& A, int t, const double* x, const double* u,
                            bool& infeas) {
  double l = 0.0;
  for (int r = 0; r < P.nw; r++) {
    const double zk = P.isx[r] ? x[P.idx[r]] : u[P.idx[r]];
    const double w = P.sgn[r] * (zk - P.bnd[r]);
    if (A.kind == AUG_BARRIER) {
      if (!(w < 0.0)) infeas = true;
      else l -= A.mu * log(-w);
    } else {
      const double q = w - A.z[(size_t)t * P.nw + r] + A.v[(size_t)t * P.nw + r] / A.rho;
      l += 0.5 * A.rho * q * q;
    }
  }
  return l;
}

template <int N, int U>
__device__ double stage_cost(const ProbS<N, U>& P, const Aug& A, int t, const double* x, const double* u,
                             bool& infeas, double* lplain = nullptr) {
  const double l = track_cost(P, t, x, u);
  if (lplain) *lplain = l;
  return l + rows_cost(P, A, t, x, u, infeas);
}

// gradient of l_t + c_t into lx, lu; with_track = false: of c_t alone (box rows)
template <int N, int U>
__device__ void stage_grad(const ProbS<N, U>& P, const Aug& A, int t, const double* x, const double* u,
                           double* lx, double* lu, bool with_track = true) {
  const double *xr = xref_at(P, t), *ur = uref_at(P, t);
#pragma unroll
  for (int i = 0; i < N; i++) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < N; j++) s += (P.Q[i * N + j] + P.Q[j * N + i]) * (x[j] - xr[j]);
    lx[i] = with_track ? s : 0.0;
  }
#pragma unroll
  for (int i = 0; i < U; i++) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < U; j++) s += (P.R[i * U + j] + P.R[j * U + i]) * (u[j] - ur[j]);
    lu[i] = with_track ? s : 0.0;
  }
  for (int r = 0; r < P.nw; r++) {
    const int k = P.idx[r];
    const double zk = P.isx[r] ? x[k] : u[k];
    const double w = P.sgn[r] * (zk - P.bnd[r]);
    double g1;
    if (A.kind == AUG_BARRIER) g1 = A.mu * P.sgn[r] / (-w);
    else g1 = A.rho * (w - A.z[(size_t)t * P.nw + r] + A.v[(size_t)t * P.nw + r] / A.rho) * P.sgn[r];
    if (P.isx[r]) lx[k] += g1;
    else lu[k] += g1;
  }
}

// adds the Hessians of l_t + c_t to P (N x N), R (U x U); l_xu = c_xu = 0 for box rows;
// with_track = false: of c_t alone
template <int N, int U, class L>
__device__ void stage_hess_add(const ProbS<N, U>& P, const Aug& A, const double* x, const double* u, L* Pm,
                               L* Rm, bool with_track = true) {
  if (with_track) {
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
      for (int j = 0; j < N; j++) Pm[i * N + j] += L(P.Q[i * N + j] + P.Q[j * N + i]);
#pragma unroll
    for (int i = 0; i < U; i++)
#pragma unroll
      for (int j = 0; j < U; j++) Rm[i * U + j] += L(P.R[i * U + j] + P.R[j * U + i]);
  }
  for (int r = 0; r < P.nw; r++) {
    const int k = P.idx[r];
    const double zk = P.isx[r] ? x[k] : u[k];
    const double w = P.sgn[r] * (zk - P.bnd[r]);
    const double g2 = (A.kind == AUG_BARRIER) ? A.mu / (w * w) : A.rho;
    if (P.isx[r]) Pm[k * N + k] += L(g2);
    else Rm[k * U + k] += L(g2);
  }
}

template <int N, int U>
__device__ double terminal_cost(const ProbS<N, U>& P, const double* x) {
  const double* xr = xref_at(P, P.Tr);
  double l = 0.0;
#pragma unroll
  for (int i = 0; i < N; i++) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < N; j++) s += P.Qf[i * N + j] * (x[j] - xr[j]);
    l += (x[i] - xr[i]) * s;
  }
  return l;
}


// FP32 stage gradient from e = x - xref, eu = u - uref (approximate co-state pass)
template <int N, int U>
__device__ void stage_grad32(const ProbS<N, U>& P, const Aug& A, int t, const double* x, const double* u,
                             float* lx, float* lu) {
  const double *xr = xref_at(P, t), *ur = uref_at(P, t);
  float e[N], eu[U];
#pragma unroll
  for (int i = 0; i < N; i++) e[i] = float(x[i] - xr[i]);
#pragma unroll
  for (int i = 0; i < U; i++) eu[i] = float(u[i] - ur[i]);
  mv<N, N>(P.Qs, e, lx);
  mv<U, U>(P.Rs, eu, lu);
  const AugF F(A);
  for (int r = 0; r < P.nw; r++) {
    const int k = P.idx[r];
    const double zk = P.isx[r] ? x[k] : u[k];
    const bool up = P.sgn[r] > 0.0;
    const float w = float(up ? zk - P.bnd[r] : P.bnd[r] - zk);
    float g1;
    if (A.kind == AUG_BARRIER) g1 = F.mu / (-w);
    else g1 = F.rho * (w - float(A.z[(size_t)t * P.nw + r])) + float(A.v[(size_t)t * P.nw + r]);
    if (!up) g1 = -g1;
    if (P.isx[r]) lx[k] += g1;
    else lu[k] += g1;
  }
}

// Change of the stage cost l_t + c_t between the nominal (x0, u0) and (x0 + dx, u0 + du),
// computed in FP32 from the deviations so that small differences keep their relative
// precision.  Barrier rows: -mu log(1 - dw / slack0); *infeas when a row is not
// strictly inside.
template <int N, int U>
__device__ float stage_delta(const ProbS<N, U>& P, const Aug& A, int t, const double* x0, const double* u0,
                             const float* dx, const float* du, bool& infeas) {
  const double *xr = xref_at(P, t), *ur = uref_at(P, t);
  float e[N], eu[U], qe[N], qd[N], re[U], rd[U];
#pragma unroll
  for (int i = 0; i < N; i++) e[i] = float(x0[i] - xr[i]);
#pragma unroll
  for (int i = 0; i < U; i++) eu[i] = float(u0[i] - ur[i]);
  mv<N, N>(P.Qs, e, qe);   // (Q + Q^T) e
  mv<N, N>(P.Qs, dx, qd);  // (Q + Q^T) dx
  mv<U, U>(P.Rs, eu, re);
  mv<U, U>(P.Rs, du, rd);
  float l = 0.0f;
#pragma unroll
  for (int i = 0; i < N; i++) l += dx[i] * (qe[i] + 0.5f * qd[i]);
#pragma unroll
  for (int i = 0; i < U; i++) l += du[i] * (re[i] + 0.5f * rd[i]);
  const AugF F(A);
  for (int r = 0; r < P.nw; r++) {
    const int k = P.idx[r];
    const double z0 = P.isx[r] ? x0[k] : u0[k];
    const bool up = P.sgn[r] > 0.0;
    const float w0 = float(up ? z0 - P.bnd[r] : P.bnd[r] - z0);
    const float dz = P.isx[r] ? dx[k] : du[k];
    const float dw = up ? dz : -dz;
    if (A.kind == AUG_BARRIER) {
      const float ratio = dw / (-w0);
      if (!(ratio < 1.0f)) infeas = true;
      else l -= F.mu * log1pf(-ratio);
    } else {
      const float q0 = w0 - float(A.z[(size_t)t * P.nw + r]) + float(A.v[(size_t)t * P.nw + r]) * F.irho;
      l += F.rho * dw * (q0 + 0.5f * dw);
    }
  }
  return l;
}

template <int N, int U>
__device__ float terminal_delta(const ProbS<N, U>& P, const double* x0, const float* dx) {
  const double* xr = xref_at(P, P.Tr);
  float e[N], qe[N], qd[N];
#pragma unroll
  for (int i = 0; i < N; i++) e[i] = float(x0[i] - xr[i]);
  mv<N, N>(P.Qfs, e, qe);
  mv<N, N>(P.Qfs, dx, qd);
  float l = 0.0f;
#pragma unroll
  for (int i = 0; i < N; i++) l += dx[i] * (qe[i] + 0.5f * qd[i]);
  return l;
}

// ---------------------------------------------------------------------------
// User-written terms (the general l_t, l_T and rows g_t(x, u) <= 0 of Sec. II-A, eq. ocp).
// A model may declare, as templates over the scalar type S (plain values, Dual and nested
// Dual numbers: derivatives come from forward-mode AD, as for its dynamics):
//   static constexpr bool USER_COST = true;
//   template <class S> static S stage_l(int t, const double* p, const S* x, const S* u);
//   template <class S> static S terminal_l(const double* p, const S* x);
// replacing the quadratic tracking terms, and
//   static constexpr int NC = ...;   // <= PTN_MAXC
//   template <class S> static void constraints(int t, const double* p, const S* x, const S* u, S* g);
// rows g_c <= 0 that join the box rows in the log barrier (interior point only).  The
// functions below give the costs and their derivatives for any model (the built-in terms
// when the model declares none).
template <class M, class = void>
struct user_cost {
  static constexpr bool value = false;
};
template <class M>
struct user_cost<M, std::void_t<decltype(M::USER_COST)>> {
  static constexpr bool value = M::USER_COST;
};
template <class M, class = void>
struct user_rows {
  static constexpr int value = 0;
};
template <class M>
struct user_rows<M, std::void_t<decltype(M::NC)>> {
  static constexpr int value = M::NC;
};
template <class M>
struct has_user_terms {
  static constexpr bool value = user_cost<M>::value || user_rows<M>::value > 0;
};

// value and gradient over z = (x, u) of the user stage cost (Dual numbers)
template <class M, int N, int U>
__device__ double user_l_grad(const ProbS<N, U>& P, int t, const double* x, const double* u, double* gz) {
  constexpr int K = N + U;
  using D = Dual<double, K>;
  D xd[N], ud[U];
#pragma unroll
  for (int i = 0; i < N; i++) { xd[i] = D(x[i]); xd[i].d[i] = 1.0; }
#pragma unroll
  for (int i = 0; i < U; i++) { ud[i] = D(u[i]); ud[i].d[N + i] = 1.0; }
  const D l = M::template stage_l<D>(t, P.prm, xd, ud);
#pragma unroll
  for (int k = 0; k < K; k++) gz[k] = l.d[k];
  return l.v;
}
// user rows and their Jacobian over z (Dual numbers): g (NC), J (NC x K)
template <class M, int N, int U>
__device__ void user_rows_jac(const ProbS<N, U>& P, int t, const double* x, const double* u, double* g, double* J) {
  constexpr int K = N + U, NC = user_rows<M>::value;
  using D = Dual<double, K>;
  D xd[N], ud[U], gd[NC];
#pragma unroll
  for (int i = 0; i < N; i++) { xd[i] = D(x[i]); xd[i].d[i] = 1.0; }
#pragma unroll
  for (int i = 0; i < U; i++) { ud[i] = D(u[i]); ud[i].d[N + i] = 1.0; }
  M::template constraints<D>(t, P.prm, xd, ud, gd);
#pragma unroll
  for (int c = 0; c < NC; c++) {
    g[c] = gd[c].v;
#pragma unroll
    for (int k = 0; k < K; k++) J[c * K + k] = gd[c].d[k];
  }
}
// second derivatives over z of the user stage cost (Hl, K x K) and rows (Hg, NC x K x K):
// one nested Dual evaluation per pair a <= b
template <class M, int N, int U>
__device__ void user_hess(const ProbS<N, U>& P, int t, const double* x, const double* u, double* Hl, double* Hg) {
  constexpr int K = N + U, NC = user_rows<M>::value;
  using D1 = Dual<double, 1>;
  using D2 = Dual<D1, 1>;
  for (int a = 0; a < K; a++)
    for (int b = a; b < K; b++) {
      D2 xd[N], ud[U];
#pragma unroll
      for (int i = 0; i < N; i++) {
        xd[i] = D2(D1(x[i]));
        xd[i].v.d[0] = (i == a) ? 1.0 : 0.0;
        xd[i].d[0] = D1((i == b) ? 1.0 : 0.0);
      }
#pragma unroll
      for (int i = 0; i < U; i++) {
        ud[i] = D2(D1(u[i]));
        ud[i].v.d[0] = (N + i == a) ? 1.0 : 0.0;
        ud[i].d[0] = D1((N + i == b) ? 1.0 : 0.0);
      }
      if constexpr (user_cost<M>::value) {
        const D2 l = M::template stage_l<D2>(t, P.prm, xd, ud);
        Hl[a * K + b] = Hl[b * K + a] = l.d[0].d[0];
      }
      if constexpr (NC > 0) {
        D2 gd[NC];
        M::template constraints<D2>(t, P.prm, xd, ud, gd);
#pragma unroll
        for (int c = 0; c < NC; c++) Hg[(c * K + a) * K + b] = Hg[(c * K + b) * K + a] = gd[c].d[0].d[0];
      }
    }
}

// l_t + c_t (+ the user rows' barrier)
template <class M, int N, int U>
__device__ double mstage_cost(const ProbS<N, U>& P, const Aug& A, int t, const double* x, const double* u,
                              bool& infeas, double* lplain = nullptr) {
  if constexpr (!has_user_terms<M>::value) {
    return stage_cost(P, A, t, x, u, infeas, lplain);
  } else {
    double l;
    if constexpr (user_cost<M>::value) l = M::template stage_l<double>(t, P.prm, x, u);
    else l = track_cost(P, t, x, u);
    if (lplain) *lplain = l;
    l += rows_cost(P, A, t, x, u, infeas);
    if constexpr (user_rows<M>::value > 0) {
      if (A.kind == AUG_BARRIER) {
        double g[user_rows<M>::value];
        M::template constraints<double>(t, P.prm, x, u, g);
#pragma unroll
        for (int c = 0; c < user_rows<M>::value; c++) {
          if (!(g[c] < 0.0)) infeas = true;
          else l -= A.mu * log(-g[c]);
        }
      }
    }
    return l;
  }
}

template <class M, int N, int U>
__device__ void mstage_grad(const ProbS<N, U>& P, const Aug& A, int t, const double* x, const double* u,
                            double* lx, double* lu) {
  if constexpr (!has_user_terms<M>::value) {
    stage_grad(P, A, t, x, u, lx, lu);
  } else {
    constexpr int K = N + U, NC = user_rows<M>::value;
    stage_grad(P, A, t, x, u, lx, lu, !user_cost<M>::value);
    if constexpr (user_cost<M>::value) {
      double gz[K];
      user_l_grad<M>(P, t, x, u, gz);
#pragma unroll
      for (int i = 0; i < N; i++) lx[i] += gz[i];
#pragma unroll
      for (int i = 0; i < U; i++) lu[i] += gz[N + i];
    }
    if constexpr (NC > 0) {
      if (A.kind == AUG_BARRIER) {
        double g[NC], J[NC * K];
        user_rows_jac<M>(P, t, x, u, g, J);
#pragma unroll
        for (int c = 0; c < NC; c++) {
          const double a = A.mu / (-g[c]);
#pragma unroll
          for (int i = 0; i < N; i++) lx[i] += a * J[c * K + i];
#pragma unroll
          for (int i = 0; i < U; i++) lu[i] += a * J[c * K + N + i];
        }
      }
    }
  }
}

// adds the Hessians of l_t + c_t (and the user terms, with the x-u block into Mm)
template <class M, int N, int U, class L>
__device__ void mstage_hess_add(const ProbS<N, U>& P, const Aug& A, int t, const double* x, const double* u,
                                L* Pm, L* Mm, L* Rm) {
  if constexpr (!has_user_terms<M>::value) {
    (void)t; (void)Mm;
    stage_hess_add(P, A, x, u, Pm, Rm);
  } else {
    constexpr int K = N + U, NC = user_rows<M>::value;
    stage_hess_add(P, A, x, u, Pm, Rm, !user_cost<M>::value);
    double H[K * K], Hg[NC > 0 ? NC * K * K : 1];
#pragma unroll
    for (int i = 0; i < K * K; i++) H[i] = 0.0;
    user_hess<M>(P, t, x, u, H, Hg);
    if constexpr (NC > 0) {
      if (A.kind == AUG_BARRIER) {
        double g[NC], J[NC * K];
        user_rows_jac<M>(P, t, x, u, g, J);
        // -mu log(-g): mu (grad g grad g^T / g^2 + Hess(g) / (-g))
#pragma unroll
        for (int c = 0; c < NC; c++) {
          const double a = A.mu / (-g[c]), b = A.mu / (g[c] * g[c]);
          for (int i = 0; i < K; i++)
            for (int j = 0; j < K; j++) H[i * K + j] += b * J[c * K + i] * J[c * K + j] + a * Hg[(c * K + i) * K + j];
        }
      }
    }
    for (int i = 0; i < N; i++) {
      for (int j = 0; j < N; j++) Pm[i * N + j] += L(H[i * K + j]);
      for (int j = 0; j < U; j++) Mm[i * U + j] += L(H[i * K + N + j]);
    }
    for (int i = 0; i < U; i++)
      for (int j = 0; j < U; j++) Rm[i * U + j] += L(H[(N + i) * K + N + j]);
  }
}

template <class M, int N, int U>
__device__ double mterminal_cost(const ProbS<N, U>& P, const double* x) {
  if constexpr (user_cost<M>::value) return M::template terminal_l<double>(P.prm, x);
  else return terminal_cost(P, x);
}
template <class M, int N, int U>
__device__ void mterminal_grad(const ProbS<N, U>& P, const double* xT, double* g) {
  if constexpr (user_cost<M>::value) {
    using D = Dual<double, N>;
    D xd[N];
#pragma unroll
    for (int i = 0; i < N; i++) { xd[i] = D(xT[i]); xd[i].d[i] = 1.0; }
    const D l = M::template terminal_l<D>(P.prm, xd);
#pragma unroll
    for (int i = 0; i < N; i++) g[i] = l.d[i];
  } else {
    terminal_grad(P, xT, g);
  }
}
// terminal Hessian (N x N) in L
template <class M, int N, int U, class L>
__device__ void mterminal_hess(const ProbS<N, U>& P, const double* xT, L* H) {
  if constexpr (user_cost<M>::value) {
    using D1 = Dual<double, 1>;
    using D2 = Dual<D1, 1>;
    for (int a = 0; a < N; a++)
      for (int b = a; b < N; b++) {
        D2 xd[N];
#pragma unroll
        for (int i = 0; i < N; i++) {
          xd[i] = D2(D1(xT[i]));
          xd[i].v.d[0] = (i == a) ? 1.0 : 0.0;
          xd[i].d[0] = D1((i == b) ? 1.0 : 0.0);
        }
        const D2 l = M::template terminal_l<D2>(P.prm, xd);
        H[a * N + b] = H[b * N + a] = L(l.d[0].d[0]);
      }
  } else {
#pragma unroll (N <= 8 ? N * N : 4)
    for (int i = 0; i < N * N; i++) H[i] = L(P.Qf[i] + P.Qf[(i % N) * N + i / N]);
  }
}

// FP32 forms of the mixed modes: the built-in terms in FP32, the user terms in FP64 and
// rounded (gradient; merit change from the nominal (x0, u0) by (dx, du))
template <class M, int N, int U>
__device__ void mstage_grad32(const ProbS<N, U>& P, const Aug& A, int t, const double* x, const double* u,
                              float* lx, float* lu) {
  if constexpr (!has_user_terms<M>::value) {
    stage_grad32(P, A, t, x, u, lx, lu);
  } else {
    double gx[N], gu[U];
    mstage_grad<M>(P, A, t, x, u, gx, gu);
#pragma unroll
    for (int i = 0; i < N; i++) lx[i] = float(gx[i]);
#pragma unroll
    for (int i = 0; i < U; i++) lu[i] = float(gu[i]);
  }
}
template <class M, int N, int U>
__device__ float mstage_delta(const ProbS<N, U>& P, const Aug& A, int t, const double* x0, const double* u0,
                              const float* dx, const float* du, bool& infeas) {
  if constexpr (!has_user_terms<M>::value) {
    return stage_delta(P, A, t, x0, u0, dx, du, infeas);
  } else {
    double x1[N], u1[U];
#pragma unroll
    for (int i = 0; i < N; i++) x1[i] = x0[i] + double(dx[i]);
#pragma unroll
    for (int i = 0; i < U; i++) u1[i] = u0[i] + double(du[i]);
    bool inf0 = false;
    const double l1 = mstage_cost<M>(P, A, t, x1, u1, infeas);
    const double l0 = mstage_cost<M>(P, A, t, x0, u0, inf0);
    return float(l1 - l0);
  }
}
template <class M, int N, int U>
__device__ float mterminal_delta(const ProbS<N, U>& P, const double* x0, const float* dx) {
  if constexpr (!user_cost<M>::value) {
    return terminal_delta(P, x0, dx);
  } else {
    double x1[N];
#pragma unroll
    for (int i = 0; i < N; i++) x1[i] = x0[i] + double(dx[i]);
    return float(mterminal_cost<M>(P, x1) - mterminal_cost<M>(P, x0));
  }
}

// ---------------------------------------------------------------------------
// device workspace: base pointers of the concatenated per-instance arrays
template <class L>
struct Work {
  double *xA, *uA;      // trajectory buffer A (the caller's output arrays)
  double *xB, *uB;      // trajectory buffer B (workspace)
  double *lam;          // (sum T+1) x N
  double *d;            // (sum T) x U           gradient d_t (FP64)
  double *F64, *G64;    // (sum T) x N*N, x N*U  exact Jacobian increments (FP64)
  L *E, *Gm;            // (sum T) x N*N, x N*U  LQR Jacobians: F - I and G
  L *Pm;                // (sum T+1) x N*N
  L *Mm, *Rm;           // (sum T) x N*U, x U*U
  L *Gam, *gam;         // (sum T) x U*N, x U
  L *dx, *du;           // (sum T+1) x N, (sum T) x U
  double *z, *v;        // (sum T) x nw (ADMM)
  double *q, *dnu;      // (sum T+1) x N  multiplier form: x-gradient q_t, dual step
  L *Sv, *sv;           // (sum T+1) x N*N, x N  multiplier form: LQR value S_t, s_t
};

template <class M, class L>
struct Inst {
  static constexpr int N = M::NX, U = M::NU;
  int T, a, b;
  bool last;
  const double* x0;
  double *xn, *un, *xc, *uc;  // nominal and candidate trajectories
  double *xA, *uA;            // the caller's output arrays
  double *lam, *d, *F64, *G64;
  L *E, *Gm, *Pm, *Mm, *Rm, *Gam, *gam, *dx, *du;
  double *z, *v;
  double *q, *dnu;
  L *Sv, *sv;
  double lamb[N];  // co-state at this chunk's right boundary (from the last co-state pass)

  __device__ void setup(const Work<L>& w, const InstDev& id, const double* x0_, int rank, int size, int nw) {
    T = id.T;
    a = (int)(((long long)rank * T) / size);
    b = (int)(((long long)(rank + 1) * T) / size);
    last = (rank == size - 1);
    x0 = x0_;
    const size_t xo = id.xoff, uo = id.uoff;
    xA = w.xA + xo * N; uA = w.uA + uo * U;
    xn = xA; un = uA;
    xc = w.xB + xo * N; uc = w.uB + uo * U;
    lam = w.lam + xo * N;
    d = w.d + uo * U;
    F64 = w.F64 + uo * N * N; G64 = w.G64 + uo * N * U;
    E = w.E + uo * N * N; Gm = w.Gm + uo * N * U;
    Pm = w.Pm + xo * N * N; Mm = w.Mm + uo * N * U; Rm = w.Rm + uo * U * U;
    Gam = w.Gam + uo * U * N; gam = w.gam + uo * U;
    dx = w.dx + xo * N; du = w.du + uo * U;
    z = w.z ? w.z + uo * nw : nullptr;
    v = w.v ? w.v + uo * nw : nullptr;
    q = w.q + xo * N; dnu = w.dnu + xo * N;
    Sv = w.Sv + xo * N * N; sv = w.sv + xo * N;
  }
};

// F = I + E in L
template <int N, class L>
__device__ __forceinline__ void load_F(const L* E, L* F) {
#pragma unroll (N <= 8 ? N * N : 4)
  for (int i = 0; i < N * N; i++) F[i] = E[i];
#pragma unroll
  for (int i = 0; i < N; i++) F[i * N + i] += L(1);
}

template <int N, int U>
__device__ void terminal_grad(const ProbS<N, U>& P, const double* xT, double* g) {
#pragma unroll
  for (int i = 0; i < N; i++) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < N; j++) s += (P.Qf[i * N + j] + P.Qf[j * N + i]) * (xT[j] - xref_at(P, P.Tr)[j]);
    g[i] = s;
  }
}

// ---------------------------------------------------------------------------
// pass 1: co-state suffix scan (Alg. 1).  Returns max_t |d_t|_inf (inf if not finite).
//
// Exact form (FP64): element (g, F^T) with F = I + E, E from FP64 forward-mode AD.
//
// lamT_in (optional): the co-state at t = T, where the horizon continues beyond T (a segment
// of a longer horizon); otherwise the terminal co-state of eq. co-state-final.
template <class M, class L, class Grp>
__device__ double costate_exact(Grp& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const Aug& A,
                                const double* lamT_in = nullptr) {
  constexpr int N = M::NX, U = M::NU;
  Aff<N, double> agg;
  set_identity(agg);
  double lamT[N];
  if (I.last) {
    // terminal co-state (eq. co-state-final): a constant map
    if (lamT_in) {
#pragma unroll
      for (int i = 0; i < N; i++) lamT[i] = lamT_in[i];
    } else {
      mterminal_grad<M>(P, I.xn + (size_t)I.T * N, lamT);
    }
#pragma unroll
    for (int i = 0; i < N; i++) {
      agg.v[i] = lamT[i];
#pragma unroll
      for (int j = 0; j < N; j++) agg.M[i * N + j] = 0.0;
    }
  }
  for (int t = I.b - 1; t >= I.a; t--) {
    double E[N * N], G[N * U], q[N], r[U];
    const double* x = I.xn + (size_t)t * N;
    const double* u = I.un + (size_t)t * U;
    MOps<M>::ijac(P, x, u, E, G);
#pragma unroll (N <= 8 ? N * N : 4)
    for (int i = 0; i < N * N; i++) { I.F64[(size_t)t * N * N + i] = E[i]; I.E[(size_t)t * N * N + i] = L(E[i]); }
#pragma unroll
    for (int i = 0; i < N * U; i++) { I.G64[(size_t)t * N * U + i] = G[i]; I.Gm[(size_t)t * N * U + i] = L(G[i]); }
    mstage_grad<M>(P, A, t, x, u, q, r);
    double vn[N];
    mtv<N, N>(E, agg.v, vn);  // (I + E)^T v = v + E^T v
#pragma unroll
    for (int i = 0; i < N; i++) agg.v[i] += vn[i] + q[i];
    if (!I.last) {
      double Mn[N * N];
      mtm<N, N, N>(E, agg.M, Mn);
#pragma unroll (N <= 8 ? N * N : 4)
      for (int i = 0; i < N * N; i++) agg.M[i] += Mn[i];
    }
  }
  bool ok = true;
  Aff<N, double> inc = g.scan(agg, CostateOp(), true, ok);
  double lam[N];
#pragma unroll
  for (int i = 0; i < N; i++) {
    lam[i] = I.last ? lamT[i] : inc.v[i];
    I.lamb[i] = lam[i];
    if (I.last) I.lam[(size_t)I.T * N + i] = lam[i];
  }
  double dmax = 0.0;
  for (int t = I.b - 1; t >= I.a; t--) {
    const double* x = I.xn + (size_t)t * N;
    const double* u = I.un + (size_t)t * U;
    const double* E = I.F64 + (size_t)t * N * N;
    const double* G = I.G64 + (size_t)t * N * U;
    double q[N], r[U], ln[N], dd[U];
    mstage_grad<M>(P, A, t, x, u, q, r);
    mtv<N, N>(E, lam, ln);
    mtv<N, U>(G, lam, dd);
#pragma unroll
    for (int i = 0; i < U; i++) {
      dd[i] += r[i];
      I.d[(size_t)t * U + i] = dd[i];
      const double ad = fabs(dd[i]);
      dmax = (ad <= dmax) ? dmax : (isfinite(ad) ? ad : INFINITY);
    }
#pragma unroll
    for (int i = 0; i < N; i++) {
      lam[i] += ln[i] + q[i];
      I.lam[(size_t)t * N + i] = lam[i];
    }
  }
  double red[1] = {dmax};
  g.template reduce<1>(red, 1u);
  return red[0];
}

// Mixed form (L = float): map v -> g + (I + D) v with g in FP64 and the matrix increment D
// in FP32; the increments E, G and the stage gradients come from FP32 AD.  Accurate to
// about 1e-7 relative in the gradient terms, which the final exact pass removes.
template <int N>
struct IncAff {
  float D[N * N];
  double g[N];
};
template <int N>
PTN_HD void set_identity(IncAff<N>& e) {
#pragma unroll
  for (int i = 0; i < N * N; i++) e.D[i] = 0.0f;
#pragma unroll
  for (int i = 0; i < N; i++) e.g[i] = 0.0;
}
// a earlier than b:  (I + Da)(I + Db) = I + Da + Db + Da Db,  g = ga + gb + Da gb
struct IncCostateOp {
  template <int N>
  PTN_HD bool operator()(const IncAff<N>& a, const IncAff<N>& b, IncAff<N>& o) const {
    IncAff<N> r;
    float DD[N * N], gb[N], Dg[N];
    mm<N, N, N>(a.D, b.D, DD);
#pragma unroll (N <= 8 ? N * N : 4)
    for (int i = 0; i < N * N; i++) r.D[i] = a.D[i] + b.D[i] + DD[i];
#pragma unroll
    for (int i = 0; i < N; i++) gb[i] = float(b.g[i]);
    mv<N, N>(a.D, gb, Dg);
#pragma unroll
    for (int i = 0; i < N; i++) r.g[i] = a.g[i] + b.g[i] + double(Dg[i]);
    o = r;
    return true;
  }
};

template <class M, class Grp>
__device__ double costate_mixed(Grp& g, Inst<M, float>& I, const ProbS<M::NX, M::NU>& P, const Aug& A) {
  constexpr int N = M::NX, U = M::NU;
  IncAff<N> agg;
  set_identity(agg);
  double lamT[N];
  if (I.last) {
    mterminal_grad<M>(P, I.xn + (size_t)I.T * N, lamT);
#pragma unroll
    for (int i = 0; i < N; i++) {
      agg.g[i] = lamT[i];
#pragma unroll
      for (int j = 0; j < N; j++) agg.D[i * N + j] = (i == j) ? -1.0f : 0.0f;  // constant map
    }
  }
  for (int t = I.b - 1; t >= I.a; t--) {
    float E[N * N], G[N * U], q[N], r[U], gf[N], Eg[N];
    const double* x = I.xn + (size_t)t * N;
    const double* u = I.un + (size_t)t * U;
    MOps<M>::ijac(P, x, u, E, G);
#pragma unroll (N <= 8 ? N * N : 4)
    for (int i = 0; i < N * N; i++) I.E[(size_t)t * N * N + i] = E[i];
#pragma unroll
    for (int i = 0; i < N * U; i++) I.Gm[(size_t)t * N * U + i] = G[i];
    mstage_grad32<M>(P, A, t, x, u, q, r);
#pragma unroll
    for (int i = 0; i < N; i++) gf[i] = float(agg.g[i]);
    mtv<N, N>(E, gf, Eg);
#pragma unroll
    for (int i = 0; i < N; i++) agg.g[i] += double(q[i] + Eg[i]);
    if (!I.last) {
      float ED[N * N];
      mtm<N, N, N>(E, agg.D, ED);
#pragma unroll (N <= 8 ? N : 4)
      for (int i = 0; i < N; i++)
#pragma unroll (N <= 8 ? N : 4)
        for (int j = 0; j < N; j++) agg.D[i * N + j] += E[j * N + i] + ED[i * N + j];
    }
  }
  bool ok = true;
  IncAff<N> inc = g.scan(agg, IncCostateOp(), true, ok);
  double lam[N];
#pragma unroll
  for (int i = 0; i < N; i++) {
    lam[i] = I.last ? lamT[i] : inc.g[i];
    I.lamb[i] = lam[i];
    if (I.last) I.lam[(size_t)I.T * N + i] = lam[i];
  }
  double dmax = 0.0;
  for (int t = I.b - 1; t >= I.a; t--) {
    const double* x = I.xn + (size_t)t * N;
    const double* u = I.un + (size_t)t * U;
    const float* E = I.E + (size_t)t * N * N;
    const float* G = I.Gm + (size_t)t * N * U;
    float q[N], r[U], lf[N], ln[N], dd[U];
    mstage_grad32<M>(P, A, t, x, u, q, r);
#pragma unroll
    for (int i = 0; i < N; i++) lf[i] = float(lam[i]);
    mtv<N, N>(E, lf, ln);
    mtv<N, U>(G, lf, dd);
#pragma unroll
    for (int i = 0; i < U; i++) {
      const double di = double(dd[i] + r[i]);
      I.d[(size_t)t * U + i] = di;
      const double ad = fabs(di);
      dmax = (ad <= dmax) ? dmax : (isfinite(ad) ? ad : INFINITY);
    }
#pragma unroll
    for (int i = 0; i < N; i++) {
      lam[i] += double(ln[i] + q[i]);
      I.lam[(size_t)t * N + i] = lam[i];
    }
  }
  double red[1] = {dmax};
  g.template reduce<1>(red, 1u);
  return red[0];
}

template <class M, class L, class Grp>
__device__ double costate_pass(Grp& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const Aug& A, bool exact) {
  if constexpr (std::is_same<L, float>::value) {
    if (!exact) return costate_mixed(g, I, P, A);
  }
  return costate_exact(g, I, P, A);
}

// pass 1, multiplier form (option costate_mode = 1; a variant of the method, not in the
// paper): the co-state suffix scan is replaced by multipliers nu of the dynamics, held in
// I.lam and moved to the LQR duals after each accepted step.  Both gradients of the
// Lagrangian  sum_t l_t + l_{N+1} + sum_t nu_{t+1}^T (f(x_t, u_t) - x_{t+1})  are local in t:
//   d_t = dl/du + G_t^T nu_{t+1},   q_t = dl/dx + F_t^T nu_{t+1} - nu_t   (t >= 1),
//   q_T = dl_T/dx - nu_T,   and nu_0 (x_0 is fixed) := dl/dx + F_0^T nu_1 with q_0 = 0,
// so no product of F_t^T is ever formed.  Jacobians in FP64 (forward-mode AD), stored as
// the exact co-state pass stores them.  Returns max(max |d|, max |q|) over the group.
template <class M, class L, class Grp>
__device__ __noinline__ double multiplier_pass(Grp& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const Aug& A) {
  constexpr int N = M::NX, U = M::NU;
  double rmax = 0.0;
  for (int t = I.a; t < I.b; t++) {
    double E[N * N], G[N * U], lx[N], lu[U], nv[N], Et[N], Gt[U];
    const double* x = I.xn + (size_t)t * N;
    const double* u = I.un + (size_t)t * U;
    MOps<M>::ijac(P, x, u, E, G);
#pragma unroll (N <= 8 ? N * N : 4)
    for (int i = 0; i < N * N; i++) { I.F64[(size_t)t * N * N + i] = E[i]; I.E[(size_t)t * N * N + i] = L(E[i]); }
#pragma unroll
    for (int i = 0; i < N * U; i++) { I.G64[(size_t)t * N * U + i] = G[i]; I.Gm[(size_t)t * N * U + i] = L(G[i]); }
    mstage_grad<M>(P, A, t, x, u, lx, lu);
#pragma unroll
    for (int i = 0; i < N; i++) nv[i] = I.lam[(size_t)(t + 1) * N + i];
    mtv<N, N>(E, nv, Et);  // F^T nu = nu + E^T nu
    mtv<N, U>(G, nv, Gt);
#pragma unroll
    for (int i = 0; i < U; i++) {
      const double d = lu[i] + Gt[i];
      I.d[(size_t)t * U + i] = d;
      const double ad = fabs(d);
      rmax = (ad <= rmax) ? rmax : (isfinite(ad) ? ad : INFINITY);
    }
#pragma unroll
    for (int i = 0; i < N; i++) {
      double v = lx[i] + nv[i] + Et[i];
      if (t == 0) {
        I.lam[i] = v;
        I.q[i] = 0.0;
        continue;
      }
      v -= I.lam[(size_t)t * N + i];
      I.q[(size_t)t * N + i] = v;
      const double av = fabs(v);
      rmax = (av <= rmax) ? rmax : (isfinite(av) ? av : INFINITY);
    }
  }
  if (I.last) {
    double gT[N];
    mterminal_grad<M>(P, I.xn + (size_t)I.T * N, gT);
#pragma unroll
    for (int i = 0; i < N; i++) {
      const double v = gT[i] - I.lam[(size_t)I.T * N + i];
      I.q[(size_t)I.T * N + i] = v;
      const double av = fabs(v);
      rmax = (av <= rmax) ? rmax : (isfinite(av) ? av : INFINITY);
    }
  }
  // nu at the chunk's right boundary for the second-order terms (the next chunk's first
  // multiplier, which this pass does not write unless it is nu_0 of an empty chunk)
  if (I.a < I.b) {
#pragma unroll
    for (int i = 0; i < N; i++) I.lamb[i] = I.lam[(size_t)I.b * N + i];
  }
  double red[1] = {rmax};
  g.template reduce<1>(red, 1u);
  return red[0];
}

// Multiplier form, mixed precision (L = float, before the FP64 endgame): the same terms
// with the Jacobian increments E = F - I, G and the stage gradients from FP32 AD, as the
// FP32-increment co-state pass has them.  Only the increment terms carry FP32 error:
//   q_t = (dl/dx + E^T nu_{t+1}) [FP32] + (nu_{t+1} - nu_t) [FP64].
template <class M, class Grp>
__device__ __noinline__ double multiplier_mixed(Grp& g, Inst<M, float>& I, const ProbS<M::NX, M::NU>& P,
                                                const Aug& A) {
  constexpr int N = M::NX, U = M::NU;
  double rmax = 0.0;
  for (int t = I.a; t < I.b; t++) {
    float E[N * N], G[N * U], lx[N], lu[U], nf[N], Et[N], Gt[U];
    double nv[N];
    const double* x = I.xn + (size_t)t * N;
    const double* u = I.un + (size_t)t * U;
    MOps<M>::ijac(P, x, u, E, G);
#pragma unroll (N <= 8 ? N * N : 4)
    for (int i = 0; i < N * N; i++) I.E[(size_t)t * N * N + i] = E[i];
#pragma unroll
    for (int i = 0; i < N * U; i++) I.Gm[(size_t)t * N * U + i] = G[i];
    mstage_grad32<M>(P, A, t, x, u, lx, lu);
#pragma unroll
    for (int i = 0; i < N; i++) {
      nv[i] = I.lam[(size_t)(t + 1) * N + i];
      nf[i] = float(nv[i]);
    }
    mtv<N, N>(E, nf, Et);
    mtv<N, U>(G, nf, Gt);
#pragma unroll
    for (int i = 0; i < U; i++) {
      const double d = double(lu[i] + Gt[i]);
      I.d[(size_t)t * U + i] = d;
      const double ad = fabs(d);
      rmax = (ad <= rmax) ? rmax : (isfinite(ad) ? ad : INFINITY);
    }
#pragma unroll
    for (int i = 0; i < N; i++) {
      const double inc = double(lx[i] + Et[i]);
      if (t == 0) {
        I.lam[i] = nv[i] + inc;
        I.q[i] = 0.0;
        continue;
      }
      const double v = inc + (nv[i] - I.lam[(size_t)t * N + i]);
      I.q[(size_t)t * N + i] = v;
      const double av = fabs(v);
      rmax = (av <= rmax) ? rmax : (isfinite(av) ? av : INFINITY);
    }
  }
  if (I.last) {
    double gT[N];
    mterminal_grad<M>(P, I.xn + (size_t)I.T * N, gT);
#pragma unroll
    for (int i = 0; i < N; i++) {
      const double v = gT[i] - I.lam[(size_t)I.T * N + i];
      I.q[(size_t)I.T * N + i] = v;
      const double av = fabs(v);
      rmax = (av <= rmax) ? rmax : (isfinite(av) ? av : INFINITY);
    }
  }
  if (I.a < I.b) {
#pragma unroll
    for (int i = 0; i < N; i++) I.lamb[i] = I.lam[(size_t)I.b * N + i];
  }
  double red[1] = {rmax};
  g.template reduce<1>(red, 1u);
  return red[0];
}

// Groups on which the multiplier form is built (all but the wide tier).
template <class Grp>
struct multiplier_form_ok {
  static constexpr bool value = true;
};

// pass 2: second-order expansion (Sec. III-C).  Needs lam from pass 1 (group-synced).
template <class M, class L, class Grp>
__device__ void quadratize(Grp& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const Aug& A) {
  constexpr int N = M::NX, U = M::NU;
  // lam_{t+1} for t = b-1 belongs to the next chunk; the co-state pass also wrote this
  // thread's own copy of it (lamb), so no group barrier is needed here
  for (int t = I.a; t < I.b; t++) {
    const double* x = I.xn + (size_t)t * N;
    const double* u = I.un + (size_t)t * U;
    L Pm[N * N], Mm[N * U], Rm[U * U];
    MOps<M>::hess(P, x, u, (t + 1 == I.b) ? I.lamb : I.lam + (size_t)(t + 1) * N, Pm, Mm, Rm);
    mstage_hess_add<M>(P, A, t, x, u, Pm, Mm, Rm);
#pragma unroll (N <= 8 ? N * N : 4)
    for (int i = 0; i < N * N; i++) I.Pm[(size_t)t * N * N + i] = Pm[i];
#pragma unroll
    for (int i = 0; i < N * U; i++) I.Mm[(size_t)t * N * U + i] = Mm[i];
#pragma unroll
    for (int i = 0; i < U * U; i++) I.Rm[(size_t)t * U * U + i] = Rm[i];
  }
  if (I.last) mterminal_hess<M>(P, I.xn + (size_t)I.T * N, I.Pm + (size_t)I.T * N * N);
}

// pass 3: value suffix scan (Alg. 2) + feedback sweep.  Returns true on success; false
// (group-uniform) when some R~_t, Q_t is not PD or some I + C J is singular.
//
// qx (optional, (T+1) x N, FP64): linear state terms q_t of the LQR stage costs, as the
// adjoint LQR has them; they enter as eta_t -= q_t (so s_t += q_t).  The Newton step's
// LQR has none (its state gradient is carried by the co-states).
//
// Sv, sv (optional, (T+1) x N*N and x N): receive S_t and s_t of the LQR value function
// V_t(dx) = 1/2 dx^T S_t dx + s_t^T dx (the multiplier form's dual step needs them).
//
// group_ok = false: return this thread's flag without the group reduction (the caller
// folds it into a later reduction).
template <class M, class L, class SV, class Grp>
__device__ bool value_pass(Grp& g, Inst<M, L>& I, double alpha, const double* qx = nullptr, L* Sv = nullptr,
                           L* sv = nullptr, bool group_ok = true) {
  constexpr int N = M::NX, U = M::NU;
  bool ok = true;
  Val<N, L> agg;
  set_identity(agg);
  if (I.last) {
    value_terminal<N, L>(I.Pm + (size_t)I.T * N * N, agg);
    if (qx) {
#pragma unroll
      for (int i = 0; i < N; i++) agg.eta[i] = L(-qx[(size_t)I.T * N + i]);
    }
  }
  // chunk aggregate: the steps' elements combined into it from the right, each in the
  // Woodbury form of the combination (value_fold_step: one U x U solve per step instead
  // of the element initialisation and an N x N inverse); the identity element starts a
  // chunk that does not end the horizon.  A one-member group needs no chunk aggregate:
  // its suffix is the terminal element.
  for (int t = I.b - 1; t >= I.a && g.size() > 1; t--) {
    L F[N * N];
    load_F<N>(I.E + (size_t)t * N * N, F);
    ok &= value_fold_sel<N, U, L, SV>(F, I.Gm + (size_t)t * N * U, I.Pm + (size_t)t * N * N,
                                      I.Mm + (size_t)t * N * U, I.Rm + (size_t)t * U * U, I.d + (size_t)t * U, alpha,
                                      agg);
    if (qx) {
#pragma unroll
      for (int i = 0; i < N; i++) agg.eta[i] -= L(qx[(size_t)t * N + i]);
    }
  }
  Val<N, L> inc = g.scan(agg, ValueOpSel<SV>(), true, ok);
  L S[N * N], s[N];
  if (I.last) {
#pragma unroll (N <= 8 ? N * N : 4)
    for (int i = 0; i < N * N; i++) S[i] = I.Pm[(size_t)I.T * N * N + i];
#pragma unroll
    for (int i = 0; i < N; i++) s[i] = qx ? L(qx[(size_t)I.T * N + i]) : L(0);
    if (Sv) {
#pragma unroll (N <= 8 ? N * N : 4)
      for (int i = 0; i < N * N; i++) Sv[(size_t)I.T * N * N + i] = S[i];
#pragma unroll
      for (int i = 0; i < N; i++) sv[(size_t)I.T * N + i] = s[i];
    }
  } else {
    // S_t = J_{t,<|}, s_t = -eta_{t,<|}
#pragma unroll (N <= 8 ? N * N : 4)
    for (int i = 0; i < N * N; i++) S[i] = inc.J[i];
#pragma unroll
    for (int i = 0; i < N; i++) s[i] = -inc.eta[i];
  }
  for (int t = I.b - 1; t >= I.a; t--) {
    L Gam[U * N], gam[U], F[N * N];
    load_F<N>(I.E + (size_t)t * N * N, F);
    ok &= riccati_step_sel<N, U, L, SV>(F, I.Gm + (size_t)t * N * U, I.Pm + (size_t)t * N * N,
                                        I.Mm + (size_t)t * N * U, I.Rm + (size_t)t * U * U, I.d + (size_t)t * U, alpha,
                                        S, s, Gam, gam);
    if (qx) {
#pragma unroll
      for (int i = 0; i < N; i++) s[i] += L(qx[(size_t)t * N + i]);
    }
    if (Sv) {
#pragma unroll (N <= 8 ? N * N : 4)
      for (int i = 0; i < N * N; i++) Sv[(size_t)t * N * N + i] = S[i];
#pragma unroll
      for (int i = 0; i < N; i++) sv[(size_t)t * N + i] = s[i];
    }
#pragma unroll
    for (int i = 0; i < U * N; i++) I.Gam[(size_t)t * U * N + i] = Gam[i];
#pragma unroll
    for (int i = 0; i < U; i++) I.gam[(size_t)t * U + i] = gam[i];
  }
  if (!group_ok) return ok;
  double red[1] = {ok ? 0.0 : 1.0};
  g.template reduce<1>(red, 1u);
  return red[0] == 0.0;
}

// multiplier form, per step t: g1 += q_t^T dx_t and dnu_t = S_t dx_t + s_t
template <int N, class L>
__device__ __noinline__ void mult_terms(int t, const L* dx, const double* qx, const L* Sv, const L* sv,
                                        double* dnu, double& g1) {
  const L* S = Sv + (size_t)t * N * N;
#pragma unroll
  for (int i = 0; i < N; i++) {
    g1 += qx[(size_t)t * N + i] * double(dx[i]);
    double v = double(sv[(size_t)t * N + i]);
#pragma unroll
    for (int j = 0; j < N; j++) v += double(S[i * N + j]) * double(dx[j]);
    dnu[(size_t)t * N + i] = v;
  }
}

// pass 4: state prefix scan (Alg. 3).  dx_1 = 0, du = Gam dx + gam, dx+ = F dx + G du.
// Returns the model terms G1, G2 (R without the alpha shift).
//
// Multiplier form (qx, Sv, sv, dnu given): G1 also carries sum_t q_t^T dx_t (the
// multiplier terms of the Lagrangian telescope along the linearised dynamics, so G1 stays
// the cost's directional derivative), and dnu_t = S_t dx_t + s_t is the dual step.
//
// fail (optional): a per-thread flag (0 or 1) reduced by maximum with G1, G2; on return
// the group's flag (the value pass's factorisation result, without a reduction of its own).
//
// dx_in (optional): dx at t = 0 where the horizon started before (a segment of a longer
// horizon); otherwise dx_0 = 0.
template <class M, class L, class Grp>
__device__ void state_pass(Grp& g, Inst<M, L>& I, double& G1, double& G2, const double* qx = nullptr,
                           const L* Sv = nullptr, const L* sv = nullptr, double* dnu = nullptr,
                           double* fail = nullptr, const L* dx_in = nullptr) {
  constexpr int N = M::NX, U = M::NU;
  Aff<N, L> agg;
  set_identity(agg);
  const bool first = (I.a == 0);
  if (first) {
#pragma unroll (N <= 8 ? N * N : 4)
    for (int i = 0; i < N * N; i++) agg.M[i] = L(0);  // the first element has F = 0
    if (dx_in)
#pragma unroll
      for (int i = 0; i < N; i++) agg.v[i] = dx_in[i];  // ... and maps to dx_in
  }
  for (int t = I.a; t < I.b; t++) {
    L Fc[N * N], e[N], GG[N * N];
    const L* G = I.Gm + (size_t)t * N * U;
    const L* Gam = I.Gam + (size_t)t * U * N;
    const L* gam = I.gam + (size_t)t * U;
    load_F<N>(I.E + (size_t)t * N * N, Fc);
    mm<N, U, N>(G, Gam, GG);
#pragma unroll (N <= 8 ? N * N : 4)
    for (int i = 0; i < N * N; i++) Fc[i] += GG[i];
    mv<N, U>(G, gam, e);
    L vn[N];
    mv<N, N>(Fc, agg.v, vn);
#pragma unroll
    for (int i = 0; i < N; i++) agg.v[i] = vn[i] + e[i];
    if (!first) {
      L Mn[N * N];
      mm<N, N, N>(Fc, agg.M, Mn);
#pragma unroll (N <= 8 ? N * N : 4)
      for (int i = 0; i < N * N; i++) agg.M[i] = Mn[i];
    }
  }
  bool ok = true;
  Aff<N, L> inc = g.scan(agg, StateOp(), false, ok);
  L dx[N];
#pragma unroll
  for (int i = 0; i < N; i++) dx[i] = first ? (dx_in ? dx_in[i] : L(0)) : inc.v[i];
  double g1 = 0.0, g2 = 0.0;
  for (int t = I.a; t < I.b; t++) {
    const L* G = I.Gm + (size_t)t * N * U;
    const L* Gam = I.Gam + (size_t)t * U * N;
    const L* gam = I.gam + (size_t)t * U;
    const L* Pm = I.Pm + (size_t)t * N * N;
    const L* Mm = I.Mm + (size_t)t * N * U;
    const L* Rm = I.Rm + (size_t)t * U * U;
    L du[U], Gd[U];
    mv<U, N>(Gam, dx, Gd);
#pragma unroll
    for (int i = 0; i < U; i++) {
      du[i] = Gd[i] + gam[i];
      I.du[(size_t)t * U + i] = du[i];
      g1 += I.d[(size_t)t * U + i] * double(du[i]);
    }
#pragma unroll
    for (int i = 0; i < N; i++) I.dx[(size_t)t * N + i] = dx[i];
    if (qx) mult_terms<N>(t, dx, qx, Sv, sv, dnu, g1);
    L Pd[N], Md[N], Rd[U];
    mv<N, N>(Pm, dx, Pd);
    mv<N, U>(Mm, du, Md);
    mv<U, U>(Rm, du, Rd);
    L q = L(0);
#pragma unroll
    for (int i = 0; i < N; i++) q += dx[i] * (L(0.5) * Pd[i] + Md[i]);
#pragma unroll
    for (int i = 0; i < U; i++) q += L(0.5) * du[i] * Rd[i];
    g2 += double(q);
    L Edx[N], Gdu[N];
    mv<N, N>(I.E + (size_t)t * N * N, dx, Edx);
    mv<N, U>(G, du, Gdu);
#pragma unroll
    for (int i = 0; i < N; i++) dx[i] += Edx[i] + Gdu[i];
  }
  if (I.last) {
    if (qx) mult_terms<N>(I.T, dx, qx, Sv, sv, dnu, g1);
    const L* PT = I.Pm + (size_t)I.T * N * N;
    L Pd[N];
    mv<N, N>(PT, dx, Pd);
    L q = L(0);
#pragma unroll
    for (int i = 0; i < N; i++) {
      I.dx[(size_t)I.T * N + i] = dx[i];
      q += L(0.5) * dx[i] * Pd[i];
    }
    g2 += double(q);
  }
  if (fail) {
    double red[3] = {g1, g2, *fail};
    g.template reduce<3>(red, 4u);
    G1 = red[0];
    G2 = red[1];
    *fail = red[2];
    return;
  }
  double red[2] = {g1, g2};
  g.template reduce<2>(red, 0u);
  G1 = red[0];
  G2 = red[1];
}

// ---------------------------------------------------------------------------
// Closed-loop nonlinear rollout for step size s (step acceptance; the paper's Alg. 4
// update x += dx leaves dynamics defects):
//   u_t = u^_t + s gam_t + Gam_t (x_t - x^_t),  x_{t+1} = f(x_t, u_t),  x_1 = x^_1,
// solved in parallel by multiple shooting: each thread integrates its chunk from a
// boundary guess (initially x^ + s dx), and Newton corrections of the boundary
// states come from a prefix scan of (chunk Jacobian, end defect) elements.
// Writes the candidate into (xc, uc).  Returns ROLL_OK when converged, finite and (for
// the barrier) strictly feasible, ROLL_INFEASIBLE when converged but not strictly
// feasible or with a non-finite merit, ROLL_FAIL otherwise.  *Jm receives the merit:
// the augmented cost J_c (FP64) or its change J_c(s) - J_c(0) accumulated from FP32
// stage differences (mixed modes, precise = false).
enum : int { ROLL_OK = 0, ROLL_FAIL = 1, ROLL_INFEASIBLE = 2 };

template <class M, class L, class Grp>
__device__ int rollout(Grp& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const OptDev& O, const Aug& A,
                       double s, bool precise, double* Jm, int* iters, int max_iter) {
  constexpr int N = M::NX, U = M::NU;
  const bool MIXED = std::is_same<L, float>::value && !precise;
  double X[N];
  const bool own = (I.a < I.b);
  const bool first = (I.a == 0);
#pragma unroll
  for (int i = 0; i < N; i++)
    X[i] = first ? I.x0[i] : I.xn[(size_t)I.a * N + i] + s * double(I.dx[(size_t)I.a * N + i]);
  bool conv = false, feas = true;
  double J = INFINITY;
  // right-hand boundary as this thread predicts it: initially the same guess the
  // neighbour starts from, afterwards E_j + Phi_j dX_j, which equals the neighbour's
  // corrected start X_{j+1} + dX_{j+1} (so no boundary exchange through memory)
  double Xn[N];
  if (own && !I.last) {
#pragma unroll
    for (int i = 0; i < N; i++) Xn[i] = I.xn[(size_t)I.b * N + i] + s * double(I.dx[(size_t)I.b * N + i]);
  }
  for (int it = 0; it < max_iter; it++) {
    if (own) {
#pragma unroll
      for (int i = 0; i < N; i++) I.xc[(size_t)I.a * N + i] = X[i];
    }
    double xt[N], cost = 0.0;
    bool inf = false;
    Aff<N, L> el;
    set_identity(el);
#pragma unroll
    for (int i = 0; i < N; i++) xt[i] = X[i];
    for (int t = I.a; t < I.b; t++) {
      const L* Gam = I.Gam + (size_t)t * U * N;
      const double* xh = I.xn + (size_t)t * N;
      const double* uh = I.un + (size_t)t * U;
      L Fc[N * N];
      if (MIXED) {
        float dxh[N], duf[U], Gd[U], dv[N], Ex[N * N], Gx[N * U], rx[N], ru[U], cx[N], cu[N];
#pragma unroll
        for (int i = 0; i < N; i++) dxh[i] = float(xt[i] - xh[i]);
        mv<U, N>(Gam, dxh, Gd);
        double ut[U];
#pragma unroll
        for (int i = 0; i < U; i++) {
          duf[i] = float(s) * I.gam[(size_t)t * U + i] + Gd[i];
          ut[i] = uh[i] + double(duf[i]);
          I.uc[(size_t)t * U + i] = ut[i];
          ru[i] = float(ut[i] - double(float(ut[i])));
        }
        if (t > I.a) {
#pragma unroll
          for (int i = 0; i < N; i++) I.xc[(size_t)t * N + i] = xt[i];
        }
        cost += double(mstage_delta<M>(P, A, t, xh, uh, dxh, duf, inf));
        // increment at the FP32-rounded point plus the first-order correction for the
        // rounding residuals, so the step map stays smooth far below FP32 resolution
        MOps<M>::ijac(P, xt, ut, Ex, Gx, dv);
#pragma unroll
        for (int i = 0; i < N; i++) rx[i] = float(xt[i] - double(float(xt[i])));
        mv<N, N>(Ex, rx, cx);
        mv<N, U>(Gx, ru, cu);
        // closed-loop Jacobian F + G Gam = I + E + G Gam
        mm<N, U, N>(Gx, Gam, Fc);
#pragma unroll (N <= 8 ? N * N : 4)
        for (int i = 0; i < N * N; i++) Fc[i] += Ex[i];
#pragma unroll
        for (int i = 0; i < N; i++) {
          Fc[i * N + i] += 1.0f;
          xt[i] += double(dv[i]) + double(cx[i] + cu[i]);
        }
      } else {
        double ut[U];
#pragma unroll
        for (int i = 0; i < U; i++) {
          double v = uh[i] + s * double(I.gam[(size_t)t * U + i]);
#pragma unroll
          for (int j = 0; j < N; j++) v += double(Gam[i * N + j]) * (xt[j] - xh[j]);
          ut[i] = v;
          I.uc[(size_t)t * U + i] = v;
        }
        if (t > I.a) {
#pragma unroll
          for (int i = 0; i < N; i++) I.xc[(size_t)t * N + i] = xt[i];
        }
        cost += mstage_cost<M>(P, A, t, xt, ut, inf);
        double xnext[N];
        // FP64 states and merits: the rollout reaches the FP64 dynamics to rounding and
        // FP64 merits stay noise-free.  The chunk Jacobian only steers the shooting Newton
        // and is stored in L: with L = FP32 it comes from FP32 forward-mode AD at the FP64
        // point (I + E + G Gam, E and G as the FP32-increment passes form them), which has
        // the same absolute accuracy as the FP64 AD Jacobian rounded to FP32 at a fraction
        // of the FP64 instructions; with L = FP64 from FP64 AD.
        if (first) {
          MOps<M>::f(P, xt, ut, xnext);  // the first chunk's map is constant: no Jacobian
        } else if constexpr (std::is_same<L, float>::value) {
          float Ex[N * N], Gx[N * U];
          MOps<M>::ijac(P, xt, ut, Ex, Gx);
          mm<N, U, N>(Gx, Gam, Fc);
#pragma unroll (N <= 8 ? N * N : 4)
          for (int i = 0; i < N * N; i++) Fc[i] += Ex[i];
#pragma unroll
          for (int i = 0; i < N; i++) Fc[i * N + i] += 1.0f;
          MOps<M>::f(P, xt, ut, xnext);
        } else {
          double Fd[N * N], Gd[U * N];
#pragma unroll
          for (int i = 0; i < U * N; i++) Gd[i] = double(Gam[i]);
          MOps<M>::cl(P, xt, ut, Gd, xnext, Fd);
#pragma unroll (N <= 8 ? N * N : 4)
          for (int i = 0; i < N * N; i++) Fc[i] = L(Fd[i]);
        }
#pragma unroll
        for (int i = 0; i < N; i++) xt[i] = xnext[i];
      }
      if (!first) {
        L Mn[N * N];
        mm<N, N, N>(Fc, el.M, Mn);
#pragma unroll (N <= 8 ? N * N : 4)
        for (int i = 0; i < N * N; i++) el.M[i] = Mn[i];
      }
    }
    double rmax = 0.0, xmax = 0.0;
    bool nonfin = !isfinite(cost);
    if (first) {
#pragma unroll (N <= 8 ? N * N : 4)
      for (int i = 0; i < N * N; i++) el.M[i] = L(0);
    }
    if (I.last) {
#pragma unroll
      for (int i = 0; i < N; i++) I.xc[(size_t)I.T * N + i] = xt[i];
      if (MIXED) {
        float dT[N];
#pragma unroll
        for (int i = 0; i < N; i++) dT[i] = float(xt[i] - I.xn[(size_t)I.T * N + i]);
        cost += double(mterminal_delta<M>(P, I.xn + (size_t)I.T * N, dT));
      } else {
        cost += mterminal_cost<M>(P, xt);
      }
#pragma unroll
      for (int i = 0; i < N; i++) el.v[i] = L(0);
    } else if (own) {
#pragma unroll
      for (int i = 0; i < N; i++) {
        const double r = xt[i] - Xn[i];
        el.v[i] = L(r);
        rmax = fmax(rmax, fabs(r));
      }
    }
#pragma unroll
    for (int i = 0; i < N; i++) {
      nonfin |= !isfinite(xt[i]);
      xmax = fmax(xmax, fabs(xt[i]));
    }
    if (nonfin) rmax = INFINITY;
    bool ok = true;
    double red[5] = {rmax, xmax, cost, inf ? 1.0 : 0.0, nonfin ? 1.0 : 0.0};
    // boundary corrections (prefix scan) and convergence/merit sums (max, max, sum, max,
    // max) behind one group barrier
    Aff<N, L> inc = g.scan_reduce(el, StateOp(), false, ok, red, 0x1bu);
    if (iters) *iters = it + 1;
    if (red[4] > 0.0) return ROLL_FAIL;
    const double rtol = MIXED ? fmax(O.roll_tol, 1e-8) : O.roll_tol;
    if (red[0] <= rtol * (1.0 + red[1])) {
      conv = true;
      feas = !(red[3] > 0.0);
      J = red[2];
      break;
    }
    if (own) {
      L d[N], Pd[N];
#pragma unroll
      for (int i = 0; i < N; i++) d[i] = first ? L(0) : inc.v[i];
      mv<N, N>(el.M, d, Pd);
#pragma unroll
      for (int i = 0; i < N; i++) {
        if (!first) X[i] += double(d[i]);
        if (!I.last) Xn[i] = xt[i] + double(Pd[i]);
      }
    }
  }
  *Jm = J;
  if (!conv) return ROLL_FAIL;
  return (feas && isfinite(J)) ? ROLL_OK : ROLL_INFEASIBLE;
}

// J_c of the current nominal (group sum); *infeas set when the barrier is undefined
template <class M, class L, class Grp>
__device__ double nominal_cost(Grp& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const Aug& A, bool* infeas,
                               double* Jplain) {
  constexpr int N = M::NX, U = M::NU;
  double c = 0.0, cp = 0.0;
  bool inf = false;
  for (int t = I.a; t < I.b; t++) {
    double lp;
    c += mstage_cost<M>(P, A, t, I.xn + (size_t)t * N, I.un + (size_t)t * U, inf, &lp);
    cp += lp;
  }
  if (I.last) {
    const double lt = mterminal_cost<M>(P, I.xn + (size_t)I.T * N);
    c += lt;
    cp += lt;
  }
  double red[3] = {c, cp, inf ? 1.0 : 0.0};
  g.template reduce<3>(red, 4u);
  if (infeas) *infeas = red[2] > 0.0;
  if (Jplain) *Jplain = red[1];
  return red[0];
}

// ---------------------------------------------------------------------------
// Threads that share one chunk (the wide tier's warps: every lane runs the solver logic for
// the warp's chunk): a read-modify-write of the chunk's entries visits entry i only from
// thread first() + k step(), and max() combines those threads' partial maxima, so that each
// entry is updated once.  One thread per chunk in the narrow tiers.
template <class Grp>
struct ChunkLanes {
  __device__ static int first() { return 0; }
  __device__ static int step() { return 1; }
  __device__ static double max(double v) { return v; }
};

struct NStats {
  int iters, ls_rejects, factor_fails, roll_fails, roll_iters, ls_evals, exact_passes;
  double alpha;
  long long cyc[6];
};

// The update of Alg. 4 as printed, into the candidate arrays: x_c = x^ + dx, u_c = u^ + du
// for this thread's (or warp's) chunk; x_0 is fixed (dx_0 = 0).
template <class M, class L, class Grp>
__device__ void literal_candidate(Grp& g, Inst<M, L>& I) {
  constexpr int N = M::NX, U = M::NU;
  using CL = ChunkLanes<Grp>;
  for (int t = I.a; t < I.b; t++) {
    for (int i = CL::first(); i < N; i += CL::step())
      I.xc[(size_t)t * N + i] = I.xn[(size_t)t * N + i] + double(I.dx[(size_t)t * N + i]);
    for (int i = CL::first(); i < U; i += CL::step())
      I.uc[(size_t)t * U + i] = I.un[(size_t)t * U + i] + double(I.du[(size_t)t * U + i]);
  }
  if (I.last)
    for (int i = CL::first(); i < N; i += CL::step())
      I.xc[(size_t)I.T * N + i] = I.xn[(size_t)I.T * N + i] + double(I.dx[(size_t)I.T * N + i]);
  g.sync();
}

// Groups whose passes are always exact (FP64 gradients, rollouts and merits whatever the
// LQR precision); the Newton loop then skips the FP32-increment phase and its endgame.
template <class Grp>
struct exact_only {
  static constexpr bool value = false;
};

// Newton iterations (Alg. 4) on the augmented sub-problem until max |d| <= tol.
// Step acceptance and the alpha rule are the same readings as the CPU oracle's.  In the
// mixed modes the gradient comes from the FP32-increment co-state pass until, at the
// final tolerance, it falls below polish * tol; from then on the exact FP64 pass decides.
template <class M, class L, class SV, class Grp>
//
// sticky_exact (optional): once a call switches to the exact FP64 path it sets the flag,
// and later calls start on that path (ADMM: every sub-problem is warm-started next to its
// solution, where the FP32-increment phase only adds iterations before the endgame).
__device__ int newton_solve(Grp& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const OptDev& O, const Aug& A,
                            double tol, bool final_level, NStats& st, double* rfinal, bool* sticky_exact = nullptr) {
  constexpr int N = M::NX;
  constexpr bool MIXED = std::is_same<L, float>::value && !exact_only<Grp>::value;
  constexpr bool CAN_MULT = multiplier_form_ok<Grp>::value;
  const bool MULT = CAN_MULT && O.costate_mode != 0;
  // first-order terms: the co-state scan, or the multiplier form's local gradients
  auto first_order = [&](bool ex) -> double {
    if constexpr (CAN_MULT) {
      if (MULT) {
        if constexpr (std::is_same<L, float>::value) {
          if (!ex) return multiplier_mixed(g, I, P, A);
        }
        return multiplier_pass(g, I, P, A);
      }
    }
    return costate_pass(g, I, P, A, ex);
  };
  bool inf;
  double J0 = nominal_cost(g, I, P, A, &inf, nullptr);
  int rc = ST_ENOTCONV;
  double r = INFINITY;
  bool exact = !MIXED || (sticky_exact && *sticky_exact);  // FP64 gradients, rollouts and merits
  if (MULT && O.costate_mode == 2) {
    // hybrid multiplier form: this sub-problem's multipliers start from the co-states of
    // the scan (written to I.lam; the pass ends with a group reduction, so they are
    // visible to the neighbouring chunks), multiplier steps take over from there
    costate_pass(g, I, P, A, exact);
  }
  bool stalled = false;  // the FP32-increment phase ran alpha past alpha_max
  // stall exit (O.stall_exit > 0, set when an FP64 finish follows on the host): on the
  // exact path of the final level, stop once stall_exit iterations have not halved max|d|
  double r_ref = INFINITY;
  int it_ref = 0;
  for (int it = 0; it <= O.max_newton; it++) {
    if (g.dead()) return ST_ETIMEOUT;
    long long c0 = clock64();
    r = first_order(exact);
    const bool near = r <= O.polish * tol;
    if (MIXED && !exact && (stalled || (it >= O.polish_after && (final_level || near)) || (final_level && near))) {
      // endgame: below the FP32 noise floor of gradients and merits, switch to FP64: at the
      // final level near its tolerance or after polish_after iterations; at an intermediate
      // level after polish_after iterations that end near its tolerance (a level whose
      // tolerance lies below the floor of a coarsely sampled instance hovers there).
      // First re-project the nominal onto the FP64 dynamics (one exact rollout with
      // s = 0 under the last feedback), so that FP64 merits compare like with like.
      exact = true;
      if (sticky_exact) *sticky_exact = true;
      st.exact_passes++;
      double mproj;
      int ri = 0;
      if (rollout(g, I, P, O, A, 0.0, true, &mproj, &ri, O.roll_max_iter) != ROLL_FAIL) {
        double* t1 = I.xn; I.xn = I.xc; I.xc = t1;
        double* t2 = I.un; I.un = I.uc; I.uc = t2;
      }
      st.roll_iters += ri;
      r = first_order(true);
      J0 = nominal_cost(g, I, P, A, &inf, nullptr);
    } else if (exact && MIXED) {
      st.exact_passes++;
    }
    long long c1 = clock64();
    st.cyc[0] += c1 - c0;
    if (r <= tol) { rc = ST_OK; break; }
    if (it == O.max_newton || !isfinite(r) || !isfinite(J0)) break;
    if (MIXED && exact && final_level && O.stall_exit > 0) {
      if (r < 0.5 * r_ref) { r_ref = r; it_ref = it; }
      else if (it - it_ref >= O.stall_exit) break;  // ST_ENOTCONV: the FP64 finish takes over
    }
    st.iters++;
    quadratize(g, I, P, A);
    long long c2 = clock64();
    st.cyc[1] += c2 - c1;
    double G1, G2;
    long long c4;
    if constexpr (CAN_MULT) {
      // value pass, then the state pass, whose group reduction also carries the value
      // pass's factorisation flag (one group reduction fewer per step); a failure anywhere
      // redoes both with a larger alpha (the state pass's results are then discarded)
      for (;;) {
        const bool okl = value_pass<M, L, SV>(g, I, st.alpha, MULT ? I.q : nullptr, MULT ? I.Sv : nullptr,
                                              MULT ? I.sv : nullptr, false);
        const long long c3 = clock64();
        st.cyc[2] += c3 - c2;
        double fail = okl ? 0.0 : 1.0;
        state_pass(g, I, G1, G2, MULT ? I.q : nullptr, MULT ? I.Sv : nullptr, MULT ? I.sv : nullptr,
                   MULT ? I.dnu : nullptr, &fail);
        c4 = clock64();
        st.cyc[3] += c4 - c3;
        if (fail == 0.0) break;
        st.factor_fails++;
        st.alpha = fmax(10.0 * st.alpha, 1e-8);
        if (st.alpha > O.alpha_max || g.dead()) { *rfinal = r; return g.dead() ? ST_ETIMEOUT : ST_ENUM; }
        c2 = clock64();
      }
    } else {
      while (!value_pass<M, L, SV>(g, I, st.alpha)) {
        st.factor_fails++;
        st.alpha = fmax(10.0 * st.alpha, 1e-8);
        if (st.alpha > O.alpha_max || g.dead()) { *rfinal = r; return g.dead() ? ST_ETIMEOUT : ST_ENUM; }
      }
      const long long c3 = clock64();
      st.cyc[2] += c3 - c2;
      state_pass(g, I, G1, G2);
      c4 = clock64();
      st.cyc[3] += c4 - c3;
    }
    bool accepted = false;
    double s = 1.0, Js = INFINITY, dJ = INFINITY;
    if (O.update_mode == 1) {
      // Alg. 4 as printed: candidate x^ + dx, u^ + du (no rollout), taken whenever its FP64
      // cost is finite; the linearised dynamics leave defects of second order
      literal_candidate(g, I);
      double* t1 = I.xn; I.xn = I.xc; I.xc = t1;
      double* t2 = I.un; I.un = I.uc; I.uc = t2;
      bool infl;
      const double Jl = nominal_cost(g, I, P, A, &infl, nullptr);
      t1 = I.xn; I.xn = I.xc; I.xc = t1;
      t2 = I.un; I.un = I.uc; I.uc = t2;
      st.ls_evals++;
      accepted = !infl && isfinite(Jl);
      Js = Jl;
      dJ = Jl - J0;
    } else {
      for (int k = 0; k < O.ls_count; k++, s *= O.ls_beta) {
        int ri = 0;
        double m;
        const bool okr = rollout(g, I, P, O, A, s, exact, &m, &ri, O.roll_max_iter) == ROLL_OK;
        st.ls_evals++;
        st.roll_iters += ri;
        if (!okr) { st.roll_fails++; continue; }
        const bool diff = MIXED && !exact;  // merits returned as FP32-accumulated differences
        dJ = diff ? m : m - J0;
        Js = diff ? J0 + m : m;
        const double eps = diff ? O.armijo_eps32 : O.armijo_eps;
        if (dJ <= O.armijo_c1 * s * G1 + eps * (1.0 + fabs(J0))) { accepted = true; break; }
      }
    }
    st.cyc[4] += clock64() - c4;
    if (accepted) {
      const double pred = -(s * G1 + s * s * G2);
      const double rho = pred > 0.0 ? -dJ / pred : 0.0;
      if (rho > 0.75) st.alpha /= 3.0;
      else if (rho < 0.25) st.alpha *= 2.0;
      st.alpha = fmin(fmax(st.alpha, O.alpha_min), O.alpha_max);
      double* t1 = I.xn; I.xn = I.xc; I.xc = t1;
      double* t2 = I.un; I.un = I.uc; I.uc = t2;
      J0 = Js;
      if constexpr (CAN_MULT) {
        if (MULT) {
          // multipliers := the duals of the LQR's linearised dynamics (full dual step
          // whatever s); the next pass reads the neighbouring chunk's nu, hence the sync
          using CL = ChunkLanes<Grp>;
          for (int t = I.a; t < I.b; t++)
            for (int i = CL::first(); i < N; i += CL::step()) I.lam[(size_t)t * N + i] += I.dnu[(size_t)t * N + i];
          if (I.last)
            for (int i = CL::first(); i < N; i += CL::step()) I.lam[(size_t)I.T * N + i] += I.dnu[(size_t)I.T * N + i];
          g.sync();
        }
      }
    } else {
      st.ls_rejects++;
      st.alpha *= 10.0;
      if (st.alpha > O.alpha_max) {
        if (MIXED && !exact) {
          // no descent found with FP32-increment gradients and merits: continue this
          // level on the exact FP64 path from alpha0 instead of giving up
          stalled = true;
          st.alpha = O.alpha0;
          continue;
        }
        rc = ST_ENUM;
        break;
      }
    }
  }
  *rfinal = r;
  return rc;
}

// final residuals: r_stat (max |d|, exact pass), r_dyn, r_feas, J, J_c; lam of the final point
// (multiplier form: r_stat = max(|d|, |q|), the Lagrangian's gradients, and lam = nu)
template <class M, class L, class Grp>
__device__ void residuals(Grp& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const Aug& A, InfoDev& info,
                          bool mult = false) {
  constexpr int N = M::NX, U = M::NU;
  if constexpr (multiplier_form_ok<Grp>::value) {
    info.r_stat = mult ? multiplier_pass(g, I, P, A) : costate_pass(g, I, P, A, true);
  } else {
    info.r_stat = costate_pass(g, I, P, A, true);
  }
  double rd = 0.0, rf = -INFINITY;
  for (int t = I.a; t < I.b; t++) {
    double xn[N];
    MOps<M>::f(P, I.xn + (size_t)t * N, I.un + (size_t)t * U, xn);
#pragma unroll
    for (int i = 0; i < N; i++) {
      const double e = fabs(I.xn[(size_t)(t + 1) * N + i] - xn[i]);
      rd = (e <= rd) ? rd : (isfinite(e) ? e : INFINITY);
    }
    for (int r = 0; r < P.nw; r++) {
      const double zk = P.isx[r] ? I.xn[(size_t)t * N + P.idx[r]] : I.un[(size_t)t * U + P.idx[r]];
      rf = fmax(rf, P.sgn[r] * (zk - P.bnd[r]));
    }
    if constexpr (user_rows<M>::value > 0) {
      double gr[user_rows<M>::value];
      M::template constraints<double>(t, P.prm, I.xn + (size_t)t * N, I.un + (size_t)t * U, gr);
#pragma unroll
      for (int c = 0; c < user_rows<M>::value; c++) rf = fmax(rf, gr[c]);
    }
  }
  double red[2] = {rd, rf};
  g.template reduce<2>(red, 3u);
  info.r_dyn = red[0];
  info.r_feas = fmax(red[1], 0.0);
  bool inf;
  double Jp;
  info.J_c = nominal_cost(g, I, P, A, &inf, &Jp);
  info.J = Jp;
}

// copy the nominal into the caller's arrays if it lives in the workspace buffer
template <class M, class L, class Grp>
__device__ void finalize_traj(Grp& g, Inst<M, L>& I) {
  constexpr int N = M::NX, U = M::NU;
  if (I.xn != I.xA) {
    for (int t = I.a; t < I.b; t++) {
#pragma unroll
      for (int i = 0; i < N; i++) I.xA[(size_t)t * N + i] = I.xn[(size_t)t * N + i];
#pragma unroll
      for (int i = 0; i < U; i++) I.uA[(size_t)t * U + i] = I.un[(size_t)t * U + i];
    }
    if (I.last)
#pragma unroll
      for (int i = 0; i < N; i++) I.xA[(size_t)I.T * N + i] = I.xn[(size_t)I.T * N + i];
  }
  g.sync();
}

// Error-free sum of two floats (Knuth): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// initial nominal: x = rollout(x0, u_init) (open loop), integrated sequentially by the
// group's first thread.  In the mixed modes the state is carried as an unevaluated sum
// of two floats (hi + lo, about 48 significant bits) updated by FP32 increments, so the
// serial chain stays on the FP32 pipes; FP64 mode integrates in FP64.
template <class M, class L, class Grp>
__device__ void initial_rollout(Grp& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P) {
  constexpr int N = M::NX, U = M::NU;
  if (g.rank() == 0) {
    if constexpr (std::is_same<L, float>::value) {
      float hi[N], lo[N], un_next[U];
#pragma unroll
      for (int i = 0; i < N; i++) {
        hi[i] = float(I.x0[i]);
        lo[i] = float(I.x0[i] - double(hi[i]));
        I.xn[i] = I.x0[i];
      }
#pragma unroll
      for (int i = 0; i < U; i++) un_next[i] = float(I.un[i]);
      for (int t = 0; t < I.T; t++) {
        float uf[U], dv[N], xf[N];
#pragma unroll
        for (int i = 0; i < U; i++) {
          uf[i] = un_next[i];
          if (t + 1 < I.T) un_next[i] = float(I.un[(size_t)(t + 1) * U + i]);
        }
#pragma unroll
        for (int i = 0; i < N; i++) xf[i] = hi[i] + lo[i];
        MOps<M>::inc32(P, xf, uf, dv);
#pragma unroll
        for (int i = 0; i < N; i++) {
          float sh, se;
          two_sum(hi[i], dv[i], sh, se);
          se += lo[i];
          hi[i] = sh + se;
          lo[i] = se - (hi[i] - sh);
          I.xn[(size_t)(t + 1) * N + i] = double(hi[i]) + double(lo[i]);
        }
      }
    } else {
      double x[N];
#pragma unroll
      for (int i = 0; i < N; i++) { x[i] = I.x0[i]; I.xn[i] = x[i]; }
      for (int t = 0; t < I.T; t++) {
        double xn[N];
        MOps<M>::f(P, x, I.un + (size_t)t * U, xn);
#pragma unroll
        for (int i = 0; i < N; i++) { x[i] = xn[i]; I.xn[(size_t)(t + 1) * N + i] = x[i]; }
      }
    }
  }
  g.sync();
}

// Initial nominal in parallel (FP32 modes, and FP64 when O.init_parallel64 is set: the
// FP64 finish of a mixed-precision solve; groups of >= 256 threads, fine time steps):
// the same open-loop trajectory x = rollout(x0, u_init), computed as
//   1. a coarse pass by the group's first thread with steps K dt (K <= 32, K dt <= 2.5 ms;
//      controls held), which gives states at t = 0, K, 2K, ...;
//   2. each thread's guess of its chunk start, integrated in fine steps (< K) from the
//      coarse state before it;
//   3. the multiple-shooting rollout with s = 0 and no feedback, which corrects the
//      guesses onto the fine trajectory (same dynamics and tolerance as later rollouts).
// Returns false (group-uniform) when not applicable (FP64 unless asked, small groups,
// coarse steps, ADMM) or when the shooting does not converge; the caller then integrates
// sequentially.
template <class M, class L, class Grp>
__device__ bool initial_rollout_parallel(Grp& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const OptDev& O,
                                         int* iters) {
  {
    constexpr int N = M::NX, U = M::NU;
    if (!std::is_same<L, float>::value && !O.init_parallel64) return false;
    int K = (int)(0.0025 / P.dt);
    K = K > 32 ? 32 : K;
    if (K < 2 || g.size() < 256 || O.method != 0) return false;  // IP only (barrier merit)
    if (g.rank() == 0) {
      double x[N];
#pragma unroll
      for (int i = 0; i < N; i++) { x[i] = I.x0[i]; I.xn[i] = x[i]; }
      for (int c = 0; c + K <= I.T; c += K) {
        float xf[N], uf[U], dv[N];
#pragma unroll
        for (int i = 0; i < N; i++) xf[i] = float(x[i]);
#pragma unroll
        for (int i = 0; i < U; i++) uf[i] = float(I.un[(size_t)c * U + i]);
        step_inc<M, float, double>(P.integ, K * P.dt, P.prm, xf, uf, dv);
#pragma unroll
        for (int i = 0; i < N; i++) {
          x[i] += double(dv[i]);
          I.xn[(size_t)(c + K) * N + i] = x[i];
        }
      }
    }
    g.sync();
    // chunk-start guesses (threads write only their own start; coarse points are read)
    if (I.a < I.b) {
      const int c = (I.a / K) * K;
      if (c != I.a) {
        double x[N];
#pragma unroll
        for (int i = 0; i < N; i++) x[i] = I.xn[(size_t)c * N + i];
        for (int t = c; t < I.a; t++) {
          float xf[N], uf[U], dv[N];
#pragma unroll
          for (int i = 0; i < N; i++) xf[i] = float(x[i]);
#pragma unroll
          for (int i = 0; i < U; i++) uf[i] = float(I.un[(size_t)t * U + i]);
          MOps<M>::inc32(P, xf, uf, dv);
#pragma unroll
          for (int i = 0; i < N; i++) x[i] += double(dv[i]);
        }
        // (I.a is not a multiple of K: no other thread reads this entry in this phase)
#pragma unroll
        for (int i = 0; i < N; i++) I.xn[(size_t)I.a * N + i] = x[i];
      }
    }
    // no step direction yet: dx = 0 where the rollout reads it (x^ + s dx with s = 0)
    for (int t = I.a; t < I.b; t++)
#pragma unroll
      for (int i = 0; i < N; i++) I.dx[(size_t)t * N + i] = L(0);
    if (I.last)
#pragma unroll
      for (int i = 0; i < N; i++) I.dx[(size_t)I.T * N + i] = L(0);
    g.sync();
    Aug A;
    A.kind = AUG_BARRIER; A.mu = O.mu0; A.rho = 1.0; A.z = nullptr; A.v = nullptr;
    double m;
    const int rc = rollout(g, I, P, O, A, 0.0, false, &m, iters, O.roll_max_iter);
    if (rc == ROLL_FAIL) return false;
    double* t1 = I.xn; I.xn = I.xc; I.xc = t1;
    double* t2 = I.un; I.un = I.uc; I.uc = t2;
    g.sync();
    return true;
  }
}

// ---------------------------------------------------------------------------
// Adjoint at a solution (x*, u*) of the barrier problem with weight mu, for the loss
//   L = gJ J* + <gx, x*> + <gu, u*>   (J* = optimal barrier objective).
// J* part: envelope theorem on the Lagrangian eq. ocp-lagrangian, dJ*/dx0 = lam_1 and
// dJ*/dtheta = dL_c/dtheta at (x*, u*, lam*).  x*, u* part: implicit function theorem on
// the KKT system.  The adjoint LQR  min 1/2 w^T H w - g^T w  s.t. the linearised dynamics
// and w_{x,1} = 0 (H the Newton-step Hessian with alpha = 0, g = (gx, gu)) is solved by
// the value and state scans of the Newton step; its multipliers
//   nu_T = q_T + P_T w_T,  nu_t = q_t + P_t w_t + M_t w_{u,t} + F_t^T nu_{t+1},  q = -gx,
// come from a co-state-type scan; then dL/dtheta -= w^T d_theta(grad_z L) + nu^T d_theta f.
// Outputs (per instance): g_x0 (N), g_Qd (N), g_Rd (U), g_Qfd (N), g_prm (PTN_MAXP).
//
// Checkpointed form (AdjSeg): a horizon longer than the workspace is taken in segments of
// at most the workspace's length, and each segment's linearisations are recomputed from
// the stored trajectory (the checkpoints x*, u*) in three sweeps over the segments:
//   1 (backward)  co-states and the adjoint LQR's value function at the segment starts,
//   2 (forward)   the adjoint LQR's state w_x at the segment ends,
//   3 (backward)  its multipliers nu at the segment starts and the gradient contributions;
// each sweep hands its boundary values to the next segment it visits.
struct AdjSeg {
  int stage;            // 1, 2 or 3
  int first, last;      // this segment starts / ends the horizon
  const double* lam_end;                   // co-state at the segment end (not last)
  const double *S_end, *s_end;             // value function at the segment end (not last)
  const double* dx_start;                  // w_x at the segment start (stages 2, 3; not first)
  const double* nu_end;                    // nu at the segment end (stage 3; not last)
  double* lam_start;                       // out, stage 1
  double *S_start, *s_start;               // out, stage 1
  double* dx_end;                          // out, stage 2
  double* nu_start;                        // out, stage 3
};

struct AdjArgs {
  const double *gx, *gu;  // (sum T+1) x N, (sum T) x U, or NULL
  double* qx;             // workspace (sum T+1) x N (the linear terms -gx)
  double mu, gJ;
  double *g_x0, *g_Qd, *g_Rd, *g_Qfd, *g_prm;  // may be NULL
  const AdjSeg* seg;      // checkpointed form: this launch's segment and stage, or NULL
};

template <int K, class Grp>
__device__ void group_sum(Grp& g, double* v) {
#pragma unroll 1
  for (int c = 0; c < K; c += 8) {
    double r[8];
#pragma unroll
    for (int i = 0; i < 8; i++) r[i] = (c + i < K) ? v[c + i] : 0.0;
    g.template reduce<8>(r, 0u);
#pragma unroll
    for (int i = 0; i < 8; i++)
      if (c + i < K) v[c + i] = r[i];
  }
}

// nu scan and the parameter contractions, in FP64 (the adjoint runs with L = double in
// every precision mode: at a solution the reduced Hessian is ill-conditioned near active
// bounds, where the barrier curvature is large, and an FP32 adjoint LQR is not accurate
// enough there even with iterative refinement).
template <class M, class L, class Grp>
__device__ void adjoint_nu_pass(Grp& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const double* qx,
                                double* envp, double* adjp, double* nu0, const double* nuT_in = nullptr) {
  static_assert(std::is_same<L, double>::value, "the adjoint runs in FP64");
  constexpr int N = M::NX, U = M::NU, NP = M::NP;
  // c_t = q_t + P_t w_t + M_t w_{u,t}
  auto cterm = [&](int t, double* c) {
    const double* Pt = I.Pm + (size_t)t * N * N;
    const double* w = I.dx + (size_t)t * N;
#pragma unroll
    for (int i = 0; i < N; i++) {
      double v = qx[(size_t)t * N + i];
#pragma unroll
      for (int j = 0; j < N; j++) v += Pt[i * N + j] * w[j];
      if (t < I.T) {
        const double* Mt = I.Mm + (size_t)t * N * U;
        const double* wu = I.du + (size_t)t * U;
#pragma unroll
        for (int j = 0; j < U; j++) v += Mt[i * U + j] * wu[j];
      }
      c[i] = v;
    }
  };
  Aff<N, double> agg;
  set_identity(agg);
  double nuT[N];
  if (I.last) {
    if (nuT_in) {
#pragma unroll
      for (int i = 0; i < N; i++) nuT[i] = nuT_in[i];
    } else {
      cterm(I.T, nuT);
    }
#pragma unroll
    for (int i = 0; i < N; i++) {
      agg.v[i] = nuT[i];
#pragma unroll
      for (int j = 0; j < N; j++) agg.M[i * N + j] = 0.0;
    }
  }
  for (int t = I.b - 1; t >= I.a; t--) {
    const double* E = I.F64 + (size_t)t * N * N;
    double c[N], vn[N];
    cterm(t, c);
    mtv<N, N>(E, agg.v, vn);
#pragma unroll
    for (int i = 0; i < N; i++) agg.v[i] += vn[i] + c[i];
    if (!I.last) {
      double Mn[N * N];
      mtm<N, N, N>(E, agg.M, Mn);
#pragma unroll (N <= 8 ? N * N : 4)
      for (int i = 0; i < N * N; i++) agg.M[i] += Mn[i];
    }
  }
  bool ok = true;
  Aff<N, double> inc = g.scan(agg, CostateOp(), true, ok);
  double nu[N];
#pragma unroll
  for (int i = 0; i < N; i++) nu[i] = I.last ? nuT[i] : inc.v[i];
  for (int t = I.b - 1; t >= I.a; t--) {
    const double* x = I.xn + (size_t)t * N;
    const double* u = I.un + (size_t)t * U;
    const double* lam1 = (t + 1 == I.b) ? I.lamb : I.lam + (size_t)(t + 1) * N;
    const double* w = I.dx + (size_t)t * N;
    const double* wu = I.du + (size_t)t * U;
    double fp[N * NP], Hzp[(N + U) * NP];
    step_param_derivs<M>(P.integ, P.dt, P.prm, x, u, lam1, fp, Hzp);
#pragma unroll
    for (int k = 0; k < NP; k++) {
      double e = 0.0, a = 0.0;
#pragma unroll
      for (int i = 0; i < N; i++) {
        e += lam1[i] * fp[i * NP + k];
        a += nu[i] * fp[i * NP + k] + w[i] * Hzp[i * NP + k];
      }
#pragma unroll
      for (int j = 0; j < U; j++) a += wu[j] * Hzp[(N + j) * NP + k];
      envp[k] += e;
      if (adjp) adjp[k] += a;
    }
    const double* E = I.F64 + (size_t)t * N * N;
    double c[N], vn[N];
    cterm(t, c);
    mtv<N, N>(E, nu, vn);
#pragma unroll
    for (int i = 0; i < N; i++) nu[i] += vn[i] + c[i];
  }
  if (I.a == 0 && I.b > 0) {
#pragma unroll
    for (int i = 0; i < N; i++) nu0[i] = nu[i];
  }
}

// envelope-only parameter term (no trajectory gradients)
template <class M, class L>
__device__ void adjoint_env_params(Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, double* envp) {
  constexpr int N = M::NX, U = M::NU, NP = M::NP;
  for (int t = I.a; t < I.b; t++) {
    const double* lam1 = (t + 1 == I.b) ? I.lamb : I.lam + (size_t)(t + 1) * N;
    double fp[N * NP], Hzp[(N + U) * NP];
    step_param_derivs<M>(P.integ, P.dt, P.prm, I.xn + (size_t)t * N, I.un + (size_t)t * U, lam1, fp, Hzp);
#pragma unroll
    for (int k = 0; k < NP; k++) {
      double e = 0.0;
#pragma unroll
      for (int i = 0; i < N; i++) e += lam1[i] * fp[i * NP + k];
      envp[k] += e;
    }
  }
}

// returns ST_OK, or ST_ENUM when the Hessian is not positive definite on the dynamics.
// Checkpointed form (aa.seg): the passes of the segment's stage, with the boundary values
// of the neighbouring segments in place of the horizon's ends; stages 1 and 2 only hand
// on boundary values, stage 3 writes the segment's share of the outputs.
template <class M, class L, class SV, class Grp>
__device__ int adjoint_instance(Grp& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const AdjArgs& aa,
                                const InstDev& id, int bi) {
  constexpr int N = M::NX, U = M::NU, NP = M::NP;
  const AdjSeg* sg = aa.seg;
  const int stage = sg ? sg->stage : 0;  // 0: the whole horizon in one launch
  const bool seg_first = !sg || sg->first, seg_last = !sg || sg->last;
  const bool owns0 = I.a == 0 && I.b > 0;  // this thread holds t = 0
  Aug A;
  A.kind = AUG_BARRIER; A.mu = aa.mu; A.rho = 1.0; A.z = nullptr; A.v = nullptr;
  costate_exact(g, I, P, A, seg_last ? nullptr : sg->lam_end);
  // lam_0 for the envelope term, read once the co-state pass has ended (its closing group
  // reduction orders the writes)
  double lam0[N];
#pragma unroll
  for (int i = 0; i < N; i++) lam0[i] = I.lam[i];
  if (stage == 1 && owns0)
#pragma unroll
    for (int i = 0; i < N; i++) sg->lam_start[i] = lam0[i];
  const bool lin = sg || aa.gx || aa.gu;
  // out = [x0 (N), Qd (N), Rd (U), Qfd (N), prm (NP)] accumulated per thread
  constexpr int KO = 3 * N + U + NP;
  double env[KO], adj[KO];
#pragma unroll
  for (int i = 0; i < KO; i++) { env[i] = 0.0; adj[i] = 0.0; }
  for (int t = I.a; t < I.b; t++) {
#pragma unroll
    for (int i = 0; i < N; i++) {
      const double e = I.xn[(size_t)t * N + i] - xref_at(P, t)[i];
      env[N + i] += e * e;
    }
#pragma unroll
    for (int i = 0; i < U; i++) {
      const double e = I.un[(size_t)t * U + i] - uref_at(P, t)[i];
      env[2 * N + i] += e * e;
    }
  }
  if (I.last && seg_last) {
#pragma unroll
    for (int i = 0; i < N; i++) {
      const double e = I.xn[(size_t)I.T * N + i] - xref_at(P, I.T)[i];
      env[2 * N + U + i] = e * e;
    }
  }
  int rc = ST_OK;
  if (!lin) {
    adjoint_env_params(I, P, env + 3 * N + U);
  } else {
    quadratize(g, I, P, A);
    // linear terms of the adjoint LQR: d_t = -gu_t, q_t = -gx_t; a segment that does not
    // end the horizon ends with the value function of the segment after it
    double* qx = aa.qx + (size_t)id.xoff * N;
    for (int t = I.a; t < I.b; t++) {
#pragma unroll
      for (int i = 0; i < U; i++) I.d[(size_t)t * U + i] = aa.gu ? -aa.gu[((size_t)id.uoff + t) * U + i] : 0.0;
#pragma unroll
      for (int i = 0; i < N; i++) qx[(size_t)t * N + i] = aa.gx ? -aa.gx[((size_t)id.xoff + t) * N + i] : 0.0;
    }
    if (I.last) {
      if (seg_last) {
#pragma unroll
        for (int i = 0; i < N; i++) qx[(size_t)I.T * N + i] = aa.gx ? -aa.gx[((size_t)id.xoff + I.T) * N + i] : 0.0;
      } else {
#pragma unroll
        for (int i = 0; i < N; i++) qx[(size_t)I.T * N + i] = sg->s_end[i];
#pragma unroll (N <= 8 ? N * N : 4)
        for (int i = 0; i < N * N; i++) I.Pm[(size_t)I.T * N * N + i] = L(sg->S_end[i]);
      }
    }
    // the value pass reads q of its own chunk and the terminal one, written by the same
    // thread, and its first group operation orders the rest
    if (!value_pass<M, L, SV>(g, I, 0.0, qx, stage == 1 ? I.Sv : nullptr, stage == 1 ? I.sv : nullptr)) {
      rc = ST_ENUM;
    } else if (stage == 1) {
      // the value function at the segment start, S_0 and s_0 (after the stage at t = 0)
      if (owns0) {
#pragma unroll (N <= 8 ? N * N : 4)
        for (int i = 0; i < N * N; i++) sg->S_start[i] = double(I.Sv[i]);
#pragma unroll
        for (int i = 0; i < N; i++) sg->s_start[i] = double(I.sv[i]);
      }
    } else {
      double G1, G2;
      const L* dx_in = seg_first ? nullptr : sg->dx_start;
      state_pass(g, I, G1, G2, (const double*)nullptr, (const L*)nullptr, (const L*)nullptr, (double*)nullptr,
                 (double*)nullptr, dx_in);  // dx = w_x, du = w_u
      if (stage == 2) {
        if (I.last)
#pragma unroll
          for (int i = 0; i < N; i++) sg->dx_end[i] = double(I.dx[(size_t)I.T * N + i]);
      } else {
        double nu0[N];
#pragma unroll
        for (int i = 0; i < N; i++) nu0[i] = 0.0;
        adjoint_nu_pass(g, I, P, qx, env + 3 * N + U, adj + 3 * N + U, nu0, seg_last ? nullptr : sg->nu_end);
        if (stage == 3 && owns0)
#pragma unroll
          for (int i = 0; i < N; i++) sg->nu_start[i] = nu0[i];
        // dJ/dx0 takes nu_0 of the horizon's first step only
#pragma unroll
        for (int i = 0; i < N; i++) adj[i] = seg_first ? nu0[i] : 0.0;
        for (int t = I.a; t < I.b; t++) {
#pragma unroll
          for (int i = 0; i < N; i++)
            adj[N + i] += double(I.dx[(size_t)t * N + i]) * 2.0 * (I.xn[(size_t)t * N + i] - xref_at(P, t)[i]);
#pragma unroll
          for (int i = 0; i < U; i++)
            adj[2 * N + i] += double(I.du[(size_t)t * U + i]) * 2.0 * (I.un[(size_t)t * U + i] - uref_at(P, t)[i]);
        }
        if (I.last && seg_last) {
#pragma unroll
          for (int i = 0; i < N; i++)
            adj[2 * N + U + i] =
                double(I.dx[(size_t)I.T * N + i]) * 2.0 * (I.xn[(size_t)I.T * N + i] - xref_at(P, I.T)[i]);
        }
      }
    }
  }
  if (stage == 1 || stage == 2) return rc;
  double out[KO];
#pragma unroll
  for (int i = 0; i < KO; i++) out[i] = (i < N ? 0.0 : aa.gJ * env[i]) - adj[i];  // x0: lam_0 below
  if constexpr (user_cost<M>::value) {
    // a user-written cost does not depend on the weights Q, R, Qf
#pragma unroll
    for (int i = N; i < 3 * N + U; i++) out[i] = 0.0;
  }
  group_sum<KO>(g, out);  // also orders the co-state writes before lam_1 is read
  if (g.rank() == 0) {
    if (seg_first)
#pragma unroll
      for (int i = 0; i < N; i++) out[i] += aa.gJ * lam0[i];
    if (aa.g_x0)
      for (int i = 0; i < N; i++) aa.g_x0[(size_t)bi * N + i] = out[i];
    if (aa.g_Qd)
      for (int i = 0; i < N; i++) aa.g_Qd[(size_t)bi * N + i] = out[N + i];
    if (aa.g_Rd)
      for (int i = 0; i < U; i++) aa.g_Rd[(size_t)bi * U + i] = out[2 * N + i];
    if (aa.g_Qfd)
      for (int i = 0; i < N; i++) aa.g_Qfd[(size_t)bi * N + i] = out[2 * N + U + i];
    if (aa.g_prm)
      for (int k = 0; k < PTN_MAXP; k++) aa.g_prm[(size_t)bi * PTN_MAXP + k] = k < NP ? out[3 * N + U + k] : 0.0;
  }
  return rc;
}

// ---------------------------------------------------------------------------
// the whole solve of one instance (IP when O.method == 0, ADMM when 1)
template <class M, class L, class SV, class Grp>
__device__ void solve_instance(Grp& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const OptDev& O,
                               const double* u_init, InfoDev* info_out) {
  constexpr int N = M::NX, U = M::NU;
  InfoDev info;
  info.status = ST_OK; info.newton_iters = 0; info.outer_iters = 0; info.ls_rejects = 0;
  info.factor_fails = 0; info.roll_fails = 0; info.roll_iters = 0; info.ls_evals = 0;
  info.mu = 0; info.alpha = 0; info.r_stat = 0; info.r_dyn = 0; info.r_feas = 0; info.r_kkt = 0;
  info.J = 0; info.J_c = 0; info.r_p = 0; info.r_d = 0; info.pad_ = 0;
  for (int t = I.a; t < I.b; t++) {
#pragma unroll
    for (int i = 0; i < U; i++) {
      I.un[(size_t)t * U + i] = u_init ? u_init[(size_t)t * U + i] : 0.0;
      I.gam[(size_t)t * U + i] = L(0);
    }
#pragma unroll
    for (int i = 0; i < U * N; i++) I.Gam[(size_t)t * U * N + i] = L(0);
    if (O.costate_mode != 0)
#pragma unroll
      for (int i = 0; i < N; i++) I.lam[(size_t)t * N + i] = 0.0;  // multipliers start at zero
  }
  if (O.costate_mode != 0 && I.last)
#pragma unroll
    for (int i = 0; i < N; i++) I.lam[(size_t)I.T * N + i] = 0.0;
  g.sync();
  const long long c_start = clock64();
  NStats st{0, 0, 0, 0, 0, 0, 0, O.alpha0, {0, 0, 0, 0, 0, 0}};
  Aug A;
  int rc = ST_OK;
  {
    int ri = 0;
    if (!initial_rollout_parallel(g, I, P, O, &ri)) initial_rollout(g, I, P);
    st.roll_iters += ri;
  }
  st.cyc[5] = clock64() - c_start;
  if (O.method == 0) {
    // ---- primal log-barrier IP (eq. lb-min, lb-step-2) ----
    A.kind = AUG_BARRIER; A.mu = O.mu0; A.rho = 1.0; A.z = nullptr; A.v = nullptr;
    bool infeas;
    nominal_cost(g, I, P, A, &infeas, nullptr);
    if (infeas) {
      rc = ST_EINFEAS;
    } else {
      int level = 0;
      double mu = O.mu0;
      for (;;) {
        const bool lastlev = mu <= O.mu_final * (1.0 + 1e-9);
        A.mu = mu;
        double r;
        rc = newton_solve<M, L, SV>(g, I, P, O, A, lastlev ? O.tol_final : O.tol_inner, lastlev, st, &r);
        level++;
        if (rc == ST_ENUM || rc == ST_ETIMEOUT || lastlev) break;
        mu = O.mu0 * pow(O.zeta, (double)level);
        if (mu < O.mu_final) mu = O.mu_final;
      }
      info.outer_iters = level;
      info.mu = A.mu;
    }
  } else {
    // ---- ADMM (eq. admm-min ... admm-step-5), z^0 = min(0, w(x^0,u^0)), v^0 = 0 ----
    A.kind = AUG_ADMM; A.mu = 0.0; A.rho = O.rho; A.z = I.z; A.v = I.v;
    for (int t = I.a; t < I.b; t++)
      for (int r = 0; r < P.nw; r++) {
        const double zk = P.isx[r] ? I.xn[(size_t)t * N + P.idx[r]] : I.un[(size_t)t * U + P.idx[r]];
        const double w = P.sgn[r] * (zk - P.bnd[r]);
        I.z[(size_t)t * P.nw + r] = w < 0.0 ? w : 0.0;
        I.v[(size_t)t * P.nw + r] = 0.0;
      }
    g.sync();
    const int kmax = O.admm_fixed_iters > 0 ? O.admm_fixed_iters : O.max_outer;
    rc = ST_ENOTCONV;
    int k;
    double rp = INFINITY, rdl = INFINITY;
    bool admm_exact = false;  // sub-problems after the first FP64 endgame start exact
    for (k = 0; k < kmax; k++) {
      double r;
      const int s = newton_solve<M, L, SV>(g, I, P, O, A, O.tol_final, true, st, &r, &admm_exact);
      if (s == ST_ENUM || s == ST_ETIMEOUT) { rc = s; k++; break; }
      using CL = ChunkLanes<Grp>;
      double lrp = 0.0, lrd = 0.0;
      for (int t = I.a; t < I.b; t++)
        for (int rr = CL::first(); rr < P.nw; rr += CL::step()) {
          const double zk = P.isx[rr] ? I.xn[(size_t)t * N + P.idx[rr]] : I.un[(size_t)t * U + P.idx[rr]];
          const double w = P.sgn[rr] * (zk - P.bnd[rr]);
          const size_t q = (size_t)t * P.nw + rr;
          double zn = w + I.v[q] / O.rho;
          zn = zn < 0.0 ? zn : 0.0;
          I.v[q] += O.rho * (w - zn);
          lrp = fmax(lrp, fabs(w - zn));
          lrd = fmax(lrd, fabs(zn - I.z[q]));
          I.z[q] = zn;
        }
      double red[2] = {CL::max(lrp), CL::max(lrd)};
      g.template reduce<2>(red, 3u);
      rp = red[0];
      rdl = red[1];
      if (O.admm_fixed_iters <= 0 && rp <= O.admm_tol && rdl <= O.admm_tol) { rc = ST_OK; k++; break; }
    }
    if (O.admm_fixed_iters > 0 && rc != ST_ENUM && rc != ST_ETIMEOUT) rc = ST_OK;
    info.outer_iters = k;
    info.r_p = rp;
    info.r_d = rdl;
  }
  if (g.dead()) rc = ST_ETIMEOUT;
  if (rc != ST_EINFEAS && rc != ST_ETIMEOUT) residuals(g, I, P, A, info, O.costate_mode != 0);
  finalize_traj(g, I);
  info.status = rc;
  info.newton_iters = st.iters;
  info.ls_rejects = st.ls_rejects;
  info.factor_fails = st.factor_fails;
  info.roll_fails = st.roll_fails;
  info.roll_iters = st.roll_iters;
  info.ls_evals = st.ls_evals;
  info.exact_passes = st.exact_passes;
  info.alpha = st.alpha;
  info.r_kkt = fmax(fmax(info.r_stat, info.r_dyn), fmax(info.r_feas, O.method == 0 ? info.mu : 0.0));
  for (int k = 0; k < 6; k++) info.cyc[k] = st.cyc[k];
  info.cyc[6] = clock64() - c_start;
  for (int k = 0; k < 6; k++) info.cyc[6] -= st.cyc[k];
  if (g.rank() == 0) *info_out = info;
}

// ---------------------------------------------------------------------------
// kernels
struct KArgs {
  const ProbDev* prob;
  const OptDev* opt;
  const InstDev* inst;
  const double* x0;      // B x N
  const double* xref;    // B x N or null
  const double* u_init;  // concatenated controls or null
  const double* xtraj;   // time-varying targets: concatenated like the states, or null
  const double* utraj;   // ... like the controls, or null
  InfoDev* info;         // B
  GridScratch gs;
  int B, pad;
};

// the time-varying targets of instance id (null when the solve has none)
template <int N>
__device__ __forceinline__ const double* inst_xtraj(const KArgs& a, const InstDev& id) {
  return a.xtraj ? a.xtraj + (size_t)id.xoff * N : nullptr;
}
template <int U>
__device__ __forceinline__ const double* inst_utraj(const KArgs& a, const InstDev& id) {
  return a.utraj ? a.utraj + (size_t)id.uoff * U : nullptr;
}

template <int N, int U, class L>
__host__ __device__ constexpr size_t scratch_bytes(int nwarps) {
  // the value scan's group form (2 nwarps + 1 + nthreads / G elements and nthreads / G
  // ints), or 8 doubles per warp; a fused scan + reduction of state elements needs
  // nwarps + 2 slots and 8 + 64 bytes
  const size_t a = scan_group_scratch<Val<N, L>, GroupOp<ValueOpSel<double>, Val<N, L>>::G>(32 * nwarps);
  const size_t b = (size_t)nwarps * 8 * 8;
  const size_t c = (size_t)(nwarps + 2) * sizeof(Aff<N, L>) + 72;
  return a > b ? (a > c ? a : c) : (b > c ? b : c);
}

// one CTA per instance (batches and short horizons)
template <class M, class L, class SV>
__global__ void __launch_bounds__(256) k_solve_cta(KArgs args, Work<L> w) {
  constexpr int N = M::NX, U = M::NU;
  extern __shared__ __align__(16) char smem[];
  ProbS<N, U>& P = *reinterpret_cast<ProbS<N, U>*>(smem);
  char* scratch = smem + ((sizeof(ProbS<N, U>) + 15) & ~size_t(15));
  const int bi = blockIdx.x;
  if (bi >= args.B) return;
  load_prob<N, U>(P, *args.prob, args.xref ? args.xref + (size_t)bi * N : nullptr, args.inst[bi].dt,
                  inst_xtraj<N>(args, args.inst[bi]), inst_utraj<U>(args, args.inst[bi]), args.inst[bi].T);
  const OptDev& O = *args.opt;  // read where used (a local copy would hold ~50 registers)
  const InstDev id = args.inst[bi];
  CtaGroup g{scratch};
  Inst<M, L> I;
  I.setup(w, id, args.x0 + (size_t)bi * N, threadIdx.x, blockDim.x, P.nw);
  solve_instance<M, L, SV>(g, I, P, O, args.u_init ? args.u_init + (size_t)id.uoff * U : nullptr, args.info + bi);
}

// the whole cooperative grid on one instance (long horizons)
template <class M, class L, class SV>
__global__ void __launch_bounds__(128) k_solve_grid(KArgs args, Work<L> w) {
  constexpr int N = M::NX, U = M::NU;
  extern __shared__ __align__(16) char smem[];
  ProbS<N, U>& P = *reinterpret_cast<ProbS<N, U>*>(smem);
  char* scratch = smem + ((sizeof(ProbS<N, U>) + 15) & ~size_t(15));
  __shared__ int sdead;
  if (threadIdx.x == 0) sdead = 0;
  load_prob<N, U>(P, *args.prob, args.xref, args.inst[0].dt,
                  inst_xtraj<N>(args, args.inst[0]), inst_utraj<U>(args, args.inst[0]), args.inst[0].T);
  const OptDev& O = *args.opt;  // read where used (a local copy would hold ~50 registers)
  const InstDev id = args.inst[0];
  GridGroup g{scratch, args.gs, 0, &sdead};
  Inst<M, L> I;
  I.setup(w, id, args.x0, g.rank(), g.size(), P.nw);
  solve_instance<M, L, SV>(g, I, P, O, args.u_init, args.info);
}

// adjoint, one CTA per instance
template <class M, class L, class SV>
__global__ void __launch_bounds__(256) k_adjoint_cta(KArgs args, Work<L> w, AdjArgs aa) {
  constexpr int N = M::NX, U = M::NU;
  extern __shared__ __align__(16) char smem[];
  ProbS<N, U>& P = *reinterpret_cast<ProbS<N, U>*>(smem);
  char* scratch = smem + ((sizeof(ProbS<N, U>) + 15) & ~size_t(15));
  const int bi = blockIdx.x;
  if (bi >= args.B) return;
  load_prob<N, U>(P, *args.prob, args.xref ? args.xref + (size_t)bi * N : nullptr, args.inst[bi].dt,
                  inst_xtraj<N>(args, args.inst[bi]), inst_utraj<U>(args, args.inst[bi]), args.inst[bi].T);
  const InstDev id = args.inst[bi];
  CtaGroup g{scratch};
  Inst<M, L> I;
  I.setup(w, id, args.x0 + (size_t)bi * N, threadIdx.x, blockDim.x, P.nw);
  const int rc = adjoint_instance<M, L, SV>(g, I, P, aa, id, bi);
  if (threadIdx.x == 0) args.info[bi].status = rc;
}

// adjoint of one instance on the cooperative grid (long horizons): the same passes on the
// grid group; a barrier that expires reports ST_ETIMEOUT
template <class M, class L, class SV>
__global__ void __launch_bounds__(128) k_adjoint_grid(KArgs args, Work<L> w, AdjArgs aa) {
  constexpr int N = M::NX, U = M::NU;
  extern __shared__ __align__(16) char smem[];
  ProbS<N, U>& P = *reinterpret_cast<ProbS<N, U>*>(smem);
  char* scratch = smem + ((sizeof(ProbS<N, U>) + 15) & ~size_t(15));
  __shared__ int sdead;
  if (threadIdx.x == 0) sdead = 0;
  load_prob<N, U>(P, *args.prob, args.xref, args.inst[0].dt,
                  inst_xtraj<N>(args, args.inst[0]), inst_utraj<U>(args, args.inst[0]), args.inst[0].T);
  const InstDev id = args.inst[0];
  GridGroup g{scratch, args.gs, 0, &sdead};
  Inst<M, L> I;
  I.setup(w, id, args.x0, g.rank(), g.size(), P.nw);
  const int rc = adjoint_instance<M, L, SV>(g, I, P, aa, id, 0);
  if (g.rank() == 0) args.info[0].status = g.dead() ? ST_ETIMEOUT : rc;
}

// ---------------------------------------------------------------------------
// Sequential-in-time baseline: one thread per instance.  With a one-member group the
// scans are identities and each pass is its serial recursion (co-states backward, the
// Riccati recursion, states forward, plain sequential rollouts).
struct SeqGroup {
  __device__ int rank() const { return 0; }
  __device__ int size() const { return 1; }
  __device__ bool dead() const { return false; }
  __device__ void sync() {}
  template <int K>
  __device__ void reduce(double (&)[K], unsigned) {}
  template <class E, class Op>
  __device__ E scan(E, const Op&, bool, bool&) {
    E id;
    set_identity(id);
    return id;
  }
  template <class E, class Op, int K>
  __device__ E scan_reduce(E v, const Op& op, bool suffix, bool& ok, double (&)[K], unsigned) {
    return scan(v, op, suffix, ok);
  }
};

// problem record for one thread (as load_prob, without the CTA-wide copy)
template <int N, int U>
__device__ void load_prob_thread(ProbS<N, U>& S, const ProbDev& P, const double* xref_override, double dt_inst,
                                 const double* xtr, const double* utr, int T) {
  const double sc = dt_inst > 0.0 ? dt_inst / P.dt : 1.0;
  for (int i = 0; i < N * N; i++) {
    S.Q[i] = sc * P.Q[i];
    S.Qf[i] = P.Qf[i];
    S.Qs[i] = float(sc * (P.Q[i] + P.Q[(i % N) * N + i / N]));
    S.Qfs[i] = float(P.Qf[i] + P.Qf[(i % N) * N + i / N]);
  }
  for (int i = 0; i < U * U; i++) {
    S.R[i] = sc * P.R[i];
    S.Rs[i] = float(sc * (P.R[i] + P.R[(i % U) * U + i / U]));
  }
  for (int i = 0; i < N; i++) S.xref[i] = xref_override ? xref_override[i] : P.xref[i];
  for (int i = 0; i < U; i++) S.uref[i] = P.uref[i];
  for (int i = 0; i < PTN_MAXP; i++) S.prm[i] = P.prm[i];
  for (int i = 0; i < P.nw; i++) {
    S.sgn[i] = P.row_sgn[i]; S.bnd[i] = P.row_bnd[i]; S.isx[i] = P.row_isx[i]; S.idx[i] = P.row_idx[i];
  }
  S.nw = P.nw; S.integ = P.integrator; S.model = P.model; S.dt = dt_inst > 0.0 ? dt_inst : P.dt;
  S.A = P.A; S.B = P.B; S.W = P.W;
  S.xtr = xtr; S.utr = utr; S.Tr = T;
}

template <class M, class L, class SV>
__global__ void __launch_bounds__(64) k_solve_seq(KArgs args, Work<L> w) {
  constexpr int N = M::NX, U = M::NU;
  const int bi = blockIdx.x * blockDim.x + threadIdx.x;
  if (bi >= args.B) return;  // no group barriers below: threads are independent
  ProbS<N, U> P;
  load_prob_thread<N, U>(P, *args.prob, args.xref ? args.xref + (size_t)bi * N : nullptr, args.inst[bi].dt,
                         inst_xtraj<N>(args, args.inst[bi]), inst_utraj<U>(args, args.inst[bi]), args.inst[bi].T);
  const OptDev& O = *args.opt;  // read where used (a local copy would hold ~50 registers)
  const InstDev id = args.inst[bi];
  SeqGroup g;
  Inst<M, L> I;
  I.setup(w, id, args.x0 + (size_t)bi * N, 0, 1, P.nw);
  solve_instance<M, L, SV>(g, I, P, O, args.u_init ? args.u_init + (size_t)id.uoff * U : nullptr, args.info + bi);
}

// one thread-block cluster on one instance (medium horizons)
template <class M, class L, class SV>
__global__ void __launch_bounds__(256) k_solve_cluster(KArgs args, Work<L> w) {
  constexpr int N = M::NX, U = M::NU;
  extern __shared__ __align__(16) char smem[];
  ProbS<N, U>& P = *reinterpret_cast<ProbS<N, U>*>(smem);
  char* scratch = smem + ((sizeof(ProbS<N, U>) + 15) & ~size_t(15));
  const int nwarps = blockDim.x >> 5;
  const size_t sbytes = scratch_bytes<N, U, L>(nwarps);
  constexpr int XB = (int)((sizeof(Val<N, double>) > 64 ? sizeof(Val<N, double>) : 64) + 15) / 16 * 16;
  char* xch = scratch + ((sbytes + 15) & ~size_t(15));
  load_prob<N, U>(P, *args.prob, args.xref, args.inst[0].dt,
                  inst_xtraj<N>(args, args.inst[0]), inst_utraj<U>(args, args.inst[0]), args.inst[0].T);
  const OptDev& O = *args.opt;  // read where used (a local copy would hold ~50 registers)
  const InstDev id = args.inst[0];
  ClusterGroup g{scratch, xch, XB, 0};
  g.sync();  // every CTA of the cluster is running before any DSMEM access
  Inst<M, L> I;
  I.setup(w, id, args.x0, g.rank(), g.size(), P.nw);
  solve_instance<M, L, SV>(g, I, P, O, args.u_init, args.info);
  g.sync();  // keep this CTA's shared memory alive until every CTA is done reading it
}

template <int N, int U, class L>
__host__ __device__ constexpr size_t cluster_xch_bytes() {
  return 2 * (size_t)(((sizeof(Val<N, double>) > 64 ? sizeof(Val<N, double>) : 64) + 15) / 16 * 16);
}

}  // namespace ptn
