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
// Precision: trajectories, co-states, gradients, costs, Cholesky factorisations and
// (I + C J)^{-1} are FP64; the LQR elements, scans and feedback use L (float or double).
#pragma once
#include "ptn_group.cuh"
#include "ptn_models.cuh"

namespace ptn {

// per-instance problem data copied to shared memory at kernel start
template <int N, int U>
struct ProbS {
  static constexpr int NW = 2 * (N + U);
  double Q[N * N], R[U * U], Qf[N * N], xref[N], uref[U];
  double prm[PTN_MAXP];
  double sgn[NW], bnd[NW];
  int isx[NW], idx[NW];
  int nw, integ, model, pad;
  double dt;
  const double *A, *B, *W;
};

template <int N, int U>
__device__ void load_prob(ProbS<N, U>& S, const ProbDev& P, const double* xref_override) {
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) { S.Q[i] = P.Q[i]; S.Qf[i] = P.Qf[i]; }
  for (int i = threadIdx.x; i < U * U; i += blockDim.x) S.R[i] = P.R[i];
  for (int i = threadIdx.x; i < N; i += blockDim.x) S.xref[i] = xref_override ? xref_override[i] : P.xref[i];
  for (int i = threadIdx.x; i < U; i += blockDim.x) S.uref[i] = P.uref[i];
  for (int i = threadIdx.x; i < PTN_MAXP; i += blockDim.x) S.prm[i] = P.prm[i];
  for (int i = threadIdx.x; i < P.nw; i += blockDim.x) {
    S.sgn[i] = P.row_sgn[i]; S.bnd[i] = P.row_bnd[i]; S.isx[i] = P.row_isx[i]; S.idx[i] = P.row_idx[i];
  }
  if (threadIdx.x == 0) {
    S.nw = P.nw; S.integ = P.integrator; S.model = P.model; S.dt = P.dt;
    S.A = P.A; S.B = P.B; S.W = P.W;
  }
  __syncthreads();
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
    step_hess<M, L>(P.integ, P.dt, P.prm, x, u, lam, Hxx, Hxu, Huu);
  }
  template <class PS, class L>
  __device__ static void cl(const PS& P, const double* x, const double* u, const L* Gam, double* xn, L* Fcl) {
    step_cl_jac<M, L>(P.integ, P.dt, P.prm, x, u, Gam, Fcl);
    step<M>(P.integ, P.dt, P.prm, x, u, xn);
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

template <int N, int U>
__device__ double stage_cost(const ProbS<N, U>& P, const Aug& A, int t, const double* x, const double* u,
                             bool& infeas, double* lplain = nullptr) {
  double l = 0.0, e[N];
#pragma unroll
  for (int i = 0; i < N; i++) e[i] = x[i] - P.xref[i];
#pragma unroll
  for (int i = 0; i < N; i++) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < N; j++) s += P.Q[i * N + j] * e[j];
    l += e[i] * s;
  }
  double eu[U];
#pragma unroll
  for (int i = 0; i < U; i++) eu[i] = u[i] - P.uref[i];
#pragma unroll
  for (int i = 0; i < U; i++) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < U; j++) s += P.R[i * U + j] * eu[j];
    l += eu[i] * s;
  }
  if (lplain) *lplain = l;
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
__device__ void stage_grad(const ProbS<N, U>& P, const Aug& A, int t, const double* x, const double* u,
                           double* lx, double* lu) {
#pragma unroll
  for (int i = 0; i < N; i++) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < N; j++) s += (P.Q[i * N + j] + P.Q[j * N + i]) * (x[j] - P.xref[j]);
    lx[i] = s;
  }
#pragma unroll
  for (int i = 0; i < U; i++) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < U; j++) s += (P.R[i * U + j] + P.R[j * U + i]) * (u[j] - P.uref[j]);
    lu[i] = s;
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

// adds the Hessians of l_t + c_t to P (N x N), R (U x U); l_xu = c_xu = 0 for box rows
template <int N, int U, class L>
__device__ void stage_hess_add(const ProbS<N, U>& P, const Aug& A, const double* x, const double* u, L* Pm,
                               L* Rm) {
#pragma unroll
  for (int i = 0; i < N; i++)
#pragma unroll
    for (int j = 0; j < N; j++) Pm[i * N + j] += L(P.Q[i * N + j] + P.Q[j * N + i]);
#pragma unroll
  for (int i = 0; i < U; i++)
#pragma unroll
    for (int j = 0; j < U; j++) Rm[i * U + j] += L(P.R[i * U + j] + P.R[j * U + i]);
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
  double l = 0.0;
#pragma unroll
  for (int i = 0; i < N; i++) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < N; j++) s += P.Qf[i * N + j] * (x[j] - P.xref[j]);
    l += (x[i] - P.xref[i]) * s;
  }
  return l;
}

// ---------------------------------------------------------------------------
// device workspace: base pointers of the concatenated per-instance arrays
template <class L>
struct Work {
  double *xA, *uA;    // trajectory buffer A (the caller's output arrays)
  double *xB, *uB;    // trajectory buffer B (workspace)
  double *lam;        // (sum T+1) x N
  double *F, *G, *d;  // (sum T) x N*N, x N*U, x U
  L *Pm;              // (sum T+1) x N*N
  L *Mm, *Rm;         // (sum T) x N*U, x U*U
  L *Gam, *gam;       // (sum T) x U*N, x U
  L *dx, *du;         // (sum T+1) x N, (sum T) x U
  double *z, *v;      // (sum T) x nw (ADMM)
};

template <class M, class L>
struct Inst {
  static constexpr int N = M::NX, U = M::NU;
  int T, a, b;
  bool last;
  const double* x0;
  double *xn, *un, *xc, *uc;  // nominal and candidate trajectories
  double *xA, *uA;            // the caller's output arrays
  double *lam, *F, *G, *d;
  L *Pm, *Mm, *Rm, *Gam, *gam, *dx, *du;
  double *z, *v;

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
    F = w.F + uo * N * N; G = w.G + uo * N * U; d = w.d + uo * U;
    Pm = w.Pm + xo * N * N; Mm = w.Mm + uo * N * U; Rm = w.Rm + uo * U * U;
    Gam = w.Gam + uo * U * N; gam = w.gam + uo * U;
    dx = w.dx + xo * N; du = w.du + uo * U;
    z = w.z ? w.z + uo * nw : nullptr;
    v = w.v ? w.v + uo * nw : nullptr;
  }
};

// ---------------------------------------------------------------------------
// pass 1: co-state suffix scan (Alg. 1).  Returns max_t |d_t|_inf (inf if not finite).
template <class M, class L, class Grp>
__device__ double costate_pass(Grp& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const Aug& A) {
  constexpr int N = M::NX, U = M::NU;
  Aff<N, double> agg;
  set_identity(agg);
  if (I.last) {
    // terminal co-state lam_{N+1} = d l_{N+1} / dx (eq. co-state-final), a constant map
#pragma unroll
    for (int i = 0; i < N; i++) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < N; j++) s += (P.Qf[i * N + j] + P.Qf[j * N + i]) * (I.xn[I.T * N + j] - P.xref[j]);
      agg.v[i] = s;
#pragma unroll
      for (int j = 0; j < N; j++) agg.M[i * N + j] = 0.0;
    }
  }
  // up-sweep: agg = a_t (x) agg for t = b-1 .. a, with a_t = (q_t, F_t^T)
  for (int t = I.b - 1; t >= I.a; t--) {
    double F[N * N], G[N * U], q[N], r[U];
    const double* x = I.xn + (size_t)t * N;
    const double* u = I.un + (size_t)t * U;
    MOps<M>::jac(P, x, u, F, G);
#pragma unroll
    for (int i = 0; i < N * N; i++) I.F[(size_t)t * N * N + i] = F[i];
#pragma unroll
    for (int i = 0; i < N * U; i++) I.G[(size_t)t * N * U + i] = G[i];
    stage_grad(P, A, t, x, u, q, r);
    double vn[N];
    mtv<N, N>(F, agg.v, vn);
#pragma unroll
    for (int i = 0; i < N; i++) agg.v[i] = vn[i] + q[i];
    if (!I.last) {
      double Mn[N * N];
      mtm<N, N, N>(F, agg.M, Mn);
#pragma unroll
      for (int i = 0; i < N * N; i++) agg.M[i] = Mn[i];
    }
  }
  bool ok = true;
  Aff<N, double> inc = g.scan(agg, CostateOp(), true, ok);
  // downsweep from lam at the chunk end (the suffix has a zero matrix part)
  double lam[N];
  if (I.last) {
#pragma unroll
    for (int i = 0; i < N; i++) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < N; j++) s += (P.Qf[i * N + j] + P.Qf[j * N + i]) * (I.xn[I.T * N + j] - P.xref[j]);
      lam[i] = s;
      I.lam[(size_t)I.T * N + i] = s;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; i++) lam[i] = inc.v[i];
  }
  double dmax = 0.0;
  for (int t = I.b - 1; t >= I.a; t--) {
    const double* x = I.xn + (size_t)t * N;
    const double* u = I.un + (size_t)t * U;
    const double* F = I.F + (size_t)t * N * N;
    const double* G = I.G + (size_t)t * N * U;
    double q[N], r[U], ln[N], dd[U];
    stage_grad(P, A, t, x, u, q, r);
    mtv<N, N>(F, lam, ln);
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
      lam[i] = ln[i] + q[i];
      I.lam[(size_t)t * N + i] = lam[i];
    }
  }
  double red[1] = {dmax};
  g.template reduce<1>(red, 1u);
  return red[0];
}

// pass 2: second-order expansion (Sec. III-C).  Needs lam from pass 1 (group-synced).
template <class M, class L, class Grp>
__device__ void quadratize(Grp& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const Aug& A) {
  constexpr int N = M::NX, U = M::NU;
  for (int t = I.a; t < I.b; t++) {
    const double* x = I.xn + (size_t)t * N;
    const double* u = I.un + (size_t)t * U;
    L Pm[N * N], Mm[N * U], Rm[U * U];
    MOps<M>::hess(P, x, u, I.lam + (size_t)(t + 1) * N, Pm, Mm, Rm);
    stage_hess_add(P, A, x, u, Pm, Rm);
#pragma unroll
    for (int i = 0; i < N * N; i++) I.Pm[(size_t)t * N * N + i] = Pm[i];
#pragma unroll
    for (int i = 0; i < N * U; i++) I.Mm[(size_t)t * N * U + i] = Mm[i];
#pragma unroll
    for (int i = 0; i < U * U; i++) I.Rm[(size_t)t * U * U + i] = Rm[i];
  }
  if (I.last) {
#pragma unroll
    for (int i = 0; i < N * N; i++) I.Pm[(size_t)I.T * N * N + i] = L(P.Qf[i] + P.Qf[(i % N) * N + i / N]);
  }
  g.sync();
}

// pass 3: value suffix scan (Alg. 2) + feedback sweep.  Returns true on success; false
// (group-uniform) when some R~_t, Q_t is not PD or some I + C J is singular.
template <class M, class L, class Grp>
__device__ bool value_pass(Grp& g, Inst<M, L>& I, double alpha) {
  constexpr int N = M::NX, U = M::NU;
  bool ok = true, have = false;
  Val<N, L> agg;
  set_identity(agg);
  if (I.last) {
    value_terminal<N, L>(I.Pm + (size_t)I.T * N * N, agg);
    have = true;
  }
  for (int t = I.b - 1; t >= I.a; t--) {
    Val<N, L> e;
    ok &= value_init<N, U, L>(I.F + (size_t)t * N * N, I.G + (size_t)t * N * U, I.Pm + (size_t)t * N * N,
                              I.Mm + (size_t)t * N * U, I.Rm + (size_t)t * U * U, I.d + (size_t)t * U, alpha, e);
    if (!have) { agg = e; have = true; }
    else ok &= ValueOp()(e, agg, agg);
  }
  Val<N, L> inc = g.scan(agg, ValueOp(), true, ok);
  L S[N * N], s[N];
  if (I.last) {
#pragma unroll
    for (int i = 0; i < N * N; i++) S[i] = I.Pm[(size_t)I.T * N * N + i];
#pragma unroll
    for (int i = 0; i < N; i++) s[i] = L(0);
  } else {
    // S_t = J_{t,<|}, s_t = -eta_{t,<|}
#pragma unroll
    for (int i = 0; i < N * N; i++) S[i] = inc.J[i];
#pragma unroll
    for (int i = 0; i < N; i++) s[i] = -inc.eta[i];
  }
  for (int t = I.b - 1; t >= I.a; t--) {
    L Gam[U * N], gam[U];
    ok &= riccati_step<N, U, L>(I.F + (size_t)t * N * N, I.G + (size_t)t * N * U, I.Pm + (size_t)t * N * N,
                                I.Mm + (size_t)t * N * U, I.Rm + (size_t)t * U * U, I.d + (size_t)t * U, alpha, S,
                                s, Gam, gam);
#pragma unroll
    for (int i = 0; i < U * N; i++) I.Gam[(size_t)t * U * N + i] = Gam[i];
#pragma unroll
    for (int i = 0; i < U; i++) I.gam[(size_t)t * U + i] = gam[i];
  }
  double red[1] = {ok ? 0.0 : 1.0};
  g.template reduce<1>(red, 1u);
  return red[0] == 0.0;
}

// pass 4: state prefix scan (Alg. 3).  dx_1 = 0, du = Gam dx + gam, dx+ = F dx + G du.
// Returns the model terms G1, G2 (R without the alpha shift).
template <class M, class L, class Grp>
__device__ void state_pass(Grp& g, Inst<M, L>& I, double& G1, double& G2) {
  constexpr int N = M::NX, U = M::NU;
  Aff<N, L> agg;
  set_identity(agg);
  const bool first = (I.a == 0);
  if (first) {
#pragma unroll
    for (int i = 0; i < N * N; i++) agg.M[i] = L(0);  // the first element has F = 0
  }
  for (int t = I.a; t < I.b; t++) {
    L Fc[N * N], e[N];
    const double* F = I.F + (size_t)t * N * N;
    const double* G = I.G + (size_t)t * N * U;
    const L* Gam = I.Gam + (size_t)t * U * N;
    const L* gam = I.gam + (size_t)t * U;
#pragma unroll
    for (int i = 0; i < N; i++) {
#pragma unroll
      for (int j = 0; j < N; j++) {
        L s = L(F[i * N + j]);
#pragma unroll
        for (int k = 0; k < U; k++) s += L(G[i * U + k]) * Gam[k * N + j];
        Fc[i * N + j] = s;
      }
      L s = L(0);
#pragma unroll
      for (int k = 0; k < U; k++) s += L(G[i * U + k]) * gam[k];
      e[i] = s;
    }
    L vn[N];
    mv<N, N>(Fc, agg.v, vn);
#pragma unroll
    for (int i = 0; i < N; i++) agg.v[i] = vn[i] + e[i];
    if (!first) {
      L Mn[N * N];
      mm<N, N, N>(Fc, agg.M, Mn);
#pragma unroll
      for (int i = 0; i < N * N; i++) agg.M[i] = Mn[i];
    }
  }
  bool ok = true;
  Aff<N, L> inc = g.scan(agg, StateOp(), false, ok);
  L dx[N];
#pragma unroll
  for (int i = 0; i < N; i++) dx[i] = first ? L(0) : inc.v[i];
  double g1 = 0.0, g2 = 0.0;
  for (int t = I.a; t < I.b; t++) {
    const double* F = I.F + (size_t)t * N * N;
    const double* G = I.G + (size_t)t * N * U;
    const L* Gam = I.Gam + (size_t)t * U * N;
    const L* gam = I.gam + (size_t)t * U;
    const L* Pm = I.Pm + (size_t)t * N * N;
    const L* Mm = I.Mm + (size_t)t * N * U;
    const L* Rm = I.Rm + (size_t)t * U * U;
    L du[U];
#pragma unroll
    for (int i = 0; i < U; i++) {
      L s = gam[i];
#pragma unroll
      for (int j = 0; j < N; j++) s += Gam[i * N + j] * dx[j];
      du[i] = s;
      I.du[(size_t)t * U + i] = s;
      g1 += I.d[(size_t)t * U + i] * double(s);
    }
#pragma unroll
    for (int i = 0; i < N; i++) I.dx[(size_t)t * N + i] = dx[i];
    double q = 0.0;
#pragma unroll
    for (int i = 0; i < N; i++) {
      double sp = 0.0, sm = 0.0;
#pragma unroll
      for (int j = 0; j < N; j++) sp += double(Pm[i * N + j]) * double(dx[j]);
#pragma unroll
      for (int j = 0; j < U; j++) sm += double(Mm[i * U + j]) * double(du[j]);
      q += double(dx[i]) * (0.5 * sp + sm);
    }
#pragma unroll
    for (int i = 0; i < U; i++) {
      double sr = 0.0;
#pragma unroll
      for (int j = 0; j < U; j++) sr += double(Rm[i * U + j]) * double(du[j]);
      q += 0.5 * double(du[i]) * sr;
    }
    g2 += q;
    L dn[N];
#pragma unroll
    for (int i = 0; i < N; i++) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < N; j++) s += F[i * N + j] * double(dx[j]);
#pragma unroll
      for (int j = 0; j < U; j++) s += G[i * U + j] * double(du[j]);
      dn[i] = L(s);
    }
#pragma unroll
    for (int i = 0; i < N; i++) dx[i] = dn[i];
  }
  if (I.last) {
    const L* PT = I.Pm + (size_t)I.T * N * N;
#pragma unroll
    for (int i = 0; i < N; i++) {
      I.dx[(size_t)I.T * N + i] = dx[i];
      double sp = 0.0;
#pragma unroll
      for (int j = 0; j < N; j++) sp += double(PT[i * N + j]) * double(dx[j]);
      g2 += 0.5 * double(dx[i]) * sp;
    }
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
// Writes the candidate into (xc, uc).  Returns true when converged, finite and (for
// the barrier) strictly feasible; *Jc receives the augmented cost J_c.
template <class M, class L, class Grp>
__device__ bool rollout(Grp& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const OptDev& O, const Aug& A,
                        double s, bool closed, double* Jc, int* iters) {
  constexpr int N = M::NX, U = M::NU;
  double X[N];
  const bool own = (I.a < I.b);
  const bool first = (I.a == 0);
#pragma unroll
  for (int i = 0; i < N; i++)
    X[i] = first ? I.x0[i] : (closed ? I.xn[(size_t)I.a * N + i] + s * double(I.dx[(size_t)I.a * N + i])
                                     : I.xc[(size_t)I.a * N + i]);
  bool conv = false, feas = true;
  double J = INFINITY;
  for (int it = 0; it < O.roll_max_iter; it++) {
    if (own) {
#pragma unroll
      for (int i = 0; i < N; i++) I.xc[(size_t)I.a * N + i] = X[i];
    }
    g.sync();
    double Xn[N];
    if (own && !I.last) {
#pragma unroll
      for (int i = 0; i < N; i++) Xn[i] = I.xc[(size_t)I.b * N + i];
    }
    g.sync();
    double xt[N], cost = 0.0;
    bool inf = false;
    Aff<N, L> el;
    set_identity(el);
#pragma unroll
    for (int i = 0; i < N; i++) xt[i] = X[i];
    for (int t = I.a; t < I.b; t++) {
      const L* Gam = I.Gam + (size_t)t * U * N;
      double ut[U];
#pragma unroll
      for (int i = 0; i < U; i++) {
        double v = I.un[(size_t)t * U + i];
        if (closed) {
          v += s * double(I.gam[(size_t)t * U + i]);
#pragma unroll
          for (int j = 0; j < N; j++) v += double(Gam[i * N + j]) * (xt[j] - I.xn[(size_t)t * N + j]);
        }
        ut[i] = v;
        I.uc[(size_t)t * U + i] = v;
      }
      if (t > I.a) {
#pragma unroll
        for (int i = 0; i < N; i++) I.xc[(size_t)t * N + i] = xt[i];
      }
      cost += stage_cost(P, A, t, xt, ut, inf);
      double xnext[N];
      L Fc[N * N];
      if (closed) {
        MOps<M>::cl(P, xt, ut, Gam, xnext, Fc);
      } else {
        L Z[U * N];
#pragma unroll
        for (int i = 0; i < U * N; i++) Z[i] = L(0);
        MOps<M>::cl(P, xt, ut, Z, xnext, Fc);
      }
      if (!first) {
        L Mn[N * N];
        mm<N, N, N>(Fc, el.M, Mn);
#pragma unroll
        for (int i = 0; i < N * N; i++) el.M[i] = Mn[i];
      }
#pragma unroll
      for (int i = 0; i < N; i++) xt[i] = xnext[i];
    }
    double rmax = 0.0, xmax = 0.0;
    bool nonfin = !isfinite(cost);
    if (first) {
#pragma unroll
      for (int i = 0; i < N * N; i++) el.M[i] = L(0);
    }
    if (I.last) {
#pragma unroll
      for (int i = 0; i < N; i++) I.xc[(size_t)I.T * N + i] = xt[i];
      cost += terminal_cost(P, xt);
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
    Aff<N, L> inc = g.scan(el, StateOp(), false, ok);
    double red[5] = {rmax, xmax, cost, inf ? 1.0 : 0.0, nonfin ? 1.0 : 0.0};
    g.template reduce<5>(red, 0x1bu);  // max, max, sum, max, max
    if (iters) *iters = it + 1;
    if (red[4] > 0.0) return false;
    if (red[0] <= O.roll_tol * (1.0 + red[1])) {
      conv = true;
      feas = !(red[3] > 0.0);
      J = red[2];
      break;
    }
    if (!first && own) {
#pragma unroll
      for (int i = 0; i < N; i++) X[i] += double(inc.v[i]);
    }
  }
  *Jc = J;
  return conv && feas && isfinite(J);
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
    c += stage_cost(P, A, t, I.xn + (size_t)t * N, I.un + (size_t)t * U, inf, &lp);
    cp += lp;
  }
  if (I.last) {
    const double lt = terminal_cost(P, I.xn + (size_t)I.T * N);
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
struct NStats {
  int iters, ls_rejects, factor_fails, roll_fails, roll_iters, ls_evals;
  double alpha;
  long long cyc[6];
};

// Newton iterations (Alg. 4) on the augmented sub-problem until max |d| <= tol.
// Step acceptance and the alpha rule are the same readings as the CPU oracle's.
template <class M, class L, class Grp>
__device__ int newton_solve(Grp& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const OptDev& O, const Aug& A,
                            double tol, NStats& st, double* rfinal) {
  bool inf;
  double J0 = nominal_cost(g, I, P, A, &inf, nullptr);
  int rc = ST_ENOTCONV;
  double r = INFINITY;
  for (int it = 0; it <= O.max_newton; it++) {
    if (g.dead()) return ST_ETIMEOUT;
    long long c0 = clock64();
    r = costate_pass(g, I, P, A);
    long long c1 = clock64();
    st.cyc[0] += c1 - c0;
    if (r <= tol) { rc = ST_OK; break; }
    if (it == O.max_newton || !isfinite(r) || !isfinite(J0)) break;
    st.iters++;
    quadratize(g, I, P, A);
    long long c2 = clock64();
    st.cyc[1] += c2 - c1;
    while (!value_pass(g, I, st.alpha)) {
      st.factor_fails++;
      st.alpha = fmax(10.0 * st.alpha, 1e-8);
      if (st.alpha > O.alpha_max || g.dead()) { *rfinal = r; return g.dead() ? ST_ETIMEOUT : ST_ENUM; }
    }
    long long c3 = clock64();
    st.cyc[2] += c3 - c2;
    double G1, G2;
    state_pass(g, I, G1, G2);
    long long c4 = clock64();
    st.cyc[3] += c4 - c3;
    bool accepted = false;
    double s = 1.0, Js = INFINITY;
    for (int k = 0; k < O.ls_count; k++, s *= O.ls_beta) {
      int ri = 0;
      const bool okr = rollout(g, I, P, O, A, s, true, &Js, &ri);
      st.ls_evals++;
      st.roll_iters += ri;
      if (!okr) { st.roll_fails++; continue; }
      if (Js <= J0 + O.armijo_c1 * s * G1 + O.armijo_eps * (1.0 + fabs(J0))) { accepted = true; break; }
    }
    st.cyc[4] += clock64() - c4;
    if (accepted) {
      const double pred = -(s * G1 + s * s * G2);
      const double rho = pred > 0.0 ? (J0 - Js) / pred : 0.0;
      if (rho > 0.75) st.alpha /= 3.0;
      else if (rho < 0.25) st.alpha *= 2.0;
      st.alpha = fmin(fmax(st.alpha, O.alpha_min), O.alpha_max);
      double* t1 = I.xn; I.xn = I.xc; I.xc = t1;
      double* t2 = I.un; I.un = I.uc; I.uc = t2;
      J0 = Js;
    } else {
      st.ls_rejects++;
      st.alpha *= 10.0;
      if (st.alpha > O.alpha_max) { rc = ST_ENUM; break; }
    }
  }
  *rfinal = r;
  return rc;
}

// final residuals: r_stat (max |d|), r_dyn, r_feas, J, J_c; lam of the final point
template <class M, class L, class Grp>
__device__ void residuals(Grp& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const Aug& A, InfoDev& info) {
  constexpr int N = M::NX, U = M::NU;
  info.r_stat = costate_pass(g, I, P, A);
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

// initial nominal: x = rollout(x0, u_init) (open loop).  The candidate buffer is first
// filled by one thread's sequential integration, which is the exact rollout.
template <class M, class L, class Grp>
__device__ void initial_rollout(Grp& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P) {
  constexpr int N = M::NX, U = M::NU;
  if (g.rank() == 0) {
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
  g.sync();
}

// ---------------------------------------------------------------------------
// the whole solve of one instance (IP when O.method == 0, ADMM when 1)
template <class M, class L, class Grp>
__device__ void solve_instance(Grp& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const OptDev& O,
                               const double* u_init, InfoDev* info_out) {
  constexpr int N = M::NX, U = M::NU;
  InfoDev info;
  info.status = ST_OK; info.newton_iters = 0; info.outer_iters = 0; info.ls_rejects = 0;
  info.factor_fails = 0; info.roll_fails = 0; info.roll_iters = 0; info.ls_evals = 0;
  info.mu = 0; info.alpha = 0; info.r_stat = 0; info.r_dyn = 0; info.r_feas = 0; info.r_kkt = 0;
  info.J = 0; info.J_c = 0; info.r_p = 0; info.r_d = 0;
  for (int t = I.a; t < I.b; t++)
#pragma unroll
    for (int i = 0; i < U; i++) I.un[(size_t)t * U + i] = u_init ? u_init[(size_t)t * U + i] : 0.0;
  g.sync();
  initial_rollout(g, I, P);
  NStats st{0, 0, 0, 0, 0, 0, O.alpha0, {0, 0, 0, 0, 0, 0}};
  const long long c_start = clock64();
  Aug A;
  int rc = ST_OK;
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
        rc = newton_solve(g, I, P, O, A, lastlev ? O.tol_final : O.tol_inner, st, &r);
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
    for (k = 0; k < kmax; k++) {
      double r;
      const int s = newton_solve(g, I, P, O, A, O.tol_final, st, &r);
      if (s == ST_ENUM || s == ST_ETIMEOUT) { rc = s; k++; break; }
      double lrp = 0.0, lrd = 0.0;
      for (int t = I.a; t < I.b; t++)
        for (int rr = 0; rr < P.nw; rr++) {
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
      double red[2] = {lrp, lrd};
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
  if (rc != ST_EINFEAS && rc != ST_ETIMEOUT) residuals(g, I, P, A, info);
  finalize_traj(g, I);
  info.status = rc;
  info.newton_iters = st.iters;
  info.ls_rejects = st.ls_rejects;
  info.factor_fails = st.factor_fails;
  info.roll_fails = st.roll_fails;
  info.roll_iters = st.roll_iters;
  info.ls_evals = st.ls_evals;
  info.alpha = st.alpha;
  for (int k = 0; k < 5; k++) info.cyc[k] = st.cyc[k];
  info.cyc[5] = clock64() - c_start - (st.cyc[0] + st.cyc[1] + st.cyc[2] + st.cyc[3] + st.cyc[4]);
  info.r_kkt = fmax(fmax(info.r_stat, info.r_dyn), fmax(info.r_feas, O.method == 0 ? info.mu : 0.0));
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
  InfoDev* info;         // B
  GridScratch gs;
  int B, pad;
};

template <int N, int U, class L>
constexpr size_t scratch_bytes(int nwarps) {
  // largest collective element (value element), nwarps + 2 slots, or 8 doubles per warp
  return ((size_t)(nwarps + 2) * sizeof(Val<N, L>) > (size_t)nwarps * 8 * 8)
             ? (size_t)(nwarps + 2) * sizeof(Val<N, L>)
             : (size_t)nwarps * 8 * 8;
}

// one CTA per instance (batches and short horizons)
template <class M, class L>
__global__ void __launch_bounds__(256) k_solve_cta(KArgs args, Work<L> w) {
  constexpr int N = M::NX, U = M::NU;
  extern __shared__ __align__(16) char smem[];
  ProbS<N, U>& P = *reinterpret_cast<ProbS<N, U>*>(smem);
  char* scratch = smem + ((sizeof(ProbS<N, U>) + 15) & ~size_t(15));
  const int bi = blockIdx.x;
  if (bi >= args.B) return;
  load_prob<N, U>(P, *args.prob, args.xref ? args.xref + (size_t)bi * N : nullptr);
  const OptDev O = *args.opt;
  const InstDev id = args.inst[bi];
  CtaGroup g{scratch};
  Inst<M, L> I;
  I.setup(w, id, args.x0 + (size_t)bi * N, threadIdx.x, blockDim.x, P.nw);
  solve_instance<M, L>(g, I, P, O, args.u_init ? args.u_init + (size_t)id.uoff * U : nullptr, args.info + bi);
}

// the whole cooperative grid on one instance (long horizons)
template <class M, class L>
__global__ void __launch_bounds__(128) k_solve_grid(KArgs args, Work<L> w) {
  constexpr int N = M::NX, U = M::NU;
  extern __shared__ __align__(16) char smem[];
  ProbS<N, U>& P = *reinterpret_cast<ProbS<N, U>*>(smem);
  char* scratch = smem + ((sizeof(ProbS<N, U>) + 15) & ~size_t(15));
  __shared__ int sdead;
  if (threadIdx.x == 0) sdead = 0;
  load_prob<N, U>(P, *args.prob, args.xref);
  const OptDev O = *args.opt;
  const InstDev id = args.inst[0];
  GridGroup g{scratch, args.gs, 0, &sdead};
  Inst<M, L> I;
  I.setup(w, id, args.x0, g.rank(), g.size(), P.nw);
  solve_instance<M, L>(g, I, P, O, args.u_init, args.info);
}

}  // namespace ptn
