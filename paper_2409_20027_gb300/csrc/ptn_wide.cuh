// ptn_wide.cuh -- the "wide" tier for state dimensions n >= 8 (quadrotor n = 12): one CTA
// per instance, one warp per time chunk, scan elements in shared memory and every
// element operation spread over the warp's lanes (ptn_wops.cuh).
//
// The solver logic is the one of ptn_solver.cuh: newton_solve, the IP and ADMM loops,
// residuals and the initial rollout are shared; the five passes of a Newton step
// (co-state, second-order expansion, value, state, rollout) are overloaded below for
// WideGroup.  Precision: the LQR data (Jacobians, Hessians, elements) are in L with the
// solves in SV, as in the narrow tier; the gradient (co-states, d), the rollouts and the
// merits are exact FP64 throughout (the exact_only trait), which keeps the per-step FP64
// work lane-parallel.
#pragma once
#include "ptn_solver.cuh"
#include "ptn_wops.cuh"

namespace ptn {

// ---------------------------------------------------------------------------
// group: rank = warp, size = number of warps of the CTA
struct WideGroup {
  char* scr;         // per-warp scratch, warp w at scr + w * scr_bytes
  size_t scr_bytes;
  char* xs;          // cross-warp scan slots: 2 buffers x nwarps x xs_bytes
  size_t xs_bytes;
  double* red;       // 8 doubles per warp

  __device__ int warp() const { return threadIdx.x >> 5; }
  __device__ int nwarps() const { return blockDim.x >> 5; }
  __device__ int rank() const { return warp(); }
  __device__ int size() const { return nwarps(); }
  __device__ bool dead() const { return false; }
  __device__ void sync() { __syncthreads(); }

  // every lane of a warp holds the warp's value; lane 0 contributes it.  Fixed order of
  // combination, so every thread gets the same result.
  template <int K>
  __device__ void reduce(double (&v)[K], unsigned maxmask) {
    static_assert(K <= 8, "at most 8 values per reduction");
    const int w = warp(), nw = nwarps();
    __syncthreads();
    if ((threadIdx.x & 31) == 0)
#pragma unroll
      for (int k = 0; k < K; k++) red[w * 8 + k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; k++) {
      double a = red[k];
      for (int i = 1; i < nw; i++) a = ((maxmask >> k) & 1u) ? fmax(a, red[i * 8 + k]) : a + red[i * 8 + k];
      v[k] = a;
    }
  }
  template <class T>
  __device__ T* slot(int buf, int w) const {
    return reinterpret_cast<T*>(xs + ((size_t)buf * nwarps() + w) * xs_bytes);
  }
};

template <>
struct multiplier_form_ok<WideGroup> {
  static constexpr bool value = false;
};
template <>
struct exact_only<WideGroup> {
  static constexpr bool value = true;
};

// per-warp shared scratch
template <class M, class L>
struct WScr {
  static constexpr int N = M::NX, U = M::NU, C = 2 * N + 1;
  // FP64 first (alignment)
  double K[N * N];       // inverse of I + C1 J2 (in SV: FP64, or FP32 in the first half)
  double col[N];
  double F64[N * N], G64[N * U];
  double x[N], u[U], xn[N], q[N], r[U], lam[N], v1[N], v2[N];
  double gr[2 * (N + U)];  // per constraint row terms
  double d[U];
  Aff<N, double> ca;     // co-state aggregate of this warp's chunk
  Val<N, L> e, agg, out;
  Aff<N, L> sa, so;      // state aggregate and a combination output
  L T1[N * N], T2[N * N], T3[N * N];
  L X[U * C];
  L F[N * N], G[N * U], Pm[N * N], Mm[N * U], Rm[U * U];
  L S[N * N], s[N], Gam[U * N], gam[U];
  L w1[N], w2[N], wu[U];
  int piv[N];
};

template <class M, class L>
__device__ __forceinline__ WScr<M, L>* wscr(const WideGroup& g) {
  return reinterpret_cast<WScr<M, L>*>(g.scr + (size_t)g.warp() * g.scr_bytes);
}

namespace wide {

using wops::lane_id;

// ---- lane-parallel stage terms (FP64) ----

// l_t (+ barrier / penalty) at (x, u); lplain: without the augmentation.  infeas is set
// when a barrier row is not strictly feasible.  gr: 2(N+U) doubles of scratch.
template <int N, int U>
__device__ double stage_cost_w(const ProbS<N, U>& P, const Aug& A, int t, const double* x, const double* u,
                               bool& infeas, double* lplain) {
  const int l = lane_id();
  double v = 0.0;
  if (l < N) {
    double s = 0.0;
    for (int j = 0; j < N; j++) s += P.Q[l * N + j] * (x[j] - P.xref[j]);
    v = (x[l] - P.xref[l]) * s;
  } else if (l < N + U) {
    const int i = l - N;
    double s = 0.0;
    for (int j = 0; j < U; j++) s += P.R[i * U + j] * (u[j] - P.uref[j]);
    v = (u[i] - P.uref[i]) * s;
  }
  const double lp = wops::wsum(v);
  if (lplain) *lplain = lp;
  double b = 0.0;
  bool bad = false;
  for (int r = l; r < P.nw; r += 32) {
    const double zk = P.isx[r] ? x[P.idx[r]] : u[P.idx[r]];
    const double w = P.sgn[r] * (zk - P.bnd[r]);
    if (A.kind == AUG_BARRIER) {
      if (!(w < 0.0)) bad = true;
      else b -= A.mu * log(-w);
    } else {
      const double qq = w - A.z[(size_t)t * P.nw + r] + A.v[(size_t)t * P.nw + r] / A.rho;
      b += 0.5 * A.rho * qq * qq;
    }
  }
  if (__any_sync(0xffffffffu, bad)) infeas = true;
  return lp + wops::wsum(b);
}

template <int N, int U>
__device__ double terminal_cost_w(const ProbS<N, U>& P, const double* x) {
  const int l = lane_id();
  double v = 0.0;
  if (l < N) {
    double s = 0.0;
    for (int j = 0; j < N; j++) s += P.Qf[l * N + j] * (x[j] - P.xref[j]);
    v = (x[l] - P.xref[l]) * s;
  }
  return wops::wsum(v);
}

// gradient of l_t + c_t into lx (N), lu (U) (shared); gr: per-row scratch (shared)
template <int N, int U>
__device__ void stage_grad_w(const ProbS<N, U>& P, const Aug& A, int t, const double* x, const double* u,
                             double* lx, double* lu, double* gr) {
  const int l = lane_id();
  for (int r = l; r < P.nw; r += 32) {
    const double zk = P.isx[r] ? x[P.idx[r]] : u[P.idx[r]];
    const double w = P.sgn[r] * (zk - P.bnd[r]);
    gr[r] = (A.kind == AUG_BARRIER) ? A.mu * P.sgn[r] / (-w)
                                    : A.rho * (w - A.z[(size_t)t * P.nw + r] + A.v[(size_t)t * P.nw + r] / A.rho) *
                                          P.sgn[r];
  }
  __syncwarp();
  if (l < N) {
    double s = 0.0;
    for (int j = 0; j < N; j++) s += (P.Q[l * N + j] + P.Q[j * N + l]) * (x[j] - P.xref[j]);
    for (int r = 0; r < P.nw; r++)
      if (P.isx[r] && P.idx[r] == l) s += gr[r];
    lx[l] = s;
  } else if (l < N + U) {
    const int i = l - N;
    double s = 0.0;
    for (int j = 0; j < U; j++) s += (P.R[i * U + j] + P.R[j * U + i]) * (u[j] - P.uref[j]);
    for (int r = 0; r < P.nw; r++)
      if (!P.isx[r] && P.idx[r] == i) s += gr[r];
    lu[i] = s;
  }
  __syncwarp();
}

template <int N, int U>
__device__ void terminal_grad_w(const ProbS<N, U>& P, const double* xT, double* g) {
  const int l = lane_id();
  if (l < N) {
    double s = 0.0;
    for (int j = 0; j < N; j++) s += (P.Qf[l * N + j] + P.Qf[j * N + l]) * (xT[j] - P.xref[j]);
    g[l] = s;
  }
  __syncwarp();
}

// adds the Hessians of l_t + c_t to Pm (N x N), Rm (U x U) (shared)
template <int N, int U, class L>
__device__ void stage_hess_add_w(const ProbS<N, U>& P, const Aug& A, const double* x, const double* u, L* Pm, L* Rm,
                                 double* gr) {
  const int l = lane_id();
  for (int r = l; r < P.nw; r += 32) {
    const double zk = P.isx[r] ? x[P.idx[r]] : u[P.idx[r]];
    const double w = P.sgn[r] * (zk - P.bnd[r]);
    gr[r] = (A.kind == AUG_BARRIER) ? A.mu / (w * w) : A.rho;
  }
  __syncwarp();
  for (int e = l; e < N * N; e += 32) {
    const int i = e / N, j = e % N;
    double v = P.Q[i * N + j] + P.Q[j * N + i];
    if (i == j)
      for (int r = 0; r < P.nw; r++)
        if (P.isx[r] && P.idx[r] == i) v += gr[r];
    Pm[e] += L(v);
  }
  for (int e = l; e < U * U; e += 32) {
    const int i = e / U, j = e % U;
    double v = P.R[i * U + j] + P.R[j * U + i];
    if (i == j)
      for (int r = 0; r < P.nw; r++)
        if (!P.isx[r] && P.idx[r] == i) v += gr[r];
    Rm[e] += L(v);
  }
  __syncwarp();
}

// ---- element operations (warp-cooperative; outputs distinct from inputs) ----

template <int N, class S>
__device__ void aff_identity(Aff<N, S>* a, bool zero_matrix) {
  for (int e = lane_id(); e < N * N; e += 32) a->M[e] = (!zero_matrix && e / N == e % N) ? S(1) : S(0);
  for (int i = lane_id(); i < N; i += 32) a->v[i] = S(0);
  __syncwarp();
}

template <int N, class L>
__device__ void val_identity(Val<N, L>* a) {
  for (int e = lane_id(); e < N * N; e += 32) {
    a->A[e] = (e / N == e % N) ? L(1) : L(0);
    a->C[e] = L(0);
    a->J[e] = L(0);
  }
  for (int i = lane_id(); i < N; i += 32) { a->eta[i] = L(0); a->b[i] = L(0); }
  __syncwarp();
}

template <int N, class S>
__device__ void aff_copy(const Aff<N, S>* a, Aff<N, S>* o) {
  wops::copy<N * N>(a->M, o->M);
  wops::copy<N>(a->v, o->v);
}
template <int N, class L>
__device__ void val_copy(const Val<N, L>* a, Val<N, L>* o) {
  wops::copy<sizeof(Val<N, L>) / sizeof(unsigned)>(reinterpret_cast<const unsigned*>(a),
                                                    reinterpret_cast<unsigned*>(o));
}

// co-state operator (M holds F^T):  v = a.v + a.M b.v,  M = a.M b.M  (a earlier)
template <int N, class S>
__device__ void costate_combine(const Aff<N, S>* a, const Aff<N, S>* b, Aff<N, S>* o) {
  wops::mm<N, N, N, false, false>(a->M, b->M, o->M);
  wops::mv<N, N, false>(a->M, b->v, o->v);
  for (int i = lane_id(); i < N; i += 32) o->v[i] += a->v[i];
  __syncwarp();
}

// state operator:  M = b.M a.M,  v = b.M a.v + b.v  (a earlier)
template <int N, class S>
__device__ void state_combine(const Aff<N, S>* a, const Aff<N, S>* b, Aff<N, S>* o) {
  wops::mm<N, N, N, false, false>(b->M, a->M, o->M);
  wops::mv<N, N, false>(b->M, a->v, o->v);
  for (int i = lane_id(); i < N; i += 32) o->v[i] += b->v[i];
  __syncwarp();
}

// value operator (e1 earlier, e2 later), same formulas as ValueOp: K = (I + C1 J2)^{-1}
// with C1 J2 formed in L and I + C1 J2 inverted in SV.  Returns false (warp-uniform)
// when I + C1 J2 is singular.
template <class SV, class M, class L>
__device__ bool val_combine(const Val<M::NX, L>* e1, const Val<M::NX, L>* e2, Val<M::NX, L>* o, WScr<M, L>* s) {
  constexpr int N = M::NX;
  const int l = lane_id();
  wops::mm<N, N, N, false, false>(e1->C, e2->J, s->T1);
  SV* K = reinterpret_cast<SV*>(s->K);
  for (int e = l; e < N * N; e += 32) K[e] = SV(s->T1[e]) + ((e / N == e % N) ? SV(1) : SV(0));
  __syncwarp();
  if (!wops::inv<N, SV>(K, s->piv, reinterpret_cast<SV*>(s->col))) return false;
  L* Kl = s->T3;
  for (int e = l; e < N * N; e += 32) Kl[e] = L(K[e]);
  __syncwarp();
  // A = A2 K A1
  wops::mm<N, N, N, false, false>(Kl, e1->A, s->T1);
  wops::mm<N, N, N, false, false>(e2->A, s->T1, o->A);
  // C = A2 K C1 A2^T + C2
  wops::mm<N, N, N, false, false>(Kl, e1->C, s->T1);
  wops::mm<N, N, N, false, false>(e2->A, s->T1, s->T2);
  wops::mm<N, N, N, false, true>(s->T2, e2->A, o->C);
  for (int e = l; e < N * N; e += 32) o->C[e] += e2->C[e];
  // b = A2 K (b1 + C1 eta2) + b2
  wops::mv<N, N, false>(e1->C, e2->eta, s->w1);
  for (int i = l; i < N; i += 32) s->w1[i] += e1->b[i];
  __syncwarp();
  wops::mv<N, N, false>(Kl, s->w1, s->w2);
  wops::mv<N, N, false>(e2->A, s->w2, o->b);
  for (int i = l; i < N; i += 32) o->b[i] += e2->b[i];
  // J = A1^T K^T J2 A1 + J1
  wops::mm<N, N, N, false, false>(e2->J, e1->A, s->T1);
  wops::mm<N, N, N, true, false>(Kl, s->T1, s->T2);
  wops::mm<N, N, N, true, false>(e1->A, s->T2, o->J);
  for (int e = l; e < N * N; e += 32) o->J[e] += e1->J[e];
  // eta = A1^T K^T (eta2 - J2 b1) + eta1
  wops::mv<N, N, false>(e2->J, e1->b, s->w1);
  for (int i = l; i < N; i += 32) s->w1[i] = e2->eta[i] - s->w1[i];
  __syncwarp();
  wops::mv<N, N, true>(Kl, s->w1, s->w2);
  wops::mv<N, N, true>(e1->A, s->w2, o->eta);
  for (int i = l; i < N; i += 32) o->eta[i] += e1->eta[i];
  __syncwarp();
  wops::symmetrize<N>(o->C);
  wops::symmetrize<N>(o->J);
  return true;
}

// element initialisation (P^-1-free form, as value_init) from the step data in s->F, G,
// Pm, Mm, Rm, d; into e.  R~ = R + alpha I factorised in SV.
template <class SV, class M, class L>
__device__ bool val_init(WScr<M, L>* s, double alpha, Val<M::NX, L>* e) {
  constexpr int N = M::NX, U = M::NU, C = 2 * N + 1;
  const int l = lane_id();
  SV Rt[U * U];
#pragma unroll
  for (int i = 0; i < U * U; i++) Rt[i] = SV(s->Rm[i]);
#pragma unroll
  for (int i = 0; i < U; i++) Rt[i * U + i] += SV(alpha);
  if (!ldlt<U, SV>(Rt)) return false;
  for (int q = l; q < U * C; q += 32) {
    const int i = q / C, c = q % C;
    s->X[q] = c < N ? s->Mm[c * U + i] : (c < 2 * N ? s->G[(c - N) * U + i] : L(s->d[i]));
  }
  __syncwarp();
  wops::ldlt_solve_cols<U, C, SV>(Rt, s->X);
  for (int q = l; q < N * N; q += 32) {
    const int i = q / N, j = q % N;
    L gm = L(0), mx = L(0), gg = L(0);
#pragma unroll
    for (int k = 0; k < U; k++) {
      gm += s->G[i * U + k] * s->X[k * C + j];
      mx += s->Mm[i * U + k] * s->X[k * C + j];
      gg += s->G[i * U + k] * s->X[k * C + N + j];
    }
    e->A[q] = s->F[q] - gm;
    e->J[q] = s->Pm[q] - mx;
    e->C[q] = gg;
  }
  for (int i = l; i < N; i += 32) {
    L et = L(0), bb = L(0);
#pragma unroll
    for (int k = 0; k < U; k++) {
      et += s->Mm[i * U + k] * s->X[k * C + 2 * N];
      bb += s->G[i * U + k] * s->X[k * C + 2 * N];
    }
    e->eta[i] = et;
    e->b[i] = -bb;
  }
  __syncwarp();
  wops::symmetrize<N>(e->J);
  wops::symmetrize<N>(e->C);
  return true;
}

// one feedback step from V_{t+1} = (s->S, s->s) with the step data in s->F, G, Pm, Mm,
// Rm, d (as riccati_step); writes s->Gam, s->gam and updates S, s in place.
template <class SV, class M, class L>
__device__ bool riccati_w(WScr<M, L>* s, double alpha) {
  constexpr int N = M::NX, U = M::NU, C = N + 1;
  const int l = lane_id();
  L* SF = s->T1;
  L* SG = s->T2;  // N x U
  wops::mm<N, N, N, false, false>(s->S, s->F, SF);
  wops::mm<N, N, U, false, false>(s->S, s->G, SG);
  // Qux = G^T S F + M^T (U x N) in X[:, :N]; d + G^T s in X[:, N]
  for (int q = l; q < U * C; q += 32) {
    const int i = q / C, j = q % C;
    L v = L(0);
    if (j < N) {
      for (int k = 0; k < N; k++) v += s->G[k * U + i] * SF[k * N + j];
      v += s->Mm[j * U + i];
    } else {
      for (int k = 0; k < N; k++) v += s->G[k * U + i] * s->s[k];
      v += L(s->d[i]);
    }
    s->X[q] = v;
  }
  // Q = R + G^T S G + alpha I, in every lane
  __syncwarp();
  SV Q[U * U];
#pragma unroll
  for (int i = 0; i < U; i++)
#pragma unroll
    for (int j = 0; j < U; j++) {
      L gsg = L(0);
      for (int k = 0; k < N; k++) gsg += s->G[k * U + i] * SG[k * U + j];
      Q[i * U + j] = SV(s->Rm[i * U + j]) + SV(gsg) + (i == j ? SV(alpha) : SV(0));
    }
  // keep Qux (U x N) for the S update, before the solve overwrites X
  L* Qux = s->T3;
  for (int q = l; q < U * N; q += 32) Qux[q] = s->X[(q / N) * C + (q % N)];
  __syncwarp();
  if (!ldlt<U, SV>(Q)) return false;
  wops::ldlt_solve_cols<U, C, SV>(Q, s->X);
  for (int q = l; q < U * N; q += 32) s->Gam[q] = -s->X[(q / N) * C + (q % N)];
  for (int i = l; i < U; i += 32) s->gam[i] = -s->X[i * C + N];
  __syncwarp();
  // S' = P + F^T S F + Qux^T Gam,  s' = F^T s + Qux^T gam
  L* Sn = s->T2;
  for (int q = l; q < N * N; q += 32) {
    const int i = q / N, j = q % N;
    L v = s->Pm[q];
    for (int k = 0; k < N; k++) v += s->F[k * N + i] * SF[k * N + j];
#pragma unroll
    for (int k = 0; k < U; k++) v += Qux[k * N + i] * s->Gam[k * N + j];
    Sn[q] = v;
  }
  for (int i = l; i < N; i += 32) {
    L v = L(0);
    for (int k = 0; k < N; k++) v += s->F[k * N + i] * s->s[k];
#pragma unroll
    for (int k = 0; k < U; k++) v += Qux[k * N + i] * s->gam[k];
    s->w1[i] = v;
  }
  __syncwarp();
  wops::copy<N * N>(Sn, s->S);
  wops::copy<N>(s->w1, s->s);
  wops::symmetrize<N>(s->S);
  return true;
}

// inclusive scan across warps of the elements in slot(0, w) of g; op(earlier, later,
// out, scratch).  Returns the buffer holding the results; ok is AND-ed with op's result.
template <class E, class Op>
__device__ int scan_warps(WideGroup& g, const Op& op, bool suffix, bool& ok) {
  const int w = g.warp(), nw = g.nwarps();
  int cur = 0;
  __syncthreads();
  for (int off = 1; off < nw; off <<= 1) {
    E* src = g.slot<E>(cur, w);
    E* dst = g.slot<E>(cur ^ 1, w);
    const int o = suffix ? w + off : w - off;
    if (o >= 0 && o < nw) {
      E* other = g.slot<E>(cur, o);
      ok &= suffix ? op(src, other, dst) : op(other, src, dst);
    } else {
      wops::copy<sizeof(E) / sizeof(unsigned)>(reinterpret_cast<const unsigned*>(src),
                                                reinterpret_cast<unsigned*>(dst));
    }
    __syncthreads();
    cur ^= 1;
  }
  return cur;
}

__device__ __forceinline__ bool wall(bool v) {
  // block-wide AND (uniform result)
  return __syncthreads_and(v ? 1 : 0) != 0;
}

}  // namespace wide

// ---------------------------------------------------------------------------
// pass 1: exact co-state pass (Alg. 1) in FP64.  Returns max_t |d_t|_inf.
template <class M, class L>
__device__ double costate_pass(WideGroup& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const Aug& A,
                               bool exact) {
  (void)exact;
  constexpr int N = M::NX, U = M::NU;
  WScr<M, L>* s = wscr<M, L>(g);
  const int l = wide::lane_id();
  Aff<N, double>* agg = &s->ca;
  wide::aff_identity<N>(agg, false);
  if (I.last) {
    wide::terminal_grad_w<N, U>(P, I.xn + (size_t)I.T * N, s->lam);
    for (int i = l; i < N; i += 32) agg->v[i] = s->lam[i];
    for (int e = l; e < N * N; e += 32) agg->M[e] = 0.0;
    __syncwarp();
  }
  for (int t = I.b - 1; t >= I.a; t--) {
    const double* x = I.xn + (size_t)t * N;
    const double* u = I.un + (size_t)t * U;
    wops::step_jac<M, double>(P.integ, P.dt, P.prm, x, u, s->F64, s->G64);
    for (int e = l; e < N * N; e += 32) {
      const double E = s->F64[e] - ((e / N == e % N) ? 1.0 : 0.0);
      I.F64[(size_t)t * N * N + e] = E;
      I.E[(size_t)t * N * N + e] = L(E);
    }
    for (int e = l; e < N * U; e += 32) {
      I.G64[(size_t)t * N * U + e] = s->G64[e];
      I.Gm[(size_t)t * N * U + e] = L(s->G64[e]);
    }
    wide::stage_grad_w<N, U>(P, A, t, x, u, s->q, s->r, s->gr);
    // agg <- (q, F^T) o agg:  v = q + F^T v,  M = F^T M (the terminal chunk keeps M = 0)
    wops::mv<N, N, true>(s->F64, agg->v, s->v1);
    for (int i = l; i < N; i += 32) agg->v[i] = s->v1[i] + s->q[i];
    __syncwarp();
    if (!I.last) {
      double* Mn = reinterpret_cast<double*>(s->K);
      wops::mm<N, N, N, true, false>(s->F64, agg->M, Mn);
      wops::copy<N * N>(Mn, agg->M);
    }
  }
  // exclusive suffix scan across warps
  wide::aff_copy<N>(agg, g.slot<Aff<N, double>>(0, g.warp()));
  bool ok = true;
  auto op = [&](const Aff<N, double>* a, const Aff<N, double>* b, Aff<N, double>* o) {
    wide::costate_combine<N>(a, b, o);
    return true;
  };
  const int cur = wide::scan_warps<Aff<N, double>>(g, op, true, ok);
  double* lam = s->lam;
  if (!I.last) {
    const Aff<N, double>* nx = g.slot<Aff<N, double>>(cur, g.warp() + 1);
    for (int i = l; i < N; i += 32) lam[i] = nx->v[i];
  }
  __syncwarp();
  for (int i = 0; i < N; i++) I.lamb[i] = lam[i];
  if (I.last)
    for (int i = l; i < N; i += 32) I.lam[(size_t)I.T * N + i] = lam[i];
  double dmax = 0.0;
  for (int t = I.b - 1; t >= I.a; t--) {
    const double* x = I.xn + (size_t)t * N;
    const double* u = I.un + (size_t)t * U;
    const double* E = I.F64 + (size_t)t * N * N;
    const double* G = I.G64 + (size_t)t * N * U;
    wide::stage_grad_w<N, U>(P, A, t, x, u, s->q, s->r, s->gr);
    // d = r + G^T lam_{t+1};  lam_t = q + (I + E)^T lam_{t+1}
    double dl = 0.0;
    if (l < U) {
      double v = s->r[l];
      for (int k = 0; k < N; k++) v += G[k * U + l] * lam[k];
      I.d[(size_t)t * U + l] = v;
      dl = fabs(v);
      dl = isfinite(dl) ? dl : INFINITY;
    }
    dmax = fmax(dmax, wops::wmax(dl));
    double ln = 0.0;
    if (l < N) {
      ln = lam[l] + s->q[l];
      for (int k = 0; k < N; k++) ln += E[k * N + l] * lam[k];
    }
    __syncwarp();
    if (l < N) {
      lam[l] = ln;
      I.lam[(size_t)t * N + l] = ln;
    }
    __syncwarp();
  }
  double red[1] = {dmax};
  g.template reduce<1>(red, 1u);
  return red[0];
}

// pass 2: second-order expansion (Sec. III-C); Hessian contractions in L by lane-parallel
// hyper-dual numbers, stage Hessians in FP64 added and rounded to L.
template <class M, class L>
__device__ void quadratize(WideGroup& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const Aug& A) {
  constexpr int N = M::NX, U = M::NU;
  WScr<M, L>* s = wscr<M, L>(g);
  const int l = wide::lane_id();
  for (int t = I.a; t < I.b; t++) {
    const double* x = I.xn + (size_t)t * N;
    const double* u = I.un + (size_t)t * U;
    const double* lam1 = (t + 1 == I.b) ? I.lamb : I.lam + (size_t)(t + 1) * N;
    wops::step_hess<M, L>(P.integ, P.dt, P.prm, x, u, lam1, s->Pm, s->Mm, s->Rm);
    wide::stage_hess_add_w<N, U, L>(P, A, x, u, s->Pm, s->Rm, s->gr);
    for (int e = l; e < N * N; e += 32) I.Pm[(size_t)t * N * N + e] = s->Pm[e];
    for (int e = l; e < N * U; e += 32) I.Mm[(size_t)t * N * U + e] = s->Mm[e];
    for (int e = l; e < U * U; e += 32) I.Rm[(size_t)t * U * U + e] = s->Rm[e];
    __syncwarp();
  }
  if (I.last)
    for (int e = l; e < N * N; e += 32)
      I.Pm[(size_t)I.T * N * N + e] = L(P.Qf[e] + P.Qf[(e % N) * N + e / N]);
  __syncwarp();
}

// loads the LQR data of step t into the warp's scratch (F = I + E)
template <class M, class L>
__device__ void load_step(Inst<M, L>& I, WScr<M, L>* s, int t) {
  constexpr int N = M::NX, U = M::NU;
  const int l = wide::lane_id();
  for (int e = l; e < N * N; e += 32) {
    s->F[e] = I.E[(size_t)t * N * N + e] + ((e / N == e % N) ? L(1) : L(0));
    s->Pm[e] = I.Pm[(size_t)t * N * N + e];
  }
  for (int e = l; e < N * U; e += 32) {
    s->G[e] = I.Gm[(size_t)t * N * U + e];
    s->Mm[e] = I.Mm[(size_t)t * N * U + e];
  }
  for (int e = l; e < U * U; e += 32) s->Rm[e] = I.Rm[(size_t)t * U * U + e];
  for (int i = l; i < U; i += 32) s->d[i] = I.d[(size_t)t * U + i];
  __syncwarp();
}

// pass 3: value suffix scan (Alg. 2) + feedback sweep
template <class M, class L, class SV>
__device__ bool value_pass(WideGroup& g, Inst<M, L>& I, double alpha, const double* qx = nullptr) {
  constexpr int N = M::NX, U = M::NU;
  WScr<M, L>* s = wscr<M, L>(g);
  const int l = wide::lane_id();
  bool ok = true, have = false;
  Val<N, L>* agg = &s->agg;
  wide::val_identity<N>(agg);
  if (I.last) {
    for (int e = l; e < N * N; e += 32) {
      agg->A[e] = L(0);
      agg->C[e] = L(0);
      agg->J[e] = I.Pm[(size_t)I.T * N * N + e];
    }
    for (int i = l; i < N; i += 32) {
      agg->eta[i] = qx ? L(-qx[(size_t)I.T * N + i]) : L(0);
      agg->b[i] = L(0);
    }
    __syncwarp();
    have = true;
  }
  for (int t = I.b - 1; t >= I.a; t--) {
    load_step(I, s, t);
    ok &= wide::val_init<SV>(s, alpha, &s->e);
    if (qx) {
      for (int i = l; i < N; i += 32) s->e.eta[i] -= L(qx[(size_t)t * N + i]);
      __syncwarp();
    }
    if (!have) {
      wide::val_copy<N>(&s->e, agg);
      have = true;
    } else {
      ok &= wide::val_combine<SV>(&s->e, agg, &s->out, s);
      wide::val_copy<N>(&s->out, agg);
    }
  }
  wide::val_copy<N>(agg, g.slot<Val<N, L>>(0, g.warp()));
  auto op = [&](const Val<N, L>* a, const Val<N, L>* b, Val<N, L>* o) { return wide::val_combine<SV>(a, b, o, s); };
  const int cur = wide::scan_warps<Val<N, L>>(g, op, true, ok);
  if (I.last) {
    for (int e = l; e < N * N; e += 32) s->S[e] = I.Pm[(size_t)I.T * N * N + e];
    for (int i = l; i < N; i += 32) s->s[i] = qx ? L(qx[(size_t)I.T * N + i]) : L(0);
  } else {
    const Val<N, L>* nx = g.slot<Val<N, L>>(cur, g.warp() + 1);
    for (int e = l; e < N * N; e += 32) s->S[e] = nx->J[e];
    for (int i = l; i < N; i += 32) s->s[i] = -nx->eta[i];
  }
  __syncwarp();
  for (int t = I.b - 1; t >= I.a; t--) {
    load_step(I, s, t);
    ok &= wide::riccati_w<SV>(s, alpha);
    if (qx) {
      for (int i = l; i < N; i += 32) s->s[i] += L(qx[(size_t)t * N + i]);
    }
    for (int e = l; e < U * N; e += 32) I.Gam[(size_t)t * U * N + e] = s->Gam[e];
    for (int i = l; i < U; i += 32) I.gam[(size_t)t * U + i] = s->gam[i];
    __syncwarp();
  }
  return wide::wall(ok);
}

// pass 4: state prefix scan (Alg. 3) and the model terms G1, G2
template <class M, class L>
__device__ void state_pass(WideGroup& g, Inst<M, L>& I, double& G1, double& G2) {
  constexpr int N = M::NX, U = M::NU;
  WScr<M, L>* s = wscr<M, L>(g);
  const int l = wide::lane_id();
  const bool first = (I.a == 0);
  Aff<N, L>* agg = &s->sa;
  wide::aff_identity<N>(agg, first);  // the first element has F = 0
  for (int t = I.a; t < I.b; t++) {
    load_step(I, s, t);
    for (int i = l; i < U * N; i += 32) s->Gam[i] = I.Gam[(size_t)t * U * N + i];
    for (int i = l; i < U; i += 32) s->gam[i] = I.gam[(size_t)t * U + i];
    __syncwarp();
    // Fc = F + G Gam (T1), e = G gam (w1)
    wops::mm<N, U, N, false, false>(s->G, s->Gam, s->T1);
    for (int q = l; q < N * N; q += 32) s->T1[q] += s->F[q];
    wops::mv<N, U, false>(s->G, s->gam, s->w1);
    // agg <- (Fc, e) after agg
    wops::mv<N, N, false>(s->T1, agg->v, s->w2);
    for (int i = l; i < N; i += 32) agg->v[i] = s->w2[i] + s->w1[i];
    __syncwarp();
    if (!first) {
      wops::mm<N, N, N, false, false>(s->T1, agg->M, s->T2);
      wops::copy<N * N>(s->T2, agg->M);
    }
  }
  wide::aff_copy<N>(agg, g.slot<Aff<N, L>>(0, g.warp()));
  bool ok = true;
  auto op = [&](const Aff<N, L>* a, const Aff<N, L>* b, Aff<N, L>* o) {
    wide::state_combine<N>(a, b, o);
    return true;
  };
  const int cur = wide::scan_warps<Aff<N, L>>(g, op, false, ok);
  L* dx = s->w2;
  if (first) {
    for (int i = l; i < N; i += 32) dx[i] = L(0);
  } else {
    const Aff<N, L>* pv = g.slot<Aff<N, L>>(cur, g.warp() - 1);
    for (int i = l; i < N; i += 32) dx[i] = pv->v[i];
  }
  __syncwarp();
  double g1 = 0.0, g2 = 0.0;
  for (int t = I.a; t < I.b; t++) {
    load_step(I, s, t);
    for (int i = l; i < U * N; i += 32) s->Gam[i] = I.Gam[(size_t)t * U * N + i];
    for (int i = l; i < U; i += 32) s->gam[i] = I.gam[(size_t)t * U + i];
    __syncwarp();
    // du = Gam dx + gam
    wops::mv<U, N, false>(s->Gam, dx, s->wu);
    for (int i = l; i < U; i += 32) {
      s->wu[i] += s->gam[i];
      I.du[(size_t)t * U + i] = s->wu[i];
    }
    for (int i = l; i < N; i += 32) I.dx[(size_t)t * N + i] = dx[i];
    __syncwarp();
    // model terms
    double a1 = 0.0, a2 = 0.0;
    if (l < U) a1 = s->d[l] * double(s->wu[l]);
    if (l < N) {
      L pd = L(0), md = L(0);
      for (int k = 0; k < N; k++) pd += s->Pm[l * N + k] * dx[k];
      for (int k = 0; k < U; k++) md += s->Mm[l * U + k] * s->wu[k];
      a2 += double(dx[l] * (L(0.5) * pd + md));
    } else if (l < N + U) {
      const int i = l - N;
      L rd = L(0);
      for (int k = 0; k < U; k++) rd += s->Rm[i * U + k] * s->wu[k];
      a2 += double(L(0.5) * s->wu[i] * rd);
    }
    g1 += wops::wsum(a1);
    g2 += wops::wsum(a2);
    // dx <- F dx + G du
    wops::mv<N, N, false>(s->F, dx, s->w1);
    wops::mv<N, U, false, true>(s->G, s->wu, s->w1);
    wops::copy<N>(s->w1, dx);
  }
  if (I.last) {
    double a2 = 0.0;
    if (l < N) {
      L pd = L(0);
      for (int k = 0; k < N; k++) pd += I.Pm[(size_t)I.T * N * N + l * N + k] * dx[k];
      a2 = double(L(0.5) * dx[l] * pd);
      I.dx[(size_t)I.T * N + l] = dx[l];
    }
    g2 += wops::wsum(a2);
    __syncwarp();
  }
  double red[2] = {g1, g2};
  g.template reduce<2>(red, 0u);
  G1 = red[0];
  G2 = red[1];
}

// closed-loop nonlinear rollout for step size s by multiple shooting (as rollout()),
// always in FP64 (precise): states and merits FP64, chunk Jacobians in L.
template <class M, class L>
__device__ int rollout(WideGroup& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const OptDev& O, const Aug& A,
                       double sstep, bool precise, double* Jm, int* iters, int max_iter) {
  (void)precise;
  constexpr int N = M::NX, U = M::NU;
  WScr<M, L>* s = wscr<M, L>(g);
  const int l = wide::lane_id();
  const bool own = (I.a < I.b);
  const bool first = (I.a == 0);
  double* X = s->v1;   // chunk start
  double* Xn = s->v2;  // predicted right boundary
  for (int i = l; i < N; i += 32) {
    X[i] = first ? I.x0[i] : I.xn[(size_t)I.a * N + i] + sstep * double(I.dx[(size_t)I.a * N + i]);
    if (own && !I.last) Xn[i] = I.xn[(size_t)I.b * N + i] + sstep * double(I.dx[(size_t)I.b * N + i]);
  }
  __syncwarp();
  bool conv = false, feas = true;
  double J = INFINITY;
  double* xt = s->x;
  double* ut = s->u;
  for (int it = 0; it < max_iter; it++) {
    if (own)
      for (int i = l; i < N; i += 32) I.xc[(size_t)I.a * N + i] = X[i];
    for (int i = l; i < N; i += 32) xt[i] = X[i];
    Aff<N, L>* el = &s->sa;
    wide::aff_identity<N>(el, false);
    double cost = 0.0;
    bool inf = false;
    __syncwarp();
    for (int t = I.a; t < I.b; t++) {
      const L* Gam = I.Gam + (size_t)t * U * N;
      const double* xh = I.xn + (size_t)t * N;
      const double* uh = I.un + (size_t)t * U;
      if (l < U) {
        double v = uh[l] + sstep * double(I.gam[(size_t)t * U + l]);
        for (int j = 0; j < N; j++) v += double(Gam[l * N + j]) * (xt[j] - xh[j]);
        ut[l] = v;
        I.uc[(size_t)t * U + l] = v;
      }
      if (t > I.a)
        for (int i = l; i < N; i += 32) I.xc[(size_t)t * N + i] = xt[i];
      __syncwarp();
      cost += wide::stage_cost_w<N, U>(P, A, t, xt, ut, inf, nullptr);
      // FP64 step (every lane) and the closed-loop Jacobian F + G Gam in L
      double xnext[N];
      step<M>(P.integ, P.dt, P.prm, xt, ut, xnext);
      wops::step_jac<M, L>(P.integ, P.dt, P.prm, xt, ut, s->F, s->G);
      for (int q = l; q < U * N; q += 32) s->Gam[q] = Gam[q];
      __syncwarp();
      wops::mm<N, U, N, false, false>(s->G, s->Gam, s->T1);
      for (int q = l; q < N * N; q += 32) s->T1[q] += s->F[q];
      __syncwarp();
      if (!first) {
        wops::mm<N, N, N, false, false>(s->T1, el->M, s->T2);
        wops::copy<N * N>(s->T2, el->M);
      }
      for (int i = l; i < N; i += 32) xt[i] = xnext[i];
      __syncwarp();
    }
    double rmax = 0.0, xmax = 0.0;
    bool nonfin = !isfinite(cost);
    if (first) {
      for (int q = l; q < N * N; q += 32) el->M[q] = L(0);
    }
    if (I.last) {
      for (int i = l; i < N; i += 32) {
        I.xc[(size_t)I.T * N + i] = xt[i];
        el->v[i] = L(0);
      }
      cost += wide::terminal_cost_w<N, U>(P, xt);
    } else if (own) {
      double rl = 0.0;
      for (int i = l; i < N; i += 32) {
        const double r = xt[i] - Xn[i];
        el->v[i] = L(r);
        rl = fmax(rl, fabs(r));
      }
      rmax = wops::wmax(rl);
    }
    double xl = 0.0;
    bool nf = false;
    for (int i = l; i < N; i += 32) {
      nf |= !isfinite(xt[i]);
      xl = fmax(xl, fabs(xt[i]));
    }
    xmax = wops::wmax(xl);
    nonfin |= __any_sync(0xffffffffu, nf);
    if (nonfin) rmax = INFINITY;
    __syncwarp();
    wide::aff_copy<N>(el, g.slot<Aff<N, L>>(0, g.warp()));
    bool ok = true;
    auto op = [&](const Aff<N, L>* a, const Aff<N, L>* b, Aff<N, L>* o) {
      wide::state_combine<N>(a, b, o);
      return true;
    };
    const int cur = wide::scan_warps<Aff<N, L>>(g, op, false, ok);
    double red[5] = {rmax, xmax, cost, inf ? 1.0 : 0.0, nonfin ? 1.0 : 0.0};
    g.template reduce<5>(red, 0x1bu);
    if (iters) *iters = it + 1;
    if (red[4] > 0.0) return ROLL_FAIL;
    if (red[0] <= O.roll_tol * (1.0 + red[1])) {
      conv = true;
      feas = !(red[3] > 0.0);
      J = red[2];
      break;
    }
    if (own) {
      L* dv = s->w1;
      if (first) {
        for (int i = l; i < N; i += 32) dv[i] = L(0);
      } else {
        const Aff<N, L>* pv = g.slot<Aff<N, L>>(cur, g.warp() - 1);
        for (int i = l; i < N; i += 32) dv[i] = pv->v[i];
      }
      __syncwarp();
      wops::mv<N, N, false>(el->M, dv, s->w2);
      for (int i = l; i < N; i += 32) {
        if (!first) X[i] += double(dv[i]);
        if (!I.last) Xn[i] = xt[i] + double(s->w2[i]);
      }
      __syncwarp();
    }
  }
  *Jm = J;
  if (!conv) return ROLL_FAIL;
  return (feas && isfinite(J)) ? ROLL_OK : ROLL_INFEASIBLE;
}

// ---------------------------------------------------------------------------
// one CTA per instance, one warp per chunk
template <class M, class L, class SV>
__global__ void __launch_bounds__(512) k_solve_wide(KArgs args, Work<L> w) {
  constexpr int N = M::NX, U = M::NU;
  extern __shared__ __align__(16) char smem[];
  ProbS<N, U>& P = *reinterpret_cast<ProbS<N, U>*>(smem);
  size_t off = (sizeof(ProbS<N, U>) + 15) & ~size_t(15);
  const int nw = blockDim.x >> 5;
  WideGroup g;
  g.red = reinterpret_cast<double*>(smem + off);
  off += (size_t)8 * 8 * nw;
  g.scr_bytes = (sizeof(WScr<M, L>) + 15) & ~size_t(15);
  g.scr = smem + off;
  off += g.scr_bytes * nw;
  constexpr size_t xb = sizeof(Val<N, L>) > sizeof(Aff<N, double>) ? sizeof(Val<N, L>) : sizeof(Aff<N, double>);
  g.xs_bytes = (xb + 15) & ~size_t(15);
  g.xs = smem + off;
  const int bi = blockIdx.x;
  if (bi >= args.B) return;
  load_prob<N, U>(P, *args.prob, args.xref ? args.xref + (size_t)bi * N : nullptr, args.inst[bi].dt);
  const OptDev& O = *args.opt;  // read where used (a local copy would hold ~50 registers)
  const InstDev id = args.inst[bi];
  Inst<M, L> I;
  I.setup(w, id, args.x0 + (size_t)bi * N, g.warp(), nw, P.nw);
  solve_instance<M, L, SV>(g, I, P, O, args.u_init ? args.u_init + (size_t)id.uoff * U : nullptr, args.info + bi);
}

template <class M, class L>
constexpr size_t wide_smem_bytes(int nwarps) {
  constexpr int N = M::NX, U = M::NU;
  constexpr size_t xb = sizeof(Val<N, L>) > sizeof(Aff<N, double>) ? sizeof(Val<N, L>) : sizeof(Aff<N, double>);
  return ((sizeof(ProbS<N, U>) + 15) & ~size_t(15)) + (size_t)8 * 8 * nwarps +
         ((sizeof(WScr<M, L>) + 15) & ~size_t(15)) * nwarps + 2 * ((xb + 15) & ~size_t(15)) * nwarps;
}

// ---------------------------------------------------------------------------
// Adjoint for the wide tier (same quantities as adjoint_instance, with L = double).
//
// Parameter derivatives of one step, lane-parallel: pair q = (j, k) of z_j = (x, u)_j and
// model constant k is one evaluation with nested dual numbers (outer: z_j, inner: p_k);
// it gives Hzp[j][k] = d2 (lam^T f) / dz_j dp_k, and for j = 0 also the column
// fp[:, k] = df / dp_k.  Calls back visit(j, k, hzp_jk) and visitp(k, fp column).
template <class M, class Fh, class Fp>
__device__ void param_pairs(int integ, double dt, const double* prm, const double* x, const double* u,
                            const double* lam, const Fh& visit, const Fp& visitp) {
  constexpr int N = M::NX, U = M::NU, K = N + U, NP = M::NP;
  using PD = Dual<double, 1>;
  using D = Dual<PD, 1>;
  for (int q = wide::lane_id(); q < K * NP; q += 32) {
    const int j = q / NP, k = q % NP;
    PD pp[NP];
#pragma unroll
    for (int i = 0; i < NP; i++) { pp[i] = PD(prm[i]); pp[i].d[0] = (i == k) ? 1.0 : 0.0; }
    D xd[N], ud[U], xn[N];
#pragma unroll
    for (int i = 0; i < N; i++) { xd[i] = D(PD(x[i])); xd[i].d[0] = PD((i == j) ? 1.0 : 0.0); }
#pragma unroll
    for (int i = 0; i < U; i++) { ud[i] = D(PD(u[i])); ud[i].d[0] = PD((N + i == j) ? 1.0 : 0.0); }
    step<M, D, PD>(integ, dt, pp, xd, ud, xn);
    double h = 0.0;
#pragma unroll
    for (int i = 0; i < N; i++) h += lam[i] * xn[i].d[0].d[0];
    visit(j, k, h);
    if (j == 0) {
      double col[N];
#pragma unroll
      for (int i = 0; i < N; i++) col[i] = xn[i].v.d[0];
      visitp(k, col);
    }
  }
}

// envelope and adjoint sums of one warp, lane 0 holds them after the calls
template <class M>
__device__ int adjoint_wide(WideGroup& g, Inst<M, double>& I, const ProbS<M::NX, M::NU>& P, const AdjArgs& aa,
                            const InstDev& id, int bi) {
  constexpr int N = M::NX, U = M::NU, NP = M::NP, KO = 3 * N + U + NP;
  using L = double;
  WScr<M, L>* s = wscr<M, L>(g);
  const int l = wide::lane_id();
  Aug A;
  A.kind = AUG_BARRIER; A.mu = aa.mu; A.rho = 1.0; A.z = nullptr; A.v = nullptr;
  costate_pass(g, I, P, A, true);
  const bool lin = aa.gx || aa.gu;
  int rc = ST_OK;
  double* qx = aa.qx + (size_t)id.xoff * N;
  if (lin) {
    quadratize(g, I, P, A);
    for (int t = I.a; t < I.b; t++) {
      for (int i = l; i < U; i += 32) I.d[(size_t)t * U + i] = aa.gu ? -aa.gu[((size_t)id.uoff + t) * U + i] : 0.0;
      for (int i = l; i < N; i += 32) qx[(size_t)t * N + i] = aa.gx ? -aa.gx[((size_t)id.xoff + t) * N + i] : 0.0;
    }
    if (I.last)
      for (int i = l; i < N; i += 32) qx[(size_t)I.T * N + i] = aa.gx ? -aa.gx[((size_t)id.xoff + I.T) * N + i] : 0.0;
    __syncwarp();
    if (!value_pass<M, L, double>(g, I, 0.0, qx)) rc = ST_ENUM;
  }
  if (__syncthreads_or(rc != ST_OK)) return ST_ENUM;
  if (lin) {
    double G1, G2;
    state_pass(g, I, G1, G2);  // dx = w_x, du = w_u
  }
  // per-warp accumulators in shared memory (T1 is free once the LQR passes are done)
  double* env = reinterpret_cast<double*>(s->T1);
  double* adj = env + KO;
  for (int i = l; i < 2 * KO; i += 32) env[i] = 0.0;
  __syncwarp();
  // quadratic-weight envelope terms
  for (int t = I.a; t < I.b; t++) {
    if (l < N) {
      const double e = I.xn[(size_t)t * N + l] - P.xref[l];
      env[N + l] += e * e;
    } else if (l < N + U) {
      const double e = I.un[(size_t)t * U + (l - N)] - P.uref[l - N];
      env[2 * N + (l - N)] += e * e;
    }
  }
  if (I.last && l < N) {
    const double e = I.xn[(size_t)I.T * N + l] - P.xref[l];
    env[2 * N + U + l] = e * e;
  }
  __syncwarp();
  double* envp = env + 3 * N + U;
  double* adjp = adj + 3 * N + U;
  if (lin) {
    // nu: co-state-type suffix scan with c_t = q_t + P_t w_t + M_t w_{u,t} (FP64)
    auto cterm = [&](int t, double* c) {
      if (l < N) {
        const double* Pt = I.Pm + (size_t)t * N * N;
        const double* w = I.dx + (size_t)t * N;
        double v = qx[(size_t)t * N + l];
        for (int j = 0; j < N; j++) v += Pt[l * N + j] * w[j];
        if (t < I.T) {
          const double* Mt = I.Mm + (size_t)t * N * U;
          const double* wu = I.du + (size_t)t * U;
          for (int j = 0; j < U; j++) v += Mt[l * U + j] * wu[j];
        }
        c[l] = v;
      }
      __syncwarp();
    };
    Aff<N, double>* agg = &s->ca;
    wide::aff_identity<N>(agg, false);
    if (I.last) {
      cterm(I.T, s->v1);
      for (int i = l; i < N; i += 32) agg->v[i] = s->v1[i];
      for (int e = l; e < N * N; e += 32) agg->M[e] = 0.0;
      __syncwarp();
    }
    for (int t = I.b - 1; t >= I.a; t--) {
      const double* E = I.F64 + (size_t)t * N * N;
      cterm(t, s->v1);
      // v = c + (I + E)^T v
      wops::mv<N, N, true>(E, agg->v, s->v2);
      for (int i = l; i < N; i += 32) agg->v[i] += s->v2[i] + s->v1[i];
      __syncwarp();
      if (!I.last) {
        double* Mn = s->K;
        wops::mm<N, N, N, true, false>(E, agg->M, Mn);
        for (int e = l; e < N * N; e += 32) agg->M[e] += Mn[e];
        __syncwarp();
      }
    }
    wide::aff_copy<N>(agg, g.slot<Aff<N, double>>(0, g.warp()));
    bool ok = true;
    auto op = [&](const Aff<N, double>* a, const Aff<N, double>* b, Aff<N, double>* o) {
      wide::costate_combine<N>(a, b, o);
      return true;
    };
    const int cur = wide::scan_warps<Aff<N, double>>(g, op, true, ok);
    double* nu = s->lam;
    if (I.last) {
      cterm(I.T, nu);
    } else {
      const Aff<N, double>* nx = g.slot<Aff<N, double>>(cur, g.warp() + 1);
      for (int i = l; i < N; i += 32) nu[i] = nx->v[i];
      __syncwarp();
    }
    for (int t = I.b - 1; t >= I.a; t--) {
      const double* lam1 = (t + 1 == I.b) ? I.lamb : I.lam + (size_t)(t + 1) * N;
      const double* w = I.dx + (size_t)t * N;
      const double* wu = I.du + (size_t)t * U;
      // contractions with nu_{t+1}, w_t and the parameter derivatives of step t
      double pa[NP], pe[NP];
#pragma unroll
      for (int k = 0; k < NP; k++) { pa[k] = 0.0; pe[k] = 0.0; }
      param_pairs<M>(
          P.integ, P.dt, P.prm, I.xn + (size_t)t * N, I.un + (size_t)t * U, lam1,
          [&](int j, int k, double h) {
            const double wj = j < N ? w[j] : wu[j - N];
#pragma unroll
            for (int kk = 0; kk < NP; kk++)
              if (kk == k) pa[kk] += wj * h;
          },
          [&](int k, const double* col) {
            double e = 0.0, a = 0.0;
            for (int i = 0; i < N; i++) {
              e += lam1[i] * col[i];
              a += nu[i] * col[i];
            }
#pragma unroll
            for (int kk = 0; kk < NP; kk++)
              if (kk == k) { pe[kk] += e; pa[kk] += a; }
          });
#pragma unroll
      for (int k = 0; k < NP; k++) {
        const double se = wops::wsum(pe[k]), sa = wops::wsum(pa[k]);
        if (l == 0) { envp[k] += se; adjp[k] += sa; }
      }
      __syncwarp();
      // nu_t = c_t + (I + E)^T nu_{t+1}
      const double* E = I.F64 + (size_t)t * N * N;
      cterm(t, s->v1);
      wops::mv<N, N, true>(E, nu, s->v2);
      for (int i = l; i < N; i += 32) nu[i] += s->v2[i] + s->v1[i];
      __syncwarp();
    }
    if (I.a == 0 && I.b > 0)
      for (int i = l; i < N; i += 32) adj[i] = nu[i];
    // quadratic-weight adjoint terms
    for (int t = I.a; t < I.b; t++) {
      if (l < N) adj[N + l] += I.dx[(size_t)t * N + l] * 2.0 * (I.xn[(size_t)t * N + l] - P.xref[l]);
      else if (l < N + U)
        adj[2 * N + (l - N)] += I.du[(size_t)t * U + (l - N)] * 2.0 * (I.un[(size_t)t * U + (l - N)] - P.uref[l - N]);
    }
    if (I.last && l < N)
      adj[2 * N + U + l] = I.dx[(size_t)I.T * N + l] * 2.0 * (I.xn[(size_t)I.T * N + l] - P.xref[l]);
    __syncwarp();
  } else {
    for (int t = I.a; t < I.b; t++) {
      const double* lam1 = (t + 1 == I.b) ? I.lamb : I.lam + (size_t)(t + 1) * N;
      double pe[NP];
#pragma unroll
      for (int k = 0; k < NP; k++) pe[k] = 0.0;
      param_pairs<M>(
          P.integ, P.dt, P.prm, I.xn + (size_t)t * N, I.un + (size_t)t * U, lam1, [&](int, int, double) {},
          [&](int k, const double* col) {
            double e = 0.0;
            for (int i = 0; i < N; i++) e += lam1[i] * col[i];
#pragma unroll
            for (int kk = 0; kk < NP; kk++)
              if (kk == k) pe[kk] += e;
          });
#pragma unroll
      for (int k = 0; k < NP; k++) {
        const double se = wops::wsum(pe[k]);
        if (l == 0) envp[k] += se;
      }
      __syncwarp();
    }
  }
  // combine over warps: out = gJ env - adj, lane 0 of each warp contributes
  for (int c = 0; c < KO; c += 8) {
    double r[8];
#pragma unroll
    for (int i = 0; i < 8; i++) r[i] = (c + i < KO) ? aa.gJ * env[c + i] - adj[c + i] : 0.0;
    g.template reduce<8>(r, 0u);
    if (g.rank() == 0 && l == 0) {
#pragma unroll
      for (int i = 0; i < 8; i++) {
        const int o = c + i;
        if (o >= KO) break;
        if (o < N) { if (aa.g_x0) aa.g_x0[(size_t)bi * N + o] = r[i] + aa.gJ * I.lam[o]; }
        else if (o < 2 * N) { if (aa.g_Qd) aa.g_Qd[(size_t)bi * N + (o - N)] = r[i]; }
        else if (o < 2 * N + U) { if (aa.g_Rd) aa.g_Rd[(size_t)bi * U + (o - 2 * N)] = r[i]; }
        else if (o < 3 * N + U) { if (aa.g_Qfd) aa.g_Qfd[(size_t)bi * N + (o - 2 * N - U)] = r[i]; }
        else if (aa.g_prm) aa.g_prm[(size_t)bi * PTN_MAXP + (o - 3 * N - U)] = r[i];
      }
    }
  }
  if (g.rank() == 0 && l == 0 && aa.g_prm)
    for (int k = NP; k < PTN_MAXP; k++) aa.g_prm[(size_t)bi * PTN_MAXP + k] = 0.0;
  return ST_OK;
}

template <class M, class SV>
__global__ void __launch_bounds__(512) k_adjoint_wide(KArgs args, Work<double> w, AdjArgs aa) {
  constexpr int N = M::NX, U = M::NU;
  extern __shared__ __align__(16) char smem[];
  ProbS<N, U>& P = *reinterpret_cast<ProbS<N, U>*>(smem);
  size_t off = (sizeof(ProbS<N, U>) + 15) & ~size_t(15);
  const int nw = blockDim.x >> 5;
  WideGroup g;
  g.red = reinterpret_cast<double*>(smem + off);
  off += (size_t)8 * 8 * nw;
  g.scr_bytes = (sizeof(WScr<M, double>) + 15) & ~size_t(15);
  g.scr = smem + off;
  off += g.scr_bytes * nw;
  constexpr size_t xb =
      sizeof(Val<N, double>) > sizeof(Aff<N, double>) ? sizeof(Val<N, double>) : sizeof(Aff<N, double>);
  g.xs_bytes = (xb + 15) & ~size_t(15);
  g.xs = smem + off;
  const int bi = blockIdx.x;
  if (bi >= args.B) return;
  load_prob<N, U>(P, *args.prob, args.xref ? args.xref + (size_t)bi * N : nullptr, args.inst[bi].dt);
  const InstDev id = args.inst[bi];
  Inst<M, double> I;
  I.setup(w, id, args.x0 + (size_t)bi * N, g.warp(), nw, P.nw);
  const int rc = adjoint_wide<M>(g, I, P, aa, id, bi);
  if (threadIdx.x == 0) args.info[bi].status = rc;
}

// host-side launch of the wide kernel (tier ignored except queries and the adjoint, which
// this tier does not have)
template <class M, class L, class SV>
cudaError_t launch_wide(LaunchReq& q) {
  constexpr int N = M::NX;
  if (q.elem_bytes) *q.elem_bytes = sizeof(Val<N, L>) > sizeof(Aff<N, double>) ? sizeof(Val<N, L>) : sizeof(Aff<N, double>);
  if (q.tier == 3) {
    // the adjoint runs with FP64 LQR data (built only in the FP64 unit)
    if constexpr (std::is_same<L, double>::value) {
      if (q.query) return cudaSuccess;
      const int nw = q.nthreads / 32;
      const size_t smem = wide_smem_bytes<M, double>(nw);
      cudaError_t e = raise_smem_limit<k_adjoint_wide<M, SV>>(smem);
      if (e != cudaSuccess) return e;
      k_adjoint_wide<M, SV><<<q.nblocks, q.nthreads, smem, q.stream>>>(q.args, typed<double>(q.w), *q.adj);
      return cudaGetLastError();
    } else {
      return cudaErrorNotSupported;
    }
  }
  if (q.query == 1) {
    if (q.max_blocks) *q.max_blocks = 0;
    return cudaSuccess;
  }
  const int nw = q.nthreads / 32;
  const size_t smem = wide_smem_bytes<M, L>(nw);
  if (!q.attrs_set) {
    cudaError_t e = raise_smem_limit<k_solve_wide<M, L, SV>>(smem);
    if (e != cudaSuccess) return e;
  }
  if (q.query == 2) return cudaSuccess;
  k_solve_wide<M, L, SV><<<q.nblocks, q.nthreads, smem, q.stream>>>(q.args, typed<L>(q.w));
  return cudaGetLastError();
}

}  // namespace ptn
