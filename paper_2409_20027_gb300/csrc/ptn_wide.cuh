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
// group: one warp per time chunk.  One CTA per instance (rank = warp, size = warps of the
// CTA), or, with grid set, the warps of the CTA range [b0, b0 + nb) of a cooperative launch
// on one instance (rank = (blockIdx.x - b0) * warps per CTA + warp; the whole launch for a
// single instance, one range per instance for a batch): barriers and reductions then also
// cross the range's CTAs (bounded barrier on the instance's own counters), and a scan ends
// with a Kogge-Stone over the CTA totals in global memory (scan_warps).
struct WideGroup {
  char* scr;         // per-warp scratch, warp w at scr + w * scr_bytes
  size_t scr_bytes;
  char* xs;          // cross-warp scan slots: 2 buffers x nwarps x xs_bytes, then the carry slot
  size_t xs_bytes;
  double* red;       // 8 doubles per warp, then 8 for the grid result
  int grid;          // nonzero: the cooperative-grid form
  int b0, nb;        // grid form: the group's CTAs blockIdx.x in [b0, b0 + nb)
  GridScratch gs;    // grid form: barrier, reduction slots, 2 x nb CTA-total slots (the group's own)
  int* sdead;        // grid form: shared flag, this CTA saw a barrier expire
  int phase;

  __device__ int warp() const { return threadIdx.x >> 5; }
  __device__ int nwarps() const { return blockDim.x >> 5; }
  __device__ int blk() const { return (int)blockIdx.x - b0; }
  __device__ int rank() const { return grid ? blk() * nwarps() + warp() : warp(); }
  __device__ int size() const { return grid ? nb * nwarps() : nwarps(); }
  __device__ bool dead() const { return grid && *(volatile int*)sdead != 0; }
  __device__ void sync() {
    __syncthreads();
    if (grid) {
      if (threadIdx.x == 0 && !*sdead) {
        if (!grid_barrier(gs, (unsigned)nb)) *sdead = 1;
      }
      __syncthreads();
    }
  }

  // every lane of a warp holds the warp's value; lane 0 contributes it.  Fixed order of
  // combination, so every thread gets the same result (in the grid form: warp 0 of each
  // CTA folds the CTAs' values in the same order).
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
    if (!grid) return;
    double* rs = gs.red + (size_t)phase * nb * 8;
    if (threadIdx.x == 0)
#pragma unroll
      for (int k = 0; k < K; k++) rs[blk() * 8 + k] = v[k];
    sync();
    double* sres = red + 8 * nw;
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      double a[K];
#pragma unroll
      for (int k = 0; k < K; k++) a[k] = ((maxmask >> k) & 1u) ? -INFINITY : 0.0;
      for (int b = lane; b < nb; b += 32)
#pragma unroll
        for (int k = 0; k < K; k++) {
          const double o = __ldcg(rs + (size_t)b * 8 + k);
          a[k] = ((maxmask >> k) & 1u) ? fmax(a[k], o) : a[k] + o;
        }
#pragma unroll
      for (int off = 1; off < 32; off <<= 1)
#pragma unroll
        for (int k = 0; k < K; k++) {
          const double o = __shfl_down_sync(0xffffffffu, a[k], off);
          if ((lane & (2 * off - 1)) == 0) a[k] = ((maxmask >> k) & 1u) ? fmax(a[k], o) : a[k] + o;
        }
      if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; k++) sres[k] = a[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = sres[k];
    __syncthreads();
    phase ^= 1;
  }

  // AND of a per-warp flag over the group (uniform result)
  __device__ bool all(bool ok) {
    double r[1] = {ok ? 0.0 : 1.0};
    reduce<1>(r, 1u);
    return r[0] == 0.0;
  }

  template <class T>
  __device__ T* slot(int buf, int w) const {
    return reinterpret_cast<T*>(xs + ((size_t)buf * nwarps() + w) * xs_bytes);
  }
  // the carry of the grid form: everything after (suffix) or before (prefix) this CTA
  template <class T>
  __device__ T* carry_slot() const {
    return reinterpret_cast<T*>(xs + (size_t)2 * nwarps() * xs_bytes);
  }
  // after a scan whose results are in buffer cur: the combination of all elements after
  // (suffix) or before (prefix) this warp's chunk -- the neighbouring warp's inclusive
  // result, or the CTA's carry at the CTA boundary (grid form).  Only for warps that have
  // such elements (not the group's last chunk for a suffix, not its first for a prefix).
  template <class T>
  __device__ const T* neighbor(int cur, bool suffix) const {
    const int w = warp(), nw = nwarps();
    if (suffix) return w + 1 < nw ? slot<T>(cur, w + 1) : carry_slot<T>();
    return w > 0 ? slot<T>(cur, w - 1) : carry_slot<T>();
  }
};

template <>
struct multiplier_form_ok<WideGroup> {
  static constexpr bool value = true;
};
template <>
struct ChunkLanes<WideGroup> {
  __device__ static int first() { return threadIdx.x & 31; }
  __device__ static int step() { return 32; }
  __device__ static double max(double v) { return wops::wmax(v); }
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
  double mdl[2 * N];     // model hooks' per-row terms
  Aff<N, L> sa;          // the rollout's chunk map (scan aggregates live in the warp's scan slot)
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

// Model terms of the wide passes, computed by the warp's lanes into shared memory: the
// Jacobians F, G of the step, the lam-contracted second derivatives (lam^T f)_zz and the
// FP64 step itself.  Models given by a continuous-time right-hand side use the lane-parallel
// forward-mode AD of ptn_wops.cuh; a model written as a discrete map specialises this.
// tmp: 2 N doubles of the warp's shared scratch.
template <class M>
struct WModel {
  static constexpr int N = M::NX, U = M::NU;
  static constexpr bool has_adjoint = true;
  template <class S>
  __device__ static void jac(const ProbS<N, U>& P, const double* x, const double* u, S* F, S* G, double* tmp) {
    (void)tmp;
    wops::step_jac<M, S>(P.integ, P.dt, P.prm, x, u, F, G);
  }
  // wrk: N x N values of L of the warp's scratch (models with closed forms use it)
  template <class L>
  __device__ static void hess(const ProbS<N, U>& P, const double* x, const double* u, const double* lam, L* Hxx,
                              L* Hxu, L* Huu, double* tmp, L* wrk) {
    (void)tmp; (void)wrk;
    wops::step_hess<M, L>(P.integ, P.dt, P.prm, x, u, lam, Hxx, Hxu, Huu);
  }
  // xn = f(x, u) in FP64 (x, u, xn in shared memory; xn must not alias x)
  __device__ static void step(const ProbS<N, U>& P, const double* x, const double* u, double* xn, double* tmp) {
    (void)tmp;
    double v[N];
    ptn::step<M>(P.integ, P.dt, P.prm, x, u, v);
    for (int i = wops::lane_id(); i < N; i += 32) xn[i] = v[i];
    __syncwarp();
  }
};

namespace wide {

using wops::lane_id;

// ---- lane-parallel stage terms (FP64) ----

// l_t (+ barrier / penalty) at (x, u); lplain: without the augmentation.  infeas is set
// when a barrier row is not strictly feasible.  gr: 2(N+U) doubles of scratch.
template <int N, int U>
__device__ double stage_cost_w(const ProbS<N, U>& P, const Aug& A, int t, const double* x, const double* u,
                               bool& infeas, double* lplain) {
  const int l = lane_id();
  const double *xr = xref_at(P, t), *ur = uref_at(P, t);
  double v = 0.0;
  for (int q = l; q < N + U; q += 32) {  // lane-strided: N + U may exceed 32
    if (q < N) {
      const double s = wops::dot4<N, double>([&](int j) { return P.Q[q * N + j] * (x[j] - xr[j]); });
      v += (x[q] - xr[q]) * s;
    } else {
      const int i = q - N;
      const double s = wops::dot4<U, double>([&](int j) { return P.R[i * U + j] * (u[j] - ur[j]); });
      v += (u[i] - ur[i]) * s;
    }
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
  const double* xr = xref_at(P, P.Tr);
  double v = 0.0;
  if (l < N) {
    const double s = wops::dot4<N, double>([&](int j) { return P.Qf[l * N + j] * (x[j] - xr[j]); });
    v = (x[l] - xr[l]) * s;
  }
  return wops::wsum(v);
}

// gradient of l_t + c_t into lx (N), lu (U) (shared); gr: per-row scratch (shared)
template <int N, int U>
__device__ void stage_grad_w(const ProbS<N, U>& P, const Aug& A, int t, const double* x, const double* u,
                             double* lx, double* lu, double* gr) {
  const int l = lane_id();
  const double *xr = xref_at(P, t), *ur = uref_at(P, t);
  for (int r = l; r < P.nw; r += 32) {
    const double zk = P.isx[r] ? x[P.idx[r]] : u[P.idx[r]];
    const double w = P.sgn[r] * (zk - P.bnd[r]);
    gr[r] = (A.kind == AUG_BARRIER) ? A.mu * P.sgn[r] / (-w)
                                    : A.rho * (w - A.z[(size_t)t * P.nw + r] + A.v[(size_t)t * P.nw + r] / A.rho) *
                                          P.sgn[r];
  }
  __syncwarp();
  for (int q = l; q < N + U; q += 32) {
    if (q < N) {
      double s = wops::dot4<N, double>([&](int j) { return (P.Q[q * N + j] + P.Q[j * N + q]) * (x[j] - xr[j]); });
      for (int r = 0; r < P.nw; r++)
        if (P.isx[r] && P.idx[r] == q) s += gr[r];
      lx[q] = s;
    } else {
      const int i = q - N;
      double s = wops::dot4<U, double>([&](int j) { return (P.R[i * U + j] + P.R[j * U + i]) * (u[j] - ur[j]); });
      for (int r = 0; r < P.nw; r++)
        if (!P.isx[r] && P.idx[r] == i) s += gr[r];
      lu[i] = s;
    }
  }
  __syncwarp();
}

template <int N, int U>
__device__ void terminal_grad_w(const ProbS<N, U>& P, const double* xT, double* g) {
  const int l = lane_id();
  const double* xr = xref_at(P, P.Tr);
  if (l < N)
    g[l] = wops::dot4<N, double>([&](int j) { return (P.Qf[l * N + j] + P.Qf[j * N + l]) * (xT[j] - xr[j]); });
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
  // Qux = G^T S F + M^T (U x N) in X[:, :N] (G^T (S F) formed in T3); d + G^T s in X[:, N];
  // G^T S G (U x U) in T3 behind it
  static_assert(U * N + U * U <= N * N, "T3 holds G^T S F and G^T S G");
  L* GSG = s->T3 + U * N;
  wops::mm<U, N, N, true, false>(s->G, SF, s->T3);
  wops::mm<U, N, U, true, false>(s->G, SG, GSG);
  for (int q = l; q < U * C; q += 32) {
    const int i = q / C, j = q % C;
    s->X[q] = (j < N) ? s->T3[i * N + j] + s->Mm[j * U + i]
                      : wops::dot4<N, L>([&](int k) { return s->G[k * U + i] * s->s[k]; }) + L(s->d[i]);
  }
  // Q = R + G^T S G + alpha I, in every lane
  __syncwarp();
  SV Q[U * U];
#pragma unroll
  for (int i = 0; i < U; i++)
#pragma unroll
    for (int j = 0; j < U; j++) Q[i * U + j] = SV(s->Rm[i * U + j]) + SV(GSG[i * U + j]) + (i == j ? SV(alpha) : SV(0));
  // keep Qux (U x N) for the S update, before the solve overwrites X
  L* Qux = s->T3;
  for (int q = l; q < U * N; q += 32) Qux[q] = s->X[(q / N) * C + (q % N)];
  __syncwarp();
  if (!ldlt<U, SV>(Q)) return false;
  wops::ldlt_solve_cols<U, C, SV>(Q, s->X);
  for (int q = l; q < U * N; q += 32) s->Gam[q] = -s->X[(q / N) * C + (q % N)];
  for (int i = l; i < U; i += 32) s->gam[i] = -s->X[i * C + N];
  __syncwarp();
  // S' = P + Qux^T Gam + F^T (S F),  s' = F^T s + Qux^T gam  (S G in T2 is used up)
  L* Sn = s->T2;
  for (int q = l; q < N * N; q += 32) {
    const int i = q / N, j = q % N;
    Sn[q] = s->Pm[q] + wops::dot4<U, L>([&](int k) { return Qux[k * N + i] * s->Gam[k * N + j]; });
  }
  __syncwarp();
  wops::mm<N, N, N, true, false, true>(s->F, SF, Sn);
  for (int i = l; i < N; i += 32) {
    L v = L(0);
    v += wops::dot4<N, L>([&](int k) { return s->F[k * N + i] * s->s[k]; });
#pragma unroll
    v += wops::dot4<U, L>([&](int k) { return Qux[k * N + i] * s->gam[k]; });
    s->w1[i] = v;
  }
  __syncwarp();
  wops::copy<N * N>(Sn, s->S);
  wops::copy<N>(s->w1, s->s);
  wops::symmetrize<N>(s->S);
  return true;
}

// step t (data in s->F, G, Pm, Mm, Rm, d) combined into the later element e, in place, in
// the Woodbury form of the value combination (as value_fold_step): with
// Q = R~ + G^T J G (U x U, inverted in SV with pivoting), H = M^T + G^T J F,
// Gam = -Q^{-1} H and gam = Q^{-1} (G^T eta - d),
//   J <- P + F^T J F + H^T Gam,  eta <- F^T eta - H^T gam,  A <- A (F + G Gam),
//   b <- b + (A G) gam,  C <- C + (A G) Q^{-1} (A G)^T.
// Returns false (warp-uniform) when Q is singular.
template <class SV, class M, class L>
__device__ bool val_fold_w(WScr<M, L>* s, double alpha, Val<M::NX, L>* e, L* tmpA) {
  constexpr int N = M::NX, U = M::NU, C = N + 1;
  static_assert(U * C <= U * (2 * N + 1) && N * U <= N * N, "scratch sizes");
  const int l = lane_id();
  L* JF = s->T1;  // N x N
  L* JG = s->T2;  // N x U
  wops::mm<N, N, N, false, false>(e->J, s->F, JF);
  wops::mm<N, N, U, false, false>(e->J, s->G, JG);
  // X[:, :N] = H = G^T J F + M^T (G^T (J F) formed in T3),  X[:, N] = G^T eta - d;
  // Q = R~ + G^T J G
  SV* Q = reinterpret_cast<SV*>(s->K);
  wops::mm<U, N, N, true, false>(s->G, JF, s->T3);
  for (int q = l; q < U * C; q += 32) {
    const int i = q / C, j = q % C;
    s->X[q] = (j < N) ? s->T3[i * N + j] + s->Mm[j * U + i]
                      : wops::dot4<N, L>([&](int k) { return s->G[k * U + i] * e->eta[k]; }) - L(s->d[i]);
  }
  for (int q = l; q < U * U; q += 32) {
    const int i = q / U, j = q % U;
    L gjg = L(0);
    gjg += wops::dot4<N, L>([&](int k) { return s->G[k * U + i] * JG[k * U + j]; });
    Q[q] = SV(s->Rm[q]) + SV(gjg) + (i == j ? SV(alpha) : SV(0));
  }
  __syncwarp();
  if (!wops::inv<U, SV>(Q, s->piv, reinterpret_cast<SV*>(s->col))) return false;
  // Gam = -Q^{-1} H, gam = Q^{-1} (G^T eta - d); H kept in T3 for the Bellman step
  L* H = s->T3;
  for (int q = l; q < U * C; q += 32) {
    const int i = q / C, j = q % C;
    SV v = SV(0);
#pragma unroll
    v += wops::dot4<U, SV>([&](int k) { return Q[i * U + k] * SV(s->X[k * C + j]); });
    if (j < N) {
      s->Gam[i * N + j] = L(-v);
      H[i * N + j] = s->X[q];
    } else {
      s->gam[i] = L(v);
    }
  }
  __syncwarp();
  // J' = P + H^T Gam + F^T (J F) (into T2: J G is used up) and eta' (into w1) from the
  // J, eta of e
  L* Jn = s->T2;
  for (int q = l; q < N * N; q += 32) {
    const int i = q / N, j = q % N;
    Jn[q] = s->Pm[q] + wops::dot4<U, L>([&](int k) { return H[k * N + i] * s->Gam[k * N + j]; });
  }
  __syncwarp();
  wops::mm<N, N, N, true, false, true>(s->F, JF, Jn);
  for (int i = l; i < N; i += 32) {
    L v = L(0);
    v += wops::dot4<N, L>([&](int k) { return s->F[k * N + i] * e->eta[k]; });
#pragma unroll
    for (int k = 0; k < U; k++) v -= H[k * N + i] * s->gam[k];
    s->w1[i] = v;
  }
  __syncwarp();
  // closed loop F + G Gam (into T1: J F is no longer needed); A G (into X)
  L* Fc = s->T1;
  L* AG = s->X;
  wops::copy<N * N>(s->F, Fc);
  wops::mm<N, U, N, false, false, true>(s->G, s->Gam, Fc);
  wops::mm<N, N, U, false, false>(e->A, s->G, AG);
  // A' = A (F + G Gam) into tmpA; (A G) Q^{-1} into T3 (H is no longer needed)
  wops::mm<N, N, N, false, false>(e->A, Fc, tmpA);
  L* AQ = s->T3;
  for (int q = l; q < N * U; q += 32) {
    const int i = q / U, j = q % U;
    SV v = SV(0);
#pragma unroll
    v += wops::dot4<U, SV>([&](int k) { return SV(AG[i * U + k]) * Q[k * U + j]; });
    AQ[q] = L(v);
  }
  __syncwarp();
  wops::mm<N, U, N, false, true, true>(AQ, AG, e->C);
  for (int q = l; q < N * N; q += 32) {
    e->A[q] = tmpA[q];
    e->J[q] = Jn[q];
  }
  for (int i = l; i < N; i += 32) {
    L v = e->b[i];
#pragma unroll
    v += wops::dot4<U, L>([&](int k) { return AG[i * U + k] * s->gam[k]; });
    e->b[i] = v;
    e->eta[i] = s->w1[i];
  }
  __syncwarp();
  wops::symmetrize<N>(e->C);
  wops::symmetrize<N>(e->J);
  return true;
}

// copy of one element through L2 (__ldcg: another CTA wrote it before a grid barrier, and
// L1 is not coherent across SMs), lane-parallel
template <class E>
__device__ void copy_cg(const E* src, E* dst) {
  const unsigned* s4 = reinterpret_cast<const unsigned*>(src);
  unsigned* d4 = reinterpret_cast<unsigned*>(dst);
  for (int i = lane_id(); i < (int)(sizeof(E) / 4); i += 32) d4[i] = __ldcg(s4 + i);
  __syncwarp();
}

// inclusive scan across warps of the elements in slot(0, w) of g; op(earlier, later, out)
// on element pointers.  Returns the buffer holding the results (read them through
// g.neighbor); ok is AND-ed with op's results.  Grid form: the CTA totals (the inclusive
// result of the CTA's first warp for a suffix, of its last for a prefix) are scanned across
// the CTAs by a Kogge-Stone in global memory, double-buffered, one combination by warp 0 of
// each CTA per level behind grid barriers, with its operands staged in shared memory; then
// every warp combines its result with its CTA's carry (the inclusive result of the next,
// or the previous, CTA), into the other buffer.
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
  if (!g.grid) return cur;
  const int nb = g.nb, b = g.blk();
  auto gslot = [&](int buf, int i) {
    return reinterpret_cast<E*>(g.gs.xs + ((size_t)buf * nb + i) * g.gs.elem_bytes);
  };
  if (w == 0) wops::copy<sizeof(E) / sizeof(unsigned)>(reinterpret_cast<const unsigned*>(g.slot<E>(cur, suffix ? 0 : nw - 1)),
                                                        reinterpret_cast<unsigned*>(gslot(0, b)));
  int gc = 0;
  g.sync();
  E* sa = g.slot<E>(cur ^ 1, 0);  // staging (free until the carry is applied)
  E* sb = g.carry_slot<E>();
  for (int off = 1; off < nb; off <<= 1) {
    const int o = suffix ? b + off : b - off;
    if (w == 0) {
      if (o >= 0 && o < nb) {
        copy_cg(gslot(gc, suffix ? b : o), sa);
        copy_cg(gslot(gc, suffix ? o : b), sb);
        ok &= op(sa, sb, gslot(gc ^ 1, b));
      } else {
        copy_cg(gslot(gc, b), gslot(gc ^ 1, b));
      }
    }
    g.sync();
    gc ^= 1;
  }
  const int cb = suffix ? b + 1 : b - 1;
  if (cb >= 0 && cb < nb) {
    if (w == 0) copy_cg(gslot(gc, cb), sb);
    __syncthreads();
    E* mine = g.slot<E>(cur, w);
    E* dst = g.slot<E>(cur ^ 1, w);
    ok &= suffix ? op(mine, sb, dst) : op(sb, mine, dst);
    cur ^= 1;
  }
  __syncthreads();
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
  Aff<N, double>* agg = g.slot<Aff<N, double>>(0, g.warp());  // the chunk aggregate, built in the scan slot
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
    WModel<M>::jac(P, x, u, s->F64, s->G64, s->mdl);
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
  bool ok = true;
  auto op = [&](const Aff<N, double>* a, const Aff<N, double>* b, Aff<N, double>* o) {
    wide::costate_combine<N>(a, b, o);
    return true;
  };
  const int cur = wide::scan_warps<Aff<N, double>>(g, op, true, ok);
  double* lam = s->lam;
  if (!I.last) {
    const Aff<N, double>* nx = g.neighbor<Aff<N, double>>(cur, true);
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
      v += wops::dot4<N, double>([&](int k) { return G[k * U + l] * lam[k]; });
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

// pass 1, multiplier form (costate_mode 1, 2; the variant of multiplier_pass in the narrow
// tiers): multipliers nu of the dynamics in I.lam, local gradients
//   d_t = dl/du + G_t^T nu_{t+1},   q_t = dl/dx + F_t^T nu_{t+1} - nu_t   (t >= 1),
//   q_T = dl_T/dx - nu_T,   nu_0 := dl/dx + F_0^T nu_1 with q_0 = 0,
// lane-parallel, FP64 Jacobians stored as the co-state pass stores them.  Returns
// max(max |d|, max |q|) over the group.
template <class M, class L>
__device__ double multiplier_pass(WideGroup& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const Aug& A) {
  constexpr int N = M::NX, U = M::NU;
  WScr<M, L>* s = wscr<M, L>(g);
  const int l = wide::lane_id();
  double rl = 0.0;
  for (int t = I.a; t < I.b; t++) {
    const double* x = I.xn + (size_t)t * N;
    const double* u = I.un + (size_t)t * U;
    WModel<M>::jac(P, x, u, s->F64, s->G64, s->mdl);
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
    const double* nv = I.lam + (size_t)(t + 1) * N;
    for (int i = l; i < U; i += 32) {
      double v = s->r[i];
      v += wops::dot4<N, double>([&](int k) { return s->G64[k * U + i] * nv[k]; });
      I.d[(size_t)t * U + i] = v;
      rl = fmax(rl, isfinite(v) ? fabs(v) : INFINITY);
    }
    for (int i = l; i < N; i += 32) {
      double v = s->q[i];
      v += wops::dot4<N, double>([&](int k) { return s->F64[k * N + i] * nv[k]; });
      if (t == 0) {
        I.lam[i] = v;
        I.q[i] = 0.0;
      } else {
        v -= I.lam[(size_t)t * N + i];
        I.q[(size_t)t * N + i] = v;
        rl = fmax(rl, isfinite(v) ? fabs(v) : INFINITY);
      }
    }
    __syncwarp();
  }
  if (I.last) {
    wide::terminal_grad_w<N, U>(P, I.xn + (size_t)I.T * N, s->lam);
    for (int i = l; i < N; i += 32) {
      const double v = s->lam[i] - I.lam[(size_t)I.T * N + i];
      I.q[(size_t)I.T * N + i] = v;
      rl = fmax(rl, isfinite(v) ? fabs(v) : INFINITY);
    }
    __syncwarp();
  }
  if (I.a < I.b)
    for (int i = 0; i < N; i++) I.lamb[i] = I.lam[(size_t)I.b * N + i];
  double red[1] = {wops::wmax(rl)};
  g.template reduce<1>(red, 1u);
  return red[0];
}

// the FP32-increment multiplier pass of the narrow tiers is not used here (exact_only)
template <class M>
__device__ double multiplier_mixed(WideGroup& g, Inst<M, float>& I, const ProbS<M::NX, M::NU>& P, const Aug& A) {
  return multiplier_pass(g, I, P, A);
}

// cost of the nominal (as nominal_cost), lane-parallel stage terms
template <class M, class L>
__device__ double nominal_cost(WideGroup& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const Aug& A, bool* infeas,
                               double* Jplain) {
  constexpr int N = M::NX, U = M::NU;
  double c = 0.0, cp = 0.0;
  bool inf = false;
  for (int t = I.a; t < I.b; t++) {
    double lp;
    c += wide::stage_cost_w<N, U>(P, A, t, I.xn + (size_t)t * N, I.un + (size_t)t * U, inf, &lp);
    cp += lp;
  }
  if (I.last) {
    const double lt = wide::terminal_cost_w<N, U>(P, I.xn + (size_t)I.T * N);
    c += lt;
    cp += lt;
  }
  double red[3] = {c, cp, inf ? 1.0 : 0.0};
  g.template reduce<3>(red, 4u);
  if (infeas) *infeas = red[2] > 0.0;
  if (Jplain) *Jplain = red[1];
  return red[0];
}

// final residuals (as residuals), the dynamics defects with the lane-parallel step
template <class M, class L>
__device__ void residuals(WideGroup& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const Aug& A, InfoDev& info,
                          bool mult = false) {
  constexpr int N = M::NX, U = M::NU;
  WScr<M, L>* s = wscr<M, L>(g);
  const int l = wide::lane_id();
  info.r_stat = mult ? multiplier_pass(g, I, P, A) : costate_pass(g, I, P, A, true);
  double rd = 0.0, rf = -INFINITY;
  for (int t = I.a; t < I.b; t++) {
    for (int i = l; i < N; i += 32) s->x[i] = I.xn[(size_t)t * N + i];
    for (int i = l; i < U; i += 32) s->u[i] = I.un[(size_t)t * U + i];
    __syncwarp();
    WModel<M>::step(P, s->x, s->u, s->xn, s->mdl);
    for (int i = l; i < N; i += 32) {
      const double e = fabs(I.xn[(size_t)(t + 1) * N + i] - s->xn[i]);
      rd = (e <= rd) ? rd : (isfinite(e) ? e : INFINITY);
    }
    for (int r = l; r < P.nw; r += 32) {
      const double zk = P.isx[r] ? s->x[P.idx[r]] : s->u[P.idx[r]];
      rf = fmax(rf, P.sgn[r] * (zk - P.bnd[r]));
    }
    __syncwarp();
  }
  double red[2] = {wops::wmax(rd), wops::wmax(rf)};
  g.template reduce<2>(red, 3u);
  info.r_dyn = red[0];
  info.r_feas = fmax(red[1], 0.0);
  bool inf;
  double Jp;
  info.J_c = nominal_cost(g, I, P, A, &inf, &Jp);
  info.J = Jp;
}

// initial nominal x = rollout(x0, u_init) (open loop, FP64), integrated by the first warp
// of the group with the lane-parallel step (the multiple-shooting form of the narrow tiers
// is not used here)
template <class M, class L>
__device__ void initial_rollout(WideGroup& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P) {
  constexpr int N = M::NX, U = M::NU;
  if (g.rank() == 0) {
    WScr<M, L>* s = wscr<M, L>(g);
    const int l = wide::lane_id();
    for (int i = l; i < N; i += 32) {
      s->x[i] = I.x0[i];
      I.xn[i] = I.x0[i];
    }
    __syncwarp();
    for (int t = 0; t < I.T; t++) {
      for (int i = l; i < U; i += 32) s->u[i] = I.un[(size_t)t * U + i];
      __syncwarp();
      WModel<M>::step(P, s->x, s->u, s->xn, s->mdl);
      for (int i = l; i < N; i += 32) {
        s->x[i] = s->xn[i];
        I.xn[(size_t)(t + 1) * N + i] = s->xn[i];
      }
      __syncwarp();
    }
  }
  g.sync();
}
template <class M, class L>
__device__ bool initial_rollout_parallel(WideGroup& g, Inst<M, L>& I, const ProbS<M::NX, M::NU>& P, const OptDev& O,
                                         int* iters) {
  (void)g; (void)I; (void)P; (void)O; (void)iters;
  return false;
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
    WModel<M>::hess(P, x, u, lam1, s->Pm, s->Mm, s->Rm, s->mdl, s->T1);
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

// pass 3: value suffix scan (Alg. 2) + feedback sweep.  qx: linear state terms of the LQR
// (adjoint, multiplier form); Sv, sv receive S_t, s_t (multiplier form); group_ok = false
// returns the warp's flag without the group reduction (as value_pass of the narrow tiers).
template <class M, class L, class SV>
__device__ bool value_pass(WideGroup& g, Inst<M, L>& I, double alpha, const double* qx = nullptr, L* Sv = nullptr,
                           L* sv = nullptr, bool group_ok = true) {
  constexpr int N = M::NX, U = M::NU;
  WScr<M, L>* s = wscr<M, L>(g);
  const int l = wide::lane_id();
  bool ok = true;
  Val<N, L>* agg = g.slot<Val<N, L>>(0, g.warp());  // the chunk aggregate, built in the scan slot
  L* tmpA = g.slot<Val<N, L>>(1, g.warp())->A;       // free until the scan
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
  }
  // the warp's chunk: each step's element combined into the aggregate from the right in
  // the Woodbury form (one U x U inverse per step instead of the element initialisation
  // and an N x N inverse); the identity element starts a chunk that does not end the horizon
  for (int t = I.b - 1; t >= I.a; t--) {
    load_step(I, s, t);
    ok &= wide::val_fold_w<SV>(s, alpha, agg, tmpA);
    if (qx) {
      for (int i = l; i < N; i += 32) agg->eta[i] -= L(qx[(size_t)t * N + i]);
      __syncwarp();
    }
  }
  auto op = [&](const Val<N, L>* a, const Val<N, L>* b, Val<N, L>* o) { return wide::val_combine<SV>(a, b, o, s); };
  const int cur = wide::scan_warps<Val<N, L>>(g, op, true, ok);
  if (I.last) {
    for (int e = l; e < N * N; e += 32) s->S[e] = I.Pm[(size_t)I.T * N * N + e];
    for (int i = l; i < N; i += 32) s->s[i] = qx ? L(qx[(size_t)I.T * N + i]) : L(0);
    if (Sv) {
      for (int e = l; e < N * N; e += 32) Sv[(size_t)I.T * N * N + e] = s->S[e];
      for (int i = l; i < N; i += 32) sv[(size_t)I.T * N + i] = s->s[i];
    }
  } else {
    const Val<N, L>* nx = g.neighbor<Val<N, L>>(cur, true);
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
    __syncwarp();
    if (Sv) {
      for (int e = l; e < N * N; e += 32) Sv[(size_t)t * N * N + e] = s->S[e];
      for (int i = l; i < N; i += 32) sv[(size_t)t * N + i] = s->s[i];
    }
    for (int e = l; e < U * N; e += 32) I.Gam[(size_t)t * U * N + e] = s->Gam[e];
    for (int i = l; i < U; i += 32) I.gam[(size_t)t * U + i] = s->gam[i];
    __syncwarp();
  }
  if (!group_ok) return ok;
  return g.all(ok);
}

// pass 4: state prefix scan (Alg. 3) and the model terms G1, G2.  Multiplier form (qx, Sv,
// sv, dnu given): G1 also carries sum_t q_t^T dx_t and dnu_t = S_t dx_t + s_t is the dual
// step (as state_pass of the narrow tiers).  fail: a per-warp flag reduced by maximum with
// G1, G2; on return the group's flag.
template <class M, class L>
__device__ void state_pass(WideGroup& g, Inst<M, L>& I, double& G1, double& G2, const double* qx = nullptr,
                           const L* Sv = nullptr, const L* sv = nullptr, double* dnu = nullptr, double* fail = nullptr) {
  constexpr int N = M::NX, U = M::NU;
  WScr<M, L>* s = wscr<M, L>(g);
  const int l = wide::lane_id();
  const bool first = (I.a == 0);
  Aff<N, L>* agg = g.slot<Aff<N, L>>(0, g.warp());  // the chunk aggregate, built in the scan slot
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
    const Aff<N, L>* pv = g.neighbor<Aff<N, L>>(cur, false);
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
    for (int q = l; q < N + U; q += 32) {
      if (q < N) {
        L pd = L(0), md = L(0);
        for (int k = 0; k < N; k++) pd += s->Pm[q * N + k] * dx[k];
        for (int k = 0; k < U; k++) md += s->Mm[q * U + k] * s->wu[k];
        a2 += double(dx[q] * (L(0.5) * pd + md));
      } else {
        const int i = q - N;
        L rd = L(0);
        for (int k = 0; k < U; k++) rd += s->Rm[i * U + k] * s->wu[k];
        a2 += double(L(0.5) * s->wu[i] * rd);
      }
    }
    if (qx) {
      // multiplier form: q_t^T dx_t in G1 and the dual step S_t dx_t + s_t
      for (int i = l; i < N; i += 32) {
        a1 += qx[(size_t)t * N + i] * double(dx[i]);
        double v = double(sv[(size_t)t * N + i]);
        v += wops::dot4<N, double>([&](int j) { return double(Sv[(size_t)t * N * N + i * N + j]) * double(dx[j]); });
        dnu[(size_t)t * N + i] = v;
      }
    }
    g1 += wops::wsum(a1);
    g2 += wops::wsum(a2);
    // dx <- F dx + G du
    wops::mv<N, N, false>(s->F, dx, s->w1);
    wops::mv<N, U, false, true>(s->G, s->wu, s->w1);
    wops::copy<N>(s->w1, dx);
  }
  if (I.last) {
    double a1 = 0.0, a2 = 0.0;
    if (l < N) {
      L pd = L(0);
      for (int k = 0; k < N; k++) pd += I.Pm[(size_t)I.T * N * N + l * N + k] * dx[k];
      a2 = double(L(0.5) * dx[l] * pd);
      I.dx[(size_t)I.T * N + l] = dx[l];
      if (qx) {
        a1 = qx[(size_t)I.T * N + l] * double(dx[l]);
        double v = double(sv[(size_t)I.T * N + l]);
        v += wops::dot4<N, double>([&](int j) { return double(Sv[(size_t)I.T * N * N + l * N + j]) * double(dx[j]); });
        dnu[(size_t)I.T * N + l] = v;
      }
    }
    g1 += wops::wsum(a1);
    g2 += wops::wsum(a2);
    __syncwarp();
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
        v += wops::dot4<N, double>([&](int j) { return double(Gam[l * N + j]) * (xt[j] - xh[j]); });
        ut[l] = v;
        I.uc[(size_t)t * U + l] = v;
      }
      if (t > I.a)
        for (int i = l; i < N; i += 32) I.xc[(size_t)t * N + i] = xt[i];
      __syncwarp();
      cost += wide::stage_cost_w<N, U>(P, A, t, xt, ut, inf, nullptr);
      // FP64 step (into s->xn) and the closed-loop Jacobian F + G Gam in L
      WModel<M>::step(P, xt, ut, s->xn, s->mdl);
      WModel<M>::jac(P, xt, ut, s->F, s->G, s->mdl);
      for (int q = l; q < U * N; q += 32) s->Gam[q] = Gam[q];
      __syncwarp();
      wops::mm<N, U, N, false, false>(s->G, s->Gam, s->T1);
      for (int q = l; q < N * N; q += 32) s->T1[q] += s->F[q];
      __syncwarp();
      if (!first) {
        wops::mm<N, N, N, false, false>(s->T1, el->M, s->T2);
        wops::copy<N * N>(s->T2, el->M);
      }
      for (int i = l; i < N; i += 32) xt[i] = s->xn[i];
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
        const Aff<N, L>* pv = g.neighbor<Aff<N, L>>(cur, false);
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
// shared memory of a wide CTA: problem record, reduction slots (8 doubles per warp and 8
// for the grid), per-warp scratch, scan slots (2 buffers per warp and the carry slot)
template <class M, class L>
__host__ __device__ constexpr size_t wide_slot_bytes() {
  constexpr int N = M::NX;
  constexpr size_t xb = sizeof(Val<N, L>) > sizeof(Aff<N, double>) ? sizeof(Val<N, L>) : sizeof(Aff<N, double>);
  return (xb + 15) & ~size_t(15);
}
template <class M, class L>
__host__ __device__ constexpr size_t wide_smem_bytes(int nwarps) {
  constexpr int N = M::NX, U = M::NU;
  return ((sizeof(ProbS<N, U>) + 15) & ~size_t(15)) + (size_t)8 * 8 * (nwarps + 1) +
         ((sizeof(WScr<M, L>) + 15) & ~size_t(15)) * nwarps + (size_t)(2 * nwarps + 1) * wide_slot_bytes<M, L>();
}

// largest CTA of the wide kernels of model M (their launch bound); a model whose warp
// scratch allows few warps per CTA lowers it, which leaves more registers per thread
template <class M>
struct WideMaxThreads {
  static constexpr int value = 256;  // the largest block_threads the options allow
};

template <class M, class L>
__device__ void wide_layout(WideGroup& g, char* smem) {
  constexpr int N = M::NX, U = M::NU;
  size_t off = (sizeof(ProbS<N, U>) + 15) & ~size_t(15);
  const int nw = blockDim.x >> 5;
  g.red = reinterpret_cast<double*>(smem + off);
  off += (size_t)8 * 8 * (nw + 1);
  g.scr_bytes = (sizeof(WScr<M, L>) + 15) & ~size_t(15);
  g.scr = smem + off;
  off += g.scr_bytes * nw;
  g.xs_bytes = wide_slot_bytes<M, L>();
  g.xs = smem + off;
}

// one CTA per instance, one warp per chunk
template <class M, class L, class SV>
__global__ void __launch_bounds__(WideMaxThreads<M>::value) k_solve_wide(KArgs args, Work<L> w) {
  constexpr int N = M::NX, U = M::NU;
  extern __shared__ __align__(16) char smem[];
  ProbS<N, U>& P = *reinterpret_cast<ProbS<N, U>*>(smem);
  const int nw = blockDim.x >> 5;
  WideGroup g{};
  wide_layout<M, L>(g, smem);
  g.grid = 0;
  const int bi = blockIdx.x;
  if (bi >= args.B) return;
  load_prob<N, U>(P, *args.prob, args.xref ? args.xref + (size_t)bi * N : nullptr, args.inst[bi].dt,
                  inst_xtraj<N>(args, args.inst[bi]), inst_utraj<U>(args, args.inst[bi]), args.inst[bi].T);
  const OptDev& O = *args.opt;  // read where used (a local copy would hold ~50 registers)
  const InstDev id = args.inst[bi];
  Inst<M, L> I;
  I.setup(w, id, args.x0 + (size_t)bi * N, g.warp(), nw, P.nw);
  solve_instance<M, L, SV>(g, I, P, O, args.u_init ? args.u_init + (size_t)id.uoff * U : nullptr, args.info + bi);
}

// one instance on every warp of a cooperative grid (long horizons)
template <class M, class L, class SV>
__global__ void __launch_bounds__(WideMaxThreads<M>::value) k_solve_wide_grid(KArgs args, Work<L> w) {
  constexpr int N = M::NX, U = M::NU;
  extern __shared__ __align__(16) char smem[];
  ProbS<N, U>& P = *reinterpret_cast<ProbS<N, U>*>(smem);
  __shared__ int sdead;
  if (threadIdx.x == 0) sdead = 0;
  WideGroup g{};
  wide_layout<M, L>(g, smem);
  g.grid = 1;
  g.b0 = 0;
  g.nb = (int)gridDim.x;
  g.gs = args.gs;
  g.sdead = &sdead;
  g.phase = 0;
  load_prob<N, U>(P, *args.prob, args.xref, args.inst[0].dt,
                  inst_xtraj<N>(args, args.inst[0]), inst_utraj<U>(args, args.inst[0]), args.inst[0].T);
  const OptDev& O = *args.opt;
  const InstDev id = args.inst[0];
  Inst<M, L> I;
  I.setup(w, id, args.x0, g.rank(), g.size(), P.nw);
  solve_instance<M, L, SV>(g, I, P, O, args.u_init, args.info);
}

// a batch on every co-resident CTA of a cooperative launch: instance i on the CTA range
// [inst[i].pad, inst[i + 1].pad) (the host sizes the ranges in proportion to the horizons),
// with its own barrier counters and scan and reduction slots: a segment of args.gs at
// offsets 2 i (counters), 2 x 8 x first CTA (reduction slots) and 2 x first CTA (element
// slots)
template <class M, class L, class SV>
__global__ void __launch_bounds__(WideMaxThreads<M>::value) k_solve_wide_bgrid(KArgs args, Work<L> w) {
  constexpr int N = M::NX, U = M::NU;
  extern __shared__ __align__(16) char smem[];
  ProbS<N, U>& P = *reinterpret_cast<ProbS<N, U>*>(smem);
  __shared__ int sdead;
  if (threadIdx.x == 0) sdead = 0;
  // the instance whose range holds this CTA: the last i with inst[i].pad <= blockIdx.x
  int lo = 0, hi = args.B - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (args.inst[mid].pad <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const int bi = lo;
  const InstDev id = args.inst[bi];
  WideGroup g{};
  wide_layout<M, L>(g, smem);
  g.grid = 1;
  g.b0 = id.pad;
  g.nb = (bi + 1 < args.B ? args.inst[bi + 1].pad : (int)gridDim.x) - id.pad;
  g.gs = args.gs;
  g.gs.bar = args.gs.bar + 2 * bi;
  g.gs.red = args.gs.red + (size_t)2 * 8 * id.pad;
  g.gs.xs = args.gs.xs + (size_t)2 * id.pad * args.gs.elem_bytes;
  g.sdead = &sdead;
  g.phase = 0;
  load_prob<N, U>(P, *args.prob, args.xref ? args.xref + (size_t)bi * N : nullptr, id.dt,
                  inst_xtraj<N>(args, id), inst_utraj<U>(args, id), id.T);
  const OptDev& O = *args.opt;
  Inst<M, L> I;
  I.setup(w, id, args.x0 + (size_t)bi * N, g.rank(), g.size(), P.nw);
  solve_instance<M, L, SV>(g, I, P, O, args.u_init ? args.u_init + (size_t)id.uoff * U : nullptr, args.info + bi);
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
  static_assert(N + U <= 32, "the wide adjoint keeps one state or control component per lane");
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
      const double e = I.xn[(size_t)t * N + l] - xref_at(P, t)[l];
      env[N + l] += e * e;
    } else if (l < N + U) {
      const double e = I.un[(size_t)t * U + (l - N)] - uref_at(P, t)[l - N];
      env[2 * N + (l - N)] += e * e;
    }
  }
  if (I.last && l < N) {
    const double e = I.xn[(size_t)I.T * N + l] - xref_at(P, I.T)[l];
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
        v += wops::dot4<N, double>([&](int j) { return Pt[l * N + j] * w[j]; });
        if (t < I.T) {
          const double* Mt = I.Mm + (size_t)t * N * U;
          const double* wu = I.du + (size_t)t * U;
          v += wops::dot4<U, double>([&](int j) { return Mt[l * U + j] * wu[j]; });
        }
        c[l] = v;
      }
      __syncwarp();
    };
    Aff<N, double>* agg = g.slot<Aff<N, double>>(0, g.warp());  // built in the scan slot
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
      const Aff<N, double>* nx = g.neighbor<Aff<N, double>>(cur, true);
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
      if (l < N) adj[N + l] += I.dx[(size_t)t * N + l] * 2.0 * (I.xn[(size_t)t * N + l] - xref_at(P, t)[l]);
      else if (l < N + U)
        adj[2 * N + (l - N)] +=
            I.du[(size_t)t * U + (l - N)] * 2.0 * (I.un[(size_t)t * U + (l - N)] - uref_at(P, t)[l - N]);
    }
    if (I.last && l < N)
      adj[2 * N + U + l] = I.dx[(size_t)I.T * N + l] * 2.0 * (I.xn[(size_t)I.T * N + l] - xref_at(P, I.T)[l]);
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
  const int nw = blockDim.x >> 5;
  WideGroup g{};
  wide_layout<M, double>(g, smem);
  g.grid = 0;
  const int bi = blockIdx.x;
  if (bi >= args.B) return;
  load_prob<N, U>(P, *args.prob, args.xref ? args.xref + (size_t)bi * N : nullptr, args.inst[bi].dt,
                  inst_xtraj<N>(args, args.inst[bi]), inst_utraj<U>(args, args.inst[bi]), args.inst[bi].T);
  const InstDev id = args.inst[bi];
  Inst<M, double> I;
  I.setup(w, id, args.x0 + (size_t)bi * N, g.warp(), nw, P.nw);
  const int rc = adjoint_wide<M>(g, I, P, aa, id, bi);
  if (threadIdx.x == 0) args.info[bi].status = rc;
}

// host-side launch of the wide kernels: tier 6 is one instance on the cooperative grid,
// tier 3 the adjoint (one CTA per instance), every other tier one CTA per instance.
// Queries: 1, the largest co-resident grid (tier 6) or 0; 2, set the function attributes;
// 4, the largest number of threads per CTA whose shared memory fits (into *max_blocks).
template <class M, class L, class SV>
cudaError_t launch_wide(LaunchReq& q) {
  if (q.elem_bytes) *q.elem_bytes = wide_slot_bytes<M, L>();
  int dev = 0, smax = 0;
  if (q.query == 4 || q.query == 1) {
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
  }
  if (q.query == 4) {
    int nw = WideMaxThreads<M>::value / 32;
    while (nw > 1 && wide_smem_bytes<M, L>(nw) > (size_t)smax) nw--;
    *q.max_blocks = wide_smem_bytes<M, L>(nw) <= (size_t)smax ? 32 * nw : 0;
    return cudaSuccess;
  }
  if (q.tier == 3) {
    // the adjoint runs with FP64 LQR data (built only in the FP64 unit)
    if constexpr (std::is_same<L, double>::value && WModel<M>::has_adjoint) {
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
  const int nw = q.nthreads / 32;
  const size_t smem = wide_smem_bytes<M, L>(nw);
  if (q.tier == 6) {
    if (!q.attrs_set) {
      cudaError_t e = raise_smem_limit<k_solve_wide_grid<M, L, SV>>(smem);
      if (e != cudaSuccess) return e;
    }
    if (q.query == 2) return cudaSuccess;
    if (q.query == 1) {
      int per = 0, sms = 0;
      cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_solve_wide_grid<M, L, SV>,
                                                                              q.nthreads, smem);
      if (e != cudaSuccess) return e;
      *q.max_blocks = per * sms;
      return cudaSuccess;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(q.nblocks);
    cfg.blockDim = dim3(q.nthreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = q.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_solve_wide_grid<M, L, SV>, q.args, typed<L>(q.w));
  }
  if (q.tier == 8) {
    if (!q.attrs_set) {
      cudaError_t e = raise_smem_limit<k_solve_wide_bgrid<M, L, SV>>(smem);
      if (e != cudaSuccess) return e;
    }
    if (q.query == 2) return cudaSuccess;
    if (q.query == 1) {
      int per = 0, sms = 0;
      cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_solve_wide_bgrid<M, L, SV>,
                                                                              q.nthreads, smem);
      if (e != cudaSuccess) return e;
      *q.max_blocks = per * sms;
      return cudaSuccess;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(q.nblocks);
    cfg.blockDim = dim3(q.nthreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = q.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_solve_wide_bgrid<M, L, SV>, q.args, typed<L>(q.w));
  }
  if (q.query == 1) {
    if (q.max_blocks) *q.max_blocks = 0;
    return cudaSuccess;
  }
  if (!q.attrs_set) {
    cudaError_t e = raise_smem_limit<k_solve_wide<M, L, SV>>(smem);
    if (e != cudaSuccess) return e;
  }
  if (q.query == 2) return cudaSuccess;
  k_solve_wide<M, L, SV><<<q.nblocks, q.nthreads, smem, q.stream>>>(q.args, typed<L>(q.w));
  return cudaGetLastError();
}

}  // namespace ptn
