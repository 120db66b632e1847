// ptn_ops.cuh -- associative elements and operators of the three scans of the
// parallel-in-time Newton step (arXiv 2409.20027, Sec. III), in register arrays.
//
//   co-state pass (Alg. 1): element (g, F^T), operator eq. co-states-comb-rule
//   value pass    (Alg. 2): element (A, b, C, eta, J), operator eq. value-fun-param,
//                           initialisation eq. value-fun-elem-init
//   state pass    (Alg. 3): element (F, e), operator eq. state-prop-comb-rule
//
// "a then b" always means a covers the earlier time interval.
#pragma once
#include "ptn_common.cuh"

namespace ptn {

// affine map (matrix part M, vector part v)
template <int N, class S>
struct Aff {
  S M[N * N];
  S v[N];
};

template <int N, class S>
PTN_HD void set_identity(Aff<N, S>& e) {
#pragma unroll
  for (int i = 0; i < N * N; i++) e.M[i] = S(0);
#pragma unroll
  for (int i = 0; i < N; i++) { e.M[i * N + i] = S(1); e.v[i] = S(0); }
}

// Co-state operator, M holds F^T:  v = a.v + a.M b.v,  M = a.M b.M.
struct CostateOp {
  template <int N, class S>
  PTN_HD bool operator()(const Aff<N, S>& a, const Aff<N, S>& b, Aff<N, S>& o) const {
    Aff<N, S> r;
    mm<N, N, N>(a.M, b.M, r.M);
    mv<N, N>(a.M, b.v, r.v);
#pragma unroll
    for (int i = 0; i < N; i++) r.v[i] += a.v[i];
    o = r;
    return true;
  }
};

// State-propagation operator:  M = b.M a.M,  v = b.M a.v + b.v.
struct StateOp {
  template <int N, class S>
  PTN_HD bool operator()(const Aff<N, S>& a, const Aff<N, S>& b, Aff<N, S>& o) const {
    Aff<N, S> r;
    mm<N, N, N>(b.M, a.M, r.M);
    mv<N, N>(b.M, a.v, r.v);
#pragma unroll
    for (int i = 0; i < N; i++) r.v[i] += b.v[i];
    o = r;
    return true;
  }
};

// value-function element; the paper's Y is stored as J
template <int N, class L>
struct Val {
  L A[N * N];
  L C[N * N];
  L J[N * N];
  L eta[N];
  L b[N];
};

template <int N, class L>
PTN_HD void set_identity(Val<N, L>& e) {
#pragma unroll
  for (int i = 0; i < N * N; i++) { e.A[i] = L(0); e.C[i] = L(0); e.J[i] = L(0); }
#pragma unroll
  for (int i = 0; i < N; i++) { e.A[i * N + i] = L(1); e.eta[i] = L(0); e.b[i] = L(0); }
}

template <int N, class L>
PTN_HD void symmetrize(L* X) {
#pragma unroll
  for (int i = 0; i < N; i++)
#pragma unroll
    for (int j = i + 1; j < N; j++) {
      L s = L(0.5) * (X[i * N + j] + X[j * N + i]);
      X[i * N + j] = s;
      X[j * N + i] = s;
    }
}

// Products of the value operator (eq. value-fun-param, with b_{t,i} as the last term of b)
// once K = (I + C1 J2)^{-1} is known:
//   A   = A2 K A1
//   C   = A2 K C1 A2^T + C2
//   b   = A2 K (b1 + C1 eta2) + b2
//   J   = A1^T K^T J2 A1 + J1      K^T = (I + J2 C1)^{-1} since C, J are symmetric
//   eta = A1^T K^T (eta2 - J2 b1) + eta1
template <int N, class L>
PTN_HD void value_apply_K(const Val<N, L>& e1, const Val<N, L>& e2, const L* K, Val<N, L>& o) {
  Val<N, L> r;
  L t1[N * N], t2[N * N], w[N], tv[N];
  // A and C
  mm<N, N, N>(K, e1.A, t1);
  mm<N, N, N>(e2.A, t1, r.A);
  mm<N, N, N>(K, e1.C, t1);
  mm<N, N, N>(e2.A, t1, t2);
  mmt<N, N, N>(t2, e2.A, r.C);
#pragma unroll
  for (int i = 0; i < N * N; i++) r.C[i] += e2.C[i];
  // b
  mv<N, N>(e1.C, e2.eta, w);
#pragma unroll
  for (int i = 0; i < N; i++) w[i] += e1.b[i];
  mv<N, N>(K, w, tv);
  mv<N, N>(e2.A, tv, r.b);
#pragma unroll
  for (int i = 0; i < N; i++) r.b[i] += e2.b[i];
  // J
  mm<N, N, N>(e2.J, e1.A, t1);
  mtm<N, N, N>(K, t1, t2);
  mtm<N, N, N>(e1.A, t2, r.J);
#pragma unroll
  for (int i = 0; i < N * N; i++) r.J[i] += e1.J[i];
  // eta
  mv<N, N>(e2.J, e1.b, w);
#pragma unroll
  for (int i = 0; i < N; i++) w[i] = e2.eta[i] - w[i];
  mtv<N, N>(K, w, tv);
  mtv<N, N>(e1.A, tv, r.eta);
#pragma unroll
  for (int i = 0; i < N; i++) r.eta[i] += e1.eta[i];
  symmetrize<N>(r.C);
  symmetrize<N>(r.J);
  o = r;
}

// Value operator (eq. value-fun-param): K = (I + C1 J2)^{-1} with C1 J2 formed in L and
// I + C1 J2 inverted in SV (FP64, or FP32 in the all-FP32 mode), then value_apply_K in L.
// Returns false when I + C1 J2 is singular.
template <class SV = double>
struct ValueOp {
  template <int N, class L>
  PTN_HD bool operator()(const Val<N, L>& e1, const Val<N, L>& e2, Val<N, L>& o) const {
    // I + C1 J2 is formed in L and solved in SV ("FP32 arrays, FP64 solves")
    L Ml[N * N];
    mm<N, N, N>(e1.C, e2.J, Ml);
    SV Md[N * N];
#pragma unroll
    for (int i = 0; i < N * N; i++) Md[i] = cvt_solve<SV>(Ml[i]);
#pragma unroll
    for (int i = 0; i < N; i++) Md[i * N + i] += SV(1);
    if (!inv_gj<N, SV>(Md)) return false;
    L K[N * N];
#pragma unroll
    for (int i = 0; i < N * N; i++) K[i] = cvt_solve<L>(Md[i]);
    value_apply_K<N, L>(e1, e2, K, o);
    return true;
  }
};

// Element initialisation eq. value-fun-elem-init in the P^{-1}-free form
//   A = F - G R~^{-1} M^T, J = P - M R~^{-1} M^T, C = G R~^{-1} G^T,
//   eta = M R~^{-1} d, b = -G R~^{-1} d,  R~ = R + alpha I,
// identical to the printed q_t, r_t form whenever P_t is invertible.  The LDL^T
// factorisation and solve of R~ run in SV; the products in L.
// Returns false when R~ is not positive definite.
template <int N, int U, class L, class SV>
PTN_HD bool value_init(const L* F, const L* G, const L* Pm, const L* Mm, const L* Rm, const double* d,
                       double alpha, Val<N, L>& e) {
  constexpr int C = 2 * N + 1;
  SV Rt[U * U], X[U * C];
#pragma unroll
  for (int i = 0; i < U * U; i++) Rt[i] = SV(Rm[i]);
#pragma unroll
  for (int i = 0; i < U; i++) Rt[i * U + i] += SV(alpha);
  if (!ldlt<U, SV>(Rt)) return false;
#pragma unroll
  for (int i = 0; i < U; i++) {
#pragma unroll (N <= 8 ? N : 4)
    for (int j = 0; j < N; j++) {
      X[i * C + j] = SV(Mm[j * U + i]);
      X[i * C + N + j] = SV(G[j * U + i]);
    }
    X[i * C + 2 * N] = SV(d[i]);
  }
  ldlt_solve<U, C, SV>(Rt, X);
  L XL[U * C];
#pragma unroll
  for (int i = 0; i < U * C; i++) XL[i] = L(X[i]);
  // XL = R~^{-1} [M^T | G^T | d]  (U x (2N+1))
#pragma unroll (N <= 8 ? N : 1)
  for (int i = 0; i < N; i++) {
#pragma unroll (N <= 8 ? N : 2)
    for (int j = 0; j < N; j++) {
      L gm = L(0), mx = L(0), gg = L(0);
#pragma unroll
      for (int k = 0; k < U; k++) {
        gm += G[i * U + k] * XL[k * C + j];
        mx += Mm[i * U + k] * XL[k * C + j];
        gg += G[i * U + k] * XL[k * C + N + j];
      }
      e.A[i * N + j] = F[i * N + j] - gm;
      e.J[i * N + j] = Pm[i * N + j] - mx;
      e.C[i * N + j] = gg;
    }
    L et = L(0), bb = L(0);
#pragma unroll
    for (int k = 0; k < U; k++) {
      et += Mm[i * U + k] * XL[k * C + 2 * N];
      bb += G[i * U + k] * XL[k * C + 2 * N];
    }
    e.eta[i] = et;
    e.b[i] = -bb;
  }
  symmetrize<N>(e.J);
  symmetrize<N>(e.C);
  return true;
}

// Value combination of one step's element nu_t (eq. value-fun-elem-init) with a later
// element e (eq. value-fun-param, nu_t first), in place: the same element as
// ValueOp(value_init(F, G, P, M, R, d), e), written through the Woodbury identity.  The
// step's C_t = G R~^{-1} G^T has rank U, so with Q = R~ + G^T J G (U x U)
//   (I + C_t J)^{-1} = I - G Q^{-1} G^T J,
// and the combination becomes one backward Bellman step of (J, eta) -- the recursion of
// eq. value-fun-feedback with S = J, s = -eta -- plus the propagation of A, b and C:
//   H = M^T + G^T J F,   Gam = -Q^{-1} H,   gam = Q^{-1} (G^T eta - d)
//   J   <- P + F^T J F + H^T Gam
//   eta <- F^T eta - H^T gam
//   A   <- A (F + G Gam)
//   b   <- b + (A G) gam
//   C   <- C + (A G) Q^{-1} (A G)^T
// (A, b, C, J, eta of e on the right-hand sides).  Q is formed in L and inverted in SV:
// one U x U solve replaces the N x N inverse of I + C_t J.  Returns false when Q is
// singular (then I + C_t J is singular as well: det(I + C_t J) = det Q / det R~).
template <int N, int U, class L, class SV>
PTN_HD bool value_fold_step(const L* F, const L* G, const L* Pm, const L* Mm, const L* Rm, const double* d,
                            double alpha, Val<N, L>& e) {
  L JG[N * U], JF[N * N], GJG[U * U], H[U * N], Ge[U];
  mm<N, N, U>(e.J, G, JG);
  mm<N, N, N>(e.J, F, JF);
  mtm<U, N, U>(G, JG, GJG);
  mtm<U, N, N>(G, JF, H);
  mtv<N, U>(G, e.eta, Ge);
#pragma unroll
  for (int i = 0; i < U; i++)
#pragma unroll (N <= 8 ? N : 4)
    for (int j = 0; j < N; j++) H[i * N + j] += Mm[j * U + i];
  SV Q[U * U];
#pragma unroll
  for (int i = 0; i < U; i++)
#pragma unroll
    for (int j = 0; j < U; j++) Q[i * U + j] = SV(Rm[i * U + j]) + SV(GJG[i * U + j]) + (i == j ? SV(alpha) : SV(0));
  if (!inv_gj<U, SV>(Q)) return false;
  L Gam[U * N], gam[U], Qi[U * U];
#pragma unroll
  for (int i = 0; i < U; i++) {
#pragma unroll (N <= 8 ? N : 4)
    for (int j = 0; j < N; j++) {
      SV s = SV(0);
#pragma unroll
      for (int k = 0; k < U; k++) s += Q[i * U + k] * SV(H[k * N + j]);
      Gam[i * N + j] = L(-s);
    }
    SV s = SV(0);
#pragma unroll
    for (int k = 0; k < U; k++) s += Q[i * U + k] * (SV(Ge[k]) - SV(d[k]));
    gam[i] = L(s);
#pragma unroll
    for (int j = 0; j < U; j++) Qi[i * U + j] = L(Q[i * U + j]);
  }
  // J and eta: the Bellman step
  L Jn[N * N], HG[N * N], Fe[N], Hg[N];
  mtm<N, N, N>(F, JF, Jn);
  mtm<N, U, N>(H, Gam, HG);
#pragma unroll (N <= 8 ? N * N : 4)
  for (int i = 0; i < N * N; i++) Jn[i] += Pm[i] + HG[i];
  symmetrize<N>(Jn);
  mtv<N, N>(F, e.eta, Fe);
  mtv<U, N>(H, gam, Hg);
  // A, b, C: propagated through the closed loop F + G Gam of this step
  L Fc[N * N], AG[N * U], An[N * N], AGg[N], AQ[N * U], Cn[N * N];
  mm<N, U, N>(G, Gam, Fc);
#pragma unroll (N <= 8 ? N * N : 4)
  for (int i = 0; i < N * N; i++) Fc[i] += F[i];
  mm<N, N, U>(e.A, G, AG);
  mm<N, N, N>(e.A, Fc, An);
  mv<N, U>(AG, gam, AGg);
  mm<N, U, U>(AG, Qi, AQ);
  mmt<N, U, N>(AQ, AG, Cn);
#pragma unroll (N <= 8 ? N * N : 4)
  for (int i = 0; i < N * N; i++) {
    e.A[i] = An[i];
    e.C[i] += Cn[i];
    e.J[i] = Jn[i];
  }
  symmetrize<N>(e.C);
#pragma unroll
  for (int i = 0; i < N; i++) {
    e.eta[i] = Fe[i] - Hg[i];
    e.b[i] += AGg[i];
  }
  return true;
}

// Terminal element nu_{N+1}: J = P_{N+1}, all other parameters zero.
template <int N, class L>
PTN_HD void value_terminal(const L* PT, Val<N, L>& e) {
#pragma unroll
  for (int i = 0; i < N * N; i++) { e.A[i] = L(0); e.C[i] = L(0); e.J[i] = L(PT[i]); }
#pragma unroll
  for (int i = 0; i < N; i++) { e.eta[i] = L(0); e.b[i] = L(0); }
}

// One backward Bellman step from V_{t+1} = (S, s) (eq. linearized-ocp-bellman): the
// element nu_t applied to a boundary value function, written through the feedback law
// eq. value-fun-feedback (reading: Q^{-1} M_t^T):
//   Q = R~ + G^T S G,  Gam = -Q^{-1}(M^T + G^T S F),  gam = -Q^{-1}(d + G^T s),
//   S_t = P + F^T S F + (M^T + G^T S F)^T Gam,  s_t = F^T s + (M^T + G^T S F)^T gam.
// Q is factorised in SV.  S, s are updated in place.  Returns false when Q is not PD.
template <int N, int U, class L, class SV>
PTN_HD bool riccati_step(const L* F, const L* G, const L* Pm, const L* Mm, const L* Rm, const double* d,
                         double alpha, L* S, L* s, L* Gam, L* gam) {
  L SG[N * U], SF[N * N], Qux[U * N], GSG[U * U];
  mm<N, N, U>(S, G, SG);
  mm<N, N, N>(S, F, SF);
  mtm<U, N, U>(G, SG, GSG);
  mtm<U, N, N>(G, SF, Qux);
  SV Q[U * U], X[U * (N + 1)];
#pragma unroll
  for (int i = 0; i < U; i++)
#pragma unroll
    for (int j = 0; j < U; j++) Q[i * U + j] = SV(Rm[i * U + j]) + SV(GSG[i * U + j]) + (i == j ? SV(alpha) : SV(0));
  L Gs[U];
  mtv<N, U>(G, s, Gs);
#pragma unroll
  for (int i = 0; i < U; i++) {
#pragma unroll (N <= 8 ? N : 4)
    for (int j = 0; j < N; j++) {
      Qux[i * N + j] += Mm[j * U + i];
      X[i * (N + 1) + j] = SV(Qux[i * N + j]);
    }
    X[i * (N + 1) + N] = SV(d[i]) + SV(Gs[i]);
  }
  if (!ldlt<U, SV>(Q)) return false;
  ldlt_solve<U, N + 1, SV>(Q, X);
#pragma unroll
  for (int i = 0; i < U; i++) {
#pragma unroll (N <= 8 ? N : 4)
    for (int j = 0; j < N; j++) Gam[i * N + j] = L(-X[i * (N + 1) + j]);
    gam[i] = L(-X[i * (N + 1) + N]);
  }
  L Sn[N * N], sn[N], FtSF[N * N], QG[N * N];
  mtm<N, N, N>(F, SF, FtSF);
  mtm<N, U, N>(Qux, Gam, QG);
#pragma unroll (N <= 8 ? N * N : 4)
  for (int i = 0; i < N * N; i++) Sn[i] = Pm[i] + FtSF[i] + QG[i];
  L Fts[N], Qg[N];
  mtv<N, N>(F, s, Fts);
  mtv<U, N>(Qux, gam, Qg);
#pragma unroll
  for (int i = 0; i < N; i++) sn[i] = Fts[i] + Qg[i];
  symmetrize<N>(Sn);
#pragma unroll
  for (int i = 0; i < N * N; i++) S[i] = Sn[i];
#pragma unroll
  for (int i = 0; i < N; i++) s[i] = sn[i];
  return true;
}

}  // namespace ptn
