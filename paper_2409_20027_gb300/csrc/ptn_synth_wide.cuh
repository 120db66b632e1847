// ptn_synth_wide.cuh -- the synthetic benchmark map x+ = A x + B u + c tanh(W x) (n = 32,
// m = 8, c = prm[0]) on the wide tier: its closed-form terms computed by the lanes of a
// warp, row i of W x by lane i (ptn_synth.cuh gives the same formulas for one thread):
//
//   F = df/dx = A + c diag(1 - tanh^2(W x)) W,      G = df/du = B,
//   (lam^T f)_xx = c W^T diag(lam o tanh''(W x)) W,  tanh''(y) = -2 tanh(y) (1 - tanh^2(y)),
//   (lam^T f)_xu = 0,  (lam^T f)_uu = 0.
//
// The map is discrete: the problem's integrator and time step do not enter.  FP32 terms use
// the problem's FP32 copies of A, B, W (one rounding of the matrices, no FP64 work).
#pragma once
#include "ptn_synth.cuh"
#include "ptn_wide.cuh"

namespace ptn {

struct Synth {
  static constexpr int NX = 32, NU = 8, NP = 1, ID = MODEL_SYNTH;
};

template <>
struct WModel<Synth> {
  static constexpr int N = Synth::NX, U = Synth::NU;
  static_assert(N <= 32, "one row of W x per lane");
  static constexpr bool has_adjoint = false;

  // tanh((W x)_l) in lane l < N (FP64)
  __device__ static double row_tanh(const ProbS<N, U>& P, const double* x) {
    const int l = wops::lane_id();
    const double y = l < N ? wops::dot4<N, double>([&](int j) { return P.W[l * N + j] * x[j]; }) : 0.0;
    return tanh(y);
  }

  template <class S>
  __device__ static void jac(const ProbS<N, U>& P, const double* x, const double* u, S* F, S* G, double* tmp) {
    (void)u;
    const int l = wops::lane_id();
    const double t = row_tanh(P, x);
    const double sc = P.prm[0] * (1.0 - t * t);
    if constexpr (std::is_same<S, float>::value) {
      float* sf = reinterpret_cast<float*>(tmp);
      if (l < N) sf[l] = float(sc);
      __syncwarp();
      for (int e = l; e < N * N; e += 32) F[e] = P.A32[e] + sf[e / N] * P.W32[e];
      for (int e = l; e < N * U; e += 32) G[e] = P.B32[e];
    } else {
      if (l < N) tmp[l] = sc;
      __syncwarp();
      for (int e = l; e < N * N; e += 32) F[e] = S(P.A[e] + tmp[e / N] * P.W[e]);
      for (int e = l; e < N * U; e += 32) G[e] = S(P.B[e]);
    }
    __syncwarp();
  }

  // wrk: N x N values of L of the warp's scratch
  template <class L>
  __device__ static void hess(const ProbS<N, U>& P, const double* x, const double* u, const double* lam, L* Hxx,
                              L* Hxu, L* Huu, double* tmp, L* wrk) {
    (void)u;
    const int l = wops::lane_id();
    const double t = row_tanh(P, x);
    const double wk = (l < N) ? P.prm[0] * lam[l] * (-2.0 * t * (1.0 - t * t)) : 0.0;
    if constexpr (std::is_same<L, float>::value) {
      // Hxx = W^T (diag(w) W): the scaled rows in wrk, the product on the tensor cores
      float* wf = reinterpret_cast<float*>(tmp);
      if (l < N) wf[l] = float(wk);
      __syncwarp();
      for (int e = l; e < N * N; e += 32) wrk[e] = wf[e / N] * P.W32[e];
      __syncwarp();
      wops::mm<N, N, N, true, false>(P.W32, wrk, Hxx);
    } else {
      if (l < N) tmp[l] = wk;
      __syncwarp();
      for (int e = l; e < N * N; e += 32) {
        const int i = e / N, j = e % N;
        Hxx[e] = L(wops::dot4<N, double>([&](int k) { return P.W[k * N + i] * tmp[k] * P.W[k * N + j]; }));
      }
    }
    for (int e = l; e < N * U; e += 32) Hxu[e] = L(0);
    for (int e = l; e < U * U; e += 32) Huu[e] = L(0);
    __syncwarp();
  }

  // xn = A x + B u + c tanh(W x) (FP64), component l by lane l
  __device__ static void step(const ProbS<N, U>& P, const double* x, const double* u, double* xn, double* tmp) {
    (void)tmp;
    const int l = wops::lane_id();
    if (l < N) {
      const double y = wops::dot4<N, double>([&](int j) { return P.W[l * N + j] * x[j]; });
      const double v = wops::dot4<N, double>([&](int j) { return P.A[l * N + j] * x[j]; }) +
                       wops::dot4<U, double>([&](int k) { return P.B[l * U + k] * u[k]; });
      xn[l] = v + P.prm[0] * tanh(y);
    }
    __syncwarp();
  }
};

// two warps' scratch per CTA fit in shared memory at n = 32
template <>
struct WideMaxThreads<Synth> {
  static constexpr int value = 64;
};

}  // namespace ptn
