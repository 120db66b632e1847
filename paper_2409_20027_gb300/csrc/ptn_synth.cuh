// ptn_synth.cuh -- the synthetic benchmark dynamics x+ = A x + B u + c tanh(W x) with
// closed-form derivatives (A, W: NX x NX, B: NX x NU, row-major; c = prm[0]).  It is a
// discrete map: the problem's integrator and time step do not enter.
//
//   F = df/dx = A + c diag(1 - tanh^2(W x)) W,      G = df/du = B,
//   lam . f_xx = c W^T diag(lam o tanh''(W x)) W,   tanh''(y) = -2 tanh(y) (1 - tanh^2(y)),
//   f_xu = 0,  f_uu = 0.
//
// Plain loops in scalar S (accumulation in S), for host and device; the building block of
// the n = 32, m = 8 workload's model terms.
#pragma once
#include <math.h>

#include "ptn_common.cuh"

namespace ptn {

template <int NX_, int NU_>
struct SynthMap {
  static constexpr int NX = NX_, NU = NU_;

  // y = W x and t = tanh(y) (FP64)
  PTN_HD static void pre(const double* W, const double* x, double* t) {
    for (int i = 0; i < NX; i++) {
      double y = 0.0;
      for (int j = 0; j < NX; j++) y += W[i * NX + j] * x[j];
      t[i] = tanh(y);
    }
  }

  // x+ (FP64)
  PTN_HD static void step(const double* A, const double* B, const double* W, double c, const double* x,
                          const double* u, double* xn) {
    double t[NX];
    pre(W, x, t);
    for (int i = 0; i < NX; i++) {
      double v = c * t[i];
      for (int j = 0; j < NX; j++) v += A[i * NX + j] * x[j];
      for (int j = 0; j < NU; j++) v += B[i * NU + j] * u[j];
      xn[i] = v;
    }
  }

  // F, G in scalar S
  template <class S>
  PTN_HD static void jac(const double* A, const double* B, const double* W, double c, const double* x, S* F,
                         S* G) {
    double t[NX];
    pre(W, x, t);
    for (int i = 0; i < NX; i++) {
      const double s = c * (1.0 - t[i] * t[i]);
      for (int j = 0; j < NX; j++) F[i * NX + j] = S(A[i * NX + j] + s * W[i * NX + j]);
      for (int j = 0; j < NU; j++) G[i * NU + j] = S(B[i * NU + j]);
    }
  }

  // Hxx = lam . f_xx in scalar S (Hxu, Huu are zero)
  template <class S>
  PTN_HD static void hess_xx(const double* W, double c, const double* x, const double* lam, S* Hxx) {
    double t[NX], w[NX];
    pre(W, x, t);
    for (int k = 0; k < NX; k++) w[k] = c * lam[k] * (-2.0 * t[k] * (1.0 - t[k] * t[k]));
    for (int i = 0; i < NX; i++)
      for (int j = i; j < NX; j++) {
        S h = S(0);
        for (int k = 0; k < NX; k++) h += S(W[k * NX + i] * w[k] * W[k * NX + j]);
        Hxx[i * NX + j] = h;
        Hxx[j * NX + i] = h;
      }
  }
};

}  // namespace ptn
