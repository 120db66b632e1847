// ptn_common.cuh -- shared device types for the parallel-in-time Newton solver
// (arXiv 2409.20027): status codes, problem/option records, small register-resident
// linear algebra and forward-mode automatic-differentiation scalars.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <type_traits>

#define PTN_MAXN 32
#define PTN_MAXM 8
#define PTN_MAXW (2 * PTN_MAXN + 2 * PTN_MAXM)
#define PTN_MAXP 8

#define PTN_HD __host__ __device__ __forceinline__

namespace ptn {

// ---- status codes (mirrors include/ptn.h) ----
enum : int {
  ST_OK = 0,
  ST_EINVAL = -1,
  ST_EINFEAS = -2,
  ST_ENOTCONV = -3,
  ST_ENUM = -4,
  ST_ETIMEOUT = -5,
  ST_ECUDA = -6,
};

enum : int { AUG_BARRIER = 1, AUG_ADMM = 2 };

// Problem record in device memory.  Constraint rows w_r = sgn_r (z_k - bnd_r) <= 0 are
// listed state rows first (per component: upper, lower), then control rows.
struct ProbDev {
  int model, nx, nu, integrator;
  int nw, pad0, pad1, pad2;
  double dt;
  double prm[PTN_MAXP];
  double Q[PTN_MAXN * PTN_MAXN];
  double R[PTN_MAXM * PTN_MAXM];
  double Qf[PTN_MAXN * PTN_MAXN];
  double xref[PTN_MAXN];
  double uref[PTN_MAXM];
  int row_isx[PTN_MAXW];
  int row_idx[PTN_MAXW];
  double row_sgn[PTN_MAXW];
  double row_bnd[PTN_MAXW];
  const double* A;  // synthetic model: nx*nx
  const double* B;  // nx*nu
  const double* W;  // nx*nx
  const float* A32;  // the same in FP32 (the model's FP32 terms)
  const float* B32;
  const float* W32;
};

struct OptDev {
  double mu0, zeta, mu_final, tol_inner, tol_final, rho, admm_tol;
  double alpha0, alpha_min, alpha_max, ls_beta, armijo_c1, armijo_eps;
  double roll_tol, polish, armijo_eps32;
  int max_newton, max_outer, ls_count, admm_fixed_iters;
  int roll_max_iter, method, polish_after, init_max_iter;
  int costate_mode;        // 0: co-state scan (Alg. 1); 1, 2: multiplier forms
  int update_mode;         // 0: step on the closed-loop rollout; 1: x += dx, u += du (Alg. 4)
  int init_parallel64;     // nonzero: FP64 kernels also build the initial nominal in parallel
  int stall_exit;          // > 0: mixed modes leave a stalled final level (FP64 finish follows)
  long long spin_limit;  // bounded waits in grid barriers
};

// per-instance description (device array)
struct InstDev {
  int T;        // horizon (controls u_0..u_{T-1}, states x_0..x_T)
  int xoff;     // offset of x_0 in state-major arrays, in steps (sum of previous T+1)
  int uoff;     // offset of u_0 in control-major arrays, in steps (sum of previous T)
  int pad;
  double dt;    // > 0: this instance's time step (stage weights scaled by dt / problem dt)
};

// per-instance statistics (device array, copied to the host)
struct InfoDev {
  int status, newton_iters, outer_iters, ls_rejects;
  int factor_fails, roll_fails, roll_iters, ls_evals;
  int exact_passes, pad_;
  double mu, alpha, r_stat, r_dyn, r_feas, r_kkt, J, J_c, r_p, r_d;
  // SM clock cycles spent by group thread 0 per phase (costate, quadratize, value,
  // state, line search, initial rollout, other)
  long long cyc[7];
};

// ---------------------------------------------------------------------------
// small dense linear algebra on row-major register arrays.  Products up to
// PTN_UNROLL_MAX multiply-adds are fully unrolled (register-resident operands);
// larger ones run as loops (operands in local memory).
// ---------------------------------------------------------------------------
#define PTN_UNROLL_MAX 512

template <int R, int K, int C, class S, class T1, class T2>
PTN_HD void mm(const T1* A, const T2* B, S* O) {
  if constexpr (R * K * C <= PTN_UNROLL_MAX) {
#pragma unroll
    for (int i = 0; i < R; i++)
#pragma unroll
      for (int j = 0; j < C; j++) {
        S s = S(0);
#pragma unroll
        for (int l = 0; l < K; l++) s += S(A[i * K + l]) * S(B[l * C + j]);
        O[i * C + j] = s;
      }
  } else {
#pragma unroll 1
    for (int i = 0; i < R; i++)
#pragma unroll 1
      for (int j = 0; j < C; j++) {
        S s = S(0);
#pragma unroll 4
        for (int l = 0; l < K; l++) s += S(A[i * K + l]) * S(B[l * C + j]);
        O[i * C + j] = s;
      }
  }
}
// O = A^T B, A is K x R, B is K x C
template <int R, int K, int C, class S, class T1, class T2>
PTN_HD void mtm(const T1* A, const T2* B, S* O) {
  if constexpr (R * K * C <= PTN_UNROLL_MAX) {
#pragma unroll
    for (int i = 0; i < R; i++)
#pragma unroll
      for (int j = 0; j < C; j++) {
        S s = S(0);
#pragma unroll
        for (int l = 0; l < K; l++) s += S(A[l * R + i]) * S(B[l * C + j]);
        O[i * C + j] = s;
      }
  } else {
#pragma unroll 1
    for (int i = 0; i < R; i++)
#pragma unroll 1
      for (int j = 0; j < C; j++) {
        S s = S(0);
#pragma unroll 4
        for (int l = 0; l < K; l++) s += S(A[l * R + i]) * S(B[l * C + j]);
        O[i * C + j] = s;
      }
  }
}
// O = A B^T, A is R x K, B is C x K
template <int R, int K, int C, class S, class T1, class T2>
PTN_HD void mmt(const T1* A, const T2* B, S* O) {
  if constexpr (R * K * C <= PTN_UNROLL_MAX) {
#pragma unroll
    for (int i = 0; i < R; i++)
#pragma unroll
      for (int j = 0; j < C; j++) {
        S s = S(0);
#pragma unroll
        for (int l = 0; l < K; l++) s += S(A[i * K + l]) * S(B[j * K + l]);
        O[i * C + j] = s;
      }
  } else {
#pragma unroll 1
    for (int i = 0; i < R; i++)
#pragma unroll 1
      for (int j = 0; j < C; j++) {
        S s = S(0);
#pragma unroll 4
        for (int l = 0; l < K; l++) s += S(A[i * K + l]) * S(B[j * K + l]);
        O[i * C + j] = s;
      }
  }
}
template <int R, int C, class S, class T1>
PTN_HD void mv(const T1* A, const S* x, S* y) {
  if constexpr (R * C <= PTN_UNROLL_MAX) {
#pragma unroll
    for (int i = 0; i < R; i++) {
      S s = S(0);
#pragma unroll
      for (int j = 0; j < C; j++) s += S(A[i * C + j]) * x[j];
      y[i] = s;
    }
  } else {
#pragma unroll 1
    for (int i = 0; i < R; i++) {
      S s = S(0);
#pragma unroll 4
      for (int j = 0; j < C; j++) s += S(A[i * C + j]) * x[j];
      y[i] = s;
    }
  }
}
// y = A^T x, A is R x C
template <int R, int C, class S, class T1>
PTN_HD void mtv(const T1* A, const S* x, S* y) {
  if constexpr (R * C <= PTN_UNROLL_MAX) {
#pragma unroll
    for (int j = 0; j < C; j++) {
      S s = S(0);
#pragma unroll
      for (int i = 0; i < R; i++) s += S(A[i * C + j]) * x[i];
      y[j] = s;
    }
  } else {
#pragma unroll 1
    for (int j = 0; j < C; j++) {
      S s = S(0);
#pragma unroll 4
      for (int i = 0; i < R; i++) s += S(A[i * C + j]) * x[i];
      y[j] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 helpers for the solves of the mixed modes.  On this GPU every FP64 warp instruction
// (DFMA, conversions to and from FP32 included) occupies the SM sub-partition's FP64 pipe
// for about 64 cycles, whatever the number of active lanes, and a correctly rounded FP64
// division takes about nine of them.  The solves of I + C1 J2 and of the U x U blocks are
// on the scans' critical paths, so their pivots and conversions avoid that pipe where
// plain arithmetic allows.

// Pivot test and reciprocal.  Device FP64: pivots with a binary exponent outside
// [-1000, 1000] count as singular (as zero or non-finite pivots do everywhere), and the
// reciprocal is the hardware's approximation (rcp.approx.ftz.f64) refined by two steps of
// Newton's iteration for f(r) = 1/r - p, r <- r + r (1 - p r), each of which squares the
// relative error; the result is within one unit in the last place of 1/p.  Elsewhere
// (FP32, host code): the division.
template <class S>
PTN_HD bool pivot_ok(S p) {
#ifdef __CUDA_ARCH__
  if constexpr (std::is_same<S, double>::value) {
    const unsigned e = (unsigned)((unsigned long long)__double_as_longlong(p) >> 52) & 0x7ffu;
    return e >= 1023u - 1000u && e <= 1023u + 1000u;
  }
#endif
  return (p != S(0)) && isfinite(p);
}
template <class S>
PTN_HD S pivot_rcp(S p) {
#ifdef __CUDA_ARCH__
  if constexpr (std::is_same<S, double>::value) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(p));
    double e = fma(-p, r, 1.0);
    r = fma(r, e, r);
    e = fma(-p, r, 1.0);
    return fma(r, e, r);
  }
#endif
  return S(1) / p;
}

// FP32 <-> FP64 conversions by integer operations on the IEEE-754 fields (device code,
// off the FP64 pipe).  Exact for zeros, normal numbers and infinities; a NaN stays a NaN
// (FP32 -> FP64: payload kept and quieted; FP64 -> FP32: the canonical quiet NaN).  Round
// to nearest even from FP64, as the conversion instruction; FP32 subnormals (below 2^-126
// in magnitude) become signed zeros in both directions.  The bit-field functions are the
// same on host and device (checked over every FP32 bit pattern on the host); host code
// converts natively.
PTN_HD void f32_bits_to_f64_bits(unsigned u, unsigned& hi, unsigned& lo) {
  const unsigned sg = u & 0x80000000u, e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  hi = sg | ((e + 896u) << 20) | (m >> 3);
  lo = m << 29;
  if (e == 0u) { hi = sg; lo = 0u; }
  if (e == 255u) hi = sg | 0x7ff00000u | (m >> 3) | (m != 0u ? 0x80000u : 0u);
}
PTN_HD unsigned f64_bits_to_f32_bits(unsigned hi, unsigned lo) {
  const unsigned sg = hi & 0x80000000u, ef = (hi >> 20) & 0x7ffu;
  const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29), rest = lo & 0x1fffffffu;
  const unsigned up = (rest > 0x10000000u || (rest == 0x10000000u && (mant & 1u))) ? 1u : 0u;
  const int e = (int)ef - 896;
  unsigned r = ((unsigned)e << 23) + mant + up;  // a carry out of the mantissa bumps e
  if (e <= 0) r = 0u;
  else if (e >= 255 || r >= 0x7f800000u) r = 0x7f800000u;
  if (ef == 0x7ffu) r = ((hi & 0xfffffu) | lo) != 0u ? 0x7fc00000u : 0x7f800000u;
  return sg | r;
}
PTN_HD double f32_to_f64(float f) {
#ifdef __CUDA_ARCH__
  unsigned hi, lo;
  f32_bits_to_f64_bits(__float_as_uint(f), hi, lo);
  return __hiloint2double((int)hi, (int)lo);
#else
  return double(f);
#endif
}
PTN_HD float f64_to_f32(double d) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(f64_bits_to_f32_bits((unsigned)__double2hiint(d), (unsigned)__double2loint(d)));
#else
  return float(d);
#endif
}
// L <-> SV conversions of the solves: the integer forms for FP32 <-> FP64
template <class To, class From>
PTN_HD To cvt_solve(From x) {
  if constexpr (std::is_same<From, float>::value && std::is_same<To, double>::value) return f32_to_f64(x);
  else if constexpr (std::is_same<From, double>::value && std::is_same<To, float>::value) return f64_to_f32(x);
  else return To(x);
}

// In-place Cholesky A = L L^T (lower triangle written, upper untouched).
// Returns false when A is not positive definite.
template <int N, class S = double>
PTN_HD bool chol(S* A) {
#pragma unroll
  for (int j = 0; j < N; j++) {
    S s = A[j * N + j];
#pragma unroll
    for (int k = 0; k < j; k++) s -= A[j * N + k] * A[j * N + k];
    if (!(s > S(0)) || !isfinite(s)) return false;
    S d = sqrt(s), id = S(1) / d;
    A[j * N + j] = d;
#pragma unroll
    for (int i = j + 1; i < N; i++) {
      S t = A[i * N + j];
#pragma unroll
      for (int k = 0; k < j; k++) t -= A[i * N + k] * A[j * N + k];
      A[i * N + j] = t * id;
    }
  }
  return true;
}
// solve (L L^T) X = B in place, B is N x C
template <int N, int C, class S = double>
PTN_HD void chol_solve(const S* L, S* B) {
#pragma unroll
  for (int c = 0; c < C; c++) {
#pragma unroll
    for (int i = 0; i < N; i++) {
      S s = B[i * C + c];
#pragma unroll
      for (int k = 0; k < i; k++) s -= L[i * N + k] * B[k * C + c];
      B[i * C + c] = s / L[i * N + i];
    }
#pragma unroll
    for (int i = N - 1; i >= 0; i--) {
      S s = B[i * C + c];
#pragma unroll
      for (int k = i + 1; k < N; k++) s -= L[k * N + i] * B[k * C + c];
      B[i * C + c] = s / L[i * N + i];
    }
  }
}

// LDL^T factorisation of a symmetric positive definite matrix in place: the unit lower
// factor below the diagonal and the reciprocal pivots 1/D_j on it.  One division per
// pivot and no square root, which matters where S = double on GB300's FP64 pipe.
// Returns false when a pivot is not positive and finite (A not positive definite).
template <int N, class S = double>
PTN_HD bool ldlt(S* A) {
  S D[N];
#pragma unroll
  for (int j = 0; j < N; j++) {
    S dj = A[j * N + j];
#pragma unroll
    for (int k = 0; k < j; k++) dj -= A[j * N + k] * A[j * N + k] * D[k];
    if (!(dj > S(0)) || !pivot_ok(dj)) return false;
    const S id = pivot_rcp(dj);
    D[j] = dj;
    A[j * N + j] = id;
#pragma unroll
    for (int i = j + 1; i < N; i++) {
      S t = A[i * N + j];
#pragma unroll
      for (int k = 0; k < j; k++) t -= A[i * N + k] * A[j * N + k] * D[k];
      A[i * N + j] = t * id;
    }
  }
  return true;
}

// solve (L D L^T) X = B in place with the factor of ldlt(), B is N x C
template <int N, int C, class S = double>
PTN_HD void ldlt_solve(const S* A, S* B) {
#pragma unroll
  for (int c = 0; c < C; c++) {
#pragma unroll
    for (int i = 0; i < N; i++) {
      S s = B[i * C + c];
#pragma unroll
      for (int k = 0; k < i; k++) s -= A[i * N + k] * B[k * C + c];
      B[i * C + c] = s;
    }
#pragma unroll
    for (int i = 0; i < N; i++) B[i * C + c] *= A[i * N + i];
#pragma unroll
    for (int i = N - 1; i >= 0; i--) {
      S s = B[i * C + c];
#pragma unroll
      for (int k = i + 1; k < N; k++) s -= A[k * N + i] * B[k * C + c];
      B[i * C + c] = s;
    }
  }
}

// magnitude order key of a float or double from its bit pattern (sign cleared, high word
// for doubles): integer comparisons, so pivot searches stay off the FP64 pipe
PTN_HD unsigned mag_key(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x) & 0x7fffffffu;
#else
  unsigned u;
  memcpy(&u, &x, sizeof(u));
  return u & 0x7fffffffu;
#endif
}
PTN_HD unsigned mag_key(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned)((unsigned long long)__double_as_longlong(x) >> 32) & 0x7fffffffu;
#else
  unsigned long long u;
  memcpy(&u, &x, sizeof(u));
  return (unsigned)(u >> 32) & 0x7fffffffu;
#endif
}

// In-place inverse by Gauss-Jordan elimination with partial pivoting (FP64).
// Returns false when a pivot is zero or not finite.
template <int N, class S = double>
PTN_HD bool inv_gj(S* A) {
  int piv[N];
#pragma unroll
  for (int i = 0; i < N; i++) piv[i] = i;
#pragma unroll (N <= 8 ? N : 1)
  for (int k = 0; k < N; k++) {
    // pivot: largest magnitude in column k at or below the diagonal (by bit pattern)
    int p = k;
    unsigned best = mag_key(A[k * N + k]);
#pragma unroll (N <= 8 ? N : 1)
    for (int i = k + 1; i < N; i++) {
      const unsigned v = mag_key(A[i * N + k]);
      if (v > best) { best = v; p = i; }
    }
    // row swap k <-> p as predicated moves with static indices (registers, not local memory)
#pragma unroll (N <= 8 ? N : 1)
    for (int i = k + 1; i < N; i++) {
      if (i == p) {
#pragma unroll (N <= 8 ? N : 4)
        for (int j = 0; j < N; j++) {
          S t = A[k * N + j]; A[k * N + j] = A[i * N + j]; A[i * N + j] = t;
        }
        int t = piv[k]; piv[k] = piv[i]; piv[i] = t;
      }
    }
    const S pv = A[k * N + k];
    if (!pivot_ok(pv)) return false;
    const S ip = pivot_rcp(pv);
    A[k * N + k] = S(1);
#pragma unroll (N <= 8 ? N : 4)
    for (int j = 0; j < N; j++) A[k * N + j] *= ip;
#pragma unroll (N <= 8 ? N : 1)
    for (int i = 0; i < N; i++) {
      if (i == k) continue;
      S f = A[i * N + k];
      A[i * N + k] = S(0);
#pragma unroll (N <= 8 ? N : 4)
      for (int j = 0; j < N; j++) A[i * N + j] -= f * A[k * N + j];
    }
  }
  // undo the row permutation as a column permutation of the inverse (column piv[j] of
  // the result is column j; selects with static indices keep A in registers)
  if constexpr (N <= 8) {
    S tmp[N * N];
#pragma unroll
    for (int i = 0; i < N; i++)
#pragma unroll
      for (int c = 0; c < N; c++) {
        S v = S(0);
#pragma unroll
        for (int j = 0; j < N; j++)
          if (piv[j] == c) v = A[i * N + j];
        tmp[i * N + c] = v;
      }
#pragma unroll
    for (int i = 0; i < N * N; i++) A[i] = tmp[i];
  } else {
    S tmp[N];
    for (int i = 0; i < N; i++) {
      for (int j = 0; j < N; j++) tmp[piv[j]] = A[i * N + j];
      for (int j = 0; j < N; j++) A[i * N + j] = tmp[j];
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// forward-mode AD scalars
// ---------------------------------------------------------------------------

// value + K first partial derivatives
template <class S, int K>
struct Dual {
  S v;
  S d[K];
  PTN_HD Dual() {}
  PTN_HD Dual(S c) : v(c) {
#pragma unroll
    for (int i = 0; i < K; i++) d[i] = S(0);
  }
};
template <class S, int K>
PTN_HD Dual<S, K> operator+(const Dual<S, K>& a, const Dual<S, K>& b) {
  Dual<S, K> r; r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < K; i++) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <class S, int K>
PTN_HD Dual<S, K> operator-(const Dual<S, K>& a, const Dual<S, K>& b) {
  Dual<S, K> r; r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < K; i++) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <class S, int K>
PTN_HD Dual<S, K> operator-(const Dual<S, K>& a) {
  Dual<S, K> r; r.v = -a.v;
#pragma unroll
  for (int i = 0; i < K; i++) r.d[i] = -a.d[i];
  return r;
}
template <class S, int K>
PTN_HD Dual<S, K> operator*(const Dual<S, K>& a, const Dual<S, K>& b) {
  Dual<S, K> r; r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < K; i++) r.d[i] = a.v * b.d[i] + a.d[i] * b.v;
  return r;
}
template <class S, int K>
PTN_HD Dual<S, K> operator*(S c, const Dual<S, K>& a) {
  Dual<S, K> r; r.v = c * a.v;
#pragma unroll
  for (int i = 0; i < K; i++) r.d[i] = c * a.d[i];
  return r;
}
template <class S, int K>
PTN_HD Dual<S, K> operator+(S c, const Dual<S, K>& a) {
  Dual<S, K> r = a; r.v = c + a.v; return r;
}
template <class S, int K>
PTN_HD Dual<S, K> recip(const Dual<S, K>& a) {
  Dual<S, K> r; S i = S(1) / a.v; r.v = i; S f = -i * i;
#pragma unroll
  for (int k = 0; k < K; k++) r.d[k] = f * a.d[k];
  return r;
}
template <class S, int K>
PTN_HD Dual<S, K> operator/(const Dual<S, K>& a, const Dual<S, K>& b) {
  return a * recip(b);
}
PTN_HD void sc_(double a, double* s, double* c) { sincos(a, s, c); }
PTN_HD void sc_(float a, float* s, float* c) { sincosf(a, s, c); }

PTN_HD void sincos_ad(double a, double& s, double& c);
PTN_HD void sincos_ad(float a, float& s, float& c);
template <class S, int K>
PTN_HD void sincos_ad(const Dual<S, K>& a, Dual<S, K>& s, Dual<S, K>& c) {
  S sv, cv;
  sincos_ad(a.v, sv, cv);
  s.v = sv; c.v = cv;
#pragma unroll
  for (int k = 0; k < K; k++) { s.d[k] = cv * a.d[k]; c.d[k] = -sv * a.d[k]; }
}

// value + K first partials + packed upper-triangular K x K second partials
template <class S, int K>
struct Jet {
  static constexpr int H = K * (K + 1) / 2;
  S v;
  S d[K];
  S h[H];
  PTN_HD Jet() {}
  PTN_HD Jet(S c) : v(c) {
#pragma unroll
    for (int i = 0; i < K; i++) d[i] = S(0);
#pragma unroll
    for (int i = 0; i < H; i++) h[i] = S(0);
  }
};
template <int K>
PTN_HD constexpr int hidx(int i, int j) {  // i <= j
  return i * K - (i * (i - 1)) / 2 + (j - i);
}
template <class S, int K>
PTN_HD Jet<S, K> operator+(const Jet<S, K>& a, const Jet<S, K>& b) {
  Jet<S, K> r; r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < K; i++) r.d[i] = a.d[i] + b.d[i];
#pragma unroll (K <= 8 ? Jet<S, K>::H : 4)
  for (int i = 0; i < Jet<S, K>::H; i++) r.h[i] = a.h[i] + b.h[i];
  return r;
}
template <class S, int K>
PTN_HD Jet<S, K> operator-(const Jet<S, K>& a, const Jet<S, K>& b) {
  Jet<S, K> r; r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < K; i++) r.d[i] = a.d[i] - b.d[i];
#pragma unroll (K <= 8 ? Jet<S, K>::H : 4)
  for (int i = 0; i < Jet<S, K>::H; i++) r.h[i] = a.h[i] - b.h[i];
  return r;
}
template <class S, int K>
PTN_HD Jet<S, K> operator-(const Jet<S, K>& a) {
  Jet<S, K> r; r.v = -a.v;
#pragma unroll
  for (int i = 0; i < K; i++) r.d[i] = -a.d[i];
#pragma unroll (K <= 8 ? Jet<S, K>::H : 4)
  for (int i = 0; i < Jet<S, K>::H; i++) r.h[i] = -a.h[i];
  return r;
}
template <class S, int K>
PTN_HD Jet<S, K> operator*(const Jet<S, K>& a, const Jet<S, K>& b) {
  Jet<S, K> r; r.v = a.v * b.v;
  if constexpr (K <= 8) {
#pragma unroll
    for (int i = 0; i < K; i++) r.d[i] = a.v * b.d[i] + a.d[i] * b.v;
#pragma unroll
    for (int i = 0; i < K; i++)
#pragma unroll
      for (int j = i; j < K; j++) {
        const int q = hidx<K>(i, j);
        r.h[q] = a.v * b.h[q] + a.h[q] * b.v + a.d[i] * b.d[j] + a.d[j] * b.d[i];
      }
  } else {
#pragma unroll 4
    for (int i = 0; i < K; i++) r.d[i] = a.v * b.d[i] + a.d[i] * b.v;
    int q = 0;
#pragma unroll 1
    for (int i = 0; i < K; i++)
#pragma unroll 2
      for (int j = i; j < K; j++, q++)
        r.h[q] = a.v * b.h[q] + a.h[q] * b.v + a.d[i] * b.d[j] + a.d[j] * b.d[i];
  }
  return r;
}
template <class S, int K>
PTN_HD Jet<S, K> operator*(S c, const Jet<S, K>& a) {
  Jet<S, K> r; r.v = c * a.v;
#pragma unroll
  for (int i = 0; i < K; i++) r.d[i] = c * a.d[i];
#pragma unroll (K <= 8 ? Jet<S, K>::H : 4)
  for (int i = 0; i < Jet<S, K>::H; i++) r.h[i] = c * a.h[i];
  return r;
}
template <class S, int K>
PTN_HD Jet<S, K> operator+(S c, const Jet<S, K>& a) {
  Jet<S, K> r = a; r.v = c + a.v; return r;
}
// chain rule for a scalar function with value f0, first derivative f1, second f2
template <class S, int K>
PTN_HD Jet<S, K> jfun(const Jet<S, K>& a, S f0, S f1, S f2) {
  Jet<S, K> r; r.v = f0;
  if constexpr (K <= 8) {
#pragma unroll
    for (int i = 0; i < K; i++) r.d[i] = f1 * a.d[i];
#pragma unroll
    for (int i = 0; i < K; i++)
#pragma unroll
      for (int j = i; j < K; j++) {
        const int q = hidx<K>(i, j);
        r.h[q] = f1 * a.h[q] + f2 * a.d[i] * a.d[j];
      }
  } else {
#pragma unroll 4
    for (int i = 0; i < K; i++) r.d[i] = f1 * a.d[i];
    int q = 0;
#pragma unroll 1
    for (int i = 0; i < K; i++)
#pragma unroll 2
      for (int j = i; j < K; j++, q++) r.h[q] = f1 * a.h[q] + f2 * a.d[i] * a.d[j];
  }
  return r;
}
template <class S, int K>
PTN_HD Jet<S, K> recip(const Jet<S, K>& a) {
  S i = S(1) / a.v;
  return jfun(a, i, -i * i, S(2) * i * i * i);
}
template <class S, int K>
PTN_HD Jet<S, K> operator/(const Jet<S, K>& a, const Jet<S, K>& b) {
  return a * recip(b);
}
template <class S, int K>
PTN_HD void sincos_ad(const Jet<S, K>& a, Jet<S, K>& s, Jet<S, K>& c) {
  S sv, cv;
  sc_(a.v, &sv, &cv);
  s = jfun(a, sv, cv, -sv);
  c = jfun(a, cv, -sv, -cv);
}

// plain scalars share the same interface
PTN_HD void sincos_ad(double a, double& s, double& c) { sincos(a, &s, &c); }
PTN_HD void sincos_ad(float a, float& s, float& c) { sincosf(a, &s, &c); }
template <class S, int K>
PTN_HD Dual<S, K> operator/(double c, const Dual<S, K>& a) {
  return recip(a) * Dual<S, K>(S(c));
}
PTN_HD double recip(double a) { return 1.0 / a; }
PTN_HD float recip(float a) { return 1.0f / a; }

// base scalar of an AD type, and products/sums with a double constant
template <class S> struct base_of { using type = S; };
template <class S, int K> struct base_of<Dual<S, K>> { using type = S; };
template <class S, int K> struct base_of<Jet<S, K>> { using type = S; };
template <class S>
PTN_HD S cmul(double c, const S& a) {
  using B = typename base_of<S>::type;
  return B(c) * a;
}
template <class S>
PTN_HD S cadd(double c, const S& a) {
  using B = typename base_of<S>::type;
  return B(c) + a;
}
// model constants may themselves be AD scalars (parameter derivatives): a constant of
// the base type, or of the same type, times a value
template <class B, int K1, int K2>
PTN_HD Dual<Dual<B, K1>, K2> cmul(const Dual<B, K1>& c, const Dual<Dual<B, K1>, K2>& a) { return c * a; }
template <class S, int K>
PTN_HD Dual<S, K> cmul(const Dual<S, K>& c, const Dual<S, K>& a) { return c * a; }
template <class B, int K1, int K2>
PTN_HD Dual<Dual<B, K1>, K2> cadd(const Dual<B, K1>& c, const Dual<Dual<B, K1>, K2>& a) { return c + a; }
template <class S, int K>
PTN_HD Dual<S, K> cadd(const Dual<S, K>& c, const Dual<S, K>& a) { return c + a; }

// model constants converted once to the evaluation's base scalar (float constants in the
// FP32 path, so no FP64 arithmetic runs inside the model), or kept as AD scalars when
// parameter derivatives are taken
template <class S>
PTN_HD typename base_of<S>::type pconv(double c) {
  return typename base_of<S>::type(c);
}
template <class S, class B, int K>
PTN_HD Dual<B, K> pconv(const Dual<B, K>& c) {
  return c;
}

template <class S>
PTN_HD S cst(double c) {
  using B = typename base_of<S>::type;
  return S(B(c));
}

}  // namespace ptn
