// ptn_wops.cuh -- warp-cooperative dense linear algebra and AD for state dimensions
// n >= 8, where one scan element no longer fits a thread's registers.  A matrix lives in
// shared memory (row-major); the 32 lanes of a warp split its entries.  Every routine
// ends with __syncwarp(), so its results are visible to the whole warp.  Operands of
// one call must not alias its output unless stated.
//
// These are the element operations of the three scans of Sec. III (Alg. 1-3), the value
// element initialisation and the feedback step, written for a warp instead of a thread.
#pragma once
#include "ptn_models.cuh"
#include "ptn_ops.cuh"

namespace ptn {
namespace wops {

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// sum over k < K of term(k), in four independent partial sums: with one warp per SM
// sub-partition nothing else hides the latency of a dependent chain of multiply-adds, so
// each lane keeps four of them in flight
template <int K, class S, class Term>
__device__ __forceinline__ S dot4(const Term& term) {
  S s0 = S(0), s1 = S(0), s2 = S(0), s3 = S(0);
#pragma unroll
  for (int k = 0; k + 3 < K; k += 4) {
    s0 += term(k);
    s1 += term(k + 1);
    s2 += term(k + 2);
    s3 += term(k + 3);
  }
#pragma unroll
  for (int k = K & ~3; k < K; k++) s0 += term(k);
  return (s0 + s1) + (s2 + s3);
}

// ---- FP32 products on the tensor cores (mma.sync m16n8k8, TF32 operands) ----
//
// A float x is split into hi = tf32(x) and lo = tf32(x - hi) (x - hi is exact in FP32);
// a product x y is taken as lo_x hi_y + hi_x lo_y + hi_x hi_y with FP32 accumulation in
// the MMA.  The dropped lo_x lo_y term and the rounding of lo are below 2^-21 of |x y|,
// so the result carries about FP32 accuracy (three MMAs per tile instead of one).
__device__ __forceinline__ unsigned tf32_rna(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split_tf32(float x, unsigned& hi, unsigned& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - __uint_as_float(hi));
}
// d += a b for one 16 x 8 tile of d, a 16 x 8 (row-major fragment), b 8 x 8 (column)
__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C (R x Cc) = op(A) (R x K) * op(B) (K x Cc) [+ C if ACC], all FP32 in shared memory, on
// the tensor cores: the output in 16 x 8 tiles held in registers, K in steps of 8, entries
// outside the matrices read as zero.  Fragment layout (PTX ISA, mma.m16n8k8 .tf32), with
// g = lane / 4 and c = lane % 4: a = {(g, c), (g + 8, c), (g, c + 4), (g + 8, c + 4)},
// b = {(c, g), (c + 4, g)}, d = {(g, 2c), (g, 2c + 1), (g + 8, 2c), (g + 8, 2c + 1)}.
template <int R, int K, int Cc, bool TA, bool TB, bool ACC>
__device__ void mm_tc(const float* A, const float* B, float* C) {
  constexpr int MT = (R + 15) / 16, NT = (Cc + 7) / 8, KT = (K + 7) / 8;
  const int l = lane_id(), g = l >> 2, c = l & 3;
  auto a_at = [&](int i, int k) -> float {
    return (i < R && k < K) ? (TA ? A[k * R + i] : A[i * K + k]) : 0.0f;
  };
  auto b_at = [&](int k, int j) -> float {
    return (k < K && j < Cc) ? (TB ? B[j * K + k] : B[k * Cc + j]) : 0.0f;
  };
  float acc[MT][NT][4];
#pragma unroll
  for (int mt = 0; mt < MT; mt++)
#pragma unroll
    for (int nt = 0; nt < NT; nt++)
#pragma unroll
      for (int q = 0; q < 4; q++) acc[mt][nt][q] = 0.0f;
#pragma unroll
  for (int kt = 0; kt < KT; kt++) {
    const int k0 = kt * 8 + c;
    unsigned ah[MT][4], al[MT][4], bh[NT][2], bl[NT][2];
#pragma unroll
    for (int mt = 0; mt < MT; mt++) {
      const int r0 = mt * 16 + g;
      split_tf32(a_at(r0, k0), ah[mt][0], al[mt][0]);
      split_tf32(a_at(r0 + 8, k0), ah[mt][1], al[mt][1]);
      split_tf32(a_at(r0, k0 + 4), ah[mt][2], al[mt][2]);
      split_tf32(a_at(r0 + 8, k0 + 4), ah[mt][3], al[mt][3]);
    }
#pragma unroll
    for (int nt = 0; nt < NT; nt++) {
      const int j = nt * 8 + g;
      split_tf32(b_at(k0, j), bh[nt][0], bl[nt][0]);
      split_tf32(b_at(k0 + 4, j), bh[nt][1], bl[nt][1]);
    }
#pragma unroll
    for (int mt = 0; mt < MT; mt++)
#pragma unroll
      for (int nt = 0; nt < NT; nt++) {
        mma_tf32(acc[mt][nt], al[mt], bh[nt]);
        mma_tf32(acc[mt][nt], ah[mt], bl[nt]);
        mma_tf32(acc[mt][nt], ah[mt], bh[nt]);
      }
  }
  __syncwarp();  // every lane's operand loads precede the first store
#pragma unroll
  for (int mt = 0; mt < MT; mt++)
#pragma unroll
    for (int nt = 0; nt < NT; nt++)
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const int i = mt * 16 + g + ((q & 2) ? 8 : 0), j = nt * 8 + 2 * c + (q & 1);
        if (i < R && j < Cc) C[i * Cc + j] = ACC ? C[i * Cc + j] + acc[mt][nt][q] : acc[mt][nt][q];
      }
  __syncwarp();
}

// C (R x Cc) = op(A) (R x K) * op(B) (K x Cc) [+ C if ACC]; op = transpose when TA / TB.
// Accumulation in the type of C.  All-FP32 products of at least 8 x 8 x 8 run on the
// tensor cores (mm_tc); the others (FP64, mixed, or thin) are lane-parallel dot products.
template <int R, int K, int Cc, bool TA, bool TB, bool ACC = false, class SA, class SB, class SC>
__device__ void mm(const SA* A, const SB* B, SC* C) {
  if constexpr (std::is_same<SA, float>::value && std::is_same<SB, float>::value &&
                std::is_same<SC, float>::value && R >= 8 && K >= 8 && Cc >= 8) {
    mm_tc<R, K, Cc, TA, TB, ACC>(A, B, C);
  } else {
    for (int e = lane_id(); e < R * Cc; e += 32) {
      const int i = e / Cc, j = e % Cc;
      const SC s = dot4<K, SC>([&](int k) {
        return SC(TA ? A[k * R + i] : A[i * K + k]) * SC(TB ? B[j * K + k] : B[k * Cc + j]);
      });
      C[e] = ACC ? C[e] + s : s;
    }
    __syncwarp();
  }
}

// y (R) = op(A) x [+ y]
template <int R, int K, bool TA, bool ACC = false, class SA, class SX, class SY>
__device__ void mv(const SA* A, const SX* x, SY* y) {
  for (int i = lane_id(); i < R; i += 32) {
    const SY s = dot4<K, SY>([&](int k) { return SY(TA ? A[k * R + i] : A[i * K + k]) * SY(x[k]); });
    y[i] = ACC ? y[i] + s : s;
  }
  __syncwarp();
}

template <int Nn, class S, class D>
__device__ void copy(const S* a, D* b) {
  for (int e = lane_id(); e < Nn; e += 32) b[e] = D(a[e]);
  __syncwarp();
}

template <int N, class S>
__device__ void symmetrize(S* X) {
  for (int e = lane_id(); e < N * N; e += 32) {
    const int i = e / N, j = e % N;
    if (i < j) {
      const S v = S(0.5) * (X[i * N + j] + X[j * N + i]);
      X[i * N + j] = v;
      X[j * N + i] = v;
    }
  }
  __syncwarp();
}

// lane with the largest key (ties: smallest index) among lanes whose key is valid
__device__ __forceinline__ int warp_argmax(unsigned key, bool valid) {
  unsigned k = valid ? key : 0u;
  int idx = valid ? lane_id() : 0x7fffffff;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned ok = __shfl_xor_sync(0xffffffffu, k, off);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, off);
    if (ok > k || (ok == k && oi < idx)) { k = ok; idx = oi; }
  }
  return idx;
}

// In-place inverse of an N x N matrix (N <= 32) by Gauss-Jordan elimination with partial
// pivoting, in scalar S.  piv: N ints of shared scratch, col: N values of shared scratch.
// Returns false (warp-uniform) when a pivot is zero or not finite.
template <int N, class S>
__device__ bool inv(S* A, int* piv, S* col) {
  static_assert(N <= 32, "pivot search spans one warp");
  const int l = lane_id();
  if (l < N) piv[l] = l;
  __syncwarp();
  for (int k = 0; k < N; k++) {
    const bool in = (l >= k && l < N);
    const unsigned key = in ? mag_key(A[l * N + k]) : 0u;
    const int p = warp_argmax(key, in);
    if (p != k) {
      for (int j = l; j < N; j += 32) {
        const S t = A[k * N + j];
        A[k * N + j] = A[p * N + j];
        A[p * N + j] = t;
      }
      if (l == 0) { const int t = piv[k]; piv[k] = piv[p]; piv[p] = t; }
    }
    __syncwarp();
    const S pv = A[k * N + k];
    if (!(pv != S(0)) || !isfinite(pv)) return false;
    const S ip = S(1) / pv;
    // column k multipliers, then the pivot row scaled, then the elimination
    if (l < N) col[l] = (l == k) ? S(0) : A[l * N + k];
    __syncwarp();
    for (int j = l; j < N; j += 32) A[k * N + j] = (j == k) ? ip : A[k * N + j] * ip;
    __syncwarp();
    for (int e = l; e < N * N; e += 32) {
      const int i = e / N, j = e % N;
      if (i == k) continue;
      const S f = col[i];
      A[e] = (j == k) ? -f * ip : A[e] - f * A[k * N + j];
    }
    __syncwarp();
  }
  // undo the row permutation as a column permutation of the inverse
  for (int i = 0; i < N; i++) {
    S v = S(0);
    if (l < N) v = A[i * N + l];
    __syncwarp();
    if (l < N) A[i * N + piv[l]] = v;
    __syncwarp();
  }
  return true;
}

// LDL^T of a U x U symmetric positive definite matrix held by every lane (registers);
// reciprocal pivots on the diagonal.  Same as ptn::ldlt, executed redundantly.
template <int U, class S>
__device__ __forceinline__ bool ldlt_regs(S* A) {
  return ldlt<U, S>(A);
}

// solve (L D L^T) X = B for the C columns of B (U x C, shared, row-major) in place; lane
// c handles column c.  F: the factor of ldlt_regs, in registers.
template <int U, int C, class S, class SB>
__device__ void ldlt_solve_cols(const S* F, SB* B) {
  for (int c = lane_id(); c < C; c += 32) {
    S y[U];
#pragma unroll
    for (int i = 0; i < U; i++) {
      S s = S(B[i * C + c]);
#pragma unroll
      for (int k = 0; k < i; k++) s -= F[i * U + k] * y[k];
      y[i] = s;
    }
#pragma unroll
    for (int i = 0; i < U; i++) y[i] *= F[i * U + i];
#pragma unroll
    for (int i = U - 1; i >= 0; i--) {
      S s = y[i];
#pragma unroll
      for (int k = i + 1; k < U; k++) s -= F[k * U + i] * y[k];
      y[i] = s;
    }
#pragma unroll
    for (int i = 0; i < U; i++) B[i * C + c] = SB(y[i]);
  }
  __syncwarp();
}

// warp sum / max of a per-lane value (result in every lane)
template <class S>
__device__ __forceinline__ S wsum(S v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
template <class S>
__device__ __forceinline__ S wmax(S v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}

// ---------------------------------------------------------------------------
// Forward-mode AD across lanes.
//
// Jacobian of the step map f(x, u) (Euler or RK4): lane j < N + U propagates one dual
// number seeded on z_j = (x, u)_j and writes column j: F (N x N) and G (N x U), in
// scalar S.  fx (N, may be null): f itself, from lane 0.
template <class M, class S>
__device__ void step_jac(int integ, double dt, const double* p, const double* x, const double* u, S* F, S* G,
                         double* fx = nullptr) {
  constexpr int N = M::NX, U = M::NU, K = N + U;
  using D = Dual<S, 1>;
  for (int j = lane_id(); j < K; j += 32) {
    D xd[N], ud[U], xn[N];
#pragma unroll
    for (int i = 0; i < N; i++) { xd[i] = D(S(x[i])); xd[i].d[0] = (i == j) ? S(1) : S(0); }
#pragma unroll
    for (int i = 0; i < U; i++) { ud[i] = D(S(u[i])); ud[i].d[0] = (N + i == j) ? S(1) : S(0); }
    step<M, D, double>(integ, dt, p, xd, ud, xn);
#pragma unroll
    for (int i = 0; i < N; i++) {
      if (j < N) F[i * N + j] = xn[i].d[0];
      else G[i * U + (j - N)] = xn[i].d[0];
    }
    if (fx && j == 0) {
#pragma unroll
      for (int i = 0; i < N; i++) fx[i] = double(xn[i].v);
    }
  }
  __syncwarp();
}

// Jacobian of the increment f(x, u) - x in scalar S (E = F - I, G), evaluated at the
// point rounded to S, as the FP32 rollouts use it; dv (N, may be null): the increment.
template <class M, class S>
__device__ void inc_jac(int integ, double dt, const double* p, const double* x, const double* u, S* E, S* G,
                        S* dv = nullptr) {
  constexpr int N = M::NX, U = M::NU, K = N + U;
  using D = Dual<S, 1>;
  for (int j = lane_id(); j < K; j += 32) {
    D xd[N], ud[U], dd[N];
#pragma unroll
    for (int i = 0; i < N; i++) { xd[i] = D(S(x[i])); xd[i].d[0] = (i == j) ? S(1) : S(0); }
#pragma unroll
    for (int i = 0; i < U; i++) { ud[i] = D(S(u[i])); ud[i].d[0] = (N + i == j) ? S(1) : S(0); }
    step_inc<M, D, double>(integ, dt, p, xd, ud, dd);
#pragma unroll
    for (int i = 0; i < N; i++) {
      if (j < N) E[i * N + j] = dd[i].d[0];
      else G[i * U + (j - N)] = dd[i].d[0];
    }
    if (dv && j == 0) {
#pragma unroll
      for (int i = 0; i < N; i++) dv[i] = dd[i].v;
    }
  }
  __syncwarp();
}

// lam-contracted second derivatives of the step map, H = sum_i lam_i d2 f_i / dz dz
// (z = (x, u), K = N + U), written as Hxx (N x N), Hxu (N x U), Huu (U x U) in scalar S.
// Lane-parallel over the K (K + 1) / 2 entries of the upper triangle, each from one
// hyper-dual evaluation (nested dual numbers seeded on z_a and z_b).
template <class M, class S>
__device__ void step_hess(int integ, double dt, const double* p, const double* x, const double* u,
                          const double* lam, S* Hxx, S* Hxu, S* Huu) {
  constexpr int N = M::NX, U = M::NU, K = N + U, NPAIR = K * (K + 1) / 2;
  using D1 = Dual<S, 1>;
  using D2 = Dual<D1, 1>;
  for (int q = lane_id(); q < NPAIR; q += 32) {
    // q -> (a, b), a <= b, row-major over the upper triangle
    int a = 0, rem = q;
    while (rem >= K - a) { rem -= K - a; a++; }
    const int b = a + rem;
    D2 xd[N], ud[U], xn[N];
#pragma unroll
    for (int i = 0; i < N; i++) {
      xd[i] = D2(D1(S(x[i])));
      xd[i].v.d[0] = (i == a) ? S(1) : S(0);
      xd[i].d[0] = D1((i == b) ? S(1) : S(0));
    }
#pragma unroll
    for (int i = 0; i < U; i++) {
      ud[i] = D2(D1(S(u[i])));
      ud[i].v.d[0] = (N + i == a) ? S(1) : S(0);
      ud[i].d[0] = D1((N + i == b) ? S(1) : S(0));
    }
    step<M, D2, double>(integ, dt, p, xd, ud, xn);
    S h = S(0);
#pragma unroll
    for (int i = 0; i < N; i++) h += S(lam[i]) * xn[i].d[0].d[0];
    auto put = [&](int r, int c, S v) {
      if (r < N && c < N) Hxx[r * N + c] = v;
      else if (r < N) Hxu[r * U + (c - N)] = v;
      else if (c >= N) Huu[(r - N) * U + (c - N)] = v;
    };
    put(a, b, h);
    if (a != b) put(b, a, h);
  }
  __syncwarp();
}

}  // namespace wops
}  // namespace ptn
