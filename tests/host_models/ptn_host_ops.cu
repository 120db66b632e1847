// Host build of the kernels' scan operators and value-element initialisation
// (ptn_ops.cuh is __host__ __device__), for comparison with the oracle's own operators
// without a GPU.  Each input line is "<op> <lqr precision> numbers..." with op one of
//   V  value combine (Alg. 2):   e1 then e2, each A(16) b(4) C(16) eta(4) J(16)
//   I  value element init:       F(16) G(4) P(16) M(4) R(1) d(1) alpha
//   C  co-state combine (Alg. 1): g1(4) Ft1(16) g2(4) Ft2(16)
//   S  state combine (Alg. 3):    F1(16) e1(4) F2(16) e2(4)
//   R  Riccati step with feedback: F(16) G(4) P(16) M(4) R(1) d(1) alpha S(16) s(4)
//      -> Gam(4) gam(1) S_t(16) s_t(4)
//   W  step folded into a later element (Woodbury form of the value combination):
//      F(16) G(4) P(16) M(4) R(1) d(1) alpha e(56: A b C eta J) -> the combined element
//   K  pivot keys: x -> mag_key(double x) mag_key(float x)
//   G  FP64 Gauss-Jordan inverse with partial pivoting: A(16) -> A^{-1}(16)
//   L  LDL^T factorisation and solve: A(16, symmetric) B(4 x 3) -> X = A^{-1} B (12)
//   D  co-state combine on FP32 increments (mixed mode): ga(4) Da(16) gb(4) Db(16)
//      -> g(4) D(16), the elements being (g, I + D)
// for n = 4, m = 1, and LQR precision 0 (FP64) or 1 (FP32 data, FP64 solves); the output
// line is the resulting element (value elements as A b C eta J).
#include <cstdio>
#include <cstring>

#include "ptn_solver.cuh"

using namespace ptn;
constexpr int N = 4, U = 1;

static bool rd(double* v, int n) {
  for (int i = 0; i < n; i++)
    if (scanf("%lf", &v[i]) != 1) return false;
  return true;
}
static void pr(const double* v, int n) {
  for (int i = 0; i < n; i++) printf("%.17g ", v[i]);
}

template <class L>
static void put_val(const double* in, Val<N, L>& e) {
  for (int i = 0; i < 16; i++) e.A[i] = L(in[i]);
  for (int i = 0; i < 4; i++) e.b[i] = L(in[16 + i]);
  for (int i = 0; i < 16; i++) e.C[i] = L(in[20 + i]);
  for (int i = 0; i < 4; i++) e.eta[i] = L(in[36 + i]);
  for (int i = 0; i < 16; i++) e.J[i] = L(in[40 + i]);
}
template <class L>
static void print_val(const Val<N, L>& e) {
  double o[56];
  for (int i = 0; i < 16; i++) o[i] = double(e.A[i]);
  for (int i = 0; i < 4; i++) o[16 + i] = double(e.b[i]);
  for (int i = 0; i < 16; i++) o[20 + i] = double(e.C[i]);
  for (int i = 0; i < 4; i++) o[36 + i] = double(e.eta[i]);
  for (int i = 0; i < 16; i++) o[40 + i] = double(e.J[i]);
  pr(o, 56);
}

template <class L>
static bool value_combine(const double* in) {
  Val<N, L> a, b, o;
  put_val(in, a);
  put_val(in + 56, b);
  if (!ValueOp<double>()(a, b, o)) return false;
  print_val(o);
  return true;
}

template <class L>
static bool value_init_op(const double* in) {
  L F[16], G[4], P[16], M[4], R[1];
  for (int i = 0; i < 16; i++) { F[i] = L(in[i]); P[i] = L(in[20 + i]); }
  for (int i = 0; i < 4; i++) { G[i] = L(in[16 + i]); M[i] = L(in[36 + i]); }
  R[0] = L(in[40]);
  const double d[1] = {in[41]};
  Val<N, L> e;
  if (!value_init<N, U, L, double>(F, G, P, M, R, d, in[42], e)) return false;
  print_val(e);
  return true;
}

template <class L>
static bool value_fold_op(const double* in) {
  L F[16], G[4], P[16], M[4], R[1];
  for (int i = 0; i < 16; i++) { F[i] = L(in[i]); P[i] = L(in[20 + i]); }
  for (int i = 0; i < 4; i++) { G[i] = L(in[16 + i]); M[i] = L(in[36 + i]); }
  R[0] = L(in[40]);
  const double d[1] = {in[41]};
  Val<N, L> e;
  put_val(in + 43, e);
  if (!value_fold_step<N, U, L, double>(F, G, P, M, R, d, in[42], e)) return false;
  print_val(e);
  return true;
}

template <class L>
static bool riccati_op(const double* in) {
  L F[16], G[4], P[16], M[4], R[1], S[16], sv[4], Gam[4], gam[1];
  for (int i = 0; i < 16; i++) { F[i] = L(in[i]); P[i] = L(in[20 + i]); S[i] = L(in[43 + i]); }
  for (int i = 0; i < 4; i++) { G[i] = L(in[16 + i]); M[i] = L(in[36 + i]); sv[i] = L(in[59 + i]); }
  R[0] = L(in[40]);
  const double d[1] = {in[41]};
  if (!riccati_step<N, U, L, double>(F, G, P, M, R, d, in[42], S, sv, Gam, gam)) return false;
  double o[25];
  for (int i = 0; i < 4; i++) o[i] = double(Gam[i]);
  o[4] = double(gam[0]);
  for (int i = 0; i < 16; i++) o[5 + i] = double(S[i]);
  for (int i = 0; i < 4; i++) o[21 + i] = double(sv[i]);
  pr(o, 25);
  return true;
}

int main() {
  char op[4];
  int prec;
  while (scanf("%3s %d", op, &prec) == 2) {
    double in[112];
    bool ok = true;
    if (op[0] == 'V') {
      if (!rd(in, 112)) return 1;
      ok = prec ? value_combine<float>(in) : value_combine<double>(in);
    } else if (op[0] == 'I') {
      if (!rd(in, 43)) return 1;
      ok = prec ? value_init_op<float>(in) : value_init_op<double>(in);
    } else if (op[0] == 'W') {
      if (!rd(in, 99)) return 1;
      ok = prec ? value_fold_op<float>(in) : value_fold_op<double>(in);
    } else if (op[0] == 'R') {
      if (!rd(in, 63)) return 1;
      ok = prec ? riccati_op<float>(in) : riccati_op<double>(in);
    } else if (op[0] == 'K') {
      if (!rd(in, 1)) return 1;
      printf("%u %u", mag_key(in[0]), mag_key(float(in[0])));
    } else if (op[0] == 'D') {
      if (!rd(in, 40)) return 1;
      IncAff<N> a, b, o;
      for (int i = 0; i < 4; i++) { a.g[i] = in[i]; b.g[i] = in[20 + i]; }
      for (int i = 0; i < 16; i++) { a.D[i] = float(in[4 + i]); b.D[i] = float(in[24 + i]); }
      IncCostateOp()(a, b, o);
      pr(o.g, 4);
      for (int i = 0; i < 16; i++) printf("%.9g ", double(o.D[i]));
    } else if (op[0] == 'L') {
      if (!rd(in, 28)) return 1;
      ok = ldlt<N, double>(in);
      if (ok) {
        ldlt_solve<N, 3, double>(in, in + 16);
        pr(in + 16, 12);
      }
    } else if (op[0] == 'G') {
      if (!rd(in, 16)) return 1;
      ok = inv_gj<N, double>(in);
      if (ok) pr(in, 16);
    } else if (op[0] == 'C' || op[0] == 'S') {
      if (!rd(in, 40)) return 1;
      Aff<N, double> a, b, o;
      if (op[0] == 'C') {
        for (int i = 0; i < 4; i++) { a.v[i] = in[i]; b.v[i] = in[20 + i]; }
        for (int i = 0; i < 16; i++) { a.M[i] = in[4 + i]; b.M[i] = in[24 + i]; }
        CostateOp()(a, b, o);
      } else {
        for (int i = 0; i < 16; i++) { a.M[i] = in[i]; b.M[i] = in[20 + i]; }
        for (int i = 0; i < 4; i++) { a.v[i] = in[16 + i]; b.v[i] = in[36 + i]; }
        StateOp()(a, b, o);
      }
      pr(o.v, 4);
      pr(o.M, 16);
    } else {
      return 2;
    }
    if (!ok) printf("FAIL");
    printf("\n");
    fflush(stdout);
  }
  return 0;
}
