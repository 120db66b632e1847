// Host build of the synthetic map's closed-form terms (ptn_synth.cuh).  Input lines:
// "n m c A(n*n) B(n*m) W(n*n) x(n) u(m) lam(n)" for (n, m) = (32, 8) or (6, 2); output:
// x+ F G Hxx.
#include <cstdio>

#include "ptn_synth.cuh"

using namespace ptn;

template <int N, int U>
static int run(double c) {
  static double A[N * N], B[N * U], W[N * N], x[N], u[U], lam[N];
  for (double& v : A) if (scanf("%lf", &v) != 1) return 1;
  for (double& v : B) if (scanf("%lf", &v) != 1) return 1;
  for (double& v : W) if (scanf("%lf", &v) != 1) return 1;
  for (double& v : x) if (scanf("%lf", &v) != 1) return 1;
  for (double& v : u) if (scanf("%lf", &v) != 1) return 1;
  for (double& v : lam) if (scanf("%lf", &v) != 1) return 1;
  static double xn[N], F[N * N], G[N * U], H[N * N];
  SynthMap<N, U>::step(A, B, W, c, x, u, xn);
  SynthMap<N, U>::template jac<double>(A, B, W, c, x, F, G);
  SynthMap<N, U>::template hess_xx<double>(W, c, x, lam, H);
  for (double v : xn) printf("%.17g ", v);
  for (double v : F) printf("%.17g ", v);
  for (double v : G) printf("%.17g ", v);
  for (double v : H) printf("%.17g ", v);
  printf("\n");
  fflush(stdout);
  return 0;
}

int main() {
  int n, m;
  double c;
  while (scanf("%d %d %lf", &n, &m, &c) == 3) {
    int rc = (n == 32 && m == 8) ? run<32, 8>(c) : (n == 6 && m == 2) ? run<6, 2>(c) : 2;
    if (rc) return rc;
  }
  return 0;
}
