// Host build of the kernels' model code (ptn_models.cuh is __host__ __device__): for each
// line of input "model integ dt p0..p7 x.. u.. lam.." it prints the step x+ = f(x, u), its
// Jacobians F, G (forward-mode Dual numbers) and the lam-contracted second derivatives
// Hxx, Hxu, Huu (Jet numbers), and the adjoint's parameter derivatives df/dprm and
// d2(lam . f)/dz dprm (nested Dual numbers) -- the same templates the solver kernels
// instantiate -- so that a test can compare them with the oracle's models without a GPU.
#include <cstdio>

#include "ptn_models.cuh"

using namespace ptn;

template <class M>
static void eval(int integ, double dt, const double* p, const double* x, const double* u, const double* lam) {
  constexpr int N = M::NX, U = M::NU;
  double xn[N], F[N * N], G[N * U], Hxx[N * N], Hxu[N * U], Huu[U * U];
  step_jac<M, double>(integ, dt, p, x, u, xn, F, G);
  step_hess<M, double>(integ, dt, p, x, u, lam, Hxx, Hxu, Huu);
  for (double v : xn) printf("%.17g ", v);
  for (double v : F) printf("%.17g ", v);
  for (double v : G) printf("%.17g ", v);
  for (double v : Hxx) printf("%.17g ", v);
  for (double v : Hxu) printf("%.17g ", v);
  for (double v : Huu) printf("%.17g ", v);
  double fp[N * M::NP], Hzp[(N + U) * M::NP];
  step_param_derivs<M>(integ, dt, p, x, u, lam, fp, Hzp);
  for (double v : fp) printf("%.17g ", v);
  for (double v : Hzp) printf("%.17g ", v);
  // increment f - x in FP64 and FP32 (the mixed rollouts' form)
  double d64[N];
  float xf[N], uf[U], d32[N];
  step_inc<M, double>(integ, dt, p, x, u, d64);
  for (int i = 0; i < N; i++) xf[i] = float(x[i]);
  for (int i = 0; i < U; i++) uf[i] = float(u[i]);
  step_inc<M, float>(integ, dt, p, xf, uf, d32);
  for (double v : d64) printf("%.17g ", v);
  for (float v : d32) printf("%.9g ", double(v));
  // closed-loop Jacobian F + G Gam with Gam = lam[0..U) in every row (a fixed test gain)
  double Gam[U * N], Fcl[N * N];
  for (int i = 0; i < U; i++)
    for (int j = 0; j < N; j++) Gam[i * N + j] = 0.1 * lam[j] / double(i + 1);
  step_cl_jac<M, double>(integ, dt, p, x, u, Gam, Fcl);
  for (double v : Fcl) printf("%.17g ", v);
  printf("\n");
}

int main() {
  int model, integ;
  double dt;
  while (scanf("%d %d %lf", &model, &integ, &dt) == 3) {
    double p[8], x[12], u[4], lam[12];
    int n = model == MODEL_PENDULUM ? 2 : model == MODEL_CARTPOLE ? 4 : 12;
    int m = model == MODEL_QUADROTOR ? 4 : 1;
    for (double& v : p) if (scanf("%lf", &v) != 1) return 1;
    for (int i = 0; i < n; i++) if (scanf("%lf", &x[i]) != 1) return 1;
    for (int i = 0; i < m; i++) if (scanf("%lf", &u[i]) != 1) return 1;
    for (int i = 0; i < n; i++) if (scanf("%lf", &lam[i]) != 1) return 1;
    if (model == MODEL_PENDULUM) eval<Pendulum>(integ, dt, p, x, u, lam);
    else if (model == MODEL_CARTPOLE) eval<CartPole>(integ, dt, p, x, u, lam);
    else if (model == MODEL_QUADROTOR) eval<Quadrotor>(integ, dt, p, x, u, lam);
    else return 2;
    fflush(stdout);
  }
  return 0;
}
