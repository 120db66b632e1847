// ptn_models.cuh -- dynamics of the paper's examples (Sec. IV) and the benchmark
// workloads, written once as templates over the scalar type so that plain values,
// Jacobians (Dual) and second-order contractions (Jet) come from the same code.
//
//   pendulum  (Sec. IV-A): theta'' = -(g/l) sin(theta) - b/(m l^2) theta' + u/(m l^2)
//   cart-pole (Sec. IV-B): Tedrake's equations with the l*theta'^2 term in p''
//   quadrotor: 12-state rigid body, ZYX Euler angles, '+' rotor layout
//   synthetic: x+ = A x + B u + c tanh(W x)
#pragma once
#include "ptn_common.cuh"

namespace ptn {

enum : int { MODEL_PENDULUM = 0, MODEL_CARTPOLE = 1, MODEL_QUADROTOR = 2, MODEL_SYNTH = 3 };
enum : int { INTEG_EULER = 0, INTEG_RK4 = 1 };

// prm = [g, l, m, b]; x = (theta, omega)
struct Pendulum {
  static constexpr int NX = 2, NU = 1, NP = 4, ID = MODEL_PENDULUM;
  template <class S, class PT>
  PTN_HD static void rhs(const PT* p, const S* x, const S* u, S* xd) {
    const auto g = pconv<S>(p[0]), l = pconv<S>(p[1]), m = pconv<S>(p[2]), b = pconv<S>(p[3]);
    const auto iml2 = decltype(g)(1) / (m * l * l);
    S s, c;
    sincos_ad(x[0], s, c);
    xd[0] = x[1];
    xd[1] = cmul(-g / l, s) + cmul(-b * iml2, x[1]) + cmul(iml2, u[0]);
  }
};

// prm = [m_c, m_p, l, g]; x = (p, theta, p', theta'), theta = 0 hanging down
struct CartPole {
  static constexpr int NX = 4, NU = 1, NP = 4, ID = MODEL_CARTPOLE;
  template <class S, class PT>
  PTN_HD static void rhs(const PT* p, const S* x, const S* u, S* xd) {
    const auto mc = pconv<S>(p[0]), mp = pconv<S>(p[1]), l = pconv<S>(p[2]), g = pconv<S>(p[3]);
    S s, c;
    sincos_ad(x[1], s, c);
    const S td2 = x[3] * x[3];
    const S den = cadd(mc, cmul(mp, s * s));
    const S iden = recip(den);
    const S pdd = (u[0] + cmul(mp, s) * (cmul(l, td2) + cmul(g, c))) * iden;
    const S num = -(u[0] * c) - cmul(mp * l, td2 * c * s) - cmul((mc + mp) * g, s);
    const S tdd = cmul(decltype(l)(1) / l, num * iden);
    (void)g;
    xd[0] = x[2];
    xd[1] = x[3];
    xd[2] = pdd;
    xd[3] = tdd;
  }
};

// prm = [mass, Ixx, Iyy, Izz, arm, k_m, g];
// x = (px,py,pz, roll,pitch,yaw, vx,vy,vz, wx,wy,wz); u = rotor thrusts 1..4
// rotor 1 on +x, 2 on +y, 3 on -x, 4 on -y; yaw torque k_m (f1 - f2 + f3 - f4)
struct Quadrotor {
  static constexpr int NX = 12, NU = 4, NP = 7, ID = MODEL_QUADROTOR;
  template <class S, class PT>
  PTN_HD static void rhs(const PT* p, const S* x, const S* u, S* xd) {
    const auto mass = pconv<S>(p[0]), Ixx = pconv<S>(p[1]), Iyy = pconv<S>(p[2]), Izz = pconv<S>(p[3]);
    const auto arm = pconv<S>(p[4]), km = pconv<S>(p[5]), g = pconv<S>(p[6]);
    using PC = decltype(g);
    S sph, cph, sth, cth, sps, cps;
    sincos_ad(x[3], sph, cph);
    sincos_ad(x[4], sth, cth);
    sincos_ad(x[5], sps, cps);
    const S icth = recip(cth);
    const S tth = sth * icth;
    const S fsum = (u[0] + u[1]) + (u[2] + u[3]);
    const S am = cmul(PC(1) / mass, fsum);
    // body z axis in the world frame (third column of Rz Ry Rx)
    const S r13 = cps * (sth * cph) + sps * sph;
    const S r23 = sps * (sth * cph) - cps * sph;
    const S r33 = cth * cph;
    xd[0] = x[6];
    xd[1] = x[7];
    xd[2] = x[8];
    xd[3] = x[9] + (sph * tth) * x[10] + (cph * tth) * x[11];
    xd[4] = cph * x[10] - sph * x[11];
    xd[5] = (sph * x[10] + cph * x[11]) * icth;
    xd[6] = am * r13;
    xd[7] = am * r23;
    xd[8] = cadd(-g, am * r33);
    (void)mass;
    const S tx = cmul(arm, u[1] - u[3]);
    const S ty = cmul(arm, u[2] - u[0]);
    const S tz = cmul(km, (u[0] + u[2]) - (u[1] + u[3]));
    xd[9] = cmul(PC(1) / Ixx, tx - cmul(Izz - Iyy, x[10] * x[11]));
    xd[10] = cmul(PC(1) / Iyy, ty - cmul(Ixx - Izz, x[11] * x[9]));
    xd[11] = cmul(PC(1) / Izz, tz - cmul(Iyy - Ixx, x[9] * x[10]));
  }
};

// Increment of one discrete step, dx = f(x, u) - x, in scalar S (no identity added, so
// FP32 keeps the relative precision of the small increment).
template <class M, class S, class PT = double>
PTN_HD void step_inc(int integ, double dt, const PT* p, const S* x, const S* u, S* dxo) {
  constexpr int N = M::NX;
  using B = typename base_of<S>::type;
  const B h = B(dt), h2 = h * B(0.5), h6 = h / B(6), two = B(2);
  S k[N];
  M::rhs(p, x, u, k);
  if (integ == INTEG_EULER) {
#pragma unroll
    for (int i = 0; i < N; i++) dxo[i] = h * k[i];
    return;
  }
  S acc[N], y[N];
#pragma unroll
  for (int i = 0; i < N; i++) { acc[i] = k[i]; y[i] = x[i] + h2 * k[i]; }
  M::rhs(p, y, u, k);
#pragma unroll
  for (int i = 0; i < N; i++) { acc[i] = acc[i] + two * k[i]; y[i] = x[i] + h2 * k[i]; }
  M::rhs(p, y, u, k);
#pragma unroll
  for (int i = 0; i < N; i++) { acc[i] = acc[i] + two * k[i]; y[i] = x[i] + h * k[i]; }
  M::rhs(p, y, u, k);
#pragma unroll
  for (int i = 0; i < N; i++) dxo[i] = h6 * (acc[i] + k[i]);
}

// One discrete step x+ = f(x, u): explicit Euler or classical RK4 with the control
// held over the step.
template <class M, class S, class PT = double>
PTN_HD void step(int integ, double dt, const PT* p, const S* x, const S* u, S* xn) {
  constexpr int N = M::NX;
  S d[N];
  step_inc<M, S, PT>(integ, dt, p, x, u, d);
#pragma unroll
  for (int i = 0; i < N; i++) xn[i] = x[i] + d[i];
}

// Jacobians of the increment: E = d(f - x)/dx (so F = I + E) and G = df/du, plus the
// increment value, by forward-mode AD in scalar S.
template <class M, class S>
PTN_HD void inc_jac(int integ, double dt, const double* p, const double* x, const double* u, S* dv, S* E,
                    S* G) {
  constexpr int N = M::NX, U = M::NU, K = N + U;
  using D = Dual<S, K>;
  D xd[N], ud[U], dn[N];
#pragma unroll
  for (int i = 0; i < N; i++) { xd[i] = D(S(x[i])); xd[i].d[i] = S(1); }
#pragma unroll
  for (int i = 0; i < U; i++) { ud[i] = D(S(u[i])); ud[i].d[N + i] = S(1); }
  step_inc<M>(integ, dt, p, xd, ud, dn);
#pragma unroll
  for (int i = 0; i < N; i++) {
    if (dv) dv[i] = dn[i].v;
#pragma unroll
    for (int j = 0; j < N; j++) E[i * N + j] = dn[i].d[j];
#pragma unroll
    for (int j = 0; j < U; j++) G[i * U + j] = dn[i].d[N + j];
  }
}

// Closed-loop increment at (x, u) with u = ub + Gam (x - xh): value dx and
// Ecl = d dx / dx = E + G Gam (so Fcl = I + Ecl), seeds (e_i, Gam e_i).
template <class M, class S>
PTN_HD void inc_cl(int integ, double dt, const double* p, const S* x, const S* u, const S* Gam, S* dv,
                   S* Ecl) {
  constexpr int N = M::NX, U = M::NU;
  using D = Dual<S, N>;
  D xd[N], ud[U], dn[N];
#pragma unroll
  for (int i = 0; i < N; i++) { xd[i] = D(x[i]); xd[i].d[i] = S(1); }
#pragma unroll
  for (int i = 0; i < U; i++) {
    ud[i] = D(u[i]);
#pragma unroll
    for (int j = 0; j < N; j++) ud[i].d[j] = Gam[i * N + j];
  }
  step_inc<M>(integ, dt, p, xd, ud, dn);
#pragma unroll
  for (int i = 0; i < N; i++) {
    dv[i] = dn[i].v;
#pragma unroll
    for (int j = 0; j < N; j++) Ecl[i * N + j] = dn[i].d[j];
  }
}

// F = df/dx (NX x NX), G = df/du (NX x NU), by forward-mode AD in scalar S.
template <class M, class S>
PTN_HD void step_jac(int integ, double dt, const double* p, const double* x, const double* u,
                     S* fx, S* F, S* G) {
  constexpr int N = M::NX, U = M::NU, K = N + U;
  using D = Dual<S, K>;
  D xd[N], ud[U], xn[N];
#pragma unroll
  for (int i = 0; i < N; i++) { xd[i] = D(S(x[i])); xd[i].d[i] = S(1); }
#pragma unroll
  for (int i = 0; i < U; i++) { ud[i] = D(S(u[i])); ud[i].d[N + i] = S(1); }
  step<M>(integ, dt, p, xd, ud, xn);
#pragma unroll
  for (int i = 0; i < N; i++) {
    if (fx) fx[i] = xn[i].v;
#pragma unroll
    for (int j = 0; j < N; j++) F[i * N + j] = xn[i].d[j];
#pragma unroll
    for (int j = 0; j < U; j++) G[i * U + j] = xn[i].d[N + j];
  }
}

// Second-order contraction lam . f_zz (Sec. III-C): Hxx, Hxu, Huu in scalar S.
template <class M, class S>
PTN_HD void step_hess(int integ, double dt, const double* p, const double* x, const double* u,
                      const double* lam, S* Hxx, S* Hxu, S* Huu) {
  constexpr int N = M::NX, U = M::NU, K = N + U;
  using J = Jet<S, K>;
  J xd[N], ud[U], xn[N];
#pragma unroll
  for (int i = 0; i < N; i++) { xd[i] = J(S(x[i])); xd[i].d[i] = S(1); }
#pragma unroll
  for (int i = 0; i < U; i++) { ud[i] = J(S(u[i])); ud[i].d[N + i] = S(1); }
  step<M>(integ, dt, p, xd, ud, xn);
  S h[J::H];
#pragma unroll (K <= 8 ? J::H : 2)
  for (int q = 0; q < J::H; q++) {
    S s = S(0);
#pragma unroll (K <= 8 ? N : 4)
    for (int k = 0; k < N; k++) s += S(lam[k]) * xn[k].h[q];
    h[q] = s;
  }
#pragma unroll
  for (int i = 0; i < K; i++)
#pragma unroll
    for (int j = i; j < K; j++) {
      const S v = h[hidx<K>(i, j)];
      if (j < N) { Hxx[i * N + j] = v; Hxx[j * N + i] = v; }
      else if (i < N) Hxu[i * U + (j - N)] = v;
      else { Huu[(i - N) * U + (j - N)] = v; Huu[(j - N) * U + (i - N)] = v; }
    }
}

// Closed-loop Jacobian of x+ = f(x, ub + Gam (x - xh)) with respect to x at (x, u):
// Fcl = F + G Gam, computed by forward mode with seeds (e_i, Gam e_i).
template <class M, class S>
PTN_HD void step_cl_jac(int integ, double dt, const double* p, const double* x, const double* u,
                        const S* Gam, S* Fcl) {
  constexpr int N = M::NX, U = M::NU;
  using D = Dual<S, N>;
  D xd[N], ud[U], xn[N];
#pragma unroll
  for (int i = 0; i < N; i++) { xd[i] = D(S(x[i])); xd[i].d[i] = S(1); }
#pragma unroll
  for (int i = 0; i < U; i++) {
    ud[i] = D(S(u[i]));
#pragma unroll
    for (int j = 0; j < N; j++) ud[i].d[j] = Gam[i * N + j];
  }
  step<M>(integ, dt, p, xd, ud, xn);
#pragma unroll
  for (int i = 0; i < N; i++)
#pragma unroll
    for (int j = 0; j < N; j++) Fcl[i * N + j] = xn[i].d[j];
}

// Parameter derivatives of one step for the adjoint:
//   fp  (NX x NP)       df/dprm
//   Hzp ((NX+NU) x NP)  d2 (lam^T f) / dz dprm
// by nested forward mode (outer: z = (x, u), inner: prm), in FP64.
template <class M>
PTN_HD void step_param_derivs(int integ, double dt, const double* prm, const double* x, const double* u,
                              const double* lam, double* fp, double* Hzp) {
  constexpr int N = M::NX, U = M::NU, K = N + U, NP = M::NP;
  using PD = Dual<double, NP>;
  using D = Dual<PD, K>;
  PD p[NP];
#pragma unroll
  for (int k = 0; k < NP; k++) { p[k] = PD(prm[k]); p[k].d[k] = 1.0; }
  D xd[N], ud[U], xn[N];
#pragma unroll
  for (int i = 0; i < N; i++) { xd[i] = D(PD(x[i])); xd[i].d[i] = PD(1.0); }
#pragma unroll
  for (int i = 0; i < U; i++) { ud[i] = D(PD(u[i])); ud[i].d[N + i] = PD(1.0); }
  step<M, D, PD>(integ, dt, p, xd, ud, xn);
#pragma unroll
  for (int i = 0; i < N; i++)
#pragma unroll
    for (int k = 0; k < NP; k++) fp[i * NP + k] = xn[i].v.d[k];
#pragma unroll
  for (int j = 0; j < K; j++)
#pragma unroll
    for (int k = 0; k < NP; k++) {
      double h = 0.0;
#pragma unroll
      for (int i = 0; i < N; i++) h += lam[i] * xn[i].d[j].d[k];
      Hzp[j * NP + k] = h;
    }
}

}  // namespace ptn
