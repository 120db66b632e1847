// A model with user-written terms (ptn_user_model.cuh): the pendulum of Sec. IV-A with its
// own stage cost (a quartic and a 1 - cos term on the angle error besides the quadratic
// ones), its own terminal cost, and a time-varying inequality row on the angular rate,
// w^2 <= 9 + 0.05 t.  The oracle's side of the same problem is given as callbacks in
// tests/test_oracle_user_terms.py (pendulum_user_problem).
#include "ptn_user_model.cuh"

struct UserCostPendulum {
  static constexpr int NX = 2, NU = 1, NP = 4, ID = 65;
  static constexpr bool USER_COST = true;
  static constexpr int NC = 1;
  static constexpr double kPi = 3.14159265358979323846;

  template <class S, class PT>
  PTN_HD static void rhs(const PT* p, const S* x, const S* u, S* xd) {
    using ptn::cmul;
    const auto g = ptn::pconv<S>(p[0]), l = ptn::pconv<S>(p[1]), m = ptn::pconv<S>(p[2]), b = ptn::pconv<S>(p[3]);
    const auto iml2 = decltype(g)(1) / (m * l * l);
    S s, c;
    ptn::sincos_ad(x[0], s, c);
    xd[0] = x[1];
    xd[1] = cmul(-g / l, s) + cmul(-b * iml2, x[1]) + cmul(iml2, u[0]);
  }

  template <class S>
  PTN_HD static S stage_l(int t, const double* p, const S* x, const S* u) {
    using ptn::cadd;
    using ptn::cmul;
    (void)t; (void)p;
    const S e = cadd(-kPi, x[0]);
    S sn, cs;
    ptn::sincos_ad(e, sn, cs);
    const S e2 = e * e;
    return e2 + cmul(0.1, x[1] * x[1]) + cmul(0.01, u[0] * u[0]) + cmul(0.05, e2 * e2) + cmul(0.3, cadd(1.0, -cs));
  }

  template <class S>
  PTN_HD static S terminal_l(const double* p, const S* x) {
    using ptn::cadd;
    using ptn::cmul;
    (void)p;
    const S e = cadd(-kPi, x[0]);
    return cmul(10.0, e * e) + x[1] * x[1];
  }

  template <class S>
  PTN_HD static void constraints(int t, const double* p, const S* x, const S* u, S* g) {
    (void)p; (void)u;
    g[0] = ptn::cadd(-(9.0 + 0.05 * t), x[1] * x[1]);
  }
};

PTN_REGISTER_MODEL(UserCostPendulum)
