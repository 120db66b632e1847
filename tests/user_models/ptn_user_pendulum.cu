// A model supplied from outside the library through ptn_user_model.cuh: the damped pendulum
// of Sec. IV-A (theta'' = -(g/l) sin(theta) - b/(m l^2) theta' + u/(m l^2)) declared again
// as user model 64, so that the registration path can be checked against the built-in
// pendulum and the oracle.  Constants p = [g, l, m, b], as for the built-in model.
#include "ptn_user_model.cuh"

struct UserPendulum {
  static constexpr int NX = 2, NU = 1, NP = 4, ID = 64;
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
};

PTN_REGISTER_MODEL_FP64(UserPendulum)
