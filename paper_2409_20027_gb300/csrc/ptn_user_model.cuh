// ptn_user_model.cuh -- adding a dynamics model to the library from outside it.
//
// The problem class of Sec. II-A is x_{t+1} = f(x_t, u_t) with quadratic tracking costs and
// box constraints.  A model supplies f as a continuous-time right-hand side written once as
// a template over the scalar type, exactly like the built-in models (ptn_models.cuh):
//
//   struct MyModel {
//     static constexpr int NX = 3, NU = 1, NP = 2, ID = 64;   // ID >= PTN_USER_MODEL_MIN
//     template <class S, class PT>
//     PTN_HD static void rhs(const PT* p, const S* x, const S* u, S* xd) { ... }
//   };
//   PTN_REGISTER_MODEL(MyModel)        // or PTN_REGISTER_MODEL_FP64(MyModel)
//
// p holds the problem's eight model constants (ptn_problem.prm); the integrator (Euler or
// RK4) and the time step come from ptn_problem.
//
// A model with NX < 8 may also replace the quadratic tracking cost and add inequality rows
// (the general l_t, l_T and g_t(x, u) <= 0 of Sec. II-A), again as templates over S:
//
//     static constexpr bool USER_COST = true;
//     template <class S> PTN_HD static S stage_l(int t, const double* p, const S* x, const S* u);
//     template <class S> PTN_HD static S terminal_l(const double* p, const S* x);
//     static constexpr int NC = 1;     // rows, at most 8
//     template <class S> PTN_HD static void constraints(int t, const double* p, const S* x, const S* u, S* g);
//
// t is the step (0 .. T-1).  The rows join the box bounds in the log barrier (interior
// point; ADMM refuses a model with rows); the start (u_init, or 0) must satisfy them
// strictly.  Gradients and Hessians come from the same Dual / nested Dual scalars;
// constants enter through cst<S>(c), cmul(c, a) and cadd(c, a).  The adjoint's gradients
// with respect to Q, R and Qf are zero for such a model.  The same code is evaluated on plain values,
// on dual numbers (Jacobians) and on second-order jets (the lambda-contracted Hessians of
// Sec. III-C), so it may use the helpers the built-in models use (pconv, cmul, cadd, recip,
// sincos_ad) and arithmetic operators on S.  Models with NX < 8 run the CTA / cluster /
// grid tiers, 8 <= NX <= 32 the wide tier (FP64 and FP32 LQR with FP64 solves only).
//
// Put the struct and the macro in a .cu file and pass it to build(extra=[...]): the file is
// compiled with this directory on the include path and linked into the library, and the
// macro registers the model's launchers when the library is loaded.  ptn_problem.model =
// ID then selects it; nx, nu must match NX, NU.
#pragma once
#include "ptn_launch.cuh"
#include "ptn_wide.cuh"

namespace ptn {

constexpr int PTN_USER_MODEL_MIN = 64;

typedef cudaError_t (*user_launch_fn)(LaunchReq&);

// Records the launchers of model `id` (defined in ptn_api.cu).  Returns 0, or -1 when the
// id is below PTN_USER_MODEL_MIN, already taken, the table is full or the sizes are out of
// range (the model is then not available and solves report an unknown model id).
int register_model(int id, int nx, int nu, user_launch_fn f64, user_launch_fn f32d, user_launch_fn f32,
                   int nrows);

template <class M, class L, class SV>
cudaError_t launch_user_model(LaunchReq& q) {
  static_assert(M::NX < 8 || !has_user_terms<M>::value,
                "user-written costs and constraint rows are built for models with NX < 8");
  static_assert(user_rows<M>::value <= 8, "at most 8 user constraint rows");
  if constexpr (M::NX >= 8) {
    return launch_wide<M, L, SV>(q);
  } else {
    return launch_typed<M, L, SV>(q);
  }
}

}  // namespace ptn

#define PTN_USER_LAUNCHERS_(M)                                                                          \
  static cudaError_t ptn_user_f64_##M(ptn::LaunchReq& q) { return ptn::launch_user_model<M, double, double>(q); } \
  static cudaError_t ptn_user_f32d_##M(ptn::LaunchReq& q) { return ptn::launch_user_model<M, float, double>(q); }

// all precisions (PTN_FP32 only for NX < 8)
#define PTN_REGISTER_MODEL(M)                                                                           \
  PTN_USER_LAUNCHERS_(M)                                                                                \
  static cudaError_t ptn_user_f32_##M(ptn::LaunchReq& q) {                                              \
    if constexpr (M::NX >= 8) return cudaErrorNotSupported;                                             \
    else return ptn::launch_user_model<M, float, float>(q);                                             \
  }                                                                                                     \
  static const int ptn_user_registered_##M =                                                            \
      ptn::register_model(M::ID, M::NX, M::NU, ptn_user_f64_##M, ptn_user_f32d_##M, ptn_user_f32_##M, \
                          ptn::user_rows<M>::value);

// PTN_FP64 only (one kernel set: the shortest build)
#define PTN_REGISTER_MODEL_FP64(M)                                                                      \
  static cudaError_t ptn_user_f64_##M(ptn::LaunchReq& q) { return ptn::launch_user_model<M, double, double>(q); } \
  static const int ptn_user_registered_##M =                                                            \
      ptn::register_model(M::ID, M::NX, M::NU, ptn_user_f64_##M, nullptr, nullptr, ptn::user_rows<M>::value);
