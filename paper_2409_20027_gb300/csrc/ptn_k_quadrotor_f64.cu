// Solver and adjoint kernels for the quadrotor model (n = 12, m = 4), wide tier in FP64.
#include "ptn_launch.cuh"
#include "ptn_wide.cuh"

cudaError_t ptn_launch_quadrotor_f64(ptn::LaunchReq& q) { return ptn::launch_wide<ptn::Quadrotor, double, double>(q); }
