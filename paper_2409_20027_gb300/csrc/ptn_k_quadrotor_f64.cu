// Solver kernels for the quadrotor model with double LQR arithmetic.
#include "ptn_launch.cuh"

cudaError_t ptn_launch_quadrotor_f64(ptn::LaunchReq& q) { return ptn::launch_typed<ptn::Quadrotor, double>(q); }
