// Solver kernels for the quadrotor model with float LQR arithmetic.
#include "ptn_launch.cuh"

cudaError_t ptn_launch_quadrotor_f32(ptn::LaunchReq& q) { return ptn::launch_typed<ptn::Quadrotor, float>(q); }
