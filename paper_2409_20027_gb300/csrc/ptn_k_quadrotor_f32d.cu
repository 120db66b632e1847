// Solver kernels for the quadrotor model (n = 12, m = 4): the wide tier, FP32 LQR data
// with FP64 solves, FP64 gradients, rollouts and merits.
#include "ptn_launch.cuh"
#include "ptn_wide.cuh"

cudaError_t ptn_launch_quadrotor_f32d(ptn::LaunchReq& q) { return ptn::launch_wide<ptn::Quadrotor, float, double>(q); }
