// Solver kernels for the pendulum model, FP32 LQR with FP64 solves.
#include "ptn_launch.cuh"

cudaError_t ptn_launch_pendulum_f32d(ptn::LaunchReq& q) { return ptn::launch_typed<ptn::Pendulum, float, double>(q); }
