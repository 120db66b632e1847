// Solver kernels for the pendulum model, FP32 LQR and solves.
#include "ptn_launch.cuh"

cudaError_t ptn_launch_pendulum_f32(ptn::LaunchReq& q) { return ptn::launch_typed<ptn::Pendulum, float, float>(q); }
