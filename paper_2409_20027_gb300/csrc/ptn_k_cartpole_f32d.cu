// Solver kernels for the cartpole model, FP32 LQR with FP64 solves.
#include "ptn_launch.cuh"

cudaError_t ptn_launch_cartpole_f32d(ptn::LaunchReq& q) { return ptn::launch_typed<ptn::CartPole, float, double>(q); }
