// Solver kernels for the cartpole model, FP32 LQR and solves.
#include "ptn_launch.cuh"

cudaError_t ptn_launch_cartpole_f32(ptn::LaunchReq& q) { return ptn::launch_typed<ptn::CartPole, float, float>(q); }
