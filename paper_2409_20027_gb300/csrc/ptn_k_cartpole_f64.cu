// Solver kernels for the cartpole model, FP64.
#include "ptn_launch.cuh"

cudaError_t ptn_launch_cartpole_f64(ptn::LaunchReq& q) { return ptn::launch_typed<ptn::CartPole, double, double>(q); }
