// Solver kernels for the pendulum model, FP64.
#include "ptn_launch.cuh"

cudaError_t ptn_launch_pendulum_f64(ptn::LaunchReq& q) { return ptn::launch_typed<ptn::Pendulum, double, double>(q); }
