// Solver kernels for the synthetic map x+ = A x + B u + c tanh(W x) (n = 32, m = 8), wide
// tier, FP32 LQR data with FP64 solves.
#include "ptn_launch.cuh"
#include "ptn_synth_wide.cuh"

cudaError_t ptn_launch_synth_f32d(ptn::LaunchReq& q) { return ptn::launch_wide<ptn::Synth, float, double>(q); }
