// ptn_launch.cuh -- host-side launch of the solver kernels for one model type.
#pragma once
#include <mutex>

#include "ptn_solver.cuh"

namespace ptn {

// Raise, never lower, a kernel's dynamic shared-memory limit (a per-function, process-wide
// attribute): a launch recorded earlier with a larger size -- in a captured CUDA graph, or
// prepared by ptn_batch_prepare -- stays valid after launches of smaller shapes.
template <auto Kernel>
cudaError_t raise_smem_limit(size_t bytes) {
  static std::mutex mu;
  static size_t limit = 0;
  std::lock_guard<std::mutex> lk(mu);
  if (bytes <= limit) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) limit = bytes;
  return e;
}

// untyped workspace pointers (LQR arrays are allocated with 8 bytes per entry so that
// either precision fits)
struct WorkRaw {
  double *xA, *uA, *xB, *uB, *lam, *d, *F64, *G64;
  void *E, *Gm, *Pm, *Mm, *Rm, *Gam, *gam, *dx, *du;
  double *z, *v;
  double *q, *dnu;  // multiplier form (may be null when it is not used)
  void *Sv, *sv;
};

template <class L>
inline Work<L> typed(const WorkRaw& r) {
  Work<L> w;
  w.xA = r.xA; w.uA = r.uA; w.xB = r.xB; w.uB = r.uB; w.lam = r.lam;
  w.d = r.d; w.F64 = r.F64; w.G64 = r.G64; w.E = (L*)r.E; w.Gm = (L*)r.Gm;
  w.Pm = (L*)r.Pm; w.Mm = (L*)r.Mm; w.Rm = (L*)r.Rm; w.Gam = (L*)r.Gam; w.gam = (L*)r.gam;
  w.dx = (L*)r.dx; w.du = (L*)r.du; w.z = r.z; w.v = r.v;
  w.q = r.q; w.dnu = r.dnu; w.Sv = (L*)r.Sv; w.sv = (L*)r.sv;
  return w;
}

struct LaunchReq {
  int tier;       // 0: one CTA per instance, 1: cooperative grid, 2: one cluster on one instance,
                  // 3: adjoint, one CTA per instance, 4: wide (n >= 8, one warp per chunk),
                  // 5: sequential-in-time baseline (one thread per instance), 6: wide on the
                  // cooperative grid (one instance), 7: adjoint of one instance on the grid,
                  // 8: wide batch on a cooperative grid, a CTA range per instance
  int precision;  // 0: FP64, 1: FP32 with FP64 solves, 2: FP32
  int nblocks, nthreads;
  int query;      // 1: only report max co-resident grid blocks in *max_blocks;
                  // 2: only set the kernel's function attributes for this launch shape
  int attrs_set;  // nonzero: the attributes were set by an earlier query 2, launch only
                  // (no runtime call besides the launch, so that it can be graph-captured)
  int* max_blocks;
  size_t* elem_bytes;  // out: bytes of the largest scan element
  KArgs args;
  WorkRaw w;
  cudaStream_t stream;
  const AdjArgs* adj;  // tier 3
};

template <class M, class L, class SV>
cudaError_t launch_typed(LaunchReq& q) {
  constexpr int N = M::NX, U = M::NU;
  const int nthreads = q.nthreads;
  const size_t smem = ((sizeof(ProbS<N, U>) + 15) & ~size_t(15)) + scratch_bytes<N, U, L>(nthreads / 32);
  if (q.elem_bytes) *q.elem_bytes = sizeof(Val<N, L>);
  if (q.tier == 0) {
    if (!q.attrs_set) {
      cudaError_t e = raise_smem_limit<k_solve_cta<M, L, SV>>(smem);
      if (e != cudaSuccess) return e;
    }
    if (q.query) return cudaSuccess;
    k_solve_cta<M, L, SV><<<q.nblocks, nthreads, smem, q.stream>>>(q.args, typed<L>(q.w));
    return cudaGetLastError();
  }
  if (q.tier == 5) {
    if (q.query) return cudaSuccess;
    k_solve_seq<M, L, SV><<<q.nblocks, q.nthreads, 0, q.stream>>>(q.args, typed<L>(q.w));
    return cudaGetLastError();
  }
  if (q.tier == 7) {
    // the adjoint of one instance on the cooperative grid (FP64 units only)
    if constexpr (std::is_same<L, double>::value) {
      cudaError_t e = raise_smem_limit<k_adjoint_grid<M, L, SV>>(smem);
      if (e != cudaSuccess) return e;
      if (q.query == 1) {
        int dev = 0, per = 0, sms = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_adjoint_grid<M, L, SV>, nthreads, smem);
        if (e != cudaSuccess) return e;
        *q.max_blocks = per * sms;
        return cudaSuccess;
      }
      if (q.query) return cudaSuccess;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(q.nblocks);
      cfg.blockDim = dim3(nthreads);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = q.stream;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeCooperative;
      at[0].val.cooperative = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      return cudaLaunchKernelEx(&cfg, k_adjoint_grid<M, L, SV>, q.args, typed<L>(q.w), *q.adj);
    } else {
      return cudaErrorNotSupported;
    }
  }
  if (q.tier == 3) {
    // the adjoint is built only in the FP64 units (it runs in FP64 in every mode)
    if constexpr (std::is_same<L, double>::value) {
      cudaError_t e = raise_smem_limit<k_adjoint_cta<M, L, SV>>(smem);
      if (e != cudaSuccess) return e;
      if (q.query) return cudaSuccess;
      k_adjoint_cta<M, L, SV><<<q.nblocks, nthreads, smem, q.stream>>>(q.args, typed<L>(q.w), *q.adj);
      return cudaGetLastError();
    } else {
      return cudaErrorNotSupported;
    }
  }
  if (q.tier == 2) {
    const size_t smc = ((smem + 15) & ~size_t(15)) + cluster_xch_bytes<N, U, L>();
    cudaError_t e = cudaSuccess;
    if (!q.attrs_set) {
      e = raise_smem_limit<k_solve_cluster<M, L, SV>>(smc);
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(k_solve_cluster<M, L, SV>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    if (q.query == 2) return cudaSuccess;
    if (q.query) {
      // largest cluster of these CTAs the device can co-schedule (the cluster
      // dimension in cfg is ignored by the query)
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(16);
      cfg.blockDim = dim3(nthreads);
      cfg.dynamicSmemBytes = smc;
      int maxc = 0;
      e = cudaOccupancyMaxPotentialClusterSize(&maxc, k_solve_cluster<M, L, SV>, &cfg);
      *q.max_blocks = maxc;
      return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(q.nblocks);
    cfg.blockDim = dim3(nthreads);
    cfg.dynamicSmemBytes = smc;
    cfg.stream = q.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = q.nblocks;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_solve_cluster<M, L, SV>, q.args, typed<L>(q.w));
  }
  cudaError_t e = cudaSuccess;
  if (!q.attrs_set) {
    e = raise_smem_limit<k_solve_grid<M, L, SV>>(smem);
    if (e != cudaSuccess) return e;
  }
  if (q.query == 2) return cudaSuccess;
  if (q.query) {
    int dev = 0, per = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_solve_grid<M, L, SV>, nthreads, smem);
    if (e != cudaSuccess) return e;
    *q.max_blocks = per * sms;
    return cudaSuccess;
  }
  // cooperative launch (all CTAs co-resident) through the extensible launch call, which a
  // stream capture records as a cooperative kernel node
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(q.nblocks);
  cfg.blockDim = dim3(nthreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = q.stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_solve_grid<M, L, SV>, q.args, typed<L>(q.w));
}


}  // namespace ptn
