// ptn_group.cuh -- collectives for the thread group that solves one instance.
//
// A group is either one CTA (CtaGroup: batches of instances, one per block) or the
// whole cooperative grid (GridGroup: one long-horizon instance across all SMs).
// Each group thread owns a contiguous chunk of time steps; the scans of the three
// passes combine the chunks' aggregates across the group with these collectives:
//
//   reduce<K>(v, maxmask)      sums / maxima of K doubles, identical in every thread
//   scan(v, op, suffix, ok)    exclusive prefix (or suffix) combination of the
//                              threads' elements in time order, op(a, b, out) meaning
//                              "a is earlier than b"
//
// Warp level: Kogge-Stone over shuffles.  Block level: warp totals in shared memory.
// Grid level: block totals in global memory behind a grid barrier whose wait is
// bounded (spin_limit); on expiry the group records ST_ETIMEOUT and stops.
#pragma once
#include <cooperative_groups.h>

#include "ptn_ops.cuh"

namespace ptn {

#define PTN_FULL 0xffffffffu

template <class E>
__device__ __forceinline__ E shfl_up_e(const E& e, int delta) {
  static_assert(sizeof(E) % 4 == 0, "element must be a multiple of 4 bytes");
  E r;
  const unsigned* s = reinterpret_cast<const unsigned*>(&e);
  unsigned* d = reinterpret_cast<unsigned*>(&r);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(E) / 4); i++) d[i] = __shfl_up_sync(PTN_FULL, s[i], delta);
  return r;
}
template <class E>
__device__ __forceinline__ E shfl_down_e(const E& e, int delta) {
  E r;
  const unsigned* s = reinterpret_cast<const unsigned*>(&e);
  unsigned* d = reinterpret_cast<unsigned*>(&r);
#pragma unroll
  for (int i = 0; i < (int)(sizeof(E) / 4); i++) d[i] = __shfl_down_sync(PTN_FULL, s[i], delta);
  return r;
}

// Block-level exclusive scan.  Writes the block total (all elements of the block
// combined in time order) into *total (shared memory) and returns each thread's
// exclusive result.  Needs blockDim.x / 32 elements of shared scratch at sw.
template <class E, class Op>
__device__ E block_scan_excl(E v, const Op& op, bool suffix, bool& ok, E* sw, E* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll 1
  for (int off = 1; off < 32; off <<= 1) {
    if (!suffix) {
      E o = shfl_up_e(v, off);
      if (lane >= off) ok &= op(o, v, v);
    } else {
      E o = shfl_down_e(v, off);
      if (lane + off < 32) ok &= op(v, o, v);
    }
  }
  E ex = suffix ? shfl_down_e(v, 1) : shfl_up_e(v, 1);
  if ((!suffix && lane == 0) || (suffix && lane == 31)) set_identity(ex);
  __syncthreads();
  if ((!suffix && lane == 31) || (suffix && lane == 0)) sw[w] = v;
  __syncthreads();
  if (!suffix) {
    if (w > 0) {
      E wt = sw[0];
#pragma unroll 1
      for (int i = 1; i < w; i++) ok &= op(wt, sw[i], wt);
      ok &= op(wt, ex, ex);
    }
  } else {
    if (w < nw - 1) {
      E wt = sw[nw - 1];
#pragma unroll 1
      for (int i = nw - 2; i > w; i--) ok &= op(sw[i], wt, wt);
      ok &= op(ex, wt, ex);
    }
  }
  if (total) {
    // block total: the fold of all warp totals in time order, by thread 0
    if (threadIdx.x == 0) {
      E t = sw[0];
#pragma unroll 1
      for (int i = 1; i < nw; i++) ok &= op(t, sw[i], t);
      *total = t;
    }
  }
  __syncthreads();
  return ex;
}

// ---------------------------------------------------------------------------
struct CtaGroup {
  char* sm;  // shared scratch (>= max(nwarps * sizeof(element)+sizeof(element), nwarps*8*K))

  __device__ int rank() const { return threadIdx.x; }
  __device__ int size() const { return blockDim.x; }
  __device__ void sync() { __syncthreads(); }
  __device__ bool dead() const { return false; }

  template <int K>
  __device__ void reduce(double (&v)[K], unsigned maxmask) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double* s = reinterpret_cast<double*>(sm);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
      for (int k = 0; k < K; k++) {
        double o = __shfl_xor_sync(PTN_FULL, v[k], off);
        v[k] = ((maxmask >> k) & 1u) ? fmax(v[k], o) : v[k] + o;
      }
    __syncthreads();
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < K; k++) s[w * K + k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; k++) {
      double a = s[k];
      for (int i = 1; i < nw; i++) a = ((maxmask >> k) & 1u) ? fmax(a, s[i * K + k]) : a + s[i * K + k];
      v[k] = a;
    }
    __syncthreads();
  }

  template <class E, class Op>
  __device__ E scan(E v, const Op& op, bool suffix, bool& ok) {
    return block_scan_excl(v, op, suffix, ok, reinterpret_cast<E*>(sm), (E*)nullptr);
  }

  // scan followed by a reduction of K values (one group barrier each within a CTA)
  template <class E, class Op, int K>
  __device__ E scan_reduce(E v, const Op& op, bool suffix, bool& ok, double (&red)[K], unsigned maxmask) {
    E r = scan(v, op, suffix, ok);
    reduce<K>(red, maxmask);
    return r;
  }
};

// ---------------------------------------------------------------------------
// Grid group: all blocks of a cooperative launch work on one instance.
struct GridScratch {
  unsigned* bar;      // [0] arrivals, [1] generation
  int* err;           // error word (ST_ETIMEOUT on an expired wait)
  double* red;        // 2 x nblocks x 8 doubles
  char* xs;           // 2 x nblocks x elem_bytes
  long long spin_limit;
  int elem_bytes;
  int pad;
};

__device__ __forceinline__ bool grid_barrier(const GridScratch& gs) {
  volatile unsigned* gen = gs.bar + 1;
  const unsigned g0 = *gen;
  __threadfence();
  const unsigned arrived = atomicAdd(gs.bar, 1u);
  if (arrived == gridDim.x - 1) {
    atomicExch(gs.bar, 0u);
    __threadfence();
    atomicAdd(gs.bar + 1, 1u);
    return true;
  }
  long long n = 0;
  while (*gen == g0) {
    if (++n > gs.spin_limit) {
      atomicExch(gs.err, ST_ETIMEOUT);
      return false;
    }
    __nanosleep(64);
  }
  __threadfence();
  return true;
}

struct GridGroup {
  char* sm;
  GridScratch gs;
  int phase;
  int* sdead;  // shared flag: this block saw a barrier expire

  __device__ int rank() const { return blockIdx.x * blockDim.x + threadIdx.x; }
  __device__ int size() const { return gridDim.x * blockDim.x; }
  __device__ bool dead() const { return *(volatile int*)sdead != 0; }

  __device__ void sync() {
    __syncthreads();
    if (threadIdx.x == 0 && !*sdead) {
      if (!grid_barrier(gs)) *sdead = 1;
    }
    __syncthreads();
  }

  // Warp 0 combines the K block values of every block (written before the barrier):
  // each lane folds blocks lane, lane + 32, ... in order, all K loads of a block issued
  // together, then an ordered shuffle tree -- the same in every block, so every block gets
  // bit-identical results; lane 0 stores them to sres.
  template <int K>
  __device__ void totals_warp0(const double* rslot, unsigned maxmask, double* sres) const {
    const int lane = threadIdx.x;
    double a[K];
#pragma unroll
    for (int k = 0; k < K; k++) a[k] = ((maxmask >> k) & 1u) ? -INFINITY : 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) {
      double o[K];
#pragma unroll
      for (int k = 0; k < K; k++) o[k] = __ldcg(rslot + (size_t)b * 8 + k);
#pragma unroll
      for (int k = 0; k < K; k++) a[k] = ((maxmask >> k) & 1u) ? fmax(a[k], o[k]) : a[k] + o[k];
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
      for (int k = 0; k < K; k++) {
        const double o = __shfl_down_sync(PTN_FULL, a[k], off);
        if ((lane & (2 * off - 1)) == 0) a[k] = ((maxmask >> k) & 1u) ? fmax(a[k], o) : a[k] + o;
      }
    }
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < K; k++) sres[k] = a[k];
  }

  // Warp 0 folds the totals of the blocks before (prefix) or after (suffix) this one: each
  // lane folds a contiguous range, then an ordered tree; lane 0 stores the carry.
  template <class E, class Op>
  __device__ void carry_warp0(const E* slot, const Op& op, bool suffix, bool& ok, E* scarry) const {
    const int lane = threadIdx.x;
    const int lo = suffix ? blockIdx.x + 1 : 0;
    const int hi = suffix ? gridDim.x : blockIdx.x;
    const int cnt = hi - lo;
    const int per = (cnt + 31) / 32;
    E acc;
    set_identity(acc);
    const int b0 = lo + lane * per;
    const int b1 = min(hi, b0 + per);
    for (int b = b0; b < b1; b++) {
      E t;
      const char* src = reinterpret_cast<const char*>(slot) + (size_t)b * gs.elem_bytes;
      // volatile-free copy through L2 (written before the barrier by another block)
      const unsigned* s4 = reinterpret_cast<const unsigned*>(src);
      unsigned* d4 = reinterpret_cast<unsigned*>(&t);
#pragma unroll
      for (int i = 0; i < (int)(sizeof(E) / 4); i++) d4[i] = __ldcg(s4 + i);
      if (b == b0) acc = t;
      else ok &= op(acc, t, acc);
    }
#pragma unroll 1
    for (int off = 1; off < 32; off <<= 1) {
      E o = shfl_down_e(acc, off);
      if ((lane & (2 * off - 1)) == 0 && lane + off < 32) ok &= op(acc, o, acc);
    }
    if (lane == 0) *scarry = acc;
  }

  template <int K>
  __device__ void reduce(double (&v)[K], unsigned maxmask) {
    static_assert(K <= 8, "at most 8 values per reduction");
    CtaGroup cg{sm};
    cg.reduce<K>(v, maxmask);
    double* slot = gs.red + (size_t)phase * gridDim.x * 8;
    if (threadIdx.x == 0)
#pragma unroll
      for (int k = 0; k < K; k++) slot[blockIdx.x * 8 + k] = v[k];
    sync();
    double* sres = reinterpret_cast<double*>(sm);
    if (threadIdx.x < 32) totals_warp0<K>(slot, maxmask, sres);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = sres[k];
    __syncthreads();
    phase ^= 1;
  }

  template <class E, class Op>
  __device__ E scan(E v, const Op& op, bool suffix, bool& ok) {
    const int nw = blockDim.x >> 5;
    E* sw = reinterpret_cast<E*>(sm);
    E* stot = sw + nw;      // block total
    E* scarry = sw + nw + 1;  // carry from other blocks
    E ex = block_scan_excl(v, op, suffix, ok, sw, stot);
    E* slot = reinterpret_cast<E*>(gs.xs + (size_t)phase * gridDim.x * gs.elem_bytes);
    if (threadIdx.x == 0) *reinterpret_cast<E*>(reinterpret_cast<char*>(slot) + (size_t)blockIdx.x * gs.elem_bytes) = *stot;
    sync();
    if (threadIdx.x < 32) carry_warp0(slot, op, suffix, ok, scarry);
    __syncthreads();
    if (!suffix) {
      if (blockIdx.x > 0) ok &= op(*scarry, ex, ex);
    } else {
      if (blockIdx.x + 1 < gridDim.x) ok &= op(ex, *scarry, ex);
    }
    __syncthreads();
    phase ^= 1;
    return ex;
  }

  // scan (as scan) and a reduction of K values (as reduce) behind one grid barrier: the
  // block reduces its values first, then scans, and thread 0 publishes both; warp 0 then
  // computes the carry and the totals from the same barrier.  Needs block scratch for
  // nwarps + 2 elements plus 8 + 8 K bytes.
  template <class E, class Op, int K>
  __device__ E scan_reduce(E v, const Op& op, bool suffix, bool& ok, double (&red)[K], unsigned maxmask) {
    static_assert(K <= 8, "at most 8 values per reduction");
    CtaGroup cg{sm};
    cg.reduce<K>(red, maxmask);  // ends with a block barrier, so the scratch is free again
    const int nw = blockDim.x >> 5;
    E* sw = reinterpret_cast<E*>(sm);
    E* stot = sw + nw;
    E* scarry = sw + nw + 1;
    double* sres = reinterpret_cast<double*>((reinterpret_cast<size_t>(scarry + 1) + 7) & ~size_t(7));
    E ex = block_scan_excl(v, op, suffix, ok, sw, stot);
    E* slot = reinterpret_cast<E*>(gs.xs + (size_t)phase * gridDim.x * gs.elem_bytes);
    double* rslot = gs.red + (size_t)phase * gridDim.x * 8;
    if (threadIdx.x == 0) {
      *reinterpret_cast<E*>(reinterpret_cast<char*>(slot) + (size_t)blockIdx.x * gs.elem_bytes) = *stot;
#pragma unroll
      for (int k = 0; k < K; k++) rslot[blockIdx.x * 8 + k] = red[k];
    }
    sync();
    if (threadIdx.x < 32) {
      carry_warp0(slot, op, suffix, ok, scarry);
      totals_warp0<K>(rslot, maxmask, sres);
    }
    __syncthreads();
    if (!suffix) {
      if (blockIdx.x > 0) ok &= op(*scarry, ex, ex);
    } else {
      if (blockIdx.x + 1 < gridDim.x) ok &= op(ex, *scarry, ex);
    }
#pragma unroll
    for (int k = 0; k < K; k++) red[k] = sres[k];
    __syncthreads();
    phase ^= 1;
    return ex;
  }
};

// ---------------------------------------------------------------------------
// Cluster group: the CTAs of one thread-block cluster (up to 16 on GB300) work on one
// instance.  Block totals are exchanged through distributed shared memory behind the
// hardware cluster barrier (barrier.cluster arrive/wait), double-buffered by parity.
struct ClusterGroup {
  char* sm;    // block scratch (nwarps + 2 scan slots)
  char* xch;   // this CTA's exchange slots: 2 x max(element bytes, 8 doubles)
  int xbytes;  // bytes per slot
  int phase;

  __device__ int nblk() const { return (int)cooperative_groups::this_cluster().num_blocks(); }
  __device__ int brank() const { return (int)cooperative_groups::this_cluster().block_rank(); }
  __device__ int rank() const { return brank() * blockDim.x + threadIdx.x; }
  __device__ int size() const { return nblk() * blockDim.x; }
  __device__ bool dead() const { return false; }
  __device__ void sync() { cooperative_groups::this_cluster().sync(); }

  template <int K>
  __device__ void reduce(double (&v)[K], unsigned maxmask) {
    static_assert(K <= 8, "at most 8 values per reduction");
    CtaGroup cg{sm};
    cg.reduce<K>(v, maxmask);
    double* mine = reinterpret_cast<double*>(xch + (size_t)phase * xbytes);
    if (threadIdx.x == 0)
#pragma unroll
      for (int k = 0; k < K; k++) mine[k] = v[k];
    sync();
    // warp 0 reads the CTAs' values (lane i: CTA i) and combines them in an ordered
    // shuffle tree, the same in every CTA; shared memory broadcasts the result
    auto cl = cooperative_groups::this_cluster();
    const int nb = nblk();
    double* sres = reinterpret_cast<double*>(sm);
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      double a[K];
#pragma unroll
      for (int k = 0; k < K; k++)
        a[k] = lane < nb ? cl.map_shared_rank(mine, lane)[k] : (((maxmask >> k) & 1u) ? -INFINITY : 0.0);
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
        for (int k = 0; k < K; k++) {
          const double o = __shfl_down_sync(0xffffffffu, a[k], off);
          if ((lane & (2 * off - 1)) == 0) a[k] = ((maxmask >> k) & 1u) ? fmax(a[k], o) : a[k] + o;
        }
      }
      if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; k++) sres[k] = a[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = sres[k];
    __syncthreads();
    phase ^= 1;
  }

  template <class E, class Op>
  __device__ E scan(E v, const Op& op, bool suffix, bool& ok) {
    const int nw = blockDim.x >> 5;
    E* sw = reinterpret_cast<E*>(sm);
    E* stot = sw + nw;
    E* scarry = sw + nw + 1;
    E ex = block_scan_excl(v, op, suffix, ok, sw, stot);
    E* mine = reinterpret_cast<E*>(xch + (size_t)phase * xbytes);
    if (threadIdx.x == 0) *mine = *stot;
    sync();
    auto cl = cooperative_groups::this_cluster();
    const int nb = nblk(), br = brank();
    if (threadIdx.x < 32) {
      // ordered tree over the totals of the CTAs before (prefix) or after (suffix) this one
      const int lane = threadIdx.x;
      const int lo = suffix ? br + 1 : 0;
      const int hi = suffix ? nb : br;
      E acc;
      set_identity(acc);
      if (lo + lane < hi) acc = *cl.map_shared_rank(mine, lo + lane);
#pragma unroll 1
      for (int off = 1; off < 32; off <<= 1) {
        E o = shfl_down_e(acc, off);
        if ((lane & (2 * off - 1)) == 0 && lane + off < 32) ok &= op(acc, o, acc);
      }
      if (lane == 0) *scarry = acc;
    }
    __syncthreads();
    if (!suffix) {
      if (br > 0) ok &= op(*scarry, ex, ex);
    } else {
      if (br + 1 < nb) ok &= op(ex, *scarry, ex);
    }
    __syncthreads();
    phase ^= 1;
    return ex;
  }

  // scan followed by a reduction of K values (the cluster barrier is cheap: no fusion)
  template <class E, class Op, int K>
  __device__ E scan_reduce(E v, const Op& op, bool suffix, bool& ok, double (&red)[K], unsigned maxmask) {
    E r = scan(v, op, suffix, ok);
    reduce<K>(red, maxmask);
    return r;
  }
};

}  // namespace ptn
