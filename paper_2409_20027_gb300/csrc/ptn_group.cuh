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

// ---------------------------------------------------------------------------
// Combinations shared by a group of G lanes (G a power of two dividing 32).  Every lane of
// the warp calls GroupOp<Op, E>::run (the groups' shuffles use the full warp), each lane of
// a group with the same two operands; each lane of the group returns the result.  The
// default is the operator itself in every lane (G = 1); value elements specialise it with
// the row-parallel form below, used where few combinations are on the critical path (the
// fold of warp totals and the carry across CTAs).
template <class Op, class E>
struct GroupOp {
  static constexpr int G = 1;
  __device__ static bool run(const Op& op, const E& a, const E& b, E& o) { return op(a, b, o); }
};

// In-place inverse of an N x N matrix by Gauss-Jordan elimination with partial pivoting
// (the same steps as inv_gj), row-parallel over the G >= N lanes of a group: lane r < N of
// the group holds row r (lanes r >= N hold unused rows).  The pivot search, row exchange
// and pivot row go through shuffles; each lane updates its own row.  Returns false in
// every lane of the group when a pivot is zero or not finite (no lane leaves early: all
// lanes of the warp take the same shuffles).
template <int N, int G, class S>
__device__ bool inv_gj_rows(S (&row)[N]) {
  static_assert(G >= N && G <= 32 && (G & (G - 1)) == 0, "group of G >= N lanes, G a power of two");
  const int lane = threadIdx.x & 31, r = lane & (G - 1), base = lane - r;
  bool ok = true;
  int perm[N];
#pragma unroll
  for (int i = 0; i < N; i++) perm[i] = i;
#pragma unroll
  for (int k = 0; k < N; k++) {
    // pivot: largest magnitude in column k among rows k..N-1 (smallest row on ties)
    const bool cand = r >= k && r < N;
    unsigned key = cand ? mag_key(row[k]) : 0u;
    int idx = cand ? r : G;
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
      const unsigned ok2 = __shfl_xor_sync(PTN_FULL, key, off);
      const int oi = __shfl_xor_sync(PTN_FULL, idx, off);
      if (ok2 > key || (ok2 == key && oi < idx)) { key = ok2; idx = oi; }
    }
    const int p = idx < N ? idx : k;
    // exchange rows k and p
    const int src = (r == k) ? p : (r == p ? k : r);
#pragma unroll
    for (int j = 0; j < N; j++) row[j] = __shfl_sync(PTN_FULL, row[j], base + src);
#pragma unroll
    for (int i = k + 1; i < N; i++)
      if (i == p) { const int t = perm[k]; perm[k] = perm[i]; perm[i] = t; }
    // the pivot row, scaled by 1 / pivot; then every other row eliminated with it
    S pk[N];
#pragma unroll
    for (int j = 0; j < N; j++) pk[j] = __shfl_sync(PTN_FULL, row[j], base + k);
    const S pv = pk[k];
    const bool good = pivot_ok(pv);
    ok &= good;
    const S ip = good ? pivot_rcp(pv) : S(0);
    pk[k] = S(1);
#pragma unroll
    for (int j = 0; j < N; j++) pk[j] *= ip;
    if (r == k) {
#pragma unroll
      for (int j = 0; j < N; j++) row[j] = pk[j];
    } else {
      const S f = row[k];
      row[k] = S(0);
#pragma unroll
      for (int j = 0; j < N; j++) row[j] -= f * pk[j];
    }
  }
  // undo the row permutation as a column permutation of the inverse
  S out[N];
#pragma unroll
  for (int j = 0; j < N; j++) {
    S v = S(0);
#pragma unroll
    for (int jj = 0; jj < N; jj++)
      if (perm[jj] == j) v = row[jj];
    out[j] = v;
  }
#pragma unroll
  for (int j = 0; j < N; j++) row[j] = out[j];
  return ok;
}

// Value operator (eq. value-fun-param) with the FP64 inverse of I + C1 J2 shared by the G
// lanes of a group (inv_gj_rows; the group's lanes hold the same operands); the products
// of value_apply_K in every lane.  Same formulas and precisions as ValueOp.
template <class SV, int G, int N, class L>
__device__ bool value_combine_rows(const Val<N, L>& e1, const Val<N, L>& e2, Val<N, L>& o) {
  const int lane = threadIdx.x & 31, r = lane & (G - 1), base = lane - r;
  L Ml[N * N];
  mm<N, N, N>(e1.C, e2.J, Ml);
  SV row[N];
#pragma unroll
  for (int j = 0; j < N; j++) {
    L v = L(0);
#pragma unroll
    for (int i = 0; i < N; i++)
      if (i == r) v = Ml[i * N + j];
    row[j] = cvt_solve<SV>(v) + (r == j ? SV(1) : SV(0));
  }
  const bool ok = inv_gj_rows<N, G, SV>(row);
  L rl[N], K[N * N];
#pragma unroll
  for (int j = 0; j < N; j++) rl[j] = cvt_solve<L>(row[j]);
#pragma unroll
  for (int i = 0; i < N; i++)
#pragma unroll
    for (int j = 0; j < N; j++) K[i * N + j] = __shfl_sync(PTN_FULL, rl[j], base + i);
  value_apply_K<N, L>(e1, e2, K, o);
  return ok;
}

// Inclusive prefix (suffix) scan of the nw warp totals in buf[0 .. nw), in time order, in
// place: buf[w] becomes the combination of totals 0..w (w..nw-1).  By the lane groups of
// the calling warp (all its lanes): Kogge-Stone over buf[0 .. nw) and buf[nw .. 2 nw).
template <class E, class Op>
__device__ void warp_totals_scan_groups(const Op& op, bool suffix, bool& ok, E* buf, int nw) {
  using GO = GroupOp<Op, E>;
  constexpr int G = GO::G;
  const int lane = threadIdx.x & 31, gi = lane / G, ng = 32 / G;
  E* cur = buf;
  E* nxt = buf + nw;
#pragma unroll 1
  for (int off = 1; off < nw; off <<= 1) {
#pragma unroll 1
    for (int i0 = 0; i0 < nw; i0 += ng) {  // the same trip count in every lane
      const int i = i0 + gi;
      const int o = suffix ? i + off : i - off;
      const bool act = i < nw;
      const bool comb = act && o >= 0 && o < nw;
      const int ia = comb ? (suffix ? i : o) : 0, ib = comb ? (suffix ? o : i) : 0;
      E a = cur[ia], b = cur[ib], res;
      const bool okc = GO::run(op, a, b, res);
      if (comb) ok &= okc;
      if (act && (lane & (G - 1)) == 0) nxt[i] = comb ? res : cur[i];
    }
    __syncwarp();
    E* t = cur; cur = nxt; nxt = t;
  }
  if (cur != buf) {
    for (int i = lane / G; i < nw; i += ng)
      if ((lane & (G - 1)) == 0) buf[i] = cur[i];
    __syncwarp();
  }
}

// The combination, in time order, of the elements [lo, hi) that load(b, e) reads (the other
// CTAs' totals), by all lane groups of the block: group g folds its contiguous range, then a
// tree over the groups through tree[0 .. ngroups) and the flags hv[0 .. ngroups).  The
// result is in *out (shared memory) after the final block barrier.  Needs hi > lo; every
// thread of the block calls it.
template <class E, class Op, class Load>
__device__ void block_fold_groups(const Op& op, bool& ok, int lo, int hi, const Load& load, E* tree, int* hv,
                                  E* out) {
  using GO = GroupOp<Op, E>;
  constexpr int G = GO::G;
  const int lane = threadIdx.x & 31, gi = threadIdx.x / G, ngr = blockDim.x / G;
  const bool lead = (lane & (G - 1)) == 0;
  const int cnt = hi - lo;
  const int used = cnt < ngr ? cnt : ngr;
  const int per = (cnt + ngr - 1) / ngr;
  // the group's first element starts its fold; the rest are combined into it
  E acc;
  bool have = lo + gi * per < hi && gi < used;
  if (have) load(lo + gi * per, acc);
  else set_identity(acc);
#pragma unroll 1
  for (int k = 1; k < per; k++) {  // the same trip count in every lane
    const int b = lo + gi * per + k;
    const bool valid = b < hi && gi < used;
    E t;
    if (valid) load(b, t);
    else set_identity(t);
    E res;
    const bool okc = GO::run(op, acc, t, res);
    if (valid) { acc = res; ok &= okc; }
  }
  if (lead && gi < ngr) {
    tree[gi] = acc;
    hv[gi] = have ? 1 : 0;
  }
  __syncthreads();
#pragma unroll 1
  for (int off = 1; off < used; off <<= 1) {
    const bool act = (gi % (2 * off)) == 0 && gi + off < used;
    const int pb = act ? gi + off : gi;
    E a = tree[gi], b = tree[pb], res;
    const bool ha = hv[gi] != 0, hb = act && hv[pb] != 0;
    const bool okc = GO::run(op, a, b, res);
    __syncthreads();
    if (act && hb) {
      if (ha) ok &= okc;
      if (lead) {
        tree[gi] = ha ? res : b;
        hv[gi] = 1;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = tree[0];
  __syncthreads();
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

// Block part of a scan for operators with a group form (GroupOp<Op, E>::G > 1): the warp
// Kogge-Stone of block_scan_excl, then the inclusive scan of the warp totals by the lane
// groups of warp 0.  Returns this thread's exclusive combination within its warp; has_ex
// is false (and the result the identity) for the warp's first element in scan order.  On
// return (after a block barrier) sw[w] holds the combination of the totals of warps 0..w
// (prefix) or w..nw-1 (suffix); sw[nw .. 2 nw) is scratch.
template <class E, class Op>
__device__ E block_scan_groups(E v, const Op& op, bool suffix, bool& ok, E* sw, bool& has_ex) {
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
  has_ex = suffix ? lane != 31 : lane != 0;
  if (!has_ex) set_identity(ex);
  __syncthreads();
  if ((!suffix && lane == 31) || (suffix && lane == 0)) sw[w] = v;
  __syncthreads();
  if (w == 0) warp_totals_scan_groups(op, suffix, ok, sw, nw);
  __syncthreads();
  return ex;
}

// this thread's exclusive result from its warp-exclusive part ex (has_ex) and the
// combination W of everything before (prefix) / after (suffix) its warp (has_w)
template <class E, class Op>
__device__ __forceinline__ void apply_outer(E& ex, bool has_ex, const E& W, const Op& op, bool suffix, bool& ok) {
  if (has_ex) ok &= suffix ? op(ex, W, ex) : op(W, ex, ex);
  else ex = W;
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
    if constexpr (GroupOp<Op, E>::G > 1) {
      E* sw = reinterpret_cast<E*>(sm);
      const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
      bool has_ex;
      E ex = block_scan_groups(v, op, suffix, ok, sw, has_ex);
      if (suffix ? w < nw - 1 : w > 0) apply_outer(ex, has_ex, sw[suffix ? w + 1 : w - 1], op, suffix, ok);
      __syncthreads();
      return ex;
    } else {
      return block_scan_excl(v, op, suffix, ok, reinterpret_cast<E*>(sm), (E*)nullptr);
    }
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

// count: the CTAs that take part (all of the launch, or the CTA range of one instance
// with its own counters)
__device__ __forceinline__ bool grid_barrier(const GridScratch& gs, unsigned count) {
  volatile unsigned* gen = gs.bar + 1;
  const unsigned g0 = *gen;
  __threadfence();
  const unsigned arrived = atomicAdd(gs.bar, 1u);
  if (arrived == count - 1) {
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
      if (!grid_barrier(gs, gridDim.x)) *sdead = 1;
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
    if constexpr (GroupOp<Op, E>::G > 1) return scan_groups(v, op, suffix, ok);
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

  // scan for operators with a group form: warp totals scanned by lane groups, the block
  // total published, then the carry over the other blocks' totals folded by all lane groups
  // of the block, merged with this warp's part by one group combination, and applied with
  // one combination per thread.  Scratch: 2 nwarps + 1 + (block / G) elements and
  // (block / G) ints (scan_group_scratch).
  template <class E, class Op>
  __device__ E scan_groups(E v, const Op& op, bool suffix, bool& ok) {
    using GO = GroupOp<Op, E>;
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5, ngr = blockDim.x / GO::G;
    E* sw = reinterpret_cast<E*>(sm);
    E* scarry = sw + 2 * nw;
    E* tree = scarry + 1;
    int* hv = reinterpret_cast<int*>(tree + ngr);
    bool has_ex;
    E ex = block_scan_groups(v, op, suffix, ok, sw, has_ex);
    char* slot = gs.xs + (size_t)phase * gridDim.x * gs.elem_bytes;
    if (threadIdx.x == 0) *reinterpret_cast<E*>(slot + (size_t)blockIdx.x * gs.elem_bytes) = sw[suffix ? 0 : nw - 1];
    sync();
    const bool has_c = suffix ? blockIdx.x + 1 < gridDim.x : blockIdx.x > 0;
    if (has_c) {
      auto load = [&](int b, E& t) {
        const unsigned* s4 = reinterpret_cast<const unsigned*>(slot + (size_t)b * gs.elem_bytes);
        unsigned* d4 = reinterpret_cast<unsigned*>(&t);
#pragma unroll
        for (int i = 0; i < (int)(sizeof(E) / 4); i++) d4[i] = __ldcg(s4 + i);
      };
      block_fold_groups<E>(op, ok, suffix ? (int)blockIdx.x + 1 : 0, suffix ? (int)gridDim.x : (int)blockIdx.x, load,
                           tree, hv, scarry);
    }
    const bool has_w = suffix ? w < nw - 1 : w > 0;
    if (has_w && has_c) {
      E W;
      if (suffix) ok &= GO::run(op, sw[w + 1], *scarry, W);
      else ok &= GO::run(op, *scarry, sw[w - 1], W);
      apply_outer(ex, has_ex, W, op, suffix, ok);
    } else if (has_w || has_c) {
      apply_outer(ex, has_ex, has_w ? sw[suffix ? w + 1 : w - 1] : *scarry, op, suffix, ok);
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
    if constexpr (GroupOp<Op, E>::G > 1) return scan_groups(v, op, suffix, ok);
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

  // scan for operators with a group form, as GridGroup::scan_groups with the block totals
  // in the CTAs' exchange slots (distributed shared memory) behind the cluster barrier
  template <class E, class Op>
  __device__ E scan_groups(E v, const Op& op, bool suffix, bool& ok) {
    using GO = GroupOp<Op, E>;
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5, ngr = blockDim.x / GO::G;
    E* sw = reinterpret_cast<E*>(sm);
    E* scarry = sw + 2 * nw;
    E* tree = scarry + 1;
    int* hv = reinterpret_cast<int*>(tree + ngr);
    bool has_ex;
    E ex = block_scan_groups(v, op, suffix, ok, sw, has_ex);
    E* mine = reinterpret_cast<E*>(xch + (size_t)phase * xbytes);
    if (threadIdx.x == 0) *mine = sw[suffix ? 0 : nw - 1];
    sync();
    auto cl = cooperative_groups::this_cluster();
    const int nb = nblk(), br = brank();
    const bool has_c = suffix ? br + 1 < nb : br > 0;
    if (has_c) {
      auto load = [&](int b, E& t) { t = *cl.map_shared_rank(mine, b); };
      block_fold_groups<E>(op, ok, suffix ? br + 1 : 0, suffix ? nb : br, load, tree, hv, scarry);
    }
    const bool has_w = suffix ? w < nw - 1 : w > 0;
    if (has_w && has_c) {
      E W;
      if (suffix) ok &= GO::run(op, sw[w + 1], *scarry, W);
      else ok &= GO::run(op, *scarry, sw[w - 1], W);
      apply_outer(ex, has_ex, W, op, suffix, ok);
    } else if (has_w || has_c) {
      apply_outer(ex, has_ex, has_w ? sw[suffix ? w + 1 : w - 1] : *scarry, op, suffix, ok);
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

// shared scratch of the group-form scans: 2 nwarps + 1 + ngroups elements and ngroups ints
template <class E, int G>
__host__ __device__ constexpr size_t scan_group_scratch(int nthreads) {
  return (size_t)(2 * (nthreads / 32) + 1 + nthreads / G) * sizeof(E) + (size_t)(nthreads / G) * sizeof(int);
}

}  // namespace ptn
