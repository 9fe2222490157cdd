// clique_kernels.cuh -- device code of the clique level engine: the
// per-launch argument block, the 32-entry batch step (forward or reverse
// intersection of N+(w) with the parent's segment) and the persistent
// warp-per-parent / block-per-parent kernels.  Included by clique.cu (the
// engine) and by every other translation unit that launches these kernels.
#pragma once

#include "common.cuh"

namespace pgm {

enum Mode : int { kCount = 0, kWrite = 1, kSum = 2 };
constexpr int kGrab = 4;    // parents taken per queue access
constexpr int kUnroll = 4;  // loads in flight per lane in the long-list loop

struct LevelArgs {
  const void* seg;            // parent segment offsets (int32 or int64)
  int64_t seg_shift;          // subtracted from seg values -> index into vid
  const int32_t* vid;         // entries of this level
  int64_t p_lo, p_hi;         // parent range
  int64_t e_base;             // output index of an entry = (its vid index) - e_base
  const int32_t* rp;          // DAG row pointers
  const int32_t* col;         // DAG columns
  uint32_t* cnt;              // kCount: child count per entry
  const int64_t* off;         // kWrite: exclusive scan of cnt
  int64_t off_shift;          // kWrite: subtracted from off -> position in out_vid
  int32_t* out_vid;           // kWrite: next level
  unsigned long long* acc;    // kSum: total count
  unsigned long long* stat;   // neighbour-list elements read (algorithmic bytes)
  unsigned long long* queue;  // [0] warp queue, [1] block queue, [2] number of hubs
  unsigned long long* err;    // non-zero: a hub parent could not be queued
  int64_t* big;               // hub parents
  int64_t big_cap;
  int hub;                    // segment length above which a parent is a hub
  int cap;                    // per-warp staging capacity (ints)
  int block_cap;              // per-block staging capacity (ints)
  int rev_ratio;              // reverse scan when d+(w) > rev_ratio * |segment|
  const int32_t* gid;         // vertex -> graph (batches) or nullptr
  unsigned long long* per_graph;  // kSum with gid: per-graph counts
  unsigned long long* carry;      // wraps of the count accumulators (add_count)
  int grab;                       // parents a warp takes per queue access (<= 0: kGrab)
};

// Flush a per-lane count to the graph's counter (warp-wide reduction).
__device__ __forceinline__ void flush_count(const LevelArgs& A, unsigned long long& tot, int g,
                                            int lane) {
  unsigned long long s = warp_sum(tot);
  if (lane == 0 && s) add_count((A.per_graph && g >= 0) ? A.per_graph + g : A.acc, s, false, A.carry);
  tot = 0;
}

// Membership in a parent's segment: a sorted list S, plus (for short
// segments staged by the warp kernel) an open-addressing hash set H of the
// same vertices in shared memory, so that a test costs ~1.4 probes instead
// of a binary search.  Empty slots hold -1 (vertex IDs are >= 0).
constexpr int kHashCap = 512;                  // hash slots per warp
constexpr int kHashMaxSeg = kHashCap / 4;      // segments up to this length are hashed
struct SegSet {
  const int32_t* S;
  int s;
  const int32_t* H;  // nullptr: binary search in S
  uint32_t shift, mask;
  int32_t smin, smax;
  __device__ __forceinline__ bool has(int32_t x) const {
    if (x < smin || x > smax) return false;
    if (H) {
      uint32_t h = ((uint32_t)x * 0x9E3779B1u) >> shift;
      for (;;) {
        const int32_t v = H[h];
        if (v == x) return true;
        if (v < 0) return false;
        h = (h + 1) & mask;
      }
    }
    return contains_dev(S, s, x);
  }
};

// dynamic shared memory of clique_warp_kernel per block
__host__ __device__ constexpr size_t clique_warp_smem(int threads, int cap) {
  return (size_t)(threads / 32) * (size_t)(cap + kHashCap + 32) * sizeof(int32_t);
}

// Build the hash set of a staged segment (one warp); returns the SegSet.
__device__ __forceinline__ SegSet make_segset(const int32_t* S, int s, int32_t* Hbuf, int lane) {
  SegSet q;
  q.S = S;
  q.s = s;
  q.smin = S[0];
  q.smax = S[s - 1];
  q.H = nullptr;
  q.shift = 0;
  q.mask = 0;
  if (s <= kHashMaxSeg) {
    int lg = 6;  // at least 64 slots, load factor <= 1/4
    while ((1 << lg) < 4 * s) lg++;
    const int T = 1 << lg;
    for (int i = lane; i < T; i += 32) Hbuf[i] = -1;
    __syncwarp();
    const uint32_t shift = 32u - (uint32_t)lg, mask = (uint32_t)T - 1u;
    for (int i = lane; i < s; i += 32) {
      const int32_t x = S[i];
      uint32_t h = ((uint32_t)x * 0x9E3779B1u) >> shift;
      while (atomicCAS(Hbuf + h, -1, x) != -1) h = (h + 1) & mask;
    }
    __syncwarp();
    q.H = Hbuf;
    q.shift = shift;
    q.mask = mask;
  }
  return q;
}

// Process entries j0 .. j0+31 of a staged segment (Q.S, length Q.s).  e0 is
// the output index of S[0].  Children of entry j are N+(S[j]) & S, found
// either forward (scan N+(w), test membership in the segment) or in reverse
// when N+(w) is much longer than S (scan S, binary-search N+(w)); both visit
// the children in ascending ID order.  Entries whose scan is at least 32
// long are processed one at a time by the whole warp (no per-element owner
// search); the remaining short scans are flattened across the lanes.
template <int MODE>
__device__ __forceinline__ void process_batch(const SegSet& Q, int j0, int64_t e0,
                                              const LevelArgs& A, int lane, uint32_t* wcnt,
                                              unsigned long long& tot, unsigned long long& lensum) {
  const int32_t* S = Q.S;
  const int s = Q.s;
  const int j = j0 + lane;
  const bool valid = j < s;
  int32_t a0 = 0, d = 0, len = 0;
  int rev = 0;
  if (valid) {
    const int32_t w = S[j];
    a0 = A.rp[w];
    d = A.rp[w + 1] - a0;
    rev = d > A.rev_ratio * s;
    len = rev ? s : d;
  }
  lensum += (unsigned long long)d;
  int64_t my_off = 0;
  if (MODE == kWrite && valid) my_off = A.off[e0 + j] - A.off_shift;
  // long scans: the whole warp strides over one entry's list
  unsigned longm = __ballot_sync(kFull, valid && len >= 32);
  while (longm) {
    const int q = __ffs(longm) - 1;
    longm &= longm - 1;
    const int aq = __shfl_sync(kFull, a0, q);
    const int dq = __shfl_sync(kFull, d, q);
    const int revq = __shfl_sync(kFull, rev, q);
    const int lq = __shfl_sync(kFull, len, q);
    const int64_t oq = __shfl_sync(kFull, my_off, q);
    uint32_t run = 0;
    // kUnroll independent loads in flight per lane before the membership tests
    for (int base = 0; base < lq; base += 32 * kUnroll) {
      int32_t xs[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; u++) {
        const int t = base + u * 32 + lane;
        xs[u] = t < lq ? (revq ? S[t] : A.col[aq + t]) : -1;
      }
#pragma unroll
      for (int u = 0; u < kUnroll; u++) {
        const int32_t x = xs[u];
        bool hit = false;
        if (x >= 0) hit = revq ? contains_dev(A.col + aq, dq, x) : Q.has(x);
        if (MODE == kSum) {
          tot += hit ? 1ull : 0ull;
        } else {
          const unsigned b = __ballot_sync(kFull, hit);
          if (MODE == kWrite && hit) A.out_vid[oq + run + __popc(b & ((1u << lane) - 1u))] = x;
          run += __popc(b);
        }
      }
    }
    if (MODE == kCount && lane == 0) A.cnt[e0 + j0 + q] = run;
  }
  // short scans: flatten the (entry, element) pairs across the lanes
  const int slen = (valid && len < 32) ? len : 0;
  const int incl = warp_inclusive_scan(slen, lane);
  const int total = __shfl_sync(kFull, incl, 31);
  const int excl = incl - slen;
  if (MODE != kSum) {
    wcnt[lane] = 0;
    __syncwarp();
  }
  for (int base = 0; base < total; base += 32) {
    const int t = base + lane;
    const bool active = t < total;
    const int q = min(warp_owner(incl, t), 31);
    const int aq = __shfl_sync(kFull, a0, q);
    const int eq = __shfl_sync(kFull, excl, q);
    const int revq = __shfl_sync(kFull, rev, q);
    const int dq = __shfl_sync(kFull, d, q);
    bool hit = false;
    int32_t x = 0;
    if (active) {
      if (!revq) {
        x = A.col[aq + (t - eq)];
        hit = Q.has(x);
      } else {
        x = S[t - eq];
        hit = contains_dev(A.col + aq, dq, x);
      }
    }
    if (MODE == kSum) {
      tot += hit ? 1ull : 0ull;
    } else {
      const unsigned b = __ballot_sync(kFull, hit);
      const int first = max(eq - base, 0);  // first lane of owner q in this round
      const unsigned from_first = ~((1u << first) - 1u);
      const unsigned upto_me = lane == 31 ? kFull : ((2u << lane) - 1u);
      if (MODE == kWrite) {
        const int64_t oq = __shfl_sync(kFull, my_off, q);
        const uint32_t rq = wcnt[q];
        if (hit) A.out_vid[oq + rq + __popc(b & from_first & ((1u << lane) - 1u))] = x;
      }
      // the last lane of each owner's run in this round advances its count
      const int qn = __shfl_down_sync(kFull, q, 1);
      const bool last = active && (lane == 31 || t + 1 >= total || qn != q);
      __syncwarp();
      if (last) wcnt[q] += __popc(b & from_first & upto_me);
      __syncwarp();
    }
  }
  if (MODE == kCount) {
    if (valid && len < 32) A.cnt[e0 + j] = wcnt[lane];
    __syncwarp();
  }
}

template <int MODE, typename OffT>
__global__ void __launch_bounds__(512) clique_warp_kernel(LevelArgs A) {
  extern __shared__ int32_t smem[];
  const OffT* __restrict__ seg = reinterpret_cast<const OffT*>(A.seg);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t* S = smem + (int64_t)wid * (A.cap + kHashCap + 32);
  int32_t* Hbuf = S + A.cap;
  uint32_t* wcnt = reinterpret_cast<uint32_t*>(Hbuf + kHashCap);
  unsigned long long tot = 0, lensum = 0;
  int cur_g = -1;
  const int64_t np = A.p_hi - A.p_lo;
  const int grab = A.grab > 0 ? A.grab : kGrab;
  for (;;) {
    unsigned long long p0 = 0;
    if (lane == 0) p0 = atomicAdd(A.queue, (unsigned long long)grab);
    p0 = __shfl_sync(kFull, p0, 0);
    if ((int64_t)p0 >= np) break;
    const int64_t pend = min((int64_t)p0 + grab, np);
    for (int64_t pi = (int64_t)p0; pi < pend; pi++) {
      const int64_t p = A.p_lo + pi;
      const int64_t sb = (int64_t)seg[p] - A.seg_shift;
      const int64_t s = (int64_t)seg[p + 1] - A.seg_shift - sb;
      if (s < 2) continue;  // a single vertex has no partner in its own segment
      if (s > A.hub) {
        if (lane == 0) {
          unsigned long long i = atomicAdd(A.queue + 2, 1ull);
          if ((int64_t)i < A.big_cap)
            A.big[i] = p;
          else
            atomicAdd(A.err, 1ull);  // cannot happen: big_cap bounds the hub count
        }
        continue;
      }
      for (int i = lane; i < s; i += 32) S[i] = A.vid[sb + i];
      __syncwarp();
      const SegSet Q = make_segset(S, (int)s, Hbuf, lane);
      if (MODE == kSum && A.gid) {
        const int g = A.gid[S[0]];
        if (g != cur_g) {
          flush_count(A, tot, cur_g, lane);
          cur_g = g;
        }
      }
      for (int j0 = 0; j0 < s; j0 += 32) process_batch<MODE>(Q, j0, sb - A.e_base, A, lane, wcnt, tot, lensum);
      __syncwarp();
    }
  }
  if (MODE == kSum) flush_count(A, tot, cur_g, lane);
  lensum = warp_sum(lensum);
  if (lane == 0 && lensum) atomicAdd(A.stat, lensum);
}

template <int MODE, typename OffT>
__global__ void __launch_bounds__(512) clique_block_kernel(LevelArgs A) {
  extern __shared__ int32_t smem[];
  __shared__ long long sh_idx;
  const OffT* __restrict__ seg = reinterpret_cast<const OffT*>(A.seg);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int32_t* stage = smem;
  uint32_t* wcnt = reinterpret_cast<uint32_t*>(smem + A.block_cap) + wid * 32;
  unsigned long long tot = 0, lensum = 0;
  int cur_g = -1;
  const long long nbig = min((long long)A.queue[2], (long long)A.big_cap);
  for (;;) {
    if (threadIdx.x == 0) sh_idx = (long long)atomicAdd(A.queue + 1, 1ull);
    __syncthreads();
    const long long idx = sh_idx;
    __syncthreads();
    if (idx >= nbig) break;
    const int64_t p = A.big[idx];
    const int64_t sb = (int64_t)seg[p] - A.seg_shift;
    const int64_t s = (int64_t)seg[p + 1] - A.seg_shift - sb;
    const int32_t* S;
    if (s <= A.block_cap) {
      for (int64_t i = threadIdx.x; i < s; i += blockDim.x) stage[i] = A.vid[sb + i];
      S = stage;
    } else {
      S = A.vid + sb;
    }
    __syncthreads();
    SegSet Q;
    Q.S = S;
    Q.s = (int)s;
    Q.H = nullptr;
    Q.shift = Q.mask = 0;
    Q.smin = S[0];
    Q.smax = S[s - 1];
    if (MODE == kSum && A.gid) {
      const int g = A.gid[S[0]];
      if (g != cur_g) {
        flush_count(A, tot, cur_g, lane);
        cur_g = g;
      }
    }
    for (int64_t j0 = (int64_t)wid * 32; j0 < s; j0 += (int64_t)nw * 32)
      process_batch<MODE>(Q, (int)j0, sb - A.e_base, A, lane, wcnt, tot, lensum);
    __syncthreads();
  }
  if (MODE == kSum) flush_count(A, tot, cur_g, lane);
  lensum = warp_sum(lensum);
  if (lane == 0 && lensum) atomicAdd(A.stat, lensum);
}

}  // namespace pgm
