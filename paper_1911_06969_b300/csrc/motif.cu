// motif.cu -- vertex-induced 3- and 4-motif counting (Sec. 3.3 Listing 4,
// Sec. 4.2 memoization and customised pattern classification).
//
// Embeddings grow by a neighbour of ANY vertex (Sec. 3.1, Algorithm 2), and a
// canonical test keeps one copy of every connected vertex set (Sec. 3.2).
// The paper does not print its canonical rule; this build uses the
// breadth-first canonical order: v0 = min(S), and each next vertex is the
// unused vertex adjacent to the prefix with the smallest key (f(u), u), where
// f(u) is the index of u's first neighbour in the prefix.  Keys of a
// canonical sequence are strictly increasing, so appending u to a canonical
// prefix (v0..v_{i-1}) is canonical iff u > v0 and either f(u) = i-1 or
// (f(v_{i-1}), v_{i-1}) < (f(u), u).
//
// Level 2: edges (v0, v1), v0 < v1, grouped by v0: segment A(v0) = the
// neighbours of v0 above v0.  Level 3 children of (v0, v1):
//   f2 = 0: u in N(v0), u > v1                    (u adjacent to v0)
//   f2 = 1: u in N(v1), u > v0, u not in N(v0)    (u adjacent to v1 only)
// stored as vid | a02 << 30 | a12 << 31 (memoised pattern of the 3-vertex
// embedding: a02 = v2~v0, a12 = v2~v1; Sec. 4.2 memoization).
// 3-motif pattern: triangle iff a02 & a12 (Listing 6), else wedge.
//
// Last level (fused count, never materialised): for a 3-embedding
// (v0, v1, v2) the 4th vertex w > v0 with adjacency mask M = (w~v0, w~v1,
// w~v2) is accepted by the canonical test iff
//   f2 = 0: M has bit 0 -> w > v2;  otherwise -> always;
//   f2 = 1: M has bit 0 -> never;   M in {2, 6} -> w > v2;  M = 4 -> always.
// The pattern follows from (a02, a12, M): edge count and maximum degree
// (customised classification, Listing 6 extended to 4 vertices):
//   3 edges: 3-star (max degree 3) or 4-path; 4 edges: tailed triangle
//   (max degree 3) or 4-cycle; 5: diamond; 6: 4-clique.
// The reduce needs only the number of accepted candidates per region, so
// with A = N(v0) & (v0, inf), B = N(v1) & (v0, inf) and I = A & B:
// candidates adjacent only to v0 and/or v1 are counted by rank queries on
// A, B and I; those adjacent to v2 come from |N(v2) & (v0, inf)|, from the
// triangle counts of arc (v0, v2) memoised by the level-3 inspection (f2 =
// 0), and from the common neighbours of v1 and v2 above v0, which are
// enumerated -- from B's side for edges with many f2 = 0 children
// (motif_l3_pairs), from N(v2) otherwise -- and looked up in A and B (hub
// bitmaps, filters, binary search, Sec. 5.4).  f2 = 1 children scan N(v2)
// & (v0, inf) against A and B.
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace pgm {

namespace {

enum MMode : int { mCount = 0, mWrite = 1, mSum = 2 };
constexpr int kMGrab = 2;
constexpr int kEdgeGrab = 4;
constexpr uint32_t kVidMask = (1u << 30) - 1u;
constexpr uint32_t kA02 = 1u << 30;
constexpr uint32_t kA12 = 1u << 31;

struct MotifArgs {
  const int32_t* rp;   // undirected CSR
  const int32_t* col;
  const int32_t* up;   // up[v] = first arc of v whose neighbour is > v
  int32_t v_lo, v_hi;  // parent (v0) range
  int64_t a_base;      // arc index that maps to entry 0 (entries are arcs)
  uint32_t* cnt;       // mCount: children per arc (index a - a_base)
  const int64_t* off;  // mWrite / level 3: exclusive scan of cnt
  int64_t off_shift;   // subtracted from off -> index into l3
  uint32_t* l3;        // mWrite output / level-3 input
  unsigned long long* acc;        // pattern counts (2 or 6)
  unsigned long long* per_graph;  // per-graph counts (batches) or nullptr
  const int32_t* gid;
  unsigned long long* stat;   // elements examined (algorithmic bytes)
  unsigned long long* queue;  // [0] warp queue [1] block queue [2] hub count
  unsigned long long* err;    // non-zero: a hub vertex could not be queued
  int32_t* big;
  int64_t big_cap;
  int cap;        // per-warp staging capacity (ints) per list
  int block_cap;  // per-block staging capacity for A
  int32_t* scratch;  // per-warp global scratch, scratch_stride ints each
  int64_t scratch_stride;
  // level 3
  const int32_t* src;       // src[a] = source vertex of arc a
  int64_t arc_lo, arc_hi;   // arcs of this chunk (absolute)
  const int32_t* hub_idx;   // vertex -> hub bitmap row or -1
  const uint32_t* hub_bits; // adjacency bitmaps of hub vertices
  int64_t hub_words;        // words per bitmap row
  uint32_t* hubctr;         // level 2, counting modes: next 32-entry batch of each hub vertex
  const int32_t* rev;       // rev[a] = index of the reverse arc of arc a
  // per arc a = (v0, v1), v1 > v0 (index a - a_base): |N(v1) & A(v0)| and
  // |N(v1) & A(v0) & (v1, inf)| (triangles on the arc above v0 / above v1),
  // written by the level-3 inspection, read by the last level (memoised
  // per level-2 edge, Sec. 4.2, instead of recomputed per level-3 entry)
  uint2* tri;
  // exclusive prefix sums over the same arcs of tri.y and of (|N(v2) above
  // v0| - tri.x) for arcs above v0 (0 elsewhere): the base region sizes of
  // all f2 = 0 children of an edge in O(1) (motif_l3_edge)
  const int64_t* py;
  const int64_t* pz;
  unsigned long long* carry;  // wraps of the count accumulators (add_count)
  int b_side_min;  // last level: edges with at least this many f2 = 0 children are counted
  // whole by motif_l3_pairs, from B's side; none of their children is stored
  // in the level-3 list, and the inspection adds their number here
  unsigned long long* skipped;
  // lengths for the checked index sites (PGM_DEBUG builds)
  int64_t narcs;        // col, rev, src
  int64_t n_arc_slots;  // cnt, tri (arcs of the launch's vertex range)
  int64_t n_l3;         // l3 entries of the chunk
  int grab;             // level 2: vertices a warp takes per queue access (<= 0: kMGrab)
};

template <int N>
__device__ __forceinline__ void flush_patterns(const MotifArgs& P, long long (&c)[N], int g,
                                               int lane) {
#pragma unroll
  for (int i = 0; i < N; i++) {
    long long s = warp_sum(c[i]);
    if (lane == 0 && s) {
      unsigned long long* dst = (P.per_graph && g >= 0) ? P.per_graph + (int64_t)g * N : P.acc;
      add_count(dst + i, (unsigned long long)s, true, P.carry);  // corrections make partials signed
    }
    c[i] = 0;
  }
}

// Membership of w in a sorted list, or by one bit of a hub's adjacency
// bitmap when the list's owner is a hub (hb >= 0).  Callers only ask about
// w above the list's lower threshold, so the bitmap of the full adjacency
// list answers for the thresholded list too.
__device__ __forceinline__ bool member(const int32_t* L, int len, int hb, const MotifArgs& P, int32_t w) {
  if (hb >= 0) return (P.hub_bits[(int64_t)hb * P.hub_words + (w >> 5)] >> (w & 31)) & 1u;
  return len > 0 && w >= L[0] && w <= L[len - 1] && contains_dev(L, len, w);
}

// ------------------------------------------------------ level 2 -> 3 / 3-motif
// Entries j0..j0+31 of v0's segment A (length s).  For entry j (v1 = A[j])
// scan N(v1): x > v0 and not in A -> f2=1 child; x in A and x > v1 -> the
// f2=0 child x is a triangle (a12 = 1).  Membership in A comes from v0's hub
// bitmap when it has one (hA >= 0: A = N(v0) above v0), the binary search
// then only placing the triangles.
template <int MODE>
__device__ __forceinline__ void l2_batch(const MotifArgs& P, const int32_t* A, int s, int hA, int j0,
                                         int32_t v0, int64_t arc0, int lane, uint32_t* wcnt,
                                         long long (&c)[2], unsigned long long& seen) {
  const int j = j0 + lane;
  const bool valid = j < s;
  int32_t v1 = 0, a0 = 0, len = 0;
  if (valid) {
    v1 = A[j];
    a0 = P.rp[v1];
    len = P.rp[v1 + 1] - a0;
  }
  seen += (unsigned long long)len;
  const int incl = warp_inclusive_scan(len, lane);
  const int total = __shfl_sync(kFull, incl, 31);
  const int excl = incl - len;
  int64_t my_off = 0;
  if (MODE == mSum && valid) c[0] += s - j - 1;  // f2 = 0 children start as wedges
  if (MODE != mSum) {
    wcnt[lane] = 0;
    if (MODE == mWrite && valid) my_off = P.off[arc0 + j] - P.off_shift;
    __syncwarp();
  }
  if (MODE == mWrite) {
    // phase 1: the f2 = 0 block A[j+1..s) with a02 = 1, a12 = 0
    for (int q = 0; q < 32; q++) {
      const int jq = j0 + q;
      if (jq >= s) break;
      const int64_t oq = __shfl_sync(kFull, my_off, q);
      if (s - jq - 1 >= P.b_side_min) continue;  // not stored (see b_side_min)
      for (int i = jq + 1 + lane; i < s; i += 32)
        if (PGM_IDX_OK(oq + (i - jq - 1), P.n_l3)) P.l3[oq + (i - jq - 1)] = (uint32_t)A[i] | kA02;
    }
    __syncwarp();
  }
  const int32_t amin = A[0], amax = A[s - 1];
  for (int base = 0; base < total; base += 32) {
    const int t = base + lane;
    const bool active = t < total;
    const int q = min(warp_owner(incl, t), 31);
    const int aq = __shfl_sync(kFull, a0, q);
    const int eq = __shfl_sync(kFull, excl, q);
    const int32_t v1q = __shfl_sync(kFull, v1, q);
    bool child = false, tri = false;
    int32_t x = 0;
    int xi = 0;
    if (active) {
      x = P.col[aq + (t - eq)];
      if (x > v0) {
        bool inA = false;
        if (x >= amin && x <= amax) {
          if (hA >= 0) {
            inA = member(A, s, hA, P, x);
          } else {
            xi = lower_bound_dev(A, s, x);
            inA = xi < s && A[xi] == x;
          }
        }
        child = !inA;
        tri = inA && x > v1q;
        if (MODE == mWrite && tri && hA >= 0) xi = lower_bound_dev(A, s, x);
      }
    }
    if (MODE == mSum) {
      c[0] += (child ? 1 : 0) - (tri ? 1 : 0);
      c[1] += tri ? 1 : 0;
    } else {
      const unsigned b = __ballot_sync(kFull, child);
      const int first = max(eq - base, 0);
      const unsigned from_first = ~((1u << first) - 1u);
      const unsigned upto_me = lane == 31 ? kFull : ((2u << lane) - 1u);
      if (MODE == mWrite) {
        const int64_t oq = __shfl_sync(kFull, my_off, q);
        const int jq = j0 + q;
        const uint32_t rq = wcnt[q];
        const bool fbq = s - jq - 1 >= P.b_side_min;  // this edge's f2 = 0 block is not stored
        const int64_t ic = oq + (fbq ? 0 : s - jq - 1) + rq + __popc(b & from_first & ((1u << lane) - 1u));
        if (child && !fbq && PGM_IDX_OK(ic, P.n_l3)) P.l3[ic] = (uint32_t)x | kA12;
        if (tri && !fbq && PGM_IDX_OK(oq + (xi - jq - 1), P.n_l3))
          P.l3[oq + (xi - jq - 1)] = (uint32_t)x | kA02 | kA12;
      }
      const int qn = __shfl_down_sync(kFull, q, 1);
      const bool last = active && (lane == 31 || t + 1 >= total || qn != q);
      __syncwarp();
      if (last) wcnt[q] += __popc(b & from_first & upto_me);
      __syncwarp();
    }
  }
  if (MODE == mCount) {
    if (valid) P.cnt[arc0 + j] = wcnt[lane] + (uint32_t)(s - j - 1);
    __syncwarp();
  }
}

// Counting modes (3-motif sum, level-3 inspection) need only the sizes of
// the intersections of A (v0's segment) with B_j = N(A[j]) & (v0, inf):
// for entry j (v1 = A[j]) the children are the f2=0 block A[j+1..s) and the
// f2=1 block B_j \ A; among the f2=0 children, those in B_j (above v1) are
// triangles.  Each intersection scans the shorter of A and B_j and tests its
// elements in the other (staged list, hub bitmap or binary search).
template <int MODE>
__device__ __forceinline__ void l2_count_batch(const MotifArgs& P, const int32_t* A, int s, int hA, int j0,
                                               int32_t v0, int64_t arc0, int lane, uint32_t* wcnt,
                                               long long (&c)[2], unsigned long long& seen) {
  const int j = j0 + lane;
  const bool valid = j < s;
  int32_t v1 = 0, r1 = 0, d1 = 0, b0 = 0, nbj = 0, len = 0, hv1 = -1, scanB = 0;
  if (valid) {
    v1 = A[j];
    r1 = P.rp[v1];
    d1 = P.rp[v1 + 1] - r1;
    // N(v1) & (v0, inf) starts after v0's own entry in N(v1) (the reverse arc)
    const int bs = P.rev[P.a_base + arc0 + j] - r1 + 1;
    b0 = r1 + bs;
    nbj = d1 - bs;
    hv1 = P.hub_idx[v1];
    scanB = nbj <= s;
    len = scanB ? nbj : s;
  }
  seen += (unsigned long long)len;
  if (MODE == mSum && valid) c[0] += (long long)(s - j - 1) + nbj;  // all children start as wedges
  const int incl = warp_inclusive_scan(len, lane);
  const int total = __shfl_sync(kFull, incl, 31);
  const int excl = incl - len;
  if (MODE == mCount) {
    wcnt[lane] = 0;
    wcnt[32 + lane] = 0;
    __syncwarp();
  }
  for (int base = 0; base < total; base += 32) {
    const int t = base + lane;
    const bool active = t < total;
    const int q = min(warp_owner(incl, t), 31);
    const int eq = __shfl_sync(kFull, excl, q);
    const int sq = __shfl_sync(kFull, scanB, q);
    const int32_t b0q = __shfl_sync(kFull, b0, q);
    const int32_t r1q = __shfl_sync(kFull, r1, q);
    const int d1q = __shfl_sync(kFull, d1, q);
    const int hq = __shfl_sync(kFull, hv1, q);
    const int32_t v1q = __shfl_sync(kFull, v1, q);
    bool in = false;
    int32_t x = 0;
    if (active) {
      const int idx = t - eq;
      if (sq) {
        x = P.col[b0q + idx];
        in = member(A, s, hA, P, x);
      } else {
        x = A[idx];
        in = member(P.col + r1q, d1q, hq, P, x);
      }
    }
    if (MODE == mSum) {
      if (in) {
        c[0] -= 1;  // in A: not an f2=1 child
        if (x > v1q) {
          c[0] -= 1;  // the f2=0 child x is a triangle
          c[1] += 1;
        }
      }
    } else {
      const unsigned b = __ballot_sync(kFull, in);
      const unsigned bg = __ballot_sync(kFull, in && x > v1q);
      const int first = max(eq - base, 0);
      const unsigned from_first = ~((1u << first) - 1u);
      const unsigned upto_me = lane == 31 ? kFull : ((2u << lane) - 1u);
      const int qn = __shfl_down_sync(kFull, q, 1);
      const bool last = active && (lane == 31 || t + 1 >= total || qn != q);
      __syncwarp();
      if (last) {
        wcnt[q] += __popc(b & from_first & upto_me);
        wcnt[32 + q] += __popc(bg & from_first & upto_me);
      }
      __syncwarp();
    }
  }
  if (MODE == mCount) {
    const bool fb = valid && s - j - 1 >= P.b_side_min;  // children not stored (see b_side_min)
    const uint32_t nch = valid ? (uint32_t)(s - j - 1) + (uint32_t)nbj - wcnt[lane] : 0u;
    if (valid && PGM_IDX_OK(arc0 + j, P.n_arc_slots)) {
      P.cnt[arc0 + j] = fb ? 0u : nch;
      P.tri[arc0 + j] = make_uint2(wcnt[lane], wcnt[32 + lane]);
    }
    const unsigned long long sk = warp_sum((unsigned long long)(fb ? nch : 0u));
    if (lane == 0 && sk) atomicAdd(P.skipped, sk);
    __syncwarp();
  }
}

// Level-2 batch: counting modes by intersection sizes, the write mode by a
// full scan of each B_j (it writes the children).
template <int MODE>
__device__ __forceinline__ void l2_any_batch(const MotifArgs& P, const int32_t* A, int s, int hA, int j0,
                                             int32_t v0, int64_t arc0, int lane, uint32_t* wcnt,
                                             long long (&c)[2], unsigned long long& seen) {
  if (MODE == mWrite)
    l2_batch<MODE>(P, A, s, hA, j0, v0, arc0, lane, wcnt, c, seen);
  else
    l2_count_batch<MODE>(P, A, s, hA, j0, v0, arc0, lane, wcnt, c, seen);
}

template <int MODE>
__global__ void __launch_bounds__(512, 2) motif_l2_warp(MotifArgs P) {
  extern __shared__ int32_t smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t* A = smem + wid * (P.cap + 64);
  uint32_t* wcnt = reinterpret_cast<uint32_t*>(A + P.cap);  // 64 counters
  long long c[2] = {0, 0};
  unsigned long long seen = 0;
  int cur_g = -1;
  const int64_t np = (int64_t)P.v_hi - P.v_lo;
  const int grab = P.grab > 0 ? P.grab : kMGrab;
  for (;;) {
    unsigned long long p0 = 0;
    if (lane == 0) p0 = atomicAdd(P.queue, (unsigned long long)grab);
    p0 = __shfl_sync(kFull, p0, 0);
    if ((int64_t)p0 >= np) break;
    const int64_t pend = min((int64_t)p0 + grab, np);
    for (int64_t pi = (int64_t)p0; pi < pend; pi++) {
      const int32_t v0 = (int32_t)(P.v_lo + pi);
      const int32_t u0 = P.up[v0], u1 = P.rp[v0 + 1];
      const int s = u1 - u0;
      if (s < 1) continue;
      if (s > P.cap) {
        if (lane == 0) {
          unsigned long long i = atomicAdd(P.queue + 2, 1ull);
          if ((int64_t)i < P.big_cap)
            P.big[i] = v0;
          else
            atomicAdd(P.err, 1ull);  // cannot happen: every vertex fits
        }
        continue;
      }
      for (int i = lane; i < s; i += 32) A[i] = P.col[u0 + i];
      __syncwarp();
      if (MODE == mSum && P.gid) {
        const int g = P.gid[v0];
        if (g != cur_g) {
          flush_patterns<2>(P, c, cur_g, lane);
          cur_g = g;
        }
      }
      const int64_t arc0 = (int64_t)u0 - P.a_base;
      const int hA = P.hub_idx[v0];
      for (int j0 = 0; j0 < s; j0 += 32) l2_any_batch<MODE>(P, A, s, hA, j0, v0, arc0, lane, wcnt, c, seen);
      __syncwarp();
    }
  }
  if (MODE == mSum) flush_patterns<2>(P, c, cur_g, lane);
  seen = warp_sum(seen);
  if (lane == 0 && seen) atomicAdd(P.stat, seen);
}

// Counting modes: the segments of the hub vertices (deferred by the warp
// kernel) in batches of 32 entries, taken by any warp from a per-hub
// counter, with A read in place (hub bitmap for membership) -- no block
// barrier, so a long batch delays no other warp.  Warps move through the
// hub list in order; `hint` (queue[3]) is the first hub not known to be
// exhausted.
template <int MODE>
__global__ void __launch_bounds__(256) motif_l2_hubs(MotifArgs P) {
  __shared__ uint32_t wcnt_all[8][64];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t* wcnt = wcnt_all[wid];
  long long c[2] = {0, 0};
  unsigned long long seen = 0;
  int cur_g = -1;
  const long long nbig = min((long long)P.queue[2], (long long)P.big_cap);
  unsigned long long* hint = P.queue + 3;
  long long i = 0;
  if (lane == 0) i = (long long)atomicAdd(hint, 0ull);
  i = __shfl_sync(kFull, i, 0);
  while (i < nbig) {
    const int32_t v0 = P.big[i];
    const int32_t u0 = P.up[v0];
    const int s = P.rp[v0 + 1] - u0;
    unsigned b = 0;
    if (lane == 0) b = atomicAdd(P.hubctr + i, 1u);
    b = __shfl_sync(kFull, b, 0);
    if ((long long)b * 32 >= s) {  // hub i exhausted: move on
      unsigned long long h = 0;
      if (lane == 0) h = atomicMax(hint, (unsigned long long)(i + 1));
      h = __shfl_sync(kFull, h, 0);
      i = max(i + 1, (long long)h);
      continue;
    }
    if (MODE == mSum && P.gid) {
      const int g = P.gid[v0];
      if (g != cur_g) {
        flush_patterns<2>(P, c, cur_g, lane);
        cur_g = g;
      }
    }
    const int64_t arc0 = (int64_t)u0 - P.a_base;
    l2_count_batch<MODE>(P, P.col + u0, s, P.hub_idx[v0], (int)b * 32, v0, arc0, lane, wcnt, c, seen);
  }
  if (MODE == mSum) flush_patterns<2>(P, c, cur_g, lane);
  seen = warp_sum(seen);
  if (lane == 0 && seen) atomicAdd(P.stat, seen);
}

template <int MODE>
__global__ void __launch_bounds__(512, 2) motif_l2_block(MotifArgs P) {
  extern __shared__ int32_t smem[];
  __shared__ long long sh_idx;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int32_t* stage = smem;
  uint32_t* wcnt = reinterpret_cast<uint32_t*>(smem + P.block_cap) + wid * 64;
  long long c[2] = {0, 0};
  unsigned long long seen = 0;
  int cur_g = -1;
  const long long nbig = min((long long)P.queue[2], (long long)P.big_cap);
  for (;;) {
    if (threadIdx.x == 0) sh_idx = (long long)atomicAdd(P.queue + 1, 1ull);
    __syncthreads();
    const long long idx = sh_idx;
    __syncthreads();
    if (idx >= nbig) break;
    const int32_t v0 = P.big[idx];
    const int32_t u0 = P.up[v0], u1 = P.rp[v0 + 1];
    const int s = u1 - u0;
    const int32_t* A;
    if (s <= P.block_cap) {
      for (int i = threadIdx.x; i < s; i += blockDim.x) stage[i] = P.col[u0 + i];
      A = stage;
    } else {
      A = P.col + u0;
    }
    __syncthreads();
    if (MODE == mSum && P.gid) {
      const int g = P.gid[v0];
      if (g != cur_g) {
        flush_patterns<2>(P, c, cur_g, lane);
        cur_g = g;
      }
    }
    const int64_t arc0 = (int64_t)u0 - P.a_base;
    const int hA = P.hub_idx[v0];
    for (int j0 = wid * 32; j0 < s; j0 += nw * 32)
      l2_any_batch<MODE>(P, A, s, hA, j0, v0, arc0, lane, wcnt, c, seen);
    __syncthreads();
  }
  if (MODE == mSum) flush_patterns<2>(P, c, cur_g, lane);
  seen = warp_sum(seen);
  if (lane == 0 && seen) atomicAdd(P.stat, seen);
}

// Per-arc terms of the f2 = 0 base region sizes, for arcs a = (v0, v2) with
// v2 > v0: tri.y, and |N(v2) & (v0, inf)| - tri.x (v2's neighbours above v0
// outside A); 0 for arcs below v0.  Scanned into py / pz.
__global__ void motif_arc_terms(MotifArgs P, int64_t E, uint32_t* __restrict__ ty, uint32_t* __restrict__ tz) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < E; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = P.a_base + k;
    const int32_t v0 = P.src[a], v2 = P.col[a];
    uint32_t y = 0, z = 0;
    if (v2 > v0) {
      const uint2 tr = P.tri[k];
      const int32_t sl = P.rp[v2 + 1] - (P.rev[a] + 1);
      y = tr.y;
      z = (uint32_t)(sl - (int32_t)tr.x);
    }
    ty[k] = y;
    tz[k] = z;
  }
}

// ------------------------------------------------------------- level 3 (last)

// Per-warp filters of the last level: one-hash bitmaps of at most kMFilterW
// words over A and over B; a clear bit proves that w is not in the list.
constexpr int kMFilterW = 256;

__device__ __forceinline__ uint32_t mf_hash(int32_t x, int shift) {
  return ((uint32_t)x * 0x9E3779B1u) >> shift;
}

// words of a filter for `count` keys, about `bits_per_key` bits each (a
// power of two in [32, kMFilterW]), and the hash shift that spans its bits
__device__ __forceinline__ int mf_words(int count, int bits_per_key) {
  int fw = 32;
  while (fw < kMFilterW && 32LL * fw < (long long)bits_per_key * count) fw <<= 1;
  return fw;
}
__device__ __forceinline__ int mf_shift(int fw) { return 32 - (__ffs(fw) - 1) - 5; }

__device__ __forceinline__ void mf_build(uint32_t* F, int fw, int shift, const int32_t* X, int nx, int lane) {
  for (int i = lane; i < fw; i += 32) F[i] = 0u;
  __syncwarp();
  for (int i = lane; i < nx; i += 32) {
    const uint32_t h = mf_hash(X[i], shift);
    atomicOr(F + (h >> 5), 1u << (h & 31));
  }
}

__device__ __forceinline__ bool mf_test(const uint32_t* F, int shift, int32_t w) {
  const uint32_t h = mf_hash(w, shift);
  return ((F[h >> 5] >> (h & 31)) & 1u) != 0;
}

// arc (v0, v2) of the f2 = 0 child at position t0 of edge (v0, A[j1])
__device__ __forceinline__ int64_t a2_of(int32_t u0, int j1, int t0) { return (int64_t)u0 + j1 + 1 + t0; }

__device__ __forceinline__ bool row_bit(const uint32_t* row, int32_t w) {
  return ((row[w >> 5] >> (w & 31)) & 1u) != 0;
}

// Shared memory of motif_l3_edge per warp, in ints: candidate queue (64
// 8-byte entries), 32 lane slots, the two filters, A, B, I staging; an even
// count keeps every warp's queue 8-byte aligned.
__host__ __device__ constexpr int64_t ml3_warp_ints(int cap) {
  return (128 + 32 + 2 * kMFilterW + 3LL * cap + 1) & ~1LL;
}

// Flattened scan of up to 32 sorted lists, one per lane (col[start ..
// start + len)), on the whole warp.  The lanes with a non-empty list move
// to the low lanes (their two tags with them); the slots of all lists are
// visited 32 at a time, the owner of slot b + lane being the owner of slot
// b plus the lists that start in slots b + 1 .. b + lane (one OR-reduce
// per 32 slots).  `test(w, tag1)` returns 0 (not a candidate) or 1 |
// knowledge bits << 1; candidates are queued and handed to `hit(entry, ok, tag0,
// tag1)` 32 at a time with the tags of their list (entry = w | (list lane
// | knowledge << 5) << 32), so the exact tests run on full warps.  The
// loads of kU chunks of 32 slots are issued before their tests.
template <int kU, class Test, class Hit>
__device__ __forceinline__ void flat_scan(const int32_t* __restrict__ col, int64_t ncol, int len, int start, int tag0,
                                          int tag1, unsigned long long* Qe, int32_t* Qs, int lane, Test test,
                                          Hit hit) {
  const unsigned lt = (1u << lane) - 1u;
  const unsigned nem = __ballot_sync(kFull, len > 0);
  if (!nem) return;
  const int nch = __popc(nem);
  if (len > 0) Qs[__popc(nem & lt)] = lane;
  __syncwarp();
  const int src = lane < nch ? Qs[lane] : lane;
  __syncwarp();
  const int ct0 = __shfl_sync(kFull, tag0, src);
  const int ct1 = __shfl_sync(kFull, tag1, src);
  const int clen = __shfl_sync(kFull, len, src) * (lane < nch);
  const int cstart = __shfl_sync(kFull, start, src);
  const int incl = warp_inclusive_scan(clen, lane);
  const int total = __shfl_sync(kFull, incl, 31);
  const int excl = incl - clen;
  const int coff = cstart - excl;  // slot t of this lane's list reads col[coff + t]
  int qn = 0, q0 = 0;
  auto drain = [&](int valid) {
    __syncwarp();
    const unsigned long long e = Qe[lane];
    const int q = (int)(e >> 32) & 31;
    const int t0 = __shfl_sync(kFull, ct0, q), t1 = __shfl_sync(kFull, ct1, q);
    hit(e, lane < valid, t0, t1);
    __syncwarp();
  };
  for (int base = 0; base < total; base += 32 * kU) {
    int32_t wv[kU];
    int qv[kU];
#pragma unroll
    for (int r = 0; r < kU; r++) {
      const int b = base + 32 * r;
      const int p = excl - b;
      const unsigned S = __reduce_or_sync(kFull, (lane < nch && p >= 1 && p <= 32) ? (1u << (p - 1)) : 0u);
      const int q = (q0 + __popc(S & lt)) & 31;
      q0 += __popc(S);
      const int t = b + lane;
      const int oq = __shfl_sync(kFull, coff, q);
      wv[r] = (t < total && PGM_IDX_OK(oq + t, ncol)) ? col[oq + t] : -1;
      qv[r] = q;
    }
#pragma unroll
    for (int r = 0; r < kU; r++) {
      const int32_t w = wv[r];
      const int tg = __shfl_sync(kFull, ct1, qv[r]);
      const int tr = w >= 0 ? test(w, tg) : 0;
      const unsigned bal = __ballot_sync(kFull, tr != 0);
      if (tr)
        Qe[qn + __popc(bal & lt)] =
            (unsigned long long)(uint32_t)w | ((unsigned long long)(qv[r] | ((tr >> 1) << 5)) << 32);
      qn += __popc(bal);
      if (qn >= 32) {
        drain(32);
        if (lane < qn - 32) Qe[lane] = Qe[lane + 32];
        qn -= 32;
        __syncwarp();
      }
    }
  }
  if (qn) drain(qn);
}

// One level-2 edge (v0, v1) per warp at a time, taken from a device queue
// over arcs, so heavy edges of hub vertices spread over the whole GPU.
// A = N(v0) & (v0, inf), B = N(v1) & (v0, inf) are staged in shared memory
// when short (else read in place, with hub bitmaps for membership);
// I = A & B is built once per edge for the rank queries.
//
// The 4th vertex w of a child (v0, v1, v2) falls in one of seven regions
// M = (w~v0, w~v1, w~v2); the canonical test (header comment) accepts a
// region's members above a threshold, and the pattern is a function of
// (a02, a12, M).  So the reduce needs region sizes, not the candidates:
//
// f2 = 0 children are A[j+1 .. s) (v1 = A[j]), the first s - j - 1 entries
// of the edge's segment, so v2's rank in A is its position; the parts of
// the regions that depend on (v0, v2) only -- |N(v2) & A| and
// |N(v2) & A & (v2, inf)| -- are memoised per arc by the inspection pass.
// What is left are the common neighbours w of v1 and v2 above v0: w in
// A & B above v2, or w in B \ A.  They are found from the side of w: every
// w in B is extended by N(w) & (v1, w) (w in A) or N(w) & (v1, inf) (w not
// in A), and each element v2 in A is such a pair (with a12 = v2 in B).
// This scans the short lists of B's members once per edge instead of
// N(v2) once per child.  Every other region size is a rank in A, B or I.
//
// f2 = 1 children (v2 in B \ A): the elements of N(v2) & (v0, inf) are
// tested in A and B; the ones in A or B leave the "adjacent to v2 only"
// region, and those in B \ A above v2 move to region (v1, v2).
//
// Both scans run flattened over 32 lists; elements pass a filter (hub
// bitmap row or shared-memory bitmap filter of A / B) and the survivors are
// tested exactly, 32 at a time.  Region moves are counted per lane as
// events and folded into the six pattern counters once per edge.
constexpr int kML3Threads = 256;  // block size of the last level (at most)
constexpr int kML3Cap = 256;      // staging capacity (ints per list per warp) of the last level

// I = A & B, sorted, into I: one warp scans the shorter list and tests its
// elements in the other; returns |I|.
__device__ __forceinline__ int build_I(const MotifArgs& P, const int32_t* A, int s, int hA, const int32_t* B, int nb,
                                       int hB, int32_t* I, int64_t icap, int lane) {
  const unsigned lt = (1u << lane) - 1u;
  const bool iterA = s <= nb;
  const int32_t* X = iterA ? A : B;
  const int32_t* Y = iterA ? B : A;
  const int nx = iterA ? s : nb, ny = iterA ? nb : s;
  const int hy = iterA ? hB : hA;
  int ni = 0;
  for (int i0 = 0; i0 < nx; i0 += 32) {
    const int i = i0 + lane;
    bool in = false;
    int32_t x = 0;
    if (i < nx) {
      x = X[i];
      in = member(Y, ny, hy, P, x);
    }
    const unsigned bal = __ballot_sync(kFull, in);
    if (in && PGM_IDX_OK(ni + __popc(bal & lt), icap)) I[ni + __popc(bal & lt)] = x;
    ni += __popc(bal);
  }
  __syncwarp();
  return ni;
}

// Base region sizes of all f2 = 0 children (v2 = A[idx], j1 < idx < s) of a
// level-2 edge, in closed form: the sums over idx of the three sizes (A only
// above v2; B only + v2 only; A & B + A & v2) come from the prefix arrays
// (tri.y, |N(v2) above v0| - tri.x) and from I (the sum of |I & (v2, inf)|
// is, over w in I above v1, the number of children below w); the a12 = 1
// children (v2 in I above v1) are taken out of the a12 = 0 sums and added
// with their own folding.
__device__ __forceinline__ void f20_closed_form(const MotifArgs& P, const int32_t* A, int s, int32_t u0, int j1,
                                                int32_t v1, int nb, const int32_t* I, int ni, int lane,
                                                long long (&c)[6]) {
  const int nf0 = s - j1 - 1;
  long long sI = 0, t1 = 0, t24 = 0, t35 = 0;
  for (int k0 = 0; k0 < ni; k0 += 32) {
    const int k = k0 + lane;
    if (k < ni) {
      const int32_t w = I[k];
      if (w > v1) {
        const int ra = lower_bound_dev(A, s, w);  // w = A[ra]
        sI += ra - j1 - 1;
        const int64_t a2 = (int64_t)u0 + ra;
        if (PGM_IDX_OK(a2 - P.a_base, P.n_arc_slots)) {
          const uint2 tr = P.tri[a2 - P.a_base];
          const int sl = P.rp[w + 1] - (P.rev[a2] + 1);
          const long long igt = ni - k - 1;  // |I & (w, inf)|
          t1 += (long long)(s - ra - 1) - igt - (long long)tr.y;
          t24 += (long long)(nb - ni) + sl - (long long)tr.x;
          t35 += igt + (long long)tr.y;
        }
      }
    }
  }
  c[0] += -sI - t1;
  c[1] += -t24;
  c[2] += sI - t35 + t1 + t24;
  c[4] += t35;
  if (lane == 0) {
    const int64_t lo = (int64_t)u0 + j1 + 1 - P.a_base, hi = (int64_t)u0 + s - P.a_base;
    if (PGM_IDX_OK(hi, P.n_arc_slots + 1)) {
      const long long sy = P.py[hi] - P.py[lo], sz = P.pz[hi] - P.pz[lo];
      c[0] += (long long)nf0 * (nf0 - 1) / 2 - sy;
      c[1] += (long long)nf0 * (nb - ni) + sz;
      c[2] += sy;
    }
  }
}

__global__ void __launch_bounds__(kML3Threads, 3) motif_l3_edge(MotifArgs P) {
  extern __shared__ __align__(16) int32_t smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int32_t* wbase = smem + (int64_t)wid * ml3_warp_ints(P.cap);
  unsigned long long* Qe = reinterpret_cast<unsigned long long*>(wbase);  // candidate queue
  int32_t* Qs = wbase + 128;                                              // compaction of lanes
  uint32_t* FA = reinterpret_cast<uint32_t*>(Qs + 32);
  uint32_t* FB = FA + kMFilterW;
  int32_t* Abuf = reinterpret_cast<int32_t*>(FB + kMFilterW);
  int32_t* Bbuf = Abuf + P.cap;
  int32_t* Ismem = Bbuf + P.cap;
  int32_t* Iglob = P.scratch + gw * P.scratch_stride;
  long long c[6] = {0, 0, 0, 0, 0, 0};
  unsigned long long seen = 0;
  int cur_g = -1;
  int32_t staged_v0 = -1;  // A (when staged) and its filter belong to this v0
  const int64_t na = P.arc_hi - P.arc_lo;
  for (;;) {
    unsigned long long p0 = 0;
    if (lane == 0) p0 = atomicAdd(P.queue, (unsigned long long)kEdgeGrab);
    p0 = __shfl_sync(kFull, p0, 0);
    if ((int64_t)p0 >= na) break;
    const int64_t pend = min((int64_t)p0 + kEdgeGrab, na);
    for (int64_t ai = (int64_t)p0; ai < pend; ai++) {
      const int64_t a = P.arc_lo + ai;
      const int64_t rel = a - P.a_base;
      const int64_t cb = P.off[rel] - P.off_shift;
      const int64_t ce = P.off[rel + 1] - P.off_shift;
      const int32_t v0 = P.src[a], v1 = P.col[a];
      if (v1 < v0) continue;  // arcs to lower neighbours are not level-2 edges
      // edges with at least b_side_min f2 = 0 children are motif_l3_pairs' (none
      // of their children is stored); childless edges
      if (P.rp[v0 + 1] - (int32_t)a - 1 >= P.b_side_min || ce <= cb) continue;
      if (P.gid) {
        const int g = P.gid[v0];
        if (g != cur_g) {
          flush_patterns<6>(P, c, cur_g, lane);
          cur_g = g;
        }
      }
      const int32_t u0 = P.up[v0];
      const int s = P.rp[v0 + 1] - u0;
      const int hA = P.hub_idx[v0], hB = P.hub_idx[v1];
      const bool restage = v0 != staged_v0;  // consecutive edges of one v0 keep A and its filter
      staged_v0 = v0;
      const int32_t* A;
      if (s <= P.cap) {
        if (restage)
          for (int i = lane; i < s; i += 32) Abuf[i] = P.col[u0 + i];
        A = Abuf;
      } else {
        A = P.col + u0;
      }
      const int32_t r0 = P.rp[v1], r1 = P.rp[v1 + 1];
      const int bstart = P.rev[a] - r0 + 1;  // after v0's own entry in N(v1)
      const int nb = r1 - r0 - bstart;
      const int32_t* B;
      if (nb <= P.cap) {
        for (int i = lane; i < nb; i += 32) Bbuf[i] = P.col[r0 + bstart + i];
        B = Bbuf;
      } else {
        B = P.col + r0 + bstart;
      }
      const uint32_t* hArow = hA >= 0 ? P.hub_bits + (int64_t)hA * P.hub_words : nullptr;
      const uint32_t* hBrow = hB >= 0 ? P.hub_bits + (int64_t)hB * P.hub_words : nullptr;
      const int j1 = (int)(a - u0);  // v1 = A[j1]
      const int nf0 = s - j1 - 1;    // f2 = 0 children, first in the segment
      const int fwA = mf_words(s, 16), shA = mf_shift(fwA);
      const int fwB = mf_words(nb, 16), shB = mf_shift(fwB);
      __syncwarp();
      if (!hArow && restage) mf_build(FA, fwA, shA, A, s, lane);
      if (!hBrow) mf_build(FB, fwB, shB, B, nb, lane);
      // I = A & B, sorted
      int32_t* I = min(s, nb) <= P.cap ? Ismem : Iglob;
      const int ni = build_I(P, A, s, hA, B, nb, hB, I, I == Ismem ? P.cap : P.scratch_stride, lane);
      if (lane == 0) seen += (unsigned long long)(nb + s);
      // region moves found by the scans (per lane): f2 = 0 children with a12
      // = 0 / 1: common neighbour in A & B above v2 (y1*), in B \ A (y2*);
      // f2 = 1 children: element in A or B (eh), in B \ A above v2 (er)
      int y1a = 0, y1b = 0, y2a = 0, y2b = 0, eh = 0, er = 0;
      // Children scans, N(v2) & (v0, inf), 32 lists at a time (tags: v2,
      // f2 = 0 | a12 << 1): always for f2 = 1 children, and for the f2 = 0
      // children of edges with fewer than b_side_min of them (the others' common
      // neighbours are found from B's side by motif_l3_pairs).  Candidates:
      // f2 = 0 children, in B; f2 = 1 children, in A or B (not v1).
      // Knowledge bits: A known, in A, B known, in B.
      auto test = [&](int32_t x, int tg) -> int {
        const bool ka = hArow != nullptr, kb = hBrow != nullptr;
        const bool xa = ka && row_bit(hArow, x), xb = kb && row_bit(hBrow, x);
        const bool ca = ka ? xa : mf_test(FA, shA, x);
        const bool cbv = kb ? xb : mf_test(FB, shB, x);
        const bool cand = (tg & 1) ? cbv : (x != v1) & (ca | cbv);
        return cand ? (1 | (ka << 1) | (xa << 2) | (kb << 3) | (xb << 4)) : 0;
      };
      auto hit = [&](unsigned long long e, bool ok, int t0, int tg) {
        if (!ok) return;
        const int32_t x = (int32_t)(uint32_t)e;
        const unsigned k = (unsigned)(e >> 37);
        const bool ib = (k & 4) ? ((k >> 3) & 1) != 0 : member(B, nb, -1, P, x);
        if ((tg & 1) && !ib) return;
        const bool ia = (k & 1) ? ((k >> 1) & 1) != 0 : member(A, s, -1, P, x);
        if (tg & 1) {  // common neighbour of v1 and v2 = t0: in A & B above v2, or in B \ A
          const bool y1 = ia && x > t0, y2 = !ia;
          if (tg & 2) {
            y1b += y1;
            y2b += y2;
          } else {
            y1a += y1;
            y2a += y2;
          }
        } else {
          eh += ia || ib;
          er += ib && !ia && x > t0;
        }
      };
      // the children, 32 at a time
      for (int64_t next = cb; next < ce; next += 32) {
        int32_t tag0 = 0;
        int len = 0, start = 0, tag1 = 0;
        {
          const int64_t ci = next + lane;
          if (ci < ce && PGM_IDX_OK(ci, P.n_l3)) {
            const uint32_t e = P.l3[ci];
            const int32_t v2 = (int32_t)(e & kVidMask);
            const int a12 = (e & kA12) ? 1 : 0;
            const int t0 = (int)(ci - cb);
            const long long I_gt2 = ni - lower_bound_dev(I, ni, v2 + 1);  // |I & (v2, inf)|
            tag0 = v2;
            if (t0 < nf0 && PGM_IDX_OK(a2_of(u0, j1, t0) - P.a_base, P.n_arc_slots)) {
              const int idx = j1 + 1 + t0;  // v2 = A[idx]
              const int64_t a2 = (int64_t)u0 + idx;
              const uint2 tr = P.tri[a2 - P.a_base];  // (|N(v2) & A|, |N(v2) & A & (v2, inf)|)
              const int st = P.rev[a2] + 1;           // N(v2) & (v0, inf) starts after (v2, v0)
              const int sl = P.rp[v2 + 1] - st;
              // region sizes before the common neighbours of v1 and v2 are moved
              const long long x1 = (long long)(s - idx - 1) - I_gt2 - (long long)tr.y;  // A only, above v2
              const long long x24 = (long long)(nb - ni) + sl - (long long)tr.x;        // B only; v2 only
              const long long x35 = I_gt2 + (long long)tr.y;                           // A & B; A & v2
              if (a12) {
                c[2] += x1 + x24;
                c[4] += x35;
              } else {
                c[0] += x1;
                c[1] += x24;
                c[2] += x35;
              }
              start = st;
              len = sl;
              tag1 = 1 | (a12 << 1);
            } else {
              const int32_t a0 = P.rp[v2];
              const int d2 = P.rp[v2 + 1] - a0;
              const int lo = lower_bound_dev(P.col + a0, d2, v0 + 1);
              const int ib = lower_bound_dev(B, nb, v2 + 1);
              start = a0 + lo;
              len = d2 - lo;
              c[0] += (long long)(nb - ib) - I_gt2;  // B only, above v2 (3-star)
              c[1] += len - 1;                       // v2 only: N(v2) above v0 but v1 (4-path)
            }
          }
        }
        seen += (unsigned long long)len;
        flat_scan<2>(P.col, P.narcs, len, start, tag0, tag1, Qe, Qs, lane, test, hit);
      }
      // fold the region moves into the pattern counters: for a12 = 0 the
      // regions (A only, B only, A&B, v2 only, A&v2, B&v2, all) are (3-star,
      // 4-path, tailed triangle, 4-path, tailed triangle, 4-cycle, diamond);
      // for a12 = 1 (tailed triangle x 2, diamond, tailed triangle, diamond x 2,
      // 4-clique); for f2 = 1, (B only, v2 only, B&v2) are (3-star, 4-path,
      // tailed triangle)
      c[0] += y1a - er;
      c[1] -= 2LL * y2a + eh;
      c[2] += y1b - 2LL * (y1a + y2b) + er;
      c[3] += y2a;
      c[4] += y1a + y2b - 2LL * y1b;
      c[5] += y1b;
    }
  }
  flush_patterns<6>(P, c, cur_g, lane);
  seen = warp_sum(seen);
  if (lane == 0 && seen) atomicAdd(P.stat, seen);
}

// The level-2 edges (v0, v1) with at least b_side_min f2 = 0 children,
// whole: none of their children is stored in the level-3 list.  Every w in
// B = N(v1) & (v0, inf) is extended by its own list:
//   w in A (an f2 = 0 child or below v1): N(w) in (v1, w); each element v2
//     in A is an f2 = 0 child with the common neighbour w of v1 and v2 in
//     A & B above v2 (y1*, a12 = v2 in B);
//   w in B \ A (an f2 = 1 child): N(w) above v0; an element v2 in A above v1
//     is an f2 = 0 child with the common neighbour w in B \ A (y2*), and any
//     element x in A or B (x != v1) is an f2 = 1 region move of the child w
//     (eh; er when x is in B \ A above w).
// Base region sizes: the f2 = 0 children in closed form (f20_closed_form);
// the f2 = 1 children's "B only above v2" regions sum to C(|B \ A|, 2) and
// their "v2 only" regions to the lengths of the lists above v0 less v1.
// All moves are folded into the six pattern counters as motif_l3_edge folds
// its own.
__global__ void __launch_bounds__(kML3Threads, 3) motif_l3_pairs(MotifArgs P) {
  extern __shared__ __align__(16) int32_t smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int32_t* wbase = smem + (int64_t)wid * ml3_warp_ints(P.cap);
  unsigned long long* Qe = reinterpret_cast<unsigned long long*>(wbase);
  int32_t* Qs = wbase + 128;
  uint32_t* FA = reinterpret_cast<uint32_t*>(Qs + 32);
  uint32_t* FB = FA + kMFilterW;
  int32_t* Abuf = reinterpret_cast<int32_t*>(FA + 2 * kMFilterW);
  int32_t* Bbuf = Abuf + P.cap;
  int32_t* Ismem = Bbuf + P.cap;
  int32_t* Iglob = P.scratch + gw * P.scratch_stride;
  long long c[6] = {0, 0, 0, 0, 0, 0};
  unsigned long long seen = 0;
  int cur_g = -1;
  int32_t staged_v0 = -1;
  const int64_t na = P.arc_hi - P.arc_lo;
  for (;;) {
    unsigned long long p0 = 0;
    if (lane == 0) p0 = atomicAdd(P.queue + 4, (unsigned long long)kEdgeGrab);
    p0 = __shfl_sync(kFull, p0, 0);
    if ((int64_t)p0 >= na) break;
    const int64_t pend = min((int64_t)p0 + kEdgeGrab, na);
    for (int64_t ai = (int64_t)p0; ai < pend; ai++) {
      const int64_t a = P.arc_lo + ai;
      const int32_t v0 = P.src[a], v1 = P.col[a];
      if (v1 < v0) continue;  // arcs to lower neighbours are not level-2 edges
      const int32_t u0 = P.up[v0];
      const int s = P.rp[v0 + 1] - u0;
      const int j1 = (int)(a - u0);  // v1 = A[j1]
      const int nf0 = s - j1 - 1;
      if (nf0 < P.b_side_min) continue;  // motif_l3_edge counts these edges from the level-3 list
      if (P.gid) {
        const int g = P.gid[v0];
        if (g != cur_g) {
          flush_patterns<6>(P, c, cur_g, lane);
          cur_g = g;
        }
      }
      const int hA = P.hub_idx[v0], hB = P.hub_idx[v1];
      const uint32_t* hArow = hA >= 0 ? P.hub_bits + (int64_t)hA * P.hub_words : nullptr;
      const uint32_t* hBrow = hB >= 0 ? P.hub_bits + (int64_t)hB * P.hub_words : nullptr;
      const bool restage = v0 != staged_v0;  // consecutive edges of one v0 keep A and its filter
      staged_v0 = v0;
      const int32_t* A;
      if (s <= P.cap) {
        if (restage)
          for (int i = lane; i < s; i += 32) Abuf[i] = P.col[u0 + i];
        A = Abuf;
      } else {
        A = P.col + u0;
      }
      const int fwA = mf_words(s, 16), shA = mf_shift(fwA);
      __syncwarp();
      if (!hArow && restage) mf_build(FA, fwA, shA, A, s, lane);
      const int32_t r0 = P.rp[v1], r1 = P.rp[v1 + 1];
      const int bstart = P.rev[a] - r0 + 1;  // after v0's own entry in N(v1)
      const int nb = r1 - r0 - bstart;
      const int32_t* B;
      if (nb <= P.cap) {
        for (int i = lane; i < nb; i += 32) Bbuf[i] = P.col[r0 + bstart + i];
        B = Bbuf;
      } else {
        B = P.col + r0 + bstart;
      }
      const int fwB = mf_words(nb, 16), shB = mf_shift(fwB);
      __syncwarp();
      if (!hBrow) mf_build(FB, fwB, shB, B, nb, lane);
      int32_t* I = min(s, nb) <= P.cap ? Ismem : Iglob;
      const int ni = build_I(P, A, s, hA, B, nb, hB, I, I == Ismem ? P.cap : P.scratch_stride, lane);
      f20_closed_form(P, A, s, u0, j1, v1, nb, I, ni, lane, c);
      if (lane == 0) c[0] += (long long)(nb - ni) * (nb - ni - 1) / 2;  // B only above v2, f2 = 1 children
      int y1a = 0, y1b = 0, y2a = 0, y2b = 0, eh = 0, er = 0;
      // candidates: from w in A, elements in A; from w in B \ A, elements in A
      // or B other than v1.  Knowledge bits: A known, in A, B known, in B.
      auto test = [&](int32_t x, int w_in_A) -> int {
        const bool ka = hArow != nullptr, kb = hBrow != nullptr;
        const bool xa = ka && row_bit(hArow, x), xb = kb && row_bit(hBrow, x);
        const bool ca = ka ? xa : mf_test(FA, shA, x);
        const bool cand = w_in_A ? ca : (x != v1) & (ca | (kb ? xb : mf_test(FB, shB, x)));
        return cand ? (1 | (ka << 1) | (xa << 2) | (kb << 3) | (xb << 4)) : 0;
      };
      auto hit = [&](unsigned long long e, bool ok, int w, int w_in_A) {
        if (!ok) return;
        const int32_t x = (int32_t)(uint32_t)e;
        const unsigned k = (unsigned)(e >> 37);
        const bool ia = (k & 1) ? ((k >> 1) & 1) != 0 : member(A, s, -1, P, x);
        if (w_in_A) {  // x in N(w) & (v1, w): an f2 = 0 child with the common neighbour w in A & B
          if (!ia) return;
          const bool a12 = (k & 4) ? ((k >> 3) & 1) != 0 : member(B, nb, -1, P, x);
          y1a += !a12;
          y1b += a12;
          return;
        }
        const bool ib = (k & 4) ? ((k >> 3) & 1) != 0 : member(B, nb, -1, P, x);
        if (!ia && !ib) return;
        eh += 1;                   // the f2 = 1 child w: x in A or B
        er += ib && !ia && x > w;  // ... in B \ A above w
        if (ia && x > v1) {        // the f2 = 0 child x with the common neighbour w in B \ A
          y2a += !ib;
          y2b += ib;
        }
      };
      long long vonly = 0;  // f2 = 1 children: |N(w) above v0| - 1 (v1), the "v2 only" regions
      for (int w0 = 0; w0 < nb; w0 += 32) {
        int len = 0, start = 0, w_in_A = 0;
        int32_t w = 0;
        if (w0 + lane < nb) {
          w = B[w0 + lane];
          w_in_A = hArow ? row_bit(hArow, w) : member(A, s, -1, P, w);
          if (w_in_A) {
            // N(w) in (v1, w): after the reverse arc (w, v1) of arc (v1, w), up to up[w]
            const int64_t ab = (int64_t)r0 + bstart + w0 + lane;  // arc (v1, w)
            start = PGM_IDX_OK(ab, P.narcs) ? P.rev[ab] + 1 : 0;
            len = max(P.up[w] - start, 0);
          } else {
            // N(w) above v0
            const int32_t wa = P.rp[w];
            const int dw = P.rp[w + 1] - wa;
            start = wa + lower_bound_dev(P.col + wa, dw, v0 + 1);
            len = wa + dw - start;
            vonly += len - 1;
          }
        }
        seen += (unsigned long long)len;
        flat_scan<4>(P.col, P.narcs, len, start, w, w_in_A, Qe, Qs, lane, test, hit);
      }
      // region moves (see motif_l3_edge): y1 = A & B & v2, y2 = B & v2 (not A);
      // f2 = 1: eh (A or B & v2), er (B & v2 above v2)
      c[0] += y1a - er;
      c[1] += vonly - 2LL * y2a - eh;
      c[2] += y1b - 2LL * (y1a + y2b) + er;
      c[3] += y2a;
      c[4] += y1a + y2b - 2LL * y1b;
      c[5] += y1b;
    }
  }
  flush_patterns<6>(P, c, cur_g, lane);
  seen = warp_sum(seen);
  if (lane == 0 && seen) atomicAdd(P.stat, seen);
}

constexpr int kQ = 0, kErr = 7, kAcc = 8, kStat = 16, kSkip = 24, kNSlots = 32;

struct MotifRun {
  Graph& g;
  Workspace& ws;
  cudaStream_t s;
  int k;
  const pgm_options o;
  int cap, block_cap;
  unsigned long long* per_graph = nullptr;
  double l3_size = 0;
  int chunks = 0;
  MotifRun(Graph& g_, Workspace& ws_, cudaStream_t s_, int k_)
      : g(g_), ws(ws_), s(s_), k(k_), o(options()) {
    cap = o.warp_stage_cap;
    block_cap = 16384;
  }
  unsigned long long* ctr() { return ws.ctr.p; }

  MotifArgs args(int32_t v_lo, int32_t v_hi) {
    MotifArgs P;
    memset(&P, 0, sizeof(P));
    P.rp = g.rp;
    P.col = g.col;
    P.up = g.up;
    P.v_lo = v_lo;
    P.v_hi = v_hi;
    P.a_base = g.h_rp[v_lo];
    P.acc = ctr() + kAcc;
    P.per_graph = per_graph;
    P.gid = g.gid;
    P.queue = ctr() + kQ;
    P.err = ctr() + kErr;
    P.big = reinterpret_cast<int32_t*>(ws.big.p);
    P.big_cap = (int64_t)ws.big.cap * 2;
    P.cap = cap;
    P.block_cap = block_cap;
    P.hub_idx = g.hub_idx;
    P.hub_bits = g.hub_bits;
    P.hub_words = g.hub_words;
    P.rev = g.rev;
    P.tri = ws.tri.p;
    P.py = ws.off[4].p;
    P.pz = ws.off[5].p;
    P.carry = ctr() + kCarrySlot;
    P.b_side_min = o.motif_b_side_min > 0 ? o.motif_b_side_min : 8;
    P.skipped = ctr() + kSkip;
    P.narcs = g.narcs;
    P.n_arc_slots = g.h_rp[v_hi] - g.h_rp[v_lo];
    return P;
  }

  template <int MODE>
  pgm_status launch_l2(MotifArgs P, const char* name) {
    PGM_TRY_CUDA(cudaMemsetAsync(ctr() + kQ, 0, 4 * sizeof(unsigned long long), s));
    if (MODE != mWrite) {
      PGM_TRY(ws.cnt[3].reserve((size_t)std::max<int64_t>(P.big_cap, 1)));
      PGM_TRY_CUDA(cudaMemsetAsync(ws.cnt[3].p, 0, (size_t)std::max<int64_t>(P.big_cap, 1) * sizeof(uint32_t), s));
      P.hubctr = ws.cnt[3].p;
    }
    P.stat = ctr() + kStat + MODE;
    const int threads = o.block_threads;
    const size_t wsmem = (size_t)(threads / 32) * (cap + 64) * sizeof(int32_t);
    const size_t bsmem = (size_t)block_cap * sizeof(int32_t) + 16 * 64 * sizeof(uint32_t);
    PGM_TRY(smem_attr((const void*)motif_l2_warp<MODE>, 160 * 1024));
    PGM_TRY(smem_attr((const void*)motif_l2_block<MODE>, 160 * 1024));
    const int64_t np = (int64_t)P.v_hi - P.v_lo;
    int wgrid = grid_for((const void*)motif_l2_warp<MODE>, threads, wsmem);
    // kMGrab vertices per queue access, one when there are fewer than that
    // many per resident warp (small graphs: a warp's vertices run in series)
    P.grab = (int)std::max<int64_t>(1, std::min<int64_t>(kMGrab, np / ((int64_t)wgrid * (threads / 32))));
    const int64_t blocks_needed = ((np + P.grab - 1) / P.grab + threads / 32 - 1) / (threads / 32);
    wgrid = (int)std::max<int64_t>(1, std::min<int64_t>(wgrid, blocks_needed));
    const int bgrid = grid_for((const void*)motif_l2_block<MODE>, 512, bsmem);
    Profiler& prof = profiler();
    int id = prof.begin(name, 2);
    motif_l2_warp<MODE><<<wgrid, threads, wsmem, s>>>(P);
    PGM_CHECK_LAUNCH();
    if (MODE == mWrite) {
      motif_l2_block<MODE><<<bgrid, 512, bsmem, s>>>(P);
      PGM_CHECK_LAUNCH();
    } else {
      const int hgrid = grid_for((const void*)motif_l2_hubs<MODE>, 256, 0);
      motif_l2_hubs<MODE><<<hgrid, 256, 0, s>>>(P);
      PGM_CHECK_LAUNCH();
    }
    prof.end(id, (double)(g.h_rp[P.v_hi] - g.h_rp[P.v_lo]) / 2.0, 0.0);
    return PGM_OK;
  }

  pgm_status launch_l3(MotifArgs P, int32_t pa, int32_t pb, double entries) {
    // queue slots: [0] motif_l3_edge, [4] motif_l3_pairs
    PGM_TRY_CUDA(cudaMemsetAsync(ctr() + kQ, 0, 5 * sizeof(unsigned long long), s));
    P.stat = ctr() + kStat + 3;
    P.src = g.src;
    P.arc_lo = g.h_rp[pa];
    P.arc_hi = g.h_rp[pb];
    P.hub_idx = g.hub_idx;
    P.hub_bits = g.hub_bits;
    P.hub_words = g.hub_words;
    const int threads = std::min(o.block_threads, kML3Threads);
    P.cap = std::min(cap, kML3Cap);
    P.b_side_min = o.motif_b_side_min > 0 ? o.motif_b_side_min : 8;
    // (threads / 32) warps of at most 5.8 KB: four blocks fit an SM
    const size_t wsmem = (size_t)(threads / 32) * ml3_warp_ints(P.cap) * sizeof(int32_t);
    PGM_TRY(smem_attr((const void*)motif_l3_edge, (int)std::max<size_t>(wsmem, 200 * 1024)));
    PGM_TRY(smem_attr((const void*)motif_l3_pairs, (int)std::max<size_t>(wsmem, 200 * 1024)));
    int grid = grid_for((const void*)motif_l3_edge, threads, wsmem);
    const int64_t na = P.arc_hi - P.arc_lo;
    const int64_t blocks_needed = ((na + kEdgeGrab - 1) / kEdgeGrab + threads / 32 - 1) / (threads / 32);
    grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid, blocks_needed));
    // per-warp scratch for I = A & B when both lists are long: |I| <= dmax
    P.scratch_stride = std::max<int64_t>(g.dmax, 1);
    PGM_TRY(ws.scratch.reserve((size_t)grid * (threads / 32) * (size_t)P.scratch_stride));
    P.scratch = ws.scratch.p;
    Profiler& prof = profiler();
    int id = prof.begin("extend_sum", 3);
    motif_l3_edge<<<grid, threads, wsmem, s>>>(P);
    PGM_CHECK_LAUNCH();
    motif_l3_pairs<<<grid, threads, wsmem, s>>>(P);
    PGM_CHECK_LAUNCH();
    prof.end(id, entries, 0.0);
    return PGM_OK;
  }

  pgm_status prepare() {
    PGM_TRY(graph_prepare_motifs(g));
    PGM_TRY(ws.big.reserve((size_t)g.n / 2 + 2));  // every vertex fits (as int32)
    PGM_TRY(ws.ctr.reserve(kNSlots));
    PGM_TRY_CUDA(cudaMemsetAsync(ctr(), 0, kNSlots * sizeof(unsigned long long), s));
    if (!per_graph) PGM_TRY(seed_counts(ctr() + kAcc, k == 3 ? 2 : 6, s));
    return PGM_OK;
  }

  pgm_status run3(int32_t v_lo, int32_t v_hi) { return launch_l2<mSum>(args(v_lo, v_hi), "extend_sum"); }

  pgm_status run4(int32_t v_lo, int32_t v_hi) {
    PGM_NVTX("motif4 levels 2-4");
    const int64_t a_lo = g.h_rp[v_lo], a_hi = g.h_rp[v_hi];
    const int64_t E = a_hi - a_lo;  // arcs; arcs to lower neighbours get zero children
    if (E == 0) return PGM_OK;
    PGM_TRY(ws.cnt[2].reserve((size_t)E));
    PGM_TRY(ws.off[2].reserve((size_t)E + 1));
    PGM_TRY(ws.tri.reserve((size_t)E));
    PGM_TRY(ws.cnt[4].reserve((size_t)E));
    PGM_TRY(ws.cnt[5].reserve((size_t)E));
    PGM_TRY(ws.off[4].reserve((size_t)E + 1));
    PGM_TRY(ws.off[5].reserve((size_t)E + 1));
    PGM_TRY_CUDA(cudaMemsetAsync(ws.cnt[2].p, 0, (size_t)E * sizeof(uint32_t), s));
    PGM_TRY_CUDA(cudaMemsetAsync(ws.tri.p, 0, (size_t)E * sizeof(uint2), s));
    MotifArgs P = args(v_lo, v_hi);
    P.cnt = ws.cnt[2].p;
    PGM_TRY(launch_l2<mCount>(P, "extend_count"));
    {
      // prefix sums of the per-arc terms of the f2 = 0 base region sizes
      P.a_base = a_lo;
      P.src = g.src;  // arc sources (set by launch_l3 for the last level; needed here too)
      motif_arc_terms<<<std::max(1, std::min(num_sms() * 8, (int)((E + 255) / 256))), 256, 0, s>>>(
          P, E, ws.cnt[4].p, ws.cnt[5].p);
      PGM_CHECK_LAUNCH();
      PGM_TRY(exclusive_scan(ws.cnt[4].p, E, ws.off[4].p, ws, s));
      PGM_TRY(exclusive_scan(ws.cnt[5].p, E, ws.off[5].p, ws, s));
    }
    {
      int id = profiler().begin("scan", 2);
      PGM_TRY(exclusive_scan(ws.cnt[2].p, E, ws.off[2].p, ws, s));
      profiler().end(id, (double)E, 12.0 * (double)E);
    }
    int64_t T = 0;
    unsigned long long skipped = 0;  // f2 = 0 children of B-side edges: counted, not stored
    PGM_TRY(read_dev(ws.off[2].p + E, &T, s));
    PGM_TRY(read_dev(ctr() + kSkip, &skipped, s));  // zeroed with the counter block by prepare()
    if (T == 0 && skipped == 0) return PGM_OK;
    l3_size += (double)T + (double)skipped;
    const int64_t Bud = o.level_budget;
    int32_t pa = v_lo;
    while (pa < v_hi) {
      int64_t base;
      PGM_TRY(read_dev(ws.off[2].p + (g.h_rp[pa] - a_lo), &base, s));
      int32_t pb;
      if (T - base <= Bud) {
        pb = v_hi;
      } else {
        int32_t lo = pa + 1, hi = v_hi;
        pb = pa + 1;
        while (lo <= hi) {
          int32_t mid = lo + (hi - lo) / 2;
          int64_t om;
          PGM_TRY(read_dev(ws.off[2].p + (g.h_rp[mid] - a_lo), &om, s));
          if (om - base <= Bud) {
            pb = mid;
            lo = mid + 1;
          } else {
            hi = mid - 1;
          }
        }
      }
      int64_t ob;
      PGM_TRY(read_dev(ws.off[2].p + (g.h_rp[pb] - a_lo), &ob, s));
      const int64_t Tp = ob - base;
      chunks++;
      if (Tp > 0 || skipped > 0) {  // a chunk without stored children may still have B-side edges
        PGM_TRY(ws.vid[3].reserve((size_t)std::max<int64_t>(Tp, 1)));
        MotifArgs W = args(pa, pb);
        W.a_base = a_lo;
        W.off = ws.off[2].p;
        W.off_shift = base;
        W.l3 = reinterpret_cast<uint32_t*>(ws.vid[3].p);
        W.n_l3 = Tp;
        W.n_arc_slots = E;
        PGM_TRY(launch_l2<mWrite>(W, "extend_write"));
        // entries of the algorithmic-bytes rule: the chunk's level-3 embeddings,
        // the unstored ones (known only in total) counted with the last chunk
        PGM_TRY(launch_l3(W, pa, pb, (double)Tp + (pb == v_hi ? (double)skipped : 0.0)));
      }
      pa = pb;
    }
    return PGM_OK;
  }
};

}  // namespace

pgm_status count_motifs_on(Graph& g, Workspace& ws, cudaStream_t s, int k, int32_t v_lo, int32_t v_hi,
                           uint64_t* out, unsigned long long* per_graph_dev);

pgm_status count_motifs(Graph& g, Workspace& ws, cudaStream_t s, int k, int32_t v_lo, int32_t v_hi,
                        uint64_t* out, unsigned long long* per_graph_dev) {
  if (k < 3 || k > 5) {
    set_error("count_motifs: k=%d unsupported (3, 4 or 5)", k);
    return PGM_EUNSUPPORTED;
  }
  if (v_lo < 0 || v_hi > g.n || v_lo > v_hi) {
    set_error("count_motifs: bad vertex range [%d, %d)", v_lo, v_hi);
    return PGM_EINVAL;
  }
  if (g.n >= (1 << 30)) {
    set_error("count_motifs: n=%d needs 30-bit vertex IDs", g.n);
    return PGM_EUNSUPPORTED;
  }
  if (v_lo == 0 && v_hi == g.n && g.n > 0 && options().motif_order == 0) {
    // full range: count on the copy relabelled by degree (same counts, less work)
    Graph* r = nullptr;
    PGM_TRY(graph_relabeled(g, k == 3 ? kOrderAscending : kOrderDescending, &r));
    return count_motifs_on(*r, ws, s, k, 0, r->n, out, per_graph_dev);
  }
  return count_motifs_on(g, ws, s, k, v_lo, v_hi, out, per_graph_dev);
}

pgm_status count_motifs_on(Graph& g, Workspace& ws, cudaStream_t s, int k, int32_t v_lo, int32_t v_hi,
                           uint64_t* out, unsigned long long* per_graph_dev) {
  if (k == 5) return count_motifs5(g, ws, s, v_lo, v_hi, out, per_graph_dev);
  MotifRun run(g, ws, s, k);
  run.per_graph = per_graph_dev;
  PGM_TRY(run.prepare());
  if (v_hi > v_lo) {
    if (k == 3)
      PGM_TRY(run.run3(v_lo, v_hi));
    else
      PGM_TRY(run.run4(v_lo, v_hi));
  }
  unsigned long long h[kNSlots];
  bool deferred = false;
  PGM_TRY(read_counters(ws.ctr.p, h, kNSlots, s, &deferred));
  if (deferred) return PGM_OK;  // replay: the caller reads the counters after the graph runs
  if (h[kErr]) {
    set_error("count_motifs: internal hub-list overflow");
    return PGM_ENOMEM;
  }
  if (h[kCarrySlot]) {
    set_error("count_motifs: a count exceeds 2^64 - 1");
    return PGM_EOVERFLOW;
  }
  const int np = k == 3 ? 2 : 6;
  for (int i = 0; i < np; i++) out[i] = h[kAcc + i] - (per_graph_dev ? 0ull : count_seed());
  pgm_profile& lp = last_profile();
  Profiler& prof = profiler();
  if (prof.on) {
    PGM_TRY(prof.finish(&lp));
    for (int i = 0; i < lp.nphases; i++) {
      pgm_phase& p = lp.phase[i];
      const int mode = !strcmp(p.name, "extend_count")   ? 0
                       : !strcmp(p.name, "extend_write") ? 1
                       : !strcmp(p.name, "extend_sum")   ? (k == 3 ? 2 : 3)
                                                         : -1;
      if (mode < 0) continue;
      // neighbour-list elements read (4 B) + per-entry records (vid, row pointers: 12 B)
      p.alg_bytes = 4.0 * (double)h[kStat + mode] + 12.0 * p.entries;
    }
  }
  const int64_t m = (g.h_rp[v_hi] - g.h_rp[v_lo]) / 2;
  lp.level_size[1] = (uint64_t)(v_hi - v_lo);
  lp.level_size[2] = (uint64_t)m;
  if (k == 3) {
    lp.level_size[3] = out[0] + out[1];
  } else {
    lp.level_size[3] = (uint64_t)run.l3_size;
    uint64_t t = 0;
    for (int i = 0; i < 6; i++) t += out[i];
    lp.level_size[4] = t;
  }
  lp.chunks = run.chunks;
  return PGM_OK;
}

}  // namespace pgm

extern "C" {

pgm_status pgm_count_motifs(pgm_graph* g, int32_t k, uint64_t* out_counts, int32_t cap) {
  PGM_NVTX("pgm_count_motifs");
  if (!g || !out_counts) {
    pgm::set_error("pgm_count_motifs: null argument");
    return PGM_EINVAL;
  }
  const int np = k == 3 ? 2 : k == 4 ? 6 : k == 5 ? 21 : 0;
  if (np && cap < np) {
    pgm::set_error("pgm_count_motifs: output capacity %d too small for k=%d", cap, k);
    return PGM_EINVAL;
  }
  pgm::profiler().start(g->g.stream);
  uint64_t c[21] = {0};
  PGM_TRY(pgm::count_motifs(g->g, g->g.ws, g->g.stream, k, 0, g->g.n, c, nullptr));
  memcpy(out_counts, c, sizeof(uint64_t) * np);
  return PGM_OK;
}

pgm_status pgm_count_motifs_range(pgm_graph* g, int32_t k, int32_t v_lo, int32_t v_hi,
                                  uint64_t* out_counts, int32_t cap) {
  PGM_NVTX("pgm_count_motifs_range");
  if (!g || !out_counts) {
    pgm::set_error("pgm_count_motifs_range: null argument");
    return PGM_EINVAL;
  }
  const int np = k == 3 ? 2 : k == 4 ? 6 : k == 5 ? 21 : 0;
  if (np && cap < np) {
    pgm::set_error("pgm_count_motifs_range: output capacity too small");
    return PGM_EINVAL;
  }
  pgm::profiler().start(g->g.stream);
  uint64_t c[21] = {0};
  PGM_TRY(pgm::count_motifs(g->g, g->g.ws, g->g.stream, k, v_lo, v_hi, c, nullptr));
  memcpy(out_counts, c, sizeof(uint64_t) * np);
  return PGM_OK;
}

}  // extern "C"
