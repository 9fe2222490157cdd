// cliquebm.cu -- k-clique counting (k = 3 .. 10) with bitset level lists.
//
// Same method as clique.cu (Sec. 3.3 Listing 3, Sec. 4.1): embeddings grow
// by the last vertex only, and a candidate is kept iff it is connected to
// every earlier vertex.  What changes is the layout of a level (the
// embedding list of Sec. 5.1): for a level-2 parent u with out-list
// P = N+(u) (d entries, sorted), the level-3 children of arc (u, P[i]) are
// N+(P[i]) & P, stored as a bit row R_i over the positions of P (W = d/32
// words).  The children of a level-3 entry (u, P[i], P[j]) are then
// R_i & R_j, so the connectivity check of 32 candidates against the whole
// embedding is one AND, and the fused last level is a population count:
//   triangles at u  = sum_i popc(R_i)
//   4-cliques at u  = sum_i sum_{j in R_i} popc(R_i & R_j)
//   5-cliques at u  = sum_i sum_{j in R_i} sum_{l in R_i & R_j} popc(R_i & R_j & R_l)
// and for k >= 6 a depth-first walk over chains j_1 in C_0 = R_i, j_2 in C_1,
// ... with C_t = C_{t-1} & R_{j_t} (the level-(t+3) children of the chain),
// whose leaves at depth k - 4 sum popc(C & R_l) over l in C.
// Each clique is counted once, at its first vertex in DAG order.
//
// Rows are built per vertex by intersecting N+(P[i]) with P, forward (scan
// N+(P[i]), find each element's position in P) or in reverse (test each
// P[j] against N+(P[i])) -- whichever list is shorter is scanned.
// Vertices with d <= 64 are handled by one warp with the rows in shared
// memory (two words each); larger ones by one block, with the rows in
// shared memory up to d = 512 and in a per-block global scratch area above.
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace pgm {
namespace {

constexpr int kBmWarpD = 64;     // warp kernel: d <= 64 (two words per row)
constexpr int kBmGrab = 8;

// counter slots: [0] warp queue, [kQPop + b] / [kQPush + b] pop / push
// counters of bucket b, [8..10] counts, [12] statistics, [15] error,
// [kDeepLvl + t] entries of level t + 3 for t = 2 .. kDeepMax (k >= 6)
constexpr int kQPop = 1, kQPush = 16, kBmBuckets = 4, kDeepLvl = 20, kBmSlots = 28;
constexpr int kDeepMax = 6;  // depth of the walk for k = 10

struct BmArgs {
  const int32_t* rp;   // DAG
  const int32_t* col;
  int32_t v_lo, v_hi;
  int k;
  unsigned long long* acc;    // [0] k-cliques, [1] level-3 entries, [2] level-4 entries
  unsigned long long* queue;  // counter block (slots above)
  unsigned long long* err;
  int32_t* big;               // vertices of bucket b at big[big_off[b] ...]
  int64_t big_off[kBmBuckets];
  int64_t big_cap[kBmBuckets];
  int smem_d;                 // out-degrees above this use the global-row bucket (3)
  int fwd_ratio;              // forward row build when d(v) <= fwd_ratio * d(u)
  uint32_t* scratch;          // per-block rows for the global-row bucket
  int64_t scratch_words;      // words per block
  unsigned long long* stat;   // adjacency elements read while building rows
  const int32_t* gid;
  unsigned long long* per_graph;
  unsigned long long* deep;   // k >= 6: [t] entries of level t + 3 (t = 2 .. k - 4)
  int clevels;                // C buffers per warp: 1, or k - 4 for k >= 6
  unsigned long long* carry;  // wraps of the count accumulators (add_count)
  int grab;                   // vertices a warp of the warp kernel takes per queue grab
  int classified;             // 1: bm_classify_kernel filled the bucket lists beforehand
};

// bucket of a vertex with out-degree d > kBmWarpD
__device__ __forceinline__ int bm_bucket(int d, int smem_d) {
  if (d > smem_d) return 3;
  return d <= 256 ? 0 : (d <= 512 ? 1 : 2);
}

__device__ __forceinline__ void bm_flush(const BmArgs& B, unsigned long long (&c)[3], int g, int lane) {
#pragma unroll
  for (int i = 0; i < 3; i++) {
    unsigned long long s = warp_sum(c[i]);
    if (lane == 0 && s) {
      if (i == 0)
        add_count((B.per_graph && g >= 0) ? B.per_graph + g : B.acc, s, false, B.carry);
      else
        atomicAdd(B.acc + i, s);
    }
    c[i] = 0;
  }
}

// Lower bound of x in the sorted list P[0, d), d >= 1, with a trip count
// that depends on d only (the lanes of a warp never diverge in the loop).
__device__ __forceinline__ int bm_lower_bound(const int32_t* P, int d, int32_t x) {
  int base = 0, n = d;
  while (n > 1) {
    const int half = n >> 1;
    base = P[base + half] < x ? base + half : base;
    n -= half;
  }
  return base + (P[base] < x ? 1 : 0);
}

// One-hash bitmap filter over the vertices of P: bit h(x) is set for every
// x in P, so a clear bit proves that x is not in P (a set bit may be a
// collision).  The filter has 32 * FW bits, FW = 2^fb >= d words.
__device__ __forceinline__ uint32_t bm_fhash(int32_t x, int fshift) {
  return ((uint32_t)x * 0x9E3779B1u) >> fshift;
}

__device__ __forceinline__ bool bm_fhit(const uint32_t* F, int fshift, int32_t x) {
  const uint32_t h = bm_fhash(x, fshift);
  return (F[h >> 5] >> (h & 31)) & 1u;
}

// Filter words and shift for a list of d entries (at most `cap` words).
__device__ __forceinline__ void bm_filter_size(int d, int cap, int& fw, int& fshift) {
  fw = 32;
  while (fw < d && fw < cap) fw <<= 1;
  fshift = 32 - (__ffs(fw) - 1) - 5;  // 32 * fw bits
}

// Position of x in P by binary search, or -1.
struct BmSearch {
  const int32_t* P;
  int d;
  __device__ __forceinline__ int operator()(int32_t x) const {
    const int j = bm_lower_bound(P, d, x);
    return (j < d && P[j] == x) ? j : -1;
  }
};

// Position of x in P by an open-addressing table (linear probing, at most
// half full): keys K (-1 = empty) and positions Pos, T = mask + 1 slots.
__device__ __forceinline__ uint32_t bm_thash(int32_t x, int shift) {
  return ((uint32_t)x * 0x85EBCA6Bu) >> shift;
}

struct BmTable {
  const int32_t* K;
  const uint16_t* Pos;
  uint32_t mask;
  int shift;
  __device__ __forceinline__ int operator()(int32_t x) const {
    uint32_t h = bm_thash(x, shift);
    for (uint32_t probe = 0; probe <= mask; probe++) {
      const int32_t k = K[h];
      if (k == x) return Pos[h];
      if (k < 0) return -1;
      h = (h + 1) & mask;
    }
    return -1;
  }
};

// Sets bit j of `row` when P[j] == x.
template <class Loc>
__device__ __forceinline__ void bm_locate(const Loc& loc, int32_t x, uint32_t* row) {
  const int j = loc(x);
  if (j >= 0) atomicOr(row + (j >> 5), 1u << (j & 31));
}

// Forward build of one row by one warp: scan N+(v) (col[b0, b0 + dv)),
// reject elements with the filter, queue the survivors in q (64 entries)
// and locate them 32 at a time, so that the binary searches run on full
// warps.  The row must be zero beforehand.
template <class Loc>
__device__ __forceinline__ void bm_row_forward(const int32_t* __restrict__ col, int32_t b0, int32_t dv,
                                               const Loc& loc, const uint32_t* F, int fshift,
                                               int32_t* q, uint32_t* row, int lane) {
  constexpr int U = 4;  // loads in flight per lane
  const unsigned lt = (1u << lane) - 1u;
  int cnt = 0;
  for (int t0 = 0; t0 < dv; t0 += 32 * U) {
    int32_t x[U];
#pragma unroll
    for (int r = 0; r < U; r++) {
      const int t = t0 + r * 32 + lane;
      x[r] = t < dv ? col[b0 + t] : -1;
    }
#pragma unroll
    for (int r = 0; r < U; r++) {
      const bool cand = (x[r] >= 0) & bm_fhit(F, fshift, x[r]);
      const unsigned bal = __ballot_sync(kFull, cand);
      if (cand) q[cnt + __popc(bal & lt)] = x[r];
      cnt += __popc(bal);
      if (cnt >= 32) {
        __syncwarp();
        bm_locate(loc, q[lane], row);
        __syncwarp();
        if (lane < cnt - 32) q[lane] = q[lane + 32];
        cnt -= 32;
        __syncwarp();
      }
    }
  }
  __syncwarp();
  if (lane < cnt) bm_locate(loc, q[lane], row);
  __syncwarp();
}

// Reverse build of one row by one warp: test each P[j] against N+(v) by
// binary search in global memory; one ballot word per 32 positions.
// N+(v) is cut into 32 segments of S elements; lane l holds the last
// element of segment l, so a search first picks the segment among the lanes
// (shuffles) and then searches S elements in memory.
__device__ __forceinline__ void bm_row_reverse(const int32_t* __restrict__ col, int32_t b0, int32_t dv,
                                               const int32_t* P, int d, uint32_t* row, int lane) {
  const int S = (dv + 31) >> 5;
  const int s0 = lane * S;
  const int32_t key = s0 < dv ? col[b0 + min(s0 + S, dv) - 1] : INT32_MAX;
  for (int j0 = 0; j0 < d; j0 += 32) {
    const int j = j0 + lane;
    const int32_t x = j < d ? P[j] : INT32_MAX;
    int seg = 0;  // first segment whose last element is >= x
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const int32_t k = __shfl_sync(kFull, key, seg + step - 1);
      if (k < x) seg += step;
    }
    const int32_t kseg = __shfl_sync(kFull, key, seg);
    bool in = false;
    const int lo = seg * S;
    if (j < d && kseg >= x && lo < dv) {
      // branch-free search of the segment: every lane's segment has S
      // elements except the last, so the trip counts agree across the warp
      const int32_t* a = col + b0 + lo;
      int base = 0;
      for (int n = min(lo + S, dv) - lo; n > 1;) {
        const int half = n >> 1;
        base = __ldg(a + base + half) <= x ? base + half : base;
        n -= half;
      }
      in = __ldg(a + base) == x;
    }
    const unsigned bal = __ballot_sync(kFull, in);
    if (lane == 0 && bal) row[j0 >> 5] |= bal;
  }
}

// k >= 6 in the warp kernel: the lane that owns row i walks the chains
// below C_T = (c0, c1) (two words); at depth D it adds popc(C_D & R_l) for
// every l in C_D.  lvl[t] counts the entries of level t + 3.
template <int T>
__device__ __forceinline__ void bm_deep_lane(uint32_t c0, uint32_t c1, const uint32_t* R, int D,
                                             unsigned long long& leaf, unsigned long long (&lvl)[kDeepMax + 1]) {
  if (T == D) {
    for (int h = 0; h < 2; h++) {
      uint32_t bits = h ? c1 : c0;
      while (bits) {
        const int l = (h << 5) + __ffs(bits) - 1;
        bits &= bits - 1;
        leaf += (unsigned long long)(__popc(c0 & R[2 * l]) + __popc(c1 & R[2 * l + 1]));
      }
    }
    return;
  }
  if constexpr (T < kDeepMax) {
    for (int h = 0; h < 2; h++) {
      uint32_t bits = h ? c1 : c0;
      while (bits) {
        const int j = (h << 5) + __ffs(bits) - 1;
        bits &= bits - 1;
        const uint32_t n0 = c0 & R[2 * j], n1 = c1 & R[2 * j + 1];
        const unsigned pc = (unsigned)(__popc(n0) + __popc(n1));
        lvl[T + 1] += pc;
        if (pc) bm_deep_lane<T + 1>(n0, n1, R, D, leaf, lvl);
      }
    }
  }
}

// per-lane level counters of the walk -> the counter block (levels 5 ..)
__device__ __forceinline__ void bm_deep_flush(const BmArgs& B, unsigned long long (&lvl)[kDeepMax + 1]) {
#pragma unroll
  for (int t = 2; t <= kDeepMax; t++) {
    const unsigned long long x = warp_sum(lvl[t]);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(B.deep + t, x);
    lvl[t] = 0;
  }
}

// ----------------------------------------------------------- warp kernel
// One vertex per warp, d <= 64: P and the rows (2 words, stride 2) in shared memory.
// DEEP: k >= 6 (the walk); otherwise k = 3, 4, 5.
template <bool DEEP>
__global__ void __launch_bounds__(256, DEEP ? 4 : 8) bm_warp_kernel(BmArgs B) {
  __shared__ int32_t sP[8][kBmWarpD];
  __shared__ int32_t sB0[8][kBmWarpD];
  __shared__ int32_t sDv[8][kBmWarpD];
  __shared__ uint32_t sR[8][kBmWarpD * 2];
  __shared__ uint32_t sF[8][kBmWarpD];  // filter: 64 words = 2048 bits
  __shared__ int32_t sQ[8][64];         // forward-build queue
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t* F = sF[wid];
  constexpr int kWarpFShift = 32 - 11;
  int32_t* P = sP[wid];
  uint32_t* R = sR[wid];
  unsigned long long c[3] = {0, 0, 0};
  unsigned long long lvl[kDeepMax + 1] = {0, 0, 0, 0, 0, 0, 0};
  unsigned long long seen = 0;
  int cur_g = -1;
  const int64_t np = (int64_t)B.v_hi - B.v_lo;
  for (;;) {
    unsigned long long p0 = 0;
    if (lane == 0) p0 = atomicAdd(B.queue, (unsigned long long)B.grab);
    p0 = __shfl_sync(kFull, p0, 0);
    if ((int64_t)p0 >= np) break;
    const int64_t pend = min((int64_t)p0 + B.grab, np);
    for (int64_t pi = (int64_t)p0; pi < pend; pi++) {
      const int32_t u = (int32_t)(B.v_lo + pi);
      const int32_t a0 = B.rp[u];
      const int d = B.rp[u + 1] - a0;
      if (d < 2) continue;  // no triangle (hence no level-3 entry) rooted at u
      if (d > kBmWarpD) {
        if (lane == 0 && !B.classified) {
          const int b = bm_bucket(d, B.smem_d);
          unsigned long long x = atomicAdd(B.queue + kQPush + b, 1ull);
          if ((int64_t)x < B.big_cap[b])
            B.big[B.big_off[b] + (int64_t)x] = u;
          else
            atomicAdd(B.err, 1ull);
        }
        continue;
      }
      if (B.gid) {
        const int g = B.gid[u];
        if (g != cur_g) {
          bm_flush(B, c, cur_g, lane);
          cur_g = g;
        }
      }
      for (int i = lane; i < d; i += 32) {
        const int32_t x = B.col[a0 + i];
        const int32_t b = B.rp[x];
        P[i] = x;
        sB0[wid][i] = b;
        sDv[wid][i] = B.rp[x + 1] - b;
      }
      for (int i = lane; i < 2 * kBmWarpD; i += 32) R[i] = 0;
      for (int i = lane; i < kBmWarpD; i += 32) F[i] = 0;
      __syncwarp();
      for (int i = lane; i < d; i += 32) {
        const uint32_t h = bm_fhash(P[i], kWarpFShift);
        atomicOr(F + (h >> 5), 1u << (h & 31));
      }
      __syncwarp();
      for (int i = 0; i < d; i++) {
        const int32_t b0 = sB0[wid][i], dv = sDv[wid][i];
        if (lane == 0) seen += (unsigned long long)dv;
        if ((int64_t)dv <= (int64_t)B.fwd_ratio * d)
          bm_row_forward(B.col, b0, dv, BmSearch{P, d}, F, kWarpFShift, sQ[wid], R + 2 * i, lane);
        else
          bm_row_reverse(B.col, b0, dv, P, d, R + 2 * i, lane);
      }
      __syncwarp();
      // lanes own rows i = lane, lane + 32
      for (int i = lane; i < d; i += 32) {
        const uint32_t r0 = R[2 * i], r1 = R[2 * i + 1];
        const unsigned long long tri = (unsigned long long)(__popc(r0) + __popc(r1));
        if (B.k == 3) {
          c[0] += tri;
          continue;
        }
        c[1] += tri;
        if constexpr (DEEP) {
          bm_deep_lane<0>(r0, r1, R, B.k - 4, c[0], lvl);
          continue;
        }
        unsigned long long k4 = 0, k5 = 0;
        for (int h = 0; h < 2; h++) {
          uint32_t bits = h ? r1 : r0;
          while (bits) {
            const int j = (h << 5) + __ffs(bits) - 1;
            bits &= bits - 1;
            const uint32_t c0 = r0 & R[2 * j], c1 = r1 & R[2 * j + 1];
            k4 += (unsigned long long)(__popc(c0) + __popc(c1));
            if (B.k == 5) {
              for (int h2 = 0; h2 < 2; h2++) {
                uint32_t b2 = h2 ? c1 : c0;
                while (b2) {
                  const int l = (h2 << 5) + __ffs(b2) - 1;
                  b2 &= b2 - 1;
                  k5 += (unsigned long long)(__popc(c0 & R[2 * l]) + __popc(c1 & R[2 * l + 1]));
                }
              }
            }
          }
        }
        if (B.k == 4) {
          c[0] += k4;
        } else {
          c[2] += k4;
          c[0] += k5;
        }
      }
      __syncwarp();
    }
  }
  bm_flush(B, c, cur_g, lane);
  if constexpr (DEEP) {
    // level 4 = lvl[1]; levels 5 .. k - 1 = lvl[2 ..]
    const unsigned long long x = warp_sum(lvl[1]);
    if (lane == 0 && x) atomicAdd(B.acc + 2, x);
    bm_deep_flush(B, lvl);
  }
  seen = warp_sum(seen);
  if (lane == 0 && seen) atomicAdd(B.stat, seen);
}

// The vertices of out-degree above kBmWarpD into their buckets' lists, one
// thread per vertex: run before the warp kernel, it lets the bucket kernels
// start without waiting for the warp kernel.
__global__ void bm_classify_kernel(BmArgs B) {
  const int64_t np = (int64_t)B.v_hi - B.v_lo;
  for (int64_t pi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pi < np; pi += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = (int32_t)(B.v_lo + pi);
    const int d = B.rp[u + 1] - B.rp[u];
    if (d <= kBmWarpD) continue;
    const int b = bm_bucket(d, B.smem_d);
    const unsigned long long x = atomicAdd(B.queue + kQPush + b, 1ull);
    if ((int64_t)x < B.big_cap[b])
      B.big[B.big_off[b] + (int64_t)x] = u;
    else
      atomicAdd(B.err, 1ull);
  }
}

// ---------------------------------------------------------- block kernels
// One big vertex (d > 64) per block, in buckets by out-degree so that the
// block size and shared memory fit the rows: DMAX > 0 keeps P, the start
// and length of each out-list, the filter and the rows (W words at stride
// W + 1, odd so that rows spread over the banks) in shared memory; DMAX = 0
// keeps P and the rows in global memory (the per-block scratch) and the
// filter (at most kBmGlobalFW words) in shared memory.
constexpr int kBmGlobalFW = 8192;

// Set bits of a row, 32 at a time: appends the set bits of the 32 words
// held one per lane (`mine`, words w0 .. w0 + 31) to the warp's buffer
// (64 entries) and calls f(j, true) on every lane for each full group of
// 32 positions j.  bm_bits_tail() hands over the last partial group.  A
// non-zero `tag` (< 2^15, rows of fewer than 2^16 positions) is stored in
// bits 16.. of each entry.
template <class F>
__device__ __forceinline__ void bm_bits(uint32_t mine, int w0, int* buf, int& cnt, int lane, F& f, int tag = 0) {
  uint32_t nz = __ballot_sync(kFull, mine != 0u);
  while (nz) {
    const int q = __ffs(nz) - 1;
    nz &= nz - 1;
    const uint32_t word = __shfl_sync(kFull, mine, q);
    if ((word >> lane) & 1u) buf[cnt + __popc(word & ((1u << lane) - 1u))] = (tag << 16) + ((w0 + q) << 5) + lane;
    cnt += __popc(word);
    if (cnt >= 32) {
      __syncwarp();
      f(buf[lane], true);
      __syncwarp();
      if (lane < cnt - 32) buf[lane] = buf[lane + 32];
      cnt -= 32;
      __syncwarp();
    }
  }
}

template <class F>
__device__ __forceinline__ void bm_bits_tail(const int* buf, int cnt, int lane, F& f) {
  __syncwarp();
  if (cnt > 0) {
    const bool v = lane < cnt;
    f(v ? buf[lane] : 0, v);
  }
  __syncwarp();
}

// Row layout of the block kernels: a row of W words occupies S4 16-byte
// chunks, S4 = ceil(W / 4) rounded up to an odd number, so that rows can be
// read with 128-bit loads and the rows taken by the 8 lanes of a
// quarter-warp (one j each) fall on different bank groups unless their
// indices agree modulo 8.
__host__ __device__ constexpr int bm_s4(int W) { return ((W + 3) >> 2) | 1; }

// |X & Y| over n4 16-byte chunks.
__device__ __forceinline__ unsigned bm_and_popc4(const uint4* X, const uint4* Y, int n4) {
  unsigned s = 0;
#pragma unroll 2
  for (int q = 0; q < n4; q++) {
    const uint4 x = X[q], y = Y[q];
    s += __popc(x.x & y.x) + __popc(x.y & y.y) + __popc(x.z & y.z) + __popc(x.w & y.w);
  }
  return s;
}

// Shared-memory bytes of bm_block_kernel<DMAX, THREADS, KV> with `clevels`
// C buffers per warp (1, or k - 4 for the walk of k >= 6).
__host__ __device__ constexpr size_t bm_block_smem(int dmax, int threads, int clevels) {
  return dmax > 0 ? (size_t)4 * dmax                       // P
                        + (size_t)8 * dmax                  // start and length of each out-list
                        + (size_t)4 * dmax                  // filter (up to dmax words)
                        + (size_t)(4 + 2) * 2 * dmax        // position table: 2 dmax keys + positions
                        + (size_t)4 * (threads / 32) * 128  // two 64-entry buffers per warp
                        + (size_t)16 * (threads / 32) * bm_s4(dmax / 32) * clevels  // C buffers per warp
                        + (size_t)16 * dmax * bm_s4(dmax / 32)                      // rows
                  : (size_t)4 * (threads / 32) * 128 + (size_t)4 * kBmGlobalFW;
}

// C buffers per warp of the 5-clique count: one per j of a group of j's
// processed together (8 for out-degrees up to 256, 2 up to 512, else 1).
__host__ __device__ constexpr int bm_c5(int dmax) { return dmax == 256 ? 8 : (dmax == 512 ? 2 : 1); }

// The largest block layout, k = 10 (kDeepMax C buffers) in the 1024 bucket,
// is 220,160 B: within the 227 KB a block may opt into on sm_103a.
static_assert(bm_block_smem(1024, 1024, kDeepMax) <= 227 * 1024, "bitset bucket exceeds 227 KB");

// resident blocks per SM that the register budget is sized for (the walk
// of k >= 6 keeps its level counters in registers: fewer, larger threads)
__host__ __device__ constexpr int bm_min_blocks(int dmax, int threads, int kv) {
  return kv >= 5 ? (threads <= 256 ? 4 : (threads <= 512 ? 2 : 1))
                 : (dmax == 0 ? 2 : (threads <= 256 ? 8 : (threads <= 512 ? 3 : 1)));
}

// k >= 6 in the block kernels: one warp walks the chains below C_T (W
// words at Ct, 16-byte chunks n4), one j at a time: C_{T+1} = C_T & R_j goes
// to buffer T of the warp (cstride words apart); at depth D the leaf adds
// |C_D & R_l| for every l in C_D, one l per lane.  lvl[t] counts the
// entries of level t + 3.
//
// At depth D - 1 (children are leaves) with G > 1 the j's go in groups of G,
// one group of 4 n4 lanes per j: C_D = C_T & R_j for the whole group into
// buffers T .. T + G - 1, then the pairs (C_D, l) of the group 32 at a time
// (buf2), so that the leaves of sibling chains share full warps.
template <int T, class RowFn>
__device__ __forceinline__ void bm_deep_walk(const uint32_t* Ct, int D, int W, int n4, uint32_t* Cbuf,
                                             int64_t cstride, const RowFn& row4, int* buf, int* buf2, int G,
                                             int lane, unsigned long long& leaf,
                                             unsigned long long (&lvl)[kDeepMax + 1]) {
  if (T == D) {
    int cnt = 0;
    auto fl = [&](int l, bool valid) {
      if (valid) leaf += bm_and_popc4(reinterpret_cast<const uint4*>(Ct), row4(l), n4);
    };
    for (int w0 = 0; w0 < W; w0 += 32) {
      const uint32_t mine = w0 + lane < W ? Ct[w0 + lane] : 0u;
      bm_bits(mine, w0, buf, cnt, lane, fl);
    }
    bm_bits_tail(buf, cnt, lane, fl);
    return;
  }
  if constexpr (T < kDeepMax) {
    if (T + 1 == D && G > 1) {
      const int L = 4 * n4;
      uint32_t* Cg0 = Cbuf + (int64_t)T * cstride;  // buffers T .. T + G - 1
      auto fl = [&](int e, bool v) {
        if (v) leaf += bm_and_popc4(reinterpret_cast<const uint4*>(Cg0 + (int64_t)(e >> 16) * cstride), row4(e & 0xffff), n4);
      };
      auto fj = [&](int j, bool valid) {
        const int nvj = __popc(__ballot_sync(kFull, valid));  // valid lanes are a prefix
        for (int g0 = 0; g0 < nvj; g0 += G) {
          const int ng = min(G, nvj - g0);
          const int gi = lane / L, w = lane - gi * L;
          const int jq = __shfl_sync(kFull, j, min(g0 + gi, 31));
          unsigned cn = 0;
          if (gi < ng) {
            const uint32_t x = Ct[w] & reinterpret_cast<const uint32_t*>(row4(jq))[w];  // padding words are zero
            Cg0[gi * cstride + w] = x;
            cn = __popc(x);
          }
          lvl[T + 1] += cn;
          __syncwarp();
          int cnt2 = 0;
          for (int g = 0; g < ng; g++)
            for (int w0 = 0; w0 < W; w0 += 32) {
              const uint32_t mine = w0 + lane < W ? Cg0[g * cstride + w0 + lane] : 0u;
              bm_bits(mine, w0, buf2, cnt2, lane, fl, g);
            }
          bm_bits_tail(buf2, cnt2, lane, fl);  // ends with __syncwarp: the group's buffers are free
        }
      };
      int cnt = 0;
      for (int w0 = 0; w0 < W; w0 += 32) {
        const uint32_t mine = w0 + lane < W ? Ct[w0 + lane] : 0u;
        bm_bits(mine, w0, buf, cnt, lane, fj);
      }
      bm_bits_tail(buf, cnt, lane, fj);
      return;
    }
    uint32_t* Cn = Cbuf + (int64_t)T * cstride;  // C_{T+1}
    for (int w0 = 0; w0 < W; w0 += 32) {
      const uint32_t mine = w0 + lane < W ? Ct[w0 + lane] : 0u;
      unsigned nz = __ballot_sync(kFull, mine != 0u);
      while (nz) {
        const int q = __ffs(nz) - 1;
        nz &= nz - 1;
        uint32_t word = __shfl_sync(kFull, mine, q);
        while (word) {
          const int j = ((w0 + q) << 5) + __ffs(word) - 1;
          word &= word - 1;
          const uint32_t* Rj = reinterpret_cast<const uint32_t*>(row4(j));
          __syncwarp();  // the previous chain's readers of Cn are done
          unsigned cn = 0;
          for (int w = lane; w < 4 * n4; w += 32) {
            const uint32_t x = Ct[w] & Rj[w];  // padding words are zero
            Cn[w] = x;
            cn += __popc(x);
          }
          lvl[T + 1] += cn;
          __syncwarp();
          if (__any_sync(kFull, cn != 0u))
            bm_deep_walk<T + 1>(Cn, D, W, n4, Cbuf, cstride, row4, buf, buf2, G, lane, leaf, lvl);
        }
      }
    }
  }
}

// KV: 4 (k = 3, 4), 5 (k = 5) or 6 (k = 6 .. 10, the walk).
template <int DMAX, int THREADS, int KV>
__global__ void __launch_bounds__(THREADS, bm_min_blocks(DMAX, THREADS, KV)) bm_block_kernel(BmArgs B, int bucket) {
  constexpr int NW = THREADS / 32;
  constexpr int S4MAX = DMAX > 0 ? bm_s4(DMAX / 32) : 0;
  extern __shared__ __align__(16) uint32_t smem_u[];
  __shared__ long long sh_idx;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // layout (DMAX > 0): P | B0 | Dv | filter | table keys | table positions | buffers | C | rows;
  // (DMAX = 0): filter | buffers
  constexpr int kHead = DMAX > 0 ? 7 * DMAX : kBmGlobalFW;
  int32_t* sP = reinterpret_cast<int32_t*>(smem_u);
  int32_t* sB0 = sP + DMAX;
  int32_t* sDv = sB0 + DMAX;
  uint32_t* sF = smem_u + (DMAX > 0 ? 3 * DMAX : 0);
  int32_t* sK = reinterpret_cast<int32_t*>(smem_u) + 4 * DMAX;
  uint16_t* sPos = reinterpret_cast<uint16_t*>(smem_u + 6 * DMAX);
  int* buf = reinterpret_cast<int*>(smem_u) + kHead + wid * 128;
  int* buf2 = buf + 64;
  // C buffers per warp: 5-cliques, one per j of a group; the walk, one per
  // depth plus the extra buffers of the grouped last level
  const int CL = KV == 6 ? B.clevels - 1 + bm_c5(DMAX) : (KV == 5 ? bm_c5(DMAX) : 1);
  uint32_t* sC = smem_u + kHead + NW * 128 + wid * 4 * S4MAX * CL;
  uint32_t* sRows = smem_u + kHead + NW * 128 + NW * 4 * S4MAX * CL;
  uint32_t* gRows = B.scratch ? B.scratch + (int64_t)blockIdx.x * B.scratch_words : nullptr;
  unsigned long long c[3] = {0, 0, 0};
  unsigned long long lvl[kDeepMax + 1] = {0, 0, 0, 0, 0, 0, 0};
  unsigned long long seen = 0;
  int cur_g = -1;
  const long long nbig = min((long long)B.queue[kQPush + bucket], (long long)B.big_cap[bucket]);
  const int32_t* big = B.big + B.big_off[bucket];
  for (;;) {
    if (threadIdx.x == 0) sh_idx = (long long)atomicAdd(B.queue + kQPop + bucket, 1ull);
    __syncthreads();
    const long long idx = sh_idx;
    __syncthreads();
    if (idx >= nbig) break;
    const int32_t u = big[idx];
    const int32_t a0 = B.rp[u];
    const int d = B.rp[u + 1] - a0;
    const int W = (d + 31) >> 5, n4 = (W + 3) >> 2, S = 4 * bm_s4(W);
    if (B.gid) {
      const int g = B.gid[u];
      if (g != cur_g) {
        bm_flush(B, c, cur_g, lane);
        cur_g = g;
      }
    }
    const int32_t* P;
    uint32_t* R;
    int fw, fshift;
    bm_filter_size(d, DMAX > 0 ? DMAX : kBmGlobalFW, fw, fshift);
    if constexpr (DMAX > 0) {
      for (int i = threadIdx.x; i < d; i += THREADS) {
        const int32_t x = B.col[a0 + i];
        const int32_t b = B.rp[x];
        sP[i] = x;
        sB0[i] = b;
        sDv[i] = B.rp[x + 1] - b;
      }
      for (int i = threadIdx.x; i < d * S; i += THREADS) sRows[i] = 0;
      P = sP;
      R = sRows;
    } else {
      for (int64_t i = threadIdx.x; i < (int64_t)d * S; i += THREADS)
        if (PGM_IDX_OK(i, B.scratch_words)) gRows[i] = 0;
      P = B.col + a0;
      R = gRows;
    }
    for (int i = threadIdx.x; i < fw; i += THREADS) sF[i] = 0;
    uint32_t tmask = 0;
    int tshift = 0;
    if constexpr (DMAX > 0) {
      int T = 64;
      while (T < 2 * d) T <<= 1;
      tmask = (uint32_t)T - 1u;
      tshift = 32 - (__ffs(T) - 1);
      for (int i = threadIdx.x; i < T; i += THREADS) sK[i] = -1;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < d; i += THREADS) {
      const int32_t x = P[i];
      const uint32_t h = bm_fhash(x, fshift);
      atomicOr(sF + (h >> 5), 1u << (h & 31));
      if constexpr (DMAX > 0) {
        uint32_t t = bm_thash(x, tshift);
        for (uint32_t probe = 0; probe <= tmask; probe++) {
          if (atomicCAS(sK + t, -1, x) == -1) {
            sPos[t] = (uint16_t)i;
            break;
          }
          t = (t + 1) & tmask;
        }
      }
    }
    __syncthreads();
    // rows R_i = N+(P[i]) & P, one warp per row
    for (int i = wid; i < d; i += NW) {
      int32_t b0, dv;
      if constexpr (DMAX > 0) {
        b0 = sB0[i];
        dv = sDv[i];
      } else {
        const int32_t v = P[i];
        b0 = B.rp[v];
        dv = B.rp[v + 1] - b0;
      }
      uint32_t* row = R + (int64_t)i * S;
      if (lane == 0) seen += (unsigned long long)dv;
      if ((int64_t)dv <= (int64_t)B.fwd_ratio * d)
        if constexpr (DMAX > 0)
          bm_row_forward(B.col, b0, dv, BmTable{sK, sPos, tmask, tshift}, sF, fshift, buf, row, lane);
        else
          bm_row_forward(B.col, b0, dv, BmSearch{P, d}, sF, fshift, buf, row, lane);
      else
        bm_row_reverse(B.col, b0, dv, P, d, row, lane);
    }
    __syncthreads();
    // level 3 and beyond: one warp per row i
    // C buffers of the warp: R_i & R_j (5-cliques) or the chain's C_1 .. C_D (k >= 6)
    uint32_t* C = DMAX > 0 ? sC : gRows + (int64_t)d * S + (int64_t)wid * S * CL;
    if (DMAX == 0 && lane == 0) PGM_IDX_OK((int64_t)d * S + (int64_t)(wid + 1) * S * CL - 1, B.scratch_words);
    const int64_t cstride = DMAX > 0 ? 4 * S4MAX : S;
    // row j (32-bit offsets when the rows are in shared memory)
    auto row4 = [&](int j) {
      return reinterpret_cast<const uint4*>(DMAX > 0 ? R + j * S : R + (int64_t)j * S);
    };
    for (int i = wid; i < d; i += NW) {
      const uint32_t* Ri = reinterpret_cast<const uint32_t*>(row4(i));
      const uint4* Ri4 = row4(i);
      unsigned tri = 0;
      for (int w = lane; w < W; w += 32) tri += __popc(Ri[w]);
      if (B.k == 3) {
        c[0] += tri;
        continue;
      }
      c[1] += tri;
      int cnt = 0;
      if constexpr (KV == 6) {
        const int L = 4 * n4;
        bm_deep_walk<0>(Ri, B.k - 4, W, n4, C, cstride, row4, buf, buf2, L <= 32 ? min(32 / L, bm_c5(DMAX)) : 1,
                        lane, c[0], lvl);
      } else if constexpr (KV == 4) {
        // 4-cliques: |R_i & R_j| for every j in R_i, one j per lane
        auto f4 = [&](int j, bool valid) {
          if (valid) c[0] += bm_and_popc4(Ri4, row4(j), n4);
        };
        for (int w0 = 0; w0 < W; w0 += 32) {
          const uint32_t mine = w0 + lane < W ? Ri[w0 + lane] : 0u;
          bm_bits(mine, w0, buf, cnt, lane, f4);
        }
        bm_bits_tail(buf, cnt, lane, f4);
      } else {
        // 5-cliques: for each j in R_i (one at a time), C = R_i & R_j; then
        // |C & R_l| for every l in C, one l per lane
        // 5-cliques: the j's of R_i in groups of G, one group of L = 4 n4 lanes
        // per j (G = 32 / L, at most the warp's C buffers): C_j = R_i & R_j for
        // the whole group in one pass, then the pairs (C_j, l), l in C_j, of the
        // group 32 at a time, |C_j & R_l| one pair per lane
        const int L = 4 * n4;
        const int G = L <= 32 ? min(32 / L, CL) : 1;
        auto f5l = [&](int e, bool v2) {
          if (v2) {
            const uint32_t* Cg = C + (int64_t)(G > 1 ? (e >> 16) : 0) * cstride;
            c[0] += bm_and_popc4(reinterpret_cast<const uint4*>(Cg), row4(G > 1 ? (e & 0xffff) : e), n4);
          }
        };
        auto f5 = [&](int j, bool valid) {
          const int nvj = __popc(__ballot_sync(kFull, valid));  // valid lanes are a prefix
          for (int g0 = 0; g0 < nvj; g0 += G) {
            const int ng = min(G, nvj - g0);
            if (G > 1) {
              const int gi = lane / L, w = lane - gi * L;
              const int jq = __shfl_sync(kFull, j, min(g0 + gi, 31));
              unsigned cnt4 = 0;
              if (gi < ng) {
                const uint32_t x = Ri[w] & reinterpret_cast<const uint32_t*>(row4(jq))[w];  // padding words are zero
                C[gi * cstride + w] = x;
                cnt4 = __popc(x);
              }
              c[2] += cnt4;
            } else {
              const int jq = __shfl_sync(kFull, j, g0);
              const uint32_t* Rj = reinterpret_cast<const uint32_t*>(row4(jq));
              unsigned cnt4 = 0;
              for (int w = lane; w < L; w += 32) {
                const uint32_t x = Ri[w] & Rj[w];
                C[w] = x;
                cnt4 += __popc(x);
              }
              c[2] += cnt4;
            }
            __syncwarp();
            int cnt2 = 0;
            for (int gi = 0; gi < ng; gi++) {
              const uint32_t* Cg = C + (int64_t)gi * cstride;
              for (int w0 = 0; w0 < W; w0 += 32) {
                const uint32_t mine = w0 + lane < W ? Cg[w0 + lane] : 0u;
                bm_bits(mine, w0, buf2, cnt2, lane, f5l, gi);
              }
            }
            bm_bits_tail(buf2, cnt2, lane, f5l);
          }
        };
        for (int w0 = 0; w0 < W; w0 += 32) {
          const uint32_t mine = w0 + lane < W ? Ri[w0 + lane] : 0u;
          bm_bits(mine, w0, buf, cnt, lane, f5);
        }
        bm_bits_tail(buf, cnt, lane, f5);
      }
    }
    __syncthreads();
  }
  bm_flush(B, c, cur_g, lane);
  if constexpr (KV == 6) {
    const unsigned long long x = warp_sum(lvl[1]);  // level 4
    if (lane == 0 && x) atomicAdd(B.acc + 2, x);
    bm_deep_flush(B, lvl);
  }
  seen = warp_sum(seen);
  if (lane == 0 && seen) atomicAdd(B.stat, seen);
}

}  // namespace

// Words of row scratch per block of the global-row bucket: d rows plus 16
// warps' C buffers (1, or k - 4 for the walk of k >= 6), 4 * S4 words each.
int64_t bitset_row_words(int64_t dmax, int k) {
  const int clevels = k >= 6 ? k - 4 : 1;
  return (dmax + 16 * (int64_t)clevels) * 4 * (int64_t)bm_s4((int)((dmax + 31) / 32));
}

// Device bytes of that scratch for a count on g (0 when every out-list fits
// the shared-memory rows): the bucket kernel's persistent grid x the words
// per block, as count_kcliques_bitset reserves them.
int64_t bitset_scratch_bytes(const Graph& g, int k) {
  const int smem_d = options().bitset_smem_degree;
  if (k < 3 || g.dag_dmax <= smem_d) return 0;
  const int kv = k <= 4 ? 4 : (k == 5 ? 5 : 6);
  const int clevels = kv == 6 ? k - 4 : 1;
  const void* fn = kv == 4 ? (const void*)bm_block_kernel<0, 512, 4>
                           : (kv == 5 ? (const void*)bm_block_kernel<0, 512, 5> : (const void*)bm_block_kernel<0, 512, 6>);
  const size_t smem = bm_block_smem(0, 512, clevels);
  if (smem_attr(fn, (int)smem) != PGM_OK) return 0;
  return (int64_t)grid_for(fn, 512, smem) * bitset_row_words(g.dag_dmax, k) * 4;
}

// Streams and events for forking the bucket launches (per thread and
// device: a call's events must not be recorded by another thread's call).
constexpr int kForks = kBmBuckets;
struct ForkStreams {
  int dev = -1;
  cudaStream_t s[kForks] = {};
  cudaEvent_t ev[1 + kForks] = {};
};

pgm_status fork_streams(ForkStreams** out) {
  thread_local ForkStreams F[8];
  const int dev = device_id();
  *out = nullptr;
  if (dev < 0 || dev >= 8) return PGM_OK;  // no fork: launches stay on the caller's stream
  ForkStreams& f = F[dev];
  if (f.dev != dev) {
    for (int i = 0; i < kForks; i++) PGM_TRY_CUDA(cudaStreamCreateWithFlags(&f.s[i], cudaStreamNonBlocking));
    for (int i = 0; i <= kForks; i++) PGM_TRY_CUDA(cudaEventCreateWithFlags(&f.ev[i], cudaEventDisableTiming));
    f.dev = dev;
  }
  *out = &f;
  return PGM_OK;
}

// Bitset engine entry: counts k-cliques (k in 3..10) rooted in [v_lo, v_hi).
// Returns PGM_EUNSUPPORTED when the DAG's largest out-degree would need more
// than `max_scratch` bytes of row scratch (the caller then uses the
// level-list engine).
pgm_status count_kcliques_bitset(Graph& g, Workspace& ws, cudaStream_t s, int k, int32_t v_lo,
                                 int32_t v_hi, uint64_t* out, unsigned long long* per_graph_dev,
                                 uint64_t* level_sizes) {
  if (k < 3 || k > 4 + kDeepMax) return PGM_EUNSUPPORTED;
  const pgm_options o = options();
  const int smem_d = o.bitset_smem_degree;
  const int64_t dmax = g.dag_dmax;
  // bucket kernels: (64, 256], (256, 512], (512, 1024] with rows in shared
  // memory (each only up to smem_d), and the rest with rows in global memory
  struct Kern {
    const void* fn;
    int threads;
    size_t smem;
    int grid;
  };
  const int kv = k <= 4 ? 4 : (k == 5 ? 5 : 6);
  const int clevels = kv == 6 ? k - 4 : 1;
  // C buffers per warp of each bucket (5-cliques: a group of j's at once)
  auto cl = [&](int dm) { return kv == 5 ? bm_c5(dm) : (kv == 6 ? clevels - 1 + bm_c5(dm) : clevels); };
  auto pick = [kv](const void* f4, const void* f5, const void* f6) { return kv == 4 ? f4 : (kv == 5 ? f5 : f6); };
  Kern kern[kBmBuckets] = {
      {pick((const void*)bm_block_kernel<256, 256, 4>, (const void*)bm_block_kernel<256, 256, 5>,
            (const void*)bm_block_kernel<256, 256, 6>),
       256, bm_block_smem(256, 256, cl(256)), 0},
      {pick((const void*)bm_block_kernel<512, 512, 4>, (const void*)bm_block_kernel<512, 512, 5>,
            (const void*)bm_block_kernel<512, 512, 6>),
       512, bm_block_smem(512, 512, cl(512)), 0},
      {pick((const void*)bm_block_kernel<1024, 1024, 4>, (const void*)bm_block_kernel<1024, 1024, 5>,
            (const void*)bm_block_kernel<1024, 1024, 6>),
       1024, bm_block_smem(1024, 1024, cl(1024)), 0},
      {pick((const void*)bm_block_kernel<0, 512, 4>, (const void*)bm_block_kernel<0, 512, 5>,
            (const void*)bm_block_kernel<0, 512, 6>),
       512, bm_block_smem(0, 512, clevels), 0},
  };
  const void* warp_fn = kv == 6 ? (const void*)bm_warp_kernel<true> : (const void*)bm_warp_kernel<false>;

  // buckets this count launches (largest out-degree first, see below); a
  // bucket whose shared memory exceeds the device's per-block opt-in limit
  // makes the engine decline (the caller falls back to the level lists)
  bool used[kBmBuckets];
  for (int b = 0; b < kBmBuckets; b++) used[b] = b < 3 ? (b == 0 ? 64 : (b == 1 ? 256 : 512)) < smem_d : dmax > smem_d;
  int optin = 0;
  PGM_TRY_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device_id()));
  for (int b = 0; b < kBmBuckets; b++) {
    if (!used[b]) continue;
    if (kern[b].smem > (size_t)optin) {
      set_error("bitset engine: bucket %d needs %zu B of shared memory per block (device limit %d)", b,
                kern[b].smem, optin);
      return PGM_EUNSUPPORTED;
    }
    PGM_TRY(smem_attr(kern[b].fn, (int)kern[b].smem));
    kern[b].grid = grid_for(kern[b].fn, kern[b].threads, kern[b].smem);
  }
  // global-row bucket: d rows plus 16 warps' C buffers per block, 4 * S4 words each
  const int64_t words = dmax > smem_d ? bitset_row_words(dmax, k) : 0;
  if (words > 0 && (double)kern[3].grid * (double)words * 4.0 > 8.0 * (double)(1ull << 30)) {
    set_error("bitset engine: out-degree %lld needs too much row scratch", (long long)dmax);
    return PGM_EUNSUPPORTED;
  }
  // bucket lists: at most arcs / (lower bound + 1) vertices exceed each lower bound
  int64_t arcs = 0;
  PGM_TRY(graph_dag_arcs(g, v_lo, v_hi, &arcs));
  const int64_t nv = (int64_t)v_hi - v_lo;
  const int64_t lo[kBmBuckets] = {kBmWarpD, 256, 512, smem_d};
  BmArgs B;
  memset(&B, 0, sizeof(B));
  int64_t total = 0;
  for (int b = 0; b < kBmBuckets; b++) {
    B.big_off[b] = total;
    B.big_cap[b] = std::min<int64_t>(nv, arcs / (lo[b] + 1)) + 1;
    total += B.big_cap[b];
  }
  PGM_TRY(ws.ctr.reserve(kBmSlots));
  PGM_TRY(ws.big.reserve((size_t)(total + 1) / 2 + 1));
  if (words > 0) PGM_TRY(ws.vid[11].reserve((size_t)kern[3].grid * (size_t)words));
  PGM_TRY_CUDA(cudaMemsetAsync(ws.ctr.p, 0, kBmSlots * sizeof(unsigned long long), s));
  if (!per_graph_dev) PGM_TRY(seed_counts(ws.ctr.p + 8, 1, s));
  B.carry = ws.ctr.p + kCarrySlot;
  B.rp = g.dag_rp;
  B.col = g.dag_col;
  B.v_lo = v_lo;
  B.v_hi = v_hi;
  B.k = k;
  B.acc = ws.ctr.p + 8;
  B.queue = ws.ctr.p;
  B.err = ws.ctr.p + 15;
  B.big = reinterpret_cast<int32_t*>(ws.big.p);
  B.smem_d = smem_d;
  B.fwd_ratio = o.bitset_forward_ratio;
  B.scratch = words > 0 ? reinterpret_cast<uint32_t*>(ws.vid[11].p) : nullptr;
  B.scratch_words = words;
  B.stat = ws.ctr.p + 12;
  B.gid = g.gid;
  B.per_graph = per_graph_dev;
  B.deep = ws.ctr.p + kDeepLvl;
  B.clevels = clevels;
  int wgrid = grid_for(warp_fn, 256, 0);
  // kBmGrab vertices per grab, fewer when the graph has too few vertices to
  // give every resident warp that many (a small graph's run time is the
  // chain of row builds of one warp's vertices)
  B.grab = (int)std::max<int64_t>(1, std::min<int64_t>(kBmGrab, nv / ((int64_t)wgrid * 8)));
  wgrid = (int)std::max<int64_t>(1, std::min<int64_t>(wgrid, ((nv + B.grab - 1) / B.grab + 7) / 8));
  // The buckets depend on their vertex lists (filled by the warp kernel, or
  // beforehand by bm_classify_kernel) but not on one another: outside a
  // stream capture or a plan recording they run on forked streams, so that
  // one bucket's tail overlaps the next.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  PGM_TRY_CUDA(cudaStreamIsCapturing(s, &cap));
  ForkStreams* F = nullptr;
  if (cap == cudaStreamCaptureStatusNone && !current_plan()) PGM_TRY(fork_streams(&F));
  Profiler& prof = profiler();
  int id = prof.begin("bitset_count", 3);
  if (nv > 0) {
    void* wargv[] = {&B};
    // forked, with bucket vertices present and a DAG that fits the L2: the
    // bucket lists first (one thread per vertex), then the warp kernel on
    // the caller's stream and the bucket kernels on the forked streams, all
    // at once.  (Measured: R-MAT 21, a 120 MB DAG, 20.60 -> 20.46 ms; R-MAT
    // scale 24, 0.7 GB, 167 -> 171 ms, the warp kernel's scattered reads
    // then sharing the L2 with the buckets' rows: there the buckets wait.)
    const int64_t dag_bytes = 4 * ((int64_t)g.narcs / 2 + (int64_t)g.n + 1);
    const bool pre = F && g.dag_dmax > kBmWarpD && dag_bytes <= l2_bytes();
    B.classified = pre ? 1 : 0;
    if (pre) {
      const int cgrid = (int)std::max<int64_t>(1, std::min<int64_t>((nv + 255) / 256, 8LL * num_sms()));
      bm_classify_kernel<<<cgrid, 256, 0, s>>>(B);
      PGM_CHECK_LAUNCH();
      PGM_TRY_CUDA(cudaEventRecord(F->ev[0], s));
    }
    PGM_TRY_CUDA(cudaLaunchKernel(warp_fn, dim3(wgrid), dim3(256), wargv, 0, s));
    PGM_CHECK_LAUNCH();
    if (F && !pre) PGM_TRY_CUDA(cudaEventRecord(F->ev[0], s));
    // largest rows first, so that the short tail of each launch is cheap
    int nf = 0;
    for (int b = kBmBuckets - 1; b >= 0; b--) {
      if (!used[b]) continue;               // bucket unused at this shared-memory limit
      if (g.dag_dmax <= lo[b]) continue;    // no out-degree reaches the bucket
      const Kern& K = kern[b];
      void* argv[] = {&B, &b};
      cudaStream_t t = s;
      if (F && nf < kForks) {
        t = F->s[nf];
        PGM_TRY_CUDA(cudaStreamWaitEvent(t, F->ev[0], 0));
      }
      PGM_TRY_CUDA(cudaLaunchKernel(K.fn, dim3(K.grid), dim3(K.threads), argv, K.smem, t));
      PGM_CHECK_LAUNCH();
      if (t != s) {
        PGM_TRY_CUDA(cudaEventRecord(F->ev[1 + nf], t));
        nf++;
      }
    }
    for (int i = 0; i < nf; i++) PGM_TRY_CUDA(cudaStreamWaitEvent(s, F->ev[1 + i], 0));
  }
  prof.end(id, (double)arcs, 0.0);
  unsigned long long h[kBmSlots];
  bool deferred = false;
  PGM_TRY(read_counters(ws.ctr.p, h, kBmSlots, s, &deferred));
  if (deferred) return PGM_OK;
  if (h[15]) {
    set_error("bitset engine: internal big-vertex list overflow");
    return PGM_ENOMEM;
  }
  if (h[kCarrySlot]) {
    set_error("count_kcliques: the count exceeds 2^64 - 1");
    return PGM_EOVERFLOW;
  }
  *out = h[8] - (per_graph_dev ? 0ull : count_seed());
  if (level_sizes) {  // [l] entries of level l (3 <= l < k), [kBmLevelRead] adjacency elements read
    level_sizes[3] = h[9];
    level_sizes[4] = h[10];
    for (int l = 5; l < k; l++) level_sizes[l] = h[kDeepLvl + (l - 3)];
    level_sizes[kBmLevelRead] = h[12];
  }
  return PGM_OK;
}

}  // namespace pgm
