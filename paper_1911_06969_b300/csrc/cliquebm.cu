// cliquebm.cu -- k-clique counting (k = 3, 4, 5) with bitset level lists.
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
// counters of bucket b, [8..10] counts, [12] statistics, [15] error
constexpr int kQPop = 1, kQPush = 16, kBmBuckets = 4, kBmSlots = 20;

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
      if (i == 0 && B.per_graph && g >= 0)
        atomicAdd(B.per_graph + g, s);
      else
        atomicAdd(B.acc + i, s);
    }
    c[i] = 0;
  }
}

// position of x in the sorted list P (length d), or -1
__device__ __forceinline__ int find_pos(const int32_t* P, int d, int32_t x) {
  if (d == 0 || x < P[0] || x > P[d - 1]) return -1;
  const int i = lower_bound_dev(P, d, x);
  return (i < d && P[i] == x) ? i : -1;
}

// Build rows R_i (i in [i0, i1), step `step`) of vertex set P (length d) into
// rows[i * stride + w]; one warp per row, lanes scan the shorter side.
// Rows must be zeroed beforehand (forward sets bits with atomicOr).
__device__ __forceinline__ void build_rows(const BmArgs& B, const int32_t* P, int d, uint32_t* rows,
                                           int stride, int i0, int i1, int step, int lane,
                                           unsigned long long& seen) {
  for (int i = i0; i < i1; i += step) {
    const int32_t v = P[i];
    const int32_t a0 = B.rp[v], dv = B.rp[v + 1] - a0;
    uint32_t* row = rows + (int64_t)i * stride;
    if (lane == 0) seen += (unsigned long long)dv;
    if (dv <= 2 * d) {
      // forward: each out-neighbour of v found in P sets its bit
      for (int t = lane; t < dv; t += 32) {
        const int j = find_pos(P, d, B.col[a0 + t]);
        if (j >= 0) atomicOr(row + (j >> 5), 1u << (j & 31));
      }
    } else {
      // reverse: one ballot word per 32 positions of P
      for (int j0 = 0; j0 < d; j0 += 32) {
        const int j = j0 + lane;
        const bool in = j < d && contains_dev(B.col + a0, dv, P[j]);
        const unsigned b = __ballot_sync(kFull, in);
        if (lane == 0 && b) row[j0 >> 5] |= b;
      }
    }
  }
}

// ----------------------------------------------------------- warp kernel
// One vertex per warp, d <= 64: P and the rows (2 words, stride 2) in shared memory.
__global__ void __launch_bounds__(256) bm_warp_kernel(BmArgs B) {
  __shared__ int32_t sP[8][kBmWarpD];
  __shared__ uint32_t sR[8][kBmWarpD * 2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t* P = sP[wid];
  uint32_t* R = sR[wid];
  unsigned long long c[3] = {0, 0, 0};
  unsigned long long seen = 0;
  int cur_g = -1;
  const int64_t np = (int64_t)B.v_hi - B.v_lo;
  for (;;) {
    unsigned long long p0 = 0;
    if (lane == 0) p0 = atomicAdd(B.queue, (unsigned long long)kBmGrab);
    p0 = __shfl_sync(kFull, p0, 0);
    if ((int64_t)p0 >= np) break;
    const int64_t pend = min((int64_t)p0 + kBmGrab, np);
    for (int64_t pi = (int64_t)p0; pi < pend; pi++) {
      const int32_t u = (int32_t)(B.v_lo + pi);
      const int32_t a0 = B.rp[u];
      const int d = B.rp[u + 1] - a0;
      if (d < 2) continue;  // no triangle (hence no level-3 entry) rooted at u
      if (d > kBmWarpD) {
        if (lane == 0) {
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
      for (int i = lane; i < d; i += 32) P[i] = B.col[a0 + i];
      for (int i = lane; i < 2 * kBmWarpD; i += 32) R[i] = 0;
      __syncwarp();
      build_rows(B, P, d, R, 2, 0, d, 1, lane, seen);
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
  seen = warp_sum(seen);
  if (lane == 0 && seen) atomicAdd(B.stat, seen);
}

// ---------------------------------------------------------- block kernels
// One big vertex (d > 64) per block, in buckets by out-degree so that the
// block size and shared memory fit the rows: DMAX > 0 keeps P, a hash map
// from vertex to position in P, and the rows (W words at stride W + 1, odd
// so that rows spread over the banks) in shared memory; DMAX = 0 keeps P
// and the rows in global memory (the per-block scratch) and finds
// positions by binary search.

// Open-addressing hash map from vertex to its position in P (linear
// probing, at most a quarter full, so the table always has empty slots).
__device__ __forceinline__ uint32_t bm_hash(int32_t x, int shift) {
  return ((uint32_t)x * 0x9E3779B1u) >> shift;
}

__device__ __forceinline__ int bm_hfind(const int32_t* key, const uint16_t* pos, uint32_t mask, int shift,
                                        int32_t x) {
  uint32_t h = bm_hash(x, shift);
  for (uint32_t probe = 0; probe <= mask; probe++) {
    const int32_t k = key[h];
    if (k == x) return pos[h];
    if (k < 0) return -1;
    h = (h + 1) & mask;
  }
  return -1;
}

// Set bits of a row, 32 at a time: appends the set bits of the 32 words
// held one per lane (`mine`, words w0 .. w0 + 31) to the warp's buffer
// (64 entries) and calls f(j, true) on every lane for each full group of
// 32 positions j.  bm_bits_tail() hands over the last partial group.
template <class F>
__device__ __forceinline__ void bm_bits(uint32_t mine, int w0, int* buf, int& cnt, int lane, F& f) {
  uint32_t nz = __ballot_sync(kFull, mine != 0u);
  while (nz) {
    const int q = __ffs(nz) - 1;
    nz &= nz - 1;
    const uint32_t word = __shfl_sync(kFull, mine, q);
    if ((word >> lane) & 1u) buf[cnt + __popc(word & ((1u << lane) - 1u))] = ((w0 + q) << 5) + lane;
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

// Shared-memory bytes of bm_block_kernel<DMAX, THREADS>.
__host__ __device__ constexpr size_t bm_block_smem(int dmax, int threads) {
  return dmax > 0 ? (size_t)4 * dmax                       // P
                        + (size_t)(4 + 2) * 4 * dmax        // hash keys + positions (4 dmax slots)
                        + (size_t)4 * (threads / 32) * 128  // two 64-entry bit buffers per warp
                        + (size_t)4 * (threads / 32) * (dmax / 32 + 1)  // C = R_i & R_j per warp
                        + (size_t)4 * dmax * (dmax / 32 + 1)            // rows
                  : (size_t)4 * (threads / 32) * 128;
}

// resident blocks per SM that the register budget is sized for
__host__ __device__ constexpr int bm_min_blocks(int dmax, int threads) {
  return dmax == 0 ? 2 : (threads <= 256 ? 6 : (threads <= 512 ? 3 : 1));
}

template <int DMAX, int THREADS>
__global__ void __launch_bounds__(THREADS, bm_min_blocks(DMAX, THREADS)) bm_block_kernel(BmArgs B, int bucket) {
  constexpr int NW = THREADS / 32;
  constexpr int HT = 4 * DMAX;
  extern __shared__ uint32_t smem_u[];
  __shared__ long long sh_idx;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t* sP = reinterpret_cast<int32_t*>(smem_u);
  int32_t* sKey = sP + DMAX;
  uint16_t* sPos = reinterpret_cast<uint16_t*>(sKey + HT);
  int* buf = reinterpret_cast<int*>(smem_u) + (DMAX > 0 ? DMAX + HT + HT / 2 : 0) + wid * 128;
  int* buf2 = buf + 64;
  uint32_t* sC = reinterpret_cast<uint32_t*>(smem_u) + (DMAX > 0 ? DMAX + HT + HT / 2 : 0) + NW * 128 +
                 wid * (DMAX / 32 + 1);
  uint32_t* sRows = reinterpret_cast<uint32_t*>(smem_u) + DMAX + HT + HT / 2 + NW * 128 + NW * (DMAX / 32 + 1);
  uint32_t* gRows = B.scratch ? B.scratch + (int64_t)blockIdx.x * B.scratch_words : nullptr;
  unsigned long long c[3] = {0, 0, 0};
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
    const int W = (d + 31) >> 5, stride = W + 1;
    if (B.gid) {
      const int g = B.gid[u];
      if (g != cur_g) {
        bm_flush(B, c, cur_g, lane);
        cur_g = g;
      }
    }
    const int32_t* P;
    uint32_t* R;
    uint32_t hmask = 0;
    int hshift = 0;
    if constexpr (DMAX > 0) {
      int T = 32;
      while (T < 4 * d) T <<= 1;
      hmask = (uint32_t)T - 1u;
      hshift = 32 - __ffs(T) + 1;
      for (int i = threadIdx.x; i < d; i += THREADS) sP[i] = B.col[a0 + i];
      for (int i = threadIdx.x; i < T; i += THREADS) sKey[i] = -1;
      for (int i = threadIdx.x; i < d * stride; i += THREADS) sRows[i] = 0;
      __syncthreads();
      for (int i = threadIdx.x; i < d; i += THREADS) {
        const int32_t x = sP[i];
        uint32_t h = bm_hash(x, hshift);
        for (int probe = 0; probe < T; probe++) {
          if (atomicCAS(sKey + h, -1, x) == -1) {
            sPos[h] = (uint16_t)i;
            break;
          }
          h = (h + 1) & hmask;
        }
      }
      P = sP;
      R = sRows;
    } else {
      for (int64_t i = threadIdx.x; i < (int64_t)d * stride; i += THREADS) gRows[i] = 0;
      P = B.col + a0;
      R = gRows;
    }
    __syncthreads();
    // rows R_i = N+(P[i]) & P, one warp per row
    const int32_t plo = P[0], phi = P[d - 1];
    for (int i = wid; i < d; i += NW) {
      const int32_t v = P[i];
      const int32_t b0 = B.rp[v], dv = B.rp[v + 1] - b0;
      uint32_t* row = R + (int64_t)i * stride;
      if (lane == 0) seen += (unsigned long long)dv;
      if (dv <= B.fwd_ratio * d) {
        // forward: each out-neighbour of v found in P sets its bit
        for (int t0 = 0; t0 < dv; t0 += 128) {
          int32_t x[4];
#pragma unroll
          for (int r = 0; r < 4; r++) {
            const int t = t0 + r * 32 + lane;
            x[r] = t < dv ? B.col[b0 + t] : -1;
          }
#pragma unroll
          for (int r = 0; r < 4; r++) {
            if (x[r] < plo || x[r] > phi) continue;
            int j;
            if constexpr (DMAX > 0) {
              j = bm_hfind(sKey, sPos, hmask, hshift, x[r]);
            } else {
              j = find_pos(P, d, x[r]);
            }
            if (j >= 0) atomicOr(row + (j >> 5), 1u << (j & 31));
          }
        }
      } else {
        // reverse: one ballot word per 32 positions of P
        for (int j0 = 0; j0 < d; j0 += 32) {
          const int j = j0 + lane;
          const bool in = j < d && contains_dev(B.col + b0, dv, P[j]);
          const unsigned bal = __ballot_sync(kFull, in);
          if (lane == 0 && bal) row[j0 >> 5] |= bal;
        }
      }
    }
    __syncthreads();
    // level 3 and beyond: one warp per row i
    for (int i = wid; i < d; i += NW) {
      const uint32_t* Ri = R + (int64_t)i * stride;
      if constexpr (DMAX > 0) {
        // W <= 32: word w of R_i is held by lane w
        const uint32_t ri = lane < W ? Ri[lane] : 0u;
        if (B.k == 3) {
          c[0] += (unsigned long long)__popc(ri);
          continue;
        }
        c[1] += (unsigned long long)__popc(ri);
        const uint32_t nzi = __ballot_sync(kFull, ri != 0u);
        if (!nzi) continue;
        int cnt = 0;
        if (B.k == 4) {
          // 4-cliques: |R_i & R_j| for every j in R_i, one j per lane
          auto f4 = [&](int j, bool valid) {
            if (!valid) return;
            const uint32_t* Rj = R + (int64_t)j * stride;
            unsigned s = 0;
            for (uint32_t m = nzi; m; m &= m - 1) {
              const int w = __ffs(m) - 1;
              s += __popc(Ri[w] & Rj[w]);
            }
            c[0] += s;
          };
          bm_bits(ri, 0, buf, cnt, lane, f4);
          bm_bits_tail(buf, cnt, lane, f4);
        } else {
          // 5-cliques: for each j in R_i (one at a time), C = R_i & R_j held
          // one word per lane; then |C & R_l| for every l in C, one l per lane
          auto f5 = [&](int j, bool valid) {
            for (unsigned mq = __ballot_sync(kFull, valid); mq; mq &= mq - 1) {
              const int q = __ffs(mq) - 1;
              const int jq = __shfl_sync(kFull, j, q);
              const uint32_t* Rj = R + (int64_t)jq * stride;
              const uint32_t cw = lane < W ? (ri & Rj[lane]) : 0u;
              c[2] += (unsigned long long)__popc(cw);
              const uint32_t nzc = __ballot_sync(kFull, cw != 0u);
              if (!nzc) continue;
              if (lane < W) sC[lane] = cw;
              __syncwarp();
              int cnt2 = 0;
              auto f5l = [&](int l, bool v2) {
                if (!v2) return;
                const uint32_t* Rl = R + (int64_t)l * stride;
                unsigned s = 0;
                for (uint32_t m = nzc; m; m &= m - 1) {
                  const int w = __ffs(m) - 1;
                  s += __popc(sC[w] & Rl[w]);
                }
                c[0] += s;
              };
              bm_bits(cw, 0, buf2, cnt2, lane, f5l);
              bm_bits_tail(buf2, cnt2, lane, f5l);
            }
          };
          bm_bits(ri, 0, buf, cnt, lane, f5);
          bm_bits_tail(buf, cnt, lane, f5);
        }
      } else {
        // rows in global memory, W > 32 words
        unsigned long long tri = 0;
        for (int w = lane; w < W; w += 32) tri += (unsigned long long)__popc(Ri[w]);
        if (B.k == 3) {
          c[0] += tri;
          continue;
        }
        c[1] += tri;
        int cnt = 0;
        if (B.k == 4) {
          auto f4 = [&](int j, bool valid) {
            if (!valid) return;
            const uint32_t* Rj = R + (int64_t)j * stride;
            unsigned long long s = 0;
            for (int w = 0; w < W; w++) {
              const uint32_t x = Ri[w];
              if (x) s += (unsigned long long)__popc(x & Rj[w]);
            }
            c[0] += s;
          };
          for (int w0 = 0; w0 < W; w0 += 32) {
            const uint32_t mine = w0 + lane < W ? Ri[w0 + lane] : 0u;
            bm_bits(mine, w0, buf, cnt, lane, f4);
          }
          bm_bits_tail(buf, cnt, lane, f4);
        } else {
          uint32_t* C = gRows + (int64_t)d * stride + (int64_t)wid * stride;
          auto f5 = [&](int j, bool valid) {
            for (unsigned mq = __ballot_sync(kFull, valid); mq; mq &= mq - 1) {
              const int q = __ffs(mq) - 1;
              const int jq = __shfl_sync(kFull, j, q);
              const uint32_t* Rj = R + (int64_t)jq * stride;
              unsigned long long cnt4 = 0;
              for (int w = lane; w < W; w += 32) {
                const uint32_t x = Ri[w] & Rj[w];
                C[w] = x;
                cnt4 += (unsigned long long)__popc(x);
              }
              c[2] += cnt4;
              __syncwarp();
              int cnt2 = 0;
              auto f5l = [&](int l, bool v2) {
                if (!v2) return;
                const uint32_t* Rl = R + (int64_t)l * stride;
                unsigned long long s = 0;
                for (int w = 0; w < W; w++) {
                  const uint32_t x = C[w];
                  if (x) s += (unsigned long long)__popc(x & Rl[w]);
                }
                c[0] += s;
              };
              for (int w0 = 0; w0 < W; w0 += 32) {
                const uint32_t mine = w0 + lane < W ? C[w0 + lane] : 0u;
                bm_bits(mine, w0, buf2, cnt2, lane, f5l);
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
    }
    __syncthreads();
  }
  bm_flush(B, c, cur_g, lane);
  seen = warp_sum(seen);
  if (lane == 0 && seen) atomicAdd(B.stat, seen);
}

}  // namespace

// Bitset engine entry: counts k-cliques (k in 3..5) rooted in [v_lo, v_hi).
// Returns PGM_EUNSUPPORTED when the DAG's largest out-degree would need more
// than `max_scratch` bytes of row scratch (the caller then uses the
// level-list engine).
pgm_status count_kcliques_bitset(Graph& g, Workspace& ws, cudaStream_t s, int k, int32_t v_lo,
                                 int32_t v_hi, uint64_t* out, unsigned long long* per_graph_dev,
                                 uint64_t* level_sizes) {
  if (k < 3 || k > 5) return PGM_EUNSUPPORTED;
  const pgm_options o = options();
  const int smem_d = o.bitset_smem_degree;
  const int64_t dmax = g.dag_dmax;
  const int64_t Wmax = (dmax + 31) / 32;
  // bucket kernels: (64, 256], (256, 512], (512, 1024] with rows in shared
  // memory (each only up to smem_d), and the rest with rows in global memory
  struct Kern {
    const void* fn;
    int threads;
    size_t smem;
    int grid;
  };
  Kern kern[kBmBuckets] = {
      {(const void*)bm_block_kernel<256, 256>, 256, bm_block_smem(256, 256), 0},
      {(const void*)bm_block_kernel<512, 512>, 512, bm_block_smem(512, 512), 0},
      {(const void*)bm_block_kernel<1024, 1024>, 1024, bm_block_smem(1024, 1024), 0},
      {(const void*)bm_block_kernel<0, 512>, 512, bm_block_smem(0, 512), 0},
  };
  for (int b = 0; b < kBmBuckets; b++) {
    PGM_TRY(smem_attr(kern[b].fn, (int)kern[b].smem));
    kern[b].grid = grid_for(kern[b].fn, kern[b].threads, kern[b].smem);
  }
  // global-row bucket: d * (W + 1) row words plus 16 warps' C buffers per block
  const int64_t words = dmax > smem_d ? (dmax + 16) * (Wmax + 1) : 0;
  if (words > 0 && (double)kern[3].grid * (double)words * 4.0 > 8.0 * (double)(1ull << 30)) {
    set_error("bitset engine: out-degree %lld needs too much row scratch", (long long)dmax);
    return PGM_EUNSUPPORTED;
  }
  // bucket lists: at most arcs / (lower bound + 1) vertices exceed each lower bound
  const int64_t arcs = g.h_dag_rp[v_hi] - g.h_dag_rp[v_lo];
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
  int wgrid = grid_for((const void*)bm_warp_kernel, 256, 0);
  wgrid = (int)std::max<int64_t>(1, std::min<int64_t>(wgrid, ((nv + kBmGrab - 1) / kBmGrab + 7) / 8));
  Profiler& prof = profiler();
  int id = prof.begin("bitset_count", 3);
  if (nv > 0) {
    bm_warp_kernel<<<wgrid, 256, 0, s>>>(B);
    PGM_CHECK_LAUNCH();
    // largest rows first, so that the short tail of each launch is cheap
    for (int b = kBmBuckets - 1; b >= 0; b--) {
      if (b < 3 && lo[b] >= smem_d) continue;  // bucket unused at this shared-memory limit
      if (b == 3 && dmax <= smem_d) continue;
      const Kern& K = kern[b];
      if (b == 0) bm_block_kernel<256, 256><<<K.grid, K.threads, K.smem, s>>>(B, b);
      if (b == 1) bm_block_kernel<512, 512><<<K.grid, K.threads, K.smem, s>>>(B, b);
      if (b == 2) bm_block_kernel<1024, 1024><<<K.grid, K.threads, K.smem, s>>>(B, b);
      if (b == 3) bm_block_kernel<0, 512><<<K.grid, K.threads, K.smem, s>>>(B, b);
      PGM_CHECK_LAUNCH();
    }
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
  *out = h[8];
  if (level_sizes) {
    level_sizes[0] = h[9];   // level 3 (triangles) for k >= 4
    level_sizes[1] = h[10];  // level 4 (4-cliques) for k = 5
    level_sizes[2] = h[12];  // adjacency elements read
  }
  return PGM_OK;
}

}  // namespace pgm
