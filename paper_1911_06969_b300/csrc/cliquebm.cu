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
constexpr int kBmSmemD = 512;    // block kernel: rows in shared memory up to this d
constexpr int kBmGrab = 8;

struct BmArgs {
  const int32_t* rp;   // DAG
  const int32_t* col;
  int32_t v_lo, v_hi;
  int k;
  unsigned long long* acc;    // [0] k-cliques, [1] level-3 entries, [2] level-4 entries
  unsigned long long* queue;  // [0] warp queue, [1] block queue, [2] big count
  unsigned long long* err;
  int32_t* big;
  int64_t big_cap;
  uint32_t* scratch;          // per-block rows for d > kBmSmemD
  int64_t scratch_words;      // words per block
  int64_t stat_elems;         // unused on device
  unsigned long long* stat;   // adjacency elements read while building rows
  const int32_t* gid;
  unsigned long long* per_graph;
};

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
          unsigned long long x = atomicAdd(B.queue + 2, 1ull);
          if ((int64_t)x < B.big_cap)
            B.big[x] = u;
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

// ---------------------------------------------------------- block kernel
// One big vertex (d > 64) per block.  Rows of W words at stride W + 1 (odd,
// spreads shared-memory banks); in shared memory when d <= kBmSmemD.
__global__ void __launch_bounds__(512) bm_block_kernel(BmArgs B) {
  extern __shared__ uint32_t smem_u[];
  __shared__ long long sh_idx;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // layout: P[kBmSmemD] | per-warp C[kBmSmemD/32 + 1] | rows (d * (W+1) words, d <= kBmSmemD)
  int32_t* sP = reinterpret_cast<int32_t*>(smem_u);
  uint32_t* sC = smem_u + kBmSmemD + wid * (kBmSmemD / 32 + 1);
  uint32_t* sRows = smem_u + kBmSmemD + nw * (kBmSmemD / 32 + 1);
  uint32_t* gRows = B.scratch + (int64_t)blockIdx.x * B.scratch_words;
  unsigned long long c[3] = {0, 0, 0};
  unsigned long long seen = 0;
  int cur_g = -1;
  const long long nbig = min((long long)B.queue[2], (long long)B.big_cap);
  for (;;) {
    if (threadIdx.x == 0) sh_idx = (long long)atomicAdd(B.queue + 1, 1ull);
    __syncthreads();
    const long long idx = sh_idx;
    __syncthreads();
    if (idx >= nbig) break;
    const int32_t u = B.big[idx];
    const int32_t a0 = B.rp[u];
    const int d = B.rp[u + 1] - a0;
    const int W = (d + 31) >> 5, stride = W + 1;
    const int32_t* P;
    if (d <= kBmSmemD) {
      for (int i = threadIdx.x; i < d; i += blockDim.x) sP[i] = B.col[a0 + i];
      P = sP;
    } else {
      P = B.col + a0;
    }
    uint32_t* R = d <= kBmSmemD ? sRows : gRows;
    // per-warp candidate buffer for 5-cliques: shared memory when it fits
    uint32_t* C = d <= kBmSmemD ? sC : gRows + (int64_t)d * stride + (int64_t)wid * stride;
    for (int64_t i = threadIdx.x; i < (int64_t)d * stride; i += blockDim.x) R[i] = 0;
    if (B.gid) {
      const int g = B.gid[u];
      if (g != cur_g) {
        bm_flush(B, c, cur_g, lane);
        cur_g = g;
      }
    }
    __syncthreads();
    build_rows(B, P, d, R, stride, wid, d, nw, lane, seen);
    __syncthreads();
    // level 3 and beyond: warps take rows i
    for (int i = wid; i < d; i += nw) {
      const uint32_t* Ri = R + (int64_t)i * stride;
      unsigned long long tri = 0;
      for (int w = lane; w < W; w += 32) tri += (unsigned long long)__popc(Ri[w]);
      if (B.k == 3) {
        c[0] += tri;
        continue;
      }
      c[1] += tri;
      // the set bits j of R_i, 32 at a time (one per lane)
      for (int w0 = 0; w0 < W; w0++) {
        const uint32_t word = Ri[w0];
        if (!word) continue;
        // lane takes the lane-th set bit of this word, if any
        const int nb = __popc(word);
        int j = -1;
        if (lane < nb) {
          uint32_t x = word;
          for (int r = 0; r < lane; r++) x &= x - 1;
          j = (w0 << 5) + __ffs(x) - 1;
        }
        if (B.k == 4) {
          if (j >= 0) {
            const uint32_t* Rj = R + (int64_t)j * stride;
            unsigned long long s = 0;
            for (int w = 0; w < W; w++) s += (unsigned long long)__popc(Ri[w] & Rj[w]);
            c[0] += s;
          }
        } else {
          // 5-cliques: for each j, C = R_i & R_j; lanes then split C's set bits
          for (int q = 0; q < nb; q++) {
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
            for (int w1 = 0; w1 < W; w1++) {
              const uint32_t cw = C[w1];
              if (!cw) continue;
              const int nb2 = __popc(cw);
              if (lane < nb2) {
                uint32_t x = cw;
                for (int r = 0; r < lane; r++) x &= x - 1;
                const int l = (w1 << 5) + __ffs(x) - 1;
                const uint32_t* Rl = R + (int64_t)l * stride;
                unsigned long long s = 0;
                for (int w = 0; w < W; w++) s += (unsigned long long)__popc(C[w] & Rl[w]);
                c[0] += s;
              }
            }
            __syncwarp();
          }
        }
      }
    }
    __syncthreads();
  }
  bm_flush(B, c, cur_g, lane);
  seen = warp_sum(seen);
  if (lane == 0 && seen) atomicAdd(B.stat, seen);
}

constexpr int kBmSlots = 16;  // [0..3] queues, [8..10] counts, [12] stat, [15] err

}  // namespace

// Bitset engine entry: counts k-cliques (k in 3..5) rooted in [v_lo, v_hi).
// Returns PGM_EUNSUPPORTED when the DAG's largest out-degree would need more
// than `max_scratch` bytes of row scratch (the caller then uses the
// level-list engine).
pgm_status count_kcliques_bitset(Graph& g, Workspace& ws, cudaStream_t s, int k, int32_t v_lo,
                                 int32_t v_hi, uint64_t* out, unsigned long long* per_graph_dev,
                                 uint64_t* level_sizes) {
  if (k < 3 || k > 5) return PGM_EUNSUPPORTED;
  const int64_t dmax = g.dag_dmax;
  const int64_t Wmax = (dmax + 31) / 32;
  // big-vertex rows in global memory: d * (W + 1) words plus 16 warps' C buffers
  const int64_t words = dmax > kBmSmemD ? (dmax + 16) * (Wmax + 1) : 0;
  const int bthreads = 512;
  const size_t bsmem = (size_t)(kBmSmemD + 16 * (kBmSmemD / 32 + 1) +
                                (int64_t)kBmSmemD * (kBmSmemD / 32 + 1)) * sizeof(uint32_t);
  PGM_TRY(smem_attr((const void*)bm_block_kernel, (int)bsmem));
  const int bgrid = grid_for((const void*)bm_block_kernel, bthreads, bsmem);
  if (words > 0 && (double)bgrid * (double)words * 4.0 > 8.0 * (double)(1ull << 30)) {
    set_error("bitset engine: out-degree %lld needs too much row scratch", (long long)dmax);
    return PGM_EUNSUPPORTED;
  }
  PGM_TRY(ws.ctr.reserve(kBmSlots));
  PGM_TRY(ws.big.reserve((size_t)std::max<int64_t>(g.n / 2 + 2, 2)));
  if (words > 0) PGM_TRY(ws.vid[11].reserve((size_t)bgrid * (size_t)words));
  PGM_TRY_CUDA(cudaMemsetAsync(ws.ctr.p, 0, kBmSlots * sizeof(unsigned long long), s));
  BmArgs B;
  memset(&B, 0, sizeof(B));
  B.rp = g.dag_rp;
  B.col = g.dag_col;
  B.v_lo = v_lo;
  B.v_hi = v_hi;
  B.k = k;
  B.acc = ws.ctr.p + 8;
  B.queue = ws.ctr.p;
  B.err = ws.ctr.p + 15;
  B.big = reinterpret_cast<int32_t*>(ws.big.p);
  B.big_cap = (int64_t)ws.big.cap * 2;
  B.scratch = words > 0 ? reinterpret_cast<uint32_t*>(ws.vid[11].p) : nullptr;
  B.scratch_words = words;
  B.stat = ws.ctr.p + 12;
  B.gid = g.gid;
  B.per_graph = per_graph_dev;
  const int64_t np = (int64_t)v_hi - v_lo;
  int wgrid = grid_for((const void*)bm_warp_kernel, 256, 0);
  wgrid = (int)std::max<int64_t>(1, std::min<int64_t>(wgrid, ((np + kBmGrab - 1) / kBmGrab + 7) / 8));
  Profiler& prof = profiler();
  int id = prof.begin("bitset_count", 3);
  if (np > 0) {
    bm_warp_kernel<<<wgrid, 256, 0, s>>>(B);
    PGM_CHECK_LAUNCH();
    bm_block_kernel<<<bgrid, bthreads, bsmem, s>>>(B);
    PGM_CHECK_LAUNCH();
  }
  prof.end(id, (double)(g.h_dag_rp[v_hi] - g.h_dag_rp[v_lo]), 0.0);
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
