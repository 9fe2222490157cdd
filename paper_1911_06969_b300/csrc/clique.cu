// clique.cu -- level-wise k-clique counting on the degree-oriented DAG.
//
// Method (Sec. 3.1 Algorithms 1-2, Sec. 3.3 Listing 3, Sec. 4.1): embeddings
// grow one vertex per level; only the last vertex is extended (eager
// pruning) and a candidate u in N+(last) is kept iff it is connected to
// every earlier vertex.  Levels are materialised with inspection-execution
// (count -> exclusive scan -> conflict-free write, Sec. 5.3); the last level
// is fused with the reduction and never written (Sec. 3.1; loop fusion,
// Sec. 5.2); the first level's parents are blocked into chunks bounded by a
// memory budget (edge blocking, Sec. 5.2).
//
// Level layout (this build's own, in place of the paper's (idx, vid) pairs
// of Sec. 5.1): level l is a vid[] array grouped into parent segments
// seg[p]..seg[p+1], each segment sorted by vertex ID.  The segment of a
// parent holds exactly the vertices connected to all of the parent's
// vertices and after its last one in DAG order, so the connectivity check
// of a candidate u of entry e = (parent p, vertex w) against all earlier
// vertices reduces to one membership test of u in segment(p): the children
// of e are N+(w) intersected with segment(p).  Level 2 is the DAG itself
// (parent = vertex u, segment = N+(u)); level l+1's segment array is the
// exclusive scan of level l's child counts.
//
// Load balancing: a persistent warp kernel takes parents from an atomic
// queue, stages the segment in shared memory and flattens the (entry,
// neighbour) pairs of 32 entries at a time across the lanes; parents whose
// segment exceeds the hub threshold are deferred to a block kernel that
// stages the segment once per block and spreads its entries over all warps.
#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace pgm {

enum Mode : int { kCount = 0, kWrite = 1, kSum = 2 };
constexpr int kGrab = 4;  // parents taken per queue access

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
};

// Flush a per-lane count to the graph's counter (warp-wide reduction).
__device__ __forceinline__ void flush_count(const LevelArgs& A, unsigned long long& tot, int g,
                                            int lane) {
  unsigned long long s = warp_sum(tot);
  if (lane == 0 && s) {
    if (A.per_graph && g >= 0)
      atomicAdd(A.per_graph + g, s);
    else
      atomicAdd(A.acc, s);
  }
  tot = 0;
}

// Process entries j0 .. j0+31 of a staged segment S (length s).  e0 is the
// output index of S[0].  Children of entry j are N+(S[j]) & S, found either
// forward (scan N+(w), binary-search S in shared memory) or in reverse when
// N+(w) is much longer than S (scan S, binary-search N+(w)); both visit the
// children in ascending ID order.
template <int MODE>
__device__ __forceinline__ void process_batch(const int32_t* S, int s, int j0, int64_t e0,
                                              const LevelArgs& A, int lane, uint32_t* wcnt,
                                              unsigned long long& tot, unsigned long long& lensum) {
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
  const int incl = warp_inclusive_scan(len, lane);
  const int total = __shfl_sync(kFull, incl, 31);
  const int excl = incl - len;
  int64_t my_off = 0;
  if (MODE != kSum) {
    wcnt[lane] = 0;
    if (MODE == kWrite && valid) my_off = A.off[e0 + j] - A.off_shift;
    __syncwarp();
  }
  const int32_t smin = S[0], smax = S[s - 1];
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
        hit = x >= smin && x <= smax && contains_dev(S, s, x);
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
    if (valid) A.cnt[e0 + j] = wcnt[lane];
    __syncwarp();
  }
}

template <int MODE, typename OffT>
__global__ void __launch_bounds__(512) clique_warp_kernel(LevelArgs A) {
  extern __shared__ int32_t smem[];
  const OffT* __restrict__ seg = reinterpret_cast<const OffT*>(A.seg);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t* S = smem + wid * (A.cap + 32);
  uint32_t* wcnt = reinterpret_cast<uint32_t*>(S + A.cap);
  unsigned long long tot = 0, lensum = 0;
  int cur_g = -1;
  const int64_t np = A.p_hi - A.p_lo;
  for (;;) {
    unsigned long long p0 = 0;
    if (lane == 0) p0 = atomicAdd(A.queue, (unsigned long long)kGrab);
    p0 = __shfl_sync(kFull, p0, 0);
    if ((int64_t)p0 >= np) break;
    const int64_t pend = min((int64_t)p0 + kGrab, np);
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
      if (MODE == kSum && A.gid) {
        const int g = A.gid[S[0]];
        if (g != cur_g) {
          flush_count(A, tot, cur_g, lane);
          cur_g = g;
        }
      }
      for (int j0 = 0; j0 < s; j0 += 32)
        process_batch<MODE>(S, (int)s, j0, sb - A.e_base, A, lane, wcnt, tot, lensum);
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
    if (MODE == kSum && A.gid) {
      const int g = A.gid[S[0]];
      if (g != cur_g) {
        flush_count(A, tot, cur_g, lane);
        cur_g = g;
      }
    }
    for (int64_t j0 = (int64_t)wid * 32; j0 < s; j0 += (int64_t)nw * 32)
      process_batch<MODE>(S, (int)s, (int)j0, sb - A.e_base, A, lane, wcnt, tot, lensum);
    __syncthreads();
  }
  if (MODE == kSum) flush_count(A, tot, cur_g, lane);
  lensum = warp_sum(lensum);
  if (lane == 0 && lensum) atomicAdd(A.stat, lensum);
}

// ---------------------------------------------------------------- host side
namespace {

struct Lvl {
  const void* seg;
  bool seg32;
  int64_t seg_shift;
  const int32_t* vid;
  const int64_t* h_seg;  // host copy of seg (level 2 only) or nullptr
  int64_t p_lo, p_hi;
  int64_t e_lo, e_hi;    // entry range (after shift) of the parents
};

// counter slots in ws.ctr
constexpr int kSlotQueue = 0;  // 4 per launch (reset per launch)
constexpr int kSlotErr = 15;   // hub-list overflow counter
constexpr int kSlotAcc = 16;   // total count
constexpr int kSlotStat = 32;  // per (level, mode): 32 + 3 l + mode
constexpr int kSlots = 96;

struct CliqueRun {
  Graph& g;
  Workspace& ws;
  cudaStream_t s;
  int k;
  const pgm_options o;
  int hub, cap, block_cap;
  int chunks = 0;
  unsigned long long* per_graph = nullptr;
  double lvl_entries[Workspace::kMaxLevels] = {0};
  double lvl_parents[Workspace::kMaxLevels] = {0};
  double lvl_size[Workspace::kMaxLevels + 4] = {0};

  CliqueRun(Graph& g_, Workspace& ws_, cudaStream_t s_, int k_)
      : g(g_), ws(ws_), s(s_), k(k_), o(options()) {
    cap = o.warp_stage_cap;
    hub = o.hub_threshold > 0 ? std::min(o.hub_threshold, cap) : cap;
    block_cap = 12288;  // ints staged per block (48 KB: four 512-thread blocks per SM)
  }

  unsigned long long* ctr() { return ws.ctr.p; }

  pgm_status e_of(const Lvl& L, int64_t p, int64_t* e) {
    if (L.h_seg) {
      *e = L.h_seg[p] - L.seg_shift;
      return PGM_OK;
    }
    if (L.seg32) {
      int32_t v;
      PGM_TRY(read_dev(reinterpret_cast<const int32_t*>(L.seg) + p, &v, s));
      *e = (int64_t)v - L.seg_shift;
    } else {
      int64_t v;
      PGM_TRY(read_dev(reinterpret_cast<const int64_t*>(L.seg) + p, &v, s));
      *e = v - L.seg_shift;
    }
    return PGM_OK;
  }

  template <int MODE>
  pgm_status launch(const Lvl& L, int level, uint32_t* cnt, const int64_t* off, int64_t off_shift,
                    int32_t* out_vid, int64_t pa, int64_t pb, int64_t e_base, const char* name,
                    double entries) {
    if (pb <= pa) return PGM_OK;
    const int64_t nparents = pb - pa;
    // at most entries / (hub + 1) parents can exceed the threshold
    const int64_t big_cap = (int64_t)(entries / std::max(hub, 1)) + 2;
    PGM_TRY(ws.big.reserve((size_t)big_cap));
    PGM_TRY_CUDA(cudaMemsetAsync(ctr() + kSlotQueue, 0, 4 * sizeof(unsigned long long), s));
    LevelArgs A;
    A.seg = L.seg;
    A.seg_shift = L.seg_shift;
    A.vid = L.vid;
    A.p_lo = pa;
    A.p_hi = pb;
    A.e_base = e_base;
    A.rp = g.dag_rp;
    A.col = g.dag_col;
    A.cnt = cnt;
    A.off = off;
    A.off_shift = off_shift;
    A.out_vid = out_vid;
    A.acc = ctr() + kSlotAcc;
    A.stat = ctr() + kSlotStat + 3 * level + MODE;
    A.queue = ctr() + kSlotQueue;
    A.err = ctr() + kSlotErr;
    A.big = ws.big.p;
    A.big_cap = big_cap;
    A.hub = hub;
    A.cap = cap;
    A.block_cap = block_cap;
    A.rev_ratio = 4;
    A.gid = g.gid;
    A.per_graph = per_graph;
    const int threads = o.block_threads;
    const size_t wsmem = (size_t)(threads / 32) * (cap + 32) * sizeof(int32_t);
    const size_t bsmem = (size_t)block_cap * sizeof(int32_t) + (size_t)(512 / 32) * 32 * 4;
    const void* wfn;
    const void* bfn;
    if (L.seg32) {
      wfn = (const void*)clique_warp_kernel<MODE, int32_t>;
      bfn = (const void*)clique_block_kernel<MODE, int32_t>;
    } else {
      wfn = (const void*)clique_warp_kernel<MODE, int64_t>;
      bfn = (const void*)clique_block_kernel<MODE, int64_t>;
    }
    PGM_TRY(smem_attr(wfn, 160 * 1024));
    PGM_TRY(smem_attr(bfn, 160 * 1024));
    int wgrid = grid_for(wfn, threads, wsmem);
    const int64_t warps_needed = (nparents + kGrab - 1) / kGrab;
    wgrid = (int)std::max<int64_t>(1, std::min<int64_t>(wgrid, (warps_needed + threads / 32 - 1) /
                                                                    (threads / 32)));
    int bgrid = grid_for(bfn, 512, bsmem);
    Profiler& prof = profiler();
    int id = prof.begin(name, level);
    if (L.seg32) {
      clique_warp_kernel<MODE, int32_t><<<wgrid, threads, wsmem, s>>>(A);
      PGM_CHECK_LAUNCH();
      clique_block_kernel<MODE, int32_t><<<bgrid, 512, bsmem, s>>>(A);
      PGM_CHECK_LAUNCH();
    } else {
      clique_warp_kernel<MODE, int64_t><<<wgrid, threads, wsmem, s>>>(A);
      PGM_CHECK_LAUNCH();
      clique_block_kernel<MODE, int64_t><<<bgrid, 512, bsmem, s>>>(A);
      PGM_CHECK_LAUNCH();
    }
    prof.end(id, entries, 0.0);
    return PGM_OK;
  }

  pgm_status level(int l, const Lvl& L) {
    const int64_t E = L.e_hi - L.e_lo;
    const int64_t P = L.p_hi - L.p_lo;
    lvl_entries[l] += (double)E;
    lvl_parents[l] += (double)P;
    lvl_size[l] += (double)E;
    if (E == 0) return PGM_OK;
    if (l == k - 1) {
      return launch<kSum>(L, l, nullptr, nullptr, 0, nullptr, L.p_lo, L.p_hi, L.e_lo, "extend_sum",
                          (double)E);
    }
    PGM_TRY(ws.cnt[l].reserve((size_t)E));
    PGM_TRY(ws.off[l].reserve((size_t)E + 1));
    PGM_TRY_CUDA(cudaMemsetAsync(ws.cnt[l].p, 0, (size_t)E * sizeof(uint32_t), s));
    PGM_TRY(launch<kCount>(L, l, ws.cnt[l].p, nullptr, 0, nullptr, L.p_lo, L.p_hi, L.e_lo,
                           "extend_count", (double)E));
    {
      Profiler& prof = profiler();
      int id = prof.begin("scan", l);
      PGM_TRY(exclusive_scan(ws.cnt[l].p, E, ws.off[l].p, ws, s));
      prof.end(id, (double)E, 12.0 * (double)E);
    }
    int64_t T = 0;
    PGM_TRY(read_dev(ws.off[l].p + E, &T, s));
    if (T == 0) return PGM_OK;
    const int64_t B = o.level_budget;
    int64_t pa = L.p_lo;
    while (pa < L.p_hi) {
      int64_t ea, pb, eb;
      PGM_TRY(e_of(L, pa, &ea));
      int64_t base;
      PGM_TRY(read_dev(ws.off[l].p + (ea - L.e_lo), &base, s));
      if (T - base <= B) {
        pb = L.p_hi;
      } else {
        // largest pb with children(pa..pb) <= B (at least one parent)
        int64_t lo = pa + 1, hi = L.p_hi;
        pb = pa + 1;
        while (lo <= hi) {
          int64_t mid = lo + (hi - lo) / 2;
          int64_t em, om;
          PGM_TRY(e_of(L, mid, &em));
          PGM_TRY(read_dev(ws.off[l].p + (em - L.e_lo), &om, s));
          if (om - base <= B) {
            pb = mid;
            lo = mid + 1;
          } else {
            hi = mid - 1;
          }
        }
      }
      PGM_TRY(e_of(L, pb, &eb));
      int64_t ob;
      PGM_TRY(read_dev(ws.off[l].p + (eb - L.e_lo), &ob, s));
      const int64_t Tp = ob - base;
      chunks++;
      if (Tp > 0) {
        PGM_TRY(ws.vid[l + 1].reserve((size_t)Tp));
        PGM_TRY(launch<kWrite>(L, l, nullptr, ws.off[l].p, base, ws.vid[l + 1].p, pa, pb, L.e_lo,
                               "extend_write", (double)(eb - ea)));
        Lvl nx;
        nx.seg = ws.off[l].p;
        nx.seg32 = false;
        nx.seg_shift = base;
        nx.vid = ws.vid[l + 1].p;
        nx.h_seg = nullptr;
        nx.p_lo = ea - L.e_lo;
        nx.p_hi = eb - L.e_lo;
        nx.e_lo = 0;
        nx.e_hi = Tp;
        PGM_TRY(level(l + 1, nx));
      }
      pa = pb;
    }
    return PGM_OK;
  }
};

}  // namespace

pgm_status count_kcliques(Graph& g, Workspace& ws, cudaStream_t s, int k, int32_t v_lo, int32_t v_hi,
                          uint64_t* out, unsigned long long* per_graph_dev) {
  if (k < 1 || k > 10) {
    set_error("count_kcliques: k=%d outside [1, 10]", k);
    return PGM_EUNSUPPORTED;
  }
  if (v_lo < 0 || v_hi > g.n || v_lo > v_hi) {
    set_error("count_kcliques: bad vertex range [%d, %d)", v_lo, v_hi);
    return PGM_EINVAL;
  }
  PGM_TRY(graph_orient(g));
  pgm_profile& lp = last_profile();
  if (k <= 2) {
    *out = k == 1 ? (uint64_t)(v_hi - v_lo) : (uint64_t)(g.h_dag_rp[v_hi] - g.h_dag_rp[v_lo]);
    return PGM_OK;
  }
  PGM_TRY(ws.ctr.reserve(kSlots));
  PGM_TRY_CUDA(cudaMemsetAsync(ws.ctr.p, 0, kSlots * sizeof(unsigned long long), s));
  CliqueRun run(g, ws, s, k);
  run.per_graph = per_graph_dev;
  Lvl L2;
  L2.seg = g.dag_rp;
  L2.seg32 = true;
  L2.seg_shift = 0;
  L2.vid = g.dag_col;
  L2.h_seg = g.h_dag_rp.data();
  L2.p_lo = v_lo;
  L2.p_hi = v_hi;
  L2.e_lo = g.h_dag_rp[v_lo];
  L2.e_hi = g.h_dag_rp[v_hi];
  run.lvl_size[1] = (double)(v_hi - v_lo);
  PGM_TRY(run.level(2, L2));
  unsigned long long h[kSlots];
  bool deferred = false;
  PGM_TRY(read_counters(ws.ctr.p, h, kSlots, s, &deferred));
  if (deferred) return PGM_OK;  // replay: the caller reads the counters after the graph runs
  if (h[kSlotErr]) {
    set_error("count_kcliques: internal hub-list overflow");
    return PGM_ENOMEM;
  }
  *out = h[kSlotAcc];
  Profiler& prof = profiler();
  if (prof.on) {
    PGM_TRY(prof.finish(&lp));
    for (int i = 0; i < lp.nphases; i++) {
      pgm_phase& p = lp.phase[i];
      const int l = p.level;
      const int mode = !strcmp(p.name, "extend_count")   ? kCount
                       : !strcmp(p.name, "extend_write") ? kWrite
                       : !strcmp(p.name, "extend_sum")   ? kSum
                                                         : -1;
      if (mode < 0 || l < 0 || l >= Workspace::kMaxLevels) continue;
      const double lens = (double)h[kSlotStat + 3 * l + mode];
      const double E = run.lvl_entries[l], P = run.lvl_parents[l];
      // entry vid (4 B) + its row-pointer pair (8 B) + parent segment offsets
      // (8 B per parent) + neighbour lists (4 B per element); count: + 4 B per
      // entry written; write: + 8 B per entry (offset) + 4 B per child written
      double b = 12.0 * E + 8.0 * P + 4.0 * lens;
      if (mode == kCount) b += 4.0 * E;
      if (mode == kWrite) b += 8.0 * E + 4.0 * run.lvl_size[l + 1];
      p.alg_bytes = b;
      p.entries = E;
    }
  }
  for (int l = 1; l <= k && l < 16; l++) lp.level_size[l] = (uint64_t)run.lvl_size[l];
  lp.level_size[k] = h[kSlotAcc];
  lp.chunks = run.chunks;
  return PGM_OK;
}

}  // namespace pgm

extern "C" {

pgm_status pgm_count_kcliques(pgm_graph* g, int32_t k, uint64_t* out_count) {
  if (!g || !out_count) {
    pgm::set_error("pgm_count_kcliques: null argument");
    return PGM_EINVAL;
  }
  pgm::profiler().start(g->g.stream);
  uint64_t c = 0;
  PGM_TRY(pgm::count_kcliques(g->g, g->g.ws, g->g.stream, k, 0, g->g.n, &c, nullptr));
  *out_count = c;
  return PGM_OK;
}

pgm_status pgm_count_kcliques_range(pgm_graph* g, int32_t k, int32_t v_lo, int32_t v_hi,
                                    uint64_t* out_count) {
  if (!g || !out_count) {
    pgm::set_error("pgm_count_kcliques_range: null argument");
    return PGM_EINVAL;
  }
  pgm::profiler().start(g->g.stream);
  uint64_t c = 0;
  PGM_TRY(pgm::count_kcliques(g->g, g->g.ws, g->g.stream, k, v_lo, v_hi, &c, nullptr));
  *out_count = c;
  return PGM_OK;
}

}  // extern "C"
