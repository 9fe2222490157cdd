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

#include "clique_kernels.cuh"

namespace pgm {

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

// Listing: every entry of the last level becomes a row of k vertex IDs.
// The vertex at position l of the row is vid_l[e_l], and the parent of a
// level-l entry e_l is the parent p whose segment holds it (the largest p
// with seg_l[p] - shift_l <= e_l); p indexes level l-1 as p + e_lo_{l-1}.
// Level 2's parents are the vertices themselves (position 1).
constexpr int kMaxK = 10;
struct EmitArgs {
  int k;
  const void* seg[kMaxK + 1];
  int seg32[kMaxK + 1];
  int64_t shift[kMaxK + 1], p_lo[kMaxK + 1], p_hi[kMaxK + 1], e_lo[kMaxK + 1];
  const int32_t* vid[kMaxK + 1];
  int64_t n;           // entries of the last level in this chunk
  int32_t* out;        // rows of k IDs
  int64_t out_base;    // first row of this chunk
};

__global__ void emit_kernel(EmitArgs A) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < A.n; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t e = t + A.e_lo[A.k];
    int32_t* row = A.out + (A.out_base + t) * A.k;
    for (int l = A.k; l >= 2; l--) {
      row[l - 1] = A.vid[l][e];
      const int64_t key = e + A.shift[l];
      int64_t lo = A.p_lo[l], hi = A.p_hi[l];  // seg[lo] <= key < seg[hi]
      while (hi - lo > 1) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        const int64_t v = A.seg32[l] ? (int64_t) reinterpret_cast<const int32_t*>(A.seg[l])[mid]
                                     : reinterpret_cast<const int64_t*>(A.seg[l])[mid];
        if (v <= key)
          lo = mid;
        else
          hi = mid;
      }
      e = lo + A.e_lo[l - 1];
    }
    row[0] = (int32_t)e;  // level 1: the vertex itself
  }
}


// counter slots in ws.ctr
constexpr int kSlotQueue = 0;  // 4 per launch (reset per launch)
constexpr int kSlotErr = 15;   // hub-list overflow counter
constexpr int kChunkedHub = 256;  // block-per-parent threshold inside chunked levels
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
  bool chunked = false;  // some level was split into several chunks
  int chunks = 0;
  unsigned long long* per_graph = nullptr;
  double lvl_entries[Workspace::kMaxLevels] = {0};
  // listing mode (list_out != nullptr): the last level is written and emitted
  int32_t* list_out = nullptr;
  int64_t list_n = 0;
  HostSink* sink = nullptr;  // rows streamed to the host (list_out unused then)
  int64_t budget;            // entries per edge-blocking chunk
  Lvl chain[Workspace::kMaxLevels + 1];
  double lvl_parents[Workspace::kMaxLevels] = {0};
  double lvl_size[Workspace::kMaxLevels + 4] = {0};

  CliqueRun(Graph& g_, Workspace& ws_, cudaStream_t s_, int k_)
      : g(g_), ws(ws_), s(s_), k(k_), o(options()) {
    cap = o.warp_stage_cap;
    hub = o.hub_threshold > 0 ? std::min(o.hub_threshold, cap) : cap;
    block_cap = 12288;  // ints staged per block (48 KB: four 512-thread blocks per SM)
    budget = o.level_budget;
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
    // Chunked levels launch once per chunk, and each launch ends with its
    // slowest warp-parent; a lower block-per-parent threshold there moves
    // the heavy parents to whole blocks (measured on R-MAT 21: 43 chunks,
    // 908 -> 685 ms; unchunked runs are unchanged by it).
    const int hub_eff = chunked ? std::min(hub, kChunkedHub) : hub;
    // at most entries / (hub + 1) parents can exceed the threshold
    const int64_t big_cap = (int64_t)(entries / std::max(hub_eff, 1)) + 2;
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
    A.carry = ctr() + kCarrySlot;
    A.big = ws.big.p;
    A.big_cap = big_cap;
    A.hub = hub_eff;
    A.cap = cap;
    A.block_cap = block_cap;
    A.rev_ratio = o.reverse_ratio;
    A.gid = g.gid;
    A.per_graph = per_graph;
    const int threads = o.block_threads;
    const size_t wsmem = clique_warp_smem(threads, cap);
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
    // kGrab parents per queue access, fewer when there are too few parents
    // to give every resident warp that many
    A.grab = (int)std::max<int64_t>(1, std::min<int64_t>(kGrab, nparents / ((int64_t)wgrid * (threads / 32))));
    const int64_t warps_needed = (nparents + A.grab - 1) / A.grab;
    wgrid = (int)std::max<int64_t>(1, std::min<int64_t>(wgrid, (warps_needed + threads / 32 - 1) /
                                                                    (threads / 32)));
    // a block takes one hub parent at a time: no more blocks than hubs can exist
    const int bgrid = (int)std::max<int64_t>(1, std::min<int64_t>(grid_for(bfn, 512, bsmem), big_cap));
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

  // rows for the last level `last` (entries 0..n) of this chunk
  pgm_status emit(const Lvl& last, int64_t n) {
    EmitArgs A;
    memset(&A, 0, sizeof(A));
    A.k = k;
    for (int l = 2; l <= k; l++) {
      const Lvl& L = l == k ? last : chain[l];
      A.seg[l] = L.seg;
      A.seg32[l] = L.seg32 ? 1 : 0;
      A.shift[l] = L.seg_shift;
      A.p_lo[l] = L.p_lo;
      A.p_hi[l] = L.p_hi;
      A.e_lo[l] = L.e_lo;
      A.vid[l] = L.vid;
    }
    A.e_lo[1] = 0;
    A.n = n;
    A.out = list_out;
    A.out_base = list_n;
    if (sink) {
      if (n > sink->cap_rows) {
        set_error("list_kcliques: %lld rows of one chunk exceed the staging buffer", (long long)n);
        return PGM_ENOMEM;
      }
      PGM_TRY(sink->reserve(n, s));
      A.out = sink->buf[sink->cur];
      A.out_base = sink->fill;
      sink->fill += n;
    }
    Profiler& prof = profiler();
    int id = prof.begin("extend_list", k);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms() * 8, (n + 255) / 256));
    emit_kernel<<<blocks, 256, 0, s>>>(A);
    PGM_CHECK_LAUNCH();
    prof.end(id, (double)n, 4.0 * (double)k * (double)n);
    list_n += n;
    return PGM_OK;
  }

  pgm_status level(int l, const Lvl& L) {
    PGM_NVTX(kNvtxLevel[l < 13 ? l : 12]);
    chain[l] = L;
    const int64_t E = L.e_hi - L.e_lo;
    const int64_t P = L.p_hi - L.p_lo;
    lvl_entries[l] += (double)E;
    lvl_parents[l] += (double)P;
    lvl_size[l] += (double)E;
    if (E == 0) return PGM_OK;
    if (l == k - 1 && !list_out && !sink) {
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
    // with rows streamed to the host, the chunks of the last level fit a staging buffer
    const int64_t B = sink && l == k - 1 ? std::min<int64_t>(budget, sink->cap_rows) : budget;
    if (T > B) chunked = true;
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
        if (l + 1 == k)
          PGM_TRY(emit(nx, Tp));
        else
          PGM_TRY(level(l + 1, nx));
      }
      pa = pb;
    }
    return PGM_OK;
  }
};

}  // namespace

// Rows for k = 1 (every vertex) and k = 2 (every DAG arc u -> v).
__global__ void list_small_kernel(int32_t n, int k, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                  int32_t* __restrict__ out) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    if (k == 1) {
      out[u] = (int32_t)u;
    } else {
      for (int32_t a = rp[u]; a < rp[u + 1]; a++) {
        out[2 * (int64_t)a] = (int32_t)u;
        out[2 * (int64_t)a + 1] = col[a];
      }
    }
  }
}

pgm_status list_small(Graph& g, int k, int32_t* out) {
  if (g.n == 0) return PGM_OK;
  const int blocks = std::max(1, std::min(num_sms() * 8, (g.n + 255) / 256));
  list_small_kernel<<<blocks, 256, 0, g.stream>>>(g.n, k, g.dag_rp, g.dag_col, out);
  PGM_CHECK_LAUNCH();
  return PGM_OK;
}

// Rows of the k-cliques of the whole graph into `out` (k IDs each, in DAG
// order), by the level lists with the last level written; `rows` must be
// the clique count.
pgm_status list_kcliques(Graph& g, Workspace& ws, cudaStream_t s, int k, int32_t* out, int64_t rows,
                         HostSink* sink) {
  PGM_TRY(graph_orient(g));
  PGM_TRY(graph_host_dag_rp(g));
  PGM_TRY(ws.ctr.reserve(kSlots));
  PGM_TRY_CUDA(cudaMemsetAsync(ws.ctr.p, 0, kSlots * sizeof(unsigned long long), s));
  CliqueRun run(g, ws, s, k);
  run.list_out = out;
  run.sink = sink;
  Lvl L2;
  L2.seg = g.dag_rp;
  L2.seg32 = true;
  L2.seg_shift = 0;
  L2.vid = g.dag_col;
  L2.h_seg = g.h_dag_rp.data();
  L2.p_lo = 0;
  L2.p_hi = g.n;
  L2.e_lo = 0;
  L2.e_hi = g.h_dag_rp[g.n];
  PGM_TRY(run.level(2, L2));
  unsigned long long h[kSlots];
  bool deferred = false;
  PGM_TRY(read_counters(ws.ctr.p, h, kSlots, s, &deferred));
  if (h[kSlotErr]) {
    set_error("list_kcliques: internal hub-list overflow");
    return PGM_ENOMEM;
  }
  if (run.list_n != rows) {
    set_error("list_kcliques: wrote %lld rows, expected %lld", (long long)run.list_n, (long long)rows);
    return PGM_ECUDA;
  }
  if (sink) {
    PGM_TRY(sink->flush(s));
    PGM_TRY(sink->finish());
  }
  return PGM_OK;
}

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
  int64_t arcs = 0;
  PGM_TRY(graph_dag_arcs(g, v_lo, v_hi, &arcs));
  if (k <= 2) {
    *out = k == 1 ? (uint64_t)(v_hi - v_lo) : (uint64_t)arcs;
    return PGM_OK;
  }
  const int engine = options().clique_engine;
  if ((engine == 0 || engine == 2) && k >= 3) {
    uint64_t ls[kBmLevelRead + 1] = {0};
    const pgm_status st = count_kcliques_bitset(g, ws, s, k, v_lo, v_hi, out, per_graph_dev, ls);
    if (st != PGM_EUNSUPPORTED) {
      if (st != PGM_OK || current_plan()) return st;
      Profiler& prof = profiler();
      if (prof.on) {
        PGM_TRY(prof.finish(&lp));
        for (int i = 0; i < lp.nphases; i++) {
          pgm_phase& p = lp.phase[i];
          // level 2 -> 3 of the extension: every level-2 embedding (DAG arc u -> v)
          // reads the out-list of its last vertex v (4 B per element) and its own
          // record (8 B), and every level-3 embedding is written (8 B) unless the
          // last level is fused (k = 3).  Deeper levels are ANDs of on-chip rows.
          if (!strcmp(p.name, "bitset_count"))
            p.alg_bytes = 4.0 * (double)ls[kBmLevelRead] + 8.0 * (double)arcs + (k > 3 ? 8.0 * (double)ls[3] : 0.0);
        }
      }
      lp.level_size[1] = (uint64_t)(v_hi - v_lo);
      lp.level_size[2] = (uint64_t)arcs;
      for (int l = 3; l < k; l++) lp.level_size[l] = ls[l];
      lp.level_size[k] = *out;
      lp.chunks = 0;
      return PGM_OK;
    }
  }
  PGM_TRY(graph_host_dag_rp(g));  // edge blocking plans on the host row pointers
  PGM_TRY(ws.ctr.reserve(kSlots));
  PGM_TRY_CUDA(cudaMemsetAsync(ws.ctr.p, 0, kSlots * sizeof(unsigned long long), s));
  if (!per_graph_dev) PGM_TRY(seed_counts(ws.ctr.p + kSlotAcc, 1, s));
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
  if (h[kCarrySlot]) {
    set_error("count_kcliques: the count exceeds 2^64 - 1");
    return PGM_EOVERFLOW;
  }
  h[kSlotAcc] -= per_graph_dev ? 0ull : count_seed();
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
  PGM_NVTX("pgm_count_kcliques");
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
  PGM_NVTX("pgm_count_kcliques_range");
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

static pgm_status list_kcliques_to(pgm_graph* g, int32_t k, int32_t* out, int64_t cap_rows, int64_t* n_rows,
                                   bool host, const char* name) {
  if (!g || !n_rows || cap_rows < 0) {
    pgm::set_error("%s: bad arguments", name);
    return PGM_EINVAL;
  }
  if (k < 1 || k > pgm::kMaxK) {
    pgm::set_error("%s: k=%d outside [1, %d]", name, k, pgm::kMaxK);
    return PGM_EUNSUPPORTED;
  }
  pgm::Graph& G = g->g;
  pgm::profiler().start(G.stream);
  uint64_t total = 0;
  PGM_TRY(pgm::count_kcliques(G, G.ws, G.stream, k, 0, G.n, &total, nullptr));
  if (total > (uint64_t)INT64_MAX / (uint64_t)k) {
    pgm::set_error("%s: %llu rows do not fit an index", name, (unsigned long long)total);
    return PGM_EOVERFLOW;
  }
  *n_rows = (int64_t)total;
  if (!out) return PGM_OK;  // size query
  if ((int64_t)total > cap_rows) {
    pgm::set_error("%s: %llu rows exceed the capacity of %lld", name, (unsigned long long)total, (long long)cap_rows);
    return PGM_EOVERFLOW;
  }
  if (total == 0) return PGM_OK;
  if (!host) {
    if (k == 1 || k == 2) {
      PGM_TRY(pgm::list_small(G, k, out));
    } else {
      pgm::profiler().start(G.stream);
      PGM_TRY(pgm::list_kcliques(G, G.ws, G.stream, k, out, (int64_t)total, nullptr));
    }
    PGM_TRY_CUDA(cudaStreamSynchronize(G.stream));
    return PGM_OK;
  }
  pgm_status st = PGM_OK;
  if (k == 1 || k == 2) {
    // n or m rows: no larger than the graph itself
    int32_t* tmp = nullptr;
    PGM_TRY_CUDA(pgm::dev_malloc(&tmp, (size_t)total * k * sizeof(int32_t)));
    st = pgm::list_small(G, k, tmp);
    if (st == PGM_OK && cudaMemcpyAsync(out, tmp, (size_t)total * k * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                        G.stream) != cudaSuccess)
      st = PGM_ECUDA;
    if (cudaStreamSynchronize(G.stream) != cudaSuccess && st == PGM_OK) st = PGM_ECUDA;
    pgm::dev_free(tmp);
    if (st == PGM_ECUDA) pgm::set_error("%s: copy to the host failed: %s", name, cudaGetErrorString(cudaGetLastError()));
    return st;
  }
  pgm::HostSink sink;
  sink.host = out;
  const int64_t staging = std::max<int64_t>(std::min<int64_t>(pgm::options().level_budget, (int64_t)1 << 26), G.dag_dmax);
  st = sink.init(k, staging);
  if (st == PGM_OK) {
    pgm::profiler().start(G.stream);
    st = pgm::list_kcliques(G, G.ws, G.stream, k, nullptr, (int64_t)total, &sink);
  }
  cudaStreamSynchronize(G.stream);
  sink.release();
  return st;
}

pgm_status pgm_list_kcliques(pgm_graph* g, int32_t k, int32_t* out_dev, int64_t cap_rows, int64_t* n_rows) {
  PGM_NVTX("pgm_list_kcliques");
  return list_kcliques_to(g, k, out_dev, cap_rows, n_rows, false, "pgm_list_kcliques");
}

pgm_status pgm_list_kcliques_host(pgm_graph* g, int32_t k, int32_t* out_host, int64_t cap_rows, int64_t* n_rows) {
  PGM_NVTX("pgm_list_kcliques_host");
  return list_kcliques_to(g, k, out_host, cap_rows, n_rows, true, "pgm_list_kcliques_host");
}

}  // extern "C"
