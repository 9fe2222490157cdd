// motifgen.cu -- the generic k-motif engine (k = 3, 4, 5): vertex-induced
// motif counting for k = 5 and motif listing for k = 3..5 (Sec. 3.3
// Listing 4 with generic pattern classification, Sec. 3.2 canonical test).
//
// Levels are embedding lists of full vertex tuples (one int32 array per
// position, plus the index f of the last vertex's first neighbour in its
// prefix), built by inspection-execution (Sec. 5.3).  An entry
// (v_0 .. v_{i-1}) is extended by every vertex u of N(v_j) (j = 0 .. i-1)
// that passes the breadth-first canonical test of the motif engine: u > v_0,
// u not in the tuple, j = f(u) (u in no earlier vertex's list, so each
// candidate is generated once), and j = i - 1 or (f(v_{i-1}), v_{i-1}) <
// (j, u).  Membership uses binary search in the sorted lists (Sec. 5.4).
// The last level is fused with the reduction (counting: a per-block class
// histogram) or written out (listing: one row per k-set): each accepted
// k-set is classified by its adjacency code through a table of the
// connected k-vertex graphs (generic classification in place of Listing
// 6's special cases).
//
// Codes: bit i = pair i of (0,1),(0,2),(0,3),(0,4),(1,2),(1,3),(1,4),(2,3),
// (2,4),(3,4) (pairs of positions in the canonical order; k < 5 uses the
// pairs of positions below k).  Class order: k = 3 wedge, triangle; k = 4
// 3-star, 4-path, tailed triangle, 4-cycle, diamond, 4-clique; k = 5 the 21
// connected 5-vertex graphs by edge count, then the degree sequence
// (non-increasing, lexicographically smaller first), then the canonical
// code (the smallest code over the 120 relabellings).
#include <algorithm>
#include <array>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace pgm {
namespace {

constexpr int kP5 = 21;
// adjacency code -> class for k = 3, 4, 5 (row k - 3), -1 if disconnected
__constant__ int8_t c_cls[3][1024];

// pair index of (a, b), a < b < 5, in the code's bit order
__host__ __device__ constexpr int pair_bit(int a, int b) {
  return a == 0 ? b - 1 : a == 1 ? 3 + b - 1 : a == 2 ? 6 + b - 2 : 9;
}

// Host: class of every code of k vertices, from the orders stated above.
std::array<int8_t, 1024> build_class_table(int k) {
  auto adj = [](int code, int a, int b) {
    if (a == b) return false;
    if (a > b) std::swap(a, b);
    return ((code >> pair_bit(a, b)) & 1) != 0;
  };
  auto relabel = [&](int code, const std::array<int, 5>& p) {
    int c = 0;
    for (int a = 0; a < 5; a++)
      for (int b = a + 1; b < 5; b++)
        if (adj(code, a, b)) {
          int x = p[a], y = p[b];
          if (x > y) std::swap(x, y);
          c |= 1 << pair_bit(x, y);
        }
    return c;
  };
  int used = 0;  // code bits of the pairs among positions < k
  for (int a = 0; a < k; a++)
    for (int b = a + 1; b < k; b++) used |= 1 << pair_bit(a, b);
  auto connected = [&](int code) {
    int reach = 1;
    for (int it = 0; it < k; it++)
      for (int a = 0; a < k; a++)
        if (reach >> a & 1)
          for (int b = 0; b < k; b++)
            if (adj(code, a, b)) reach |= 1 << b;
    return reach == (1 << k) - 1;
  };
  auto degrees = [&](int code, int* e) {
    std::array<int, 5> deg = {0, 0, 0, 0, 0};
    *e = 0;
    for (int a = 0; a < k; a++)
      for (int b = a + 1; b < k; b++)
        if (adj(code, a, b)) deg[a]++, deg[b]++, ++*e;
    std::sort(deg.begin(), deg.end(), [](int x, int y) { return x > y; });
    return deg;
  };
  std::array<int8_t, 1024> t;
  t.fill(-1);
  if (k == 3 || k == 4) {
    for (int code = 0; code < 1024; code++) {
      if ((code & ~used) || !connected(code)) continue;
      int e = 0;
      const int dmax = degrees(code, &e)[0];
      t[code] = (int8_t)(k == 3 ? e - 2 : e == 3 ? (dmax == 3 ? 0 : 1) : e == 4 ? (dmax == 3 ? 2 : 3) : e == 5 ? 4 : 5);
    }
    return t;
  }
  std::vector<int> canon(1024, -1);
  std::vector<int> reps;
  for (int code = 0; code < 1024; code++) {
    if (!connected(code)) continue;
    std::array<int, 5> p = {0, 1, 2, 3, 4};
    int best = 1 << 10;
    do best = std::min(best, relabel(code, p));
    while (std::next_permutation(p.begin(), p.end()));
    canon[code] = best;
    if (best == code) reps.push_back(code);
  }
  auto key = [&](int code) {
    int e = 0;
    const auto deg = degrees(code, &e);
    return std::make_tuple(e, deg, code);
  };
  std::sort(reps.begin(), reps.end(), [&](int x, int y) { return key(x) < key(y); });
  for (int code = 0; code < 1024; code++)
    if (canon[code] >= 0)
      t[code] = (int8_t)(std::find(reps.begin(), reps.end(), canon[code]) - reps.begin());
  return t;
}

pgm_status upload_class_tables() {
  static std::mutex mu;
  static bool done[64] = {false};
  const int dev = device_id();
  std::lock_guard<std::mutex> lk(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return PGM_OK;
  static const std::array<std::array<int8_t, 1024>, 3> tables = {build_class_table(3), build_class_table(4),
                                                                 build_class_table(5)};
  int8_t flat[3][1024];
  for (int r = 0; r < 3; r++) memcpy(flat[r], tables[r].data(), 1024);
  PGM_TRY_CUDA(cudaMemcpyToSymbol(c_cls, flat, sizeof(flat)));
  if (dev >= 0 && dev < 64) done[dev] = true;
  return PGM_OK;
}

// count: children per entry; write: the next level; hist: last level into
// the class histogram; emit: last level as rows (k IDs + class)
enum MgMode : int { mgCount = 0, mgWrite = 1, mgHist = 2, mgEmit = 3 };

struct MgArgs {
  const int32_t* rp;
  const int32_t* col;
  const int32_t* src;     // level 2 (implicit): source of every arc
  int64_t E;              // entries of this level (arcs for level 2)
  int64_t e_lo;           // level 2: first arc
  const int32_t* tup;     // (I + 1) arrays of E: vertices, then f of the last one
  uint32_t* cnt;          // count mode: children per entry
  const int64_t* off;     // write mode: first child of every entry (minus off_shift)
  int64_t off_shift;
  int64_t p_lo, p_hi;     // entries of this chunk
  int32_t* out;           // write mode: (I + 2) arrays of out_E; emit mode: rows of I + 2
  int64_t out_E;          // write mode: entries of `out`; emit mode: row capacity
  unsigned long long* rows;  // emit mode: rows written so far (row cursor)
  unsigned long long* err;   // emit mode: set when a row would pass the capacity
  unsigned long long* hist;  // hist mode: class counts
  const int32_t* gid;        // batches: vertex -> graph (nullptr otherwise)
  unsigned long long* per_graph;  // batches: 21 class counts per graph (hist mode)
  unsigned long long* queue;
  unsigned long long* stat;  // neighbour elements scanned
  unsigned long long* carry; // wraps of the count accumulators (add_count)
};

// a[j] for a runtime j < N, without dynamic indexing (keeps `a` in registers)
template <int N>
__device__ __forceinline__ int32_t pick(const int32_t (&a)[N], int j) {
  int32_t r = a[0];
#pragma unroll
  for (int q = 1; q < N; q++) r = j == q ? a[q] : r;
  return r;
}

// x in a[0, len): branch-free binary search whose trip count depends only on
// len, so a warp searching one list for 32 keys does not diverge
__device__ __forceinline__ bool member_u(const int32_t* __restrict__ a, int len, int32_t x) {
  if (len <= 0) return false;
  int lo = 0;
  for (int n = len; n > 1;) {
    const int half = n >> 1;
    lo = __ldg(a + lo + half) <= x ? lo + half : lo;
    n -= half;
  }
  return __ldg(a + lo) == x;
}

// one warp per entry of a level of I-vertex tuples
template <int MODE, int I>
__global__ void __launch_bounds__(256) mg_extend(MgArgs A) {
  constexpr bool kLast = MODE == mgHist || MODE == mgEmit;
  __shared__ unsigned long long hist[kP5];
  __shared__ int8_t cls_of[kLast ? 1024 : 1];  // lanes look up different codes
  if (kLast) {
    if (MODE == mgHist)
      for (int t = threadIdx.x; t < kP5; t += blockDim.x) hist[t] = 0;
    for (int t = threadIdx.x; t < 1024; t += blockDim.x) cls_of[t] = c_cls[I - 2][t];
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  unsigned long long seen = 0;
  for (;;) {
    unsigned long long pe = 0;
    if (lane == 0) pe = atomicAdd(A.queue, 1ull);
    pe = __shfl_sync(kFull, pe, 0);
    const int64_t e = A.p_lo + (int64_t)pe;
    if (e >= A.p_hi) break;
    int32_t v[I];
    int fl = 0;
    bool valid = true;
    if (I == 2) {
      const int64_t a = A.e_lo + e;
      v[0] = A.src[a];
      v[1] = A.col[a];
      valid = v[1] > v[0];
    } else {
#pragma unroll
      for (int t = 0; t < I; t++) v[t] = A.tup[(int64_t)t * A.E + e];
      fl = A.tup[(int64_t)I * A.E + e];
    }
    int32_t st[I], ln[I], pre[I + 1];
    pre[0] = 0;
#pragma unroll
    for (int t = 0; t < I; t++) {
      st[t] = A.rp[v[t]];
      ln[t] = A.rp[v[t] + 1] - st[t];
    }
    // every candidate and every later vertex is above v_0: skip each list's prefix up to v_0
    {
      int skip = 0;
      if (lane < I) skip = lower_bound_dev(A.col + pick<I>(st, lane), pick<I>(ln, lane), v[0] + 1);
#pragma unroll
      for (int t = 0; t < I; t++) {
        const int x = __shfl_sync(kFull, skip, t);
        st[t] += x;
        ln[t] -= x;
        pre[t + 1] = pre[t] + ln[t];
      }
    }
    const int total = valid ? pre[I] : 0;
    int code_in = 0;  // adjacency among the I vertices of the entry
    if (kLast && valid) {
      // pairs (a, b) of positions, one per lane
      bool in = false;
      if (lane < I * (I - 1) / 2) {
        int a = 0, r = lane;
        while (r >= I - 1 - a) r -= I - 1 - a++;
        const int b = a + 1 + r;
        in = contains_dev(A.col + pick<I>(st, a), pick<I>(ln, a), pick<I>(v, b));
      }
      const unsigned bal = __ballot_sync(kFull, in);
      int q = 0;
#pragma unroll
      for (int a = 0; a < I; a++)
#pragma unroll
        for (int b = a + 1; b < I; b++, q++)
          if (bal >> q & 1) code_in |= 1 << pair_bit(a, b);
    }
    int64_t wpos = 0;
    if (MODE == mgWrite) wpos = A.off[e - A.p_lo] - A.off_shift;
    uint32_t cnt = 0;
    if (lane == 0) seen += (unsigned long long)total;
    for (int t0 = 0; t0 < total; t0 += 32) {
      const int t = t0 + lane;
      bool ok = false;
      int j = 0;
      int32_t u = 0;
      if (t < total) {
#pragma unroll
        for (int q = 1; q < I; q++) j += t >= pre[q] ? 1 : 0;
        u = A.col[pick<I>(st, j) + (t - pick<I + 1>(pre, j))];
        ok = u > v[0];
#pragma unroll
        for (int q = 1; q < I; q++) ok = ok && u != v[q];
        // first neighbour: u in no list of an earlier position (the lanes
        // that search list q search it with the same trip count)
#pragma unroll
        for (int q = 0; q < I - 1; q++)
          if (q < j && ok) ok = !member_u(A.col + st[q], ln[q], u);
        ok = ok && (j == I - 1 || fl < j || (fl == j && v[I - 1] < u));
      }
      if (MODE == mgCount) {
        cnt += ok ? 1u : 0u;
      } else if (MODE == mgWrite) {
        const unsigned bal = __ballot_sync(kFull, ok);
        if (ok) {
          const int64_t pos = wpos + __popc(bal & lt);
#pragma unroll
          for (int q = 0; q < I; q++) A.out[(int64_t)q * A.out_E + pos] = v[q];
          A.out[(int64_t)I * A.out_E + pos] = u;
          A.out[(int64_t)(I + 1) * A.out_E + pos] = j;
        }
        wpos += __popc(bal);
      } else {
        int cls = -1;
        if (ok) {
          // u's adjacency: j is its first neighbour; test the later positions
          int code = code_in | (1 << pair_bit(j, I));
#pragma unroll
          for (int q = 1; q < I; q++)
            if (q > j && member_u(A.col + st[q], ln[q], u)) code |= 1 << pair_bit(q, I);
          cls = cls_of[code];
        }
        if (MODE == mgHist) {
          // one atomic per distinct class among the 32 candidates (all of
          // one entry, so of one graph of a batch)
          const unsigned same = __match_any_sync(kFull, cls);
          if (cls >= 0 && lane == __ffs(same) - 1) {
            if (A.per_graph)
              add_count(A.per_graph + (int64_t)A.gid[v[0]] * kP5 + cls, (unsigned long long)__popc(same), false,
                        A.carry);
            else
              atomicAdd(&hist[cls], (unsigned long long)__popc(same));
          }
        } else {
          const unsigned bal = __ballot_sync(kFull, ok);
          unsigned long long base = 0;
          if (lane == 0 && bal) base = atomicAdd(A.rows, (unsigned long long)__popc(bal));
          base = __shfl_sync(kFull, base, 0);
          if (ok) {
            const unsigned long long pos = base + __popc(bal & lt);
            if (pos < (unsigned long long)A.out_E) {
              int32_t* row = A.out + (int64_t)pos * (I + 2);
#pragma unroll
              for (int q = 0; q < I; q++) row[q] = v[q];
              row[I] = u;
              row[I + 1] = cls;
            } else {
              atomicOr(A.err, 1ull);
            }
          }
        }
      }
    }
    if (MODE == mgCount) {
      cnt = warp_sum(cnt);
      if (lane == 0) A.cnt[e - A.p_lo] = cnt;
    }
  }
  if (MODE == mgHist) {
    __syncthreads();
    for (int t = threadIdx.x; t < kP5; t += blockDim.x)
      if (hist[t]) add_count(A.hist + t, hist[t], false, A.carry);
  }
  seen = warp_sum(seen);
  if (lane == 0 && seen) atomicAdd(A.stat, seen);
}

constexpr int kQg = 0, kRowsg = 1, kErrg = 2, kHistg = 8, kStatg = 32, kSlotsg = 40;

const char* mg_phase(int mode) {
  return mode == mgCount ? "extend_count" : mode == mgWrite ? "extend_write" : mode == mgHist ? "extend_sum" : "extend_emit";
}

struct MgRun {
  Graph& g;
  Workspace& ws;
  cudaStream_t s;
  int k;                  // motif size
  int64_t budget;
  int32_t* rows_out = nullptr;  // listing: caller's row buffer
  int64_t rows_cap = 0;
  HostSink* sink = nullptr;     // listing to host memory: staging buffers
  int64_t host_rows = 0;
  unsigned long long* per_graph = nullptr;  // batches: per-graph class counts
  double lvl_size[6] = {0, 0, 0, 0, 0, 0};
  int chunks = 0;

  template <int MODE, int I>
  pgm_status launch_t(MgArgs A) {
    A.queue = ws.ctr.p + kQg;
    A.rows = ws.ctr.p + kRowsg;
    A.err = ws.ctr.p + kErrg;
    A.hist = ws.ctr.p + kHistg;
    A.stat = ws.ctr.p + kStatg + I;
    A.carry = ws.ctr.p + kCarrySlot;
    PGM_TRY_CUDA(cudaMemsetAsync(A.queue, 0, sizeof(unsigned long long), s));
    const int64_t n = A.p_hi - A.p_lo;
    if (n <= 0) return PGM_OK;
    int grid = grid_for((const void*)mg_extend<MODE, I>, 256, 0);
    grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid, (n + 7) / 8));
    Profiler& prof = profiler();
    int id = prof.begin(mg_phase(MODE), I);
    mg_extend<MODE, I><<<grid, 256, 0, s>>>(A);
    PGM_CHECK_LAUNCH();
    prof.end(id, (double)n, 0.0);
    return PGM_OK;
  }

  template <int MODE>
  pgm_status launch(const MgArgs& A, int i) {
    switch (i) {
      case 2: return launch_t<MODE, 2>(A);
      case 3: return launch_t<MODE, 3>(A);
      case 4: return launch_t<MODE == mgWrite ? mgHist : MODE, 4>(A);  // never extended
    }
    set_error("motif engine: level %d", i);
    return PGM_EINVAL;
  }

  // entries [0, E) of level i (tuples `tup`, or arcs [e_lo, e_lo + E) for i = 2)
  pgm_status level(int i, const int32_t* tup, int64_t E, int64_t e_lo) {
    PGM_NVTX(kNvtxLevel[i < 13 ? i : 12]);
    if (E <= 0) return PGM_OK;
    lvl_size[i] += (double)E;
    MgArgs A;
    memset(&A, 0, sizeof(A));
    A.rp = g.rp;
    A.col = g.col;
    A.src = g.src;
    A.E = E;
    A.e_lo = e_lo;
    A.tup = tup;
    A.p_lo = 0;
    A.p_hi = E;
    A.gid = g.gid;
    A.per_graph = per_graph;
    const bool last = i == k - 1;
    if (last && !sink) {
      if (rows_out) {
        A.out = rows_out;
        A.out_E = rows_cap;
        return launch<mgEmit>(A, i);
      }
      return launch<mgHist>(A, i);
    }
    // inspection: children per entry (the rows themselves at the last level)
    PGM_TRY(ws.cnt[i].reserve((size_t)E));
    PGM_TRY(ws.off[i].reserve((size_t)E + 1));
    A.cnt = ws.cnt[i].p;
    PGM_TRY(launch<mgCount>(A, i));
    PGM_TRY(exclusive_scan(ws.cnt[i].p, E, ws.off[i].p, ws, s));
    int64_t T = 0;
    PGM_TRY(read_dev(ws.off[i].p + E, &T, s));
    if (T == 0) return PGM_OK;
    const int64_t B = last ? std::min<int64_t>(budget, sink->cap_rows) : budget;
    // children of entries [pa, pb) fit the budget (at least one entry per chunk)
    int64_t pa = 0;
    while (pa < E) {
      int64_t base, pb = E;
      PGM_TRY(read_dev(ws.off[i].p + pa, &base, s));
      if (T - base > B) {
        int64_t lo = pa + 1, hi = E;
        pb = pa + 1;
        while (lo <= hi) {
          const int64_t mid = lo + (hi - lo) / 2;
          int64_t om;
          PGM_TRY(read_dev(ws.off[i].p + mid, &om, s));
          if (om - base <= B) {
            pb = mid;
            lo = mid + 1;
          } else {
            hi = mid - 1;
          }
        }
      }
      int64_t ob;
      PGM_TRY(read_dev(ws.off[i].p + pb, &ob, s));
      const int64_t Tp = ob - base;
      chunks++;
      if (Tp > 0 && last) {
        // this chunk's rows into the current staging buffer
        if (Tp > sink->cap_rows) {
          set_error("list_motifs: %lld rows of one entry range exceed the staging buffer", (long long)Tp);
          return PGM_ENOMEM;
        }
        PGM_TRY(sink->reserve(Tp, s));
        PGM_TRY_CUDA(cudaMemsetAsync(ws.ctr.p + kRowsg, 0, sizeof(unsigned long long), s));
        A.p_lo = pa;
        A.p_hi = pb;
        A.out = sink->buf[sink->cur] + sink->fill * (int64_t)(k + 1);
        A.out_E = Tp;
        PGM_TRY(launch<mgEmit>(A, i));
        sink->fill += Tp;
        host_rows += Tp;
      } else if (Tp > 0) {
        PGM_TRY(ws.vid[i + 1].reserve((size_t)(i + 2) * (size_t)Tp));
        A.off = ws.off[i].p + pa;
        A.off_shift = base;
        A.p_lo = pa;
        A.p_hi = pb;
        A.out = ws.vid[i + 1].p;
        A.out_E = Tp;
        PGM_TRY(launch<mgWrite>(A, i));
        PGM_TRY(level(i + 1, ws.vid[i + 1].p, Tp, 0));
      }
      pa = pb;
    }
    return PGM_OK;
  }

  // the connected k-sets whose minimum vertex is in [v_lo, v_hi)
  // (*deferred: replaying a recorded plan, the counters are read by the caller later)
  pgm_status run(int32_t v_lo, int32_t v_hi, unsigned long long* h, bool* deferred) {
    if (g.n >= (1 << 30)) {
      set_error("motif engine: n=%d needs 30-bit vertex IDs", g.n);
      return PGM_EUNSUPPORTED;
    }
    PGM_TRY(upload_class_tables());
    PGM_TRY(graph_prepare_motifs(g));
    PGM_TRY(ws.ctr.reserve(kSlotsg));
    PGM_TRY_CUDA(cudaMemsetAsync(ws.ctr.p, 0, kSlotsg * sizeof(unsigned long long), s));
    if (!per_graph) PGM_TRY(seed_counts(ws.ctr.p + kHistg, kP5, s));
    const int64_t a_lo = g.h_rp[v_lo], a_hi = g.h_rp[v_hi];
    PGM_TRY(level(2, nullptr, a_hi - a_lo, a_lo));
    PGM_TRY(read_counters(ws.ctr.p, h, kSlotsg, s, deferred));
    if (*deferred) return PGM_OK;
    pgm_profile& lp = last_profile();
    Profiler& prof = profiler();
    if (prof.on) PGM_TRY(prof.finish(&lp));
    lp.level_size[1] = (uint64_t)(v_hi - v_lo);
    for (int l = 2; l < k; l++) lp.level_size[l] = (uint64_t)lvl_size[l];
    lp.chunks = chunks;
    return PGM_OK;
  }
};

}  // namespace

pgm_status count_motifs5(Graph& g, Workspace& ws, cudaStream_t s, int32_t v_lo, int32_t v_hi, uint64_t* out,
                         unsigned long long* per_graph_dev) {
  MgRun run{g, ws, s, 5, std::max<int64_t>(options().level_budget / 8, 1024)};
  run.per_graph = per_graph_dev;
  unsigned long long h[kSlotsg];
  bool deferred = false;
  PGM_TRY(run.run(v_lo, v_hi, h, &deferred));
  if (deferred) return PGM_OK;
  if (h[kCarrySlot]) {
    set_error("count_motifs: a count exceeds 2^64 - 1");
    return PGM_EOVERFLOW;
  }
  uint64_t t = 0;
  for (int c = 0; c < kP5; c++) t += out[c] = h[kHistg + c] - (per_graph_dev ? 0ull : count_seed());
  last_profile().level_size[5] = t;
  return PGM_OK;
}

pgm_status list_motifs(Graph& g, Workspace& ws, cudaStream_t s, int k, int32_t* out_dev, int64_t cap_rows,
                       int64_t* n_rows, HostSink* sink) {
  MgRun run{g, ws, s, k, std::max<int64_t>(options().level_budget / 8, 1024)};
  run.rows_out = out_dev;
  run.rows_cap = cap_rows;
  run.sink = sink;
  unsigned long long h[kSlotsg];
  bool deferred = false;
  PGM_TRY(run.run(0, g.n, h, &deferred));
  if (sink) {
    PGM_TRY(sink->flush(s));
    PGM_TRY(sink->finish());
    h[kRowsg] = (unsigned long long)run.host_rows;
  }
  *n_rows = (int64_t)h[kRowsg];
  if (h[kErrg] || (int64_t)h[kRowsg] > cap_rows) {
    set_error("list_motifs: %llu rows exceed the capacity of %lld", h[kRowsg], (long long)cap_rows);
    return PGM_EOVERFLOW;
  }
  last_profile().level_size[k] = h[kRowsg];
  return PGM_OK;
}

}  // namespace pgm

extern "C" {

static pgm_status list_motifs_to(pgm_graph* g, int32_t k, int32_t* out, int64_t cap_rows, int64_t* n_rows,
                                  bool host, const char* name) {
  if (!g || !n_rows || cap_rows < 0) {
    pgm::set_error("%s: bad arguments", name);
    return PGM_EINVAL;
  }
  if (k < 3 || k > 5) {
    pgm::set_error("%s: k=%d unsupported (3, 4 or 5)", name, k);
    return PGM_EUNSUPPORTED;
  }
  pgm::Graph& G = g->g;
  pgm::profiler().start(G.stream);
  uint64_t c[21] = {0};
  PGM_TRY(pgm::count_motifs(G, G.ws, G.stream, k, 0, G.n, c, nullptr));
  uint64_t total = 0;
  for (int i = 0; i < 21; i++) total += c[i];
  if (total > (uint64_t)INT64_MAX / (uint64_t)(k + 1)) {
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
  int64_t written = 0;
  pgm_status st = PGM_OK;
  if (!host) {
    pgm::profiler().start(G.stream);
    st = pgm::list_motifs(G, G.ws, G.stream, k, out, (int64_t)total, &written, nullptr);
  } else {
    // staging rows: a chunk holds at least one entry, whose rows are at most
    // the neighbours of its k - 1 vertices
    pgm::HostSink sink;
    sink.host = out;
    const int64_t staging = std::max<int64_t>(std::min<int64_t>(pgm::options().level_budget, (int64_t)1 << 26),
                                              (int64_t)(k - 1) * G.dmax);
    st = sink.init(k + 1, staging);
    if (st == PGM_OK) {
      pgm::profiler().start(G.stream);
      st = pgm::list_motifs(G, G.ws, G.stream, k, nullptr, (int64_t)total, &written, &sink);
    }
    cudaStreamSynchronize(G.stream);
    sink.release();
  }
  PGM_TRY(st);
  if (written != (int64_t)total) {
    pgm::set_error("%s: %lld rows written, %llu counted", name, (long long)written, (unsigned long long)total);
    return PGM_EINVAL;
  }
  return PGM_OK;
}

pgm_status pgm_list_motifs(pgm_graph* g, int32_t k, int32_t* out_dev, int64_t cap_rows, int64_t* n_rows) {
  PGM_NVTX("pgm_list_motifs");
  return list_motifs_to(g, k, out_dev, cap_rows, n_rows, false, "pgm_list_motifs");
}

pgm_status pgm_list_motifs_host(pgm_graph* g, int32_t k, int32_t* out_host, int64_t cap_rows, int64_t* n_rows) {
  PGM_NVTX("pgm_list_motifs_host");
  return list_motifs_to(g, k, out_host, cap_rows, n_rows, true, "pgm_list_motifs_host");
}

}  // extern "C"
