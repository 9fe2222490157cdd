// motif5.cu -- vertex-induced 5-motif counting (Sec. 3.3 Listing 4 with
// generic pattern classification, Sec. 3.2 canonical test).
//
// Levels are embedding lists of full vertex tuples (one int32 array per
// position, plus the index f of the last vertex's first neighbour in its
// prefix), built by inspection-execution (Sec. 5.3).  An entry
// (v_0 .. v_{i-1}) is extended by every vertex u of N(v_j) (j = 0 .. i-1)
// that passes the breadth-first canonical test of the motif engine: u > v_0,
// u not in the tuple, j = f(u) (u in no earlier vertex's list, so each
// candidate is generated once), and j = i - 1 or (f(v_{i-1}), v_{i-1}) <
// (j, u).  Membership uses binary search in the sorted lists (Sec. 5.4).
// The last level is fused with the reduction: each accepted 5-set is
// classified by its 10-bit adjacency code through a table of the 21
// connected 5-vertex graphs (generic classification in place of Listing
// 6's special cases) and counted in a per-block histogram.
//
// Class order: edge count, then the degree sequence (non-increasing,
// lexicographically smaller first), then the canonical code (the smallest
// adjacency code over the 120 relabellings; bit i = pair i of (0,1),(0,2),
// (0,3),(0,4),(1,2),(1,3),(1,4),(2,3),(2,4),(3,4)).
#include <algorithm>
#include <array>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace pgm {
namespace {

constexpr int kP5 = 21;
__constant__ int8_t c_p5_class[1024];  // adjacency code -> class, -1 if disconnected

// pair index of (a, b), a < b < 5, in the code's bit order
__host__ __device__ constexpr int pair_bit(int a, int b) {
  return a == 0 ? b - 1 : a == 1 ? 3 + b - 1 : a == 2 ? 6 + b - 2 : 9;
}

// Host: class of every code, from the definition above.
std::array<int8_t, 1024> build_p5_table() {
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
  auto connected = [&](int code) {
    int reach = 1;
    for (int it = 0; it < 5; it++)
      for (int a = 0; a < 5; a++)
        if (reach >> a & 1)
          for (int b = 0; b < 5; b++)
            if (adj(code, a, b)) reach |= 1 << b;
    return reach == 31;
  };
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
    std::array<int, 5> deg = {0, 0, 0, 0, 0};
    int e = 0;
    for (int a = 0; a < 5; a++)
      for (int b = a + 1; b < 5; b++)
        if (adj(code, a, b)) deg[a]++, deg[b]++, e++;
    std::sort(deg.begin(), deg.end(), [](int x, int y) { return x > y; });
    return std::make_tuple(e, deg, code);
  };
  std::sort(reps.begin(), reps.end(), [&](int x, int y) { return key(x) < key(y); });
  std::array<int8_t, 1024> t;
  t.fill(-1);
  for (int code = 0; code < 1024; code++)
    if (canon[code] >= 0)
      t[code] = (int8_t)(std::find(reps.begin(), reps.end(), canon[code]) - reps.begin());
  return t;
}

pgm_status upload_p5_table() {
  static std::mutex mu;
  static bool done[64] = {false};
  const int dev = device_id();
  std::lock_guard<std::mutex> lk(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return PGM_OK;
  static const std::array<int8_t, 1024> table = build_p5_table();
  PGM_TRY_CUDA(cudaMemcpyToSymbol(c_p5_class, table.data(), sizeof(c_p5_class)));
  if (dev >= 0 && dev < 64) done[dev] = true;
  return PGM_OK;
}

enum M5Mode : int { m5Count = 0, m5Write = 1, m5Last = 2 };

struct M5Args {
  const int32_t* rp;
  const int32_t* col;
  const int32_t* src;     // level 2 (implicit): source of every arc
  int i;                  // vertices per entry of this level
  int64_t E;              // entries of this level (arcs for level 2)
  int64_t e_lo;           // level 2: first arc
  const int32_t* tup;     // (i + 1) arrays of E: vertices, then f of the last one
  uint32_t* cnt;          // count mode: children per entry
  const int64_t* off;     // write mode: first child of every entry (minus off_shift)
  int64_t off_shift;
  int64_t p_lo, p_hi;     // entries of this chunk
  int32_t* out;           // write mode: (i + 2) arrays of out_E
  int64_t out_E;
  unsigned long long* hist;  // last mode: 21 class counts
  unsigned long long* queue;
  unsigned long long* stat;  // neighbour elements scanned
};

__device__ __forceinline__ bool m5_member(const int32_t* col, int32_t st, int32_t len, int32_t x) {
  return contains_dev(col + st, len, x);
}

// one warp per entry
template <int MODE>
__global__ void __launch_bounds__(256) m5_extend(M5Args A) {
  __shared__ unsigned long long hist[kP5];
  if (MODE == m5Last) {
    for (int t = threadIdx.x; t < kP5; t += blockDim.x) hist[t] = 0;
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
    int32_t v[4] = {0, 0, 0, 0};
    int fl = 0;
    const int i = A.i;
    bool valid = true;
    if (i == 2) {
      const int64_t a = A.e_lo + e;
      v[0] = A.src[a];
      v[1] = A.col[a];
      valid = v[1] > v[0];
    } else {
      for (int t = 0; t < i; t++) v[t] = A.tup[(int64_t)t * A.E + e];
      fl = A.tup[(int64_t)i * A.E + e];
    }
    int32_t st[4], ln[4], pre[5];
    pre[0] = 0;
    for (int t = 0; t < 4; t++) {
      st[t] = t < i ? A.rp[v[t]] : 0;
      ln[t] = t < i ? A.rp[v[t] + 1] - st[t] : 0;
      pre[t + 1] = pre[t] + ln[t];
    }
    const int total = valid ? pre[i] : 0;
    int code4 = 0;
    if (MODE == m5Last && valid) {
      // adjacency among the four vertices (6 pairs, one per lane)
      bool in = false;
      int a = 0, b = 0;
      if (lane < 6) {
        a = lane < 3 ? 0 : lane < 5 ? 1 : 2;
        b = lane < 3 ? lane + 1 : lane < 5 ? lane - 1 : 3;
        in = m5_member(A.col, st[a], ln[a], v[b]);
      }
      const unsigned bal = __ballot_sync(kFull, in);
      for (int q = 0; q < 6; q++) {
        const int qa = q < 3 ? 0 : q < 5 ? 1 : 2;
        const int qb = q < 3 ? q + 1 : q < 5 ? q - 1 : 3;
        if (bal >> q & 1) code4 |= 1 << pair_bit(qa, qb);
      }
    }
    int64_t wpos = 0;
    if (MODE == m5Write) wpos = A.off[e - A.p_lo] - A.off_shift;
    uint32_t cnt = 0;
    if (lane == 0) seen += (unsigned long long)total;
    for (int t0 = 0; t0 < total; t0 += 32) {
      const int t = t0 + lane;
      bool ok = false;
      int j = 0;
      int32_t u = 0;
      if (t < total) {
        j = t < pre[1] ? 0 : t < pre[2] ? 1 : t < pre[3] ? 2 : 3;
        u = A.col[st[j] + (t - pre[j])];
        ok = u > v[0];
        for (int q = 0; q < i; q++) ok = ok && u != v[q];
        for (int q = 0; q < j && ok; q++) ok = !m5_member(A.col, st[q], ln[q], u);
        ok = ok && (j == i - 1 || fl < j || (fl == j && v[i - 1] < u));
      }
      if (MODE == m5Count) {
        cnt += ok ? 1u : 0u;
      } else if (MODE == m5Write) {
        const unsigned bal = __ballot_sync(kFull, ok);
        if (ok) {
          const int64_t pos = wpos + __popc(bal & lt);
          for (int q = 0; q < i; q++) A.out[(int64_t)q * A.out_E + pos] = v[q];
          A.out[(int64_t)i * A.out_E + pos] = u;
          A.out[(int64_t)(i + 1) * A.out_E + pos] = j;
        }
        wpos += __popc(bal);
      } else if (ok) {
        // u's adjacency: j is its first neighbour; test the later ones
        int code = code4 | (1 << pair_bit(j, 4));
        for (int q = j + 1; q < 4; q++)
          if (m5_member(A.col, st[q], ln[q], u)) code |= 1 << pair_bit(q, 4);
        const int cls = c_p5_class[code];
        if (cls >= 0) atomicAdd(&hist[cls], 1ull);
      }
    }
    if (MODE == m5Count) {
      cnt = warp_sum(cnt);
      if (lane == 0) A.cnt[e - A.p_lo] = cnt;
    }
  }
  if (MODE == m5Last) {
    __syncthreads();
    for (int t = threadIdx.x; t < kP5; t += blockDim.x)
      if (hist[t]) atomicAdd(A.hist + t, hist[t]);
  }
  seen = warp_sum(seen);
  if (lane == 0 && seen) atomicAdd(A.stat, seen);
}

constexpr int kQ5 = 0, kHist5 = 8, kStat5 = 32, kSlots5 = 40;

struct M5Run {
  Graph& g;
  Workspace& ws;
  cudaStream_t s;
  int64_t budget;
  double lvl_size[6] = {0, 0, 0, 0, 0, 0};
  int chunks = 0;

  template <int MODE>
  pgm_status launch(const M5Args& A0) {
    M5Args A = A0;
    A.queue = ws.ctr.p + kQ5;
    A.hist = ws.ctr.p + kHist5;
    A.stat = ws.ctr.p + kStat5 + A.i;
    PGM_TRY_CUDA(cudaMemsetAsync(A.queue, 0, sizeof(unsigned long long), s));
    const int64_t n = A.p_hi - A.p_lo;
    if (n <= 0) return PGM_OK;
    int grid = grid_for((const void*)m5_extend<MODE>, 256, 0);
    grid = (int)std::max<int64_t>(1, std::min<int64_t>(grid, (n + 7) / 8));
    Profiler& prof = profiler();
    int id = prof.begin(MODE == m5Count ? "extend_count" : MODE == m5Write ? "extend_write" : "extend_sum", A.i);
    m5_extend<MODE><<<grid, 256, 0, s>>>(A);
    PGM_CHECK_LAUNCH();
    prof.end(id, (double)n, 0.0);
    return PGM_OK;
  }

  // entries [0, E) of level i (tuples `tup`, or arcs [e_lo, e_lo + E) for i = 2)
  pgm_status level(int i, const int32_t* tup, int64_t E, int64_t e_lo) {
    if (E <= 0) return PGM_OK;
    lvl_size[i] += (double)E;
    M5Args A;
    memset(&A, 0, sizeof(A));
    A.rp = g.rp;
    A.col = g.col;
    A.src = g.src;
    A.i = i;
    A.E = E;
    A.e_lo = e_lo;
    A.tup = tup;
    if (i == 4) {
      A.p_lo = 0;
      A.p_hi = E;
      return launch<m5Last>(A);
    }
    PGM_TRY(ws.cnt[i].reserve((size_t)E));
    PGM_TRY(ws.off[i].reserve((size_t)E + 1));
    A.cnt = ws.cnt[i].p;
    A.p_lo = 0;
    A.p_hi = E;
    PGM_TRY(launch<m5Count>(A));
    PGM_TRY(exclusive_scan(ws.cnt[i].p, E, ws.off[i].p, ws, s));
    int64_t T = 0;
    PGM_TRY(read_dev(ws.off[i].p + E, &T, s));
    if (T == 0) return PGM_OK;
    // children of entries [pa, pb) fit the budget (at least one entry per chunk)
    int64_t pa = 0;
    while (pa < E) {
      int64_t base, pb = E;
      PGM_TRY(read_dev(ws.off[i].p + pa, &base, s));
      if (T - base > budget) {
        int64_t lo = pa + 1, hi = E;
        pb = pa + 1;
        while (lo <= hi) {
          const int64_t mid = lo + (hi - lo) / 2;
          int64_t om;
          PGM_TRY(read_dev(ws.off[i].p + mid, &om, s));
          if (om - base <= budget) {
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
      if (Tp > 0) {
        PGM_TRY(ws.vid[i + 1].reserve((size_t)(i + 2) * (size_t)Tp));
        A.off = ws.off[i].p + pa;
        A.off_shift = base;
        A.p_lo = pa;
        A.p_hi = pb;
        A.out = ws.vid[i + 1].p;
        A.out_E = Tp;
        PGM_TRY(launch<m5Write>(A));
        PGM_TRY(level(i + 1, ws.vid[i + 1].p, Tp, 0));
      }
      pa = pb;
    }
    return PGM_OK;
  }
};

}  // namespace

pgm_status count_motifs5(Graph& g, Workspace& ws, cudaStream_t s, int32_t v_lo, int32_t v_hi, uint64_t* out) {
  if (g.n >= (1 << 30)) {
    set_error("count_motifs: n=%d needs 30-bit vertex IDs", g.n);
    return PGM_EUNSUPPORTED;
  }
  PGM_TRY(upload_p5_table());
  PGM_TRY(graph_prepare_motifs(g));
  PGM_TRY(ws.ctr.reserve(kSlots5));
  PGM_TRY_CUDA(cudaMemsetAsync(ws.ctr.p, 0, kSlots5 * sizeof(unsigned long long), s));
  M5Run run{g, ws, s, std::max<int64_t>(options().level_budget / 8, 1024)};
  const int64_t a_lo = g.h_rp[v_lo], a_hi = g.h_rp[v_hi];
  PGM_TRY(run.level(2, nullptr, a_hi - a_lo, a_lo));
  unsigned long long h[kSlots5];
  bool deferred = false;
  PGM_TRY(read_counters(ws.ctr.p, h, kSlots5, s, &deferred));
  for (int c = 0; c < kP5; c++) out[c] = h[kHist5 + c];
  pgm_profile& lp = last_profile();
  Profiler& prof = profiler();
  if (prof.on) PGM_TRY(prof.finish(&lp));
  lp.level_size[1] = (uint64_t)(v_hi - v_lo);
  for (int l = 2; l <= 4; l++) lp.level_size[l] = (uint64_t)run.lvl_size[l];
  uint64_t t = 0;
  for (int c = 0; c < kP5; c++) t += out[c];
  lp.level_size[5] = t;
  lp.chunks = run.chunks;
  return PGM_OK;
}

}  // namespace pgm
