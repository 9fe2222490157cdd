// common.cuh -- internals shared by the libpgm translation units: error
// reporting, options, device workspaces, launch profiling, record/replay
// plans and the warp-level primitives of the level engine (sorted-list
// search, warp scan).
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <string>
#include <memory>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pgm.h"

namespace pgm {

// ------------------------------------------------------------------ errors
void set_error(const char* fmt, ...);
const char* get_error();

#define PGM_TRY_CUDA(expr)                                                                     \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      ::pgm::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__,      \
                       __LINE__);                                                              \
      return e_ == cudaErrorMemoryAllocation ? PGM_ENOMEM : PGM_ECUDA;                         \
    }                                                                                          \
  } while (0)

#define PGM_TRY(expr)            \
  do {                           \
    pgm_status s_ = (expr);      \
    if (s_ != PGM_OK) return s_; \
  } while (0)

// every kernel launch of the library is followed by this check, which also
// counts it (pgm_kernel_launches)
void note_launches(uint64_t n);
#define PGM_CHECK_LAUNCH()              \
  do {                                  \
    ::pgm::note_launches(1);            \
    PGM_TRY_CUDA(cudaGetLastError());   \
  } while (0)

// NVTX range over a scope: every public counting, listing, mining and
// batch call (and each level of the level-wise engines) appears as a named
// range in Nsight Systems; without a tool attached a push/pop is a no-op.
struct NvtxScope {
  explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
  ~NvtxScope() { nvtxRangePop(); }
  NvtxScope(const NvtxScope&) = delete;
  NvtxScope& operator=(const NvtxScope&) = delete;
};
#define PGM_NVTX_CAT2(a, b) a##b
#define PGM_NVTX_CAT(a, b) PGM_NVTX_CAT2(a, b)
#define PGM_NVTX(name) ::pgm::NvtxScope PGM_NVTX_CAT(nvtx_scope_, __LINE__)(name)
// names of the level ranges of the level-wise engines
constexpr const char* kNvtxLevel[13] = {"level 0", "level 1", "level 2",  "level 3",  "level 4",  "level 5", "level 6",
                                        "level 7", "level 8", "level 9", "level 10", "level 11", "level 12"};

// ----------------------------------------------------------------- options
pgm_options& options();  // current options (defaults filled); read-only while counting
// Start value of the count accumulators (options.count_headroom_log2: 2^64 -
// 2^x, else 0) and the host write of it into n device slots (not while a
// plan is replayed).  Readback subtracts count_seed() again.
unsigned long long count_seed();
// counter-block slot of every engine that accumulates add_count() wraps
constexpr int kCarrySlot = 5;
pgm_status seed_counts(unsigned long long* dev, int n, cudaStream_t s);
int num_sms();            // SM count of the current device
int64_t l2_bytes();       // L2 cache size of the current device (bytes)
int device_id();

// ----------------------------------------------------------- device memory
// All device memory of the library (graphs, workspaces, scratch) comes from
// a stream-ordered pool of its own per device, which keeps up to
// kPoolKeepBytes of freed memory mapped: building and dropping graph
// handles, orientations and workspaces call after call then costs no
// mapping work (dropping an R-MAT 21 handle: 0.4 ms of cudaFree before,
// 0.02 ms from the pool).  dev_malloc returns memory that every
// stream may use (the allocation is complete on return); dev_free waits for
// the device like cudaFree, then returns the block to the pool.  An
// allocation that fails is retried once after the pool's cached memory is
// released.
constexpr uint64_t kPoolKeepBytes = (uint64_t)8 << 30;
cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t dev_free(void* p);
template <typename T>
cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc(reinterpret_cast<void**>(p), bytes);
}

// ------------------------------------------------------------ device array
// Grow-only device buffer owned by a handle; never shrinks until freed.
template <typename T>
struct DevArr {
  T* p = nullptr;
  size_t cap = 0;  // elements
  pgm_status reserve(size_t n) {
    if (n <= cap && p) return PGM_OK;
    if (p) dev_free(p);
    p = nullptr;
    cap = 0;
    size_t want = n ? n : 1;
    cudaError_t e = dev_malloc(&p, want * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      set_error("device allocation of %zu bytes failed: %s", want * sizeof(T), cudaGetErrorString(e));
      return PGM_ENOMEM;
    }
    cap = want;
    return PGM_OK;
  }
  void release() {
    if (p) dev_free(p);
    p = nullptr;
    cap = 0;
  }
};

// --------------------------------------------------------------- profiling
// Records CUDA events around each kernel launch on the launching stream
// when options().profile is set; folded into pgm_phase rows at the end of
// a public call.
struct Profiler {
  struct Rec {
    std::string name;
    int level;
    cudaEvent_t a, b;
    double entries, alg_bytes;
  };
  cudaStream_t stream = nullptr;
  bool on = false;
  std::vector<Rec> recs;
  void start(cudaStream_t s);
  int begin(const char* name, int level);             // returns record id or -1
  void end(int id, double entries, double alg_bytes);  // after the launch
  pgm_status finish(pgm_profile* out);                 // sync + fold into out
};
Profiler& profiler();         // thread-local
pgm_profile& last_profile();  // thread-local result of the last call

// ------------------------------------------------------------ graph state
// Scratch of one counting call: level lists, counters, hub queues.  A graph
// handle owns one; the server owns one per in-flight slot.
struct Workspace {
  static constexpr int kMaxLevels = 12;
  DevArr<uint32_t> cnt[kMaxLevels];  // per-entry child counts (inspection)
  DevArr<int64_t> off[kMaxLevels];   // exclusive scan of cnt (execution offsets)
  DevArr<int32_t> vid[kMaxLevels];   // materialised level lists
  DevArr<int64_t> big;               // hub parents of one launch
  DevArr<unsigned long long> ctr;    // queue counters + accumulators
  DevArr<int64_t> scan_tmp;          // block partials of the scan
  DevArr<int32_t> scratch;           // per-warp spill lists of the hub kernels
  DevArr<uint2> tri;                 // motifs: per-arc triangle counts of the level-2 edges
  DevArr<uint32_t> dom;              // frequent subgraph mining: domain bitmaps
  void release_all();
};

// Device-resident graph.  Everything but `ws` is immutable after
// orientation and motif preparation, so several streams may count on it
// concurrently with their own workspaces.
struct Graph {
  int32_t n = 0;
  int64_t narcs = 0;           // 2 m
  int32_t* rp = nullptr;       // int32[n+1] undirected CSR
  int32_t* col = nullptr;      // int32[narcs]
  int32_t* dag_rp = nullptr;   // int32[n+1] oriented DAG
  int32_t* dag_col = nullptr;  // int32[m]
  int32_t* up = nullptr;       // up[v] = first arc of v whose neighbour is > v
  int32_t* gid = nullptr;      // batches: vertex -> graph id (nullptr otherwise)
  int32_t* src = nullptr;      // motifs: source vertex of every arc
  int32_t* rev = nullptr;      // motifs: index of the reverse arc (v -> u) of every arc u -> v
  int32_t* labels = nullptr;   // frequent subgraph mining: vertex labels (pgm_graph_set_labels)
  int32_t* label_rank = nullptr;       // vertex -> its index among the vertices of its label
  std::vector<int64_t> h_label_count;  // vertices per label
  int32_t* wedge_centres = nullptr;    // vertices of degree >= 2 in (label, ID) order
  int64_t* wedge_prefix = nullptr;     // exclusive prefix of C(d, 2) over wedge_centres (n_centres + 1)
  int64_t n_wedge_centres = 0, n_wedges = 0;
  int32_t* hub_idx = nullptr;  // motifs: vertex -> row of hub_bits, or -1
  uint32_t* hub_bits = nullptr;  // motifs: adjacency bitmaps of the highest-degree vertices
  int64_t hub_words = 0;       // 32-bit words per bitmap row
  int32_t nhubs = 0;
  int32_t G = 1;
  int64_t dmax = 0, dag_dmax = 0;
  bool oriented = false;
  cudaStream_t stream = nullptr;
  std::vector<int64_t> h_dag_rp;  // host copy of the DAG row pointers (edge blocking), lazy
  std::vector<int64_t> h_rp;      // host copy of the CSR row pointers, lazy
  std::recursive_mutex mu;        // orientation, lazy host copies, motif helpers, relabelled copies
  Workspace ws;                   // workspace of calls made through the handle
  std::unique_ptr<Graph> relabeled[2];  // copies with IDs in ascending / descending degree order
};

constexpr int kOrderAscending = 0, kOrderDescending = 1;

pgm_status graph_upload(Graph& g, int32_t n, const int64_t* rowptr, const int32_t* col,
                        bool rowptr_on_device, int64_t narcs, uint32_t flags, cudaStream_t s);
pgm_status graph_orient(Graph& g);
pgm_status graph_prepare_motifs(Graph& g);
// host copies of the row pointers (g.h_rp, g.h_dag_rp), made on first use;
// never called while a stream capture is open (a batch records first)
pgm_status graph_host_rp(Graph& g);
pgm_status graph_host_dag_rp(Graph& g);
// arcs of the DAG whose source lies in [v_lo, v_hi)
pgm_status graph_dag_arcs(Graph& g, int32_t v_lo, int32_t v_hi, int64_t* arcs);
// 5-motif counts (21 classes) of the connected 5-sets whose minimum vertex is in [v_lo, v_hi)
// (per_graph_dev: batches, 21 counts per graph added on the device instead)
pgm_status count_motifs5(Graph& g, Workspace& ws, cudaStream_t s, int32_t v_lo, int32_t v_hi, uint64_t* out,
                         unsigned long long* per_graph_dev);
// rows of k IDs (canonical order) + class of every connected k-set, k = 3..5, into out_dev
struct HostSink;
// (sink: rows streamed to host memory instead, out_dev unused)
pgm_status list_motifs(Graph& g, Workspace& ws, cudaStream_t s, int k, int32_t* out_dev, int64_t cap_rows,
                       int64_t* n_rows, HostSink* sink);
// motif count on exactly this graph's IDs (count_motifs may switch to a relabelled copy)
pgm_status count_motifs_on(Graph& g, Workspace& ws, cudaStream_t s, int k, int32_t v_lo, int32_t v_hi,
                           uint64_t* out, unsigned long long* per_graph_dev);
// copy of g with vertex IDs in degree order (kOrderAscending / kOrderDescending),
// each graph of a batch within its own block; built on first use
pgm_status graph_relabeled(Graph& g, int order, Graph** out);
// out[i] = (int32) in[i] on the stream
void narrow_rowptr(const int64_t* in, int32_t* out, int64_t len, cudaStream_t s);
void graph_free(Graph& g);

// Rows streamed to host memory: the last level of every edge-blocking chunk
// is emitted into one of two device staging buffers; a full buffer is
// copied to the host on a copy stream while the counting stream fills the
// other.  Chunks are cut so that one chunk's rows fit a staging buffer;
// device memory stays bounded by the staging size whatever the number of
// rows.
struct HostSink {
  int32_t* host = nullptr;  // caller's rows
  int64_t cap_rows = 0;     // rows per staging buffer
  int64_t written = 0;      // rows already copied (or being copied) to the host
  int64_t fill = 0;         // rows in the current staging buffer
  int cur = 0;
  int32_t* buf[2] = {nullptr, nullptr};
  cudaStream_t copy = nullptr;
  cudaEvent_t filled[2] = {nullptr, nullptr};  // on the counting stream: buffer's rows written
  cudaEvent_t done[2] = {nullptr, nullptr};    // on the copy stream: buffer copied out
  int k = 0;  // int32 per row

  pgm_status init(int row_ints, int64_t rows) {
    k = row_ints;
    cap_rows = rows;
    PGM_TRY_CUDA(cudaStreamCreateWithFlags(&copy, cudaStreamNonBlocking));
    for (int b = 0; b < 2; b++) {
      PGM_TRY_CUDA(dev_malloc(&buf[b], (size_t)rows * k * sizeof(int32_t)));
      PGM_TRY_CUDA(cudaEventCreateWithFlags(&filled[b], cudaEventDisableTiming));
      PGM_TRY_CUDA(cudaEventCreateWithFlags(&done[b], cudaEventDisableTiming));
    }
    return PGM_OK;
  }
  // hand the current buffer to the copy stream; the counting stream then
  // writes the other one once its previous copy has finished
  pgm_status flush(cudaStream_t s) {
    if (fill > 0) {
      PGM_TRY_CUDA(cudaEventRecord(filled[cur], s));
      PGM_TRY_CUDA(cudaStreamWaitEvent(copy, filled[cur], 0));
      PGM_TRY_CUDA(cudaMemcpyAsync(host + written * k, buf[cur], (size_t)fill * k * sizeof(int32_t),
                                   cudaMemcpyDeviceToHost, copy));
      PGM_TRY_CUDA(cudaEventRecord(done[cur], copy));
      written += fill;
      fill = 0;
      cur ^= 1;
      PGM_TRY_CUDA(cudaStreamWaitEvent(s, done[cur], 0));  // no-op before the buffer's first copy
    }
    return PGM_OK;
  }
  pgm_status finish() {
    if (copy) PGM_TRY_CUDA(cudaStreamSynchronize(copy));
    return PGM_OK;
  }
  // staging space for n more rows (n <= cap_rows)
  pgm_status reserve(int64_t n, cudaStream_t s) {
    if (fill + n > cap_rows) PGM_TRY(flush(s));
    return PGM_OK;
  }
  void release() {
    if (copy) cudaStreamSynchronize(copy);
    for (int b = 0; b < 2; b++) {
      if (buf[b]) dev_free(buf[b]);
      if (filled[b]) cudaEventDestroy(filled[b]);
      if (done[b]) cudaEventDestroy(done[b]);
      buf[b] = nullptr;
      filled[b] = done[b] = nullptr;
    }
    if (copy) cudaStreamDestroy(copy);
    copy = nullptr;
  }
};

// scan: out[i] = sum cnt[0..i), out[len] = total (device pointers)
pgm_status exclusive_scan(const uint32_t* cnt, int64_t len, int64_t* out, Workspace& ws,
                          cudaStream_t s);

// ------------------------------------------------------- record / replay
// The engines read a few values back from the device (level totals and
// edge-blocking boundaries).  A Plan recorded on a first run lets the same
// launch sequence be replayed without those reads -- the condition for
// capturing it in a CUDA graph.  In replay mode the final counter readback
// is an async copy into `pinned_ctr`, read by the caller after the stream
// (or graph launch) completes.
struct Plan {
  bool record = false;
  bool replay = false;
  std::vector<int64_t> v;
  size_t cur = 0;
  unsigned long long* pinned_ctr = nullptr;  // host-pinned copy target (replay)
};
Plan*& current_plan();  // thread-local, nullptr when not planning

template <typename T>
pgm_status read_dev(const T* p, T* out, cudaStream_t s) {
  Plan* pl = current_plan();
  if (pl && pl->replay) {
    if (pl->cur >= pl->v.size()) {
      set_error("plan replay: more reads than recorded");
      return PGM_EINVAL;
    }
    *out = (T)pl->v[pl->cur++];
    return PGM_OK;
  }
  PGM_TRY_CUDA(cudaMemcpyAsync(out, p, sizeof(T), cudaMemcpyDeviceToHost, s));
  PGM_TRY_CUDA(cudaStreamSynchronize(s));
  if (pl && pl->record) pl->v.push_back((int64_t)*out);
  return PGM_OK;
}

// Final readback of an engine's counter block: synchronous normally, an
// async copy into the plan's pinned buffer when replaying (then *deferred
// is set and the values are not yet on the host).
pgm_status read_counters(const unsigned long long* dev, unsigned long long* host, size_t n,
                         cudaStream_t s, bool* deferred);

// counting engines (results written on PGM_OK; per_graph_dev: batches)
pgm_status count_kcliques(Graph& g, Workspace& ws, cudaStream_t s, int k, int32_t v_lo,
                          int32_t v_hi, uint64_t* out, unsigned long long* per_graph_dev);
// bitset engine: level_sizes[l] = entries of level l (3 <= l < k),
// level_sizes[kBmLevelRead] = adjacency elements read (array of kBmLevelRead + 1)
constexpr int kBmLevelRead = 11;
pgm_status count_kcliques_bitset(Graph& g, Workspace& ws, cudaStream_t s, int k, int32_t v_lo,
                                 int32_t v_hi, uint64_t* out, unsigned long long* per_graph_dev,
                                 uint64_t* level_sizes);
pgm_status count_motifs(Graph& g, Workspace& ws, cudaStream_t s, int k, int32_t v_lo,
                        int32_t v_hi, uint64_t* out, unsigned long long* per_graph_dev);
// device bytes of the bitset engine's global row scratch for a k-clique
// count on g, as count_kcliques_bitset reserves it (0 if all rows fit in
// shared memory); used by the server's memory prediction
int64_t bitset_scratch_bytes(const Graph& g, int k);
int64_t bitset_row_words(int64_t dmax, int k);

// persistent-grid size for a kernel
int grid_for(const void* fn, int threads, size_t smem);
// raise a kernel's dynamic shared-memory limit once per process
pgm_status smem_attr(const void* fn, int bytes);

// -------------------------------------------------------- checked indexing
// Builds with PGM_DEBUG check the index of every marked global access
// against the length of its array (PGM_IDX_OK(i, n)): a violation adds one
// to a device error word of the translation unit, the first one records its
// source line and index, and the caller skips the access (a load yields a
// neutral value).  Nothing traps.  Without PGM_DEBUG the check compiles to
// `true`.  pgm_debug_errors() sums the words of all translation units.
#ifdef PGM_DEBUG
struct DebugWord {
  unsigned long long count, line, index;
};
static __device__ DebugWord g_pgm_debug;
__device__ __forceinline__ bool idx_ok(long long i, long long n, int line) {
  if (i >= 0 && i < n) return true;
  if (atomicAdd(&g_pgm_debug.count, 1ull) == 0ull) {
    g_pgm_debug.line = (unsigned long long)line;
    g_pgm_debug.index = (unsigned long long)i;
  }
  return false;
}
// host: register this translation unit's word (reader and reset) by name
int register_debug_word(const char* file, cudaError_t (*read)(DebugWord*), cudaError_t (*reset)());
static cudaError_t read_debug_word(DebugWord* out) { return cudaMemcpyFromSymbol(out, g_pgm_debug, sizeof(DebugWord)); }
static cudaError_t reset_debug_word() {
  DebugWord z = {0, 0, 0};
  return cudaMemcpyToSymbol(g_pgm_debug, &z, sizeof(z));
}
static const int g_debug_registered = register_debug_word(__FILE__, read_debug_word, reset_debug_word);
#else
__device__ __forceinline__ bool idx_ok(long long, long long, int) { return true; }
#endif
#define PGM_IDX_OK(i, n) ::pgm::idx_ok((long long)(i), (long long)(n), __LINE__)

// -------------------------------------------------------- device helpers
constexpr unsigned kFull = 0xffffffffu;

// first index i in [0, n) with a[i] >= x (n if none)
__device__ __forceinline__ int lower_bound_dev(const int32_t* __restrict__ a, int n, int32_t x) {
  int lo = 0;
  while (n > 0) {
    int half = n >> 1;
    int32_t v = a[lo + half];
    if (v < x) {
      lo += half + 1;
      n -= half + 1;
    } else {
      n = half;
    }
  }
  return lo;
}

__device__ __forceinline__ bool contains_dev(const int32_t* __restrict__ a, int n, int32_t x) {
  int i = lower_bound_dev(a, n, x);
  return i < n && a[i] == x;
}

__device__ __forceinline__ int warp_inclusive_scan(int v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    int t = __shfl_up_sync(kFull, v, d);
    if (lane >= d) v += t;
  }
  return v;
}

// lane of the owner of item t, given each lane's inclusive prefix `incl`
// of item counts (non-decreasing): the number of incl values <= t
__device__ __forceinline__ int warp_owner(int incl, int t) {
  int q = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1) {
    int v = __shfl_sync(kFull, incl, q + step - 1);
    if (v <= t) q += step;
  }
  return q;
}

// Adds one warp's partial count s to a uint64 accumulator and records a
// wrap in *carry: +1 when the sum passes 2^64 - 1 upward, -1 (two's
// complement) when a negative partial of a signed sum (sgn) passes 0
// downward.  The accumulated total lies in [0, 2^64) exactly when *carry
// ends at 0 (PGM_EOVERFLOW otherwise).
__device__ __forceinline__ void add_count(unsigned long long* acc, unsigned long long s, bool sgn,
                                          unsigned long long* carry) {
  const unsigned long long old = atomicAdd(acc, s);
  const unsigned long long now = old + s;
  if (sgn && (long long)s < 0) {
    if (now > old) atomicAdd(carry, ~0ull);
  } else if (now < old) {
    atomicAdd(carry, 1ull);
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
  return v;
}

}  // namespace pgm

struct pgm_graph {
  pgm::Graph g;
};
