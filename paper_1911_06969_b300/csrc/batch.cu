// batch.cu -- counting many graphs in one pass (not in the paper: the
// many-small-graphs batching pattern).
//
// A batch is the disjoint union of G graphs in one CSR.  Because no arc
// leaves its graph, one run of the level engine over the union enumerates
// exactly the embeddings of every graph; each kernel attributes a count to
// the graph of the embedding's first vertex (vertex -> graph map `gid`),
// flushing its per-warp counters only when the graph changes.  The engine's
// persistent kernels pull parents from a device queue, so small graphs of
// very different sizes share the whole GPU instead of each under-filling it.
//
// The launch sequence can be captured once in a CUDA graph and replayed: a
// first run records the few values the host reads back (level totals and
// edge-blocking boundaries, identical on every run of the same batch), and
// the capture replays them, so the graph contains no host synchronisation.
// Each captured configuration owns its workspace, so its device pointers
// stay valid for the lifetime of the batch.
//
// The baseline the batch is measured against, pgm_batch_count_motifs_loop,
// runs the plain per-graph path (pgm_count_motifs_range on each graph's
// vertex range) in a host loop, with its natural per-level syncs.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>
#include <memory>
#include <new>

#include "common.cuh"

namespace pgm {

__global__ void gid_kernel(int32_t n, const int64_t* __restrict__ vtx_off, int32_t G,
                           int32_t* __restrict__ gid) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    // last graph whose first vertex is <= v
    int lo = 0, hi = G - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (vtx_off[mid] <= v) lo = mid;
      else hi = mid - 1;
    }
    gid[v] = lo;
  }
}

__global__ void crossing_kernel(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                const int32_t* __restrict__ gid, unsigned* __restrict__ bad) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int g = gid[v];
    for (int32_t a = rp[v]; a < rp[v + 1]; a++) {
      const int32_t u = col[a];
      if (u < 0 || u >= n || gid[u] != g) {
        atomicOr(bad, 1u);
        break;
      }
    }
  }
}

}  // namespace pgm

struct pgm_batch {
  pgm::Graph g;
  int32_t G = 0;
  std::vector<int64_t> vtx_off;
  pgm::DevArr<unsigned long long> per_graph;  // G * 21 (the largest pattern count, k = 5)
  unsigned long long* pinned_pg = nullptr;    // host-pinned copy of per_graph
  unsigned long long* pinned_ctr = nullptr;   // host-pinned counter block
  cudaStream_t own_stream = nullptr;          // created when the caller passes NULL
  struct Cap {
    int kind, k;
    pgm_tune t;
    cudaGraphExec_t exec = nullptr;
    uint64_t kernel_nodes = 0;
    std::unique_ptr<pgm::Workspace> ws;
  };
  std::vector<std::unique_ptr<Cap>> caps;
};

namespace pgm {
namespace {

enum Kind { kMotif = 0, kClique = 1 };

// apply a tune to the process options for the duration of one call
struct TuneScope {
  pgm_options saved;
  explicit TuneScope(const pgm_tune* t) : saved(options()) {
    if (!t) return;
    pgm_options& o = options();
    if (t->block_threads) o.block_threads = t->block_threads;
    if (t->warp_stage_cap) o.warp_stage_cap = t->warp_stage_cap;
    if (t->hub_threshold) o.hub_threshold = t->hub_threshold;
    if (t->blocks_per_sm) o.blocks_per_sm = t->blocks_per_sm;
    if (t->motif_b_side_min) o.motif_b_side_min = t->motif_b_side_min;
    if (t->reverse_ratio) o.reverse_ratio = t->reverse_ratio;
    if (t->bitset_forward_ratio) o.bitset_forward_ratio = t->bitset_forward_ratio;
  }
  ~TuneScope() { options() = saved; }
};

pgm_status check_tune(const pgm_tune* t) {
  if (!t) return PGM_OK;
  if (t->block_threads && (t->block_threads < 64 || t->block_threads > 512 || t->block_threads % 32)) {
    set_error("tune: block_threads must be a multiple of 32 in [64, 512]");
    return PGM_EINVAL;
  }
  if (t->warp_stage_cap && (t->warp_stage_cap < 32 || t->warp_stage_cap > 4096)) {
    set_error("tune: warp_stage_cap must be in [32, 4096]");
    return PGM_EINVAL;
  }
  {
    const int th = t->block_threads ? t->block_threads : options().block_threads;
    const int cp = t->warp_stage_cap ? t->warp_stage_cap : options().warp_stage_cap;
    if ((th / 32) * cp > 16384) {
      set_error("tune: block_threads / 32 * warp_stage_cap must be <= 16384 (shared memory)");
      return PGM_EINVAL;
    }
  }
  if (t->hub_threshold && t->hub_threshold < 2) {
    set_error("tune: hub_threshold must be >= 2");
    return PGM_EINVAL;
  }
  if (t->blocks_per_sm < 0) {
    set_error("tune: blocks_per_sm must be >= 0");
    return PGM_EINVAL;
  }
  return PGM_OK;
}

int npat(int kind, int k) { return kind == kClique ? 1 : (k == 3 ? 2 : k == 4 ? 6 : 21); }

pgm_status engine(pgm_batch* b, Workspace& ws, int kind, int k, unsigned long long* pg) {
  uint64_t tmp[21];
  Graph& g = b->g;
  if (kind == kMotif) return count_motifs(g, ws, g.stream, k, 0, g.n, tmp, pg);
  return count_kcliques(g, ws, g.stream, k, 0, g.n, tmp, pg);
}

bool same_tune(const pgm_tune& a, const pgm_tune& c) {
  return a.block_threads == c.block_threads && a.warp_stage_cap == c.warp_stage_cap &&
         a.hub_threshold == c.hub_threshold && a.blocks_per_sm == c.blocks_per_sm &&
         a.motif_b_side_min == c.motif_b_side_min && a.reverse_ratio == c.reverse_ratio &&
         a.bitset_forward_ratio == c.bitset_forward_ratio;
}

// counters block layout shared with the engines: error slots to inspect
pgm_status check_err_slots(const unsigned long long* h, int kind) {
  const unsigned long long e = kind == kMotif ? h[7] : h[15];
  if (e) {
    set_error("batch: internal hub-list overflow");
    return PGM_ENOMEM;
  }
  if (h[kCarrySlot]) {
    set_error("batch: a count exceeds 2^64 - 1");
    return PGM_EOVERFLOW;
  }
  return PGM_OK;
}

pgm_status run_batch(pgm_batch* b, int kind, int k, uint64_t* out, const pgm_tune* t) {
  PGM_TRY(check_tune(t));
  Graph& g = b->g;
  cudaStream_t s = g.stream;
  const int np = npat(kind, k);
  if (kind == kClique && k <= 2) {
    PGM_TRY(graph_host_rp(g));
    for (int i = 0; i < b->G; i++) {
      const int64_t v0 = b->vtx_off[i], v1 = b->vtx_off[i + 1];
      out[i] = k == 1 ? (uint64_t)(v1 - v0) : (uint64_t)((g.h_rp[v1] - g.h_rp[v0]) / 2);
    }
    return PGM_OK;
  }
  if (kind == kMotif && (k < 3 || k > 5)) {
    set_error("batch: motif size k=%d unsupported (3, 4 or 5)", k);
    return PGM_EUNSUPPORTED;
  }
  if (kind == kClique && (k < 1 || k > 10)) {
    set_error("batch: clique size k=%d outside [1, 10]", k);
    return PGM_EUNSUPPORTED;
  }
  TuneScope scope(t);
  const size_t pg_bytes = (size_t)b->G * np * sizeof(unsigned long long);
  const bool use_graph = t && t->use_graph;
  if (!use_graph) {
    profiler().start(s);
    PGM_TRY_CUDA(cudaMemsetAsync(b->per_graph.p, 0, pg_bytes, s));
    PGM_TRY(engine(b, g.ws, kind, k, b->per_graph.p));
    PGM_TRY_CUDA(cudaMemcpyAsync(b->pinned_pg, b->per_graph.p, pg_bytes, cudaMemcpyDeviceToHost, s));
    PGM_TRY_CUDA(cudaStreamSynchronize(s));
    memcpy(out, b->pinned_pg, pg_bytes);
    return PGM_OK;
  }
  pgm_batch::Cap* cap = nullptr;
  for (auto& c : b->caps)
    if (c->kind == kind && c->k == k && same_tune(c->t, *t)) cap = c.get();
  if (!cap) {
    if (b->caps.size() >= 4) {  // bound the memory held by captured workspaces
      auto& old = b->caps.front();
      if (old->exec) cudaGraphExecDestroy(old->exec);
      old->ws->release_all();
      b->caps.erase(b->caps.begin());
    }
    auto c = std::make_unique<pgm_batch::Cap>();
    c->kind = kind;
    c->k = k;
    c->t = *t;
    c->ws = std::make_unique<Workspace>();
    // 1) record the host reads (and size every buffer of the workspace)
    Plan plan;
    plan.record = true;
    current_plan() = &plan;
    profiler().start(s);
    profiler().on = false;
    pgm_status st = cudaMemsetAsync(b->per_graph.p, 0, pg_bytes, s) == cudaSuccess ? PGM_OK : PGM_ECUDA;
    if (st == PGM_OK) st = engine(b, *c->ws, kind, k, b->per_graph.p);
    current_plan() = nullptr;
    PGM_TRY(st);
    // 2) capture the same sequence, replaying the recorded reads
    plan.record = false;
    plan.replay = true;
    plan.cur = 0;
    plan.pinned_ctr = b->pinned_ctr;
    cudaGraph_t graph = nullptr;
    PGM_TRY_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    current_plan() = &plan;
    st = PGM_OK;
    if (cudaMemsetAsync(b->per_graph.p, 0, pg_bytes, s) != cudaSuccess) st = PGM_ECUDA;
    if (st == PGM_OK) st = engine(b, *c->ws, kind, k, b->per_graph.p);
    if (st == PGM_OK &&
        cudaMemcpyAsync(b->pinned_pg, b->per_graph.p, pg_bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      st = PGM_ECUDA;
    current_plan() = nullptr;
    cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (st != PGM_OK || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      if (st == PGM_OK) set_error("batch: stream capture failed: %s", cudaGetErrorString(ce));
      return st == PGM_OK ? PGM_ECUDA : st;
    }
    if (plan.cur != plan.v.size()) {
      cudaGraphDestroy(graph);
      set_error("batch: replay consumed %zu of %zu recorded reads", plan.cur, plan.v.size());
      return PGM_EINVAL;
    }
    size_t nn = 0;
    if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn > 0) {
      std::vector<cudaGraphNode_t> nodes(nn);
      if (cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess)
        for (size_t i = 0; i < nn; i++) {
          cudaGraphNodeType ty;
          if (cudaGraphNodeGetType(nodes[i], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel)
            c->kernel_nodes++;
        }
    }
    cudaGetLastError();
    cudaError_t ie = cudaGraphInstantiate(&c->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      c->exec = nullptr;
      set_error("batch: graph instantiation failed: %s", cudaGetErrorString(ie));
      return PGM_ECUDA;
    }
    cap = c.get();
    b->caps.push_back(std::move(c));
  }
  PGM_TRY_CUDA(cudaGraphLaunch(cap->exec, s));
  note_launches(cap->kernel_nodes);
  PGM_TRY_CUDA(cudaStreamSynchronize(s));
  PGM_TRY(check_err_slots(b->pinned_ctr, kind));
  memcpy(out, b->pinned_pg, pg_bytes);
  return PGM_OK;
}

// --------------------------------------------------------- autotune cache
// Winners of pgm_batch_autotune_ex kept in a small JSON object, one entry
// per line: "<key>": {"block_threads": .., "warp_stage_cap": ..,
// "hub_threshold": .., "blocks_per_sm": .., "motif_b_side_min": ..,
// "reverse_ratio": .., "bitset_forward_ratio": .., "ms": ..}.  The key holds
// the motif size and the batch's features rounded down to powers of two:
// graphs, vertices, arcs and largest degree.
int ilog2(int64_t x) {
  int l = 0;
  while (x > 1) {
    x >>= 1;
    l++;
  }
  return l;
}

std::string tune_key(pgm_batch* b, int k) {
  char buf[128];
  snprintf(buf, sizeof(buf), "motif%d_G2^%d_n2^%d_arcs2^%d_dmax2^%d", k, ilog2(b->G), ilog2(b->g.n),
           ilog2(b->g.narcs), ilog2(b->g.dmax));
  return buf;
}

// every "key": {...} line of the file (an absent or unreadable file is empty)
std::vector<std::pair<std::string, std::string>> tune_cache_read(const char* path) {
  std::vector<std::pair<std::string, std::string>> out;
  FILE* f = fopen(path, "r");
  if (!f) return out;
  char line[1024];
  while (fgets(line, sizeof(line), f)) {
    const char* q0 = strchr(line, '"');
    const char* q1 = q0 ? strchr(q0 + 1, '"') : nullptr;
    const char* b0 = q1 ? strchr(q1, '{') : nullptr;
    const char* b1 = b0 ? strchr(b0, '}') : nullptr;
    if (!b1) continue;
    out.emplace_back(std::string(q0 + 1, q1), std::string(b0, b1 + 1));
  }
  fclose(f);
  return out;
}

bool json_field(const std::string& body, const char* name, double* v) {
  const std::string pat = std::string("\"") + name + "\":";
  const size_t i = body.find(pat);
  if (i == std::string::npos) return false;
  return sscanf(body.c_str() + i + pat.size(), "%lf", v) == 1;
}

bool tune_cache_get(const char* path, const std::string& key, pgm_tune* t, double* ms) {
  for (const auto& e : tune_cache_read(path)) {
    if (e.first != key) continue;
    double v[8];
    static const char* names[8] = {"block_threads", "warp_stage_cap", "hub_threshold", "blocks_per_sm",
                                   "motif_b_side_min", "reverse_ratio", "bitset_forward_ratio", "ms"};
    for (int i = 0; i < 8; i++)
      if (!json_field(e.second, names[i], &v[i])) return false;
    memset(t, 0, sizeof(*t));
    t->block_threads = (int32_t)v[0];
    t->warp_stage_cap = (int32_t)v[1];
    t->hub_threshold = (int32_t)v[2];
    t->blocks_per_sm = (int32_t)v[3];
    t->motif_b_side_min = (int32_t)v[4];
    t->reverse_ratio = (int32_t)v[5];
    t->bitset_forward_ratio = (int32_t)v[6];
    t->use_graph = 1;
    *ms = v[7];
    return check_tune(t) == PGM_OK;
  }
  return false;
}

pgm_status tune_cache_put(const char* path, const std::string& key, const pgm_tune& t, double ms) {
  auto entries = tune_cache_read(path);
  char body[512];
  snprintf(body, sizeof(body),
           "{\"block_threads\": %d, \"warp_stage_cap\": %d, \"hub_threshold\": %d, \"blocks_per_sm\": %d, "
           "\"motif_b_side_min\": %d, \"reverse_ratio\": %d, \"bitset_forward_ratio\": %d, \"ms\": %.3f}",
           t.block_threads, t.warp_stage_cap, t.hub_threshold, t.blocks_per_sm, t.motif_b_side_min,
           t.reverse_ratio, t.bitset_forward_ratio, ms);
  bool found = false;
  for (auto& e : entries)
    if (e.first == key) {
      e.second = body;
      found = true;
    }
  if (!found) entries.emplace_back(key, body);
  const std::string tmp = std::string(path) + ".tmp";
  FILE* f = fopen(tmp.c_str(), "w");
  if (!f) {
    set_error("autotune cache: cannot write %s", tmp.c_str());
    return PGM_EINVAL;
  }
  fprintf(f, "{\n");
  for (size_t i = 0; i < entries.size(); i++)
    fprintf(f, " \"%s\": %s%s\n", entries[i].first.c_str(), entries[i].second.c_str(),
            i + 1 < entries.size() ? "," : "");
  fprintf(f, "}\n");
  fclose(f);
  if (rename(tmp.c_str(), path) != 0) {
    set_error("autotune cache: cannot replace %s", path);
    return PGM_EINVAL;
  }
  return PGM_OK;
}

}  // namespace
}  // namespace pgm

// ------------------------------------------------------------------- C ABI
extern "C" {

pgm_status pgm_batch_create(int32_t G, const int64_t* vtx_off, const int64_t* rowptr_cat,
                            const int32_t* col_cat, uint32_t flags, void* stream, pgm_batch** out) {
  PGM_NVTX("pgm_batch_create");
  if (!out || G < 0 || !vtx_off || !rowptr_cat) {
    pgm::set_error("pgm_batch_create: bad arguments");
    return PGM_EINVAL;
  }
  if (vtx_off[0] != 0) {
    pgm::set_error("pgm_batch_create: vtx_off[0] must be 0");
    return PGM_EINVAL;
  }
  for (int32_t i = 0; i < G; i++)
    if (vtx_off[i + 1] < vtx_off[i]) {
      pgm::set_error("pgm_batch_create: vtx_off decreases at graph %d", i);
      return PGM_EINVAL;
    }
  const int64_t n = vtx_off[G];
  if (n >= INT32_MAX) {
    pgm::set_error("pgm_batch_create: %lld vertices exceed int32", (long long)n);
    return PGM_EUNSUPPORTED;
  }
  pgm_batch* b = new (std::nothrow) pgm_batch();
  if (!b) return PGM_ENOMEM;
  auto fail = [&](pgm_status st) {
    pgm_batch_destroy(b);
    return st;
  };
  cudaStream_t s = (cudaStream_t)stream;
  if (!s) {
    // the legacy default stream cannot be captured into a CUDA graph
    if (cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      pgm::set_error("pgm_batch_create: stream creation failed");
      return fail(PGM_ECUDA);
    }
    s = b->own_stream;
  }
  pgm::profiler().start(s);
  pgm_status st = pgm::graph_upload(b->g, (int32_t)n, rowptr_cat, col_cat, false, 0,
                                    flags & ~PGM_SANITIZE, s);
  if (st != PGM_OK) return fail(st);
  b->G = G;
  b->g.G = G;
  b->vtx_off.assign(vtx_off, vtx_off + G + 1);
  // vertex -> graph map and the no-crossing-arc check
  int64_t* d_off = nullptr;
  unsigned* d_bad = nullptr;
  if (pgm::dev_malloc(&b->g.gid, (size_t)std::max<int64_t>(n, 1) * sizeof(int32_t)) != cudaSuccess ||
      pgm::dev_malloc(&d_off, ((size_t)G + 1) * sizeof(int64_t)) != cudaSuccess ||
      pgm::dev_malloc(&d_bad, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    if (d_off) pgm::dev_free(d_off);
    if (d_bad) pgm::dev_free(d_bad);
    pgm::set_error("pgm_batch_create: device allocation failed");
    return fail(PGM_ENOMEM);
  }
  unsigned hbad = 0;
  cudaMemcpyAsync(d_off, vtx_off, ((size_t)G + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(d_bad, 0, sizeof(unsigned), s);
  if (n > 0 && G > 0) {
    const int blocks = std::max(1, std::min(pgm::num_sms() * 8, (int)((n + 255) / 256)));
    pgm::gid_kernel<<<blocks, 256, 0, s>>>((int32_t)n, d_off, G, b->g.gid);
    pgm::crossing_kernel<<<blocks, 256, 0, s>>>((int32_t)n, b->g.rp, b->g.col, b->g.gid, d_bad);
  }
  cudaMemcpyAsync(&hbad, d_bad, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  pgm::dev_free(d_off);
  pgm::dev_free(d_bad);
  if (e != cudaSuccess) {
    pgm::set_error("pgm_batch_create: %s", cudaGetErrorString(e));
    return fail(PGM_ECUDA);
  }
  if (hbad) {
    pgm::set_error("pgm_batch_create: an arc leaves its graph");
    return fail(PGM_EINVAL);
  }
  st = pgm::graph_orient(b->g);
  if (st == PGM_OK) st = pgm::graph_prepare_motifs(b->g);
  if (st != PGM_OK) return fail(st);
  st = b->per_graph.reserve((size_t)std::max(G, 1) * 21);
  if (st != PGM_OK) return fail(st);
  if (cudaMallocHost(&b->pinned_pg, (size_t)std::max(G, 1) * 21 * sizeof(unsigned long long)) != cudaSuccess ||
      cudaMallocHost(&b->pinned_ctr, 128 * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    pgm::set_error("pgm_batch_create: pinned host allocation failed");
    return fail(PGM_ENOMEM);
  }
  *out = b;
  return PGM_OK;
}

pgm_status pgm_batch_count_motifs(pgm_batch* b, int32_t k, uint64_t* out, const pgm_tune* t) {
  PGM_NVTX("pgm_batch_count_motifs");
  if (!b || !out) {
    pgm::set_error("pgm_batch_count_motifs: null argument");
    return PGM_EINVAL;
  }
  return pgm::run_batch(b, pgm::kMotif, k, out, t);
}

pgm_status pgm_batch_count_kcliques(pgm_batch* b, int32_t k, uint64_t* out, const pgm_tune* t) {
  PGM_NVTX("pgm_batch_count_kcliques");
  if (!b || !out) {
    pgm::set_error("pgm_batch_count_kcliques: null argument");
    return PGM_EINVAL;
  }
  return pgm::run_batch(b, pgm::kClique, k, out, t);
}

pgm_status pgm_batch_count_motifs_loop(pgm_batch* b, int32_t k, uint64_t* out) {
  PGM_NVTX("pgm_batch_count_motifs_loop");
  if (!b || !out) {
    pgm::set_error("pgm_batch_count_motifs_loop: null argument");
    return PGM_EINVAL;
  }
  if (k < 3 || k > 5) {
    pgm::set_error("pgm_batch_count_motifs_loop: k=%d unsupported", k);
    return PGM_EUNSUPPORTED;
  }
  const int np = k == 3 ? 2 : k == 4 ? 6 : 21;
  // the same graph the batched pass counts on (the relabelled copy keeps
  // every graph's block of IDs), restricted to one graph's range per call
  // (no per-graph attribution; one plain engine call per graph)
  pgm::Graph* gp = &b->g;
  if (pgm::options().motif_order == 0) {
    pgm_status rs = pgm::graph_relabeled(b->g, k == 3 ? pgm::kOrderAscending : pgm::kOrderDescending, &gp);
    if (rs != PGM_OK) return rs;
  }
  pgm::Graph& g = *gp;
  int32_t* gid = g.gid;
  g.gid = nullptr;
  pgm_status st = PGM_OK;
  for (int32_t i = 0; i < b->G && st == PGM_OK; i++) {
    pgm::profiler().start(g.stream);
    uint64_t c[21];
    st = pgm::count_motifs_on(g, b->g.ws, g.stream, k, (int32_t)b->vtx_off[i], (int32_t)b->vtx_off[i + 1], c,
                              nullptr);
    if (st == PGM_OK) memcpy(out + (int64_t)i * np, c, np * sizeof(uint64_t));
  }
  g.gid = gid;
  return st;
}

pgm_status pgm_batch_autotune(pgm_batch* b, int32_t k, pgm_tune* best, double* best_ms) {
  return pgm_batch_autotune_ex(b, k, nullptr, best, best_ms, nullptr, 0, nullptr, nullptr);
}

pgm_status pgm_batch_autotune_ex(pgm_batch* b, int32_t k, const char* cache_path, pgm_tune* best, double* best_ms,
                                 pgm_tune_trial* trials, int32_t cap, int32_t* n_trials, int32_t* from_cache) {
  PGM_NVTX("pgm_batch_autotune_ex");
  if (!b || !best || !best_ms || cap < 0 || (cap > 0 && !trials)) {
    pgm::set_error("pgm_batch_autotune: bad arguments");
    return PGM_EINVAL;
  }
  if (k != 3 && k != 4) {
    pgm::set_error("pgm_batch_autotune: k=%d unsupported", k);
    return PGM_EUNSUPPORTED;
  }
  if (n_trials) *n_trials = 0;
  if (from_cache) *from_cache = 0;
  const std::string key = pgm::tune_key(b, k);
  if (cache_path) {
    pgm_tune t;
    double ms = 0;
    if (pgm::tune_cache_get(cache_path, key, &t, &ms)) {
      *best = t;
      *best_ms = ms;
      if (from_cache) *from_cache = 1;
      return PGM_OK;
    }
  }
  // coordinate descent over the knobs of the motif engine, from the
  // defaults: block size, staging capacity, persistent blocks per SM, and
  // the intersection variant of the last level (B-side threshold); each
  // knob's values are timed with the others at their best so far
  const int np = k == 3 ? 2 : 6;
  std::vector<uint64_t> ref((size_t)std::max(b->G, 1) * np), got(ref.size());
  cudaStream_t s = b->g.stream;
  cudaEvent_t e0, e1;
  PGM_TRY_CUDA(cudaEventCreate(&e0));
  PGM_TRY_CUDA(cudaEventCreate(&e1));
  pgm_tune cur;
  memset(&cur, 0, sizeof(cur));
  cur.block_threads = 256;
  cur.warp_stage_cap = 512;
  cur.motif_b_side_min = 8;
  double bms = 1e30;
  bool have_ref = false;
  int nt = 0;
  std::vector<pgm_tune> tried;
  auto time_one = [&](const pgm_tune& t, double* out_ms) -> pgm_status {
    PGM_TRY(pgm::run_batch(b, pgm::kMotif, k, got.data(), &t));  // warm-up + exactness check
    if (!have_ref) {
      ref = got;
      have_ref = true;
    } else if (got != ref) {
      pgm::set_error("pgm_batch_autotune: counts differ between schedules");
      return PGM_EINVAL;
    }
    double tot = 0;
    for (int rep = 0; rep < 2; rep++) {
      cudaEventRecord(e0, s);
      PGM_TRY(pgm::run_batch(b, pgm::kMotif, k, got.data(), &t));
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      tot += ms;
    }
    *out_ms = tot / 2;
    return PGM_OK;
  };
  static const int kThreads[] = {128, 256, 512};
  static const int kCaps[] = {128, 256, 512, 1024};
  static const int kPerSM[] = {0, 2, 4};
  static const int kBSide[] = {8, 32, 128, 1 << 30};
  pgm_status st = PGM_OK;
  for (int knob = 0; knob < 4 && st == PGM_OK; knob++) {
    const int* vals = knob == 0 ? kThreads : knob == 1 ? kCaps : knob == 2 ? kPerSM : kBSide;
    const int nv = knob == 0 ? 3 : knob == 2 ? 3 : 4;
    pgm_tune base = cur;
    for (int i = 0; i < nv && st == PGM_OK; i++) {
      pgm_tune t = base;
      int* f = knob == 0 ? &t.block_threads : knob == 1 ? &t.warp_stage_cap : knob == 2 ? &t.blocks_per_sm
                                                                                       : &t.motif_b_side_min;
      *f = vals[i];
      if ((t.block_threads / 32) * t.warp_stage_cap > 16384) continue;  // shared memory of the warp kernels
      bool seen = false;
      for (const auto& u : tried) seen = seen || (u.block_threads == t.block_threads &&
                                                  u.warp_stage_cap == t.warp_stage_cap &&
                                                  u.blocks_per_sm == t.blocks_per_sm &&
                                                  u.motif_b_side_min == t.motif_b_side_min);
      if (seen) continue;
      tried.push_back(t);
      double ms = 0;
      st = time_one(t, &ms);
      if (st != PGM_OK) break;
      if (nt < cap) {
        trials[nt].tune = t;
        trials[nt].ms = ms;
      }
      nt++;
      if (ms < bms) {
        bms = ms;
        cur = t;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != PGM_OK) return st;
  cur.use_graph = 1;
  *best = cur;
  *best_ms = bms;
  if (n_trials) *n_trials = std::min(nt, cap);
  if (cache_path) PGM_TRY(pgm::tune_cache_put(cache_path, key, cur, bms));
  return PGM_OK;
}

int32_t pgm_batch_size(const pgm_batch* b) { return b ? b->G : 0; }

void pgm_batch_destroy(pgm_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->g.stream);
  for (auto& c : b->caps) {
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->ws) c->ws->release_all();
  }
  b->caps.clear();
  b->per_graph.release();
  if (b->pinned_pg) cudaFreeHost(b->pinned_pg);
  if (b->pinned_ctr) cudaFreeHost(b->pinned_ctr);
  pgm::graph_free(b->g);
  if (b->own_stream) cudaStreamDestroy(b->own_stream);
  delete b;
}

}  // extern "C"
