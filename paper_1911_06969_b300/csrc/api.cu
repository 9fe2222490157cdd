// api.cu -- process-wide state of libpgm: error messages, options, device
// queries, the launch profiler, record/replay plans and the small C-ABI
// entry points.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "common.cuh"

namespace pgm {

static thread_local std::string t_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_err = buf;
}

const char* get_error() { return t_err.c_str(); }

static std::atomic<uint64_t> g_launches{0};
void note_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static pgm_options g_opts = {256, 512, 0, 0, (int64_t)1 << 31, 0, 2, 0, 4, 1024, 0, 0, 8, 0};

pgm_options& options() { return g_opts; }

unsigned long long count_seed() {
  const int x = g_opts.count_headroom_log2;
  return (x > 0 && x < 64) ? 0ull - (1ull << x) : 0ull;
}

pgm_status seed_counts(unsigned long long* dev, int n, cudaStream_t s) {
  const unsigned long long seed = count_seed();
  if (!seed || current_plan()) return PGM_OK;
  std::vector<unsigned long long> h((size_t)n, seed);
  PGM_TRY_CUDA(cudaMemcpyAsync(dev, h.data(), (size_t)n * sizeof(unsigned long long), cudaMemcpyHostToDevice, s));
  PGM_TRY_CUDA(cudaStreamSynchronize(s));
  return PGM_OK;
}

int device_id() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}

int num_sms() {
  static int cached[64] = {0};
  static std::mutex mu;
  int d = device_id();
  if (d < 0 || d >= 64) return 148;
  std::lock_guard<std::mutex> lk(mu);
  if (!cached[d]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 148;
    }
    cached[d] = v;
  }
  return cached[d];
}

int64_t l2_bytes() {
  static int64_t cached[64] = {0};
  static std::mutex mu;
  int d = device_id();
  if (d < 0 || d >= 64) return 0;
  std::lock_guard<std::mutex> lk(mu);
  if (!cached[d]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, d) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 0;
    }
    cached[d] = v > 0 ? v : -1;
  }
  return cached[d] > 0 ? cached[d] : 0;
}

// occupancy is cached per (kernel, block size, shared memory) so that no
// runtime query happens while a stream is being captured
int grid_for(const void* fn, int threads, size_t smem) {
  int per_sm = options().blocks_per_sm;
  if (per_sm <= 0) {
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, size_t>, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_tuple(fn, threads, smem);
    auto it = cache.find(key);
    if (it != cache.end()) {
      per_sm = it->second;
    } else {
      int occ = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess ||
          occ <= 0) {
        cudaGetLastError();
        occ = 1;
      }
      cache[key] = occ;
      per_sm = occ;
    }
  }
  return per_sm * num_sms();
}

pgm_status smem_attr(const void* fn, int bytes) {
  static std::mutex mu;
  static std::map<const void*, int> done;
  std::lock_guard<std::mutex> lk(mu);
  auto it = done.find(fn);
  if (it != done.end() && it->second >= bytes) return PGM_OK;
  PGM_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done[fn] = bytes;
  return PGM_OK;
}

// ---------------------------------------------------------------- profiler
static thread_local Profiler t_prof;
static thread_local pgm_profile t_last;
static thread_local std::vector<cudaEvent_t> t_event_pool;

Profiler& profiler() { return t_prof; }
pgm_profile& last_profile() { return t_last; }

static cudaEvent_t take_event() {
  if (!t_event_pool.empty()) {
    cudaEvent_t e = t_event_pool.back();
    t_event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

void Profiler::start(cudaStream_t s) {
  for (auto& r : recs) {
    if (r.a) t_event_pool.push_back(r.a);
    if (r.b) t_event_pool.push_back(r.b);
  }
  recs.clear();
  stream = s;
  on = options().profile != 0;
  memset(&t_last, 0, sizeof(t_last));
}

int Profiler::begin(const char* name, int level) {
  if (!on) return -1;
  Rec r;
  r.name = name;
  r.level = level;
  r.a = take_event();
  r.b = take_event();
  r.entries = 0;
  r.alg_bytes = 0;
  if (!r.a || !r.b) return -1;
  cudaEventRecord(r.a, stream);
  recs.push_back(r);
  return (int)recs.size() - 1;
}

void Profiler::end(int id, double entries, double alg_bytes) {
  if (id < 0 || id >= (int)recs.size()) return;
  cudaEventRecord(recs[id].b, stream);
  recs[id].entries = entries;
  recs[id].alg_bytes = alg_bytes;
}

pgm_status Profiler::finish(pgm_profile* out) {
  if (!on) return PGM_OK;
  PGM_TRY_CUDA(cudaStreamSynchronize(stream));
  std::map<std::pair<std::string, int>, int> slot;
  for (auto& r : recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
      cudaGetLastError();
      ms = 0.f;
    }
    auto key = std::make_pair(r.name, r.level);
    auto it = slot.find(key);
    int i;
    if (it == slot.end()) {
      if (out->nphases >= PGM_PROFILE_MAX) continue;
      i = out->nphases++;
      slot[key] = i;
      pgm_phase& p = out->phase[i];
      memset(&p, 0, sizeof(p));
      strncpy(p.name, r.name.c_str(), sizeof(p.name) - 1);
      p.level = r.level;
    } else {
      i = it->second;
    }
    pgm_phase& p = out->phase[i];
    p.launches += 1;
    p.ms += ms;
    p.entries += r.entries;
    p.alg_bytes += r.alg_bytes;
  }
  return PGM_OK;
}

// ------------------------------------------------------------------ plans
static thread_local Plan* t_plan = nullptr;
Plan*& current_plan() { return t_plan; }

pgm_status read_counters(const unsigned long long* dev, unsigned long long* host, size_t n,
                         cudaStream_t s, bool* deferred) {
  Plan* pl = current_plan();
  if (pl && pl->replay && pl->pinned_ctr) {
    PGM_TRY_CUDA(cudaMemcpyAsync(pl->pinned_ctr, dev, n * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, s));
    *deferred = true;
    return PGM_OK;
  }
  // through a page-locked staging buffer of this thread: a copy to pageable
  // memory takes the driver's own staging path, which costs several
  // microseconds per call on the small counts where launch latency is the
  // whole run time
  struct Staging {
    unsigned long long* p = nullptr;
    size_t n = 0;
    ~Staging() {
      if (p) cudaFreeHost(p);
    }
  };
  static thread_local Staging st;
  if (st.n < n) {
    if (st.p) cudaFreeHost(st.p);
    st.p = nullptr;
    st.n = 0;
    const size_t want = std::max<size_t>(n, 256);
    if (cudaHostAlloc(&st.p, want * sizeof(unsigned long long), cudaHostAllocPortable) == cudaSuccess) {
      st.n = want;
    } else {
      cudaGetLastError();
      st.p = nullptr;
    }
  }
  unsigned long long* dst = st.p ? st.p : host;
  PGM_TRY_CUDA(cudaMemcpyAsync(dst, dev, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  PGM_TRY_CUDA(cudaStreamSynchronize(s));
  if (dst != host) memcpy(host, dst, n * sizeof(unsigned long long));
  *deferred = false;
  return PGM_OK;
}

// ----------------------------------------------------------- device memory
namespace {
struct DevPool {
  cudaMemPool_t pool = nullptr;
  cudaStream_t s = nullptr;  // stream of the pool's allocations and frees
};
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
DevPool g_pools[kMaxDevices];

DevPool* pool_here(cudaError_t& e) {
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nullptr;
  if (dev < 0 || dev >= kMaxDevices) {
    e = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_pool_mu);
  DevPool& P = g_pools[dev];
  if (!P.pool) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    e = cudaMemPoolCreate(&P.pool, &props);
    if (e != cudaSuccess) {
      P.pool = nullptr;
      return nullptr;
    }
    uint64_t keep = kPoolKeepBytes;
    e = cudaMemPoolSetAttribute(P.pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&P.s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(P.pool);
      P.pool = nullptr;
      P.s = nullptr;
      return nullptr;
    }
  }
  e = cudaSuccess;
  return &P;
}
}  // namespace

cudaError_t dev_malloc(void** p, size_t bytes) {
  *p = nullptr;
  cudaError_t e;
  DevPool* P = pool_here(e);
  if (!P) return e;
  e = cudaMallocFromPoolAsync(p, bytes, P->pool, P->s);
  if (e == cudaErrorMemoryAllocation) {  // give the cached blocks back and try once more
    cudaGetLastError();
    cudaStreamSynchronize(P->s);
    cudaMemPoolTrimTo(P->pool, 0);
    e = cudaMallocFromPoolAsync(p, bytes, P->pool, P->s);
  }
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  e = cudaStreamSynchronize(P->s);  // complete: usable from every stream
  if (e != cudaSuccess) {
    cudaFreeAsync(*p, P->s);
    *p = nullptr;
  }
  return e;
}

cudaError_t dev_free(void* p) {
  if (!p) return cudaSuccess;
  cudaError_t e;
  DevPool* P = pool_here(e);
  if (!P) return e;
  e = cudaDeviceSynchronize();  // every user of the block has finished, as with cudaFree
  const cudaError_t f = cudaFreeAsync(p, P->s);
  return e != cudaSuccess ? e : f;
}

void Workspace::release_all() {
  for (int i = 0; i < kMaxLevels; i++) {
    cnt[i].release();
    off[i].release();
    vid[i].release();
  }
  big.release();
  ctr.release();
  scan_tmp.release();
  scratch.release();
  tri.release();
  dom.release();
}

}  // namespace pgm

#ifdef PGM_DEBUG
namespace pgm {
namespace {
struct DebugReg {
  const char* file;
  cudaError_t (*read)(DebugWord*);
  cudaError_t (*reset)();
};
std::vector<DebugReg>& debug_regs() {
  static std::vector<DebugReg> v;
  return v;
}
}  // namespace
int register_debug_word(const char* file, cudaError_t (*read)(DebugWord*), cudaError_t (*reset)()) {
  debug_regs().push_back({file, read, reset});
  return (int)debug_regs().size();
}
}  // namespace pgm
#endif

// ------------------------------------------------------------------- C ABI
extern "C" {

uint64_t pgm_debug_errors(int32_t reset) {
#ifdef PGM_DEBUG
  uint64_t total = 0;
  bool first = true;
  for (const auto& r : pgm::debug_regs()) {
    pgm::DebugWord w = {0, 0, 0};
    if (r.read(&w) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (w.count && first) {
      pgm::set_error("out-of-range index %lld at %s:%llu (%llu violations in that file)", (long long)w.index,
                     r.file, w.line, w.count);
      first = false;
    }
    total += w.count;
    if (reset && r.reset() != cudaSuccess) cudaGetLastError();
  }
  return total;
#else
  (void)reset;
  return 0;
#endif
}

const char* pgm_last_error(void) { return pgm::get_error(); }

const char* pgm_version(void) { return "libpgm 0.2 (sm_103a)"; }

uint64_t pgm_kernel_launches(void) { return pgm::g_launches.load(std::memory_order_relaxed); }

pgm_status pgm_set_options(const pgm_options* o) {
  if (!o) {
    pgm::set_error("pgm_set_options: null options");
    return PGM_EINVAL;
  }
  const pgm_options v = *o;
  pgm_options next = pgm::options();  // validated as a whole, then applied
  if (v.block_threads) {
    if (v.block_threads < 64 || v.block_threads > 512 || v.block_threads % 32) {
      pgm::set_error("block_threads must be a multiple of 32 in [64, 512]");
      return PGM_EINVAL;
    }
    next.block_threads = v.block_threads;
  }
  if (v.warp_stage_cap) {
    if (v.warp_stage_cap < 32 || v.warp_stage_cap > 4096) {
      pgm::set_error("warp_stage_cap must be in [32, 4096]");
      return PGM_EINVAL;
    }
    next.warp_stage_cap = v.warp_stage_cap;
  }
  // shared memory of the warp kernels: (threads / 32) * cap ints per staged list
  if ((next.block_threads / 32) * next.warp_stage_cap > 16384) {
    pgm::set_error("block_threads / 32 * warp_stage_cap must be <= 16384 (shared memory)");
    return PGM_EINVAL;
  }
  if (v.hub_threshold) {
    if (v.hub_threshold < 2) {
      pgm::set_error("hub_threshold must be >= 2");
      return PGM_EINVAL;
    }
    next.hub_threshold = v.hub_threshold;
  }
  if (v.blocks_per_sm) next.blocks_per_sm = v.blocks_per_sm < 0 ? 0 : v.blocks_per_sm;
  if (v.level_budget) {
    if (v.level_budget < 1024) {
      pgm::set_error("level_budget must be >= 1024 entries");
      return PGM_EINVAL;
    }
    next.level_budget = v.level_budget;
  }
  if (v.reverse_ratio) {
    if (v.reverse_ratio < 1) {
      pgm::set_error("reverse_ratio must be >= 1");
      return PGM_EINVAL;
    }
    next.reverse_ratio = v.reverse_ratio;
  }
  if (v.clique_engine < 0 || v.clique_engine > 2) {
    pgm::set_error("clique_engine must be 0 (auto), 1 (level lists) or 2 (bitset levels)");
    return PGM_EINVAL;
  }
  next.clique_engine = v.clique_engine;
  if (v.bitset_forward_ratio) {
    if (v.bitset_forward_ratio < 1) {
      pgm::set_error("bitset_forward_ratio must be >= 1");
      return PGM_EINVAL;
    }
    next.bitset_forward_ratio = v.bitset_forward_ratio;
  }
  if (v.bitset_smem_degree) {
    const int b = v.bitset_smem_degree;
    if (b != 64 && b != 256 && b != 512 && b != 1024) {
      pgm::set_error("bitset_smem_degree must be 64, 256, 512 or 1024");
      return PGM_EINVAL;
    }
    next.bitset_smem_degree = b;
  }
  if (v.motif_order < 0 || v.motif_order > 1) {
    pgm::set_error("motif_order must be 0 (degree-ordered copy) or 1 (input IDs)");
    return PGM_EINVAL;
  }
  next.motif_order = v.motif_order;
  if (v.count_headroom_log2 < 0 || v.count_headroom_log2 > 63) {
    pgm::set_error("count_headroom_log2 must be 0 (off) or in [1, 63]");
    return PGM_EINVAL;
  }
  next.count_headroom_log2 = v.count_headroom_log2;
  if (v.motif_b_side_min) {
    if (v.motif_b_side_min < 1) {
      pgm::set_error("motif_b_side_min must be >= 1");
      return PGM_EINVAL;
    }
    next.motif_b_side_min = v.motif_b_side_min;
  }
  if (v.fsm_domain_order < 0 || v.fsm_domain_order > 2) {
    pgm::set_error("fsm_domain_order must be 0 (auto), 1 (by first edge) or 2 (by centre)");
    return PGM_EINVAL;
  }
  next.fsm_domain_order = v.fsm_domain_order;
  next.profile = v.profile ? 1 : 0;
  pgm::options() = next;
  return PGM_OK;
}

pgm_status pgm_get_options(pgm_options* o) {
  if (!o) return PGM_EINVAL;
  *o = pgm::options();
  if (!o->hub_threshold) o->hub_threshold = o->warp_stage_cap;
  return PGM_OK;
}

pgm_status pgm_last_profile(pgm_profile* out) {
  if (!out) return PGM_EINVAL;
  *out = pgm::last_profile();
  return PGM_OK;
}

}  // extern "C"
