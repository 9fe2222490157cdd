// graph.cu -- CSR ingest, validation, degree orientation and statistics.
//
// Input format (Sec. 6.1): simple undirected graph, CSR with neighbour
// lists sorted by ascending ID, symmetric, without self-loops or duplicate
// edges.  On the device the graph is int32 row pointers + int32 columns.
//
// Orientation (Sec. 4.1, "Directed Acyclic Graph"): arc u->v is kept iff
// (d(u), u) < (d(v), v) -- edges point to the higher degree, ties to the
// larger ID.  Each vertex's out-list keeps the ID order of its undirected
// list, so DAG lists stay sorted.
#include <algorithm>
#include <cstring>
#include <new>

#include "common.cuh"

namespace pgm {

enum : unsigned {
  kBadRange = 1u,    // neighbour ID outside [0, n)
  kUnsorted = 2u,    // list not strictly ascending (unsorted or duplicate)
  kSelfLoop = 4u,
  kAsymmetric = 8u,
};

// one warp per vertex: checks IDs, order, loops and symmetry
__global__ void validate_kernel(int32_t n, const int32_t* __restrict__ rp,
                                const int32_t* __restrict__ col, unsigned* __restrict__ flags) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned bad = 0;
  for (int64_t u = warp; u < n; u += nwarps) {
    const int32_t a0 = rp[u], a1 = rp[u + 1];
    for (int32_t a = a0 + lane; a < a1; a += 32) {
      int32_t v = col[a];
      if (v < 0 || v >= n) {
        bad |= kBadRange;
        continue;
      }
      if (v == u) bad |= kSelfLoop;
      if (a > a0 && col[a - 1] >= v) bad |= kUnsorted;
      // symmetry: u must appear in N(v)
      if (!contains_dev(col + rp[v], rp[v + 1] - rp[v], (int32_t)u)) bad |= kAsymmetric;
    }
  }
  bad = __reduce_or_sync(kFull, bad);
  if (lane == 0 && bad) atomicOr(flags, bad);
}

__device__ __forceinline__ bool keep_arc(int32_t u, int32_t du, int32_t v, int32_t dv) {
  return du < dv || (du == dv && u < v);
}

// Row pointers: checks rp[0] = 0, rp[n] = narcs and that they never
// decrease, narrows them to int32 and records the largest degree.
// info[0] = max degree, info[1] = first vertex whose pointer decreases
// (initialised to all ones), info[2] = 1 if rp[0] or rp[n] is wrong.
__global__ void rowptr_kernel(int32_t n, const int64_t* __restrict__ rp64, int64_t narcs,
                              int32_t* __restrict__ rp32, unsigned long long* __restrict__ info) {
  long long dmax = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = rp64[v];
    rp32[v] = (int32_t)a;
    if ((v == 0 && a != 0) || (v == n && a != narcs)) atomicOr(info + 2, 1ull);
    if (v < n) {
      const int64_t b = rp64[v + 1];
      if (b < a)
        atomicMin(info + 1, (unsigned long long)v);
      else
        dmax = max(dmax, (long long)(b - a));
    }
  }
  dmax = __reduce_max_sync(kFull, (unsigned)min(dmax, (long long)INT32_MAX));
  if ((threadIdx.x & 31) == 0 && dmax) atomicMax(info, (unsigned long long)dmax);
}

// Orientation, pass 1 (one warp per vertex): out-degree per vertex, one
// keep flag per arc and the largest out-degree (atomicMax into *dmax).
// Orientation, arc-parallel (per-vertex warps left the R-MAT hubs, tens of
// thousands of arcs each, as a long tail).  Arcs are taken in words of 32;
// a warp owns kOrientWords consecutive words, finds the source of its first
// arc by binary search in rp and carries it along; each lane walks from the
// word's first source to its own arc's source (the arcs of a vertex are
// contiguous).  orient_mask_kernel writes the keep flags of each word as a
// bit mask and its population count; an exclusive scan of the counts gives
// every kept arc its DAG position (word offset + rank within the word).
constexpr int kOrientWords = 64;

__global__ void __launch_bounds__(256) orient_mask_kernel(int32_t n, int64_t narcs, const int32_t* __restrict__ rp,
                                                          const int32_t* __restrict__ col, uint32_t* __restrict__ mask,
                                                          uint32_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nwords = (narcs + 31) >> 5;
  for (int64_t w0 = warp * kOrientWords; w0 < nwords; w0 += nwarps * kOrientWords) {
    // source of arc 32 w0: the largest u with rp[u] <= 32 w0 (rp[0] = 0)
    int32_t u = 0;
    if (lane == 0) {
      int32_t lo = 0, hi = n - 1;
      const int64_t a0 = w0 << 5;
      while (lo < hi) {
        const int32_t mid = lo + ((hi - lo + 1) >> 1);
        if (rp[mid] <= a0) lo = mid; else hi = mid - 1;
      }
      u = lo;
    }
    u = __shfl_sync(kFull, u, 0);
    const int64_t w1 = min(w0 + kOrientWords, nwords);
    for (int64_t w = w0; w < w1; w++) {
      const int64_t a = (w << 5) + lane;
      bool k = false;
      int32_t su = u;
      if (a < narcs) {
        while (rp[su + 1] <= a) su++;  // su < n: rp[n] = narcs > a
        const int32_t v = col[a];
        k = keep_arc(su, rp[su + 1] - rp[su], v, rp[v + 1] - rp[v]);
      }
      const unsigned bal = __ballot_sync(kFull, k);
      if (lane == 0) {
        mask[w] = bal;
        cnt[w] = __popc(bal);
      }
      u = __shfl_sync(kFull, su, 31);  // the last lane's source starts the next word
    }
  }
}

// DAG position of arc a: kept arcs before it
__device__ __forceinline__ int64_t orient_pos(const uint32_t* mask, const int64_t* off, int64_t a) {
  const int64_t w = a >> 5;
  const int b = (int)(a & 31);
  return off[w] + (b ? __popc(mask[w] & ((1u << b) - 1u)) : 0);
}

// The kept arcs into dag_col (thread per arc), and dag_rp plus the largest
// out-degree (thread per vertex, u = n gives the end pointer).
__global__ void __launch_bounds__(256) orient_write_kernel(int64_t narcs, const int32_t* __restrict__ col,
                                                           const uint32_t* __restrict__ mask,
                                                           const int64_t* __restrict__ off,
                                                           int32_t* __restrict__ dag_col) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < narcs; a += (int64_t)gridDim.x * blockDim.x) {
    const int64_t w = a >> 5;
    const int b = (int)(a & 31);
    const uint32_t m = mask[w];
    if ((m >> b) & 1u) dag_col[off[w] + __popc(m & ((1u << b) - 1u))] = col[a];
  }
}

__global__ void __launch_bounds__(256) orient_rows_kernel(int32_t n, const int32_t* __restrict__ rp,
                                                          const uint32_t* __restrict__ mask,
                                                          const int64_t* __restrict__ off,
                                                          int32_t* __restrict__ dag_rp,
                                                          unsigned long long* __restrict__ dmax) {
  unsigned cmax = 0;
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u <= n; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p0 = orient_pos(mask, off, rp[u]);
    dag_rp[u] = (int32_t)p0;
    if (u < n) cmax = max(cmax, (unsigned)(orient_pos(mask, off, rp[u + 1]) - p0));
  }
  cmax = __reduce_max_sync(kFull, cmax);
  if ((threadIdx.x & 31) == 0 && cmax) atomicMax(dmax, (unsigned long long)cmax);
}

__global__ void narrow_kernel(const int64_t* __restrict__ in, int32_t* __restrict__ out, int64_t len) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int32_t)in[i];
}

// up[v] = index of the first arc of v whose neighbour is greater than v
__global__ void upper_kernel(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                             int32_t* __restrict__ up) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a0 = rp[v], a1 = rp[v + 1];
    up[v] = a0 + lower_bound_dev(col + a0, a1 - a0, (int32_t)v + 1);
  }
}

// src[a] = v for every arc a of v
__global__ void src_kernel(int32_t n, const int32_t* __restrict__ rp, int32_t* __restrict__ src) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t v = warp; v < n; v += nwarps)
    for (int32_t a = rp[v] + lane; a < rp[v + 1]; a += 32) src[a] = (int32_t)v;
}

// rev[a] = index of arc v -> u for every arc a = u -> v (binary search in N(v))
__global__ void rev_kernel(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                           int32_t* __restrict__ rev) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u = warp; u < n; u += nwarps)
    for (int32_t a = rp[u] + lane; a < rp[u + 1]; a += 32) {
      const int32_t v = col[a];
      rev[a] = rp[v] + lower_bound_dev(col + rp[v], rp[v + 1] - rp[v], (int32_t)u);
    }
}

// one block per hub: set the bits of its neighbours in its bitmap row
__global__ void hub_bits_kernel(const int32_t* __restrict__ hubs, int32_t nh, const int32_t* __restrict__ rp,
                                const int32_t* __restrict__ col, uint32_t* __restrict__ bits, int64_t words) {
  for (int32_t h = blockIdx.x; h < nh; h += gridDim.x) {
    const int32_t v = hubs[h];
    uint32_t* row = bits + (int64_t)h * words;
    for (int32_t a = rp[v] + threadIdx.x; a < rp[v + 1]; a += blockDim.x) {
      const int32_t w = col[a];
      atomicOr(row + (w >> 5), 1u << (w & 31));
    }
  }
}

static int warp_grid(int64_t items, int threads) {
  int64_t blocks = (items * 32 + threads - 1) / threads;
  int64_t cap = (int64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  return (int)std::max<int64_t>(blocks, 1);
}

// host-side repair: symmetrise, drop loops and duplicates, sort
static void sanitize_host(int32_t n, const int64_t* rowptr, const int32_t* col,
                          std::vector<int64_t>& rp_out, std::vector<int32_t>& col_out) {
  std::vector<uint64_t> keys;
  keys.reserve((size_t)rowptr[n] * 2);
  for (int32_t u = 0; u < n; u++)
    for (int64_t a = rowptr[u]; a < rowptr[u + 1]; a++) {
      int32_t v = col[a];
      if (v < 0 || v >= n || v == u) continue;
      keys.push_back(((uint64_t)(uint32_t)u << 32) | (uint32_t)v);
      keys.push_back(((uint64_t)(uint32_t)v << 32) | (uint32_t)u);
    }
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  rp_out.assign((size_t)n + 1, 0);
  col_out.resize(keys.size());
  for (size_t i = 0; i < keys.size(); i++) {
    rp_out[(keys[i] >> 32) + 1]++;
    col_out[i] = (int32_t)(keys[i] & 0xffffffffu);
  }
  for (int32_t v = 0; v < n; v++) rp_out[v + 1] += rp_out[v];
}

void narrow_rowptr(const int64_t* in, int32_t* out, int64_t len, cudaStream_t s) {
  narrow_kernel<<<std::max(1, std::min(num_sms() * 8, (int)((len + 255) / 256))), 256, 0, s>>>(in, out, len);
  note_launches(1);
}

void graph_free(Graph& g) {
  for (auto& r : g.relabeled)
    if (r) {
      graph_free(*r);
      r.reset();
    }
  if (g.rp) pgm::dev_free(g.rp);
  if (g.col) pgm::dev_free(g.col);
  if (g.dag_rp) pgm::dev_free(g.dag_rp);
  if (g.dag_col) pgm::dev_free(g.dag_col);
  if (g.gid) pgm::dev_free(g.gid);
  if (g.up) pgm::dev_free(g.up);
  if (g.src) pgm::dev_free(g.src);
  if (g.rev) pgm::dev_free(g.rev);
  if (g.hub_idx) pgm::dev_free(g.hub_idx);
  if (g.labels) pgm::dev_free(g.labels);
  if (g.label_rank) pgm::dev_free(g.label_rank);
  if (g.wedge_centres) pgm::dev_free(g.wedge_centres);
  if (g.wedge_prefix) pgm::dev_free(g.wedge_prefix);
  if (g.hub_bits) pgm::dev_free(g.hub_bits);
  g.rp = g.col = g.dag_rp = g.dag_col = g.gid = g.up = g.src = g.hub_idx = g.rev = nullptr;
  g.hub_bits = nullptr;
  g.labels = nullptr;
  g.label_rank = nullptr;
  g.wedge_centres = nullptr;
  g.wedge_prefix = nullptr;
  g.n_wedge_centres = g.n_wedges = 0;
  g.h_label_count.clear();
  g.nhubs = 0;
  g.ws.release_all();
  g.oriented = false;
}

pgm_status graph_upload(Graph& g, int32_t n, const int64_t* rowptr, const int32_t* col,
                        bool rowptr_on_device, int64_t narcs, uint32_t flags, cudaStream_t s) {
  if (n < 0 || !rowptr || (flags & ~(PGM_VALIDATE | PGM_SANITIZE))) {
    set_error("graph: bad arguments (n=%d)", n);
    return PGM_EINVAL;
  }
  g.stream = s;
  g.n = n;
  std::vector<int64_t> rp_s;
  std::vector<int32_t> col_s;
  if (!rowptr_on_device) {
    if (rowptr[0] != 0) {
      set_error("graph: rowptr[0] must be 0");
      return PGM_EINVAL;
    }
    if (flags & PGM_SANITIZE) {
      for (int32_t v = 0; v < n; v++)
        if (rowptr[v + 1] < rowptr[v]) {
          set_error("graph: rowptr decreases at vertex %d", v);
          return PGM_EINVAL;
        }
      if (rowptr[n] > 0 && !col) {
        set_error("graph: null col");
        return PGM_EINVAL;
      }
      sanitize_host(n, rowptr, col, rp_s, col_s);
      rowptr = rp_s.data();
      col = col_s.data();
    }
    narcs = rowptr[n];
    if (narcs > 0 && !col) {
      set_error("graph: null col");
      return PGM_EINVAL;
    }
  } else if (flags & PGM_SANITIZE) {
    set_error("graph: PGM_SANITIZE needs host arrays");
    return PGM_EINVAL;
  }
  if (narcs < 0 || narcs >= INT32_MAX) {
    set_error("graph: %lld arcs outside the int32 device index range", (long long)narcs);
    return narcs < 0 ? PGM_EINVAL : PGM_EUNSUPPORTED;
  }
  g.narcs = narcs;
  PGM_TRY_CUDA(pgm::dev_malloc(&g.rp, ((size_t)n + 1) * sizeof(int32_t)));
  PGM_TRY_CUDA(pgm::dev_malloc(&g.col, (size_t)std::max<int64_t>(narcs, 1) * sizeof(int32_t)));
  const int64_t* rp64 = rowptr;
  if (!rowptr_on_device) {
    PGM_TRY(g.ws.off[0].reserve((size_t)n + 1));
    PGM_TRY_CUDA(cudaMemcpyAsync(g.ws.off[0].p, rowptr, ((size_t)n + 1) * sizeof(int64_t),
                                 cudaMemcpyHostToDevice, s));
    rp64 = g.ws.off[0].p;
  }
  if (narcs > 0)
    PGM_TRY_CUDA(cudaMemcpyAsync(g.col, col, (size_t)narcs * sizeof(int32_t),
                                 rowptr_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                 s));
  // row pointers checked and narrowed on the device; max degree by reduction
  PGM_TRY(g.ws.ctr.reserve(16));
  unsigned long long* info = g.ws.ctr.p;
  PGM_TRY_CUDA(cudaMemsetAsync(info, 0, 3 * sizeof(unsigned long long), s));
  PGM_TRY_CUDA(cudaMemsetAsync(info + 1, 0xff, sizeof(unsigned long long), s));
  rowptr_kernel<<<std::max(1, std::min(num_sms() * 8, (int)((n + 256) / 256))), 256, 0, s>>>(n, rp64, narcs,
                                                                                          g.rp, info);
  PGM_CHECK_LAUNCH();
  unsigned long long h[3];
  PGM_TRY_CUDA(cudaMemcpyAsync(h, info, sizeof(h), cudaMemcpyDeviceToHost, s));
  PGM_TRY_CUDA(cudaStreamSynchronize(s));
  if (h[1] != ~0ull) {
    set_error("graph: rowptr decreases at vertex %llu", h[1]);
    return PGM_EINVAL;
  }
  if (h[2]) {
    set_error("graph: rowptr must start at 0 and end at the number of arcs (%lld)", (long long)narcs);
    return PGM_EINVAL;
  }
  g.dmax = (int64_t)h[0];
  g.h_rp.clear();  // host copy made on first use (graph_host_rp)
  if ((flags & PGM_VALIDATE) && n > 0) {
    unsigned* fl = reinterpret_cast<unsigned*>(info);
    PGM_TRY_CUDA(cudaMemsetAsync(fl, 0, sizeof(unsigned), s));
    validate_kernel<<<warp_grid(n, 256), 256, 0, s>>>(n, g.rp, g.col, fl);
    PGM_CHECK_LAUNCH();
    unsigned hf = 0;
    PGM_TRY_CUDA(cudaMemcpyAsync(&hf, fl, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    PGM_TRY_CUDA(cudaStreamSynchronize(s));
    if (hf) {
      set_error("graph: invalid CSR:%s%s%s%s", (hf & kBadRange) ? " neighbour-out-of-range" : "",
                (hf & kUnsorted) ? " unsorted-or-duplicate" : "", (hf & kSelfLoop) ? " self-loop" : "",
                (hf & kAsymmetric) ? " asymmetric" : "");
      return PGM_EINVAL;
    }
  }
  return PGM_OK;
}

// Host copies of the row pointers, made on first use (they are not needed
// by the clique path).  Not to be called while a stream capture is open.
static pgm_status host_copy(const int32_t* dev, int32_t n, cudaStream_t s, std::vector<int64_t>& out) {
  std::vector<int32_t> tmp((size_t)n + 1);
  PGM_TRY_CUDA(cudaMemcpyAsync(tmp.data(), dev, ((size_t)n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  PGM_TRY_CUDA(cudaStreamSynchronize(s));
  out.assign(tmp.begin(), tmp.end());
  return PGM_OK;
}

pgm_status graph_host_rp(Graph& g) {
  std::lock_guard<std::recursive_mutex> lk(g.mu);
  if (g.h_rp.size() == (size_t)g.n + 1) return PGM_OK;
  return host_copy(g.rp, g.n, g.stream, g.h_rp);
}

pgm_status graph_host_dag_rp(Graph& g) {
  std::lock_guard<std::recursive_mutex> lk(g.mu);
  PGM_TRY(graph_orient(g));
  if (g.h_dag_rp.size() == (size_t)g.n + 1) return PGM_OK;
  return host_copy(g.dag_rp, g.n, g.stream, g.h_dag_rp);
}

pgm_status graph_dag_arcs(Graph& g, int32_t v_lo, int32_t v_hi, int64_t* arcs) {
  PGM_TRY(graph_orient(g));
  if (v_lo == 0 && v_hi == g.n) {
    *arcs = g.narcs / 2;
    return PGM_OK;
  }
  PGM_TRY(graph_host_dag_rp(g));
  *arcs = g.h_dag_rp[v_hi] - g.h_dag_rp[v_lo];
  return PGM_OK;
}

pgm_status graph_orient(Graph& g) {
  std::lock_guard<std::recursive_mutex> lk(g.mu);
  if (g.oriented) return PGM_OK;
  cudaStream_t s = g.stream;
  const int32_t n = g.n;
  const int64_t m = g.narcs / 2;
  if (g.narcs % 2) {
    set_error("orient: odd number of arcs (input not symmetric)");
    return PGM_EINVAL;
  }
  if (!g.dag_rp) PGM_TRY_CUDA(pgm::dev_malloc(&g.dag_rp, ((size_t)n + 1) * sizeof(int32_t)));
  if (!g.dag_col) PGM_TRY_CUDA(pgm::dev_malloc(&g.dag_col, (size_t)std::max<int64_t>(m, 1) * sizeof(int32_t)));
  const int64_t nwords = (g.narcs + 31) / 32;
  PGM_TRY(g.ws.cnt[0].reserve((size_t)std::max<int64_t>(nwords, 1)));
  PGM_TRY(g.ws.off[0].reserve((size_t)nwords + 1));
  PGM_TRY(g.ws.ctr.reserve(16));
  DevArr<uint32_t> mask;  // keep flags, one word per 32 arcs, freed on return
  PGM_TRY(mask.reserve((size_t)std::max<int64_t>(nwords, 1)));
  struct Free {
    DevArr<uint32_t>& k;
    ~Free() { k.release(); }
  } free_mask{mask};
  unsigned long long* dmax_dev = g.ws.ctr.p + 3;
  PGM_TRY_CUDA(cudaMemsetAsync(dmax_dev, 0, sizeof(unsigned long long), s));
  Profiler& prof = profiler();
  int id = prof.begin("orient", 1);
  const int grid = std::max(1, num_sms() * 8);
  if (g.narcs > 0) {
    const int64_t ranges = (nwords + kOrientWords - 1) / kOrientWords;
    orient_mask_kernel<<<(int)std::min<int64_t>(grid, (ranges + 7) / 8), 256, 0, s>>>(n, g.narcs, g.rp, g.col,
                                                                                      mask.p, g.ws.cnt[0].p);
    PGM_CHECK_LAUNCH();
  }
  PGM_TRY(exclusive_scan(g.ws.cnt[0].p, nwords, g.ws.off[0].p, g.ws, s));
  int64_t kept = 0;
  PGM_TRY_CUDA(cudaMemcpyAsync(&kept, g.ws.off[0].p + nwords, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  PGM_TRY_CUDA(cudaStreamSynchronize(s));
  if (kept != m) {
    // not symmetric: the kept-arc count differs from m; refuse before writing
    set_error("orient: kept %lld arcs, expected %lld (input not symmetric?)", (long long)kept, (long long)m);
    return PGM_EINVAL;
  }
  if (g.narcs > 0) {
    orient_write_kernel<<<(int)std::min<int64_t>(grid, (g.narcs + 255) / 256), 256, 0, s>>>(
        g.narcs, g.col, mask.p, g.ws.off[0].p, g.dag_col);
    PGM_CHECK_LAUNCH();
  }
  orient_rows_kernel<<<(int)std::min<int64_t>(grid, ((int64_t)n + 256) / 256), 256, 0, s>>>(
      n, g.rp, mask.p, g.ws.off[0].p, g.dag_rp, dmax_dev);
  PGM_CHECK_LAUNCH();
  prof.end(id, (double)n, 8.0 * (double)g.narcs);
  unsigned long long dd = 0;
  PGM_TRY_CUDA(cudaMemcpyAsync(&dd, dmax_dev, sizeof(dd), cudaMemcpyDeviceToHost, s));
  PGM_TRY_CUDA(cudaStreamSynchronize(s));
  g.dag_dmax = (int64_t)dd;
  g.h_dag_rp.clear();  // host copy made on first use (graph_host_dag_rp)
  g.oriented = true;
  return PGM_OK;
}

// Motif helpers, built once per graph: up[] (first arc to a larger ID),
// src[] (source vertex of each arc) and adjacency bitmaps of the vertices
// of degree >= kHubDegree (highest degrees first, at most kHubBytes), used
// for O(1) membership tests against hub adjacency lists.
constexpr int64_t kHubDegree = 512;  // longer lists than the default staging capacity
constexpr int64_t kHubBytes = (int64_t)512 << 20;

pgm_status graph_prepare_motifs(Graph& g) {
  std::lock_guard<std::recursive_mutex> lk(g.mu);
  if (g.up) return PGM_OK;
  PGM_TRY(graph_host_rp(g));
  cudaStream_t s = g.stream;
  const int32_t n = g.n;
  PGM_TRY_CUDA(pgm::dev_malloc(&g.up, ((size_t)n + 1) * sizeof(int32_t)));
  PGM_TRY_CUDA(pgm::dev_malloc(&g.src, (size_t)std::max<int64_t>(g.narcs, 1) * sizeof(int32_t)));
  PGM_TRY_CUDA(pgm::dev_malloc(&g.rev, (size_t)std::max<int64_t>(g.narcs, 1) * sizeof(int32_t)));
  PGM_TRY_CUDA(pgm::dev_malloc(&g.hub_idx, ((size_t)n + 1) * sizeof(int32_t)));
  PGM_TRY_CUDA(cudaMemsetAsync(g.hub_idx, 0xff, ((size_t)n + 1) * sizeof(int32_t), s));
  if (n > 0) {
    const int blocks = std::max(1, std::min(num_sms() * 8, (n + 255) / 256));
    upper_kernel<<<blocks, 256, 0, s>>>(n, g.rp, g.col, g.up);
    PGM_CHECK_LAUNCH();
    src_kernel<<<warp_grid(n, 256), 256, 0, s>>>(n, g.rp, g.src);
    PGM_CHECK_LAUNCH();
    rev_kernel<<<warp_grid(n, 256), 256, 0, s>>>(n, g.rp, g.col, g.rev);
    PGM_CHECK_LAUNCH();
  }
  // hubs: highest degrees first
  std::vector<std::pair<int64_t, int32_t>> cand;
  for (int32_t v = 0; v < n; v++) {
    const int64_t d = g.h_rp[v + 1] - g.h_rp[v];
    if (d >= kHubDegree) cand.push_back({-d, v});
  }
  std::sort(cand.begin(), cand.end());
  g.hub_words = ((int64_t)n + 31) / 32;
  int64_t maxh = g.hub_words > 0 ? kHubBytes / (g.hub_words * 4) : 0;
  const int32_t nh = (int32_t)std::min<int64_t>((int64_t)cand.size(), maxh);
  if (nh > 0) {
    std::vector<int32_t> hubs(nh), idx(nh);
    for (int32_t h = 0; h < nh; h++) hubs[h] = cand[h].second;
    PGM_TRY_CUDA(pgm::dev_malloc(&g.hub_bits, (size_t)nh * g.hub_words * sizeof(uint32_t)));
    PGM_TRY_CUDA(cudaMemsetAsync(g.hub_bits, 0, (size_t)nh * g.hub_words * sizeof(uint32_t), s));
    int32_t* d_hubs = nullptr;
    PGM_TRY_CUDA(pgm::dev_malloc(&d_hubs, (size_t)nh * sizeof(int32_t)));
    PGM_TRY_CUDA(cudaMemcpyAsync(d_hubs, hubs.data(), (size_t)nh * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    hub_bits_kernel<<<std::min(nh, num_sms() * 4), 256, 0, s>>>(d_hubs, nh, g.rp, g.col, g.hub_bits,
                                                                g.hub_words);
    PGM_CHECK_LAUNCH();
    for (int32_t h = 0; h < nh; h++) idx[h] = h;
    // scatter the row numbers into hub_idx (one small copy per hub)
    for (int32_t h = 0; h < nh; h++)
      PGM_TRY_CUDA(cudaMemcpyAsync(g.hub_idx + hubs[h], &idx[h], sizeof(int32_t), cudaMemcpyHostToDevice, s));
    PGM_TRY_CUDA(cudaStreamSynchronize(s));
    pgm::dev_free(d_hubs);
  }
  g.nhubs = nh;
  PGM_TRY_CUDA(cudaStreamSynchronize(s));
  return PGM_OK;
}

}  // namespace pgm

// ------------------------------------------------------------------- C ABI
extern "C" {

pgm_status pgm_graph_create_csr(int32_t n, const int64_t* rowptr, const int32_t* col, uint32_t flags,
                                void* stream, pgm_graph** out) {
  PGM_NVTX("pgm_graph_create_csr");
  if (!out) {
    pgm::set_error("pgm_graph_create_csr: null out");
    return PGM_EINVAL;
  }
  pgm_graph* h = new (std::nothrow) pgm_graph();
  if (!h) return PGM_ENOMEM;
  pgm::profiler().start((cudaStream_t)stream);
  pgm_status st = pgm::graph_upload(h->g, n, rowptr, col, false, 0, flags, (cudaStream_t)stream);
  if (st != PGM_OK) {
    pgm::graph_free(h->g);
    delete h;
    return st;
  }
  *out = h;
  return PGM_OK;
}

pgm_status pgm_graph_create_csr_dev(int32_t n, const int64_t* rowptr_dev, const int32_t* col_dev,
                                    int64_t narcs, uint32_t flags, void* stream, pgm_graph** out) {
  PGM_NVTX("pgm_graph_create_csr_dev");
  if (!out || (narcs > 0 && !col_dev)) {
    pgm::set_error("pgm_graph_create_csr_dev: bad arguments");
    return PGM_EINVAL;
  }
  pgm_graph* h = new (std::nothrow) pgm_graph();
  if (!h) return PGM_ENOMEM;
  pgm::profiler().start((cudaStream_t)stream);
  pgm_status st = pgm::graph_upload(h->g, n, rowptr_dev, col_dev, true, narcs, flags,
                                    (cudaStream_t)stream);
  if (st != PGM_OK) {
    pgm::graph_free(h->g);
    delete h;
    return st;
  }
  *out = h;
  return PGM_OK;
}

pgm_status pgm_graph_orient_by_degree(pgm_graph* g) {
  PGM_NVTX("pgm_graph_orient_by_degree");
  if (!g) {
    pgm::set_error("pgm_graph_orient_by_degree: null graph");
    return PGM_EINVAL;
  }
  pgm::profiler().start(g->g.stream);
  return pgm::graph_orient(g->g);
}

pgm_status pgm_graph_stats_get(const pgm_graph* gh, pgm_graph_stats* out) {
  if (!gh || !out) {
    pgm::set_error("pgm_graph_stats_get: null argument");
    return PGM_EINVAL;
  }
  pgm::Graph& g = const_cast<pgm_graph*>(gh)->g;
  PGM_TRY(pgm::graph_host_rp(g));
  unsigned __int128 s2 = 0, s3 = 0;
  for (int32_t v = 0; v < g.n; v++) {
    unsigned __int128 d = (unsigned __int128)(g.h_rp[v + 1] - g.h_rp[v]);
    if (d >= 2) s2 += d * (d - 1) / 2;
    if (d >= 3) s3 += d * (d - 1) * (d - 2) / 6;
  }
  pgm_graph_stats r;
  memset(&r, 0, sizeof(r));
  r.n = g.n;
  r.m = g.narcs / 2;
  r.dmax = g.dmax;
  r.dag_dmax = g.oriented ? g.dag_dmax : 0;
  r.sum_c2[0] = (uint64_t)s2;
  r.sum_c2[1] = (uint64_t)(s2 >> 64);
  r.sum_c3[0] = (uint64_t)s3;
  r.sum_c3[1] = (uint64_t)(s3 >> 64);
  *out = r;
  return PGM_OK;
}

void pgm_graph_destroy(pgm_graph* g) {
  if (!g) return;
  cudaStreamSynchronize(g->g.stream);
  pgm::graph_free(g->g);
  delete g;
}

}  // extern "C"
