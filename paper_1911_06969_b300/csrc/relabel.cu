// relabel.cu -- a copy of the graph with vertex IDs assigned by degree.
//
// The motif counts are invariant under any relabelling of the vertices
// (an isomorphism maps every connected k-set to one of the same pattern),
// but the work of the level-wise extension is not: the canonical order of
// an embedding starts at its smallest ID (Sec. 3.2 canonical test), and the
// lists the extension scans are the neighbours above that vertex.  Counting
// on a copy whose IDs follow the degrees moves the hub vertices to the end
// (ascending order) or to the front (descending order) of the ID range.
// Each graph of a batch is relabelled within its own block of IDs, so the
// block structure (and the per-graph attribution) is unchanged.
#include <algorithm>
#include <cstring>
#include <memory>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_segmented_sort.cuh>

#include "common.cuh"

namespace pgm {
namespace {

// sort key of vertex v: graph block (batches) major, then degree (or its
// complement for descending order); ties keep the input order (stable sort)
__global__ void relabel_keys_kernel(int32_t n, const int32_t* __restrict__ rp, const int32_t* __restrict__ gid,
                                    bool descending, unsigned long long* __restrict__ key,
                                    int32_t* __restrict__ val) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t d = (uint32_t)(rp[v + 1] - rp[v]);
    const uint32_t g = gid ? (uint32_t)gid[v] : 0u;
    key[v] = ((unsigned long long)g << 32) | (descending ? 0xffffffffu - d : d);
    val[v] = (int32_t)v;
  }
}

// new ID of every old vertex, degrees in the new order, new graph IDs
__global__ void relabel_map_kernel(int32_t n, const int32_t* __restrict__ order, const int32_t* __restrict__ rp,
                                   const int32_t* __restrict__ gid, int32_t* __restrict__ newid,
                                   uint32_t* __restrict__ deg_new, int32_t* __restrict__ gid_new) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = order[i];
    newid[u] = (int32_t)i;
    deg_new[i] = (uint32_t)(rp[u + 1] - rp[u]);
    if (gid) gid_new[i] = gid[u];
  }
}

// one warp per new vertex: its list, relabelled (unsorted)
__global__ void relabel_lists_kernel(int32_t n, const int32_t* __restrict__ order, const int32_t* __restrict__ rp,
                                     const int32_t* __restrict__ col, const int32_t* __restrict__ newid,
                                     const int32_t* __restrict__ rp_new, int32_t* __restrict__ col_new) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp; i < n; i += nwarps) {
    const int32_t u = order[i];
    const int32_t a0 = rp[u], d = rp[u + 1] - a0, b0 = rp_new[i];
    for (int t = lane; t < d; t += 32) col_new[b0 + t] = newid[col[a0 + t]];
  }
}

pgm_status build_relabeled(Graph& g, bool descending, Graph& r) {
  cudaStream_t s = g.stream;
  const int32_t n = g.n;
  const int64_t narcs = g.narcs;
  r.stream = s;
  r.n = n;
  r.narcs = narcs;
  r.G = g.G;
  r.dmax = g.dmax;
  DevArr<unsigned long long> key, key2;
  DevArr<int32_t> val, order, newid;
  DevArr<uint32_t> deg_new;
  DevArr<unsigned char> tmp;
  const size_t nn = (size_t)std::max<int32_t>(n, 1);
  PGM_TRY(key.reserve(nn));
  PGM_TRY(key2.reserve(nn));
  PGM_TRY(val.reserve(nn));
  PGM_TRY(order.reserve(nn));
  PGM_TRY(newid.reserve(nn));
  PGM_TRY(deg_new.reserve(nn + 1));
  PGM_TRY_CUDA(pgm::dev_malloc(&r.rp, ((size_t)n + 1) * sizeof(int32_t)));
  PGM_TRY_CUDA(pgm::dev_malloc(&r.col, (size_t)std::max<int64_t>(narcs, 1) * sizeof(int32_t)));
  if (g.gid) PGM_TRY_CUDA(pgm::dev_malloc(&r.gid, nn * sizeof(int32_t)));
  int32_t* col_unsorted = nullptr;
  struct Cleanup {
    DevArr<unsigned long long>& a;
    DevArr<unsigned long long>& b;
    DevArr<int32_t>& c;
    DevArr<int32_t>& d;
    DevArr<int32_t>& e;
    DevArr<uint32_t>& f;
    DevArr<unsigned char>& t;
    int32_t*& cu;
    ~Cleanup() {
      a.release();
      b.release();
      c.release();
      d.release();
      e.release();
      f.release();
      t.release();
      if (cu) pgm::dev_free(cu);
    }
  } cleanup{key, key2, val, order, newid, deg_new, tmp, col_unsorted};
  const int blocks = std::max(1, std::min(num_sms() * 8, (int)((n + 255) / 256)));
  if (n > 0) {
    relabel_keys_kernel<<<blocks, 256, 0, s>>>(n, g.rp, g.gid, descending, key.p, val.p);
    PGM_CHECK_LAUNCH();
    size_t tb = 0;
    PGM_TRY_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, tb, key.p, key2.p, val.p, order.p, (int64_t)n, 0, 64, s));
    PGM_TRY(tmp.reserve(std::max<size_t>(tb, 1)));
    PGM_TRY_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, tb, key.p, key2.p, val.p, order.p, (int64_t)n, 0, 64, s));
    relabel_map_kernel<<<blocks, 256, 0, s>>>(n, order.p, g.rp, g.gid, newid.p, deg_new.p, r.gid);
    PGM_CHECK_LAUNCH();
  }
  // row pointers of the copy: exclusive scan of the degrees in the new order
  PGM_TRY(r.ws.off[0].reserve((size_t)n + 1));
  PGM_TRY(exclusive_scan(deg_new.p, n, r.ws.off[0].p, r.ws, s));
  narrow_rowptr(r.ws.off[0].p, r.rp, (int64_t)n + 1, s);
  if (n > 0 && narcs > 0) {
    PGM_TRY_CUDA(pgm::dev_malloc(&col_unsorted, (size_t)narcs * sizeof(int32_t)));
    const int wblocks = std::max(1, std::min(num_sms() * 16, (int)(((int64_t)n * 32 + 255) / 256)));
    relabel_lists_kernel<<<wblocks, 256, 0, s>>>(n, order.p, g.rp, g.col, newid.p, r.rp, col_unsorted);
    PGM_CHECK_LAUNCH();
    // sort every list
    size_t tb = 0;
    PGM_TRY_CUDA(cub::DeviceSegmentedSort::SortKeys(nullptr, tb, col_unsorted, r.col, (int64_t)narcs, (int64_t)n,
                                                    r.rp, r.rp + 1, s));
    PGM_TRY(tmp.reserve(std::max<size_t>(tb, 1)));
    PGM_TRY_CUDA(cub::DeviceSegmentedSort::SortKeys(tmp.p, tb, col_unsorted, r.col, (int64_t)narcs, (int64_t)n,
                                                    r.rp, r.rp + 1, s));
  }
  PGM_TRY_CUDA(cudaStreamSynchronize(s));
  return PGM_OK;
}

}  // namespace

pgm_status graph_relabeled(Graph& g, int order, Graph** out) {
  if (order < 0 || order > 1) return PGM_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(g.mu);
  if (!g.relabeled[order]) {
    std::unique_ptr<Graph> r(new (std::nothrow) Graph());
    if (!r) {
      set_error("relabel: out of host memory");
      return PGM_ENOMEM;
    }
    const pgm_status st = build_relabeled(g, order == kOrderDescending, *r);
    if (st != PGM_OK) {
      graph_free(*r);
      return st;
    }
    g.relabeled[order] = std::move(r);
  }
  *out = g.relabeled[order].get();
  return PGM_OK;
}

}  // namespace pgm
