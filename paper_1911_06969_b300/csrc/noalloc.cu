// noalloc.cu -- triangle counting that allocates no device memory.
//
// For callers that must not call cudaMalloc (for example a plugin inside a
// host application whose allocator owns the whole device memory budget, or
// a latency-critical process that cannot afford the implicit device-wide
// synchronisation of an allocation).  They pass the oriented graph and the
// output slot in memory they already own; the kernels' scratch -- queue
// counters, the accumulator and the list of hub parents handed from the
// warp kernel to the block kernel -- lives in one fixed-size file-scope
// device array instead of library-allocated buffers.
//
// The array is a __device__ variable: in host code its name stands for a
// host-side shadow, not a device address, so the host obtains the device
// address once per device with cudaGetSymbolAddress (with that device
// current) and passes it to the kernels.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "clique_kernels.cuh"

namespace pgm {
namespace {

constexpr int64_t kNoAllocMaxHubs = (int64_t)1 << 20;  // hub-parent slots (8 MiB)
constexpr int kNoAllocSlots = 64;                       // counters (512 B)
constexpr int kNaQueue = 0, kNaErr = 15, kNaAcc = 16, kNaStat = 32;

struct NoAllocScratch {
  unsigned long long ctr[kNoAllocSlots];  // queues, error flag, accumulator, statistics
  int64_t big[kNoAllocMaxHubs];           // hub parents deferred to the block kernel
};

// Shared by every call on a device; holds the last call's contents.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

std::mutex g_na_mu;
NoAllocScratch* g_na_ptr[64] = {nullptr};

// Device address of the scratch array on the current device (resolved on
// the first call per device, with that device current).
pgm_status noalloc_scratch(NoAllocScratch** out) {
  int dev = 0;
  PGM_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    set_error("pgm_count_triangles_noalloc: device ordinal %d out of range", dev);
    return PGM_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      set_error("pgm_count_triangles_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return PGM_ECUDA;
    }
    g_na_ptr[dev] = reinterpret_cast<NoAllocScratch*>(p);
  }
  *out = g_na_ptr[dev];
  return PGM_OK;
}

}  // namespace
}  // namespace pgm

extern "C" pgm_status pgm_count_triangles_noalloc(int32_t n, const int32_t* dag_rowptr_dev,
                                                  const int32_t* dag_col_dev, int64_t m,
                                                  unsigned long long* count_dev, void* stream) {
  using namespace pgm;
  if (n < 0 || m < 0 || !count_dev || (n > 0 && !dag_rowptr_dev) || (m > 0 && !dag_col_dev)) {
    set_error("pgm_count_triangles_noalloc: bad arguments");
    return PGM_EINVAL;
  }
  const pgm_options o = options();
  const int cap = o.warp_stage_cap;
  const int hub = o.hub_threshold > 0 ? std::min(o.hub_threshold, cap) : cap;
  // at most m / (hub + 1) parents have more than `hub` out-neighbours
  const int64_t big_need = m / (hub + 1) + 2;
  if (m >= INT32_MAX || big_need > kNoAllocMaxHubs) {
    set_error("pgm_count_triangles_noalloc: %lld arcs exceed the fixed scratch (at most %lld hub parents "
              "of more than %d out-neighbours)", (long long)m, (long long)kNoAllocMaxHubs, hub);
    return PGM_EUNSUPPORTED;
  }
  NoAllocScratch* sc = nullptr;
  PGM_TRY(noalloc_scratch(&sc));
  cudaStream_t s = (cudaStream_t)stream;
  // the array keeps the previous call's contents: clear the counters
  PGM_TRY_CUDA(cudaMemsetAsync(sc->ctr, 0, sizeof(sc->ctr), s));
  if (n > 0 && m > 0) {
    LevelArgs A;
    memset(&A, 0, sizeof(A));
    A.seg = dag_rowptr_dev;  // level 2: parent u's segment is N+(u)
    A.seg_shift = 0;
    A.vid = dag_col_dev;
    A.p_lo = 0;
    A.p_hi = n;
    A.e_base = 0;
    A.rp = dag_rowptr_dev;
    A.col = dag_col_dev;
    A.acc = sc->ctr + kNaAcc;
    A.stat = sc->ctr + kNaStat;
    A.queue = sc->ctr + kNaQueue;
    A.err = sc->ctr + kNaErr;
    A.carry = sc->ctr + kCarrySlot;
    A.big = sc->big;
    A.big_cap = big_need;
    A.hub = hub;
    A.cap = cap;
    A.block_cap = 12288;
    A.rev_ratio = o.reverse_ratio;
    const int threads = o.block_threads;
    const size_t wsmem = clique_warp_smem(threads, cap);
    const size_t bsmem = (size_t)A.block_cap * sizeof(int32_t) + (size_t)(512 / 32) * 32 * 4;
    const void* wfn = (const void*)clique_warp_kernel<kSum, int32_t>;
    const void* bfn = (const void*)clique_block_kernel<kSum, int32_t>;
    PGM_TRY(smem_attr(wfn, 160 * 1024));
    PGM_TRY(smem_attr(bfn, 160 * 1024));
    int wgrid = grid_for(wfn, threads, wsmem);
    A.grab = (int)std::max<int64_t>(1, std::min<int64_t>(kGrab, (int64_t)n / ((int64_t)wgrid * (threads / 32))));
    const int64_t warps_needed = ((int64_t)n + A.grab - 1) / A.grab;
    wgrid = (int)std::max<int64_t>(1, std::min<int64_t>(wgrid, (warps_needed + threads / 32 - 1) / (threads / 32)));
    const int bgrid = (int)std::max<int64_t>(1, std::min<int64_t>(grid_for(bfn, 512, bsmem), big_need));
    clique_warp_kernel<kSum, int32_t><<<wgrid, threads, wsmem, s>>>(A);
    PGM_CHECK_LAUNCH();
    clique_block_kernel<kSum, int32_t><<<bgrid, 512, bsmem, s>>>(A);
    PGM_CHECK_LAUNCH();
  }
  PGM_TRY_CUDA(cudaMemcpyAsync(count_dev, sc->ctr + kNaAcc, sizeof(unsigned long long),
                               cudaMemcpyDeviceToDevice, s));
  // the carry and error slots in one readback (slots kCarrySlot .. kNaErr)
  static_assert(kCarrySlot < kNaErr, "carry slot below the error slot");
  unsigned long long h[kNaErr - kCarrySlot + 1];
  PGM_TRY_CUDA(cudaMemcpyAsync(h, sc->ctr + kCarrySlot, sizeof(h), cudaMemcpyDeviceToHost, s));
  PGM_TRY_CUDA(cudaStreamSynchronize(s));
  const unsigned long long err = h[kNaErr - kCarrySlot], carry = h[0];
  if (err) {
    set_error("pgm_count_triangles_noalloc: hub list overflow");
    return PGM_ENOMEM;
  }
  if (carry) {
    set_error("pgm_count_triangles_noalloc: the count exceeds 2^64 - 1");
    return PGM_EOVERFLOW;
  }
  return PGM_OK;
}
