// scan.cu -- exclusive prefix sum of per-embedding child counts: the
// allocation step of inspection-execution (Sec. 5.3).  uint32 counts in,
// int64 offsets out, out[len] = total.  Three passes: block partial sums,
// a single-block scan of the partials, and a block-local scan that adds the
// block's carry.  Loads and stores go through shared memory so that every
// global access is coalesced.
#include "common.cuh"

namespace pgm {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096 counts per block

// inclusive block scan of one int64 per thread; *total receives the block total
__device__ __forceinline__ long long block_inclusive_scan(long long v, long long* sh_warp,
                                                          long long* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    long long t = __shfl_up_sync(kFull, v, d);
    if (lane >= d) v += t;
  }
  if (lane == 31) sh_warp[wid] = v;
  __syncthreads();
  if (wid == 0) {
    long long w = lane < nw ? sh_warp[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      long long t = __shfl_up_sync(kFull, w, d);
      if (lane >= d) w += t;
    }
    if (lane < nw) sh_warp[lane] = w;
  }
  __syncthreads();
  long long base = wid > 0 ? sh_warp[wid - 1] : 0;
  *total = sh_warp[nw - 1];
  __syncthreads();
  return v + base;
}

__global__ void __launch_bounds__(kScanThreads) scan_partials_kernel(const uint32_t* __restrict__ cnt,
                                                                     int64_t len,
                                                                     long long* __restrict__ part) {
  __shared__ long long sh_warp[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  long long s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    int64_t j = base + (int64_t)i * kScanThreads + threadIdx.x;
    if (j < len) s += cnt[j];
  }
  long long total;
  block_inclusive_scan(s, sh_warp, &total);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// exclusive scan of the partials in place (one block, sequential tiles)
__global__ void __launch_bounds__(1024) scan_partials_single_kernel(long long* __restrict__ part,
                                                                    int64_t nparts,
                                                                    int64_t* __restrict__ out_total) {
  __shared__ long long sh_warp[32];
  long long carry = 0;
  for (int64_t t0 = 0; t0 < nparts; t0 += blockDim.x) {
    int64_t j = t0 + threadIdx.x;
    long long v = j < nparts ? part[j] : 0;
    long long total;
    long long incl = block_inclusive_scan(v, sh_warp, &total);
    if (j < nparts) part[j] = carry + incl - v;
    carry += total;
  }
  if (threadIdx.x == 0) *out_total = carry;
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const uint32_t* __restrict__ cnt,
                                                                  int64_t len,
                                                                  const long long* __restrict__ part,
                                                                  int64_t* __restrict__ out) {
  __shared__ uint32_t sh_in[kScanTile];
  __shared__ long long sh_warp[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    int idx = i * kScanThreads + threadIdx.x;
    int64_t j = base + idx;
    sh_in[idx] = j < len ? cnt[j] : 0u;
  }
  __syncthreads();
  // each thread owns kScanItems consecutive counts
  uint32_t loc[kScanItems];
  long long s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; i++) {
    loc[i] = sh_in[threadIdx.x * kScanItems + i];
    s += loc[i];
  }
  long long total;
  long long incl = block_inclusive_scan(s, sh_warp, &total);
  long long run = part[blockIdx.x] + incl - s;
  __syncthreads();
  // write back through shared memory, half a tile of int64 at a time
  long long* sh_out = reinterpret_cast<long long*>(sh_in);
#pragma unroll
  for (int half = 0; half < 2; half++) {
    const int lo = half * (kScanTile / 2);
    long long r = run;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
      int idx = threadIdx.x * kScanItems + i;
      if (idx >= lo && idx < lo + kScanTile / 2) sh_out[idx - lo] = r;
      r += loc[i];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < kScanTile / 2; idx += kScanThreads) {
      int64_t j = base + lo + idx;
      if (j < len) out[j] = sh_out[idx];
    }
    __syncthreads();
  }
}

pgm_status exclusive_scan(const uint32_t* cnt, int64_t len, int64_t* out, Workspace& ws,
                          cudaStream_t s) {
  if (len < 0) return PGM_EINVAL;
  if (len == 0) {
    PGM_TRY_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return PGM_OK;
  }
  const int64_t nb = (len + kScanTile - 1) / kScanTile;
  if (nb > INT32_MAX) {
    set_error("scan length %lld too large", (long long)len);
    return PGM_EUNSUPPORTED;
  }
  PGM_TRY(ws.scan_tmp.reserve((size_t)nb));
  long long* part = reinterpret_cast<long long*>(ws.scan_tmp.p);
  scan_partials_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(cnt, len, part);
  PGM_CHECK_LAUNCH();
  scan_partials_single_kernel<<<1, 1024, 0, s>>>(part, nb, out + len);
  PGM_CHECK_LAUNCH();
  scan_apply_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(cnt, len, part, out);
  PGM_CHECK_LAUNCH();
  return PGM_OK;
}

}  // namespace pgm

extern "C" pgm_status pgm_exclusive_scan_dev(const uint32_t* cnt_dev, int64_t len, int64_t* out_dev,
                                             void* stream) {
  if (len < 0 || (len > 0 && !cnt_dev) || !out_dev) {
    pgm::set_error("pgm_exclusive_scan_dev: bad arguments");
    return PGM_EINVAL;
  }
  static thread_local pgm::Workspace ws;
  cudaStream_t s = (cudaStream_t)stream;
  PGM_TRY(pgm::exclusive_scan(cnt_dev, len, out_dev, ws, s));
  PGM_TRY_CUDA(cudaStreamSynchronize(s));
  return PGM_OK;
}
