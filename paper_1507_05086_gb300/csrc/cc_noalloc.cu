// cc_noalloc.cu -- cc_disagreements_static: the disagreement count of a
// labelling with no memory allocation at all.
//
// Some callers cannot allocate device memory at the moment they need this
// number: code that runs inside a pre-sized memory pool or arena, callers
// that run under a strict "no allocation after start-up" rule (serving
// loops, real-time paths), or callers that must not touch the allocator
// while other work is in flight.  This entry point works only on buffers the
// caller already owns plus one fixed scratch area that is part of the
// library's image: a file-scope __device__ array that, once mapped on a GPU,
// stays there until the process exits.
//
// With CUDA's lazy module loading (the default) the array is mapped when this
// file's module is first used on a device, which is the first call of this
// entry point there (its cudaGetSymbolAddress lookup).  That first call may
// therefore make the driver allocate device memory, and it can fail with
// CC_ERR_OOM on a full GPU: make one call at start-up on each device, before
// any no-allocation phase or stream capture begins.  Later calls allocate
// nothing.
//
// The scratch is shared by every call on that device, so calls whose work
// overlaps on the GPU race with each other and must be serialised by the
// caller (one stream, or events).
#include <cstdint>
#include <mutex>

#include "../../include/cc.h"
#include "cc_device.cuh"

namespace {

constexpr int64_t kStaticMaxN = CC_STATIC_MAX_N;
constexpr int kMaxDevices = 64;

// Scratch: per-cluster sizes and the three accumulators (intra-cluster CSR
// entries, sum of C(s, 2), bad-label flag).  Cleared by every call.
__device__ __align__(256) int32_t g_static_size[kStaticMaxN];
__device__ __align__(256) unsigned long long g_static_acc[4];

struct StaticScratch {
  int32_t* size = nullptr;
  unsigned long long* acc = nullptr;
};

std::mutex g_mu;
StaticScratch g_dev[kMaxDevices];

__global__ void k_static_sizes(int64_t n, const int32_t* __restrict__ labels, int32_t* __restrict__ size,
                               unsigned long long* acc) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = labels[v];
    if (c < 0 || c >= n) { atomicExch(acc + 2, 1ull); continue; }
    atomicAdd(size + c, 1);
  }
}

// Entries (u, w) of the CSR with label[u] == label[w].  One warp per row;
// a row longer than kStaticLongRow (a hub of a power-law graph) is queued in
// shared memory and read by the whole block once the block's warps are done
// with their short rows, so that one hub does not hold a single warp for the
// whole kernel (a full queue sends the row back to its warp).
constexpr int kStaticLongRow = 2048;
constexpr int kStaticLongCap = 64;

__global__ void k_static_intra(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                               const int32_t* __restrict__ labels, unsigned long long* acc) {
  __shared__ int32_t longq[kStaticLongCap];
  __shared__ int nlong;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x == 0) nlong = 0;
  __syncthreads();
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long cnt = 0;
  for (int64_t u = gw; u < n; u += nw) {
    const int64_t e0 = off[u], e1 = off[u + 1];
    if (e1 - e0 > kStaticLongRow) {
      int slot = 0;
      if (lane == 0) slot = atomicAdd(&nlong, 1);
      slot = __shfl_sync(ccg::FULL, slot, 0);
      if (slot < kStaticLongCap) {
        if (lane == 0) longq[slot] = (int32_t)u;
        continue;
      }
    }
    const int32_t lu = labels[u];
    for (int64_t e = e0 + lane; e < e1; e += 32) cnt += labels[col[e]] == lu ? 1 : 0;
  }
  __syncthreads();
  const int nq = nlong < kStaticLongCap ? nlong : kStaticLongCap;
  for (int q = 0; q < nq; ++q) {
    const int32_t u = longq[q];
    const int32_t lu = labels[u];
    const int64_t e1 = off[u + 1];
    for (int64_t e = off[u] + threadIdx.x; e < e1; e += blockDim.x) cnt += labels[col[e]] == lu ? 1 : 0;
  }
  cnt = ccg::warp_sum(cnt);
  if (lane == 0 && cnt) atomicAdd(acc, cnt);
}

__global__ void k_static_pairs(int64_t n, const int32_t* __restrict__ size, unsigned long long* acc) {
  unsigned long long p = 0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long s = (unsigned long long)size[c];
    p += s * (s - 1) / 2;
  }
  p = ccg::warp_sum(p);
  if ((threadIdx.x & 31) == 0 && p) atomicAdd(acc + 1, p);
}

// D = m - intra_dir + sum C(s, 2) with m = off[n] / 2; -1 when a label was
// out of range.
__global__ void k_static_finish(const int64_t* __restrict__ off, int64_t n, const unsigned long long* acc,
                                int64_t* out) {
  if (acc[2]) { *out = -1; return; }
  const int64_t nnz = n > 0 ? off[n] : 0;
  *out = nnz / 2 - (int64_t)acc[0] + (int64_t)acc[1];
}

int scratch_for_device(int dev, StaticScratch* out) {
  if (dev < 0 || dev >= kMaxDevices) return CC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev[dev].size) {
    // Under lazy module loading (the CUDA default) this lookup is what loads
    // the module, and with it maps the scratch array on this device: a lack
    // of memory shows up here, and is reported as such.
    void* ps = nullptr;
    void* pa = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ps, g_static_size);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&pa, g_static_acc);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? CC_ERR_OOM : CC_ERR_CUDA;
    }
    g_dev[dev].size = static_cast<int32_t*>(ps);
    g_dev[dev].acc = static_cast<unsigned long long*>(pa);
  }
  *out = g_dev[dev];
  return CC_OK;
}

}  // namespace

extern "C" int cc_disagreements_static(int64_t n, const int64_t* row_offsets, const int32_t* col_idx,
                                       const int32_t* labels, int64_t* out, void* cuda_stream) {
  if (n < 0 || n > kStaticMaxN || !out) return CC_ERR_INVALID_ARG;
  if (n > 0 && (!row_offsets || !col_idx || !labels)) return CC_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CC_ERR_CUDA;
  StaticScratch sc;
  const int rc = scratch_for_device(dev, &sc);
  if (rc != CC_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (cudaMemsetAsync(sc.acc, 0, 4 * sizeof(unsigned long long), s) != cudaSuccess) return CC_ERR_CUDA;
  if (n == 0) {
    k_static_finish<<<1, 1, 0, s>>>(row_offsets, 0, sc.acc, out);
    return cudaGetLastError() == cudaSuccess ? CC_OK : CC_ERR_CUDA;
  }
  if (cudaMemsetAsync(sc.size, 0, sizeof(int32_t) * (size_t)n, s) != cudaSuccess) return CC_ERR_CUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = sms > 0 ? sms * 4 : 128;
  k_static_sizes<<<grid, 256, 0, s>>>(n, labels, sc.size, sc.acc);
  k_static_intra<<<grid, 256, 0, s>>>(n, row_offsets, col_idx, labels, sc.acc);
  k_static_pairs<<<grid, 256, 0, s>>>(n, sc.size, sc.acc);
  // the edge count comes from the offsets on the device, so read it there
  k_static_finish<<<1, 1, 0, s>>>(row_offsets, n, sc.acc, out);
  return cudaGetLastError() == cudaSuccess ? CC_OK : CC_ERR_CUDA;
}
