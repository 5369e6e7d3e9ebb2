// cc_noalloc.cu -- cc_disagreements_static: the disagreement count of a
// labelling with no memory allocation at all.
//
// Some callers cannot allocate device memory at the moment they need this
// number: code that runs inside a pre-sized memory pool or arena, callers
// that run under a strict "no allocation after start-up" rule (serving
// loops, real-time paths), or callers that must not touch the allocator
// while other work is in flight.  This entry point works only on buffers the
// caller already owns plus one fixed scratch area that is part of the
// library's image: a file-scope __device__ array reserved when the library is
// loaded on a GPU and kept until the process exits.
//
// The scratch is shared by every call on that device, so calls whose work
// overlaps on the GPU race with each other and must be serialised by the
// caller (one stream, or events).  The first call on a device looks up the
// device address of the scratch with cudaGetSymbolAddress; make that first
// call before any stream capture begins.
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

// One warp per row: entries (u, w) of the CSR with label[u] == label[w].
__global__ void k_static_intra(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                               const int32_t* __restrict__ labels, unsigned long long* acc) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long cnt = 0;
  for (int64_t u = gw; u < n; u += nw) {
    const int32_t lu = labels[u];
    for (int64_t e = off[u] + lane; e < off[u + 1]; e += 32) cnt += labels[col[e]] == lu ? 1 : 0;
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
    void* ps = nullptr;
    void* pa = nullptr;
    if (cudaGetSymbolAddress(&ps, g_static_size) != cudaSuccess) return CC_ERR_CUDA;
    if (cudaGetSymbolAddress(&pa, g_static_acc) != cudaSuccess) return CC_ERR_CUDA;
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
