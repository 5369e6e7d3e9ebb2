// cc_api.cu -- the C ABI (include/cc.h): argument checks, device memory,
// launches and result transfer.  All computation happens in the kernels of
// cc_perm.cu, cc_rounds.cu, cc_async.cu and cc_objective.cu.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/cc.h"
#include "cc_async.h"
#include "cc_graph_impl.h"
#include "cc_internal.h"
#include "cc_nvtx.h"

using namespace ccg;

// ---- the library's device memory pools ---------------------------------------
namespace {
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxPoolDevices] = {};
}  // namespace

namespace ccg {

// One pool per device, created on first use, that keeps freed memory
// reserved (release threshold: unlimited) so that repeated graph creation and
// destruction does not map and unmap device memory every time.
cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxPoolDevices) return cudaErrorInvalidDevice;
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[dev]) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      cudaMemPool_t created;
      if ((e = cudaMemPoolCreate(&created, &props)) != cudaSuccess) return e;
      uint64_t keep = UINT64_MAX;
      if ((e = cudaMemPoolSetAttribute(created, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
        cudaMemPoolDestroy(created);
        return e;
      }
      g_pool[dev] = created;
    }
    pool = g_pool[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, stream);
}

}  // namespace ccg

extern "C" int cc_release_memory(void) {
  std::lock_guard<std::mutex> lock(g_pool_mu);
  int rc = CC_OK;
  for (int d = 0; d < kMaxPoolDevices; ++d)
    if (g_pool[d] && cudaMemPoolTrimTo(g_pool[d], 0) != cudaSuccess) rc = CC_ERR_CUDA;
  return rc;
}

namespace {
// batched size classes (defaults): up to batch_small_n vertices one block
// runs a job, up to batch_team_n a team of batch_team_blocks blocks, beyond
// that the whole grid
constexpr int64_t kBatchSmallN = 1 << 16;
constexpr int64_t kBatchTeamN = 1 << 21;
constexpr int kBatchTeamBlocks = 8;

cc_tuning public_default_tuning() {
  const Tuning d = default_tuning();
  cc_tuning t{};
  t.walk_batches = d.walk_batches;
  t.prefetch_ahead = d.prefetch_ahead;
  t.inline_heavy = d.inline_heavy;
  t.inline_decide = d.inline_decide;
  t.inline_rebuild = d.inline_rebuild;
  t.heavy_shift = d.heavy_shift;
  t.batch_small_n = kBatchSmallN;
  t.batch_team_n = kBatchTeamN;
  t.batch_team_blocks = kBatchTeamBlocks;
  t.warp_resolve_row = d.warp_resolve_row;
  return t;
}

bool tuning_valid(const cc_tuning& t) {
  return t.walk_batches >= 1 && t.walk_batches <= 8 && t.prefetch_ahead >= 0 && t.prefetch_ahead <= 8 &&
         t.inline_heavy >= 0 && t.inline_heavy <= 65536 && t.inline_decide >= 0 && t.inline_decide <= 65536 &&
         t.inline_rebuild >= 0 && t.inline_rebuild <= 65536 && t.heavy_shift >= 1 && t.heavy_shift <= 4 &&
         t.batch_small_n >= 1 && t.batch_small_n <= (1 << 20) && t.batch_team_n >= t.batch_small_n &&
         t.batch_team_n <= (1 << 24) && t.batch_team_blocks >= 2 && t.batch_team_blocks <= 16 &&
         t.warp_resolve_row >= 0 && t.warp_resolve_row <= (1 << 24);
}

Tuning device_tuning(const cc_tuning& t) {
  return Tuning{t.walk_batches, t.prefetch_ahead, t.inline_heavy, t.inline_decide, t.inline_rebuild, t.heavy_shift,
                t.warp_resolve_row};
}

std::mutex g_tune_mu;
bool g_batch_tuning_set = false;
cc_tuning g_batch_tuning;

cc_tuning batch_tuning() {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  return g_batch_tuning_set ? g_batch_tuning : public_default_tuning();
}
}  // namespace


namespace {

int from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return CC_OK;
  if (e == cudaErrorMemoryAllocation) return CC_ERR_OOM;
  return CC_ERR_CUDA;
}

#define CC_TRY(expr)                          \
  do {                                        \
    cudaError_t _e = (expr);                  \
    if (_e != cudaSuccess) return from_cuda(_e); \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
cudaError_t dalloc(T** p, size_t bytes, cudaStream_t s) {
  void* q = nullptr;
  cudaError_t e = pool_malloc(&q, bytes > 0 ? bytes : 1, s);
  *p = static_cast<T*>(q);
  return e;
}

template <class T>
void dfree(T*& p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
  p = nullptr;
}

int ensure_cluster_ws(cc_graph* g) {
  if (!g->order) CC_TRY(dalloc(&g->order, 4 * (size_t)g->n, g->stream));
  const size_t pb = perm_workspace_bytes(g->n);
  if (g->perm_ws_bytes < pb) {
    dfree(g->perm_ws, g->stream);
    CC_TRY(dalloc(&g->perm_ws, pb, g->stream));
    g->perm_ws_bytes = pb;
  }
  if (!g->grid) g->grid = rounds_grid_size(g->device);
  const size_t rb = rounds_workspace_bytes(g->n, g->max_deg, g->grid);
  if (g->round_ws_bytes < rb) {
    dfree(g->round_ws, g->stream);
    CC_TRY(dalloc(&g->round_ws, rb, g->stream));
    g->round_ws_bytes = rb;
  }
  if (!g->perm_err) CC_TRY(dalloc(&g->perm_err, sizeof(int), g->stream));
  if (!g->ctl_host) CC_TRY(cudaMallocHost(&g->ctl_host, sizeof(Ctl)));
  return CC_OK;
}

int ensure_labels_tmp(cc_graph* g) {
  if (!g->labels_tmp) CC_TRY(dalloc(&g->labels_tmp, 4 * (size_t)g->n, g->stream));
  return CC_OK;
}

int ensure_objective_ws(cc_graph* g) {
  if (!g->obj_ws) CC_TRY(dalloc(&g->obj_ws, objective_workspace_bytes(g->n), g->stream));
  if (!g->obj_out) CC_TRY(dalloc(&g->obj_out, 4 * sizeof(unsigned long long), g->stream));
  if (!g->obj_host) CC_TRY(cudaMallocHost(&g->obj_host, 4 * sizeof(unsigned long long)));
  return CC_OK;
}

int status_of_device_err(int e) {
  if (e == CC_OK) return CC_OK;
  if (e == CC_ERR_TIMEOUT) return CC_ERR_TIMEOUT;
  return CC_ERR_INTERNAL;
}

int eps_ppm_of(double eps, int64_t* out) {
  if (!(eps > 0.0) || !(eps <= 1.0)) return CC_ERR_INVALID_ARG;
  const long long ppm = std::llround(eps * 1e6);
  if (ppm < 1 || ppm > 1000000) return CC_ERR_INVALID_ARG;
  *out = ppm;
  return CC_OK;
}

}  // namespace

extern "C" {

const char* cc_status_string(int status) {
  switch (status) {
    case CC_OK: return "ok";
    case CC_ERR_INVALID_ARG: return "invalid argument";
    case CC_ERR_INVALID_GRAPH: return "invalid graph";
    case CC_ERR_OOM: return "out of memory";
    case CC_ERR_CUDA: return "CUDA error";
    case CC_ERR_TIMEOUT: return "device wait timed out";
    case CC_ERR_BUSY: return "busy";
    case CC_ERR_INTERNAL: return "internal consistency check failed";
    default: return "unknown status";
  }
}

int cc_graph_destroy(cc_graph* g) {
  if (!g) return CC_OK;
  cudaSetDevice(g->device);
  cudaStream_t s = g->stream;
  if (g->own_off) dfree(g->off, s);
  if (g->own_col) dfree(g->col, s);
  dfree(g->nz_row, s);
  dfree(g->nz_pos, s);
  dfree(g->dsort, s);
  dfree(g->dge, s);
  dfree(g->perm_ws, s);
  dfree(g->order, s);
  dfree(g->round_ws, s);
  dfree(g->labels_tmp, s);
  dfree(g->obj_ws, s);
  dfree(g->obj_out, s);
  dfree(g->stats_dev, s);
  dfree(g->perm_err, s);
  cudaStreamSynchronize(s);
  for (auto& e : g->ev)
    if (e) cudaEventDestroy(e);
  if (g->ctl_host) cudaFreeHost(g->ctl_host);
  if (g->obj_host) cudaFreeHost(g->obj_host);
  delete g;
  return CC_OK;
}

int cc_graph_create(int64_t n, const void* row_offsets, const int32_t* col_idx, uint32_t flags,
                    void* cuda_stream, cc_graph** out) {
  NvtxRange range("cc_graph_create");
  if (!out) return CC_ERR_INVALID_ARG;
  *out = nullptr;
  if (n < 0 || n > 2147483616LL || !row_offsets) return CC_ERR_INVALID_ARG;
  if (flags & ~(CC_VALIDATE | CC_DEVICE_PTRS | CC_OFFSETS_I32 | CC_VALIDATE_EXACT)) return CC_ERR_INVALID_ARG;
  const bool dev = (flags & CC_DEVICE_PTRS) != 0, i32 = (flags & CC_OFFSETS_I32) != 0;
  cc_graph* g = new (std::nothrow) cc_graph();
  if (!g) return CC_ERR_OOM;
  g->stream = static_cast<cudaStream_t>(cuda_stream);
  g->n = n;
  int rc = CC_OK;
  do {
    if (cudaGetDevice(&g->device) != cudaSuccess) { rc = CC_ERR_CUDA; break; }
    cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    cudaStream_t s = g->stream;
    // nnz = off[n]
    int64_t nnz = 0;
    if (dev) {
      if (i32) {
        int32_t t = 0;
        if (cudaMemcpy(&t, static_cast<const int32_t*>(row_offsets) + n, 4, cudaMemcpyDeviceToHost) != cudaSuccess) { rc = CC_ERR_CUDA; break; }
        nnz = t;
      } else if (cudaMemcpy(&nnz, static_cast<const int64_t*>(row_offsets) + n, 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
        rc = CC_ERR_CUDA; break;
      }
    } else {
      nnz = i32 ? static_cast<const int32_t*>(row_offsets)[n] : static_cast<const int64_t*>(row_offsets)[n];
    }
    if (nnz < 0 || nnz >= (int64_t(1) << 33)) { rc = CC_ERR_INVALID_GRAPH; break; }
    if (nnz > 0 && !col_idx) { rc = CC_ERR_INVALID_ARG; break; }
    g->nnz = nnz;
    // offsets
    if (dev && !i32) {
      g->off = const_cast<int64_t*>(static_cast<const int64_t*>(row_offsets));
    } else {
      if ((rc = from_cuda(dalloc(&g->off, 8 * (size_t)(n + 1), s))) != CC_OK) break;
      g->own_off = true;
      if (i32) {
        int32_t* tmp = nullptr;
        if ((rc = from_cuda(dalloc(&tmp, 4 * (size_t)(n + 1), s))) != CC_OK) break;
        cudaMemcpyAsync(tmp, row_offsets, 4 * (size_t)(n + 1), dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
        launch_offsets_i32_to_i64(n, tmp, g->off, s);
        dfree(tmp, s);
      } else if ((rc = from_cuda(cudaMemcpyAsync(g->off, row_offsets, 8 * (size_t)(n + 1), cudaMemcpyHostToDevice, s))) != CC_OK) {
        break;
      }
    }
    // columns: from the host in kColChunks pieces on a copy stream, each
    // checked on s as soon as it has landed, so validation hides under the
    // transfer
    const int chunks = (!dev && nnz > 0) ? kColChunks : 1;
    int64_t cut[kColChunks + 1];
    for (int c = 0; c <= chunks; ++c) cut[c] = nnz / chunks * c + (c == chunks ? nnz % chunks : 0);
    if (dev) {
      g->col = const_cast<int32_t*>(col_idx);
    } else {
      if ((rc = from_cuda(dalloc(&g->col, 4 * (size_t)nnz, s))) != CC_OK) break;
      g->own_col = true;
      if (nnz > 0) {
        cudaEvent_t alloc_done;
        if ((rc = from_cuda(cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking))) != CC_OK) break;
        if ((rc = from_cuda(cudaEventCreateWithFlags(&alloc_done, cudaEventDisableTiming))) != CC_OK) break;
        cudaEventRecord(alloc_done, s);                    // the allocation is ordered on s
        cudaStreamWaitEvent(g->copy_stream, alloc_done, 0);
        cudaEventDestroy(alloc_done);
        for (int c = 0; c < chunks; ++c) {
          if ((rc = from_cuda(cudaEventCreateWithFlags(&g->col_ready[c], cudaEventDisableTiming))) != CC_OK) break;
          if ((rc = from_cuda(cudaMemcpyAsync(g->col + cut[c], col_idx + cut[c], 4 * (size_t)(cut[c + 1] - cut[c]),
                                              cudaMemcpyHostToDevice, g->copy_stream))) != CC_OK)
            break;
          cudaEventRecord(g->col_ready[c], g->copy_stream);
        }
        if (rc != CC_OK) break;
      }
    }
    // validation: offsets first (the non-empty-row list relies on them)
    void* vws = nullptr;
    if ((rc = from_cuda(dalloc(&vws, validate_workspace_bytes(), s))) != CC_OK) break;
    int* vflags_dev = reinterpret_cast<int*>(static_cast<char*>(vws) + align_up(8 * sizeof(unsigned long long)));
    int vflags[2] = {0, 0};
    launch_validate_offsets(n, nnz, g->off, vws, g->num_sms, s);
    cudaMemcpyAsync(vflags, vflags_dev, sizeof(vflags), cudaMemcpyDeviceToHost, s);
    if ((rc = from_cuda(cudaStreamSynchronize(s))) != CC_OK) { dfree(vws, s); break; }
    if (vflags[0] != 0) { dfree(vws, s); rc = CC_ERR_INVALID_GRAPH; break; }
    g->max_deg = vflags[1];
    // non-empty rows (for the edge-balanced passes over the whole CSR)
    if ((rc = from_cuda(dalloc(&g->nz_row, 4 * (size_t)(n > 0 ? n : 1), s))) != CC_OK) { dfree(vws, s); break; }
    if ((rc = from_cuda(dalloc(&g->nz_pos, 8 * (size_t)(n > 0 ? n : 1), s))) != CC_OK) { dfree(vws, s); break; }
    void* nws = nullptr;
    if ((rc = from_cuda(dalloc(&nws, nonempty_workspace_bytes(n), s))) != CC_OK) { dfree(vws, s); break; }
    int64_t* nz_dev = reinterpret_cast<int64_t*>(static_cast<char*>(nws) + nonempty_workspace_bytes(n) - 256);
    launch_nonempty_rows(n, g->off, g->nz_row, g->nz_pos, nws, nz_dev, g->num_sms, s);
    cudaMemcpyAsync(&g->nz_n, nz_dev, 8, cudaMemcpyDeviceToHost, s);
    if ((rc = from_cuda(cudaStreamSynchronize(s))) != CC_OK) { dfree(vws, s); dfree(nws, s); break; }
    // the non-isolated vertices by degree (for the round kernel's Delta)
    {
      void* dws = nullptr;
      if ((rc = from_cuda(dalloc(&g->dsort, 4 * (size_t)(g->nz_n > 0 ? g->nz_n : 1), s))) != CC_OK ||
          (rc = from_cuda(dalloc(&g->dge, 8 * ((size_t)g->max_deg + 2), s))) != CC_OK ||
          (rc = from_cuda(dalloc(&dws, degree_order_workspace_bytes(g->max_deg), s))) != CC_OK) {
        dfree(dws, s); dfree(vws, s); dfree(nws, s);
        break;
      }
      rc = from_cuda(launch_degree_order(g->nz_n, g->nz_row, g->off, g->max_deg, g->dsort, g->dge, dws, g->num_sms, s));
      dfree(dws, s);
      if (rc != CC_OK) { dfree(vws, s); dfree(nws, s); break; }
    }
    for (int c = 0; c < chunks; ++c) {
      if (g->col_ready[c]) cudaStreamWaitEvent(s, g->col_ready[c], 0);
      launch_validate_edges(n, cut[c], cut[c + 1], c == chunks - 1, g->nz_row, g->nz_pos, g->nz_n, g->col, vws,
                            g->num_sms, s);
    }
    if (flags & CC_VALIDATE_EXACT)
      launch_validate_reverse(nnz, g->off, g->nz_row, g->nz_pos, g->nz_n, g->col, vws, g->num_sms, s);
    cudaMemcpyAsync(vflags, vflags_dev, sizeof(vflags), cudaMemcpyDeviceToHost, s);
    dfree(vws, s);
    dfree(nws, s);
    if ((rc = from_cuda(cudaStreamSynchronize(s))) != CC_OK) break;
    if ((rc = from_cuda(cudaGetLastError())) != CC_OK) break;
    if (vflags[0] != 0) { rc = CC_ERR_INVALID_GRAPH; break; }
  } while (false);
  // the copy stream and its events are no longer needed (every chunk is
  // ordered before the work on s, or the graph is being thrown away)
  if (g->copy_stream) {
    cudaStreamSynchronize(g->copy_stream);
    for (auto& e : g->col_ready)
      if (e) { cudaEventDestroy(e); e = nullptr; }
    cudaStreamDestroy(g->copy_stream);
    g->copy_stream = nullptr;
  }
  if (rc != CC_OK) {
    cc_graph_destroy(g);
    return rc;
  }
  *out = g;
  return CC_OK;
}

int cc_graph_info(const cc_graph* g, int64_t* n, int64_t* nnz, int64_t* max_degree) {
  if (!g) return CC_ERR_INVALID_ARG;
  if (n) *n = g->n;
  if (nnz) *nnz = g->nnz;
  if (max_degree) *max_degree = g->max_deg;
  return CC_OK;
}

int cc_permutation(cc_graph* g, uint64_t seed, int32_t* order_out) {
  if (!g || (!order_out && g->n > 0)) return CC_ERR_INVALID_ARG;
  if (g->n == 0) return CC_OK;
  cudaSetDevice(g->device);
  int rc = ensure_cluster_ws(g);
  if (rc != CC_OK) return rc;
  cudaStream_t s = g->stream;
  CC_TRY(cudaMemsetAsync(g->perm_err, 0, sizeof(int), s));
  const bool dev = is_device_ptr(order_out);
  int32_t* dst = dev ? order_out : g->order;
  CC_TRY(launch_permutation(g->n, seed, dst, g->perm_ws, g->num_sms, g->perm_err, s));
  if (!dev) CC_TRY(cudaMemcpyAsync(order_out, g->order, 4 * (size_t)g->n, cudaMemcpyDeviceToHost, s));
  int err = 0;
  CC_TRY(cudaMemcpyAsync(&err, g->perm_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CC_TRY(cudaStreamSynchronize(s));
  return status_of_device_err(err);
}

// C4 without rounds (Alg. 3): permutation, the asynchronous decisions and
// pushes, labels, then the objective from the labels.  One statistics record
// describes the whole run; there are no rounds.
static int cluster_async(cc_graph* g, uint64_t seed, int32_t* labels_out, int32_t* rounds_out,
                         int64_t* disagreements_out, cc_round_stats* stats, int32_t stats_cap, int32_t* stats_len) {
  cudaStream_t s = g->stream;
  int rc = ensure_objective_ws(g);
  if (rc != CC_OK) return rc;
  if (!g->async_grid) g->async_grid = async_grid_size(g->device);
  RoundBuffers b;
  rounds_carve(g->round_ws, g->n, g->max_deg, g->grid, &b);
  b.n = g->n;
  b.nnz = g->nnz;
  b.max_deg = g->max_deg;
  b.off = g->off;
  b.col = g->col;
  b.order = g->order;
  b.nz_static = g->nz_row;
  b.nz_n = g->nz_n;
  b.dsort = g->dsort;
  b.dge = g->dge;
  const bool dev = is_device_ptr(labels_out);
  int32_t* lab = labels_out;
  if (!dev) {
    if ((rc = ensure_labels_tmp(g)) != CC_OK) return rc;
    lab = g->labels_tmp;
  }
  CC_TRY(cudaMemsetAsync(g->perm_err, 0, sizeof(int), s));
  if (g->timing) CC_TRY(cudaEventRecord(g->ev[0], s));
  CC_TRY(launch_permutation(g->n, seed, g->order, g->perm_ws, g->num_sms, g->perm_err, s));
  if (g->timing) CC_TRY(cudaEventRecord(g->ev[1], s));
  CC_TRY(launch_async_c4(b, g->async_grid, lab, s));
  if (g->timing) CC_TRY(cudaEventRecord(g->ev[2], s));
  CC_TRY(launch_disagreements(g->n, g->nnz, g->off, g->col, g->nz_row, g->nz_pos, g->nz_n, lab, g->obj_ws,
                              g->obj_out, g->num_sms, s));
  if (labels_out && !dev) CC_TRY(cudaMemcpyAsync(labels_out, lab, 4 * (size_t)g->n, cudaMemcpyDeviceToHost, s));
  if (g->timing) CC_TRY(cudaEventRecord(g->ev[3], s));
  CC_TRY(cudaMemcpyAsync(g->ctl_host, b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  CC_TRY(cudaMemcpyAsync(g->obj_host, g->obj_out, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  int perr = 0;
  CC_TRY(cudaMemcpyAsync(&perr, g->perm_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CC_TRY(cudaStreamSynchronize(s));
  const Ctl& c = *g->ctl_host;
  if (g->timing) {
    for (int i = 0; i < 3; ++i) CC_TRY(cudaEventElapsedTime(&g->last_ms[i], g->ev[i], g->ev[i + 1]));
    g->timed = true;
  }
  for (auto& x : g->last_phase_ns) x = 0;
  g->phases_valid = true;
  if (perr != 0) return status_of_device_err(perr);
  if (c.err != 0) return status_of_device_err(c.err);
  if (c.r_centers + c.r_noncenter != g->n || g->obj_host[2]) return CC_ERR_INTERNAL;
  if (stats_cap > 0) {
    cc_round_stats& r = stats[0];
    r.n_alive = g->n;
    r.delta = g->max_deg;
    r.k = g->n;
    r.centers = c.r_centers;
    r.removed = g->n;
    r.blocked = c.r_blocked;
    r.edges = c.r_attached;
    r.ns = 0;
  }
  if (stats_len) *stats_len = 1;
  if (rounds_out) *rounds_out = 0;
  if (disagreements_out) *disagreements_out = g->nnz / 2 - (int64_t)g->obj_host[0] + (int64_t)g->obj_host[1];
  return CC_OK;
}

int cc_cluster_ex(cc_graph* g, int algo, double eps, uint64_t seed, int32_t* labels_out, int32_t* rounds_out,
                  int64_t* disagreements_out, cc_round_stats* stats, int32_t stats_cap, int32_t* stats_len) {
  NvtxRange range("cc_cluster");
  if (!g) return CC_ERR_INVALID_ARG;
  // the test hook belongs to this call whatever its outcome (a bad argument,
  // an empty graph, a failed allocation, the asynchronous algorithm)
  const int32_t withhold = g->withhold;
  g->withhold = 0;
  if (algo < CC_ALGO_C4 || algo > CC_ALGO_C4_ASYNC) return CC_ERR_INVALID_ARG;
  if (stats_cap < 0 || (stats_cap > 0 && !stats)) return CC_ERR_INVALID_ARG;
  int64_t ppm = 0;
  int rc = eps_ppm_of(eps, &ppm);
  if (rc != CC_OK) return rc;
  if (g->n == 0) {
    if (rounds_out) *rounds_out = 0;
    if (disagreements_out) *disagreements_out = 0;
    if (stats_len) *stats_len = 0;
    return CC_OK;
  }
  cudaSetDevice(g->device);
  if ((rc = ensure_cluster_ws(g)) != CC_OK) return rc;
  cudaStream_t s = g->stream;
  if (stats_cap > g->stats_dev_cap) {
    dfree(g->stats_dev, s);
    CC_TRY(dalloc(&g->stats_dev, sizeof(RoundStat) * (size_t)stats_cap, s));
    g->stats_dev_cap = stats_cap;
  }
  if (algo == CC_ALGO_C4_ASYNC)
    return cluster_async(g, seed, labels_out, rounds_out, disagreements_out, stats, stats_cap, stats_len);
  RoundBuffers b;
  rounds_carve(g->round_ws, g->n, g->max_deg, g->grid, &b);
  b.tune = g->tune;
  b.n = g->n;
  b.nnz = g->nnz;
  b.max_deg = g->max_deg;
  b.off = g->off;
  b.col = g->col;
  b.order = g->order;
  b.nz_static = g->nz_row;
  b.nz_n = g->nz_n;
  b.dsort = g->dsort;
  b.dge = g->dge;
  b.stats = g->stats_dev;
  b.stats_cap = stats_cap;
  CC_TRY(cudaMemsetAsync(g->perm_err, 0, sizeof(int), s));
  if (g->timing) CC_TRY(cudaEventRecord(g->ev[0], s));
  {
    NvtxRange r("permutation");
    CC_TRY(launch_permutation(g->n, seed, g->order, g->perm_ws, g->num_sms, g->perm_err, s));
  }
  if (g->timing) CC_TRY(cudaEventRecord(g->ev[1], s));
  {
    NvtxRange r("rounds");
    CC_TRY(launch_rounds(b, algo, ppm, seed, g->grid, s, withhold));
  }
  if (g->timing) CC_TRY(cudaEventRecord(g->ev[2], s));
  NvtxRange labels_range("labels");
  const bool dev = is_device_ptr(labels_out);
  if (labels_out && !dev) {
    if ((rc = ensure_labels_tmp(g)) != CC_OK) return rc;
    CC_TRY(launch_finalize_labels(b, g->labels_tmp, s));
    CC_TRY(cudaMemcpyAsync(labels_out, g->labels_tmp, 4 * (size_t)g->n, cudaMemcpyDeviceToHost, s));
  } else {
    CC_TRY(launch_finalize_labels(b, labels_out, s));   // also the objective's pair term
  }
  if (g->timing) CC_TRY(cudaEventRecord(g->ev[3], s));
  CC_TRY(cudaMemcpyAsync(g->ctl_host, b.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s));
  int perr = 0;
  CC_TRY(cudaMemcpyAsync(&perr, g->perm_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CC_TRY(cudaStreamSynchronize(s));
  const Ctl& c = *g->ctl_host;
  if (g->timing) {
    for (int i = 0; i < 3; ++i) CC_TRY(cudaEventElapsedTime(&g->last_ms[i], g->ev[i], g->ev[i + 1]));
    g->timed = true;
  }
  for (int i = 0; i < 8; ++i) g->last_phase_ns[i] = c.ph_ns[i];
  g->phases_valid = true;
  if (perr != 0) return status_of_device_err(perr);
  if (c.err != 0) return status_of_device_err(c.err);
  if (c.n_alive != 0 || !c.done) return CC_ERR_INTERNAL;
  const int64_t rounds = c.round;
  if (stats_cap > 0) {
    const int64_t cnt = rounds < stats_cap ? rounds : stats_cap;
    static_assert(sizeof(cc_round_stats) == sizeof(RoundStat), "round stats layout");
    if (cnt > 0) CC_TRY(cudaMemcpy(stats, g->stats_dev, sizeof(RoundStat) * (size_t)cnt, cudaMemcpyDeviceToHost));
  }
  if (stats_len) *stats_len = (int32_t)rounds;
  if (rounds_out) *rounds_out = (int32_t)rounds;
  if (disagreements_out) {
    const int64_t m = g->nnz / 2;
    *disagreements_out = m - 2 * (int64_t)c.mc - (int64_t)c.mm + (int64_t)c.pairs;
  }
  return CC_OK;
}

int cc_debug_withhold_release(cc_graph* g, int32_t round) {
  if (!g || round < 0 || round > 2147483646) return CC_ERR_INVALID_ARG;
  g->withhold = round + 1;
  return CC_OK;
}

int cc_graph_set_timing(cc_graph* g, int enable) {
  if (!g) return CC_ERR_INVALID_ARG;
  cudaSetDevice(g->device);
  if (enable)
    for (auto& e : g->ev)
      if (!e) CC_TRY(cudaEventCreate(&e));
  g->timing = enable != 0;
  g->timed = false;
  return CC_OK;
}

int cc_last_timings(const cc_graph* g, float* ms_out) {
  if (!g || !ms_out || !g->timing || !g->timed) return CC_ERR_INVALID_ARG;
  for (int i = 0; i < 3; ++i) ms_out[i] = g->last_ms[i];
  return CC_OK;
}

int cc_last_phase_times(const cc_graph* g, double* ms_out, int32_t cap) {
  if (!g || !ms_out || cap < 0 || !g->phases_valid) return CC_ERR_INVALID_ARG;
  for (int32_t i = 0; i < cap && i < 7; ++i) ms_out[i] = (double)g->last_phase_ns[i] * 1e-6;
  return CC_OK;
}

int cc_cluster(cc_graph* g, int algo, double eps, uint64_t seed, int32_t* labels_out, int32_t* rounds_out,
               int64_t* disagreements_out) {
  return cc_cluster_ex(g, algo, eps, seed, labels_out, rounds_out, disagreements_out, nullptr, 0, nullptr);
}

int cc_disagreements(cc_graph* g, const int32_t* labels, int64_t* out) {
  NvtxRange range("cc_disagreements");
  if (!g || !out || (!labels && g->n > 0)) return CC_ERR_INVALID_ARG;
  if (g->n == 0) { *out = 0; return CC_OK; }
  cudaSetDevice(g->device);
  cudaStream_t s = g->stream;
  int orc = ensure_objective_ws(g);
  if (orc != CC_OK) return orc;
  const int32_t* lab = labels;
  if (!is_device_ptr(labels)) {
    int rc = ensure_labels_tmp(g);
    if (rc != CC_OK) return rc;
    CC_TRY(cudaMemcpyAsync(g->labels_tmp, labels, 4 * (size_t)g->n, cudaMemcpyHostToDevice, s));
    lab = g->labels_tmp;
  }
  CC_TRY(launch_disagreements(g->n, g->nnz, g->off, g->col, g->nz_row, g->nz_pos, g->nz_n, lab, g->obj_ws,
                              g->obj_out, g->num_sms, s));
  CC_TRY(cudaMemcpyAsync(g->obj_host, g->obj_out, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  CC_TRY(cudaStreamSynchronize(s));
  if (g->obj_host[2]) return CC_ERR_INVALID_ARG;
  *out = g->nnz / 2 - (int64_t)g->obj_host[0] + (int64_t)g->obj_host[1];
  return CC_OK;
}

}  // extern "C"

namespace {

// Runs every (graph, permutation) job; jobs[i * k_perms + j] gets its rounds
// and disagreements.
int run_batch_jobs(cc_graph* const* gs, int32_t count, int algo, double eps, const uint64_t* seeds, int32_t k_perms,
                   std::vector<BatchJob>& jobs) {
  NvtxRange range("cc_batch_jobs");
  if (count < 0 || k_perms < 1 || (count > 0 && (!gs || !seeds))) return CC_ERR_INVALID_ARG;
  if (algo < CC_ALGO_C4 || algo > CC_ALGO_CLUSTERWILD_EST) return CC_ERR_INVALID_ARG;
  int64_t ppm = 0;
  int rc = eps_ppm_of(eps, &ppm);
  if (rc != CC_OK) return rc;
  if (count == 0) { jobs.clear(); return CC_OK; }
  for (int32_t i = 0; i < count; ++i)
    if (!gs[i] || gs[i]->device != gs[0]->device) return CC_ERR_INVALID_ARG;
  cudaSetDevice(gs[0]->device);
  cudaStream_t s = gs[0]->stream;
  for (int32_t i = 1; i < count; ++i)
    if (gs[i]->stream != s) CC_TRY(cudaStreamSynchronize(gs[i]->stream));
  // one job per (graph, permutation)
  const int64_t njobs = (int64_t)count * k_perms;
  jobs.assign((size_t)njobs, BatchJob{});
  for (int32_t i = 0; i < count; ++i)
    for (int32_t j = 0; j < k_perms; ++j) {
      BatchJob& jb = jobs[(size_t)i * k_perms + j];
      const cc_graph* g = gs[i];
      jb = BatchJob{};
      jb.off = g->off; jb.col = g->col; jb.nz = g->nz_row; jb.nz_n = g->nz_n;
      jb.dsort = g->dsort; jb.dge = g->dge;
      jb.n = g->n; jb.nnz = g->nnz; jb.max_deg = g->max_deg;
      jb.seed = seeds[i] + (uint64_t)j;
      jb.err = 1;
      jb.rounds = 0;
      jb.D = 0;
    }
  // size classes: one block per job, eight-block teams, or the whole grid
  const cc_tuning tune = batch_tuning();
  std::vector<int64_t> cls[3];
  for (int64_t q = 0; q < njobs; ++q) {
    const int64_t n = jobs[(size_t)q].n;
    cls[n <= tune.batch_small_n ? 0 : (n <= tune.batch_team_n ? 1 : 2)].push_back(q);
  }
  const int grid0 = batch_grid_size(gs[0]->device);
  for (int c = 0; c < 2; ++c) {
    std::vector<int64_t>& ids = cls[c];
    if (ids.empty()) continue;
    std::sort(ids.begin(), ids.end(), [&](int64_t a, int64_t b2) { return jobs[(size_t)a].n > jobs[(size_t)b2].n; });
    const int team = c == 0 ? 1 : tune.batch_team_blocks;
    const int teams = grid0 / team;
    if (teams < 1) return CC_ERR_INTERNAL;
    const int grid = teams * team;
    const int64_t n_max = jobs[(size_t)ids[0]].n;
    const size_t slot = align_up(batch_slot_bytes(n_max, team));
    void* ws = nullptr;
    CC_TRY(dalloc(&ws, slot * (size_t)teams, s));
    std::vector<RoundBuffers> slots((size_t)teams);
    for (int t = 0; t < teams; ++t) {
      batch_slot_carve(static_cast<char*>(ws) + slot * (size_t)t, n_max, team, &slots[(size_t)t]);
      slots[(size_t)t].tune = device_tuning(tune);
      CC_TRY(cudaMemsetAsync(slots[(size_t)t].ctl, 0, sizeof(Ctl), s));
    }
    std::vector<BatchJob> sub(ids.size());
    for (size_t q = 0; q < ids.size(); ++q) sub[q] = jobs[(size_t)ids[q]];
    BatchJob* jobs_dev = nullptr;
    RoundBuffers* slots_dev = nullptr;
    CC_TRY(dalloc(&jobs_dev, sizeof(BatchJob) * sub.size(), s));
    CC_TRY(dalloc(&slots_dev, sizeof(RoundBuffers) * slots.size(), s));
    CC_TRY(cudaMemcpyAsync(jobs_dev, sub.data(), sizeof(BatchJob) * sub.size(), cudaMemcpyHostToDevice, s));
    CC_TRY(cudaMemcpyAsync(slots_dev, slots.data(), sizeof(RoundBuffers) * slots.size(), cudaMemcpyHostToDevice, s));
    CC_TRY(launch_batch(jobs_dev, (int)sub.size(), slots_dev, team, grid, algo, ppm, s));
    CC_TRY(cudaMemcpyAsync(sub.data(), jobs_dev, sizeof(BatchJob) * sub.size(), cudaMemcpyDeviceToHost, s));
    dfree(jobs_dev, s);
    dfree(slots_dev, s);
    dfree(ws, s);
    CC_TRY(cudaStreamSynchronize(s));
    for (size_t q = 0; q < ids.size(); ++q) {
      if (sub[q].err != 0) return sub[q].err == CC_ERR_TIMEOUT ? CC_ERR_TIMEOUT : CC_ERR_INTERNAL;
      jobs[(size_t)ids[q]].rounds = sub[q].rounds;
      jobs[(size_t)ids[q]].D = sub[q].D;
      jobs[(size_t)ids[q]].err = 0;
    }
  }
  for (int64_t q : cls[2]) {   // graphs too large for a team: the whole grid per job
    BatchJob& jb = jobs[(size_t)q];
    int32_t r = 0;
    int64_t d = 0;
    rc = cc_cluster(gs[q / k_perms], algo, eps, jb.seed, nullptr, &r, &d);
    if (rc != CC_OK) return rc;
    jb.rounds = r;
    jb.D = d;
    jb.err = 0;
  }
  return CC_OK;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace ccg {
// The process-wide batch settings (cc_set_batch_tuning) as the server reads
// them when it is created.
Tuning batch_settings(int64_t* small_n, int64_t* team_n, int* team_blocks) {
  const cc_tuning t = batch_tuning();
  *small_n = t.batch_small_n;
  *team_n = t.batch_team_n;
  *team_blocks = t.batch_team_blocks;
  return device_tuning(t);
}
}  // namespace ccg

extern "C" {

int cc_tuning_default(cc_tuning* out) {
  if (!out) return CC_ERR_INVALID_ARG;
  *out = public_default_tuning();
  return CC_OK;
}

int cc_graph_set_tuning(cc_graph* g, const cc_tuning* t) {
  if (!g || !t || !tuning_valid(*t)) return CC_ERR_INVALID_ARG;
  g->tune = device_tuning(*t);
  return CC_OK;
}

int cc_graph_get_tuning(const cc_graph* g, cc_tuning* out) {
  if (!g || !out) return CC_ERR_INVALID_ARG;
  const cc_tuning b = batch_tuning();
  *out = b;
  out->walk_batches = g->tune.walk_batches;
  out->prefetch_ahead = g->tune.prefetch_ahead;
  out->inline_heavy = g->tune.inline_heavy;
  out->inline_decide = g->tune.inline_decide;
  out->inline_rebuild = g->tune.inline_rebuild;
  out->heavy_shift = g->tune.heavy_shift;
  out->warp_resolve_row = g->tune.warp_resolve_row;
  return CC_OK;
}

int cc_set_batch_tuning(const cc_tuning* t) {
  if (!t || !tuning_valid(*t)) return CC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_batch_tuning = *t;
  g_batch_tuning_set = true;
  return CC_OK;
}

int cc_get_batch_tuning(cc_tuning* out) {
  if (!out) return CC_ERR_INVALID_ARG;
  *out = batch_tuning();
  return CC_OK;
}

int cc_batch_jobs(cc_graph* const* gs, int32_t count, int algo, double eps, const uint64_t* seeds, int32_t k_perms,
                  int64_t* D_out, int32_t* rounds_out) {
  std::vector<BatchJob> jobs;
  const int rc = run_batch_jobs(gs, count, algo, eps, seeds, k_perms, jobs);
  if (rc != CC_OK) return rc;
  for (size_t q = 0; q < jobs.size(); ++q) {
    if (D_out) D_out[q] = jobs[q].D;
    if (rounds_out) rounds_out[q] = (int32_t)jobs[q].rounds;
  }
  return CC_OK;
}

int cc_batch_run(cc_graph* const* gs, int32_t count, int algo, double eps, const uint64_t* seeds, int32_t k_perms,
                 int32_t* const* labels_out, int32_t* best_j, int64_t* best_D, int32_t* rounds) {
  std::vector<BatchJob> jobs;
  int rc = run_batch_jobs(gs, count, algo, eps, seeds, k_perms, jobs);
  if (rc != CC_OK) return rc;
  // best of k per graph: lowest D, ties to the lowest j
  for (int32_t i = 0; i < count; ++i) {
    int32_t bj = 0;
    for (int32_t j = 1; j < k_perms; ++j)
      if (jobs[(size_t)i * k_perms + j].D < jobs[(size_t)i * k_perms + bj].D) bj = j;
    const BatchJob& b = jobs[(size_t)i * k_perms + bj];
    if (best_j) best_j[i] = bj;
    if (best_D) best_D[i] = b.D;
    if (rounds) rounds[i] = (int32_t)b.rounds;
    if (labels_out && labels_out[i]) {
      // labels of the winning permutation (the same deterministic clustering)
      rc = cc_cluster(gs[i], algo, eps, b.seed, labels_out[i], nullptr, nullptr);
      if (rc != CC_OK) return rc;
    }
  }
  return CC_OK;
}

}  // extern "C"
