// cc_objective.cu -- the disagreement objective (Sec. 2) of an arbitrary
// labelling, CSR validation and small graph utilities.
//
// Disagreements: with m positive edges, intra = positive edges inside a
// cluster and s_c the cluster sizes,
//     D = (m - intra) + (sum_c C(s_c, 2) - intra) = m - intra_dir + sum_c C(s_c, 2)
// where intra_dir = 2 * intra counts CSR entries (u, w) with label[u] == label[w].
// One pass counts cluster sizes, one edge-balanced pass over the non-empty
// rows counts intra_dir, one pass sums C(s_c, 2).
#include <cstdint>

#include "cc_device.cuh"
#include "cc_internal.h"

namespace ccg {
namespace {

constexpr int kObjThreads = 512;

__global__ void k_cluster_sizes(int64_t n, const int32_t* __restrict__ labels, int32_t* __restrict__ size,
                                unsigned long long* out) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = labels[v];
    if (c < 0 || c >= n) { atomicExch(out + 2, 1ull); continue; }
    atomicAdd(size + c, 1);
  }
}

__global__ void __launch_bounds__(kObjThreads) k_intra(int64_t nz_n, const int32_t* __restrict__ nz_row,
                                                      const int64_t* __restrict__ nz_pos, int64_t nnz,
                                                      const int32_t* __restrict__ col,
                                                      const int32_t* __restrict__ labels, unsigned long long* out) {
  __shared__ LbsWarp lbs[kObjThreads / 32];
  __shared__ int64_t scr[33];
  int64_t cnt = 0;
  // the non-empty rows are contiguous in the CSR, so virtual edge e is CSR entry e
  lbs_for_each(nz_pos, nz_n, nnz, &lbs[threadIdx.x >> 5], [&](const Lbs& L) {
    int32_t lu[kLbsK], w[kLbsK];
#pragma unroll
    for (int t = 0; t < kLbsK; ++t) {
      lu[t] = L.ok(t) ? __ldg(labels + __ldg(nz_row + L.item(t))) : 0;
      w[t] = L.ok(t) ? __ldg(col + L.edge(t)) : 0;
    }
#pragma unroll
    for (int t = 0; t < kLbsK; ++t)
      if (L.ok(t)) cnt += (__ldg(labels + w[t]) == lu[t]) ? 1 : 0;
  }, nullptr, nullptr, 0, col);
  cnt = block_sum<int64_t>(cnt, scr);
  if (threadIdx.x == 0 && cnt) atomicAdd(out + 0, (unsigned long long)cnt);
}

__global__ void k_pairs(int64_t n, const int32_t* __restrict__ size, unsigned long long* out) {
  __shared__ int64_t scr[33];
  int64_t acc = 0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = size[c];
    acc += s * (s - 1) / 2;
  }
  acc = block_sum<int64_t>(acc, scr);
  if (threadIdx.x == 0 && acc) atomicAdd(out + 1, (unsigned long long)acc);
}

// ---- validation ---------------------------------------------------------------
// Error codes written to flags[0] (first one wins).
constexpr int kBadOffsets = 1, kBadColumn = 2, kSelfLoop = 3, kUnsorted = 4, kAsymmetric = 5;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 33)) * 0xFF51AFD7ED558CCDull;
  z = (z ^ (z >> 33)) * 0xC4CEB9FE1A85EC53ull;
  return z ^ (z >> 33);
}

// Offsets: monotone, inside [0, nnz]; largest degree.
__global__ void k_validate_offsets(int64_t n, int64_t nnz, const int64_t* __restrict__ off, int* flags) {
  int dmax = 0;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = off[u], b = off[u + 1];
    if (a < 0 || b < a || b > nnz) { atomicCAS(flags, 0, kBadOffsets); continue; }
    const int64_t d = b - a;
    dmax = max(dmax, d > 0x7FFFFFFF ? 0x7FFFFFFF : (int)d);
  }
  dmax = warp_max(dmax);
  if ((threadIdx.x & 31) == 0 && dmax > 0) atomicMax(flags + 1, dmax);
}

// Entries, edge-balanced over the non-empty rows: range, order, self loops;
// symmetry by comparing two hash sums of the pairs (min, max) seen from the
// lower and from the upper endpoint (equal multisets give equal sums).
constexpr int kValThreads = 512;

__global__ void __launch_bounds__(kValThreads) k_validate_edges(int64_t n, int64_t e0, int64_t e1, int64_t nz_n,
                                                               const int32_t* __restrict__ nz_row,
                                                               const int64_t* __restrict__ nz_pos,
                                                               const int32_t* __restrict__ col, int* flags,
                                                               unsigned long long* sums) {
  __shared__ LbsWarp lbs[kValThreads / 32];
  unsigned long long lo1 = 0, lo2 = 0, up1 = 0, up2 = 0;
  long long nlo = 0, nup = 0;
  int bad = 0;
  lbs_for_each(nz_pos, nz_n, e1, &lbs[threadIdx.x >> 5], [&](const Lbs& L) {
#pragma unroll
    for (int t = 0; t < kLbsK; ++t) {
      if (!L.ok(t)) continue;
      const int64_t e = L.edge(t);
      const int32_t u = __ldg(nz_row + L.item(t));
      const int32_t w = __ldg(col + e);
      if (w < 0 || w >= n) { bad = bad ? bad : kBadColumn; continue; }
      if (w == u) { bad = bad ? bad : kSelfLoop; continue; }
      if (L.in_row(t) > 0 && __ldg(col + e - 1) >= w) bad = bad ? bad : kUnsorted;
      const uint64_t key = u < w ? (((uint64_t)u << 32) | (uint32_t)w) : (((uint64_t)w << 32) | (uint32_t)u);
      const uint64_t h1 = mix64(key ^ 0x9E3779B97F4A7C15ull), h2 = mix64(key + 0x632BE59BD9B4E019ull);
      if (u < w) { lo1 += h1; lo2 += h2; ++nlo; } else { up1 += h1; up2 += h2; ++nup; }
    }
  }, nullptr, nullptr, e0, col);
  if (bad) atomicCAS(flags, 0, bad);
  lo1 = warp_sum(lo1); lo2 = warp_sum(lo2); up1 = warp_sum(up1); up2 = warp_sum(up2);
  nlo = warp_sum(nlo); nup = warp_sum(nup);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(sums + 0, lo1); atomicAdd(sums + 1, lo2);
    atomicAdd(sums + 2, up1); atomicAdd(sums + 3, up2);
    atomicAdd(sums + 4, (unsigned long long)nlo); atomicAdd(sums + 5, (unsigned long long)nup);
  }
}

// Exact symmetry (opt-in): every entry (u, w) with u < w must have u in row w,
// found by binary search in that sorted row.  Together with the equal counts
// of lower and upper entries (k_validate_symmetry) this makes the entries
// seen from the two ends the same set of pairs.
__global__ void __launch_bounds__(kValThreads) k_validate_reverse(int64_t nz_n, const int32_t* __restrict__ nz_row,
                                                                 const int64_t* __restrict__ nz_pos, int64_t nnz,
                                                                 const int64_t* __restrict__ off,
                                                                 const int32_t* __restrict__ col, int* flags) {
  __shared__ LbsWarp lbs[kValThreads / 32];
  int bad = 0;
  lbs_for_each(nz_pos, nz_n, nnz, &lbs[threadIdx.x >> 5], [&](const Lbs& L) {
#pragma unroll
    for (int t = 0; t < kLbsK; ++t) {
      if (!L.ok(t)) continue;
      const int32_t u = __ldg(nz_row + L.item(t));
      const int32_t w = __ldg(col + L.edge(t));
      if (w <= u) continue;
      int64_t lo = __ldg(off + w), hi = __ldg(off + w + 1);
      while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(col + mid) < u) lo = mid + 1;
        else hi = mid;
      }
      if (lo >= __ldg(off + w + 1) || __ldg(col + lo) != u) bad = kAsymmetric;
    }
  }, nullptr, nullptr, 0, col);
  if (bad) atomicCAS(flags, 0, bad);
}

__global__ void k_validate_finish(int64_t n, const int64_t* __restrict__ off, int64_t nnz, int* flags,
                                  const unsigned long long* sums) {
  (void)sums;
  if (off[0] != 0 || off[n] != nnz) atomicCAS(flags, 0, kBadOffsets);
}

__global__ void k_validate_symmetry(int* flags, const unsigned long long* sums) {
  if (sums[0] != sums[2] || sums[1] != sums[3] || sums[4] != sums[5]) atomicCAS(flags, 0, kAsymmetric);
}

__global__ void k_off32_to_64(int64_t n, const int32_t* __restrict__ in, int64_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}

// Non-empty rows: per-block counts, a single-block scan, then the write.
constexpr int kNzTile = 1024;

__global__ void k_nz_count(int64_t n, const int64_t* __restrict__ off, int64_t* __restrict__ tile_cnt) {
  __shared__ int64_t scr[33];
  const int64_t ntiles = (n + kNzTile - 1) / kNzTile;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t v = t * kNzTile + threadIdx.x;
    int64_t c = (v < n && off[v + 1] > off[v]) ? 1 : 0;
    c = block_sum<int64_t>(c, scr);
    if (threadIdx.x == 0) tile_cnt[t] = c;
  }
}

__global__ void k_nz_scan(int64_t ntiles, int64_t* __restrict__ tile_cnt, int64_t* __restrict__ total) {
  __shared__ int64_t scr[33];
  int64_t run = 0;
  for (int64_t base = 0; base < ntiles; base += blockDim.x) {
    const int64_t t = base + threadIdx.x;
    const int64_t x = t < ntiles ? tile_cnt[t] : 0;
    int64_t tot;
    const int64_t ex = block_exclusive_sum<int64_t>(x, scr, &tot);
    if (t < ntiles) tile_cnt[t] = run + ex;
    run += tot;
  }
  if (threadIdx.x == 0) *total = run;
}

__global__ void k_nz_write(int64_t n, const int64_t* __restrict__ off, const int64_t* __restrict__ tile_off,
                           int32_t* __restrict__ nz_row, int64_t* __restrict__ nz_pos) {
  __shared__ int64_t scr[33];
  const int64_t ntiles = (n + kNzTile - 1) / kNzTile;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t v = t * kNzTile + threadIdx.x;
    const int64_t c = (v < n && off[v + 1] > off[v]) ? 1 : 0;
    int64_t tot;
    const int64_t ex = block_exclusive_sum<int64_t>(c, scr, &tot);
    if (c) {
      nz_row[tile_off[t] + ex] = (int32_t)v;
      nz_pos[tile_off[t] + ex] = off[v];
    }
  }
}

// ---- the non-isolated vertices ordered by degree --------------------------
// dsort lists the non-isolated vertices, largest degree first (ties in any
// order), and dge[t] (t = 0 .. max_deg + 1) counts the vertices of degree
// >= t, so dsort[0 .. dge[t]) are exactly the vertices of degree >= t.  The
// round kernel's Delta rebuild reads such a prefix.  Degrees below kDegSmall
// are counted and placed through shared-memory bins (one global atomic per
// block and bin), larger ones (few vertices) directly.
constexpr int kDegSmall = 2048;
constexpr int kDegThreads = 1024;
constexpr int kDegPer = 4;

__global__ void __launch_bounds__(kDegThreads) k_deg_hist(int64_t nz_n, const int32_t* __restrict__ nz_row,
                                                         const int64_t* __restrict__ off,
                                                         unsigned long long* __restrict__ cnt) {
  __shared__ int bin[kDegSmall];
  for (int b = threadIdx.x; b < kDegSmall; b += blockDim.x) bin[b] = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nz_n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = nz_row[i];
    const int64_t d = off[v + 1] - off[v];
    if (d < kDegSmall) atomicAdd(&bin[d], 1);
    else atomicAdd(cnt + d, 1ull);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kDegSmall; b += blockDim.x)
    if (bin[b]) atomicAdd(cnt + b, (unsigned long long)bin[b]);
}

// dge[t] = sum of cnt[d] over d >= t (suffix sums), in three steps over tiles
// of kDegThreads entries: each tile's own suffix sums and total, a suffix
// scan of the tile totals by one block, then each entry adds the totals of
// the tiles after its own.  cnt[d] then becomes the first position of degree
// d in dsort, dge[d + 1] = dge[d] - cnt[d].
__global__ void __launch_bounds__(kDegThreads) k_deg_suffix_tiles(int64_t len, const unsigned long long* __restrict__ cnt,
                                                                 int64_t* __restrict__ dge, int64_t* __restrict__ tile_tot) {
  __shared__ int64_t scr[33];
  // tile t covers indices [len - (t + 1) * kDegThreads, len - t * kDegThreads), read top down
  const int64_t idx = len - 1 - ((int64_t)blockIdx.x * kDegThreads + threadIdx.x);
  const int64_t x = idx >= 0 ? (int64_t)cnt[idx] : 0;
  int64_t tot;
  const int64_t ex = block_exclusive_sum<int64_t>(x, scr, &tot);
  if (idx >= 0) dge[idx] = ex + x;
  if (threadIdx.x == 0) tile_tot[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kDegThreads) k_deg_suffix_totals(int64_t ntiles, int64_t* __restrict__ tile_tot) {
  __shared__ int64_t scr[33];
  int64_t run = 0;
  for (int64_t base = 0; base < ntiles; base += blockDim.x) {
    const int64_t t = base + threadIdx.x;
    const int64_t x = t < ntiles ? tile_tot[t] : 0;
    int64_t tot;
    const int64_t ex = block_exclusive_sum<int64_t>(x, scr, &tot);
    if (t < ntiles) tile_tot[t] = run + ex;     // the totals of the tiles above tile t
    run += tot;
  }
}

__global__ void __launch_bounds__(kDegThreads) k_deg_suffix_add(int64_t len, unsigned long long* __restrict__ cnt,
                                                               int64_t* __restrict__ dge,
                                                               const int64_t* __restrict__ tile_tot) {
  const int64_t idx = len - 1 - ((int64_t)blockIdx.x * kDegThreads + threadIdx.x);
  if (idx < 0) return;
  const int64_t d = dge[idx] + tile_tot[blockIdx.x];
  dge[idx] = d;
  if (idx < len - 1) cnt[idx] = (unsigned long long)(d - (int64_t)cnt[idx]);
}

__global__ void __launch_bounds__(kDegThreads) k_deg_scatter(int64_t nz_n, const int32_t* __restrict__ nz_row,
                                                            const int64_t* __restrict__ off,
                                                            unsigned long long* __restrict__ cur,
                                                            int32_t* __restrict__ dsort) {
  __shared__ int bin[kDegSmall];
  __shared__ unsigned long long base[kDegSmall];
  const int64_t tile = (int64_t)kDegThreads * kDegPer;
  for (int64_t t0 = blockIdx.x * tile; t0 < nz_n; t0 += (int64_t)gridDim.x * tile) {
    for (int b = threadIdx.x; b < kDegSmall; b += blockDim.x) bin[b] = 0;
    __syncthreads();
    int32_t v[kDegPer];
    int32_t d[kDegPer];
    int r[kDegPer];
#pragma unroll
    for (int q = 0; q < kDegPer; ++q) {
      const int64_t i = t0 + (int64_t)q * blockDim.x + threadIdx.x;
      v[q] = i < nz_n ? nz_row[i] : -1;
      d[q] = v[q] >= 0 ? (int32_t)(off[v[q] + 1] - off[v[q]]) : 0;
      r[q] = 0;
      if (v[q] < 0) continue;
      if (d[q] < kDegSmall) r[q] = atomicAdd(&bin[d[q]], 1);
      else dsort[atomicAdd(cur + d[q], 1ull)] = v[q];
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kDegSmall; b += blockDim.x)
      if (bin[b]) base[b] = atomicAdd(cur + b, (unsigned long long)bin[b]);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kDegPer; ++q)
      if (v[q] >= 0 && d[q] < kDegSmall) dsort[base[d[q]] + r[q]] = v[q];
    __syncthreads();
  }
}

}  // namespace

size_t degree_order_workspace_bytes(int32_t max_deg) {
  const size_t len = (size_t)max_deg + 2;
  return align_up(8 * len) + align_up(8 * ((len + kDegThreads - 1) / kDegThreads));
}

cudaError_t launch_degree_order(int64_t nz_n, const int32_t* nz_row, const int64_t* off, int32_t max_deg,
                                int32_t* dsort, int64_t* dge, void* ws, int num_sms, cudaStream_t stream) {
  const int64_t len = (int64_t)max_deg + 2;             // degrees 0 .. max_deg + 1
  const int64_t ntiles = (len + kDegThreads - 1) / kDegThreads;
  unsigned long long* cnt = static_cast<unsigned long long*>(ws);
  int64_t* tile_tot = reinterpret_cast<int64_t*>(static_cast<char*>(ws) + align_up(8 * (size_t)len));
  cudaError_t e = cudaMemsetAsync(cnt, 0, 8 * (size_t)len, stream);
  if (e != cudaSuccess) return e;
  const int g = num_sms > 0 ? num_sms : 1;
  if (nz_n > 0) k_deg_hist<<<g, kDegThreads, 0, stream>>>(nz_n, nz_row, off, cnt);
  k_deg_suffix_tiles<<<(unsigned)ntiles, kDegThreads, 0, stream>>>(len, cnt, dge, tile_tot);
  k_deg_suffix_totals<<<1, kDegThreads, 0, stream>>>(ntiles, tile_tot);
  k_deg_suffix_add<<<(unsigned)ntiles, kDegThreads, 0, stream>>>(len, cnt, dge, tile_tot);
  if (nz_n > 0) k_deg_scatter<<<g, kDegThreads, 0, stream>>>(nz_n, nz_row, off, cnt, dsort);
  return cudaGetLastError();
}

size_t objective_workspace_bytes(int64_t n) {
  return align_up(4 * (size_t)(n > 0 ? n : 1)) + align_up(8 * 4);
}

cudaError_t launch_disagreements(int64_t n, int64_t nnz, const int64_t* off, const int32_t* col,
                                 const int32_t* nz_row, const int64_t* nz_pos, int64_t nz_n,
                                 const int32_t* labels, void* ws, unsigned long long* out, int num_sms,
                                 cudaStream_t stream) {
  (void)off;
  int32_t* size = static_cast<int32_t*>(ws);
  cudaError_t e = cudaMemsetAsync(size, 0, 4 * (size_t)(n > 0 ? n : 1), stream);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(out, 0, 3 * sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return e;
  if (n <= 0) return cudaSuccess;
  const int g = num_sms * 4;
  k_cluster_sizes<<<g, 256, 0, stream>>>(n, labels, size, out);
  if (nnz > 0) k_intra<<<num_sms * 2, kObjThreads, 0, stream>>>(nz_n, nz_row, nz_pos, nnz, col, labels, out);
  k_pairs<<<g, 256, 0, stream>>>(n, size, out);
  return cudaGetLastError();
}

size_t validate_workspace_bytes() { return align_up(8 * sizeof(unsigned long long)) + align_up(2 * sizeof(int)); }

cudaError_t launch_validate_offsets(int64_t n, int64_t nnz, const int64_t* off, void* ws, int num_sms,
                                    cudaStream_t stream) {
  int* flags = reinterpret_cast<int*>(static_cast<char*>(ws) + align_up(8 * sizeof(unsigned long long)));
  cudaError_t e = cudaMemsetAsync(ws, 0, validate_workspace_bytes(), stream);
  if (e != cudaSuccess) return e;
  if (n > 0) k_validate_offsets<<<num_sms * 8, 256, 0, stream>>>(n, nnz, off, flags);
  k_validate_finish<<<1, 1, 0, stream>>>(n, off, nnz, flags, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_validate_edges(int64_t n, int64_t e0, int64_t e1, bool last, const int32_t* nz_row,
                                  const int64_t* nz_pos, int64_t nz_n, const int32_t* col, void* ws, int num_sms,
                                  cudaStream_t stream) {
  unsigned long long* sums = static_cast<unsigned long long*>(ws);
  int* flags = reinterpret_cast<int*>(static_cast<char*>(ws) + align_up(8 * sizeof(unsigned long long)));
  if (e1 > e0)
    k_validate_edges<<<num_sms * 2, kValThreads, 0, stream>>>(n, e0, e1, nz_n, nz_row, nz_pos, col, flags, sums);
  if (last) k_validate_symmetry<<<1, 1, 0, stream>>>(flags, sums);
  return cudaGetLastError();
}

cudaError_t launch_validate_reverse(int64_t nnz, const int64_t* off, const int32_t* nz_row, const int64_t* nz_pos,
                                    int64_t nz_n, const int32_t* col, void* ws, int num_sms, cudaStream_t stream) {
  int* flags = reinterpret_cast<int*>(static_cast<char*>(ws) + align_up(8 * sizeof(unsigned long long)));
  if (nnz > 0) k_validate_reverse<<<num_sms * 2, kValThreads, 0, stream>>>(nz_n, nz_row, nz_pos, nnz, off, col, flags);
  return cudaGetLastError();
}

cudaError_t launch_offsets_i32_to_i64(int64_t n, const int32_t* in, int64_t* out, cudaStream_t stream) {
  const int64_t want = (n + 256) / 256;
  k_off32_to_64<<<(int)(want < 4096 ? want : 4096), 256, 0, stream>>>(n, in, out);
  return cudaGetLastError();
}

size_t nonempty_workspace_bytes(int64_t n) {
  const int64_t ntiles = (n + kNzTile - 1) / kNzTile;
  return align_up(8 * (size_t)(ntiles + 1)) + align_up(8);
}

// nz_row/nz_pos get the non-empty rows and their first CSR positions; the
// count is written to *count_dev (device int64).
cudaError_t launch_nonempty_rows(int64_t n, const int64_t* off, int32_t* nz_row, int64_t* nz_pos, void* ws,
                                 int64_t* count_dev, int num_sms, cudaStream_t stream) {
  if (n <= 0) return cudaMemsetAsync(count_dev, 0, sizeof(int64_t), stream);
  const int64_t ntiles = (n + kNzTile - 1) / kNzTile;
  int64_t* tile = static_cast<int64_t*>(ws);
  const int g = (int)(ntiles < (int64_t)num_sms * 4 ? ntiles : (int64_t)num_sms * 4);
  k_nz_count<<<g, kNzTile, 0, stream>>>(n, off, tile);
  k_nz_scan<<<1, 1024, 0, stream>>>(ntiles, tile, count_dev);
  k_nz_write<<<g, kNzTile, 0, stream>>>(n, off, tile, nz_row, nz_pos);
  return cudaGetLastError();
}

}  // namespace ccg
