// cc_perm.cu -- the random order pi of Alg. 1 / Alg. 2 on the device.
//
// pi lists the vertices by ascending (splitmix64(seed ^ v), v).  The keys are
// uniform 64-bit values, so a two-level sort suffices:
//   1. bucket vertices by the top b key bits (b chosen so a bucket holds about
//      384-768 vertices): a histogram, an exclusive scan and a scatter;
//   2. sort each bucket in shared memory by the full (key, v): a counting sort
//      on the next 10 key bits, then an insertion sort per sub-bucket of
//      about one element, and write its slice of order[].
// Keys are recomputed from v wherever needed instead of being stored, so the
// only global traffic is 4 bytes per vertex scattered and 4+4 bytes per vertex
// read and written by the bucket sort.  A bucket larger than the shared-memory
// capacity (vanishingly unlikely for a hash) falls back to a rank-by-counting
// pass that is slow but exact.
#include <cstdint>

#include "cc_device.cuh"
#include "cc_internal.h"

namespace ccg {
namespace {

constexpr int kBucketCap = 1536;      // vertices per bucket sorted in shared memory
constexpr int kSortThreads = 512;
constexpr int kMaxOverflow = 1023;    // buckets above capacity handled by the fallback

__device__ __forceinline__ uint32_t bucket_of(uint64_t key, int bits) {
  return bits == 0 ? 0u : (uint32_t)(key >> (64 - bits));
}

__global__ void k_bucket_hist(int64_t n, uint64_t seed, int bits, uint32_t* __restrict__ count) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&count[bucket_of(perm_key(seed, (uint64_t)v), bits)], 1u);
}

// Exclusive scan of the nb counts into start[0..nb] (start[nb] = n) and
// cursor = start, in three steps: every block of kScanTile threads scans its
// tile of counts (tile totals to tot[]), one block scans the totals, every
// block adds its tile's offset.
constexpr int kScanTile = 1024;

__global__ void __launch_bounds__(kScanTile) k_scan_tiles(const uint32_t* __restrict__ count, int64_t nb,
                                                        int64_t* __restrict__ start, int64_t* __restrict__ tot) {
  __shared__ int64_t scratch[33];
  const int64_t i = blockIdx.x * (int64_t)kScanTile + threadIdx.x;
  int64_t t;
  const int64_t ex = block_exclusive_sum<int64_t>(i < nb ? (int64_t)count[i] : 0, scratch, &t);
  if (i < nb) start[i] = ex;
  if (threadIdx.x == 0) tot[blockIdx.x] = t;
}

__global__ void k_scan_totals(int64_t ntiles, int64_t nb, int64_t* __restrict__ tot, int64_t* __restrict__ start) {
  __shared__ int64_t scratch[33];
  int64_t run = 0;
  for (int64_t base = 0; base < ntiles; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    int64_t t;
    const int64_t ex = block_exclusive_sum<int64_t>(i < ntiles ? tot[i] : 0, scratch, &t);
    if (i < ntiles) tot[i] = run + ex;
    run += t;
  }
  if (threadIdx.x == 0) start[nb] = run;
}

__global__ void __launch_bounds__(kScanTile) k_scan_add(int64_t nb, const int64_t* __restrict__ tot,
                                                      int64_t* __restrict__ start, uint32_t* __restrict__ cursor) {
  const int64_t i = blockIdx.x * (int64_t)kScanTile + threadIdx.x;
  if (i < nb) {
    const int64_t s = start[i] + tot[blockIdx.x];
    start[i] = s;
    cursor[i] = (uint32_t)s;              // positions are below n < 2^31
  }
}

__global__ void k_bucket_scatter(int64_t n, uint64_t seed, int bits, uint32_t* __restrict__ cursor,
                                 int32_t* __restrict__ tmp) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    uint32_t b = bucket_of(perm_key(seed, (uint64_t)v), bits);
    const int64_t pos = (int64_t)atomicAdd(&cursor[b], 1u);
    tmp[pos] = (int32_t)v;
  }
}

__device__ __forceinline__ bool kv_less(uint64_t ka, int32_t va, uint64_t kb, int32_t vb) {
  return ka < kb || (ka == kb && va < vb);
}

// One block per bucket (grid-stride).  Inside a bucket the keys share their
// top `bits` bits and the next kSubBits bits are still uniform, so a counting
// sort on those bits spreads the bucket over kSub sub-buckets of about one
// element each; one thread then finishes each sub-bucket with an insertion
// sort on the full (key, v).
constexpr int kSubBits = 10;
constexpr int kSub = 1 << kSubBits;
// the sub-bucket counts are scanned two per thread
static_assert(2 * kSortThreads >= kSub, "k_bucket_sort needs 2 * kSortThreads >= kSub");

__global__ void __launch_bounds__(kSortThreads)
k_bucket_sort(uint64_t seed, int bits, int64_t nb, const int64_t* __restrict__ start,
              const int32_t* __restrict__ tmp, int32_t* __restrict__ order, int* __restrict__ overflow) {
  __shared__ uint64_t sk[kBucketCap];
  __shared__ int32_t sv[kBucketCap];
  __shared__ uint64_t ok_[kBucketCap];
  __shared__ int32_t ov[kBucketCap];
  __shared__ int32_t cnt[kSub + 1];
  __shared__ int64_t scr[33];
  const int shift = 64 - bits - kSubBits;
  for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
    const int64_t s0 = start[b], len = start[b + 1] - s0;
    if (len <= 0) continue;
    if (len > kBucketCap) {   // handled by k_bucket_sort_large
      if (threadIdx.x == 0) {
        int slot = atomicAdd(overflow, 1);
        if (slot < kMaxOverflow) overflow[1 + slot] = (int)b;
      }
      continue;
    }
    for (int i = threadIdx.x; i < kSub; i += blockDim.x) cnt[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      const int32_t v = tmp[s0 + i];
      const uint64_t k = perm_key(seed, (uint64_t)v);
      sv[i] = v;
      sk[i] = k;
      atomicAdd(&cnt[(int)((k >> shift) & (kSub - 1))], 1);
    }
    __syncthreads();
    // exclusive scan of the sub-bucket counts (two per thread)
    {
      const int i0 = threadIdx.x * 2;
      const int c0 = i0 < kSub ? cnt[i0] : 0, c1 = i0 + 1 < kSub ? cnt[i0 + 1] : 0;
      int64_t tot;
      const int64_t ex = block_exclusive_sum<int64_t>(c0 + c1, scr, &tot);
      if (i0 < kSub) cnt[i0] = (int)ex;
      if (i0 + 1 < kSub) cnt[i0 + 1] = (int)ex + c0;
      if (threadIdx.x == 0) cnt[kSub] = (int)tot;
    }
    __syncthreads();
    // scatter into sub-buckets (arbitrary order inside a sub-bucket); the
    // counters end at the next sub-bucket's start
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      const uint64_t k = sk[i];
      const int pos = atomicAdd(&cnt[(int)((k >> shift) & (kSub - 1))], 1);
      ok_[pos] = k;
      ov[pos] = sv[i];
    }
    __syncthreads();
    // sub-bucket q now spans [q == 0 ? 0 : cnt[q-1], cnt[q]): insertion sort
    for (int q = threadIdx.x; q < kSub; q += blockDim.x) {
      const int lo = q == 0 ? 0 : cnt[q - 1], hi = cnt[q];
      for (int i = lo + 1; i < hi; ++i) {
        const uint64_t k = ok_[i];
        const int32_t v = ov[i];
        int j = i - 1;
        while (j >= lo && kv_less(k, v, ok_[j], ov[j])) {
          ok_[j + 1] = ok_[j];
          ov[j + 1] = ov[j];
          --j;
        }
        ok_[j + 1] = k;
        ov[j + 1] = v;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) order[s0 + i] = ov[i];
    __syncthreads();
  }
}

// Exact fallback for buckets above kBucketCap: each element's position is the
// number of bucket elements smaller than it.
__global__ void k_bucket_sort_large(uint64_t seed, const int* __restrict__ overflow,
                                    const int64_t* __restrict__ start, const int32_t* __restrict__ tmp,
                                    int32_t* __restrict__ order, int* __restrict__ err) {
  const int cnt = overflow[0];
  if (cnt > kMaxOverflow) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(err, kOk, kErrInternal);
    return;
  }
  for (int q = 0; q < cnt; ++q) {
    const int64_t b = overflow[1 + q];
    const int64_t s0 = start[b], len = start[b + 1] - s0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len;
         i += (int64_t)gridDim.x * blockDim.x) {
      const int32_t vi = tmp[s0 + i];
      const uint64_t ki = perm_key(seed, (uint64_t)vi);
      int64_t r = 0;
      for (int64_t j = 0; j < len; ++j) {
        const int32_t vj = tmp[s0 + j];
        r += kv_less(perm_key(seed, (uint64_t)vj), vj, ki, vi) ? 1 : 0;
      }
      order[s0 + r] = vi;
    }
  }
}

}  // namespace

int perm_bucket_bits(int64_t n) {
  int bits = 0;
  while (bits < 40 && (n >> bits) > 768) ++bits;
  return bits;
}

size_t perm_workspace_bytes(int64_t n) {
  const int64_t nb = int64_t(1) << perm_bucket_bits(n);
  return align_up(sizeof(uint32_t) * nb) + align_up(sizeof(int64_t) * (nb + 1)) +
         align_up(sizeof(int64_t) * nb) + align_up(sizeof(int32_t) * (n > 0 ? n : 1)) +
         align_up(sizeof(int) * (kMaxOverflow + 1)) + align_up(sizeof(int64_t) * ((nb + kScanTile - 1) / kScanTile));
}

// order[0..n) = pi for `seed`.  ws must hold perm_workspace_bytes(n).  A
// failed device-side check is reported through *err.
cudaError_t launch_permutation(int64_t n, uint64_t seed, int32_t* order, void* ws, int num_sms,
                               int* err, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int bits = perm_bucket_bits(n);
  const int64_t nb = int64_t(1) << bits;
  char* p = static_cast<char*>(ws);
  uint32_t* count = reinterpret_cast<uint32_t*>(p); p += align_up(sizeof(uint32_t) * nb);
  int64_t* start = reinterpret_cast<int64_t*>(p);   p += align_up(sizeof(int64_t) * (nb + 1));
  uint32_t* cursor = reinterpret_cast<uint32_t*>(p); p += align_up(sizeof(int64_t) * nb);
  int32_t* tmp = reinterpret_cast<int32_t*>(p);     p += align_up(sizeof(int32_t) * n);
  int* overflow = reinterpret_cast<int*>(p);         p += align_up(sizeof(int) * (kMaxOverflow + 1));
  int64_t* tot = reinterpret_cast<int64_t*>(p);
  const int64_t stiles = (nb + kScanTile - 1) / kScanTile;
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(uint32_t) * nb, stream);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(overflow, 0, sizeof(int), stream);
  if (e != cudaSuccess) return e;
  const int64_t want = (n + 255) / 256;
  const int grid = (int)(want < (int64_t)num_sms * 8 ? want : (int64_t)num_sms * 8);
  k_bucket_hist<<<grid, 256, 0, stream>>>(n, seed, bits, count);
  k_scan_tiles<<<(unsigned)stiles, kScanTile, 0, stream>>>(count, nb, start, tot);
  k_scan_totals<<<1, 1024, 0, stream>>>(stiles, nb, tot, start);
  k_scan_add<<<(unsigned)stiles, kScanTile, 0, stream>>>(nb, tot, start, cursor);
  k_bucket_scatter<<<grid, 256, 0, stream>>>(n, seed, bits, cursor, tmp);
  const int sgrid = (int)(nb < (int64_t)num_sms * 4 ? nb : (int64_t)num_sms * 4);
  k_bucket_sort<<<sgrid, kSortThreads, 0, stream>>>(seed, bits, nb, start, tmp, order, overflow);
  // The fallback kernel returns at once when no bucket overflowed, so it
  // always runs; this keeps the host free of a sync.
  k_bucket_sort_large<<<num_sms, 256, 0, stream>>>(seed, overflow, start, tmp, order, err);
  return cudaGetLastError();
}

}  // namespace ccg
