// cc_async.cu -- C4 without rounds: the asynchronous execution of Alg. 3 with
// attemptCluster (the concurrency control of C4).
//
// Vertices are taken in pi order and nothing separates them into rounds.  A
// vertex v is a cluster center iff none of its earlier-ranked neighbours is a
// center (the serial KwikCluster rule, which C4 preserves by Sec. 4's
// serializability argument); a non-center joins the earliest-ranked center
// among its neighbours.  On the GPU:
//
//   k_async_init      rank = pi^-1, labels "none", decisions "undecided".
//   k_async_decide    one persistent cooperative launch; warp w decides the
//                     vertices of rank w, w + W, w + 2W, ... (W warps, numbered
//                     across the blocks first).  A vertex that an earlier
//                     center already attached is a non-center at once;
//                     otherwise the warp reads its row: an earlier neighbour
//                     that is a center decides "non-center", an undecided
//                     earlier neighbour is waited for (isCenter's wait), and a
//                     row with neither decides "center".  A center pushes its
//                     rank to its neighbours with atomicMin (createCluster) at
//                     once when its row is short, else it is queued.
//   k_async_push_long the queued centers' rows, edge-balanced.
//   k_async_labels    labels[v] = pi(label rank of v).
//
// Waits only go to strictly earlier ranks, whose warps are resident (the
// launch is cooperative): the smallest undecided rank never waits, so every
// wait ends.  Each wait is still bounded (kBarrierLimitNs, then kErrTimeout).
// A push reaches only non-centers: an earlier neighbour was decided before the
// center (the center waited for it), a later one is a non-center because of
// this center.  So a vertex found already attached is a non-center, no center
// is ever pushed to, and the final label of a non-center is the smallest rank
// among its center neighbours, which is the KwikCluster label.
#include <cstdint>

#include "cc_async.h"
#include "cc_device.cuh"

namespace ccg {
namespace {

constexpr int kAThreads = 256;
constexpr int kAK = 4;                        // adjacency entries per lane per step
constexpr int64_t kEagerMax = 4096;           // centers with longer rows push after the decisions
constexpr uint32_t kNone = 0xFFFFFFFFu;       // no center rank yet
constexpr uint32_t kUndecided = 0, kCenter = 1, kNonCenter = 2;

__device__ __forceinline__ uint32_t ld_volatile_u8(const uint8_t* p) {
  return *reinterpret_cast<const volatile uint8_t*>(p);
}
__device__ __forceinline__ void st_volatile_u8(uint8_t* p, uint32_t v) {
  *reinterpret_cast<volatile uint8_t*>(p) = (uint8_t)v;
}
__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}

// rank[order[r]] = r; label[v] = none; decision[v] = undecided.  An entry
// of order outside [0, n) (a failed permutation) is reported, not used.
__global__ void k_async_init(const __grid_constant__ RoundBuffers B) {
  const int64_t n = B.n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    B.st[i] = kNone;
    B.blk_flag[i] = (uint8_t)kUndecided;
    const int32_t v = __ldg(B.order + i);
    if (v < 0 || v >= n) {
      atomicCAS(&B.ctl->err, kOk, kErrInternal);
      continue;
    }
    B.arank[v] = (int32_t)i;
  }
}

__global__ void __launch_bounds__(kAThreads) k_async_decide(const __grid_constant__ RoundBuffers B) {
  __shared__ unsigned long long tal[4];
  if (threadIdx.x < 4) tal[threadIdx.x] = 0;
  __syncthreads();
  Ctl* const C = B.ctl;
  uint32_t* const label = B.st;
  uint8_t* const decision = B.blk_flag;
  const int lane = threadIdx.x & 31;
  const int64_t n = B.n;
  const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long centers = 0, noncenters = 0, blocked = 0, scanned = 0;
  bool abort = ld_volatile_int(&C->err) != kOk;
  for (int64_t r = (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x; r < n && !abort; r += W) {
    const int32_t v = __ldg(B.order + r);
    if (v < 0 || v >= n) break;                          // reported by k_async_init
    if (ld_volatile_u32(label + v) != kNone) {          // attached by an earlier center
      if (lane == 0) st_volatile_u8(decision + v, kNonCenter);
      noncenters += lane == 0;
      continue;
    }
    const int64_t row = __ldg(B.off + v), len = __ldg(B.off + v + 1) - row;
    bool center = true, waited = false;
    for (int64_t base = 0; base < len; base += 32 * kAK) {
      int32_t u[kAK];
#pragma unroll
      for (int t = 0; t < kAK; ++t) {
        const int64_t e = base + lane + 32 * t;
        u[t] = e < len ? __ldg(B.col + row + e) : -1;
      }
      // the decision of each earlier neighbour (later ones do not matter)
      uint32_t s[kAK];
#pragma unroll
      for (int t = 0; t < kAK; ++t) {
        const bool earlier = u[t] >= 0 && (int64_t)__ldg(B.arank + u[t]) < r;
        s[t] = earlier ? ld_volatile_u8(decision + u[t]) : kNonCenter;
      }
      if (lane == 0) scanned += (unsigned long long)(len - base < 32 * kAK ? len - base : 32 * kAK);
      bool hit = false, pend = false;
#pragma unroll
      for (int t = 0; t < kAK; ++t) {
        hit |= s[t] == kCenter;
        pend |= s[t] == kUndecided;
      }
      if (__any_sync(FULL, hit)) { center = false; break; }
      if (!__any_sync(FULL, pend)) continue;
      // isCenter: wait for the undecided earlier neighbours of this step
      waited = true;
      bool gave_up = false;
      const uint64_t t0 = globaltimer_ns();
#pragma unroll
      for (int t = 0; t < kAK; ++t) {
        unsigned spins = 0;
        while (s[t] == kUndecided && !gave_up) {
          if ((++spins & 63) == 0 &&
              (ld_volatile_int(&C->err) != kOk || globaltimer_ns() - t0 > kBarrierLimitNs)) {
            atomicCAS(&C->err, kOk, kErrTimeout);
            gave_up = true;
            break;
          }
          s[t] = ld_volatile_u8(decision + u[t]);
        }
        hit |= s[t] == kCenter;
      }
      if (__any_sync(FULL, gave_up)) { abort = true; break; }
      if (__any_sync(FULL, hit)) { center = false; break; }
    }
    if (abort) break;
    if (lane == 0) {
      if (center) label[v] = (uint32_t)r;
      st_volatile_u8(decision + v, center ? kCenter : kNonCenter);
    }
    blocked += lane == 0 && waited;
    if (!center) {
      noncenters += lane == 0;
      continue;
    }
    centers += lane == 0;
    // createCluster: push this center's rank to its neighbours
    if (len <= kEagerMax) {
      for (int64_t base = 0; base < len; base += 32 * kAK) {
#pragma unroll
        for (int t = 0; t < kAK; ++t) {
          const int64_t e = base + lane + 32 * t;
          if (e < len) atomicMin(label + __ldg(B.col + row + e), (uint32_t)r);
        }
      }
    } else if (lane == 0) {
      const unsigned long long old = atomicAdd(&C->act_pack, (1ull << kPackShift) | (unsigned long long)len);
      const int64_t j = (int64_t)(old >> kPackShift), ep = (int64_t)(old & kPackEdgeMask);
      B.act_v[j] = v;
      B.act_r[j] = (int32_t)r;
      B.act_e[j] = ep;
      B.act_d[j] = row - ep;
    }
  }
  if (lane == 0) {
    if (centers) atomicAdd(&tal[0], centers);
    if (noncenters) atomicAdd(&tal[1], noncenters);
    if (blocked) atomicAdd(&tal[2], blocked);
    if (scanned) atomicAdd(&tal[3], scanned);
  }
  __syncthreads();
  if (threadIdx.x < 4 && tal[threadIdx.x]) {
    long long* dst = threadIdx.x == 0 ? &C->r_centers
                   : threadIdx.x == 1 ? &C->r_noncenter
                   : threadIdx.x == 2 ? &C->r_blocked
                                      : &C->r_attached;
    atomicAdd(reinterpret_cast<unsigned long long*>(dst), tal[threadIdx.x]);
  }
}

// The queued (long-row) centers push their ranks, edge-balanced.
__global__ void __launch_bounds__(kAThreads) k_async_push_long(const __grid_constant__ RoundBuffers B) {
  __shared__ LbsWarp ws[kAThreads / 32];
  const unsigned long long pk = ldcg(&B.ctl->act_pack);
  const int64_t items = (int64_t)(pk >> kPackShift), E = (int64_t)(pk & kPackEdgeMask);
  lbs_for_each(B.act_e, items, E, &ws[threadIdx.x >> 5], [&](const Lbs& L) {
#pragma unroll
    for (int t = 0; t < kLbsK; ++t)
      if (L.ok(t)) atomicMin(B.st + __ldg(B.col + L.csr(t)), (uint32_t)L.vtx(t));
  }, B.act_d, B.act_r);
}

// labels[v] = order[label rank of v]; a vertex without a center is an error
__global__ void k_async_labels(const __grid_constant__ RoundBuffers B, int32_t* __restrict__ labels) {
  const int64_t n = B.n;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t x = B.st[v];
    if ((int64_t)x >= n) {
      atomicCAS(&B.ctl->err, kOk, kErrInternal);
      labels[v] = -1;
      continue;
    }
    labels[v] = __ldg(B.order + x);
  }
}

}  // namespace

int async_grid_size(int device) {
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_async_decide, kAThreads, 0);
  if (per < 1) per = 1;
  return sms * per;
}

cudaError_t launch_async_c4(const RoundBuffers& b, int grid, int32_t* labels, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(b.ctl, 0, sizeof(Ctl), stream);
  if (e != cudaSuccess || b.n <= 0) return e;
  k_async_init<<<grid, kAThreads, 0, stream>>>(b);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  RoundBuffers arg = b;
  void* args[] = {&arg};
  e = cudaLaunchCooperativeKernel((const void*)k_async_decide, dim3(grid), dim3(kAThreads), args, 0, stream);
  if (e != cudaSuccess) return e;
  k_async_push_long<<<grid, kAThreads, 0, stream>>>(b);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_async_labels<<<grid, kAThreads, 0, stream>>>(b, labels);
  return cudaGetLastError();
}

}  // namespace ccg
