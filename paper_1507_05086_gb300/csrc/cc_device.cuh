// cc_device.cuh -- device-side building blocks shared by the library's kernels:
// the permutation hash, a grid barrier with a bounded wait, warp/block scans
// and the edge-balanced list walker used by every adjacency pass.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ccg {

constexpr unsigned FULL = 0xFFFFFFFFu;

// Status codes, mirrored from include/cc.h.
constexpr int kOk = 0;
constexpr int kErrTimeout = -5;
constexpr int kErrInternal = -7;

// ---------------------------------------------------------------------------
// Permutation hash: the SplitMix64 output function (Steele, Lea & Flood,
// OOPSLA 2014) applied to seed ^ v.  pi orders vertices by (key, v).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t perm_key(uint64_t seed, uint64_t v) {
  uint64_t z = (seed ^ v) + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// ---------------------------------------------------------------------------
// Memory access helpers.  Data that other blocks of the same persistent
// kernel write is read at L2 (ld.cg); L1 is not coherent across SMs.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T ldcg(const T* p) { return __ldcg(p); }

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_int(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// Grid barrier for a cooperative (co-resident) launch.  The last block to
// arrive may run a "leader" step with the whole block before releasing the
// others.  Every wait is bounded: after kBarrierLimitNs the waiter records
// kErrTimeout in *err and returns false, and the kernel unwinds.
// ---------------------------------------------------------------------------
constexpr uint64_t kBarrierLimitNs = 4000000000ull;   // 4 s

struct GridBarrier {
  unsigned count;
  unsigned gen;
};

// Phase 1: arrive.  Returns true in every thread of the block that arrived
// last.  *gen_out (shared) receives the generation to wait on.
__device__ __forceinline__ bool bar_arrive(GridBarrier* b, unsigned nblocks, unsigned* s_gen,
                                           int* s_leader) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned g = ld_acquire(&b->gen);
    __threadfence();
    unsigned t = atomicAdd(&b->count, 1u);
    *s_gen = g;
    *s_leader = (t == nblocks - 1) ? 1 : 0;
  }
  __syncthreads();
  return *s_leader != 0;
}

// Phase 2: the leader releases; everyone else waits (bounded).
__device__ __forceinline__ bool bar_finish(GridBarrier* b, bool leader, unsigned* s_gen, int* err,
                                           int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (leader) {
      b->count = 0;
      __threadfence();
      st_release(&b->gen, *s_gen + 1);
    } else {
      uint64_t t0 = globaltimer_ns();
      unsigned spins = 0;
      while (ld_acquire(&b->gen) == *s_gen) {
        if (ld_volatile_int(err) != kOk) { ok = 0; break; }
        if (++spins > 64) __nanosleep(128);
        if ((spins & 255) == 0 && globaltimer_ns() - t0 > kBarrierLimitNs) {
          atomicCAS(err, kOk, kErrTimeout);
          ok = 0;
          break;
        }
      }
      __threadfence();
    }
    if (ld_volatile_int(err) != kOk) ok = 0;
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// ---------------------------------------------------------------------------
// Scans
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T warp_inclusive_sum(T x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

template <class T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  return x;
}

template <class T>
__device__ __forceinline__ T warp_max(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T y = __shfl_xor_sync(FULL, x, o);
    x = y > x ? y : x;
  }
  return x;
}

// Block-wide exclusive sum; *total receives the block total.  scratch must
// hold 33 elements.  All threads of the block must call it.
template <class T>
__device__ __forceinline__ T block_exclusive_sum(T x, T* scratch, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  T inc = warp_inclusive_sum(x);
  __syncthreads();
  if (lane == 31) scratch[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    T w = lane < nwarps ? scratch[lane] : T(0);
    T wi = warp_inclusive_sum(w);
    scratch[lane] = wi - w;
    if (lane == 31) scratch[32] = wi;   // lane 31 holds the grand total
  }
  __syncthreads();
  T res = scratch[warp] + inc - x;
  *total = scratch[32];
  __syncthreads();
  return res;
}

template <class T>
__device__ __forceinline__ T block_sum(T x, T* scratch) {
  T tot;
  block_exclusive_sum(x, scratch, &tot);
  return tot;
}

template <class T>
__device__ __forceinline__ T block_max(T x, T* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  x = warp_max(x);
  __syncthreads();
  if (lane == 0) scratch[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T w = lane < nwarps ? scratch[lane] : scratch[0];
    w = warp_max(w);
    if (lane == 0) scratch[0] = w;
  }
  __syncthreads();
  T r = scratch[0];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// Edge-balanced walk over a list of adjacency rows.
//
// Item j of the list owns the virtual edges [epos[j], epos[j+1]) (epos[j] is
// non-decreasing in j and every item owns at least one edge); E is the total.
// Every warp of the grid takes chunks of kLbsChunk consecutive virtual edges,
// so a hub row is spread over many warps and short rows are packed together.
// f(valid, j, k) is called by all 32 lanes of a warp together for each step of
// 32 edges, with k the edge's index inside item j's row; lanes with
// valid == false must do nothing but take part in warp collectives.
// ---------------------------------------------------------------------------
constexpr int kLbsSteps = 8;
constexpr int64_t kLbsChunk = 32 * kLbsSteps;

__device__ __forceinline__ int64_t upper_bound_i64(const int64_t* a, int64_t n, int64_t x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (ldcg(a + mid) <= x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

template <class F>
__device__ __forceinline__ void lbs_for_each(const int64_t* epos, int64_t nitems, int64_t E,
                                             int* warp_buf /* 32 ints for this warp */, F&& f) {
  if (E <= 0) return;
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t base0 = gwarp * kLbsChunk; base0 < E; base0 += nwarps * kLbsChunk) {
    int64_t j0 = 0;
    if (lane == 0) j0 = upper_bound_i64(epos, nitems, base0) - 1;
    j0 = __shfl_sync(FULL, j0, 0);
    const int64_t end = base0 + kLbsChunk < E ? base0 + kLbsChunk : E;
    for (int64_t base = base0; base < end; base += 32) {
      const int64_t jj = j0 + lane;
      const int64_t s = jj < nitems ? ldcg(epos + jj) : INT64_MAX;
      warp_buf[lane] = -1;
      __syncwarp();
      if (s >= base && s < base + 32) warp_buf[s - base] = lane;
      __syncwarp();
      int t = warp_buf[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL, t, o);
        if (lane >= o) t = y > t ? y : t;
      }
      if (t < 0) t = 0;
      const int64_t sj = __shfl_sync(FULL, s, t);
      const int64_t e = base + lane;
      f(e < end, j0 + t, e - sj);
      j0 += __shfl_sync(FULL, t, 31);
      __syncwarp();
    }
  }
}

// Warp-aggregated append to a list whose counter packs (items << 33 | edges).
// Lanes with want == true add one item of `edges` edges; the function returns
// (item index, first edge) for those lanes.  All 32 lanes must call it.
constexpr int kPackShift = 33;
constexpr uint64_t kPackEdgeMask = (1ull << kPackShift) - 1;

__device__ __forceinline__ void warp_append_packed(bool want, int64_t edges, unsigned long long* counter,
                                                   int64_t* item_out, int64_t* epos_out) {
  const int lane = threadIdx.x & 31;
  const unsigned mask = __ballot_sync(FULL, want);
  if (mask == 0) return;
  const int64_t ex = warp_inclusive_sum<int64_t>(want ? edges : 0) - (want ? edges : 0);
  const int64_t tot = __shfl_sync(FULL, ex + (want ? edges : 0), 31);
  const int leader = __ffs(mask) - 1;
  unsigned long long old = 0;
  if (lane == leader)
    old = atomicAdd(counter, ((unsigned long long)__popc(mask) << kPackShift) | (unsigned long long)tot);
  old = __shfl_sync(FULL, old, leader);
  if (want) {
    *item_out = (int64_t)(old >> kPackShift) + __popc(mask & ((1u << lane) - 1u));
    *epos_out = (int64_t)(old & kPackEdgeMask) + ex;
  }
}

}  // namespace ccg
