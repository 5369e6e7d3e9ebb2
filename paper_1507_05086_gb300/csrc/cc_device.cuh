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
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_volatile_int(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounds checks of the debug build (nvcc -DCC_DEBUG; build(debug=True)): an
// index outside [0, cap) records CC_ERR_INTERNAL in the kernel's error word
// and the access is skipped, so a bookkeeping mistake reports an error
// instead of touching memory out of range.  Release builds compile the
// checks away.
#ifdef CC_DEBUG
constexpr bool kDebugChecks = true;
#else
constexpr bool kDebugChecks = false;
#endif
__device__ __forceinline__ bool in_bounds(int64_t i, int64_t cap, int* err) {
  if (!kDebugChecks) return true;
  if (i >= 0 && i < cap) return true;
  if (err) atomicCAS(err, kOk, kErrInternal);
  return false;
}
// The checks as written at the access sites: in release builds the macro is
// the constant true and its arguments are not compiled at all, so the kernels
// are the same code as without the checks (register allocation included).
#ifdef CC_DEBUG
#define CC_IN_BOUNDS(i, cap, err) in_bounds((i), (cap), (err))
#define CC_ROWLIST_CHECK(cap, err) , (cap), (err)
#else
#define CC_IN_BOUNDS(i, cap, err) true
#define CC_ROWLIST_CHECK(cap, err)
#endif

// Every spin-wait of the kernels is bounded: after kBarrierLimitNs the waiter
// records kErrTimeout in the error word and the kernel unwinds.
constexpr uint64_t kBarrierLimitNs = 4000000000ull;   // 4 s

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

__device__ __forceinline__ int32_t warp_min_i32(int32_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int32_t y = __shfl_xor_sync(FULL, x, o);
    x = y < x ? y : x;
  }
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
// Warps take chunks of kLbsBatches * kLbsW consecutive virtual edges, so a hub
// row is spread over many warps and short rows are packed together.  Within a
// chunk a warp handles kLbsW = 32 * kLbsK edges at a time: each lane gets kLbsK
// edges (e = base + lane + 32 t), so kLbsK independent loads per lane are in
// flight instead of one.  f(L) receives an Lbs view of the batch (item, virtual
// edge and position in the item of each of the lane's edges); all 32 lanes
// call f together (edges with L.ok(t) == false must be skipped, but their
// lanes still take part in warp collectives).
// ---------------------------------------------------------------------------
constexpr int kLbsK = 4;
#ifndef CC_LBS_PF_AHEAD
#define CC_LBS_PF_AHEAD 2
#endif
constexpr int kLbsPfAhead = CC_LBS_PF_AHEAD;   // batches of a long row prefetched into L2 ahead

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
constexpr int kLbsW = 32 * kLbsK;
#ifndef CC_LBS_BATCHES
#define CC_LBS_BATCHES 4
#endif
constexpr int kLbsBatches = CC_LBS_BATCHES;   // batches per chunk of a long walk

// Run-time shape of a walk (the defaults above unless a tuning says
// otherwise): batches per chunk (1..8) and batches of a long row prefetched
// ahead (0..8).  Neither changes what a walk visits, only its schedule.
struct WalkShape {
  int batches = kLbsBatches;
  int pf_ahead = kLbsPfAhead;
};

struct LbsWarp {
  int32_t mark[kLbsW];   // relative item index per position
  int32_t rel[kLbsW];    // item start relative to the batch base
  int64_t dlt[kLbsW];    // per-item CSR delta (prefetched when given)
  int32_t vtx[kLbsW];    // per-item vertex or payload (prefetched when given)
  int32_t next;          // relative index of the item starting the next batch
  int32_t pad;
};

// One batch of kLbsW virtual edges as seen by one lane.
struct Lbs {
  int64_t j0, base;
  const LbsWarp* ws;
  int32_t ri[kLbsK];
  unsigned valid;
  __device__ __forceinline__ bool ok(int t) const { return (valid >> t) & 1u; }
  __device__ __forceinline__ int64_t item(int t) const { return j0 + ri[t]; }
  __device__ __forceinline__ int64_t edge(int t) const { return base + (threadIdx.x & 31) + 32 * t; }
  // index of the edge inside its item's row
  __device__ __forceinline__ int64_t in_row(int t) const {
    return (int64_t)((threadIdx.x & 31) + 32 * t) - ws->rel[ri[t]];
  }
  // prefetched per-item data (only when the walk was given the arrays)
  __device__ __forceinline__ int64_t csr(int t) const { return edge(t) + ws->dlt[ri[t]]; }
  __device__ __forceinline__ int32_t vtx(int t) const { return ws->vtx[ri[t]]; }
};

// Number of elements of the sorted array a[0..n) that are <= x, by a 33-ary
// search of the whole warp (about log_33(n) dependent loads).
__device__ __forceinline__ int64_t warp_upper_bound(const int64_t* a, int64_t n, int64_t x) {
  const int lane = threadIdx.x & 31;
  int64_t lo = 0, hi = n;
  while (hi - lo > 32) {
    const int64_t span = hi - lo;
    const int64_t p = lo + (span * (lane + 1)) / 33;
    const unsigned b = __ballot_sync(FULL, ldcg(a + p) <= x);
    const int c = __popc(b);
    const int64_t pp = __shfl_sync(FULL, p, c > 0 ? c - 1 : 0);
    const int64_t pn = __shfl_sync(FULL, p, c < 32 ? c : 31);
    lo = c > 0 ? pp + 1 : lo;
    hi = c < 32 ? pn : hi;
  }
  const int64_t p = lo + lane;
  const bool le = p < hi && ldcg(a + p) <= x;
  return lo + __popc(__ballot_sync(FULL, le));
}

// One chunk [c0, cend) of the walk: find the item holding c0, then batches
// of kLbsW virtual edges.  A batch that lies inside one item (a long row)
// needs none of the per-item loads: the warp keeps the range, delta and
// vertex of its current item, taken from the previous batch's loads, and
// only a batch that crosses an item boundary loads and scans item starts,
// in groups of 32 items: a group is loaded only while the previous one ends
// inside the batch, so a batch spanning a few rows costs one group, not
// kLbsK (every item owns at least one edge, so kLbsK groups always suffice,
// and the item after the batch's last one is always among those loaded).
// With vmap, the per-item payload is vmap[vtx[j]] - vsub instead of vtx[j]
// (one load per item, not per edge).
//
// With colp (the CSR column array; the walk's CSR position of virtual edge e
// of item j is e + delta[j], or e without delta), the column ids of the
// batch kLbsPfAhead ahead in the current row are prefetched into L2, so a
// long row streams from DRAM ahead of its use.  E: the walk's end.
template <class F>
__device__ __forceinline__ void lbs_chunk(const int64_t* epos, int64_t nitems, int64_t c0, int64_t cend, LbsWarp* ws,
                                          F& f, const int64_t* delta, const int32_t* vtx,
                                          const uint32_t* vmap = nullptr, uint32_t vsub = 0,
                                          const int32_t* colp = nullptr, int64_t E = 0, int pf_ahead = kLbsPfAhead) {
  const int lane = threadIdx.x & 31;
  int64_t j0 = warp_upper_bound(epos, nitems, c0) - 1;
  // cached item (warp-uniform): valid when cur_j == j0
  int64_t cur_j = -1, cur_start = 0, cur_end = 0, cur_dlt = 0;
  int32_t cur_vtx = 0;
  for (int64_t base = c0; base < cend; base += kLbsW) {
    Lbs L;
    L.j0 = j0;
    L.base = base;
    L.ws = ws;
    L.valid = 0;
    if (cur_j == j0 && cur_end >= base + kLbsW) {
      // the whole batch belongs to item j0
      if (lane == 0) {
        ws->rel[0] = (int32_t)(cur_start - base);
        ws->dlt[0] = cur_dlt;
        ws->vtx[0] = cur_vtx;
      }
      __syncwarp();
#pragma unroll
      for (int t = 0; t < kLbsK; ++t) {
        L.ri[t] = 0;
        if (base + lane + 32 * t < cend) L.valid |= 1u << t;
      }
      if (colp && pf_ahead > 0 && lane < kLbsW / 32) {
        const int64_t pe = base + (int64_t)pf_ahead * kLbsW + 32 * lane;
        if (pe < cur_end && pe < E) prefetch_l2(colp + pe + cur_dlt);
      }
      f(L);
      __syncwarp();
      if (cur_end == base + kLbsW) ++j0;          // the next batch starts the next item
      continue;
    }
    int64_t s[kLbsK];
#pragma unroll
    for (int t = 0; t < kLbsK; ++t) {
      s[t] = INT64_MAX;
      ws->mark[lane + 32 * t] = -1;
    }
#pragma unroll
    for (int t = 0; t < kLbsK; ++t) {
      // a group of 32 items is needed while the previous group's last item
      // starts inside the batch or at its end
      if (t > 0 && __shfl_sync(FULL, s[t - 1], 31) > base + kLbsW) break;
      const int64_t jj = j0 + lane + 32 * t;
      const bool in = jj < nitems;
      s[t] = in ? ldcg(epos + jj) : INT64_MAX;
      // per-item data loads issue together with the start offsets
      if (delta) ws->dlt[lane + 32 * t] = in ? ldcg(delta + jj) : 0;
      if (vtx) ws->vtx[lane + 32 * t] = in ? ldcg(vtx + jj) : 0;
    }
    if (lane == 0) ws->next = -1;
    __syncwarp();
    if (vmap) {
      // payload of the items that own edges of this batch, and of the one
      // that starts the next batch (it may be kept for that batch)
#pragma unroll
      for (int t = 0; t < kLbsK; ++t) {
        const int i = lane + 32 * t;
        if (s[t] <= base + kLbsW) ws->vtx[i] = (int32_t)(ldcg(vmap + ws->vtx[i]) - vsub);
      }
    }
#pragma unroll
    for (int t = 0; t < kLbsK; ++t) {
      const int i = lane + 32 * t;
      // start relative to the batch, clamped to int32 (items past the end of
      // the list, or starting 2^31 edges later, read as INT32_MAX)
      const int64_t r = s[t] - base;
      ws->rel[i] = s[t] == INT64_MAX || r > INT32_MAX - 1 ? INT32_MAX : (int32_t)r;
      if (s[t] < base + kLbsW) {
        if (s[t] >= base) ws->mark[s[t] - base] = i;
      } else if (s[t] == base + kLbsW) {
        ws->next = i;                  // the item that starts the next batch
      }
    }
    __syncwarp();
    // segmented max-scan: each position takes the last item starting at or before it
    int v[kLbsK];
    int run = -1;
#pragma unroll
    for (int t = 0; t < kLbsK; ++t) {
      const int m = ws->mark[lane * kLbsK + t];
      run = m > run ? m : run;
      v[t] = run;
    }
    int inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, inc, o);
      if (lane >= o) inc = y > inc ? y : inc;
    }
    int exc = __shfl_up_sync(FULL, inc, 1);
    if (lane == 0) exc = -1;
    __syncwarp();
#pragma unroll
    for (int t = 0; t < kLbsK; ++t) {
      int m = v[t] > exc ? v[t] : exc;
      ws->mark[lane * kLbsK + t] = m < 0 ? 0 : m;
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < kLbsK; ++t) {
      const int p = lane + 32 * t;
      L.ri[t] = ws->mark[p];
      if (base + p < cend) L.valid |= 1u << t;
    }
    const int last = ws->mark[kLbsW - 1];
    const int nxt = ws->next;
    // next batch: the item holding its first edge is the last item of this
    // batch or, when an item starts exactly at the next base, that item (the
    // item after `last` is always among the ones loaded here unless `last`
    // is the final loaded slot, in which case one load decides)
    int m = nxt >= 0 ? nxt : last;
    if (nxt < 0 && last == kLbsW - 1 && j0 + kLbsW < nitems && ldcg(epos + j0 + kLbsW) <= base + kLbsW) m = kLbsW;
    // remember the next batch's item when its range is among the loaded ones
    if (m + 1 < kLbsW) {
      const int32_t r1 = ws->rel[m + 1];
      cur_j = j0 + m;
      cur_start = base + ws->rel[m];
      cur_end = r1 == INT32_MAX ? INT64_MAX : base + r1;
      cur_dlt = delta ? ws->dlt[m] : 0;
      cur_vtx = vtx ? ws->vtx[m] : 0;
      // the next batches of that item: start streaming them
      if (colp) {
        for (int a = 1; a <= pf_ahead; ++a) {
          const int64_t pe = base + (int64_t)a * kLbsW + 32 * lane;
          if (lane < kLbsW / 32 && pe >= cur_start && pe < cur_end && pe < E) prefetch_l2(colp + pe + cur_dlt);
        }
      }
    }
    f(L);
    __syncwarp();
    j0 += m;
  }
}

// gwarp / nwarps: this warp's index among, and the number of, the warps that
// share the walk (the whole grid, or one team of blocks).  The walk covers
// the virtual edges [E0, E); warp w takes chunks w, w + nwarps, ...
template <class F>
__device__ __forceinline__ void lbs_for_each_in(int64_t gwarp, int64_t nwarps, const int64_t* epos, int64_t nitems,
                                                int64_t E, LbsWarp* ws, F&& f, const int64_t* delta = nullptr,
                                                const int32_t* vtx = nullptr, int64_t E0 = 0,
                                                const uint32_t* vmap = nullptr, uint32_t vsub = 0,
                                                const int32_t* colp = nullptr, WalkShape shape = WalkShape{}) {
  if (E <= E0) return;
  // up to shape.batches batches per chunk, fewer when the list is short, so
  // that short lists still spread over many warps
  int64_t nb = (E - E0) / (nwarps * (int64_t)kLbsW * 2);
  nb = nb < 1 ? 1 : (nb > shape.batches ? shape.batches : nb);
  const int64_t kChunk = (int64_t)kLbsW * nb;
  for (int64_t c0 = E0 + gwarp * kChunk; c0 < E; c0 += nwarps * kChunk)
    lbs_chunk(epos, nitems, c0, c0 + kChunk < E ? c0 + kChunk : E, ws, f, delta, vtx, vmap, vsub, colp, E,
              shape.pf_ahead);
}

template <class F>
__device__ __forceinline__ void lbs_for_each(const int64_t* epos, int64_t nitems, int64_t E, LbsWarp* ws, F&& f,
                                             const int64_t* delta = nullptr, const int32_t* vtx = nullptr,
                                             int64_t E0 = 0, const int32_t* colp = nullptr) {
  lbs_for_each_in(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5, ((int64_t)gridDim.x * blockDim.x) >> 5,
                  epos, nitems, E, ws, f, delta, vtx, E0, nullptr, 0, colp);
}

// Lists of adjacency rows.  A list counter packs (items << 33 | edges): one
// atomicAdd hands out an item index and the item's first virtual edge, so
// epos stays non-decreasing in the item index.  For every item the list keeps
// its vertex, epos and delta = (CSR row start) - epos, so the CSR position of
// virtual edge e of item j is e + delta[j].
constexpr int kPackShift = 33;
constexpr uint64_t kPackEdgeMask = (1ull << kPackShift) - 1;

struct RowList {
  int32_t* v;
  int64_t* epos;
  int64_t* delta;
  int32_t* aux;                 // optional per-item payload (may be null)
  unsigned long long* counter;  // packed (items << 33 | edges)
#ifdef CC_DEBUG
  int64_t cap;                  // items the arrays hold
  int* err;                     // error word for a failed check
#endif
};

// Warp-aggregated append of one item per lane with want == true.  All 32
// lanes must call it.
__device__ __forceinline__ void warp_append_rows(bool want, int32_t v, int64_t row, int64_t edges, int32_t aux,
                                                 const RowList& L) {
  const int lane = threadIdx.x & 31;
  const unsigned mask = __ballot_sync(FULL, want);
  if (mask == 0) return;
  const int64_t mine = want ? edges : 0;
  const int64_t ex = warp_inclusive_sum<int64_t>(mine) - mine;
  const int64_t tot = __shfl_sync(FULL, ex + mine, 31);
  const int leader = __ffs(mask) - 1;
  unsigned long long old = 0;
  if (lane == leader)
    old = atomicAdd(L.counter, ((unsigned long long)__popc(mask) << kPackShift) | (unsigned long long)tot);
  old = __shfl_sync(FULL, old, leader);
  if (want) {
    const int64_t j = (int64_t)(old >> kPackShift) + __popc(mask & ((1u << lane) - 1u));
    const int64_t ep = (int64_t)(old & kPackEdgeMask) + ex;
    if (!CC_IN_BOUNDS(j, L.cap, L.err)) return;
    L.v[j] = v;
    L.epos[j] = ep;
    L.delta[j] = row - ep;
    if (L.aux) L.aux[j] = aux;
  }
}

// Per-warp staging of list appends, so that many items share one atomic on
// the list counter.
constexpr int kAppCap = 128;

struct AppendBuf {
  int32_t v[kAppCap];
  int32_t len[kAppCap];
  int64_t row[kAppCap];
  int n;
};

__device__ __forceinline__ void append_flush(AppendBuf* b, const RowList& L) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  const int n = b->n;
  if (n == 0) return;
  constexpr int kPer = kAppCap / 32;
  int64_t loc = 0;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int i = lane * kPer + q;
    if (i < n) loc += b->len[i];
  }
  const int64_t ex = warp_inclusive_sum<int64_t>(loc) - loc;
  const int64_t tot = __shfl_sync(FULL, ex + loc, 31);
  unsigned long long old = 0;
  if (lane == 0) old = atomicAdd(L.counter, ((unsigned long long)n << kPackShift) | (unsigned long long)tot);
  old = __shfl_sync(FULL, old, 0);
  const int64_t j0 = (int64_t)(old >> kPackShift);
  int64_t ep = (int64_t)(old & kPackEdgeMask) + ex;
#pragma unroll
  for (int q = 0; q < kPer; ++q) {
    const int i = lane * kPer + q;
    if (i < n && CC_IN_BOUNDS(j0 + i, L.cap, L.err)) {
      L.v[j0 + i] = b->v[i];
      L.epos[j0 + i] = ep;
      L.delta[j0 + i] = b->row[i] - ep;
      ep += b->len[i];
    }
  }
  __syncwarp();
  if (lane == 0) b->n = 0;
  __syncwarp();
}

__device__ __forceinline__ void append_stage(AppendBuf* b, bool want, int32_t v, int64_t row, int32_t len,
                                             const RowList& L) {
  const int lane = threadIdx.x & 31;
  const unsigned mask = __ballot_sync(FULL, want);
  if (mask == 0) return;
  __syncwarp();
  if (b->n + __popc(mask) > kAppCap) append_flush(b, L);
  const int pos = b->n + __popc(mask & ((1u << lane) - 1u));
  if (want) {
    b->v[pos] = v;
    b->len[pos] = len;
    b->row[pos] = row;
  }
  __syncwarp();
  if (lane == 0) b->n += __popc(mask);
  __syncwarp();
}

}  // namespace ccg
