// cc_rounds.cu -- the bulk-synchronous rounds of C4 and ClusterWild! (Alg. 2)
// as one persistent cooperative kernel.
//
// All rounds run inside a single launch.  Phases are separated by grid
// barriers; block 0 is the coordinator: at every barrier it waits for all
// blocks, does the serial bookkeeping of the round (Delta walk, batch size,
// selection windows, statistics) on state it keeps in its own shared memory,
// publishes a 128-byte plan and releases the others, which copy the plan with
// one vector load.  Every wait is bounded.  The host is not involved between
// rounds.
//
// Per-vertex state: one 32-bit word st[v]
//   alive ............ kAlive | residual degree
//   clustered ........ kLab + center rank
//   active ............ kActive / kActCenter / kActNon (undecided or
//                       ClusterWild! center / C4 center / C4 non-center)
// An active's rank is kept in arank[v].  A center keeps its active marker for
// good (its label is its own rank, arank); the actives of the current round
// are the ones whose rank is >= r0, the round's first active rank.
//
// Attachment (createCluster, concurrency rule 2): a center of rank r lowers
// st[u] with atomicMin(kLab + r).  Alive words compare above every label and
// active markers below, so one compare-then-atomicMin does rule 2 and skips
// clustered and active vertices.
//
// Residual degrees live in the alive word itself, so the decrement that
// follows the removal of a vertex is a fire-and-forget atomic on that word.
// The alive tests of the hot passes read a separate removal tag instead:
// 4 bits per vertex, 0 while alive, else 1 + (removal round mod 15), an
// eighth of the state words' footprint, so the random reads of the edge
// passes and of the selection scans mostly hit L2.  A tag equal to the
// current round's only says "maybe removed this round" (a vertex removed
// 15, 30, ... rounds earlier carries it too); the state word decides.
//
// Delta_i (max residual degree, exact every round) comes from a heavy list H:
// every alive vertex whose degree was >= tau when H was built.  Degrees only
// fall, so if the largest current degree in H is still >= tau it is the
// maximum over the whole graph; otherwise a rebuild scans the compact list of
// alive non-isolated vertices, takes the exact maximum D, sets tau = D/2 and
// refills H.  No work per decrement.  Selection scans pi itself from a cursor
// (entry i is the vertex of rank i) and skips removed vertices by their tag;
// a selected vertex of residual degree 0 is a singleton center for which
// nothing is written (the label pass reads its alive word of degree 0).
//
// Every adjacency pass is edge-balanced (lbs_for_each), so hub rows of
// power-law graphs are split across many warps.
#include <cstdint>

#include "cc_device.cuh"
#include "cc_internal.h"

namespace ccg {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kScanU = 4;                    // list entries per thread per scan step
constexpr int kSelU = 2;                     // window entries per thread per selection step
constexpr int64_t kDescStride = 16;          // look-back descriptors: one per 128-byte line
constexpr int kAlgoC4 = 1, kAlgoCW = 2;
constexpr int kRun = 0, kDone = 1, kAbort = 3, kRebuildDelta = 4, kScanH = 5, kDrawBatch = 6;
constexpr int kRebuildDeg = 7, kRebuildHeavy = 8;   // Delta search over the degree order, heavy refill
// Defaults of the run-time schedule settings (Tuning; cc_tuning in the C ABI)
constexpr int32_t kInlineH = 8192;           // heavy lists up to this size are scanned by the coordinator
constexpr int32_t kInlineDecide = 4096;      // C4 blocked lists up to this size are decided by the coordinator
constexpr int32_t kInlineRebuild = 8192;     // heavy-list rebuilds over prefixes up to this size run in the coordinator
constexpr int32_t kHeavyShift = 1;           // heavy-list threshold tau = max(1, D >> kHeavyShift)
// C4 blocked actives are resolved one warp each (one grid phase) when every
// one of them has a warp and no blocked row is longer than this
constexpr int32_t kWarpResolveRow = 1024;

// State word of a vertex (uint32):
//   alive ........... kAlive | residual degree
//   clustered ....... kLab + center rank
//   active this round kActive (undecided, or a ClusterWild! center),
//                     kActCenter / kActNon (C4 center / non-center)
constexpr uint32_t kAlive = 0x80000000u, kDegMask = 0x7FFFFFFFu, kLab = 16;
constexpr uint32_t kActive = 1, kActCenter = 2, kActNon = 3;
constexpr int kTagCycle = 15;                // removal tags 1..15
__device__ __forceinline__ bool is_alive(uint32_t x) { return x >= kAlive; }
__device__ __forceinline__ uint32_t deg_of(uint32_t x) { return x & kDegMask; }
__device__ __forceinline__ bool is_active(uint32_t x) { return x < kLab; }

__device__ __forceinline__ int64_t rtag_words(int64_t n) { return (n >> 3) + 1; }
__device__ __forceinline__ uint32_t rtag_of(const uint32_t* rtag, int32_t v) {
  return (ldcg(rtag + (v >> 3)) >> ((v & 7) * 4)) & 15u;
}
__device__ __forceinline__ void set_rtag(uint32_t* rtag, int32_t v, uint32_t tag) {
  atomicOr(rtag + (v >> 3), tag << ((v & 7) * 4));      // result unused
}

// ---- the practical schedule of Sec. 5 ------------------------------------------
// Delta-hat starts at the maximum degree and halves every P rounds,
// P = (2/eps) ln(n log Delta / delta) with delta = 1/10, in integers: ln x =
// ln 2 log2 x with log2 rounded up to a bit length.  The batch B_i is
// binomial over the n - cursor unprocessed ranks of pi with p = eps /
// Delta-hat_i: the number of the round's SplitMix64 draws (a stream seeded
// from the seed of pi and the round) below T_i = floor(p 2^64).  A_i = the
// alive vertices among the next B_i ranks.
__device__ __forceinline__ int64_t bit_length(uint64_t x) { return x ? 64 - __clzll((long long)x) : 0; }

__device__ __forceinline__ int64_t sec5_period(int64_t n, int64_t max_deg, int64_t eps_ppm) {
  const int64_t l = bit_length((uint64_t)n) + bit_length((uint64_t)bit_length((uint64_t)(max_deg > 2 ? max_deg : 2))) + 4;
  return (int64_t)((2ull * 693147ull * (uint64_t)l + (uint64_t)eps_ppm - 1) / (uint64_t)eps_ppm);
}

__device__ __forceinline__ int64_t sec5_delta_hat(int64_t max_deg, int64_t period, int64_t round) {
  const int64_t h = round / period;
  const int64_t d = h >= 63 ? 0 : (max_deg >> h);
  return d > 1 ? d : 1;
}

// floor(eps_ppm 2^64 / (10^6 dhat)) for eps_ppm < 10^6 dhat: 64 quotient bits
// by long division (12, 12, 12, 12, 12, 4 bits; the remainder stays < 2^51).
__device__ __forceinline__ uint64_t sec5_threshold(int64_t eps_ppm, int64_t dhat, bool* all) {
  const uint64_t den = 1000000ull * (uint64_t)dhat;
  *all = (uint64_t)eps_ppm >= den;
  if (*all) return ~0ull;
  uint64_t r = (uint64_t)eps_ppm, t = 0;
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    r <<= 12;
    t = (t << 12) | (r / den);
    r %= den;
  }
  r <<= 4;
  return (t << 4) | (r / den);
}

// Draw j of round i's stream: the j-th output of SplitMix64 seeded with s.
__device__ __forceinline__ uint64_t sec5_draw(uint64_t s, uint64_t j) {
  return perm_key(0, s + j * 0x9E3779B97F4A7C15ull);     // state s + (j+1) gamma, mixed
}

template <class T>
__device__ __forceinline__ T vload(const T* p) { return *reinterpret_cast<const volatile T*>(p); }

__device__ __forceinline__ void atom_add_release(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Coordinator state, in block 0's shared memory for the whole kernel.
struct Coord {
  int64_t n, n_alive, cursor, al_len, k, round, stats_cap, eps_ppm;
  int64_t need, win_lo, win_len, r_edges, fix_iter;
  int64_t clusters;              // centers opened so far
  int64_t h_len;                 // heavy list length
  int64_t nz_len, nz_total;      // compact list of alive non-isolated vertices
  int64_t rb_lo, rb_hi;          // degree-order search: next segment of the prefix
  int32_t rb_t, rb_D;            // every vertex of full degree >= rb_t read; largest current degree seen
  int32_t tau, delta, max_deg, d_new;
  int algo, rebuilds_in_row;
  int nz_sel, nz_static;
  int delta_zero;                // a rebuild found no alive vertex with an alive neighbour
  int est;                       // the Sec. 5 schedule: Delta-hat and binomial batches
  int64_t period, rank_cursor;   // rounds per halving of Delta-hat; ranks of pi passed
  int32_t withhold;              // test hook (Ctl::withhold)
  int64_t batch_end;             // rank (index in pi) that ends the round's batch
  unsigned long long t0, round_t0;
  unsigned long long ph_ns[8];
};

// Shared memory of one block (dynamic: larger than the 48 KB static limit).
// Bucket-sort scratch of the in-kernel permutation (batched jobs).
constexpr int kPermCap = 1536;        // vertices per bucket sorted in shared memory
constexpr int kPermSubBits = 10;
constexpr int kPermSub = 1 << kPermSubBits;
constexpr int kPermMaxBuckets = 4096;

struct PermSmem {
  uint64_t sk[kPermCap];
  uint64_t ok[kPermCap];
  int32_t sv[kPermCap];
  int32_t ov[kPermCap];
  int32_t cnt[kPermSub + 1];
  int32_t hist[kPermMaxBuckets];
};

struct Shared {
  Plan plan;
  Coord co;
  int ok;
  int dec;
  int64_t scr[33];
  int64_t bcast[8];
  unsigned long long tal[5];     // round tallies of the block (flushed at round end)
  union {
    struct {
      LbsWarp lbs[kWarps];
      AppendBuf app[kWarps];
    } w;
    PermSmem perm;
  } u;
};

// Per-thread tallies of one round (flushed at every round end).
// The member-center edges of the objective need no tally: every member of a
// cluster is adjacent to its center (it was attached through that edge) and
// to no other center of its cluster, so they number n - (number of clusters).
struct Tally {
  int32_t centers, attached, noncenter, blocked;
  uint32_t mm;                  // member-member entries inside a cluster
};

// The blocks that run one clustering job: the whole grid, or a team of
// G blocks inside a batched launch (bid = this block's rank in the team).
struct K {
  const RoundBuffers& B;
  Ctl* C;
  Shared* S;
  unsigned G;
  unsigned bid;
  unsigned epoch;
  Tally t;

  template <class F>
  __device__ __forceinline__ void lbs(const int64_t* epos, int64_t nitems, int64_t E, F&& f,
                                      const int64_t* delta = nullptr, const int32_t* vtx = nullptr,
                                      const uint32_t* vmap = nullptr, uint32_t vsub = 0) {
    // every walk with a delta array walks CSR rows: stream them ahead.
    // Warps are numbered across the blocks first (warp w of block b is
    // w * G + b), so a short walk spreads over every SM instead of the
    // first few blocks.
    lbs_for_each_in((int64_t)(threadIdx.x >> 5) * G + bid, ((int64_t)G * blockDim.x) >> 5, epos, nitems,
                    E, lbs_ws(), f, delta, vtx, 0, vmap, vsub, delta ? B.col : nullptr,
                    WalkShape{B.tune.walk_batches, B.tune.prefetch_ahead});
  }

  __device__ __forceinline__ const Plan& P() const { return S->plan; }
  // heavy-list threshold for a maximum degree D
  __device__ __forceinline__ int32_t tau_of(int32_t D) const {
    const int32_t t = D >> B.tune.heavy_shift;
    return t >= 1 ? t : 1;
  }
  __device__ __forceinline__ Coord& co() const { return S->co; }
  __device__ void fail(int code) { atomicCAS(&C->err, kOk, code); }

  // ---------------- grid barrier with the coordinator -------------------------
  // All blocks call sync(); block 0 waits for every arrival, books the time
  // since the previous barrier to phase `cat`, runs act() with its whole
  // block (writing S->plan), publishes the plan and releases.  The others
  // wait for the release and copy the plan.  Returns false once the run
  // must stop (error, or the plan says so).
  template <class A>
  __device__ bool sync(int cat, A&& act) {
    __syncthreads();
    ++epoch;
    if (G == 1) {                       // a one-block team is its own coordinator
      if (threadIdx.x == 0) {
        const unsigned long long now = globaltimer_ns();
        S->co.ph_ns[cat] += now - S->co.t0;
        S->co.t0 = now;
      }
      __syncthreads();
      if (ld_volatile_int(&C->err) == kOk) act();
      __syncthreads();
      if (threadIdx.x == 0 && ld_volatile_int(&C->err) != kOk) S->plan.state = kAbort;
      __syncthreads();
      return S->plan.state != kAbort;
    }
    if (threadIdx.x == 0) atom_add_release(&C->arrive, 1u);
    if (bid == 0) {
      if (threadIdx.x == 0) {
        const unsigned target = G * epoch;
        const uint64_t t0 = globaltimer_ns();
        unsigned spins = 0;
        int ok = 1;
        while (ld_acquire(&C->arrive) < target) {
          if ((++spins & 63) == 0) {
            if (ld_volatile_int(&C->err) != kOk) { ok = 0; break; }
            if (globaltimer_ns() - t0 > kBarrierLimitNs) { atomicCAS(&C->err, kOk, kErrTimeout); ok = 0; break; }
          }
        }
        if (ld_volatile_int(&C->err) != kOk) ok = 0;
        const unsigned long long now = globaltimer_ns();
        S->co.ph_ns[cat] += now - S->co.t0;
        S->co.t0 = now;
        S->ok = ok;
      }
      __syncthreads();
      if (S->ok) act();
      __syncthreads();
      // an error (here or in any block) travels in the plan as the abort state
      if (threadIdx.x == 0 && (!S->ok || ld_volatile_int(&C->err) != kOk)) S->plan.state = kAbort;
      // test hook: after the chosen round the release is withheld; the other
      // blocks' bounded waits run out (kErrTimeout) and every block unwinds
      if (threadIdx.x == 0 && cat == 6 && S->co.withhold != 0 && S->co.round == S->co.withhold) {
        S->plan.state = kAbort;
        S->ok = 2;
      }
      __syncthreads();
      if (S->ok != 2) {
        // publish: 128 bytes as eight 16-byte stores, then release
        if (threadIdx.x < sizeof(Plan) / 16)
          reinterpret_cast<int4*>(&C->plan)[threadIdx.x] = reinterpret_cast<const int4*>(&S->plan)[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 0) st_release(&C->gen, epoch);
      }
    } else {
      if (threadIdx.x == 0) {
        const uint64_t t0 = globaltimer_ns();
        unsigned spins = 0;
        int released = 1;
        while (ld_acquire(&C->gen) < epoch) {
          if ((++spins & 63) == 0) {
            if (ld_volatile_int(&C->err) != kOk) { released = 0; break; }
            if (globaltimer_ns() - t0 > kBarrierLimitNs) {
              atomicCAS(&C->err, kOk, kErrTimeout);
              released = 0;
              break;
            }
          }
        }
        S->ok = released;
      }
      __syncthreads();
      // the plan (its last 16 bytes hold the state word; without a release
      // the copy is stale and the state becomes the abort state)
      if (threadIdx.x < sizeof(Plan) / 16) {
        int4 q = __ldcg(reinterpret_cast<const int4*>(&C->plan) + threadIdx.x);
        if (threadIdx.x == sizeof(Plan) / 16 - 1 && !S->ok) q.x = kAbort;
        reinterpret_cast<int4*>(&S->plan)[threadIdx.x] = q;
      }
      __syncthreads();
    }
    return S->plan.state != kAbort;
  }
  __device__ bool sync(int cat) {
    return sync(cat, [] {});
  }

  __device__ RowList new_list() const { return RowList{B.new_v, B.new_e, B.new_d, nullptr, &C->new_pack CC_ROWLIST_CHECK(B.n, &C->err)}; }
  // blocked actives; the payload initialises each one's pull slot (no center yet)
  __device__ RowList blk_list() const { return RowList{B.b_j, B.b_e, B.b_d, B.pull, &C->blk_pack CC_ROWLIST_CHECK(B.n, &C->err)}; }
  __device__ LbsWarp* lbs_ws() const { return &S->u.w.lbs[threadIdx.x >> 5]; }
  __device__ AppendBuf* app_buf() const { return &S->u.w.app[threadIdx.x >> 5]; }

  // Entry i of the rank-ordered candidate list: (rank, vertex) = (i, pi(i)).
  // Selection scans it from the cursor and skips removed vertices by their
  // removal tag; the list is never compacted (every entry is scanned about
  // once anyway, so a compaction pass would cost more than it saves).
  __device__ int2 al_at(int64_t i) const { return make_int2((int32_t)i, __ldg(B.order + i)); }

  // contiguous slice of [lo, lo+len) for this block
  __device__ void slice(int64_t lo, int64_t len, int64_t* s, int64_t* e) const {
    const int64_t chunk = (len + G - 1) / G;
    *s = lo + chunk * bid;
    *e = *s + chunk < lo + len ? *s + chunk : lo + len;
    if (*s > *e) *s = *e;
  }

  // Coordinator: exclusive prefix of blk_a[0..G) in place; returns the total.
  __device__ int64_t prefix_blocks() {
    int64_t run = 0;
    for (unsigned base = 0; base < G; base += blockDim.x) {
      const unsigned b = base + threadIdx.x;
      const int64_t x = b < G ? ldcg(B.blk_a + b) : 0;
      int64_t tot;
      const int64_t ex = block_exclusive_sum<int64_t>(x, S->scr, &tot);
      if (b < G) B.blk_a[b] = run + ex;
      run += tot;
    }
    __syncthreads();
    return run;
  }

  // ---------------- coordinator actions ----------------------------------------
  __device__ void co_init() {
    if (threadIdx.x == 0) {
      Coord& c = co();
      c.n = B.n;
      c.n_alive = B.n;
      c.cursor = 0;
      c.al_len = B.n;
      c.max_deg = B.max_deg;
      c.tau = 0x7FFFFFFF;         // empty heavy list: the first round rebuilds it
      c.h_len = 0;
      c.nz_len = B.nz_n;          // non-isolated vertices, from the graph
      c.nz_static = 1;
      c.nz_sel = 0;
      c.delta_zero = 0;
      c.round = 0;
      c.clusters = 0;
      c.rebuilds_in_row = 0;
      c.algo = vload(&C->algo);
      c.eps_ppm = vload(&C->eps_ppm);
      c.withhold = vload(&C->withhold);
      c.est = c.algo >= 3;                // the Sec. 5 schedule
      if (c.est) c.algo -= 2;
      c.period = c.est ? sec5_period(c.n, c.max_deg, c.eps_ppm) : 0;
      c.rank_cursor = 0;
      c.stats_cap = B.stats_cap;
      Plan& p = S->plan;
      p = Plan{};
      p.r0 = -1;
    }
    __syncthreads();
    co_decide_delta();
  }

  // Coordinator: with Delta known, set k and the first selection window.
  __device__ void plan_selection(int32_t delta) {
    if (threadIdx.x == 0) {
      Coord& c = co();
      Plan& p = S->plan;
      int64_t k;
      if (delta <= 0) k = c.n_alive;
      else {
        const unsigned long long num = (unsigned long long)c.eps_ppm * (unsigned long long)c.n_alive;
        const unsigned long long den = 1000000ull * (unsigned long long)delta;
        k = (int64_t)((num + den - 1) / den);
        if (k < 1) k = 1;
        if (k > c.n_alive) k = c.n_alive;
      }
      c.delta = delta;
      c.k = k;
      c.need = k;
      c.win_lo = c.cursor;
      const int64_t avail = c.al_len - c.cursor;
      const int64_t est = (int64_t)((double)k * (double)avail / (double)c.n_alive * 1.05) + 256;
      c.win_len = est < avail ? est : avail;
      if (c.est) {
        // Sec. 5: the whole window of the round's batch, every alive entry of it
        c.k = 0;                          // set from the window's alive count
        c.need = INT64_MAX / 4;
        c.win_len = c.batch_end - c.cursor;
      }
      c.r_edges = 0;
      C->act_pack = 0; C->new_pack = 0; C->blk_pack = 0; C->blk_maxlen = 0;
      C->r_centers = 0; C->r_attached = 0; C->r_noncenter = 0; C->r_blocked = 0;
      C->r0 = -1;
      p.state = kRun;
      p.k = c.k;
      p.need = c.need;
      p.win_lo = c.win_lo;
      p.win_len = c.win_len;
      p.th = 0;
      p.r0 = -1;
      p.tag = (int32_t)(c.round % kTagCycle) + 1;
    }
    __syncthreads();
  }

  // Coordinator, at a round boundary: finish, draw the Sec. 5 batch, or get
  // Delta from the heavy list (inline when short, else by a grid scan), or
  // rebuild the heavy list.
  __device__ __noinline__ void co_decide_delta() {
    Coord& c = co();
    Plan& p = S->plan;
    if (threadIdx.x == 0) {
      int dec = 1;
      if (c.n_alive <= 0) p.state = kDone;
      else if (c.est) {
        p.state = kDrawBatch;             // Sec. 5: draw the batch, no Delta
        const int64_t dh = sec5_delta_hat(c.max_deg, c.period, c.round);
        bool all;
        const uint64_t thr = sec5_threshold(c.eps_ppm, dh, &all);
        c.delta = (int32_t)dh;
        p.win_len = c.n - c.rank_cursor;                            // trials
        p.need = (int64_t)thr;                                      // threshold bits
        p.take = all ? 1 : 0;
        p.k = (int64_t)perm_key(vload(&C->seed) ^ 0x5851F42D4C957F2Dull, (uint64_t)c.round);   // stream seed
      } else if (c.delta_zero) {
        dec = 2;                          // every alive vertex is isolated: Delta = 0
      } else if (c.h_len == 0) {
        dec = 3;                          // no heavy list yet: build it
      } else if (c.h_len > B.tune.inline_heavy) {
        p.state = kScanH; p.win_lo = 0; p.win_len = c.h_len;
      } else {
        dec = 0;                          // scan the short heavy list here
      }
      S->dec = dec;
    }
    __syncthreads();
    if (S->dec == 2) { plan_selection(0); return; }
    if (S->dec == 3) {
      // before the first round every vertex is alive with its full degree:
      // the search starts at the largest degree, which it finds at once
      start_rebuild(co().round == 0 ? co().max_deg : 1);
      return;
    }
    if (S->dec) return;
    // the whole block reads the heavy list, eight entries per thread at a time
    // so that the dependent loads overlap
    int64_t mx = -1;
    for (int64_t base = 0; base < c.h_len; base += 8 * (int64_t)blockDim.x) {
      int32_t h[8];
      uint32_t x[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int64_t i = base + threadIdx.x + (int64_t)q * blockDim.x;
        h[q] = i < c.h_len ? ldcg(B.hv + i) : -1;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) x[q] = h[q] >= 0 ? ldcg(B.st + h[q]) : 0u;
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (is_alive(x[q])) mx = (int64_t)deg_of(x[q]) > mx ? (int64_t)deg_of(x[q]) : mx;
    }
    mx = block_max<int64_t>(mx, S->scr);
    co_after_heavy((int32_t)mx);
  }

  // Coordinator: the largest current degree in the heavy list is mx (-1 if
  // none is alive).  It is the global maximum when it is still >= tau.
  __device__ void co_after_heavy(int32_t mx) {
    if (threadIdx.x == 0) S->dec = mx >= co().tau ? 1 : 0;
    __syncthreads();
    if (S->dec) { plan_selection(mx); return; }
    // The new maximum D lies in [max(mx, 0), tau): every vertex outside the
    // heavy list had a degree below tau when the list was built.
    start_rebuild(co().tau >= 2 ? co().tau >> 1 : 1);
  }

  // ---------------- Delta rebuild: where to look -------------------------------
  // A rebuild needs the exact maximum D over the alive vertices and a new heavy
  // list holding every alive vertex of degree >= max(1, D/2).  Degrees only
  // fall, so a vertex of current degree >= x has full degree >= x.  The search
  // reads the degree order (dsort, largest full degree first) in segments:
  // after every vertex of full degree >= t has been read, the largest current
  // degree seen is D exactly if it is >= t (no unread vertex can reach t);
  // otherwise t halves and the next segment is read.  The heavy list then
  // comes from the prefix of full degree >= D/2.  Segments up to
  // inline_rebuild vertices (a tuning setting) are read by the coordinator block inside the
  // barrier; longer ones by the grid.  Once the prefix to read exceeds a
  // quarter of the compact list of alive non-isolated vertices (vertex order,
  // dead vertices dropped at each of its rebuilds), that list is cheaper and
  // the rebuild switches to it.
  __device__ __noinline__ void start_rebuild(int32_t t0) {
    if (threadIdx.x == 0) {
      Coord& c = co();
      const int32_t hi = c.max_deg + 1;
      c.rb_t = t0 < 1 ? 1 : (t0 > hi ? hi : t0);
      c.rb_lo = 0;
      c.rb_hi = __ldg(B.dge + c.rb_t);
      c.rb_D = 0;
      c.rebuilds_in_row += 1;
      if (c.rebuilds_in_row > 2) fail(kErrInternal);
    }
    __syncthreads();
    rebuild_advance();
  }

  // Coordinator block: read segments inline until D is known (then refill the
  // heavy list, inline or by planning a grid pass), or plan a grid step.
  __device__ __noinline__ void rebuild_advance() {
    for (;;) {
      if (threadIdx.x == 0) {
        Coord& c = co();
        Plan& p = S->plan;
        const int64_t limit = c.nz_len / 4;
        const int64_t seg = c.rb_hi - c.rb_lo;
        int dec;
        if (seg > 0) {
          dec = seg <= B.tune.inline_rebuild ? 0 : (c.rb_hi > limit ? 4 : 1);
        } else if (c.rb_D >= c.rb_t || c.rb_t <= 1) {
          if (c.rb_D <= 0) {
            dec = 5;                                  // nothing alive has an alive neighbour
          } else {
            c.tau = tau_of(c.rb_D);
            c.rb_hi = __ldg(B.dge + c.tau);           // heavy candidates: full degree >= tau
            dec = c.rb_hi <= B.tune.inline_rebuild ? 2 : (c.rb_hi > limit ? 4 : 3);
          }
        } else {
          c.rb_t = c.rb_t >= 2 ? c.rb_t >> 1 : 1;
          c.rb_hi = __ldg(B.dge + c.rb_t);
          dec = -1;
        }
        if (dec == 1) { p.state = kRebuildDeg; p.win_lo = c.rb_lo; p.win_len = seg; }
        if (dec == 3) { p.state = kRebuildHeavy; p.win_lo = 0; p.win_len = c.rb_hi; p.th = c.tau; C->h_pack = 0; }
        if (dec == 4) { p.state = kRebuildDelta; set_nz_plan(); }
        S->dec = dec;
      }
      __syncthreads();
      const int dec = S->dec;
      __syncthreads();
      if (dec == -1) continue;
      if (dec == 0) {                                 // read a short segment here
        const int64_t m = deg_max_over(co().rb_lo, co().rb_hi);
        if (threadIdx.x == 0) {
          Coord& c = co();
          c.rb_D = m > c.rb_D ? (int32_t)m : c.rb_D;
          c.rb_lo = c.rb_hi;
        }
        __syncthreads();
        continue;
      }
      if (dec == 2) {                                 // refill a short heavy list here
        const int32_t tau = co().tau;
        const int64_t len = co().rb_hi;
        if (threadIdx.x == 0) S->bcast[0] = 0;
        __syncthreads();
        for (int64_t base = threadIdx.x; base < len; base += (int64_t)kScanU * blockDim.x) {
          int32_t v[kScanU];
          uint32_t x[kScanU];
#pragma unroll
          for (int q = 0; q < kScanU; ++q) {
            const int64_t i = base + (int64_t)q * blockDim.x;
            v[q] = i < len ? __ldg(B.dsort + i) : -1;
          }
#pragma unroll
          for (int q = 0; q < kScanU; ++q) x[q] = v[q] >= 0 ? ldcg(B.st + v[q]) : 0u;
#pragma unroll
          for (int q = 0; q < kScanU; ++q)
            if (is_alive(x[q]) && deg_of(x[q]) > 0 && (int64_t)deg_of(x[q]) >= tau)
            {
              const int64_t h = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(&S->bcast[0]), 1ull);
              if (CC_IN_BOUNDS(h, B.n, &C->err)) B.hv[h] = v[q];
            }
        }
        __syncthreads();
        finish_rebuild(co().rb_D, S->bcast[0]);
        return;
      }
      if (dec == 5) { finish_rebuild(0, 0); return; }
      return;                                         // a grid step is planned
    }
  }

  // Coordinator block: the largest current degree of an alive vertex among
  // dsort[lo, hi) (0 if none).
  __device__ int64_t deg_max_over(int64_t lo, int64_t hi) {
    int64_t mx = 0;
    for (int64_t base = lo + threadIdx.x; base < hi; base += (int64_t)kScanU * blockDim.x) {
      uint32_t x[kScanU];
#pragma unroll
      for (int q = 0; q < kScanU; ++q) {
        const int64_t i = base + (int64_t)q * blockDim.x;
        x[q] = i < hi ? ldcg(B.st + __ldg(B.dsort + i)) : 0u;
      }
#pragma unroll
      for (int q = 0; q < kScanU; ++q)
        if (is_alive(x[q])) mx = (int64_t)deg_of(x[q]) > mx ? (int64_t)deg_of(x[q]) : mx;
    }
    return block_max<int64_t>(mx, S->scr);
  }

  __device__ void set_nz_plan() {
    Coord& c = co();
    S->plan.win_lo = 0;
    S->plan.win_len = c.nz_len;
    S->plan.pad0 = (c.nz_static ? 2 : 0) | c.nz_sel;
  }

  // Coordinator: the new maximum D and heavy list of hcount entries are in
  // place; plan the round's selection.
  __device__ void finish_rebuild(int32_t D, int64_t hcount) {
    if (threadIdx.x == 0) {
      Coord& c = co();
      c.tau = tau_of(D);
      c.h_len = D > 0 ? hcount : 0;
      if (D <= 0) c.delta_zero = 1;
    }
    __syncthreads();
    plan_selection(D > 0 ? D : 0);
  }

  // Statistics and n_i update after the removal phase, then the next plan.
  __device__ void co_end_round() {
    Coord& c = co();
    if (threadIdx.x < 6) {
      const long long* src[6] = {&C->r_centers, &C->r_attached, &C->r_noncenter, &C->r_blocked,
                                 reinterpret_cast<const long long*>(&C->new_pack), nullptr};
      if (threadIdx.x < 5) S->bcast[threadIdx.x] = vload(src[threadIdx.x]);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const int64_t centers_seen = S->bcast[0], attached = S->bcast[1], noncenter = S->bcast[2];
      const int64_t blocked = S->bcast[3];
      const unsigned long long np = (unsigned long long)S->bcast[4];
      const int64_t k = c.k;
      const int64_t removed = k + attached;
      const int64_t centers = k - noncenter;
      const int64_t r = c.round;
      if (r < c.stats_cap) {
        RoundStat s;
        s.n_alive = c.n_alive; s.delta = c.delta; s.k = k; s.centers = centers;
        s.removed = removed; s.blocked = blocked; s.edges = c.r_edges + (int64_t)(np & kPackEdgeMask);
        s.ns = (int64_t)(globaltimer_ns() - c.round_t0);
        B.stats[r] = s;
      }
      c.round_t0 = globaltimer_ns();
      if (centers_seen != centers) fail(kErrInternal);
      c.n_alive -= removed;
      c.clusters += centers;
      if (c.n_alive < 0) fail(kErrInternal);
      c.round = r + 1;
      c.rebuilds_in_row = 0;
      if (!c.est && c.round > c.n + 1) fail(kErrInternal);   // Sec. 5 rounds may hold no active vertex
    }
    __syncthreads();
    co_decide_delta();
  }

  // ---------------- Sec. 5: the round's binomial batch ------------------------
  // Every block counts its share of the round's draws below the threshold
  // (plan: win_len trials, need = threshold bits, take = every trial
  // succeeds, k = stream seed); the coordinator adds them up, moves the rank
  // cursor past the batch and plans the round's single selection window, the
  // batch's ranks of pi.
  __device__ bool draw_batch() {
    const int64_t trials = P().win_len;
    const uint64_t thr = (uint64_t)P().need, s = (uint64_t)P().k;
    int64_t cnt = 0;
    if (P().take) {
      cnt = bid == 0 && threadIdx.x == 0 ? trials : 0;
    } else {
      for (int64_t j = (int64_t)bid * blockDim.x + threadIdx.x; j < trials; j += (int64_t)G * blockDim.x)
        cnt += sec5_draw(s, (uint64_t)j) < thr ? 1 : 0;
    }
    cnt = block_sum<int64_t>(cnt, S->scr);
    if (threadIdx.x == 0) B.blk_a[bid] = cnt;
    return sync(2, [&] {
      const int64_t b = prefix_blocks();
      Coord& c = co();
      const int64_t end_rank = c.rank_cursor + b;
      // the list entry of rank end_rank ends the batch (entry i has rank i)
      const int64_t end = end_rank < c.al_len ? end_rank : c.al_len;
      if (threadIdx.x == 0) {
        c.batch_end = end;
        c.rank_cursor = end_rank;
        if (end_rank > c.n) fail(kErrInternal);
      }
      __syncthreads();
      plan_selection(c.delta);
    });
  }

  // ---------------- heavy list: per-round maximum ----------------------------
  __device__ bool heavy_scan() {
    int64_t s, e;
    slice(0, P().win_len, &s, &e);
    int64_t mx = -1;
    for (int64_t base = s; base < e; base += (int64_t)blockDim.x * kScanU) {
      int32_t v[kScanU];
#pragma unroll
      for (int q = 0; q < kScanU; ++q) {
        const int64_t i = base + (int64_t)threadIdx.x * kScanU + q;
        v[q] = i < e ? ldcg(B.hv + i) : -1;
      }
#pragma unroll
      for (int q = 0; q < kScanU; ++q) {
        if (v[q] < 0) continue;
        const uint32_t x = ldcg(B.st + v[q]);
        if (is_alive(x)) mx = (int64_t)deg_of(x) > mx ? (int64_t)deg_of(x) : mx;
      }
    }
    mx = block_max<int64_t>(mx, S->scr);
    if (threadIdx.x == 0) B.blk_b[bid] = mx;
    return sync(0, [&] {
      const int64_t m = max_blocks_signed();
      co_after_heavy((int32_t)m);
    });
  }

  // ---------------- Delta rebuild: grid passes ---------------------------------
  // Over the compact list (vertex order): A, count the vertices that are still
  // alive with a degree > 0 and find the largest degree D; B, compact the list
  // and put every survivor of degree >= tau = max(1, D/2) on the heavy list.
  __device__ int32_t nz_at(int flags, int64_t i) const {
    if (flags & 2) return __ldg(B.nz_static + i);
    return ldcg(((flags & 1) ? B.nz1 : B.nz0) + i);
  }

  __device__ bool delta_rebuild() {
    const int flags = P().pad0;
    const int64_t len = P().win_len;
    int64_t s, e;
    slice(0, len, &s, &e);
    int64_t cnt = 0, mx = 0;
    for (int64_t base = s; base < e; base += (int64_t)blockDim.x * kScanU) {
      int32_t v[kScanU];
#pragma unroll
      for (int q = 0; q < kScanU; ++q) {
        const int64_t i = base + (int64_t)threadIdx.x * kScanU + q;
        v[q] = i < e ? nz_at(flags, i) : -1;
      }
#pragma unroll
      for (int q = 0; q < kScanU; ++q) {
        if (v[q] < 0) continue;
        const uint32_t x = ldcg(B.st + v[q]);
        if (is_alive(x) && deg_of(x) > 0) {
          ++cnt;
          mx = (int64_t)deg_of(x) > mx ? (int64_t)deg_of(x) : mx;
        }
      }
    }
    cnt = block_sum<int64_t>(cnt, S->scr);
    mx = block_max<int64_t>(mx, S->scr);
    if (threadIdx.x == 0) { B.blk_a[bid] = cnt; B.blk_b[bid] = mx; }
    if (!sync(0, [&] {
          const int64_t tot = prefix_blocks();
          const int64_t D = max_blocks_signed();
          if (threadIdx.x == 0) {
            Coord& c = co();
            c.nz_total = tot;
            c.d_new = (int32_t)(D > 0 ? D : 0);
            S->plan.th = tau_of((int32_t)D);
            C->h_pack = 0;
          }
        }))
      return false;
    const int32_t tau = P().th;
    int32_t* dst = (flags & 2) ? B.nz0 : ((flags & 1) ? B.nz0 : B.nz1);
    int64_t run = ldcg(B.blk_a + bid);
    for (int64_t base = s; base < e; base += (int64_t)blockDim.x * kScanU) {
      int32_t v[kScanU];
      uint32_t d[kScanU];
      int64_t mine = 0, heavy = 0;
#pragma unroll
      for (int q = 0; q < kScanU; ++q) {
        const int64_t i = base + (int64_t)threadIdx.x * kScanU + q;
        v[q] = i < e ? nz_at(flags, i) : -1;
      }
#pragma unroll
      for (int q = 0; q < kScanU; ++q) {
        d[q] = 0;
        if (v[q] < 0) continue;
        const uint32_t x = ldcg(B.st + v[q]);
        if (is_alive(x)) d[q] = deg_of(x);
        mine += d[q] > 0 ? 1 : 0;
        heavy += (d[q] > 0 && (int64_t)d[q] >= tau) ? 1 : 0;
      }
      int64_t tot, htot;
      int64_t o = run + block_exclusive_sum<int64_t>(mine, S->scr, &tot);
      int64_t ho = block_exclusive_sum<int64_t>(heavy, S->scr, &htot);
      if (htot > 0) {
        if (threadIdx.x == 0) S->bcast[0] = (int64_t)atomicAdd(&C->h_pack, (unsigned long long)htot);
        __syncthreads();
        ho += S->bcast[0];
        __syncthreads();
      }
#pragma unroll
      for (int q = 0; q < kScanU; ++q) {
        if (d[q] == 0) continue;
        if (CC_IN_BOUNDS(o, B.n, &C->err)) dst[o++] = v[q];
        if ((int64_t)d[q] >= tau && CC_IN_BOUNDS(ho, B.n, &C->err)) B.hv[ho++] = v[q];
      }
      run += tot;
    }
    return sync(1, [&] {
      if (threadIdx.x == 0) {
        Coord& c = co();
        c.nz_sel = (flags & 2) ? 0 : ((flags & 1) ? 0 : 1);
        c.nz_static = 0;
        c.nz_len = c.nz_total;
      }
      __syncthreads();
      finish_rebuild(co().d_new, (int64_t)vload(&C->h_pack));
    });
  }

  // One segment dsort[win_lo, win_lo + win_len) of the degree-order search:
  // the largest current degree of an alive vertex in it.
  __device__ bool rebuild_segment() {
    int64_t s, e;
    slice(P().win_lo, P().win_len, &s, &e);
    int64_t mx = 0;
    for (int64_t base = s; base < e; base += (int64_t)blockDim.x * kScanU) {
      uint32_t x[kScanU];
#pragma unroll
      for (int q = 0; q < kScanU; ++q) {
        const int64_t i = base + (int64_t)threadIdx.x * kScanU + q;
        x[q] = i < e ? ldcg(B.st + __ldg(B.dsort + i)) : 0u;
      }
#pragma unroll
      for (int q = 0; q < kScanU; ++q)
        if (is_alive(x[q])) mx = (int64_t)deg_of(x[q]) > mx ? (int64_t)deg_of(x[q]) : mx;
    }
    mx = block_max<int64_t>(mx, S->scr);
    if (threadIdx.x == 0) B.blk_b[bid] = mx;
    return sync(0, [&] {
      const int64_t m = max_blocks_signed();
      if (threadIdx.x == 0) {
        Coord& c = co();
        c.rb_D = m > c.rb_D ? (int32_t)m : c.rb_D;
        c.rb_lo = c.rb_hi;
      }
      __syncthreads();
      rebuild_advance();
    });
  }

  // The heavy list from dsort[0, win_len): every alive vertex of current
  // degree >= th (> 0).
  __device__ bool heavy_fill() {
    int64_t s, e;
    slice(0, P().win_len, &s, &e);
    const int64_t tau = P().th;
    for (int64_t base = s; base < e; base += (int64_t)blockDim.x * kScanU) {
      int32_t v[kScanU];
      uint32_t x[kScanU];
      int64_t heavy = 0;
#pragma unroll
      for (int q = 0; q < kScanU; ++q) {
        const int64_t i = base + (int64_t)threadIdx.x * kScanU + q;
        v[q] = i < e ? __ldg(B.dsort + i) : -1;
      }
#pragma unroll
      for (int q = 0; q < kScanU; ++q) {
        x[q] = v[q] >= 0 ? ldcg(B.st + v[q]) : 0u;
        if (!(is_alive(x[q]) && deg_of(x[q]) > 0 && (int64_t)deg_of(x[q]) >= tau)) v[q] = -1;
        heavy += v[q] >= 0 ? 1 : 0;
      }
      int64_t htot;
      int64_t ho = block_exclusive_sum<int64_t>(heavy, S->scr, &htot);
      if (htot > 0) {
        if (threadIdx.x == 0) S->bcast[0] = (int64_t)atomicAdd(&C->h_pack, (unsigned long long)htot);
        __syncthreads();
        ho += S->bcast[0];
        __syncthreads();
      }
#pragma unroll
      for (int q = 0; q < kScanU; ++q)
        if (v[q] >= 0 && CC_IN_BOUNDS(ho, B.n, &C->err)) B.hv[ho++] = v[q];
    }
    return sync(1, [&] { finish_rebuild(co().rb_D, (int64_t)vload(&C->h_pack)); });
  }

  __device__ int64_t max_blocks_signed() {
    int64_t m = -1;
    for (unsigned b = threadIdx.x; b < G; b += blockDim.x) {
      const int64_t x = ldcg(B.blk_b + b);
      m = x > m ? x : m;
    }
    return block_max<int64_t>(m, S->scr);
  }

  // ---------------- active-set selection (Alg. 2: A = next k alive of pi) ----
  // Called by every thread of the block for one tile of the window; entry q
  // of a thread is an active vertex (rank a[q].x, vertex a[q].y) when want[q].
  __device__ void emit_actives(const int2* a, const bool* want, int algo) {
    int64_t deg0[kSelU], row[kSelU];
    bool listed[kSelU];
    int64_t nl = 0, el = 0;
#pragma unroll
    for (int q = 0; q < kSelU; ++q) {
      listed[q] = false;
      deg0[q] = 0;
      row[q] = 0;
      if (!want[q]) continue;
      const int32_t r = a[q].x, v = a[q].y;
      const uint32_t d = deg_of(ldcg(B.st + v));
      if (d == 0) {
        // no alive neighbour: a singleton center.  No pass can reach it
        // again (its neighbours are all clustered, and later windows start
        // past it), so it keeps its alive word and zero tag; the label pass
        // reads an alive word of degree 0 as its own cluster.
        t.centers += 1;
      } else {
        set_rtag(B.rtag, v, (uint32_t)P().tag);
        row[q] = __ldg(B.off + v);
        deg0[q] = __ldg(B.off + v + 1) - row[q];
        B.arank[v] = r;
        B.st[v] = kActive;
        listed[q] = true;
        nl += 1;
        el += deg0[q];
        if (algo == kAlgoCW) t.centers += 1;
      }
    }
    // one atomic per block and tile on the packed list counter
    int64_t tot;
    const int64_t pkx = block_exclusive_sum<int64_t>((nl << 40) | el, S->scr, &tot);
    const int64_t jx = pkx >> 40, ex = pkx & ((1ll << 40) - 1);
    const int64_t cnt_tot = tot >> 40, e_tot = tot & ((1ll << 40) - 1);
    if (cnt_tot == 0) return;
    if (threadIdx.x == 0) {
      const unsigned long long old =
          atomicAdd(&C->act_pack, ((unsigned long long)cnt_tot << kPackShift) | (unsigned long long)e_tot);
      S->bcast[0] = (int64_t)(old >> kPackShift);
      S->bcast[1] = (int64_t)(old & kPackEdgeMask);
    }
    __syncthreads();
    int64_t j = S->bcast[0] + jx, ep = S->bcast[1] + ex;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kSelU; ++q) {
      if (!listed[q] || !CC_IN_BOUNDS(j, B.n, &C->err)) continue;
      B.act_v[j] = a[q].y;
      B.act_r[j] = a[q].x;
      B.act_e[j] = ep;
      B.act_d[j] = row[q] - ep;
      B.blk_flag[j] = 0;
      ++j;
      ep += deg0[q];
    }
  }

  // Look-back over the team (one pass instead of count, barrier, emit):
  // block bid publishes its alive count in desc[bid * kDescStride] (one
  // 128-byte line per block, so that the pollers of different blocks'
  // counts meet in different L2 slices), tagged with the barrier
  // epoch; thread q of the block waits for the counts of predecessors q,
  // q + blockDim.x, ... and the block sums them (a single round of loads
  // while the team has at most blockDim.x blocks).  The last block also
  // stores the window's total in desc[G * kDescStride] for the coordinator.  A cleared
  // descriptor (flag 0) is never taken for a count, whatever the epoch.
  // Returns this block's exclusive prefix to every thread; every wait is
  // bounded.
  static constexpr unsigned long long kDescVal = (1ull << 38) - 1;
  __device__ __forceinline__ unsigned long long pack_desc(unsigned flag, long long v) const {
    return ((unsigned long long)(epoch & 0xFFFFFFu) << 40) | ((unsigned long long)flag << 38) |
           ((unsigned long long)v & kDescVal);
  }
  __device__ long long lookback(long long mine) {
    volatile unsigned long long* d = B.desc;
    if (threadIdx.x == 0) d[(int64_t)bid * kDescStride] = pack_desc(1, mine);
    const unsigned tag = epoch & 0xFFFFFFu;
    long long v = 0;
    const uint64_t t0 = globaltimer_ns();
    for (int64_t q = threadIdx.x; q < (int64_t)bid; q += blockDim.x) {
      unsigned long long x = d[q * kDescStride];
      unsigned spins = 0;
      while ((unsigned)(x >> 40) != tag || ((x >> 38) & 3u) == 0) {
        if ((++spins & 63) == 0 && (ld_volatile_int(&C->err) != kOk || globaltimer_ns() - t0 > kBarrierLimitNs)) {
          atomicCAS(&C->err, kOk, kErrTimeout);
          x = 0;
          break;
        }
        x = d[q * kDescStride];
      }
      v += (long long)(x & kDescVal);
    }
    const long long excl = block_sum<int64_t>(v, S->scr);
    if (threadIdx.x == 0 && bid == G - 1) d[(int64_t)G * kDescStride] = pack_desc(2, excl + mine);
    return excl;
  }

  __device__ bool select(int algo) {
    for (;;) {
      const int64_t wlo = P().win_lo, wlen = P().win_len;
      int64_t s, e;
      slice(wlo, wlen, &s, &e);
      // Centers keep their active marker for good (a center's label is its
      // arank): an active of this round is told from an earlier round's
      // center by its rank, which is >= r0, the round's first active rank.
      // count this block's alive entries (the first tile stays in registers)
      const int64_t tile = (int64_t)blockDim.x * kSelU;
      int2 a0[kSelU];
      bool alive0[kSelU];
      int64_t mine0 = 0;
#pragma unroll
      for (int q = 0; q < kSelU; ++q) {
        const int64_t i = s + (int64_t)threadIdx.x * kSelU + q;
        a0[q] = i < e ? al_at(i) : make_int2(0, -1);
      }
#pragma unroll
      for (int q = 0; q < kSelU; ++q) {
        alive0[q] = a0[q].y >= 0 && rtag_of(B.rtag, a0[q].y) == 0;
        mine0 += alive0[q] ? 1 : 0;
      }
      int64_t cnt = mine0;
      for (int64_t base = s + tile; base < e; base += 2 * tile) {
        int2 a[2 * kSelU];
#pragma unroll
        for (int q = 0; q < 2 * kSelU; ++q) {
          const int64_t i = base + (int64_t)q * blockDim.x + threadIdx.x;
          a[q] = i < e ? al_at(i) : make_int2(0, -1);
        }
#pragma unroll
        for (int q = 0; q < 2 * kSelU; ++q)
          cnt += (a[q].y >= 0 && rtag_of(B.rtag, a[q].y) == 0) ? 1 : 0;
      }
      cnt = block_sum<int64_t>(cnt, S->scr);
      // this block's first alive entry is number `run` of the window
      int64_t run = lookback(cnt);
      // emit the alive entries of the window numbered below `need`
      const int64_t need = P().need;
      const bool first_window = P().r0 < 0;
      if (run < need) {
        for (int64_t base = s; base < e; base += tile) {
          int2 a[kSelU];
          bool alive[kSelU];
          int64_t mine = 0;
          if (base == s) {
#pragma unroll
            for (int q = 0; q < kSelU; ++q) {
              a[q] = a0[q];
              alive[q] = alive0[q];
            }
            mine = mine0;
          } else {
#pragma unroll
            for (int q = 0; q < kSelU; ++q) {
              const int64_t i = base + (int64_t)threadIdx.x * kSelU + q;
              a[q] = i < e ? al_at(i) : make_int2(0, -1);
            }
#pragma unroll
            for (int q = 0; q < kSelU; ++q) {
              alive[q] = a[q].y >= 0 && rtag_of(B.rtag, a[q].y) == 0;
              mine += alive[q] ? 1 : 0;
            }
          }
          int64_t tot;
          int64_t g = run + block_exclusive_sum<int64_t>(mine, S->scr, &tot);
          bool want[kSelU];
#pragma unroll
          for (int q = 0; q < kSelU; ++q) {
            want[q] = alive[q] && g < need;
            if (want[q] && g == 0 && first_window) C->r0 = a[q].x;
            if (want[q] && g == need - 1) C->cursor_next = base + (int64_t)threadIdx.x * kSelU + q + 1;
            g += alive[q] ? 1 : 0;
          }
          emit_actives(a, want, algo);
          run += tot;
          if (run >= need) break;           // uniform across the block
        }
      }
      if (!sync(3, [&] {
            // the four words this decision reads, loaded side by side
            if (threadIdx.x < 4) {
              const int i = threadIdx.x;
              S->bcast[i] = i == 0 ? (int64_t)(ldcg(B.desc + (int64_t)G * kDescStride) & kDescVal)
                                   : i == 1 ? (int64_t)vload(&C->r0)
                                   : i == 2 ? vload(&C->cursor_next) : (int64_t)vload(&C->act_pack);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
              Coord& c = co();
              Plan& p = S->plan;
              // the last block's inclusive prefix: the window's alive count
              const int64_t total = S->bcast[0];
              p.take = total < c.need ? total : c.need;
              if (c.est) { c.k = total; p.k = total; }   // Sec. 5: all of the window
              if (p.r0 < 0) p.r0 = (int32_t)S->bcast[1];
              const int64_t left = c.est ? 0 : c.need - p.take;
              c.need = left;
              p.need = left;
              if (left == 0) {
                c.cursor = c.est ? c.batch_end : S->bcast[2];
                const unsigned long long pk = (unsigned long long)S->bcast[3];
                p.act_n = (int64_t)(pk >> kPackShift);
                p.act_E = (int64_t)(pk & kPackEdgeMask);
                // adjacency passes over the active rows: attach (and C4 detection)
                c.r_edges = p.act_E * (c.algo == kAlgoC4 ? 2 : 1);
              } else {
                const int64_t lo2 = c.win_lo + c.win_len;
                const int64_t avail = c.al_len - lo2;
                const int64_t alive_left = c.n_alive - (c.k - left);
                if (avail <= 0 || alive_left <= 0) {
                  fail(kErrInternal);
                } else {
                  const int64_t est = (int64_t)((double)left * (double)avail / (double)alive_left * 1.1) + 1024;
                  c.win_lo = lo2;
                  c.win_len = est < avail ? est : avail;
                  p.win_lo = c.win_lo;
                  p.win_len = c.win_len;
                }
              }
            }
          }))
        return false;
      if (P().need == 0) return true;
    }
  }

  // Coordinator: list sizes after the attachment passes.
  __device__ void co_lists_ready() {
    if (threadIdx.x == 0) {
      const unsigned long long pk = vload(&C->new_pack);
      S->plan.new_n = (int64_t)(pk >> kPackShift);
      S->plan.new_E = (int64_t)(pk & kPackEdgeMask);
    }
  }

  // ---------------- createCluster: push a center's rank to its neighbours ----
  // Lanes with push == true try to attach u (state word x, read earlier) to
  // the center of rank r.  All 32 lanes must call it.
  __device__ void attach_one(bool push, int32_t u, int32_t r, uint32_t x) {
    bool fresh = false;
    uint32_t d_old = 0;
    const uint32_t nv = kLab + (uint32_t)r;
    if (push && x > nv) {
      const uint32_t old = atomicMin(B.st + u, nv);
      if (is_alive(old)) {
        fresh = true;
        d_old = deg_of(old);
        set_rtag(B.rtag, u, (uint32_t)P().tag);
      }
    }
    if (fresh) t.attached += 1;
    // The center is the only alive neighbour of a fresh vertex of residual
    // degree 1: nothing to decrement, and no other center can reach it, so
    // its label is already final.
    const bool single = fresh && d_old == 1;
    if (single && CC_IN_BOUNDS(r, B.n, &C->err)) atomicAdd(B.size + r, 1);   // one more member (result unused)
    const bool want = fresh && d_old != 1;
    int64_t row = 0;
    int32_t len = 0;
    if (want) {
      row = __ldg(B.off + u);
      len = (int32_t)(__ldg(B.off + u + 1) - row);
    }
    append_stage(app_buf(), want, u, row, len, new_list());
  }

  __device__ void attach_from_actives(bool skip_blocked) {
    const int64_t an = P().act_n, aE = P().act_E;
    lbs(B.act_e, an, aE, [&](const Lbs& L) {
      bool push[kLbsK];
      int32_t u[kLbsK];
      uint32_t x[kLbsK];
#pragma unroll
      for (int q = 0; q < kLbsK; ++q) {
        push[q] = L.ok(q) && (!skip_blocked || ldcg(B.blk_flag + L.item(q)) == 0);
        u[q] = push[q] ? __ldg(B.col + L.csr(q)) : 0;
        if (push[q] && !CC_IN_BOUNDS(u[q], B.n, &C->err)) push[q] = false;
      }
      // alive (tag 0): try the atomicMin directly; tagged this round (or 15k
      // rounds ago): the state word decides; removed earlier: nothing to do
      uint32_t tg[kLbsK];
#pragma unroll
      for (int q = 0; q < kLbsK; ++q) tg[q] = push[q] ? rtag_of(B.rtag, u[q]) : 16u;
#pragma unroll
      for (int q = 0; q < kLbsK; ++q)
        x[q] = tg[q] == 0 ? 0xFFFFFFFFu : (tg[q] == (uint32_t)P().tag ? ldcg(B.st + u[q]) : 0u);
#pragma unroll
      for (int q = 0; q < kLbsK; ++q) attach_one(push[q], u[q], L.vtx(q), x[q]);
    }, B.act_d, B.act_r);
    append_flush(app_buf(), new_list());
  }

  // ---------------- C4: blocked detection ------------------------------------
  __device__ void c4_detect() {
    const int64_t an = P().act_n, aE = P().act_E;
    lbs(B.act_e, an, aE, [&](const Lbs& L) {
      int32_t u[kLbsK];
#pragma unroll
      for (int q = 0; q < kLbsK; ++q) u[q] = L.ok(q) ? __ldg(B.col + L.csr(q)) : 0;
#pragma unroll
      for (int q = 0; q < kLbsK; ++q) {
        if (!L.ok(q)) continue;
        // an earlier active neighbour: v must wait (isCenter); actives carry
        // this round's tag
        if (rtag_of(B.rtag, u[q]) != (uint32_t)P().tag) continue;
        if (is_active(ldcg(B.st + u[q]))) {
          const int32_t ru = ldcg(B.arank + u[q]);
          if (ru >= P().r0 && ru < L.vtx(q)) B.blk_flag[L.item(q)] = 1;
        }
      }
    }, B.act_d, B.act_r);
  }

  // C4: unblocked actives become centers; blocked ones go to the blocked list.
  __device__ void c4_classify() {
    const int64_t an = P().act_n;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)bid * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)G * blockDim.x) >> 5;
    for (int64_t base = gw * 32; base < an; base += nw * 32) {
      const int64_t j = base + lane;
      bool blocked = false;
      int64_t len = 0, row = 0;
      if (j < an) {
        const int32_t v = ldcg(B.act_v + j), r = ldcg(B.act_r + j);
        if (ldcg(B.blk_flag + j)) {
          blocked = true;
          row = ldcg(B.act_e + j) + ldcg(B.act_d + j);
          len = __ldg(B.off + v + 1) - __ldg(B.off + v);
          t.blocked += 1;
        } else {
          B.st[v] = kActCenter;
          (void)r;
          t.centers += 1;
        }
      }
      warp_append_rows(blocked, (int32_t)j, row, len, 0x7FFFFFFF, blk_list());
      const int64_t ml = warp_max<int64_t>(len);
      if (lane == 0 && ml > 0) atomicMax(&C->blk_maxlen, (unsigned long long)ml);
    }
  }

  // C4, a round's blocked actives one warp each (every one has a warp of its
  // own and no row is longer than warp_resolve_row): the warp waits until each
  // earlier-ranked active neighbour of its vertex is decided; the vertex is a
  // center iff none of them is a center (isCenter), otherwise it joins the
  // lowest-ranked one (every earlier center is known by then, so the label is
  // final at once).  A center then pushes its rank to its alive neighbours
  // (createCluster).  Waits go only to strictly earlier ranks and every vertex
  // has a resident warp, so the earliest undecided vertex always progresses:
  // the same decisions as the fixpoint, in one grid phase.  Every wait is
  // bounded.
  __device__ void c4_resolve_by_warp() {
    const int64_t bn = P().b_n;
    const int lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)(threadIdx.x >> 5) * G + bid;     // warps numbered across the blocks first
    const uint32_t tag = (uint32_t)P().tag;
    const int32_t r0 = P().r0;
    int32_t v = 0, rv = 0;
    int64_t row = 0, len = 0;
    if (gw < bn) {                                                 // warp-uniform
      const int32_t j = ldcg(B.b_j + gw);
      v = ldcg(B.act_v + j);
      rv = ldcg(B.act_r + j);
      row = ldcg(B.b_e + gw) + ldcg(B.b_d + gw);
      len = __ldg(B.off + v + 1) - __ldg(B.off + v);
    }
    int32_t minc = 0x7FFFFFFF;
    bool late = false;
    const uint64_t t0 = globaltimer_ns();
    for (int64_t base = 0; base < len; base += 32) {
      const int64_t e = base + lane;
      if (e >= len || late) continue;
      const int32_t u = __ldg(B.col + row + e);
      if (rtag_of(B.rtag, u) != tag) continue;                     // not an active of this round
      uint32_t x = ldcg(B.st + u);
      if (!is_active(x)) continue;                                 // a decided non-center, or attached
      const int32_t ru = ldcg(B.arank + u);
      if (ru < r0 || ru >= rv) continue;                           // not earlier in this round
      unsigned spins = 0;
      while (x == kActive) {
        if ((++spins & 63) == 0 && (globaltimer_ns() - t0 > kBarrierLimitNs || ld_volatile_int(&C->err) != kOk)) {
          late = true;
          break;
        }
        x = ld_relaxed_u32(B.st + u);
      }
      if (x == kActCenter) minc = ru < minc ? ru : minc;
    }
    if (__any_sync(FULL, late)) {
      if (lane == 0) fail(kErrTimeout);
      return;
    }
    minc = warp_min_i32(minc);
    const bool center = gw < bn && minc == 0x7FFFFFFF;
    if (gw < bn && lane == 0) {
      if (center) {
        atomicExch(B.st + v, kActCenter);
        t.centers += 1;
      } else {
        atomicExch(B.st + v, kLab + (uint32_t)minc);
        t.noncenter += 1;
      }
    }
    // a non-center leaves with its row (the removal phase walks it)
    warp_append_rows(gw < bn && !center && lane == 0, v, row, len, 0, new_list());
    if (!center) return;
    for (int64_t base = 0; base < len; base += 32) {
      const int64_t e = base + lane;
      const bool in = e < len;
      const int32_t u = in ? __ldg(B.col + row + e) : 0;
      const uint32_t tg = in ? rtag_of(B.rtag, u) : 16u;
      const uint32_t x = tg == 0 ? 0xFFFFFFFFu : (tg == tag ? ldcg(B.st + u) : 0u);
      attach_one(in, u, rv, x);
    }
    append_flush(app_buf(), new_list());
  }

  // C4 fixpoint, step 1: look at the earlier active neighbours of every
  // undecided blocked vertex.
  __device__ void c4_fix_scan() {
    const int64_t bn = P().b_n, bE = P().b_E;
    lbs(B.b_e, bn, bE, [&](const Lbs& L) {
#pragma unroll
      for (int i = 0; i < kLbsK; ++i) {
        if (!L.ok(i)) continue;
        const int32_t j = ldcg(B.b_j + L.item(i));
        const int32_t v = ldcg(B.act_v + j), rv = ldcg(B.act_r + j);
        if (ldcg(B.st + v) != kActive) continue;
        const int32_t u = __ldg(B.col + L.edge(i) + ldcg(B.b_d + L.item(i)));
        if (rtag_of(B.rtag, u) != (uint32_t)P().tag) continue;     // not an active of this round
        const uint32_t x = ldcg(B.st + u);
        const int32_t ru = is_active(x) ? ldcg(B.arank + u) : -1;
        if (ru >= P().r0 && ru < rv) {
          if (x == kActCenter) B.hit_c[L.item(i)] = 1;
          else if (x == kActive) B.hit_p[L.item(i)] = 1;
        }
      }
    });
  }

  // C4 fixpoint, step 2: decide (isCenter without waiting) for blocked items
  // q = first, first + stride, ...  The hit flags go back to zero, so they
  // are zero whenever a fixpoint starts.
  __device__ long long c4_fix_decide(int64_t first, int64_t stride) {
    const int64_t bn = P().b_n;
    long long left = 0;
    for (int64_t q = first; q < bn; q += stride) {
      const int32_t j = ldcg(B.b_j + q);
      const int32_t v = ldcg(B.act_v + j), r = ldcg(B.act_r + j);
      (void)r;
      if (ldcg(B.st + v) != kActive) continue;
      if (ldcg(B.hit_c + q)) B.st[v] = kActNon;
      else if (!ldcg(B.hit_p + q)) { B.st[v] = kActCenter; t.centers += 1; }
      else left += 1;
      B.hit_c[q] = 0;
      B.hit_p[q] = 0;
    }
    return left;
  }

  // C4 after the fixpoint: blocked centers push, blocked non-centers pull the
  // lowest center rank among their neighbours.
  __device__ void c4_blocked_attach() {
    const int64_t bn = P().b_n, bE = P().b_E;
    lbs(B.b_e, bn, bE, [&](const Lbs& L) {
#pragma unroll
      for (int i = 0; i < kLbsK; ++i) {
        bool push = false;
        int32_t u = 0, r = 0;
        uint32_t x = 0;
        if (L.ok(i)) {
          const int32_t j = ldcg(B.b_j + L.item(i));
          const int32_t v = ldcg(B.act_v + j);
          r = ldcg(B.act_r + j);
          u = __ldg(B.col + L.edge(i) + ldcg(B.b_d + L.item(i)));
          x = ldcg(B.st + u);
          if (ldcg(B.st + v) == kActCenter) {
            push = true;
          } else if (x == kActCenter) {
            const int32_t ru = ldcg(B.arank + u);
            if (ru >= P().r0) atomicMin(B.pull + L.item(i), ru);   // a center of this round
          }
        }
        attach_one(push, u, r, x);
      }
    });
    append_flush(app_buf(), new_list());
  }

  // C4: a non-center active takes its pulled label and joins the removal list.
  __device__ void c4_pull_finalize() {
    const int64_t bn = P().b_n;
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)bid * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)G * blockDim.x) >> 5;
    for (int64_t base = gw * 32; base < bn; base += nw * 32) {
      const int64_t q = base + lane;
      bool want = false;
      int32_t v = 0;
      int64_t len = 0, row = 0;
      if (q < bn) {
        const int32_t j = ldcg(B.b_j + q);
        v = ldcg(B.act_v + j);
        if (ldcg(B.st + v) == kActNon) {
          const int32_t lab = ldcg(B.pull + q);
          if (lab == 0x7FFFFFFF) fail(kErrInternal);   // a non-center always has a center neighbour
          B.st[v] = kLab + (uint32_t)lab;
          t.noncenter += 1;
          row = ldcg(B.b_e + q) + ldcg(B.b_d + q);
          len = __ldg(B.off + v + 1) - __ldg(B.off + v);
          want = true;
        }
      }
      warp_append_rows(want, v, row, len, 0, new_list());
    }
  }

  // ---------------- removal: residual degrees and the objective --------------
  // ---------------- removal: residual degrees and the objective --------------
  __device__ void decrement() {
    const int64_t nn = P().new_n, nE = P().new_E;
    lbs(B.new_e, nn, nE, [&](const Lbs& L) {
      int32_t w[kLbsK];
      uint32_t lu[kLbsK], x[kLbsK];
#pragma unroll
      for (int q = 0; q < kLbsK; ++q) {
        w[q] = L.ok(q) ? __ldg(B.col + L.csr(q)) : 0;
        lu[q] = (uint32_t)L.vtx(q);                             // the member's (final) label
      }
      uint32_t tg[kLbsK];
#pragma unroll
      for (int q = 0; q < kLbsK; ++q) tg[q] = L.ok(q) && CC_IN_BOUNDS(w[q], B.n, &C->err) ? rtag_of(B.rtag, w[q]) : 16u;
      // alive: decrement; maybe removed this round: the state word decides
      // whether w shares the member's cluster; removed earlier: nothing
      const uint32_t tag = (uint32_t)P().tag;
#pragma unroll
      for (int q = 0; q < kLbsK; ++q) x[q] = tg[q] == tag ? ldcg(B.st + w[q]) : 0;
#pragma unroll
      for (int q = 0; q < kLbsK; ++q) {
        if (!L.ok(q) || !CC_IN_BOUNDS(w[q], B.n, &C->err)) continue;
        if (L.in_row(q) == 0 && CC_IN_BOUNDS(lu[q], B.n, &C->err)) atomicAdd(B.size + lu[q], 1);   // once per removed member
        if (tg[q] == 0) {
          atomicSub(B.st + w[q], 1u);                          // result unused
        } else if (tg[q] != tag) {
          continue;
        } else if (is_active(x[q])) {                          // a center of this round: counted per member
        } else if (x[q] - kLab == lu[q]) {
          t.mm += 1;
        }
      }
    }, B.new_d, B.new_v, B.st, kLab);       // payload: the member's label, st[v] - kLab
  }

  // Reduce the round tallies of this block into the control block.
  __device__ void flush_round_tallies() {
    long long v[5] = {t.centers, t.attached, t.noncenter, t.blocked, (long long)t.mm};
#pragma unroll
    for (int i = 0; i < 5; ++i) v[i] = warp_sum(v[i]);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
      for (int i = 0; i < 5; ++i)
        if (v[i]) atomicAdd(&S->tal[i], (unsigned long long)v[i]);
    }
    __syncthreads();
    if (threadIdx.x < 5) {
      unsigned long long* dst[5] = {reinterpret_cast<unsigned long long*>(&C->r_centers),
                                    reinterpret_cast<unsigned long long*>(&C->r_attached),
                                    reinterpret_cast<unsigned long long*>(&C->r_noncenter),
                                    reinterpret_cast<unsigned long long*>(&C->r_blocked), &C->mm};
      const unsigned long long x = S->tal[threadIdx.x];
      if (x) { atomicAdd(dst[threadIdx.x], x); S->tal[threadIdx.x] = 0; }
    }
    t = Tally{0, 0, 0, 0, 0};
  }
};

// All rounds of one clustering job, run by the team of blocks in k.  The
// state words, the control block and the lists in k.B belong to this job.
__device__ void run_job(K& k, int algo) {
  Shared& S = *k.S;
  Ctl* C = k.C;
  if (algo >= 3) algo -= 2;             // the Sec. 5 schedule: same rounds, C4 or ClusterWild!
  if (k.bid == 0 && threadIdx.x == 0) {
    for (int i = 0; i < 8; ++i) S.co.ph_ns[i] = 0;
    S.co.t0 = globaltimer_ns();
    S.co.round_t0 = S.co.t0;
  }
  __syncthreads();
  if (!k.sync(7, [&] { k.co_init(); })) goto out;

  for (;;) {
    if (S.plan.state == kDone) break;
    if (S.plan.state == kRebuildDelta) {
      if (!k.delta_rebuild()) goto out;
      continue;
    }
    if (S.plan.state == kRebuildDeg) {
      if (!k.rebuild_segment()) goto out;
      continue;
    }
    if (S.plan.state == kRebuildHeavy) {
      if (!k.heavy_fill()) goto out;
      continue;
    }
    if (S.plan.state == kScanH) {
      if (!k.heavy_scan()) goto out;
      continue;
    }
    if (S.plan.state == kDrawBatch) {
      if (!k.draw_batch()) goto out;
      continue;
    }
    if (!k.select(algo)) goto out;
    {
      if (algo == kAlgoCW) {
        k.attach_from_actives(false);
        if (!k.sync(4, [&] { k.co_lists_ready(); })) goto out;
      } else {
        k.c4_detect();
        if (!k.sync(4)) goto out;
        k.c4_classify();
        k.attach_from_actives(true);
        if (!k.sync(4, [&] {
              if (threadIdx.x < 2) S.bcast[threadIdx.x] = (int64_t)vload(threadIdx.x == 0 ? &C->blk_pack : &C->blk_maxlen);
              __syncthreads();
              if (threadIdx.x == 0) {
                const unsigned long long pk = (unsigned long long)S.bcast[0];
                S.plan.b_n = (int64_t)(pk >> kPackShift);
                S.plan.b_E = (int64_t)(pk & kPackEdgeMask);
                S.plan.undecided = S.plan.b_n;
                S.co.fix_iter = 0;
                S.co.r_edges += 2 * S.plan.b_E;       // first fixpoint scan, blocked attach / pull
                const int64_t warps = (int64_t)k.G * (blockDim.x >> 5);
                S.plan.pad4 = (S.plan.b_n > 0 && S.plan.b_n <= warps &&
                               S.bcast[1] <= (int64_t)k.B.tune.warp_resolve_row) ? 1 : 0;
              }
              k.co_lists_ready();
            }))
          goto out;
        if (S.plan.b_n > 0 && S.plan.pad4 == 1) {
          k.c4_resolve_by_warp();
          if (!k.sync(5, [&] { k.co_lists_ready(); })) goto out;
        } else if (S.plan.b_n > 0) {
          // the pull slots were set when the list was built; the hit flags are zero
          auto after_decide = [&](long long left) {
            if (threadIdx.x == 0) {
              S.plan.undecided = left;
              S.co.fix_iter += 1;
              if (S.co.fix_iter > 1) S.co.r_edges += S.plan.b_E;
              if (S.co.fix_iter > S.plan.b_n + 1) { k.fail(kErrInternal); S.plan.undecided = 0; }
            }
          };
          while (S.plan.undecided > 0) {
            k.c4_fix_scan();
            if (S.plan.b_n <= k.B.tune.inline_decide) {
              // a short blocked list: the coordinator decides inside the barrier
              if (!k.sync(5, [&] {
                    const long long left = block_sum<int64_t>(k.c4_fix_decide(threadIdx.x, blockDim.x), S.scr);
                    after_decide(left);
                  }))
                goto out;
            } else {
              if (!k.sync(5, [&] { if (threadIdx.x == 0) C->undecided = 0; })) goto out;
              const long long left = block_sum<int64_t>(
                  k.c4_fix_decide((int64_t)k.bid * blockDim.x + threadIdx.x, (int64_t)k.G * blockDim.x), S.scr);
              if (threadIdx.x == 0 && left)
                atomicAdd(reinterpret_cast<unsigned long long*>(&C->undecided), (unsigned long long)left);
              if (!k.sync(5, [&] { after_decide((long long)vload(&C->undecided)); })) goto out;
            }
          }
          k.c4_blocked_attach();
          if (!k.sync(5)) goto out;
          k.c4_pull_finalize();
          if (!k.sync(5, [&] { k.co_lists_ready(); })) goto out;
        }
      }
      k.decrement();
      k.flush_round_tallies();
      if (!k.sync(6, [&] { k.co_end_round(); })) goto out;
    }
  }
out:
  // coordinator: results for the host
  if (k.bid == 0 && threadIdx.x == 0) {
    C->round = S.co.round;
    C->n_alive = S.co.n_alive;
    C->mc = (unsigned long long)(S.co.n - S.co.clusters);   // member-center edges
    C->done = S.plan.state == kDone ? 1 : 0;
    for (int i = 0; i < 8; ++i) C->ph_ns[i] = S.co.ph_ns[i];
  }
}

__global__ void __launch_bounds__(kThreads, 2) k_rounds(const __grid_constant__ RoundBuffers B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Shared& S = *reinterpret_cast<Shared*>(smem_raw);
  K k{B, B.ctl, &S, gridDim.x, blockIdx.x, 0u, Tally{0, 0, 0, 0, 0}};
  if ((threadIdx.x & 31) == 0) S.u.w.app[threadIdx.x >> 5].n = 0;
  if (threadIdx.x < 5) S.tal[threadIdx.x] = 0;
  // look-back descriptors of an earlier launch could carry the same epochs:
  // clear this block's before the first barrier
  if (threadIdx.x == 0) B.desc[(int64_t)blockIdx.x * kDescStride] = 0;
  __syncthreads();
  run_job(k, vload(&B.ctl->algo));
}


// ---------------------------------------------------------------------------
// Batched engine: many (graph, permutation) jobs in one persistent launch.
// The grid is cut into teams of G blocks; team t runs jobs t, t + T, ...
// (jobs arrive sorted by size, largest first).  A job is the whole pipeline:
// permutation, state set-up, all rounds, objective.  Each team owns one
// scratch slot, reused job after job.
// ---------------------------------------------------------------------------

// pi for the job in k.B, computed by the team: bucket by the top key bits
// (histogram, exclusive scan, scatter), then a counting sort on the next
// kPermSubBits bits plus an insertion sort inside each bucket.  Also writes
// the initial state words.
__device__ bool team_permutation(K& k, uint64_t seed) {
  const RoundBuffers& B = k.B;
  Shared& S = *k.S;
  const int64_t n = B.n;
  int bits = 0;
  while (bits < 12 && (n >> bits) > 768) ++bits;
  const int nb = 1 << bits;
  int64_t* cursor = B.pcnt;            // nb counts, then cursors
  int64_t* start = B.pcnt + nb + 1;    // nb + 1 bucket starts
  const int64_t tid = (int64_t)k.bid * blockDim.x + threadIdx.x, nthr = (int64_t)k.G * blockDim.x;
  // 1: histogram (shared memory, then one global add per non-empty bucket) and state words
  for (int i = threadIdx.x; i < nb; i += blockDim.x) S.u.perm.hist[i] = 0;
  __syncthreads();
  for (int64_t v = tid; v < n; v += nthr) {
    const uint64_t key = perm_key(seed, (uint64_t)v);
    atomicAdd(&S.u.perm.hist[bits == 0 ? 0 : (int)(key >> (64 - bits))], 1);
    const int64_t d = __ldg(B.off + v + 1) - __ldg(B.off + v);
    B.st[v] = kAlive | (uint32_t)d;
    B.size[v] = 0;
    B.hit_c[v] = 0;
    B.hit_p[v] = 0;
  }
  for (int64_t i = tid; i < rtag_words(n); i += nthr) B.rtag[i] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    const int h = S.u.perm.hist[i];
    if (h) atomicAdd(reinterpret_cast<unsigned long long*>(cursor + i), (unsigned long long)h);
  }
  if (!k.sync(7, [&] {
        int64_t run = 0;
        for (int base = 0; base < nb; base += blockDim.x) {
          const int b = base + threadIdx.x;
          const int64_t c = b < nb ? ldcg(cursor + b) : 0;
          int64_t tot;
          const int64_t ex = block_exclusive_sum<int64_t>(c, S.scr, &tot);
          if (b < nb) { start[b] = run + ex; cursor[b] = run + ex; }
          run += tot;
        }
        if (threadIdx.x == 0) start[nb] = run;
      }))
    return false;
  // 2: scatter
  for (int64_t v = tid; v < n; v += nthr) {
    const uint64_t key = perm_key(seed, (uint64_t)v);
    const int b = bits == 0 ? 0 : (int)(key >> (64 - bits));
    const int64_t pos = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(cursor + b), 1ull);
    B.ptmp[pos] = (int32_t)v;
  }
  if (!k.sync(7)) return false;
  // 3: sort each bucket by (key, v)
  PermSmem& P = S.u.perm;
  const int shift = 64 - bits - kPermSubBits;
  for (int b = (int)k.bid; b < nb; b += (int)k.G) {
    const int64_t s0 = ldcg(start + b), len = ldcg(start + b + 1) - s0;
    if (len <= 0) continue;
    if (len > kPermCap) {
      // rare: rank by counting (exact, quadratic)
      for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
        const int32_t vi = ldcg(B.ptmp + s0 + i);
        const uint64_t ki = perm_key(seed, (uint64_t)vi);
        int64_t r = 0;
        for (int64_t j = 0; j < len; ++j) {
          const int32_t vj = ldcg(B.ptmp + s0 + j);
          const uint64_t kj = perm_key(seed, (uint64_t)vj);
          r += (kj < ki || (kj == ki && vj < vi)) ? 1 : 0;
        }
        B.order_w[s0 + r] = vi;
      }
      __syncthreads();
      continue;
    }
    for (int i = threadIdx.x; i < kPermSub; i += blockDim.x) P.cnt[i] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      const int32_t v = ldcg(B.ptmp + s0 + i);
      const uint64_t key = perm_key(seed, (uint64_t)v);
      P.sv[i] = v;
      P.sk[i] = key;
      atomicAdd(&P.cnt[(int)((key >> shift) & (kPermSub - 1))], 1);
    }
    __syncthreads();
    {
      const int i0 = threadIdx.x * 2;
      const int c0 = i0 < kPermSub ? P.cnt[i0] : 0, c1 = i0 + 1 < kPermSub ? P.cnt[i0 + 1] : 0;
      int64_t tot;
      const int64_t ex = block_exclusive_sum<int64_t>(c0 + c1, S.scr, &tot);
      if (i0 < kPermSub) P.cnt[i0] = (int)ex;
      if (i0 + 1 < kPermSub) P.cnt[i0 + 1] = (int)ex + c0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      const uint64_t key = P.sk[i];
      const int pos = atomicAdd(&P.cnt[(int)((key >> shift) & (kPermSub - 1))], 1);
      P.ok[pos] = key;
      P.ov[pos] = P.sv[i];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kPermSub; q += blockDim.x) {
      const int lo = q == 0 ? 0 : P.cnt[q - 1], hi = P.cnt[q];
      for (int i = lo + 1; i < hi; ++i) {
        const uint64_t key = P.ok[i];
        const int32_t v = P.ov[i];
        int j = i - 1;
        while (j >= lo && (key < P.ok[j] || (key == P.ok[j] && v < P.ov[j]))) {
          P.ok[j + 1] = P.ok[j];
          P.ov[j + 1] = P.ov[j];
          --j;
        }
        P.ok[j + 1] = key;
        P.ov[j + 1] = v;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < len; i += blockDim.x) B.order_w[s0 + i] = P.ov[i];
    __syncthreads();
  }
  return k.sync(7);
}

__global__ void __launch_bounds__(kThreads, 2)
k_batch(BatchJob* __restrict__ jobs, int njobs, const RoundBuffers* __restrict__ slots, int team_size, int algo,
        int64_t eps_ppm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Shared& S = *reinterpret_cast<Shared*>(smem_raw);
  __shared__ RoundBuffers rb;
  const unsigned G = (unsigned)team_size;
  const unsigned team = blockIdx.x / G, nteams = gridDim.x / G;
  if (team >= nteams) return;
  Ctl* C = slots[team].ctl;
  K k{rb, C, &S, G, blockIdx.x % G, 0u, Tally{0, 0, 0, 0, 0}};
  if (threadIdx.x == 0) S.plan.state = kDone;
  __syncthreads();
  for (int j = (int)team; j < njobs; j += (int)nteams) {
    if (threadIdx.x == 0) {
      rb = slots[team];
      const BatchJob& jb = jobs[j];
      rb.n = jb.n;
      rb.nnz = jb.nnz;
      rb.max_deg = jb.max_deg;
      rb.off = jb.off;
      rb.col = jb.col;
      rb.dsort = jb.dsort;
      rb.dge = jb.dge;
      rb.nz_static = jb.nz;
      rb.nz_n = jb.nz_n;
      rb.order = rb.order_w;
      rb.stats = nullptr;
      rb.stats_cap = 0;
      if (k.bid == 0) jobs[j].t0 = (int64_t)globaltimer_ns();   // device clock at the job's start
    }
    __syncthreads();
    // zero the permutation counters, reset the control block (not the barrier counters)
    const int64_t zn = 2 * (int64_t)kPermMaxBuckets + 2;
    for (int64_t i = (int64_t)k.bid * blockDim.x + threadIdx.x; i < zn; i += (int64_t)G * blockDim.x) rb.pcnt[i] = 0;
    if (threadIdx.x == 0) rb.desc[(int64_t)k.bid * kDescStride] = 0;   // look-back descriptors of an earlier launch
    if (!k.sync(7, [&] {
          if (threadIdx.x == 0) {
            C->err = 0;
            C->algo = algo;
            C->eps_ppm = eps_ppm;
            C->seed = jobs[j].seed;
            C->mc = 0; C->mm = 0; C->pairs = 0;
            C->undecided = 0; C->h_pack = 0;
            S.plan.state = kRun;
          }
        }))
      break;
    if (!team_permutation(k, jobs[j].seed)) break;
    if ((threadIdx.x & 31) == 0) S.u.w.app[threadIdx.x >> 5].n = 0;
    if (threadIdx.x < 5) S.tal[threadIdx.x] = 0;
    __syncthreads();
    run_job(k, algo);
    if (S.plan.state == kAbort) {
      if (k.bid == 0 && threadIdx.x == 0) jobs[j].err = ld_volatile_int(&C->err) ? ld_volatile_int(&C->err) : kErrInternal;
      break;
    }
    // labels and the pair term of the objective (see k_finalize_labels)
    unsigned long long pairs = 0;
    int32_t* const lab = jobs[j].labels;
    for (int64_t v = (int64_t)k.bid * blockDim.x + threadIdx.x; v < rb.n; v += (int64_t)G * blockDim.x) {
      const uint32_t x = ldcg(rb.st + v);
      if (x == kAlive) {                   // selected with residual degree 0: its own cluster
        if (lab) lab[v] = (int32_t)v;
        continue;
      }
      const int64_t c = is_active(x) ? (int64_t)ldcg(rb.arank + v) : (int64_t)x - kLab;
      if (is_alive(x) || c < 0 || c >= rb.n) { k.fail(kErrInternal); continue; }
      const int32_t cv = ldcg(rb.order + c);
      if (lab) lab[v] = cv;
      if (cv == v) {
        const unsigned long long sz = 1ull + (unsigned long long)ldcg(rb.size + c);
        pairs += sz * (sz - 1) / 2;
      }
    }
    pairs = (unsigned long long)block_sum<int64_t>((int64_t)pairs, S.scr);
    if (threadIdx.x == 0 && pairs) atomicAdd(&C->pairs, pairs);
    if (!k.sync(6, [&] {
          if (threadIdx.x == 0) {
            BatchJob& jb = jobs[j];
            const int done = S.plan.state == kDone && S.co.n_alive == 0;
            jb.rounds = S.co.round;
            jb.D = jb.nnz / 2 - 2 * (int64_t)vload(&C->mc) - (int64_t)vload(&C->mm) + (int64_t)vload(&C->pairs);
            jb.err = done ? 0 : kErrInternal;
            jb.t1 = (int64_t)globaltimer_ns();
            S.plan.state = kDone;
          }
        }))
      break;
  }
}

__global__ void k_init_state(RoundBuffers B, int algo, int64_t eps_ppm, uint64_t seed, int32_t withhold) {
  const int64_t n = B.n;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = __ldg(B.off + v + 1) - __ldg(B.off + v);
    B.st[v] = kAlive | (uint32_t)d;
    B.size[v] = 0;                     // members per center rank
    B.hit_c[v] = 0;                    // C4 fixpoint flags start (and stay) zero
    B.hit_p[v] = 0;
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rtag_words(n); i += (int64_t)gridDim.x * blockDim.x)
    B.rtag[i] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Ctl* C = B.ctl;
    C->algo = algo;
    C->eps_ppm = eps_ppm;
    C->seed = seed;
    C->withhold = withhold;
    C->n_alive = n;
    C->done = n > 0 ? 0 : 1;
  }
}

// Labels (center vertex id = order[center rank]) and the pair term of the
// objective: vertex v is the center of cluster c exactly when order[c] == v,
// and its cluster has 1 + size[c] vertices.
__global__ void k_finalize_labels(RoundBuffers B, int32_t* __restrict__ labels) {
  __shared__ int64_t scr[33];
  const int64_t n = B.n;
  unsigned long long pairs = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t x = B.st[v];
    if (x == kAlive) {                     // selected with residual degree 0: its own cluster
      if (labels) labels[v] = (int32_t)v;
      continue;
    }
    const int64_t c = is_active(x) ? (int64_t)B.arank[v] : (int64_t)x - kLab;   // last round's centers
    if (is_alive(x) || c < 0 || c >= n) {
      atomicCAS(&B.ctl->err, kOk, kErrInternal);
      if (labels) labels[v] = -1;
      continue;
    }
    const int32_t cv = __ldg(B.order + c);
    if (labels) labels[v] = cv;
    if (cv == v) {
      const unsigned long long sz = 1ull + (unsigned long long)B.size[c];
      pairs += sz * (sz - 1) / 2;
    }
  }
  pairs = (unsigned long long)block_sum<int64_t>((int64_t)pairs, scr);
  if (threadIdx.x == 0 && pairs) atomicAdd(&B.ctl->pairs, pairs);
}

}  // namespace

Tuning default_tuning() {
  return Tuning{kLbsBatches, kLbsPfAhead, kInlineH, kInlineDecide, kInlineRebuild, kHeavyShift, kWarpResolveRow};
}

size_t rounds_workspace_bytes(int64_t n, int32_t max_deg, int grid) {
  const size_t nn = (size_t)(n > 0 ? n : 1);
  size_t b = 0;
  b += align_up(sizeof(Ctl));
  b += align_up(4 * nn);                 // st
  b += align_up(4 * ((nn >> 3) + 1));    // rtag
  b += align_up(4 * nn);                 // arank
  b += 2 * align_up(4 * nn) + 2 * align_up(8 * nn);   // act_v, act_r, act_e, act_d
  b += align_up(4 * nn) + 2 * align_up(8 * nn);       // new_v, new_e, new_d
  b += align_up(4 * nn);                 // size
  b += 3 * align_up(4 * nn);             // hv, nz0, nz1
  b += 3 * align_up(nn);                 // blk_flag, hit_c, hit_p
  b += align_up(4 * nn);                 // pull
  b += align_up(4 * nn) + 2 * align_up(8 * nn);       // b_j, b_e, b_d
  b += 2 * align_up(8 * ((size_t)grid + 1));          // blk_a, blk_b
  b += align_up(8 * kDescStride * ((size_t)grid + 1)); // desc
  return b;
}

void rounds_carve(void* ws, int64_t n, int32_t max_deg, int grid, RoundBuffers* B) {
  const size_t nn = (size_t)(n > 0 ? n : 1);
  B->tune = default_tuning();
  char* p = static_cast<char*>(ws);
  auto take = [&](size_t bytes) { char* q = p; p += align_up(bytes); return q; };
  B->ctl = reinterpret_cast<Ctl*>(take(sizeof(Ctl)));
  B->st = reinterpret_cast<uint32_t*>(take(4 * nn));
  B->rtag = reinterpret_cast<uint32_t*>(take(4 * ((nn >> 3) + 1)));
  B->arank = reinterpret_cast<int32_t*>(take(4 * nn));
  B->act_v = reinterpret_cast<int32_t*>(take(4 * nn));
  B->act_r = reinterpret_cast<int32_t*>(take(4 * nn));
  B->act_e = reinterpret_cast<int64_t*>(take(8 * nn));
  B->act_d = reinterpret_cast<int64_t*>(take(8 * nn));
  B->new_v = reinterpret_cast<int32_t*>(take(4 * nn));
  B->new_e = reinterpret_cast<int64_t*>(take(8 * nn));
  B->new_d = reinterpret_cast<int64_t*>(take(8 * nn));
  B->size = reinterpret_cast<int32_t*>(take(4 * nn));
  B->hv = reinterpret_cast<int32_t*>(take(4 * nn));
  B->nz0 = reinterpret_cast<int32_t*>(take(4 * nn));
  B->nz1 = reinterpret_cast<int32_t*>(take(4 * nn));
  B->blk_flag = reinterpret_cast<uint8_t*>(take(nn));
  B->hit_c = reinterpret_cast<uint8_t*>(take(nn));
  B->hit_p = reinterpret_cast<uint8_t*>(take(nn));
  B->pull = reinterpret_cast<int32_t*>(take(4 * nn));
  B->b_j = reinterpret_cast<int32_t*>(take(4 * nn));
  B->b_e = reinterpret_cast<int64_t*>(take(8 * nn));
  B->b_d = reinterpret_cast<int64_t*>(take(8 * nn));
  B->blk_a = reinterpret_cast<int64_t*>(take(8 * ((size_t)grid + 1)));
  B->blk_b = reinterpret_cast<int64_t*>(take(8 * ((size_t)grid + 1)));
  B->desc = reinterpret_cast<unsigned long long*>(take(8 * kDescStride * ((size_t)grid + 1)));
}

int rounds_grid_size(int device) {
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaFuncSetAttribute(k_rounds, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Shared));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_rounds, kThreads, sizeof(Shared));
  if (per < 1) per = 1;
  if (per > 2) per = 2;
  return sms * per;
}

cudaError_t launch_rounds(const RoundBuffers& b, int algo, int64_t eps_ppm, uint64_t seed, int grid,
                          cudaStream_t stream, int32_t withhold) {
  cudaError_t e = cudaMemsetAsync(b.ctl, 0, sizeof(Ctl), stream);
  if (e != cudaSuccess) return e;
  k_init_state<<<grid, 256, 0, stream>>>(b, algo, eps_ppm, seed, withhold);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (b.n <= 0) return cudaSuccess;
  RoundBuffers arg = b;
  void* args[] = {&arg};
  e = cudaFuncSetAttribute(k_rounds, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Shared));
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel((const void*)k_rounds, dim3(grid), dim3(kThreads), args, sizeof(Shared),
                                     stream);
}

cudaError_t launch_finalize_labels(const RoundBuffers& b, int32_t* labels_out, cudaStream_t stream) {
  if (b.n <= 0) return cudaSuccess;
  const int64_t want = (b.n + 255) / 256;
  const int grid = (int)(want < 2048 ? want : 2048);
  k_finalize_labels<<<grid, 256, 0, stream>>>(b, labels_out);
  return cudaGetLastError();
}


int batch_grid_size(int device) {
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Shared));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch, kThreads, sizeof(Shared));
  if (per < 1) per = 1;
  if (per > 2) per = 2;
  return sms * per;
}

size_t batch_slot_bytes(int64_t n_max, int team_size) {
  const size_t nn = (size_t)(n_max > 0 ? n_max : 1);
  return rounds_workspace_bytes(n_max, 0, team_size) + 2 * align_up(4 * nn) +
         align_up(8 * (2 * (size_t)kPermMaxBuckets + 2));
}

void batch_slot_carve(void* ws, int64_t n_max, int team_size, RoundBuffers* B) {
  const size_t nn = (size_t)(n_max > 0 ? n_max : 1);
  rounds_carve(ws, n_max, 0, team_size, B);
  char* p = static_cast<char*>(ws) + rounds_workspace_bytes(n_max, 0, team_size);
  B->order_w = reinterpret_cast<int32_t*>(p); p += align_up(4 * nn);
  B->ptmp = reinterpret_cast<int32_t*>(p); p += align_up(4 * nn);
  B->pcnt = reinterpret_cast<int64_t*>(p);
  B->order = B->order_w;
}

// One block per job (team size 1): no block waits on another, so an
// ordinary launch suffices and several batches can share the GPU.
cudaError_t launch_batch_blocks(const BatchJob* jobs_dev, int njobs, const RoundBuffers* slots_dev, int blocks,
                                int algo, int64_t eps_ppm, cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Shared));
  if (e != cudaSuccess) return e;
  k_batch<<<blocks, kThreads, sizeof(Shared), stream>>>(const_cast<BatchJob*>(jobs_dev), njobs, slots_dev, 1, algo,
                                                       eps_ppm);
  return cudaGetLastError();
}

cudaError_t launch_batch(const BatchJob* jobs_dev, int njobs, const RoundBuffers* slots_dev, int team_size,
                         int grid, int algo, int64_t eps_ppm, cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Shared));
  if (e != cudaSuccess) return e;
  BatchJob* jobs = const_cast<BatchJob*>(jobs_dev);
  void* args[] = {&jobs, &njobs, &slots_dev, &team_size, &algo, &eps_ppm};
  return cudaLaunchCooperativeKernel((const void*)k_batch, dim3(grid), dim3(kThreads), args, sizeof(Shared), stream);
}

}  // namespace ccg
