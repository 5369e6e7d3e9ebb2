// cc_rounds.cu -- the bulk-synchronous rounds of C4 and ClusterWild! (Alg. 2)
// as one persistent cooperative kernel.
//
// All rounds run inside a single launch; the barrier at the end of each
// phase is a grid barrier (bounded wait), and the last block to reach a
// barrier does that barrier's serial bookkeeping (the Delta walk, batch size,
// statistics) before releasing the others.  The host is not involved between
// rounds.
//
// Per-vertex state: one 64-bit word st[v] = (hi:int32, lo:uint32)
//   alive ............ hi = 0x7FFFFFFF, lo = residual degree
//   clustered ........ hi = center rank (>= 0), lo = 0
//   active this round  hi = ~rank (< 0), lo = status (undecided/center/non-center)
// Centers keep hi = ~rank after their round; decoding a label is
// hi < 0 ? ~hi : hi.  Because rank order is the clustering order, every
// round's actives have ranks above every earlier center, so "active this
// round" is hi < 0 with ~hi >= r0 (the round's first active rank).
//
// Attachment (createCluster, concurrency rule 2): a center of rank r lowers
// st[u] with a 64-bit atomicMin of (r << 32).  Alive words compare above any
// (r << 32), clustered and active words compare below their own center's, so
// one compare-then-atomicMin does rule 2 and skips dead and active vertices.
//
// Residual degrees live in the low word, so the decrement that follows the
// removal of a vertex is a 32-bit atomic on the same cache sector the alive
// test just read.  Delta_i (max residual degree, exact every round) comes
// from a count-per-degree table kept only for degrees >= th; when no tracked
// vertex is left, a rebuild rescans the alive list, compacts it, lowers th
// and refills the table.
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
constexpr int kHist = 2048;                  // shared-memory window of the degree table
constexpr int32_t kAliveHi = 0x7FFFFFFF;
constexpr uint32_t kUndecided = 0, kCenter = 1, kNonCenter = 2;
constexpr int kAlgoC4 = 1, kAlgoCW = 2;

__device__ __forceinline__ int32_t hi_of(unsigned long long x) { return (int32_t)(x >> 32); }
__device__ __forceinline__ uint32_t lo_of(unsigned long long x) { return (uint32_t)x; }
__device__ __forceinline__ int32_t decode_label(int32_t hi) { return hi < 0 ? ~hi : hi; }
__device__ __forceinline__ unsigned long long word(int32_t hi, uint32_t lo) {
  return ((unsigned long long)(uint32_t)hi << 32) | lo;
}

template <class T>
__device__ __forceinline__ T vload(const T* p) { return *reinterpret_cast<const volatile T*>(p); }

// Shared memory of one block (dynamic: larger than the 48 KB static limit).
struct Shared {
  unsigned gen;
  int leader, ok;
  int64_t scr[33];
  int64_t bcast[2];
  int32_t hist[kHist];
  LbsWarp lbs[kWarps];
  AppendBuf app[kWarps];
};

// Per-thread tallies of one round (flushed at every round end).
struct Tally {
  int32_t centers, attached, noncenter, blocked;
  uint32_t mc, mm;              // member-center and member-member edges
  unsigned long long pairs;     // growth of sum_c C(s_c, 2)
};

struct K {
  const RoundBuffers& B;
  Ctl* C;
  Shared* S;
  unsigned G;
  Tally t;

  // plain control-block fields, always accessed at L2
  __device__ __forceinline__ volatile Ctl* vc() const { return C; }

  // ---------------- degree-count table --------------------------------------
  __device__ void hist_add(int32_t th, uint32_t d, int delta) {
    if ((int64_t)d < th) return;
    const int64_t i = (int64_t)d - th;
    if (i < kHist) atomicAdd(&S->hist[i], delta);
    else atomicAdd(&B.cnt[d], delta);
  }
  __device__ void hist_flush(int32_t th) {
    __syncthreads();
    for (int i = threadIdx.x; i < kHist; i += blockDim.x) {
      const int32_t v = S->hist[i];
      if (v != 0) {
        if ((int64_t)th + i <= (int64_t)B.max_deg) atomicAdd(&B.cnt[th + i], v);
        S->hist[i] = 0;
      }
    }
    __syncthreads();
  }

  // ---------------- barrier --------------------------------------------------
  // Arrive at a grid barrier; the leader books the time since the previous
  // barrier to phase category `cat` (a cheap always-on profile of the rounds).
  __device__ bool arrive(int cat) {
    const bool lead = bar_arrive(reinterpret_cast<GridBarrier*>(&C->bar), G, &S->gen, &S->leader);
    if (lead && threadIdx.x == 0) {
      const unsigned long long now = globaltimer_ns();
      vc()->ph_ns[cat] += now - vc()->ph_t0;
      vc()->ph_t0 = now;
    }
    return lead;
  }
  __device__ bool finish(bool lead) {
    return bar_finish(reinterpret_cast<GridBarrier*>(&C->bar), lead, &S->gen, &C->err, &S->ok);
  }
  __device__ void fail(int code) { atomicCAS(&C->err, kOk, code); }

  __device__ RowList new_list() const { return RowList{B.new_v, B.new_e, B.new_d, nullptr, &C->new_pack}; }
  __device__ RowList blk_list() const { return RowList{B.b_j, B.b_e, B.b_d, nullptr, &C->blk_pack}; }
  __device__ LbsWarp* lbs_ws() const { return &S->lbs[threadIdx.x >> 5]; }
  __device__ AppendBuf* app_buf() const { return &S->app[threadIdx.x >> 5]; }

  // Pair tally of cluster growth: a member joining the cluster of center rank
  // c adds (current size) new pairs, sum_c C(s_c, 2) in total.  Lanes with the
  // same c share one atomic.
  __device__ void add_member(bool want, int32_t c) {
    const int lane = threadIdx.x & 31;
    const int key = want ? c : -1;
    const unsigned grp = __match_any_sync(FULL, key);
    const int leader = __ffs(grp) - 1;
    int old = 0;
    if (want && lane == leader) old = atomicAdd(B.size + c, __popc(grp));
    old = __shfl_sync(FULL, old, leader);
    if (want) t.pairs += 1ull + (unsigned long long)(old + __popc(grp & ((1u << lane) - 1u)));
  }

  __device__ int32_t al_at(int sel, int identity, int64_t i) const {
    if (identity) return (int32_t)i;
    return ldcg((sel ? B.al1 : B.al0) + i);
  }

  // contiguous slice of [lo, lo+len) for this block
  __device__ void slice(int64_t lo, int64_t len, int64_t* s, int64_t* e) const {
    const int64_t chunk = (len + G - 1) / G;
    *s = lo + chunk * blockIdx.x;
    *e = *s + chunk < lo + len ? *s + chunk : lo + len;
    if (*s > *e) *s = *e;
  }

  // Exclusive prefix of blk_a[0..G) in place; returns the total.  Leader only.
  __device__ int64_t leader_prefix_blocks() {
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

  __device__ int64_t leader_max_blocks() {
    int64_t m = 0;
    for (unsigned b = threadIdx.x; b < G; b += blockDim.x) {
      const int64_t x = ldcg(B.blk_b + b);
      m = x > m ? x : m;
    }
    return block_max<int64_t>(m, S->scr);
  }

  // ---------------- round planning (leader) ----------------------------------
  // Sets Delta, k and the first selection window, or asks for a rebuild.
  __device__ void plan_round() {
    __shared__ int s_dec;
    if (threadIdx.x == 0) {
      const int64_t n_alive = vc()->n_alive;
      int dec = 0;
      if (n_alive <= 0) { vc()->done = 1; dec = 1; }
      else if (!vc()->al_identity && vc()->al_len - vc()->cursor > 4 * n_alive + 65536) { vc()->need_rebuild = 1; dec = 1; }
      s_dec = dec;
    }
    __syncthreads();
    if (s_dec) return;
    // walk the degree table down from `top`
    const int32_t th = vc()->th;
    int32_t t = vc()->top;
    int32_t found = -1;
    while (t >= th) {
      // four bins per thread per step: t, t-1, ... t-4*blockDim+1
      int32_t hit = -1;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int32_t d = t - (int32_t)(threadIdx.x * 4 + q);
        if (d >= th && hit < 0 && ldcg(B.cnt + d) > 0) hit = d;
      }
      found = (int32_t)block_max<int64_t>(hit, S->scr);
      if (found >= 0) break;
      t -= 4 * (int32_t)blockDim.x;
    }
    if (threadIdx.x == 0) {
      int32_t delta;
      if (found >= 0) { delta = found; vc()->top = found; }
      else if (th <= 1) { delta = 0; vc()->top = 0; }
      else { vc()->need_rebuild = 1; s_dec = 1; }
      if (!s_dec) {
        const int64_t n_alive = vc()->n_alive;
        int64_t k;
        if (delta <= 0) k = n_alive;
        else {
          const unsigned long long num = (unsigned long long)vc()->eps_ppm * (unsigned long long)n_alive;
          const unsigned long long den = 1000000ull * (unsigned long long)delta;
          k = (int64_t)((num + den - 1) / den);
          if (k < 1) k = 1;
          if (k > n_alive) k = n_alive;
        }
        vc()->delta = delta;
        vc()->k = k;
        vc()->need = k;
        vc()->win_lo = vc()->cursor;
        const int64_t avail = vc()->al_len - vc()->cursor;
        const int64_t est = (int64_t)((double)k * (double)avail / (double)n_alive * 1.05) + 256;
        vc()->win_len = est < avail ? est : avail;
        vc()->act_pack = 0; vc()->new_pack = 0; vc()->blk_pack = 0;
        vc()->r_centers = 0; vc()->r_attached = 0; vc()->r_noncenter = 0; vc()->r_blocked = 0; vc()->r_edges = 0;
        vc()->r0 = -1;
      }
    }
    __syncthreads();
  }

  // ---------------- rebuild: compact the alive list, refill the table -------
  __device__ bool rebuild() {
    const int sel = vload(&C->al_sel), ident = vload(&C->al_identity);
    const int64_t lo = vload(&C->cursor), len = vload(&C->al_len) - lo;
    const int32_t top = vload(&C->top);
    // A: zero the table, count alive and find the largest degree per block
    const int64_t zhi = (int64_t)top + 1 + kHist;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < zhi && i <= (int64_t)B.max_deg + 1 + kHist;
         i += (int64_t)G * blockDim.x)
      B.cnt[i] = 0;
    int64_t s, e;
    slice(lo, len, &s, &e);
    int64_t cnt = 0, mx = 0;
    for (int64_t i = s + threadIdx.x; i < e; i += blockDim.x) {
      const int32_t r = al_at(sel, ident, i);
      const unsigned long long x = ldcg(B.st + __ldg(B.order + r));
      if (hi_of(x) == kAliveHi) { ++cnt; mx = lo_of(x) > mx ? lo_of(x) : mx; }
    }
    cnt = block_sum<int64_t>(cnt, S->scr);
    mx = block_max<int64_t>(mx, S->scr);
    if (threadIdx.x == 0) { B.blk_a[blockIdx.x] = cnt; B.blk_b[blockIdx.x] = mx; }
    bool lead = arrive(0);
    if (lead) {
      const int64_t tot = leader_prefix_blocks();
      const int64_t D = leader_max_blocks();
      if (threadIdx.x == 0) {
        if (tot != vc()->n_alive) fail(kErrInternal);
        vc()->take = tot;                 // new list length
        vc()->top = (int32_t)D;
        const int32_t th = (int32_t)(D >> 2);
        vc()->th = th < 1 ? 1 : th;
      }
    }
    if (!finish(lead)) return false;
    // B: stable compaction into the other buffer, refill the table
    const int32_t th = vload(&C->th);
    int32_t* dst = sel ? B.al0 : B.al1;
    int64_t run = ldcg(B.blk_a + blockIdx.x);
    for (int64_t base = s; base < e; base += blockDim.x) {
      const int64_t i = base + threadIdx.x;
      int32_t r = 0;
      uint32_t d = 0;
      int64_t alive = 0;
      if (i < e) {
        r = al_at(sel, ident, i);
        const unsigned long long x = ldcg(B.st + __ldg(B.order + r));
        if (hi_of(x) == kAliveHi) { alive = 1; d = lo_of(x); }
      }
      int64_t tot;
      const int64_t ex = block_exclusive_sum<int64_t>(alive, S->scr, &tot);
      if (alive) {
        dst[run + ex] = r;
        hist_add(th, d, 1);
      }
      run += tot;
    }
    hist_flush(th);
    lead = arrive(1);
    if (lead) {
      if (threadIdx.x == 0) {
        vc()->al_sel = sel ^ 1;
        vc()->al_identity = 0;
        vc()->al_len = vc()->take;
        vc()->cursor = 0;
        vc()->need_rebuild = 0;
        // a rebuild always leaves a tracked vertex (or Delta = 0), so two in a
        // row without a round in between mean the table is inconsistent
        vc()->rebuilds_in_row += 1;
        if (vc()->rebuilds_in_row > 2) fail(kErrInternal);
      }
      __syncthreads();
      plan_round();
    }
    return finish(lead);
  }

  // ---------------- active-set selection (Alg. 2: A = next k alive of pi) ----
  // Called by every thread of the block for one tile of the window; threads
  // with want == true hold an active vertex v of rank r.
  __device__ void emit_actives(int32_t v, int32_t r, int algo, int32_t th, bool want) {
    uint32_t d = 0;
    int64_t deg0 = 0, row = 0;
    int64_t listed = 0;
    if (want) {
      const unsigned long long x = ldcg(B.st + v);
      d = lo_of(x);
      hist_add(th, d, -1);                      // v leaves the graph this round
      B.size[r] = 0;
      if (d == 0) {                             // no alive neighbour: singleton center
        B.st[v] = word(r, 0);
        t.centers += 1;
      } else {
        row = __ldg(B.off + v);
        deg0 = __ldg(B.off + v + 1) - row;
        B.st[v] = word(~r, algo == kAlgoCW ? kCenter : kUndecided);
        listed = 1;
        if (algo == kAlgoCW) t.centers += 1;
      }
    }
    // one atomic per block and tile on the packed list counter
    int64_t cnt_tot, e_tot;
    const int64_t jx = block_exclusive_sum<int64_t>(listed, S->scr, &cnt_tot);
    const int64_t ex = block_exclusive_sum<int64_t>(listed ? deg0 : 0, S->scr, &e_tot);
    if (cnt_tot == 0) return;
    if (threadIdx.x == 0) {
      const unsigned long long old =
          atomicAdd(&C->act_pack, ((unsigned long long)cnt_tot << kPackShift) | (unsigned long long)e_tot);
      S->bcast[0] = (int64_t)(old >> kPackShift);
      S->bcast[1] = (int64_t)(old & kPackEdgeMask);
    }
    __syncthreads();
    const int64_t j = S->bcast[0] + jx, ep = S->bcast[1] + ex;
    __syncthreads();
    if (listed) {
      B.act_v[j] = v;
      B.act_r[j] = r;
      B.act_e[j] = ep;
      B.act_d[j] = row - ep;
      B.blk_flag[j] = 0;
    }
  }

  __device__ bool select(int algo) {
    for (;;) {
      const int sel = vload(&C->al_sel), ident = vload(&C->al_identity);
      const int64_t wlo = vload(&C->win_lo), wlen = vload(&C->win_len);
      int64_t s, e;
      slice(wlo, wlen, &s, &e);
      // S1: alive count per block
      int64_t cnt = 0;
      for (int64_t i = s + threadIdx.x; i < e; i += blockDim.x) {
        const int32_t r = al_at(sel, ident, i);
        if (hi_of(ldcg(B.st + __ldg(B.order + r))) == kAliveHi) ++cnt;
      }
      cnt = block_sum<int64_t>(cnt, S->scr);
      if (threadIdx.x == 0) B.blk_a[blockIdx.x] = cnt;
      bool lead = arrive(2);
      if (lead) {
        const int64_t tot = leader_prefix_blocks();
        if (threadIdx.x == 0) {
          const int64_t need = vc()->need;
          vc()->take = tot < need ? tot : need;
        }
      }
      if (!finish(lead)) return false;
      // S2: emit the first `take` alive entries of the window
      const int64_t take = vload(&C->take), need = vload(&C->need);
      const bool first_window = vload(&C->r0) < 0;
      const int32_t th = vload(&C->th);
      int64_t run = ldcg(B.blk_a + blockIdx.x);
      if (run < take) {
        for (int64_t base = s; base < e; base += blockDim.x) {
          const int64_t i = base + threadIdx.x;
          int32_t r = 0, v = 0;
          int64_t alive = 0;
          if (i < e) {
            r = al_at(sel, ident, i);
            v = __ldg(B.order + r);
            alive = hi_of(ldcg(B.st + v)) == kAliveHi ? 1 : 0;
          }
          int64_t tot;
          const int64_t g = run + block_exclusive_sum<int64_t>(alive, S->scr, &tot);
          const bool want = alive && g < take;
          if (want && g == 0 && first_window) vc()->r0 = r;
          if (want && take == need && g == take - 1) vc()->cursor_next = i + 1;
          emit_actives(v, r, algo, th, want);
          run += tot;
          if (run >= take) break;           // uniform across the block
        }
      }
      hist_flush(th);
      lead = arrive(3);
      if (lead && threadIdx.x == 0) {
        const int64_t left = vc()->need - vc()->take;
        vc()->need = left;
        if (left == 0) {
          vc()->cursor = vc()->cursor_next;
          const unsigned long long p = vc()->act_pack;
          vc()->act_n = (int64_t)(p >> kPackShift);
          vc()->act_E = (int64_t)(p & kPackEdgeMask);
          // adjacency passes over the active rows: attach (and C4 detection)
          vc()->r_edges = vc()->act_E * (vc()->algo == kAlgoC4 ? 2 : 1);
        } else {
          const int64_t lo2 = vc()->win_lo + vc()->win_len;
          const int64_t avail = vc()->al_len - lo2;
          const int64_t alive_left = vc()->n_alive - (vc()->k - left);
          if (avail <= 0 || alive_left <= 0) {
            fail(kErrInternal);
          } else {
            const int64_t est = (int64_t)((double)left * (double)avail / (double)alive_left * 1.1) + 1024;
            vc()->win_lo = lo2;
            vc()->win_len = est < avail ? est : avail;
          }
        }
      }
      if (!finish(lead)) return false;
      if (vload(&C->need) == 0) return true;
    }
  }

  // ---------------- createCluster: push a center's rank to its neighbours ----
  // Lanes with push == true try to attach u (state word x, read earlier) to
  // the center of rank r.  All 32 lanes must call it.
  __device__ void attach_one(bool push, int32_t u, int32_t r, unsigned long long x, int32_t th) {
    bool fresh = false;
    uint32_t d_old = 0;
    const unsigned long long nv = (unsigned long long)(uint32_t)r << 32;
    if (push && (long long)x > (long long)nv) {
      const unsigned long long old =
          (unsigned long long)atomicMin(reinterpret_cast<long long*>(B.st + u), (long long)nv);
      if (hi_of(old) == kAliveHi) { fresh = true; d_old = lo_of(old); }
    }
    if (fresh) {
      hist_add(th, d_old, -1);
      t.attached += 1;
    }
    // The center is the only alive neighbour of a fresh vertex of residual
    // degree 1: nothing to decrement, and no other center can reach it, so
    // its label is already final.
    const bool single = fresh && d_old == 1;
    if (single) t.mc += 1;
    add_member(single, r);
    const bool want = fresh && d_old != 1;
    int64_t row = 0;
    int32_t len = 0;
    if (want) {
      row = __ldg(B.off + u);
      len = (int32_t)(__ldg(B.off + u + 1) - row);
    }
    append_stage(app_buf(), want, u, row, len, new_list());
  }

  __device__ void attach_from_actives(bool skip_blocked, int32_t th) {
    const int64_t an = vload(&C->act_n), aE = vload(&C->act_E);
    lbs_for_each(B.act_e, an, aE, lbs_ws(), [&](const Lbs& L) {
      bool push[kLbsK];
      int32_t r[kLbsK], u[kLbsK];
      int64_t pos[kLbsK];
      unsigned long long x[kLbsK];
#pragma unroll
      for (int q = 0; q < kLbsK; ++q) {
        push[q] = L.ok(q) && (!skip_blocked || ldcg(B.blk_flag + L.item(q)) == 0);
        r[q] = push[q] ? ldcg(B.act_r + L.item(q)) : 0;
        pos[q] = push[q] ? L.edge(q) + ldcg(B.act_d + L.item(q)) : 0;
      }
#pragma unroll
      for (int q = 0; q < kLbsK; ++q) u[q] = push[q] ? __ldg(B.col + pos[q]) : 0;
#pragma unroll
      for (int q = 0; q < kLbsK; ++q) x[q] = push[q] ? ldcg(B.st + u[q]) : 0;
#pragma unroll
      for (int q = 0; q < kLbsK; ++q) attach_one(push[q], u[q], r[q], x[q], th);
    });
    append_flush(app_buf(), new_list());
  }

  // ---------------- C4: blocked detection ------------------------------------
  __device__ void c4_detect() {
    const int64_t an = vload(&C->act_n), aE = vload(&C->act_E);
    const int32_t r0 = vload(&C->r0);
    lbs_for_each(B.act_e, an, aE, lbs_ws(), [&](const Lbs& L) {
      int32_t rv[kLbsK], u[kLbsK];
      int64_t pos[kLbsK];
#pragma unroll
      for (int q = 0; q < kLbsK; ++q) {
        rv[q] = L.ok(q) ? ldcg(B.act_r + L.item(q)) : 0;
        pos[q] = L.ok(q) ? L.edge(q) + ldcg(B.act_d + L.item(q)) : 0;
      }
#pragma unroll
      for (int q = 0; q < kLbsK; ++q) u[q] = L.ok(q) ? __ldg(B.col + pos[q]) : 0;
#pragma unroll
      for (int q = 0; q < kLbsK; ++q) {
        if (!L.ok(q)) continue;
        const int32_t hw = hi_of(ldcg(B.st + u[q]));
        // an earlier active neighbour: v must wait (isCenter)
        if (hw < 0 && ~hw >= r0 && ~hw < rv[q]) B.blk_flag[L.item(q)] = 1;
      }
    });
  }

  // C4: unblocked actives become centers; blocked ones go to the blocked list.
  __device__ void c4_classify() {
    const int64_t an = vload(&C->act_n);
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
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
          B.st[v] = word(~r, kCenter);
          t.centers += 1;
        }
      }
      warp_append_rows(blocked, (int32_t)j, row, len, 0, blk_list());
    }
  }

  // Reset the per-item scratch of the blocked list (after its counter is known).
  __device__ void c4_blocked_init() {
    const int64_t bn = vload(&C->b_n);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < bn; q += (int64_t)G * blockDim.x) {
      B.hit_c[q] = 0;
      B.hit_p[q] = 0;
      B.pull[q] = 0x7FFFFFFF;
    }
  }

  // C4 fixpoint, step 1: look at the earlier active neighbours of every
  // undecided blocked vertex.
  __device__ void c4_fix_scan() {
    const int64_t bn = vload(&C->b_n), bE = vload(&C->b_E);
    const int32_t r0 = vload(&C->r0);
    lbs_for_each(B.b_e, bn, bE, lbs_ws(), [&](const Lbs& L) {
#pragma unroll
      for (int i = 0; i < kLbsK; ++i) {
        if (!L.ok(i)) continue;
        const int32_t j = ldcg(B.b_j + L.item(i));
        const int32_t v = ldcg(B.act_v + j), rv = ldcg(B.act_r + j);
        if (lo_of(ldcg(B.st + v)) != kUndecided) continue;
        const int32_t u = __ldg(B.col + L.edge(i) + ldcg(B.b_d + L.item(i)));
        const unsigned long long x = ldcg(B.st + u);
        const int32_t hw = hi_of(x);
        if (hw < 0 && ~hw >= r0 && ~hw < rv) {
          const uint32_t su = lo_of(x);
          if (su == kCenter) B.hit_c[L.item(i)] = 1;
          else if (su == kUndecided) B.hit_p[L.item(i)] = 1;
        }
      }
    });
  }

  // C4 fixpoint, step 2: decide (isCenter without waiting).
  __device__ long long c4_fix_decide() {
    const int64_t bn = vload(&C->b_n);
    long long left = 0;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < bn; q += (int64_t)G * blockDim.x) {
      const int32_t j = ldcg(B.b_j + q);
      const int32_t v = ldcg(B.act_v + j), r = ldcg(B.act_r + j);
      if (lo_of(ldcg(B.st + v)) != kUndecided) continue;
      if (ldcg(B.hit_c + q)) B.st[v] = word(~r, kNonCenter);
      else if (!ldcg(B.hit_p + q)) { B.st[v] = word(~r, kCenter); t.centers += 1; }
      else left += 1;
      B.hit_c[q] = 0;
      B.hit_p[q] = 0;
    }
    return left;
  }

  // C4 after the fixpoint: blocked centers push, blocked non-centers pull the
  // lowest center rank among their neighbours.
  __device__ void c4_blocked_attach(int32_t th) {
    const int64_t bn = vload(&C->b_n), bE = vload(&C->b_E);
    const int32_t r0 = vload(&C->r0);
    lbs_for_each(B.b_e, bn, bE, lbs_ws(), [&](const Lbs& L) {
#pragma unroll
      for (int i = 0; i < kLbsK; ++i) {
        bool push = false;
        int32_t u = 0, r = 0;
        unsigned long long x = 0;
        if (L.ok(i)) {
          const int32_t j = ldcg(B.b_j + L.item(i));
          const int32_t v = ldcg(B.act_v + j);
          r = ldcg(B.act_r + j);
          u = __ldg(B.col + L.edge(i) + ldcg(B.b_d + L.item(i)));
          x = ldcg(B.st + u);
          if (lo_of(ldcg(B.st + v)) == kCenter) {
            push = true;
          } else {
            const int32_t hw = hi_of(x);
            if (hw < 0 && ~hw >= r0 && lo_of(x) == kCenter) atomicMin(B.pull + L.item(i), ~hw);
          }
        }
        attach_one(push, u, r, x, th);
      }
    });
    append_flush(app_buf(), new_list());
  }

  // C4: a non-center active takes its pulled label and joins the removal list.
  __device__ void c4_pull_finalize() {
    const int64_t bn = vload(&C->b_n);
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)G * blockDim.x) >> 5;
    for (int64_t base = gw * 32; base < bn; base += nw * 32) {
      const int64_t q = base + lane;
      bool want = false;
      int32_t v = 0;
      int64_t len = 0, row = 0;
      if (q < bn) {
        const int32_t j = ldcg(B.b_j + q);
        v = ldcg(B.act_v + j);
        if (lo_of(ldcg(B.st + v)) == kNonCenter) {
          const int32_t lab = ldcg(B.pull + q);
          if (lab == 0x7FFFFFFF) fail(kErrInternal);   // a non-center always has a center neighbour
          B.st[v] = word(lab, 0);
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
  __device__ void decrement(int32_t th) {
    const unsigned long long p = vload(&C->new_pack);
    const int64_t nn = (int64_t)(p >> kPackShift), nE = (int64_t)(p & kPackEdgeMask);
    lbs_for_each(B.new_e, nn, nE, lbs_ws(), [&](const Lbs& L) {
      int32_t u[kLbsK], w[kLbsK], lu[kLbsK];
      int64_t pos[kLbsK];
      unsigned long long x[kLbsK];
#pragma unroll
      for (int q = 0; q < kLbsK; ++q) {
        u[q] = L.ok(q) ? ldcg(B.new_v + L.item(q)) : 0;
        pos[q] = L.ok(q) ? L.edge(q) + ldcg(B.new_d + L.item(q)) : 0;
      }
#pragma unroll
      for (int q = 0; q < kLbsK; ++q) w[q] = L.ok(q) ? __ldg(B.col + pos[q]) : 0;
#pragma unroll
      for (int q = 0; q < kLbsK; ++q) {
        lu[q] = L.ok(q) ? hi_of(ldcg(B.st + u[q])) : 0;
        x[q] = L.ok(q) ? ldcg(B.st + w[q]) : 0;
      }
#pragma unroll
      for (int q = 0; q < kLbsK; ++q) {
        add_member(L.ok(q) && L.in_row(q) == 0, lu[q]);   // once per removed member
        if (!L.ok(q)) continue;
        const int32_t hw = hi_of(x[q]);
        if (hw == kAliveHi) {
          const uint32_t d = atomicSub(reinterpret_cast<unsigned*>(B.st + w[q]), 1u);   // low word
          if (d == 0) { fail(kErrInternal); continue; }
          hist_add(th, d, -1);
          hist_add(th, d - 1, 1);
        } else if (decode_label(hw) == lu[q]) {
          if (hw < 0) t.mc += 1; else t.mm += 1;
        }
      }
    });
  }

  // Reduce the round tallies of this block into the control block.
  __device__ void flush_round_tallies() {
    const long long v[6] = {t.centers, t.attached, t.noncenter, t.blocked, (long long)t.mc, (long long)t.mm};
    long long* dst[6] = {&C->r_centers, &C->r_attached, &C->r_noncenter, &C->r_blocked,
                         reinterpret_cast<long long*>(&C->mc), reinterpret_cast<long long*>(&C->mm)};
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const long long s = block_sum<int64_t>(v[i], S->scr);
      if (threadIdx.x == 0 && s != 0) atomicAdd(reinterpret_cast<unsigned long long*>(dst[i]), (unsigned long long)s);
    }
    const unsigned long long pr = (unsigned long long)block_sum<int64_t>((int64_t)t.pairs, S->scr);
    if (threadIdx.x == 0 && pr != 0) atomicAdd(&C->pairs, pr);
    t = Tally{0, 0, 0, 0, 0, 0, 0};
  }

  // Leader at the end of a round: statistics, n_i update, plan the next round.
  __device__ void end_round() {
    if (threadIdx.x == 0) {
      const int64_t k = vc()->k;
      const int64_t removed = k + vc()->r_attached;
      const int64_t centers = k - vc()->r_noncenter;
      const int64_t r = vc()->round;
      if (r < B.stats_cap) {
        RoundStat s;
        s.n_alive = vc()->n_alive; s.delta = vc()->delta; s.k = k; s.centers = centers;
        s.removed = removed; s.blocked = vc()->r_blocked; s.edges = vc()->r_edges + (int64_t)(vc()->new_pack & kPackEdgeMask);
        B.stats[r] = s;
      }
      if (vc()->r_centers != centers) fail(kErrInternal);
      vc()->n_alive -= removed;
      if (vc()->n_alive < 0) fail(kErrInternal);
      vc()->round = r + 1;
      vc()->rebuilds_in_row = 0;
      if (vc()->round > vc()->n + 1) fail(kErrInternal);
    }
    __syncthreads();
    plan_round();
  }
};

__global__ void __launch_bounds__(kThreads, 2) k_rounds(const __grid_constant__ RoundBuffers B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Shared& S = *reinterpret_cast<Shared*>(smem_raw);
  K k{B, B.ctl, &S, gridDim.x, Tally{0, 0, 0, 0, 0, 0, 0}};
  for (int i = threadIdx.x; i < kHist; i += blockDim.x) S.hist[i] = 0;
  if ((threadIdx.x & 31) == 0) S.app[threadIdx.x >> 5].n = 0;
  __syncthreads();
  Ctl* C = B.ctl;
  volatile Ctl* V = B.ctl;
  const int algo = V->algo;
  if (blockIdx.x == 0 && threadIdx.x == 0) V->ph_t0 = globaltimer_ns();

  for (;;) {
    if (vload(&C->need_rebuild)) {
      if (!k.rebuild()) return;
      continue;
    }
    if (vload(&C->done)) break;
    if (!k.select(algo)) return;
    const int32_t th = vload(&C->th);
    bool lead;
    if (algo == kAlgoCW) {
      k.attach_from_actives(false, th);
      k.hist_flush(th);
      lead = k.arrive(4);
      if (!k.finish(lead)) return;
    } else {
      k.c4_detect();
      lead = k.arrive(4);
      if (!k.finish(lead)) return;
      k.c4_classify();
      k.attach_from_actives(true, th);
      k.hist_flush(th);
      lead = k.arrive(4);
      if (lead && threadIdx.x == 0) {
        const unsigned long long p = V->blk_pack;
        V->b_n = (int64_t)(p >> kPackShift);
        V->b_E = (int64_t)(p & kPackEdgeMask);
        V->undecided = V->b_n;
        V->fix_iter = 0;
        V->r_edges += 2 * V->b_E;          // blocked attach / pull pass, first fixpoint scan
      }
      if (!k.finish(lead)) return;
      if (vload(&C->b_n) > 0) {
        k.c4_blocked_init();
        lead = k.arrive(5);
        if (!k.finish(lead)) return;
        while (vload(&C->undecided) > 0) {
          k.c4_fix_scan();
          lead = k.arrive(5);
          if (lead && threadIdx.x == 0) V->undecided = 0;
          if (!k.finish(lead)) return;
          const long long left = block_sum<int64_t>(k.c4_fix_decide(), S.scr);
          if (threadIdx.x == 0 && left) atomicAdd(reinterpret_cast<unsigned long long*>(&C->undecided),
                                                  (unsigned long long)left);
          lead = k.arrive(5);
          if (lead && threadIdx.x == 0) {
            V->fix_iter += 1;
            if (V->fix_iter > 1) V->r_edges += V->b_E;
            if (V->fix_iter > V->b_n + 1) { k.fail(kErrInternal); V->undecided = 0; }
          }
          if (!k.finish(lead)) return;
        }
        k.c4_blocked_attach(th);
        k.hist_flush(th);
        lead = k.arrive(5);
        if (!k.finish(lead)) return;
        k.c4_pull_finalize();
        lead = k.arrive(5);
        if (!k.finish(lead)) return;
      }
    }
    k.decrement(th);
    k.hist_flush(th);
    k.flush_round_tallies();
    lead = k.arrive(6);
    if (lead) k.end_round();
    if (!k.finish(lead)) return;
  }
}

__global__ void k_init_state(RoundBuffers B, int algo, int64_t eps_ppm) {
  const int64_t n = B.n;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = __ldg(B.off + v + 1) - __ldg(B.off + v);
    B.st[v] = word(kAliveHi, (uint32_t)d);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Ctl* C = B.ctl;
    C->algo = algo;
    C->eps_ppm = eps_ppm;
    C->n = n;
    C->nnz = B.nnz;
    C->max_deg = B.max_deg;
    C->n_alive = n;
    C->cursor = 0;
    C->al_len = n;
    C->al_identity = 1;
    C->al_sel = 0;
    C->th = B.max_deg + 1;       // nothing tracked: the first rebuild fills the table
    C->top = B.max_deg;
    C->need_rebuild = n > 0 ? 1 : 0;
    C->done = n > 0 ? 0 : 1;
    C->r0 = -1;
  }
}

__global__ void k_finalize_labels(RoundBuffers B, int32_t* __restrict__ labels) {
  const int64_t n = B.n;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t hw = hi_of(B.st[v]);
    const int32_t c = decode_label(hw);
    if (hw == kAliveHi || c < 0 || c >= n) {
      atomicCAS(&B.ctl->err, kOk, kErrInternal);
      labels[v] = -1;
    } else {
      labels[v] = __ldg(B.order + c);
    }
  }
}

}  // namespace

size_t rounds_workspace_bytes(int64_t n, int32_t max_deg, int grid) {
  const size_t nn = (size_t)(n > 0 ? n : 1);
  size_t b = 0;
  b += align_up(sizeof(Ctl));
  b += align_up(8 * nn);                 // st
  b += 2 * align_up(4 * nn);             // al0, al1
  b += 2 * align_up(4 * nn) + 2 * align_up(8 * nn);   // act_v, act_r, act_e, act_d
  b += align_up(4 * nn) + 2 * align_up(8 * nn);       // new_v, new_e, new_d
  b += align_up(4 * nn);                 // size
  b += align_up(4 * ((size_t)max_deg + 2 + kHist));   // cnt
  b += 3 * align_up(nn);                 // blk_flag, hit_c, hit_p
  b += align_up(4 * nn);                 // pull
  b += align_up(4 * nn) + 2 * align_up(8 * nn);       // b_j, b_e, b_d
  b += 2 * align_up(8 * ((size_t)grid + 1));          // blk_a, blk_b
  return b;
}

void rounds_carve(void* ws, int64_t n, int32_t max_deg, int grid, RoundBuffers* B) {
  const size_t nn = (size_t)(n > 0 ? n : 1);
  char* p = static_cast<char*>(ws);
  auto take = [&](size_t bytes) { char* q = p; p += align_up(bytes); return q; };
  B->ctl = reinterpret_cast<Ctl*>(take(sizeof(Ctl)));
  B->st = reinterpret_cast<unsigned long long*>(take(8 * nn));
  B->al0 = reinterpret_cast<int32_t*>(take(4 * nn));
  B->al1 = reinterpret_cast<int32_t*>(take(4 * nn));
  B->act_v = reinterpret_cast<int32_t*>(take(4 * nn));
  B->act_r = reinterpret_cast<int32_t*>(take(4 * nn));
  B->act_e = reinterpret_cast<int64_t*>(take(8 * nn));
  B->act_d = reinterpret_cast<int64_t*>(take(8 * nn));
  B->new_v = reinterpret_cast<int32_t*>(take(4 * nn));
  B->new_e = reinterpret_cast<int64_t*>(take(8 * nn));
  B->new_d = reinterpret_cast<int64_t*>(take(8 * nn));
  B->size = reinterpret_cast<int32_t*>(take(4 * nn));
  B->cnt = reinterpret_cast<int32_t*>(take(4 * ((size_t)max_deg + 2 + kHist)));
  B->blk_flag = reinterpret_cast<uint8_t*>(take(nn));
  B->hit_c = reinterpret_cast<uint8_t*>(take(nn));
  B->hit_p = reinterpret_cast<uint8_t*>(take(nn));
  B->pull = reinterpret_cast<int32_t*>(take(4 * nn));
  B->b_j = reinterpret_cast<int32_t*>(take(4 * nn));
  B->b_e = reinterpret_cast<int64_t*>(take(8 * nn));
  B->b_d = reinterpret_cast<int64_t*>(take(8 * nn));
  B->blk_a = reinterpret_cast<int64_t*>(take(8 * ((size_t)grid + 1)));
  B->blk_b = reinterpret_cast<int64_t*>(take(8 * ((size_t)grid + 1)));
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

cudaError_t launch_rounds(const RoundBuffers& b, int algo, int64_t eps_ppm, int grid, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(b.ctl, 0, sizeof(Ctl), stream);
  if (e != cudaSuccess) return e;
  k_init_state<<<grid, 256, 0, stream>>>(b, algo, eps_ppm);
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
  const int grid = (int)(want < 4096 ? want : 4096);
  k_finalize_labels<<<grid, 256, 0, stream>>>(b, labels_out);
  return cudaGetLastError();
}

}  // namespace ccg
