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

struct Shared {
  unsigned gen;
  int leader, ok;
  int64_t scr[33];
  int lbs[kWarps][32];
  int32_t hist[kHist];
};

// Per-thread tallies carried through a round.
struct Tally {
  long long centers, attached, noncenter, blocked, edges;
  unsigned long long mc, mm, pairs;
};

struct K {
  const RoundBuffers& B;
  Ctl* C;
  volatile Ctl* V;     // plain control-block fields, always read at L2
  Shared* S;
  unsigned G;
  Tally t;

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
  __device__ bool arrive() { return bar_arrive(reinterpret_cast<GridBarrier*>(&C->bar), G, &S->gen, &S->leader); }
  __device__ bool finish(bool lead) {
    return bar_finish(reinterpret_cast<GridBarrier*>(&C->bar), lead, &S->gen, &C->err, &S->ok);
  }
  __device__ void fail(int code) { atomicCAS(&C->err, kOk, code); }

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
      const int64_t n_alive = V->n_alive;
      int dec = 0;
      if (n_alive <= 0) { V->done = 1; dec = 1; }
      else if (!V->al_identity && V->al_len - V->cursor > 4 * n_alive + 65536) { V->need_rebuild = 1; dec = 1; }
      s_dec = dec;
    }
    __syncthreads();
    if (s_dec) return;
    // walk the degree table down from `top`
    const int32_t th = V->th;
    int32_t t = V->top;
    int32_t found = -1;
    while (t >= th) {
      const int32_t d = t - (int32_t)threadIdx.x;
      const int32_t hit = (d >= th && ldcg(B.cnt + d) > 0) ? d : -1;
      found = (int32_t)block_max<int64_t>(hit, S->scr);
      if (found >= 0) break;
      t -= (int32_t)blockDim.x;
    }
    if (threadIdx.x == 0) {
      int32_t delta;
      if (found >= 0) { delta = found; V->top = found; }
      else if (th <= 1) { delta = 0; V->top = 0; }
      else { V->need_rebuild = 1; s_dec = 1; }
      if (!s_dec) {
        const int64_t n_alive = V->n_alive;
        int64_t k;
        if (delta <= 0) k = n_alive;
        else {
          const unsigned long long num = (unsigned long long)V->eps_ppm * (unsigned long long)n_alive;
          const unsigned long long den = 1000000ull * (unsigned long long)delta;
          k = (int64_t)((num + den - 1) / den);
          if (k < 1) k = 1;
          if (k > n_alive) k = n_alive;
        }
        V->delta = delta;
        V->k = k;
        V->need = k;
        V->win_lo = V->cursor;
        const int64_t avail = V->al_len - V->cursor;
        const int64_t est = (int64_t)((double)k * (double)avail / (double)n_alive * 1.05) + 256;
        V->win_len = est < avail ? est : avail;
        V->act_pack = 0; V->new_pack = 0; V->blk_pack = 0;
        V->r_centers = 0; V->r_attached = 0; V->r_noncenter = 0; V->r_blocked = 0; V->r_edges = 0;
        V->r0 = -1;
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
    bool lead = arrive();
    if (lead) {
      const int64_t tot = leader_prefix_blocks();
      const int64_t D = leader_max_blocks();
      if (threadIdx.x == 0) {
        if (tot != V->n_alive) fail(kErrInternal);
        V->take = tot;                 // new list length
        V->top = (int32_t)D;
        const int32_t th = (int32_t)(D >> 2);
        V->th = th < 1 ? 1 : th;
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
    lead = arrive();
    if (lead) {
      if (threadIdx.x == 0) {
        V->al_sel = sel ^ 1;
        V->al_identity = 0;
        V->al_len = V->take;
        V->cursor = 0;
        V->need_rebuild = 0;
        // a rebuild always leaves a tracked vertex (or Delta = 0), so two in a
        // row without a round in between mean the table is inconsistent
        V->rebuilds_in_row += 1;
        if (V->rebuilds_in_row > 2) fail(kErrInternal);
      }
      __syncthreads();
      plan_round();
    }
    return finish(lead);
  }

  // ---------------- active-set selection (Alg. 2: A = next k alive of pi) ----
  __device__ void emit_active(int32_t v, int32_t r, int algo, int32_t th, bool want) {
    uint32_t d = 0;
    int64_t deg0 = 0, row = 0;
    bool listed = false;
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
        listed = true;
      }
    }
    int64_t j = 0, ep = 0;
    warp_append_packed(listed, deg0, &C->act_pack, &j, &ep);
    if (listed) {
      B.act_v[j] = v;
      B.act_r[j] = r;
      B.act_e[j] = ep;
      B.act_row[j] = row;
      B.blk_flag[j] = 0;
      if (algo == kAlgoCW) t.centers += 1;
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
      bool lead = arrive();
      if (lead) {
        const int64_t tot = leader_prefix_blocks();
        if (threadIdx.x == 0) {
          const int64_t need = V->need;
          V->take = tot < need ? tot : need;
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
          if (want && g == 0 && first_window) V->r0 = r;
          if (want && take == need && g == take - 1) V->cursor_next = i + 1;
          emit_active(v, r, algo, th, want);
          run += tot;
          if (run >= take) break;           // uniform across the block
        }
      }
      hist_flush(th);
      lead = arrive();
      if (lead && threadIdx.x == 0) {
        const int64_t left = V->need - V->take;
        V->need = left;
        if (left == 0) {
          V->cursor = V->cursor_next;
          const unsigned long long p = V->act_pack;
          V->act_n = (int64_t)(p >> kPackShift);
          V->act_E = (int64_t)(p & kPackEdgeMask);
        } else {
          const int64_t lo2 = V->win_lo + V->win_len;
          const int64_t avail = V->al_len - lo2;
          const int64_t alive_left = V->n_alive - (V->k - left);
          if (avail <= 0 || alive_left <= 0) {
            fail(kErrInternal);
          } else {
            const int64_t est = (int64_t)((double)left * (double)avail / (double)alive_left * 1.1) + 1024;
            V->win_lo = lo2;
            V->win_len = est < avail ? est : avail;
          }
        }
      }
      if (!finish(lead)) return false;
      if (vload(&C->need) == 0) return true;
    }
  }

  // ---------------- createCluster: push a center's rank to its neighbours ----
  // Lanes with `push` set try to attach u to the center of rank r.
  __device__ void attach_lanes(bool push, int32_t u, int32_t r, int32_t th) {
    bool fresh = false;
    uint32_t d_old = 0;
    if (push) {
      const unsigned long long nv = (unsigned long long)(uint32_t)r << 32;
      const unsigned long long x = ldcg(B.st + u);
      if ((long long)x > (long long)nv) {
        const unsigned long long old =
            (unsigned long long)atomicMin(reinterpret_cast<long long*>(B.st + u), (long long)nv);
        if (hi_of(old) == kAliveHi) { fresh = true; d_old = lo_of(old); }
      }
    }
    bool want = false;
    int64_t deg0 = 0, row = 0;
    if (fresh) {
      hist_add(th, d_old, -1);
      t.attached += 1;
      if (d_old == 1) {
        // the center is u's only alive neighbour: nothing to decrement, and
        // no other center can reach u, so the label is already final
        t.mc += 1;
        t.pairs += 1ull + (unsigned long long)atomicAdd(B.size + r, 1);
      } else {
        row = __ldg(B.off + u);
        deg0 = __ldg(B.off + u + 1) - row;
        want = true;
      }
    }
    int64_t j = 0, ep = 0;
    warp_append_packed(want, deg0, &C->new_pack, &j, &ep);
    if (want) {
      B.new_v[j] = u;
      B.new_e[j] = ep;
      B.new_row[j] = row;
    }
  }

  __device__ void attach_from_actives(bool skip_blocked, int32_t th) {
    const int64_t an = vload(&C->act_n), aE = vload(&C->act_E);
    int* wb = S->lbs[threadIdx.x >> 5];
    lbs_for_each(B.act_e, an, aE, wb, [&](bool valid, int64_t j, int64_t k) {
      bool push = false;
      int32_t u = 0, r = 0;
      if (valid) {
        t.edges += 1;
        if (!skip_blocked || ldcg(B.blk_flag + j) == 0) {
          r = ldcg(B.act_r + j);
          u = __ldg(B.col + ldcg(B.act_row + j) + k);
          push = true;
        }
      }
      attach_lanes(push, u, r, th);
    });
  }

  // ---------------- C4: blocked detection ------------------------------------
  __device__ void c4_detect() {
    const int64_t an = vload(&C->act_n), aE = vload(&C->act_E);
    const int32_t r0 = vload(&C->r0);
    int* wb = S->lbs[threadIdx.x >> 5];
    lbs_for_each(B.act_e, an, aE, wb, [&](bool valid, int64_t j, int64_t k) {
      if (!valid) return;
      t.edges += 1;
      const int32_t rv = ldcg(B.act_r + j);
      const int32_t u = __ldg(B.col + ldcg(B.act_row + j) + k);
      const int32_t hw = hi_of(ldcg(B.st + u));
      if (hw < 0) {
        const int32_t ru = ~hw;
        if (ru >= r0 && ru < rv) B.blk_flag[j] = 1;   // an earlier active neighbour: v must wait
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
      int64_t deg0 = 0;
      if (j < an) {
        const int32_t v = ldcg(B.act_v + j), r = ldcg(B.act_r + j);
        if (ldcg(B.blk_flag + j)) {
          blocked = true;
          deg0 = __ldg(B.off + v + 1) - __ldg(B.off + v);
          t.blocked += 1;
        } else {
          B.st[v] = word(~r, kCenter);
          t.centers += 1;
        }
      }
      int64_t q = 0, ep = 0;
      warp_append_packed(blocked, deg0, &C->blk_pack, &q, &ep);
      if (blocked) {
        B.b_j[q] = (int32_t)j;
        B.b_e[q] = ep;
        B.hit_c[q] = 0;
        B.hit_p[q] = 0;
        B.pull[q] = 0x7FFFFFFF;
      }
    }
  }

  // C4 fixpoint, step 1: look at the earlier active neighbours of every
  // undecided blocked vertex.
  __device__ void c4_fix_scan() {
    const int64_t bn = vload(&C->b_n), bE = vload(&C->b_E);
    const int32_t r0 = vload(&C->r0);
    int* wb = S->lbs[threadIdx.x >> 5];
    lbs_for_each(B.b_e, bn, bE, wb, [&](bool valid, int64_t q, int64_t k) {
      if (!valid) return;
      const int32_t j = ldcg(B.b_j + q);
      const int32_t v = ldcg(B.act_v + j), rv = ldcg(B.act_r + j);
      if (lo_of(ldcg(B.st + v)) != kUndecided) return;
      t.edges += 1;
      const int32_t u = __ldg(B.col + ldcg(B.act_row + j) + k);
      const unsigned long long x = ldcg(B.st + u);
      const int32_t hw = hi_of(x);
      if (hw < 0) {
        const int32_t ru = ~hw;
        if (ru >= r0 && ru < rv) {
          const uint32_t su = lo_of(x);
          if (su == kCenter) B.hit_c[q] = 1;
          else if (su == kUndecided) B.hit_p[q] = 1;
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
    int* wb = S->lbs[threadIdx.x >> 5];
    lbs_for_each(B.b_e, bn, bE, wb, [&](bool valid, int64_t q, int64_t k) {
      bool push = false;
      int32_t u = 0, r = 0;
      if (valid) {
        t.edges += 1;
        const int32_t j = ldcg(B.b_j + q);
        const int32_t v = ldcg(B.act_v + j);
        r = ldcg(B.act_r + j);
        u = __ldg(B.col + ldcg(B.act_row + j) + k);
        const uint32_t sv = lo_of(ldcg(B.st + v));
        if (sv == kCenter) {
          push = true;
        } else {
          const unsigned long long x = ldcg(B.st + u);
          const int32_t hw = hi_of(x);
          if (hw < 0 && ~hw >= r0 && lo_of(x) == kCenter) atomicMin(B.pull + q, ~hw);
        }
      }
      attach_lanes(push, u, r, th);
    });
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
      int64_t deg0 = 0, row = 0;
      if (q < bn) {
        const int32_t j = ldcg(B.b_j + q);
        v = ldcg(B.act_v + j);
        if (lo_of(ldcg(B.st + v)) == kNonCenter) {
          const int32_t lab = ldcg(B.pull + q);
          if (lab == 0x7FFFFFFF) fail(kErrInternal);   // a non-center always has a center neighbour
          B.st[v] = word(lab, 0);
          t.noncenter += 1;
          row = __ldg(B.off + v);
          deg0 = __ldg(B.off + v + 1) - row;
          want = true;
        }
      }
      int64_t j2 = 0, ep = 0;
      warp_append_packed(want, deg0, &C->new_pack, &j2, &ep);
      if (want) {
        B.new_v[j2] = v;
        B.new_e[j2] = ep;
        B.new_row[j2] = row;
      }
    }
  }

  // ---------------- removal: residual degrees and the objective --------------
  __device__ void decrement(int32_t th) {
    const unsigned long long p = vload(&C->new_pack);
    const int64_t nn = (int64_t)(p >> kPackShift), nE = (int64_t)(p & kPackEdgeMask);
    int* wb = S->lbs[threadIdx.x >> 5];
    lbs_for_each(B.new_e, nn, nE, wb, [&](bool valid, int64_t j, int64_t k) {
      if (!valid) return;
      t.edges += 1;
      const int32_t u = ldcg(B.new_v + j);
      const int32_t lu = hi_of(ldcg(B.st + u));
      if (k == 0) t.pairs += 1ull + (unsigned long long)atomicAdd(B.size + lu, 1);
      const int32_t w = __ldg(B.col + ldcg(B.new_row + j) + k);
      const unsigned long long x = ldcg(B.st + w);
      const int32_t hw = hi_of(x);
      if (hw == kAliveHi) {
        const uint32_t d = atomicSub(reinterpret_cast<unsigned*>(B.st + w), 1u);   // low word
        if (d == 0) { fail(kErrInternal); return; }
        hist_add(th, d, -1);
        hist_add(th, d - 1, 1);
      } else if (decode_label(hw) == lu) {
        if (hw < 0) t.mc += 1; else t.mm += 1;
      }
    });
  }

  // Reduce the round tallies of this block into the control block.
  __device__ void flush_round_tallies() {
    long long v[5] = {t.centers, t.attached, t.noncenter, t.blocked, t.edges};
    long long* dst[5] = {&C->r_centers, &C->r_attached, &C->r_noncenter, &C->r_blocked, &C->r_edges};
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const long long s = block_sum<int64_t>(v[i], S->scr);
      if (threadIdx.x == 0 && s != 0) atomicAdd(reinterpret_cast<unsigned long long*>(dst[i]), (unsigned long long)s);
    }
    t.centers = t.attached = t.noncenter = t.blocked = t.edges = 0;
  }

  // Leader at the end of a round: statistics, n_i update, plan the next round.
  __device__ void end_round() {
    if (threadIdx.x == 0) {
      const int64_t k = V->k;
      const int64_t removed = k + V->r_attached;
      const int64_t centers = k - V->r_noncenter;
      const int64_t r = V->round;
      if (r < B.stats_cap) {
        RoundStat s;
        s.n_alive = V->n_alive; s.delta = V->delta; s.k = k; s.centers = centers;
        s.removed = removed; s.blocked = V->r_blocked; s.edges = V->r_edges;
        B.stats[r] = s;
      }
      if (V->r_centers != centers) fail(kErrInternal);
      V->n_alive -= removed;
      if (V->n_alive < 0) fail(kErrInternal);
      V->round = r + 1;
      V->rebuilds_in_row = 0;
      if (V->round > V->n + 1) fail(kErrInternal);
    }
    __syncthreads();
    plan_round();
  }
};

__global__ void __launch_bounds__(kThreads, 2) k_rounds(const __grid_constant__ RoundBuffers B) {
  __shared__ Shared S;
  K k{B, B.ctl, B.ctl, &S, gridDim.x, Tally{0, 0, 0, 0, 0, 0, 0, 0}};
  for (int i = threadIdx.x; i < kHist; i += blockDim.x) S.hist[i] = 0;
  __syncthreads();
  Ctl* C = B.ctl;
  volatile Ctl* V = B.ctl;
  const int algo = V->algo;

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
      lead = k.arrive();
      if (!k.finish(lead)) return;
    } else {
      k.c4_detect();
      lead = k.arrive();
      if (!k.finish(lead)) return;
      k.c4_classify();
      k.attach_from_actives(true, th);
      k.hist_flush(th);
      lead = k.arrive();
      if (lead && threadIdx.x == 0) {
        const unsigned long long p = V->blk_pack;
        V->b_n = (int64_t)(p >> kPackShift);
        V->b_E = (int64_t)(p & kPackEdgeMask);
        V->undecided = V->b_n;
        V->fix_iter = 0;
      }
      if (!k.finish(lead)) return;
      if (vload(&C->b_n) > 0) {
        while (vload(&C->undecided) > 0) {
          k.c4_fix_scan();
          lead = k.arrive();
          if (lead && threadIdx.x == 0) V->undecided = 0;
          if (!k.finish(lead)) return;
          const long long left = block_sum<int64_t>(k.c4_fix_decide(), S.scr);
          if (threadIdx.x == 0 && left) atomicAdd(reinterpret_cast<unsigned long long*>(&C->undecided),
                                                  (unsigned long long)left);
          lead = k.arrive();
          if (lead && threadIdx.x == 0) {
            V->fix_iter += 1;
            if (V->fix_iter > V->b_n + 1) { k.fail(kErrInternal); V->undecided = 0; }
          }
          if (!k.finish(lead)) return;
        }
        k.c4_blocked_attach(th);
        k.hist_flush(th);
        lead = k.arrive();
        if (!k.finish(lead)) return;
        k.c4_pull_finalize();
        lead = k.arrive();
        if (!k.finish(lead)) return;
      }
    }
    k.decrement(th);
    k.hist_flush(th);
    k.flush_round_tallies();
    lead = k.arrive();
    if (lead) k.end_round();
    if (!k.finish(lead)) return;
  }
  // objective tallies of the whole run
  const unsigned long long mc = block_sum<int64_t>((int64_t)k.t.mc, S.scr);
  const unsigned long long mm = block_sum<int64_t>((int64_t)k.t.mm, S.scr);
  const unsigned long long pr = block_sum<int64_t>((int64_t)k.t.pairs, S.scr);
  if (threadIdx.x == 0) {
    if (mc) atomicAdd(&C->mc, mc);
    if (mm) atomicAdd(&C->mm, mm);
    if (pr) atomicAdd(&C->pairs, pr);
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
  b += 2 * align_up(4 * nn) + 2 * align_up(8 * nn);   // act_v, act_r, act_e, act_row
  b += align_up(4 * nn) + 2 * align_up(8 * nn);       // new_v, new_e, new_row
  b += align_up(4 * nn);                 // size
  b += align_up(4 * ((size_t)max_deg + 2 + kHist));   // cnt
  b += 3 * align_up(nn);                 // blk_flag, hit_c, hit_p
  b += align_up(4 * nn);                 // pull
  b += align_up(4 * nn) + align_up(8 * nn);           // b_j, b_e
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
  B->act_row = reinterpret_cast<int64_t*>(take(8 * nn));
  B->new_v = reinterpret_cast<int32_t*>(take(4 * nn));
  B->new_e = reinterpret_cast<int64_t*>(take(8 * nn));
  B->new_row = reinterpret_cast<int64_t*>(take(8 * nn));
  B->size = reinterpret_cast<int32_t*>(take(4 * nn));
  B->cnt = reinterpret_cast<int32_t*>(take(4 * ((size_t)max_deg + 2 + kHist)));
  B->blk_flag = reinterpret_cast<uint8_t*>(take(nn));
  B->hit_c = reinterpret_cast<uint8_t*>(take(nn));
  B->hit_p = reinterpret_cast<uint8_t*>(take(nn));
  B->pull = reinterpret_cast<int32_t*>(take(4 * nn));
  B->b_j = reinterpret_cast<int32_t*>(take(4 * nn));
  B->b_e = reinterpret_cast<int64_t*>(take(8 * nn));
  B->blk_a = reinterpret_cast<int64_t*>(take(8 * ((size_t)grid + 1)));
  B->blk_b = reinterpret_cast<int64_t*>(take(8 * ((size_t)grid + 1)));
}

int rounds_grid_size(int device) {
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_rounds, kThreads, 0);
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
  return cudaLaunchCooperativeKernel((const void*)k_rounds, dim3(grid), dim3(kThreads), args, 0, stream);
}

cudaError_t launch_finalize_labels(const RoundBuffers& b, int32_t* labels_out, cudaStream_t stream) {
  if (b.n <= 0) return cudaSuccess;
  const int64_t want = (b.n + 255) / 256;
  const int grid = (int)(want < 4096 ? want : 4096);
  k_finalize_labels<<<grid, 256, 0, stream>>>(b, labels_out);
  return cudaGetLastError();
}

}  // namespace ccg
