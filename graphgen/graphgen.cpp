// graphgen.cpp -- seeded synthetic graph generators, shared input module.
//
// Stand-ins for the WebGraph crawls of the paper's Table 1 (not available
// here): Erdos-Renyi G(n,p), a planted partition with Zipf cluster sizes, R-MAT
// and Chung-Lu power-law graphs.  Every generator returns an undirected simple
// graph as a symmetric CSR (int64 offsets, int32 columns, each row sorted, no
// self loops, no duplicates).
//
// This module holds no step of the clustering method.  Both the oracle and the
// CUDA library read the graphs it writes, and neither is linked into it.  Its
// random numbers come from its own SplitMix64 stream (Steele, Lea & Flood,
// OOPSLA 2014): out_j = mix(s0 + (j+1)*gamma), written out here independently.
//
// Results are identical for any thread count: every random draw is a pure
// function of (seed, index).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

inline uint64_t sm_mix(uint64_t x) {
  uint64_t z = x + kGamma;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct Stream {  // SplitMix64 sequence from state s
  uint64_t s;
  explicit Stream(uint64_t seed) : s(seed) {}
  uint64_t next() { uint64_t r = sm_mix(s); s += kGamma; return r; }
  double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }  // [0,1)
  uint64_t below(uint64_t bound) {  // uniform integer in [0,bound), bound >= 1 (Lemire-style reject)
    uint64_t threshold = (0 - bound) % bound;
    for (;;) {
      uint64_t r = next();
      unsigned __int128 m = (unsigned __int128)r * bound;
      if ((uint64_t)m >= threshold) return (uint64_t)(m >> 64);
    }
  }
};

int num_threads(int requested) {
  if (requested > 0) return requested;
  unsigned h = std::thread::hardware_concurrency();
  return h ? (int)h : 1;
}

template <class F>
void parallel_for(int64_t count, int threads, F f) {  // f(begin, end, tid)
  if (count <= 0) return;
  threads = (int)std::max<int64_t>(1, std::min<int64_t>(threads, count));
  std::vector<std::thread> ts;
  for (int t = 0; t < threads; ++t) {
    int64_t b = count * t / threads, e = count * (t + 1) / threads;
    ts.emplace_back([=] { f(b, e, t); });
  }
  for (auto& th : ts) th.join();
}

template <class F>
void parallel_dynamic(int64_t count, int64_t chunk, int threads, F f) {  // f(begin, end)
  std::atomic<int64_t> next{0};
  std::vector<std::thread> ts;
  for (int t = 0; t < threads; ++t)
    ts.emplace_back([&] {
      for (;;) {
        int64_t b = next.fetch_add(chunk);
        if (b >= count) break;
        f(b, std::min(count, b + chunk));
      }
    });
  for (auto& th : ts) th.join();
}

}  // namespace

struct gg_graph {
  int64_t n = 0;
  std::vector<int64_t> off;
  std::vector<int32_t> col;
  std::vector<int32_t> aux;  // planted labels etc. (may be empty)
};

namespace {

// Undirected pairs (u[i], v[i]) -> symmetric simple CSR.  Self loops and
// duplicates are dropped.  Pairs with u < 0 are ignored.
void build_csr(int64_t n, const int32_t* u, const int32_t* v, int64_t m, int threads, gg_graph* g) {
  g->n = n;
  std::vector<std::atomic<uint32_t>> cnt(n > 0 ? n : 1);
  parallel_for(n, threads, [&](int64_t b, int64_t e, int) {
    for (int64_t i = b; i < e; ++i) cnt[i].store(0, std::memory_order_relaxed);
  });
  parallel_for(m, threads, [&](int64_t b, int64_t e, int) {
    for (int64_t i = b; i < e; ++i) {
      if (u[i] < 0 || u[i] == v[i]) continue;
      cnt[u[i]].fetch_add(1, std::memory_order_relaxed);
      cnt[v[i]].fetch_add(1, std::memory_order_relaxed);
    }
  });
  std::vector<int64_t> off(n + 1);
  off[0] = 0;
  for (int64_t i = 0; i < n; ++i) off[i + 1] = off[i] + cnt[i].load(std::memory_order_relaxed);
  std::vector<int32_t> col(off[n] > 0 ? off[n] : 1);
  // Rows above kHub entries are split into one contiguous sub-range per
  // thread (no shared cache lines while filling); other rows use an atomic
  // cursor.
  constexpr uint32_t kHub = 1024;
  std::vector<int32_t> hub_of(n > 0 ? n : 1, -1);
  std::vector<int64_t> hubs;
  for (int64_t i = 0; i < n; ++i)
    if (cnt[i].load(std::memory_order_relaxed) > kHub) { hub_of[i] = (int32_t)hubs.size(); hubs.push_back(i); }
  const int64_t H = (int64_t)hubs.size();
  const int T = (int)std::max<int64_t>(1, std::min<int64_t>(threads, m > 0 ? m : 1));
  std::vector<int64_t> hub_cur((size_t)T * (H > 0 ? H : 1), 0);
  parallel_for(m, T, [&](int64_t b, int64_t e, int t) {
    int64_t* hc = hub_cur.data() + (size_t)t * H;
    for (int64_t i = b; i < e; ++i) {
      if (u[i] < 0 || u[i] == v[i]) continue;
      if (hub_of[u[i]] >= 0) ++hc[hub_of[u[i]]];
      if (hub_of[v[i]] >= 0) ++hc[hub_of[v[i]]];
    }
  });
  for (int64_t h = 0; h < H; ++h) {          // per-thread start inside each hub row
    int64_t run = off[hubs[h]];
    for (int t = 0; t < T; ++t) {
      int64_t c = hub_cur[(size_t)t * H + h];
      hub_cur[(size_t)t * H + h] = run;
      run += c;
    }
  }
  parallel_for(n, threads, [&](int64_t b, int64_t e, int) {
    for (int64_t i = b; i < e; ++i) cnt[i].store(0, std::memory_order_relaxed);
  });
  parallel_for(m, T, [&](int64_t b, int64_t e, int t) {
    int64_t* hc = hub_cur.data() + (size_t)t * H;
    for (int64_t i = b; i < e; ++i) {
      if (u[i] < 0 || u[i] == v[i]) continue;
      const int32_t a = u[i], c = v[i];
      if (hub_of[a] >= 0) col[hc[hub_of[a]]++] = c;
      else col[off[a] + cnt[a].fetch_add(1, std::memory_order_relaxed)] = c;
      if (hub_of[c] >= 0) col[hc[hub_of[c]]++] = a;
      else col[off[c] + cnt[c].fetch_add(1, std::memory_order_relaxed)] = a;
    }
  });
  // sort + dedup each row; new lengths into cnt
  parallel_dynamic(n, 4096, threads, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) {
      int32_t* r0 = col.data() + off[i];
      int32_t* r1 = col.data() + off[i + 1];
      std::sort(r0, r1);
      cnt[i].store((uint32_t)(std::unique(r0, r1) - r0), std::memory_order_relaxed);
    }
  });
  g->off.assign(n + 1, 0);
  for (int64_t i = 0; i < n; ++i) g->off[i + 1] = g->off[i] + cnt[i].load(std::memory_order_relaxed);
  // compact rows leftwards in increasing row order (each destination starts at
  // or before its source, so a forward memmove never clobbers unread data)
  for (int64_t i = 0; i < n; ++i) {
    int64_t len = g->off[i + 1] - g->off[i];
    if (len && g->off[i] != off[i])
      std::memmove(col.data() + g->off[i], col.data() + off[i], (size_t)len * sizeof(int32_t));
  }
  g->col.swap(col);   // capacity may exceed off[n]; only the prefix is used
}

}  // namespace

extern "C" {

// Erdos-Renyi G(n, p) by geometric skipping over the pairs u < v in
// lexicographic order (Batagelj & Brandes 2005), one SplitMix64 stream.
int gg_er(int64_t n, double p, uint64_t seed, int threads, gg_graph** out) {
  if (n < 0 || n > 2147483646 || !(p >= 0.0 && p <= 1.0) || !out) return -1;
  auto* g = new (std::nothrow) gg_graph();
  if (!g) return -3;
  std::vector<int32_t> us, vs;
  if (p > 0.0 && n > 1) {
    Stream rng(seed);
    const double lq = std::log1p(-p);
    int64_t v = 1, w = -1;  // current pair (w, v) with w < v
    for (;;) {
      double r = rng.uniform();
      int64_t skip = (p >= 1.0) ? 0 : (int64_t)std::floor(std::log1p(-r) / lq);
      w += 1 + skip;
      while (w >= v && v < n) { w -= v; ++v; }
      if (v >= n) break;
      us.push_back((int32_t)w);
      vs.push_back((int32_t)v);
    }
  }
  build_csr(n, us.data(), vs.data(), (int64_t)us.size(), num_threads(threads), g);
  *out = g;
  return 0;
}

// Planted partition: n vertices in q clusters of rank-size Zipf sizes
// s_i = min_size + floor((n - q*min_size) * i^-zipf / sum_j j^-zipf), the
// remainder added one by one to the largest clusters; vertices assigned by a
// seeded Fisher-Yates shuffle; each intra pair kept with probability
// min(p_max, mean_intra / (s - 1)); every kept intra edge then dropped with
// probability drop; finally `noise` uniform pairs (self loops redrawn,
// duplicates merged).  aux = planted cluster index of each vertex.
int gg_planted(int64_t n, int64_t q, int64_t min_size, double zipf, double p_max,
               double mean_intra, double drop, int64_t noise, uint64_t seed, int threads,
               gg_graph** out) {
  if (n <= 0 || q <= 0 || q * min_size > n || n > 2147483646 || !out) return -1;
  auto* g = new (std::nothrow) gg_graph();
  if (!g) return -3;
  std::vector<int64_t> size(q);
  double z = 0.0;
  for (int64_t i = 1; i <= q; ++i) z += std::pow((double)i, -zipf);
  int64_t total = 0;
  for (int64_t i = 1; i <= q; ++i) {
    size[i - 1] = min_size + (int64_t)std::floor((double)(n - q * min_size) * std::pow((double)i, -zipf) / z);
    total += size[i - 1];
  }
  for (int64_t i = 0; total < n; i = (i + 1) % q) { size[i] += 1; total += 1; }
  // shuffle vertices, cut into clusters
  std::vector<int32_t> perm(n);
  for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  Stream sh(sm_mix(seed ^ 0x5EED0001ull));
  for (int64_t i = n - 1; i > 0; --i) std::swap(perm[i], perm[(int64_t)sh.below((uint64_t)i + 1)]);
  g->aux.assign(n, 0);
  std::vector<int64_t> start(q + 1, 0);
  for (int64_t c = 0; c < q; ++c) start[c + 1] = start[c] + size[c];
  for (int64_t c = 0; c < q; ++c)
    for (int64_t j = start[c]; j < start[c + 1]; ++j) g->aux[perm[j]] = (int32_t)c;
  // intra edges, cluster by cluster, each with its own stream
  std::vector<std::vector<int32_t>> cu(q), cv(q);
  parallel_dynamic(q, 1, num_threads(threads), [&](int64_t b, int64_t e) {
    for (int64_t c = b; c < e; ++c) {
      int64_t s = size[c];
      if (s < 2) continue;
      double p = std::min(p_max, mean_intra / (double)(s - 1));
      Stream rng(sm_mix(seed ^ (0xC1A5000000000000ull + (uint64_t)c)));
      const double lq = std::log1p(-p);
      int64_t v = 1, w = -1;
      for (;;) {
        double r = rng.uniform();
        int64_t skip = (p >= 1.0) ? 0 : (int64_t)std::floor(std::log1p(-r) / lq);
        w += 1 + skip;
        while (w >= v && v < s) { w -= v; ++v; }
        if (v >= s) break;
        if (rng.uniform() < drop) continue;  // removal of intra edges
        cu[c].push_back(perm[start[c] + w]);
        cv[c].push_back(perm[start[c] + v]);
      }
    }
  });
  std::vector<int32_t> us, vs;
  for (int64_t c = 0; c < q; ++c) {
    us.insert(us.end(), cu[c].begin(), cu[c].end());
    vs.insert(vs.end(), cv[c].begin(), cv[c].end());
    std::vector<int32_t>().swap(cu[c]);
    std::vector<int32_t>().swap(cv[c]);
  }
  Stream nz(sm_mix(seed ^ 0x4015E00000000000ull));
  for (int64_t i = 0; i < noise; ++i) {
    int32_t a, b;
    do { a = (int32_t)nz.below((uint64_t)n); b = (int32_t)nz.below((uint64_t)n); } while (a == b);
    us.push_back(a);
    vs.push_back(b);
  }
  build_csr(n, us.data(), vs.data(), (int64_t)us.size(), num_threads(threads), g);
  *out = g;
  return 0;
}

// R-MAT (Chakrabarti, Zhan & Faloutsos 2004): 2^scale vertices, ef * 2^scale
// generated edges; edge i descends `scale` levels choosing quadrant
// (a, b, c, d) with 32-bit uniforms from the stream seeded mix(seed ^ i).
// Symmetrised, deduplicated, self loops removed; no noise, no relabelling.
int gg_rmat(int scale, int64_t ef, double a, double b, double c, uint64_t seed, int threads,
            gg_graph** out) {
  if (scale < 1 || scale > 30 || ef < 1 || !out) return -1;
  if (!(a >= 0 && b >= 0 && c >= 0 && a + b + c <= 1.0)) return -1;
  auto* g = new (std::nothrow) gg_graph();
  if (!g) return -3;
  const int64_t n = int64_t(1) << scale;
  const int64_t m = ef * n;
  const uint64_t ta = (uint64_t)std::floor(a * 4294967296.0);
  const uint64_t tb = (uint64_t)std::floor((a + b) * 4294967296.0);
  const uint64_t tc = (uint64_t)std::floor((a + b + c) * 4294967296.0);
  std::vector<int32_t> us(m), vs(m);
  int th = num_threads(threads);
  parallel_for(m, th, [&](int64_t lo, int64_t hi, int) {
    for (int64_t i = lo; i < hi; ++i) {
      Stream rng(sm_mix(seed ^ (uint64_t)i));
      uint32_t row = 0, colv = 0;
      uint64_t word = 0;
      for (int l = 0; l < scale; ++l) {
        uint64_t r;
        if ((l & 1) == 0) { word = rng.next(); r = word >> 32; } else { r = word & 0xFFFFFFFFull; }
        // quadrant a: (0,0), b: (0,1), c: (1,0), d: (1,1)
        const uint32_t rbit = r >= tb ? 1u : 0u;
        const uint32_t cbit = ((r >= ta) & (r < tb)) | (r >= tc) ? 1u : 0u;
        row = (row << 1) | rbit;
        colv = (colv << 1) | cbit;
      }
      us[i] = (int32_t)row;
      vs[i] = (int32_t)colv;
    }
  });
  build_csr(n, us.data(), vs.data(), m, th, g);
  *out = g;
  return 0;
}

// Chung-Lu power-law graph: weights w_i = (i + 1)^(-1/(beta-1)), scaled to the
// mean degree d and capped at sqrt(n*d); n*d/2 endpoint pairs drawn
// independently in proportion to w (inverse CDF on the prefix sums);
// deduplicated, self loops removed.
int gg_chung_lu(int64_t n, double d, double beta, uint64_t seed, int threads, gg_graph** out) {
  if (n < 1 || n > 2147483646 || !(d > 0) || !(beta > 1.0) || !out) return -1;
  auto* g = new (std::nothrow) gg_graph();
  if (!g) return -3;
  std::vector<double> w(n), cdf(n);
  double sum = 0.0;
  for (int64_t i = 0; i < n; ++i) { w[i] = std::pow((double)(i + 1), -1.0 / (beta - 1.0)); sum += w[i]; }
  const double cap = std::sqrt((double)n * d);
  double scale = d * (double)n / sum;
  for (int64_t i = 0; i < n; ++i) w[i] = std::min(w[i] * scale, cap);
  double acc = 0.0;
  for (int64_t i = 0; i < n; ++i) { acc += w[i]; cdf[i] = acc; }
  const int64_t m = (int64_t)std::llround((double)n * d / 2.0);
  std::vector<int32_t> us(m), vs(m);
  int th = num_threads(threads);
  parallel_for(m, th, [&](int64_t lo, int64_t hi, int) {
    for (int64_t i = lo; i < hi; ++i) {
      Stream rng(sm_mix(seed ^ (uint64_t)i));
      double x = rng.uniform() * acc, y = rng.uniform() * acc;
      us[i] = (int32_t)std::min<int64_t>(n - 1, std::upper_bound(cdf.begin(), cdf.end(), x) - cdf.begin());
      vs[i] = (int32_t)std::min<int64_t>(n - 1, std::upper_bound(cdf.begin(), cdf.end(), y) - cdf.begin());
    }
  });
  build_csr(n, us.data(), vs.data(), m, th, g);
  *out = g;
  return 0;
}

// Undirected edge list (u[i], v[i]) -> symmetric simple CSR.
int gg_from_edges(int64_t n, const int32_t* u, const int32_t* v, int64_t m, int threads, gg_graph** out) {
  if (n < 0 || m < 0 || !out) return -1;
  for (int64_t i = 0; i < m; ++i)
    if (u[i] < 0 || v[i] < 0 || u[i] >= n || v[i] >= n) return -2;
  auto* g = new (std::nothrow) gg_graph();
  if (!g) return -3;
  build_csr(n, u, v, m, num_threads(threads), g);
  *out = g;
  return 0;
}

int64_t gg_n(const gg_graph* g) { return g->n; }
int64_t gg_nnz(const gg_graph* g) { return g->off.empty() ? 0 : g->off[g->n]; }

int64_t gg_aux_len(const gg_graph* g) { return (int64_t)g->aux.size(); }

int gg_copy(const gg_graph* g, int64_t* off, int32_t* col, int32_t* aux) {
  if (off) std::memcpy(off, g->off.data(), (size_t)(g->n + 1) * sizeof(int64_t));
  if (col && gg_nnz(g)) std::memcpy(col, g->col.data(), (size_t)gg_nnz(g) * sizeof(int32_t));
  if (aux && !g->aux.empty()) std::memcpy(aux, g->aux.data(), g->aux.size() * sizeof(int32_t));
  return 0;
}

void gg_free(gg_graph* g) { delete g; }

}  // extern "C"
