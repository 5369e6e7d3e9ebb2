/*
 * cc_oracle.c -- plain, serial, obviously-correct CPU oracle for parallel
 * correlation clustering (KwikCluster, C4, ClusterWild!) and for the
 * disagreement objective.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
 * Python binding) includes, links or calls this file.  Only the test suite,
 * the smoke check of the package entry module and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header or table with the CUDA
 * path: the permutation hash below is written out separately here from its
 * published definition.
 *
 * Every routine follows the paper "Parallel Correlation Clustering on Big
 * Graphs" (Pan, Papailiopoulos, Oymak, Recht, Ramchandran, Jordan, 2015):
 *   - objective ............ Sec. 2, definition of correlation clustering
 *                            (disagreements = negative pairs inside clusters
 *                            plus positive edges across clusters)
 *   - KwikCluster(pi) ...... Alg. 1
 *   - C4 / ClusterWild! .... Alg. 2 with createCluster, attemptCluster and
 *                            isCenter (Sec. 2.1, 2.2)
 *
 * Input graph: n vertices, symmetric CSR of the positive edges (off[n+1] int64,
 * col[off[n]] int32), no self loops, no duplicate entries.  Every pair that is
 * not a positive edge is a negative edge (the complete signed graph, Sec. 1).
 *
 * Readings of the paper that this oracle fixes (the CUDA path takes the same):
 *   R1 pi is 0-based: rank[v] in [0,n).  order[r] is the vertex at rank r.
 *      pi = ascending (splitmix64(seed ^ v), v).
 *   R2 attemptCluster tests clusterID(v) (the printed clusterID(u) has no u
 *      in scope).
 *   R3 "n" in eps*n/Delta is n_i, the number of unclustered vertices at the
 *      start of the round (the analysis of Sec. 3 and of the appendix uses
 *      n_i and Delta_i).
 *   R4 k_i = ceil(eps_ppm * n_i / (10^6 * Delta_i)) in integer arithmetic,
 *      clamped to [1, n_i]; k_i = n_i when Delta_i = 0.  eps_ppm =
 *      round(eps * 10^6).
 *   R5 Delta_i = maximum residual degree (alive neighbours only) over the
 *      vertices alive at the start of round i, exact every round.
 *   R6 Gamma(v) = neighbours of v alive at the start of the round.
 *   R7 C4's createCluster labels every alive neighbour, active ones included;
 *      ClusterWild!'s createCluster skips the active set (Gamma(v) \ A).
 *   R8 clusterID holds the center's rank; the reported label is the center's
 *      vertex id.
 *
 * The practical schedule of Sec. 5 ("Estimating but not computing Delta",
 * "Binomial sampling instead of fixed-size batches"), orc_rounds_bsp:
 *   R13 the proxy Delta-hat starts at the maximum degree and halves every P
 *      rounds, P = ceil((2/eps) ln(n log Delta / delta)) with delta = 1/10,
 *      computed in integers: ln x = ln 2 * log2 x with log2 x rounded up to a
 *      bit length, P = ceil(2 * 693147 * L / eps_ppm), L = bits(n) +
 *      bits(bits(max(Delta, 2))) + 4 (bits(x) = number of binary digits, and
 *      4 = bits(10) for 1/delta).  Delta-hat_i = max(1, Delta >> floor(i / P)).
 *   R14 B_i ~ Bin(N_i, eps / Delta-hat_i) with N_i the unprocessed suffix of
 *      pi (ranks cursor .. n-1, clustered or not), drawn as the number of
 *      successes of N_i Bernoulli trials: trial j succeeds when the j-th
 *      output of SplitMix64 seeded with s_i = splitmix64(seed ^ C ^ i)
 *      (C = 0x5851F42D4C957F2D) is below T_i = floor(eps_ppm 2^64 /
 *      (10^6 Delta-hat_i)); every trial succeeds when eps_ppm = 10^6 and
 *      Delta-hat_i = 1.
 *   R15 A_i = the alive vertices among the next B_i ranks of pi; the cursor
 *      moves past all B_i.  Rounds continue while a vertex is unclustered (a
 *      round may have no active vertex).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INF INT64_MAX

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_OOM = -3, ORC_ERR_STATE = -7 };
enum { ORC_ALGO_C4 = 1, ORC_ALGO_CW = 2 };

/* ------------------------------------------------------------------------ */
/* SplitMix64 output function (Steele, Lea & Flood, "Fast splittable        */
/* pseudorandom number generators", OOPSLA 2014): add the golden gamma, then */
/* two xor-shift-multiply steps and a final xor-shift.                        */
/* ------------------------------------------------------------------------ */
uint64_t orc_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Permutation key of vertex v (reading R1). */
uint64_t orc_perm_key(uint64_t seed, int64_t v)
{
    return orc_splitmix64(seed ^ (uint64_t)v);
}

typedef struct { uint64_t key; int64_t v; } orc_kv;

static int orc_kv_cmp(const void *a, const void *b)
{
    const orc_kv *x = (const orc_kv *)a, *y = (const orc_kv *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->v != y->v) return x->v < y->v ? -1 : 1;
    return 0;
}

/* pi (Alg. 1 and Alg. 2, "a random permutation"): order[r] = the vertex with the r-th
 * smallest (key, v).  The comparison is a total order, so the result does not
 * depend on the sort routine. */
int orc_permutation(int64_t n, uint64_t seed, int32_t *order)
{
    if (n < 0 || (n > 0 && !order)) return ORC_ERR_ARG;
    orc_kv *a = (orc_kv *)malloc((size_t)(n > 0 ? n : 1) * sizeof(orc_kv));
    if (!a) return ORC_ERR_OOM;
    for (int64_t v = 0; v < n; ++v) { a[v].key = orc_perm_key(seed, v); a[v].v = v; }
    qsort(a, (size_t)n, sizeof(orc_kv), orc_kv_cmp);
    for (int64_t r = 0; r < n; ++r) order[r] = (int32_t)a[r].v;
    free(a);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* KwikCluster with pi (Alg. 1).  Walking pi in order and skipping clustered  */
/* vertices is the same as repeatedly taking the first remaining vertex of pi */
/* and peeling C_v = {v} u N(v) restricted to the unclustered vertices.       */
/* label[v] = center vertex id.                                               */
/* ------------------------------------------------------------------------ */
int orc_kwik(int64_t n, const int64_t *off, const int32_t *col,
             const int32_t *order, int32_t *label)
{
    if (n < 0) return ORC_ERR_ARG;
    for (int64_t v = 0; v < n; ++v) label[v] = -1;           /* unclustered */
    for (int64_t r = 0; r < n; ++r) {
        int32_t v = order[r];
        if (label[v] != -1) continue;                         /* already peeled */
        label[v] = v;                                         /* v is a center */
        for (int64_t e = off[v]; e < off[v + 1]; ++e) {
            int32_t u = col[e];
            if (label[u] == -1) label[u] = v;                 /* peel N(v) */
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* C4 and ClusterWild! rounds (Alg. 2), executed serially.                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t n_alive;   /* n_i: unclustered vertices at round start          */
    int64_t delta;     /* Delta_i: max residual degree                      */
    int64_t k;         /* |A_i|                                             */
    int64_t centers;   /* cluster centers created this round                */
    int64_t removed;   /* vertices clustered this round (A_i included)      */
    int64_t blocked;   /* C4: actives with an earlier alive neighbour       */
} orc_round_stat;

/* ---- Sec. 5 schedule (readings R13-R15) ----------------------------------- */
static int64_t orc_bits(uint64_t x)
{
    int64_t b = 0;
    while (x) { ++b; x >>= 1; }
    return b;
}

/* Rounds between two halvings of Delta-hat (R13). */
int64_t orc_bsp_period(int64_t n, int64_t max_deg, int64_t eps_ppm)
{
    const int64_t d = max_deg > 2 ? max_deg : 2;
    const int64_t l = orc_bits((uint64_t)n) + orc_bits((uint64_t)orc_bits((uint64_t)d)) + 4;
    const uint64_t num = 2ull * 693147ull * (uint64_t)l;
    return (int64_t)((num + (uint64_t)eps_ppm - 1) / (uint64_t)eps_ppm);
}

/* Delta-hat of round i (R13). */
int64_t orc_bsp_delta_hat(int64_t max_deg, int64_t period, int64_t round)
{
    const int64_t h = round / period;
    const int64_t d = h >= 63 ? 0 : (max_deg >> h);
    return d > 1 ? d : 1;
}

/* T = floor(eps_ppm 2^64 / (10^6 dhat)) by long division, 12 bits at a time
 * (the remainder stays below 2^51); *all = 1 when every trial succeeds. */
uint64_t orc_bsp_threshold(int64_t eps_ppm, int64_t dhat, int *all)
{
    const uint64_t den = 1000000ull * (uint64_t)dhat;
    *all = (uint64_t)eps_ppm >= den;
    if (*all) return UINT64_MAX;
    uint64_t r = (uint64_t)eps_ppm, t = 0;
    for (int step = 0; step < 5; ++step) {            /* 60 bits */
        r <<= 12;
        t = (t << 12) | (r / den);
        r %= den;
    }
    r <<= 4;                                          /* the last 4 bits */
    t = (t << 4) | (r / den);
    return t;
}

/* B_i: successes among the N trials of round i (R14). */
int64_t orc_bsp_batch(uint64_t seed, int64_t round, int64_t trials, uint64_t thr, int all)
{
    if (all) return trials;
    const uint64_t s = orc_splitmix64(seed ^ 0x5851F42D4C957F2Dull ^ (uint64_t)round);
    int64_t b = 0;
    uint64_t state = s;
    for (int64_t j = 0; j < trials; ++j) {
        state += 0x9E3779B97F4A7C15ull;          /* the SplitMix64 generator: */
        uint64_t z = state;                      /* advance, then mix          */
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        b += z < thr;
    }
    return b;
}

/* Round-i batch size (readings R3, R4). */
int64_t orc_batch_size(int64_t eps_ppm, int64_t n_i, int64_t delta_i)
{
    if (n_i <= 0) return 0;
    if (delta_i <= 0) return n_i;
    uint64_t num = (uint64_t)eps_ppm * (uint64_t)n_i;
    uint64_t den = 1000000ull * (uint64_t)delta_i;
    int64_t k = (int64_t)((num + den - 1) / den);
    if (k < 1) k = 1;
    if (k > n_i) k = n_i;
    return k;
}

/*
 * algo: ORC_ALGO_C4 or ORC_ALGO_CW.  eps_ppm in [1, 10^6].
 * delta_mode 0: Delta_i by a scan over all alive vertices, as Alg. 2 states it.
 * delta_mode 1: the same maximum read from a count-per-degree table whose
 *               top pointer only moves down (residual degrees never grow).
 * label_out[v] = center vertex id.  active_round (optional) gets the round in
 * which v was in the active set, or -1.  stats (optional) receives up to
 * stats_cap rounds.  Returns the number of rounds through *rounds_out.
 */
static int rounds_impl(int64_t n, const int64_t *off, const int32_t *col,
                       const int32_t *order, int algo, int64_t eps_ppm, int delta_mode,
                       uint64_t seed, int32_t *label_out, int64_t *rounds_out,
                       int32_t *active_round, orc_round_stat *stats, int64_t stats_cap)
{
    if (n < 0 || eps_ppm < 1 || eps_ppm > 1000000) return ORC_ERR_ARG;
    if (algo != ORC_ALGO_C4 && algo != ORC_ALGO_CW) return ORC_ERR_ARG;
    size_t nn = (size_t)(n > 0 ? n : 1);
    int64_t *rank = (int64_t *)malloc(nn * sizeof(int64_t));
    int64_t *cid = (int64_t *)malloc(nn * sizeof(int64_t));   /* clusterID (rank) */
    int64_t *deg = (int64_t *)malloc(nn * sizeof(int64_t));   /* residual degree */
    char *alive = (char *)malloc(nn);
    char *in_a = (char *)malloc(nn);
    char *center = (char *)malloc(nn);
    int32_t *act = (int32_t *)malloc(nn * sizeof(int32_t));
    int32_t *rem = (int32_t *)malloc(nn * sizeof(int32_t));
    int64_t maxdeg0 = 0;
    for (int64_t v = 0; v < n; ++v)
        if (off[v + 1] - off[v] > maxdeg0) maxdeg0 = off[v + 1] - off[v];
    int64_t *cnt = (int64_t *)calloc((size_t)maxdeg0 + 1, sizeof(int64_t));
    if (!rank || !cid || !deg || !alive || !in_a || !center || !act || !rem || !cnt) {
        free(rank); free(cid); free(deg); free(alive); free(in_a); free(center);
        free(act); free(rem); free(cnt);
        return ORC_ERR_OOM;
    }
    for (int64_t r = 0; r < n; ++r) rank[order[r]] = r;
    for (int64_t v = 0; v < n; ++v) {
        cid[v] = ORC_INF;                                    /* clusterID = inf */
        deg[v] = off[v + 1] - off[v];
        alive[v] = 1; in_a[v] = 0; center[v] = 0;
        cnt[deg[v]] += 1;
        if (active_round) active_round[v] = -1;
    }
    int64_t n_alive = n, cursor = 0, rounds = 0, top = maxdeg0;
    const int64_t period = delta_mode == 2 ? orc_bsp_period(n, maxdeg0, eps_ppm) : 0;
    int status = ORC_OK;

    while (n_alive > 0) {                                    /* while V != empty */
        int64_t delta = 0, na = 0;
        if (delta_mode == 2) {
            /* Sec. 5: Delta-hat, B ~ Bin(unprocessed, eps / Delta-hat), A = the
             * alive vertices among the next B of pi (R13-R15) */
            if (cursor >= n) { status = ORC_ERR_STATE; goto done; }
            delta = orc_bsp_delta_hat(maxdeg0, period, rounds);
            int all;
            const uint64_t thr = orc_bsp_threshold(eps_ppm, delta, &all);
            const int64_t b = orc_bsp_batch(seed, rounds, n - cursor, thr, all);
            for (int64_t r = cursor; r < cursor + b; ++r) {
                int32_t v = order[r];
                if (alive[v]) { act[na++] = v; in_a[v] = 1; }
            }
            cursor += b;
        } else {
            /* Delta = max residual degree over alive vertices (R5) */
            if (delta_mode == 0) {
                for (int64_t v = 0; v < n; ++v)
                    if (alive[v] && deg[v] > delta) delta = deg[v];
            } else {
                while (top > 0 && cnt[top] == 0) --top;
                delta = top;
            }
            /* A = the first k alive vertices of pi (R3, R4) */
            int64_t k = orc_batch_size(eps_ppm, n_alive, delta);
            while (na < k) {
                int32_t v = order[cursor++];
                if (alive[v]) { act[na++] = v; in_a[v] = 1; }
            }
        }
        int64_t centers = 0, blocked = 0, nr = 0;
        /* process A in pi order: attemptCluster (C4) or createCluster (CW) */
        for (int64_t i = 0; i < na; ++i) {
            int32_t v = act[i];
            if (algo == ORC_ALGO_C4) {
                /* blocked: v has an earlier-ranked alive neighbour to wait on */
                int waits = 0;
                for (int64_t e = off[v]; e < off[v + 1]; ++e) {
                    int32_t u = col[e];
                    if (alive[u] && rank[u] < rank[v]) { waits = 1; break; }
                }
                blocked += waits;
                /* attemptCluster(v): clusterID(v) = inf and isCenter(v) */
                if (cid[v] != ORC_INF) continue;
                int is_center = 1;                           /* isCenter(v) */
                for (int64_t e = off[v]; e < off[v + 1]; ++e) {
                    int32_t u = col[e];
                    if (alive[u] && rank[u] < rank[v] && center[u]) { is_center = 0; break; }
                }
                if (!is_center) continue;
            }
            /* createCluster(v); a vertex whose clusterID leaves inf is
             * clustered this round and goes on the removal list */
            center[v] = 1; ++centers;
            if (cid[v] == ORC_INF) rem[nr++] = v;
            cid[v] = rank[v];
            for (int64_t e = off[v]; e < off[v + 1]; ++e) {
                int32_t u = col[e];
                if (!alive[u]) continue;                     /* u not in Gamma(v) */
                if (algo == ORC_ALGO_CW && in_a[u]) continue; /* Gamma(v) \ A */
                if (rank[v] < cid[u]) {
                    if (cid[u] == ORC_INF) rem[nr++] = u;
                    cid[u] = rank[v];
                }
            }
        }
        /* every active vertex is clustered by the end of its round */
        for (int64_t i = 0; i < na; ++i) {
            if (cid[act[i]] == ORC_INF) { status = ORC_ERR_STATE; goto done; }
            if (active_round) active_round[act[i]] = (int32_t)rounds;
            in_a[act[i]] = 0;
        }
        /* remove clustered vertices from V and pi; update residual degrees */
        for (int64_t i = 0; i < nr; ++i) {
            int32_t v = rem[i];
            alive[v] = 0;
            cnt[deg[v]] -= 1;
        }
        for (int64_t i = 0; i < nr; ++i) {
            int32_t v = rem[i];
            for (int64_t e = off[v]; e < off[v + 1]; ++e) {
                int32_t w = col[e];
                if (alive[w]) { cnt[deg[w]] -= 1; deg[w] -= 1; cnt[deg[w]] += 1; }
            }
        }
        if (stats && rounds < stats_cap) {
            stats[rounds].n_alive = n_alive; stats[rounds].delta = delta;
            stats[rounds].k = na; stats[rounds].centers = centers;
            stats[rounds].removed = nr; stats[rounds].blocked = blocked;
        }
        n_alive -= nr;
        ++rounds;
    }
    for (int64_t v = 0; v < n; ++v) label_out[v] = order[cid[v]];
    if (rounds_out) *rounds_out = rounds;
done:
    free(rank); free(cid); free(deg); free(alive); free(in_a); free(center);
    free(act); free(rem); free(cnt);
    return status;
}

int orc_rounds(int64_t n, const int64_t *off, const int32_t *col,
               const int32_t *order, int algo, int64_t eps_ppm, int delta_mode,
               int32_t *label_out, int64_t *rounds_out, int32_t *active_round,
               orc_round_stat *stats, int64_t stats_cap)
{
    if (delta_mode != 0 && delta_mode != 1) return ORC_ERR_ARG;
    return rounds_impl(n, off, col, order, algo, eps_ppm, delta_mode, 0, label_out, rounds_out,
                       active_round, stats, stats_cap);
}

/* The practical schedule of Sec. 5 (R13-R15): same rounds, Delta-hat and the
 * binomial batch of seed `seed` (the seed of pi).  stats[i].delta holds
 * Delta-hat_i and stats[i].k the number of active vertices. */
int orc_rounds_bsp(int64_t n, const int64_t *off, const int32_t *col,
                   const int32_t *order, int algo, int64_t eps_ppm, uint64_t seed,
                   int32_t *label_out, int64_t *rounds_out, int32_t *active_round,
                   orc_round_stat *stats, int64_t stats_cap)
{
    return rounds_impl(n, off, col, order, algo, eps_ppm, 2, seed, label_out, rounds_out,
                       active_round, stats, stats_cap);
}

/* ------------------------------------------------------------------------ */
/* Objective (Sec. 2 definition): disagreements of a labelling.               */
/* ------------------------------------------------------------------------ */

/* By pairs: every unordered pair {u,v} costs 1 when it is a positive edge cut
 * by the labelling or a negative pair placed in one cluster.  O(n^2) time. */
int64_t orc_disagreements_pairs(int64_t n, const int64_t *off, const int32_t *col,
                                const int32_t *label)
{
    char *adj = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    if (!adj) return -1;
    int64_t d = 0;
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t e = off[u]; e < off[u + 1]; ++e) adj[col[e]] = 1;
        for (int64_t v = u + 1; v < n; ++v) {
            int positive = adj[v] != 0;
            int together = label[u] == label[v];
            if (positive != together) ++d;
        }
        for (int64_t e = off[u]; e < off[u + 1]; ++e) adj[col[e]] = 0;
    }
    free(adj);
    return d;
}

static int orc_i32_cmp(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* By counts: with m positive edges, intra = positive edges inside clusters and
 * s_c the cluster sizes, positive edges cut = m - intra and negative pairs
 * inside = sum_c s_c (s_c - 1)/2 - intra, so
 *     D = m - 2 intra + sum_c s_c (s_c - 1)/2.
 * Any int32 label values are accepted. */
int64_t orc_disagreements(int64_t n, const int64_t *off, const int32_t *col,
                          const int32_t *label)
{
    int64_t m2 = off[n], intra2 = 0;
    for (int64_t u = 0; u < n; ++u)
        for (int64_t e = off[u]; e < off[u + 1]; ++e)
            if (label[u] == label[col[e]]) ++intra2;
    int32_t *s = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!s) return -1;
    memcpy(s, label, (size_t)n * sizeof(int32_t));
    qsort(s, (size_t)n, sizeof(int32_t), orc_i32_cmp);
    int64_t pairs = 0;
    for (int64_t i = 0; i < n;) {
        int64_t j = i;
        while (j < n && s[j] == s[i]) ++j;
        pairs += (j - i) * (j - i - 1) / 2;
        i = j;
    }
    free(s);
    return m2 / 2 - intra2 + pairs;   /* m - 2*intra + pairs, with intra = intra2/2 */
}

/* ------------------------------------------------------------------------ */
/* Exhaustive optimum (the OPT of Sec. 2) for n <= 12, by enumerating every   */
/* set partition as a restricted-growth string a[0..n-1]: a[0] = 0 and        */
/* a[i] <= 1 + max(a[0..i-1]).  adj is a row-major n x n 0/1 matrix.           */
/* Returns OPT; *count gets the number of partitions visited (Bell(n)).       */
/* ------------------------------------------------------------------------ */
int64_t orc_opt_bruteforce(int n, const uint8_t *adj, int64_t *count, int32_t *best_label)
{
    if (n < 1 || n > 12) return -1;
    int a[12], mx[12];
    int64_t best = INT64_MAX, visited = 0;
    for (int i = 0; i < n; ++i) { a[i] = 0; mx[i] = 0; }
    for (;;) {
        int64_t d = 0;
        for (int u = 0; u < n; ++u)
            for (int v = u + 1; v < n; ++v)
                if ((adj[u * n + v] != 0) != (a[u] == a[v])) ++d;
        ++visited;
        if (d < best) {
            best = d;
            if (best_label) for (int i = 0; i < n; ++i) best_label[i] = a[i];
        }
        /* next restricted-growth string */
        int i = n - 1;
        while (i > 0 && a[i] == mx[i - 1] + 1) --i;
        if (i == 0) break;
        a[i] += 1;
        mx[i] = a[i] > mx[i - 1] ? a[i] : mx[i - 1];
        for (int j = i + 1; j < n; ++j) { a[j] = 0; mx[j] = mx[i]; }
    }
    if (count) *count = visited;
    return best;
}

/* KwikCluster cost summed over all n! permutations (n <= 10), for the
 * expected-cost statement "E_pi[KC] <= 3 OPT" (Sec. 1, Sec. 3.2).  adj is a
 * row-major n x n 0/1 matrix.  *perms gets n!. */
int64_t orc_kwik_all_perms_total(int n, const uint8_t *adj, int64_t *perms,
                                 int64_t *worst, int64_t *bestc)
{
    if (n < 1 || n > 10) return -1;
    int p[10], lab[10];
    for (int i = 0; i < n; ++i) p[i] = i;
    int64_t total = 0, count = 0, mx = 0, mn = INT64_MAX;
    for (;;) {
        for (int i = 0; i < n; ++i) lab[i] = -1;
        for (int r = 0; r < n; ++r) {
            int v = p[r];
            if (lab[v] != -1) continue;
            lab[v] = v;
            for (int u = 0; u < n; ++u)
                if (adj[v * n + u] && lab[u] == -1) lab[u] = v;
        }
        int64_t d = 0;
        for (int u = 0; u < n; ++u)
            for (int v = u + 1; v < n; ++v)
                if ((adj[u * n + v] != 0) != (lab[u] == lab[v])) ++d;
        total += d; ++count;
        if (d > mx) mx = d;
        if (d < mn) mn = d;
        /* next permutation in lexicographic order */
        int i = n - 2;
        while (i >= 0 && p[i] > p[i + 1]) --i;
        if (i < 0) break;
        int j = n - 1;
        while (p[j] < p[i]) --j;
        int t = p[i]; p[i] = p[j]; p[j] = t;
        for (int l = i + 1, r = n - 1; l < r; ++l, --r) { t = p[l]; p[l] = p[r]; p[r] = t; }
    }
    if (perms) *perms = count;
    if (worst) *worst = mx;
    if (bestc) *bestc = mn;
    return total;
}
