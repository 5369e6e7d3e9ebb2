/*
 * cc.h -- C ABI of the GB300 library for parallel correlation clustering.
 *
 * Implements the bulk-synchronous round of C4 and ClusterWild! and the
 * disagreement objective from "Parallel Correlation Clustering on Big Graphs"
 * (Pan, Papailiopoulos, Oymak, Recht, Ramchandran, Jordan; NIPS 2015).
 *
 * Problem (Sec. 2, definition of correlation clustering): a complete signed
 * graph on n vertices is given by its positive edges as a symmetric CSR; every
 * other pair is a negative edge.  A clustering is scored by its disagreements:
 * positive edges between clusters plus negative pairs inside clusters.
 *
 * Method (Alg. 2): pi is a random order of the vertices.  Each round
 *   1. Delta = maximum residual degree of the unclustered graph,
 *   2. A = the next ceil(eps * n_i / Delta) unclustered vertices of pi,
 *   3. centers: all of A (ClusterWild!), or the vertices of A with no
 *      earlier-ranked center among their neighbours (C4; the greedy maximal
 *      independent set of A in pi order),
 *   4. every unclustered neighbour joins its lowest-ranked adjacent center
 *      (createCluster; concurrency rule 2 of Sec. 2.1),
 *   5. clustered vertices leave the graph and residual degrees drop.
 * C4 returns exactly the KwikCluster (Alg. 1) clustering of pi (Sec. 3.2).
 *
 * Readings fixed by this library (the paper leaves them open):
 *   - pi sorts vertices by (splitmix64(seed ^ v), v) ascending; rank 0 first.
 *   - n_i in the batch size is the number of unclustered vertices at round
 *     start; k_i = ceil(eps_ppm * n_i / (10^6 * Delta_i)) in integers, with
 *     eps_ppm = round(eps * 10^6), clamped to [1, n_i]; k_i = n_i if Delta_i = 0.
 *   - Delta_i is exact every round (not the halving estimate of the
 *     implementation appendix).
 *   - C4's createCluster also labels non-center active vertices; ClusterWild!
 *     skips the active set.
 *   - A cluster id is the center's vertex id.
 *
 * Everything runs in the library's own sm_103a kernels on one GPU.  Host code
 * only validates arguments, allocates and launches.
 *
 * Threading: a cc_graph is not re-entrant; calls on one graph must not overlap.
 * Different graphs may be used from different threads.
 * Errors: every call returns CC_OK (0) or a negative CC_ERR_* code; nothing
 * else crosses the ABI.  After CC_ERR_INVALID_ARG the graph stays usable.
 */
#ifndef CC_H_
#define CC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define CC_OK                 0
#define CC_ERR_INVALID_ARG   -1   /* bad argument (null pointer, eps out of (0,1], ...) */
#define CC_ERR_INVALID_GRAPH -2   /* CSR is not a symmetric simple graph           */
#define CC_ERR_OOM           -3   /* device or host allocation failed              */
#define CC_ERR_CUDA          -4   /* a CUDA runtime call failed                    */
#define CC_ERR_TIMEOUT       -5   /* a bounded device-side wait ran out            */
#define CC_ERR_BUSY          -6   /* server queue full / job not finished          */
#define CC_ERR_INTERNAL      -7   /* device-side consistency check failed          */

/* ---- algorithms ---------------------------------------------------------- */
#define CC_ALGO_C4          1     /* serializable: equals KwikCluster(pi)          */
#define CC_ALGO_CLUSTERWILD 2     /* coordination-free                             */
/* The same two with the practical schedule of Sec. 5 (estimating Delta,
 * binomial batches) instead of Alg. 2's exact Delta_i and k_i:
 *   Delta-hat starts at the maximum degree and halves every
 *   P = ceil(2 * 693147 * L / eps_ppm) rounds, L = bits(n) +
 *   bits(bits(max(Delta, 2))) + 4 (the paper's (2/eps) ln(n log Delta /
 *   delta) with delta = 1/10, logarithms rounded up to bit lengths);
 *   B_i = the number of the round's n - cursor draws below
 *   floor(eps_ppm 2^64 / (10^6 Delta-hat_i)) (all when that is 2^64), draw j
 *   being the j-th output of SplitMix64 seeded with
 *   splitmix64(seed ^ 0x5851F42D4C957F2D ^ i), seed = the seed of pi;
 *   A_i = the alive vertices among the next B_i ranks of pi.
 * cc_round_stats.delta then reports Delta-hat_i and .k the active count. */
#define CC_ALGO_C4_EST          3
#define CC_ALGO_CLUSTERWILD_EST 4
/* C4 with no rounds at all: the asynchronous execution of Alg. 3 with
 * attemptCluster.  Vertices are decided in pi order by whichever warp holds
 * them; a vertex waits (bounded) only for its undecided earlier-ranked
 * neighbours, and becomes a center iff none of them is one.  The output
 * equals KwikCluster(pi) and CC_ALGO_C4 (Sec. 4).  eps is checked but
 * unused; rounds_out is 0; cc_cluster_ex writes one statistics record for
 * the whole run (n_alive = k = removed = n, delta = the maximum degree,
 * centers, blocked = vertices that waited on an undecided neighbour,
 * edges = adjacency entries read by the decisions, ns = 0).
 * cc_cluster / cc_cluster_ex only (not the batch or server entry points). */
#define CC_ALGO_C4_ASYNC        5

/* ---- cc_graph_create flags ----------------------------------------------- */
#define CC_VALIDATE     1u   /* validate the CSR (always done; accepted for clarity) */
#define CC_DEVICE_PTRS  2u   /* row_offsets/col_idx are device pointers, adopted by
                                reference (caller keeps them alive until destroy) */
#define CC_OFFSETS_I32  4u   /* row_offsets is int32[n+1] instead of int64[n+1]  */
#define CC_VALIDATE_EXACT 8u /* check symmetry exactly: every entry (u, w) with u < w is
                                looked up in row w by binary search (slower: about 10
                                random reads per entry); without it symmetry is checked by
                                two order-independent 64-bit hash sums of the pairs seen
                                from either end, which a crafted graph could defeat */

/* Limits: 0 <= n <= 2^31 - 32 (a 32-bit state word per vertex), nnz < 2^33. */

typedef struct cc_graph cc_graph;

/* Per-round statistics of one clustering (Alg. 2 loop body). */
typedef struct cc_round_stats {
  int64_t n_alive;   /* n_i: unclustered vertices at round start              */
  int64_t delta;     /* Delta_i: maximum residual degree                      */
  int64_t k;         /* |A_i|                                                 */
  int64_t centers;   /* clusters opened this round                            */
  int64_t removed;   /* vertices clustered this round (A_i included)          */
  int64_t blocked;   /* C4: actives with an earlier-ranked active neighbour   */
  int64_t edges;     /* adjacency entries read by this round's passes         */
  int64_t ns;        /* device time of the round (from the previous round's end,
                        its Delta work included), nanoseconds                 */
} cc_round_stats;

/*
 * cc_graph_create -- upload (or adopt) the positive edges of a graph.
 *   n            number of vertices.
 *   row_offsets  int64[n+1] (int32[n+1] with CC_OFFSETS_I32), off[0] = 0,
 *                non-decreasing; row v is col_idx[off[v] .. off[v+1]).
 *   col_idx      int32[off[n]]: each row strictly increasing, no self loop,
 *                every entry in [0,n), and the graph symmetric (u in row v iff
 *                v in row u).  Isolated vertices are allowed.
 *   flags        CC_VALIDATE / CC_DEVICE_PTRS / CC_OFFSETS_I32 / CC_VALIDATE_EXACT
 *                (any other bit: CC_ERR_INVALID_ARG).
 *   cuda_stream  cudaStream_t for all work on this graph (NULL = legacy stream).
 *   out          receives the handle.
 * Host arrays are copied; the caller may free them on return.  The CSR is
 * validated on the device (range, order, self loops, symmetry):
 * CC_ERR_INVALID_GRAPH on failure.
 */
int cc_graph_create(int64_t n, const void* row_offsets, const int32_t* col_idx,
                    uint32_t flags, void* cuda_stream, cc_graph** out);

/* Release the graph and every device buffer it owns. NULL is accepted. */
int cc_graph_destroy(cc_graph* g);

/* n, nnz (= 2m) and the largest degree of a created graph. Any out may be NULL. */
int cc_graph_info(const cc_graph* g, int64_t* n, int64_t* nnz, int64_t* max_degree);

/*
 * cc_permutation -- pi of Alg. 1/2: order_out[r] = the vertex of rank r, the
 * vertices sorted by (splitmix64(seed ^ v), v).  order_out: int32[n], host or
 * device memory.  Uses the graph's stream; blocks until done.
 */
int cc_permutation(cc_graph* g, uint64_t seed, int32_t* order_out);

/*
 * cc_cluster -- one full clustering (Alg. 2) of graph g.
 *   algo               CC_ALGO_C4, CC_ALGO_CLUSTERWILD, CC_ALGO_C4_EST,
 *                      CC_ALGO_CLUSTERWILD_EST or CC_ALGO_C4_ASYNC.
 *   eps                0 < eps <= 1 (Sec. 3 assumes eps <= 1).
 *   seed               selects pi.
 *   labels_out         int32[n], host or device memory: the center vertex id
 *                      of each vertex's cluster.  May be NULL.
 *   rounds_out         number of rounds (NULL allowed).
 *   disagreements_out  the objective of the result, int64 (NULL allowed).
 * Blocks until the result is available.
 */
int cc_cluster(cc_graph* g, int algo, double eps, uint64_t seed, int32_t* labels_out,
               int32_t* rounds_out, int64_t* disagreements_out);

/* cc_cluster plus per-round statistics: the first min(rounds, stats_cap)
 * rounds are written to stats (host memory); *stats_len = rounds
 * (CC_ALGO_C4_ASYNC: one record for the whole run, *stats_len = 1). */
int cc_cluster_ex(cc_graph* g, int algo, double eps, uint64_t seed, int32_t* labels_out,
                  int32_t* rounds_out, int64_t* disagreements_out, cc_round_stats* stats,
                  int32_t stats_cap, int32_t* stats_len);

/*
 * cc_disagreements -- objective (Sec. 2) of an arbitrary labelling:
 * positive edges across clusters plus negative pairs inside clusters.
 * labels: int32[n], host or device, values in [0, n) (CC_ERR_INVALID_ARG
 * otherwise).  out: host int64.
 */
int cc_disagreements(cc_graph* g, const int32_t* labels, int64_t* out);

/*
 * cc_batch_run -- best-of-k over many graphs (the paper runs each graph
 * under 100 random orders; this keeps the best of k).  For graph i and
 * j = 0..k_perms-1 the job is cc_cluster(gs[i], algo, eps, seeds[i] + j).
 *   gs[count], seeds[count]  graphs and base seeds.
 *   labels_out[i]            int32[n_i] (host or device) or NULL: labels of the
 *                            best job of graph i.
 *   best_j[i], best_D[i], rounds[i]  host arrays (NULL allowed): index of the
 *                            best permutation (lowest D, ties to lowest j), its
 *                            disagreements and its round count.
 * Jobs run concurrently on the device; each result is the same as the
 * corresponding single cc_cluster call.  algo: CC_ALGO_C4 ..
 * CC_ALGO_CLUSTERWILD_EST (CC_ALGO_C4_ASYNC is CC_ERR_INVALID_ARG here).
 */
int cc_batch_run(cc_graph* const* gs, int32_t count, int algo, double eps,
                 const uint64_t* seeds, int32_t k_perms, int32_t* const* labels_out,
                 int32_t* best_j, int64_t* best_D, int32_t* rounds);

/*
 * cc_batch_jobs -- the jobs of cc_batch_run without the best-of-k reduction:
 * D_out[i * k_perms + j] and rounds_out[i * k_perms + j] (host arrays, either
 * may be NULL) for graph i under seed seeds[i] + j.  Small graphs run one per
 * thread block, medium graphs one per team of blocks, all in one launch per
 * size class; graphs above 2^21 vertices run on the whole GPU one at a time.
 * All graphs must live on the same device.
 */
int cc_batch_jobs(cc_graph* const* gs, int32_t count, int algo, double eps,
                  const uint64_t* seeds, int32_t k_perms, int64_t* D_out,
                  int32_t* rounds_out);

/*
 * Kernel timing hook.  cc_graph_set_timing(g, 1) makes later cc_cluster /
 * cc_cluster_ex calls on g record CUDA events on the graph's stream around
 * their three device stages; cc_last_timings then writes the durations in
 * milliseconds of the last call to ms_out[0..2] = {permutation, rounds
 * kernel, label output}.  cc_last_timings returns CC_ERR_INVALID_ARG when
 * timing is off or nothing has been timed yet.
 */
int cc_graph_set_timing(cc_graph* g, int enable);
int cc_last_timings(const cc_graph* g, float* ms_out);

/*
 * Device-side breakdown of the last clustering's round kernel (always
 * recorded; globaltimer at every grid barrier).  ms_out[0..min(cap,7)) =
 * milliseconds spent in: Delta from the heavy list (grid scans) and the
 * count pass of its rebuild, the rebuild's compaction and refill, the Sec. 5
 * batch draws, active-set selection, centers + attachment (C4: detection
 * and classification too), C4 fixpoint and blocked actives, removal and
 * degree updates.  (Zeros for CC_ALGO_C4_ASYNC.)
 */
int cc_last_phase_times(const cc_graph* g, double* ms_out, int32_t cap);

/*
 * Test hook for the bounded waits (failure detection without a fault): the
 * next cc_cluster / cc_cluster_ex call on g (CC_ALGO_C4 .. _EST) withholds the
 * round kernel's barrier release after round `round` (0-based).  Every other
 * block's wait on that release runs out after its 4 s bound, records
 * CC_ERR_TIMEOUT and returns, so the call returns CC_ERR_TIMEOUT after about
 * 4 s and the graph stays usable.  The hook applies to the next clustering
 * call on g only, whatever that call's outcome: a call that fails its
 * argument checks, runs on an empty graph, fails to allocate or uses
 * CC_ALGO_C4_ASYNC consumes it without effect; a clustering with fewer
 * rounds ends normally.  round < 0: CC_ERR_INVALID_ARG.
 */
int cc_debug_withhold_release(cc_graph* g, int32_t round);

/*
 * cc_disagreements_static -- the same objective as cc_disagreements, for
 * callers that cannot allocate memory when they need it: code running inside
 * a fixed memory pool or arena, or under a "no allocation after start-up"
 * rule.  Besides the caller's buffers it uses one scratch area compiled into
 * the library (about 4 MB per GPU, held until the process exits).  Under
 * CUDA's lazy module loading (the default) that area is mapped on a device
 * by the first call there, which may therefore make the driver allocate and
 * can return CC_ERR_OOM on a full GPU: make one call per device at start-up,
 * before any no-allocation phase or stream capture.  Later calls allocate
 * nothing.  The paper has no counterpart; this is a deployment variant.
 *   n            number of vertices, 0 <= n <= CC_STATIC_MAX_N (larger n:
 *                CC_ERR_INVALID_ARG).
 *   row_offsets  device int64[n+1], col_idx device int32[off[n]]: a CSR as
 *                cc_graph_create accepts it (not validated here).
 *   labels       device int32[n], values in [0, n).
 *   out          device int64: receives D, or -1 if a label is out of range.
 *   cuda_stream  stream for the work; the call returns without waiting.
 * Every call shares the one scratch area (cleared by each call): calls whose
 * work overlaps on the GPU race and must be ordered by the caller.  The
 * first call on a device looks up the scratch address (cudaGetSymbolAddress).
 */
#define CC_STATIC_MAX_N (1 << 20)
int cc_disagreements_static(int64_t n, const int64_t* row_offsets, const int32_t* col_idx,
                            const int32_t* labels, int64_t* out, void* cuda_stream);

/*
 * Serving loop with continuous batching.  cc_server_submit queues a request
 * (graph g, algo, eps, seed) and returns a ticket at once.  A dispatcher
 * thread starts the waiting requests of one size class as one launch on one
 * of sixteen streams as soon as a stream is free and the device-memory budget
 * covers the launch's scratch, so requests that arrive while others run are
 * admitted and their work overlaps on the device with the work in flight.
 * Size classes: up to 2^16 vertices one thread block per request; up to 2^21
 * one team of eight blocks per request (cooperative launches of up to
 * sixteen teams, two such launches in flight at a time, together at most two
 * thirds of the GPU); larger graphs the whole
 * GPU, one request at a time, on a worker thread of their own.  The
 * dispatcher never waits for the GPU (results come back by asynchronous
 * copies into pinned host memory).  A launch that fails fails its own
 * requests only.  Graphs stay resident (they are the caller's, must outlive
 * their requests, and must not be used by the caller while a request on them
 * is pending; submit does not wait for the graph's stream).  The result of a
 * request is exactly that of
 * cc_cluster with the same arguments.  algo: CC_ALGO_C4 ..
 * CC_ALGO_CLUSTERWILD_EST (CC_ALGO_C4_ASYNC is CC_ERR_INVALID_ARG here).
 *   mem_budget   bytes of device memory for batch scratch (a request whose
 *                scratch alone exceeds it fails with CC_ERR_OOM).
 *   max_batch    largest number of requests per launch.
 *   labels_out   device int32[n] or NULL.
 * cc_server_poll returns CC_ERR_BUSY while the request is pending;
 * cc_server_wait blocks (at most 10 minutes).  latency_ms = time from submit
 * to completion as seen by the dispatcher.  cc_server_device_times gives the
 * device clock (%globaltimer, ns) at which a finished request's job started
 * and ended on the GPU (-1 for requests that ran on the whole GPU), so that
 * callers can see which requests overlapped; CC_ERR_BUSY while pending.
 * cc_server_destroy finishes the queued work first.  A server is thread safe.
 */
typedef struct cc_server cc_server;
int cc_server_create(size_t mem_budget, int32_t max_batch, cc_server** out);
int cc_server_submit(cc_server* s, cc_graph* g, int algo, double eps, uint64_t seed,
                     int32_t* labels_out, int64_t* ticket);
int cc_server_poll(cc_server* s, int64_t ticket, int32_t* rounds, int64_t* disagreements,
                   double* latency_ms);
int cc_server_wait(cc_server* s, int64_t ticket, int32_t* rounds, int64_t* disagreements,
                   double* latency_ms);
int cc_server_device_times(cc_server* s, int64_t ticket, int64_t* start_ns, int64_t* end_ns);
int cc_server_destroy(cc_server* s);

/*
 * Schedule settings (the autotuner's knobs).  None of them changes any
 * result -- labels, rounds and disagreements are the same under every valid
 * setting -- only how the work is cut into pieces and where it runs.  The
 * paper has no counterpart (its implementation ran on CPU threads).
 *   walk_batches     edge walker: 128-entry batches per warp chunk, 1..8 (4)
 *   prefetch_ahead   edge walker: batches of a long row prefetched into L2,
 *                    0..8 (2)
 *   inline_heavy     exact Delta: heavy lists up to this long are scanned
 *                    inside the grid barrier by one block, 0..65536 (8192)
 *   inline_decide    C4: blocked lists up to this long are decided inside the
 *                    barrier, 0..65536 (4096)
 *   inline_rebuild   Delta rebuild: degree-order segments up to this long are
 *                    read inside the barrier, 0..65536 (8192)
 *   heavy_shift      heavy-list threshold tau = max(1, Delta >> heavy_shift),
 *                    1..4 (1)
 *   batch_small_n    batched jobs and served requests: one thread block per
 *                    job up to this many vertices, 1..2^20 (65536)
 *   batch_team_n     one team of blocks per job up to this many vertices,
 *                    >= batch_small_n, <= 2^24 (2^21)
 *   batch_team_blocks  blocks per team, 2..16 (8)
 *   warp_resolve_row C4: a round's blocked actives are decided one warp per
 *                    vertex in one grid phase when each has a warp and no
 *                    blocked row is longer than this (else by the fixpoint of
 *                    synchronous passes), 0..2^24 (1024; 0 = always the fixpoint)
 * cc_tuning_default fills the defaults (in brackets).  cc_graph_set_tuning
 * sets the round-kernel settings (all but the batch_* ones) for the clusterings of one
 * graph; cc_set_batch_tuning sets them, and the size classes, for every
 * later cc_batch_jobs / cc_batch_run call and every server created later
 * (process-wide).  Out-of-range values: CC_ERR_INVALID_ARG, nothing changed.
 */
typedef struct cc_tuning {
  int32_t walk_batches;
  int32_t prefetch_ahead;
  int32_t inline_heavy;
  int32_t inline_decide;
  int32_t inline_rebuild;
  int32_t heavy_shift;
  int64_t batch_small_n;
  int64_t batch_team_n;
  int32_t batch_team_blocks;
  int32_t warp_resolve_row;
} cc_tuning;
int cc_tuning_default(cc_tuning* out);
int cc_graph_set_tuning(cc_graph* g, const cc_tuning* t);
int cc_graph_get_tuning(const cc_graph* g, cc_tuning* out);
int cc_set_batch_tuning(const cc_tuning* t);
int cc_get_batch_tuning(cc_tuning* out);

/*
 * Device memory.  Every device allocation of the library (graphs, clustering
 * workspaces, batch and serving scratch) comes from one memory pool per GPU,
 * owned by the library, on the caller's stream (stream-ordered).  Memory a
 * destroyed graph or a finished batch gives back stays reserved in the pool,
 * so the next graph of a similar size maps no new memory.  cc_release_memory
 * returns the pools' unused reserved memory to the system (for example
 * before handing the GPU to another allocator); memory still in use is not
 * affected.  Returns CC_OK, or CC_ERR_CUDA.  The paper has no counterpart.
 */
int cc_release_memory(void);

/* Human-readable name of a status code (static storage). */
const char* cc_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* CC_H_ */
