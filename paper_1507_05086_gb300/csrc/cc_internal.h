// cc_internal.h -- host-side declarations shared by the library's translation
// units (not part of the public ABI; see include/cc.h for that).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace ccg {

inline size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// pieces of the column array copied (and validated) one after another when a
// graph is created from host memory
constexpr int kColChunks = 8;

// ---- device memory (cc_api.cu) -----------------------------------------------
// Stream-ordered allocation from the library's pool on the current device
// (freed blocks stay reserved for reuse); free with cudaFreeAsync.
cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t stream);

// ---- permutation (cc_perm.cu) ----------------------------------------------
int perm_bucket_bits(int64_t n);
size_t perm_workspace_bytes(int64_t n);
cudaError_t launch_permutation(int64_t n, uint64_t seed, int32_t* order, void* ws, int num_sms,
                               int* err, cudaStream_t stream);

// ---- rounds (cc_rounds.cu) ---------------------------------------------------
// Per-round statistics as written by the device (layout of cc_round_stats).
struct RoundStat {
  int64_t n_alive, delta, k, centers, removed, blocked, edges, ns;
};

// Plan of the next phase, published by the coordinator block at every grid
// barrier (128 bytes, copied by every block with one vector load).
struct Plan {
  int64_t k, need, win_lo, win_len;
  int64_t take, act_n, act_E, new_n;
  int64_t new_E, b_n, b_E, undecided;
  int32_t th, r0, pad3, pad4;
  int32_t state, pad0, tag, pad2;      // tag: removal tag of the current round
};
static_assert(sizeof(Plan) == 128, "plan layout");
static_assert(offsetof(Plan, state) == 112, "the state word opens the last 16 bytes of the plan");

// Device control block of one clustering job.  Zeroed by the host before
// each launch; written by the kernels only.
struct Ctl {
  unsigned arrive, gen;           // grid barrier (monotonic counters)
  int err;
  int algo;                       // 1 / 2: C4 / ClusterWild!; 3 / 4: the same with the Sec. 5 schedule
  int64_t eps_ppm;
  uint64_t seed;                  // seed of pi (the Sec. 5 batch draws derive from it)
  // test hook: 1 + the round after which the coordinator withholds its
  // release, so that every other block's bounded wait runs out (0: off)
  int32_t withhold;
  alignas(16) Plan plan;
  // per-round counters, written by every block (lists pack items << 33 | edges)
  unsigned long long act_pack, new_pack, blk_pack;
  long long r_centers, r_attached, r_noncenter, r_blocked;
  long long undecided;
  unsigned long long h_pack;      // heavy-list appends
  unsigned long long blk_maxlen;  // C4: longest row of a blocked active this round
  int32_t r0;
  int64_t cursor_next;
  // objective tallies: member-center edges, member-member edges (counted from
  // both ends), sum over clusters of C(size, 2)
  unsigned long long mc, mm, pairs;
  // results, written by the coordinator at the end
  int64_t round, n_alive;
  int done;
  // time per phase category (ns): Delta scan (heavy list, rebuild count),
  // Delta rebuild (compaction, heavy refill), Sec. 5 draws, selection,
  // centers+attach, C4 fixpoint and blocked actives, removal+decrement, setup
  unsigned long long ph_ns[8];
};

// Schedule settings of the round kernel (the device side of cc_tuning in
// include/cc.h).  None of them changes a result, only how the work is cut.
struct Tuning {
  int32_t walk_batches;      // edge walker: 128-entry batches per warp chunk
  int32_t prefetch_ahead;    // edge walker: batches of a long row prefetched into L2
  int32_t inline_heavy;      // heavy lists up to this long are scanned by the coordinator block
  int32_t inline_decide;     // C4 blocked lists up to this long are decided inside the barrier
  int32_t inline_rebuild;    // degree-order segments up to this long are read by the coordinator
  int32_t heavy_shift;       // heavy-list threshold tau = max(1, D >> heavy_shift)
  int32_t warp_resolve_row;  // C4: blocked sets with rows up to this long resolved one warp per vertex
};
Tuning default_tuning();
// Process-wide settings of batched jobs (cc_set_batch_tuning): the size
// classes and the round-kernel settings of their jobs.
Tuning batch_settings(int64_t* small_n, int64_t* team_n, int* team_blocks);

struct RoundBuffers {
  int64_t n, nnz;
  int32_t max_deg;
  const int64_t* off;
  const int32_t* col;
  const int32_t* order;
  uint32_t* st;                // per-vertex state word
  uint32_t* rtag;              // per-vertex removal tag, 4 bits (8 vertices per word)
  int32_t* arank;              // rank of a vertex while it is active
  // row lists (see RowList in cc_device.cuh): vertex, first virtual edge,
  // CSR delta; actives also keep their rank, the blocked list stores the
  // active-list index in place of a vertex
  int32_t* act_v;
  int32_t* act_r;
  int64_t* act_e;
  int64_t* act_d;
  int32_t* new_v;
  int64_t* new_e;
  int64_t* new_d;
  int32_t* size;
  int32_t* hv;                 // heavy list (Delta candidates)
  int32_t* nz0;                // alive non-isolated vertices (double buffer)
  int32_t* nz1;
  const int32_t* nz_static;    // the graph's non-isolated vertices
  int64_t nz_n;
  // the graph's non-isolated vertices by degree, largest first, and the
  // number of vertices of degree >= t for t = 0 .. max_deg + 1 (the Delta
  // rebuild reads the prefix that can still hold the maximum)
  const int32_t* dsort;
  const int64_t* dge;
  uint8_t* blk_flag;
  uint8_t* hit_c;
  uint8_t* hit_p;
  int32_t* pull;
  int32_t* b_j;
  int64_t* b_e;
  int64_t* b_d;
  int64_t* blk_a;              // per-block scratch
  int64_t* blk_b;
  unsigned long long* desc;    // per-block scan descriptors of the selection (decoupled look-back)
  RoundStat* stats;
  int64_t stats_cap;
  Ctl* ctl;
  Tuning tune;
  // batched jobs only: writable order, permutation scratch
  int32_t* order_w;
  int32_t* ptmp;
  int64_t* pcnt;
};

// One job of a batched launch: a graph and a permutation seed, plus results.
struct BatchJob {
  const int64_t* off;
  const int32_t* col;
  const int32_t* nz;
  int64_t nz_n;
  const int32_t* dsort;
  const int64_t* dge;
  int64_t n, nnz;
  int32_t max_deg;
  int32_t err;          // result: device status (0 = ok, 1 = not run)
  uint64_t seed;
  int32_t* labels;      // optional device int32[n]: center vertex id of each vertex
  int64_t rounds;       // result
  int64_t D;            // result: disagreements
  int64_t t0, t1;       // result: device clock (%globaltimer, ns) at the job's start and end
};

// Largest co-resident grid of the batched kernel on this device.
int batch_grid_size(int device);
// Per-team scratch of a batched launch, sized for the largest job of the launch.
size_t batch_slot_bytes(int64_t n_max, int team_size);
void batch_slot_carve(void* ws, int64_t n_max, int team_size, RoundBuffers* B);
cudaError_t launch_batch(const BatchJob* jobs_dev, int njobs, const RoundBuffers* slots_dev, int team_size,
                         int grid, int algo, int64_t eps_ppm, cudaStream_t stream);
// Team size 1 with an ordinary (not cooperative) launch of `blocks` blocks.
cudaError_t launch_batch_blocks(const BatchJob* jobs_dev, int njobs, const RoundBuffers* slots_dev, int blocks,
                                int algo, int64_t eps_ppm, cudaStream_t stream);

size_t rounds_workspace_bytes(int64_t n, int32_t max_deg, int grid);
// Carve a workspace of rounds_workspace_bytes() into RoundBuffers (pointers only).
void rounds_carve(void* ws, int64_t n, int32_t max_deg, int grid, RoundBuffers* b);
// Largest co-resident grid for the persistent round kernel on this device.
int rounds_grid_size(int device);
cudaError_t launch_rounds(const RoundBuffers& b, int algo, int64_t eps_ppm, uint64_t seed, int grid,
                          cudaStream_t stream, int32_t withhold = 0);
// labels_out[v] = center vertex id (order[center rank]) when labels_out is
// not null; always adds the pair term sum_c C(s_c, 2) to ctl->pairs.
cudaError_t launch_finalize_labels(const RoundBuffers& b, int32_t* labels_out, cudaStream_t stream);

// ---- objective and validation (cc_objective.cu) ------------------------------
size_t objective_workspace_bytes(int64_t n);
// out[0] = intra-cluster CSR entries, out[1] = sum_c C(s_c, 2), out[2] = 1 if a
// label was outside [0, n).  out: 3 device words.
cudaError_t launch_disagreements(int64_t n, int64_t nnz, const int64_t* off, const int32_t* col,
                                 const int32_t* nz_row, const int64_t* nz_pos, int64_t nz_n,
                                 const int32_t* labels, void* ws, unsigned long long* out, int num_sms,
                                 cudaStream_t stream);
size_t validate_workspace_bytes();
// Validation in two steps sharing ws (validate_workspace_bytes()): offsets
// first (zeroes ws), then the entries over the non-empty rows.  The int pair
// at ws + align_up(64) holds (first error code, max degree).
cudaError_t launch_validate_offsets(int64_t n, int64_t nnz, const int64_t* off, void* ws, int num_sms,
                                    cudaStream_t stream);
// Entries [e0, e1) of the CSR; `last` adds the symmetry verdict over every
// range validated since launch_validate_offsets cleared the workspace.
cudaError_t launch_validate_edges(int64_t n, int64_t e0, int64_t e1, bool last, const int32_t* nz_row,
                                  const int64_t* nz_pos, int64_t nz_n, const int32_t* col, void* ws, int num_sms,
                                  cudaStream_t stream);
// Exact symmetry check (CC_VALIDATE_EXACT): reverse-entry search for every
// lower entry; shares ws (and its error word) with the validation above.
cudaError_t launch_validate_reverse(int64_t nnz, const int64_t* off, const int32_t* nz_row, const int64_t* nz_pos,
                                    int64_t nz_n, const int32_t* col, void* ws, int num_sms, cudaStream_t stream);
cudaError_t launch_offsets_i32_to_i64(int64_t n, const int32_t* in, int64_t* out, cudaStream_t stream);
// dsort (int32[nz_n]): the non-isolated vertices, largest degree first;
// dge (int64[max_deg + 2]): dge[t] = number of vertices of degree >= t.
// ws: degree_order_workspace_bytes(max_deg), free once the work is done.
size_t degree_order_workspace_bytes(int32_t max_deg);
cudaError_t launch_degree_order(int64_t nz_n, const int32_t* nz_row, const int64_t* off, int32_t max_deg,
                                int32_t* dsort, int64_t* dge, void* ws, int num_sms, cudaStream_t stream);
size_t nonempty_workspace_bytes(int64_t n);
cudaError_t launch_nonempty_rows(int64_t n, const int64_t* off, int32_t* nz_row, int64_t* nz_pos, void* ws,
                                 int64_t* count_dev, int num_sms, cudaStream_t stream);

}  // namespace ccg
