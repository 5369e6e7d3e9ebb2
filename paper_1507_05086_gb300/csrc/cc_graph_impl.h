// cc_graph_impl.h -- the layout of the opaque cc_graph handle, shared by the
// translation units of the C ABI (not part of the public interface).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "cc_internal.h"

struct cc_graph {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int64_t n = 0, nnz = 0;
  int32_t max_deg = 0;
  int64_t* off = nullptr;
  int32_t* col = nullptr;
  bool own_off = false, own_col = false;
  int32_t* nz_row = nullptr;
  int64_t* nz_pos = nullptr;
  int64_t nz_n = 0;
  // non-isolated vertices by degree, largest first, and counts of degree >= t
  int32_t* dsort = nullptr;
  int64_t* dge = nullptr;
  // cached workspaces (grown on demand)
  void* perm_ws = nullptr;
  size_t perm_ws_bytes = 0;
  int32_t* order = nullptr;
  void* round_ws = nullptr;
  size_t round_ws_bytes = 0;
  int grid = 0;
  ccg::Tuning tune = ccg::default_tuning();   // schedule settings of this graph's clusterings
  int async_grid = 0;            // co-resident grid of the asynchronous C4 decisions
  int32_t withhold = 0;          // test hook for the next clustering (cc_debug_withhold_release)
  int32_t* labels_tmp = nullptr;
  void* obj_ws = nullptr;
  unsigned long long* obj_out = nullptr;
  ccg::RoundStat* stats_dev = nullptr;
  int64_t stats_dev_cap = 0;
  int* perm_err = nullptr;
  // optional event timing of the last clustering
  bool timing = false;
  bool timed = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  float last_ms[3] = {0, 0, 0};
  unsigned long long last_phase_ns[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  bool phases_valid = false;
  // pinned host staging for the small results
  ccg::Ctl* ctl_host = nullptr;
  unsigned long long* obj_host = nullptr;
  // graph creation from host arrays: the column copy runs on its own stream
  // in kColChunks pieces (released once creation ends)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t col_ready[ccg::kColChunks] = {};
};
