// cc_async.h -- host-side declarations of the asynchronous C4 (Alg. 3).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "cc_internal.h"

namespace ccg {

// Largest co-resident grid of the asynchronous decision kernel on this device.
int async_grid_size(int device);

// C4 without rounds (Alg. 3 with attemptCluster), on the workspace of the
// round kernel: b.order holds pi; on return labels[v] (device int32[n]) is
// the center vertex id of v, and b.ctl holds the counters:
//   r_centers  centers,  r_noncenter  non-centers,
//   r_blocked  vertices that waited on an undecided earlier neighbour,
//   r_attached adjacency entries read by the decisions,
//   err        device status (kErrTimeout when a wait ran out).
// The arrays st, arank, blk_flag and the active list of b are overwritten.
cudaError_t launch_async_c4(const RoundBuffers& b, int grid, int32_t* labels, cudaStream_t stream);

}  // namespace ccg
