// dscan.cuh -- device-wide exclusive scan of int32 counts into int64 offsets
// (three launches: per-block totals, one-block scan of the totals, apply).
#pragma once

#include "amc_internal.cuh"

namespace amc {

// Workspace bytes for scanning n counts.
size_t dscan_workspace_bytes(int64_t n);

// out[i] = sum(in[0..i)), out[n] = total.  `out` has n + 1 entries.
int dscan_exclusive(const int32_t* in, int64_t* out, int64_t n, void* workspace, cudaStream_t s);

}  // namespace amc
