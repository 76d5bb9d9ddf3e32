// autotune.cuh -- launch-shape autotuner (see autotune.cu).
#pragma once

#include <functional>
#include <string>

#include "amc_internal.cuh"

namespace amc {

// Runs run(i) for the cached / tuned / default candidate i of key.
int autotune_run(const std::string& key, int n_cand, int default_idx, cudaStream_t s,
                 const std::function<int(int)>& run);
// Cached choice for key, or -1.
int autotune_lookup(const std::string& key);
// "kind:log2(a):log2(b):extra"
std::string shape_key(const char* kind, int64_t a, int64_t b, int64_t extra);

}  // namespace amc
