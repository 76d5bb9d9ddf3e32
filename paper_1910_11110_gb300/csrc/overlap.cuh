// overlap.cuh -- the overlap sets r_v (Section 4.3) as ascending lists.
#pragma once

#include "amc_internal.cuh"

namespace amc {

struct OverlapBuild {
    const int32_t* arr_start = nullptr;
    const int32_t* arr_len = nullptr;
    const int32_t* arr_born = nullptr;    // nullable: every array live throughout
    const int32_t* arr_died = nullptr;
    int32_t n_arrays = 0;
    int64_t cap = 0;                      // listed pairs the output holds; 0: count only
    int64_t* ov_off = nullptr;            // [n_arrays + 1] list offsets (always written)
    uint32_t* ov_idx = nullptr;           // [cap] list entries (with cap > 0)
    int64_t* n_pairs = nullptr;           // nullable, device: listed pairs (both directions)
    int* err = nullptr;
    void* workspace = nullptr;
};

size_t overlap_workspace_bytes(int32_t n_arrays, int64_t cap);
int launch_overlaps(const OverlapBuild& O, cudaStream_t s);

}  // namespace amc
