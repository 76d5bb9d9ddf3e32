// overlap.cuh -- the overlap sets r_v (Section 4.3) as ascending lists.
#pragma once

#include "amc_internal.cuh"

namespace amc {

// time buckets of the lists with lifetimes (a call reads its bucket's list)
constexpr int32_t OV_MAX_BUCKETS = 256;

struct OverlapBuild {
    const int32_t* arr_start = nullptr;
    const int32_t* arr_len = nullptr;
    const int32_t* arr_born = nullptr;    // nullable: every array live throughout
    const int32_t* arr_died = nullptr;
    int32_t n_arrays = 0;
    int32_t n_buckets = 1;                // lists per array (with lifetimes)
    int64_t bucket_len = 1;               // calls per bucket
    int64_t cap = 0;                      // list entries the output holds; 0: count only
    int64_t* ov_off = nullptr;            // [n_arrays * n_buckets + 1] offsets of list (a, bucket)
    uint32_t* ov_idx = nullptr;           // [cap] list entries (with cap > 0)
    int64_t* n_pairs = nullptr;           // nullable, device: listed pairs (both directions)
    int* err = nullptr;
    void* workspace = nullptr;
};

size_t overlap_workspace_bytes(int32_t n_arrays, int32_t n_buckets, int64_t cap);
// buckets for a run of n_calls calls (1 without lifetimes), and their length
int32_t overlap_buckets(int64_t n_calls, bool lifetimes);
int64_t overlap_bucket_len(int64_t n_calls, int32_t n_buckets);
int launch_overlaps(const OverlapBuild& O, cudaStream_t s);

}  // namespace amc
