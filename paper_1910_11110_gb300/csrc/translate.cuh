// translate.cuh -- launch interface of the VectorPU translation.
#pragma once

#include "amc_internal.cuh"

namespace amc {

struct TranslateLaunch {
    const int32_t* arr_start = nullptr;
    const int32_t* arr_len = nullptr;
    int32_t n_arrays = 0;
    const uint8_t* call_side = nullptr;
    const int32_t* call_off = nullptr;
    int64_t n_calls = 0;
    const int32_t* opnd_array = nullptr;
    const uint8_t* opnd_mode = nullptr;
    int64_t n_operands = 0;
    int infer = 1;
    uint8_t* out_ks = nullptr;
    int32_t* out_var = nullptr;
    int64_t out_cap = 0;
    int64_t* out_n = nullptr;
    int64_t* call_first_op = nullptr;
    int* err = nullptr;
    void* workspace = nullptr;
    int profile = 0;
    // lifetimes (arr_born == nullptr: every array live throughout)
    const int32_t* arr_born = nullptr;
    const int32_t* arr_died = nullptr;
    const int32_t* arr_parent = nullptr;
    int64_t max_pairs = 0;                 // listed overlap pairs the workspace holds
    int64_t* arr_probe = nullptr;          // [n_arrays] creation records
};

size_t translate_workspace_bytes(int32_t n_arrays, int64_t n_calls);
size_t translate_lifetimes_workspace_bytes(int32_t n_arrays, int64_t n_calls, int64_t max_pairs);
int launch_translate(const TranslateLaunch& T, cudaStream_t s);
// Initial statuses (2 n_arrays) of the second pass of a check of a trace with
// creation records: (V,I) for vectors, for a pvector the statuses step gives
// the Noop v, Noop v# of its record (its vector's at its creation).
int launch_inherit(const int32_t* var, int64_t n_ops, int32_t n_arrays, const int32_t* arr_parent,
                   const int64_t* arr_probe, const uint8_t* step, uint8_t* init, int* err, cudaStream_t s);
// The overlap-list entries (both directions, one per time bucket two
// lifetimes share) into *n_pairs (device): the max_pairs a lifetimes
// translation of n_calls calls needs.
size_t overlap_count_workspace_bytes(int32_t n_arrays, int64_t n_calls, bool lifetimes);
int launch_overlap_count(const int32_t* arr_start, const int32_t* arr_len, const int32_t* arr_born,
                         const int32_t* arr_died, int32_t n_arrays, int64_t n_calls, int64_t* n_pairs, int* err,
                         void* workspace, cudaStream_t s);

}  // namespace amc
