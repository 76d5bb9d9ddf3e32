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
};

size_t translate_workspace_bytes(int32_t n_arrays, int64_t n_calls);
int launch_translate(const TranslateLaunch& T, cudaStream_t s);

}  // namespace amc
