// kloc.cuh -- launch interface of the trace check over k memory locations.
#pragma once

#include "amc_internal.cuh"

namespace amc {

struct KlocLaunch {
    const uint8_t* op = nullptr;
    const int32_t* var = nullptr;
    int64_t n_ops = 0;
    int32_t n_vars = 0;
    int k = 2;
    const uint8_t* init = nullptr;
    uint8_t* step = nullptr;
    uint8_t* final_status = nullptr;
    int32_t* vff = nullptr;
    int64_t* first_fault = nullptr;
    void* workspace = nullptr;
    int* err = nullptr;
    int profile = 0;
};

size_t kloc_workspace_bytes(int64_t n_ops);
int launch_kloc(const KlocLaunch& L, cudaStream_t s);

}  // namespace amc
