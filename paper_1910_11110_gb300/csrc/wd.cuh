// wd.cuh -- launch interface of the static well-declaredness check.
#pragma once

#include "amc_internal.cuh"

namespace amc {

struct WdLaunch {
    const int64_t* arr_loc_off = nullptr;
    int32_t n_arrays = 0;
    const int32_t* loc_owner = nullptr;
    const int64_t* call_tok_off = nullptr;
    int64_t n_calls = 0;
    const uint8_t* tok = nullptr;
    const int32_t* payload = nullptr;
    int64_t n_tokens = 0;
    const int64_t* call_am_off = nullptr;
    const int32_t* am_array = nullptr;
    const uint8_t* am_mode = nullptr;
    int64_t n_decls = 0;
    uint32_t* violations = nullptr;
    int64_t* first_bad = nullptr;
    int32_t* first_unmet = nullptr;
    void* workspace = nullptr;
    int* err = nullptr;
    int profile = 0;
};

size_t wd_workspace_bytes();
int launch_well_declared(const WdLaunch& L, cudaStream_t s);

}  // namespace amc
