// batch_ps.cuh -- launch interface of the path-sensitive relation mode.
#pragma once

#include "amc_internal.cuh"

namespace amc {

struct PsParams {
    const uint8_t* tok;
    const int32_t* payload;
    const int64_t* prog_tok_off;
    const int32_t* prog_nvars;
    const int64_t* prog_var_off;
    const int32_t* prog_guard;     // guard variable per program, -1 none
    int64_t n_progs;
    int64_t n_tokens;
    int64_t total_vars;
    const uint8_t* init_mask;      // nullable: every variable starts as {(V,I)}
    uint8_t* step_mask;
    uint8_t* final_mask;
    int64_t* prog_first_fault;
    uint32_t* J;                   // [total_vars] pair sets of programs with many variables
    uint32_t* save;                // [AMC_MAX_DEPTH][2][total_vars] construct copies
    const int32_t* order;
    uint64_t* queue_head;
    int* err;
    SetTables tab;
};

struct PsLaunch {
    const uint8_t* tok = nullptr;
    const int32_t* payload = nullptr;
    const int64_t* prog_tok_off = nullptr;
    const int32_t* prog_nvars = nullptr;
    const int64_t* prog_var_off = nullptr;
    const int32_t* prog_guard = nullptr;
    int64_t n_progs = 0;
    int64_t n_tokens = 0;
    int64_t total_vars = 0;
    const uint8_t* init_mask = nullptr;
    uint8_t* step_mask = nullptr;
    uint8_t* final_mask = nullptr;
    int64_t* prog_first_fault = nullptr;
    int* err = nullptr;
    void* workspace = nullptr;
    int profile = 0;
};

size_t batch_ps_workspace_bytes(int64_t n_progs, int64_t total_vars);
int launch_batch_ps(const PsLaunch& B, cudaStream_t s);

}  // namespace amc
