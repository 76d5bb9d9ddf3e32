// batch.cuh -- launch interface of the relation-mode batch checker.
#pragma once

#include "amc_internal.cuh"

namespace amc {

struct BatchParams {
    const uint8_t* tok;
    const int32_t* payload;
    const int64_t* prog_tok_off;
    const int32_t* prog_nvars;
    const int64_t* prog_var_off;
    int64_t n_progs;
    int64_t n_tokens;
    const uint8_t* init_mask;      // nullable: every variable starts as {(V,I)}
    uint8_t* step_mask;
    uint8_t* final_mask;
    int64_t* prog_first_fault;
    uint8_t* save;                 // [AMC_MAX_DEPTH][n_tokens]
    uint8_t* alt;                  // [AMC_MAX_DEPTH][n_tokens]
    const int32_t* order;          // nullable: program queue order
    uint64_t* queue_head;
    int* err;
    int64_t split;                 // segment length of split programs
    int save_rows;                 // construct levels the save / alt rows hold (deeper: AMC_E_INVALID)
    SetTables tab;
};

struct BatchLaunch {
    const uint8_t* tok = nullptr;
    const int32_t* payload = nullptr;
    const int64_t* prog_tok_off = nullptr;
    const int32_t* prog_nvars = nullptr;
    const int64_t* prog_var_off = nullptr;
    int64_t n_progs = 0;
    int64_t n_tokens = 0;
    const uint8_t* init_mask = nullptr;
    uint8_t* step_mask = nullptr;
    uint8_t* final_mask = nullptr;
    int64_t* prog_first_fault = nullptr;
    int* err = nullptr;
    void* workspace = nullptr;
    int longest_first = 1;
    int max_ctas = 0;
    int regs_capped = 1;           // registers fitted to 6 CTAs per SM (else to 4)
    int no_split = 0;              // never split a program (no reduce-pass scratch)
    int save_rows = AMC_MAX_DEPTH; // construct levels with save / alt rows (0: straight-line only)
    int profile = 0;
};

size_t batch_workspace_bytes(int64_t n_tokens, int64_t n_progs);
size_t batch_workspace_bytes(int64_t n_tokens, int64_t n_progs, bool no_split, int save_rows);
int launch_batch(const BatchLaunch& B, cudaStream_t s);

}  // namespace amc
