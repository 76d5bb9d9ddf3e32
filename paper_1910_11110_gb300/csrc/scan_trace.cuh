// scan_trace.cuh -- launch interface of the per-variable trace scan.
#pragma once

#include "amc_internal.cuh"

namespace amc {

struct ScanParams {
    const uint8_t* kind_side;
    const int32_t* var;
    int64_t n_ops;              // ops (with n_dev: the capacity of the arrays)
    const int64_t* n_dev;       // nullable: device word with the op count (clamped to n_ops)
    const int* gate;            // nullable: the launch works only while (*gate != 0) == gate_on
    int gate_on;
    int32_t n_vars;
    const uint8_t* init;        // nullable: all (V,I)
    uint8_t* step;              // [n_ops] post-statuses (pre-statuses in pre_mode)
    int32_t* vff;               // [n_vars] first fault per var (-1 none); also the stuck index
    int64_t* first_fault;       // [1]
    const uint8_t* guard;       // pre-statuses from the guard pass (GT resolution)
    int pre_mode;               // 1 = guard pass: GT is Noop, outputs are pre-statuses
    int* err;
    uint32_t* head;             // [n_vars] newest registered node of each var
    uint32_t* node_next;        // [n_tiles * T]
    uint8_t* node_status;       // [n_tiles * T]
    uint32_t* regbits;          // bit t set: tile t's nodes are in their lists
    uint32_t* fbits;            // bit v set: variable v is known to be stuck
    int fbw;                    // words of fbits copied to shared memory (multiple of 4)
    int fbits_words;            // words per copy of fbits (two copies)
    int fb_mode;                // 0 none, 1 shared copy, 2 L1-cached global copies, 3 both
    uint32_t* tile_counter;
    uint32_t* front;            // every tile < *front has registered
    int n_tiles;
    int passes;
    int digit_bits;
    int bulk_ok;
    int phase_on;               // accumulate per-phase cycle counters
    int group_max;              // most tiles per claim (1: tile path only)
    int group_force;            // 1: every claim takes group_max tiles
    Tables tab;
};

struct ScanLaunch {
    const uint8_t* kind_side = nullptr;
    const int32_t* var = nullptr;
    int64_t n_ops = 0;
    int32_t n_vars = 0;
    const uint8_t* init = nullptr;
    uint8_t* step = nullptr;
    uint8_t* final_status = nullptr;    // nullable: skip the final-status pass
    int32_t* vff = nullptr;
    int64_t* first_fault = nullptr;
    const uint8_t* guard = nullptr;
    int pre_mode = 0;
    int* err = nullptr;
    void* workspace = nullptr;
    int max_ctas = 0;                   // 0 = one wave of resident CTAs
    int profile = 0;                    // bit 0: record the start event, bit 1: the stop event
    int fb_max_bits = 0;                // shared stuck bitmap size in variables (0 = default,
                                        // -1 = no bitmap, -2 = bitmap read through L1)
    int group_max = 0;                  // most tiles per claim (0 = default, 1 = tile path only)
    int ctas_per_sm = 0;                // resident CTAs per SM (0 = as many as fit)
    int dense = -1;                     // reduce / carry / apply path: -1 when eligible, 0 never
    const int64_t* n_dev = nullptr;     // device op count, read by the kernel (n_ops = capacity);
                                        // single-pass kernel only, not with a guard
    int prefix_log2 = 0;                // > 0: a 2^k-op reduce / carry / apply prefix whatever the
                                        // size, initial statuses or device count (many variables)
    const int* gate = nullptr;          // device flag: the scan and its final-status pass do
    int gate_on = 0;                    // nothing unless (*gate != 0) == gate_on (single-pass only)
    int tail = -1;                      // epoch path: -1 by size (2^29 ops or more), 1 whenever
                                        // eligible (more than 2^22 ops), 0 never
};

int scan_tile_size();
size_t scan_workspace_bytes(int64_t n_ops, int32_t n_vars, bool with_dense = true);
int launch_scan_trace(const ScanLaunch& L, cudaStream_t s);
// Traces over at most 16,384 variables take the reduce / carry / apply path of
// scan_dense.cu by size (or whenever AMC_SCAN_DENSE=1 or the launch forces it;
// never when AMC_SCAN_DENSE=0); its scratch follows the single-pass workspace.
// By size: at least 1,024 ops and at least 2^(15 + 2 (12 - log2 n_vars)) ops (the crossover with the
// single-pass scan measured on random traces with the Zipf workload's kind
// mix: 2^11 ops at 2^14 variables, 2^15 at 2^12, 2^21 at 2^9).
bool scan_dense_eligible(int64_t n_ops, int32_t n_vars);
// Whether a launch may force the reduce / carry / apply path on these sizes
// (at most 16,384 variables; up to 2^20 with global rows from 2^20 ops on).
bool dense_forced_ok(int64_t n_ops, int32_t n_vars);
size_t scan_dense_workspace_bytes(int64_t n_ops, int32_t n_vars);
int launch_scan_dense(const ScanLaunch& L, uint8_t* ws, cudaStream_t s);
// Traces over more than 16,384 (at most 2^20) variables and of 2^24 ops or
// more, without initial statuses: the first 2^22 ops take that path with
// per-chunk rows in global memory and the rest the single-pass kernel, from the
// prefix's final statuses.
bool scan_prefix_eligible(int64_t n_ops, int32_t n_vars, bool has_init);
int launch_scan_prefix(const ScanLaunch& L, uint8_t* ws, cudaStream_t s);
// Scratch of a P-op prefix (after the single-pass workspace); and whether L
// asks for a forced prefix that applies.
size_t scan_prefix_workspace_bytes(int64_t P, int32_t n_vars);
bool scan_forced_prefix(const ScanLaunch& L);
// First faults of a check of ops [offset, ...) folded into those of the ops
// before it: vff[v] = vff_part[v] + offset where vff[v] is -1 and vff_part[v]
// is not; the same for *ff.  With only_if, nothing happens while *only_if == 0.
int launch_merge_faults(int32_t* vff, const int32_t* vff_part, int32_t n_vars, int64_t* ff,
                        const int64_t* ff_part, int64_t offset, cudaStream_t s, const int* only_if = nullptr);
// Traces over 16,385 to 2^20 variables and of 2^29 ops or more, without a
// guard: the first 2^22 ops checked by sorting them by variable, the rest in
// epochs that each end at four times their start (stream filter on the stuck
// bitmap, the compacted candidates checked by sorting them by variable from
// the epoch's start statuses); its scratch replaces the single-pass workspace
// (scan_workspace_bytes covers both).
bool scan_tail_eligible(const ScanLaunch& L);
// Traces of at most 2^16 ops over at most 2,048 variables, without a guard:
// one CTA does the whole check (small.cu), no workspace.
bool scan_small_eligible(const ScanLaunch& L);
int launch_scan_small(const ScanLaunch& L, cudaStream_t s);
size_t scan_tail_workspace_bytes(int64_t n_ops, int32_t n_vars);
int launch_scan_tail(const ScanLaunch& L, cudaStream_t s);
// Kernels one launch_scan_tail of L runs (0 when L does not take that path).
int scan_tail_launches(const ScanLaunch& L);
// Radix passes of a sort by variable id over n_vars variables.
int ss_radix_passes(int32_t n_vars);
// The path launch_scan_trace takes for L (AMC_PATH_*) and the kernels it runs.
int scan_trace_plan(const ScanLaunch& L, int* launches);
// A set of ops checked by sorting it by variable (scan_sorted.cu): the pairs
// (variable id, set index << 4 | 4-bit code of the op byte) sit in key[0] /
// val[0]; key[1] / val[1] are the sort's second buffers.  Writes the status of
// every op whose status is not F to step[pos] (the caller wrote F at every
// position), the first fault of each variable that faults in the set
// (vff[v] = offset + pos, only ever written for variables not F at entry),
// folds them into *ff, and writes final statuses to fin (the caller copies the
// entry statuses there first).  Nothing runs while *gate != 0.
struct SortedCheck {
    uint32_t* key[2] = {nullptr, nullptr};
    uint32_t* val[2] = {nullptr, nullptr};
    const uint32_t* pos = nullptr;      // nullable: set index j is at position j
    const int64_t* n_dev = nullptr;     // nullable: the set's size on the device (clamped to cap)
    int64_t cap = 0;                    // the set's size, or its capacity with n_dev
    const int* gate = nullptr;
    int32_t n_vars = 0;
    const uint8_t* init = nullptr;      // entry statuses; nullable: all (V,I)
    uint8_t* step = nullptr;
    uint8_t* fin = nullptr;
    int32_t* vff = nullptr;
    int64_t* ff = nullptr;
    int64_t offset = 0;
    void* scratch = nullptr;            // sorted_check_scratch_bytes(cap)
    int* err = nullptr;                 // device error word (an expired bounded wait)
    uint32_t* bm = nullptr;             // nullable: stuck bitmap; bits set for variables that end F
};
// 4-bit code of an op byte in a pair: kind (bits 0-2) and side (bit 3)
__host__ __device__ __forceinline__ uint32_t sorted_code_of(uint32_t ks) { return (ks & 7u) | ((ks >> 1) & 8u); }
size_t sorted_check_scratch_bytes(int64_t cap);
int launch_sorted_check(const SortedCheck& C, cudaStream_t s);
// The same outputs for a set whose ops spread over the variable ids (an
// epoch's candidates; C.pos required): one radix pass groups the pairs into
// 128 buckets by the low seven bits of the id, one CTA checks each bucket.
// Final statuses and stuck bits are written only where a status changes, so
// C.fin must hold the entry statuses.  At most 2^20 variables
// (bucket_check_ok).
bool bucket_check_ok(int32_t n_vars);
int launch_bucket_check(const SortedCheck& C, cudaStream_t s);
// The sort alone: stable LSD radix sort of the pairs key[0] / val[0] by key
// (keys < n_vars), 7-bit digits, key[1] / val[1] as the second buffers; the
// result is in buffer (*passes & 1).  scratch: sorted_check_scratch_bytes(cap).
int launch_ss_radix(uint32_t* const key[2], uint32_t* const val[2], const int64_t* n_dev, int64_t cap,
                    int32_t n_vars, void* scratch, const int* gate, cudaStream_t s, int* passes);
// Ops [0, n) of a trace as pairs for launch_sorted_check, checked for bad
// bytes, ids out of range and GT without its EN; F written to step[0, n).
int launch_ss_keys(const uint8_t* kind_side, const int32_t* var, int64_t n, int64_t n_after, int32_t n_vars,
                   uint32_t* key, uint32_t* val, uint8_t* step, int* err, cudaStream_t s);
// enable >= 0: switch phase counting on/off and zero the counters; host_out
// (nullable): copy the 8 counters (cycles summed over CTAs).
int scan_phase_profile(int enable, unsigned long long* host_out);

}  // namespace amc
