/*
 * oracle.h -- plain CPU reference of the access-mode consistency calculus of
 * Henrio, Kessler and Li, "Leveraging Access Mode Declarations in a Model for
 * Memory Consistency in Heterogeneous Systems" (arXiv 1910.11110).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py load this library.  The product
 * path (the CUDA library under paper_1910_11110_gb300/) never links, loads or
 * calls it, and it shares no code, header or table with that path: the byte
 * encodings below are restated here on purpose.
 *
 * Encodings (inputs and outputs, identical to the product's C ABI):
 *   status code  = cpuValid | gpuValid << 1, plus 4 = F (stuck, absorbing).
 *                  The paper's pair is (local, remote) with local = CPU
 *                  (Section 3.1; data starts in CPU memory, Section 3.2).
 *   op byte      = kind | side << 4, side 0 = "E x", side 1 = "rem(E x)".
 *                  kinds: r=0 w=1 Push=2 Pull=3 Noop=4 pw=5 GT=6 EN=7;
 *                  structure tokens (relation mode): IF=8 ELSE=9 WHILE=10 END=11.
 *   status mask  = bit k set <=> status code k is possible (relation mode).
 *
 * Every function returns 0 on success and a negative code on malformed input
 * (-1 invalid, -2 id out of range, -3 out of host memory, -4 output capacity
 * exceeded); outputs are then unspecified.
 */
#ifndef AMC_ORACLE_H
#define AMC_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* Status code of applying one op (kind 0..5, side 0/1) to status code s.
 * Section 3.1 effect signatures + Fig. Opsem rules Effect / Remote Effect. */
int oracle_apply(int kind, int side, int status);

/* Straight-line trace mode (Fig. Opsem, initial store of Section 3.2). */
int oracle_check_trace(const uint8_t* kind_side, const int32_t* var, int64_t n_ops,
                       int32_t n_vars, const uint8_t* init_status,
                       uint8_t* step_status, uint8_t* final_status,
                       int32_t* var_first_fault, int64_t* first_fault);

/* oracle_check_trace restricted to the variables v % n_shards == shard (core
 * kinds only, initial statuses (V,I)); outputs written for those variables. */
int oracle_check_trace_shard(const uint8_t* kind_side, const int32_t* var, int64_t n_ops,
                             int32_t n_vars, int32_t n_shards, int32_t shard,
                             uint8_t* step_status, uint8_t* final_status,
                             int32_t* var_first_fault, int64_t* first_fault);

/* Relation mode for one structured program (If = union, While = closure). */
int oracle_check_program(const uint8_t* tok, const int32_t* payload, int64_t n_tok,
                         int32_t n_vars, const uint8_t* init_mask,
                         uint8_t* step_mask, uint8_t* final_mask, int64_t* first_fault);

/* Relation mode over a batch of independent programs (CSR layout). */
int oracle_check_batch(const uint8_t* tok, const int32_t* payload, const int64_t* prog_tok_off,
                       const int32_t* prog_nvars, const int64_t* prog_var_off, int64_t n_progs,
                       uint8_t* step_mask, uint8_t* final_mask, int64_t* prog_first_fault);

/* Path-sensitive relation mode: IF / WHILE token bits 4-5 = condition
 * (0 opaque x (+) y, 1 isValid g, 2 remIsValid g) on the program's guard
 * variable g (guard = -1: none, every condition opaque).  Pair sets (status
 * of g, status of x) per variable; a stuck g satisfies no condition rule (the
 * path ends).  Outputs as oracle_check_program (step_mask = statuses of the
 * op's variable after it, 0 when the op is unreachable). */
int oracle_check_program_guarded(const uint8_t* tok, const int32_t* payload, int64_t n_tok, int32_t n_vars,
                                 int32_t guard, const uint8_t* init_mask, uint8_t* step_mask,
                                 uint8_t* final_mask, int64_t* first_fault);
int oracle_check_batch_guarded(const uint8_t* tok, const int32_t* payload, const int64_t* prog_tok_off,
                               const int32_t* prog_nvars, const int64_t* prog_var_off, const int32_t* prog_guard,
                               int64_t n_progs, uint8_t* step_mask, uint8_t* final_mask, int64_t* prog_first_fault);

/* Overlap sets of half-open intervals [start, start+len): CSR, ascending ids. */
int oracle_overlaps(const int32_t* arr_start, const int32_t* arr_len, int32_t n_arrays,
                    int64_t* ov_off, int32_t* ov_idx, int64_t ov_cap);

/* VectorPU-annotated calls (Fig. sem-AM, Table Overlap-ext-tab, Section 4.3). */
int oracle_vectorpu(const int32_t* arr_start, const int32_t* arr_len, int32_t n_arrays,
                    const uint8_t* call_side, const int32_t* call_off, int64_t n_calls,
                    const int32_t* opnd_array, const uint8_t* opnd_mode, int infer_overlap,
                    uint8_t* out_kind_side, int32_t* out_var, int64_t out_cap, int64_t* out_n,
                    int64_t* call_first_op, uint8_t* step_status, uint8_t* final_status,
                    int32_t* var_first_fault, int64_t* first_fault);

/* oracle_vectorpu over pvectors with lifetimes (Section 4.3: r_v updated at
 * creations and deletions; a pvector inherits its mother vector's coherence
 * state when declared).  Array a is live at calls arr_born[a] <= c <
 * arr_died[a] (0 <= born < died <= n_calls); arr_parent[a] = -1 for a vector,
 * else the vector (parent -1) whose range and lifetime hold a's.  Before call
 * c each pvector born at c (ascending id) takes its vector's real and
 * abstract statuses, recorded as Noop v, Noop v# (CPU side) at the head of
 * call c's statements; arr_probe[a] = index of the first (-1 for vectors).
 * Operands must be live; O(M), shadows and write projections use the live
 * arrays only. */
int oracle_vectorpu_lifetimes(const int32_t* arr_start, const int32_t* arr_len, const int32_t* arr_parent,
                              const int32_t* arr_born, const int32_t* arr_died, int32_t n_arrays,
                              const uint8_t* call_side, const int32_t* call_off, int64_t n_calls,
                              const int32_t* opnd_array, const uint8_t* opnd_mode, int infer_overlap,
                              uint8_t* out_kind_side, int32_t* out_var, int64_t out_cap, int64_t* out_n,
                              int64_t* call_first_op, int64_t* arr_probe, uint8_t* step_status,
                              uint8_t* final_status, int32_t* var_first_fault, int64_t* first_fault);

/* Static well-declaredness of VectorPU-style calls AM{S} (Section 3.3,
 * Definitions "Occurs in all execution paths" and "Well-declared program";
 * Section 3.5, "Well-declared program with array access").  Locations of
 * array a are [arr_loc_off[a], arr_loc_off[a+1]) (loc_owner[l] = a; a scalar
 * is an array of one location).  Call c has body tokens [call_tok_off[c],
 * call_tok_off[c+1]) (ops r/w/Push/Pull/Noop on locations, IF/ELSE/WHILE/END
 * as in relation mode) and declarations [call_am_off[c], call_am_off[c+1])
 * (am_array, am_mode = mode (R 1, W 2, RW 3) | side << 4).  violations[c]:
 * bit 0 Push / Pull in the body, bit 1 a write not declared W / RW on its
 * side, bit 2 a read not declared R / RW on its side, bit 3 a W declaration
 * whose array has a location not written on that side in all execution
 * paths, bit 4 an array declared twice; first_bad[c] = call-relative token of
 * the first bit 0-2 violation (-1 none); first_unmet[c] = smallest array id
 * with a bit-3 violation (-1 none). */
int oracle_well_declared(const int64_t* arr_loc_off, int32_t n_arrays, const int32_t* loc_owner,
                         const int64_t* call_tok_off, int64_t n_calls, const uint8_t* tok,
                         const int32_t* payload, const int64_t* call_am_off, const int32_t* am_array,
                         const uint8_t* am_mode, uint32_t* violations, int64_t* first_bad,
                         int32_t* first_unmet);

/* Traces over k memory locations (k = 1..7): the Section 3.1 signatures on a
 * vector of k validity flags.  Op byte: bits 0-1 kind (r 0, w 1, copy 2,
 * Noop 3), bits 2-4 location a, bits 5-7 location b (copy a -> b only).
 * Status byte: bit i = location i valid, 0x80 = F.  init_status NULL: valid
 * in location 0 only.  Outputs as oracle_check_trace. */
int oracle_apply_k(int op, int status, int k);
int oracle_check_trace_k(const uint8_t* op, const int32_t* var, int64_t n_ops, int32_t n_vars, int32_t k,
                         const uint8_t* init_status, uint8_t* step_status, uint8_t* final_status,
                         int32_t* var_first_fault, int64_t* first_fault);

#ifdef __cplusplus
}
#endif
#endif
