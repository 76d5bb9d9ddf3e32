/*
 * amc.h -- C ABI of the GB300 access-mode consistency checker.
 *
 * The checker runs the calculus of Henrio, Kessler and Li, "Leveraging Access
 * Mode Declarations in a Model for Memory Consistency in Heterogeneous Systems"
 * (arXiv 1910.11110) over large inputs on one GPU (sm_103a):
 *   - straight-line op traces (Section 3.2, rules Effect / Remote Effect of
 *     Fig. Opsem over the effect signatures of Section 3.1);
 *   - VectorPU component calls with R / W / RW access modes over possibly
 *     overlapping arrays (translation of Fig. sem-AM, arrays of Section 3.5,
 *     overlap inference of Table Overlap-ext-tab and Section 4.3);
 *   - batches of structured If / While programs, with If read as the union of
 *     its branches and While as the closure of its body (Fig. Opsem rules
 *     IF-True/IF-False and While-True/While-False with opaque conditions);
 *   - a serving loop over such requests with device-resident session state.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Status code (uint8):  cpuValid | gpuValid << 1, i.e. 0 = (I,I), 1 = (V,I),
 *   2 = (I,V), 3 = (V,V), and 4 = F, the stuck state of Property Progress.
 *   F absorbs: once a variable is stuck every later op on it reports F, while
 *   other variables keep being checked.  The paper's pair is (local, remote)
 *   with local = CPU memory (Section 3.1); every variable starts at (V,I)
 *   (initial store of Section 3.2) unless an initial status is passed.
 * Status mask (uint8): bit k set <=> status code k is possible (relation mode).
 * Op byte (uint8):  kind | side << 4, bits 5-7 zero.  side 0 = "E x" (local,
 *   CPU), side 1 = "rem(E x)" (remote, GPU).  Kinds:
 *     0 r, 1 w, 2 Push, 3 Pull, 4 Noop           (Section 3.1 effects)
 *     5 pw   partial write of an overlapping array: own side keeps its
 *            validity, the other side becomes invalid (per-array summary)
 *     6 GT   guarded transfer on a real array: acts as the Fig. sem-AM
 *            transfer (CPU side: Pull, GPU side: Push, both local statements)
 *            exactly when the side is invalid in the status, before the next
 *            op, of the next op's variable; must be followed by an EN of the
 *            same side on another variable (amc_check_guarded_trace only)
 *     7 EN   the same test and transfer on an abstract variable itself
 *     8 IF, 9 ELSE, 10 WHILE, 11 END   structure tokens (programs only)
 * Pointers are DEVICE pointers unless marked "host".  Buffers are owned by
 *   the caller; the library never frees them.  Every call is asynchronous on
 *   the given stream (a cudaStream_t passed as void*, NULL = legacy default
 *   stream) and allocates no device memory: callers size `workspace` with the
 *   matching *_workspace() query (256-byte aligned).
 * Return value: argument / launch errors only (AMC_E_*).  A semantic fault is
 *   a result, never an error.  Data-dependent errors found on the device
 *   (a var id out of range, a malformed op byte, an expired bounded wait) are
 *   reported by amc_sync_status(); when it reports one, the outputs of the
 *   calls since the previous amc_sync_status() are unspecified.
 */
#ifndef AMC_H
#define AMC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define AMC_API __attribute__((visibility("default")))
#else
#define AMC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

enum {
    AMC_OK = 0,
    AMC_E_INVALID = -1,   /* malformed input (bad op byte, unbalanced tokens, duplicate operand ...) */
    AMC_E_RANGE = -2,     /* variable / array id out of range, capacity exceeded */
    AMC_E_NOMEM = -3,     /* workspace too small, or memory budget exceeded */
    AMC_E_TIMEOUT = -4,   /* a bounded device-side wait expired */
    AMC_E_CUDA = -5,      /* a CUDA runtime call failed */
    AMC_E_AGAIN = -6      /* serving: no slot free yet (back-pressure) */
};

enum { AMC_ST_II = 0, AMC_ST_VI = 1, AMC_ST_IV = 2, AMC_ST_VV = 3, AMC_ST_F = 4 };
enum { AMC_K_R = 0, AMC_K_W = 1, AMC_K_PUSH = 2, AMC_K_PULL = 3, AMC_K_NOOP = 4,
       AMC_K_PW = 5, AMC_K_GT = 6, AMC_K_EN = 7,
       AMC_T_IF = 8, AMC_T_ELSE = 9, AMC_T_WHILE = 10, AMC_T_END = 11 };
enum { AMC_MODE_R = 1, AMC_MODE_W = 2, AMC_MODE_RW = 3, AMC_MODE_DROPPED = 0x80 };

/* Library version (major * 10000 + minor * 100 + patch). */
AMC_API int amc_version(void);

/* Static message for an AMC_* code. */
AMC_API const char* amc_error_string(int code);

/* Synchronises `stream` and returns the first device-side error raised on
 * the current device since the previous call (AMC_OK if none), clearing it.
 * A CUDA error while synchronising is returned as AMC_E_CUDA. */
AMC_API int amc_sync_status(void* stream);

/* Profiling aid (no counterpart in the paper): while set, every call made by
 * this host thread records `start_event` on its stream just before its
 * dominant kernel and `stop_event` just after it (cudaEvent_t handles passed
 * as void*; NULL, NULL turns it off).  Returns AMC_OK. */
AMC_API int amc_set_profile_events(void* start_event, void* stop_event);

/* Profiling aid (no counterpart in the paper): counters of the trace scan
 * kernel, summed over CTAs: cycles per phase (0 tile staging, 1 decode and
 * compaction, 2 sort, 3 segmented scan, 4 run entry and list insertion,
 * 5 registration frontier, 6 look-back, 7 outputs), then 8 tiles, 9 tiles
 * with live ops, 10 live ops, 11 tiles with runs that look back.  enable >= 0
 * switches counting on (1) or off (0) for later launches and zeroes the
 * counters; host_out (12 host uint64, nullable) receives the counters. */
AMC_API int amc_debug_scan_phases(int enable, uint64_t* host_out);

/* ------------------------------------------------------------------------ */
/* (1) Straight-line traces -- Section 3.2 (Fig. Opsem, Effect and Remote    */
/*     Effect rules; signatures of Section 3.1; initial store sigma_0).      */
/* ------------------------------------------------------------------------ */

/* Workspace bytes amc_check_trace needs for these sizes. */
AMC_API size_t amc_check_trace_workspace(int64_t n_ops, int32_t n_vars);

/* Checks one trace of kinds 0..5 and 7: for every op i (0 <= i < n_ops,
 * n_ops <= 2^31 - 1) on
 * variable var[i] (0 <= var[i] < n_vars) writes the variable's status after
 * the op to step_status[i]; writes every variable's status after the trace to
 * final_status[v], the index of the op at which v first became F to
 * var_first_fault[v] (-1 if never) and the minimum of those to *first_fault
 * (-1 if none; a real execution stops there, Property Progress).
 *   kind_side   [n_ops]  op bytes (a GT is reported as AMC_E_INVALID)
 *   var         [n_ops]  int32 variable ids
 *   init_status [n_vars] initial status codes, or NULL for all (V,I); must
 *                        not overlap final_status (the first call of a size
 *                        class may run the check once per launch shape to
 *                        time them, each run reading init_status)
 *   step_status [n_ops], final_status [n_vars], var_first_fault [n_vars],
 *   first_fault [1]      outputs (int64)
 * Once the size class is tuned, a call on a stream other than the legacy
 * default stream (and not being captured by the caller) captures its launch
 * sequence into a CUDA graph, kept until exit and keyed by every argument and
 * the AMC_SCAN_* tuning knobs, and later calls with the same key replay it
 * (AMC_TRACE_GRAPH=0 turns this off; past 256 captured argument sets, new ones
 * run without a graph); the results are the same either way.
 * Errors: AMC_E_INVALID for negative sizes, NULL or overlapping buffers,
 * AMC_E_NOMEM when ws_bytes is too small.  Ids out of range or malformed op
 * bytes are reported through amc_sync_status (AMC_E_RANGE / AMC_E_INVALID). */
AMC_API int amc_check_trace(const uint8_t* kind_side, const int32_t* var, int64_t n_ops, int32_t n_vars,
                    const uint8_t* init_status, uint8_t* step_status, uint8_t* final_status,
                    int32_t* var_first_fault, int64_t* first_fault,
                    void* workspace, size_t ws_bytes, void* stream);

/* Which path the next amc_check_trace of these sizes takes and how many
 * kernels it launches (profiling aid, no counterpart in the paper): the
 * choice timed on the first call of the size class when one was made in this
 * process, else the size rule.  Writes one of AMC_PATH_* to *path (nullable)
 * and the kernel count to *launches (nullable).  Host only, no device work.
 * Returns AMC_E_INVALID for negative sizes. */
enum { AMC_PATH_SCAN = 0,        /* single-pass scan over linked runs */
       AMC_PATH_SMALL = 1,       /* one CTA: at most 2^16 ops over at most 2,048 variables */
       AMC_PATH_WARP_DENSE = 2,  /* reduce / carry / apply, warp-sequential chunks */
       AMC_PATH_DENSE = 3,       /* reduce / carry / apply, sorted tiles */
       AMC_PATH_PREFIX = 4,      /* a reduce / carry / apply prefix, then the scan */
       AMC_PATH_EPOCHS = 5 };    /* first part sorted by variable, then filtered epochs */
AMC_API int amc_check_trace_plan(int64_t n_ops, int32_t n_vars, int has_init, int32_t* path, int32_t* launches);

/* Workspace bytes amc_check_guarded_trace needs. */
AMC_API size_t amc_check_guarded_trace_workspace(int64_t n_ops, int32_t n_vars);

/* amc_check_trace for traces that also contain GT (kind 6), as produced by
 * amc_translate_vectorpu.  Runs two scans: the first yields the status of
 * every EN's variable before the EN with GT read as Noop (guards only read
 * abstract variables, which GT never touches); the second resolves each GT
 * from that status (the condition of Fig. sem-AM is checked on the abstract
 * value, Section 3.3) and checks the trace.  Same outputs and errors as
 * amc_check_trace; a GT not followed by an EN of the same side on another
 * variable is reported as AMC_E_INVALID. */
AMC_API int amc_check_guarded_trace(const uint8_t* kind_side, const int32_t* var, int64_t n_ops, int32_t n_vars,
                            const uint8_t* init_status, uint8_t* step_status, uint8_t* final_status,
                            int32_t* var_first_fault, int64_t* first_fault,
                            void* workspace, size_t ws_bytes, void* stream);

/* Allocation-free variant of amc_check_trace (the paper has no counterpart).
 * For callers that cannot allocate device memory themselves: code that runs
 * inside a host application whose allocator owns all device memory, plug-ins
 * that are handed only their inputs and outputs, and latency-critical loops
 * where an allocation call would synchronise the device.  The caller still
 * passes inputs and outputs exactly as for amc_check_trace; the scratch comes
 * from one fixed device array inside this library instead of a workspace.
 *   - Limits: n_ops <= AMC_NOALLOC_MAX_OPS and n_vars <= AMC_NOALLOC_MAX_VARS;
 *     larger sizes are rejected with AMC_E_RANGE before any GPU work.
 *   - The array (AMC_NOALLOC_SCRATCH_BYTES) is held by every GPU that loads
 *     the library until the process exits.
 *   - The first call on a device looks up the array's device address with
 *     that device current; make that first call before any stream capture.
 *   - All calls share the array: calls whose GPU work overlaps (other streams,
 *     other host threads) race on it and give unspecified results.  Each call
 *     re-initialises what must start at zero, so sequential calls are safe.
 *   - It calls no cudaMalloc / cudaFree and no allocating library routine.
 * Same outputs and device-side error reporting as amc_check_trace. */
#define AMC_NOALLOC_MAX_OPS (1 << 22)
#define AMC_NOALLOC_MAX_VARS (1 << 20)
#define AMC_NOALLOC_SCRATCH_BYTES (25u << 20)
AMC_API int amc_check_trace_noalloc(const uint8_t* kind_side, const int32_t* var, int64_t n_ops, int32_t n_vars,
                                    const uint8_t* init_status, uint8_t* step_status, uint8_t* final_status,
                                    int32_t* var_first_fault, int64_t* first_fault, void* stream);

/* amc_check_trace over HOST buffers: Section 3.2's check of one straight-line
 * trace (same op kinds, statuses and first-fault rules), with the inputs read
 * from and the outputs written to host memory.  The trace is cut into chunks
 * of chunk_ops ops (<= 0: 2^25; rounded up to a multiple of 4,096).  Chunk c
 * is checked from the final statuses of chunk c - 1 (Section 3.2: a trace's
 * statuses depend only on the statuses before it), and its first faults are
 * offset and folded into those of the earlier chunks.  Three chunks are in
 * flight: while chunk c is checked on `stream`, chunk c + 1 is copied in and
 * the step statuses of chunk c - 1 are copied out on two copy streams of this
 * library.
 *   kind_side, var [n_ops]        host inputs, as for amc_check_trace
 *   init_status [n_vars]          host, or NULL for all (V,I)
 *   step_status [n_ops], final_status, var_first_fault [n_vars],
 *   first_fault [1]               host outputs, as for amc_check_trace
 *   workspace, ws_bytes           DEVICE workspace, 256-byte aligned, at
 *                                 least amc_check_trace_host_workspace(...)
 *   stream                        the check's stream; the call waits for the
 *                                 work already on it and returns at once.
 * The outputs are complete once `stream` has synchronised (amc_sync_status).
 * Host buffers should be page-locked (cudaHostAlloc / cudaHostRegister): the
 * copies then overlap the checks; pageable buffers give the same results with
 * the copies serialised.  The caller keeps every buffer alive and untouched
 * until the stream has synchronised.  Concurrent calls from several host
 * threads are serialised while they enqueue.
 * Errors: as amc_check_trace; AMC_E_NOMEM when ws_bytes is too small. */
AMC_API size_t amc_check_trace_host_workspace(int64_t n_ops, int32_t n_vars, int64_t chunk_ops);
AMC_API int amc_check_trace_host(const uint8_t* kind_side, const int32_t* var, int64_t n_ops, int32_t n_vars,
                                 const uint8_t* init_status, uint8_t* step_status, uint8_t* final_status,
                                 int32_t* var_first_fault, int64_t* first_fault, int64_t chunk_ops,
                                 void* workspace, size_t ws_bytes, void* stream);

/* Traces over K memory locations (K = 1..AMC_K_MAX): the effects of Section
 * 3.1 on a vector of K validity flags instead of a pair (Section 3 states that
 * the results extend to multiple memory locations).  Location 0 is main
 * memory, where every variable starts valid (Section 3.2).  An op runs at a
 * location a:  r at a needs flag a valid and changes nothing; w at a makes a
 * the only valid flag; copy a -> b (a Push at a towards b, or a Pull at b
 * from a) needs flag a valid and makes flag b valid; Noop.  A failed need is
 * the stuck status.  With K = 2, local = 0 and remote = 1, Push = copy 0->1,
 * Pull = copy 1->0, rem Push = copy 1->0, rem Pull = copy 0->1.
 *   op [n_ops]           bits 0-1 kind (0 r, 1 w, 2 copy, 3 Noop), bits 2-4
 *                        location a, bits 5-7 location b (copy only, b != a;
 *                        0 for r / w; a = b = 0 for Noop)
 *   var [n_ops]          variable ids, 0 <= var < n_vars
 *   init_status [n_vars] status bytes (bit i = location i valid, AMC_KL_F =
 *                        stuck), or NULL for "valid in location 0 only"; must
 *                        not be the final_status buffer
 *   step_status, final_status, var_first_fault, first_fault: as for
 *                        amc_check_trace, with status bytes of this encoding
 * n_ops < 2^31.  Errors: host: AMC_E_INVALID for bad sizes, K out of range or
 * aliased buffers, AMC_E_NOMEM for a small workspace; device (amc_sync_status):
 * AMC_E_INVALID for a malformed op or initial status, AMC_E_RANGE for an id
 * out of range. */
#define AMC_K_MAX 7
#define AMC_KL_F 0x80
AMC_API size_t amc_check_trace_k_workspace(int64_t n_ops, int32_t n_vars);
AMC_API int amc_check_trace_k(const uint8_t* op, const int32_t* var, int64_t n_ops, int32_t n_vars, int32_t k,
                              const uint8_t* init_status, uint8_t* step_status, uint8_t* final_status,
                              int32_t* var_first_fault, int64_t* first_fault, void* workspace, size_t ws_bytes,
                              void* stream);

/* ------------------------------------------------------------------------ */
/* (2) VectorPU calls -> core trace -- Fig. sem-AM (translation of access    */
/*     modes), Section 3.5 (one abstract status per array), Table            */
/*     Overlap-ext-tab (inference O(M)) and Section 4.3 (overlap sets r_v,   */
/*     shadow arguments, no recursive application).                          */
/* ------------------------------------------------------------------------ */

/* Most operands one call may have. */
#define AMC_MAX_OPERANDS 32

/* Workspace bytes amc_translate_vectorpu needs (grows as n_arrays^2: the
 * overlap lists are sized for every array overlapping every other; they are
 * built by sorting the ranges by start and sweeping, in O(A log A + pairs)). */
AMC_API size_t amc_translate_vectorpu_workspace(int32_t n_arrays, int64_t n_calls, int64_t n_operands);

/* Translates n_calls component calls into a core trace over 2 * n_arrays
 * variables: real arrays 0..A-1 and their abstract variables A..2A-1.
 *   arr_start, arr_len [n_arrays]  half-open intervals [start, start + len)
 *                                  of one shared index space (len >= 1)
 *   call_side [n_calls]            0 = CPU component, 1 = GPU component
 *   call_off  [n_calls + 1]        CSR offsets into the operand arrays
 *   opnd_array, opnd_mode          operand array id and mode (1 R, 2 W, 3 RW;
 *                                  bit 7 = annotation dropped: the body still
 *                                  accesses the operand but it is not declared)
 *   infer_overlap                  1 = extend each call's declarations to O(M)
 * Per call, in this order (each statement touches one variable, so per
 * variable this is the paper's order [[M]]; S):
 *   for each operand in argument order: if declared with effective mode R or
 *   RW: GT x, EN x#; if W or RW: w x#; then the body accesses of its own mode
 *   (R: r x; W: w x; RW: r x, w x);
 *   for each shadow RW(y), ascending y: GT y, EN y#, w y#;
 *   for each operand x that the body writes and each y != x overlapping x,
 *   ascending y: w y if y lies inside x, else pw y.
 * All statements carry the call's side.  Outputs: out_kind_side / out_var
 * [out_cap] and *out_n (device int64) = statements written; call_first_op
 * [n_calls + 1] = index of each call's first statement.  When the
 * translation needs more than out_cap statements nothing but *out_n (the
 * needed count) is written and amc_sync_status reports AMC_E_RANGE.
 * Feed the result to amc_check_guarded_trace with n_vars = 2 * n_arrays.
 * Errors (host): AMC_E_INVALID for bad sizes; (device, via amc_sync_status)
 * AMC_E_INVALID for a bad mode / side / interval, a duplicate operand or more
 * than AMC_MAX_OPERANDS operands in a call,
 * AMC_E_RANGE for an array id out of range or an overflowing output. */
AMC_API int amc_translate_vectorpu(const int32_t* arr_start, const int32_t* arr_len, int32_t n_arrays,
                           const uint8_t* call_side, const int32_t* call_off, int64_t n_calls,
                           const int32_t* opnd_array, const uint8_t* opnd_mode, int64_t n_operands,
                           int infer_overlap,
                           uint8_t* out_kind_side, int32_t* out_var, int64_t out_cap, int64_t* out_n,
                           int64_t* call_first_op, void* workspace, size_t ws_bytes, void* stream);

/* pvectors created and deleted during the run -- Section 4.3 (r_v is
 * initialised when a vector is declared, updated at pvector creations and
 * deletions, queried at calls) and Section 5's account of VectorPU's partial
 * vectors (a new pvector inherits the coherence state of its mother vector).
 *   arr_parent [n_arrays]  -1 for a vector (its elements are a fresh
 *                          allocation), else the id of the vector the pvector
 *                          is a window of: a vector (parent -1), not the
 *                          pvector itself, whose range holds its range
 *   arr_born, arr_died     the array is live at calls born <= c < died
 *                          (0 <= born < died <= n_calls); a pvector's lifetime
 *                          lies within its vector's
 * Overlap lists keep only the pairs whose lifetimes meet; at call c, O(M),
 * the shadows and the projections of body writes take only the arrays live
 * at c, and every operand must be live at c.  Before call c, each pvector
 * created there (ascending id) takes its vector's real and abstract
 * statuses; the translated trace records this at the head of call c's
 * statements as Noop v, Noop v# (CPU side, no effect), and arr_probe[a]
 * (device int64 [n_arrays]) = index of the first of the two (-1 for vectors).
 *
 * The overlap lists are kept per time bucket (up to 256 stretches of equal
 * length of the n_calls calls): a pair of overlapping arrays is listed, for
 * each of the two, in every bucket their lifetimes share.
 * amc_vectorpu_overlap_pairs writes to *n_pairs (device int64) the number of
 * list entries for a run of n_calls calls (with arr_born = arr_died = NULL:
 * every overlapping pair, both directions, one bucket): the max_pairs the
 * translation needs.  amc_translate_vectorpu_lifetimes is then
 * amc_translate_vectorpu with those rules; more than max_pairs list entries
 * give AMC_E_RANGE (device).  Feed its trace to amc_check_inherited_trace.
 * Errors (device): AMC_E_INVALID for a malformed lifetime or vector link or an
 * operand that is not live at its call, AMC_E_RANGE for a vector id out of
 * range; the rest as amc_translate_vectorpu. */
AMC_API size_t amc_vectorpu_overlap_pairs_workspace(int32_t n_arrays, int64_t n_calls);
AMC_API int amc_vectorpu_overlap_pairs(const int32_t* arr_start, const int32_t* arr_len, const int32_t* arr_born,
                                       const int32_t* arr_died, int32_t n_arrays, int64_t n_calls, int64_t* n_pairs,
                                       void* workspace, size_t ws_bytes, void* stream);
AMC_API size_t amc_translate_vectorpu_lifetimes_workspace(int32_t n_arrays, int64_t n_calls, int64_t n_operands,
                                                          int64_t max_pairs);
AMC_API int amc_translate_vectorpu_lifetimes(const int32_t* arr_start, const int32_t* arr_len,
                                             const int32_t* arr_parent, const int32_t* arr_born,
                                             const int32_t* arr_died, int32_t n_arrays, const uint8_t* call_side,
                                             const int32_t* call_off, int64_t n_calls, const int32_t* opnd_array,
                                             const uint8_t* opnd_mode, int64_t n_operands, int infer_overlap,
                                             int64_t max_pairs, uint8_t* out_kind_side, int32_t* out_var,
                                             int64_t out_cap, int64_t* out_n, int64_t* call_first_op,
                                             int64_t* arr_probe, void* workspace, size_t ws_bytes, void* stream);

/* amc_check_guarded_trace of a trace with creation records (from
 * amc_translate_vectorpu_lifetimes) over 2 * n_arrays variables: every
 * variable starts from the initial store, except that each pvector starts
 * from the statuses its vector has at its creation record.  Two passes: the
 * first from the initial store gives every vector's statuses at the records
 * (a vector's statuses never depend on a pvector's), the second runs from the
 * inherited statuses and writes the outputs.  arr_parent and arr_probe as
 * given to / written by the translation.  Errors: as amc_check_guarded_trace;
 * AMC_E_INVALID (device) for a record that is not Noop v, Noop v#. */
AMC_API size_t amc_check_inherited_trace_workspace(int64_t n_ops, int32_t n_arrays);
AMC_API int amc_check_inherited_trace(const uint8_t* kind_side, const int32_t* var, int64_t n_ops, int32_t n_arrays,
                                      const int32_t* arr_parent, const int64_t* arr_probe, uint8_t* step_status,
                                      uint8_t* final_status, int32_t* var_first_fault, int64_t* first_fault,
                                      void* workspace, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* (3) Batches of structured programs, relation mode -- Fig. Opsem with      */
/*     opaque conditions: If = union of both branches, While = closure of    */
/*     its body.                                                             */
/* ------------------------------------------------------------------------ */

/* Largest If/While nesting depth amc_check_batch accepts. */
#define AMC_MAX_DEPTH 8

/* Workspace bytes amc_check_batch needs. */
AMC_API size_t amc_check_batch_workspace(int64_t n_tokens, int64_t n_progs, int64_t total_vars);

/* Checks n_progs independent programs in one launch sequence.  Program p owns
 * tokens [prog_tok_off[p], prog_tok_off[p+1]) of tok_kind_side / tok_payload
 * and variables 0..prog_nvars[p]-1 (stored at prog_var_off[p] in final_mask).
 * Op tokens carry their program-local variable id in the payload; IF, ELSE and
 * WHILE carry the token length of the branch / body that follows, END 0:
 *   IF(n_then) <then> ELSE(n_else) <else> END,   WHILE(n_body) <body> END.
 * Every variable starts as the set {(V,I)}.  Outputs: step_mask[token] = set
 * of possible statuses of the op's variable after the op (0 for structure
 * tokens); final_mask[prog_var_off[p] + v]; prog_first_fault[p] = smallest
 * program-relative token index of an op whose possible pre-statuses include a
 * non-stuck status that the op makes stuck (-1 if none).
 * graph_capture = 1 launches through a cached CUDA graph for this shape.
 * Errors: host-side checks of sizes; device-side (amc_sync_status)
 * AMC_E_INVALID for unbalanced tokens, depth > AMC_MAX_DEPTH or bad op bytes,
 * AMC_E_RANGE for a var id out of its program's range. */
AMC_API int amc_check_batch(const uint8_t* tok_kind_side, const int32_t* tok_payload,
                    const int64_t* prog_tok_off, const int32_t* prog_nvars,
                    const int64_t* prog_var_off, int64_t n_progs, int64_t n_tokens,
                    uint8_t* step_mask, uint8_t* final_mask, int64_t* prog_first_fault,
                    int graph_capture, void* workspace, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* (3b) Static well-declaredness of calls AM{S} -- Section 3.3, Definitions   */
/*      "Occurs in all execution paths" and "Well-declared program";         */
/*      Section 3.5, "Well-declared program with array access".              */
/* ------------------------------------------------------------------------ */

/* Most declarations one call may have. */
#define AMC_WD_MAX_DECLS 32

/* Workspace bytes amc_check_well_declared needs (a work-queue counter). */
AMC_API size_t amc_check_well_declared_workspace(int64_t n_calls);

/* Checks n_calls calls AM{S}, each a function body S guarded by access-mode
 * declarations AM, against the definition of a well-declared program.
 * Locations: a scalar variable or one element of an array; array a owns the
 * locations [arr_loc_off[a], arr_loc_off[a+1]) and is represented by one
 * abstract variable (loc_owner[l] = the array owning location l).
 *   arr_loc_off [n_arrays + 1], loc_owner [arr_loc_off[n_arrays]]
 *   call_tok_off [n_calls + 1]  body tokens of call c: [off[c], off[c+1]) of
 *                               tok / payload [n_tokens]: ops r / w / Push /
 *                               Pull / Noop (kind | side << 4, payload = a
 *                               location) and IF / ELSE / WHILE / END (payload
 *                               = branch / body length, as in amc_check_batch),
 *                               nested at most AMC_MAX_DEPTH deep
 *   call_am_off [n_calls + 1]   declarations of call c: [off[c], off[c+1]) of
 *                               am_array / am_mode [n_decls] (mode R 1, W 2,
 *                               RW 3, | side << 4), at most AMC_WD_MAX_DECLS
 * Outputs per call: violations[c] bit 0 a Push or Pull in the body (only the
 * declarations may synchronise), bit 1 a write whose array has no W / RW
 * declaration on the write's side, bit 2 a read without R / RW on its side,
 * bit 3 a W declaration with a location of its array that is not written, on
 * that side, in all execution paths of the body (conditions are opaque: both
 * branches of an If, and zero or more runs of a While, are paths), bit 4 an
 * array declared twice; first_bad[c] = call-relative index of the first token
 * with a bit 0-2 violation (-1 none); first_unmet[c] = smallest array id with
 * a bit-3 violation (-1 none).  A call is well-declared iff violations[c] = 0.
 * Errors (via amc_sync_status): AMC_E_INVALID for malformed tokens (unbalanced
 * or too deep constructs, pw / GT / EN in a body), bad modes or more than
 * AMC_WD_MAX_DECLS declarations; AMC_E_RANGE for ids out of range. */
AMC_API int amc_check_well_declared(const int64_t* arr_loc_off, int32_t n_arrays, const int32_t* loc_owner,
                                    const int64_t* call_tok_off, int64_t n_calls, const uint8_t* tok,
                                    const int32_t* payload, int64_t n_tokens, const int64_t* call_am_off,
                                    const int32_t* am_array, const uint8_t* am_mode, int64_t n_decls,
                                    uint32_t* violations, int64_t* first_bad, int32_t* first_unmet,
                                    void* workspace, size_t ws_bytes, void* stream);

/* Path-sensitive relation mode -- Fig. Opsem with the conditions of Section
 * 3.2 evaluated (rules valid / invalid / rem-valid / rem-invalid): IF and
 * WHILE token bits 4-5 give the condition, 0 = opaque (x (+) y, both
 * outcomes), 1 = isValid g, 2 = remIsValid g, on the program's guard
 * variable g = prog_guard[p] (-1: none, every condition must be opaque).
 * For every variable x other than g the set of reachable pairs (status of g,
 * status of x) is tracked (exact, as control flow depends on g alone); a
 * stuck g satisfies no condition rule, so its paths end at the next
 * condition; each variable's F is absorbing and does not stop the others.
 * Outputs as amc_check_batch: step_mask[token] = statuses the op's variable
 * may have after the op (0 for structure tokens and for ops no path reaches),
 * final_mask, prog_first_fault.  Errors (device): AMC_E_INVALID for
 * malformed tokens, a condition without a guard, a guard out of range or
 * depth > AMC_MAX_DEPTH; AMC_E_RANGE for a variable id out of range. */
AMC_API size_t amc_check_batch_guarded_workspace(int64_t n_tokens, int64_t n_progs, int64_t total_vars);
AMC_API int amc_check_batch_guarded(const uint8_t* tok_kind_side, const int32_t* tok_payload,
                                    const int64_t* prog_tok_off, const int32_t* prog_nvars,
                                    const int64_t* prog_var_off, const int32_t* prog_guard, int64_t n_progs,
                                    int64_t n_tokens, int64_t total_vars, uint8_t* step_mask, uint8_t* final_mask,
                                    int64_t* prog_first_fault, void* workspace, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* (4) Serving -- continuous batching of check requests with per-session     */
/*     variable statuses kept on the device between requests.                */
/* ------------------------------------------------------------------------ */
typedef struct amc_server amc_server;

enum { AMC_REQ_TRACE = 0, AMC_REQ_PROGRAM = 1 };
enum { AMC_REQ_BORROW = 1 };

/* A request, described on the host.  Buffers are HOST pointers, copied into
 * the server's pinned staging before amc_serve_submit returns -- unless flags
 * holds AMC_REQ_BORROW: then the server reads them when the request runs, and
 * the caller keeps them valid and unchanged until amc_serve_poll reports the
 * request done (page-locked buffers make that copy asynchronous).
 * TRACE: kind_side / var of n_items ops, as for amc_check_trace; they are
 * checked on the device (a bad byte or id is the request's `error`).
 * PROGRAM: kind_side / var hold the token bytes and payloads of n_items
 * tokens, checked at submission.  n_vars sizes the session on its first
 * request and must match afterwards.  A session takes both kinds in any
 * order: it keeps, per variable, the set of statuses the variable may have
 * (every variable starts as {(V,I)}). */
typedef struct {
    int kind;
    int32_t n_vars;
    int64_t n_items;
    const uint8_t* kind_side;
    const int32_t* var;
    int flags;               /* 0 or AMC_REQ_BORROW */
} amc_request;

/* Result of a finished request.  `status` holds n_items host bytes, valid
 * until amc_serve_release(ticket): status masks (is_mask = 1) for a PROGRAM,
 * and for a TRACE whose session has run a program with If / While before it
 * (its variables may then hold sets of several statuses; the trace is checked
 * in relation mode, first_fault as for amc_check_batch); else status codes
 * (is_mask = 0, first_fault as for amc_check_trace). */
typedef struct {
    int error;               /* AMC_OK, or the device-side error of this request's check */
    int64_t first_fault;     /* request-relative index, -1 none */
    int64_t n_items;
    const uint8_t* status;
    double t_submit, t_admit, t_done;   /* seconds, server clock */
    int is_mask;             /* 1: `status` holds masks, 0: status codes */
} amc_result;

/* Creates a server on the current device that holds at most max_slots
 * requests on the device at once and at most mem_budget_bytes of device
 * memory for requests and sessions. */
AMC_API int amc_server_create(size_t mem_budget_bytes, int max_slots, amc_server** out);
/* Queues a request of a session (requests of one session run in submission
 * order; different sessions overlap on the device).  Returns AMC_E_AGAIN when
 * the queue is full. */
AMC_API int amc_serve_submit(amc_server* srv, uint64_t session_id, const amc_request* req, uint64_t* ticket);
/* Non-blocking: *done = 1 and *out filled once the request finished.  A
 * request that reports an error leaves its session's statuses unspecified. */
AMC_API int amc_serve_poll(amc_server* srv, uint64_t ticket, int* done, amc_result* out);
/* Non-blocking: writes to tickets[0..*n) up to cap tickets of requests that
 * finished since the previous call (each reported once, in finishing order),
 * so that a client polls only what is done. */
AMC_API int amc_serve_completed(amc_server* srv, uint64_t* tickets, int32_t cap, int32_t* n);
/* Frees a finished request's host result. */
AMC_API int amc_serve_release(amc_server* srv, uint64_t ticket);
/* Copies a session's current variable status sets (status masks, bit k set
 * <=> status code k is possible) to host memory, after its queued requests. */
AMC_API int amc_session_export(amc_server* srv, uint64_t session_id, uint8_t* host_status, int32_t n_vars);
/* Waits for all queued requests, then frees the server. */
AMC_API int amc_server_destroy(amc_server* srv);

#ifdef __cplusplus
}
#endif
#endif /* AMC_H */
