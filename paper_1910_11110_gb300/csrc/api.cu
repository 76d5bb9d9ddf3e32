// api.cu -- C ABI entry points: argument checks, workspace layout, launches.
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "amc_internal.cuh"
#include "scan_trace.cuh"
#include "translate.cuh"
#include "batch.cuh"
#include "batch_ps.cuh"
#include "autotune.cuh"
#include "wd.cuh"
#include "kloc.cuh"

using namespace amc;

namespace {

inline bool aligned256(const void* p) { return ((uintptr_t)p & 255) == 0; }

// the guard pass's first faults (discarded), then its pre-statuses: the guards
// of the second pass, in a buffer of their own so that no pass reads what it
// writes
size_t guarded_extra_bytes(int64_t n_ops, int32_t n_vars)
{
    return align_up(4 * (size_t)n_vars, 256) + 256 + align_up((size_t)n_ops, 256);
}

int check_trace_args(const uint8_t* kind_side, const int32_t* var, int64_t n_ops, int32_t n_vars,
                     uint8_t* step_status, uint8_t* final_status, int32_t* var_first_fault,
                     int64_t* first_fault)
{
    if (n_ops < 0 || n_ops > INT32_MAX || n_vars < 0) return AMC_E_INVALID;
    if (n_ops > 0 && (n_vars < 1 || !kind_side || !var || !step_status)) return AMC_E_INVALID;
    if (n_vars > 0 && (!final_status || !var_first_fault)) return AMC_E_INVALID;
    if (!first_fault) return AMC_E_INVALID;
    return AMC_OK;
}

// CUDA graphs of amc_check_batch, one per (device, stream, arguments)
struct GraphCache {
    std::mutex mu;
    std::map<std::vector<uintptr_t>, cudaGraphExec_t> execs;
};
GraphCache& graph_cache()
{
    static GraphCache* c = new GraphCache();      // never destroyed: graphs live until exit
    return *c;
}

constexpr int MAX_TRACE_GRAPHS = 256;

// Trace-check graphs captured so far (under the graph cache's lock).
int& trace_graph_count()
{
    static int n = 0;
    return n;
}

// Repeated trace checks replay a captured graph unless AMC_TRACE_GRAPH=0 or
// the stream is the legacy default stream (which cannot be captured) or is
// being captured by the caller.
bool trace_graphs_enabled(cudaStream_t s)
{
    const char* e = getenv("AMC_TRACE_GRAPH");
    if (e && e[0] == '0') return false;
    if (s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread) return false;
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess || st != cudaStreamCaptureStatusNone) return false;
    return true;
}

// The tuning knobs the launch functions read per call, as part of a graph key
// (a changed knob captures a new graph).
void append_knobs(std::vector<uintptr_t>& key)
{
    static const char* const knobs[] = {"AMC_SCAN_FB_BITS", "AMC_SCAN_GROUP", "AMC_SCAN_CTAS_PER_SM",
                                        "AMC_SCAN_DENSE", "AMC_SCAN_DENSE_SORT", "AMC_SCAN_PREFIX",
                                        "AMC_SCAN_TAIL"};
    for (const char* k : knobs) {
        const char* v = getenv(k);
        uintptr_t h = 1469598103934665603ull;         // FNV-1a of the value (0 when unset)
        if (!v) {
            h = 0;
        } else {
            for (const char* c = v; *c; ++c) h = (h ^ (uint8_t)*c) * 1099511628211ull;
        }
        key.push_back(h);
    }
}

}  // namespace

extern "C" {

int amc_version(void) { return 10000; }

int amc_set_profile_events(void* start_event, void* stop_event)
{
    amc::set_profile_events(static_cast<cudaEvent_t>(start_event), static_cast<cudaEvent_t>(stop_event));
    return AMC_OK;
}

int amc_debug_scan_phases(int enable, uint64_t* host_out)
{
    return scan_phase_profile(enable, reinterpret_cast<unsigned long long*>(host_out));
}

const char* amc_error_string(int code)
{
    switch (code) {
    case AMC_OK: return "ok";
    case AMC_E_INVALID: return "malformed input";
    case AMC_E_RANGE: return "id out of range or capacity exceeded";
    case AMC_E_NOMEM: return "workspace too small or memory budget exceeded";
    case AMC_E_TIMEOUT: return "a bounded device-side wait expired";
    case AMC_E_CUDA: return "CUDA runtime error";
    case AMC_E_AGAIN: return "no slot free yet";
    }
    return "unknown error";
}

int amc_sync_status(void* stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return AMC_E_CUDA;
    int* w = device_error_word();
    if (!w) return AMC_E_CUDA;
    int v = 0;
    if (cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return AMC_E_CUDA;
    if (v != 0) {
        int z = 0;
        if (cudaMemcpy(w, &z, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return AMC_E_CUDA;
    }
    return v;
}

size_t amc_check_trace_workspace(int64_t n_ops, int32_t n_vars)
{
    if (n_ops < 0 || n_vars < 0) return 0;
    return scan_workspace_bytes(n_ops, n_vars);
}

int amc_check_trace(const uint8_t* kind_side, const int32_t* var, int64_t n_ops, int32_t n_vars,
                    const uint8_t* init_status, uint8_t* step_status, uint8_t* final_status,
                    int32_t* var_first_fault, int64_t* first_fault, void* workspace, size_t ws_bytes,
                    void* stream)
{
    int rc = check_trace_args(kind_side, var, n_ops, n_vars, step_status, final_status, var_first_fault,
                              first_fault);
    if (rc) return rc;
    if (init_status && n_vars > 0 && init_status < final_status + n_vars && final_status < init_status + n_vars)
        return AMC_E_INVALID;
    if (!workspace || !aligned256(workspace) || ws_bytes < scan_workspace_bytes(n_ops, n_vars))
        return AMC_E_NOMEM;
    int* err = device_error_word();
    if (!err) return AMC_E_CUDA;
    ScanLaunch L;
    L.kind_side = kind_side;
    L.var = var;
    L.n_ops = n_ops;
    L.n_vars = n_vars;
    L.init = init_status;
    L.step = step_status;
    L.final_status = final_status;
    L.vff = var_first_fault;
    L.first_fault = first_fault;
    L.err = err;
    L.workspace = workspace;
    L.profile = 3;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // candidates, timed on the first call of a shape bucket: the path by size
    // with the single-pass scan's stuck bitmap read through L1 (three CTAs per
    // SM), in shared memory (2^20 variables, one CTA per SM) or none, each with
    // groups of up to 16 tiles per claim; or L1 and single tiles; the reduce /
    // carry / apply path at any size; the epoch path at any size (else the
    // single-pass scan alone)
    static const int fb[6] = {-2, 1 << 20, -1, -2, -2, -2};
    static const int grp[6] = {16, 16, 16, 1, 16, 16};
    static const int dns[6] = {-1, -1, -1, -1, 1, 0};
    static const int tl[6] = {-1, -1, -1, -1, 0, 1};
    auto run = [&](int i) {
        ScanLaunch C = L;
        C.fb_max_bits = fb[i];
        C.group_max = grp[i];
        C.dense = dns[i];
        C.tail = tl[i];
        return launch_scan_trace(C, s);
    };
    if (const char* e = getenv("AMC_TRACE_CANDIDATE")) {        // test override: one candidate, untimed
        const int i = atoi(e);
        if (i >= 0 && i < 6) return run(i);
    }
    const std::string key = shape_key("trace", n_ops, n_vars, init_status ? 1 : 0);
    const int pick = autotune_lookup(key);
    if (pick < 0 || !trace_graphs_enabled(s)) return autotune_run(key, 6, 0, s, run);
    // the size class is decided: the launch sequence depends only on the
    // arguments and the tuning knobs, so it is captured once into a CUDA graph
    // and replayed (one launch instead of one per kernel)
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<uintptr_t> gkey = {0x7472616365,        (uintptr_t)dev,           (uintptr_t)s,
                                  (uintptr_t)kind_side, (uintptr_t)var,           (uintptr_t)n_ops,
                                  (uintptr_t)n_vars,    (uintptr_t)init_status,   (uintptr_t)step_status,
                                  (uintptr_t)final_status, (uintptr_t)var_first_fault, (uintptr_t)first_fault,
                                  (uintptr_t)workspace, (uintptr_t)pick};
    append_knobs(gkey);
    GraphCache& gc = graph_cache();
    std::lock_guard<std::mutex> lock(gc.mu);
    auto it = gc.execs.find(gkey);
    if (it == gc.execs.end()) {
        // graphs are kept until exit: past MAX_TRACE_GRAPHS distinct argument
        // sets, further ones run without a graph
        if (++trace_graph_count() > MAX_TRACE_GRAPHS) return run(pick);
        L.profile = 0;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return AMC_E_CUDA;
        const int rc = run(pick);
        const cudaError_t ce = cudaStreamEndCapture(s, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ce != cudaSuccess) return AMC_E_CUDA;
        cudaGraphExec_t ex = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return AMC_E_CUDA;
        it = gc.execs.emplace(gkey, ex).first;
    }
    profile_begin(s);
    const cudaError_t le = cudaGraphLaunch(it->second, s);
    profile_end(s);
    return le == cudaSuccess ? AMC_OK : AMC_E_CUDA;
}

int amc_check_trace_plan(int64_t n_ops, int32_t n_vars, int has_init, int32_t* path, int32_t* launches)
{
    if (n_ops < 0 || n_vars < 0) return AMC_E_INVALID;
    static const int dns[6] = {-1, -1, -1, -1, 1, 0};
    static const int tl[6] = {-1, -1, -1, -1, 0, 1};
    int pick = autotune_lookup(shape_key("trace", n_ops, n_vars, has_init ? 1 : 0));
    if (const char* e = getenv("AMC_TRACE_CANDIDATE")) pick = atoi(e);
    if (pick < 0 || pick >= 6) pick = 0;
    ScanLaunch L;
    L.n_ops = n_ops;
    L.n_vars = n_vars;
    static uint8_t stand_in = 0;                     // the plan only tests these against null
    L.init = has_init ? &stand_in : nullptr;
    L.final_status = &stand_in;
    L.dense = dns[pick];
    L.tail = tl[pick];
    int n = 0;
    const int p = scan_trace_plan(L, &n);
    if (path) *path = p;
    if (launches) *launches = n;
    return AMC_OK;
}

size_t amc_check_guarded_trace_workspace(int64_t n_ops, int32_t n_vars)
{
    if (n_ops < 0 || n_vars < 0) return 0;
    return scan_workspace_bytes(n_ops, n_vars) + guarded_extra_bytes(n_ops, n_vars);
}

int amc_check_guarded_trace(const uint8_t* kind_side, const int32_t* var, int64_t n_ops, int32_t n_vars,
                            const uint8_t* init_status, uint8_t* step_status, uint8_t* final_status,
                            int32_t* var_first_fault, int64_t* first_fault, void* workspace,
                            size_t ws_bytes, void* stream)
{
    int rc = check_trace_args(kind_side, var, n_ops, n_vars, step_status, final_status, var_first_fault,
                              first_fault);
    if (rc) return rc;
    if (!workspace || !aligned256(workspace) || ws_bytes < amc_check_guarded_trace_workspace(n_ops, n_vars))
        return AMC_E_NOMEM;
    int* err = device_error_word();
    if (!err) return AMC_E_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t* w = static_cast<uint8_t*>(workspace);
    uint8_t* extra = w + scan_workspace_bytes(n_ops, n_vars);
    int32_t* vff_scratch = reinterpret_cast<int32_t*>(extra);
    int64_t* ff_scratch = reinterpret_cast<int64_t*>(extra + align_up(4 * (size_t)n_vars, 256));
    uint8_t* guard = extra + align_up(4 * (size_t)n_vars, 256) + 256;
    // pass 1: pre-statuses of every op with GT as Noop (guards read abstract
    // variables, which GT never touches)
    ScanLaunch A;
    A.kind_side = kind_side;
    A.var = var;
    A.n_ops = n_ops;
    A.n_vars = n_vars;
    A.init = init_status;
    A.step = guard;
    A.vff = vff_scratch;
    A.first_fault = ff_scratch;
    A.pre_mode = 1;
    A.err = err;
    A.workspace = workspace;
    A.profile = 1;          // the profiled span covers both scans
    // the choice tuned for plain traces of this shape, if any (the epoch path
    // does not take guards)
    static const int fb[6] = {-2, 1 << 20, -1, -2, -2, -2};
    static const int grp[6] = {16, 16, 16, 1, 16, 16};
    static const int dns[6] = {-1, -1, -1, -1, 1, 0};
    int pick = autotune_lookup(shape_key("trace", n_ops, n_vars, init_status ? 1 : 0));
    if (pick < 0 || pick >= 6) pick = 0;
    A.fb_max_bits = fb[pick];
    A.group_max = grp[pick];
    A.dense = dns[pick];
    // candidates, timed on the first call of a size class: that choice, or
    // both passes on the reduce / carry / apply path (a translated trace of a
    // well-declared program gets almost nothing stuck, so every op stays live)
    auto run = [&](int i) {
        ScanLaunch P1 = A;
        if (i == 1) P1.dense = 1;
        int r = launch_scan_trace(P1, s);
        if (r) return r;
        // pass 2: GT resolved from the pre-status of the EN that follows it
        ScanLaunch P2 = P1;
        P2.step = step_status;
        P2.final_status = final_status;
        P2.vff = var_first_fault;
        P2.first_fault = first_fault;
        P2.guard = guard;
        P2.pre_mode = 0;
        P2.profile = 2;
        return launch_scan_trace(P2, s);
    };
    if (const char* e = getenv("AMC_GUARDED_CANDIDATE")) {      // test override: one candidate, untimed
        const int i = atoi(e);
        if (i == 0 || i == 1) return run(i);
    }
    return autotune_run(shape_key("guarded", n_ops, n_vars, init_status ? 1 : 0), 2, 0, s, run);
}

size_t amc_translate_vectorpu_workspace(int32_t n_arrays, int64_t n_calls, int64_t n_operands)
{
    if (n_arrays < 0 || n_calls < 0 || n_operands < 0) return 0;
    return translate_workspace_bytes(n_arrays, n_calls);
}

int amc_translate_vectorpu(const int32_t* arr_start, const int32_t* arr_len, int32_t n_arrays,
                           const uint8_t* call_side, const int32_t* call_off, int64_t n_calls,
                           const int32_t* opnd_array, const uint8_t* opnd_mode, int64_t n_operands,
                           int infer_overlap, uint8_t* out_kind_side, int32_t* out_var, int64_t out_cap,
                           int64_t* out_n, int64_t* call_first_op, void* workspace, size_t ws_bytes,
                           void* stream)
{
    if (n_arrays < 0 || n_arrays > INT32_MAX / 2 || n_calls < 0 || n_calls > INT32_MAX || n_operands < 0 ||
        out_cap < 0)
        return AMC_E_INVALID;
    if (!out_n || !call_first_op || !call_off) return AMC_E_INVALID;
    if (n_arrays > 0 && (!arr_start || !arr_len)) return AMC_E_INVALID;
    if (n_calls > 0 && !call_side) return AMC_E_INVALID;
    if (n_operands > 0 && (!opnd_array || !opnd_mode)) return AMC_E_INVALID;
    if (out_cap > 0 && (!out_kind_side || !out_var)) return AMC_E_INVALID;
    if (!workspace || !aligned256(workspace) || ws_bytes < translate_workspace_bytes(n_arrays, n_calls))
        return AMC_E_NOMEM;
    int* err = device_error_word();
    if (!err) return AMC_E_CUDA;
    TranslateLaunch T;
    T.arr_start = arr_start;
    T.arr_len = arr_len;
    T.n_arrays = n_arrays;
    T.call_side = call_side;
    T.call_off = call_off;
    T.n_calls = n_calls;
    T.opnd_array = opnd_array;
    T.opnd_mode = opnd_mode;
    T.n_operands = n_operands;
    T.infer = infer_overlap ? 1 : 0;
    T.out_ks = out_kind_side;
    T.out_var = out_var;
    T.out_cap = out_cap;
    T.out_n = out_n;
    T.call_first_op = call_first_op;
    T.err = err;
    T.workspace = workspace;
    T.profile = 3;
    return launch_translate(T, static_cast<cudaStream_t>(stream));
}

size_t amc_vectorpu_overlap_pairs_workspace(int32_t n_arrays, int64_t n_calls)
{
    if (n_arrays < 0 || n_calls < 0) return 0;
    return overlap_count_workspace_bytes(n_arrays, n_calls, true);
}

int amc_vectorpu_overlap_pairs(const int32_t* arr_start, const int32_t* arr_len, const int32_t* arr_born,
                               const int32_t* arr_died, int32_t n_arrays, int64_t n_calls, int64_t* n_pairs,
                               void* workspace, size_t ws_bytes, void* stream)
{
    if (n_arrays < 0 || n_calls < 0 || !n_pairs || (n_arrays > 0 && (!arr_start || !arr_len)) ||
        (!arr_born != !arr_died))
        return AMC_E_INVALID;
    if (!workspace || !aligned256(workspace) ||
        ws_bytes < overlap_count_workspace_bytes(n_arrays, n_calls, arr_born != nullptr))
        return AMC_E_NOMEM;
    int* err = device_error_word();
    if (!err) return AMC_E_CUDA;
    return launch_overlap_count(arr_start, arr_len, arr_born, arr_died, n_arrays, n_calls, n_pairs, err, workspace,
                                static_cast<cudaStream_t>(stream));
}

size_t amc_translate_vectorpu_lifetimes_workspace(int32_t n_arrays, int64_t n_calls, int64_t n_operands,
                                                  int64_t max_pairs)
{
    if (n_arrays < 0 || n_calls < 0 || n_operands < 0 || max_pairs < 0) return 0;
    return translate_lifetimes_workspace_bytes(n_arrays, n_calls, max_pairs);
}

int amc_translate_vectorpu_lifetimes(const int32_t* arr_start, const int32_t* arr_len, const int32_t* arr_parent,
                                     const int32_t* arr_born, const int32_t* arr_died, int32_t n_arrays,
                                     const uint8_t* call_side, const int32_t* call_off, int64_t n_calls,
                                     const int32_t* opnd_array, const uint8_t* opnd_mode, int64_t n_operands,
                                     int infer_overlap, int64_t max_pairs, uint8_t* out_kind_side, int32_t* out_var,
                                     int64_t out_cap, int64_t* out_n, int64_t* call_first_op, int64_t* arr_probe,
                                     void* workspace, size_t ws_bytes, void* stream)
{
    if (n_arrays < 0 || n_arrays > INT32_MAX / 2 || n_calls < 0 || n_calls >= INT32_MAX || n_operands < 0 ||
        out_cap < 0 || max_pairs < 0)
        return AMC_E_INVALID;
    if (!out_n || !call_first_op || !call_off) return AMC_E_INVALID;
    if (n_arrays > 0 && (!arr_start || !arr_len || !arr_parent || !arr_born || !arr_died || !arr_probe))
        return AMC_E_INVALID;
    if (n_calls > 0 && !call_side) return AMC_E_INVALID;
    if (n_operands > 0 && (!opnd_array || !opnd_mode)) return AMC_E_INVALID;
    if (out_cap > 0 && (!out_kind_side || !out_var)) return AMC_E_INVALID;
    if (!workspace || !aligned256(workspace) ||
        ws_bytes < translate_lifetimes_workspace_bytes(n_arrays, n_calls, max_pairs))
        return AMC_E_NOMEM;
    int* err = device_error_word();
    if (!err) return AMC_E_CUDA;
    TranslateLaunch T;
    T.arr_start = arr_start;
    T.arr_len = arr_len;
    T.n_arrays = n_arrays;
    T.call_side = call_side;
    T.call_off = call_off;
    T.n_calls = n_calls;
    T.opnd_array = opnd_array;
    T.opnd_mode = opnd_mode;
    T.n_operands = n_operands;
    T.infer = infer_overlap ? 1 : 0;
    T.out_ks = out_kind_side;
    T.out_var = out_var;
    T.out_cap = out_cap;
    T.out_n = out_n;
    T.call_first_op = call_first_op;
    T.err = err;
    T.workspace = workspace;
    T.profile = 3;
    T.arr_born = n_arrays > 0 ? arr_born : nullptr;
    T.arr_died = arr_died;
    T.arr_parent = arr_parent;
    T.max_pairs = max_pairs;
    T.arr_probe = arr_probe;
    return launch_translate(T, static_cast<cudaStream_t>(stream));
}

size_t amc_check_inherited_trace_workspace(int64_t n_ops, int32_t n_arrays)
{
    if (n_ops < 0 || n_arrays < 0 || n_arrays > INT32_MAX / 2) return 0;
    return amc_check_guarded_trace_workspace(n_ops, 2 * n_arrays) + align_up(2 * (size_t)n_arrays + 1, 256);
}

int amc_check_inherited_trace(const uint8_t* kind_side, const int32_t* var, int64_t n_ops, int32_t n_arrays,
                              const int32_t* arr_parent, const int64_t* arr_probe, uint8_t* step_status,
                              uint8_t* final_status, int32_t* var_first_fault, int64_t* first_fault,
                              void* workspace, size_t ws_bytes, void* stream)
{
    if (n_arrays < 0 || n_arrays > INT32_MAX / 2 || n_ops < 0) return AMC_E_INVALID;
    if (n_arrays > 0 && (!arr_parent || !arr_probe)) return AMC_E_INVALID;
    const size_t gws = amc_check_guarded_trace_workspace(n_ops, 2 * n_arrays);
    if (!workspace || !aligned256(workspace) || ws_bytes < amc_check_inherited_trace_workspace(n_ops, n_arrays))
        return AMC_E_NOMEM;
    int* err = device_error_word();
    if (!err) return AMC_E_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint8_t* init = static_cast<uint8_t*>(workspace) + gws;
    // pass 1 from the initial store: the vectors' statuses at every creation
    // record (a vector's ops do not depend on any pvector's statuses)
    int rc = amc_check_guarded_trace(kind_side, var, n_ops, 2 * n_arrays, nullptr, step_status, final_status,
                                     var_first_fault, first_fault, workspace, gws, stream);
    if (rc) return rc;
    rc = launch_inherit(var, n_ops, n_arrays, arr_parent, arr_probe, step_status, init, err, s);
    if (rc) return rc;
    // pass 2 from the inherited statuses
    return amc_check_guarded_trace(kind_side, var, n_ops, 2 * n_arrays, n_arrays > 0 ? init : nullptr, step_status,
                                   final_status, var_first_fault, first_fault, workspace, gws, stream);
}

size_t amc_check_batch_guarded_workspace(int64_t n_tokens, int64_t n_progs, int64_t total_vars)
{
    if (n_tokens < 0 || n_progs < 0 || total_vars < 0) return 0;
    return batch_ps_workspace_bytes(n_progs, total_vars);
}

int amc_check_batch_guarded(const uint8_t* tok_kind_side, const int32_t* tok_payload, const int64_t* prog_tok_off,
                            const int32_t* prog_nvars, const int64_t* prog_var_off, const int32_t* prog_guard,
                            int64_t n_progs, int64_t n_tokens, int64_t total_vars, uint8_t* step_mask,
                            uint8_t* final_mask, int64_t* prog_first_fault, void* workspace, size_t ws_bytes,
                            void* stream)
{
    if (n_progs < 0 || n_tokens < 0 || total_vars < 0) return AMC_E_INVALID;
    if (n_progs > 0 && (!prog_tok_off || !prog_nvars || !prog_var_off || !prog_guard || !prog_first_fault))
        return AMC_E_INVALID;
    if (n_tokens > 0 && (!tok_kind_side || !tok_payload || !step_mask)) return AMC_E_INVALID;
    if (total_vars > 0 && !final_mask) return AMC_E_INVALID;
    if (!workspace || !aligned256(workspace) || ws_bytes < batch_ps_workspace_bytes(n_progs, total_vars))
        return AMC_E_NOMEM;
    int* err = device_error_word();
    if (!err) return AMC_E_CUDA;
    PsLaunch B;
    B.tok = tok_kind_side;
    B.payload = tok_payload;
    B.prog_tok_off = prog_tok_off;
    B.prog_nvars = prog_nvars;
    B.prog_var_off = prog_var_off;
    B.prog_guard = prog_guard;
    B.n_progs = n_progs;
    B.n_tokens = n_tokens;
    B.total_vars = total_vars;
    B.step_mask = step_mask;
    B.final_mask = final_mask;
    B.prog_first_fault = prog_first_fault;
    B.err = err;
    B.workspace = workspace;
    B.profile = 3;
    return launch_batch_ps(B, static_cast<cudaStream_t>(stream));
}

size_t amc_check_batch_workspace(int64_t n_tokens, int64_t n_progs, int64_t total_vars)
{
    if (n_tokens < 0 || n_progs < 0 || total_vars < 0) return 0;
    return batch_workspace_bytes(n_tokens, n_progs);
}

int amc_check_batch(const uint8_t* tok_kind_side, const int32_t* tok_payload, const int64_t* prog_tok_off,
                    const int32_t* prog_nvars, const int64_t* prog_var_off, int64_t n_progs, int64_t n_tokens,
                    uint8_t* step_mask, uint8_t* final_mask, int64_t* prog_first_fault, int graph_capture,
                    void* workspace, size_t ws_bytes, void* stream)
{
    if (n_progs < 0 || n_tokens < 0 || n_progs > INT32_MAX) return AMC_E_INVALID;
    if (n_progs > 0 && (!prog_tok_off || !prog_nvars || !prog_var_off || !prog_first_fault || !final_mask))
        return AMC_E_INVALID;
    if (n_tokens > 0 && (!tok_kind_side || !tok_payload || !step_mask)) return AMC_E_INVALID;
    if (!workspace || !aligned256(workspace) || ws_bytes < batch_workspace_bytes(n_tokens, n_progs))
        return AMC_E_NOMEM;
    int* err = device_error_word();
    if (!err) return AMC_E_CUDA;
    BatchLaunch B;
    B.tok = tok_kind_side;
    B.payload = tok_payload;
    B.prog_tok_off = prog_tok_off;
    B.prog_nvars = prog_nvars;
    B.prog_var_off = prog_var_off;
    B.n_progs = n_progs;
    B.n_tokens = n_tokens;
    B.step_mask = step_mask;
    B.final_mask = final_mask;
    B.prog_first_fault = prog_first_fault;
    B.err = err;
    B.workspace = workspace;
    B.profile = 3;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // candidates (longest-first queue): registers fitted to six or four CTAs
    // per SM
    auto shape = [&](BatchLaunch X, int i) {
        X.longest_first = 1;
        X.regs_capped = (i & 1) ? 0 : 1;
        return X;
    };
    const std::string key = shape_key("batch", n_tokens, n_progs, 0);
    if (!graph_capture || s == nullptr)
        return autotune_run(key, 2, 0, s, [&](int i) { return launch_batch(shape(B, i), s); });
    {
        // tune outside the capture first (no-op when the key is cached)
        const int rc0 = autotune_lookup(key) >= 0
                            ? AMC_OK
                            : autotune_run(key, 2, 0, s, [&](int i) { return launch_batch(shape(B, i), s); });
        if (rc0) return rc0;
        const int pick = autotune_lookup(key);
        B = shape(B, pick >= 0 ? pick : 0);
    }
    int dev = 0;
    cudaGetDevice(&dev);
    std::vector<uintptr_t> gkey = {(uintptr_t)dev,          (uintptr_t)s,           (uintptr_t)tok_kind_side,
                                  (uintptr_t)tok_payload,  (uintptr_t)prog_tok_off, (uintptr_t)prog_nvars,
                                  (uintptr_t)prog_var_off, (uintptr_t)n_progs,      (uintptr_t)n_tokens,
                                  (uintptr_t)step_mask,    (uintptr_t)final_mask,   (uintptr_t)prog_first_fault,
                                  (uintptr_t)workspace};
    GraphCache& gc = graph_cache();
    std::lock_guard<std::mutex> lock(gc.mu);
    auto it = gc.execs.find(gkey);
    if (it == gc.execs.end()) {
        B.profile = 0;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return AMC_E_CUDA;
        const int rc = launch_batch(B, s);
        const cudaError_t ce = cudaStreamEndCapture(s, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ce != cudaSuccess) return AMC_E_CUDA;
        cudaGraphExec_t ex = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) return AMC_E_CUDA;
        it = gc.execs.emplace(gkey, ex).first;
    }
    profile_begin(s);
    const cudaError_t le = cudaGraphLaunch(it->second, s);
    profile_end(s);
    return le == cudaSuccess ? AMC_OK : AMC_E_CUDA;
}

size_t amc_check_trace_k_workspace(int64_t n_ops, int32_t n_vars)
{
    if (n_ops < 0 || n_vars < 0) return 0;
    return kloc_workspace_bytes(n_ops);
}

int amc_check_trace_k(const uint8_t* op, const int32_t* var, int64_t n_ops, int32_t n_vars, int32_t k,
                      const uint8_t* init_status, uint8_t* step_status, uint8_t* final_status,
                      int32_t* var_first_fault, int64_t* first_fault, void* workspace, size_t ws_bytes,
                      void* stream)
{
    if (k < 1 || k > AMC_K_MAX) return AMC_E_INVALID;
    int rc = check_trace_args(op, var, n_ops, n_vars, step_status, final_status, var_first_fault, first_fault);
    if (rc) return rc;
    if (init_status && init_status == final_status) return AMC_E_INVALID;
    if (!workspace || !aligned256(workspace) || ws_bytes < kloc_workspace_bytes(n_ops)) return AMC_E_NOMEM;
    int* err = device_error_word();
    if (!err) return AMC_E_CUDA;
    KlocLaunch L;
    L.op = op;
    L.var = var;
    L.n_ops = n_ops;
    L.n_vars = n_vars;
    L.k = k;
    L.init = init_status;
    L.step = step_status;
    L.final_status = final_status;
    L.vff = var_first_fault;
    L.first_fault = first_fault;
    L.workspace = workspace;
    L.err = err;
    L.profile = 3;
    return launch_kloc(L, static_cast<cudaStream_t>(stream));
}

size_t amc_check_well_declared_workspace(int64_t n_calls)
{
    if (n_calls < 0) return 0;
    return wd_workspace_bytes();
}

int amc_check_well_declared(const int64_t* arr_loc_off, int32_t n_arrays, const int32_t* loc_owner,
                            const int64_t* call_tok_off, int64_t n_calls, const uint8_t* tok, const int32_t* payload,
                            int64_t n_tokens, const int64_t* call_am_off, const int32_t* am_array,
                            const uint8_t* am_mode, int64_t n_decls, uint32_t* violations, int64_t* first_bad,
                            int32_t* first_unmet, void* workspace, size_t ws_bytes, void* stream)
{
    if (n_arrays < 0 || n_calls < 0 || n_tokens < 0 || n_decls < 0) return AMC_E_INVALID;
    if (!arr_loc_off || !call_tok_off || !call_am_off) return AMC_E_INVALID;
    if (n_calls > 0 && (!violations || !first_bad || !first_unmet)) return AMC_E_INVALID;
    if (n_tokens > 0 && (!tok || !payload || !loc_owner)) return AMC_E_INVALID;
    if (n_decls > 0 && (!am_array || !am_mode)) return AMC_E_INVALID;
    if (!workspace || !aligned256(workspace) || ws_bytes < wd_workspace_bytes()) return AMC_E_NOMEM;
    int* err = device_error_word();
    if (!err) return AMC_E_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    WdLaunch L;
    L.arr_loc_off = arr_loc_off;
    L.n_arrays = n_arrays;
    L.loc_owner = loc_owner;
    L.call_tok_off = call_tok_off;
    L.n_calls = n_calls;
    L.tok = tok;
    L.payload = payload;
    L.n_tokens = n_tokens;
    L.call_am_off = call_am_off;
    L.am_array = am_array;
    L.am_mode = am_mode;
    L.n_decls = n_decls;
    L.violations = violations;
    L.first_bad = first_bad;
    L.first_unmet = first_unmet;
    L.workspace = workspace;
    L.err = err;
    L.profile = 3;
    return launch_well_declared(L, s);
}

}  // extern "C"
