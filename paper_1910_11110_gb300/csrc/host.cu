// host.cu -- amc_check_trace_host: the trace check over host buffers, cut into
// chunks whose copies in, checks and copies out overlap.
//
// Section 3.2: the status of a variable after an op depends only on its
// status before the op, so a trace can be checked chunk by chunk, each chunk
// from the final statuses of the one before.  First faults of a later chunk
// count only where no earlier chunk faulted on that variable (a variable that
// entered the chunk as F is never reported again: F is absorbing).
//
// Pipeline (K = 3 device slots, each holding one chunk's op bytes, variable
// ids and step statuses):
//   copy-in stream   H2D chunk c into slot c % K once the check of chunk c - K
//                    has finished reading that slot
//   caller's stream  check chunk c (statuses ping-pong between two buffers),
//                    fold its first faults, once chunk c is in and the copy
//                    out of chunk c - K has drained the slot's step statuses
//   copy-out stream  D2H chunk c's step statuses once its check is done
// The caller's stream finally waits for the copy-out stream, so that a
// synchronise on it covers every output.
#include <map>
#include <mutex>

#include "amc_internal.cuh"
#include "scan_trace.cuh"
#include "autotune.cuh"

using namespace amc;

namespace {

constexpr int SLOTS = 3;
constexpr int64_t DEFAULT_CHUNK = (int64_t)1 << 25;
constexpr int64_t CHUNK_ROUND = 4096;

int64_t chunk_of(int64_t n_ops, int64_t chunk_ops)
{
    int64_t c = chunk_ops > 0 ? chunk_ops : DEFAULT_CHUNK;
    c = (c + CHUNK_ROUND - 1) / CHUNK_ROUND * CHUNK_ROUND;
    const int64_t whole = (n_ops + CHUNK_ROUND - 1) / CHUNK_ROUND * CHUNK_ROUND;
    if (c > whole) c = whole;
    return c > 0 ? c : CHUNK_ROUND;
}

size_t slot_bytes(int64_t chunk) { return align_up((size_t)chunk, 256) * 2 + align_up(4 * (size_t)chunk, 256); }

// statuses x2, first faults running and per chunk
size_t state_bytes(int32_t n_vars) { return 2 * align_up((size_t)n_vars, 256) + 2 * align_up(4 * (size_t)n_vars, 256) + 512; }

// Copy streams and slot events of one device, made on first use and kept.
struct HostPipe {
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t fork = nullptr, done = nullptr;
    cudaEvent_t in[SLOTS] = {}, checked[SLOTS] = {}, out[SLOTS] = {};
};

std::mutex& pipe_mutex()
{
    static std::mutex* m = new std::mutex();
    return *m;
}

// Call with pipe_mutex held.
HostPipe* pipe_for_current_device()
{
    static std::map<int, HostPipe*>* pipes = new std::map<int, HostPipe*>();   // kept until exit
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    auto it = pipes->find(dev);
    if (it != pipes->end()) return it->second;
    HostPipe* P = new HostPipe();
    bool ok = cudaStreamCreateWithFlags(&P->h2d, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&P->d2h, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&P->done, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; ok && i < SLOTS; ++i)
        ok = cudaEventCreateWithFlags(&P->in[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&P->checked[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&P->out[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) return nullptr;     // the partial objects stay alive; the call reports AMC_E_CUDA
    (*pipes)[dev] = P;
    return P;
}

inline bool ok(cudaError_t e) { return e == cudaSuccess; }

}  // namespace

extern "C" {

size_t amc_check_trace_host_workspace(int64_t n_ops, int32_t n_vars, int64_t chunk_ops)
{
    if (n_ops < 0 || n_vars < 0) return 0;
    const int64_t chunk = chunk_of(n_ops, chunk_ops);
    return SLOTS * slot_bytes(chunk) + state_bytes(n_vars) + scan_workspace_bytes(chunk, n_vars);
}

int amc_check_trace_host(const uint8_t* kind_side, const int32_t* var, int64_t n_ops, int32_t n_vars,
                         const uint8_t* init_status, uint8_t* step_status, uint8_t* final_status,
                         int32_t* var_first_fault, int64_t* first_fault, int64_t chunk_ops, void* workspace,
                         size_t ws_bytes, void* stream)
{
    if (n_ops < 0 || n_ops > INT32_MAX || n_vars < 0) return AMC_E_INVALID;
    if (n_ops > 0 && (n_vars < 1 || !kind_side || !var || !step_status)) return AMC_E_INVALID;
    if (n_vars > 0 && (!final_status || !var_first_fault)) return AMC_E_INVALID;
    if (!first_fault) return AMC_E_INVALID;
    if (!workspace || ((uintptr_t)workspace & 255) ||
        ws_bytes < amc_check_trace_host_workspace(n_ops, n_vars, chunk_ops))
        return AMC_E_NOMEM;
    int* err = device_error_word();
    if (!err) return AMC_E_CUDA;
    const int64_t chunk = chunk_of(n_ops, chunk_ops);
    const int64_t n_chunks = n_ops > 0 ? (n_ops + chunk - 1) / chunk : 1;

    // workspace: K slots, statuses x2, first faults (running, chunk), scan scratch
    uint8_t* w = static_cast<uint8_t*>(workspace);
    uint8_t* slot_ks[SLOTS];
    int32_t* slot_var[SLOTS];
    uint8_t* slot_step[SLOTS];
    for (int i = 0; i < SLOTS; ++i) {
        slot_ks[i] = w;
        w += align_up((size_t)chunk, 256);
        slot_var[i] = reinterpret_cast<int32_t*>(w);
        w += align_up(4 * (size_t)chunk, 256);
        slot_step[i] = w;
        w += align_up((size_t)chunk, 256);
    }
    uint8_t* st[2];
    st[0] = w;
    w += align_up((size_t)n_vars, 256);
    st[1] = w;
    w += align_up((size_t)n_vars, 256);
    int32_t* vff_run = reinterpret_cast<int32_t*>(w);
    w += align_up(4 * (size_t)n_vars, 256);
    int32_t* vff_part = reinterpret_cast<int32_t*>(w);
    w += align_up(4 * (size_t)n_vars, 256);
    int64_t* ff_run = reinterpret_cast<int64_t*>(w);
    int64_t* ff_part = reinterpret_cast<int64_t*>(w + 256);
    w += 512;
    void* scan_ws = w;

    // launch shape: the choice tuned for plain traces of the chunk's shape, if any
    static const int fb[4] = {-2, 1 << 20, -1, -2};
    static const int grp[4] = {16, 16, 16, 1};
    const int pick = autotune_lookup(shape_key("trace", chunk, n_vars, 0));

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lock(pipe_mutex());
    HostPipe* P = pipe_for_current_device();
    if (!P) return AMC_E_CUDA;
    // the copy streams start after the work already on the caller's stream
    if (!ok(cudaEventRecord(P->fork, s)) || !ok(cudaStreamWaitEvent(P->h2d, P->fork, 0)) ||
        !ok(cudaStreamWaitEvent(P->d2h, P->fork, 0)))
        return AMC_E_CUDA;
    if (init_status && n_vars > 0 &&
        !ok(cudaMemcpyAsync(st[0], init_status, (size_t)n_vars, cudaMemcpyHostToDevice, P->h2d)))
        return AMC_E_CUDA;

    for (int64_t c = 0; c < n_chunks; ++c) {
        const int k = (int)(c % SLOTS);
        const int64_t off = c * chunk;
        const int64_t n = n_ops - off < chunk ? n_ops - off : chunk;
        // copy in, after the check of chunk c - K has read the slot
        if (c >= SLOTS && !ok(cudaStreamWaitEvent(P->h2d, P->checked[k], 0))) return AMC_E_CUDA;
        if (n > 0) {
            if (!ok(cudaMemcpyAsync(slot_ks[k], kind_side + off, (size_t)n, cudaMemcpyHostToDevice, P->h2d)) ||
                !ok(cudaMemcpyAsync(slot_var[k], var + off, 4 * (size_t)n, cudaMemcpyHostToDevice, P->h2d)))
                return AMC_E_CUDA;
        }
        if (!ok(cudaEventRecord(P->in[k], P->h2d))) return AMC_E_CUDA;
        // check, once the chunk is in and the slot's earlier step statuses are out
        if (!ok(cudaStreamWaitEvent(s, P->in[k], 0))) return AMC_E_CUDA;
        if (c >= SLOTS && !ok(cudaStreamWaitEvent(s, P->out[k], 0))) return AMC_E_CUDA;
        ScanLaunch L;
        L.kind_side = slot_ks[k];
        L.var = slot_var[k];
        L.n_ops = n;
        L.n_vars = n_vars;
        L.init = c == 0 ? (init_status ? st[0] : nullptr) : st[c & 1];
        L.step = slot_step[k];
        L.final_status = st[(c + 1) & 1];
        L.vff = c == 0 ? vff_run : vff_part;
        L.first_fault = c == 0 ? ff_run : ff_part;
        L.err = err;
        L.workspace = scan_ws;
        L.profile = 0;
        L.fb_max_bits = fb[pick >= 0 && pick < 4 ? pick : 0];
        L.group_max = grp[pick >= 0 && pick < 4 ? pick : 0];
        int rc = launch_scan_trace(L, s);
        if (rc) return rc;
        if (c > 0 && (rc = launch_merge_faults(vff_run, vff_part, n_vars, ff_run, ff_part, off, s))) return rc;
        if (!ok(cudaEventRecord(P->checked[k], s))) return AMC_E_CUDA;
        // copy out
        if (!ok(cudaStreamWaitEvent(P->d2h, P->checked[k], 0))) return AMC_E_CUDA;
        if (n > 0 && !ok(cudaMemcpyAsync(step_status + off, slot_step[k], (size_t)n, cudaMemcpyDeviceToHost, P->d2h)))
            return AMC_E_CUDA;
        if (!ok(cudaEventRecord(P->out[k], P->d2h))) return AMC_E_CUDA;
    }
    // the last check's final statuses and the folded first faults
    uint8_t* fin = st[n_chunks & 1];
    if (n_vars > 0 &&
        (!ok(cudaMemcpyAsync(final_status, fin, (size_t)n_vars, cudaMemcpyDeviceToHost, P->d2h)) ||
         !ok(cudaMemcpyAsync(var_first_fault, vff_run, 4 * (size_t)n_vars, cudaMemcpyDeviceToHost, P->d2h))))
        return AMC_E_CUDA;
    if (!ok(cudaMemcpyAsync(first_fault, ff_run, 8, cudaMemcpyDeviceToHost, P->d2h))) return AMC_E_CUDA;
    if (!ok(cudaEventRecord(P->done, P->d2h)) || !ok(cudaStreamWaitEvent(s, P->done, 0))) return AMC_E_CUDA;
    return AMC_OK;
}

}  // extern "C"
