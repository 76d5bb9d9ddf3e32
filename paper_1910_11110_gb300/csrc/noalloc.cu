// noalloc.cu -- amc_check_trace_noalloc: the trace check with its scratch in a
// fixed device array that belongs to this library, for callers that cannot
// allocate device memory.
//
// The scratch is one file-scope __device__ array: every GPU that loads the
// library holds it (AMC_NOALLOC_SCRATCH_BYTES) until the process exits.  Its
// device address is looked up once per device, with that device current, on
// the first call made on it; later calls reuse the cached address.  Calls
// share the array, so two calls whose work overlaps on the GPU race on it;
// every call clears what must start at zero before its kernels run.
#include <map>
#include <mutex>

#include "amc_internal.cuh"
#include "scan_trace.cuh"

static __device__ __align__(256) uint8_t noalloc_scratch[AMC_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of noalloc_scratch on the current device (nullptr if the
// lookup fails).  In host code the array's name is only a host-side stand-in,
// so kernels must be handed this address instead.
void* scratch_on_current_device()
{
    static std::mutex mu;
    static std::map<int, void*> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, noalloc_scratch) != cudaSuccess || !ptr) return nullptr;
    cache[dev] = ptr;
    return ptr;
}

}  // namespace

extern "C" int amc_check_trace_noalloc(const uint8_t* kind_side, const int32_t* var, int64_t n_ops,
                                       int32_t n_vars, const uint8_t* init_status, uint8_t* step_status,
                                       uint8_t* final_status, int32_t* var_first_fault, int64_t* first_fault,
                                       void* stream)
{
    if (n_ops < 0 || n_vars < 0) return AMC_E_INVALID;
    if (n_ops > AMC_NOALLOC_MAX_OPS || n_vars > AMC_NOALLOC_MAX_VARS) return AMC_E_RANGE;
    // the single-pass path only: its scratch fits the array at the maximum sizes
    if (amc::scan_workspace_bytes(n_ops, n_vars, false) > (size_t)AMC_NOALLOC_SCRATCH_BYTES) return AMC_E_RANGE;
    if (n_ops > 0 && (n_vars < 1 || !kind_side || !var || !step_status)) return AMC_E_INVALID;
    if (n_vars > 0 && (!final_status || !var_first_fault)) return AMC_E_INVALID;
    if (!first_fault) return AMC_E_INVALID;
    void* scratch = scratch_on_current_device();
    int* err = amc::device_error_word();
    if (!scratch || !err) return AMC_E_CUDA;
    amc::ScanLaunch L;
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
    L.workspace = scratch;
    L.dense = 0;
    return amc::launch_scan_trace(L, static_cast<cudaStream_t>(stream));
}
