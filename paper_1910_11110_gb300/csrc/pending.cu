// pending.cu -- entry points whose kernels are not in this build yet; they
// reject every call with AMC_E_INVALID.
#include "amc_internal.cuh"

extern "C" {
size_t amc_check_batch_workspace(int64_t, int64_t, int64_t) { return 0; }
int amc_check_batch(const uint8_t*, const int32_t*, const int64_t*, const int32_t*, const int64_t*, int64_t,
                    int64_t, uint8_t*, uint8_t*, int64_t*, int, void*, size_t, void*) { return AMC_E_INVALID; }
int amc_server_create(size_t, int, amc_server**) { return AMC_E_INVALID; }
int amc_serve_submit(amc_server*, uint64_t, const amc_request*, uint64_t*) { return AMC_E_INVALID; }
int amc_serve_poll(amc_server*, uint64_t, int*, amc_result*) { return AMC_E_INVALID; }
int amc_serve_release(amc_server*, uint64_t) { return AMC_E_INVALID; }
int amc_session_export(amc_server*, uint64_t, uint8_t*, int32_t) { return AMC_E_INVALID; }
int amc_server_destroy(amc_server*) { return AMC_E_INVALID; }
}
