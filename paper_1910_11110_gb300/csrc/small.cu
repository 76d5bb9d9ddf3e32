// small.cu -- the trace check of a small trace in one CTA (Section 3.2, rules
// Effect / Remote Effect of Fig. Opsem; sequencing is associative).
//
// For traces of at most SMALL_MAX_OPS ops over at most SMALL_MAX_VARS
// variables, one launch of one CTA does the whole check: its 32 warps take
// consecutive stretches of the trace; (1) each warp folds its stretch into
// one transfer function per variable (32 ops at a time, lanes with the same
// variable grouped by match.any, the group's first lane composing them in
// order), kept in shared memory; (2) a thread per variable carries the
// initial status through the warps' functions, giving every stretch its entry
// statuses and the final status; (3) each warp re-runs its stretch from those
// statuses and writes every op's status and the first faults.  No workspace,
// no memset, one kernel: the latency of a check is one launch.  The initial
// and final statuses may share a buffer: a variable's initial status is read
// and its final status written by the same thread in step (2).
#include "amc_internal.cuh"
#include "scan_trace.cuh"

namespace amc {

namespace {

constexpr int SMALL_MAX_OPS = 1 << 16;
constexpr int SMALL_MAX_VARS = 2048;
constexpr int SNW = 32;                      // warps

struct SmallSmem {
    uint8_t comp[MAX_ELEMS * MAX_ELEMS];
    uint8_t app[MAX_ELEMS * 8];
    uint8_t elem_of[256];
    uint8_t mb[SNW][32];
    uint8_t row[SNW][SMALL_MAX_VARS];        // per warp: folded functions, then current statuses
    unsigned long long ff;
};

__global__ void __launch_bounds__(SNW * 32, 1) small_trace_kernel(const uint8_t* __restrict__ kind_side,
                                                                   const int32_t* __restrict__ var, int32_t n,
                                                                   int32_t n_vars, const uint8_t* init,
                                                                   uint8_t* __restrict__ step,
                                                                   uint8_t* fin, int32_t* __restrict__ vff,
                                                                   int64_t* first_fault, int* err, const Tables tab)
{
    extern __shared__ __align__(16) uint8_t smraw[];
    SmallSmem& S = *reinterpret_cast<SmallSmem*>(smraw);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t lt = lanemask_lt();
    for (int i = tid; i < MAX_ELEMS * MAX_ELEMS; i += SNW * 32) S.comp[i] = tab.comp[i];
    for (int i = tid; i < MAX_ELEMS * 8; i += SNW * 32) S.app[i] = tab.app[i];
    for (int i = tid; i < 256; i += SNW * 32) S.elem_of[i] = tab.elem_of[i];
    const uint32_t ID = tab.identity;
    for (int v = lane; v < n_vars; v += 32) S.row[w][v] = (uint8_t)ID;
    if (tid == 0) S.ff = ~0ull;
    __syncthreads();
    const int per = (n + SNW - 1) / SNW;
    const int lo = min(n, w * per), hi = min(n, lo + per);
    // (1) fold each stretch per variable
    for (int b = lo; b < hi; b += 32) {
        const int i = b + lane;
        const bool ok = i < hi;
        const uint32_t ks = ok ? kind_side[i] : 0u;
        int32_t v = ok ? var[i] : 0;
        uint32_t m = ID;
        if (ok) {
            if (v < 0 || v >= n_vars) {
                raise_error(err, AMC_E_RANGE);
                v = 0;
            }
            m = S.elem_of[ks];
            if (m == ELEM_BAD || m == ELEM_GT) {         // GT only in a guarded check
                raise_error(err, AMC_E_INVALID);
                m = ID;
            }
        }
        S.mb[w][lane] = (uint8_t)m;
        const uint32_t peers = __match_any_sync(0xffffffffu, ok ? (uint32_t)v : 0xFFFFFFFFu);
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) {
            uint32_t acc = S.row[w][v];
            for (uint32_t q = peers; q; q &= q - 1) acc = S.comp[acc * MAX_ELEMS + S.mb[w][__ffs(q) - 1]];
            S.row[w][v] = (uint8_t)acc;
        }
        __syncwarp();
    }
    __syncthreads();
    // (2) carry: entry status of every stretch, final statuses
    for (int v = tid; v < n_vars; v += SNW * 32) {
        uint32_t s = init ? (uint32_t)(init[v] & 7u) : (uint32_t)AMC_ST_VI;
        for (int k = 0; k < SNW; ++k) {
            const uint32_t e = S.row[k][v];
            S.row[k][v] = (uint8_t)s;
            s = S.app[e * 8 + s];
        }
        fin[v] = (uint8_t)s;
        vff[v] = -1;
    }
    __syncthreads();
    // (3) statuses of every op from the stretch's entry statuses
    for (int b = lo; b < hi; b += 32) {
        const int i = b + lane;
        const bool ok = i < hi;
        const uint32_t ks = ok ? kind_side[i] : 0u;
        int32_t v = ok ? var[i] : 0;
        if (v < 0 || v >= n_vars) v = 0;
        uint32_t m = ok ? S.elem_of[ks] : ID;
        if (m == ELEM_BAD || m == ELEM_GT) m = ID;
        S.mb[w][lane] = (uint8_t)m;
        const uint32_t peers = __match_any_sync(0xffffffffu, ok ? (uint32_t)v : 0xFFFFFFFFu);
        __syncwarp();
        const uint32_t cur = ok ? S.row[w][v] : 0u;
        __syncwarp();
        if (ok) {
            uint32_t acc = ID;
            for (uint32_t q = peers & lt; q; q &= q - 1) acc = S.comp[acc * MAX_ELEMS + S.mb[w][__ffs(q) - 1]];
            const uint32_t pre = S.app[acc * 8 + cur];
            const uint32_t post = S.app[S.comp[acc * MAX_ELEMS + m] * 8 + cur];
            step[i] = (uint8_t)post;
            if (post == ST_F && pre != ST_F) {
                vff[v] = i;                              // a variable becomes stuck once
                atomicMin(&S.ff, (unsigned long long)i);
            }
            if (lane == 31 - __clz(peers)) S.row[w][v] = (uint8_t)post;
        }
        __syncwarp();
    }
    __syncthreads();
    if (tid == 0) *first_fault = S.ff == ~0ull ? -1 : (int64_t)S.ff;
}

}  // namespace

bool scan_small_eligible(const ScanLaunch& L)
{
    return L.dense != 0 && !L.n_dev && !L.gate && !L.guard && !L.pre_mode && L.n_ops <= SMALL_MAX_OPS &&
           L.n_vars >= 1 && L.n_vars <= SMALL_MAX_VARS && L.final_status != nullptr;
}

int launch_scan_small(const ScanLaunch& L, cudaStream_t s)
{
    static bool attr_done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 64 || !attr_done[dev]) {
        if (cudaFuncSetAttribute(small_trace_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(SmallSmem)) != cudaSuccess)
            return AMC_E_CUDA;
        if (dev < 64) attr_done[dev] = true;
    }
    if (L.profile & 1) profile_begin(s);
    small_trace_kernel<<<1, SNW * 32, sizeof(SmallSmem), s>>>(L.kind_side, L.var, (int32_t)L.n_ops, L.n_vars, L.init,
                                                              L.step, L.final_status, L.vff, L.first_fault, L.err,
                                                              host_tables());
    if (L.profile & 2) profile_end(s);
    return cudaGetLastError() == cudaSuccess ? AMC_OK : AMC_E_CUDA;
}

}  // namespace amc
