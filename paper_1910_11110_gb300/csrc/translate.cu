// translate.cu -- VectorPU component calls -> core trace (sm_103a).
//
// Arrays are half-open intervals of one index space; each has a real status
// (id a) and an abstract status (id A + a), one validity pair per array
// (Section 3.5).  Per call:
//   - O(M), Table Overlap-ext-tab: a declared W or RW operand x upgrades an
//     overlapping declared R operand to RW, an overlapping declared W operand
//     only when x is RW, and adds a shadow RW(y) for every overlapping array
//     that is not an argument of the call (Section 4.3; the rules read the
//     declared set only, they are not applied again to what they add).  A
//     dropped annotation is not declared: it takes part in no rule.
//   - translation of each declaration (Fig. sem-AM): R / RW -> GT x, EN x#
//     (the guarded transfers on the real and abstract variable), W / RW ->
//     w x#; then the body accesses of the operand's own mode;
//   - shadows RW(y) in ascending order: GT y, EN y#, w y#;
//   - every body write of x also writes the shared elements of each array y
//     overlapping x: w y when y lies inside x, otherwise pw y.
// Kernels: overlap sets r_v (count / fill, one warp per array), per-call
// statement counts, device-wide exclusive scan of the counts, emission.
#include "amc_internal.cuh"
#include "dscan.cuh"
#include "translate.cuh"

namespace amc {

namespace {

constexpr int MAX_OPND = 32;

struct TrParams {
    const int32_t* arr_start;
    const int32_t* arr_len;
    int32_t n_arrays;
    const uint8_t* call_side;
    const int32_t* call_off;
    int64_t n_calls;
    const int32_t* opnd_array;
    const uint8_t* opnd_mode;
    int64_t n_operands;
    int infer;
    uint8_t* out_ks;
    int32_t* out_var;
    int64_t out_cap;
    int64_t* out_n;
    int64_t* call_first_op;
    const int64_t* ov_off;
    int32_t* ov_idx;
    int32_t* ov_cnt;
    int32_t* call_cnt;
    int* err;
};

__device__ __forceinline__ bool iv_overlap(int32_t s1, int32_t l1, int32_t s2, int32_t l2)
{
    return (int64_t)s1 < (int64_t)s2 + l2 && (int64_t)s2 < (int64_t)s1 + l1;
}
__device__ __forceinline__ bool iv_contains(int32_t so, int32_t lo, int32_t si, int32_t li)
{
    return so <= si && (int64_t)si + li <= (int64_t)so + lo;
}

// One warp per array: count (FILL = false) or list (FILL = true) the arrays
// overlapping it, in ascending id order.
template <bool FILL>
__global__ void overlap_kernel(const TrParams p)
{
    const int64_t a = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (a >= p.n_arrays) return;
    const int32_t sa = p.arr_start[a], la = p.arr_len[a];
    if (!FILL && lane == 0 && (sa < 0 || la < 1 || (int64_t)sa + la > INT32_MAX)) raise_error(p.err, AMC_E_INVALID);
    int64_t run = FILL ? p.ov_off[a] : 0;
    const uint32_t lt = lanemask_lt();
    for (int32_t b0 = 0; b0 < p.n_arrays; b0 += 32) {
        const int32_t b = b0 + lane;
        const bool ov = b < p.n_arrays && b != a && iv_overlap(sa, la, p.arr_start[b], p.arr_len[b]);
        const uint32_t m = __ballot_sync(0xffffffffu, ov);
        if (FILL && ov) p.ov_idx[run + __popc(m & lt)] = b;
        run += __popc(m);
    }
    if (!FILL && lane == 0) p.ov_cnt[a] = (int32_t)run;
}

// Statements of call c.  EMIT = false only counts; EMIT = true writes them at
// out_base.  Returns the count, or -1 for a malformed call.
// One call.  NMAX >= the call's operand count; every array below is indexed
// only by unrolled loop counters (the operand that matches an array id is
// found by comparing against all slots), so for small NMAX they stay in
// registers.  The statements and their order are the same for every NMAX.
template <bool EMIT, int NMAX>
__device__ int64_t translate_call_n(const TrParams& p, int64_t c, int64_t out_base, const int32_t k0, const int n,
                                    const uint32_t side)
{
    const int32_t A = p.n_arrays;
    int32_t arr[NMAX];
    uint8_t mode[NMAX], eff[NMAX];
#pragma unroll
    for (int i = 0; i < NMAX; ++i) {
        arr[i] = -1;
        mode[i] = eff[i] = 0;
        if (i < n) {
            arr[i] = p.opnd_array[k0 + i];
            mode[i] = p.opnd_mode[k0 + i];
        }
    }
#pragma unroll
    for (int i = 0; i < NMAX; ++i) {
        if (i >= n) break;
        if ((mode[i] & 0x7C) || (mode[i] & 3) == 0) {
            if (!EMIT) raise_error(p.err, AMC_E_INVALID);
            return -1;
        }
        if (arr[i] < 0 || arr[i] >= A) {
            if (!EMIT) raise_error(p.err, AMC_E_RANGE);
            return -1;
        }
        bool dup = false;
#pragma unroll
        for (int j = 0; j < NMAX; ++j) dup |= j < i && arr[j] == arr[i];
        if (dup) {                          // one declaration per variable (Section 3.3)
            if (!EMIT) raise_error(p.err, AMC_E_INVALID);
            return -1;
        }
        eff[i] = (mode[i] & AMC_MODE_DROPPED) ? 0 : (mode[i] & 3);
    }
    auto is_arg = [&](int32_t y) {
        bool f = false;
#pragma unroll
        for (int j = 0; j < NMAX; ++j) f |= j < n && arr[j] == y;
        return f;
    };
    if (p.infer) {
#pragma unroll
        for (int i = 0; i < NMAX; ++i) {
            if (i >= n) break;
            if ((mode[i] & AMC_MODE_DROPPED) || !(mode[i] & AMC_MODE_W)) continue;
            const bool x_rw = (mode[i] & 3) == AMC_MODE_RW;
            for (int64_t q = p.ov_off[arr[i]]; q < p.ov_off[arr[i] + 1]; ++q) {
                const int32_t y = p.ov_idx[q];
#pragma unroll
                for (int j = 0; j < NMAX; ++j)
                    if (j < n && arr[j] == y && !(mode[j] & AMC_MODE_DROPPED) && (x_rw || (mode[j] & 3) != AMC_MODE_W))
                        eff[j] = AMC_MODE_RW;
            }
        }
    }
    int64_t o = out_base;
    const uint8_t sb = (uint8_t)(side << 4);
    auto put = [&](uint32_t kind, int32_t v) {
        if (EMIT) {
            p.out_ks[o] = (uint8_t)(kind | sb);
            p.out_var[o] = v;
        }
        ++o;
    };
#pragma unroll
    for (int i = 0; i < NMAX; ++i) {
        if (i >= n) break;
        const int32_t x = arr[i];
        const int me = eff[i], mo = mode[i] & 3;
        if (me == AMC_MODE_R || me == AMC_MODE_RW) {
            put(AMC_K_GT, x);
            put(AMC_K_EN, A + x);
        }
        if (me == AMC_MODE_W || me == AMC_MODE_RW) put(AMC_K_W, A + x);
        if (mo == AMC_MODE_R || mo == AMC_MODE_RW) put(AMC_K_R, x);
        if (mo == AMC_MODE_W || mo == AMC_MODE_RW) put(AMC_K_W, x);
    }
    if (p.infer) {
        // shadows: union of the overlap lists of declared written operands,
        // minus the call's arguments, ascending (merge of sorted lists)
        int64_t cur[NMAX], end[NMAX];
#pragma unroll
        for (int l = 0; l < NMAX; ++l) {
            cur[l] = end[l] = 0;
            if (l < n && !(mode[l] & AMC_MODE_DROPPED) && (mode[l] & AMC_MODE_W)) {
                cur[l] = p.ov_off[arr[l]];
                end[l] = p.ov_off[arr[l] + 1];
            }
        }
        for (;;) {
            int32_t y = INT32_MAX;
#pragma unroll
            for (int l = 0; l < NMAX; ++l)
                if (cur[l] < end[l]) y = min(y, p.ov_idx[cur[l]]);
            if (y == INT32_MAX) break;
#pragma unroll
            for (int l = 0; l < NMAX; ++l)
                if (cur[l] < end[l] && p.ov_idx[cur[l]] == y) ++cur[l];
            if (is_arg(y)) continue;
            put(AMC_K_GT, y);
            put(AMC_K_EN, A + y);
            put(AMC_K_W, A + y);
        }
    }
#pragma unroll
    for (int i = 0; i < NMAX; ++i) {
        if (i >= n) break;
        if (!(mode[i] & AMC_MODE_W)) continue;           // the body writes x (declared or not)
        const int32_t x = arr[i];
        const int32_t sx = p.arr_start[x], lx = p.arr_len[x];
        for (int64_t q = p.ov_off[x]; q < p.ov_off[x + 1]; ++q) {
            const int32_t y = p.ov_idx[q];
            put(iv_contains(sx, lx, p.arr_start[y], p.arr_len[y]) ? AMC_K_W : AMC_K_PW, y);
        }
    }
    return o - out_base;
}

// Calls with more than 8 operands (rare): the same statements, arrays in local memory.
template <bool EMIT>
__device__ __noinline__ int64_t translate_call_dyn(const TrParams& p, int64_t c, int64_t out_base)
{
    const uint32_t side = p.call_side[c];
    const int32_t k0 = p.call_off[c], k1 = p.call_off[c + 1];
    const int32_t A = p.n_arrays;
    if (side > 1 || k0 < 0 || k1 < k0 || (int64_t)k1 > p.n_operands || k1 - k0 > MAX_OPND) {
        if (!EMIT) raise_error(p.err, AMC_E_INVALID);
        return -1;
    }
    const int n = k1 - k0;
    int32_t arr[MAX_OPND];
    uint8_t mode[MAX_OPND], eff[MAX_OPND];
    for (int i = 0; i < n; ++i) {
        arr[i] = p.opnd_array[k0 + i];
        mode[i] = p.opnd_mode[k0 + i];
        if ((mode[i] & 0x7C) || (mode[i] & 3) == 0) {
            if (!EMIT) raise_error(p.err, AMC_E_INVALID);
            return -1;
        }
        if (arr[i] < 0 || arr[i] >= A) {
            if (!EMIT) raise_error(p.err, AMC_E_RANGE);
            return -1;
        }
        for (int j = 0; j < i; ++j)
            if (arr[j] == arr[i]) {       // one declaration per variable (Section 3.3)
                if (!EMIT) raise_error(p.err, AMC_E_INVALID);
                return -1;
            }
        eff[i] = (mode[i] & AMC_MODE_DROPPED) ? 0 : (mode[i] & 3);
    }
    auto find = [&](int32_t y) -> int {
        for (int j = 0; j < n; ++j)
            if (arr[j] == y) return j;
        return -1;
    };
    if (p.infer) {
        for (int i = 0; i < n; ++i) {
            if ((mode[i] & AMC_MODE_DROPPED) || !(mode[i] & AMC_MODE_W)) continue;
            for (int64_t q = p.ov_off[arr[i]]; q < p.ov_off[arr[i] + 1]; ++q) {
                const int j = find(p.ov_idx[q]);
                if (j < 0 || (mode[j] & AMC_MODE_DROPPED)) continue;
                if ((mode[i] & 3) == AMC_MODE_RW || (mode[j] & 3) != AMC_MODE_W) eff[j] = AMC_MODE_RW;
            }
        }
    }
    int64_t o = out_base;
    const uint8_t sb = (uint8_t)(side << 4);
    auto put = [&](uint32_t kind, int32_t v) {
        if (EMIT) {
            p.out_ks[o] = (uint8_t)(kind | sb);
            p.out_var[o] = v;
        }
        ++o;
    };
    for (int i = 0; i < n; ++i) {
        const int32_t x = arr[i];
        const int me = eff[i], mo = mode[i] & 3;
        if (me == AMC_MODE_R || me == AMC_MODE_RW) {
            put(AMC_K_GT, x);
            put(AMC_K_EN, A + x);
        }
        if (me == AMC_MODE_W || me == AMC_MODE_RW) put(AMC_K_W, A + x);
        if (mo == AMC_MODE_R || mo == AMC_MODE_RW) put(AMC_K_R, x);
        if (mo == AMC_MODE_W || mo == AMC_MODE_RW) put(AMC_K_W, x);
    }
    if (p.infer) {
        // shadows: union of the overlap lists of declared written operands,
        // minus the call's arguments, ascending (merge of sorted lists)
        int64_t cur[MAX_OPND], end[MAX_OPND];
        int nl = 0;
        for (int i = 0; i < n; ++i) {
            if ((mode[i] & AMC_MODE_DROPPED) || !(mode[i] & AMC_MODE_W)) continue;
            cur[nl] = p.ov_off[arr[i]];
            end[nl] = p.ov_off[arr[i] + 1];
            ++nl;
        }
        for (;;) {
            int32_t y = INT32_MAX;
            for (int l = 0; l < nl; ++l)
                if (cur[l] < end[l]) y = min(y, p.ov_idx[cur[l]]);
            if (y == INT32_MAX) break;
            for (int l = 0; l < nl; ++l)
                if (cur[l] < end[l] && p.ov_idx[cur[l]] == y) ++cur[l];
            if (find(y) >= 0) continue;
            put(AMC_K_GT, y);
            put(AMC_K_EN, A + y);
            put(AMC_K_W, A + y);
        }
    }
    for (int i = 0; i < n; ++i) {
        if (!(mode[i] & AMC_MODE_W)) continue;           // the body writes x (declared or not)
        const int32_t x = arr[i];
        const int32_t sx = p.arr_start[x], lx = p.arr_len[x];
        for (int64_t q = p.ov_off[x]; q < p.ov_off[x + 1]; ++q) {
            const int32_t y = p.ov_idx[q];
            put(iv_contains(sx, lx, p.arr_start[y], p.arr_len[y]) ? AMC_K_W : AMC_K_PW, y);
        }
    }
    return o - out_base;
}

template <bool EMIT>
__device__ int64_t translate_call(const TrParams& p, int64_t c, int64_t out_base)
{
    const uint32_t side = p.call_side[c];
    const int32_t k0 = p.call_off[c], k1 = p.call_off[c + 1];
    if (side > 1 || k0 < 0 || k1 < k0 || (int64_t)k1 > p.n_operands || k1 - k0 > MAX_OPND) {
        if (!EMIT) raise_error(p.err, AMC_E_INVALID);
        return -1;
    }
    const int n = k1 - k0;
    if (n <= 4) return translate_call_n<EMIT, 4>(p, c, out_base, k0, n, side);
    if (n <= 8) return translate_call_n<EMIT, 8>(p, c, out_base, k0, n, side);
    return translate_call_dyn<EMIT>(p, c, out_base);
}

__global__ void count_kernel(const TrParams p)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p.n_calls) return;
    const int64_t k = translate_call<false>(p, c, 0);
    p.call_cnt[c] = k < 0 ? 0 : (int32_t)k;
}

__global__ void emit_kernel(const TrParams p)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p.n_calls) return;
    if (p.call_first_op[p.n_calls] > p.out_cap) return;     // nothing but out_n is written
    translate_call<true>(p, c, p.call_first_op[c]);
}

__global__ void total_kernel(const TrParams p)
{
    const int64_t total = p.call_first_op[p.n_calls];
    *p.out_n = total;
    if (total > p.out_cap) raise_error(p.err, AMC_E_RANGE);
}

struct TrLayout {
    size_t ov_cnt, ov_off, ov_idx, call_cnt, scan, total;
};

TrLayout layout(int32_t A, int64_t n_calls)
{
    TrLayout L;
    size_t o = 0;
    L.ov_cnt = o;
    o += align_up(4 * (size_t)A, 256);
    L.ov_off = o;
    o += align_up(8 * ((size_t)A + 1), 256);
    L.ov_idx = o;
    o += align_up(4 * (size_t)A * (size_t)(A > 0 ? A - 1 : 0) + 4, 256);
    L.call_cnt = o;
    o += align_up(4 * (size_t)n_calls + 4, 256);
    L.scan = o;
    o += dscan_workspace_bytes(n_calls > A ? n_calls : A);
    L.total = o;
    return L;
}

}  // namespace

size_t translate_workspace_bytes(int32_t n_arrays, int64_t n_calls)
{
    return layout(n_arrays, n_calls).total;
}

int launch_translate(const TranslateLaunch& T, cudaStream_t s)
{
    TrParams p{};
    p.arr_start = T.arr_start;
    p.arr_len = T.arr_len;
    p.n_arrays = T.n_arrays;
    p.call_side = T.call_side;
    p.call_off = T.call_off;
    p.n_calls = T.n_calls;
    p.opnd_array = T.opnd_array;
    p.opnd_mode = T.opnd_mode;
    p.n_operands = T.n_operands;
    p.infer = T.infer;
    p.out_ks = T.out_ks;
    p.out_var = T.out_var;
    p.out_cap = T.out_cap;
    p.out_n = T.out_n;
    p.call_first_op = T.call_first_op;
    p.err = T.err;
    const TrLayout L = layout(T.n_arrays, T.n_calls);
    uint8_t* w = static_cast<uint8_t*>(T.workspace);
    p.ov_cnt = reinterpret_cast<int32_t*>(w + L.ov_cnt);
    int64_t* ov_off = reinterpret_cast<int64_t*>(w + L.ov_off);
    p.ov_off = ov_off;
    p.ov_idx = reinterpret_cast<int32_t*>(w + L.ov_idx);
    p.call_cnt = reinterpret_cast<int32_t*>(w + L.call_cnt);
    void* scan_ws = w + L.scan;

    if (T.n_arrays > 0) {
        const int64_t threads = (int64_t)T.n_arrays * 32;
        const unsigned blocks = (unsigned)((threads + 255) / 256);
        overlap_kernel<false><<<blocks, 256, 0, s>>>(p);
        int rc = dscan_exclusive(p.ov_cnt, ov_off, T.n_arrays, scan_ws, s);
        if (rc) return rc;
        overlap_kernel<true><<<blocks, 256, 0, s>>>(p);
    } else if (cudaMemsetAsync(ov_off, 0, 8, s) != cudaSuccess) {
        return AMC_E_CUDA;
    }
    if (T.n_calls > 0) {
        const unsigned blocks = (unsigned)((T.n_calls + 255) / 256);
        count_kernel<<<blocks, 256, 0, s>>>(p);
        int rc = dscan_exclusive(p.call_cnt, T.call_first_op, T.n_calls, scan_ws, s);
        if (rc) return rc;
        if (T.profile & 1) profile_begin(s);
        emit_kernel<<<blocks, 256, 0, s>>>(p);
        if (T.profile & 2) profile_end(s);
    } else if (cudaMemsetAsync(T.call_first_op, 0, 8, s) != cudaSuccess) {
        return AMC_E_CUDA;
    }
    total_kernel<<<1, 1, 0, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? AMC_OK : AMC_E_CUDA;
}

}  // namespace amc
