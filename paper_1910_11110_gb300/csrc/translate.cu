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
// With lifetimes (pvectors created and deleted during the run, Section 4.3:
// r_v is updated at creations and deletions): array a is live at the calls
// born[a] <= c < died[a]; operands must be live; O(M), the shadows and the
// projections of body writes take only the arrays live at the call; and each
// pvector created before call c (ascending id) is recorded at the head of
// call c's statements as Noop v, Noop v# (CPU side) on its vector v, the
// point where it takes v's statuses (arr_probe[a] = index of the first).
// Kernels: overlap sets r_v (sort and sweep, overlap.cu; with lifetimes only
// the pairs whose lifetimes meet), the pvectors sorted by creation call,
// per-call statement counts, device-wide exclusive scan of the counts,
// emission.
#include "amc_internal.cuh"
#include "dscan.cuh"
#include "overlap.cuh"
#include "scan_trace.cuh"
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
    const int64_t* ov_off;        // [n_arrays * nb + 1]: list (a, bucket)
    const int32_t* ov_idx;
    int32_t nb;                   // time buckets of the lists (1 without lifetimes)
    int64_t bl;                   // calls per bucket
    int32_t* call_cnt;
    int* err;
    // lifetimes (born == nullptr: every array live throughout)
    const int32_t* born;
    const int32_t* died;
    const int32_t* parent;
    const uint32_t* b_key;        // creation call of each pvector, ascending (n_calls for vectors)
    const uint32_t* b_id;         // the pvector ids in that order
    int64_t* arr_probe;
};

// overlap list of array a read at call c (its time bucket's list)
__device__ __forceinline__ int64_t list_lo(const TrParams& p, int32_t a, int64_t c)
{
    return p.ov_off[(int64_t)a * p.nb + (p.nb > 1 ? c / p.bl : 0)];
}
__device__ __forceinline__ int64_t list_hi(const TrParams& p, int32_t a, int64_t c)
{
    return p.ov_off[(int64_t)a * p.nb + (p.nb > 1 ? c / p.bl : 0) + 1];
}

// Where statement o goes: ks[o - base], var[o - base] (the output itself, or
// a warp's staging buffer in shared memory)
struct Out {
    uint8_t* ks;
    int32_t* var;
    int64_t base;
};

__device__ __forceinline__ bool live_at(const TrParams& p, int32_t a, int64_t c)
{
    return !p.born || (c >= p.born[a] && c < p.died[a]);
}

// [*lo, *hi): the pvectors created before call c
__device__ __forceinline__ void births_of(const TrParams& p, int64_t c, int32_t* lo, int32_t* hi)
{
    int32_t a = 0, b = p.n_arrays;
    while (a < b) {
        const int32_t m = (a + b) >> 1;
        if ((int64_t)p.b_key[m] < c) a = m + 1;
        else b = m;
    }
    *lo = a;
    b = p.n_arrays;
    while (a < b) {
        const int32_t m = (a + b) >> 1;
        if ((int64_t)p.b_key[m] <= c) a = m + 1;
        else b = m;
    }
    *hi = a;
}

__device__ __forceinline__ bool iv_contains(int32_t so, int32_t lo, int32_t si, int32_t li)
{
    return so <= si && (int64_t)si + li <= (int64_t)so + lo;
}

// The creation records at the head of call c: Noop v, Noop v# (CPU side)
// for every pvector created before it, ascending id.  Returns the count.
template <bool EMIT>
__device__ __forceinline__ int64_t put_births(const TrParams& p, int64_t c, int64_t o, const Out& out)
{
    int32_t lo, hi;
    births_of(p, c, &lo, &hi);
    for (int32_t k = lo; k < hi; ++k) {
        if (EMIT) {
            const int32_t y = (int32_t)p.b_id[k];
            const int32_t v = p.parent[y];
            p.arr_probe[y] = o;
            out.ks[o - out.base] = (uint8_t)AMC_K_NOOP;
            out.var[o - out.base] = v;
            out.ks[o + 1 - out.base] = (uint8_t)AMC_K_NOOP;
            out.var[o + 1 - out.base] = p.n_arrays + v;
        }
        o += 2;
    }
    return 2 * (int64_t)(hi - lo);
}

// Statements of call c.  EMIT = false only counts; EMIT = true writes them at
// out_base.  Returns the count, or -1 for a malformed call.
// One call.  NMAX >= the call's operand count; every array below is indexed
// only by unrolled loop counters (the operand that matches an array id is
// found by comparing against all slots), so for small NMAX they stay in
// registers.  The statements and their order are the same for every NMAX.
template <bool EMIT, int NMAX>
__device__ int64_t translate_call_n(const TrParams& p, const Out& out, int64_t c, int64_t out_base, const int32_t k0,
                                    const int n,
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
        if (!live_at(p, arr[i], c)) {       // not live at this call
            if (!EMIT) raise_error(p.err, AMC_E_INVALID);
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
            for (int64_t q = list_lo(p, arr[i], c); q < list_hi(p, arr[i], c); ++q) {
                const int32_t y = p.ov_idx[q];
                if (!live_at(p, y, c)) continue;
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
            out.ks[o - out.base] = (uint8_t)(kind | sb);
            out.var[o - out.base] = v;
        }
        ++o;
    };
    if (p.b_key) o += put_births<EMIT>(p, c, o, out);
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
                cur[l] = list_lo(p, arr[l], c);
                end[l] = list_hi(p, arr[l], c);
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
            if (is_arg(y) || !live_at(p, y, c)) continue;
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
        for (int64_t q = list_lo(p, x, c); q < list_hi(p, x, c); ++q) {
            const int32_t y = p.ov_idx[q];
            if (!live_at(p, y, c)) continue;
            put(iv_contains(sx, lx, p.arr_start[y], p.arr_len[y]) ? AMC_K_W : AMC_K_PW, y);
        }
    }
    return o - out_base;
}

// Calls with more than 8 operands (rare): the same statements, arrays in local memory.
template <bool EMIT>
__device__ __noinline__ int64_t translate_call_dyn(const TrParams& p, const Out& out, int64_t c, int64_t out_base)
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
        if (!live_at(p, arr[i], c)) {
            if (!EMIT) raise_error(p.err, AMC_E_INVALID);
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
            for (int64_t q = list_lo(p, arr[i], c); q < list_hi(p, arr[i], c); ++q) {
                if (!live_at(p, p.ov_idx[q], c)) continue;
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
            out.ks[o - out.base] = (uint8_t)(kind | sb);
            out.var[o - out.base] = v;
        }
        ++o;
    };
    if (p.b_key) o += put_births<EMIT>(p, c, o, out);
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
            cur[nl] = list_lo(p, arr[i], c);
            end[nl] = list_hi(p, arr[i], c);
            ++nl;
        }
        for (;;) {
            int32_t y = INT32_MAX;
            for (int l = 0; l < nl; ++l)
                if (cur[l] < end[l]) y = min(y, p.ov_idx[cur[l]]);
            if (y == INT32_MAX) break;
            for (int l = 0; l < nl; ++l)
                if (cur[l] < end[l] && p.ov_idx[cur[l]] == y) ++cur[l];
            if (find(y) >= 0 || !live_at(p, y, c)) continue;
            put(AMC_K_GT, y);
            put(AMC_K_EN, A + y);
            put(AMC_K_W, A + y);
        }
    }
    for (int i = 0; i < n; ++i) {
        if (!(mode[i] & AMC_MODE_W)) continue;           // the body writes x (declared or not)
        const int32_t x = arr[i];
        const int32_t sx = p.arr_start[x], lx = p.arr_len[x];
        for (int64_t q = list_lo(p, x, c); q < list_hi(p, x, c); ++q) {
            const int32_t y = p.ov_idx[q];
            if (!live_at(p, y, c)) continue;
            put(iv_contains(sx, lx, p.arr_start[y], p.arr_len[y]) ? AMC_K_W : AMC_K_PW, y);
        }
    }
    return o - out_base;
}

template <bool EMIT>
__device__ int64_t translate_call(const TrParams& p, const Out& out, int64_t c, int64_t out_base)
{
    const uint32_t side = p.call_side[c];
    const int32_t k0 = p.call_off[c], k1 = p.call_off[c + 1];
    if (side > 1 || k0 < 0 || k1 < k0 || (int64_t)k1 > p.n_operands || k1 - k0 > MAX_OPND) {
        if (!EMIT) raise_error(p.err, AMC_E_INVALID);
        return -1;
    }
    const int n = k1 - k0;
    if (n <= 4) return translate_call_n<EMIT, 4>(p, out, c, out_base, k0, n, side);
    if (n <= 8) return translate_call_n<EMIT, 8>(p, out, c, out_base, k0, n, side);
    return translate_call_dyn<EMIT>(p, out, c, out_base);
}

__global__ void count_kernel(const TrParams p)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p.n_calls) return;
    const int64_t k = translate_call<false>(p, Out{nullptr, nullptr, 0}, c, 0);
    p.call_cnt[c] = k < 0 ? 0 : (int32_t)k;
}

// Emission: a thread per call writes its statements in order.  (Staging a
// warp's statements in shared memory to coalesce the stores cost more in
// occupancy than it saved: 37.4 -> 42.0 ms per VectorPU step.)
__global__ void emit_kernel(const TrParams p)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= p.n_calls) return;
    if (p.call_first_op[p.n_calls] > p.out_cap) return;     // nothing but out_n is written
    translate_call<true>(p, Out{p.out_ks, p.out_var, 0}, c, p.call_first_op[c]);
}

__global__ void total_kernel(const TrParams p)
{
    const int64_t total = p.call_first_op[p.n_calls];
    *p.out_n = total;
    if (total > p.out_cap) raise_error(p.err, AMC_E_RANGE);
}

// pvector lifetimes: 0 <= born < died <= n_calls; a pvector's vector is a
// vector (parent -1) other than itself whose range and lifetime hold its own.
// Sort keys: the creation call of each pvector, n_calls for vectors.
__global__ void lifetimes_kernel(const TrParams p, uint32_t* __restrict__ key, uint32_t* __restrict__ val)
{
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= p.n_arrays) return;
    p.arr_probe[a] = -1;
    const int32_t b = p.born[a], d = p.died[a], v = p.parent[a];
    bool ok = b >= 0 && b < d && (int64_t)d <= p.n_calls;
    if (v != -1) {
        if (v < 0 || v >= p.n_arrays) {
            raise_error(p.err, AMC_E_RANGE);
            ok = true;                        // reported
        } else {
            ok = ok && v != a && p.parent[v] == -1 && p.born[v] <= b && d <= p.died[v] &&
                 iv_contains(p.arr_start[v], p.arr_len[v], p.arr_start[a], p.arr_len[a]);
        }
    }
    if (!ok) raise_error(p.err, AMC_E_INVALID);
    key[a] = (v >= 0 && v < p.n_arrays && b >= 0 && b < p.n_calls) ? (uint32_t)b : (uint32_t)p.n_calls;
    val[a] = (uint32_t)a;
}

struct TrLayout {
    size_t ov_off, ov_idx, ovws, bk0, bv0, bk1, bv1, bscr, call_cnt, scan, total;
    int64_t cap;
    int32_t nb;
};

TrLayout layout(int32_t A, int64_t n_calls, int64_t max_pairs, bool lifetimes)
{
    TrLayout L;
    size_t o = 0;
    auto take = [&](size_t b) { const size_t at = o; o += align_up(b, 256); return at; };
    // without lifetimes every array may overlap every other
    L.cap = lifetimes ? max_pairs : (int64_t)A * (A > 0 ? A - 1 : 0);
    L.nb = overlap_buckets(n_calls, lifetimes);
    L.ov_off = take(8 * ((size_t)A * L.nb + 1));
    L.ov_idx = take(4 * (size_t)(L.cap > 0 ? L.cap : 1));
    L.ovws = take(overlap_workspace_bytes(A, L.nb, L.cap));
    const size_t a4 = lifetimes ? 4 * (size_t)(A > 0 ? A : 1) : 0;
    L.bk0 = take(a4);
    L.bv0 = take(a4);
    L.bk1 = take(a4);
    L.bv1 = take(a4);
    L.bscr = take(lifetimes ? sorted_check_scratch_bytes(A > 0 ? A : 1) : 0);
    L.call_cnt = take(4 * (size_t)n_calls + 4);
    L.scan = take(dscan_workspace_bytes(n_calls > 0 ? n_calls : 1));
    L.total = o;
    return L;
}

}  // namespace

size_t translate_workspace_bytes(int32_t n_arrays, int64_t n_calls)
{
    return layout(n_arrays, n_calls, 0, false).total;
}

size_t translate_lifetimes_workspace_bytes(int32_t n_arrays, int64_t n_calls, int64_t max_pairs)
{
    return layout(n_arrays, n_calls, max_pairs, true).total;
}

size_t overlap_count_workspace_bytes(int32_t n_arrays, int64_t n_calls, bool lifetimes)
{
    const int32_t nb = overlap_buckets(n_calls, lifetimes);
    return align_up(8 * ((size_t)n_arrays * nb + 1), 256) + overlap_workspace_bytes(n_arrays, nb, 0);
}

int launch_overlap_count(const int32_t* arr_start, const int32_t* arr_len, const int32_t* arr_born,
                         const int32_t* arr_died, int32_t n_arrays, int64_t n_calls, int64_t* n_pairs, int* err,
                         void* workspace, cudaStream_t s)
{
    OverlapBuild O;
    O.arr_start = arr_start;
    O.arr_len = arr_len;
    O.arr_born = arr_born;
    O.arr_died = arr_died;
    O.n_arrays = n_arrays;
    O.n_buckets = overlap_buckets(n_calls, arr_born != nullptr);
    O.bucket_len = overlap_bucket_len(n_calls, O.n_buckets);
    O.cap = 0;
    O.ov_off = static_cast<int64_t*>(workspace);
    O.n_pairs = n_pairs;
    O.err = err;
    O.workspace = static_cast<uint8_t*>(workspace) + align_up(8 * ((size_t)n_arrays * O.n_buckets + 1), 256);
    return launch_overlaps(O, s);
}

int launch_translate(const TranslateLaunch& T, cudaStream_t s)
{
    const bool lifetimes = T.arr_born != nullptr;
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
    p.born = T.arr_born;
    p.died = T.arr_died;
    p.parent = T.arr_parent;
    p.arr_probe = T.arr_probe;
    const TrLayout L = layout(T.n_arrays, T.n_calls, T.max_pairs, lifetimes);
    uint8_t* w = static_cast<uint8_t*>(T.workspace);
    int64_t* ov_off = reinterpret_cast<int64_t*>(w + L.ov_off);
    p.ov_off = ov_off;
    p.ov_idx = reinterpret_cast<int32_t*>(w + L.ov_idx);
    p.call_cnt = reinterpret_cast<int32_t*>(w + L.call_cnt);
    void* scan_ws = w + L.scan;

    OverlapBuild O;
    O.arr_start = T.arr_start;
    O.arr_len = T.arr_len;
    O.arr_born = T.arr_born;
    O.arr_died = T.arr_died;
    O.n_arrays = T.n_arrays;
    O.n_buckets = L.nb;
    O.bucket_len = overlap_bucket_len(T.n_calls, L.nb);
    p.nb = L.nb;
    p.bl = O.bucket_len;
    O.cap = L.cap > 0 ? L.cap : 1;
    O.ov_off = ov_off;
    O.ov_idx = reinterpret_cast<uint32_t*>(w + L.ov_idx);
    O.err = T.err;
    O.workspace = w + L.ovws;
    int rc = launch_overlaps(O, s);
    if (rc) return rc;
    if (lifetimes && T.n_arrays > 0) {
        uint32_t* bk[2] = {reinterpret_cast<uint32_t*>(w + L.bk0), reinterpret_cast<uint32_t*>(w + L.bk1)};
        uint32_t* bv[2] = {reinterpret_cast<uint32_t*>(w + L.bv0), reinterpret_cast<uint32_t*>(w + L.bv1)};
        lifetimes_kernel<<<(unsigned)((T.n_arrays + 255) / 256), 256, 0, s>>>(p, bk[0], bv[0]);
        int passes = 0;
        const int64_t kr = T.n_calls + 1 < INT32_MAX ? T.n_calls + 1 : INT32_MAX;
        rc = launch_ss_radix(bk, bv, nullptr, T.n_arrays, (int32_t)kr, w + L.bscr, nullptr, s, &passes);
        if (rc) return rc;
        p.b_key = bk[passes & 1];
        p.b_id = bv[passes & 1];
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

namespace amc {

namespace {

// Initial statuses of the second check pass: a vector's are those of the
// initial store, (V,I); a pvector's real and abstract statuses are its
// vector's at its creation record (the statuses the first pass gave the two
// Noops there).
__global__ void inherit_kernel(const int32_t* __restrict__ var, int64_t n_ops, int32_t A,
                               const int32_t* __restrict__ parent, const int64_t* __restrict__ probe,
                               const uint8_t* __restrict__ step, uint8_t* __restrict__ init, int* err)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= 2 * (int64_t)A) return;
    const int32_t a = (int32_t)(v < A ? v : v - A);
    const int32_t pv = parent[a];
    uint8_t st = (uint8_t)AMC_ST_VI;
    if (pv != -1) {
        const int64_t q = probe[a];
        const bool ok = pv >= 0 && pv < A && q >= 0 && q + 1 < n_ops && var[q] == pv && var[q + 1] == A + pv;
        if (ok) st = step[q + (v < A ? 0 : 1)];
        else raise_error(err, AMC_E_INVALID);
    }
    init[v] = st;
}

}  // namespace

int launch_inherit(const int32_t* var, int64_t n_ops, int32_t n_arrays, const int32_t* arr_parent,
                   const int64_t* arr_probe, const uint8_t* step, uint8_t* init, int* err, cudaStream_t s)
{
    if (n_arrays <= 0) return AMC_OK;
    const int64_t n = 2 * (int64_t)n_arrays;
    inherit_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(var, n_ops, n_arrays, arr_parent, arr_probe, step,
                                                                init, err);
    return cudaGetLastError() == cudaSuccess ? AMC_OK : AMC_E_CUDA;
}

}  // namespace amc
