// overlap.cu -- the overlap sets r_v of Section 4.3 as lists (sm_103a).
//
// For every array a, the ids of the other arrays whose index ranges overlap
// a's range and, when lifetimes are given, whose lifetimes meet a's
// (max(born) < min(died)), ascending.  With lifetimes the lists are kept per
// time bucket (n_buckets stretches of bucket_len calls): list (a, b) holds
// the overlapping arrays whose lifetime meets a's within bucket b, so that a
// call at c reads list (a, c / bucket_len) -- about the arrays live near c,
// not every array that ever overlaps a -- and keeps the entries live at c:
// r_v as the paper queries it at that call.  Sort and sweep, O(A log A + P)
// for P listed entries:
//   1. the arrays sorted by range start (stable LSD radix sort, ids as values);
//   2. a warp per sorted position p: the arrays after p whose start lies below
//      p's end overlap it (they start no earlier and have at least one
//      element), found by a binary search for that end; every overlapping
//      pair is seen once, from its earlier position; the warp counts, for
//      both ends, one entry per bucket the two lifetimes share (atomics);
//   3. exclusive scan of the counts: list offsets and the total, checked
//      against the capacity (over it: AMC_E_RANGE, and every list is left
//      empty);
//   4. the same sweep writes each entry into its list (atomic cursors, any
//      order) as (other, owner list) pairs;
//   5. a stable sort of the pairs by other, then by owner list: each list in
//      ascending order.
#include "amc_internal.cuh"
#include "dscan.cuh"
#include "overlap.cuh"
#include "scan_trace.cuh"

namespace amc {

namespace {

struct OvParams {
    const int32_t* start;
    const int32_t* len;
    const int32_t* born;          // nullable: every pair meets
    const int32_t* died;
    int32_t A;
    int32_t nb;                   // time buckets (1 without lifetimes)
    int64_t bl;                   // calls per bucket
    const uint32_t* skey;         // range starts, sorted
    const uint32_t* sval;         // their ids
    int32_t* cnt;                 // [A * nb] list lengths, then fill cursors
    const int64_t* off;           // [A * nb + 1]
    int64_t cap;
    uint32_t* pkey;               // [cap] other
    uint32_t* pval;               // [cap] owner list (owner * nb + bucket)
    int* err;
};

__global__ void ov_keys_kernel(const int32_t* __restrict__ start, const int32_t* __restrict__ len, int32_t A,
                               uint32_t* __restrict__ key, uint32_t* __restrict__ val, int* err)
{
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A) return;
    const int32_t s = start[a], l = len[a];
    if (s < 0 || l < 1 || (int64_t)s + l > INT32_MAX) raise_error(err, AMC_E_INVALID);
    key[a] = s < 0 ? 0u : (uint32_t)s;
    val[a] = (uint32_t)a;
}

// first position in (lo, A) whose start is >= e (A if none)
__device__ __forceinline__ int32_t upper_pos(const uint32_t* skey, int32_t lo, int32_t A, int64_t e)
{
    int32_t a = lo + 1, b = A;
    while (a < b) {
        const int32_t m = (a + b) >> 1;
        if ((int64_t)skey[m] < e) a = m + 1;
        else b = m;
    }
    return a;
}

template <bool FILL>
__global__ void ov_sweep_kernel(const OvParams p)
{
    const int64_t pos = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (pos >= p.A) return;
    if (FILL && p.off[p.A] > p.cap) return;                  // over capacity: reported by the count pass
    const int32_t i = (int32_t)p.sval[pos];
    const int64_t e = (int64_t)p.start[i] + p.len[i];
    const int32_t ub = upper_pos(p.skey, (int32_t)pos, p.A, e);
    const int32_t bi = p.born ? p.born[i] : 0, di = p.born ? p.died[i] : 1;
    for (int32_t q = (int32_t)pos + 1 + lane; q < ub; q += 32) {
        const int32_t j = (int32_t)p.sval[q];
        // the shared part of the two lifetimes, and its buckets
        const int32_t lo = p.born ? max(bi, p.born[j]) : 0, hi = p.born ? min(di, p.died[j]) : 1;
        if (lo >= hi) continue;
        const int32_t b0 = p.born ? (int32_t)(lo / p.bl) : 0, b1 = p.born ? (int32_t)((hi - 1) / p.bl) : 0;
        for (int32_t b = b0; b <= b1; ++b) {
            const int64_t li = (int64_t)i * p.nb + b, lj = (int64_t)j * p.nb + b;
            if (FILL) {
                const int64_t wi = p.off[li] + atomicAdd(&p.cnt[li], 1);
                const int64_t wj = p.off[lj] + atomicAdd(&p.cnt[lj], 1);
                p.pkey[wi] = (uint32_t)j;
                p.pval[wi] = (uint32_t)li;
                p.pkey[wj] = (uint32_t)i;
                p.pval[wj] = (uint32_t)lj;
            } else {
                atomicAdd(&p.cnt[li], 1);
                atomicAdd(&p.cnt[lj], 1);
            }
        }
    }
}

// the total; over capacity: an error, and the gate that turns off the fill,
// the sorts and the copy
__global__ void ov_total_kernel(const int64_t* __restrict__ off, int64_t NL, int64_t cap, int64_t* n_pairs, int* err,
                                int* gate)
{
    const int64_t t = off[NL];
    if (n_pairs) *n_pairs = t;
    const bool over = cap > 0 && t > cap;
    if (over) raise_error(err, AMC_E_RANGE);
    if (gate) *gate = over ? 1 : 0;
}

// over capacity: every list empty, so that no later kernel reads an entry
// that was not written
__global__ void ov_clear_kernel(int64_t* __restrict__ off, int64_t NL, const int* gate)
{
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (*gate && a <= NL) off[a] = 0;
}

__global__ void ov_zero_kernel(int32_t* __restrict__ cnt, int64_t NL)
{
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a < NL) cnt[a] = 0;
}

// the pairs after the sort, as ov_idx
__global__ void ov_copy_kernel(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst, const int64_t* off,
                               int64_t NL, int64_t cap)
{
    if (off[NL] > cap) return;
    const int64_t n = off[NL];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

struct OvLayout {
    size_t k0, v0, k1, v1, sscr, cnt, scan, gate, p0, p1, p2, p3, pscr, total;
};

OvLayout layout(int32_t A, int32_t nb, int64_t cap)
{
    OvLayout L;
    size_t o = 0;
    auto take = [&](size_t b) { const size_t at = o; o += align_up(b, 256); return at; };
    const size_t a4 = 4 * (size_t)(A > 0 ? A : 1);
    const int64_t NL = (int64_t)(A > 0 ? A : 1) * (nb > 0 ? nb : 1);
    L.k0 = take(a4);
    L.v0 = take(a4);
    L.k1 = take(a4);
    L.v1 = take(a4);
    L.sscr = take(sorted_check_scratch_bytes(A > 0 ? A : 1));
    L.cnt = take(4 * (size_t)NL);
    L.scan = take(dscan_workspace_bytes(NL));
    L.gate = take(4);
    const size_t c4 = 4 * (size_t)(cap > 0 ? cap : 1);
    L.p0 = take(c4);
    L.p1 = take(c4);
    L.p2 = take(c4);
    L.p3 = take(c4);
    L.pscr = take(sorted_check_scratch_bytes(cap > 0 ? cap : 1));
    L.total = o;
    return L;
}

}  // namespace

size_t overlap_workspace_bytes(int32_t n_arrays, int32_t n_buckets, int64_t cap)
{
    return layout(n_arrays, n_buckets, cap).total;
}

int32_t overlap_buckets(int64_t n_calls, bool lifetimes)
{
    if (!lifetimes || n_calls <= 1) return 1;
    return (int32_t)(n_calls < OV_MAX_BUCKETS ? n_calls : OV_MAX_BUCKETS);
}

int64_t overlap_bucket_len(int64_t n_calls, int32_t n_buckets)
{
    return n_calls <= 0 ? 1 : (n_calls + n_buckets - 1) / n_buckets;
}

int launch_overlaps(const OverlapBuild& O, cudaStream_t s)
{
    const int32_t A = O.n_arrays;
    const int32_t nb = O.arr_born ? (O.n_buckets > 0 ? O.n_buckets : 1) : 1;
    const int64_t NL = (int64_t)A * nb;
    if (A <= 0) {
        if (cudaMemsetAsync(O.ov_off, 0, 8, s) != cudaSuccess) return AMC_E_CUDA;
        if (O.n_pairs && cudaMemsetAsync(O.n_pairs, 0, 8, s) != cudaSuccess) return AMC_E_CUDA;
        return AMC_OK;
    }
    const OvLayout L = layout(A, nb, O.cap);
    uint8_t* w = static_cast<uint8_t*>(O.workspace);
    uint32_t* k[2] = {reinterpret_cast<uint32_t*>(w + L.k0), reinterpret_cast<uint32_t*>(w + L.k1)};
    uint32_t* v[2] = {reinterpret_cast<uint32_t*>(w + L.v0), reinterpret_cast<uint32_t*>(w + L.v1)};
    OvParams p{};
    p.start = O.arr_start;
    p.len = O.arr_len;
    p.born = O.arr_born;
    p.died = O.arr_died;
    p.A = A;
    p.nb = nb;
    p.bl = O.bucket_len > 0 ? O.bucket_len : 1;
    p.cnt = reinterpret_cast<int32_t*>(w + L.cnt);
    p.off = O.ov_off;
    p.cap = O.cap;
    p.err = O.err;
    const unsigned ab = (unsigned)((A + 255) / 256);
    const unsigned lb = (unsigned)((NL + 256) / 256);
    ov_keys_kernel<<<ab, 256, 0, s>>>(O.arr_start, O.arr_len, A, k[0], v[0], O.err);
    ov_zero_kernel<<<lb, 256, 0, s>>>(p.cnt, NL);
    int passes = 0;
    // starts are < 2^31: 31 key bits
    int rc = launch_ss_radix(k, v, nullptr, A, INT32_MAX, w + L.sscr, nullptr, s, &passes);
    if (rc) return rc;
    p.skey = k[passes & 1];
    p.sval = v[passes & 1];
    const unsigned wb = (unsigned)(((int64_t)A * 32 + 255) / 256);
    ov_sweep_kernel<false><<<wb, 256, 0, s>>>(p);
    rc = dscan_exclusive(p.cnt, O.ov_off, NL, w + L.scan, s);
    if (rc) return rc;
    int* gate = reinterpret_cast<int*>(w + L.gate);
    ov_total_kernel<<<1, 1, 0, s>>>(O.ov_off, NL, O.cap, O.n_pairs, O.err, gate);
    if (O.cap <= 0 || !O.ov_idx) return cudaGetLastError() == cudaSuccess ? AMC_OK : AMC_E_CUDA;   // count only
    ov_zero_kernel<<<lb, 256, 0, s>>>(p.cnt, NL);
    uint32_t* pk[2] = {reinterpret_cast<uint32_t*>(w + L.p0), reinterpret_cast<uint32_t*>(w + L.p1)};
    uint32_t* pv[2] = {reinterpret_cast<uint32_t*>(w + L.p2), reinterpret_cast<uint32_t*>(w + L.p3)};
    p.pkey = pk[0];
    p.pval = pv[0];
    ov_sweep_kernel<true><<<wb, 256, 0, s>>>(p);
    // by other, then (stably) by owner list; the count is read on the device
    const int64_t* n_dev = O.ov_off + NL;
    rc = launch_ss_radix(pk, pv, n_dev, O.cap, A, w + L.pscr, gate, s, &passes);
    if (rc) return rc;
    const int b1 = passes & 1;
    uint32_t* k2[2] = {pv[b1], pv[b1 ^ 1]};          // owner list as the key
    uint32_t* v2[2] = {pk[b1], pk[b1 ^ 1]};          // other as the value
    int passes2 = 0;
    rc = launch_ss_radix(k2, v2, n_dev, O.cap, (int32_t)(NL < INT32_MAX ? NL : INT32_MAX), w + L.pscr, gate, s,
                         &passes2);
    if (rc) return rc;
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    ov_copy_kernel<<<(unsigned)(n_sm > 0 ? 4 * n_sm : 256), 256, 0, s>>>(v2[passes2 & 1], O.ov_idx, O.ov_off, NL,
                                                                           O.cap);
    ov_clear_kernel<<<lb, 256, 0, s>>>(O.ov_off, NL, gate);
    return cudaGetLastError() == cudaSuccess ? AMC_OK : AMC_E_CUDA;
}

}  // namespace amc
