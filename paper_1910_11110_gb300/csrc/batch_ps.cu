// batch_ps.cu -- path-sensitive relation mode over a batch of structured
// programs (sm_103a).
//
// Semantics (Fig. Opsem: rules valid / invalid / rem-valid / rem-invalid,
// IF-True / IF-False, While-True / While-False): the conditions of If and
// While are isValid g or remIsValid g on the program's guard variable g, or
// opaque (x (+) y: both outcomes).  Control flow then depends on g alone, so
// for every other variable x the set of reachable pairs (status of g, status
// of x) -- a 5x5 bit matrix, bit 5 i + j for g = i, x = j -- is exactly the
// projection of the reachable stores; g's own statuses are a 5-bit set.  An
// op on x maps each row (a fixed g status) through the op's set image; an op
// on g moves whole rows; a condition keeps the rows whose g status makes it
// true (or false), never the stuck one (no rule applies to it, the path
// ends).  If: both branches from the filtered entry state, joined.  While:
// the loop-head state is the least X with X = entry U body(X restricted to
// the condition), the body's step sets are those of the pass from that
// fixpoint, and the loop is left with X restricted to the condition's
// negation.  Each variable's F is absorbing and does not stop the others, as
// in the opaque relation mode.  Step output: the statuses the op's variable
// may have after it (the union of its pair set's rows; 0 where the op is not
// reachable).
//
// Work: one warp per program from a longest-first queue.  Runs of up to 32
// op tokens on variables other than g are applied 32 at a time (lanes with
// the same variable grouped by match.any, the group's first lane applying
// them in order); an op on g, and every condition, touches every variable's
// pair set (lanes stride the variables).  Entering a construct copies the
// whole state (every variable's pair set and g's set) to that level's save
// row, ELSE to the alt row.  Pair sets live in shared memory for programs of
// at most PS_SMEM_VARS variables, else in the workspace.
#include <cstdlib>

#include "amc_internal.cuh"
#include "batch_ps.cuh"

namespace amc {

namespace {

constexpr int PS_WARPS = 8;
constexpr int PS_SMEM_VARS = 1024;
constexpr uint32_t PS_MAX_PASSES = 64;
constexpr uint8_t ROWS_ALL = 31;

__device__ __forceinline__ bool ps_is_op(uint32_t ks) { return (ks & 0xE0u) == 0 && (ks & 15u) <= AMC_K_PW; }

struct PsTab {
    uint8_t img[16 * 32];         // set image per op index (kind << 1 | side)
    uint32_t flt[16];             // bit m: the set m may get stuck under the op
    uint8_t tgt[16 * 8];          // status an op maps status i to (row moves of an op on g)
};

struct PsWarp {
    uint32_t J[PS_SMEM_VARS];
    uint8_t stage[32];
};

__device__ __forceinline__ uint32_t row_mask(uint32_t rows)
{
    uint32_t m = 0;
#pragma unroll
    for (int i = 0; i < 5; ++i)
        if ((rows >> i) & 1u) m |= 31u << (5 * i);
    return m;
}

__device__ __forceinline__ uint32_t proj(uint32_t J)
{
    return (J | (J >> 5) | (J >> 10) | (J >> 15) | (J >> 20)) & 31u;
}

// rows kept on the then side (t) and the else side (e) of condition c
__device__ __forceinline__ void cond_rows(uint32_t c, uint32_t& t, uint32_t& e)
{
    if (c == 0) {
        t = e = ROWS_ALL;
        return;
    }
    // statuses 0 (I,I) 1 (V,I) 2 (I,V) 3 (V,V): local flag bit 0, remote bit 1
    const uint32_t bit = c == 1 ? 1u : 2u;
    t = 0;
    e = 0;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        if (s & bit) t |= 1u << s;
        else e |= 1u << s;
    }
}

template <bool SMEM>
__device__ void run_ps(const PsParams& p, int64_t prog, PsWarp& S, const PsTab& T)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    const int64_t t0 = p.prog_tok_off[prog], t1 = p.prog_tok_off[prog + 1];
    const int32_t nv = p.prog_nvars[prog];
    const int64_t vo = p.prog_var_off[prog];
    const int32_t g = p.prog_guard[prog];
    if (t0 < 0 || t1 < t0 || t1 > p.n_tokens || nv < 0 || vo < 0 || p.prog_var_off[prog + 1] - vo != nv ||
        g < -1 || g >= nv) {
        if (lane == 0) raise_error(p.err, AMC_E_INVALID);
        return;
    }
    uint32_t* J = SMEM ? S.J : p.J + vo;
    auto row_of = [&](int d, int k) { return p.save + ((int64_t)d * 2 + k) * p.total_vars + vo; };
    const uint32_t vi = 1u << AMC_ST_VI;
    uint32_t G = g >= 0 ? (p.init_mask ? p.init_mask[vo + g] : vi) : 1u;     // no guard: a single row
    for (int32_t x = lane; x < nv; x += 32) {
        const uint32_t m = p.init_mask ? p.init_mask[vo + x] : vi;
        uint32_t j = 0;
#pragma unroll
        for (int i = 0; i < 5; ++i)
            if ((G >> i) & 1u) j |= m << (5 * i);
        J[x] = x == g ? 0u : j;
    }
    __syncwarp();
    // frames: kind | cond << 4, passes; construct, ELSE and END tokens; g sets
    int fk[AMC_MAX_DEPTH], fpass[AMC_MAX_DEPTH];
    int64_t fpos[AMC_MAX_DEPTH * 3] = {};
    uint32_t gsave[AMC_MAX_DEPTH], galt[AMC_MAX_DEPTH];
    int depth = 0;
    int64_t ff = INT64_MAX;
    bool bad = false;
    int64_t pos = t0;
    auto range_end = [&]() -> int64_t { return depth ? fpos[(depth - 1) * 3 + 2] : t1; };
    auto keep = [&](uint32_t rows) {            // every pair set restricted to rows
        const uint32_t m = row_mask(rows);
        for (int32_t x = lane; x < nv; x += 32) J[x] &= m;
        G &= rows;
    };
    while (pos < t1 && !bad) {
        const uint32_t ks0 = p.tok[pos];
        const uint32_t k0 = ks0 & 15u;
        if (ps_is_op(ks0)) {
            const int32_t v0 = p.payload[pos];
            if (v0 == g && g >= 0) {
                // an op on g: rows move, g's set maps through the op
                const uint32_t o = (k0 << 1) | ((ks0 >> 4) & 1u);
                if ((T.flt[o] >> G) & 1u) ff = min(ff, pos - t0);
                for (int32_t x = lane; x < nv; x += 32) {
                    if (x == g) continue;
                    const uint32_t j = J[x];
                    uint32_t out = 0;
#pragma unroll
                    for (int i = 0; i < 5; ++i) out |= ((j >> (5 * i)) & 31u) << (5 * T.tgt[o * 8 + i]);
                    J[x] = out;
                }
                G = T.img[o * 32 + G];
                if (lane == 0) p.step_mask[pos] = (uint8_t)G;
                __syncwarp();
                ++pos;
                continue;
            }
            // a run of up to 32 op tokens on variables other than g
            const int64_t lim = range_end();
            const int64_t q = pos + lane;
            const uint32_t ks = q < lim ? p.tok[q] : 0xFFu;
            const int32_t pl = q < lim ? p.payload[q] : -1;
            const bool opx = ps_is_op(ks) && !(pl == g && g >= 0);
            const uint32_t opm = __ballot_sync(0xffffffffu, opx);
            const int cnt = (~opm) ? __ffs(~opm) - 1 : 32;
            const bool act = lane < cnt;
            int32_t v = act ? pl : -1;
            if (act && (v < 0 || v >= nv)) {
                raise_error(p.err, AMC_E_RANGE);
                v = -1;
            }
            S.stage[lane] = (uint8_t)(((ks & 15u) << 1) | ((ks >> 4) & 1u));
            __syncwarp();
            const uint32_t key = (act && v >= 0) ? (uint32_t)v : 0x80000000u + lane;
            const uint32_t peers = __match_any_sync(0xffffffffu, key);
            if (act && v >= 0 && (peers & lt) == 0) {
                uint32_t j = J[v];
                for (uint32_t rest = peers; rest; rest &= rest - 1) {
                    const int L = __ffs(rest) - 1;
                    const uint32_t o = S.stage[L];
                    if ((T.flt[o] >> proj(j)) & 1u) ff = min(ff, pos + L - t0);
                    uint32_t out = 0;
#pragma unroll
                    for (int i = 0; i < 5; ++i) out |= (uint32_t)T.img[o * 32 + ((j >> (5 * i)) & 31u)] << (5 * i);
                    j = out;
                    p.step_mask[pos + L] = (uint8_t)proj(j);
                }
                J[v] = j;
            }
            if (act && v < 0) p.step_mask[q] = 0;
            __syncwarp();
            pos += cnt;
        } else if (k0 == AMC_T_IF || k0 == AMC_T_WHILE) {
            const uint32_t c = ks0 >> 4;
            const int64_t lim = range_end();
            const int64_t len = p.payload[pos];
            int64_t e = -1, end;
            if (k0 == AMC_T_IF) {
                e = pos + 1 + len;
                end = (len >= 0 && e < lim && p.tok[e] == AMC_T_ELSE) ? e + 1 + (int64_t)p.payload[e] : -1;
            } else {
                end = pos + 1 + len;
            }
            if (c > 2 || (c && g < 0) || len < 0 || end <= pos || end >= lim || p.tok[end] != AMC_T_END ||
                depth >= AMC_MAX_DEPTH) {
                bad = true;
                break;
            }
            const int d = depth;
            uint32_t* sv = row_of(d, 0);
            for (int32_t x = lane; x < nv; x += 32) sv[x] = J[x];
            gsave[d] = G;
            __syncwarp();
            uint32_t tr, er;
            cond_rows(c, tr, er);
            if (tr != ROWS_ALL) keep(tr);
            __syncwarp();
            fk[d] = (int)(k0 | (c << 4));
            fpass[d] = 0;
            fpos[d * 3 + 0] = pos;
            fpos[d * 3 + 1] = e;
            fpos[d * 3 + 2] = end;
            ++depth;
            if (lane == 0) p.step_mask[pos] = 0;
            ++pos;
        } else if (ks0 == AMC_T_ELSE) {
            if (!depth || (fk[depth - 1] & 15) != AMC_T_IF || fpos[(depth - 1) * 3 + 1] != pos) {
                bad = true;
                break;
            }
            const int d = depth - 1;
            uint32_t tr, er;
            cond_rows((uint32_t)fk[d] >> 4, tr, er);
            uint32_t* sv = row_of(d, 0);
            uint32_t* al = row_of(d, 1);
            const uint32_t m = row_mask(er);
            for (int32_t x = lane; x < nv; x += 32) {
                al[x] = J[x];                    // then-results
                J[x] = sv[x] & m;                // the entry state on the IF-False paths
            }
            galt[d] = G;
            G = gsave[d] & er;
            __syncwarp();
            if (lane == 0) p.step_mask[pos] = 0;
            ++pos;
        } else if (ks0 == AMC_T_END) {
            if (!depth || fpos[(depth - 1) * 3 + 2] != pos) {
                bad = true;
                break;
            }
            const int d = depth - 1;
            if (lane == 0) p.step_mask[pos] = 0;
            uint32_t tr, er;
            cond_rows((uint32_t)fk[d] >> 4, tr, er);
            uint32_t* sv = row_of(d, 0);
            if ((fk[d] & 15) == AMC_T_IF) {
                const uint32_t* al = row_of(d, 1);
                for (int32_t x = lane; x < nv; x += 32) J[x] |= al[x];
                G |= galt[d];
                __syncwarp();
                --depth;
                ++pos;
            } else {
                // loop head: X = X U body(X on the While-True paths)
                bool grew = false;
                for (int32_t x = lane; x < nv; x += 32) {
                    const uint32_t a = sv[x], b = a | J[x];
                    grew |= b != a;
                    sv[x] = b;
                }
                const uint32_t gn = gsave[d] | G;
                grew |= gn != gsave[d];
                gsave[d] = gn;
                __syncwarp();
                const uint32_t rows = __any_sync(0xffffffffu, grew) ? tr : er;
                const uint32_t m = row_mask(rows);
                for (int32_t x = lane; x < nv; x += 32) J[x] = sv[x] & m;
                G = gn & rows;
                __syncwarp();
                if (rows == tr && __any_sync(0xffffffffu, grew)) {
                    if (++fpass[d] > (int)PS_MAX_PASSES) {
                        bad = true;
                        break;
                    }
                    pos = fpos[d * 3] + 1;          // the body again from the grown head
                } else {
                    --depth;                        // While-False: leave with the head's other rows
                    ++pos;
                }
            }
        } else {
            bad = true;
        }
    }
    if (!bad && depth) bad = true;
    if (bad && lane == 0) raise_error(p.err, AMC_E_INVALID);
    __syncwarp();
#pragma unroll
    for (int o = 16; o; o >>= 1) ff = min(ff, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)ff, o));
    if (lane == 0) p.prog_first_fault[prog] = ff == INT64_MAX ? -1 : ff;
    for (int32_t x = lane; x < nv; x += 32) p.final_mask[vo + x] = (uint8_t)(x == g ? G : proj(J[x]));
}

__global__ void __launch_bounds__(PS_WARPS * 32) ps_kernel(const PsParams p)
{
    __shared__ PsWarp warps[PS_WARPS];
    __shared__ PsTab tab;
    for (int i = threadIdx.x; i < 16 * 32; i += blockDim.x) tab.img[i] = p.tab.img[i];
    if (threadIdx.x < 16) tab.flt[threadIdx.x] = p.tab.flt[threadIdx.x];
    for (int i = threadIdx.x; i < 16 * 8; i += blockDim.x) {
        const int o = i >> 3, s = i & 7;
        const uint32_t im = s < 5 ? p.tab.img[o * 32 + (1 << s)] : 0u;
        tab.tgt[i] = (uint8_t)(im ? __ffs(im) - 1 : 0);
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        int64_t i = 0;
        if (lane == 0) i = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(p.queue_head), 1ull);
        i = __shfl_sync(0xffffffffu, (long long)i, 0);
        if (i >= p.n_progs) break;
        const int64_t prog = p.order ? p.order[i] : i;
        if (p.prog_nvars[prog] <= PS_SMEM_VARS)
            run_ps<true>(p, prog, warps[w], tab);
        else
            run_ps<false>(p, prog, warps[w], tab);
        __syncwarp();
    }
}

// queue order: programs by decreasing length bucket (counting sort by
// floor(log2(tokens)), any order within a bucket)
__device__ __forceinline__ int ps_bucket(int64_t len) { return len <= 0 ? 63 : 63 - (64 - __clzll(len)); }

__global__ void ps_count_kernel(const int64_t* __restrict__ tok_off, int64_t n, int32_t* __restrict__ counts)
{
    __shared__ int32_t c[64];
    if (threadIdx.x < 64) c[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&c[ps_bucket(tok_off[i + 1] - tok_off[i])], 1);
    __syncthreads();
    if (threadIdx.x < 64 && c[threadIdx.x]) atomicAdd(&counts[threadIdx.x], c[threadIdx.x]);
}

__global__ void ps_scan_kernel(int32_t* __restrict__ counts, int64_t* __restrict__ boff)
{
    if (threadIdx.x == 0) {
        int64_t s = 0;
        for (int b = 0; b < 64; ++b) {
            boff[b] = s;
            s += counts[b];
            counts[b] = 0;
        }
    }
}

__global__ void ps_order_kernel(const int64_t* __restrict__ tok_off, int64_t n, const int64_t* __restrict__ boff,
                                int32_t* __restrict__ cursor, int32_t* __restrict__ order)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = ps_bucket(tok_off[i + 1] - tok_off[i]);
    order[boff[b] + atomicAdd(&cursor[b], 1)] = (int32_t)i;
}

struct PsLayout {
    size_t J, save, order, counts, boff, head, total;
};

PsLayout layout(int64_t n_progs, int64_t total_vars)
{
    PsLayout L;
    size_t o = 0;
    auto take = [&](size_t b) { const size_t at = o; o += align_up(b, 256); return at; };
    const size_t tv = (size_t)(total_vars > 0 ? total_vars : 1);
    L.J = take(4 * tv);
    L.save = take(4 * tv * 2 * AMC_MAX_DEPTH);
    L.order = take(4 * (size_t)n_progs + 4);
    L.counts = take(256);
    L.boff = take(512);
    L.head = take(256);
    L.total = o;
    return L;
}

}  // namespace

size_t batch_ps_workspace_bytes(int64_t n_progs, int64_t total_vars) { return layout(n_progs, total_vars).total; }

int launch_batch_ps(const PsLaunch& B, cudaStream_t s)
{
    PsParams p{};
    p.tok = B.tok;
    p.payload = B.payload;
    p.prog_tok_off = B.prog_tok_off;
    p.prog_nvars = B.prog_nvars;
    p.prog_var_off = B.prog_var_off;
    p.prog_guard = B.prog_guard;
    p.n_progs = B.n_progs;
    p.n_tokens = B.n_tokens;
    p.total_vars = B.total_vars;
    p.init_mask = B.init_mask;
    p.step_mask = B.step_mask;
    p.final_mask = B.final_mask;
    p.prog_first_fault = B.prog_first_fault;
    p.err = B.err;
    p.tab = host_set_tables();
    const PsLayout L = layout(B.n_progs, B.total_vars);
    uint8_t* w = static_cast<uint8_t*>(B.workspace);
    p.J = reinterpret_cast<uint32_t*>(w + L.J);
    p.save = reinterpret_cast<uint32_t*>(w + L.save);
    p.queue_head = reinterpret_cast<uint64_t*>(w + L.head);
    int32_t* order = reinterpret_cast<int32_t*>(w + L.order);
    int32_t* counts = reinterpret_cast<int32_t*>(w + L.counts);
    int64_t* boff = reinterpret_cast<int64_t*>(w + L.boff);
    if (B.n_progs <= 0) return AMC_OK;
    if (cudaMemsetAsync(p.queue_head, 0, 8, s) != cudaSuccess) return AMC_E_CUDA;
    if (cudaMemsetAsync(counts, 0, 256, s) != cudaSuccess) return AMC_E_CUDA;
    ps_count_kernel<<<128, 256, 0, s>>>(B.prog_tok_off, B.n_progs, counts);
    ps_scan_kernel<<<1, 32, 0, s>>>(counts, boff);
    ps_order_kernel<<<(unsigned)((B.n_progs + 255) / 256), 256, 0, s>>>(B.prog_tok_off, B.n_progs, boff, counts,
                                                                          order);
    p.order = order;
    int dev = 0, n_sm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ps_kernel, PS_WARPS * 32, 0);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)n_sm * per_sm;
    const int64_t need = (B.n_progs + PS_WARPS - 1) / PS_WARPS;
    if (grid > need) grid = need;
    if (B.profile & 1) profile_begin(s);
    ps_kernel<<<(unsigned)grid, PS_WARPS * 32, 0, s>>>(p);
    if (B.profile & 2) profile_end(s);
    return cudaGetLastError() == cudaSuccess ? AMC_OK : AMC_E_CUDA;
}

}  // namespace amc
