// batch.cu -- relation mode over a batch of structured programs (sm_103a).
//
// Semantics (Fig. Opsem with opaque conditions): every variable carries the
// SET of statuses it may have (a 5-bit mask); an op maps the set to its image;
// If joins the sets its two branches produce from the same entry sets; While
// loops until the set at its head stops growing (X = entry U body(X)), and the
// ops of its body report the sets of the pass that starts from that fixpoint.
// A program's "first fault" is the smallest token of an op whose possible
// pre-statuses include a non-stuck status that the op makes stuck.
//
// Work: one warp per program, programs taken from a queue ordered longest
// first (work split by op count).  Consecutive op tokens are handled 32 at a
// time: lanes with the same variable are grouped (match.any) and the group's
// first lane applies their images in token order.  Structure tokens are
// handled by the whole warp: entering an If or While saves, for every op token
// inside it, its variable's set (save[level][token]); at ELSE the then-results
// are kept (alt[level][token]) and the entry sets restored; at the If's END
// the two results are joined; at the While's END the sets are joined into the
// loop-head sets and the body runs again if any grew.  Because every variable
// a construct touches has an op token inside it, these per-token copies cover
// exactly the variables that matter.  Sets live in shared memory when the
// program has at most SMEM_VARS variables, else in the final_mask output.
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "amc_internal.cuh"
#include "batch.cuh"

namespace amc {

namespace {

constexpr int SMEM_VARS = 4096;
constexpr int WARPS = 8;
constexpr uint32_t MAX_WHILE_PASSES = 32;

__device__ __forceinline__ bool is_op(uint32_t ks) { return (ks & 0xE0u) == 0 && (ks & 15u) <= AMC_K_PW; }

template <bool SMEM>
__device__ void run_program(const BatchParams& p, int64_t prog, uint8_t* smM, uint8_t* stage)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    const int64_t t0 = p.prog_tok_off[prog], t1 = p.prog_tok_off[prog + 1];
    const int32_t nv = p.prog_nvars[prog];
    uint8_t* gM = p.final_mask + p.prog_var_off[prog];
    uint8_t* M = SMEM ? smM : gM;
    if (t0 < 0 || t1 < t0 || t1 > p.n_tokens || nv < 0 || p.prog_var_off[prog] < 0 ||
        p.prog_var_off[prog + 1] - p.prog_var_off[prog] != nv) {
        if (lane == 0) raise_error(p.err, AMC_E_INVALID);
        return;
    }
    for (int32_t v = lane; v < nv; v += 32) M[v] = p.init_mask ? p.init_mask[p.prog_var_off[prog] + v] : 2u;
    __syncwarp();
    // frames (identical in every lane): kind (8 = IF, 10 = WHILE) and pass
    // count; construct token, ELSE token and END token
    int fk[AMC_MAX_DEPTH * 2];
    int64_t fpos[AMC_MAX_DEPTH * 3] = {};
    int depth = 0;
    int64_t ff = INT64_MAX;
    bool bad = false;
    int64_t pos = t0;
    auto range_end = [&]() -> int64_t { return depth ? fpos[(depth - 1) * 3 + 2] : t1; };
    // parallel helper over the op tokens of (a, b)
    auto for_ops = [&](int64_t a, int64_t b, auto&& f) {
        for (int64_t q = a + lane; q < b; q += 32) {
            const uint32_t ks = p.tok[q];
            if (is_op(ks)) {
                const int32_t v = p.payload[q];
                if (v >= 0 && v < nv) f(q, v);
            }
        }
    };
    while (pos < t1 && !bad) {
        const uint32_t ks0 = p.tok[pos];
        const uint32_t k0 = ks0 & 15u;
        if (is_op(ks0)) {
            // a run of up to 32 op tokens
            const int64_t lim = range_end();
            const int64_t q = pos + lane;
            const uint32_t ks = q < lim ? p.tok[q] : 0xFFu;
            const uint32_t opm = __ballot_sync(0xffffffffu, is_op(ks));
            const int cnt = __ffs(~opm) - 1 < 0 ? 32 : __ffs(~opm) - 1;
            const bool act = lane < cnt;
            int32_t v = act ? p.payload[q] : -1;
            if (act && (v < 0 || v >= nv)) {
                raise_error(p.err, AMC_E_RANGE);
                v = -1;
            }
            const uint32_t oi = ((ks & 15u) << 1) | ((ks >> 4) & 1u);
            stage[lane] = (uint8_t)oi;
            __syncwarp();
            const uint32_t key = (act && v >= 0) ? (uint32_t)v : 0x80000000u + lane;
            const uint32_t peers = __match_any_sync(0xffffffffu, key);
            if (act && v >= 0 && (peers & lt) == 0) {
                // group leader: apply the group's ops in token order
                uint32_t m = M[v];
                uint32_t rest = peers;
                while (rest) {
                    const int L = __ffs(rest) - 1;
                    rest &= rest - 1;
                    const uint32_t o = stage[L];
                    if ((p.tab.flt[o] >> m) & 1u) ff = min(ff, pos + L - t0);
                    m = p.tab.img[o * 32 + m];
                    p.step_mask[pos + L] = (uint8_t)m;
                }
                M[v] = (uint8_t)m;
            }
            __syncwarp();
            pos += cnt;
        } else if (k0 == AMC_T_IF || k0 == AMC_T_WHILE) {
            const int64_t lim = range_end();
            const int64_t len = p.payload[pos];
            int64_t e = -1, end;
            if (k0 == AMC_T_IF) {
                e = pos + 1 + len;
                end = (len >= 0 && e < lim && (p.tok[e] & 0xEFu) == AMC_T_ELSE) ? e + 1 + (int64_t)p.payload[e] : -1;
            } else {
                end = pos + 1 + len;
            }
            if ((ks0 >> 4) || len < 0 || end <= pos || end >= lim || (p.tok[end] & 0xEFu) != AMC_T_END ||
                (p.tok[end] >> 4) || depth >= AMC_MAX_DEPTH) {
                bad = true;
                break;
            }
            uint8_t* save = p.save + (int64_t)depth * p.n_tokens;
            for_ops(pos + 1, end, [&](int64_t q, int32_t v) { save[q] = M[v]; });
            __syncwarp();
            fk[depth * 2] = (int)k0;
            fk[depth * 2 + 1] = 0;
            fpos[depth * 3 + 0] = pos;
            fpos[depth * 3 + 1] = e;
            fpos[depth * 3 + 2] = end;
            ++depth;
            if (lane == 0) p.step_mask[pos] = 0;
            ++pos;
        } else if (k0 == AMC_T_ELSE) {
            if (!depth || fk[(depth - 1) * 2] != AMC_T_IF || fpos[(depth - 1) * 3 + 1] != pos || (ks0 >> 4)) {
                bad = true;
                break;
            }
            const int d = depth - 1;
            const int64_t a = fpos[d * 3], b = fpos[d * 3 + 2];
            uint8_t* save = p.save + (int64_t)d * p.n_tokens;
            uint8_t* alt = p.alt + (int64_t)d * p.n_tokens;
            for_ops(a + 1, b, [&](int64_t q, int32_t v) { alt[q] = M[v]; });      // then-results
            __syncwarp();
            for_ops(a + 1, b, [&](int64_t q, int32_t v) { M[v] = save[q]; });     // entry sets again
            __syncwarp();
            if (lane == 0) p.step_mask[pos] = 0;
            ++pos;
        } else if (k0 == AMC_T_END) {
            if (!depth || fpos[(depth - 1) * 3 + 2] != pos || (ks0 >> 4)) {
                bad = true;
                break;
            }
            const int d = depth - 1;
            const int64_t a = fpos[d * 3], b = pos;
            uint8_t* save = p.save + (int64_t)d * p.n_tokens;
            if (lane == 0) p.step_mask[pos] = 0;
            if (fk[d * 2] == AMC_T_IF) {
                uint8_t* alt = p.alt + (int64_t)d * p.n_tokens;
                for_ops(a + 1, b, [&](int64_t q, int32_t v) { M[v] = (uint8_t)(M[v] | alt[q]); });
                __syncwarp();
                --depth;
                ++pos;
            } else {
                bool grew = false;
                for_ops(a + 1, b, [&](int64_t q, int32_t v) {
                    const uint32_t x = save[q], nx = x | M[v];
                    grew |= nx != x;
                    save[q] = (uint8_t)nx;
                    M[v] = (uint8_t)nx;
                });
                __syncwarp();
                if (__any_sync(0xffffffffu, grew)) {
                    if (++fk[d * 2 + 1] > (int)MAX_WHILE_PASSES) {
                        bad = true;
                        break;
                    }
                    pos = a + 1;            // run the body again from the grown sets
                } else {
                    --depth;
                    ++pos;
                }
            }
        } else {
            bad = true;                     // GT / EN / unknown byte in a program
        }
    }
    if (!bad && depth) bad = true;          // construct not closed
    if (bad && lane == 0) raise_error(p.err, AMC_E_INVALID);
    // program first fault: min over lanes
#pragma unroll
    for (int o = 16; o; o >>= 1) ff = min(ff, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)ff, o));
    if (lane == 0) p.prog_first_fault[prog] = ff == INT64_MAX ? -1 : ff;
    if (SMEM) {
        __syncwarp();
        for (int32_t v = lane; v < nv; v += 32) gM[v] = M[v];
    }
}

__global__ void __launch_bounds__(WARPS * 32) batch_kernel(const BatchParams p)
{
    __shared__ uint8_t smM[WARPS][SMEM_VARS];
    __shared__ uint8_t stage[WARPS][32];
    const int w = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    for (;;) {
        int64_t i = 0;
        if (lane == 0) i = atomicAdd(reinterpret_cast<unsigned long long*>(p.queue_head), 1ull);
        i = __shfl_sync(0xffffffffu, (long long)i, 0);
        if (i >= p.n_progs) break;
        const int64_t prog = p.order ? p.order[i] : i;
        if (p.prog_nvars[prog] <= SMEM_VARS)
            run_program<true>(p, prog, smM[w], stage[w]);
        else
            run_program<false>(p, prog, smM[w], stage[w]);
        __syncwarp();
    }
}

// Work list: programs by decreasing token count (stable), by a key of
// (length bucket) in a counting sort done on the host side of the queue.
__global__ void order_kernel(const int64_t* __restrict__ tok_off, int64_t n, const int64_t* __restrict__ bucket_off,
                             int32_t* __restrict__ cursor, int32_t* __restrict__ order)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t len = tok_off[i + 1] - tok_off[i];
    const int b = len <= 0 ? 63 : 63 - (64 - __clzll(len));      // longer programs, smaller bucket
    const int slot = atomicAdd(&cursor[b], 1);
    order[bucket_off[b] + slot] = (int32_t)i;
}

__global__ void bucket_count_kernel(const int64_t* __restrict__ tok_off, int64_t n, int32_t* __restrict__ counts)
{
    __shared__ int32_t c[64];
    if (threadIdx.x < 64) c[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t len = tok_off[i + 1] - tok_off[i];
        const int b = len <= 0 ? 63 : 63 - (64 - __clzll(len));
        atomicAdd(&c[b], 1);
    }
    __syncthreads();
    if (threadIdx.x < 64 && c[threadIdx.x]) atomicAdd(&counts[threadIdx.x], c[threadIdx.x]);
}

__global__ void bucket_scan_kernel(const int32_t* __restrict__ counts, int64_t* __restrict__ off,
                                   int32_t* __restrict__ cursor)
{
    if (threadIdx.x == 0) {
        int64_t s = 0;
        for (int b = 0; b < 64; ++b) {
            off[b] = s;
            s += counts[b];
            cursor[b] = 0;
        }
    }
}

struct BatchLayout {
    size_t save, alt, order, counts, cursor, boff, head, total;
};

BatchLayout layout(int64_t n_tokens, int64_t n_progs)
{
    BatchLayout L;
    size_t o = 0;
    L.save = o;
    o += align_up((size_t)AMC_MAX_DEPTH * (size_t)n_tokens + 1, 256);
    L.alt = o;
    o += align_up((size_t)AMC_MAX_DEPTH * (size_t)n_tokens + 1, 256);
    L.order = o;
    o += align_up(4 * (size_t)n_progs + 4, 256);
    L.counts = o;
    o += 256;
    L.cursor = o;
    o += 256;
    L.boff = o;
    o += 512;
    L.head = o;
    o += 256;
    L.total = o;
    return L;
}

}  // namespace

size_t batch_workspace_bytes(int64_t n_tokens, int64_t n_progs) { return layout(n_tokens, n_progs).total; }

int launch_batch(const BatchLaunch& B, cudaStream_t s)
{
    BatchParams p{};
    p.tok = B.tok;
    p.payload = B.payload;
    p.prog_tok_off = B.prog_tok_off;
    p.prog_nvars = B.prog_nvars;
    p.prog_var_off = B.prog_var_off;
    p.n_progs = B.n_progs;
    p.n_tokens = B.n_tokens;
    p.init_mask = B.init_mask;
    p.step_mask = B.step_mask;
    p.final_mask = B.final_mask;
    p.prog_first_fault = B.prog_first_fault;
    p.err = B.err;
    p.tab = host_set_tables();
    const BatchLayout L = layout(B.n_tokens, B.n_progs);
    uint8_t* w = static_cast<uint8_t*>(B.workspace);
    p.save = w + L.save;
    p.alt = w + L.alt;
    int32_t* order = reinterpret_cast<int32_t*>(w + L.order);
    int32_t* counts = reinterpret_cast<int32_t*>(w + L.counts);
    int32_t* cursor = reinterpret_cast<int32_t*>(w + L.cursor);
    int64_t* boff = reinterpret_cast<int64_t*>(w + L.boff);
    p.queue_head = reinterpret_cast<uint64_t*>(w + L.head);
    if (B.n_progs <= 0) return AMC_OK;
    if (cudaMemsetAsync(p.queue_head, 0, 8, s) != cudaSuccess) return AMC_E_CUDA;
    if (B.longest_first) {
        if (cudaMemsetAsync(counts, 0, 256, s) != cudaSuccess) return AMC_E_CUDA;
        bucket_count_kernel<<<128, 256, 0, s>>>(B.prog_tok_off, B.n_progs, counts);
        bucket_scan_kernel<<<1, 32, 0, s>>>(counts, boff, cursor);
        order_kernel<<<(unsigned)((B.n_progs + 255) / 256), 256, 0, s>>>(B.prog_tok_off, B.n_progs, boff, cursor,
                                                                           order);
        p.order = order;
    }
    int dev = 0, n_sm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, WARPS * 32, 0);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)n_sm * per_sm;
    const int64_t need = (B.n_progs + WARPS - 1) / WARPS;
    if (grid > need) grid = need;
    if (B.max_ctas > 0 && grid > B.max_ctas) grid = B.max_ctas;
    if (B.profile & 1) profile_begin(s);
    batch_kernel<<<(unsigned)grid, WARPS * 32, 0, s>>>(p);
    if (B.profile & 2) profile_end(s);
    return cudaGetLastError() == cudaSuccess ? AMC_OK : AMC_E_CUDA;
}

}  // namespace amc
