// scan_sorted.cu -- a set of ops checked by grouping it by variable: a stable
// radix sort of (variable, index) pairs, then a segmented scan of the transfer
// functions over each variable's run.
//
// It computes what the single-pass scan computes for the same ops in the same
// order.  An op's status depends only on the earlier ops on its variable (Fig.
// Opsem, rules Effect / Remote Effect touch sigma(x) alone) and sequencing is
// associative (Section 3.2), so the ops may be regrouped by variable as long as
// each variable keeps its own order, and every op's status is the composition
// of its variable's earlier transfer functions and its own, applied to the
// variable's entry status.
//   1. pairs: key = variable id, value = index of the op in the set << 4 | its
//      kind and side (4 bits);
//   2. LSD radix sort by key, 7-bit digits; per pass a histogram per tile of
//      4,096 pairs, an exclusive scan of each digit's row over the tiles (one
//      CTA per digit; the digits' totals are scanned by every scatter CTA),
//      and a stable scatter
//      (each pair's rank from per-thread digit counters in shared memory over a
//      blocked arrangement, the tile staged in shared memory in digit order);
//   3. segmented scan over the sorted pairs in one pass (decoupled look-back
//      over the tiles' published values gives the carry into each tile's
//      leading run), every op's prefix applied to its variable's entry status.
// Outputs: the status of every op whose status is not F (the caller has
// written F at every position of the set), the first fault of each variable
// that faults in the set, the global first fault, and the final statuses.
#include <cstdio>

#include "amc_internal.cuh"
#include "scan_trace.cuh"

namespace amc {

namespace {

constexpr int ST = 4096;                 // pairs per tile
constexpr int SNT = 256;                 // threads per CTA
constexpr int SE = ST / SNT;             // pairs per thread (blocked)
constexpr int SDIG = 7;                  // digit bits
constexpr int SRAD = 1 << SDIG;
constexpr int CROWS = SRAD / 2;          // counter rows: digit d and d + 64 share a word (16-bit halves)
constexpr int CWORDS = CROWS * SNT;      // logical counter words
constexpr int CPHYS = CWORDS + CWORDS / 64;   // one pad word per 64: conflict-free row scans
constexpr uint32_t NOKEY = 0xFFFFFFFFu;  // no variable id equals it

__device__ __forceinline__ int cphys(int l) { return l + (l >> 6); }

__device__ __forceinline__ int64_t set_count(const int64_t* n_dev, int64_t cap)
{
    if (!n_dev) return cap;
    const int64_t n = *n_dev;
    return n < 0 ? 0 : (n < cap ? n : cap);
}

__device__ __forceinline__ bool gated(const int* gate) { return gate && *gate != 0; }

// 4-bit code (sorted_code_of) -> op byte
__device__ __forceinline__ uint32_t byte_of(uint32_t c) { return (c & 7u) | ((c & 8u) << 1); }

// Segmented-scan value: bits 0-4 the composed element, bit 8 "a run starts
// inside".  (x then y): y's element alone when a run starts in y, else x's
// element followed by y's.
__device__ __forceinline__ uint32_t seg_combine(uint32_t x, uint32_t y, const uint8_t* comp)
{
    if (y & 0x100u) return y;
    return (x & 0x100u) | comp[(x & 31u) * MAX_ELEMS + (y & 31u)];
}

// Thread loads of a tile's keys / values in blocked arrangement (thread t:
// pairs [16 t, 16 t + 16) of the tile); pairs past m are left as NOKEY.
__device__ __forceinline__ void load_blocked(const uint32_t* __restrict__ a, int64_t b, int m, uint32_t (&x)[SE],
                                             uint32_t fill)
{
    const int i0 = threadIdx.x * SE;
    if (m == ST) {
        const uint4* p = reinterpret_cast<const uint4*>(a + b + i0);
#pragma unroll
        for (int h = 0; h < SE / 4; ++h) {
            const uint4 q = p[h];
            x[4 * h] = q.x;
            x[4 * h + 1] = q.y;
            x[4 * h + 2] = q.z;
            x[4 * h + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int u = 0; u < SE; ++u) x[u] = (i0 + u < m) ? a[b + i0 + u] : fill;
    }
}

// (1) digit histogram of every tile: hist[d * n_tiles + t]
__global__ void __launch_bounds__(SNT) ss_hist_kernel(const uint32_t* __restrict__ key, const int64_t* n_dev,
                                                      int64_t cap, int shift, uint32_t* __restrict__ hist,
                                                      const int* gate)
{
    __shared__ uint32_t cnt[SRAD];
    if (gated(gate)) return;
    const int64_t n = set_count(n_dev, cap);
    const int64_t nt = (n + ST - 1) / ST;
    for (int64_t t = blockIdx.x; t < nt; t += gridDim.x) {
        if (threadIdx.x < SRAD) cnt[threadIdx.x] = 0;
        __syncthreads();
        const int64_t b = t * ST;
        const int m = (int)(n - b < ST ? n - b : ST);
        uint32_t k[SE];
        load_blocked(key, b, m, k, NOKEY);
#pragma unroll
        for (int u = 0; u < SE; ++u)
            if (k[u] != NOKEY) atomicAdd(&cnt[(k[u] >> shift) & (SRAD - 1)], 1u);
        __syncthreads();
        if (threadIdx.x < SRAD) hist[(int64_t)threadIdx.x * nt + t] = cnt[threadIdx.x];
        __syncthreads();
    }
}

// (2) CTA d: exclusive scan of digit d's row hist[d * n_tiles, + n_tiles) in
// place; the row's total to dtot[d]
__global__ void __launch_bounds__(1024) ss_hscan_kernel(uint32_t* __restrict__ hist, uint32_t* __restrict__ dtot,
                                                        const int64_t* n_dev, int64_t cap, const int* gate)
{
    __shared__ int tmp[1024 / 32 + 1];
    if (gated(gate)) return;
    const int64_t n = set_count(n_dev, cap);
    const int64_t nt = (n + ST - 1) / ST;
    uint32_t* row = hist + (int64_t)blockIdx.x * nt;
    const int64_t per = (nt + 1023) / 1024;
    const int64_t lo = threadIdx.x * per, hi = lo + per < nt ? lo + per : nt;
    uint32_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += row[i];
    int total = 0;
    uint32_t run = (uint32_t)block_excl_sum<1024>((int)s, tmp, &total);
    for (int64_t i = lo; i < hi; ++i) {
        const uint32_t x = row[i];
        row[i] = run;
        run += x;
    }
    if (threadIdx.x == 0) dtot[blockIdx.x] = (uint32_t)total;
}

// (3) stable scatter of one pass.  Counters: thread t's count of digit d sits
// in the 16-bit half (d >> 6) of logical word (d & 63) * 256 + t; an exclusive
// scan of the words in logical order, plus the low halves' total added to the
// high halves, gives every (digit, thread) its first rank in the tile.
__global__ void __launch_bounds__(SNT, 3) ss_scatter_kernel(const uint32_t* __restrict__ kin,
                                                         const uint32_t* __restrict__ vin,
                                                         uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                         const int64_t* n_dev, int64_t cap, int shift,
                                                         const uint32_t* __restrict__ hist,
                                                         const uint32_t* __restrict__ dtot, const int* gate)
{
    extern __shared__ __align__(16) uint32_t sm[];          // CPHYS counter words, then the staged tile
    __shared__ uint32_t gbase[SRAD];
    __shared__ uint32_t dpre[SRAD];                         // pairs of all tiles with a smaller digit
    __shared__ int tmp[SNT / 32 + 1];
    if (gated(gate)) return;
    const int64_t n = set_count(n_dev, cap);
    const int64_t nt = (n + ST - 1) / ST;
    const int t = threadIdx.x;
    {
        const int x = t < SRAD ? (int)dtot[t] : 0;
        const int e = block_excl_sum<SNT>(x, tmp, nullptr);
        if (t < SRAD) dpre[t] = (uint32_t)e;
    }
    for (int64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const int64_t b = tile * ST;
        const int m = (int)(n - b < ST ? n - b : ST);
        uint32_t k[SE], v[SE], r[SE];           // r: rank among the thread's own digit, then in the tile
        load_blocked(kin, b, m, k, NOKEY);
        load_blocked(vin, b, m, v, 0u);
        for (int i = t; i < CPHYS / 4; i += SNT) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
        __syncthreads();
#pragma unroll
        for (int u = 0; u < SE; ++u) {
            if (k[u] == NOKEY) continue;
            const uint32_t d = (k[u] >> shift) & (SRAD - 1);
            const int p = cphys((int)(d & (CROWS - 1)) * SNT + t);
            const uint32_t sh = (d >> 6) * 16;
            r[u] = (sm[p] >> sh) & 0xFFFFu;
            sm[p] += 1u << sh;
        }
        __syncthreads();
        // thread t scans logical words [64 t, 64 t + 64): physical 65 t + i
        uint32_t s = 0;
#pragma unroll 8
        for (int i = 0; i < 64; ++i) s += sm[65 * t + i];
        int total = 0;
        uint32_t run = (uint32_t)block_excl_sum<SNT>((int)s, tmp, &total);
#pragma unroll 8
        for (int i = 0; i < 64; ++i) {
            const uint32_t x = sm[65 * t + i];
            sm[65 * t + i] = run;
            run += x;
        }
        const uint32_t low_total = (uint32_t)total & 0xFFFFu;       // pairs with digits 0..63
        __syncthreads();
#pragma unroll
        for (int u = 0; u < SE; ++u) {
            if (k[u] == NOKEY) continue;
            const uint32_t d = (k[u] >> shift) & (SRAD - 1);
            const int p = cphys((int)(d & (CROWS - 1)) * SNT + t);
            const uint32_t sh = (d >> 6) * 16;
            r[u] += ((sm[p] >> sh) & 0xFFFFu) + (sh ? low_total : 0u);
        }
        if (t < SRAD) {
            const uint32_t d = (uint32_t)t;
            const int p = cphys((int)(d & (CROWS - 1)) * SNT);
            const uint32_t sh = (d >> 6) * 16;
            const uint32_t dstart = ((sm[p] >> sh) & 0xFFFFu) + (sh ? low_total : 0u);
            gbase[t] = dpre[t] + hist[(int64_t)t * nt + tile] - dstart;
        }
        __syncthreads();
        uint32_t* sk = sm;
        uint32_t* sv = sm + ST;
#pragma unroll
        for (int u = 0; u < SE; ++u) {
            if (k[u] == NOKEY) continue;
            sk[r[u]] = k[u];
            sv[r[u]] = v[u];
        }
        __syncthreads();
        for (int i = t; i < m; i += SNT) {
            const uint32_t kk = sk[i];
            const uint32_t o = gbase[(kk >> shift) & (SRAD - 1)] + (uint32_t)i;
            kout[o] = kk;
            vout[o] = sv[i];
        }
        __syncthreads();
    }
}

struct SegTables {
    uint8_t comp[MAX_ELEMS * MAX_ELEMS];
    uint8_t app[MAX_ELEMS * 8];
    uint8_t elem[16];               // element of each 4-bit code (identity for GT and bad bytes)
    uint8_t id;
};

__device__ __forceinline__ void load_seg_tables(SegTables& S, const Tables& tab)
{
    for (int i = threadIdx.x; i < MAX_ELEMS * MAX_ELEMS; i += blockDim.x) S.comp[i] = tab.comp[i];
    for (int i = threadIdx.x; i < MAX_ELEMS * 8; i += blockDim.x) S.app[i] = tab.app[i];
    if (threadIdx.x < 16) {
        const uint32_t m = tab.elem_of[byte_of(threadIdx.x)];
        S.elem[threadIdx.x] = (uint8_t)(m < MAX_ELEMS ? m : tab.identity);
    }
    if (threadIdx.x == 0) S.id = tab.identity;
}

// Exclusive segmented scan over the CTA's threads of one value each; returns
// this thread's exclusive value and (in *all) the CTA's inclusive total.
__device__ __forceinline__ uint32_t seg_block_excl(uint32_t x, uint32_t ident, const uint8_t* comp, uint32_t* wtot,
                                                   uint32_t* all)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int NW = SNT / 32;
    uint32_t incl = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl = seg_combine(y, incl, comp);
    }
    uint32_t ex = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) ex = ident;
    if (lane == 31) wtot[warp] = incl;
    __syncthreads();
    uint32_t pre = ident;
    for (int w = 0; w < warp; ++w) pre = seg_combine(pre, wtot[w], comp);
    if (all) {
        uint32_t a = ident;
        for (int w = 0; w < NW; ++w) a = seg_combine(a, wtot[w], comp);
        *all = a;
    }
    __syncthreads();
    return seg_combine(pre, ex, comp);
}

struct SegParams {
    const uint32_t* key;        // sorted
    const uint32_t* val;
    const int64_t* n_dev;
    int64_t cap;
    const int* gate;
    const uint32_t* pos;        // nullable: set index -> position (identity when null)
    const uint8_t* init;        // nullable: all (V,I)
    uint8_t* step;
    uint8_t* fin;
    int32_t* vff;
    int64_t* ff;
    int64_t offset;
    uint32_t* tstat;            // [n_tiles] published scan value of each tile (zeroed before)
    uint32_t* tile_counter;     // tiles claimed so far (zeroed before)
    int* err;
    uint32_t* bm;               // nullable: stuck bitmap, bits set for variables that end F
    Tables tab;
};

// Per thread: its 16 sorted pairs, run starts and the fold of its pairs.
struct ThreadRun {
    uint32_t k[SE], v[SE];
    uint32_t heads;             // bit u: pair u starts a variable's run
    uint32_t agg;
};

__device__ __forceinline__ void thread_run(const SegParams& p, const SegTables& S, int64_t n, int64_t b, int m,
                                           ThreadRun& R)
{
    load_blocked(p.key, b, m, R.k, NOKEY);
    load_blocked(p.val, b, m, R.v, 0u);
    const int64_t i0 = b + threadIdx.x * SE;
    uint32_t prev = (i0 > 0 && i0 - 1 < n) ? p.key[i0 - 1] : NOKEY;
    R.heads = 0;
    uint32_t a = S.id;
#pragma unroll
    for (int u = 0; u < SE; ++u) {
        if (R.k[u] == NOKEY) break;
        const uint32_t e = S.elem[R.v[u] & 15u];
        if (R.k[u] != prev) {
            R.heads |= 1u << u;
            a = 0x100u | e;
        } else {
            a = (a & 0x100u) | S.comp[(a & 31u) * MAX_ELEMS + e];
        }
        prev = R.k[u];
    }
    R.agg = a;
}

// (4) every pair's prefix, applied to its variable's entry status, in one
// pass: CTAs claim tiles in order; a tile publishes its aggregate (the fold of
// its trailing run, and whether a run starts inside), then looks back over the
// earlier tiles' published values until one that covers everything before it
// (an inclusive value, or an aggregate in which a run starts), publishes its
// inclusive value and carries the exclusive one into its leading run.  A
// claimed tile belongs to a running CTA that publishes its aggregate before it
// waits on anything, so every look-back ends; the wait is bounded all the same
// (AMC_E_TIMEOUT).
constexpr uint32_t TS_AGG = 1u << 30, TS_INCL = 2u << 30, TS_FLAGS = 3u << 30, TS_VAL = 0x1FFu;

__global__ void __launch_bounds__(SNT) ss_seg_kernel(const SegParams p)
{
    __shared__ SegTables S;
    __shared__ uint32_t wtot[SNT / 32];
    __shared__ uint32_t s_tile, s_carry;
    if (gated(p.gate)) return;
    load_seg_tables(S, p.tab);
    __syncthreads();
    const int64_t n = set_count(p.n_dev, p.cap);
    const int64_t nt = (n + ST - 1) / ST;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(p.tile_counter, 1u);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= nt) break;
        const int64_t b = tile * ST;
        const int m = (int)(n - b < ST ? n - b : ST);
        ThreadRun R;
        thread_run(p, S, n, b, m, R);
        uint32_t all;
        const uint32_t ex = seg_block_excl(R.agg, S.id, S.comp, wtot, &all);
        if (threadIdx.x == 0) {
            uint32_t carry = S.id;
            if (tile == 0) {
                st_release(p.tstat, TS_INCL | (all & TS_VAL));
            } else {
                st_release(p.tstat + tile, TS_AGG | (all & TS_VAL));
                uint32_t prefix = S.id;                   // over tiles [t2, tile), earlier ones folded in front
                for (int64_t t2 = tile - 1; t2 >= 0; --t2) {
                    uint32_t v = 0;
                    for (uint32_t it = 0; it < (1u << 24); ++it) {
                        v = ld_acquire(p.tstat + t2);
                        if (v & TS_FLAGS) break;
                    }
                    if (!(v & TS_FLAGS)) {
                        if (p.err) raise_error(p.err, AMC_E_TIMEOUT);
                        break;
                    }
                    prefix = seg_combine(v & TS_VAL, prefix, S.comp);
                    if ((v & TS_INCL) || (v & 0x100u)) break;
                }
                st_release(p.tstat + tile, TS_INCL | (seg_combine(prefix, all, S.comp) & TS_VAL));
                if (p.key[b - 1] == p.key[b]) carry = prefix & 31u;
            }
            s_carry = carry;
        }
        __syncthreads();
        const uint32_t c = s_carry;
        uint32_t run = (ex & 0x100u) ? (ex & 31u) : S.comp[c * MAX_ELEMS + (ex & 31u)];
        const int64_t i0 = b + threadIdx.x * SE;
        const uint32_t after = (i0 + SE < n) ? p.key[i0 + SE] : NOKEY;
#pragma unroll
        for (int u = 0; u < SE; ++u) {
            const uint32_t kv = R.k[u];
            if (kv == NOKEY) break;
            const uint32_t e = S.elem[R.v[u] & 15u];
            const uint32_t before = (R.heads >> u) & 1u ? S.id : run;
            run = (R.heads >> u) & 1u ? e : S.comp[run * MAX_ELEMS + e];
            const uint32_t s0 = p.init ? (p.init[kv] & 7u) : (uint32_t)AMC_ST_VI;
            const uint32_t pre = S.app[before * 8 + s0];
            const uint32_t post = S.app[run * 8 + s0];
            const uint32_t j = R.v[u] >> 4;
            if (post != ST_F || pre != ST_F) {
                const int64_t pos = p.pos ? (int64_t)p.pos[j] : (int64_t)j;
                if (post != ST_F) {
                    p.step[pos] = (uint8_t)post;
                } else {
                    const int64_t g = p.offset + pos;
                    p.vff[kv] = (int32_t)g;
                    if ((unsigned long long)g < *reinterpret_cast<volatile unsigned long long*>(p.ff))
                        atomicMin(reinterpret_cast<unsigned long long*>(p.ff), (unsigned long long)g);
                }
            }
            const uint32_t next = u + 1 < SE ? R.k[u + 1] : after;
            if (next != kv) {
                p.fin[kv] = (uint8_t)post;
                if (p.bm && post == ST_F) atomicOr(p.bm + (kv >> 5), 1u << (kv & 31));
            }
        }
        __syncthreads();
    }
}

// Raw ops [0, n) as pairs: checked like the filter checks them (bad bytes,
// ids out of range, GT not followed by its EN), F written at every position,
// pairs (id, i << 4 | code) with bad ids replaced by 0.
__global__ void ss_keys_kernel(const uint8_t* __restrict__ kind_side, const int32_t* __restrict__ var, int64_t n,
                               int64_t n_after, int32_t n_vars, uint32_t* __restrict__ key,
                               uint32_t* __restrict__ val, uint8_t* __restrict__ step, int* err)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t ks = kind_side[i];
        const int32_t v = var[i];
        if ((ks & 0xE0u) || (ks & 15u) > AMC_K_EN) raise_error(err, AMC_E_INVALID);
        uint32_t uv = (uint32_t)v;
        if (v < 0 || v >= n_vars) {
            raise_error(err, AMC_E_RANGE);
            uv = 0;
        }
        if ((ks & 15u) == AMC_K_GT) {
            uint32_t nks = 0xFF;
            int32_t nv = (int32_t)uv;
            if (i + 1 < n_after) {
                nks = kind_side[i + 1];
                nv = var[i + 1];
            }
            if (!((nks & 15) == AMC_K_EN && (nks >> 4) == (ks >> 4) && nv != (int32_t)uv))
                raise_error(err, AMC_E_INVALID);
        }
        key[i] = uv;
        val[i] = (uint32_t)i << 4 | sorted_code_of(ks);
        step[i] = (uint8_t)ST_F;
    }
}

int sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

int key_bits_of(int32_t n_vars)
{
    int kb = 1;
    while (kb < 31 && ((int64_t)1 << kb) < (int64_t)n_vars) ++kb;
    return kb;
}

}  // namespace

size_t sorted_check_scratch_bytes(int64_t cap)
{
    const size_t nt = (size_t)((cap + ST - 1) / ST);
    return align_up(4 * SRAD * nt, 256) + align_up(4 * SRAD, 256) + align_up(4 * nt, 256) + 256;
}

int launch_ss_keys(const uint8_t* kind_side, const int32_t* var, int64_t n, int64_t n_after, int32_t n_vars,
                   uint32_t* key, uint32_t* val, uint8_t* step, int* err, cudaStream_t s)
{
    if (n <= 0) return AMC_OK;
    const int64_t blocks = (n + 255) / 256;
    const int grid = (int)(blocks < (int64_t)sm_count() * 8 ? blocks : (int64_t)sm_count() * 8);
    ss_keys_kernel<<<grid, 256, 0, s>>>(kind_side, var, n, n_after, n_vars, key, val, step, err);
    return cudaGetLastError() == cudaSuccess ? AMC_OK : AMC_E_CUDA;
}

int ss_radix_passes(int32_t n_vars) { return (key_bits_of(n_vars) + SDIG - 1) / SDIG; }

int launch_ss_radix(uint32_t* const key[2], uint32_t* const val[2], const int64_t* n_dev, int64_t cap,
                    int32_t n_vars, void* scratch, const int* gate, cudaStream_t s, int* passes_out)
{
    static bool attr_done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    const size_t smem = (size_t)CPHYS * 4;
    static_assert(CPHYS >= 2 * ST, "the staged tile reuses the counter words");
    if (dev >= 64 || !attr_done[dev]) {
        if (cudaFuncSetAttribute(ss_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return AMC_E_CUDA;
        if (dev < 64) attr_done[dev] = true;
    }
    const int n_sm = sm_count();
    const int64_t tiles = (cap + ST - 1) / ST;
    auto grid = [&](int per_sm) { return (int)(tiles < (int64_t)n_sm * per_sm ? tiles : (int64_t)n_sm * per_sm); };
    uint8_t* w = static_cast<uint8_t*>(scratch);
    uint32_t* hist = reinterpret_cast<uint32_t*>(w);
    w += align_up(4 * SRAD * (size_t)tiles, 256);
    uint32_t* dtot = reinterpret_cast<uint32_t*>(w);
    const int kb = key_bits_of(n_vars);
    const int passes = (kb + SDIG - 1) / SDIG;
    for (int ps = 0; ps < passes; ++ps) {
        const int src = ps & 1;
        const int shift = ps * SDIG;
        ss_hist_kernel<<<grid(8), SNT, 0, s>>>(key[src], n_dev, cap, shift, hist, gate);
        ss_hscan_kernel<<<SRAD, 1024, 0, s>>>(hist, dtot, n_dev, cap, gate);
        ss_scatter_kernel<<<grid(3), SNT, smem, s>>>(key[src], val[src], key[src ^ 1], val[src ^ 1], n_dev, cap, shift,
                                                     hist, dtot, gate);
        if (cudaGetLastError() != cudaSuccess) return AMC_E_CUDA;
    }
    *passes_out = passes;
    return AMC_OK;
}

int launch_sorted_check(const SortedCheck& C, cudaStream_t s)
{
    if (C.cap <= 0) return AMC_OK;
    if (C.cap > ((int64_t)1 << 28)) return AMC_E_INVALID;        // set index << 4 must fit 32 bits
    const int n_sm = sm_count();
    const int64_t tiles = (C.cap + ST - 1) / ST;
    auto grid = [&](int per_sm) { return (int)(tiles < (int64_t)n_sm * per_sm ? tiles : (int64_t)n_sm * per_sm); };
    uint8_t* w = static_cast<uint8_t*>(C.scratch);
    uint32_t* hist = reinterpret_cast<uint32_t*>(w);
    w += align_up(4 * SRAD * (size_t)tiles, 256);
    uint32_t* dtot = reinterpret_cast<uint32_t*>(w);
    w += align_up(4 * SRAD, 256);
    uint32_t* tstat = reinterpret_cast<uint32_t*>(w);
    w += align_up(4 * (size_t)tiles, 256);
    uint32_t* tile_counter = reinterpret_cast<uint32_t*>(w);

    int passes = 0;
    const int rc = launch_ss_radix(C.key, C.val, C.n_dev, C.cap, C.n_vars, C.scratch, C.gate, s, &passes);
    if (rc) return rc;
    SegParams p;
    p.key = C.key[passes & 1];
    p.val = C.val[passes & 1];
    p.n_dev = C.n_dev;
    p.cap = C.cap;
    p.gate = C.gate;
    p.pos = C.pos;
    p.init = C.init;
    p.step = C.step;
    p.fin = C.fin;
    p.vff = C.vff;
    p.ff = C.ff;
    p.offset = C.offset;
    p.tstat = tstat;
    p.tile_counter = tile_counter;
    p.err = C.err;
    p.bm = C.bm;
    p.tab = host_tables();
    if (cudaMemsetAsync(tstat, 0, 4 * (size_t)tiles, s) != cudaSuccess) return AMC_E_CUDA;
    if (cudaMemsetAsync(tile_counter, 0, 4, s) != cudaSuccess) return AMC_E_CUDA;
    ss_seg_kernel<<<grid(8), SNT, 0, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? AMC_OK : AMC_E_CUDA;
}

}  // namespace amc
