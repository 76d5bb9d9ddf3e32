// scan_sorted.cu -- a set of ops checked by grouping it by variable: a stable
// radix sort of (variable, index) pairs, then a segmented scan of the transfer
// functions over each variable's run; or, for a set whose ops spread over the
// variable ids, one radix pass into buckets checked one CTA each.
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
//      2,048 pairs, an exclusive scan of each digit's row over the tiles (one
//      CTA per digit; the digits' totals are scanned by every scatter CTA),
//      and a stable scatter (ranks within each warp from one ballot per digit
//      bit, per-warp digit counters, the tile staged in shared memory in
//      digit order);
//   3. segmented scan over the sorted pairs as reduce / carry / apply over the
//      tiles, every op's prefix applied to its variable's entry status.
// The bucket check (5) replaces 2-3 by one radix pass on the low seven bits
// of the id and one CTA per bucket.
// Outputs: the status of every op whose status is not F (the caller has
// written F at every position of the set), the first fault of each variable
// that faults in the set, the global first fault, and the final statuses.
#include <cstdio>

#include "amc_internal.cuh"
#include "scan_trace.cuh"

namespace amc {

namespace {

constexpr int ST = 2048;                 // pairs per tile
constexpr int SNT = 256;                 // threads per CTA
constexpr int SE = ST / SNT;             // pairs per thread (blocked)
constexpr int SDIG = 7;                  // digit bits
constexpr int SRAD = 1 << SDIG;
constexpr uint32_t NOKEY = 0xFFFFFFFFu;  // no variable id equals it


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

// (3) stable scatter of one pass, ranked warp by warp: warp w holds pairs
// [256 w, 256 w + 256) of the tile, lane L pair 256 w + 32 r + L in round r
// (loads coalesce).  In each round the lanes with equal digits find each
// other (one ballot per digit bit); the lowest of them adds the group's size
// to the warp's counter of that digit, and each lane's rank within the warp
// is the counter's old value plus the group's lanes below it.  Ranks follow
// (warp, round, lane), i.e. the pairs' order in the tile, so the pass is
// stable.  Per digit an exclusive sum over the warps' counters and over the
// digits' tile totals turns warp ranks into tile ranks; the tile is staged in
// shared memory in digit order, so the stores of each digit's run coalesce.
constexpr int SCT = 256;                       // scatter threads per CTA
constexpr int SCW = SCT / 32;                  // its warps
constexpr int SWR = ST / SCW / 32;             // rounds per warp (8)

__global__ void __launch_bounds__(SCT, 5) ss_scatter_kernel(const uint32_t* __restrict__ kin,
                                                         const uint32_t* __restrict__ vin,
                                                         uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                         const int64_t* n_dev, int64_t cap, int shift,
                                                         const uint32_t* __restrict__ hist,
                                                         const uint32_t* __restrict__ dtot, const int* gate)
{
    __shared__ __align__(16) uint32_t sk[ST];
    __shared__ __align__(16) uint32_t sv[ST];
    __shared__ uint32_t wcnt[SCW][SRAD];                    // per-warp digit counters, then their prefixes
    __shared__ uint32_t gbase[SRAD];
    __shared__ uint32_t dpre[SRAD];                         // pairs of all tiles with a smaller digit
    __shared__ uint32_t dstart[SRAD];                       // first rank of each digit in the tile
    __shared__ int tmp[SCT / 32 + 1];
    if (gated(gate)) return;
    const int64_t n = set_count(n_dev, cap);
    const int64_t nt = (n + ST - 1) / ST;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t lt = lanemask_lt();
    {
        const int x = t < SRAD ? (int)dtot[t] : 0;
        const int e = block_excl_sum<SCT>(x, tmp, nullptr);
        if (t < SRAD) dpre[t] = (uint32_t)e;
    }
    for (int64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const int64_t b = tile * ST;
        const int m = (int)(n - b < ST ? n - b : ST);
        // the tile's first pair of each digit among all tiles: its row entry (loaded early)
        const uint32_t hrow = t < SRAD ? hist[(int64_t)t * nt + tile] : 0u;
        uint32_t k[SWR], r[SWR];
        const int w0 = warp * (ST / SCW);
#pragma unroll
        for (int u = 0; u < SWR; ++u) {
            const int i = w0 + 32 * u + lane;
            const bool ok = i < m;
            k[u] = ok ? kin[b + i] : NOKEY;
            sv[i] = ok ? vin[b + i] : 0u;                   // values wait in shared memory
        }
        for (int i = t; i < SCW * SRAD; i += SCT) (&wcnt[0][0])[i] = 0;
        __syncthreads();
#pragma unroll
        for (int u = 0; u < SWR; ++u) {
            const bool ok = k[u] != NOKEY;
            const uint32_t d = (k[u] >> shift) & (SRAD - 1);
            const uint32_t valid = __ballot_sync(0xffffffffu, ok);
            uint32_t peers = ok ? valid : ~valid;
#pragma unroll
            for (int bit = 0; bit < SDIG; ++bit) {
                const uint32_t bal = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
                peers &= ((d >> bit) & 1u) ? bal : ~bal;
            }
            const int lead = __ffs(peers) - 1;
            uint32_t old = 0;
            if (ok && lane == lead) {
                old = wcnt[warp][d];
                wcnt[warp][d] = old + (uint32_t)__popc(peers);
            }
            old = __shfl_sync(0xffffffffu, old, lead);
            r[u] = old + (uint32_t)__popc(peers & lt);
        }
        __syncthreads();
        uint32_t cnt = 0;
        if (t < SRAD) {
#pragma unroll
            for (int w = 0; w < SCW; ++w) {
                const uint32_t x = wcnt[w][t];
                wcnt[w][t] = cnt;
                cnt += x;
            }
        }
        const uint32_t ds = (uint32_t)block_excl_sum<SCT>((int)cnt, tmp, nullptr);
        if (t < SRAD) {
            dstart[t] = ds;
            gbase[t] = dpre[t] + hrow - ds;
        }
        uint32_t v[SWR];
#pragma unroll
        for (int u = 0; u < SWR; ++u) v[u] = sv[w0 + 32 * u + lane];
        __syncthreads();
#pragma unroll
        for (int u = 0; u < SWR; ++u) {
            if (k[u] == NOKEY) continue;
            const uint32_t d = (k[u] >> shift) & (SRAD - 1);
            const uint32_t rr = r[u] + wcnt[warp][d] + dstart[d];
            sk[rr] = k[u];
            sv[rr] = v[u];
        }
        __syncthreads();
        for (int i = t; i < m; i += SCT) {
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
    uint32_t* tstat;            // [n_tiles] each tile's scan value, then the value before it
    int* err;
    uint32_t* bm;               // nullable: stuck bitmap, bits set for variables that end F
    Tables tab;
};

constexpr uint32_t TS_VAL = 0x1FFu;      // a scan value: element (bits 0-4), "a run starts inside" (bit 8)

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

// (4) every pair's prefix, applied to its variable's entry status, as
// reduce / carry / apply over the sorted tiles (no CTA waits on another):
//   (a) each tile's value: the fold of its trailing run, bit 8 set when a run
//       starts inside (what a later tile needs from it);
//   (b) one CTA folds the tile values into exclusive prefixes in place (the
//       value of everything before the tile: the fold of the run that the
//       tile's first pair may continue);
//   (c) each tile carries that prefix into its leading run (when the run
//       continues across the boundary) and composes every pair's prefix;
//       each pair's entry status and output position are loaded before the
//       tile's scan so that their latency overlaps it.
__global__ void __launch_bounds__(SNT, 6) ss_red_kernel(const SegParams p)
{
    __shared__ SegTables S;
    __shared__ uint32_t wtot[SNT / 32];
    if (gated(p.gate)) return;
    load_seg_tables(S, p.tab);
    __syncthreads();
    const int64_t n = set_count(p.n_dev, p.cap);
    const int64_t nt = (n + ST - 1) / ST;
    for (int64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const int64_t b = tile * ST;
        const int m = (int)(n - b < ST ? n - b : ST);
        ThreadRun R;
        thread_run(p, S, n, b, m, R);
        uint32_t all;
        seg_block_excl(R.agg, S.id, S.comp, wtot, &all);
        if (threadIdx.x == 0) p.tstat[tile] = all & TS_VAL;
    }
}

constexpr int CNT = 1024;                  // threads of the carry CTA

__global__ void __launch_bounds__(CNT) ss_carry_kernel(const SegParams p)
{
    __shared__ uint8_t comp[MAX_ELEMS * MAX_ELEMS];
    __shared__ uint32_t wtot[CNT / 32];
    __shared__ uint8_t s_id;
    if (gated(p.gate)) return;
    for (int i = threadIdx.x; i < MAX_ELEMS * MAX_ELEMS; i += CNT) comp[i] = p.tab.comp[i];
    if (threadIdx.x == 0) s_id = p.tab.identity;
    __syncthreads();
    const uint32_t id = s_id;
    const int64_t n = set_count(p.n_dev, p.cap);
    const int64_t nt = (n + ST - 1) / ST;
    const int64_t per = (nt + CNT - 1) / CNT;
    const int64_t lo = threadIdx.x * per, hi = lo + per < nt ? lo + per : nt;
    uint32_t a = id;
    for (int64_t i = lo; i < hi; ++i) a = seg_combine(a, p.tstat[i], comp);
    // exclusive segmented scan of the threads' folds
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = a;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl = seg_combine(y, incl, comp);
    }
    uint32_t ex = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) ex = id;
    if (lane == 31) wtot[warp] = incl;
    __syncthreads();
    uint32_t pre = id;
    for (int w = 0; w < warp; ++w) pre = seg_combine(pre, wtot[w], comp);
    uint32_t run = seg_combine(pre, ex, comp);
    for (int64_t i = lo; i < hi; ++i) {
        const uint32_t x = p.tstat[i];
        p.tstat[i] = run;
        run = seg_combine(run, x, comp);
    }
}

__global__ void __launch_bounds__(SNT, 4) ss_apply_kernel(const SegParams p)
{
    __shared__ SegTables S;
    __shared__ uint32_t wtot[SNT / 32];
    if (gated(p.gate)) return;
    load_seg_tables(S, p.tab);
    __syncthreads();
    const int64_t n = set_count(p.n_dev, p.cap);
    const int64_t nt = (n + ST - 1) / ST;
    const uint8_t* __restrict__ init = p.init;
    const uint32_t* __restrict__ posm = p.pos;
    for (int64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const int64_t b = tile * ST;
        const int m = (int)(n - b < ST ? n - b : ST);
        const uint32_t before_tile = p.tstat[tile];
        const bool cont = tile > 0 && p.key[b - 1] == p.key[b];
        ThreadRun R;
        thread_run(p, S, n, b, m, R);
        // entry statuses (3 bits each, packed) and positions of the thread's pairs
        uint32_t s0lo = 0, s0hi = 0;
        uint32_t posv[SE];
#pragma unroll
        for (int u = 0; u < SE; ++u) {
            const bool ok = R.k[u] != NOKEY;
            const uint32_t s0 = (init && ok) ? (init[R.k[u]] & 7u) : (uint32_t)AMC_ST_VI;
            if (u < 8) s0lo |= s0 << (3 * u);
            else s0hi |= s0 << (3 * (u - 8));
            const uint32_t j = R.v[u] >> 4;
            posv[u] = (posm && ok) ? posm[j] : j;
        }
        const uint32_t ex = seg_block_excl(R.agg, S.id, S.comp, wtot, nullptr);
        const uint32_t c = cont ? (before_tile & 31u) : S.id;
        uint32_t run = (ex & 0x100u) ? (ex & 31u) : S.comp[c * MAX_ELEMS + (ex & 31u)];
        const int64_t i0 = b + threadIdx.x * SE;
        const uint32_t after = (i0 + SE < n) ? p.key[i0 + SE] : NOKEY;
        unsigned long long gmin = ~0ull;
#pragma unroll
        for (int u = 0; u < SE; ++u) {
            const uint32_t kv = R.k[u];
            if (kv == NOKEY) break;
            const uint32_t e = S.elem[R.v[u] & 15u];
            const uint32_t before = (R.heads >> u) & 1u ? S.id : run;
            run = (R.heads >> u) & 1u ? e : S.comp[run * MAX_ELEMS + e];
            const uint32_t s0 = ((u < 8 ? s0lo : s0hi) >> (3 * (u & 7))) & 7u;
            const uint32_t pre = S.app[before * 8 + s0];
            const uint32_t post = S.app[run * 8 + s0];
            if (post != ST_F || pre != ST_F) {
                const int64_t pos = (int64_t)posv[u];
                if (post != ST_F) {
                    p.step[pos] = (uint8_t)post;
                } else {
                    const int64_t g = p.offset + pos;
                    p.vff[kv] = (int32_t)g;
                    if ((unsigned long long)g < gmin) gmin = (unsigned long long)g;
                }
            }
            const uint32_t next = u + 1 < SE ? R.k[u + 1] : after;
            if (next != kv) {
                p.fin[kv] = (uint8_t)post;
                if (p.bm && post == ST_F) atomicOr(p.bm + (kv >> 5), 1u << (kv & 31));
            }
        }
        // the warp's smallest first fault, one atomic per warp
#pragma unroll
        for (int d = 16; d; d >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, gmin, d);
            if (o < gmin) gmin = o;
        }
        if ((threadIdx.x & 31) == 0 && gmin != ~0ull) atomicMin(reinterpret_cast<unsigned long long*>(p.ff), gmin);
        __syncthreads();
    }
}

// (5) A set over many variables whose ops spread over the variable ids (an
// epoch's candidates), checked per bucket: one stable radix pass on the low
// seven bits of the id groups the pairs into 128 buckets (bucket b: the ids
// v with v mod 128 = b, strided over the whole id range, so hot and cold ids
// mix and the buckets come out about equal), each still in position order;
// then one CTA per bucket does the whole check of its bucket, as a reduce /
// carry / apply over its warps' stretches (no CTA waits on another):
//   (a) warp w folds its stretch of the bucket, 32 pairs at a time, into one
//       function per variable of the bucket (a row of ceil(n_vars / 128)
//       bytes in shared memory, indexed by v / 128): when the batch's
//       variables are distinct (a bit per variable in shared memory tells)
//       each lane composes its own, else lanes with the same variable are
//       grouped (match.any) and the group's first lane composes them in order;
//   (b) a thread per variable carries the entry status through the warps'
//       functions: every stretch's entry statuses, and the final status (and
//       stuck bit) of a variable whose status changed;
//   (c) each warp re-runs its stretch from those entry statuses, writing the
//       statuses that are not F (the caller wrote F everywhere) and the first
//       faults.
constexpr int BKW = 16;                   // warps of a bucket CTA
constexpr int BK_MAX_W = 8192;            // variables per bucket (n_vars <= 2^20): 128 KB of rows
constexpr int BKU = 16;                   // batches of 32 pairs loaded at once
constexpr uint32_t BK_ABSENT = 0xFF;      // row byte of a variable with no pair in the stretch

// row bytes per bucket: one per id b, b + 128, ... below n_vars, padded to 16
__host__ __device__ __forceinline__ int bucket_width(int32_t n_vars)
{
    return (int)((((int64_t)n_vars + SRAD - 1) / SRAD + 15) & ~(int64_t)15);
}

struct BucketParams {
    const uint32_t* key;        // grouped by bucket, position order inside
    const uint32_t* val;
    const int64_t* n_dev;
    int64_t cap;
    const int* gate;
    const uint32_t* dtot;       // pairs per bucket
    int32_t n_vars;
    const uint32_t* pos;        // set index -> position in the epoch
    const uint8_t* init;        // nullable: all (V,I)
    uint8_t* step;
    uint8_t* fin;
    int32_t* vff;
    int64_t* ff;
    int64_t offset;
    uint32_t* bm;               // nullable: stuck bitmap, bits set for variables that become F
    Tables tab;
};

// Duplicate test of a batch without match.any (slow on this part): each lane
// sets its variable's bit in the warp's bitmap; a bit already set means that
// an earlier lane of the batch has the same variable.  The bits are cleared
// after the batch.
__device__ __forceinline__ bool seen_before(uint32_t* seen, uint32_t lv)
{
    const uint32_t bit = 1u << (lv & 31);
    return (atomicOr(seen + (lv >> 5), bit) & bit) != 0;
}
__device__ __forceinline__ void forget(uint32_t* seen, uint32_t lv) { atomicAnd(seen + (lv >> 5), ~(1u << (lv & 31))); }

__global__ void __launch_bounds__(BKW * 32, 1) ss_bucket_kernel(const BucketParams p)
{
    extern __shared__ __align__(16) uint8_t rows[];        // [BKW][W], then seen bits [BKW][W / 32]
    __shared__ uint8_t comp[MAX_ELEMS * MAX_ELEMS];
    __shared__ uint8_t app[MAX_ELEMS * 8];
    __shared__ uint8_t elem[16];
    __shared__ uint8_t mb[BKW][32];
    __shared__ uint32_t bstart[SRAD];
    __shared__ int tmp[BKW + 1];
    if (gated(p.gate)) return;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t lt = lanemask_lt();
    for (int i = tid; i < MAX_ELEMS * MAX_ELEMS; i += BKW * 32) comp[i] = p.tab.comp[i];
    for (int i = tid; i < MAX_ELEMS * 8; i += BKW * 32) app[i] = p.tab.app[i];
    if (tid < 16) {
        const uint32_t m = p.tab.elem_of[byte_of(tid)];
        elem[tid] = (uint8_t)(m < MAX_ELEMS ? m : p.tab.identity);
    }
    {
        const int x = tid < SRAD ? (int)p.dtot[tid] : 0;
        const int e = block_excl_sum<BKW * 32>(x, tmp, nullptr);
        if (tid < SRAD) bstart[tid] = (uint32_t)e;
    }
    const uint32_t ID = p.tab.identity;
    const int W = bucket_width(p.n_vars);
    const int64_t n = set_count(p.n_dev, p.cap);
    uint32_t* const seen_all = reinterpret_cast<uint32_t*>(rows + (size_t)BKW * W);
    const int WS = (W + 31) >> 5;
    uint32_t* const seen = seen_all + w * WS;             // this warp's bits
    for (int i = tid; i < BKW * WS; i += BKW * 32) seen_all[i] = 0;
    __syncthreads();
    for (int b = blockIdx.x; b < SRAD; b += gridDim.x) {
        const int nv = (int)(((int64_t)p.n_vars - b + SRAD - 1) / SRAD);   // ids b, b + 128, ... below n_vars
        const int lo_b = (int)bstart[b];
        const int hi_b = (int)min(n, (int64_t)lo_b + (int64_t)p.dtot[b]);
        const int per = (hi_b - lo_b + BKW - 1) / BKW;
        const int lo = min(hi_b, lo_b + w * per), hi = min(hi_b, lo + per);
        uint8_t* row = rows + (size_t)w * W;
        // rows start as "absent" (no pair of the variable in the stretch yet)
        for (int v = lane; v < W / 16; v += 32) reinterpret_cast<uint4*>(row)[v] = make_uint4(~0u, ~0u, ~0u, ~0u);
        __syncwarp();
        // (a) fold the stretch per variable; BKU batches of 32 pairs are
        // loaded at once (their loads overlap), then folded one by one
        for (int g0 = lo; g0 < hi; g0 += 32 * BKU) {
            uint32_t kk[BKU], vv[BKU];
#pragma unroll
            for (int u = 0; u < BKU; ++u) {
                const int i = g0 + 32 * u + lane;
                kk[u] = i < hi ? p.key[i] >> SDIG : 0xFFFFFFFFu;
                vv[u] = i < hi ? p.val[i] : 0u;
            }
#pragma unroll
            for (int u = 0; u < BKU; ++u) {
                if (g0 + 32 * u >= hi) break;
                const uint32_t lv = kk[u];
                const bool ok = lv != 0xFFFFFFFFu;
                const uint32_t m = ok ? elem[vv[u] & 15u] : ID;
                if (!__ballot_sync(0xffffffffu, ok && seen_before(seen, lv))) {
                    // every variable once in the batch: each lane composes alone
                    if (ok) {
                        const uint32_t r = row[lv];
                        row[lv] = r == BK_ABSENT ? (uint8_t)m : comp[r * MAX_ELEMS + m];
                    }
                } else {
                    mb[w][lane] = (uint8_t)m;
                    const uint32_t peers = __match_any_sync(0xffffffffu, lv);
                    __syncwarp();
                    if (ok && lane == __ffs(peers) - 1) {
                        uint32_t acc = row[lv];
                        if (acc == BK_ABSENT) acc = ID;
                        for (uint32_t r = peers; r; r &= r - 1) acc = comp[acc * MAX_ELEMS + mb[w][__ffs(r) - 1]];
                        row[lv] = (uint8_t)acc;
                    }
                }
                if (ok) forget(seen, lv);
                __syncwarp();
            }
        }
        __syncthreads();
        // (b) carry, four variables per step: entry statuses of every
        // stretch; final statuses and stuck bits of the variables whose status
        // changed (the others keep theirs).  Four variables that no stretch
        // touches ("absent" in every row) are skipped.
        for (int l4 = tid; l4 < (nv + 3) / 4; l4 += BKW * 32) {
            uint32_t e4[BKW];
            uint32_t all = ~0u;
#pragma unroll
            for (int k = 0; k < BKW; ++k) {
                e4[k] = reinterpret_cast<const uint32_t*>(rows + (size_t)k * W)[l4];
                all &= e4[k];
            }
            if (all == ~0u) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int lv = 4 * l4 + j;
                if (lv >= nv) break;
                const int64_t v = (int64_t)lv * SRAD + b;
                const uint32_t s0 = p.init ? (uint32_t)(p.init[v] & 7u) : (uint32_t)AMC_ST_VI;
                uint32_t st = s0;
#pragma unroll
                for (int k = 0; k < BKW; ++k) {
                    const uint32_t e = (e4[k] >> (8 * j)) & 0xFFu;
                    rows[(size_t)k * W + lv] = (uint8_t)st;
                    if (e != BK_ABSENT) st = app[e * 8 + st];
                }
                if (st != s0) {
                    p.fin[v] = (uint8_t)st;
                    if (p.bm && st == ST_F) atomicOr(p.bm + (v >> 5), 1u << (v & 31));
                }
            }
        }
        __syncthreads();
        // (c) every pair's status from its stretch's entry statuses
        unsigned long long gmin = ~0ull;
        for (int g0 = lo; g0 < hi; g0 += 32 * BKU) {
            uint32_t kk[BKU], vv[BKU], pp[BKU];
#pragma unroll
            for (int u = 0; u < BKU; ++u) {
                const int i = g0 + 32 * u + lane;
                kk[u] = i < hi ? p.key[i] >> SDIG : 0xFFFFFFFFu;
                vv[u] = i < hi ? p.val[i] : 0u;
            }
#pragma unroll
            for (int u = 0; u < BKU; ++u) pp[u] = kk[u] != 0xFFFFFFFFu ? p.pos[vv[u] >> 4] : 0u;
#pragma unroll
            for (int u = 0; u < BKU; ++u) {
                if (g0 + 32 * u >= hi) break;
                const uint32_t lv = kk[u];
                const bool ok = lv != 0xFFFFFFFFu;
                const uint32_t m = ok ? elem[vv[u] & 15u] : ID;
                const uint32_t posi = pp[u];
                // pre / post: the variable's status before / after the pair
                uint32_t pre = 0, post = 0;
                if (!__ballot_sync(0xffffffffu, ok && seen_before(seen, lv))) {
                    if (ok) {
                        pre = row[lv];
                        post = app[m * 8 + pre];
                        row[lv] = (uint8_t)post;
                    }
                } else {
                    mb[w][lane] = (uint8_t)m;
                    const uint32_t peers = __match_any_sync(0xffffffffu, lv);
                    __syncwarp();
                    const uint32_t cur = ok ? row[lv] : 0u;
                    __syncwarp();
                    if (ok) {
                        uint32_t acc = ID;
                        for (uint32_t r = peers & lt; r; r &= r - 1) acc = comp[acc * MAX_ELEMS + mb[w][__ffs(r) - 1]];
                        pre = app[acc * 8 + cur];
                        post = app[comp[acc * MAX_ELEMS + m] * 8 + cur];
                        if (lane == 31 - __clz(peers)) row[lv] = (uint8_t)post;
                    }
                }
                if (ok) {
                    forget(seen, lv);
                    if (post != ST_F) {
                        p.step[posi] = (uint8_t)post;
                    } else if (pre != ST_F) {
                        const int64_t g = p.offset + (int64_t)posi;
                        p.vff[(int64_t)lv * SRAD + b] = (int32_t)g;
                        if ((unsigned long long)g < gmin) gmin = (unsigned long long)g;
                    }
                }
                __syncwarp();
            }
        }
#pragma unroll
        for (int d = 16; d; d >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, gmin, d);
            if (o < gmin) gmin = o;
        }
        if (lane == 0 && gmin != ~0ull) atomicMin(reinterpret_cast<unsigned long long*>(p.ff), gmin);
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
        ss_scatter_kernel<<<grid(5), SCT, 0, s>>>(key[src], val[src], key[src ^ 1], val[src ^ 1], n_dev, cap, shift,
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
    // scratch: the sort's digit rows and totals, then the tile values
    uint8_t* w = static_cast<uint8_t*>(C.scratch) + align_up(4 * SRAD * (size_t)tiles, 256) + align_up(4 * SRAD, 256);
    uint32_t* tstat = reinterpret_cast<uint32_t*>(w);

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
    p.err = C.err;
    p.bm = C.bm;
    p.tab = host_tables();
    ss_red_kernel<<<grid(6), SNT, 0, s>>>(p);
    ss_carry_kernel<<<1, CNT, 0, s>>>(p);
    ss_apply_kernel<<<grid(4), SNT, 0, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? AMC_OK : AMC_E_CUDA;
}

bool bucket_check_ok(int32_t n_vars) { return n_vars >= 1 && bucket_width(n_vars) <= BK_MAX_W; }

int launch_bucket_check(const SortedCheck& C, cudaStream_t s)
{
    if (C.cap <= 0) return AMC_OK;
    if (C.cap > ((int64_t)1 << 28) || !C.pos || !bucket_check_ok(C.n_vars)) return AMC_E_INVALID;
    const int W = bucket_width(C.n_vars);
    const size_t smem = (size_t)BKW * W + (size_t)BKW * 4 * ((W + 31) / 32);
    static size_t attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 64 || attr_set[dev] < smem) {
        if (cudaFuncSetAttribute(ss_bucket_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return AMC_E_CUDA;
        if (dev < 64) attr_set[dev] = smem;
    }
    const int n_sm = sm_count();
    const int64_t tiles = (C.cap + ST - 1) / ST;
    auto grid = [&](int per_sm) { return (int)(tiles < (int64_t)n_sm * per_sm ? tiles : (int64_t)n_sm * per_sm); };
    uint8_t* w = static_cast<uint8_t*>(C.scratch);
    uint32_t* hist = reinterpret_cast<uint32_t*>(w);
    uint32_t* dtot = reinterpret_cast<uint32_t*>(w + align_up(4 * SRAD * (size_t)tiles, 256));
    ss_hist_kernel<<<grid(8), SNT, 0, s>>>(C.key[0], C.n_dev, C.cap, 0, hist, C.gate);
    ss_hscan_kernel<<<SRAD, 1024, 0, s>>>(hist, dtot, C.n_dev, C.cap, C.gate);
    ss_scatter_kernel<<<grid(5), SCT, 0, s>>>(C.key[0], C.val[0], C.key[1], C.val[1], C.n_dev, C.cap, 0, hist,
                                              dtot, C.gate);
    BucketParams p;
    p.key = C.key[1];
    p.val = C.val[1];
    p.n_dev = C.n_dev;
    p.cap = C.cap;
    p.gate = C.gate;
    p.dtot = dtot;
    p.n_vars = C.n_vars;
    p.pos = C.pos;
    p.init = C.init;
    p.step = C.step;
    p.fin = C.fin;
    p.vff = C.vff;
    p.ff = C.ff;
    p.offset = C.offset;
    p.bm = C.bm;
    p.tab = host_tables();
    ss_bucket_kernel<<<C.n_vars < SRAD ? C.n_vars : SRAD, BKW * 32, smem, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? AMC_OK : AMC_E_CUDA;
}

}  // namespace amc
