// scan_tail.cu -- long traces checked in epochs: stream filter, compacted
// candidates, each set checked grouped by variable.
//
// Section 3.2: F is absorbing, so once a variable's status is F every later
// op on it yields F (Property Progress: a stuck variable stays stuck).  On a
// long trace nearly every op after the first few per variable is such an op.
// The first part of the trace, [0, S), is checked by sorting its ops by
// variable (scan_sorted.cu); the rest is cut into epochs (by default each
// ends at four times its start), and for each epoch
//   1. the statuses at its start are exact (the previous part's final
//      statuses); variables with status F form a bitmap;
//   2. a streaming kernel writes F at every position and collects the ops on
//      variables outside the bitmap ("candidates"), in position order;
//   3. the candidates, a set of ops over the same variables (an op's status
//      depends only on the earlier ops on its variable), are checked from the
//      epoch's start statuses, with their count read from device memory: one
//      radix pass groups them into 128 buckets by the low seven bits of the
//      variable id (position order kept inside a bucket), one CTA checks each
//      bucket (scan_sorted.cu, bucket check); the statuses that are not F go
//      to their positions, first faults to trace positions, final statuses
//      start the next epoch.
// Outputs are identical to one scan over the whole trace.  An epoch whose
// candidates overflow their slots is rechecked whole by the single-pass scan.
#include <cstdio>
#include <cstdlib>

#include "amc_internal.cuh"
#include "scan_trace.cuh"

namespace amc {

namespace {

constexpr int TF_THREADS = 1024;          // filter CTA: one per SM (the bitmap fills shared memory)
constexpr int TF_CHUNK = 4096;            // ops per warp chunk in epochs of 2^27 ops or more,
constexpr int TF_CHUNK_SHORT = 1024;      // in shorter epochs (more warps busy)
constexpr int64_t TF_LONG_CHUNKS_FROM = (int64_t)1 << 27;
constexpr int TF_SLOT_DIV = 4;            // candidate slots per chunk: a quarter (more: the epoch falls back)
constexpr int CAND_DIV = 4;               // candidate capacity: epoch ops / 4 (more: falls back)
constexpr int64_t CAND_MAX = (int64_t)1 << 27;   // and at most 2^27 (set index << 4 fits 32 bits)
constexpr int TF_PER = 16;                // ops per lane and step
constexpr int TAIL_MIN_VARS = 16385;      // fewer variables take the reduce / carry / apply path
constexpr int TAIL_MAX_VARS = 1 << 20;    // bitmap of 128 KB in shared memory
constexpr int DEFAULT_FIRST_LOG2 = 21;    // first part 2^21 ops,
constexpr int DEFAULT_GROW = 2;           // then epochs ending at 4 times their start
constexpr int64_t DEFAULT_MIN_OPS = (int64_t)1 << 29;

struct TailShape {
    int64_t S = 0;        // ops of the first part
    int64_t E = 0;        // ops per epoch (grow == 0)
    int grow = 0;         // > 0: each epoch ends at 2^grow times its start
};

// AMC_SCAN_TAIL="s,e": first part 2^s ops, epochs of 2^e ops; "s,-g": first
// part 2^s ops, each epoch ending at 2^g times its start; for every trace
// longer than 2^s ops (test and tuning override); "0" disables.
// force: -1 by size (from DEFAULT_MIN_OPS ops), 1 for every trace longer than
// 2^21 ops (first part 2^21 ops from 2^23 ops on, else a quarter of the trace),
// 0 never.
bool tail_shape(int64_t n_ops, int32_t n_vars, bool guarded, TailShape& sh, int force)
{
    if (guarded || n_vars < TAIL_MIN_VARS || n_vars > TAIL_MAX_VARS || !bucket_check_ok(n_vars)) return false;
    if (const char* e = getenv("AMC_SCAN_TAIL")) {
        if (e[0] == '0' && e[1] == 0) return false;
        int a = 0, b = 0;
        if (sscanf(e, "%d,%d", &a, &b) == 2 && a >= 12 && a <= 27 && ((b >= 12 && b < 31) || (b >= -4 && b <= -1))) {
            sh.S = (int64_t)1 << a;
            if (n_ops <= sh.S) return false;
            if (b > 0) {
                sh.E = (int64_t)1 << b;
                if (sh.E > n_ops - sh.S) sh.E = n_ops - sh.S;
            } else {
                sh.grow = -b;
            }
            return true;
        }
    }
    if (force == 0) return false;
    if (force == 1 ? n_ops <= ((int64_t)1 << DEFAULT_FIRST_LOG2) : n_ops < DEFAULT_MIN_OPS) return false;
    int lg = DEFAULT_FIRST_LOG2;
    while (lg > 12 && ((int64_t)1 << (lg + 2)) > n_ops) --lg;      // first part at most a quarter
    sh.S = (int64_t)1 << lg;
    sh.grow = DEFAULT_GROW;
    return true;
}

// ops per filter chunk of an epoch of n ops
int chunk_for(int64_t n) { return n < TF_LONG_CHUNKS_FROM ? TF_CHUNK_SHORT : TF_CHUNK; }
int64_t chunks_of(int64_t n) { return (n + chunk_for(n) - 1) / chunk_for(n); }
// candidate slots per chunk: a quarter of it
int slots_for(int64_t n) { return chunk_for(n) / TF_SLOT_DIV; }

int64_t epoch_end(const TailShape& sh, int64_t e0, int64_t n_ops)
{
    const int64_t e1 = sh.grow ? (e0 << sh.grow) : e0 + sh.E;
    return e1 < n_ops ? e1 : n_ops;
}

int64_t longest_epoch(const TailShape& sh, int64_t n_ops)
{
    int64_t m = 0;
    for (int64_t e0 = sh.S; e0 < n_ops; e0 = epoch_end(sh, e0, n_ops)) {
        const int64_t len = epoch_end(sh, e0, n_ops) - e0;
        if (len > m) m = len;
    }
    return m;
}

// candidate capacity of an epoch of E ops
int64_t cand_cap(int64_t E)
{
    int64_t C = (E + CAND_DIV - 1) / CAND_DIV;
    C = (C + TF_CHUNK - 1) / TF_CHUNK * TF_CHUNK;
    return C < CAND_MAX ? C : CAND_MAX;
}

struct TailLayout {
    int64_t K = 0;        // pairs the sort buffers hold: the first part or an epoch's candidates
    size_t st0, st1, bm, cnt, off, coff, ncand, ovf, fvff, fff;
    size_t region;        // shared region: pairs and slots, or the fallback scan
    size_t key0, val0, pos, key1, val1, sks, svar, spos, scratch;   // offsets inside the region
    size_t total;
};

// Scratch: a few per-variable arrays, then one region used in turn by the
// first part's pairs, by an epoch's candidates (chunk slots, sharing their
// space with the sort's second buffers, the pairs, their positions, the sort's
// scratch), and by the epoch's fallback scan over all its ops (taken when the
// candidates overflow their slots).
TailLayout tail_layout(const TailShape& sh, int32_t n_vars, int64_t n_ops)
{
    TailLayout t;
    const int64_t Emax = longest_epoch(sh, n_ops);
    size_t n_chunks = 0, n_slots = 0;          // most chunks, most slots of one epoch
    for (int64_t e0 = sh.S; e0 < n_ops; e0 = epoch_end(sh, e0, n_ops)) {
        const int64_t n = epoch_end(sh, e0, n_ops) - e0;
        if ((size_t)chunks_of(n) > n_chunks) n_chunks = (size_t)chunks_of(n);
        if ((size_t)(chunks_of(n) * slots_for(n)) > n_slots) n_slots = (size_t)(chunks_of(n) * slots_for(n));
    }
    const int64_t C = cand_cap(Emax);
    t.K = C > sh.S ? C : sh.S;
    const size_t K = (size_t)t.K;
    size_t o = 0;
    auto take = [&](size_t b) { const size_t at = o; o += align_up(b, 256); return at; };
    t.st0 = take((size_t)n_vars);
    t.st1 = take((size_t)n_vars);
    t.bm = take(4 * (size_t)((n_vars + 31) / 32));
    t.cnt = take(4 * n_chunks);
    t.off = take(4 * n_chunks);
    t.coff = take(4 * n_chunks);
    t.ncand = take(8);
    t.ovf = take(4);
    t.fvff = take(4 * (size_t)n_vars);
    t.fff = take(8);
    t.region = o;
    size_t r = 0;
    auto rtake = [&](size_t b) { const size_t at = r; r += align_up(b, 256); return at; };
    t.key0 = rtake(4 * K);
    t.val0 = rtake(4 * K);
    t.pos = rtake(4 * K);
    t.scratch = rtake(sorted_check_scratch_bytes(t.K));
    // the slots live until the gather; the sort's second buffers after it
    const size_t shared_at = r;
    t.key1 = shared_at;
    t.val1 = shared_at + align_up(4 * K, 256);
    const size_t second = 2 * align_up(4 * K, 256);
    t.sks = shared_at;
    t.svar = t.sks + align_up(n_slots, 256);
    t.spos = t.svar + align_up(4 * n_slots, 256);
    const size_t slots = align_up(n_slots, 256) + align_up(4 * n_slots, 256) + align_up(2 * n_slots, 256);
    r += second > slots ? second : slots;
    size_t reg = r;
    const size_t fallback = scan_workspace_bytes(Emax, n_vars, false);
    if (fallback > reg) reg = fallback;
    t.total = o + reg;
    return t;
}

// bit v: status of v is F
__global__ void tail_bitmap_kernel(const uint8_t* __restrict__ st, int32_t n_vars, uint32_t* __restrict__ bm)
{
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool f = v < n_vars && st[v] == ST_F;
    const uint32_t m = __ballot_sync(0xffffffffu, f);
    if ((threadIdx.x & 31) == 0 && v < n_vars) bm[v >> 5] = m;
}

struct FilterParams {
    const uint8_t* kind_side;   // the epoch's first op
    const int32_t* var;
    int64_t n;                  // ops in the epoch
    int64_t n_after;            // ops of the trace from the epoch's first op on (GT pairing)
    int32_t n_vars;
    const uint32_t* bm;         // stuck bitmap at the epoch's start
    int bm_words;
    uint8_t* step;              // the epoch's outputs
    uint8_t* sks;               // candidate slots: a quarter of the chunk
    int32_t* svar;
    uint16_t* spos;             // position within the chunk
    uint32_t* cnt;              // candidates per chunk
    int* ovf;                   // set when a chunk has more candidates than slots
    int* err;
    int bulk_ok;
};

// Each warp takes chunks of CHUNK ops in steps of 32 x 16 (lane L: ops
// [16 L, 16 L + 16) of a step: one 16-byte load of op bytes and four of ids);
// every position gets F (the candidates' statuses that are not F are written
// after their check), the ops on variables outside the bitmap are staged in
// the chunk's slots in position order.  Op bytes and ids are checked as in the
// scan (malformed bytes, ids out of range, GT not followed by its EN); an id
// out of range is staged as 0.
template <int CHUNK>
__global__ void __launch_bounds__(TF_THREADS, 1) tail_filter_kernel(const FilterParams q)
{
    extern __shared__ __align__(16) uint32_t sbm[];
    for (int i = threadIdx.x; i < q.bm_words; i += TF_THREADS) sbm[i] = q.bm[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t n_chunks = (q.n + CHUNK - 1) / CHUNK;
    for (int64_t c = (int64_t)blockIdx.x * (TF_THREADS / 32) + warp; c < n_chunks;
         c += (int64_t)gridDim.x * (TF_THREADS / 32)) {
        const int64_t c0 = c * CHUNK;
        const int cn = (int)min((int64_t)CHUNK, q.n - c0);
        int wcount = 0;
        bool full = false;                                   // slots exhausted (warp-uniform)
        for (int s0 = 0; s0 < cn; s0 += 32 * TF_PER) {
            const int off = s0 + lane * TF_PER;              // offset in the chunk
            const int64_t i0 = c0 + off;                     // offset in the epoch
            const int nl = (int)min((int64_t)TF_PER, q.n - i0);
            const bool vec = nl == TF_PER && q.bulk_ok;
            uint32_t kw[TF_PER / 4];
            int32_t va[TF_PER];
            uint32_t liveMask = 0;
            if (vec) {
                // full step: four op bytes per 32-bit word are checked at once
                const uint4 kk = __ldcs(reinterpret_cast<const uint4*>(q.kind_side + i0));
                kw[0] = kk.x;
                kw[1] = kk.y;
                kw[2] = kk.z;
                kw[3] = kk.w;
#pragma unroll
                for (int h = 0; h < TF_PER / 4; ++h) {
                    const int4 v4 = __ldcs(reinterpret_cast<const int4*>(q.var + i0) + h);
                    va[4 * h] = v4.x;
                    va[4 * h + 1] = v4.y;
                    va[4 * h + 2] = v4.z;
                    va[4 * h + 3] = v4.w;
                }
                uint32_t badk = 0, gt = 0, badv = 0;
#pragma unroll
                for (int h = 0; h < TF_PER / 4; ++h) {
                    // a valid byte has bits 3 and 5-7 clear (kinds 0..7, side bit 4)
                    badk |= kw[h] & 0xE8E8E8E8u;
                    // bytes whose kind is GT (6): zero bytes of (kind ^ 6)
                    const uint32_t x = (kw[h] & 0x0F0F0F0Fu) ^ 0x06060606u;
                    gt |= (x - 0x01010101u) & ~x & 0x80808080u;
                }
#pragma unroll
                for (int u = 0; u < TF_PER; ++u) {
                    const uint32_t v = (uint32_t)va[u];
                    const bool ok = v < (uint32_t)q.n_vars;
                    badv |= !ok;
                    const uint32_t uv = ok ? v : 0u;
                    va[u] = (int32_t)uv;
                    const uint32_t stuck = (sbm[uv >> 5] >> (uv & 31)) & 1u;
                    liveMask |= (stuck ^ 1u) << u;
                }
                if (badk) raise_error(q.err, AMC_E_INVALID);
                if (badv) raise_error(q.err, AMC_E_RANGE);
                if (gt) {
                    // GT must be followed by EN of the same side on another variable
#pragma unroll
                    for (int u = 0; u < TF_PER; ++u) {
                        const uint32_t ks = (kw[u >> 2] >> (8 * (u & 3))) & 0xFFu;
                        if ((ks & 15u) != AMC_K_GT) continue;
                        const uint32_t uv = (uint32_t)va[u] < (uint32_t)q.n_vars ? (uint32_t)va[u] : 0u;
                        uint32_t nks = 0xFF;
                        int32_t nv = (int32_t)uv;
                        if (i0 + u + 1 < q.n_after) {
                            nks = q.kind_side[i0 + u + 1];
                            nv = q.var[i0 + u + 1];
                        }
                        if (!((nks & 15) == AMC_K_EN && (nks >> 4) == (ks >> 4) && nv != (int32_t)uv))
                            raise_error(q.err, AMC_E_INVALID);
                    }
                }
                constexpr uint32_t F4 = 0x01010101u * ST_F;
                __stcs(reinterpret_cast<uint4*>(q.step + i0), make_uint4(F4, F4, F4, F4));
            } else {
#pragma unroll
                for (int h = 0; h < TF_PER / 4; ++h) kw[h] = 0;
#pragma unroll
                for (int u = 0; u < TF_PER; ++u) {
                    va[u] = 0;
                    if (u < nl) {
                        kw[u >> 2] |= (uint32_t)q.kind_side[i0 + u] << (8 * (u & 3));
                        va[u] = q.var[i0 + u];
                    }
                }
#pragma unroll
                for (int u = 0; u < TF_PER; ++u) {
                    const uint32_t ks = (kw[u >> 2] >> (8 * (u & 3))) & 0xFFu;
                    if (u < nl) {
                        if ((ks & 0xE0u) || (ks & 15u) > AMC_K_EN) raise_error(q.err, AMC_E_INVALID);
                        uint32_t uv = (uint32_t)va[u];
                        if (va[u] < 0 || va[u] >= q.n_vars) {
                            raise_error(q.err, AMC_E_RANGE);
                            uv = 0;
                        }
                        if ((ks & 15u) == AMC_K_GT) {
                            uint32_t nks = 0xFF;
                            int32_t nv = (int32_t)uv;
                            if (i0 + u + 1 < q.n_after) {
                                nks = q.kind_side[i0 + u + 1];
                                nv = q.var[i0 + u + 1];
                            }
                            if (!((nks & 15) == AMC_K_EN && (nks >> 4) == (ks >> 4) && nv != (int32_t)uv))
                                raise_error(q.err, AMC_E_INVALID);
                        }
                        va[u] = (int32_t)uv;
                        if (!((sbm[uv >> 5] >> (uv & 31)) & 1u)) liveMask |= 1u << u;
                        q.step[i0 + u] = (uint8_t)ST_F;
                    }
                }
            }
            const int cl = __popc(liveMask);
            if (full || !__any_sync(0xffffffffu, cl != 0)) continue;
            int pre = 0, wtot = 0;
#pragma unroll
            for (int bit = 0; bit < 6; ++bit) {                 // counts 0..32
                const uint32_t bal = __ballot_sync(0xffffffffu, (cl >> bit) & 1);
                pre += __popc(bal & lt) << bit;
                wtot += __popc(bal) << bit;
            }
            if (wcount + wtot > CHUNK / TF_SLOT_DIV) {
                // more candidates than slots: the epoch is rechecked whole
                if (lane == 0) atomicExch(q.ovf, 1);
                full = true;
                continue;
            }
            int64_t idx = c * (CHUNK / TF_SLOT_DIV) + wcount + pre;
#pragma unroll
            for (int u = 0; u < TF_PER; ++u) {
                if (liveMask & (1u << u)) {
                    q.sks[idx] = (uint8_t)((kw[u >> 2] >> (8 * (u & 3))) & 0xFFu);
                    q.svar[idx] = va[u];
                    q.spos[idx] = (uint16_t)(off + u);
                    ++idx;
                }
            }
            wcount += wtot;
        }
        if (lane == 0) q.cnt[c] = (uint32_t)wcount;
    }
}

// Candidates per block of 1024 chunks.
__global__ void __launch_bounds__(1024) tail_blocksum_kernel(const uint32_t* __restrict__ cnt, int n_chunks,
                                                             uint32_t* __restrict__ bsum)
{
    __shared__ uint32_t ws[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * 1024 + threadIdx.x;
    uint32_t x = i < n_chunks ? cnt[i] : 0u;
#pragma unroll
    for (int d = 16; d; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
    if (lane == 0) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t y = ws[lane];
#pragma unroll
        for (int d = 16; d; d >>= 1) y += __shfl_xor_sync(0xffffffffu, y, d);
        if (lane == 0) bsum[blockIdx.x] = y;
    }
}

// Offsets of the chunks' candidates in the compacted set, in position order.  Block b takes
// chunks [1024 b, 1024 b + 1024): its base is the sum of the earlier blocks'
// counts, its chunks' offsets a block scan; each warp copies 32 chunks.  Every
// block also forms the grand total, so all agree on an overflow (more
// candidates than the compacted trace holds, or a chunk with more than its
// slots): then nothing is copied and the epoch's fallback scan runs instead.
__global__ void __launch_bounds__(1024) tail_offsets_kernel(const uint32_t* __restrict__ cnt, int n_chunks,
                                                            const uint32_t* __restrict__ bsum, int n_blocks,
                                                            int64_t cap, uint32_t* __restrict__ coff,
                                                            int64_t* __restrict__ n_cand, int* ovf)
{
    __shared__ unsigned long long rb[32], rt[32];
    __shared__ uint32_t wsum[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int b = blockIdx.x;
    unsigned long long before = 0, total = 0;
    for (int j = tid; j < n_blocks; j += 1024) {
        const unsigned long long v = bsum[j];
        total += v;
        if (j < b) before += v;
    }
#pragma unroll
    for (int d = 16; d; d >>= 1) {
        before += __shfl_xor_sync(0xffffffffu, before, d);
        total += __shfl_xor_sync(0xffffffffu, total, d);
    }
    if (lane == 0) {
        rb[warp] = before;
        rt[warp] = total;
    }
    const int filter_ovf = *ovf;              // read before any block can write it
    __syncthreads();
    before = total = 0;
#pragma unroll 4
    for (int w = 0; w < 32; ++w) {
        before += rb[w];
        total += rt[w];
    }
    if (filter_ovf || total > (unsigned long long)cap) {
        if (b == 0 && tid == 0) {
            *ovf = 1;
            *n_cand = 0;
        }
        return;
    }
    if (b == 0 && tid == 0) *n_cand = (int64_t)total;
    const int i = b * 1024 + tid;
    const uint32_t x = i < n_chunks ? cnt[i] : 0u;
    uint32_t incl = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = wsum[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, v, d);
            if (lane >= d) v += y;
        }
        wsum[lane] = v;                      // inclusive over warps
    }
    __syncthreads();
    if (i < n_chunks) coff[i] = (uint32_t)before + (warp > 0 ? wsum[warp - 1] : 0u) + incl - x;
}

// Warp per G consecutive chunks (G a power of two up to 32, larger where the
// epoch has many chunks and few candidates each), whose candidates are
// contiguous in the compacted set: lane L copies entries L, L + 32, ... of
// that stretch (the stores coalesce), finding each entry's chunk by a binary
// search over the G chunks' prefix counts, which lanes 0..G-1 hold.
__global__ void __launch_bounds__(256) tail_gather_kernel(const uint8_t* __restrict__ sks,
                                                          const int32_t* __restrict__ svar,
                                                          const uint16_t* __restrict__ spos,
                                                          const uint32_t* __restrict__ cnt,
                                                          const uint32_t* __restrict__ coff, int n_chunks,
                                                          uint32_t* __restrict__ ckey, uint32_t* __restrict__ cval,
                                                          uint32_t* __restrict__ cpos, int G, int chunk, int slots,
                                                          const int* ovf)
{
    if (*ovf) return;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g * G < n_chunks; g += nw) {
        const int64_t c = g * G + lane;
        const bool mine = lane < G && c < n_chunks;
        const uint32_t nk = mine ? cnt[c] : 0u;
        const uint32_t base = __shfl_sync(0xffffffffu, mine ? coff[c] : 0u, 0);
        uint32_t incl = nk;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t excl = incl - nk;
        for (uint32_t i0 = 0; i0 < total; i0 += 32) {
            const uint32_t idx = i0 + lane;
            int k = 0;                                      // largest k < G with excl_k <= idx
            for (int step = G >> 1; step; step >>= 1) {
                const uint32_t e = __shfl_sync(0xffffffffu, excl, k + step);
                if (e <= idx) k += step;
            }
            const uint32_t first = __shfl_sync(0xffffffffu, excl, k);
            if (idx < total) {
                const int64_t ch = g * G + k;
                const int64_t src = ch * slots + (idx - first);
                const uint32_t o = base + idx;
                ckey[o] = (uint32_t)svar[src];
                cval[o] = o << 4 | sorted_code_of(sks[src]);
                cpos[o] = (uint32_t)ch * (uint32_t)chunk + spos[src];
            }
        }
    }
}

// After an epoch's fallback scan (gated on by its overflow flag): the scan's
// first faults folded into the trace's, the stuck bitmap rebuilt from the
// statuses the scan wrote.
__global__ void tail_post_kernel(const int* gate, const uint8_t* __restrict__ st, int32_t n_vars,
                                 uint32_t* __restrict__ bm, int32_t* __restrict__ vff,
                                 const int32_t* __restrict__ fvff, int64_t* __restrict__ ff,
                                 const int64_t* __restrict__ fff, int64_t offset)
{
    if (*gate == 0) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_words = ((int64_t)n_vars + 31) / 32 * 32;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_words; v += stride) {
        bool f = false;
        if (v < n_vars) {
            if (vff[v] == -1 && fvff[v] != -1) vff[v] = (int32_t)(fvff[v] + offset);
            f = st[v] == ST_F;
        }
        const uint32_t m = __ballot_sync(0xffffffffu, f);
        if ((threadIdx.x & 31) == 0) bm[v >> 5] = m;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && *fff != -1) {
        const unsigned long long g = (unsigned long long)(*fff + offset);
        atomicMin(reinterpret_cast<unsigned long long*>(ff), g);
    }
}

}  // namespace

bool scan_tail_eligible(const ScanLaunch& L)
{
    TailShape sh;
    return (L.dense != 0 || L.tail == 1) && !L.n_dev && !L.gate && !L.guard && !L.pre_mode &&
           tail_shape(L.n_ops, L.n_vars, false, sh, L.tail);
}

size_t scan_tail_workspace_bytes(int64_t n_ops, int32_t n_vars)
{
    TailShape sh;                          // the largest shape a launch may take (forced)
    if (!tail_shape(n_ops, n_vars, false, sh, 1)) return 0;
    size_t b = tail_layout(sh, n_vars, n_ops).total;
    TailShape sd;
    if (tail_shape(n_ops, n_vars, false, sd, -1)) {
        const size_t d = tail_layout(sd, n_vars, n_ops).total;
        if (d > b) b = d;
    }
    return b;
}

int scan_tail_launches(const ScanLaunch& L)
{
    TailShape sh;
    if (!scan_tail_eligible(L) || !tail_shape(L.n_ops, L.n_vars, false, sh, L.tail)) return 0;
    // a sorted check: three kernels per radix pass, then the segmented scan's
    // reduce, carry and apply; a bucket check: one radix pass, the bucket kernel
    const int sorted = 3 + 3 * ss_radix_passes(L.n_vars);
    const int bucketed = 3 + 1;
    int epochs = 0;
    for (int64_t e0 = sh.S; e0 < L.n_ops; e0 = epoch_end(sh, e0, L.n_ops)) ++epochs;
    // first part: pairs, its sorted check, the stuck bitmap; per epoch filter,
    // block sums, offsets, gather (which writes the pairs), the candidates'
    // bucket check, gated set-up / scan / final statuses and the gated merge
    // with bitmap rebuild
    return 1 + sorted + 1 + epochs * (4 + bucketed + 3 + 1);
}

int launch_scan_tail(const ScanLaunch& L, cudaStream_t s)
{
    TailShape sh;
    if (!tail_shape(L.n_ops, L.n_vars, false, sh, L.tail)) return AMC_E_INVALID;
    const TailLayout lay = tail_layout(sh, L.n_vars, L.n_ops);
    uint8_t* w = static_cast<uint8_t*>(L.workspace);
    uint8_t* st[2] = {w + lay.st0, w + lay.st1};
    uint32_t* bm = reinterpret_cast<uint32_t*>(w + lay.bm);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(w + lay.cnt);
    uint32_t* bsum = reinterpret_cast<uint32_t*>(w + lay.off);    // candidates per 1024 chunks
    uint32_t* coff = reinterpret_cast<uint32_t*>(w + lay.coff);   // first candidate of each chunk
    int64_t* ncand = reinterpret_cast<int64_t*>(w + lay.ncand);
    int* ovf = reinterpret_cast<int*>(w + lay.ovf);
    int32_t* fvff = reinterpret_cast<int32_t*>(w + lay.fvff);
    int64_t* fff = reinterpret_cast<int64_t*>(w + lay.fff);
    uint8_t* reg = w + lay.region;
    uint8_t* sks = reg + lay.sks;
    int32_t* svar = reinterpret_cast<int32_t*>(reg + lay.svar);
    uint16_t* spos = reinterpret_cast<uint16_t*>(reg + lay.spos);
    uint32_t* key0 = reinterpret_cast<uint32_t*>(reg + lay.key0);
    uint32_t* val0 = reinterpret_cast<uint32_t*>(reg + lay.val0);
    uint32_t* key1 = reinterpret_cast<uint32_t*>(reg + lay.key1);
    uint32_t* val1 = reinterpret_cast<uint32_t*>(reg + lay.val1);
    uint32_t* cpos = reinterpret_cast<uint32_t*>(reg + lay.pos);
    void* scratch = reg + lay.scratch;

    int dev = 0, n_sm = 0, max_optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int bm_words = (L.n_vars + 31) / 32;
    const size_t fsmem = 4 * (size_t)bm_words;
    if ((int)fsmem > max_optin) return AMC_E_INVALID;
    static size_t attr_set[64] = {};
    if (dev >= 64 || attr_set[dev] < fsmem) {
        if (cudaFuncSetAttribute(tail_filter_kernel<TF_CHUNK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fsmem) != cudaSuccess ||
            cudaFuncSetAttribute(tail_filter_kernel<TF_CHUNK_SHORT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)fsmem) != cudaSuccess)
            return AMC_E_CUDA;
        if (dev < 64) attr_set[dev] = fsmem;
    }
    if (L.profile & 1) profile_begin(s);

    // first part: ops [0, S) checked by sorting them by variable, from the
    // initial statuses; final statuses to st[0]
    if (cudaMemsetAsync(L.vff, 0xFF, 4 * (size_t)L.n_vars, s) != cudaSuccess) return AMC_E_CUDA;
    if (cudaMemsetAsync(L.first_fault, 0xFF, 8, s) != cudaSuccess) return AMC_E_CUDA;
    if (L.init) {
        if (cudaMemcpyAsync(st[0], L.init, (size_t)L.n_vars, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return AMC_E_CUDA;
    } else if (cudaMemsetAsync(st[0], AMC_ST_VI, (size_t)L.n_vars, s) != cudaSuccess) {
        return AMC_E_CUDA;
    }
    int rc = launch_ss_keys(L.kind_side, L.var, sh.S, L.n_ops, L.n_vars, key0, val0, L.step, L.err, s);
    if (rc) return rc;
    SortedCheck A;
    A.key[0] = key0;
    A.key[1] = key1;
    A.val[0] = val0;
    A.val[1] = val1;
    A.cap = sh.S;
    A.n_vars = L.n_vars;
    A.init = L.init;
    A.step = L.step;
    A.fin = st[0];
    A.vff = L.vff;
    A.ff = L.first_fault;
    A.scratch = scratch;
    A.err = L.err;
    rc = launch_sorted_check(A, s);
    if (rc) return rc;
    // the stuck bitmap at the first epoch's start; later epochs add the
    // variables that become stuck (the bucket checks set their bits, the
    // fallback rebuilds it)
    tail_bitmap_kernel<<<(unsigned)((L.n_vars + 255) / 256), 256, 0, s>>>(st[0], L.n_vars, bm);

    int cur = 0;
    for (int64_t e0 = sh.S; e0 < L.n_ops;) {
        const int64_t e1 = epoch_end(sh, e0, L.n_ops);
        const int64_t n = e1 - e0;
        const bool last = e1 >= L.n_ops;
        uint8_t* fin = (last && L.final_status) ? L.final_status : st[cur ^ 1];
        if (cudaMemsetAsync(ovf, 0, sizeof(int), s) != cudaSuccess) return AMC_E_CUDA;
        const int chunk = chunk_for(n);
        const int slots = slots_for(n);
        FilterParams q;
        q.kind_side = L.kind_side + e0;
        q.var = L.var + e0;
        q.n = n;
        q.n_after = L.n_ops - e0;
        q.n_vars = L.n_vars;
        q.bm = bm;
        q.bm_words = bm_words;
        q.step = L.step + e0;
        q.sks = sks;
        q.svar = svar;
        q.spos = spos;
        q.cnt = cnt;
        q.ovf = ovf;
        q.err = L.err;
        q.bulk_ok = ((uintptr_t)q.kind_side % 16 == 0) && ((uintptr_t)q.var % 16 == 0) &&
                    ((uintptr_t)q.step % 16 == 0);
        const int n_chunks = (int)chunks_of(n);
        const int fgrid = (int)min((int64_t)n_sm, ((int64_t)n_chunks + TF_THREADS / 32 - 1) / (TF_THREADS / 32));
        if (chunk == TF_CHUNK)
            tail_filter_kernel<TF_CHUNK><<<fgrid, TF_THREADS, fsmem, s>>>(q);
        else
            tail_filter_kernel<TF_CHUNK_SHORT><<<fgrid, TF_THREADS, fsmem, s>>>(q);
        const int n_blocks = (n_chunks + 1023) / 1024;
        const int64_t C = cand_cap(n);
        tail_blocksum_kernel<<<n_blocks, 1024, 0, s>>>(cnt, n_chunks, bsum);
        tail_offsets_kernel<<<n_blocks, 1024, 0, s>>>(cnt, n_chunks, bsum, n_blocks, C, coff, ncand, ovf);
        int G = 1;                                   // chunks per gather warp: about 8,192 warps
        while (G < 32 && n_chunks / (2 * G) >= 8192) G *= 2;
        const int64_t groups = ((int64_t)n_chunks + G - 1) / G;
        const int ggrid = (int)min((int64_t)n_sm * 8, (groups + 7) / 8);
        tail_gather_kernel<<<ggrid, 256, 0, s>>>(sks, svar, spos, cnt, coff, n_chunks, key0, val0, cpos, G, chunk, slots,
                                                 ovf);
        if (cudaGetLastError() != cudaSuccess) return AMC_E_CUDA;
        // the candidates, at most C (count on the device), from the epoch's
        // start statuses, checked per bucket of ids (final statuses written
        // where they change); gated off when they overflowed
        if (cudaMemcpyAsync(fin, st[cur], (size_t)L.n_vars, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return AMC_E_CUDA;
        SortedCheck K;
        K.key[0] = key0;
        K.key[1] = key1;
        K.val[0] = val0;
        K.val[1] = val1;
        K.pos = cpos;
        K.n_dev = ncand;
        K.cap = C;
        K.gate = ovf;
        K.n_vars = L.n_vars;
        K.init = st[cur];
        K.step = L.step + e0;
        K.fin = fin;
        K.vff = L.vff;
        K.ff = L.first_fault;
        K.offset = e0;
        K.scratch = scratch;
        K.err = L.err;
        K.bm = bm;
        rc = launch_bucket_check(K, s);
        if (rc) return rc;
        // fallback, gated on by an overflow: the single-pass scan over all the
        // epoch's ops from its start statuses
        ScanLaunch F = L;
        F.kind_side = L.kind_side + e0;
        F.var = L.var + e0;
        F.n_ops = n;
        F.gate = ovf;
        F.gate_on = 1;
        F.init = st[cur];
        F.step = L.step + e0;
        F.final_status = fin;
        F.vff = fvff;
        F.first_fault = fff;
        F.workspace = reg;
        F.dense = 0;
        F.profile = 0;
        rc = launch_scan_trace(F, s);
        if (rc) return rc;
        tail_post_kernel<<<n_sm * 2, 256, 0, s>>>(ovf, fin, L.n_vars, bm, L.vff, fvff, L.first_fault, fff, e0);
        if (cudaGetLastError() != cudaSuccess) return AMC_E_CUDA;
        cur ^= 1;
        e0 = e1;
    }
    if (L.profile & 2) profile_end(s);
    return AMC_OK;
}

}  // namespace amc
