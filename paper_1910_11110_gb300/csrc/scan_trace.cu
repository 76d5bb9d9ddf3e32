// scan_trace.cu -- single-pass per-variable scan of an op trace (sm_103a).
//
// What it computes: for every op i on variable v = var[i] the status of v after
// the op, by applying each op's transfer function in trace order (rules Effect
// and Remote Effect of Fig. Opsem; sequencing is associative with Noop as unit,
// Section 3.2, so per-variable prefix compositions give the same statuses).
//
// How (one CTA per tile of T = 4096 ops, persistent CTAs taking tiles in order):
//  1. the tile's op bytes and var ids are staged into shared memory by bulk
//     async copies (cp.async.bulk + mbarrier);
//  2. each op byte becomes a monoid element (5-bit id, table lookup) and each
//     op a packed key (var << 12 | position);
//  3. a stable LSD radix sort of the keys in shared memory (at most 10 bits
//     per pass, warp ranking with match.any, per-warp histogram rows) groups
//     the tile's ops per variable ("runs"); arrays are padded one word per 32
//     so that each thread's blocked slice is read without bank conflicts;
//  4. a segmented scan over the sorted runs composes each op's in-tile prefix
//     (thread-serial composition, then a warp-shuffle segmented scan);
//  5. each run needs the status of its variable at tile entry.  Runs of a
//     variable already known to be stuck take F at once (F is absorbing; the
//     first-fault table doubles as that index; its loads are issued before the
//     scan so the scan hides their latency).  The other runs add a node (the
//     tile's aggregate) to the variable's list of touching tiles, kept sorted
//     by tile with lock-free insertion, then -- once every earlier tile has
//     registered -- walk that list back composing aggregates until a node with
//     a published inclusive status or the list end (initial status): decoupled
//     look-back restricted to the tiles that touch the variable;
//  6. outputs are written in original order (coalesced 16-byte stores), first
//     faults by atomicMin.
// Where few ops are live (the stuck bitmap filters nearly all of them) a CTA
// takes up to 16 tiles per claim instead ("group path"): it streams them from
// global memory, writes the stuck ops' outputs at once, and runs steps 3-6 once
// for the live ops of the whole group, with runs split per tile so that nodes
// and registration stay per tile.  The claim size follows the live ops per
// tile the CTA saw lately; a group with more live ops than one tile's buffers
// hold is processed tile by tile.  A look-back walk stops early once the
// aggregates it has passed send every status to F.
// The only waits are on the registration frontier and on the mbarrier, both
// bounded; an expired wait raises AMC_E_TIMEOUT and the kernel carries on.
#include <cstdlib>

#include "amc_internal.cuh"
#include "scan_trace.cuh"

namespace amc {

namespace {

constexpr int TILE = 4096;
constexpr int THREADS = 256;
constexpr int POS_BITS = 12;                // log2(TILE)
constexpr int MAX_DIGIT_BITS = 7;                // radix digit: 2 KB of histogram rows
constexpr uint8_t RUN_PENDING = 0xFF;
constexpr uint32_t NO_NODE = 0x80000000u;      // pending-run flag: constant-F run, no list node
// A first-fault entry with this bit set is a bound, not a position: the
// variable is stuck by the end of the position in the low bits (a run of that
// tile sends every status to F).  An exact fault is never larger than a bound
// of its variable, so atomicMin keeps it once recorded; a bound that is still
// there at the end belongs to a variable that was already F at the start
// (no fault inside the trace) and is cleared by the final-status pass.
constexpr uint32_t VFF_BOUND = 0x80000000u;
constexpr uint32_t NODE_AGG = 0x40;
constexpr uint32_t NODE_INCL = 0x80;
constexpr uint32_t SPIN_LIMIT = 1u << 22;
constexpr int DEFAULT_FB_BITS = 1 << 20;      // shared stuck bitmap: 128 KB
constexpr int N_PHASES = 12;
constexpr int RANK_SORT_MAX = 128;             // live ops below which a rank sort replaces the radix passes
constexpr int GROUP_MAX = 16;                  // tiles per claim in the group path (positions fit 16 bits)
constexpr int MAX_CTAS_PER_SM = 3;             // resident CTAs per SM the launch bounds and carve-out assume
constexpr int GROUP_LIVE_TARGET = 2048;        // expected live ops per group when choosing its size

}  // namespace

// Cycle counters per phase of the scan kernel (debug aid, summed over CTAs).
__device__ unsigned long long g_scan_phase_cycles[N_PHASES];

namespace {

__device__ __forceinline__ int pad(int i) { return i + (i >> 5); }

template <typename KeyT, int T, int NT>
struct __align__(16) ScanSmem {
    KeyT vbuf[1][T + T / 32];        // bulk target of the var ids (first 4T bytes); after the
                                     // decode it holds the live ops' packed keys
    KeyT keyA[T + T / 32];
    union {
        struct {
            uint8_t kind[1][T];      // op bytes (tile path)
            uint8_t out[T];          // output tile (tile path)
        };
        uint16_t livePos[T];         // group path: tile in group << 12 | position, per live op
    };
    uint8_t mel[T];                  // element ids of live ops (by position; by live index in groups)
    uint8_t runEntry[T];
    uint16_t hist[(NT / 32) << MAX_DIGIT_BITS];   // per-warp rows of the radix histogram
    uint8_t comp[MAX_ELEMS * MAX_ELEMS];
    uint8_t app[MAX_ELEMS * 8];
    uint8_t elem_of[256];
    uint32_t constF;                 // bit e: element e sends every status to F
    int scanTmp[NT / 32 + 2];
    uint8_t segF[NT / 32];
    uint8_t segV[NT / 32];
    uint16_t cnt[(T / NT) * (NT / 32)];   // live ops per (slot, warp), then their offsets
    uint64_t mbar[1];
    int tile[1];
    int viaBulk[1];
    int nPend;
    int nLive;
    uint32_t frontVal;
    int grp[1];                      // tiles in the current claim
    int64_t nOps;                    // ops of the trace (the host count, or the device one)
    int nTiles;
    // followed (dynamic shared memory) by the stuck bitmap: fbw 32-bit words
};
// three CTAs per SM with 32-bit keys within a 164 KB shared-memory carve-out (1 KB reserved
// per CTA), which leaves 92 KB of L1 for the stuck bitmap read through it
static_assert(MAX_CTAS_PER_SM * (sizeof(ScanSmem<uint32_t, TILE, THREADS>) + 1024) <= 164 * 1024,
              "shared memory per CTA");

__device__ __forceinline__ uint32_t comp_of(const uint8_t* comp, uint32_t a, uint32_t b)
{
    return comp[a * MAX_ELEMS + b];
}

template <typename KeyT, int T, int NT>
__device__ void process_tile(const ScanParams& p, ScanSmem<KeyT, T, NT>& S, uint32_t* fsm, const int t, const int b,
                             const uint32_t refresh, long long& last)
{
#define PHASE(k)                                                                                 \
    if (p.phase_on && threadIdx.x == 0) {                                                        \
        const long long now = clock64();                                                         \
        atomicAdd(&g_scan_phase_cycles[k], (unsigned long long)(now - last));                     \
        last = now;                                                                              \
    }
    constexpr int E = T / NT;
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)t * T;
    const int n = (int)min((int64_t)T, S.nOps - base);
    uint8_t* kb = S.kind[b];
    int32_t* vraw = reinterpret_cast<int32_t*>(S.vbuf[b]);
    const uint32_t ID = 0;
    const uint32_t lt = lanemask_lt();

    if (!S.viaBulk[b]) {
        for (int i = tid; i < n; i += NT) {
            kb[i] = p.kind_side[base + i];
            vraw[i] = p.var[base + i];
        }
        __syncthreads();
    }
    // L1-cached copy of the stuck bitmap: the two global copies alternate every
    // 64 tiles of this CTA, so cached lines never get older than that
    const uint32_t* fbl1 = p.fbits + ((refresh >> 6) & 1u) * (uint32_t)p.fbits_words;
    // rolling refresh of the shared copy of the stuck bitmap (16 bytes per
    // thread per tile).  Bits are only ever set, so a stale word is merely
    // less complete, never wrong.
    if (p.fbw) {
        const uint32_t nq = (uint32_t)p.fbw / 4;
#pragma unroll
        for (uint32_t r = 0; r < 2; ++r) {
            const uint32_t q = ((2 * refresh + r) * NT + tid) % nq;
            reinterpret_cast<uint4*>(fsm)[q] = __ldcg(reinterpret_cast<const uint4*>(p.fbits) + q);
        }
    }

    // ---- 2. decode: four consecutive ops per thread and step (one 32-bit load
    // of op bytes, one 16-byte load of ids).  Ops on variables known to be
    // stuck output F at once; the others ("live") get their element ids and
    // are compacted in position order.
    constexpr int G = 4;
    constexpr int STEPS = E / G;
    uint32_t liveBits = 0;                 // bit 4k+u: op u of step k is live
    int excl[STEPS];
    // all loads first: op bytes, ids and (L1 mode) bitmap words of every step
    uint32_t kwa[STEPS];
    int4 vva[STEPS];
    uint32_t fwa[STEPS][G];
#pragma unroll
    for (int k = 0; k < STEPS; ++k) {
        const int i0 = (k * NT + tid) * G;
        kwa[k] = 0;
        vva[k] = make_int4(0, 0, 0, 0);
        if (i0 < n) {
            kwa[k] = *reinterpret_cast<const uint32_t*>(kb + i0);
            vva[k] = *reinterpret_cast<const int4*>(vraw + i0);
        }
    }
#pragma unroll
    for (int k = 0; k < STEPS; ++k) {
        const int32_t va[G] = {vva[k].x, vva[k].y, vva[k].z, vva[k].w};
#pragma unroll
        for (int u = 0; u < G; ++u) {
            const uint32_t uv = (va[u] < 0 || va[u] >= p.n_vars) ? 0u : (uint32_t)va[u];
            fwa[k][u] = uv < (uint32_t)p.fbw * 32u ? fsm[uv >> 5] : (p.fb_mode >= 2 ? __ldg(fbl1 + (uv >> 5)) : 0u);
        }
    }
#pragma unroll
    for (int k = 0; k < STEPS; ++k) {
        const int g = k * NT + tid;
        const int i0 = g * G;
        uint32_t cnt = 0;
        if (i0 < n) {
            const uint32_t kw = kwa[k];
            const int4 vv = vva[k];
            const int32_t va[G] = {vv.x, vv.y, vv.z, vv.w};
            uint32_t outw = 0;
#pragma unroll
            for (int u = 0; u < G; ++u) {
                const int i = i0 + u;
                const uint32_t ks = (kw >> (8 * u)) & 0xFFu;
                uint32_t o = ST_F;
                if (i < n) {
                    if ((ks & 0xE0u) || (ks & 15u) > AMC_K_EN) raise_error(p.err, AMC_E_INVALID);
                    uint32_t uv = (uint32_t)va[u];
                    if (va[u] < 0 || va[u] >= p.n_vars) {
                        raise_error(p.err, AMC_E_RANGE);
                        uv = 0;
                    }
                    bool gt_ok = true;
                    if ((ks & 15u) == AMC_K_GT) {
                        // GT must be followed by EN of the same side on another variable
                        const int64_t gi = base + i;
                        uint32_t nks = 0xFF;
                        int32_t nv = (int32_t)uv;
                        if (gi + 1 < S.nOps) {
                            nks = (i + 1 < n) ? kb[i + 1] : p.kind_side[gi + 1];
                            nv = (i + 1 < n) ? vraw[i + 1] : p.var[gi + 1];
                        }
                        gt_ok = (nks & 15) == AMC_K_EN && (nks >> 4) == (ks >> 4) && nv != (int32_t)uv;
                        if (!gt_ok) raise_error(p.err, AMC_E_INVALID);
                    }
                    const bool stuck = ((fwa[k][u] >> (uv & 31)) & 1u) != 0;
                    if (!stuck) {
                        uint32_t m = S.elem_of[ks];
                        if (m == ELEM_GT) {
                            if (!gt_ok || p.pre_mode) {
                                m = ID;                      // guard pass: GT does not touch guards
                            } else if (!p.guard) {
                                raise_error(p.err, AMC_E_INVALID);   // GT needs the guarded entry point
                                m = ID;
                            } else {
                                // guard = status of the EN's variable before the EN,
                                // written at the next position by the guard pass
                                const uint32_t gs = p.guard[base + i + 1];
                                const int side = ks >> 4;
                                const bool valid = gs != ST_F && (gs & (side == 0 ? 1u : 2u));
                                m = valid ? ID : p.tab.pull_of_side[side];
                            }
                        } else if (m == ELEM_BAD) {
                            m = ID;
                        }
                        S.mel[i] = (uint8_t)m;
                        liveBits |= 1u << (k * G + u);
                        ++cnt;
                        o = 0;                       // written by the live path
                    }
                }
                outw |= o << (8 * u);
            }
            *reinterpret_cast<uint32_t*>(S.out + i0) = outw;   // stuck before the op: stuck after it
        }
        const int incl = warp_incl_sum((int)cnt);
        excl[k] = incl - (int)cnt;
        if (lane == 31) S.cnt[k * NW + warp] = (uint16_t)incl;
    }
    __syncthreads();
    if (warp == 0) {
        // exclusive scan of the live counts in (step, warp) = position order
        constexpr int C = STEPS * NW;
        constexpr int PER = (C + 31) / 32;
        int v[PER];
        int sum = 0;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int idx = lane * PER + u;
            v[u] = idx < C ? S.cnt[idx] : 0;
            sum += v[u];
        }
        const int incl = warp_incl_sum(sum);
        int run = incl - sum;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int idx = lane * PER + u;
            if (idx < C) S.cnt[idx] = (uint16_t)run;
            run += v[u];
        }
        if (lane == 31) S.nLive = incl;
        if (lane == 0) S.nPend = 0;
    }
    __syncthreads();
    if (p.phase_on && tid == 0) atomicAdd(&g_scan_phase_cycles[8], 1ull);
    if (S.nLive == 0 && !p.guard) {
        // every op's variable was already stuck: outputs are all F
        if (tid == 0) {
            __threadfence();
            atomicOr(p.regbits + (t >> 5), 1u << (t & 31));
        }
        if (n == T && p.bulk_ok) {
            const uint4* src = reinterpret_cast<const uint4*>(S.out);
            uint4* dst = reinterpret_cast<uint4*>(p.step + base);
            for (int i = tid; i < T / 16; i += NT) dst[i] = src[i];
        } else {
            for (int i = tid; i < n; i += NT) p.step[base + i] = S.out[i];
        }
        return;
    }
    KeyT* keyIn = S.keyA;
#pragma unroll
    for (int k = 0; k < STEPS; ++k) {
        if (!((liveBits >> (k * G)) & 0xFu)) continue;
        const int i0 = (k * NT + tid) * G;
        int c = S.cnt[k * NW + warp] + excl[k];
#pragma unroll
        for (int u = 0; u < G; ++u) {
            if (liveBits & (1u << (k * G + u))) {
                const int i = i0 + u;
                int32_t v = vraw[i];
                if (v < 0 || v >= p.n_vars) v = 0;
                keyIn[pad(c++)] = ((KeyT)(uint32_t)v << POS_BITS) | (KeyT)i;
            }
        }
    }
    const int nl = S.nLive;                // live ops: the sort and the scan see only these
    if (p.phase_on && tid == 0) {
        atomicAdd(&g_scan_phase_cycles[9], 1ull);
        atomicAdd(&g_scan_phase_cycles[10], (unsigned long long)nl);
    }
    // own histogram row cleared before the first ranking
    const int D0 = 1 << p.digit_bits;
    for (int i = lane; i < D0; i += 32) S.hist[warp * D0 + i] = 0;
    __syncthreads();
    PHASE(1)

    // ---- 3. stable LSD radix sort of the packed keys ------------------------
    KeyT* kin = keyIn;
    KeyT* kout = S.vbuf[b];
    const bool rank_sort = nl <= RANK_SORT_MAX;
    if (nl > 0 && rank_sort) {
        // few live ops: each key's rank is the number of smaller keys (keys are
        // unique: they carry the position)
        if (tid < nl) {
            const KeyT kj = kin[pad(tid)];
            int r = 0;
            for (int i = 0; i < nl; ++i) r += kin[pad(i)] < kj;
            kout[pad(r)] = kj;
        }
        __syncthreads();
        KeyT* tk = kin;
        kin = kout;
        kout = tk;
    }
    for (int pass = 0; pass < (nl && !rank_sort ? p.passes : 0); ++pass) {
        const int D = 1 << p.digit_bits;
        const int shift = POS_BITS + pass * p.digit_bits;
        uint16_t* hrow = S.hist + warp * D;
        if (pass > 0) {
            for (int i = lane; i < D; i += 32) hrow[i] = 0;
            __syncwarp();
        }
        KeyT kk[E];
        uint16_t lr[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int pos = warp * 32 * E + e * 32 + lane;
            const bool ok = pos < nl;
            const KeyT key = ok ? kin[pad(pos)] : (KeyT)0;
            kk[e] = key;
            const uint32_t dig = ok ? (uint32_t)((key >> shift) & (KeyT)(D - 1)) : 0xFFFFFFFFu;
            const uint32_t peers = __match_any_sync(0xffffffffu, dig);
            const uint32_t rank = __popc(peers & lt);
            uint16_t c = 0;
            if (ok) c = hrow[dig];
            lr[e] = (uint16_t)(c + rank);
            __syncwarp();
            if (ok && rank == 0) hrow[dig] = (uint16_t)(c + __popc(peers));
            __syncwarp();
        }
        __syncthreads();
        {
            // exclusive scan of the counts in (digit, warp) order
            const int per = (D + NT - 1) / NT;
            const int d0 = tid * per;
            int sum = 0;
            for (int d = d0; d < d0 + per && d < D; ++d)
#pragma unroll
                for (int w = 0; w < NW; ++w) sum += S.hist[w * D + d];
            int run = block_excl_sum<NT>(sum, S.scanTmp, nullptr);
            for (int d = d0; d < d0 + per && d < D; ++d)
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    const int c = S.hist[w * D + d];
                    S.hist[w * D + d] = (uint16_t)run;
                    run += c;
                }
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int pos = warp * 32 * E + e * 32 + lane;
            if (pos < nl) {
                const uint32_t dig = (uint32_t)((kk[e] >> shift) & (KeyT)(D - 1));
                kout[pad(hrow[dig] + lr[e])] = kk[e];
            }
        }
        __syncthreads();
        KeyT* tk = kin;
        kin = kout;
        kout = tk;
    }
    PHASE(2)
    const KeyT* K = kin;                       // sorted keys
    uint32_t* pend = reinterpret_cast<uint32_t*>(kout);   // the free buffer
    auto kvar = [&](int j) -> uint32_t { return (uint32_t)(K[pad(j)] >> POS_BITS); };
    auto kpos = [&](int j) -> int { return (int)(K[pad(j)] & (KeyT)(T - 1)); };

    // ---- 4a. run boundaries; the stuck-shortcut loads are issued here so
    // that the segmented scan below hides their latency --------------------
    const int j0 = tid * E;
    uint32_t headMask = 0, lastMask = 0;
    uint32_t ffv[E];
    {
        uint32_t prev = (j0 > 0 && j0 - 1 < nl) ? kvar(j0 - 1) : 0xFFFFFFFFu;
        uint32_t cur = (j0 < nl) ? kvar(j0) : 0xFFFFFFFEu;
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const int j = j0 + k;
            const uint32_t nxt = (j + 1 < nl) ? kvar(j + 1) : 0xFFFFFFFDu;
            ffv[k] = 0xFFFFFFFFu;
            if (j < nl) {
                if (cur != prev) headMask |= 1u << k;
                if (nxt != cur) {
                    lastMask |= 1u << k;
                    ffv[k] = __ldcg(reinterpret_cast<const unsigned int*>(p.vff) + cur);
                }
            }
            prev = cur;
            cur = nxt;
        }
    }

    // ---- 4b. segmented scan over runs (blocked: thread owns E sorted slots) --
    // per-slot prefix (pm) and exclusive prefix (xm), four bytes per word
#define getb(w, k) (((w)[(k) >> 2] >> (8 * ((k) & 3))) & 0xFFu)
#define setb(w, k, v) ((w)[(k) >> 2] = ((w)[(k) >> 2] & ~(0xFFu << (8 * ((k) & 3)))) | ((uint32_t)(v) << (8 * ((k) & 3))))
    uint32_t pmw[E / 4], xmw[E / 4];
#pragma unroll
    for (int i = 0; i < E / 4; ++i) pmw[i] = xmw[i] = 0;    // identity is element 0
    const int nHeads = __popc(headMask);
    uint32_t acc = ID;
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const int j = j0 + k;
        if (j < nl) {
            const uint32_t m = S.mel[kpos(j)];
            if (headMask & (1u << k)) {
                acc = m;
            } else {
                setb(xmw, k, acc);
                acc = comp_of(S.comp, acc, m);
            }
            setb(pmw, k, acc);
        }
    }
    uint32_t carry;
    {
        uint32_t f = headMask != 0, v = acc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t fu = __shfl_up_sync(0xffffffffu, f, o);
            const uint32_t vu = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) {
                if (!f) v = comp_of(S.comp, vu, v);
                f |= fu;
            }
        }
        uint32_t fe = __shfl_up_sync(0xffffffffu, f, 1);
        uint32_t ve = __shfl_up_sync(0xffffffffu, v, 1);
        if (lane == 0) { fe = 0; ve = ID; }
        if (lane == 31) { S.segF[warp] = (uint8_t)f; S.segV[warp] = (uint8_t)v; }
        __syncthreads();
        if (warp == 0) {
            uint32_t wf = lane < NW ? S.segF[lane] : 0, wv = lane < NW ? S.segV[lane] : ID;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t fu = __shfl_up_sync(0xffffffffu, wf, o);
                const uint32_t vu = __shfl_up_sync(0xffffffffu, wv, o);
                if (lane >= o) {
                    if (!wf) wv = comp_of(S.comp, vu, wv);
                    wf |= fu;
                }
            }
            uint32_t xf = __shfl_up_sync(0xffffffffu, wf, 1);
            uint32_t xv = __shfl_up_sync(0xffffffffu, wv, 1);
            if (lane == 0) { xf = 0; xv = ID; }
            if (lane < NW) { S.segF[lane] = (uint8_t)xf; S.segV[lane] = (uint8_t)xv; }
        }
        __syncthreads();
        carry = fe ? ve : comp_of(S.comp, S.segV[warp], ve);
    }
    // elements before the thread's first head continue a run from earlier threads
#pragma unroll
    for (int k = 0; k < E; ++k) {
        if ((headMask & ((2u << k) - 1)) == 0) {
            setb(pmw, k, comp_of(S.comp, carry, getb(pmw, k)));
            setb(xmw, k, comp_of(S.comp, carry, getb(xmw, k)));
        }
    }
    const int runBase = block_excl_sum<NT>(nHeads, S.scanTmp, nullptr);
    auto run_id = [&](int k) { return runBase - 1 + __popc(headMask & ((2u << k) - 1)); };
    PHASE(3)

    // ---- 5a. run entry: stuck shortcut, or a node in the variable's list ----
    const uint32_t nodeBase = (uint32_t)t * (uint32_t)T;
#pragma unroll
    for (int k = 0; k < E; ++k) {
        if (lastMask & (1u << k)) {
            const int r = run_id(k);
            if ((ffv[k] & ~VFF_BOUND) < (uint32_t)base) {
                S.runEntry[r] = ST_F;
                // stuck before this tile, hence before every later tile of this CTA
                const uint32_t v = kvar(j0 + k);
                if (v < (uint32_t)p.fbw * 32u) atomicOr(fsm + (v >> 5), 1u << (v & 31));
            } else {
                const uint32_t agg = getb(pmw, k);
                S.runEntry[r] = RUN_PENDING;
                if ((S.constF >> agg) & 1u) {
                    // stuck by the end of this tile whatever its entry: publish
                    // that bound as the first fault (the exact one, recorded
                    // below or earlier, is never larger) instead of a node;
                    // later tiles take the stuck shortcut
                    atomicMin(reinterpret_cast<uint32_t*>(p.vff) + kvar(j0 + k), (uint32_t)(base + T - 1) | VFF_BOUND);
                    pend[atomicAdd(&S.nPend, 1)] = (uint32_t)r | ((uint32_t)(j0 + k) << 16) | NO_NODE;
                } else {
                    pend[atomicAdd(&S.nPend, 1)] = (uint32_t)r | ((uint32_t)(j0 + k) << 16);
                    p.node_status[nodeBase + r] = (uint8_t)(NODE_AGG | agg);
                }
            }
        }
    }
    __syncthreads();
    const int nPend = S.nPend;
    if (p.phase_on && tid == 0 && nPend) atomicAdd(&g_scan_phase_cycles[11], 1ull);
    constexpr int PW = 4;                 // pending runs a thread handles in step
    for (int lo = 0; lo < nPend; lo += NT * PW) {
        // insert each node into its variable's list (sorted by decreasing
        // tile): one attempt for PW runs at once, then retries one by one
        uint32_t c[PW], old[PW], node[PW], var[PW];
        uint32_t mine = 0, simple = 0;
#pragma unroll
        for (int u = 0; u < PW; ++u) {
            const int i = lo + u * NT + tid;
            c[u] = NIL;
            node[u] = var[u] = 0;
            if (i < nPend && !(pend[i] & NO_NODE)) {
                const uint32_t e = pend[i];
                mine |= 1u << u;
                node[u] = nodeBase + (e & 0xFFFFu);
                var[u] = kvar((int)(e >> 16));
                c[u] = __ldcg(p.head + var[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < PW; ++u)
            if ((mine & (1u << u)) && (c[u] == NIL || c[u] / T < (uint32_t)t)) {
                p.node_next[node[u]] = c[u];
                simple |= 1u << u;
            }
        __threadfence();
#pragma unroll
        for (int u = 0; u < PW; ++u) old[u] = (simple & (1u << u)) ? atomicCAS(p.head + var[u], c[u], node[u]) : c[u];
#pragma unroll
        for (int u = 0; u < PW; ++u) {
            if (!(mine & (1u << u)) || ((simple & (1u << u)) && old[u] == c[u])) continue;
            uint32_t* link = p.head + var[u];
            for (uint32_t it = 0;; ++it) {
                const uint32_t cc = ld_acquire(link);
                if (cc == NIL || cc / T < (uint32_t)t) {
                    p.node_next[node[u]] = cc;
                    __threadfence();
                    if (atomicCAS(link, cc, node[u]) == cc) break;
                } else {
                    link = p.node_next + cc;
                }
                if (it > SPIN_LIMIT) { raise_error(p.err, AMC_E_TIMEOUT); break; }
            }
        }
    }
    __syncthreads();

    PHASE(4)
    // ---- 5b. registration frontier ------------------------------------------
    // bit t of regbits is set once tile t's nodes are all in their lists;
    // *front = F means every tile < F has registered.  Only tiles that look
    // back (and all tiles of the guard-resolving pass, whose first input status
    // is read by the previous tile) wait for the frontier to reach them.
    if (tid == 0) {
        __threadfence();
        atomicOr(p.regbits + (t >> 5), 1u << (t & 31));
    }
    if (nPend > 0 || p.guard) {
        // check every tile in [front, t) at once, 32 per word, starting from the
        // frontier this CTA last knew (checking more tiles than needed is safe)
        uint32_t f0 = min(S.frontVal, (uint32_t)t);
        for (uint32_t it = 0;; ++it) {
            bool all = true;
            for (uint32_t w = (f0 >> 5) + tid; f0 < (uint32_t)t && w <= ((uint32_t)t - 1) >> 5; w += NT) {
                const uint32_t lo = max(f0, w << 5), hi = min((uint32_t)t, (w << 5) + 32);
                const uint32_t need = (hi - lo == 32) ? 0xFFFFFFFFu : (((1u << (hi - lo)) - 1u) << (lo & 31));
                all &= (__ldcg(p.regbits + w) & need) == need;
            }
            if (__syncthreads_and(all)) {
                if (tid == 0) {
                    __threadfence();
                    atomicMax(p.front, (uint32_t)t);
                    S.frontVal = (uint32_t)t;
                }
                break;
            }
            if (it > SPIN_LIMIT) { if (tid == 0) raise_error(p.err, AMC_E_TIMEOUT); break; }
            __nanosleep(128);
            if (tid == 0) S.frontVal = ld_acquire(p.front);
            __syncthreads();
            f0 = min(max(f0, S.frontVal), (uint32_t)t);
            __syncthreads();
        }
        __threadfence();
    }

    PHASE(5)
    // ---- 5c. look-back along the lists, PW runs per thread in step -----------
    for (int lo = 0; lo < nPend; lo += NT * PW) {
        uint32_t q[PW], a[PW], st[PW], node[PW], var[PW], rr[PW], ffw[PW], ag[PW];
        uint32_t active = 0, nonode = 0;
#pragma unroll
        for (int u = 0; u < PW; ++u) {
            const int i = lo + u * NT + tid;
            a[u] = ID;
            st[u] = 0;
            q[u] = NIL;
            node[u] = var[u] = rr[u] = ag[u] = 0;
            ffw[u] = 0xFFFFFFFFu;
            if (i < nPend) {
                const uint32_t e = pend[i];
                active |= 1u << u;
                rr[u] = e & 0xFFFFu;
                var[u] = kvar((int)((e >> 16) & 0x7FFFu));
                if (e & NO_NODE) {
                    nonode |= 1u << u;
                    q[u] = ld_acquire(p.head + var[u]);         // from the newest node
                } else {
                    node[u] = nodeBase + rr[u];
                    q[u] = ld_acquire(p.node_next + node[u]);
                    ag[u] = __ldcg(p.node_status + node[u]) & 31u;   // the run's aggregate (AGG status)
                }
                ffw[u] = ld_acquire(reinterpret_cast<const uint32_t*>(p.vff) + var[u]);
            }
        }
        const uint32_t mine = active;
#pragma unroll
        for (int u = 0; u < PW; ++u)
            if ((active & (1u << u)) && (ffw[u] & ~VFF_BOUND) < (uint32_t)base) {
                st[u] = ST_F;                  // stuck before this tile (bound published since)
                active &= ~(1u << u);
            }
        for (uint32_t hop = 0; active; ++hop) {
            // a node's status and its next pointer are read together: below
            // the walking tile the list no longer changes (every earlier tile
            // has inserted before the frontier passed), and either status of
            // a node (aggregate or inclusive) is a valid answer
            uint32_t sv[PW], nx[PW];
#pragma unroll
            for (int u = 0; u < PW; ++u) {
                sv[u] = 0;
                nx[u] = NIL;
                if ((active & (1u << u)) && q[u] != NIL) {
                    sv[u] = ld_relaxed_u8(p.node_status + q[u]);
                    nx[u] = ld_relaxed(p.node_next + q[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < PW; ++u) {
                if (!(active & (1u << u))) continue;
                if (q[u] == NIL) {
                    st[u] = p.init ? p.init[var[u]] : (uint32_t)AMC_ST_VI;
                    active &= ~(1u << u);
                } else if (q[u] / T >= (uint32_t)t) {
                    // a node of this or a later tile (walks that start at the head)
                } else if (sv[u] & NODE_INCL) {
                    st[u] = sv[u] & 7u;
                    active &= ~(1u << u);
                } else {
                    a[u] = comp_of(S.comp, sv[u] & 31u, a[u]);     // earlier tile first
                    // F is absorbing: once the tiles passed so far send every
                    // status to F, the entry is F whatever came before them
                    if ((S.constF >> a[u]) & 1u) {
                        st[u] = 0;
                        active &= ~(1u << u);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < PW; ++u)
                if (active & (1u << u)) q[u] = nx[u];
            if (hop > SPIN_LIMIT) { raise_error(p.err, AMC_E_TIMEOUT); break; }
        }
#pragma unroll
        for (int u = 0; u < PW; ++u) {
            if (!(mine & (1u << u))) continue;
            const uint32_t entry = S.app[a[u] * 8 + st[u]];
            S.runEntry[rr[u]] = (uint8_t)entry;
            if (!(nonode & (1u << u)))
                st_relaxed_u8(p.node_status + node[u], NODE_INCL | S.app[ag[u] * 8 + entry]);
        }
    }
    __syncthreads();

    PHASE(6)
    // ---- 6. outputs in original order; first faults --------------------------
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const int j = j0 + k;
        if (j < nl) {
            const uint32_t e = S.runEntry[run_id(k)];
            const uint32_t pre = S.app[getb(xmw, k) * 8 + e];
            const uint32_t post = S.app[getb(pmw, k) * 8 + e];
            const int pos = kpos(j);
            S.out[pos] = (uint8_t)(p.pre_mode ? pre : post);
            if (post == ST_F && pre != ST_F) {
                const uint32_t gi = (uint32_t)(base + pos);
                const uint32_t v = kvar(j);
                atomicMin(reinterpret_cast<uint32_t*>(p.vff) + v, gi);
                atomicOr(p.fbits + (v >> 5), 1u << (v & 31));
                atomicOr(p.fbits + p.fbits_words + (v >> 5), 1u << (v & 31));
                if (v < (uint32_t)p.fbw * 32u) atomicOr(fsm + (v >> 5), 1u << (v & 31));
                // the global minimum only falls: skip the atomic once it is below gi
                if ((unsigned long long)gi < *reinterpret_cast<volatile unsigned long long*>(p.first_fault))
                    atomicMin(reinterpret_cast<unsigned long long*>(p.first_fault), (unsigned long long)gi);
            }
        }
    }
#undef getb
#undef setb
    __syncthreads();
    if (n == T && p.bulk_ok) {
        const uint4* src = reinterpret_cast<const uint4*>(S.out);
        uint4* dst = reinterpret_cast<uint4*>(p.step + base);
        for (int i = tid; i < T / 16; i += NT) dst[i] = src[i];
    } else {
        for (int i = tid; i < n; i += NT) p.step[base + i] = S.out[i];
    }
    PHASE(7)
#undef PHASE
}

// Group path: G consecutive tiles taken in one claim and read straight from
// global memory.  Ops on variables known to be stuck get F at once (written
// with the rest of their output word); the live ops of all G tiles -- at most T
// of them -- are sorted, scanned, inserted, registered and looked back
// together.  Runs are (variable, tile) pairs, so list nodes and registration
// bits stay per tile and other CTAs see exactly the tile path's protocol.
// Returns false, having registered nothing, when the group holds more than T
// live ops; the caller then runs its tiles through the tile path.
template <typename KeyT, int T, int NT>
__device__ __noinline__ bool process_group(const ScanParams& p, ScanSmem<KeyT, T, NT>& S, uint32_t* fsm, const int t0, const int G,
                              const uint32_t refresh, long long& last)
{
#define PHASE(k)                                                                                 \
    if (p.phase_on && threadIdx.x == 0) {                                                        \
        const long long now = clock64();                                                         \
        atomicAdd(&g_scan_phase_cycles[k], (unsigned long long)(now - last));                     \
        last = now;                                                                              \
    }
    constexpr int E = T / NT;
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t ID = 0;
    const uint32_t lt = lanemask_lt();
    const int64_t gbase = (int64_t)t0 * T;
    const int nTiles = (int)min((int64_t)G, (int64_t)S.nTiles - t0);

    const uint32_t* fbl1 = p.fbits + ((refresh >> 6) & 1u) * (uint32_t)p.fbits_words;
    if (p.fbw) {
        const uint32_t nq = (uint32_t)p.fbw / 4;
        const uint32_t reps = min(2u * (uint32_t)nTiles, (nq + NT - 1) / NT);   // at most one full pass
        for (uint32_t r = 0; r < reps; ++r) {
            const uint32_t q = ((2 * refresh + r) * NT + tid) % nq;
            reinterpret_cast<uint4*>(fsm)[q] = __ldcg(reinterpret_cast<const uint4*>(p.fbits) + q);
        }
    }

    // ---- 1-2. stream and decode the tiles; compact the live ops ------------
    // Warp w takes the contiguous ops [w R, (w + 1) R) of the group (R =
    // nTiles * T / NW) in steps of 32 * 16 ops; lane L takes ops [16 L, 16 L +
    // 16) of a step (one 16-byte load of op bytes, four of ids, one 16-byte
    // store of outputs).  No block barrier inside the loop: each warp stages
    // its live ops, in position order, in a slice of its own (T / NW entries;
    // a fuller slice sends the group to the tile path), and one barrier at
    // the end concatenates the slices.
    constexpr int PER = T / NT;
    static_assert(PER == 16, "16 ops per thread and step");
    constexpr int CAP = T / NW;                                  // staged live ops per warp
    KeyT* const keyIn = S.keyA;
    uint32_t* const stVar = reinterpret_cast<uint32_t*>(S.vbuf[0]);   // staged var ids
    uint32_t* const stPos = reinterpret_cast<uint32_t*>(S.keyA);      // staged offset | element << 16
    const int gops = (int)min((int64_t)nTiles * T, S.nOps - gbase);  // ops in the group (<= 2^16)
    const int R = nTiles * (T / NW);
    int wcount = 0;                          // live ops staged by this warp (warp-uniform)
    bool over = false;
    for (int s0 = warp * R; s0 < (warp + 1) * R && s0 < gops; s0 += 32 * PER) {
        const int i0 = s0 + lane * PER;                          // group offset of the lane's first op
        const int n = min(PER, gops - i0);                       // its ops in the trace (may be <= 0)
        const int64_t base = gbase + i0;
        const bool vec = n == PER && p.bulk_ok;
        uint32_t kw[PER / 4];
        int32_t va[PER];
        uint32_t outw[PER / 4], melw[PER / 4];
        uint32_t liveMask = 0;
        // element of a live op (GT resolved from its guard, malformed bytes as identity)
        auto live_elem = [&](const uint32_t ks, const uint32_t uv, const int u) -> uint32_t {
            uint32_t m = S.elem_of[ks];
            if (m == ELEM_GT) {
                const int64_t gi = base + u;
                uint32_t nks = 0xFF;
                int32_t nv = (int32_t)uv;
                if (gi + 1 < S.nOps) {
                    nks = p.kind_side[gi + 1];
                    nv = p.var[gi + 1];
                }
                const bool gt_ok = (nks & 15) == AMC_K_EN && (nks >> 4) == (ks >> 4) && nv != (int32_t)uv;
                if (!gt_ok || p.pre_mode) {
                    m = ID;
                } else if (!p.guard) {
                    raise_error(p.err, AMC_E_INVALID);
                    m = ID;
                } else {
                    const uint32_t gs = p.guard[gi + 1];
                    const int side = ks >> 4;
                    const bool valid = gs != ST_F && (gs & (side == 0 ? 1u : 2u));
                    m = valid ? ID : p.tab.pull_of_side[side];
                }
            } else if (m == ELEM_BAD) {
                m = ID;
            }
            return m;
        };
        if (vec) {
            // full step: four op bytes per 32-bit word are checked at once
            const uint4 kk = __ldcs(reinterpret_cast<const uint4*>(p.kind_side + base));
            kw[0] = kk.x;
            kw[1] = kk.y;
            kw[2] = kk.z;
            kw[3] = kk.w;
#pragma unroll
            for (int q = 0; q < PER / 4; ++q) {
                const int4 v4 = __ldcs(reinterpret_cast<const int4*>(p.var + base) + q);
                va[4 * q] = v4.x;
                va[4 * q + 1] = v4.y;
                va[4 * q + 2] = v4.z;
                va[4 * q + 3] = v4.w;
            }
            uint32_t badk = 0, gtw = 0, badv = 0;
#pragma unroll
            for (int q = 0; q < PER / 4; ++q) {
                // a valid byte has bits 3 and 5-7 clear (kinds 0..7, side bit 4)
                badk |= kw[q] & 0xE8E8E8E8u;
                // bytes whose kind is GT (6): zero bytes of (kind ^ 6)
                const uint32_t x = (kw[q] & 0x0F0F0F0Fu) ^ 0x06060606u;
                gtw |= (x - 0x01010101u) & ~x & 0x80808080u;
                outw[q] = melw[q] = 0;
            }
            uint32_t fw[PER];
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const uint32_t v = (uint32_t)va[u];
                const uint32_t uv = v < (uint32_t)p.n_vars ? v : 0u;
                badv |= v >= (uint32_t)p.n_vars;
                fw[u] = uv < (uint32_t)p.fbw * 32u ? fsm[uv >> 5] : (p.fb_mode >= 2 ? __ldg(fbl1 + (uv >> 5)) : 0u);
            }
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const uint32_t v = (uint32_t)va[u];
                const uint32_t uv = v < (uint32_t)p.n_vars ? v : 0u;
                const uint32_t stuck = (fw[u] >> (uv & 31)) & 1u;
                liveMask |= (stuck ^ 1u) << u;
                outw[u >> 2] |= stuck << (8 * (u & 3) + 2);      // F = 4 where stuck; live: set later
            }
            if (badk) raise_error(p.err, AMC_E_INVALID);
            if (badv) raise_error(p.err, AMC_E_RANGE);
            if (gtw) {
                // GT must be followed by EN of the same side on another variable
#pragma unroll
                for (int u = 0; u < PER; ++u) {
                    const uint32_t ks = (kw[u >> 2] >> (8 * (u & 3))) & 0xFFu;
                    if ((ks & 15u) != AMC_K_GT) continue;
                    const uint32_t uv = (uint32_t)va[u] < (uint32_t)p.n_vars ? (uint32_t)va[u] : 0u;
                    const int64_t gi = base + u;
                    uint32_t nks = 0xFF;
                    int32_t nv = (int32_t)uv;
                    if (gi + 1 < S.nOps) {
                        nks = p.kind_side[gi + 1];
                        nv = p.var[gi + 1];
                    }
                    if (!((nks & 15) == AMC_K_EN && (nks >> 4) == (ks >> 4) && nv != (int32_t)uv))
                        raise_error(p.err, AMC_E_INVALID);
                }
            }
            if (liveMask) {
#pragma unroll
                for (int u = 0; u < PER; ++u) {
                    if (!(liveMask & (1u << u))) continue;
                    const uint32_t ks = (kw[u >> 2] >> (8 * (u & 3))) & 0xFFu;
                    const uint32_t uv = (uint32_t)va[u] < (uint32_t)p.n_vars ? (uint32_t)va[u] : 0u;
                    melw[u >> 2] |= live_elem(ks, uv, u) << (8 * (u & 3));
                }
            }
            __stcs(reinterpret_cast<uint4*>(p.step + base), make_uint4(outw[0], outw[1], outw[2], outw[3]));
        } else {
#pragma unroll
            for (int q = 0; q < PER / 4; ++q) kw[q] = outw[q] = melw[q] = 0;
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                va[u] = 0;
                if (u < n) {
                    kw[u >> 2] |= (uint32_t)p.kind_side[base + u] << (8 * (u & 3));
                    va[u] = p.var[base + u];
                }
            }
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                if (u >= n) continue;
                const uint32_t ks = (kw[u >> 2] >> (8 * (u & 3))) & 0xFFu;
                if ((ks & 0xE0u) || (ks & 15u) > AMC_K_EN) raise_error(p.err, AMC_E_INVALID);
                uint32_t uv = (uint32_t)va[u];
                if (va[u] < 0 || va[u] >= p.n_vars) {
                    raise_error(p.err, AMC_E_RANGE);
                    uv = 0;
                }
                if ((ks & 15u) == AMC_K_GT) {
                    const int64_t gi = base + u;
                    uint32_t nks = 0xFF;
                    int32_t nv = (int32_t)uv;
                    if (gi + 1 < S.nOps) {
                        nks = p.kind_side[gi + 1];
                        nv = p.var[gi + 1];
                    }
                    if (!((nks & 15) == AMC_K_EN && (nks >> 4) == (ks >> 4) && nv != (int32_t)uv))
                        raise_error(p.err, AMC_E_INVALID);
                }
                const uint32_t fwu =
                    uv < (uint32_t)p.fbw * 32u ? fsm[uv >> 5] : (p.fb_mode >= 2 ? __ldg(fbl1 + (uv >> 5)) : 0u);
                uint32_t o = ST_F;
                if (!((fwu >> (uv & 31)) & 1u)) {
                    melw[u >> 2] |= live_elem(ks, uv, u) << (8 * (u & 3));
                    liveMask |= 1u << u;
                    o = 0;                       // written once the run's entry is known
                }
                p.step[base + u] = (uint8_t)o;
            }
        }
        // live-op prefix within the warp (counts are 0..16: five bits)
        const int c = __popc(liveMask);
        if (!__any_sync(0xffffffffu, c != 0)) continue;
        int pre = 0, wtot = 0;
#pragma unroll
        for (int bit = 0; bit < 5; ++bit) {
            const uint32_t bal = __ballot_sync(0xffffffffu, (c >> bit) & 1);
            pre += __popc(bal & lt) << bit;
            wtot += __popc(bal) << bit;
        }
        if (wcount + wtot > CAP) {               // too many live ops for the warp's slice
            over = true;
            break;
        }
        if (liveMask) {
            int idx = warp * CAP + wcount + pre;
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                if (liveMask & (1u << u)) {
                    stVar[idx] = (va[u] < 0 || va[u] >= p.n_vars) ? 0u : (uint32_t)va[u];
                    stPos[idx] = (uint32_t)(i0 + u) | (((melw[u >> 2] >> (8 * (u & 3))) & 0xFFu) << 16);
                    ++idx;
                }
            }
        }
        wcount += wtot;
    }
    if (lane == 0) S.cnt[warp] = over ? 0xFFFFu : (uint16_t)wcount;
    __syncthreads();
    int total = 0, woff[NW];
    bool anyOver = false;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const int cw = S.cnt[w];
        anyOver |= cw == 0xFFFF;
        woff[w] = total;
        total += cw == 0xFFFF ? 0 : cw;
    }
    if (anyOver) return false;               // the tile path takes the group (every thread agrees)
    if (total > 0) {
        // slices -> position-ordered live indices (keys, offsets, elements)
        uint32_t sv[PER], sp[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = k * NT + tid;
            sv[k] = sp[k] = 0;
            if (i < total) {
                int w = 0;
#pragma unroll
                for (int x = 1; x < NW; ++x)
                    if (i >= woff[x]) w = x;
                const int src = w * CAP + (i - woff[w]);
                sv[k] = stVar[src];
                sp[k] = stPos[src];
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = k * NT + tid;
            if (i < total) {
                keyIn[pad(i)] = ((KeyT)sv[k] << POS_BITS) | (KeyT)i;
                S.livePos[i] = (uint16_t)(sp[k] & 0xFFFFu);
                S.mel[i] = (uint8_t)(sp[k] >> 16);
            }
        }
    }
    if (tid == 0) {
        S.nLive = total;
        S.nPend = 0;
    }
    __syncthreads();
    const int nl = total;
    if (p.phase_on && tid == 0) {
        atomicAdd(&g_scan_phase_cycles[8], (unsigned long long)nTiles);
        if (nl) atomicAdd(&g_scan_phase_cycles[9], 1ull);
        atomicAdd(&g_scan_phase_cycles[10], (unsigned long long)nl);
    }
    auto register_tiles = [&]() {
        if (tid == 0) {
            __threadfence();
            uint32_t w = (uint32_t)t0 >> 5, m = 0;
            for (int u = 0; u < nTiles; ++u) {
                const uint32_t tt = (uint32_t)(t0 + u);
                if ((tt >> 5) != w) {
                    atomicOr(p.regbits + w, m);
                    w = tt >> 5;
                    m = 0;
                }
                m |= 1u << (tt & 31);
            }
            atomicOr(p.regbits + w, m);
        }
    };
    if (nl == 0 && !p.guard) {
        // every op's variable was already stuck: all outputs are written
        register_tiles();
        return true;
    }
    const int D0 = 1 << p.digit_bits;
    for (int i = lane; i < D0; i += 32) S.hist[warp * D0 + i] = 0;
    __syncthreads();
    PHASE(1)

    // ---- 3. stable LSD radix sort of the live keys (by variable) -----------
    KeyT* kin = keyIn;
    KeyT* kout = S.vbuf[0];
    const bool rank_sort = nl <= RANK_SORT_MAX;
    if (nl > 0 && rank_sort) {
        if (tid < nl) {
            const KeyT kj = kin[pad(tid)];
            int r = 0;
            for (int i = 0; i < nl; ++i) r += kin[pad(i)] < kj;
            kout[pad(r)] = kj;
        }
        __syncthreads();
        KeyT* tk = kin;
        kin = kout;
        kout = tk;
    }
    for (int pass = 0; pass < (nl && !rank_sort ? p.passes : 0); ++pass) {
        const int D = 1 << p.digit_bits;
        const int shift = POS_BITS + pass * p.digit_bits;
        uint16_t* hrow = S.hist + warp * D;
        if (pass > 0) {
            for (int i = lane; i < D; i += 32) hrow[i] = 0;
            __syncwarp();
        }
        KeyT kk[E];
        uint16_t lr[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int pos = warp * 32 * E + e * 32 + lane;
            const bool ok = pos < nl;
            const KeyT key = ok ? kin[pad(pos)] : (KeyT)0;
            kk[e] = key;
            const uint32_t dig = ok ? (uint32_t)((key >> shift) & (KeyT)(D - 1)) : 0xFFFFFFFFu;
            const uint32_t peers = __match_any_sync(0xffffffffu, dig);
            const uint32_t rank = __popc(peers & lt);
            uint16_t c = 0;
            if (ok) c = hrow[dig];
            lr[e] = (uint16_t)(c + rank);
            __syncwarp();
            if (ok && rank == 0) hrow[dig] = (uint16_t)(c + __popc(peers));
            __syncwarp();
        }
        __syncthreads();
        {
            const int per = (D + NT - 1) / NT;
            const int d0 = tid * per;
            int sum = 0;
            for (int d = d0; d < d0 + per && d < D; ++d)
#pragma unroll
                for (int w = 0; w < NW; ++w) sum += S.hist[w * D + d];
            int run = block_excl_sum<NT>(sum, S.scanTmp, nullptr);
            for (int d = d0; d < d0 + per && d < D; ++d)
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    const int c = S.hist[w * D + d];
                    S.hist[w * D + d] = (uint16_t)run;
                    run += c;
                }
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int pos = warp * 32 * E + e * 32 + lane;
            if (pos < nl) {
                const uint32_t dig = (uint32_t)((kk[e] >> shift) & (KeyT)(D - 1));
                kout[pad(hrow[dig] + lr[e])] = kk[e];
            }
        }
        __syncthreads();
        KeyT* tk = kin;
        kin = kout;
        kout = tk;
    }
    PHASE(2)
    const KeyT* K = kin;                       // sorted keys: (variable, position in group)
    uint32_t* pend = reinterpret_cast<uint32_t*>(kout);   // the free buffer
    auto kvar = [&](int j) -> uint32_t { return (uint32_t)(K[pad(j)] >> POS_BITS); };
    auto kidx = [&](int j) -> int { return (int)(K[pad(j)] & (KeyT)(T - 1)); };
    // run key: variable and tile in group (runs never cross a tile)
    auto rkey = [&](int j) -> uint64_t {
        return ((uint64_t)kvar(j) << 8) | (uint64_t)(S.livePos[kidx(j)] >> POS_BITS);
    };

    // ---- 4a. run boundaries; stuck-shortcut loads ---------------------------
    const int j0 = tid * E;
    uint32_t headMask = 0, lastMask = 0;
    uint32_t ffv[E];
    {
        uint64_t prev = (j0 > 0 && j0 - 1 < nl) ? rkey(j0 - 1) : ~0ull;
        uint64_t cur = (j0 < nl) ? rkey(j0) : ~1ull;
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const int j = j0 + k;
            const uint64_t nxt = (j + 1 < nl) ? rkey(j + 1) : ~2ull;
            ffv[k] = 0xFFFFFFFFu;
            if (j < nl) {
                if (cur != prev) headMask |= 1u << k;
                if (nxt != cur) {
                    lastMask |= 1u << k;
                    const uint32_t v = (uint32_t)(cur >> 8);
                    ffv[k] = __ldcg(reinterpret_cast<const unsigned int*>(p.vff) + v);
                }
            }
            prev = cur;
            cur = nxt;
        }
    }

    // ---- 4b. segmented scan over runs (as in the tile path) ----------------
#define getb(w, k) (((w)[(k) >> 2] >> (8 * ((k) & 3))) & 0xFFu)
#define setb(w, k, v) ((w)[(k) >> 2] = ((w)[(k) >> 2] & ~(0xFFu << (8 * ((k) & 3)))) | ((uint32_t)(v) << (8 * ((k) & 3))))
    uint32_t pmw[E / 4], xmw[E / 4];
#pragma unroll
    for (int i = 0; i < E / 4; ++i) pmw[i] = xmw[i] = 0;
    const int nHeads = __popc(headMask);
    uint32_t acc = ID;
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const int j = j0 + k;
        if (j < nl) {
            const uint32_t m = S.mel[kidx(j)];
            if (headMask & (1u << k)) {
                acc = m;
            } else {
                setb(xmw, k, acc);
                acc = comp_of(S.comp, acc, m);
            }
            setb(pmw, k, acc);
        }
    }
    uint32_t carry;
    {
        uint32_t f = headMask != 0, v = acc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t fu = __shfl_up_sync(0xffffffffu, f, o);
            const uint32_t vu = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) {
                if (!f) v = comp_of(S.comp, vu, v);
                f |= fu;
            }
        }
        uint32_t fe = __shfl_up_sync(0xffffffffu, f, 1);
        uint32_t ve = __shfl_up_sync(0xffffffffu, v, 1);
        if (lane == 0) { fe = 0; ve = ID; }
        if (lane == 31) { S.segF[warp] = (uint8_t)f; S.segV[warp] = (uint8_t)v; }
        __syncthreads();
        if (warp == 0) {
            uint32_t wf = lane < NW ? S.segF[lane] : 0, wv = lane < NW ? S.segV[lane] : ID;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t fu = __shfl_up_sync(0xffffffffu, wf, o);
                const uint32_t vu = __shfl_up_sync(0xffffffffu, wv, o);
                if (lane >= o) {
                    if (!wf) wv = comp_of(S.comp, vu, wv);
                    wf |= fu;
                }
            }
            uint32_t xf = __shfl_up_sync(0xffffffffu, wf, 1);
            uint32_t xv = __shfl_up_sync(0xffffffffu, wv, 1);
            if (lane == 0) { xf = 0; xv = ID; }
            if (lane < NW) { S.segF[lane] = (uint8_t)xf; S.segV[lane] = (uint8_t)xv; }
        }
        __syncthreads();
        carry = fe ? ve : comp_of(S.comp, S.segV[warp], ve);
    }
#pragma unroll
    for (int k = 0; k < E; ++k) {
        if ((headMask & ((2u << k) - 1)) == 0) {
            setb(pmw, k, comp_of(S.comp, carry, getb(pmw, k)));
            setb(xmw, k, comp_of(S.comp, carry, getb(xmw, k)));
        }
    }
    const int runBase = block_excl_sum<NT>(nHeads, S.scanTmp, nullptr);
    auto run_id = [&](int k) { return runBase - 1 + __popc(headMask & ((2u << k) - 1)); };
    PHASE(3)

    // ---- 5a. run entry: stuck shortcut, or a node in the variable's list ----
    // node of run r in group tile g: (t0 + g) * T + r  (r < T: one per live op at most)
#pragma unroll
    for (int k = 0; k < E; ++k) {
        if (lastMask & (1u << k)) {
            const int r = run_id(k);
            const int g = S.livePos[kidx(j0 + k)] >> POS_BITS;
            const int64_t rbase = gbase + (int64_t)g * T;
            if ((ffv[k] & ~VFF_BOUND) < (uint32_t)rbase) {
                S.runEntry[r] = ST_F;
                const uint32_t v = kvar(j0 + k);
                if (v < (uint32_t)p.fbw * 32u) atomicOr(fsm + (v >> 5), 1u << (v & 31));
            } else {
                const uint32_t agg = getb(pmw, k);
                S.runEntry[r] = RUN_PENDING;
                if ((S.constF >> agg) & 1u) {
                    // stuck by the end of its tile: bound as first fault, no node
                    atomicMin(reinterpret_cast<uint32_t*>(p.vff) + kvar(j0 + k), (uint32_t)(rbase + T - 1) | VFF_BOUND);
                    pend[atomicAdd(&S.nPend, 1)] = (uint32_t)r | ((uint32_t)(j0 + k) << 16) | NO_NODE;
                } else {
                    pend[atomicAdd(&S.nPend, 1)] = (uint32_t)r | ((uint32_t)(j0 + k) << 16);
                    p.node_status[(uint32_t)(t0 + g) * (uint32_t)T + (uint32_t)r] = (uint8_t)(NODE_AGG | agg);
                }
            }
        }
    }
    __syncthreads();
    const int nPend = S.nPend;
    if (p.phase_on && tid == 0 && nPend) atomicAdd(&g_scan_phase_cycles[11], 1ull);
    constexpr int PW = 4;
    for (int lo = 0; lo < nPend; lo += NT * PW) {
        uint32_t c[PW], old[PW], node[PW], var[PW], ntile[PW];
        uint32_t mine = 0, simple = 0;
#pragma unroll
        for (int u = 0; u < PW; ++u) {
            const int i = lo + u * NT + tid;
            c[u] = NIL;
            node[u] = var[u] = ntile[u] = 0;
            if (i < nPend && !(pend[i] & NO_NODE)) {
                const uint32_t e = pend[i];
                const int j = (int)(e >> 16);
                mine |= 1u << u;
                ntile[u] = (uint32_t)t0 + (uint32_t)(S.livePos[kidx(j)] >> POS_BITS);
                node[u] = ntile[u] * (uint32_t)T + (e & 0xFFFFu);
                var[u] = kvar(j);
                c[u] = __ldcg(p.head + var[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < PW; ++u)
            if ((mine & (1u << u)) && (c[u] == NIL || c[u] / T < ntile[u])) {
                p.node_next[node[u]] = c[u];
                simple |= 1u << u;
            }
        __threadfence();
#pragma unroll
        for (int u = 0; u < PW; ++u) old[u] = (simple & (1u << u)) ? atomicCAS(p.head + var[u], c[u], node[u]) : c[u];
#pragma unroll
        for (int u = 0; u < PW; ++u) {
            if (!(mine & (1u << u)) || ((simple & (1u << u)) && old[u] == c[u])) continue;
            uint32_t* link = p.head + var[u];
            for (uint32_t it = 0;; ++it) {
                const uint32_t cc = ld_acquire(link);
                if (cc == NIL || cc / T < ntile[u]) {
                    p.node_next[node[u]] = cc;
                    __threadfence();
                    if (atomicCAS(link, cc, node[u]) == cc) break;
                } else {
                    link = p.node_next + cc;
                }
                if (it > SPIN_LIMIT) { raise_error(p.err, AMC_E_TIMEOUT); break; }
            }
        }
    }
    __syncthreads();
    PHASE(4)

    // ---- 5b. registration of the group's tiles; frontier --------------------
    register_tiles();
    if (nPend > 0 || p.guard) {
        uint32_t f0 = min(S.frontVal, (uint32_t)t0);
        for (uint32_t it = 0;; ++it) {
            bool all = true;
            for (uint32_t w = (f0 >> 5) + tid; f0 < (uint32_t)t0 && w <= ((uint32_t)t0 - 1) >> 5; w += NT) {
                const uint32_t lo = max(f0, w << 5), hi = min((uint32_t)t0, (w << 5) + 32);
                const uint32_t need = (hi - lo == 32) ? 0xFFFFFFFFu : (((1u << (hi - lo)) - 1u) << (lo & 31));
                all &= (__ldcg(p.regbits + w) & need) == need;
            }
            if (__syncthreads_and(all)) {
                if (tid == 0) {
                    __threadfence();
                    // the group's own tiles registered above
                    atomicMax(p.front, (uint32_t)(t0 + nTiles));
                    S.frontVal = (uint32_t)(t0 + nTiles);
                }
                break;
            }
            if (it > SPIN_LIMIT) { if (tid == 0) raise_error(p.err, AMC_E_TIMEOUT); break; }
            __nanosleep(128);
            if (tid == 0) S.frontVal = ld_acquire(p.front);
            __syncthreads();
            f0 = min(max(f0, S.frontVal), (uint32_t)t0);
            __syncthreads();
        }
        __threadfence();
    }
    PHASE(5)

    // ---- 5c. look-back along the lists -------------------------------------
    for (int lo = 0; lo < nPend; lo += NT * PW) {
        uint32_t q[PW], a[PW], st[PW], node[PW], var[PW], rr[PW], ffw[PW], rt[PW], ag[PW];
        uint32_t active = 0, nonode = 0;
#pragma unroll
        for (int u = 0; u < PW; ++u) {
            const int i = lo + u * NT + tid;
            a[u] = ID;
            st[u] = 0;
            q[u] = NIL;
            node[u] = var[u] = rr[u] = rt[u] = ag[u] = 0;
            ffw[u] = 0xFFFFFFFFu;
            if (i < nPend) {
                const uint32_t e = pend[i];
                const int j = (int)((e >> 16) & 0x7FFFu);
                active |= 1u << u;
                rr[u] = e & 0xFFFFu;
                rt[u] = (uint32_t)t0 + (uint32_t)(S.livePos[kidx(j)] >> POS_BITS);     // the run's tile
                var[u] = kvar(j);
                if (e & NO_NODE) {
                    nonode |= 1u << u;
                    q[u] = ld_acquire(p.head + var[u]);         // from the newest node
                } else {
                    node[u] = rt[u] * (uint32_t)T + rr[u];
                    q[u] = ld_acquire(p.node_next + node[u]);
                    ag[u] = __ldcg(p.node_status + node[u]) & 31u;   // the run's aggregate (AGG status)
                }
                ffw[u] = ld_acquire(reinterpret_cast<const uint32_t*>(p.vff) + var[u]);
            }
        }
        const uint32_t mine = active;
#pragma unroll
        for (int u = 0; u < PW; ++u)
            if ((active & (1u << u)) && (ffw[u] & ~VFF_BOUND) < rt[u] * (uint32_t)T) {
                st[u] = ST_F;                  // stuck before the run's tile (bound published since)
                active &= ~(1u << u);
            }
        for (uint32_t hop = 0; active; ++hop) {
            // a node's status and its next pointer are read together: below
            // the walking tile the list no longer changes (every earlier tile
            // has inserted before the frontier passed), and either status of
            // a node (aggregate or inclusive) is a valid answer
            uint32_t sv[PW], nx[PW];
#pragma unroll
            for (int u = 0; u < PW; ++u) {
                sv[u] = 0;
                nx[u] = NIL;
                if ((active & (1u << u)) && q[u] != NIL) {
                    sv[u] = ld_relaxed_u8(p.node_status + q[u]);
                    nx[u] = ld_relaxed(p.node_next + q[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < PW; ++u) {
                if (!(active & (1u << u))) continue;
                if (q[u] == NIL) {
                    st[u] = p.init ? p.init[var[u]] : (uint32_t)AMC_ST_VI;
                    active &= ~(1u << u);
                } else if (q[u] / T >= rt[u]) {
                    // a node of the run's tile or a later one (walks that start at the head)
                } else if (sv[u] & NODE_INCL) {
                    st[u] = sv[u] & 7u;
                    active &= ~(1u << u);
                } else {
                    a[u] = comp_of(S.comp, sv[u] & 31u, a[u]);     // earlier tile first
                    if ((S.constF >> a[u]) & 1u) {                  // entry F (absorbing)
                        st[u] = 0;
                        active &= ~(1u << u);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < PW; ++u)
                if (active & (1u << u)) q[u] = nx[u];
            if (hop > SPIN_LIMIT) { raise_error(p.err, AMC_E_TIMEOUT); break; }
        }
#pragma unroll
        for (int u = 0; u < PW; ++u) {
            if (!(mine & (1u << u))) continue;
            const uint32_t entry = S.app[a[u] * 8 + st[u]];
            S.runEntry[rr[u]] = (uint8_t)entry;
            if (!(nonode & (1u << u)))
                st_relaxed_u8(p.node_status + node[u], NODE_INCL | S.app[ag[u] * 8 + entry]);
        }
    }
    __syncthreads();
    PHASE(6)

    // ---- 6. outputs of the live ops (byte stores); first faults -------------
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const int j = j0 + k;
        if (j < nl) {
            const uint32_t e = S.runEntry[run_id(k)];
            const uint32_t pre = S.app[getb(xmw, k) * 8 + e];
            const uint32_t post = S.app[getb(pmw, k) * 8 + e];
            const int64_t gpos = gbase + (int64_t)S.livePos[kidx(j)];
            p.step[gpos] = (uint8_t)(p.pre_mode ? pre : post);
            if (post == ST_F && pre != ST_F) {
                const uint32_t gi = (uint32_t)gpos;
                const uint32_t v = kvar(j);
                atomicMin(reinterpret_cast<uint32_t*>(p.vff) + v, gi);
                atomicOr(p.fbits + (v >> 5), 1u << (v & 31));
                atomicOr(p.fbits + p.fbits_words + (v >> 5), 1u << (v & 31));
                if (v < (uint32_t)p.fbw * 32u) atomicOr(fsm + (v >> 5), 1u << (v & 31));
                // the global minimum only falls: skip the atomic once it is below gi
                if ((unsigned long long)gi < *reinterpret_cast<volatile unsigned long long*>(p.first_fault))
                    atomicMin(reinterpret_cast<unsigned long long*>(p.first_fault), (unsigned long long)gi);
            }
        }
    }
#undef getb
#undef setb
    PHASE(7)
#undef PHASE
    return true;
}

template <typename KeyT, int T, int NT>
__device__ __forceinline__ void issue_tile(const ScanParams& p, ScanSmem<KeyT, T, NT>& S, int b, int t)
{
    const int64_t base = (int64_t)t * T;
    S.viaBulk[b] = 0;
    if (t < S.nTiles && base + T <= S.nOps && p.bulk_ok) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&S.mbar[b], (uint32_t)(T + 4 * T));
        bulk_g2s(S.kind[b], p.kind_side + base, T, &S.mbar[b]);
        bulk_g2s(S.vbuf[b], p.var + base, 4 * T, &S.mbar[b]);
        S.viaBulk[b] = 1;
    }
}

template <typename KeyT, int T, int NT>
__global__ void __launch_bounds__(NT, MAX_CTAS_PER_SM) scan_trace_kernel(const ScanParams p)
{
    extern __shared__ __align__(128) uint8_t smem_raw[];
    // gated off: return before touching the tile counter or any other state
    // (a gated launch's set-up is gated the same way, so that state is stale)
    if (p.gate && ((*p.gate != 0) != (p.gate_on != 0))) return;
    ScanSmem<KeyT, T, NT>& S = *reinterpret_cast<ScanSmem<KeyT, T, NT>*>(smem_raw);
    uint32_t* fsm = reinterpret_cast<uint32_t*>(smem_raw + sizeof(ScanSmem<KeyT, T, NT>));
    const int tid = threadIdx.x;
    for (int i = tid; i < MAX_ELEMS * MAX_ELEMS; i += NT) S.comp[i] = p.tab.comp[i];
    for (int i = tid; i < MAX_ELEMS * 8; i += NT) S.app[i] = p.tab.app[i];
    for (int i = tid; i < 256; i += NT) S.elem_of[i] = p.tab.elem_of[i];
    if (tid < 32) {
        // element e is the constant F function when it sends all four
        // non-stuck statuses to F (F itself is absorbing)
        const uint32_t e = (uint32_t)tid;
        bool cf = e < (uint32_t)p.tab.n_elems;
        for (int st = 0; st < 4; ++st) cf = cf && p.tab.app[e * 8 + st] == ST_F;
        const uint32_t m = __ballot_sync(0xffffffffu, cf);
        if (tid == 0) S.constF = m;
    }
    for (int i = tid; i < p.fbw; i += NT) fsm[i] = __ldcg(p.fbits + i);
    if (tid == 0) {
        mbar_init(&S.mbar[0], 1);
        fence_mbar_init();
        S.frontVal = 0;
        int64_t n = p.n_ops;
        if (p.n_dev) {
            const int64_t d = *p.n_dev;
            n = d < 0 ? 0 : (d < n ? d : n);
        }
        if (p.gate && ((*p.gate != 0) != (p.gate_on != 0))) n = 0;    // gated off: no work
        S.nOps = n;
        S.nTiles = (int)((n + T - 1) / T);
    }
    uint32_t parity = 0;
    long long last = clock64();
    uint32_t done = 0;               // tiles this CTA has processed (bitmap refresh clock)
    uint32_t est = T;                // live ops per tile lately (thread 0's estimate)
    bool failed = false;
    // A CTA takes the next tile ids only when it starts them: every tile below
    // an id being processed has then started too, so it reaches its
    // registration within one pre-registration phase (no queued tiles, no
    // convoys of waits through other CTAs' queues).  Where few ops are live
    // the CTA takes a group of tiles at once (group path), sized so that the
    // expected live ops fill about half of the shared buffers.
    while (!failed) {
        if (tid == 0) {
            int G = 1;
            if (p.group_max > 1) {
                G = p.group_max;
                while (!p.group_force && G > 1 && (uint32_t)G * est > (uint32_t)GROUP_LIVE_TARGET) G >>= 1;
            }
            const int t = (int)atomicAdd(p.tile_counter, (uint32_t)G);
            S.tile[0] = t;
            S.grp[0] = G;
            if (G == 1) issue_tile<KeyT, T, NT>(p, S, 0, t);
        }
        __syncthreads();
        const int t = S.tile[0];
        const int G = S.grp[0];
        if (t >= S.nTiles) break;
        if (G > 1) {
            if (process_group<KeyT, T, NT>(p, S, fsm, t, G, done, last)) {
                const int nt = min(G, S.nTiles - t);
                if (tid == 0) est = (est + (uint32_t)S.nLive / (uint32_t)nt + 1) / 2;
                done += (uint32_t)nt;
                __syncthreads();
                continue;
            }
            // more live ops than one group holds: its tiles one by one
            if (tid == 0) est = T;
            for (int u = 0; u < G && t + u < S.nTiles && !failed; ++u) {
                __syncthreads();
                if (tid == 0) issue_tile<KeyT, T, NT>(p, S, 0, t + u);
                __syncthreads();
                bool ok = true;
                if (S.viaBulk[0]) {
                    ok = mbar_wait_bounded(&S.mbar[0], parity, p.err);
                    parity ^= 1;
                }
                if (__syncthreads_or(!ok)) {
                    if (tid == 0) mbar_wait_bounded(&S.mbar[0], parity ^ 1, p.err);   // drain, bounded
                    failed = true;
                    break;
                }
                process_tile<KeyT, T, NT>(p, S, fsm, t + u, 0, done++, last);
                __syncthreads();
            }
            continue;
        }
        bool ok = true;
        if (S.viaBulk[0]) {
            ok = mbar_wait_bounded(&S.mbar[0], parity, p.err);
            parity ^= 1;
        }
        if (__syncthreads_or(!ok)) {
            if (tid == 0) mbar_wait_bounded(&S.mbar[0], parity ^ 1, p.err);   // drain, bounded
            break;
        }
        if (p.phase_on && tid == 0) {
            const long long now = clock64();
            atomicAdd(&g_scan_phase_cycles[0], (unsigned long long)(now - last));
            last = now;
        }
        process_tile<KeyT, T, NT>(p, S, fsm, t, 0, done++, last);
        if (tid == 0) est = (est + (uint32_t)S.nLive + 1) / 2;
        __syncthreads();
    }
}

__global__ void finalize_trace_kernel(int32_t* __restrict__ vff, const uint32_t* __restrict__ head,
                                      const uint8_t* __restrict__ node_status, const uint8_t* __restrict__ init,
                                      int32_t n_vars, uint8_t* __restrict__ final_status, const int* gate,
                                      int gate_on)
{
    if (gate && ((*gate != 0) != (gate_on != 0))) return;     // gated off: the other launch writes
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_vars; v += stride) {
        const uint32_t ff = (uint32_t)vff[v];
        uint8_t f;
        if (ff != 0xFFFFFFFFu) {
            f = ST_F;
            if (ff & VFF_BOUND) vff[v] = -1;   // stuck from the start: no fault inside the trace
        } else {
            const uint32_t h = head[v];
            f = (h == NIL) ? (init ? init[v] : (uint8_t)AMC_ST_VI) : (uint8_t)(node_status[h] & 7u);
        }
        if (final_status) final_status[v] = f;
    }
}

// Variables whose initial status is F are stuck before the first op: their
// bits go into both copies of the stuck bitmap before the scan starts.
__global__ void seed_stuck_kernel(const uint8_t* __restrict__ init, int32_t n_vars, uint32_t* __restrict__ fbits,
                                  int fbits_words, const int* gate, int gate_on)
{
    if (gate && ((*gate != 0) != (gate_on != 0))) return;
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool f = v < n_vars && init[v] == ST_F;
    const uint32_t m = __ballot_sync(0xffffffffu, f);
    if ((threadIdx.x & 31) == 0 && m) {
        const int64_t w = v >> 5;
        fbits[w] = m;
        fbits[w + fbits_words] = m;
    }
}

// The set-up of a gated launch, done on the device so that a launch gated off
// costs no memsets: list heads, first faults and the global first fault to -1,
// registration bits and the tile counter / frontier to 0, both copies of the
// stuck bitmap from the initial statuses (F: stuck before the first op).
__global__ void gated_init_kernel(const int* gate, int gate_on, uint32_t* __restrict__ head,
                                  int32_t* __restrict__ vff, int32_t n_vars, int64_t* __restrict__ ff,
                                  uint32_t* __restrict__ regbits, int64_t reg_words, uint32_t* __restrict__ fbits,
                                  int64_t f_words, const uint8_t* __restrict__ init,
                                  uint32_t* __restrict__ tile_counter)
{
    if ((*gate != 0) != (gate_on != 0)) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t v = g; v < n_vars; v += stride) {
        head[v] = NIL;
        vff[v] = -1;
    }
    for (int64_t w = g; w < reg_words; w += stride) regbits[w] = 0;
    for (int64_t w = g; w < f_words; w += stride) {            // f_words per copy
        uint32_t m = 0;
        if (init)
            for (int j = 0; j < 32; ++j) {
                const int64_t v = 32 * w + j;
                if (v < n_vars && init[v] == ST_F) m |= 1u << j;
            }
        fbits[w] = m;
        fbits[w + f_words] = m;
    }
    if (g == 0) {
        *ff = -1;
        tile_counter[0] = 0;
        tile_counter[1] = 0;
    }
}

template <typename KeyT>
int launch_kernel(ScanParams p, const ScanLaunch& L, cudaStream_t s)
{
    int dev = 0;
    cudaGetDevice(&dev);
    int max_optin = 0;
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int64_t room = ((int64_t)max_optin - (int64_t)sizeof(ScanSmem<KeyT, TILE, THREADS>) - 1024) / 16 * 4;
    if (p.fbw > room) p.fbw = room > 0 ? (int)room : 0;          // shared bitmap words (multiple of 4)
    const size_t smem = sizeof(ScanSmem<KeyT, TILE, THREADS>) + 4 * (size_t)p.fbw;
    static size_t attr_set[64] = {};
    if (dev >= 64 || attr_set[dev] != smem) {
        if (cudaFuncSetAttribute(scan_trace_kernel<KeyT, TILE, THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return AMC_E_CUDA;
        // ask for the smallest shared-memory carve-out that still holds the
        // resident CTAs, so that the rest of the SM's memory serves as L1 for
        // the stuck bitmap
        int per_sm_smem = 0;
        cudaDeviceGetAttribute(&per_sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (per_sm_smem > 0) {
            const size_t need = (size_t)MAX_CTAS_PER_SM * (smem + 1024);
            const int pct = (int)min((size_t)100, (need * 100 + (size_t)per_sm_smem - 1) / (size_t)per_sm_smem);
            cudaFuncSetAttribute(scan_trace_kernel<KeyT, TILE, THREADS>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout, pct);
        }
        if (dev < 64) attr_set[dev] = smem;
    }
    int n_sm = 0, per_sm = 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scan_trace_kernel<KeyT, TILE, THREADS>, THREADS, smem);
    if (per_sm < 1) per_sm = 1;
    if (L.ctas_per_sm > 0 && L.ctas_per_sm < per_sm) per_sm = L.ctas_per_sm;
    if (const char* e = getenv("AMC_SCAN_CTAS_PER_SM")) per_sm = max(1, min(atoi(e), per_sm));   // tuning override
    int grid = n_sm * per_sm;
    if (grid > p.n_tiles) grid = p.n_tiles;
    if (L.max_ctas > 0 && grid > L.max_ctas) grid = L.max_ctas;
    if (L.profile & 1) profile_begin(s);
    scan_trace_kernel<KeyT, TILE, THREADS><<<grid, THREADS, smem, s>>>(p);
    if (cudaGetLastError() != cudaSuccess) return AMC_E_CUDA;
    if (L.profile & 2) profile_end(s);
    return AMC_OK;
}

}  // namespace

int scan_tile_size() { return TILE; }

namespace {
bool g_phase_on = false;
}

int scan_phase_profile(int enable, unsigned long long* host_out)
{
    if (host_out &&
        cudaMemcpyFromSymbol(host_out, g_scan_phase_cycles, sizeof(unsigned long long) * N_PHASES) != cudaSuccess)
        return AMC_E_CUDA;
    if (enable >= 0) {
        g_phase_on = enable != 0;
        unsigned long long z[N_PHASES] = {};
        if (cudaMemcpyToSymbol(g_scan_phase_cycles, z, sizeof(z)) != cudaSuccess) return AMC_E_CUDA;
    }
    return AMC_OK;
}

size_t scan_workspace_bytes(int64_t n_ops, int32_t n_vars, bool with_dense)
{
    const int64_t n_tiles = (n_ops + TILE - 1) / TILE;
    size_t b = 0;
    b += align_up(4 * (size_t)n_vars, 256);                 // head
    b += align_up(4 * (size_t)n_tiles * TILE, 256);         // node_next
    b += align_up((size_t)n_tiles * TILE, 256);             // node_status
    b += align_up(4 * (size_t)((n_tiles + 31) / 32), 256);  // registration bits
    b += 2 * align_up(16 * (size_t)((n_vars + 127) / 128), 256); // stuck bitmap, two copies
    b += 256;                                               // tile counter, frontier
    if (with_dense) {
        b += scan_dense_workspace_bytes(n_ops, n_vars);    // reduce / carry / apply path
        const size_t t = scan_tail_workspace_bytes(n_ops, n_vars);   // epochs of a long trace
        if (t > b) b = t;
    }
    return b;
}

int scan_trace_plan(const ScanLaunch& L, int* launches)
{
    int n = 2, path = AMC_PATH_SCAN;                        // scan, final statuses
    const bool plain = !L.n_dev && !L.gate;
    if (scan_small_eligible(L)) {
        n = 1;
        path = AMC_PATH_SMALL;
    } else if (scan_tail_eligible(L)) {
        n = scan_tail_launches(L);
        path = AMC_PATH_EPOCHS;
    } else if (L.dense != 0 && plain &&
               ((L.dense == 1 && dense_forced_ok(L.n_ops, L.n_vars)) || scan_dense_eligible(L.n_ops, L.n_vars))) {
        const char* e = getenv("AMC_SCAN_DENSE_SORT");
        const bool warp = L.n_vars <= 8192 && !(e && e[0] == '1');
        n = warp ? 5 : 3;                                   // chunk, reduce, carry, expand, chunk; or reduce, carry, apply
        path = warp ? AMC_PATH_WARP_DENSE : AMC_PATH_DENSE;
    } else if (L.dense != 0 && (L.prefix_log2 > 0 ? scan_forced_prefix(L)
                                                  : plain && scan_prefix_eligible(L.n_ops, L.n_vars, L.init != nullptr))) {
        n = 7;                                              // prefix (3), bitmap seed, scan (2), merge
        path = AMC_PATH_PREFIX;
    }
    if (launches) *launches = n;
    return path;
}

int launch_scan_trace(const ScanLaunch& L, cudaStream_t s)
{
    if (scan_small_eligible(L)) return launch_scan_small(L, s);
    if (scan_tail_eligible(L)) return launch_scan_tail(L, s);
    ScanParams p{};
    p.kind_side = L.kind_side;
    p.var = L.var;
    p.n_ops = L.n_ops;
    p.n_dev = L.n_dev;
    p.gate = L.gate;
    p.gate_on = L.gate_on;
    p.n_vars = L.n_vars;
    p.init = L.init;
    p.step = L.step;
    p.vff = L.vff;
    p.first_fault = L.first_fault;
    p.guard = L.guard;
    p.pre_mode = L.pre_mode;
    p.err = L.err;
    p.phase_on = g_phase_on;
    p.tab = host_tables();
    p.n_tiles = (int)((L.n_ops + TILE - 1) / TILE);
    uint8_t* w = static_cast<uint8_t*>(L.workspace);
    p.head = reinterpret_cast<uint32_t*>(w);
    w += align_up(4 * (size_t)L.n_vars, 256);
    p.node_next = reinterpret_cast<uint32_t*>(w);
    w += align_up(4 * (size_t)p.n_tiles * TILE, 256);
    p.node_status = w;
    w += align_up((size_t)p.n_tiles * TILE, 256);
    p.regbits = reinterpret_cast<uint32_t*>(w);
    const size_t regbytes = 4 * (size_t)((p.n_tiles + 31) / 32);
    w += align_up(regbytes, 256);
    p.fbits = reinterpret_cast<uint32_t*>(w);
    const size_t fbytes = 2 * align_up(16 * (size_t)((L.n_vars + 127) / 128), 256);
    p.fbits_words = (int)(fbytes / 8);
    w += fbytes;
    {
        // shared copy of the stuck bitmap: the first fb_max_bits variables
        const int64_t words = (int64_t)(fbytes / 4);
        int64_t bits = L.fb_max_bits ? L.fb_max_bits : DEFAULT_FB_BITS;
        if (const char* e = getenv("AMC_SCAN_FB_BITS")) bits = atoll(e);       // tuning override
        // > 0: shared copy of the first `bits` variables, the rest live;
        // -2: L1-cached global copies; < -2: shared copy of the first -bits
        // variables (the most frequent ids of a Zipf trace), the rest L1
        p.fb_mode = bits > 0 ? 1 : (bits == -2 ? 2 : (bits < -2 ? 3 : 0));
        const int64_t cap = (bits > 0 ? bits / 32 : (bits < -2 ? -bits / 32 : 0)) & ~(int64_t)3;
        p.fbw = (int)(words < cap ? words : cap);
    }
    p.tile_counter = reinterpret_cast<uint32_t*>(w);
    p.front = p.tile_counter + 1;
    const bool plain = !L.n_dev && !L.gate;
    const bool dense_forced = L.dense == 1 && dense_forced_ok(L.n_ops, L.n_vars);
    if (L.dense != 0 && plain && (dense_forced || scan_dense_eligible(L.n_ops, L.n_vars)))
        return launch_scan_dense(L, w + 256, s);
    if (L.dense != 0 && (L.prefix_log2 > 0 ? scan_forced_prefix(L)
                                           : plain && scan_prefix_eligible(L.n_ops, L.n_vars, L.init != nullptr)))
        return launch_scan_prefix(L, w + 256, s);
    // key bits: var ids are < n_vars; at most MAX_DIGIT_BITS per pass
    int kb = 1;
    while (kb < 31 && ((int64_t)1 << kb) < (int64_t)L.n_vars) ++kb;
    p.passes = (kb + MAX_DIGIT_BITS - 1) / MAX_DIGIT_BITS;
    p.group_max = L.group_max > 0 ? min(L.group_max, GROUP_MAX) : GROUP_MAX;
    if (const char* e = getenv("AMC_SCAN_GROUP")) {
        // tuning and test override: N = at most N tiles per claim, -N = always N
        const int g = atoi(e);
        p.group_max = max(1, min(g < 0 ? -g : g, GROUP_MAX));
        p.group_force = g < 0;
    }
    p.digit_bits = (kb + p.passes - 1) / p.passes;
    p.bulk_ok = ((uintptr_t)L.kind_side % 16 == 0) && ((uintptr_t)L.var % 16 == 0) &&
                ((uintptr_t)L.step % 16 == 0);

    if (L.gate) {
        // a gated launch (the epoch path's fallback) sets itself up on the device
        const int64_t nw = L.n_vars > (int64_t)(fbytes / 4) ? L.n_vars : (int64_t)(fbytes / 4);
        int n_sm = 0, dv = 0;
        cudaGetDevice(&dv);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dv);
        const int64_t cap = n_sm > 0 ? 4 * (int64_t)n_sm : 4096;       // grid-stride; a gated-off launch is cheap
        const int nb = (int)((nw + 255) / 256 < cap ? (nw + 255) / 256 : cap);
        gated_init_kernel<<<nb > 0 ? nb : 1, 256, 0, s>>>(L.gate, L.gate_on, p.head, L.vff, L.n_vars,
                                                          L.first_fault, p.regbits, L.n_ops > 0 ? regbytes / 4 : 0,
                                                          p.fbits, L.n_ops > 0 ? p.fbits_words : 0, L.init,
                                                          p.tile_counter);
        if (cudaGetLastError() != cudaSuccess) return AMC_E_CUDA;
    } else {
        if (cudaMemsetAsync(p.head, 0xFF, 4 * (size_t)L.n_vars, s) != cudaSuccess) return AMC_E_CUDA;
        if (cudaMemsetAsync(L.vff, 0xFF, 4 * (size_t)L.n_vars, s) != cudaSuccess) return AMC_E_CUDA;
        if (cudaMemsetAsync(L.first_fault, 0xFF, 8, s) != cudaSuccess) return AMC_E_CUDA;
    }
    if (L.n_ops > 0) {
        if (!L.gate) {
            if (cudaMemsetAsync(p.regbits, 0, regbytes, s) != cudaSuccess) return AMC_E_CUDA;
            if (fbytes && cudaMemsetAsync(p.fbits, 0, fbytes, s) != cudaSuccess) return AMC_E_CUDA;
        }
        if (L.init && L.n_vars > 0 && !L.gate) {
            seed_stuck_kernel<<<(unsigned)((L.n_vars + 255) / 256), 256, 0, s>>>(L.init, L.n_vars, p.fbits,
                                                                                p.fbits_words, L.gate, L.gate_on);
            if (cudaGetLastError() != cudaSuccess) return AMC_E_CUDA;
        }
        if (!L.gate && cudaMemsetAsync(p.tile_counter, 0, 8, s) != cudaSuccess) return AMC_E_CUDA;
        // keys pack (var << 12 | position): 32-bit while var ids fit 20 bits
        const int rc = kb + POS_BITS <= 32 ? launch_kernel<uint32_t>(p, L, s) : launch_kernel<uint64_t>(p, L, s);
        if (rc) return rc;
    }
    {
        // final statuses (when asked for) and first-fault bounds cleared
        int n_sm = 0, dv = 0;
        cudaGetDevice(&dv);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dv);
        const int64_t cap = n_sm > 0 ? 8 * (int64_t)n_sm : 4096;       // grid-stride
        const int nb = (int)((L.n_vars + 255) / 256 < cap ? (L.n_vars + 255) / 256 : cap);
        if (nb > 0) {
            finalize_trace_kernel<<<nb, 256, 0, s>>>(L.vff, p.head, p.node_status, L.init, L.n_vars,
                                                     L.final_status, L.gate, L.gate_on);
            if (cudaGetLastError() != cudaSuccess) return AMC_E_CUDA;
        }
    }
    return AMC_OK;
}

}  // namespace amc
