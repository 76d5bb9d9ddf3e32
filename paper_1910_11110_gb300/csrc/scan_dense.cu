// scan_dense.cu -- the trace check for traces over few variables (reduce,
// carry, apply), where nearly every op stays live.
//
// What it computes is what scan_trace.cu computes: for every op the status of
// its variable after (or, in the guard pass, before) the op, by applying the
// transfer functions of Fig. Opsem in trace order; sequencing is associative
// (Section 3.2), so the trace may be cut into chunks whose per-variable
// compositions are combined afterwards.
//
// Over few variables the per-variable lists of the single-pass kernel become
// long and every tile in flight contends for the same ones.  Here instead:
//  1. reduce: CTA c takes chunk c (consecutive 4,096-op tiles) and, tile by
//     tile, sorts the ops by variable, composes each variable's run and folds
//     it into a dense per-variable element vector in shared memory; the vector
//     is written out (one byte per variable and chunk);
//  2. carry: one thread per variable walks the chunks in order, applying the
//     chunk aggregates to the initial status: the status at every chunk entry
//     and the final status;
//  3. apply: CTA c runs its tiles again from the entry statuses, writes every
//     op's status, the per-variable first faults (atomicMin) and the global one.
// No CTA waits on another, so the grid may exceed what is resident.
#include <cstdlib>

#include "amc_internal.cuh"
#include "scan_trace.cuh"

namespace amc {

namespace {

constexpr int DT = 4096;                 // ops per tile
constexpr int DNT = 256;                 // threads per CTA
constexpr int DE = DT / DNT;             // sorted slots per thread
constexpr int DNW = DNT / 32;
constexpr int DPOS = 12;                 // log2(DT): position bits of a key
constexpr int DDIG = 7;                  // radix digit bits
constexpr int DENSE_MAX_VARS = 16384;    // the dense vector lives in shared memory
constexpr int DENSE_MAX_CHUNKS = 2048;
constexpr int64_t DENSE_MIN_OPS = 1 << 10;

__device__ __forceinline__ int dpad(int i) { return i + (i >> 5); }

struct DenseParams {
    const uint8_t* kind_side;
    const int32_t* var;
    int64_t n_ops;
    int64_t n_ops_follow;                // ops readable after position i (a GT's EN may lie beyond n_ops)
    int32_t n_vars;
    const uint8_t* init;
    uint8_t* step;
    int32_t* vff;
    int64_t* first_fault;
    uint8_t* final_status;
    const uint8_t* guard;
    int pre_mode;
    int* err;
    uint8_t* aggs;                       // [n_chunks][n_vars] chunk aggregates (elements)
    uint8_t* entry;                      // [n_chunks][n_vars] statuses at chunk entry
    int n_tiles;
    int n_chunks;
    int tiles_per_chunk;
    int passes;
    int digit_bits;
    Tables tab;
};

struct __align__(16) DenseSmem {
    uint32_t keyA[DT + DT / 32];
    uint32_t keyB[DT + DT / 32];         // staged var ids, then a sort buffer
    uint8_t kind[DT];
    uint8_t mel[DT];                     // element of each op, by position
    uint8_t out[DT];
    uint16_t hist[DNW << DDIG];
    uint8_t comp[MAX_ELEMS * MAX_ELEMS];
    uint8_t app[MAX_ELEMS * 8];
    uint8_t elem_of[256];
    int scanTmp[DNW + 2];
    uint8_t segF[DNW];
    uint8_t segV[DNW];
    // followed (dynamic shared memory) by the per-variable vector: n_vars bytes
};

// One tile: load, decode, sort by variable, segmented scan; then either fold
// the runs into the aggregate vector (REDUCE) or emit the ops' statuses from
// the status vector and advance it (APPLY).
template <bool APPLY>
__device__ void dense_tile(const DenseParams& p, DenseSmem& S, uint8_t* vec, const int t)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = lanemask_lt();
    const uint32_t ID = p.tab.identity;
    const int64_t base = (int64_t)t * DT;
    const int n = (int)min((int64_t)DT, p.n_ops - base);
    int32_t* vraw = reinterpret_cast<int32_t*>(S.keyB);

    // ---- load (coalesced 16-byte loads for a full, aligned tile) ------------
    const bool vec16 = n == DT && ((uintptr_t)(p.kind_side + base) % 16 == 0) && ((uintptr_t)(p.var + base) % 16 == 0);
    if (vec16) {
        for (int i = tid; i < DT / 16; i += DNT)
            reinterpret_cast<uint4*>(S.kind)[i] = __ldcs(reinterpret_cast<const uint4*>(p.kind_side + base) + i);
        for (int i = tid; i < DT / 4; i += DNT)
            reinterpret_cast<int4*>(vraw)[i] = __ldcs(reinterpret_cast<const int4*>(p.var + base) + i);
    } else {
        for (int i = tid; i < n; i += DNT) {
            S.kind[i] = p.kind_side[base + i];
            vraw[i] = p.var[base + i];
        }
    }
    __syncthreads();

    // ---- decode: element per op, validation, keys (var << 12 | position) ----
    for (int i = tid; i < n; i += DNT) {
        const uint32_t ks = S.kind[i];
        if ((ks & 0xE0u) || (ks & 15u) > AMC_K_EN) raise_error(p.err, AMC_E_INVALID);
        int32_t v = vraw[i];
        if (v < 0 || v >= p.n_vars) {
            raise_error(p.err, AMC_E_RANGE);
            v = 0;
        }
        uint32_t m = S.elem_of[ks];
        if (m == ELEM_GT) {
            // GT must be followed by EN of the same side on another variable
            const int64_t gi = base + i;
            uint32_t nks = 0xFF;
            int32_t nv = v;
            if (gi + 1 < p.n_ops_follow) {
                nks = (i + 1 < n) ? S.kind[i + 1] : p.kind_side[gi + 1];
                nv = (i + 1 < n) ? vraw[i + 1] : p.var[gi + 1];
            }
            const bool gt_ok = (nks & 15) == AMC_K_EN && (nks >> 4) == (ks >> 4) && nv != v;
            if (!gt_ok) raise_error(p.err, AMC_E_INVALID);
            if (!gt_ok || p.pre_mode) {
                m = ID;                              // guard pass: GT does not touch guards
            } else if (!p.guard) {
                raise_error(p.err, AMC_E_INVALID);   // GT needs the guarded entry point
                m = ID;
            } else {
                // guard = status of the EN's variable before the EN (guard pass)
                const uint32_t gs = p.guard[gi + 1];
                const int side = ks >> 4;
                const bool valid = gs != ST_F && (gs & (side == 0 ? 1u : 2u));
                m = valid ? ID : p.tab.pull_of_side[side];
            }
        } else if (m == ELEM_BAD) {
            m = ID;
        }
        S.mel[i] = (uint8_t)m;
        S.keyA[dpad(i)] = ((uint32_t)v << DPOS) | (uint32_t)i;
    }
    __syncthreads();

    // ---- stable LSD radix sort by variable (warp ranking with match.any) ----
    uint32_t* kin = S.keyA;
    uint32_t* kout = S.keyB;
    for (int pass = 0; pass < p.passes; ++pass) {
        const int D = 1 << p.digit_bits;
        const int shift = DPOS + pass * p.digit_bits;
        uint16_t* hrow = S.hist + warp * D;
        for (int i = lane; i < D; i += 32) hrow[i] = 0;
        __syncwarp();
        uint32_t kk[DE];
        uint16_t lr[DE];
#pragma unroll
        for (int e = 0; e < DE; ++e) {
            const int pos = warp * 32 * DE + e * 32 + lane;
            const bool ok = pos < n;
            const uint32_t key = ok ? kin[dpad(pos)] : 0u;
            kk[e] = key;
            const uint32_t dig = ok ? ((key >> shift) & (uint32_t)(D - 1)) : 0xFFFFFFFFu;
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
            const int per = (D + DNT - 1) / DNT;
            const int d0 = tid * per;
            int sum = 0;
            for (int d = d0; d < d0 + per && d < D; ++d)
#pragma unroll
                for (int w = 0; w < DNW; ++w) sum += S.hist[w * D + d];
            int run = block_excl_sum<DNT>(sum, S.scanTmp, nullptr);
            for (int d = d0; d < d0 + per && d < D; ++d)
#pragma unroll
                for (int w = 0; w < DNW; ++w) {
                    const int c = S.hist[w * D + d];
                    S.hist[w * D + d] = (uint16_t)run;
                    run += c;
                }
        }
        __syncthreads();
#pragma unroll
        for (int e = 0; e < DE; ++e) {
            const int pos = warp * 32 * DE + e * 32 + lane;
            if (pos < n) {
                const uint32_t dig = (kk[e] >> shift) & (uint32_t)(D - 1);
                kout[dpad(hrow[dig] + lr[e])] = kk[e];
            }
        }
        __syncthreads();
        uint32_t* tk = kin;
        kin = kout;
        kout = tk;
    }
    const uint32_t* K = kin;
    auto kvar = [&](int j) -> uint32_t { return K[dpad(j)] >> DPOS; };
    auto kpos = [&](int j) -> int { return (int)(K[dpad(j)] & (uint32_t)(DT - 1)); };

    // ---- segmented scan over runs (blocked: thread owns DE sorted slots) -----
    const int j0 = tid * DE;
    uint32_t headMask = 0, lastMask = 0;
    {
        uint32_t prev = (j0 > 0 && j0 - 1 < n) ? kvar(j0 - 1) : 0xFFFFFFFFu;
        uint32_t cur = (j0 < n) ? kvar(j0) : 0xFFFFFFFEu;
#pragma unroll
        for (int k = 0; k < DE; ++k) {
            const int j = j0 + k;
            const uint32_t nxt = (j + 1 < n) ? kvar(j + 1) : 0xFFFFFFFDu;
            if (j < n) {
                if (cur != prev) headMask |= 1u << k;
                if (nxt != cur) lastMask |= 1u << k;
            }
            prev = cur;
            cur = nxt;
        }
    }
    uint8_t pm[DE], xm[DE];
    uint32_t acc = ID;
#pragma unroll
    for (int k = 0; k < DE; ++k) {
        const int j = j0 + k;
        pm[k] = xm[k] = (uint8_t)ID;
        if (j < n) {
            const uint32_t m = S.mel[kpos(j)];
            if (headMask & (1u << k)) {
                acc = m;
            } else {
                xm[k] = (uint8_t)acc;
                acc = S.comp[acc * MAX_ELEMS + m];
            }
            pm[k] = (uint8_t)acc;
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
                if (!f) v = S.comp[vu * MAX_ELEMS + v];
                f |= fu;
            }
        }
        uint32_t fe = __shfl_up_sync(0xffffffffu, f, 1);
        uint32_t ve = __shfl_up_sync(0xffffffffu, v, 1);
        if (lane == 0) { fe = 0; ve = ID; }
        if (lane == 31) { S.segF[warp] = (uint8_t)f; S.segV[warp] = (uint8_t)v; }
        __syncthreads();
        if (warp == 0) {
            uint32_t wf = lane < DNW ? S.segF[lane] : 0, wv = lane < DNW ? S.segV[lane] : ID;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t fu = __shfl_up_sync(0xffffffffu, wf, o);
                const uint32_t vu = __shfl_up_sync(0xffffffffu, wv, o);
                if (lane >= o) {
                    if (!wf) wv = S.comp[vu * MAX_ELEMS + wv];
                    wf |= fu;
                }
            }
            uint32_t xf = __shfl_up_sync(0xffffffffu, wf, 1);
            uint32_t xv = __shfl_up_sync(0xffffffffu, wv, 1);
            if (lane == 0) { xf = 0; xv = ID; }
            if (lane < DNW) { S.segF[lane] = (uint8_t)xf; S.segV[lane] = (uint8_t)xv; }
        }
        __syncthreads();
        carry = fe ? ve : S.comp[S.segV[warp] * MAX_ELEMS + ve];
    }
    // slots before the thread's first head continue a run from earlier threads
#pragma unroll
    for (int k = 0; k < DE; ++k) {
        if ((headMask & ((2u << k) - 1)) == 0) {
            pm[k] = S.comp[carry * MAX_ELEMS + pm[k]];
            xm[k] = S.comp[carry * MAX_ELEMS + xm[k]];
        }
    }

    if constexpr (!APPLY) {
        // fold each run (one per variable in the tile) into the chunk aggregate
#pragma unroll
        for (int k = 0; k < DE; ++k)
            if (lastMask & (1u << k)) {
                const uint32_t v = kvar(j0 + k);
                vec[v] = S.comp[vec[v] * MAX_ELEMS + pm[k]];
            }
        __syncthreads();
    } else {
    // ---- apply: statuses from the variable's status at tile entry ------------
    uint8_t post_last[DE];
#pragma unroll
    for (int k = 0; k < DE; ++k) {
        const int j = j0 + k;
        post_last[k] = 0;
        if (j < n) {
            const uint32_t v = kvar(j);
            const uint32_t e = vec[v];
            const uint32_t pre = S.app[xm[k] * 8 + e];
            const uint32_t post = S.app[pm[k] * 8 + e];
            const int pos = kpos(j);
            S.out[pos] = (uint8_t)(p.pre_mode ? pre : post);
            post_last[k] = (uint8_t)post;
            if (post == ST_F && pre != ST_F) {
                const uint32_t gi = (uint32_t)(base + pos);
                atomicMin(reinterpret_cast<uint32_t*>(p.vff) + v, gi);
                atomicMin(reinterpret_cast<unsigned long long*>(p.first_fault), (unsigned long long)gi);
            }
        }
    }
    __syncthreads();                         // every op has read its entry status
#pragma unroll
    for (int k = 0; k < DE; ++k)
        if (lastMask & (1u << k)) vec[kvar(j0 + k)] = post_last[k];
    if (vec16 && ((uintptr_t)(p.step + base) % 16 == 0)) {
        for (int i = tid; i < DT / 16; i += DNT)
            reinterpret_cast<uint4*>(p.step + base)[i] = reinterpret_cast<const uint4*>(S.out)[i];
    } else {
        for (int i = tid; i < n; i += DNT) p.step[base + i] = S.out[i];
    }
    __syncthreads();
    }
}

// GV: the per-variable vector is the chunk's own row of aggs (reduce) or entry
// (apply) in global memory, for variable counts beyond shared memory; the
// CTA's tiles run in order and only this CTA touches the row.
template <bool APPLY, bool GV>
__global__ void __launch_bounds__(DNT) dense_chunk_kernel(const DenseParams p)
{
    extern __shared__ __align__(16) uint8_t smem[];
    DenseSmem& S = *reinterpret_cast<DenseSmem*>(smem);
    const int tid = threadIdx.x;
    for (int i = tid; i < MAX_ELEMS * MAX_ELEMS; i += DNT) S.comp[i] = p.tab.comp[i];
    for (int i = tid; i < MAX_ELEMS * 8; i += DNT) S.app[i] = p.tab.app[i];
    for (int i = tid; i < 256; i += DNT) S.elem_of[i] = p.tab.elem_of[i];
    const int c = blockIdx.x;
    const size_t V = (size_t)p.n_vars;
    uint8_t* vec;
    if (GV) {
        vec = (APPLY ? p.entry : p.aggs) + (size_t)c * V;
        if (!APPLY) {
            const uint32_t id4 = p.tab.identity * 0x01010101u;
            const size_t n16 = (V % 16 == 0) ? V / 16 : 0;
            for (size_t i = tid; i < n16; i += DNT) reinterpret_cast<uint4*>(vec)[i] = make_uint4(id4, id4, id4, id4);
            for (size_t v = n16 * 16 + tid; v < V; v += DNT) vec[v] = p.tab.identity;
        }
    } else {
        vec = smem + sizeof(DenseSmem);
        for (int v = tid; v < p.n_vars; v += DNT) vec[v] = APPLY ? p.entry[(size_t)c * V + v] : p.tab.identity;
    }
    __syncthreads();
    const int t0 = c * p.tiles_per_chunk;
    const int t1 = min(t0 + p.tiles_per_chunk, p.n_tiles);
    for (int t = t0; t < t1; ++t) dense_tile<APPLY>(p, S, vec, t);
    if (!APPLY && !GV)
        for (int v = tid; v < p.n_vars; v += DNT) p.aggs[(size_t)c * V + v] = vec[v];
}

// Thread per four variables (one 32-bit word of every chunk row; rows are
// n_vars bytes long, a multiple of 4 here): status at every chunk entry, then
// the final status.
__global__ void dense_carry4_kernel(const DenseParams p)
{
    __shared__ uint8_t app[MAX_ELEMS * 8];
    for (int i = threadIdx.x; i < MAX_ELEMS * 8; i += blockDim.x) app[i] = p.tab.app[i];
    __syncthreads();
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;      // word: variables 4w .. 4w+3
    const size_t V = (size_t)p.n_vars;
    if (4 * w >= (int64_t)V) return;
    uint32_t e[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) e[b] = p.init ? p.init[4 * w + b] : (uint32_t)AMC_ST_VI;
    const size_t W = V / 4;
#pragma unroll 4
    for (int c = 0; c < p.n_chunks; ++c) {
        const uint32_t a = reinterpret_cast<const uint32_t*>(p.aggs)[(size_t)c * W + w];
        reinterpret_cast<uint32_t*>(p.entry)[(size_t)c * W + w] = e[0] | (e[1] << 8) | (e[2] << 16) | (e[3] << 24);
#pragma unroll
        for (int b = 0; b < 4; ++b) e[b] = app[((a >> (8 * b)) & 0xFFu) * 8 + e[b]];
    }
    if (p.final_status)
#pragma unroll
        for (int b = 0; b < 4; ++b) p.final_status[4 * w + b] = (uint8_t)e[b];
}

// Thread per variable (any row length).
__global__ void dense_carry_kernel(const DenseParams p)
{
    __shared__ uint8_t app[MAX_ELEMS * 8];
    for (int i = threadIdx.x; i < MAX_ELEMS * 8; i += blockDim.x) app[i] = p.tab.app[i];
    __syncthreads();
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= p.n_vars) return;
    uint32_t e = p.init ? p.init[v] : (uint32_t)AMC_ST_VI;
    const size_t V = (size_t)p.n_vars;
#pragma unroll 8
    for (int c = 0; c < p.n_chunks; ++c) {
        p.entry[(size_t)c * V + v] = (uint8_t)e;
        e = app[p.aggs[(size_t)c * V + v] * 8 + e];
    }
    if (p.final_status) p.final_status[v] = (uint8_t)e;
}

// ---------------------------------------------------------------------------
// Warp-sequential variant for at most 8,192 variables: every warp owns a
// contiguous sub-chunk (a multiple of 32 ops) and a dense per-variable vector
// in shared memory, and walks its sub-chunk in batches of 32 consecutive ops.
// The lanes of a batch that touch the same variable are grouped by match.any;
// a group's ops are composed in lane (= trace) order from a per-warp staging
// array, so no sort is needed.  The sub-chunks are the carry's chunks.
constexpr int WARP_MAX_VARS = 8192;
constexpr int WARP_CHUNKS_MAX = 8192;
constexpr int SEG = 64;                 // chunks per carry segment

template <bool APPLY>
__global__ void __launch_bounds__(256) warp_chunk_kernel(const DenseParams p, const int64_t cs)
{
    extern __shared__ __align__(16) uint8_t wsm[];
    uint8_t* comp = wsm;                                  // [32 * 32]
    uint8_t* app = comp + MAX_ELEMS * MAX_ELEMS;          // [32 * 8]
    uint8_t* elem_of = app + MAX_ELEMS * 8;               // [256]
    uint8_t* mbuf = elem_of + 256;                        // [8 warps][32]
    uint8_t* vecs = mbuf + 256;                           // [8 warps][n_vars]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < MAX_ELEMS * MAX_ELEMS; i += 256) comp[i] = p.tab.comp[i];
    for (int i = tid; i < MAX_ELEMS * 8; i += 256) app[i] = p.tab.app[i];
    for (int i = tid; i < 256; i += 256) elem_of[i] = p.tab.elem_of[i];
    __syncthreads();
    const int64_t g = (int64_t)blockIdx.x * 8 + warp;
    if (g >= p.n_chunks) return;                          // no block barrier below
    const size_t V = (size_t)p.n_vars;
    const uint32_t ID = p.tab.identity;
    const uint32_t lt = lanemask_lt();
    uint8_t* vec = vecs + (size_t)warp * V;
    uint8_t* mb = mbuf + warp * 32;
    for (size_t v = lane; v < V; v += 32) vec[v] = APPLY ? p.entry[(size_t)g * V + v] : (uint8_t)ID;
    __syncwarp();
    const int64_t lo = g * cs;
    const int64_t hi = min(lo + cs, p.n_ops);
    constexpr int UB = 8;                                 // batches whose loads are in flight together
    for (int64_t b0 = lo; b0 < hi; b0 += 32 * UB) {
    uint32_t ksb[UB];
    int32_t vb[UB];
#pragma unroll
    for (int u = 0; u < UB; ++u) {
        const int64_t i = b0 + 32 * u + lane;
        ksb[u] = i < hi ? (uint32_t)__ldcs(p.kind_side + i) : 0u;
        vb[u] = i < hi ? __ldcs(p.var + i) : 0;
    }
#pragma unroll
    for (int u = 0; u < UB; ++u) {
        const int64_t b = b0 + 32 * u;
        if (b >= hi) break;                               // warp-uniform
        const int64_t i = b + lane;
        const bool ok = i < hi;
        uint32_t ks = ksb[u];
        int32_t v = vb[u];
        if (ok) {
            if ((ks & 0xE0u) || (ks & 15u) > AMC_K_EN) raise_error(p.err, AMC_E_INVALID);
            if (v < 0 || v >= p.n_vars) {
                raise_error(p.err, AMC_E_RANGE);
                v = 0;
            }
        }
        const uint32_t nks_l = __shfl_down_sync(0xffffffffu, ks, 1);
        const int32_t nv_l = __shfl_down_sync(0xffffffffu, v, 1);
        uint32_t m = ok ? elem_of[ks] : ID;
        if (ok && m == ELEM_GT) {
            // GT must be followed by EN of the same side on another variable
            uint32_t nks = 0xFF;
            int32_t nv = v;
            if (i + 1 < p.n_ops_follow) {
                const bool in_batch = lane < 31 && i + 1 < hi;
                nks = in_batch ? nks_l : p.kind_side[i + 1];
                nv = in_batch ? nv_l : p.var[i + 1];
            }
            const bool gt_ok = (nks & 15) == AMC_K_EN && (nks >> 4) == (ks >> 4) && nv != v;
            if (!gt_ok) raise_error(p.err, AMC_E_INVALID);
            if (!gt_ok || p.pre_mode) {
                m = ID;
            } else if (!p.guard) {
                raise_error(p.err, AMC_E_INVALID);
                m = ID;
            } else {
                const uint32_t gs = p.guard[i + 1];
                const int side = ks >> 4;
                const bool valid = gs != ST_F && (gs & (side == 0 ? 1u : 2u));
                m = valid ? ID : p.tab.pull_of_side[side];
            }
        } else if (m == ELEM_BAD) {
            m = ID;
        }
        mb[lane] = (uint8_t)m;
        const uint32_t peers = __match_any_sync(0xffffffffu, ok ? (uint32_t)v : 0xFFFFFFFFu);
        __syncwarp();
        if constexpr (!APPLY) {
            if (ok && lane == __ffs(peers) - 1) {             // the group's first lane folds it in
                uint32_t acc = vec[v];
                for (uint32_t q = peers; q; q &= q - 1) acc = comp[acc * MAX_ELEMS + mb[__ffs(q) - 1]];
                vec[v] = (uint8_t)acc;
            }
        } else {
            const uint32_t e = ok ? vec[v] : 0u;                  // the variable's status before the batch
            __syncwarp();
            if (ok) {
                uint32_t acc = ID;
                for (uint32_t q = peers & lt; q; q &= q - 1) acc = comp[acc * MAX_ELEMS + mb[__ffs(q) - 1]];
                const uint32_t pre = app[acc * 8 + e];
                const uint32_t post = app[comp[acc * MAX_ELEMS + m] * 8 + e];
                p.step[i] = (uint8_t)(p.pre_mode ? pre : post);
                if (post == ST_F && pre != ST_F) {
                    atomicMin(reinterpret_cast<uint32_t*>(p.vff) + v, (uint32_t)i);
                    atomicMin(reinterpret_cast<unsigned long long*>(p.first_fault), (unsigned long long)i);
                }
                if (lane == 31 - __clz(peers)) vec[v] = (uint8_t)post;   // the group's last lane
            }
        }
        __syncwarp();
    }
    }
    if constexpr (!APPLY)
        for (size_t v = lane; v < V; v += 32) p.aggs[(size_t)g * V + v] = vec[v];
}

// Segmented carry over many chunks: (1) compose each segment's chunk
// aggregates, (2) carry the initial statuses over the segments, (3) expand
// every chunk's entry statuses inside its segment.  Thread per (segment,
// variable); composition is associative, so this equals the serial carry.
__global__ void seg_reduce_kernel(const DenseParams p, uint8_t* __restrict__ seg_agg, int n_segs)
{
    __shared__ uint8_t comp[MAX_ELEMS * MAX_ELEMS];
    for (int i = threadIdx.x; i < MAX_ELEMS * MAX_ELEMS; i += blockDim.x) comp[i] = p.tab.comp[i];
    __syncthreads();
    const size_t V = (size_t)p.n_vars;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_segs * (int64_t)V) return;
    const int s = (int)(t / (int64_t)V);
    const size_t v = (size_t)(t % (int64_t)V);
    uint32_t acc = p.tab.identity;
    const int c1 = min((s + 1) * SEG, p.n_chunks);
    for (int c = s * SEG; c < c1; ++c) acc = comp[acc * MAX_ELEMS + p.aggs[(size_t)c * V + v]];
    seg_agg[(size_t)s * V + v] = (uint8_t)acc;
}

__global__ void seg_carry_kernel(const DenseParams p, const uint8_t* __restrict__ seg_agg,
                                 uint8_t* __restrict__ seg_entry, int n_segs)
{
    __shared__ uint8_t app[MAX_ELEMS * 8];
    for (int i = threadIdx.x; i < MAX_ELEMS * 8; i += blockDim.x) app[i] = p.tab.app[i];
    __syncthreads();
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= p.n_vars) return;
    const size_t V = (size_t)p.n_vars;
    uint32_t e = p.init ? p.init[v] : (uint32_t)AMC_ST_VI;
    for (int s = 0; s < n_segs; ++s) {
        seg_entry[(size_t)s * V + v] = (uint8_t)e;
        e = app[seg_agg[(size_t)s * V + v] * 8 + e];
    }
    if (p.final_status) p.final_status[v] = (uint8_t)e;
}

__global__ void seg_expand_kernel(const DenseParams p, const uint8_t* __restrict__ seg_entry, int n_segs)
{
    __shared__ uint8_t app[MAX_ELEMS * 8];
    for (int i = threadIdx.x; i < MAX_ELEMS * 8; i += blockDim.x) app[i] = p.tab.app[i];
    __syncthreads();
    const size_t V = (size_t)p.n_vars;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_segs * (int64_t)V) return;
    const int s = (int)(t / (int64_t)V);
    const size_t v = (size_t)(t % (int64_t)V);
    uint32_t e = seg_entry[(size_t)s * V + v];
    const int c1 = min((s + 1) * SEG, p.n_chunks);
    for (int c = s * SEG; c < c1; ++c) {
        p.entry[(size_t)c * V + v] = (uint8_t)e;
        e = app[p.aggs[(size_t)c * V + v] * 8 + e];
    }
}

// Warp sub-chunks of a trace: chunk length (a multiple of 32) and count.
void warp_shape(int64_t n_ops, int64_t& cs, int& n_chunks)
{
    int64_t want = (n_ops + 4095) / 4096;                 // at least a tile's worth per warp
    if (want > WARP_CHUNKS_MAX) want = WARP_CHUNKS_MAX;
    if (want < 1) want = 1;
    cs = ((n_ops + want - 1) / want + 31) / 32 * 32;
    if (cs < 32) cs = 32;
    n_chunks = (int)((n_ops + cs - 1) / cs);
}

size_t warp_workspace_bytes(int64_t n_ops, int32_t n_vars)
{
    int64_t cs;
    int n_chunks;
    warp_shape(n_ops, cs, n_chunks);
    const int n_segs = (n_chunks + SEG - 1) / SEG;
    return 2 * align_up((size_t)n_chunks * (size_t)n_vars, 256) + 2 * align_up((size_t)n_segs * (size_t)n_vars, 256);
}

int launch_warp_dense(const ScanLaunch& L, uint8_t* ws, cudaStream_t s)
{
    DenseParams p{};
    p.kind_side = L.kind_side;
    p.var = L.var;
    p.n_ops = L.n_ops;
    p.n_ops_follow = L.n_ops;
    p.n_vars = L.n_vars;
    p.init = L.init;
    p.step = L.step;
    p.vff = L.vff;
    p.first_fault = L.first_fault;
    p.final_status = L.final_status;
    p.guard = L.guard;
    p.pre_mode = L.pre_mode;
    p.err = L.err;
    p.tab = host_tables();
    int64_t cs;
    warp_shape(L.n_ops, cs, p.n_chunks);
    const int n_segs = (p.n_chunks + SEG - 1) / SEG;
    const size_t V = (size_t)L.n_vars;
    p.aggs = ws;
    p.entry = ws + align_up((size_t)p.n_chunks * V, 256);
    uint8_t* seg_agg = p.entry + align_up((size_t)p.n_chunks * V, 256);
    uint8_t* seg_entry = seg_agg + align_up((size_t)n_segs * V, 256);
    if (cudaMemsetAsync(L.vff, 0xFF, 4 * V, s) != cudaSuccess) return AMC_E_CUDA;
    if (cudaMemsetAsync(L.first_fault, 0xFF, 8, s) != cudaSuccess) return AMC_E_CUDA;
    const size_t smem = MAX_ELEMS * MAX_ELEMS + MAX_ELEMS * 8 + 256 + 256 + 8 * V;
    if (cudaFuncSetAttribute(warp_chunk_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaFuncSetAttribute(warp_chunk_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return AMC_E_CUDA;
    const unsigned grid = (unsigned)((p.n_chunks + 7) / 8);
    const unsigned segv = (unsigned)(((int64_t)n_segs * (int64_t)V + 255) / 256);
    if (L.profile & 1) profile_begin(s);
    warp_chunk_kernel<false><<<grid, 256, smem, s>>>(p, cs);
    if (cudaGetLastError() != cudaSuccess) return AMC_E_CUDA;
    seg_reduce_kernel<<<segv, 256, 0, s>>>(p, seg_agg, n_segs);
    seg_carry_kernel<<<(unsigned)((V + 255) / 256), 256, 0, s>>>(p, seg_agg, seg_entry, n_segs);
    seg_expand_kernel<<<segv, 256, 0, s>>>(p, seg_entry, n_segs);
    if (cudaGetLastError() != cudaSuccess) return AMC_E_CUDA;
    warp_chunk_kernel<true><<<grid, 256, smem, s>>>(p, cs);
    if (cudaGetLastError() != cudaSuccess) return AMC_E_CUDA;
    if (L.profile & 2) profile_end(s);
    return AMC_OK;
}

void dense_shape(int64_t n_ops, int max_chunks, int& n_tiles, int& n_chunks, int& tpc)
{
    n_tiles = (int)((n_ops + DT - 1) / DT);
    const int want = n_tiles < max_chunks ? n_tiles : max_chunks;
    tpc = want > 0 ? (n_tiles + want - 1) / want : 1;
    n_chunks = tpc > 0 ? (n_tiles + tpc - 1) / tpc : 0;
}

// Large traces over many variables (more than 16,384, at most 2^20): the first
// PREFIX_OPS ops -- where nearly every op is live and the single-pass kernel's
// lists are most contended -- take this path with global per-chunk rows; the
// rest continues in the single-pass kernel from the prefix's final statuses.
constexpr int PREFIX_LOG2 = 22;
constexpr int PREFIX_CHUNKS = 256;
constexpr int64_t PREFIX_MIN_OPS = (int64_t)1 << 24;

// has_init: a caller's initial statuses may already make most variables
// stuck (a trace continued from an earlier one), so the start is not dense:
// the prefix is then taken only when forced.
int64_t prefix_ops(int64_t n_ops, int32_t n_vars, bool has_init)
{
    if (n_vars <= DENSE_MAX_VARS || n_vars > (1 << 20)) return 0;
    int lg = PREFIX_LOG2;
    int64_t min_ops = PREFIX_MIN_OPS;
    if (const char* e = getenv("AMC_SCAN_DENSE"))
        if (e[0] == '0') return 0;
    if (const char* e = getenv("AMC_SCAN_PREFIX")) {   // test override: prefix of 2^k ops at any size
        lg = atoi(e);
        min_ops = 0;
        if (lg < 12 || lg > 30) return 0;
    }
    if (has_init && min_ops > 0) return 0;
    const int64_t P = (int64_t)1 << lg;
    return (n_ops >= min_ops && n_ops > P) ? P : 0;
}

int launch_dense_range(const ScanLaunch& L, int max_chunks, int64_t n_follow, uint8_t* ws, cudaStream_t s)
{
    DenseParams p{};
    p.kind_side = L.kind_side;
    p.var = L.var;
    p.n_ops = L.n_ops;
    p.n_ops_follow = n_follow;
    p.n_vars = L.n_vars;
    p.init = L.init;
    p.step = L.step;
    p.vff = L.vff;
    p.first_fault = L.first_fault;
    p.final_status = L.final_status;
    p.guard = L.guard;
    p.pre_mode = L.pre_mode;
    p.err = L.err;
    p.tab = host_tables();
    dense_shape(L.n_ops, max_chunks, p.n_tiles, p.n_chunks, p.tiles_per_chunk);
    const size_t vb = align_up((size_t)p.n_chunks * (size_t)L.n_vars, 256);
    p.aggs = ws;
    p.entry = ws + vb;
    int kb = 1;
    while (kb < 31 && ((int64_t)1 << kb) < (int64_t)L.n_vars) ++kb;
    p.passes = (kb + DDIG - 1) / DDIG;
    p.digit_bits = (kb + p.passes - 1) / p.passes;
    const bool gv = L.n_vars > DENSE_MAX_VARS;

    if (cudaMemsetAsync(L.vff, 0xFF, 4 * (size_t)L.n_vars, s) != cudaSuccess) return AMC_E_CUDA;
    if (cudaMemsetAsync(L.first_fault, 0xFF, 8, s) != cudaSuccess) return AMC_E_CUDA;
    const size_t smem = sizeof(DenseSmem) + (gv ? 0 : (size_t)L.n_vars);
    auto kr = gv ? dense_chunk_kernel<false, true> : dense_chunk_kernel<false, false>;
    auto ka = gv ? dense_chunk_kernel<true, true> : dense_chunk_kernel<true, false>;
    if (cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(ka, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return AMC_E_CUDA;
    if (L.profile & 1) profile_begin(s);
    kr<<<p.n_chunks, DNT, smem, s>>>(p);
    if (cudaGetLastError() != cudaSuccess) return AMC_E_CUDA;
    if (L.n_vars % 4 == 0)       // rows start 256-byte aligned; 4-byte words when n_vars is a multiple of 4
        dense_carry4_kernel<<<(unsigned)((L.n_vars / 4 + 255) / 256), 256, 0, s>>>(p);
    else
        dense_carry_kernel<<<(unsigned)((L.n_vars + 255) / 256), 256, 0, s>>>(p);
    if (cudaGetLastError() != cudaSuccess) return AMC_E_CUDA;
    ka<<<p.n_chunks, DNT, smem, s>>>(p);
    if (cudaGetLastError() != cudaSuccess) return AMC_E_CUDA;
    if (L.profile & 2) profile_end(s);
    return AMC_OK;
}

// First faults of a prefix and the suffix after it: the prefix's where it has
// one, else the suffix's moved by the prefix length.
__global__ void merge_faults_kernel(int32_t* __restrict__ vff, const int32_t* __restrict__ vff_suffix, int32_t n_vars,
                                    int64_t* __restrict__ ff, const int64_t* __restrict__ ff_suffix, int64_t P,
                                    const int* only_if)
{
    if (only_if && *only_if == 0) return;
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n_vars && vff[v] == -1 && vff_suffix[v] != -1) vff[v] = (int32_t)(vff_suffix[v] + P);
    if (v == 0 && *ff == -1 && *ff_suffix != -1) *ff = *ff_suffix + P;
}

}  // namespace

bool scan_dense_eligible(int64_t n_ops, int32_t n_vars)
{
    if (n_vars < 1 || n_vars > DENSE_MAX_VARS || n_ops < 1) return false;
    if (const char* e = getenv("AMC_SCAN_DENSE")) return e[0] == '1';   // tuning and test override
    int lv = 0, ln = 0;
    while (lv < 31 && ((int64_t)1 << lv) < (int64_t)n_vars) ++lv;
    while (ln < 62 && ((int64_t)1 << ln) < n_ops) ++ln;
    return ln >= 15 + 2 * (12 - lv) && n_ops >= DENSE_MIN_OPS;
}

// The whole trace over more than 16,384 (at most 2^20) variables with global
// per-chunk rows: where nothing gets stuck (a well-declared program's guarded
// trace) every op stays live and the single-pass kernel's lists are long and
// contended.  Taken when the launch forces it (the tuner times it) on traces
// of at least GV_MIN_OPS ops; chunk count from the row budget (about 2^28
// row bytes, 256 .. 1,024 chunks).
constexpr int64_t GV_MIN_OPS = (int64_t)1 << 20;
constexpr int32_t GV_MAX_VARS = 1 << 20;

int gv_chunks(int32_t n_vars)
{
    int64_t c = ((int64_t)1 << 28) / (n_vars > 0 ? n_vars : 1);
    return (int)(c < 256 ? 256 : (c > 1024 ? 1024 : c));
}

bool dense_forced_ok(int64_t n_ops, int32_t n_vars)
{
    if (n_vars < 1 || n_ops < 1) return false;
    return n_vars <= DENSE_MAX_VARS || (n_vars <= GV_MAX_VARS && n_ops >= GV_MIN_OPS);
}

size_t scan_dense_workspace_bytes(int64_t n_ops, int32_t n_vars)
{
    int n_tiles, n_chunks, tpc;
    if (n_vars > DENSE_MAX_VARS && n_vars <= GV_MAX_VARS && n_ops >= GV_MIN_OPS) {
        dense_shape(n_ops, gv_chunks(n_vars), n_tiles, n_chunks, tpc);
        size_t b = 2 * align_up((size_t)n_chunks * (size_t)n_vars, 256);
        if (const int64_t P = prefix_ops(n_ops, n_vars, false)) {
            dense_shape(P, PREFIX_CHUNKS, n_tiles, n_chunks, tpc);
            const size_t pb = 2 * align_up((size_t)n_chunks * (size_t)n_vars, 256) + align_up(4 * (size_t)n_vars, 256) +
                              256 + align_up((size_t)n_vars, 256) + 256;
            if (pb > b) b = pb;
        }
        return b;
    }
    if (const int64_t P = prefix_ops(n_ops, n_vars, false)) {   // the larger workspace
        // prefix rows, then the suffix's first faults and the prefix's final statuses
        dense_shape(P, PREFIX_CHUNKS, n_tiles, n_chunks, tpc);
        return 2 * align_up((size_t)n_chunks * (size_t)n_vars, 256) + align_up(4 * (size_t)n_vars, 256) + 256 +
               align_up((size_t)n_vars, 256) + 256;
    }
    if (n_vars < 1 || n_vars > DENSE_MAX_VARS || n_ops < 1) return 0;
    dense_shape(n_ops, DENSE_MAX_CHUNKS, n_tiles, n_chunks, tpc);
    const size_t sorted = 2 * align_up((size_t)n_chunks * (size_t)n_vars, 256);
    const size_t warped = n_vars <= WARP_MAX_VARS ? warp_workspace_bytes(n_ops, n_vars) : 0;
    return sorted > warped ? sorted : warped;
}

bool scan_prefix_eligible(int64_t n_ops, int32_t n_vars, bool has_init)
{
    return prefix_ops(n_ops, n_vars, has_init) > 0;
}

namespace {

// the prefix a launch takes: forced (prefix_log2) or by size
int64_t launch_prefix_ops(const ScanLaunch& L)
{
    if (L.prefix_log2 > 0) {
        if (L.n_vars <= DENSE_MAX_VARS || L.n_vars > (1 << 20) || L.prefix_log2 < 12 || L.prefix_log2 > 30) return 0;
        const int64_t P = (int64_t)1 << L.prefix_log2;
        return L.n_ops > P ? P : 0;
    }
    return prefix_ops(L.n_ops, L.n_vars, L.init != nullptr);
}

// *out = max(0, *n - P): the suffix's op count when the trace's count is on the device
__global__ void suffix_count_kernel(const int64_t* n, int64_t P, int64_t* out)
{
    const int64_t r = *n - P;
    *out = r > 0 ? r : 0;
}

}  // namespace

size_t scan_prefix_workspace_bytes(int64_t P, int32_t n_vars)
{
    int n_tiles, n_chunks, tpc;
    dense_shape(P, PREFIX_CHUNKS, n_tiles, n_chunks, tpc);
    return 2 * align_up((size_t)n_chunks * (size_t)n_vars, 256) + align_up(4 * (size_t)n_vars, 256) + 256 +
           align_up((size_t)n_vars, 256) + 256;
}

bool scan_forced_prefix(const ScanLaunch& L) { return launch_prefix_ops(L) > 0 && L.prefix_log2 > 0; }

int launch_scan_prefix(const ScanLaunch& L, uint8_t* ws, cudaStream_t s)
{
    const int64_t P = launch_prefix_ops(L);
    int n_tiles, n_chunks, tpc;
    dense_shape(P, PREFIX_CHUNKS, n_tiles, n_chunks, tpc);
    uint8_t* w = ws + 2 * align_up((size_t)n_chunks * (size_t)L.n_vars, 256);
    int32_t* vff_suffix = reinterpret_cast<int32_t*>(w);
    w += align_up(4 * (size_t)L.n_vars, 256);
    int64_t* ff_suffix = reinterpret_cast<int64_t*>(w);
    w += 256;
    uint8_t* pfinal = w;
    w += align_up((size_t)L.n_vars, 256);
    int64_t* n_suffix = reinterpret_cast<int64_t*>(w);      // with a device count: the suffix's

    ScanLaunch A = L;                       // the prefix: faults straight into the outputs
    A.n_ops = P;
    A.n_dev = nullptr;                      // the first P ops are always there (padded by the caller)
    A.gate = nullptr;
    A.final_status = pfinal;
    A.profile = L.profile & 1;
    int rc = launch_dense_range(A, PREFIX_CHUNKS, L.n_ops, ws, s);
    if (rc) return rc;
    ScanLaunch B = L;                       // the rest, from the prefix's final statuses
    B.kind_side = L.kind_side + P;
    B.var = L.var + P;
    B.n_ops = L.n_ops - P;
    B.step = L.step + P;
    B.guard = L.guard ? L.guard + P : nullptr;
    B.init = pfinal;
    B.vff = vff_suffix;
    B.first_fault = ff_suffix;
    B.dense = 0;
    B.prefix_log2 = 0;
    B.profile = 0;
    if (L.n_dev) {
        suffix_count_kernel<<<1, 1, 0, s>>>(L.n_dev, P, n_suffix);
        if (cudaGetLastError() != cudaSuccess) return AMC_E_CUDA;
        B.n_dev = n_suffix;
    }
    rc = launch_scan_trace(B, s);
    if (rc) return rc;
    merge_faults_kernel<<<(unsigned)((L.n_vars + 255) / 256), 256, 0, s>>>(L.vff, vff_suffix, L.n_vars,
                                                                           L.first_fault, ff_suffix, P, nullptr);
    if (cudaGetLastError() != cudaSuccess) return AMC_E_CUDA;
    if (L.profile & 2) profile_end(s);
    return AMC_OK;
}

int launch_scan_dense(const ScanLaunch& L, uint8_t* ws, cudaStream_t s)
{
    // up to 8,192 variables: warp-sequential batches; else tile sorts (rows
    // in shared memory up to 16,384 variables, in global memory above)
    const char* e = getenv("AMC_SCAN_DENSE_SORT");                // test override: the sorted variant
    if (L.n_vars <= WARP_MAX_VARS && !(e && e[0] == '1')) return launch_warp_dense(L, ws, s);
    if (L.n_vars > DENSE_MAX_VARS) return launch_dense_range(L, gv_chunks(L.n_vars), L.n_ops, ws, s);
    return launch_dense_range(L, DENSE_MAX_CHUNKS, L.n_ops, ws, s);
}

int launch_merge_faults(int32_t* vff, const int32_t* vff_part, int32_t n_vars, int64_t* ff,
                        const int64_t* ff_part, int64_t offset, cudaStream_t s, const int* only_if)
{
    merge_faults_kernel<<<(unsigned)((n_vars + 255) / 256 > 0 ? (n_vars + 255) / 256 : 1), 256, 0, s>>>(
        vff, vff_part, n_vars, ff, ff_part, offset, only_if);
    return cudaGetLastError() == cudaSuccess ? AMC_OK : AMC_E_CUDA;
}

}  // namespace amc
