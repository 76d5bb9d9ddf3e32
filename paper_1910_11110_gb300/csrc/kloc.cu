// kloc.cu -- traces over k memory locations (k = 1..7): the Section 3.1
// effects on a vector of k validity flags.  Section 3 states that the
// two-location results extend to many locations; an op runs at one location:
// r at a needs flag a valid; w at a makes a the only valid flag; copy a -> b
// (Push at a towards b, Pull at b from a) needs flag a valid and makes b
// valid; Noop.  A failed need is the stuck status F (Property Progress).
//
// Every composition of these functions has the form
//     f(s) = F                     if s = F, or f is constant F, or G is not inside s
//     f(s) = (s AND K) OR S        otherwise
// for flag sets G (needed), K (kept) and S (set): r at a = (G {a}, K all,
// S {}), w at a = ({}, {}, {a}), copy a -> b = ({a}, all, {b}), Noop = ({},
// all, {}).  For f then g: a flag g needs is either set by f, or kept by f
// and then needed from s, or neither -- then the composition is constant F;
// so G = Gf | (Gg & ~Sf), K = Kf & Kg, S = (Sf & Kg) | Sg.  These 22-bit
// elements compose with a few bit operations, so the check groups the ops by
// variable (stable radix sort of (variable, index) pairs, scan_sorted.cu) and
// runs one segmented scan of the elements over the sorted pairs (decoupled
// look-back over tiles claimed in order), applying each prefix to its
// variable's initial status.  The pairs' keys carry the op byte above the
// variable id's bits (up to 2^21 variables), so the scan reads its ops in
// sorted order instead of gathering them; F is written at every position
// first (F is absorbing: on a long trace nearly every op sees it), and the
// scan writes only the statuses that are not F.
#include "amc_internal.cuh"
#include "kloc.cuh"
#include "scan_trace.cuh"

namespace amc {

namespace {

constexpr int KT = 2048;                 // pairs per tile
constexpr int KNT = 256;
constexpr int KE = KT / KNT;
constexpr uint32_t KL_F = 0x80u;
constexpr uint32_t KCF = 1u << 21;       // constant F
constexpr uint32_t KRUN = 1u << 22;      // segmented-scan value: a variable's run starts inside
constexpr uint32_t KVAL = (1u << 23) - 1u;
constexpr uint32_t KIDENT = 0x7Fu << 7;  // G {}, K all, S {}
constexpr uint32_t KNOKEY = 0xFFFFFFFFu;
constexpr uint32_t TS_AGG = 1u << 30, TS_INCL = 2u << 30, TS_FLAGS = 3u << 30;
constexpr int KOP_SHIFT = 21;            // op byte in key bits 21-28 when n_vars <= 2^21

__device__ __forceinline__ uint32_t kcomp(uint32_t f, uint32_t g)
{
    if ((f | g) & KCF) return KCF;
    const uint32_t fG = f & 0x7Fu, fK = (f >> 7) & 0x7Fu, fS = (f >> 14) & 0x7Fu;
    const uint32_t gG = g & 0x7Fu, gK = (g >> 7) & 0x7Fu, gS = (g >> 14) & 0x7Fu;
    const uint32_t need = gG & ~fS;
    if (need & ~fK) return KCF;
    return (fG | need) | (fK & gK) << 7 | ((fS & gK) | gS) << 14;
}

__device__ __forceinline__ uint32_t kapply(uint32_t f, uint32_t s)
{
    if ((s & KL_F) || (f & KCF)) return KL_F;
    const uint32_t G = f & 0x7Fu;
    if ((s & G) != G) return KL_F;
    return (s & ((f >> 7) & 0x7Fu)) | ((f >> 14) & 0x7Fu);
}

__device__ __forceinline__ bool kvalid(uint32_t op, int k)
{
    const uint32_t kind = op & 3u, a = (op >> 2) & 7u, b = (op >> 5) & 7u;
    if (kind == 3u) return a == 0 && b == 0;
    if (a >= (uint32_t)k) return false;
    if (kind == 2u) return b < (uint32_t)k && b != a;
    return b == 0;
}

__device__ __forceinline__ uint32_t kelem(uint32_t op)
{
    const uint32_t kind = op & 3u, a = (op >> 2) & 7u, b = (op >> 5) & 7u;
    if (kind == 0u) return (1u << a) | KIDENT;                  // r
    if (kind == 1u) return (1u << a) << 14;                     // w
    if (kind == 2u) return (1u << a) | KIDENT | (1u << b) << 14;   // copy
    return KIDENT;                                              // Noop
}

// segmented combine of (value, run-start) words: y alone when a run starts in y
__device__ __forceinline__ uint32_t kseg(uint32_t x, uint32_t y)
{
    if (y & KRUN) return y;
    return (x & KRUN) | kcomp(x & (KRUN - 1u), y & (KRUN - 1u));
}

// pairs (var | op << KOP_SHIFT when packed, index); every op byte and id
// checked; F written at every position; initial statuses checked; final
// statuses and first faults initialised
__global__ void kl_keys_kernel(const uint8_t* __restrict__ op, const int32_t* __restrict__ var, int64_t n,
                               int32_t n_vars, int k, int pack, uint32_t* __restrict__ key, uint32_t* __restrict__ val,
                               uint8_t* __restrict__ step, const uint8_t* __restrict__ init, uint8_t* __restrict__ fin,
                               int32_t* __restrict__ vff, int64_t* ff, int* err)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = g; i < n; i += stride) {
        const uint32_t o = op[i];
        const int32_t v = var[i];
        if (!kvalid(o, k)) raise_error(err, AMC_E_INVALID);
        uint32_t uv = (uint32_t)v;
        if (v < 0 || v >= n_vars) {
            raise_error(err, AMC_E_RANGE);
            uv = 0;
        }
        key[i] = pack ? (uv | o << KOP_SHIFT) : uv;
        val[i] = (uint32_t)i;
        step[i] = (uint8_t)KL_F;
    }
    for (int64_t v = g; v < n_vars; v += stride) {
        uint8_t s = 1;                                          // valid in location 0 only
        if (init) {
            s = init[v];
            if (s != KL_F && (s >> k)) raise_error(err, AMC_E_INVALID);
        }
        fin[v] = s;
        vff[v] = -1;
    }
    if (g == 0) *ff = -1;
}

struct KSegParams {
    uint32_t vmask;         // variable bits of a key
    int pack;               // keys carry the op byte
    const uint32_t* key;
    const uint32_t* val;
    int64_t n;
    const uint8_t* op;
    const uint8_t* init;
    uint8_t* step;
    uint8_t* fin;
    int32_t* vff;
    int64_t* ff;
    uint32_t* tstat;        // per tile, zeroed before the launch
    uint32_t* tile_counter; // zeroed before the launch
    int* err;
};

__global__ void __launch_bounds__(KNT) kl_seg_kernel(const KSegParams p)
{
    __shared__ uint32_t wtot[KNT / 32];
    __shared__ uint32_t s_tile, s_carry;
    const int64_t nt = (p.n + KT - 1) / KT;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(p.tile_counter, 1u);
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= nt) break;
        const int64_t b = tile * KT;
        const int m = (int)(p.n - b < KT ? p.n - b : KT);
        const int i0 = threadIdx.x * KE;
        uint32_t kk[KE], vv[KE], el[KE];
#pragma unroll
        for (int u = 0; u < KE; ++u) {
            const bool in = i0 + u < m;
            kk[u] = in ? p.key[b + i0 + u] : KNOKEY;
            vv[u] = in ? p.val[b + i0 + u] : 0u;
        }
#pragma unroll
        for (int u = 0; u < KE; ++u) {
            if (kk[u] == KNOKEY) {
                el[u] = KIDENT;
                continue;
            }
            el[u] = kelem(p.pack ? (kk[u] >> KOP_SHIFT) & 0xFFu : p.op[vv[u]]);
            kk[u] &= p.vmask;                                   // the variable alone from here on
        }
        uint32_t prev = (b + i0 > 0 && b + i0 - 1 < p.n) ? (p.key[b + i0 - 1] & p.vmask) : KNOKEY;
        uint32_t heads = 0, agg = KIDENT;
#pragma unroll
        for (int u = 0; u < KE; ++u) {
            if (kk[u] == KNOKEY) break;
            if (kk[u] != prev) {
                heads |= 1u << u;
                agg = KRUN | el[u];
            } else {
                agg = (agg & KRUN) | kcomp(agg & (KRUN - 1u), el[u]);
            }
            prev = kk[u];
        }
        // exclusive segmented scan of the threads' folds
        uint32_t incl = agg;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl = kseg(y, incl);
        }
        uint32_t ex = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane == 0) ex = KIDENT;
        if (lane == 31) wtot[warp] = incl;
        __syncthreads();
        uint32_t pre = KIDENT;
        for (int w = 0; w < warp; ++w) pre = kseg(pre, wtot[w]);
        uint32_t all = KIDENT;
        for (int w = 0; w < KNT / 32; ++w) all = kseg(all, wtot[w]);
        ex = kseg(pre, ex);
        if (threadIdx.x == 0) {
            uint32_t carry = KIDENT;
            if (tile == 0) {
                st_release(p.tstat, TS_INCL | (all & KVAL));
            } else {
                st_release(p.tstat + tile, TS_AGG | (all & KVAL));
                uint32_t prefix = KIDENT;                  // over tiles [t2, tile)
                for (int64_t t2 = tile - 1; t2 >= 0; --t2) {
                    uint32_t v = 0;
                    for (uint32_t it = 0; it < (1u << 24); ++it) {
                        v = ld_acquire(p.tstat + t2);
                        if (v & TS_FLAGS) break;
                    }
                    if (!(v & TS_FLAGS)) {
                        raise_error(p.err, AMC_E_TIMEOUT);
                        break;
                    }
                    prefix = kseg(v & KVAL, prefix);
                    if ((v & TS_INCL) || (v & KRUN)) break;
                }
                st_release(p.tstat + tile, TS_INCL | (kseg(prefix, all) & KVAL));
                if (((p.key[b - 1] ^ p.key[b]) & p.vmask) == 0) carry = prefix & (KRUN - 1u);
            }
            s_carry = carry;
        }
        __syncthreads();
        // the carry reaches this thread's first run only if no run starts
        // before it in the tile
        uint32_t run = (ex & KRUN) ? (ex & (KRUN - 1u)) : kcomp(s_carry, ex & (KRUN - 1u));
        const uint32_t after = (b + i0 + KE < p.n) ? (p.key[b + i0 + KE] & p.vmask) : KNOKEY;
        unsigned long long gmin = ~0ull;
#pragma unroll
        for (int u = 0; u < KE; ++u) {
            const uint32_t kv = kk[u];
            if (kv == KNOKEY) break;
            const bool head = (heads >> u) & 1u;
            const uint32_t before = head ? KIDENT : run;
            run = head ? el[u] : kcomp(run, el[u]);
            const uint32_t s0 = p.init ? p.init[kv] : 1u;
            const uint32_t pre_s = kapply(before, s0);
            const uint32_t post = kapply(run, s0);
            if (post != KL_F) p.step[vv[u]] = (uint8_t)post;    // F is there already
            if (post == KL_F && pre_s != KL_F) {
                p.vff[kv] = (int32_t)vv[u];
                if ((unsigned long long)vv[u] < gmin) gmin = vv[u];
            }
            const uint32_t next = u + 1 < KE ? kk[u + 1] : after;
            if (next != kv) p.fin[kv] = (uint8_t)post;
        }
        // the warp's smallest first fault, one atomic per warp
#pragma unroll
        for (int d = 16; d; d >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, gmin, d);
            if (o < gmin) gmin = o;
        }
        if (lane == 0 && gmin != ~0ull) atomicMin(reinterpret_cast<unsigned long long*>(p.ff), gmin);
        __syncthreads();
    }
}

struct KLayout {
    size_t key0, val0, key1, val1, scratch, tstat, ctr, total;
};

KLayout klayout(int64_t n)
{
    KLayout L;
    size_t o = 0;
    auto take = [&](size_t b) { const size_t at = o; o += align_up(b, 256); return at; };
    L.key0 = take(4 * (size_t)n);
    L.val0 = take(4 * (size_t)n);
    L.key1 = take(4 * (size_t)n);
    L.val1 = take(4 * (size_t)n);
    L.scratch = take(sorted_check_scratch_bytes(n));
    L.tstat = take(4 * (size_t)((n + KT - 1) / KT + 1));
    L.ctr = take(4);
    L.total = o;
    return L;
}

}  // namespace

size_t kloc_workspace_bytes(int64_t n_ops) { return klayout(n_ops).total; }

int launch_kloc(const KlocLaunch& L, cudaStream_t s)
{
    const KLayout lay = klayout(L.n_ops);
    uint8_t* w = static_cast<uint8_t*>(L.workspace);
    uint32_t* key[2] = {reinterpret_cast<uint32_t*>(w + lay.key0), reinterpret_cast<uint32_t*>(w + lay.key1)};
    uint32_t* val[2] = {reinterpret_cast<uint32_t*>(w + lay.val0), reinterpret_cast<uint32_t*>(w + lay.val1)};
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (L.profile & 1) profile_begin(s);
    const int64_t work = L.n_ops > L.n_vars ? L.n_ops : L.n_vars;
    const int64_t blocks = (work + 255) / 256;
    const int kgrid = (int)(blocks < (int64_t)n_sm * 8 ? (blocks > 0 ? blocks : 1) : (int64_t)n_sm * 8);
    const int pack = L.n_vars <= (1 << KOP_SHIFT) ? 1 : 0;
    kl_keys_kernel<<<kgrid, 256, 0, s>>>(L.op, L.var, L.n_ops, L.n_vars, L.k, pack, key[0], val[0], L.step, L.init,
                                         L.final_status, L.vff, L.first_fault, L.err);
    if (cudaGetLastError() != cudaSuccess) return AMC_E_CUDA;
    if (L.n_ops > 0) {
        int passes = 0;
        const int rc = launch_ss_radix(key, val, nullptr, L.n_ops, L.n_vars, w + lay.scratch, nullptr, s, &passes);
        if (rc) return rc;
        const int64_t tiles = (L.n_ops + KT - 1) / KT;
        if (cudaMemsetAsync(w + lay.tstat, 0, lay.total - lay.tstat, s) != cudaSuccess) return AMC_E_CUDA;
        KSegParams p;
        p.vmask = pack ? (1u << KOP_SHIFT) - 1u : 0xFFFFFFFFu;
        p.pack = pack;
        p.key = key[passes & 1];
        p.val = val[passes & 1];
        p.n = L.n_ops;
        p.op = L.op;
        p.init = L.init;
        p.step = L.step;
        p.fin = L.final_status;
        p.vff = L.vff;
        p.ff = L.first_fault;
        p.tstat = reinterpret_cast<uint32_t*>(w + lay.tstat);
        p.tile_counter = reinterpret_cast<uint32_t*>(w + lay.ctr);
        p.err = L.err;
        const int sgrid = (int)(tiles < (int64_t)n_sm * 8 ? tiles : (int64_t)n_sm * 8);
        kl_seg_kernel<<<sgrid, KNT, 0, s>>>(p);
        if (cudaGetLastError() != cudaSuccess) return AMC_E_CUDA;
    }
    if (L.profile & 2) profile_end(s);
    return AMC_OK;
}

}  // namespace amc
