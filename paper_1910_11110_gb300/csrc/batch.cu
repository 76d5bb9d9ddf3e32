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
// Work is split by op count.  A program longer than the split length (with at
// most SPLIT_VARS variables) is cut into segments of about that length at
// top-level boundaries (never inside an If or While); every other program is
// one segment.  Per variable, a segment maps the set its variable enters with
// to the set it leaves with through a relation over the five statuses (a 5x5
// boolean matrix, 25 bits: row i = the set reached from {i}; If is the union
// of the branches' relations, While the closure of its body's, both exactly
// what the set semantics computes from a singleton entry set).  So:
//   reduce  every segment but the last of a split program is run five times,
//           from {i} for every variable (i = 0..4): the five exit sets are the
//           rows of each variable's relation;
//   carry   per split program and variable, the entry set of segment s + 1 is
//           the image of segment s's entry set through its relation;
//   apply   every segment runs from its entry sets, writing the step sets, the
//           program's first fault (the minimum over its segments) and, for the
//           last segment, the final sets.
// A segment runs on one warp: consecutive op tokens 32 at a time, the lanes
// with the same variable grouped (match.any) and the group's first lane
// applying their images in token order; structure tokens by the whole warp:
// entering an If or While saves, for every op token inside it, its variable's
// set (save[level][token]); at ELSE the then-results are kept (alt) and the
// entry sets restored; at the If's END the two results are joined; at the
// While's END the sets are joined into the loop-head sets and the body runs
// again if any grew.  Because every variable a construct touches has an op
// token inside it, these per-token copies cover exactly the variables that
// matter.  A While that runs again because an enclosing While does starts
// from its previous loop-head sets joined with its new entry sets: the sets
// only grow from one pass of an enclosing loop to the next, so that start lies
// below the new fixpoint and the iteration still ends on it, in fewer passes.
// Sets live in shared memory for programs of at most SMEM_VARS variables,
// else in the final_mask output; the image and fault tables in shared memory.
#include <cstdlib>

#include "amc_internal.cuh"
#include "batch.cuh"

namespace amc {

namespace {

constexpr int SMEM_VARS = 4096;
constexpr int BWARPS = 8;                  // warps per CTA
constexpr uint32_t MAX_WHILE_PASSES = 32;
constexpr int64_t SPLIT_DEFAULT = 65536;   // segment length of split programs (tokens)
constexpr int32_t SPLIT_VARS = 4096;       // programs with more variables are not split
constexpr int RED_CTAS = 64;               // CTAs of the reduce phase: each warp has its own save / alt rows

// Segment length (AMC_BATCH_SPLIT overrides it, 1,024 .. 2^30 tokens).  A
// program is split when one warp would take longer on it alone than the rest
// of the batch takes on all of them; at the measured rate of a lone warp that
// is far beyond the longest programs of the 100,000-program workload.
int64_t batch_split()
{
    int64_t v = SPLIT_DEFAULT;
    if (const char* e = getenv("AMC_BATCH_SPLIT")) {
        const long long x = atoll(e);
        if (x >= 1024 && x <= (1ll << 30)) v = x;
    }
    return v;
}
// longest segment a reduce pass takes (else the program is not split)
__host__ __device__ __forceinline__ int64_t seg_max_of(int64_t split) { return split + split / 2; }

__device__ __forceinline__ bool is_op(uint32_t ks) { return (ks & 0xE0u) == 0 && (ks & 15u) <= AMC_K_PW; }

struct WarpSmem {
    uint8_t M[SMEM_VARS];
    uint8_t stage[32];
    uint8_t outm[32];
};

struct TabSmem {
    uint8_t img[16 * 32];
    uint32_t flt[16];
};

// A unit of work: tokens [t0, t1) of program `prog`.
struct Unit {
    int64_t prog;
    int64_t t0, t1;
    int mode;                     // 0 apply; 1..5 reduce pass for entry status (mode - 1)
    int last;                     // apply: the program's last segment (writes final sets)
    const uint8_t* entry;         // apply of a later segment: entry sets (nv bytes); else null
    uint32_t* rel;                // reduce: relation row of the segment (nv words)
    uint8_t* rsave;               // reduce: the warp's save / alt rows ([AMC_MAX_DEPTH][seg_max] each)
    uint8_t* ralt;
    int whole;                    // apply of a whole program under the simple plan
};

// Runs one unit on the calling warp.
template <bool SMEM>
__device__ void run_unit(const BatchParams& p, const Unit& u, WarpSmem& S, const TabSmem& T)
{
    const int lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    const int64_t prog = u.prog;
    const int64_t pt0 = p.prog_tok_off[prog];          // program start (first-fault offsets)
    const int64_t t0 = u.t0, t1 = u.t1;
    const int32_t nv = p.prog_nvars[prog];
    uint8_t* gM = p.final_mask + p.prog_var_off[prog];
    uint8_t* M = SMEM ? S.M : gM;
    const bool apply = u.mode == 0;
    // entry sets
    for (int32_t v = lane; v < nv; v += 32) {
        uint8_t m;
        if (!apply) m = (uint8_t)(1u << (u.mode - 1));
        else if (u.entry) m = u.entry[v];
        else m = p.init_mask ? p.init_mask[p.prog_var_off[prog] + v] : (uint8_t)(1u << AMC_ST_VI);
        M[v] = m;
    }
    __syncwarp();
    int fk[AMC_MAX_DEPTH * 2];
    int64_t fpos[AMC_MAX_DEPTH * 3] = {};
    int depth = 0;
    int64_t ff = INT64_MAX;
    bool bad = false;
    int64_t pos = t0;
    // construct copies: per token in the apply phase; in a reduce pass per
    // token of the segment in the warp's own rows (the five passes of a
    // segment run at once on different warps)
    auto save_at = [&](int d, int64_t q) -> uint8_t* {
        return apply ? p.save + (int64_t)d * p.n_tokens + q : u.rsave + (int64_t)d * seg_max_of(p.split) + (q - t0);
    };
    auto alt_at = [&](int d, int64_t q) -> uint8_t* {
        return apply ? p.alt + (int64_t)d * p.n_tokens + q : u.ralt + (int64_t)d * seg_max_of(p.split) + (q - t0);
    };
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
            const int32_t pl = q < lim ? p.payload[q] : -1;
            const uint32_t opm = __ballot_sync(0xffffffffu, is_op(ks));
            const int cnt = __ffs(~opm) - 1 < 0 ? 32 : __ffs(~opm) - 1;
            const bool act = lane < cnt;
            int32_t v = act ? pl : -1;
            if (act && (v < 0 || v >= nv)) {
                raise_error(p.err, AMC_E_RANGE);
                v = -1;
            }
            const uint32_t oi = ((ks & 15u) << 1) | ((ks >> 4) & 1u);
            S.stage[lane] = (uint8_t)oi;
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
                    const uint32_t o = S.stage[L];
                    if (apply && ((T.flt[o] >> m) & 1u)) ff = min(ff, pos + L - pt0);
                    m = T.img[o * 32 + m];
                    S.outm[L] = (uint8_t)m;
                }
                M[v] = (uint8_t)m;
            }
            __syncwarp();
            if (apply && act) p.step_mask[q] = v >= 0 ? S.outm[lane] : 0;
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
                (p.tok[end] >> 4) || depth >= p.save_rows) {
                bad = true;
                break;
            }
            const int d = depth;
            // a While run again by an enclosing While restarts from its last
            // loop-head sets joined with the new entry sets
            bool rerun = false;
            if (k0 == AMC_T_WHILE)
                for (int e2 = 0; e2 < depth; ++e2) rerun |= fk[e2 * 2] == AMC_T_WHILE && fk[e2 * 2 + 1] > 0;
            if (rerun) {
                for_ops(pos + 1, end, [&](int64_t q2, int32_t v2) {
                    uint8_t* sp = save_at(d, q2);
                    *sp = (uint8_t)(*sp | M[v2]);
                });
                __syncwarp();
                for_ops(pos + 1, end, [&](int64_t q2, int32_t v2) { M[v2] = *save_at(d, q2); });
            } else {
                for_ops(pos + 1, end, [&](int64_t q2, int32_t v2) { *save_at(d, q2) = M[v2]; });
            }
            __syncwarp();
            fk[depth * 2] = (int)k0;
            fk[depth * 2 + 1] = 0;
            fpos[depth * 3 + 0] = pos;
            fpos[depth * 3 + 1] = e;
            fpos[depth * 3 + 2] = end;
            ++depth;
            if (apply && lane == 0) p.step_mask[pos] = 0;
            ++pos;
        } else if (k0 == AMC_T_ELSE) {
            if (!depth || fk[(depth - 1) * 2] != AMC_T_IF || fpos[(depth - 1) * 3 + 1] != pos || (ks0 >> 4)) {
                bad = true;
                break;
            }
            const int d = depth - 1;
            const int64_t a = fpos[d * 3], b = fpos[d * 3 + 2];
            for_ops(a + 1, b, [&](int64_t q2, int32_t v2) { *alt_at(d, q2) = M[v2]; });      // then-results
            __syncwarp();
            for_ops(a + 1, b, [&](int64_t q2, int32_t v2) { M[v2] = *save_at(d, q2); });   // entry sets again
            __syncwarp();
            if (apply && lane == 0) p.step_mask[pos] = 0;
            ++pos;
        } else if (k0 == AMC_T_END) {
            if (!depth || fpos[(depth - 1) * 3 + 2] != pos || (ks0 >> 4)) {
                bad = true;
                break;
            }
            const int d = depth - 1;
            const int64_t a = fpos[d * 3], b = pos;
            if (apply && lane == 0) p.step_mask[pos] = 0;
            if (fk[d * 2] == AMC_T_IF) {
                for_ops(a + 1, b, [&](int64_t q2, int32_t v2) { M[v2] = (uint8_t)(M[v2] | *alt_at(d, q2)); });
                __syncwarp();
                --depth;
                ++pos;
            } else {
                bool grew = false;
                for_ops(a + 1, b, [&](int64_t q2, int32_t v2) {
                    uint8_t* sp = save_at(d, q2);
                    const uint32_t x = *sp, nx = x | M[v2];
                    grew |= nx != x;
                    *sp = (uint8_t)nx;
                    M[v2] = (uint8_t)nx;
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
    __syncwarp();
    if (apply) {
        // program first fault: min over lanes, then over the program's segments
#pragma unroll
        for (int o = 16; o; o >>= 1) ff = min(ff, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)ff, o));
        if (lane == 0) {
            if (u.whole)                    // the only segment: the program's first fault
                p.prog_first_fault[prog] = ff == INT64_MAX ? -1 : ff;
            else if (ff != INT64_MAX)
                atomicMin(reinterpret_cast<unsigned long long*>(p.prog_first_fault + prog), (unsigned long long)ff);
        }
        if (SMEM && u.last)
            for (int32_t v = lane; v < nv; v += 32) gM[v] = M[v];
    } else {
        // the five passes of a segment run on different warps: each adds its row
        const int sh = 5 * (u.mode - 1);
        for (int32_t v = lane; v < nv; v += 32) atomicOr(u.rel + v, (uint32_t)M[v] << sh);
    }
}

// Segments: program p owns slots [slot_off[p], slot_off[p + 1]) when it is
// split (seg_t0[slot] = first token of the segment, -1 for a slot left empty
// because no top-level boundary fell in its stretch), none otherwise; its
// apply units are [unit_off[p], unit_off[p + 1]) -- one per slot, or one.
struct Plan {
    const int64_t* slot_off;      // [P + 1]
    const int64_t* unit_off;      // [P + 1]
    int64_t* seg_t0;              // [slots]
    uint8_t* E;                   // [slots][SPLIT_VARS] entry sets
    uint32_t* R;                  // [slots][SPLIT_VARS] relations
    uint8_t* rsave;               // [reduce warps][2][AMC_MAX_DEPTH][seg_max] reduce-pass copies
    int64_t* ord_off;             // [P + 1] apply units before the k-th program of the queue order
    int simple;                   // no program can be split: one unit per program, no planning
};

__device__ __forceinline__ int64_t split_slots(int64_t len, int32_t nv, int64_t split)
{
    return (len > split && nv >= 0 && nv <= SPLIT_VARS) ? (len + split - 1) / split : 0;
}

// largest p in [0, n) with off[p] <= i (off ascending, off[0] = 0)
__device__ __forceinline__ int64_t find_owner(const int64_t* off, int64_t n, int64_t i)
{
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// the segment of `slot` (program prog): [*a, *b), and whether it is the last
__device__ __forceinline__ bool segment_of(const BatchParams& p, const Plan& pl, int64_t prog, int64_t slot, int64_t* a,
                                           int64_t* b)
{
    *a = pl.seg_t0[slot];
    *b = p.prog_tok_off[prog + 1];
    const int64_t s_end = pl.slot_off[prog + 1];
    for (int64_t s2 = slot + 1; s2 < s_end; ++s2)
        if (pl.seg_t0[s2] >= 0) {
            *b = pl.seg_t0[s2];
            return false;
        }
    return true;
}

// phase 0: reduce passes, unit i = (slot i / 5, entry status i % 5);
// phase 1: apply, unit i of program find_owner(unit_off, P, i)
// MINB: resident CTAs per SM the register budget is fitted to (6: 40
// registers with a few spills, 48 warps per SM; 4: 64 registers, 32 warps)
// -- the tuner times both
template <int MINB>
__global__ void __launch_bounds__(BWARPS * 32, MINB) batch_kernel(const BatchParams p, const Plan pl, int phase)
{
    __shared__ WarpSmem smem[BWARPS];
    __shared__ TabSmem tab;
    const int w = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    WarpSmem& S = smem[w];
    for (int i = threadIdx.x; i < 16 * 32; i += blockDim.x) tab.img[i] = p.tab.img[i];
    if (threadIdx.x < 16) tab.flt[threadIdx.x] = p.tab.flt[threadIdx.x];
    __syncthreads();
    const int64_t wid = (int64_t)blockIdx.x * BWARPS + w;
    const int64_t sm = seg_max_of(p.split);
    uint8_t* rsave = pl.rsave + wid * 2 * (int64_t)AMC_MAX_DEPTH * sm;
    uint8_t* ralt = rsave + (int64_t)AMC_MAX_DEPTH * sm;
    // without any split program (simple plan) unit i is program i of the queue
    const int64_t n_slots = pl.simple ? 0 : pl.slot_off[p.n_progs];
    const int64_t n_units = pl.simple ? p.n_progs : pl.unit_off[p.n_progs];
    for (;;) {
        int64_t i = 0;
        if (lane == 0) i = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(p.queue_head), 1ull);
        i = __shfl_sync(0xffffffffu, (long long)i, 0);
        Unit u;
        if (phase == 0) {
            if (i >= 5 * n_slots) break;
            const int64_t slot = i / 5;
            const int64_t prog = find_owner(pl.slot_off, p.n_progs, slot);
            int64_t a, b;
            if (pl.seg_t0[slot] < 0 || segment_of(p, pl, prog, slot, &a, &b)) continue;   // empty, or last
            u.prog = prog;
            u.t0 = a;
            u.t1 = b;
            u.mode = 1 + (int)(i % 5);
            u.last = 0;
            u.whole = 0;
            u.entry = nullptr;
            u.rel = pl.R + slot * (int64_t)SPLIT_VARS;
            u.rsave = rsave;
            u.ralt = ralt;
        } else {
            if (i >= n_units) break;
            int64_t prog, j;
            if (pl.simple) {
                prog = p.order ? p.order[i] : i;
                j = 0;
            } else if (p.order) {           // programs longest first, their units in order
                const int64_t k = find_owner(pl.ord_off, p.n_progs, i);
                prog = p.order[k];
                j = i - pl.ord_off[k];
            } else {
                prog = find_owner(pl.unit_off, p.n_progs, i);
                j = i - pl.unit_off[prog];
            }
            const int64_t ns = pl.simple ? 0 : pl.slot_off[prog + 1] - pl.slot_off[prog];
            u.prog = prog;
            u.mode = 0;
            u.rel = nullptr;
            u.rsave = u.ralt = nullptr;
            u.whole = pl.simple;
            if (ns == 0) {
                u.t0 = p.prog_tok_off[prog];
                u.t1 = p.prog_tok_off[prog + 1];
                u.last = 1;
                u.entry = nullptr;
            } else {
                const int64_t slot = pl.slot_off[prog] + j;
                if (pl.seg_t0[slot] < 0) continue;
                int64_t a, b;
                u.last = segment_of(p, pl, prog, slot, &a, &b) ? 1 : 0;
                u.t0 = a;
                u.t1 = b;
                u.entry = j == 0 ? nullptr : pl.E + slot * (int64_t)SPLIT_VARS;
            }
        }
        const int32_t nv = p.prog_nvars[u.prog];
        const int64_t pt0 = p.prog_tok_off[u.prog], pt1 = p.prog_tok_off[u.prog + 1];
        if (pt0 < 0 || pt1 < pt0 || pt1 > p.n_tokens || nv < 0 || p.prog_var_off[u.prog] < 0 ||
            p.prog_var_off[u.prog + 1] - p.prog_var_off[u.prog] != nv) {
            if (lane == 0) raise_error(p.err, AMC_E_INVALID);
            continue;
        }
        if (nv <= SMEM_VARS)
            run_unit<true>(p, u, S, tab);
        else
            run_unit<false>(p, u, S, tab);
        __syncwarp();
    }
}

// One CTA: slot and unit offsets of every program (exclusive scans), and the
// programs' first faults set to -1 (then lowered by atomicMin).
__global__ void __launch_bounds__(1024) plan_offsets_kernel(const int64_t* __restrict__ tok_off,
                                                            const int32_t* __restrict__ nvars, int64_t P,
                                                            int64_t* __restrict__ slot_off,
                                                            int64_t* __restrict__ unit_off,
                                                            int64_t* __restrict__ prog_ff, int64_t split)
{
    __shared__ unsigned long long tmp_s[32], tmp_u[32];
    __shared__ unsigned long long carry_s, carry_u;
    if (threadIdx.x == 0) {
        carry_s = 0;
        carry_u = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t b0 = 0; b0 < P; b0 += 1024) {
        const int64_t pr = b0 + threadIdx.x;
        unsigned long long ns = 0, nu = 0;
        if (pr < P) {
            ns = (unsigned long long)split_slots(tok_off[pr + 1] - tok_off[pr], nvars[pr], split);
            nu = ns ? ns : 1ull;
            prog_ff[pr] = -1;
        }
        unsigned long long is = ns, iu = nu;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long ys = __shfl_up_sync(0xffffffffu, is, d);
            const unsigned long long yu = __shfl_up_sync(0xffffffffu, iu, d);
            if (lane >= d) {
                is += ys;
                iu += yu;
            }
        }
        if (lane == 31) {
            tmp_s[warp] = is;
            tmp_u[warp] = iu;
        }
        __syncthreads();
        unsigned long long ps = carry_s, pu = carry_u;
        for (int w2 = 0; w2 < warp; ++w2) {
            ps += tmp_s[w2];
            pu += tmp_u[w2];
        }
        if (pr < P) {
            slot_off[pr] = (int64_t)(ps + is - ns);
            unit_off[pr] = (int64_t)(pu + iu - nu);
        }
        __syncthreads();
        if (threadIdx.x == 1023) {
            carry_s = ps + is;
            carry_u = pu + iu;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        slot_off[P] = (int64_t)carry_s;
        unit_off[P] = (int64_t)carry_u;
    }
}

// Warp per split program: the segment starts.  Slot j's segment starts at the
// first top-level token boundary at or after the program start + j * split
// (slot 0 at the program start); a slot whose stretch has no such boundary
// before the next slot's target is left empty (-1).  Depth is tracked with a
// warp prefix sum of +1 (IF, WHILE) / -1 (END) over 32 tokens at a time.
__global__ void plan_cuts_kernel(const uint8_t* __restrict__ tok, const int64_t* __restrict__ tok_off,
                                 const int32_t* __restrict__ nvars, int64_t P, const int64_t* __restrict__ slot_off,
                                 int64_t* __restrict__ seg_t0, int64_t split)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t pr = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; pr < P; pr += nw) {
        const int64_t s0 = slot_off[pr], s1 = slot_off[pr + 1];
        if (s1 == s0) continue;
        const int64_t t0 = tok_off[pr], t1 = tok_off[pr + 1];
        for (int64_t s = s0 + lane; s < s1; s += 32) seg_t0[s] = s == s0 ? t0 : -1;
        __syncwarp();
        int depth = 0;                 // before the batch
        int64_t next = 1;              // next slot (relative) to place
        for (int64_t q0 = t0; q0 < t1 && next < s1 - s0; q0 += 32) {
            const int64_t q = q0 + lane;
            int delta = 0;
            if (q < t1) {
                const uint32_t k = tok[q] & 15u;
                delta = (k == AMC_T_IF || k == AMC_T_WHILE) ? 1 : (k == AMC_T_END ? -1 : 0);
            }
            int incl = delta;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            const int before = depth + incl - delta;         // depth before token q
            // token q starts a segment when it is at top level and at or past the next target
            bool cut = q < t1 && before == 0 && q > t0;
            uint32_t cand = __ballot_sync(0xffffffffu, cut);
            while (cand && next < s1 - s0) {
                const int L = __ffs(cand) - 1;
                const int64_t qq = q0 + L;
                const int64_t target = t0 + next * split;
                if (qq >= target) {
                    // the stretch of slot `next` is [target, target + split); later slots whose
                    // targets this boundary passes stay empty
                    while (next < s1 - s0 && t0 + (next + 1) * split <= qq) ++next;
                    if (lane == 0) seg_t0[s0 + next] = qq;
                    ++next;
                }
                cand &= cand - 1;
            }
            depth += __shfl_sync(0xffffffffu, incl, 31);
        }
        // a reduce pass keeps its construct copies for seg_max tokens: with a
        // longer segment before the last, the program runs as one segment
        __syncwarp();
        bool too_long = false;
        int64_t prev = t0;
        for (int64_t s = s0 + 1; s < s1; ++s) {
            const int64_t b = seg_t0[s];
            if (b < 0) continue;
            too_long |= b - prev > seg_max_of(split);
            prev = b;
        }
        __syncwarp();
        if (too_long)
            for (int64_t s = s0 + 1 + lane; s < s1; s += 32) seg_t0[s] = -1;
    }
}

// Queue order of the apply phase: programs by decreasing length bucket
// (floor(log2(tokens))); the order within a bucket is whatever the cursors
// give (it only decides which warp starts which program first).
__device__ __forceinline__ int len_bucket(int64_t len) { return len <= 0 ? 63 : 63 - (64 - __clzll(len)); }

__global__ void bucket_count_kernel(const int64_t* __restrict__ tok_off, int64_t n, int32_t* __restrict__ counts)
{
    __shared__ int32_t c[64];
    if (threadIdx.x < 64) c[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&c[len_bucket(tok_off[i + 1] - tok_off[i])], 1);
    __syncthreads();
    if (threadIdx.x < 64 && c[threadIdx.x]) atomicAdd(&counts[threadIdx.x], c[threadIdx.x]);
}

// bucket offsets, and the counters reused as the order kernel's cursors
__global__ void bucket_scan_kernel(int32_t* __restrict__ counts, int64_t* __restrict__ boff)
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

__global__ void order_kernel(const int64_t* __restrict__ tok_off, int64_t n, const int64_t* __restrict__ boff,
                             int32_t* __restrict__ cursor, int32_t* __restrict__ order)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = len_bucket(tok_off[i + 1] - tok_off[i]);
    order[boff[b] + atomicAdd(&cursor[b], 1)] = (int32_t)i;
}

// One CTA: ord_off[k] = apply units of the programs before position k of
// the queue order (exclusive scan).
__global__ void __launch_bounds__(1024) order_units_kernel(const int32_t* __restrict__ order,
                                                           const int64_t* __restrict__ unit_off, int64_t P,
                                                           int64_t* __restrict__ ord_off)
{
    __shared__ unsigned long long tmp[32];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t b0 = 0; b0 < P; b0 += 1024) {
        const int64_t k = b0 + threadIdx.x;
        unsigned long long c = 0;
        if (k < P) {
            const int64_t pr = order[k];
            c = (unsigned long long)(unit_off[pr + 1] - unit_off[pr]);
        }
        unsigned long long inc = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += y;
        }
        if (lane == 31) tmp[warp] = inc;
        __syncthreads();
        unsigned long long pre = carry;
        for (int w2 = 0; w2 < warp; ++w2) pre += tmp[w2];
        if (k < P) ord_off[k] = (int64_t)(pre + inc - c);
        __syncthreads();
        if (threadIdx.x == 1023) carry = pre + inc;
        __syncthreads();
    }
    if (threadIdx.x == 0) ord_off[P] = (int64_t)carry;
}

// Per split program and variable: entry sets of every segment from the
// relations of the ones before (image of the set through the 25-bit rows).
__global__ void carry_kernel(const BatchParams p, const Plan pl)
{
    // program by block, variable by thread
    for (int64_t pr = blockIdx.x; pr < p.n_progs; pr += gridDim.x) {
        const int64_t s0 = pl.slot_off[pr], s1 = pl.slot_off[pr + 1];
        if (s1 == s0) continue;
        const int32_t nv = p.prog_nvars[pr];
        for (int32_t v = threadIdx.x; v < nv; v += blockDim.x) {
            uint32_t m = p.init_mask ? p.init_mask[p.prog_var_off[pr] + v] : (1u << AMC_ST_VI);
            for (int64_t s = s0; s < s1; ++s) {
                if (pl.seg_t0[s] < 0) continue;
                pl.E[s * (int64_t)SPLIT_VARS + v] = (uint8_t)m;
                const uint32_t r = pl.R[s * (int64_t)SPLIT_VARS + v];
                uint32_t nm = 0;
#pragma unroll
                for (int i = 0; i < 5; ++i)
                    if ((m >> i) & 1u) nm |= (r >> (5 * i)) & 31u;
                m = nm;
            }
        }
    }
}

__global__ void zero_rel_kernel(const BatchParams p, const Plan pl)
{
    const int64_t n = pl.slot_off[p.n_progs] * (int64_t)SPLIT_VARS;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) pl.R[i] = 0;
}

struct BatchLayout {
    size_t save, alt, slot_off, unit_off, seg_t0, E, R, rsave, order, ord_off, counts, boff, head, total;
    int64_t max_slots;
    int64_t red_ctas;             // CTAs of the reduce phase (each warp owns construct-copy rows)
};

BatchLayout layout(int64_t n_tokens, int64_t n_progs, int64_t split, int save_rows)
{
    BatchLayout L;
    // a split program of length len has ceil(len / split) <= 2 len / split slots
    L.max_slots = 2 * (n_tokens / split) + 1;
    size_t o = 0;
    auto take = [&](size_t b) { const size_t at = o; o += align_up(b, 256); return at; };
    L.save = take((size_t)save_rows * (size_t)n_tokens + 1);
    L.alt = take((size_t)save_rows * (size_t)n_tokens + 1);
    L.slot_off = take(8 * ((size_t)n_progs + 1));
    L.unit_off = take(8 * ((size_t)n_progs + 1));
    L.seg_t0 = take(8 * (size_t)L.max_slots);
    L.E = take((size_t)L.max_slots * SPLIT_VARS);
    L.R = take(4 * (size_t)L.max_slots * SPLIT_VARS);
    // reduce-pass copies: one warp per reduce unit at most (five per slot)
    L.red_ctas = n_tokens > split ? (5 * L.max_slots + BWARPS - 1) / BWARPS : 0;
    if (L.red_ctas > RED_CTAS) L.red_ctas = RED_CTAS;
    L.rsave = take((size_t)L.red_ctas * BWARPS * 2 * AMC_MAX_DEPTH * (size_t)seg_max_of(split));
    L.order = take(4 * (size_t)n_progs + 4);
    L.ord_off = take(8 * ((size_t)n_progs + 1));
    L.counts = take(256);
    L.boff = take(512);
    L.head = take(256);
    L.total = o;
    return L;
}

}  // namespace

// no_split: programs are never split (a split length past any program)
int64_t split_of(bool no_split) { return no_split ? (int64_t)1 << 60 : batch_split(); }

size_t batch_workspace_bytes(int64_t n_tokens, int64_t n_progs)
{
    return layout(n_tokens, n_progs, batch_split(), AMC_MAX_DEPTH).total;
}

size_t batch_workspace_bytes(int64_t n_tokens, int64_t n_progs, bool no_split, int save_rows)
{
    return layout(n_tokens, n_progs, split_of(no_split), save_rows).total;
}

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
    p.split = split_of(B.no_split != 0);
    p.save_rows = B.save_rows < 0 ? 0 : (B.save_rows > AMC_MAX_DEPTH ? AMC_MAX_DEPTH : B.save_rows);
    const BatchLayout L = layout(B.n_tokens, B.n_progs, p.split, p.save_rows);
    uint8_t* w = static_cast<uint8_t*>(B.workspace);
    p.save = w + L.save;
    p.alt = w + L.alt;
    p.order = nullptr;
    p.queue_head = reinterpret_cast<uint64_t*>(w + L.head);
    Plan pl;
    pl.slot_off = reinterpret_cast<int64_t*>(w + L.slot_off);
    pl.unit_off = reinterpret_cast<int64_t*>(w + L.unit_off);
    pl.seg_t0 = reinterpret_cast<int64_t*>(w + L.seg_t0);
    pl.E = w + L.E;
    pl.R = reinterpret_cast<uint32_t*>(w + L.R);
    pl.rsave = w + L.rsave;
    pl.ord_off = reinterpret_cast<int64_t*>(w + L.ord_off);
    int32_t* order = reinterpret_cast<int32_t*>(w + L.order);
    int32_t* counts = reinterpret_cast<int32_t*>(w + L.counts);
    int64_t* boff = reinterpret_cast<int64_t*>(w + L.boff);
    if (B.n_progs <= 0) return AMC_OK;
    int dev = 0, n_sm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    auto kern = B.regs_capped ? batch_kernel<6> : batch_kernel<4>;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BWARPS * 32, 0);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)n_sm * per_sm;
    if (B.max_ctas > 0 && grid > B.max_ctas) grid = B.max_ctas;
    // no program longer than the split length: one unit per program, no planning
    pl.simple = B.n_tokens <= p.split ? 1 : 0;
    if (pl.simple) {
        const int64_t need = (B.n_progs + BWARPS - 1) / BWARPS;
        if (grid > need) grid = need;
    }
    if (B.profile & 1) profile_begin(s);
    if (!pl.simple) {
        plan_offsets_kernel<<<1, 1024, 0, s>>>(B.prog_tok_off, B.prog_nvars, B.n_progs,
                                               const_cast<int64_t*>(pl.slot_off), const_cast<int64_t*>(pl.unit_off),
                                               B.prog_first_fault, p.split);
        plan_cuts_kernel<<<n_sm * 4, 256, 0, s>>>(B.tok, B.prog_tok_off, B.prog_nvars, B.n_progs, pl.slot_off,
                                                  pl.seg_t0, p.split);
        zero_rel_kernel<<<n_sm * 4, 256, 0, s>>>(p, pl);
    }
    if (B.longest_first) {
        if (cudaMemsetAsync(counts, 0, 256, s) != cudaSuccess) return AMC_E_CUDA;
        bucket_count_kernel<<<128, 256, 0, s>>>(B.prog_tok_off, B.n_progs, counts);
        bucket_scan_kernel<<<1, 32, 0, s>>>(counts, boff);
        order_kernel<<<(unsigned)((B.n_progs + 255) / 256), 256, 0, s>>>(B.prog_tok_off, B.n_progs, boff, counts,
                                                                           order);
        if (!pl.simple) order_units_kernel<<<1, 1024, 0, s>>>(order, pl.unit_off, B.n_progs, pl.ord_off);
        p.order = order;
    }
    if (!pl.simple) {
        if (cudaMemsetAsync(p.queue_head, 0, 8, s) != cudaSuccess) return AMC_E_CUDA;
        const int64_t rgrid = grid < L.red_ctas ? grid : L.red_ctas;
        if (rgrid > 0) kern<<<(unsigned)rgrid, BWARPS * 32, 0, s>>>(p, pl, 0);      // reduce
        carry_kernel<<<n_sm * 4, 256, 0, s>>>(p, pl);
    }
    if (cudaMemsetAsync(p.queue_head, 0, 8, s) != cudaSuccess) return AMC_E_CUDA;
    kern<<<(unsigned)grid, BWARPS * 32, 0, s>>>(p, pl, 1);       // apply
    if (B.profile & 2) profile_end(s);
    return cudaGetLastError() == cudaSuccess ? AMC_OK : AMC_E_CUDA;
}

}  // namespace amc
