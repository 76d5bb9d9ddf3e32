// wd.cu -- static well-declaredness of calls AM{S} (Section 3.3, Definitions
// "Occurs in all execution paths" and "Well-declared program"; Section 3.5,
// "Well-declared program with array access").
//
// Per call, one warp:
//   * each statement of the body is checked against the call's declarations:
//     no Push / Pull; a write needs W or RW on its side, a read R or RW, for
//     the array that owns the location (one abstract variable per array);
//   * every W declaration obliges a write, on its side, of every location of
//     the array in all execution paths of the body.  That is relation mode
//     over a two-state machine per tracked location -- N "not written yet",
//     Y "written" -- with conditions opaque: w maps any state to Y, other ops
//     keep it, If is the union of its branches' sets and While the closure of
//     its body.  The obligation holds iff N is not in the set at the end.  The
//     warp keeps, per tracked location, the bit "N is not in the set" (lane j
//     owns 64 locations per word): an op sets its bit; at an If the then- and
//     else-sets come from the same entry, so the bit after it is entry OR
//     (then AND else); a While may run zero times, so its body adds nothing.
// The warp walks the body 32 tokens at a time: ops are checked in parallel,
// structure tokens by the whole warp with a stack of the entry / then bits.
#include "amc_internal.cuh"
#include "wd.cuh"

namespace amc {

namespace {

constexpr int WD_WARPS = 4;                   // warps per CTA
constexpr int WD_WORDS = 32;                  // tracked words per warp pass: 32 lanes x 64 locations

struct WdParams {
    const int64_t* arr_loc_off;
    int32_t n_arrays;
    const int32_t* loc_owner;
    const int64_t* call_tok_off;
    int64_t n_calls;
    const uint8_t* tok;
    const int32_t* payload;
    int64_t n_tokens;
    const int64_t* call_am_off;
    const int32_t* am_array;
    const uint8_t* am_mode;
    int64_t n_decls;
    uint32_t* violations;
    int64_t* first_bad;
    int32_t* first_unmet;
    unsigned long long* queue;     // next call to take
    int* err;
};

struct WdWarp {
    int32_t arr[AMC_WD_MAX_DECLS];
    uint8_t mode[AMC_WD_MAX_DECLS];
    int64_t base[AMC_WD_MAX_DECLS];       // first tracked bit of a W entry, -1 for R / RW
    uint64_t stack[2 * AMC_MAX_DEPTH][32];  // per level: entry bits, then-branch bits (per lane word)
    int64_t fend[AMC_MAX_DEPTH];          // END token of each open construct
    int64_t felse[AMC_MAX_DEPTH];         // ELSE token of an open If (-1 for While)
};

__device__ __forceinline__ bool wd_op_kind(uint32_t k) { return k <= AMC_K_NOOP; }

// One call: declarations into shared memory, then one pass over the body per
// window of WD_WORDS * 64 tracked locations (at least one pass, for the
// statement checks).
__device__ void wd_call(const WdParams& p, int64_t c, WdWarp& S)
{
    const int lane = threadIdx.x & 31;
    const int64_t n_locs = p.n_arrays > 0 ? p.arr_loc_off[p.n_arrays] : 0;
    const int64_t t0 = p.call_tok_off[c], t1 = p.call_tok_off[c + 1];
    const int64_t m0 = p.call_am_off[c], m1 = p.call_am_off[c + 1];
    if (t0 < 0 || t1 < t0 || t1 > p.n_tokens || m0 < 0 || m1 < m0 || m1 > p.n_decls ||
        m1 - m0 > AMC_WD_MAX_DECLS) {
        if (lane == 0) raise_error(p.err, AMC_E_INVALID);
        return;
    }
    const int nd = (int)(m1 - m0);
    uint32_t viol = 0;
    // declarations: range, mode, duplicates, tracked bases of the W entries
    int32_t a = -1;
    uint32_t md = 0;
    int64_t len = 0;
    if (lane < nd) {
        a = p.am_array[m0 + lane];
        md = p.am_mode[m0 + lane];
        if (a < 0 || a >= p.n_arrays) {
            raise_error(p.err, AMC_E_RANGE);
            a = -1;
        } else {
            len = p.arr_loc_off[a + 1] - p.arr_loc_off[a];
        }
        if ((md & 0xE0u) || (md & 15u) < 1 || (md & 15u) > 3) raise_error(p.err, AMC_E_INVALID);
    }
    for (int j = 0; j < nd; ++j) {
        const int32_t aj = __shfl_sync(0xffffffffu, a, j);
        if (lane > j && lane < nd && a >= 0 && a == aj) viol |= 16u;     // declared twice
    }
    const bool isw = lane < nd && a >= 0 && (md & 15u) == 2u;
    int64_t wl = isw ? len : 0;
    int64_t incl = wl;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    const int64_t tracked = __shfl_sync(0xffffffffu, incl, 31);
    if (lane < nd) {
        S.arr[lane] = a;
        S.mode[lane] = (uint8_t)md;
        S.base[lane] = isw ? incl - wl : -1;
    }
    __syncwarp();
    int64_t bad = INT64_MAX;
    int32_t unmet = INT32_MAX;
    bool malformed = false;
    const int64_t window = (int64_t)WD_WORDS * 64;
    for (int64_t w0 = 0; w0 == 0 || w0 < tracked; w0 += window) {
        const bool first_pass = w0 == 0;
        uint64_t cur = 0;                    // this lane's word: locations w0 + 64 lane + [0, 64)
        int depth = 0;
        for (int64_t pos = t0; pos < t1 && !malformed;) {
            const int64_t q = pos + lane;
            const bool in = q < t1;
            const uint32_t ks = in ? p.tok[q] : 0xFFu;
            const int32_t pl = in ? p.payload[q] : 0;
            const uint32_t k = ks & 15u;
            const bool op = in && !(ks & 0xE0u) && wd_op_kind(k);
            // the run of op tokens at the head of this batch
            const uint32_t nonop = __ballot_sync(0xffffffffu, !op);
            const int cnt = nonop ? __ffs(nonop) - 1 : 32;
            int64_t bit = -1;
            if (lane < cnt && k != AMC_K_NOOP) {
                if (pl < 0 || pl >= n_locs) {
                    raise_error(p.err, AMC_E_RANGE);
                } else if (k == AMC_K_PUSH || k == AMC_K_PULL) {
                    if (first_pass) {
                        viol |= 1u;
                        bad = min(bad, q - t0);
                    }
                } else {
                    const int32_t own = p.loc_owner[pl];
                    const uint32_t side = (ks >> 4) & 1u;
                    bool ok = false;
                    for (int j = 0; j < nd; ++j) {
                        if (S.arr[j] != own || ((S.mode[j] >> 4) & 1u) != side) continue;
                        const uint32_t m = S.mode[j] & 15u;
                        if (k == AMC_K_W && (m == 2u || m == 3u)) ok = true;
                        if (k == AMC_K_R && (m == 1u || m == 3u)) ok = true;
                        if (k == AMC_K_W && m == 2u) bit = S.base[j] + (pl - p.arr_loc_off[own]) - w0;
                    }
                    if (!ok && first_pass) {
                        viol |= k == AMC_K_W ? 2u : 4u;
                        bad = min(bad, q - t0);
                    }
                }
            }
            // the run's tracked writes set their bits in the owning lanes' words
            for (int L = 0; L < cnt; ++L) {
                const int64_t b = __shfl_sync(0xffffffffu, bit, L);
                if (b >= 0 && b < window && (int)(b >> 6) == lane) cur |= 1ull << (b & 63);
            }
            pos += cnt;
            if (cnt == 32) continue;
            if (pos >= t1) break;
            // one structure token, by the whole warp
            const uint32_t sks = __shfl_sync(0xffffffffu, ks, cnt);
            const int32_t spl = __shfl_sync(0xffffffffu, pl, cnt);
            const uint32_t sk = sks & 15u;
            const int64_t lim = depth ? S.fend[depth - 1] : t1;
            if (sks & 0xF0u) {                                // structure tokens carry no side
                malformed = true;
                break;
            }
            if (sk == AMC_T_IF || sk == AMC_T_WHILE) {
                int64_t e = -1, end = -1;
                if (spl >= 0) {
                    if (sk == AMC_T_IF) {
                        e = pos + 1 + spl;
                        if (e < lim && p.tok[e] == AMC_T_ELSE && p.payload[e] >= 0) end = e + 1 + p.payload[e];
                    } else {
                        end = pos + 1 + spl;
                    }
                }
                if (end <= pos || end >= lim || p.tok[end] != AMC_T_END || depth >= AMC_MAX_DEPTH) {
                    malformed = true;
                    break;
                }
                S.stack[2 * depth][lane] = cur;             // entry bits
                S.fend[depth] = end;
                S.felse[depth] = sk == AMC_T_IF ? e : -1;
                ++depth;
                cur = 0;                                     // the branch / body from scratch
                ++pos;
            } else if (sk == AMC_T_ELSE) {
                if (!depth || S.felse[depth - 1] != pos) {
                    malformed = true;
                    break;
                }
                S.stack[2 * (depth - 1) + 1][lane] = cur;   // then-branch bits
                cur = 0;
                ++pos;
            } else if (sk == AMC_T_END) {
                if (!depth || S.fend[depth - 1] != pos) {
                    malformed = true;
                    break;
                }
                --depth;
                const uint64_t entry = S.stack[2 * depth][lane];
                cur = S.felse[depth] >= 0 ? (entry | (S.stack[2 * depth + 1][lane] & cur)) : entry;
                ++pos;
            } else {
                malformed = true;                            // pw / GT / EN, or a byte out of range
                break;
            }
            __syncwarp();
        }
        if (depth) malformed = true;
        if (malformed) break;
        // W obligations whose tracked bits fall in this window
        for (int j = 0; j < nd; ++j) {
            const int64_t b0 = S.base[j];
            if (b0 < 0) continue;
            const int32_t aj = S.arr[j];
            const int64_t n = p.arr_loc_off[aj + 1] - p.arr_loc_off[aj];
            const int64_t lo = max(b0, w0) - w0, hi = min(b0 + n, w0 + window) - w0;
            if (lo >= hi) continue;
            // bits [lo, hi) of the window: lane words [64 lane, 64 lane + 64)
            const int64_t wlo = (int64_t)lane * 64, whi = wlo + 64;
            const int64_t a0 = max(lo, wlo), a1 = min(hi, whi);
            bool miss = false;
            if (a0 < a1) {
                const int s0 = (int)(a0 - wlo), s1 = (int)(a1 - wlo);
                const uint64_t need = (s1 - s0 == 64) ? ~0ull : (((1ull << (s1 - s0)) - 1ull) << s0);
                miss = (cur & need) != need;
            }
            if (__any_sync(0xffffffffu, miss)) {
                viol |= 8u;
                unmet = min(unmet, aj);
            }
        }
    }
    if (malformed) {
        if (lane == 0) raise_error(p.err, AMC_E_INVALID);
        return;
    }
    // combine the lanes' findings
    viol = __reduce_or_sync(0xffffffffu, viol);
#pragma unroll
    for (int d = 16; d; d >>= 1) bad = min(bad, (int64_t)__shfl_xor_sync(0xffffffffu, (long long)bad, d));
    unmet = __reduce_min_sync(0xffffffffu, unmet);
    if (lane == 0) {
        p.violations[c] = viol;
        p.first_bad[c] = bad == INT64_MAX ? -1 : bad;
        p.first_unmet[c] = unmet == INT32_MAX ? -1 : unmet;
    }
}

__global__ void __launch_bounds__(WD_WARPS * 32) wd_kernel(const WdParams p)
{
    __shared__ WdWarp S[WD_WARPS];
    const int w = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    for (;;) {
        long long c = 0;
        if (lane == 0) c = (long long)atomicAdd(p.queue, 1ull);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= p.n_calls) break;
        wd_call(p, c, S[w]);
        __syncwarp();
    }
}

}  // namespace

size_t wd_workspace_bytes() { return 256; }

int launch_well_declared(const WdLaunch& L, cudaStream_t s)
{
    if (L.n_calls == 0) return AMC_OK;
    WdParams p;
    p.arr_loc_off = L.arr_loc_off;
    p.n_arrays = L.n_arrays;
    p.loc_owner = L.loc_owner;
    p.call_tok_off = L.call_tok_off;
    p.n_calls = L.n_calls;
    p.tok = L.tok;
    p.payload = L.payload;
    p.n_tokens = L.n_tokens;
    p.call_am_off = L.call_am_off;
    p.am_array = L.am_array;
    p.am_mode = L.am_mode;
    p.n_decls = L.n_decls;
    p.violations = L.violations;
    p.first_bad = L.first_bad;
    p.first_unmet = L.first_unmet;
    p.queue = static_cast<unsigned long long*>(L.workspace);
    p.err = L.err;
    if (cudaMemsetAsync(p.queue, 0, sizeof(unsigned long long), s) != cudaSuccess) return AMC_E_CUDA;
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t need = (L.n_calls + WD_WARPS - 1) / WD_WARPS;
    const int grid = (int)(need < (int64_t)n_sm * 8 ? need : (int64_t)n_sm * 8);
    if (L.profile & 1) profile_begin(s);
    wd_kernel<<<grid, WD_WARPS * 32, 0, s>>>(p);
    if (L.profile & 2) profile_end(s);
    return cudaGetLastError() == cudaSuccess ? AMC_OK : AMC_E_CUDA;
}

}  // namespace amc
