// amc_internal.cuh -- device helpers and tables shared by the kernels of the
// access-mode consistency checker (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "amc.h"

namespace amc {

// ---------------------------------------------------------------------------
// Encodings (mirrors include/amc.h)
// ---------------------------------------------------------------------------
constexpr int ST_F = 4;
constexpr uint32_t NIL = 0xFFFFFFFFu;
constexpr uint8_t ELEM_BAD = 0xFF;      // op byte that is not a trace op
constexpr uint8_t ELEM_GT = 0xFE;       // guarded transfer: resolved at decode
constexpr int MAX_ELEMS = 32;

// Transfer functions of single ops form a finite monoid under composition
// (the sequencing of Section 3.2 is associative with Noop as unit).  Each op
// byte maps to an element id; comp[a][b] is "a then b"; app[a][s] applies a
// to status s.  Built on the host (monoid.cu) from the effect rules and passed
// to kernels by value.
struct Tables {
    uint8_t comp[MAX_ELEMS * MAX_ELEMS];
    uint8_t app[MAX_ELEMS * 8];
    uint8_t elem_of[256];           // op byte -> element id / ELEM_BAD / ELEM_GT
    uint8_t pull_of_side[2];        // element of the Fig. sem-AM transfer per side
    uint8_t identity;
    uint8_t n_elems;
};

// Host: the tables (built once per process).
const Tables& host_tables();

// Status-set images for relation mode.  Op index o = kind << 1 | side for
// kinds 0..5; img[o * 32 + m] = image of the set m; bit m of flt[o] is set when
// the set m holds a non-stuck status that op o makes stuck.
struct SetTables {
    uint8_t img[16 * 32];
    uint32_t flt[16];
};
const SetTables& host_set_tables();

// Host: address of the device-side error word of the current device (first
// error wins), or nullptr if it could not be resolved.
int* device_error_word();

// Host: profiling events of the calling thread (see amc_set_profile_events).
void set_profile_events(cudaEvent_t start, cudaEvent_t stop);
void profile_begin(cudaStream_t s);
void profile_end(cudaStream_t s);

__device__ __forceinline__ void raise_error(int* err, int code)
{
    atomicCAS(err, 0, code);
}

// ---------------------------------------------------------------------------
// Memory-order helpers (PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_acquire_u8(const uint8_t* p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u8 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_u8(const uint8_t* p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u8 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_u8(uint8_t* p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.u8 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---------------------------------------------------------------------------
// Bulk copies global -> shared through the async proxy, completion tracked by
// an mbarrier (no tensor map, no multicast).  Addresses and sizes are
// multiples of 16 bytes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bounded wait on an mbarrier phase.  Returns false (and raises
// AMC_E_TIMEOUT) when the phase did not complete within the bound.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* err)
{
    for (uint32_t it = 0; it < (1u << 24); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
    }
    raise_error(err, AMC_E_TIMEOUT);
    return false;
}

// ---------------------------------------------------------------------------
// Block-wide helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int warp_incl_sum(int x)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive block sum; tmp needs (NT/32 + 1) ints.  Contains __syncthreads.
template <int NT>
__device__ __forceinline__ int block_excl_sum(int x, int* tmp, int* total)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = warp_incl_sum(x);
    if (lane == 31) tmp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int w = lane < NW ? tmp[lane] : 0;
        int wi = warp_incl_sum(w);
        if (lane < NW) tmp[lane] = wi - w;
        if (lane == NW - 1) tmp[NW] = wi;
    }
    __syncthreads();
    int res = incl - x + tmp[warp];
    if (total) *total = tmp[NW];
    __syncthreads();
    return res;
}

__host__ __device__ constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace amc
