// dscan.cu -- device-wide exclusive scan (int32 counts -> int64 offsets).
#include "dscan.cuh"

namespace amc {

namespace {

constexpr int SCAN_NT = 512;
constexpr int SCAN_IPT = 16;
constexpr int SCAN_TILE = SCAN_NT * SCAN_IPT;

__device__ __forceinline__ long long warp_incl_sum64(long long x)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// exclusive block scan of one value per thread; returns the block total in *total
__device__ long long block_excl_sum64(long long x, long long* tmp, long long* total)
{
    constexpr int NW = SCAN_NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long incl = warp_incl_sum64(x);
    if (lane == 31) tmp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < NW ? tmp[lane] : 0;
        long long wi = warp_incl_sum64(w);
        if (lane < NW) tmp[lane] = wi - w;
        if (lane == NW - 1) tmp[NW] = wi;
    }
    __syncthreads();
    long long r = incl - x + tmp[warp];
    *total = tmp[NW];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SCAN_NT) scan_reduce(const int32_t* __restrict__ in, int64_t n,
                                                       long long* __restrict__ block_sums)
{
    __shared__ long long tmp[SCAN_NT / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    long long s = 0;
    for (int k = 0; k < SCAN_IPT; ++k) {
        const int64_t i = base + (int64_t)k * SCAN_NT + threadIdx.x;
        if (i < n) s += in[i];
    }
    long long total;
    block_excl_sum64(s, tmp, &total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_NT) scan_top(long long* __restrict__ block_sums, int64_t n_blocks)
{
    __shared__ long long tmp[SCAN_NT / 32 + 1];
    long long carry = 0;
    for (int64_t lo = 0; lo < n_blocks; lo += SCAN_NT) {
        const int64_t i = lo + threadIdx.x;
        const long long x = i < n_blocks ? block_sums[i] : 0;
        long long total;
        const long long e = block_excl_sum64(x, tmp, &total);
        if (i < n_blocks) block_sums[i] = carry + e;
        carry += total;
    }
    if (threadIdx.x == 0) block_sums[n_blocks] = carry;
}

__global__ void __launch_bounds__(SCAN_NT) scan_apply(const int32_t* __restrict__ in, int64_t n,
                                                      const long long* __restrict__ block_sums,
                                                      int64_t* __restrict__ out, int64_t n_blocks)
{
    __shared__ long long tmp[SCAN_NT / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_IPT;
    long long v[SCAN_IPT];
    long long s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        const int64_t i = base + k;
        v[k] = i < n ? in[i] : 0;
        s += v[k];
    }
    long long total;
    long long run = block_excl_sum64(s, tmp, &total) + block_sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) {
        const int64_t i = base + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = block_sums[n_blocks];
}

}  // namespace

size_t dscan_workspace_bytes(int64_t n)
{
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    return align_up(8 * (size_t)(nb + 1), 256);
}

int dscan_exclusive(const int32_t* in, int64_t* out, int64_t n, void* workspace, cudaStream_t s)
{
    long long* bs = static_cast<long long*>(workspace);
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 0) {
        if (cudaMemsetAsync(out, 0, 8, s) != cudaSuccess) return AMC_E_CUDA;
        return AMC_OK;
    }
    scan_reduce<<<(unsigned)nb, SCAN_NT, 0, s>>>(in, n, bs);
    scan_top<<<1, SCAN_NT, 0, s>>>(bs, nb);
    scan_apply<<<(unsigned)nb, SCAN_NT, 0, s>>>(in, n, bs, out, nb);
    return cudaGetLastError() == cudaSuccess ? AMC_OK : AMC_E_CUDA;
}

}  // namespace amc
