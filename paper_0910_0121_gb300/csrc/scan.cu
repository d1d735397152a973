// Device-wide exclusive prefix sum of uint32 arrays (reduce, scan the block sums,
// scan again with offsets).  Used for the node-ownership counts, group flags and
// radix-sort histograms.
#include "common.cuh"

namespace greem {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048

static inline size_t ceil_div(size_t a, size_t b) { return (a + b - 1) / b; }

size_t scan_scratch_elems(size_t n)
{
    size_t tot = 0;
    while (n > 1) {
        n = ceil_div(n, kScanTile);
        tot += n + 1;
    }
    return tot + 4;
}

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total)
{
    __shared__ uint32_t wsum[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < kScanThreads / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kScanThreads / 32) wsum[lane] = s;
    }
    __syncthreads();
    uint32_t before = (w > 0 ? wsum[w - 1] : 0) + x - v;
    *total = wsum[kScanThreads / 32 - 1];
    __syncthreads();
    return before;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ in, size_t n,
                                                               uint32_t *__restrict__ sums)
{
    size_t base = (size_t)blockIdx.x * kScanTile;
    uint32_t s = 0;
#pragma unroll
    for (int t = 0; t < kScanItems; t++) {
        size_t i = base + (size_t)t * kScanThreads + threadIdx.x;
        if (i < n) s += in[i];
    }
    uint32_t tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Each thread owns kScanItems consecutive elements.
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t *in, size_t n,
                                                             const uint32_t *__restrict__ offs, uint32_t *out)
{
    size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int t = 0; t < kScanItems; t++) {
        size_t i = base + t;
        v[t] = i < n ? in[i] : 0;
        s += v[t];
    }
    uint32_t tot;
    uint32_t run = block_exclusive_scan(s, &tot) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
    for (int t = 0; t < kScanItems; t++) {
        size_t i = base + t;
        if (i < n) out[i] = run;
        run += v[t];
    }
    // the thread holding element n-1 also writes the total at out[n]
    if (base < n && n - 1 < base + kScanItems) out[n] = run;
}

void scan_u32(const uint32_t *in, uint32_t *out, size_t n, uint32_t *scratch, cudaStream_t s)
{
    if (n == 0) {
        cudaMemsetAsync(out, 0, sizeof(uint32_t), s);
        return;
    }
    size_t nb = ceil_div(n, kScanTile);
    if (nb == 1) {
        k_scan_down<<<1, kScanThreads, 0, s>>>(in, n, nullptr, out);
        g_launches++;
        return;
    }
    uint32_t *sums = scratch;  // nb + 1 entries
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums);
    g_launches++;
    scan_u32(sums, sums, nb, scratch + nb + 1, s);
    k_scan_down<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums, out);
    g_launches++;
}

}  // namespace greem
