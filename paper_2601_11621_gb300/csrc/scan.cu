// scan.cu -- in-place exclusive prefix sum of uint32 arrays (segment counts
// of the sieve, digit counts of the radix grouping), in three passes: block
// sums, a scan of the block sums, and the per-block scans with offsets.
#include "cat_internal.cuh"

namespace cat {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ uint32_t block_exclusive_sum(uint32_t v, uint32_t *wsm, uint32_t *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc += o;
    }
    __syncthreads();
    if (lane == 31) wsm[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < nw ? wsm[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += o;
        }
        wsm[lane] = w;
    }
    __syncthreads();
    *total = wsm[nw - 1];
    return (wid > 0 ? wsm[wid - 1] : 0) + inc - v;
}

__global__ void __launch_bounds__(kScanThreads) scan_block_sums(const uint32_t *d, size_t n,
                                                                uint32_t *sums)
{
    __shared__ uint32_t wsm[32];
    const size_t base = (size_t)blockIdx.x * kScanChunk + (size_t)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++)
        if (base + k < n) s += d[base + k];
    uint32_t total;
    block_exclusive_sum(s, wsm, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Single block: exclusive scan of n values (any n), chunk by chunk.
__global__ void __launch_bounds__(kScanThreads) scan_single(uint32_t *d, size_t n)
{
    __shared__ uint32_t wsm[32];
    uint32_t run = 0;
    for (size_t base = 0; base < n; base += kScanChunk) {
        const size_t i0 = base + (size_t)threadIdx.x * kScanItems;
        uint32_t v[kScanItems], s = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            v[k] = i0 + k < n ? d[i0 + k] : 0;
            s += v[k];
        }
        uint32_t total;
        uint32_t ex = block_exclusive_sum(s, wsm, &total) + run;
#pragma unroll
        for (int k = 0; k < kScanItems; k++) {
            if (i0 + k < n) d[i0 + k] = ex;
            ex += v[k];
        }
        run += total;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanThreads) scan_apply(uint32_t *d, size_t n,
                                                           const uint32_t *offs)
{
    __shared__ uint32_t wsm[32];
    const size_t i0 = (size_t)blockIdx.x * kScanChunk + (size_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems], s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        v[k] = i0 + k < n ? d[i0 + k] : 0;
        s += v[k];
    }
    uint32_t total;
    uint32_t ex = block_exclusive_sum(s, wsm, &total) + offs[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        if (i0 + k < n) d[i0 + k] = ex;
        ex += v[k];
    }
}

void exclusive_scan_u32(Ctx &c, uint32_t *data, size_t n, cudaStream_t s)
{
    if (n == 0) return;
    const size_t blocks = (n + kScanChunk - 1) / kScanChunk;
    if (blocks <= 4) {
        scan_single<<<1, kScanThreads, 0, s>>>(data, n);
        CAT_LAUNCH("scan_single");
        return;
    }
    DevBuf<uint32_t> sums(c, blocks, s);
    scan_block_sums<<<(unsigned)blocks, kScanThreads, 0, s>>>(data, n, sums.get());
    CAT_LAUNCH("scan_block_sums");
    scan_single<<<1, kScanThreads, 0, s>>>(sums.get(), blocks);
    CAT_LAUNCH("scan_single");
    scan_apply<<<(unsigned)blocks, kScanThreads, 0, s>>>(data, n, sums.get());
    CAT_LAUNCH("scan_apply");
}

}  // namespace cat
