// hostcopy.cu -- a finished result copied into host memory.  When the whole
// destination range is page-locked host memory that this device can address,
// the copy is a kernel whose stores travel straight over the CPU-GPU link;
// otherwise (pageable memory) it is a copy-engine transfer.  On GB300 with a
// Grace host both reach about 190 GB/s for a 512 MB result, but repeated
// copy-engine transfers were measured to stall for 5 to 35 ms about every
// half second on a system that had been busy for a while, while the SM stores
// into the same pinned buffer never did.
#include "cat_internal.cuh"

#include <algorithm>
#include <cstddef>

namespace cat {

constexpr int kToHostThreads = 512;
constexpr int kToHostBlocks = 608;  // 4 per SM: enough stores in flight for the link

__global__ void __launch_bounds__(kToHostThreads) to_host_u4(const uint4 *__restrict__ src,
                                                            uint4 *__restrict__ dst, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

__global__ void __launch_bounds__(kToHostThreads) to_host_u32(const uint32_t *__restrict__ src,
                                                             uint32_t *__restrict__ dst, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// The device address of host range [p, p + bytes) when both of its ends lie in
// page-locked host memory mapped for the current device at device addresses
// exactly bytes - 1 apart; null otherwise.  (The range is the caller's one
// output buffer, so its ends lie in the same allocation.)
static void *mapped_host_range(void *p, size_t bytes)
{
    cudaPointerAttributes a{}, b{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    char *last = static_cast<char *>(p) + bytes - 1;
    if (cudaPointerGetAttributes(&b, last) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (b.type != cudaMemoryTypeHost || !b.devicePointer) return nullptr;
    if (static_cast<char *>(b.devicePointer) - static_cast<char *>(a.devicePointer) !=
        (std::ptrdiff_t)(bytes - 1))
        return nullptr;
    return a.devicePointer;
}

void copy_to_host(Ctx &c, uint32_t *host, const uint32_t *dev, size_t n, cudaStream_t s)
{
    if (n == 0) return;
    void *d = mapped_host_range(host, 4 * n);
    if (!d) {
        CAT_CUDA(cudaMemcpyAsync(host, dev, 4 * n, cudaMemcpyDeviceToHost, s));
        return;
    }
    const int tok = prof_begin(c, "to_host", s);
    const bool wide = ((reinterpret_cast<uintptr_t>(d) | reinterpret_cast<uintptr_t>(dev)) & 15) == 0;
    const size_t items = wide ? n / 4 : n;
    const unsigned blocks = (unsigned)std::min<size_t>(
        kToHostBlocks, std::max<size_t>(1, (items + kToHostThreads - 1) / kToHostThreads));
    if (wide) {
        if (items)
            to_host_u4<<<blocks, kToHostThreads, 0, s>>>(reinterpret_cast<const uint4 *>(dev),
                                                         static_cast<uint4 *>(d), items);
        const size_t done = 4 * items;
        if (done < n)  // the last one to three limbs
            to_host_u32<<<1, 32, 0, s>>>(dev + done, static_cast<uint32_t *>(d) + done, n - done);
    } else {
        to_host_u32<<<blocks, kToHostThreads, 0, s>>>(dev, static_cast<uint32_t *>(d), n);
    }
    CAT_LAUNCH("to_host");
    prof_end(c, tok, s, 8.0 * (double)n);
}

}  // namespace cat
