// comba.cu -- the lower levels of the balanced product tree (Sec. 3.2):
// many independent small products, by column-wise schoolbook ("Comba")
// multiplication with 96-bit column accumulators built from 32x32->64
// multiply-add chains.
//
// Layout: a tree level is an array of nodes in fixed slots of S limbs (node i
// at [i S, (i+1) S)), zero-padded.  A product of 2^k values below 2^32 always
// fits in 2^k limbs, so the product of adjacent nodes (2i, 2i+1) fits the
// next level's slot of 2S limbs exactly.
#include "cat_internal.cuh"

namespace cat {

// c2:c1:c0 += a * b  (96-bit accumulator)
__device__ __forceinline__ void mac96(uint32_t a, uint32_t b, uint32_t &c0, uint32_t &c1,
                                      uint32_t &c2)
{
    asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
        "addc.u32 %2, %2, 0;\n\t"
        : "+r"(c0), "+r"(c1), "+r"(c2)
        : "r"(a), "r"(b));
}

// --------------------------------------------------------------- leaves

constexpr int kLeafSlot = 8;

// Node i (eight limbs) = product of values[lpn i .. lpn i + lpn) (values
// past `count` count as 1; the caller picks lpn so that the product fits),
// accumulated by single-limb multiplications.
__global__ void leaf_products(const uint32_t *v, size_t count, uint32_t *out, size_t nodes,
                              int lpn)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nodes) return;
    uint32_t acc[kLeafSlot];
#pragma unroll
    for (int j = 0; j < kLeafSlot; j++) acc[j] = 0;
    acc[0] = 1;
    for (int k = 0; k < lpn; k++) {
        const size_t idx = i * (size_t)lpn + k;
        const uint32_t x = idx < count ? v[idx] : 1u;
        uint32_t carry = 0;
#pragma unroll
        for (int j = 0; j < kLeafSlot; j++) {
            const uint64_t t = (uint64_t)acc[j] * x + carry;
            acc[j] = (uint32_t)t;
            carry = (uint32_t)(t >> 32);
        }
    }
    uint4 *o = reinterpret_cast<uint4 *>(out + i * kLeafSlot);
    o[0] = make_uint4(acc[0], acc[1], acc[2], acc[3]);
    o[1] = make_uint4(acc[4], acc[5], acc[6], acc[7]);
}

// ---------------------------------------------- one product per thread

template <int S>
__global__ void comba_thread(const uint32_t *in, size_t nprod, uint32_t *out,
                             const uint32_t *out_index)
{
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nprod) return;
    const uint4 *a4 = reinterpret_cast<const uint4 *>(in + 2 * k * S);
    uint32_t A[S], B[S], O[2 * S];
#pragma unroll
    for (int i = 0; i < S / 4; i++) {
        const uint4 x = a4[i], y = a4[S / 4 + i];
        A[4 * i] = x.x; A[4 * i + 1] = x.y; A[4 * i + 2] = x.z; A[4 * i + 3] = x.w;
        B[4 * i] = y.x; B[4 * i + 1] = y.y; B[4 * i + 2] = y.z; B[4 * i + 3] = y.w;
    }
    uint32_t c0 = 0, c1 = 0, c2 = 0;
#pragma unroll
    for (int col = 0; col < 2 * S - 1; col++) {
#pragma unroll
        for (int i = 0; i < S; i++) {
            const int j = col - i;
            if (j >= 0 && j < S) mac96(A[i], B[j], c0, c1, c2);
        }
        O[col] = c0;
        c0 = c1;
        c1 = c2;
        c2 = 0;
    }
    O[2 * S - 1] = c0;
    const size_t node = out_index ? (size_t)out_index[k] : k;
    uint4 *o4 = reinterpret_cast<uint4 *>(out + 2 * node * S);
#pragma unroll
    for (int i = 0; i < S / 2; i++)
        o4[i] = make_uint4(O[4 * i], O[4 * i + 1], O[4 * i + 2], O[4 * i + 3]);
}

// ------------------------------------------------ one product per warp

constexpr int kWarpsPerBlock = 8;

// Lane l owns output columns [l W, l W + W), W = 2S/32 >= 2, and the lanes
// step through i = 0 .. S-1 together: column col gains A[i] B[col - i], B read
// as zero outside [0, S).  At step i lane l needs B[l W - i + w], w < W: a
// window that slides down by one word per step, so a step is one broadcast
// read of A[i], one new word of B and W multiply-adds.  The zero-padded copy
// of B (word j at j' = j + S, j' < 3S) is stored skewed, j' at j' + j' / W, so
// that the lanes' reads, W words apart, fall in distinct banks (W + 1 is odd).
//
// The column sums form a number N_l = low_l + high_l 2^(32W) per lane with
// high_l < 2^41; the product is sum_l (low_l + high_{l-1}) 2^(32 W l).  Each
// lane's addition low_l + high_{l-1} carries at most one bit out, and the
// one-bit carries are resolved by a generate/propagate scan across the warp.
template <int S>
__global__ void __launch_bounds__(32 * kWarpsPerBlock) comba_warp(const uint32_t *in,
                                                                  size_t nprod, uint32_t *out,
                                                                  const uint32_t *out_index)
{
    constexpr int W = 2 * S / 32;
    static_assert(W >= 2, "warp Comba needs at least two columns per lane");
    constexpr int PADN = 3 * S;              // padded indices j' in [0, 3S)
    constexpr int BWORDS = PADN + PADN / W;  // skewed layout
    __shared__ uint32_t smA[kWarpsPerBlock][S];
    __shared__ uint32_t smB[kWarpsPerBlock][BWORDS];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const size_t k = (size_t)blockIdx.x * kWarpsPerBlock + wid;
    if (k >= nprod) return;
    const uint32_t *src = in + 2 * k * S;
    uint32_t *A = smA[wid], *Bs = smB[wid];
    for (int i = lane; i < S; i += 32) A[i] = src[i];
    for (int jp = lane; jp < PADN; jp += 32) {
        const int j = jp - S;
        Bs[jp + jp / W] = (j >= 0 && j < S) ? src[S + j] : 0u;
    }
    __syncwarp();
    uint32_t c0[W], c1[W], c2[W], b[W];
#pragma unroll
    for (int w = 0; w < W; w++) {
        c0[w] = c1[w] = c2[w] = 0;
        const int jp = lane * W + w + S;
        b[w] = Bs[jp + jp / W];
    }
#pragma unroll
    for (int i = 0; i < S; i++) {
        const uint32_t a = A[i];
#pragma unroll
        for (int w = 0; w < W; w++) mac96(a, b[w], c0[w], c1[w], c2[w]);
        if (i + 1 < S) {
#pragma unroll
            for (int w = W - 1; w > 0; w--) b[w] = b[w - 1];
            // j' = l W + (S - i - 1) with S - i - 1 >= 0: j' / W = l + (S - i - 1) / W
            b[0] = Bs[lane * (W + 1) + (S - i - 1) + (S - i - 1) / W];
        }
    }
    uint32_t limb[W];
    // carry the running 96-bit sum through the lane's columns
    uint32_t r0 = 0, r1 = 0, r2 = 0;
#pragma unroll
    for (int w = 0; w < W; w++) {
        asm("add.cc.u32 %0, %0, %3;\n\t"
            "addc.cc.u32 %1, %1, %4;\n\t"
            "addc.u32 %2, %2, %5;\n\t"
            : "+r"(r0), "+r"(r1), "+r"(r2)
            : "r"(c0[w]), "r"(c1[w]), "r"(c2[w]));
        limb[w] = r0;
        r0 = r1;
        r1 = r2;
        r2 = 0;
    }
    const uint64_t high = ((uint64_t)r1 << 32) | r0;
    uint64_t hprev = __shfl_up_sync(0xffffffffu, high, 1);
    if (lane == 0) hprev = 0;
    // low + hprev
    uint64_t t = (uint64_t)limb[0] + (uint32_t)hprev;
    limb[0] = (uint32_t)t;
    t = (t >> 32) + limb[1] + (uint32_t)(hprev >> 32);
    limb[1] = (uint32_t)t;
    uint32_t cy = (uint32_t)(t >> 32);
#pragma unroll
    for (int w = 2; w < W; w++) {
        t = (uint64_t)limb[w] + cy;
        limb[w] = (uint32_t)t;
        cy = (uint32_t)(t >> 32);
    }
    bool ones = true;
#pragma unroll
    for (int w = 0; w < W; w++) ones = ones && limb[w] == 0xffffffffu;
    // generate/propagate scan: (g, p) o (g', p') = (g | (p & g'), p & p')
    uint32_t g = cy, p = ones ? 1u : 0u;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t go = __shfl_up_sync(0xffffffffu, g, off);
        const uint32_t po = __shfl_up_sync(0xffffffffu, p, off);
        if (lane >= off) {
            g = g | (p & go);
            p = p & po;
        }
    }
    uint32_t cin = __shfl_up_sync(0xffffffffu, g, 1);
    if (lane == 0) cin = 0;
#pragma unroll
    for (int w = 0; w < W; w++) {
        t = (uint64_t)limb[w] + cin;
        limb[w] = (uint32_t)t;
        cin = (uint32_t)(t >> 32);
    }
    const size_t node = out_index ? (size_t)out_index[k] : k;
    uint32_t *o = out + 2 * node * S + lane * W;
#pragma unroll
    for (int w = 0; w < W; w++) o[w] = limb[w];
}

// ------------------------------------------------------------ utilities

// Largest i + 1 with x[i] != 0, reduced into *top (0 if all zero).
__global__ void find_top(const uint32_t *x, size_t n, unsigned long long *top)
{
    unsigned long long best = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        if (x[i]) best = i + 1;
    for (int off = 16; off; off >>= 1) {
        const unsigned long long o = __shfl_down_sync(0xffffffffu, best, off);
        best = o > best ? o : best;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(top, best);
}

// ----------------------------------------------------------- host side

void leaf_level(Ctx &c, const uint32_t *values, size_t count, uint32_t *out, size_t nodes,
                int lpn, cudaStream_t s)
{
    const int tok = prof_begin(c, "leaf_products", s);
    leaf_products<<<(unsigned)((nodes + 255) / 256), 256, 0, s>>>(values, count, out, nodes,
                                                                    lpn);
    CAT_LAUNCH("leaf_products");
    prof_end(c, tok, s, 4.0 * (double)count + 32.0 * (double)nodes,
             4.0 * (double)count + 32.0 * (double)nodes);
}

// Products of adjacent slot-limb nodes into 2*slot-limb slots, for slots
// handled by schoolbook multiplication.  Returns false if slot is too large.
bool comba_level(Ctx &c, const uint32_t *in, size_t slot, size_t nprod, uint32_t *out,
                 cudaStream_t s, const uint32_t *out_index)
{
    if (nprod == 0) return true;
    if (slot > 256) return false;
    const int tok = prof_begin(c, slot <= 16 ? "comba_thread" : "comba_warp", s);
    const unsigned tb = 256;
    const unsigned gt = (unsigned)((nprod + tb - 1) / tb);
    const unsigned gw = (unsigned)((nprod + kWarpsPerBlock - 1) / kWarpsPerBlock);
    switch (slot) {
    case 8: comba_thread<8><<<gt, tb, 0, s>>>(in, nprod, out, out_index); break;
    case 16: comba_thread<16><<<gt, tb, 0, s>>>(in, nprod, out, out_index); break;
    case 32: comba_warp<32><<<gw, 32 * kWarpsPerBlock, 0, s>>>(in, nprod, out, out_index); break;
    case 64: comba_warp<64><<<gw, 32 * kWarpsPerBlock, 0, s>>>(in, nprod, out, out_index); break;
    case 128: comba_warp<128><<<gw, 32 * kWarpsPerBlock, 0, s>>>(in, nprod, out, out_index); break;
    case 256: comba_warp<256><<<gw, 32 * kWarpsPerBlock, 0, s>>>(in, nprod, out, out_index); break;
    default: return false;
    }
    CAT_LAUNCH("comba_level");
    prof_end(c, tok, s, 16.0 * (double)slot * (double)nprod, 16.0 * (double)slot * (double)nprod);
    return true;
}

size_t normalized_length(Ctx &c, const uint32_t *x, size_t n, cudaStream_t s)
{
    if (n == 0) return 0;
    DevBuf<unsigned long long> scratch;
    unsigned long long *top = c.dev_word;
    if (!top) {
        scratch = DevBuf<unsigned long long>(c, 1, s);
        top = scratch.get();
    }
    CAT_CUDA(cudaMemsetAsync(top, 0, sizeof(unsigned long long), s));
    const size_t threads = 256;
    size_t blocks = (n + threads - 1) / threads;
    const size_t cap = (size_t)c.num_sms * 8;
    if (blocks > cap) blocks = cap;
    find_top<<<(unsigned)blocks, threads, 0, s>>>(x, n, top);
    CAT_LAUNCH("find_top");
    unsigned long long local = 0;
    unsigned long long *h = c.host_word ? reinterpret_cast<unsigned long long *>(c.host_word) : &local;
    CAT_CUDA(cudaMemcpyAsync(h, top, sizeof(*h), cudaMemcpyDeviceToHost, s));
    CAT_CUDA(cudaStreamSynchronize(s));
    return (size_t)*h;
}

}  // namespace cat
