// decimal.cu -- binary to decimal conversion: the optional decimal text
// output of the reconstructed number (Sec. 3.2; Table 1 gives the digit count
// of C(2,050,572,903), 1,234,567,890).
//
// Method (no division of long numbers).  The little-endian 2^32-limbs are cut
// into leaves of 59 limbs, each converted to base 10^9 ("chunks" of nine
// digits) by Horner's rule in one thread.  Then, level by level, adjacent
// nodes (lo, hi) of w limbs each are joined into lo + hi 2^(32 w), computed in
// base 10^9: one batched product of all hi nodes with the common power
// P_j = 2^(32 w) written in base 10^9 (transformed once), whose remaindering
// splits every exact coefficient into base-10^9 digits, adds the lo node and
// carries in base 10^9.  P_{j+1} = P_j^2 by the same product.  An odd last
// node of a level (no hi) moves up unchanged.  The top node is the whole
// number in base 10^9; a last pass prints nine digits per chunk (the top
// chunk without leading zeros).
//
// Leaf size.  A w-limb value has at most 1.0704 w chunks, so 59-limb leaves
// fill 64 chunks (2^1888 < 10^569) and a level-j node at most 64 2^j: the
// product hi P_j then has at most 2^(7 + j) coefficients, exactly one
// transform size.  (64-limb leaves would need 69 chunks, and every product a
// transform twice its length.)
//
// Exactness: a level's product coefficients are below min(len) (10^9)^2 <
// 2^26 10^18 < 10^26, inside the three-prime range, and each node sum lo +
// hi 2^(32 w) < 2^(64 w) fits the next level's chunk count, so no carry
// leaves a node.  The one product too long for a single transform (the top
// level of very long numbers) goes by pieces (mul_acc).
#include "cat_internal.cuh"

#include <math.h>

#include <algorithm>
#include <vector>

namespace cat {

constexpr int kDecLeafLimbs = 59;
constexpr int kDecLeafChunks = 64;  // 2^1888 < 10^569: 64 chunks of nine digits

// chunks of nine digits that hold any value below 2^bits (a little spare)
static size_t chunks_for_bits(double bits)
{
    return (size_t)ceil((bits * log10(2.0) + 2.0) / 9.0);
}

// Leaf i: limbs [59 i, 59 i + 59) of x (zero past n) in base 10^9, by
// acc <- acc 2^32 + limb from the top limb down.  After m limbs acc < 2^(32 m)
// has at most ceil(32 m log10(2) / 9) + 1 chunks, so step m touches only those.
__global__ void __launch_bounds__(128) dec_leaves(const uint32_t *x, size_t n, size_t leaves,
                                                  uint32_t *out)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= leaves) return;
    uint32_t acc[kDecLeafChunks];
#pragma unroll
    for (int c = 0; c < kDecLeafChunks; c++) acc[c] = 0;
#pragma unroll
    for (int m = 1; m <= kDecLeafLimbs; m++) {
        const size_t idx = i * kDecLeafLimbs + (kDecLeafLimbs - m);
        uint64_t carry = idx < n ? x[idx] : 0u;
        // 32 m log10(2) / 9 < 1.0703 m: chunks in use after this step
        constexpr int kSpare = 2;
        const int used = (int)((m * 10703) / 10000) + kSpare;
#pragma unroll
        for (int c = 0; c < kDecLeafChunks; c++) {
            if (c < used) {
                const uint64_t v = ((uint64_t)acc[c] << 32) + carry;  // < 10^9 2^32 + 2^33
                carry = v / kDecBase;
                acc[c] = (uint32_t)(v - carry * kDecBase);
            }
        }
    }
    uint32_t *o = out + i * kDecLeafChunks;
#pragma unroll
    for (int c = 0; c < kDecLeafChunks; c++) o[c] = acc[c];
}

// Digits of the chunks ch[0 .. top] (top the highest non-zero one), most
// significant first: chunk top gives its `lead` digits, every lower chunk
// exactly nine.
__global__ void dec_print(const uint32_t *ch, size_t top, int lead, char *out)
{
    const size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c > top) return;
    uint32_t v = ch[c];
    const int nd = c == top ? lead : 9;
    char *o = out + (c == top ? 0 : lead + 9 * (top - 1 - c));
    for (int d = nd - 1; d >= 0; d--) {
        o[d] = (char)('0' + v % 10u);
        v /= 10u;
    }
}

size_t decimal_bound(size_t n)
{
    // floor(32 n log10 2) + 1 digits at most; a little spare against rounding
    return (size_t)floor((double)n * 32.0 * log10(2.0)) + 2;
}

// P_0 = 2^(32 * 59) in base 10^9, on the host.
static std::vector<uint32_t> leaf_power()
{
    std::vector<uint32_t> p(1, 1u);
    for (int b = 0; b < 32 * kDecLeafLimbs; b++) {
        uint32_t carry = 0;
        for (uint32_t &d : p) {
            const uint32_t v = 2 * d + carry;
            carry = v >= kDecBase ? 1u : 0u;
            d = v - carry * kDecBase;
        }
        if (carry) p.push_back(carry);
    }
    return p;
}

int to_decimal_dev(Ctx &c, const uint32_t *x, size_t n, char *out, size_t cap, size_t *needed,
                   cudaStream_t s)
{
    NvtxRange range("to_decimal");
    n = n ? normalized_length(c, x, n, s) : 0;
    if (n == 0) {
        *needed = 1;
        if (cap < 1) return CAT_ERANGE;
        const char zero = '0';
        CAT_CUDA(cudaMemcpyAsync(out, &zero, 1, cudaMemcpyHostToDevice, s));
        CAT_CUDA(cudaStreamSynchronize(s));
        return CAT_OK;
    }
    const size_t leaves = (n + kDecLeafLimbs - 1) / kDecLeafLimbs;
    int h = 0;
    while (((size_t)1 << h) < leaves) h++;

    // level 0: leaves of 59 limbs in 64 chunks
    size_t S = kDecLeafChunks, nodes = leaves;
    DevBuf<uint32_t> cur(c, nodes * S, s);
    {
        const int tok = prof_begin(c, "dec_leaves", s);
        dec_leaves<<<(unsigned)((nodes + 127) / 128), 128, 0, s>>>(x, n, nodes, cur.get());
        CAT_LAUNCH("dec_leaves");
        prof_end(c, tok, s, 4.0 * (double)n + 4.0 * (double)(nodes * S));
    }
    const std::vector<uint32_t> p0 = leaf_power();
    size_t plen = p0.size();
    DevBuf<uint32_t> P(c, plen, s);
    CAT_CUDA(cudaMemcpyAsync(P.get(), p0.data(), 4 * plen, cudaMemcpyHostToDevice, s));

    for (int j = 0; j < h; j++) {
        const size_t nprod = nodes / 2, odd = nodes & 1, nn = nprod + odd;
        // node width 59 * 2^j limbs -> the joined node holds 2^(32 * 59 * 2^(j+1))
        const size_t S1 = chunks_for_bits(32.0 * kDecLeafLimbs * (double)((size_t)2 << j));
        DevBuf<uint32_t> nxt(c, nn * S1, s);
        if (nprod && S + plen <= ((size_t)1 << c.max_log)) {
            mul_broadcast(c, cur.get() + S, 2 * S, S, nprod, P.get(), plen,
                          Sink{nxt.get(), S1, S1, true, cur.get(), 2 * S, S}, s);
        } else {
            for (size_t k = 0; k < nprod; k++) {
                uint32_t *acc = nxt.get() + k * S1;
                const uint32_t *hi = cur.get() + (2 * k + 1) * S;
                CAT_CUDA(cudaMemcpyAsync(acc, cur.get() + 2 * k * S, 4 * S,
                                         cudaMemcpyDeviceToDevice, s));
                CAT_CUDA(cudaMemsetAsync(acc + S, 0, 4 * (S1 - S), s));
                // the top node's hi part may be much shorter than its slot
                mul_acc(c, hi, normalized_length(c, hi, S, s), P.get(), plen, acc, S1, true, s);
            }
        }
        if (odd) {  // no hi: the last node moves up
            uint32_t *dst = nxt.get() + nprod * S1;
            CAT_CUDA(cudaMemcpyAsync(dst, cur.get() + 2 * nprod * S, 4 * S,
                                     cudaMemcpyDeviceToDevice, s));
            CAT_CUDA(cudaMemsetAsync(dst + S, 0, 4 * (S1 - S), s));
        }
        cur = std::move(nxt);
        S = S1;
        nodes = nn;
        if (j + 1 < h) {  // P_{j+1} = P_j^2
            DevBuf<uint32_t> P2(c, 2 * plen, s);
            if (2 * plen <= ((size_t)1 << c.max_log)) {
                mul_broadcast(c, P.get(), 0, plen, 1, P.get(), plen,
                              Sink{P2.get(), 0, 2 * plen, true, nullptr, 0, 0}, s);
            } else {
                CAT_CUDA(cudaMemsetAsync(P2.get(), 0, 8 * plen, s));
                mul_acc(c, P.get(), plen, P.get(), plen, P2.get(), 2 * plen, true, s);
            }
            plen = normalized_length(c, P2.get(), 2 * plen, s);
            P = std::move(P2);
        }
    }
    // cur: the number in S chunks of base 10^9
    const size_t nch = normalized_length(c, cur.get(), S, s);
    const size_t top = nch - 1;
    uint32_t lead_chunk = 0;
    CAT_CUDA(cudaMemcpyAsync(&lead_chunk, cur.get() + top, 4, cudaMemcpyDeviceToHost, s));
    CAT_CUDA(cudaStreamSynchronize(s));
    int lead = 1;
    for (uint32_t v = lead_chunk; v >= 10; v /= 10) lead++;
    const size_t total = (size_t)lead + 9 * top;
    *needed = total;
    if (cap < total) return CAT_ERANGE;
    const int tok = prof_begin(c, "dec_print", s);
    dec_print<<<(unsigned)((nch + 255) / 256), 256, 0, s>>>(cur.get(), top, lead, out);
    CAT_LAUNCH("dec_print");
    prof_end(c, tok, s, 4.0 * (double)nch + (double)total);
    CAT_CUDA(cudaStreamSynchronize(s));
    return CAT_OK;
}

}  // namespace cat
