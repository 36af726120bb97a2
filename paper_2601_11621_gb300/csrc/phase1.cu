// phase1.cu -- Phase 1 of the method on the device (Sec. 3.1, Algorithm 1):
// the primes up to the sieve limit by a segmented Sieve of Eratosthenes, the
// exponent of each prime by Legendre's formula (Sec. 2), and the grouping of
// the primes with e > 0 by exponent into CSR form.
//
// Sieve.  Seed primes up to sqrt(limit) come from one thread block.  The odd
// numbers up to the limit are cut into segments of 2^18 (one bit each, 32 KiB
// of shared memory per block).  Primes 3..31 are struck word by word from
// precomputed bit patterns; primes 37..511 are struck by whole warps (one
// multiple per lane); larger seed primes by one thread each.  Each segment's
// bitmap and prime count go to global memory; an exclusive scan of the
// counts gives every segment its first output position.
//
// Exponents.  2n < 2^32, so every term floor(m / p^k) is a 32-bit division;
// primes above sqrt(m) take one division per factorial.  c_p = v_p(n+1) is
// the valuation of n+1 at p, which equals the exponent of p in the
// trial-division factorisation of n+1 of Algorithm 1 step 2.
//
// Grouping.  (e, p) pairs are sorted stably by e (least-significant-digit
// radix sort, pairs with e = 0 dropped in the first pass), so primes stay
// ascending within each group; group starts are then collected.
//
// Binomial kinds.  For C(n) and C(2n, n) every prime above sqrt(2n) has
// exponent 0 or 1 (one base-p carry), found with one division inside the
// sieve; the sieve keeps only the primes with exponent 1 and they are written
// in order straight into the e = 1 group.  Only the seed primes (below
// sqrt(2n) <= 65536) go through Legendre's formula and the radix grouping.
#include "cat_internal.cuh"
#include "legendre.cuh"

#include <algorithm>
#include <math.h>

namespace cat {

void exclusive_scan_u32(Ctx &c, uint32_t *data, size_t n, cudaStream_t s);

constexpr int kSegBits = 1 << 18;           // odd numbers per segment
constexpr int kSegWords = kSegBits / 32;    // 8192 words
constexpr int kSieveThreads = 512;
constexpr uint32_t kMediumPrime = 37;       // first prime struck by atomics
constexpr uint32_t kLargePrime = 512;       // thread-per-prime from here (measured best)

// ---------------------------------------------------------------- seeds

// All primes <= root (root < 2^16) in ascending order, by one block.
__global__ void __launch_bounds__(1024) seed_sieve(uint32_t root, uint32_t *seeds,
                                                   uint32_t *nseeds)
{
    __shared__ uint32_t bm[2048];  // bit x set = x composite, x < 65536
    __shared__ uint32_t pre[1024];
    for (int i = threadIdx.x; i < 2048; i += blockDim.x) bm[i] = 0;
    __syncthreads();
    if (threadIdx.x == 0) atomicOr(&bm[0], 3u);  // 0 and 1
    for (uint32_t p = 2; p * p <= root; p++)
        for (uint32_t j = p * p + threadIdx.x * p; j <= root; j += blockDim.x * p)
            atomicOr(&bm[j >> 5], 1u << (j & 31));
    __syncthreads();
    // thread t owns numbers [64 t, 64 t + 64)
    const uint32_t lo = threadIdx.x * 64;
    uint32_t w0 = ~bm[2 * threadIdx.x], w1 = ~bm[2 * threadIdx.x + 1];
    if (lo > root) { w0 = 0; w1 = 0; }
    else if (lo + 64 > root + 1) {
        const uint32_t keep = root + 1 - lo;  // 1..64 numbers kept
        if (keep < 32) { w0 &= (1u << keep) - 1; w1 = 0; }
        else if (keep < 64) { w1 &= (1u << (keep - 32)) - 1; }
    }
    const uint32_t cnt = __popc(w0) + __popc(w1);
    pre[threadIdx.x] = cnt;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        uint32_t v = threadIdx.x >= (unsigned)off ? pre[threadIdx.x - off] : 0;
        __syncthreads();
        pre[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t pos = pre[threadIdx.x] - cnt;
    for (int b = 0; b < 32; b++)
        if (w0 >> b & 1) seeds[pos++] = lo + b;
    for (int b = 0; b < 32; b++)
        if (w1 >> b & 1) seeds[pos++] = lo + 32 + b;
    if (threadIdx.x == 1023) *nseeds = pre[1023];
}

// ------------------------------------------------------------ segments

struct SieveArgs {
    const uint32_t *seeds;  // ascending primes <= sqrt(limit)
    uint32_t i_med, i_large, nseeds;  // index ranges: [0,i_med) small (3..31 are
                                       // patterned), [i_med,i_large) medium, rest large
    uint32_t imax;          // largest odd index i with 2i+1 <= limit
    uint32_t *bits;         // out: per segment, bit set = prime
    uint32_t *counts;       // out: primes per segment
    // unit_kind >= 0: keep only the primes p > root (p^2 > 2 unit_n) whose
    // exponent in the quantity of that kind is 1 (all others are 0 there);
    // counts then count the kept primes, and *total gets every odd prime.
    int unit_kind;
    uint32_t unit_n, root;
    unsigned int *total;
};

__constant__ uint32_t c_small_primes[10] = {3, 5, 7, 11, 13, 17, 19, 23, 29, 31};

__global__ void __launch_bounds__(kSieveThreads) sieve_segments(SieveArgs a)
{
    __shared__ uint32_t bm[kSegWords];
    __shared__ uint32_t red[kSieveThreads / 32], red_all[kSieveThreads / 32];
    const uint32_t seg = blockIdx.x;
    const uint32_t ibase = seg * (uint32_t)kSegBits;  // odd index of bit 0
    // words of this segment at or below the last odd index (the last segment,
    // or the only one of a small limit, is sieved only that far)
    const uint32_t used = (uint32_t)std::min<uint64_t>(kSegWords, (a.imax - ibase) / 32 + 1);
    const uint64_t used_bits = 32ull * used;
    // primes 3..31: bit b of word w is odd number x = 2(ibase + 32 w + b) + 1;
    // p | x  <=>  ibase + 32 w + b = (p - 1)/2 (mod p)
    // (the primes are compile-time constants, so i0 mod p is a multiply and a
    // shift; the word's bits b0, b0 + p, ... are one shift of the pattern
    // of p's multiples below 64)
    constexpr uint32_t kSmall[10] = {3, 5, 7, 11, 13, 17, 19, 23, 29, 31};
    for (int w = threadIdx.x; w < (int)used; w += blockDim.x) {
        const uint32_t i0 = ibase + 32u * w;
        uint32_t m = 0;
#pragma unroll
        for (int k = 0; k < 10; k++) {
            const uint32_t p = kSmall[k];
            uint64_t multiples = 0;
            for (uint32_t b = 0; b < 64; b += p) multiples |= 1ull << b;
            const uint32_t r = i0 % p;
            uint32_t b0 = (p - 1) / 2 + p - r;  // in (0, 2p)
            if (b0 >= p) b0 -= p;
            m |= (uint32_t)(multiples << b0);
        }
        bm[w] = m;
    }
    __syncthreads();
    // smallest odd number here (below the limit, so below 2^32)
    const uint32_t lo_num = 2u * ibase + 1u;
    const uint32_t ubits = (uint32_t)used_bits;
    // bit index of the first odd multiple of p at or above max(lo_num, p^2),
    // or ubits when there is none in this segment (32-bit remainder: lo_num
    // and p < 2^16 fit 32 bits; the sums in 64 bits)
    auto first_bit = [&](uint32_t p) -> uint32_t {
        const uint32_t r = lo_num % p;
        uint64_t x0 = (uint64_t)lo_num + (r ? p - r : 0u);
        if (x0 < (uint64_t)p * p) x0 = (uint64_t)p * p;
        if (!(x0 & 1)) x0 += p;
        const uint64_t f = (x0 - 1) / 2 - ibase;
        return f < ubits ? (uint32_t)f : ubits;
    };
    // medium primes: one warp per prime, one multiple per lane
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint32_t j = a.i_med + wid; j < a.i_large; j += nw) {
        const uint32_t p = a.seeds[j];
        for (uint32_t i = first_bit(p) + (uint32_t)lane * p; i < ubits; i += 32 * p)
            atomicOr(&bm[i >> 5], 1u << (i & 31));
    }
    // large primes: one thread per prime
    for (uint32_t j = a.i_large + threadIdx.x; j < a.nseeds; j += blockDim.x) {
        const uint32_t p = a.seeds[j];
        for (uint32_t i = first_bit(p); i < ubits; i += p)
            atomicOr(&bm[i >> 5], 1u << (i & 31));
    }
    __syncthreads();
    if (seg == 0 && threadIdx.x == 0) {
        uint32_t w0 = bm[0];
        w0 |= 1u;  // 1 is not prime
        for (int k = 0; k < 10; k++) {  // the pattern struck p itself
            const uint32_t i = (c_small_primes[k] - 1) / 2;
            w0 &= ~(1u << i);
        }
        bm[0] = w0;
    }
    __syncthreads();
    uint32_t cnt = 0, all = 0;
    uint32_t *out = a.bits + (size_t)seg * kSegWords;
    for (int w = threadIdx.x; w < kSegWords; w += blockDim.x) {
        const uint64_t i0 = (uint64_t)ibase + 32u * w;
        uint32_t v = w < (int)used ? ~bm[w] : 0u;
        if (i0 > a.imax) v = 0;
        else if (i0 + 31 > a.imax) v &= (uint32_t)((2ull << (a.imax - i0)) - 1);
        if (a.unit_kind >= 0) {
            all += __popc(v);
            if (2 * i0 + 1 > a.unit_n) {
                // every number of the word is above n (so above root): a prime
                // p in (n, 2n] has e_p = 1 (floor(2n/p) = 1, floor(n/p) = 0),
                // except p = n + 1 for C(n), which divides n + 1
                if (a.unit_kind == CAT_CATALAN && ((a.unit_n + 1) & 1)) {
                    const uint64_t j = (uint64_t)a.unit_n / 2;  // odd index of n + 1
                    if (j >= i0 && j < i0 + 32) v &= ~(1u << (j - i0));
                }
            } else {
                uint32_t keep = 0;
                for (uint32_t m = v; m; m &= m - 1) {
                    const int b = __ffs(m) - 1;
                    const uint32_t p = (uint32_t)(2 * (i0 + b) + 1);
                    if (p > a.root && unit_exponent(p, a.unit_n, a.unit_kind)) keep |= 1u << b;
                }
                v = keep;
            }
        }
        out[w] = v;
        cnt += __popc(v);
    }
    for (int off = 16; off; off >>= 1) {
        cnt += __shfl_down_sync(0xffffffffu, cnt, off);
        all += __shfl_down_sync(0xffffffffu, all, off);
    }
    if (lane == 0) {
        red[wid] = cnt;
        red_all[wid] = all;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0, ta = 0;
        for (int k = 0; k < nw; k++) {
            t += red[k];
            ta += red_all[k];
        }
        a.counts[seg] = t;
        if (a.unit_kind >= 0) atomicAdd(a.total, ta);
    }
}

// ----------------------------------------------------------- exponents

struct ExpandArgs {
    const uint32_t *bits;
    const uint32_t *seg_offsets;  // exclusive scan of the per-segment counts
    Ratio r;                      // the quantity (a kind of n, or a factorial ratio)
    int has_two;                  // limit >= 2: item 0 is the prime 2
    uint64_t *items;              // out: (e << 32) | p, all primes ascending
    unsigned int *max_e;
    unsigned int *negative;
};

// One block per segment: list its primes in order with their exponents.
__global__ void __launch_bounds__(kSieveThreads) expand_exponents(ExpandArgs a)
{
    __shared__ uint32_t pre[kSieveThreads];
    __shared__ uint32_t red[kSieveThreads / 32];
    constexpr int kWordsPerThread = kSegWords / kSieveThreads;  // 16
    const uint32_t seg = blockIdx.x;
    const uint32_t *bits = a.bits + (size_t)seg * kSegWords + threadIdx.x * kWordsPerThread;
    uint32_t w[kWordsPerThread];
    uint32_t cnt = 0;
#pragma unroll
    for (int k = 0; k < kWordsPerThread; k++) {
        w[k] = bits[k];
        cnt += __popc(w[k]);
    }
    pre[threadIdx.x] = cnt;
    __syncthreads();
    for (int off = 1; off < kSieveThreads; off <<= 1) {
        const uint32_t v = threadIdx.x >= (unsigned)off ? pre[threadIdx.x - off] : 0;
        __syncthreads();
        pre[threadIdx.x] += v;
        __syncthreads();
    }
    size_t pos = (size_t)a.seg_offsets[seg] + pre[threadIdx.x] - cnt + (a.has_two ? 1 : 0);
    const uint32_t ibase = seg * (uint32_t)kSegBits + threadIdx.x * kWordsPerThread * 32;
    uint32_t emax = 0, neg = 0;
#pragma unroll
    for (int k = 0; k < kWordsPerThread; k++) {
        uint32_t v = w[k];
        while (v) {
            const int b = __ffs(v) - 1;
            v &= v - 1;
            const uint32_t p = 2 * (ibase + 32 * k + b) + 1;
            const int64_t e = exponent_of(p, a.r);
            if (e < 0) neg = 1;
            const uint32_t eu = e < 0 ? 0u : (uint32_t)e;
            emax = max(emax, eu);
            a.items[pos++] = ((uint64_t)eu << 32) | p;
        }
    }
    if (seg == 0 && threadIdx.x == 0 && a.has_two) {
        const int64_t e = exponent_of(2, a.r);
        if (e < 0) neg = 1;
        const uint32_t eu = e < 0 ? 0u : (uint32_t)e;
        emax = max(emax, eu);
        a.items[0] = ((uint64_t)eu << 32) | 2u;
    }
    for (int off = 16; off; off >>= 1) {
        emax = max(emax, __shfl_down_sync(0xffffffffu, emax, off));
        neg |= __shfl_down_sync(0xffffffffu, neg, off);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = emax | (neg ? 0x80000000u : 0u);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t m = 0, ng = 0;
        for (int k = 0; k < kSieveThreads / 32; k++) {
            m = max(m, red[k] & 0x7fffffffu);
            ng |= red[k] >> 31;
        }
        atomicMax(a.max_e, m);
        if (ng) atomicOr(a.negative, 1u);
    }
}

// ------------------------------------------------------- radix grouping

constexpr int kRsThreads = 256;
constexpr int kRsItems = 16;                     // per thread
constexpr int kRsTile = kRsThreads * kRsItems;   // 4096
constexpr int kRsWarps = kRsThreads / 32;

// item (warp w, iteration it, lane) of a tile is element
// tile*4096 + w*512 + it*32 + lane: warp-major, so warp order = element order.
__device__ __forceinline__ size_t rs_index(size_t tile, int w, int it, int lane)
{
    return tile * kRsTile + (size_t)w * (32 * kRsItems) + it * 32 + lane;
}

struct RsArgs {
    const uint64_t *in;
    uint64_t *out;
    size_t count;
    int shift, bits;    // digit = (e >> shift) & (2^bits - 1), e = item >> 32
    int drop_zero;      // first pass: items with e == 0 are dropped
    uint32_t *counts;   // [digit][tile]
    size_t tiles;
};

__global__ void __launch_bounds__(kRsThreads) rs_histogram(RsArgs a)
{
    __shared__ uint32_t h[256];
    const int nb = 1 << a.bits;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const size_t tile = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int it = 0; it < kRsItems; it++) {
        const size_t i = rs_index(tile, w, it, lane);
        if (i < a.count) {
            const uint32_t e = (uint32_t)(a.in[i] >> 32);
            if (!(a.drop_zero && e == 0)) atomicAdd(&h[(e >> a.shift) & (nb - 1)], 1u);
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nb; d += blockDim.x) a.counts[(size_t)d * a.tiles + tile] = h[d];
}

__global__ void __launch_bounds__(kRsThreads) rs_scatter(RsArgs a)
{
    __shared__ uint32_t wh[kRsWarps][256];
    const int nb = 1 << a.bits;
    for (int i = threadIdx.x; i < kRsWarps * 256; i += blockDim.x) (&wh[0][0])[i] = 0;
    __syncthreads();
    const size_t tile = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t item[kRsItems];
    uint32_t rank[kRsItems];
    int digit[kRsItems];
    for (int it = 0; it < kRsItems; it++) {
        const size_t i = rs_index(tile, w, it, lane);
        int d = -1;
        uint64_t v = 0;
        if (i < a.count) {
            v = a.in[i];
            const uint32_t e = (uint32_t)(v >> 32);
            if (!(a.drop_zero && e == 0)) d = (int)((e >> a.shift) & (nb - 1));
        }
        item[it] = v;
        digit[it] = d;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (d >= 0 && lane == leader) {
            base = wh[w][d];
            wh[w][d] = base + __popc(peers);
        }
        base = __shfl_sync(0xffffffffu, base, leader);
        rank[it] = base + __popc(peers & ((1u << lane) - 1));
        __syncwarp();
    }
    __syncthreads();
    // exclusive scan over warps per digit, plus the global digit offset
    for (int d = threadIdx.x; d < nb; d += blockDim.x) {
        uint32_t run = a.counts[(size_t)d * a.tiles + tile];
        for (int k = 0; k < kRsWarps; k++) {
            const uint32_t c = wh[k][d];
            wh[k][d] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int it = 0; it < kRsItems; it++)
        if (digit[it] >= 0) a.out[wh[w][digit[it]] + rank[it]] = item[it];
}

// group starts: positions i with e_i != e_{i-1}, appended as (e, i)
__global__ void group_starts(const uint64_t *items, size_t count, uint64_t *starts,
                             unsigned int *nstarts, uint32_t *primes)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint64_t v = items[i];
    primes[i] = (uint32_t)v;
    const uint32_t e = (uint32_t)(v >> 32);
    if (i == 0 || (uint32_t)(items[i - 1] >> 32) != e) {
        const unsigned k = atomicAdd(nstarts, 1u);
        starts[2 * k] = e;
        starts[2 * k + 1] = i;
    }
}

// One block per segment: the primes of its bitmap in ascending order, written
// to primes[first + seg_offsets[seg] + ...]; with_two also puts 2 at primes[0].
// Each warp owns 1024 consecutive words and takes them 32 at a time (one word
// a lane): a warp scan of the bit counts places each lane's primes in a
// per-warp shared stage, which the warp then copies out contiguously.
constexpr int kExpandThreads = 256;
constexpr int kExpandWarps = kExpandThreads / 32;
constexpr int kWordsPerWarp = kSegWords / kExpandWarps;  // 1024
constexpr int kExpandIters = kWordsPerWarp / 32;          // 32

__global__ void __launch_bounds__(kExpandThreads) expand_primes(const uint32_t *bits,
                                                               const uint32_t *seg_offsets,
                                                               uint32_t *primes, uint32_t first,
                                                               int with_two)
{
    __shared__ uint32_t stage[kExpandWarps][32 * 32];
    __shared__ uint32_t wsum[kExpandWarps];
    const uint32_t seg = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t word0 = (uint32_t)wid * kWordsPerWarp;
    const uint32_t *b = bits + (size_t)seg * kSegWords + word0;
    uint32_t w[kExpandIters];
    uint32_t cnt = 0;
#pragma unroll
    for (int it = 0; it < kExpandIters; it++) {
        w[it] = b[it * 32 + lane];
        cnt += __popc(w[it]);
    }
    for (int off = 16; off; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
    if (lane == 0) wsum[wid] = cnt;
    __syncthreads();
    size_t pos = (size_t)seg_offsets[seg] + first;
    for (int k = 0; k < wid; k++) pos += wsum[k];
    uint32_t *st = stage[wid];
#pragma unroll
    for (int it = 0; it < kExpandIters; it++) {
        const uint32_t c = __popc(w[it]);
        uint32_t incl = c;
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += v;
        }
        const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
        uint32_t at = incl - c;
        const uint32_t ibase = seg * (uint32_t)kSegBits + 32u * (word0 + it * 32 + lane);
        for (uint32_t m = w[it]; m; m &= m - 1) st[at++] = 2 * (ibase + __ffs(m) - 1) + 1;
        __syncwarp();
        for (uint32_t k = lane; k < tot; k += 32) primes[pos + k] = st[k];
        pos += tot;
        __syncwarp();
    }
    if (with_two && seg == 0 && threadIdx.x == 0) primes[0] = 2;
}

// The exponents of the seed primes (all primes <= sqrt(2n)), one thread each.
__global__ void seed_items(const uint32_t *seeds, uint32_t ns, Ratio r, uint64_t *items,
                           unsigned int *max_e, unsigned int *negative)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns) return;
    const uint32_t p = seeds[i];
    const int64_t e = exponent_of(p, r);
    if (e < 0) atomicOr(negative, 1u);
    const uint32_t eu = e < 0 ? 0u : (uint32_t)e;
    atomicMax(max_e, eu);
    items[i] = ((uint64_t)eu << 32) | p;
}

// ------------------------------------------------------------ host side

static uint64_t isqrt64(uint64_t x)
{
    uint64_t r = (uint64_t)sqrtl((long double)x);
    while (r > 0 && r * r > x) r--;
    while ((r + 1) * (r + 1) <= x) r++;
    return r;
}

// The segmented sieve up to `limit` (>= 2): per-segment bitmaps of the odd
// primes and the exclusive scan of their counts.  sieved = pi(limit).
// With unit_kind >= 0 (a binomial kind of n, limit = 2n) the bitmaps keep only
// the primes above sqrt(2n) with exponent 1, the offsets scan their counts
// (kept in total), and the seeds are exactly the primes up to sqrt(2n).
struct SieveOut {
    DevBuf<uint32_t> bits, offsets, seeds;
    uint32_t nsegs = 0, nseeds = 0;
    uint64_t sieved = 0, kept = 0;
};

static SieveOut run_sieve(Ctx &c, uint64_t limit, cudaStream_t s, int unit_kind = -1,
                          uint32_t unit_n = 0)
{
    SieveOut o;
    const uint64_t root = isqrt64(limit);
    o.seeds = DevBuf<uint32_t>(c, 8192, s);
    DevBuf<uint32_t> &seeds = o.seeds;
    DevBuf<uint32_t> nseeds(c, 2, s);
    CAT_CUDA(cudaMemsetAsync(nseeds.get(), 0, 8, s));
    seed_sieve<<<1, 1024, 0, s>>>((uint32_t)root, seeds.get(), nseeds.get());
    CAT_LAUNCH("seed_sieve");
    uint32_t ns = 0;
    CAT_CUDA(cudaMemcpyAsync(&ns, nseeds.get(), 4, cudaMemcpyDeviceToHost, s));
    CAT_CUDA(cudaStreamSynchronize(s));
    o.nseeds = ns;
    std::vector<uint32_t> hs(ns);
    if (ns)
        CAT_CUDA(cudaMemcpyAsync(hs.data(), seeds.get(), 4 * ns, cudaMemcpyDeviceToHost, s));
    CAT_CUDA(cudaStreamSynchronize(s));
    // odd seeds only for the segment sieve
    const uint32_t *odd = seeds.get() + (ns > 0 && hs[0] == 2 ? 1 : 0);
    const uint32_t nodd = ns > 0 ? ns - 1 : 0;
    uint32_t i_med = 0, i_large = 0;
    for (uint32_t k = 0; k < nodd; k++) {
        const uint32_t p = hs[k + 1];
        if (p < kMediumPrime) i_med = k + 1;
        if (p < kLargePrime) i_large = k + 1;
    }
    // segments over odd indices 0..imax (odd number 2i+1 <= limit)
    const uint32_t imax = (uint32_t)((limit - 1) / 2);
    o.nsegs = imax / kSegBits + 1;
    o.bits = DevBuf<uint32_t>(c, (size_t)o.nsegs * kSegWords, s);
    o.offsets = DevBuf<uint32_t>(c, o.nsegs, s);
    SieveArgs sa{odd, i_med, i_large, nodd, imax, o.bits.get(), o.offsets.get(),
                 unit_kind, unit_n, (uint32_t)root, nseeds.get() + 1};
    const int tok = prof_begin(c, "sieve_segments", s);
    sieve_segments<<<o.nsegs, kSieveThreads, 0, s>>>(sa);
    CAT_LAUNCH("sieve_segments");
    prof_end(c, tok, s, 4.0 * (double)o.nsegs * kSegWords);
    uint32_t last_count = 0;
    CAT_CUDA(cudaMemcpyAsync(&last_count, o.offsets.get() + o.nsegs - 1, 4,
                             cudaMemcpyDeviceToHost, s));
    exclusive_scan_u32(c, o.offsets.get(), o.nsegs, s);
    uint32_t last_off = 0, total = 0;
    CAT_CUDA(cudaMemcpyAsync(&last_off, o.offsets.get() + o.nsegs - 1, 4,
                             cudaMemcpyDeviceToHost, s));
    CAT_CUDA(cudaMemcpyAsync(&total, nseeds.get() + 1, 4, cudaMemcpyDeviceToHost, s));
    CAT_CUDA(cudaStreamSynchronize(s));
    o.kept = (uint64_t)last_off + last_count;
    o.sieved = (unit_kind >= 0 ? (uint64_t)total : o.kept) + 1;  // plus the prime 2
    return o;
}

void factor(Ctx &c, uint64_t n, int kind, cat_factorization *out, cudaStream_t s)
{
    if (n >= (1ull << 31)) fail(CAT_EINVAL, "n must be below 2^31");
    if (kind < CAT_CATALAN || kind > CAT_FACTORIAL) fail(CAT_EINVAL, "unknown kind");
    Ratio r{};
    r.kind = kind;
    r.n = (uint32_t)n;
    factor_ratio(c, r, out, s);
}

// (e, p) items with e = 0 dropped, grouped by e: primes ascending within each
// group, groups by ascending e, offs[k] = start of group k (offs has one more
// entry than exps, ending in count).
struct Grouped {
    DevBuf<uint32_t> primes;
    std::vector<uint64_t> exps, offs{0};
    uint64_t count = 0;
};

static Grouped group_items(Ctx &c, DevBuf<uint64_t> &items, size_t count, uint32_t max_e,
                           cudaStream_t s)
{
    Grouped g;
    // stable radix sort by e, dropping e = 0
    int ebits = 0;
    while (ebits < 32 && (max_e >> ebits)) ebits++;
    DevBuf<uint64_t> alt(c, std::max<size_t>(count, 1), s);
    uint64_t *src = items.get(), *dst = alt.get();
    int tok;
    for (int shift = 0, pass = 0; pass == 0 || shift < ebits; pass++) {
        const int bitsd = std::max(1, std::min(8, ebits - shift));
        const size_t tiles = (count + kRsTile - 1) / kRsTile;
        if (tiles == 0) break;
        const size_t nbins = (size_t)1 << bitsd;
        DevBuf<uint32_t> cnt(c, nbins * tiles, s);
        RsArgs ra{src, dst, count, shift, bitsd, pass == 0 ? 1 : 0, cnt.get(), tiles};
        tok = prof_begin(c, "rs_histogram", s);
        rs_histogram<<<(unsigned)tiles, kRsThreads, 0, s>>>(ra);
        CAT_LAUNCH("rs_histogram");
        prof_end(c, tok, s, 8.0 * (double)count);
        uint32_t lastc = 0, lasto = 0;
        CAT_CUDA(cudaMemcpyAsync(&lastc, cnt.get() + nbins * tiles - 1, 4,
                                 cudaMemcpyDeviceToHost, s));
        exclusive_scan_u32(c, cnt.get(), nbins * tiles, s);
        CAT_CUDA(cudaMemcpyAsync(&lasto, cnt.get() + nbins * tiles - 1, 4,
                                 cudaMemcpyDeviceToHost, s));
        tok = prof_begin(c, "rs_scatter", s);
        rs_scatter<<<(unsigned)tiles, kRsThreads, 0, s>>>(ra);
        CAT_LAUNCH("rs_scatter");
        prof_end(c, tok, s, 16.0 * (double)count);
        CAT_CUDA(cudaStreamSynchronize(s));
        count = (size_t)lasto + lastc;
        std::swap(src, dst);
        shift += bitsd;
        if (ebits == 0) break;
    }
    g.count = count;
    if (count == 0) return g;
    g.primes = DevBuf<uint32_t>(c, count, s);
    DevBuf<uint64_t> starts(c, 2 * count, s);
    DevBuf<unsigned int> nst(c, 1, s);
    CAT_CUDA(cudaMemsetAsync(nst.get(), 0, 4, s));
    group_starts<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(src, count, starts.get(),
                                                                  nst.get(), g.primes.get());
    CAT_LAUNCH("group_starts");
    unsigned int ng = 0;
    CAT_CUDA(cudaMemcpyAsync(&ng, nst.get(), 4, cudaMemcpyDeviceToHost, s));
    CAT_CUDA(cudaStreamSynchronize(s));
    std::vector<uint64_t> hst(2 * (size_t)ng);
    CAT_CUDA(cudaMemcpyAsync(hst.data(), starts.get(), 16 * (size_t)ng, cudaMemcpyDeviceToHost,
                             s));
    CAT_CUDA(cudaStreamSynchronize(s));
    std::vector<std::pair<uint64_t, uint64_t>> gs(ng);
    for (size_t k = 0; k < ng; k++) gs[k] = {hst[2 * k], hst[2 * k + 1]};
    std::sort(gs.begin(), gs.end());
    g.offs.clear();
    for (auto &x : gs) {
        g.exps.push_back(x.first);
        g.offs.push_back(x.second);
    }
    g.offs.push_back(count);
    return g;
}

// Catalan or central binomial kinds with n >= 2.  Every prime above sqrt(2n)
// has exponent 0 or 1; the sieve keeps those with 1 and they are written in
// order straight into the e = 1 group, after the seed primes with e = 1.  The
// seed primes (<= sqrt(2n), fewer than 6600) take Legendre's formula and the
// radix grouping; their groups with e >= 2 follow.
static void factor_unit(Ctx &c, const Ratio &r, uint64_t limit, DevBuf<uint32_t> &primes_out,
                        std::vector<uint64_t> &h_exps, std::vector<uint64_t> &h_offs,
                        uint64_t &sieved, uint64_t &npos, cudaStream_t s)
{
    SieveOut sv = run_sieve(c, limit, s, r.kind, r.n);
    sieved = sv.sieved;
    const uint32_t ns = sv.nseeds;
    DevBuf<uint64_t> items(c, std::max<uint32_t>(ns, 1), s);
    DevBuf<unsigned int> flags(c, 2, s);
    CAT_CUDA(cudaMemsetAsync(flags.get(), 0, 8, s));
    if (ns) {
        seed_items<<<(ns + 255) / 256, 256, 0, s>>>(sv.seeds.get(), ns, r, items.get(),
                                                    flags.get(), flags.get() + 1);
        CAT_LAUNCH("seed_items");
    }
    unsigned int hf[2];
    CAT_CUDA(cudaMemcpyAsync(hf, flags.get(), 8, cudaMemcpyDeviceToHost, s));
    CAT_CUDA(cudaStreamSynchronize(s));
    if (hf[1]) fail(CAT_ENOTINTEGRAL, "a prime exponent is negative");
    Grouped g = group_items(c, items, ns, hf[0], s);
    const uint64_t nl = sv.kept;
    const uint64_t n1 = (!g.exps.empty() && g.exps[0] == 1) ? g.offs[1] : 0;
    npos = g.count + nl;
    h_exps.clear();
    h_offs.assign(1, 0);
    if (npos == 0) return;
    primes_out = DevBuf<uint32_t>(c, npos, s);
    uint32_t *d = primes_out.get();
    if (n1)
        CAT_CUDA(cudaMemcpyAsync(d, g.primes.get(), 4 * n1, cudaMemcpyDeviceToDevice, s));
    if (nl) {
        const int tok = prof_begin(c, "expand_primes", s);
        expand_primes<<<sv.nsegs, kExpandThreads, 0, s>>>(sv.bits.get(), sv.offsets.get(),
                                                           d + n1, 0, 0);
        CAT_LAUNCH("expand_primes");
        prof_end(c, tok, s, 4.0 * (double)sv.nsegs * kSegWords + 4.0 * (double)nl);
    }
    if (g.count > n1)
        CAT_CUDA(cudaMemcpyAsync(d + n1 + nl, g.primes.get() + n1, 4 * (g.count - n1),
                                 cudaMemcpyDeviceToDevice, s));
    h_offs.clear();
    if (n1 + nl) {
        h_exps.push_back(1);
        h_offs.push_back(0);
    }
    for (size_t k = n1 ? 1 : 0; k < g.exps.size(); k++) {
        h_exps.push_back(g.exps[k]);
        h_offs.push_back(g.offs[k] + nl);
    }
    h_offs.push_back(npos);
    CAT_CUDA(cudaStreamSynchronize(s));  // the copies read g.primes before it is freed
}

// Phase 1 for any Ratio: primes up to the largest factorial argument (2n for
// the binomial kinds, n for n!, the largest term of a ratio).
void factor_ratio(Ctx &c, const Ratio &r, cat_factorization *out, cudaStream_t s)
{
    NvtxRange range("phase1: sieve, exponents, grouping");
    *out = cat_factorization{};
    const int kind = r.kind;
    const uint64_t n = r.n;
    uint64_t limit = kind == CAT_FACTORIAL ? n : 2 * n;
    if (kind == kRatioKind) {
        limit = 0;
        for (int i = 0; i < r.ka; i++) limit = std::max<uint64_t>(limit, r.a[i]);
        for (int j = 0; j < r.kb; j++) limit = std::max<uint64_t>(limit, r.b[j]);
    }
    std::vector<uint64_t> h_exps, h_offs{0};
    DevBuf<uint32_t> primes_out;
    uint64_t sieved = 0, npos = 0;
    if ((kind == CAT_CATALAN || kind == CAT_CENTRAL_BINOMIAL) && n >= 2) {
        factor_unit(c, r, limit, primes_out, h_exps, h_offs, sieved, npos, s);
    } else if (limit >= 2) {
        SieveOut sv = run_sieve(c, limit, s);
        const uint32_t nsegs = sv.nsegs;
        sieved = sv.sieved;
        // exponents
        DevBuf<uint64_t> items(c, sieved, s);
        DevBuf<unsigned int> flags(c, 2, s);
        CAT_CUDA(cudaMemsetAsync(flags.get(), 0, 8, s));
        ExpandArgs ea{sv.bits.get(), sv.offsets.get(), r, 1, items.get(), flags.get(),
                      flags.get() + 1};
        const int tok = prof_begin(c, "expand_exponents", s);
        expand_exponents<<<nsegs, kSieveThreads, 0, s>>>(ea);
        CAT_LAUNCH("expand_exponents");
        prof_end(c, tok, s, 4.0 * (double)nsegs * kSegWords + 8.0 * (double)sieved);
        sv.bits.reset();
        sv.offsets.reset();
        sv.seeds.reset();
        unsigned int hf[2];
        CAT_CUDA(cudaMemcpyAsync(hf, flags.get(), 8, cudaMemcpyDeviceToHost, s));
        CAT_CUDA(cudaStreamSynchronize(s));
        if (hf[1]) fail(CAT_ENOTINTEGRAL, "a prime exponent is negative");
        Grouped g = group_items(c, items, sieved, hf[0], s);
        npos = g.count;
        primes_out = std::move(g.primes);
        h_exps = std::move(g.exps);
        h_offs = std::move(g.offs);
    }
    const size_t ng = h_exps.size();
    DevBuf<uint64_t> d_exps(c, ng + 1, s), d_offs(c, ng + 1, s);
    if (!primes_out.get()) primes_out = DevBuf<uint32_t>(c, 1, s);
    out->host_exps = new uint64_t[ng + 1];
    out->host_offsets = new uint64_t[ng + 1];
    for (size_t k = 0; k < ng; k++) out->host_exps[k] = h_exps[k];
    out->host_exps[ng] = 0;
    for (size_t k = 0; k <= ng; k++) out->host_offsets[k] = h_offs[k];
    CAT_CUDA(cudaMemcpyAsync(d_exps.get(), out->host_exps, 8 * (ng + 1),
                             cudaMemcpyHostToDevice, s));
    CAT_CUDA(cudaMemcpyAsync(d_offs.get(), out->host_offsets, 8 * (ng + 1),
                             cudaMemcpyHostToDevice, s));
    CAT_CUDA(cudaStreamSynchronize(s));
    out->num_groups = ng;
    out->num_primes = npos;
    out->primes_sieved = sieved;
    out->exps = d_exps.release();
    out->offsets = d_offs.release();
    out->primes = primes_out.release();
}

DevBuf<uint32_t> sieve_primes(Ctx &c, uint64_t limit, uint64_t *count, cudaStream_t s)
{
    *count = 0;
    if (limit < 2) return DevBuf<uint32_t>(c, 1, s);
    SieveOut sv = run_sieve(c, limit, s);
    DevBuf<uint32_t> primes(c, sv.sieved, s);
    const int tok = prof_begin(c, "expand_primes", s);
    expand_primes<<<sv.nsegs, kExpandThreads, 0, s>>>(sv.bits.get(), sv.offsets.get(),
                                                       primes.get(), 1, 1);
    CAT_LAUNCH("expand_primes");
    prof_end(c, tok, s, 4.0 * (double)sv.nsegs * kSegWords + 4.0 * (double)sv.sieved);
    *count = sv.sieved;
    return primes;
}

void factor_free(Ctx &c, cat_factorization *f)
{
    if (!f) return;
    dev_free(c, f->exps, 8 * (f->num_groups + 1), nullptr);
    dev_free(c, f->offsets, 8 * (f->num_groups + 1), nullptr);
    dev_free(c, f->primes, 4 * (f->num_primes ? f->num_primes : 1), nullptr);
    delete[] f->host_exps;
    delete[] f->host_offsets;
    *f = cat_factorization{};
}

}  // namespace cat
