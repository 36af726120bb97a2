// cat_internal.cuh -- shared internals of libcatalan (context, errors, device
// memory, 32-bit Montgomery arithmetic for the NTT primes).
//
// Integer representation: little-endian uint32 limbs.  The NTT works modulo
// three primes q = k * 2^m + 1 below 2^32 whose multiplicative groups contain
// 2^27-th roots of unity, so one transform covers up to 2^27 points; the
// product of the three primes (~2^93.6) exceeds the largest convolution
// coefficient 2^26 * (2^32 - 1)^2 < 2^90 of two operands whose lengths add up
// to at most 2^27 limbs, so the Chinese remaindering is exact.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <string>
#include <vector>

#include "catalan.h"

namespace cat {

// ----------------------------------------------------------------- errors

struct Error {
    int code;
    std::string msg;
};

[[noreturn]] void fail(int code, const std::string &msg);
void check_cuda(cudaError_t e, const char *what);
#define CAT_CUDA(call) ::cat::check_cuda((call), #call)
#define CAT_LAUNCH(what) ::cat::check_cuda(cudaGetLastError(), what)

// ------------------------------------------------------------- constants

constexpr int kNumPrimes = 3;
constexpr int kLogMaxNtt = 27;  // largest transform: 2^27 points
// Two sets of three NTT primes.  Set 0: q < 2^31 with 2^26 | q - 1, for
// transforms up to 2^26 points (product ~2^90.5 > 2^25 (2^32 - 1)^2, the
// largest coefficient when na + nb <= 2^26); q < 2^31 makes a modular add,
// subtract or Montgomery correction three integer instructions (a min of
// two candidates).  Set 1: q < 2^32 with 2^27 | q - 1, for 2^27 points
// (product ~2^93.6 > 2^26 (2^32 - 1)^2).  Primes ascend within a set.
constexpr int kNumSets = 2;
constexpr int kLogMaxSmallSet = 26;
// Twiddle tables per (prime, direction), w the primitive 2^27-th root of
// unity (or its inverse), entries (Montgomery form, that times q^-1 mod 2^32):
//   [0, 2^13)               w^(j 2^14): the roots of order <= 2^13 used by
//                           the butterfly stages of a sub-transform;
//   three tables of 512     w^j, w^(512 j), w^(2^18 j): any w^E, E < 2^27,
//                           as a product of three small-table entries.
constexpr int kTwStage = 1 << 13;
constexpr int kTwSmall = 512;
constexpr int kTwPerDir = kTwStage + 3 * kTwSmall;  // uint2 entries per (prime, direction)

__host__ __device__ constexpr uint32_t ntt_prime(int set, int i)
{
    return set == 0 ? (i == 0 ? 469762049u : (i == 1 ? 1811939329u : 2013265921u))
                    : (i == 0 ? 2013265921u : (i == 1 ? 2281701377u : 3221225473u));
}

// log2 of the order of the root of unity the twiddle tables of a set use
__host__ __device__ constexpr int set_log_root(int set) { return set == 0 ? kLogMaxSmallSet : kLogMaxNtt; }

// the prime set a transform of 2^n points uses
__host__ __device__ constexpr int set_for(int n) { return n <= kLogMaxSmallSet ? 0 : 1; }

// q^-1 mod 2^32 by Newton's iteration x <- x (2 - q x)
__host__ __device__ constexpr uint32_t inv32(uint32_t q)
{
    uint32_t x = q;
    for (int i = 0; i < 5; i++) x *= 2u - q * x;
    return x;
}

__host__ __device__ constexpr uint32_t mulmod_u64(uint64_t a, uint64_t b, uint32_t q)
{
    return (uint32_t)((a % q) * (b % q) % q);
}

__host__ __device__ constexpr uint32_t powmod_u32(uint64_t a, uint64_t e, uint32_t q)
{
    uint64_t r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = r * a % q;
        a = a * a % q;
        e >>= 1;
    }
    return (uint32_t)r;
}

// x * 2^32 mod q (Montgomery form of x)
__host__ __device__ constexpr uint32_t to_mont_c(uint64_t x, uint32_t q)
{
    return (uint32_t)(((x % q) << 32) % q);
}

// ------------------------------------------------ device modular arithmetic

// a + b mod q for a, b < q < 2^32 (no 32-bit overflow).
__device__ __forceinline__ uint32_t add_mod(uint32_t a, uint32_t b, uint32_t q)
{
    uint32_t t = q - b;
    return a >= t ? a - t : a + b;
}

// a - b mod q for a, b < q.
__device__ __forceinline__ uint32_t sub_mod(uint32_t a, uint32_t b, uint32_t q)
{
    uint32_t d = a - b;
    return a >= b ? d : d + q;
}

// Montgomery product a * b * 2^-32 mod q, for a < 2^32 and b < q.
// With m = (a b mod 2^32) q^-1 mod 2^32 the low words of a b and m q agree,
// so (a b - m q) / 2^32 = hi(a b) - hi(m q), which lies in (-q, q).
__device__ __forceinline__ uint32_t mont_mul(uint32_t a, uint32_t b, uint32_t q, uint32_t qinv)
{
    uint32_t lo = a * b;
    uint32_t hi = __umulhi(a, b);
    uint32_t m = lo * qinv;
    uint32_t u = __umulhi(m, q);
    uint32_t r = hi - u;
    return hi < u ? r + q : r;
}

// Same product with the multiplier's companion wp = w * q^-1 mod 2^32
// precomputed (saves one multiply); w < q, a < 2^32.
__device__ __forceinline__ uint32_t mont_mul_pre(uint32_t a, uint32_t w, uint32_t wp, uint32_t q)
{
    uint32_t hi = __umulhi(a, w);
    uint32_t m = a * wp;
    uint32_t u = __umulhi(m, q);
    uint32_t r = hi - u;
    return hi < u ? r + q : r;
}

// x mod q for any 32-bit x (q > 2^30, so at most two subtractions).
__device__ __forceinline__ uint32_t reduce32(uint32_t x, uint32_t q)
{
    if (x >= q) x -= q;
    if (x >= q) x -= q;
    return x;
}

// The same operations for a prime set: S (q < 2^31) takes the min-of-two
// forms, whose candidates never wrap because 2q < 2^32.
template <bool S>
__device__ __forceinline__ uint32_t add_m(uint32_t a, uint32_t b, uint32_t q)
{
    if (S) {
        const uint32_t s = a + b;
        return min(s, s - q);
    }
    return add_mod(a, b, q);
}

template <bool S>
__device__ __forceinline__ uint32_t sub_m(uint32_t a, uint32_t b, uint32_t q)
{
    if (S) {
        const uint32_t d = a - b + q;
        return min(d, d - q);
    }
    return sub_mod(a, b, q);
}

template <bool S>
__device__ __forceinline__ uint32_t mont_pre(uint32_t a, uint32_t w, uint32_t wp, uint32_t q)
{
    if (S) {
        const uint32_t hi = __umulhi(a, w);
        const uint32_t m = a * wp;
        const uint32_t t = hi - __umulhi(m, q) + q;
        return min(t, t - q);
    }
    return mont_mul_pre(a, w, wp, q);
}

template <bool S>
__device__ __forceinline__ uint32_t mont(uint32_t a, uint32_t b, uint32_t q, uint32_t qinv)
{
    if (S) {
        const uint32_t hi = __umulhi(a, b);
        const uint32_t m = (a * b) * qinv;
        const uint32_t t = hi - __umulhi(m, q) + q;
        return min(t, t - q);
    }
    return mont_mul(a, b, q, qinv);
}

// x mod q for any 32-bit x: for S one Montgomery product with 2^32 mod q
// (x 2^32 2^-32), otherwise at most two subtractions (q > 2^30).
template <bool S>
__device__ __forceinline__ uint32_t reduce_m(uint32_t x, uint32_t q, uint32_t qinv, uint32_t r1)
{
    if (S) return mont<true>(x, r1, q, qinv);
    return reduce32(x, q);
}

__device__ __forceinline__ uint32_t bitrev(uint32_t x, int bits)
{
    return bits == 0 ? 0u : (__brev(x) >> (32 - bits));
}

// ---------------------------------------------------------------- context

// Per-kernel timing by CUDA events around each launch (off unless enabled):
// launch count, total device milliseconds and algorithmic bytes per kernel
// name.  Events are resolved when an entry point finishes.
struct ProfEntry {
    std::string name;
    uint64_t launches = 0;
    double ms = 0;
    double bytes = 0;
    double ops = 0;  // algorithmic 32-bit integer operations
};

struct ProfPending {
    int idx;
    cudaEvent_t a, b;
    double bytes;
    double ops;
};

struct Ctx {
    int device = 0;
    size_t budget = 0;   // 0 = unlimited
    size_t in_use = 0;
    size_t peak = 0;
    std::string last_error;
    uint2 *twiddles = nullptr;  // [prime][dir][kTwPerDir] (Montgomery w, w q^-1)
    int num_sms = 0;
    size_t comba_max_slot = 128;  // tree levels with slots up to this use schoolbook
    bool profiling = false;
    std::vector<ProfEntry> prof;
    std::vector<ProfPending> pending;
    std::vector<cudaEvent_t> event_pool;
};

// Launch bracketing for the profiler: prof_begin returns a token (or -1 when
// profiling is off); prof_end records the stop event and the launch's
// algorithmic bytes.  prof_resolve turns finished pairs into totals.
int prof_begin(Ctx &c, const char *name, cudaStream_t s);
void prof_end(Ctx &c, int token, cudaStream_t s, double bytes, double ops = 0);
void prof_resolve(Ctx &c);

// Fills h[kTwTotal] with the twiddle tables of both sets (host side).
constexpr size_t kTwTotal = (size_t)kNumSets * kNumPrimes * 2 * kTwPerDir;
void twiddle_tables_host(uint2 *h);

// Device allocation from the context's stream-ordered pool (cudaMallocAsync on
// the device's default memory pool, whose release threshold is raised at
// context creation so freed blocks stay cached).
void *dev_alloc(Ctx &c, size_t bytes, cudaStream_t s);
void dev_free(Ctx &c, void *p, size_t bytes, cudaStream_t s);

template <typename T>
struct DevBuf {
    Ctx *c = nullptr;
    T *p = nullptr;
    size_t n = 0;
    cudaStream_t s = nullptr;
    DevBuf() = default;
    DevBuf(Ctx &ctx, size_t count, cudaStream_t st) : c(&ctx), n(count), s(st)
    {
        p = count ? (T *)dev_alloc(ctx, count * sizeof(T), st) : nullptr;
    }
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept { *this = std::move(o); }
    DevBuf &operator=(DevBuf &&o) noexcept
    {
        if (this != &o) {
            reset();
            c = o.c; p = o.p; n = o.n; s = o.s;
            o.p = nullptr; o.n = 0;
        }
        return *this;
    }
    ~DevBuf() { reset(); }
    void reset()
    {
        if (p && c) dev_free(*c, p, n * sizeof(T), s);
        p = nullptr;
        n = 0;
    }
    T *get() const { return p; }
    // Hands the allocation to the caller (who frees it with dev_free).
    T *release()
    {
        T *r = p;
        p = nullptr;
        n = 0;
        return r;
    }
};

// A device big integer held by the library: n limbs (upper bound on the
// normalised length; the top limbs may be zero).
struct Big {
    DevBuf<uint32_t> buf;
    size_t n = 0;
};

// A device copy job: `len` limbs from src to dst, then dst zero-filled up to
// `cap`; src == null writes the value 1.  run_copy_jobs runs a list of them
// in one launch and waits for it.
struct CopyJob {
    const uint32_t *src;
    uint32_t *dst;
    uint64_t len, cap;
};
void run_copy_jobs(Ctx &c, const std::vector<CopyJob> &jobs, cudaStream_t s);

// Where the product of one segment of a segmented product tree goes: into a
// caller's region of `cap` limbs (zero-filled above the value), or, with dst
// null, into `big` (length = an upper bound on the normalised length).
struct TreeRoot {
    uint32_t *dst = nullptr;
    uint64_t cap = 0;
    Big big;
};

// Products of the segments leaves[seg[j] .. seg[j+1]) for all j at once: one
// level-synchronous tree in which every level of every segment is a single
// batched multiplication.  An empty segment's product is 1.
void segmented_tree(Ctx &c, const uint32_t *leaves, const std::vector<uint64_t> &seg,
                    std::vector<TreeRoot> &roots, cudaStream_t s);

// ------------------------------------------------------- internal entry points
// (all on stream s; lengths are limb counts)

// out[0 .. na+nb) = a * b (exact, zero-padded).  out must hold na + nb limbs.
void mul_into(Ctx &c, const uint32_t *a, size_t na, const uint32_t *b, size_t nb,
              uint32_t *out, cudaStream_t s);
// Normalised length of x[0..n) (reads the device array).
size_t normalized_length(Ctx &c, const uint32_t *x, size_t n, cudaStream_t s);
// Product of count 32-bit values (balanced tree).  Returns the result.
Big tree_product(Ctx &c, const uint32_t *values, size_t count, cudaStream_t s);
// a^e.
Big power(Ctx &c, const uint32_t *a, size_t na, uint64_t e, cudaStream_t s);
// Phase 1 on the device.  The arrays of *out come from the context's pool
// and are released by factor_free.
void factor(Ctx &c, uint64_t n, int kind, cat_factorization *out, cudaStream_t s);
void factor_free(Ctx &c, cat_factorization *f);
// Algorithm 2 on a factorisation; returns the result (normalised length).
Big reconstruct(Ctx &c, const cat_factorization *f, cudaStream_t s);

size_t bound_limbs(uint64_t n, int kind);

}  // namespace cat
