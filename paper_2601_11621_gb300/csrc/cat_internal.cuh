// cat_internal.cuh -- shared internals of libcatalan (context, errors, device
// memory, 32-bit modular arithmetic for the NTT primes).
//
// Integer representation: little-endian uint32 limbs.  The NTT works modulo
// three primes q = k * 2^m + 1 (one of three prime sets, by transform size,
// see below); one transform covers up to 2^27 points.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <atomic>
#include <string>
#include <vector>

#include "catalan.h"

#include <nvtx3/nvToolsExt.h>

namespace cat {

// ----------------------------------------------------------------- errors

struct Error {
    int code;
    std::string msg;
};

[[noreturn]] void fail(int code, const std::string &msg);
void check_cuda(cudaError_t e, const char *what);
// after every kernel launch: counts it (cat_launch_count) and checks it
void launched(const char *what);
#define CAT_CUDA(call) ::cat::check_cuda((call), #call)
#define CAT_LAUNCH(what) ::cat::launched(what)

// ------------------------------------------------------------- constants

constexpr int kNumPrimes = 3;
constexpr int kLogMaxNtt = 27;  // largest transform: 2^27 points
// Three sets of three NTT primes q = k 2^m + 1, chosen by the transform size
// 2^n.  In each set the product of the primes exceeds the largest convolution
// coefficient 2^(n-1) (2^32 - 1)^2 of two operands whose lengths add up to 2^n
// limbs, so the Chinese remaindering is exact.
//   set 0, n <= 23: q < 2^30, 2^23 | q - 1 (product ~2^89.35 > 2^86).  As
//          4q < 2^32, residues stay unreduced inside a transform: in [0, 2q)
//          in the forward direction and [0, 4q) in the inverse one (Harvey's
//          lazy butterflies), one correction per butterfly;
//   set 1, n <= 26: q < 2^31, 2^26 | q - 1 (product ~2^90.47 > 2^89);
//          residues in [0, q), every correction a min of two candidates,
//          which cannot wrap because 2q < 2^32;
//   set 2, n = 27:  q < 2^32, 2^27 | q - 1 (product ~2^93.6 > 2^90);
//          residues in [0, q), compare-and-subtract corrections.
// Sets 0 and 1 multiply by known factors with Shoup's method (the factor w and
// floor(w 2^32 / q) are stored); set 2 with Montgomery's (2^32 w mod q and
// that times q^-1 mod 2^32).  Primes ascend within a set.
constexpr int kNumSets = 3;
constexpr int kLogSet0 = 23;
constexpr int kLogSet1 = 26;
// Twiddle tables per (set, prime, direction), w the set's primitive 2^L-th
// root of unity (L = set_log_root) or its inverse, entries as pairs in the
// set's multiplier form:
//   [2^s, 2^(s+1))          w_{2^(s+1)}^j, j < 2^s, for s < 13: the twiddles
//                           of butterfly stage s (half-span 2^s) of a
//                           sub-transform, consecutive in j so that the
//                           lanes of a warp read consecutive entries;
//   three tables of 512     w^j, w^(512 j), w^(2^18 j): any w^E, E < 2^L,
//                           as a product of three small-table entries (in
//                           Shoup-form sets the third table is stored times
//                           2^32 mod q, so the product is w^E's Montgomery
//                           form).
constexpr int kTwStage = 1 << 13;
constexpr int kTwSmall = 512;
constexpr int kTwPerDir = kTwStage + 3 * kTwSmall;  // uint2 entries per (prime, direction)

__host__ __device__ constexpr uint32_t ntt_prime(int set, int i)
{
    return set == 0   ? (i == 0 ? 880803841u : (i == 1 ? 897581057u : 998244353u))
           : set == 1 ? (i == 0 ? 469762049u : (i == 1 ? 1811939329u : 2013265921u))
                      : (i == 0 ? 2013265921u : (i == 1 ? 2281701377u : 3221225473u));
}

// log2 of the order of the root of unity the twiddle tables of a set use
__host__ __device__ constexpr int set_log_root(int set)
{
    return set == 0 ? kLogSet0 : (set == 1 ? kLogSet1 : kLogMaxNtt);
}

// the prime set a transform of 2^n points uses
__host__ __device__ constexpr int set_for(int n)
{
    return n <= kLogSet0 ? 0 : (n <= kLogSet1 ? 1 : 2);
}

// whether a set stores its multipliers in Shoup's form
__host__ __device__ constexpr bool set_shoup(int set) { return set < 2; }

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

// floor(w 2^32 / q): Shoup's companion of a multiplier w < q
__host__ __device__ constexpr uint32_t shoup_c(uint32_t w, uint32_t q)
{
    return (uint32_t)(((uint64_t)w << 32) / q);
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

// Shoup's product: a w - floor(a wp / 2^32) q with wp = floor(w 2^32 / q)
// equals a w mod q or that plus q, for any a < 2^32 and w < q < 2^31
// (the quotient estimate is short by at most one), so it lies in [0, 2q) and
// the 32-bit wrap-around arithmetic is exact.
__device__ __forceinline__ uint32_t shoup(uint32_t a, uint32_t w, uint32_t wp, uint32_t q)
{
    return a * w - __umulhi(a, wp) * q;
}

// x - m when x >= m, for x < 2m <= 2^32: when x < m the difference wraps to
// at least 2^32 - m > x, so the smaller candidate is always the answer.
__device__ __forceinline__ uint32_t csub(uint32_t x, uint32_t m) { return min(x, x - m); }

// Modular add, subtract and Montgomery products for q < 2^31 (S) in the
// min-of-two form, or for any q < 2^32.  Inputs below q, results below q.
template <bool S>
__device__ __forceinline__ uint32_t add_m(uint32_t a, uint32_t b, uint32_t q)
{
    if (S) return csub(a + b, q);
    return add_mod(a, b, q);
}

template <bool S>
__device__ __forceinline__ uint32_t sub_m(uint32_t a, uint32_t b, uint32_t q)
{
    if (S) return csub(a - b + q, q);
    return sub_mod(a, b, q);
}

template <bool S>
__device__ __forceinline__ uint32_t mont(uint32_t a, uint32_t b, uint32_t q, uint32_t qinv)
{
    if (S) {
        const uint32_t hi = __umulhi(a, b);
        const uint32_t m = (a * b) * qinv;
        return csub(hi - __umulhi(m, q) + q, q);
    }
    return mont_mul(a, b, q, qinv);
}

// ------------------------------------------- the transform data per set
//
// Forward-transform residues lie in [0, 2q) for set 0 and in [0, q)
// otherwise; inverse-transform residues in [0, 4q) for set 0 and [0, q)
// otherwise.  A multiplier is a uint2 in the set's form.

// a w for any 32-bit a, into the forward range
template <int PS>
__device__ __forceinline__ uint32_t mul_w(uint32_t a, uint2 w, uint32_t q)
{
    if constexpr (PS == 0) return shoup(a, w.x, w.y, q);
    else if constexpr (PS == 1) return csub(shoup(a, w.x, w.y, q), q);
    else return mont_mul_pre(a, w.x, w.y, q);
}

// Forward (decimation-in-frequency) butterfly (x, y) <- (x + y, (x - y) w)
// on forward-range residues.
template <int PS>
__device__ __forceinline__ void bf_dif(uint32_t &x, uint32_t &y, uint2 w, uint32_t q)
{
    const uint32_t a = x, b = y;
    if constexpr (PS == 0) {
        x = csub(a + b, 2 * q);                 // [0, 4q) -> [0, 2q)
        y = shoup(a - b + 2 * q, w.x, w.y, q);  // (0, 4q) times w -> [0, 2q)
    } else if constexpr (PS == 1) {
        x = csub(a + b, q);
        y = csub(shoup(a - b + q, w.x, w.y, q), q);
    } else {
        x = add_mod(a, b, q);
        y = mont_mul_pre(sub_mod(a, b, q), w.x, w.y, q);
    }
}

// the same with w = 1
template <int PS>
__device__ __forceinline__ void bf_dif1(uint32_t &x, uint32_t &y, uint32_t q)
{
    const uint32_t a = x, b = y;
    if constexpr (PS == 0) {
        x = csub(a + b, 2 * q);
        y = csub(a - b + 2 * q, 2 * q);
    } else {
        x = add_m<PS == 1>(a, b, q);
        y = sub_m<PS == 1>(a, b, q);
    }
}

// Inverse (decimation-in-time) butterfly (x, y) <- (x + y w, x - y w) on
// inverse-range residues.
template <int PS>
__device__ __forceinline__ void bf_dit(uint32_t &x, uint32_t &y, uint2 w, uint32_t q)
{
    if constexpr (PS == 0) {
        const uint32_t a = csub(x, 2 * q);          // [0, 2q)
        const uint32_t t = shoup(y, w.x, w.y, q);   // [0, 2q)
        x = a + t;                                  // [0, 4q)
        y = a - t + 2 * q;                          // (0, 4q)
    } else {
        const uint32_t a = x, t = mul_w<PS>(y, w, q);
        x = add_m<PS == 1>(a, t, q);
        y = sub_m<PS == 1>(a, t, q);
    }
}

template <int PS>
__device__ __forceinline__ void bf_dit1(uint32_t &x, uint32_t &y, uint32_t q)
{
    if constexpr (PS == 0) {
        const uint32_t a = csub(x, 2 * q), t = csub(y, 2 * q);
        x = a + t;
        y = a - t + 2 * q;
    } else {
        const uint32_t a = x, b = y;
        x = add_m<PS == 1>(a, b, q);
        y = sub_m<PS == 1>(a, b, q);
    }
}

// A raw 32-bit limb into the forward range: Shoup's product with 1
// (wp1 = floor(2^32 / q)) for sets 0 and 1, two subtractions for set 2.
template <int PS>
__device__ __forceinline__ uint32_t reduce_in(uint32_t x, uint32_t q, uint32_t wp1)
{
    if constexpr (PS == 0) return shoup(x, 1u, wp1, q);
    else if constexpr (PS == 1) return csub(shoup(x, 1u, wp1, q), q);
    else return reduce32(x, q);
}

// Pointwise product of two forward-range residues times the scale factor:
// x y 2^-32 by Montgomery's reduction, then times sc = 2^32 2^-n (Shoup) for
// sets 0 and 1 or sc = 2^64 2^-n (Montgomery) for set 2, giving x y 2^-n.
// For set 0, x y < 4 q^2 < 2^32 q keeps hi(x y) - hi(m q) in (-q, q).
template <int PS>
__device__ __forceinline__ uint32_t pmul(uint32_t x, uint32_t y, uint2 sc, uint32_t q,
                                         uint32_t qinv)
{
    if constexpr (PS == 0) {
        const uint32_t hi = __umulhi(x, y);
        const uint32_t m = (x * y) * qinv;
        return shoup(hi - __umulhi(m, q) + q, sc.x, sc.y, q);
    } else if constexpr (PS == 1) {
        return csub(shoup(mont<true>(x, y, q, qinv), sc.x, sc.y, q), q);
    } else {
        return mont_mul(mont_mul(x, y, q, qinv), sc.x, q, qinv);
    }
}

// An inverse-range residue reduced into [0, q).
template <int PS>
__device__ __forceinline__ uint32_t final_red(uint32_t r, uint32_t q)
{
    if constexpr (PS == 0) return csub(csub(r, 2 * q), q);
    return r;
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
    double unit_bytes = 0;  // algorithmic bytes of the products the launches completed
};

struct ProfPending {
    int idx;
    cudaEvent_t a, b;
    double bytes;
    double unit_bytes;
};

struct Ctx {
    int device = 0;
    size_t budget = 0;   // 0 = unlimited
    size_t in_use = 0;
    // A budget shared with other contexts (the serving engine's workers): the
    // bytes all of them hold, and their common cap (0 = none).
    std::atomic<size_t> *shared_in_use = nullptr;
    std::atomic<size_t> *shared_peak = nullptr;  // high-water mark of *shared_in_use
    size_t shared_budget = 0;
    size_t peak = 0;
    std::string last_error;
    uint2 *twiddles = nullptr;  // [set][prime][dir][kTwPerDir] multiplier pairs
    int num_sms = 0;
    size_t comba_max_slot = 128;  // tree levels with slots up to this use schoolbook
    int max_log = kLogMaxNtt;     // longest single transform; longer products go by pieces
    // row-pass size (log2 points) of the multi-pass transform of 2^n points,
    // as tuned on this device (cat_autotune); 0 = the default plan
    int row_log[kLogMaxNtt + 1] = {};
    std::string tuning;           // where the tuned values came from ("" = defaults)
    // twiddle tables of the column passes (built on first use, kept until the
    // context is released; contexts with a budget compute the twiddles)
    struct ColTwTable {
        int ps, m, lr, dir;
        bool scaled;  // entries times 2^(32-m): operand b's first forward pass
        uint32_t *p;
    };
    std::vector<ColTwTable> col_tw;
    bool col_tw_tables = true;
    // largest block (log2 points) whose passes read a table: for the first
    // forward pass (which runs once per operand) and for the others (all by
    // default; smaller values are for measurements)
    int col_tw_first_max_log = kLogMaxNtt, col_tw_max_log = kLogMaxNtt;
    // small read-backs (lengths of results): a pinned host word and a device
    // word, allocated once per context
    uint64_t *host_word = nullptr;
    unsigned long long *dev_word = nullptr;
    bool profiling = false;
    std::vector<ProfEntry> prof;
    std::vector<ProfPending> pending;
    std::vector<cudaEvent_t> event_pool;
};

// Launch bracketing for the profiler: prof_begin returns a token (or -1 when
// profiling is off); prof_end records the stop event and the launch's
// algorithmic bytes.  prof_resolve turns finished pairs into totals.
int prof_begin(Ctx &c, const char *name, cudaStream_t s);
// unit_bytes: the algorithmic bytes of the products the launch completes
// (operands read once and the product written once, 4 bytes per limb each),
// counted on the one launch of a product that holds its pointwise step (the
// row pass, the one-block multiply, a schoolbook or leaf kernel); 0 elsewhere.
void prof_end(Ctx &c, int token, cudaStream_t s, double bytes, double unit_bytes = 0);
void prof_resolve(Ctx &c);

// Where the limbs of a batch of products go: product k at out + k *
// out_tstride, out_len limbs, in base 2^32 or (dec) in base 10^9; with `add`,
// the limbs add + k * add_tstride (add_len of them, zero beyond) are added in
// before the carries (the sum must fit out_len limbs).
struct Sink {
    uint32_t *out;
    size_t out_tstride, out_len;
    bool dec;
    const uint32_t *add;
    size_t add_tstride, add_len;
    // when set, product k goes to out + out_index[k] * out_tstride (a device
    // table), else to out + k * out_tstride
    const uint32_t *out_index = nullptr;
};

__host__ __device__ __forceinline__ size_t sink_node(const Sink &o, size_t k)
{
    return o.out_index ? (size_t)o.out_index[k] : k;
}

constexpr uint32_t kDecBase = 1000000000u;

inline Sink plain_sink(uint32_t *out, size_t out_tstride, size_t out_len)
{
    return Sink{out, out_tstride, out_len, false, nullptr, 0, 0};
}

// An NVTX range over a scope (phases and tree levels show up by name in
// profilers; no cost without one attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Fills h[kTwTotal] with the twiddle tables of all sets (host side).
constexpr size_t kTwTotal = (size_t)kNumSets * kNumPrimes * 2 * kTwPerDir;
void twiddle_tables_host(uint2 *h);
// Copies the first 16 entries of every stage table of h into the constant
// memory of the current device (ntt.cu).
void upload_low_twiddles(const uint2 *h);

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

// Leaves of a product tree per first-level node (eight limbs) when every
// leaf is below 2^bits: their product stays below 2^256.
inline int leaves_per_node(int bits)
{
    bits = bits < 1 ? 1 : (bits > 32 ? 32 : bits);
    const int k = 256 / bits;
    return k > 32 ? 32 : k;
}

// Bits of the largest value <= limit (limit < 2^32): a bound on the primes
// of a factorisation whose sieve stopped at limit.
inline int bits_below(uint64_t limit)
{
    int b = 1;
    while (b < 32 && (limit >> b)) b++;
    return b;
}

// Products of the segments leaves[seg[j] .. seg[j+1]) for all j at once: one
// level-synchronous tree in which every level of every segment is a single
// batched multiplication.  An empty segment's product is 1.  Every leaf is
// below 2^leaf_bits, so that a first-level node of eight limbs takes
// floor(256 / leaf_bits) leaves (at most 32).
void segmented_tree(Ctx &c, const uint32_t *leaves, const std::vector<uint64_t> &seg,
                    std::vector<TreeRoot> &roots, cudaStream_t s, int leaf_bits = 32);

// ------------------------------------------------------- internal entry points
// (all on stream s; lengths are limb counts)

// One level of a product tree: nprod products of adjacent slot-limb nodes
// (in[2k] times in[2k+1]) into 2*slot-limb nodes of out.  Product k goes to
// node out_index[k] of out (a device table; out_index_host, where given, is
// its host copy) or, without a table, to node k.  comba_level returns false
// for slots it has no schoolbook kernel for.
bool comba_level(Ctx &c, const uint32_t *in, size_t slot, size_t nprod, uint32_t *out,
                 cudaStream_t s, const uint32_t *out_index = nullptr);
void ntt_level(Ctx &c, const uint32_t *level, size_t slot, size_t nprod, uint32_t *out,
               cudaStream_t s, const uint32_t *out_index = nullptr,
               const uint32_t *out_index_host = nullptr);

// out[0 .. na+nb) = a * b (exact, zero-padded).  out must hold na + nb limbs.
void mul_into(Ctx &c, const uint32_t *a, size_t na, const uint32_t *b, size_t nb,
              uint32_t *out, cudaStream_t s);
// nprod products x_k y (x_k at x + k xstride, xlen limbs; one y of ylen
// limbs, transformed once) into `sink`; xlen + ylen <= 2^27.
void mul_broadcast(Ctx &c, const uint32_t *x, size_t xstride, size_t xlen, size_t nprod,
                   const uint32_t *y, size_t ylen, const Sink &sink, cudaStream_t s);
// acc[0 .. R) += t[0 .. tn), base 2^32 or (dec) 10^9, carries through acc.
void add_into(Ctx &c, uint32_t *acc, size_t R, const uint32_t *t, size_t tn, bool dec,
              cudaStream_t s);
// out[0 .. nx + ny) = x y for ny <= 2^k - ny: chunks of 2^k - ny limbs of x
// times y in one batch (y transformed once), overlap-added.
void mul_chunked(Ctx &c, const uint32_t *x, size_t nx, const uint32_t *y, size_t ny, int k,
                 uint32_t *out, cudaStream_t s);
// acc[0 .. R) += x y for any lengths (pieces of <= 2^26 limbs when long).
void mul_acc(Ctx &c, const uint32_t *x, size_t xlen, const uint32_t *y, size_t ylen,
             uint32_t *acc, size_t R, bool dec, cudaStream_t s);
// Decimal digits of x[0..n) into out (device, no sign, no terminator, "0"
// for zero); returns the digit count.  Fails with CAT_ERANGE (and the count
// in *needed) when cap is too small.
size_t decimal_bound(size_t n);
int to_decimal_dev(Ctx &c, const uint32_t *x, size_t n, char *out, size_t cap, size_t *needed,
                   cudaStream_t s);
// Normalised length of x[0..n) (reads the device array).
size_t normalized_length(Ctx &c, const uint32_t *x, size_t n, cudaStream_t s);
// The same, reading only the top four limbs when one of them is nonzero (the
// usual case for a product of normalised operands).
size_t trim(Ctx &c, const uint32_t *x, size_t n, cudaStream_t s);
// Product of count 32-bit values (balanced tree).  Returns the result.
// The product of values[0 .. count), times *extra when given; exact = false
// returns a length bound (zero top limbs) without a host read-back (tree.cu).
// Every value is below 2^leaf_bits: a first-level node of eight limbs then
// takes leaves_per_node(leaf_bits) values.
Big tree_product(Ctx &c, const uint32_t *values, size_t count, cudaStream_t s,
                 const Big *extra = nullptr, bool exact = true, int leaf_bits = 32);
// a^e.
Big power(Ctx &c, const uint32_t *a, size_t na, uint64_t e, cudaStream_t s, bool exact = true);
// Factorial ratios (Sec. 6.3): N = prod_i a_i! / prod_j b_j!.  A Ratio also
// describes the three kinds (kind < kRatioKind: the quantity of n).  Every
// term is below 2^32 and the a_i sum to less than 2^32, so every exponent
// fits 32 bits.
constexpr int kRatioKind = 3;
constexpr int kMaxRatioTerms = 16;

struct Ratio {
    int kind;
    uint32_t n;
    int ka, kb;
    uint32_t a[kMaxRatioTerms], b[kMaxRatioTerms];
};

// Phase 1 on the device.  The arrays of *out come from the context's pool
// and are released by factor_free.
void factor(Ctx &c, uint64_t n, int kind, cat_factorization *out, cudaStream_t s);
void factor_ratio(Ctx &c, const Ratio &r, cat_factorization *out, cudaStream_t s);
void factor_free(Ctx &c, cat_factorization *f);

// n limbs from device memory into host memory, on stream s (not synchronised):
// a store kernel when the host range is page-locked and mapped for the
// device, a copy-engine transfer otherwise.
void copy_to_host(Ctx &c, uint32_t *host, const uint32_t *dev, size_t n, cudaStream_t s);
// Algorithm 2 on a factorisation; returns the result (normalised length).
// Every prime of f is below 2^leaf_bits (32 when nothing smaller is known).
Big reconstruct(Ctx &c, const cat_factorization *f, cudaStream_t s, int leaf_bits = 32);
// Kernels launched by the library so far (every CAT_LAUNCH).
unsigned long long launch_count();

// Frees the context's column-pass twiddle tables.
void drop_col_twiddles(Ctx &c);

// Whether the in-core reconstruction of f would exceed the context's HBM
// budget, and Algorithm 2 within the budget (ooc.cu): copies f's primes to
// pinned host memory (and, with release, frees f's device arrays), multiplies
// by chunks and pieces, and copies the result (*out_len limbs) to out, device
// memory or (to_host) host memory.
bool reconstruct_out_of_core(const Ctx &c, const cat_factorization *f);
void reconstruct_into(Ctx &c, cat_factorization *f, uint32_t *out, size_t cap, bool to_host,
                      size_t *out_len, cudaStream_t s, bool release = true);

// The factorisation as the paper's text layout (Sec. 3.1) into out (device),
// titled `name`; the binary result file (bytes 01 01, then the magnitude
// little-endian).  Both fail with CAT_ERANGE when cap is short (*needed set).
int factor_text(Ctx &c, const cat_factorization *f, const char *name, char *out, size_t cap,
                size_t *needed, cudaStream_t s);
int binary_file(Ctx &c, const uint32_t *x, size_t n, uint8_t *out, size_t cap, size_t *needed,
                cudaStream_t s);

size_t bound_limbs(uint64_t n, int kind);

// The tuned choices of the multiplication (autotune.cu): measure and apply
// them, write or read a table, and the table a new context reads.
void autotune(Ctx &c, cudaStream_t s);
void save_tuning(const Ctx &c, const char *path);
bool load_tuning(Ctx &c, const char *path);
std::string default_tuning_path();
size_t ratio_bound_limbs(const Ratio &r);

}  // namespace cat
