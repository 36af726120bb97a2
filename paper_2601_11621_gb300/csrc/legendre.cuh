// legendre.cuh -- the exponent of a prime in the three quantities (Sec. 2,
// Legendre's formula, and Sec. 3.1, Algorithm 1), shared by the single and
// batched Phase-1 kernels.  2n < 2^32, so every term floor(m / p^k) is a
// 32-bit division; primes above sqrt(m) take one division per factorial.
#pragma once

#include "cat_internal.cuh"

namespace cat {

// v_p(m!) = sum_k floor(m / p^k)
__device__ __forceinline__ uint32_t legendre32(uint32_t m, uint32_t p)
{
    uint32_t s = 0;
    uint64_t pk = p;
    while (pk <= m) {
        s += m / (uint32_t)pk;
        pk *= p;
    }
    return s;
}

// v_p(x) for x > 0
__device__ __forceinline__ uint32_t valuation32(uint32_t x, uint32_t p)
{
    uint32_t v = 0;
    while (x % p == 0) {
        x /= p;
        v++;
    }
    return v;
}

// e_p by kind: Catalan v_p((2n)!) - 2 v_p(n!) - v_p(n+1); central binomial
// v_p((2n)!) - 2 v_p(n!); factorial v_p(n!).  c_p = v_p(n+1) is the exponent
// of p in the trial-division factorisation of n+1 (Algorithm 1 step 2).
__device__ __forceinline__ int64_t exponent_of(uint32_t p, uint32_t n, int kind)
{
    if (kind == CAT_FACTORIAL) return legendre32(n, p);
    int64_t e = (int64_t)legendre32(2 * n, p) - 2 * (int64_t)legendre32(n, p);
    if (kind == CAT_CATALAN) e -= valuation32(n + 1, p);
    return e;
}

// The same exponent for a prime with p^2 > 2n (Catalan or central binomial
// kinds).  Then v_p((2n)!) = floor(2n/p) and v_p(n!) = floor(n/p), so with
// r = n mod p the difference is floor(2r/p) in {0, 1} (one carry when n + n
// is added in base p), and v_p(n+1) = [p | n+1] = [r = p-1].  One division,
// none for p > n (r = n there: half of the primes up to 2n).
__device__ __forceinline__ uint32_t unit_exponent(uint32_t p, uint32_t n, int kind)
{
    const uint32_t r = p > n ? n : n % p;
    uint32_t e = 2 * r >= p ? 1u : 0u;  // 2r < 2^32: r <= n < 2^31
    if (kind == CAT_CATALAN && r == p - 1) e = 0;
    return e;
}

// v_p of a Ratio (Sec. 6.3: v_p(N) = sum_i v_p(a_i!) - sum_j v_p(b_j!)).
__device__ __forceinline__ int64_t exponent_of(uint32_t p, const Ratio &r)
{
    if (r.kind != kRatioKind) return exponent_of(p, r.n, r.kind);
    int64_t e = 0;
    for (int i = 0; i < r.ka; i++) e += legendre32(r.a[i], p);
    for (int j = 0; j < r.kb; j++) e -= legendre32(r.b[j], p);
    return e;
}

}  // namespace cat
