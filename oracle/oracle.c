/*
 * oracle.c -- plain, slow, obviously-correct CPU oracle for the exact
 * Catalan / central-binomial / factorial computation of arXiv 2601.11621.
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no source, header,
 * table or helper with the CUDA library; the two meet only through the seeded
 * input generators and through the tests that compare their outputs.
 *
 * Every function follows the paper's definitions in the paper's order:
 *   - Sec. 2 (Legendre's formula)   : v_p(m!) = sum_k floor(m / p^k)
 *   - Sec. 2 (Catalan valuation)    : e_p = v_p((2n)!) - 2 v_p(n!) - v_p(n+1)
 *   - Sec. 3.1, Algorithm 1         : sieve, trial-division of n+1, exponent
 *                                      loop dropping e = 0, grouping by e,
 *                                      digit-count estimate
 *   - Sec. 3.2, Algorithm 2         : Q_e = BalancedProductTree(G_e),
 *                                      P_e = Q_e^e, C = BalancedProductTree(P)
 *   - Sec. 6.3 (factorial ratios)   : v_p(N) = sum_i v_p(a_i!) - sum_j v_p(b_j!)
 * plus two verification helpers the paper names but does not define
 * ("modular checks", abstract and Sec. 1): the residue of the exact integer
 * modulo a prime q > 2n, computed from factorial products with no sieve.
 *
 * Big integers are little-endian arrays of uint32_t limbs.  A result length is
 * always normalised (top limb non-zero); zero has length 0, one is {1}.
 *
 * Parity status: every exported function is pinned by a CPU test against an
 * independent fact (brute force, CPython integers, textbook prime counts,
 * Kummer's theorem, the paper's printed digit and bit counts).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Multi-threaded runs (orc_exact_mt only): the two halves of a product tree
 * and the three sub-products of a Karatsuba step become OpenMP tasks when they
 * are at least this large.  Outside a parallel region a task runs at once in
 * the calling thread, so every other entry point stays single-threaded and
 * computes in exactly the order written. */
#define ORC_TASK_MIN_LIMBS 2048
#define ORC_TASK_MIN_VALUES 4096

typedef uint32_t limb_t;
typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------ */
/* Primes: Sieve of Eratosthenes (Sec. 3.1, Algorithm 1 step 1).             */
/* A plain byte-per-integer sieve, cut into blocks only so that the memory   */
/* stays bounded at large limits.  The paper's parallel segmented sieve      */
/* finds the same set.                                                        */
/* ------------------------------------------------------------------------ */

static uint64_t isqrt_u64(uint64_t x)
{
    uint64_t r = (uint64_t)sqrtl((long double)x);
    while (r > 0 && r * r > x) r--;
    while ((r + 1) * (r + 1) <= x) r++;
    return r;
}

/* Writes the primes <= limit in ascending order to out (at most cap of them)
 * and returns how many primes <= limit exist (which may exceed cap). */
uint64_t orc_sieve(uint64_t limit, uint32_t *out, uint64_t cap)
{
    if (limit < 2) return 0;
    uint64_t root = isqrt_u64(limit);
    unsigned char *small = calloc(root + 1, 1); /* 1 = composite */
    uint64_t nseeds = 0;
    uint64_t *seeds = malloc(sizeof(uint64_t) * (root + 1));
    for (uint64_t i = 2; i <= root; i++) {
        if (small[i]) continue;
        seeds[nseeds++] = i;
        for (uint64_t j = i * i; j <= root; j += i) small[j] = 1;
    }
    free(small);

    const uint64_t block = (uint64_t)1 << 24;
    unsigned char *seg = malloc(block);
    uint64_t count = 0;
    for (uint64_t lo = 2; lo <= limit; lo += block) {
        uint64_t hi = lo + block; /* exclusive */
        if (hi > limit + 1) hi = limit + 1;
        memset(seg, 0, hi - lo);
        for (uint64_t s = 0; s < nseeds; s++) {
            uint64_t p = seeds[s];
            uint64_t start = p * p;
            if (start >= hi) break;
            if (start < lo) start = ((lo + p - 1) / p) * p;
            for (uint64_t j = start; j < hi; j += p) seg[j - lo] = 1;
        }
        for (uint64_t x = lo; x < hi; x++) {
            if (!seg[x - lo]) {
                if (count < cap) out[count] = (uint32_t)x;
                count++;
            }
        }
    }
    free(seg);
    free(seeds);
    return count;
}

/* The primes in [lo, hi] (same plain block sieve, started at lo).  Used to
 * time a bounded slice of a large sieve.  Returns the count; writes at most
 * cap of them. */
uint64_t orc_sieve_range(uint64_t lo, uint64_t hi, uint32_t *out, uint64_t cap)
{
    if (hi < 2 || hi < lo) return 0;
    if (lo < 2) lo = 2;
    uint64_t root = isqrt_u64(hi);
    unsigned char *small = calloc(root + 1, 1);
    uint64_t nseeds = 0;
    uint64_t *seeds = malloc(sizeof(uint64_t) * (root + 1));
    for (uint64_t i = 2; i <= root; i++) {
        if (small[i]) continue;
        seeds[nseeds++] = i;
        for (uint64_t j = i * i; j <= root; j += i) small[j] = 1;
    }
    free(small);
    const uint64_t block = (uint64_t)1 << 24;
    unsigned char *seg = malloc(block);
    uint64_t count = 0;
    for (uint64_t b = lo; b <= hi; b += block) {
        uint64_t e = b + block;
        if (e > hi + 1) e = hi + 1;
        memset(seg, 0, e - b);
        for (uint64_t s = 0; s < nseeds; s++) {
            uint64_t p = seeds[s];
            uint64_t start = p * p;
            if (start >= e) break;
            if (start < b) start = ((b + p - 1) / p) * p;
            for (uint64_t j = start; j < e; j += p) seg[j - b] = 1;
        }
        for (uint64_t x = b; x < e; x++) {
            if (!seg[x - b]) {
                if (count < cap) out[count] = (uint32_t)x;
                count++;
            }
        }
    }
    free(seg);
    free(seeds);
    return count;
}

/* ------------------------------------------------------------------------ */
/* Legendre's formula (Sec. 2): v_p(m!) = sum_{k>=1} floor(m / p^k).         */
/* The loop stops once p^(k+1) would exceed m, so p^k never overflows.       */
/* ------------------------------------------------------------------------ */
uint64_t orc_legendre(uint64_t m, uint64_t p)
{
    uint64_t s = 0, pk = p;
    for (;;) {
        s += m / pk;
        if (pk > m / p) break;
        pk *= p;
    }
    return s;
}

/* Algorithm 1 step 2: factor m = n+1 by trial division with the primes up to
 * sqrt(m); whatever cofactor > 1 remains is itself prime (exponent 1).
 * Writes up to cap (prime, exponent) pairs and returns how many there are. */
int orc_factor_trial(uint64_t m, const uint32_t *primes, uint64_t nprimes,
                     uint64_t *fac_p, uint64_t *fac_e, int cap)
{
    int k = 0;
    for (uint64_t i = 0; i < nprimes; i++) {
        uint64_t p = primes[i];
        if (p * p > m) break;
        if (m % p == 0) {
            uint64_t e = 0;
            while (m % p == 0) { m /= p; e++; }
            if (k < cap) { fac_p[k] = p; fac_e[k] = e; }
            k++;
        }
    }
    if (m > 1) {
        if (k < cap) { fac_p[k] = m; fac_e[k] = 1; }
        k++;
    }
    return k;
}

/* Kinds of quantity (Sec. 6.3 special cases). */
enum { ORC_CATALAN = 0, ORC_CENTRAL_BINOMIAL = 1, ORC_FACTORIAL = 2 };

/* Largest prime that can divide the quantity: 2n for the binomial kinds,
 * n for n!. */
uint64_t orc_prime_limit(int kind, uint64_t n)
{
    return kind == ORC_FACTORIAL ? n : 2 * n;
}

/* Algorithm 1 steps 3-9 for every prime of primes[0..count): writes the signed
 * exponent e_p of the requested kind.
 *   Catalan          : a - 2b - c, a = v_p((2n)!), b = v_p(n!), c = v_p(n+1)
 *                      (c from the trial-division factorisation of n+1)
 *   central binomial : a - 2b
 *   factorial        : v_p(n!)
 * Returns 0, or -1 if n+1 has more prime factors than the local table. */
int orc_exponents(int kind, uint64_t n, const uint32_t *primes, uint64_t count,
                  int64_t *e_out)
{
    uint64_t fp[64], fe[64];
    int nf = 0;
    if (kind == ORC_CATALAN) {
        nf = orc_factor_trial(n + 1, primes, count, fp, fe, 64);
        if (nf > 64) return -1;
    }
    for (uint64_t i = 0; i < count; i++) {
        uint64_t p = primes[i];
        int64_t e;
        if (kind == ORC_FACTORIAL) {
            e = (int64_t)orc_legendre(n, p);
        } else {
            uint64_t a = orc_legendre(2 * n, p);
            uint64_t b = orc_legendre(n, p);
            e = (int64_t)a - 2 * (int64_t)b;
            if (kind == ORC_CATALAN) {
                for (int j = 0; j < nf; j++)
                    if (fp[j] == p) e -= (int64_t)fe[j];
            }
        }
        e_out[i] = e;
    }
    return 0;
}

/* Sec. 6.3: v_p(N) for N = prod a_i! / prod b_j!, for each prime. */
void orc_ratio_exponents(const uint64_t *a, int ka, const uint64_t *b, int kb,
                         const uint32_t *primes, uint64_t count, int64_t *e_out)
{
    for (uint64_t i = 0; i < count; i++) {
        int64_t e = 0;
        for (int j = 0; j < ka; j++) e += (int64_t)orc_legendre(a[j], primes[i]);
        for (int j = 0; j < kb; j++) e -= (int64_t)orc_legendre(b[j], primes[i]);
        e_out[i] = e;
    }
}

/* Algorithm 1 steps 10-13 and 14: keep the primes with e > 0 and group them by
 * exponent.  Output in CSR form: exps[g] ascending, group g's primes are
 * grouped_primes[offsets[g] .. offsets[g+1]) in ascending prime order.
 * Returns the number of groups.  exps/offsets need room for (distinct e)+1. */
static int cmp_u64(const void *x, const void *y)
{
    uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
    return (a > b) - (a < b);
}

static uint64_t find_group(const uint64_t *exps, uint64_t ng, uint64_t v)
{
    uint64_t lo = 0, hi = ng; /* exps[lo..hi) sorted; v is present */
    while (hi - lo > 1) {
        uint64_t mid = (lo + hi) / 2;
        if (exps[mid] <= v) lo = mid; else hi = mid;
    }
    return lo;
}

uint64_t orc_group(const uint32_t *primes, const int64_t *e, uint64_t count,
                   uint64_t *exps, uint64_t *offsets, uint32_t *grouped_primes)
{
    /* distinct positive exponents, ascending */
    uint64_t npos = 0;
    for (uint64_t i = 0; i < count; i++)
        if (e[i] > 0) exps[npos++] = (uint64_t)e[i];
    qsort(exps, npos, sizeof(uint64_t), cmp_u64);
    uint64_t ng = 0;
    for (uint64_t i = 0; i < npos; i++)
        if (ng == 0 || exps[ng - 1] != exps[i]) exps[ng++] = exps[i];
    /* count per group, prefix sums, then place primes in input order */
    for (uint64_t g = 0; g <= ng; g++) offsets[g] = 0;
    for (uint64_t i = 0; i < count; i++)
        if (e[i] > 0) offsets[find_group(exps, ng, (uint64_t)e[i]) + 1]++;
    for (uint64_t g = 0; g < ng; g++) offsets[g + 1] += offsets[g];
    uint64_t *fill = calloc(ng + 1, sizeof(uint64_t));
    for (uint64_t i = 0; i < count; i++) {
        if (e[i] <= 0) continue;
        uint64_t g = find_group(exps, ng, (uint64_t)e[i]);
        grouped_primes[offsets[g] + fill[g]++] = primes[i];
    }
    free(fill);
    return ng;
}

/* Digit-count estimate (Algorithm 1, last step): sum of e_p log10 p, summed
 * with Kahan compensation in long double.  floor(result) + 1 = digits. */
long double orc_log10_estimate(const uint32_t *primes, const int64_t *e,
                               uint64_t count)
{
    long double s = 0.0L, c = 0.0L;
    for (uint64_t i = 0; i < count; i++) {
        if (e[i] == 0) continue;
        long double term = (long double)e[i] * log10l((long double)primes[i]);
        long double y = term - c;
        long double t = s + y;
        c = (t - s) - y;
        s = t;
    }
    return s;
}

/* ------------------------------------------------------------------------ */
/* Big-integer arithmetic: schoolbook and Karatsuba multiplication.          */
/* ------------------------------------------------------------------------ */

static uint64_t norm_len(const limb_t *a, uint64_t n)
{
    while (n > 0 && a[n - 1] == 0) n--;
    return n;
}

/* out[0 .. na+nb) = a * b, schoolbook.  out must not alias a or b. */
static void mul_school(const limb_t *a, uint64_t na, const limb_t *b, uint64_t nb,
                       limb_t *out)
{
    memset(out, 0, sizeof(limb_t) * (na + nb));
    for (uint64_t i = 0; i < na; i++) {
        uint64_t carry = 0;
        for (uint64_t j = 0; j < nb; j++) {
            uint64_t t = (uint64_t)out[i + j] + (uint64_t)a[i] * b[j] + carry;
            out[i + j] = (limb_t)t;
            carry = t >> 32;
        }
        out[i + nb] = (limb_t)carry;
    }
}

/* r[0..n) += x[0..m) (m <= n); returns the carry out of r[n-1]. */
static limb_t add_into(limb_t *r, uint64_t n, const limb_t *x, uint64_t m)
{
    uint64_t carry = 0;
    for (uint64_t i = 0; i < n; i++) {
        uint64_t t = (uint64_t)r[i] + (i < m ? x[i] : 0) + carry;
        r[i] = (limb_t)t;
        carry = t >> 32;
        if (i >= m && carry == 0) break;
    }
    return (limb_t)carry;
}

/* r[0..n) -= x[0..m) (m <= n), assuming the result is non-negative. */
static void sub_from(limb_t *r, uint64_t n, const limb_t *x, uint64_t m)
{
    int64_t borrow = 0;
    for (uint64_t i = 0; i < n; i++) {
        int64_t t = (int64_t)r[i] - (i < m ? (int64_t)x[i] : 0) - borrow;
        borrow = t < 0;
        r[i] = (limb_t)(t + (borrow ? ((int64_t)1 << 32) : 0));
        if (i >= m && borrow == 0) break;
    }
}

#define KARATSUBA_CUTOFF 32

static void mul_any(const limb_t *a, uint64_t na, const limb_t *b, uint64_t nb,
                    limb_t *out);

/* Textbook Karatsuba for equal lengths n (= na = nb), n >= cutoff:
 *   a = a1 B + a0, b = b1 B + b0, B = 2^(32h)
 *   z0 = a0 b0, z2 = a1 b1, z1 = (a0+a1)(b0+b1) - z0 - z2
 *   a b = z2 B^2 + z1 B + z0.  out gets 2n limbs. */
static void mul_karatsuba(const limb_t *a, const limb_t *b, uint64_t n, limb_t *out)
{
    if (n < KARATSUBA_CUTOFF) { mul_school(a, n, b, n, out); return; }
    uint64_t h = n / 2, hh = n - h; /* low part h limbs, high part hh >= h */
    const limb_t *a0 = a, *a1 = a + h, *b0 = b, *b1 = b + h;
    limb_t *sa = calloc(hh + 1, sizeof(limb_t));
    limb_t *sb = calloc(hh + 1, sizeof(limb_t));
    memcpy(sa, a1, sizeof(limb_t) * hh);
    memcpy(sb, b1, sizeof(limb_t) * hh);
    sa[hh] = add_into(sa, hh, a0, h);
    sb[hh] = add_into(sb, hh, b0, h);
    limb_t *z1 = calloc(2 * (hh + 1), sizeof(limb_t));
    memset(out, 0, sizeof(limb_t) * 2 * n);
    /* the three products are independent (disjoint outputs) */
#pragma omp task if (n >= ORC_TASK_MIN_LIMBS)
    mul_karatsuba(sa, sb, hh + 1, z1);
#pragma omp task if (n >= ORC_TASK_MIN_LIMBS)
    mul_karatsuba(a0, b0, h, out);                 /* z0 -> out[0, 2h)     */
    mul_karatsuba(a1, b1, hh, out + 2 * h);        /* z2 -> out[2h, 2n)    */
#pragma omp taskwait
    sub_from(z1, 2 * (hh + 1), out, 2 * h);         /* z1 -= z0             */
    sub_from(z1, 2 * (hh + 1), out + 2 * h, 2 * hh); /* z1 -= z2            */
    add_into(out + h, 2 * n - h, z1, norm_len(z1, 2 * (hh + 1)));
    free(sa); free(sb); free(z1);
}

/* out[0 .. na+nb) = a * b for any lengths.  Operands within a factor of two
 * of each other go through Karatsuba after zero-extending the shorter one; a
 * much longer operand is cut into blocks of the shorter one's length and the
 * partial products are added at their offsets. */
static void mul_any(const limb_t *a, uint64_t na, const limb_t *b, uint64_t nb,
                    limb_t *out)
{
    if (na < nb) { const limb_t *t = a; a = b; b = t; uint64_t u = na; na = nb; nb = u; }
    if (nb == 0) { memset(out, 0, sizeof(limb_t) * na); return; }
    if (nb < KARATSUBA_CUTOFF) { mul_school(a, na, b, nb, out); return; }
    if (na == nb) { mul_karatsuba(a, b, na, out); return; }
    if (2 * nb >= na) {
        limb_t *bp = calloc(na, sizeof(limb_t));
        limb_t *full = malloc(sizeof(limb_t) * 2 * na);
        memcpy(bp, b, sizeof(limb_t) * nb);
        mul_karatsuba(a, bp, na, full);
        memcpy(out, full, sizeof(limb_t) * (na + nb)); /* the rest is zero */
        free(bp); free(full);
        return;
    }
    memset(out, 0, sizeof(limb_t) * (na + nb));
    limb_t *part = malloc(sizeof(limb_t) * 2 * nb);
    for (uint64_t off = 0; off < na; off += nb) {
        uint64_t len = na - off < nb ? na - off : nb;
        mul_any(a + off, len, b, nb, part);
        add_into(out + off, na + nb - off, part, norm_len(part, len + nb));
    }
    free(part);
}

/* Exported multiply: writes normalised a*b into out (room for na+nb limbs);
 * returns the normalised length. */
uint64_t orc_mul(const limb_t *a, uint64_t na, const limb_t *b, uint64_t nb,
                 limb_t *out)
{
    na = norm_len(a, na);
    nb = norm_len(b, nb);
    if (na == 0 || nb == 0) return 0;
    mul_any(a, na, b, nb, out);
    return norm_len(out, na + nb);
}

/* ------------------------------------------------------------------------ */
/* A minimal owned big-integer for the recursive algorithms.                 */
/* ------------------------------------------------------------------------ */
typedef struct { limb_t *d; uint64_t n; } big_t;

static big_t big_from_u64(uint64_t v)
{
    big_t r;
    r.d = malloc(sizeof(limb_t) * 2);
    r.d[0] = (limb_t)v;
    r.d[1] = (limb_t)(v >> 32);
    r.n = norm_len(r.d, 2);
    return r;
}

static big_t big_mul(big_t a, big_t b)
{
    big_t r;
    r.d = malloc(sizeof(limb_t) * (a.n + b.n + 1));
    r.n = orc_mul(a.d, a.n, b.d, b.n, r.d);
    return r;
}

/* BalancedProductTree (Sec. 3.2): recursive divide-and-conquer product of
 * the values v[0..count), splitting the list in halves. */
static big_t tree_u32(const uint32_t *v, uint64_t count)
{
    if (count == 0) return big_from_u64(1);
    if (count == 1) return big_from_u64(v[0]);
    uint64_t h = count / 2;
    big_t l, r;
#pragma omp task shared(l) if (count >= ORC_TASK_MIN_VALUES)
    l = tree_u32(v, h);
    r = tree_u32(v + h, count - h);
#pragma omp taskwait
    big_t p = big_mul(l, r);
    free(l.d); free(r.d);
    return p;
}

static big_t tree_big(big_t *v, uint64_t count)
{
    if (count == 0) return big_from_u64(1);
    if (count == 1) {
        big_t c; c.n = v[0].n; c.d = malloc(sizeof(limb_t) * (c.n + 1));
        memcpy(c.d, v[0].d, sizeof(limb_t) * c.n);
        return c;
    }
    uint64_t h = count / 2;
    big_t l, r;
#pragma omp task shared(l) if (count >= 4)
    l = tree_big(v, h);
    r = tree_big(v + h, count - h);
#pragma omp taskwait
    big_t p = big_mul(l, r);
    free(l.d); free(r.d);
    return p;
}

/* "fast pow" of Algorithm 2: left-to-right binary exponentiation. */
static big_t big_pow(big_t a, uint64_t e)
{
    if (e == 0) return big_from_u64(1);
    big_t r; r.n = a.n; r.d = malloc(sizeof(limb_t) * (a.n + 1));
    memcpy(r.d, a.d, sizeof(limb_t) * a.n);
    int top = 63;
    while (!((e >> top) & 1)) top--;
    for (int bit = top - 1; bit >= 0; bit--) {
        big_t s = big_mul(r, r);
        free(r.d);
        r = s;
        if ((e >> bit) & 1) {
            big_t t = big_mul(r, a);
            free(r.d);
            r = t;
        }
    }
    return r;
}

/* Exported product tree over a list of 32-bit values. Returns the length;
 * writes at most cap limbs. */
uint64_t orc_product_tree(const uint32_t *v, uint64_t count, limb_t *out, uint64_t cap)
{
    big_t r = tree_u32(v, count);
    uint64_t n = r.n;
    memcpy(out, r.d, sizeof(limb_t) * (n < cap ? n : cap));
    free(r.d);
    return n;
}

/* Exported power a^e. Returns the length; writes at most cap limbs. */
uint64_t orc_pow(const limb_t *a, uint64_t na, uint64_t e, limb_t *out, uint64_t cap)
{
    big_t x; x.n = norm_len(a, na); x.d = malloc(sizeof(limb_t) * (x.n + 1));
    memcpy(x.d, a, sizeof(limb_t) * x.n);
    big_t r = big_pow(x, e);
    uint64_t n = r.n;
    memcpy(out, r.d, sizeof(limb_t) * (n < cap ? n : cap));
    free(r.d); free(x.d);
    return n;
}

/* Algorithm 2 on a grouped factorisation (CSR, as written by orc_group):
 * Q_e = tree(G_e), P_e = Q_e^e, result = tree(P).  Returns the length. */
uint64_t orc_reconstruct(uint64_t ngroups, const uint64_t *exps,
                         const uint64_t *offsets, const uint32_t *gprimes,
                         limb_t *out, uint64_t cap)
{
    big_t *P = malloc(sizeof(big_t) * (ngroups + 1));
    for (uint64_t g = 0; g < ngroups; g++) {
        big_t Q = tree_u32(gprimes + offsets[g], offsets[g + 1] - offsets[g]);
        P[g] = big_pow(Q, exps[g]);
        free(Q.d);
    }
    big_t C = tree_big(P, ngroups);
    for (uint64_t g = 0; g < ngroups; g++) free(P[g].d);
    free(P);
    uint64_t n = C.n;
    memcpy(out, C.d, sizeof(limb_t) * (n < cap ? n : cap));
    free(C.d);
    return n;
}

/* Algorithms 1 and 2 end to end for one kind.  Returns the normalised length
 * (writes at most cap limbs), or UINT64_MAX if some exponent is negative. */
uint64_t orc_exact(int kind, uint64_t n, limb_t *out, uint64_t cap)
{
    uint64_t lim = orc_prime_limit(kind, n);
    uint64_t np = orc_sieve(lim, NULL, 0);
    uint32_t *pr = malloc(sizeof(uint32_t) * (np + 1));
    orc_sieve(lim, pr, np);
    int64_t *e = malloc(sizeof(int64_t) * (np + 1));
    orc_exponents(kind, n, pr, np, e);
    for (uint64_t i = 0; i < np; i++)
        if (e[i] < 0) { free(pr); free(e); return UINT64_MAX; }
    /* distinct exponents never exceed the number of primes + 1 */
    uint64_t *exps = malloc(sizeof(uint64_t) * (np + 2));
    uint64_t *offs = malloc(sizeof(uint64_t) * (np + 2));
    uint32_t *gp = malloc(sizeof(uint32_t) * (np + 1));
    uint64_t ng = orc_group(pr, e, np, exps, offs, gp);
    uint64_t len = orc_reconstruct(ng, exps, offs, gp, out, cap);
    free(pr); free(e); free(exps); free(offs); free(gp);
    return len;
}

/* orc_exact run by `threads` threads: the same steps and the same code, with
 * the product tree's halves and the large Karatsuba sub-products executed as
 * OpenMP tasks (the integer is the same; only the schedule changes).  Used to
 * time the oracle on all host cores.  Without OpenMP it runs single-threaded. */
uint64_t orc_exact_mt(int kind, uint64_t n, limb_t *out, uint64_t cap, int threads)
{
    uint64_t len = 0;
    if (threads < 1) threads = 1;
#pragma omp parallel num_threads(threads)
#pragma omp single
    len = orc_exact(kind, n, out, cap);
    return len;
}

/* Threads orc_exact_mt can use: the processors OpenMP sees, or 1 without it. */
int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_num_procs();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Modular checks.                                                           */
/* ------------------------------------------------------------------------ */

/* Plain modular multiply through a 128-bit product (any q < 2^64). */
uint64_t orc_mulmod_plain(uint64_t a, uint64_t b, uint64_t q)
{
    return (uint64_t)(((u128)a * b) % q);
}

/* Montgomery multiplication (Montgomery 1985) with R = 2^64 for odd q < 2^63:
 * REDC(T) = (T + m q) / R, m = (T mod R) * (-q^-1) mod R, for T < q R.
 * The plain division-free form; pinned against orc_mulmod_plain. */
typedef struct { uint64_t q, qneg_inv, r2; } mont_t;

static mont_t mont_init(uint64_t q)
{
    mont_t m;
    m.q = q;
    uint64_t inv = 1; /* Newton iteration for q^-1 mod 2^64 */
    for (int i = 0; i < 7; i++) inv *= 2 - q * inv;
    m.qneg_inv = (uint64_t)0 - inv;
    u128 r = ((u128)1 << 64) % q;      /* R mod q   */
    m.r2 = (uint64_t)((r * r) % q);     /* R^2 mod q */
    return m;
}

static uint64_t redc(const mont_t *m, u128 t)
{
    uint64_t mm = (uint64_t)t * m->qneg_inv;
    u128 s = t + (u128)mm * m->q;
    uint64_t r = (uint64_t)(s >> 64);
    return r >= m->q ? r - m->q : r;
}

static uint64_t to_mont(const mont_t *m, uint64_t a) { return redc(m, (u128)(a % m->q) * m->r2); }
static uint64_t from_mont(const mont_t *m, uint64_t a) { return redc(m, a); }
static uint64_t mont_mul(const mont_t *m, uint64_t a, uint64_t b) { return redc(m, (u128)a * b); }

uint64_t orc_mulmod_mont(uint64_t a, uint64_t b, uint64_t q)
{
    mont_t m = mont_init(q);
    return from_mont(&m, mont_mul(&m, to_mont(&m, a), to_mont(&m, b)));
}

/* prod_{k=lo}^{hi} k mod q (1 when lo > hi), q odd < 2^63.  The factor k is
 * carried in Montgomery form and stepped by +1 each iteration. */
uint64_t orc_range_product_mod(uint64_t lo, uint64_t hi, uint64_t q)
{
    mont_t m = mont_init(q);
    uint64_t one = to_mont(&m, 1);
    uint64_t acc = one;
    if (lo > hi) return 1 % q;
    uint64_t km = to_mont(&m, lo);
    for (uint64_t k = lo;; k++) {
        acc = mont_mul(&m, acc, km);
        if (k == hi) break;
        km += one;
        if (km >= q) km -= q;
    }
    return from_mont(&m, acc);
}

static uint64_t powmod(uint64_t a, uint64_t e, uint64_t q)
{
    uint64_t r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = orc_mulmod_plain(r, a, q);
        a = orc_mulmod_plain(a, a, q);
        e >>= 1;
    }
    return r;
}

/* The exact quantity modulo a prime q, straight from its factorial
 * definition and with no sieve (Sec. 1):
 *   Catalan          C(n) = (2n)! / (n! (n+1)!) = [prod_{k=n+2}^{2n} k] / n!
 *   central binomial      = [prod_{k=n+1}^{2n} k] / n!
 *   factorial        n!   = prod_{k=1}^{n} k
 * For the binomial kinds q must be a prime > 2n so that n! is invertible.
 * Returns UINT64_MAX if q is too small for the kind. */
uint64_t orc_exact_mod(int kind, uint64_t n, uint64_t q)
{
    if (kind == ORC_FACTORIAL) return orc_range_product_mod(1, n, q);
    if (q <= 2 * n) return UINT64_MAX;
    uint64_t num = orc_range_product_mod(kind == ORC_CATALAN ? n + 2 : n + 1, 2 * n, q);
    uint64_t den = orc_range_product_mod(1, n, q);
    return orc_mulmod_plain(num, powmod(den, q - 2, q), q);
}

/* Limbs reduced modulo q by Horner's rule from the top limb:
 * r <- (r * 2^32 + limb) mod q. */
uint64_t orc_limbs_mod(const limb_t *a, uint64_t n, uint64_t q)
{
    mont_t m = mont_init(q);
    uint64_t base = to_mont(&m, (uint64_t)1 << 32);
    uint64_t r = 0; /* Montgomery form of 0 is 0 */
    for (uint64_t i = n; i-- > 0;) {
        r = mont_mul(&m, r, base);
        uint64_t l = to_mont(&m, a[i]);
        r += l;
        if (r >= q) r -= q;
    }
    return from_mont(&m, r);
}

/* Deterministic Miller-Rabin for 64-bit integers (bases 2..37 suffice
 * below 3.3e24).  Used to pick the check primes. */
int orc_is_prime(uint64_t x)
{
    if (x < 2) return 0;
    static const uint64_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (int i = 0; i < 12; i++) {
        if (x == small[i]) return 1;
        if (x % small[i] == 0) return 0;
    }
    uint64_t d = x - 1; int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        uint64_t y = powmod(small[i], d, x);
        if (y == 1 || y == x - 1) continue;
        int composite = 1;
        for (int r = 1; r < s; r++) {
            y = orc_mulmod_plain(y, y, x);
            if (y == x - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

/* Smallest prime >= x. */
uint64_t orc_next_prime(uint64_t x)
{
    if (x <= 2) return 2;
    if ((x & 1) == 0) x++;
    while (!orc_is_prime(x)) x += 2;
    return x;
}

/* ------------------------------------------------------------------------ */
/* Decimal text of a result (Sec. 3.2: the optional decimal output; Table 1: */
/* 1,234,567,890 digits at the paper's n).  The definition written out: the  */
/* digits are the remainders of repeated division by ten, taken here nine at */
/* a time (schoolbook long division of the limb array by 10^9, quadratic).   */
/* Writes the digits most significant first, no sign, no terminator, "0" for */
/* zero; returns the digit count, or UINT64_MAX when cap is too small.       */
uint64_t orc_to_decimal(const limb_t *a, uint64_t n, char *out, uint64_t cap)
{
    n = norm_len(a, n);
    if (n == 0) {
        if (cap < 1) return UINT64_MAX;
        out[0] = '0';
        return 1;
    }
    limb_t *w = (limb_t *)malloc(n * sizeof(limb_t));
    /* at most ceil(n * 32 / 29.89) + 1 chunks of nine digits */
    uint64_t maxch = (n * 32) / 29 + 2;
    uint32_t *ch = (uint32_t *)malloc(maxch * sizeof(uint32_t));
    memcpy(w, a, n * sizeof(limb_t));
    uint64_t len = n, nch = 0;
    while (len > 0) {
        uint64_t rem = 0; /* w = w / 10^9, rem = w mod 10^9 */
        for (uint64_t i = len; i-- > 0;) {
            uint64_t cur = (rem << 32) | w[i];
            w[i] = (limb_t)(cur / 1000000000u);
            rem = cur % 1000000000u;
        }
        ch[nch++] = (uint32_t)rem;
        while (len > 0 && w[len - 1] == 0) len--;
    }
    /* the top chunk without leading zeros, every other chunk as nine digits */
    char top[10];
    int lead = 0;
    for (uint32_t v = ch[nch - 1]; v; v /= 10) top[lead++] = (char)('0' + v % 10);
    uint64_t total = (uint64_t)lead + 9 * (nch - 1);
    if (total > cap) {
        free(w);
        free(ch);
        return UINT64_MAX;
    }
    uint64_t pos = 0;
    for (int i = lead - 1; i >= 0; i--) out[pos++] = top[i];
    for (uint64_t c = nch - 1; c-- > 0;) {
        uint32_t v = ch[c];
        for (int d = 8; d >= 0; d--) {
            out[pos + d] = (char)('0' + v % 10);
            v /= 10;
        }
        pos += 9;
    }
    free(w);
    free(ch);
    return total;
}
