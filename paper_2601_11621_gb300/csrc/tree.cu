// tree.cu -- Phase 2 of the method (Sec. 3.2, Algorithm 2): the balanced
// product tree, binary powering and the final product, as level-synchronous
// batched multiplications on the device.
//
// Product tree.  The leaves (32-bit primes) are combined eight at a time into
// 8-limb nodes; every further level multiplies adjacent nodes (2i, 2i+1) of a
// fixed slot size S into slots of 2S limbs (a product of 2^k values below 2^32
// always fits 2^k limbs), with an odd last node carried up unchanged.  All
// products of one level are one batched launch: schoolbook (Comba) kernels
// for small slots, a one-block transform for products up to 2^12 limbs, and
// the multi-pass transform above.  Nodes of a level hold equally many primes,
// which is what keeps the tree balanced.
#include "cat_internal.cuh"

#include <math.h>

#include <algorithm>
#include <vector>

namespace cat {

// comba.cu
void leaf_level(Ctx &c, const uint32_t *values, size_t count, uint32_t *out, size_t nodes,
                int lpn, cudaStream_t s);
// ntt.cu
void ntt_mul(Ctx &c, const uint32_t *a, size_t na, const uint32_t *b, size_t nb,
             uint32_t *out, cudaStream_t s);

constexpr size_t kLeafSlot = 8;

static Big make_one(Ctx &c, cudaStream_t s)
{
    Big r;
    r.buf = DevBuf<uint32_t>(c, 1, s);
    static const uint32_t one = 1;
    CAT_CUDA(cudaMemcpyAsync(r.buf.get(), &one, 4, cudaMemcpyHostToDevice, s));
    CAT_CUDA(cudaStreamSynchronize(s));
    r.n = 1;
    return r;
}

// Length of x[0..n) after dropping zero top limbs, reading only the top few
// limbs when they decide it.
size_t trim(Ctx &c, const uint32_t *x, size_t n, cudaStream_t s)
{
    if (n == 0) return 0;
    const size_t k = std::min<size_t>(n, 4);
    uint32_t local[4];
    uint32_t *h = c.host_word ? reinterpret_cast<uint32_t *>(c.host_word) : local;
    CAT_CUDA(cudaMemcpyAsync(h, x + n - k, 4 * k, cudaMemcpyDeviceToHost, s));
    CAT_CUDA(cudaStreamSynchronize(s));
    for (size_t i = k; i-- > 0;)
        if (h[i]) return n - k + i + 1;
    return normalized_length(c, x, n - k, s);
}

// Relative cost of a butterfly in the prime set of a 2^n-point transform
// (measured: set 1 ~1.1x and set 2 ~1.5x the lazy set 0).
static double set_cost(int n) { return n <= kLogSet0 ? 1.0 : (n <= kLogSet1 ? 1.1 : 1.5); }

static int clog2(size_t x)
{
    int n = 0;
    while (((size_t)1 << n) < x) n++;
    return n;
}

// For a long x and a short y: the chunk transform size 2^k whose estimated
// cost (transform points x log2 points x set cost, plus the overlap pass)
// beats one product of nx + ny limbs, or 0 if none does.
static int chunk_log(const Ctx &c, size_t nx, size_t ny)
{
    if (nx < 2 * ny || nx + ny <= 4096) return 0;
    const int nf = clog2(nx + ny);
    double best = nf <= c.max_log ? 3.0 * ldexp(1.0, nf) * nf * set_cost(nf) : 1e300;
    int bk = 0;
    for (int k = std::max(1, clog2(2 * ny)); k <= std::min(c.max_log, nf); k++) {
        const double L = ldexp(1.0, k), M = L - (double)ny;
        const double chunks = ceil((double)nx / M);
        const double cost = (2.0 * chunks + 1.0) * L * k * set_cost(k) + 4.0 * (double)(nx + ny);
        if (cost < best) {
            best = cost;
            bk = k;
        }
    }
    return bk;
}

void mul_into(Ctx &c, const uint32_t *a, size_t na, const uint32_t *b, size_t nb,
              uint32_t *out, cudaStream_t s)
{
    if (na == 0 || nb == 0) {
        if (na + nb) CAT_CUDA(cudaMemsetAsync(out, 0, 4 * (na + nb), s));
        return;
    }
    // unbalanced: chunks of the long operand against the short one
    {
        const bool swap = na < nb;
        const uint32_t *x = swap ? b : a, *y = swap ? a : b;
        const size_t nx = swap ? nb : na, ny = swap ? na : nb;
        if (const int k = chunk_log(c, nx, ny)) {
            mul_chunked(c, x, nx, y, ny, k, out, s);
            return;
        }
    }
    if (na + nb <= ((size_t)1 << c.max_log)) {
        ntt_mul(c, a, na, b, nb, out, s);
        return;
    }
    // longer than one transform: pieces of at most 2^26 limbs, accumulated
    CAT_CUDA(cudaMemsetAsync(out, 0, 4 * (na + nb), s));
    mul_acc(c, a, na, b, nb, out, na + nb, false, s);
}

static Big copy_big(Ctx &c, const uint32_t *a, size_t n, cudaStream_t s);
static Big mul_big(Ctx &c, const Big &x, const Big &y, cudaStream_t s, bool exact = true);

// Levels above the leaves of a tree over `count` values, lpn to a node.
static int tree_depth(size_t count, int lpn)
{
    size_t nodes = (count + lpn - 1) / lpn;
    int d = 0;
    for (; nodes > 1; d++) nodes = (nodes + 1) / 2;
    return d;
}

// The product of values[0 .. count) (times *extra when given).  extra joins
// the tree as one node: the count is padded with values 1 up to a multiple of
// a slot size S >= extra's length, plus S more, so that at slot S the last
// node is exactly 1 and extra takes its place.  Every node still fits its
// slot, so the levels above are unchanged; only when the padding would add a
// level is extra multiplied in at the end instead.  exact = false returns the
// top slot (zero-padded) as the length instead of reading the true length
// back: no host synchronisation.
Big tree_product(Ctx &c, const uint32_t *values, size_t count, cudaStream_t s, const Big *extra,
                 bool exact, int leaf_bits)
{
    NvtxRange range("product tree");
    if (count == 0) return extra ? copy_big(c, extra->buf.get(), extra->n, s) : make_one(c, s);
    const int lpn = leaves_per_node(leaf_bits);
    size_t total = count, inj_slot = 0;
    if (extra) {
        size_t S = 2 * kLeafSlot;
        while (S < extra->n) S <<= 1;
        const size_t per = S / kLeafSlot * (size_t)lpn;  // leaves under one node of slot S
        const size_t padded = (count + per - 1) / per * per + per;
        if (tree_depth(padded, lpn) == tree_depth(count, lpn)) {
            total = padded;
            inj_slot = S;
        }
    }
    size_t slot = kLeafSlot;
    size_t nodes = (total + lpn - 1) / lpn;
    DevBuf<uint32_t> cur(c, nodes * slot, s);
    leaf_level(c, values, count, cur.get(), nodes, lpn, s);
    while (nodes > 1) {
        NvtxRange level("tree level");
        const size_t nprod = nodes / 2, odd = nodes & 1, nn = nprod + odd, ns = 2 * slot;
        DevBuf<uint32_t> nxt(c, nn * ns, s);
        if (slot > c.comba_max_slot || !comba_level(c, cur.get(), slot, nprod, nxt.get(), s))
            ntt_level(c, cur.get(), slot, nprod, nxt.get(), s);
        if (odd) {
            CAT_CUDA(cudaMemcpyAsync(nxt.get() + nprod * ns, cur.get() + (nodes - 1) * slot,
                                     4 * slot, cudaMemcpyDeviceToDevice, s));
            CAT_CUDA(cudaMemsetAsync(nxt.get() + nprod * ns + slot, 0, 4 * slot, s));
        }
        if (ns == inj_slot) {  // the last node covers only padding: replace its 1 by extra
            uint32_t *last = nxt.get() + (nn - 1) * ns;
            CAT_CUDA(cudaMemcpyAsync(last, extra->buf.get(), 4 * extra->n,
                                     cudaMemcpyDeviceToDevice, s));
            if (extra->n < ns)
                CAT_CUDA(cudaMemsetAsync(last + extra->n, 0, 4 * (ns - extra->n), s));
            inj_slot = 0;
            extra = nullptr;
        }
        cur = std::move(nxt);
        nodes = nn;
        slot = ns;
    }
    Big r;
    r.n = exact ? normalized_length(c, cur.get(), slot, s) : slot;
    r.buf = std::move(cur);
    if (extra) return mul_big(c, r, *extra, s, exact);
    return r;
}

static Big copy_big(Ctx &c, const uint32_t *a, size_t n, cudaStream_t s)
{
    Big r;
    r.buf = DevBuf<uint32_t>(c, n ? n : 1, s);
    if (n) CAT_CUDA(cudaMemcpyAsync(r.buf.get(), a, 4 * n, cudaMemcpyDeviceToDevice, s));
    r.n = n;
    return r;
}

// x y; exact = false keeps the bound x.n + y.n as the length (zero top limbs)
// instead of reading the true length back.
static Big mul_big(Ctx &c, const Big &x, const Big &y, cudaStream_t s, bool exact)
{
    Big r;
    const size_t n = x.n + y.n;
    r.buf = DevBuf<uint32_t>(c, n ? n : 1, s);
    mul_into(c, x.buf.get(), x.n, y.buf.get(), y.n, r.buf.get(), s);
    r.n = exact ? trim(c, r.buf.get(), n, s) : n;
    return r;
}

// a^e, left-to-right binary (the powering step of Algorithm 2).  Squarings reuse
// one forward transform.  exact = false takes a (nonzero) as given, with zero
// top limbs allowed, and returns a bound as the length: no host
// synchronisation.
Big power(Ctx &c, const uint32_t *a, size_t na, uint64_t e, cudaStream_t s, bool exact)
{
    NvtxRange range("power");
    if (exact) na = normalized_length(c, a, na, s);
    if (e == 0) return make_one(c, s);
    if (na == 0) return copy_big(c, a, 0, s);
    Big base = copy_big(c, a, na, s);
    Big r = copy_big(c, a, na, s);
    int top = 63;
    while (!((e >> top) & 1)) top--;
    for (int bit = top - 1; bit >= 0; bit--) {
        r = mul_big(c, r, r, s, exact);
        if ((e >> bit) & 1) r = mul_big(c, r, base, s, exact);
    }
    return r;
}

// Factorisations with more exponent groups than this (n! has about 2 sqrt(n))
// take the bit-decomposed form below; Catalan numbers and central binomials
// (at most 33 groups) always take Algorithm 2 as written.
constexpr uint64_t kManyGroups = 64;

// prod_e Q_e^e = prod_b R_b^(2^b), R_b = prod of Q_e over the groups whose
// exponent has bit b set.  All R_b come from one segmented tree over the
// primes (segment b = the primes of those groups), then
// X = R_top; X = X^2 R_b for b below the top bit.  Same integer as
// Algorithm 2 with about 2 log2(max e) large multiplications instead of one
// powering chain per group.
static Big reconstruct_bits(Ctx &c, const cat_factorization *f, cudaStream_t s, int leaf_bits)
{
    uint64_t emax = 0;
    for (uint64_t g = 0; g < f->num_groups; g++) emax = std::max(emax, f->host_exps[g]);
    int B = 0;
    while (B < 64 && (emax >> B)) B++;
    std::vector<uint64_t> seg(B + 1, 0);
    for (uint64_t g = 0; g < f->num_groups; g++)
        for (int b = 0; b < B; b++)
            if ((f->host_exps[g] >> b) & 1)
                seg[b + 1] += f->host_offsets[g + 1] - f->host_offsets[g];
    for (int b = 0; b < B; b++) seg[b + 1] += seg[b];
    DevBuf<uint32_t> leaves(c, std::max<uint64_t>(seg[B], 1), s);
    std::vector<CopyJob> jobs;
    std::vector<uint64_t> at(seg.begin(), seg.end() - 1);
    for (uint64_t g = 0; g < f->num_groups; g++) {
        const uint64_t off = f->host_offsets[g], cnt = f->host_offsets[g + 1] - off;
        if (!cnt) continue;
        for (int b = 0; b < B; b++)
            if ((f->host_exps[g] >> b) & 1) {
                jobs.push_back(CopyJob{f->primes + off, leaves.get() + at[b], cnt, cnt});
                at[b] += cnt;
            }
    }
    run_copy_jobs(c, jobs, s);
    std::vector<TreeRoot> R(B);
    segmented_tree(c, leaves.get(), seg, R, s, leaf_bits);
    leaves.reset();
    for (int b = 0; b < B; b++) R[b].big.n = trim(c, R[b].big.buf.get(), R[b].big.n, s);
    Big X = std::move(R[B - 1].big);
    for (int b = B - 2; b >= 0; b--) {
        X = mul_big(c, X, X, s);
        if (seg[b + 1] > seg[b]) X = mul_big(c, X, R[b].big, s);
    }
    return X;
}

// Algorithm 2: Q_e by the tree, P_e = Q_e^e, then the P_e combined by
// repeatedly multiplying the two shortest (equal-length operands meet
// first, so intermediates stay as short as possible).
Big reconstruct(Ctx &c, const cat_factorization *f, cudaStream_t s, int leaf_bits)
{
    NvtxRange range("phase2: reconstruction");
    if (f->num_groups > kManyGroups) return reconstruct_bits(c, f, s, leaf_bits);
    // P_e = Q_e^e for e >= 2 first, combined into R; then Q_1's tree takes R
    // in as one of its nodes, so that the long P_1 needs no final product
    // (the same integer: the final product of the P_e, re-associated).  The
    // small P_e and R carry length bounds (zero top limbs), so that none of
    // their many short steps waits for a read-back; only the end result is
    // normalised.
    std::vector<Big> P;
    int64_t g1 = -1;
    for (uint64_t g = 0; g < f->num_groups; g++) {
        if (f->host_exps[g] == 1) {
            g1 = (int64_t)g;
            continue;
        }
        const uint64_t off = f->host_offsets[g], cnt = f->host_offsets[g + 1] - off;
        Big Q = tree_product(c, f->primes + off, cnt, s, nullptr, false, leaf_bits);
        P.push_back(power(c, Q.buf.get(), Q.n, f->host_exps[g], s, false));
    }
    while (P.size() > 1) {
        std::sort(P.begin(), P.end(), [](const Big &x, const Big &y) { return x.n > y.n; });
        Big x = std::move(P.back());
        P.pop_back();
        Big y = std::move(P.back());
        P.pop_back();
        P.push_back(mul_big(c, x, y, s, false));
    }
    if (g1 < 0) {
        if (P.empty()) return make_one(c, s);
        P[0].n = normalized_length(c, P[0].buf.get(), P[0].n, s);
        return std::move(P[0]);
    }
    const uint64_t off = f->host_offsets[g1], cnt = f->host_offsets[g1 + 1] - off;
    return tree_product(c, f->primes + off, cnt, s, P.empty() ? nullptr : &P[0], true, leaf_bits);
}

}  // namespace cat
