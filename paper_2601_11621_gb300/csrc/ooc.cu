// ooc.cu -- Phase 2 within a device budget smaller than its in-core peak.
//
// The paper keeps its memory bounded by multiplying the primes in chunks
// (about 10^5 at a time) and by keeping partial products outside the working
// set (Sec. 3.2, Algorithm 2 and its remarks on chunking; Sec. 6.2 on memory).
// This file is that mode for a context whose HBM budget cannot hold the
// in-core reconstruction (level arrays plus the three-prime transforms of a
// whole tree level, ~120 bytes per result limb):
//   - the grouped primes move to pinned host memory;
//   - each group's primes are multiplied in chunks of K consecutive primes,
//     every chunk by the device product tree, its root copied to pinned host
//     memory (K sized to the budget);
//   - the chunk roots, the powers Q_e^e and the final product are combined
//     by balanced trees whose operands live in host memory: a product whose
//     operands, result and transform scratch fit the budget runs as one
//     device multiplication; a larger one runs by pieces of M limbs (M sized
//     to the budget), the piece products added into a sliding window of
//     2M + 2 limbs on the device, whose low M limbs are final and copied back
//     after every output block.
// Every step is exact, so the integer equals the in-core result.
#include "cat_internal.cuh"

#include <algorithm>
#include <vector>

namespace cat {

namespace {

// A big integer in pinned host memory (n limbs, normalised).
struct HostBig {
    uint32_t *p = nullptr;
    size_t n = 0;
    HostBig() = default;
    explicit HostBig(size_t cap)
    {
        if (cap) CAT_CUDA(cudaMallocHost(&p, 4 * cap));
    }
    HostBig(const HostBig &) = delete;
    HostBig &operator=(const HostBig &) = delete;
    HostBig(HostBig &&o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    HostBig &operator=(HostBig &&o) noexcept
    {
        if (this != &o) {
            if (p) cudaFreeHost(p);
            p = o.p;
            n = o.n;
            o.p = nullptr;
            o.n = 0;
        }
        return *this;
    }
    ~HostBig()
    {
        if (p) cudaFreeHost(p);
    }
};

constexpr size_t kMargin = 256u << 10;  // bytes kept free for small scratch

size_t avail(const Ctx &c)
{
    if (!c.budget) return ~(size_t)0 >> 1;
    return c.budget > c.in_use + kMargin ? c.budget - c.in_use - kMargin : 0;
}

size_t pow2_floor(size_t x)
{
    size_t p = 1;
    while (p <= x / 2) p <<= 1;
    return x ? p : 0;
}

size_t pow2_ceil(size_t x)
{
    size_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Device bytes one in-core product of na + nb limbs holds at its peak: both
// operands, the product, and the transform scratch (three residues of two
// operands and of the product per point, 36 bytes, for the transform of the
// product's length or of the longest piece), with headroom.
size_t mul_need(const Ctx &c, size_t na, size_t nb)
{
    const size_t n = na + nb;
    const size_t L = std::min(pow2_ceil(n), (size_t)1 << c.max_log);
    return 8 * n + 48 * L + (64u << 10);
}

HostBig to_host(Ctx &c, const uint32_t *dev, size_t n, cudaStream_t s)
{
    const size_t len = normalized_length(c, dev, n, s);
    HostBig h(len ? len : 1);
    h.n = len;
    if (len) CAT_CUDA(cudaMemcpyAsync(h.p, dev, 4 * len, cudaMemcpyDeviceToHost, s));
    CAT_CUDA(cudaStreamSynchronize(s));
    return h;
}

HostBig host_one()
{
    HostBig h(1);
    h.p[0] = 1;
    h.n = 1;
    return h;
}

// a * b for host operands, by pieces of M limbs: piece products A_i B_j for
// i + j = s are added into a device window holding limbs [sM, sM + 2M + 2) of
// the sum (2M + 2 limbs always hold it: the pending sum is below (pieces + 1)
// 2^(64 M)); after step s the window's low M limbs are final (no later piece
// product reaches below (s + 1) M), go back to the host, and the window
// shifts down by M limbs into the other buffer.
HostBig mul_pieces(Ctx &c, const HostBig &a, const HostBig &b, cudaStream_t s)
{
    size_t M = pow2_floor(avail(c) / 112);
    M = std::min(M, (size_t)1 << (c.max_log - 1));
    if (M < 1024) fail(CAT_ENOMEM, "HBM budget too small for a product by pieces");
    const size_t na = a.n, nb = b.n, nA = (na + M - 1) / M, nB = (nb + M - 1) / M;
    const size_t total = na + nb, W = 2 * M + 2;
    HostBig r(total);
    DevBuf<uint32_t> Ai(c, M, s), Bj(c, M, s), P(c, 2 * M, s), W0(c, W, s), W1(c, W, s);
    uint32_t *win = W0.get(), *nxt = W1.get();
    CAT_CUDA(cudaMemsetAsync(win, 0, 4 * W, s));
    size_t done = 0;  // limbs of r written
    for (size_t st = 0; st + 1 < nA + nB; st++) {
        const size_t i0 = st >= nB ? st - nB + 1 : 0, i1 = std::min(st, nA - 1);
        for (size_t i = i0; i <= i1; i++) {
            const size_t j = st - i;
            const size_t li = std::min(M, na - i * M), lj = std::min(M, nb - j * M);
            CAT_CUDA(cudaMemcpyAsync(Ai.get(), a.p + i * M, 4 * li, cudaMemcpyHostToDevice, s));
            CAT_CUDA(cudaMemcpyAsync(Bj.get(), b.p + j * M, 4 * lj, cudaMemcpyHostToDevice, s));
            mul_into(c, Ai.get(), li, Bj.get(), lj, P.get(), s);
            add_into(c, win, W, P.get(), li + lj, false, s);
        }
        const size_t take = std::min(M, total - done);
        CAT_CUDA(cudaMemcpyAsync(r.p + done, win, 4 * take, cudaMemcpyDeviceToHost, s));
        done += take;
        CAT_CUDA(cudaMemcpyAsync(nxt, win + M, 4 * (M + 2), cudaMemcpyDeviceToDevice, s));
        CAT_CUDA(cudaMemsetAsync(nxt + M + 2, 0, 4 * (W - M - 2), s));
        std::swap(win, nxt);
        // keep the host copies of the pieces alive until their transfers ran
        CAT_CUDA(cudaStreamSynchronize(s));
    }
    if (done < total)
        CAT_CUDA(cudaMemcpyAsync(r.p + done, win, 4 * std::min(W, total - done),
                                 cudaMemcpyDeviceToHost, s));
    CAT_CUDA(cudaStreamSynchronize(s));
    size_t n = total;
    while (n && r.p[n - 1] == 0) n--;
    r.n = n;
    return r;
}

// a * b for host operands: one device multiplication when it fits the
// budget, else by pieces.
HostBig mul_host(Ctx &c, const HostBig &a, const HostBig &b, cudaStream_t s)
{
    if (!a.n || !b.n) return HostBig();
    if (mul_need(c, a.n, b.n) > avail(c)) return mul_pieces(c, a, b, s);
    const size_t n = a.n + b.n;
    DevBuf<uint32_t> da(c, a.n, s), db(c, b.n, s), dr(c, n, s);
    CAT_CUDA(cudaMemcpyAsync(da.get(), a.p, 4 * a.n, cudaMemcpyHostToDevice, s));
    CAT_CUDA(cudaMemcpyAsync(db.get(), b.p, 4 * b.n, cudaMemcpyHostToDevice, s));
    mul_into(c, da.get(), a.n, db.get(), b.n, dr.get(), s);
    da.reset();
    db.reset();
    return to_host(c, dr.get(), n, s);
}

// Balanced product of host values (Sec. 3.2), adjacent pairs level by level.
HostBig tree_host(Ctx &c, std::vector<HostBig> v, cudaStream_t s)
{
    if (v.empty()) return host_one();
    while (v.size() > 1) {
        std::vector<HostBig> nx;
        for (size_t i = 0; i + 1 < v.size(); i += 2) nx.push_back(mul_host(c, v[i], v[i + 1], s));
        if (v.size() & 1) nx.push_back(std::move(v.back()));
        v = std::move(nx);
    }
    return std::move(v[0]);
}

// The product of count 32-bit values in host memory: chunks of K values, each
// by the device product tree (its root to the host), then a balanced tree
// over the chunk roots.  The tree of K values holds about 8 K bytes of level
// arrays and 36 K bytes of transform scratch at its top level; K is the
// largest power of two that fits 80 K bytes into the budget.
HostBig chunk_product(Ctx &c, const uint32_t *vals, size_t count, cudaStream_t s)
{
    if (count == 0) return host_one();
    size_t K = pow2_floor(avail(c) / 80);
    if (K < 64) fail(CAT_ENOMEM, "HBM budget too small for chunked products");
    std::vector<HostBig> roots;
    for (size_t off = 0; off < count; off += K) {
        const size_t k = std::min(K, count - off);
        Big r;
        {
            DevBuf<uint32_t> dv(c, k, s);
            CAT_CUDA(cudaMemcpyAsync(dv.get(), vals + off, 4 * k, cudaMemcpyHostToDevice, s));
            r = tree_product(c, dv.get(), k, s, nullptr, false);
        }
        roots.push_back(to_host(c, r.buf.get(), r.n, s));
    }
    return tree_host(c, std::move(roots), s);
}

// a^e by left-to-right binary powering (Algorithm 2's powering step).
HostBig power_host(Ctx &c, HostBig a, uint64_t e, cudaStream_t s)
{
    if (e == 0) return host_one();
    if (e == 1 || a.n == 0) return a;
    int top = 63;
    while (!((e >> top) & 1)) top--;
    HostBig r = mul_host(c, a, a, s);
    if ((e >> (top - 1)) & 1) r = mul_host(c, r, a, s);
    for (int bit = top - 2; bit >= 0; bit--) {
        r = mul_host(c, r, r, s);
        if ((e >> bit) & 1) r = mul_host(c, r, a, s);
    }
    return r;
}

}  // namespace

// Upper bound on the device bytes of the in-core reconstruction of f: about
// 120 bytes per result limb (measured), and a result of at most
// sum_g e_g |G_g| limbs (every prime is below 2^32).
size_t reconstruct_need(const cat_factorization *f)
{
    double limbs = 0;
    for (uint64_t g = 0; g < f->num_groups; g++)
        limbs += (double)f->host_exps[g] * (double)(f->host_offsets[g + 1] - f->host_offsets[g]);
    return (size_t)(128.0 * limbs) + (4u << 20);
}

bool reconstruct_out_of_core(const Ctx &c, const cat_factorization *f)
{
    return c.budget && reconstruct_need(f) > avail(c);
}

// Algorithm 2 within the context's budget: the grouped primes go to pinned
// host memory (the device factorisation is released when it belongs to this
// call), Q_e = product of G_e by chunks, P_e = Q_e^e, C = balanced product of
// the P_e.  The result is copied to `out` (device memory, or host memory with
// to_host), cap limbs.
void reconstruct_into(Ctx &c, cat_factorization *f, uint32_t *out, size_t cap, bool to_host_out,
                      size_t *out_len, cudaStream_t s, bool release)
{
    NvtxRange range("phase2: reconstruction by chunks");
    const uint64_t ng = f->num_groups, np = f->num_primes;
    std::vector<uint64_t> exps(f->host_exps, f->host_exps + ng);
    std::vector<uint64_t> offs(f->host_offsets, f->host_offsets + ng + 1);
    HostBig primes(np ? np : 1);
    if (np)
        CAT_CUDA(cudaMemcpyAsync(primes.p, f->primes, 4 * np, cudaMemcpyDeviceToHost, s));
    CAT_CUDA(cudaStreamSynchronize(s));
    if (release) factor_free(c, f);
    std::vector<HostBig> P;
    for (uint64_t g = 0; g < ng; g++) {
        HostBig Q = chunk_product(c, primes.p + offs[g], offs[g + 1] - offs[g], s);
        P.push_back(power_host(c, std::move(Q), exps[g], s));
    }
    HostBig r = tree_host(c, std::move(P), s);
    *out_len = r.n;
    if (r.n > cap) fail(CAT_ERANGE, "output capacity too small");
    if (r.n)
        CAT_CUDA(cudaMemcpyAsync(out, r.p, 4 * r.n,
                                 to_host_out ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice, s));
    CAT_CUDA(cudaStreamSynchronize(s));
}

}  // namespace cat
