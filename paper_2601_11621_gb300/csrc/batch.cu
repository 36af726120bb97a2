// batch.cu -- many exact quantities computed together (uneven n, mixed kinds).
//
// Phase 1 (Sec. 3.1) once for the whole batch: one sieve up to the largest
// limit, then one thread per (request, prime) computes e_p (Sec. 2) and the
// primes of request r are written out e_p times each, request after request.
// Phase 2 (Sec. 3.2) as one segmented, level-synchronous product tree: every
// level of every request's tree is multiplied by the same batched launches
// (schoolbook, one-block transform or multi-pass transform, by slot size).
// A segment with an odd node count at some level gets a node of value 1
// appended, so adjacent pairs never straddle two requests.  The product over
// a request's primes, each repeated e_p times, is prod_e Q_e^e: the powers
// P_e = Q_e^e of Algorithm 2 are formed inside the tree rather than by
// separate square-and-multiply chains, which keeps the whole batch in a
// handful of launches per level.
#include "cat_internal.cuh"
#include "legendre.cuh"

#include <string.h>

#include <algorithm>
#include <vector>

namespace cat {

DevBuf<uint32_t> sieve_primes(Ctx &c, uint64_t limit, uint64_t *count, cudaStream_t s);
void exclusive_scan_u32(Ctx &c, uint32_t *data, size_t n, cudaStream_t s);

namespace {

constexpr int kBatchLeafSlot = 8;

// index r with pre[r] <= t < pre[r+1] (pre ascending, pre[0] = 0)
__device__ __forceinline__ int find_segment(const uint64_t *pre, int count, uint64_t t)
{
    int lo = 0, hi = count;  // pre[lo] <= t < pre[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// The segment of flat index t (< pre[count]) for a block of consecutive
// indices: one binary search per block (for its first index), then a short
// walk forward; a thread more than a few segments past the block's first one
// searches for itself.  Every thread of the block must call it.
__device__ __forceinline__ int block_segment(const uint64_t *pre, int count, uint64_t t)
{
    __shared__ int first;
    const uint64_t total = pre[count];
    if (threadIdx.x == 0) {
        const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x;
        first = t0 < total ? find_segment(pre, count, t0) : 0;
    }
    __syncthreads();
    if (t >= total) return 0;
    int r = first;
    for (int k = 0; k < 8 && pre[r + 1] <= t; k++) r++;
    if (pre[r + 1] <= t) r = find_segment(pre, count, t);
    return r;
}

// pi(limit_r) for each request: binary search in the ascending prime list
__global__ void count_primes_le(const uint32_t *primes, uint64_t np, const uint64_t *limits,
                                int count, uint64_t *out)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= count) return;
    uint64_t lo = 0, hi = np;  // first index with primes[i] > limit
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if ((uint64_t)primes[mid] <= limits[r]) lo = mid + 1; else hi = mid;
    }
    out[r] = lo;
}

struct ReqDev {
    uint32_t n;
    int kind;
};

// e_p for flat index t = (request r, prime index t - pre[r]); counts into e
__global__ void batch_exponents(const uint32_t *primes, const uint64_t *pre, int count,
                                const ReqDev *reqs, uint32_t *e, unsigned int *negative)
{
    const uint64_t total = pre[count];
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = block_segment(pre, count, t);
    if (t >= total) return;
    const uint32_t p = primes[t - pre[r]], n = reqs[r].n;
    const int kind = reqs[r].kind;
    // primes above sqrt(2n) of the binomial kinds: one division at most
    if (kind != CAT_FACTORIAL && (uint64_t)p * p > 2 * (uint64_t)n) {
        e[t] = unit_exponent(p, n, kind);
        return;
    }
    const int64_t v = exponent_of(p, n, kind);
    if (v < 0) atomicOr(negative, 1u);
    e[t] = v < 0 ? 0u : (uint32_t)v;
}

// after the scan: pos[t] = first leaf slot of flat index t, and the exponent
// of flat index t is pos[t + 1] - pos[t]; write p that many times
__global__ void batch_leaves(const uint32_t *primes, const uint64_t *pre, int count,
                             const uint32_t *pos, uint32_t *leaves)
{
    const uint64_t total = pre[count];
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = block_segment(pre, count, t);
    if (t >= total) return;
    uint32_t at = pos[t];
    const uint32_t end = pos[t + 1];
    if (at == end) return;
    const uint32_t p = primes[t - pre[r]];
    for (; at < end; at++) leaves[at] = p;
}

// leaf segment start of every request (flat index pre[r] -> its position
// after the scan; pos[pre[count]] is the total leaf count)
__global__ void batch_seg_starts(const uint64_t *pre, int count, const uint32_t *pos,
                                 uint64_t *seg)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r > count) return;
    seg[r] = (r < count && pre[r] < pre[count]) ? pos[pre[r]] : pos[pre[count]];
}

// node j of segment r = product of its leaves [lpn j, lpn j + lpn) (missing
// ones = 1; the caller picks lpn so that the product fits eight limbs),
// written to node dpos[r] + j of out
__global__ void batch_leaf_nodes(const uint32_t *leaves, const uint64_t *seg,
                                 const uint64_t *node_pre, const uint64_t *dpos, int count,
                                 int lpn, uint32_t *out)
{
    const uint64_t total = node_pre[count];
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int r = block_segment(node_pre, count, t);
    if (t >= total) return;
    const uint64_t first = seg[r] + (t - node_pre[r]) * (uint64_t)lpn, end = seg[r + 1];
    uint32_t acc[kBatchLeafSlot];
#pragma unroll
    for (int j = 0; j < kBatchLeafSlot; j++) acc[j] = j == 0;
    for (int k = 0; k < lpn; k++) {
        const uint32_t x = first + k < end ? leaves[first + k] : 1u;
        uint32_t carry = 0;
#pragma unroll
        for (int j = 0; j < kBatchLeafSlot; j++) {
            const uint64_t v = (uint64_t)acc[j] * x + carry;
            acc[j] = (uint32_t)v;
            carry = (uint32_t)(v >> 32);
        }
    }
#pragma unroll
    const uint64_t node = dpos[r] + (t - node_pre[r]);
#pragma unroll
    for (int j = 0; j < kBatchLeafSlot; j++) out[node * kBatchLeafSlot + j] = acc[j];
}

__global__ void batch_copy(const CopyJob *jobs, int njobs)
{
    for (int j = blockIdx.y; j < njobs; j += gridDim.y) {
        const CopyJob J = jobs[j];
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < J.cap;
             i += (uint64_t)gridDim.x * blockDim.x) {
            uint32_t v;
            if (!J.src)
                v = i == 0;
            else
                v = i < J.len ? J.src[i] : 0u;
            J.dst[i] = v;
        }
    }
}

// normalised length of each output region (one block per request, scanning
// down from the top)
__global__ void batch_lengths(const uint32_t *out, const uint64_t *off, const uint64_t *cap,
                              uint64_t *len)
{
    __shared__ unsigned long long best;
    const int r = blockIdx.x;
    if (threadIdx.x == 0) best = 0;
    __syncthreads();
    const uint32_t *o = out + off[r];
    const uint64_t n = cap[r];
    for (uint64_t top = n; top > 0 && best == 0;) {
        const uint64_t lo = top > blockDim.x ? top - blockDim.x : 0;
        const uint64_t i = lo + threadIdx.x;
        if (i < top && o[i]) atomicMax(&best, (unsigned long long)(i + 1));
        __syncthreads();
        top = lo;
    }
    if (threadIdx.x == 0) len[r] = best;
}

template <typename T>
DevBuf<T> upload(Ctx &c, const std::vector<T> &h, cudaStream_t s)
{
    DevBuf<T> d(c, h.size() ? h.size() : 1, s);
    if (!h.empty())
        CAT_CUDA(cudaMemcpyAsync(d.get(), h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice,
                                 s));
    return d;
}

}  // namespace

void run_copy_jobs(Ctx &c, const std::vector<CopyJob> &jobs, cudaStream_t s)
{
    if (jobs.empty()) return;
    DevBuf<CopyJob> d_jobs = upload(c, jobs, s);
    const int nj = (int)jobs.size();
    batch_copy<<<dim3(64, std::min(nj, 4096)), 256, 0, s>>>(d_jobs.get(), nj);
    CAT_LAUNCH("batch_copy");
    CAT_CUDA(cudaStreamSynchronize(s));
}

namespace {

// A copy job of the segmented tree, planned before the level buffers exist:
// offsets into the launch's source and destination levels (src == kOne
// writes the value 1; dst_abs, when set, replaces the destination level).
struct LevelJob {
    uint64_t src, dst;
    uint32_t *dst_abs;
    uint64_t len, cap;
};
constexpr uint64_t kOne = ~(uint64_t)0;

__global__ void batch_copy_level(const LevelJob *jobs, int njobs, const uint32_t *src_base,
                                 uint32_t *dst_base)
{
    for (int j = blockIdx.y; j < njobs; j += gridDim.y) {
        const LevelJob J = jobs[j];
        uint32_t *dst = J.dst_abs ? J.dst_abs : dst_base + J.dst;
        const uint32_t *src = J.src == kOne ? nullptr : src_base + J.src;
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < J.cap;
             i += (uint64_t)gridDim.x * blockDim.x)
            dst[i] = src ? (i < J.len ? src[i] : 0u) : (uint32_t)(i == 0);
    }
}

// Output nodes of all the tree's products, every level's products numbered
// one after another: run i covers products [rs[i], rs[i+1]) and sends them
// to nodes dst[i], dst[i] + 1, ... of their level's output.
__global__ void batch_level_index(const uint64_t *rs, const uint64_t *dst, int runs,
                                  uint32_t *index)
{
    const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= rs[runs]) return;
    const int i = find_segment(rs, runs, k);
    index[k] = (uint32_t)(dst[i] + (k - rs[i]));
}

}  // namespace

// The segmented level-synchronous product tree (see segmented_tree in
// cat_internal.cuh).  Level 0 multiplies eight leaves per node; every later
// level multiplies adjacent pairs of the whole level in one batched call.
//
// Every level's node counts follow from the segment lengths alone, so the
// whole schedule is planned on the host first and uploaded once; the levels
// then run back to back without waiting for the device.  A level's buffer
// holds the segments still multiplying, each padded to an even node count
// by a node of value 1, then the segments that are down to one node (their
// roots, copied out).  Each product is written straight to its node of the
// next level's buffer through an index table, so that no level is gathered
// or re-packed between products.
void segmented_tree(Ctx &c, const uint32_t *leaves, const std::vector<uint64_t> &seg,
                    std::vector<TreeRoot> &roots, cudaStream_t s, int leaf_bits)
{
    const size_t count = seg.size() - 1;
    const int nr = (int)count;
    // leaves per first-level node: their product stays below 2^(32 * 8)
    const int lpn = leaves_per_node(leaf_bits);
    struct Level {
        size_t slot;
        uint64_t padded, nodes;  // padded multiplying nodes; all nodes of the buffer
        size_t job0, njobs;      // pads and root copies of this level's buffer
        uint64_t maxcap;         // the longest of them (limbs), which sizes the launch
        uint64_t prod0;          // first product (all levels numbered in turn)
        size_t run0, nruns;      // runs of this level's products
    };
    std::vector<LevelJob> jobs;
    std::vector<Level> levels;
    std::vector<uint64_t> rs{0}, rdst;  // runs of products
    auto root_dst = [&](size_t r, uint64_t len, uint64_t &cap) -> uint32_t * {
        TreeRoot &t = roots[r];
        if (t.dst) {
            cap = t.cap;
            return t.dst;
        }
        const uint64_t n = std::max<uint64_t>(len, 1);
        t.big.buf = DevBuf<uint32_t>(c, n, s);
        t.big.n = n;
        cap = n;
        return t.big.buf.get();
    };
    // positions of a level's nodes: multiplying segments first, each padded
    // to an even count, then the one-node segments
    auto layout = [&](const std::vector<uint64_t> &cnt, std::vector<uint64_t> &pos,
                      uint64_t &padded, uint64_t &nodes) {
        uint64_t at = 0;
        for (size_t r = 0; r < count; r++)
            if (cnt[r] >= 2) {
                pos[r] = at;
                at += cnt[r] + (cnt[r] & 1);
            }
        padded = at;
        for (size_t r = 0; r < count; r++)
            if (cnt[r] == 1) pos[r] = at++;
        nodes = at;
    };
    std::vector<uint64_t> cnt(count), node_pre(count + 1, 0), pos(count, 0), nxt_cnt(count),
        nxt_pos(count, 0);
    for (size_t r = 0; r < count; r++) {
        cnt[r] = (seg[r + 1] - seg[r] + lpn - 1) / lpn;
        node_pre[r + 1] = node_pre[r] + cnt[r];
    }
    uint64_t padded = 0, nodes = 0, prod = 0;
    layout(cnt, pos, padded, nodes);
    const std::vector<uint64_t> pos0 = pos;
    const uint64_t nodes0 = nodes;
    for (size_t r = 0; r < count; r++)  // empty segments: the value 1
        if (seg[r + 1] == seg[r]) {
            uint64_t cap = 0;
            uint32_t *d = root_dst(r, 1, cap);
            jobs.push_back(LevelJob{kOne, 0, d, 1, cap});
        }
    for (size_t slot = kBatchLeafSlot;; slot *= 2) {
        Level lv{slot, padded, nodes, 0, 0, 0, prod, rs.size() - 1, 0};
        lv.job0 = levels.empty() ? 0 : jobs.size();
        for (size_t r = 0; r < count; r++) {
            if (cnt[r] >= 2 && (cnt[r] & 1))
                jobs.push_back(LevelJob{kOne, (pos[r] + cnt[r]) * slot, nullptr, 1, slot});
            if (cnt[r] == 1) {
                const uint64_t len = std::min<uint64_t>(slot, seg[r + 1] - seg[r]);
                uint64_t cap = 0;
                uint32_t *d = root_dst(r, len, cap);
                jobs.push_back(LevelJob{pos[r] * slot, 0, d, std::min(len, cap), cap});
            }
        }
        lv.njobs = jobs.size() - lv.job0;
        for (size_t j = lv.job0; j < jobs.size(); j++) lv.maxcap = std::max(lv.maxcap, jobs[j].cap);
        if (padded == 0) {
            levels.push_back(lv);
            break;
        }
        for (size_t r = 0; r < count; r++) nxt_cnt[r] = cnt[r] >= 2 ? (cnt[r] + 1) / 2 : 0;
        uint64_t npadded = 0, nnodes = 0;
        layout(nxt_cnt, nxt_pos, npadded, nnodes);
        for (size_t r = 0; r < count; r++)
            if (cnt[r] >= 2) {
                rs.push_back(rs.back() + nxt_cnt[r]);
                rdst.push_back(nxt_pos[r]);
            }
        lv.nruns = rs.size() - 1 - lv.run0;
        prod += padded / 2;
        levels.push_back(lv);
        cnt.swap(nxt_cnt);
        pos.swap(nxt_pos);
        padded = npadded;
        nodes = nnodes;
    }
    const uint64_t total_prod = prod;
    const int runs = (int)rdst.size();
    // one upload: segment starts, level-0 node offsets and positions, runs,
    // jobs
    std::vector<uint64_t> blob;
    auto put = [&](const std::vector<uint64_t> &v) {
        const size_t at = blob.size();
        blob.insert(blob.end(), v.begin(), v.end());
        return at;
    };
    const size_t at_seg = put(seg), at_np = put(node_pre), at_pos = put(pos0), at_rs = put(rs),
                 at_rd = put(rdst), at_jobs = blob.size();
    static_assert(sizeof(LevelJob) % sizeof(uint64_t) == 0, "LevelJob packs into words");
    blob.resize(at_jobs + jobs.size() * (sizeof(LevelJob) / sizeof(uint64_t)));
    if (!jobs.empty()) memcpy(blob.data() + at_jobs, jobs.data(), jobs.size() * sizeof(LevelJob));
    DevBuf<uint64_t> d_blob = upload(c, blob, s);
    const uint64_t *d = d_blob.get();
    const LevelJob *d_jobs = reinterpret_cast<const LevelJob *>(d + at_jobs);
    DevBuf<uint32_t> index(c, std::max<uint64_t>(total_prod, 1), s);
    if (total_prod) {
        batch_level_index<<<(unsigned)((total_prod + 255) / 256), 256, 0, s>>>(
            d + at_rs, d + at_rd, runs, index.get());
        CAT_LAUNCH("batch_level_index");
    }
    const uint64_t tn = node_pre[count];
    DevBuf<uint32_t> cur(c, std::max<uint64_t>(nodes0, 1) * kBatchLeafSlot, s);
    {
        const int tok = prof_begin(c, "batch_leaf_nodes", s);
        if (tn)
            batch_leaf_nodes<<<(unsigned)((tn + 255) / 256), 256, 0, s>>>(
                leaves, d + at_seg, d + at_np, d + at_pos, nr, lpn, cur.get());
        CAT_LAUNCH("batch_leaf_nodes");
        prof_end(c, tok, s, 4.0 * (double)(seg[count] - seg[0]) + 32.0 * (double)tn);
    }
    for (size_t li = 0; li < levels.size(); li++) {
        const Level &lv = levels[li];
        if (lv.njobs) {
            // blocks per job by the longest job (2,048 limbs a block), jobs
            // spread over the grid's second dimension
            const unsigned gx = (unsigned)std::min<uint64_t>(64, (lv.maxcap + 2047) / 2048);
            batch_copy_level<<<dim3(std::max(1u, gx), (unsigned)std::min<size_t>(lv.njobs, 65535)),
                               256, 0, s>>>(
                d_jobs + lv.job0, (int)lv.njobs, cur.get(), cur.get());
            CAT_LAUNCH("batch_copy_level");
        }
        if (lv.padded == 0) break;
        const size_t slot = lv.slot, nprod = lv.padded / 2, ns = 2 * slot;
        DevBuf<uint32_t> nxt(c, levels[li + 1].nodes * ns, s);
        const uint32_t *ix = index.get() + lv.prod0;
        if (slot > c.comba_max_slot || !comba_level(c, cur.get(), slot, nprod, nxt.get(), s, ix)) {
            std::vector<uint32_t> host_ix;
            if (ns > ((size_t)1 << c.max_log)) {  // products by pieces, placed from the host
                host_ix.resize(nprod);
                for (size_t i = lv.run0; i < lv.run0 + lv.nruns; i++)
                    for (uint64_t k = rs[i]; k < rs[i + 1]; k++)
                        host_ix[k - lv.prod0] = (uint32_t)(rdst[i] + (k - rs[i]));
            }
            ntt_level(c, cur.get(), slot, nprod, nxt.get(), s, ix,
                      host_ix.empty() ? nullptr : host_ix.data());
        }
        cur = std::move(nxt);
    }
}

// Batched Phase 1 + Phase 2 for requests whose exponents are small (every
// prime written e_p times); request r's result goes to out + offsets[r]
// (room for bound_limbs limbs), its normalised length to lengths[r].
static void batch_core(Ctx &c, const cat_request *reqs, size_t count, uint32_t *out,
                       const uint64_t *offsets, uint64_t *lengths, cudaStream_t s)
{
    if (count == 0) return;
    std::vector<uint64_t> limits(count), caps(count);
    std::vector<ReqDev> rd(count);
    uint64_t M = 0;
    for (size_t r = 0; r < count; r++) {
        rd[r] = ReqDev{(uint32_t)reqs[r].n, reqs[r].kind};
        limits[r] = reqs[r].kind == CAT_FACTORIAL ? reqs[r].n : 2 * reqs[r].n;
        M = std::max(M, limits[r]);
        caps[r] = bound_limbs(reqs[r].n, reqs[r].kind);
    }
    const int nr = (int)count;
    // ---- Phase 1: shared sieve, exponents, leaves
    uint64_t np = 0;
    DevBuf<uint32_t> primes = sieve_primes(c, std::max<uint64_t>(M, 2), &np, s);
    DevBuf<uint64_t> d_limits = upload(c, limits, s);
    DevBuf<uint64_t> d_pi(c, count, s);
    count_primes_le<<<(nr + 255) / 256, 256, 0, s>>>(primes.get(), np, d_limits.get(), nr,
                                                     d_pi.get());
    CAT_LAUNCH("count_primes_le");
    std::vector<uint64_t> pi(count), pre(count + 1, 0);
    CAT_CUDA(cudaMemcpyAsync(pi.data(), d_pi.get(), 8 * count, cudaMemcpyDeviceToHost, s));
    CAT_CUDA(cudaStreamSynchronize(s));
    for (size_t r = 0; r < count; r++) pre[r + 1] = pre[r] + pi[r];
    const uint64_t F = pre[count];
    if (F >= (1ull << 32)) fail(CAT_EINVAL, "batch too large");
    DevBuf<uint64_t> d_pre = upload(c, pre, s);
    DevBuf<ReqDev> d_req = upload(c, rd, s);
    DevBuf<uint32_t> pos(c, F + 1, s);
    DevBuf<unsigned int> neg(c, 1, s);
    CAT_CUDA(cudaMemsetAsync(neg.get(), 0, 4, s));
    CAT_CUDA(cudaMemsetAsync(pos.get() + F, 0, 4, s));
    const unsigned fb = (unsigned)((F + 255) / 256);
    int tok = prof_begin(c, "batch_exponents", s);
    if (F) batch_exponents<<<fb, 256, 0, s>>>(primes.get(), d_pre.get(), nr, d_req.get(),
                                              pos.get(), neg.get());
    CAT_LAUNCH("batch_exponents");
    prof_end(c, tok, s, 8.0 * (double)F);
    // exclusive scan over F + 1 entries: pos[F] becomes the total leaf count
    exclusive_scan_u32(c, pos.get(), F + 1, s);
    // the segment starts (the last one the total leaf count) and the sign
    // flag in one read-back
    DevBuf<uint64_t> d_seg(c, count + 1, s);
    batch_seg_starts<<<(nr + 256) / 256, 256, 0, s>>>(d_pre.get(), nr, pos.get(), d_seg.get());
    CAT_LAUNCH("batch_seg_starts");
    std::vector<uint64_t> seg(count + 1);
    unsigned int hneg = 0;
    CAT_CUDA(cudaMemcpyAsync(seg.data(), d_seg.get(), 8 * (count + 1), cudaMemcpyDeviceToHost, s));
    CAT_CUDA(cudaMemcpyAsync(&hneg, neg.get(), 4, cudaMemcpyDeviceToHost, s));
    CAT_CUDA(cudaStreamSynchronize(s));
    if (hneg) fail(CAT_ENOTINTEGRAL, "a prime exponent is negative");
    const uint32_t total_leaves = (uint32_t)seg[count];
    DevBuf<uint32_t> leaves(c, total_leaves ? total_leaves : 1, s);
    tok = prof_begin(c, "batch_leaves", s);
    if (F) batch_leaves<<<fb, 256, 0, s>>>(primes.get(), d_pre.get(), nr, pos.get(),
                                           leaves.get());
    CAT_LAUNCH("batch_leaves");
    prof_end(c, tok, s, 8.0 * (double)F + 4.0 * total_leaves);
    primes.reset();
    pos.reset();

    // ---- Phase 2: one segmented tree over all requests
    std::vector<TreeRoot> roots(count);
    for (size_t r = 0; r < count; r++) {
        roots[r].dst = out + offsets[r];
        roots[r].cap = caps[r];
    }
    segmented_tree(c, leaves.get(), seg, roots, s, bits_below(M));  // leaves: primes <= M
    leaves.reset();
    // ---- lengths
    DevBuf<uint64_t> d_off = upload(c, std::vector<uint64_t>(offsets, offsets + count), s);
    DevBuf<uint64_t> d_cap = upload(c, caps, s);
    DevBuf<uint64_t> d_len(c, count, s);
    batch_lengths<<<nr, 256, 0, s>>>(out, d_off.get(), d_cap.get(), d_len.get());
    CAT_LAUNCH("batch_lengths");
    CAT_CUDA(cudaMemcpyAsync(lengths, d_len.get(), 8 * count, cudaMemcpyDeviceToHost, s));
    CAT_CUDA(cudaStreamSynchronize(s));
}

// Factorials beyond this n have exponents far above 1 (v_2(n!) ~ n), so
// writing every prime e_p times would blow up the tree; they are computed one
// by one through the grouped path instead.
constexpr uint64_t kBatchFactorialMax = 64;

// out: the results back to back, request r at offsets[r] with room for
// bound_limbs(n_r, kind_r) limbs; lengths[r] = normalised length.
void exact_batch(Ctx &c, const cat_request *reqs, size_t count, uint32_t *out, size_t cap,
                 uint64_t *offsets, uint64_t *lengths, cudaStream_t s)
{
    NvtxRange range("batch");
    if (count == 0) return;
    uint64_t total_cap = 0;
    for (size_t r = 0; r < count; r++) {
        if (reqs[r].n >= (1ull << 31)) fail(CAT_EINVAL, "n must be below 2^31");
        if (reqs[r].kind < CAT_CATALAN || reqs[r].kind > CAT_FACTORIAL)
            fail(CAT_EINVAL, "unknown kind");
        offsets[r] = total_cap;
        total_cap += bound_limbs(reqs[r].n, reqs[r].kind);
    }
    if (total_cap > cap) {
        lengths[0] = total_cap;
        fail(CAT_ERANGE, "output capacity too small for the batch");
    }
    std::vector<cat_request> small;
    std::vector<uint64_t> small_off, small_len;
    std::vector<size_t> small_idx, single_idx;
    for (size_t r = 0; r < count; r++) {
        if (reqs[r].kind == CAT_FACTORIAL && reqs[r].n >= kBatchFactorialMax) {
            single_idx.push_back(r);
        } else {
            small_idx.push_back(r);
            small.push_back(reqs[r]);
            small_off.push_back(offsets[r]);
        }
    }
    small_len.resize(small.size());
    batch_core(c, small.data(), small.size(), out, small_off.data(), small_len.data(), s);
    for (size_t i = 0; i < small_idx.size(); i++) lengths[small_idx[i]] = small_len[i];
    for (size_t r : single_idx) {
        cat_factorization f{};
        factor(c, reqs[r].n, reqs[r].kind, &f, s);
        Big v;
        try {
            v = reconstruct(c, &f, s, bits_below(reqs[r].n));  // primes <= n
        } catch (...) {
            factor_free(c, &f);
            throw;
        }
        factor_free(c, &f);
        const uint64_t capr = bound_limbs(reqs[r].n, reqs[r].kind);
        if (v.n > capr) fail(CAT_ERANGE, "result longer than its bound");
        run_copy_jobs(c, {CopyJob{v.buf.get(), out + offsets[r], v.n, capr}}, s);
        lengths[r] = v.n;
    }
}

size_t batch_bound(const cat_request *reqs, size_t count)
{
    size_t t = 0;
    for (size_t r = 0; r < count; r++) t += bound_limbs(reqs[r].n, reqs[r].kind);
    return t;
}

}  // namespace cat
