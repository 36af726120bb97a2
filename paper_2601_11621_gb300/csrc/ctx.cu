// ctx.cu -- context, error plumbing, the stream-ordered scratch pool and the
// NTT twiddle tables.
#include "cat_internal.cuh"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <string>
#include <vector>

namespace cat {

void fail(int code, const std::string &msg) { throw Error{code, msg}; }

void check_cuda(cudaError_t e, const char *what)
{
    if (e != cudaSuccess) {
        std::string m = std::string(what) + ": " + cudaGetErrorString(e);
        if (e == cudaErrorMemoryAllocation) fail(CAT_ENOMEM, m);
        fail(CAT_ECUDA, m);
    }
}

// kernels launched by this library in this process
static std::atomic<unsigned long long> g_launches{0};

void launched(const char *what)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    check_cuda(cudaGetLastError(), what);
}

unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

// ------------------------------------------------------------------ memory

namespace {
struct PoolHolder {
    cudaMemPool_t pool = nullptr;
};
}  // namespace

static cudaMemPool_t g_pools[64] = {};

static cudaMemPool_t pool_for(int device)
{
    if (device < 0 || device >= 64) fail(CAT_EINVAL, "device index out of range");
    if (!g_pools[device]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t p;
        CAT_CUDA(cudaMemPoolCreate(&p, &props));
        uint64_t thr = UINT64_MAX;  // keep freed blocks cached in the pool
        CAT_CUDA(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr));
        g_pools[device] = p;
    }
    return g_pools[device];
}

void *dev_alloc(Ctx &c, size_t bytes, cudaStream_t s)
{
    if (bytes == 0) return nullptr;
    bytes = (bytes + 255) & ~(size_t)255;
    if (c.budget && c.in_use + bytes > c.budget)
        fail(CAT_ENOMEM, "scratch would exceed the context's HBM budget (" +
                             std::to_string(c.in_use + bytes) + " > " +
                             std::to_string(c.budget) + " bytes)");
    if (c.shared_in_use) {
        const size_t before = c.shared_in_use->fetch_add(bytes);
        if (c.shared_budget && before + bytes > c.shared_budget) {
            c.shared_in_use->fetch_sub(bytes);
            fail(CAT_ENOMEM, "scratch would exceed the shared HBM budget (" +
                                 std::to_string(before + bytes) + " > " +
                                 std::to_string(c.shared_budget) + " bytes)");
        }
        if (c.shared_peak) {
            size_t pk = c.shared_peak->load();
            while (before + bytes > pk && !c.shared_peak->compare_exchange_weak(pk, before + bytes)) {
            }
        }
    }
    void *p = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, pool_for(c.device), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (c.shared_in_use) c.shared_in_use->fetch_sub(bytes);
        fail(CAT_ENOMEM, "device allocation of " + std::to_string(bytes) +
                             " bytes failed: " + cudaGetErrorString(e));
    }
    c.in_use += bytes;
    if (c.in_use > c.peak) c.peak = c.in_use;
    return p;
}

void dev_free(Ctx &c, void *p, size_t bytes, cudaStream_t s)
{
    if (!p) return;
    bytes = (bytes + 255) & ~(size_t)255;
    cudaFreeAsync(p, s);
    c.in_use -= bytes;
    if (c.shared_in_use) c.shared_in_use->fetch_sub(bytes);
}

// --------------------------------------------------------------- profiler

static cudaEvent_t take_event(Ctx &c)
{
    if (!c.event_pool.empty()) {
        cudaEvent_t e = c.event_pool.back();
        c.event_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    CAT_CUDA(cudaEventCreate(&e));
    return e;
}

int prof_begin(Ctx &c, const char *name, cudaStream_t s)
{
    if (!c.profiling) return -1;
    int idx = -1;
    for (size_t i = 0; i < c.prof.size(); i++)
        if (c.prof[i].name == name) { idx = (int)i; break; }
    if (idx < 0) {
        c.prof.push_back(ProfEntry{name, 0, 0.0, 0.0, 0.0});
        idx = (int)c.prof.size() - 1;
    }
    ProfPending p{idx, take_event(c), take_event(c), 0.0, 0.0};
    CAT_CUDA(cudaEventRecord(p.a, s));
    c.pending.push_back(p);
    return (int)c.pending.size() - 1;
}

void prof_end(Ctx &c, int token, cudaStream_t s, double bytes, double unit_bytes)
{
    if (token < 0) return;
    ProfPending &p = c.pending[token];
    p.bytes = bytes;
    p.unit_bytes = unit_bytes;
    CAT_CUDA(cudaEventRecord(p.b, s));
}

void prof_resolve(Ctx &c)
{
    for (ProfPending &p : c.pending) {
        cudaEventSynchronize(p.b);
        float ms = 0;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            ProfEntry &e = c.prof[p.idx];
            e.launches++;
            e.ms += ms;
            e.bytes += p.bytes;
            e.unit_bytes += p.unit_bytes;
        }
        c.event_pool.push_back(p.a);
        c.event_pool.push_back(p.b);
    }
    c.pending.clear();
    cudaGetLastError();
}

// --------------------------------------------------------------- twiddles

static uint32_t find_generator(uint32_t q)
{
    std::vector<uint64_t> f;
    uint64_t m = q - 1;
    for (uint64_t d = 2; d * d <= m; d++) {
        if (m % d == 0) {
            f.push_back(d);
            while (m % d == 0) m /= d;
        }
    }
    if (m > 1) f.push_back(m);
    for (uint32_t g = 2;; g++) {
        bool ok = true;
        for (uint64_t d : f)
            if (powmod_u32(g, (q - 1) / d, q) == 1) { ok = false; break; }
        if (ok) return g;
    }
}

// Powers f, f s, f s^2, ... (count of them) of `step` into T as multiplier
// pairs: (x, floor(x 2^32 / q)) in Shoup's form, else (x 2^32 mod q, that
// times q^-1 mod 2^32) in Montgomery's.
static void fill_powers(uint2 *T, int count, uint32_t step, uint32_t q, bool shoup,
                        uint32_t first = 1)
{
    const uint32_t qi = inv32(q);
    uint64_t x = first % q;
    for (int j = 0; j < count; j++) {
        if (shoup) {
            T[j] = make_uint2((uint32_t)x, shoup_c((uint32_t)x, q));
        } else {
            const uint32_t m = to_mont_c(x, q);
            T[j] = make_uint2(m, m * qi);
        }
        x = x * step % q;
    }
}

// Table layout per (set, prime i, direction d), w the primitive 2^L-th root
// of unity of the set (L = set_log_root) (d = 0) or its inverse (d = 1): see
// kTwStage / kTwSmall.
void twiddle_tables_host(uint2 *h)
{
    for (int set = 0; set < kNumSets; set++)
    for (int i = 0; i < kNumPrimes; i++) {
        const int L = set_log_root(set);
        const bool sh = set_shoup(set);
        const uint32_t q = ntt_prime(set, i);
        if ((q - 1) % (1u << L)) fail(CAT_ECUDA, "prime without the needed roots of unity");
        const uint32_t w = powmod_u32(find_generator(q), (q - 1) >> L, q);
        if (powmod_u32(w, 1u << (L - 1), q) != q - 1)
            fail(CAT_ECUDA, "twiddle root check failed");
        for (int d = 0; d < 2; d++) {
            const uint32_t root = d == 0 ? w : powmod_u32(w, (1u << L) - 1, q);
            uint2 *T = h + (((size_t)set * kNumPrimes + i) * 2 + d) * kTwPerDir;
            // stage s (half-span 2^s, s < 13): w_{2^(s+1)}^j at 2^s + j, j < 2^s
            fill_powers(T, 1, 1, q, sh);
            for (int st = 0; st < 13; st++)
                fill_powers(T + (1 << st), 1 << st, powmod_u32(root, 1u << (L - 1 - st), q), q,
                            sh);
            fill_powers(T + kTwStage, kTwSmall, root, q, sh);
            fill_powers(T + kTwStage + kTwSmall, kTwSmall, powmod_u32(root, 1u << 9, q), q, sh);
            // the third table times 2^32 in Shoup-form sets, so that products
            // of small-table entries come out in Montgomery form
            fill_powers(T + kTwStage + 2 * kTwSmall, kTwSmall, powmod_u32(root, 1u << 18, q), q,
                        sh, sh ? to_mont_c(1, q) : 1u);
        }
    }
}

static void build_twiddles(Ctx &c)
{
    std::vector<uint2> h(kTwTotal);
    twiddle_tables_host(h.data());
    CAT_CUDA(cudaMalloc(&c.twiddles, h.size() * sizeof(uint2)));
    CAT_CUDA(cudaMemcpy(c.twiddles, h.data(), h.size() * sizeof(uint2),
                        cudaMemcpyHostToDevice));
    upload_low_twiddles(h.data());
}

void ctx_init(Ctx &c, int device, size_t budget)
{
    int ndev = 0;
    CAT_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) fail(CAT_EINVAL, "no such CUDA device");
    CAT_CUDA(cudaSetDevice(device));
    c.device = device;
    c.budget = budget;
    CAT_CUDA(cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, device));
    // a tuning table made on this kind of device, if there is one
    const std::string tp = default_tuning_path();
    if (!tp.empty()) load_tuning(c, tp.c_str());
    if (const char *e = getenv("CAT_COMBA_MAX_SLOT")) c.comba_max_slot = strtoull(e, nullptr, 10);
    // column-pass twiddles from tables (default) or computed in the passes
    if (const char *e = getenv("CAT_COL_TWIDDLE_TABLES")) c.col_tw_tables = atoi(e) != 0;
    if (const char *e = getenv("CAT_COL_TW_FIRST_MAX_LOG")) c.col_tw_first_max_log = atoi(e);
    if (const char *e = getenv("CAT_COL_TW_MAX_LOG")) c.col_tw_max_log = atoi(e);
    // a lower single-transform limit sends shorter products through the piece
    // path (used to exercise it at small sizes)
    if (const char *e = getenv("CAT_MAX_TRANSFORM_LOG")) {
        const long v = strtol(e, nullptr, 10);
        if (v >= 13 && v <= kLogMaxNtt) c.max_log = (int)v;
    }
    pool_for(device);
    build_twiddles(c);
    CAT_CUDA(cudaMallocHost(&c.host_word, 4 * sizeof(uint64_t)));
    CAT_CUDA(cudaMalloc(&c.dev_word, sizeof(unsigned long long)));
}

void ctx_release(Ctx &c)
{
    cudaSetDevice(c.device);
    drop_col_twiddles(c);
    if (c.twiddles) {
        cudaFree(c.twiddles);
        c.twiddles = nullptr;
    }
    if (c.dev_word) {
        cudaFree(c.dev_word);
        c.dev_word = nullptr;
    }
    if (c.host_word) {
        cudaFreeHost(c.host_word);
        c.host_word = nullptr;
    }
}

// --------------------------------------------------------------- bounds

// log2 of the quantity from log-gamma, plus a margin of two limbs.  The
// double-precision error of lgamma at x <= 2^32 is below 1e-5 nats, far inside
// the margin.
size_t bound_limbs(uint64_t n, int kind)
{
    double x = (double)n, ln;
    if (kind == CAT_FACTORIAL)
        ln = lgamma(x + 1.0);
    else if (kind == CAT_CENTRAL_BINOMIAL)
        ln = lgamma(2.0 * x + 1.0) - 2.0 * lgamma(x + 1.0);
    else
        ln = lgamma(2.0 * x + 1.0) - lgamma(x + 1.0) - lgamma(x + 2.0);
    if (ln < 0) ln = 0;
    double bits = ln / log(2.0);
    return (size_t)(bits / 32.0) + 2;
}

// The same for a factorial ratio: sum_i ln a_i! - sum_j ln b_j!, each term's
// lgamma error far below the two spare limbs.
size_t ratio_bound_limbs(const Ratio &r)
{
    double ln = 0;
    for (int i = 0; i < r.ka; i++) ln += lgamma((double)r.a[i] + 1.0);
    for (int j = 0; j < r.kb; j++) ln -= lgamma((double)r.b[j] + 1.0);
    if (ln < 0) ln = 0;
    return (size_t)(ln / log(2.0) / 32.0) + 2;
}

}  // namespace cat
