// capi.cu -- the extern "C" entry points of libcatalan (include/catalan.h).
// Each converts the internal exceptions into status codes and records the
// message in the context.
#include "cat_internal.cuh"

#include <string.h>

#include <new>

struct cat_ctx {
    cat::Ctx c;
};

namespace cat {
void ctx_init(Ctx &c, int device, size_t budget);
void ctx_release(Ctx &c);
void exact_batch(Ctx &c, const cat_request *reqs, size_t count, uint32_t *out, size_t cap,
                 uint64_t *offsets, uint64_t *lengths, cudaStream_t s);
size_t batch_bound(const cat_request *reqs, size_t count);
}  // namespace cat

namespace {

template <typename F>
int guarded(cat_ctx *ctx, F &&body)
{
    try {
        if (ctx) {
            ctx->c.last_error.clear();
            cat::check_cuda(cudaSetDevice(ctx->c.device), "cudaSetDevice");
        }
        body();
        if (ctx) cat::prof_resolve(ctx->c);
        return CAT_OK;
    } catch (const cat::Error &e) {
        if (ctx) {
            ctx->c.last_error = e.msg;
            cat::prof_resolve(ctx->c);
        }
        return e.code;
    } catch (const std::bad_alloc &) {
        if (ctx) ctx->c.last_error = "host allocation failed";
        return CAT_ENOMEM;
    } catch (...) {
        if (ctx) ctx->c.last_error = "unexpected internal error";
        return CAT_ECUDA;
    }
}

inline cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

// A factorial ratio from the ABI's arrays; false if the arguments are out of
// range (term count, a term >= 2^32, numerator sum >= 2^32, null arrays).
bool make_ratio(const uint64_t *a, int ka, const uint64_t *b, int kb, cat::Ratio *r)
{
    if (ka < 0 || kb < 0 || ka > cat::kMaxRatioTerms || kb > cat::kMaxRatioTerms) return false;
    if ((ka && !a) || (kb && !b)) return false;
    *r = cat::Ratio{};
    r->kind = cat::kRatioKind;
    r->ka = ka;
    r->kb = kb;
    uint64_t sum = 0;
    for (int i = 0; i < ka; i++) {
        if (a[i] >= (1ull << 32)) return false;
        sum += a[i];
        r->a[i] = (uint32_t)a[i];
    }
    if (sum >= (1ull << 32)) return false;
    for (int j = 0; j < kb; j++) {
        if (b[j] >= (1ull << 32)) return false;
        r->b[j] = (uint32_t)b[j];
    }
    return true;
}

void copy_out(cat::Ctx &c, const cat::Big &r, uint32_t *out, size_t cap, size_t *out_len,
              cudaStream_t s)
{
    *out_len = r.n;
    if (r.n > cap) cat::fail(CAT_ERANGE, "output capacity too small");
    if (r.n)
        CAT_CUDA(cudaMemcpyAsync(out, r.buf.get(), 4 * r.n, cudaMemcpyDeviceToDevice, s));
    CAT_CUDA(cudaStreamSynchronize(s));
    (void)c;
}

}  // namespace

extern "C" {

int cat_ctx_create(int device, size_t hbm_budget_bytes, cat_ctx **out)
{
    if (!out) return CAT_EINVAL;
    *out = nullptr;
    cat_ctx *ctx = new (std::nothrow) cat_ctx;
    if (!ctx) return CAT_ENOMEM;
    int rc = guarded(nullptr, [&] { cat::ctx_init(ctx->c, device, hbm_budget_bytes); });
    if (rc != CAT_OK) {
        cat::ctx_release(ctx->c);
        delete ctx;
        return rc;
    }
    *out = ctx;
    return CAT_OK;
}

void cat_ctx_destroy(cat_ctx *ctx)
{
    if (!ctx) return;
    cat::ctx_release(ctx->c);
    delete ctx;
}

const char *cat_last_error(const cat_ctx *ctx)
{
    return ctx ? ctx->c.last_error.c_str() : "";
}

int cat_autotune(cat_ctx *ctx, const char *path, void *stream)
{
    if (!ctx) return CAT_EINVAL;
    return guarded(ctx, [&] {
        cat::autotune(ctx->c, as_stream(stream));
        if (path) cat::save_tuning(ctx->c, path);
    });
}

int cat_ctx_load_tuning(cat_ctx *ctx, const char *path)
{
    if (!ctx || !path) return CAT_EINVAL;
    return guarded(ctx, [&] {
        if (!cat::load_tuning(ctx->c, path))
            cat::fail(CAT_EINVAL, std::string("no tuning table for this device at ") + path);
    });
}

int cat_ctx_tuning(const cat_ctx *ctx, size_t *comba_max_slot, int *row_log, size_t count)
{
    if (!ctx || (count && !row_log)) return CAT_EINVAL;
    if (comba_max_slot) *comba_max_slot = ctx->c.comba_max_slot;
    for (size_t n = 0; n < count; n++)
        row_log[n] = n <= (size_t)cat::kLogMaxNtt ? ctx->c.row_log[n] : 0;
    return CAT_OK;
}

int cat_ctx_memory(const cat_ctx *ctx, size_t *in_use, size_t *peak)
{
    if (!ctx) return CAT_EINVAL;
    if (in_use) *in_use = ctx->c.in_use;
    if (peak) *peak = ctx->c.peak;
    return CAT_OK;
}

unsigned long long cat_launch_count(void) { return cat::launch_count(); }

int cat_ctx_set_profiling(cat_ctx *ctx, int on)
{
    if (!ctx) return CAT_EINVAL;
    ctx->c.profiling = on != 0;
    ctx->c.prof.clear();
    return CAT_OK;
}

int cat_ctx_profile(const cat_ctx *ctx, size_t i, const char **name, uint64_t *launches,
                    double *ms, double *bytes, double *unit_bytes)
{
    if (!ctx) return CAT_EINVAL;
    if (i >= ctx->c.prof.size()) return CAT_ERANGE;
    const cat::ProfEntry &e = ctx->c.prof[i];
    if (name) *name = e.name.c_str();
    if (launches) *launches = e.launches;
    if (ms) *ms = e.ms;
    if (bytes) *bytes = e.bytes;
    if (unit_bytes) *unit_bytes = e.unit_bytes;
    return CAT_OK;
}

int catalan_factor(cat_ctx *ctx, uint64_t n, int kind, cat_factorization *out, void *stream)
{
    if (!ctx || !out) return CAT_EINVAL;
    return guarded(ctx, [&] { cat::factor(ctx->c, n, kind, out, as_stream(stream)); });
}

void cat_factor_free(cat_ctx *ctx, cat_factorization *f)
{
    if (!ctx || !f) return;
    cudaSetDevice(ctx->c.device);
    cat::factor_free(ctx->c, f);
}

int cat_factor_copy_primes(cat_ctx *ctx, const cat_factorization *f, uint32_t *dst,
                           size_t cap, void *stream)
{
    if (!ctx || !f || (cap && !dst)) return CAT_EINVAL;
    return guarded(ctx, [&] {
        if (f->num_primes > cap) cat::fail(CAT_ERANGE, "destination too small");
        cudaStream_t s = as_stream(stream);
        if (f->num_primes)
            CAT_CUDA(cudaMemcpyAsync(dst, f->primes, 4 * f->num_primes,
                                     cudaMemcpyDeviceToDevice, s));
        CAT_CUDA(cudaStreamSynchronize(s));
    });
}

int bigint_mul(cat_ctx *ctx, const uint32_t *a, size_t na, const uint32_t *b, size_t nb,
               uint32_t *out, size_t cap, size_t *out_len, void *stream)
{
    if (!ctx || !out_len || (na && !a) || (nb && !b) || (cap && !out)) return CAT_EINVAL;
    return guarded(ctx, [&] {
        cudaStream_t s = as_stream(stream);
        const size_t n = na + nb;
        // straight into out when it holds na + nb limbs and overlaps neither
        // operand; otherwise through a scratch product
        auto apart = [&](const uint32_t *x, size_t nx) {
            const uintptr_t o = (uintptr_t)out, xs = (uintptr_t)x;
            return o + 4 * cap <= xs || xs + 4 * nx <= o;
        };
        if (cap >= n && apart(a, na) && apart(b, nb)) {
            cat::mul_into(ctx->c, a, na, b, nb, out, s);
            *out_len = cat::trim(ctx->c, out, n, s);
            return;
        }
        cat::Big r;
        r.buf = cat::DevBuf<uint32_t>(ctx->c, n ? n : 1, s);
        cat::mul_into(ctx->c, a, na, b, nb, r.buf.get(), s);
        r.n = cat::trim(ctx->c, r.buf.get(), n, s);
        copy_out(ctx->c, r, out, cap, out_len, s);
    });
}

int bigint_pow(cat_ctx *ctx, const uint32_t *a, size_t na, uint64_t e, uint32_t *out,
               size_t cap, size_t *out_len, void *stream)
{
    if (!ctx || !out_len || (na && !a) || (cap && !out)) return CAT_EINVAL;
    return guarded(ctx, [&] {
        cudaStream_t s = as_stream(stream);
        cat::Big r = cat::power(ctx->c, a, na, e, s);
        copy_out(ctx->c, r, out, cap, out_len, s);
    });
}

int product_tree(cat_ctx *ctx, const uint32_t *values, size_t count, uint32_t *out,
                 size_t cap, size_t *out_len, void *stream)
{
    if (!ctx || !out_len || (count && !values) || (cap && !out)) return CAT_EINVAL;
    return guarded(ctx, [&] {
        cudaStream_t s = as_stream(stream);
        cat::Big r = cat::tree_product(ctx->c, values, count, s);
        copy_out(ctx->c, r, out, cap, out_len, s);
    });
}

int cat_reconstruct(cat_ctx *ctx, const cat_factorization *f, uint32_t *out, size_t cap,
                    size_t *out_len, void *stream)
{
    if (!ctx || !f || !out_len || (cap && !out)) return CAT_EINVAL;
    return guarded(ctx, [&] {
        cudaStream_t s = as_stream(stream);
        if (cat::reconstruct_out_of_core(ctx->c, f)) {
            // the caller's factorisation stays as it is
            cat::reconstruct_into(ctx->c, const_cast<cat_factorization *>(f), out, cap, false,
                                  out_len, s, false);
            return;
        }
        cat::Big r = cat::reconstruct(ctx->c, f, s);
        copy_out(ctx->c, r, out, cap, out_len, s);
    });
}

int cat_bound_limbs(uint64_t n, int kind, size_t *limbs)
{
    if (!limbs || n >= (1ull << 31) || kind < CAT_CATALAN || kind > CAT_FACTORIAL)
        return CAT_EINVAL;
    *limbs = cat::bound_limbs(n, kind);
    return CAT_OK;
}

int cat_exact(cat_ctx *ctx, int kind, uint64_t n, uint32_t *out, size_t cap,
              size_t *out_len, void *stream)
{
    if (!ctx || !out_len || (cap && !out)) return CAT_EINVAL;
    if (n >= (1ull << 31) || kind < CAT_CATALAN || kind > CAT_FACTORIAL) return CAT_EINVAL;
    return guarded(ctx, [&] {
        cudaStream_t s = as_stream(stream);
        cat_factorization f{};
        cat::factor(ctx->c, n, kind, &f, s);
        try {
            if (cat::reconstruct_out_of_core(ctx->c, &f)) {
                cat::reconstruct_into(ctx->c, &f, out, cap, false, out_len, s);
                return;
            }
            // the primes are at most the sieve limit
            cat::Big r = cat::reconstruct(ctx->c, &f, s,
                                          cat::bits_below(kind == CAT_FACTORIAL ? n : 2 * n));
            cat::factor_free(ctx->c, &f);
            copy_out(ctx->c, r, out, cap, out_len, s);
        } catch (...) {
            cat::factor_free(ctx->c, &f);
            throw;
        }
    });
}

int cat_ratio_bound_limbs(const uint64_t *a, int ka, const uint64_t *b, int kb, size_t *limbs)
{
    cat::Ratio r;
    if (!limbs || !make_ratio(a, ka, b, kb, &r)) return CAT_EINVAL;
    *limbs = cat::ratio_bound_limbs(r);
    return CAT_OK;
}

int cat_ratio_factor(cat_ctx *ctx, const uint64_t *a, int ka, const uint64_t *b, int kb,
                     cat_factorization *out, void *stream)
{
    cat::Ratio r;
    if (!ctx || !out || !make_ratio(a, ka, b, kb, &r)) return CAT_EINVAL;
    return guarded(ctx, [&] { cat::factor_ratio(ctx->c, r, out, as_stream(stream)); });
}

int cat_ratio_exact(cat_ctx *ctx, const uint64_t *a, int ka, const uint64_t *b, int kb,
                    uint32_t *out, size_t cap, size_t *out_len, void *stream)
{
    cat::Ratio q;
    if (!ctx || !out_len || (cap && !out) || !make_ratio(a, ka, b, kb, &q)) return CAT_EINVAL;
    return guarded(ctx, [&] {
        cudaStream_t s = as_stream(stream);
        cat_factorization f{};
        cat::factor_ratio(ctx->c, q, &f, s);
        try {
            if (cat::reconstruct_out_of_core(ctx->c, &f)) {
                cat::reconstruct_into(ctx->c, &f, out, cap, false, out_len, s);
                return;
            }
            uint64_t top = 1;  // the primes are at most the largest numerator term
            for (int i = 0; i < q.ka; i++) top = std::max<uint64_t>(top, q.a[i]);
            cat::Big r = cat::reconstruct(ctx->c, &f, s, cat::bits_below(top));
            cat::factor_free(ctx->c, &f);
            copy_out(ctx->c, r, out, cap, out_len, s);
        } catch (...) {
            cat::factor_free(ctx->c, &f);
            throw;
        }
    });
}

int cat_batch_bound(const cat_request *reqs, size_t count, size_t *total)
{
    if (!total || (count && !reqs)) return CAT_EINVAL;
    for (size_t r = 0; r < count; r++)
        if (reqs[r].n >= (1ull << 31) || reqs[r].kind < CAT_CATALAN ||
            reqs[r].kind > CAT_FACTORIAL)
            return CAT_EINVAL;
    *total = cat::batch_bound(reqs, count);
    return CAT_OK;
}

int cat_exact_batch(cat_ctx *ctx, const cat_request *reqs, size_t count, uint32_t *out,
                    size_t cap, uint64_t *offsets, uint64_t *lengths, void *stream)
{
    if (!ctx || (count && (!reqs || !offsets || !lengths)) || (cap && !out)) return CAT_EINVAL;
    return guarded(ctx, [&] {
        cat::exact_batch(ctx->c, reqs, count, out, cap, offsets, lengths, as_stream(stream));
    });
}

int catalan_exact(cat_ctx *ctx, uint64_t n, uint32_t *out, size_t cap, size_t *out_len,
                  void *stream)
{
    return cat_exact(ctx, CAT_CATALAN, n, out, cap, out_len, stream);
}

int cat_exact_host(cat_ctx *ctx, int kind, uint64_t n, uint32_t *host_out, size_t cap,
                   size_t *out_len, void *stream)
{
    if (!ctx || !out_len || (cap && !host_out)) return CAT_EINVAL;
    if (n >= (1ull << 31) || kind < CAT_CATALAN || kind > CAT_FACTORIAL) return CAT_EINVAL;
    return guarded(ctx, [&] {
        cudaStream_t s = as_stream(stream);
        cat_factorization f{};
        cat::factor(ctx->c, n, kind, &f, s);
        cat::Big r;
        try {
            if (cat::reconstruct_out_of_core(ctx->c, &f)) {
                cat::reconstruct_into(ctx->c, &f, host_out, cap, true, out_len, s);
                return;
            }
            r = cat::reconstruct(ctx->c, &f, s,
                                 cat::bits_below(kind == CAT_FACTORIAL ? n : 2 * n));
        } catch (...) {
            cat::factor_free(ctx->c, &f);
            throw;
        }
        cat::factor_free(ctx->c, &f);
        *out_len = r.n;
        if (r.n > cap) cat::fail(CAT_ERANGE, "output capacity too small");
        cat::copy_to_host(ctx->c, host_out, r.buf.get(), r.n, s);
        CAT_CUDA(cudaStreamSynchronize(s));
    });
}

int cat_factor_text(cat_ctx *ctx, const cat_factorization *f, const char *name, char *out,
                    size_t cap, size_t *out_len, void *stream)
{
    if (!ctx || !f || !name || !out_len || (cap && !out)) return CAT_EINVAL;
    return guarded(ctx, [&] {
        if (cat::factor_text(ctx->c, f, name, out, cap, out_len, as_stream(stream)) != CAT_OK)
            cat::fail(CAT_ERANGE, "output capacity too small");
    });
}

int cat_binary(cat_ctx *ctx, const uint32_t *limbs, size_t n, uint8_t *out, size_t cap,
               size_t *out_len, void *stream)
{
    if (!ctx || !out_len || (n && !limbs) || (cap && !out)) return CAT_EINVAL;
    return guarded(ctx, [&] {
        if (cat::binary_file(ctx->c, limbs, n, out, cap, out_len, as_stream(stream)) != CAT_OK)
            cat::fail(CAT_ERANGE, "output capacity too small");
    });
}

size_t cat_decimal_bound(size_t n) { return cat::decimal_bound(n); }

int to_decimal(cat_ctx *ctx, const uint32_t *limbs, size_t n, char *out, size_t cap,
               size_t *out_len, void *stream)
{
    if (!ctx || !out_len || (n && !limbs) || (cap && !out)) return CAT_EINVAL;
    return guarded(ctx, [&] {
        const int rc =
            cat::to_decimal_dev(ctx->c, limbs, n, out, cap, out_len, as_stream(stream));
        if (rc == CAT_ERANGE) cat::fail(CAT_ERANGE, "output capacity too small");
    });
}

}  // extern "C"
