/*
 * catalan.h -- C ABI of libcatalan, a GB300 (sm_103a) library for exact
 * Catalan numbers C(n), central binomials C(2n, n) and factorials n!, built on
 * the two-phase prime-exponent method of arXiv 2601.11621.
 *
 *   Phase 1 (Sec. 3.1, Algorithm 1): sieve the primes p <= 2n, compute
 *   e_p = v_p((2n)!) - 2 v_p(n!) - v_p(n+1) by Legendre's formula (Sec. 2),
 *   drop e_p = 0 and group the primes by exponent.
 *   Phase 2 (Sec. 3.2, Algorithm 2): Q_e = BalancedProductTree(G_e),
 *   P_e = Q_e^e, C(n) = BalancedProductTree({P_e}).
 *
 * Conventions shared by every entry point
 *   - Big integers are arrays of little-endian uint32_t limbs.  Lengths
 *     written back through *out_len are normalised: the top limb is non-zero;
 *     zero has length 0 and one is {1} with length 1.  Input lengths may
 *     include leading zero limbs.
 *   - Every data pointer (inputs and outputs) is a DEVICE pointer owned by
 *     the caller, unless the function name ends in _host.  Inputs are read
 *     only and must not overlap the output.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  All work
 *     is issued on it.  The functions plan on the host from small device
 *     read-backs, so they return only after the result has been computed;
 *     the output is complete and visible on `stream` when they return CAT_OK.
 *   - Scratch memory comes from the context's pool (stream-ordered, cached),
 *     bounded by the context's HBM budget.
 *   - Errors: argument errors are reported before any work is issued.  A
 *     CUDA error is reported as CAT_ECUDA and its text is kept in the
 *     context (cat_last_error).  After an error the output contents are
 *     unspecified.
 *   - Supported n: 0 <= n <= 2^31 - 1, so every prime involved is < 2^32.
 *   - One context must not be used by two host threads at the same time.
 */
#ifndef CATALAN_H
#define CATALAN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CAT_OK = 0,
    CAT_EINVAL = -1,        /* bad argument (null pointer, n out of range, ...) */
    CAT_ENOMEM = -2,        /* device allocation failed or HBM budget exceeded  */
    CAT_ERANGE = -3,        /* output capacity too small; *out_len = needed     */
    CAT_ENOTINTEGRAL = -4,  /* a prime exponent came out negative (Sec. 6.3)    */
    CAT_ETIMEOUT = -5,      /* a bounded device wait gave up                    */
    CAT_ECUDA = -6,         /* CUDA runtime error; see cat_last_error           */
    CAT_EBUSY = -7          /* request still pending                            */
} cat_status;

/* Quantity selected by its exponent rule (Sec. 2 and the Sec. 6.3 special
 * cases): Catalan e = v_p((2n)!) - 2 v_p(n!) - v_p(n+1) over p <= 2n;
 * central binomial e = v_p((2n)!) - 2 v_p(n!) over p <= 2n;
 * factorial e = v_p(n!) over p <= n. */
typedef enum {
    CAT_CATALAN = 0,
    CAT_CENTRAL_BINOMIAL = 1,
    CAT_FACTORIAL = 2
} cat_kind;

typedef struct cat_ctx cat_ctx;

/* Creates a context on CUDA device `device`.  hbm_budget_bytes caps the
 * scratch the context may hold at once (0 = no cap).  When the in-core
 * reconstruction of a quantity would not fit the cap (about 128 bytes per
 * result limb), cat_exact, catalan_exact, cat_exact_host and cat_ratio_exact
 * (and cat_reconstruct, which leaves the caller's factorisation as it is)
 * reconstruct it within the cap instead, the paper's chunked products with
 * partial products kept in pinned host memory (Sec. 3.2): the primes are
 * multiplied in chunks sized to the cap, and products too large for it run by
 * pieces through a sliding device window.  The result is the same integer,
 * computed more slowly.  Phase 1 itself runs in-core (about 0.5 bytes per
 * integer up to 2n plus 4 bytes per prime) and fails with CAT_ENOMEM if that
 * does not fit.  The context owns the NTT twiddle tables and the scratch pool.
 * A context without a cap also keeps, built on first use, a table of the
 * inter-pass twiddles of every column-pass shape it has run (2^m words per
 * prime for blocks of 2^m points: about 10 GB after C(2,050,572,903)); it is
 * not scratch (not counted by cat_ctx_memory) and is freed with the context.
 * A capped context computes those twiddles instead.
 * Returns CAT_OK and *out, or an error (CAT_EINVAL, CAT_ECUDA). */
int cat_ctx_create(int device, size_t hbm_budget_bytes, cat_ctx **out);

/* Frees the context and everything it owns.  NULL is ignored. */
void cat_ctx_destroy(cat_ctx *ctx);

/* Text of the last error recorded in ctx ("" if none).  Owned by ctx. */
const char *cat_last_error(const cat_ctx *ctx);

/* ------------------------------------------------------------ autotuning
 * The device-dependent choices of the product tree's multiplications (the
 * paper leaves them to its bignum library): the row-pass size of the
 * multi-pass transform for each transform size 2^13 .. 2^27, and the largest
 * tree-level slot (32 .. 256 limbs) multiplied by schoolbook (Comba) rather
 * than by the transform.
 *
 * cat_autotune: times every candidate on a synthetic tree level of 2^24
 * limbs (one product of 2^n limbs above that) on ctx's device (about a
 * second; up to about 6 GB of scratch from the context's pool),
 * applies the fastest to ctx and, when path is not NULL, writes them as a
 * text table tagged with the device's name and SM count.  Results of every
 * entry point are the same integers with any choice; only speed changes.
 * cat_ctx_load_tuning: applies a table written by cat_autotune
 * (CAT_EINVAL when it is unreadable or was made on another kind of device).
 * A new context reads the table at $CAT_TUNE_FILE, else autotune.txt next to
 * libcatalan.so, when it exists and matches the device.
 * cat_ctx_tuning: the values in use: the crossover slot, and row_log[n] for
 * n < count (0 = the default plan).  Errors: CAT_EINVAL, CAT_ENOMEM,
 * CAT_ECUDA. */
int cat_autotune(cat_ctx *ctx, const char *path, void *stream);
int cat_ctx_load_tuning(cat_ctx *ctx, const char *path);
int cat_ctx_tuning(const cat_ctx *ctx, size_t *comba_max_slot, int *row_log, size_t count);

/* Bytes of scratch currently held / the high-water mark since creation. */
int cat_ctx_memory(const cat_ctx *ctx, size_t *in_use, size_t *peak);

/* The number of kernels this library has launched in this process, over all
 * contexts and threads, each counted when it is issued (a measurement aid:
 * the difference across a call is that call's launches). */
unsigned long long cat_launch_count(void);

/* Per-kernel device timing (tracing aid, not part of the method).  When on,
 * every kernel launch is bracketed by CUDA events on its stream; each entry
 * point resolves them before returning.  Turning it on or off clears the
 * totals.  Errors: CAT_EINVAL. */
int cat_ctx_set_profiling(cat_ctx *ctx, int on);

/* Totals for the i-th kernel name seen since profiling was switched on:
 * launches, summed device milliseconds, summed pass bytes (the bytes the
 * launch itself must read and write at minimum, e.g. three residue arrays in
 * and out for a transform pass) and summed unit bytes: the algorithmic bytes
 * of the products the launches completed, 4 bytes per limb of each operand
 * read once and of each product written once (for a level of the product
 * tree, 8 bytes per limb of the level).  A product's unit bytes are counted
 * on the one launch that holds its pointwise step (the transform's row pass,
 * the one-block multiply, a schoolbook or leaf kernel) and are 0 for its other
 * launches.  *name is owned by ctx.  Returns CAT_ERANGE when i is past the
 * last entry. */
int cat_ctx_profile(const cat_ctx *ctx, size_t i, const char **name, uint64_t *launches,
                    double *ms, double *bytes, double *unit_bytes);

/* ------------------------------------------------------------------ Phase 1
 * Grouped prime factorisation of the quantity (Sec. 3.1, Algorithm 1):
 * the primes with e_p > 0 in CSR form.  Group g has exponent exps[g]
 * (ascending) and its primes are primes[offsets[g] .. offsets[g+1]) in
 * ascending order.  Device arrays are owned by the context and released by
 * cat_factor_free; host_exps / host_offsets are host copies.
 * primes_sieved = the number of primes <= the sieve limit (2n, or n for n!). */
typedef struct {
    uint64_t num_groups;
    uint64_t num_primes;
    uint64_t primes_sieved;
    uint64_t *exps;          /* device, num_groups      */
    uint64_t *offsets;       /* device, num_groups + 1  */
    uint32_t *primes;        /* device, num_primes      */
    uint64_t *host_exps;     /* host,   num_groups      */
    uint64_t *host_offsets;  /* host,   num_groups + 1  */
} cat_factorization;

/* Phase 1 on the device: segmented sieve of the primes <= 2n (n for n!),
 * Legendre exponents by kind, and grouping by exponent.
 * Errors: CAT_EINVAL (n >= 2^31, bad kind), CAT_ENOMEM, CAT_ENOTINTEGRAL,
 * CAT_ECUDA. */
int catalan_factor(cat_ctx *ctx, uint64_t n, int kind, cat_factorization *out,
                   void *stream);

/* Releases the arrays of a factorisation returned by catalan_factor.  Work
 * that reads them must have completed. */
void cat_factor_free(cat_ctx *ctx, cat_factorization *f);

/* Copies the grouped primes of f (num_primes values) into the caller's
 * device buffer dst of cap entries.  Errors: CAT_EINVAL, CAT_ERANGE. */
int cat_factor_copy_primes(cat_ctx *ctx, const cat_factorization *f, uint32_t *dst,
                           size_t cap, void *stream);

/* ------------------------------------------------------------------ Phase 2
 * out = a * b.  a has na limbs, b has nb limbs (device).  out has room for
 * cap limbs; na + nb limbs always suffice.  *out_len = normalised length.
 * out may overlap a or b (the product is then formed in library scratch and
 * copied); a disjoint out of at least na + nb limbs receives it directly.
 * Errors: CAT_EINVAL, CAT_ERANGE (cap < normalised length), CAT_ENOMEM,
 * CAT_ECUDA.  Products of up to 2^27 limbs take one three-prime transform;
 * longer ones are summed from products of pieces of at most 2^26 limbs (any
 * length that fits device memory). */
int bigint_mul(cat_ctx *ctx, const uint32_t *a, size_t na, const uint32_t *b,
               size_t nb, uint32_t *out, size_t cap, size_t *out_len, void *stream);

/* out = a * b without allocating any device memory.  The paper has no
 * counterpart: this is for callers that cannot call cudaMalloc, such as an
 * application whose own allocator already holds the device's memory (a new
 * allocation would fail or fragment it), or code that must not take
 * cudaMalloc/cudaFree's implicit synchronisation of the whole device (this
 * call waits only for its own stream), or a service that must not meet an
 * out-of-memory failure in the middle of a request.  There is no context: the
 * transform scratch and the twiddle tables live in fixed-size __device__
 * arrays of the library (about 2.4 MB of scratch and 1.4 MB of tables),
 * which every GPU that loads the library holds until the process exits.
 *   - Limit: na + nb <= 65,536 limbs; larger products return CAT_ENOMEM
 *     (checked before any device work).
 *   - out must have room for na + nb limbs (cap >= na + nb, else
 *     CAT_ERANGE); *out_len = the normalised length.  a, b, out are device
 *     pointers; stream as elsewhere.  Every call synchronises `stream` before
 *     it returns (it reads the normalised length back), so the result is
 *     complete on return.
 *   - Runs on the current CUDA device.  The first call on a device sets that
 *     device up (looks up the arrays' device addresses and uploads the
 *     twiddle table with a synchronous copy); make that first call before any
 *     stream capture.
 *   - Every call shares the same scratch array: calls that overlap on the GPU
 *     (other streams or other host threads) race; serialise them.
 *   - Errors: CAT_EINVAL (null pointer), CAT_ENOMEM (too large), CAT_ERANGE,
 *     CAT_ECUDA. */
int bigint_mul_noalloc(const uint32_t *a, size_t na, const uint32_t *b, size_t nb,
                       uint32_t *out, size_t cap, size_t *out_len, void *stream);

/* out = a^e by left-to-right binary exponentiation ("fast pow",
 * Algorithm 2).  a^0 = 1.  Errors as bigint_mul. */
int bigint_pow(cat_ctx *ctx, const uint32_t *a, size_t na, uint64_t e,
               uint32_t *out, size_t cap, size_t *out_len, void *stream);

/* out = product of the count 32-bit values (device array), by the balanced
 * product tree of Sec. 3.2.  The empty product is 1.  A result of count
 * limbs always fits.  Errors as bigint_mul. */
int product_tree(cat_ctx *ctx, const uint32_t *values, size_t count, uint32_t *out,
                 size_t cap, size_t *out_len, void *stream);

/* Algorithm 2 on a factorisation: out = prod_g (prod_{p in G_g} p)^exps[g].
 * The P_e with e >= 2 are combined by always multiplying the two shortest,
 * which keeps every intermediate as short as possible (the aim Sec. 3.2
 * states for the balanced tree); their product then joins the tree of Q_1
 * as one node, so the longest factor needs no final multiplication (the same
 * integer, re-associated). */
int cat_reconstruct(cat_ctx *ctx, const cat_factorization *f, uint32_t *out,
                    size_t cap, size_t *out_len, void *stream);

/* Upper bound on the limb count of the quantity (from log-gamma with a
 * safety margin); a buffer of that many limbs always suffices.
 * Errors: CAT_EINVAL. */
int cat_bound_limbs(uint64_t n, int kind, size_t *limbs);

/* Phase 1 + Phase 2 end to end for one kind: out = the exact quantity.
 * Errors: those of catalan_factor and bigint_mul. */
int cat_exact(cat_ctx *ctx, int kind, uint64_t n, uint32_t *out, size_t cap,
              size_t *out_len, void *stream);

/* cat_exact for the Catalan number C(n) = (2n)! / (n! (n+1)!). */
int catalan_exact(cat_ctx *ctx, uint64_t n, uint32_t *out, size_t cap,
                  size_t *out_len, void *stream);

/* cat_exact writing into a HOST buffer: the device result is copied back
 * before returning (the copy is part of the call).  When host_out lies in
 * page-locked memory mapped for the device (cudaHostAlloc, cudaHostRegister),
 * the copy is a kernel storing straight into it; for pageable memory it is a
 * copy-engine transfer.  host_out must hold cap limbs in one buffer. */
int cat_exact_host(cat_ctx *ctx, int kind, uint64_t n, uint32_t *host_out,
                   size_t cap, size_t *out_len, void *stream);

/* ------------------------------------------------------------------ batches
 * One request of a batch: the quantity `kind` at n. */
typedef struct {
    int kind;
    uint64_t n;
} cat_request;

/* Limbs a batch needs in total: the sum of cat_bound_limbs over the
 * requests.  Errors: CAT_EINVAL. */
int cat_batch_bound(const cat_request *reqs, size_t count, size_t *total);

/* The exact quantities of `count` requests computed together: Phase 1 once
 * for the batch (one sieve up to the largest limit, exponents for every
 * request) and Phase 2 as one segmented product tree whose every level, for
 * all requests at once, is a single batched multiplication (each request's
 * product runs over its primes with multiplicity e_p, which equals
 * prod_e Q_e^e of Algorithm 2).  Factorials with n >= 64, whose exponents
 * are large, are computed one by one through the grouped path of cat_exact
 * inside the same call.  Results go back to back into the device
 * buffer out (cap limbs, at least cat_batch_bound): request r at
 * offsets[r] (host array, written by the call; the prefix sums of
 * cat_bound_limbs), normalised length lengths[r] (host array).
 * Errors: CAT_EINVAL, CAT_ERANGE (cap too small; lengths[0] = the total
 * needed), CAT_ENOMEM, CAT_ENOTINTEGRAL, CAT_ECUDA. */
int cat_exact_batch(cat_ctx *ctx, const cat_request *reqs, size_t count, uint32_t *out,
                    size_t cap, uint64_t *offsets, uint64_t *lengths, void *stream);

/* -------------------------------------------------------- factorial ratios
 * N = prod_{i<ka} a_i! / prod_{j<kb} b_j! (Sec. 6.3): binomials C(n, k) =
 * n!/(k!(n-k)!), multinomials, and any other ratio of factorial products.
 * Phase 1 sieves the primes up to the largest term and sums Legendre's
 * formula over the terms, v_p(N) = sum_i v_p(a_i!) - sum_j v_p(b_j!); Phase 2
 * is the same reconstruction as for C(n).  a and b are HOST arrays.
 * Limits: 0 <= ka, kb <= 16; every term below 2^32; the a_i sum to less than
 * 2^32 (so every exponent fits 32 bits).  An empty product is 1.
 *
 * cat_ratio_bound_limbs: an upper bound on N's limb count (log-gamma, two
 * spare limbs).  cat_ratio_factor: the grouped factorisation, as
 * catalan_factor (free with cat_factor_free).  cat_ratio_exact: N into the
 * device buffer out of cap limbs, *out_len its normalised length.
 * Errors: CAT_EINVAL (limits above, null pointers), CAT_ENOTINTEGRAL (some
 * v_p(N) < 0: N is not an integer), CAT_ERANGE (cap too small), CAT_ENOMEM,
 * CAT_ECUDA. */
int cat_ratio_bound_limbs(const uint64_t *a, int ka, const uint64_t *b, int kb, size_t *limbs);
int cat_ratio_factor(cat_ctx *ctx, const uint64_t *a, int ka, const uint64_t *b, int kb,
                     cat_factorization *out, void *stream);
int cat_ratio_exact(cat_ctx *ctx, const uint64_t *a, int ka, const uint64_t *b, int kb,
                    uint32_t *out, size_t cap, size_t *out_len, void *stream);

/* ---------------------------------------------------------------- artifacts
 * cat_factor_text: the grouped factorisation f in the text layout of Sec. 3.1,
 * as ASCII into the device buffer out of cap bytes:
 *     # Prime factorization of <name>
 *     # exponent=E count=K            (one block per group, ascending E)
 *     p1 p2 ... pK                    (its primes, ascending, one line)
 * Lines end with '\n'; no terminator.  *out_len = the byte count (the exact
 * size is returned with CAT_ERANGE when cap is short).  At most 390,000,000
 * primes.  Errors: CAT_EINVAL, CAT_ERANGE, CAT_ENOMEM, CAT_ECUDA.
 *
 * cat_binary: the result file of Algorithm 2's last step: the bytes 01 01
 * followed by the magnitude of limbs[0..n) in little-endian byte order, its
 * minimal length ceil(bits / 8) (the layout whose SHA-256 is the one Table 1
 * prints for C(2,050,572,903); the paper states the magnitude's size,
 * 512,643,220 bytes), into the device buffer out of cap bytes.  Zero is the
 * two header bytes alone.  Errors: CAT_EINVAL, CAT_ERANGE, CAT_ECUDA. */
int cat_factor_text(cat_ctx *ctx, const cat_factorization *f, const char *name, char *out,
                    size_t cap, size_t *out_len, void *stream);
int cat_binary(cat_ctx *ctx, const uint32_t *limbs, size_t n, uint8_t *out, size_t cap,
               size_t *out_len, void *stream);

/* ----------------------------------------------------------- decimal output
 * The optional decimal text output of the reconstructed number (Sec. 3.2;
 * Table 1 of Sec. 5 states 1,234,567,890 digits for C(2,050,572,903)).
 *
 * cat_decimal_bound: an upper bound on the digit count of any number of n
 * limbs (floor(32 n log10 2) + 2).
 *
 * to_decimal: the decimal digits of the little-endian uint32 number
 * limbs[0..n) (device pointer; leading zero limbs allowed) as ASCII into the
 * device buffer out of cap bytes: most significant digit first, no sign, no
 * leading zeros, no terminator; "0" for zero.  *out_len = the digit count.
 * Converted by a tree over the limbs in base 10^9 (batched three-prime
 * products with the powers 2^(32 w), carries in base 10^9); scratch comes
 * from the context's pool and is about 3x the input.  Returns when done.
 * Errors: CAT_EINVAL (null pointer), CAT_ERANGE (cap too small; *out_len is
 * the exact count, which cat_decimal_bound never undercuts), CAT_ENOMEM,
 * CAT_ECUDA. */
size_t cat_decimal_bound(size_t n);
int to_decimal(cat_ctx *ctx, const uint32_t *limbs, size_t n, char *out, size_t cap,
               size_t *out_len, void *stream);

/* ------------------------------------------------------------------ serving
 * A continuous-batching request engine on one device (the paper has a single
 * offline run; this is the serving layer around the same computation).
 * `workers` threads each own a context and a CUDA stream.  An idle worker
 * admits the queued requests in arrival order, at most max_batch of them
 * (0 = 4096), while their estimated device footprint plus the estimates of
 * the batches already running plus the results still held fits
 * hbm_budget_bytes (0 = no cap; a worker admits one request when nothing
 * else is running), and computes them together with cat_exact_batch.  The
 * footprint estimate is 256 bytes per limb of the result bound
 * (cat_bound_limbs) plus 2 MiB (cat_batch_footprint); cat_server_submit
 * denies (CAT_ENOMEM) a request whose estimate alone exceeds the budget.  All workers' scratch and results count
 * against one shared cap of hbm_budget_bytes, so a batch that still outgrows
 * it fails with CAT_ENOMEM for its tickets.  Requests that arrive while
 * batches are running are admitted by the next idle worker, so batches
 * overlap on the GPU.  Results stay in device memory until released.
 * All functions are thread-safe. */
typedef struct cat_server cat_server;

typedef struct {
    int kind;
    uint64_t n;
    const uint32_t *limbs;     /* device pointer, valid until release   */
    uint64_t length;           /* normalised limb count                  */
    uint64_t t_submit_ns;      /* steady-clock times of submission,      */
    uint64_t t_start_ns;       /* admission into a batch and completion  */
    uint64_t t_end_ns;
    uint64_t batch;            /* id of the batch that computed it       */
} cat_server_result;

/* Errors: CAT_EINVAL (workers outside 1..64), CAT_ECUDA. */
int cat_server_create(int device, size_t hbm_budget_bytes, int workers, size_t max_batch,
                      cat_server **out);

/* Queues one request; *ticket identifies it.  Errors: CAT_EINVAL, CAT_ENOMEM
 * (estimated footprint above the whole budget). */
int cat_server_submit(cat_server *sv, int kind, uint64_t n, uint64_t *ticket);

/* CAT_EBUSY while queued or running; CAT_OK with *res filled when done; the
 * request's error code if it failed; CAT_EINVAL for an unknown ticket. */
int cat_server_poll(cat_server *sv, uint64_t ticket, cat_server_result *res);

/* As cat_server_poll, waiting up to timeout_ms (CAT_ETIMEOUT if still busy). */
int cat_server_wait(cat_server *sv, uint64_t ticket, uint64_t timeout_ms,
                    cat_server_result *res);

/* Copies a finished result (length limbs) into dst (host memory if to_host,
 * else device memory) of cap limbs; *out_len = its length.  The ticket stays
 * valid.  Errors: CAT_EBUSY, CAT_ERANGE, CAT_EINVAL, CAT_ECUDA. */
int cat_server_fetch(cat_server *sv, uint64_t ticket, uint32_t *dst, size_t cap, int to_host,
                     size_t *out_len);

/* Forgets a finished ticket and frees its result (CAT_EBUSY while pending). */
int cat_server_release(cat_server *sv, uint64_t ticket);

/* The serving engine's estimate of the device bytes `count` requests hold
 * while they are computed together: for each request 2 MiB plus 256 bytes per
 * limb of cat_bound_limbs (measured peaks: at most 1.35 MB for tiny n and at
 * most 124 bytes per limb from n = 10^4 to 3 * 10^8), summed.  Admission
 * compares it with the budget.  Errors: CAT_EINVAL. */
int cat_batch_footprint(const cat_request *reqs, size_t count, size_t *bytes);

/* Device bytes all workers hold now (scratch and results) and their
 * high-water mark since creation; both stay within hbm_budget_bytes when it
 * is set.  Errors: CAT_EINVAL. */
int cat_server_memory(cat_server *sv, size_t *in_use, size_t *peak);

/* Requests waiting for admission / tickets held (queued, running, done). */
int cat_server_pending(cat_server *sv, size_t *queued, size_t *total);

/* Stops the workers (running batches finish), frees all results. */
void cat_server_destroy(cat_server *sv);

#ifdef __cplusplus
}
#endif

#endif /* CATALAN_H */
