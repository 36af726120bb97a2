// artifacts.cu -- the run's files as the paper describes them: the grouped
// factorisation as text (Sec. 3.1: a title line, then per exponent group a
// line "# exponent=E count=K" and a line of its primes) and the binary result
// file whose SHA-256 Table 1 prints (Sec. 3.2, Algorithm 2's last step).
#include "cat_internal.cuh"

#include <string>
#include <vector>

namespace cat {

void exclusive_scan_u32(Ctx &c, uint32_t *data, size_t n, cudaStream_t s);

__device__ __forceinline__ int dec_digits(uint32_t p)
{
    int d = 1;
    while (p >= 10) {
        p /= 10;
        d++;
    }
    return d;
}

// first[g] = off[goffs[g]]: where group g's primes start in the primes' text.
__global__ void text_group_starts(const uint32_t *off, const uint64_t *goffs, uint64_t ngroups,
                                  uint32_t *first)
{
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g < ngroups) first[g] = off[goffs[g]];
}

// Bytes of prime i's text: its digits and one separator.  len[count] = 0.
__global__ void text_lengths(const uint32_t *primes, size_t count, uint32_t *len)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) len[i] = (uint32_t)dec_digits(primes[i]) + 1;
    if (i == count) len[i] = 0;
}

// Prime i goes to off[i] (its place in the concatenated primes' text) plus
// the bytes of the title and of the headers of groups 0..g, g its group: each
// header sits just before its group's first prime.  A group's last prime ends
// its line with '\n', the others with ' '.
__global__ void text_write(const uint32_t *primes, size_t count, const uint32_t *off,
                           const uint64_t *goffs, uint64_t ngroups, const uint64_t *hdr_through,
                           char *out)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    // group g: the largest g with goffs[g] <= i
    uint64_t lo = 0, hi = ngroups;  // goffs[lo] <= i < goffs[hi]
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) / 2;
        if (goffs[mid] <= i) lo = mid;
        else hi = mid;
    }
    char *o = out + hdr_through[lo] + off[i];
    uint32_t p = primes[i];
    const int nd = dec_digits(p);
    for (int d = nd - 1; d >= 0; d--) {
        o[d] = (char)('0' + p % 10u);
        p /= 10u;
    }
    o[nd] = (i + 1 == goffs[lo + 1]) ? '\n' : ' ';
}

int factor_text(Ctx &c, const cat_factorization *f, const char *name, char *out, size_t cap,
                size_t *needed, cudaStream_t s)
{
    const uint64_t G = f->num_groups, count = f->num_primes;
    if (count > 390000000ull) fail(CAT_EINVAL, "factorisation too large for 32-bit text offsets");
    // headers on the host: the title, then one line per group
    const std::string title = std::string("# Prime factorization of ") + name + "\n";
    std::vector<std::string> hdr(G);
    std::vector<uint64_t> through(G);  // title + headers of groups 0..g
    uint64_t acc = title.size();
    for (uint64_t g = 0; g < G; g++) {
        hdr[g] = "# exponent=" + std::to_string(f->host_exps[g]) +
                 " count=" + std::to_string(f->host_offsets[g + 1] - f->host_offsets[g]) + "\n";
        acc += hdr[g].size();
        through[g] = acc;
    }
    DevBuf<uint32_t> off(c, count + 1, s);
    const unsigned blocks = (unsigned)((count + 1 + 255) / 256);
    text_lengths<<<blocks, 256, 0, s>>>(f->primes, count, off.get());
    CAT_LAUNCH("text_lengths");
    exclusive_scan_u32(c, off.get(), count + 1, s);
    uint32_t body = 0;
    CAT_CUDA(cudaMemcpyAsync(&body, off.get() + count, 4, cudaMemcpyDeviceToHost, s));
    CAT_CUDA(cudaStreamSynchronize(s));
    const size_t total = acc + body;
    *needed = total;
    if (cap < total) return CAT_ERANGE;
    // the title and each header go in front of their group's primes
    std::vector<uint32_t> first(G + 1, 0);
    if (G) {
        DevBuf<uint32_t> d_first(c, G, s);
        text_group_starts<<<(unsigned)((G + 255) / 256), 256, 0, s>>>(off.get(), f->offsets, G,
                                                                      d_first.get());
        CAT_LAUNCH("text_group_starts");
        CAT_CUDA(cudaMemcpyAsync(first.data(), d_first.get(), 4 * G, cudaMemcpyDeviceToHost, s));
        CAT_CUDA(cudaStreamSynchronize(s));
    }
    CAT_CUDA(cudaMemcpyAsync(out, title.data(), title.size(), cudaMemcpyHostToDevice, s));
    for (uint64_t g = 0; g < G; g++) {
        const uint64_t at = (through[g] - hdr[g].size()) + first[g];
        CAT_CUDA(cudaMemcpyAsync(out + at, hdr[g].data(), hdr[g].size(), cudaMemcpyHostToDevice,
                                 s));
    }
    if (count) {
        DevBuf<uint64_t> d_through(c, G, s);
        CAT_CUDA(cudaMemcpyAsync(d_through.get(), through.data(), 8 * G, cudaMemcpyHostToDevice,
                                 s));
        const int tok = prof_begin(c, "text_write", s);
        text_write<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(
            f->primes, count, off.get(), f->offsets, G, d_through.get(), out);
        CAT_LAUNCH("text_write");
        prof_end(c, tok, s, 4.0 * (double)count + (double)body);
    }
    CAT_CUDA(cudaStreamSynchronize(s));
    return CAT_OK;
}

size_t binary_bytes(Ctx &c, const uint32_t *x, size_t n, cudaStream_t s, size_t *mag_bytes)
{
    n = n ? normalized_length(c, x, n, s) : 0;
    uint32_t top = 0;
    if (n) {
        CAT_CUDA(cudaMemcpyAsync(&top, x + n - 1, 4, cudaMemcpyDeviceToHost, s));
        CAT_CUDA(cudaStreamSynchronize(s));
    }
    int tb = 0;
    while (tb < 32 && (top >> tb)) tb++;
    const uint64_t bits = n ? (uint64_t)(n - 1) * 32 + tb : 0;
    *mag_bytes = (size_t)((bits + 7) / 8);
    return 2 + *mag_bytes;
}

int binary_file(Ctx &c, const uint32_t *x, size_t n, uint8_t *out, size_t cap, size_t *needed,
                cudaStream_t s)
{
    size_t mag = 0;
    const size_t total = binary_bytes(c, x, n, s, &mag);
    *needed = total;
    if (cap < total) return CAT_ERANGE;
    const uint8_t header[2] = {1, 1};
    CAT_CUDA(cudaMemcpyAsync(out, header, 2, cudaMemcpyHostToDevice, s));
    if (mag) CAT_CUDA(cudaMemcpyAsync(out + 2, x, mag, cudaMemcpyDeviceToDevice, s));
    CAT_CUDA(cudaStreamSynchronize(s));
    return CAT_OK;
}

}  // namespace cat
