// autotune.cu -- measures the device-dependent choices of the product tree's
// multiplications on the current GPU and applies them to a context:
//   - the row-pass size (2^9 .. 2^12 points) of the multi-pass transform for
//     every transform size 2^13 .. 2^27, the rest of the transform going to
//     one or two column passes;
//   - the largest tree-level slot (32 .. 256 limbs) whose products the
//     schoolbook (Comba) kernels finish faster than the transform.
// Each candidate multiplies a synthetic tree level of 2^24 limbs (one product
// of 2^n limbs above that; seeded words) and is timed with CUDA events on the
// context's stream; the fastest wins.  The largest trial holds about 6 GB of
// scratch and 4.5 GB of column twiddle tables (dropped after every trial).
// The table is written as text, tagged with the device's name and SM count,
// and read back by contexts created later on the same kind of device.
#include "cat_internal.cuh"

#include <dlfcn.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <fstream>
#include <sstream>
#include <string>

namespace cat {

bool plan_row_ok(int n, int rrow);

namespace {

constexpr size_t kTuneLimbs = (size_t)1 << 24;
constexpr int kTuneMinLog = 13, kTuneMaxLog = kLogMaxNtt;
const size_t kCombaSlots[] = {32, 64, 128, 256};

// Seeded pseudo-random words (an integer hash of the index), so that no
// limb is zero and no product degenerates.
__global__ void tune_fill(uint32_t *x, size_t n, uint32_t seed)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        uint32_t v = (uint32_t)i * 2654435761u ^ seed;
        v ^= v << 13;
        v ^= v >> 17;
        v ^= v << 5;
        x[i] = v | 1u;
    }
}

// Median device milliseconds of five runs of f after one warm-up run.
template <class F>
float time_ms(cudaStream_t s, F &&f)
{
    cudaEvent_t a, b;
    CAT_CUDA(cudaEventCreate(&a));
    CAT_CUDA(cudaEventCreate(&b));
    f();
    float t[5];
    for (float &x : t) {
        CAT_CUDA(cudaEventRecord(a, s));
        f();
        CAT_CUDA(cudaEventRecord(b, s));
        CAT_CUDA(cudaEventSynchronize(b));
        CAT_CUDA(cudaEventElapsedTime(&x, a, b));
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    std::sort(t, t + 5);
    return t[2];
}

// The default row-pass size of a 2^n-point transform (the plan without a
// tuned value).
int default_row(int n) { return std::min(12, n - 4); }

std::string device_tag(int device)
{
    cudaDeviceProp p;
    CAT_CUDA(cudaGetDeviceProperties(&p, device));
    std::string name = p.name;
    for (char &ch : name)
        if (ch == ' ') ch = '_';
    return name + " " + std::to_string(p.multiProcessorCount);
}

}  // namespace

void autotune(Ctx &c, cudaStream_t s)
{
    NvtxRange range("autotune");
    const int top = std::min(kTuneMaxLog, c.max_log);
    const size_t limbs = std::max(kTuneLimbs, (size_t)1 << top);
    DevBuf<uint32_t> in(c, limbs, s), out(c, limbs, s);
    tune_fill<<<c.num_sms * 4, 256, 0, s>>>(in.get(), limbs, 0x9e3779b9u);
    CAT_LAUNCH("tune_fill");
    // row-pass size per transform size (one product per trial above 2^24 points)
    for (int n = kTuneMinLog; n <= top; n++) {
        const size_t slot = (size_t)1 << (n - 1), nprod = std::max<size_t>(1, kTuneLimbs >> n);
        // the default plan first; another size replaces it only when at least
        // 1 % faster, so that near-ties keep the default
        const int def = default_row(n);
        c.row_log[n] = 0;
        int best = def;
        // each trial's column twiddle tables (built by its warm-up run) are
        // dropped after it, so that at most one plan's tables are held
        float best_ms = time_ms(s, [&] { ntt_level(c, in.get(), slot, nprod, out.get(), s); });
        drop_col_twiddles(c);
        for (int r = 9; r <= 12; r++) {
            if (r == def || !plan_row_ok(n, r)) continue;
            c.row_log[n] = r;
            const float ms =
                time_ms(s, [&] { ntt_level(c, in.get(), slot, nprod, out.get(), s); });
            drop_col_twiddles(c);
            if (ms < 0.99f * best_ms) {
                best = r;
                best_ms = ms;
            }
        }
        c.row_log[n] = plan_row_ok(n, best) ? best : 0;
    }
    // schoolbook / transform crossover: the largest slot up to which Comba wins
    size_t cross = 16;
    for (size_t slot : kCombaSlots) {
        const size_t nprod = kTuneLimbs / (2 * slot);
        const float tc =
            time_ms(s, [&] { comba_level(c, in.get(), slot, nprod, out.get(), s); });
        const float tn = time_ms(s, [&] { ntt_level(c, in.get(), slot, nprod, out.get(), s); });
        if (tc > tn) break;
        cross = slot;
    }
    c.comba_max_slot = cross;
    c.tuning = "measured";
    drop_col_twiddles(c);
}

void save_tuning(const Ctx &c, const char *path)
{
    std::ofstream f(path);
    if (!f) fail(CAT_EINVAL, std::string("cannot write the tuning table ") + path);
    f << "# libcatalan tuning table (cat_autotune): device name and SM count, the\n"
         "# schoolbook/transform crossover slot, and the row-pass size per transform size\n";
    f << "device " << device_tag(c.device) << "\n";
    f << "comba_max_slot " << c.comba_max_slot << "\n";
    for (int n = 0; n <= kLogMaxNtt; n++)
        if (c.row_log[n]) f << "row_log " << n << " " << c.row_log[n] << "\n";
    if (!f) fail(CAT_EINVAL, std::string("cannot write the tuning table ") + path);
}

// Applies the table at path when it was made on this kind of device; returns
// false (and changes nothing) otherwise.
bool load_tuning(Ctx &c, const char *path)
{
    std::ifstream f(path);
    if (!f) return false;
    std::string line, tag = device_tag(c.device);
    size_t slot = 0;
    int rows[kLogMaxNtt + 1] = {};
    bool device_ok = false;
    while (std::getline(f, line)) {
        if (line.empty() || line[0] == '#') continue;
        std::istringstream is(line);
        std::string key;
        is >> key;
        if (key == "device") {
            std::string name, sms;
            is >> name >> sms;
            device_ok = (name + " " + sms) == tag;
        } else if (key == "comba_max_slot") {
            is >> slot;
        } else if (key == "row_log") {
            int n = 0, r = 0;
            is >> n >> r;
            if (n < 0 || n > kLogMaxNtt || !plan_row_ok(n, r)) return false;
            rows[n] = r;
        } else {
            return false;
        }
    }
    if (!device_ok || (slot != 16 && slot != 32 && slot != 64 && slot != 128 && slot != 256))
        return false;
    c.comba_max_slot = slot;
    for (int n = 0; n <= kLogMaxNtt; n++) c.row_log[n] = rows[n];
    c.tuning = path;
    return true;
}

// The table a context reads when it is created: $CAT_TUNE_FILE, else
// autotune.txt in the directory of this library.
std::string default_tuning_path()
{
    if (const char *e = getenv("CAT_TUNE_FILE")) return e;
    Dl_info info;
    if (dladdr((void *)&default_tuning_path, &info) && info.dli_fname) {
        std::string p = info.dli_fname;
        const size_t slash = p.rfind('/');
        return (slash == std::string::npos ? std::string(".") : p.substr(0, slash)) +
               "/autotune.txt";
    }
    return "";
}

}  // namespace cat
