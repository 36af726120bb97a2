// ntt.cu -- exact big-integer multiplication by a three-prime number-theoretic
// transform (NTT), Chinese remaindering and carry propagation.
//
// This is the multiplication the reconstruction phase spends its time in
// (Sec. 3.2; Sec. 6 reports that the big products dominate the run time, and
// Sec. 6.3 assumes an FFT-based multiplication for large operands).  The
// method is the classical one: the limbs of a and b are the coefficients of
// two polynomials; their cyclic convolution of length L = 2^n >= na + nb is
// computed modulo three primes q_i (forward transforms, pointwise product,
// inverse transform), the exact coefficients are recovered by Garner's
// mixed-radix Chinese remaindering, and their 96-bit values are summed into
// 32-bit limbs with carry propagation.
//
// Transform layout.  The forward transform is an in-place decimation-in-
// frequency transform (natural order in, bit-reversed order out); the inverse
// is the matching decimation-in-time transform (bit-reversed in, natural out),
// so no permutation pass is needed.  A length-2^n transform is split into
// passes that each run 2^r-point sub-transforms in shared memory (the
// "four-step" factorisation L = L1 * L2 applied recursively): column passes
// over strided sub-arrays, each followed by the twiddle w_M^(col * k1), and a
// final row pass over contiguous runs of 2^r points.  The last forward row
// pass, the pointwise product and the first inverse row pass are fused.
// Transforms of up to 2^12 points run entirely inside one thread block,
// including the remaindering and carries.
#include "cat_internal.cuh"

#include <algorithm>
#include <mutex>

namespace cat {

// --------------------------------------------------------------- constants

#define CAT_SET_CONST(f)                                                              \
    {{f(ntt_prime(0, 0)), f(ntt_prime(0, 1)), f(ntt_prime(0, 2))},                    \
     {f(ntt_prime(1, 0)), f(ntt_prime(1, 1)), f(ntt_prime(1, 2))},                    \
     {f(ntt_prime(2, 0)), f(ntt_prime(2, 1)), f(ntt_prime(2, 2))}}
#define CAT_Q(q) (q)
#define CAT_WP1(q) shoup_c(1u, q)
__constant__ uint32_t c_q[kNumSets][kNumPrimes] = CAT_SET_CONST(CAT_Q);
__constant__ uint32_t c_qinv[kNumSets][kNumPrimes] = CAT_SET_CONST(inv32);
// floor(2^32 / q): Shoup's companion of 1, which reduces raw limbs
__constant__ uint32_t c_wp1[kNumSets][kNumPrimes] = CAT_SET_CONST(CAT_WP1);

#undef CAT_SET_CONST
#undef CAT_Q
#undef CAT_WP1

// Entries [0, 16) of every stage table (the twiddles of stage bits below 4,
// [set][prime][direction][index] in the stage table's own layout and
// multiplier form), for the register rounds with B = 0, whose twiddle indices
// are compile-time constants: served from constant memory they are uniform
// operands instead of registers held across the round.
__constant__ uint2 c_tw_low[kNumSets][kNumPrimes][2][16];

void upload_low_twiddles(const uint2 *tables)
{
    uint2 h[kNumSets][kNumPrimes][2][16];
    for (int set = 0; set < kNumSets; set++)
        for (int p = 0; p < kNumPrimes; p++)
            for (int d = 0; d < 2; d++)
                for (int j = 0; j < 16; j++)
                    h[set][p][d][j] = tables[(((size_t)set * kNumPrimes + p) * 2 + d) * kTwPerDir + j];
    CAT_CUDA(cudaMemcpyToSymbol(c_tw_low, h, sizeof(h)));
}

// Garner constants of a set, in Montgomery form.
template <int PS>
struct Garner {
    static constexpr uint32_t q0 = ntt_prime(PS, 0), q1 = ntt_prime(PS, 1), q2 = ntt_prime(PS, 2);
    static constexpr uint32_t qinv1 = inv32(q1), qinv2 = inv32(q2);
    static constexpr uint32_t inv_q0_mod_q1 = to_mont_c(powmod_u32(q0 % q1, q1 - 2, q1), q1);
    static constexpr uint32_t q0_mod_q2 = to_mont_c(q0 % q2, q2);
    static constexpr uint32_t inv_q0q1_mod_q2 =
        to_mont_c(powmod_u32(mulmod_u64(q0, q1, q2), q2 - 2, q2), q2);
    static_assert(q0 < q1 && q1 < q2, "Garner order assumes q0 < q1 < q2");
    // the same three factors as plain residues with Shoup's companions
    static constexpr uint32_t s1 = powmod_u32(q0 % q1, q1 - 2, q1), s1p = shoup_c(s1, q1);
    static constexpr uint32_t s2 = q0 % q2, s2p = shoup_c(s2, q2);
    static constexpr uint32_t s3 = powmod_u32(mulmod_u64(q0, q1, q2), q2 - 2, q2),
                              s3p = shoup_c(s3, q2);
};

// Pointwise scale 2^-n folded into the product's second factor: 2^32 2^-n mod
// q in Shoup's form for sets 0 and 1, 2^64 2^-n mod q (Montgomery) for set 2,
// so that pmul(x, y) = x y 2^-n.
struct Scale {
    uint2 c[kNumPrimes];
};

static Scale make_scale(int set, int n)
{
    Scale s;
    for (int i = 0; i < kNumPrimes; i++) {
        const uint32_t q = ntt_prime(set, i);
        const uint32_t inv2n = powmod_u32((q + 1) / 2, (uint64_t)n, q);  // 2^-n
        const uint32_t r = to_mont_c(inv2n, q);                           // 2^32 2^-n
        s.c[i] = set_shoup(set) ? make_uint2(r, shoup_c(r, q)) : make_uint2(to_mont_c(r, q), 0u);
    }
    return s;
}

// -------------------------------------------------------------- twiddles

__device__ __forceinline__ const uint2 *tw_table(const uint2 *tw, int set, int p, int dir)
{
    return tw + (((size_t)set * kNumPrimes + p) * 2 + dir) * kTwPerDir;
}

// w^E 2^32 mod q (the Montgomery form of w^E, below q) from the three small
// tables.  In Shoup-form sets the third table holds w^(2^18 j) 2^32, so two
// Shoup products give the Montgomery form directly; in set 2 all entries are
// Montgomery forms and Montgomery products keep that form.
template <int PS>
__device__ __forceinline__ uint32_t tw_pow_mont(const uint2 *T, uint32_t E, uint32_t q,
                                                uint32_t qinv)
{
    const uint2 a = __ldg(&T[kTwStage + (E & (kTwSmall - 1))]);
    const uint2 b = __ldg(&T[kTwStage + kTwSmall + ((E >> 9) & (kTwSmall - 1))]);
    const uint2 c = __ldg(&T[kTwStage + 2 * kTwSmall + (E >> 18)]);
    if constexpr (PS == 2) {
        return mont_mul_pre(mont_mul_pre(a.x, b.x, b.y, q), c.x, c.y, q);
    } else {
        return csub(shoup(shoup(a.x, b.x, b.y, q), c.x, c.y, q), q);
    }
}

// x v for any 32-bit x and a Montgomery-form multiplier vm = v 2^32 mod q,
// into the set's forward range (set 0: hi(x vm) - hi(m q) + q lies in (0, 2q)).
template <int PS>
__device__ __forceinline__ uint32_t mul_mont(uint32_t x, uint32_t vm, uint32_t q, uint32_t qinv)
{
    if constexpr (PS == 0) {
        const uint32_t hi = __umulhi(x, vm);
        const uint32_t m = (x * vm) * qinv;
        return hi - __umulhi(m, q) + q;
    } else if constexpr (PS == 1) {
        return mont<true>(x, vm, q, qinv);
    } else {
        return mont_mul(x, vm, q, qinv);
    }
}

// Product of two Montgomery-form multipliers, reduced below q, with the
// second one's companion up = um q^-1 mod 2^32 precomputed (three multiplies:
// the low word of vm um times q^-1 is vm up).
template <int PS>
__device__ __forceinline__ uint32_t mont_step(uint32_t vm, uint32_t um, uint32_t up, uint32_t q)
{
    if constexpr (PS == 2) return mont_mul_pre(vm, um, up, q);
    const uint32_t hi = __umulhi(vm, um);
    const uint32_t m = vm * up;
    return csub(hi - __umulhi(m, q) + q, q);
}

// ----------------------------------------------- remaindering and carries

// Garner: the coefficient c < q0 q1 q2 with c = r_i mod q_i, as three words,
// from inverse-transform residues (reduced into [0, q_i) first).
template <int PS>
__device__ __forceinline__ void crt3(uint32_t r0, uint32_t r1, uint32_t r2, uint32_t &c0,
                                     uint32_t &c1, uint32_t &c2)
{
    using G = Garner<PS>;
    uint32_t x0, x1, x2;
    if constexpr (PS == 2) {
        x0 = r0;  // < q0 < q1 < q2
        x1 = mont_mul(sub_mod(r1, x0, G::q1), G::inv_q0_mod_q1, G::q1, G::qinv1);
        uint32_t t = sub_mod(r2, x0, G::q2);
        t = sub_mod(t, mont_mul(x1, G::q0_mod_q2, G::q2, G::qinv2), G::q2);
        x2 = mont_mul(t, G::inv_q0q1_mod_q2, G::q2, G::qinv2);
    } else {
        // Shoup products take any 32-bit input, so the differences go in
        // unreduced: set 0's lazy residues need only r0 fully reduced (it is
        // the exact low digit) and r1, r2 below 2q; set 1's are below q.
        x0 = final_red<PS>(r0, G::q0);
        if constexpr (PS == 0) {
            r1 = csub(r1, 2 * G::q1);  // [0, 2 q1)
            r2 = csub(r2, 2 * G::q2);  // [0, 2 q2)
        }
        // (r1 - x0) / q0 mod q1, the input in (0, 3 q1)
        x1 = csub(shoup(r1 - x0 + G::q1, G::s1, G::s1p, G::q1), G::q1);
        const uint32_t u = csub(shoup(x1, G::s2, G::s2p, G::q2), G::q2);  // x1 q0 mod q2
        uint32_t t;
        if constexpr (PS == 0)
            t = r2 - x0 - u + 2 * G::q2;  // (0, 4 q2), below 2^32 as 4 q2 < 2^32
        else
            t = sub_m<true>(r2, x0, G::q2) - u + G::q2;  // (0, 2 q2)
        x2 = csub(shoup(t, G::s3, G::s3p, G::q2), G::q2);
    }
    const uint64_t y = (uint64_t)G::q1 * x2 + x1;                 // < q1 q2
    const uint64_t lo = (uint64_t)G::q0 * (uint32_t)y + x0;
    const uint64_t hi = (uint64_t)G::q0 * (uint32_t)(y >> 32) + (lo >> 32);
    c0 = (uint32_t)lo;
    c1 = (uint32_t)hi;
    c2 = (uint32_t)(hi >> 32);
}

// The carry map of a run in compact form.  A run takes its carry-in c in
// {0,1,2,3} into its lowest limb, and one more carry leaves it only if that
// limb overflows and every other limb is the largest digit; so its map is
// c -> b + [c >= t] with b the carry-out for c = 0 and t in {1,2,3} (or 4,
// never).  Compositions keep the form, (f o g)(c) = b_f + [b_g + [c >= t_g]
// >= t_f], with t = 0 for "always".  Packed as b << 4 | t; kUnitId (t = 15)
// is the identity, for threads without limbs.
constexpr uint32_t kUnitId = 15u;

__device__ __forceinline__ uint32_t unit_eval(uint32_t m, uint32_t c)
{
    return m == kUnitId ? c : (m >> 4) + (c >= (m & 15u) ? 1u : 0u);
}

// f o g
__device__ __forceinline__ uint32_t unit_compose(uint32_t f, uint32_t g)
{
    const uint32_t tf = f & 15u, bg = g >> 4, tg = g & 15u;
    const uint32_t t = bg >= tf ? 0u : (bg + 1u == tf ? tg : 4u);
    uint32_t r = (f & ~15u) | t;
    r = g == kUnitId ? f : r;
    return f == kUnitId ? g : r;
}

// Scan of compact run maps over the threads of the block, in thread order:
// returns the carry into thread t's run for a carry-in of 0 ahead of thread 0,
// and the composition of all the block's maps through *total.  wsm holds 32
// words.  Synchronises internally.
__device__ uint32_t block_carry_scan(uint32_t f, uint32_t *wsm, uint32_t *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    uint32_t inc = f;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, inc, off);
        if (lane >= off) inc = unit_compose(inc, o);
    }
    __syncthreads();
    if (lane == 31) wsm[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < nw ? wsm[lane] : kUnitId;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t o = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w = unit_compose(w, o);
        }
        wsm[lane] = w;
    }
    __syncthreads();
    const uint32_t cin_warp = wid > 0 ? unit_eval(wsm[wid - 1], 0u) : 0u;
    const uint32_t ex = __shfl_up_sync(0xffffffffu, inc, 1);
    *total = wsm[nw - 1];
    return lane > 0 ? unit_eval(ex, cin_warp) : cin_warp;
}

constexpr int kLimbsPerThread = 8;

// Coefficient words of a thread's run of kLimbsPerThread consecutive
// coefficients j0 + i (c0 the low word, c1 the middle, c2 the high).  Limb j
// sums c0[j] + c1[j-1] + c2[j-2], so the first two limbs of a run also need
// c1[j0-1], c2[j0-2] and c2[j0-1] of the preceding run.
struct CoefRun {
    uint32_t c0[kLimbsPerThread], c1[kLimbsPerThread], c2[kLimbsPerThread];
};

// Those three halo words from the preceding thread: by shuffle inside a warp,
// through hsm (3 x 32 words) across warps; thread 0 takes first1/first2a/
// first2b (the block's predecessor).  Every thread of the block calls this.
__device__ __forceinline__ void run_halo(const CoefRun &r, uint32_t first1, uint32_t first2a,
                                         uint32_t first2b, uint32_t *hsm, uint32_t &h1,
                                         uint32_t &h2a, uint32_t &h2b)
{
    constexpr int L = kLimbsPerThread;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    h1 = __shfl_up_sync(0xffffffffu, r.c1[L - 1], 1);
    h2a = __shfl_up_sync(0xffffffffu, r.c2[L - 2], 1);
    h2b = __shfl_up_sync(0xffffffffu, r.c2[L - 1], 1);
    if (lane == 31) {
        hsm[wid] = r.c1[L - 1];
        hsm[32 + wid] = r.c2[L - 2];
        hsm[64 + wid] = r.c2[L - 1];
    }
    __syncthreads();
    if (lane == 0) {
        h1 = wid ? hsm[wid - 1] : first1;
        h2a = wid ? hsm[32 + wid - 1] : first2a;
        h2b = wid ? hsm[64 + wid - 1] : first2b;
    }
}

// The exact coefficient c = w2 2^64 + w1 2^32 + w0 < 10^26 as three base-10^9
// digits (c < min(na, nb) (10^9 - 1)^2 < 2^26 10^18 for digit operands and
// transforms of at most 2^27 points, so the top digit is below 10^8).
__device__ __forceinline__ void words_to_dec(uint32_t &w0, uint32_t &w1, uint32_t &w2)
{
    const uint64_t hi = ((uint64_t)w2 << 32) | w1;
    const uint64_t qh = hi / kDecBase;
    const uint32_t rh = (uint32_t)(hi - qh * kDecBase);
    const uint64_t lo = ((uint64_t)rh << 32) | w0;
    const uint64_t ql = lo / kDecBase;
    const uint64_t q = (qh << 32) + ql;  // floor(c / 10^9) < 10^17
    const uint64_t q2 = q / kDecBase;
    w0 = (uint32_t)(lo - ql * kDecBase);
    w1 = (uint32_t)(q - q2 * kDecBase);
    w2 = (uint32_t)q2;
}

// Limb sums and carries for one tile of coefficient runs, one run per thread
// (run j0 = kLimbsPerThread * threadIdx.x; coefficients at or past tile_len
// are zero), in base 2^32 or (dec) 10^9, plus the addend limbs add[j] for
// j < add_count.  In both bases a limb sums two full words, the coefficient's
// top word or digit (below 2^26 or 10^8: coefficients stay below 2^90, or
// 10^26 for digit operands), the addend and a carry <= 3, so carries stay in
// {0, 1, 2, 3}.  Writes limbs j < min(tile_len, out_count) to out and returns
// the tile's carry map in compact form in *tile_map (valid in every thread; it
// fits a byte).  The tile's own carry-in is assumed 0.
// DEC / ADD: 1 or 0 when known at compile time, -1 when the runtime flag
// (dec, add != null) decides.
template <int DEC, int ADD>
__device__ __forceinline__ void tile_carry_t(const CoefRun &r, uint32_t h1, uint32_t h2a,
                                             uint32_t h2b, int tile_len, uint32_t *out,
                                             long out_count, bool dec_rt, const uint32_t *add,
                                             long add_count, uint32_t *wsm, uint32_t *tile_map)
{
    const bool dec = DEC < 0 ? dec_rt : DEC == 1;
    if (ADD == 0) add = nullptr;
    const int j0 = threadIdx.x * kLimbsPerThread;
    const uint32_t top = dec ? kDecBase - 1 : 0xffffffffu;  // largest limb
    uint32_t limb[kLimbsPerThread];
    uint32_t carry = 0;
    uint32_t f = kUnitId;
    if (j0 < tile_len) {
#pragma unroll
        for (int i = 0; i < kLimbsPerThread; i++) {
            const uint32_t m1 = i >= 1 ? r.c1[i - 1] : h1;
            const uint32_t m2 = i >= 2 ? r.c2[i - 2] : (i == 0 ? h2a : h2b);
            const uint32_t ad = (add && j0 + i < add_count) ? add[j0 + i] : 0u;
            const uint64_t v = (uint64_t)r.c0[i] + m1 + m2 + ad + carry;
            if (dec) {
                const uint32_t v32 = (uint32_t)v;  // < 3.1 10^9 + 3 < 2^32
                carry = (v32 >= kDecBase) + (v32 >= 2 * kDecBase) + (v32 >= 3 * kDecBase);
                limb[i] = v32 - carry * kDecBase;
            } else {
                limb[i] = (uint32_t)v;
                carry = (uint32_t)(v >> 32);
            }
        }
        bool ones = true;
#pragma unroll
        for (int i = 1; i < kLimbsPerThread; i++) ones = ones && limb[i] == top;
        // a carry-in c leaves the run iff ones and limb[0] + c > top
        const uint32_t t = (ones && limb[0] >= top - 2u) ? top + 1u - limb[0] : 4u;
        f = (carry << 4) | t;
    }
    const uint32_t cin = block_carry_scan(f, wsm, tile_map);
    if (j0 < tile_len) {
        uint32_t c = cin;
#pragma unroll
        for (int i = 0; i < kLimbsPerThread; i++) {
            const uint64_t v = (uint64_t)limb[i] + c;
            c = dec ? (uint32_t)(v >= kDecBase) : (uint32_t)(v >> 32);
            limb[i] = dec ? (uint32_t)(v - (uint64_t)c * kDecBase) : (uint32_t)v;
        }
        if (j0 + kLimbsPerThread <= tile_len && j0 + kLimbsPerThread <= out_count &&
            (reinterpret_cast<uintptr_t>(out + j0) & 15) == 0) {
            uint4 *o4 = reinterpret_cast<uint4 *>(out + j0);
            o4[0] = make_uint4(limb[0], limb[1], limb[2], limb[3]);
            o4[1] = make_uint4(limb[4], limb[5], limb[6], limb[7]);
        } else {
#pragma unroll
            for (int i = 0; i < kLimbsPerThread; i++)
                if (j0 + i < tile_len && j0 + i < out_count) out[j0 + i] = limb[i];
        }
    }
}

__device__ void tile_carry(const CoefRun &r, uint32_t h1, uint32_t h2a, uint32_t h2b, int tile_len,
                           uint32_t *out, long out_count, bool dec, const uint32_t *add,
                           long add_count, uint32_t *wsm, uint32_t *tile_map)
{
    tile_carry_t<-1, -1>(r, h1, h2a, h2b, tile_len, out, out_count, dec, add, add_count, wsm,
                         tile_map);
}

constexpr int kTileThreads = 256;
constexpr int kTile = kTileThreads * kLimbsPerThread;  // 2048 limbs

struct CrtArgs {
    const uint32_t *G;  // inverse-transformed residues [prime][product][L]
    size_t gpstride;
    int n;              // log2 L
    Sink sink;          // product k's limbs (out_len <= L)
    uint8_t *tile_maps; // [product][tiles], compact carry maps
};

// One tile of 2048 coefficients per block: each thread remainders its run of
// eight (two 16-byte loads per prime: tiles, runs and the prime arrays are
// multiples of 8 words apart) and sums them into limbs.
template <int PS, bool DEC, bool ADD>
__global__ void __launch_bounds__(kTileThreads) crt_carry_tiles(CrtArgs a)
{
    __shared__ uint32_t wsm[32];
    __shared__ uint32_t hsm[96];
    const size_t tiles = ((size_t)1 << a.n) / kTile;
    const size_t k = blockIdx.x / tiles;
    const size_t t = blockIdx.x % tiles;
    const size_t jt = t * kTile;
    const size_t node = sink_node(a.sink, k);
    const uint32_t *g0 = a.G + (k << a.n) + jt;
    const int j0 = threadIdx.x * kLimbsPerThread;
    constexpr bool dec = DEC;
    uint32_t r[3][kLimbsPerThread];
#pragma unroll
    for (int p = 0; p < 3; p++) {
        const uint4 *v = reinterpret_cast<const uint4 *>(g0 + p * a.gpstride + j0);
        const uint4 x = v[0], y = v[1];
        r[p][0] = x.x; r[p][1] = x.y; r[p][2] = x.z; r[p][3] = x.w;
        r[p][4] = y.x; r[p][5] = y.y; r[p][6] = y.z; r[p][7] = y.w;
    }
    // the tile's predecessor: coefficients jt - 2 and jt - 1 (none for tile 0),
    // loaded by thread 0 beside its run so that the latencies overlap
    const bool pred = threadIdx.x == 0 && t > 0;
    uint32_t pr[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    if (pred) {
#pragma unroll
        for (int p = 0; p < 3; p++) {
            pr[p][0] = g0[p * a.gpstride - 2];
            pr[p][1] = g0[p * a.gpstride - 1];
        }
    }
    CoefRun run;
#pragma unroll
    for (int i = 0; i < kLimbsPerThread; i++) {
        crt3<PS>(r[0][i], r[1][i], r[2][i], run.c0[i], run.c1[i], run.c2[i]);
        if (dec) words_to_dec(run.c0[i], run.c1[i], run.c2[i]);
    }
    uint32_t f1 = 0, f2a = 0, f2b = 0;
    if (pred) {
        uint32_t d0, d1, e0;
        crt3<PS>(pr[0][0], pr[1][0], pr[2][0], d0, d1, f2a);
        if (dec) words_to_dec(d0, d1, f2a);
        crt3<PS>(pr[0][1], pr[1][1], pr[2][1], e0, f1, f2b);
        if (dec) words_to_dec(e0, f1, f2b);
    }
    uint32_t h1, h2a, h2b;
    run_halo(run, f1, f2a, f2b, hsm, h1, h2a, h2b);
    const Sink &o = a.sink;
    const long remaining = (long)o.out_len - (long)jt;
    const uint32_t *add = ADD ? o.add + k * o.add_tstride + jt : nullptr;
    uint32_t map;
    tile_carry_t<DEC ? 1 : 0, ADD ? 1 : 0>(run, h1, h2a, h2b, kTile,
                                           o.out + node * o.out_tstride + jt, remaining, dec, add,
                                           (long)o.add_len - (long)jt, wsm, &map);
    if (threadIdx.x == 0) a.tile_maps[blockIdx.x] = (uint8_t)map;
}

// Carry into each tile of a product (one block per product), in place of the
// tiles' compact maps: each thread folds the maps of its stretch of
// consecutive tiles, a block scan carries between the stretches, and each
// thread replays its stretch, writing every tile's carry-in.
__global__ void __launch_bounds__(1024) carry_tile_scan(uint8_t *tile_maps, size_t tiles)
{
    __shared__ uint32_t wsm[32];
    uint8_t *m = tile_maps + blockIdx.x * tiles;
    const size_t per = (tiles + blockDim.x - 1) / blockDim.x;
    const size_t i0 = threadIdx.x * per, i1 = std::min(tiles, i0 + per);
    uint32_t f = kUnitId;
    for (size_t i = i0; i < i1; i++) f = unit_compose(m[i], f);
    uint32_t total;
    uint32_t c = block_carry_scan(f, wsm, &total);
    for (size_t i = i0; i < i1; i++) {
        const uint32_t g = m[i];
        m[i] = (uint8_t)c;  // now the tile's carry-in
        c = unit_eval(g, c);
    }
}

// Add each tile's carry-in to its first limbs (rarely more than one), in
// base 2^32 or (dec) 10^9.
__global__ void carry_fix(const uint8_t *tile_cin, size_t tiles_total, size_t tiles, int n,
                          uint32_t *out, size_t out_tstride, size_t out_len, bool dec,
                          const uint32_t *out_index = nullptr)
{
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= tiles_total) return;
    uint32_t c = tile_cin[t];
    if (!c) return;
    const size_t k = t / tiles, tt = t % tiles;
    uint32_t *o = out + (out_index ? (size_t)out_index[k] : k) * out_tstride;
    size_t j = tt * kTile;
    const size_t end = std::min(j + kTile, out_len);
    for (; c && j < end; j++) {
        const uint64_t v = (uint64_t)o[j] + c;
        if (dec) {
            c = v >= kDecBase ? 1u : 0u;
            o[j] = (uint32_t)(v - (uint64_t)c * kDecBase);
        } else {
            o[j] = (uint32_t)v;
            c = (uint32_t)(v >> 32);
        }
    }
}

#include "ntt_kernels.cuh"

// ------------------------------------------ whole product in one block

struct FusedArgs {
    const uint32_t *A;
    size_t a_tstride, a_len;
    const uint32_t *B;  // null: square A; b_tstride 0: the same B for every product
    size_t b_tstride, b_len;
    Sink sink;
    const uint2 *tw;
    Scale scale;
};

constexpr int kFusedMaxLog = 12;
constexpr int kFusedThreads = 512;

// The one-block multiply's first forward round input: raw limbs (shared
// memory, unswizzled) reduced into the forward range; column 0 is operand a,
// column 1 operand b (a again when squaring).  With sb, operand b's limbs are
// multiplied by sb (the pointwise step's normalisation 2^(32-n), taken in
// advance) instead of by 1: the same Shoup product.
struct RawIn {
    const uint32_t *a, *b;
    uint32_t q, wp1;
    uint2 sb;  // (multiplier, Shoup companion) for operand b, or (1, wp1)
    template <int E, int B, int NA>
    __device__ __forceinline__ void load(uint32_t (&x)[NA][1 << E], int base, int c) const
    {
        const uint32_t *r = c ? b : a;
        const uint32_t w = c ? sb.x : 1u, wp = c ? sb.y : wp1;
#pragma unroll
        for (int k = 0; k < (1 << E); k++) x[0][k] = shoup(r[base + (k << B)], w, wp, q);
    }
};

// One product per block: per prime the forward transforms of both operands,
// the pointwise product and the inverse transform in shared memory (register
// rounds, the middle one fused as in the row pass), then remaindering and
// carries over one tile.
// Layout (words): residues R0 [0,L) R1 [L,2L) R2 [2L,3L); raw A shares R2's
// space (it is last read before R2 is written), raw B [3L,4L), transform pair
// XY [4L,6L).  Every thread owns a run of eight coefficients for the carries
// (L <= 8 x threads).
// Two blocks per SM (64 registers; a small spill in the remaindering phase):
// measured faster than one block per SM without the spill.
template <int LR>
__global__ void __launch_bounds__(kFusedThreads, 2) ntt_mul_fused(FusedArgs a)
{
    extern __shared__ uint32_t sm[];
    __shared__ uint32_t wsm[32];
    constexpr int L = 1 << LR;
    uint32_t *Rr[3] = {sm, sm + L, sm + 2 * L};
    uint32_t *rawA = sm + 2 * L;
    uint32_t *rawB = sm + 3 * L;
    uint32_t *X = sm + 4 * L;  // X [4L,5L), Y [5L,6L): two arrays for the dual rounds
    uint32_t *Y = X + L;
    const size_t k = blockIdx.x;
    const uint32_t *ga = a.A + k * a.a_tstride;
    const uint32_t *gb = a.B ? a.B + k * a.b_tstride : nullptr;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        rawA[i] = (size_t)i < a.a_len ? ga[i] : 0u;
        rawB[i] = (gb && (size_t)i < a.b_len) ? gb[i] : 0u;
    }
    __syncthreads();
    constexpr int NR = rounds_of(LR);
#pragma unroll 1
    for (int p = 0; p < kNumPrimes; p++) {
        const uint32_t q = c_q[0][p], qinv = c_qinv[0][p], wp1 = c_wp1[0][p];
        const TwRef T{tw_table(a.tw, 0, p, 0), p};
        const TwRef Ti{tw_table(a.tw, 0, p, 1), p};
        const uint2 sc = p == 0 ? a.scale.c[0] : (p == 1 ? a.scale.c[1] : a.scale.c[2]);
        uint32_t *Z = Rr[p];
        if constexpr (NR == 1) {
            // up to 16 points: reduce, transform both, multiply, transform back
            // operand b (when there is one) takes the normalisation in advance
            for (int i = threadIdx.x; i < L; i += blockDim.x) {
                X[swz(i)] = reduce_in<0>(rawA[i], q, wp1);
                Y[swz(i)] = gb ? shoup(rawB[i], sc.x, sc.y, q) : reduce_in<0>(rawA[i], q, wp1);
            }
            __syncthreads();
            dif_smem<LR, 2, 0>(X, T, q);  // X and Y as two arrays
            // elementwise in the swizzled space: Z, X, Y share the permutation
            for (int i = threadIdx.x; i < L; i += blockDim.x)
                Z[i] = gb ? mul_mont<0>(X[i], Y[i], q, qinv) : pmul<0>(X[i], Y[i], sc, q, qinv);
            __syncthreads();
            dit_smem<LR, 1, 0>(Z, Ti, q);
        } else {
            // The first forward round reads the raw limbs and reduces them; X and
            // Y are two arrays of the round (twice the groups of one pair).
            const SmemIO<LR, 2, false> xy{X};
            const RawIn ri{rawA, gb ? rawB : rawA, q, wp1, gb ? sc : make_uint2(1u, wp1)};
            round_io<LR, 2, dif_base(LR, 0), round_size(LR, 0), true, 1, false, 0>(ri, xy, T, q);
            __syncthreads();
            if constexpr (NR == 3) {
                round_io<LR, 2, dif_base(LR, 1), round_size(LR, 1), true, 1, false, 0>(xy, xy, T,
                                                                                      q);
                __syncthreads();
            }
            // The last forward round of both operands, the pointwise product and
            // the first inverse round share one register round (their stage bits
            // coincide), as in the row pass.
            constexpr int EL = round_size(LR, NR - 1);
            static_assert(EL == dit_size(LR, 0), "mirrored rounds");
            const SmemIO<LR, 1, false> pair{X};  // NA = 2: X and Y = X + L
            const SmemIO<LR, 1, false> zs{Z};
            for (int g = threadIdx.x; g < (L >> EL); g += blockDim.x) {
                const int base = g << EL;
                uint32_t x[2][1 << EL];
                pair.template load<EL, 0, 2>(x, base, 0);
                dif_stages<EL, 0, 2, 0>(x, 0, T, q);
                uint32_t zz[1][1 << EL];
#pragma unroll
                for (int j = 0; j < (1 << EL); j++)
                    zz[0][j] = gb ? mul_mont<0>(x[0][j], x[1][j], q, qinv)
                                  : pmul<0>(x[0][j], x[1][j], sc, q, qinv);
                dit_stages<EL, 0, 1, 0>(zz, 0, Ti, q);
                zs.template store<EL, 0, 1>(zz, base, 0);
            }
            __syncthreads();
            round_io<LR, 1, dit_base(LR, 1), dit_size(LR, 1), false, 1, false, 0>(zs, zs, Ti, q);
            __syncthreads();
            if constexpr (NR == 3) {
                round_io<LR, 1, dit_base(LR, 2), dit_size(LR, 2), false, 1, false, 0>(zs, zs, Ti,
                                                                                      q);
                __syncthreads();
            }
        }
    }
    // each thread remainders its run of eight coefficients straight from the
    // swizzled residues (for a fixed i the lanes' words 8 t + i fall in
    // distinct banks under swz)
    __shared__ uint32_t hsm[96];
    const int j0 = threadIdx.x * kLimbsPerThread;
    CoefRun run;
#pragma unroll
    for (int i = 0; i < kLimbsPerThread; i++) {
        run.c0[i] = run.c1[i] = run.c2[i] = 0;
        if (j0 + i < L) {
            const int j = swz(j0 + i);
            crt3<0>(Rr[0][j], Rr[1][j], Rr[2][j], run.c0[i], run.c1[i], run.c2[i]);
        }
    }
    const Sink &o = a.sink;
    if (o.dec)
#pragma unroll
        for (int i = 0; i < kLimbsPerThread; i++) words_to_dec(run.c0[i], run.c1[i], run.c2[i]);
    uint32_t h1, h2a, h2b, map;
    run_halo(run, 0u, 0u, 0u, hsm, h1, h2a, h2b);
    tile_carry(run, h1, h2a, h2b, L, o.out + sink_node(o, k) * o.out_tstride, (long)o.out_len, o.dec,
               o.add ? o.add + k * o.add_tstride : nullptr, (long)o.add_len, wsm, &map);
}

// ------------------------------------------------------------ host side

struct NttPlan {
    int n = 0;
    int ncol = 0;
    int rcol[3] = {0, 0, 0};
    int rrow = 0;
};

// Row pass of up to 2^12 points (at least 2^4 so column passes keep 16
// columns), column passes of at most 2^10 rows, split as evenly as possible.
// A row-pass size tuned for this device (Ctx::row_log: rows of 2^9 .. 2^12
// points, at most two column passes of at least 2 rows, at least 2^4 rows in
// prime sets 1 and 2, whose column passes are built for 2^4 .. 2^10 rows)
// replaces the default.
bool plan_row_ok(int n, int rrow)
{
    if (n > kLogMaxNtt || rrow < 9 || rrow > kRowMaxLog) return false;
    const int rem = n - rrow;
    const int ncol = (rem + kColMaxLog - 1) / kColMaxLog;
    if (rem < 2 || ncol > 2) return false;
    return rem / ncol >= (set_for(n) == 0 ? 2 : kColMinLog);
}

static NttPlan make_plan(const Ctx &c, int n)
{
    NttPlan P;
    P.n = n;
    P.rrow = std::min(kRowMaxLog, n - kColMinLog);
    if (n <= kLogMaxNtt && c.row_log[n] && plan_row_ok(n, c.row_log[n])) P.rrow = c.row_log[n];
    int rem = n - P.rrow;
    P.ncol = (rem + kColMaxLog - 1) / kColMaxLog;
    for (int i = 0; i < P.ncol; i++) {
        P.rcol[i] = rem / (P.ncol - i);
        rem -= P.rcol[i];
    }
    std::sort(P.rcol, P.rcol + P.ncol, [](int x, int y) { return x > y; });
    return P;
}

// Raise the kernel's dynamic shared-memory limit when dynamic plus static
// shared memory (a few hundred bytes here) could pass the default 48 KiB.
template <typename K>
static void set_smem(K kernel, size_t bytes)
{
    if (bytes > 40 * 1024)
        CAT_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)bytes));
}

template <int LR, int PS>
static void launch_col(bool fwd, dim3 grid, cudaStream_t s, const ColArgs &a)
{
    const size_t smem = ((size_t)1 << (LR + col_log_c(LR))) * sizeof(uint32_t);
    // the first pass of operands of at most half the transform (every tree
    // level) knows its upper half is zero
    const bool zt = fwd && a.src && a.src_len <= ((size_t)1 << (a.m - 1));
    if (zt) {
        set_smem(ntt_col_fwd<LR, PS, kColV, true>, smem);
        ntt_col_fwd<LR, PS, kColV, true><<<grid, kColFwdThreads, smem, s>>>(a);
    } else if (fwd) {
        set_smem(ntt_col_fwd<LR, PS, kColV, false>, smem);
        ntt_col_fwd<LR, PS, kColV, false><<<grid, kColFwdThreads, smem, s>>>(a);
    } else {
        set_smem(ntt_col_inv<LR, PS, kColV>, smem);
        ntt_col_inv<LR, PS, kColV><<<grid, kColInvThreads, smem, s>>>(a);
    }
}

// ps: the prime set of the transform (set_for)
// The twiddles of a column pass of 2^r rows over blocks of 2^m points (set
// ps, direction dir): entry row 2^(m-r) + col = w^((col bitrev_r(row)) << shift)
// in Montgomery form, the value the pass would otherwise compute for that
// point (tw_pow_mont, exactly as the stepping reaches it).
// With scale (per prime, nonzero), every entry is multiplied by it mod q.
template <int PS>
__global__ void col_twiddle_table(const uint2 *tw, int m, int r, int dir, uint3 scale,
                                  uint32_t *tab)
{
    const int p = blockIdx.y;
    const uint32_t q = c_q[PS][p], qinv = c_qinv[PS][p];
    const uint32_t sp = p == 0 ? scale.x : (p == 1 ? scale.y : scale.z);
    const uint2 *T = tw_table(tw, PS, p, dir);
    const int shift = set_log_root(PS) - m;
    const uint32_t cols = 1u << (m - r);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < (1u << m);
         i += gridDim.x * blockDim.x) {
        const uint32_t row = i >> (m - r), col = i & (cols - 1);
        uint32_t v = tw_pow_mont<PS>(T, (col * bitrev(row, r)) << shift, q, qinv);
        if (sp) v = (uint32_t)((uint64_t)v * sp % q);
        tab[((size_t)p << m) + i] = v;
    }
}

// A column pass's twiddle table, built on first use; null when the context
// computes its twiddles (a budgeted context, or no room for the table).
// scaled: the entries times 2^(32-m) mod q, for operand b of a product whose
// pointwise step then needs no normalisation (forward first passes, m = n).
static const uint32_t *col_twiddles(Ctx &c, int ps, int m, int r, int dir, cudaStream_t s,
                                    bool scaled = false)
{
    if (!c.col_tw_tables || c.budget || c.shared_budget) return nullptr;
    for (const Ctx::ColTwTable &t : c.col_tw)
        if (t.ps == ps && t.m == m && t.lr == r && t.dir == dir && t.scaled == scaled) return t.p;
    uint32_t *p = nullptr;
    if (cudaMalloc(&p, ((size_t)kNumPrimes << m) * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    uint3 sc = make_uint3(0, 0, 0);
    if (scaled) {
        uint32_t v[kNumPrimes];
        for (int i = 0; i < kNumPrimes; i++) {
            const uint32_t q = ntt_prime(ps, i);
            v[i] = to_mont_c(powmod_u32((q + 1) / 2, (uint64_t)m, q), q);  // 2^32 2^-m
        }
        sc = make_uint3(v[0], v[1], v[2]);
    }
    const unsigned blocks = (unsigned)std::min<size_t>(((size_t)1 << m) / 256 + 1, 4096);
    const dim3 grid(blocks, kNumPrimes);
    if (ps == 0) col_twiddle_table<0><<<grid, 256, 0, s>>>(c.twiddles, m, r, dir, sc, p);
    else if (ps == 1) col_twiddle_table<1><<<grid, 256, 0, s>>>(c.twiddles, m, r, dir, sc, p);
    else col_twiddle_table<2><<<grid, 256, 0, s>>>(c.twiddles, m, r, dir, sc, p);
    CAT_LAUNCH("col_twiddle_table");
    c.col_tw.push_back(Ctx::ColTwTable{ps, m, r, dir, scaled, p});
    return p;
}

void drop_col_twiddles(Ctx &c)
{
    if (c.col_tw.empty()) return;
    cudaDeviceSynchronize();  // no pass still reads them
    for (const Ctx::ColTwTable &t : c.col_tw) cudaFree(t.p);
    c.col_tw.clear();
}

// scaled (first forward passes): 1 = every transform of the call is an
// operand b, 2 = the odd ones are (adjacent pairs); their twiddles then carry
// the pointwise step's normalisation.  Returns whether they did (the scaled
// table exists), i.e. whether the row pass must skip the normalisation.
static bool col_pass(Ctx &c, int ps, bool fwd, uint32_t *data, size_t pstride, size_t total,
                     int m, int r, const uint32_t *src, size_t src_tstride, size_t src_len,
                     cudaStream_t s, int scaled = 0)
{
    ColArgs a;
    a.twtab_odd = nullptr;
    // (measured per C(2,050,572,903): tables in every pass beat computed
    // twiddles at every block size, the first forward passes' large tables
    // included, once the table loads go through the read-only path)
    const int tmax = src ? c.col_tw_first_max_log : c.col_tw_max_log;
    a.twtab = m <= tmax ? col_twiddles(c, ps, m, r, fwd ? 0 : 1, s) : nullptr;
    bool prescaled = false;
    if (scaled && a.twtab) {
        const uint32_t *sct = col_twiddles(c, ps, m, r, 0, s, true);
        if (sct) {
            if (scaled == 1) a.twtab = sct;
            else a.twtab_odd = sct;
            prescaled = true;
        }
    }
    a.data = data;
    a.pstride = pstride;
    a.m = m;
    a.src = src;
    a.src_tstride = src_tstride;
    a.src_len = src_len;
    a.tw = c.twiddles;
    const size_t ctas = total >> (r + col_log_c(r));
    dim3 grid((unsigned)ctas, kNumPrimes);
    // algorithmic bytes: every point of the three prime arrays read and
    // written once (the first forward pass reads limbs instead)
    double bytes = 24.0 * (double)total;
    if (src) bytes = 12.0 * (double)total + 4.0 * (double)src_len * (double)(total >> m);
    const int tok = prof_begin(c, fwd ? (src ? "ntt_col_fwd_first" : "ntt_col_fwd") : "ntt_col_inv", s);
    if (ps == 0) {
        switch (r) {
        case 1: launch_col<1, 0>(fwd, grid, s, a); break;
        case 2: launch_col<2, 0>(fwd, grid, s, a); break;
        case 3: launch_col<3, 0>(fwd, grid, s, a); break;
        case 4: launch_col<4, 0>(fwd, grid, s, a); break;
        case 5: launch_col<5, 0>(fwd, grid, s, a); break;
        case 6: launch_col<6, 0>(fwd, grid, s, a); break;
        case 7: launch_col<7, 0>(fwd, grid, s, a); break;
        case 8: launch_col<8, 0>(fwd, grid, s, a); break;
        case 9: launch_col<9, 0>(fwd, grid, s, a); break;
        case 10: launch_col<10, 0>(fwd, grid, s, a); break;
        default: fail(CAT_EINVAL, "column pass size out of range");
        }
    } else if (ps == 1) {
        // 2^24 .. 2^26 points: default plans [6, 6], [7, 6], [7, 7] + 12; tuned
        // plans column passes of 2^4 .. 2^10 rows
        switch (r) {
        case 4: launch_col<4, 1>(fwd, grid, s, a); break;
        case 5: launch_col<5, 1>(fwd, grid, s, a); break;
        case 6: launch_col<6, 1>(fwd, grid, s, a); break;
        case 7: launch_col<7, 1>(fwd, grid, s, a); break;
        case 8: launch_col<8, 1>(fwd, grid, s, a); break;
        case 9: launch_col<9, 1>(fwd, grid, s, a); break;
        case 10: launch_col<10, 1>(fwd, grid, s, a); break;
        default: fail(CAT_EINVAL, "column pass size out of range");
        }
    } else {
        // 2^27 points: default plan [8, 7] + 12; tuned plans 2^4 .. 2^10 rows
        switch (r) {
        case 4: launch_col<4, 2>(fwd, grid, s, a); break;
        case 5: launch_col<5, 2>(fwd, grid, s, a); break;
        case 6: launch_col<6, 2>(fwd, grid, s, a); break;
        case 7: launch_col<7, 2>(fwd, grid, s, a); break;
        case 8: launch_col<8, 2>(fwd, grid, s, a); break;
        case 9: launch_col<9, 2>(fwd, grid, s, a); break;
        case 10: launch_col<10, 2>(fwd, grid, s, a); break;
        default: fail(CAT_EINVAL, "column pass size out of range");
        }
    }
    CAT_LAUNCH(fwd ? "ntt_col_fwd" : "ntt_col_inv");
    prof_end(c, tok, s, bytes);
    return prescaled;
}

template <int LR, int PS>
static void launch_row_t(dim3 grid, cudaStream_t s, const RowArgs &a, bool pre)
{
    if (a.prescaled && a.mode != PAIR_SQUARE && !pre) {  // operand b carries the scale
        const size_t smem = ((size_t)2 << kRowMaxLog) * sizeof(uint32_t);
        set_smem(ntt_row_mul_ns<LR, PS>, smem);
        ntt_row_mul_ns<LR, PS><<<grid, kRowThreads, smem, s>>>(a);
    } else if (pre) {  // broadcast products, the common transform complete
        const size_t smem = ((size_t)1 << kRowMaxLog) * sizeof(uint32_t);
        set_smem(ntt_row_mul_bcast<LR, PS>, smem);
        ntt_row_mul_bcast<LR, PS><<<grid, kRowThreads, smem, s>>>(a);
    } else if (a.mode == PAIR_SQUARE) {
        const size_t smem = ((size_t)1 << kRowMaxLog) * sizeof(uint32_t);
        set_smem(ntt_row_mul<LR, true, PS>, smem);
        ntt_row_mul<LR, true, PS><<<grid, kRowThreads, smem, s>>>(a);
    } else {
        const size_t smem = ((size_t)2 << kRowMaxLog) * sizeof(uint32_t);
        set_smem(ntt_row_mul<LR, false, PS>, smem);
        ntt_row_mul<LR, false, PS><<<grid, kRowThreads, smem, s>>>(a);
    }
}

// The fused row pass of nprod products of 2^n points with prime set ps
// (pre: broadcast products whose common transform ntt_row_fwd completed).
static void launch_row(int ps, int lr, size_t nprod, int n, cudaStream_t s, const RowArgs &a,
                       bool pre = false)
{
    dim3 grid((unsigned)(nprod << (n - kRowMaxLog)), kNumPrimes);
    if (ps == 0) {
        switch (lr) {
        case 9: launch_row_t<9, 0>(grid, s, a, pre); break;
        case 10: launch_row_t<10, 0>(grid, s, a, pre); break;
        case 11: launch_row_t<11, 0>(grid, s, a, pre); break;
        case 12: launch_row_t<12, 0>(grid, s, a, pre); break;
        default: fail(CAT_EINVAL, "row pass size out of range");
        }
    } else if (ps == 1) {
        switch (lr) {
        case 9: launch_row_t<9, 1>(grid, s, a, pre); break;
        case 10: launch_row_t<10, 1>(grid, s, a, pre); break;
        case 11: launch_row_t<11, 1>(grid, s, a, pre); break;
        case 12: launch_row_t<12, 1>(grid, s, a, pre); break;
        default: fail(CAT_EINVAL, "row pass size out of range");
        }
    } else {
        switch (lr) {
        case 9: launch_row_t<9, 2>(grid, s, a, pre); break;
        case 10: launch_row_t<10, 2>(grid, s, a, pre); break;
        case 11: launch_row_t<11, 2>(grid, s, a, pre); break;
        case 12: launch_row_t<12, 2>(grid, s, a, pre); break;
        default: fail(CAT_EINVAL, "row pass size out of range");
        }
    }
    CAT_LAUNCH("ntt_row_mul");
}

template <int LR, int PS>
static void launch_row_fwd_t(dim3 grid, cudaStream_t s, const RowArgs &a)
{
    const size_t smem = ((size_t)1 << kRowMaxLog) * sizeof(uint32_t);
    set_smem(ntt_row_fwd<LR, PS>, smem);
    ntt_row_fwd<LR, PS><<<grid, kRowThreads, smem, s>>>(a);
}

// The row pass's forward rounds of one transform of 2^n points in place (the
// common operand of broadcast products; a.F at its slot).
static void launch_row_fwd(int ps, int lr, int n, cudaStream_t s, const RowArgs &a)
{
    dim3 grid((unsigned)((size_t)1 << (n - kRowMaxLog)), kNumPrimes);
    switch (ps * 16 + lr) {
    case 9: launch_row_fwd_t<9, 0>(grid, s, a); break;
    case 10: launch_row_fwd_t<10, 0>(grid, s, a); break;
    case 11: launch_row_fwd_t<11, 0>(grid, s, a); break;
    case 12: launch_row_fwd_t<12, 0>(grid, s, a); break;
    case 16 + 9: launch_row_fwd_t<9, 1>(grid, s, a); break;
    case 16 + 10: launch_row_fwd_t<10, 1>(grid, s, a); break;
    case 16 + 11: launch_row_fwd_t<11, 1>(grid, s, a); break;
    case 16 + 12: launch_row_fwd_t<12, 1>(grid, s, a); break;
    case 32 + 9: launch_row_fwd_t<9, 2>(grid, s, a); break;
    case 32 + 10: launch_row_fwd_t<10, 2>(grid, s, a); break;
    case 32 + 11: launch_row_fwd_t<11, 2>(grid, s, a); break;
    case 32 + 12: launch_row_fwd_t<12, 2>(grid, s, a); break;
    default: fail(CAT_EINVAL, "row pass size out of range");
    }
    CAT_LAUNCH("ntt_row_fwd");
}

// Remaindering of a batch, specialised by prime set and by the sink's mode
// (base 10^9 or 2^32, with or without an addend).
template <int PS>
static void launch_crt_ps(unsigned grid, cudaStream_t s, const CrtArgs &a)
{
    const bool dec = a.sink.dec, add = a.sink.add != nullptr;
    if (dec && add)
        crt_carry_tiles<PS, true, true><<<grid, kTileThreads, 0, s>>>(a);
    else if (dec)
        crt_carry_tiles<PS, true, false><<<grid, kTileThreads, 0, s>>>(a);
    else if (add)
        crt_carry_tiles<PS, false, true><<<grid, kTileThreads, 0, s>>>(a);
    else
        crt_carry_tiles<PS, false, false><<<grid, kTileThreads, 0, s>>>(a);
}

static void launch_crt(int ps, unsigned grid, cudaStream_t s, const CrtArgs &a)
{
    if (ps == 0)
        launch_crt_ps<0>(grid, s, a);
    else if (ps == 1)
        launch_crt_ps<1>(grid, s, a);
    else
        launch_crt_ps<2>(grid, s, a);
}

// One operand source of a batched product.
struct Operand {
    const uint32_t *p;
    size_t tstride;  // limbs between consecutive transforms (for batches)
    size_t len;      // valid limbs per transform
};

// Batched products through the multi-pass transform, L = 2^n > 2^12.
//  mode PAIR_ADJACENT:  nprod products of transforms (2k, 2k+1) of `x`
//                       (2 nprod transforms, tstride apart);
//  mode PAIR_FIRST_TWO: one product of x and y;
//  mode PAIR_SQUARE:    nprod squares of x's transforms;
//  mode PAIR_BROADCAST: nprod products of x's transforms (tstride apart) with
//                       one y, whose transform is computed once.
static void ntt_mul_multipass(Ctx &c, int n, int mode, size_t nprod, Operand x, Operand y,
                              const Sink &sink, cudaStream_t s)
{
    const NttPlan P = make_plan(c, n);
    const int PS = set_for(n);
    const size_t L = (size_t)1 << n;
    const size_t ntf = mode == PAIR_ADJACENT ? 2 * nprod
                       : mode == PAIR_SQUARE ? nprod
                       : mode == PAIR_BROADCAST ? nprod + 1
                                                : 2;
    const size_t fp = ntf * L;
    DevBuf<uint32_t> F(c, fp * kNumPrimes, s);
    // forward column passes (operand b's first pass takes the pointwise
    // step's normalisation into its twiddles when it has a table)
    bool prescaled = false;
    if (mode == PAIR_FIRST_TWO) {
        col_pass(c, PS, true, F.get(), fp, L, n, P.rcol[0], x.p, 0, x.len, s);
        prescaled = col_pass(c, PS, true, F.get() + L, fp, L, n, P.rcol[0], y.p, 0, y.len, s, 1);
    } else if (mode == PAIR_BROADCAST) {
        col_pass(c, PS, true, F.get(), fp, nprod * L, n, P.rcol[0], x.p, x.tstride, x.len, s);
        col_pass(c, PS, true, F.get() + nprod * L, fp, L, n, P.rcol[0], y.p, 0, y.len, s);
    } else {
        prescaled = col_pass(c, PS, true, F.get(), fp, fp, n, P.rcol[0], x.p, x.tstride, x.len, s,
                             mode == PAIR_ADJACENT ? 2 : 0);
    }
    int m = n - P.rcol[0];
    for (int i = 1; i < P.ncol; i++) {
        col_pass(c, PS, true, F.get(), fp, fp, m, P.rcol[i], nullptr, 0, 0, s);
        m -= P.rcol[i];
    }
    // fused row pass
    const size_t gp = nprod * L;
    DevBuf<uint32_t> G(c, gp * kNumPrimes, s);
    RowArgs ra;
    ra.F = F.get();
    ra.fpstride = fp;
    ra.G = G.get();
    ra.gpstride = gp;
    ra.n = n;
    ra.mode = mode;
    ra.prescaled = prescaled ? 1 : 0;
    ra.tw = c.twiddles;
    ra.scale = make_scale(PS, n);
    // broadcast products: y's transform completed once, in its slot, so that
    // the row pass transforms only the x's
    const bool pre = mode == PAIR_BROADCAST && nprod >= 2;
    int tok;
    if (pre) {
        RowArgs ya = ra;
        ya.F = F.get() + nprod * L;
        tok = prof_begin(c, "ntt_row_fwd", s);
        launch_row_fwd(PS, P.rrow, n, s, ya);
        prof_end(c, tok, s, 8.0 * (double)L * kNumPrimes);
    }
    tok = prof_begin(c, "ntt_row_mul", s);
    launch_row(PS, P.rrow, nprod, n, s, ra, pre);
    // the products' own bytes: operands read and products written once
    const double unit = 4.0 * (double)nprod * (double)(x.len + sink.out_len) +
                        (mode == PAIR_SQUARE ? 0.0
                         : mode == PAIR_BROADCAST ? 4.0 * (double)y.len
                                                  : 4.0 * (double)nprod * (double)y.len);
    prof_end(c, tok, s, (mode == PAIR_SQUARE ? 24.0 : 36.0) * (double)gp, unit);
    F.reset();
    // inverse column passes, reverse order
    for (int i = P.ncol - 1; i >= 0; i--) {
        int mi = n;
        for (int j = 0; j < i; j++) mi -= P.rcol[j];
        col_pass(c, PS, false, G.get(), gp, gp, mi, P.rcol[i], nullptr, 0, 0, s);
    }
    // remaindering and carries
    const size_t tiles = L / kTile;
    DevBuf<uint8_t> maps(c, nprod * tiles, s);
    CrtArgs ca;
    ca.G = G.get();
    ca.gpstride = gp;
    ca.n = n;
    ca.sink = sink;
    ca.tile_maps = maps.get();
    tok = prof_begin(c, "crt_carry_tiles", s);
    launch_crt(PS, (unsigned)(nprod * tiles), s, ca);
    CAT_LAUNCH("crt_carry_tiles");
    prof_end(c, tok, s, 12.0 * (double)gp + 4.0 * (double)nprod * (double)sink.out_len);
    tok = prof_begin(c, "carry_tile_scan", s);
    carry_tile_scan<<<(unsigned)nprod, 1024, 0, s>>>(maps.get(), tiles);
    CAT_LAUNCH("carry_tile_scan");
    prof_end(c, tok, s, 2.0 * (double)(nprod * tiles));
    const size_t tt = nprod * tiles;
    tok = prof_begin(c, "carry_fix", s);
    carry_fix<<<(unsigned)((tt + 255) / 256), 256, 0, s>>>(maps.get(), tt, tiles, n, sink.out,
                                                             sink.out_tstride, sink.out_len,
                                                             sink.dec, sink.out_index);
    CAT_LAUNCH("carry_fix");
    prof_end(c, tok, s, (double)tt);
}

template <int LR>
static void launch_fused(unsigned grid, cudaStream_t s, const FusedArgs &a)
{
    const size_t smem = 6 * ((size_t)1 << LR) * sizeof(uint32_t);
    set_smem(ntt_mul_fused<LR>, smem);
    const int threads = std::min(kFusedThreads, std::max(64, (1 << LR) / 8));
    ntt_mul_fused<LR><<<grid, threads, smem, s>>>(a);
}

static void ntt_mul_small(Ctx &c, int n, size_t nprod, Operand x, Operand y, bool square,
                          const Sink &sink, cudaStream_t s)
{
    FusedArgs a;
    a.A = x.p;
    a.a_tstride = x.tstride;
    a.a_len = x.len;
    a.B = square ? nullptr : y.p;
    a.b_tstride = y.tstride;
    a.b_len = y.len;
    a.sink = sink;
    a.tw = c.twiddles;
    a.scale = make_scale(0, n);
    const unsigned grid = (unsigned)nprod;
    const int tok = prof_begin(c, "ntt_mul_fused", s);
    switch (n) {
    case 1: launch_fused<1>(grid, s, a); break;
    case 2: launch_fused<2>(grid, s, a); break;
    case 3: launch_fused<3>(grid, s, a); break;
    case 4: launch_fused<4>(grid, s, a); break;
    case 5: launch_fused<5>(grid, s, a); break;
    case 6: launch_fused<6>(grid, s, a); break;
    case 7: launch_fused<7>(grid, s, a); break;
    case 8: launch_fused<8>(grid, s, a); break;
    case 9: launch_fused<9>(grid, s, a); break;
    case 10: launch_fused<10>(grid, s, a); break;
    case 11: launch_fused<11>(grid, s, a); break;
    case 12: launch_fused<12>(grid, s, a); break;
    default: fail(CAT_EINVAL, "one-block transform size out of range");
    }
    CAT_LAUNCH("ntt_mul_fused");
    const double unit =
        4.0 * (double)nprod * (double)(x.len + (square ? 0 : y.len) + sink.out_len);
    prof_end(c, tok, s, unit, unit);
}

static int ceil_log2(size_t x)
{
    int n = 0;
    while (((size_t)1 << n) < x) n++;
    return n;
}

// Level products of the fixed-slot product tree: nprod products of adjacent
// slot-limb nodes of `level`, each written into a 2*slot-limb slot of out.
void ntt_level(Ctx &c, const uint32_t *level, size_t slot, size_t nprod, uint32_t *out,
               cudaStream_t s, const uint32_t *out_index, const uint32_t *out_index_host)
{
    const int n = ceil_log2(2 * slot);
    Operand x{level, slot, slot};
    if (n > c.max_log) {  // longer than one transform: each pair by pieces
        if (out_index && !out_index_host) fail(CAT_EINVAL, "indexed level needs its host table");
        for (size_t k = 0; k < nprod; k++) {
            uint32_t *o = out + 2 * (out_index ? (size_t)out_index_host[k] : k) * slot;
            CAT_CUDA(cudaMemsetAsync(o, 0, 8 * slot, s));
            mul_acc(c, level + 2 * k * slot, slot, level + (2 * k + 1) * slot, slot, o, 2 * slot,
                    false, s);
        }
        return;
    }
    Sink sink = plain_sink(out, 2 * slot, 2 * slot);
    sink.out_index = out_index;
    if (n <= kFusedMaxLog) {
        Operand a{level, 2 * slot, slot}, b{level + slot, 2 * slot, slot};
        ntt_mul_small(c, n, nprod, a, b, false, sink, s);
    } else {
        ntt_mul_multipass(c, n, PAIR_ADJACENT, nprod, x, x, sink, s);
    }
}

// out[0 .. na+nb) = a * b by the transform (na + nb <= 2^27).
void ntt_mul(Ctx &c, const uint32_t *a, size_t na, const uint32_t *b, size_t nb,
             uint32_t *out, cudaStream_t s)
{
    const size_t len = na + nb;
    const int n = std::max(1, ceil_log2(len));
    if (n > kLogMaxNtt) fail(CAT_EINVAL, "operands too long for one transform");
    const bool square = (a == b && na == nb);
    Operand x{a, 0, na}, y{b, 0, nb};
    if (n <= kFusedMaxLog) {
        ntt_mul_small(c, n, 1, x, y, square, plain_sink(out, 0, len), s);
    } else if (square) {
        ntt_mul_multipass(c, n, PAIR_SQUARE, 1, x, x, plain_sink(out, 0, len), s);
    } else {
        ntt_mul_multipass(c, n, PAIR_FIRST_TWO, 1, x, y, plain_sink(out, 0, len), s);
    }
}

// nprod products x_k y, x_k at x + k xstride (xlen limbs each), one y (ylen
// limbs), into `sink`; xlen + ylen <= 2^27.  y is transformed once.
void mul_broadcast(Ctx &c, const uint32_t *x, size_t xstride, size_t xlen, size_t nprod,
                   const uint32_t *y, size_t ylen, const Sink &sink, cudaStream_t s)
{
    if (nprod == 0) return;
    const int n = std::max(1, ceil_log2(xlen + ylen));
    if (n > kLogMaxNtt) fail(CAT_EINVAL, "operands too long for one transform");
    Operand ox{x, xstride, xlen}, oy{y, 0, ylen};
    if (nprod == 1 && x == y && xlen == ylen) {  // a square: one forward transform
        if (n <= kFusedMaxLog)
            ntt_mul_small(c, n, 1, ox, ox, true, sink, s);
        else
            ntt_mul_multipass(c, n, PAIR_SQUARE, 1, ox, ox, sink, s);
        return;
    }
    if (n <= kFusedMaxLog)
        ntt_mul_small(c, n, nprod, ox, oy, false, sink, s);
    else
        ntt_mul_multipass(c, n, PAIR_BROADCAST, nprod, ox, oy, sink, s);
}

// ------------------------------------------------ long products by pieces

// acc[j] += t[j] (t zero past tn) over one tile of 2048 limbs, carries within
// the tile; the tile's carry map goes to tile_maps.
__global__ void __launch_bounds__(kTileThreads) add_tiles(uint32_t *acc, size_t R,
                                                          const uint32_t *t, size_t tn, bool dec,
                                                          uint8_t *tile_maps)
{
    __shared__ uint32_t wsm[32];
    const size_t jt = (size_t)blockIdx.x * kTile;
    const int j0 = threadIdx.x * kLimbsPerThread;
    CoefRun run;
#pragma unroll
    for (int i = 0; i < kLimbsPerThread; i++) {
        const size_t j = jt + j0 + i;
        run.c0[i] = j < tn ? t[j] : 0u;
        run.c1[i] = run.c2[i] = 0u;
    }
    const int tile_len = (int)(R - jt < (size_t)kTile ? R - jt : (size_t)kTile);
    uint32_t map;
    tile_carry(run, 0u, 0u, 0u, tile_len, acc + jt, tile_len, dec, acc + jt, tile_len, wsm, &map);
    if (threadIdx.x == 0) tile_maps[blockIdx.x] = (uint8_t)map;
}

// acc[0 .. R) += t[0 .. tn) in base 2^32 or (dec) 10^9, the carries carried
// through all of acc (the sum must fit R limbs; limbs of t past R are zero).
void add_into(Ctx &c, uint32_t *acc, size_t R, const uint32_t *t, size_t tn, bool dec,
              cudaStream_t s)
{
    if (R == 0 || tn == 0) return;
    const size_t tiles = (R + kTile - 1) / kTile;
    if (tiles > 0x7fffffffu) fail(CAT_EINVAL, "addition too long");
    DevBuf<uint8_t> maps(c, tiles, s);
    const int tok = prof_begin(c, "add_tiles", s);
    add_tiles<<<(unsigned)tiles, kTileThreads, 0, s>>>(acc, R, t, tn, dec, maps.get());
    CAT_LAUNCH("add_tiles");
    carry_tile_scan<<<1, 1024, 0, s>>>(maps.get(), tiles);
    CAT_LAUNCH("carry_tile_scan");
    carry_fix<<<(unsigned)((tiles + 255) / 256), 256, 0, s>>>(maps.get(), tiles, tiles, 0, acc, 0,
                                                              R, dec);
    CAT_LAUNCH("carry_fix");
    prof_end(c, tok, s, 8.0 * (double)R + 4.0 * (double)tn);
}

// acc[0 .. R) += x y for operands of any length: pieces of Mx and My limbs
// with Mx + My <= 2^max_log, so that every piece product fits one transform,
// each added in at its offset (the sum must fit R limbs).  Both pieces are
// 2^(max_log - 1) limbs, or an operand shorter than that is one piece and the
// other takes the rest of the transform.
void mul_acc(Ctx &c, const uint32_t *x, size_t xlen, const uint32_t *y, size_t ylen,
             uint32_t *acc, size_t R, bool dec, cudaStream_t s)
{
    if (xlen == 0 || ylen == 0) return;
    const size_t L = (size_t)1 << c.max_log, M = L / 2;
    size_t Mx = M, My = M;
    if (xlen < M) {
        Mx = xlen;
        My = L - xlen;
    } else if (ylen < M) {
        My = ylen;
        Mx = L - ylen;
    }
    for (size_t i = 0; i < xlen; i += Mx)
        for (size_t j = 0; j < ylen; j += My) {
            if (i + j >= R) continue;
            const size_t lx = std::min(Mx, xlen - i), ly = std::min(My, ylen - j);
            DevBuf<uint32_t> t(c, lx + ly, s);
            mul_broadcast(c, x + i, 0, lx, 1, y + j, ly,
                          Sink{t.get(), 0, lx + ly, dec, nullptr, 0, 0}, s);
            add_into(c, acc + i + j, R - (i + j), t.get(), lx + ly, dec, s);
        }
}

// ------------------------------------------- unbalanced products by chunks

// The product of a long x (nx limbs) and a short y (ny limbs) from chunk
// products: chunk i = x[iM, iM + M) times y lies in slot i of T (M + ny
// words), and belongs at offset iM, so it overlaps the next chunk's product by
// ny limbs.  Limb j of the result sums t1 = slot k's word j - kM (k = j / M,
// the last slot also covers its tail) and t2 = slot k-1's word M + (j - kM)
// when j - kM < ny.  Per tile: run words c0[i] = t1(j0 + i) and c1[i] =
// t2(j0 + i + 1), so tile_carry's c1[j - 1] term adds t2(j) to limb j.
__device__ __forceinline__ void overlap_terms(const uint32_t *T, size_t M, size_t ny,
                                              size_t chunks, size_t j, uint32_t &t1,
                                              uint32_t &t2)
{
    size_t k = j / M;
    const bool past = k >= chunks;
    if (past) k = chunks - 1;
    const size_t r = j - k * M;
    t1 = r < M + ny ? T[k * (M + ny) + r] : 0u;
    t2 = (!past && k >= 1 && r < ny) ? T[(k - 1) * (M + ny) + M + r] : 0u;
}

__global__ void __launch_bounds__(kTileThreads) overlap_tiles(const uint32_t *T, size_t M,
                                                              size_t ny, size_t chunks,
                                                              uint32_t *out, size_t R,
                                                              uint8_t *tile_maps)
{
    __shared__ uint32_t wsm[32];
    __shared__ uint32_t hsm[96];
    const size_t jt = (size_t)blockIdx.x * kTile;
    const size_t j0 = jt + threadIdx.x * kLimbsPerThread;
    CoefRun run;
#pragma unroll
    for (int i = 0; i < kLimbsPerThread; i++) {
        uint32_t a = 0, b = 0, dummy = 0;
        if (j0 + i < R) overlap_terms(T, M, ny, chunks, j0 + i, a, dummy);
        if (j0 + i + 1 < R) overlap_terms(T, M, ny, chunks, j0 + i + 1, dummy, b);
        run.c0[i] = a;
        run.c1[i] = b;
        run.c2[i] = 0u;
    }
    uint32_t first1 = 0, dummy = 0;
    if (threadIdx.x == 0 && jt < R) overlap_terms(T, M, ny, chunks, jt, dummy, first1);
    uint32_t h1, h2a, h2b;
    run_halo(run, first1, 0u, 0u, hsm, h1, h2a, h2b);
    const int tile_len = (int)(R - jt < (size_t)kTile ? R - jt : (size_t)kTile);
    uint32_t map;
    tile_carry(run, h1, 0u, 0u, tile_len, out + jt, tile_len, false, nullptr, 0, wsm, &map);
    if (threadIdx.x == 0) tile_maps[blockIdx.x] = (uint8_t)map;
}

// out[0 .. nx + ny) = x y by chunks of M = 2^k - ny >= ny limbs of x, each
// multiplied by y in one batch (y transformed once).
void mul_chunked(Ctx &c, const uint32_t *x, size_t nx, const uint32_t *y, size_t ny, int k,
                 uint32_t *out, cudaStream_t s)
{
    const size_t L = (size_t)1 << k, M = L - ny, slot = L;
    if (ny == 0 || M < ny) fail(CAT_EINVAL, "chunk size below the short operand");
    const size_t full = nx / M, rem = nx - full * M, chunks = full + (rem ? 1 : 0);
    DevBuf<uint32_t> T(c, chunks * slot, s);
    if (full) mul_broadcast(c, x, M, M, full, y, ny, plain_sink(T.get(), slot, slot), s);
    if (rem) {
        uint32_t *last = T.get() + full * slot;
        CAT_CUDA(cudaMemsetAsync(last, 0, 4 * slot, s));
        mul_broadcast(c, x + full * M, 0, rem, 1, y, ny, plain_sink(last, 0, rem + ny), s);
    }
    const size_t R = nx + ny, tiles = (R + kTile - 1) / kTile;
    DevBuf<uint8_t> maps(c, tiles, s);
    const int tok = prof_begin(c, "overlap_tiles", s);
    overlap_tiles<<<(unsigned)tiles, kTileThreads, 0, s>>>(T.get(), M, ny, chunks, out, R,
                                                            maps.get());
    CAT_LAUNCH("overlap_tiles");
    carry_tile_scan<<<1, 1024, 0, s>>>(maps.get(), tiles);
    CAT_LAUNCH("carry_tile_scan");
    carry_fix<<<(unsigned)((tiles + 255) / 256), 256, 0, s>>>(maps.get(), tiles, tiles, 0, out, 0,
                                                              R, false);
    CAT_LAUNCH("carry_fix");
    prof_end(c, tok, s, 4.0 * (double)(chunks * slot) + 4.0 * (double)R);
}

// --------------------------------------- multiplication without allocation
//
// For callers that must not allocate device memory: code running where
// cudaMalloc is not allowed or not wanted (inside a host callback, a caller
// that owns all device memory through its own arena, or a process whose
// allocator is already saturated).  The transform scratch and the twiddle
// tables of this variant live in file-scope __device__ arrays of fixed size,
// reserved when the library is loaded, on every device that loads it, until
// the process exits.  Products of up to kNoAllocMaxLimbs limbs fit.

constexpr int kNoAllocLog = 16;
constexpr size_t kNoAllocMaxLimbs = (size_t)1 << kNoAllocLog;   // na + nb limit
constexpr size_t kNoAllocL = kNoAllocMaxLimbs;
// words: F (3 primes x 2 transforms x L), G (3 x L), tile maps, top index
constexpr size_t kNoAllocF = 6 * kNoAllocL;
constexpr size_t kNoAllocG = 3 * kNoAllocL;
constexpr size_t kNoAllocMapWords = 64;
constexpr size_t kNoAllocWords = kNoAllocF + kNoAllocG + kNoAllocMapWords + 2;

static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];
static __device__ __align__(256) uint2 g_noalloc_twiddles[kTwTotal];

// Largest i + 1 with x[i] != 0 into *top (which the caller clears).
__global__ void noalloc_top(const uint32_t *x, size_t n, unsigned long long *top)
{
    unsigned long long best = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        if (x[i]) best = i + 1;
    for (int off = 16; off; off >>= 1) {
        const unsigned long long o = __shfl_down_sync(0xffffffffu, best, off);
        best = o > best ? o : best;
    }
    if ((threadIdx.x & 31) == 0 && best) atomicMax(top, best);
}

struct NoAllocDevice {
    bool ready = false;
    uint32_t *scratch = nullptr;  // device address of g_noalloc_scratch
    uint2 *twiddles = nullptr;    // device address of g_noalloc_twiddles
};
static NoAllocDevice g_noalloc_dev[64];
static uint2 g_noalloc_tw_host[kTwTotal];

// Once per device, with that device current: resolve the device addresses of
// the two arrays and fill the twiddle table (same layout as the context's).
static std::mutex g_noalloc_mutex;

static int noalloc_setup(int dev)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoAllocDevice &d = g_noalloc_dev[dev];
    if (d.ready) return CAT_OK;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return CAT_ECUDA;
    d.scratch = (uint32_t *)p;
    if (cudaGetSymbolAddress(&p, g_noalloc_twiddles) != cudaSuccess) return CAT_ECUDA;
    d.twiddles = (uint2 *)p;
    try {
        twiddle_tables_host(g_noalloc_tw_host);
    } catch (...) {
        return CAT_ECUDA;
    }
    if (cudaMemcpyToSymbol(g_noalloc_twiddles, g_noalloc_tw_host, sizeof(g_noalloc_tw_host)) !=
        cudaSuccess)
        return CAT_ECUDA;
    try {
        upload_low_twiddles(g_noalloc_tw_host);
    } catch (...) {
        return CAT_ECUDA;
    }
    d.ready = true;
    return CAT_OK;
}

// The product through the same kernels as ntt_mul, with all scratch taken
// from the static array.
static void noalloc_mul(const NoAllocDevice &d, const uint32_t *a, size_t na, const uint32_t *b,
                        size_t nb, uint32_t *out, cudaStream_t s)
{
    Ctx local;  // no device resources: only the twiddle pointer is used
    local.twiddles = d.twiddles;
    local.col_tw_tables = false;  // the passes compute their twiddles: nothing allocated
    const size_t len = na + nb;
    const int n = std::max(1, ceil_log2(len));
    Operand x{a, 0, na}, y{b, 0, nb};
    if (n <= kFusedMaxLog) {
        ntt_mul_small(local, n, 1, x, y, false, plain_sink(out, 0, len), s);
        return;
    }
    const NttPlan P = make_plan(local, n);
    const size_t L = (size_t)1 << n;
    uint32_t *F = d.scratch;
    uint32_t *G = d.scratch + kNoAllocF;
    uint8_t *maps = (uint8_t *)(d.scratch + kNoAllocF + kNoAllocG);
    const size_t fp = 2 * L, gp = L;
    col_pass(local, 0, true, F, fp, L, n, P.rcol[0], x.p, 0, x.len, s);
    col_pass(local, 0, true, F + L, fp, L, n, P.rcol[0], y.p, 0, y.len, s);
    int m = n - P.rcol[0];
    for (int i = 1; i < P.ncol; i++) {
        col_pass(local, 0, true, F, fp, fp, m, P.rcol[i], nullptr, 0, 0, s);
        m -= P.rcol[i];
    }
    RowArgs ra;
    ra.F = F;
    ra.fpstride = fp;
    ra.G = G;
    ra.gpstride = gp;
    ra.n = n;
    ra.mode = PAIR_FIRST_TWO;
    ra.prescaled = 0;  // computed twiddles: the row pass normalises
    ra.tw = d.twiddles;
    ra.scale = make_scale(0, n);
    launch_row(0, P.rrow, 1, n, s, ra);
    for (int i = P.ncol - 1; i >= 0; i--) {
        int mi = n;
        for (int j = 0; j < i; j++) mi -= P.rcol[j];
        col_pass(local, 0, false, G, gp, gp, mi, P.rcol[i], nullptr, 0, 0, s);
    }
    const size_t tiles = L / kTile;
    CrtArgs ca;
    ca.G = G;
    ca.gpstride = gp;
    ca.n = n;
    ca.sink = plain_sink(out, 0, len);
    ca.tile_maps = maps;
    launch_crt(0, (unsigned)tiles, s, ca);
    CAT_LAUNCH("crt_carry_tiles");
    carry_tile_scan<<<1, 1024, 0, s>>>(maps, tiles);
    CAT_LAUNCH("carry_tile_scan");
    carry_fix<<<(unsigned)((tiles + 255) / 256), 256, 0, s>>>(maps, tiles, tiles, n, out, 0, len,
                                                            false);
    CAT_LAUNCH("carry_fix");
}

}  // namespace cat

extern "C" int bigint_mul_noalloc(const uint32_t *a, size_t na, const uint32_t *b, size_t nb,
                                  uint32_t *out, size_t cap, size_t *out_len, void *stream)
{
    using namespace cat;
    if (!out_len || (na && !a) || (nb && !b) || (cap && !out)) return CAT_EINVAL;
    // beyond the static scratch (written so that na + nb cannot wrap around)
    if (na > kNoAllocMaxLimbs || nb > kNoAllocMaxLimbs - na) return CAT_ENOMEM;
    if (cap < na + nb) return CAT_ERANGE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return CAT_ECUDA;
    const int rc = noalloc_setup(dev);
    if (rc != CAT_OK) return rc;
    const NoAllocDevice &d = g_noalloc_dev[dev];
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    try {
        if (na == 0 || nb == 0) {
            if (na + nb) CAT_CUDA(cudaMemsetAsync(out, 0, 4 * (na + nb), s));
            CAT_CUDA(cudaStreamSynchronize(s));
            *out_len = 0;
            return CAT_OK;
        }
        noalloc_mul(d, a, na, b, nb, out, s);
        unsigned long long *top = (unsigned long long *)(d.scratch + kNoAllocF + kNoAllocG +
                                                         kNoAllocMapWords);
        CAT_CUDA(cudaMemsetAsync(top, 0, sizeof(*top), s));
        noalloc_top<<<64, 256, 0, s>>>(out, na + nb, top);
        CAT_LAUNCH("noalloc_top");
        unsigned long long h = 0;
        CAT_CUDA(cudaMemcpyAsync(&h, top, sizeof(h), cudaMemcpyDeviceToHost, s));
        CAT_CUDA(cudaStreamSynchronize(s));
        *out_len = (size_t)h;
        return CAT_OK;
    } catch (const Error &e) {
        return e.code;
    } catch (...) {
        return CAT_ECUDA;
    }
}
