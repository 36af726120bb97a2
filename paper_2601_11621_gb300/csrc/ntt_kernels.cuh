// ntt_kernels.cuh -- the sub-transform engine and the pass kernels of the
// multi-pass NTT (included once by ntt.cu, after the constants, twiddle
// helpers and the remaindering code).
//
// A 2^LR-point sub-transform runs in "rounds" of up to four radix-2 stages.
// In a round covering stage bits [B, B + E), a thread holds the 2^E elements
// base + k 2^B (k < 2^E) of one group in registers and runs the E stages
// there.  The forward (DIF) rounds go from the top bits down, the inverse
// (DIT) rounds mirror them from the bottom up.  A pass kernel reads its first
// round straight from global memory and writes its last round straight to
// global memory; rounds in between exchange through shared memory (one
// barrier per round).  Stage s (half-span 2^s) multiplies by
// w_{2^(s+1)}^(i mod 2^s), entry 2^s + (i mod 2^s) of the stage table
// (2^(s+1) <= 2^13).
#pragma once

#include <type_traits>

__host__ __device__ constexpr int rounds_of(int lr) { return (lr + 3) / 4; }

// Whether an input of a register round knows that the upper half of its
// points (k >= 2^(E-1), the top stage's second inputs) are zero: the first
// forward round of an operand no longer than half the transform.
template <class T, class = void>
struct zero_top : std::false_type {};
template <class T>
struct zero_top<T, std::void_t<decltype(T::kZeroTop)>> : std::bool_constant<T::kZeroTop> {};

// size of DIF round rd of nr rounds (counted from the top stage bits); when
// the stages do not split evenly the last rounds take the extra ones, so that
// the round at stage bits [0, E) (which carries the column twiddles) is the
// largest
__host__ __device__ constexpr int round_size(int lr, int rd, int nr)
{
    return lr / nr + (rd >= nr - lr % nr ? 1 : 0);
}
__host__ __device__ constexpr int round_size(int lr, int rd)
{
    return round_size(lr, rd, rounds_of(lr));
}

// lowest stage bit of DIF round rd
__host__ __device__ constexpr int dif_base(int lr, int rd, int nr)
{
    int b = lr;
    for (int j = 0; j <= rd; j++) b -= round_size(lr, j, nr);
    return b;
}
__host__ __device__ constexpr int dif_base(int lr, int rd) { return dif_base(lr, rd, rounds_of(lr)); }

// DIT round rd (counted from the bottom) mirrors DIF round NR-1-rd
__host__ __device__ constexpr int dit_size(int lr, int rd, int nr)
{
    return round_size(lr, nr - 1 - rd, nr);
}
__host__ __device__ constexpr int dit_size(int lr, int rd) { return dit_size(lr, rd, rounds_of(lr)); }

__host__ __device__ constexpr int dit_base(int lr, int rd, int nr)
{
    int b = 0;
    for (int j = 0; j < rd; j++) b += dit_size(lr, j, nr);
    return b;
}
__host__ __device__ constexpr int dit_base(int lr, int rd) { return dit_base(lr, rd, rounds_of(lr)); }

// Shared-memory address swizzle: the bank bits of address a are XORed with a
// GF(2)-linear image f(t) of its row-of-32 index t = (a >> 5) mod 32, f
// sending the bits of t to 1, 10, 20, 24, 16.  In a round with base bit
// B < 5 the lanes of a warp differ in address bits [0, B) and in bits at and
// above B + E; f is chosen so that those five bits always land on five
// independent bank bits for the round shapes used here (E = 3 or 4 with
// B = 0, 3 or 4 on contiguous rows; the group bit 7 of 16-column tiles; in the
// column passes' interleaved tiles every shape from E = 2 to 4 at the bases
// they use, checked lane by lane), so no round has a bank conflict.  Rounds
// with B >= 5 are conflict-free under any such XOR.
__host__ __device__ constexpr int swz(int a)
{
    const int t = (a >> 5) & 31;
    return a ^ t ^ ((t & 6) << 2) ^ ((t & 8) << 1);
}

// The twiddles of one direction of one prime: the stage table in global
// memory, and the prime's index for the entries of stage bits below 4, which
// rounds with B = 0 read from constant memory (c_tw_low): their indices are
// compile-time constants, so the reads are uniform and need no registers.
struct TwRef {
    const uint2 *t;
    int prime;
};

template <int PS, int DIR, bool LOW>
__device__ __forceinline__ uint2 tw_at(const TwRef &T, int idx)
{
    if constexpr (LOW)
        return c_tw_low[PS][T.prime][DIR][idx];
    else
        return __ldg(&T.t[idx]);
}

// In a round with B = 0 the twiddle index is a compile-time constant, and the
// butterflies with (k mod 2^st) = 0 have twiddle w^0 = 1: no multiply.  With
// ZT the top stage's second inputs are zero, so its butterflies are
// (x, 0) -> (x, x w): one product, no sum or difference.
template <int E, int B, int NA, int PS, bool ZT = false>
__device__ __forceinline__ void dif_stages(uint32_t (&x)[NA][1 << E], int glow, const TwRef &T,
                                           uint32_t q)
{
#pragma unroll
    for (int st = E - 1; st >= 0; st--) {
#pragma unroll
        for (int k = 0; k < (1 << E); k++) {
            if (k & (1 << st)) continue;
            if (ZT && st == E - 1) {
                if (B == 0 && k == 0) {
#pragma unroll
                    for (int a = 0; a < NA; a++) x[a][k + (1 << st)] = x[a][k];
                } else {
                    const uint2 w = tw_at<PS, 0, (B == 0 && E <= 4)>(T, (1 << (B + st)) + glow +
                                                                            (k << B));
#pragma unroll
                    for (int a = 0; a < NA; a++) x[a][k + (1 << st)] = mul_w<PS>(x[a][k], w, q);
                }
                continue;
            }
            if (B == 0 && (k & ((1 << st) - 1)) == 0) {
#pragma unroll
                for (int a = 0; a < NA; a++) bf_dif1<PS>(x[a][k], x[a][k + (1 << st)], q);
                continue;
            }
            const int p = glow + ((k & ((1 << st) - 1)) << B);
            const uint2 w = tw_at<PS, 0, (B == 0 && E <= 4)>(T, (1 << (B + st)) + p);
#pragma unroll
            for (int a = 0; a < NA; a++) bf_dif<PS>(x[a][k], x[a][k + (1 << st)], w, q);
        }
    }
}

template <int E, int B, int NA, int PS>
__device__ __forceinline__ void dit_stages(uint32_t (&x)[NA][1 << E], int glow, const TwRef &Ti,
                                           uint32_t q)
{
#pragma unroll
    for (int st = 0; st < E; st++) {
#pragma unroll
        for (int k = 0; k < (1 << E); k++) {
            if (k & (1 << st)) continue;
            if (B == 0 && (k & ((1 << st) - 1)) == 0) {
#pragma unroll
                for (int a = 0; a < NA; a++) bf_dit1<PS>(x[a][k], x[a][k + (1 << st)], q);
                continue;
            }
            const int p = glow + ((k & ((1 << st) - 1)) << B);
            const uint2 w = tw_at<PS, 1, (B == 0 && E <= 4)>(Ti, (1 << (B + st)) + p);
#pragma unroll
            for (int a = 0; a < NA; a++) bf_dit<PS>(x[a][k], x[a][k + (1 << st)], w, q);
        }
    }
}

// One round over C independent sub-transforms ("columns") of 2^LR points:
// every group of this thread is loaded by `in`, transformed, and stored by
// `out`.  COLFAST: consecutive threads take consecutive columns (strided
// columns in global memory); otherwise consecutive threads take consecutive
// groups of one column (contiguous rows in global memory).  No barrier.
template <int LR, int C, int B, int E, bool FWD, int NA, bool COLFAST, int PS, class IN, class OUT>
__device__ __forceinline__ void round_io(const IN &in, const OUT &out, const TwRef &T, uint32_t q)
{
    constexpr int NGC = (1 << LR) >> E;  // groups per column
    constexpr int NG = C * NGC;
    for (int g = threadIdx.x; g < NG; g += blockDim.x) {
        const int c = COLFAST ? (g & (C - 1)) : (g / NGC);
        const int gg = COLFAST ? (g / C) : (g & (NGC - 1));
        const int glow = gg & ((1 << B) - 1);
        const int base = ((gg >> B) << (B + E)) | glow;
        uint32_t x[NA][1 << E];
        in.template load<E, B, NA>(x, base, c);
        if (FWD)
            dif_stages<E, B, NA, PS, zero_top<IN>::value>(x, glow, T, q);
        else
            dit_stages<E, B, NA, PS>(x, glow, T, q);
        out.template store<E, B, NA>(x, base, c);
    }
}

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }

// NA arrays of 2^LR x C words each, back to back, swizzled.  COLFAST: the
// columns interleave (point i of column c at i C + c); otherwise each column
// is contiguous (at c 2^LR + i).  A group's points base + k 2^B have offsets
// d_k = k 2^B (times C when interleaved) whose bits the group's own address
// a0 never has, and swz is linear over XOR on disjoint bits, so the swizzled
// address is swz(a0) ^ swz(d_k): one XOR with a compile-time constant.
template <int LR, int C, bool COLFAST>
struct SmemIO {
    uint32_t *s;
    static constexpr int LC = ilog2c(C);
    template <int B>
    __device__ __forceinline__ static int group_addr(int base, int c)
    {
        return COLFAST ? swz(base * C + c) : (c << LR) + swz(base);
    }
    template <int E, int B, int NA>
    __device__ __forceinline__ void load(uint32_t (&x)[NA][1 << E], int base, int c) const
    {
        constexpr int SH = COLFAST ? B + LC : B;
        const int a0 = group_addr<B>(base, c);
#pragma unroll
        for (int a = 0; a < NA; a++)
#pragma unroll
            for (int k = 0; k < (1 << E); k++)
                x[a][k] = s[a * ((1 << LR) * C) + (a0 ^ swz(k << SH))];
    }
    template <int E, int B, int NA>
    __device__ __forceinline__ void store(uint32_t (&x)[NA][1 << E], int base, int c) const
    {
        constexpr int SH = COLFAST ? B + LC : B;
        const int a0 = group_addr<B>(base, c);
#pragma unroll
        for (int a = 0; a < NA; a++)
#pragma unroll
            for (int k = 0; k < (1 << E); k++)
                s[a * ((1 << LR) * C) + (a0 ^ swz(k << SH))] = x[a][k];
    }
};

// All-shared-memory transforms (used by the one-block multiply) of C arrays
// of 2^LR words each, back to back (swizzled); every group holds one array's
// points, so a round has C 2^(LR - E) groups for the block's threads.  Caller
// synchronises before; these return synchronised.
template <int LR, int C, int PS>
__device__ __forceinline__ void dif_smem(uint32_t *s, const TwRef &T, uint32_t q)
{
    constexpr int NR = rounds_of(LR);
    SmemIO<LR, C, false> S{s};
    round_io<LR, C, dif_base(LR, 0), round_size(LR, 0), true, 1, false, PS>(S, S, T, q);
    __syncthreads();
    if constexpr (NR >= 2) {
        round_io<LR, C, dif_base(LR, 1), round_size(LR, 1), true, 1, false, PS>(S, S, T, q);
        __syncthreads();
    }
    if constexpr (NR >= 3) {
        round_io<LR, C, dif_base(LR, 2), round_size(LR, 2), true, 1, false, PS>(S, S, T, q);
        __syncthreads();
    }
}

template <int LR, int C, int PS>
__device__ __forceinline__ void dit_smem(uint32_t *s, const TwRef &Ti, uint32_t q)
{
    constexpr int NR = rounds_of(LR);
    SmemIO<LR, C, false> S{s};
    round_io<LR, C, dit_base(LR, 0), dit_size(LR, 0), false, 1, false, PS>(S, S, Ti, q);
    __syncthreads();
    if constexpr (NR >= 2) {
        round_io<LR, C, dit_base(LR, 1), dit_size(LR, 1), false, 1, false, PS>(S, S, Ti, q);
        __syncthreads();
    }
    if constexpr (NR >= 3) {
        round_io<LR, C, dit_base(LR, 2), dit_size(LR, 2), false, 1, false, PS>(S, S, Ti, q);
        __syncthreads();
    }
}

// ---------------------------------------------------------- column passes

// A column pass block holds C columns of 2^LR rows: 16 columns at 2^10 rows
// (64 KiB), otherwise 2^(13-LR) columns (8192 points, 32 KiB), so that
// every thread has a group to work on even for short columns.
// Launch shapes of the passes (compile-time knobs; the defaults are the
// fastest measured per C(2,050,572,903) on GB300, 142.0 -> 125.7 ms with the
// two-column groups below): threads per forward / inverse column-pass block,
// the most stages per register round in those passes, and the minimum
// resident blocks per SM of the row pass and of the forward column pass
// (which cap their registers at 64: four blocks per SM).
#ifndef CAT_COL_FWD_THREADS
#define CAT_COL_FWD_THREADS 256
#endif
#ifndef CAT_COL_INV_THREADS
#define CAT_COL_INV_THREADS 256
#endif
#ifndef CAT_COL_FWD_RMAX
#define CAT_COL_FWD_RMAX 4
#endif
#ifndef CAT_COL_INV_RMAX
#define CAT_COL_INV_RMAX 3
#endif
#ifndef CAT_ROW_MINB
#define CAT_ROW_MINB 4
#endif
#ifndef CAT_COL_FWD_MINB
#define CAT_COL_FWD_MINB 4
#endif
#ifndef CAT_COL_INV_MINB
#define CAT_COL_INV_MINB 1
#endif
__host__ __device__ constexpr int col_log_c(int lr) { return lr >= 10 ? 4 : 13 - lr; }
constexpr int kColFwdThreads = CAT_COL_FWD_THREADS;
constexpr int kColInvThreads = CAT_COL_INV_THREADS;
constexpr int kColMinLog = 4;   // columns of at least 2^4 rows
constexpr int kColMaxLog = 10;  // and at most 2^10
// Most stages per register round in the forward and inverse column passes
// (measured per C(2,050,572,903) with two-column groups: forward passes
// 39.2 -> 35.0 ms with four-stage rounds at 64 registers, inverse passes
// 17.7 ms with three-stage rounds against 18.9 with four).
constexpr int kColFwdRoundMax = CAT_COL_FWD_RMAX;
constexpr int kColInvRoundMax = CAT_COL_INV_RMAX;
__host__ __device__ constexpr int col_rounds(int lr, int most) { return (lr + most - 1) / most; }

struct ColArgs {
    uint32_t *data;        // prime p's array at data + p * pstride
    size_t pstride;
    int m;                 // block size 2^m (the sub-problem this pass splits)
    const uint32_t *src;   // first forward pass: limb source (else null)
    size_t src_tstride;    // limbs between consecutive transforms' sources
    size_t src_len;        // valid limbs per transform (rest are zero)
    const uint2 *tw;
    // the pass's inter-pass twiddles, w^(col bitrev(row)) in the multiplier
    // form the pass applies, point (row, col) of a 2^m block at row 2^(m-LR) +
    // col, 2^m per prime; null: the pass computes them
    const uint32_t *twtab;
    // first forward pass of adjacent pairs: the odd transforms' (operand b's)
    // table, its entries times 2^(32-m) (the pointwise product's 2^-m
    // normalisation taken in advance), or null
    const uint32_t *twtab_odd;
};

// Column tiles hold V adjacent columns per thread group: the group's V
// columns c V + a (a < V) are the V arrays of the register round (NA = V), so
// they share every stage twiddle, and global memory moves V adjacent words
// with one V-word access.  In shared memory array a holds the columns
// c V + a, back to back (SmemIO with C / V columns and NA = V).
#ifndef CAT_COL_V
#define CAT_COL_V 2
#endif
constexpr int kColV = CAT_COL_V;

template <int V>
__device__ __forceinline__ void load_v(const uint32_t *p, uint32_t (&w)[V])
{
    if constexpr (V == 4) {
        const uint4 t = *reinterpret_cast<const uint4 *>(p);
        w[0] = t.x; w[1] = t.y; w[2] = t.z; w[3] = t.w;
    } else if constexpr (V == 2) {
        const uint2 t = *reinterpret_cast<const uint2 *>(p);
        w[0] = t.x; w[1] = t.y;
    } else {
        w[0] = *p;
    }
}

// The same through the read-only path, for tables no kernel writes: the
// loads may then be issued ahead of the pass's own stores.
template <int V>
__device__ __forceinline__ void load_v_ro(const uint32_t *p, uint32_t (&w)[V])
{
    if constexpr (V == 4) {
        const uint4 t = __ldg(reinterpret_cast<const uint4 *>(p));
        w[0] = t.x; w[1] = t.y; w[2] = t.z; w[3] = t.w;
    } else if constexpr (V == 2) {
        const uint2 t = __ldg(reinterpret_cast<const uint2 *>(p));
        w[0] = t.x; w[1] = t.y;
    } else {
        w[0] = __ldg(p);
    }
}

template <int V>
__device__ __forceinline__ void store_v(uint32_t *p, const uint32_t (&w)[V])
{
    if constexpr (V == 4)
        *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    else if constexpr (V == 2)
        *reinterpret_cast<uint2 *>(p) = make_uint2(w[0], w[1]);
    else
        *p = w[0];
}

// Column tile in global memory: element (row, col) at p[row * S + col0 + col],
// group c covering columns c V .. c V + V - 1 (V-word aligned: S, col0 and
// the array bases are multiples of 16 words).  With `src`, elements come from
// limbs instead (zero past src_len, reduced), word by word, since a caller's
// limbs need not be aligned.
template <int PS, int V, bool ZT = false>
struct ColIn {
    // ZT: the first round of the first pass of an operand of at most half the
    // transform's length, whose points k >= 2^(E-1) lie in the zero upper half
    static constexpr bool kZeroTop = ZT;
    const uint32_t *p;
    const uint32_t *src;
    uint32_t S, col0, src_len;  // offsets within one transform fit in 32 bits
    uint32_t q, wp1;
    template <int E, int B, int NA>
    __device__ __forceinline__ void load(uint32_t (&x)[NA][1 << E], int base, int c) const
    {
        static_assert(NA == V, "one array per column of the group");
        const uint32_t i0 = (uint32_t)base * S + col0 + (uint32_t)c * V;
#pragma unroll
        for (int k = 0; k < (1 << E); k++) {
            if (ZT && k >= (1 << (E - 1))) {
#pragma unroll
                for (int a = 0; a < V; a++) x[a][k] = 0u;
                continue;
            }
            const uint32_t idx = i0 + (uint32_t)k * (S << B);
            if (src) {
#pragma unroll
                for (int a = 0; a < V; a++)
                    x[a][k] = idx + a < src_len ? reduce_in<PS>(src[idx + a], q, wp1) : 0u;
            } else {
                uint32_t w[V];
                load_v<V>(p + idx, w);
#pragma unroll
                for (int a = 0; a < V; a++) x[a][k] = w[a];
            }
        }
    }
};

__host__ __device__ constexpr int bitrev_c(int j, int bits)
{
    int r = 0;
    for (int b = 0; b < bits; b++) r |= ((j >> b) & 1) << (bits - 1 - b);
    return r;
}

// The twiddle w_M^(col * bitrev(row)) of the last forward (first inverse)
// round, whose groups are 2^E consecutive rows base + k (B = 0): with
// bitrev_LR(base + k) = bitrev_LR(base) + bitrev_E(k) 2^(LR - E) it is
// W0 U^bitrev_E(k), W0 = w^(col bitrev_LR(base)), U = w^(col 2^(LR - E)) (in
// units of the root order, hence the shift), so a group takes two table
// products and one Montgomery product per point to step through the powers,
// for each of its V columns.
template <int LR, int PS, int NR, int THREADS, int V>
struct ColTw {
    const uint2 *T;
    uint32_t q, qinv;
    int shift;      // log2(root order) - m
    uint32_t u[V];  // U of this thread's columns, when its groups share them
    // when set, the twiddles are read from this table (row stride S) instead
    const uint32_t *tab = nullptr;
    uint32_t S = 0;
    static constexpr int E = round_size(LR, NR - 1, NR);
    static constexpr int CV = (1 << col_log_c(LR)) / V;  // column groups per tile
    static constexpr bool kOneColumn = CV <= THREADS;
    __device__ __forceinline__ uint32_t step_of(uint32_t gcol) const
    {
        return tw_pow_mont<PS>(T, gcol << (LR - E + shift), q, qinv);
    }
    // Each thread's groups share their columns when the tile has at most as
    // many column groups as the block has threads (c = threadIdx mod CV): U
    // once per thread and column.
    __device__ __forceinline__ void init(uint32_t col0)
    {
        if (kOneColumn && !tab) {
            const uint32_t c0 = col0 + (threadIdx.x & (CV - 1)) * V;
#pragma unroll
            for (int a = 0; a < V; a++) u[a] = step_of(c0 + a);
        }
    }
    // f(k, v) for the group's rows k (in the order bitrev_E(j)), v[a] the
    // twiddle of column gcol + a at row base + k
    template <int EE, class F>
    __device__ __forceinline__ void each(uint32_t gcol, int base, F &&f) const
    {
        static_assert(EE == E, "twiddles are applied in the round at stage bits [0, E)");
        if (tab) {  // one table word per point (V adjacent columns in one access)
#pragma unroll
            for (int j = 0; j < (1 << E); j++) {
                const int k = bitrev_c(j, E);
                uint32_t w[V];
                load_v_ro<V>(tab + (uint32_t)(base + k) * S + gcol, w);
                f(k, w);
            }
            return;
        }
        const uint32_t br = bitrev((uint32_t)base, LR);
        uint32_t v[V], uu[V], up[V];
#pragma unroll
        for (int a = 0; a < V; a++) {
            v[a] = tw_pow_mont<PS>(T, ((gcol + a) * br) << shift, q, qinv);
            uu[a] = kOneColumn ? u[a] : step_of(gcol + a);
            up[a] = uu[a] * qinv;
        }
#pragma unroll
        for (int j = 0; j < (1 << E); j++) {
            f(bitrev_c(j, E), v);
            if (j + 1 < (1 << E))
#pragma unroll
                for (int a = 0; a < V; a++) v[a] = mont_step<PS>(v[a], uu[a], up[a], q);
        }
    }
};

// Forward pass output: element (row, col) times w_M^(col * bitrev(row)).
template <int LR, int PS, int NR, int V>
struct ColOutTw {
    uint32_t *p;
    uint32_t S, col0;
    ColTw<LR, PS, NR, kColFwdThreads, V> tw;
    template <int E, int B, int NA>
    __device__ __forceinline__ void store(uint32_t (&x)[NA][1 << E], int base, int c) const
    {
        static_assert(B == 0 && NA == V, "the twiddled round has contiguous rows");
        const uint32_t gcol = col0 + (uint32_t)c * V;
        const uint32_t i0 = (uint32_t)base * S + gcol;
        tw.template each<E>(gcol, base, [&](int k, const uint32_t(&v)[V]) {
            uint32_t w[V];
#pragma unroll
            for (int a = 0; a < V; a++) w[a] = mul_mont<PS>(x[a][k], v[a], tw.q, tw.qinv);
            store_v<V>(p + i0 + (uint32_t)k * S, w);
        });
    }
};

// Inverse pass input: element (row, col) times w_M^-(col * bitrev(row)).
template <int LR, int PS, int NR, int V>
struct ColInTw {
    const uint32_t *p;
    uint32_t S, col0;
    ColTw<LR, PS, NR, kColInvThreads, V> tw;
    template <int E, int B, int NA>
    __device__ __forceinline__ void load(uint32_t (&x)[NA][1 << E], int base, int c) const
    {
        static_assert(B == 0 && NA == V, "the twiddled round has contiguous rows");
        const uint32_t gcol = col0 + (uint32_t)c * V;
        const uint32_t i0 = (uint32_t)base * S + gcol;
        tw.template each<E>(gcol, base, [&](int k, const uint32_t(&v)[V]) {
            uint32_t w[V];
            load_v<V>(p + i0 + (uint32_t)k * S, w);
#pragma unroll
            for (int a = 0; a < V; a++) x[a][k] = mul_mont<PS>(w[a], v[a], tw.q, tw.qinv);
        });
    }
};

template <int V>
struct ColOut {
    uint32_t *p;
    uint32_t S, col0;
    template <int E, int B, int NA>
    __device__ __forceinline__ void store(uint32_t (&x)[NA][1 << E], int base, int c) const
    {
        static_assert(NA == V, "one array per column of the group");
        const uint32_t i0 = (uint32_t)base * S + col0 + (uint32_t)c * V;
#pragma unroll
        for (int k = 0; k < (1 << E); k++) {
            uint32_t w[V];
#pragma unroll
            for (int a = 0; a < V; a++) w[a] = x[a][k];
            store_v<V>(p + i0 + (uint32_t)k * (S << B), w);
        }
    }
};

// Forward column pass: a 2^LR-point DIF down each of C consecutive columns of
// one block (row stride S = 2^(m-LR)), then the twiddle w_M^(col * bitrev(row)).
template <int LR, int PS, int V, bool ZT>
__global__ void __launch_bounds__(kColFwdThreads, CAT_COL_FWD_MINB) ntt_col_fwd(ColArgs a)
{
    extern __shared__ uint32_t sm[];
    constexpr int LC = col_log_c(LR), C = 1 << LC, CV = C / V;
    // 2^4-row columns in one round, straight from global to global memory
    constexpr int NR = LR <= 4 ? 1 : col_rounds(LR, kColFwdRoundMax);
    static_assert(NR <= 4, "at most four rounds");
    const int p = blockIdx.y;
    const uint32_t q = c_q[PS][p];
    const size_t Sr = (size_t)1 << (a.m - LR);
    const size_t groups = Sr >> LC;
    const size_t blk = blockIdx.x / groups;
    const size_t col0 = (blockIdx.x % groups) << LC;
    uint32_t *base = a.data + p * a.pstride + (blk << a.m);
    const uint2 *T = tw_table(a.tw, PS, p, 0);
    const TwRef TR{T, p};
    const ColIn<PS, V, ZT> in{base, a.src ? a.src + blk * a.src_tstride : nullptr, (uint32_t)Sr,
                              (uint32_t)col0, (uint32_t)a.src_len, q, c_wp1[PS][p]};
    ColTw<LR, PS, NR, kColFwdThreads, V> tw{T, q, c_qinv[PS][p], set_log_root(PS) - a.m, {}};
    const uint32_t *tt = ((blk & 1) && a.twtab_odd) ? a.twtab_odd : a.twtab;
    if (tt) {
        tw.tab = tt + ((size_t)p << a.m);
        tw.S = (uint32_t)Sr;
    }
    tw.init((uint32_t)col0);
    const ColOutTw<LR, PS, NR, V> out{base, (uint32_t)Sr, (uint32_t)col0, tw};
    if constexpr (NR == 1) {
        round_io<LR, CV, 0, LR, true, V, true, PS>(in, out, TR, q);
    } else {
        const SmemIO<LR, CV, true> sio{sm};
        round_io<LR, CV, dif_base(LR, 0, NR), round_size(LR, 0, NR), true, V, true, PS>(in, sio,
                                                                                       TR, q);
        __syncthreads();
        if constexpr (NR >= 3) {
            round_io<LR, CV, dif_base(LR, 1, NR), round_size(LR, 1, NR), true, V, true, PS>(
                sio, sio, TR, q);
            __syncthreads();
        }
        if constexpr (NR >= 4) {
            round_io<LR, CV, dif_base(LR, 2, NR), round_size(LR, 2, NR), true, V, true, PS>(
                sio, sio, TR, q);
            __syncthreads();
        }
        round_io<LR, CV, 0, round_size(LR, NR - 1, NR), true, V, true, PS>(sio, out, TR, q);
    }
}

// Inverse column pass: undo the twiddle, then the DIT down each column.
template <int LR, int PS, int V>
__global__ void __launch_bounds__(kColInvThreads, CAT_COL_INV_MINB) ntt_col_inv(ColArgs a)
{
    extern __shared__ uint32_t sm[];
    constexpr int LC = col_log_c(LR), C = 1 << LC, CV = C / V;
    constexpr int NR = col_rounds(LR, kColInvRoundMax);
    static_assert(NR <= 4, "at most four rounds");
    const int p = blockIdx.y;
    const uint32_t q = c_q[PS][p];
    const size_t Sr = (size_t)1 << (a.m - LR);
    const size_t groups = Sr >> LC;
    const size_t blk = blockIdx.x / groups;
    const size_t col0 = (blockIdx.x % groups) << LC;
    uint32_t *base = a.data + p * a.pstride + (blk << a.m);
    const uint2 *Ti = tw_table(a.tw, PS, p, 1);
    const TwRef TRi{Ti, p};
    ColTw<LR, PS, NR, kColInvThreads, V> tw{Ti, q, c_qinv[PS][p], set_log_root(PS) - a.m, {}};
    if (a.twtab) {
        tw.tab = a.twtab + ((size_t)p << a.m);
        tw.S = (uint32_t)Sr;
    }
    tw.init((uint32_t)col0);
    const ColInTw<LR, PS, NR, V> in{base, (uint32_t)Sr, (uint32_t)col0, tw};
    const ColOut<V> out{base, (uint32_t)Sr, (uint32_t)col0};
    if constexpr (NR == 1) {
        round_io<LR, CV, 0, LR, false, V, true, PS>(in, out, TRi, q);
    } else {
        const SmemIO<LR, CV, true> sio{sm};
        round_io<LR, CV, 0, dit_size(LR, 0, NR), false, V, true, PS>(in, sio, TRi, q);
        __syncthreads();
        if constexpr (NR >= 3) {
            round_io<LR, CV, dit_base(LR, 1, NR), dit_size(LR, 1, NR), false, V, true, PS>(
                sio, sio, TRi, q);
            __syncthreads();
        }
        if constexpr (NR >= 4) {
            round_io<LR, CV, dit_base(LR, 2, NR), dit_size(LR, 2, NR), false, V, true, PS>(
                sio, sio, TRi, q);
            __syncthreads();
        }
        round_io<LR, CV, dit_base(LR, NR - 1, NR), dit_size(LR, NR - 1, NR), false, V, true, PS>(
            sio, out, TRi, q);
    }
}

// ------------------------------------------------------------ row pass

enum { PAIR_ADJACENT = 0, PAIR_SQUARE = 1, PAIR_FIRST_TWO = 2, PAIR_BROADCAST = 3 };

constexpr int kRowThreads = 256;
constexpr int kRowMaxLog = 12;
// rows of 2^LR points per block: 4096 points per block in all
__host__ __device__ constexpr int row_log_rows(int lr) { return kRowMaxLog - lr; }

struct RowArgs {
    const uint32_t *F;  // forward data after the column passes
    size_t fpstride;
    uint32_t *G;        // products (transform domain, then inverse rows)
    size_t gpstride;
    int n;              // log2 L
    int mode;           // which transforms product k multiplies
    int prescaled;      // operand b's transform already carries 2^(32-n): no scale
    const uint2 *tw;
    Scale scale;
};

// Consecutive rows in global memory (operands a, b): point i of row c at
// c 2^LR + i from the block's first row.
template <int LR>
struct RowIn {
    const uint32_t *pa, *pb;
    template <int E, int B, int NA>
    __device__ __forceinline__ void load(uint32_t (&x)[NA][1 << E], int base, int c) const
    {
#pragma unroll
        for (int k = 0; k < (1 << E); k++) {
            x[0][k] = pa[(c << LR) + base + (k << B)];
            if (NA > 1) x[NA - 1][k] = pb[(c << LR) + base + (k << B)];
        }
    }
};

// The product's inverse rounds with two rows per group (rows c and c + CH,
// CH = half the block's rows): they are the two arrays of the register round,
// so each stage twiddle and every index serves both rows.
#ifndef CAT_ROW_PAIR
#define CAT_ROW_PAIR 1
#endif

// The forward rounds but the last with two rows per group and both operands:
// arrays a-row c, a-row c + CH, b-row c, b-row c + CH (NA = 4, or 2 when
// squaring), which is the layout of SmemIO with CH columns and NA arrays.
#ifndef CAT_ROW_PAIR_FWD
#define CAT_ROW_PAIR_FWD 1
#endif

template <int LR, int CH>
struct RowInPair {
    const uint32_t *pa, *pb;
    template <int E, int B, int NA>
    __device__ __forceinline__ void load(uint32_t (&x)[NA][1 << E], int base, int c) const
    {
#pragma unroll
        for (int k = 0; k < (1 << E); k++) {
            x[0][k] = pa[(c << LR) + base + (k << B)];
            x[1][k] = pa[((c + CH) << LR) + base + (k << B)];
            if (NA > 2) {
                x[NA - 2][k] = pb[(c << LR) + base + (k << B)];
                x[NA - 1][k] = pb[((c + CH) << LR) + base + (k << B)];
            }
        }
    }
};

template <int LR, int CH>
struct RowOutPair {
    uint32_t *p;
    template <int E, int B, int NA>
    __device__ __forceinline__ void store(uint32_t (&x)[NA][1 << E], int base, int c) const
    {
#pragma unroll
        for (int a = 0; a < NA; a++)
#pragma unroll
            for (int k = 0; k < (1 << E); k++) p[((c + a * CH) << LR) + base + (k << B)] = x[a][k];
    }
};

template <int LR>
struct RowOut {
    uint32_t *p;
    template <int E, int B, int NA>
    __device__ __forceinline__ void store(uint32_t (&x)[NA][1 << E], int base, int c) const
    {
#pragma unroll
        for (int k = 0; k < (1 << E); k++) p[(c << LR) + base + (k << B)] = x[0][k];
    }
};

// Last forward pass of both operands (or one, squaring), pointwise product
// and first inverse pass, on 2^(12-LR) consecutive rows of 2^LR points of
// product k.  The last forward round, the product and the first inverse round
// share one register round (their stage bits coincide).  YH (broadcast
// products): the common operand's transform is already complete in its slot
// (ntt_row_fwd), in the order the product loop reads it, so only x is
// transformed here.
template <int LR, bool SQ, int PS, bool YH, bool NS = false>
__device__ __forceinline__ void row_mul_body(const RowArgs &a, uint32_t *sm)
{
    constexpr int NR = rounds_of(LR);
    constexpr int NA = (SQ || YH) ? 1 : 2;
    constexpr int EL = round_size(LR, NR - 1);
    constexpr int RB = row_log_rows(LR), C = 1 << RB;
    static_assert(EL == dit_size(LR, 0), "mirrored rounds");
    const int p = blockIdx.y;
    const uint32_t q = c_q[PS][p], qinv = c_qinv[PS][p];
    const size_t blocks = (size_t)1 << (a.n - LR - RB);  // row blocks per product
    const size_t k = blockIdx.x / blocks;
    const size_t off = (blockIdx.x % blocks) << (LR + RB);
    size_t ta, tb;
    if (a.mode == PAIR_ADJACENT) { ta = 2 * k; tb = 2 * k + 1; }
    else if (a.mode == PAIR_SQUARE) { ta = k; tb = k; }
    else if (a.mode == PAIR_BROADCAST) { ta = k; tb = gridDim.x / blocks; }  // y after the x's
    else { ta = 0; tb = 1; }
    const uint32_t *fa = a.F + p * a.fpstride + (ta << a.n) + off;
    const uint32_t *fb = a.F + p * a.fpstride + (tb << a.n) + off;
    const TwRef T{tw_table(a.tw, PS, p, 0), p};
    const TwRef Ti{tw_table(a.tw, PS, p, 1), p};
    const uint2 sc = p == 0 ? a.scale.c[0] : (p == 1 ? a.scale.c[1] : a.scale.c[2]);
    const SmemIO<LR, C, false> sio{sm};
    // forward rounds but the last, two rows per group when every thread still
    // gets a group
    constexpr int CF = C / 2 > 0 ? C / 2 : 1;
    constexpr bool kPairFwd =
        CAT_ROW_PAIR_FWD && C >= 2 && CF * ((1 << LR) >> round_size(LR, 0)) >= kRowThreads &&
        (NR == 2 || CF * ((1 << LR) >> round_size(LR, 1)) >= kRowThreads);
    if constexpr (kPairFwd) {
        const SmemIO<LR, CF, false> sp{sm};
        round_io<LR, CF, dif_base(LR, 0), round_size(LR, 0), true, 2 * NA, false, PS>(
            RowInPair<LR, CF>{fa, fb}, sp, T, q);
        __syncthreads();
        if constexpr (NR == 3) {
            round_io<LR, CF, dif_base(LR, 1), round_size(LR, 1), true, 2 * NA, false, PS>(sp, sp, T,
                                                                                       q);
            __syncthreads();
        }
    } else {
        round_io<LR, C, dif_base(LR, 0), round_size(LR, 0), true, NA, false, PS>(
            RowIn<LR>{fa, fb}, sio, T, q);
        __syncthreads();
        if constexpr (NR == 3) {
            round_io<LR, C, dif_base(LR, 1), round_size(LR, 1), true, NA, false, PS>(sio, sio, T,
                                                                                   q);
            __syncthreads();
        }
    }
    // last forward round + pointwise product + first inverse round
    constexpr int NGC = (1 << LR) >> EL;
    for (int g = threadIdx.x; g < C * NGC; g += blockDim.x) {
        const int c = g / NGC;
        const int base = (g & (NGC - 1)) << EL;
        uint32_t x[NA][1 << EL];
        sio.template load<EL, 0, NA>(x, base, c);
        dif_stages<EL, 0, NA, PS>(x, 0, T, q);
        uint32_t yv[1 << EL];
        if constexpr (YH) {
            static_assert(EL >= 2, "the common transform is read 16 bytes at a time");
            const uint4 *y4 = reinterpret_cast<const uint4 *>(fb + (c << LR) + base);
#pragma unroll
            for (int j = 0; j < (1 << EL) / 4; j++) {
                const uint4 v = y4[j];
                yv[4 * j] = v.x; yv[4 * j + 1] = v.y; yv[4 * j + 2] = v.z; yv[4 * j + 3] = v.w;
            }
        }
        uint32_t z[1][1 << EL];
#pragma unroll
        for (int j = 0; j < (1 << EL); j++)
            z[0][j] = NS ? mul_mont<PS>(x[0][j], x[NA - 1][j], q, qinv)
                         : pmul<PS>(x[0][j], YH ? yv[j] : x[NA - 1][j], sc, q, qinv);
        dit_stages<EL, 0, 1, PS>(z, 0, Ti, q);
        sio.template store<EL, 0, 1>(z, base, c);
    }
    __syncthreads();
    uint32_t *g = a.G + p * a.gpstride + (k << a.n) + off;
    // rows in pairs when the block has two rows or more and the paired rounds
    // still give every thread a group; the single-array layout (row r at
    // r 2^LR) is the paired layout's (array a at a CH 2^LR, column c at c 2^LR)
    constexpr int CH = C / 2 > 0 ? C / 2 : 1;
    constexpr bool kPair =
        CAT_ROW_PAIR && C >= 2 && CH * ((1 << LR) >> dit_size(LR, 1)) >= kRowThreads &&
        (NR == 2 || CH * ((1 << LR) >> dit_size(LR, 2)) >= kRowThreads);
    if constexpr (kPair) {
        const SmemIO<LR, CH, false> sp{sm};
        if constexpr (NR == 2) {
            round_io<LR, CH, dit_base(LR, 1), dit_size(LR, 1), false, 2, false, PS>(
                sp, RowOutPair<LR, CH>{g}, Ti, q);
        } else {
            round_io<LR, CH, dit_base(LR, 1), dit_size(LR, 1), false, 2, false, PS>(sp, sp, Ti, q);
            __syncthreads();
            round_io<LR, CH, dit_base(LR, 2), dit_size(LR, 2), false, 2, false, PS>(
                sp, RowOutPair<LR, CH>{g}, Ti, q);
        }
    } else if constexpr (NR == 2) {
        round_io<LR, C, dit_base(LR, 1), dit_size(LR, 1), false, 1, false, PS>(sio, RowOut<LR>{g},
                                                                               Ti, q);
    } else {
        round_io<LR, C, dit_base(LR, 1), dit_size(LR, 1), false, 1, false, PS>(sio, sio, Ti, q);
        __syncthreads();
        round_io<LR, C, dit_base(LR, 2), dit_size(LR, 2), false, 1, false, PS>(sio, RowOut<LR>{g},
                                                                               Ti, q);
    }
}

template <int LR, bool SQ, int PS>
__global__ void __launch_bounds__(kRowThreads, CAT_ROW_MINB) ntt_row_mul(RowArgs a)
{
    extern __shared__ uint32_t sm[];
    row_mul_body<LR, SQ, PS, false>(a, sm);
}

// Products whose operand b transform already carries the normalisation
// 2^(32-n) (its first pass took the scaled twiddle table): the pointwise
// product is one Montgomery product.
template <int LR, int PS>
__global__ void __launch_bounds__(kRowThreads, CAT_ROW_MINB) ntt_row_mul_ns(RowArgs a)
{
    extern __shared__ uint32_t sm[];
    row_mul_body<LR, false, PS, false, true>(a, sm);
}

// Broadcast products x_k y whose y transform ntt_row_fwd has completed.
template <int LR, int PS>
__global__ void __launch_bounds__(kRowThreads, CAT_ROW_MINB) ntt_row_mul_bcast(RowArgs a)
{
    extern __shared__ uint32_t sm[];
    row_mul_body<LR, false, PS, true>(a, sm);
}

// The row pass's forward rounds alone, for the common operand y of broadcast
// products: a.F points at y's slot, 2^(12-LR) consecutive rows of 2^LR points
// per block; the last forward round's output goes back to the same rows,
// point base + j of row c at (c << LR) + base + j (the order in which the
// product loop of ntt_row_mul_bcast reads it).  Each block reads its rows
// into shared memory before it writes any of them.
template <int LR, int PS>
__global__ void __launch_bounds__(kRowThreads, CAT_ROW_MINB) ntt_row_fwd(RowArgs a)
{
    extern __shared__ uint32_t sm[];
    constexpr int NR = rounds_of(LR);
    constexpr int EL = round_size(LR, NR - 1);
    constexpr int RB = row_log_rows(LR), C = 1 << RB;
    static_assert(EL >= 2, "rows are written 16 bytes at a time");
    const int p = blockIdx.y;
    const uint32_t q = c_q[PS][p];
    const size_t off = (size_t)blockIdx.x << (LR + RB);
    uint32_t *fy = const_cast<uint32_t *>(a.F) + p * a.fpstride + off;
    const TwRef T{tw_table(a.tw, PS, p, 0), p};
    const SmemIO<LR, C, false> sio{sm};
    constexpr int CF = C / 2 > 0 ? C / 2 : 1;
    constexpr bool kPairFwd =
        CAT_ROW_PAIR_FWD && C >= 2 && CF * ((1 << LR) >> round_size(LR, 0)) >= kRowThreads &&
        (NR == 2 || CF * ((1 << LR) >> round_size(LR, 1)) >= kRowThreads);
    if constexpr (kPairFwd) {
        const SmemIO<LR, CF, false> sp{sm};
        round_io<LR, CF, dif_base(LR, 0), round_size(LR, 0), true, 2, false, PS>(
            RowInPair<LR, CF>{fy, fy}, sp, T, q);
        __syncthreads();
        if constexpr (NR == 3) {
            round_io<LR, CF, dif_base(LR, 1), round_size(LR, 1), true, 2, false, PS>(sp, sp, T, q);
            __syncthreads();
        }
    } else {
        round_io<LR, C, dif_base(LR, 0), round_size(LR, 0), true, 1, false, PS>(
            RowIn<LR>{fy, fy}, sio, T, q);
        __syncthreads();
        if constexpr (NR == 3) {
            round_io<LR, C, dif_base(LR, 1), round_size(LR, 1), true, 1, false, PS>(sio, sio, T, q);
            __syncthreads();
        }
    }
    constexpr int NGC = (1 << LR) >> EL;
    for (int g = threadIdx.x; g < C * NGC; g += blockDim.x) {
        const int c = g / NGC;
        const int base = (g & (NGC - 1)) << EL;
        uint32_t x[1][1 << EL];
        sio.template load<EL, 0, 1>(x, base, c);
        dif_stages<EL, 0, 1, PS>(x, 0, T, q);
        uint4 *o4 = reinterpret_cast<uint4 *>(fy + (c << LR) + base);
#pragma unroll
        for (int j = 0; j < (1 << EL) / 4; j++)
            o4[j] = make_uint4(x[0][4 * j], x[0][4 * j + 1], x[0][4 * j + 2], x[0][4 * j + 3]);
    }
}
