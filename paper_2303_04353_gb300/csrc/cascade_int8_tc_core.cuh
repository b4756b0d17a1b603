// The tcgen05 INT8-form kernel (see cascade_int8_tc.cu for the method),
// templated on where its tiles come from: one problem (cascade_int8_tc.cu)
// or a planned list of (problem, tile) items (batched_int8_tc.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>

#include "dd_device.cuh"
#include "ddgemm_internal.h"
#include "tma.cuh"
#include "umma.cuh"

namespace ddg {
namespace {

constexpr int BM = INT8_TC_BM, BN = INT8_TC_BN, BK = 16;
// What follows from the digit width TB of the pieces: the chunk over which
// an FP32 accumulator stays exact (up to 16 products of |digit| <= 2^(TB-1)
// per entry, so 2^24 / (16 2^(2 TB - 2)) entries: 256 for seven bits, 64
// for eight), the chunks per k-block, and the split of a block value
// T = H 2^SPLIT + L (L holds the eight smallest diagonals).
template <int TB>
struct TcWidth {
    static constexpr int CHUNK_STEPS = (1 << 24) / (16 << (2 * TB - 2)) / 16;  // k-steps of 16
    static constexpr int BLOCK_CHUNKS = kblock_of_bits(TB) / (BK * CHUNK_STEPS);
    static constexpr int SPLIT = 8 * TB;
    static_assert(TB == 7 || TB == 8, "seven- or eight-bit pieces");
    static_assert(CHUNK_STEPS >= 1 && SPLIT <= 64, "digit width");
};
// Drain warps: four per tensor-memory lane quadrant (a warp reaches only the
// quadrant warp % 4), each taking DCOLS of the 16 columns of every diagonal.
// Sixteen warps hide the read-out latency better than eight and leave each
// thread half the state (its outputs' exact block values).
constexpr int EPI_WARPS = 16;
constexpr int DRAIN_PARTS = EPI_WARPS / 4;
constexpr int DCOLS = BN / DRAIN_PARTS;
static_assert(DCOLS == 4, "the drain reads 4 columns per diagonal");
constexpr int NTHREADS = 32 * (2 + EPI_WARPS);
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t ACC_STRIDE = 256;                  // columns between the two sets
constexpr int TILE_GROUP = 4;

constexpr int MAX_SMEM = 227 * 1024;                  // dynamic shared memory per CTA
constexpr int BAR_BYTES = 256;

template <int S>
struct TcGeom {
    static constexpr int A_PLANE = BM * BK * 2;       // 4 KB
    static constexpr int B_PLANE = BN * BK * 2;       // 512 bytes
    static constexpr int A_STAGE = S * A_PLANE;
    static constexpr int TX = S * (A_PLANE + B_PLANE);  // bytes the two copies deliver
    static constexpr int STAGE = (TX + 1023) / 1024 * 1024;
    // as many stages as fit, at most 4 (3 at s = 16)
    static constexpr int NST_FIT = (MAX_SMEM - BAR_BYTES - 1024) / STAGE;
    static constexpr int NST = NST_FIT < 4 ? NST_FIT : 4;
    static constexpr size_t SMEM = (size_t)NST * STAGE + BAR_BYTES + 1024;
    static_assert(NST >= 2, "at least two stages");
    static_assert(S * BN <= (int)ACC_STRIDE, "one accumulator set is 16 s columns");
};

template <int NST>
struct Shared {
    uint64_t full[NST], empty[NST], acc_full[2], acc_empty[2], mma_done;
    uint32_t tmem_base;
    int abort_flag;
};

// A wait bounded by limit_ns that also gives up when another role has
// aborted.  sleep_ns > 0: sleep between polls (the drain warps, which share
// their SM sub-partitions with the copy and MMA threads and can wait a
// little longer: measured 0.8 % off the eight-bit form at 4096^3).
template <class SH>
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, SH *sh,
                                              unsigned int *status, uint64_t limit_ns,
                                              unsigned sleep_ns = 0) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    volatile int *flag = &sh->abort_flag;
    while (!mbar_try_wait(bar, parity)) {
        if (*flag) return false;
        if (global_ns() - t0 > limit_ns) {
            *flag = 1;
            if (status) atomicOr(status, DEV_TIMEOUT_BIT);
            return false;
        }
        if (sleep_ns) __nanosleep(sleep_ns);
    }
    return true;
}

__device__ __forceinline__ int bitlen128(unsigned __int128 x) {
    const unsigned long long h = (unsigned long long)(x >> 64), l = (unsigned long long)x;
    if (h) return 128 - __clzll((long long)h);
    return l ? 64 - __clzll((long long)l) : 0;
}

// m 2^e as a double, for 0 < m <= 2^53 (every such m is exact in a double):
// the IEEE bits are put together on the integer pipes when the result is a
// normal number (the FP64 pipe is narrow on this GPU and the epilogues run
// this per output), otherwise scalbn does it.
__device__ __forceinline__ double scaled(unsigned long long m, int e) {
    const int b = 64 - __clzll((long long)m);  // 1 .. 54
    if (b > 53) {                              // m = 2^53
        m >>= 1;
        e += 1;
    } else {
        m <<= 53 - b;
        e -= 53 - b;
    }
    const int be = e + 52 + 1023;              // biased exponent of m 2^e
    if (be >= 1 && be <= 2046)
        return __longlong_as_double(((long long)be << 52) | (long long)(m & ((1ull << 52) - 1)));
    return scalbn((double)m, e);
}

__device__ __forceinline__ double with_sign(double v, bool neg) {
    return __longlong_as_double(__double_as_longlong(v) ^ ((long long)neg << 63));
}

// Nearest double (ties to even) to the signed integer r times 2^e, |r| < 2^127.
__device__ __forceinline__ double round_int(__int128 r, int e) {
    if (r == 0) return 0.0;
    const bool neg = r < 0;
    const unsigned __int128 u = neg ? (unsigned __int128)(-r) : (unsigned __int128)r;
    const int q = bitlen128(u);
    double v;
    if (q <= 53) {
        v = scaled((unsigned long long)u, e);
    } else {
        const int sh = q - 53;
        unsigned long long m = (unsigned long long)(u >> sh);
        const unsigned __int128 rem = u & (((unsigned __int128)1 << sh) - 1);
        const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
        if (rem > half || (rem == half && (m & 1ull))) ++m;
        v = scaled(m, sh + e);
    }
    return with_sign(v, neg);
}

// The FP64x2 nearest to T 2^e with T = H 2^SPLIT + L (|H| < 2^80,
// |L| < 2^90, SPLIT <= 64): hi = RN(T 2^e), lo = RN(T 2^e - hi).
template <int SPLIT>
__device__ __forceinline__ void round_dd(__int128 H, __int128 L, int e, double &hi, double &lo) {
    // carry L's bits above 2^SPLIT into H: T = H1 2^SPLIT + L0,
    // 0 <= L0 < 2^SPLIT (floor division)
    const __int128 unit = (__int128)1 << SPLIT;
    const __int128 qs = L / unit;
    const __int128 carry = (L < 0 && qs * unit != L) ? qs - 1 : qs;
    const unsigned long long L0 = (unsigned long long)(L - carry * unit);
    __int128 H1 = H + carry;
    const bool neg = H1 < 0;
    unsigned __int128 Hm;
    unsigned long long Lm;
    if (!neg) {
        Hm = (unsigned __int128)H1;
        Lm = L0;
    } else if (L0 != 0) {  // -T = (-H1 - 1) 2^SPLIT + (2^SPLIT - L0)
        Hm = (unsigned __int128)(-H1 - 1);
        Lm = (unsigned long long)(unit - (__int128)L0);
    } else {
        Hm = (unsigned __int128)(-H1);
        Lm = 0;
    }
    if (Hm == 0 && Lm == 0) {
        hi = 0.0;
        lo = 0.0;
        return;
    }
    const int p = Hm ? SPLIT + bitlen128(Hm) : 64 - __clzll((long long)Lm);
    if (p <= 53) {  // then Hm = 0 and |T| = Lm < 2^53
        hi = with_sign(scaled(Lm, e), neg);
        lo = 0.0;
        return;
    }
    // |T| = m 2^sh + r with m the 53-bit significand rounded to nearest even
    const int sh = p - 53;
    unsigned __int128 q, rem;
    if (sh >= SPLIT) {
        const int s2 = sh - SPLIT;
        q = Hm >> s2;
        rem = ((Hm & (((unsigned __int128)1 << s2) - 1)) << SPLIT) | Lm;
    } else {
        const unsigned __int128 x = (Hm << SPLIT) | Lm;  // p < 53 + SPLIT: fits
        q = x >> sh;
        rem = x & (((unsigned __int128)1 << sh) - 1);
    }
    unsigned long long m = (unsigned long long)q;
    const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
    __int128 r;
    if (rem > half || (rem == half && (m & 1ull))) {
        ++m;
        r = (__int128)rem - ((__int128)1 << sh);
    } else {
        r = (__int128)rem;
    }
    hi = with_sign(scaled(m, sh + e), neg);
    lo = round_int(neg ? -r : r, e);
}

// Diagonal t's term of T = sum_t S_t 2^(TB (s-1-t)) = H 2^SPLIT + L: the
// eight smallest diagonals go to L, the others to H (multiplications by
// powers of two: shifts of negative values are not defined in C++17).
template <int S, int TB>
__device__ __forceinline__ void add_diagonal(int t, int v, __int128 &H, __int128 &L) {
    if (t < S - 8)
        H += (__int128)v * ((__int128)1 << (TB * (S - 9 - t)));
    else
        L += (__int128)v * ((__int128)1 << (TB * (S - 1 - t)));
}

// The diagonals in groups of up to four: the H half [0, S-8) and the L half
// [S-8, S) of T = H 2^SPLIT + L, each cut from its start.  Within its half
// the last diagonal has weight 1 and each earlier one 2^TB more, so group q
// enters its half with weight 2^shift(q) times its own combination.
template <int S, int TB>
struct Groups {
    static constexpr int H_GROUPS = (S - 8 + 3) / 4;
    static constexpr int COUNT = H_GROUPS + 2;
    __device__ static constexpr int first(int q) {
        return q < H_GROUPS ? 4 * q : S - 8 + 4 * (q - H_GROUPS);
    }
    __device__ static constexpr int end(int q) { return q < H_GROUPS ? S - 8 : S; }
    __device__ static constexpr int len(int q) {
        return end(q) - first(q) < 4 ? end(q) - first(q) : 4;
    }
    __device__ static constexpr int shift(int q) { return TB * (end(q) - first(q) - len(q)); }
};

// Group q of one chunk: its diagonals read from tensor memory (DCOLS
// columns each, at base + 16 t) with one wait, combined exactly in an int64
// (each FP32 value is an integer of magnitude <= 2^24, so the combination
// stays below 2^(25 + 3 TB)) and added to the group's k-block sums acc[j].
// Over a k-block a diagonal sums to below 2^31 (the k-block is chosen for
// it), so a group's sum stays below 2^(32 + 3 TB) <= 2^56: exact in int64.
template <int S, int TB, int Q>
__device__ __forceinline__ void read_group(uint32_t base, long long (&acc)[DCOLS]) {
    using Gr = Groups<S, TB>;
    constexpr int g0 = Gr::first(Q), len = Gr::len(Q);
    uint32_t r[4 * DCOLS];
    if constexpr (len == 4) {
        const uint32_t t[4] = {base + g0 * BN, base + (g0 + 1) * BN, base + (g0 + 2) * BN,
                               base + (g0 + 3) * BN};
        umma::ld_x4_n(t, r);
    } else if constexpr (len == 3) {
        const uint32_t t[3] = {base + g0 * BN, base + (g0 + 1) * BN, base + (g0 + 2) * BN};
        uint32_t r3[3 * DCOLS];
        umma::ld_x4_n(t, r3);
#pragma unroll
        for (int j = 0; j < 3 * DCOLS; ++j) r[j] = r3[j];
    } else if constexpr (len == 2) {
        const uint32_t t[2] = {base + g0 * BN, base + (g0 + 1) * BN};
        uint32_t r2[2 * DCOLS];
        umma::ld_x4_n(t, r2);
#pragma unroll
        for (int j = 0; j < 2 * DCOLS; ++j) r[j] = r2[j];
    } else {
        const uint32_t t[1] = {base + g0 * BN};
        uint32_t r1[DCOLS];
        umma::ld_x4_n(t, r1);
#pragma unroll
        for (int j = 0; j < DCOLS; ++j) r[j] = r1[j];
    }
#pragma unroll
    for (int j = 0; j < DCOLS; ++j) {
        long long g = __float2int_rn(__uint_as_float(r[j]));
#pragma unroll
        for (int d = 1; d < len; ++d)
            g = g * (1 << TB) + __float2int_rn(__uint_as_float(r[DCOLS * d + j]));
        acc[j] += g;
    }
}

template <int S, int TB, int Q = 0>
__device__ __forceinline__ void read_groups(uint32_t base,
                                            long long (&acc)[Groups<S, TB>::COUNT][DCOLS]) {
    if constexpr (Q < Groups<S, TB>::COUNT) {
        read_group<S, TB, Q>(base, acc[Q]);
        read_groups<S, TB, Q + 1>(base, acc);
    }
}

// The k-block value of column x, T = H 2^SPLIT + L, from the group sums.
template <int S, int TB, int Q = 0>
__device__ __forceinline__ void block_value(const long long (&acc)[Groups<S, TB>::COUNT][DCOLS],
                                            int x, __int128 &H, __int128 &L) {
    if constexpr (Q < Groups<S, TB>::COUNT) {
        using Gr = Groups<S, TB>;
        const __int128 v = (__int128)acc[Q][x] * ((__int128)1 << Gr::shift(Q));
        if (Q < Gr::H_GROUPS)
            H += v;
        else
            L += v;
        block_value<S, TB, Q + 1>(acc, x, H, L);
    }
}

// T = sum_q acc_q 2^(W_q) as a 192-bit two's complement th 2^128 + tl, with
// W_q the weight of group q in T = H 2^SPLIT + L (block_value's terms).
template <int S, int TB, int Q = 0>
__device__ __forceinline__ void block_value_192(const long long (&acc)[Groups<S, TB>::COUNT][DCOLS],
                                                int x, long long &th, unsigned __int128 &tl) {
    if constexpr (Q < Groups<S, TB>::COUNT) {
        using Gr = Groups<S, TB>;
        constexpr int W = (Q < Gr::H_GROUPS ? TcWidth<TB>::SPLIT : 0) + Gr::shift(Q);
        static_assert(W < 64 + 32, "a group's term fits 128 bits before its shift by 64");
        unsigned __int128 low;
        long long high;
        if constexpr (W < 64) {
            const __int128 v = (__int128)acc[Q][x] * ((__int128)1 << W);  // |v| < 2^120
            low = (unsigned __int128)v;
            high = v < 0 ? -1 : 0;
        } else {
            const __int128 v = (__int128)acc[Q][x] * ((__int128)1 << (W - 64));  // < 2^88
            low = (unsigned __int128)v << 64;
            high = (long long)(v >> 64);
        }
        const unsigned __int128 sum = tl + low;
        th += high + (sum < tl ? 1 : 0);
        tl = sum;
        block_value_192<S, TB, Q + 1>(acc, x, th, tl);
    }
}

// RN((u + f) 2^e) for 2^53 <= u < 2^75 and a fraction 0 <= f < 1 of which
// only f != 0 (sticky) is known; or u < 2^53 and f = 0 (exact).
__device__ __forceinline__ double round_mag75(unsigned __int128 u, bool sticky, int e) {
    const int q = bitlen128(u);
    if (q <= 53) return scaled((unsigned long long)u, e);
    const int sh = q - 53;                       // 1 .. 22
    unsigned long long m = (unsigned long long)(u >> sh);
    const unsigned long long rem = (unsigned long long)u & ((1ull << sh) - 1ull);
    const unsigned long long half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (sticky || (m & 1ull)))) ++m;
    return scaled(m, sh + e);
}

// The k-block value of column x, T 2^e with T from the group sums, rounded
// to the nearest FP64x2: hi = RN(T 2^e), lo = RN(T 2^e - hi), the same
// values as round_dd on block_value's (H, L).  The magnitude is left-aligned
// once into 128 bits (bits below the window, when |T| >= 2^128, only make a
// sticky bit), so that hi's 53 bits, its rounding bit and the remainder are
// fixed bit fields.  Only a remainder that is both inexact in the window and
// below 2^53 of its units (about one value in 2^22 above 2^128) takes
// round_dd.
template <int S, int TB>
__device__ __forceinline__ void round_block(const long long (&acc)[Groups<S, TB>::COUNT][DCOLS],
                                            int x, int e, double &hi, double &lo) {
    long long th = 0;
    unsigned __int128 tl = 0;
    block_value_192<S, TB>(acc, x, th, tl);
    const bool neg = th < 0;
    if (neg) {  // the magnitude, two's complement negation over 192 bits
        tl = ~tl + 1;
        th = ~th + (tl == 0 ? 1 : 0);
    }
    unsigned __int128 w;  // |T| 2^(128 - p), most significant bit at 127
    int p;                // bit length of |T|
    bool sticky = false;  // bits of |T| below the window
    if (th != 0) {
        const int sb = 64 - __clzll(th);         // 1 .. 63: |T| < 2^191
        p = 128 + sb;
        w = ((unsigned __int128)(unsigned long long)th << (128 - sb)) | (tl >> sb);
        sticky = ((unsigned long long)tl & ((1ull << sb) - 1ull)) != 0;
    } else {
        if (tl == 0) {
            hi = 0.0;
            lo = 0.0;
            return;
        }
        p = bitlen128(tl);
        if (p <= 53) {
            hi = with_sign(scaled((unsigned long long)tl, e), neg);
            lo = 0.0;
            return;
        }
        w = tl << (128 - p);
    }
    const unsigned long long mant = (unsigned long long)(w >> 75);
    const unsigned __int128 low75 = w & (((unsigned __int128)1 << 75) - 1);
    const bool rbit = (unsigned long long)(w >> 74) & 1ull;
    const bool rest = sticky || (w & (((unsigned __int128)1 << 74) - 1)) != 0;
    const bool up = rbit && (rest || (mant & 1ull));
    // |T - hi| in units of 2^(p - 128): r + f, 0 <= f < 1 (f != 0 iff sticky)
    const unsigned __int128 r =
        up ? ((unsigned __int128)1 << 75) - low75 - (sticky ? 1 : 0) : low75;
    if (sticky && bitlen128(r) <= 53) {
        __int128 H = 0, L = 0;
        block_value<S, TB>(acc, x, H, L);
        round_dd<TcWidth<TB>::SPLIT>(H, L, e, hi, lo);
        return;
    }
    hi = with_sign(scaled(mant + (up ? 1ull : 0ull), p - 53 + e), neg);
    lo = (r == 0 && !sticky) ? 0.0 : with_sign(round_mag75(r, sticky, p - 128 + e), neg != up);
}

// One output tile of one problem, as a CTA sees it.  The tile's rows (the
// MMA's M side) are vectors of a_tiles and its columns (N side) vectors of
// b_tiles; output (row, col) is stored at row * ldc + col, or, for a product
// computed transposed (trans: C^T = B^T A^T), at col * ldc + row, straight
// into C.
struct TcJob {
    int m, n, k;   // rows and columns of the tile grid's product, and k
    int tm;        // row tile
    int tn_load;   // column tile whose B digits are loaded
    int col0;      // first column this CTA stores (>= n: nothing is stored)
    const uint16_t *a_tiles, *b_tiles;
    const int *exp_a, *exp_b;
    double *c_hi, *c_lo;
    long long ldc;
    bool trans;
    __device__ long long out_index(int row, int col) const {
        return trans ? (long long)col * ldc + row : (long long)row * ldc + col;
    }
};

// The tiles of one problem (Int8TcArgs), in groups of TILE_GROUP row tiles.
struct SingleSource {
    Int8TcArgs a;
    int tiles_m, tiles_n;
    __device__ long long items() const { return (long long)tiles_m * tiles_n; }
    __device__ unsigned int *status() const { return a.status; }
    __device__ const WaitPlan &wait() const { return a.wait; }
    __device__ TcJob job(long long item, int &) const {
        int tm, tn;
        grouped_tile((unsigned)item, tiles_m, tiles_n, TILE_GROUP, tm, tn);
        TcJob j;
        j.m = a.m;
        j.n = a.n;
        j.k = a.k;
        j.tm = tm;
        j.tn_load = tn;
        j.col0 = tn * BN;
        j.a_tiles = a.a_tiles;
        j.b_tiles = a.b_tiles;
        j.exp_a = a.exp_a;
        j.exp_b = a.exp_b;
        j.c_hi = a.c_hi;
        j.c_lo = a.c_lo;
        j.ldc = a.ldc;
        j.trans = false;
        return j;
    }
};

// PLANES: the order of a k-step's MMAs over the A planes,
// DDGEMM_PLANES_INTERLEAVED (0) or DDGEMM_PLANES_ASCENDING (1).
template <int S, int TB, class Src, int PLANES = DDGEMM_PLANES_INTERLEAVED>
__global__ void __launch_bounds__(NTHREADS, 1)
cascade_int8_tc_kernel(const Src src) {
    using G = TcGeom<S>;
    using W = TcWidth<TB>;
    constexpr int CHUNK_STEPS = W::CHUNK_STEPS, BLOCK_CHUNKS = W::BLOCK_CHUNKS;
    constexpr int NST = G::NST;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    auto *sh = reinterpret_cast<Shared<NST> *>(smem + NST * G::STAGE);
    static_assert(sizeof(Shared<NST>) <= BAR_BYTES, "barriers fit their region");

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long tiles = src.items();
    const long long first = blockIdx.x, stride = gridDim.x;
    unsigned int *status = src.status();
    const uint64_t limit = src.wait().limit_ns;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(smem_addr(&sh->full[s]), 1);
            mbar_init(smem_addr(&sh->empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_addr(&sh->acc_full[b]), 1);
            mbar_init(smem_addr(&sh->acc_empty[b]), EPI_WARPS);
        }
        mbar_init(smem_addr(&sh->mma_done), 1);
        sh->abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 1) {
        umma::alloc(smem_addr(&sh->tmem_base), TMEM_COLS);
        umma::relinquish();
    }
    umma::fence_before();
    __syncthreads();
    umma::fence_after();
    const uint32_t tmem = sh->tmem_base;

    if (warp == 0) {
        // ---- TMA producer -----------------------------------------------
        if (lane == 0) {
            // the failure-handling tests withhold one ring iteration's copies
            const long long withheld =
                (int)blockIdx.x == src.wait().cta ? src.wait().step : -1;
            uint32_t it = 0;
            bool ok = true;
            int hint = 0;  // the job source's position (items come in order)
            for (long long tile = first; ok && tile < tiles; tile += stride) {
                const TcJob j = src.job(tile, hint);
                const int ksteps = (j.k + BK - 1) / BK;
                for (int ks = 0; ks < ksteps; ++ks, ++it) {
                    const int stage = it % NST;
                    const uint32_t use = it / NST;
                    if (use > 0 && !wait_or_abort(smem_addr(&sh->empty[stage]), (use - 1) & 1, sh,
                                                  status, limit)) {
                        ok = false;
                        break;
                    }
                    if ((long long)it == withheld) continue;
                    unsigned char *dst = smem + stage * G::STAGE;
                    const uint32_t bar = smem_addr(&sh->full[stage]);
                    mbar_arrive_expect_tx(bar, (uint32_t)G::TX);
                    // k-step ks of all S planes: S consecutive blocks
                    const uint16_t *src_a =
                        j.a_tiles + ((long long)j.tm * ksteps + ks) * S * (BM * BK);
                    const uint16_t *src_b =
                        j.b_tiles + ((long long)j.tn_load * ksteps + ks) * S * (BN * BK);
                    bulk_load(smem_addr(dst), src_a, (uint32_t)G::A_STAGE, bar);
                    bulk_load(smem_addr(dst + G::A_STAGE), src_b, (uint32_t)(S * G::B_PLANE),
                              bar);
                }
            }
            if (!ok) {
                // copies issued but perhaps not consumed: let them land (bounded)
                for (uint32_t u = it > (uint32_t)NST ? it - NST : 0; u < it; ++u)
                    if ((long long)u != withheld)
                        mbar_wait_limit(smem_addr(&sh->full[u % NST]), (u / NST) & 1, limit);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---- MMA issuer ---------------------------------------------------
        if (lane == 0) {
            uint32_t it = 0, chunk = 0;
            bool ok = true;
            int hint = 0;
            for (long long tile = first; ok && tile < tiles; tile += stride) {
                const TcJob j = src.job(tile, hint);
                const int ksteps = (j.k + BK - 1) / BK;
                const int nchunks = (ksteps + CHUNK_STEPS - 1) / CHUNK_STEPS;
                for (int c = 0; ok && c < nchunks; ++c, ++chunk) {
                    const int b = chunk & 1;
                    const uint32_t use = chunk >> 1;
                    if (use > 0 && !wait_or_abort(smem_addr(&sh->acc_empty[b]), (use - 1) & 1,
                                                  sh, status, limit)) {
                        ok = false;
                        break;
                    }
                    umma::fence_after();
                    const uint32_t d_base = tmem + b * ACC_STRIDE;
                    const int ks0 = c * CHUNK_STEPS;
                    const int ks1 = min(ksteps, ks0 + CHUNK_STEPS);
                    for (int ks = ks0; ks < ks1; ++ks, ++it) {
                        const int stage = it % NST;
                        if (!wait_or_abort(smem_addr(&sh->full[stage]), (it / NST) & 1, sh,
                                           status, limit)) {
                            ok = false;
                            break;
                        }
                        umma::fence_after();
                        const uint32_t a0 = smem_addr(smem + stage * G::STAGE);
                        const uint64_t bdesc = umma::desc_k_sw32(a0 + G::A_STAGE);
                        // plane i's descriptor: the start-address field
                        // (address / 16, bits 0-13) advanced by i A_PLANE / 16;
                        // shared addresses stay below 2^18, so it never carries
                        const uint64_t adesc0 = umma::desc_k_sw32(a0);
                        // planes in the order 0, S-1, 1, S-2, ...: a narrow MMA
                        // (plane i near S, N = 16 (S - i)) follows a wide one.
                        // A narrow M = 128, K = 16 MMA takes about as long as a
                        // much wider one, so the narrow ones are the triangle's
                        // waste; interleaved with the wide ones they cost less
                        // (measured: 5 % less kernel time at 4096^3).  Plane 0
                        // comes first in either order: its MMA covers every
                        // column of the set and starts the chunk's sums
                        // (accumulate = 0).  The sums are exact integers, so
                        // the order changes no bit.
#pragma unroll
                        for (int q = 0; q < S; ++q) {
                            const int i = PLANES == DDGEMM_PLANES_ASCENDING ? q
                                          : (q & 1) ? S - 1 - (q >> 1) : (q >> 1);
                            umma::mma_bf16(d_base + i * BN,
                                           adesc0 + (uint64_t)(i * (G::A_PLANE >> 4)), bdesc,
                                           umma::idesc_bf16_f32(BM, (S - i) * BN),
                                           (ks > ks0 || q > 0) ? 1u : 0u);
                        }
                        // the stage is free once these MMAs have read it
                        umma::commit(smem_addr(&sh->empty[stage]));
                    }
                    if (ok) umma::commit(smem_addr(&sh->acc_full[b]));
                }
            }
            // every product of this CTA is done before tensor memory is freed
            umma::commit(smem_addr(&sh->mma_done));
            mbar_wait_limit(smem_addr(&sh->mma_done), 0, limit);
        }
        __syncwarp();
    } else {
        // ---- drain and assembly ---------------------------------------------
        const int quad = warp & 3;               // tensor-memory lanes 32 quad ..
        const int part = (warp - 2) >> 2;        // columns DCOLS part .. of each diagonal
        const int row_in_tile = quad * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16) + part * DCOLS;
        uint32_t chunk = 0;
        bool ok = true;
        int hint = 0;
        for (long long tile = first; ok && tile < tiles; tile += stride) {
            const TcJob j = src.job(tile, hint);
            const int ksteps = (j.k + BK - 1) / BK;
            const int nchunks = (ksteps + CHUNK_STEPS - 1) / CHUNK_STEPS;
            const int row = j.tm * BM + row_in_tile;
            const int col0 = j.col0 + part * DCOLS;
            if (nchunks == 0 && row < j.m) {  // k = 0: C = 0 on this tile
                for (int x = 0; x < DCOLS; ++x)
                    if (col0 + x < j.n) {
                        const long long o = j.out_index(row, col0 + x);
                        j.c_hi[o] = 0.0;
                        j.c_lo[o] = 0.0;
                    }
            }
            // per group of diagonals and column, the k-block's exact sums
            long long acc[Groups<S, TB>::COUNT][DCOLS];
#pragma unroll
            for (int q = 0; q < Groups<S, TB>::COUNT; ++q)
#pragma unroll
                for (int x = 0; x < DCOLS; ++x) acc[q][x] = 0;
            for (int c = 0; c < nchunks; ++c, ++chunk) {
                const int b = chunk & 1;
                // every lane waits; the warp goes on only together (the
                // tensor-memory loads below are warp-wide)
                const bool lane_ok = wait_or_abort(smem_addr(&sh->acc_full[b]), (chunk >> 1) & 1,
                                                   sh, status, limit, 200);
                if (!__all_sync(0xffffffffu, lane_ok)) {
                    ok = false;
                    break;
                }
                umma::fence_after();
                const uint32_t base = lane_base + b * ACC_STRIDE;
                // diagonals 0 .. S-9 belong to H, S-8 .. S-1 to L
                read_groups<S, TB>(base, acc);
                umma::fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_addr(&sh->acc_empty[b]));

                if ((c + 1) % BLOCK_CHUNKS == 0 || c + 1 == nchunks) {
                    // end of a k-block: its value, rounded once, into C
                    const int p = c / BLOCK_CHUNKS;
                    if (row < j.m) {
                        const int ea = j.exp_a[(long long)p * j.m + row];
                        // this thread's DCOLS outputs: o_base + x o_step
                        const long long o_base = j.out_index(row, col0);
                        const long long o_step = j.trans ? j.ldc : 1;
#pragma unroll
                        for (int x = 0; x < DCOLS; ++x) {
                            const int col = col0 + x;
                            if (col < j.n) {
                                const int e = ea + j.exp_b[(long long)p * j.n + col] - 12 -
                                              TB * (S - 1);
                                double h, l;
                                round_block<S, TB>(acc, x, e, h, l);
                                const long long o = o_base + x * o_step;
                                if (p > 0) {
                                    double ch = j.c_hi[o], cl = j.c_lo[o];
                                    dd_add(ch, cl, h, l, ch, cl);
                                    j.c_hi[o] = ch;
                                    j.c_lo[o] = cl;
                                } else {
                                    // C = (0, 0) + (h, l) is (h, l) itself, with no
                                    // FP64 operation (the FP64 pipe is narrow here):
                                    // the FP64x2 add reduces to FastTwoSum(h, l) and
                                    // the add of a zero low word.  round_dd gives
                                    // |l| <= ulp(h)/2, with |l| = ulp(h)/2 only when
                                    // h = RN(T) was a tie and so even: h + l rounds
                                    // to h, the FastTwoSum returns (h, l), and l is
                                    // never -0 (round_dd returns +0 for a zero), so
                                    // adding +0 leaves it.
                                    j.c_hi[o] = h;
                                    j.c_lo[o] = l;
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int q = 0; q < Groups<S, TB>::COUNT; ++q)
#pragma unroll
                        for (int x = 0; x < DCOLS; ++x) acc[q][x] = 0;
                }
            }
        }
    }
    umma::fence_before();
    __syncthreads();
    if (warp == 1) {
        umma::fence_after();
        umma::dealloc(tmem, TMEM_COLS);
    }
}

// One problem's tiles on a persistent grid: one CTA per SM (at most one per
// tile).
template <int S, int TB>
cudaError_t launch_tc_single(const Int8TcArgs &a, cudaStream_t stream) {
    using G = TcGeom<S>;
    auto kernel = cascade_int8_tc_kernel<S, TB, SingleSource>;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)G::SMEM);
    if (e != cudaSuccess) return e;
    const long long tiles_m = (a.m + BM - 1) / BM, tiles_n = (a.n + BN - 1) / BN;
    if (tiles_m * tiles_n > 0x7fffffffLL) return cudaErrorInvalidValue;
    SingleSource src;
    src.a = a;
    src.tiles_m = (int)tiles_m;
    src.tiles_n = (int)tiles_n;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return e;
    const long long tiles = tiles_m * tiles_n;
    const unsigned grid = (unsigned)(tiles < sms ? tiles : sms);
    kernel<<<grid, NTHREADS, G::SMEM, stream>>>(src);
    return cudaGetLastError();
}

}  // namespace
}  // namespace ddg
