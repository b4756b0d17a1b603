// Device units of the INT8 split (phase one of the INT8 forms), shared by
// the single-problem kernels (split_int8.cu) and the batched tcgen05 form
// (batched_int8_tc.cu).  See split_int8.cu for the method.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "ddgemm_internal.h"

namespace ddg {
namespace split8 {

constexpr unsigned DEV_NONFINITE = 0x1u;

// The block maxima and exponents are formed on the integer pipes (the FP64
// pipe is narrow on this GPU): the bit patterns of non-negative doubles
// order as their values, so max |x| is the largest pattern with the sign
// cleared (an Inf or NaN in the block wins, and gives e = 0).
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// e with |x| = f 2^e, f in [1/2, 1) (frexp's exponent), from the pattern of
// |x|; 0 for zero, Inf and NaN.
__device__ __forceinline__ int block_exponent(unsigned long long b) {
    const int be = (int)(b >> 52);
    if (b == 0 || be == 0x7ff) return 0;
    if (be > 0) return be - 1022;                      // normal
    return (64 - __clzll((long long)b)) - 1074;         // subnormal
}

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

// One warp: the exponent of block p (of kb entries) of vector v, whose
// entries are contiguous (element l at row[l]).
__device__ __forceinline__ void exps_contig_unit(int lane, int v, int p, int nvec, int kdim,
                                                 int kb, const double *__restrict__ x,
                                                 long long ldx, int *__restrict__ exps) {
    const double *row = x + (long long)v * ldx;
    const int lend = min((p + 1) * kb, kdim);
    // four independent chains keep four loads of each lane in flight
    unsigned long long m0 = 0, m1 = 0, m2 = 0, m3 = 0;
    int l = p * kb + lane;
    for (; l + 96 < lend; l += 128) {
        m0 = umax64(m0, abs_bits(row[l]));
        m1 = umax64(m1, abs_bits(row[l + 32]));
        m2 = umax64(m2, abs_bits(row[l + 64]));
        m3 = umax64(m3, abs_bits(row[l + 96]));
    }
    for (; l < lend; l += 32) m0 = umax64(m0, abs_bits(row[l]));
    unsigned long long mx = umax64(umax64(m0, m1), umax64(m2, m3));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        mx = umax64(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0) exps[(long long)p * nvec + v] = block_exponent(mx);
}

// One CTA of 64 RG threads: the exponents of block p (of kb entries) of
// vectors [64 vt, 64 vt + 64), whose entries are strided (element l at
// x[l*ldx + v]); RG row groups take every RG-th entry, four loads in flight
// each.
template <int RG>
__device__ __forceinline__ void exps_strided_unit(int vt, int p, int nvec, int kdim, int kb,
                                                  const double *__restrict__ x, long long ldx,
                                                  int *__restrict__ exps,
                                                  unsigned long long (&part)[RG][64]) {
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
    const int v = vt * 64 + tx;
    const int lend = min((p + 1) * kb, kdim);
    unsigned long long mx = 0;
    if (v < nvec) {
        unsigned long long m0 = 0, m1 = 0, m2 = 0, m3 = 0;
        int l = p * kb + ty;
        for (; l + 3 * RG < lend; l += 4 * RG) {
            m0 = umax64(m0, abs_bits(x[(long long)l * ldx + v]));
            m1 = umax64(m1, abs_bits(x[(long long)(l + RG) * ldx + v]));
            m2 = umax64(m2, abs_bits(x[(long long)(l + 2 * RG) * ldx + v]));
            m3 = umax64(m3, abs_bits(x[(long long)(l + 3 * RG) * ldx + v]));
        }
        for (; l < lend; l += RG) m0 = umax64(m0, abs_bits(x[(long long)l * ldx + v]));
        mx = umax64(umax64(m0, m1), umax64(m2, m3));
    }
    part[ty][tx] = mx;
    __syncthreads();
    if (ty == 0 && v < nvec) {
#pragma unroll
        for (int g = 1; g < RG; ++g) mx = umax64(mx, part[g][tx]);
        exps[(long long)p * nvec + v] = block_exponent(mx);
    }
    __syncthreads();  // part is reused by the next unit
}

// The upper word of (hi:lo) << (s mod 32).
__host__ __device__ __forceinline__ uint32_t funnel_l(uint32_t lo, uint32_t hi, int s) {
#ifdef __CUDA_ARCH__
    return __funnelshift_l(lo, hi, (unsigned)s);
#else
    const int r = s & 31;
    return r ? (hi << r) | (lo >> (32 - r)) : hi;
#endif
}

__host__ __device__ __forceinline__ unsigned long long double_bits(double x) {
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long b;
    __builtin_memcpy(&b, &x, sizeof b);
    return b;
#endif
}

// round-half-even(|x| 2^sh) as a 128-bit magnitude in 32-bit words v[0..3]
// (least significant first), from the two words of x's bit pattern (hw:
// sign, exponent and the fraction's top 20 bits).  The shifts are word
// funnel shifts and the rounding one carry trick, on the integer pipes.
// Returns false for Inf and NaN (v = 0; the caller flags them).  An entry
// with |x| 2^sh >= 2^74 (a lo part far above its block's max |hi|, outside
// the form's range) gives 0.
__host__ __device__ __forceinline__ bool scaled_magnitude(uint32_t hw, uint32_t lw, int sh,
                                                          uint32_t (&v)[4]) {
    const int ex = (int)((hw >> 20) & 0x7ffu);
    uint32_t m1 = hw & 0xfffffu;  // |x| = (m1:lw) 2^(p - sh)
    int p;
    if (ex == 0) {
        p = 1 - 1075 + sh;        // zero or subnormal: no implicit bit
    } else {
        m1 |= 0x100000u;
        p = ex - 1075 + sh;
    }
    v[0] = v[1] = v[2] = v[3] = 0u;
    if (ex == 0x7ff) return false;
    if (p > 127 - 54) return true;
    if (p >= 0) {
        // (m1:lw) << p: three words from word p / 32 up (the third is zero
        // when p >= 64, as m1 < 2^21 and p <= 73)
        const uint32_t t0 = lw << (p & 31), t1 = funnel_l(lw, m1, p), t2 = funnel_l(m1, 0u, p);
        const int q = p >> 5;
        v[0] = q == 0 ? t0 : 0u;
        v[1] = q == 0 ? t1 : (q == 1 ? t0 : 0u);
        v[2] = q == 0 ? t2 : (q == 1 ? t1 : t0);
        v[3] = q == 1 ? t2 : (q == 2 ? t1 : 0u);
    } else if (p >= -63) {
        // m / 2^r rounded half to even is (m + 2^(r-1) - 1 + bit r of m) >> r
        // (no overflow: m < 2^53); below 2^-63 the value rounds to 0
        const int r = -p;
        const unsigned long long m = ((unsigned long long)m1 << 32) | lw;
        const unsigned long long q = (m + ((1ull << (r - 1)) - 1ull) + ((m >> r) & 1ull)) >> r;
        v[0] = (uint32_t)q;
        v[1] = (uint32_t)(q >> 32);
    }
    return true;
}

__host__ __device__ __forceinline__ unsigned __int128 words128(const uint32_t (&v)[4], uint32_t mask) {
    return ((unsigned __int128)(((unsigned long long)(v[3] ^ mask) << 32) | (v[2] ^ mask)) << 64) |
           (((unsigned long long)(v[1] ^ mask) << 32) | (v[0] ^ mask));
}

// C + rne(hi 2^sh) + rne(lo 2^sh) as a 128-bit two's complement integer,
// each term rounded on its own; clears `finite` when hi or lo is Inf or
// NaN.  A negative term -v enters as ~v + 1: its words XORed with all ones
// and the 1 added to the constant C.
__host__ __device__ __forceinline__ __int128 fixed_sum(double hi, double lo, int sh, __int128 c,
                                                       bool &finite) {
    const unsigned long long bh = double_bits(hi), bl = double_bits(lo);
    uint32_t vh[4], vl[4];
    finite &= scaled_magnitude((uint32_t)(bh >> 32), (uint32_t)bh, sh, vh);
    finite &= scaled_magnitude((uint32_t)(bl >> 32), (uint32_t)bl, sh, vl);
    const uint32_t nh = (uint32_t)(bh >> 63), nl = (uint32_t)(bl >> 63);
    return (__int128)(words128(vh, 0u - nh) + words128(vl, 0u - nl) +
                      ((unsigned __int128)c + nh + nl));
}

constexpr int TV = 32, TK = 64;  // tile: 32 vectors x 64 k

// sum_{i < S-1} 2^(BITS-1) 2^(BITS i): adding it turns the balanced digits
// of X into plain BITS-bit fields offset by 2^(BITS-1).
template <int S, int BITS>
__host__ __device__ constexpr __int128 digit_offset() {
    __int128 c = 0;
    for (int i = 0; i < S - 1; ++i) c = c * (1 << BITS) + (1 << (BITS - 1));
    return c;
}

// Field i (least significant first) of the offset value Y, 0 <= field <
// 2^BITS + 1: digit i plus 2^(BITS-1).  The top field (i = S-1) is Y's
// signed top part plus 2^(BITS-1).
template <int S, int BITS>
__device__ __forceinline__ uint32_t digit_field(__int128 Y, int i) {
    if (i == S - 1) return (uint32_t)((int)(Y >> (BITS * (S - 1))) + (1 << (BITS - 1)));
    const int b0 = BITS * i;
    const unsigned long long y_lo = (unsigned long long)Y;
    const unsigned long long y_hi = (unsigned long long)(Y >> 64);
    unsigned long long field;
    if (b0 + BITS <= 64)
        field = y_lo >> b0;
    else if (b0 >= 64)
        field = y_hi >> (b0 - 64);
    else
        field = (y_lo >> b0) | (y_hi << (64 - b0));
    return (uint32_t)field & ((1u << BITS) - 1u);
}

// The FP32 encoding of the digit d = f - 2^(BITS-1) for a field
// 0 <= f < 2^23: the bit pattern 0x4B000000 | f is the float 2^23 + f, and
// subtracting 2^23 + 2^(BITS-1) is exact (every operand and the result are
// integers below 2^24).  Its upper half is the bf16 encoding of d, exact
// because |d| <= 2^BITS has at most 8 significant bits (bf16 keeps 8).
template <int BITS>
__device__ __forceinline__ uint32_t digit_fp32(uint32_t f) {
    constexpr float bias = 8388608.0f + (float)(1 << (BITS - 1));
    return __float_as_uint(__fsub_rn(__uint_as_float(0x4B000000u | f), bias));
}

// Element offset of the 8-entry group (v, l .. l+7) of plane s in the tiled
// bf16 order (l a multiple of 8).
template <int S>
__device__ __forceinline__ long long tiled_offset(int v, int l, int s, int th, int ksteps) {
    const int r = v % th;
    const long long block = ((long long)(v / th) * ksteps + l / 16) * S + s;
    return block * th * 16 + r * 16 + ((((l >> 3) & 1) ^ ((r >> 2) & 1)) << 3);
}

// One CTA of 256 threads: the BITS-bit digits of the tile of TV vectors x
// TK entries at (v0, l0), through shared memory (sh, sl) so that both input
// layouts are read coalesced.  CONTIG: element (v, l) at x[v*ldx + l]; else
// at x[l*ldx + v].  BF16: the tiled bf16 order with tile height th; else
// int8 planes with leading dimension ld_out.  exps per k-block of
// kblock_of_bits(BITS).
template <int S, bool CONTIG, bool BF16, int BITS>
__device__ __forceinline__ void digits_unit(int v0, int l0, int nvec, int kdim,
                                            const double *__restrict__ xh,
                                            const double *__restrict__ xl, long long ldx,
                                            void *__restrict__ out_v, long long ld_out, int th,
                                            const int *__restrict__ exps, unsigned int *status,
                                            double (&sh)[TV][TK + 1], double (&sl)[TV][TK + 1]) {
    const int tid = threadIdx.x;
    // coalesced tile load in the input's own layout
#pragma unroll
    for (int it = 0; it < TV * TK / 256; ++it) {
        const int idx = it * 256 + tid;
        int v, l;
        if (CONTIG) {
            v = idx / TK; l = idx % TK;
        } else {
            l = idx / TV; v = idx % TV;
        }
        const int gv = v0 + v, gl = l0 + l;
        double a = 0.0, b = 0.0;
        if (gv < nvec && gl < kdim) {
            const long long o = CONTIG ? (long long)gv * ldx + gl : (long long)gl * ldx + gv;
            a = xh[o];
            b = xl[o];
        }
        sh[v][l] = a;
        sl[v][l] = b;
    }
    __syncthreads();
    // each thread: one vector, 8 consecutive k.  For the tiled bf16 order a
    // warp takes one k-step of 16 entries (two lanes per vector) of 16
    // vectors: the k-steps a ragged tile has past its end, and a vector half
    // past nvec, then leave whole warps idle instead of lanes of every warp,
    // and a warp's stores of a plane are 512 contiguous bytes.  The int8
    // planes keep a vector's 64 entries in one warp (64-byte rows).
    const int warp = tid >> 5, lane = tid & 31;
    const int v = BF16 ? (warp >> 2) * 16 + (lane >> 1) : tid >> 3;
    const int lg = BF16 ? (warp & 3) * 2 + (lane & 1) : tid & 7;
    const int gv = v0 + v;
    if (gv >= nvec) return;
    const int gl = l0 + lg * 8;
    // the tiled bf16 order is read a whole k-step of 16 at a time: groups
    // past kdim up to the next multiple of 16 are written with zero digits
    // (their entries were loaded as zeros); the int8 planes stop at kdim
    if (gl >= (BF16 ? (kdim + 15) / 16 * 16 : kdim)) return;
    const int e = exps[(long long)(l0 / kblock_of_bits(BITS)) * nvec + gv];
    constexpr int F = 6 + BITS * (S - 1);
    if constexpr (BF16) {
        // Balanced base-2^BITS digits as bit fields: with Y = X +
        // sum_{i<s-1} 2^(BITS-1) 2^(BITS i), digit i (least significant
        // first) is field i of Y minus 2^(BITS-1), and the top digit is
        // Y >> BITS (s-1) (the same digits as peeling d = ((X + h) mod 2 h)
        // - h, X = (X - d) / 2h with h = 2^(BITS-1)).
        __int128 Y[8];
        bool finite = true;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            Y[j] = fixed_sum(sh[v][lg * 8 + j], sl[v][lg * 8 + j], F - e,
                             digit_offset<S, BITS>(), finite);
        if (!finite && status) atomicOr(status, DEV_NONFINITE);
        const int ksteps = (kdim + 15) / 16;
        // plane s holds digit S-1-s; two entries' bf16 digits share a
        // 32-bit word, each plane's 8 entries one 16-byte store
#pragma unroll
        for (int s = 0; s < S; ++s) {
            uint32_t w[4];
#pragma unroll
            for (int jp = 0; jp < 4; ++jp)
                w[jp] = __byte_perm(digit_fp32<BITS>(digit_field<S, BITS>(Y[2 * jp], S - 1 - s)),
                                    digit_fp32<BITS>(digit_field<S, BITS>(Y[2 * jp + 1], S - 1 - s)),
                                    0x7632);
            *reinterpret_cast<uint4 *>(static_cast<uint16_t *>(out_v) +
                                       tiled_offset<S>(gv, gl, s, th, ksteps)) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
    } else {
        // int8 planes (eight-bit pieces): 8 entries per plane in one 8-byte
        // word
        static_assert(BITS == 8, "int8 planes hold eight-bit pieces");
        unsigned long long word[S];
#pragma unroll
        for (int s = 0; s < S; ++s) word[s] = 0;
        bool finite = true;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            // the digits as in the bf16 branch; the int8 digit d = f - 128 is
            // the byte f ^ 0x80
            const __int128 Y = fixed_sum(sh[v][lg * 8 + j], sl[v][lg * 8 + j], F - e,
                                         digit_offset<S, BITS>(), finite);
#pragma unroll
            for (int s = 0; s < S; ++s)
                word[s] |= (unsigned long long)((digit_field<S, BITS>(Y, S - 1 - s) ^ 0x80u) &
                                                0xffu)
                           << (8 * j);
        }
        if (!finite && status) atomicOr(status, DEV_NONFINITE);
        // entries past kdim in the last group of 8 carry zero digits; they
        // sit in the row padding (ld_out >= kdim rounded up to 16) and are
        // never read
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const long long o = ((long long)s * nvec + gv) * ld_out + gl;
            *reinterpret_cast<unsigned long long *>(static_cast<int8_t *>(out_v) + o) = word[s];
        }
    }
}


}  // namespace split8
}  // namespace ddg
