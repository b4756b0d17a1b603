// The FP64 cascade's per-tile arithmetic, shared by the single-problem
// kernel (TMA-staged) and the batched persistent kernel (cp.async-staged).
//
// A k-step of 8 holds, in shared memory, the step's slice of the four A
// pieces ([4][BM][8]) and of the seven B panels ([7][8][BN]).  A warp owns a
// 16 x 32 sub-tile: 2 x 4 fragments of the m8n8k4 f64 MMA, four
// accumulators each (bin 0, bin 1, bin 2, bin 3-6).  The ten products of
// eq. (Gemm10) are issued per fragment, each A fragment reused against all
// its B partners.
#pragma once
#include <cstdint>

#include "dd_device.cuh"

namespace ddg {

constexpr int CBK = 8;  // k per shared-memory stage

template <int WM, int WN>
struct Fp64Tile {
    static constexpr int BM = 16 * WM, BN = 32 * WN, NTHREADS = 32 * WM * WN;
    static constexpr int A_STAGE = 4 * BM * CBK;  // doubles
    static constexpr int B_STAGE = 7 * CBK * BN;  // doubles
    static constexpr int STAGE = A_STAGE + B_STAGE;
};

using Acc = double[4][2][4][2];  // [bin][m fragment][n fragment][2 values]

// D = A B + D for one m8n8k4 f64 fragment.
__device__ __forceinline__ void dmma(double (&d)[2], double a, double b) {
    asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                 : "+d"(d[0]), "+d"(d[1])
                 : "d"(a), "d"(b));
}

__device__ __forceinline__ void zero_acc(Acc &acc) {
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[b][i][j][0] = acc[b][i][j][1] = 0.0;
}

// Which products feed the bins (PRODUCTS):
//   0  eq. (Gemm10): the method, bins 3-6 folded into four products;
//   1  eq. (Gemm16): all sixteen products (accuracy ablation);
//   2  bins 0-3 of eq. (Gemm16) only, bins 4-6 dropped (accuracy ablation).
constexpr int PRODUCTS_GEMM10 = 0, PRODUCTS_GEMM16 = 1, PRODUCTS_DROP456 = 2;

// The products for one k-step held in shared memory.
template <int BM, int BN, int PRODUCTS = PRODUCTS_GEMM10>
__device__ __forceinline__ void mma_stage(Acc &acc, const double *As, const double *Bs, int wm,
                                          int wn, int lane) {
    constexpr int NB = PRODUCTS == PRODUCTS_GEMM10 ? 7 : 4;  // B panels the products use
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
        double a[4][2];
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int i = 0; i < 2; ++i)
                a[s][i] = As[s * BM * CBK + (wm * 16 + i * 8 + (lane >> 2)) * CBK + ks * 4 +
                             (lane & 3)];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            double b[NB];
#pragma unroll
            for (int s = 0; s < NB; ++s)
                b[s] = Bs[s * CBK * BN + (ks * 4 + (lane & 3)) * BN + wn * 32 + j * 8 + (lane >> 2)];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                dmma(acc[0][i][j], a[0][i], b[0]);  // bin 0:   A0 B0
                dmma(acc[1][i][j], a[0][i], b[1]);  // bin 1:   A0 s1B1
                dmma(acc[1][i][j], a[1][i], b[0]);  //          s1A1 B0
                dmma(acc[2][i][j], a[0][i], b[2]);  // bin 2:   A0 s2B2
                dmma(acc[2][i][j], a[1][i], b[1]);  //          s1A1 s1B1
                dmma(acc[2][i][j], a[2][i], b[0]);  //          s2A2 B0
                if constexpr (PRODUCTS == PRODUCTS_GEMM10) {
                    dmma(acc[3][i][j], a[0][i], b[3]);  // bin 3-6: A0 s3B3
                    dmma(acc[3][i][j], a[1][i], b[4]);  //          s1A1 s2B4
                    dmma(acc[3][i][j], a[2][i], b[5]);  //          s2A2 s1B5
                    dmma(acc[3][i][j], a[3][i], b[6]);  //          s3A3 B6
                } else if constexpr (PRODUCTS == PRODUCTS_GEMM16) {
                    dmma(acc[3][i][j], a[0][i], b[3]);  // bins 3-6, row by row of eq. Gemm16
                    dmma(acc[3][i][j], a[1][i], b[2]);
                    dmma(acc[3][i][j], a[1][i], b[3]);
                    dmma(acc[3][i][j], a[2][i], b[1]);
                    dmma(acc[3][i][j], a[2][i], b[2]);
                    dmma(acc[3][i][j], a[2][i], b[3]);
                    dmma(acc[3][i][j], a[3][i], b[0]);
                    dmma(acc[3][i][j], a[3][i], b[1]);
                    dmma(acc[3][i][j], a[3][i], b[2]);
                    dmma(acc[3][i][j], a[3][i], b[3]);
                } else {
                    dmma(acc[3][i][j], a[0][i], b[3]);  // bin 3 only
                    dmma(acc[3][i][j], a[1][i], b[2]);
                    dmma(acc[3][i][j], a[2][i], b[1]);
                    dmma(acc[3][i][j], a[3][i], b[0]);
                }
            }
        }
    }
}

// Where a k-block's results go.
struct EpilogueOut {
    int m, n;
    const int *exp_a;  // [k-block][m]
    const int *exp_b;  // [k-block][n]
    double *c_hi, *c_lo;
    long long ldc;
    int *flags;        // optional m x n
    double *bins;      // when non-null: the four raw bins of k-block 0
};

// End of k-block p for one warp's sub-tile at (row0, col0): bins 3-6 -> 2
// -> 1 -> 0 in FP64x2, scale by 2^(e_a + e_b), FP64x2-add into C (C holds
// the running sum between k-blocks; `first` marks the first k-block summed
// into this output, which starts from zero), then clear the bins.
template <bool DUMP_BINS>
__device__ __forceinline__ void epilogue(Acc &acc, int p, bool first, int row0, int col0,
                                         int lane, const EpilogueOut &o) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int row = row0 + i * 8 + (lane >> 2);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int col = col0 + j * 8 + 2 * (lane & 3) + h;
                if (row < o.m && col < o.n) {
                    const double b0 = acc[0][i][j][h], b1 = acc[1][i][j][h];
                    const double b2 = acc[2][i][j][h], b36 = acc[3][i][j][h];
                    if constexpr (DUMP_BINS) {
                        const long long mn = (long long)o.m * o.n;
                        const long long x = (long long)row * o.n + col;
                        o.bins[x] = b0;
                        o.bins[mn + x] = b1;
                        o.bins[2 * mn + x] = b2;
                        o.bins[3 * mn + x] = b36;
                    } else {
                        double sh, sl;
                        assemble_bins(b0, b1, b2, b36, sh, sl);
                        const int sc = o.exp_a[(long long)p * o.m + row] +
                                       o.exp_b[(long long)p * o.n + col];
                        sh = scalbn(sh, sc);
                        sl = scalbn(sl, sc);
                        const long long x = (long long)row * o.ldc + col;
                        double ch = 0.0, cl = 0.0;
                        if (!first) {
                            ch = o.c_hi[x];
                            cl = o.c_lo[x];
                        }
                        dd_add(ch, cl, sh, sl, ch, cl);
                        o.c_hi[x] = ch;
                        o.c_lo[x] = cl;
                        if (o.flags) {
                            const long long fx = (long long)row * o.n + col;
                            int f = first ? 0 : o.flags[fx];
                            if (b0 == 0.0 && (sh != 0.0 || sl != 0.0)) ++f;
                            o.flags[fx] = f;
                        }
                    }
                }
                acc[0][i][j][h] = acc[1][i][j][h] = 0.0;
                acc[2][i][j][h] = acc[3][i][j][h] = 0.0;
            }
        }
    }
}

// NaN into every output of one warp's sub-tile at (row0, col0) (hi and lo):
// what a CTA whose wait gave up leaves, so that no later pass can mistake
// its outputs for results.
__device__ __forceinline__ void poison(int row0, int col0, int lane, const EpilogueOut &o) {
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int row = row0 + i * 8 + (lane >> 2);
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int col = col0 + j * 8 + 2 * (lane & 3) + h;
                if (row < o.m && col < o.n) {
                    const long long x = (long long)row * o.ldc + col;
                    o.c_hi[x] = nan;
                    o.c_lo[x] = nan;
                }
            }
    }
}

}  // namespace ddg
