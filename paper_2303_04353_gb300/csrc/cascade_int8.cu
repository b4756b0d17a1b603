// Phases two and three of the INT8 form (Sec. "FP64x2 in terms of INT8",
// Sec. "Safely dropping lower order bins"): the triangle of digit-pair
// products i + j <= s - 1 on the integer tensor path (mma.sync m16n8k32 s8,
// exact int32 accumulation), one int32 accumulator per diagonal t = i + j,
// and the FP64x2 sum of the diagonals, smallest first, once per k-block.
//
// Tiling.  A CTA owns a 32 x 32 tile of C; 8 warps each own 16 x 8 (one
// MMA tile).  Per k-step of 32, two TMA copies bring all s digit planes of
// A ([s][32][32] int8) and of B ([s][32][32], k contiguous) into a
// three-deep ring (two CTAs per SM).  Each warp loads its s A fragments (ldmatrix.x4) and s B
// fragments (ldmatrix.x2) once and issues the s(s+1)/2 products from
// registers.  The s accumulators of 4 registers each are what bound the
// tile size per warp (s = 15: 60 accumulator + 90 operand registers).
//
// Exactness.  |digit| <= 128, so a product is at most 2^14 and a diagonal
// holds at most s <= 15 of them per k: over a k-block of 8192 a diagonal sum
// is below 15 2^27 < 2^31.  The int32 -> FP64 conversion and the scaling by
// 2^(-12-8t) are exact; only the FP64x2 additions round.
//
// Waits are bounded as in the FP64 kernel (DDGEMM_DEV_TIMEOUT).
#include <cuda_runtime.h>

#include <cstdint>

#include "dd_device.cuh"
#include "ddgemm_internal.h"
#include "tma.cuh"

namespace ddg {
namespace {

constexpr int BM = 32, BN = 32, BKB = 32, NST = 3, NTHREADS = 256;
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2(uint32_t (&r)[2], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
                 : "=r"(r[0]), "=r"(r[1])
                 : "r"(addr));
}

// D = A B + D for one m16n8k32 s8 tile with s32 accumulation.
__device__ __forceinline__ void imma(int (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+r"(d[0]), "+r"(d[1]), "+r"(d[2]), "+r"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int S>
struct Geometry {
    static constexpr int PLANE = BM * BKB;              // bytes of one digit plane tile
    static constexpr int A_STAGE = S * PLANE;
    static constexpr int B_STAGE = S * BN * BKB;
    static constexpr int STAGE = A_STAGE + B_STAGE;
    static constexpr size_t SMEM = (size_t)NST * STAGE + NST * sizeof(uint64_t) + 1024;
};

// Two CTAs per SM while the registers allow it (<= 128 per thread): one
// CTA's FP64x2 epilogue then overlaps the other's integer MMAs.
template <int S>
constexpr int ctas_per_sm() { return S <= 17 ? 2 : 1; }

template <int S>
__global__ void __launch_bounds__(NTHREADS, ctas_per_sm<S>())
cascade_int8_kernel(const __grid_constant__ CUtensorMap tm_a,
                    const __grid_constant__ CUtensorMap tm_b, const Int8Args args) {
    using G = Geometry<S>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NST * G::STAGE);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;
    int tm, tn;
    grouped_tile(blockIdx.x, (args.m + BM - 1) / BM, (args.n + BN - 1) / BN, 16, tm, tn);
    const int m0 = tm * BM, n0 = tn * BN;
    const int ksteps = (args.k + BKB - 1) / BKB;
    constexpr int STEPS_PER_BLOCK = KB8 / BKB;

    if (tid == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(smem_addr(&bars[s]), 1);
        mbar_fence_init();
    }
    __syncthreads();

    // the failure-handling tests withhold one k-step's copy of one CTA
    const long long withheld = (int)blockIdx.x == args.wait.cta ? args.wait.step : -1;
    const unsigned long long limit = args.wait.limit_ns;
    auto issue = [&](int t, int stage) {
        if (t == withheld) return;
        const uint32_t bar = smem_addr(&bars[stage]);
        unsigned char *dst = smem + stage * G::STAGE;
        mbar_arrive_expect_tx(bar, (uint32_t)G::STAGE);
        tma_load_3d(smem_addr(dst), &tm_a, bar, t * BKB, m0, 0);
        tma_load_3d(smem_addr(dst + G::A_STAGE), &tm_b, bar, t * BKB, n0, 0);
    };
    if (tid == 0)
        for (int s = 0; s < NST && s < ksteps; ++s) issue(s, s);

    int acc[S][4];
#pragma unroll
    for (int t = 0; t < S; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0;

    // ldmatrix row addresses (bytes, relative to a plane tile)
    const uint32_t a_off = (uint32_t)((wm * 16 + (lane & 7) + ((lane >> 3) & 1) * 8) * BKB +
                                      (lane >> 4) * 16);
    const uint32_t b_off = (uint32_t)((wn * 8 + (lane & 7)) * BKB + ((lane >> 3) & 1) * 16);

    for (int t = 0; t < ksteps; ++t) {
        const int stage = t % NST;
        const bool ok = mbar_wait_limit(smem_addr(&bars[stage]), (t / NST) & 1, limit);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                if (args.status) atomicOr(args.status, DEV_TIMEOUT_BIT);
                for (int u = t; u < t + NST && u < ksteps; ++u)
                    if (u != withheld)
                        mbar_wait_limit(smem_addr(&bars[u % NST]), (u / NST) & 1, limit);
            }
            return;
        }
        const uint32_t base = smem_addr(smem + stage * G::STAGE);
        uint32_t a[S][4], b[S][2];
#pragma unroll
        for (int i = 0; i < S; ++i) ldsm_x4(a[i], base + i * G::PLANE + a_off);
#pragma unroll
        for (int j = 0; j < S; ++j) ldsm_x2(b[j], base + G::A_STAGE + j * (BN * BKB) + b_off);
#pragma unroll
        for (int i = 0; i < S; ++i)
#pragma unroll
            for (int j = 0; j < S - i; ++j) imma(acc[i + j], a[i], b[j]);
        __syncthreads();
        if (tid == 0 && t + NST < ksteps) issue(t + NST, stage);

        if ((t + 1) % STEPS_PER_BLOCK == 0 || t + 1 == ksteps) {
            const int p = t / STEPS_PER_BLOCK;
            const int g = lane >> 2, q4 = lane & 3;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int row = m0 + wm * 16 + g + (q >> 1) * 8;
                const int col = n0 + wn * 8 + 2 * q4 + (q & 1);
                if (row < args.m && col < args.n) {
                    double h = 0.0, l = 0.0;
#pragma unroll
                    for (int d = S - 1; d >= 0; --d) {
                        // S_d 2^(-12-8d): exact; the power of two is a constant
                        const double v = __dmul_rn(__int2double_rn(acc[d][q]),
                                                   __longlong_as_double(
                                                       (long long)(1023 - 12 - 8 * d) << 52));
                        dd_add_d(h, l, v);
                    }
                    const int sc = args.exp_a[(long long)p * args.m + row] +
                                   args.exp_b[(long long)p * args.n + col];
                    h = scalbn(h, sc);
                    l = scalbn(l, sc);
                    const long long o = (long long)row * args.ldc + col;
                    double ch = 0.0, cl = 0.0;
                    if (p > 0) {
                        ch = args.c_hi[o];
                        cl = args.c_lo[o];
                    }
                    dd_add(ch, cl, h, l, ch, cl);
                    args.c_hi[o] = ch;
                    args.c_lo[o] = cl;
                }
            }
#pragma unroll
            for (int d = 0; d < S; ++d) acc[d][0] = acc[d][1] = acc[d][2] = acc[d][3] = 0;
        }
    }
}

template <int S>
cudaError_t launch_s(const Int8Args &a, cudaStream_t stream) {
    using G = Geometry<S>;
    CUtensorMap tm_a, tm_b;
    // digit planes [S][rows][ld] (int8, k contiguous), box [S][32][32]
    if (!encode_map_3d(&tm_a, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, a.a_digits, a.k, a.m, S,
                       a.ld_digits, BKB, 32, S) ||
        !encode_map_3d(&tm_b, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, a.b_digits, a.k, a.n, S,
                       a.ld_digits, BKB, 32, S))
        return cudaErrorInvalidValue;
    const cudaError_t e = cudaFuncSetAttribute(
        cascade_int8_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    if (e != cudaSuccess) return e;
    const long long tiles = (long long)((a.n + BN - 1) / BN) * ((a.m + BM - 1) / BM);
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    cascade_int8_kernel<S><<<(unsigned)tiles, NTHREADS, G::SMEM, stream>>>(tm_a, tm_b, a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cascade_int8(const Int8Args &a, cudaStream_t stream) {
    if (a.m <= 0 || a.n <= 0 || a.k <= 0) return cudaSuccess;
    switch (a.slices) {
#define DDG_CASE(S) \
    case S:         \
        return launch_s<S>(a, stream);
        DDG_INT8_SLICE_CASES
#undef DDG_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace ddg
