// Phases two and three of the cascade (Sec. "Practical considerations") in
// one kernel: the ten FP64 products of eq. (Gemm10) on the FP64 tensor path,
// accumulated into four bins, and the FP64x2 assembly of the bins into C
// after every k-block of K_C = 256 (Sec. "Simple").
//
// Tiling.  One CTA owns a 64 x 64 tile of C and walks k in steps of 8.  Per
// step, two TMA copies bring the step's slice of all four A pieces
// ([4][64][8] doubles) and of all seven B panels ([7][8][64]) into shared
// memory; a three-deep ring of such stages keeps copies ahead of the math.
// Each of the eight warps owns a 16 x 32 sub-tile, i.e. 2 x 4 fragments of
// the m8n8k4 f64 MMA, and keeps four accumulators per fragment (bin 0,
// bin 1, bin 2, bin 3-6).  Every A fragment is loaded once per step and
// reused against all the B panels it pairs with in eq. (Gemm10):
//   A0 x {B0, s1B1, s2B2, s3B3},  s1A1 x {B0, s1B1, s2B4},
//   s2A2 x {B0, s1B5},            s3A3 x {B6}.
// This is the data reuse the paper gets from cascading while packing
// (Sec. "BLIS-like"), here at the level of shared memory and registers.
//
// Exactness.  With the pieces pre-scaled by sigma_i, every product of bins
// 0-2 and every partial sum of a bin over one k-block is an integer multiple
// of that bin's unit (2^-42, 2^-63, 2^-84) below 2^53 units, so the FP64 MMA
// accumulates them without rounding, in any order.  Bin 3-6 rounds.
//
// Epilogue per k-block: bin 3-6 -> bin 2 -> bin 1 -> bin 0 with TwoSum-based
// FP64x2 additions, scale by 2^(e_a + e_b) (exact), FP64x2-add into C (C
// itself holds the running sum between k-blocks; each CTA owns its tile).
//
// Waits.  Every mbarrier wait gives up after ~2 s of global time: the CTA
// then sets DDGEMM_DEV_TIMEOUT, waits (again bounded) for its own copies
// still in flight and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "cascade_core.cuh"
#include "ddgemm_internal.h"

namespace ddg {
namespace {

using Tile = Fp64Tile<4, 2>;  // 64 x 64, 8 warps
constexpr int BM = Tile::BM, BN = Tile::BN, BK = CBK, NST = 3, NTHREADS = Tile::NTHREADS;
constexpr int A_STAGE = Tile::A_STAGE;
constexpr int B_STAGE = Tile::B_STAGE;
constexpr int STAGE = Tile::STAGE;
constexpr uint32_t STAGE_BYTES = STAGE * sizeof(double);
constexpr int STEPS_PER_BLOCK = KC / BK;
constexpr size_t SMEM_BYTES = (size_t)NST * STAGE * sizeof(double) + NST * sizeof(uint64_t) + 1024;
constexpr unsigned DEV_TIMEOUT = 0x2u;
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on one phase of an mbarrier.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > WAIT_LIMIT_NS) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                            int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y), "r"(z)
        : "memory");
}

template <bool DUMP_BINS>
__global__ void __launch_bounds__(NTHREADS, 1)
cascade_fp64_kernel(const __grid_constant__ CUtensorMap tm_a,
                    const __grid_constant__ CUtensorMap tm_b, const CascadeArgs args) {
    extern __shared__ unsigned char smem_raw[];
    double *smem = reinterpret_cast<double *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NST * STAGE);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 3, wn = warp >> 2;
    int tm, tn;
    grouped_tile(blockIdx.x, (args.m + BM - 1) / BM, (args.n + BN - 1) / BN, 8, tm, tn);
    const int m0 = tm * BM, n0 = tn * BN;
    const int ksteps = (args.k + BK - 1) / BK;

    if (tid == 0) {
        for (int s = 0; s < NST; ++s) mbar_init(smem_addr(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    auto issue = [&](int t, int stage) {
        const uint32_t bar = smem_addr(&bars[stage]);
        double *dst = smem + stage * STAGE;
        mbar_arrive_expect_tx(bar, STAGE_BYTES);
        tma_load_3d(smem_addr(dst), &tm_a, bar, t * BK, m0, 0);
        tma_load_3d(smem_addr(dst + A_STAGE), &tm_b, bar, n0, t * BK, 0);
    };
    if (tid == 0) {
        for (int s = 0; s < NST && s < ksteps; ++s) issue(s, s);
    }

    Acc acc;
    zero_acc(acc);
    const EpilogueOut out{args.m, args.n, args.exp_a, args.exp_b, args.c_hi, args.c_lo,
                          args.ldc, args.flags, args.bins};

    for (int t = 0; t < ksteps; ++t) {
        const int stage = t % NST;
        const uint32_t parity = (t / NST) & 1;
        const bool ok = mbar_wait(smem_addr(&bars[stage]), parity);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                if (args.status) atomicOr(args.status, DEV_TIMEOUT);
                // Copies already issued for steps t .. t+NST-1 may still be in
                // flight into this CTA's shared memory: wait for them, bounded.
                for (int u = t; u < t + NST && u < ksteps; ++u)
                    mbar_wait(smem_addr(&bars[u % NST]), (u / NST) & 1);
            }
            return;
        }
        const double *As = smem + stage * STAGE;
        mma_stage<BM, BN>(acc, As, As + A_STAGE, wm, wn, lane);
        __syncthreads();  // every warp is done with this stage
        if (tid == 0 && t + NST < ksteps) issue(t + NST, stage);

        if ((t + 1) % STEPS_PER_BLOCK == 0 || t + 1 == ksteps) {
            epilogue<DUMP_BINS>(acc, t / STEPS_PER_BLOCK, m0 + wm * 16, n0 + wn * 32, lane, out);
            if constexpr (DUMP_BINS) return;
        }
    }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 3-D tensor map over a stack of `nz` row-major FP64 matrices of `rows` x
// `cols` (row stride ld doubles); box = [bz][by][bx].  Reads outside the
// extents are filled with zeros.
bool make_map(CUtensorMap *map, const double *base, uint64_t cols, uint64_t rows, uint64_t nz,
              uint64_t ld, uint32_t bx, uint32_t by, uint32_t bz) {
    auto enc = get_encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[3] = {cols, rows, nz};
    const cuuint64_t strides[2] = {ld * sizeof(double), ld * rows * sizeof(double)};
    const cuuint32_t box[3] = {bx, by, bz};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<double *>(base),
                           dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <bool DUMP>
cudaError_t launch_impl(const CascadeArgs &a, cudaStream_t stream) {
    CUtensorMap tm_a, tm_b;
    if (!make_map(&tm_a, a.a_slices, a.k, a.m, 4, a.lda_s, BK, BM, 4)) return cudaErrorInvalidValue;
    if (!make_map(&tm_b, a.b_slices, a.n, a.k, 7, a.ldb_s, BN, BK, 7)) return cudaErrorInvalidValue;
    // per device and cheap: set on every launch
    const cudaError_t attr_err = cudaFuncSetAttribute(
        cascade_fp64_kernel<DUMP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    if (attr_err != cudaSuccess) return attr_err;
    const long long tiles = (long long)((a.n + BN - 1) / BN) * ((a.m + BM - 1) / BM);
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    cascade_fp64_kernel<DUMP><<<(unsigned)tiles, NTHREADS, SMEM_BYTES, stream>>>(tm_a, tm_b, a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cascade_fp64(const CascadeArgs &a, cudaStream_t stream) {
    if (a.m <= 0 || a.n <= 0 || a.k <= 0) return cudaSuccess;
    return a.bins ? launch_impl<true>(a, stream) : launch_impl<false>(a, stream);
}

}  // namespace ddg
