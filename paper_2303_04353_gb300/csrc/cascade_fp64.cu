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
// Waits.  Every mbarrier wait gives up after args.wait.limit_ns (~2 s) of
// global time: the CTA then sets DDGEMM_DEV_TIMEOUT, writes NaN into the
// outputs it owns (its C tile, or its partial tile under split-k, so that
// the fix-up cannot add stale partial sums into a plausible C), waits
// (again bounded) for its own copies still in flight and returns.
#include <cuda_runtime.h>

#include <cstdint>

#include "cascade_core.cuh"
#include "ddgemm_internal.h"
#include "tma.cuh"

namespace ddg {
namespace {

using Tile = Fp64Tile<4, 2>;  // 64 x 64, 8 warps
constexpr int BM = Tile::BM, BN = Tile::BN, BK = CBK, NST = 3, NTHREADS = Tile::NTHREADS;
constexpr int A_STAGE = Tile::A_STAGE;
constexpr int STAGE = Tile::STAGE;
constexpr uint32_t STAGE_BYTES = STAGE * sizeof(double);
constexpr int STEPS_PER_BLOCK = KC / BK;
constexpr size_t SMEM_BYTES = (size_t)NST * STAGE * sizeof(double) + NST * sizeof(uint64_t) + 1024;
template <bool DUMP_BINS, int PRODUCTS>
__global__ void __launch_bounds__(NTHREADS, 1)
cascade_fp64_kernel(const __grid_constant__ CUtensorMap tm_a,
                    const __grid_constant__ CUtensorMap tm_b, const CascadeArgs args) {
    extern __shared__ unsigned char smem_raw[];
    double *smem = reinterpret_cast<double *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NST * STAGE);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 3, wn = warp >> 2;
    const int tiles_m = (args.m + BM - 1) / BM, tiles_n = (args.n + BN - 1) / BN;
    const unsigned tiles = (unsigned)tiles_m * (unsigned)tiles_n;
    const int part = (int)(blockIdx.x / tiles);     // k-block group (split-k)
    int tm, tn;
    grouped_tile(blockIdx.x % tiles, tiles_m, tiles_n, 8, tm, tn);
    const int m0 = tm * BM, n0 = tn * BN;
    const int total_steps = (args.k + BK - 1) / BK;
    const int kblocks = (args.k + KC - 1) / KC;
    const int kb_begin = part * kblocks / args.split, kb_end = (part + 1) * kblocks / args.split;
    const int t0 = kb_begin * STEPS_PER_BLOCK;
    const int ksteps = min(kb_end * STEPS_PER_BLOCK, total_steps) - t0;

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
        double *dst = smem + stage * STAGE;
        mbar_arrive_expect_tx(bar, STAGE_BYTES);
        tma_load_3d(smem_addr(dst), &tm_a, bar, (t0 + t) * BK, m0, 0);
        tma_load_3d(smem_addr(dst + A_STAGE), &tm_b, bar, n0, (t0 + t) * BK, 0);
    };
    if (tid == 0) {
        for (int s = 0; s < NST && s < ksteps; ++s) issue(s, s);
    }

    Acc acc;
    zero_acc(acc);
    // group 0 sums into C; the others into their partial buffers
    const long long mn = (long long)args.m * args.n;
    const EpilogueOut out =
        part == 0 ? EpilogueOut{args.m, args.n, args.exp_a, args.exp_b, args.c_hi, args.c_lo,
                                args.ldc, args.flags, args.bins}
                  : EpilogueOut{args.m, args.n, args.exp_a, args.exp_b,
                                args.part_hi + (part - 1) * mn, args.part_lo + (part - 1) * mn,
                                args.n, nullptr, nullptr};

    for (int t = 0; t < ksteps; ++t) {
        const int stage = t % NST;
        const uint32_t parity = (t / NST) & 1;
        const bool ok = mbar_wait_limit(smem_addr(&bars[stage]), parity, limit);
        if (__syncthreads_or(!ok)) {
            if constexpr (!DUMP_BINS) poison(m0 + wm * 16, n0 + wn * 32, lane, out);
            if (tid == 0) {
                if (args.status) atomicOr(args.status, DEV_TIMEOUT_BIT);
                // Copies already issued for steps t .. t+NST-1 may still be in
                // flight into this CTA's shared memory: wait for them, bounded.
                for (int u = t; u < t + NST && u < ksteps; ++u)
                    if (u != withheld)
                        mbar_wait_limit(smem_addr(&bars[u % NST]), (u / NST) & 1, limit);
            }
            return;
        }
        const double *As = smem + stage * STAGE;
        mma_stage<BM, BN, PRODUCTS>(acc, As, As + A_STAGE, wm, wn, lane);
        __syncthreads();  // every warp is done with this stage
        if (tid == 0 && t + NST < ksteps) issue(t + NST, stage);

        const int ta = t0 + t;  // the k-step in the whole of k
        if ((ta + 1) % STEPS_PER_BLOCK == 0 || ta + 1 == total_steps) {
            const int p = ta / STEPS_PER_BLOCK;
            // group 0's first k-block starts C from zero unless the launch
            // continues an earlier product; the partials always start from zero
            epilogue<DUMP_BINS>(acc, p, p == kb_begin && !(args.accumulate && part == 0),
                                m0 + wm * 16, n0 + wn * 32, lane, out);
            if constexpr (DUMP_BINS) return;
        }
    }
}

// Split-k: C (group 0) += the partial sums of groups 1..parts-1, in order,
// in FP64x2.
__global__ void __launch_bounds__(256)
split_fixup_kernel(int m, int n, double *c_hi, double *c_lo, long long ldc, const double *p_hi,
                   const double *p_lo, int parts) {
    const long long mn = (long long)m * n;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < mn;
         x += (long long)gridDim.x * blockDim.x) {
        const long long o = (x / n) * ldc + x % n;
        double h = c_hi[o], l = c_lo[o];
        for (int q = 0; q < parts - 1; ++q) dd_add(h, l, p_hi[q * mn + x], p_lo[q * mn + x], h, l);
        c_hi[o] = h;
        c_lo[o] = l;
    }
}

template <bool DUMP, int PRODUCTS>
cudaError_t launch_impl(const CascadeArgs &a, cudaStream_t stream) {
    CUtensorMap tm_a, tm_b;
    // A pieces [4][m][lda_s], box [4][64][8]; B panels [7][k][ldb_s], box [7][8][64]
    if (!encode_map_3d(&tm_a, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, a.a_slices, a.k, a.m, 4,
                       a.lda_s, BK, BM, 4) ||
        !encode_map_3d(&tm_b, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, a.b_slices, a.n, a.k, 7,
                       a.ldb_s, BN, BK, 7))
        return cudaErrorInvalidValue;
    // per device and cheap: set on every launch
    const cudaError_t attr_err = cudaFuncSetAttribute(
        cascade_fp64_kernel<DUMP, PRODUCTS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)SMEM_BYTES);
    if (attr_err != cudaSuccess) return attr_err;
    const long long tiles = (long long)((a.n + BN - 1) / BN) * ((a.m + BM - 1) / BM);
    if (tiles * a.split > 0x7fffffffLL || a.split < 1) return cudaErrorInvalidValue;
    cascade_fp64_kernel<DUMP, PRODUCTS><<<(unsigned)(tiles * a.split), NTHREADS, SMEM_BYTES,
                                          stream>>>(tm_a, tm_b, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || a.split == 1) return e;
    const long long mn = (long long)a.m * a.n;
    const long long blocks = (mn + 255) / 256;
    split_fixup_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, stream>>>(
        a.m, a.n, a.c_hi, a.c_lo, a.ldc, a.part_hi, a.part_lo, a.split);
    return cudaGetLastError();
}

}  // namespace

int choose_split(long long tiles, int kblocks, int slots, int cap) {
    // Estimated span in k-block times: ceil(CTAs / slots) waves of the
    // longest group (ceil(kblocks / s) k-blocks), plus a 0.2% charge per
    // extra group for the partial sums and the fix-up pass (measured on
    // GB300: a CTA's start-up and epilogue cost well under 1% of a k-block);
    // the least wins, ties to fewer groups.
    if (tiles <= 0 || kblocks <= 0 || slots <= 0) return 1;
    int best = 1;
    double best_span = 0.0;
    for (int s = 1; s <= cap && s <= kblocks; ++s) {
        const long long waves = (tiles * s + slots - 1) / slots;
        const int longest = (kblocks + s - 1) / s;
        const double span = (double)(waves * longest) * (1.0 + 0.002 * (s - 1));
        if (s == 1 || span < best_span) {
            best_span = span;
            best = s;
        }
    }
    return best;
}

cudaError_t launch_cascade_fp64(const CascadeArgs &a, cudaStream_t stream) {
    if (a.m <= 0 || a.n <= 0 || a.k <= 0) return cudaSuccess;
    if (a.bins) return launch_impl<true, PRODUCTS_GEMM10>(a, stream);
    switch (a.products) {
        case PRODUCTS_GEMM16: return launch_impl<false, PRODUCTS_GEMM16>(a, stream);
        case PRODUCTS_DROP456: return launch_impl<false, PRODUCTS_DROP456>(a, stream);
        default: return launch_impl<false, PRODUCTS_GEMM10>(a, stream);
    }
}

}  // namespace ddg
