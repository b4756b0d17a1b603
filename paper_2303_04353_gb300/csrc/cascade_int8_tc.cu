// Phases two and three of the INT8 form (Sec. "FP64x2 in terms of INT8",
// Sec. "Safely dropping lower order bins") on the fifth-generation tensor
// cores.  tcgen05 on this GPU has no integer MMA, but the digits are small
// integers, exact in bf16, and their products are summed exactly by an FP32
// accumulator while every partial sum stays below 2^24.
//
// Digits.  This form takes seven-bit pieces (balanced base 128, |digit| <=
// 64; the mma.sync form takes eight-bit ones): a product is at most 2^12 and
// diagonal t holds t + 1 <= 16 products per k, so over a chunk of 256
// entries every partial sum of a diagonal is an integer of magnitude
// <= 256 * 16 * 2^12 = 2^24: exact in FP32.  With eight-bit pieces
// (cascade_int8_tc8.cu, the same kernel core) the chunk is 64 entries, and
// four times as many read-outs and accumulator switches make that form
// slower per product.  After each chunk the FP32 sums are read out of
// tensor memory, converted (exactly) to integers and added into each
// output's exact k-block sums; over a k-block of 16384 entries a
// diagonal's sum stays within 2^30.
//
// Assembly.  Per k-block the exact value sum_t S_t 2^(-12-7t) sigma tau is
// formed in 192-bit integer arithmetic and rounded once to the nearest
// FP64x2 (hi = RN(x), lo = RN(x - hi)) from one left alignment of its
// magnitude; the blocks are added into C with the FP64x2 add (the first
// block is stored as it is).  This is one rounding where the paper's
// smallest-first FP64x2 sum of the diagonals has s.
//
// Tiling.  A C tile is 128 rows x 16 columns; k advances by 16.  The split
// wrote the digits tiled and pre-swizzled (split_int8.cu), so one bulk copy
// per operand and stage brings all s digit planes of A ([s][128][16] bf16,
// 64 KB at s = 16) and of B ([s][16][16]) into a three-deep ring, already in
// the 32-byte-swizzled K-major layout the MMA reads (a tensor-map copy with
// 32-byte rows would issue one request per row; the bulk copy issues few and
// large ones).  Per stage, one MMA per A plane i: M = 128,
// N = 16 (s - i) (B planes 0..s-1-i side by side), K = 16, accumulating
// into tensor-memory columns 16 i .. 16 s - 1, so that the product of
// planes i and j lands on diagonal i + j's 16 columns.  Two accumulator sets
// of 16 s columns alternate between chunks, so the drain of one overlaps
// the products of the next.
//
// Warps.  Warp 0 issues the bulk copies, warp 1 allocates tensor memory and
// issues the MMAs (one thread), warps 2-17 drain the accumulators and
// assemble: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (rows of
// the tile) and columns 4 ((w - 2) / 4) .. + 3 of every diagonal.  Per
// output it keeps the k-block's sums exactly in int64s, one per group of up
// to four consecutive diagonals (a group's chunk sum, combined with powers
// of 2^7, stays below 2^46 and its k-block sum below 2^56), and forms the
// block value from them once at the k-block's end.  The kernel is
// persistent: one CTA per SM walks the tiles in groups of 4 row tiles.
//
// Waits.  Every wait gives up after ~2 s, sets DDGEMM_DEV_TIMEOUT and a flag
// that ends the other roles' loops; the producer then waits (bounded) for
// its copies in flight, the MMA thread for its products, and tensor memory
// is released before the CTA exits.
#include "cascade_int8_tc_core.cuh"

namespace ddg {
namespace {

template <int S>
cudaError_t launch_tc(const Int8TcArgs &a, cudaStream_t stream) {
    if ((uintptr_t)a.a_tiles % 16 || (uintptr_t)a.b_tiles % 16) return cudaErrorInvalidValue;
    return launch_tc_single<S, INT8_TC_BITS>(a, stream);
}

template <int S>
__global__ void __launch_bounds__(256)
assemble_kernel(int count, const int *__restrict__ diag, const int *__restrict__ scale,
                double *__restrict__ hi, double *__restrict__ lo) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    __int128 H = 0, L = 0;
#pragma unroll
    for (int t = 0; t < S; ++t)
        add_diagonal<S, INT8_TC_BITS>(t, diag[(long long)t * count + i], H, L);
    round_dd<TcWidth<INT8_TC_BITS>::SPLIT>(H, L, scale[i] - 12 - INT8_TC_BITS * (S - 1), hi[i],
                                           lo[i]);
}

}  // namespace

cudaError_t launch_cascade_int8_tc(const Int8TcArgs &a, cudaStream_t stream) {
    if (a.m <= 0 || a.n <= 0 || a.k <= 0) return cudaSuccess;
    if (a.bits == INT8_BITS) return launch_cascade_int8_tc8(a, stream);
    if (a.bits != INT8_TC_BITS) return cudaErrorInvalidValue;
    switch (a.slices) {
        case 12: return launch_tc<12>(a, stream);
        case 13: return launch_tc<13>(a, stream);
        case 14: return launch_tc<14>(a, stream);
        case 15: return launch_tc<15>(a, stream);
        case 16: return launch_tc<16>(a, stream);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_assemble_int8(int count, int slices, const int *diag, const int *scale,
                                 double *hi, double *lo, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((count + 255) / 256);
    switch (slices) {
#define DDG_ASM(S)                                                                          \
    case S:                                                                                 \
        assemble_kernel<S><<<blocks, 256, 0, stream>>>(count, diag, scale, hi, lo);         \
        return cudaGetLastError();
        DDG_ASM(12) DDG_ASM(13) DDG_ASM(14) DDG_ASM(15) DDG_ASM(16)
#undef DDG_ASM
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace ddg
