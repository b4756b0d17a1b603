// Phase one of the INT8 form (Sec. "FP64x2 in terms of INT8"): every FP64x2
// entry becomes s signed 7-bit digits of a fixed-point value.
//
// Per (vector, k-block of 16384 entries): sigma = 2^e with e the frexp
// exponent of max |hi| (as in the FP64 form).  Per entry, on the integer
// ALU (the FP64 pipe of this GPU is narrow, the integer pipes are not):
//   X = rne(hi 2^(F-e)) + rne(lo 2^(F-e)), F = 6 + b (s-1)   (exact, 128 bits)
//   balanced base-2^b digits d_0..d_{s-1} of X, most significant first,
//   |d_i| <= 2^(b-1) (d_0 within +-65), so x / sigma ~ sum_i d_i 2^(-6-b i),
//   with b = 8 for the int8 planes and b = 7 for the tcgen05 form's bf16.
// Output, for A (vectors = rows) and B (vectors = columns; transposed
// through shared memory) alike, either
//   * int8 digit planes [s][vector][ld] with k contiguous (mma.sync
//     m16n8k32 s8), or
//   * bf16 digits (a digit of at most 8 significant bits is exact in bf16)
//     in the tcgen05 form's tiled order: for every tile of TH vectors
//     (TH = 128 for A, 16 for B) and every k-step of 16 entries, the s
//     planes' TH x 16 blocks follow one another, each block being the
//     shared-memory image of a K-major operand with 32-byte swizzling (row r
//     at byte 32 r, its two 16-byte halves exchanged when bit 2 of r is
//     set).  One contiguous copy then stages a whole k-step of all planes.
#include <cuda_runtime.h>
#include <cstdint>

#include "ddgemm_internal.h"
#include "split_int8_device.cuh"

namespace ddg {
namespace {

using namespace split8;

// Per (vector, k-block) exponents, element (v, l) at x[v*ldx + l]: one warp
// per vector and block.
__global__ void __launch_bounds__(256)
int8_exps_contig_kernel(int nvec, int kdim, int blk, const double *__restrict__ x, long long ldx,
                        int *__restrict__ exps) {
    const int kb = (kdim + blk - 1) / blk;
    const int lane = threadIdx.x & 31;
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= (long long)nvec * kb) return;
    exps_contig_unit(lane, (int)(w / kb), (int)(w % kb), nvec, kdim, blk, x, ldx, exps);
}

// The same with element (v, l) at x[l*ldx + v]: one CTA per 64 vectors and
// block, with 16 row groups, as one problem has few such units (64 at
// n = 4096) and each must keep many loads in flight.
constexpr int EXPS_RG = 16;
__global__ void __launch_bounds__(64 * EXPS_RG)
int8_exps_strided_kernel(int nvec, int kdim, int blk, const double *__restrict__ x,
                         long long ldx, int *__restrict__ exps) {
    __shared__ unsigned long long part[EXPS_RG][64];
    exps_strided_unit<EXPS_RG>(blockIdx.x, blockIdx.y, nvec, kdim, blk, x, ldx, exps, part);
}

// BITS-bit digits: int8 planes (eight bits) or the tiled bf16 order (seven
// or eight).
template <int S, bool CONTIG, bool BF16, int BITS>
__global__ void __launch_bounds__(256)
int8_digits_kernel(int nvec, int kdim, const double *__restrict__ xh,
                   const double *__restrict__ xl, long long ldx, void *__restrict__ out_v,
                   long long ld_out, int th, const int *__restrict__ exps, unsigned int *status) {
    __shared__ double sh[TV][TK + 1];
    __shared__ double sl[TV][TK + 1];
    digits_unit<S, CONTIG, BF16, BITS>(blockIdx.y * TV, blockIdx.x * TK, nvec, kdim, xh, xl, ldx,
                                       out_v, ld_out, th, exps, status, sh, sl);
}

template <int S, bool BF16, int BITS>
cudaError_t launch_digits_t(int nvec, int kdim, const double *xh, const double *xl, long long ldx,
                            bool contig, void *out, long long ld_out, int th, const int *exps,
                            unsigned int *status, cudaStream_t stream) {
    const dim3 grid((kdim + TK - 1) / TK, (nvec + TV - 1) / TV);
    if (grid.y > 65535) return cudaErrorInvalidValue;
    if (contig)
        int8_digits_kernel<S, true, BF16, BITS><<<grid, 256, 0, stream>>>(
            nvec, kdim, xh, xl, ldx, out, ld_out, th, exps, status);
    else
        int8_digits_kernel<S, false, BF16, BITS><<<grid, 256, 0, stream>>>(
            nvec, kdim, xh, xl, ldx, out, ld_out, th, exps, status);
    return cudaGetLastError();
}

// int8 planes: eight-bit digits, s in 12..15.  Tiled bf16: seven-bit digits
// with s in 12..16, eight-bit ones with s in 12..15 (the fixed-point value
// needs 6 + bits (s - 1) + 2 <= 127 bits).
template <int S>
cudaError_t launch_digits(int nvec, int kdim, const double *xh, const double *xl, long long ldx,
                          bool contig, void *out, int tile_rows, int bits, long long ld_out,
                          const int *exps, unsigned int *status, cudaStream_t stream) {
    if (tile_rows && bits == INT8_TC_BITS)
        return launch_digits_t<S, true, INT8_TC_BITS>(nvec, kdim, xh, xl, ldx, contig, out, 0,
                                                      tile_rows, exps, status, stream);
    if constexpr (S <= 15) {
        if (bits != INT8_BITS) return cudaErrorInvalidValue;
        if (tile_rows)
            return launch_digits_t<S, true, INT8_BITS>(nvec, kdim, xh, xl, ldx, contig, out, 0,
                                                       tile_rows, exps, status, stream);
        return launch_digits_t<S, false, INT8_BITS>(nvec, kdim, xh, xl, ldx, contig, out, ld_out,
                                                    0, exps, status, stream);
    } else {
        return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_split_int8(int slices, int nvec, int kdim, const double *x_hi,
                              const double *x_lo, long long ldx, bool vec_contig, void *out,
                              int tile_rows, int bits, long long ld_out, int *exps,
                              unsigned int *status, cudaStream_t stream) {
    if (nvec <= 0 || kdim <= 0) return cudaSuccess;
    if (bits != INT8_BITS && bits != INT8_TC_BITS) return cudaErrorInvalidValue;
    if (tile_rows == 0 && (bits != INT8_BITS || ld_out % 16 != 0 || ld_out < kdim))
        return cudaErrorInvalidValue;
    if (tile_rows != 0 && tile_rows % 8 != 0) return cudaErrorInvalidValue;
    // block exponents per k-block of the digit width in use
    const int blk = kblock_of_bits(bits);
    const int kb = (kdim + blk - 1) / blk;
    if (vec_contig) {
        const long long blocks = ((long long)nvec * kb + 7) / 8;
        if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
        int8_exps_contig_kernel<<<(unsigned)blocks, 256, 0, stream>>>(nvec, kdim, blk, x_hi, ldx,
                                                                      exps);
    } else {
        if (kb > 65535) return cudaErrorInvalidValue;
        int8_exps_strided_kernel<<<dim3((nvec + 63) / 64, kb), 64 * EXPS_RG, 0, stream>>>(
            nvec, kdim, blk, x_hi, ldx, exps);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    switch (slices) {
        case 12: return launch_digits<12>(nvec, kdim, x_hi, x_lo, ldx, vec_contig, out, tile_rows,
                                          bits, ld_out, exps, status, stream);
        case 13: return launch_digits<13>(nvec, kdim, x_hi, x_lo, ldx, vec_contig, out, tile_rows,
                                          bits, ld_out, exps, status, stream);
        case 14: return launch_digits<14>(nvec, kdim, x_hi, x_lo, ldx, vec_contig, out, tile_rows,
                                          bits, ld_out, exps, status, stream);
        case 15: return launch_digits<15>(nvec, kdim, x_hi, x_lo, ldx, vec_contig, out, tile_rows,
                                          bits, ld_out, exps, status, stream);
        case 16: return launch_digits<16>(nvec, kdim, x_hi, x_lo, ldx, vec_contig, out, tile_rows,
                                          bits, ld_out, exps, status, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ddg
