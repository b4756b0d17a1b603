// Phase one of the cascade (Sec. "Practical considerations"): the fused
// scale + split kernels of the FP64 form.
//
// For every vector (a row of A or a column of B) and every k-block of
// K_C = 256 entries, one pass finds sigma = 2^e with e the frexp exponent of
// the largest |hi| in the block ("the smallest power of two greater than"
// the largest element, Sec. "Cascading vectors and dot products"), and a
// second pass over the same entries (L1/L2-resident) cascades each FP64x2
// entry following Appendix A (see split_device.cuh).  The pieces are written
// pre-multiplied by sigma_i in the order of eq. Gemm10:
// A -> [A0, s1 A1, s2 A2, s3 A3]; B -> [B0, s1 B1, s2 B2, s3 B3, s2 B4,
// s1 B5, B6], with B4, B5, B6 the FP64 roundings of the exact tails the
// split already holds.
#include "split_device.cuh"

namespace ddg {
namespace {

using namespace split_detail;

// Vectors run along memory (A not transposed, B transposed): one warp per
// (vector, k-block); lanes read 16-byte pairs, 512 contiguous bytes per warp
// instruction.
template <int NS, bool VEC>
__global__ void __launch_bounds__(256)
split_contig_kernel(int nvec, int kdim, const double *__restrict__ xh,
                    const double *__restrict__ xl, long long ldx, double *__restrict__ out,
                    long long ld_out, PanelLayout layout, int *__restrict__ exps,
                    unsigned int *status) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int kb = (kdim + KC - 1) / KC;
    if (warp >= (long long)nvec * kb) return;
    split_contig_unit<NS, VEC>(lane, (int)(warp / kb), (int)(warp % kb), nvec, kdim, xh, xl, ldx,
                               out, ld_out, layout, exps, status);
}

// Vectors are strided in memory (B not transposed, A transposed): one CTA
// per (k-block, 64 vectors); a warp reads 64 consecutive vectors of one row
// with 16-byte pairs.  Block maxima are combined in shared memory.
template <int NS, bool VEC>
__global__ void __launch_bounds__(256)
split_strided_kernel(int nvec, int kdim, const double *__restrict__ xh,
                     const double *__restrict__ xl, long long ldx, double *__restrict__ out,
                     long long ld_out, PanelLayout layout, int *__restrict__ exps,
                     unsigned int *status) {
    __shared__ double part[8][64];
    __shared__ int sexp[64];
    split_strided_unit<NS, VEC>(blockIdx.x, blockIdx.y, nvec, kdim, xh, xl, ldx, out, ld_out,
                                layout, exps, status, part, sexp);
}

template <int NS>
cudaError_t launch_split_ns(int nvec, int kdim, const double *xh, const double *xl,
                            long long ldx, bool vec_contig, double *out, long long ld_out,
                            PanelLayout layout, int *exps, unsigned int *status,
                            cudaStream_t stream) {
    const int kb = (kdim + KC - 1) / KC;
    const bool vec = (ldx % 2 == 0) && ((uintptr_t)xh % 16 == 0) && ((uintptr_t)xl % 16 == 0);
    if (vec_contig) {
        const long long warps = (long long)nvec * kb;
        const long long blocks = (warps + 7) / 8;
        if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
        if (vec)
            split_contig_kernel<NS, true><<<(unsigned)blocks, 256, 0, stream>>>(
                nvec, kdim, xh, xl, ldx, out, ld_out, layout, exps, status);
        else
            split_contig_kernel<NS, false><<<(unsigned)blocks, 256, 0, stream>>>(
                nvec, kdim, xh, xl, ldx, out, ld_out, layout, exps, status);
    } else {
        if (kb > 65535) return cudaErrorInvalidValue;
        dim3 grid((nvec + 63) / 64, kb);
        if (vec)
            split_strided_kernel<NS, true><<<grid, 256, 0, stream>>>(
                nvec, kdim, xh, xl, ldx, out, ld_out, layout, exps, status);
        else
            split_strided_kernel<NS, false><<<grid, 256, 0, stream>>>(
                nvec, kdim, xh, xl, ldx, out, ld_out, layout, exps, status);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_split(int nslices, int nvec, int kdim, const double *x_hi,
                         const double *x_lo, long long ldx, bool vec_contig, double *out,
                         long long ld_out, PanelLayout layout, int *exps, unsigned int *status,
                         cudaStream_t stream) {
    if (nvec <= 0 || kdim <= 0) return cudaSuccess;
    if (nslices == 4)
        return launch_split_ns<4>(nvec, kdim, x_hi, x_lo, ldx, vec_contig, out, ld_out, layout,
                                  exps, status, stream);
    if (nslices == 7)
        return launch_split_ns<7>(nvec, kdim, x_hi, x_lo, ldx, vec_contig, out, ld_out, layout,
                                  exps, status, stream);
    return cudaErrorInvalidValue;
}

}  // namespace ddg
