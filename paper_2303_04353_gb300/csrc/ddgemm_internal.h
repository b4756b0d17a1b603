// Launchers shared between the translation units of libddgemm (not part of
// the public C ABI, which is include/ddgemm.h).
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

namespace ddg {

// k-block of the exactness argument (Sec. "Blocking for the k dimension").
constexpr int KC = 256;
// Digits of the fixed-width pieces at k = 256 (Sec. "Cascading vectors and
// dot products"): c0 = 22, c1 = 21, c2 = 21.
constexpr int C0 = 22, C1 = 21, C2 = 21;

// Output orientation of the cascaded panels.
//   VEC_MAJOR: out[(s * nvec + v) * ld + l]   (A: slices x m x k)
//   K_MAJOR:   out[(s * kdim + l) * ld + v]   (B: slices x k x n)
enum class PanelLayout { VEC_MAJOR, K_MAJOR };

// Cascade `nvec` vectors of length `kdim` (Appendix A) into 4 pieces (for A)
// or 7 panels (for B).  Element (v, l) of the input is at
//   x[v * ldx + l]  when vec_contig (the vector runs along memory), else
//   x[l * ldx + v].
// exps[p * nvec + v] receives the block exponent.  Returns a cudaError_t.
cudaError_t launch_split(int nslices, int nvec, int kdim, const double *x_hi,
                         const double *x_lo, long long ldx, bool vec_contig,
                         double *out, long long ld_out, PanelLayout layout, int *exps,
                         unsigned int *status, cudaStream_t stream);

struct CascadeArgs {
    int m, n, k;
    const double *a_slices;  // 4 x m x lda_s   (VEC_MAJOR)
    long long lda_s;
    const double *b_slices;  // 7 x k x ldb_s   (K_MAJOR)
    long long ldb_s;
    const int *exp_a;        // ceil(k/256) x m
    const int *exp_b;        // ceil(k/256) x n
    double *c_hi, *c_lo;
    long long ldc;
    int *flags;              // optional m x n
    unsigned int *status;    // optional
    double *bins;            // when non-null: write the bins of k-block 0 instead of C
};

// The ten products of eq. Gemm10 on the FP64 tensor path with the bin
// assembly fused in (one launch).
cudaError_t launch_cascade_fp64(const CascadeArgs &a, cudaStream_t stream);

}  // namespace ddg
