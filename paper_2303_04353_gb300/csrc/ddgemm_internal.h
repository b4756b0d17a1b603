// Launchers shared between the translation units of libddgemm (not part of
// the public C ABI, which is include/ddgemm.h).
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "../../include/ddgemm.h"

namespace ddg {

// k-block of the exactness argument (Sec. "Blocking for the k dimension").
constexpr int KC = 256;
// Digits of the fixed-width pieces at k = 256 (Sec. "Cascading vectors and
// dot products"): c0 = 22, c1 = 21, c2 = 21.
constexpr int C0 = 22, C1 = 21, C2 = 21;

// The kernels' bounded waits.  Every mbarrier wait gives up after limit_ns
// of global time, sets DDGEMM_DEV_TIMEOUT and ends the CTA's work.  For the
// failure-handling tests, a plan may also name one copy that is never issued
// (the producer of CTA `cta` skips its k-step or stage `step`): the barrier
// it would complete then never does, and the wait runs out without any fault.
// Only the diagnostic entry points (include/ddgemm_diag.h) set cta >= 0.
constexpr unsigned long long WAIT_LIMIT_DEFAULT_NS = 2000000000ull;  // ~2 s
struct WaitPlan {
    unsigned long long limit_ns = WAIT_LIMIT_DEFAULT_NS;
    int cta = -1;         // CTA whose copy is withheld (-1: none)
    long long step = -1;  // the producer's k-step (or ring iteration) withheld
};

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
    int products;            // 0: eq. Gemm10 (the method); 1: Gemm16; 2: bins 4-6 dropped
    int split;               // k-block groups per tile (1: no split)
    double *part_hi, *part_lo;  // split > 1: partial C of groups 1..split-1, [split-1][m][n]
    WaitPlan wait{};
    // add the k-blocks into C's (and the flags') current values instead of
    // starting from zero: a product over a range of k that continues an
    // earlier one, in the same k-block order as one launch over both
    bool accumulate = false;
};

// Split-k over whole k-blocks: the number of groups for a grid of `tiles`
// CTAs on `slots` resident CTAs, at most `cap` (and one k-block per group).
int choose_split(long long tiles, int kblocks, int slots, int cap);

// The least workspace ddgemm() accepts: ddgemm_workspace_size() without the
// room for split-k partial sums (api.cu).
size_t base_workspace_size(int m, int n, int k, const ddgemm_opts *opts);

// The ten products of eq. Gemm10 on the FP64 tensor path with the bin
// assembly fused in (one launch).
cudaError_t launch_cascade_fp64(const CascadeArgs &a, cudaStream_t stream);

// ---- INT8 form ------------------------------------------------------------
// The INT8 pieces are balanced digits of INT8_BITS bits for the mma.sync
// form (eight, as the paper's estimate of about 15 pieces implies) and of
// INT8_TC_BITS bits for the tcgen05 form (seven: its FP32 accumulators then
// stay exact over 256 entries instead of 64).
constexpr int INT8_BITS = 8, INT8_TC_BITS = 7;
// k-block: the longest power of two whose int32 diagonal sums stay exact
// (8 bits: 15 * 8192 * 2^14 < 2^31; 7 bits: 16 * 16384 * 2^12 <= 2^30).
__host__ __device__ constexpr int kblock_of_bits(int bits) { return bits == 8 ? 8192 : 16384; }
constexpr int KB8 = kblock_of_bits(INT8_BITS);
constexpr int KB8_TC = kblock_of_bits(INT8_TC_BITS);
// Piece counts with a compiled kernel (the fixed-point value needs
// 6 + 8 (s - 1) + 2 <= 127 bits, so s <= 15).
#define DDG_INT8_SLICE_CASES DDG_CASE(12) DDG_CASE(13) DDG_CASE(14) DDG_CASE(15)
constexpr int INT8_SLICES_DEFAULT = 15;
inline bool int8_slices_supported(int s) { return s >= 12 && s <= 15; }

// The tcgen05 form puts the products of plane i with planes 0..s-1-i in one
// MMA of N = 16 (s - i) <= 256 columns: s <= 16.  With eight-bit pieces
// (DDGEMM_VARIANT_INT8_TC8) the fixed-point bound above keeps s <= 15.
constexpr int INT8_TC_MAX_SLICES = 16;
constexpr int INT8_TC_SLICES_DEFAULT = 16;
inline bool int8_tc_slices_supported(int s) { return s >= 12 && s <= INT8_TC_MAX_SLICES; }
constexpr int INT8_TC8_SLICES_DEFAULT = 15;
inline bool int8_tc8_slices_supported(int s) { return s >= 12 && s <= 15; }

// tile_rows = 0: int8 digit planes out[(s * nvec + v) * ld_out + l] of
// eight-bit digits (bits = 8), ld_out a multiple of 16 and >= kdim.
// tile_rows = TH (a multiple of 8): bf16 digits of `bits` bits (7 or 8) in
// the tcgen05 form's tiled, pre-swizzled order (split_int8.cu),
// ceil(nvec / TH) * ceil(kdim / 16) * s blocks of TH x 16; entries past kdim
// up to a multiple of 16 are zero, rows past nvec are not written.
// exps[p * nvec + v] per k-block of kblock_of_bits(bits) entries.  Element
// (v, l) of the input is at x[v * ldx + l] when vec_contig, else
// x[l * ldx + v].
cudaError_t launch_split_int8(int slices, int nvec, int kdim, const double *x_hi,
                              const double *x_lo, long long ldx, bool vec_contig, void *out,
                              int tile_rows, int bits, long long ld_out, int *exps,
                              unsigned int *status, cudaStream_t stream);

struct Int8Args {
    int m, n, k, slices;
    const int8_t *a_digits;  // slices x m x ld_digits
    const int8_t *b_digits;  // slices x n x ld_digits
    long long ld_digits;
    const int *exp_a;        // ceil(k/KB8) x m
    const int *exp_b;        // ceil(k/KB8) x n
    double *c_hi, *c_lo;
    long long ldc;
    unsigned int *status;
    WaitPlan wait{};
};

cudaError_t launch_cascade_int8(const Int8Args &a, cudaStream_t stream);

// The INT8 form on the fifth-generation tensor cores: bf16 digit planes,
// tcgen05.mma with FP32 accumulation in tensor memory (exact over 256
// entries of seven-bit digits, 64 of eight-bit ones), int32 diagonal sums,
// exact assembly rounded once to FP64x2.  Tile heights of the tcgen05
// form's tiled digit order: rows of C per tile (A) and columns (B).  Its
// k-blocks are kblock_of_bits(bits) long.
constexpr int INT8_TC_BM = 128, INT8_TC_BN = 16;

struct Int8TcArgs {
    int m, n, k, slices;
    int bits;                  // digit width: 7 (INT8_TC) or 8 (INT8_TC8)
    const uint16_t *a_tiles;   // bf16, tiled order with TH = INT8_TC_BM
    const uint16_t *b_tiles;   // bf16, tiled order with TH = INT8_TC_BN
    const int *exp_a;          // ceil(k/kblock_of_bits(bits)) x m
    const int *exp_b;          // ceil(k/kblock_of_bits(bits)) x n
    double *c_hi, *c_lo;
    long long ldc;
    unsigned int *status;
    WaitPlan wait{};
};

cudaError_t launch_cascade_int8_tc(const Int8TcArgs &a, cudaStream_t stream);
// The eight-bit instantiations (cascade_int8_tc8.cu), reached through
// launch_cascade_int8_tc.
cudaError_t launch_cascade_int8_tc8(const Int8TcArgs &a, cudaStream_t stream);

// The batched tcgen05 INT8 form (batched_int8_tc.cu): workspace bytes, and
// the whole pass (returns a DDGEMM_* code).
// bits: 7 (DDGEMM_VARIANT_INT8_TC) or 8 (DDGEMM_VARIANT_INT8_TC8).
size_t batched_int8_tc_workspace_size(int count, const ddgemm_problem *probs_host, int slices,
                                      int bits);
// config: NULL (defaults) or checked by the caller.  events: NULL or three
// cudaEvent_t recorded before the plan, before the persistent kernel and
// after it.
int run_batched_int8_tc(int count, const ddgemm_problem *probs_host,
                        const ddgemm_problem *probs_dev, void *workspace, size_t ws_bytes,
                        cudaStream_t s, int slices, int bits, unsigned int *status,
                        const ddgemm_batch_config *config, const WaitPlan &wait = WaitPlan{},
                        void *const *events = nullptr);

// Whether a batch configuration's fields are in range (both forms).
inline bool batch_config_ok(const ddgemm_batch_config *c) {
    return !c || (c->tile >= DDGEMM_TILE_64x64 && c->tile <= DDGEMM_TILE_32x32 &&
                  c->order >= DDGEMM_ORDER_GIVEN && c->order <= DDGEMM_ORDER_LONGEST_K_FIRST &&
                  c->orient >= DDGEMM_ORIENT_FEWER_TILES && c->orient <= DDGEMM_ORIENT_GIVEN &&
                  c->planes >= DDGEMM_PLANES_INTERLEAVED && c->planes <= DDGEMM_PLANES_ASCENDING &&
                  c->row_group >= 0 && c->row_group <= 8);
}

// The exact assembly alone: (hi[i], lo[i]) = the FP64x2 nearest to
// sum_t diag[t * count + i] 2^(-12-7t) 2^scale[i].
cudaError_t launch_assemble_int8(int count, int slices, const int *diag, const int *scale,
                                 double *hi, double *lo, cudaStream_t stream);

}  // namespace ddg
