/*
 * ddgemm.h - cascading double-double GEMM on one GB300 GPU (sm_103a).
 *
 * C := A B with A, B, C in double-double (FP64x2): every matrix is a pair of
 * FP64 arrays (hi, lo) and an entry's value is the exact real hi + lo
 * (Parikh, van de Geijn, Henry, "Cascading GEMM: High Precision from Low
 * Precision", Sec. "FP64 and FP64x2 numbers", eq. doubledouble).  The paper
 * states the operation as C := A B, with no alpha or beta (Sec.
 * "Introduction"); so does this library.
 *
 * Method (Sec. "Cascading matrices and GEMM", eq. Gemm10; Sec. "Simple";
 * Appendix A): k is staged in blocks of K_C = 256.  For every k-block each
 * row of A and each column of B is scaled by a power of two (sigma, tau)
 * and split into four FP64 pieces holding 22, 21 and 21 fixed-point digits
 * (more for a block shorter than 256) plus an FP64 remainder; B also gets
 * the combined panels B4, B5, B6.  Ten FP64 products land in four bins
 * (0, 1, 2 exact; 3-6 rounded), which are added from bin 3-6 up to bin 0
 * in FP64x2, scaled back by sigma tau and accumulated into C in FP64x2.
 *
 * Conventions for every entry point:
 *   - Matrices are row-major.  Element (r, c) of a matrix with leading
 *     dimension ld is at ptr[r * ld + c].
 *   - Every matrix pointer is DEVICE memory owned by the caller (except
 *     ddgemm_host(), whose matrices are in host memory), and the library
 *     never allocates device memory, frees or keeps a pointer after the
 *     call: scratch space is the caller's `workspace`.
 *   - When a call sets DDGEMM_DEV_TIMEOUT in the status word, its outputs
 *     are undefined (the FP64 form writes NaN into the tiles whose wait gave
 *     up; the other forms leave the tiles they did not finish as they were).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued on it and the call returns without waiting.
 *   - The return value reports host-side checks and launch errors only.
 *     Conditions found on the device are OR-ed into the optional word
 *     opts->status_dev (DDGEMM_DEV_* bits), which the caller reads after
 *     synchronising the stream.
 *   - Inputs need not be normalised (|lo| may reach ulp(hi)); outputs are
 *     normalised: hi == fl(hi + lo).
 *   - Results near the FP64 overflow threshold or in the subnormal range are
 *     outside the paper's error analysis; non-finite inputs set
 *     DDGEMM_DEV_NONFINITE and leave the affected outputs unspecified.
 */
#ifndef DDGEMM_H
#define DDGEMM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Host-side return codes. */
#define DDGEMM_OK            0 /* work enqueued */
#define DDGEMM_EINVAL        1 /* bad size, leading dimension, pointer or option */
#define DDGEMM_EWORKSPACE    2 /* workspace NULL, misaligned or smaller than required */
#define DDGEMM_ECUDA         3 /* a CUDA runtime call or kernel launch failed */
#define DDGEMM_EUNSUPPORTED  4 /* valid request this build does not implement */

/* Device status bits, OR-ed into *opts->status_dev. */
#define DDGEMM_DEV_NONFINITE 0x1u /* an input entry was Inf or NaN */
#define DDGEMM_DEV_TIMEOUT   0x2u /* a bounded wait inside a kernel gave up;
                                     outputs of that call are undefined */

/* opts->variant */
#define DDGEMM_VARIANT_FP64  0    /* ten FP64 products on the FP64 tensor path */
#define DDGEMM_VARIANT_INT8  1    /* the cascade re-sliced into INT8 pieces (below) */
/* Accuracy ablations of the FP64 form (same pieces, other products): */
#define DDGEMM_VARIANT_FP64_GEMM16  2 /* all sixteen products of eq. Gemm16 */
#define DDGEMM_VARIANT_FP64_DROP456 3 /* bins 0-3 of eq. Gemm16 only: bins 4-6
                                         dropped (ten products, not folded) */
/* The INT8 form with its digit products on the fifth-generation tensor
 * cores (tcgen05.mma, bf16 digits, FP32 accumulation, exact) and the exact
 * assembly (below): seven-bit pieces (INT8_TC), or the mma.sync form's
 * eight-bit pieces and accuracy (INT8_TC8): */
#define DDGEMM_VARIANT_INT8_TC 4
#define DDGEMM_VARIANT_INT8_TC8 5

typedef struct ddgemm_opts {
    /* 0: A is m x k (lda >= k).  1: A is stored k x m (lda >= m) and the
     * operation uses its transpose.  Same for B: 0 = k x n (ldb >= n),
     * 1 = stored n x k (ldb >= k). */
    int trans_a;
    int trans_b;
    /* DDGEMM_VARIANT_FP64 (default) or DDGEMM_VARIANT_INT8.
     *
     * INT8 (Sec. "FP64x2 in terms of INT8", Sec. "Safely dropping lower
     * order bins"): per (row of A, k-block of 8192) and (k-block, column of
     * B), sigma = 2^e as in the FP64 form; each entry becomes the fixed-point
     * integer X = rne(hi 2^(F-e)) + rne(lo 2^(F-e)), F = 6 + 8 (s - 1),
     * written as s balanced base-256 digits in [-128, 127] (eight-bit INT8
     * pieces, the first within +-65).  The products of digit planes i, j
     * with i + j <= s - 1 are accumulated exactly in int32 per diagonal
     * t = i + j on the integer tensor path, and the diagonals are added
     * smallest first in FP64x2.  Error per entry and k-block: at most about
     * (4 s + 2) 2^-8s k sigma tau (conversion and dropped diagonals) plus
     * FP64x2 rounding.  flags_dev is not supported with it
     * (DDGEMM_EUNSUPPORTED).
     *
     * INT8_TC: the same cascade with seven-bit pieces (balanced base-128
     * digits in [-64, 64], F = 6 + 7 (s - 1), k-blocks of 16384) and the
     * digit products on the tcgen05 tensor cores: a digit is exact in
     * bf16, a product is at most 2^12, and over 256 entries a diagonal's
     * FP32 accumulator holds integers of at most 2^24, so it is exact; it
     * is read out every 256 entries into an exact integer sum (eight-bit
     * pieces would allow 64 entries only).  Per k-block the value
     * sum_t S_t 2^(-12-7t) sigma tau is formed exactly and rounded once to
     * the nearest FP64x2 (hi = RN(x), lo = RN(x - hi)) before the FP64x2
     * add into C: a more accurate reading of "add the results across bins
     * in FP64x2" than the smallest-first sum.  flags_dev is not supported.
     *
     * INT8_TC8: INT8_TC with the eight-bit pieces of INT8 (balanced
     * base-256 digits, F = 6 + 8 (s - 1), k-blocks of 8192, s in 12..15):
     * the fixed point and accuracy of INT8 at the speed of the tensor
     * cores.  An eight-bit product is at most 2^14, so the FP32
     * accumulators are read out every 64 entries instead of 256, which
     * makes it slower than INT8_TC.  Assembly as for INT8_TC, with weights
     * 2^(-12-8t). */
    int variant;
    /* Optional device word (or NULL): DDGEMM_DEV_* bits are OR-ed into it.
     * The library never clears it. */
    unsigned int *status_dev;
    /* Optional device int32 array of m * n entries, row-major with leading
     * dimension n (or NULL).  Written with, per output entry, the number of
     * k-blocks whose bin 0 came out zero while that block's contribution
     * did not: the paper's cheap cancellation detection (Sec. "Detecting
     * cancellation error", Sec. "Adding detection of cancellation errors").
     * Nothing is corrected. */
    int *flags_dev;
    /* Optional (or NULL): three cudaEvent_t handles, passed as void*, that
     * ddgemm() records on `stream` before the split (phase one), between the
     * split and the ten products (phases two and three, one kernel) and
     * after it, so that a caller can time each phase on the device
     * (ddgemm_batched(): before its plan, before its persistent kernel and
     * after it). */
    void **phase_events;
    /* INT8 forms only: pieces per entry, s (s + 1) / 2 digit products per k.
     * INT8: s in {12, 13, 14, 15}, 0 = 15 (the paper estimates 14-15; 120
     * products).  INT8_TC: s in {12, ..., 16}, 0 = 16 (seven-bit pieces;
     * 136 products).  INT8_TC8: s in {12, ..., 15}, 0 = 15. */
    int int8_slices;
    /* FP64 forms: split-k over whole 256-entry k-blocks when a grid of 64 x 64
     * tiles would leave SMs idle.  Group g of a tile sums its run of k-blocks
     * into C (g = 0) or into a partial buffer in the workspace, and one more
     * kernel adds the partials into C in group order, in FP64x2.  0 = chosen
     * per launch from the SM count (grids below 4096 tiles only, at most
     * min(16, ceil(8192 / tiles)) groups, only as many as the workspace
     * holds); 1 = never (C then follows the paper's k order bit for bit);
     * 2-16 = that many groups (capped by the k-blocks and the workspace).
     * Not used with flags_dev. */
    int split_k;
} ddgemm_opts;

/* Bytes of device workspace ddgemm() can use for this problem (0 when m, n
 * or k is 0).  Holds the four cascaded pieces of A (4 m k doubles, Appendix
 * A), the seven cascaded panels of B (7 k n doubles), the per-block
 * exponents of sigma and tau, and, for grids of fewer than 4096 tiles of
 * 64 x 64, room for split-k partial C (2 m n doubles each, at most 15 and
 * at most about 0.5 GB in all; see split_k).  ddgemm() accepts a smaller
 * workspace down to the size without the partials and then splits less or
 * not at all.  opts may be NULL (all defaults).  Returns 0 on invalid
 * sizes. */
size_t ddgemm_workspace_size(int m, int n, int k, const ddgemm_opts *opts);

/* How many split-k groups ddgemm() launches for this problem (see split_k;
 * the paper's k-blocking, Sec. "Blocking for the k dimension", summed in
 * groups) on a GPU with `sms` multiprocessors and a workspace of ws_bytes:
 * 1 for the INT8 form, with flags_dev, or when there is no room for
 * partials.  Host only, no GPU needed.  Returns 0 on invalid arguments. */
int ddgemm_split_groups(int m, int n, int k, int sms, size_t ws_bytes, const ddgemm_opts *opts);

/* C := A B in FP64x2 by the ten-GEMM cascade (eq. Gemm10).
 *   m, n, k      sizes of op(A) (m x k), op(B) (k x n) and C (m x n); >= 0.
 *                k = 0 writes C = 0.
 *   A_hi, A_lo   op(A) as described for opts->trans_a, leading dim lda.
 *   B_hi, B_lo   op(B) likewise, leading dim ldb.
 *   C_hi, C_lo   output, m x n, leading dim ldc >= n.  Must not overlap the
 *                inputs or the workspace.
 *   workspace    device buffer of ddgemm_workspace_size() bytes (at the
 *                least that size less the split-k partials), 256-byte
 *                aligned; its contents on return are the cascaded panels
 *                (unspecified layout).
 *   opts         may be NULL.
 * Returns DDGEMM_OK or an error code; on error nothing was enqueued. */
int ddgemm(int m, int n, int k,
           const double *A_hi, const double *A_lo, int lda,
           const double *B_hi, const double *B_lo, int ldb,
           double *C_hi, double *C_lo, int ldc,
           void *workspace, size_t ws_bytes, void *stream,
           const ddgemm_opts *opts);

/* Backward pass of C = op(A) op(B) for a loss L with dL/dC = dC (all FP64x2):
 * dA = dC op(B)^T and dB = op(A)^T dC, each computed by the same cascade
 * (two ddgemm() calls on `stream`).  The paper has no backward pass; this is
 * the chain rule applied to its product.
 *   A, B, opts   as passed to the forward ddgemm() (trans flags included).
 *   dC_hi/lo     m x n, leading dim lddc >= n.
 *   dA_hi/lo     op(A)'s storage shape: m x k (ldda >= k) if trans_a = 0,
 *                else k x m (ldda >= m).
 *   dB_hi/lo     B's storage shape: k x n (lddb >= n) if trans_b = 0, else
 *                n x k (lddb >= k).
 *   workspace    at least ddgemm_backward_workspace_size() bytes, reused by
 *                both products.
 * opts->flags_dev and opts->phase_events are ignored. */
size_t ddgemm_backward_workspace_size(int m, int n, int k, const ddgemm_opts *opts);
int ddgemm_backward(int m, int n, int k,
                    const double *A_hi, const double *A_lo, int lda,
                    const double *B_hi, const double *B_lo, int ldb,
                    const double *dC_hi, const double *dC_lo, int lddc,
                    double *dA_hi, double *dA_lo, int ldda,
                    double *dB_hi, double *dB_lo, int lddb,
                    void *workspace, size_t ws_bytes, void *stream,
                    const ddgemm_opts *opts);

/* ---- Batched: many independent problems in one pass ----------------------
 * The paper has no batched form; this schedules its FP64 cascade (eq.
 * Gemm10, Sec. "Simple") over many problems at once.  Each C is
 * bit-identical to what ddgemm() computes for that problem alone. */
typedef struct ddgemm_problem {
    int m, n, k;        /* C (m x n) := A (m x k) B (k x n); any may be 0 */
    int lda, ldb, ldc;  /* row-major leading dimensions (>= k, n, n) */
    const double *A_hi, *A_lo, *B_hi, *B_lo;  /* device */
    double *C_hi, *C_lo;                      /* device */
} ddgemm_problem;

#define DDGEMM_TILE_64x64 0
#define DDGEMM_TILE_32x64 1
#define DDGEMM_TILE_64x32 2
#define DDGEMM_TILE_32x32 3
#define DDGEMM_ORDER_GIVEN           0 /* tiles in problem order */
#define DDGEMM_ORDER_LONGEST_K_FIRST 1 /* problems by k, then m n, descending */
/* tcgen05 forms: the tile grid of a problem */
#define DDGEMM_ORIENT_FEWER_TILES 0 /* C or C^T = B^T A^T, whichever needs fewer tiles */
#define DDGEMM_ORIENT_GIVEN       1 /* always C */
/* tcgen05 forms: the order of a k-step's MMAs over the A digit planes */
#define DDGEMM_PLANES_INTERLEAVED 0 /* 0, S-1, 1, S-2, ...: a narrow MMA after a wide one */
#define DDGEMM_PLANES_ASCENDING   1 /* 0, 1, ..., S-1 */

typedef struct ddgemm_batch_config {
    int tile;      /* FP64 form: DDGEMM_TILE_*, the C tile of the persistent
                      kernel's CTAs (the tcgen05 forms' tile is 128 x 16) */
    int order;     /* both forms: DDGEMM_ORDER_*, the order in which the
                      persistent CTAs take the problems' tiles */
    int orient;    /* tcgen05 forms: DDGEMM_ORIENT_* */
    int planes;    /* tcgen05 forms: DDGEMM_PLANES_* */
    int row_group; /* tcgen05 forms: row tiles per group of a problem's tile
                      order (the CTAs walk a group's columns, then the next
                      group), 1 .. 8; 0 = 4 */
} ddgemm_batch_config;

/* Workspace bytes for ddgemm_batched() over these problems (host array)
 * with these opts (NULL: the FP64 form): a plan area plus every problem's
 * cascaded panels, or digit tiles for INT8_TC. */
size_t ddgemm_batched_workspace_size(int count, const ddgemm_problem *probs_host,
                                     const ddgemm_opts *opts);

/* C_i := A_i B_i for count problems.  The schedule (config) changes the
 * time, never a bit of any C_i: every configuration computes each problem
 * bit-identically.  FP64 form: four launches on `stream`:
 *   1. a one-CTA plan kernel that reads probs_dev and writes the problems'
 *      workspace offsets, the tile schedule and a work counter into the
 *      workspace;
 *   2. and 3. the split of every A and every B (grid-stride kernels);
 *   4. one persistent cascade kernel (CTAs pull (problem, tile) items from
 *      the counter until none are left).
 *   probs_host  the problems, on the host: checked, and used to size the
 *               launches and the workspace.
 *   probs_dev   the same array in device memory (the caller uploads it); all
 *               device-side information comes from it, so the call can be
 *               captured into a CUDA graph once it has been uploaded.
 *   workspace   >= ddgemm_batched_workspace_size() bytes, 256-byte aligned.
 *   opts        NULL or: trans flags 0, variant FP64, INT8_TC or INT8_TC8,
 *               no flags_dev (else DDGEMM_EUNSUPPORTED); status_dev is
 *               honoured; int8_slices for INT8_TC (12-16; 0 = 16) and
 *               INT8_TC8 (12-15; 0 = 15); phase_events NULL or three
 *               cudaEvent_t (as void *) recorded on `stream` before the
 *               plan, after the splits (before the persistent kernel) and
 *               after the persistent kernel.
 *   config      NULL = {DDGEMM_TILE_64x64, DDGEMM_ORDER_LONGEST_K_FIRST,
 *               DDGEMM_ORIENT_FEWER_TILES, DDGEMM_PLANES_INTERLEAVED, 4}.
 *               Out-of-range fields: DDGEMM_EINVAL.
 * INT8_TC and INT8_TC8 (the INT8 form on the tcgen05 tensor cores, see
 * DDGEMM_VARIANT_INT8_TC): four launches, a plan, the exponents of every A
 * and of every B (one launch), the digits of all of them, and one persistent tcgen05
 * kernel over the (problem, 128 x 16 tile) items (tile grids over C or C^T
 * and the tile order as config says); each C_i is bit-identical to ddgemm()
 * with that variant.  The workspace size depends on opts (pass the same opts
 * to both calls), not on config.
 * Problems with m or n = 0 are skipped; k = 0 writes C = 0.  The ordering
 * by k costs count^2 / 256 comparisons in the plan kernel. */
int ddgemm_batched(int count, const ddgemm_problem *probs_host,
                   const ddgemm_problem *probs_dev, void *workspace, size_t ws_bytes,
                   void *stream, const ddgemm_opts *opts,
                   const ddgemm_batch_config *config);

/* Bytes of device buffer ddgemm_host() needs for this problem: dense device
 * copies of A, B and C (hi and lo of each) and the workspace for the row
 * chunks it runs.  0 when m or n is 0 or the arguments are invalid. */
size_t ddgemm_host_buffer_size(int m, int n, int k, const ddgemm_opts *opts);

/* ddgemm() on HOST operands: C := op(A) op(B) with A_hi, A_lo, B_hi, B_lo,
 * C_hi and C_lo in host memory (same shapes, leading dimensions and trans
 * flags as ddgemm()).  The paper has no counterpart (its operands are in
 * the CPU's memory already); this packages the host-to-device copies with
 * the cascade so that they overlap it.
 *
 *   - buffer: device memory of >= ddgemm_host_buffer_size() bytes, 256-byte
 *     aligned, owned by the caller; it holds the copies and the workspace.
 *   - The copies run on two streams of the library's own, ordered by
 *     fifteen events: a call takes such a set from a per-device pool and
 *     returns it when it returns, so only the first call on a device (and a
 *     call that overlaps another one on the host) creates them; they live
 *     until the process exits (do not reset the device between calls).
 *     op(A) is copied in up to four chunks of rows: every chunk's split and
 *     products run on `stream` as soon as its rows (and B) have arrived,
 *     and its rows of C are copied back while the next chunk computes.
 *     Chunks hold at least 1024 tiles of the form's kernel (about seven
 *     waves of the GPU), so small problems run as one chunk.  The INT8
 *     forms copy B whole first.  The FP64 forms, when there are several
 *     chunks, copy the first chunk of A first and then B in up to four
 *     parts of whole 256-entry k-blocks, and multiply the first chunk part
 *     by part as the parts arrive (each part's product added into C in
 *     k-block order, as ddgemm() does).
 *   - Each chunk computes exactly what ddgemm() computes for those rows:
 *     C is bit-identical to ddgemm() on device copies of the operands,
 *     except that the FP64 form may choose a different split-k grouping
 *     for a chunk (split_k = 1 makes it bit-identical there too).
 *   - `stream` waits for the last copy, so synchronising it (or an event
 *     recorded on it after the call) means C is on the host.  Nothing of the
 *     call starts before the work already enqueued on `stream`, so calls on
 *     one stream may reuse one buffer.  The host arrays must stay valid and
 *     unchanged until then.
 *   - Page-locked host memory (cudaHostAlloc, cudaHostRegister) lets the
 *     copies run asynchronously and the call return at once.  With pageable
 *     memory the driver stages the copies and the call returns only when the
 *     copies to the host have completed.  Device or managed pointers work
 *     too (the copies are then device to device).
 *   - opts as for ddgemm(); phase_events is ignored.  flags_dev, if given,
 *     is a device array as for ddgemm().
 *   - Errors: DDGEMM_EINVAL, DDGEMM_EUNSUPPORTED as for ddgemm();
 *     DDGEMM_EWORKSPACE for a missing, misaligned or small buffer;
 *     DDGEMM_ECUDA if a stream, event, copy or launch call fails (work
 *     enqueued before the failure may still be running: synchronise the
 *     device before reusing the buffer or the host arrays).
 *   - Not for stream capture (it records and waits on events of its own
 *     streams and may create a set of them). */
int ddgemm_host(int m, int n, int k,
                const double *A_hi, const double *A_lo, int lda,
                const double *B_hi, const double *B_lo, int ldb,
                double *C_hi, double *C_lo, int ldc,
                void *buffer, size_t buffer_bytes, void *stream,
                const ddgemm_opts *opts);

/* Size of the static device scratch array that ddgemm_noalloc() uses. */
#define DDGEMM_NOALLOC_SCRATCH_BYTES (64u << 20) /* 64 MiB */

/* ddgemm() for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a packaging of ddgemm(), not part of the method.
 *
 * Who needs it: code that runs while a stream is being captured into a CUDA
 * graph (allocation is not allowed there), plug-ins inside a framework whose
 * memory pool owns the GPU, latency-bound paths that cannot afford
 * cudaMalloc's implicit device synchronisation, and callers from other
 * languages with no GPU allocator.  They pass inputs and outputs only; the
 * scratch space is a file-scope __device__ array of
 * DDGEMM_NOALLOC_SCRATCH_BYTES that every GPU loading this library keeps
 * until the process exits.
 *
 *   - Arguments, layouts and results are those of ddgemm() (opts may be
 *     NULL); the work is enqueued on `stream` and the call does not wait.
 *   - Problems whose workspace without the split-k partial sums (see
 *     ddgemm_workspace_size) is above DDGEMM_NOALLOC_SCRATCH_BYTES are
 *     rejected with DDGEMM_EWORKSPACE (872 x 872 x 872 is the largest cube
 *     that fits); the rest of the array is used for split-k when it fits.
 *   - The first call on each device looks up the array's device address
 *     with cudaGetSymbolAddress (with that device current) and caches it;
 *     make that first call before any stream capture.
 *   - It calls no cudaMalloc, cudaFree or other allocating routine.
 *   - Every call on a device shares the one array, which keeps the last
 *     call's contents (nothing in it needs clearing between calls): calls
 *     whose work overlaps on the GPU (different streams, no ordering) race
 *     and give wrong results.  Serialise them, e.g. on one stream.
 *   - C is undefined when the status word reports DDGEMM_DEV_TIMEOUT; a
 *     split-k group whose wait gave up writes NaN into its partial tile, so
 *     an earlier call's partial sums left in the array never reach C. */
int ddgemm_noalloc(int m, int n, int k,
                   const double *A_hi, const double *A_lo, int lda,
                   const double *B_hi, const double *B_lo, int ldb,
                   double *C_hi, double *C_lo, int ldc,
                   void *stream, const ddgemm_opts *opts);

/* The split step alone for A (Appendix A; Sec. "Cascading matrices and
 * GEMM"): per row i and k-block p, sigma = 2^e with e the frexp exponent of
 * max |A_hi| over the block (e = 0 for an all-zero block); every entry is
 * scaled by 2^-e and cascaded into four pieces.  The pieces hold c0, c1, c2
 * digits from the paper's digit budget for the block's length L (ceil of
 * log2): 2 c0 + L <= 53, c0 + c1 + L + 1 <= 53, 2 c1 + L + 2 <= 53,
 * c0 + c2 + L + 2 <= 53, i.e. (22, 21, 21) for a full block of 256 entries
 * and wider for a shorter last block or small k (the paper widens them too).
 *   slices  device, 4 x m x ld_slices doubles: slices[(s*m + i)*ld_slices + l]
 *           = sigma_s * A_s(i, l) with sigma_0 = 1, sigma_1 = 2^-c0,
 *           sigma_2 = 2^-(c0+c1), sigma_3 = 2^-(c0+c1+c2) (2^-22, 2^-43,
 *           2^-64 for a full block): the left factor of eq. Gemm10.
 *           ld_slices >= k.  Columns l >= k are not written.
 *   exps    device int32, ceil(k/256) x m: exps[p*m + i] = e.
 * trans_a as in ddgemm_opts.  status_dev optional (DDGEMM_DEV_NONFINITE). */
int ddgemm_split_a(int m, int k, const double *A_hi, const double *A_lo, int lda,
                   int trans_a, double *slices, int ld_slices, int *exps,
                   unsigned int *status_dev, void *stream);

/* The split step alone for B: per k-block p and column j, tau = 2^e as
 * above; seven panels [B0 | s1 B1 | s2 B2 | s3 B3 || s2 B4 | s1 B5 | B6]
 * (the right factor of eq. Gemm10), where B4, B5, B6 are the FP64 roundings
 * of the exact tails B2 + B3 s3/s2, B1 + B2 s2/s1 + B3 s3/s1 and
 * B0 + s1 B1 + s2 B2 + s3 B3.
 *   slices  device, 7 x k x ld_slices doubles: slices[(s*k + l)*ld_slices + j].
 *           ld_slices >= n.  Columns j >= n are not written.
 *   exps    device int32, ceil(k/256) x n: exps[p*n + j] = e. */
int ddgemm_split_b(int k, int n, const double *B_hi, const double *B_lo, int ldb,
                   int trans_b, double *slices, int ld_slices, int *exps,
                   unsigned int *status_dev, void *stream);

/* The split step of the INT8 form alone (Sec. "FP64x2 in terms of INT8";
 * see ddgemm_opts.variant).
 *   slices      s, as for ddgemm_opts.int8_slices (no 0 default here).
 *   digits      device int8, s x m x ld_digits for A (row i of A is row i of
 *               each plane) and s x n x ld_digits for B (column j of B is row
 *               j of each plane): digits[(d*nvec + v)*ld_digits + l] is digit
 *               d (most significant first) of entry l of vector v.
 *               ld_digits >= k and a multiple of 16; the bytes of the last
 *               8-byte group past k in a row are written with zero digits.
 *               Digits are in [-128, 127].
 *   exps        device int32, ceil(k/8192) x m (or x n): e of sigma = 2^e. */
int ddgemm_split_int8_a(int m, int k, const double *A_hi, const double *A_lo, int lda,
                        int trans_a, int slices, signed char *digits, int ld_digits,
                        int *exps, unsigned int *status_dev, void *stream);
int ddgemm_split_int8_b(int k, int n, const double *B_hi, const double *B_lo, int ldb,
                        int trans_b, int slices, signed char *digits, int ld_digits,
                        int *exps, unsigned int *status_dev, void *stream);

/* The assembly step of DDGEMM_VARIANT_INT8_TC alone (the diagonal sums
 * added "in FP64x2", Sec. "FP64x2 in terms of INT8", read as one exact sum
 * rounded once), on the device: for
 * i < count, (hi[i], lo[i]) = the FP64x2 nearest to
 *     x_i = sum_{t < slices} diag[t*count + i] 2^(-12-7t) 2^scale[i]
 * (hi = RN(x_i), lo = RN(x_i - hi), round to nearest, ties to even), x_i
 * formed exactly (the form's seven-bit pieces).  diag: device int32 (any
 * value; a k-block's diagonal sums stay within 2^30); scale: device int32;
 * hi, lo: device doubles.  Results in the subnormal range are rounded twice
 * (outside the method's range).  slices in {12, ..., 16}. */
int ddgemm_assemble_int8(int count, int slices, const int *diag, const int *scale, double *hi,
                         double *lo, void *stream);

/* The ten products of one k-block without the FP64x2 assembly (for
 * checking that bins 0-2 are exact, Sec. "Cascading vectors and dot
 * products").  Requires 0 < k <= 256.  bins: device, 4 x m x n doubles,
 * bins[(b*m + i)*n + j] for b = bin 0, bin 1, bin 2, bin 3-6, each in the
 * scaled units of eq. Gemm10 (sigma tau not applied).  Other arguments as
 * for ddgemm. */
int ddgemm_bins(int m, int n, int k,
                const double *A_hi, const double *A_lo, int lda,
                const double *B_hi, const double *B_lo, int ldb,
                double *bins, void *workspace, size_t ws_bytes, void *stream,
                const ddgemm_opts *opts);

/* Static text for a return code. */
const char *ddgemm_status_string(int code);

#ifdef __cplusplus
}
#endif

#endif /* DDGEMM_H */
