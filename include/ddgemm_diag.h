/*
 * ddgemm_diag.h - measurement and failure-handling aids of libddgemm.
 *
 * Nothing here is part of the cascade (the paper has no counterpart for any
 * of it): these entry points exist for the benchmark, which measures the
 * tensor-path ceilings the kernels are compared against, and for the tests
 * of the kernels' bounded waits.  They are exported by the same library as
 * include/ddgemm.h and follow its conventions (device pointers owned by the
 * caller, `stream` a cudaStream_t passed as void*, DDGEMM_* return codes).
 */
#ifndef DDGEMM_DIAG_H
#define DDGEMM_DIAG_H

#include <stddef.h>

#include "ddgemm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Enqueue a throughput kernel of the FP64 tensor path (mma.sync m8n8k4 f64,
 * 4 CTAs of 256 threads per SM, eight independent accumulator chains per
 * warp, `iters` rounds) on `stream` and return the number of FP64 flops it
 * performs (-1 on error).  The caller times it; flops / time is the
 * measured ceiling of the ten products.  sink: device pointer to one double
 * (never written in practice). */
double ddgemm_probe_fp64(int iters, double *sink, void *stream);

/* The same for the integer tensor path of the INT8 form (mma.sync m16n8k32
 * s8 with s32 accumulation, four independent chains per warp); returns the
 * number of integer operations (2 per multiply-add), or -1 on error. */
double ddgemm_probe_int8(int iters, double *sink, void *stream);

/* One thread waits, with the same bounded mbarrier wait the cascade kernels
 * use, on a barrier that nothing arrives on.  After limit_ns nanoseconds
 * (1 .. 10^10) it gives up and ORs DDGEMM_DEV_TIMEOUT into *status_dev, as
 * a cascade kernel does when a wait runs out; the context stays usable.
 * Returns DDGEMM_EINVAL for a null status or a limit out of range. */
int ddgemm_probe_wait_timeout(unsigned long long limit_ns, unsigned int *status_dev,
                              void *stream);

/* ddgemm() with one of its cascade kernel's copies withheld, to exercise
 * the kernel's own timeout path without any fault.  The copy producer of
 * CTA `cta` skips the copy of its ring iteration `step` (the k-step of the
 * tile for the FP64 and mma.sync INT8 forms; the CTA's running stage count
 * over its tiles for the tcgen05 forms); the barrier that copy would
 * complete never does, so the CTA's waits run out after limit_ns.  The CTA
 * then ORs DDGEMM_DEV_TIMEOUT into *opts->status_dev, lets its other copies
 * land (bounded), releases its tensor memory (tcgen05 forms) and returns;
 * every other CTA computes as usual.  Every wait of the launch uses limit_ns
 * in place of the default (~2 s).
 *   Arguments as for ddgemm(); opts and opts->status_dev are required.
 *   cta >= 0, step >= 0 (a CTA or step that does not exist withholds
 *   nothing), limit_ns in 10^3 .. 10^10.  flags_dev and phase_events are
 *   not used (DDGEMM_EUNSUPPORTED / ignored); split_k as for ddgemm().
 * C is undefined afterwards (the FP64 form writes NaN into the tile whose
 * wait gave up). */
int ddgemm_diag_withheld_copy(int m, int n, int k,
                              const double *A_hi, const double *A_lo, int lda,
                              const double *B_hi, const double *B_lo, int ldb,
                              double *C_hi, double *C_lo, int ldc,
                              void *workspace, size_t ws_bytes, void *stream,
                              const ddgemm_opts *opts, int cta, long long step,
                              unsigned long long limit_ns);

/* The same for the persistent tcgen05 kernel of ddgemm_batched() (variants
 * INT8_TC and INT8_TC8; the FP64 batched kernel stages its operands with
 * cp.async groups and has no barrier wait to run out: DDGEMM_EUNSUPPORTED).
 * `step` counts the CTA's stages over the planned items it takes.  Arguments
 * as for ddgemm_batched(); opts->status_dev is required. */
int ddgemm_diag_batched_withheld_copy(int count, const ddgemm_problem *probs_host,
                                      const ddgemm_problem *probs_dev, void *workspace,
                                      size_t ws_bytes, void *stream, const ddgemm_opts *opts,
                                      int cta, long long step, unsigned long long limit_ns);

#ifdef __cplusplus
}
#endif

#endif /* DDGEMM_DIAG_H */
