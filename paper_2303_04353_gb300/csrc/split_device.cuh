// Device side of phase one of the FP64 form (Appendix A), shared by the
// single-problem split kernels (split.cu) and the batched ones (batched.cu).
#pragma once
#include <cuda_runtime.h>
#include <cmath>
#include <cstdint>

#include "dd_device.cuh"
#include "ddgemm_internal.h"

namespace ddg {
namespace split_detail {

constexpr unsigned DEV_NONFINITE = 0x1u;

// Appendix A round-to-d-digits constants 2^(53-d) + 2^(52-d).
__device__ __forceinline__ double round_c0(double x) {
    const double m = 3221225472.0;            // 2^31 + 2^30
    return __dsub_rn(__dadd_rn(x, m), m);
}
__device__ __forceinline__ double round_c12(double x) {
    const double m = 6442450944.0;            // 2^32 + 2^31
    return __dsub_rn(__dadd_rn(x, m), m);
}

struct Pieces {
    double x0, x1, x2, x3;  // the four splits
    double r0, r1, r2;      // running values before each rounding stage
};

// Appendix A for one FP64 value already scaled by 2^-e.
__device__ __forceinline__ Pieces split_fp64(double x) {
    Pieces q;
    q.r0 = x;
    q.x0 = round_c0(q.r0);
    q.r1 = __dmul_rn(__dsub_rn(q.r0, q.x0), 4194304.0);    // 2^22
    q.x1 = round_c12(q.r1);
    q.r2 = __dmul_rn(__dsub_rn(q.r1, q.x1), 2097152.0);    // 2^21
    q.x2 = round_c12(q.r2);
    q.x3 = __dmul_rn(__dsub_rn(q.r2, q.x2), 2097152.0);    // 2^21
    return q;
}

// Cascade one FP64x2 entry with block exponent e into NS outputs.
template <int NS>
__device__ __forceinline__ void cascade_entry(double hi, double lo, int e, double (&o)[NS]) {
    const Pieces h = split_fp64(scalbn(hi, -e));
    const Pieces l = split_fp64(scalbn(lo, -e));
    o[0] = __dadd_rn(h.x0, l.x0);
    o[1] = __dmul_rn(__dadd_rn(h.x1, l.x1), 0x1p-22);
    o[2] = __dmul_rn(__dadd_rn(h.x2, l.x2), 0x1p-43);
    o[3] = __dmul_rn(__dadd_rn(h.x3, l.x3), 0x1p-64);
    if constexpr (NS == 7) {
        o[4] = __dmul_rn(__dadd_rn(h.r2, l.r2), 0x1p-43);  // s2 B4
        o[5] = __dmul_rn(__dadd_rn(h.r1, l.r1), 0x1p-22);  // s1 B5
        o[6] = __dadd_rn(h.r0, l.r0);                      // B6
    }
}

__device__ __forceinline__ int block_exponent(double mx) {
    int e = 0;
    if (mx > 0.0 && isfinite(mx)) frexp(mx, &e);
    return e;
}

template <int NS>
__device__ __forceinline__ void store_entry(double *out, long long ld_out, PanelLayout layout,
                                            int nvec, int kdim, int v, int l,
                                            const double (&o)[NS]) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const long long idx = layout == PanelLayout::VEC_MAJOR
                                  ? ((long long)s * nvec + v) * ld_out + l
                                  : ((long long)s * kdim + l) * ld_out + v;
        out[idx] = o[s];
    }
}

// Vectors run along memory (A not transposed, B transposed): one warp per
// (vector, k-block); lanes read 16-byte pairs, 512 contiguous bytes per warp
// instruction.
template <int NS, bool VEC>
__device__ __forceinline__ void split_contig_unit(int lane, int v, int p, int nvec, int kdim,
                                                  const double *__restrict__ xh,
                                                  const double *__restrict__ xl, long long ldx,
                                                  double *__restrict__ out, long long ld_out,
                                                  PanelLayout layout, int *__restrict__ exps,
                                                  unsigned int *status) {
    const double *rh = xh + (long long)v * ldx;
    const double *rl = xl + (long long)v * ldx;
    double h[8], lo[8];
    double mx = 0.0;
    bool bad = false;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int l = p * KC + 64 * t + 2 * lane;
        if (VEC && l + 1 < kdim) {
            const double2 a = *reinterpret_cast<const double2 *>(rh + l);
            const double2 b = *reinterpret_cast<const double2 *>(rl + l);
            h[2 * t] = a.x; h[2 * t + 1] = a.y; lo[2 * t] = b.x; lo[2 * t + 1] = b.y;
        } else {
            h[2 * t] = l < kdim ? rh[l] : 0.0;
            lo[2 * t] = l < kdim ? rl[l] : 0.0;
            h[2 * t + 1] = l + 1 < kdim ? rh[l + 1] : 0.0;
            lo[2 * t + 1] = l + 1 < kdim ? rl[l + 1] : 0.0;
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            mx = fmax(mx, fabs(h[2 * t + c]));
            bad |= !isfinite(h[2 * t + c]) || !isfinite(lo[2 * t + c]);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    const int e = block_exponent(mx);
    if (lane == 0) exps[(long long)p * nvec + v] = e;
    if (bad && status) atomicOr(status, DEV_NONFINITE);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int l = p * KC + 64 * t + 2 * lane + c;
            if (l < kdim) {
                double o[NS];
                cascade_entry<NS>(h[2 * t + c], lo[2 * t + c], e, o);
                store_entry<NS>(out, ld_out, layout, nvec, kdim, v, l, o);
            }
        }
    }
}

// Vectors are strided in memory (B not transposed, A transposed): one CTA
// per (k-block, 64 vectors); a warp reads 64 consecutive vectors of one row
// with 16-byte pairs.  Block maxima are combined in shared memory.
// One CTA of 256 threads: vectors vt*64 .. vt*64+63, k-block p.  Uses the
// caller's shared arrays; ends with the CTA synchronised.
template <int NS, bool VEC>
__device__ __forceinline__ void split_strided_unit(int vt, int p, int nvec, int kdim,
                                                   const double *__restrict__ xh,
                                                   const double *__restrict__ xl, long long ldx,
                                                   double *__restrict__ out, long long ld_out,
                                                   PanelLayout layout, int *__restrict__ exps,
                                                   unsigned int *status, double (&part)[8][64],
                                                   int (&sexp)[64]) {
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int v = vt * 64 + 2 * tx;
    const int lbeg = p * KC, lend = min(lbeg + KC, kdim);
    auto load_pair = [&](const double *x, int l, double &a, double &b) {
        const double *row = x + (long long)l * ldx;
        if (VEC && v + 1 < nvec) {
            const double2 q = *reinterpret_cast<const double2 *>(row + v);
            a = q.x; b = q.y;
        } else {
            a = v < nvec ? row[v] : 0.0;
            b = v + 1 < nvec ? row[v + 1] : 0.0;
        }
    };
    double m0 = 0.0, m1 = 0.0;
    for (int l = lbeg + ty; l < lend; l += 8) {
        double a, b;
        load_pair(xh, l, a, b);
        m0 = fmax(m0, fabs(a));
        m1 = fmax(m1, fabs(b));
    }
    part[ty][2 * tx] = m0;
    part[ty][2 * tx + 1] = m1;
    __syncthreads();
    if (ty == 0) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            double mx = 0.0;
#pragma unroll
            for (int r = 0; r < 8; ++r) mx = fmax(mx, part[r][2 * tx + c]);
            const int e = block_exponent(mx);
            sexp[2 * tx + c] = e;
            if (v + c < nvec) exps[(long long)p * nvec + v + c] = e;
        }
    }
    __syncthreads();
    const int e0 = sexp[2 * tx], e1 = sexp[2 * tx + 1];
    bool bad = false;
    for (int l = lbeg + ty; l < lend; l += 8) {
        double ha, hb, la, lb;
        load_pair(xh, l, ha, hb);
        load_pair(xl, l, la, lb);
        bad |= !isfinite(ha) || !isfinite(la) || !isfinite(hb) || !isfinite(lb);
        double o[NS];
        if (v < nvec) {
            cascade_entry<NS>(ha, la, e0, o);
            store_entry<NS>(out, ld_out, layout, nvec, kdim, v, l, o);
        }
        if (v + 1 < nvec) {
            cascade_entry<NS>(hb, lb, e1, o);
            store_entry<NS>(out, ld_out, layout, nvec, kdim, v + 1, l, o);
        }
    }
    if (bad && status) atomicOr(status, DEV_NONFINITE);
    __syncthreads();  // the caller may reuse part/sexp for the next unit
}

}  // namespace split_detail
}  // namespace ddg
