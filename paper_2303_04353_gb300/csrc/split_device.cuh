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

// Exact powers of two and the Appendix A rounding constant
// 2^(53-c) + 2^(52-c), built from their bit patterns.
__device__ __forceinline__ double pow2(int e) {
    return __longlong_as_double((long long)(1023 + e) << 52);
}
__device__ __forceinline__ double round_const(int c) {
    return __longlong_as_double(((long long)(1023 + 53 - c) << 52) | (1ll << 51));
}

// The digit budget of a k-block of `len` entries (Sec. "Cascading vectors
// and dot products", with L = ceil(log2 len) in place of log2 k):
//   2 c0 + L <= 53;  c0 + c1 + L + 1 <= 53;  2 c1 + L + 2 <= 53;
//   c0 + c2 + L + 2 <= 53.
// (22, 21, 21) for a full block of 256; wider for shorter blocks, as the
// paper allows for smaller k.  Kept with the constants the split needs.
struct Digits {
    double m0, m1, m2;     // rounding constants for c0, c1, c2
    double up0, up1, up2;  // 2^c0, 2^c1, 2^c2
    double s1, s2, s3;     // sigma_1 = 2^-c0, sigma_2 = 2^-(c0+c1), sigma_3 = 2^-(c0+c1+c2)
};

__device__ __forceinline__ Digits block_digits(int len) {
    const int L = len > 1 ? 32 - __clz(len - 1) : 0;
    const int c0 = (53 - L) / 2;
    const int c1 = min(53 - c0 - L - 1, (53 - L - 2) / 2);
    const int c2 = 53 - c0 - L - 2;
    Digits d;
    d.m0 = round_const(c0);
    d.m1 = round_const(c1);
    d.m2 = round_const(c2);
    d.up0 = pow2(c0);
    d.up1 = pow2(c1);
    d.up2 = pow2(c2);
    d.s1 = pow2(-c0);
    d.s2 = pow2(-(c0 + c1));
    d.s3 = pow2(-(c0 + c1 + c2));
    return d;
}

// Appendix A: round to a digit grid by adding and subtracting the constant.
__device__ __forceinline__ double round_to(double x, double m) {
    return __dsub_rn(__dadd_rn(x, m), m);
}

struct Pieces {
    double x0, x1, x2, x3;  // the four splits
    double r0, r1, r2;      // running values before each rounding stage
};

// Appendix A for one FP64 value already scaled by 2^-e.
__device__ __forceinline__ Pieces split_fp64(double x, const Digits &d) {
    Pieces q;
    q.r0 = x;
    q.x0 = round_to(q.r0, d.m0);
    q.r1 = __dmul_rn(__dsub_rn(q.r0, q.x0), d.up0);
    q.x1 = round_to(q.r1, d.m1);
    q.r2 = __dmul_rn(__dsub_rn(q.r1, q.x1), d.up1);
    q.x2 = round_to(q.r2, d.m2);
    q.x3 = __dmul_rn(__dsub_rn(q.r2, q.x2), d.up2);
    return q;
}

// Cascade one FP64x2 entry with block exponent e into NS outputs.
template <int NS>
__device__ __forceinline__ void cascade_entry(double hi, double lo, int e, const Digits &d,
                                              double (&o)[NS]) {
    const Pieces h = split_fp64(scalbn(hi, -e), d);
    const Pieces l = split_fp64(scalbn(lo, -e), d);
    o[0] = __dadd_rn(h.x0, l.x0);
    o[1] = __dmul_rn(__dadd_rn(h.x1, l.x1), d.s1);
    o[2] = __dmul_rn(__dadd_rn(h.x2, l.x2), d.s2);
    o[3] = __dmul_rn(__dadd_rn(h.x3, l.x3), d.s3);
    if constexpr (NS == 7) {
        o[4] = __dmul_rn(__dadd_rn(h.r2, l.r2), d.s2);  // s2 B4
        o[5] = __dmul_rn(__dadd_rn(h.r1, l.r1), d.s1);  // s1 B5
        o[6] = __dadd_rn(h.r0, l.r0);                   // B6
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
    const Digits dg = block_digits(min(KC, kdim - p * KC));
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
                cascade_entry<NS>(h[2 * t + c], lo[2 * t + c], e, dg, o);
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
    const Digits dg = block_digits(lend - lbeg);
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
            cascade_entry<NS>(ha, la, e0, dg, o);
            store_entry<NS>(out, ld_out, layout, nvec, kdim, v, l, o);
        }
        if (v + 1 < nvec) {
            cascade_entry<NS>(hb, lb, e1, dg, o);
            store_entry<NS>(out, ld_out, layout, nvec, kdim, v + 1, l, o);
        }
    }
    if (bad && status) atomicOr(status, DEV_NONFINITE);
    __syncthreads();  // the caller may reuse part/sexp for the next unit
}

}  // namespace split_detail
}  // namespace ddg
