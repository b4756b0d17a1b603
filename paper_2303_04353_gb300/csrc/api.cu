// The C ABI of libddgemm (declared in include/ddgemm.h): argument checks,
// workspace carving and the launches of the split and cascade kernels.
// Nothing here allocates device memory.
#include <cuda_runtime.h>
#include <algorithm>
#include <cstddef>
#include <cstdint>

#include "../../include/ddgemm.h"
#include "ddgemm_internal.h"

namespace {

constexpr size_t ALIGN = 256;

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Split-k groups the workspace has room for: one k-block each at least, at
// most 16, and when chosen automatically only for grids below 4096 tiles of
// 64 x 64 (bigger grids fill the GPU in many waves) and at most
// ceil(8192 / tiles), which bounds the partial sums at (8192 + tiles) tiles'
// worth of FP64x2 C, about 0.5 GB.  split_k = 1 in the options reserves none.
constexpr int SPLIT_MAX = 16;
constexpr long long SPLIT_TILE_LIMIT = 4096;

long long fp64_tiles(int m, int n) { return (long long)((m + 63) / 64) * ((n + 63) / 64); }

int auto_split_cap(int m, int n, int k) {
    const long long tiles = fp64_tiles(m, n);
    const int kb = (k + ddg::KC - 1) / ddg::KC;
    if (tiles <= 0 || tiles >= SPLIT_TILE_LIMIT) return 1;
    const long long by_tiles = (2 * SPLIT_TILE_LIMIT + tiles - 1) / tiles;
    return (int)std::min<long long>(std::min<long long>(SPLIT_MAX, kb), by_tiles);
}

int split_reserve(int m, int n, int k, int split_k) {
    const int kb = (k + ddg::KC - 1) / ddg::KC;
    if (split_k == 1) return 1;
    if (split_k > 1) return std::min(std::min(split_k, SPLIT_MAX), kb);
    return auto_split_cap(m, n, k);
}

// Workspace carve: A pieces, B panels, exponents of A, exponents of B, then
// room for the partial C of split-k groups 1..reserve-1.
struct Layout {
    long long lda_s, ldb_s;
    size_t off_a, off_b, off_ea, off_eb, base, off_part, part_bytes, total;
};

Layout layout_for(int m, int n, int k, int split_reserve_groups = 1) {
    Layout L;
    const long long kb = (k + ddg::KC - 1) / ddg::KC;
    L.lda_s = (long long)round_up((size_t)k, 8);
    L.ldb_s = (long long)round_up((size_t)n, 8);
    L.off_a = 0;
    L.off_b = L.off_a + round_up((size_t)4 * m * L.lda_s * sizeof(double), ALIGN);
    L.off_ea = L.off_b + round_up((size_t)7 * k * L.ldb_s * sizeof(double), ALIGN);
    L.off_eb = L.off_ea + round_up((size_t)kb * m * sizeof(int), ALIGN);
    L.base = L.off_eb + round_up((size_t)kb * n * sizeof(int), ALIGN);
    L.off_part = L.base;
    L.part_bytes = round_up((size_t)m * n * sizeof(double), ALIGN);   // one hi or lo plane
    L.total = L.base + (size_t)(split_reserve_groups - 1) * 2 * L.part_bytes;
    return L;
}

struct Parsed {
    int trans_a = 0, trans_b = 0, variant = DDGEMM_VARIANT_FP64;
    unsigned int *status = nullptr;
    int *flags = nullptr;
    void **events = nullptr;
    int slices = 0;  // 0: the form's default
    int split_k = 0;
};

bool is_int8(int variant) {
    return variant == DDGEMM_VARIANT_INT8 || variant == DDGEMM_VARIANT_INT8_TC;
}

// Workspace carve of the INT8 forms: digit planes of A and B (int8, or bf16
// for the tensor-core form), exponents.
struct Layout8 {
    long long ld;
    size_t off_a, off_b, off_ea, off_eb, total;
};

Layout8 layout8_for(int m, int n, int k, int slices, int variant) {
    Layout8 L;
    const int blk = variant == DDGEMM_VARIANT_INT8_TC ? ddg::KB8_TC : ddg::KB8;
    const long long kb = (k + blk - 1) / blk;
    L.ld = (long long)round_up((size_t)k, 64);
    L.off_a = 0;
    if (variant == DDGEMM_VARIANT_INT8_TC) {
        // bf16 digits in whole tiles of 128 rows (A) and 16 columns (B) by
        // k-steps of 16
        const size_t kpad = round_up((size_t)k, 16);
        L.off_b = round_up((size_t)slices * round_up((size_t)m, ddg::INT8_TC_BM) * kpad * 2, ALIGN);
        L.off_ea = L.off_b +
                   round_up((size_t)slices * round_up((size_t)n, ddg::INT8_TC_BN) * kpad * 2, ALIGN);
    } else {
        L.off_b = round_up((size_t)slices * m * L.ld, ALIGN);
        L.off_ea = L.off_b + round_up((size_t)slices * n * L.ld, ALIGN);
    }
    L.off_eb = L.off_ea + round_up((size_t)kb * m * sizeof(int), ALIGN);
    L.total = L.off_eb + round_up((size_t)kb * n * sizeof(int), ALIGN);
    return L;
}

bool parse(const ddgemm_opts *o, Parsed &p) {
    if (o) {
        p.trans_a = o->trans_a;
        p.trans_b = o->trans_b;
        p.variant = o->variant;
        p.status = o->status_dev;
        p.flags = o->flags_dev;
        p.events = o->phase_events;
        if (o->int8_slices) p.slices = o->int8_slices;
        p.split_k = o->split_k;
    }
    if (p.split_k < 0) return false;
    if (p.slices == 0)
        p.slices = p.variant == DDGEMM_VARIANT_INT8_TC ? ddg::INT8_TC_SLICES_DEFAULT
                                                       : ddg::INT8_SLICES_DEFAULT;
    if (p.variant == DDGEMM_VARIANT_INT8 && !ddg::int8_slices_supported(p.slices)) return false;
    if (p.variant == DDGEMM_VARIANT_INT8_TC && !ddg::int8_tc_slices_supported(p.slices))
        return false;
    return (p.trans_a == 0 || p.trans_a == 1) && (p.trans_b == 0 || p.trans_b == 1);
}

bool dims_ok(int m, int n, int k) {
    if (m < 0 || n < 0 || k < 0) return false;
    // tensor-map extents and grid limits
    return (long long)m <= (1LL << 31) - 1 && (long long)n <= (1LL << 31) - 1;
}

int check_operands(int m, int n, int k, const void *ah, const void *al, int lda, const void *bh,
                   const void *bl, int ldb, const Parsed &p) {
    if (m > 0 && k > 0) {
        if (!ah || !al) return DDGEMM_EINVAL;
        if (lda < (p.trans_a ? m : k)) return DDGEMM_EINVAL;
    }
    if (n > 0 && k > 0) {
        if (!bh || !bl) return DDGEMM_EINVAL;
        if (ldb < (p.trans_b ? k : n)) return DDGEMM_EINVAL;
    }
    return DDGEMM_OK;
}

// split-k groups of an FP64-form launch: as many as the workspace holds,
// within the choice for this grid
int split_groups(int m, int n, int k, int sms, size_t ws_bytes, const Parsed &p) {
    if (is_int8(p.variant) || p.flags || p.split_k == 1) return 1;
    if (m <= 0 || n <= 0 || k <= 0) return 1;
    const Layout L = layout_for(m, n, k);
    if (ws_bytes < L.base) return 1;
    const int kb = (k + ddg::KC - 1) / ddg::KC;
    const int room = 1 + (int)std::min<size_t>((ws_bytes - L.base) / (2 * L.part_bytes),
                                                SPLIT_MAX - 1);
    int split = 1;
    if (p.split_k > 1)
        split = std::min(std::min(p.split_k, SPLIT_MAX), kb);
    else
        split = ddg::choose_split(fp64_tiles(m, n), kb, sms, auto_split_cap(m, n, k));
    return std::min(split, room);
}

int run(int m, int n, int k, const double *A_hi, const double *A_lo, int lda,
        const double *B_hi, const double *B_lo, int ldb, double *C_hi, double *C_lo, int ldc,
        double *bins, void *workspace, size_t ws_bytes, cudaStream_t stream, const Parsed &p) {
    const Layout L = layout_for(m, n, k);
    if (!workspace || ws_bytes < L.base || (uintptr_t)workspace % ALIGN) return DDGEMM_EWORKSPACE;
    int split = 1;
    if (!bins && !p.flags && p.split_k != 1) {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return DDGEMM_ECUDA;
        split = split_groups(m, n, k, sms, ws_bytes, p);
    }
    char *ws = static_cast<char *>(workspace);
    double *a_s = reinterpret_cast<double *>(ws + L.off_a);
    double *b_s = reinterpret_cast<double *>(ws + L.off_b);
    int *e_a = reinterpret_cast<int *>(ws + L.off_ea);
    int *e_b = reinterpret_cast<int *>(ws + L.off_eb);
    auto mark = [&](int i) {
        return !p.events || cudaEventRecord(static_cast<cudaEvent_t>(p.events[i]), stream) ==
                                cudaSuccess;
    };
    if (!mark(0)) return DDGEMM_ECUDA;
    // A: a row of op(A) is a vector; it runs along memory unless trans_a.
    cudaError_t e = ddg::launch_split(4, m, k, A_hi, A_lo, lda, !p.trans_a, a_s, L.lda_s,
                                      ddg::PanelLayout::VEC_MAJOR, e_a, p.status, stream);
    if (e != cudaSuccess) return DDGEMM_ECUDA;
    // B: a column of op(B) is a vector; it runs along memory only if trans_b.
    e = ddg::launch_split(7, n, k, B_hi, B_lo, ldb, p.trans_b != 0, b_s, L.ldb_s,
                          ddg::PanelLayout::K_MAJOR, e_b, p.status, stream);
    if (e != cudaSuccess || !mark(1)) return DDGEMM_ECUDA;
    const int products = p.variant == DDGEMM_VARIANT_FP64_GEMM16    ? 1
                         : p.variant == DDGEMM_VARIANT_FP64_DROP456 ? 2
                                                                      : 0;
    double *part = reinterpret_cast<double *>(ws + L.off_part);
    double *part_lo = reinterpret_cast<double *>(ws + L.off_part + (size_t)(split - 1) * L.part_bytes);
    ddg::CascadeArgs ca{m, n, k, a_s, L.lda_s, b_s, L.ldb_s, e_a, e_b, C_hi, C_lo,
                        (long long)ldc, p.flags, p.status, bins, products, split, part, part_lo};
    e = ddg::launch_cascade_fp64(ca, stream);
    return e == cudaSuccess && mark(2) ? DDGEMM_OK : DDGEMM_ECUDA;
}

int run_int8(int m, int n, int k, const double *A_hi, const double *A_lo, int lda,
             const double *B_hi, const double *B_lo, int ldb, double *C_hi, double *C_lo, int ldc,
             void *workspace, size_t ws_bytes, cudaStream_t stream, const Parsed &p) {
    const bool tc = p.variant == DDGEMM_VARIANT_INT8_TC;
    const Layout8 L = layout8_for(m, n, k, p.slices, p.variant);
    if (!workspace || ws_bytes < L.total || (uintptr_t)workspace % ALIGN) return DDGEMM_EWORKSPACE;
    char *ws = static_cast<char *>(workspace);
    void *da = ws + L.off_a;
    void *db = ws + L.off_b;
    int *e_a = reinterpret_cast<int *>(ws + L.off_ea);
    int *e_b = reinterpret_cast<int *>(ws + L.off_eb);
    auto mark = [&](int i) {
        return !p.events || cudaEventRecord(static_cast<cudaEvent_t>(p.events[i]), stream) ==
                                cudaSuccess;
    };
    if (!mark(0)) return DDGEMM_ECUDA;
    cudaError_t e = ddg::launch_split_int8(p.slices, m, k, A_hi, A_lo, lda, !p.trans_a, da,
                                           tc ? ddg::INT8_TC_BM : 0, L.ld, e_a, p.status, stream);
    if (e != cudaSuccess) return DDGEMM_ECUDA;
    e = ddg::launch_split_int8(p.slices, n, k, B_hi, B_lo, ldb, p.trans_b != 0, db,
                               tc ? ddg::INT8_TC_BN : 0, L.ld, e_b, p.status, stream);
    if (e != cudaSuccess || !mark(1)) return DDGEMM_ECUDA;
    if (tc) {
        ddg::Int8TcArgs a{m, n, k, p.slices, static_cast<const uint16_t *>(da),
                          static_cast<const uint16_t *>(db), e_a, e_b, C_hi, C_lo,
                          (long long)ldc, p.status};
        e = ddg::launch_cascade_int8_tc(a, stream);
    } else {
        ddg::Int8Args a{m, n, k, p.slices, static_cast<const int8_t *>(da),
                        static_cast<const int8_t *>(db), L.ld, e_a, e_b, C_hi, C_lo,
                        (long long)ldc, p.status};
        e = ddg::launch_cascade_int8(a, stream);
    }
    return e == cudaSuccess && mark(2) ? DDGEMM_OK : DDGEMM_ECUDA;
}

}  // namespace

namespace ddg {

size_t base_workspace_size(int m, int n, int k, const ddgemm_opts *opts) {
    Parsed p;
    if (!parse(opts, p) || !dims_ok(m, n, k)) return 0;
    if (m == 0 || n == 0 || k == 0) return 0;
    if (is_int8(p.variant)) return layout8_for(m, n, k, p.slices, p.variant).total;
    return layout_for(m, n, k).base;
}

}  // namespace ddg

extern "C" {

size_t ddgemm_workspace_size(int m, int n, int k, const ddgemm_opts *opts) {
    Parsed p;
    if (!parse(opts, p) || !dims_ok(m, n, k)) return 0;
    if (m == 0 || n == 0 || k == 0) return 0;
    if (is_int8(p.variant)) return layout8_for(m, n, k, p.slices, p.variant).total;
    return layout_for(m, n, k, split_reserve(m, n, k, p.split_k)).total;
}

int ddgemm_split_groups(int m, int n, int k, int sms, size_t ws_bytes, const ddgemm_opts *opts) {
    Parsed p;
    if (!parse(opts, p) || !dims_ok(m, n, k) || sms <= 0) return 0;
    return split_groups(m, n, k, sms, ws_bytes, p);
}

int ddgemm(int m, int n, int k, const double *A_hi, const double *A_lo, int lda,
           const double *B_hi, const double *B_lo, int ldb, double *C_hi, double *C_lo, int ldc,
           void *workspace, size_t ws_bytes, void *stream, const ddgemm_opts *opts) {
    Parsed p;
    if (!parse(opts, p) || !dims_ok(m, n, k)) return DDGEMM_EINVAL;
    if (p.variant < DDGEMM_VARIANT_FP64 || p.variant > DDGEMM_VARIANT_INT8_TC)
        return DDGEMM_EUNSUPPORTED;
    if (is_int8(p.variant) && p.flags) return DDGEMM_EUNSUPPORTED;
    if (int r = check_operands(m, n, k, A_hi, A_lo, lda, B_hi, B_lo, ldb, p)) return r;
    if (m == 0 || n == 0) return DDGEMM_OK;
    if (!C_hi || !C_lo || ldc < n) return DDGEMM_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (k == 0) {
        // C := A B with k = 0 is the zero matrix
        if (cudaMemset2DAsync(C_hi, (size_t)ldc * 8, 0, (size_t)n * 8, m, s) != cudaSuccess ||
            cudaMemset2DAsync(C_lo, (size_t)ldc * 8, 0, (size_t)n * 8, m, s) != cudaSuccess ||
            (p.flags && cudaMemsetAsync(p.flags, 0, (size_t)m * n * sizeof(int), s) != cudaSuccess))
            return DDGEMM_ECUDA;
        return DDGEMM_OK;
    }
    if (is_int8(p.variant))
        return run_int8(m, n, k, A_hi, A_lo, lda, B_hi, B_lo, ldb, C_hi, C_lo, ldc, workspace,
                        ws_bytes, s, p);
    return run(m, n, k, A_hi, A_lo, lda, B_hi, B_lo, ldb, C_hi, C_lo, ldc, nullptr, workspace,
               ws_bytes, s, p);
}

int ddgemm_split_int8_a(int m, int k, const double *A_hi, const double *A_lo, int lda,
                        int trans_a, int slices, signed char *digits, int ld_digits, int *exps,
                        unsigned int *status_dev, void *stream) {
    if (m < 0 || k < 0 || (trans_a != 0 && trans_a != 1) || !ddg::int8_slices_supported(slices))
        return DDGEMM_EINVAL;
    if (m == 0 || k == 0) return DDGEMM_OK;
    if (!A_hi || !A_lo || !digits || !exps || lda < (trans_a ? m : k) || ld_digits < k ||
        ld_digits % 16)
        return DDGEMM_EINVAL;
    const cudaError_t e = ddg::launch_split_int8(slices, m, k, A_hi, A_lo, lda, !trans_a, digits,
                                                 0, ld_digits, exps, status_dev,
                                                 static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? DDGEMM_OK : DDGEMM_ECUDA;
}

int ddgemm_split_int8_b(int k, int n, const double *B_hi, const double *B_lo, int ldb,
                        int trans_b, int slices, signed char *digits, int ld_digits, int *exps,
                        unsigned int *status_dev, void *stream) {
    if (n < 0 || k < 0 || (trans_b != 0 && trans_b != 1) || !ddg::int8_slices_supported(slices))
        return DDGEMM_EINVAL;
    if (n == 0 || k == 0) return DDGEMM_OK;
    if (!B_hi || !B_lo || !digits || !exps || ldb < (trans_b ? k : n) || ld_digits < k ||
        ld_digits % 16)
        return DDGEMM_EINVAL;
    const cudaError_t e = ddg::launch_split_int8(slices, n, k, B_hi, B_lo, ldb, trans_b != 0,
                                                 digits, 0, ld_digits, exps, status_dev,
                                                 static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? DDGEMM_OK : DDGEMM_ECUDA;
}

int ddgemm_bins(int m, int n, int k, const double *A_hi, const double *A_lo, int lda,
                const double *B_hi, const double *B_lo, int ldb, double *bins, void *workspace,
                size_t ws_bytes, void *stream, const ddgemm_opts *opts) {
    Parsed p;
    if (!parse(opts, p) || !dims_ok(m, n, k)) return DDGEMM_EINVAL;
    if (k <= 0 || k > ddg::KC || m <= 0 || n <= 0 || !bins) return DDGEMM_EINVAL;
    if (p.variant != DDGEMM_VARIANT_FP64) return DDGEMM_EUNSUPPORTED;
    if (int r = check_operands(m, n, k, A_hi, A_lo, lda, B_hi, B_lo, ldb, p)) return r;
    p.flags = nullptr;
    return run(m, n, k, A_hi, A_lo, lda, B_hi, B_lo, ldb, nullptr, nullptr, n, bins, workspace,
               ws_bytes, static_cast<cudaStream_t>(stream), p);
}

int ddgemm_split_a(int m, int k, const double *A_hi, const double *A_lo, int lda, int trans_a,
                   double *slices, int ld_slices, int *exps, unsigned int *status_dev,
                   void *stream) {
    if (m < 0 || k < 0 || (trans_a != 0 && trans_a != 1)) return DDGEMM_EINVAL;
    if (m == 0 || k == 0) return DDGEMM_OK;
    if (!A_hi || !A_lo || !slices || !exps || lda < (trans_a ? m : k) || ld_slices < k)
        return DDGEMM_EINVAL;
    const cudaError_t e =
        ddg::launch_split(4, m, k, A_hi, A_lo, lda, !trans_a, slices, ld_slices,
                          ddg::PanelLayout::VEC_MAJOR, exps, status_dev,
                          static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? DDGEMM_OK : DDGEMM_ECUDA;
}

int ddgemm_split_b(int k, int n, const double *B_hi, const double *B_lo, int ldb, int trans_b,
                   double *slices, int ld_slices, int *exps, unsigned int *status_dev,
                   void *stream) {
    if (n < 0 || k < 0 || (trans_b != 0 && trans_b != 1)) return DDGEMM_EINVAL;
    if (n == 0 || k == 0) return DDGEMM_OK;
    if (!B_hi || !B_lo || !slices || !exps || ldb < (trans_b ? k : n) || ld_slices < n)
        return DDGEMM_EINVAL;
    const cudaError_t e =
        ddg::launch_split(7, n, k, B_hi, B_lo, ldb, trans_b != 0, slices, ld_slices,
                          ddg::PanelLayout::K_MAJOR, exps, status_dev,
                          static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? DDGEMM_OK : DDGEMM_ECUDA;
}

// The two products of the backward pass, each a plain ddgemm on the stream.
// With C = op(A) op(B) and dC given:
//   dA: trans_a = 0 -> dA (m x k) = dC op(B)^T;  trans_a = 1 -> dA (k x m) = op(B) dC^T
//   dB: trans_b = 0 -> dB (k x n) = op(A)^T dC;  trans_b = 1 -> dB (n x k) = dC^T op(A)
struct BwdCall {
    int m, n, k;
    const double *ah, *al;
    int lda, ta;
    const double *bh, *bl;
    int ldb, tb;
};

static void backward_calls(int m, int n, int k, const double *A_hi, const double *A_lo, int lda,
                           const double *B_hi, const double *B_lo, int ldb, const double *dC_hi,
                           const double *dC_lo, int lddc, const Parsed &p, BwdCall &ca,
                           BwdCall &cb) {
    if (!p.trans_a)
        ca = {m, k, n, dC_hi, dC_lo, lddc, 0, B_hi, B_lo, ldb, !p.trans_b};
    else
        ca = {k, m, n, B_hi, B_lo, ldb, p.trans_b, dC_hi, dC_lo, lddc, 1};
    if (!p.trans_b)
        cb = {k, n, m, A_hi, A_lo, lda, !p.trans_a, dC_hi, dC_lo, lddc, 0};
    else
        cb = {n, k, m, dC_hi, dC_lo, lddc, 1, A_hi, A_lo, lda, p.trans_a};
}

size_t ddgemm_backward_workspace_size(int m, int n, int k, const ddgemm_opts *opts) {
    Parsed p;
    if (!parse(opts, p) || !dims_ok(m, n, k)) return 0;
    ddgemm_opts plain{0, 0, p.variant, nullptr, nullptr, nullptr, p.slices, p.split_k};
    const size_t a = ddgemm_workspace_size(p.trans_a ? k : m, p.trans_a ? m : k, n, &plain);
    const size_t b = ddgemm_workspace_size(p.trans_b ? n : k, p.trans_b ? k : n, m, &plain);
    return a > b ? a : b;
}

int ddgemm_backward(int m, int n, int k, const double *A_hi, const double *A_lo, int lda,
                    const double *B_hi, const double *B_lo, int ldb, const double *dC_hi,
                    const double *dC_lo, int lddc, double *dA_hi, double *dA_lo, int ldda,
                    double *dB_hi, double *dB_lo, int lddb, void *workspace, size_t ws_bytes,
                    void *stream, const ddgemm_opts *opts) {
    Parsed p;
    if (!parse(opts, p) || !dims_ok(m, n, k)) return DDGEMM_EINVAL;
    if (p.variant != DDGEMM_VARIANT_FP64 && !is_int8(p.variant))
        return DDGEMM_EUNSUPPORTED;
    if (int r = check_operands(m, n, k, A_hi, A_lo, lda, B_hi, B_lo, ldb, p)) return r;
    if (m > 0 && n > 0 && (!dC_hi || !dC_lo || lddc < n)) return DDGEMM_EINVAL;
    BwdCall ca, cb;
    backward_calls(m, n, k, A_hi, A_lo, lda, B_hi, B_lo, ldb, dC_hi, dC_lo, lddc, p, ca, cb);
    if (ca.m > 0 && ca.n > 0 && (!dA_hi || !dA_lo || ldda < ca.n)) return DDGEMM_EINVAL;
    if (cb.m > 0 && cb.n > 0 && (!dB_hi || !dB_lo || lddb < cb.n)) return DDGEMM_EINVAL;
    if (ws_bytes < ddgemm_backward_workspace_size(m, n, k, opts)) return DDGEMM_EWORKSPACE;
    ddgemm_opts oa{ca.ta, ca.tb, p.variant, p.status, nullptr, nullptr, p.slices, p.split_k};
    ddgemm_opts ob{cb.ta, cb.tb, p.variant, p.status, nullptr, nullptr, p.slices, p.split_k};
    // both products run on one stream, so the second may reuse the workspace
    int r = ddgemm(ca.m, ca.n, ca.k, ca.ah, ca.al, ca.lda, ca.bh, ca.bl, ca.ldb, dA_hi, dA_lo,
                   ldda, workspace, ws_bytes, stream, &oa);
    if (r != DDGEMM_OK) return r;
    return ddgemm(cb.m, cb.n, cb.k, cb.ah, cb.al, cb.lda, cb.bh, cb.bl, cb.ldb, dB_hi, dB_lo, lddb,
                  workspace, ws_bytes, stream, &ob);
}

int ddgemm_assemble_int8(int count, int slices, const int *diag, const int *scale, double *hi,
                         double *lo, void *stream) {
    if (count < 0 || !ddg::int8_tc_slices_supported(slices)) return DDGEMM_EINVAL;
    if (count == 0) return DDGEMM_OK;
    if (!diag || !scale || !hi || !lo) return DDGEMM_EINVAL;
    const cudaError_t e = ddg::launch_assemble_int8(count, slices, diag, scale, hi, lo,
                                                    static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? DDGEMM_OK : DDGEMM_ECUDA;
}

const char *ddgemm_status_string(int code) {
    switch (code) {
        case DDGEMM_OK: return "ok";
        case DDGEMM_EINVAL: return "invalid argument";
        case DDGEMM_EWORKSPACE: return "workspace missing, misaligned or too small";
        case DDGEMM_ECUDA: return "CUDA error";
        case DDGEMM_EUNSUPPORTED: return "unsupported option";
        default: return "unknown status";
    }
}

}  // extern "C"
