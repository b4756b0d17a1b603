// The C ABI of libddgemm (declared in include/ddgemm.h): argument checks,
// workspace carving and the launches of the split and cascade kernels.
// Nothing here allocates device memory.
#include <cuda_runtime.h>
#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "../../include/ddgemm.h"
#include "../../include/ddgemm_diag.h"
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
    ddg::WaitPlan wait{};  // only the diagnostic entry point changes it
};

bool is_int8(int variant) {
    return variant == DDGEMM_VARIANT_INT8 || variant == DDGEMM_VARIANT_INT8_TC ||
           variant == DDGEMM_VARIANT_INT8_TC8;
}

// The INT8 forms on the tcgen05 tensor cores, and their digit widths.
bool is_tc(int variant) {
    return variant == DDGEMM_VARIANT_INT8_TC || variant == DDGEMM_VARIANT_INT8_TC8;
}
int int8_bits(int variant) {
    return variant == DDGEMM_VARIANT_INT8_TC ? ddg::INT8_TC_BITS : ddg::INT8_BITS;
}

// Workspace carve of the INT8 forms: digit planes of A and B (int8, or bf16
// for the tensor-core form), exponents.
struct Layout8 {
    long long ld;
    size_t off_a, off_b, off_ea, off_eb, total;
};

Layout8 layout8_for(int m, int n, int k, int slices, int variant) {
    Layout8 L;
    const int blk = ddg::kblock_of_bits(int8_bits(variant));
    const long long kb = (k + blk - 1) / blk;
    L.ld = (long long)round_up((size_t)k, 64);
    L.off_a = 0;
    if (is_tc(variant)) {
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
        p.slices = p.variant == DDGEMM_VARIANT_INT8_TC    ? ddg::INT8_TC_SLICES_DEFAULT
                   : p.variant == DDGEMM_VARIANT_INT8_TC8 ? ddg::INT8_TC8_SLICES_DEFAULT
                                                          : ddg::INT8_SLICES_DEFAULT;
    if (p.variant == DDGEMM_VARIANT_INT8 && !ddg::int8_slices_supported(p.slices)) return false;
    if (p.variant == DDGEMM_VARIANT_INT8_TC && !ddg::int8_tc_slices_supported(p.slices))
        return false;
    if (p.variant == DDGEMM_VARIANT_INT8_TC8 && !ddg::int8_tc8_slices_supported(p.slices))
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

// A workspace carved for row chunks of at most mc rows of op(A) against all
// of op(B): the B regions and their offsets depend on mc, n and k only, so
// one split of B serves every chunk, and a chunk of mr <= mc rows puts its
// pieces of A, its exponents and its split-k partials in regions sized for
// mc.  ddgemm() is the single chunk mc = mr = m.
struct Carve {
    int mc = 0;
    bool int8 = false;
    Layout L{};
    Layout8 L8{};
    size_t base = 0;  // bytes without split-k partials
};

Carve carve_for(int mc, int n, int k, const Parsed &p) {
    Carve c;
    c.mc = mc;
    c.int8 = is_int8(p.variant);
    if (c.int8) {
        c.L8 = layout8_for(mc, n, k, p.slices, p.variant);
        c.base = c.L8.total;
    } else {
        c.L = layout_for(mc, n, k);
        c.base = c.L.base;
    }
    return c;
}

// split-k groups of an FP64-form launch of mr rows in a workspace carved for
// mc >= mr rows: as many as the workspace holds, within the choice for the
// grid of mr x n
int split_groups_in(int mr, int n, int k, int sms, size_t ws_bytes, const Carve &c,
                    const Parsed &p) {
    if (c.int8 || p.flags || p.split_k == 1) return 1;
    if (mr <= 0 || n <= 0 || k <= 0) return 1;
    if (ws_bytes < c.base) return 1;
    const int kb = (k + ddg::KC - 1) / ddg::KC;
    const int room = 1 + (int)std::min<size_t>((ws_bytes - c.base) / (2 * c.L.part_bytes),
                                                SPLIT_MAX - 1);
    int split = 1;
    if (p.split_k > 1)
        split = std::min(std::min(p.split_k, SPLIT_MAX), kb);
    else
        split = ddg::choose_split(fp64_tiles(mr, n), kb, sms, auto_split_cap(mr, n, k));
    return std::min(split, room);
}

int split_groups(int m, int n, int k, int sms, size_t ws_bytes, const Parsed &p) {
    if (m <= 0 || n <= 0 || k <= 0) return 1;
    return split_groups_in(m, n, k, sms, ws_bytes, carve_for(m, n, k, p), p);
}

int sm_count(int &sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DDGEMM_ECUDA;
    return DDGEMM_OK;
}

// Phase one for B (Appendix A; Sec. "FP64x2 in terms of INT8" for the INT8
// forms): the exponents of tau and the seven panels, or the digit planes.
// A column of op(B) is a vector; it runs along memory only if trans_b.
cudaError_t split_b_into(const Carve &c, int n, int k, const double *B_hi, const double *B_lo,
                         int ldb, char *ws, cudaStream_t s, const Parsed &p) {
    if (c.int8) {
        return ddg::launch_split_int8(p.slices, n, k, B_hi, B_lo, ldb, p.trans_b != 0,
                                      ws + c.L8.off_b, is_tc(p.variant) ? ddg::INT8_TC_BN : 0,
                                      int8_bits(p.variant), c.L8.ld,
                                      reinterpret_cast<int *>(ws + c.L8.off_eb), p.status, s);
    }
    return ddg::launch_split(7, n, k, B_hi, B_lo, ldb, p.trans_b != 0,
                             reinterpret_cast<double *>(ws + c.L.off_b), c.L.ldb_s,
                             ddg::PanelLayout::K_MAJOR, reinterpret_cast<int *>(ws + c.L.off_eb),
                             p.status, s);
}

// Phase one for mr rows of op(A) (a row is a vector; it runs along memory
// unless trans_a).
cudaError_t split_a_into(const Carve &c, int mr, int k, const double *A_hi, const double *A_lo,
                         int lda, char *ws, cudaStream_t s, const Parsed &p) {
    if (c.int8) {
        return ddg::launch_split_int8(p.slices, mr, k, A_hi, A_lo, lda, !p.trans_a,
                                      ws + c.L8.off_a, is_tc(p.variant) ? ddg::INT8_TC_BM : 0,
                                      int8_bits(p.variant), c.L8.ld,
                                      reinterpret_cast<int *>(ws + c.L8.off_ea), p.status, s);
    }
    return ddg::launch_split(4, mr, k, A_hi, A_lo, lda, !p.trans_a,
                             reinterpret_cast<double *>(ws + c.L.off_a), c.L.lda_s,
                             ddg::PanelLayout::VEC_MAJOR, reinterpret_cast<int *>(ws + c.L.off_ea),
                             p.status, s);
}

// Phases two and three for the mr rows whose pieces split_a_into wrote: the
// products, the bins' assembly and the FP64x2 accumulation into C (or, with
// bins, the bins of the single k-block).
cudaError_t products_into(const Carve &c, int mr, int n, int k, double *C_hi, double *C_lo,
                          int ldc, int *flags, double *bins, int split, char *ws, cudaStream_t s,
                          const Parsed &p, bool accumulate = false) {
    if (c.int8) {
        const Layout8 &L = c.L8;
        const int *e_a = reinterpret_cast<const int *>(ws + L.off_ea);
        const int *e_b = reinterpret_cast<const int *>(ws + L.off_eb);
        if (is_tc(p.variant)) {
            ddg::Int8TcArgs a{mr, n, k, p.slices, int8_bits(p.variant),
                              reinterpret_cast<const uint16_t *>(ws + L.off_a),
                              reinterpret_cast<const uint16_t *>(ws + L.off_b), e_a, e_b, C_hi,
                              C_lo, (long long)ldc, p.status, p.wait};
            return ddg::launch_cascade_int8_tc(a, s);
        }
        ddg::Int8Args a{mr, n, k, p.slices, reinterpret_cast<const int8_t *>(ws + L.off_a),
                        reinterpret_cast<const int8_t *>(ws + L.off_b), L.ld, e_a, e_b, C_hi,
                        C_lo, (long long)ldc, p.status, p.wait};
        return ddg::launch_cascade_int8(a, s);
    }
    const Layout &L = c.L;
    const int products = p.variant == DDGEMM_VARIANT_FP64_GEMM16    ? 1
                         : p.variant == DDGEMM_VARIANT_FP64_DROP456 ? 2
                                                                      : 0;
    double *part = reinterpret_cast<double *>(ws + L.off_part);
    double *part_lo =
        reinterpret_cast<double *>(ws + L.off_part + (size_t)(split - 1) * L.part_bytes);
    ddg::CascadeArgs ca{mr, n, k, reinterpret_cast<const double *>(ws + L.off_a), L.lda_s,
                        reinterpret_cast<const double *>(ws + L.off_b), L.ldb_s,
                        reinterpret_cast<const int *>(ws + L.off_ea),
                        reinterpret_cast<const int *>(ws + L.off_eb), C_hi, C_lo,
                        (long long)ldc, flags, p.status, bins, products, split, part, part_lo,
                        p.wait, accumulate};
    return ddg::launch_cascade_fp64(ca, s);
}

// One whole problem on device operands: the split of A, the split of B, and
// the products, with the optional phase events around them.
int run(int m, int n, int k, const double *A_hi, const double *A_lo, int lda,
        const double *B_hi, const double *B_lo, int ldb, double *C_hi, double *C_lo, int ldc,
        double *bins, void *workspace, size_t ws_bytes, cudaStream_t stream, const Parsed &p) {
    const Carve c = carve_for(m, n, k, p);
    if (!workspace || ws_bytes < c.base || (uintptr_t)workspace % ALIGN) return DDGEMM_EWORKSPACE;
    int split = 1;
    if (!c.int8 && !bins && !p.flags && p.split_k != 1) {
        int sms = 0;
        if (sm_count(sms) != DDGEMM_OK) return DDGEMM_ECUDA;
        split = split_groups_in(m, n, k, sms, ws_bytes, c, p);
    }
    char *ws = static_cast<char *>(workspace);
    auto mark = [&](int i) {
        return !p.events || cudaEventRecord(static_cast<cudaEvent_t>(p.events[i]), stream) ==
                                cudaSuccess;
    };
    if (!mark(0)) return DDGEMM_ECUDA;
    if (split_a_into(c, m, k, A_hi, A_lo, lda, ws, stream, p) != cudaSuccess ||
        split_b_into(c, n, k, B_hi, B_lo, ldb, ws, stream, p) != cudaSuccess || !mark(1))
        return DDGEMM_ECUDA;
    const cudaError_t e =
        products_into(c, m, n, k, C_hi, C_lo, ldc, p.flags, bins, split, ws, stream, p);
    return e == cudaSuccess && mark(2) ? DDGEMM_OK : DDGEMM_ECUDA;
}

// Workspace bytes of ddgemm() for a valid problem (m, n, k all positive),
// split-k partials included.
size_t workspace_total(int m, int n, int k, const Parsed &p) {
    if (is_int8(p.variant)) return layout8_for(m, n, k, p.slices, p.variant).total;
    return layout_for(m, n, k, split_reserve(m, n, k, p.split_k)).total;
}

// ---- host buffers: ddgemm_host ---------------------------------------------
//
// The operands are copied in and C is copied out by two streams of the call's
// own, so that the copies overlap the kernels on the caller's stream: A in
// row chunks, each split and multiplied as soon as its rows (and B) have
// arrived, and its rows of C copied back while the next chunk computes.  B
// is needed whole by every chunk; in the FP64 forms it comes in parts of
// whole k-blocks after the first chunk of A, and that chunk is multiplied
// part by part as they arrive (each part's product added into C in k-block
// order, as one launch would), so that only the first part of B stays
// exposed; B is then split whole for the other chunks.  The INT8 forms take
// B whole first.  Exposed: the copy of the first chunk of A and of B (or of
// its first part), their splits, and the copy of the last chunk of C.

constexpr int HOST_MAX_CHUNKS = 4;
constexpr int HOST_B_PARTS = 4;
constexpr long long HOST_MIN_TILES = 1024;

// Rows of op(A) per chunk: at least HOST_MIN_TILES tiles of the form's own
// tile shape per chunk, so that a chunk still fills the GPU, and at most
// HOST_MAX_CHUNKS chunks; a multiple of 128 (every form's tile height divides it).
int host_chunk_rows(int m, int n, const Parsed &p) {
    int tm = 64, tn = 64;
    if (is_tc(p.variant)) {
        tm = ddg::INT8_TC_BM;
        tn = ddg::INT8_TC_BN;
    } else if (p.variant == DDGEMM_VARIANT_INT8) {
        tm = 32;
        tn = 32;
    }
    const long long col_tiles = (n + tn - 1) / tn;
    const long long rows_min = (HOST_MIN_TILES + col_tiles - 1) / col_tiles * tm;
    long long mc = std::max<long long>(rows_min, (m + HOST_MAX_CHUNKS - 1) / HOST_MAX_CHUNKS);
    mc = (mc + 127) / 128 * 128;
    return (int)std::min<long long>(mc, m);
}

// Device buffer of ddgemm_host: dense copies of A (chunk after chunk), B and
// C, each as a hi plane then a lo plane, then the workspace for chunks of
// mc rows.
struct HostLayout {
    int mc = 0;
    size_t a_plane = 0, b_plane = 0, c_plane = 0;
    size_t off_a = 0, off_b = 0, off_c = 0, off_ws = 0, ws_bytes = 0, total = 0;
};

HostLayout host_layout(int m, int n, int k, const Parsed &p) {
    HostLayout H;
    H.mc = k == 0 ? m : host_chunk_rows(m, n, p);
    H.a_plane = round_up((size_t)m * k * sizeof(double), ALIGN);
    H.b_plane = round_up((size_t)k * n * sizeof(double), ALIGN);
    H.c_plane = round_up((size_t)m * n * sizeof(double), ALIGN);
    H.off_a = 0;
    H.off_b = H.off_a + 2 * H.a_plane;
    H.off_c = H.off_b + 2 * H.b_plane;
    H.off_ws = H.off_c + 2 * H.c_plane;
    H.ws_bytes = k == 0 ? 0 : workspace_total(H.mc, n, k, p);
    H.total = H.off_ws + H.ws_bytes;
    return H;
}

// The copy streams and events of one ddgemm_host call.  A call takes a set
// from its device's pool and puts it back when it returns: the first call on
// a device (and each call that overlaps another on the host) creates one,
// later calls reuse them, so a call creates nothing.  A set is used by one
// call at a time, so its event records and waits cannot interleave with
// another call's; work a call left on the set's streams only orders the next
// call's copies after it (both wait for their own caller's stream anyway).
// The sets live until the process exits.
struct HostStreams {
    static constexpr int MAX_EVENTS = 3 + 2 * HOST_MAX_CHUNKS + HOST_B_PARTS;
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t ev[MAX_EVENTS] = {};
    bool init() {
        if (cudaStreamCreateWithFlags(&h2d, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&d2h, cudaStreamNonBlocking) != cudaSuccess)
            return false;
        for (auto &e : ev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return false;
        return true;
    }
    void release() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e), e = nullptr;
        if (h2d) cudaStreamDestroy(h2d), h2d = nullptr;
        if (d2h) cudaStreamDestroy(d2h), d2h = nullptr;
    }
};

std::mutex g_host_pool_mutex;
std::unordered_map<int, std::vector<HostStreams *>> g_host_pool;  // by device

// A set of copy streams and events on the current device, from the pool or
// new (nullptr if creating one fails); returned with put_host_streams.
HostStreams *take_host_streams(int dev) {
    {
        std::lock_guard<std::mutex> lock(g_host_pool_mutex);
        auto &free = g_host_pool[dev];
        if (!free.empty()) {
            HostStreams *h = free.back();
            free.pop_back();
            return h;
        }
    }
    HostStreams *h = new HostStreams;
    if (!h->init()) {
        h->release();
        delete h;
        return nullptr;
    }
    return h;
}

void put_host_streams(int dev, HostStreams *h) {
    std::lock_guard<std::mutex> lock(g_host_pool_mutex);
    g_host_pool[dev].push_back(h);
}

// Holds a pooled set for the length of one call.
struct PooledHostStreams {
    int dev = -1;
    HostStreams *h = nullptr;
    bool acquire() {
        if (cudaGetDevice(&dev) != cudaSuccess) return false;
        h = take_host_streams(dev);
        return h != nullptr;
    }
    ~PooledHostStreams() {
        if (h) put_host_streams(dev, h);
    }
};

// `to` waits for the work enqueued so far on `from`.
bool after(cudaStream_t to, cudaStream_t from, cudaEvent_t e) {
    return cudaEventRecord(e, from) == cudaSuccess && cudaStreamWaitEvent(to, e, 0) == cudaSuccess;
}

// A rows x cols block of doubles (row pitches in elements), either way
// between host and device.
bool copy2d(double *dst, long long dpitch, const double *src, long long spitch, long long cols,
            long long rows, cudaStream_t s) {
    if (rows == 0 || cols == 0) return true;
    return cudaMemcpy2DAsync(dst, (size_t)dpitch * sizeof(double), src,
                             (size_t)spitch * sizeof(double), (size_t)cols * sizeof(double),
                             (size_t)rows, cudaMemcpyDefault, s) == cudaSuccess;
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
    return workspace_total(m, n, k, p);
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
    if (p.variant < DDGEMM_VARIANT_FP64 || p.variant > DDGEMM_VARIANT_INT8_TC8)
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
    return run(m, n, k, A_hi, A_lo, lda, B_hi, B_lo, ldb, C_hi, C_lo, ldc, nullptr, workspace,
               ws_bytes, s, p);
}

size_t ddgemm_host_buffer_size(int m, int n, int k, const ddgemm_opts *opts) {
    Parsed p;
    if (!parse(opts, p) || !dims_ok(m, n, k)) return 0;
    if (p.variant < DDGEMM_VARIANT_FP64 || p.variant > DDGEMM_VARIANT_INT8_TC8) return 0;
    if (m == 0 || n == 0) return 0;
    return host_layout(m, n, k, p).total;
}

int ddgemm_diag_withheld_copy(int m, int n, int k, const double *A_hi, const double *A_lo,
                              int lda, const double *B_hi, const double *B_lo, int ldb,
                              double *C_hi, double *C_lo, int ldc, void *workspace,
                              size_t ws_bytes, void *stream, const ddgemm_opts *opts, int cta,
                              long long step, unsigned long long limit_ns) {
    Parsed p;
    if (!opts || !opts->status_dev || !parse(opts, p) || !dims_ok(m, n, k)) return DDGEMM_EINVAL;
    if (cta < 0 || step < 0 || limit_ns < 1000ull || limit_ns > 10000000000ull)
        return DDGEMM_EINVAL;
    if (p.variant < DDGEMM_VARIANT_FP64 || p.variant > DDGEMM_VARIANT_INT8_TC8 || p.flags)
        return DDGEMM_EUNSUPPORTED;
    if (int r = check_operands(m, n, k, A_hi, A_lo, lda, B_hi, B_lo, ldb, p)) return r;
    if (m == 0 || n == 0 || k == 0) return DDGEMM_EINVAL;  // no kernel to withhold from
    if (!C_hi || !C_lo || ldc < n) return DDGEMM_EINVAL;
    p.events = nullptr;
    p.wait.limit_ns = limit_ns;
    p.wait.cta = cta;
    p.wait.step = step;
    return run(m, n, k, A_hi, A_lo, lda, B_hi, B_lo, ldb, C_hi, C_lo, ldc, nullptr, workspace,
               ws_bytes, static_cast<cudaStream_t>(stream), p);
}

int ddgemm_host(int m, int n, int k, const double *A_hi, const double *A_lo, int lda,
                const double *B_hi, const double *B_lo, int ldb, double *C_hi, double *C_lo,
                int ldc, void *buffer, size_t buffer_bytes, void *stream,
                const ddgemm_opts *opts) {
    Parsed p;
    if (!parse(opts, p) || !dims_ok(m, n, k)) return DDGEMM_EINVAL;
    if (p.variant < DDGEMM_VARIANT_FP64 || p.variant > DDGEMM_VARIANT_INT8_TC8)
        return DDGEMM_EUNSUPPORTED;
    if (is_int8(p.variant) && p.flags) return DDGEMM_EUNSUPPORTED;
    if (int r = check_operands(m, n, k, A_hi, A_lo, lda, B_hi, B_lo, ldb, p)) return r;
    if (m == 0 || n == 0) return DDGEMM_OK;
    if (!C_hi || !C_lo || ldc < n) return DDGEMM_EINVAL;
    p.events = nullptr;
    const HostLayout H = host_layout(m, n, k, p);
    if (!buffer || buffer_bytes < H.total || (uintptr_t)buffer % ALIGN) return DDGEMM_EWORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *buf = static_cast<char *>(buffer);
    double *a_hi = reinterpret_cast<double *>(buf + H.off_a);
    double *a_lo = reinterpret_cast<double *>(buf + H.off_a + H.a_plane);
    double *b_hi = reinterpret_cast<double *>(buf + H.off_b);
    double *b_lo = reinterpret_cast<double *>(buf + H.off_b + H.b_plane);
    double *c_hi = reinterpret_cast<double *>(buf + H.off_c);
    double *c_lo = reinterpret_cast<double *>(buf + H.off_c + H.c_plane);
    char *ws = buf + H.off_ws;

    PooledHostStreams pooled;
    if (!pooled.acquire()) return DDGEMM_ECUDA;
    HostStreams &hs = *pooled.h;
    // event slots: the entry, B copied, chunk r of A copied, chunk r of C
    // done, part q of B copied
    constexpr int E_ENTRY = 0, E_B = 1, E_A = 2, E_C = 2 + HOST_MAX_CHUNKS,
                  E_BP = 2 + 2 * HOST_MAX_CHUNKS;
    // nothing of this call starts before the work already on the caller's
    // stream (which may still be using the buffer)
    if (!after(hs.h2d, s, hs.ev[E_ENTRY]) ||
        cudaStreamWaitEvent(hs.d2h, hs.ev[E_ENTRY], 0) != cudaSuccess)
        return DDGEMM_ECUDA;
    const int nchunks = (m + H.mc - 1) / H.mc;  // 1 when k = 0
    if (k == 0) {
        // C := 0 on the device (and the flags), then back
        ddgemm_opts z{p.trans_a, p.trans_b, p.variant, p.status, p.flags, nullptr, p.slices,
                      p.split_k};
        if (int r = ddgemm(m, n, 0, nullptr, nullptr, 0, nullptr, nullptr, 0, c_hi, c_lo, n,
                           nullptr, 0, stream, &z))
            return r;
        if (cudaEventRecord(hs.ev[E_C], s) != cudaSuccess) return DDGEMM_ECUDA;
    } else {
        const long long bk = p.trans_b ? n : k, bn = p.trans_b ? k : n;  // stored shape
        const Carve c = carve_for(H.mc, n, k, p);
        int sms = 0;
        if (!c.int8 && sm_count(sms) != DDGEMM_OK) return DDGEMM_ECUDA;
        // chunk r of A: its device rows and the copy of them
        auto chunk_a = [&](int r, double *&ah, double *&al, int &mr, int &lda_c) {
            const int r0 = r * H.mc;
            mr = std::min(H.mc, m - r0);
            ah = a_hi + (size_t)r0 * k;
            al = a_lo + (size_t)r0 * k;
            // the chunk keeps A's stored orientation: rows r0.. of A, or
            // columns r0.. of the stored k x m matrix
            lda_c = p.trans_a ? mr : k;
            return p.trans_a ? copy2d(ah, mr, A_hi + r0, lda, mr, k, hs.h2d) &&
                                   copy2d(al, mr, A_lo + r0, lda, mr, k, hs.h2d)
                             : copy2d(ah, k, A_hi + (size_t)r0 * lda, lda, k, mr, hs.h2d) &&
                                   copy2d(al, k, A_lo + (size_t)r0 * lda, lda, k, mr, hs.h2d);
        };
        // B in parts of whole k-blocks for the first chunk (FP64 forms, when
        // there is a second chunk to hide it behind and the parts' workspace
        // fits where B's pieces go later)
        const int kblocks = (k + ddg::KC - 1) / ddg::KC;
        int parts = 1, kpart = k;
        Carve cp;
        size_t cp_bytes = 0;
        if (!c.int8 && nchunks > 1 && kblocks > 1) {
            parts = std::min(HOST_B_PARTS, kblocks);
            kpart = (kblocks + parts - 1) / parts * ddg::KC;
            parts = (k + kpart - 1) / kpart;
            cp = carve_for(H.mc, n, kpart, p);
            cp_bytes = H.ws_bytes - c.L.off_b;
            if (cp.base > cp_bytes) parts = 1;
        }
        int r_first = 0;
        if (parts > 1) {
            // copies: the first chunk of A, then B part by part
            double *ah, *al;
            int mr, lda_c;
            if (!chunk_a(0, ah, al, mr, lda_c) || !after(s, hs.h2d, hs.ev[E_A])) return DDGEMM_ECUDA;
            for (int q = 0; q < parts; ++q) {
                const long long k0 = (long long)q * kpart, kq = std::min<long long>(kpart, k - k0);
                const bool ok =
                    p.trans_b ? copy2d(b_hi + k0, bn, B_hi + k0, ldb, kq, bk, hs.h2d) &&
                                    copy2d(b_lo + k0, bn, B_lo + k0, ldb, kq, bk, hs.h2d)
                              : copy2d(b_hi + k0 * bn, bn, B_hi + k0 * ldb, ldb, bn, kq, hs.h2d) &&
                                    copy2d(b_lo + k0 * bn, bn, B_lo + k0 * ldb, ldb, bn, kq, hs.h2d);
                if (!ok || cudaEventRecord(hs.ev[E_BP + q], hs.h2d) != cudaSuccess)
                    return DDGEMM_ECUDA;
            }
            // the first chunk's products part by part, in the parts' own
            // workspace (where B's pieces go later), each added into C
            char *wp = ws + c.L.off_b;
            for (int q = 0; q < parts; ++q) {
                const int k0 = q * kpart, kq = std::min(kpart, k - k0);
                const double *aph = p.trans_a ? ah + (size_t)k0 * mr : ah + k0;
                const double *apl = p.trans_a ? al + (size_t)k0 * mr : al + k0;
                const double *bph = p.trans_b ? b_hi + k0 : b_hi + (size_t)k0 * bn;
                const double *bpl = p.trans_b ? b_lo + k0 : b_lo + (size_t)k0 * bn;
                const int split = split_groups_in(mr, n, kq, sms, cp_bytes, cp, p);
                if (cudaStreamWaitEvent(s, hs.ev[E_BP + q], 0) != cudaSuccess ||
                    split_a_into(cp, mr, kq, aph, apl, lda_c, wp, s, p) != cudaSuccess ||
                    split_b_into(cp, n, kq, bph, bpl, (int)bn, wp, s, p) != cudaSuccess ||
                    products_into(cp, mr, n, kq, c_hi, c_lo, n, p.flags, nullptr, split, wp, s, p,
                                  q > 0) != cudaSuccess)
                    return DDGEMM_ECUDA;
            }
            if (cudaEventRecord(hs.ev[E_C], s) != cudaSuccess) return DDGEMM_ECUDA;
            r_first = 1;
        } else {
            // B whole first
            if (!copy2d(b_hi, bn, B_hi, ldb, bn, bk, hs.h2d) ||
                !copy2d(b_lo, bn, B_lo, ldb, bn, bk, hs.h2d) || !after(s, hs.h2d, hs.ev[E_B]))
                return DDGEMM_ECUDA;
        }
        // B split whole (all of it has arrived: the stream waited for its
        // copy or for its last part) for the remaining chunks
        if (r_first < nchunks && split_b_into(c, n, k, b_hi, b_lo, (int)bn, ws, s, p) != cudaSuccess)
            return DDGEMM_ECUDA;
        for (int r = r_first; r < nchunks; ++r) {
            const int r0 = r * H.mc;
            double *ah, *al;
            int mr, lda_c;
            if (!chunk_a(r, ah, al, mr, lda_c) || !after(s, hs.h2d, hs.ev[E_A + r]))
                return DDGEMM_ECUDA;
            const int split = c.int8 ? 1 : split_groups_in(mr, n, k, sms, H.ws_bytes, c, p);
            if (split_a_into(c, mr, k, ah, al, lda_c, ws, s, p) != cudaSuccess ||
                products_into(c, mr, n, k, c_hi + (size_t)r0 * n, c_lo + (size_t)r0 * n, n,
                              p.flags ? p.flags + (size_t)r0 * n : nullptr, nullptr, split, ws, s,
                              p) != cudaSuccess ||
                cudaEventRecord(hs.ev[E_C + r], s) != cudaSuccess)
                return DDGEMM_ECUDA;
        }
    }
    // C back, chunk by chunk as each is done (all enqueued after the kernels,
    // so that a pageable destination, which makes a copy wait on the host,
    // cannot hold back a launch)
    for (int r = 0; r < nchunks; ++r) {
        const int r0 = r * H.mc, mr = std::min(H.mc, m - r0);
        if (cudaStreamWaitEvent(hs.d2h, hs.ev[E_C + r], 0) != cudaSuccess ||
            !copy2d(C_hi + (size_t)r0 * ldc, ldc, c_hi + (size_t)r0 * n, n, n, mr, hs.d2h) ||
            !copy2d(C_lo + (size_t)r0 * ldc, ldc, c_lo + (size_t)r0 * n, n, n, mr, hs.d2h))
            return DDGEMM_ECUDA;
    }
    // the caller's stream ends after the last copy
    return after(s, hs.d2h, hs.ev[HostStreams::MAX_EVENTS - 1]) ? DDGEMM_OK : DDGEMM_ECUDA;
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
                                                 0, ddg::INT8_BITS, ld_digits, exps, status_dev,
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
                                                 digits, 0, ddg::INT8_BITS, ld_digits, exps,
                                                 status_dev,
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
