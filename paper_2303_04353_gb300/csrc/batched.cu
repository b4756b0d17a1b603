// Many FP64x2 GEMMs of uneven shapes in one pass of four launches: a plan,
// the batched split of every A, the batched split of every B, and one
// persistent cascade kernel whose CTAs pull (problem, tile) items from an
// atomic counter.  The paper has no batched form; this is the FP64 cascade
// (eq. Gemm10, Sec. "Simple") scheduled for many small problems at once,
// which one launch per problem would spread over a few SMs only.
//
// Everything the kernels need is computed on the device from the caller's
// device copy of the problem list, so the whole call can be captured into a
// CUDA graph.  The per-tile arithmetic is cascade_core.cuh, the same as the
// single-problem kernel's, so every problem's C is bit-identical to what
// ddgemm() computes for it.  Tiles are staged with cp.async (16-byte copies
// with zero fill at the problem's edges): one tensor map per problem would
// not fit in the kernel's parameters.
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "../../include/ddgemm.h"
#include "../../include/ddgemm_diag.h"
#include "cascade_core.cuh"
#include "ddgemm_internal.h"
#include "split_device.cuh"

namespace ddg {
namespace {

constexpr size_t ALIGN = 256;
constexpr int NST = 3;  // cp.async stages

__host__ __device__ inline size_t ru(size_t x, size_t a) { return (x + a - 1) / a * a; }

// One problem as the kernels see it (index order).
struct Entry {
    int m, n, k, kb;
    int lda, ldb, vec_a, vec_b;
    long long lda_s, ldb_s, ldc;
    const double *a_hi, *a_lo, *b_hi, *b_lo;
    double *a_s, *b_s;
    int *e_a, *e_b;
    double *c_hi, *c_lo;
    int tiles_n, tiles;
    long long a_units, b_units;
};

struct Header {
    long long total_tiles, total_a, total_b;
    unsigned long long counter;
    int count;
};

// Workspace: [Header][Entry x count][order][tile prefix][a prefix][b prefix] | panels
struct PlanLayout {
    size_t entries, order, tile_pre, a_pre, b_pre, panels;
};

__host__ __device__ inline PlanLayout plan_layout(int count) {
    PlanLayout L;
    L.entries = ru(sizeof(Header), ALIGN);
    L.order = ru(L.entries + (size_t)count * sizeof(Entry), ALIGN);
    L.tile_pre = ru(L.order + (size_t)count * sizeof(int), ALIGN);
    L.a_pre = ru(L.tile_pre + (size_t)(count + 1) * sizeof(long long), ALIGN);
    L.b_pre = ru(L.a_pre + (size_t)(count + 1) * sizeof(long long), ALIGN);
    L.panels = ru(L.b_pre + (size_t)(count + 1) * sizeof(long long), ALIGN);
    return L;
}

// Panel bytes of one problem, with the single-problem layout.
__host__ __device__ inline size_t panel_bytes(int m, int n, int k) {
    if (m <= 0 || n <= 0 || k <= 0) return 0;
    const size_t kb = (size_t)(k + KC - 1) / KC;
    const size_t lda_s = ru((size_t)k, 8), ldb_s = ru((size_t)n, 8);
    return ru(4 * (size_t)m * lda_s * 8, ALIGN) + ru(7 * (size_t)k * ldb_s * 8, ALIGN) +
           ru(kb * m * 4, ALIGN) + ru(kb * n * 4, ALIGN);
}

__device__ inline long long find(const long long *prefix, int count, long long u) {
    int lo = 0, hi = count;  // prefix[lo] <= u < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= u) lo = mid; else hi = mid;
    }
    return lo;
}

// Ordering key for "longest k first": larger k, then larger m n, then index
// (false for a = b).  Without branches: the lanes of the rank loop compare
// different problems, and branching on the keys diverged.
__device__ inline bool before(int ka, long long sa, int ia, int kb, long long sb, int ib) {
    return (ka > kb) | ((ka == kb) & ((sa > sb) | ((sa == sb) & (ia < ib))));
}

// Problems whose ordering keys the plan kernel keeps in shared memory.
constexpr int PLAN_SMEM_KEYS = 2048;

// One CTA of 256 threads.  Every thread fills the entries of its problems
// and their ranks in the schedule (a rank compares the problem with every
// other one); then the prefix sums over the problems (split units,
// workspace bytes) and over the ranks (tiles): thread t takes a contiguous
// segment, the 256 segment totals are scanned by one warp per quantity, and
// every thread walks its segment again from its offsets.
__global__ void __launch_bounds__(256)
plan_kernel(int count, const ddgemm_problem *__restrict__ probs, char *ws, int order_mode, int bm,
            int bn) {
    const PlanLayout L = plan_layout(count);
    Header *hdr = reinterpret_cast<Header *>(ws);
    Entry *ent = reinterpret_cast<Entry *>(ws + L.entries);
    int *order = reinterpret_cast<int *>(ws + L.order);
    long long *tile_pre = reinterpret_cast<long long *>(ws + L.tile_pre);
    long long *a_pre = reinterpret_cast<long long *>(ws + L.a_pre);
    long long *b_pre = reinterpret_cast<long long *>(ws + L.b_pre);
    const bool by_k = order_mode == DDGEMM_ORDER_LONGEST_K_FIRST;
    __shared__ int key_k[PLAN_SMEM_KEYS];
    __shared__ long long key_mn[PLAN_SMEM_KEYS];
    const bool keys_in_smem = by_k && count <= PLAN_SMEM_KEYS;
    if (keys_in_smem) {
        for (int i = threadIdx.x; i < count; i += blockDim.x) {
            key_k[i] = probs[i].k;
            key_mn[i] = (long long)probs[i].m * probs[i].n;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        const ddgemm_problem q = probs[i];
        Entry e;
        e.m = q.m; e.n = q.n; e.k = q.k;
        e.kb = q.k > 0 ? (q.k + KC - 1) / KC : 0;
        e.lda = q.lda; e.ldb = q.ldb; e.ldc = q.ldc;
        e.a_hi = q.A_hi; e.a_lo = q.A_lo; e.b_hi = q.B_hi; e.b_lo = q.B_lo;
        e.c_hi = q.C_hi; e.c_lo = q.C_lo;
        e.vec_a = (q.lda % 2 == 0) && ((uintptr_t)q.A_hi % 16 == 0) && ((uintptr_t)q.A_lo % 16 == 0);
        e.vec_b = (q.ldb % 2 == 0) && ((uintptr_t)q.B_hi % 16 == 0) && ((uintptr_t)q.B_lo % 16 == 0);
        e.lda_s = (long long)ru((size_t)(q.k > 0 ? q.k : 0), 8);
        e.ldb_s = (long long)ru((size_t)(q.n > 0 ? q.n : 0), 8);
        const bool mn = q.m > 0 && q.n > 0;
        e.tiles_n = mn ? (q.n + bn - 1) / bn : 0;
        e.tiles = mn ? ((q.m + bm - 1) / bm) * e.tiles_n : 0;
        const bool work = mn && q.k > 0;
        e.a_units = work ? (long long)q.m * e.kb : 0;
        e.b_units = work ? (long long)e.kb * ((q.n + 63) / 64) : 0;
        e.a_s = e.b_s = nullptr;
        e.e_a = e.e_b = nullptr;
        ent[i] = e;
        // rank for the schedule
        int r = i;
        if (by_k) {
            const long long qmn = (long long)q.m * q.n;
            r = 0;
            if (keys_in_smem) {
#pragma unroll 4
                for (int j = 0; j < count; ++j) r += before(key_k[j], key_mn[j], j, q.k, qmn, i);
            } else {
                for (int j = 0; j < count; ++j)
                    r += before(probs[j].k, (long long)probs[j].m * probs[j].n, j, q.k, qmn, i);
            }
        }
        order[r] = i;
    }
    __syncthreads();
    constexpr int NQ = 4;  // a units, b units, workspace bytes, tiles (rank order)
    __shared__ long long part[NQ][256];  // blockDim.x <= 256
    const int nt = blockDim.x, t = threadIdx.x;
    const int seg = (count + nt - 1) / nt;
    const int i0 = min(count, t * seg), i1 = min(count, i0 + seg);
    {
        long long acc[NQ] = {0, 0, 0, 0};
        for (int i = i0; i < i1; ++i) {
            const Entry &e = ent[i];
            acc[0] += e.a_units;
            acc[1] += e.b_units;
            acc[2] += (long long)panel_bytes(e.m, e.n, e.k);
            acc[3] += ent[order[i]].tiles;
        }
        for (int q = 0; q < NQ; ++q) part[q][t] = acc[q];
    }
    __syncthreads();
    {
        // exclusive scan of part[q][0 .. nt-1] by warp q (nt <= 256)
        const int w = t >> 5, lane = t & 31;
        if (w < NQ) {
            long long v[8], run = 0;
            for (int j = 0; j < 8; ++j) {
                const int x = lane * 8 + j;
                v[j] = x < nt ? part[w][x] : 0;
                run += v[j];
            }
            long long incl = run;
            for (int off = 1; off < 32; off <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += y;
            }
            long long pre = incl - run;
            for (int j = 0; j < 8; ++j) {
                const int x = lane * 8 + j;
                if (x < nt) part[w][x] = pre;
                pre += v[j];
            }
        }
    }
    __syncthreads();
    {
        long long ta = part[0][t], tb = part[1][t], tt = part[3][t];
        size_t off = L.panels + (size_t)part[2][t];
        for (int i = i0; i < i1; ++i) {
            Entry &e = ent[i];
            a_pre[i] = ta;
            b_pre[i] = tb;
            ta += e.a_units;
            tb += e.b_units;
            if (e.a_units > 0) {
                e.a_s = reinterpret_cast<double *>(ws + off);
                off += ru(4 * (size_t)e.m * e.lda_s * 8, ALIGN);
                e.b_s = reinterpret_cast<double *>(ws + off);
                off += ru(7 * (size_t)e.k * e.ldb_s * 8, ALIGN);
                e.e_a = reinterpret_cast<int *>(ws + off);
                off += ru((size_t)e.kb * e.m * 4, ALIGN);
                e.e_b = reinterpret_cast<int *>(ws + off);
                off += ru((size_t)e.kb * e.n * 4, ALIGN);
            }
            tile_pre[i] = tt;
            tt += ent[order[i]].tiles;
        }
        if (i1 == count && i0 < i1) {  // the last non-empty segment: the totals
            a_pre[count] = ta;
            b_pre[count] = tb;
            tile_pre[count] = tt;
            hdr->total_tiles = tt;
            hdr->total_a = ta;
            hdr->total_b = tb;
            hdr->counter = 0ull;
            hdr->count = count;
        }
    }
}

// A: one warp per (problem, row, k-block), grid-stride over all of them.
__global__ void __launch_bounds__(256) batched_split_a_kernel(const char *ws, unsigned int *status) {
    const Header *hdr = reinterpret_cast<const Header *>(ws);
    const int count = hdr->count;
    const PlanLayout L = plan_layout(count);
    const Entry *ent = reinterpret_cast<const Entry *>(ws + L.entries);
    const long long *a_pre = reinterpret_cast<const long long *>(ws + L.a_pre);
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < hdr->total_a;
         u += nw) {
        const int i = (int)find(a_pre, count, u);
        const Entry &e = ent[i];
        const long long local = u - a_pre[i];
        const int v = (int)(local / e.kb), p = (int)(local % e.kb);
        if (e.vec_a)
            split_detail::split_contig_unit<4, true>(lane, v, p, e.m, e.k, e.a_hi, e.a_lo, e.lda,
                                                     e.a_s, e.lda_s, PanelLayout::VEC_MAJOR,
                                                     e.e_a, status);
        else
            split_detail::split_contig_unit<4, false>(lane, v, p, e.m, e.k, e.a_hi, e.a_lo, e.lda,
                                                      e.a_s, e.lda_s, PanelLayout::VEC_MAJOR,
                                                      e.e_a, status);
    }
}

// B: one CTA per (problem, k-block, 64 columns), grid-stride.
__global__ void __launch_bounds__(256) batched_split_b_kernel(const char *ws, unsigned int *status) {
    __shared__ double part[8][64];
    __shared__ int sexp[64];
    const Header *hdr = reinterpret_cast<const Header *>(ws);
    const int count = hdr->count;
    const PlanLayout L = plan_layout(count);
    const Entry *ent = reinterpret_cast<const Entry *>(ws + L.entries);
    const long long *b_pre = reinterpret_cast<const long long *>(ws + L.b_pre);
    for (long long u = blockIdx.x; u < hdr->total_b; u += gridDim.x) {
        const int i = (int)find(b_pre, count, u);
        const Entry &e = ent[i];
        const long long local = u - b_pre[i];
        const int vtiles = (e.n + 63) / 64;
        const int vt = (int)(local % vtiles), p = (int)(local / vtiles);
        if (e.vec_b)
            split_detail::split_strided_unit<7, true>(vt, p, e.n, e.k, e.b_hi, e.b_lo, e.ldb,
                                                      e.b_s, e.ldb_s, PanelLayout::K_MAJOR, e.e_b,
                                                      status, part, sexp);
        else
            split_detail::split_strided_unit<7, false>(vt, p, e.n, e.k, e.b_hi, e.b_lo, e.ldb,
                                                       e.b_s, e.ldb_s, PanelLayout::K_MAJOR,
                                                       e.e_b, status, part, sexp);
    }
}

__device__ __forceinline__ void cp_async16(double *dst, const double *src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The step-t slices of the four A pieces and seven B panels of one tile,
// 16 bytes per copy; entries outside the problem are zero-filled.
template <int BM, int BN, int NT>
__device__ __forceinline__ void load_stage(const Entry &e, int m0, int n0, int t, double *As,
                                           double *Bs) {
    const int k0 = t * CBK;
    for (int c = threadIdx.x; c < 16 * BM; c += NT) {
        const int s = c / (4 * BM), rem = c % (4 * BM), r = rem >> 2, q = rem & 3;
        const int row = m0 + r, col = k0 + 2 * q;
        const int valid = row < e.m ? max(0, min(2, e.k - col)) : 0;
        const double *src = valid ? e.a_s + ((long long)s * e.m + row) * e.lda_s + col : e.a_s;
        cp_async16(As + s * BM * CBK + r * CBK + 2 * q, src, valid * 8);
    }
    constexpr int HALF = BN / 2;
    for (int c = threadIdx.x; c < 7 * CBK * HALF; c += NT) {
        const int s = c / (CBK * HALF), rem = c % (CBK * HALF), kk = rem / HALF, q = rem % HALF;
        const int krow = k0 + kk, col = n0 + 2 * q;
        const int valid = krow < e.k ? max(0, min(2, e.n - col)) : 0;
        const double *src = valid ? e.b_s + ((long long)s * e.k + krow) * e.ldb_s + col : e.b_s;
        cp_async16(Bs + s * CBK * BN + kk * BN + 2 * q, src, valid * 8);
    }
}

template <int WM, int WN>
__global__ void __launch_bounds__(32 * WM * WN)
batched_cascade_kernel(char *ws) {
    using T = Fp64Tile<WM, WN>;
    constexpr int BM = T::BM, BN = T::BN, NT = T::NTHREADS;
    extern __shared__ unsigned char smem_raw[];
    double *smem = reinterpret_cast<double *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    __shared__ long long s_item;
    Header *hdr = reinterpret_cast<Header *>(ws);
    const int count = hdr->count;
    const PlanLayout L = plan_layout(count);
    const Entry *ent = reinterpret_cast<const Entry *>(ws + L.entries);
    const int *order = reinterpret_cast<const int *>(ws + L.order);
    const long long *tile_pre = reinterpret_cast<const long long *>(ws + L.tile_pre);
    const long long total = hdr->total_tiles;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp % WM, wn = warp / WM;
    constexpr int STEPS_PER_BLOCK = KC / CBK;

    for (;;) {
        if (tid == 0) s_item = (long long)atomicAdd(&hdr->counter, 1ull);
        __syncthreads();
        const long long item = s_item;
        __syncthreads();
        if (item >= total) break;
        const int r = (int)find(tile_pre, count, item);
        const Entry &e = ent[order[r]];
        const long long local = item - tile_pre[r];
        const int m0 = (int)(local / e.tiles_n) * BM, n0 = (int)(local % e.tiles_n) * BN;
        const int ksteps = (e.k + CBK - 1) / CBK;
        if (ksteps == 0) {  // k = 0: C = 0 on this tile
            for (int x = tid; x < BM * BN; x += NT) {
                const int row = m0 + x / BN, col = n0 + x % BN;
                if (row < e.m && col < e.n) {
                    e.c_hi[(long long)row * e.ldc + col] = 0.0;
                    e.c_lo[(long long)row * e.ldc + col] = 0.0;
                }
            }
            continue;
        }
        const EpilogueOut out{e.m, e.n, e.e_a, e.e_b, e.c_hi, e.c_lo, e.ldc, nullptr, nullptr};
        Acc acc;
        zero_acc(acc);
#pragma unroll
        for (int s = 0; s < NST - 1; ++s) {
            if (s < ksteps)
                load_stage<BM, BN, NT>(e, m0, n0, s, smem + s * T::STAGE,
                                       smem + s * T::STAGE + T::A_STAGE);
            cp_async_commit();
        }
        for (int t = 0; t < ksteps; ++t) {
            cp_async_wait<NST - 2>();
            __syncthreads();  // step t is in shared memory; step t-1 is consumed
            const double *As = smem + (t % NST) * T::STAGE;
            mma_stage<BM, BN>(acc, As, As + T::A_STAGE, wm, wn, lane);
            const int nxt = t + NST - 1;
            if (nxt < ksteps)
                load_stage<BM, BN, NT>(e, m0, n0, nxt, smem + (nxt % NST) * T::STAGE,
                                       smem + (nxt % NST) * T::STAGE + T::A_STAGE);
            cp_async_commit();
            if ((t + 1) % STEPS_PER_BLOCK == 0 || t + 1 == ksteps)
                epilogue<false>(acc, t / STEPS_PER_BLOCK, t < STEPS_PER_BLOCK, m0 + wm * 16,
                                n0 + wn * 32, lane, out);
        }
        cp_async_wait<0>();
        __syncthreads();  // the next tile refills the stages
    }
}

template <int WM, int WN>
size_t smem_of() {
    return (size_t)NST * Fp64Tile<WM, WN>::STAGE * sizeof(double) + 128;
}

template <int WM, int WN>
cudaError_t launch_cascade(char *ws, int sms, cudaStream_t stream) {
    const size_t smem = smem_of<WM, WN>();
    cudaError_t e = cudaFuncSetAttribute(batched_cascade_kernel<WM, WN>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_cascade_kernel<WM, WN>,
                                                      32 * WM * WN, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    batched_cascade_kernel<WM, WN><<<sms * per_sm, 32 * WM * WN, smem, stream>>>(ws);
    return cudaGetLastError();
}

void tile_shape(int tile, int &bm, int &bn) {
    switch (tile) {
        case DDGEMM_TILE_32x64: bm = 32; bn = 64; break;
        case DDGEMM_TILE_64x32: bm = 64; bn = 32; break;
        case DDGEMM_TILE_32x32: bm = 32; bn = 32; break;
        default: bm = 64; bn = 64; break;
    }
}

bool problem_ok(const ddgemm_problem &q) {
    if (q.m < 0 || q.n < 0 || q.k < 0) return false;
    if (q.m > 0 && q.n > 0) {
        if (!q.C_hi || !q.C_lo || q.ldc < q.n) return false;
        if (q.k > 0 && (!q.A_hi || !q.A_lo || !q.B_hi || !q.B_lo || q.lda < q.k || q.ldb < q.n))
            return false;
    }
    return true;
}

}  // namespace
}  // namespace ddg

extern "C" size_t ddgemm_batched_workspace_size(int count, const ddgemm_problem *probs_host,
                                                const ddgemm_opts *opts) {
    if (count <= 0 || !probs_host) return 0;
    if (opts && opts->variant == DDGEMM_VARIANT_INT8_TC) {
        const int s = opts->int8_slices ? opts->int8_slices : ddg::INT8_TC_SLICES_DEFAULT;
        if (!ddg::int8_tc_slices_supported(s)) return 0;
        return ddg::batched_int8_tc_workspace_size(count, probs_host, s, ddg::INT8_TC_BITS);
    }
    if (opts && opts->variant == DDGEMM_VARIANT_INT8_TC8) {
        const int s = opts->int8_slices ? opts->int8_slices : ddg::INT8_TC8_SLICES_DEFAULT;
        if (!ddg::int8_tc8_slices_supported(s)) return 0;
        return ddg::batched_int8_tc_workspace_size(count, probs_host, s, ddg::INT8_BITS);
    }
    size_t total = ddg::plan_layout(count).panels;
    for (int i = 0; i < count; ++i) {
        const ddgemm_problem &q = probs_host[i];
        total += ddg::panel_bytes(q.m, q.n, q.k);
    }
    return total;
}

extern "C" int ddgemm_batched(int count, const ddgemm_problem *probs_host,
                              const ddgemm_problem *probs_dev, void *workspace, size_t ws_bytes,
                              void *stream, const ddgemm_opts *opts,
                              const ddgemm_batch_config *config) {
    using namespace ddg;
    if (count < 0 || (count > 0 && (!probs_host || !probs_dev))) return DDGEMM_EINVAL;
    if (!batch_config_ok(config)) return DDGEMM_EINVAL;
    if (count == 0) return DDGEMM_OK;
    unsigned int *status = nullptr;
    if (opts) {
        if (opts->trans_a || opts->trans_b || opts->flags_dev ||
            (opts->variant != DDGEMM_VARIANT_FP64 && opts->variant != DDGEMM_VARIANT_INT8_TC &&
             opts->variant != DDGEMM_VARIANT_INT8_TC8))
            return DDGEMM_EUNSUPPORTED;
        status = opts->status_dev;
        if (opts->variant == DDGEMM_VARIANT_INT8_TC) {
            const int s = opts->int8_slices ? opts->int8_slices : INT8_TC_SLICES_DEFAULT;
            if (!int8_tc_slices_supported(s)) return DDGEMM_EINVAL;
            return run_batched_int8_tc(count, probs_host, probs_dev, workspace, ws_bytes,
                                       static_cast<cudaStream_t>(stream), s, INT8_TC_BITS,
                                       status, config, WaitPlan{}, opts->phase_events);
        }
        if (opts->variant == DDGEMM_VARIANT_INT8_TC8) {
            const int s = opts->int8_slices ? opts->int8_slices : INT8_TC8_SLICES_DEFAULT;
            if (!int8_tc8_slices_supported(s)) return DDGEMM_EINVAL;
            return run_batched_int8_tc(count, probs_host, probs_dev, workspace, ws_bytes,
                                       static_cast<cudaStream_t>(stream), s, INT8_BITS, status,
                                       config, WaitPlan{}, opts->phase_events);
        }
    }
    const int tile = config ? config->tile : DDGEMM_TILE_64x64;
    const int order = config ? config->order : DDGEMM_ORDER_LONGEST_K_FIRST;
    if (tile < 0 || tile > DDGEMM_TILE_32x32 || order < 0 || order > DDGEMM_ORDER_LONGEST_K_FIRST)
        return DDGEMM_EINVAL;
    long long total_a = 0, total_b = 0;
    for (int i = 0; i < count; ++i) {
        const ddgemm_problem &q = probs_host[i];
        if (!problem_ok(q)) return DDGEMM_EINVAL;
        if (q.m > 0 && q.n > 0 && q.k > 0) {
            const long long kb = (q.k + KC - 1) / KC;
            total_a += (long long)q.m * kb;
            total_b += kb * ((q.n + 63) / 64);
        }
    }
    const size_t need = ddgemm_batched_workspace_size(count, probs_host, opts);
    if (!workspace || ws_bytes < need || (uintptr_t)workspace % ALIGN) return DDGEMM_EWORKSPACE;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DDGEMM_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    void *const *events = opts ? opts->phase_events : nullptr;
    auto mark = [&](int i) {
        return !events || cudaEventRecord(static_cast<cudaEvent_t>(events[i]), s) == cudaSuccess;
    };
    int bm, bn;
    tile_shape(tile, bm, bn);
    if (!mark(0)) return DDGEMM_ECUDA;
    plan_kernel<<<1, 256, 0, s>>>(count, probs_dev, ws, order, bm, bn);
    if (cudaGetLastError() != cudaSuccess) return DDGEMM_ECUDA;
    if (total_a > 0) {
        const long long blocks = (total_a + 7) / 8;
        batched_split_a_kernel<<<(unsigned)(blocks < 8LL * sms ? blocks : 8LL * sms), 256, 0, s>>>(
            ws, status);
        batched_split_b_kernel<<<(unsigned)(total_b < 8LL * sms ? total_b : 8LL * sms), 256, 0,
                                 s>>>(ws, status);
        if (cudaGetLastError() != cudaSuccess) return DDGEMM_ECUDA;
    }
    if (!mark(1)) return DDGEMM_ECUDA;
    cudaError_t e;
    switch (tile) {
        case DDGEMM_TILE_32x64: e = launch_cascade<2, 2>(ws, sms, s); break;
        case DDGEMM_TILE_64x32: e = launch_cascade<4, 1>(ws, sms, s); break;
        case DDGEMM_TILE_32x32: e = launch_cascade<2, 1>(ws, sms, s); break;
        default: e = launch_cascade<4, 2>(ws, sms, s); break;
    }
    return e == cudaSuccess && mark(2) ? DDGEMM_OK : DDGEMM_ECUDA;
}

extern "C" int ddgemm_diag_batched_withheld_copy(int count, const ddgemm_problem *probs_host,
                                                 const ddgemm_problem *probs_dev, void *workspace,
                                                 size_t ws_bytes, void *stream,
                                                 const ddgemm_opts *opts, int cta, long long step,
                                                 unsigned long long limit_ns) {
    using namespace ddg;
    if (!opts || !opts->status_dev || count <= 0 || !probs_host || !probs_dev)
        return DDGEMM_EINVAL;
    if (cta < 0 || step < 0 || limit_ns < 1000ull || limit_ns > 10000000000ull)
        return DDGEMM_EINVAL;
    if (opts->trans_a || opts->trans_b || opts->flags_dev) return DDGEMM_EUNSUPPORTED;
    int bits, s;
    if (opts->variant == DDGEMM_VARIANT_INT8_TC) {
        bits = INT8_TC_BITS;
        s = opts->int8_slices ? opts->int8_slices : INT8_TC_SLICES_DEFAULT;
        if (!int8_tc_slices_supported(s)) return DDGEMM_EINVAL;
    } else if (opts->variant == DDGEMM_VARIANT_INT8_TC8) {
        bits = INT8_BITS;
        s = opts->int8_slices ? opts->int8_slices : INT8_TC8_SLICES_DEFAULT;
        if (!int8_tc8_slices_supported(s)) return DDGEMM_EINVAL;
    } else {
        return DDGEMM_EUNSUPPORTED;
    }
    WaitPlan wait;
    wait.limit_ns = limit_ns;
    wait.cta = cta;
    wait.step = step;
    return run_batched_int8_tc(count, probs_host, probs_dev, workspace, ws_bytes,
                               static_cast<cudaStream_t>(stream), s, bits, opts->status_dev,
                               nullptr, wait);
}
