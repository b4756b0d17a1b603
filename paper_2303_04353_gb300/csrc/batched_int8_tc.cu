// Many FP64x2 GEMMs of uneven shapes with the INT8 form on the tcgen05
// tensor cores, in four launches: a plan, the block exponents of every A
// (one warp per row and k-block) and of every B (one CTA per 64 columns
// and k-block) in one launch, the tiled bf16 digits of every A and B (one
// CTA per 32 x 64 input tile), and one persistent tcgen05 kernel that walks the planned list
// of (problem, 128 x 16 tile) items in the configured order (longest k
// first unless ddgemm_batch_config says otherwise).  The paper has no
// batched form; this is the tcgen05 INT8 form (cascade_int8_tc.cu) scheduled
// for many small problems at once, with seven- or eight-bit pieces.  Every
// unit runs the single-problem form's device code on that problem's data,
// so each C is bit-identical to what ddgemm() computes for it with
// DDGEMM_VARIANT_INT8_TC (or DDGEMM_VARIANT_INT8_TC8).
//
// Everything the kernels need is computed on the device from the caller's
// device copy of the problem list (the host copy only sizes the launches),
// so the call can be captured into a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>

#include "../../include/ddgemm.h"
#include "cascade_int8_tc_core.cuh"
#include "split_int8_device.cuh"

namespace ddg {
namespace {

constexpr size_t TC_ALIGN = 256;

__host__ __device__ inline size_t ru_tc(size_t x, size_t a) { return (x + a - 1) / a * a; }

// One problem as the kernels see it.  trans: the tile grid covers C^T =
// B^T A^T (B's columns are the 128-row side, A's rows the 16-column side),
// chosen when that needs fewer tiles; every diagonal sum, so every bit of C,
// is the same either way (each is a sum over the same digit products).
struct TcEntry {
    int m, n, k, kb8, lda, ldb, trans;
    long long ldc;
    const double *a_hi, *a_lo, *b_hi, *b_lo;
    double *c_hi, *c_lo;
    uint16_t *a_tiles, *b_tiles;
    int *e_a, *e_b;
    // the same seen from the tile grid (swapped when trans): its rows and
    // columns, the digits and exponents of its row side and column side
    int g_m, g_n;
    const uint16_t *g_a_tiles, *g_b_tiles;
    const int *g_e_a, *g_e_b;
    int tiles_n;
    long long tiles;
    long long ea_units, eb_units, da_units, db_units;
};

struct TcHeader {
    long long total_tiles, total_ea, total_eb, total_d;
    int count;
    int kblk;                  // k-block of the digit width (8192 or 16384)
    unsigned int *status;
    unsigned long long next_d;   // the digit kernel's unit counter (the plan zeroes it)
    unsigned long long next_eb;  // the same for the exponents of B
};

// Workspace: [header][entries][order][tile prefix][4 unit prefixes] | digits
struct TcPlanLayout {
    size_t entries, order, tile_pre, ea_pre, eb_pre, da_pre, db_pre, data;
};

__host__ __device__ inline TcPlanLayout tc_plan_layout(int count) {
    TcPlanLayout L;
    const size_t pre = (size_t)(count + 1) * sizeof(long long);
    L.entries = ru_tc(sizeof(TcHeader), TC_ALIGN);
    L.order = ru_tc(L.entries + (size_t)count * sizeof(TcEntry), TC_ALIGN);
    L.tile_pre = ru_tc(L.order + (size_t)count * sizeof(int), TC_ALIGN);
    L.ea_pre = ru_tc(L.tile_pre + pre, TC_ALIGN);
    L.eb_pre = ru_tc(L.ea_pre + pre, TC_ALIGN);
    L.da_pre = ru_tc(L.eb_pre + pre, TC_ALIGN);
    L.db_pre = ru_tc(L.da_pre + pre, TC_ALIGN);
    L.data = ru_tc(L.db_pre + pre, TC_ALIGN);
    return L;
}

// Tiles of 128 x 16 over C (m x n), or over C^T (n x m) when transposed.
__host__ __device__ inline long long tc_tiles(int m, int n, bool trans) {
    const int rows = trans ? n : m, cols = trans ? m : n;
    return (long long)((rows + INT8_TC_BM - 1) / INT8_TC_BM) *
           ((cols + INT8_TC_BN - 1) / INT8_TC_BN);
}

// The orientation with fewer tiles (ties: as given).
__host__ __device__ inline bool tc_trans(int m, int n) {
    return tc_tiles(m, n, true) < tc_tiles(m, n, false);
}

// Tile heights of A's rows and B's columns in the digit order.
__host__ __device__ inline int tc_th_a(bool trans) { return trans ? INT8_TC_BN : INT8_TC_BM; }
__host__ __device__ inline int tc_th_b(bool trans) { return trans ? INT8_TC_BM : INT8_TC_BN; }

// Digit and exponent bytes of one problem (the single-problem layout, with
// the tile heights of the orientation tr).
__host__ __device__ inline size_t tc_problem_bytes(int m, int n, int k, int slices, int kblk,
                                                   bool tr) {
    if (m <= 0 || n <= 0 || k <= 0) return 0;
    const size_t kpad = ru_tc((size_t)k, 16), kb8 = (size_t)(k + kblk - 1) / kblk;
    return ru_tc((size_t)slices * ru_tc((size_t)m, tc_th_a(tr)) * kpad * 2, TC_ALIGN) +
           ru_tc((size_t)slices * ru_tc((size_t)n, tc_th_b(tr)) * kpad * 2, TC_ALIGN) +
           ru_tc(kb8 * m * 4, TC_ALIGN) + ru_tc(kb8 * n * 4, TC_ALIGN);
}

__device__ inline int find_tc(const long long *prefix, int count, long long u) {
    int lo = 0, hi = count;  // prefix[lo] <= u < prefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= u) lo = mid; else hi = mid;
    }
    return lo;
}

// The same search for a caller that visits units in increasing order:
// from its previous answer `i` it gallops forward (a few steps when the next
// unit is near), falling back to the full search if u lies before it.
__device__ inline int advance_tc(const long long *prefix, int count, long long u, int i) {
    if (prefix[i] > u) return find_tc(prefix, count, u);
    int lo = i, step = 1, hi;
    for (;;) {
        hi = lo + step;
        if (hi >= count) {
            hi = count;  // prefix[count] = total > u
            break;
        }
        if (prefix[hi] > u) break;
        lo = hi;
        step <<= 1;
    }
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= u) lo = mid; else hi = mid;
    }
    return lo;
}

// Longest k first, then larger m n, then index (false for a = b).  Without
// branches: every lane of the plan's rank loop compares against another
// problem, and branches on the keys diverged and made that loop the plan's
// slowest phase.
__device__ inline bool before_tc(int ka, long long sa, int ia, int kb, long long sb, int ib) {
    return (ka > kb) | ((ka == kb) & ((sa > sb) | ((sa == sb) & (ia < ib))));
}

// Problems whose ordering keys the plan kernel keeps in shared memory.
constexpr int PLAN_SMEM_KEYS = 2048;

// order: DDGEMM_ORDER_* (the rank of a problem in the tile list); orient:
// DDGEMM_ORIENT_* (whether a problem's grid may cover C^T).
__global__ void __launch_bounds__(256)
tc_plan_kernel(int count, const ddgemm_problem *__restrict__ probs, char *ws, int slices,
               int kblk, unsigned int *status, int order_rule, int orient) {
    const TcPlanLayout L = tc_plan_layout(count);
    TcHeader *hdr = reinterpret_cast<TcHeader *>(ws);
    TcEntry *ent = reinterpret_cast<TcEntry *>(ws + L.entries);
    int *order = reinterpret_cast<int *>(ws + L.order);
    long long *tile_pre = reinterpret_cast<long long *>(ws + L.tile_pre);
    long long *ea_pre = reinterpret_cast<long long *>(ws + L.ea_pre);
    long long *eb_pre = reinterpret_cast<long long *>(ws + L.eb_pre);
    long long *da_pre = reinterpret_cast<long long *>(ws + L.da_pre);
    long long *db_pre = reinterpret_cast<long long *>(ws + L.db_pre);
    // the ordering keys (k, m n) in shared memory when they fit: the rank of
    // a problem compares it with every other one
    __shared__ int key_k[PLAN_SMEM_KEYS];
    __shared__ long long key_mn[PLAN_SMEM_KEYS];
    const bool keys_in_smem = count <= PLAN_SMEM_KEYS;
    if (keys_in_smem) {
        for (int i = threadIdx.x; i < count; i += blockDim.x) {
            key_k[i] = probs[i].k;
            key_mn[i] = (long long)probs[i].m * probs[i].n;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        const ddgemm_problem q = probs[i];
        TcEntry e;
        e.m = q.m; e.n = q.n; e.k = q.k;
        e.kb8 = q.k > 0 ? (q.k + kblk - 1) / kblk : 0;
        e.lda = q.lda; e.ldb = q.ldb; e.ldc = q.ldc;
        e.a_hi = q.A_hi; e.a_lo = q.A_lo; e.b_hi = q.B_hi; e.b_lo = q.B_lo;
        e.c_hi = q.C_hi; e.c_lo = q.C_lo;
        const bool mn = q.m > 0 && q.n > 0, work = mn && q.k > 0;
        e.trans = mn && orient == DDGEMM_ORIENT_FEWER_TILES && tc_trans(q.m, q.n);
        e.tiles_n = mn ? ((e.trans ? q.m : q.n) + INT8_TC_BN - 1) / INT8_TC_BN : 0;
        e.tiles = mn ? tc_tiles(q.m, q.n, e.trans) : 0;
        const long long ktiles = work ? (q.k + split8::TK - 1) / split8::TK : 0;
        e.ea_units = work ? (long long)q.m * e.kb8 : 0;
        e.eb_units = work ? (long long)((q.n + 63) / 64) * e.kb8 : 0;
        e.da_units = work ? (long long)((q.m + split8::TV - 1) / split8::TV) * ktiles : 0;
        e.db_units = work ? (long long)((q.n + split8::TV - 1) / split8::TV) * ktiles : 0;
        ent[i] = e;
        const long long qmn = (long long)q.m * q.n;
        int r = i;  // DDGEMM_ORDER_GIVEN
        if (order_rule == DDGEMM_ORDER_LONGEST_K_FIRST) {
            r = 0;
            if (keys_in_smem) {
#pragma unroll 4
                for (int j = 0; j < count; ++j)
                    r += before_tc(key_k[j], key_mn[j], j, q.k, qmn, i);
            } else {
                for (int j = 0; j < count; ++j)
                    r += before_tc(probs[j].k, (long long)probs[j].m * probs[j].n, j, q.k, qmn, i);
            }
        }
        order[r] = i;
    }
    __syncthreads();
    // Prefix sums over the problems (units, workspace bytes) and over the
    // ranks (tiles): thread t takes a contiguous segment, the 256 segment
    // totals are scanned by one warp per quantity, then every thread walks
    // its segment again from its offsets.
    constexpr int NQ = 6;  // ea, eb, da, db units; bytes; tiles (rank order)
    __shared__ long long part[NQ][256];  // blockDim.x <= 256
    const int nt = blockDim.x, t = threadIdx.x;
    const int seg = (count + nt - 1) / nt;
    const int i0 = min(count, t * seg), i1 = min(count, i0 + seg);
    auto bytes_of = [&](const TcEntry &e) -> size_t {
        if (e.ea_units <= 0) return 0;
        return tc_problem_bytes(e.m, e.n, e.k, slices, kblk, e.trans != 0);
    };
    {
        long long acc[NQ] = {0, 0, 0, 0, 0, 0};
        for (int i = i0; i < i1; ++i) {
            const TcEntry &e = ent[i];
            acc[0] += e.ea_units;
            acc[1] += e.eb_units;
            acc[2] += e.da_units;
            acc[3] += e.db_units;
            acc[4] += (long long)bytes_of(e);
            acc[5] += ent[order[i]].tiles;
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
        long long ta = part[0][t], tb = part[1][t], tda = part[2][t],
                  tdb = part[3][t], tt = part[5][t];
        size_t off = L.data + (size_t)part[4][t];
        for (int i = i0; i < i1; ++i) {
            TcEntry &e = ent[i];
            ea_pre[i] = ta;
            eb_pre[i] = tb;
            da_pre[i] = tda;
            db_pre[i] = tdb;
            ta += e.ea_units;
            tb += e.eb_units;
            tda += e.da_units;
            tdb += e.db_units;
            e.a_tiles = e.b_tiles = nullptr;
            e.e_a = e.e_b = nullptr;
            if (e.ea_units > 0) {
                const size_t kpad = ru_tc((size_t)e.k, 16);
                e.a_tiles = reinterpret_cast<uint16_t *>(ws + off);
                off += ru_tc((size_t)slices * ru_tc((size_t)e.m, tc_th_a(e.trans)) * kpad * 2,
                             TC_ALIGN);
                e.b_tiles = reinterpret_cast<uint16_t *>(ws + off);
                off += ru_tc((size_t)slices * ru_tc((size_t)e.n, tc_th_b(e.trans)) * kpad * 2,
                             TC_ALIGN);
                e.e_a = reinterpret_cast<int *>(ws + off);
                off += ru_tc((size_t)e.kb8 * e.m * 4, TC_ALIGN);
                e.e_b = reinterpret_cast<int *>(ws + off);
                off += ru_tc((size_t)e.kb8 * e.n * 4, TC_ALIGN);
            }
            e.g_m = e.trans ? e.n : e.m;
            e.g_n = e.trans ? e.m : e.n;
            e.g_a_tiles = e.trans ? e.b_tiles : e.a_tiles;
            e.g_b_tiles = e.trans ? e.a_tiles : e.b_tiles;
            e.g_e_a = e.trans ? e.e_b : e.e_a;
            e.g_e_b = e.trans ? e.e_a : e.e_b;
            tile_pre[i] = tt;
            tt += ent[order[i]].tiles;
        }
        if (i1 == count && i0 < i1) {  // the last non-empty segment: the totals
            ea_pre[count] = ta;
            eb_pre[count] = tb;
            da_pre[count] = tda;
            db_pre[count] = tdb;
            tile_pre[count] = tt;
            hdr->total_tiles = tt;
            hdr->total_ea = ta;
            hdr->total_eb = tb;
            hdr->total_d = tda + tdb;
            hdr->count = count;
            hdr->kblk = kblk;
            hdr->status = status;
            hdr->next_d = 0;
            hdr->next_eb = 0;
        }
    }
}

struct TcView {
    const TcHeader *hdr;
    const TcEntry *ent;
    const int *order;
    const long long *tile_pre, *ea_pre, *eb_pre, *da_pre, *db_pre;
    __device__ explicit TcView(const char *ws) {
        hdr = reinterpret_cast<const TcHeader *>(ws);
        const TcPlanLayout L = tc_plan_layout(hdr->count);
        ent = reinterpret_cast<const TcEntry *>(ws + L.entries);
        order = reinterpret_cast<const int *>(ws + L.order);
        tile_pre = reinterpret_cast<const long long *>(ws + L.tile_pre);
        ea_pre = reinterpret_cast<const long long *>(ws + L.ea_pre);
        eb_pre = reinterpret_cast<const long long *>(ws + L.eb_pre);
        da_pre = reinterpret_cast<const long long *>(ws + L.da_pre);
        db_pre = reinterpret_cast<const long long *>(ws + L.db_pre);
    }
};

// The exponents of every A and every B in one launch: CTAs [0, blocks_a)
// take A's units, the others B's, so that the two latency-bound halves
// overlap instead of running one after the other.
//   A: one warp per (problem, row, k-block).  Neighbouring warps take
//   neighbouring chunks of units (a contiguous run per warp measured
//   slower: the runs differ in length of rows); a search of the unit prefix
//   serves a chunk's units, mostly rows of one problem.
//   B: one CTA per (problem, 64 columns, k-block), taken from a counter.
constexpr int EA_CHUNK = 8;
__global__ void __launch_bounds__(256) tc_exps_kernel(const char *ws, int blocks_a) {
    __shared__ unsigned long long part[4][64];
    const TcView V(ws);
    const int count = V.hdr->count, kblk = V.hdr->kblk;
    int i = 0;
    if ((int)blockIdx.x < blocks_a) {
        const int lane = threadIdx.x & 31;
        const long long total = V.hdr->total_ea;
        const long long nw = ((long long)blocks_a * blockDim.x) >> 5;
        for (long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
             c * EA_CHUNK < total; c += nw) {
            const long long u1 =
                c * EA_CHUNK + EA_CHUNK < total ? c * EA_CHUNK + EA_CHUNK : total;
            for (long long u = c * EA_CHUNK; u < u1; ++u) {
                i = advance_tc(V.ea_pre, count, u, i);
                const TcEntry &e = V.ent[i];
                const int local = (int)(u - V.ea_pre[i]);
                const int row = e.kb8 == 1 ? local : local / e.kb8;
                split8::exps_contig_unit(lane, row, local - row * e.kb8, e.m, e.k, kblk, e.a_hi,
                                         e.lda, e.e_a);
            }
        }
    } else {
        // B's units (of uneven size: k rows each) from a counter
        __shared__ long long s_next;
        for (;;) {
            __syncthreads();  // every thread has read s_next
            if (threadIdx.x == 0)
                s_next = (long long)atomicAdd(const_cast<unsigned long long *>(&V.hdr->next_eb),
                                              1ull);
            __syncthreads();
            const long long u = s_next;
            if (u >= V.hdr->total_eb) break;
            i = advance_tc(V.eb_pre, count, u, i);
            const TcEntry &e = V.ent[i];
            const long long local = u - V.eb_pre[i];
            const int vtiles = (e.n + 63) / 64;
            split8::exps_strided_unit<4>((int)(local % vtiles), (int)(local / vtiles), e.n, e.k,
                                         kblk, e.b_hi, e.ldb, e.e_b, part);
        }
    }
}

// Digits of every A, then of every B: one CTA per 32 x 64 input tile.
constexpr int DIGIT_CHUNK = 1;
template <int S, int BITS>
__global__ void __launch_bounds__(256, 4) tc_digits_kernel(const char *ws) {
    __shared__ double sh[split8::TV][split8::TK + 1];
    __shared__ double sl[split8::TV][split8::TK + 1];
    const TcView V(ws);
    const int count = V.hdr->count;
    const long long total_a = V.da_pre[count];
    unsigned int *status = V.hdr->status;
    // CTAs take chunks of DIGIT_CHUNK consecutive units from a counter, so
    // that units of uneven cost (ragged tiles) do not leave some CTAs with
    // the last of the work; chunks come in increasing order, so each CTA's
    // problem lookups gallop forward (one unit per chunk measured best: 1.73
    // ms for plan and split against 1.73, 1.75 and 1.78 for 2, 4 and 8)
    const long long total = V.hdr->total_d;
    __shared__ long long s_next;
    int ia = 0, ib = 0;
    for (;;) {
        __syncthreads();  // every thread has read s_next and is done with sh, sl
        if (threadIdx.x == 0)
            s_next = (long long)atomicAdd(const_cast<unsigned long long *>(&V.hdr->next_d),
                                          (unsigned long long)DIGIT_CHUNK);
        __syncthreads();
        const long long u0 = s_next;
        if (u0 >= total) break;
        const long long u1 = u0 + DIGIT_CHUNK < total ? u0 + DIGIT_CHUNK : total;
        for (long long u = u0; u < u1; ++u) {
            if (u > u0) __syncthreads();  // the previous unit is done with sh, sl
            if (u < total_a) {
                const int i = ia = advance_tc(V.da_pre, count, u, ia);
                const TcEntry &e = V.ent[i];
                const long long local = u - V.da_pre[i];
                const int ktiles = (e.k + split8::TK - 1) / split8::TK;
                split8::digits_unit<S, true, true, BITS>((int)(local / ktiles) * split8::TV,
                                                         (int)(local % ktiles) * split8::TK, e.m,
                                                         e.k, e.a_hi, e.a_lo, e.lda, e.a_tiles, 0,
                                                         tc_th_a(e.trans), e.e_a, status, sh, sl);
            } else {
                const long long ub = u - total_a;
                const int i = ib = advance_tc(V.db_pre, count, ub, ib);
                const TcEntry &e = V.ent[i];
                const long long local = ub - V.db_pre[i];
                const int ktiles = (e.k + split8::TK - 1) / split8::TK;
                split8::digits_unit<S, false, true, BITS>((int)(local / ktiles) * split8::TV,
                                                          (int)(local % ktiles) * split8::TK, e.n,
                                                          e.k, e.b_hi, e.b_lo, e.ldb, e.b_tiles, 0,
                                                          tc_th_b(e.trans), e.e_b, status, sh, sl);
            }
        }
    }
}

// The planned (problem, tile) items in the plan's problem order; within a
// problem the tiles go in groups of row_group row tiles.
struct BatchSource {
    const char *ws;
    int row_group;  // row tiles per group of a problem's tile order
    WaitPlan plan;
    __device__ long long items() const {
        return reinterpret_cast<const TcHeader *>(ws)->total_tiles;
    }
    __device__ unsigned int *status() const {
        return reinterpret_cast<const TcHeader *>(ws)->status;
    }
    __device__ const WaitPlan &wait() const { return plan; }
    // hint: the rank of the caller's previous item (items come in
    // increasing order)
    __device__ TcJob job(long long item, int &hint) const {
        const TcView V(ws);
        const int r = hint = advance_tc(V.tile_pre, V.hdr->count, item, hint);
        const TcEntry &e = V.ent[V.order[r]];
        const long long local = item - V.tile_pre[r];
        TcJob j;
        // transposed: the grid's rows are B's columns, its columns A's rows
        j.m = e.g_m;
        j.n = e.g_n;
        j.k = e.k;
        int tm, tn;
        grouped_tile((unsigned)local, (j.m + BM - 1) / BM, e.tiles_n, row_group, tm, tn);
        j.tm = tm;
        j.tn_load = tn;
        j.col0 = tn * BN;
        j.a_tiles = e.g_a_tiles;
        j.b_tiles = e.g_b_tiles;
        j.exp_a = e.g_e_a;
        j.exp_b = e.g_e_b;
        j.c_hi = e.c_hi;
        j.c_lo = e.c_lo;
        j.ldc = e.ldc;
        j.trans = e.trans != 0;
        return j;
    }
};

template <int S, int BITS, int PLANES>
cudaError_t launch_batched_tc(char *ws, long long tiles, long long units_ea, long long units_eb,
                              long long units_d, int sms, cudaStream_t s, int row_group,
                              const WaitPlan &wait, void *const *events) {
    const long long cap = 8LL * sms;
    const long long ba = std::min(cap, (units_ea + 8 * EA_CHUNK - 1) / (8 * EA_CHUNK)),
                    bb = std::min(cap, units_eb);
    if (ba + bb > 0) tc_exps_kernel<<<(unsigned)(ba + bb), 256, 0, s>>>(ws, (int)ba);
    if (units_d > 0)
        tc_digits_kernel<S, BITS><<<(unsigned)(units_d < cap ? units_d : cap), 256, 0, s>>>(ws);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && events)
        e = cudaEventRecord(static_cast<cudaEvent_t>(events[1]), s);
    if (e != cudaSuccess) return e;
    if (tiles == 0)
        return events ? cudaEventRecord(static_cast<cudaEvent_t>(events[2]), s) : cudaSuccess;
    using G = TcGeom<S>;
    auto kernel = cascade_int8_tc_kernel<S, BITS, BatchSource, PLANES>;
    if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)G::SMEM)) != cudaSuccess)
        return e;
    const int grid = (int)(tiles < sms ? tiles : sms);
    BatchSource src{ws, row_group, wait};
    kernel<<<grid, NTHREADS, G::SMEM, s>>>(src);
    e = cudaGetLastError();
    if (e == cudaSuccess && events) e = cudaEventRecord(static_cast<cudaEvent_t>(events[2]), s);
    return e;
}

bool tc_problem_ok(const ddgemm_problem &q) {
    if (q.m < 0 || q.n < 0 || q.k < 0) return false;
    if (q.m > 0 && q.n > 0) {
        if (!q.C_hi || !q.C_lo || q.ldc < q.n) return false;
        if (q.k > 0 && (!q.A_hi || !q.A_lo || !q.B_hi || !q.B_lo || q.lda < q.k || q.ldb < q.n))
            return false;
    }
    return true;
}

}  // namespace

size_t batched_int8_tc_workspace_size(int count, const ddgemm_problem *probs_host, int slices,
                                      int bits) {
    if (count <= 0 || !probs_host) return 0;
    const int kblk = kblock_of_bits(bits);
    size_t total = tc_plan_layout(count).data;
    // room for either orientation, so that one workspace serves every config
    for (int i = 0; i < count; ++i) {
        const ddgemm_problem &q = probs_host[i];
        const size_t a = tc_problem_bytes(q.m, q.n, q.k, slices, kblk, false);
        const size_t b = tc_problem_bytes(q.m, q.n, q.k, slices, kblk, true);
        total += a > b ? a : b;
    }
    return total;
}

int run_batched_int8_tc(int count, const ddgemm_problem *probs_host,
                        const ddgemm_problem *probs_dev, void *workspace, size_t ws_bytes,
                        cudaStream_t s, int slices, int bits, unsigned int *status,
                        const ddgemm_batch_config *config, const WaitPlan &wait,
                        void *const *events) {
    if (bits != INT8_TC_BITS && bits != INT8_BITS) return DDGEMM_EINVAL;
    if (bits == INT8_BITS && slices > 15) return DDGEMM_EINVAL;
    const int kblk = kblock_of_bits(bits);
    const int order_rule = config ? config->order : DDGEMM_ORDER_LONGEST_K_FIRST;
    const int orient = config ? config->orient : DDGEMM_ORIENT_FEWER_TILES;
    const int planes = config ? config->planes : DDGEMM_PLANES_INTERLEAVED;
    const int row_group = config && config->row_group ? config->row_group : TILE_GROUP;
    long long tiles = 0, ea = 0, eb = 0, d = 0;
    for (int i = 0; i < count; ++i) {
        const ddgemm_problem &q = probs_host[i];
        if (!tc_problem_ok(q)) return DDGEMM_EINVAL;
        if (q.m > 0 && q.n > 0) {
            tiles += tc_tiles(q.m, q.n,
                              orient == DDGEMM_ORIENT_FEWER_TILES && tc_trans(q.m, q.n));
            if (q.k > 0) {
                const long long kb8 = (q.k + kblk - 1) / kblk,
                                kt = (q.k + split8::TK - 1) / split8::TK;
                ea += (long long)q.m * kb8;
                eb += (long long)((q.n + 63) / 64) * kb8;
                d += (long long)((q.m + split8::TV - 1) / split8::TV) * kt +
                     (long long)((q.n + split8::TV - 1) / split8::TV) * kt;
            }
        }
    }
    const size_t need = batched_int8_tc_workspace_size(count, probs_host, slices, bits);
    if (!workspace || ws_bytes < need || (uintptr_t)workspace % TC_ALIGN) return DDGEMM_EWORKSPACE;
    if (tiles > 0x7fffffffLL) return DDGEMM_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DDGEMM_ECUDA;
    char *ws = static_cast<char *>(workspace);
    if (events && cudaEventRecord(static_cast<cudaEvent_t>(events[0]), s) != cudaSuccess)
        return DDGEMM_ECUDA;
    tc_plan_kernel<<<1, 256, 0, s>>>(count, probs_dev, ws, slices, kblk, status, order_rule,
                                     orient);
    if (cudaGetLastError() != cudaSuccess) return DDGEMM_ECUDA;
    cudaError_t e;
#define DDG_TC(S, B)                                                                     \
    (planes == DDGEMM_PLANES_ASCENDING                                                   \
         ? launch_batched_tc<S, B, 1>(ws, tiles, ea, eb, d, sms, s, row_group, wait, events) \
         : launch_batched_tc<S, B, 0>(ws, tiles, ea, eb, d, sms, s, row_group, wait, events))
    if (bits == INT8_BITS) {
        switch (slices) {
            case 12: e = DDG_TC(12, INT8_BITS); break;
            case 13: e = DDG_TC(13, INT8_BITS); break;
            case 14: e = DDG_TC(14, INT8_BITS); break;
            case 15: e = DDG_TC(15, INT8_BITS); break;
            default: return DDGEMM_EINVAL;
        }
    } else {
        switch (slices) {
            case 12: e = DDG_TC(12, INT8_TC_BITS); break;
            case 13: e = DDG_TC(13, INT8_TC_BITS); break;
            case 14: e = DDG_TC(14, INT8_TC_BITS); break;
            case 15: e = DDG_TC(15, INT8_TC_BITS); break;
            case 16: e = DDG_TC(16, INT8_TC_BITS); break;
            default: return DDGEMM_EINVAL;
        }
    }
#undef DDG_TC
    return e == cudaSuccess ? DDGEMM_OK : DDGEMM_ECUDA;
}

}  // namespace ddg
