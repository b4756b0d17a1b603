// ddgemm_noalloc: the cascade GEMM for callers that cannot allocate device
// memory.  The paper has no counterpart; this is a packaging of ddgemm().
//
// Some callers cannot call cudaMalloc or hand the library a workspace:
// code that runs while a stream is being captured into a CUDA graph (where
// an allocation is not allowed), plug-ins living inside a framework whose
// memory pool owns the whole GPU, latency-bound paths that cannot afford
// cudaMalloc's implicit device synchronisation, and foreign-language callers
// with no binding to a GPU allocator.  For them the scratch space lives in a
// file-scope __device__ array of DDGEMM_NOALLOC_SCRATCH_BYTES: every GPU that
// loads this library holds it until the process exits.
//
// In host code the array's name is only a host-side stand-in, not a device
// address, so its device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and cached.
#include <cuda_runtime.h>

#include <mutex>
#include <unordered_map>

#include "../../include/ddgemm.h"
#include "ddgemm_internal.h"

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[DDGEMM_NOALLOC_SCRATCH_BYTES];

std::mutex g_mutex;
std::unordered_map<int, void *> g_scratch_by_device;

// Device address of the scratch array on the current device, or nullptr.
void *scratch_for_current_device() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lock(g_mutex);
    auto it = g_scratch_by_device.find(dev);
    if (it != g_scratch_by_device.end()) return it->second;
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return nullptr;
    g_scratch_by_device.emplace(dev, ptr);
    return ptr;
}

}  // namespace

extern "C" int ddgemm_noalloc(int m, int n, int k, const double *A_hi, const double *A_lo,
                              int lda, const double *B_hi, const double *B_lo, int ldb,
                              double *C_hi, double *C_lo, int ldc, void *stream,
                              const ddgemm_opts *opts) {
    if (m < 0 || n < 0 || k < 0) return DDGEMM_EINVAL;
    // ddgemm() needs at least the base workspace; the rest of the array gives
    // it room for split-k partial sums when they fit
    const size_t need = ddg::base_workspace_size(m, n, k, opts);
    if (need > (size_t)DDGEMM_NOALLOC_SCRATCH_BYTES) return DDGEMM_EWORKSPACE;
    if (need == 0) {
        // empty problem or k = 0: ddgemm needs no workspace
        return ddgemm(m, n, k, A_hi, A_lo, lda, B_hi, B_lo, ldb, C_hi, C_lo, ldc, nullptr, 0,
                      stream, opts);
    }
    void *scratch = scratch_for_current_device();
    if (!scratch) return DDGEMM_ECUDA;
    // Nothing in the scratch needs clearing: the split kernels of this call
    // write every panel entry and block exponent that the cascade kernel of
    // this call reads (reads past k and n are outside the tensor maps and
    // come back as zeros).
    return ddgemm(m, n, k, A_hi, A_lo, lda, B_hi, B_lo, ldb, C_hi, C_lo, ldc, scratch,
                  (size_t)DDGEMM_NOALLOC_SCRATCH_BYTES, stream, opts);
}
