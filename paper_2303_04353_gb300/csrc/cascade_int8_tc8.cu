// The tcgen05 INT8 form with eight-bit pieces (DDGEMM_VARIANT_INT8_TC8): the
// digits of the mma.sync form (balanced base 256, |digit| <= 128, s <= 15,
// k-blocks of 8192), so the same fixed point (6 + 8 (s - 1) fraction bits)
// and accuracy, on the tcgen05 tensor cores.  The kernel is the seven-bit
// form's (cascade_int8_tc_core.cuh, see cascade_int8_tc.cu) with the width
// as a template argument.  An eight-bit product is at most 2^14, so an FP32
// accumulator stays exact over 64 entries (64 * 16 * 2^14 = 2^24): the
// tensor memory is read out four times as often as with seven-bit pieces.
#include "cascade_int8_tc_core.cuh"

namespace ddg {

cudaError_t launch_cascade_int8_tc8(const Int8TcArgs &a, cudaStream_t stream) {
    if (a.m <= 0 || a.n <= 0 || a.k <= 0) return cudaSuccess;
    if (a.bits != INT8_BITS) return cudaErrorInvalidValue;
    if ((uintptr_t)a.a_tiles % 16 || (uintptr_t)a.b_tiles % 16) return cudaErrorInvalidValue;
    switch (a.slices) {
        case 12: return launch_tc_single<12, INT8_BITS>(a, stream);
        case 13: return launch_tc_single<13, INT8_BITS>(a, stream);
        case 14: return launch_tc_single<14, INT8_BITS>(a, stream);
        case 15: return launch_tc_single<15, INT8_BITS>(a, stream);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ddg
