// Device-side bounds checks of the SP_DEBUG build (compile with -DSP_DEBUG; the library built
// that way is libsvdphat_debug.so).  A failed check sets bit kDebugBit of the device status word
// (sp_check_status then returns SP_EBOUNDS) and the guarded access is skipped, so a bad index
// is reported instead of faulting.  In the release build every check compiles away.
#pragma once

namespace sp {

constexpr int kDebugBit = 0x100;

#ifdef SP_DEBUG
// true when cond holds; otherwise records the failure and returns false
__device__ __forceinline__ bool dcheck(bool cond, int *status) {
    if (!cond) atomicOr(status, kDebugBit);
    return cond;
}
#else
__device__ __forceinline__ constexpr bool dcheck(bool, int *) { return true; }
#endif

}  // namespace sp
