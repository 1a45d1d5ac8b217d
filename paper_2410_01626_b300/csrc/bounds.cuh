// Index checks of the bounds-checked build (compiled with -DFMM_BOUNDS_CHECK into
// libfmmcph_checked.so).  FMM_IN(i, n) is 0 <= i < n and FMM_OK(c) is c.  A failed check records
// the source line of the first failure of this translation unit in a device word, and the caller
// skips the guarded access (it never returns early from code that a warp or a block runs
// together, so a failed check cannot leave a barrier or shuffle waiting).  fmm_status_word reads
// and clears the words (FMM_DEV_BOUNDS, and the file and line in fmm_last_error).  In the normal
// build both macros are the constant true and cost nothing.
#pragma once
#include <cuda_runtime.h>

#ifdef FMM_BOUNDS_CHECK
namespace {
__device__ int fmm_bc_line;  // first failing line in this translation unit, 0 = none
__device__ __forceinline__ bool fmm_bc(bool ok, int line) {
    if (!ok) atomicCAS(&fmm_bc_line, 0, line);
    return ok;
}
}  // namespace
#define FMM_IN(i, n) fmm_bc((long long)(i) >= 0 && (long long)(i) < (long long)(n), __LINE__)
#define FMM_OK(c) fmm_bc((c), __LINE__)
// host: the line this translation unit recorded (0 = none), clearing it
#define FMM_BC_TAKE(fn)                                                   \
    int fn() {                                                            \
        int v = 0;                                                        \
        if (cudaMemcpyFromSymbol(&v, fmm_bc_line, sizeof v) != cudaSuccess) { \
            cudaGetLastError();                                           \
            return 0;                                                     \
        }                                                                 \
        if (v) {                                                          \
            const int z = 0;                                              \
            cudaMemcpyToSymbol(fmm_bc_line, &z, sizeof z);                \
        }                                                                 \
        return v;                                                         \
    }
#else
#define FMM_IN(i, n) true
#define FMM_OK(c) true
#define FMM_BC_TAKE(fn) \
    int fn() { return 0; }
#endif
