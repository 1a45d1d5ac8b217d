// M2L on the 5th-generation tensor cores (tcgen05, TF32) -- placeholder until the kernel lands.
#include "fmm_internal.h"

namespace fmmcph {

bool m2l_tc_supported(const Handle*) { return false; }
void launch_m2l_tc(Handle*, cudaStream_t) {}

}  // namespace fmmcph
