// Instantiations of the batched forward kernel for programs that use at
// most 7 stack slots (template heights 7 and 8), with the pow instructions.
#include "kernels.cuh"

namespace gg {
const void* fwd_ptr_d7_pow(int variant) { return fwd_table<7, true>(variant); }
}  // namespace gg
