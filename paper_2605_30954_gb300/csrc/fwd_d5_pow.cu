// Instantiations of the batched forward kernel for programs that use at
// most 5 stack slots (template heights 5 and 6), with the pow instructions.
#include "kernels.cuh"

namespace gg {
const void* fwd_ptr_d5_pow(int variant) { return fwd_table<5, true>(variant); }
}  // namespace gg
