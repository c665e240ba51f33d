// Instantiations of the batched forward kernel for programs that use at
// most 7 stack slots (template heights 7 and 8).
#include "kernels.cuh"

namespace gg {
const void* fwd_ptr_d7(int variant) { return fwd_table<7, false>(variant); }
}  // namespace gg
