// Instantiations of the batched forward kernel for programs that use at
// most 5 stack slots (template heights 5 and 6).
#include "kernels.cuh"

namespace gg {
const void* fwd_ptr_d5(int variant) { return fwd_table<5, false>(variant); }
}  // namespace gg
