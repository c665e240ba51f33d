// Instantiations of the batched forward kernel for programs that use at
// most 3 stack slots (template heights up to 4).
#include "kernels.cuh"

namespace gg {
const void* fwd_ptr_d3(int variant) { return fwd_table<3, false>(variant); }
}  // namespace gg
