// Instantiations of the batched forward kernel for programs that use at
// most 3 stack slots (template heights up to 4), with the pow instructions.
#include "kernels.cuh"

namespace gg {
const void* fwd_ptr_d3_pow(int variant) { return fwd_table<3, true>(variant); }
}  // namespace gg
