// Instantiations of the batched forward kernel, with the pow instructions.
#include "kernels.cuh"

namespace gg {
const void* fwd_ptr_pow(int variant) { return fwd_table<true>(variant); }
}  // namespace gg
