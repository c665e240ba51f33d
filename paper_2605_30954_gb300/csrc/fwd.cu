// Instantiations of the batched forward kernel.
#include "kernels.cuh"

namespace gg {
const void* fwd_ptr_plain(int variant) { return fwd_table<false>(variant); }
}  // namespace gg
