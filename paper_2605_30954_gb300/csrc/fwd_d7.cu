// Instantiations of the batched forward kernel for programs that use at
// most 7 stack slots (template heights up to 8).
#include "kernels.cuh"

namespace gg {
const void* fwd_ptr_d7(int variant) {
  switch (variant) {
    case 0: return reinterpret_cast<const void*>(&fwd_kernel<7, 8, false, false>);
    case 1: return reinterpret_cast<const void*>(&fwd_kernel<7, 4, false, false>);
    case 2: return reinterpret_cast<const void*>(&fwd_kernel<7, 4, true, false>);
    case 3: return reinterpret_cast<const void*>(&fwd_kernel<7, 4, true, true>);
    default: return nullptr;
  }
}
}  // namespace gg
