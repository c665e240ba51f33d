// Instantiations of the batched forward kernel for programs that use at
// most 3 stack slots (template heights up to 4).
#include "kernels.cuh"

namespace gg {
const void* fwd_ptr_d3(int variant) {
  switch (variant) {
    case 0: return reinterpret_cast<const void*>(&fwd_kernel<3, 8, false, false, 1>);
    case 1: return reinterpret_cast<const void*>(&fwd_kernel<3, 4, false, false, 1>);
    case 2: return reinterpret_cast<const void*>(&fwd_kernel<3, 4, true, false, 1>);
    case 3: return reinterpret_cast<const void*>(&fwd_kernel<3, 4, true, true, 1>);
    case 4: return reinterpret_cast<const void*>(&fwd_kernel<3, 8, false, false, 2>);
    case 5: return reinterpret_cast<const void*>(&fwd_kernel<3, 4, false, false, 2>);
    case 6: return reinterpret_cast<const void*>(&fwd_kernel<3, 4, true, false, 2>);
    default: return nullptr;
  }
}
}  // namespace gg
