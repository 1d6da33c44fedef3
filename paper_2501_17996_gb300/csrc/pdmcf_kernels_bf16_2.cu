// Kernel instantiations: P = float (iterates), S = __nv_bfloat16 (storage of F), shape part 2.
#include "pdmcf_kernels.h"

namespace pdmcf {
void fill_bf16_2(KernelTable<float, __nv_bfloat16>& t) {
  fill_shape<float, __nv_bfloat16, 7>(t);
  fill_shape<float, __nv_bfloat16, 8>(t);
  fill_shape<float, __nv_bfloat16, 9>(t);
}
}  // namespace pdmcf
