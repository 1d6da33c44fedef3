// Kernel instantiations: P = float (iterates), S = __nv_bfloat16 (storage of F), shape part 1.
#include "pdmcf_kernels.h"

namespace pdmcf {
void fill_bf16_1(KernelTable<float, __nv_bfloat16>& t) {
  fill_shape<float, __nv_bfloat16, 4>(t);
  fill_shape<float, __nv_bfloat16, 5>(t);
  fill_shape<float, __nv_bfloat16, 6>(t);
}
}  // namespace pdmcf
