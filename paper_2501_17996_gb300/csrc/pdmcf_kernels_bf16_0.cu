// Kernel instantiations: P = float (iterates), S = __nv_bfloat16 (storage of F), shape part 0.
#include "pdmcf_kernels.h"

namespace pdmcf {
void fill_bf16_0(KernelTable<float, __nv_bfloat16>& t) {
  fill_shape<float, __nv_bfloat16, 0>(t);
  fill_shape<float, __nv_bfloat16, 1>(t);
  fill_shape<float, __nv_bfloat16, 2>(t);
  fill_shape<float, __nv_bfloat16, 3>(t);
}
}  // namespace pdmcf
