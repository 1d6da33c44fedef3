// Kernel instantiations: P = float (iterates), S = __nv_bfloat16 (storage of F), shape part 3.
#include "pdmcf_kernels.h"

namespace pdmcf {
void fill_bf16_3(KernelTable<float, __nv_bfloat16>& t) {
  fill_shape<float, __nv_bfloat16, 10>(t);
  fill_shape<float, __nv_bfloat16, 11>(t);
}
}  // namespace pdmcf
