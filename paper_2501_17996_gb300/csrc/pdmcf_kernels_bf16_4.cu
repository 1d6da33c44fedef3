// Kernel instantiations: P = float (iterates), S = __nv_bfloat16 (storage of F), shape part 4.
#include "pdmcf_kernels.h"

namespace pdmcf {
void fill_bf16_4(KernelTable<float, __nv_bfloat16>& t) {
  fill_shape<float, __nv_bfloat16, 12>(t);
  fill_shape<float, __nv_bfloat16, 13>(t);
}
}  // namespace pdmcf
