// Kernel instantiations: P = float (iterates), S = float (storage of F), shape part 1.
#include "pdmcf_kernels.h"

namespace pdmcf {
void fill_f32_1(KernelTable<float, float>& t) {
  fill_shape<float, float, 4>(t);
  fill_shape<float, float, 5>(t);
  fill_shape<float, float, 6>(t);
}
}  // namespace pdmcf
