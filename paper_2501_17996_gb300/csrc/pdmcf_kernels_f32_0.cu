// Kernel instantiations: P = float (iterates), S = float (storage of F), shape part 0.
#include "pdmcf_kernels.h"

namespace pdmcf {
void fill_f32_0(KernelTable<float, float>& t) {
  fill_shape<float, float, 0>(t);
  fill_shape<float, float, 1>(t);
  fill_shape<float, float, 2>(t);
  fill_shape<float, float, 3>(t);
}
}  // namespace pdmcf
