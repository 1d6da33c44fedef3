// Kernel instantiations: P = float (iterates), S = float (storage of F), shape part 2.
#include "pdmcf_kernels.h"

namespace pdmcf {
void fill_f32_2(KernelTable<float, float>& t) {
  fill_shape<float, float, 7>(t);
  fill_shape<float, float, 8>(t);
  fill_shape<float, float, 9>(t);
}
}  // namespace pdmcf
