// Kernel instantiations: P = float (iterates), S = float (storage of F), shape part 3.
#include "pdmcf_kernels.h"

namespace pdmcf {
void fill_f32_3(KernelTable<float, float>& t) {
  fill_shape<float, float, 10>(t);
  fill_shape<float, float, 11>(t);
}
}  // namespace pdmcf
