// Kernel instantiations: P = float (iterates), S = float (storage of F), shape part 4.
#include "pdmcf_kernels.h"

namespace pdmcf {
void fill_f32_4(KernelTable<float, float>& t) {
  fill_shape<float, float, 12>(t);
  fill_shape<float, float, 13>(t);
}
}  // namespace pdmcf
