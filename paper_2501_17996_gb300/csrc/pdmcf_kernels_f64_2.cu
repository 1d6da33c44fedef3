// Kernel instantiations: P = double (iterates), S = double (storage of F), shape part 2.
#include "pdmcf_kernels.h"

namespace pdmcf {
void fill_f64_2(KernelTable<double, double>& t) {
  fill_shape<double, double, 7>(t);
  fill_shape<double, double, 8>(t);
  fill_shape<double, double, 9>(t);
}
}  // namespace pdmcf
