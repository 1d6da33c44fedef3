// Kernel instantiations: P = double (iterates), S = double (storage of F), shape part 1.
#include "pdmcf_kernels.h"

namespace pdmcf {
void fill_f64_1(KernelTable<double, double>& t) {
  fill_shape<double, double, 4>(t);
  fill_shape<double, double, 5>(t);
  fill_shape<double, double, 6>(t);
}
}  // namespace pdmcf
