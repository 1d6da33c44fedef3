// Kernel instantiations: P = double (iterates), S = double (storage of F), shape part 0.
#include "pdmcf_kernels.h"

namespace pdmcf {
void fill_f64_0(KernelTable<double, double>& t) {
  fill_shape<double, double, 0>(t);
  fill_shape<double, double, 1>(t);
  fill_shape<double, double, 2>(t);
  fill_shape<double, double, 3>(t);
}
}  // namespace pdmcf
