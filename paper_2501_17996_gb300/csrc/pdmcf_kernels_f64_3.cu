// Kernel instantiations: P = double (iterates), S = double (storage of F), shape part 3.
#include "pdmcf_kernels.h"

namespace pdmcf {
void fill_f64_3(KernelTable<double, double>& t) {
}
}  // namespace pdmcf
