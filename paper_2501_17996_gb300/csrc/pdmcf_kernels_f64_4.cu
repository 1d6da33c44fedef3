// Kernel instantiations: P = double (iterates), S = double (storage of F), shape part 4.
#include "pdmcf_kernels.h"

namespace pdmcf {
void fill_f64_4(KernelTable<double, double>& t) {
}
}  // namespace pdmcf
