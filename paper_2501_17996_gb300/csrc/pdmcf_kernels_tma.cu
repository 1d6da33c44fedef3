// Kernel instantiations of the pipelined edge phase and its node phase (FP32 iterates,
// F stored as FP32 or BF16).
#include "pdmcf_kernels.h"

namespace pdmcf {

const TmaTable<float>& tma_table_f32() {
  static const TmaTable<float> t = [] {
    TmaTable<float> t{};
    fill_tma<float, 0>(t); fill_tma<float, 1>(t); fill_tma<float, 2>(t);
    fill_tma<float, 3>(t); fill_tma<float, 4>(t);
    return t;
  }();
  return t;
}

}  // namespace pdmcf
