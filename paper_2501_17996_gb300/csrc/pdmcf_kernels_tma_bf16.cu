// Kernel instantiations of the pipelined edge phase and its node phase, F stored as BF16.
#include "pdmcf_kernels.h"

namespace pdmcf {

const TmaTable<__nv_bfloat16>& tma_table_bf16() {
  static const TmaTable<__nv_bfloat16> t = [] {
    TmaTable<__nv_bfloat16> t{};
    fill_tma<__nv_bfloat16, 0>(t); fill_tma<__nv_bfloat16, 1>(t); fill_tma<__nv_bfloat16, 2>(t);
    fill_tma<__nv_bfloat16, 3>(t); fill_tma<__nv_bfloat16, 4>(t);
    return t;
  }();
  return t;
}

}  // namespace pdmcf
