// Kernel instantiations of the batched iteration (FP32 iterates), one entry per launch shape.
#include "pdmcf_batch_engine.h"

namespace pdmcf {

template <int IDX>
static void fill_batch(BatchTable& t) {
  constexpr ShapeDesc d = kShapes[IDX];
  constexpr int MB = min_blocks<float, d.vpt, 4, d.block>();
  // the node phase works one chunk at a time (its registers do not grow with vpt): 1024
  // threads per SM
  constexpr int MBN = 1024 / d.block > 0 ? 1024 / d.block : 1;
  t.edge[IDX] = batch_edge_kernel<d.vpt, d.group, d.block, MB>;
  t.node[IDX] = batch_node_kernel<d.vpt, d.group, d.block, MBN>;
  t.check[IDX] = batch_check_kernel<d.vpt, d.group, d.block, MB>;
}

const BatchTable& batch_table() {
  static const BatchTable t = [] {
    BatchTable t{};
    fill_batch<0>(t); fill_batch<1>(t); fill_batch<2>(t); fill_batch<3>(t); fill_batch<4>(t);
    fill_batch<5>(t); fill_batch<6>(t); fill_batch<7>(t); fill_batch<8>(t); fill_batch<9>(t);
    fill_batch<10>(t); fill_batch<11>(t); fill_batch<12>(t); fill_batch<13>(t);
    return t;
  }();
  return t;
}

}  // namespace pdmcf
