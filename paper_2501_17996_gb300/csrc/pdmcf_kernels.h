// pdmcf_kernels.h — launch shapes and per-precision kernel tables.
#pragma once

#include <cuda_bf16.h>

#include "pdmcf_device.cuh"

namespace pdmcf {

// One edge (or node) vector of ld elements is split into ld/VW 16-byte chunks; a group
// of `group` threads owns one edge/node and each thread holds `vpt` chunks in registers.
// capacity = group * vpt chunks.
struct ShapeDesc {
  int group, vpt, block;
};
constexpr int NUM_SHAPES = 14;
constexpr ShapeDesc kShapes[NUM_SHAPES] = {
    {32, 1, 256},  {32, 2, 256},  {32, 4, 256},  {32, 8, 256},  {128, 3, 128},
    {128, 4, 128}, {128, 6, 128}, {256, 4, 256}, {256, 6, 256}, {256, 8, 256},
    {512, 5, 512}, {512, 6, 512}, {512, 8, 512}, {512, 16, 512},
};

template <typename P, typename S>
struct KernelTable {
  void (*edge[NUM_SHAPES])(IterArgs<P, S>);
  void (*node[NUM_SHAPES])(IterArgs<P, S>);
  void (*node_chk[NUM_SHAPES])(IterArgs<P, S>);   // the node phase of check iterations
  void (*check[NUM_SHAPES])(IterArgs<P, S>);
};

// Pipelined (bulk-copy) edge phase for long vectors: one 512-thread CTA per SM, `vpt`
// 16-byte chunks of F per thread; the matching node phase reads the per-head in-sums.
constexpr int TMA_BLOCK = 512;
constexpr int TMA_NODE_BLOCK = 512;
constexpr int NUM_TMA = 5;
constexpr int kTmaVpt[NUM_TMA] = {2, 3, 4, 5, 7};

template <typename S>
struct TmaTable {
  void (*edge[NUM_TMA])(IterArgs<float, S>);
  void (*node[NUM_TMA])(IterArgs<float, S>);
  void (*node_chk[NUM_TMA])(IterArgs<float, S>);
  void (*insum[NUM_TMA])(IterArgs<float, S>);   // register edge phase with in-sums
};
const TmaTable<float>& tma_table_f32();
const TmaTable<__nv_bfloat16>& tma_table_bf16();

const KernelTable<float, float>& table_f32();
const KernelTable<double, double>& table_f64();
const KernelTable<float, __nv_bfloat16>& table_bf16();

// Smallest shape whose capacity covers nchunks (-1 if none).
inline int pick_shape(int nchunks) {
  int best = -1, best_cap = 0;
  for (int s = 0; s < NUM_SHAPES; ++s) {
    const int cap = kShapes[s].group * kShapes[s].vpt;
    if (cap >= nchunks && (best < 0 || cap < best_cap)) { best = s; best_cap = cap; }
  }
  return best;
}

}  // namespace pdmcf

// Residency target: keep 1024 threads per SM when a thread's register arrays are small,
// 512 when they are large (2 * VPT * VW values per thread in the edge phase).
template <typename P, int VPT, int VW, int BLOCK>
constexpr int min_blocks() {
  return (VPT * VW * (int)sizeof(P) <= 96) ? (1024 / BLOCK > 0 ? 1024 / BLOCK : 1)
                                           : (512 / BLOCK > 0 ? 512 / BLOCK : 1);
}

// The node phase works one chunk at a time, so its registers do not grow with VPT: 1024
// threads per SM.
template <typename P, int VPT, int VW, int BLOCK>
constexpr int min_blocks_node() {
  return 1024 / BLOCK > 0 ? 1024 / BLOCK : 1;
}

namespace pdmcf {
template <typename P, typename S, int IDX>
void fill_shape(KernelTable<P, S>& t) {
  constexpr ShapeDesc d = kShapes[IDX];
  constexpr int MB = min_blocks<P, d.vpt, StoreTraits<S>::VW, d.block>();
  t.edge[IDX] = edge_kernel<P, S, d.vpt, d.group, d.block, MB>;
  constexpr int MBN = min_blocks_node<P, d.vpt, StoreTraits<S>::VW, d.block>();
  t.node[IDX] = node_kernel<P, S, d.vpt, d.group, d.block, MBN, false, false>;
  t.node_chk[IDX] = node_kernel<P, S, d.vpt, d.group, d.block, 1, false, true>;
  t.check[IDX] = check_kernel<P, S, d.vpt, d.group, d.block, MB>;
}

template <typename S, int IDX>
void fill_tma(TmaTable<S>& t) {
  constexpr int V = kTmaVpt[IDX];
  t.edge[IDX] = edge_tma_kernel<S, V, TMA_BLOCK>;
  t.node[IDX] = node_kernel<float, S, V, TMA_NODE_BLOCK, TMA_NODE_BLOCK, 2, true, false>;
  t.node_chk[IDX] = node_kernel<float, S, V, TMA_NODE_BLOCK, TMA_NODE_BLOCK, 1, true, true>;
  t.insum[IDX] = edge_insum_kernel<float, S, V, TMA_BLOCK>;
}

// Defined in the pdmcf_kernels_<precision>_<part>.cu translation units (compiled in
// parallel); each fills a range of shapes.
#define PDMCF_PARTS(name, P, S)                        \
  void fill_##name##_0(KernelTable<P, S>& t);          \
  void fill_##name##_1(KernelTable<P, S>& t);          \
  void fill_##name##_2(KernelTable<P, S>& t);          \
  void fill_##name##_3(KernelTable<P, S>& t);          \
  void fill_##name##_4(KernelTable<P, S>& t);
PDMCF_PARTS(f32, float, float)
PDMCF_PARTS(f64, double, double)
PDMCF_PARTS(bf16, float, __nv_bfloat16)
#undef PDMCF_PARTS
}  // namespace pdmcf
