// pdmcf_batch_engine.h — host engine that advances many resident instances together.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <tuple>
#include <vector>

#include "pdmcf_batch.cuh"
#include "pdmcf_internal.h"
#include "pdmcf_kernels.h"

namespace pdmcf {

using BatchKernel = void (*)(const BatchInst*, BatchClassDev);
struct BatchTable {
  BatchKernel edge[NUM_SHAPES];
  BatchKernel node[NUM_SHAPES];
  BatchKernel check[NUM_SHAPES];
};
const BatchTable& batch_table();

// Device buffers of one instance the engine owns besides the problem's DeviceState.
struct BatchSlot {
  bool used = false;
  mcf_problem* p = nullptr;
  mcf_options opts{};
  void* tag = nullptr;
  int cls = -1;
  double* pe = nullptr;
  double* pn = nullptr;
  double* pc = nullptr;
  int64_t bytes = 0;
  bool finished = false;
  int status = MCF_PENDING;
  mcf_result res{};
};

// Advances every resident instance by one PDHG iteration per step with one launch per
// phase and shape class. Not thread-safe: one owner thread drives it.
class BatchEngine {
 public:
  BatchEngine(int device, int max_slots);
  ~BatchEngine();
  int init();                         // allocate the tables; MCF_OK or an error
  int device() const { return device_; }
  int free_slots() const;
  int active_count() const;
  // Admit an FP32 request: allocates/initialises the instance state (cold or warm).
  int add(mcf_problem* p, const mcf_options& o, void* tag, int* slot_out, int cls = -1);
  // Run `iters` batched iterations (graph-captured), then refresh the host scalar mirror
  // and mark instances whose stop rule fired as finished.
  int step(int iters);
  // Finished slots since the last call.
  std::vector<int> take_finished();
  // Copy the slot's final state back into its problem and free the slot.
  void release(int slot);
  const BatchSlot& slot(int s) const { return slots_[s]; }
  static int64_t extra_bytes(const mcf_problem* p);   // engine buffers per instance

 private:
  int step_impl(int iters);
  int upload_lists();
  int launch_iteration(cudaStream_t st, bool with_check);
  uint64_t check_iterations(int iters) const;
  void destroy_graphs();

  int device_;
  int max_slots_;
  cudaStream_t stream_ = nullptr;
  int sms_ = 0;
  BatchInst* d_insts_ = nullptr;
  BatchScalars* d_sc_ = nullptr;
  BatchScalars* h_sc_ = nullptr;       // pinned mirror
  int* d_slot_list_ = nullptr;
  int* d_nslots_ = nullptr;
  int* d_cls_count_ = nullptr;          // [NUM_SHAPES]
  int* d_cls_inst_ = nullptr;           // [NUM_SHAPES * max_slots]
  long long* d_cls_eoff_ = nullptr;     // [NUM_SHAPES * (max_slots + 1)]
  long long* d_cls_noff_ = nullptr;
  int grid_[3][NUM_SHAPES] = {};
  std::vector<BatchSlot> slots_;
  std::vector<BatchInst> h_insts_;
  bool lists_dirty_ = true;
  unsigned class_mask_ = 0;
  // key: class mask, iterations per chunk, iterations of the chunk with a stop test
  std::map<std::tuple<unsigned, int, uint64_t>, cudaGraphExec_t> graphs_;
  bool graphs_broken_ = false;
  std::vector<int> finished_;
};

int batch_admit_shape(const mcf_problem* p);   // default shape class of an FP32 instance
// Shape class the batched engine uses for an instance with this many 16-byte chunks per
// vector: the default class, or the autotuned choice once tuning has run for it.
int batch_class_for(int device, int nchunks, bool autotune);

}  // namespace pdmcf
