// Executor: turns a Plan into kernel launches on one device and stream.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "kernels.h"
#include "planner.h"

namespace qtpu {

struct Leaf {
  Inds ids;
  std::vector<int64_t> dims, strides;  // strides in elements
  int dt = DT_F64;
  const void* ptr = nullptr;
};

enum StepKind { SK_GENERIC = 0, SK_TC = 1 };

struct StepExec {
  int kind = SK_GENERIC;
  int x = 0, y = 0, out = 0;
  int dtx = DT_F64, dty = DT_F64;
  bool x_leaf = false, y_leaf = false;
  ContractArgs c;            // generic
  SplitArgs sa, sb;          // tensor-core path
  GemmArgs g;
  size_t out_off = 0;        // arena byte offset (unused for the last step)
  bool last = false;
  double flops = 0;          // useful flops per slice
};

struct Executor {
  int device = 0;
  int sm_count = 148;
  cudaStream_t stream = nullptr;
  int prec = 3;
  int kc_blocks = 0;
  std::vector<StepExec> steps;
  // per leaf: (stride, dim) of each sliced index it carries, in slice order
  std::vector<std::vector<std::pair<int, int64_t>>> leaf_slice;  // (slice position, stride)
  std::vector<int64_t> slice_dims;  // dims of the sliced indices, plan order
  int64_t n_slices = 1;
  int64_t final_size = 1;           // entries of the last step's output per slice
  ContractArgs reduce;              // partial[slices][final] -> out
  bool reduce_from_leaf = false;    // single-tensor network: reduce the leaf
  int reduce_leaf = 0;
  // device memory (owned)
  uint8_t* arena = nullptr;
  size_t arena_bytes = 0;
  uint8_t* splitbuf = nullptr;
  size_t split_bytes = 0;
  double* partial = nullptr;
  uint32_t* status = nullptr;
  double* out_stage = nullptr;     // staging buffer of the host-buffer entry point
  int n_tc_steps = 0;
  size_t workspace_bytes() const { return arena_bytes + split_bytes + (size_t)n_slices * final_size * 8; }
};

// Build launch descriptors and allocate the workspace.  Returns an empty
// string on success, else an error message (*code receives a qtpu_status).
std::string exec_build(Executor* ex, const Plan& plan, const std::vector<Leaf>& leaves, const DimMap& dims,
                       int prec, int* code);
// Enqueue the whole contraction; writes output_size FP64 entries to dev_out.
std::string exec_run(Executor* ex, const std::vector<Leaf>& leaves, double* dev_out, cudaStream_t st, int* code);
void exec_free(Executor* ex);

}  // namespace qtpu
