// Naive circuit knitting (Eq. knitting, section 2.1): the sum over every
// global instance, as a device-side table of the network.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace qtpu {

constexpr int kKnitMaxT = 32;    // tensors
constexpr int kKnitMaxSum = 40;  // summed (non-output) indices
constexpr int kKnitMaxOut = 8;   // output indices

// The network for k_knit_terms (in device memory): per tensor its data and
// dtype; per summed index its extent and its element stride in each tensor
// (0 where the tensor does not carry it); the same for the output indices.
// Summed indices are enumerated as one mixed-radix number, the last fastest.
struct KnitTable {
  int n_t = 0, n_sum = 0, n_outi = 0;
  uint64_t n_inst = 1;
  const void* ptr[kKnitMaxT] = {};
  int dt[kKnitMaxT] = {};
  int64_t dim[kKnitMaxSum] = {};
  int64_t stride[kKnitMaxSum][kKnitMaxT] = {};
  int64_t out_dim[kKnitMaxOut] = {};
  int64_t out_stride[kKnitMaxOut][kKnitMaxT] = {};
};

// out[o] = FP64 sum over the n_inst instances, partials[n_out][n_chunks]
cudaError_t launch_knit(const KnitTable* d_table, uint64_t n_inst, uint64_t n_out, double* partial,
                        uint64_t n_chunks, double* out, cudaStream_t st);

}  // namespace qtpu
