// QPD sampling and h-TN simplification: device-side descriptors and
// launchers (section 4.3; Step 1 of section 6.1).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace qtpu {

constexpr int kQpdMaxCts = 8;    // gate-cut CTs fused into one
constexpr int kQpdMaxAxes = 16;  // axes of a truncated QT

// One fused CT: its gate-cut vectors (device pointers, dtype, extent, stride
// in elements), its length D = prod(dim) and its offset in the per-value
// buffers (fused values, prefix sums, counts, kept values).
struct QpdGroup {
  int n_ct = 0;
  int64_t D = 0, base = 0;
  const void* ct[kQpdMaxCts] = {};
  int dt[kQpdMaxCts] = {};
  int64_t dim[kQpdMaxCts] = {}, stride[kQpdMaxCts] = {};
};

// The truncated copy of one QT: output axes in C order, each either plain
// (element stride `stride` in the source) or fused (`table` gives the source
// offset of each kept value).
struct QpdGather {
  const void* src = nullptr;
  void* dst = nullptr;
  int dt = 0;  // DT_F32 or DT_F64, the same for source and copy
  int n_axes = 0;
  int64_t n_out = 0;
  int64_t dim[kQpdMaxAxes] = {}, stride[kQpdMaxAxes] = {};
  const int64_t* table[kQpdMaxAxes] = {};
};

// fused[base + f] for every group (max_D: the largest D)
cudaError_t qpd_fuse(const QpdGroup* d_groups, int n_groups, int64_t max_D, double* fused, cudaStream_t st);
// counts[base + i] += draws of i, from u[x * s + j]; gamma[x] = P_{D-1}
cudaError_t qpd_draw(const QpdGroup* d_groups, int n_groups, const double* fused, double* prefix, double* gamma,
                     const double* u, uint64_t s, uint32_t* counts, cudaStream_t st);
// kept_idx[base + k], kept_ct[base + k] for k < n_kept[x]
cudaError_t qpd_compact(const QpdGroup* d_groups, int n_groups, const double* fused, const double* gamma,
                        const uint32_t* counts, uint64_t s, int32_t* kept_idx, double* kept_ct, int32_t* n_kept,
                        cudaStream_t st);
// out[k] = sum_j digit_j(kept_idx[k]) * qstride[j] over the group's dims
cudaError_t qpd_table(int n_ct, const int64_t* dims, const int64_t* qstride, const int32_t* kept_idx, int64_t n_kept,
                      int64_t* out, cudaStream_t st);
cudaError_t qpd_gather(const QpdGather& a, int sm_count, cudaStream_t st);

}  // namespace qtpu
