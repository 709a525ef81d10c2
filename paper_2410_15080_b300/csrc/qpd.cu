// QPD sampling and h-TN simplification (section 4.3; Step 1 of section 6.1).
//
// The gate-cut coefficient vectors between the same two QTs are fused into
// one CT (their tensor product, first vector slowest); each fused CT c is
// sampled s times with probability |c_i| / gamma; the sampled CT is
// c'_i = sign(c_i) * ((gamma * count_i) / s); values never drawn are dropped
// from the CT and from the two QTs along the fused index.  The kernels here:
//
//   k_qpd_fuse     fused CT entries c_1[i_1] * c_2[i_2] * ..., FP64, left to
//                  right (every group in one launch);
//   k_qpd_draw     one block per group: thread 0 accumulates the prefix sums
//                  P_i = |c_0| + ... + |c_i| left to right in FP64 (the draws
//                  are integer decisions taken from floating point, so the
//                  order is fixed), then the block maps each uniform u to the
//                  first i with P_i > u * gamma (binary search; the last
//                  nonzero entry if there is none) and counts it atomically;
//   k_qpd_compact  one block per group: the drawn values in ascending order,
//                  their sampled coefficients, and the kept count;
//   k_qpd_table    per (QT, group): the QT element offset of every kept fused
//                  value (its digits times the QT's strides of the group's
//                  indices);
//   k_qpd_gather   the truncated QT: every entry of the new C-order layout
//                  read from the source QT through plain strides and the
//                  fused tables, the trailing axes' offsets tabulated once
//                  per block in shared memory (HBM-bound: one read and one
//                  write per kept entry).
#include <cuda_runtime.h>

#include "kernels.h"
#include "qpd.h"

namespace qtpu {

namespace {

__device__ __forceinline__ double load_val(const void* p, int dt, int64_t i) {
  return dt == DT_F64 ? ((const double*)p)[i] : (double)((const float*)p)[i];
}

__global__ void k_qpd_fuse(const QpdGroup* __restrict__ groups, int n_groups, double* __restrict__ fused) {
  const int x = blockIdx.y;
  if (x >= n_groups) return;
  const QpdGroup& G = groups[x];
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < G.D; f += (int64_t)gridDim.x * blockDim.x) {
    int64_t digit[kQpdMaxCts];
    int64_t r = f;
    for (int j = G.n_ct - 1; j >= 0; --j) {
      digit[j] = r % G.dim[j];
      r /= G.dim[j];
    }
    double p = load_val(G.ct[0], G.dt[0], digit[0] * G.stride[0]);
    for (int j = 1; j < G.n_ct; ++j) p = __dmul_rn(p, load_val(G.ct[j], G.dt[j], digit[j] * G.stride[j]));
    fused[G.base + f] = p;
  }
}

__global__ void k_qpd_draw(const QpdGroup* __restrict__ groups, const double* __restrict__ fused,
                           double* __restrict__ prefix, double* __restrict__ gamma_out, const double* __restrict__ u,
                           uint64_t s, uint32_t* __restrict__ counts) {
  const int x = blockIdx.x;
  const QpdGroup& G = groups[x];
  const double* c = fused + G.base;
  double* P = prefix + G.base;
  __shared__ double s_gamma;
  __shared__ int64_t s_last;
  if (threadIdx.x == 0) {
    double acc = 0.0;
    int64_t last = G.D - 1, lastnz = -1;
    for (int64_t i = 0; i < G.D; ++i) {
      const double a = fabs(c[i]);
      acc = __dadd_rn(acc, a);
      P[i] = acc;
      if (a != 0.0) lastnz = i;
    }
    s_gamma = acc;
    s_last = lastnz >= 0 ? lastnz : last;
    gamma_out[x] = acc;
  }
  __syncthreads();
  const double gamma = s_gamma;
  const int64_t last = s_last;
  const double* ux = u + (uint64_t)x * s;
  for (uint64_t j = threadIdx.x; j < s; j += blockDim.x) {
    const double t = __dmul_rn(ux[j], gamma);
    // first i with P[i] > t
    int64_t lo = 0, hi = G.D;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (P[mid] > t)
        hi = mid;
      else
        lo = mid + 1;
    }
    atomicAdd(&counts[G.base + (lo < G.D ? lo : last)], 1u);
  }
}

__global__ void k_qpd_compact(const QpdGroup* __restrict__ groups, const double* __restrict__ fused,
                              const double* __restrict__ gamma, const uint32_t* __restrict__ counts, uint64_t s,
                              int32_t* __restrict__ kept_idx, double* __restrict__ kept_ct,
                              int32_t* __restrict__ n_kept) {
  const int x = blockIdx.x;
  if (threadIdx.x != 0) return;
  const QpdGroup& G = groups[x];
  const double g = gamma[x];
  const double sd = (double)s;
  int32_t k = 0;
  for (int64_t i = 0; i < G.D; ++i) {
    const uint32_t n = counts[G.base + i];
    if (!n) continue;
    const double c = fused[G.base + i];
    const double m = __ddiv_rn(__dmul_rn(g, (double)n), sd);
    kept_idx[G.base + k] = (int32_t)i;
    kept_ct[G.base + k] = c > 0.0 ? m : (c < 0.0 ? -m : 0.0);
    ++k;
  }
  n_kept[x] = k;
}

struct TableArgs {
  int n_ct;
  int64_t dim[kQpdMaxCts], qstride[kQpdMaxCts];
};

__global__ void k_qpd_table(TableArgs a, const int32_t* __restrict__ kept_idx, int64_t n_kept,
                            int64_t* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_kept; k += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = kept_idx[k], off = 0;
    for (int j = a.n_ct - 1; j >= 0; --j) {
      off += (r % a.dim[j]) * a.qstride[j];
      r /= a.dim[j];
    }
    out[k] = off;
  }
}

// Output axes [0, split) are the outer axes, [split, n_axes) the inner ones
// (at most kQpdInner entries together).  Each block builds the source offsets
// of the inner entries once in shared memory; then per outer row (grid-
// stride) one offset from the outer coordinates, and the row's entries are
// copied with contiguous writes.
constexpr int kQpdInner = 4096;

template <typename T>
__global__ void __launch_bounds__(256) k_qpd_gather(const __grid_constant__ QpdGather a, int split, int64_t inner) {
  __shared__ int64_t tab[kQpdInner];
  const T* __restrict__ src = (const T*)a.src;
  T* __restrict__ dst = (T*)a.dst;
  for (int64_t j = threadIdx.x; j < inner; j += blockDim.x) {
    int64_t r = j, off = 0;
    for (int m = a.n_axes - 1; m >= split; --m) {
      const int64_t i = r % a.dim[m];
      r /= a.dim[m];
      off += a.table[m] ? a.table[m][i] : i * a.stride[m];
    }
    tab[j] = off;
  }
  __syncthreads();
  const int64_t rows = a.n_out / inner;
  for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
    int64_t r = row, base = 0;
    for (int m = split - 1; m >= 0; --m) {
      const int64_t i = r % a.dim[m];
      r /= a.dim[m];
      base += a.table[m] ? a.table[m][i] : i * a.stride[m];
    }
    T* d = dst + row * inner;
    for (int64_t j = threadIdx.x; j < inner; j += blockDim.x) d[j] = src[base + tab[j]];
  }
}

}  // namespace

cudaError_t qpd_fuse(const QpdGroup* d_groups, int n_groups, int64_t max_D, double* fused, cudaStream_t st) {
  if (n_groups <= 0) return cudaSuccess;
  const int64_t bx = (max_D + 255) / 256;
  k_qpd_fuse<<<dim3((unsigned)(bx < 4096 ? bx : 4096), (unsigned)n_groups), 256, 0, st>>>(d_groups, n_groups, fused);
  return cudaGetLastError();
}

cudaError_t qpd_draw(const QpdGroup* d_groups, int n_groups, const double* fused, double* prefix, double* gamma,
                     const double* u, uint64_t s, uint32_t* counts, cudaStream_t st) {
  if (n_groups <= 0) return cudaSuccess;
  k_qpd_draw<<<n_groups, 256, 0, st>>>(d_groups, fused, prefix, gamma, u, s, counts);
  return cudaGetLastError();
}

cudaError_t qpd_compact(const QpdGroup* d_groups, int n_groups, const double* fused, const double* gamma,
                        const uint32_t* counts, uint64_t s, int32_t* kept_idx, double* kept_ct, int32_t* n_kept,
                        cudaStream_t st) {
  if (n_groups <= 0) return cudaSuccess;
  k_qpd_compact<<<n_groups, 32, 0, st>>>(d_groups, fused, gamma, counts, s, kept_idx, kept_ct, n_kept);
  return cudaGetLastError();
}

cudaError_t qpd_table(int n_ct, const int64_t* dims, const int64_t* qstride, const int32_t* kept_idx, int64_t n_kept,
                      int64_t* out, cudaStream_t st) {
  if (n_kept <= 0) return cudaSuccess;
  if (n_ct < 1 || n_ct > kQpdMaxCts) return cudaErrorInvalidValue;
  TableArgs a{};
  a.n_ct = n_ct;
  for (int j = 0; j < n_ct; ++j) a.dim[j] = dims[j], a.qstride[j] = qstride[j];
  const int64_t b = (n_kept + 255) / 256;
  k_qpd_table<<<(unsigned)(b < 1024 ? b : 1024), 256, 0, st>>>(a, kept_idx, n_kept, out);
  return cudaGetLastError();
}

cudaError_t qpd_gather(const QpdGather& a, int sm_count, cudaStream_t st) {
  if (a.n_out <= 0) return cudaSuccess;
  if (a.n_axes < 0 || a.n_axes > kQpdMaxAxes) return cudaErrorInvalidValue;
  // the longest run of trailing axes within kQpdInner entries
  int split = a.n_axes;
  int64_t inner = 1;
  while (split > 0 && inner * a.dim[split - 1] <= kQpdInner) inner *= a.dim[--split];
  const int64_t rows = a.n_out / inner;
  const int64_t cap = (int64_t)sm_count * 4;
  const unsigned grid = (unsigned)(rows < cap ? rows : cap);
  if (a.dt == DT_F64)
    k_qpd_gather<double><<<grid, 256, 0, st>>>(a, split, inner);
  else
    k_qpd_gather<float><<<grid, 256, 0, st>>>(a, split, inner);
  return cudaGetLastError();
}

}  // namespace qtpu
