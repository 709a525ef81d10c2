// Naive circuit knitting on the GPU (Eq. knitting, section 2.1): the
// expectation value as the sum, over every global instance -- every
// assignment of every cut index, the tensor product of the QPD coefficient
// sets -- of the instance's coefficient times the product of its subcircuit
// results.  In h-TN terms: every non-output index assignment, the product of
// one entry of every tensor (QTs and CTs), summed in FP64.  Its cost grows
// with the product of all cut dimensions; it is the baseline the h-TN
// contraction is measured against (sections 2.1 and 4.2).
//
// k_knit_terms: grid (chunks, outputs); each thread walks a contiguous run of
// instances as a mixed-radix counter (last summed index fastest) with running
// per-tensor offsets (an increment adds one stride per tensor carrying that
// index, a carry subtracts the wrapped extent), multiplies one entry per
// tensor in FP64 and accumulates in FP64; the block sums its threads in a
// fixed tree and writes one partial.  k_knit_finish adds an output's
// partials in chunk order, so the result is deterministic.
#include <cuda_runtime.h>

#include "kernels.h"
#include "knit.h"

namespace qtpu {

namespace {

__device__ __forceinline__ double entry(const void* p, int dt, int64_t i) {
  return dt == DT_F64 ? ((const double*)p)[i] : (double)((const float*)p)[i];
}

__global__ void __launch_bounds__(256) k_knit_terms(const KnitTable* __restrict__ T, uint64_t per_chunk,
                                                    double* __restrict__ partial) {
  const int n_t = T->n_t, n_s = T->n_sum;
  const uint64_t chunk = blockIdx.x, o = blockIdx.y;
  const uint64_t c0 = chunk * per_chunk;
  const uint64_t c1 = min(T->n_inst, c0 + per_chunk);
  // this thread's run inside the chunk
  const uint64_t len = c1 > c0 ? c1 - c0 : 0;
  const uint64_t per_t = (len + blockDim.x - 1) / blockDim.x;
  const uint64_t i0 = c0 + min(len, (uint64_t)threadIdx.x * per_t);
  const uint64_t i1 = c0 + min(len, (uint64_t)(threadIdx.x + 1) * per_t);
  double acc = 0.0;
  if (i0 < i1) {
    int64_t off[kKnitMaxT];
    // output coordinates
    for (int t = 0; t < n_t; ++t) off[t] = 0;
    uint64_t r = o;
    for (int m = T->n_outi - 1; m >= 0; --m) {
      const uint64_t d = r % (uint64_t)T->out_dim[m];
      r /= (uint64_t)T->out_dim[m];
      for (int t = 0; t < n_t; ++t) off[t] += (int64_t)d * T->out_stride[m][t];
    }
    // digits of the first instance
    int64_t dig[kKnitMaxSum];
    r = i0;
    for (int m = n_s - 1; m >= 0; --m) {
      dig[m] = (int64_t)(r % (uint64_t)T->dim[m]);
      r /= (uint64_t)T->dim[m];
      for (int t = 0; t < n_t; ++t) off[t] += dig[m] * T->stride[m][t];
    }
    for (uint64_t i = i0; i < i1; ++i) {
      double p = entry(T->ptr[0], T->dt[0], off[0]);
      for (int t = 1; t < n_t; ++t) p = __dmul_rn(p, entry(T->ptr[t], T->dt[t], off[t]));
      acc = __dadd_rn(acc, p);
      // next instance
      int m = n_s - 1;
      while (m >= 0) {
        ++dig[m];
        for (int t = 0; t < n_t; ++t) off[t] += T->stride[m][t];
        if (dig[m] < T->dim[m]) break;
        for (int t = 0; t < n_t; ++t) off[t] -= T->dim[m] * T->stride[m][t];
        dig[m] = 0;
        --m;
      }
    }
  }
  // fixed-order block sum
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[o * gridDim.x + chunk] = red[0];
}

__global__ void k_knit_finish(const double* __restrict__ partial, uint64_t n_chunks, uint64_t n_out,
                              double* __restrict__ out) {
  const uint64_t o = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (o >= n_out) return;
  double s = 0.0;
  for (uint64_t c = 0; c < n_chunks; ++c) s = __dadd_rn(s, partial[o * n_chunks + c]);
  out[o] = s;
}

}  // namespace

cudaError_t launch_knit(const KnitTable* d_table, uint64_t n_inst, uint64_t n_out, double* partial,
                        uint64_t n_chunks, double* out, cudaStream_t st) {
  if (n_out == 0) return cudaSuccess;
  if (n_chunks == 0 || n_chunks > 65535u * 1024u || n_out > 65535) return cudaErrorInvalidValue;
  const uint64_t per_chunk = (n_inst + n_chunks - 1) / n_chunks;
  k_knit_terms<<<dim3((unsigned)n_chunks, (unsigned)n_out), 256, 0, st>>>(d_table, per_chunk, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_knit_finish<<<(unsigned)((n_out + 255) / 256), 256, 0, st>>>(partial, n_chunks, n_out, out);
  return cudaGetLastError();
}

}  // namespace qtpu
