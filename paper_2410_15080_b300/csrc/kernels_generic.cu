// FP64 CUDA-core kernels of the h-TN contraction:
//
//  * k_contract_*: one pairwise contraction over strided operand views,
//      out[o] = sum_l A[offA(o) + offA(l)] * B[offB(o) + offB(l)],
//    used for every step that is not a large dense GEMM: absorbing a QPD
//    coefficient tensor into a QT (a gate CT scales along its hyper-index,
//    the 4x4 wire CT of Eq. wire-tensor mixes one index; section 4.1), dot
//    products over the last shared indices (the final contraction to <O>,
//    section 4.1), skinny products, and with B absent the slice sum and the
//    final reduction to the output indices.  Everything accumulates in FP64
//    in a fixed order, so results are deterministic.  HBM-bound: each output
//    is written once and operand runs are read along the innermost mode.

#include "common.cuh"
#include "kernels.h"

namespace qtpu {

namespace {

template <typename T>
__device__ __forceinline__ double ld(const T* p, int64_t i) {
  return (double)__ldg(p + i);
}

// offsets of flat index o over the modes of t (last mode fastest)
__device__ __forceinline__ void decompose(int64_t o, const ModeTab& t, int64_t& oa, int64_t& ob) {
  oa = 0;
  ob = 0;
  for (int j = t.n - 1; j >= 0; --j) {
    const int64_t d = t.dim[j];
    const int64_t q = o / d;
    const int64_t i = o - q * d;
    o = q;
    oa += i * t.sa[j];
    ob += i * t.sb[j];
  }
}

template <typename TA, typename TB, bool HAS_B>
__device__ __forceinline__ double loop_sum(const TA* A, const TB* B, int64_t oa, int64_t ob,
                                           const ContractArgs& a) {
  const ModeTab& L = a.loop;
  if (L.n == 0) return HAS_B ? ld(A, oa) * ld(B, ob) : ld(A, oa);
  if (L.n == 1) {
    double acc = 0.0;
    const int64_t d = L.dim[0], sa = L.sa[0], sb = L.sb[0];
    for (int64_t i = 0; i < d; ++i) acc += HAS_B ? ld(A, oa + i * sa) * ld(B, ob + i * sb) : ld(A, oa + i * sa);
    return acc;
  }
  if (L.n == 2) {
    double acc = 0.0;
    for (int64_t i0 = 0; i0 < L.dim[0]; ++i0) {
      const int64_t a0 = oa + i0 * L.sa[0], b0 = ob + i0 * L.sb[0];
      for (int64_t i1 = 0; i1 < L.dim[1]; ++i1)
        acc += HAS_B ? ld(A, a0 + i1 * L.sa[1]) * ld(B, b0 + i1 * L.sb[1]) : ld(A, a0 + i1 * L.sa[1]);
    }
    return acc;
  }
  // general odometer over the loop modes
  int64_t idx[kMaxModes];
  for (int j = 0; j < L.n; ++j) idx[j] = 0;
  int64_t pa = oa, pb = ob;
  double acc = 0.0;
  for (int64_t l = 0; l < a.n_loop; ++l) {
    acc += HAS_B ? ld(A, pa) * ld(B, pb) : ld(A, pa);
    int j = L.n - 1;
    ++idx[j];
    pa += L.sa[j];
    pb += L.sb[j];
    while (j > 0 && idx[j] == L.dim[j]) {
      pa -= L.dim[j] * L.sa[j];
      pb -= L.dim[j] * L.sb[j];
      idx[j] = 0;
      --j;
      ++idx[j];
      pa += L.sa[j];
      pb += L.sb[j];
    }
  }
  return acc;
}

// one thread per output entry
template <typename TA, typename TB, bool HAS_B>
__global__ void __launch_bounds__(256) k_contract_thread(const TA* __restrict__ A, const TB* __restrict__ B,
                                                         double* __restrict__ out, const ContractArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < a.n_out; o += stride) {
    int64_t oa, ob;
    decompose(o, a.out, oa, ob);
    const double v = loop_sum<TA, TB, HAS_B>(A, B, oa, ob, a);
    out[o] = a.accum ? out[o] + v : v;
  }
}

// one block per output entry, the loop split over the threads, then a
// fixed-shape tree (deterministic)
template <typename TA, typename TB, bool HAS_B>
__global__ void __launch_bounds__(256) k_contract_block(const TA* __restrict__ A, const TB* __restrict__ B,
                                                        double* __restrict__ out, const ContractArgs a) {
  __shared__ double red[8];
  for (int64_t o = blockIdx.x; o < a.n_out; o += gridDim.x) {
    int64_t oa, ob;
    decompose(o, a.out, oa, ob);
    double acc = 0.0;
    for (int64_t l = threadIdx.x; l < a.n_loop; l += blockDim.x) {
      int64_t la, lb;
      decompose(l, a.loop, la, lb);
      acc += HAS_B ? ld(A, oa + la) * ld(B, ob + lb) : ld(A, oa + la);
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      out[o] = a.accum ? out[o] + t : t;
    }
    __syncthreads();
  }
}

template <typename TA, typename TB, bool HAS_B>
cudaError_t launch3(const void* A, const void* B, double* out, const ContractArgs& a, int sm, cudaStream_t st) {
  if (a.n_out <= 0) return cudaSuccess;
  const bool block_mode = a.n_loop >= 1024 && a.n_out <= (int64_t)sm * 16;
  if (block_mode) {
    const int64_t g = a.n_out < (int64_t)sm * 16 ? a.n_out : (int64_t)sm * 16;
    k_contract_block<TA, TB, HAS_B><<<(int)g, 256, 0, st>>>((const TA*)A, (const TB*)B, out, a);
  } else {
    int64_t g = (a.n_out + 255) / 256;
    if (g > (int64_t)sm * 32) g = (int64_t)sm * 32;
    k_contract_thread<TA, TB, HAS_B><<<(int)g, 256, 0, st>>>((const TA*)A, (const TB*)B, out, a);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_contract(const void* A, int dtA, const void* B, int dtB, double* out, const ContractArgs& a,
                            int sm, cudaStream_t st) {
  if (!B) {
    return dtA == DT_F64 ? launch3<double, double, false>(A, nullptr, out, a, sm, st)
                         : launch3<float, double, false>(A, nullptr, out, a, sm, st);
  }
  if (dtA == DT_F64 && dtB == DT_F64) return launch3<double, double, true>(A, B, out, a, sm, st);
  if (dtA == DT_F64 && dtB == DT_F32) return launch3<double, float, true>(A, B, out, a, sm, st);
  if (dtA == DT_F32 && dtB == DT_F64) return launch3<float, double, true>(A, B, out, a, sm, st);
  return launch3<float, float, true>(A, B, out, a, sm, st);
}


}  // namespace qtpu
