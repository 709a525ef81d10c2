// Multi-operand gather-contract kernel with compensated FP32 arithmetic.
//
//   value(o) = sum_{l} prod_{j < nops} X_j[off_j(o) + off_j(l)]
//
// over strided operand views, written either as an FP32 pair (hi, lo) per
// entry (an intermediate tensor), as FP64 (the final output), or split into
// tensor-core pieces laid out [rows][Kp] (a GEMM operand).  One kernel covers
// every non-GEMM piece of the contraction: absorbing the QPD coefficient
// tensors into a QT (section 4.1: a gate CT scales along its hyper-index, the
// wire CT of Eq. wire-tensor mixes one index; the executor folds chains of
// such absorptions into the operand gather of the step that consumes them),
// dot products over the last shared indices, small pairwise steps, and the
// gather + split of each GEMM operand.
//
// Why FP32 pairs: FP64 throughput on B300 is ~1/64 of FP32, so FP64 values
// are decoded into (hi, lo) floats with integer operations only, products and
// sums use error-free transformations (TwoProd via FMA, TwoSum), and
// intermediates are stored as pairs (value = hi + lo, ~44 significant bits).
#include <cuda_bf16.h>

#include "arith.cuh"
#include "common.cuh"
#include "kernels.h"

namespace qtpu {

namespace {
using namespace arith;

template <int NOPS>
__device__ __forceinline__ float2 term(const GatherArgs& a, const int64_t* off) {
  float2 v = load_any(a.ptr[0], a.dt[0], off[0]);
#pragma unroll
  for (int j = 1; j < NOPS; ++j) v = mul_pair(v, load_any(a.ptr[j], a.dt[j], off[j]));
  return v;
}

// loop positions [l0, l1) of one output entry (base offsets) as an odometer
// walk over the loop modes, started from the digits of l0
template <int NOPS, typename ACC>
__device__ __forceinline__ void entry_range(const GatherArgs& a, const int64_t* base, uint32_t l0, uint32_t l1,
                                            ACC& acc) {
  if (l0 >= l1) return;
  uint32_t idx[kMaxModes];
  int64_t off[NOPS];
#pragma unroll
  for (int j = 0; j < NOPS; ++j) off[j] = base[j];
  digits<NOPS>(l0, a.loop, idx, off);
  for (uint32_t l = l0; l < l1; ++l) {
    acc.add(term<NOPS>(a, off));
    int m = a.loop.n - 1;
    ++idx[m];
#pragma unroll
    for (int j = 0; j < NOPS; ++j) off[j] += a.loop.stride[m][j];
    while (m > 0 && idx[m] == a.loop.dim[m]) {
#pragma unroll
      for (int j = 0; j < NOPS; ++j) off[j] -= (int64_t)a.loop.dim[m] * a.loop.stride[m][j];
      idx[m] = 0;
      --m;
      ++idx[m];
#pragma unroll
      for (int j = 0; j < NOPS; ++j) off[j] += a.loop.stride[m][j];
    }
  }
}

// value of one output entry: base offsets + sum over the loop modes, in the
// accumulator ACC (FP32 pairs for intermediates, FP64 for output values)
template <int NOPS, typename ACC>
__device__ __forceinline__ ACC entry(const GatherArgs& a, const int64_t* base) {
  ACC acc;
  if (a.loop.n == 0) {
    acc.add(term<NOPS>(a, base));
    return acc;
  }
  if (a.loop.n == 1) {
    int64_t off[NOPS];
#pragma unroll
    for (int j = 0; j < NOPS; ++j) off[j] = base[j];
    for (uint32_t i = 0; i < a.loop.dim[0]; ++i) {
      acc.add(term<NOPS>(a, off));
#pragma unroll
      for (int j = 0; j < NOPS; ++j) off[j] += a.loop.stride[0][j];
    }
    return acc;
  }
  uint32_t idx[kMaxModes];
  int64_t off[NOPS];
  for (int m = 0; m < a.loop.n; ++m) idx[m] = 0;
#pragma unroll
  for (int j = 0; j < NOPS; ++j) off[j] = base[j];
  for (uint32_t l = 0; l < a.n_loop; ++l) {
    acc.add(term<NOPS>(a, off));
    int m = a.loop.n - 1;
    ++idx[m];
#pragma unroll
    for (int j = 0; j < NOPS; ++j) off[j] += a.loop.stride[m][j];
    while (m > 0 && idx[m] == a.loop.dim[m]) {
#pragma unroll
      for (int j = 0; j < NOPS; ++j) off[j] -= (int64_t)a.loop.dim[m] * a.loop.stride[m][j];
      idx[m] = 0;
      --m;
      ++idx[m];
#pragma unroll
      for (int j = 0; j < NOPS; ++j) off[j] += a.loop.stride[m][j];
    }
  }
  return acc;
}

// ------------------------------------------------------------ dense writers
// out[o] for o < n_out, one thread per entry (FP32 pair, or FP64 output
// accumulated in FP64).  With lanes_log2 > 0 (few outputs, a long loop),
// 2^lanes_log2 consecutive lanes share an entry, each summing a contiguous
// run of the loop, and the runs' sums meet by shuffles in a fixed order.
template <int NOPS, bool F64OUT>
__global__ void __launch_bounds__(256) k_gather_dense(const GatherArgs a, void* __restrict__ out, int lanes_log2) {
  using ACC = typename AccSel<F64OUT>::T;
  pdl_wait();
  pdl_launch_dependents();
  if (lanes_log2 > 0) {
    const uint32_t S = 1u << lanes_log2;
    const uint32_t per = (a.n_loop + S - 1) / S;
    const uint64_t total = (uint64_t)a.n_out << lanes_log2;
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    // i0 is the same for the 32 lanes of a warp: every lane takes part in the shuffles
    for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < total; i0 += step) {
      const uint64_t i = i0 + (threadIdx.x & 31u);
      const uint32_t o = (uint32_t)(i >> lanes_log2), sub = (uint32_t)(i & (S - 1));
      ACC acc;
      if (o < a.n_out) {
        int64_t base[NOPS];
        offsets<NOPS>(o, a.out, base);
        const uint32_t l0 = (uint32_t)min((uint64_t)a.n_loop, (uint64_t)sub * per);
        entry_range<NOPS, ACC>(a, base, l0, (uint32_t)min((uint64_t)a.n_loop, (uint64_t)l0 + per), acc);
      }
      if (F64OUT) {
        double v = acc.as_double();
        for (uint32_t d = S >> 1; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
        if (o < a.n_out && sub == 0) store_out((double*)out, o, v, a.accum);
        continue;
      }
      float2 v = acc.get();
      for (uint32_t d = S >> 1; d > 0; d >>= 1) {
        Acc t;
        t.hi = v.x;
        t.lo = v.y;
        t.add(make_float2(__shfl_xor_sync(0xffffffffu, v.x, d), __shfl_xor_sync(0xffffffffu, v.y, d)));
        v = t.get();
      }
      if (o < a.n_out && sub == 0) store_out((float2*)out, o, v, a.accum);
    }
    return;
  }
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t o = blockIdx.x * blockDim.x + threadIdx.x; o < a.n_out; o += stride) {
    int64_t base[NOPS];
    offsets<NOPS>(o, a.out, base);
    const ACC v = entry<NOPS, ACC>(a, base);
    if (F64OUT)
      store_out((double*)out, o, v.as_double(), a.accum);
    else
      store_out((float2*)out, o, v.get(), a.accum);
  }
}

// one block per output entry for long sums (deterministic fixed-shape tree);
// with F64OUT every partial sum, the shuffles and the block sum are FP64
template <int NOPS, bool F64OUT>
__global__ void __launch_bounds__(256) k_gather_block(const GatherArgs a, void* __restrict__ out) {
  __shared__ float2 red[8];
  __shared__ double redd[8];
  pdl_wait();
  pdl_launch_dependents();
  for (uint32_t o = blockIdx.x; o < a.n_out; o += gridDim.x) {
    int64_t base[NOPS];
    offsets<NOPS>(o, a.out, base);
    if (F64OUT) {
      AccD acc;
      for (uint32_t l = threadIdx.x; l < a.n_loop; l += blockDim.x) {
        int64_t lo[NOPS];
        offsets<NOPS>(l, a.loop, lo);
#pragma unroll
        for (int j = 0; j < NOPS; ++j) lo[j] += base[j];
        acc.add(term<NOPS>(a, lo));
      }
      double v = acc.s;
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
      if ((threadIdx.x & 31) == 0) redd[threadIdx.x >> 5] = v;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += redd[w];
        store_out((double*)out, o, t, a.accum);
      }
      __syncthreads();
      continue;
    }
    Acc acc;
    for (uint32_t l = threadIdx.x; l < a.n_loop; l += blockDim.x) {
      int64_t lo[NOPS];
      offsets<NOPS>(l, a.loop, lo);
#pragma unroll
      for (int j = 0; j < NOPS; ++j) lo[j] += base[j];
      acc.add(term<NOPS>(a, lo));
    }
    float2 v = acc.get();
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      Acc t;
      t.hi = v.x;
      t.lo = v.y;
      t.add(make_float2(__shfl_xor_sync(0xffffffffu, v.x, s), __shfl_xor_sync(0xffffffffu, v.y, s)));
      v = t.get();
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      Acc t;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t.add(red[w]);
      store_out((float2*)out, o, t.get(), a.accum);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ split writer
// GEMM operand [rows][Kp]: out modes = row modes (a.out) x K modes (a.kmodes).
// A block takes a tile of kTR rows x kTK k: (1) the per-operand offsets of
// the tile's rows and ks go to shared memory (the offset of an entry is
// row part + k part), (2) the entries are computed in the order in which the
// leading operand is contiguous (rows or k fastest) and staged in shared
// memory, (3) every thread splits 8 consecutive k of one row into pieces and
// writes each piece plane with 16-byte stores.
constexpr int kTR = 32, kTK = 64;

template <int NOPS, int KIND, int NP>
__global__ void __launch_bounds__(256) k_gather_split(const GatherArgs a, void* __restrict__ dst) {
  __shared__ int64_t rowoff[kTR][NOPS];
  __shared__ int64_t koff[kTK][NOPS];
  __shared__ float2 tile[kTR][kTK + 1];
  pdl_wait();
  pdl_launch_dependents();
  const uint32_t n_rt = (a.n_rows + kTR - 1) / kTR;
  const uint32_t n_kt = (a.Kp + kTK - 1) / kTK;
  const int64_t piece = (int64_t)a.n_rows * a.Kp;
  const int tid = threadIdx.x;
  for (uint32_t t = blockIdx.x; t < n_rt * n_kt; t += gridDim.x) {
    const uint32_t rt = t / n_kt, kt = t - rt * n_kt;
    const uint32_t r0 = rt * kTR, k0 = kt * kTK;
    if (tid < kTR) {
      int64_t o[NOPS];
      offsets<NOPS>(min(r0 + tid, a.n_rows - 1), a.out, o);
#pragma unroll
      for (int j = 0; j < NOPS; ++j) rowoff[tid][j] = o[j];
    } else if (tid < kTR + kTK) {
      int64_t o[NOPS];
      offsets<NOPS>(min(k0 + (tid - kTR), a.K - 1), a.kmodes, o);
#pragma unroll
      for (int j = 0; j < NOPS; ++j) koff[tid - kTR][j] = o[j];
    }
    __syncthreads();
#pragma unroll 2
    for (int e = tid; e < kTR * kTK; e += 256) {
      int r, k;
      if (a.row_fast) {
        r = e % kTR;
        k = e / kTR;
      } else {
        k = e % kTK;
        r = e / kTK;
      }
      float2 v = make_float2(0.f, 0.f);
      if (r0 + r < a.n_rows && k0 + k < a.K) {
        int64_t b[NOPS];
#pragma unroll
        for (int j = 0; j < NOPS; ++j) b[j] = rowoff[r][j] + koff[k][j];
        v = entry<NOPS, Acc>(a, b).get();
      }
      tile[r][k] = v;
    }
    __syncthreads();
    {
      const int r = tid >> 3, kk = (tid & 7) * 8;
      const uint32_t row = r0 + r, kb = k0 + kk;
      const bool in = row < a.n_rows && kb < a.Kp;
      if (KIND == 0) {
        // BF16 pieces on the grid of this row's 64-entry k-block (the 8
        // threads of a row are 8 consecutive lanes)
        float m = 0.f;
#pragma unroll
        for (int e = 0; e < 8; ++e) m = fmaxf(m, fabsf(tile[r][kk + e].x));
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 4));
        const int E = grid_exp(m);
        if (in) {
          const int64_t base = (int64_t)row * a.Kp + kb;
          __nv_bfloat16 h[3][8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            float pc[3];
            grid_pieces(tile[r][kk + e], E, pc);
#pragma unroll
            for (int p = 0; p < 3; ++p) h[p][e] = __float2bfloat16_rn(pc[p]);  // exact
          }
          __nv_bfloat16* d = (__nv_bfloat16*)dst;
#pragma unroll
          for (int p = 0; p < 3; ++p) *(uint4*)(d + p * piece + base) = *(const uint4*)h[p];
        }
      } else if (in) {
        const int64_t base = (int64_t)row * a.Kp + kb;
        {
          float f[NP][8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const float2 v = tile[r][kk + e];
            const float t0 = tf32_rna(v.x);
            f[0][e] = t0;
            if (NP > 1) f[NP - 1][e] = tf32_rna(__fadd_rn(__fsub_rn(v.x, t0), v.y));
          }
          float* d = (float*)dst;
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            *(float4*)(d + p * piece + base) = *(const float4*)&f[p][0];
            *(float4*)(d + p * piece + base + 4) = *(const float4*)&f[p][4];
          }
        }
      }
    }
    __syncthreads();
  }
}

template <int NOPS>
cudaError_t launch_n(const GatherArgs& a, void* out, int sm, cudaStream_t st) {
  if (a.mode == GW_SPLIT_BF16X3 || a.mode == GW_SPLIT_TF32X2 || a.mode == GW_SPLIT_TF32) {
    const int64_t tiles = (int64_t)((a.n_rows + kTR - 1) / kTR) * ((a.Kp + kTK - 1) / kTK);
    if (tiles <= 0) return cudaSuccess;
    int64_t g = tiles < (int64_t)sm * 8 ? tiles : (int64_t)sm * 8;
    if (a.mode == GW_SPLIT_BF16X3) return launch_k(k_gather_split<NOPS, 0, 3>, dim3((unsigned)g), dim3(256), 0, st, a, out);
    if (a.mode == GW_SPLIT_TF32X2) return launch_k(k_gather_split<NOPS, 1, 2>, dim3((unsigned)g), dim3(256), 0, st, a, out);
    return launch_k(k_gather_split<NOPS, 1, 1>, dim3((unsigned)g), dim3(256), 0, st, a, out);
  }
  if (a.n_out == 0) return cudaSuccess;
  const bool f64 = a.mode == GW_DENSE_F64;
  const bool block_mode = a.n_loop >= 1024 && a.n_out <= (uint32_t)sm * 16;
  if (block_mode) {
    const uint32_t g = a.n_out < (uint32_t)sm * 16 ? a.n_out : (uint32_t)sm * 16;
    if (f64) return launch_k(k_gather_block<NOPS, true>, dim3(g), dim3(256), 0, st, a, out);
    return launch_k(k_gather_block<NOPS, false>, dim3(g), dim3(256), 0, st, a, out);
  }
  const int lg = a.loop.n > 0 ? lanes_for_long_sum(a.n_out, a.n_loop, sm) : 0;
  int64_t g = (((int64_t)a.n_out << lg) + 255) / 256;
  if (g > (int64_t)sm * 32) g = (int64_t)sm * 32;
  if (f64) return launch_k(k_gather_dense<NOPS, true>, dim3((unsigned)g), dim3(256), 0, st, a, out, lg);
  return launch_k(k_gather_dense<NOPS, false>, dim3((unsigned)g), dim3(256), 0, st, a, out, lg);
}

}  // namespace

FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  uint32_t l = 0;
  while (l < 32 && (1ull << l) < d) ++l;
  f.shift = l;
  f.magic = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
  if (d == 1) f.magic = 0, f.shift = 0;
  return f;
}

cudaError_t launch_gather(const GatherArgs& a, void* out, int sm, cudaStream_t st) {
  switch (a.nops) {
    case 1: return launch_n<1>(a, out, sm, st);
    case 2: return launch_n<2>(a, out, sm, st);
    case 3: return launch_n<3>(a, out, sm, st);
    case 4: return launch_n<4>(a, out, sm, st);
    case 5: return launch_n<5>(a, out, sm, st);
    case 6: return launch_n<6>(a, out, sm, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace qtpu
