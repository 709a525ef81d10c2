// Typed fast path of the gather kernels.
//
// Same computation as kernels_gather.cu,
//   value(o) = sum_l prod_j X_j[...],
// specialised for the shapes the h-TN contraction produces: at most two
// large operands (a QT or an intermediate, typed at compile time as FP64 or
// FP32 pair), and any number of small leaves -- the QPD coefficient tensors
// absorbed into the step (section 4.1) -- whose product over their joint
// index space is computed once per block into a table W in shared memory.
// Each term then costs one typed load per large operand, one shared-memory
// load and one compensated multiply-add.
#include <cuda_bf16.h>


#include "arith.cuh"
#include "common.cuh"
#include "kernels.h"

namespace qtpu {

namespace {
using namespace arith;

// W[u] = prod over the small operands of their entry at u (u dense over a.wmodes)
// entry u of W
__device__ __forceinline__ float2 w_entry(const GatherArgs& a, uint32_t u) {
  const int nsmall = a.nops - a.nbig;
  int64_t off[kMaxOps];
  for (int j = 0; j < nsmall; ++j) off[j] = 0;
  uint32_t o = u;
  for (int m = a.wmodes.n - 1; m >= 0; --m) {
    const uint32_t q = fdiv(o, a.wmodes.div[m]);
    const uint32_t i = o - q * a.wmodes.dim[m];
    o = q;
    for (int j = 0; j < nsmall; ++j) off[j] += (int64_t)i * a.wmodes.stride[m][j];
  }
  float2 v = load_any(a.ptr[a.nbig], a.dt[a.nbig], off[0]);
  for (int j = 1; j < nsmall; ++j) v = mul_pair(v, load_any(a.ptr[a.nbig + j], a.dt[a.nbig + j], off[j]));
  return v;
}

// a large W, once per launch: one entry per thread
__global__ void __launch_bounds__(256) k_build_w(const GatherArgs a, float2* __restrict__ wg) {
  pdl_wait();
  pdl_launch_dependents();
  const uint32_t u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < a.w_size) wg[u] = w_entry(a, u);
}

// W from the buffer filled by the preceding k_build_w launch
__device__ __forceinline__ void copy_w(const GatherArgs& a, float2* W) {
  pdl_wait();
  for (uint32_t u = threadIdx.x; u < a.w_size; u += blockDim.x) W[u] = a.wg[u];
}

__device__ void build_w(const GatherArgs& a, float2* W) {
  const int nsmall = a.nops - a.nbig;
  for (uint32_t u = threadIdx.x; u < a.w_size; u += blockDim.x) {
    int64_t off[kMaxOps];
    for (int j = 0; j < nsmall; ++j) off[j] = 0;
    uint32_t o = u;
    for (int m = a.wmodes.n - 1; m >= 0; --m) {
      const uint32_t q = fdiv(o, a.wmodes.div[m]);
      const uint32_t i = o - q * a.wmodes.dim[m];
      o = q;
      for (int j = 0; j < nsmall; ++j) off[j] += (int64_t)i * a.wmodes.stride[m][j];
    }
    float2 v = load_any(a.ptr[a.nbig], a.dt[a.nbig], off[0]);
    for (int j = 1; j < nsmall; ++j) v = mul_pair(v, load_any(a.ptr[a.nbig + j], a.dt[a.nbig + j], off[j]));
    W[u] = v;
  }
}

// Offsets of every loop position (summed terms) per operand, built once per
// block when the loop is short: the terms of an entry then issue independent
// loads instead of walking the loop modes one dependent step at a time.
constexpr uint32_t kLoopTab = 64;
template <int NOPS>
__device__ void build_loop_tab(const GatherArgs& a, int64_t (*lt)[NOPS]) {
  if (a.n_loop > kLoopTab || a.loop.n == 0) return;
  for (uint32_t l = threadIdx.x; l < a.n_loop; l += blockDim.x) offsets<NOPS>(l, a.loop, lt[l]);
}
__device__ __forceinline__ bool use_loop_tab(const GatherArgs& a) { return a.loop.n > 0 && a.n_loop <= kLoopTab; }

template <int NB, int DT0, int DT1, bool HW>
struct Op {
  static constexpr int NOPS = NB + (HW ? 1 : 0);
  __device__ static __forceinline__ float2 term(const GatherArgs& a, const float2* W, const int64_t* off) {
    float2 v = load_pair<DT0>(a.ptr[0], off[0]);
    if (NB == 2) v = mul_pair(v, load_pair<DT1>(a.ptr[1], off[1]));
    if (HW) v = mul_pair(v, W[off[NB]]);
    return v;
  }
  template <typename ACC>
  __device__ static __forceinline__ ACC entry(const GatherArgs& a, const float2* W, const int64_t* base,
                                              const int64_t (*lt)[NOPS]) {
    ACC acc;
    if (a.loop.n == 0) {
      acc.add(term(a, W, base));
      return acc;
    }
    if (use_loop_tab(a)) {
      if (a.n_loop == 4) {  // a wire CT's loop: unrolled, no loop control
#pragma unroll
        for (uint32_t l = 0; l < 4; ++l) {
          int64_t off[NOPS];
#pragma unroll
          for (int j = 0; j < NOPS; ++j) off[j] = base[j] + lt[l][j];
          acc.add(term(a, W, off));
        }
        return acc;
      }
#pragma unroll 4
      for (uint32_t l = 0; l < a.n_loop; ++l) {
        int64_t off[NOPS];
#pragma unroll
        for (int j = 0; j < NOPS; ++j) off[j] = base[j] + lt[l][j];
        acc.add(term(a, W, off));
      }
      return acc;
    }
    int64_t off[NOPS];
#pragma unroll
    for (int j = 0; j < NOPS; ++j) off[j] = base[j];
    if (a.loop.n == 1) {
      const uint32_t d = a.loop.dim[0];
      for (uint32_t i = 0; i < d; ++i) {
        acc.add(term(a, W, off));
#pragma unroll
        for (int j = 0; j < NOPS; ++j) off[j] += a.loop.stride[0][j];
      }
      return acc;
    }
    walk(a, W, off, 0, a.n_loop, acc);
    return acc;
  }
  // loop positions [l0, l1) of the entry at base as an odometer walk over the
  // loop modes, started from the digits of l0
  template <typename ACC>
  __device__ static __forceinline__ void range(const GatherArgs& a, const float2* W, const int64_t* base,
                                               uint32_t l0, uint32_t l1, ACC& acc) {
    if (l0 >= l1) return;
    int64_t off[NOPS];
#pragma unroll
    for (int j = 0; j < NOPS; ++j) off[j] = base[j];
    walk(a, W, off, l0, l1, acc);
  }
  template <typename ACC>
  __device__ static __forceinline__ void walk(const GatherArgs& a, const float2* W, int64_t* off, uint32_t l0,
                                              uint32_t l1, ACC& acc) {
    uint32_t idx[kMaxModes];
    for (int m = 0; m < a.loop.n; ++m) idx[m] = 0;
    if (l0 > 0) digits<NOPS>(l0, a.loop, idx, off);
    for (uint32_t l = l0; l < l1; ++l) {
      acc.add(term(a, W, off));
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
};

// F entries that share every large-operand offset (they differ only along a
// mode that W alone carries): W offsets per entry in wof[F]
template <int DT0, int F>
__device__ __forceinline__ void entry_fan(const GatherArgs& a, const float2* W, int64_t xo, const int* wof,
                                          float2* v, const int64_t (*lt)[2]) {
  Acc acc[F];
  if (a.loop.n == 0) {
    const float2 x = load_pair<DT0>(a.ptr[0], xo);
#pragma unroll
    for (int f = 0; f < F; ++f) v[f] = mul_pair(x, W[wof[f]]);
    return;
  }
  if (use_loop_tab(a) && a.n_loop == 4) {  // a wire CT's loop: unrolled, no loop control
#pragma unroll
    for (uint32_t l = 0; l < 4; ++l) {
      const float2 x = load_pair<DT0>(a.ptr[0], xo + lt[l][0]);
      const int ow = (int)lt[l][1];
#pragma unroll
      for (int f = 0; f < F; ++f) acc[f].add(mul_pair(x, W[wof[f] + ow]));
    }
  } else if (use_loop_tab(a)) {
#pragma unroll 4
    for (uint32_t l = 0; l < a.n_loop; ++l) {
      const float2 x = load_pair<DT0>(a.ptr[0], xo + lt[l][0]);
      const int ow = (int)lt[l][1];
#pragma unroll
      for (int f = 0; f < F; ++f) acc[f].add(mul_pair(x, W[wof[f] + ow]));
    }
  } else if (a.loop.n == 1) {
    const uint32_t d = a.loop.dim[0];
    const int64_t sx = a.loop.stride[0][0];
    const int sw = (int)a.loop.stride[0][1];
    for (uint32_t i = 0; i < d; ++i) {
      const float2 x = load_pair<DT0>(a.ptr[0], xo + (int64_t)i * sx);
#pragma unroll
      for (int f = 0; f < F; ++f) acc[f].add(mul_pair(x, W[wof[f] + (int)i * sw]));
    }
  } else {
    uint32_t idx[kMaxModes];
    for (int m = 0; m < a.loop.n; ++m) idx[m] = 0;
    int64_t ox = xo;
    int ow = 0;
    for (uint32_t l = 0; l < a.n_loop; ++l) {
      const float2 x = load_pair<DT0>(a.ptr[0], ox);
#pragma unroll
      for (int f = 0; f < F; ++f) acc[f].add(mul_pair(x, W[wof[f] + ow]));
      int m = a.loop.n - 1;
      ++idx[m];
      ox += a.loop.stride[m][0];
      ow += (int)a.loop.stride[m][1];
      while (m > 0 && idx[m] == a.loop.dim[m]) {
        ox -= (int64_t)a.loop.dim[m] * a.loop.stride[m][0];
        ow -= (int)(a.loop.dim[m] * a.loop.stride[m][1]);
        idx[m] = 0;
        --m;
        ++idx[m];
        ox += a.loop.stride[m][0];
        ow += (int)a.loop.stride[m][1];
      }
    }
  }
#pragma unroll
  for (int f = 0; f < F; ++f) v[f] = acc[f].get();
}

// ------------------------------------------------------------ dense output
template <int NB, int DT0, int DT1, bool HW, bool F64OUT>
__global__ void __launch_bounds__(256) k_dense_fast(const GatherArgs a, void* __restrict__ out, int lanes_log2) {
  using O = Op<NB, DT0, DT1, HW>;
  using ACC = typename AccSel<F64OUT>::T;  // FP64 when the values are outputs
  extern __shared__ float2 W[];  // w_size entries (dynamic shared memory)
  __shared__ int64_t lt[kLoopTab][O::NOPS];
  if (HW) {
    if (a.wg)
      copy_w(a, W);
    else
      build_w(a, W);
  }
  build_loop_tab<O::NOPS>(a, lt);
  __syncthreads();
  pdl_wait();
  pdl_launch_dependents();
  if (lanes_log2 > 0) {
    // few outputs: 2^lanes_log2 consecutive lanes share an output, each
    // summing every 2^lanes_log2-th term of a tabulated loop, or a contiguous
    // run of a longer one; the partial sums then meet by shuffles
    // (compensated pairs, or FP64)
    const uint32_t S = 1u << lanes_log2;
    const bool tab = use_loop_tab(a);
    const uint32_t per = (a.n_loop + S - 1) / S;
    const uint64_t total = (uint64_t)a.n_out << lanes_log2;
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    // i0 is the same for the 32 lanes of a warp: every lane takes part in the shuffles
    for (uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < total; i0 += step) {
      const uint64_t i = i0 + (threadIdx.x & 31u);
      const uint32_t o = (uint32_t)(i >> lanes_log2), sub = (uint32_t)(i & (S - 1));
      ACC acc;
      if (o < a.n_out) {
        int64_t base[O::NOPS];
        offsets<O::NOPS>(o, a.out, base);
        if (tab) {
#pragma unroll 2
          for (uint32_t l = sub; l < a.n_loop; l += S) {
            int64_t off[O::NOPS];
#pragma unroll
            for (int j = 0; j < O::NOPS; ++j) off[j] = base[j] + lt[l][j];
            acc.add(O::term(a, W, off));
          }
        } else {
          const uint32_t l0 = (uint32_t)min((uint64_t)a.n_loop, (uint64_t)sub * per);
          O::range(a, W, base, l0, (uint32_t)min((uint64_t)a.n_loop, (uint64_t)l0 + per), acc);
        }
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
    int64_t base[O::NOPS];
    offsets<O::NOPS>(o, a.out, base);
    const ACC v = O::template entry<ACC>(a, W, base, lt);
    if (F64OUT)
      store_out((double*)out, o, v.as_double(), a.accum);
    else
      store_out((float2*)out, o, v.get(), a.accum);
  }
}

// ------------------------------------------------------------ dot reduction
// value(o) = sum over the loop of X0 * X1 for few outputs and a long loop.
// Block (c, o) walks its range of outer tuples; per tuple it stages the
// operand-0 tile in shared memory in operand 1's order (both global reads
// run along each operand's own unit stride), then multiplies it with the
// operand-1 tile read straight from global memory.
__host__ __device__ __forceinline__ uint32_t dot_slot(uint32_t u) { return u + (u >> 4); }  // padded: fewer bank conflicts

// F64: the values are outputs (the final dot of a slice).  Each thread then
// sums the products of at most kDotFold tuples (<= kDotFold * 8 terms) as a
// compensated FP32 pair, folds that sub-sum into an FP64 accumulator, and
// the block and chunk sums are FP64.  A pair sub-sum of n terms is within
// about n * 2^-47 of its exact value relative to the sum of the magnitudes,
// far inside FP64's own bound for the long sum (terms * 2^-53), so the
// output keeps FP64 accuracy while the FP64 pipe (1/64 of the FP32 rate on
// B300) runs once per kDotFold tuples instead of once per term.
constexpr int kDotFold = 8;

template <int DT0, int DT1, bool F64, int PER>
__global__ void __launch_bounds__(256) k_dot_fast(const GatherArgs a) {
  // PER >= tile_n / 256 entries of the tile per thread
  extern __shared__ float2 dsm[];
  const uint32_t T = a.tile_n;
  float2* sX = dsm;                                                   // T + T/16 slots
  int2* tx = reinterpret_cast<int2*>(dsm + dot_slot(T) + 1);          // v -> (slot, op-0 offset)
  int* ty = reinterpret_cast<int*>(tx + T);                           // slot -> op-1 offset
  for (uint32_t v = threadIdx.x; v < T; v += blockDim.x) {
    int64_t off[2];
    offsets<2>(v, a.kmodes, off);
    tx[v] = make_int2((int)dot_slot((uint32_t)off[1]), (int)off[0]);
    int64_t yo[1];
    offsets<1>(v, a.wmodes, yo);
    ty[v] = (int)yo[0];
  }
  __syncthreads();
  pdl_wait();
  pdl_launch_dependents();
  const uint32_t o = blockIdx.y;
  int64_t base[2];
  offsets<2>(o, a.out, base);
  const uint32_t per = (a.n_outer + a.chunks - 1) / a.chunks;
  const uint32_t t0 = blockIdx.x * per;
  const uint32_t t1 = min(a.n_outer, t0 + per);
  const void* X = a.ptr[0];
  const void* Y = a.ptr[1];
  Acc acc;
  double accd = 0.0;
  int fold = 0;
  // two register buffers: the loads of the next two tuples are in flight
  // while the current tuple is multiplied (the buffers alternate, so no
  // register copy waits on a load)
  float2 xa[PER], ya[PER], xb[PER], yb[PER];
  auto load = [&](uint32_t t, float2* xv, float2* yv) {
    int64_t ot[2];
    offsets<2>(t, a.loop, ot);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const uint32_t v = threadIdx.x + k * 256;
      if (v < T) {
        xv[k] = load_pair<DT0>(X, base[0] + ot[0] + tx[v].y);
        yv[k] = load_pair<DT1>(Y, base[1] + ot[1] + ty[v]);
      }
    }
  };
  auto step = [&](uint32_t t, float2* xv, float2* yv) {
    __syncthreads();  // the previous tuple's tile is consumed
    float2 yc[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const uint32_t v = threadIdx.x + k * 256;
      if (v < T) sX[tx[v].x] = xv[k];
      yc[k] = yv[k];
    }
    __syncthreads();
    if (t + 2 < t1) load(t + 2, xv, yv);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const uint32_t u = threadIdx.x + k * 256;
      if (u < T) acc.add(mul_pair(sX[dot_slot(u)], yc[k]));
    }
    if (F64 && ++fold == kDotFold) {
      accd += acc.as_double();
      acc = Acc();
      fold = 0;
    }
  };
  if (t0 < t1) load(t0, xa, ya);
  if (t0 + 1 < t1) load(t0 + 1, xb, yb);
  for (uint32_t t = t0; t < t1; t += 2) {
    step(t, xa, ya);
    if (t + 1 < t1) step(t + 1, xb, yb);
  }
  if (F64) {
    // FP64 block sum -> scratch[o][c] (the scratch holds doubles here)
    __shared__ double redd[8];
    double v = accd + acc.as_double();
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
    if ((threadIdx.x & 31) == 0) redd[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += redd[w];
      reinterpret_cast<double*>(a.scratch)[(size_t)o * a.chunks + blockIdx.x] = t;
    }
    return;
  }
  // block sum (compensated) -> scratch[o][c]
  __shared__ float2 red[8];
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
    for (int w = 0; w < 8; ++w) t.add(red[w]);
    a.scratch[(size_t)o * a.chunks + blockIdx.x] = t.get();
  }
}

// sum of the chunk partials of every output: FP64 partials summed in FP64
// (F64OUT), or compensated pairs
template <bool F64OUT>
__global__ void __launch_bounds__(256) k_dot_finish(const float2* __restrict__ part, uint32_t n_out,
                                                    uint32_t chunks, void* __restrict__ out, int accum) {
  pdl_wait();
  pdl_launch_dependents();
  for (uint32_t o = blockIdx.x * blockDim.x + threadIdx.x; o < n_out; o += gridDim.x * blockDim.x) {
    if (F64OUT) {
      const double* pd = reinterpret_cast<const double*>(part);
      double s = 0.0;
      for (uint32_t c = 0; c < chunks; ++c) s += pd[(size_t)o * chunks + c];
      store_out((double*)out, o, s, accum);
      continue;
    }
    Acc acc;
    for (uint32_t c = 0; c < chunks; ++c) acc.add(part[(size_t)o * chunks + c]);
    store_out((float2*)out, o, acc.get(), accum);
  }
}

size_t dot_smem_bytes(uint32_t T) { return (dot_slot(T) + 1) * sizeof(float2) + T * (sizeof(int2) + sizeof(int)); }

template <int DT0, int DT1, int PER>
cudaError_t dot_main(const GatherArgs& a, size_t sm_bytes, bool f64, cudaStream_t st) {
  auto kern = f64 ? k_dot_fast<DT0, DT1, true, PER> : k_dot_fast<DT0, DT1, false, PER>;
  cudaError_t e = cudaSuccess;
  if (sm_bytes > 40960) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_bytes);
  if (e != cudaSuccess) return e;
  return launch_k(kern, dim3(a.chunks, a.n_out), dim3(256), sm_bytes, st, a);
}

template <int DT0, int DT1>
cudaError_t dot_launch(const GatherArgs& a, void* out, cudaStream_t st) {
  const size_t sm_bytes = dot_smem_bytes(a.tile_n);
  const bool f64 = a.mode == GW_DENSE_F64;
  // tile entries per thread, rounded up to an instantiated count
  const uint32_t per = (a.tile_n + 255) / 256;
  cudaError_t e = per <= 2   ? dot_main<DT0, DT1, 2>(a, sm_bytes, f64, st)
                  : per <= 4 ? dot_main<DT0, DT1, 4>(a, sm_bytes, f64, st)
                  : per <= 6 ? dot_main<DT0, DT1, 6>(a, sm_bytes, f64, st)
                             : dot_main<DT0, DT1, kDotMaxTile / 256>(a, sm_bytes, f64, st);
  if (e != cudaSuccess) return e;
  const uint32_t g = (a.n_out + 255) / 256;
  const float2* part = a.scratch;
  if (f64) return launch_k(k_dot_finish<true>, dim3(g), dim3(256), 0, st, part, a.n_out, a.chunks, out, a.accum);
  return launch_k(k_dot_finish<false>, dim3(g), dim3(256), 0, st, part, a.n_out, a.chunks, out, a.accum);
}

// ------------------------------------------------------------ split output
constexpr int kTR = 32, kTK = 64;

template <int DT0, bool HW, int KIND, int NP, int F>
__global__ void __launch_bounds__(256) k_split_fast(const GatherArgs a, void* __restrict__ dst) {
  using O = Op<1, DT0, DT0, HW>;
  constexpr int NOPS = O::NOPS;
  extern __shared__ float2 W[];  // w_size entries (dynamic shared memory)
  __shared__ int64_t rowoff[kTR][NOPS];
  __shared__ int64_t koff[kTK][NOPS];
  __shared__ float2 tile[kTR][kTK + 1];
  __shared__ int64_t lt[kLoopTab][NOPS];
  if (HW) build_w(a, W);
  build_loop_tab<NOPS>(a, lt);
  __syncthreads();
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
    if (F > 1) {
      // work item = F entries along the fan mode (rows or ks), one operand load each
      constexpr int NI = kTR * kTK / F;
#pragma unroll
      for (int e = tid; e < NI; e += 256) {
        int r, k;
        if (a.fan == 2) {  // F consecutive rows
          const int ng = kTR / F;
          if (a.row_fast) {
            r = (e % ng) * F;
            k = e / ng;
          } else {
            k = e % kTK;
            r = (e / kTK) * F;
          }
        } else {  // F consecutive ks
          const int ng = kTK / F;
          if (a.row_fast) {
            r = e % kTR;
            k = (e / kTR) * F;
          } else {
            k = (e % ng) * F;
            r = e / ng;
          }
        }
        float2 v[F];
        if (r0 + r < a.n_rows && k0 + k < a.K) {
          int wof[F];
#pragma unroll
          for (int f = 0; f < F; ++f)
            wof[f] = (int)(a.fan == 2 ? rowoff[r + f][1] + koff[k][1] : rowoff[r][1] + koff[k + f][1]);
          entry_fan<DT0, F>(a, W, rowoff[r][0] + koff[k][0], wof, v, (const int64_t (*)[2])lt);
        } else {
#pragma unroll
          for (int f = 0; f < F; ++f) v[f] = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int f = 0; f < F; ++f) {
          const int rr = a.fan == 2 ? r + f : r, kk = a.fan == 2 ? k : k + f;
          const bool in = r0 + rr < a.n_rows && k0 + kk < a.K;
          tile[rr][kk] = in ? v[f] : make_float2(0.f, 0.f);
        }
      }
    } else if (a.loop.n == 0) {
      // one term per entry: every load of the tile issued before any use
      constexpr int PER = kTR * kTK / 256;
      float2 v[PER];
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int e = tid + u * 256;
        const int r = a.row_fast ? e % kTR : e / kTK;
        const int k = a.row_fast ? e / kTR : e % kTK;
        v[u] = r0 + r < a.n_rows && k0 + k < a.K ? load_pair<DT0>(a.ptr[0], rowoff[r][0] + koff[k][0])
                                                  : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int e = tid + u * 256;
        const int r = a.row_fast ? e % kTR : e / kTK;
        const int k = a.row_fast ? e / kTR : e % kTK;
        if (HW) v[u] = mul_pair(v[u], W[rowoff[r][NOPS - 1] + koff[k][NOPS - 1]]);
        tile[r][k] = v[u];
      }
    } else {
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
        v = O::template entry<Acc>(a, W, b, lt).get();
      }
      tile[r][k] = v;
    }
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

// ------------------------------------------------------------ split, one term
// Tiles like k_split_fast's (but 64 rows high) for entries of one term (a
// large operand, times W when small factors are absorbed), software-pipelined: a block loads
// its next tile into registers before it writes the current one, so the load
// latency overlaps the piece arithmetic, the stores and the barriers.  The
// index tables of the next tile are built during the current write.
// Tiles of TR rows x 64 k: with 64 rows each block has 32 KB of loads in
// flight, and three blocks per SM (80 registers a thread) 96 KB.
constexpr int kPipeTR = 64;
template <int DT0, bool HW, int KIND, int NP, int TR>
__global__ void __launch_bounds__(256, 3) k_split_pipe(const GatherArgs a, void* __restrict__ dst) {
  constexpr int NOPS = 1 + (HW ? 1 : 0);
  constexpr int PER = TR * kTK / 256;
  extern __shared__ float2 W[];  // w_size entries (dynamic shared memory)
  __shared__ int64_t rowoff[2][TR][NOPS];
  __shared__ int64_t koff[2][kTK][NOPS];
  __shared__ float2 tile[TR][kTK + 1];
  if (HW) build_w(a, W);
  __syncthreads();
  pdl_wait();
  pdl_launch_dependents();
  const uint32_t n_rt = (a.n_rows + TR - 1) / TR;
  const uint32_t n_kt = (a.Kp + kTK - 1) / kTK;
  const uint32_t n_tiles = n_rt * n_kt;
  const int64_t piece = (int64_t)a.n_rows * a.Kp;
  const int tid = threadIdx.x;
  auto tables = [&](uint32_t t, int buf) {
    const uint32_t rt = t / n_kt, kt = t - rt * n_kt;
    const uint32_t r0 = rt * TR, k0 = kt * kTK;
    if (tid < TR) {
      int64_t o[NOPS];
      offsets<NOPS>(min(r0 + tid, a.n_rows - 1), a.out, o);
#pragma unroll
      for (int j = 0; j < NOPS; ++j) rowoff[buf][tid][j] = o[j];
    } else if (tid < TR + kTK) {
      int64_t o[NOPS];
      offsets<NOPS>(min(k0 + (tid - TR), a.K - 1), a.kmodes, o);
#pragma unroll
      for (int j = 0; j < NOPS; ++j) koff[buf][tid - TR][j] = o[j];
    }
  };
  float2 v[PER];
  auto load = [&](uint32_t t, int buf) {
    const uint32_t rt = t / n_kt, kt = t - rt * n_kt;
    const uint32_t r0 = rt * TR, k0 = kt * kTK;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = tid + u * 256;
      const int r = a.row_fast ? e % TR : e / kTK;
      const int k = a.row_fast ? e / TR : e % kTK;
      v[u] = r0 + r < a.n_rows && k0 + k < a.K ? load_pair<DT0>(a.ptr[0], rowoff[buf][r][0] + koff[buf][k][0])
                                                : make_float2(0.f, 0.f);
    }
  };
  auto stage = [&](int buf) {  // registers -> tile (times W)
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = tid + u * 256;
      const int r = a.row_fast ? e % TR : e / kTK;
      const int k = a.row_fast ? e / TR : e % kTK;
      float2 x = v[u];
      if (HW) x = mul_pair(x, W[rowoff[buf][r][NOPS - 1] + koff[buf][k][NOPS - 1]]);
      tile[r][k] = x;
    }
  };
  uint32_t t = blockIdx.x;
  if (t >= n_tiles) return;
  tables(t, 0);
  __syncthreads();
  load(t, 0);
  stage(0);
  int buf = 0;
  if (t + gridDim.x < n_tiles) tables(t + gridDim.x, 1);
  __syncthreads();
  for (;;) {
    const uint32_t nt = t + gridDim.x;
    const bool more = nt < n_tiles;
    if (more) load(nt, buf ^ 1);  // in flight during this tile's write
    const uint32_t rt = t / n_kt, kt = t - rt * n_kt;
    const uint32_t r0 = rt * TR, k0 = kt * kTK;
#pragma unroll
    for (int rr = 0; rr < TR; rr += 32) {
      const int r = (tid >> 3) + rr, kk = (tid & 7) * 8;
      const uint32_t row = r0 + r, kb = k0 + kk;
      const bool in = row < a.n_rows && kb < a.Kp;
      if (KIND == 0) {
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
        float f[NP][8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const float2 x = tile[r][kk + e];
          const float t0 = tf32_rna(x.x);
          f[0][e] = t0;
          if (NP > 1) f[NP - 1][e] = tf32_rna(__fadd_rn(__fsub_rn(x.x, t0), x.y));
        }
        float* d = (float*)dst;
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          *(float4*)(d + p * piece + base) = *(const float4*)&f[p][0];
          *(float4*)(d + p * piece + base + 4) = *(const float4*)&f[p][4];
        }
      }
    }
    if (!more) break;
    __syncthreads();  // the tile and this tile's tables are consumed
    stage(buf ^ 1);
    if (nt + gridDim.x < n_tiles) tables(nt + gridDim.x, buf);
    __syncthreads();
    buf ^= 1;
    t = nt;
  }
}

// dynamic shared memory above the 48 KB default needs a one-time opt-in
template <typename K>
cudaError_t allow_smem(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kMaxW * sizeof(float2)));
}

template <int DT0, bool HW, int F>
cudaError_t split_f(const GatherArgs& a, void* out, int g, cudaStream_t st) {
  const size_t sm_bytes = HW ? a.w_size * sizeof(float2) : 0;
  cudaError_t e = cudaSuccess;
  if (a.mode == GW_SPLIT_BF16X3) {
    if (sm_bytes > 16384) e = allow_smem(k_split_fast<DT0, HW, 0, 3, F>);
    if (e == cudaSuccess) e = launch_k(k_split_fast<DT0, HW, 0, 3, F>, dim3(g), dim3(256), sm_bytes, st, a, out);
  } else if (a.mode == GW_SPLIT_TF32X2) {
    if (sm_bytes > 16384) e = allow_smem(k_split_fast<DT0, HW, 1, 2, F>);
    if (e == cudaSuccess) e = launch_k(k_split_fast<DT0, HW, 1, 2, F>, dim3(g), dim3(256), sm_bytes, st, a, out);
  } else {
    if (sm_bytes > 16384) e = allow_smem(k_split_fast<DT0, HW, 1, 1, F>);
    if (e == cudaSuccess) e = launch_k(k_split_fast<DT0, HW, 1, 1, F>, dim3(g), dim3(256), sm_bytes, st, a, out);
  }
  return e;
}

template <int DT0, bool HW>
cudaError_t split_dt(const GatherArgs& a, void* out, int sm, cudaStream_t st) {
  const int64_t tiles = (int64_t)((a.n_rows + kTR - 1) / kTR) * ((a.Kp + kTK - 1) / kTK);
  if (tiles <= 0) return cudaSuccess;
  // blocks loop over tiles; with a large W table fewer blocks, each building
  // the table once
  const int64_t cap = HW && a.w_size > 1024 ? (int64_t)sm * 4 : (int64_t)sm * 8;
  const int g = (int)(tiles < cap ? tiles : cap);
  if (a.loop.n == 0 && !(HW && a.fan)) {  // one term per entry: the pipelined kernel
    const size_t sm_bytes = HW ? a.w_size * sizeof(float2) : 0;
    auto go = [&](auto kernel) -> cudaError_t {
      if (sm_bytes > 16384) {
        cudaError_t e = allow_smem(kernel);
        if (e != cudaSuccess) return e;
      }
      // 64-row tiles, 80 registers a thread: 3 blocks of 256 per SM stay resident
      const int64_t tp = (int64_t)((a.n_rows + kPipeTR - 1) / kPipeTR) * ((a.Kp + kTK - 1) / kTK);
      const int gp = (int)(tp < (int64_t)sm * 3 ? tp : (int64_t)sm * 3);
      return launch_k(kernel, dim3(gp), dim3(256), sm_bytes, st, a, out);
    };
    if (a.mode == GW_SPLIT_BF16X3) return go(k_split_pipe<DT0, HW, 0, 3, kPipeTR>);
    if (a.mode == GW_SPLIT_TF32X2) return go(k_split_pipe<DT0, HW, 1, 2, kPipeTR>);
    return go(k_split_pipe<DT0, HW, 1, 1, kPipeTR>);
  }
  if (HW && a.fan && a.fan_f == 4) return split_f<DT0, HW, 4>(a, out, g, st);
  if (HW && a.fan && a.fan_f == 2) return split_f<DT0, HW, 2>(a, out, g, st);
  return split_f<DT0, HW, 1>(a, out, g, st);
}

template <int NB, int DT0, int DT1, bool HW>
cudaError_t dense_dt(const GatherArgs& a, void* out, int sm, cudaStream_t st) {
  if (a.n_out == 0) return cudaSuccess;
  // lanes per output: up to 8 while the SMs are not yet full and each lane
  // keeps at least 4 terms of a tabulated loop; for a longer loop, up to 32
  // when the outputs are few (each lane a run of at least 8 terms)
  int lg = 0;
  if (a.loop.n > 0 && a.n_loop <= kLoopTab)
    while (lg < 3 && (4u << (lg + 1)) <= a.n_loop && ((uint64_t)a.n_out << (lg + 1)) <= (uint64_t)sm * 4096) ++lg;
  else if (a.loop.n > 0)
    lg = lanes_for_long_sum(a.n_out, a.n_loop, sm);
  int64_t g = (((int64_t)a.n_out << lg) + 255) / 256;
  if (g > (int64_t)sm * 8) g = (int64_t)sm * 8;
  const size_t sm_bytes = HW ? a.w_size * sizeof(float2) : 0;
  cudaError_t e = cudaSuccess;
  if (a.mode == GW_DENSE_F64) {
    if (sm_bytes > 40960) e = allow_smem(k_dense_fast<NB, DT0, DT1, HW, true>);
    if (e == cudaSuccess) e = launch_k(k_dense_fast<NB, DT0, DT1, HW, true>, dim3((unsigned)g), dim3(256), sm_bytes, st, a, out, lg);
  } else {
    if (sm_bytes > 40960) e = allow_smem(k_dense_fast<NB, DT0, DT1, HW, false>);
    if (e == cudaSuccess) e = launch_k(k_dense_fast<NB, DT0, DT1, HW, false>, dim3((unsigned)g), dim3(256), sm_bytes, st, a, out, lg);
  }
  return e;
}

template <int NB, int DT0, int DT1>
cudaError_t dense_w(const GatherArgs& a, void* out, int sm, cudaStream_t st) {
  return a.w_size ? dense_dt<NB, DT0, DT1, true>(a, out, sm, st) : dense_dt<NB, DT0, DT1, false>(a, out, sm, st);
}

bool typed(int dt) { return dt == DT_F64 || dt == DT_F32X2; }

}  // namespace

cudaError_t launch_gather_fast(const GatherArgs& a, void* out, int sm, cudaStream_t st) {
  if (a.nbig < 1 || a.nbig > 2 || a.w_size > kMaxW) return cudaErrorNotSupported;
  for (int j = 0; j < a.nbig; ++j)
    if (!typed(a.dt[j])) return cudaErrorNotSupported;
  if (a.wg && a.w_size) {
    const cudaError_t e = launch_k(k_build_w, dim3((a.w_size + 255) / 256), dim3(256), 0, st, a, a.wg);
    if (e != cudaSuccess) return e;
  }
  const bool split = a.mode == GW_SPLIT_BF16X3 || a.mode == GW_SPLIT_TF32X2 || a.mode == GW_SPLIT_TF32;
  if (split) {
    if (a.nbig != 1) return cudaErrorNotSupported;
    if (a.dt[0] == DT_F64)
      return a.w_size ? split_dt<DT_F64, true>(a, out, sm, st) : split_dt<DT_F64, false>(a, out, sm, st);
    return a.w_size ? split_dt<DT_F32X2, true>(a, out, sm, st) : split_dt<DT_F32X2, false>(a, out, sm, st);
  }
  if (a.dot) {
    if (a.nbig != 2 || a.w_size || a.tile_n == 0 || a.tile_n > kDotMaxTile || a.chunks == 0 || a.n_out > 65535 ||
        (size_t)a.n_out * a.chunks > dot_scratch_entries(sm) || !a.scratch)
      return cudaErrorNotSupported;
    if (a.dt[0] == DT_F64)
      return a.dt[1] == DT_F64 ? dot_launch<DT_F64, DT_F64>(a, out, st) : dot_launch<DT_F64, DT_F32X2>(a, out, st);
    return a.dt[1] == DT_F64 ? dot_launch<DT_F32X2, DT_F64>(a, out, st) : dot_launch<DT_F32X2, DT_F32X2>(a, out, st);
  }
  // long sums over few outputs go to the block-reduction kernel of the generic path
  if (a.n_loop >= 1024 && a.n_out <= (uint32_t)sm * 16) return cudaErrorNotSupported;
  if (a.nbig == 1)
    return a.dt[0] == DT_F64 ? dense_w<1, DT_F64, DT_F64>(a, out, sm, st) : dense_w<1, DT_F32X2, DT_F64>(a, out, sm, st);
  if (a.dt[0] == DT_F64)
    return a.dt[1] == DT_F64 ? dense_w<2, DT_F64, DT_F64>(a, out, sm, st) : dense_w<2, DT_F64, DT_F32X2>(a, out, sm, st);
  return a.dt[1] == DT_F64 ? dense_w<2, DT_F32X2, DT_F64>(a, out, sm, st)
                           : dense_w<2, DT_F32X2, DT_F32X2>(a, out, sm, st);
}

}  // namespace qtpu
