// Persistent batched execution: the gather launches of many networks in one
// kernel.
//
// Section 6.1 step 4 contracts each evaluated network; a batch of small
// networks is bound by launch latency, not by arithmetic or bandwidth.  Here
// every gather launch of every network in the batch is a task of one
// persistent launch: blocks claim work units (256 outputs of a task, or one
// output of a long sum) from a global counter in task order, which is level
// by level across networks, and before a unit is processed the block waits
// until every unit of the task's predecessor (the previous launch of the
// same network) is done.  Units are claimed in order and a block only waits
// on earlier tasks whose units are all claimed by running blocks, so the wait
// ends; it is still bounded by a time limit, after which the block sets the
// network's status bit and an abort flag, and every later unit completes
// without computing and flags its own network (the host reads QTPU_ETIMEOUT
// from the status word of every network whose result is incomplete).  Operands are read with L2-only loads: producers and consumers of
// an intermediate run on different SMs inside the same launch.
#include <cuda_runtime.h>

#include "arith.cuh"
#include "common.cuh"
#include "kernels.h"

namespace qtpu {

namespace {
using namespace arith;

__device__ __forceinline__ float2 load_cg(const void* p, int dt, int64_t i) {
  if (dt == DT_F64) {
    const double x = __ldcg((const double*)p + i);
    return decode_f64(x);
  }
  if (dt == DT_F32X2) return __ldcg((const float2*)p + i);
  return make_float2(__ldcg((const float*)p + i), 0.f);
}

__device__ __forceinline__ float2 term_cg(const GatherArgs& a, const int64_t* off) {
  float2 v = load_cg(a.ptr[0], a.dt[0], off[0]);
  for (int j = 1; j < a.nops; ++j) v = mul_pair(v, load_cg(a.ptr[j], a.dt[j], off[j]));
  return v;
}

__device__ __forceinline__ void offsets_n(uint32_t o, const GModes& t, int nops, int64_t* off) {
  for (int j = 0; j < nops; ++j) off[j] = 0;
  for (int m = t.n - 1; m >= 0; --m) {
    const uint32_t q = fdiv(o, t.div[m]);
    const uint32_t i = o - q * t.dim[m];
    o = q;
    for (int j = 0; j < nops; ++j) off[j] += (int64_t)i * t.stride[m][j];
  }
}

// one output: the loop modes walked with running offsets (no divisions)
template <typename ACC>
__device__ ACC dense_entry(const GatherArgs& a, uint32_t o) {
  int64_t off[kMaxOps];
  offsets_n(o, a.out, a.nops, off);
  ACC acc;
  if (a.loop.n == 0) {
    acc.add(term_cg(a, off));
    return acc;
  }
  uint32_t idx[kMaxModes];
  for (int m = 0; m < a.loop.n; ++m) idx[m] = 0;
  for (uint32_t l = 0; l < a.n_loop; ++l) {
    acc.add(term_cg(a, off));
    int m = a.loop.n - 1;
    ++idx[m];
    for (int j = 0; j < a.nops; ++j) off[j] += a.loop.stride[m][j];
    while (m > 0 && idx[m] == a.loop.dim[m]) {
      for (int j = 0; j < a.nops; ++j) off[j] -= (int64_t)a.loop.dim[m] * a.loop.stride[m][j];
      idx[m] = 0;
      --m;
      ++idx[m];
      for (int j = 0; j < a.nops; ++j) off[j] += a.loop.stride[m][j];
    }
  }
  return acc;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__global__ void __launch_bounds__(256) k_batch_persistent(const BatchTask* __restrict__ tasks, int n_tasks,
                                                          const uint64_t* __restrict__ unit_start,
                                                          unsigned long long* next_unit, uint32_t* done,
                                                          uint64_t limit_ns, int* abort_flag) {
  __shared__ int s_task;
  __shared__ unsigned long long s_unit;
  __shared__ int s_run;
  __shared__ double redd[8];
  __shared__ float2 red[8];
  const uint64_t total = unit_start[n_tasks];
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned long long u = atomicAdd(next_unit, 1ull);
      s_unit = u;
      if (u < total) {
        int lo = 0, hi = n_tasks - 1;  // the task t with unit_start[t] <= u < unit_start[t + 1]
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (unit_start[mid] <= u)
            lo = mid;
          else
            hi = mid - 1;
        }
        s_task = lo;
        const BatchTask& T = tasks[lo];
        int run = *(volatile int*)abort_flag == 0;
        if (!run) atomicOr(T.status, ST_TIMEOUT_DEP);  // skipped: this network's result is not valid
        if (run && T.dep >= 0) {
          const uint64_t t0 = global_ns();
          uint32_t spin = 0;
          while (ld_acquire(&done[T.dep]) < T.dep_units) {
            if (*(volatile int*)abort_flag) {
              atomicOr(T.status, ST_TIMEOUT_DEP);
              run = 0;
              break;
            }
            if (global_ns() - t0 > limit_ns) {
              atomicOr(T.status, ST_TIMEOUT_DEP);
              atomicExch(abort_flag, 1);
              run = 0;
              break;
            }
            __nanosleep(spin < 256 ? 32 : 256);
            ++spin;
          }
        }
        s_run = run;
      }
    }
    __syncthreads();
    const unsigned long long u = s_unit;
    if (u >= total) return;
    const int t = s_task;
    const BatchTask& T = tasks[t];
    const GatherArgs& a = T.g;
    const uint32_t unit = (uint32_t)(u - unit_start[t]);
    if (s_run) {
      if (!T.block_mode) {
        const uint32_t o = unit * blockDim.x + threadIdx.x;
        if (o < a.n_out) {
          if (T.f64out)
            ((double*)T.dst)[o] = dense_entry<AccD>(a, o).as_double();
          else
            ((float2*)T.dst)[o] = dense_entry<Acc>(a, o).get();
        }
      } else {
        // one output, its loop split over the block; fixed-shape tree
        const uint32_t o = unit;
        int64_t base[kMaxOps];
        offsets_n(o, a.out, a.nops, base);
        if (T.f64out) {
          AccD acc;
          for (uint32_t l = threadIdx.x; l < a.n_loop; l += blockDim.x) {
            int64_t off[kMaxOps];
            offsets_n(l, a.loop, a.nops, off);
            for (int j = 0; j < a.nops; ++j) off[j] += base[j];
            acc.add(term_cg(a, off));
          }
          double v = acc.s;
          for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
          if ((threadIdx.x & 31) == 0) redd[threadIdx.x >> 5] = v;
          __syncthreads();
          if (threadIdx.x == 0) {
            double r = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += redd[w];
            ((double*)T.dst)[o] = r;
          }
        } else {
          Acc acc;
          for (uint32_t l = threadIdx.x; l < a.n_loop; l += blockDim.x) {
            int64_t off[kMaxOps];
            offsets_n(l, a.loop, a.nops, off);
            for (int j = 0; j < a.nops; ++j) off[j] += base[j];
            acc.add(term_cg(a, off));
          }
          float2 v = acc.get();
          for (int s = 16; s > 0; s >>= 1) v = pair_sum(v, make_float2(__shfl_xor_sync(0xffffffffu, v.x, s),
                                                                      __shfl_xor_sync(0xffffffffu, v.y, s)));
          if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
          __syncthreads();
          if (threadIdx.x == 0) {
            Acc r;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r.add(red[w]);
            ((float2*)T.dst)[o] = r.get();
          }
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&done[t], 1u);
    }
  }
}

}  // namespace

cudaError_t launch_batch_persistent(const BatchTask* tasks, int n_tasks, const uint64_t* unit_start,
                                    unsigned long long* next_unit, uint32_t* done, uint64_t limit_ns, int* abort_flag,
                                    int grid, cudaStream_t st) {
  if (n_tasks <= 0) return cudaSuccess;
  k_batch_persistent<<<grid, 256, 0, st>>>(tasks, n_tasks, unit_start, next_unit, done, limit_ns, abort_flag);
  return cudaGetLastError();
}

}  // namespace qtpu
