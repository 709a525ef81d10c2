// Allocation-free pairwise contraction: C[b] = A[b] * B[b] on the tensor cores
// with every piece of scratch memory taken from one fixed device array.
//
// Who needs this: callers that must not allocate device memory at call time.
// Examples are code running inside a pre-sized memory pool or arena owned by
// someone else (a serving process that reserved the GPU's memory up front), a
// real-time loop where a cudaMalloc / cudaFree would synchronise the device or
// stall for an unbounded time, and hosts where the caller has no allocator at
// all (a plain C caller that only receives device pointers).  The regular
// entry points allocate their workspace when a network is planned; this one
// never allocates: its scratch is a file-scope __device__ array of
// kNoallocScratchBytes that every GPU which loads this library holds until the
// process exits.
//
// The scratch is shared by all calls and keeps the contents of the last call.
// Nothing in it must start at zero (every byte a call reads was written earlier
// in the same call), except the status word, which each call clears.  Calls
// whose GPU work overlaps (on different streams, or from different threads)
// race on the scratch: serialise them.
//
// Device-side failures: the GEMM's bounded waits (and a kernel that rejects
// its arguments) record a bit in the status word at the start of the scratch
// instead of faulting.  qtpu_noalloc_status waits for the caller's stream,
// copies that word to the host (no allocation: one 4-byte copy into a host
// variable), clears it and maps it to a status code, so a caller learns that
// C is not valid.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/qtpu_htn.h"
#include "exec.h"
#include "kernels.h"

namespace qtpu {

namespace {

constexpr size_t kNoallocScratchBytes = QTPU_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};  // device address of the array, per device

size_t up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool push(GModes& t, uint32_t d, int64_t s) {
  if (d == 1) return true;
  if (t.n >= kMaxModes) return false;
  t.dim[t.n] = d;
  t.div[t.n] = make_fastdiv(d);
  for (int j = 0; j < kMaxOps; ++j) t.stride[t.n][j] = 0;
  t.stride[t.n][0] = s;
  t.n++;
  return true;
}

qtpu_status fail(qtpu_status s, const char* msg) {
  set_global_error(msg);
  return s;
}

// device address of the scratch array on the current device (resolved once per
// device with that device current), or nullptr
void* scratch_base(int* dev_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  *dev_out = dev;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return nullptr;
    g_scratch_addr[dev] = p;
  }
  return g_scratch_addr[dev];
}

}  // namespace

// Scratch bytes a call of these sizes needs (status word, BF16x3 pieces of A
// and B, the FP32-pair product).
static size_t noalloc_need(int batch, int M, int N, int K, size_t* a_off, size_t* b_off, size_t* c_off) {
  const size_t Kp = up((size_t)K, 8);
  *a_off = 1024;
  *b_off = up(*a_off + 3ull * batch * M * Kp * 2, 1024);
  *c_off = up(*b_off + 3ull * batch * N * Kp * 2, 256);
  return *c_off + (size_t)batch * M * N * 8;
}

}  // namespace qtpu

using namespace qtpu;

extern "C" qtpu_status qtpu_pairwise_contract_noalloc(const double* A, const double* B, double* C, int batch,
                                                      int M, int N, int K, void* cuda_stream) {
  if (!A || !B || !C) return fail(QTPU_EINVAL, "noalloc: NULL pointer");
  if (batch < 1 || M < 1 || N < 1 || K < 1) return fail(QTPU_EINVAL, "noalloc: sizes must be >= 1");
  size_t a_off, b_off, c_off;
  const size_t need = noalloc_need(batch, M, N, K, &a_off, &b_off, &c_off);
  if (need > kNoallocScratchBytes) return fail(QTPU_ELIMIT, "noalloc: the sizes need more than the fixed scratch");
  // one-time set-up per device (the first call on a device): resolve the
  // array's device address with that device current
  int dev = 0;
  void* base = scratch_base(&dev);
  if (!base) return fail(QTPU_ECUDA, "noalloc: no current device or the scratch address cannot be resolved");
  cudaError_t e = cudaSuccess;
  int sm = 148;
  cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  uint8_t* s = (uint8_t*)base;
  uint32_t* status = (uint32_t*)s;
  const uint32_t Kp = (uint32_t)up((size_t)K, 8);

  e = cudaMemsetAsync(status, 0, 16, st);  // the only state that must start at zero
  // split A[b][m][k] (rows = b*M + m, K contiguous) into BF16x3 planes
  GatherArgs ga;
  ga.nops = 1;
  ga.mode = GW_SPLIT_BF16X3;
  ga.ptr[0] = A;
  ga.dt[0] = DT_F64;
  bool ok = push(ga.out, (uint32_t)((uint64_t)batch * M), K) && push(ga.kmodes, (uint32_t)K, 1);
  ga.n_rows = (uint32_t)((uint64_t)batch * M);
  ga.K = (uint32_t)K;
  ga.Kp = Kp;
  ga.row_fast = 0;
  // split B[b][k][n]: rows = (b, n), K strided by N
  GatherArgs gb;
  gb.nops = 1;
  gb.mode = GW_SPLIT_BF16X3;
  gb.ptr[0] = B;
  gb.dt[0] = DT_F64;
  ok = ok && push(gb.out, (uint32_t)batch, (int64_t)K * N) && push(gb.out, (uint32_t)N, 1) &&
       push(gb.kmodes, (uint32_t)K, N);
  gb.n_rows = (uint32_t)((uint64_t)batch * N);
  gb.K = (uint32_t)K;
  gb.Kp = Kp;
  gb.row_fast = N > 1 ? 1 : 0;
  // convert the FP32-pair product [b][n][m] to FP64 C[b][m][n]
  GatherArgs gc;
  gc.nops = 1;
  gc.mode = GW_DENSE_F64;
  gc.ptr[0] = s + c_off;
  gc.dt[0] = DT_F32X2;
  ok = ok && push(gc.out, (uint32_t)batch, (int64_t)M * N) && push(gc.out, (uint32_t)M, 1) &&
       push(gc.out, (uint32_t)N, M);
  gc.n_out = (uint32_t)((uint64_t)batch * M * N);
  gc.n_loop = 1;
  if (!ok || (uint64_t)batch * M * N > 0x7FFFFFFFull) return fail(QTPU_ENOTSUP, "noalloc: shape too large");
  GemmArgs g;
  if (!make_operand_map(&g.maps.a[0], s + a_off, 3, batch, M, K, Kp, 128) ||
      !make_operand_map(&g.maps.b[0], s + b_off, 3, batch, N, K, Kp, g.bn))
    return fail(QTPU_ECUDA, "noalloc: cuTensorMapEncodeTiled failed");
  g.C = s + c_off;
  g.batch = batch;
  g.M = M;
  g.N = N;
  g.K = K;
  g.prec = 3;
  g.status = status;
  if (e == cudaSuccess) e = gemm_prepare();
  if (e == cudaSuccess) e = launch_gather(ga, s + a_off, sm, st);
  if (e == cudaSuccess) e = launch_gather(gb, s + b_off, sm, st);
  if (e == cudaSuccess) e = launch_gemm(g, sm, st);
  if (e == cudaSuccess) e = launch_gather(gc, C, sm, st);
  if (e != cudaSuccess) return fail(QTPU_ECUDA, "noalloc: launch failed");
  set_global_error("no error");
  return QTPU_OK;
}

extern "C" qtpu_status qtpu_pairwise_noalloc_scratch_bytes(int batch, int M, int N, int K, size_t* bytes) {
  if (!bytes) return fail(QTPU_EINVAL, "noalloc: bytes is NULL");
  if (batch < 1 || M < 1 || N < 1 || K < 1) return fail(QTPU_EINVAL, "noalloc: sizes must be >= 1");
  size_t a_off, b_off, c_off;
  *bytes = noalloc_need(batch, M, N, K, &a_off, &b_off, &c_off);
  return QTPU_OK;
}

extern "C" qtpu_status qtpu_noalloc_status(void* cuda_stream) {
  int dev = 0;
  void* base = scratch_base(&dev);
  if (!base) return fail(QTPU_ECUDA, "noalloc: no current device or the scratch address cannot be resolved");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return fail(QTPU_ECUDA, cudaGetErrorString(e));
  uint32_t st = 0;
  e = cudaMemcpy(&st, base, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(QTPU_ECUDA, cudaGetErrorString(e));
  if (st) {
    e = cudaMemset(base, 0, 4);  // reported once
    if (e != cudaSuccess) return fail(QTPU_ECUDA, cudaGetErrorString(e));
  }
  if (st & (ST_TIMEOUT_TMA | ST_TIMEOUT_MMA | ST_TIMEOUT_EPI | ST_TIMEOUT_DEP))
    return fail(QTPU_ETIMEOUT, "noalloc: a bounded device-side wait gave up; C is not valid");
  if (st) return fail(QTPU_ECUDA, "noalloc: a kernel rejected its arguments; C is not valid");
  set_global_error("no error");
  return QTPU_OK;
}

extern "C" qtpu_status qtpu_noalloc_selftest_timeout(uint64_t limit_ns, void* cuda_stream) {
  if (limit_ns == 0 || limit_ns > 10000000000ull) return fail(QTPU_EINVAL, "noalloc: limit must be in (0, 10 s]");
  int dev = 0;
  void* base = scratch_base(&dev);
  if (!base) return fail(QTPU_ECUDA, "noalloc: no current device or the scratch address cannot be resolved");
  cudaError_t e = launch_bounded_wait_probe((uint32_t*)base, limit_ns, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return fail(QTPU_ECUDA, cudaGetErrorString(e));
  return QTPU_OK;
}
