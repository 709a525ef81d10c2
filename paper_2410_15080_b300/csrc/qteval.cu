// QT evaluation on the GPU: a statevector simulator of subcircuit instances
// (section 4.1: each subcircuit is a QT whose entries are the expectation
// values of its instances; section 6.2 Step 2 evaluates them -- on QPUs in
// the paper, here exactly, as a mock QPU).
//
// A program is one subcircuit of at most 15 qubits: single-qubit unitaries,
// CZ gates, and at each gate cut the local operation of the cut's instance
// (a term of the CZ decomposition of section 2.1: I, Z, e^{+-i pi/4 Z} or a
// signed Z measurement, then e^{-i pi/4 Z}); wire cuts prepare a qubit in
// |0>, |1>, |+>, |i> or measure it in I, Z, X, Y (Eq. wire-tensor).  The QT
// is written as FP64 [observable][cut values...] in C order: the layout the
// contraction reads.
//
// k_qt_instances: one block per instance (grid-stride).  A signed
// measurement M(rho) = P0 rho P0 - P1 rho P1 is carried as two branches,
// the projected (unnormalised) pure states, whose expectation values add
// with sign -1 for outcome 1; the block runs the instance's branches one
// after another.  The state (2^n FP64 complex amplitudes, qubit 0 the most
// significant bit) lives in shared memory up to 12 qubits, else in a global
// slice of the block.  Each operation is one pass of the block over the
// amplitudes, separated by barriers; each observable O_k is
// sum_x conj(psi[x ^ f]) i^{ny} (-1)^{|x & p|} psi[x] (f: X/Y qubits, p: Y/Z
// qubits), reduced over the block in a fixed tree, so results are
// deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/qtpu_htn.h"
#include "exec.h"

namespace qtpu {

namespace {

constexpr int kQtMaxQubits = 15;
constexpr int kQtSmemQubits = 12;
constexpr int kQtMaxCuts = 16;
constexpr int kQtMaxObs = 64;
constexpr int kQtThreads = 256;

struct QOp {
  int kind, q0, q1, cut, side;
  double2 u[4];
};

struct QtProg {
  int n, n_ops, n_cuts, n_obs;
  uint64_t n_inst;
  int dim[kQtMaxCuts], cut_kind[kQtMaxCuts], cut_qubit[kQtMaxCuts];
  uint32_t fm[kQtMaxObs], pm[kQtMaxObs];
  int ny[kQtMaxObs];
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(__dsub_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)),
                      __dadd_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x)));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// local operation of gate-cut term g on side s: 0 = phase (d0, d1), 1 = measure
__device__ __forceinline__ void local_op(int side, int g, int* kind, double2* d0, double2* d1) {
  const double r = 0.70710678118654752440;  // cos(pi/4) = sin(pi/4)
  const double2 one = make_double2(1.0, 0.0), mone = make_double2(-1.0, 0.0);
  const double2 ep = make_double2(r, r), em = make_double2(r, -r);  // e^{+i pi/4}, e^{-i pi/4}
  // side 0: I, Z, M, M, e^{+i pi/4 Z}, e^{-i pi/4 Z}; side 1: I, Z, e^{+}, e^{-}, M, M
  int t;
  if (g == 0) t = 0;
  else if (g == 1) t = 1;
  else if (side == 0) t = g <= 3 ? 4 : (g == 4 ? 2 : 3);
  else t = g >= 4 ? 4 : (g == 2 ? 2 : 3);
  *kind = t == 4 ? 1 : 0;
  if (t == 0) *d0 = one, *d1 = one;
  if (t == 1) *d0 = one, *d1 = mone;
  if (t == 2) *d0 = ep, *d1 = em;  // e^{+i pi/4 Z} = diag(e^{+i pi/4}, e^{-i pi/4})
  if (t == 3) *d0 = em, *d1 = ep;
  if (t == 4) *d0 = one, *d1 = one;
}

__global__ void __launch_bounds__(kQtThreads) k_qt_instances(const QtProg* __restrict__ P, const QOp* __restrict__ ops,
                                                           double2* __restrict__ gscratch, double* __restrict__ out) {
  extern __shared__ double2 smem_state[];
  __shared__ double red[kQtThreads];
  __shared__ double acc[kQtMaxObs];
  const int n = P->n;
  const uint32_t N = 1u << n;
  double2* psi = n <= kQtSmemQubits ? smem_state : gscratch + (size_t)blockIdx.x * N;
  const double r = 0.70710678118654752440;
  const double2 post0 = make_double2(r, -r), post1 = make_double2(r, r);  // e^{-i pi/4 Z}
  for (uint64_t inst = blockIdx.x; inst < P->n_inst; inst += gridDim.x) {
    int val[kQtMaxCuts];
    uint64_t rr = inst;
    for (int c = P->n_cuts - 1; c >= 0; --c) {
      val[c] = (int)(rr % (uint64_t)P->dim[c]);
      rr /= (uint64_t)P->dim[c];
    }
    int n_meas = 0;
    for (int o = 0; o < P->n_ops; ++o)
      if (ops[o].kind == QTPU_OP_GATE_CUT) {
        int kd;
        double2 a, b;
        local_op(ops[o].side, val[ops[o].cut], &kd, &a, &b);
        n_meas += kd;
      }
    // measured wires: A = I, Z, X, Y on their qubit (flip / parity / Y count)
    uint32_t wfm = 0, wpm = 0;
    int wny = 0;
    for (int c = 0; c < P->n_cuts; ++c)
      if (P->cut_kind[c] == QTPU_CUT_MEASURE) {
        const uint32_t bit = 1u << (n - 1 - P->cut_qubit[c]);
        const int a = val[c];
        if (a == 2 || a == 3) wfm |= bit;
        if (a == 1 || a == 3) wpm |= bit;
        if (a == 3) ++wny;
      }
    if (threadIdx.x < (unsigned)P->n_obs) acc[threadIdx.x] = 0.0;
    for (uint32_t br = 0; br < (1u << n_meas); ++br) {
      // initial product state
      for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) {
        double2 amp = make_double2(1.0, 0.0);
        for (int q = 0; q < n; ++q) {
          const int b = (x >> (n - 1 - q)) & 1;
          int prep = -1;
          for (int c = 0; c < P->n_cuts; ++c)
            if (P->cut_kind[c] == QTPU_CUT_PREPARE && P->cut_qubit[c] == q) prep = val[c];
          double2 k = make_double2(b ? 0.0 : 1.0, 0.0);  // |0>
          if (prep == 1) k = make_double2(b ? 1.0 : 0.0, 0.0);
          if (prep == 2) k = make_double2(r, 0.0);                          // |+>
          if (prep == 3) k = b ? make_double2(0.0, r) : make_double2(r, 0.0);  // |i>
          amp = cmul(amp, k);
        }
        psi[x] = amp;
      }
      __syncthreads();
      double sign = 1.0;
      int mi = 0;
      for (int o = 0; o < P->n_ops; ++o) {
        const QOp& op = ops[o];
        if (op.kind == QTPU_OP_U1) {
          const int p = n - 1 - op.q0;
          const uint32_t lo = (1u << p) - 1;
          for (uint32_t t = threadIdx.x; t < N / 2; t += blockDim.x) {
            const uint32_t i0 = ((t & ~lo) << 1) | (t & lo), i1 = i0 | (1u << p);
            const double2 a0 = psi[i0], a1 = psi[i1];
            psi[i0] = cadd(cmul(op.u[0], a0), cmul(op.u[1], a1));
            psi[i1] = cadd(cmul(op.u[2], a0), cmul(op.u[3], a1));
          }
        } else if (op.kind == QTPU_OP_CZ) {
          const uint32_t m = (1u << (n - 1 - op.q0)) | (1u << (n - 1 - op.q1));
          for (uint32_t x = threadIdx.x; x < N; x += blockDim.x)
            if ((x & m) == m) psi[x] = make_double2(-psi[x].x, -psi[x].y);
        } else {
          int kd;
          double2 d0, d1;
          local_op(op.side, val[op.cut], &kd, &d0, &d1);
          const uint32_t bit = 1u << (n - 1 - op.q0);
          if (kd) {  // signed measurement: this branch's outcome, then the phase
            const uint32_t outc = (br >> mi) & 1;
            ++mi;
            if (outc) sign = -sign;
            for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) {
              const uint32_t b = (x & bit) ? 1 : 0;
              psi[x] = b != outc ? make_double2(0.0, 0.0) : cmul(psi[x], b ? post1 : post0);
            }
          } else {
            const double2 c0 = cmul(d0, post0), c1 = cmul(d1, post1);
            for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) psi[x] = cmul(psi[x], (x & bit) ? c1 : c0);
          }
        }
        __syncthreads();
      }
      // observables
      for (int k = 0; k < P->n_obs; ++k) {
        const uint32_t fm = P->fm[k] | wfm, pm = P->pm[k] | wpm;
        const int ny = (P->ny[k] + wny) & 3;
        double s = 0.0;
        for (uint32_t x = threadIdx.x; x < N; x += blockDim.x) {
          const double2 a = psi[x ^ fm], b = psi[x];
          // conj(a) * b
          double2 v = make_double2(__dadd_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)),
                                   __dsub_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x)));
          // times i^{ny}: real part of the product
          double re = ny == 0 ? v.x : (ny == 1 ? -v.y : (ny == 2 ? -v.x : v.y));
          if (__popc(x & pm) & 1) re = -re;
          s = __dadd_rn(s, re);
        }
        red[threadIdx.x] = s;
        __syncthreads();
        for (int h = blockDim.x / 2; h > 0; h >>= 1) {
          if ((int)threadIdx.x < h) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + h]);
          __syncthreads();
        }
        if (threadIdx.x == 0) acc[k] = __dadd_rn(acc[k], sign * red[0]);
        __syncthreads();
      }
    }
    __syncthreads();
    if (threadIdx.x < (unsigned)P->n_obs) out[(uint64_t)threadIdx.x * P->n_inst + inst] = acc[threadIdx.x];
    __syncthreads();
  }
}

qtpu_status qt_fail(qtpu_status s, const std::string& m) {
  set_global_error(m.c_str());
  return s;
}

}  // namespace

}  // namespace qtpu

using namespace qtpu;

extern "C" qtpu_status qtpu_qt_evaluate(int device, void* cuda_stream, const qtpu_qt_program* prog,
                                        double* dev_out, double* n_instances) {
  if (n_instances) *n_instances = 0;
  if (!prog || !dev_out) return qt_fail(QTPU_EINVAL, "qt_evaluate: NULL program or output");
  const int n = prog->n_qubits;
  if (n < 1 || n > kQtMaxQubits) return qt_fail(QTPU_EINVAL, "qt_evaluate: 1..15 qubits");
  if (prog->n_ops < 0 || prog->n_ops > 4096 || (prog->n_ops > 0 && !prog->ops))
    return qt_fail(QTPU_EINVAL, "qt_evaluate: 0..4096 operations");
  if (prog->n_cuts < 0 || prog->n_cuts > kQtMaxCuts || (prog->n_cuts > 0 && (!prog->cut_kind || !prog->cut_qubit)))
    return qt_fail(QTPU_EINVAL, "qt_evaluate: 0..16 cuts");
  if (prog->n_obs < 1 || prog->n_obs > kQtMaxObs || !prog->paulis)
    return qt_fail(QTPU_EINVAL, "qt_evaluate: 1..64 observables");
  QtProg P{};
  P.n = n;
  P.n_ops = prog->n_ops;
  P.n_cuts = prog->n_cuts;
  P.n_obs = prog->n_obs;
  P.n_inst = 1;
  std::vector<int> used(prog->n_cuts, 0), wire_q(n, 0);
  for (int c = 0; c < prog->n_cuts; ++c) {
    const int k = prog->cut_kind[c];
    if (k != QTPU_CUT_GATE && k != QTPU_CUT_MEASURE && k != QTPU_CUT_PREPARE)
      return qt_fail(QTPU_EINVAL, "qt_evaluate: bad cut kind");
    P.cut_kind[c] = k;
    P.dim[c] = k == QTPU_CUT_GATE ? 6 : 4;
    P.n_inst *= (uint64_t)P.dim[c];
    P.cut_qubit[c] = -1;
    if (k != QTPU_CUT_GATE) {
      const int q = prog->cut_qubit[c];
      if (q < 0 || q >= n || wire_q[q]) return qt_fail(QTPU_EINVAL, "qt_evaluate: bad or repeated wire-cut qubit");
      wire_q[q] = 1;
      P.cut_qubit[c] = q;
    }
  }
  std::vector<QOp> ops(prog->n_ops);
  for (int o = 0; o < prog->n_ops; ++o) {
    const qtpu_qop& s = prog->ops[o];
    QOp& d = ops[o];
    d.kind = s.kind;
    d.q0 = s.q0;
    d.q1 = s.q1;
    d.cut = s.cut;
    d.side = s.side;
    if (s.q0 < 0 || s.q0 >= n) return qt_fail(QTPU_EINVAL, "qt_evaluate: bad qubit");
    if (s.kind == QTPU_OP_U1) {
      for (int j = 0; j < 4; ++j) d.u[j] = make_double2(s.u[2 * j], s.u[2 * j + 1]);
    } else if (s.kind == QTPU_OP_CZ) {
      if (s.q1 < 0 || s.q1 >= n || s.q1 == s.q0) return qt_fail(QTPU_EINVAL, "qt_evaluate: bad CZ qubits");
    } else if (s.kind == QTPU_OP_GATE_CUT) {
      if (s.cut < 0 || s.cut >= prog->n_cuts || prog->cut_kind[s.cut] != QTPU_CUT_GATE || used[s.cut]++ ||
          (s.side != 0 && s.side != 1))
        return qt_fail(QTPU_EINVAL, "qt_evaluate: a gate-cut operation needs its own gate cut and side 0 or 1");
    } else {
      return qt_fail(QTPU_EINVAL, "qt_evaluate: bad operation kind");
    }
  }
  for (int c = 0; c < prog->n_cuts; ++c)
    if (prog->cut_kind[c] == QTPU_CUT_GATE && !used[c])
      return qt_fail(QTPU_EINVAL, "qt_evaluate: a gate cut without its operation");
  for (int k = 0; k < prog->n_obs; ++k) {
    P.fm[k] = P.pm[k] = 0;
    P.ny[k] = 0;
    for (int q = 0; q < n; ++q) {
      const char ch = prog->paulis[(size_t)k * n + q];
      const uint32_t bit = 1u << (n - 1 - q);
      if (ch != 'I' && wire_q[q]) {
        for (int c = 0; c < prog->n_cuts; ++c)
          if (prog->cut_kind[c] == QTPU_CUT_MEASURE && prog->cut_qubit[c] == q)
            return qt_fail(QTPU_EINVAL, "qt_evaluate: an observable acts on a measured wire qubit");
      }
      if (ch == 'X') P.fm[k] |= bit;
      else if (ch == 'Y') P.fm[k] |= bit, P.pm[k] |= bit, P.ny[k]++;
      else if (ch == 'Z') P.pm[k] |= bit;
      else if (ch != 'I') return qt_fail(QTPU_EINVAL, "qt_evaluate: Pauli characters are I, X, Y, Z");
    }
  }
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return qt_fail(QTPU_ECUDA, cudaGetErrorString(e));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int sm = 148;
  cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, device);
  const uint64_t grid = std::min<uint64_t>(P.n_inst, (uint64_t)sm * (n <= kQtSmemQubits ? 4 : 2));
  const size_t smem = n <= kQtSmemQubits ? ((size_t)1 << n) * sizeof(double2) : 0;
  if (smem > 48 * 1024) {
    e = cudaFuncSetAttribute(k_qt_instances, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return qt_fail(QTPU_ECUDA, cudaGetErrorString(e));
  }
  QtProg* dP = nullptr;
  QOp* dops = nullptr;
  double2* scratch = nullptr;
  e = cudaMallocAsync((void**)&dP, sizeof(QtProg), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&dops, sizeof(QOp) * std::max(1, P.n_ops), st);
  if (e == cudaSuccess && n > kQtSmemQubits)
    e = cudaMallocAsync((void**)&scratch, grid * ((size_t)1 << n) * sizeof(double2), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dP, &P, sizeof(QtProg), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && P.n_ops)
    e = cudaMemcpyAsync(dops, ops.data(), sizeof(QOp) * P.n_ops, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_qt_instances<<<(unsigned)grid, kQtThreads, smem, st>>>(dP, dops, scratch, dev_out);
    e = cudaGetLastError();
  }
  // the program is copied from host memory of this call: finish before returning
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (dP) cudaFreeAsync(dP, st);
  if (dops) cudaFreeAsync(dops, st);
  if (scratch) cudaFreeAsync(scratch, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return qt_fail(e == cudaErrorMemoryAllocation ? QTPU_ENOMEM : QTPU_ECUDA,
                   std::string("qt_evaluate: ") + cudaGetErrorString(e));
  }
  if (n_instances) *n_instances = (double)P.n_inst;
  return QTPU_OK;
}
