// Learned cost model: a 3-layer perceptron trained and evaluated with this
// library's own CUDA kernels.
//
//   h1 = relu(x W1 + b1),  h2 = relu(h1 W2 + b2),  y = h2 W3 + b3
//
// x: plan features (FP32), y: predicted log contraction time.  Weights are
// used in BF16 (rounded from FP32 master copies that the optimiser updates),
// every product is accumulated in FP32, the loss is the mean squared error
// and the optimiser is Adam.  The model only ranks candidate plans; the
// exact FLOP cost stays the fallback and every chosen plan is contracted
// exactly as any other.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "../../include/qtpu_htn.h"

struct qtpu_mlp {
  int device = 0;
  cudaStream_t stream = nullptr;
  int din = 0, hid = 0;
  int64_t n_params = 0;
  float* master = nullptr;       // FP32 parameters (W1 b1 W2 b2 W3 b3)
  float* grad = nullptr;         // FP32 gradients, same layout
  float* m1 = nullptr;           // Adam moments
  float* m2 = nullptr;
  __nv_bfloat16* wbf = nullptr;  // BF16 copies of W1, W2, W3 (same offsets as master)
  float* act = nullptr;          // work: z1 a1 z2 a2 y, dy, da2, dz2, da1, dz1, loss
  int cap = 0;                   // batch capacity of `act`
  int64_t step = 0;
};

namespace {

constexpr int T = 32;  // tile edge of the small GEMM kernel

// C[M x N] = op(A) op(B) (+ bias[n]); A FP32, B FP32 or BF16; row-major with
// leading dimensions; TA / TB read the stored matrix transposed.  256 threads,
// each computing 4 entries of a 32 x 32 tile; FP32 accumulation.
template <bool TA, bool TB, typename TBT>
__global__ void __launch_bounds__(256) k_mm(const float* __restrict__ A, const TBT* __restrict__ B,
                                            float* __restrict__ C, int M, int N, int K, int lda, int ldb,
                                            int ldc, const float* __restrict__ bias) {
  __shared__ float As[T][T + 1];
  __shared__ float Bs[T][T + 1];
  const int tx = threadIdx.x % T, ty = threadIdx.x / T;  // ty 0..7
  const int m0 = blockIdx.y * T, n0 = blockIdx.x * T;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < K; k0 += T) {
    for (int r = ty; r < T; r += 8) {
      const int m = m0 + r, k = k0 + tx;
      As[r][tx] = (m < M && k < K) ? (TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k]) : 0.f;
      const int kk = k0 + r, n = n0 + tx;
      float bv = 0.f;
      if (kk < K && n < N) bv = (float)(TB ? B[(size_t)n * ldb + kk] : B[(size_t)kk * ldb + n]);
      Bs[r][tx] = bv;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < T; ++k) {
      const float b = Bs[k][tx];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i] = fmaf(As[ty + 8 * i][k], b, acc[i]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 8 * i, n = n0 + tx;
    if (m < M && n < N) C[(size_t)m * ldc + n] = acc[i] + (bias ? bias[n] : 0.f);
  }
}

__global__ void k_relu(const float* __restrict__ z, float* __restrict__ a, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a[i] = z[i] > 0.f ? z[i] : 0.f;
}
__global__ void k_relu_bwd(const float* __restrict__ z, const float* __restrict__ da, float* __restrict__ dz,
                           int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dz[i] = z[i] > 0.f ? da[i] : 0.f;
}
// dy = 2 (y - t) / B and the loss sum (one block, fixed reduction order)
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dy,
                      float* __restrict__ loss, int B) {
  __shared__ float red[256];
  float s = 0.f;
  for (int i = threadIdx.x; i < B; i += blockDim.x) {
    const float d = y[i] - t[i];
    dy[i] = 2.f * d / (float)B;
    s += d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0] / (float)B;
}
// column sums of dz [B x N] (bias gradients)
__global__ void k_colsum(const float* __restrict__ dz, float* __restrict__ db, int B, int N) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += dz[(size_t)b * N + n];
  db[n] = s;
}
// Adam (Kingma and Ba) on the master copy, then the BF16 copy of weights
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, __nv_bfloat16* __restrict__ wbf, int64_t n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    w[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
    wbf[i] = __float2bfloat16_rn(w[i]);
  }
}
__global__ void k_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ o, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    o[i] = __float2bfloat16_rn(w[i]);
}

// parameter offsets
struct Off {
  int64_t W1, b1, W2, b2, W3, b3, n;
};
Off offs(int din, int hid) {
  Off o;
  o.W1 = 0;
  o.b1 = o.W1 + (int64_t)din * hid;
  o.W2 = o.b1 + hid;
  o.b2 = o.W2 + (int64_t)hid * hid;
  o.W3 = o.b2 + hid;
  o.b3 = o.W3 + hid;
  o.n = o.b3 + 1;
  return o;
}

template <bool TA, bool TB, typename TBT>
cudaError_t mm(cudaStream_t st, const float* A, const TBT* B, float* C, int M, int N, int K, int lda, int ldb, int ldc,
               const float* bias) {
  dim3 grid((N + T - 1) / T, (M + T - 1) / T);
  k_mm<TA, TB, TBT><<<grid, 256, 0, st>>>(A, B, C, M, N, K, lda, ldb, ldc, bias);
  return cudaGetLastError();
}

int blocks(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); }

// activations for a batch of B: z1 a1 z2 a2 (B x hid each), y (B), dy (B),
// da2 dz2 da1 dz1 (B x hid each), loss (1)
struct Act {
  float *z1, *a1, *z2, *a2, *y, *dy, *da2, *dz2, *da1, *dz1, *loss;
};
Act act_ptrs(qtpu_mlp* m, int B) {
  Act a;
  float* p = m->act;
  const int64_t H = (int64_t)B * m->hid;
  a.z1 = p; p += H;
  a.a1 = p; p += H;
  a.z2 = p; p += H;
  a.a2 = p; p += H;
  a.y = p; p += B;
  a.dy = p; p += B;
  a.da2 = p; p += H;
  a.dz2 = p; p += H;
  a.da1 = p; p += H;
  a.dz1 = p; p += H;
  a.loss = p;
  return a;
}

bool ensure(qtpu_mlp* m, int B) {
  if (B <= m->cap) return true;
  if (m->act) cudaFree(m->act);
  m->act = nullptr;
  const size_t n = (size_t)8 * B * m->hid + 2 * (size_t)B + 16;
  if (cudaMalloc(&m->act, n * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    m->cap = 0;
    return false;
  }
  m->cap = B;
  return true;
}

cudaError_t forward(qtpu_mlp* m, const float* x, int B, const Act& a, float* y) {
  const Off o = offs(m->din, m->hid);
  const int H = m->hid;
  cudaStream_t st = m->stream;
  cudaError_t e = mm<false, false>(st, x, m->wbf + o.W1, a.z1, B, H, m->din, m->din, H, H, m->master + o.b1);
  if (e == cudaSuccess) k_relu<<<blocks((int64_t)B * H), 256, 0, st>>>(a.z1, a.a1, (int64_t)B * H);
  if (e == cudaSuccess) e = mm<false, false>(st, a.a1, m->wbf + o.W2, a.z2, B, H, H, H, H, H, m->master + o.b2);
  if (e == cudaSuccess) k_relu<<<blocks((int64_t)B * H), 256, 0, st>>>(a.z2, a.a2, (int64_t)B * H);
  if (e == cudaSuccess) e = mm<false, false>(st, a.a2, m->wbf + o.W3, y, B, 1, H, H, 1, 1, m->master + o.b3);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

// forward + backward of the MSE loss; gradients into m->grad
cudaError_t backward(qtpu_mlp* m, const float* x, const float* t, int B, const Act& a) {
  const Off o = offs(m->din, m->hid);
  const int H = m->hid;
  cudaStream_t st = m->stream;
  cudaError_t e = forward(m, x, B, a, a.y);
  if (e != cudaSuccess) return e;
  k_mse<<<1, 256, 0, st>>>(a.y, t, a.dy, a.loss, B);
  float* g = m->grad;
  // layer 3: y = a2 W3 + b3
  e = mm<true, false>(st, a.a2, a.dy, g + o.W3, H, 1, B, H, 1, 1, nullptr);  // dW3 = a2^T dy
  if (e == cudaSuccess) k_colsum<<<1, 32, 0, st>>>(a.dy, g + o.b3, B, 1);
  if (e == cudaSuccess) e = mm<false, true>(st, a.dy, m->wbf + o.W3, a.da2, B, H, 1, 1, 1, H, nullptr);
  // layer 2
  if (e == cudaSuccess) k_relu_bwd<<<blocks((int64_t)B * H), 256, 0, st>>>(a.z2, a.da2, a.dz2, (int64_t)B * H);
  if (e == cudaSuccess) e = mm<true, false>(st, a.a1, a.dz2, g + o.W2, H, H, B, H, H, H, nullptr);
  if (e == cudaSuccess) k_colsum<<<(H + 127) / 128, 128, 0, st>>>(a.dz2, g + o.b2, B, H);
  if (e == cudaSuccess) e = mm<false, true>(st, a.dz2, m->wbf + o.W2, a.da1, B, H, H, H, H, H, nullptr);
  // layer 1
  if (e == cudaSuccess) k_relu_bwd<<<blocks((int64_t)B * H), 256, 0, st>>>(a.z1, a.da1, a.dz1, (int64_t)B * H);
  if (e == cudaSuccess) e = mm<true, false>(st, x, a.dz1, g + o.W1, m->din, H, B, m->din, H, H, nullptr);
  if (e == cudaSuccess) k_colsum<<<(H + 127) / 128, 128, 0, st>>>(a.dz1, g + o.b1, B, H);
  return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace

extern "C" {

qtpu_status qtpu_mlp_create(qtpu_mlp** out, int device, void* cuda_stream, int in_dim, int hidden, uint64_t seed) {
  if (!out || in_dim < 1 || hidden < 1 || in_dim > 4096 || hidden > 4096) return QTPU_EINVAL;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return QTPU_ECUDA;
  qtpu_mlp* m = new (std::nothrow) qtpu_mlp();
  if (!m) return QTPU_ENOMEM;
  m->device = device;
  m->stream = (cudaStream_t)cuda_stream;
  m->din = in_dim;
  m->hid = hidden;
  const Off o = offs(in_dim, hidden);
  m->n_params = o.n;
  bool ok = cudaMalloc(&m->master, o.n * 4) == cudaSuccess && cudaMalloc(&m->grad, o.n * 4) == cudaSuccess &&
            cudaMalloc(&m->m1, o.n * 4) == cudaSuccess && cudaMalloc(&m->m2, o.n * 4) == cudaSuccess &&
            cudaMalloc(&m->wbf, o.n * 2) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    qtpu_mlp_destroy(m);
    return QTPU_ENOMEM;
  }
  // He-style uniform initialisation from SplitMix64(seed) on the host
  std::vector<float> w(o.n, 0.f);
  uint64_t s = seed;
  auto next = [&]() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);  // [0, 1)
  };
  auto fill = [&](int64_t off, int64_t n, int fan_in) {
    const double a = std::sqrt(6.0 / fan_in);
    for (int64_t i = 0; i < n; ++i) w[off + i] = (float)((2.0 * next() - 1.0) * a);
  };
  fill(o.W1, (int64_t)in_dim * hidden, in_dim);
  fill(o.W2, (int64_t)hidden * hidden, hidden);
  fill(o.W3, hidden, hidden);
  if (cudaMemcpy(m->master, w.data(), o.n * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(m->m1, 0, o.n * 4) != cudaSuccess || cudaMemset(m->m2, 0, o.n * 4) != cudaSuccess) {
    qtpu_mlp_destroy(m);
    return QTPU_ECUDA;
  }
  k_to_bf16<<<blocks(o.n), 256>>>(m->master, m->wbf, o.n);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    qtpu_mlp_destroy(m);
    return QTPU_ECUDA;
  }
  *out = m;
  return QTPU_OK;
}

qtpu_status qtpu_mlp_num_params(const qtpu_mlp* m, int64_t* n) {
  if (!m || !n) return QTPU_EINVAL;
  *n = m->n_params;
  return QTPU_OK;
}

qtpu_status qtpu_mlp_params(qtpu_mlp* m, float* host_out, const float* host_in) {
  if (!m) return QTPU_EINVAL;
  if (cudaSetDevice(m->device) != cudaSuccess) return QTPU_ECUDA;
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return QTPU_ECUDA;
  if (host_in) {
    if (cudaMemcpy(m->master, host_in, m->n_params * 4, cudaMemcpyHostToDevice) != cudaSuccess) return QTPU_ECUDA;
    k_to_bf16<<<blocks(m->n_params), 256, 0, m->stream>>>(m->master, m->wbf, m->n_params);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return QTPU_ECUDA;
  }
  if (host_out && cudaMemcpy(host_out, m->master, m->n_params * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return QTPU_ECUDA;
  return QTPU_OK;
}

qtpu_status qtpu_mlp_forward(qtpu_mlp* m, const float* dev_x, int batch, float* dev_y) {
  if (!m || !dev_x || !dev_y || batch < 1) return QTPU_EINVAL;
  if (cudaSetDevice(m->device) != cudaSuccess) return QTPU_ECUDA;
  if (!ensure(m, batch)) return QTPU_ENOMEM;
  Act a = act_ptrs(m, batch);
  return forward(m, dev_x, batch, a, dev_y) == cudaSuccess ? QTPU_OK : QTPU_ECUDA;
}

qtpu_status qtpu_mlp_gradients(qtpu_mlp* m, const float* dev_x, const float* dev_t, int batch, float* host_grads,
                               float* host_loss) {
  if (!m || !dev_x || !dev_t || batch < 1) return QTPU_EINVAL;
  if (cudaSetDevice(m->device) != cudaSuccess) return QTPU_ECUDA;
  if (!ensure(m, batch)) return QTPU_ENOMEM;
  Act a = act_ptrs(m, batch);
  if (backward(m, dev_x, dev_t, batch, a) != cudaSuccess) return QTPU_ECUDA;
  if (cudaStreamSynchronize(m->stream) != cudaSuccess) return QTPU_ECUDA;
  if (host_grads && cudaMemcpy(host_grads, m->grad, m->n_params * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return QTPU_ECUDA;
  if (host_loss && cudaMemcpy(host_loss, a.loss, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return QTPU_ECUDA;
  return QTPU_OK;
}

qtpu_status qtpu_mlp_train_step(qtpu_mlp* m, const float* dev_x, const float* dev_t, int batch, float lr,
                                float* host_loss) {
  if (!m || !dev_x || !dev_t || batch < 1 || !(lr > 0.f)) return QTPU_EINVAL;
  if (cudaSetDevice(m->device) != cudaSuccess) return QTPU_ECUDA;
  if (!ensure(m, batch)) return QTPU_ENOMEM;
  Act a = act_ptrs(m, batch);
  if (backward(m, dev_x, dev_t, batch, a) != cudaSuccess) return QTPU_ECUDA;
  m->step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
  k_adam<<<blocks(m->n_params), 256, 0, m->stream>>>(m->master, m->grad, m->m1, m->m2, m->wbf, m->n_params, lr, b1,
                                                      b2, 1e-8f, c1, c2);
  if (cudaGetLastError() != cudaSuccess) return QTPU_ECUDA;
  if (host_loss) {
    if (cudaMemcpyAsync(host_loss, a.loss, 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess) return QTPU_ECUDA;
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return QTPU_ECUDA;
  }
  return QTPU_OK;
}

qtpu_status qtpu_mlp_destroy(qtpu_mlp* m) {
  if (!m) return QTPU_EINVAL;
  cudaSetDevice(m->device);
  for (void* p : {(void*)m->master, (void*)m->grad, (void*)m->m1, (void*)m->m2, (void*)m->wbf, (void*)m->act})
    if (p) cudaFree(p);
  delete m;
  return QTPU_OK;
}

}  // extern "C"
