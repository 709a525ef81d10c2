// Compensated FP32 arithmetic shared by the gather kernels.
//
// FP64 throughput on B300 is ~1/64 of FP32, so the tensor-core path keeps
// values as (hi, lo) float pairs (value = hi + lo) and never uses the FP64
// pipe: FP64 inputs are decoded with integer operations, products use TwoProd
// (exact via FMA), sums use TwoSum (Knuth).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.h"

namespace qtpu {
namespace arith {

// ------------------------------------------------------------ FP64 decode
// x = hi + lo with hi = x truncated to 24 significant bits and lo the next
// bits truncated to 24 (|x - hi - lo| < 2^-47 |x|), using integer operations
// only.  Zeros and subnormals decode to 0; exponents outside the FP32 range
// fall back to conversions.
__device__ __forceinline__ float2 decode_f64(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint32_t uh = (uint32_t)(u >> 32), ul = (uint32_t)u;
  const uint32_t sign = uh & 0x80000000u;
  const int e = (int)((uh >> 20) & 0x7FF) - 1023;
  if (e < -126 || e > 127) {
    if (e == -1023) return make_float2(0.f, 0.f);
    const float h = (float)x;  // out of FP32 range: inf / denormal path
    return make_float2(h, (float)(x - (double)h));
  }
  const uint32_t mhi = ((uh & 0xFFFFFu) << 3) | (ul >> 29);  // top 23 mantissa bits
  const float hi = __uint_as_float(sign | ((uint32_t)(e + 127) << 23) | mhi);
  const uint32_t rem = ul & 0x1FFFFFFFu;  // remaining 29 mantissa bits, weight 2^(e-52)
  // lo without branches: its bits are formed whatever rem is and selected
  // only when rem is nonzero and lo is a normal float
  const int p = 31 - __clz(rem);  // leading one, 0..28 (-1 when rem is 0)
  const int el = e - 52 + p;
  const uint32_t m = p >= 23 ? (rem >> (p - 23)) : (rem << (23 - p));
  const uint32_t lob = sign | ((uint32_t)(el + 127) << 23) | (m & 0x7FFFFFu);
  const float lo = (rem != 0u && el >= -126) ? __uint_as_float(lob) : 0.f;
  return make_float2(hi, lo);
}

template <int DT>
__device__ __forceinline__ float2 load_pair(const void* p, int64_t i) {
  if (DT == DT_F32) return make_float2(__ldg((const float*)p + i), 0.f);
  if (DT == DT_F64) return decode_f64(__ldg((const double*)p + i));
  return __ldg((const float2*)p + i);
}

__device__ __forceinline__ float2 load_any(const void* p, int dt, int64_t i) {
  if (dt == DT_F64) return load_pair<DT_F64>(p, i);
  if (dt == DT_F32X2) return load_pair<DT_F32X2>(p, i);
  return load_pair<DT_F32>(p, i);
}

// (a_hi + a_lo) * (b_hi + b_lo) as an unnormalised pair
__device__ __forceinline__ float2 mul_pair(float2 a, float2 b) {
  const float p = a.x * b.x;
  const float e = fmaf(a.x, b.x, -p);
  return make_float2(p, e + fmaf(a.x, b.y, a.y * b.x));
}

struct Acc {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float2 v) {
    const float s = __fadd_rn(hi, v.x);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v.x, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, v.y));
  }
  __device__ __forceinline__ float2 get() const {  // renormalised (Fast2Sum)
    const float s = __fadd_rn(hi, lo);
    return make_float2(s, __fsub_rn(lo, __fsub_rn(s, hi)));
  }
  __device__ __forceinline__ double as_double() const { return (double)hi + (double)lo; }
};

// FP64 accumulator of FP32-pair terms: used wherever a sum produces a value
// of the final output (the last step of every slice, the slice sum, the
// final dot product), because a sum over signed QPD coefficients may cancel
// and FP64 keeps 53 bits through it.  Each term hi + lo enters exactly (up to
// one FP64 rounding) and is added in FP64.
struct AccD {
  double s = 0.0;
  __device__ __forceinline__ void add(float2 v) { s += (double)v.x + (double)v.y; }
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double as_double() const { return s; }
  __device__ __forceinline__ float2 get() const {
    const float h = (float)s;
    return make_float2(h, (float)(s - (double)h));
  }
};

// (hi, lo) pair plus (hi, lo) pair, compensated and renormalised
__device__ __forceinline__ float2 pair_sum(float2 a, float2 b) {
  Acc t;
  t.hi = a.x;
  t.lo = a.y;
  t.add(b);
  return t.get();
}
// store an output value, or add it to the stored one
__device__ __forceinline__ void store_out(float2* out, uint32_t o, float2 v, int accum) {
  out[o] = accum ? pair_sum(out[o], v) : v;
}
__device__ __forceinline__ void store_out(double* out, uint32_t o, double v, int accum) {
  out[o] = accum ? out[o] + v : v;
}

// FP64 on the output side, FP32 pairs elsewhere
template <bool F64>
struct AccSel {
  using T = Acc;
};
template <>
struct AccSel<true> {
  using T = AccD;
};

// ------------------------------------------------------------ BF16x3 pieces
// The three BF16 pieces of the values of one operand row over one 64-entry
// k-block share a grid: with 2^E above every |x| of the block, the pieces are
// integer multiples of 2^(E-7), 2^(E-16) and 2^(E-25), the first of magnitude
// at most 2^7 units and the others at most 2^8 (at most 8 significant bits,
// so exact in BF16), and |x - x0 - x1 - x2| <= 2^(E-26).  A product of two
// leading pieces is an integer multiple of 2^(Ea+Eb-14) of at most 2^14
// units, so the sum of up to 1024 of them on one grid (16 k-blocks) stays
// within 2^24 units and is exact in the tensor cores' FP32 accumulator
// whatever rounding it applies.
__device__ __forceinline__ int grid_exp(float m) {  // E with |m| < 2^E, clamped to [-123, 111]
  const int e = (int)((__float_as_uint(fabsf(m)) >> 23) & 0xffu) - 126;
  return e > 111 ? 111 : (e < -123 ? -123 : e);
}
// x rounded to a multiple of 2^(e-23) (round to nearest even); |x| < 2^(e-1),
// e + 127 in [1, 254].  x + 1.5*2^e lies in [2^e, 2^(e+1)), where the spacing
// of floats is 2^(e-23), and the subtraction is exact.
__device__ __forceinline__ float grid_round(float x, int e) {
  const float c = __uint_as_float(((uint32_t)(e + 127) << 23) | 0x400000u);
  return __fsub_rn(__fadd_rn(x, c), c);
}
// pieces of v = v.x + v.y on the grid of exponent E
__device__ __forceinline__ void grid_pieces(float2 v, int E, float* p) {
  const float h0 = grid_round(v.x, E + 16);              // multiple of 2^(E-7)
  const float r1 = __fadd_rn(__fsub_rn(v.x, h0), v.y);  // v.x - h0 is exact
  const float h1 = grid_round(r1, E + 7);                // multiple of 2^(E-16)
  const float r2 = __fsub_rn(r1, h1);                    // exact
  p[0] = h0;
  p[1] = h1;
  p[2] = grid_round(r2, E - 2);                          // multiple of 2^(E-25)
}

// ------------------------------------------------------------ indexing
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& d) {
  return (uint32_t)(((uint64_t)__umulhi(n, d.magic) + n) >> d.shift);
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}


template <int NOPS>
__device__ __forceinline__ void offsets(uint32_t o, const GModes& t, int64_t* off) {
#pragma unroll
  for (int j = 0; j < NOPS; ++j) off[j] = 0;
  for (int m = t.n - 1; m >= 0; --m) {
    const uint32_t q = fdiv(o, t.div[m]);
    const uint32_t i = o - q * t.dim[m];
    o = q;
#pragma unroll
    for (int j = 0; j < NOPS; ++j) off[j] += (int64_t)i * t.stride[m][j];
  }
}

// digits of position l over the modes of t (outermost first) and the
// operand offsets they add: the start state of an odometer walk from l
template <int NOPS>
__device__ __forceinline__ void digits(uint32_t l, const GModes& t, uint32_t* idx, int64_t* off) {
  for (int m = t.n - 1; m >= 0; --m) {
    const uint32_t q = fdiv(l, t.div[m]);
    const uint32_t i = l - q * t.dim[m];
    l = q;
    idx[m] = i;
#pragma unroll
    for (int j = 0; j < NOPS; ++j) off[j] += (int64_t)i * t.stride[m][j];
  }
}

// lanes per output for a sum of n_loop terms: groups of 2^lg consecutive
// lanes share an output (each lane a contiguous run of at least 8 terms)
// while the lanes stay within half of what the SMs hold at once (1024 a
// SM); with more outputs than that, one lane per output already fills them
inline int lanes_for_long_sum(uint32_t n_out, uint32_t n_loop, int sm_count) {
  int lg = 0;
  while (lg < 5 && (8u << (lg + 1)) <= n_loop && ((uint64_t)n_out << (lg + 1)) <= (uint64_t)sm_count * 1024) ++lg;
  return lg;
}

}  // namespace arith
}  // namespace qtpu
