// Batched GEMM on the 5th-generation tensor cores (tcgen05 + TMEM + TMA).
//
// Pairwise contraction of two h-TN tensors (section 4.2: the post-processing
// is a sequence of pairwise contractions) is, after regrouping indices, a
// batched GEMM  C[b, m, n] = sum_k A[b, m, k] * B[b, n, k]  (both operands
// K-major; C stored [b][n][m], the layout in which the epilogue's stores are
// contiguous).  FP64 operands are split into low-precision pieces by the split
// kernel (x = x0 + x1 + x2, BF16 or TF32 pieces); the products of the pieces
// whose combined weight is at or above 2^-16 (BF16x3: 6 products) or 2^-11
// (3xTF32: 3 products) accumulate in FP32 in TMEM.  The tensor cores'
// FP32 accumulation loses precision with every MMA added into an accumulator
// (measured: the error grows linearly with K), so (1) the leading product
// x0*y0 has its own accumulator X and the smaller cross terms share Y, and
// (2) BF16x3 pieces are cut on a grid shared by each operand row's 64-entry
// block of k (see grid_pieces): every block's sum of leading products, and a
// chunk of up to 1024 k on one grid, is then exact in X, so one chunk covers
// K <= 1024 and the accumulators are drained once per tile.  Longer K (and
// the TF32 forms, 128 or 1024 k per chunk) add each chunk's X + Y to the
// stored result with compensated (TwoSum) FP32 arithmetic; FP64 math is
// avoided (FP64 throughput on B300 is ~1/64 of FP32).
//
// The N tile BN is a template parameter (128, 112, 96, 80, 64 or 48 columns,
// and 160 or 144 for BF16x3 on one CTA: 160 for a fused-split producer whose
// N side is at most 160 wide, and either for a plain GEMM whose tile table
// entry picks it;
// the executor picks it per GEMM, with the orientation, from a measured tile
// table or by padding): a 216-wide side fills two 112-column tiles to 96 %
// where 128-column tiles fill 84 %.  The M tile is 128 rows.  Every k-block
// issues all its K-steps, zero-filled past K: on B300 skipping the K-steps
// past K made every launch slower, even those with no partial k-block
// (1296 x 1296 x 576: 0.675 ms with a bound check in the MMA issue loop and
// 0.660 ms with unrolled per-count variants, 0.591-0.597 ms without).
//
// BF16x3 GEMMs can also run on CTA pairs (clusters of two, cta_group::2
// MMAs of M = 256): each CTA stages its 128 rows of A and half of B's BN
// rows, so a stage is 25 % smaller and three fit instead of two; the tile
// table picks the form per problem (on B300 the 4-pair 216 x 7776 x 216 step
// of the 100-qubit plan runs 12 % faster on pairs, 1296 x 1296 x 576 is
// fastest on single CTAs).
//
// One CTA (or CTA pair) per SM (pair of SMs), persistent over (batch,
// m-tile, n-tile) tiles:
//   warp 0      TMA producer (one lane): pieces of A and B for one k-block
//               (KB k: 64 for BF16x3, 32 for TF32) per pipeline stage, each
//               piece p (A_p and B_p) counted on its own mbarrier; as many
//               stages as fit (BF16x3: 2 with 128-column tiles on one CTA,
//               3 with 64 or 48 columns or on a pair, 2 with a pair's 224 or
//               256 columns);
//   warp 1      TMEM owner and MMA issuer (one lane; rank 0 of a pair): per
//               k-block and piece p as it lands, the K-steps of the products
//               whose later piece is p (x0*y0; x0*y1, x1*y0, x1*y1; x0*y2,
//               x2*y0), into one of two TMEM accumulator buffers
//               (double-buffered so the epilogue of one chunk overlaps the
//               MMAs of the next; one buffer for N tiles above 128 columns);
//   warps 2..17 epilogue: tcgen05.ld 32 lanes x 8-column groups of both
//               accumulators, X + Y as an exact (hi, lo) float pair (TwoSum)
//               stored, or added to the stored pair for later chunks.
// Every wait is bounded (global timer); on give-up the kernel sets a status
// bit, lets in-flight copies and MMAs land, frees TMEM and returns.
#include <cstdio>

#include <cuda_bf16.h>

#include "arith.cuh"
#include "common.cuh"
#include "kernels.h"

namespace qtpu {

namespace {

constexpr int BM = 128;
constexpr int kFuseBN = 128;                   // N tile of the fused-split epilogue
constexpr int kEpiWarps = 16;
constexpr int kThreads = 64 + 32 * kEpiWarps;  // producer, MMA, 16 epilogue warps
constexpr uint32_t kTmemCols = 512;            // 2 buffers x (X, Y) x BN columns (BN <= 128)
constexpr int kSmemLimit = 232448;             // dynamic shared memory per CTA (227 KB)

// Product list: entry 0 is the leading product x0*y0 (accumulator X), the
// rest are the cross terms (accumulator Y, a factor 2^-8 or 2^-11 smaller).
template <int PREC>
struct Cfg;
// KB: k per pipeline stage (one 128-byte swizzled shared-memory row: 64
// BF16 or 32 TF32; measured on B300, 32-k BF16x3 stages in 64-byte swizzle,
// twice as many in flight, ran the 100-qubit GEMMs 8-20 % slower); KC:
// stages per accumulator chunk.
template <>
struct Cfg<3> {  // BF16x3: pieces of 8 significant bits, products of weight >= 2^-16
  static constexpr int NP = 3, NPROD = 6, ES = 2, KB = 64, UK = 16, FMT = 1, KC = 16;
  __host__ __device__ static constexpr int pa(int i) { return i == 2 || i == 4 ? 1 : (i == 5 ? 2 : 0); }
  __host__ __device__ static constexpr int pb(int i) { return i == 1 || i == 4 ? 1 : (i == 3 ? 2 : 0); }
};
template <>
struct Cfg<2> {  // 3xTF32: pieces of 11 significant bits, products of weight >= 2^-11
  static constexpr int NP = 2, NPROD = 3, ES = 4, KB = 32, UK = 8, FMT = 2, KC = 4;
  __host__ __device__ static constexpr int pa(int i) { return i == 2 ? 1 : 0; }
  __host__ __device__ static constexpr int pb(int i) { return i == 1 ? 1 : 0; }
};
template <>
struct Cfg<1> {  // TF32: one piece, one product
  static constexpr int NP = 1, NPROD = 1, ES = 4, KB = 32, UK = 8, FMT = 2, KC = 32;
  __host__ __device__ static constexpr int pa(int) { return 0; }
  __host__ __device__ static constexpr int pb(int) { return 0; }
};

// Shared memory: the pipeline stages (as many as fit, at most 8), the
// barriers and, for the fused-split epilogue (BF16x3, one CTA per tile, BN =
// 128, or 160 for an N side of at most 160 columns), its tables.  In a CTA pair each CTA stages its own 128 rows of
// A and half of B's BN rows.
template <int PREC, int BN, bool PAIR = false>
struct Layout {
  using C = Cfg<PREC>;
  static constexpr bool FUSE = PREC == 3 && !PAIR && (BN == kFuseBN || BN == kFuseWideBN);
  static constexpr int ROW = C::KB * C::ES;  // bytes per smem row (= swizzle span)
  static_assert(ROW == 64 || ROW == 128, "64- or 128-byte swizzle rows");
  static constexpr int B_ROWS = PAIR ? BN / 2 : BN;  // B rows staged by one CTA
  static_assert(B_ROWS % 8 == 0, "B rows in whole 8-row swizzle atoms");
  static constexpr int TM = PAIR ? 2 * BM : BM;      // rows of a tile
  // TMEM accumulator buffers of (X, Y) x BN columns: two (the epilogue of a
  // chunk overlaps the next chunk's MMAs) while they fit in 512 columns
  static constexpr int ACC_BUFS = 4 * BN <= (int)kTmemCols ? 2 : 1;
  // TMEM columns allocated, a power of two; a pair's allocation covers both CTAs
  static constexpr uint32_t TMEM_COLS = !PAIR || 2 * ACC_BUFS * BN > 256 ? kTmemCols : 256;
  static constexpr int A_PIECE = BM * ROW;
  static constexpr int B_PIECE = B_ROWS * ROW;
  static constexpr int STAGE = C::NP * (A_PIECE + B_PIECE);
  static constexpr int FUSE_W = (BN == kFuseBN ? (int)kFuseMaxW : (int)kFuseMaxWWide) * 8;
  // maxima: [4][BN] per lane quarter and column (k along the rows), or per
  // column group and row: [4][128] (BN 128), [4][2][128] (BN 160: a group of
  // 40 columns meets two 64-entry k-blocks)
  static constexpr int FUSE_XF = BN == kFuseBN ? 4 * 128 : (4 * BN > 8 * 128 ? 4 * BN : 8 * 128);
  static constexpr int FUSE_BYTES = FUSE ? FUSE_W + 2 * 128 * 4 + 2 * BN * 4 + FUSE_XF * 4 + 16 : 0;
  static constexpr int FIT = (kSmemLimit - 1024 - 256 - FUSE_BYTES) / STAGE;
  static constexpr int STAGES = FIT < 8 ? FIT : 8;
  static_assert(STAGES >= 2, "two pipeline stages must fit");
  static_assert(BN % 16 == 0 && BN >= 16 && 2 * ACC_BUFS * BN <= (int)kTmemCols, "UMMA N tile");
  static_assert(BN <= 128 || PAIR || (PREC == 3 && (BN == kGemmWideN[0] || BN == kGemmWideN[1])),
                "N tiles above 128 columns: CTA pairs, or 160 and 144 in BF16x3");
  static constexpr int BAR_OFF = STAGES * STAGE;
  // full[S][NP] (one per piece of a stage), empty[S], accfull[2],
  // accempty[2], mma_done
  static constexpr int N_BARS = STAGES * C::NP + STAGES + 5;
  static constexpr int FUSE_OFF = (BAR_OFF + N_BARS * 8 + 16 + 15) / 16 * 16;
  static constexpr int SMEM = FUSE_OFF + FUSE_BYTES + 1024;
  static_assert(SMEM <= kSmemLimit, "shared memory");
};

__device__ __forceinline__ void set_abort(volatile int* abort, uint32_t* status, uint32_t bit) {
  *abort = 1;
  if (status) atomicOr(status, bit);
}

// s + e = a + b exactly (TwoSum, Knuth)
__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return make_float2(s, e);
}
// (hi, lo) pair plus (hi, lo) pair, renormalised (Fast2Sum)
__device__ __forceinline__ float2 pair_add(float2 p, float2 q) {
  const float2 t = two_sum(p.x, q.x);
  const float lo = __fadd_rn(t.y, __fadd_rn(p.y, q.y));
  const float hi = __fadd_rn(t.x, lo);
  return make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, t.x)));
}

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpiWarps) : "memory"); }

// offsets of x over digit modes: stride 0 -> *r, stride 1 -> *w
__device__ __forceinline__ void digits(uint32_t x, const GModes& t, int* r, int* w) {
  int64_t a = 0, b = 0;
  for (int m = t.n - 1; m >= 0; --m) {
    const uint32_t q = arith::fdiv(x, t.div[m]);
    const uint32_t i = x - q * t.dim[m];
    x = q;
    a += (int64_t)i * t.stride[m][0];
    b += (int64_t)i * t.stride[m][1];
  }
  *r = (int)a;
  *w = (int)b;
}

// Epilogue that writes the consumer operand's BF16x3 pieces (GemmFuse).  Per
// tile: digit tables of the tile's rows and columns, then pass 1 (X + Y times
// W, maxima per consumer row and 64-entry k-block, exchanged through shared
// memory), then pass 2 (pieces on each block's grid, stored).  Both passes
// read the accumulator, which is handed back after pass 2.  Every epilogue
// warp reaches every named barrier of a tile; a timeout (abort) ends the tile
// loop for all of them after the second barrier.
template <int PREC, int BN>
__device__ void fused_epilogue(const GemmFuse& fz, const float2* fW, uint8_t* smem, uint32_t tmem, uint64_t* accfull,
                               uint64_t* accempty, volatile int* abort, uint32_t* status, uint64_t limit_ns, int batch,
                               int M, int N, int mt, int nt, int n_tiles, __nv_bfloat16* out) {
  using L = Layout<PREC, BN>;
  static_assert(L::FUSE, "the fused epilogue has 128- or 160-column tiles");
  constexpr int kEpiCols = BN / (kEpiWarps / 4);  // columns per thread (4 column groups)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ew = warp - 2, q = warp & 3, h = ew >> 2;
  const int et = threadIdx.x - 64;
  int* rm = reinterpret_cast<int*>(smem + L::FUSE_OFF + L::FUSE_W);
  int* wm = rm + 128;
  int* rn = wm + 128;
  int* wn = rn + BN;
  float* xmax = reinterpret_cast<float*>(wn + BN);  // L::FUSE_XF entries
  // set only by epilogue threads, and only before a tile's last barrier, so
  // every epilogue warp reads the same value after it
  volatile int* epi_abort = reinterpret_cast<volatile int*>(xmax + L::FUSE_XF);
  // BN 160: the 64-entry k-blocks (columns) a group of 40 columns meets,
  // first and last (the only N tile starts at column 0)
  const int blk0 = h * kEpiCols / 64, blk1 = (h * kEpiCols + kEpiCols - 1) / 64;
  if (et == 0) *epi_abort = 0;
  const bool hasW = fz.w_size != 0;
  const uint32_t Kp = fz.Kp;
  int item = 0;
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x, ++item) {
    const int ntile = (int)(t % nt);
    const int r = t / nt;
    const int mtile = (int)(r % mt);
    const int b = (int)(r / mt);
    epi_bar();  // the previous tile's readers of the tables are done
    if (et < 128) {  // entries outside the matrix get offset 0 (never stored)
      const int m = mtile * BM + et;
      rm[et] = wm[et] = 0;
      if (m < M) digits((uint32_t)m, fz.mmodes, &rm[et], &wm[et]);
    } else if (et < 128 + BN) {
      const int n = ntile * BN + (et - 128);
      rn[et - 128] = wn[et - 128] = 0;
      if (n < N) digits((uint32_t)n, fz.nmodes, &rn[et - 128], &wn[et - 128]);
    }
    int rb, wb;
    digits((uint32_t)b, fz.bmodes, &rb, &wb);
    epi_bar();
    const int acc = item % L::ACC_BUFS;
    const uint32_t aph = (uint32_t)((item / L::ACC_BUFS) & 1);
    const bool got = mbar_wait_bounded(&accfull[acc], aph, limit_ns, abort);
    const bool all = __all_sync(0xffffffffu, got);
    if (!all && lane == 0) {
      set_abort(abort, status, ST_TIMEOUT_EPI);
      *epi_abort = 1;
    }
    if (all) tc_fence_after();
    const uint32_t tX = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * 2 * BN + h * kEpiCols);
    const int ml = q * 32 + lane;
    const int m = mtile * BM + ml;
    // pass 1: maxima of |X + Y| * W
    float tmax = 0.f, tmax1 = 0.f;  // (tmax1: BN 160, the group's second k-block)
#pragma unroll 1
    for (int g = 0; g < kEpiCols / 8 && all; ++g) {
      uint32_t rx[8], ry[8];
      tmem_ld8_nowait(tX + g * 8, rx);
      tmem_ld8_nowait(tX + BN + g * 8, ry);
      tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int cl = h * kEpiCols + g * 8 + j;
        float2 v = two_sum(__uint_as_float(rx[j]), __uint_as_float(ry[j]));
        if (hasW) v = arith::mul_pair(v, fW[wb + wm[ml] + wn[cl]]);
        float a = (m < M && ntile * BN + cl < N) ? fabsf(v.x) : 0.f;
        if (fz.k_is_m) {  // k runs over the lanes: maximum per column over the warp
#pragma unroll
          for (int s = 16; s > 0; s >>= 1) a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, s));
          if (lane == 0) xmax[q * BN + cl] = a;
        } else if (BN == kFuseBN || cl / 64 == blk0) {
          tmax = fmaxf(tmax, a);
        } else {
          tmax1 = fmaxf(tmax1, a);
        }
      }
    }
    if (!fz.k_is_m) {
      if (BN == kFuseBN) {
        xmax[h * 128 + ml] = tmax;
      } else {
        xmax[(h * 2) * 128 + ml] = tmax;
        xmax[(h * 2 + 1) * 128 + ml] = tmax1;
      }
    }
    epi_bar();
    if (*epi_abort) break;
    // pass 2: pieces
    if (fz.k_is_m) {
#pragma unroll 1
      for (int g = 0; g < kEpiCols / 8; ++g) {
        uint32_t rx[8], ry[8];
        tmem_ld8_nowait(tX + g * 8, rx);
        tmem_ld8_nowait(tX + BN + g * 8, ry);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int cl = h * kEpiCols + g * 8 + j;
          const int n = ntile * BN + cl;
          if (m >= M || n >= N) continue;
          float2 v = two_sum(__uint_as_float(rx[j]), __uint_as_float(ry[j]));
          if (hasW) v = arith::mul_pair(v, fW[wb + wm[ml] + wn[cl]]);
          const int qb = q & 2;  // the two lane quarters of this 64-entry k-block
          const int E = arith::grid_exp(fmaxf(xmax[qb * BN + cl], xmax[(qb + 1) * BN + cl]));
          float pc[3];
          arith::grid_pieces(v, E, pc);
          const int64_t dst = (int64_t)(rb + rn[cl]) * Kp + m;
#pragma unroll
          for (int p = 0; p < 3; ++p) out[p * fz.piece + dst] = __float2bfloat16_rn(pc[p]);
        }
      }
    } else {
      // the grid exponent of each k-block this thread's columns meet: BN 128,
      // the two column groups of the one block; BN 160, every group's
      // partial maximum for the block (0, the neutral maximum, where a group
      // does not meet it)
      int E0, E1 = 0;
      if (BN == kFuseBN) {
        const int hb = h & ~1;
        E0 = arith::grid_exp(fmaxf(xmax[hb * 128 + ml], xmax[(hb + 1) * 128 + ml]));
      } else {
        float m0 = 0.f, m1 = 0.f;
#pragma unroll
        for (int hh = 0; hh < 4; ++hh) {
          const int b0 = hh * kEpiCols / 64;
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            const float v = xmax[(hh * 2 + s) * 128 + ml];
            if (b0 + s == blk0) m0 = fmaxf(m0, v);
            if (b0 + s == blk1) m1 = fmaxf(m1, v);
          }
        }
        E0 = arith::grid_exp(m0);
        E1 = arith::grid_exp(m1);
      }
#pragma unroll 1
      for (int g = 0; g < kEpiCols / 8; ++g) {
        uint32_t rx[8], ry[8];
        tmem_ld8_nowait(tX + g * 8, rx);
        tmem_ld8_nowait(tX + BN + g * 8, ry);
        tmem_wait_ld();
        const int c0 = h * kEpiCols + g * 8;
        const int n0 = ntile * BN + c0;
        if (m >= M || n0 >= N) continue;
        const int E = (BN == kFuseBN || c0 / 64 == blk0) ? E0 : E1;
        __nv_bfloat16 hp[3][8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float2 v = two_sum(__uint_as_float(rx[j]), __uint_as_float(ry[j]));
          if (hasW) v = arith::mul_pair(v, fW[wb + wm[ml] + wn[c0 + j]]);
          float pc[3];
          arith::grid_pieces(v, E, pc);
#pragma unroll
          for (int p = 0; p < 3; ++p) hp[p][j] = __float2bfloat16_rn(pc[p]);
        }
        const int64_t dst = (int64_t)(rb + rm[ml]) * Kp + n0;
        if (n0 + 8 <= N) {
#pragma unroll
          for (int p = 0; p < 3; ++p) *reinterpret_cast<uint4*>(out + p * fz.piece + dst) = *reinterpret_cast<const uint4*>(hp[p]);
        } else {
          for (int j = 0; j < 8 && n0 + j < N; ++j)
#pragma unroll
            for (int p = 0; p < 3; ++p) out[p * fz.piece + dst + j] = hp[p][j];
        }
      }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&accempty[acc]);
  }
}

// The MMAs of one stage (all its K-steps) for the products whose later
// piece is p (p is a constant after the caller's unrolling).
template <int PREC, int BN, bool PAIR>
__device__ __forceinline__ void issue_piece(int p, uint64_t dA0, uint64_t dB0, uint32_t dX, uint32_t dY,
                                            uint32_t idesc, bool first_kb) {
  using C = Cfg<PREC>;
  using L = Layout<PREC, BN, PAIR>;
#pragma unroll
  for (int kk = 0; kk < C::KB / C::UK; ++kk) {
    const bool first = first_kb && kk == 0;
#pragma unroll
    for (int pr = 0; pr < C::NPROD; ++pr) {
      if ((C::pa(pr) > C::pb(pr) ? C::pa(pr) : C::pb(pr)) != p) continue;
      const uint64_t ad = dA0 + (uint64_t)((C::pa(pr) * L::A_PIECE + kk * C::UK * C::ES) >> 4);
      const uint64_t bd = dB0 + (uint64_t)((C::pb(pr) * L::B_PIECE + kk * C::UK * C::ES) >> 4);
      const uint32_t accum = (first && pr <= 1) ? 0u : 1u;
      const uint32_t d = pr == 0 ? dX : dY;
      if constexpr (PAIR)
        umma_f16_pair(d, ad, bd, idesc, accum);
      else if (C::FMT == 1)
        umma_f16(d, ad, bd, idesc, accum);
      else
        umma_tf32(d, ad, bd, idesc, accum);
    }
  }
}

// PAIR: a cluster of two CTAs computes each 256 x BN tile with cta_group::2
// MMAs issued by rank 0 (the leader): each CTA loads its 128 rows of A and
// BN/2 rows of B into its own shared memory and completes the bytes on the
// leader's stage barriers; the leader's commits arrive on the stage and
// accumulator barriers of both CTAs; each CTA's epilogue drains its own TMEM
// (its 128 rows) and hands the accumulator back on the leader's barrier.
template <int PREC, int BN, bool PAIR>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_tc(const __grid_constant__ GemmMaps maps, int nval,
              float2* __restrict__ Cout, int batch, int M, int N, int K, int kc_blocks, uint32_t* status,
              uint64_t limit_ns, const __grid_constant__ GemmFuse fz, int accum, int test_no_loads) {
  using C = Cfg<PREC>;
  using L = Layout<PREC, BN, PAIR>;
  static_assert(!PAIR || PREC == 3, "CTA pairs for BF16x3 only");
  constexpr int NG = BN / 8;  // 8-column groups of a tile
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + L::BAR_OFF);
  uint64_t* full = bars;  // [stage * NP + piece]
  uint64_t* empty = bars + L::STAGES * C::NP;
  uint64_t* accfull = empty + L::STAGES;
  uint64_t* accempty = accfull + 2;
  uint64_t* mma_done = accempty + 2;
  uint32_t* tmem_holder = (uint32_t*)(bars + L::N_BARS);
  volatile int* abort = (volatile int*)(tmem_holder + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t rank = PAIR ? cluster_rank() : 0u;
  const bool leader = rank == 0;
  // tiles are dealt to CTAs (or CTA pairs) round robin
  const int tile0 = PAIR ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
  const int tstep = PAIR ? (int)(gridDim.x >> 1) : (int)gridDim.x;
  const int mt = (M + L::TM - 1) / L::TM, nt = (N + BN - 1) / BN;
  const int n_tiles = batch * mt * nt;  // host checks n_tiles < 2^31
  // k-blocks of one operand pair, and of all nval pairs in sequence (pair v
  // owns k-blocks [v * nkb1, (v + 1) * nkb1))
  const int nkb1 = (K + C::KB - 1) / C::KB;
  const int nkb = nkb1 * nval;
  // the fused split takes the whole K in one accumulator chunk (host: K <= 1024)
  const int kc0 = (L::FUSE && fz.on) ? nkb : (kc_blocks > 0 ? kc_blocks : C::KC);
  const int kc = kc0 < nkb ? kc0 : nkb;
  const int nchunks = (nkb + kc - 1) / kc;

  if (threadIdx.x == 0) {
    for (int s = 0; s < L::STAGES; ++s) {
      for (int p = 0; p < C::NP; ++p) mbar_init(&full[s * C::NP + p], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&accfull[a], 1);
      // a pair's accumulator is free once the epilogue warps of both CTAs are done
      mbar_init(&accempty[a], PAIR ? 2 * kEpiWarps : kEpiWarps);
    }
    mbar_init(mma_done, 1);
    *abort = 0;
    mbar_fence_init();
  }
  if (warp == 1) {
    if constexpr (PAIR) {
      tmem_alloc_pair(tmem_holder, L::TMEM_COLS);
      tmem_relinquish_pair();
    } else {
      tmem_alloc(tmem_holder, L::TMEM_COLS);
      tmem_relinquish();
    }
  }
  if (warp == 0 && lane < nval) {
    tma_prefetch_desc(&maps.a[lane]);
    tma_prefetch_desc(&maps.b[lane]);
  }
  tc_fence_before();
  if constexpr (PAIR)
    cluster_sync();  // the peer's barriers are initialised before either CTA signals them
  else
    __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;
  float2* fW = reinterpret_cast<float2*>(smem + L::FUSE_OFF);
  if (L::FUSE && fz.on && fz.w_size) {  // product of the absorbed small leaves
    for (uint32_t u = threadIdx.x; u < fz.w_size; u += blockDim.x) {
      int64_t off[kMaxOps];
      for (int j = 0; j < fz.nsmall; ++j) off[j] = 0;
      uint32_t o = u;
      for (int m = fz.wmodes.n - 1; m >= 0; --m) {
        const uint32_t qq = arith::fdiv(o, fz.wmodes.div[m]);
        const uint32_t i = o - qq * fz.wmodes.dim[m];
        o = qq;
        for (int j = 0; j < fz.nsmall; ++j) off[j] += (int64_t)i * fz.wmodes.stride[m][j];
      }
      float2 v = arith::load_any(fz.wptr[0], fz.wdt[0], off[0]);
      for (int j = 1; j < fz.nsmall; ++j) v = arith::mul_pair(v, arith::load_any(fz.wptr[j], fz.wdt[j], off[j]));
      fW[u] = v;
    }
    __syncthreads();
  }
  // operands and the output buffer belong to earlier kernels of the stream
  pdl_wait();
  pdl_launch_dependents();

  if (warp == 0) {
    // (test_no_loads: a self-test issues no copies, so that every wait of
    // the MMA issuer and the epilogue gives up after limit_ns)
    if (lane == 0 && !test_no_loads) {
      // ------------------------------------------------------------ producer
      int stage = 0;
      uint32_t phase = 0;
      int issued[L::STAGES];
      uint32_t issued_phase[L::STAGES];
      for (int s = 0; s < L::STAGES; ++s) issued[s] = 0, issued_phase[s] = 0;
      bool ok = true;
      for (int t = tile0; t < n_tiles && ok; t += tstep) {
        const int ntile = (int)(t % nt);
        const int r = t / nt;
        const int mtile = (int)(r % mt);
        const int b = (int)(r / mt);
        // this CTA's rows of A and of B
        const int arow = mtile * L::TM + (int)rank * BM;
        const int brow = ntile * BN + (int)rank * L::B_ROWS;
        for (int kb = 0; kb < nkb; ++kb) {
          if (!mbar_wait_bounded(&empty[stage], phase ^ 1, limit_ns, abort)) {
            set_abort(abort, status, ST_TIMEOUT_TMA);
            ok = false;
            break;
          }
          uint8_t* sA = smem + stage * L::STAGE;
          uint8_t* sB = sA + C::NP * L::A_PIECE;
          const int v = kb / nkb1, kb1 = kb - v * nkb1;
          // piece by piece, each on its own barrier, so the MMAs of the
          // leading pieces start while the later ones are in flight
#pragma unroll
          for (int p = 0; p < C::NP; ++p) {
            uint64_t* fb = &full[stage * C::NP + p];
            if constexpr (PAIR) {
              // the leader expects both CTAs' bytes; the peer's copies may
              // complete before that (the barrier's pending count goes below zero)
              if (leader) mbar_arrive_expect_tx(fb, 2 * (L::A_PIECE + L::B_PIECE));
              const uint32_t cfb = cluster_addr(fb, 0);
              tma_load_4d_pair(sA + p * L::A_PIECE, &maps.a[v], cfb, kb1 * C::KB, arow, b, p);
              tma_load_4d_pair(sB + p * L::B_PIECE, &maps.b[v], cfb, kb1 * C::KB, brow, b, p);
            } else {
              mbar_arrive_expect_tx(fb, L::A_PIECE + L::B_PIECE);
              tma_load_4d(sA + p * L::A_PIECE, &maps.a[v], fb, kb1 * C::KB, arow, b, p);
              tma_load_4d(sB + p * L::B_PIECE, &maps.b[v], fb, kb1 * C::KB, brow, b, p);
            }
          }
          issued[stage] = 1;
          issued_phase[stage] = phase;
          if (++stage == L::STAGES) stage = 0, phase ^= 1;
        }
      }
      if (!ok) {  // let copies already in flight land before the CTA exits
        if constexpr (PAIR) {
          // the pair's copies complete on the leader's barriers, whose phases
          // the peer does not see: give them a fixed time (copies of a stage
          // take microseconds)
          const uint64_t t0 = global_ns();
          while (global_ns() - t0 < 2000000ull) {
          }
        } else {
          for (int s = 0; s < L::STAGES; ++s)
            if (issued[s]) {
              volatile int no_abort = 0;
              for (int p = 0; p < C::NP; ++p)
                mbar_wait_bounded(&full[s * C::NP + p], issued_phase[s], limit_ns, &no_abort);
            }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && leader) {
      // ------------------------------------------------------------ MMA issuer
      const uint32_t idesc = make_idesc(C::FMT, L::TM, BN);
      int stage = 0;
      uint32_t phase = 0;
      int item = 0;
      bool ok = true, any = false;
      for (int t = tile0; t < n_tiles && ok; t += tstep) {
        for (int ch = 0; ch < nchunks && ok; ++ch, ++item) {
          const int acc = item % L::ACC_BUFS;
          const uint32_t aph = (uint32_t)((item / L::ACC_BUFS) & 1);
          const bool free_acc = PAIR ? mbar_wait_bounded_cluster(&accempty[acc], aph ^ 1, limit_ns, abort)
                                     : mbar_wait_bounded(&accempty[acc], aph ^ 1, limit_ns, abort);
          if (!free_acc) {
            set_abort(abort, status, ST_TIMEOUT_MMA);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t dX = tmem + (uint32_t)(acc * 2 * BN);
          const uint32_t dY = dX + BN;
          const int kb0 = ch * kc, kb1 = min(nkb, kb0 + kc);
          for (int kb = kb0; kb < kb1 && ok; ++kb) {
            const uint32_t sA = smem_u32(smem + stage * L::STAGE);
            const uint32_t sB = sA + C::NP * L::A_PIECE;
            // descriptors of the stage's pieces; each K-step and piece adds its
            // byte offset / 16 to the start-address field (the stage lies
            // below 256 KB of shared memory, so the 14-bit field cannot carry)
            const uint64_t dA0 = smem_desc_k<L::ROW>(sA), dB0 = smem_desc_k<L::ROW>(sB);
            // piece p's barrier releases the products whose later piece is p
            // (x0y0; then x0y1, x1y0, x1y1; then x0y2, x2y0), so the leading
            // products run while the smaller pieces still arrive
#pragma unroll
            for (int p = 0; p < C::NP; ++p) {
              if (!mbar_wait_bounded(&full[stage * C::NP + p], phase, limit_ns, abort)) {
                set_abort(abort, status, ST_TIMEOUT_MMA);
                ok = false;
                break;
              }
              tc_fence_after();
              issue_piece<PREC, BN, PAIR>(p, dA0, dB0, dX, dY, idesc, kb == kb0);
              any = true;
            }
            if (!ok) break;
            if constexpr (PAIR)
              umma_commit_pair(&empty[stage], 3);
            else
              umma_commit(&empty[stage]);
            any = true;
            if (++stage == L::STAGES) stage = 0, phase ^= 1;
          }
          if (ok) {
            if constexpr (PAIR)
              umma_commit_pair(&accfull[acc], 3);
            else
              umma_commit(&accfull[acc]);
          }
        }
      }
      if (!ok && any) {  // let issued MMAs finish before TMEM is freed
        if constexpr (PAIR)
          umma_commit_pair(mma_done, 1);
        else
          umma_commit(mma_done);
        volatile int no_abort = 0;
        mbar_wait_bounded(mma_done, 0, limit_ns, &no_abort);
      }
    }
  } else {
    // -------------------------------------------------------------- epilogue
    bool fused = false;
    if constexpr (L::FUSE) {
      if (fz.on) {
        fused_epilogue<PREC, BN>(fz, fW, smem, tmem, accfull, accempty, abort, status, limit_ns, batch, M, N, mt,
                                 nt, n_tiles, reinterpret_cast<__nv_bfloat16*>(Cout));
        fused = true;
      }
    }
    if (!fused) {
    // warp w owns TMEM lane quarter (w % 4) and the 8-column groups
    // h, h + 4, h + 8, ... of the tile; per chunk each thread loads its row's
    // columns of X and Y group by group, hands the accumulator back to the
    // MMA warp after its last group, and stores X + Y as an exact (hi, lo)
    // pair -- added to the stored pair for chunks after the first (the same
    // thread owns the same outputs in every chunk).
    const int ew = warp - 2;
    const int q = warp & 3;
    const int h = ew >> 2;
    int item = 0;
    bool ok = true;
    for (int t = tile0; t < n_tiles && ok; t += tstep) {
      const int ntile = (int)(t % nt);
      const int r = t / nt;
      const int mtile = (int)(r % mt);
      const int b = (int)(r / mt);
      // C is stored [batch][N][M] (M fastest): for a fixed column the 32
      // lanes of a warp write 32 consecutive rows, 256 contiguous bytes
      const int row = mtile * L::TM + (int)rank * BM + q * 32 + lane;
      float2* cb = Cout + (long long)b * M * N + row;
      const int n0 = ntile * BN;
      for (int ch = 0; ch < nchunks; ++ch, ++item) {
        const int acc = item % L::ACC_BUFS;
        const uint32_t aph = (uint32_t)((item / L::ACC_BUFS) & 1);
        // every lane waits, then the warp agrees (tcgen05.ld is warp-collective)
        const bool got = mbar_wait_bounded(&accfull[acc], aph, limit_ns, abort);
        if (!__all_sync(0xffffffffu, got)) {
          if (lane == 0) set_abort(abort, status, ST_TIMEOUT_EPI);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tX = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * 2 * BN);
        // groups of 8 columns: X and Y of a group in 16 registers (all
        // register indices compile-time constants)
#pragma unroll 1
        for (int g = h; g < NG; g += 4) {
          uint32_t rx[8], ry[8];
          tmem_ld8_nowait(tX + g * 8, rx);
          if (C::NPROD > 1) tmem_ld8_nowait(tX + BN + g * 8, ry);
          tmem_wait_ld();
          if (g + 4 >= NG) {  // this warp's last group: the accumulator is free for the next chunk
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
              if constexpr (PAIR)
                mbar_arrive_cluster(cluster_addr(&accempty[acc], 0));
              else
                mbar_arrive(&accempty[acc]);
            }
          }
          if (row < M) {
            const int c0 = n0 + g * 8;
            float2* dst = cb + (long long)c0 * M;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              if (c0 + j < N) {
                float2 v = two_sum(__uint_as_float(rx[j]), C::NPROD > 1 ? __uint_as_float(ry[j]) : 0.f);
                if (ch > 0 || accum) v = pair_add(dst[(long long)j * M], v);
                dst[(long long)j * M] = v;
              }
            }
          }
        }
      }
    }
    }
  }

  tc_fence_before();
  if constexpr (PAIR)
    cluster_sync();  // neither CTA frees TMEM or exits while the pair still works
  else
    __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    if constexpr (PAIR)
      tmem_dealloc_pair(tmem, L::TMEM_COLS);
    else
      tmem_dealloc(tmem, L::TMEM_COLS);
  }
}

// clusters of two that can be resident at once, per device (measured once
// by gemm_prepare; half the SMs when unknown)
constexpr int kMaxDevices = 64;
template <int PREC, int BN>
int* pair_clusters() {
  static int n[kMaxDevices] = {};
  return n;
}

template <int PREC, int BN, bool PAIR>
cudaError_t launch_t(const GemmArgs& a, int sm_count, cudaStream_t st) {
  using L = Layout<PREC, BN, PAIR>;
  const long long tiles = (long long)a.batch * ((a.M + L::TM - 1) / L::TM) * ((a.N + BN - 1) / BN);
  if (tiles <= 0) return cudaSuccess;
  if (a.fuse.on && (!L::FUSE || a.fuse.w_size > (uint32_t)(L::FUSE_W / 8) || a.accum || a.nval != 1))
    return cudaErrorInvalidValue;
  if (a.nval < 1 || a.nval > kGemmVals) return cudaErrorInvalidValue;
  if constexpr (PAIR) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorInvalidDevice;
    int ncl = dev >= 0 && dev < kMaxDevices ? pair_clusters<PREC, BN>()[dev] : 0;
    if (ncl <= 0) ncl = sm_count / 2;
    const int grid = 2 * (int)(tiles < ncl ? tiles : ncl);
    return launch_k_pair(k_gemm_tc<PREC, BN, true>, dim3(grid), dim3(kThreads), (size_t)L::SMEM, st, a.maps, a.nval,
                         (float2*)a.C, a.batch, a.M, a.N, a.K, a.kc_blocks, a.status, a.limit_ns, a.fuse, a.accum,
                         a.test_no_loads);
  } else {
    const int grid = (int)(tiles < sm_count ? tiles : sm_count);
    return launch_k(k_gemm_tc<PREC, BN, false>, dim3(grid), dim3(kThreads), (size_t)L::SMEM, st, a.maps, a.nval,
                    (float2*)a.C, a.batch, a.M, a.N, a.K, a.kc_blocks, a.status, a.limit_ns, a.fuse, a.accum,
                         a.test_no_loads);
  }
}

template <int PREC, int BN, bool PAIR>
cudaError_t prepare_t() {
  using L = Layout<PREC, BN, PAIR>;
  cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<PREC, BN, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
  if (e != cudaSuccess || !PAIR) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * (unsigned)(sms / 2));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = L::SMEM;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if ((e = cudaOccupancyMaxActiveClusters(&n, k_gemm_tc<PREC, BN, PAIR>, &cfg)) != cudaSuccess) return e;
  if (dev >= 0 && dev < kMaxDevices) pair_clusters<PREC, BN>()[dev] = n > 0 ? n : sms / 2;
  return cudaSuccess;
}

// the N tiles instantiated, in kGemmBlockN order; CTA pairs for BF16x3 only
template <int PREC, bool PAIR>
cudaError_t launch_p(const GemmArgs& a, int sm_count, cudaStream_t st) {
  if constexpr (PAIR) {
    if (a.bn == 256) return launch_t<PREC, 256, PAIR>(a, sm_count, st);
    if (a.bn == 224) return launch_t<PREC, 224, PAIR>(a, sm_count, st);
  }
  if constexpr (PREC == 3 && !PAIR) {
    if (a.bn == kGemmWideN[0]) return launch_t<PREC, kGemmWideN[0], PAIR>(a, sm_count, st);
    if (a.bn == kGemmWideN[1]) return launch_t<PREC, kGemmWideN[1], PAIR>(a, sm_count, st);
  }
  switch (a.bn) {
    case 128: return launch_t<PREC, 128, PAIR>(a, sm_count, st);
    case 112: return launch_t<PREC, 112, PAIR>(a, sm_count, st);
    case 96: return launch_t<PREC, 96, PAIR>(a, sm_count, st);
    case 80: return launch_t<PREC, 80, PAIR>(a, sm_count, st);
    case 64: return launch_t<PREC, 64, PAIR>(a, sm_count, st);
    case 48: return launch_t<PREC, 48, PAIR>(a, sm_count, st);
    default: return cudaErrorInvalidValue;
  }
}
template <int PREC, bool PAIR>
cudaError_t prepare_p() {
  cudaError_t e = cudaSuccess;
  for (cudaError_t x : {prepare_t<PREC, 128, PAIR>(), prepare_t<PREC, 112, PAIR>(), prepare_t<PREC, 96, PAIR>(),
                        prepare_t<PREC, 80, PAIR>(), prepare_t<PREC, 64, PAIR>(), prepare_t<PREC, 48, PAIR>()})
    if (e == cudaSuccess) e = x;
  if constexpr (PAIR) {
    if (e == cudaSuccess) e = prepare_t<PREC, 256, PAIR>();
    if (e == cudaSuccess) e = prepare_t<PREC, 224, PAIR>();
  }
  if constexpr (PREC == 3 && !PAIR) {
    if (e == cudaSuccess) e = prepare_t<PREC, kGemmWideN[0], PAIR>();
    if (e == cudaSuccess) e = prepare_t<PREC, kGemmWideN[1], PAIR>();
  }
  return e;
}

// A single warp waits on an mbarrier that nothing completes, with the same
// bounded wait the GEMM pipeline uses; after limit_ns it gives up and sets
// the dependency-timeout bit of the status word.  Exercises the device-side
// failure path without faulting or hanging the GPU.
__global__ void k_bounded_wait_probe(uint32_t* status, uint64_t limit_ns) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    mbar_fence_init();
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(&bar, 0, limit_ns, &abort_flag);
  if (!__all_sync(0xffffffffu, ok) && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT_DEP);
}

}  // namespace

cudaError_t launch_bounded_wait_probe(uint32_t* status, uint64_t limit_ns, cudaStream_t st) {
  k_bounded_wait_probe<<<1, 32, 0, st>>>(status, limit_ns);
  return cudaGetLastError();
}

bool gemm_bn_supported(int bn, int pair, int prec) {
  for (int b : kGemmBlockN)
    if (b == bn) return true;
  if (!pair && prec == 3)
    for (int b : kGemmWideN)
      if (b == bn) return true;
  if (pair)
    for (int b : kGemmPairWideN)
      if (b == bn) return true;
  return false;
}

cudaError_t gemm_prepare() {
  cudaError_t e = prepare_p<1, false>();
  if (e == cudaSuccess) e = prepare_p<2, false>();
  if (e == cudaSuccess) e = prepare_p<3, false>();
  if (e == cudaSuccess) e = prepare_p<3, true>();
  return e;
}
int gemm_k_block(int prec) { return prec == 3 ? Cfg<3>::KB : Cfg<1>::KB; }

cudaError_t launch_gemm(const GemmArgs& a, int sm_count, cudaStream_t st) {
  if (a.pair && (a.prec != 3 || a.fuse.on)) return cudaErrorInvalidValue;
  switch (a.prec) {
    case 1: return launch_p<1, false>(a, sm_count, st);
    case 2: return launch_p<2, false>(a, sm_count, st);
    case 3: return a.pair ? launch_p<3, true>(a, sm_count, st) : launch_p<3, false>(a, sm_count, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace qtpu
