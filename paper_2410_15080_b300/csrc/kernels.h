// Launch interfaces of the h-TN kernels (host side).
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace qtpu {

constexpr int kMaxModes = 12;

// device status word bits (OR-ed in by any thread that gives up)
enum : uint32_t {
  ST_TIMEOUT_TMA = 1u << 0,   // producer waited too long for a free stage
  ST_TIMEOUT_MMA = 1u << 1,   // MMA issuer waited too long for data / accumulator
  ST_TIMEOUT_EPI = 1u << 2,   // epilogue waited too long for an accumulator
  ST_TIMEOUT_DEP = 1u << 3,   // a dependency counter never completed
  ST_BAD_ARG = 1u << 8,       // a kernel saw inconsistent arguments and did nothing
};

// A group of tensor modes (outermost first) with element strides into two
// operands.  A stride of 0 means the operand does not carry that mode.
struct ModeTab {
  int n = 0;
  int64_t dim[kMaxModes];
  int64_t sa[kMaxModes];
  int64_t sb[kMaxModes];
};

// out[o] = sum_l A[offA(o) + offA(l)] * B[offB(o) + offB(l)]   (FP64)
// o runs over the `out` modes (dense output, last mode fastest), l over the
// `loop` modes.  B may be null (single-operand reduction: B == 1).
struct ContractArgs {
  ModeTab out, loop;
  int64_t n_out = 1, n_loop = 1;
  int accum = 0;  // add to the output instead of overwriting it
};

enum DType { DT_F32 = 0, DT_F64 = 1, DT_F32X2 = 2 /* (hi, lo) float pair per entry */ };

// ---------------------------------------------------------------- gather
constexpr int kMaxOps = 6;

// n / d for 32-bit n via a multiply-high and a shift (d fixed per launch)
struct FastDiv {
  uint32_t magic = 0, shift = 0;
};
FastDiv make_fastdiv(uint32_t d);

// modes (outermost first) with their element strides in every operand
struct GModes {
  int n = 0;
  uint32_t dim[kMaxModes];
  FastDiv div[kMaxModes];
  int64_t stride[kMaxModes][kMaxOps];
};

enum GatherMode {
  GW_DENSE_PAIR = 0,   // write (hi, lo) float pairs, dense in out-mode order
  GW_DENSE_F64 = 1,    // write FP64, dense
  GW_SPLIT_BF16X3 = 2, // write 3 BF16 piece planes [rows][Kp]
  GW_SPLIT_TF32X2 = 3, // write 2 TF32 piece planes
  GW_SPLIT_TF32 = 4    // write 1 TF32 plane
};

// value(o) = sum over loop modes of prod_j X_j[...]; for the split modes the
// entry index is (row over `out`, k over `kmodes`).
struct GatherArgs {
  int nops = 1;
  int mode = GW_DENSE_PAIR;
  const void* ptr[kMaxOps] = {};
  float2* wg = nullptr;  // large W (fast dense path): computed once per launch into
                         // this global buffer by a small kernel, then copied by every block
  int dt[kMaxOps] = {};
  GModes out, loop, kmodes;
  uint32_t n_out = 1, n_loop = 1;        // dense modes
  uint32_t n_rows = 0, K = 0, Kp = 0;   // split modes
  int row_fast = 0;  // split: operand 0 is contiguous along rows (read rows fastest)
  // fast path: operands [0, nbig) are large stored tensors; the small leaves
  // that follow are pre-multiplied into a table W held in shared memory, W
  // dense over `wmodes` (per small operand j: stride[m][nbig + j]); in the
  // out/loop/k tables the W operand occupies slot nbig with W's own strides
  int nbig = 0;          // 0 = fast path not set up
  int fan = 0;           // split fast path: 1 = innermost k mode, 2 = innermost row
                         // mode is carried by W alone (dim fan_f): one thread
                         // computes the fan_f entries from one operand load
  int fan_f = 1;
  uint32_t w_size = 0;   // entries of W (0 = no small operands)
  GModes wmodes;
  // fast dot path (two large operands, no W, a long sum over few outputs):
  // the loop splits into a tile of `tile_n` entries over the modes nearest
  // unit stride in either operand, and the outer modes left in `loop`.  The
  // tile's modes sit in `kmodes` in operand-0 stride order (stride 0: operand
  // 0, stride 1: slot in the tile) and in `wmodes` in slot order (stride 0:
  // operand 1).  Each block adds `chunks`-th of one output's tiles into
  // `scratch`, and a second kernel adds the chunks of every output.
  int dot = 0;
  uint32_t tile_n = 0, n_outer = 0, chunks = 0;
  float2* scratch = nullptr;
  // dense modes: add to the output instead of overwriting it (a sum over a
  // sliced index that the step contracts, accumulated slice value by value)
  int accum = 0;
};
constexpr uint32_t kDotMaxTile = 2048;
// scratch entries a dot launch may use (float2)
inline size_t dot_scratch_entries(int sm_count) { return (size_t)sm_count * 24; }
cudaError_t launch_gather(const GatherArgs& a, void* out, int sm_count, cudaStream_t st);
// The same computation through the typed fast kernels (shared-memory table of
// the small factors); cudaErrorNotSupported when no instantiation fits.
constexpr uint32_t kMaxW = 4096;
constexpr uint32_t kGlobalW = 1024;  // dense-gather W tables from this size go through GatherArgs::wg
cudaError_t launch_gather_fast(const GatherArgs& a, void* out, int sm_count, cudaStream_t st);

cudaError_t launch_contract(const void* A, int dtA, const void* B, int dtB, double* out,
                            const ContractArgs& a, int sm_count, cudaStream_t st);

// Fused operand split (BF16x3, a single accumulator chunk): the GEMM's
// epilogue writes the BF16x3 pieces of the next GEMM's operand, on the grid of
// grid_pieces, straight from the accumulators instead of the (hi, lo) result.
// The consumer's K is the tile's M rows (k_is_m) or its N columns, in the same
// order; batch and the other tile coordinate map onto consumer rows through
// per-digit row strides, and absorbed small factors multiply each entry
// through a table W over their joint indices (per-digit W strides).
constexpr uint32_t kFuseMaxW = 1024;
// a fused-epilogue producer whose N side is 129-160 wide may run one 160-column
// tile instead of two of 128 (one CTA, one TMEM buffer); its table of small
// factors holds at most kFuseMaxWWide entries (shared memory)
constexpr int kFuseWideBN = 160;
constexpr uint32_t kFuseMaxWWide = 256;
struct GemmFuse {
  int on = 0;
  int k_is_m = 1;
  uint32_t Kp = 0;                // consumer row length
  int64_t piece = 0;              // entries per piece plane
  GModes bmodes, mmodes, nmodes;  // digits of batch / m / n: stride 0 = consumer row
                                  // contribution, stride 1 = W offset contribution
  int nsmall = 0;                 // small factors in W
  const void* wptr[kMaxOps] = {};
  int wdt[kMaxOps] = {};
  GModes wmodes;                  // W's modes, stride j = small factor j
  uint32_t w_size = 0;
};

// A GEMM may add up the products of several operand pairs (one per value of
// a sliced index the step contracts): C = sum_v A_v B_v, all accumulated in
// TMEM before one epilogue.
constexpr int kGemmVals = 8;
struct GemmMaps {
  CUtensorMap a[kGemmVals], b[kGemmVals];  // 4-D maps over [pieces][batch][rows][Kp]
};

// prec: 1 = TF32 (1 piece, 1 product), 2 = 3xTF32 (2 pieces, 3 products),
//       3 = BF16x3 (3 pieces, 6 products)
struct GemmArgs {
  GemmMaps maps;         // operand pair v in maps.a[v], maps.b[v], v < nval
  int nval = 1;
  void* C = nullptr;     // [batch][N][M] (hi, lo) float pairs, dense (M fastest)
  int batch = 0, M = 0, N = 0, K = 0;
  int kc_blocks = 0;     // k-blocks per TMEM accumulation chunk (0 = all)
  int prec = 3;
  uint32_t* status = nullptr;
  uint64_t limit_ns = 2000000000ull;
  GemmFuse fuse;         // fuse.on: C receives the consumer's piece planes
  int accum = 0;         // add the product to the stored (hi, lo) result (not with fuse)
  int bn = 128;          // N tile: kGemmBlockN, kGemmPairWideN with pair, kGemmWideN in BF16x3 without (fuse: 128, 160)
  int pair = 0;          // BF16x3 without fuse: 256-row tiles on a cluster of two CTAs
                         // (cta_group::2), each staging BN/2 rows of B (the B map's box)
  int test_no_loads = 0;  // failure-path self-test: no copies are issued, every wait gives up
};
cudaError_t launch_gemm(const GemmArgs& a, int sm_count, cudaStream_t st);
// one warp waiting (bounded) on a barrier nothing completes: sets ST_TIMEOUT_DEP
cudaError_t launch_bounded_wait_probe(uint32_t* status, uint64_t limit_ns, cudaStream_t st);
// one-time per-device setup of the GEMM kernels (shared-memory attribute)
cudaError_t gemm_prepare();

// One task of the persistent batched kernel: a gather launch of one network
// with its operand pointers resolved.  Dense tasks have one work unit per 256
// outputs; block-mode tasks (long sums over few outputs) one per output.  A
// unit runs after `dep_units` units of task `dep` (the network's previous
// launch) are done.
struct BatchTask {
  GatherArgs g;
  void* dst = nullptr;
  uint32_t n_units = 0;
  int block_mode = 0;
  int f64out = 0;
  int dep = -1;
  uint32_t dep_units = 0;
  uint32_t* status = nullptr;  // the network's status word
};
cudaError_t launch_batch_persistent(const BatchTask* tasks, int n_tasks, const uint64_t* unit_start,
                                    unsigned long long* next_unit, uint32_t* done, uint64_t limit_ns, int* abort_flag,
                                    int grid, cudaStream_t st);

// Build the 4-D TMA map of a split operand buffer (returns false on failure).
bool make_operand_map(CUtensorMap* map, void* base, int prec, int64_t batch, int64_t rows, int64_t K,
                      int64_t Kp, int box_rows);

// N tiles of the GEMM kernel (the M tile is 128 rows); B operand maps use a
// box of bn rows
constexpr int kGemmBlockN[6] = {128, 112, 96, 80, 64, 48};
// wider N tiles, on CTA pairs only (one TMEM accumulator buffer)
constexpr int kGemmPairWideN[2] = {256, 224};
// wider N tiles of BF16x3 on one CTA (one TMEM accumulator buffer): 160 (also
// the fused-split producer's), and 144 for N sides that are multiples of 144
constexpr int kGemmWideN[2] = {kFuseWideBN, 144};
bool gemm_bn_supported(int bn, int pair = 0, int prec = 3);
int gemm_k_block(int prec);  // K elements per pipeline stage

}  // namespace qtpu
