// Executor: turns a Plan into a list of kernel launches on one device/stream.
#pragma once
#include <algorithm>
#include <array>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/qtpu_htn.h"
#include "kernels.h"
#include "planner.h"

namespace qtpu {

struct Leaf {
  Inds ids;
  std::vector<int64_t> dims, strides;  // strides in elements
  int dt = DT_F64;
  const void* ptr = nullptr;
  int kind = 0;  // QTPU_QT or QTPU_CT
};

enum KernelClass { KC_CONTRACT = 0, KC_SPLIT = 1, KC_GEMM = 2, KC_REDUCE = 3, KC_COUNT = 4 };

enum LaunchKind { LK_GATHER = 0, LK_GEMM = 1, LK_CONTRACT64 = 2 };

// Destinations of a launch's output
enum : int { DST_PARTIAL = -1, DST_SPLIT_A = -2, DST_SPLIT_B = -3, DST_OUT = -4, DST_SIDE = -5, DST_KEPT = -6 };

struct Launch {
  int kind = LK_GATHER;
  int kclass = KC_CONTRACT;
  int nsrc = 0;
  int src[kMaxOps] = {};  // operand tensor ids: leaf (< n_leaves) or intermediate
  int dst = DST_PARTIAL;  // intermediate id (>= n_leaves) or a DST_* code
  GatherArgs g;           // LK_GATHER (operand pointers patched per slice)
  bool has_fast = false;  // typed fast path available (gf, operands gf_src)
  GatherArgs gf;
  int gf_src[kMaxOps] = {};
  GemmArgs gemm;          // LK_GEMM (split buffers fixed; C patched)
  ContractArgs c64;       // LK_CONTRACT64 (FP64 path)
  double flops = 0, bytes = 0;
  // side stream: a split whose operands are all leaves runs on a second
  // stream into its own buffer (side_off) ahead of the chain; the GEMM that
  // consumes it waits for its event (wait_side: indices into side events)
  int side = -1;
  size_t side_off = 0;
  int wait_side[2] = {-1, -1};
  // LK_GEMM operands: index of the split launch that writes each one, or the
  // intermediate whose arena slot holds its pieces (written by the epilogue
  // of the GEMM that produced it), with that layout's row length
  int opnd_split[2] = {-1, -1};
  int opnd_fused[2] = {-1, -1};
  uint32_t opnd_kp[2] = {0, 0};
  // LK_GEMM with gemm.fuse.on: the small leaves of the fused W (patched per slice)
  int fuse_src[kMaxOps] = {};
  // fast gather/split with a large W table: its byte offset in Executor::wbuf
  int64_t wg_off = -1;
  // slice reuse: the sliced positions the launch loops over (the values its
  // inputs depend on) and those its result depends on (one kept copy per
  // value); it adds up over din \ dout.  runs = executions per contraction.
  uint64_t din = 0, dout = 0;
  int64_t runs = 1;      // its operand products per contraction (FLOPs = flops x runs)
  int64_t n_launch = 1;  // its kernel launches per contraction (a GEMM sums up to kGemmVals runs)
  // LK_GEMM whose operand is a kept result with several copies (pieces
  // written by the producing GEMM's epilogue): one map per copy, and the
  // intermediate holding them
  std::vector<CUtensorMap> tm_copies[2];
  int opnd_owner[2] = {-1, -1};
  // LK_GEMM: its problem as the tile table keys it (prec, batch, m, n, k:
  // the step's own index-group sizes, before orientation), and whether the
  // orientation and N tile are fixed (by a fused-split consumer)
  int64_t tile_key[5] = {};
  bool tile_fixed = false;
  // a split whose result is kept per value of its own sliced positions
  // (DST_KEPT): the slot count, bytes per slot, its region in keptbuf and the
  // GEMM side it feeds; the GEMM it feeds holds one map per slot
  int64_t kept_slots = 0;
  size_t kept_slot_bytes = 0, kept_off = 0;
  int kept_side = 0;
  std::vector<CUtensorMap> kept_maps[2];
};

// One unit of the slice-reuse schedule: a launch, preceded (for a GEMM) by
// the splits of its operands.  The group loops over the values of the main
// launch's din in `order` (last fastest); a split runs only when the values
// of its own din change.
struct Group {
  int main = -1;
  int split[2] = {-1, -1};
  std::vector<int> order;
  // a GEMM group: the positions it contracts (outside the blocked ones),
  // summed inside one launch over up to kGemmVals operand pairs
  uint64_t sum_pos = 0;
};

// Where an intermediate lives: arena offset of copy 0, bytes per copy, and
// the sliced positions indexing its copies (those its value depends on,
// outside the blocked positions).
struct Stored {
  size_t off = 0, bytes = 0;
  std::vector<int> cpos;
};

struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> ev;  // pairs
  std::vector<int> kind;
  std::vector<int> lidx;        // launch index (-1: the reduction)
  std::vector<double> flops, bytes;
  size_t used = 0;
  size_t graph_events = 0;  // event pairs inside the profiling graph
};

struct Executor {
  int device = 0;
  int sm_count = 148;
  cudaStream_t stream = nullptr;
  int prec = 3;
  int kc_blocks = 0;
  int n_leaves = 0;
  std::vector<Launch> launches;  // one slice, in order
  Launch reduce;                 // slice sum + final reduction -> dev_out
  std::vector<size_t> inter_off; // arena byte offset per intermediate (id - n_leaves)
  // per leaf: (slice position, stride) of each sliced index it carries
  std::vector<std::vector<std::pair<int, int64_t>>> leaf_slice;
  std::vector<int64_t> slice_dims;
  int64_t n_slices = 1;
  int64_t final_size = 1;        // entries of the last step's result per slice
  int inter_dt = DT_F32X2;       // storage of intermediates
  int partial_dt = DT_F64;       // storage of the per-slice results (FP64, or pairs after a GEMM)
  size_t split_a_bytes = 0;      // offset of the B operand region
  // operand splits of one GEMM launch over several values of a sliced index
  // it contracts each get a slot: slot bytes per side, slots
  size_t split_slot[2] = {0, 0};
  int n_split_slots = 1;
  // device memory (owned)
  uint8_t* arena = nullptr;
  size_t arena_bytes = 0;
  uint8_t* splitbuf = nullptr;
  size_t split_bytes = 0;
  uint8_t* partial = nullptr;
  uint32_t* status = nullptr;
  double* out_stage = nullptr;   // staging buffer of the host-buffer entry point
  float2* dot_scratch = nullptr; // per-chunk sums of the dot-reduction kernel
  uint8_t* wbuf = nullptr;       // precomputed large W tables, one region per launch
  size_t wbuf_bytes = 0;
  int n_tc_steps = 0;
  int n_fused_steps = 0;         // absorption steps folded into a consumer
  int n_fused_splits = 0;        // operand splits written by the producing GEMM's epilogue
  int64_t launches_per_contract = 0;
  bool lowered = false;
  Profiler prof;
  // CUDA graph of one whole contraction, replayed on a private stream
  // (index 0: plain, 1: with profiling events)
  bool use_graph = true;
  cudaStream_t own = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  // concurrent leaf splits (graph mode, unsliced plans only)
  int n_side = 0;
  uint8_t* sidebuf = nullptr;
  size_t side_bytes = 0;
  // kept split results (sliced plans): one region per kept split
  uint8_t* keptbuf = nullptr;
  size_t kept_split_bytes = 0;
  cudaStream_t side_stream = nullptr;
  std::vector<cudaEvent_t> side_ev;  // one per side launch, plus fork and join
  double planned_side_bytes = 0;
  // slice reuse (sliced plans): the schedule's groups, the positions held
  // fixed per block (bit mask), the layout of every intermediate
  std::vector<Group> groups;
  uint64_t fixed = 0;
  uint64_t reuse_budget = 0;
  size_t kept_bytes = 0;         // arena bytes beyond the one-slice-at-a-time layout
  std::vector<Stored> stored;    // per intermediate (id - n_leaves)
  double flops_executed = 0;     // useful FLOPs one full contraction executes
  double flops_no_reuse = 0;     // the same with every slice computed in full
  size_t workspace_bytes() const {
    return arena_bytes + split_bytes + side_bytes + kept_split_bytes + wbuf_bytes +
           (size_t)std::max<int64_t>(final_size, 1) * 8;
  }
};

// Build launch descriptors and allocate the workspace.  Returns an empty
// string on success, else an error message (*code receives a qtpu_status).
// reuse_bytes: device memory for results kept across slices (0 = default).
// GEMM tile table: per problem (prec, batch, m, n, k -- m and n the sizes of
// the step's own index groups), the orientation (swap: m along the N tile)
// and the N tile, with the measured times of that choice and of the padding
// rule's choice.
struct TileChoice {
  int swap = 0;
  int bn = 128;
  int pair = 0;  // BF16x3: 256-row tiles on a CTA pair
  double ms = 0, ms_rule = 0, ms_base = 0;
};
using TileKey = std::array<int64_t, 5>;
using TileTable = std::map<TileKey, TileChoice>;
// "" on success; the file holds lines "prec batch m n k : swap bn [ms ms_rule
// ms_base]"
std::string load_tile_table(const std::string& path, TileTable* t);
std::string save_tile_table(const std::string& path, const TileTable& t);
// the gemm_tiles_b300.txt beside the library
std::string default_tile_table_path();
// Orientation and N tile of a GEMM step: the table's entry when it has one
// (for m x n or n x m), else the padding rule: the fewest tiles weighted by
// (N + 128) for a tile of N columns -- on B300 a tile's time grows far less
// than its width (112-column tiles of a 1296 x 1296 x 576 step took 0.98 of
// the time of 128-column ones) -- ties keeping *swap as given and the wider
// tile.
void choose_tile(const TileTable* t, int prec, double nb, double nm, double nn, double nk, bool* swap, int* bn,
                 int* pair);

std::string exec_build(Executor* ex, const Plan& plan, const std::vector<Leaf>& leaves, const DimMap& dims,
                       int prec, int* code, bool dry_run = false, uint64_t reuse_bytes = 0,
                       const TileTable* tiles = nullptr);
// Time every GEMM problem of the lowered plan (fixed tiles excepted) in each
// valid orientation and N tile on synthetic operand pieces on the current
// device, `reps` timed launches each (median), and store the fastest choice
// per problem in *t.  *n receives the number of problems timed.
std::string exec_autotune(const Executor* ex, int reps, TileTable* t, int* n, int* code);
// One line per launch of the lowered contraction (kind, operands, shape,
// useful FLOPs, algorithmic bytes) -- available after exec_build, also on a
// dry run.
std::string exec_describe(const Executor* ex);
// Enqueue the whole contraction; writes output_size FP64 entries to dev_out.
std::string exec_run(Executor* ex, const std::vector<Leaf>& leaves, double* dev_out, cudaStream_t st, int* code);
// The same with direct launches, each waiting for the events (one per leaf,
// recorded after that leaf's upload) of the leaves it reads.
std::string exec_run_host(Executor* ex, const std::vector<Leaf>& leaves, double* dev_out, cudaStream_t st,
                          const cudaEvent_t* leaf_ready, int* code);
// Tasks of one network for the persistent batched kernel (unsliced, gather
// launches only), its final reduction writing dev_out; false if the network
// is not eligible.
bool exec_batch_tasks(const Executor* ex, const std::vector<Leaf>& leaves, double* dev_out,
                      std::vector<BatchTask>* out);
// Leaves in the order the schedule first reads them (upload order).
std::vector<int> exec_leaf_order(const Executor* ex, int n_leaves);
// Enqueue one whole contraction on `st` with direct launches, result to out
// (used to capture several networks into one graph).
cudaError_t exec_enqueue(Executor* ex, const std::vector<Leaf>& leaves, double* out, cudaStream_t st);
// Contract slices [first, first + count) only (direct launches); dev_out
// receives their sum.
std::string exec_run_slices(Executor* ex, const std::vector<Leaf>& leaves, int64_t first, int64_t count,
                            double* dev_out, cudaStream_t st, int* code);
void exec_free(Executor* ex);
// Set the message qtpu_last_error(NULL) returns (calls that take no handle).
void set_global_error(const char* msg);
// The learned cost model's plan choice (qtpu_plan_opts.cost_model = 1); returns
// a qtpu_status, *err on failure.
int plan_by_cost_model(const std::vector<Inds>& li, const DimMap& dims, const Inds& output,
                       const qtpu_plan_opts& o, const std::vector<Leaf>& leaves, int device, void* stream,
                       const TileTable* tiles, Plan* chosen, std::string* err);
// Hyper-search over the exact tree and randomised greedy candidates, ranked
// by the FLOPs their lowered launch lists execute (search.cpp).  Returns a
// qtpu_status.
int plan_hyper(const std::vector<Inds>& li, const DimMap& dims, const Inds& output, const qtpu_plan_opts& o,
               const std::vector<Leaf>& leaves, const TileTable* tiles, Plan* chosen, std::string* err);
// Sum the timed launches per class (after a stream sync) and reset.
std::string exec_profile_read(Executor* ex, double* ms, int64_t* launches, double* flops, double* bytes);
// Every timed launch (launch index, ms) in order (after a stream sync), and reset.
std::string exec_profile_launches(Executor* ex, std::vector<int>* index, std::vector<double>* ms);

// Features of one lowered launch for the learned cost model: kind, work,
// shape, tile fill and access pattern (kLaunchFeatures floats).
constexpr int kLaunchFeatures = 32;
void exec_launch_features(const Executor* ex, size_t i, float* f);

}  // namespace qtpu
