// Host contraction planner: greedy pairwise order + slicing on exact costs.
//
// Section 4.2: an h-TN's post-processing cost is the cost of contracting its
// classical TN and depends on the pairwise order; section 6.1 step 3 plans
// that order before the contraction.  The rules (candidates, cost key,
// tie-breaks, index grouping, slicing key) are stated in planner.cpp and are
// the same as the FP64 reference planner the tests compare against.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "u256.h"

namespace qtpu {

using Inds = std::vector<int64_t>;

struct PlanStep {
  int x = 0, y = 0, out = 0;  // operand ids (x < y) and result id
  Inds batch, m, n, k, sa, sb;
  Inds out_inds() const {
    Inds r(batch);
    r.insert(r.end(), m.begin(), m.end());
    r.insert(r.end(), n.begin(), n.end());
    return r;
  }
};

struct Plan {
  int n_leaves = 0;
  Inds output;
  std::vector<Inds> tensor_inds;  // every id: leaves then step results
  std::vector<PlanStep> steps;
  Inds final_inds, final_sum;
  Inds sliced;
  U256 n_slices{1};
  // per-slice accounting (sliced indices count as dim 1)
  std::vector<U256> step_size, step_flops;
  U256 flops_per_slice, flops_total, peak;
  uint32_t search = 0;     // candidates searched (0: a single plan)
  uint64_t search_seed = 0;
  int search_exact = -1;   // >= 0: an exact-search plan over this many tensors
  std::string search_note; // a hyper-search's choice (plan text line)
};

// index id -> dim lookup
struct DimMap {
  std::vector<std::pair<int64_t, int64_t>> kv;  // sorted by id
  int64_t get(int64_t id) const;
  bool has(int64_t id) const;
  void set(int64_t id, int64_t d);
  std::vector<int64_t> ids() const;
};

enum PlanErr { PLAN_OK = 0, PLAN_OVERFLOW = 1, PLAN_LIMIT = 2, PLAN_TOO_MANY = 3 };

// Greedy order then slicing.  Returns PLAN_OK, PLAN_OVERFLOW (a size >= 2^255)
// or PLAN_LIMIT (peak limit unreachable).
// seed != 0: randomised greedy (candidate plans for the cost model): at each
// step the pair is drawn uniformly among the kRandTop best keys with the
// SplitMix64 generator seeded by `seed`.
constexpr int kRandTop = 3;
int make_plan(const std::vector<Inds>& leaves, const DimMap& dims, const Inds& output,
              uint64_t max_bytes, uint64_t n_slices, int64_t slice_dim, Plan* plan, uint64_t seed = 0);

// Best of n candidates (seeds seed .. seed+n-1) by total FLOPs; ties keep the
// lower seed.  *chosen receives the winning seed.
int make_plan_best(const std::vector<Inds>& leaves, const DimMap& dims, const Inds& output, uint64_t max_bytes,
                   uint64_t n_slices, int64_t slice_dim, uint64_t seed, uint32_t n, Plan* plan, uint64_t* chosen);

// Slice a plan's fixed tree (same rule as make_plan) and fill its accounting.
int finish_plan(const DimMap& dims, const Inds& output, uint64_t max_bytes, uint64_t n_slices, int64_t slice_dim,
                Plan* plan);

// Exact order search (section 6.1 step 3, beyond greedy): every small leaf
// (<= 256 entries) is first contracted, in ascending id, into the lowest-id
// large leaf sharing an index with it; over the m tensors left (ascending
// id) the cheapest contraction tree is found by dynamic programming over
// subsets with the planner's step cost: cost(S) = min over A (containing S's
// lowest member, A != S) of cost(A) + cost(S \ A) + flops(A, S \ A), an
// index kept when carried outside S or by the output, ties to the smallest
// A as a bit mask; the tree is emitted in post order (A's subtree first,
// operands as (min id, max id)) and sliced by finish_plan.  PLAN_TOO_MANY
// when m > kExactMax or the network has more than 128 indices or a cost
// above 2^126.
constexpr int kExactMax = 16;
int make_plan_exact(const std::vector<Inds>& leaves, const DimMap& dims, const Inds& output, uint64_t max_bytes,
                    uint64_t n_slices, int64_t slice_dim, Plan* plan);

std::string plan_text(const Plan& plan);

}  // namespace qtpu
