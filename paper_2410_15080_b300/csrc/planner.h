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
};

// index id -> dim lookup
struct DimMap {
  std::vector<std::pair<int64_t, int64_t>> kv;  // sorted by id
  int64_t get(int64_t id) const;
  bool has(int64_t id) const;
  void set(int64_t id, int64_t d);
  std::vector<int64_t> ids() const;
};

enum PlanErr { PLAN_OK = 0, PLAN_OVERFLOW = 1, PLAN_LIMIT = 2 };

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

std::string plan_text(const Plan& plan);

}  // namespace qtpu
