// Contraction-order hyper-search (section 6.1 step 3: the order is computed
// before the contraction by a search over candidate trees).
//
// Candidates: the exact subset-DP tree (make_plan_exact, when the network
// has at most kExactMax tensors after absorption) and n randomised greedy
// orders.  Each candidate is sliced like any plan and lowered without device
// memory; the one whose lowered launch list executes the fewest FLOPs under
// slice reuse wins (ties: fewer plan FLOPs, then candidate order, the exact
// tree first).  Candidates are planned and lowered on the host cores in
// parallel, so the search runs while the caller does other work on the
// device (such as producing the QTs).
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <thread>

#include "exec.h"

namespace qtpu {

int plan_hyper(const std::vector<Inds>& li, const DimMap& dims, const Inds& output, const qtpu_plan_opts& o,
               const std::vector<Leaf>& leaves, const TileTable* tiles, Plan* chosen, std::string* err) {
  const uint32_t ng = o.n_candidates > 1 ? o.n_candidates : 64;
  const int nc = (int)ng + 1;  // candidate 0: the exact tree
  struct Cand {
    Plan plan;
    int status = PLAN_LIMIT;
    bool lowered = false;
    double executed = 0;
  };
  std::vector<Cand> cands(nc);
  std::atomic<int> next{0};
  auto work = [&]() {
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= nc) return;
      Cand& c = cands[k];
      c.status = k == 0 ? make_plan_exact(li, dims, output, o.max_intermediate_bytes, o.n_slices, o.slice_dim,
                                          &c.plan)
                        : make_plan(li, dims, output, o.max_intermediate_bytes, o.n_slices, o.slice_dim, &c.plan,
                                    o.seed + (uint64_t)(k - 1));
      if (c.status != PLAN_OK) continue;
      Executor ex;
      int code = QTPU_OK;
      exec_build(&ex, c.plan, leaves, dims, (int)o.prec, &code, true, o.reuse_bytes, tiles);
      if (code != QTPU_OK || !ex.lowered) continue;
      c.lowered = true;
      c.executed = ex.flops_executed;
    }
  };
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  const int nt = std::min(nc, std::min(hw, 32));
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(work);
  work();
  for (auto& t : pool) t.join();
  int best = -1;
  for (int k = 0; k < nc; ++k) {
    const Cand& c = cands[k];
    if (c.status == PLAN_OVERFLOW) {
      *err = "a contraction size reaches 2^255";
      return QTPU_ENOTSUP;
    }
    if (!c.lowered) continue;
    if (best < 0 || c.executed < cands[best].executed ||
        (c.executed == cands[best].executed && c.plan.flops_total < cands[best].plan.flops_total))
      best = k;
  }
  if (best < 0) {
    *err = "the peak-intermediate limit cannot be met by slicing";
    return QTPU_ELIMIT;
  }
  *chosen = cands[best].plan;
  chosen->search = 0;
  chosen->search_exact = -1;
  char fl[64];
  std::snprintf(fl, sizeof fl, "%.0f", cands[best].executed);
  chosen->search_note = "search hyper candidates=" + std::to_string(nc) + " chosen=" +
                        (best == 0 ? std::string("exact") : "seed:" + std::to_string(o.seed + best - 1)) +
                        " executed_flops=" + fl;
  return QTPU_OK;
}

}  // namespace qtpu
