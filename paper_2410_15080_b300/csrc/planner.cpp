// Greedy pairwise contraction order and slicing (host side).
//
// Rules (section 4.2 makes the cost order-dependent; the rules below fix one
// deterministic order so that plans are reproducible bit for bit):
//  * candidates: live pairs (x < y) sharing an index; all live pairs if no
//    pair shares one (disconnected pieces become outer products);
//  * an index of x or y is KEPT if the output or another live tensor carries
//    it.  kept & in both -> batch; kept & only x -> M; kept & only y -> N;
//    not kept & in both -> K (summed by the GEMM); not kept & on one side
//    only -> summed out of that operand first (sa / sb);
//  * key(x, y) = (size(out) - size(x) - size(y), flops, x, y), minimised,
//    flops = 2 * batch * M * N * K (+ size(x) if sa, + size(y) if sb);
//  * the result's axes are [batch, M, N], groups ordered as in x (batch, M)
//    and y (N), and it takes the next id;
//  * randomised variant (seed != 0): the pair is drawn uniformly among the
//    kRandTop smallest keys, with SplitMix64 (Steele, Lea and Flood 2014;
//    the constants of Vigna's reference version) advanced once per step;
//  * slicing keeps the tree fixed and repeatedly slices the non-output index
//    (of dim slice_dim if nonzero) minimising (peak entries per slice, total
//    flops over all slices, index id) until 8 * peak <= max_bytes and the
//    slice count reaches n_slices.
#include "planner.h"

#include <algorithm>
#include <functional>
#include <map>
#include <set>
#include <sstream>

namespace qtpu {

int64_t DimMap::get(int64_t id) const {
  auto it = std::lower_bound(kv.begin(), kv.end(), std::make_pair(id, (int64_t)INT64_MIN));
  return (it != kv.end() && it->first == id) ? it->second : -1;
}
bool DimMap::has(int64_t id) const { return get(id) >= 0; }
void DimMap::set(int64_t id, int64_t d) {
  auto it = std::lower_bound(kv.begin(), kv.end(), std::make_pair(id, (int64_t)INT64_MIN));
  if (it != kv.end() && it->first == id)
    it->second = d;
  else
    kv.insert(it, {id, d});
}
std::vector<int64_t> DimMap::ids() const {
  std::vector<int64_t> r;
  for (auto& p : kv) r.push_back(p.first);
  return r;
}

namespace {

struct Ctx {
  const DimMap* dims;
  const std::set<int64_t>* sliced = nullptr;
  bool ovf = false;
  U256 prod(const Inds& v) {
    U256 r(1);
    for (int64_t i : v) {
      int64_t d = (sliced && sliced->count(i)) ? 1 : dims->get(i);
      r = U256::mul_u64(r, (uint64_t)d, &ovf);
    }
    return r;
  }
  U256 prod2(const Inds& a, const Inds& b, const Inds& c, const Inds& d) {
    U256 r = prod(a);
    r = U256::mul(r, prod(b), &ovf);
    r = U256::mul(r, prod(c), &ovf);
    r = U256::mul(r, prod(d), &ovf);
    return r;
  }
  U256 flops(const Inds& ia, const Inds& ib, const PlanStep& s) {
    U256 f = U256::mul_u64(prod2(s.batch, s.m, s.n, s.k), 2, &ovf);
    if (!s.sa.empty()) f = U256::add(f, prod(ia), &ovf);
    if (!s.sb.empty()) f = U256::add(f, prod(ib), &ovf);
    return f;
  }
};

bool contains(const Inds& v, int64_t x) { return std::find(v.begin(), v.end(), x) != v.end(); }

void classify(const Inds& ia, const Inds& ib, const std::set<int64_t>& keep, PlanStep* s) {
  s->batch.clear(); s->m.clear(); s->n.clear(); s->k.clear(); s->sa.clear(); s->sb.clear();
  for (int64_t i : ia) {
    bool inb = contains(ib, i), kp = keep.count(i) > 0;
    if (inb && kp) s->batch.push_back(i);
    else if (inb) s->k.push_back(i);
    else if (kp) s->m.push_back(i);
    else s->sa.push_back(i);
  }
  for (int64_t i : ib) {
    if (contains(ia, i)) continue;
    if (keep.count(i)) s->n.push_back(i);
    else s->sb.push_back(i);
  }
}

// exact compare of (o1 - a1 - b1) < (o2 - a2 - b2) as o1 + a2 + b2 < o2 + a1 + b1
struct Wide { U256 v; int carry = 0; };
Wide add3(const U256& a, const U256& b, const U256& c) {
  Wide r;
  unsigned __int128 cy = 0;
  for (int i = 0; i < 4; ++i) {
    cy += (unsigned __int128)a.w[i] + b.w[i] + c.w[i];
    r.v.w[i] = (uint64_t)cy;
    cy >>= 64;
  }
  r.carry = (int)cy;
  return r;
}
bool wide_less(const Wide& a, const Wide& b) {
  if (a.carry != b.carry) return a.carry < b.carry;
  return a.v < b.v;
}

struct Key {
  U256 out, sa, sb, flops;
  int x, y;
};
bool key_less(const Key& p, const Key& q) {
  Wide l = add3(p.out, q.sa, q.sb), r = add3(q.out, p.sa, p.sb);
  if (wide_less(l, r)) return true;
  if (wide_less(r, l)) return false;
  if (p.flops != q.flops) return p.flops < q.flops;
  if (p.x != q.x) return p.x < q.x;
  return p.y < q.y;
}

void stats(const Plan& p, Ctx& c, U256* peak, U256* fl) {
  *peak = U256(0);
  *fl = U256(0);
  for (auto& st : p.steps) {
    U256 sz = c.prod(st.out_inds());
    if (*peak < sz) *peak = sz;
    *fl = U256::add(*fl, c.flops(p.tensor_inds[st.x], p.tensor_inds[st.y], st), &c.ovf);
  }
}

}  // namespace

namespace {
uint64_t splitmix64(uint64_t* state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
}  // namespace

int make_plan(const std::vector<Inds>& leaves, const DimMap& dims, const Inds& output,
              uint64_t max_bytes, uint64_t n_slices, int64_t slice_dim, Plan* plan, uint64_t seed) {
  uint64_t rng = seed;
  Ctx c{&dims};
  Plan& p = *plan;
  p = Plan();
  p.n_leaves = (int)leaves.size();
  p.output = output;
  p.tensor_inds = leaves;
  std::map<int, Inds> live;
  std::map<int64_t, int> count;
  for (int t = 0; t < (int)leaves.size(); ++t) {
    live[t] = leaves[t];
    std::set<int64_t> u(leaves[t].begin(), leaves[t].end());
    for (int64_t i : u) count[i]++;
  }
  for (int64_t i : output) count[i]++;
  int nxt = (int)leaves.size();
  while (live.size() > 1) {
    std::vector<int> ids;
    for (auto& kv : live) ids.push_back(kv.first);
    std::vector<std::pair<int, int>> pairs;
    for (size_t a = 0; a < ids.size(); ++a)
      for (size_t b = a + 1; b < ids.size(); ++b) {
        const Inds& ia = live[ids[a]];
        const Inds& ib = live[ids[b]];
        bool share = false;
        for (int64_t i : ia) if (contains(ib, i)) { share = true; break; }
        if (share) pairs.push_back({ids[a], ids[b]});
      }
    if (pairs.empty())
      for (size_t a = 0; a < ids.size(); ++a)
        for (size_t b = a + 1; b < ids.size(); ++b) pairs.push_back({ids[a], ids[b]});
    bool have = false;
    Key best{};
    PlanStep best_step;
    std::vector<std::pair<Key, PlanStep>> top;  // randomised: the kRandTop best
    for (auto& pr : pairs) {
      const Inds& ia = live[pr.first];
      const Inds& ib = live[pr.second];
      std::set<int64_t> keep;
      for (int64_t i : ia) if (count[i] - 1 - (contains(ib, i) ? 1 : 0) > 0) keep.insert(i);
      for (int64_t i : ib) if (count[i] - 1 - (contains(ia, i) ? 1 : 0) > 0) keep.insert(i);
      PlanStep st;
      st.x = pr.first; st.y = pr.second; st.out = nxt;
      classify(ia, ib, keep, &st);
      Key k;
      k.out = c.prod(st.out_inds());
      k.sa = c.prod(ia);
      k.sb = c.prod(ib);
      k.flops = c.flops(ia, ib, st);
      k.x = pr.first; k.y = pr.second;
      if (c.ovf) return PLAN_OVERFLOW;
      if (!have || key_less(k, best)) { best = k; best_step = st; have = true; }
      if (seed) {
        top.push_back({k, st});
        std::sort(top.begin(), top.end(), [](const std::pair<Key, PlanStep>& a, const std::pair<Key, PlanStep>& b) {
          return key_less(a.first, b.first);
        });
        if ((int)top.size() > kRandTop) top.pop_back();
      }
    }
    if (seed) best_step = top[splitmix64(&rng) % top.size()].second;
    for (int64_t i : std::set<int64_t>(live[best_step.x].begin(), live[best_step.x].end())) count[i]--;
    for (int64_t i : std::set<int64_t>(live[best_step.y].begin(), live[best_step.y].end())) count[i]--;
    live.erase(best_step.x);
    live.erase(best_step.y);
    Inds ni = best_step.out_inds();
    live[nxt] = ni;
    for (int64_t i : std::set<int64_t>(ni.begin(), ni.end())) count[i]++;
    p.steps.push_back(best_step);
    p.tensor_inds.push_back(ni);
    nxt++;
  }
  p.final_inds = live.begin()->second;
  for (int64_t i : p.final_inds)
    if (!contains(output, i)) p.final_sum.push_back(i);
  return finish_plan(dims, output, max_bytes, n_slices, slice_dim, &p);
}

// Slicing on the fixed tree, then the per-slice accounting.
int finish_plan(const DimMap& dims, const Inds& output, uint64_t max_bytes, uint64_t n_slices, int64_t slice_dim,
                Plan* plan) {
  Plan& p = *plan;
  Ctx c{&dims};
  std::set<int64_t> sl;
  U256 nsl(1);
  std::vector<int64_t> all_ix = dims.ids();
  for (;;) {
    c.sliced = &sl;
    U256 peak, fl;
    stats(p, c, &peak, &fl);
    if (c.ovf) return PLAN_OVERFLOW;
    bool ok_bytes = true;
    if (max_bytes) {
      bool o2 = false;
      U256 pb = U256::mul_u64(peak, 8, &o2);
      ok_bytes = !o2 && !(U256(max_bytes) < pb);
    }
    if (ok_bytes && !(nsl < U256(n_slices))) break;
    bool have = false;
    U256 bp, bf;
    int64_t bi = -1;
    for (int64_t i : all_ix) {
      if (contains(output, i) || sl.count(i)) continue;
      if (slice_dim != 0 && dims.get(i) != slice_dim) continue;
      std::set<int64_t> s2 = sl;
      s2.insert(i);
      c.sliced = &s2;
      U256 pk, f;
      stats(p, c, &pk, &f);
      U256 tot = U256::mul(U256::mul_u64(nsl, (uint64_t)dims.get(i), &c.ovf), f, &c.ovf);
      if (c.ovf) return PLAN_OVERFLOW;
      bool better = !have || pk < bp || (pk == bp && (tot < bf || (tot == bf && i < bi)));
      if (better) { have = true; bp = pk; bf = tot; bi = i; }
    }
    c.sliced = &sl;
    if (!have) return PLAN_LIMIT;
    sl.insert(bi);
    p.sliced.push_back(bi);
    nsl = U256::mul_u64(nsl, (uint64_t)dims.get(bi), &c.ovf);
    if (c.ovf) return PLAN_OVERFLOW;
  }
  p.n_slices = nsl;
  c.sliced = &sl;
  p.step_size.clear();
  p.step_flops.clear();
  p.flops_per_slice = U256(0);
  p.peak = U256(0);
  for (auto& st : p.steps) {
    U256 sz = c.prod(st.out_inds());
    U256 f = c.flops(p.tensor_inds[st.x], p.tensor_inds[st.y], st);
    p.step_size.push_back(sz);
    p.step_flops.push_back(f);
    p.flops_per_slice = U256::add(p.flops_per_slice, f, &c.ovf);
    if (p.peak < sz) p.peak = sz;
  }
  p.flops_total = U256::mul(p.flops_per_slice, p.n_slices, &c.ovf);
  if (c.ovf) return PLAN_OVERFLOW;
  return PLAN_OK;
}

int make_plan_best(const std::vector<Inds>& leaves, const DimMap& dims, const Inds& output, uint64_t max_bytes,
                   uint64_t n_slices, int64_t slice_dim, uint64_t seed, uint32_t n, Plan* plan, uint64_t* chosen) {
  int last_err = PLAN_LIMIT;
  bool have = false;
  Plan cand;
  for (uint32_t i = 0; i < n; ++i) {
    const uint64_t s = seed + i;
    const int r = make_plan(leaves, dims, output, max_bytes, n_slices, slice_dim, &cand, s);
    if (r != PLAN_OK) {
      last_err = r;
      continue;
    }
    if (!have || cand.flops_total < plan->flops_total) {
      *plan = cand;
      *chosen = s;
      have = true;
    }
  }
  if (!have) return last_err;
  plan->search = n;
  plan->search_seed = *chosen;
  return PLAN_OK;
}

static std::string lst(const Inds& v) {
  if (v.empty()) return "-";
  std::ostringstream o;
  for (size_t i = 0; i < v.size(); ++i) {
    if (i) o << ",";
    o << v[i];
  }
  return o.str();
}

std::string plan_text(const Plan& p) {
  std::ostringstream o;
  o << "qtpu-plan 1 leaves=" << p.n_leaves << " output=" << lst(p.output) << "\n";
  for (size_t s = 0; s < p.steps.size(); ++s) {
    const PlanStep& st = p.steps[s];
    o << "step " << s << " " << st.x << " " << st.y << " -> " << st.out << " batch=" << lst(st.batch)
      << " m=" << lst(st.m) << " n=" << lst(st.n) << " k=" << lst(st.k) << " sa=" << lst(st.sa)
      << " sb=" << lst(st.sb) << " size=" << p.step_size[s].str() << " flops=" << p.step_flops[s].str()
      << "\n";
  }
  o << "final inds=" << lst(p.final_inds) << " sum=" << lst(p.final_sum) << "\n";
  o << "slices n=" << p.n_slices.str() << " idx=" << lst(p.sliced) << "\n";
  o << "cost flops_per_slice=" << p.flops_per_slice.str() << " flops_total=" << p.flops_total.str()
    << " peak=" << p.peak.str() << "\n";
  if (p.search) o << "search candidates=" << p.search << " seed=" << p.search_seed << "\n";
  if (p.search_exact >= 0) o << "search exact tensors=" << p.search_exact << "\n";
  if (!p.search_note.empty()) o << p.search_note << "\n";
  return o.str();
}

// ------------------------------------------------------------ exact search
namespace {
using u128 = unsigned __int128;
constexpr u128 kCostCap = (u128)1 << 126;

struct Bits {
  uint64_t w[2] = {0, 0};
  void set(int i) { w[i >> 6] |= 1ull << (i & 63); }
  bool any() const { return w[0] | w[1]; }
  Bits operator|(const Bits& o) const { Bits r; r.w[0] = w[0] | o.w[0]; r.w[1] = w[1] | o.w[1]; return r; }
  Bits operator&(const Bits& o) const { Bits r; r.w[0] = w[0] & o.w[0]; r.w[1] = w[1] & o.w[1]; return r; }
  Bits operator~() const { Bits r; r.w[0] = ~w[0]; r.w[1] = ~w[1]; return r; }
};

// product of the dims of the set bits; false when it reaches the cap
bool prod_bits(const Bits& b, const std::vector<int64_t>& dim, u128* out) {
  u128 r = 1;
  for (int q = 0; q < 2; ++q) {
    uint64_t x = b.w[q];
    while (x) {
      const int i = q * 64 + __builtin_ctzll(x);
      x &= x - 1;
      r *= (u128)dim[i];
      if (r >= kCostCap) return false;
    }
  }
  *out = r;
  return true;
}

// one pairwise step with the planner's keep rule (count-based)
void apply_step(std::map<int, Inds>& live, std::map<int64_t, int>& count, int x, int y, int nxt, Plan* p) {
  const Inds& ia = live[x];
  const Inds& ib = live[y];
  std::set<int64_t> keep;
  for (int64_t i : ia) if (count[i] - 1 - (contains(ib, i) ? 1 : 0) > 0) keep.insert(i);
  for (int64_t i : ib) if (count[i] - 1 - (contains(ia, i) ? 1 : 0) > 0) keep.insert(i);
  PlanStep st;
  st.x = x; st.y = y; st.out = nxt;
  classify(ia, ib, keep, &st);
  for (int64_t i : std::set<int64_t>(ia.begin(), ia.end())) count[i]--;
  for (int64_t i : std::set<int64_t>(ib.begin(), ib.end())) count[i]--;
  live.erase(x);
  live.erase(y);
  Inds ni = st.out_inds();
  live[nxt] = ni;
  for (int64_t i : std::set<int64_t>(ni.begin(), ni.end())) count[i]++;
  p->steps.push_back(st);
  p->tensor_inds.push_back(ni);
}
}  // namespace

int make_plan_exact(const std::vector<Inds>& leaves, const DimMap& dims, const Inds& output, uint64_t max_bytes,
                    uint64_t n_slices, int64_t slice_dim, Plan* plan) {
  Plan& p = *plan;
  p = Plan();
  p.n_leaves = (int)leaves.size();
  p.output = output;
  p.tensor_inds = leaves;
  const int n = (int)leaves.size();
  std::map<int, Inds> live;
  std::map<int64_t, int> count;
  for (int t = 0; t < n; ++t) {
    live[t] = leaves[t];
    for (int64_t i : std::set<int64_t>(leaves[t].begin(), leaves[t].end())) count[i]++;
  }
  for (int64_t i : output) count[i]++;
  // 1. absorption of the small leaves
  std::vector<int> small, large;
  for (int t = 0; t < n; ++t) {
    double sz = 1;
    for (int64_t i : leaves[t]) sz *= (double)dims.get(i);
    (sz <= 256.0 ? small : large).push_back(t);
  }
  std::map<int, int> cur;
  for (int t : large) cur[t] = t;
  int nxt = n;
  for (int t : small) {
    int h = -1;
    for (int q : large) {
      bool share = false;
      for (int64_t i : leaves[t]) if (contains(leaves[q], i)) { share = true; break; }
      if (share) { h = q; break; }  // large is ascending: the lowest id
    }
    if (h < 0) continue;
    const int x = std::min(cur[h], t), y = std::max(cur[h], t);
    apply_step(live, count, x, y, nxt, &p);
    cur[h] = nxt++;
  }
  // 2. exact tree over the live tensors
  std::vector<int> ids;
  for (auto& kv : live) ids.push_back(kv.first);
  const int m = (int)ids.size();
  if (m > kExactMax) return PLAN_TOO_MANY;
  std::vector<int64_t> all = dims.ids();
  if (all.size() > 128) return PLAN_TOO_MANY;
  std::map<int64_t, int> pos;
  std::vector<int64_t> dim(all.size());
  for (size_t q = 0; q < all.size(); ++q) pos[all[q]] = (int)q, dim[q] = dims.get(all[q]);
  Bits outb;
  for (int64_t i : output) outb.set(pos[i]);
  std::vector<Bits> carried(m);
  for (int j = 0; j < m; ++j)
    for (int64_t i : live[ids[j]]) carried[j].set(pos[i]);
  const uint32_t full = m ? (1u << m) - 1 : 0;
  std::vector<Bits> uni(full + 1), tup(full + 1);
  std::vector<u128> size(full + 1, 0), cost(full + 1, 0);
  std::vector<uint32_t> split(full + 1, 0);
  for (uint32_t s = 1; s <= full; ++s) uni[s] = uni[s & (s - 1)] | carried[__builtin_ctz(s)];
  auto kept = [&](uint32_t s) { return uni[s] & (uni[full ^ s] | outb); };
  for (uint32_t s = 1; s <= full; ++s) {
    tup[s] = (s & (s - 1)) ? kept(s) : carried[__builtin_ctz(s)];
    if (!prod_bits(tup[s], dim, &size[s])) return PLAN_TOO_MANY;
  }
  for (uint32_t s = 1; s <= full; ++s) {
    if (!(s & (s - 1))) continue;
    const uint32_t low = s & (~s + 1), rest = s ^ low;
    const Bits keep = kept(s);
    bool have = false;
    u128 best = 0;
    uint32_t besta = 0;
    for (uint32_t sub = rest;; sub = (sub - 1) & rest) {
      const uint32_t a = low | sub;
      if (a != s) {
        const uint32_t b = s ^ a;
        const Bits& ia = tup[a];
        const Bits& ib = tup[b];
        const Bits sa = ia & ~ib & ~keep, sb = ib & ~ia & ~keep;
        u128 core;
        if (!prod_bits((ia | ib) & ~(sa | sb), dim, &core)) return PLAN_TOO_MANY;
        u128 f = 2 * core + (sa.any() ? size[a] : 0) + (sb.any() ? size[b] : 0);
        const u128 c = cost[a] + cost[b] + f;
        if (c >= kCostCap) return PLAN_TOO_MANY;
        if (!have || c < best || (c == best && a < besta)) best = c, besta = a, have = true;
      }
      if (sub == 0) break;
    }
    cost[s] = best;
    split[s] = besta;
  }
  // 3. the tree in post order
  std::function<int(uint32_t)> build = [&](uint32_t s) -> int {
    if (!(s & (s - 1))) return ids[__builtin_ctz(s)];
    const uint32_t a = split[s];
    const int xa = build(a);
    const int xb = build(s ^ a);
    apply_step(live, count, std::min(xa, xb), std::max(xa, xb), nxt, &p);
    return nxt++;
  };
  if (m > 1) build(full);
  p.final_inds = live.begin()->second;
  for (int64_t i : p.final_inds)
    if (!contains(output, i)) p.final_sum.push_back(i);
  p.search_exact = m;
  return finish_plan(dims, output, max_bytes, n_slices, slice_dim, &p);
}

}  // namespace qtpu
