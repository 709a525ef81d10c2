// Executor: lowers a contraction plan to a flat list of kernel launches.
//
// Section 6.1 step 4 contracts the evaluated classical TN on the available
// accelerator.  With a tensor-core precision each planned pairwise step
// becomes one of:
//   * absorbed: a step that contracts a tensor with a small leaf (a QPD
//     coefficient tensor, section 4.1; or any leaf of <= 256 entries) is not
//     run on its own; the result stays a "virtual" tensor (base operands +
//     small factors + internal summed indices) and the step that consumes it
//     gathers the product on the fly (the h-TN simplification of section 4.3
//     fuses the CTs between two QTs; here they are fused into the QT read);
//   * tensor-core step (large dense GEMM): two gather-split launches lay the
//     operands out as [batch][rows][K] piece planes, then the tcgen05 GEMM
//     writes the result [batch][M][N] as (hi, lo) float pairs;
//   * gather step: everything else (dot products, skinny or small steps),
//     one multi-operand gather kernel with compensated FP32 arithmetic.
// With QTPU_PREC_FP64 every step is an FP64 CUDA-core contraction and
// intermediates are FP64.  Intermediates live in one device arena laid out at
// build time (first-fit over the steps' lifetimes).  Slices (fixed values of
// the sliced indices) run one after another through the same launches with
// shifted leaf pointers; each slice's final tensor lands in partial[slice],
// and one reduction sums the slices (and any leftover indices) in a fixed
// order into the FP64 output.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <sstream>
#include <unordered_map>

#include "exec.h"
#include "../../include/qtpu_htn.h"

namespace qtpu {

namespace {

struct Err {
  std::string msg;
  int code = QTPU_OK;
};

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

bool contains(const Inds& v, int64_t x) { return std::find(v.begin(), v.end(), x) != v.end(); }

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// first-fit arena over byte ranges
struct Arena {
  std::map<size_t, size_t> free_;  // offset -> size
  size_t top = 0;
  size_t alloc(size_t n) {
    n = align_up(n, 256);
    for (auto it = free_.begin(); it != free_.end(); ++it)
      if (it->second >= n) {
        size_t off = it->first, rem = it->second - n;
        free_.erase(it);
        if (rem) free_[off + n] = rem;
        return off;
      }
    size_t off = top;
    top += n;
    return off;
  }
  void release(size_t off, size_t n) {
    n = align_up(n, 256);
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

// Append a mode, dropping dim-1 modes.
bool push_mode(ModeTab& t, int64_t d, int64_t sa, int64_t sb) {
  if (d == 1) return true;
  if (t.n >= kMaxModes) return false;
  t.dim[t.n] = d;
  t.sa[t.n] = sa;
  t.sb[t.n] = sb;
  t.n++;
  return true;
}

// Merge adjacent modes j, j+1 that are contiguous in both operands.
void merge_modes(ModeTab& t) {
  int w = 0;
  for (int j = 0; j < t.n; ++j) {
    if (w > 0 && t.sa[w - 1] == t.sa[j] * t.dim[j] && t.sb[w - 1] == t.sb[j] * t.dim[j]) {
      t.dim[w - 1] *= t.dim[j];
      t.sa[w - 1] = t.sa[j];
      t.sb[w - 1] = t.sb[j];
    } else {
      t.dim[w] = t.dim[j];
      t.sa[w] = t.sa[j];
      t.sb[w] = t.sb[j];
      ++w;
    }
  }
  t.n = w;
}

// largest element offset a mode table reaches in operand a (which = 0) or b
int64_t max_off(const ModeTab& t, int which) {
  int64_t m = 0;
  for (int j = 0; j < t.n; ++j) m += (t.dim[j] - 1) * (which == 0 ? t.sa[j] : t.sb[j]);
  return m;
}

int64_t tab_size(const ModeTab& t) {
  int64_t s = 1;
  for (int j = 0; j < t.n; ++j) s *= t.dim[j];
  return s;
}

}  // namespace

bool make_operand_map(CUtensorMap* map, void* base, int prec, int64_t batch, int64_t rows, int64_t K, int64_t Kp,
                      int box_rows) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  const int np = prec == 3 ? 3 : (prec == 2 ? 2 : 1);
  const int es = prec == 3 ? 2 : 4;
  const int kb = gemm_k_block(prec);
  cuuint64_t gdim[4] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)batch, (cuuint64_t)np};
  cuuint64_t gstr[3] = {(cuuint64_t)(Kp * es), (cuuint64_t)(rows * Kp * es), (cuuint64_t)(batch * rows * Kp * es)};
  cuuint32_t box[4] = {(cuuint32_t)kb, (cuuint32_t)box_rows, 1, 1};
  cuuint32_t est[4] = {1, 1, 1, 1};
  // the swizzle span is the stage's row: kb elements
  const CUtensorMapSwizzle swz = kb * es == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
  CUresult r = enc(map, prec == 3 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base,
                   gdim, gstr, box, est, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

namespace {

constexpr int64_t kSmallLeaf = 256;   // leaves up to this size are absorbed
constexpr int kMaxVirtualOps = 5;     // operands of one virtual tensor
constexpr int64_t kMaxVirtualLoop = 256;
// QTPU_GEMM_PAIR=0/1 sets the CTA-pair form of every BF16x3 GEMM whose tile
// the lowering chooses (unset: the tile table's choice)
int gemm_pair_override() {
  static const int v = [] {
    const char* e = std::getenv("QTPU_GEMM_PAIR");
    return e ? (std::atoi(e) != 0 ? 1 : 0) : -1;
  }();
  return v;
}
// rows of B one TMA box loads: a CTA of a pair stages half of the N tile
int gemm_b_box(const GemmArgs& g) { return g.pair ? g.bn / 2 : g.bn; }
constexpr size_t kKeptSplitBudget = (size_t)8 << 30;  // device bytes for kept split results

size_t dt_bytes(int dt) { return dt == DT_F32 ? 4 : 8; }

// Add a mode to a gather table (dim-1 modes dropped), strides per operand.
bool gpush(GModes& t, int64_t d, const int64_t* st, int nops) {
  if (d == 1) return true;
  if (t.n >= kMaxModes || d > 0xFFFFFFFFll) return false;
  t.dim[t.n] = (uint32_t)d;
  for (int j = 0; j < kMaxOps; ++j) t.stride[t.n][j] = j < nops ? st[j] : 0;
  t.n++;
  return true;
}

void gmerge(GModes& t, int nops) {
  int w = 0;
  for (int m = 0; m < t.n; ++m) {
    bool can = w > 0;
    for (int j = 0; j < nops && can; ++j) can = t.stride[w - 1][j] == t.stride[m][j] * (int64_t)t.dim[m];
    if (can && (uint64_t)t.dim[w - 1] * t.dim[m] <= 0xFFFFFFFFull) {
      t.dim[w - 1] *= t.dim[m];
      for (int j = 0; j < kMaxOps; ++j) t.stride[w - 1][j] = t.stride[m][j];
    } else {
      t.dim[w] = t.dim[m];
      for (int j = 0; j < kMaxOps; ++j) t.stride[w][j] = t.stride[m][j];
      ++w;
    }
  }
  t.n = w;
  for (int m = 0; m < t.n; ++m) t.div[m] = make_fastdiv(t.dim[m]);
}

uint64_t gsize(const GModes& t) {
  uint64_t s = 1;
  for (int m = 0; m < t.n; ++m) s *= t.dim[m];
  return s;
}

int64_t gmax(const GModes& t, int j) {
  int64_t m = 0;
  for (int k = 0; k < t.n; ++k) m += (int64_t)(t.dim[k] - 1) * t.stride[k][j];
  return m;
}

// Dot layout of a fast two-operand gather with a long loop (see GatherArgs):
// the tile takes, for each operand, its loop modes in rising stride order
// while they stay contiguous and until its run reaches 32 entries; a
// unit-stride mode too long for the tile is split at a divisor first.
bool dot_setup(GatherArgs& g, int sm) {
  GModes L = g.loop;
  for (int j = 0; j < 2; ++j)
    for (int m = 0; m < L.n; ++m) {
      if (L.stride[m][j] != 1 || L.dim[m] <= 256 || L.n >= kMaxModes) continue;
      uint32_t d2 = 0;
      for (uint32_t d = 256; d >= 16 && !d2; --d)
        if (L.dim[m] % d == 0) d2 = d;
      if (!d2) continue;
      for (int k = L.n; k > m + 1; --k) {
        L.dim[k] = L.dim[k - 1];
        for (int q = 0; q < kMaxOps; ++q) L.stride[k][q] = L.stride[k - 1][q];
      }
      L.n++;
      L.dim[m + 1] = d2;
      for (int q = 0; q < kMaxOps; ++q) L.stride[m + 1][q] = L.stride[m][q];
      L.dim[m] /= d2;
      for (int q = 0; q < kMaxOps; ++q) L.stride[m][q] *= d2;
    }
  std::vector<int> in_tile(L.n, 0);
  uint64_t T = 1;
  for (int j = 0; j < 2; ++j) {
    std::vector<int> ord;
    for (int m = 0; m < L.n; ++m)
      if (L.stride[m][j] > 0) ord.push_back(m);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return L.stride[a][j] < L.stride[b][j]; });
    int64_t run = 1;
    for (int m : ord) {
      if (L.stride[m][j] != run || run >= 32) break;
      if (!in_tile[m]) {
        if (T * L.dim[m] > kDotMaxTile) break;
        T *= L.dim[m];
        in_tile[m] = 1;
      }
      run *= L.dim[m];
    }
  }
  // widen the tile (fewer block barriers per entry): the remaining modes in
  // rising operand-1 stride order while the tile stays within bounds
  {
    std::vector<int> ord;
    for (int m = 0; m < L.n; ++m)
      if (!in_tile[m]) ord.push_back(m);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return L.stride[a][1] < L.stride[b][1]; });
    for (int m : ord) {
      if (T >= 1024) break;
      if (T * L.dim[m] <= kDotMaxTile) {
        T *= L.dim[m];
        in_tile[m] = 1;
        continue;
      }
      // the largest divisor of the mode that still fits: split it, the inner
      // part joins the tile
      uint32_t d2 = 0;
      for (uint32_t d = (uint32_t)(kDotMaxTile / T); d >= 2 && !d2; --d)
        if (L.dim[m] % d == 0) d2 = d;
      if (!d2 || L.n >= kMaxModes) continue;
      for (int k = L.n; k > m + 1; --k) {
        L.dim[k] = L.dim[k - 1];
        for (int q = 0; q < kMaxOps; ++q) L.stride[k][q] = L.stride[k - 1][q];
      }
      in_tile.insert(in_tile.begin() + m + 1, 1);
      L.n++;
      L.dim[m + 1] = d2;
      for (int q = 0; q < kMaxOps; ++q) L.stride[m + 1][q] = L.stride[m][q];
      L.dim[m] /= d2;
      for (int q = 0; q < kMaxOps; ++q) L.stride[m][q] *= d2;
      T *= d2;
      break;
    }
  }
  if (T < 32) return false;
  std::vector<int> tile;
  for (int m = 0; m < L.n; ++m)
    if (in_tile[m]) tile.push_back(m);
  // slot order: operand 1's strides, outermost first
  std::vector<int> so = tile;
  std::stable_sort(so.begin(), so.end(), [&](int a, int b) { return L.stride[a][1] > L.stride[b][1]; });
  std::map<int, int64_t> slot;
  int64_t acc = 1;
  for (int k = (int)so.size() - 1; k >= 0; --k) {
    slot[so[k]] = acc;
    acc *= L.dim[so[k]];
  }
  GModes tx, ty, outer;
  for (int m : so) {
    ty.dim[ty.n] = L.dim[m];
    for (int q = 0; q < kMaxOps; ++q) ty.stride[ty.n][q] = q == 0 ? L.stride[m][1] : 0;
    ty.div[ty.n] = make_fastdiv(L.dim[m]);
    ty.n++;
  }
  std::vector<int> xo = tile;
  std::stable_sort(xo.begin(), xo.end(), [&](int a, int b) { return L.stride[a][0] > L.stride[b][0]; });
  for (int m : xo) {
    tx.dim[tx.n] = L.dim[m];
    for (int q = 0; q < kMaxOps; ++q) tx.stride[tx.n][q] = q == 0 ? L.stride[m][0] : (q == 1 ? slot[m] : 0);
    tx.div[tx.n] = make_fastdiv(L.dim[m]);
    tx.n++;
  }
  // outer tuples: the mode with the smallest strides runs fastest, so a
  // block's consecutive tuples read neighbouring runs of both operands while
  // their cache lines are still in L2
  std::vector<int> om;
  for (int m = 0; m < L.n; ++m)
    if (!in_tile[m]) om.push_back(m);
  std::stable_sort(om.begin(), om.end(), [&](int a, int b) {
    return L.stride[a][0] + L.stride[a][1] > L.stride[b][0] + L.stride[b][1];
  });
  for (int m : om) {
    outer.dim[outer.n] = L.dim[m];
    for (int q = 0; q < kMaxOps; ++q) outer.stride[outer.n][q] = L.stride[m][q];
    outer.n++;
  }
  gmerge(outer, 2);
  if (gmax(tx, 0) >= 0x7FFFFFFF || gmax(ty, 0) >= 0x7FFFFFFF || gsize(outer) > 0xFFFFFFFFull) return false;
  g.n_outer = (uint32_t)gsize(outer);
  g.loop = outer;
  g.kmodes = tx;
  g.wmodes = ty;
  g.tile_n = (uint32_t)T;
  uint32_t c = (uint32_t)((sm * 8 + g.n_out - 1) / g.n_out);
  g.chunks = std::max<uint32_t>(1, std::min<uint32_t>(c, g.n_outer));
  g.dot = 1;
  return true;
}

// a tensor during lowering: either stored (one operand: itself) or virtual
struct Repr {
  std::vector<int> ops;  // stored tensor ids whose product forms the tensor
  Inds L;                // indices summed inside a virtual tensor
  bool virt = false;
  double flops = 0;      // useful flops of absorbed steps not yet executed
};

}  // namespace

std::string exec_build(Executor* ex, const Plan& plan, const std::vector<Leaf>& leaves, const DimMap& dims,
                       int prec, int* code, bool dry_run, uint64_t reuse_bytes, const TileTable* tiles) {
  *code = QTPU_OK;
  ex->prec = prec;
  ex->n_leaves = plan.n_leaves;
  ex->launches.clear();
  ex->inter_off.clear();
  ex->n_tc_steps = ex->n_fused_steps = 0;
  if (const char* e = std::getenv("QTPU_KC")) ex->kc_blocks = std::atoi(e);
  const bool fp64 = prec == QTPU_PREC_FP64;
  ex->inter_dt = fp64 ? DT_F64 : DT_F32X2;
  std::set<int64_t> sliced(plan.sliced.begin(), plan.sliced.end());
  const int nl = plan.n_leaves;
  const int n_plan = (int)plan.tensor_inds.size();
  auto fail = [&](int c, const std::string& m) {
    *code = c;
    return m;
  };

  if (!plan.n_slices.fits_u64() || plan.n_slices.w[0] > ((uint64_t)1 << 40)) return fail(QTPU_ENOTSUP, "slice count too large");
  ex->n_slices = (int64_t)plan.n_slices.w[0];
  ex->slice_dims.clear();
  for (int64_t i : plan.sliced) ex->slice_dims.push_back(dims.get(i));
  ex->leaf_slice.assign(nl, {});
  for (int t = 0; t < nl; ++t)
    for (size_t p = 0; p < plan.sliced.size(); ++p)
      for (size_t a = 0; a < leaves[t].ids.size(); ++a)
        if (leaves[t].ids[a] == plan.sliced[p]) ex->leaf_slice[t].push_back({(int)p, leaves[t].strides[a]});

  // Slice reuse.  tout[t] is the set of sliced positions the value of tensor
  // t depends on: those carried by the leaves below it, minus those its steps
  // have already contracted (a sliced index is an index of the network like
  // any other; the step that contracts it sums its values one slice value
  // after another).  A launch loops over the values of the positions its
  // inputs depend on (din) and keeps one copy of its result per value of the
  // positions the result depends on (dout), adding up over the positions it
  // contracts; a position can instead be held fixed in an outer loop (a
  // block) to save memory.  Every distinct value of a result is then
  // computed once per block.
  const int nsp = (int)plan.sliced.size();
  if (nsp > 62) return fail(QTPU_ENOTSUP, "more than 62 sliced indices");
  bool reuse = ex->n_slices > 1;
  if (const char* e = std::getenv("QTPU_NO_REUSE")) reuse = reuse && std::atoi(e) == 0;
  if (reuse_bytes == 1) reuse = false;
  ex->reuse_budget = reuse_bytes ? reuse_bytes : ((uint64_t)64 << 30);
  std::map<int64_t, int> spos;  // sliced index id -> position
  for (int p = 0; p < nsp; ++p) spos[plan.sliced[p]] = p;
  auto smask = [&](const Inds& v) {
    uint64_t m = 0;
    for (int64_t i : v) {
      auto it = spos.find(i);
      if (it != spos.end()) m |= 1ull << it->second;
    }
    return m;
  };
  std::unordered_map<int, uint64_t> tout;
  for (int t = 0; t < nl; ++t)
    for (auto& ps : ex->leaf_slice[t]) tout[t] |= 1ull << ps.first;
  for (const PlanStep& ps : plan.steps)
    tout[ps.out] = (tout[ps.x] | tout[ps.y]) & ~(smask(ps.k) | smask(ps.sa) | smask(ps.sb));
  auto toutof = [&](int t) -> uint64_t {
    auto it = tout.find(t);
    return it == tout.end() ? 0 : it->second;
  };

  // per-slice layout of every stored tensor: leaves keep their strides, step
  // results are dense over their non-sliced indices in [batch, M, N] order
  std::unordered_map<int, std::map<int64_t, int64_t>> stride;
  std::unordered_map<int, Inds> live_inds;
  std::unordered_map<int, int64_t> extent, slice_max;
  auto nsl = [&](const Inds& v) {
    Inds r;
    for (int64_t i : v)
      if (!sliced.count(i)) r.push_back(i);
    return r;
  };
  auto prod = [&](const Inds& v) {
    double s = 1;
    for (int64_t i : v) s *= (double)dims.get(i);
    return s;
  };
  for (int t = 0; t < nl; ++t) {
    int64_t e = 1;
    for (size_t a = 0; a < leaves[t].ids.size(); ++a) {
      e += (leaves[t].dims[a] - 1) * leaves[t].strides[a];
      if (!sliced.count(leaves[t].ids[a])) {
        live_inds[t].push_back(leaves[t].ids[a]);
        stride[t][leaves[t].ids[a]] = leaves[t].strides[a];
      }
    }
    extent[t] = e;
    int64_t sm = 0;
    for (auto& ps : ex->leaf_slice[t]) sm += (ex->slice_dims[ps.first] - 1) * ps.second;
    slice_max[t] = sm;
  }
  auto set_dense = [&](int t, const Inds& inds) {
    live_inds[t] = inds;
    int64_t st = 1;
    for (int j = (int)inds.size() - 1; j >= 0; --j) {
      stride[t][inds[j]] = st;
      st *= dims.get(inds[j]);
    }
    extent[t] = st;
    slice_max[t] = 0;
  };
  auto sof = [&](int t, int64_t i) -> int64_t {
    auto it = stride[t].find(i);
    return it == stride[t].end() ? 0 : it->second;
  };
  auto dt_of = [&](int t) { return t < nl ? leaves[t].dt : ex->inter_dt; };
  auto bytes_of = [&](int t) { return prod(live_inds[t]) * (double)dt_bytes(dt_of(t)); };

  // intermediates' lifetimes in launch order (+1 placed, -1 released); the
  // arena is laid out after lowering, when the copies of each are known
  std::vector<std::pair<int, int>> events;
  std::set<int> placed;
  std::map<int, size_t> offs;
  auto place = [&](int t) {
    events.push_back({t, 1});
    placed.insert(t);
  };
  auto release = [&](int t) {
    if (t >= nl && placed.count(t)) {
      events.push_back({t, -1});
      placed.erase(t);
    }
  };
  // every operand view must stay inside its tensor's storage
  auto check = [&](const GatherArgs& g, const std::vector<int>& src) {
    for (int j = 0; j < g.nops; ++j) {
      const int64_t m = gmax(g.out, j) + gmax(g.loop, j) + gmax(g.kmodes, j) + slice_max[src[j]];
      if (m >= extent[src[j]]) return false;
    }
    return true;
  };

  std::vector<Repr> repr(n_plan);
  // GEMM results not yet consumed: producing launch, index groups of the
  // stored [batch][N][M] layout, and K (for the fused operand split)
  struct GemmOut {
    size_t li;
    Inds batch, inner, outer;
    int64_t K;
  };
  std::map<int, GemmOut> gemm_out;
  bool fuse_off = false, fuse_keep_layout = false;
  if (const char* e = std::getenv("QTPU_NO_FUSE")) fuse_off = std::atoi(e) != 0;
  // QTPU_FUSE_KEEP_LAYOUT=1: no operand swap in favour of the fused split
  // (exercises the epilogue form with K along the tile's rows)
  if (const char* e = std::getenv("QTPU_FUSE_KEEP_LAYOUT")) fuse_keep_layout = std::atoi(e) != 0;
  for (int t = 0; t < nl; ++t) repr[t].ops = {t};
  size_t split_need_a = 0, split_need_b = 0;
  const int np = prec == 3 ? 3 : (prec == 2 ? 2 : 1);
  const int es = prec == 3 ? 2 : 4;
  const int split_mode = prec == 3 ? GW_SPLIT_BF16X3 : (prec == 2 ? GW_SPLIT_TF32X2 : GW_SPLIT_TF32);
  int next_tmp = n_plan;  // ids of materialised virtual tensors
  bool fast_off = false;
  if (const char* e = std::getenv("QTPU_NO_FAST")) fast_off = std::atoi(e) != 0;

  // Typed fast-path arguments: large operands first, small leaves folded
  // into a table W (dense over their joint non-sliced indices).  `groups`
  // are the index lists of the out / k / loop tables.
  auto fast_args = [&](const std::vector<int>& src, const Inds& outg, const Inds& kg, const Inds& loopg,
                       GatherArgs g, Launch* L) -> bool {
    std::vector<int> big, small;
    for (int t : src) {
      const bool is_small = t < nl && prod(live_inds[t]) <= (double)kSmallLeaf;
      (is_small ? small : big).push_back(t);
    }
    if (big.empty() || big.size() > 2) return false;
    auto w_entries = [&](const std::vector<int>& sm) {
      Inds u;
      for (int t : sm)
        for (int64_t i : live_inds[t])
          if (!contains(u, i)) u.push_back(i);
      return prod(u);
    };
    // a W table too large for shared memory: read the small leaf whose
    // removal shrinks it most directly, as a second large operand
    if (big.size() == 1 && small.size() > 1 && w_entries(small) > (double)kMaxW) {
      size_t best = 0;
      double best_w = 0;
      for (size_t j = 0; j < small.size(); ++j) {
        std::vector<int> rest = small;
        rest.erase(rest.begin() + j);
        const double w = w_entries(rest);
        if (j == 0 || w < best_w) best = j, best_w = w;
      }
      if (best_w <= (double)kMaxW && (dt_of(small[best]) == DT_F64 || dt_of(small[best]) == DT_F32X2)) {
        big.push_back(small[best]);
        small.erase(small.begin() + best);
      }
    }
    for (int t : big)
      if (dt_of(t) != DT_F64 && dt_of(t) != DT_F32X2) return false;
    Inds U;
    for (int t : small)
      for (int64_t i : live_inds[t])
        if (!contains(U, i)) U.push_back(i);
    std::map<int64_t, int64_t> wst;
    int64_t wsz = 1;
    for (int j = (int)U.size() - 1; j >= 0; --j) {
      wst[U[j]] = wsz;
      wsz *= dims.get(U[j]);
    }
    if (small.empty()) wsz = 0;
    if (wsz > (int64_t)kMaxW) return false;
    const int nb = (int)big.size();
    const int ne = nb + (wsz ? 1 : 0);
    g.nops = nb + (int)small.size();
    g.nbig = nb;
    g.w_size = (uint32_t)wsz;
    std::vector<int> order = big;
    order.insert(order.end(), small.begin(), small.end());
    for (int j = 0; j < g.nops; ++j) {
      g.dt[j] = dt_of(order[j]);
      L->gf_src[j] = order[j];
    }
    g.out = GModes();
    g.kmodes = GModes();
    g.loop = GModes();
    g.wmodes = GModes();
    int64_t st[kMaxOps];
    bool ok = true;
    auto fill = [&](GModes& t, const Inds& grp, bool is_loop) {
      for (int64_t i : grp) {
        if (sliced.count(i)) continue;
        for (int j = 0; j < nb; ++j) st[j] = sof(big[j], i);
        if (wsz) st[nb] = wst.count(i) ? wst[i] : 0;
        ok &= gpush(t, is_loop ? dims.get(i) : dims.get(i), st, ne);
      }
      gmerge(t, ne);
    };
    fill(g.out, outg, false);
    fill(g.kmodes, kg, false);
    fill(g.loop, loopg, true);
    for (int64_t i : U) {
      for (int j = 0; j < (int)small.size(); ++j) st[j] = sof(small[j], i);
      ok &= gpush(g.wmodes, dims.get(i), st, (int)small.size());
    }
    if (!ok) return false;
    // keep W's modes unmerged but set up their divisions
    for (int m = 0; m < g.wmodes.n; ++m) g.wmodes.div[m] = make_fastdiv(g.wmodes.dim[m]);
    for (int j = 0; j < nb; ++j) {
      const int64_t mx = gmax(g.out, j) + gmax(g.loop, j) + gmax(g.kmodes, j) + slice_max[big[j]];
      if (mx >= extent[big[j]]) return false;
    }
    for (int j = 0; j < (int)small.size(); ++j)
      if (gmax(g.wmodes, j) + slice_max[small[j]] >= extent[small[j]]) return false;
    if (wsz && gmax(g.out, nb) + gmax(g.loop, nb) + gmax(g.kmodes, nb) >= wsz) return false;
    // a long sum over few outputs: the tiled dot kernel, else the generic
    // path's block reduction
    if (g.mode == GW_DENSE_PAIR || g.mode == GW_DENSE_F64) {
      const int64_t nl_ = (int64_t)gsize(g.loop), no_ = (int64_t)gsize(g.out);
      if (nl_ >= 1024 && no_ <= (int64_t)ex->sm_count * 16) {
        g.n_out = (uint32_t)no_;
        g.n_loop = (uint32_t)nl_;
        if (nb != 2 || wsz || !dot_setup(g, ex->sm_count)) return false;
      }
    }
    L->gf = g;
    L->has_fast = true;
    return true;
  };

  // gather launch writing `inds` (dense) from the product of reprs
  auto gather_launch = [&](const std::vector<const Repr*>& rs, const Inds& out_inds, const Inds& extra_loop,
                           int mode, int dst, double flops, int kclass, Launch* L) -> bool {
    GatherArgs g;
    std::vector<int> src;
    Inds loop;
    for (auto* r : rs) {
      for (int o : r->ops) src.push_back(o);
      for (int64_t i : r->L) loop.push_back(i);
    }
    for (int64_t i : extra_loop) loop.push_back(i);
    if ((int)src.size() > kMaxOps) return false;
    g.nops = (int)src.size();
    g.mode = mode;
    for (int j = 0; j < g.nops; ++j) g.dt[j] = dt_of(src[j]);
    int64_t st[kMaxOps];
    bool ok = true;
    for (int64_t i : out_inds) {
      if (sliced.count(i)) continue;
      for (int j = 0; j < g.nops; ++j) st[j] = sof(src[j], i);
      ok &= gpush(g.out, dims.get(i), st, g.nops);
    }
    for (int64_t i : loop) {
      if (sliced.count(i)) continue;
      for (int j = 0; j < g.nops; ++j) st[j] = sof(src[j], i);
      ok &= gpush(g.loop, dims.get(i), st, g.nops);
    }
    if (!ok) return false;
    gmerge(g.out, g.nops);
    gmerge(g.loop, g.nops);
    if (gsize(g.out) > 0x7FFFFFFFull || gsize(g.loop) > 0x7FFFFFFFull) return false;
    g.n_out = (uint32_t)gsize(g.out);
    g.n_loop = (uint32_t)gsize(g.loop);
    if (!check(g, src)) return false;
    L->kind = LK_GATHER;
    L->kclass = kclass;
    L->nsrc = g.nops;
    for (int j = 0; j < g.nops; ++j) L->src[j] = src[j];
    L->din = 0;
    for (int j = 0; j < g.nops; ++j) L->din |= toutof(src[j]);
    L->dout = dst >= nl ? toutof(dst) : 0;
    L->dst = dst;
    L->g = g;
    L->flops = flops;
    if (!fast_off) fast_args(src, out_inds, {}, loop, g, L);
    double by = (double)g.n_out * (mode == GW_DENSE_F64 ? 8 : 8);
    for (int s : std::set<int>(src.begin(), src.end())) by += bytes_of(s);
    L->bytes = by;
    return true;
  };
  // split launch: rows = row_inds, K = k_inds, from one repr
  auto split_launch = [&](const Repr& r, const Inds& row_inds, const Inds& k_inds, int dst, Launch* L,
                          int64_t* rows_out, int64_t* K_out) -> bool {
    GatherArgs g;
    const std::vector<int>& src = r.ops;
    if ((int)src.size() > kMaxOps) return false;
    g.nops = (int)src.size();
    g.mode = split_mode;
    for (int j = 0; j < g.nops; ++j) g.dt[j] = dt_of(src[j]);
    int64_t st[kMaxOps];
    bool ok = true;
    for (int64_t i : row_inds) {
      for (int j = 0; j < g.nops; ++j) st[j] = sof(src[j], i);
      ok &= gpush(g.out, dims.get(i), st, g.nops);
    }
    for (int64_t i : k_inds) {
      for (int j = 0; j < g.nops; ++j) st[j] = sof(src[j], i);
      ok &= gpush(g.kmodes, dims.get(i), st, g.nops);
    }
    for (int64_t i : r.L) {
      if (sliced.count(i)) continue;
      for (int j = 0; j < g.nops; ++j) st[j] = sof(src[j], i);
      ok &= gpush(g.loop, dims.get(i), st, g.nops);
    }
    if (!ok) return false;
    gmerge(g.out, g.nops);
    gmerge(g.kmodes, g.nops);
    gmerge(g.loop, g.nops);
    // read rows fastest when the leading operand is contiguous along a row mode
    int64_t min_row = INT64_MAX, min_k = INT64_MAX;
    for (int q = 0; q < g.out.n; ++q)
      if (g.out.stride[q][0] > 0) min_row = std::min(min_row, g.out.stride[q][0]);
    for (int q = 0; q < g.kmodes.n; ++q)
      if (g.kmodes.stride[q][0] > 0) min_k = std::min(min_k, g.kmodes.stride[q][0]);
    g.row_fast = min_row < min_k ? 1 : 0;
    const uint64_t rows = gsize(g.out), K = gsize(g.kmodes);
    if (rows * ((K + 7) / 8) > 0x7FFFFFFFull || gsize(g.loop) > 0x7FFFFFFFull) return false;
    g.n_rows = (uint32_t)rows;
    g.K = (uint32_t)K;
    g.Kp = (uint32_t)align_up(K, 8);
    g.n_loop = (uint32_t)gsize(g.loop);
    if (!check(g, src)) return false;
    L->kind = LK_GATHER;
    L->kclass = KC_SPLIT;
    L->nsrc = g.nops;
    for (int j = 0; j < g.nops; ++j) L->src[j] = src[j];
    L->din = 0;
    for (int j = 0; j < g.nops; ++j) L->din |= toutof(src[j]);
    L->dout = L->din;  // pieces are never summed over slice values
    L->dst = dst;
    L->g = g;
    if (!fast_off) {
      Inds rl, kl;
      for (int64_t i : row_inds) rl.push_back(i);
      for (int64_t i : k_inds) kl.push_back(i);
      if (fast_args(src, rl, kl, r.L, g, L)) {
        // same read order as the generic table: decided by the leading operand
        int64_t mr = INT64_MAX, mk = INT64_MAX;
        for (int q = 0; q < L->gf.out.n; ++q)
          if (L->gf.out.stride[q][0] > 0) mr = std::min(mr, L->gf.out.stride[q][0]);
        for (int q = 0; q < L->gf.kmodes.n; ++q)
          if (L->gf.kmodes.stride[q][0] > 0) mk = std::min(mk, L->gf.kmodes.stride[q][0]);
        L->gf.row_fast = mr < mk ? 1 : 0;
        // fan-out: innermost k (or row) mode carried by W alone, dim 2 or 4
        GatherArgs& f = L->gf;
        f.fan = 0;
        f.fan_f = 1;
        if (f.w_size && f.nbig == 1) {
          auto fan_ok = [&](const GModes& t) {
            if (t.n == 0) return 0;
            const int m = t.n - 1;
            const uint32_t d = t.dim[m];
            return (t.stride[m][0] == 0 && t.stride[m][1] != 0 && (d == 2 || d == 4)) ? (int)d : 0;
          };
          if (int d = fan_ok(f.kmodes)) {
            f.fan = 1;
            f.fan_f = d;
          } else if (int d2 = fan_ok(f.out)) {
            f.fan = 2;
            f.fan_f = d2;
          }
        }
      }
    }
    // algorithmic bytes: the operand read once (the piece planes the split
    // writes are this implementation's staging, not work of the method)
    double by = 0;
    for (int s : std::set<int>(src.begin(), src.end())) by += bytes_of(s);
    L->bytes = by;
    *rows_out = (int64_t)rows;
    *K_out = (int64_t)K;
    return true;
  };

  // The (non-sliced) indices the step consuming tensor t contracts, following
  // t through absorptions of small leaves; empty if there is none.
  auto consumer_k = [&](int t, size_t from) -> Inds {
    for (size_t u = from + 1; u < plan.steps.size(); ++u) {
      const PlanStep& q = plan.steps[u];
      if (q.x != t && q.y != t) continue;
      const int other = q.x == t ? q.y : q.x;
      if (other < nl && prod(live_inds[other]) <= (double)kSmallLeaf && u + 1 < plan.steps.size()) {
        t = q.out;  // folded into the consumer of the absorption's result
        continue;
      }
      return nsl(q.k);
    }
    return Inds();
  };

  // Can operand R (rows, K in the consumer's order) be written in piece form
  // by the epilogue of the GEMM that produced its one large factor?  It must
  // be that GEMM result times small leaves, with no summed index, carry
  // exactly the result's indices, have K equal to the result's M or N index
  // group in stored order, and fit the result's arena slot.
  auto fuse_check = [&](const Repr& R, const Inds& rows, const Inds& K, GemmFuse* F, std::vector<int>* small_ids,
                        int* T_out) -> bool {
    if (fuse_off || prec != 3 || !R.L.empty()) return false;
    int T = -1;
    std::vector<int> small;
    for (int o : R.ops) {
      if (o < nl && prod(live_inds[o]) <= (double)kSmallLeaf) {
        small.push_back(o);
      } else {
        if (T >= 0) return false;
        T = o;
      }
    }
    auto it = gemm_out.find(T);
    if (T < 0 || it == gemm_out.end()) return false;
    const GemmOut& P = it->second;
    const Launch& LP = ex->launches[P.li];
    // the fused epilogue's tiles: 128 columns, or one 160-column tile over the
    // whole N side (its k-blocks then never cross a tile)
    const bool fuse_tile = !LP.gemm.pair && (LP.gemm.bn == 128 || (LP.gemm.bn == kFuseWideBN && LP.gemm.N <= kFuseWideBN));
    const uint32_t w_cap = LP.gemm.bn == kFuseWideBN ? kFuseMaxWWide : kFuseMaxW;
    if (LP.kind != LK_GEMM || LP.gemm.fuse.on || LP.gemm.prec != 3 || !fuse_tile || (P.K + 63) / 64 > 16)
      return false;
    // pieces cannot be added up: the producer must not sum over slice values
    if (LP.din != LP.dout) return false;
    int k_is_m;
    if (K == P.inner)
      k_is_m = 1;
    else if (K == P.outer)
      k_is_m = 0;
    else
      return false;
    std::set<int64_t> mine(rows.begin(), rows.end()), theirs;
    for (int64_t i : K) mine.insert(i);
    for (const Inds* g : {&P.batch, &P.inner, &P.outer}) theirs.insert(g->begin(), g->end());
    if (mine != theirs || mine.size() != rows.size() + K.size()) return false;
    const double rows_total = prod(rows);
    const uint64_t Kp = align_up((uint64_t)prod(K), 8);
    if (rows_total * (double)Kp >= 2147483647.0 || 3.0 * rows_total * (double)Kp * 2.0 > (double)extent[T] * 8.0)
      return false;
    // W over the small leaves' non-sliced indices, dense in first-seen order
    Inds U;
    for (int t : small)
      for (int64_t i : live_inds[t])
        if (!sliced.count(i) && !contains(U, i)) U.push_back(i);
    std::map<int64_t, int64_t> wst;
    int64_t wsz = 1;
    for (int j = (int)U.size() - 1; j >= 0; --j) {
      wst[U[j]] = wsz;
      wsz *= dims.get(U[j]);
    }
    if (small.empty()) wsz = 0;
    if (wsz > (int64_t)w_cap || (int)small.size() > kMaxOps) return false;
    for (int64_t i : U)
      if (!mine.count(i)) return false;
    std::map<int64_t, int64_t> rst;
    int64_t acc = 1;
    for (int j = (int)rows.size() - 1; j >= 0; --j) {
      rst[rows[j]] = acc;
      acc *= dims.get(rows[j]);
    }
    GemmFuse f;
    f.on = 1;
    f.k_is_m = k_is_m;
    f.Kp = (uint32_t)Kp;
    f.piece = (int64_t)rows_total * (int64_t)Kp;
    auto add = [&](GModes& t, const Inds& g, bool to_rows) {
      for (int64_t i : g) {
        if (t.n >= kMaxModes) return false;
        t.dim[t.n] = (uint32_t)dims.get(i);
        t.div[t.n] = make_fastdiv(t.dim[t.n]);
        for (int q = 0; q < kMaxOps; ++q) t.stride[t.n][q] = 0;
        if (to_rows) t.stride[t.n][0] = rst.at(i);
        t.stride[t.n][1] = wst.count(i) ? wst[i] : 0;
        t.n++;
      }
      return true;
    };
    if (!add(f.bmodes, P.batch, true) || !add(f.mmodes, P.inner, !k_is_m) || !add(f.nmodes, P.outer, k_is_m))
      return false;
    for (int64_t i : P.batch)
      if (!rst.count(i)) return false;
    f.nsmall = (int)small.size();
    f.w_size = (uint32_t)wsz;
    for (int j = 0; j < f.nsmall; ++j) f.wdt[j] = dt_of(small[j]);
    int64_t st[kMaxOps];
    for (int64_t i : U) {
      for (int j = 0; j < f.nsmall; ++j) st[j] = sof(small[j], i);
      if (!gpush(f.wmodes, dims.get(i), st, f.nsmall)) return false;
    }
    for (int m = 0; m < f.wmodes.n; ++m) f.wmodes.div[m] = make_fastdiv(f.wmodes.dim[m]);
    for (int j = 0; j < f.nsmall; ++j)
      if (gmax(f.wmodes, j) + slice_max[small[j]] >= extent[small[j]]) return false;
    *F = f;
    *small_ids = small;
    *T_out = T;
    return true;
  };

  for (size_t s = 0; s < plan.steps.size(); ++s) {
    const PlanStep& ps = plan.steps[s];
    const bool last = s + 1 == plan.steps.size();
    const Inds batch = nsl(ps.batch), m = nsl(ps.m), n = nsl(ps.n), k = nsl(ps.k), sa = nsl(ps.sa),
               sb = nsl(ps.sb);
    const Inds &m_plan = m, &n_plan = n, &k_plan = k;
    Inds out_inds = batch;
    out_inds.insert(out_inds.end(), m.begin(), m.end());
    out_inds.insert(out_inds.end(), n.begin(), n.end());
    const double nb = prod(batch), nm = prod(m), nn = prod(n), nk = prod(k);
    const double step_flops = 2.0 * nb * nm * nn * nk;
    Repr& X = repr[ps.x];
    Repr& Y = repr[ps.y];
    const int dst = last ? DST_PARTIAL : ps.out;

    if (fp64) {
      // plain FP64 CUDA-core step
      ContractArgs c;
      memset(&c.out, 0, sizeof(ModeTab));
      memset(&c.loop, 0, sizeof(ModeTab));
      bool ok = true;
      for (int64_t i : batch) ok &= push_mode(c.out, dims.get(i), sof(ps.x, i), sof(ps.y, i));
      for (int64_t i : m) ok &= push_mode(c.out, dims.get(i), sof(ps.x, i), 0);
      for (int64_t i : n) ok &= push_mode(c.out, dims.get(i), 0, sof(ps.y, i));
      for (int64_t i : k) ok &= push_mode(c.loop, dims.get(i), sof(ps.x, i), sof(ps.y, i));
      for (int64_t i : sa) ok &= push_mode(c.loop, dims.get(i), sof(ps.x, i), 0);
      for (int64_t i : sb) ok &= push_mode(c.loop, dims.get(i), 0, sof(ps.y, i));
      if (!ok) return fail(QTPU_ENOTSUP, "a step has more than 12 modes in one group");
      merge_modes(c.out);
      merge_modes(c.loop);
      c.n_out = tab_size(c.out);
      c.n_loop = tab_size(c.loop);
      if (max_off(c.out, 0) + max_off(c.loop, 0) + slice_max[ps.x] >= extent[ps.x] ||
          max_off(c.out, 1) + max_off(c.loop, 1) + slice_max[ps.y] >= extent[ps.y])
        return fail(QTPU_ENOTSUP, "internal: operand view out of bounds");
      Launch L;
      L.kind = LK_CONTRACT64;
      L.kclass = KC_CONTRACT;
      L.din = toutof(ps.x) | toutof(ps.y);
      L.dout = last ? 0 : toutof(ps.out);
      L.nsrc = 2;
      L.src[0] = ps.x;
      L.src[1] = ps.y;
      L.dst = dst;
      L.c64 = c;
      L.flops = step_flops;
      L.bytes = bytes_of(ps.x) + bytes_of(ps.y) + (double)c.n_out * 8;
      set_dense(ps.out, out_inds);
      if (!last) place(ps.out);
      release(ps.x);
      release(ps.y);
      ex->launches.push_back(L);
      continue;
    }

    // ---- absorption of a small leaf: keep the result virtual
    auto small_leaf = [&](const Repr& r, int t) {
      return !r.virt && t < nl && prod(live_inds[t]) <= (double)kSmallLeaf;
    };
    const bool sx = small_leaf(X, ps.x), sy = small_leaf(Y, ps.y);
    const double big_size = sx ? prod(live_inds[ps.y]) : prod(live_inds[ps.x]);
    Inds vL = X.L;
    vL.insert(vL.end(), Y.L.begin(), Y.L.end());
    Inds stepL;
    for (const Inds* g : {&k, &sa, &sb}) stepL.insert(stepL.end(), g->begin(), g->end());
    vL.insert(vL.end(), stepL.begin(), stepL.end());
    // A virtual result sums prod(vL) terms per entry where it is finally read;
    // evaluating its parts step by step sums prod(X.L) + prod(Y.L) +
    // prod(stepL) at a comparable output size.  Keep it virtual only when
    // the product is not larger than that sum: a QT absorbing five 4 x 4
    // wire CTs at once would sum 4^5 = 1024 terms per entry instead of 5 x 4.
    const bool loop_ok = prod(vL) <= prod(X.L) + prod(Y.L) + prod(stepL);
    if (!last && (sx || sy) && !(sx && sy && nb * nm * nn > 4 * kSmallLeaf) &&
        nb * nm * nn <= 4.0 * big_size && (int)(X.ops.size() + Y.ops.size()) <= kMaxVirtualOps &&
        prod(vL) <= (double)kMaxVirtualLoop && loop_ok) {
      Repr V;
      V.ops = X.ops;
      V.ops.insert(V.ops.end(), Y.ops.begin(), Y.ops.end());
      V.L = vL;
      V.virt = true;
      V.flops = X.flops + Y.flops + step_flops;
      live_inds[ps.out] = out_inds;
      repr[ps.out] = V;
      ex->n_fused_steps++;
      continue;
    }

    // ---- tensor-core GEMM step (operands swapped when M is the skinny side:
    // C^T = B^T A^T, so the 128-row tile runs along the longer dimension)
    const double lim = 2147483647.0;
    bool swap = nm < 64 && nn >= 64;
    int bn = 128, pair = 0;
    bool oriented = false;  // fixed by the fused split of the consumer
    // when the next GEMM will contract this result over exactly the m (or n)
    // indices, make that group the stored outer (N) one: the epilogue then
    // writes the next operand's pieces along each thread's own columns
    // (with QTPU_FUSE_KEEP_LAYOUT the default orientation stays).  Such a
    // result keeps the 128-column tile the fused epilogue needs: dropping a
    // split launch saves more than a narrower tile.
    // (a result summed over slice values never becomes pieces in the
    // epilogue: such a step takes its tile like any other)
    uint64_t din_step = 0;
    for (const Repr* R : {&X, &Y})
      for (int o : R->ops) din_step |= toutof(o);
    if (!fuse_off && prec == 3 && !last && din_step == toutof(ps.out)) {
      const Inds ck = consumer_k(ps.out, s);
      const std::set<int64_t> cks(ck.begin(), ck.end());
      int pref = -1;
      if (!ck.empty() && cks == std::set<int64_t>(m.begin(), m.end())) pref = 1;
      if (!ck.empty() && cks == std::set<int64_t>(n.begin(), n.end())) pref = 0;
      if (pref >= 0) {
        if (!fuse_keep_layout && (pref ? nn : nm) >= 64 && (pref ? nm : nn) >= 16) swap = pref == 1;
        oriented = true;
      }
    }
    if (!oriented) {
      choose_tile(tiles, prec, nb, nm, nn, nk, &swap, &bn, &pair);
      if (gemm_pair_override() >= 0) pair = gemm_pair_override();
    }
    if (prec != 3) pair = 0;
    // the tiles above 128 columns: 224 and 256 on CTA pairs, 160 and 144 on one CTA in BF16x3
    if (!gemm_bn_supported(bn, pair, prec)) bn = 128;
    const double gM = swap ? nn : nm, gN = swap ? nm : nn;
    // a result the next GEMM may take in piece form keeps a tile the fused
    // epilogue has: 128 columns, or one 160-column tile when the N side is
    // 129-160 wide and that fits the problem in one wave of CTAs where
    // 128-column tiles need two or more (small latency-bound steps)
    if (oriented && prec == 3 && gN > 128 && gN <= kFuseWideBN) {
      const double sms = ex->sm_count;
      const double t128 = nb * std::ceil(gM / 128.0) * std::ceil(gN / 128.0);
      const double t160 = nb * std::ceil(gM / 128.0);
      if (t128 > sms && t160 <= sms) bn = kFuseWideBN;
    }
    const bool tc = sa.empty() && sb.empty() && gM >= 64 && gN >= 16 && nk >= 8 &&
                    nb * nm * nn * nk >= (double)(1 << 22) && nb < lim && nm < lim && nn < lim && nk < lim &&
                    nb * std::ceil(gM / 128.0) * std::ceil(gN / (double)bn) < lim;
    if (tc) {
      // Mode order inside each split operand is free (K only has to agree
      // between the two): rows follow their operand's source strides, and K
      // follows the larger operand's, so its split reads and writes run
      // along the same unit-stride direction.
      auto rep_stride = [&](const Repr& r, int64_t i) {
        int64_t best = 0;
        double bsz = -1;
        for (int o : r.ops) {
          const double sz = prod(live_inds[o]);
          if (sz > bsz && sof(o, i)) best = sof(o, i), bsz = sz;
        }
        return best;
      };
      auto by_stride = [&](Inds v, const Repr& r) {
        std::stable_sort(v.begin(), v.end(),
                         [&](int64_t a, int64_t b) { return rep_stride(r, a) > rep_stride(r, b); });
        return v;
      };
      const double szX = prod(live_inds[ps.x]), szY = prod(live_inds[ps.y]);
      const Inds m = by_stride(m_plan, X), n = by_stride(n_plan, Y), k = by_stride(k_plan, szX >= szY ? X : Y);
      Inds rowsX = batch, rowsY = batch;
      rowsX.insert(rowsX.end(), m.begin(), m.end());
      rowsY.insert(rowsY.end(), n.begin(), n.end());
      const Repr& RA = swap ? Y : X;
      const Repr& RB = swap ? X : Y;
      const Inds& rowsA = swap ? rowsY : rowsX;
      const Inds& rowsB = swap ? rowsX : rowsY;
      // an operand that is a GEMM result is written in piece form by that
      // GEMM's epilogue when K can follow the result's M or N index group
      Inds kk = k;
      for (const Repr* R : {&RA, &RB}) {
        int T = -1;
        for (int o : R->ops)
          if (!(o < nl && prod(live_inds[o]) <= (double)kSmallLeaf)) T = o;
        auto it = gemm_out.find(T);
        if (it == gemm_out.end()) continue;
        const std::set<int64_t> ks(k.begin(), k.end());
        if (ks == std::set<int64_t>(it->second.inner.begin(), it->second.inner.end()) && k.size() == it->second.inner.size()) {
          kk = it->second.inner;
          break;
        }
        if (ks == std::set<int64_t>(it->second.outer.begin(), it->second.outer.end()) && k.size() == it->second.outer.size()) {
          kk = it->second.outer;
          break;
        }
      }
      GemmFuse FA, FB;
      std::vector<int> smA, smB;
      int TA = -1, TB = -1;
      const bool fa = fuse_check(RA, rowsA, kk, &FA, &smA, &TA);
      const bool fb = fuse_check(RB, rowsB, kk, &FB, &smB, &TB) && TB != TA;
      Launch LA, LB, LG;
      int64_t ra = 0, rb = 0, Ka = 0, Kb = 0;
      if (fa) ra = (int64_t)prod(rowsA), Ka = (int64_t)prod(kk);
      if (fb) rb = (int64_t)prod(rowsB), Kb = (int64_t)prod(kk);
      if ((fa || split_launch(RA, rowsA, kk, DST_SPLIT_A, &LA, &ra, &Ka)) &&
          (fb || split_launch(RB, rowsB, kk, DST_SPLIT_B, &LB, &rb, &Kb)) && Ka == Kb) {
        const size_t abytes = align_up((size_t)np * ra * align_up(Ka, 8) * es, 1024);
        const size_t bbytes = align_up((size_t)np * rb * align_up(Kb, 8) * es, 1024);
        if (!fa) split_need_a = std::max(split_need_a, abytes);
        if (!fb) split_need_b = std::max(split_need_b, bbytes);
        for (int side = 0; side < 2; ++side) {
          const bool f = side ? fb : fa;
          if (!f) continue;
          const int T = side ? TB : TA;
          Launch& LP = ex->launches[gemm_out[T].li];
          LP.gemm.fuse = side ? FB : FA;
          LP.tile_fixed = true;
          const std::vector<int>& sm = side ? smB : smA;
          for (size_t j = 0; j < sm.size(); ++j) LP.fuse_src[j] = sm[j];
          // the pieces it now writes carry the absorbed factors' slices too
          for (int t : sm) LP.din |= toutof(t), LP.dout |= toutof(t);
          LG.opnd_fused[side] = T;
          LG.opnd_kp[side] = (uint32_t)align_up(Ka, 8);
          ex->n_fused_splits++;
        }
        // the last step of a sliced plan writes an intermediate that one more
        // launch adds into the FP64 partial (the slice sum stays FP64)
        const bool last_sliced = last && nsp > 0;
        LG.kind = LK_GEMM;
        LG.kclass = KC_GEMM;
        LG.dst = last_sliced ? ps.out : dst;
        for (const Repr* R : {&X, &Y})
          for (int o : R->ops) LG.din |= toutof(o);
        LG.dout = (last && !last_sliced) ? 0 : toutof(ps.out);
        LG.gemm.batch = (int)nb;
        LG.gemm.M = (int)gM;
        LG.gemm.N = (int)gN;
        LG.gemm.K = (int)Ka;
        LG.gemm.prec = prec;
        LG.gemm.bn = bn;
        LG.gemm.pair = pair;
        LG.tile_key[0] = prec, LG.tile_key[1] = (int64_t)nb, LG.tile_key[2] = (int64_t)nm;
        LG.tile_key[3] = (int64_t)nn, LG.tile_key[4] = (int64_t)nk;
        LG.tile_fixed = oriented;
        LG.gemm.kc_blocks = ex->kc_blocks;
        LG.flops = step_flops + X.flops + Y.flops;
        // algorithmic bytes: the result written once (its operands are
        // counted by the splits that read them)
        LG.bytes = nb * nm * nn * 8.0;
        // the GEMM stores [batch][its N][its M]
        Inds stored = batch;
        const Inds& outer = swap ? m : n;
        const Inds& inner = swap ? n : m;
        stored.insert(stored.end(), outer.begin(), outer.end());
        stored.insert(stored.end(), inner.begin(), inner.end());
        set_dense(ps.out, stored);
        if (!last || last_sliced) place(ps.out);
        for (int o : X.ops) release(o);
        for (int o : Y.ops) release(o);
        for (int t : {TA, TB})
          if (t >= 0) gemm_out.erase(t);
        if (!fa) {
          LG.opnd_split[0] = (int)ex->launches.size();
          ex->launches.push_back(LA);
        }
        if (!fb) {
          LG.opnd_split[1] = (int)ex->launches.size();
          ex->launches.push_back(LB);
        }
        if (!last) gemm_out[ps.out] = GemmOut{ex->launches.size(), batch, inner, outer, (int64_t)Ka};
        ex->launches.push_back(LG);
        ex->n_tc_steps++;
        repr[ps.out] = Repr();
        repr[ps.out].ops = {ps.out};
        if (last_sliced) {
          Launch LF;
          if (!gather_launch({&repr[ps.out]}, stored, {}, GW_DENSE_F64, DST_PARTIAL, 0, KC_REDUCE, &LF))
            return fail(QTPU_ENOTSUP, "internal: the last result does not fit the gather kernel");
          ex->launches.push_back(LF);
          release(ps.out);
        }
        continue;
      }
    }

    // ---- gather step (materialises the result)
    Inds extra = k;
    extra.insert(extra.end(), sa.begin(), sa.end());
    extra.insert(extra.end(), sb.begin(), sb.end());
    // a virtual operand is materialised first when it has too many factors
    // for one gather, when this step would recompute each of its entries
    // many times (every output reads it over the whole loop), or when the
    // product of its loop and this step's sums more terms than the two
    // done one after the other
    for (Repr* r : {&X, &Y}) {
      const double vsize = r->virt ? prod(live_inds[r == &X ? ps.x : ps.y]) : 1.0;
      const double reuse = r->virt ? (nb * nm * nn) * prod(extra) / vsize : 0.0;
      // terms summed by this gather with r virtual, and by materialising r
      // first (its own loop once per entry) and then gathering without it
      const double fused_terms = (nb * nm * nn) * prod(X.L) * prod(Y.L) * prod(extra);
      const double split_terms = vsize * prod(r->L) + fused_terms / prod(r->L);
      if (r->virt && ((int)(X.ops.size() + Y.ops.size()) > kMaxOps || reuse > 4.0 || fused_terms > split_terms)) {
        const int tid = next_tmp++;
        const Inds vin = live_inds[r == &X ? ps.x : ps.y];
        tout[tid] = toutof(r == &X ? ps.x : ps.y);
        Launch L;
        if (!gather_launch({r}, vin, {}, GW_DENSE_PAIR, tid, r->flops, KC_CONTRACT, &L))
          return fail(QTPU_ENOTSUP, "internal: cannot lower a fused tensor");
        set_dense(tid, vin);
        place(tid);
        for (int o : r->ops) release(o);
        ex->launches.push_back(L);
        *r = Repr();
        r->ops = {tid};
      }
    }
    Launch L;
    // the last step of a slice produces output values: FP64 accumulation and
    // an FP64 partial (the slice sum then stays in FP64 throughout)
    if (!gather_launch({&X, &Y}, out_inds, extra, last ? GW_DENSE_F64 : GW_DENSE_PAIR, dst,
                       step_flops + X.flops + Y.flops, KC_CONTRACT, &L))
      return fail(QTPU_ENOTSUP, "internal: a step does not fit the gather kernel (modes or operand views)");
    set_dense(ps.out, out_inds);
    if (!last) place(ps.out);
    for (int o : X.ops) release(o);
    for (int o : Y.ops) release(o);
    ex->launches.push_back(L);
    repr[ps.out] = Repr();
    repr[ps.out].ops = {ps.out};
  }

  // ---- final reduction: slices and leftover indices -> output order (FP64)
  Launch R;
  if (plan.steps.empty()) {
    const Leaf& Lf = leaves[0];
    Inds loop;
    for (size_t a = 0; a < Lf.ids.size(); ++a)
      if (!contains(plan.output, Lf.ids[a])) loop.push_back(Lf.ids[a]);
    // the leaf's sliced indices are summed here as well
    stride[0].clear();
    for (size_t a = 0; a < Lf.ids.size(); ++a) stride[0][Lf.ids[a]] = Lf.strides[a];
    std::set<int64_t> saved = sliced;
    sliced.clear();
    slice_max[0] = 0;
    Repr r0;
    r0.ops = {0};
    const bool ok = gather_launch({&r0}, plan.output, loop, GW_DENSE_F64, DST_OUT, 0, KC_REDUCE, &R);
    sliced = saved;
    if (!ok) return fail(QTPU_ENOTSUP, "the output does not fit the reduction kernel");
    ex->final_size = 0;
  } else {
    const int last = plan.steps.back().out;
    ex->final_size = extent[last];
    // partial[final]: the last launch adds every slice's result into it (in
    // FP64 when it is a gather), then this reduction sums the leftover
    // indices in a fixed order into the output order
    const int pid = next_tmp++;
    live_inds[pid] = live_inds[last];
    stride[pid] = stride[last];
    extent[pid] = ex->final_size;
    slice_max[pid] = 0;
    Inds loop;
    for (int64_t i : plan.final_sum)
      if (!sliced.count(i)) loop.push_back(i);
    // a gather as last launch writes FP64; a GEMM (unsliced plans only) its
    // (hi, lo) pairs, read exactly into the FP64 sum
    ex->partial_dt = (!fp64 && ex->launches.back().kind == LK_GEMM) ? DT_F32X2 : DT_F64;
    GatherArgs g;
    g.nops = 1;
    g.mode = GW_DENSE_F64;
    g.dt[0] = ex->partial_dt;
    int64_t st[kMaxOps] = {};
    bool ok = true;
    for (int64_t i : plan.output) {
      st[0] = sof(pid, i);
      ok &= gpush(g.out, dims.get(i), st, 1);
    }
    for (int64_t i : loop) {
      st[0] = sof(pid, i);
      ok &= gpush(g.loop, dims.get(i), st, 1);
    }
    if (!ok) return fail(QTPU_ENOTSUP, "the output does not fit the reduction kernel");
    gmerge(g.out, 1);
    gmerge(g.loop, 1);
    if (gsize(g.out) > 0x7FFFFFFFull || gsize(g.loop) > 0x7FFFFFFFull)
      return fail(QTPU_ENOTSUP, "the output does not fit the reduction kernel");
    g.n_out = (uint32_t)gsize(g.out);
    g.n_loop = (uint32_t)gsize(g.loop);
    if (gmax(g.out, 0) + gmax(g.loop, 0) >= extent[pid]) return fail(QTPU_ENOTSUP, "internal: reduction out of bounds");
    R.kind = LK_GATHER;
    R.kclass = KC_REDUCE;
    R.nsrc = 1;
    R.src[0] = pid;
    R.dst = DST_OUT;
    R.g = g;
    R.bytes = (double)ex->final_size * 8 + (double)g.n_out * 8;
    offs[pid] = 0;  // resolved to the partial buffer at run time
  }
  if (fp64) {
    // the FP64 path reduces with the FP64 kernel (same views)
    ContractArgs c;
    memset(&c.out, 0, sizeof(ModeTab));
    memset(&c.loop, 0, sizeof(ModeTab));
    for (int m = 0; m < R.g.out.n; ++m) push_mode(c.out, R.g.out.dim[m], R.g.out.stride[m][0], 0);
    for (int m = 0; m < R.g.loop.n; ++m) push_mode(c.loop, R.g.loop.dim[m], R.g.loop.stride[m][0], 0);
    c.n_out = tab_size(c.out);
    c.n_loop = tab_size(c.loop);
    R.kind = LK_CONTRACT64;
    R.c64 = c;
  }
  ex->reduce = R;

  // ---- slice reuse schedule (see the comment at tout): groups, blocked
  // positions, copies and the arena layout.
  // A GEMM forms a group with the splits of its operands; every other launch
  // is a group of its own.
  ex->groups.clear();
  for (size_t i = 0; i < ex->launches.size(); ++i) {
    const Launch& L = ex->launches[i];
    if (L.kind == LK_GATHER && (L.dst == DST_SPLIT_A || L.dst == DST_SPLIT_B)) continue;
    Group G;
    G.main = (int)i;
    if (L.kind == LK_GEMM) G.split[0] = L.opnd_split[0], G.split[1] = L.opnd_split[1];
    ex->groups.push_back(G);
  }
  std::vector<int> producer(next_tmp + 1, -1);
  for (size_t i = 0; i < ex->launches.size(); ++i)
    if (ex->launches[i].dst >= nl) producer[ex->launches[i].dst] = (int)i;
  const std::vector<int64_t>& sd = ex->slice_dims;
  auto count_of = [&](uint64_t m) {
    double c = 1;
    for (int p = 0; p < nsp; ++p)
      if ((m >> p) & 1) c *= (double)sd[p];
    return c;
  };
  auto tbytes = [&](int t) { return align_up((size_t)extent[t] * 8, 1024); };
  auto copies_of = [&](int t, uint64_t F) {
    const int pr = producer[t];
    return pr < 0 ? 1.0 : count_of(ex->launches[pr].dout & ~F);
  };
  // arena layout with the copies of every intermediate under blocked set F
  auto layout = [&](uint64_t F, std::map<int, size_t>* off_out) -> double {
    Arena ar;
    std::map<int, size_t> off;
    std::map<int, size_t> sz;
    for (auto& ev : events) {
      const int t = ev.first;
      if (ev.second > 0) {
        const double c = copies_of(t, F);
        if ((double)tbytes(t) * c > 1e15) return 1e30;
        sz[t] = (size_t)c * tbytes(t);
        off[t] = ar.alloc(sz[t]);
      } else {
        ar.release(off[t], sz[t]);
      }
    }
    if (off_out) *off_out = off;
    return (double)ar.top;
  };
  auto cost_of = [&](uint64_t F) {
    double c = 0;
    for (const Launch& L : ex->launches) c += L.flops * count_of(L.din | F);
    return c;
  };
  const uint64_t all_pos = nsp ? ((nsp >= 64 ? ~0ull : (1ull << nsp) - 1)) : 0;
  uint64_t F = all_pos;  // every position blocked: each slice on its own
  if (reuse && nsp > 0) {
    double best_c = cost_of(F);
    const double budget = (double)ex->reuse_budget;
    auto consider = [&](uint64_t f) {
      const double c = cost_of(f);
      if (c < best_c && layout(f, nullptr) <= budget) best_c = c, F = f;
    };
    if (nsp <= 12) {
      for (uint64_t f = 0; f < all_pos; ++f) consider(f);
    } else {  // release blocked positions one at a time while it fits
      for (bool more = true; more;) {
        more = false;
        const uint64_t base = F;
        for (int p = 0; p < nsp; ++p)
          if ((base >> p) & 1) {
            const uint64_t f = base & ~(1ull << p);
            const double c0 = best_c;
            consider(f);
            if (best_c < c0) more = true;
          }
      }
    }
  }
  ex->fixed = F;
  std::map<int, size_t> toff;
  ex->arena_bytes = std::max<size_t>((size_t)layout(F, &toff), 256);
  {
    const double per_slice = layout(all_pos, nullptr);
    ex->kept_bytes = (double)ex->arena_bytes > per_slice ? (size_t)((double)ex->arena_bytes - per_slice) : 0;
  }
  ex->stored.assign(next_tmp - nl + 1, Stored());
  for (auto& kv : toff) {
    const int t = kv.first;
    if (t < nl) continue;
    Stored& S = ex->stored[t - nl];
    S.off = kv.second;
    S.bytes = tbytes(t);
    const int pr = producer[t];
    if (pr >= 0)
      for (int q = 0; q < nsp; ++q)
        if (((ex->launches[pr].dout & ~F) >> q) & 1) S.cpos.push_back(q);
    offs[t] = kv.second;
  }
  // group loop orders and executions per contraction
  const double blocks = count_of(F);
  size_t kept_total = 0;
  bool kept_on = true;
  if (const char* e = std::getenv("QTPU_NO_KEPT_SPLITS")) kept_on = std::atoi(e) == 0;
  ex->flops_executed = ex->flops_no_reuse = 0;
  ex->launches_per_contract = 1;
  ex->n_split_slots = 1;
  std::vector<double> launches_of(ex->launches.size(), 0);
  for (Group& G : ex->groups) {
    Launch& M = ex->launches[G.main];
    // a GEMM sums the values of the positions it contracts inside one launch
    // (operand pair per value): those positions go innermost, and each split
    // that depends on them fills one slot per value
    G.sum_pos = M.kind == LK_GEMM ? (M.din & ~M.dout & ~F) : 0;
    uint64_t A = 0, B = 0;
    double ba = 0, bb = 0;
    if (G.split[0] >= 0) A = ex->launches[G.split[0]].din & ~F & ~G.sum_pos, ba = ex->launches[G.split[0]].bytes;
    if (G.split[1] >= 0) B = ex->launches[G.split[1]].din & ~F & ~G.sum_pos, bb = ex->launches[G.split[1]].bytes;
    if (bb > ba) std::swap(A, B);  // the larger split's positions outermost
    G.order.clear();
    for (uint64_t part : {A & B, A & ~B, B & ~A, (M.din & ~F) & ~(A | B) & ~G.sum_pos, G.sum_pos})
      for (int q = 0; q < nsp; ++q)
        if ((part >> q) & 1) G.order.push_back(q);
    const double V = count_of(G.sum_pos);
    M.runs = (int64_t)(count_of(M.din & ~F) * blocks);
    launches_of[G.main] = (double)M.runs / V * std::ceil(V / kGemmVals);
    if (G.sum_pos) ex->n_split_slots = std::max<int>(ex->n_split_slots, (int)std::min<double>(V, kGemmVals));
    // a split reruns when the outer positions up to its innermost own one
    // change; one that depends on a contracted position fills a slot per value
    std::vector<int> outer_order;
    for (int q : G.order)
      if (!((G.sum_pos >> q) & 1)) outer_order.push_back(q);
    for (int sp : G.split) {
      if (sp < 0) continue;
      Launch& S = ex->launches[sp];
      int last_j = -1;
      for (size_t j = 0; j < outer_order.size(); ++j)
        if (((S.din & ~F) >> outer_order[j]) & 1) last_j = (int)j;
      double r = 1;
      for (int j = 0; j <= last_j; ++j) r *= (double)sd[outer_order[j]];
      if (S.din & G.sum_pos) r *= V;
      // a split that would rerun for values it has already produced (an
      // outer position it does not depend on varies before its own) keeps
      // one result per value of its own positions instead, within a budget
      const double distinct = count_of(S.din & ~F);
      if (r > distinct && !fp64 && kept_on && (S.dst == DST_SPLIT_A || S.dst == DST_SPLIT_B)) {
        const GatherArgs& g = S.has_fast ? S.gf : S.g;
        const size_t slot_bytes = align_up((size_t)np * g.n_rows * g.Kp * es, 1024);
        if (kept_total + slot_bytes * (size_t)distinct <= kKeptSplitBudget) {
          S.kept_slots = (int64_t)distinct;
          S.kept_slot_bytes = slot_bytes;
          S.kept_off = kept_total;
          S.kept_side = S.dst == DST_SPLIT_A ? 0 : 1;
          S.dst = DST_KEPT;
          kept_total += slot_bytes * (size_t)distinct;
          r = distinct;
        }
      }
      S.runs = (int64_t)(r * blocks);
      launches_of[sp] = (double)S.runs;
    }
  }
  for (size_t i = 0; i < ex->launches.size(); ++i) {
    Launch& L = ex->launches[i];
    L.n_launch = (int64_t)(launches_of[i] > 0 ? launches_of[i] : (double)L.runs);
    ex->flops_executed += L.flops * (double)L.runs;
    ex->flops_no_reuse += L.flops * (double)ex->n_slices;
    ex->launches_per_contract += L.n_launch;
  }

  // ---- concurrent leaf splits: in an unsliced plan, a GEMM operand gathered
  // from leaves only does not depend on the chain; give it its own buffer
  // and run it on a second stream
  if (const char* e = std::getenv("QTPU_NO_GRAPH")) ex->use_graph = std::atoi(e) == 0;
  bool side_ok = !fp64 && ex->n_slices == 1 && ex->use_graph;
  if (const char* e = std::getenv("QTPU_NO_SIDE")) side_ok = side_ok && std::atoi(e) == 0;
  size_t side_total = 0;
  ex->n_side = 0;
  if (side_ok) {
    bool first = true;
    for (size_t i = 0; i < ex->launches.size(); ++i) {
      Launch& L = ex->launches[i];
      if (L.kind != LK_GATHER || (L.dst != DST_SPLIT_A && L.dst != DST_SPLIT_B)) continue;
      bool leaves_only = true;
      for (int j = 0; j < L.nsrc; ++j) leaves_only = leaves_only && L.src[j] < nl;
      if (!leaves_only) continue;
      // the first one stays on the main stream: the first GEMM's two leaf
      // splits then run side by side instead of one after the other
      if (first) {
        first = false;
        continue;
      }
      const GatherArgs& g = L.has_fast ? L.gf : L.g;
      const size_t bytes = align_up((size_t)np * g.n_rows * g.Kp * es, 1024);
      if (side_total + bytes > ((size_t)4 << 30)) continue;
      L.side = ex->n_side++;
      L.side_off = side_total;
      side_total += bytes;
      // the GEMM right after its two splits waits for this one
      for (size_t q = i + 1; q < ex->launches.size() && q <= i + 2; ++q)
        if (ex->launches[q].kind == LK_GEMM) {
          ex->launches[q].wait_side[L.dst == DST_SPLIT_A ? 0 : 1] = L.side;
          break;
        }
      L.dst = DST_SIDE;
    }
  }
  ex->side_bytes = side_total;
  ex->kept_split_bytes = kept_total;
  // large W tables are computed once per launch into a buffer of their own
  ex->wbuf_bytes = 0;
  for (auto& L : ex->launches)
    if (L.kind == LK_GATHER && L.has_fast && L.gf.w_size >= kGlobalW && !L.gf.dot &&
        (L.gf.mode == GW_DENSE_PAIR || L.gf.mode == GW_DENSE_F64)) {
      L.wg_off = (int64_t)ex->wbuf_bytes;
      ex->wbuf_bytes += align_up((size_t)L.gf.w_size * sizeof(float2), 256);
    }
  ex->split_slot[0] = split_need_a;
  ex->split_slot[1] = split_need_b;
  ex->split_a_bytes = split_need_a * ex->n_split_slots;
  ex->split_bytes = (split_need_a + split_need_b) * ex->n_split_slots;
  ex->lowered = true;
  if (dry_run) return "";

  // ---- device memory
  cudaError_t ce = cudaSetDevice(ex->device);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&ex->sm_count, cudaDevAttrMultiProcessorCount, ex->device);
  if (ce != cudaSuccess) return fail(QTPU_ECUDA, std::string("cuda: ") + cudaGetErrorString(ce));
  // QTPU_TEST_FAIL_ALLOC=1 makes the workspace allocation fail (a host-side
  // injection point for the out-of-memory path)
  const char* fa = std::getenv("QTPU_TEST_FAIL_ALLOC");
  const bool force_fail = fa && std::atoi(fa) != 0;
  auto dalloc = [&](void** p, size_t nbytes) -> bool {
    if (force_fail) return false;
    if (!nbytes) return true;
    if (cudaMalloc(p, nbytes) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  };
  if (!dalloc((void**)&ex->arena, ex->arena_bytes) || !dalloc((void**)&ex->splitbuf, ex->split_bytes) ||
      !dalloc((void**)&ex->partial, (size_t)std::max<int64_t>(ex->final_size, 1) * 8) ||
      !dalloc((void**)&ex->status, 16) || !dalloc((void**)&ex->out_stage, (size_t)R.g.n_out * 8 + 8) ||
      !dalloc((void**)&ex->dot_scratch, dot_scratch_entries(ex->sm_count) * sizeof(float2)) ||
      !dalloc((void**)&ex->wbuf, ex->wbuf_bytes) || !dalloc((void**)&ex->keptbuf, ex->kept_split_bytes)) {
    exec_free(ex);
    return fail(QTPU_ENOMEM, "device workspace allocation failed");
  }
  if (ex->n_side) {
    bool ok = dalloc((void**)&ex->sidebuf, ex->side_bytes) &&
              cudaStreamCreateWithFlags(&ex->side_stream, cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; ok && k < ex->n_side + 2; ++k) {
      cudaEvent_t e;
      ok = cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
      if (ok) ex->side_ev.push_back(e);
    }
    if (!ok) {
      cudaGetLastError();
      exec_free(ex);
      return fail(QTPU_ENOMEM, "side buffers");
    }
  }
  cudaMemset(ex->status, 0, 16);
  if (ex->n_tc_steps) {
    ce = gemm_prepare();
    if (ce != cudaSuccess) {
      exec_free(ex);
      return fail(QTPU_ECUDA, std::string("GEMM setup: ") + cudaGetErrorString(ce));
    }
  }
  if (const char* e = std::getenv("QTPU_NO_GRAPH")) ex->use_graph = std::atoi(e) == 0;
  if (ex->launches_per_contract > 20000) ex->use_graph = false;  // graph too large to be worth it
  if (ex->use_graph) {
    if (cudaStreamCreateWithFlags(&ex->own, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ex->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ex->ev_out, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      ex->use_graph = false;
    }
  }
  ex->inter_off.assign(next_tmp - nl + 1, 0);
  for (auto& kv : offs)
    if (kv.first >= nl) ex->inter_off[kv.first - nl] = kv.second;
  // tensor maps of the split buffers (fixed addresses); an operand whose
  // pieces are a kept result with several copies gets one map per copy
  for (size_t i = 0; i < ex->launches.size(); ++i) {
    Launch& L = ex->launches[i];
    if (L.kind != LK_GEMM) continue;
    uint8_t* base[2];
    int64_t kp[2];
    for (int side = 0; side < 2; ++side) {
      L.opnd_owner[side] = -1;
      L.tm_copies[side].clear();
      L.kept_maps[side].clear();
      if (L.opnd_split[side] >= 0 && ex->launches[L.opnd_split[side]].kept_slots) {
        // one map per kept result
        const Launch& S = ex->launches[L.opnd_split[side]];
        base[side] = ex->keptbuf + S.kept_off;
        kp[side] = S.g.Kp;
        const int64_t rows = side ? L.gemm.N : L.gemm.M;
        const int box = side ? gemm_b_box(L.gemm) : 128;
        L.kept_maps[side].resize((size_t)S.kept_slots);
        for (int64_t c = 0; c < S.kept_slots; ++c)
          if (!make_operand_map(&L.kept_maps[side][c], base[side] + (size_t)c * S.kept_slot_bytes, prec,
                                L.gemm.batch, rows, L.gemm.K, kp[side], box)) {
            exec_free(ex);
            return fail(QTPU_ECUDA, "cuTensorMapEncodeTiled failed");
          }
        continue;
      }
      if (L.opnd_split[side] >= 0) {
        const Launch& S = ex->launches[L.opnd_split[side]];
        base[side] = S.side >= 0 ? ex->sidebuf + S.side_off : ex->splitbuf + (side ? ex->split_a_bytes : 0);
        kp[side] = S.g.Kp;
        // one map per split slot (slot 0 is the map set below)
        const int64_t rows = side ? L.gemm.N : L.gemm.M;
        const int box = side ? gemm_b_box(L.gemm) : 128;
        for (int v = 1; v < ex->n_split_slots && S.side < 0; ++v) {
          CUtensorMap* m = side ? &L.gemm.maps.b[v] : &L.gemm.maps.a[v];
          if (!make_operand_map(m, base[side] + (size_t)v * ex->split_slot[side], prec, L.gemm.batch, rows, L.gemm.K,
                                kp[side], box)) {
            exec_free(ex);
            return fail(QTPU_ECUDA, "cuTensorMapEncodeTiled failed");
          }
        }
        continue;
      }
      const int T = L.opnd_fused[side];
      const Stored& St = ex->stored[T - nl];
      base[side] = ex->arena + St.off;
      kp[side] = L.opnd_kp[side];
      int64_t nc = 1;
      for (int q : St.cpos) nc *= ex->slice_dims[q];
      if (nc > 1) {
        L.opnd_owner[side] = T;
        const int64_t rows = side ? L.gemm.N : L.gemm.M;
        const int box = side ? gemm_b_box(L.gemm) : 128;
        L.tm_copies[side].resize((size_t)nc);
        for (int64_t c = 0; c < nc; ++c)
          if (!make_operand_map(&L.tm_copies[side][c], base[side] + (size_t)c * St.bytes, prec, L.gemm.batch, rows,
                                L.gemm.K, kp[side], box)) {
            exec_free(ex);
            return fail(QTPU_ECUDA, "cuTensorMapEncodeTiled failed");
          }
      }
    }
    if (!make_operand_map(&L.gemm.maps.a[0], base[0], prec, L.gemm.batch, L.gemm.M, L.gemm.K, kp[0], 128) ||
        !make_operand_map(&L.gemm.maps.b[0], base[1], prec, L.gemm.batch, L.gemm.N, L.gemm.K, kp[1],
                          gemm_b_box(L.gemm))) {
      exec_free(ex);
      return fail(QTPU_ECUDA, "cuTensorMapEncodeTiled failed");
    }
    L.gemm.status = ex->status;
  }
  return "";
}

namespace {
// event pair around one launch when profiling is on
struct Timed {
  Profiler& p;
  cudaStream_t st;
  size_t i = 0;
  bool on;
  unsigned flags = 0;  // external record nodes inside a stream capture
  Timed(Profiler& pr, cudaStream_t s, int kind, double fl, double by, int li = -1) : p(pr), st(s), on(pr.on) {
    if (!on) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
      flags = cudaEventRecordExternal;
    if (p.used * 2 + 2 > p.ev.size()) {
      for (int k = 0; k < 2; ++k) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
          on = false;
          return;
        }
        p.ev.push_back(e);
      }
      p.kind.push_back(0);
      p.lidx.push_back(-1);
      p.flops.push_back(0);
      p.bytes.push_back(0);
    }
    i = p.used++;
    p.kind[i] = kind;
    p.lidx[i] = li;
    p.flops[i] = fl;
    p.bytes[i] = by;
    cudaEventRecordWithFlags(p.ev[2 * i], st, flags);
  }
  ~Timed() {
    if (on) cudaEventRecordWithFlags(p.ev[2 * i + 1], st, flags);
  }
};
}  // namespace

std::string exec_describe(const Executor* ex) {
  std::ostringstream o;
  const char* cls[] = {"contract", "split", "gemm", "reduce"};
  auto one = [&](const Launch& L, size_t i) {
    o << "launch " << i << " " << cls[L.kclass] << " ";
    if (L.kind == LK_GEMM) {
      o << "gemm batch=" << L.gemm.batch << " M=" << L.gemm.M << " N=" << L.gemm.N << " K=" << L.gemm.K
        << " bn=" << L.gemm.bn << (L.gemm.pair ? " pair" : "");
      if (L.gemm.fuse.on) o << " writes-pieces k=" << (L.gemm.fuse.k_is_m ? "M" : "N") << " w=" << L.gemm.fuse.w_size;
    } else if (L.kind == LK_CONTRACT64) {
      o << "fp64 out=" << L.c64.n_out << " loop=" << L.c64.n_loop;
    } else {
      const GatherArgs& g = L.has_fast ? L.gf : L.g;
      o << (L.has_fast ? "fast" : "generic") << " ops=" << g.nops;
      if (L.has_fast) o << " big=" << g.nbig << " w=" << g.w_size << " fan=" << g.fan_f;
      if (L.has_fast && g.dot) o << " dot tile=" << g.tile_n << " outer=" << g.n_outer << " chunks=" << g.chunks;
      if (g.mode >= GW_SPLIT_BF16X3)
        o << " rows=" << g.n_rows << " K=" << g.K;
      else
        o << " out=" << g.n_out;
      o << " loop=" << g.n_loop;
      // per mode: dim:stride of each operand (0 = operand does not carry it)
      auto modes = [&](const char* name, const GModes& t) {
        o << " " << name << "=";
        for (int m = 0; m < t.n; ++m) {
          o << (m ? "," : "") << t.dim[m];
          for (int j = 0; j < g.nops && j < kMaxOps; ++j) o << (j ? "/" : ":") << t.stride[m][j];
        }
        if (!t.n) o << "-";
      };
      modes("om", g.out);
      if (g.mode >= GW_SPLIT_BF16X3) modes("km", g.kmodes);
      modes("lm", g.loop);
    }
    o << " src=";
    for (int j = 0; j < L.nsrc; ++j) o << (j ? "," : "") << L.src[j];
    if (L.kind == LK_GEMM) o << "-";
    o << " dst=" << L.dst << (L.side >= 0 ? " side" : "") << " flops=" << (long long)L.flops
      << " bytes=" << (long long)L.bytes;
    if (!ex->slice_dims.empty()) {
      auto pos = [&](uint64_t m) {
        std::string r;
        for (size_t q = 0; q < ex->slice_dims.size(); ++q)
          if ((m >> q) & 1) r += (r.empty() ? "" : ",") + std::to_string(q);
        return r.empty() ? std::string("-") : r;
      };
      o << " din=" << pos(L.din) << " dout=" << pos(L.dout) << " runs=" << L.runs << " launches=" << L.n_launch;
    }
    o << "\n";
  };
  for (size_t i = 0; i < ex->launches.size(); ++i) one(ex->launches[i], i);
  o << "reduce slices=" << ex->n_slices << " out=" << ex->reduce.g.n_out << " loop=" << ex->reduce.g.n_loop << "\n";
  o << "summary launches_per_slice=" << ex->launches.size() << " tensor_core_steps=" << ex->n_tc_steps
    << " fused_steps=" << ex->n_fused_steps << " fused_splits=" << ex->n_fused_splits << " side_splits=" << ex->n_side << " arena_bytes=" << ex->arena_bytes
    << " split_bytes=" << ex->split_bytes << "\n";
  o << "reuse blocked=";
  {
    std::string r;
    for (size_t q = 0; q < ex->slice_dims.size(); ++q)
      if ((ex->fixed >> q) & 1) r += (r.empty() ? "" : ",") + std::to_string(q);
    o << (r.empty() ? "-" : r);
  }
  o << " launches_per_contract=" << ex->launches_per_contract << " flops_executed=" << (long long)ex->flops_executed
    << " flops_all_slices=" << (long long)ex->flops_no_reuse << "\n";
  return o.str();
}

std::string exec_profile_read(Executor* ex, double* ms, int64_t* launches, double* flops, double* bytes) {
  for (int k = 0; k < KC_COUNT; ++k) ms[k] = 0, launches[k] = 0, flops[k] = 0, bytes[k] = 0;
  Profiler& p = ex->prof;
  for (size_t i = 0; i < p.used; ++i) {
    float t = 0;
    cudaError_t e = cudaEventElapsedTime(&t, p.ev[2 * i], p.ev[2 * i + 1]);
    if (e != cudaSuccess) {
      p.used = 0;
      return std::string("cudaEventElapsedTime: ") + cudaGetErrorString(e);
    }
    ms[p.kind[i]] += t;
    launches[p.kind[i]] += 1;
    flops[p.kind[i]] += p.flops[i];
    bytes[p.kind[i]] += p.bytes[i];
  }
  p.used = 0;
  return "";
}

std::string exec_profile_launches(Executor* ex, std::vector<int>* index, std::vector<double>* ms) {
  index->clear();
  ms->clear();
  Profiler& p = ex->prof;
  for (size_t i = 0; i < p.used; ++i) {
    float t = 0;
    cudaError_t e = cudaEventElapsedTime(&t, p.ev[2 * i], p.ev[2 * i + 1]);
    if (e != cudaSuccess) {
      p.used = 0;
      return std::string("cudaEventElapsedTime: ") + cudaGetErrorString(e);
    }
    index->push_back(p.lidx[i]);
    ms->push_back(t);
  }
  p.used = 0;
  return "";
}

void exec_launch_features(const Executor* ex, size_t i, float* f) {
  for (int j = 0; j < kLaunchFeatures; ++j) f[j] = 0.f;
  const Launch& L = ex->launches[i];
  auto lg = [](double x) { return (float)std::log2(1.0 + std::max(0.0, x)); };
  const double nv = L.kind == LK_GEMM ? std::max(1.0, (double)L.runs / (double)std::max<int64_t>(L.n_launch, 1)) : 1.0;
  f[31] = 1.f;
  f[6] = lg(L.flops * nv);
  f[7] = lg(L.bytes);
  const bool accum = L.din != L.dout;
  f[22] = accum ? 1.f : 0.f;
  if (L.kind == LK_GEMM) {
    const GemmArgs& g = L.gemm;
    f[0] = 1.f;
    f[8] = lg((double)g.batch * g.M * g.N);
    f[9] = lg((double)g.K * nv);
    f[10] = 2.f;
    f[13] = lg(g.M);
    f[14] = lg(g.N);
    f[15] = lg(g.K);
    f[16] = lg(g.batch);
    f[17] = (float)nv;
    const double mt = std::ceil(g.M / (g.pair ? 256.0 : 128.0)), nt = std::ceil(g.N / (double)g.bn);
    f[18] = (float)(g.M / ((g.pair ? 256.0 : 128.0) * mt));
    f[19] = (float)(g.N / ((double)g.bn * nt));
    f[20] = (float)(g.K / (64.0 * std::ceil(g.K / 64.0)));
    f[21] = g.fuse.on ? 1.f : 0.f;
    f[25] = lg((double)g.batch * mt * nt);
    return;
  }
  if (L.kind == LK_CONTRACT64) {
    f[5] = 1.f;
    f[8] = lg((double)L.c64.n_out);
    f[9] = lg((double)L.c64.n_loop);
    f[10] = (float)L.nsrc;
    f[28] = 1.f;
    return;
  }
  const GatherArgs& g = L.has_fast ? L.gf : L.g;
  const bool split = g.mode >= GW_SPLIT_BF16X3;
  if (split)
    f[1] = 1.f;
  else if (L.has_fast && g.dot)
    f[3] = 1.f;
  else if (L.has_fast)
    f[2] = 1.f;
  else
    f[4] = 1.f;
  f[8] = split ? lg((double)g.n_rows * g.Kp) : lg((double)g.n_out);
  f[9] = lg((double)g.n_loop);
  f[10] = (float)g.nops;
  f[11] = lg((double)g.w_size);
  f[12] = (float)g.fan_f;
  auto min_stride = [](const GModes& t) {
    int64_t m = 0;
    for (int q = 0; q < t.n; ++q)
      if (t.stride[q][0] > 0 && (m == 0 || t.stride[q][0] < m)) m = t.stride[q][0];
    return (double)m;
  };
  f[23] = lg(min_stride(g.out));
  f[24] = lg(min_stride(split ? g.kmodes : g.loop));
  f[25] = split ? lg(std::ceil(g.n_rows / 32.0) * std::ceil(g.Kp / 64.0)) : lg(g.n_out / 256.0);
  f[26] = (float)g.row_fast;
  f[27] = (float)(g.tile_n / 2048.0);
  f[28] = g.dt[0] == DT_F64 ? 1.f : 0.f;
  f[29] = L.has_fast ? 0.f : 1.f;
  f[30] = lg((double)g.loop.n);
}

namespace {
// A block of the slice space: per sliced position the value range [lo, hi).
struct Block {
  std::vector<int64_t> lo, hi;
};

// The blocks of slices [first, first + count) in slice-id order (slice id =
// mixed radix of the position values, last position fastest): the largest
// aligned runs, each a run of values of one position with every later
// position free and every earlier one fixed.
std::vector<Block> range_blocks(const std::vector<int64_t>& dims, int64_t first, int64_t count) {
  const int n = (int)dims.size();
  std::vector<int64_t> span(n + 1, 1);  // span[j]: slices per value of position j-1
  for (int j = n - 1; j >= 0; --j) span[j] = span[j + 1] * dims[j];
  std::vector<Block> out;
  int64_t a = first;
  const int64_t b = first + count;
  while (a < b) {
    // the coarsest position j whose whole values fit at a
    int j = n;
    while (j > 0 && a % span[j - 1] == 0 && a + span[j - 1] <= b) --j;
    Block B;
    B.lo.assign(n, 0);
    B.hi.assign(n, 0);
    int64_t r = a;
    for (int q = n - 1; q >= 0; --q) {
      B.lo[q] = r % dims[q];
      r /= dims[q];
    }
    if (j == n) {  // a single slice
      for (int q = 0; q < n; ++q) B.hi[q] = B.lo[q] + 1;
      a += 1;
    } else {
      // position j-1 (if any) runs over as many values as fit; later free
      for (int q = 0; q < n; ++q) B.hi[q] = B.lo[q] + 1;
      for (int q = j; q < n; ++q) B.lo[q] = 0, B.hi[q] = dims[q];
      if (j > 0) {
        const int64_t m = std::min<int64_t>((b - a) / span[j], dims[j - 1] - B.lo[j - 1]);
        B.hi[j - 1] = B.lo[j - 1] + m;
        a += m * span[j];
      } else {
        a += span[0];
      }
    }
    out.push_back(B);
  }
  return out;
}

// Enqueue every launch of one contraction (or of slices [first, first +
// count)) on `st`; the result goes to `out`.  Sliced plans run the groups of
// the slice-reuse schedule once per block: a group loops over the values of
// its main launch's din (within the block), re-running a split only when
// its own din values change, and the main launch adds up over the positions
// it contracts (the last launch over everything, into the FP64 partial).
//
// leaf_ready (optional, one event per leaf): each launch first makes its
// stream wait for the events of the leaves it reads (their uploads), once
// per stream.
cudaError_t enqueue_all(Executor* ex, const std::vector<Leaf>& leaves, double* out, cudaStream_t st,
                        int64_t first = 0, int64_t count = -1, const cudaEvent_t* leaf_ready = nullptr) {
  if (count < 0) count = ex->n_slices;
  const int nl = (int)leaves.size();
  const int nsp = (int)ex->slice_dims.size();
  std::vector<int64_t> loff(nl, 0);
  std::vector<int64_t> digit(nsp, 0);
  cudaError_t ce = cudaSuccess;
  std::vector<std::vector<cudaStream_t>> waited(leaf_ready ? nl : 0);
  auto wait_leaf = [&](int t, cudaStream_t s) -> cudaError_t {
    if (!leaf_ready || t < 0 || t >= nl) return cudaSuccess;
    for (cudaStream_t w : waited[t])
      if (w == s) return cudaSuccess;
    waited[t].push_back(s);
    return cudaStreamWaitEvent(s, leaf_ready[t], 0);
  };
  auto wait_sources = [&](const Launch& L, cudaStream_t s) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < L.nsrc && e == cudaSuccess; ++j) e = wait_leaf(L.src[j], s);
    if (L.kind == LK_GEMM && L.gemm.fuse.on)
      for (int j = 0; j < L.gemm.fuse.nsmall && e == cudaSuccess; ++j) e = wait_leaf(L.fuse_src[j], s);
    return e;
  };
  // copy index of an intermediate under the current position values
  auto copy_of = [&](const Stored& S) {
    int64_t c = 0;
    for (int q : S.cpos) c = c * ex->slice_dims[q] + digit[q];
    return c;
  };
  auto inter_ptr = [&](int t) -> uint8_t* {
    const Stored& S = ex->stored[t - nl];
    return ex->arena + S.off + (size_t)copy_of(S) * S.bytes;
  };
  auto src_ptr = [&](int t) -> const void* {
    if (t < nl) return (const uint8_t*)leaves[t].ptr + loff[t] * (int64_t)dt_bytes(leaves[t].dt);
    return inter_ptr(t);
  };
  const bool sided = ex->n_side > 0 && count == ex->n_slices && ex->n_slices == 1;
  const Launch* cur = nullptr;
  int cur_slot = 0;  // split slot of the launch being enqueued
  // operand maps of the values a GEMM launch sums (nullptr: its own maps)
  struct ValMaps {
    int n = 0;
    const CUtensorMap* a[kGemmVals];
    const CUtensorMap* b[kGemmVals];
  };
  const ValMaps* cur_vals = nullptr;
  auto dst_ptr = [&](int d) -> void* {
    switch (d) {
      case DST_SIDE: return ex->sidebuf + cur->side_off;
      case DST_KEPT: return ex->keptbuf + cur->kept_off + (size_t)cur_slot * cur->kept_slot_bytes;
      case DST_PARTIAL: return ex->partial;
      case DST_SPLIT_A: return ex->splitbuf + (size_t)cur_slot * ex->split_slot[0];
      case DST_SPLIT_B: return ex->splitbuf + ex->split_a_bytes + (size_t)cur_slot * ex->split_slot[1];
      case DST_OUT: return out;
      default: return inter_ptr(d);
    }
  };
  auto run_one_on = [&](const Launch& L, bool reduce, int accum, cudaStream_t st) -> cudaError_t {
    if (!reduce) {
      const cudaError_t we = wait_sources(L, st);
      if (we != cudaSuccess) return we;
    }
    cur = &L;
    // a GEMM launch summing several operand pairs does that many products
    const double nv = (L.kind == LK_GEMM && cur_vals) ? (double)cur_vals->n : 1.0;
    Timed t(ex->prof, st, L.kclass, L.flops * nv, L.bytes,
            reduce ? -1 : (int)(&L - ex->launches.data()));
    const bool from_partial = reduce && !ex->launches.empty();
    if (L.kind == LK_GATHER) {
      if (L.has_fast && !from_partial) {
        GatherArgs g = L.gf;
        for (int j = 0; j < g.nops; ++j) g.ptr[j] = src_ptr(L.gf_src[j]);
        g.scratch = ex->dot_scratch;
        g.accum = accum;
        if (L.wg_off >= 0) g.wg = reinterpret_cast<float2*>(ex->wbuf + L.wg_off);
        cudaError_t e = launch_gather_fast(g, dst_ptr(L.dst), ex->sm_count, st);
        if (e != cudaErrorNotSupported) return e;
        cudaGetLastError();
      }
      GatherArgs g = L.g;
      g.accum = accum;
      for (int j = 0; j < L.nsrc; ++j) g.ptr[j] = from_partial ? (const void*)ex->partial : src_ptr(L.src[j]);
      return launch_gather(g, dst_ptr(L.dst), ex->sm_count, st);
    }
    if (L.kind == LK_GEMM) {
      GemmArgs g = L.gemm;
      g.C = dst_ptr(L.dst);
      g.accum = accum;
      if (cur_vals) {
        g.nval = cur_vals->n;
        for (int v = 0; v < cur_vals->n; ++v) g.maps.a[v] = *cur_vals->a[v], g.maps.b[v] = *cur_vals->b[v];
      } else {
        if (L.opnd_owner[0] >= 0) g.maps.a[0] = L.tm_copies[0][(size_t)copy_of(ex->stored[L.opnd_owner[0] - nl])];
        if (L.opnd_owner[1] >= 0) g.maps.b[0] = L.tm_copies[1][(size_t)copy_of(ex->stored[L.opnd_owner[1] - nl])];
      }
      for (int j = 0; g.fuse.on && j < g.fuse.nsmall; ++j) g.fuse.wptr[j] = src_ptr(L.fuse_src[j]);
      return launch_gemm(g, ex->sm_count, st);
    }
    ContractArgs c = L.c64;
    c.accum = accum;
    const void* A = from_partial ? (const void*)ex->partial : src_ptr(L.src[0]);
    const void* B = reduce ? nullptr : src_ptr(L.src[1]);
    const int dta = from_partial ? ex->partial_dt : (L.src[0] < nl ? leaves[L.src[0]].dt : ex->inter_dt);
    const int dtb = reduce ? DT_F64 : (L.src[1] < nl ? leaves[L.src[1]].dt : ex->inter_dt);
    return launch_contract(A, dta, B, dtb, (double*)dst_ptr(L.dst), c, ex->sm_count, st);
  };
  auto run_one = [&](const Launch& L, bool reduce, int accum) { return run_one_on(L, reduce, accum, st); };
  if (sided) {
    // fork: every leaf-only split on the side stream first, one event each
    cudaStream_t ss = ex->side_stream;
    cudaEvent_t fork = ex->side_ev[ex->n_side], join = ex->side_ev[ex->n_side + 1];
    ce = cudaEventRecord(fork, st);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(ss, fork, 0);
    for (auto& L : ex->launches) {
      if (ce != cudaSuccess) break;
      if (L.side < 0) continue;
      ce = run_one_on(L, false, 0, ss);
      if (ce == cudaSuccess) ce = cudaEventRecord(ex->side_ev[L.side], ss);
    }
    for (auto& L : ex->launches) {
      if (ce != cudaSuccess) break;
      if (L.side >= 0) continue;
      for (int w : L.wait_side)
        if (w >= 0 && ce == cudaSuccess) ce = cudaStreamWaitEvent(st, ex->side_ev[w], 0);
      if (ce == cudaSuccess) ce = run_one(L, false, 0);
    }
    if (ce == cudaSuccess) ce = cudaEventRecord(join, ss);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(st, join, 0);
    if (ce == cudaSuccess) ce = run_one(ex->reduce, true, 0);
    return ce;
  }
  // blocks: a slice range in id order, split further over the blocked
  // positions (each blocked position takes one value per block)
  std::vector<Block> blocks;
  if (nsp == 0) {
    blocks.push_back(Block());
  } else {
    for (const Block& R : range_blocks(ex->slice_dims, first, count)) {
      std::vector<int> free_fixed;
      for (int q = 0; q < nsp; ++q)
        if (((ex->fixed >> q) & 1) && R.hi[q] - R.lo[q] > 1) free_fixed.push_back(q);
      int64_t n = 1;
      for (int q : free_fixed) n *= R.hi[q] - R.lo[q];
      for (int64_t k = 0; k < n; ++k) {
        Block B = R;
        int64_t r = k;
        for (int j = (int)free_fixed.size() - 1; j >= 0; --j) {
          const int q = free_fixed[j];
          const int64_t w = R.hi[q] - R.lo[q];
          B.lo[q] = R.lo[q] + r % w;
          B.hi[q] = B.lo[q] + 1;
          r /= w;
        }
        blocks.push_back(B);
      }
    }
  }
  bool final_written = false;
  const size_t n_launch = ex->launches.size();
  // per split and slot: the values of the split's positions it last ran with
  std::vector<std::vector<int64_t>> split_epoch(n_launch);
  auto set_leaf_offsets = [&]() {
    for (int t = 0; t < nl; ++t) {
      int64_t o = 0;
      for (auto& ps : ex->leaf_slice[t]) o += digit[ps.first] * ps.second;
      loff[t] = o;
    }
  };
  auto set_digits = [&](const std::vector<int>& pos, int64_t k, const Block& B) {
    for (int j = (int)pos.size() - 1; j >= 0; --j) {
      const int q = pos[j];
      const int64_t w = B.hi[q] - B.lo[q];
      digit[q] = B.lo[q] + k % w;
      k /= w;
    }
  };
  for (const Block& B : blocks) {
    if (ce != cudaSuccess) break;
    for (int q = 0; q < nsp; ++q) digit[q] = B.lo[q];
    for (const Group& G : ex->groups) {
      if (ce != cudaSuccess) break;
      const Launch& M = ex->launches[G.main];
      // positions that vary in this block: the outer ones (a loop of
      // launches) and, for a GEMM, the contracted ones (summed inside each
      // launch, up to kGemmVals operand pairs at a time)
      std::vector<int> outer, inner;
      for (int q : G.order)
        if (B.hi[q] - B.lo[q] > 1) (((G.sum_pos >> q) & 1) ? inner : outer).push_back(q);
      uint64_t inner_mask = 0;
      for (int q : inner) inner_mask |= 1ull << q;
      for (int q = 0; q < nsp; ++q)
        if ((M.din >> q) & 1) digit[q] = B.lo[q];
      for (int sp : G.split)
        if (sp >= 0)
          split_epoch[sp].assign((size_t)std::max<int64_t>(ex->launches[sp].kept_slots, ex->n_split_slots), -1);
      int64_t n_outer = 1, n_inner = 1;
      for (int q : outer) n_outer *= B.hi[q] - B.lo[q];
      for (int q : inner) n_inner *= B.hi[q] - B.lo[q];
      for (int64_t ko = 0; ko < n_outer && ce == cudaSuccess; ++ko) {
        set_digits(outer, ko, B);
        for (int64_t c0 = 0; c0 < n_inner && ce == cudaSuccess; c0 += kGemmVals) {
          const int nv = (int)std::min<int64_t>(kGemmVals, n_inner - c0);
          ValMaps vm;
          vm.n = nv;
          for (int j = 0; j < nv && ce == cudaSuccess; ++j) {
            set_digits(inner, c0 + j, B);
            set_leaf_offsets();
            int slot_of[2] = {0, 0};
            for (int side = 0; side < 2; ++side) {
              const int sp = G.split[side];
              if (sp < 0) continue;
              const Launch& S = ex->launches[sp];
              int slot = (S.din & inner_mask) ? j : 0;
              if (S.kept_slots) {  // the kept result of the current values of its positions
                int64_t k = 0;
                for (int q = 0; q < nsp; ++q)
                  if (((S.din >> q) & 1) && B.hi[q] - B.lo[q] > 1) k = k * (B.hi[q] - B.lo[q]) + (digit[q] - B.lo[q]);
                slot = (int)k;
              }
              slot_of[side] = slot;
              int64_t ep = 0;  // the values of the split's own positions
              for (int q = 0; q < nsp; ++q)
                if ((S.din >> q) & 1) ep = ep * ex->slice_dims[q] + digit[q];
              if (ep == split_epoch[sp][slot]) continue;
              split_epoch[sp][slot] = ep;
              cur_slot = slot;
              ce = run_one(S, false, 0);
              cur_slot = 0;
              if (ce != cudaSuccess) break;
            }
            if (M.kind == LK_GEMM) {
              for (int side = 0; side < 2; ++side) {
                const CUtensorMap* m;
                if (!M.kept_maps[side].empty())
                  m = &M.kept_maps[side][(size_t)slot_of[side]];
                else if (M.opnd_split[side] >= 0)
                  m = side ? &M.gemm.maps.b[slot_of[side]] : &M.gemm.maps.a[slot_of[side]];
                else if (M.opnd_owner[side] >= 0)
                  m = &M.tm_copies[side][(size_t)copy_of(ex->stored[M.opnd_owner[side] - nl])];
                else
                  m = side ? &M.gemm.maps.b[0] : &M.gemm.maps.a[0];
                (side ? vm.b : vm.a)[j] = m;
              }
            }
          }
          if (ce != cudaSuccess) break;
          // add up over the positions the launch contracts: a GEMM over its
          // later batches of values; any other launch on every visit after
          // the first with the same dout values; the last launch on every
          // visit after the contraction's first
          int accum = 0;
          if (M.dst == DST_PARTIAL) {
            accum = final_written ? 1 : 0;
            final_written = true;
          } else if (M.kind == LK_GEMM && inner_mask) {
            accum = c0 > 0 ? 1 : 0;
          } else {
            for (int q = 0; q < nsp; ++q)
              if ((((M.din & ~M.dout) >> q) & 1) && digit[q] != B.lo[q]) accum = 1;
          }
          cur_vals = (M.kind == LK_GEMM) ? &vm : nullptr;
          ce = run_one(M, false, accum);
          cur_vals = nullptr;
        }
      }
    }
  }
  if (ce == cudaSuccess) ce = run_one(ex->reduce, true, 0);
  return ce;
}
}  // namespace

std::string exec_run(Executor* ex, const std::vector<Leaf>& leaves, double* dev_out, cudaStream_t st, int* code) {
  *code = QTPU_OK;
  cudaError_t ce = cudaSuccess;
  if (!ex->use_graph) {
    ce = enqueue_all(ex, leaves, dev_out, st);
  } else {
    // the graph writes the output to the staging buffer; one small copy
    // moves it to the caller's buffer on the caller's stream
    const int gi = ex->prof.on ? 1 : 0;
    if (!ex->graph[gi]) {
      if (ex->prof.on) ex->prof.used = 0;
      cudaGraph_t g = nullptr;
      cudaGetLastError();  // a launch error left by earlier work must not fail this capture
      ce = cudaStreamBeginCapture(ex->own, cudaStreamCaptureModeThreadLocal);
      if (ce == cudaSuccess) {
        cudaError_t e1 = enqueue_all(ex, leaves, ex->out_stage, ex->own);
        ce = cudaStreamEndCapture(ex->own, &g);
        if (e1 != cudaSuccess) ce = e1;
      }
      if (ce == cudaSuccess) ce = cudaGraphInstantiate(&ex->graph[gi], g, 0);
      if (g) cudaGraphDestroy(g);
      if (ce != cudaSuccess) {
        cudaGetLastError();
        *code = QTPU_ECUDA;
        return std::string("graph capture failed: ") + cudaGetErrorString(ce);
      }
      if (ex->prof.on) ex->prof.graph_events = ex->prof.used;
    }
    // each replay records the captured events again: a profile read sees the
    // launches of the most recent contraction
    if (ex->prof.on) ex->prof.used = ex->prof.graph_events;
    ce = cudaEventRecord(ex->ev_in, st);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(ex->own, ex->ev_in, 0);
    if (ce == cudaSuccess) ce = cudaGraphLaunch(ex->graph[gi], ex->own);
    if (ce == cudaSuccess) ce = cudaEventRecord(ex->ev_out, ex->own);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(st, ex->ev_out, 0);
    if (ce == cudaSuccess && dev_out != ex->out_stage)
      ce = cudaMemcpyAsync(dev_out, ex->out_stage, (size_t)ex->reduce.g.n_out * 8, cudaMemcpyDeviceToDevice, st);
  }
  if (ce != cudaSuccess) {
    *code = QTPU_ECUDA;
    return std::string("launch failed: ") + cudaGetErrorString(ce);
  }
  return "";
}

std::string exec_run_host(Executor* ex, const std::vector<Leaf>& leaves, double* dev_out, cudaStream_t st,
                          const cudaEvent_t* leaf_ready, int* code) {
  *code = QTPU_OK;
  cudaError_t ce = enqueue_all(ex, leaves, dev_out, st, 0, -1, leaf_ready);
  if (ce != cudaSuccess) {
    *code = QTPU_ECUDA;
    return std::string("launch failed: ") + cudaGetErrorString(ce);
  }
  return "";
}

bool exec_batch_tasks(const Executor* ex, const std::vector<Leaf>& leaves, double* dev_out,
                      std::vector<BatchTask>* out) {
  out->clear();
  if (!ex->lowered || ex->n_slices != 1 || ex->launches.empty()) return false;
  // small networks only: the persistent kernel runs the generic gather; a
  // launch above this many terms keeps the typed kernels of a graph branch
  // (measured on B300: a batch of 512 networks of <= 2^14-entry QTs runs
  // 2.1x faster in the persistent kernel than as graph branches; in a batch
  // whose time is set by networks with GEMMs, moving networks with launches
  // above 2^16 terms into it only lengthened the batch)
  double max_terms = (double)(1 << 16);
  if (const char* e = std::getenv("QTPU_BATCH_MAX_TERMS")) max_terms = std::atof(e);
  for (const Launch& L : ex->launches) {
    if (L.kind != LK_GATHER || L.g.mode >= GW_SPLIT_BF16X3 || L.side >= 0) return false;
    if ((double)L.g.n_out * (double)L.g.n_loop > max_terms) return false;
  }
  const int nl = (int)leaves.size();
  auto src_ptr = [&](int t) -> const void* {
    if (t < nl) return leaves[t].ptr;
    return ex->arena + ex->stored[t - nl].off;
  };
  auto add = [&](const GatherArgs& g0, const int* src, int nsrc, bool from_partial, void* dst) {
    BatchTask T;
    T.g = g0;
    for (int j = 0; j < nsrc; ++j) T.g.ptr[j] = from_partial ? (const void*)ex->partial : src_ptr(src[j]);
    T.g.accum = 0;
    T.dst = dst;
    T.f64out = g0.mode == GW_DENSE_F64 ? 1 : 0;
    T.block_mode = (g0.n_loop >= 1024 && g0.n_out <= (uint32_t)ex->sm_count * 16) ? 1 : 0;
    T.n_units = T.block_mode ? g0.n_out : (g0.n_out + 255) / 256;
    T.status = ex->status;
    if (T.n_units == 0) T.n_units = 1;  // an empty task still completes one unit
    out->push_back(T);
  };
  for (const Launch& L : ex->launches) {
    void* dst = L.dst == DST_PARTIAL ? (void*)ex->partial
                                     : (L.dst == DST_OUT ? (void*)dev_out : (void*)(ex->arena + ex->stored[L.dst - nl].off));
    add(L.g, L.src, L.nsrc, false, dst);
  }
  add(ex->reduce.g, ex->reduce.src, ex->reduce.nsrc, true, dev_out);
  return true;
}

std::vector<int> exec_leaf_order(const Executor* ex, int n_leaves) {
  std::vector<int> order;
  std::vector<char> seen(n_leaves, 0);
  auto add = [&](int t) {
    if (t >= 0 && t < n_leaves && !seen[t]) seen[t] = 1, order.push_back(t);
  };
  // the side-stream splits run first in an unsliced plan
  for (const Launch& L : ex->launches)
    if (L.side >= 0)
      for (int j = 0; j < L.nsrc; ++j) add(L.src[j]);
  for (const Launch& L : ex->launches) {
    for (int j = 0; j < L.nsrc; ++j) add(L.src[j]);
    if (L.kind == LK_GEMM && L.gemm.fuse.on)
      for (int j = 0; j < L.gemm.fuse.nsmall; ++j) add(L.fuse_src[j]);
  }
  for (int t = 0; t < n_leaves; ++t) add(t);
  return order;
}

cudaError_t exec_enqueue(Executor* ex, const std::vector<Leaf>& leaves, double* out, cudaStream_t st) {
  return enqueue_all(ex, leaves, out, st);
}

std::string exec_run_slices(Executor* ex, const std::vector<Leaf>& leaves, int64_t first, int64_t count,
                            double* dev_out, cudaStream_t st, int* code) {
  *code = QTPU_OK;
  if (ex->launches.empty()) {
    *code = QTPU_ENOTSUP;
    return "slice ranges need a network with at least one pairwise step";
  }
  cudaError_t ce = enqueue_all(ex, leaves, dev_out, st, first, count);
  if (ce != cudaSuccess) {
    *code = QTPU_ECUDA;
    return std::string("launch failed: ") + cudaGetErrorString(ce);
  }
  return "";
}

void exec_free(Executor* ex) {
  for (int i = 0; i < 2; ++i)
    if (ex->graph[i]) cudaGraphExecDestroy(ex->graph[i]), ex->graph[i] = nullptr;
  if (ex->own) cudaStreamDestroy(ex->own), ex->own = nullptr;
  if (ex->ev_in) cudaEventDestroy(ex->ev_in), ex->ev_in = nullptr;
  if (ex->ev_out) cudaEventDestroy(ex->ev_out), ex->ev_out = nullptr;
  for (auto e : ex->prof.ev) cudaEventDestroy(e);
  ex->prof.ev.clear();
  ex->prof.used = 0;
  if (ex->arena) cudaFree(ex->arena);
  if (ex->splitbuf) cudaFree(ex->splitbuf);
  if (ex->partial) cudaFree(ex->partial);
  if (ex->status) cudaFree(ex->status);
  if (ex->out_stage) cudaFree(ex->out_stage);
  if (ex->dot_scratch) cudaFree(ex->dot_scratch);
  ex->dot_scratch = nullptr;
  if (ex->wbuf) cudaFree(ex->wbuf);
  ex->wbuf = nullptr;
  if (ex->keptbuf) cudaFree(ex->keptbuf);
  ex->keptbuf = nullptr;
  ex->arena = ex->splitbuf = ex->partial = nullptr;
  ex->status = nullptr;
  ex->out_stage = nullptr;
}

}  // namespace qtpu
