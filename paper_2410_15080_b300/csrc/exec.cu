// Executor: lowers a contraction plan to kernel launches.
//
// Section 6.1 step 4 contracts the evaluated classical TN on the available
// accelerator.  Each planned pairwise step becomes either
//   * a tensor-core step (large dense GEMM): two split kernels gather the
//     operands into [batch][rows][K] piece planes, then the tcgen05 GEMM
//     writes the FP64 result [batch][M][N]; or
//   * a generic FP64 step (CT absorption, dot products, skinny shapes).
// Intermediates live in one device arena laid out at build time (first-fit
// over the steps' lifetimes).  Slices (fixed values of the sliced indices)
// run one after another through the same launches with shifted leaf
// pointers; each slice's final tensor lands in partial[slice], and one FP64
// reduction sums the slices (and any leftover indices) in a fixed order into
// the output.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <sstream>

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
  CUresult r = enc(map, prec == 3 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base,
                   gdim, gstr, box, est, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

std::string exec_build(Executor* ex, const Plan& plan, const std::vector<Leaf>& leaves, const DimMap& dims,
                       int prec, int* code) {
  *code = QTPU_OK;
  ex->prec = prec;
  if (const char* e = std::getenv("QTPU_KC")) ex->kc_blocks = std::atoi(e);
  std::set<int64_t> sliced(plan.sliced.begin(), plan.sliced.end());
  const int nl = plan.n_leaves;
  const size_t n_t = plan.tensor_inds.size();

  // slice bookkeeping
  if (!plan.n_slices.fits_u64() || plan.n_slices.w[0] > (uint64_t)1 << 40) {
    *code = QTPU_ENOTSUP;
    return "slice count too large";
  }
  ex->n_slices = (int64_t)plan.n_slices.w[0];
  ex->slice_dims.clear();
  for (int64_t i : plan.sliced) ex->slice_dims.push_back(dims.get(i));
  ex->leaf_slice.assign(nl, {});
  for (int t = 0; t < nl; ++t)
    for (size_t p = 0; p < plan.sliced.size(); ++p) {
      const Leaf& L = leaves[t];
      for (size_t a = 0; a < L.ids.size(); ++a)
        if (L.ids[a] == plan.sliced[p]) ex->leaf_slice[t].push_back({(int)p, L.strides[a]});
    }

  // per-slice layout of every tensor: leaves keep their strides, step
  // results are dense over their non-sliced indices
  std::vector<Inds> live_inds(n_t);
  std::vector<std::map<int64_t, int64_t>> stride(n_t);
  for (int t = 0; t < nl; ++t)
    for (size_t a = 0; a < leaves[t].ids.size(); ++a)
      if (!sliced.count(leaves[t].ids[a])) {
        live_inds[t].push_back(leaves[t].ids[a]);
        stride[t][leaves[t].ids[a]] = leaves[t].strides[a];
      }
  for (size_t s = 0; s < plan.steps.size(); ++s) {
    const int o = plan.steps[s].out;
    for (int64_t i : plan.tensor_inds[o])
      if (!sliced.count(i)) live_inds[o].push_back(i);
    int64_t st = 1;
    for (int j = (int)live_inds[o].size() - 1; j >= 0; --j) {
      stride[o][live_inds[o][j]] = st;
      st *= dims.get(live_inds[o][j]);
    }
  }
  auto sof = [&](int t, int64_t i) -> int64_t {
    auto it = stride[t].find(i);
    return it == stride[t].end() ? 0 : it->second;
  };
  auto tsize = [&](int t) -> int64_t {
    int64_t s = 1;
    for (int64_t i : live_inds[t]) s *= dims.get(i);
    return s;
  };

  // extent (elements) of every tensor's storage and the largest offset the
  // slice loop adds to a leaf: every launch is checked to stay inside
  std::vector<int64_t> extent(n_t, 0), slice_max(n_t, 0);
  for (int t = 0; t < nl; ++t) {
    int64_t e = 1;
    for (size_t a = 0; a < leaves[t].ids.size(); ++a) e += (leaves[t].dims[a] - 1) * leaves[t].strides[a];
    extent[t] = e;
    for (auto& ps : ex->leaf_slice[t]) slice_max[t] += (ex->slice_dims[ps.first] - 1) * ps.second;
  }
  for (size_t s = 0; s < plan.steps.size(); ++s) extent[plan.steps[s].out] = tsize(plan.steps[s].out);
  auto inside = [&](int t, int64_t off) { return off + slice_max[t] < extent[t]; };

  Arena arena;
  std::map<int, std::pair<size_t, size_t>> where;  // intermediate id -> (offset, bytes)
  size_t split_need = 0;
  ex->steps.clear();
  ex->n_tc_steps = 0;
  const int np = prec == 3 ? 3 : (prec == 2 ? 2 : 1);
  const int es = prec == 3 ? 2 : 4;
  for (size_t s = 0; s < plan.steps.size(); ++s) {
    const PlanStep& ps = plan.steps[s];
    StepExec e;
    e.x = ps.x;
    e.y = ps.y;
    e.out = ps.out;
    e.x_leaf = ps.x < nl;
    e.y_leaf = ps.y < nl;
    e.dtx = e.x_leaf ? leaves[ps.x].dt : DT_F64;
    e.dty = e.y_leaf ? leaves[ps.y].dt : DT_F64;
    e.last = (s + 1 == plan.steps.size());
    auto nsl = [&](const Inds& v) {
      Inds r;
      for (int64_t i : v)
        if (!sliced.count(i)) r.push_back(i);
      return r;
    };
    const Inds batch = nsl(ps.batch), m = nsl(ps.m), n = nsl(ps.n), k = nsl(ps.k), sa = nsl(ps.sa),
               sb = nsl(ps.sb);
    double nb = 1, nm = 1, nn = 1, nk = 1;
    for (int64_t i : batch) nb *= (double)dims.get(i);
    for (int64_t i : m) nm *= (double)dims.get(i);
    for (int64_t i : n) nn *= (double)dims.get(i);
    for (int64_t i : k) nk *= (double)dims.get(i);
    e.flops = 2.0 * nb * nm * nn * nk;
    const double lim = 2147483647.0;
    bool tc = prec != QTPU_PREC_FP64 && sa.empty() && sb.empty() && nm >= 64 && nn >= 32 && nk >= 32 &&
              nb * nm * nn * nk >= (double)(1 << 22) && nb < lim && nm < lim && nn < lim && nk < lim;
    if (tc) {
      SplitArgs A, B;
      memset(&A.row, 0, sizeof(ModeTab));
      memset(&A.k, 0, sizeof(ModeTab));
      memset(&B.row, 0, sizeof(ModeTab));
      memset(&B.k, 0, sizeof(ModeTab));
      bool ok = true;
      for (int64_t i : batch) ok &= push_mode(A.row, dims.get(i), sof(ps.x, i), 0);
      for (int64_t i : m) ok &= push_mode(A.row, dims.get(i), sof(ps.x, i), 0);
      for (int64_t i : k) ok &= push_mode(A.k, dims.get(i), sof(ps.x, i), 0);
      for (int64_t i : batch) ok &= push_mode(B.row, dims.get(i), sof(ps.y, i), 0);
      for (int64_t i : n) ok &= push_mode(B.row, dims.get(i), sof(ps.y, i), 0);
      for (int64_t i : k) ok &= push_mode(B.k, dims.get(i), sof(ps.y, i), 0);
      if (ok) {
        merge_modes(A.row);
        merge_modes(A.k);
        merge_modes(B.row);
        merge_modes(B.k);
        const int64_t K = (int64_t)nk, Kp = (int64_t)align_up((size_t)K, 8);
        A.n_rows = (int64_t)(nb * nm);
        B.n_rows = (int64_t)(nb * nn);
        A.K = B.K = K;
        A.Kp = B.Kp = Kp;
        A.pieces = B.pieces = np;
        A.kind = B.kind = prec == 3 ? 0 : 1;
        if (!inside(ps.x, max_off(A.row, 0) + max_off(A.k, 0)) ||
            !inside(ps.y, max_off(B.row, 0) + max_off(B.k, 0))) {
          *code = QTPU_ENOTSUP;
          return "internal: operand view out of bounds";
        }
        e.sa = A;
        e.sb = B;
        e.kind = SK_TC;
        e.g.batch = (int)nb;
        e.g.M = (int)nm;
        e.g.N = (int)nn;
        e.g.K = (int)K;
        e.g.prec = prec;
        e.g.kc_blocks = ex->kc_blocks;
        const size_t abytes = align_up((size_t)np * A.n_rows * Kp * es, 1024);
        const size_t bbytes = align_up((size_t)np * B.n_rows * Kp * es, 1024);
        split_need = std::max(split_need, abytes + bbytes);
        ex->n_tc_steps++;
      } else {
        tc = false;
      }
    }
    if (!tc) {
      e.kind = SK_GENERIC;
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
      if (!ok) {
        *code = QTPU_ENOTSUP;
        return "a step has more than 12 modes in one group";
      }
      merge_modes(c.out);
      merge_modes(c.loop);
      c.n_out = tab_size(c.out);
      c.n_loop = tab_size(c.loop);
      if (!inside(ps.x, max_off(c.out, 0) + max_off(c.loop, 0)) ||
          !inside(ps.y, max_off(c.out, 1) + max_off(c.loop, 1)) || c.n_out != tsize(ps.out)) {
        *code = QTPU_ENOTSUP;
        return "internal: operand view out of bounds";
      }
      e.c = c;
    }
    // output placement
    const size_t obytes = (size_t)tsize(ps.out) * 8;
    if (!e.last) {
      e.out_off = arena.alloc(obytes);
      where[ps.out] = {e.out_off, obytes};
    }
    for (int t : {ps.x, ps.y})
      if (t >= nl) {
        arena.release(where[t].first, where[t].second);
        where.erase(t);
      }
    ex->steps.push_back(e);
  }

  // final reduction: slices and leftover indices -> output order
  ContractArgs r;
  memset(&r.out, 0, sizeof(ModeTab));
  memset(&r.loop, 0, sizeof(ModeTab));
  bool ok = true;
  if (plan.steps.empty()) {
    ex->reduce_from_leaf = true;
    ex->reduce_leaf = 0;
    const Leaf& L = leaves[0];
    for (int64_t i : plan.output) {
      size_t a = std::find(L.ids.begin(), L.ids.end(), i) - L.ids.begin();
      ok &= push_mode(r.out, L.dims[a], L.strides[a], 0);
    }
    for (size_t a = 0; a < L.ids.size(); ++a)
      if (!contains(plan.output, L.ids[a])) ok &= push_mode(r.loop, L.dims[a], L.strides[a], 0);
    ex->final_size = 0;
  } else {
    ex->reduce_from_leaf = false;
    const int last = plan.steps.back().out;
    ex->final_size = tsize(last);
    for (int64_t i : plan.output) ok &= push_mode(r.out, dims.get(i), sof(last, i), 0);
    ok &= push_mode(r.loop, ex->n_slices, ex->final_size, 0);
    for (int64_t i : plan.final_sum)
      if (!sliced.count(i)) ok &= push_mode(r.loop, dims.get(i), sof(last, i), 0);
  }
  if (!ok) {
    *code = QTPU_ENOTSUP;
    return "the output has more than 12 modes";
  }
  merge_modes(r.out);
  merge_modes(r.loop);
  r.n_out = tab_size(r.out);
  r.n_loop = tab_size(r.loop);
  {
    const int64_t src_extent = plan.steps.empty() ? extent[0] : ex->n_slices * ex->final_size;
    if (max_off(r.out, 0) + max_off(r.loop, 0) >= src_extent) {
      *code = QTPU_ENOTSUP;
      return "internal: reduction view out of bounds";
    }
  }
  ex->reduce = r;

  // device memory
  cudaError_t ce = cudaSetDevice(ex->device);
  if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&ex->sm_count, cudaDevAttrMultiProcessorCount, ex->device);
  if (ce != cudaSuccess) {
    *code = QTPU_ECUDA;
    return std::string("cuda: ") + cudaGetErrorString(ce);
  }
  ex->arena_bytes = std::max<size_t>(arena.top, 256);
  ex->split_bytes = split_need;
  auto dalloc = [&](void** p, size_t n) -> bool {
    if (!n) return true;
    if (cudaMalloc(p, n) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    return true;
  };
  if (!dalloc((void**)&ex->arena, ex->arena_bytes) || !dalloc((void**)&ex->splitbuf, ex->split_bytes) ||
      !dalloc((void**)&ex->partial, (size_t)ex->n_slices * std::max<int64_t>(ex->final_size, 1) * 8) ||
      !dalloc((void**)&ex->status, 16) || !dalloc((void**)&ex->out_stage, (size_t)r.n_out * 8)) {
    exec_free(ex);
    *code = QTPU_ENOMEM;
    return "device workspace allocation failed";
  }
  cudaMemset(ex->status, 0, 16);
  // tensor maps of the split buffers (fixed addresses)
  for (auto& e : ex->steps) {
    if (e.kind != SK_TC) continue;
    const size_t abytes = align_up((size_t)np * e.sa.n_rows * e.sa.Kp * es, 1024);
    if (!make_operand_map(&e.g.tmA, ex->splitbuf, prec, e.g.batch, e.g.M, e.g.K, e.sa.Kp, 128) ||
        !make_operand_map(&e.g.tmB, ex->splitbuf + abytes, prec, e.g.batch, e.g.N, e.g.K, e.sb.Kp,
                          gemm_block_n())) {
      exec_free(ex);
      *code = QTPU_ECUDA;
      return "cuTensorMapEncodeTiled failed";
    }
    e.g.status = ex->status;
  }
  return "";
}

static size_t dt_size(int dt) { return dt == DT_F64 ? 8 : 4; }

std::string exec_run(Executor* ex, const std::vector<Leaf>& leaves, double* dev_out, cudaStream_t st, int* code) {
  *code = QTPU_OK;
  const int nl = (int)leaves.size();
  std::vector<int64_t> loff(nl, 0);
  std::vector<int64_t> digit(ex->slice_dims.size(), 0);
  cudaError_t ce = cudaSuccess;
  if (!ex->reduce_from_leaf) {
    for (int64_t s = 0; s < ex->n_slices && ce == cudaSuccess; ++s) {
      int64_t r = s;
      for (int j = (int)ex->slice_dims.size() - 1; j >= 0; --j) {
        digit[j] = r % ex->slice_dims[j];
        r /= ex->slice_dims[j];
      }
      for (int t = 0; t < nl; ++t) {
        int64_t o = 0;
        for (auto& ps : ex->leaf_slice[t]) o += digit[ps.first] * ps.second;
        loff[t] = o;
      }
      for (auto& e : ex->steps) {
        const void* A = e.x_leaf ? (const void*)((const uint8_t*)leaves[e.x].ptr + loff[e.x] * dt_size(e.dtx))
                                 : nullptr;
        const void* B = e.y_leaf ? (const void*)((const uint8_t*)leaves[e.y].ptr + loff[e.y] * dt_size(e.dty))
                                 : nullptr;
        if (!e.x_leaf) A = ex->arena + ex->steps[e.x - nl].out_off;
        if (!e.y_leaf) B = ex->arena + ex->steps[e.y - nl].out_off;
        double* out = e.last ? ex->partial + s * ex->final_size : (double*)(ex->arena + e.out_off);
        if (e.kind == SK_GENERIC) {
          ce = launch_contract(A, e.dtx, B, e.dty, out, e.c, ex->sm_count, st);
        } else {
          const int np = ex->prec == 3 ? 3 : (ex->prec == 2 ? 2 : 1);
          const int es = ex->prec == 3 ? 2 : 4;
          const size_t abytes = align_up((size_t)np * e.sa.n_rows * e.sa.Kp * es, 1024);
          ce = launch_split(A, e.dtx, ex->splitbuf, e.sa, ex->sm_count, st);
          if (ce == cudaSuccess) ce = launch_split(B, e.dty, ex->splitbuf + abytes, e.sb, ex->sm_count, st);
          if (ce == cudaSuccess) {
            GemmArgs g = e.g;
            g.C = out;
            ce = launch_gemm(g, ex->sm_count, st);
          }
        }
        if (ce != cudaSuccess) break;
      }
    }
  }
  if (ce == cudaSuccess) {
    if (ex->reduce_from_leaf)
      ce = launch_contract(leaves[ex->reduce_leaf].ptr, leaves[ex->reduce_leaf].dt, nullptr, DT_F64, dev_out,
                           ex->reduce, ex->sm_count, st);
    else
      ce = launch_contract(ex->partial, DT_F64, nullptr, DT_F64, dev_out, ex->reduce, ex->sm_count, st);
  }
  if (ce != cudaSuccess) {
    *code = QTPU_ECUDA;
    return std::string("launch failed: ") + cudaGetErrorString(ce);
  }
  return "";
}

void exec_free(Executor* ex) {
  if (ex->arena) cudaFree(ex->arena);
  if (ex->splitbuf) cudaFree(ex->splitbuf);
  if (ex->partial) cudaFree(ex->partial);
  if (ex->status) cudaFree(ex->status);
  if (ex->out_stage) cudaFree(ex->out_stage);
  ex->out_stage = nullptr;
  ex->arena = ex->splitbuf = nullptr;
  ex->partial = nullptr;
  ex->status = nullptr;
}

}  // namespace qtpu
