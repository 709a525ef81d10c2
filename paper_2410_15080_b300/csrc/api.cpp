// C ABI of the h-TN contraction library (declared in include/qtpu_htn.h).
//
// Holds the network description (borrowed device tensors with their index
// ids), runs the host planner, and hands the plan to the executor.  Every
// entry point validates its arguments and returns a status; messages are
// kept per handle.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <vector>

#include "../../include/qtpu_htn.h"
#include "exec.h"
#include "knit.h"
#include "qpd.h"
#include "planner.h"

using namespace qtpu;

struct qtpu_htn {
  int device = -1;
  cudaStream_t stream = nullptr;
  bool host_only = true;
  std::vector<Leaf> leaves;
  Inds output;
  DimMap dims;
  bool planned = false;
  Plan plan;
  qtpu_plan_opts opts{};
  Executor ex;
  bool built = false;
  std::string err;
  // contract_host: a copy stream for the leaf uploads, one event per leaf,
  // and an event that orders the uploads after earlier work on the stream
  cudaStream_t up_stream = nullptr;
  std::vector<cudaEvent_t> leaf_ev;
  cudaEvent_t up_start = nullptr;
  // a network made by qtpu_htn_qpd_sample: the device memory it owns (its
  // fused CTs, truncated QTs and sampling scratch) and, per group, the fused
  // length before sampling and the values kept
  std::vector<void*> owned;
  std::vector<std::pair<int64_t, int64_t>> qpd;
};

// message of the last failed create or allocation-free call, per thread
static thread_local std::string g_create_err = "no error";

namespace qtpu {
void set_global_error(const char* msg) { g_create_err = msg ? msg : "no error"; }
}  // namespace qtpu

static qtpu_status fail(qtpu_htn* h, qtpu_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

namespace {
// QPD sampling groups (section 4.3): the gate-cut CTs (rank 1, kind CT,
// index on exactly two QTs and nothing else, not an output index) between
// the same QT pair, pairs ascending, CTs ascending within a pair.
struct QpdGroupHost {
  int qa = -1, qb = -1;
  std::vector<int> cts;
  std::vector<int64_t> ids, dims;
  int64_t D = 1;
};
// Device memory of sampled networks comes from one stream-ordered pool per
// device that keeps freed memory (release threshold: never), so repeated
// sampling reuses it instead of mapping fresh pages on every call.
cudaMemPool_t qpd_pool(int dev) {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  if (dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> g(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = p;
  }
  return pools[dev];
}

std::vector<QpdGroupHost> qpd_groups_of(const qtpu_htn* h) {
  std::map<int64_t, std::vector<int>> carriers;
  for (size_t t = 0; t < h->leaves.size(); ++t)
    for (int64_t i : h->leaves[t].ids) carriers[i].push_back((int)t);
  const std::set<int64_t> outs(h->output.begin(), h->output.end());
  std::map<std::pair<int, int>, QpdGroupHost> by_pair;
  for (size_t t = 0; t < h->leaves.size(); ++t) {
    const Leaf& L = h->leaves[t];
    if (L.kind != QTPU_CT || L.ids.size() != 1 || outs.count(L.ids[0])) continue;
    std::vector<int> others;
    for (int u : carriers[L.ids[0]])
      if (u != (int)t) others.push_back(u);
    if (others.size() != 2 || h->leaves[others[0]].kind != QTPU_QT || h->leaves[others[1]].kind != QTPU_QT) continue;
    const int a = std::min(others[0], others[1]), b = std::max(others[0], others[1]);
    QpdGroupHost& G = by_pair[{a, b}];
    G.qa = a, G.qb = b;
    G.cts.push_back((int)t);
    G.ids.push_back(L.ids[0]);
    G.dims.push_back(L.dims[0]);
    G.D *= L.dims[0];
  }
  std::vector<QpdGroupHost> out;
  for (auto& kv : by_pair) out.push_back(kv.second);
  return out;
}
}  // namespace

extern "C" {

qtpu_status qtpu_htn_create(qtpu_htn** out, int device, void* cuda_stream) {
  if (!out) {
    g_create_err = "out is NULL";
    return QTPU_EINVAL;
  }
  *out = nullptr;
  qtpu_htn* h = new (std::nothrow) qtpu_htn();
  if (!h) {
    g_create_err = "host allocation failed";
    return QTPU_ENOMEM;
  }
  h->device = device;
  h->stream = (cudaStream_t)cuda_stream;
  h->host_only = device < 0;
  if (!h->host_only) {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || device >= n) {
      cudaGetLastError();
      g_create_err = std::string("device ") + std::to_string(device) + " not available: " +
                     (e != cudaSuccess ? cudaGetErrorString(e) : "index out of range");
      delete h;
      return QTPU_ECUDA;
    }
    e = cudaSetDevice(device);
    if (e != cudaSuccess) {
      g_create_err = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
      delete h;
      return QTPU_ECUDA;
    }
    h->ex.device = device;
    h->ex.stream = h->stream;
  }
  *out = h;
  return QTPU_OK;
}

qtpu_status qtpu_htn_add_tensor(qtpu_htn* h, qtpu_kind kind, int rank, const int64_t* index_ids,
                                const int64_t* dims, qtpu_dtype dtype, const void* dev_ptr,
                                const int64_t* strides, int* tensor_id) {
  if (!h) return QTPU_EINVAL;
  if (h->planned) return fail(h, QTPU_ESTATE, "add_tensor after plan");
  if (kind != QTPU_QT && kind != QTPU_CT) return fail(h, QTPU_EINVAL, "bad kind");
  if (rank < 0 || rank > 16) return fail(h, QTPU_EINVAL, "rank must be 0..16");
  if (rank > 0 && (!index_ids || !dims)) return fail(h, QTPU_EINVAL, "index_ids/dims NULL");
  if (dtype != QTPU_F32 && dtype != QTPU_F64) return fail(h, QTPU_EINVAL, "bad dtype");
  if (!dev_ptr && !h->host_only) return fail(h, QTPU_EINVAL, "dev_ptr NULL");
  Leaf L;
  std::set<int64_t> seen;
  for (int a = 0; a < rank; ++a) {
    if (index_ids[a] < 0) return fail(h, QTPU_EINVAL, "negative index id");
    if (dims[a] < 1) return fail(h, QTPU_EINVAL, "dim < 1");
    if (!seen.insert(index_ids[a]).second) return fail(h, QTPU_EINVAL, "repeated index id within a tensor");
    int64_t d = h->dims.get(index_ids[a]);
    if (d >= 0 && d != dims[a])
      return fail(h, QTPU_EINVAL,
                  "index " + std::to_string(index_ids[a]) + ": dim " + std::to_string(dims[a]) +
                      " != " + std::to_string(d));
    if (strides && strides[a] < 0) return fail(h, QTPU_EINVAL, "negative stride");
  }
  for (int a = 0; a < rank; ++a) h->dims.set(index_ids[a], dims[a]);
  L.ids.assign(index_ids, index_ids + rank);
  L.dims.assign(dims, dims + rank);
  L.strides.resize(rank);
  int64_t st = 1;
  for (int a = rank - 1; a >= 0; --a) {
    L.strides[a] = strides ? strides[a] : st;
    st *= dims[a];
  }
  L.dt = dtype == QTPU_F64 ? DT_F64 : DT_F32;
  L.ptr = dev_ptr;
  L.kind = kind;
  h->leaves.push_back(L);
  if (tensor_id) *tensor_id = (int)h->leaves.size() - 1;
  return QTPU_OK;
}

qtpu_status qtpu_htn_set_output(qtpu_htn* h, int n, const int64_t* index_ids) {
  if (!h) return QTPU_EINVAL;
  if (h->planned) return fail(h, QTPU_ESTATE, "set_output after plan");
  if (n < 0 || (n > 0 && !index_ids)) return fail(h, QTPU_EINVAL, "bad output list");
  std::set<int64_t> seen;
  for (int a = 0; a < n; ++a)
    if (!seen.insert(index_ids[a]).second) return fail(h, QTPU_EINVAL, "repeated output id");
  h->output.assign(index_ids, index_ids + n);
  return QTPU_OK;
}

qtpu_status qtpu_htn_plan(qtpu_htn* h, const qtpu_plan_opts* opts) {
  if (!h) return QTPU_EINVAL;
  if (h->planned) return fail(h, QTPU_ESTATE, "already planned");
  if (h->leaves.empty()) return fail(h, QTPU_ESTATE, "plan before any tensor");
  qtpu_plan_opts o{};
  o.prec = QTPU_PREC_BF16X3;
  if (opts) o = *opts;
  if (o.prec < QTPU_PREC_FP64 || o.prec > QTPU_PREC_BF16X3) return fail(h, QTPU_EINVAL, "bad precision");
  if (o.cost_model != 0 && o.cost_model != 1) return fail(h, QTPU_EINVAL, "cost_model must be 0 or 1");
  if (o.search > 2) return fail(h, QTPU_EINVAL, "search must be 0, 1 or 2");
  if (o.search && o.cost_model) return fail(h, QTPU_EINVAL, "search and cost_model exclude each other");
  if (o.cost_model == 1 && h->host_only)
    return fail(h, QTPU_ENOTSUP, "the learned cost model runs its perceptron on the device");
  for (int64_t i : h->output)
    if (!h->dims.has(i)) return fail(h, QTPU_EINVAL, "output index " + std::to_string(i) + " is on no tensor");
  // GEMM tile table: the given file (it must load), or the measured table
  // beside the library when there is one ("" = the padding rule alone)
  TileTable tiles;
  {
    const bool given = o.autotune_table != nullptr;
    const std::string tp = given ? std::string(o.autotune_table) : default_tile_table_path();
    if (!tp.empty()) {
      FILE* fp = std::fopen(tp.c_str(), "r");
      if (fp) std::fclose(fp);
      if (fp || given) {
        const std::string m = load_tile_table(tp, &tiles);
        if (!m.empty()) return fail(h, QTPU_EINVAL, m);
      }
    }
  }
  std::vector<Inds> li;
  for (auto& L : h->leaves) li.push_back(L.ids);
  int r;
  if (o.cost_model == 1) {
    std::string err;
    const int st = plan_by_cost_model(li, h->dims, h->output, o, h->leaves, h->device, (void*)h->stream, &tiles,
                                      &h->plan, &err);
    if (st != QTPU_OK) return fail(h, (qtpu_status)st, err);
    r = PLAN_OK;
  } else if (o.search == 1) {
    std::string err;
    const int st = plan_hyper(li, h->dims, h->output, o, h->leaves, &tiles, &h->plan, &err);
    if (st != QTPU_OK) return fail(h, (qtpu_status)st, err);
    r = PLAN_OK;
  } else if (o.search == 2) {
    r = make_plan_exact(li, h->dims, h->output, o.max_intermediate_bytes, o.n_slices, o.slice_dim, &h->plan);
    if (r == PLAN_TOO_MANY)
      return fail(h, QTPU_ENOTSUP, "exact search: more than 16 tensors after absorption, 128 indices or 2^126");
  } else if (o.n_candidates > 1) {
    uint64_t chosen = 0;
    r = make_plan_best(li, h->dims, h->output, o.max_intermediate_bytes, o.n_slices, o.slice_dim, o.seed,
                       o.n_candidates, &h->plan, &chosen);
  } else {
    r = make_plan(li, h->dims, h->output, o.max_intermediate_bytes, o.n_slices, o.slice_dim, &h->plan, o.seed);
  }
  if (r == PLAN_OVERFLOW) return fail(h, QTPU_ENOTSUP, "a contraction size reaches 2^255");
  if (r == PLAN_LIMIT) return fail(h, QTPU_ELIMIT, "the peak-intermediate limit cannot be met by slicing");
  h->opts = o;
  {
    // a host-only handle lowers the plan too (no device work), so its
    // launch list can be inspected
    int code = QTPU_OK;
    std::string m =
        exec_build(&h->ex, h->plan, h->leaves, h->dims, (int)o.prec, &code, h->host_only, o.reuse_bytes, &tiles);
    if (code != QTPU_OK && !h->host_only) return fail(h, (qtpu_status)code, m);
    if (code != QTPU_OK) h->ex.lowered = false;  // planning still succeeded
    h->built = !h->host_only;
  }
  h->planned = true;
  return QTPU_OK;
}

qtpu_status qtpu_htn_autotune(qtpu_htn* h, int device, const char* table_path, int reps, int* n_problems) {
  if (!h) return QTPU_EINVAL;
  if (n_problems) *n_problems = 0;
  if (!table_path || !*table_path) return fail(h, QTPU_EINVAL, "table_path is NULL or empty");
  if (reps < 1 || reps > 1000) return fail(h, QTPU_EINVAL, "reps outside 1..1000");
  if (!h->planned) return fail(h, QTPU_ESTATE, "autotune before plan");
  if (device < 0 && h->host_only) return fail(h, QTPU_ENOTSUP, "host-only handle: give a device to time on");
  if (!h->ex.lowered) return fail(h, QTPU_ESTATE, "no lowered plan");
  cudaError_t e = cudaSetDevice(device < 0 ? h->device : device);
  if (e != cudaSuccess) return fail(h, QTPU_ECUDA, cudaGetErrorString(e));
  TileTable t;
  FILE* fp = std::fopen(table_path, "r");
  if (fp) {
    std::fclose(fp);
    const std::string m = load_tile_table(table_path, &t);
    if (!m.empty()) return fail(h, QTPU_EINVAL, m);
  }
  int n = 0, code = QTPU_OK;
  std::string m = exec_autotune(&h->ex, reps, &t, &n, &code);
  if (code != QTPU_OK) return fail(h, (qtpu_status)code, m);
  m = save_tile_table(table_path, t);
  if (!m.empty()) return fail(h, QTPU_EINVAL, m);
  if (n_problems) *n_problems = n;
  return QTPU_OK;
}

qtpu_status qtpu_htn_qpd_groups(const qtpu_htn* h, int* n_groups) {
  if (!h || !n_groups) return QTPU_EINVAL;
  *n_groups = (int)qpd_groups_of(h).size();
  return QTPU_OK;
}

qtpu_status qtpu_htn_qpd_sample(const qtpu_htn* h, uint64_t s_qpd, const double* dev_uniforms, qtpu_htn** out) {
  if (!out) return QTPU_EINVAL;
  *out = nullptr;
  if (!h) return QTPU_EINVAL;
  qtpu_htn* hs = const_cast<qtpu_htn*>(h);  // only its error message is written
  if (h->host_only) return fail(hs, QTPU_ENOTSUP, "host-only handle cannot sample");
  if (s_qpd < 1 || s_qpd > (1ull << 32)) return fail(hs, QTPU_EINVAL, "s_qpd outside 1..2^32");
  const std::vector<QpdGroupHost> gs = qpd_groups_of(h);
  const int ng = (int)gs.size();
  if (ng > 0 && !dev_uniforms) return fail(hs, QTPU_EINVAL, "dev_uniforms NULL");
  int64_t total = 0, maxD = 0;
  for (const QpdGroupHost& G : gs) {
    if ((int)G.cts.size() > kQpdMaxCts) return fail(hs, QTPU_ENOTSUP, "more than 8 gate cuts between two QTs");
    if (G.D > 0x7FFFFFFF) return fail(hs, QTPU_ENOTSUP, "fused CT of 2^31 entries or more");
    total += G.D;
    maxD = std::max(maxD, G.D);
  }
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return fail(hs, QTPU_ECUDA, cudaGetErrorString(e));
  qtpu_htn* nh = new (std::nothrow) qtpu_htn();
  if (!nh) return fail(hs, QTPU_ENOMEM, "host allocation failed");
  nh->device = h->device;
  nh->stream = h->stream;
  nh->host_only = false;
  nh->output = h->output;
  cudaStream_t st = h->stream;
  auto bail = [&](cudaError_t x, const char* what) {
    cudaGetLastError();
    qtpu_htn_destroy(nh);
    return fail(hs, x == cudaErrorMemoryAllocation ? QTPU_ENOMEM : QTPU_ECUDA,
                std::string("qpd_sample: ") + what + ": " + cudaGetErrorString(x));
  };
  cudaMemPool_t pool = qpd_pool(h->device);
  if (!pool) {
    qtpu_htn_destroy(nh);
    return fail(hs, QTPU_ECUDA, "qpd_sample: memory pool");
  }
  auto dalloc = [&](size_t bytes, void** p) {
    *p = nullptr;
    cudaError_t x = cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 16), pool, st);
    if (x == cudaSuccess) nh->owned.push_back(*p);
    return x;
  };
  // scratch: groups, fused values, prefix sums, gamma, counts, kept values
  // and coefficients, kept counts (8-byte fields first)
  const size_t n8 = (size_t)std::max<int64_t>(total, 1);
  const size_t off_groups = 0, off_fused = (sizeof(QpdGroup) * std::max(ng, 1) + 255) / 256 * 256;
  const size_t off_prefix = off_fused + n8 * 8, off_gamma = off_prefix + n8 * 8;
  const size_t off_keptct = off_gamma + std::max(ng, 1) * 8, off_counts = off_keptct + n8 * 8;
  const size_t off_keptidx = off_counts + n8 * 4, off_nkept = off_keptidx + n8 * 4;
  const size_t scratch_bytes = off_nkept + std::max(ng, 1) * 4;
  void* scratch = nullptr;
  if ((e = dalloc(scratch_bytes, &scratch)) != cudaSuccess) return bail(e, "scratch");
  uint8_t* sb = (uint8_t*)scratch;
  QpdGroup* d_groups = (QpdGroup*)(sb + off_groups);
  double* fused = (double*)(sb + off_fused);
  double* prefix = (double*)(sb + off_prefix);
  double* gamma = (double*)(sb + off_gamma);
  double* kept_ct = (double*)(sb + off_keptct);
  uint32_t* counts = (uint32_t*)(sb + off_counts);
  int32_t* kept_idx = (int32_t*)(sb + off_keptidx);
  int32_t* n_kept = (int32_t*)(sb + off_nkept);
  std::vector<QpdGroup> hg(ng);
  int64_t base = 0;
  for (int x = 0; x < ng; ++x) {
    QpdGroup& G = hg[x];
    G.n_ct = (int)gs[x].cts.size();
    G.D = gs[x].D;
    G.base = base;
    base += G.D;
    for (int j = 0; j < G.n_ct; ++j) {
      const Leaf& L = h->leaves[gs[x].cts[j]];
      G.ct[j] = L.ptr;
      G.dt[j] = L.dt;
      G.dim[j] = L.dims[0];
      G.stride[j] = L.strides[0];
    }
  }
  std::vector<int32_t> kept(ng, 0);
  if (ng > 0) {
    if ((e = cudaMemcpyAsync(d_groups, hg.data(), sizeof(QpdGroup) * ng, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return bail(e, "group upload");
    if ((e = cudaMemsetAsync(counts, 0, (size_t)total * 4, st)) != cudaSuccess) return bail(e, "counts");
    if ((e = qpd_fuse(d_groups, ng, maxD, fused, st)) != cudaSuccess) return bail(e, "fuse");
    if ((e = qpd_draw(d_groups, ng, fused, prefix, gamma, dev_uniforms, s_qpd, counts, st)) != cudaSuccess)
      return bail(e, "draw");
    if ((e = qpd_compact(d_groups, ng, fused, gamma, counts, s_qpd, kept_idx, kept_ct, n_kept, st)) != cudaSuccess)
      return bail(e, "compact");
    // the kept counts fix the new shapes
    if ((e = cudaMemcpyAsync(kept.data(), n_kept, (size_t)ng * 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return bail(e, "kept counts");
  }
  int sm = 148;
  cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, h->device);
  int64_t max_id = -1;
  for (const Leaf& L : h->leaves)
    for (int64_t i : L.ids) max_id = std::max(max_id, i);
  std::set<int> dropped;
  for (const QpdGroupHost& G : gs) dropped.insert(G.cts.begin(), G.cts.end());
  for (size_t t = 0; t < h->leaves.size(); ++t) {
    if (dropped.count((int)t)) continue;
    const Leaf& L = h->leaves[t];
    std::vector<int> mine;
    for (int x = 0; x < ng; ++x)
      if (gs[x].qa == (int)t || gs[x].qb == (int)t) mine.push_back(x);
    if (mine.empty()) {
      nh->leaves.push_back(L);  // borrowed
      continue;
    }
    // the axis list of the truncated copy: groups applied in order, each
    // group's axes replaced by its fused axis at the first of their places
    struct Ax {
      int64_t id, dim, stride;
      int group;
    };
    std::vector<Ax> ax;
    for (size_t a = 0; a < L.ids.size(); ++a) ax.push_back({L.ids[a], L.dims[a], L.strides[a], -1});
    for (int x : mine) {
      std::vector<size_t> pos;
      for (int64_t id : gs[x].ids)
        for (size_t a = 0; a < ax.size(); ++a)
          if (ax[a].group < 0 && ax[a].id == id) pos.push_back(a);
      const size_t first = *std::min_element(pos.begin(), pos.end());
      std::vector<Ax> nx;
      for (size_t a = 0; a < ax.size(); ++a) {
        if (a == first) nx.push_back({max_id + 1 + x, kept[x], 0, x});
        if (std::find(pos.begin(), pos.end(), a) == pos.end()) nx.push_back(ax[a]);
      }
      ax = nx;
    }
    QpdGather g;
    g.src = L.ptr;
    g.dt = L.dt;
    g.n_axes = (int)ax.size();
    g.n_out = 1;
    for (size_t a = 0; a < ax.size(); ++a) {
      g.dim[a] = ax[a].dim;
      g.stride[a] = ax[a].stride;
      g.n_out *= ax[a].dim;
      if (ax[a].group < 0) continue;
      const int x = ax[a].group;
      std::vector<int64_t> qstride;
      for (int64_t id : gs[x].ids)
        for (size_t b = 0; b < L.ids.size(); ++b)
          if (L.ids[b] == id) qstride.push_back(L.strides[b]);
      void* tab = nullptr;
      if ((e = dalloc((size_t)kept[x] * 8, &tab)) != cudaSuccess) return bail(e, "table");
      if ((e = qpd_table((int)gs[x].dims.size(), gs[x].dims.data(), qstride.data(), kept_idx + hg[x].base, kept[x],
                         (int64_t*)tab, st)) != cudaSuccess)
        return bail(e, "table");
      g.table[a] = (const int64_t*)tab;
    }
    void* dst = nullptr;
    if ((e = dalloc((size_t)g.n_out * (L.dt == DT_F64 ? 8 : 4), &dst)) != cudaSuccess) return bail(e, "QT copy");
    g.dst = dst;
    if ((e = qpd_gather(g, sm, st)) != cudaSuccess) return bail(e, "gather");
    Leaf N;
    N.kind = L.kind;
    N.dt = L.dt;
    N.ptr = dst;
    int64_t stc = 1;
    N.strides.assign(ax.size(), 1);
    for (int a = (int)ax.size() - 1; a >= 0; --a) N.strides[a] = stc, stc *= ax[a].dim;
    for (const Ax& a : ax) N.ids.push_back(a.id), N.dims.push_back(a.dim);
    nh->leaves.push_back(N);
  }
  for (int x = 0; x < ng; ++x) {
    Leaf C;
    C.kind = QTPU_CT;
    C.dt = DT_F64;
    C.ptr = kept_ct + hg[x].base;
    C.ids = {max_id + 1 + x};
    C.dims = {(int64_t)kept[x]};
    C.strides = {1};
    nh->leaves.push_back(C);
    nh->qpd.push_back({gs[x].D, (int64_t)kept[x]});
  }
  for (const Leaf& L : nh->leaves)
    for (size_t a = 0; a < L.ids.size(); ++a) nh->dims.set(L.ids[a], L.dims[a]);
  *out = nh;
  return QTPU_OK;
}

qtpu_status qtpu_htn_qpd_info(const qtpu_htn* h, int max, int64_t* dim_before, int64_t* dim_kept, int* n_groups) {
  if (!h || !n_groups || max < 0 || (max > 0 && (!dim_before || !dim_kept))) return QTPU_EINVAL;
  *n_groups = (int)h->qpd.size();
  for (int x = 0; x < max && x < (int)h->qpd.size(); ++x) dim_before[x] = h->qpd[x].first, dim_kept[x] = h->qpd[x].second;
  return QTPU_OK;
}

qtpu_status qtpu_htn_tensor_info(const qtpu_htn* h, int t, int max_rank, int* rank, int64_t* index_ids,
                                 int64_t* dims, int64_t* strides, qtpu_dtype* dtype, qtpu_kind* kind,
                                 const void** dev_ptr) {
  if (!h || !rank) return QTPU_EINVAL;
  if (t < 0 || t >= (int)h->leaves.size()) return QTPU_EINVAL;
  const Leaf& L = h->leaves[t];
  *rank = (int)L.ids.size();
  if (max_rank < *rank && (index_ids || dims || strides)) return QTPU_EINVAL;
  for (int a = 0; a < *rank; ++a) {
    if (index_ids) index_ids[a] = L.ids[a];
    if (dims) dims[a] = L.dims[a];
    if (strides) strides[a] = L.strides[a];
  }
  if (dtype) *dtype = L.dt == DT_F64 ? QTPU_F64 : QTPU_F32;
  if (kind) *kind = (qtpu_kind)L.kind;
  if (dev_ptr) *dev_ptr = L.ptr;
  return QTPU_OK;
}

qtpu_status qtpu_htn_knit_naive(qtpu_htn* h, double* dev_out, double* n_instances) {
  if (!h) return QTPU_EINVAL;
  if (n_instances) *n_instances = 0;
  if (h->host_only) return fail(h, QTPU_ENOTSUP, "host-only handle cannot contract");
  if (!dev_out) return fail(h, QTPU_EINVAL, "dev_out NULL");
  if (h->leaves.empty()) return fail(h, QTPU_ESTATE, "no tensors");
  if ((int)h->leaves.size() > kKnitMaxT) return fail(h, QTPU_ENOTSUP, "more than 32 tensors");
  for (int64_t i : h->output)
    if (!h->dims.has(i)) return fail(h, QTPU_EINVAL, "output index " + std::to_string(i) + " is on no tensor");
  const std::set<int64_t> outs(h->output.begin(), h->output.end());
  std::set<int64_t> summed;
  for (const Leaf& L : h->leaves)
    for (int64_t i : L.ids)
      if (!outs.count(i)) summed.insert(i);
  if ((int)summed.size() > kKnitMaxSum) return fail(h, QTPU_ENOTSUP, "more than 40 summed indices");
  if ((int)h->output.size() > kKnitMaxOut) return fail(h, QTPU_ENOTSUP, "more than 8 output indices");
  KnitTable T;
  T.n_t = (int)h->leaves.size();
  T.n_sum = (int)summed.size();
  T.n_outi = (int)h->output.size();
  double ninst = 1, nout = 1;
  for (int t = 0; t < T.n_t; ++t) T.ptr[t] = h->leaves[t].ptr, T.dt[t] = h->leaves[t].dt;
  auto strides_of = [&](int64_t id, int64_t* row) {
    for (int t = 0; t < T.n_t; ++t) {
      const Leaf& L = h->leaves[t];
      row[t] = 0;
      for (size_t a = 0; a < L.ids.size(); ++a)
        if (L.ids[a] == id) row[t] = L.strides[a];
    }
  };
  int m = 0;
  for (int64_t i : summed) {
    T.dim[m] = h->dims.get(i);
    ninst *= (double)T.dim[m];
    strides_of(i, T.stride[m]);
    ++m;
  }
  for (int a = 0; a < T.n_outi; ++a) {
    T.out_dim[a] = h->dims.get(h->output[a]);
    nout *= (double)T.out_dim[a];
    strides_of(h->output[a], T.out_stride[a]);
  }
  if (ninst >= 4.0e18 || nout > 65535) return fail(h, QTPU_ENOTSUP, "instance or output count too large");
  T.n_inst = (uint64_t)ninst;
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return fail(h, QTPU_ECUDA, cudaGetErrorString(e));
  int sm = 148;
  cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, h->device);
  // about 8 blocks per SM in all, at least 256 instances per block
  uint64_t chunks = (uint64_t)std::ceil(sm * 8.0 / nout);
  chunks = std::max<uint64_t>(1, std::min<uint64_t>(chunks, (T.n_inst + 255) / 256));
  cudaStream_t st = h->stream;
  KnitTable* dT = nullptr;
  double* part = nullptr;
  e = cudaMallocAsync((void**)&dT, sizeof(KnitTable), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&part, (size_t)nout * chunks * 8, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dT, &T, sizeof(KnitTable), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_knit(dT, T.n_inst, (uint64_t)nout, part, chunks, dev_out, st);
  // the table is copied from this stack frame: finish the copy before returning
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (dT) cudaFreeAsync(dT, st);
  if (part) cudaFreeAsync(part, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, e == cudaErrorMemoryAllocation ? QTPU_ENOMEM : QTPU_ECUDA,
                std::string("knit_naive: ") + cudaGetErrorString(e));
  }
  if (n_instances) *n_instances = ninst;
  return QTPU_OK;
}

qtpu_status qtpu_htn_num_tensors(const qtpu_htn* h, int* n) {
  if (!h || !n) return QTPU_EINVAL;
  *n = (int)h->leaves.size();
  return QTPU_OK;
}

qtpu_status qtpu_htn_plan_info(const qtpu_htn* h, char* buf, size_t len, size_t* needed) {
  if (!h) return QTPU_EINVAL;
  if (!h->planned) return QTPU_ESTATE;
  std::string t = plan_text(h->plan);
  if (needed) *needed = t.size() + 1;
  if (buf && len) {
    size_t n = std::min(len - 1, t.size());
    memcpy(buf, t.data(), n);
    buf[n] = 0;
  }
  return QTPU_OK;
}

qtpu_status qtpu_htn_lowering_info(const qtpu_htn* h, char* buf, size_t len, size_t* needed) {
  if (!h) return QTPU_EINVAL;
  if (!h->planned || !h->ex.lowered) return QTPU_ESTATE;
  std::string t = exec_describe(&h->ex);
  if (needed) *needed = t.size() + 1;
  if (buf && len) {
    size_t n = std::min(len - 1, t.size());
    memcpy(buf, t.data(), n);
    buf[n] = 0;
  }
  return QTPU_OK;
}

qtpu_status qtpu_htn_output_size(const qtpu_htn* h, int64_t* n) {
  if (!h || !n) return QTPU_EINVAL;
  int64_t s = 1;
  for (int64_t i : h->output) s *= h->dims.get(i);
  *n = s;
  return QTPU_OK;
}

qtpu_status qtpu_htn_plan_stats(const qtpu_htn* h, double* flops_total, int* n_steps, int* n_tc,
                                uint64_t* ws, int64_t* launches) {
  if (!h) return QTPU_EINVAL;
  if (!h->planned) return QTPU_ESTATE;
  if (launches) *launches = h->ex.lowered ? h->ex.launches_per_contract : 0;
  if (flops_total) *flops_total = h->plan.flops_total.to_double();
  if (n_steps) *n_steps = (int)h->plan.steps.size();
  if (n_tc) *n_tc = h->built ? h->ex.n_tc_steps : 0;
  if (ws) *ws = h->ex.lowered ? (uint64_t)h->ex.workspace_bytes() : 0;
  return QTPU_OK;
}

qtpu_status qtpu_htn_exec_stats(const qtpu_htn* h, double* flops_executed, double* flops_all_slices,
                                uint64_t* kept_bytes, int64_t* launches) {
  if (!h) return QTPU_EINVAL;
  if (!h->planned || !h->ex.lowered) return QTPU_ESTATE;
  if (flops_executed) *flops_executed = h->ex.flops_executed;
  if (flops_all_slices) *flops_all_slices = h->ex.flops_no_reuse;
  if (kept_bytes) *kept_bytes = (uint64_t)h->ex.kept_bytes;
  if (launches) *launches = h->ex.launches_per_contract;
  return QTPU_OK;
}

qtpu_status qtpu_htn_launch_features(const qtpu_htn* h, int max_rows, float* features, int64_t* launches,
                                     int* n_rows) {
  if (!h || max_rows < 0 || (max_rows > 0 && !features)) return QTPU_EINVAL;
  if (!h->planned || !h->ex.lowered) return QTPU_ESTATE;
  const int n = (int)h->ex.launches.size();
  if (n_rows) *n_rows = n;
  for (int i = 0; i < n && i < max_rows; ++i) {
    exec_launch_features(&h->ex, (size_t)i, features + (size_t)i * kLaunchFeatures);
    if (launches) launches[i] = h->ex.launches[i].n_launch;
  }
  return QTPU_OK;
}

qtpu_status qtpu_htn_profile_launches(qtpu_htn* h, int max, int* launch_index, double* ms, int* n) {
  if (!h || max < 0 || !n) return QTPU_EINVAL;
  if (h->host_only || !h->built) return fail(h, QTPU_ESTATE, "nothing to read");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess && h->ex.own) e = cudaStreamSynchronize(h->ex.own);
  if (e != cudaSuccess) return fail(h, QTPU_ECUDA, cudaGetErrorString(e));
  if ((size_t)max < h->ex.prof.used) {  // too small: report the count, keep the timings
    *n = (int)h->ex.prof.used;
    return QTPU_OK;
  }
  std::vector<int> idx;
  std::vector<double> t;
  std::string err = exec_profile_launches(&h->ex, &idx, &t);
  if (!err.empty()) return fail(h, QTPU_ECUDA, err);
  *n = (int)idx.size();
  for (int i = 0; i < *n && i < max; ++i) {
    if (launch_index) launch_index[i] = idx[i];
    if (ms) ms[i] = t[i];
  }
  return QTPU_OK;
}

qtpu_status qtpu_htn_contract(qtpu_htn* h, double* dev_out) {
  if (!h) return QTPU_EINVAL;
  if (!h->planned) return fail(h, QTPU_ESTATE, "contract before plan");
  if (h->host_only) return fail(h, QTPU_ENOTSUP, "host-only handle cannot contract");
  if (!dev_out) return fail(h, QTPU_EINVAL, "dev_out NULL");
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return fail(h, QTPU_ECUDA, cudaGetErrorString(e));
  int code = QTPU_OK;
  std::string m = exec_run(&h->ex, h->leaves, dev_out, h->stream, &code);
  if (code != QTPU_OK) return fail(h, (qtpu_status)code, m);
  return QTPU_OK;
}

qtpu_status qtpu_htn_contract_slices(qtpu_htn* h, int64_t first, int64_t count, double* dev_out) {
  if (!h) return QTPU_EINVAL;
  if (!h->planned) return fail(h, QTPU_ESTATE, "contract before plan");
  if (h->host_only) return fail(h, QTPU_ENOTSUP, "host-only handle cannot contract");
  if (!dev_out) return fail(h, QTPU_EINVAL, "dev_out NULL");
  if (first < 0 || count < 1 || first + count > h->ex.n_slices)
    return fail(h, QTPU_EINVAL, "slice range outside [0, n_slices)");
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return fail(h, QTPU_ECUDA, cudaGetErrorString(e));
  int code = QTPU_OK;
  std::string m = exec_run_slices(&h->ex, h->leaves, first, count, dev_out, h->stream, &code);
  if (code != QTPU_OK) return fail(h, (qtpu_status)code, m);
  return QTPU_OK;
}

qtpu_status qtpu_htn_sync(qtpu_htn* h) {
  if (!h) return QTPU_EINVAL;
  if (h->host_only || !h->built) return QTPU_OK;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(h, QTPU_ECUDA, cudaGetErrorString(e));
  if (h->ex.own) {
    e = cudaStreamSynchronize(h->ex.own);
    if (e != cudaSuccess) return fail(h, QTPU_ECUDA, cudaGetErrorString(e));
  }
  uint32_t st = 0;
  e = cudaMemcpy(&st, h->ex.status, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(h, QTPU_ECUDA, cudaGetErrorString(e));
  if (st) cudaMemset(h->ex.status, 0, 4);  // reported once
  if (st & (ST_TIMEOUT_TMA | ST_TIMEOUT_MMA | ST_TIMEOUT_EPI | ST_TIMEOUT_DEP))
    return fail(h, QTPU_ETIMEOUT, "a bounded device-side wait gave up (status 0x" + std::to_string(st) + ")");
  if (st) return fail(h, QTPU_ECUDA, "device status word " + std::to_string(st));
  return QTPU_OK;
}

qtpu_status qtpu_htn_contract_host(qtpu_htn* h, const void* const* host_ptrs, double* host_out) {
  if (!h) return QTPU_EINVAL;
  if (!h->planned) return fail(h, QTPU_ESTATE, "contract before plan");
  if (h->host_only) return fail(h, QTPU_ENOTSUP, "host-only handle cannot contract");
  if (!host_ptrs || !host_out) return fail(h, QTPU_EINVAL, "NULL host buffer");
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return fail(h, QTPU_ECUDA, cudaGetErrorString(e));
  for (size_t t = 0; t < h->leaves.size(); ++t)
    if (!host_ptrs[t]) return fail(h, QTPU_EINVAL, "NULL host buffer");
  const size_t nl = h->leaves.size();
  if (!h->up_stream) {
    e = cudaStreamCreateWithFlags(&h->up_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->up_start, cudaEventDisableTiming);
    for (size_t t = 0; t < nl && e == cudaSuccess; ++t) {
      cudaEvent_t ev;
      e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) h->leaf_ev.push_back(ev);
    }
    if (e != cudaSuccess) return fail(h, QTPU_ECUDA, cudaGetErrorString(e));
  }
  // The uploads run on a copy stream, leaf by leaf in the order the schedule
  // first reads them, after the work already enqueued on the handle's stream
  // (which may still read the device buffers); each launch of the
  // contraction waits only for the leaves it reads, so the contraction starts
  // while later leaves are still being copied.
  e = cudaEventRecord(h->up_start, h->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->up_stream, h->up_start, 0);
  for (int t : exec_leaf_order(&h->ex, (int)nl)) {
    if (e != cudaSuccess) break;
    const Leaf& L = h->leaves[t];
    int64_t n = 1;
    for (int64_t d : L.dims) n *= d;
    e = cudaMemcpyAsync((void*)L.ptr, host_ptrs[t], (size_t)n * (L.dt == DT_F64 ? 8 : 4), cudaMemcpyHostToDevice,
                        h->up_stream);
    if (e == cudaSuccess) e = cudaEventRecord(h->leaf_ev[t], h->up_stream);
  }
  if (e != cudaSuccess) return fail(h, QTPU_ECUDA, cudaGetErrorString(e));
  int64_t no = 1;
  qtpu_htn_output_size(h, &no);
  double* dout = h->ex.out_stage;  // allocated with the workspace by plan
  int code = QTPU_OK;
  std::string m = exec_run_host(&h->ex, h->leaves, dout, h->stream, h->leaf_ev.data(), &code);
  if (code != QTPU_OK) return fail(h, (qtpu_status)code, m);
  // every upload is done before the call returns (a leaf no launch reads too)
  for (size_t t = 0; t < nl && e == cudaSuccess; ++t) e = cudaStreamWaitEvent(h->stream, h->leaf_ev[t], 0);
  if (e != cudaSuccess) return fail(h, QTPU_ECUDA, cudaGetErrorString(e));
  e = cudaMemcpyAsync(host_out, dout, (size_t)no * 8, cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return fail(h, QTPU_ECUDA, cudaGetErrorString(e));
  return qtpu_htn_sync(h);
}

// ---------------------------------------------------------------- batches
// Many networks in one CUDA graph.  Networks whose launches are all gathers
// (unsliced) become tasks of one persistent kernel (batch.cu) on branch 0;
// every other network's launch sequence is captured on one of kBranches
// parallel streams (networks own disjoint workspaces, so they may run
// concurrently), followed by the copy of its output.  The graph is cached per
// (handles, outputs, options) and replayed with one graph launch.
namespace {
constexpr int kBranches = 16;
struct BatchGraph {
  std::vector<qtpu_htn*> hs;
  std::vector<double*> outs;
  int device = 0;
  int persistent = 1;
  uint64_t limit_ns = 0;
  int stall = -1;
  cudaGraphExec_t exec = nullptr;
  // persistent kernel: tasks, unit prefix, counters
  int n_tasks = 0, n_persistent = 0;
  BatchTask* d_tasks = nullptr;
  uint64_t* d_start = nullptr;
  unsigned long long* d_next = nullptr;
  uint32_t* d_done = nullptr;
  int* d_abort = nullptr;
};
struct BatchState {
  std::mutex mu;
  std::vector<BatchGraph*> cache;  // most recent last, at most 4
  cudaStream_t cap[64] = {};
  cudaStream_t br[64][kBranches] = {};
  cudaEvent_t fork[64] = {}, join[64][kBranches] = {}, in[64] = {}, out[64] = {};
};
BatchState g_batch;

void batch_free(BatchGraph* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (void* p : {(void*)b->d_tasks, (void*)b->d_start, (void*)b->d_next, (void*)b->d_done, (void*)b->d_abort})
    if (p) cudaFree(p);
  delete b;
}

bool batch_streams(int dev) {
  if (g_batch.cap[dev]) return true;
  if (cudaStreamCreateWithFlags(&g_batch.cap[dev], cudaStreamNonBlocking) != cudaSuccess) return false;
  for (int i = 0; i < kBranches; ++i) {
    if (cudaStreamCreateWithFlags(&g_batch.br[dev][i], cudaStreamNonBlocking) != cudaSuccess) return false;
    if (cudaEventCreateWithFlags(&g_batch.join[dev][i], cudaEventDisableTiming) != cudaSuccess) return false;
  }
  return cudaEventCreateWithFlags(&g_batch.fork[dev], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&g_batch.in[dev], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&g_batch.out[dev], cudaEventDisableTiming) == cudaSuccess;
}

// blocks of the persistent kernel per SM (QTPU_BATCH_BLOCKS_PER_SM overrides
// the default of 4, the fastest of 1, 2 and 4 measured on a batch of small
// networks)
int batch_grid(int sm) {
  int per = 4;
  if (const char* s = getenv("QTPU_BATCH_BLOCKS_PER_SM")) per = std::max(1, std::min(8, atoi(s)));
  return sm * per;
}

void batch_forget(qtpu_htn* h) {
  std::lock_guard<std::mutex> g(g_batch.mu);
  for (size_t i = 0; i < g_batch.cache.size();) {
    BatchGraph* b = g_batch.cache[i];
    if (std::find(b->hs.begin(), b->hs.end(), h) != b->hs.end()) {
      batch_free(b);
      g_batch.cache.erase(g_batch.cache.begin() + i);
    } else {
      ++i;
    }
  }
}

// The persistent kernel's tasks: level by level across the eligible networks
// (task l of every network, then l + 1, ...), each depending on the same
// network's previous task.  Returns a CUDA error; eligible[i] is set for the
// networks the kernel contracts.
cudaError_t batch_build_tasks(BatchGraph* b, qtpu_htn* const* hs, int n, double* const* dev_out, int stall,
                              int mode, std::vector<char>* eligible) {
  std::vector<std::vector<BatchTask>> per(n);
  eligible->assign(n, 0);
  size_t max_len = 0;
  int n_el = 0;
  for (int i = 0; i < n; ++i)
    if (exec_batch_tasks(&hs[i]->ex, hs[i]->leaves, dev_out[i], &per[i])) (*eligible)[i] = 1, ++n_el;
  // mode 2: only a batch that is at least half small networks
  if (mode == 2 && 2 * n_el < n) {
    eligible->assign(n, 0);
    return cudaSuccess;
  }
  for (int i = 0; i < n; ++i)
    if ((*eligible)[i]) {
      max_len = std::max(max_len, per[i].size());
      b->n_persistent++;
    }
  std::vector<BatchTask> tasks;
  std::vector<uint64_t> start(1, 0);
  std::vector<int> last(n, -1);
  for (size_t l = 0; l < max_len; ++l)
    for (int i = 0; i < n; ++i) {
      if (!(*eligible)[i] || l >= per[i].size()) continue;
      BatchTask T = per[i][l];
      T.dep = last[i];
      T.dep_units = T.dep >= 0 ? tasks[T.dep].n_units : 0;
      // test hook: one dependency of this network never completes
      if (i == stall && T.dep >= 0) T.dep_units = tasks[T.dep].n_units + 1;
      last[i] = (int)tasks.size();
      tasks.push_back(T);
      start.push_back(start.back() + T.n_units);
    }
  b->n_tasks = (int)tasks.size();
  if (!b->n_tasks) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)&b->d_tasks, tasks.size() * sizeof(BatchTask));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_start, start.size() * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_next, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_done, tasks.size() * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_abort, sizeof(int));
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_tasks, tasks.data(), tasks.size() * sizeof(BatchTask), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_start, start.data(), start.size() * sizeof(uint64_t), cudaMemcpyHostToDevice);
  return e;
}
}  // namespace

qtpu_status qtpu_htn_contract_batch(qtpu_htn* const* hs, int n, double* const* dev_out, void* cuda_stream) {
  return qtpu_htn_contract_batch_ex(hs, n, dev_out, cuda_stream, nullptr);
}

qtpu_status qtpu_htn_contract_batch_ex(qtpu_htn* const* hs, int n, double* const* dev_out, void* cuda_stream,
                                       const qtpu_batch_opts* opts) {
  if (n < 0 || (n > 0 && (!hs || !dev_out))) return QTPU_EINVAL;
  if (n == 0) return QTPU_OK;
  qtpu_batch_opts o{2, 0, -1};
  if (opts) o = *opts;
  if (o.persistent < 0 || o.persistent > 2) return fail(hs[0], QTPU_EINVAL, "persistent must be 0, 1 or 2");
  if (o.wait_limit_ns == 0) o.wait_limit_ns = 2000000000ull;
  if (o.wait_limit_ns > 10000000000ull) return fail(hs[0], QTPU_EINVAL, "wait limit above 10 s");
  for (int i = 0; i < n; ++i) {
    qtpu_htn* h = hs[i];
    if (!h) return QTPU_EINVAL;
    if (!h->planned) return fail(h, QTPU_ESTATE, "contract before plan");
    if (h->host_only) return fail(h, QTPU_ENOTSUP, "host-only handle cannot contract");
    if (h->device != hs[0]->device) return fail(h, QTPU_EINVAL, "handles on different devices");
    if (!dev_out[i]) return fail(h, QTPU_EINVAL, "dev_out NULL");
    for (int j = 0; j < i; ++j)
      if (hs[j] == h) return fail(h, QTPU_EINVAL, "a handle appears twice in the batch");
  }
  const int dev = hs[0]->device;
  if (dev >= 64) return fail(hs[0], QTPU_ENOTSUP, "device index >= 64");
  cudaError_t e = cudaSetDevice(dev);
  if (e != cudaSuccess) return fail(hs[0], QTPU_ECUDA, cudaGetErrorString(e));
  cudaStream_t user = cuda_stream ? (cudaStream_t)cuda_stream : hs[0]->stream;
  std::lock_guard<std::mutex> g(g_batch.mu);
  if (!batch_streams(dev)) return fail(hs[0], QTPU_ECUDA, "batch streams");
  BatchGraph* b = nullptr;
  for (BatchGraph* c : g_batch.cache)
    if (c->device == dev && (int)c->hs.size() == n && std::equal(c->hs.begin(), c->hs.end(), hs) &&
        std::equal(c->outs.begin(), c->outs.end(), dev_out) && c->persistent == o.persistent &&
        c->limit_ns == o.wait_limit_ns && c->stall == o.test_stall_network)
      b = c;
  if (!b) {
    b = new BatchGraph();
    b->hs.assign(hs, hs + n);
    b->outs.assign(dev_out, dev_out + n);
    b->device = dev;
    b->persistent = o.persistent;
    b->limit_ns = o.wait_limit_ns;
    b->stall = o.test_stall_network;
    std::vector<char> eligible(n, 0);
    if (b->persistent) {
      e = batch_build_tasks(b, hs, n, dev_out, o.test_stall_network, o.persistent, &eligible);
      if (e != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return fail(hs[0], QTPU_ENOMEM, std::string("batch tasks: ") + cudaGetErrorString(e));
      }
    }
    int sm = 148;
    cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
    cudaStream_t cs = g_batch.cap[dev];
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e1 = cudaEventRecord(g_batch.fork[dev], cs);
      for (int i = 0; i < kBranches && e1 == cudaSuccess; ++i)
        e1 = cudaStreamWaitEvent(g_batch.br[dev][i], g_batch.fork[dev], 0);
      if (e1 == cudaSuccess && b->n_tasks) {
        cudaStream_t s0 = g_batch.br[dev][0];
        e1 = cudaMemsetAsync(b->d_next, 0, sizeof(unsigned long long), s0);
        if (e1 == cudaSuccess) e1 = cudaMemsetAsync(b->d_done, 0, (size_t)b->n_tasks * 4, s0);
        if (e1 == cudaSuccess) e1 = cudaMemsetAsync(b->d_abort, 0, sizeof(int), s0);
        if (e1 == cudaSuccess)
          e1 = launch_batch_persistent(b->d_tasks, b->n_tasks, b->d_start, b->d_next, b->d_done, o.wait_limit_ns,
                                       b->d_abort, batch_grid(sm), s0);
      }
      int k = 0;
      for (int i = 0; i < n && e1 == cudaSuccess; ++i) {
        if (eligible[i]) continue;
        qtpu_htn* h = hs[i];
        // branch 0 carries the persistent kernel when there is one
        const int br = b->n_tasks ? 1 + (k++ % (kBranches - 1)) : (k++ % kBranches);
        cudaStream_t bs = g_batch.br[dev][br];
        int64_t no = 1;
        qtpu_htn_output_size(h, &no);
        e1 = exec_enqueue(&h->ex, h->leaves, h->ex.out_stage, bs);
        if (e1 == cudaSuccess)
          e1 = cudaMemcpyAsync(dev_out[i], h->ex.out_stage, (size_t)no * 8, cudaMemcpyDeviceToDevice, bs);
      }
      for (int i = 0; i < kBranches && e1 == cudaSuccess; ++i) {
        e1 = cudaEventRecord(g_batch.join[dev][i], g_batch.br[dev][i]);
        if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(cs, g_batch.join[dev][i], 0);
      }
      e = cudaStreamEndCapture(cs, &graph);
      if (e1 != cudaSuccess) e = e1;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      cudaGetLastError();
      batch_free(b);
      return fail(hs[0], QTPU_ECUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    }
    g_batch.cache.push_back(b);
    if (g_batch.cache.size() > 4) {
      batch_free(g_batch.cache.front());
      g_batch.cache.erase(g_batch.cache.begin());
    }
  }
  cudaStream_t cs = g_batch.cap[dev];
  e = cudaEventRecord(g_batch.in[dev], user);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, g_batch.in[dev], 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, cs);
  if (e == cudaSuccess) e = cudaEventRecord(g_batch.out[dev], cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(user, g_batch.out[dev], 0);
  if (e != cudaSuccess) return fail(hs[0], QTPU_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
  return QTPU_OK;
}

qtpu_status qtpu_htn_batch_info(qtpu_htn* const* hs, int n, double* const* dev_out, int* n_persistent,
                                int* n_tasks) {
  if (!hs || !dev_out || n < 1) return QTPU_EINVAL;
  std::lock_guard<std::mutex> g(g_batch.mu);
  for (auto it = g_batch.cache.rbegin(); it != g_batch.cache.rend(); ++it) {
    BatchGraph* c = *it;
    if ((int)c->hs.size() == n && std::equal(c->hs.begin(), c->hs.end(), hs) &&
        std::equal(c->outs.begin(), c->outs.end(), dev_out)) {
      if (n_persistent) *n_persistent = c->n_persistent;
      if (n_tasks) *n_tasks = c->n_tasks;
      return QTPU_OK;
    }
  }
  return QTPU_ESTATE;
}

qtpu_status qtpu_htn_profile(qtpu_htn* h, int enable) {
  if (!h) return QTPU_EINVAL;
  h->ex.prof.on = enable != 0;
  return QTPU_OK;
}

qtpu_status qtpu_htn_profile_read(qtpu_htn* h, int n, double* ms, int64_t* launches, double* flops,
                                  double* bytes) {
  if (!h || n < 0 || n > KC_COUNT) return QTPU_EINVAL;
  if (h->host_only || !h->built) return fail(h, QTPU_ESTATE, "nothing to read");
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess && h->ex.own) e = cudaStreamSynchronize(h->ex.own);
  if (e != cudaSuccess) return fail(h, QTPU_ECUDA, cudaGetErrorString(e));
  double m[KC_COUNT], f[KC_COUNT], b[KC_COUNT];
  int64_t l[KC_COUNT];
  std::string err = exec_profile_read(&h->ex, m, l, f, b);
  if (!err.empty()) return fail(h, QTPU_ECUDA, err);
  for (int k = 0; k < n; ++k) {
    if (ms) ms[k] = m[k];
    if (launches) launches[k] = l[k];
    if (flops) flops[k] = f[k];
    if (bytes) bytes[k] = b[k];
  }
  return QTPU_OK;
}

qtpu_status qtpu_htn_selftest_timeout(qtpu_htn* h, uint64_t limit_ns) {
  if (!h) return QTPU_EINVAL;
  if (h->host_only || !h->built) return fail(h, QTPU_ESTATE, "needs a planned device handle");
  if (limit_ns == 0 || limit_ns > 10000000000ull) return fail(h, QTPU_EINVAL, "limit must be in (0, 10 s]");
  cudaError_t e = cudaSetDevice(h->device);
  if (e == cudaSuccess) e = launch_bounded_wait_probe(h->ex.status, limit_ns, h->stream);
  if (e != cudaSuccess) return fail(h, QTPU_ECUDA, cudaGetErrorString(e));
  return QTPU_OK;
}

qtpu_status qtpu_htn_selftest_gemm_timeout(qtpu_htn* h, int pair, uint64_t limit_ns) {
  if (!h) return QTPU_EINVAL;
  if (h->host_only || !h->built) return fail(h, QTPU_ESTATE, "needs a planned device handle");
  if (limit_ns == 0 || limit_ns > 10000000000ull) return fail(h, QTPU_EINVAL, "limit must be in (0, 10 s]");
  if (pair != 0 && pair != 1) return fail(h, QTPU_EINVAL, "pair must be 0 or 1");
  // one 256 x 128 x 64 BF16x3 problem on zeroed operand pieces, in memory
  // ordered on the handle's stream
  const int M = 256, N = 128, K = 64;
  const size_t a_bytes = (size_t)3 * M * K * 2, b_bytes = (size_t)3 * N * K * 2, c_bytes = (size_t)M * N * 8;
  void *A = nullptr, *B = nullptr, *Cb = nullptr;
  cudaError_t e = cudaSetDevice(h->device);
  if (e == cudaSuccess) e = gemm_prepare();
  if (e == cudaSuccess) e = cudaMallocAsync(&A, a_bytes, h->stream);
  if (e == cudaSuccess) e = cudaMallocAsync(&B, b_bytes, h->stream);
  if (e == cudaSuccess) e = cudaMallocAsync(&Cb, c_bytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(A, 0, a_bytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(B, 0, b_bytes, h->stream);
  if (e == cudaSuccess) {
    GemmArgs g;
    g.nval = 1;
    g.C = Cb;
    g.batch = 1;
    g.M = M;
    g.N = N;
    g.K = K;
    g.prec = 3;
    g.bn = 128;
    g.pair = pair;
    g.status = h->ex.status;
    g.limit_ns = limit_ns;
    g.test_no_loads = 1;
    if (!make_operand_map(&g.maps.a[0], A, 3, 1, M, K, K, 128) ||
        !make_operand_map(&g.maps.b[0], B, 3, 1, N, K, K, pair ? 64 : 128))
      e = cudaErrorInvalidValue;
    if (e == cudaSuccess) e = launch_gemm(g, h->ex.sm_count, h->stream);
  }
  for (void* p : {A, B, Cb})
    if (p) cudaFreeAsync(p, h->stream);
  if (e != cudaSuccess) return fail(h, QTPU_ECUDA, cudaGetErrorString(e));
  return QTPU_OK;
}

qtpu_status qtpu_htn_destroy(qtpu_htn* h) {
  if (!h) return QTPU_EINVAL;
  batch_forget(h);
  if (h->built) {
    cudaSetDevice(h->device);
    exec_free(&h->ex);
  }
  for (cudaEvent_t ev : h->leaf_ev) cudaEventDestroy(ev);
  if (h->up_start) cudaEventDestroy(h->up_start);
  if (h->up_stream) cudaStreamDestroy(h->up_stream);
  if (!h->owned.empty()) {
    // pool memory, freed in stream order after the work that uses it
    cudaSetDevice(h->device);
    for (void* p : h->owned) cudaFreeAsync(p, h->stream);
  }
  delete h;
  return QTPU_OK;
}

const char* qtpu_last_error(const qtpu_htn* h) {
  if (!h) return g_create_err.c_str();
  return h->err.empty() ? "no error" : h->err.c_str();
}

}  // extern "C"
