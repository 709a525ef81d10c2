// Learned cost model at plan time (qtpu_plan_opts.cost_model = 1).
//
// Section 6.1 step 3 chooses a contraction sequence before contracting.  The
// exact FLOP count ranks candidates by arithmetic alone; the time of a
// contraction also depends on how its launches map onto the hardware (tile
// fill of the tensor-core steps, memory-bound gathers and splits, launch
// counts).  A small perceptron trained on the executor's own per-launch
// timings predicts the device time of every launch of a candidate plan from
// the launch's features (exec_launch_features); a candidate's time is the sum
// over its launches of (launches per contraction) x exp(predicted log us).
// The choice is the candidate with the smallest predicted time among those
// whose executed FLOPs are within `factor` of the fewest (the exact cost
// model bounds the model's error; the factor is stored with the weights).
// The model only chooses among plans: every plan is contracted by the same
// kernels, so results are unaffected.
#include <dlfcn.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/qtpu_htn.h"
#include "exec.h"
#include "planner.h"

namespace qtpu {

namespace {

struct CmFile {
  int din = 0, hid = 0;
  float factor = 1.f, ymu = 0.f;
  std::vector<float> mu, sd, params;
};

// Weights file (little-endian): "QTPUCM1" NUL, int32 in_dim, int32 hidden,
// float factor, float ymu, float mu[in_dim], float sd[in_dim], then the
// perceptron's FP32 parameters in the layout of qtpu_mlp_params.
bool load_model(const std::string& path, CmFile* m, std::string* err) {
  FILE* fp = std::fopen(path.c_str(), "rb");
  if (!fp) {
    *err = "cannot open the cost model file " + path;
    return false;
  }
  char magic[8] = {};
  bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, "QTPUCM1", 8) == 0;
  int32_t dims[2] = {0, 0};
  ok = ok && std::fread(dims, 4, 2, fp) == 2 && dims[0] > 0 && dims[1] > 0 && dims[0] <= 4096 && dims[1] <= 4096;
  float fy[2] = {0, 0};
  ok = ok && std::fread(fy, 4, 2, fp) == 2;
  if (ok) {
    m->din = dims[0];
    m->hid = dims[1];
    m->factor = fy[0];
    m->ymu = fy[1];
    m->mu.resize(m->din);
    m->sd.resize(m->din);
    const size_t np = (size_t)m->din * m->hid + m->hid + (size_t)m->hid * m->hid + m->hid + m->hid + 1;
    m->params.resize(np);
    ok = std::fread(m->mu.data(), 4, m->din, fp) == (size_t)m->din &&
         std::fread(m->sd.data(), 4, m->din, fp) == (size_t)m->din &&
         std::fread(m->params.data(), 4, np, fp) == np;
  }
  std::fclose(fp);
  if (!ok) *err = "the cost model file " + path + " is not a valid weights file";
  return ok;
}

}  // namespace

std::string default_cost_model_path() {
  Dl_info info;
  if (dladdr((void*)&default_cost_model_path, &info) && info.dli_fname) {
    std::string p = info.dli_fname;
    const size_t s = p.find_last_of('/');
    return (s == std::string::npos ? std::string(".") : p.substr(0, s)) + "/costmodel_b300.bin";
  }
  return "costmodel_b300.bin";
}

// Plan n candidates (seeds seed .. seed+n-1 under the given slicing options),
// lower each (no device memory), predict each one's contraction time with
// the perceptron on `device`, and return the chosen plan.  Returns a
// qtpu_status.
int plan_by_cost_model(const std::vector<Inds>& li, const DimMap& dims, const Inds& output,
                       const qtpu_plan_opts& o, const std::vector<Leaf>& leaves, int device, void* stream,
                       const TileTable* tiles, Plan* chosen, std::string* err) {
  CmFile cm;
  const std::string path = o.cost_model_path ? std::string(o.cost_model_path) : default_cost_model_path();
  if (!load_model(path, &cm, err)) return QTPU_EINVAL;
  if (cm.din != kLaunchFeatures) {
    *err = "the cost model expects " + std::to_string(cm.din) + " launch features";
    return QTPU_EINVAL;
  }
  const uint32_t nc = o.n_candidates > 1 ? o.n_candidates : 64;
  struct Cand {
    Plan plan;
    uint64_t seed;
    double flops;
    size_t row0, rows;
  };
  std::vector<Cand> cands;
  std::vector<float> X;
  std::vector<double> weight;
  for (uint64_t s = o.seed; s < o.seed + nc; ++s) {
    Cand c;
    const int r = make_plan(li, dims, output, o.max_intermediate_bytes, o.n_slices, o.slice_dim, &c.plan, s);
    if (r == PLAN_OVERFLOW) {
      *err = "a contraction size reaches 2^255";
      return QTPU_ENOTSUP;
    }
    if (r != PLAN_OK) continue;
    Executor ex;
    ex.device = device;
    int code = QTPU_OK;
    exec_build(&ex, c.plan, leaves, dims, (int)o.prec, &code, true, o.reuse_bytes, tiles);
    if (code != QTPU_OK || !ex.lowered) continue;
    c.seed = s;
    c.flops = ex.flops_executed;
    c.row0 = weight.size();
    c.rows = ex.launches.size();
    for (size_t i = 0; i < ex.launches.size(); ++i) {
      float f[kLaunchFeatures];
      exec_launch_features(&ex, i, f);
      for (int j = 0; j < kLaunchFeatures; ++j) X.push_back((f[j] - cm.mu[j]) / cm.sd[j]);
      weight.push_back((double)ex.launches[i].n_launch);
    }
    cands.push_back(std::move(c));
  }
  if (cands.empty()) {
    *err = "the peak-intermediate limit cannot be met by slicing";
    return QTPU_ELIMIT;
  }
  // predicted log(us) of every launch, on the device with the library's
  // perceptron kernels
  const int n = (int)weight.size();
  std::vector<float> y(n, 0.f);
  qtpu_mlp* m = nullptr;
  qtpu_status st = qtpu_mlp_create(&m, device, stream, cm.din, cm.hid, 1);
  if (st == QTPU_OK) st = qtpu_mlp_params(m, nullptr, cm.params.data());
  float *dx = nullptr, *dy = nullptr;
  if (st == QTPU_OK && (cudaMalloc((void**)&dx, X.size() * 4) != cudaSuccess ||
                        cudaMalloc((void**)&dy, (size_t)n * 4) != cudaSuccess))
    st = QTPU_ENOMEM;
  if (st == QTPU_OK && cudaMemcpyAsync(dx, X.data(), X.size() * 4, cudaMemcpyHostToDevice, (cudaStream_t)stream) !=
                           cudaSuccess)
    st = QTPU_ECUDA;
  if (st == QTPU_OK) st = qtpu_mlp_forward(m, dx, n, dy);
  if (st == QTPU_OK && cudaMemcpyAsync(y.data(), dy, (size_t)n * 4, cudaMemcpyDeviceToHost, (cudaStream_t)stream) !=
                           cudaSuccess)
    st = QTPU_ECUDA;
  if (st == QTPU_OK && cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) st = QTPU_ECUDA;
  if (dx) cudaFree(dx);
  if (dy) cudaFree(dy);
  if (m) qtpu_mlp_destroy(m);
  if (st != QTPU_OK) {
    cudaGetLastError();
    *err = "cost model inference failed";
    return st;
  }
  double fmin = cands[0].flops;
  for (const Cand& c : cands) fmin = std::min(fmin, c.flops);
  int best = -1;
  double best_t = 0;
  for (size_t k = 0; k < cands.size(); ++k) {
    const Cand& c = cands[k];
    if (c.flops > (double)cm.factor * fmin) continue;
    double t = 0;
    for (size_t r = c.row0; r < c.row0 + c.rows; ++r) t += weight[r] * std::exp((double)y[r] + cm.ymu);
    if (best < 0 || t < best_t || (t == best_t && c.flops < cands[best].flops)) best = (int)k, best_t = t;
  }
  *chosen = cands[best].plan;
  chosen->search = nc;
  chosen->search_seed = cands[best].seed;
  return QTPU_OK;
}

}  // namespace qtpu
