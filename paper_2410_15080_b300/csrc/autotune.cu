// GEMM tile table: the orientation and N tile of each tensor-core GEMM
// problem, measured on the device.
//
// The pairwise contractions of section 4.2 become batched GEMMs whose sizes
// are products of small index dimensions (6, 24, 36, 216, 1296, ...): rarely
// multiples of the kernel's 128-row M tile.  Which side runs along M and how
// wide the N tile is decide how much of every tile is padding; the padding
// rule below picks by counted tile area, and exec_autotune measures every
// valid choice of a plan's GEMM problems on synthetic operand pieces and
// records the fastest in a tile table, which the lowering then follows.
// Each GEMM is timed alone: the layout its result leaves for the next step
// (set by the orientation) is not part of the measurement, so the tuner
// keeps a problem's orientation unless the other one is clearly faster.
#include <cuda_runtime.h>
#include <dlfcn.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <set>
#include <vector>

#include "exec.h"

namespace qtpu {

namespace {

// the least gain (fraction of the time) for which the tuner changes a
// problem's orientation
constexpr double kSwapGain = 0.03;

bool valid_tile(double nm, double nn, bool swap, int bn, int pair = 0, int prec = 3) {
  const double gM = swap ? nn : nm, gN = swap ? nm : nn;
  return gM >= 64 && gN >= 16 && gemm_bn_supported(bn, pair, prec);
}

// synthetic operand pieces: values uniform in [-1, 1) from a 32-bit hash of
// the entry index (their bits only load the tensor cores like real data)
__global__ void k_fill_pieces(void* p, size_t n, int es, uint32_t seed) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)i * 0x9E3779B1u ^ seed;
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    const float v = (float)(h >> 8) * (2.0f / 16777216.0f) - 1.0f;
    if (es == 2) {
      const uint32_t b = __float_as_uint(v) >> 16;  // truncated to BF16
      ((uint16_t*)p)[i] = (uint16_t)b;
    } else {
      ((float*)p)[i] = v;
    }
  }
}

}  // namespace

std::string load_tile_table(const std::string& path, TileTable* t) {
  FILE* fp = std::fopen(path.c_str(), "r");
  if (!fp) return "cannot open the tile table " + path;
  char line[512];
  int ln = 0;
  std::string err;
  while (std::fgets(line, sizeof line, fp)) {
    ++ln;
    const char* c = line;
    while (*c == ' ' || *c == '\t') ++c;
    if (*c == '#' || *c == '\n' || *c == 0) continue;
    long long k[5];
    int swap = 0, bn = 0, pair = 0;
    double ms = 0, ms_rule = 0, ms_base = 0;
    const int got = std::sscanf(c, "%lld %lld %lld %lld %lld : %d %d %lf %lf %lf %d", &k[0], &k[1], &k[2], &k[3],
                                &k[4], &swap, &bn, &ms, &ms_rule, &ms_base, &pair);
    if (got < 7 || (swap != 0 && swap != 1) || (pair != 0 && pair != 1) || !gemm_bn_supported(bn, pair, (int)k[0]) ||
        k[0] < 0 || k[0] > 3 || (pair && k[0] != 3)) {
      err = path + ":" + std::to_string(ln) + ": not a tile table line";
      break;
    }
    TileChoice ch;
    ch.swap = swap;
    ch.bn = bn;
    ch.pair = pair;
    ch.ms = ms;
    ch.ms_rule = ms_rule;
    ch.ms_base = ms_base;
    (*t)[TileKey{k[0], k[1], k[2], k[3], k[4]}] = ch;
  }
  std::fclose(fp);
  return err;
}

std::string save_tile_table(const std::string& path, const TileTable& t) {
  FILE* fp = std::fopen(path.c_str(), "w");
  if (!fp) return "cannot write the tile table " + path;
  std::fprintf(fp,
               "# GEMM tile table: prec batch m n k : swap bn ms ms_rule ms_base pair\n"
               "# (m, n: the step's index-group sizes; swap 1: m runs along the N tile of bn columns;\n"
               "#  median times in ms of that choice, of the padding rule's choice, and of 128-column\n"
               "#  tiles with m along M unless m < 64; pair 1: 256-row tiles on a pair of CTAs)\n");
  for (const auto& kv : t)
    std::fprintf(fp, "%lld %lld %lld %lld %lld : %d %d %.6f %.6f %.6f %d\n", (long long)kv.first[0],
                 (long long)kv.first[1], (long long)kv.first[2], (long long)kv.first[3], (long long)kv.first[4],
                 kv.second.swap, kv.second.bn, kv.second.ms, kv.second.ms_rule, kv.second.ms_base, kv.second.pair);
  const bool ok = std::fclose(fp) == 0;
  return ok ? "" : "cannot write the tile table " + path;
}

std::string default_tile_table_path() {
  Dl_info info;
  if (dladdr((void*)&default_tile_table_path, &info) && info.dli_fname) {
    std::string p = info.dli_fname;
    const size_t s = p.find_last_of('/');
    return (s == std::string::npos ? std::string(".") : p.substr(0, s)) + "/gemm_tiles_b300.txt";
  }
  return "gemm_tiles_b300.txt";
}

void choose_tile(const TileTable* t, int prec, double nb, double nm, double nn, double nk, bool* swap, int* bn,
                 int* pair) {
  *pair = 0;
  if (t && !t->empty()) {
    auto it = t->find(TileKey{prec, (int64_t)nb, (int64_t)nm, (int64_t)nn, (int64_t)nk});
    if (it != t->end() && valid_tile(nm, nn, it->second.swap != 0, it->second.bn, it->second.pair, prec)) {
      *swap = it->second.swap != 0;
      *bn = it->second.bn;
      *pair = prec == 3 ? it->second.pair : 0;
      return;
    }
    it = t->find(TileKey{prec, (int64_t)nb, (int64_t)nn, (int64_t)nm, (int64_t)nk});
    if (it != t->end() && valid_tile(nm, nn, it->second.swap == 0, it->second.bn, it->second.pair, prec)) {
      *swap = it->second.swap == 0;
      *bn = it->second.bn;
      *pair = prec == 3 ? it->second.pair : 0;
      return;
    }
  }
  double best = std::numeric_limits<double>::infinity();
  bool bs = *swap;
  int bb = *bn;
  for (int o = 0; o < 2; ++o) {
    const bool sw = o == 0 ? *swap : !*swap;
    for (int b : kGemmBlockN) {
      if (!valid_tile(nm, nn, sw, b)) continue;
      const double gM = sw ? nn : nm, gN = sw ? nm : nn;
      const double c = std::ceil(gM / 128.0) * std::ceil(gN / b) * (b + 128);
      if (c < best) best = c, bs = sw, bb = b;
    }
  }
  if (best < std::numeric_limits<double>::infinity()) *swap = bs, *bn = bb;
}

std::string exec_autotune(const Executor* ex, int reps, TileTable* t, int* n, int* code) {
  *n = 0;
  *code = QTPU_OK;
  if (!ex->lowered) {
    *code = QTPU_ESTATE;
    return "no lowered plan";
  }
  if (reps < 1) reps = 1;
  cudaError_t e = gemm_prepare();
  if (e != cudaSuccess) {
    *code = QTPU_ECUDA;
    return cudaGetErrorString(e);
  }
  int sm = 148;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  uint32_t* status = nullptr;
  std::string err;
  auto cuda_fail = [&](cudaError_t x) {
    cudaGetLastError();
    *code = x == cudaErrorMemoryAllocation ? QTPU_ENOMEM : QTPU_ECUDA;
    err = cudaGetErrorString(x);
  };
  if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess ||
      (e = cudaMalloc((void**)&status, 4)) != cudaSuccess || (e = cudaMemset(status, 0, 4)) != cudaSuccess)
    cuda_fail(e);
  std::set<TileKey> done;
  for (const Launch& L : ex->launches) {
    if (!err.empty()) break;
    if (L.kind != LK_GEMM || L.tile_fixed) continue;
    const TileKey key{L.tile_key[0], L.tile_key[1], L.tile_key[2], L.tile_key[3], L.tile_key[4]};
    if (done.count(key)) continue;
    done.insert(key);
    const int prec = (int)key[0];
    const int64_t nb = key[1], nm = key[2], nn = key[3], nk = key[4];
    const int nval = (int)std::max<int64_t>(1, std::min<int64_t>(kGemmVals, L.runs / std::max<int64_t>(1, L.n_launch)));
    const int np = prec == 3 ? 3 : (prec == 2 ? 2 : 1);
    const int es = prec == 3 ? 2 : 4;
    const int64_t Kp = (nk + 7) / 8 * 8;
    const int64_t rows = std::max(nm, nn);
    const size_t piece_bytes = (size_t)np * nb * rows * Kp * es;
    const size_t c_bytes = (size_t)nb * nm * nn * 8;
    std::vector<void*> bufs;
    void* C = nullptr;
    // one buffer per operand and pair, each large enough for either side
    for (int v = 0; v < 2 * nval && err.empty(); ++v) {
      void* p = nullptr;
      if ((e = cudaMalloc(&p, piece_bytes)) != cudaSuccess) {
        cuda_fail(e);
        break;
      }
      bufs.push_back(p);
      k_fill_pieces<<<sm * 8, 256, 0, st>>>(p, piece_bytes / es, es, 0x51ED270Bu + 977u * (uint32_t)v);
    }
    if (err.empty() && (e = cudaMalloc(&C, c_bytes)) != cudaSuccess) cuda_fail(e);
    const bool base_swap = nm < 64 && nn >= 64;
    bool rule_swap = base_swap;
    int rule_bn = 128, rule_pair = 0;
    choose_tile(nullptr, prec, (double)nb, (double)nm, (double)nn, (double)nk, &rule_swap, &rule_bn, &rule_pair);
    // the orientation also sets the layout the next step reads, which a GEMM
    // timed alone does not show: the other orientation replaces the one of
    // the problem's present entry (else the padding rule's) only when it is
    // more than kSwapGain faster
    bool ref_swap = rule_swap;
    {
      const auto it = t->find(key);
      const auto jt = t->find(TileKey{key[0], key[1], key[3], key[2], key[4]});
      if (it != t->end())
        ref_swap = it->second.swap != 0;
      else if (jt != t->end())
        ref_swap = jt->second.swap == 0;
    }
    TileChoice best, best_ref;
    best.ms = best_ref.ms = std::numeric_limits<double>::infinity();
    // every width on one CTA and on a CTA pair; valid_tile drops the ones a
    // form lacks (224 and 256 on one CTA, 160 and 144 on pairs or outside BF16x3)
    std::vector<int> widths(std::begin(kGemmPairWideN), std::end(kGemmPairWideN));
    widths.insert(widths.end(), std::begin(kGemmWideN), std::end(kGemmWideN));
    widths.insert(widths.end(), std::begin(kGemmBlockN), std::end(kGemmBlockN));
    for (int o = 0; o < 4 && err.empty(); ++o)
      for (int bn : widths) {
        if (!err.empty()) break;
        const bool sw = (o & 1) != 0;
        const int pair = o >> 1;  // CTA pairs: BF16x3 only
        if (pair && prec != 3) continue;
        if (!valid_tile((double)nm, (double)nn, sw, bn, pair, prec)) continue;
        GemmArgs g;
        g.nval = nval;
        g.C = C;
        g.batch = (int)nb;
        g.M = (int)(sw ? nn : nm);
        g.N = (int)(sw ? nm : nn);
        g.K = (int)nk;
        g.kc_blocks = ex->kc_blocks;
        g.prec = prec;
        g.bn = bn;
        g.pair = pair;
        g.status = status;
        bool ok = true;
        for (int v = 0; v < nval && ok; ++v)
          ok = make_operand_map(&g.maps.a[v], bufs[2 * v], prec, nb, g.M, nk, Kp, 128) &&
               make_operand_map(&g.maps.b[v], bufs[2 * v + 1], prec, nb, g.N, nk, Kp, pair ? bn / 2 : bn);
        if (!ok) {
          *code = QTPU_ECUDA;
          err = "cuTensorMapEncodeTiled failed";
          break;
        }
        std::vector<float> ms;
        for (int r = -1; r < reps && err.empty(); ++r) {  // one warm-up launch
          if ((e = cudaEventRecord(e0, st)) != cudaSuccess || (e = launch_gemm(g, sm, st)) != cudaSuccess ||
              (e = cudaEventRecord(e1, st)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess) {
            cuda_fail(e);
            break;
          }
          float x = 0;
          cudaEventElapsedTime(&x, e0, e1);
          if (r >= 0) ms.push_back(x);
        }
        if (!err.empty()) break;
        std::sort(ms.begin(), ms.end());
        const double med = ms[ms.size() / 2];
        if (sw == rule_swap && bn == rule_bn && !pair) best.ms_rule = med;
        if (sw == base_swap && bn == 128 && !pair) best.ms_base = med;
        if (med < best.ms) best.ms = med, best.swap = sw ? 1 : 0, best.bn = bn, best.pair = pair;
        if (sw == ref_swap && med < best_ref.ms) best_ref.ms = med, best_ref.swap = sw ? 1 : 0, best_ref.bn = bn,
                                                 best_ref.pair = pair;
      }
    if ((best.swap != 0) != ref_swap && best_ref.ms <= best.ms * (1.0 + kSwapGain)) {
      best_ref.ms_rule = best.ms_rule;
      best_ref.ms_base = best.ms_base;
      best = best_ref;
    }
    uint32_t hs = 0;
    if (err.empty() && (e = cudaMemcpy(&hs, status, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) cuda_fail(e);
    if (err.empty() && hs) {
      *code = QTPU_ETIMEOUT;
      err = "a GEMM's bounded wait gave up while timing tiles";
    }
    for (void* p : bufs) cudaFree(p);
    if (C) cudaFree(C);
    if (err.empty() && best.ms < std::numeric_limits<double>::infinity()) {
      (*t)[key] = best;
      ++*n;
    }
  }
  if (status) cudaFree(status);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  return err;
}

}  // namespace qtpu
