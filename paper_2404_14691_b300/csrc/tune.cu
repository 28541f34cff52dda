// Autotuner of the tensor-core GEMM tiles.
//
// For a GEMM shape (kind, M bucket, N, K) it times every tile configuration the
// kernels offer (N tile x pipeline depth) on scratch operands with CUDA events
// and keeps the fastest in a process-wide table; launches then use the table.
// M is bucketed to the next power of two (>= 128), since the best tile depends
// on how many waves of CTAs the batch makes.  The table can be saved to and
// loaded from a text file keyed by the GPU's name, so a box tunes once.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/sage.h"
#include "kernels.h"

namespace sage {
namespace {

using Key = std::tuple<int, int, int, int>;  // kind, M bucket, N, K
std::mutex g_mu;
std::map<Key, GemmCfg> g_table;

int bucket(int M) {
  int b = 128;
  while (b < M && b < (1 << 30)) b <<= 1;
  return b;
}

std::string gpu_name() {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  std::string s = p.name;
  std::replace(s.begin(), s.end(), ' ', '_');
  return s;
}

// Median of five timed runs (CUDA events on the stream; the run was warmed up once).
template <class Run>
float median_of_5(Run& run, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  float t[5];
  for (int r = 0; r < 5; ++r) {
    cudaEventRecord(e0, s);
    run();
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    t[r] = 0;
    cudaEventElapsedTime(&t[r], e0, e1);
  }
  std::sort(t, t + 5);
  return t[2];
}

}  // namespace

GemmCfg tuned_gemm(int kind, int M, int N, int K) {
  std::lock_guard<std::mutex> g(g_mu);
  auto it = g_table.find(Key{kind, bucket(M), N, K});
  return it == g_table.end() ? GemmCfg{0, 0} : it->second;
}

// Times each candidate for one shape; returns the chosen config (or {0,0}).
sage_status autotune_gemm(int kind, int M, int N, int K, cudaStream_t s, GemmCfg* chosen, double* best_ms) {
  const int Mb = bucket(M);
  const size_t es = kind == kGemmBf16 ? 2 : 4;
  void *x = nullptr, *w = nullptr, *y = nullptr, *b = nullptr;
  int* err = nullptr;
  auto cleanup = [&] {
    cudaFree(x);
    cudaFree(w);
    cudaFree(y);
    cudaFree(b);
    cudaFree(err);
  };
  if (cudaMalloc(&x, static_cast<size_t>(Mb) * K * es) != cudaSuccess ||
      cudaMalloc(&w, static_cast<size_t>(N) * K * es) != cudaSuccess ||
      cudaMalloc(&y, static_cast<size_t>(Mb) * N * es) != cudaSuccess ||
      cudaMalloc(&b, static_cast<size_t>(N) * 4) != cudaSuccess || cudaMalloc(&err, 256) != cudaSuccess) {
    cleanup();
    cudaGetLastError();
    set_last_error("autotune: scratch allocation failed");
    return SAGE_ERR_NOMEM;
  }
  // small nonzero operands (0x3c3c.. patterns), zero bias
  cudaMemsetAsync(x, 0x3c, static_cast<size_t>(Mb) * K * es, s);
  cudaMemsetAsync(w, 0x3c, static_cast<size_t>(N) * K * es, s);
  cudaMemsetAsync(b, 0, static_cast<size_t>(N) * 4, s);
  cudaMemsetAsync(err, 0, 256, s);
  GemmCfg cands[16];
  const int nc = gemm_candidates(kind, cands, 16);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  GemmCfg best{0, 0};
  float best_t = 1e30f;
  for (int c = 0; c < nc; ++c) {
    if (N % cands[c].bn) continue;
    auto run = [&] {
      if (kind == kGemmBf16)
        return launch_linear_bf16_tc(Mb, N, K, x, K, w, static_cast<float*>(b), 1, y, N, err, s, cands[c]);
      if (kind == kGemmTf32Pre)  // the same buffer serves as both planes: timing only
        return launch_linear_f32_tc_presplit(Mb, N, K, static_cast<float*>(x), static_cast<float*>(x), K,
                                             static_cast<float*>(w), static_cast<float*>(w), static_cast<float*>(b),
                                             1, static_cast<float*>(y), static_cast<float*>(y), N, err, s, cands[c]);
      return launch_linear_f32_tc(Mb, N, K, static_cast<float*>(x), K, static_cast<float*>(w),
                                  static_cast<float*>(b), 1, static_cast<float*>(y), N, err, s, cands[c]);
    };
    if (run() != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    const float t = median_of_5(run, s, e0, e1);
    if (t < best_t) {
      best_t = t;
      best = cands[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaError_t ce = cudaStreamSynchronize(s);
  cleanup();
  if (ce != cudaSuccess) {
    set_last_error("autotune: a timing run failed");
    return SAGE_ERR_CUDA;
  }
  if (best.bn) {
    std::lock_guard<std::mutex> g(g_mu);
    g_table[Key{kind, Mb, N, K}] = best;
  }
  if (chosen) *chosen = best;
  if (best_ms) *best_ms = best_t;
  return SAGE_OK;
}

// Bottom layers 0 and 1 (and 2 when N2 > 0) of a pre-split fp32 function (K0 dense
// inputs, N0, N1 and N2 outputs): times the fused kernel's tiles against bottom0
// followed by the layer GEMMs at their own tuned tiles (so tune those first); when
// N2 > 0 every candidate includes layer 2 -- its GEMM, or the three-layer kernel
// (256, 202) where the shape allows it.  Records the fastest under (kBottom01,
// M bucket, N1, N0); {1, 1} records that separate kernels won.
sage_status autotune_bottom01(int M, int K0, int N0, int N1, int N2, cudaStream_t s, GemmCfg* chosen) {
  if (!bottom01_fusable(K0, N0, N1)) return set_last_error("autotune: shape cannot fuse"), SAGE_ERR_INVALID;
  const int Mb = bucket(M);
  const int n2 = N2 > 0 ? N2 : 0;
  const size_t sizes[] = {static_cast<size_t>(Mb) * K0,     static_cast<size_t>(N0) * K0,
                          static_cast<size_t>(N0),          static_cast<size_t>(N1) * N0,
                          static_cast<size_t>(N1),          2 * static_cast<size_t>(Mb) * N0,
                          2 * static_cast<size_t>(Mb) * N1, static_cast<size_t>(n2 ? n2 : 1) * N1,
                          static_cast<size_t>(n2 ? n2 : 1), 2 * static_cast<size_t>(Mb) * (n2 ? n2 : 1),
                          64};
  constexpr int kBufs = sizeof(sizes) / sizeof(sizes[0]);
  float* b[kBufs] = {};
  auto cleanup = [&] {
    for (float* p : b) cudaFree(p);
  };
  for (int i = 0; i < kBufs; ++i) {
    if (cudaMalloc(&b[i], sizes[i] * 4) != cudaSuccess) {
      cleanup();
      cudaGetLastError();
      return set_last_error("autotune: scratch allocation failed"), SAGE_ERR_NOMEM;
    }
    cudaMemsetAsync(b[i], i == kBufs - 1 ? 0 : 0x3c, sizes[i] * 4, s);
  }
  float *dense = b[0], *w0 = b[1], *b0 = b[2], *w1 = b[3], *b1 = b[4], *y0 = b[5], *y1 = b[6];
  float *w2 = b[7], *b2 = b[8], *y2 = b[9];
  int* err = reinterpret_cast<int*>(b[10]);
  std::unique_ptr<InvTable> tab(new InvTable());
  tab->n = 1;
  tab->M = Mb;
  tab->d[0] = InvDesc{dense, nullptr, nullptr, nullptr, Mb, 0, 0};
  const GemmCfg g1 = tuned_gemm(kGemmTf32Pre, Mb, N1, N0);
  const GemmCfg g2 = n2 ? tuned_gemm(kGemmTf32Pre, Mb, n2, N1) : GemmCfg{0, 0};
  float* y1l = y1 + static_cast<size_t>(Mb) * N1;
  float* y2l = y2 + static_cast<size_t>(Mb) * (n2 ? n2 : 1);
  auto layer2 = [&]() -> cudaError_t {
    if (!n2) return cudaSuccess;
    return launch_linear_f32_tc_presplit(Mb, n2, N1, y1, y1l, N1, w2, w2, b2, 1, y2, y2l, n2, err, s, g2);
  };
  GemmCfg cands[16];
  const int nc = bottom01_candidates(cands, 16);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  GemmCfg best{0, 0};
  float best_t = 1e30f;
  for (int c = 0; c < nc; ++c) {
    if (N1 % cands[c].bn) continue;
    const bool three = cands[c].stages == 202;
    if (three && !(n2 && bottom012_fusable(N1, n2, Mb))) continue;
    auto run = [&]() -> cudaError_t {
      cudaError_t ce;
      if (cands[c].bn == 1) {
        ce = launch_bottom0(0, *tab, K0, N0, w0, b0, y0, N0, s, y0 + static_cast<size_t>(Mb) * N0);
        if (ce != cudaSuccess) return ce;
        ce = launch_linear_f32_tc_presplit(Mb, N1, N0, y0, y0 + static_cast<size_t>(Mb) * N0, N0, w1, w1, b1, 1, y1,
                                           y1l, N1, err, s, g1);
        return ce != cudaSuccess ? ce : layer2();
      }
      if (three)
        return launch_bottom01_f32(*tab, K0, N0, w0, b0, N1, w1, w1, b1, y2, y2l, n2, err, s, cands[c], w2, w2, b2,
                                   n2);
      ce = launch_bottom01_f32(*tab, K0, N0, w0, b0, N1, w1, w1, b1, y1, y1l, N1, err, s, cands[c]);
      return ce != cudaSuccess ? ce : layer2();
    };
    if (run() != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    const float t = median_of_5(run, s, e0, e1);
    if (t < best_t) {
      best_t = t;
      best = cands[c];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaError_t ce = cudaStreamSynchronize(s);
  cleanup();
  if (ce != cudaSuccess) return set_last_error("autotune: a timing run failed"), SAGE_ERR_CUDA;
  if (best.bn) {
    std::lock_guard<std::mutex> g(g_mu);
    g_table[Key{kBottom01, Mb, N1, N0}] = best;
  }
  if (chosen) *chosen = best;
  return SAGE_OK;
}

}  // namespace sage

extern "C" sage_status sage_tuning_set(int kind, int rows, int N, int K, int bn, int stages) {
  sage::GemmCfg cands[16];
  const int nc = sage::gemm_candidates(kind, cands, 16);
  bool known = false;
  for (int c = 0; c < nc; ++c) known |= cands[c].bn == bn && cands[c].stages == stages;
  if (!known || rows < 1 || N < 1 || K < 1 || (N % bn))
    return sage::set_last_error("unknown tile configuration for this GEMM kind or shape"), SAGE_ERR_INVALID;
  std::lock_guard<std::mutex> g(sage::g_mu);
  sage::g_table[sage::Key{kind, sage::bucket(rows), N, K}] = sage::GemmCfg{bn, stages};
  return SAGE_OK;
}

extern "C" sage_status sage_tuning_save(const char* path) {
  if (!path) return sage::set_last_error("null path"), SAGE_ERR_INVALID;
  FILE* f = fopen(path, "w");
  if (!f) return sage::set_last_error("cannot write the tuning file"), SAGE_ERR_INVALID;
  const std::string gpu = sage::gpu_name();
  std::lock_guard<std::mutex> g(sage::g_mu);
  fprintf(f, "# gpu kind m_bucket N K bn stages\n");
  for (auto& kv : sage::g_table)
    fprintf(f, "%s %d %d %d %d %d %d\n", gpu.c_str(), std::get<0>(kv.first), std::get<1>(kv.first),
            std::get<2>(kv.first), std::get<3>(kv.first), kv.second.bn, kv.second.stages);
  fclose(f);
  return SAGE_OK;
}

extern "C" sage_status sage_tuning_load(const char* path) {
  if (!path) return sage::set_last_error("null path"), SAGE_ERR_INVALID;
  FILE* f = fopen(path, "r");
  if (!f) return sage::set_last_error("cannot read the tuning file"), SAGE_ERR_INVALID;
  const std::string gpu = sage::gpu_name();
  char line[512], name[256];
  int kind, mb, n, k, bn, st, loaded = 0;
  std::lock_guard<std::mutex> g(sage::g_mu);
  while (fgets(line, sizeof(line), f)) {
    if (line[0] == '#') continue;
    if (sscanf(line, "%255s %d %d %d %d %d %d", name, &kind, &mb, &n, &k, &bn, &st) != 7) continue;
    if (gpu != name) continue;  // tuned on another GPU model
    sage::GemmCfg cands[16];
    const int nc = sage::gemm_candidates(kind, cands, 16);
    bool known = false;
    for (int c = 0; c < nc; ++c) known |= cands[c].bn == bn && cands[c].stages == st;
    if (!known) continue;
    sage::g_table[sage::Key{kind, mb, n, k}] = sage::GemmCfg{bn, st};
    ++loaded;
  }
  fclose(f);
  return loaded > 0 ? SAGE_OK : (sage::set_last_error("no entries for this GPU"), SAGE_ERR_INVALID);
}
