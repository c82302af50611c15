// Autotuner over the interval count P (the paper's Exp 2, Section IV-B2).
// Each candidate is built and timed on the device; results can be cached in a
// plain text file, one "key best_P" line per tuned workload.
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>

#include "nx_internal.cuh"

namespace nx {
namespace {

std::string tune_key(uint64_t m, uint32_t n, uint32_t flags, nx_program prog, const uint32_t* cand,
                     uint32_t count) {
  cudaDeviceProp prop{};
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  std::ostringstream k;
  std::string name = prop.name;
  for (char& ch : name)
    if (ch == ' ') ch = '_';
  k << name << "|n=" << n << "|m=" << m << "|flags=" << flags << "|prog=" << (int)prog << "|P=";
  for (uint32_t q = 0; q < count; ++q) k << (q ? "," : "") << cand[q];
  return k.str();
}

bool cache_lookup(const char* path, const std::string& key, uint32_t* P) {
  if (!path) return false;
  std::ifstream f(path);
  std::string k;
  uint32_t v;
  while (f >> k >> v)
    if (k == key) {
      *P = v;
      return true;
    }
  return false;
}

void cache_store(const char* path, const std::string& key, uint32_t P) {
  if (!path) return;
  std::ofstream f(path, std::ios::app);
  f << key << " " << P << "\n";
}

}  // namespace
}  // namespace nx

extern "C" nx_status nx_autotune(const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n,
                                 uint32_t flags, const float* w, nx_program program,
                                 const uint32_t* candidates, uint32_t count, uint32_t iters,
                                 uint32_t* best_P, float* ms_per_iter, const char* cache_path) {
  if (!candidates || count == 0 || !best_P) return nx::invalid("nx_autotune: no candidates");
  if (iters == 0) return nx::invalid("nx_autotune: iters must be >= 1");
  if (program == NX_WCC) flags |= NX_WITH_TRANSPOSE;
  const std::string key = nx::tune_key(m, n, flags, program, candidates, count);
  uint32_t cached = 0;
  if (nx::cache_lookup(cache_path, key, &cached)) {
    *best_P = cached;
    if (ms_per_iter)
      for (uint32_t q = 0; q < count; ++q) ms_per_iter[q] = -1.f;
    return NX_OK;
  }
  float best = 0.f;
  uint32_t bestP = 0;
  for (uint32_t q = 0; q < count; ++q) {
    nx_graph* g = nullptr;
    NX_TRY(nx_build_dsss(src, dst, m, n, candidates[q], flags, w, &g));
    nx_params p{};
    p.alpha = 0.85f;
    nx_run_stats st{};
    nx_status s1 = nx_run(g, program, &p, iters, NX_SPU, 0, &st);  // warm-up (plans, buffers)
    if (s1 == NX_OK) s1 = nx_run(g, program, &p, iters, NX_SPU, 0, &st);
    nx_graph_free(g);
    NX_TRY(s1);
    const float per = st.iters_done ? st.ms / (float)st.iters_done : st.ms;
    if (ms_per_iter) ms_per_iter[q] = per;
    if (bestP == 0 || per < best) {
      best = per;
      bestP = candidates[q];
    }
  }
  *best_P = bestP;
  nx::cache_store(cache_path, key, bestP);
  return NX_OK;
}
