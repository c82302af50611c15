// Autotuners (the paper's Exp 2, Section IV-B2, finds P = 12..48 good on its
// CPU; here the partition and the tile and batch shapes below it are timed on
// the device). Results can be cached in a plain text file, one
// "key best_index" line per tuned workload and candidate list.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "nx_internal.cuh"

namespace nx {
namespace {

std::string device_name() {
  cudaDeviceProp prop{};
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  std::string name = prop.name;
  for (char& ch : name)
    if (ch == ' ') ch = '_';
  return name;
}

std::string shape_key(uint64_t m, uint32_t n, uint32_t flags, nx_program prog, const nx_shape* cand,
                      uint32_t count) {
  std::ostringstream k;
  k << device_name() << "|n=" << n << "|m=" << m << "|flags=" << flags << "|prog=" << (int)prog
    << "|shapes=";
  for (uint32_t q = 0; q < count; ++q)
    k << (q ? ";" : "") << cand[q].P << "," << cand[q].tile_cap_log2 << ","
      << cand[q].tile_edges_log2;
  return k.str();
}

bool cache_lookup(const char* path, const std::string& key, uint32_t count, uint32_t* idx) {
  if (!path) return false;
  std::ifstream f(path);
  std::string k;
  uint32_t v;
  while (f >> k >> v)
    if (k == key && v < count) {
      *idx = v;
      return true;
    }
  return false;
}

void cache_store(const char* path, const std::string& key, uint32_t idx) {
  if (!path) return;
  std::ofstream f(path, std::ios::app);
  f << key << " " << idx << "\n";
}

}  // namespace
}  // namespace nx

extern "C" nx_status nx_autotune_shape(const uint32_t* src, const uint32_t* dst, uint64_t m,
                                       uint32_t n, uint32_t flags, const float* w,
                                       nx_program program, const nx_shape* candidates,
                                       uint32_t count, uint32_t iters, uint32_t* best,
                                       float* ms_per_iter, const char* cache_path) {
  if (!candidates || count == 0 || !best) return nx::invalid("nx_autotune: no candidates");
  if (iters == 0) return nx::invalid("nx_autotune: iters must be >= 1");
  if ((int)program < 0 || (int)program > 5) return nx::invalid("nx_autotune: unknown program");
  if (program == NX_WCC || program == NX_SCC) flags |= NX_WITH_TRANSPOSE;
  flags &= ~(NX_TILE_CAP_LOG2(0xF) | NX_TILE_EDGES_LOG2(0x1F));  // the candidates set the shape
  const std::string key = nx::shape_key(m, n, flags, program, candidates, count);
  uint32_t cached = 0;
  if (nx::cache_lookup(cache_path, key, count, &cached)) {
    *best = cached;
    if (ms_per_iter)
      for (uint32_t q = 0; q < count; ++q) ms_per_iter[q] = -1.f;
    return NX_OK;
  }
  float best_ms = 0.f;
  uint32_t best_q = count;
  for (uint32_t q = 0; q < count; ++q) {
    const nx_shape& c = candidates[q];
    const uint32_t f = flags | NX_TILE_CAP_LOG2(c.tile_cap_log2) | NX_TILE_EDGES_LOG2(c.tile_edges_log2);
    nx_graph* g = nullptr;
    NX_TRY(nx_build_dsss(src, dst, m, n, c.P, f, w, &g));
    nx_params p{};
    p.alpha = 0.85f;
    nx_run_stats st{};
    nx_status s1 = nx_run(g, program, &p, iters, NX_SPU, 0, &st);  // warm-up (plans, buffers)
    if (s1 == NX_OK) s1 = nx_run(g, program, &p, iters, NX_SPU, 0, &st);
    nx_graph_free(g);
    NX_TRY(s1);
    const float per = st.iters_done ? st.ms / (float)st.iters_done : st.ms;
    if (ms_per_iter) ms_per_iter[q] = per;
    if (best_q == count || per < best_ms) {
      best_ms = per;
      best_q = q;
    }
  }
  *best = best_q;
  nx::cache_store(cache_path, key, best_q);
  return NX_OK;
}

extern "C" nx_status nx_autotune(const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n,
                                 uint32_t flags, const float* w, nx_program program,
                                 const uint32_t* candidates, uint32_t count, uint32_t iters,
                                 uint32_t* best_P, float* ms_per_iter, const char* cache_path) {
  if (!candidates || count == 0 || !best_P) return nx::invalid("nx_autotune: no candidates");
  std::vector<nx_shape> shapes(count);
  const uint32_t cap = (flags >> 8) & 0xFu, edges = (flags >> 12) & 0x1Fu;
  for (uint32_t q = 0; q < count; ++q) shapes[q] = nx_shape{candidates[q], cap, edges, 0};
  uint32_t idx = 0;
  NX_TRY(nx_autotune_shape(src, dst, m, n, flags, w, program, shapes.data(), count, iters, &idx,
                           ms_per_iter, cache_path));
  *best_P = candidates[idx];
  return NX_OK;
}

extern "C" nx_status nx_set_batch_shape(nx_graph* g, uint32_t rows, uint32_t sub) {
  if (!g) return nx::invalid("nx_set_batch_shape: graph is NULL");
  if (rows != 2 && rows != 4 && rows != 8)
    return nx::invalid("nx_set_batch_shape: rows in flight must be 2, 4 or 8");
  if (sub != 32 && sub != 64 && sub != 128 && sub != 256)
    return nx::invalid("nx_set_batch_shape: sub-tile must be 32, 64, 128 or 256 destinations");
  g->ppr_rows = rows;
  g->ppr_sub = sub;
  return NX_OK;
}

extern "C" nx_status nx_autotune_ppr_batch(nx_graph* g, const float* teleport, uint32_t B,
                                           uint32_t iters, float alpha, int32_t ptrs_are_device,
                                           const nx_batch_shape* candidates, uint32_t count,
                                           uint32_t* best, float* ms_per_iter,
                                           const char* cache_path) {
  if (!g || !teleport || !candidates || count == 0 || !best)
    return nx::invalid("nx_autotune_ppr_batch: NULL argument or no candidates");
  if (iters == 0) return nx::invalid("nx_autotune_ppr_batch: iters must be >= 1");
  for (uint32_t q = 0; q < count; ++q) {
    const nx_batch_shape& c = candidates[q];
    if ((c.rows != 2 && c.rows != 4 && c.rows != 8) ||
        (c.sub != 32 && c.sub != 64 && c.sub != 128 && c.sub != 256))
      return nx::invalid("nx_autotune_ppr_batch: a candidate shape is out of range");
  }
  nx_graph_info info{};
  NX_TRY(nx_graph_get_info(g, &info));
  std::ostringstream k;
  k << nx::device_name() << "|batch|n=" << info.n << "|m=" << info.m << "|P=" << info.P
    << "|tiles=" << info.ntiles << "|B=" << (B <= 32 ? 32 : 64) << "|shapes=";
  for (uint32_t q = 0; q < count; ++q) k << (q ? ";" : "") << candidates[q].rows << "," << candidates[q].sub;
  const std::string key = k.str();
  uint32_t cached = 0;
  if (nx::cache_lookup(cache_path, key, count, &cached)) {
    *best = cached;
    g->ppr_rows = candidates[cached].rows;
    g->ppr_sub = candidates[cached].sub;
    if (ms_per_iter)
      for (uint32_t q = 0; q < count; ++q) ms_per_iter[q] = -1.f;
    return NX_OK;
  }
  // ranks go where the teleport lives (a scratch buffer either way)
  nx::DevBuf out;
  std::vector<float> host_out;
  float* ranks = nullptr;
  if (ptrs_are_device) {
    NX_TRY(out.alloc((size_t)info.n * B * 4));
    ranks = out.as<float>();
  } else {
    host_out.resize((size_t)info.n * B);
    ranks = host_out.data();
  }
  const uint32_t rows0 = g->ppr_rows, sub0 = g->ppr_sub;
  float best_ms = 0.f;
  uint32_t best_q = count;
  for (uint32_t q = 0; q < count; ++q) {
    g->ppr_rows = candidates[q].rows;
    g->ppr_sub = candidates[q].sub;
    nx_run_stats st{};
    nx_status s1 = nx_run_ppr_batch(g, teleport, B, iters, alpha, ranks, ptrs_are_device, &st);
    if (s1 == NX_OK)  // the first run was the warm-up
      s1 = nx_run_ppr_batch(g, teleport, B, iters, alpha, ranks, ptrs_are_device, &st);
    if (s1 != NX_OK) {
      g->ppr_rows = rows0;
      g->ppr_sub = sub0;
      return s1;
    }
    const float per = st.ms / (float)iters;
    if (ms_per_iter) ms_per_iter[q] = per;
    if (best_q == count || per < best_ms) {
      best_ms = per;
      best_q = q;
    }
  }
  *best = best_q;
  g->ppr_rows = candidates[best_q].rows;
  g->ppr_sub = candidates[best_q].sub;
  nx::cache_store(cache_path, key, best_q);
  return NX_OK;
}
