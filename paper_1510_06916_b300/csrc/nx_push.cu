// Exp 1 / Table IV ablation: the sub-shard model NXgraph is compared against.
// The same sub-shards SS_ij are read in source order (the transpose DSSS holds
// each SS_ij sorted by (source, destination)), and each edge pushes its
// source's contribution into the destination accumulator with an atomic add,
// so writes from different threads to one destination conflict (Section IV-B1:
// "src-sorted" versus "dst-sorted" sub-shards).
//   coarse: one thread block per sub-shard (the coarse-grained model: the
//           skew of sub-shard sizes becomes load imbalance);
//   fine:   edge-balanced chunks of the same source-sorted order (isolates the
//           ordering from the parallel model).
// PageRank / personalized PageRank only. The destination accumulators are
// FP64: FP32 atomic adds of many small contributions into one hub lose up to a
// few percent of its rank (a 300k-edge in-star measured 1.8%), while the DSSS
// sweep compensates its FP32 sums; FP64 keeps the comparison at equal accuracy.
#include <algorithm>

#include "nx_internal.cuh"

namespace nx {
namespace {

constexpr int kPushThreads = 256;

struct PushItem {
  uint64_t e0, e1;  // edge range in the transpose DSSS
  uint32_t p;       // the piece holding e0
  uint32_t t;       // that piece's source tile
  uint32_t j;       // destination interval of the sub-shard
  uint32_t pad;
};

// Transpose-DSSS word: ((source - tile_start) << lb) | (destination - j L).
__global__ void __launch_bounds__(kPushThreads)
    k_push(const PushItem* __restrict__ items, const uint32_t* __restrict__ ew,
           const uint64_t* __restrict__ piece_off, const uint32_t* __restrict__ tile_start,
           uint32_t L, uint32_t lb, const float* __restrict__ c, double* __restrict__ acc) {
  const PushItem it = items[blockIdx.x];
  const uint32_t mask = (1u << lb) - 1u;
  double* accj = acc + (uint64_t)it.j * L;
  uint32_t p = it.p, t = it.t;
  uint64_t pend = piece_off[p + 1];
  uint32_t ubase = tile_start[t];
  for (uint64_t e = it.e0 + threadIdx.x; e < it.e1; e += kPushThreads) {
    // pieces of one sub-shard are consecutive, one per source tile
    while (e >= pend) {
      ++p;
      ++t;
      pend = piece_off[p + 1];
      ubase = tile_start[t];
    }
    const uint32_t w = ew[e];
    atomicAdd(accj + (w & mask), (double)c[ubase + (w >> lb)]);
  }
}

// r' = (1 - a) t_v + a (acc_v + Dm s_v), c' = r' / outdeg, acc cleared, and the
// per-block dangling partials of r'.
__global__ void k_push_apply(uint32_t n, float alpha, const float* __restrict__ tele,
                             int dang_by_tele, const double* __restrict__ dm_in,
                             const uint32_t* __restrict__ outdeg, double* __restrict__ acc,
                             float* __restrict__ r, float* __restrict__ c,
                             double* __restrict__ part) {
  __shared__ double red[kPushThreads / 32];
  const float inv_n = 1.0f / (float)n;
  const float dm = (float)(*dm_in);
  double s = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const float tv = tele ? tele[v] : inv_n;
    const float spread = dang_by_tele ? tv : inv_n;
    const float rv = (1.0f - alpha) * tv + alpha * ((float)acc[v] + dm * spread);
    acc[v] = 0.0;
    r[v] = rv;
    const uint32_t od = outdeg[v];
    c[v] = od ? rv / (float)od : 0.0f;
    if (od == 0) s += (double)rv;
  }
  for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int q = 0; q < kPushThreads / 32; ++q) tot += red[q];
    part[blockIdx.x] = tot;
  }
}

// Fixed-order fold of the partials (one block).
__global__ void k_push_fold(const double* __restrict__ part, uint32_t k, double* __restrict__ out) {
  __shared__ double red[kPushThreads];
  double t = 0.0;
  for (uint32_t q = threadIdx.x; q < k; q += kPushThreads) t += part[q];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int d = kPushThreads / 2; d > 0; d >>= 1) {
    if ((int)threadIdx.x < d) red[threadIdx.x] += red[threadIdx.x + d];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// Items over the transpose DSSS: sub-shard SS_ij is the run of pieces
// (row j, tiles of column i), edges sorted by (source, destination).
std::vector<PushItem> push_items(const nx_graph* g, bool coarse, uint64_t chunk) {
  const uint32_t P = g->geo.P;
  const auto& tb = g->geo.h_col_tb;
  const auto& po = g->tr.h_piece_off;
  std::vector<PushItem> items;
  for (uint32_t i = 0; i < P; ++i) {
    const uint32_t nt = tb[i + 1] - tb[i];
    if (nt == 0) continue;
    for (uint32_t j = 0; j < P; ++j) {
      const uint64_t pf = piece_index(P, tb[i], nt, j, tb[i]);
      const uint64_t e0 = po[pf], e1 = po[pf + nt];
      if (e1 == e0) continue;
      const uint64_t step = coarse ? e1 - e0 : chunk;
      uint64_t p = pf;
      for (uint64_t e = e0; e < e1; e += step) {
        while (po[p + 1] <= e) ++p;  // the piece holding e (skips empty pieces)
        PushItem it;
        it.e0 = e;
        it.e1 = std::min(e1, e + step);
        it.p = (uint32_t)p;
        it.t = tb[i] + (uint32_t)(p - pf);
        it.j = j;
        it.pad = 0;
        items.push_back(it);
      }
    }
  }
  return items;
}

}  // namespace

nx_status push_run(nx_graph* g, const PushRun& r, uint32_t* launches, float* ms) {
  const uint32_t n = g->geo.n;
  const uint64_t chunk = std::max<uint64_t>(4096, ceil_div(g->m, 8ull * (uint64_t)num_sms()));
  const std::vector<PushItem> h = push_items(g, r.coarse, chunk);
  DevBuf items, acc, part;
  NX_TRY(items.alloc(std::max<size_t>(h.size(), 1) * sizeof(PushItem)));
  NX_TRY(acc.alloc((size_t)n * 8));
  const unsigned ga = (unsigned)std::min<uint64_t>(ceil_div(n, kPushThreads), (uint64_t)num_sms() * 8);
  NX_TRY(part.alloc((size_t)ga * 8));
  if (!h.empty())
    NX_CUDA(cudaMemcpyAsync(items.p, h.data(), h.size() * sizeof(PushItem), cudaMemcpyHostToDevice,
                            stream()));
  NX_CUDA(cudaMemsetAsync(acc.p, 0, (size_t)n * 8, stream()));
  NX_CUDA(cudaStreamSynchronize(stream()));  // h is a host temporary
  EventPair ev;
  NX_TRY(ev.create());
  NX_CUDA(cudaEventRecord(ev.e0, stream()));
  for (uint32_t it = 0; it < r.iters; ++it) {
    const int c = g->cur, nx_ = 1 - g->cur;
    if (!h.empty()) {
      k_push<<<(unsigned)h.size(), kPushThreads, 0, stream()>>>(
          items.as<PushItem>(), g->tr.ew.as<uint32_t>(), g->tr.piece_off.as<uint64_t>(),
          g->geo.tile_start.as<uint32_t>(), g->geo.L, g->geo.lb, g->aux[c].as<float>(),
          acc.as<double>());
      NX_LAUNCH_CHECK();
      ++*launches;
    }
    k_push_apply<<<ga, kPushThreads, 0, stream()>>>(
        n, r.alpha, r.tele, r.dang_by_tele, r.dm + c, g->outdeg.as<uint32_t>(), acc.as<double>(),
        g->val[nx_].as<float>(), g->aux[nx_].as<float>(), part.as<double>());
    NX_LAUNCH_CHECK();
    k_push_fold<<<1, kPushThreads, 0, stream()>>>(part.as<double>(), ga, r.dm + nx_);
    NX_LAUNCH_CHECK();
    *launches += 2;
    g->cur = nx_;
  }
  NX_CUDA(cudaEventRecord(ev.e1, stream()));
  return ev.elapsed(ms);
}

}  // namespace nx
