// nx_pagerank_step_noalloc: one PageRank step that allocates no memory.
//
// Who needs this: callers that cannot call cudaMalloc at the time they step
// the iteration — for example an application that has already handed the
// whole device to its own memory pool (where a new cudaMalloc would fail or
// fragment the pool), or a latency-critical loop that must not pay for an
// allocation or for the device-wide synchronisation of cudaFree. nx_run()
// allocates its ping-pong arrays, plans and scratch on first use; this entry
// point uses only the graph built earlier, the caller's input and output
// arrays, and the file-scope scratch array below.
#include <mutex>

#include "nx_sweep.cuh"

namespace nx {
namespace {

// Scratch of the allocation-free step: [0, 64) scalars (dangling mass in and
// out, the completion counter), then per-tile dangling partials (double per
// destination tile), then per-block partials of the dangling-mass reduction.
// Every GPU that loads the library holds these 4 MiB until the process exits.
constexpr size_t kScratchBytes = 4u << 20;
constexpr size_t kHeadBytes = 256;
constexpr unsigned kDangBlocks = 1024;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr size_t kMaxTiles = (kScratchBytes - kHeadBytes - kDangBlocks * sizeof(double)) / sizeof(double);

std::mutex g_mu;
void* g_addr[128] = {};  // device address of the scratch array, per device

// Device address of the scratch on the current device, looked up once.
nx_status scratch_address(void** out) {
  int dev = 0;
  NX_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return invalid("nx_pagerank_step_noalloc: device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    NX_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return NX_OK;
}

// Per-block sums of the dangling mass sum_{outdeg(u) = 0} r[u].
__global__ void k_dangling_partials(const float* __restrict__ r, const uint32_t* __restrict__ od,
                                    uint32_t n, double* __restrict__ part) {
  __shared__ double red[8];
  double s = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    if (od[v] == 0) s += (double)r[v];
  for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    part[blockIdx.x] = t;
  }
}

// Folds the partials in a fixed order; one block of 256 threads.
__global__ void k_fold(const double* __restrict__ part, uint32_t k, double* __restrict__ out) {
  __shared__ double red[256];
  double t = 0.0;
  for (uint32_t q = threadIdx.x; q < k; q += blockDim.x) t += part[q];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int d = 128; d > 0; d >>= 1) {
    if ((int)threadIdx.x < d) red[threadIdx.x] += red[threadIdx.x + d];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

}  // namespace
}  // namespace nx

extern "C" nx_status nx_pagerank_step_noalloc(const nx_graph* g, float alpha, const float* r_in,
                                              float* r_out) {
  if (!g || !r_in || !r_out) return nx::invalid("nx_pagerank_step_noalloc: NULL argument");
  if (r_in == r_out) return nx::invalid("nx_pagerank_step_noalloc: r_in and r_out must differ");
  if (!(alpha >= 0.f && alpha < 1.f))
    return nx::invalid("nx_pagerank_step_noalloc: alpha must be in [0, 1)");
  if (g->relabeled)  // mapping caller order would need scratch of n entries
    return nx::invalid("nx_pagerank_step_noalloc: the graph was built with NX_RELABEL");
  const uint32_t ntiles = g->geo.ntiles, n = g->geo.n;
  if (!nx::fully_resident(g))
    return nx::invalid("nx_pagerank_step_noalloc: part of the graph is in host memory after a run "
                       "with a device budget; run nx_run without a budget first");
  if (ntiles > nx::kMaxTiles)
    return nx::invalid("nx_pagerank_step_noalloc: the graph has more destination tiles than the "
                       "4 MiB scratch holds (at most 523,232)");
  void* base = nullptr;
  NX_TRY(nx::scratch_address(&base));
  unsigned char* b = static_cast<unsigned char*>(base);
  double* dm = reinterpret_cast<double*>(b);  // [0] in, [1] out
  uint32_t* ticket = reinterpret_cast<uint32_t*>(b + 16);
  double* tile_part = reinterpret_cast<double*>(b + nx::kHeadBytes);
  double* dang_part = tile_part + ntiles;
  cudaStream_t s = nx::stream();
  // the completion counter must start at zero; the rest is overwritten
  NX_CUDA(cudaMemsetAsync(ticket, 0, sizeof(uint32_t), s));
  nx::k_dangling_partials<<<nx::kDangBlocks, 256, 0, s>>>(r_in, g->outdeg.as<uint32_t>(), n,
                                                          dang_part);
  NX_LAUNCH_CHECK();
  nx::k_fold<<<1, 256, 0, s>>>(dang_part, nx::kDangBlocks, dm);
  NX_LAUNCH_CHECK();
  nx::SweepArgs a;
  a.src[0].ew = g->fwd.ew.as<uint32_t>();
  a.src[0].piece_off = g->fwd.piece_off.as<uint64_t>();
  a.nsrc = 1;
  a.src_lo = 0;
  a.src_hi = g->geo.P;
  a.items = nullptr;  // one block per tile
  a.tile_start = g->geo.tile_start.as<uint32_t>();
  a.col_tb = g->geo.col_tb.as<uint32_t>();
  a.P = g->geo.P;
  a.L = g->geo.L;
  a.lb = g->geo.lb;
  a.n = n;
  a.tile_max = g->geo.tile_max;
  a.gsrc = r_in;
  a.vnew = r_out;
  a.cnew = nullptr;
  a.outdeg = g->outdeg.as<uint32_t>();
  a.alpha = alpha;
  a.dm_in = dm;
  a.dm_out = dm + 1;
  a.tile_part = tile_part;
  a.ticket = ticket;
  a.n_epi = ntiles;
  NX_TRY(nx::launch_sweep(nx::PK_PRD, a, ntiles, s));
  NX_CUDA(cudaStreamSynchronize(s));
  return NX_OK;
}
