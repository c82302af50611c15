// Degree-ordered vertex ids (the "degreeing" step of Section III-A maps the
// input's vertex indices to the ids the sharder uses). Here the map is a
// permutation of [0, n): internal id k is the caller vertex with the k-th
// largest out-degree (ties by caller id), so the most-read source values share
// cache lines. No vertex is dropped, so n and every result are unchanged; the
// ABI maps vertex-indexed inputs and outputs between the two numberings.
#include <algorithm>

#include "nx_internal.cuh"

namespace nx {
namespace {

__global__ void k_max_u32(const uint32_t* __restrict__ a, uint32_t n, uint32_t* __restrict__ out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint32_t mx = 0;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    mx = max(mx, a[v]);
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

// key = max_deg - outdeg (ascending keys = descending degree), value = v: the
// stable sort leaves equal degrees in id order.
__global__ void k_order_keys(const uint32_t* __restrict__ od, uint32_t n, uint32_t max_deg,
                             uint64_t* __restrict__ keys, uint32_t* __restrict__ ids) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    keys[v] = max_deg - od[v];
    ids[v] = (uint32_t)v;
  }
}

__global__ void k_order_perm(const uint32_t* __restrict__ ids, uint32_t n,
                             uint32_t* __restrict__ old_of_new, uint32_t* __restrict__ new_of_old) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
    const uint32_t old = ids[k];
    old_of_new[k] = old;
    new_of_old[old] = (uint32_t)k;
  }
}

__global__ void k_rename(const uint32_t* __restrict__ map, const uint32_t* s, const uint32_t* d,
                         uint64_t m, uint32_t* s_out, uint32_t* d_out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    const uint32_t a = s[e], b = d[e];
    s_out[e] = map[a];
    d_out[e] = map[b];
  }
}

__global__ void k_gather(const uint32_t* __restrict__ idx, const uint32_t* __restrict__ in,
                         uint64_t n, uint32_t* __restrict__ out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride)
    out[k] = in[idx[k]];
}

unsigned grid_of(uint64_t work) {
  return (unsigned)std::min<uint64_t>(ceil_div(work ? work : 1, 256), (uint64_t)num_sms() * 8);
}

}  // namespace

nx_status relabel_edges(nx_graph* g, const uint32_t* s, const uint32_t* d, uint64_t m,
                        uint32_t* s_out, uint32_t* d_out, const uint32_t* outdeg) {
  const uint32_t n = g->geo.n;
  if (n == 0) return invalid("relabel_edges: the graph's n is not set");
  DevBuf keys, ids, mx;
  NX_TRY(mx.alloc(4));
  NX_CUDA(cudaMemsetAsync(mx.p, 0, 4, stream()));
  k_max_u32<<<grid_of(n), 256, 0, stream()>>>(outdeg, n, mx.as<uint32_t>());
  NX_LAUNCH_CHECK();
  uint32_t max_deg = 0;
  NX_CUDA(cudaMemcpyAsync(&max_deg, mx.p, 4, cudaMemcpyDeviceToHost, stream()));
  NX_CUDA(cudaStreamSynchronize(stream()));
  NX_TRY(keys.alloc((uint64_t)n * 8));
  NX_TRY(ids.alloc((uint64_t)n * 4));
  k_order_keys<<<grid_of(n), 256, 0, stream()>>>(outdeg, n, max_deg, keys.as<uint64_t>(),
                                                 ids.as<uint32_t>());
  NX_LAUNCH_CHECK();
  NX_TRY(radix_sort_u64(keys, &ids, n, bits_for((uint64_t)max_deg + 1)));
  NX_TRY(g->old_of_new.alloc((uint64_t)n * 4));
  NX_TRY(g->new_of_old.alloc((uint64_t)n * 4));
  k_order_perm<<<grid_of(n), 256, 0, stream()>>>(ids.as<uint32_t>(), n, g->old_of_new.as<uint32_t>(),
                                                 g->new_of_old.as<uint32_t>());
  NX_LAUNCH_CHECK();
  if (m && s_out) {
    k_rename<<<grid_of(m), 256, 0, stream()>>>(g->new_of_old.as<uint32_t>(), s, d, m, s_out, d_out);
    NX_LAUNCH_CHECK();
  }
  NX_CUDA(cudaStreamSynchronize(stream()));  // od and keys are freed on return
  g->relabeled = true;
  return NX_OK;
}

nx_status rename_edges(const nx_graph* g, uint32_t* s, uint32_t* d, uint64_t m) {
  if (!m) return NX_OK;
  k_rename<<<grid_of(m), 256, 0, stream()>>>(g->new_of_old.as<uint32_t>(), s, d, m, s, d);
  NX_LAUNCH_CHECK();
  return NX_OK;
}

nx_status gather_u32(const uint32_t* idx, const void* in, void* out, uint64_t n) {
  if (!n) return NX_OK;
  k_gather<<<grid_of(n), 256, 0, stream()>>>(idx, static_cast<const uint32_t*>(in), n,
                                             static_cast<uint32_t*>(out));
  NX_LAUNCH_CHECK();
  return NX_OK;
}

nx_status vertex_to_internal(const nx_graph* g, const void* in, void* out) {
  const uint64_t n = g->geo.n;
  if (!g->relabeled) {
    NX_CUDA(cudaMemcpyAsync(out, in, n * 4, cudaMemcpyDeviceToDevice, stream()));
    return NX_OK;
  }
  return gather_u32(g->old_of_new.as<uint32_t>(), in, out, n);
}

nx_status vertex_to_caller(const nx_graph* g, const void* in, void* out) {
  const uint64_t n = g->geo.n;
  if (!g->relabeled) {
    NX_CUDA(cudaMemcpyAsync(out, in, n * 4, cudaMemcpyDeviceToDevice, stream()));
    return NX_OK;
  }
  return gather_u32(g->new_of_old.as<uint32_t>(), in, out, n);
}

}  // namespace nx

extern "C" nx_status nx_get_relabel(const nx_graph* g, uint32_t* old_of_new, uint64_t count,
                                    int32_t out_is_device) {
  if (!g || !old_of_new) return nx::invalid("nx_get_relabel: NULL argument");
  if (!g->relabeled) return nx::invalid("nx_get_relabel: the graph was built without NX_RELABEL");
  if (count != g->geo.n) return nx::invalid("nx_get_relabel: count must equal n");
  NX_CUDA(cudaMemcpyAsync(old_of_new, g->old_of_new.p, count * 4,
                          out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          nx::stream()));
  NX_CUDA(cudaStreamSynchronize(nx::stream()));
  return NX_OK;
}
