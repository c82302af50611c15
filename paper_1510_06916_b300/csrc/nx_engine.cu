// Update engine (Section III-B): Initialize, the per-iteration schedules of
// SPU / DPU / MPU (Algorithms 5-7), activity-driven termination (Algorithm 1),
// value access, and the I/O model of Table II.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "nx_sweep.cuh"

namespace nx {
namespace {

constexpr uint32_t kInf = 0xFFFFFFFFu;

// ---------------------------------------------------------------- init kernels
__global__ void k_init_pr(uint32_t n, const float* __restrict__ tele, const float* __restrict__ rin,
                          const uint32_t* __restrict__ outdeg, float* __restrict__ r,
                          float* __restrict__ c, double* __restrict__ part) {
  __shared__ double red[8];
  double s = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    float rv = rin ? rin[v] : (tele ? tele[v] : 1.0f / (float)n);
    r[v] = rv;
    uint32_t od = outdeg[v];
    if (c) c[v] = od ? rv / (float)od : 0.0f;
    if (od == 0) s += (double)rv;
  }
  for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    part[blockIdx.x] = t;
  }
}

// One block of 256 threads; a fixed summation order (deterministic).
__global__ void k_sum_parts(const double* __restrict__ part, uint32_t k, double* __restrict__ out) {
  __shared__ double red[256];
  double t = 0.0;
  for (uint32_t q = threadIdx.x; q < k; q += blockDim.x) t += part[q];
  red[threadIdx.x] = t;
  __syncthreads();
  for (int d = blockDim.x / 2; d > 0; d >>= 1) {
    if ((int)threadIdx.x < d) red[threadIdx.x] += red[threadIdx.x + d];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// WCC labels start as the caller's ids (ids: internal -> caller, nullable).
__global__ void k_init_min(uint32_t n, int bfs, uint32_t root, const uint32_t* __restrict__ ids,
                           uint32_t* __restrict__ v) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride)
    v[x] = bfs ? (x == root ? 0u : kInf) : (ids ? ids[x] : (uint32_t)x);
}

unsigned grid_for(uint64_t work) {
  uint64_t b = ceil_div(work ? work : 1, 256);
  return (unsigned)std::min<uint64_t>(b, (uint64_t)num_sms() * 8);
}

ProgKind kind_of(nx_program p) {
  switch (p) {
    case NX_WPR: return PK_WPR;
    case NX_BFS: return PK_BFS;
    case NX_WCC: return PK_WCC;
    default: return PK_PR;
  }
}
bool is_min(nx_program p) { return p == NX_BFS || p == NX_WCC; }

// ---------------------------------------------------------------- plans
struct PlanOut {
  std::vector<Item> items;
  std::vector<uint64_t> cost;  // edges per item (sort key)
  uint32_t slots = 0;
};

uint64_t piece_len(const nx_graph* g, const Dsss& d, uint32_t i, uint32_t t, uint32_t j) {
  const auto& tb = g->geo.h_col_tb;
  uint64_t pc = piece_index(g->geo.P, tb[j], tb[j + 1] - tb[j], i, t);
  return d.h_piece_off[pc + 1] - d.h_piece_off[pc];
}

uint64_t target_block_edges(uint64_t total) {
  uint64_t e = total / ((uint64_t)num_sms() * 8);
  return std::max<uint64_t>(16384, e);
}

// Appends the items to `out` heaviest first: a counting sort on the cost
// rounded down to 8 steps per octave (ties and near-ties in the order they
// were made), linear in the item count.
void emit_heaviest_first(const std::vector<std::pair<uint64_t, uint32_t>>& key,
                         const std::vector<Item>& made, PlanOut& out) {
  auto bucket = [](uint64_t c) -> uint32_t {  // c >= 1
    const uint32_t e = 63u - (uint32_t)__builtin_clzll(c);
    const uint32_t frac = e >= 3 ? (uint32_t)(c >> (e - 3)) & 7u : (uint32_t)(c << (3 - e)) & 7u;
    return e * 8 + frac;
  };
  constexpr uint32_t kBuckets = 64 * 8;
  std::vector<uint32_t> start(kBuckets + 1, 0);
  for (const auto& k : key) ++start[kBuckets - 1 - bucket(k.first)];
  uint32_t acc = 0;
  for (uint32_t b = 0; b <= kBuckets; ++b) {
    const uint32_t c = start[b];
    start[b] = acc;
    acc += c;
  }
  std::vector<uint32_t> order(key.size());
  for (uint32_t q = 0; q < (uint32_t)key.size(); ++q)
    order[start[kBuckets - 1 - bucket(key[q].first)]++] = q;
  const size_t base = out.items.size();
  out.items.resize(base + key.size());
  out.cost.resize(base + key.size());
  for (size_t q = 0; q < order.size(); ++q) {
    out.items[base + q] = made[key[order[q]].second];
    out.cost[base + q] = key[order[q]].first;
  }
}

// Items of one tile (or piece) of `cost` edges: split into k parts of about
// `blk` edges when it is heavier than 2 blk.
void make_items(uint32_t t, uint64_t cost, bool allow_split, uint64_t blk, uint32_t row,
                uint32_t sx, std::vector<std::pair<uint64_t, uint32_t>>& key,
                std::vector<Item>& made, PlanOut& out) {
  uint32_t k = 1;
  if (allow_split && cost > 2 * blk) k = (uint32_t)ceil_div(cost, blk);
  for (uint32_t q = 0; q < k; ++q) {
    Item it{};
    it.tile = t;
    it.nsplit = k;
    it.slot = k > 1 ? out.slots : 0;
    it.sub = q;
    it.row = row;
    it.pad = sx;
    it.vbeg = cost * q / k;
    it.vend = (q + 1 == k) ? ~0ull : cost * (q + 1) / k;
    key.push_back({cost / k + 1, (uint32_t)made.size()});
    made.push_back(it);
  }
  if (k > 1) out.slots += k;
}

// Tiles of columns [c0, c1) (those in [tlo, thi) only), sweeping sources
// [i0, i1) over `ds`.
void plan_tiles(const nx_graph* g, const std::vector<const Dsss*>& ds, uint32_t i0, uint32_t i1,
                uint32_t c0, uint32_t c1, bool allow_split, uint64_t blk, PlanOut& out,
                uint32_t tlo = 0, uint32_t thi = 0xFFFFFFFFu) {
  const auto& tb = g->geo.h_col_tb;
  const uint32_t P = g->geo.P, t0 = tb[c0], t1 = tb[c1];
  // edges per tile: pieces (i, t) of one column and source are consecutive
  std::vector<uint64_t> cost((size_t)(t1 - t0), 0);
  for (uint32_t j = c0; j < c1; ++j) {
    const uint32_t nt = tb[j + 1] - tb[j];
    uint64_t* cj = cost.data() + (tb[j] - t0);
    for (const Dsss* d : ds)
      for (uint32_t i = i0; i < i1; ++i) {
        const uint64_t* po = d->h_piece_off.data() + piece_index(P, tb[j], nt, i, tb[j]);
        for (uint32_t q = 0; q < nt; ++q) cj[q] += po[q + 1] - po[q];
      }
  }
  std::vector<std::pair<uint64_t, uint32_t>> key;
  std::vector<Item> made;
  key.reserve(cost.size() + 64);
  made.reserve(cost.size() + 64);
  for (uint32_t t = std::max(t0, tlo); t < std::min(t1, thi); ++t)
    make_items(t, cost[t - t0], allow_split, blk, 0, 0, key, made, out);
  emit_heaviest_first(key, made, out);
}

// Single pieces (i, t) of row i of DSSS number `sx` for tiles of columns
// [c0, c1) (ToHub / row pass).
void plan_row(const nx_graph* g, const Dsss& d, uint32_t sx, uint32_t i, uint32_t c0, uint32_t c1,
              uint64_t blk, PlanOut& out) {
  const auto& tb = g->geo.h_col_tb;
  std::vector<std::pair<uint64_t, uint32_t>> key;
  std::vector<Item> made;
  for (uint32_t j = c0; j < c1; ++j)
    for (uint32_t t = tb[j]; t < tb[j + 1]; ++t) {
      const uint64_t cost = piece_len(g, d, i, t, j);
      if (cost) make_items(t, cost, true, blk, i, sx, key, made, out);
    }
  emit_heaviest_first(key, made, out);
}

// ---------------------------------------------------------------- buffers
nx_status ensure(DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return NX_OK;
  return b.alloc(bytes);
}

// Scalar slots (doubles): [0..1] dangling mass ping-pong; u32 counters after.
struct Scal {
  double* dm;          // [2]
  uint32_t* ticket;    // [1]
  uint32_t* act_count; // [1]
};
Scal scal_of(nx_graph* g) {
  Scal s;
  s.dm = g->scal.as<double>();
  s.ticket = reinterpret_cast<uint32_t*>(s.dm + 2);
  s.act_count = s.ticket + 1;
  return s;
}

nx_status prepare(nx_graph* g) {
  const uint64_t n = g->geo.n;
  for (int k = 0; k < 2; ++k) {
    NX_TRY(ensure(g->val[k], n * 4));
    NX_TRY(ensure(g->act[k], ((size_t)g->geo.P + 1) * 4));
  }
  if (!g->scal.p) {
    NX_TRY(g->scal.alloc(64));
    NX_CUDA(cudaMemsetAsync(g->scal.p, 0, 64, stream()));
  }
  if (!g->tile_part.p) NX_TRY(g->tile_part.alloc(((size_t)g->geo.ntiles + 1) * 8));
  if (!g->tile_ticket.p) {  // per (tile, DSSS)
    NX_TRY(g->tile_ticket.alloc((2 * (size_t)g->geo.ntiles + 1) * 4));
    NX_CUDA(cudaMemsetAsync(g->tile_ticket.p, 0, (2 * (size_t)g->geo.ntiles + 1) * 4, stream()));
  }
  return NX_OK;
}

nx_status upload_items(nx_graph*, PlanOut& plan, nx_graph::Plan& dst) {
  NX_TRY(dst.items.alloc(std::max<size_t>(plan.items.size(), 1) * sizeof(Item)));
  if (!plan.items.empty())
    NX_CUDA(cudaMemcpyAsync(dst.items.p, plan.items.data(), plan.items.size() * sizeof(Item),
                            cudaMemcpyHostToDevice, stream()));
  NX_CUDA(cudaStreamSynchronize(stream()));  // plan.items is a host temporary
  dst.slots = plan.slots;
  dst.h_cost = std::move(plan.cost);
  dst.h_items = std::move(plan.items);
  return NX_OK;
}

// Split slots are transient within a launch: one buffer sized for the largest plan.
nx_status ensure_split(nx_graph* g, uint32_t slots) {
  const uint64_t need = (uint64_t)slots * g->geo.tile_max * 8;  // hi + lo per slot
  if (g->split_buf.bytes >= std::max<uint64_t>(need, 4)) return NX_OK;
  NX_CUDA(cudaStreamSynchronize(stream()));
  return g->split_buf.alloc(std::max<uint64_t>(need, 4));
}

// ---------------------------------------------------------------- initialize
nx_status initialize(nx_graph* g, nx_program prog, const nx_params& p, const float* tele,
                     const void* resume) {
  const uint32_t n = g->geo.n;
  Scal sc = scal_of(g);
  g->cur = 0;
  if (!is_min(prog)) {
    const bool need_c = prog != NX_WPR;
    if (need_c) {
      NX_TRY(ensure(g->aux[0], (size_t)n * 4));
      NX_TRY(ensure(g->aux[1], (size_t)n * 4));
    }
    const unsigned gb = grid_for(n);
    NX_TRY(ensure(g->init_part, (size_t)gb * 8));
    DevBuf& part = g->init_part;
    const float* r0_tele = (prog == NX_PPR) ? tele : nullptr;  // PPR: r0 = t
    k_init_pr<<<gb, 256, 0, stream()>>>(n, r0_tele, static_cast<const float*>(resume),
                                        g->outdeg.as<uint32_t>(), g->val[0].as<float>(),
                                        need_c ? g->aux[0].as<float>() : nullptr, part.as<double>());
    NX_LAUNCH_CHECK();
    k_sum_parts<<<1, 256, 0, stream()>>>(part.as<double>(), gb, sc.dm);
    NX_LAUNCH_CHECK();
  } else {
    const uint32_t P = g->geo.P;
    std::vector<uint32_t> a0(P + 1, 0);
    if (resume) {
      NX_CUDA(cudaMemcpyAsync(g->val[0].p, resume, (size_t)n * 4, cudaMemcpyDeviceToDevice,
                              stream()));
      std::fill(a0.begin(), a0.begin() + P, 1u);
    } else {
      k_init_min<<<grid_for(n), 256, 0, stream()>>>(
          n, prog == NX_BFS, p.root, g->relabeled ? g->old_of_new.as<uint32_t>() : nullptr,
          g->val[0].as<uint32_t>());
      NX_LAUNCH_CHECK();
      if (prog == NX_BFS) a0[p.root / g->geo.L] = 1u;
      else std::fill(a0.begin(), a0.begin() + P, 1u);
    }
    NX_CUDA(cudaMemcpyAsync(g->act[0].p, a0.data(), (P + 1) * 4, cudaMemcpyHostToDevice, stream()));
    NX_CUDA(cudaMemsetAsync(g->act[1].p, 0, (P + 1) * 4, stream()));
    NX_CUDA(cudaStreamSynchronize(stream()));
  }
  return NX_OK;
}

// ---------------------------------------------------------------- common args
SweepArgs base_args(nx_graph* g, nx_program prog, const nx_params& p, const float* tele) {
  SweepArgs a;
  const bool tr = (prog == NX_WCC);
  a.src[0].ew = g->fwd.ew.as<uint32_t>();
  a.src[0].wt = g->fwd.wt.as<float>();
  a.src[0].piece_off = g->fwd.piece_off.as<uint64_t>();
  a.nsrc = 1;
  if (tr) {
    a.src[1].ew = g->tr.ew.as<uint32_t>();
    a.src[1].wt = g->tr.wt.as<float>();
    a.src[1].piece_off = g->tr.piece_off.as<uint64_t>();
    a.nsrc = 2;
  }
  a.tile_start = g->geo.tile_start.as<uint32_t>();
  a.col_tb = g->geo.col_tb.as<uint32_t>();
  a.P = g->geo.P;
  a.L = g->geo.L;
  a.lb = g->geo.lb;
  a.n = g->geo.n;
  a.tile_max = g->geo.tile_max;
  a.outdeg = g->outdeg.as<uint32_t>();
  a.tele = (prog == NX_PPR || prog == NX_WPR) ? tele : nullptr;
  a.dang_by_tele = (prog == NX_PPR) ? 1 : 0;
  a.alpha = p.alpha;
  a.tile_part = g->tile_part.as<double>();
  Scal sc = scal_of(g);
  a.ticket = sc.ticket;
  a.act_count = sc.act_count;
  a.split = g->split_buf.p;
  a.tile_ticket = g->tile_ticket.as<uint32_t>();
  a.n_epi = g->geo.ntiles;
  a.src_lo = 0;
  a.src_hi = g->geo.P;
  a.hub_off[0] = g->fwd.hub_off.as<uint64_t>();
  a.hub_dst[0] = g->fwd.hub_dst.as<uint16_t>();
  a.hubs[0] = g->hubs.p;
  if (tr) {
    a.hub_off[1] = g->tr.hub_off.as<uint64_t>();
    a.hub_dst[1] = g->tr.hub_dst.as<uint16_t>();
    a.hubs[1] = g->hubs_t.p;
  }
  // Flattened step schedule (a tile's pieces as one sequence of warp steps):
  // measured faster for every program once the shared-memory carveout leaves
  // L1 to the gathers -- PageRank at R-MAT scale 26 by 3% (P = 16) to 16%
  // (P = 64), where pieces are short; BFS / WCC skip inactive pieces in it.
  const uint32_t npieces = (uint32_t)a.nsrc * g->geo.P;
  a.flat_cap = npieces <= 256 ? npieces : 0;
  return a;
}

void set_iter_ptrs(nx_graph* g, nx_program prog, SweepArgs& a) {
  const int c = g->cur, n = 1 - g->cur;
  Scal sc = scal_of(g);
  a.gsrc = (prog == NX_WPR || is_min(prog)) ? g->val[c].p : g->aux[c].p;
  a.vold = g->val[c].p;
  a.vnew = g->val[n].p;
  a.cnew = (prog == NX_PR || prog == NX_PPR) ? g->aux[n].as<float>() : nullptr;
  a.dm_in = sc.dm + c;
  a.dm_out = sc.dm + n;
  if (is_min(prog)) {
    a.act_in = g->act[c].as<uint32_t>();
    a.act_out = g->act[n].as<uint32_t>();
  } else {
    a.act_in = nullptr;
    a.act_out = nullptr;
  }
}

uint64_t bytes_per_sweep(const nx_graph* g, nx_program prog, uint64_t edges) {
  const uint64_t n = g->geo.n;
  uint64_t b = 4 * edges;             // edge words
  if (prog == NX_WPR) b += 4 * edges;  // weights
  if (is_min(prog)) b += 12 * n;       // gather-read, previous, new
  else b += 16 * n;                    // gather-read c (r), write r, write c (tele), outdeg
  return b;
}

// One SPU iteration: every tile of every column in one launch (Algorithm 5;
// the order of sub-shards does not matter in SPU, Section III-B1).
nx_status spu_iteration(nx_graph* g, nx_program prog, SweepArgs& a, uint32_t nitems) {
  set_iter_ptrs(g, prog, a);
  a.mode = 0;
  NX_TRY(launch_sweep(kind_of(prog), a, nitems, stream()));
  g->cur ^= 1;
  return NX_OK;
}

// One DPU iteration (Algorithm 6): ToHub over every piece (row-major items),
// then FromHub + epilogue per destination tile.
nx_status dpu_iteration(nx_graph* g, nx_program prog, SweepArgs& a, uint32_t n_tohub,
                        uint32_t n_fromhub) {
  set_iter_ptrs(g, prog, a);
  const Item* all = a.items;
  SweepArgs th = a;
  th.mode = 1;
  th.q_res = 0;
  th.items = all;
  NX_TRY(launch_sweep(kind_of(prog), th, n_tohub, stream()));
  SweepArgs fh = a;
  fh.mode = 0;
  fh.items = all + n_tohub;
  fh.src_lo = fh.src_hi = 0;
  fh.hub_lo = 0;
  fh.hub_hi = g->geo.P;
  NX_TRY(launch_sweep(kind_of(prog), fh, n_fromhub, stream()));
  g->cur ^= 1;
  return NX_OK;
}

}  // namespace

// ---------------------------------------------------------------- residency
// Whole-array moves between the device and pinned host memory (no-ops when
// the array is already where it is asked to be).
nx_status move_to_host(DevBuf& d, PinnedBuf& h) {
  if (!d.p) return NX_OK;
  NX_TRY(h.alloc(d.bytes));
  NX_CUDA(cudaMemcpyAsync(h.p, d.p, d.bytes, cudaMemcpyDeviceToHost, stream()));
  NX_CUDA(cudaStreamSynchronize(stream()));
  d.release();
  return NX_OK;
}

nx_status move_to_device(PinnedBuf& h, DevBuf& d) {
  if (d.p || !h.p) return NX_OK;
  NX_TRY(d.alloc(h.bytes));
  NX_CUDA(cudaMemcpyAsync(d.p, h.p, h.bytes, cudaMemcpyHostToDevice, stream()));
  NX_CUDA(cudaStreamSynchronize(stream()));
  h.release();
  return NX_OK;
}

nx_status set_edge_residency(Dsss& d, uint64_t dev_words, uint64_t host_first) {
  dev_words = std::min(dev_words, d.words);
  host_first = std::min(host_first, dev_words);
  const bool need_host = dev_words < d.words;
  cudaStream_t s = stream();
  if (need_host && (!d.h_ew.p || d.h_ew_first > host_first)) {
    // a host image of words [host_first, words): the part below the old image
    // comes from the device (which holds it: h_ew_first <= dev_words)
    PinnedBuf nh;
    NX_TRY(nh.alloc((d.words - host_first) * 4));
    const uint64_t dev_end = d.h_ew.p ? d.h_ew_first : d.words;
    if (dev_end > host_first)
      NX_CUDA(cudaMemcpyAsync(nh.p, d.ew.as<uint32_t>() + host_first, (dev_end - host_first) * 4,
                              cudaMemcpyDeviceToHost, s));
    NX_CUDA(cudaStreamSynchronize(s));
    if (d.h_ew.p)
      memcpy(nh.as<uint32_t>() + (dev_end - host_first), d.h_ew.p, (d.words - dev_end) * 4);
    std::swap(nh.p, d.h_ew.p);
    std::swap(nh.bytes, d.h_ew.bytes);
    d.h_ew_first = host_first;
  }
  if (dev_words != d.dev_words) {
    // the new device prefix: words the device held, then words from the host image
    DevBuf nb;
    if (dev_words) {
      NX_TRY(nb.alloc(dev_words * 4));
      const uint64_t kept = std::min(dev_words, d.dev_words);
      if (kept)
        NX_CUDA(cudaMemcpyAsync(nb.p, d.ew.p, kept * 4, cudaMemcpyDeviceToDevice, s));
      if (dev_words > kept)
        NX_CUDA(cudaMemcpyAsync(nb.as<uint32_t>() + kept, d.h_ew.as<uint32_t>() + (kept - d.h_ew_first),
                                (dev_words - kept) * 4, cudaMemcpyHostToDevice, s));
    }
    NX_CUDA(cudaStreamSynchronize(s));
    d.ew = std::move(nb);
    d.dev_words = dev_words;
  }
  if (!need_host && d.h_ew.p) {
    d.h_ew.release();
    d.h_ew_first = 0;
  }
  return NX_OK;
}

nx_status ensure_resident(nx_graph* g) {
  Dsss* all_ds[2] = {&g->fwd, g->has_tr ? &g->tr : nullptr};
  for (Dsss* d : all_ds) {
    if (!d) continue;
    NX_TRY(set_edge_residency(*d, d->words, 0));
    NX_TRY(move_to_device(d->h_piece_pin, d->piece_off));
    NX_TRY(move_to_device(d->h_hub_off, d->hub_off));
    NX_TRY(move_to_device(d->h_hub_dst, d->hub_dst));
    NX_TRY(move_to_device(d->h_wt, d->wt));
  }
  NX_TRY(move_to_device(g->h_orig_src, g->orig_src));
  NX_TRY(move_to_device(g->h_orig_dst, g->orig_dst));
  if (g->oc.built) {
    NX_TRY(move_to_device(g->oc.h_ew, g->oc.ew));
    NX_TRY(move_to_device(g->oc.h_hub_dst, g->oc.hub_dst));
    if (!g->oc.hub_val.p) NX_TRY(g->oc.hub_val.alloc(std::max<uint64_t>(g->oc.H, 1) * 4));
  }
  return NX_OK;
}

bool fully_resident(const nx_graph* g) {
  const Dsss* all_ds[2] = {&g->fwd, g->has_tr ? &g->tr : nullptr};
  for (const Dsss* d : all_ds)
    if (d && (d->dev_words != d->words || d->h_hub_dst.p || d->h_wt.p || d->h_piece_pin.p ||
              d->h_hub_off.p))
      return false;
  return !g->h_orig_src.p && !g->h_orig_dst.p && !g->oc.h_ew.p && !g->oc.h_hub_dst.p;
}

namespace {

// ---------------------------------------------------------------- shard streaming
// A streamed column is swept in bands of consecutive source intervals whose
// edge words (over the DSSS of the sweep) fit one staging buffer of this many
// words (64 MB), unless one sub-shard alone is larger; tile accumulators carry
// between the bands of a column in device memory.
constexpr uint64_t kStreamChunkWords = 16ull << 20;

struct StreamBand {
  uint32_t j, i0, i1;     // column and its source intervals [i0, i1)
  uint32_t t0, t1;        // its tiles [t0, t1) (the whole column unless a sub-shard is split)
  uint64_t e0[2], e1[2];  // word range of each DSSS (aligned, padded)
  bool first, last;       // the band starts / ends the source range of its tiles
};

// Bands of the streamed columns [Jc, P) (deterministic: plans are cached):
// consecutive source intervals of a column up to kStreamChunkWords words; a
// single sub-shard above that is cut into ranges of its tiles (its pieces
// (i, t) are consecutive), so the staging buffers stay about that size
// however skewed the graph (degree-ordered ids put most edges in SS_00).
std::vector<StreamBand> stream_bands(const nx_graph* g, const std::vector<const Dsss*>& ds,
                                     uint32_t Jc) {
  const uint32_t P = g->geo.P;
  const auto& tb = g->geo.h_col_tb;
  std::vector<StreamBand> out;
  for (uint32_t j = Jc; j < P; ++j) {
    const uint32_t nt = tb[j + 1] - tb[j];
    if (nt == 0) continue;  // empty trailing interval: no tiles
    // start of piece (i, t) in DSSS s; (i, tb[j + 1]) is the end of SS_ij and
    // (P, tb[j]) the column's end
    auto at = [&](size_t sx, uint32_t i, uint32_t t) {
      return ds[sx]->h_piece_off[piece_index(P, tb[j], nt, i, t)];
    };
    auto words = [&](uint32_t ia, uint32_t ta, uint32_t ib, uint32_t tb_) {
      uint64_t w = 0;
      for (size_t sx = 0; sx < ds.size(); ++sx) w += at(sx, ib, tb_) - at(sx, ia, ta);
      return w;
    };
    auto push = [&](uint32_t i0, uint32_t i1, uint32_t t0, uint32_t t1, uint32_t ta, uint32_t ie,
                    uint32_t te) {
      StreamBand b{};
      b.j = j;
      b.i0 = i0;
      b.i1 = i1;
      b.t0 = t0;
      b.t1 = t1;
      for (size_t sx = 0; sx < ds.size(); ++sx) {
        b.e0[sx] = at(sx, i0, ta) & ~(kEdgeAlign - 1);
        b.e1[sx] = round_up(at(sx, ie, te), kEdgeAlign) + kEdgeAlign;
      }
      b.first = (i0 == 0);
      b.last = (i1 == P);
      out.push_back(b);
    };
    uint32_t i0 = 0;
    while (i0 < P) {
      uint32_t i1 = i0 + 1;
      while (i1 < P && words(i0, tb[j], i1 + 1, tb[j]) <= kStreamChunkWords) ++i1;
      if (i1 == i0 + 1 && words(i0, tb[j], i0 + 1, tb[j]) > kStreamChunkWords) {
        // one sub-shard above the chunk: ranges of its tiles
        for (uint32_t t = tb[j]; t < tb[j + 1];) {
          uint32_t te = t + 1;
          while (te < tb[j + 1] && words(i0, t, i0, te + 1) <= kStreamChunkWords) ++te;
          push(i0, i0 + 1, t, te, t, i0, te);
          t = te;
        }
      } else {
        push(i0, i1, tb[j], tb[j + 1], tb[j], i1, tb[j]);
      }
      i0 = i1;
    }
  }
  return out;
}

struct Streamer {
  cudaStream_t side = nullptr;
  cudaEvent_t copied[2] = {nullptr, nullptr}, used[2] = {nullptr, nullptr};
  ~Streamer() {
    if (side) cudaStreamSynchronize(side);  // no copy outlives the run (early error returns)
    for (int k = 0; k < 2; ++k) {
      if (copied[k]) cudaEventDestroy(copied[k]);
      if (used[k]) cudaEventDestroy(used[k]);
    }
    if (side) cudaStreamDestroy(side);
  }
  nx_status init() {
    NX_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
      NX_CUDA(cudaEventCreateWithFlags(&copied[k], cudaEventDisableTiming));
      NX_CUDA(cudaEventCreateWithFlags(&used[k], cudaEventDisableTiming));
      NX_CUDA(cudaEventRecord(used[k], stream()));
    }
    return NX_OK;
  }
};

// ---------------------------------------------------------------- run
struct RunCtx {
  nx_graph* g;
  nx_program prog;
  std::vector<const Dsss*> ds;
  uint32_t P, Q, Jc;
  uint64_t keep[2] = {0, 0};  // leading words of shard Jc (per DSSS) cached in device memory
  uint64_t stage_off[2] = {0, 0};  // word offset of each DSSS's segment in a staging buffer
  const uint32_t* act_host = nullptr;  // BFS / WCC: this iteration's interval flags (host)
  const float* tele;
  uint64_t h2d = 0, d2h = 0;
  uint32_t launches = 0;
};

// SPU iteration with columns [Jc, P) streamed from pinned host memory on a
// side stream (double-buffered), band by band; columns [0, Jc) are read in
// place. Words below each DSSS's device-resident prefix (the cached head of
// column Jc) are read from the device, the rest cross the host link.
nx_status spu_stream_iteration(RunCtx& c, SweepArgs& a, const std::vector<uint32_t>& off,
                               const std::vector<StreamBand>& bands, Streamer& sm) {
  nx_graph* g = c.g;
  set_iter_ptrs(g, c.prog, a);
  a.mode = 0;
  const Item* all = a.items;
  {  // resident columns
    SweepArgs r = a;
    r.items = all;
    NX_TRY(launch_sweep(kind_of(c.prog), r, off[0], stream()));
    ++c.launches;
  }
  uint32_t nstaged = 0;
  for (size_t q = 0; q < bands.size(); ++q) {
    const StreamBand& bd = bands[q];
    SweepArgs sa = a;
    sa.items = all + off[q];
    sa.src_lo = bd.i0;
    sa.src_hi = bd.i1;
    sa.acc_base = bd.j * g->geo.L;
    sa.accres = g->accres.p;
    sa.acc_in = bd.first ? nullptr : g->accres.p;
    sa.mode = bd.last ? 0 : 2;
    const int b = (int)(nstaged & 1);
    bool staged = false;
    for (size_t sx = 0; sx < c.ds.size(); ++sx) {
      const Dsss& d = *c.ds[sx];
      if (bd.e1[sx] <= d.dev_words) {  // the whole band is on the device
        sa.src[sx].ew = d.ew.as<uint32_t>();
        sa.ew_lo[sx] = 0;
        continue;
      }
      if (!staged) {
        NX_CUDA(cudaStreamWaitEvent(sm.side, sm.used[b], 0));  // the launch two bands back is done
        staged = true;
      }
      uint32_t* dst = g->stage[b].as<uint32_t>() + c.stage_off[sx];
      const uint64_t e0 = bd.e0[sx], e1 = bd.e1[sx];
      const uint64_t mid = std::max(e0, std::min(e1, d.dev_words));
      if (mid > e0)
        NX_CUDA(cudaMemcpyAsync(dst, d.ew.as<uint32_t>() + e0, (mid - e0) * 4,
                                cudaMemcpyDeviceToDevice, sm.side));
      NX_CUDA(cudaMemcpyAsync(dst + (mid - e0), d.h_ew.as<uint32_t>() + (mid - d.h_ew_first),
                              (e1 - mid) * 4, cudaMemcpyHostToDevice, sm.side));
      c.h2d += (e1 - mid) * 4;
      sa.src[sx].ew = dst;
      sa.ew_lo[sx] = e0;
    }
    if (staged) {
      NX_CUDA(cudaEventRecord(sm.copied[b], sm.side));
      NX_CUDA(cudaStreamWaitEvent(stream(), sm.copied[b], 0));
    }
    NX_TRY(launch_sweep(kind_of(c.prog), sa, off[q + 1] - off[q], stream()));
    ++c.launches;
    if (staged) {
      NX_CUDA(cudaEventRecord(sm.used[b], stream()));
      ++nstaged;
    }
  }
  g->cur ^= 1;
  return NX_OK;
}

// SPU iteration in bands of source intervals: band 0 stores the raw tile
// accumulators, the middle bands add to them, the last band adds and applies
// the epilogue. Every tile is owned by one block per band (split tiles merge
// their slots first), so no band needs atomics in device memory.
nx_status spu_band_iteration(RunCtx& c, SweepArgs& a, const std::vector<uint32_t>& off,
                             uint32_t band) {
  nx_graph* g = c.g;
  set_iter_ptrs(g, c.prog, a);
  const uint32_t nb = (uint32_t)off.size() - 1;
  for (uint32_t b = 0; b < nb; ++b) {
    SweepArgs ab = a;
    ab.items = a.items + off[b];
    ab.src_lo = b * band;
    ab.src_hi = std::min(c.P, (b + 1) * band);
    ab.acc_in = b == 0 ? nullptr : g->accres.p;
    ab.accres = g->accres.p;
    ab.mode = (b + 1 == nb) ? 0 : 2;
    NX_TRY(launch_sweep(kind_of(c.prog), ab, off[b + 1] - off[b], stream()));
    ++c.launches;
  }
  g->cur ^= 1;
  return NX_OK;
}

// MPU iteration (Algorithm 7) with intervals [Q, P) in pinned host memory.
// Their transfers run on a side stream, double-buffered against the sweeps:
// vstage[0..1] source rows (lines 7-16), vstage[2..3] / [4..5] new values /
// contributions of a staged column, vstage[6..7] its previous values (BFS,
// WCC; lines 17-26).
struct Staged {
  uint32_t n_res = 0, nh = 0;
  std::vector<uint32_t> off;  // launch boundaries in the item array
  cudaStream_t side = nullptr;
  // row_in/row_used: source row copied / its sweep done; col_in: previous
  // values copied; col_done: column swept; col_out: its results copied out
  cudaEvent_t row_in[2] = {}, row_used[2] = {}, col_in[2] = {}, col_done[2] = {}, col_out[2] = {};
  uint32_t nrow = 0, ncol = 0;  // buffers handed out so far (parity picks the buffer)
  ~Staged() {
    if (side) cudaStreamSynchronize(side);  // no copy outlives the run (early error returns)
    for (cudaEvent_t* e : {row_in, row_used, col_in, col_done, col_out})
      for (int k = 0; k < 2; ++k)
        if (e[k]) cudaEventDestroy(e[k]);
    if (side) cudaStreamDestroy(side);
  }
  nx_status init() {
    NX_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    for (cudaEvent_t* e : {row_in, row_used, col_in, col_done, col_out})
      for (int k = 0; k < 2; ++k) {
        NX_CUDA(cudaEventCreateWithFlags(&e[k], cudaEventDisableTiming));
        NX_CUDA(cudaEventRecord(e[k], stream()));
      }
    return NX_OK;
  }
  // the main stream waits for everything queued on the side stream
  nx_status join() {
    NX_CUDA(cudaEventRecord(col_out[0], side));
    NX_CUDA(cudaStreamWaitEvent(stream(), col_out[0], 0));
    return NX_OK;
  }
};

nx_status mpu_iteration(RunCtx& c, SweepArgs& a, Staged& S) {
  nx_graph* g = c.g;
  const uint32_t P = c.P, Q = c.Q, L = g->geo.L, n = g->geo.n;
  const bool pr = !is_min(c.prog);
  const bool has_c = (c.prog == NX_PR || c.prog == NX_PPR);
  const int cur = g->cur, nxt = 1 - g->cur;
  set_iter_ptrs(g, c.prog, a);
  const Item* all = a.items;
  const ProgKind K = kind_of(c.prog);
  uint32_t li = 0;  // launch index into S.off
  auto items_of = [&](uint32_t k) { return std::make_pair(all + S.off[k], S.off[k + 1] - S.off[k]); };
  // host arrays of this iteration
  float* hv_old = g->hval[cur].as<float>();
  float* hv_new = g->hval[nxt].as<float>();
  const uint32_t nh = S.nh;
  float* hc_old = has_c ? g->hval[cur].as<float>() + nh : nullptr;
  float* hc_new = has_c ? g->hval[nxt].as<float>() + nh : nullptr;
  // 1. resident block: sources [0, Q) into columns [0, Q), stored raw (lines 2-6)
  {
    auto [it, k] = items_of(li++);
    SweepArgs m2 = a;
    m2.mode = 2;
    m2.items = it;
    m2.src_lo = 0;
    m2.src_hi = Q;
    m2.accres = g->accres.p;
    NX_TRY(launch_sweep(K, m2, k, stream()));
    ++c.launches;
  }
  // 2. rows i >= Q: load I_i, update resident columns in place, ToHub the rest (lines 7-16).
  // BFS / WCC skip inactive rows (the run's host copy of this iteration's flags).
  for (uint32_t i = Q; i < P; ++i) {
    auto [it, k] = items_of(li++);
    if ((!pr && !c.act_host[i]) || k == 0) continue;
    const uint32_t v0 = i * L, v1 = std::min<uint32_t>(n, v0 + L);
    if (v1 <= v0) continue;
    const float* src_host = (has_c ? hc_old : hv_old) + (v0 - S.n_res);
    const int b = (int)(S.nrow++ & 1);
    NX_CUDA(cudaStreamWaitEvent(S.side, S.row_used[b], 0));  // the sweep two rows back is done
    NX_CUDA(cudaMemcpyAsync(g->vstage[b].p, src_host, (size_t)(v1 - v0) * 4,
                            cudaMemcpyHostToDevice, S.side));
    NX_CUDA(cudaEventRecord(S.row_in[b], S.side));
    c.h2d += (uint64_t)(v1 - v0) * 4;
    SweepArgs m1 = a;
    m1.mode = 1;
    m1.items = it;
    m1.q_res = Q;
    m1.accres = g->accres.p;
    m1.gstage = g->vstage[b].p;
    m1.stage_i = i;
    NX_CUDA(cudaStreamWaitEvent(stream(), S.row_in[b], 0));
    NX_TRY(launch_sweep(K, m1, k, stream()));
    NX_CUDA(cudaEventRecord(S.row_used[b], stream()));
    ++c.launches;
  }
  // 3. epilogue of the resident columns from their accumulators
  {
    auto [it, k] = items_of(li++);
    SweepArgs m3 = a;
    m3.mode = 3;
    m3.items = it;
    m3.accres = g->accres.p;
    NX_TRY(launch_sweep(K, m3, k, stream()));
    ++c.launches;
  }
  // 4. columns j >= Q: SPU from resident rows + FromHub, save to the host (lines 17-26)
  for (uint32_t j = Q; j < P; ++j) {
    auto [it, k] = items_of(li++);
    const uint32_t v0 = j * L, v1 = std::min<uint32_t>(n, v0 + L);
    if (v1 <= v0) continue;
    const size_t bytes = (size_t)(v1 - v0) * 4;
    const int b = (int)(S.ncol++ & 1);
    SweepArgs m0 = a;
    m0.mode = 0;
    m0.items = it;
    m0.src_lo = 0;
    m0.src_hi = Q;
    m0.hub_lo = Q;
    m0.hub_hi = P;
    m0.out_base = v0;
    m0.vnew = g->vstage[2 + b].p;
    m0.cnew = has_c ? g->vstage[4 + b].as<float>() : nullptr;
    if (!pr) {  // previous values: the sweep two columns back is done with the buffer
      NX_CUDA(cudaStreamWaitEvent(S.side, S.col_done[b], 0));
      NX_CUDA(cudaMemcpyAsync(g->vstage[6 + b].p, hv_old + (v0 - S.n_res), bytes,
                              cudaMemcpyHostToDevice, S.side));
      NX_CUDA(cudaEventRecord(S.col_in[b], S.side));
      NX_CUDA(cudaStreamWaitEvent(stream(), S.col_in[b], 0));
      c.h2d += bytes;
      m0.vold = g->vstage[6 + b].p;
    }
    NX_CUDA(cudaStreamWaitEvent(stream(), S.col_out[b], 0));  // outputs two columns back copied out
    NX_TRY(launch_sweep(K, m0, k, stream()));
    NX_CUDA(cudaEventRecord(S.col_done[b], stream()));
    ++c.launches;
    NX_CUDA(cudaStreamWaitEvent(S.side, S.col_done[b], 0));
    NX_CUDA(cudaMemcpyAsync(hv_new + (v0 - S.n_res), g->vstage[2 + b].p, bytes,
                            cudaMemcpyDeviceToHost, S.side));
    c.d2h += bytes;
    if (has_c) {
      NX_CUDA(cudaMemcpyAsync(hc_new + (v0 - S.n_res), g->vstage[4 + b].p, bytes,
                              cudaMemcpyDeviceToHost, S.side));
      c.d2h += bytes;
    }
    NX_CUDA(cudaEventRecord(S.col_out[b], S.side));
  }
  g->cur ^= 1;
  return NX_OK;
}

nx_status run_impl(nx_graph* g, nx_program prog, const nx_params& p, uint32_t iters,
                   nx_strategy strategy, uint64_t budget, nx_run_stats* st) {
  const uint32_t n = g->geo.n, P = g->geo.P, L = g->geo.L;
  if (prog == NX_WCC && !g->has_tr)
    return invalid("nx_run: WCC needs the transpose DSSS (build with NX_WITH_TRANSPOSE)");
  if (prog == NX_WPR && !g->has_w) return invalid("nx_run: WPR needs NX_WITH_WEIGHTS");
  if (prog == NX_BFS && p.root >= n) return invalid("nx_run: BFS root >= n");
  const bool push = (strategy == NX_SRC_COARSE || strategy == NX_SRC_FINE);
  if (push && prog != NX_PR && prog != NX_PPR)
    return invalid("nx_run: the source-sorted ablation runs PR and PPR only");
  if (push && !g->has_tr)
    return invalid("nx_run: the source-sorted ablation reads the transpose DSSS (NX_WITH_TRANSPOSE)");
  if (push && budget) return invalid("nx_run: the source-sorted ablation takes no budget");
  // NX_AUTO picks the fastest strategy the graph and the budget allow (the
  // paper's adaptive choice, Section III-B3): for PageRank on a graph built
  // with NX_ONCHIP_HUBS and no budget, the on-chip double-phase update (1.4x
  // the SPU sweep at R-MAT scale 26); otherwise SPU when the budget holds
  // every interval, else MPU (below).
  const bool onchip = (strategy == NX_DPU_ONCHIP) ||
                      (strategy == NX_AUTO && !budget && g->oc.built && (prog == NX_PR || prog == NX_PPR));
  if (onchip && prog != NX_PR && prog != NX_PPR)
    return invalid("nx_run: NX_DPU_ONCHIP runs PR and PPR only");
  if (onchip && !g->oc.built)
    return invalid("nx_run: NX_DPU_ONCHIP needs a graph built with NX_ONCHIP_HUBS");
  if (onchip && budget) return invalid("nx_run: NX_DPU_ONCHIP takes no budget");
  // strategy from the budget (Section III-B3: Q <= B_M P / (2 n B_a))
  const double Ba = 4.0;
  uint32_t Qb = P;
  if (budget) Qb = (uint32_t)std::min<double>(P, std::floor((double)budget * P / (2.0 * n * Ba)));
  nx_strategy strat = strategy;
  if (strat == NX_AUTO) strat = (Qb >= P) ? NX_SPU : NX_MPU;
  if (strat == NX_SPU && Qb < P) {
    set_error("nx_run: SPU needs 2 n B_a bytes of budget for the ping-pong intervals");
    return NX_ERR_BUDGET_TOO_SMALL;
  }
  if (strat == NX_MPU && Qb >= P) strat = NX_SPU;  // Q = P: MPU is SPU (Section III-B3)
  const bool staged = (strat == NX_MPU) || (strat == NX_DPU && Qb < P);
  const uint32_t Q = strat == NX_MPU ? Qb : (strat == NX_DPU ? 0 : P);
  if (budget && (strat == NX_DPU || strat == NX_MPU) && budget < 2ull * L * 4) {
    set_error("nx_run: the budget is below one interval pair (2 L B_a)");
    return NX_ERR_BUDGET_TOO_SMALL;
  }

  NX_TRY(prepare(g));
  // teleport
  const float* tele = nullptr;
  if ((prog == NX_PPR || prog == NX_WPR) && p.teleport) {
    if (p.teleport_is_device && !g->relabeled) {
      tele = p.teleport;
    } else {
      NX_TRY(ensure(g->tele, (size_t)n * 4));
      if (g->relabeled) {  // caller order -> internal order
        DevBuf tmp;
        const void* in = p.teleport;
        if (!p.teleport_is_device) {
          NX_TRY(tmp.alloc((size_t)n * 4));
          NX_CUDA(cudaMemcpyAsync(tmp.p, p.teleport, (size_t)n * 4, cudaMemcpyHostToDevice,
                                  stream()));
          in = tmp.p;
        }
        NX_TRY(vertex_to_internal(g, in, g->tele.p));
        NX_CUDA(cudaStreamSynchronize(stream()));  // tmp is freed on leaving
      } else {
        NX_CUDA(cudaMemcpyAsync(g->tele.p, p.teleport, (size_t)n * 4, cudaMemcpyHostToDevice,
                                stream()));
      }
      tele = g->tele.as<float>();
    }
  }
  if (prog == NX_PPR && !tele) {  // uniform teleport: PPR equals PageRank
    NX_TRY(ensure(g->tele, (size_t)n * 4));
    std::vector<float> u(n, 1.0f / (float)n);
    NX_CUDA(cudaMemcpyAsync(g->tele.p, u.data(), (size_t)n * 4, cudaMemcpyHostToDevice, stream()));
    NX_CUDA(cudaStreamSynchronize(stream()));
    tele = g->tele.as<float>();
  }
  // initialize or resume
  const bool resume = (g->values_set_for == (int)prog);
  if (resume) {
    DevBuf tmp;
    NX_TRY(tmp.alloc((size_t)n * 4));
    NX_CUDA(cudaMemcpyAsync(tmp.p, g->val[g->cur].p, (size_t)n * 4, cudaMemcpyDeviceToDevice,
                            stream()));
    NX_TRY(initialize(g, prog, p, tele, tmp.p));
  } else {
    NX_TRY(initialize(g, prog, p, tele, nullptr));
  }
  g->values_set_for = -1;
  g->last_prog = (int)prog;
  if (prog == NX_WPR) g->wpr_alpha = p.alpha;
  if (onchip) {
    NX_TRY(ensure_resident(g));
    Scal sc = scal_of(g);
    EventPair ev;
    NX_TRY(ev.create());
    NX_CUDA(cudaEventRecord(ev.e0, stream()));
    for (uint32_t it = 0; it < iters; ++it) {
      const int c = g->cur, nn = 1 - g->cur;
      OcRun r;
      r.c_in = g->aux[c].as<float>();
      r.r_out = g->val[nn].as<float>();
      r.c_out = g->aux[nn].as<float>();
      r.tele = (prog == NX_PPR) ? tele : nullptr;
      r.dang_by_tele = (prog == NX_PPR) ? 1 : 0;
      r.alpha = p.alpha;
      r.dm_in = sc.dm + c;
      r.dm_out = sc.dm + nn;
      NX_TRY(onchip_iteration(g, r, stream()));
      g->cur ^= 1;
    }
    NX_CUDA(cudaEventRecord(ev.e1, stream()));
    float ms = 0.f;
    NX_TRY(ev.elapsed(&ms));
    if (st) {
      const uint64_t n64 = g->geo.n;
      memset(st, 0, sizeof *st);
      st->iters_done = iters;
      st->Q = P;
      st->strategy = (uint32_t)NX_DPU_ONCHIP;
      st->ms = ms;
      st->edges_swept = g->m * iters;
      // 16-bit edge entries, hub values written and read, hub offsets, staged c, outdeg, r, c
      st->bytes_model = (uint64_t)iters * (2 * g->m + 10 * g->oc.H + 16 * n64);
      st->launches = (g->oc.na ? 2 : 1) * iters;
    }
    return NX_OK;
  }
  if (push) {
    NX_TRY(ensure_resident(g));
    PushRun r;
    r.coarse = (strategy == NX_SRC_COARSE);
    r.iters = iters;
    r.alpha = p.alpha;
    r.tele = tele;
    r.dang_by_tele = (prog == NX_PPR) ? 1 : 0;
    r.dm = scal_of(g).dm;
    uint32_t launches = 0;
    float ms = 0.f;
    NX_TRY(push_run(g, r, &launches, &ms));
    if (st) {
      memset(st, 0, sizeof *st);
      st->iters_done = iters;
      st->Q = P;
      st->strategy = (uint32_t)strategy;
      st->ms = ms;
      st->edges_swept = g->m * iters;
      st->bytes_model = bytes_per_sweep(g, prog, g->m) * iters;
      st->launches = launches;
    }
    return NX_OK;
  }

  RunCtx c;
  c.g = g;
  c.prog = prog;
  c.ds = {&g->fwd};
  if (prog == NX_WCC) c.ds.push_back(&g->tr);
  c.P = P;
  c.Q = Q;
  c.tele = tele;
  const auto& tb = g->geo.h_col_tb;
  // SPU: shards that do not fit next to the intervals stream from pinned host memory
  c.Jc = P;
  if (strat == NX_SPU && budget) {
    const uint64_t vert = (uint64_t)2 * n * 4;
    uint64_t left = budget > vert ? budget - vert : 0;
    uint32_t j = 0;
    for (; j < P; ++j) {
      uint64_t bytes = 0;
      for (const Dsss* d : c.ds)
        bytes += 4 * (d->h_piece_off[(uint64_t)P * tb[j + 1]] - d->h_piece_off[(uint64_t)P * tb[j]]);
      if (prog == NX_WPR) bytes *= 2;
      if (bytes > left) break;
      left -= bytes;
    }
    c.Jc = j;
    if (c.Jc < P) {  // the rest of the budget caches the head of shard Jc
      for (size_t s = 0; s < c.ds.size(); ++s) {
        const Dsss* d = c.ds[s];
        const uint64_t w = d->h_piece_off[(uint64_t)P * tb[j + 1]] - d->h_piece_off[(uint64_t)P * tb[j]];
        const uint64_t kw = std::min<uint64_t>(w, left / 4) & ~(kEdgeAlign - 1);
        c.keep[s] = kw;
        left -= kw * 4;
      }
    }
    if (c.Jc < P && prog == NX_WPR) {
      set_error("nx_run: weighted PageRank needs its edges on the device (budget too small)");
      return NX_ERR_BUDGET_TOO_SMALL;
    }
  }
  const bool streaming = (strat == NX_SPU && c.Jc < P);
  // Residency: under an SPU budget the device keeps only the words the
  // schedule reads in place (shards [0, Jc) and the cached head of shard Jc);
  // the streamed rest, every DSSS the program does not read, the hub index and
  // (unless weighted PageRank reads them) the weights live in pinned host
  // memory only. Other runs need their DSSS (and hubs) on the device.
  const bool budgeted_spu = (strat == NX_SPU && budget != 0);
  std::vector<StreamBand> bands;
  if (streaming) bands = stream_bands(g, c.ds, c.Jc);
  {
    Dsss* all_ds[2] = {&g->fwd, g->has_tr ? &g->tr : nullptr};
    for (Dsss* d : all_ds) {
      if (!d) continue;
      const auto it = std::find(c.ds.begin(), c.ds.end(), d);
      const bool used = it != c.ds.end();
      if (!budgeted_spu) {
        if (used) {
          NX_TRY(set_edge_residency(*d, d->words, 0));
          if (strat == NX_DPU || staged) NX_TRY(move_to_device(d->h_hub_dst, d->hub_dst));
        }
        continue;
      }
      NX_TRY(move_to_host(d->hub_dst, d->h_hub_dst));
      if (prog != NX_WPR) NX_TRY(move_to_host(d->wt, d->h_wt));
      else if (used) NX_TRY(move_to_device(d->h_wt, d->wt));
      if (!used) {  // nothing of it stays on the device
        NX_TRY(set_edge_residency(*d, 0, 0));
        NX_TRY(move_to_host(d->piece_off, d->h_piece_pin));
        NX_TRY(move_to_host(d->hub_off, d->h_hub_off));
      } else if (c.Jc >= P) {
        NX_TRY(set_edge_residency(*d, d->words, 0));
      } else {
        const size_t sx = (size_t)(it - c.ds.begin());
        const uint64_t ej = d->h_piece_off[(uint64_t)P * tb[c.Jc]];
        const uint64_t head = (ej & ~(kEdgeAlign - 1)) + c.keep[sx];
        NX_TRY(set_edge_residency(*d, std::max(round_up(ej, kEdgeAlign), head), ej & ~(kEdgeAlign - 1)));
      }
    }
    if (budgeted_spu) {
      NX_TRY(move_to_host(g->orig_src, g->h_orig_src));
      NX_TRY(move_to_host(g->orig_dst, g->h_orig_dst));
      // scratch of other programs and schedules (reallocated when they run)
      DevBuf* scratch[] = {&g->hubs, &g->hubs_t, &g->lam[0], &g->lam[1], &g->ybuf, &g->accres,
                           &g->split_buf, &g->stage[0], &g->stage[1], &g->vstage[0],
                           &g->vstage[1], &g->vstage[2], &g->vstage[3], &g->vstage[4],
                           &g->vstage[5], &g->vstage[6], &g->vstage[7]};
      for (DevBuf* b : scratch) b->release();
      if (prog != NX_PPR && prog != NX_WPR) g->tele.release();
      if (g->oc.built) {  // the on-chip double-phase structure
        NX_TRY(move_to_host(g->oc.ew, g->oc.h_ew));
        NX_TRY(move_to_host(g->oc.hub_dst, g->oc.h_hub_dst));
        g->oc.hub_val.release();
      }
    }
  }
  for (const Dsss* d : c.ds) {  // the piece and hub offsets of every DSSS the run reads
    NX_TRY(move_to_device(const_cast<Dsss*>(d)->h_piece_pin, const_cast<Dsss*>(d)->piece_off));
    NX_TRY(move_to_device(const_cast<Dsss*>(d)->h_hub_off, const_cast<Dsss*>(d)->hub_off));
  }
  // SPU bands (on request): launches over groups of source intervals, the
  // tile accumulators carried between them. One launch over all sources is
  // the default: at R-MAT scale 26 (268 MB of values, beyond L2) it beat two
  // 128 MB bands by 7.4% with degree-ordered ids (5.82 vs 6.28 ms per sweep at
  // P = 64, 5.70 vs 6.15 at P = 32) and by 2.4% with the generator's ids: the
  // most-read values stay in L2 either way, and a band pays for the carried
  // accumulators and a second pass over every tile.
  uint32_t band = P;
  if (strat == NX_SPU && !streaming && p.band_intervals) band = std::min<uint32_t>(p.band_intervals, P);
  const uint32_t nbands = (uint32_t)ceil_div(P, band);

  // plan (cached: the graph never changes)
  const int key = (((int)strat * 16 + (int)c.ds.size()) * 4096 + (int)(staged ? Q + 1 : 0) +
                   (streaming ? (int)(c.Jc + 2048) : 0)) * 2048 + (int)(nbands > 1 ? band : 0);
  auto& slot_plan = g->plans[key];
  if (!slot_plan) {  // built aside and cached only once complete (a failed call caches nothing)
    TraceRange trace_plan("plan");
    std::unique_ptr<nx_graph::Plan> fresh(new nx_graph::Plan());
    nx_graph::Plan& pl = *fresh;
    const uint64_t total = g->m * c.ds.size();
    const uint64_t blk = target_block_edges(total);
    PlanOut plan;
    std::vector<uint32_t> launch_off;
    uint32_t n_a = 0, n_b = 0;
    if (strat == NX_SPU && !streaming && nbands == 1) {
      plan_tiles(g, c.ds, 0, P, 0, P, true, blk, plan);
      n_a = (uint32_t)plan.items.size();
    } else if (strat == NX_SPU && !streaming) {  // one launch per band of source intervals
      for (uint32_t i0 = 0; i0 < P; i0 += band) {
        launch_off.push_back((uint32_t)plan.items.size());
        plan_tiles(g, c.ds, i0, std::min(P, i0 + band), 0, P, true,
                   std::max<uint64_t>(blk / nbands, 4096), plan);
      }
      launch_off.push_back((uint32_t)plan.items.size());
    } else if (strat == NX_SPU) {  // columns [0, Jc) in place, then one launch per streamed band
      plan_tiles(g, c.ds, 0, P, 0, c.Jc, true, blk, plan);
      for (const StreamBand& bd : bands) {
        launch_off.push_back((uint32_t)plan.items.size());
        plan_tiles(g, c.ds, bd.i0, bd.i1, bd.j, bd.j + 1, true, blk, plan, bd.t0, bd.t1);
      }
      launch_off.push_back((uint32_t)plan.items.size());  // launch_off[0]: resident item count
    } else if (!staged) {  // DPU, intervals resident: ToHub items (all rows), then FromHub tiles
      for (size_t sx = 0; sx < c.ds.size(); ++sx)
        for (uint32_t i = 0; i < P; ++i) plan_row(g, *c.ds[sx], (uint32_t)sx, i, 0, P, blk, plan);
      n_a = (uint32_t)plan.items.size();
      plan_tiles(g, c.ds, 0, 0, 0, P, false, blk, plan);
      n_b = (uint32_t)plan.items.size() - n_a;
    } else {  // MPU / staged DPU: launches of Algorithm 7
      launch_off.push_back(0);
      plan_tiles(g, c.ds, 0, Q, 0, Q, true, blk, plan);  // resident block (mode 2)
      launch_off.push_back((uint32_t)plan.items.size());
      for (uint32_t i = Q; i < P; ++i) {  // rows (mode 1), every DSSS of the program
        for (size_t sx = 0; sx < c.ds.size(); ++sx)
          plan_row(g, *c.ds[sx], (uint32_t)sx, i, 0, P, blk, plan);
        launch_off.push_back((uint32_t)plan.items.size());
      }
      plan_tiles(g, c.ds, 0, 0, 0, Q, false, blk, plan);  // resident epilogue (mode 3)
      launch_off.push_back((uint32_t)plan.items.size());
      for (uint32_t j = Q; j < P; ++j) {  // staged columns (mode 0)
        plan_tiles(g, c.ds, 0, Q, j, j + 1, true, blk, plan);
        launch_off.push_back((uint32_t)plan.items.size());
      }
    }
    NX_TRY(upload_items(g, plan, pl));
    pl.na = n_a;
    pl.nb = n_b;
    pl.off = launch_off;
    slot_plan = std::move(fresh);
  }
  nx_graph::Plan& pl = *slot_plan;
  NX_TRY(ensure_split(g, pl.slots));
  const uint32_t n_a = pl.na, n_b = pl.nb;
  if (strat == NX_DPU || staged) {
    NX_TRY(ensure(g->hubs, std::max<uint64_t>(g->fwd.D, 1) * 4));
    if (prog == NX_WCC) NX_TRY(ensure(g->hubs_t, std::max<uint64_t>(g->tr.D, 1) * 4));
  }

  if (nbands > 1) NX_TRY(ensure(g->accres, (size_t)n * 4));
  SweepArgs a = base_args(g, prog, p, tele);
  a.items = pl.items.as<Item>();

  a.split = g->split_buf.p;

  // streaming buffers: two staging buffers, each with one segment per DSSS
  // sized for that DSSS's largest band, and a column of tile accumulators
  Streamer sm;
  if (streaming) {
    uint64_t seg[2] = {0, 0};
    for (const StreamBand& bd : bands)
      for (size_t sx = 0; sx < c.ds.size(); ++sx)
        if (bd.e1[sx] > c.ds[sx]->dev_words) seg[sx] = std::max(seg[sx], bd.e1[sx] - bd.e0[sx]);
    c.stage_off[0] = 0;
    c.stage_off[1] = seg[0];
    for (int b = 0; b < 2; ++b) NX_TRY(ensure(g->stage[b], std::max<uint64_t>(seg[0] + seg[1], 1) * 4));
    NX_TRY(ensure(g->accres, (size_t)L * 4));
    NX_TRY(sm.init());
  }
  // staged intervals (MPU): device accumulators for resident columns, pinned
  // host arrays for the rest, per-interval staging buffers
  Staged S;
  if (staged) {
    S.n_res = std::min<uint64_t>((uint64_t)Q * L, n);
    S.nh = n - S.n_res;
    S.off = pl.off;
    NX_TRY(ensure(g->accres, std::max<size_t>(S.n_res, 1) * 4));
    for (int b = 0; b < 8; ++b) NX_TRY(ensure(g->vstage[b], (size_t)L * 4));
    const bool has_c = (prog == NX_PR || prog == NX_PPR);
    const size_t hbytes = (size_t)S.nh * 4 * (has_c ? 2 : 1);
    for (int b = 0; b < 2; ++b)
      if (g->hval[b].bytes < std::max<size_t>(hbytes, 4)) NX_TRY(g->hval[b].alloc(std::max<size_t>(hbytes, 4)));
    // move the initial values of intervals [Q, P) to the host
    const int cc = g->cur;
    if (S.nh) {
      NX_CUDA(cudaMemcpyAsync(g->hval[cc].p, g->val[cc].as<uint32_t>() + S.n_res, (size_t)S.nh * 4,
                              cudaMemcpyDeviceToHost, stream()));
      if (has_c)
        NX_CUDA(cudaMemcpyAsync(g->hval[cc].as<uint32_t>() + S.nh, g->aux[cc].as<uint32_t>() + S.n_res,
                                (size_t)S.nh * 4, cudaMemcpyDeviceToHost, stream()));
    }
    NX_CUDA(cudaStreamSynchronize(stream()));
    NX_TRY(S.init());
  }

  // per-interval edge counts (edges streamed by a sweep of active sources)
  std::vector<uint64_t> row_edges(P, 0);
  for (uint32_t j = 0; j < P; ++j) {
    const uint32_t nt = tb[j + 1] - tb[j];
    if (nt == 0) continue;  // empty trailing interval
    for (uint32_t i = 0; i < P; ++i)
      for (const Dsss* d : c.ds) {
        uint64_t p0 = d->h_piece_off[piece_index(P, tb[j], nt, i, tb[j])];
        uint64_t p1 = d->h_piece_off[piece_index(P, tb[j], nt, i, tb[j + 1] - 1) + 1];
        row_edges[i] += p1 - p0;
      }
  }

  EventPair ev;
  NX_TRY(ev.create());
  Scal sc = scal_of(g);
  TraceRange trace_loop("iterations");
  uint64_t swept = 0;
  uint32_t done = 0, skipped = 0;
  // activity: [0] = active-interval count, [1 + i] = flag of interval i (pinned)
  if (g->hact.bytes < ((size_t)P + 1) * 4) NX_TRY(g->hact.alloc(((size_t)P + 1) * 4));
  uint32_t* hact = g->hact.as<uint32_t>();
  const uint32_t* act_h = hact + 1;
  c.act_host = act_h;
  std::fill(hact, hact + P + 1, 1u);
  if (is_min(prog)) {  // the flags Initialize left (later ones arrive with each count)
    NX_CUDA(cudaMemcpyAsync(hact + 1, g->act[g->cur].p, (size_t)P * 4, cudaMemcpyDeviceToHost,
                            stream()));
    NX_CUDA(cudaStreamSynchronize(stream()));
    c.d2h += (uint64_t)P * 4;
  }
  NX_CUDA(cudaEventRecord(ev.e0, stream()));
  for (uint32_t it = 0; it < iters; ++it) {
    for (uint32_t i = 0; i < P; ++i) {
      if (act_h[i]) swept += row_edges[i];
      else ++skipped;
    }
    if (strat == NX_SPU && !streaming && nbands == 1) {
      NX_TRY(spu_iteration(g, prog, a, n_a));
      ++c.launches;
    } else if (strat == NX_SPU && !streaming) {
      NX_TRY(spu_band_iteration(c, a, pl.off, band));
    } else if (streaming) {
      NX_TRY(spu_stream_iteration(c, a, pl.off, bands, sm));
    } else if (!staged) {
      NX_TRY(dpu_iteration(g, prog, a, n_a, n_b));
      c.launches += 2;
    } else {
      NX_TRY(mpu_iteration(c, a, S));
    }
    ++done;
    if (is_min(prog)) {  // Algorithm 1: stop when no interval is active; one round trip
      NX_CUDA(cudaMemcpyAsync(hact, sc.act_count, 4, cudaMemcpyDeviceToHost, stream()));
      NX_CUDA(cudaMemcpyAsync(hact + 1, g->act[g->cur].p, (size_t)P * 4, cudaMemcpyDeviceToHost,
                              stream()));
      NX_CUDA(cudaStreamSynchronize(stream()));
      c.d2h += 4 + (uint64_t)P * 4;
      if (hact[0] == 0) break;
    }
  }
  if (staged) NX_TRY(S.join());  // the last results reach the host inside the timed region
  NX_CUDA(cudaEventRecord(ev.e1, stream()));
  float ms = 0.f;
  NX_TRY(ev.elapsed(&ms));
  if (staged && S.nh) {  // results of the host-side intervals back into the value arrays
    const int cc = g->cur;
    const bool has_c = (prog == NX_PR || prog == NX_PPR);
    NX_CUDA(cudaMemcpyAsync(g->val[cc].as<uint32_t>() + S.n_res, g->hval[cc].p, (size_t)S.nh * 4,
                            cudaMemcpyHostToDevice, stream()));
    if (has_c)
      NX_CUDA(cudaMemcpyAsync(g->aux[cc].as<uint32_t>() + S.n_res, g->hval[cc].as<uint32_t>() + S.nh,
                              (size_t)S.nh * 4, cudaMemcpyHostToDevice, stream()));
    NX_CUDA(cudaStreamSynchronize(stream()));
  }
  if (st) {
    memset(st, 0, sizeof *st);
    st->iters_done = done;
    st->Q = (strat == NX_SPU) ? P : Q;
    st->strategy = (uint32_t)strat;
    st->streamed_cols = streaming ? P - c.Jc : 0;
    st->ms = ms;
    st->edges_swept = swept;
    st->intervals_skipped = skipped;
    st->bytes_model = bytes_per_sweep(g, prog, 0) * done + 4 * swept + (prog == NX_WPR ? 4 * swept : 0);
    if (strat == NX_DPU && !staged) st->bytes_model += (uint64_t)done * 3 * 4 * g->fwd.D;
    st->h2d_bytes = c.h2d;
    st->d2h_bytes = c.d2h;
    st->launches = c.launches;
  }
  return NX_OK;
}

// ---------------------------------------------------------------- gather probe
// Times the PageRank sweep's loads and gathers alone (PK_PROBE) with the
// launches an SPU PageRank run would make: the same plan (bands included).
nx_status probe_impl(nx_graph* g, uint32_t sweeps, float* ms_per_sweep) {
  const uint32_t n = g->geo.n, P = g->geo.P;
  NX_TRY(ensure_resident(g));
  NX_TRY(prepare(g));
  NX_TRY(ensure(g->aux[0], (size_t)n * 4));
  NX_TRY(ensure(g->aux[1], (size_t)n * 4));
  // one launch over all sources, as the SPU run's default
  const int key = (((int)NX_SPU * 16 + 1) * 4096) * 2048;
  auto& slot = g->plans[key];
  if (!slot) {  // cached only once complete
    std::unique_ptr<nx_graph::Plan> fresh(new nx_graph::Plan());
    PlanOut plan;
    std::vector<const Dsss*> ds{&g->fwd};
    plan_tiles(g, ds, 0, P, 0, P, true, target_block_edges(g->m), plan);
    NX_TRY(upload_items(g, plan, *fresh));
    fresh->na = (uint32_t)fresh->h_items.size();
    slot = std::move(fresh);
  }
  NX_TRY(ensure_split(g, slot->slots));
  nx_params p{};
  p.alpha = 0.85f;
  SweepArgs a = base_args(g, NX_PR, p, nullptr);
  a.items = slot->items.as<Item>();
  a.split = g->split_buf.p;
  a.gsrc = g->aux[0].p;
  a.vnew = g->aux[1].p;  // the probe's sink (never written in practice)
  EventPair ev;
  NX_TRY(ev.create());
  NX_CUDA(cudaEventRecord(ev.e0, stream()));
  for (uint32_t q = 0; q < sweeps; ++q) NX_TRY(launch_sweep(PK_PROBE, a, slot->na, stream()));
  NX_CUDA(cudaEventRecord(ev.e1, stream()));
  float ms = 0.f;
  NX_TRY(ev.elapsed(&ms));
  *ms_per_sweep = sweeps ? ms / (float)sweeps : 0.f;
  return NX_OK;
}

// ---------------------------------------------------------------- SCC
// Strongly connected components (Section IV-D names SCC; the paper gives no
// algorithm) by coloring over the DSSS and its transpose. Each round:
//  1. every unassigned vertex v takes color(v) = its own label (caller id);
//     forward min-propagation along edges between unassigned vertices makes
//     color(v) the smallest label of a vertex that reaches v;
//  2. a vertex whose color is its own label is a root; the vertices of its
//     color that reach it form its component (a vertex u of that color
//     reaches the root, and the root reaches u because it has the smallest
//     label among u's reachers), found by backward reach over the transpose
//     DSSS; each is assigned the root's label, the smallest in the component;
//  3. repeat over the vertices left unassigned.
// Colors never increase along an edge between unassigned vertices, so a
// vertex's out-neighbours of its own color are exactly those whose reach
// value (color + 1) equals its color + 1: the backward sweep is a max
// reduction compared against the vertex's own color.
__global__ void k_scc_fwd_init(uint32_t n, const uint32_t* __restrict__ lab,
                               const uint32_t* __restrict__ ids, uint32_t* __restrict__ col) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    col[v] = lab[v] == kInf ? (ids ? ids[v] : (uint32_t)v) : kInf;
}

// Roots (color == own label) start reached; their intervals start active.
__global__ void k_scc_bwd_init(uint32_t n, uint32_t L, const uint32_t* __restrict__ col,
                               const uint32_t* __restrict__ ids, uint32_t* __restrict__ bw,
                               uint32_t* __restrict__ act) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const uint32_t c = col[v];
    const bool root = c != kInf && c == (ids ? ids[v] : (uint32_t)v);
    bw[v] = root ? c + 1u : 0u;
    if (root) act[v / L] = 1u;
  }
}

// Reached vertices take their color as label; counts the vertices left.
__global__ void k_scc_assign(uint32_t n, const uint32_t* __restrict__ col,
                             const uint32_t* __restrict__ bw, uint32_t* __restrict__ lab,
                             uint32_t* __restrict__ left) {
  uint32_t c = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    uint32_t l = lab[v];
    if (l == kInf && bw[v] != 0u) lab[v] = l = col[v];
    c += l == kInf ? 1u : 0u;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(left, c);
}

constexpr int kTrPlanKey = -7;  // plan over the transpose DSSS (adjoint, SCC)

nx_status tr_plan(nx_graph* g, nx_graph::Plan** out) {
  auto& slot = g->plans[kTrPlanKey];
  if (!slot) {  // cached only once complete
    std::unique_ptr<nx_graph::Plan> fresh(new nx_graph::Plan());
    PlanOut plan;
    std::vector<const Dsss*> ds{&g->tr};
    plan_tiles(g, ds, 0, g->geo.P, 0, g->geo.P, true, target_block_edges(g->m), plan);
    NX_TRY(upload_items(g, plan, *fresh));
    fresh->na = (uint32_t)fresh->h_items.size();
    slot = std::move(fresh);
  }
  NX_TRY(ensure_split(g, slot->slots));
  *out = slot.get();
  return NX_OK;
}

nx_status scc_impl(nx_graph* g, uint32_t max_sweeps, nx_run_stats* st) {
  const uint32_t n = g->geo.n, P = g->geo.P;
  cudaStream_t s = stream();
  NX_TRY(ensure_resident(g));
  NX_TRY(prepare(g));
  for (int k = 0; k < 2; ++k) NX_TRY(ensure(g->aux[k], (size_t)n * 4));
  NX_TRY(ensure(g->ybuf, (size_t)n * 4));  // labels while the rounds run
  // plans: tiles over the forward DSSS and over the transpose
  const int fkey = ((int)NX_SPU * 16 + 1) * 4096 * 2048;
  auto& fslot = g->plans[fkey];
  if (!fslot) {  // cached only once complete
    std::unique_ptr<nx_graph::Plan> fresh(new nx_graph::Plan());
    PlanOut plan;
    std::vector<const Dsss*> ds{&g->fwd};
    plan_tiles(g, ds, 0, P, 0, P, true, target_block_edges(g->m), plan);
    NX_TRY(upload_items(g, plan, *fresh));
    fresh->na = (uint32_t)fresh->h_items.size();
    fslot = std::move(fresh);
  }
  NX_TRY(ensure_split(g, fslot->slots));
  nx_graph::Plan* tpl = nullptr;
  NX_TRY(tr_plan(g, &tpl));
  nx_params p{};
  p.alpha = 0.85f;
  SweepArgs fa = base_args(g, NX_BFS, p, nullptr);
  fa.items = fslot->items.as<Item>();
  fa.split = g->split_buf.p;
  SweepArgs ba = fa;
  ba.src[0].ew = g->tr.ew.as<uint32_t>();
  ba.src[0].wt = nullptr;
  ba.src[0].piece_off = g->tr.piece_off.as<uint64_t>();
  ba.items = tpl->items.as<Item>();
  const uint32_t* ids = g->relabeled ? g->old_of_new.as<uint32_t>() : nullptr;
  uint32_t* lab = g->ybuf.as<uint32_t>();
  uint32_t* col[2] = {g->val[0].as<uint32_t>(), g->val[1].as<uint32_t>()};
  uint32_t* bw[2] = {g->aux[0].as<uint32_t>(), g->aux[1].as<uint32_t>()};
  uint32_t* act[2] = {g->act[0].as<uint32_t>(), g->act[1].as<uint32_t>()};
  Scal sc = scal_of(g);
  uint32_t* left = reinterpret_cast<uint32_t*>(g->scal.as<unsigned char>() + 36);
  if (g->hact.bytes < ((size_t)P + 1) * 4) NX_TRY(g->hact.alloc(((size_t)P + 1) * 4));
  uint32_t* hact = g->hact.as<uint32_t>();
  const unsigned gb = grid_for(n);
  EventPair ev;
  NX_TRY(ev.create());
  NX_CUDA(cudaMemsetAsync(lab, 0xFF, (size_t)n * 4, s));
  NX_CUDA(cudaEventRecord(ev.e0, s));
  uint32_t sweeps = 0, rounds = 0, cc = 0;
  uint64_t swept = 0;
  uint32_t remaining = n;
  // one propagation to a fixed point: sweeps until no interval changed
  auto propagate = [&](ProgKind K, SweepArgs& a, uint32_t nitems, uint32_t** vals, int& cur,
                       uint32_t& ca) -> nx_status {
    for (;;) {
      if (sweeps >= max_sweeps) return NX_OK;
      a.gsrc = vals[cur];
      a.vold = vals[cur];
      a.vnew = vals[1 - cur];
      a.act_in = act[ca];
      a.act_out = act[1 - ca];
      NX_TRY(launch_sweep(K, a, nitems, s));
      ++sweeps;
      swept += g->m;
      cur ^= 1;
      ca ^= 1;
      NX_CUDA(cudaMemcpyAsync(hact, sc.act_count, 4, cudaMemcpyDeviceToHost, s));
      NX_CUDA(cudaStreamSynchronize(s));
      if (hact[0] == 0) return NX_OK;
    }
  };
  while (remaining && sweeps < max_sweeps) {
    ++rounds;
    int cf = 0, cb = 0;
    uint32_t ca = 0;
    k_scc_fwd_init<<<gb, 256, 0, s>>>(n, lab, ids, col[0]);
    NX_LAUNCH_CHECK();
    std::vector<uint32_t> ones(P, 1u);
    NX_CUDA(cudaMemcpyAsync(act[0], ones.data(), (size_t)P * 4, cudaMemcpyHostToDevice, s));
    NX_CUDA(cudaMemsetAsync(act[1], 0, (size_t)P * 4, s));
    NX_TRY(propagate(PK_SCCF, fa, fslot->na, col, cf, ca));
    if (sweeps >= max_sweeps) break;
    const uint32_t* colf = col[cf];
    NX_CUDA(cudaMemsetAsync(act[ca], 0, (size_t)P * 4, s));
    NX_CUDA(cudaMemsetAsync(act[1 - ca], 0, (size_t)P * 4, s));
    k_scc_bwd_init<<<gb, 256, 0, s>>>(n, g->geo.L, colf, ids, bw[0], act[ca]);
    NX_LAUNCH_CHECK();
    ba.aux_u32 = colf;
    NX_TRY(propagate(PK_SCCB, ba, tpl->na, bw, cb, ca));
    NX_CUDA(cudaMemsetAsync(left, 0, 4, s));
    k_scc_assign<<<gb, 256, 0, s>>>(n, colf, bw[cb], lab, left);
    NX_LAUNCH_CHECK();
    NX_CUDA(cudaMemcpyAsync(&remaining, left, 4, cudaMemcpyDeviceToHost, s));
    NX_CUDA(cudaStreamSynchronize(s));
    if (sweeps >= max_sweeps) break;
  }
  NX_CUDA(cudaMemcpyAsync(col[cc], lab, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
  NX_CUDA(cudaEventRecord(ev.e1, s));
  float ms = 0.f;
  NX_TRY(ev.elapsed(&ms));
  g->cur = cc;
  g->last_prog = NX_SCC;
  g->values_set_for = -1;
  if (st) {
    memset(st, 0, sizeof *st);
    st->iters_done = sweeps;
    st->Q = rounds;  // coloring rounds
    st->strategy = NX_SPU;
    st->ms = ms;
    st->edges_swept = swept;
    st->bytes_model = (uint64_t)sweeps * (4 * g->m + 12 * (uint64_t)n);
    st->launches = sweeps + 3 * rounds;
  }
  return NX_OK;
}

// ---------------------------------------------------------------- adjoint
// dL/dw_e = a r_u / W_u (lambda_v - y_u) for edge e = (u, v) in caller order;
// dL/dt_v = (1 - a) lambda_v.
__global__ void k_edge_grad(const uint32_t* __restrict__ src, const uint32_t* __restrict__ dst,
                            uint64_t m, const float* __restrict__ r, const float* __restrict__ W,
                            const float* __restrict__ lam, const float* __restrict__ y, float alpha,
                            float* __restrict__ dw) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    const uint32_t u = src[e], v = dst[e];
    dw[e] = alpha * __ldg(r + u) / __ldg(W + u) * (__ldg(lam + v) - __ldg(y + u));
  }
}

__global__ void k_scale(const float* __restrict__ x, uint32_t n, float f, float* __restrict__ out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    out[v] = f * x[v];
}

__global__ void k_partial_sum(const float* __restrict__ x, uint32_t n, double* __restrict__ part) {
  __shared__ double red[8];
  double s = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    s += (double)x[v];
  for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    part[blockIdx.x] = t;
  }
}


nx_status adjoint_impl(nx_graph* g, const float* grad_r, uint32_t K, float* grad_w, float* grad_t,
                       int dev, nx_run_stats* st) {
  const uint32_t n = g->geo.n, P = g->geo.P;
  const uint64_t m = g->m;
  cudaStream_t s = stream();
  NX_TRY(prepare(g));
  for (int k = 0; k < 2; ++k) NX_TRY(ensure(g->lam[k], (size_t)n * 4));
  NX_TRY(ensure(g->ybuf, (size_t)n * 4));
  NX_TRY(ensure(g->tele, (size_t)n * 4));  // holds g = dL/dr
  if (g->relabeled) {  // caller order -> internal order
    NX_CUDA(cudaMemcpyAsync(g->lam[1].p, grad_r, (size_t)n * 4,
                            dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    NX_TRY(vertex_to_internal(g, g->lam[1].p, g->tele.p));
  } else {
    NX_CUDA(cudaMemcpyAsync(g->tele.p, grad_r, (size_t)n * 4,
                            dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  }
  NX_CUDA(cudaMemcpyAsync(g->lam[0].p, g->tele.p, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
  // S0 = sum of lambda^0
  Scal sc = scal_of(g);
  const unsigned gb = grid_for(n);
  NX_TRY(ensure(g->init_part, (size_t)gb * 8));
  k_partial_sum<<<gb, 256, 0, s>>>(g->lam[0].as<float>(), n, g->init_part.as<double>());
  k_sum_parts<<<1, 256, 0, s>>>(g->init_part.as<double>(), gb, sc.dm);
  NX_LAUNCH_CHECK();
  // plan over the transpose DSSS
  nx_graph::Plan* slotp = nullptr;
  NX_TRY(tr_plan(g, &slotp));
  auto* slot = slotp;
  nx_params p{};
  p.alpha = g->wpr_alpha;
  SweepArgs a = base_args(g, NX_WPR, p, nullptr);
  a.src[0].ew = g->tr.ew.as<uint32_t>();
  a.src[0].wt = g->tr.wt.as<float>();
  a.src[0].piece_off = g->tr.piece_off.as<uint64_t>();
  a.nsrc = 1;
  a.items = slot->items.as<Item>();
  a.split = g->split_buf.p;
  a.tele = g->tele.as<float>();
  a.alpha = g->wpr_alpha;
  EventPair ev;
  NX_TRY(ev.create());
  NX_CUDA(cudaEventRecord(ev.e0, s));
  int cur = 0;
  uint32_t launches = 0;
  for (uint32_t k = 1; k < K; ++k) {  // lambda^{k} = M^T lambda^{k-1} + g
    SweepArgs b = a;
    b.mode = 0;
    b.gsrc = g->lam[cur].p;
    b.vnew = g->lam[1 - cur].p;
    b.dm_in = sc.dm + cur;
    b.dm_out = sc.dm + 1 - cur;
    NX_TRY(launch_sweep(PK_ADJ, b, slot->na, s));
    ++launches;
    cur = 1 - cur;
  }
  {  // y_u = sum_v w^_uv lambda_v: the same sweep, raw accumulators stored
    SweepArgs b = a;
    b.mode = 2;
    b.gsrc = g->lam[cur].p;
    b.accres = g->ybuf.p;
    NX_TRY(launch_sweep(PK_WPR, b, slot->na, s));
    ++launches;
  }
  DevBuf dw_dev;
  float* dwp = grad_w;
  if (!dev) {
    NX_TRY(dw_dev.alloc(std::max<uint64_t>(m, 1) * 4));
    dwp = dw_dev.as<float>();
  }
  if (m) {
    k_edge_grad<<<grid_for(m), 256, 0, s>>>(g->orig_src.as<uint32_t>(), g->orig_dst.as<uint32_t>(),
                                            m, g->val[g->cur].as<float>(), g->wsum.as<float>(),
                                            g->lam[cur].as<float>(), g->ybuf.as<float>(),
                                            g->wpr_alpha, dwp);
    NX_LAUNCH_CHECK();
    ++launches;
  }
  NX_CUDA(cudaEventRecord(ev.e1, s));
  if (!dev && m) NX_CUDA(cudaMemcpyAsync(grad_w, dwp, m * 4, cudaMemcpyDeviceToHost, s));
  if (grad_t) {
    DevBuf dt_dev;
    float* dtp = grad_t;
    if (!dev) {
      NX_TRY(dt_dev.alloc((size_t)n * 4));
      dtp = dt_dev.as<float>();
    }
    if (g->relabeled) {  // internal order -> caller order (lam[1-cur] is free now)
      k_scale<<<grid_for(n), 256, 0, s>>>(g->lam[cur].as<float>(), n, 1.0f - g->wpr_alpha,
                                          g->lam[1 - cur].as<float>());
      NX_LAUNCH_CHECK();
      NX_TRY(vertex_to_caller(g, g->lam[1 - cur].p, dtp));
    } else {
      k_scale<<<grid_for(n), 256, 0, s>>>(g->lam[cur].as<float>(), n, 1.0f - g->wpr_alpha, dtp);
      NX_LAUNCH_CHECK();
    }
    if (!dev) NX_CUDA(cudaMemcpyAsync(grad_t, dtp, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    NX_CUDA(cudaStreamSynchronize(s));
  }
  float ms = 0.f;
  NX_TRY(ev.elapsed(&ms));
  NX_CUDA(cudaStreamSynchronize(s));
  if (st) {
    memset(st, 0, sizeof *st);
    st->iters_done = K;
    st->Q = P;
    st->ms = ms;
    st->edges_swept = m * K;
    // K transpose sweeps (edge word + weight per edge, 16 n per sweep) + the edge pass
    st->bytes_model = (uint64_t)K * (8 * m + 16 * (uint64_t)n) + m * (4 + 4 + 4 + 4 * 4);
    st->launches = launches;
  }
  return NX_OK;
}

// ---------------------------------------------------------------- many graphs
// The executable CUDA graph of a multi-graph run (counter resets + the
// persistent kernel) and the device copies of its arguments. A later call on
// the same graphs with the same program, iteration count, damping and barrier
// limit, whose per-graph arguments are byte-identical (no buffer of any graph
// was reallocated), replays it without capturing again.
struct MultiExec {
  int device = -1;
  std::vector<nx_graph*> graphs;
  int prog = -1;
  float alpha = 0.f;
  uint32_t iters = 0;
  long long limit = 0;
  std::vector<unsigned char> args_img, items_img;
  DevBuf d_args, d_items, d_ctr, d_sync;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  ~MultiExec() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};
constexpr size_t kMultiCacheSize = 4;
std::mutex g_multi_mu;
// most recent last; never destroyed (at process exit the CUDA context and the
// caller's streams may already be gone)
std::vector<std::unique_ptr<MultiExec>>& g_multi_cache = *new std::vector<std::unique_ptr<MultiExec>>();
std::atomic<long long> g_barrier_limit{0};

// Drops the cached executable graphs that sweep `g` (it is being freed).
void multi_cache_drop(const nx_graph* g) {
  std::lock_guard<std::mutex> lock(g_multi_mu);
  auto& c = g_multi_cache;
  for (size_t q = 0; q < c.size();) {
    if (std::find(c[q]->graphs.begin(), c[q]->graphs.end(), g) != c[q]->graphs.end())
      c.erase(c.begin() + q);
    else
      ++q;
  }
}

nx_status multi_impl(nx_graph** gs, uint32_t count, nx_program prog, float alpha, uint32_t iters,
                     nx_run_stats* st) {
  nx_params p{};
  p.alpha = alpha;
  p.root = 0;
  const ProgKind K = kind_of(prog);
  std::vector<SweepArgs> args(2 * (size_t)count);
  std::vector<MItem> items;
  std::vector<uint64_t> costs;
  uint32_t tile_max = 1;
  uint64_t edges = 0;
  for (uint32_t gi = 0; gi < count; ++gi) {
    nx_graph* g = gs[gi];
    NX_TRY(ensure_resident(g));
    NX_TRY(prepare(g));
    NX_TRY(initialize(g, prog, p, nullptr, nullptr));  // sets cur = 0
    g->values_set_for = -1;
    g->last_prog = (int)prog;
    std::vector<const Dsss*> ds{&g->fwd};
    if (prog == NX_WCC) ds.push_back(&g->tr);
    const int key = ((int)NX_SPU * 16 + (int)ds.size()) * 4096;
    auto& slot = g->plans[key];
    if (!slot) {  // cached only once complete
      std::unique_ptr<nx_graph::Plan> fresh(new nx_graph::Plan());
      PlanOut plan;
      plan_tiles(g, ds, 0, g->geo.P, 0, g->geo.P, true, target_block_edges(g->m * ds.size()), plan);
      NX_TRY(upload_items(g, plan, *fresh));
      fresh->na = (uint32_t)fresh->h_items.size();
      slot = std::move(fresh);
    }
    NX_TRY(ensure_split(g, slot->slots));
    SweepArgs a = base_args(g, prog, p, nullptr);
    a.items = nullptr;
    a.split = g->split_buf.p;
    // many small graphs: the flattened schedule keeps all warps busy
    const uint32_t npieces = (uint32_t)a.nsrc * g->geo.P;
    a.flat_cap = npieces <= 256 ? npieces : 0;
    for (int par = 0; par < 2; ++par) {
      g->cur = par;
      set_iter_ptrs(g, prog, a);
      args[2 * (size_t)gi + par] = a;
    }
    g->cur = 0;
    for (size_t q = 0; q < slot->h_items.size(); ++q) {
      MItem mi;
      mi.gid = gi;
      mi.pad = 0;
      mi.it = slot->h_items[q];
      items.push_back(mi);
      costs.push_back(slot->h_cost[q]);
    }
    tile_max = std::max(tile_max, g->geo.tile_max);
    edges += g->m * ds.size();
  }
  // heaviest items first over all graphs
  std::vector<uint32_t> order(items.size());
  for (uint32_t q = 0; q < order.size(); ++q) order[q] = q;
  std::stable_sort(order.begin(), order.end(),
                   [&](uint32_t x, uint32_t y) { return costs[x] > costs[y]; });
  std::vector<MItem> sorted(items.size());
  for (size_t q = 0; q < order.size(); ++q) sorted[q] = items[order[q]];
  const long long limit = barrier_limit();
  int device = 0;
  NX_CUDA(cudaGetDevice(&device));
  const unsigned char* ab = reinterpret_cast<const unsigned char*>(args.data());
  const unsigned char* ib = reinterpret_cast<const unsigned char*>(sorted.data());
  std::vector<unsigned char> args_img(ab, ab + args.size() * sizeof(SweepArgs));
  std::vector<unsigned char> items_img(ib, ib + sorted.size() * sizeof(MItem));
  cudaStream_t s = stream();

  std::lock_guard<std::mutex> lock(g_multi_mu);
  MultiExec* ex = nullptr;
  for (size_t q = 0; q < g_multi_cache.size(); ++q) {
    MultiExec* c = g_multi_cache[q].get();
    if (c->device == device && c->prog == (int)prog && c->alpha == alpha && c->iters == iters &&
        c->limit == limit && c->graphs == std::vector<nx_graph*>(gs, gs + count) &&
        c->args_img == args_img && c->items_img == items_img) {
      std::unique_ptr<MultiExec> keep = std::move(g_multi_cache[q]);  // most recent last
      g_multi_cache.erase(g_multi_cache.begin() + q);
      g_multi_cache.push_back(std::move(keep));
      ex = g_multi_cache.back().get();
      break;
    }
  }
  const bool hit = ex != nullptr;
  if (!hit) {
    std::unique_ptr<MultiExec> c(new MultiExec());
    c->device = device;
    c->graphs.assign(gs, gs + count);
    c->prog = (int)prog;
    c->alpha = alpha;
    c->iters = iters;
    c->limit = limit;
    NX_TRY(c->d_args.alloc(args.size() * sizeof(SweepArgs)));
    NX_TRY(c->d_items.alloc(std::max<size_t>(sorted.size(), 1) * sizeof(MItem)));
    NX_TRY(c->d_ctr.alloc(std::max<size_t>(iters, 1) * 4));
    NX_TRY(c->d_sync.alloc(sizeof(MultiSync)));
    NX_CUDA(cudaMemcpyAsync(c->d_args.p, args.data(), args.size() * sizeof(SweepArgs),
                            cudaMemcpyHostToDevice, s));
    if (!sorted.empty())
      NX_CUDA(cudaMemcpyAsync(c->d_items.p, sorted.data(), sorted.size() * sizeof(MItem),
                              cudaMemcpyHostToDevice, s));
    NX_CUDA(cudaStreamSynchronize(s));
    uint32_t nblocks = 0;
    NX_TRY(multi_blocks(K, tile_max, &nblocks));
    // the whole iteration loop as one CUDA graph: counters reset, then the kernel
    cudaStream_t cs = nullptr;
    NX_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    nx_status rc = NX_OK;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaMemsetAsync(c->d_ctr.p, 0, std::max<size_t>(iters, 1) * 4, cs);
      cudaMemsetAsync(c->d_sync.p, 0, sizeof(MultiSync), cs);
      rc = launch_multi(K, c->d_args.as<SweepArgs>(), c->d_items.as<MItem>(),
                        (uint32_t)sorted.size(), iters, c->d_ctr.as<uint32_t>(),
                        c->d_sync.as<MultiSync>(), tile_max, nblocks, limit, cs);
      cudaError_t e2 = cudaStreamEndCapture(cs, &c->graph);
      if (rc == NX_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "cudaStreamEndCapture", __FILE__, __LINE__);
    } else {
      rc = cuda_fail(e, "cudaStreamBeginCapture", __FILE__, __LINE__);
    }
    cudaStreamDestroy(cs);
    NX_TRY(rc);
    NX_CUDA(cudaGraphInstantiate(&c->exec, c->graph, 0));
    c->args_img.swap(args_img);
    c->items_img.swap(items_img);
    if (g_multi_cache.size() >= kMultiCacheSize) g_multi_cache.erase(g_multi_cache.begin());
    g_multi_cache.push_back(std::move(c));
    ex = g_multi_cache.back().get();
  }
  float ms = 0.f;
  {
    EventPair ev;
    NX_TRY(ev.create());
    NX_CUDA(cudaEventRecord(ev.e0, s));
    NX_CUDA(cudaGraphLaunch(ex->exec, s));
    NX_CUDA(cudaEventRecord(ev.e1, s));
    NX_TRY(ev.elapsed(&ms));
  }
  MultiSync hs{};
  NX_CUDA(cudaMemcpy(&hs, ex->d_sync.p, sizeof hs, cudaMemcpyDeviceToHost));
  if (hs.err) {
    // Blocks that gave up left per-iteration and split-tile completion
    // counters part-way: clear them so the graphs' next runs start clean.
    for (uint32_t gi = 0; gi < count; ++gi) {
      nx_graph* g = gs[gi];
      NX_CUDA(cudaMemsetAsync(scal_of(g).ticket, 0, 8, s));
      NX_CUDA(cudaMemsetAsync(g->tile_ticket.p, 0, g->tile_ticket.bytes, s));
      g->last_prog = -1;
    }
    NX_CUDA(cudaStreamSynchronize(s));
    set_error("nx_run_multi: a grid barrier timed out; values are undefined");
    return NX_ERR_TIMEOUT;
  }
  for (uint32_t gi = 0; gi < count; ++gi) gs[gi]->cur = (int)(iters & 1u);
  if (st) {
    memset(st, 0, sizeof *st);
    st->iters_done = iters;
    st->ms = ms;
    st->edges_swept = edges * iters;
    st->launches = 1;
    st->Q = hit ? 1u : 0u;  // 1: the cached executable graph was replayed
    uint64_t bytes = 0;
    for (uint32_t gi = 0; gi < count; ++gi) bytes += bytes_per_sweep(gs[gi], prog, gs[gi]->m);
    st->bytes_model = bytes * iters;
  }
  return NX_OK;
}

// Largest finite value of a uint32 array plus one (0: none finite).
__global__ void k_max_finite(const uint32_t* __restrict__ v, uint32_t n, uint32_t* __restrict__ out) {
  uint32_t mx = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
    const uint32_t d = v[x];
    if (d != kInf && d + 1 > mx) mx = d + 1;
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

}  // namespace
}  // namespace nx

namespace nx {
long long barrier_limit() {
  const long long v = g_barrier_limit.load();
  return v > 0 ? v : 4000000000ll;  // default: about two seconds at 2 GHz
}
}  // namespace nx

// ---------------------------------------------------------------- C ABI
extern "C" nx_status nx_graph_get_info(const nx_graph* g, nx_graph_info* info) {
  if (!g || !info) return nx::invalid("nx_graph_get_info: NULL argument");
  memset(info, 0, sizeof *info);
  info->n = g->geo.n;
  info->P = g->geo.P;
  info->L = g->geo.L;
  info->ntiles = g->geo.ntiles;
  info->tile_max = g->geo.tile_max;
  info->lb = g->geo.lb;
  info->m = g->m;
  info->D = g->fwd.D;
  info->D_t = g->has_tr ? g->tr.D : 0;
  info->device_bytes = g->device_bytes();
  info->build_ms = g->build_ms;
  info->has_transpose = g->has_tr;
  info->has_weights = g->has_w;
  info->host_bytes = g->host_bytes();
  info->H_onchip = g->oc.built ? g->oc.H : 0;
  return NX_OK;
}

extern "C" nx_status nx_run(nx_graph* g, nx_program program, const nx_params* params,
                            uint32_t iters, nx_strategy strategy, uint64_t mem_budget_bytes,
                            nx_run_stats* stats) {
  if (!g) return nx::invalid("nx_run: graph is NULL");
  if ((int)program < 0 || (int)program > 5) return nx::invalid("nx_run: unknown program");
  nx::TraceRange trace("nx_run");
  if ((int)strategy < 0 || (int)strategy > 6) return nx::invalid("nx_run: unknown strategy");
  if (program == NX_SCC) {
    if (!g->has_tr) return nx::invalid("nx_run: SCC needs the transpose DSSS (NX_WITH_TRANSPOSE)");
    if ((strategy != NX_SPU && strategy != NX_AUTO) || mem_budget_bytes)
      return nx::invalid("nx_run: SCC runs under SPU without a budget");
    return nx::scc_impl(g, iters, stats);
  }
  nx_params p{};
  p.alpha = 0.85f;
  if (params) p = *params;
  if (!(p.alpha >= 0.f && p.alpha < 1.f)) return nx::invalid("nx_run: alpha must be in [0, 1)");
  if (program == NX_BFS && g->relabeled && p.root < g->geo.n) {  // caller id -> internal id
    NX_CUDA(cudaMemcpyAsync(&p.root, g->new_of_old.as<uint32_t>() + p.root, 4,
                            cudaMemcpyDeviceToHost, nx::stream()));
    NX_CUDA(cudaStreamSynchronize(nx::stream()));
  }
  return nx::run_impl(g, program, p, iters, strategy, mem_budget_bytes, stats);
}

extern "C" nx_status nx_adjoint_wpr(nx_graph* g, const float* grad_r, uint32_t adj_terms,
                                    float* grad_w, float* grad_t, int32_t ptrs_are_device,
                                    nx_run_stats* stats) {
  if (!g || !grad_r || !grad_w) return nx::invalid("nx_adjoint_wpr: NULL argument");
  if (!g->has_w || !g->has_tr)
    return nx::invalid("nx_adjoint_wpr: needs NX_WITH_WEIGHTS and NX_WITH_TRANSPOSE");
  if (g->last_prog != NX_WPR)
    return nx::invalid("nx_adjoint_wpr: run NX_WPR first (its ranks are the forward state)");
  if (adj_terms == 0) return nx::invalid("nx_adjoint_wpr: adj_terms must be >= 1");
  nx::TraceRange trace("nx_adjoint_wpr");
  NX_TRY(nx::ensure_resident(g));
  return nx::adjoint_impl(g, grad_r, adj_terms, grad_w, grad_t, ptrs_are_device, stats);
}

extern "C" nx_status nx_run_multi(nx_graph** graphs, uint32_t count, nx_program program,
                                  float alpha, uint32_t iters, nx_run_stats* stats) {
  if (!graphs || count == 0) return nx::invalid("nx_run_multi: no graphs");
  if (program == NX_PPR) return nx::invalid("nx_run_multi: PPR needs a teleport; use PR, WPR, BFS, WCC");
  if ((int)program < 0 || (int)program > 4)
    return nx::invalid("nx_run_multi: unknown program (SCC runs through nx_run)");
  if (!(alpha >= 0.f && alpha < 1.f)) return nx::invalid("nx_run_multi: alpha must be in [0, 1)");
  for (uint32_t q = 0; q < count; ++q) {
    const nx_graph* g = graphs[q];
    if (!g) return nx::invalid("nx_run_multi: a graph is NULL");
    for (uint32_t r = 0; r < q; ++r)
      if (graphs[r] == g) return nx::invalid("nx_run_multi: a graph appears twice");
    if (program == NX_WCC && !g->has_tr) return nx::invalid("nx_run_multi: WCC needs the transpose");
    if (program == NX_WPR && !g->has_w) return nx::invalid("nx_run_multi: WPR needs weights");
    if (g->relabeled) return nx::invalid("nx_run_multi: a graph was built with NX_RELABEL");
  }
  nx::TraceRange trace("nx_run_multi");
  return nx::multi_impl(graphs, count, program, alpha, iters, stats);
}

extern "C" nx_status nx_gather_probe(nx_graph* g, uint32_t sweeps, float* ms_per_sweep) {
  if (!g || !ms_per_sweep) return nx::invalid("nx_gather_probe: NULL argument");
  if (sweeps == 0) return nx::invalid("nx_gather_probe: sweeps must be >= 1");
  return nx::probe_impl(g, sweeps, ms_per_sweep);
}

extern "C" nx_status nx_set_barrier_limit(uint64_t cycles) {
  if (cycles > (1ull << 62)) return nx::invalid("nx_set_barrier_limit: limit too large");
  nx::g_barrier_limit.store((long long)cycles);
  return NX_OK;
}

extern "C" nx_status nx_bfs_max_depth(const nx_graph* g, int64_t* max_depth) {
  if (!g || !max_depth) return nx::invalid("nx_bfs_max_depth: NULL argument");
  if (g->last_prog != NX_BFS)
    return nx::invalid("nx_bfs_max_depth: the graph's current values are not BFS depths");
  uint32_t* slot = reinterpret_cast<uint32_t*>(g->scal.as<unsigned char>() + 32);
  NX_CUDA(cudaMemsetAsync(slot, 0, 4, nx::stream()));
  nx::k_max_finite<<<nx::grid_for(g->geo.n), 256, 0, nx::stream()>>>(
      g->val[g->cur].as<uint32_t>(), g->geo.n, slot);
  NX_LAUNCH_CHECK();
  uint32_t h = 0;
  NX_CUDA(cudaMemcpyAsync(&h, slot, 4, cudaMemcpyDeviceToHost, nx::stream()));
  NX_CUDA(cudaStreamSynchronize(nx::stream()));
  *max_depth = (int64_t)h - 1;
  return NX_OK;
}

extern "C" nx_status nx_get_values(const nx_graph* g, void* out, uint64_t count,
                                   int32_t out_is_device) {
  if (!g || !out) return nx::invalid("nx_get_values: NULL argument");
  if (count != g->geo.n) return nx::invalid("nx_get_values: count must equal n");
  if (g->last_prog < 0 && g->values_set_for < 0) return nx::invalid("nx_get_values: nothing run yet");
  if (g->relabeled) {  // internal order -> caller order
    nx::DevBuf tmp;
    void* dst = out;
    if (!out_is_device) {
      NX_TRY(tmp.alloc(count * 4));
      dst = tmp.p;
    }
    NX_TRY(nx::vertex_to_caller(g, g->val[g->cur].p, dst));
    if (!out_is_device)
      NX_CUDA(cudaMemcpyAsync(out, tmp.p, count * 4, cudaMemcpyDeviceToHost, nx::stream()));
    NX_CUDA(cudaStreamSynchronize(nx::stream()));
    return NX_OK;
  }
  NX_CUDA(cudaMemcpyAsync(out, g->val[g->cur].p, count * 4,
                          out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          nx::stream()));
  NX_CUDA(cudaStreamSynchronize(nx::stream()));
  return NX_OK;
}

extern "C" nx_status nx_set_values(nx_graph* g, nx_program program, const void* in, uint64_t count,
                                   int32_t in_is_device) {
  if (!g || !in) return nx::invalid("nx_set_values: NULL argument");
  if (count != g->geo.n) return nx::invalid("nx_set_values: count must equal n");
  if ((int)program < 0 || (int)program > 4)
    return nx::invalid("nx_set_values: unknown program (SCC does not resume)");
  NX_TRY(nx::prepare(g));
  if (g->relabeled) {  // caller order -> internal order
    nx::DevBuf tmp;
    const void* src = in;
    if (!in_is_device) {
      NX_TRY(tmp.alloc(count * 4));
      NX_CUDA(cudaMemcpyAsync(tmp.p, in, count * 4, cudaMemcpyHostToDevice, nx::stream()));
      src = tmp.p;
    }
    NX_TRY(nx::vertex_to_internal(g, src, g->val[g->cur].p));
  } else {
    NX_CUDA(cudaMemcpyAsync(g->val[g->cur].p, in, count * 4,
                            in_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            nx::stream()));
  }
  NX_CUDA(cudaStreamSynchronize(nx::stream()));
  g->values_set_for = (int)program;
  g->last_prog = (int)program;
  return NX_OK;
}

extern "C" void nx_graph_free(nx_graph* g) {
  if (!g) return;
  cudaStreamSynchronize(nx::stream());
  nx::multi_cache_drop(g);
  delete g;
}

extern "C" nx_status nx_io_model(nx_strategy s, double n, double m, double P, double B_M,
                                 double B_a, double B_v, double B_e, double d, double* Q,
                                 double* bytes_read, double* bytes_write) {
  if (n <= 0 || P <= 0 || B_a <= 0 || d <= 0) return nx::invalid("nx_io_model: bad sizes");
  double q = std::min(P, std::floor(B_M * P / (2.0 * n * B_a)));
  double rd = 0, wr = 0;
  switch (s) {
    case NX_SPU:  // Section III-B1: B_read = m B_e + 2 n B_a - B_M (>= 0), no writes
      q = P;
      rd = std::max(0.0, m * B_e + 2.0 * n * B_a - B_M);
      wr = 0;
      break;
    case NX_DPU:  // Section III-B2
      q = 0;
      rd = m * (B_e + (B_a + B_v) / d) + n * B_a;
      wr = m * (B_a + B_v) / d + n * B_a;
      break;
    case NX_MPU:
    case NX_AUTO: {  // Section III-B3 (sub-shards of equal size)
      if (q < 0) q = 0;
      // Table II form: the hubbed (P-Q)^2 sub-shards carry (B_a + B_v)/d per edge
      const double f = (P - q) / P;
      rd = m * (B_e + f * f * (B_a + B_v) / d) + f * n * B_a;
      wr = f * f * m * (B_a + B_v) / d + f * n * B_a;
      break;
    }
    default:  // the Table IV ablation strategies have no I/O model in the paper
      return nx::invalid("nx_io_model: the model covers SPU, DPU, MPU and AUTO only");
  }
  if (Q) *Q = q;
  if (bytes_read) *bytes_read = rd;
  if (bytes_write) *bytes_write = wr;
  return NX_OK;
}


namespace nx {
namespace {
// Decodes stored edge words back to endpoints (tile geometry + piece table).
__global__ void k_export(const uint32_t* __restrict__ ew, const uint64_t* __restrict__ piece_off,
                         const uint32_t* __restrict__ tile_start, const uint32_t* __restrict__ col_tb,
                         uint32_t P, uint32_t L, uint32_t lb, uint64_t npieces,
                         uint32_t* __restrict__ s_out, uint32_t* __restrict__ d_out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t pc = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; pc < npieces; pc += stride) {
    // invert piece_index: column j from the tile prefix, then (i, t)
    uint32_t lo = 0, hi = P;  // find j with P*tb[j] <= pc < P*tb[j+1]
    while (hi - lo > 1) {
      uint32_t mid = (lo + hi) / 2;
      if ((uint64_t)P * col_tb[mid] <= pc) lo = mid; else hi = mid;
    }
    const uint32_t j = lo, tb = col_tb[j], nt = col_tb[j + 1] - tb;
    if (nt == 0) continue;
    const uint64_t r = pc - (uint64_t)P * tb;
    const uint32_t i = (uint32_t)(r / nt), t = tb + (uint32_t)(r % nt);
    const uint32_t mask = (1u << lb) - 1u;
    for (uint64_t e = piece_off[pc]; e < piece_off[pc + 1]; ++e) {
      const uint32_t w = ew[e];
      s_out[e] = i * L + (w & mask);
      d_out[e] = tile_start[t] + (w >> lb);
    }
  }
}
}  // namespace
}  // namespace nx

extern "C" nx_status nx_dsss_export(const nx_graph* g, int32_t transpose, uint32_t* src,
                                    uint32_t* dst, uint64_t* sub_off) {
  if (!g || !src || !dst) return nx::invalid("nx_dsss_export: NULL argument");
  if (transpose && !g->has_tr) return nx::invalid("nx_dsss_export: no transpose DSSS");
  NX_TRY(nx::ensure_resident(const_cast<nx_graph*>(g)));
  const nx::Dsss& d = transpose ? g->tr : g->fwd;
  const uint64_t m = g->m, np = (uint64_t)g->geo.P * g->geo.ntiles;
  nx::DevBuf s, t;
  NX_TRY(s.alloc(std::max<uint64_t>(m, 1) * 4));
  NX_TRY(t.alloc(std::max<uint64_t>(m, 1) * 4));
  nx::k_export<<<nx::grid_for(np), 256, 0, nx::stream()>>>(
      d.ew.as<uint32_t>(), d.piece_off.as<uint64_t>(), g->geo.tile_start.as<uint32_t>(),
      g->geo.col_tb.as<uint32_t>(), g->geo.P, g->geo.L, g->geo.lb, np, s.as<uint32_t>(),
      t.as<uint32_t>());
  NX_LAUNCH_CHECK();
  // the transpose stores (original dst, original src): swap back
  uint32_t* so = transpose ? dst : src;
  uint32_t* dout = transpose ? src : dst;
  if (m) {
    NX_CUDA(cudaMemcpyAsync(so, s.p, m * 4, cudaMemcpyDeviceToHost, nx::stream()));
    NX_CUDA(cudaMemcpyAsync(dout, t.p, m * 4, cudaMemcpyDeviceToHost, nx::stream()));
  }
  NX_CUDA(cudaStreamSynchronize(nx::stream()));
  if (sub_off) {
    const uint32_t P = g->geo.P;
    const auto& tb = g->geo.h_col_tb;
    for (uint32_t j = 0; j < P; ++j)
      for (uint32_t i = 0; i < P; ++i) {
        const uint32_t nt = tb[j + 1] - tb[j];
        sub_off[(uint64_t)j * P + i] =
            nt ? d.h_piece_off[nx::piece_index(P, tb[j], nt, i, tb[j])]
               : d.h_piece_off[(uint64_t)P * tb[j]];
      }
    sub_off[(uint64_t)P * P] = m;
  }
  return NX_OK;
}
