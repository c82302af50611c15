// Batched personalized PageRank: B teleport vectors solved by one DSSS sweep
// per iteration (an extension of the paper's PageRank task).
//
// Values are stored vertex-major, [n][Bp] floats with Bp = 32 or 64 (B padded),
// so every edge gathers one contiguous Bp-float row of its source — 128 or
// 256 bytes, all of it used — instead of one scalar. A thread block owns a
// sub-tile of SUB destinations of a DSSS tile; for each source interval i it
// binary-searches the sub-tile's range inside piece (i, t) (edges are sorted
// by destination inside a piece) and its warps walk those edges 32 at a time:
// lane l loads edge word l, then the warp broadcasts each edge and gathers the
// source row with 16-byte loads by Bp/4 lanes, so one warp instruction serves
// 2 (Bp = 64) or 4 (Bp = 32) edges. Runs of equal destination accumulate in
// registers (at most the edges of one lane group in a 32-edge chunk) and are
// flushed to the shared-memory row of that destination with one atomic per
// column.
//
//   r'[v][b] = (1-a) t[v][b] + a (sum_{u->v} c[u][b] + Dm[b] t[v][b]),
//   c'[v][b] = r'[v][b] / outdeg(v) (0 if dangling), Dm[b] = sum_{dangling} r[v][b].
// Teleport vectors are sparse (a few seeds each), so the sweep's epilogue
// writes a * acc only and a second small kernel adds the teleport terms at the
// seed entries (their c and, when dangling, the next dangling mass). The rank
// array itself is written by the last iteration only; every iteration writes
// the contributions c it needs next.
#include <algorithm>
#include <cstring>

#include "nx_sweep.cuh"

namespace nx {
namespace {

constexpr int kBT = 256;  // threads per block
constexpr int kBW = kBT / 32;
// Shape (run-time choices, nx_set_batch_shape / nx_autotune_ppr_batch): the
// destinations per sub-tile (a block's shared-memory rows) and the source
// rows each lane group keeps in flight (a template parameter: 2, 4 or 8).

struct BItem {
  uint32_t tile, sub;      // tile and sub-tile index inside it
  uint32_t nsplit, part;   // blocks sharing the sub-tile, this block's index
  uint32_t slot, group;    // first split slot, completion counter of the group
  uint64_t vbeg, vend;     // range of the sub-tile's virtual edge sequence
};

struct BArgs {
  int write_r;        // last iteration: also store r
  const uint32_t* ew;
  const uint64_t* piece_off;
  const uint32_t* tile_start;
  const uint32_t* col_tb;
  const uint32_t* outdeg;
  uint32_t P, L, lb, n;
  const BItem* items;
  const float* c_in;  // [n][Bp]
  float* r_out;       // [n][Bp]
  float* c_out;       // [n][Bp]
  const double* dm_in;  // [Bp]
  double* dm_out;       // [Bp] (accumulated with atomics; zeroed before)
  float* split;         // split slots [sub * Bp] each
  uint32_t* ticket;     // per split group
  float alpha;
  uint32_t sub;         // destinations per sub-tile
};

// First position in ew[p0, p1) whose destination offset (word >> lb) is >= key.
__device__ __forceinline__ uint64_t lower_key(const uint32_t* __restrict__ ew, uint64_t p0,
                                              uint64_t p1, uint32_t lb, uint32_t key) {
  while (p0 < p1) {
    const uint64_t mid = p0 + ((p1 - p0) >> 1);
    if ((__ldg(ew + mid) >> lb) < key) p0 = mid + 1;
    else p1 = mid;
  }
  return p0;
}

// Lanes per edge: a BP-float row is read with 16-byte loads by LPE = BP / 4
// lanes, so a warp works on 32 / LPE edges at once. In shared memory, column b
// of a destination row is stored at (b % 4) * LPE + b / 4: the q-th component
// of the float4 of lane gl goes to q * LPE + gl, so the lanes of one group add
// into consecutive words.
template <int BP>
__device__ __forceinline__ uint32_t acc_pos(uint32_t b) {
  return (b % 4) * (BP / 4) + b / 4;
}

// Register budget for five blocks per SM with up to four rows in flight (four
// blocks with eight): the extra warps' row gathers in flight made the tuned
// shape (4 rows, 128-destination sub-tiles) 10.7% faster at R-MAT scale 24
// with 64 vectors (13.06 vs 14.63 ms per iteration), despite a few spilled
// registers.
template <int BP, int kRows>
__global__ void __launch_bounds__(kBT, kRows <= 4 ? 5 : 4) k_ppr_batch(const BArgs a) {
  constexpr int C = BP / 32;   // columns per lane in the epilogue
  constexpr int LPE = BP / 4;  // lanes per edge in the sweep
  constexpr int NG = 32 / LPE; // edge groups per warp
  constexpr int EPG = 32 / NG; // chunk edges per group
  static_assert(EPG % kRows == 0, "kRows must divide the edges of a group");
  extern __shared__ __align__(16) unsigned char smem[];
  const uint32_t kSub = a.sub;
  float* acc = reinterpret_cast<float*>(smem);                          // [sub][BP]
  uint64_t* rlo = reinterpret_cast<uint64_t*>(acc + kSub * BP);          // [P]
  uint64_t* rlen = rlo + a.P;                                             // [P + 1] (prefix)
  __shared__ int s_last;
  const BItem it = a.items[blockIdx.x];
  const uint32_t t = it.tile;
  const uint32_t ts = a.tile_start[t], te = a.tile_start[t + 1];
  const uint32_t j = ts / a.L;
  const uint32_t tb = a.col_tb[j], nt = a.col_tb[j + 1] - tb;
  const uint32_t k0 = it.sub * kSub;  // destination offsets [k0, k1) in the tile
  const uint32_t k1 = min(k0 + kSub, te - ts);
  const uint32_t nrows = k1 - k0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / LPE, gl = lane % LPE;
  auto flush = [&](float* arow, const float4 v) {
    atomicAdd(arow + gl, v.x);
    atomicAdd(arow + LPE + gl, v.y);
    atomicAdd(arow + 2 * LPE + gl, v.z);
    atomicAdd(arow + 3 * LPE + gl, v.w);
  };
  for (uint32_t q = threadIdx.x; q < kSub * BP; q += kBT) acc[q] = 0.f;
  // sub-tile range inside every piece (i, t)
  for (uint32_t i = threadIdx.x; i < a.P; i += kBT) {
    const uint64_t pc = piece_index(a.P, tb, nt, i, t);
    const uint64_t p0 = a.piece_off[pc], p1 = a.piece_off[pc + 1];
    const uint64_t lo = lower_key(a.ew, p0, p1, a.lb, k0);
    const uint64_t hi = lower_key(a.ew, lo, p1, a.lb, k1);
    rlo[i] = lo;
    rlen[i] = hi - lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // exclusive prefix of the range lengths
    uint64_t s = 0;
    for (uint32_t i = 0; i < a.P; ++i) {
      const uint64_t l = rlen[i];
      rlen[i] = s;
      s += l;
    }
    rlen[a.P] = s;
  }
  __syncthreads();
  const uint32_t smask = (1u << a.lb) - 1u;
  // walk the virtual sequence in 32-edge chunks, chunk q to warp q % kBW
  uint32_t rot = 0;
  for (uint32_t i = 0; i < a.P; ++i) {
    const uint64_t v0 = rlen[i], v1 = rlen[i + 1];
    const uint64_t vb = v0 > it.vbeg ? v0 : it.vbeg;
    const uint64_t ve = v1 < it.vend ? v1 : it.vend;
    if (vb >= ve) continue;
    const uint64_t e0 = rlo[i] + (vb - v0), e1 = rlo[i] + (ve - v0);
    const uint32_t nch = (uint32_t)((e1 - e0 + 31) >> 5);
    const uint32_t first = (uint32_t)((warp - (int)rot) & (kBW - 1));
    rot = (rot + nch) & (kBW - 1);
    const uint32_t sbase = i * a.L;
    for (uint32_t ch = first; ch < nch; ch += kBW) {
      const uint64_t e = e0 + (uint64_t)ch * 32 + lane;
      const uint32_t w = e < e1 ? __ldcs(a.ew + e) : 0xFFFFFFFFu;
      const uint64_t left = e1 - (e0 + (uint64_t)ch * 32);
      const uint32_t cnt = left < 32 ? (uint32_t)left : 32u;
      // group grp takes the chunk's edges [grp * EPG, (grp + 1) * EPG); a run in
      // registers spans at most those edges: plain sums
      float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
      uint32_t curk = 0xFFFFFFFFu;
      const uint32_t g0 = (uint32_t)grp * EPG;
      for (uint32_t x = 0; x < (uint32_t)EPG; x += kRows) {
        float4 row[kRows];
        uint32_t key[kRows];
#pragma unroll
        for (int y = 0; y < kRows; ++y) {  // kRows rows in flight per group
          const uint32_t ce = g0 + x + y;
          const uint32_t wy = __shfl_sync(0xffffffffu, w, ce);
          const bool ok = ce < cnt;
          key[y] = ok ? (wy >> a.lb) - k0 : 0xFFFFFFFFu;
          const float4* src = reinterpret_cast<const float4*>(
              a.c_in + (size_t)(sbase + (wy & smask)) * BP + gl * 4);
          row[y] = ok ? __ldg(src) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int y = 0; y < kRows; ++y) {
          if (key[y] == 0xFFFFFFFFu) continue;
          if (key[y] != curk) {
            if (curk != 0xFFFFFFFFu) flush(acc + curk * BP, sum);
            curk = key[y];
            sum = row[y];
          } else {
            sum.x += row[y].x;
            sum.y += row[y].y;
            sum.z += row[y].z;
            sum.w += row[y].w;
          }
        }
      }
      if (curk != 0xFFFFFFFFu) flush(acc + curk * BP, sum);
    }
  }
  __syncthreads();
  if (it.nsplit > 1) {  // combine the blocks of a split sub-tile in slot order
    float* mine = a.split + (size_t)(it.slot + it.part) * kSub * BP;
    for (uint32_t q = threadIdx.x; q < nrows * BP; q += kBT) mine[q] = acc[q];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(a.ticket + it.group, 1u) == it.nsplit - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) a.ticket[it.group] = 0;
    for (uint32_t q = threadIdx.x; q < nrows * BP; q += kBT) {
      double v = 0.0;
      for (uint32_t z = 0; z < it.nsplit; ++z)
        v += (double)__ldcg(a.split + (size_t)(it.slot + z) * kSub * BP + q);
      acc[q] = (float)v;
    }
    __syncthreads();
  }
  // epilogue: warp w takes rows w, w + kBW, ...; lane l columns [l*C, l*C + C)
  double dang[C];
#pragma unroll
  for (int q = 0; q < C; ++q) dang[q] = 0.0;
  const float al = a.alpha;
  for (uint32_t rr = warp; rr < nrows; rr += kBW) {
    const uint32_t v = ts + k0 + rr;
    const uint32_t od = a.outdeg[v];
#pragma unroll
    for (int q = 0; q < C; ++q) {
      const size_t o = (size_t)v * BP + lane * C + q;
      // the teleport terms are added afterwards at the seed entries
      const float r = al * acc[rr * BP + acc_pos<BP>(lane * C + q)];
      if (a.write_r) a.r_out[o] = r;
      a.c_out[o] = od ? r / (float)od : 0.0f;
      if (od == 0) dang[q] += (double)r;
    }
  }
  // per-column dangling mass: fold warps through shared memory, one atomic per column
  __syncthreads();
  double* red = reinterpret_cast<double*>(acc);  // reuse: [kBW][BP]
#pragma unroll
  for (int q = 0; q < C; ++q) red[warp * BP + lane * C + q] = dang[q];
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < BP; b += kBT) {
    double s2 = 0.0;
    for (int w2 = 0; w2 < kBW; ++w2) s2 += red[w2 * BP + b];
    if (s2 != 0.0) atomicAdd(a.dm_out + b, s2);
  }
}

// Per sub-tile edge counts (for the work plan): one thread per (sub-tile, piece).
__global__ void k_subtile_cost(const uint32_t* __restrict__ ew, const uint64_t* __restrict__ po,
                               const uint32_t* __restrict__ tile_start,
                               const uint32_t* __restrict__ col_tb, const uint32_t* __restrict__ sub_of,
                               const uint32_t* __restrict__ sub_tile, uint32_t nsub, uint32_t P,
                               uint32_t L, uint32_t lb, uint32_t kSub,
                               unsigned long long* __restrict__ cost) {
  const uint64_t total = (uint64_t)nsub * P;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += stride) {
    const uint32_t sidx = (uint32_t)(x / P), i = (uint32_t)(x % P);
    const uint32_t t = sub_tile[sidx];
    const uint32_t k0 = (sidx - sub_of[t]) * kSub;
    const uint32_t ts = tile_start[t], te = tile_start[t + 1];
    const uint32_t k1 = min(k0 + kSub, te - ts);
    const uint32_t j = ts / L, tb = col_tb[j], nt = col_tb[j + 1] - tb;
    const uint64_t pc = piece_index(P, tb, nt, i, t);
    const uint64_t p0 = po[pc], p1 = po[pc + 1];
    const uint64_t lo = lower_key(ew, p0, p1, lb, k0);
    const uint64_t hi = lower_key(ew, lo, p1, lb, k1);
    if (hi > lo) atomicAdd(cost + sidx, (unsigned long long)(hi - lo));
  }
}

// Nonzero teleport entries (vertex, column, value), appended in any order;
// rows are in caller order, vertices stored as internal ids (map nullable).
__global__ void k_seed_list(const float* __restrict__ t_in, uint32_t B, uint32_t n,
                            const uint32_t* __restrict__ map, uint32_t* __restrict__ cnt,
                            uint32_t cap, uint32_t* __restrict__ sv, uint32_t* __restrict__ sb,
                            float* __restrict__ st) {
  const uint64_t total = (uint64_t)n * B;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += stride) {
    const float tv = t_in[x];
    if (tv != 0.f) {
      const uint32_t k = atomicAdd(cnt, 1u);
      if (k < cap) {
        const uint32_t v = (uint32_t)(x / B);
        sv[k] = map ? map[v] : v;
        sb[k] = (uint32_t)(x % B);
        st[k] = tv;
      }
    }
  }
}

// Teleport terms at the seeds: delta = a Dm_in[b] t + (1 - a) t added to r
// (through c = r / outdeg, or to the next dangling mass when v is dangling).
// init != 0: r0 = t, c0 = t / outdeg, Dm0 = sum of dangling t.
__global__ void k_seed_apply(uint32_t nnz, const uint32_t* __restrict__ sv,
                             const uint32_t* __restrict__ sb, const float* __restrict__ st,
                             uint32_t BP, const uint32_t* __restrict__ od, float alpha, int init,
                             const double* __restrict__ dm_in, double* __restrict__ dm_out,
                             float* __restrict__ c, float* __restrict__ r) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += stride) {
    const uint32_t v = sv[k], b = sb[k];
    const float tv = st[k];
    const float delta = init ? tv : (alpha * (float)dm_in[b] * tv + (1.0f - alpha) * tv);
    const size_t o = (size_t)v * BP + b;
    const uint32_t d = od[v];
    if (d) c[o] += delta / (float)d;
    else atomicAdd(dm_out + b, (double)delta);
    if (r) r[o] += delta;
  }
}

// [n][B] output rows in caller order (map: caller -> internal id, nullable).
__global__ void k_ppr_out(const float* __restrict__ r, uint32_t B, uint32_t BP, uint32_t n,
                          const uint32_t* __restrict__ map, float* __restrict__ out) {
  const uint64_t total = (uint64_t)n * B;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += stride) {
    const uint32_t v = (uint32_t)(x / B);
    out[x] = r[(size_t)(map ? map[v] : v) * BP + (x % B)];
  }
}

// The kernel instance for B padded to BP and `rows` source rows in flight.
void (*batch_kernel(uint32_t BP, uint32_t rows))(const BArgs) {
  if (BP == 32) {
    if (rows == 2) return k_ppr_batch<32, 2>;
    if (rows == 4) return k_ppr_batch<32, 4>;
    if (rows == 8) return k_ppr_batch<32, 8>;
  } else {
    if (rows == 2) return k_ppr_batch<64, 2>;
    if (rows == 4) return k_ppr_batch<64, 4>;
    if (rows == 8) return k_ppr_batch<64, 8>;
  }
  return nullptr;
}

unsigned grid_of(uint64_t work) {
  return (unsigned)std::min<uint64_t>(ceil_div(work ? work : 1, 256), (uint64_t)num_sms() * 16);
}

nx_status ppr_batch_impl(nx_graph* g, const float* tele_in, uint32_t B, uint32_t iters,
                         float alpha, float* ranks, int dev_ptrs, nx_run_stats* st) {
  const uint32_t n = g->geo.n, P = g->geo.P, L = g->geo.L;
  const uint32_t BP = B <= 32 ? 32 : 64;
  const uint32_t kSub = g->ppr_sub;
  cudaStream_t s = stream();
  // sub-tiles
  const auto& tsh = g->geo.h_tile_start;
  const uint32_t ntiles = g->geo.ntiles;
  std::vector<uint32_t> sub_of(ntiles + 1, 0);
  for (uint32_t t = 0; t < ntiles; ++t)
    sub_of[t + 1] = sub_of[t] + (uint32_t)ceil_div(tsh[t + 1] - tsh[t], kSub);
  const uint32_t nsub = sub_of[ntiles];
  std::vector<uint32_t> sub_tile(nsub);
  for (uint32_t t = 0; t < ntiles; ++t)
    for (uint32_t q = sub_of[t]; q < sub_of[t + 1]; ++q) sub_tile[q] = t;
  DevBuf d_sub_of, d_sub_tile, d_cost;
  NX_TRY(d_sub_of.alloc((ntiles + 1) * 4));
  NX_TRY(d_sub_tile.alloc(std::max<size_t>(nsub, 1) * 4));
  NX_TRY(d_cost.alloc(std::max<size_t>(nsub, 1) * 8));
  NX_CUDA(cudaMemcpyAsync(d_sub_of.p, sub_of.data(), (ntiles + 1) * 4, cudaMemcpyHostToDevice, s));
  NX_CUDA(cudaMemcpyAsync(d_sub_tile.p, sub_tile.data(), (size_t)nsub * 4, cudaMemcpyHostToDevice, s));
  NX_CUDA(cudaMemsetAsync(d_cost.p, 0, std::max<size_t>(nsub, 1) * 8, s));
  k_subtile_cost<<<grid_of((uint64_t)nsub * P), 256, 0, s>>>(
      g->fwd.ew.as<uint32_t>(), g->fwd.piece_off.as<uint64_t>(), g->geo.tile_start.as<uint32_t>(),
      g->geo.col_tb.as<uint32_t>(), d_sub_of.as<uint32_t>(), d_sub_tile.as<uint32_t>(), nsub, P, L,
      g->geo.lb, kSub, d_cost.as<unsigned long long>());
  NX_LAUNCH_CHECK();
  std::vector<uint64_t> cost(nsub);
  NX_CUDA(cudaMemcpyAsync(cost.data(), d_cost.p, (size_t)nsub * 8, cudaMemcpyDeviceToHost, s));
  NX_CUDA(cudaStreamSynchronize(s));
  // plan: heavy sub-tiles are split over several blocks
  const uint64_t blk = std::max<uint64_t>(2048, g->m / ((uint64_t)num_sms() * 16));
  std::vector<std::pair<uint64_t, BItem>> tmp;
  uint32_t slots = 0, groups = 0;
  for (uint32_t q = 0; q < nsub; ++q) {
    const uint64_t c = cost[q];
    const uint32_t k = c > 2 * blk ? (uint32_t)ceil_div(c, blk) : 1;
    for (uint32_t z = 0; z < k; ++z) {
      BItem it{};
      it.tile = sub_tile[q];
      it.sub = q - sub_of[it.tile];
      it.nsplit = k;
      it.part = z;
      it.slot = k > 1 ? slots : 0;
      it.group = k > 1 ? groups : 0;
      it.vbeg = c * z / k;
      it.vend = (z + 1 == k) ? ~0ull : c * (z + 1) / k;
      tmp.push_back({c / k + 1, it});
    }
    if (k > 1) {
      slots += k;
      ++groups;
    }
  }
  std::stable_sort(tmp.begin(), tmp.end(),
                   [](const auto& x, const auto& y) { return x.first > y.first; });
  std::vector<BItem> items;
  items.reserve(tmp.size());
  for (auto& x : tmp) items.push_back(x.second);
  DevBuf d_items, d_split, d_ticket, rv, cv[2], dm;
  NX_TRY(d_items.alloc(std::max<size_t>(items.size(), 1) * sizeof(BItem)));
  NX_CUDA(cudaMemcpyAsync(d_items.p, items.data(), items.size() * sizeof(BItem),
                          cudaMemcpyHostToDevice, s));
  NX_TRY(d_split.alloc(std::max<size_t>((size_t)slots * kSub * BP * 4, 4)));
  NX_TRY(d_ticket.alloc(std::max<size_t>(groups, 1) * 4));
  NX_CUDA(cudaMemsetAsync(d_ticket.p, 0, std::max<size_t>(groups, 1) * 4, s));
  const size_t vb = (size_t)n * BP * 4;
  NX_TRY(rv.alloc(vb));
  for (int k = 0; k < 2; ++k) NX_TRY(cv[k].alloc(vb));
  NX_TRY(dm.alloc(2 * BP * 8));
  NX_CUDA(cudaMemsetAsync(dm.p, 0, 2 * BP * 8, s));
  // teleport (host or device) -> list of seed entries
  DevBuf tin, cnt, sv, sb, sval;
  const float* t_dev = tele_in;
  if (!dev_ptrs) {
    NX_TRY(tin.alloc((size_t)n * B * 4));
    NX_CUDA(cudaMemcpyAsync(tin.p, tele_in, (size_t)n * B * 4, cudaMemcpyHostToDevice, s));
    t_dev = tin.as<float>();
  }
  NX_TRY(cnt.alloc(4));
  NX_CUDA(cudaMemsetAsync(cnt.p, 0, 4, s));
  const uint32_t* map = g->relabeled ? g->new_of_old.as<uint32_t>() : nullptr;
  k_seed_list<<<grid_of((uint64_t)n * B), 256, 0, s>>>(t_dev, B, n, map, cnt.as<uint32_t>(), 0,
                                                       nullptr, nullptr, nullptr);
  NX_LAUNCH_CHECK();
  uint32_t nnz = 0;
  NX_CUDA(cudaMemcpyAsync(&nnz, cnt.p, 4, cudaMemcpyDeviceToHost, s));
  NX_CUDA(cudaStreamSynchronize(s));
  NX_TRY(sv.alloc(std::max<size_t>(nnz, 1) * 4));
  NX_TRY(sb.alloc(std::max<size_t>(nnz, 1) * 4));
  NX_TRY(sval.alloc(std::max<size_t>(nnz, 1) * 4));
  NX_CUDA(cudaMemsetAsync(cnt.p, 0, 4, s));
  k_seed_list<<<grid_of((uint64_t)n * B), 256, 0, s>>>(t_dev, B, n, map, cnt.as<uint32_t>(), nnz,
                                                       sv.as<uint32_t>(), sb.as<uint32_t>(),
                                                       sval.as<float>());
  NX_LAUNCH_CHECK();
  // r0 = t (stored only when no iteration runs), c0 = t / outdeg, Dm0
  NX_CUDA(cudaMemsetAsync(cv[0].p, 0, vb, s));
  if (iters == 0) NX_CUDA(cudaMemsetAsync(rv.p, 0, vb, s));
  k_seed_apply<<<grid_of(nnz), 256, 0, s>>>(nnz, sv.as<uint32_t>(), sb.as<uint32_t>(),
                                            sval.as<float>(), BP, g->outdeg.as<uint32_t>(), alpha,
                                            1, nullptr, dm.as<double>(), cv[0].as<float>(),
                                            iters == 0 ? rv.as<float>() : nullptr);
  NX_LAUNCH_CHECK();
  BArgs a{};
  a.ew = g->fwd.ew.as<uint32_t>();
  a.piece_off = g->fwd.piece_off.as<uint64_t>();
  a.tile_start = g->geo.tile_start.as<uint32_t>();
  a.col_tb = g->geo.col_tb.as<uint32_t>();
  a.outdeg = g->outdeg.as<uint32_t>();
  a.P = P;
  a.L = L;
  a.lb = g->geo.lb;
  a.n = n;
  a.items = d_items.as<BItem>();
  a.split = d_split.as<float>();
  a.ticket = d_ticket.as<uint32_t>();
  a.alpha = alpha;
  a.sub = kSub;
  a.r_out = rv.as<float>();
  const size_t smem = (size_t)kSub * BP * 4 + (size_t)(2 * P + 1) * 8;
  void (*kern)(const BArgs) = batch_kernel(BP, g->ppr_rows);
  if (!kern) return invalid("nx_run_ppr_batch: unsupported rows in flight");
  if (smem > 48 * 1024)
    NX_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  NX_TRY(prefer_l1(reinterpret_cast<const void*>(kern), kBT, smem));
  EventPair ev;
  NX_TRY(ev.create());
  NX_CUDA(cudaEventRecord(ev.e0, s));
  int cur = 0;
  for (uint32_t itn = 0; itn < iters; ++itn) {
    const bool last = itn + 1 == iters;
    a.write_r = last ? 1 : 0;
    a.c_in = cv[cur].as<float>();
    a.c_out = cv[1 - cur].as<float>();
    a.dm_in = dm.as<double>() + cur * BP;
    a.dm_out = dm.as<double>() + (1 - cur) * BP;
    NX_CUDA(cudaMemsetAsync(dm.as<double>() + (1 - cur) * BP, 0, BP * 8, s));
    kern<<<(unsigned)items.size(), kBT, smem, s>>>(a);
    NX_LAUNCH_CHECK();
    k_seed_apply<<<grid_of(nnz), 256, 0, s>>>(nnz, sv.as<uint32_t>(), sb.as<uint32_t>(),
                                              sval.as<float>(), BP, g->outdeg.as<uint32_t>(),
                                              alpha, 0, a.dm_in, a.dm_out, cv[1 - cur].as<float>(),
                                              last ? rv.as<float>() : nullptr);
    NX_LAUNCH_CHECK();
    cur = 1 - cur;
  }
  NX_CUDA(cudaEventRecord(ev.e1, s));
  float ms = 0.f;
  NX_TRY(ev.elapsed(&ms));
  // output [n][B]
  if (dev_ptrs) {
    k_ppr_out<<<grid_of((uint64_t)n * B), 256, 0, s>>>(rv.as<float>(), B, BP, n, map, ranks);
    NX_LAUNCH_CHECK();
  } else {
    DevBuf o;
    NX_TRY(o.alloc((size_t)n * B * 4));
    k_ppr_out<<<grid_of((uint64_t)n * B), 256, 0, s>>>(rv.as<float>(), B, BP, n, map,
                                                       o.as<float>());
    NX_LAUNCH_CHECK();
    NX_CUDA(cudaMemcpyAsync(ranks, o.p, (size_t)n * B * 4, cudaMemcpyDeviceToHost, s));
  }
  NX_CUDA(cudaStreamSynchronize(s));
  if (st) {
    memset(st, 0, sizeof *st);
    st->iters_done = iters;
    st->Q = P;
    st->ms = ms;
    st->edges_swept = g->m * iters;
    // per iteration: edge words, one read of every source row, one write of c
    st->bytes_model = (uint64_t)iters * (4 * g->m + (uint64_t)n * BP * 4 * 2);
    st->launches = 2 * iters;
  }
  return NX_OK;
}

}  // namespace
}  // namespace nx

extern "C" nx_status nx_run_ppr_batch(nx_graph* g, const float* teleport, uint32_t B,
                                      uint32_t iters, float alpha, float* ranks,
                                      int32_t ptrs_are_device, nx_run_stats* stats) {
  if (!g || !teleport || !ranks) return nx::invalid("nx_run_ppr_batch: NULL argument");
  if (B == 0 || B > 64) return nx::invalid("nx_run_ppr_batch: B must be in [1, 64]");
  if (!(alpha >= 0.f && alpha < 1.f)) return nx::invalid("nx_run_ppr_batch: alpha must be in [0, 1)");
  if (g->geo.P > 1024) return nx::invalid("nx_run_ppr_batch: P too large");
  nx::TraceRange trace("nx_run_ppr_batch");
  NX_TRY(nx::ensure_resident(g));
  return nx::ppr_batch_impl(g, teleport, B, iters, alpha, ranks, ptrs_are_device, stats);
}
