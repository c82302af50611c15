// DSSS builder (Section III-A "Sharding"): edge list -> P x P destination-sorted
// sub-shards, entirely on the device.
//
// Layout produced (per DSSS):
//   * Vertices: P equal intervals of L = ceil(n/P) (the paper's equal-size
//     partitioning). Each interval is cut further into destination tiles of at
//     most tile_max vertices and about E_tile in-edges (a tile never crosses an
//     interval). Tiles are the unit a thread block owns in a sweep.
//   * Edges: sorted by (j, i, dst, src) — shard j (destination interval), then
//     sub-shard SS_ij (source interval i), then destination, then source
//     (Section III-A: edges sorted by destination, ties by source).
//     The run of SS_ij that falls in tile t is the "piece" (i, t).
//   * Each edge is one 32-bit word ((dst - tile_start) << lb) | src_local, with
//     src_local = src - i*L < 2^lb. This is the paper's "compressed sparse
//     format": destination and source high bits are implied by the position.
//   * Hub index (Table I, H_ij): one entry per distinct destination of each
//     sub-shard, in order, with its destination offset inside its tile.
//
// Steps: ids checked and out-degrees counted as the edges arrive; with
// NX_RELABEL the degree order of the vertices; keys (j*P + i, dst - jL,
// src - iL) radix-sorted (host edges: chunk by chunk as the chunks land, the
// sorted chunks merged by merge path); in-degrees counted from the sorted
// forward keys and the tiles cut by them; one pass writes the edge words, run
// heads and piece starts; the hub index follows from the run heads.
#include <algorithm>
#include <cstdio>

#include "nx_internal.cuh"

namespace nx {
namespace {

// Most vertices in a destination tile unless the build flags choose another
// cap (NX_TILE_CAP_LOG2): the block's accumulators (hi + lo floats) take 8 B
// per vertex of shared memory.
constexpr uint32_t kTileMaxCap = 2048;

// Degree histogram of ids a[0..m) into h[0..n) (h nullable: the check only);
// ids >= n are counted nowhere and raise *bad (the build reads it before
// anything indexes by an id).
__global__ void k_check_count(const uint32_t* __restrict__ a, uint64_t m, uint32_t n,
                              uint32_t* __restrict__ h, uint32_t* __restrict__ bad) {
  uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  bool any = false;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    const uint32_t v = a[e];
    if (v >= n) any = true;
    else if (h) atomicAdd(&h[v], 1u);
  }
  if (__any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}

__global__ void k_deg_sum(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b,
                          uint32_t n, uint64_t* __restrict__ out) {
  uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    out[v] = (uint64_t)a[v] + (b ? b[v] : 0u);
}

// A vertex starts a tile at an interval start, every tile_max vertices inside
// an interval, and where the in-edge prefix crosses a multiple of E_tile.
__global__ void k_tile_flags(const uint64_t* __restrict__ pre, uint32_t n, uint32_t L,
                             uint32_t tile_max, uint64_t E, uint32_t* __restrict__ flag) {
  uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    uint32_t p = (uint32_t)(v % L);
    bool s = (p == 0) || (p % tile_max == 0) || (pre[v] / E != pre[v - 1] / E);
    flag[v] = s ? 1u : 0u;
  }
}

__global__ void k_tile_ids(const uint32_t* __restrict__ flag, uint32_t* __restrict__ tid,
                           uint32_t n, uint32_t* __restrict__ tile_start) {
  uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    uint32_t t = tid[v] + flag[v] - 1;  // tid holds the exclusive scan of flags
    tid[v] = t;
    if (flag[v]) tile_start[t] = (uint32_t)v;
  }
}

// vt[v] = tile of v << 32 | v's offset in its tile.
__global__ void k_vertex_tiles(const uint32_t* __restrict__ tid, const uint32_t* __restrict__ tile_start,
                               uint32_t n, uint64_t* __restrict__ vt) {
  uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const uint32_t t = tid[v];
    vt[v] = ((uint64_t)t << 32) | (uint32_t)(v - tile_start[t]);
  }
}

struct KeyCodec {
  uint32_t P, L, lb;
  __host__ __device__ uint64_t encode(uint32_t s, uint32_t d) const {
    uint32_t i = s / L, j = d / L;
    return ((uint64_t)(j * P + i) << (2 * lb)) | ((uint64_t)(d - j * L) << lb) | (s - i * L);
  }
  __device__ void decode(uint64_t k, uint32_t* i, uint32_t* j, uint32_t* d, uint32_t* sl) const {
    uint32_t sub = (uint32_t)(k >> (2 * lb));
    uint64_t mask = lb ? ((1ull << lb) - 1) : 0ull;
    *sl = (uint32_t)(k & mask);
    uint32_t dl = (uint32_t)((k >> lb) & mask);
    *j = sub / P;
    *i = sub - *j * P;
    *d = *j * L + dl;
  }
};

// rename (nullable): internal id of each input id, applied on the fly. Ids
// >= n read no map entry and raise *bad (nullable) instead; the build rejects
// them before the keys are used.
__global__ void k_make_keys(const uint32_t* __restrict__ s, const uint32_t* __restrict__ d,
                            uint64_t m, uint32_t n, KeyCodec kc, const uint32_t* __restrict__ rename,
                            uint64_t* __restrict__ keys, uint32_t* __restrict__ idx,
                            uint32_t* __restrict__ bad) {
  uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  bool any = false;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    uint32_t a = s[e], b = d[e];
    any |= (a >= n) || (b >= n);
    a = a < n ? a : 0u;
    b = b < n ? b : 0u;
    keys[e] = rename ? kc.encode(rename[a], rename[b]) : kc.encode(a, b);
    if (idx) idx[e] = (uint32_t)e;
  }
  if (bad && __any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}

// In-degrees from sorted keys: each group of 32 keys adds the length of each
// of its runs of equal destination to indeg (a destination's edges form one
// run per sub-shard, cut at group boundaries).
__global__ void k_indeg_from_keys(const uint64_t* __restrict__ keys, uint64_t m, KeyCodec kc,
                                  uint32_t* __restrict__ indeg) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t ng = (m + 31) / 32;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t g = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < ng; g += nwarps) {
    const uint64_t e = g * 32 + lane;
    const bool valid = e < m;
    uint32_t i = 0, j = 0, dv = 0, sl = 0;
    if (valid) kc.decode(keys[e], &i, &j, &dv, &sl);
    const uint32_t key = valid ? (j * kc.P + i) : 0xFFFFFFFFu;  // sub-shard: runs never span two
    const uint32_t up_d = __shfl_up_sync(0xffffffffu, dv, 1), up_k = __shfl_up_sync(0xffffffffu, key, 1);
    const uint32_t dn_d = __shfl_down_sync(0xffffffffu, dv, 1), dn_k = __shfl_down_sync(0xffffffffu, key, 1);
    const bool head = valid && (lane == 0 || up_d != dv || up_k != key);
    const bool tail = valid && (lane == 31 || dn_d != dv || dn_k != key || e + 1 == m);
    const uint32_t tails = __ballot_sync(0xffffffffu, tail);
    if (head) {
      const uint32_t last = lane + __ffs(tails >> lane) - 1;  // this run's tail lane
      atomicAdd(&indeg[dv], last - lane + 1);
    }
  }
}

// Piece and destination of a key. vt[v] = (tile of v) << 32 | (v's offset in
// its tile), so a key costs one lookup that depends on it.
struct PieceMap {
  KeyCodec kc;
  const uint64_t* vt;      // [n]
  const uint32_t* col_tb;  // [P+1]
  struct Dec {
    uint32_t i, j, d, sl;
  };
  __device__ Dec decode(uint64_t key) const {
    Dec x;
    kc.decode(key, &x.i, &x.j, &x.d, &x.sl);
    return x;
  }
  // piece of a decoded key whose vt entry is `v`; *off: offset in the tile
  __device__ uint64_t piece(const Dec& x, uint64_t v, uint32_t* off) const {
    const uint32_t t = (uint32_t)(v >> 32);
    const uint32_t tb = col_tb[x.j], nt = col_tb[x.j + 1] - tb;
    *off = (uint32_t)v;
    return piece_index(kc.P, tb, nt, x.i, t);
  }
  __device__ uint64_t piece(uint64_t key, uint32_t* d) const {
    const Dec x = decode(key);
    uint32_t off;
    *d = x.d;
    return piece(x, vt[x.d], &off);
  }
};

// Edge words, run-head bits and piece starts. A run is the edges of one
// (piece, destination); its first edge is its head, and each head owns one hub
// entry. Edges go in groups of 32 (w = e / 32): hbits[w] holds their head bits
// and hcnt[w] the number of heads; pieces (pc(e-1), pc(e)] start at edge e.
// Each warp takes kWordGroups consecutive groups per iteration and issues
// their key loads, then their vertex lookups, together: the key -> vertex
// chain is latency-bound, so the groups overlap their waits.
constexpr int kWordGroups = 4;
__global__ void k_words(const uint64_t* __restrict__ keys, uint64_t m, PieceMap pm,
                        uint32_t* __restrict__ ew, uint32_t* __restrict__ hbits,
                        uint32_t* __restrict__ hcnt, uint64_t* __restrict__ piece_off) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t nw = (m + 31) / 32;
  const uint64_t ng = (nw + kWordGroups - 1) / kWordGroups;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t g = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < ng; g += nwarps) {
    const uint64_t e0 = g * kWordGroups * 32;
    uint64_t key[kWordGroups];
#pragma unroll
    for (int q = 0; q < kWordGroups; ++q) {
      const uint64_t e = e0 + q * 32 + lane;
      key[q] = e < m ? keys[e] : 0ull;
    }
    // the edge before the first group belongs to the previous iteration's range
    const uint64_t kprev = (lane == 0 && e0 > 0) ? keys[e0 - 1] : 0ull;
    PieceMap::Dec x[kWordGroups];
    uint64_t v[kWordGroups];
#pragma unroll
    for (int q = 0; q < kWordGroups; ++q) {
      x[q] = pm.decode(key[q]);
      v[q] = (e0 + q * 32 + lane < m) ? pm.vt[x[q].d] : 0ull;
    }
    const PieceMap::Dec xp = pm.decode(kprev);
    const uint64_t vp = (lane == 0 && e0 > 0) ? pm.vt[xp.d] : 0ull;
    uint32_t offp;
    uint64_t pc_last = pm.piece(xp, vp, &offp);  // the previous edge's piece (lane 0)
    uint32_t d_last = xp.d;
#pragma unroll
    for (int q = 0; q < kWordGroups; ++q) {
      const uint64_t w = g * kWordGroups + q;
      const uint64_t e = e0 + q * 32 + lane;
      const bool valid = e < m;
      uint32_t off = 0;
      uint64_t pc = 0;
      if (valid) {
        pc = pm.piece(x[q], v[q], &off);
        ew[e] = (off << pm.kc.lb) | x[q].sl;
      }
      const uint32_t d = valid ? x[q].d : 0u;
      uint64_t pc0 = __shfl_up_sync(0xffffffffu, pc, 1);
      uint32_t d0 = __shfl_up_sync(0xffffffffu, d, 1);
      if (lane == 0) {
        pc0 = pc_last;
        d0 = d_last;
      }
      pc_last = __shfl_sync(0xffffffffu, pc, 31);  // lane 31 precedes the next group's lane 0
      d_last = __shfl_sync(0xffffffffu, d, 31);
      const bool head = valid && (e == 0 || pc0 != pc || d0 != d);
      const uint32_t bits = __ballot_sync(0xffffffffu, head);
      if (lane == 0 && w < nw) {
        hbits[w] = bits;
        hcnt[w] = __popc(bits);
      }
      if (valid) {
        const uint64_t k0 = (e == 0) ? 0 : pc0 + 1;
        for (uint64_t k = k0; k <= pc; ++k) piece_off[k] = e;
      }
    }
  }
}

// Pieces after the last edge's start at m.
__global__ void k_piece_tail(const uint64_t* __restrict__ keys, uint64_t m, PieceMap pm,
                             uint64_t* __restrict__ piece_off, uint64_t npieces) {
  uint64_t k0 = 0;
  if (m) {
    uint32_t d;
    k0 = pm.piece(keys[m - 1], &d) + 1;
  }
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = k0 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= npieces; k += stride)
    piece_off[k] = m;
}

// Hub entry of edge e: the heads before it (hpre = exclusive scan of hcnt).
__device__ __forceinline__ uint64_t hub_index(const uint32_t* hbits, const uint32_t* hpre, uint64_t e) {
  const uint64_t w = e >> 5;
  const uint32_t lt = (1u << (e & 31)) - 1u;
  return (uint64_t)hpre[w] + __popc(hbits[w] & lt);
}

// Destination offset (within its tile) of every hub entry.
__global__ void k_hub_dst(const uint32_t* __restrict__ ew, const uint32_t* __restrict__ hbits,
                          const uint32_t* __restrict__ hpre, uint64_t m, uint32_t lb,
                          uint16_t* __restrict__ hub_dst) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride)
    if ((hbits[e >> 5] >> (e & 31)) & 1u) hub_dst[hub_index(hbits, hpre, e)] = (uint16_t)(ew[e] >> lb);
}

// First hub entry of every piece (D for pieces that start at m).
__global__ void k_hub_off(const uint64_t* __restrict__ piece_off, const uint32_t* __restrict__ hbits,
                          const uint32_t* __restrict__ hpre, uint64_t m, uint64_t D,
                          uint64_t* __restrict__ hub_off, uint64_t npieces) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= npieces; k += stride) {
    const uint64_t e = piece_off[k];
    hub_off[k] = e >= m ? D : hub_index(hbits, hpre, e);
  }
}

__global__ void k_wsum(const uint32_t* __restrict__ s, const float* __restrict__ w, uint64_t m,
                       double* __restrict__ W) {
  uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride)
    atomicAdd(&W[s[e]], (double)w[e]);
}

__global__ void k_wnorm(const uint32_t* __restrict__ s, const float* __restrict__ w, uint64_t m,
                        const double* __restrict__ W, float* __restrict__ wn) {
  uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride)
    wn[e] = (float)((double)w[e] / W[s[e]]);
}

__global__ void k_wsum_f(const double* __restrict__ W, uint32_t n, float* __restrict__ Wf) {
  uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    Wf[v] = (float)W[v];
}

__global__ void k_gather_f(const float* __restrict__ src, const uint32_t* __restrict__ idx,
                           uint64_t m, float* __restrict__ out) {
  uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride)
    out[e] = src[idx[e]];
}

unsigned grid_for(uint64_t work, unsigned threads = 256) {
  uint64_t b = ceil_div(work ? work : 1, threads);
  uint64_t cap = (uint64_t)num_sms() * 16;
  return (unsigned)std::min<uint64_t>(b, cap);
}

// DSSS keys of (s, d) over the geometry's P, L, lb, sorted; with want_idx,
// idx[k] is the input position of the k-th key. rename (nullable): applied to
// s and d while the keys are made.
nx_status sort_keys(const uint32_t* s, const uint32_t* d, uint64_t m, const Geometry& geo,
                    const uint32_t* rename, bool want_idx, DevBuf& keys, DevBuf& idx) {
  const KeyCodec kc{geo.P, geo.L, geo.lb};
  const uint32_t key_bits = bits_for((uint64_t)geo.P * geo.P) + 2 * geo.lb;
  if (key_bits > 64) return invalid("DSSS key does not fit 64 bits (n too large for P)");
  NX_TRY(keys.alloc(std::max<uint64_t>(m, 1) * sizeof(uint64_t)));
  if (want_idx) NX_TRY(idx.alloc(std::max<uint64_t>(m, 1) * sizeof(uint32_t)));
  if (m) {
    k_make_keys<<<grid_for(m), 256, 0, stream()>>>(s, d, m, geo.n, kc, rename, keys.as<uint64_t>(),
                                                   want_idx ? idx.as<uint32_t>() : nullptr, nullptr);
    NX_LAUNCH_CHECK();
    NX_TRY(radix_sort_u64(keys, want_idx ? &idx : nullptr, m, key_bits));
  }
  return NX_OK;
}

// Builds one DSSS from (s, d) over the geometry; wn (nullable) are the
// normalised weights in input order.
// rename (nullable): applied to s and d while the keys are made.
// sorted / sorted_idx (nullable): the keys of (s, d) already sorted, and with
// weights their input positions (both taken over).
nx_status build_one(const uint32_t* s, const uint32_t* d, uint64_t m, const Geometry& geo,
                    const uint64_t* vt, const float* wn, Dsss& out,
                    const uint32_t* rename = nullptr, DevBuf* sorted = nullptr,
                    DevBuf* sorted_idx = nullptr) {
  out.m = m;
  const uint64_t npieces = (uint64_t)geo.P * geo.ntiles;
  KeyCodec kc{geo.P, geo.L, geo.lb};
  DevBuf keys, idx;
  if (sorted && sorted->p) {
    if (wn && !(sorted_idx && sorted_idx->p)) return invalid("build_one: presorted keys without positions");
    keys = std::move(*sorted);
    if (wn) idx = std::move(*sorted_idx);
  } else {
    NX_TRY(sort_keys(s, d, m, geo, rename, wn != nullptr, keys, idx));
  }
  const uint64_t mpad = round_up(m, kEdgeAlign) + kEdgeAlign;
  NX_TRY(out.ew.alloc(mpad * sizeof(uint32_t)));
  NX_CUDA(cudaMemsetAsync(out.ew.p, 0, mpad * sizeof(uint32_t), stream()));
  NX_TRY(out.piece_off.alloc((npieces + 1) * sizeof(uint64_t)));
  NX_TRY(out.hub_off.alloc((npieces + 1) * sizeof(uint64_t)));
  PieceMap pm{kc, vt, geo.col_tb.as<uint32_t>()};
  const uint64_t nw = (m + 31) / 32;
  DevBuf hbits, hcnt, dtot;
  NX_TRY(hbits.alloc(std::max<uint64_t>(nw, 1) * sizeof(uint32_t)));
  NX_TRY(hcnt.alloc(std::max<uint64_t>(nw, 1) * sizeof(uint32_t)));
  NX_TRY(dtot.alloc(sizeof(uint32_t)));
  if (m) {
    k_words<<<grid_for(m), 256, 0, stream()>>>(keys.as<uint64_t>(), m, pm, out.ew.as<uint32_t>(),
                                               hbits.as<uint32_t>(), hcnt.as<uint32_t>(),
                                               out.piece_off.as<uint64_t>());
    NX_LAUNCH_CHECK();
    NX_TRY(exclusive_scan_u32(hcnt.as<uint32_t>(), hcnt.as<uint32_t>(), nw, dtot.as<uint32_t>()));
    uint32_t D32 = 0;
    NX_CUDA(cudaMemcpyAsync(&D32, dtot.p, sizeof D32, cudaMemcpyDeviceToHost, stream()));
    NX_CUDA(cudaStreamSynchronize(stream()));
    out.D = D32;
  } else {
    out.D = 0;
  }
  k_piece_tail<<<grid_for(npieces + 1), 256, 0, stream()>>>(keys.as<uint64_t>(), m, pm,
                                                           out.piece_off.as<uint64_t>(), npieces);
  NX_LAUNCH_CHECK();
  NX_TRY(out.hub_dst.alloc(std::max<uint64_t>(out.D, 1) * sizeof(uint16_t)));
  if (m) {
    k_hub_dst<<<grid_for(m), 256, 0, stream()>>>(out.ew.as<uint32_t>(), hbits.as<uint32_t>(),
                                                 hcnt.as<uint32_t>(), m, geo.lb,
                                                 out.hub_dst.as<uint16_t>());
    NX_LAUNCH_CHECK();
  }
  k_hub_off<<<grid_for(npieces + 1), 256, 0, stream()>>>(
      out.piece_off.as<uint64_t>(), hbits.as<uint32_t>(), hcnt.as<uint32_t>(), m, out.D,
      out.hub_off.as<uint64_t>(), npieces);
  NX_LAUNCH_CHECK();
  if (wn) {
    NX_TRY(out.wt.alloc(mpad * sizeof(float)));
    NX_CUDA(cudaMemsetAsync(out.wt.p, 0, mpad * sizeof(float), stream()));
    if (m) {
      k_gather_f<<<grid_for(m), 256, 0, stream()>>>(wn, idx.as<uint32_t>(), m, out.wt.as<float>());
      NX_LAUNCH_CHECK();
    }
  }
  NX_TRY(out.h_piece_off.resize(npieces + 1));
  NX_CUDA(cudaMemcpyAsync(out.h_piece_off.data(), out.piece_off.p, (npieces + 1) * sizeof(uint64_t),
                          cudaMemcpyDeviceToHost, stream()));
  NX_CUDA(cudaStreamSynchronize(stream()));
  out.words = mpad;
  out.dev_words = mpad;
  return NX_OK;
}

// vt: the tile of every vertex and its offset in the tile (k_vertex_tiles).
nx_status build_geometry(nx_graph* g, const uint32_t* deg_a, const uint32_t* deg_b,
                         uint64_t m_bal, uint32_t edges_log2, DevBuf& vt) {
  Geometry& geo = g->geo;
  const uint32_t n = geo.n;
  // E_tile: about m / (8 x SMs), within [2^14, 2^20]. The vertex cap bounds
  // most tiles; E_tile cuts the heavy ones (and gives small graphs enough
  // tiles), and the planner splits what is still heavy over several blocks.
  // The upper bound was 2^16: lifting it made the R-MAT scale-26 PageRank
  // sweep (P = 64, E_tile 2^20) 4% faster (5.58 vs 5.81 ms) and DPU sweeps
  // 15-30% faster at scales 22-24; the staged MPU columns want smaller tiles
  // (scale 22, P = 16, Q = 8: 15.5 / 16.2 / 20.1 ms at 2^16 / 2^17 / 2^18),
  // which m / (8 x SMs) still gives there (2^17 with the transpose).
  uint64_t E = m_bal / ((uint64_t)num_sms() * 8);
  E = std::max<uint64_t>(16384, std::min<uint64_t>(E, 1ull << 20));
  if (edges_log2) E = 1ull << edges_log2;
  DevBuf pre, flag, tile_of;
  NX_TRY(pre.alloc((uint64_t)n * sizeof(uint64_t)));
  NX_TRY(flag.alloc((uint64_t)n * sizeof(uint32_t)));
  NX_TRY(tile_of.alloc((uint64_t)n * sizeof(uint32_t)));
  k_deg_sum<<<grid_for(n), 256, 0, stream()>>>(deg_a, deg_b, n, pre.as<uint64_t>());
  NX_LAUNCH_CHECK();
  NX_TRY(exclusive_scan_u64(pre.as<uint64_t>(), pre.as<uint64_t>(), n, nullptr));
  k_tile_flags<<<grid_for(n), 256, 0, stream()>>>(pre.as<uint64_t>(), n, geo.L, geo.tile_max, E,
                                                  flag.as<uint32_t>());
  NX_LAUNCH_CHECK();
  DevBuf tot;
  NX_TRY(tot.alloc(sizeof(uint32_t)));
  NX_TRY(exclusive_scan_u32(flag.as<uint32_t>(), tile_of.as<uint32_t>(), n, tot.as<uint32_t>()));
  uint32_t ntiles = 0;
  NX_CUDA(cudaMemcpyAsync(&ntiles, tot.p, sizeof ntiles, cudaMemcpyDeviceToHost, stream()));
  NX_CUDA(cudaStreamSynchronize(stream()));
  geo.ntiles = ntiles;
  NX_TRY(geo.tile_start.alloc(((uint64_t)ntiles + 1) * sizeof(uint32_t)));
  k_tile_ids<<<grid_for(n), 256, 0, stream()>>>(flag.as<uint32_t>(), tile_of.as<uint32_t>(), n,
                                                geo.tile_start.as<uint32_t>());
  NX_LAUNCH_CHECK();
  NX_CUDA(cudaMemcpyAsync(geo.tile_start.as<uint32_t>() + ntiles, &geo.n, sizeof(uint32_t),
                          cudaMemcpyHostToDevice, stream()));
  NX_TRY(vt.alloc((uint64_t)n * sizeof(uint64_t)));
  k_vertex_tiles<<<grid_for(n), 256, 0, stream()>>>(tile_of.as<uint32_t>(), geo.tile_start.as<uint32_t>(),
                                                    n, vt.as<uint64_t>());
  NX_LAUNCH_CHECK();
  geo.h_tile_start.resize((size_t)ntiles + 1);
  NX_CUDA(cudaMemcpyAsync(geo.h_tile_start.data(), geo.tile_start.p,
                          ((uint64_t)ntiles + 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                          stream()));
  NX_CUDA(cudaStreamSynchronize(stream()));
  // first tile of every column (empty trailing intervals get ntiles)
  geo.h_col_tb.assign((size_t)geo.P + 1, ntiles);
  {
    uint32_t t = 0;
    for (uint32_t j = 0; j < geo.P; ++j) {
      uint64_t v0 = (uint64_t)j * geo.L;
      while (t < ntiles && geo.h_tile_start[t] < v0) ++t;
      geo.h_col_tb[j] = t;
    }
  }
  NX_TRY(geo.col_tb.alloc(((size_t)geo.P + 1) * sizeof(uint32_t)));
  NX_CUDA(cudaMemcpyAsync(geo.col_tb.p, geo.h_col_tb.data(), ((size_t)geo.P + 1) * sizeof(uint32_t),
                          cudaMemcpyHostToDevice, stream()));
  NX_CUDA(cudaStreamSynchronize(stream()));
  return NX_OK;
}

// Side stream and events of a chunked host-to-device upload.
struct Upload {
  cudaStream_t side = nullptr;
  cudaEvent_t ready = nullptr;
  std::vector<cudaEvent_t> copied;
  ~Upload() {
    // copies still in flight (an early error return) must land before the
    // buffers they write are freed on the main stream
    if (side) cudaStreamSynchronize(side);
    for (cudaEvent_t e : copied)
      if (e) cudaEventDestroy(e);
    if (ready) cudaEventDestroy(ready);
    if (side) cudaStreamDestroy(side);
  }
  nx_status init(int chunks) {
    NX_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    NX_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    copied.assign(chunks, nullptr);
    for (auto& e : copied) NX_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return NX_OK;
  }
};

// Host edges without weights: the src chunks cross the link first, then the
// dst chunks, on a side stream. The out-degrees are complete once src has
// landed, so NX_RELABEL's order is computed while dst arrives; each dst
// chunk's keys (forward, and transpose when asked) are made in the new ids and
// sorted as it lands, and only the merge of the sorted chunks is left once the
// last chunk is in (pairs of sorted chunks are merged while later ones
// arrive). The keys are the same as build_one's, so is their order.
nx_status upload_and_sort(nx_graph* g, const uint32_t* src, const uint32_t* dst, uint64_t m,
                          uint32_t n, uint32_t P, bool relabel, bool want_t, uint32_t* hs,
                          uint32_t* hd, uint32_t* bad, DevBuf* sorted) {
  const uint32_t L = (uint32_t)ceil_div(n, P), lb = bits_for(L);
  const KeyCodec kc{P, L, lb};
  const uint32_t key_bits = bits_for((uint64_t)P * P) + 2 * lb;
  if (key_bits > 64) return invalid("DSSS key does not fit 64 bits (n too large for P)");
  constexpr uint64_t kChunks = 8;
  const uint64_t chunk = round_up(ceil_div(m, kChunks), 1024);
  const int nc = (int)ceil_div(m, chunk);
  Upload up;
  NX_TRY(up.init(2 * nc));
  NX_CUDA(cudaEventRecord(up.ready, stream()));  // the buffers exist in stream order
  NX_CUDA(cudaStreamWaitEvent(up.side, up.ready, 0));
  auto range = [&](int c, uint64_t* e0, uint64_t* len) {
    *e0 = (uint64_t)c * chunk;
    *len = std::min<uint64_t>(chunk, m - *e0);
  };
  // Copies from pinned memory are queued at once (the host returns at once,
  // the link never waits for the relabel step); from pageable memory the host
  // thread stages each copy itself, so each chunk's copy is issued just before
  // its work, which then runs while the host stages the next chunk.
  auto pinned = [](const void* p) {
    cudaPointerAttributes at{};
    return cudaPointerGetAttributes(&at, p) == cudaSuccess && at.type == cudaMemoryTypeHost;
  };
  const bool queue_all = pinned(src) && pinned(dst);
  cudaGetLastError();  // a failed attribute query leaves no error behind
  auto copy = [&](int c, bool second) -> nx_status {
    uint64_t a0, n0;
    range(c, &a0, &n0);
    NX_CUDA(cudaMemcpyAsync((second ? hd : hs) + a0, (second ? dst : src) + a0, n0 * 4,
                            cudaMemcpyHostToDevice, up.side));
    NX_CUDA(cudaEventRecord(up.copied[(second ? nc : 0) + c], up.side));
    return NX_OK;
  };
  if (queue_all)
    for (int c = 0; c < 2 * nc; ++c) NX_TRY(copy(c % nc, c >= nc));
  uint64_t e0, len;
  for (int c = 0; c < nc; ++c) {
    range(c, &e0, &len);
    if (!queue_all) NX_TRY(copy(c, false));
    NX_CUDA(cudaStreamWaitEvent(stream(), up.copied[c], 0));
    k_check_count<<<grid_for(len), 256, 0, stream()>>>(hs + e0, len, n, g->outdeg.as<uint32_t>(), bad);
    NX_LAUNCH_CHECK();
  }
  if (relabel) NX_TRY(relabel_edges(g, nullptr, nullptr, 0, nullptr, nullptr, g->outdeg.as<uint32_t>()));
  const uint32_t* ren = relabel ? g->new_of_old.as<uint32_t>() : nullptr;
  const int nk = want_t ? 2 : 1;
  for (int k = 0; k < nk; ++k) NX_TRY(sorted[k].alloc(m * sizeof(uint64_t)));
  DevBuf scratch, counts;
  NX_TRY(scratch.alloc(chunk * sizeof(uint64_t)));
  NX_TRY(counts.alloc(radix_sort_count_words(chunk) * sizeof(uint32_t)));
  RunMerger mg[2];
  for (int k = 0; k < nk; ++k) NX_TRY(mg[k].init(sorted[k], m));
  for (int c = 0; c < nc; ++c) {
    range(c, &e0, &len);
    if (!queue_all) NX_TRY(copy(c, true));
    NX_CUDA(cudaStreamWaitEvent(stream(), up.copied[nc + c], 0));
    for (int k = 0; k < nk; ++k) {
      uint64_t* kk = sorted[k].as<uint64_t>() + e0;
      k_make_keys<<<grid_for(len), 256, 0, stream()>>>(k ? hd + e0 : hs + e0, k ? hs + e0 : hd + e0,
                                                       len, n, kc, ren, kk, nullptr, k ? nullptr : bad);
      NX_LAUNCH_CHECK();
      bool in_b = false;
      NX_TRY(radix_sort_u64_raw(kk, scratch.as<uint64_t>(), nullptr, nullptr, counts.as<uint32_t>(),
                                len, key_bits, &in_b));
      if (in_b)
        NX_CUDA(cudaMemcpyAsync(kk, scratch.p, len * sizeof(uint64_t), cudaMemcpyDeviceToDevice, stream()));
      NX_TRY(mg[k].push(e0, e0 + len));
    }
  }
  for (int k = 0; k < nk; ++k) NX_TRY(mg[k].finish());  // synchronises
  return NX_OK;
}

nx_status build_impl(const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n, uint32_t P,
                     uint32_t flags, const float* w, nx_graph* g) {
  const bool on_dev = flags & NX_DEV_PTRS;
  const bool want_t = flags & NX_WITH_TRANSPOSE;
  const bool want_w = flags & NX_WITH_WEIGHTS;
  EventPair ev;
  NX_TRY(ev.create());
  NX_CUDA(cudaEventRecord(ev.e0, stream()));
  g->geo.n = n;  // relabel_edges reads it, during the upload of host edges too
  // Degrees of the input ids are counted as the edges arrive (overlapping the
  // upload of host edges); NX_RELABEL orders the vertices by them and then
  // permutes them to the new ids (a renamed vertex keeps its degrees).
  DevBuf indeg, bad, od_new;
  // The value and contribution arrays every run gathers from, and the
  // out-degrees in new ids, are allocated before the build's temporaries
  // (about 40 GB at R-MAT scale 26) pass through the device pool: carved out
  // of the memory those leave behind, the same arrays made the scale-26
  // PageRank sweep 1.5% slower (6.37 vs 6.28 ms, measured on one GPU).
  for (int k = 0; k < 2; ++k) {
    NX_TRY(g->val[k].alloc((uint64_t)n * 4));
    NX_TRY(g->aux[k].alloc((uint64_t)n * 4));
  }
  if (flags & NX_RELABEL) NX_TRY(od_new.alloc((uint64_t)n * 4));
  NX_TRY(g->outdeg.alloc((uint64_t)n * 4));
  NX_TRY(indeg.alloc((uint64_t)n * 4));
  NX_TRY(bad.alloc(4));
  NX_CUDA(cudaMemsetAsync(g->outdeg.p, 0, (uint64_t)n * 4, stream()));
  NX_CUDA(cudaMemsetAsync(indeg.p, 0, (uint64_t)n * 4, stream()));
  NX_CUDA(cudaMemsetAsync(bad.p, 0, 4, stream()));
  // per range of edges: ids < n, and the degree histograms
  // per range of edges: ids < n and the out-degrees (the in-degrees are
  // counted from the sorted forward keys, in the ids the DSSS uses)
  auto scan_edges = [&](const uint32_t* s0, const uint32_t* d0, uint64_t len) -> nx_status {
    k_check_count<<<grid_for(len), 256, 0, stream()>>>(s0, len, n, g->outdeg.as<uint32_t>(),
                                                       bad.as<uint32_t>());
    k_check_count<<<grid_for(len), 256, 0, stream()>>>(d0, len, n, nullptr, bad.as<uint32_t>());
    NX_LAUNCH_CHECK();
    return NX_OK;
  };
  // device copies of host inputs, uploaded in chunks on a side stream so the
  // checks and histograms of one chunk overlap the copy of the next
  DevBuf ds, dd, dw;
  DevBuf sorted[2];  // forward / transpose keys sorted while the host edges arrive
  const uint32_t *s = src, *d = dst;
  const float* wp = w;
  const bool presorted = !on_dev && m && !want_w;
  if (!on_dev) {
    NX_TRY(ds.alloc(std::max<uint64_t>(m, 1) * 4));
    NX_TRY(dd.alloc(std::max<uint64_t>(m, 1) * 4));
    if (want_w) NX_TRY(dw.alloc(std::max<uint64_t>(m, 1) * 4));
    s = ds.as<uint32_t>();
    d = dd.as<uint32_t>();
    if (want_w) wp = dw.as<float>();
    if (presorted) {
      TraceRange tr("upload and sort");
      NX_TRY(upload_and_sort(g, src, dst, m, n, P, (flags & NX_RELABEL) != 0, want_t, ds.as<uint32_t>(),
                             dd.as<uint32_t>(), bad.as<uint32_t>(), sorted));
    } else if (m) {
      constexpr int kChunks = 8;
      Upload up;
      NX_TRY(up.init(kChunks));
      NX_CUDA(cudaEventRecord(up.ready, stream()));  // the buffers exist in stream order
      NX_CUDA(cudaStreamWaitEvent(up.side, up.ready, 0));
      const uint64_t chunk = round_up(ceil_div(m, kChunks), 1024);
      for (int c = 0; c < kChunks && (uint64_t)c * chunk < m; ++c) {
        const uint64_t e0 = (uint64_t)c * chunk, len = std::min<uint64_t>(chunk, m - e0);
        NX_CUDA(cudaMemcpyAsync(ds.as<uint32_t>() + e0, src + e0, len * 4, cudaMemcpyHostToDevice, up.side));
        NX_CUDA(cudaMemcpyAsync(dd.as<uint32_t>() + e0, dst + e0, len * 4, cudaMemcpyHostToDevice, up.side));
        NX_CUDA(cudaEventRecord(up.copied[c], up.side));
        NX_CUDA(cudaStreamWaitEvent(stream(), up.copied[c], 0));
        NX_TRY(scan_edges(s + e0, d + e0, len));
      }
      if (want_w) {
        NX_CUDA(cudaMemcpyAsync(dw.p, w, m * 4, cudaMemcpyHostToDevice, up.side));
        NX_CUDA(cudaEventRecord(up.ready, up.side));
        NX_CUDA(cudaStreamWaitEvent(stream(), up.ready, 0));
      }
    }
  } else if (m) {
    NX_TRY(scan_edges(s, d, m));
  }
  {  // ids < n
    uint32_t hb = 0;
    NX_CUDA(cudaMemcpyAsync(&hb, bad.p, 4, cudaMemcpyDeviceToHost, stream()));
    NX_CUDA(cudaStreamSynchronize(stream()));
    if (hb) return invalid("nx_build_dsss: an edge endpoint is >= n");
  }
  g->m = m;
  Geometry& geo = g->geo;
  geo.n = n;
  DevBuf rs, rd;
  // With nothing but the forward DSSS to build, the keys apply the new ids
  // themselves and the renamed endpoint arrays are never written.
  const bool rename_in_keys = (flags & NX_RELABEL) && !want_t && !want_w && !(flags & NX_ONCHIP_HUBS);
  if ((flags & NX_RELABEL) && presorted) {
    // the order exists and the keys carry the new ids; only the on-chip
    // structure reads the endpoint arrays, in the new ids
    if (flags & NX_ONCHIP_HUBS) NX_TRY(rename_edges(g, ds.as<uint32_t>(), dd.as<uint32_t>(), m));
  } else if ((flags & NX_RELABEL) && rename_in_keys) {
    NX_TRY(relabel_edges(g, s, d, m, nullptr, nullptr, g->outdeg.as<uint32_t>()));
  } else if (flags & NX_RELABEL) {  // host inputs are renamed in their device copies
    uint32_t* so = ds.as<uint32_t>();
    uint32_t* dout = dd.as<uint32_t>();
    if (on_dev) {
      NX_TRY(rs.alloc(std::max<uint64_t>(m, 1) * 4));
      NX_TRY(rd.alloc(std::max<uint64_t>(m, 1) * 4));
      so = rs.as<uint32_t>();
      dout = rd.as<uint32_t>();
    }
    NX_TRY(relabel_edges(g, s, d, m, so, dout, g->outdeg.as<uint32_t>()));
    s = so;
    d = dout;
  }
  if (flags & NX_RELABEL) {
    {  // out-degrees of the renamed ids: new vertex k is caller vertex old_of_new[k]
      DevBuf od2 = std::move(od_new);
      NX_TRY(gather_u32(g->old_of_new.as<uint32_t>(), g->outdeg.p, od2.p, n));
      g->outdeg = std::move(od2);
    }
  }
  geo.P = P;
  geo.L = (uint32_t)ceil_div(n, P);
  geo.lb = bits_for(geo.L);
  const uint32_t cap_log2 = (flags >> 8) & 0xFu, edges_log2 = (flags >> 12) & 0x1Fu;
  const uint64_t cap = cap_log2 ? (1ull << cap_log2) : kTileMaxCap;
  geo.tile_max = (uint32_t)std::min<uint64_t>(cap, 1ull << (32 - geo.lb));
  // the forward keys, sorted (host edges: already, as they arrived), give the
  // in-degrees the tiles are cut by
  DevBuf sorted_idx;
  TraceRange tr_rest("keys, geometry, words");
  if (!presorted)
    NX_TRY(sort_keys(s, d, m, geo, rename_in_keys ? g->new_of_old.as<uint32_t>() : nullptr, want_w,
                     sorted[0], sorted_idx));
  if (m) {
    const KeyCodec kc{geo.P, geo.L, geo.lb};
    k_indeg_from_keys<<<grid_for(m), 256, 0, stream()>>>(sorted[0].as<uint64_t>(), m, kc,
                                                         indeg.as<uint32_t>());
    NX_LAUNCH_CHECK();
  }
  DevBuf vt;
  NX_TRY(build_geometry(g, indeg.as<uint32_t>(), want_t ? g->outdeg.as<uint32_t>() : nullptr,
                        want_t ? 2 * m : m, edges_log2, vt));
  indeg.release();
  // weights: W_u in FP64, normalised weights in input order
  DevBuf wn;
  if (want_w) {
    DevBuf W;
    NX_TRY(W.alloc((uint64_t)n * 8));
    NX_CUDA(cudaMemsetAsync(W.p, 0, (uint64_t)n * 8, stream()));
    NX_TRY(wn.alloc(std::max<uint64_t>(m, 1) * 4));
    NX_TRY(g->wsum.alloc((uint64_t)n * 4));
    if (m) {
      k_wsum<<<grid_for(m), 256, 0, stream()>>>(s, wp, m, W.as<double>());
      k_wnorm<<<grid_for(m), 256, 0, stream()>>>(s, wp, m, W.as<double>(), wn.as<float>());
      NX_LAUNCH_CHECK();
    }
    k_wsum_f<<<grid_for(n), 256, 0, stream()>>>(W.as<double>(), n, g->wsum.as<float>());
    NX_LAUNCH_CHECK();
    NX_CUDA(cudaStreamSynchronize(stream()));
    g->has_w = true;
  }
  NX_TRY(build_one(s, d, m, geo, vt.as<uint64_t>(), want_w ? wn.as<float>() : nullptr, g->fwd,
                   rename_in_keys ? g->new_of_old.as<uint32_t>() : nullptr, &sorted[0], &sorted_idx));
  if (flags & NX_ONCHIP_HUBS) NX_TRY(build_onchip(g, s, d, m));
  if (want_t) {
    NX_TRY(build_one(d, s, m, geo, vt.as<uint64_t>(), want_w ? wn.as<float>() : nullptr,
                     g->tr, nullptr, &sorted[1]));
    g->has_tr = true;
  }
  if (want_w) {  // caller-order endpoints for the edge gradients
    NX_TRY(g->orig_src.alloc(std::max<uint64_t>(m, 1) * 4));
    NX_TRY(g->orig_dst.alloc(std::max<uint64_t>(m, 1) * 4));
    if (m) {
      NX_CUDA(cudaMemcpyAsync(g->orig_src.p, s, m * 4, cudaMemcpyDeviceToDevice, stream()));
      NX_CUDA(cudaMemcpyAsync(g->orig_dst.p, d, m * 4, cudaMemcpyDeviceToDevice, stream()));
    }
  }
  NX_CUDA(cudaEventRecord(ev.e1, stream()));
  NX_TRY(ev.elapsed(&g->build_ms));
  return NX_OK;
}

}  // namespace
}  // namespace nx

uint64_t nx_graph::device_bytes() const {
  const nx::DevBuf* bufs[] = {&geo.tile_start, &geo.col_tb, &fwd.ew, &fwd.wt, &fwd.piece_off,
                              &fwd.hub_off, &fwd.hub_dst, &tr.ew, &tr.wt, &tr.piece_off,
                              &tr.hub_off, &tr.hub_dst, &outdeg, &wsum, &orig_src, &orig_dst,
                              &val[0], &val[1], &aux[0], &aux[1], &act[0], &act[1], &scal,
                              &tile_part, &split_buf, &tile_ticket, &hubs, &hubs_t, &tele,
                              &lam[0], &lam[1], &ybuf, &stage[0], &stage[1], &vstage[0],
                              &vstage[1], &vstage[2], &vstage[3], &vstage[4], &vstage[5],
                              &vstage[6], &vstage[7], &accres, &init_part};
  uint64_t s = 0;
  for (auto* b : bufs) s += b->bytes;
  for (const auto& kv : plans) s += kv.second->items.bytes;
  s += old_of_new.bytes + new_of_old.bytes;
  const nx::DevBuf* ocb[] = {&oc.ew, &oc.seg_e, &oc.seg_h, &oc.hub_dst, &oc.hub_val, &oc.chunks,
                             &oc.items_a, &oc.items_b, &oc.split, &oc.ticket, &oc.part};
  for (auto* b : ocb) s += b->bytes;
  return s;
}

uint64_t nx_graph::host_bytes() const {
  const nx::PinnedBuf* bufs[] = {&fwd.h_ew, &fwd.h_hub_dst, &fwd.h_wt, &fwd.h_piece_pin,
                                 &fwd.h_hub_off, &tr.h_ew, &tr.h_hub_dst, &tr.h_wt,
                                 &tr.h_piece_pin, &tr.h_hub_off, &h_orig_src, &h_orig_dst,
                                 &hval[0], &hval[1], &hact, &oc.h_ew, &oc.h_hub_dst};
  uint64_t s = 0;
  for (auto* b : bufs) s += b->bytes;
  return s;
}

extern "C" nx_status nx_build_dsss(const uint32_t* src, const uint32_t* dst, uint64_t m,
                                   uint32_t n, uint32_t P, uint32_t flags, const float* w,
                                   nx_graph** out) {
  if (!out) return nx::invalid("nx_build_dsss: out is NULL");
  *out = nullptr;
  if (n == 0 || n > (1u << 30)) return nx::invalid("nx_build_dsss: n must be in [1, 2^30]");
  if (P == 0 || P > n || P > 1024)
    return nx::invalid("nx_build_dsss: P must be in [1, min(n, 1024)]");
  if (m >= (1ull << 32)) return nx::invalid("nx_build_dsss: m must be < 2^32");
  if (m && (!src || !dst)) return nx::invalid("nx_build_dsss: src/dst is NULL");
  {
    const uint32_t cap_log2 = (flags >> 8) & 0xFu, edges_log2 = (flags >> 12) & 0x1Fu;
    if (cap_log2 && (cap_log2 < 8 || cap_log2 > 13))
      return nx::invalid("nx_build_dsss: NX_TILE_CAP_LOG2 must be in [8, 13]");
    if (edges_log2 && (edges_log2 < 10 || edges_log2 > 20))
      return nx::invalid("nx_build_dsss: NX_TILE_EDGES_LOG2 must be in [10, 20]");
    if (flags & ~0x1FFFFu) return nx::invalid("nx_build_dsss: unknown flag bits");
  }
  if ((flags & NX_WITH_WEIGHTS) && m && !w)
    return nx::invalid("nx_build_dsss: NX_WITH_WEIGHTS needs w");
  nx::TraceRange trace("nx_build_dsss");
  nx_graph* g = new (std::nothrow) nx_graph();
  if (!g) return nx::invalid("nx_build_dsss: out of host memory");
  nx_status st = nx::build_impl(src, dst, m, n, P, flags, w, g);
  if (st != NX_OK) {
    cudaStreamSynchronize(nx::stream());
    delete g;
    return st;
  }
  *out = g;
  return NX_OK;
}
