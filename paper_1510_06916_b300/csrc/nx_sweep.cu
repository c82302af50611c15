// The DSSS update sweep (Section III-B, III-D) for sm_103a.
//
// A thread block owns one destination tile (a slice of a destination interval
// I_j) and walks the tile's piece of every sub-shard SS_ij, i = 0..P-1. Each
// warp takes 256 consecutive edge words per step (two 16-byte loads per lane),
// gathers the source values, and reduces runs of equal destination first in
// registers and then across lanes with a segmented shuffle scan. One shared-
// memory atomic per destination run folds the run into the tile accumulator,
// so there are no global atomics (Section III-D: a destination belongs to one
// worker, sorted destinations make the reduction a segmented one). After the
// last piece the block applies the program's epilogue to its tile
// (InitializeIteration / Update of Algorithm 1, 5) and writes the new values.
//
// Tiles too heavy for one block are split over several blocks; each writes its
// accumulator to a private slot and the last block to finish (a completion
// counter) combines the slots in a fixed order, so results do not depend on
// block scheduling except for the order of shared-memory atomics inside a block.
#include <mutex>
#include <type_traits>
#include <set>
#include <utility>

#include "nx_sweep.cuh"

namespace nx {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kSent = 0xFFFFFFFFu;  // run key of edges outside the range
constexpr uint32_t kInf = 0xFFFFFFFFu;

// Tile accumulator in shared memory: hi[T] plus, for sums, lo[T] holding the
// exact rounding error of every atomic add into hi (TwoSum, Knuth TAOCP vol. 2
// 4.2.2), so long runs into one destination stay compensated.
template <class V>
struct Acc {
  V* hi;
  float* lo;
};

struct PrSum {  // PageRank family: compensated sum of float contributions
  using V = float;
  static constexpr bool compensated = true;
  __device__ static V identity() { return 0.f; }
  __device__ static V op(V a, V b) { return a + b; }
  __device__ static void emit(Acc<V> acc, uint32_t k, V v) {
    const float old = atomicAdd(acc.hi + k, v);
    const float s = old + v;
    const float bb = s - old;
    const float err = (old - (s - bb)) + (v - bb);
    atomicAdd(acc.lo + k, err);
  }
  // Runs that end inside one lane (at most 8 edges): a plain add. A destination
  // gets few of these (at most two per piece), so their rounding stays small;
  // long runs cross lanes and take the compensated path above.
  __device__ static void emit_short(Acc<V> acc, uint32_t k, V v) { atomicAdd(acc.hi + k, v); }
  __device__ static V read(Acc<V> acc, uint32_t k) { return acc.hi[k] + acc.lo[k]; }
  __device__ static void emit_global(V* p, V v) { *p += v; }
};
struct MinU {  // BFS / WCC: min of uint32
  using V = uint32_t;
  static constexpr bool compensated = false;
  __device__ static V identity() { return kInf; }
  __device__ static V op(V a, V b) { return a < b ? a : b; }
  __device__ static void emit(Acc<V> acc, uint32_t k, V v) {
    if (v != kInf) atomicMin(acc.hi + k, v);
  }
  __device__ static void emit_short(Acc<V> acc, uint32_t k, V v) { emit(acc, k, v); }
  __device__ static V read(Acc<V> acc, uint32_t k) { return acc.hi[k]; }
  // row passes of WCC update a resident label from the forward and the
  // transpose DSSS in the same launch: an atomic min keeps that race benign
  __device__ static void emit_global(V* p, V v) {
    if (v < *p) atomicMin(p, v);
  }
};

struct MaxU {  // SCC backward reach: max of uint32 (0 = nothing reached)
  using V = uint32_t;
  static constexpr bool compensated = false;
  __device__ static V identity() { return 0u; }
  __device__ static V op(V a, V b) { return a > b ? a : b; }
  __device__ static void emit(Acc<V> acc, uint32_t k, V v) {
    if (v != 0u) atomicMax(acc.hi + k, v);
  }
  __device__ static void emit_short(Acc<V> acc, uint32_t k, V v) { emit(acc, k, v); }
  __device__ static V read(Acc<V> acc, uint32_t k) { return acc.hi[k]; }
  __device__ static void emit_global(V* p, V v) {
    if (v > *p) atomicMax(p, v);
  }
};

// Load of a gathered source value (random 4-byte access). NX_GATHER_MODE picks
// the cache operator: 0 = read-only path (ld.global.nc), 1 = L2 only (.cg).
#ifndef NX_GATHER_MODE
#define NX_GATHER_MODE 0
#endif
template <class T>
__device__ __forceinline__ T ld_gather(const T* p) {
#if NX_GATHER_MODE == 1
  return __ldcg(p);
#else
  return __ldg(p);
#endif
}

template <int K>
struct Prog;
// gather(raw, od, u, w): the contribution of source u whose stored value is
// `raw` (its value read from device memory).
template <>
struct Prog<PK_PR> : PrSum {  // c[u] = r[u] / outdeg[u]
  static constexpr bool weighted = false;
  __device__ static float gather(float raw, const uint32_t*, uint32_t, float) { return raw; }
};
template <>
struct Prog<PK_WPR> : PrSum {  // w^_uv r[u]
  static constexpr bool weighted = true;
  __device__ static float gather(float raw, const uint32_t*, uint32_t, float w) { return w * raw; }
};
template <>
struct Prog<PK_ADJ> : PrSum {  // w^_uv lambda[v] over the transpose DSSS
  static constexpr bool weighted = true;
  __device__ static float gather(float raw, const uint32_t*, uint32_t, float w) { return w * raw; }
};
template <>
struct Prog<PK_PRD> : PrSum {  // r[u] / outdeg[u] (u has an out-edge)
  static constexpr bool weighted = false;
  __device__ static float gather(float raw, const uint32_t* od, uint32_t u, float) {
    return raw / (float)__ldg(od + u);
  }
};
template <>
struct Prog<PK_BFS> : MinU {  // depth[u] + 1 (infinity stays infinity)
  static constexpr bool weighted = false;
  __device__ static uint32_t gather(uint32_t raw, const uint32_t*, uint32_t, float) {
    return raw == kInf ? kInf : raw + 1;
  }
};
template <>
struct Prog<PK_WCC> : MinU {  // label[u]
  static constexpr bool weighted = false;
  __device__ static uint32_t gather(uint32_t raw, const uint32_t*, uint32_t, float) { return raw; }
};
// The gather probe: the PageRank sweep's loads and gathers without the
// reduction (each warp step adds its 256 gathered values into one float).
template <>
struct Prog<PK_PROBE> : PrSum {
  static constexpr bool weighted = false;
  __device__ static float gather(float raw, const uint32_t*, uint32_t, float) { return raw; }
};
template <>
struct Prog<PK_SCCF> : MinU {  // color[u] (assigned: 0xFFFFFFFF, the identity)
  static constexpr bool weighted = false;
  __device__ static uint32_t gather(uint32_t raw, const uint32_t*, uint32_t, float) { return raw; }
};
template <>
struct Prog<PK_SCCB> : MaxU {  // reach value of the out-neighbour v (transpose DSSS)
  static constexpr bool weighted = false;
  __device__ static uint32_t gather(uint32_t raw, const uint32_t*, uint32_t, float) { return raw; }
};

__device__ __forceinline__ uint4 ld_stream(const uint32_t* p) {
  return __ldcs(reinterpret_cast<const uint4*>(p));
}
__device__ __forceinline__ float4 ld_stream_f(const float* p) {
  return __ldcs(reinterpret_cast<const float4*>(p));
}

// Edges per lane in one warp step (8 or 16): two or four 16-byte loads.
#ifndef NX_EPL
#define NX_EPL 8
#endif
constexpr int kEPL = NX_EPL;
constexpr int kStep = 32 * kEPL;  // edges per warp step
static_assert(kEPL == 8 || kEPL == 16, "edges per lane");
static_assert(kEPL <= (int)kEdgeAlign, "edge padding");

template <int N>
struct EdgeRegs {
  uint4 q[N / 4];
  float4 f[N / 4];
};

// Edge words of a step; prefetched one step ahead. The weights of weighted
// programs are loaded when their step is processed (not prefetched): without
// the second set of weight registers the weighted sweeps fit five blocks per
// SM, 2-3% faster than four blocks with prefetched weights.
template <class PG>
__device__ __forceinline__ void load_step(EdgeRegs<kEPL>& r, const uint32_t* __restrict__ ew,
                                          const float* __restrict__ wt, uint64_t idx) {
#pragma unroll
  for (int k = 0; k < kEPL / 4; ++k) r.q[k] = ld_stream(ew + idx + 4 * k);
}
__device__ __forceinline__ void load_weights(EdgeRegs<kEPL>& r, const float* __restrict__ wt,
                                             uint64_t idx) {
#pragma unroll
  for (int k = 0; k < kEPL / 4; ++k) r.f[k] = ld_stream_f(wt + idx + 4 * k);
}

// One warp step: the kStep edge words in `cur` start at edge index `base`;
// edges outside [a, b) are masked. Gathers the sources, reduces runs of equal
// destination in registers and across lanes, and folds them into `acc`.
template <class PG>
__device__ __forceinline__ void process_step(const EdgeRegs<kEPL>& cur, uint64_t base, uint64_t a,
                                             uint64_t b, const void* __restrict__ g,
                                             uint32_t sbase, uint32_t lb, Acc<typename PG::V> acc,
                                             const uint32_t* __restrict__ od) {
  using V = typename PG::V;
  const int lane = threadIdx.x & 31;
  const uint32_t smask = (1u << lb) - 1u;
  const uint32_t lo = base < a ? (uint32_t)(a - base) : 0u;
  const uint32_t hi = (b - base) < (uint64_t)kStep ? (uint32_t)(b - base) : (uint32_t)kStep;
  const uint32_t span = hi - lo;
  uint32_t key[kEPL];
  V val[kEPL];
#pragma unroll
  for (int k = 0; k < kEPL; ++k) {
    const uint4 q = cur.q[k / 4];
    const float4 f = cur.f[k / 4];
    const uint32_t w = (k & 3) == 0 ? q.x : (k & 3) == 1 ? q.y : (k & 3) == 2 ? q.z : q.w;
    const float wf = (k & 3) == 0 ? f.x : (k & 3) == 1 ? f.y : (k & 3) == 2 ? f.z : f.w;
    const bool valid = ((uint32_t)(lane * kEPL + k) - lo) < span;
    key[k] = valid ? (w >> lb) : kSent;
    const uint32_t u = sbase + (w & smask);
    V raw = PG::identity();
    if (valid) raw = ld_gather(static_cast<const V*>(g) + u);
    val[k] = valid ? PG::gather(raw, od, u, wf) : PG::identity();
  }
  if constexpr (std::is_same<PG, Prog<PK_PROBE>>::value) {
    float x = 0.f;
#pragma unroll
    for (int k = 0; k < kEPL; ++k) x += val[k];
    for (int d = 16; d > 0; d >>= 1) x += __shfl_down_sync(0xffffffffu, x, d);
    if (lane == 0) atomicAdd(acc.hi, x);
    return;
  }
  // runs of equal destination inside the lane: first (head), middle, last (tail)
  uint32_t hk = key[0], ck = key[0];
  V hs = val[0], cs = val[0];
  bool single = true;
#pragma unroll
  for (int k = 1; k < kEPL; ++k) {
    const bool brk = key[k] != ck;
    if (brk && !single && ck != kSent) PG::emit_short(acc, ck, cs);
    if (brk && single) {
      hk = ck;
      hs = cs;
    }
    single = single && !brk;
    cs = brk ? val[k] : PG::op(cs, val[k]);
    ck = key[k];
  }
  const uint32_t first_key = single ? ck : hk;
  uint32_t prev_tail = __shfl_up_sync(0xffffffffu, ck, 1);
  if (lane == 0) prev_tail = kSent;
  uint32_t next_first = __shfl_down_sync(0xffffffffu, first_key, 1);
  if (lane == 31) next_first = kSent;
  // segmented inclusive scan of the tail runs across lanes
  const bool starts = (lane == 0) || !single || (ck != prev_tail);
  const uint32_t smask_b = __ballot_sync(0xffffffffu, starts);
  const uint32_t le = smask_b & (0xffffffffu >> (31 - lane));
  const int seg0 = 31 - __clz(le);
  V x = cs;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    V y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane - d >= seg0) x = PG::op(y, x);
  }
  const V prev_x = __shfl_up_sync(0xffffffffu, x, 1);
  // the head run joins the chain of the lanes before it when the key matches
  if (!single && hk != kSent) {
    if (lane > 0 && hk == prev_tail) PG::emit(acc, hk, PG::op(prev_x, hs));
    else PG::emit_short(acc, hk, hs);
  }
  if (ck != kSent && next_first != ck) {
    if (seg0 < lane) PG::emit(acc, ck, x);  // the run crossed lanes
    else PG::emit_short(acc, ck, x);
  }
}

// Folds edges [a, b) of one piece into the tile accumulator. Edge e is read at
// ew[e - ew_lo]; its source value at g[sbase + src_local]. The piece is cut
// into kStep-edge steps from a rounded down to kEPL; step k goes to warp
// (k + rot) % 8 so that short pieces do not all land on the same warps (rot
// advances by the piece's step count). Each warp loads its next step's edge
// words before it gathers and reduces the current one.
template <class PG>
__device__ __forceinline__ void sweep_range(const uint32_t* __restrict__ ew,
                                            const float* __restrict__ wt, uint64_t ew_lo,
                                            uint64_t a, uint64_t b, const void* __restrict__ g,
                                            uint32_t sbase, uint32_t lb,
                                            Acc<typename PG::V> acc, uint32_t& rot,
                                            const uint32_t* __restrict__ od) {
  using V = typename PG::V;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t a0 = a & ~(uint64_t)(kEPL - 1);
  const uint32_t nsteps = (uint32_t)((b - a0 + kStep - 1) / kStep);
  const uint32_t k0 = (uint32_t)((warp - (int)rot) & (kWarps - 1));
  rot = (rot + nsteps) & (kWarps - 1);
  uint64_t base = a0 + (uint64_t)k0 * kStep;
  if (base >= b) return;
  EdgeRegs<kEPL> nxt;
#pragma unroll
  for (int k = 0; k < kEPL / 4; ++k) {
    nxt.q[k] = make_uint4(0, 0, 0, 0);
    nxt.f[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  {
    const uint64_t p = base + (uint64_t)lane * kEPL;
    if (p < b) load_step<PG>(nxt, ew, wt, p - ew_lo);
  }
  while (base < b) {
    EdgeRegs<kEPL> cur = nxt;
    if (PG::weighted) {
      const uint64_t p = base + (uint64_t)lane * kEPL;
      if (p < b) load_weights(cur, wt, p - ew_lo);
    }
    const uint64_t nbase = base + (uint64_t)kWarps * kStep;
    {  // prefetch the warp's next step
      const uint64_t pn = nbase + (uint64_t)lane * kEPL;
      if (pn < b) load_step<PG>(nxt, ew, wt, pn - ew_lo);
    }
    process_step<PG>(cur, base, a, b, g, sbase, lb, acc, od);
    base = nbase;
  }
}

// Block-wide exclusive scan (all kThreads threads call it); returns this
// thread's prefix and writes the total to *total.
template <class T>
__device__ __forceinline__ T block_scan_excl(T v, T* total) {
  __shared__ T wsum[kWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  T before = 0, all = 0;
#pragma unroll
  for (int q = 0; q < kWarps; ++q) {
    const T t = wsum[q];
    before += q < w ? t : T(0);
    all += t;
  }
  __syncthreads();
  *total = all;
  return before + x - v;
}

// The item's pieces as one sequence of warp steps (at most kThreads pieces):
// warps take steps w, w + 8, ... over the whole sequence, so they stay
// balanced and each prefetches its next step even across piece boundaries.
// The table lives in dynamic shared memory after the accumulators, 16 bytes
// per piece: valid range [a, b) (edge indices < 2^32), the warp steps before
// the piece (low 24 bits) with the DSSS index (bit 24) and a staged-source
// flag (bit 25), and the source interval base.
struct FlatEnt {
  uint32_t a, b, cum, sb;
};

template <class PG>
__device__ __forceinline__ void sweep_flat(const SweepArgs& a, const Item& it, uint32_t t,
                                           uint32_t tb, uint32_t nt, uint32_t i_lo, uint32_t i_hi,
                                           Acc<typename PG::V> acc, FlatEnt* tab) {
  const uint32_t npi = i_hi - i_lo;
  const uint32_t np = (uint32_t)a.nsrc * npi;
  const uint32_t k = threadIdx.x;
  uint64_t p0 = 0, len = 0;
  bool active = false;
  uint32_t s = 0, i = 0;
  if (k < np) {
    s = k / npi;
    i = i_lo + k % npi;
    const uint64_t* po = a.src[s].piece_off;
    const uint64_t pc = piece_index(a.P, tb, nt, i, t);
    p0 = po[pc];
    len = po[pc + 1] - p0;
    active = !a.act_in || a.act_in[i];
  }
  uint64_t vtot;
  const uint64_t vo = block_scan_excl<uint64_t>(len, &vtot);
  uint32_t steps = 0;
  uint64_t ea = 0, eb = 0;
  if (k < np && active) {
    const uint64_t lo = vo > it.vbeg ? vo : it.vbeg;
    const uint64_t hi = (vo + len) < it.vend ? (vo + len) : it.vend;
    if (lo < hi) {
      ea = p0 + (lo - vo);
      eb = p0 + (hi - vo);
      steps = (uint32_t)((eb - (ea & ~(uint64_t)(kEPL - 1)) + kStep - 1) / kStep);
    }
  }
  uint32_t stot;
  const uint32_t before = block_scan_excl<uint32_t>(steps, &stot);
  const bool staged = (i == a.stage_i);
  if (k < np) {
    FlatEnt e;
    e.a = (uint32_t)ea;
    e.b = (uint32_t)eb;
    e.cum = before | (s << 24) | (staged ? (1u << 25) : 0u);
    e.sb = staged ? 0u : i * a.L;
    tab[k] = e;
  }
  if (k == 0) tab[np].cum = stot;
  __syncthreads();
  constexpr uint32_t kCum = (1u << 24) - 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t q = warp, p = 0;
  if (q >= stot) return;
  while ((tab[p + 1].cum & kCum) <= q) ++p;
  FlatEnt ep = tab[p];
  uint64_t base = (uint64_t)(ep.a & ~(uint32_t)(kEPL - 1)) + (uint64_t)(q - (ep.cum & kCum)) * kStep;
  EdgeRegs<kEPL> nxt;
#pragma unroll
  for (int z = 0; z < kEPL / 4; ++z) {
    nxt.q[z] = make_uint4(0, 0, 0, 0);
    nxt.f[z] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  {
    const uint32_t sx = (ep.cum >> 24) & 1u;
    const uint64_t e = base + (uint64_t)lane * kEPL;
    if (e < ep.b) load_step<PG>(nxt, a.src[sx].ew, a.src[sx].wt, e - a.ew_lo[sx]);
  }
  while (q < stot) {
    EdgeRegs<kEPL> cur = nxt;
    const FlatEnt ec = ep;
    const uint64_t bc = base;
    if (PG::weighted) {
      const uint32_t sxc = (ec.cum >> 24) & 1u;
      const uint64_t e = bc + (uint64_t)lane * kEPL;
      if (e < ec.b) load_weights(cur, a.src[sxc].wt, e - a.ew_lo[sxc]);
    }
    const uint32_t qn = q + kWarps;
    if (qn < stot) {  // prefetch the warp's next step, possibly in a later piece
      while ((tab[p + 1].cum & kCum) <= qn) ++p;
      ep = tab[p];
      base = (uint64_t)(ep.a & ~(uint32_t)(kEPL - 1)) + (uint64_t)(qn - (ep.cum & kCum)) * kStep;
      const uint32_t sx = (ep.cum >> 24) & 1u;
      const uint64_t e = base + (uint64_t)lane * kEPL;
      if (e < ep.b) load_step<PG>(nxt, a.src[sx].ew, a.src[sx].wt, e - a.ew_lo[sx]);
    }
    const void* g = (ec.cum & (1u << 25)) ? a.gstage : a.gsrc;
    process_step<PG>(cur, bc, ec.a, ec.b, g, ec.sb, a.lb, acc, a.outdeg);
    q = qn;
  }
}

__device__ __forceinline__ double block_sum_d(double v, double* red) {
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < kWarps; ++q) t += red[q];
  return t;  // valid in thread 0
}

// One work item: the tile's pieces, the split merge and the epilogue. Called
// by k_sweep (one item per block) and by the persistent multi-graph kernel.
template <int K>
__device__ __forceinline__ void sweep_item(const SweepArgs& a, Item it, unsigned char* smem_raw) {
  using PG = Prog<K>;
  using V = typename PG::V;
  Acc<V> acc;
  acc.hi = reinterpret_cast<V*>(smem_raw);
  acc.lo = PG::compensated ? reinterpret_cast<float*>(smem_raw) + a.tile_max : nullptr;
  __shared__ double red[kWarps];
  __shared__ int s_flag;
  const uint32_t t = it.tile;
  const uint32_t ts = a.tile_start[t], te = a.tile_start[t + 1];
  const uint32_t T = te - ts;
  const uint32_t j = ts / a.L;
  const uint32_t tb = a.col_tb[j], nt = a.col_tb[j + 1] - tb;

  if (a.mode == 3) {  // epilogue from the stored accumulators of resident columns
    const V* ar = static_cast<const V*>(a.accres) + (ts - a.acc_base);
    for (uint32_t k = threadIdx.x; k < T; k += kThreads) acc.hi[k] = ar[k];
  } else if (a.acc_in && it.sub == 0) {  // banded sweep: continue from the earlier bands
    const V* ai = static_cast<const V*>(a.acc_in) + (ts - a.acc_base);
    for (uint32_t k = threadIdx.x; k < T; k += kThreads) acc.hi[k] = ai[k];
  } else {
    for (uint32_t k = threadIdx.x; k < T; k += kThreads) acc.hi[k] = PG::identity();
  }
  if (PG::compensated)
    for (uint32_t k = threadIdx.x; k < T; k += kThreads) acc.lo[k] = 0.f;
  __syncthreads();

  if (a.mode != 3) {
    // edges: pieces (i, t) for i in [src_lo, src_hi) of every DSSS of the sweep
    uint64_t vo = 0;
    uint32_t rot = 0;
    const uint32_t i_lo = a.mode == 1 ? it.row : a.src_lo;
    const uint32_t i_hi = a.mode == 1 ? it.row + 1 : a.src_hi;
    const bool flat = a.flat_cap && a.mode != 1 && (uint32_t)a.nsrc * (i_hi - i_lo) <= a.flat_cap;
    // a row-pass item sweeps one piece of one DSSS
    const int s_lo = a.mode == 1 ? (int)it.pad : 0;
    const int s_hi = a.mode == 1 ? (int)it.pad + 1 : a.nsrc;
    if (flat) {
      FlatEnt* tab = reinterpret_cast<FlatEnt*>(smem_raw + (size_t)a.tile_max * (PG::compensated ? 8 : 4));
      if (i_hi > i_lo) sweep_flat<PG>(a, it, t, tb, nt, i_lo, i_hi, acc, tab);
    } else
    for (int s = s_lo; s < s_hi && vo < it.vend; ++s) {
      const uint64_t* po = a.src[s].piece_off;
      for (uint32_t i = i_lo; i < i_hi && vo < it.vend; ++i) {
        const uint64_t pc = piece_index(a.P, tb, nt, i, t);
        const uint64_t p0 = po[pc], len = po[pc + 1] - p0;
        const uint64_t lo = vo > it.vbeg ? vo : it.vbeg;
        const uint64_t hi = (vo + len) < it.vend ? (vo + len) : it.vend;
        if (lo < hi && (!a.act_in || a.act_in[i])) {
          const bool staged = (i == a.stage_i);
          const void* g = staged ? a.gstage : a.gsrc;
          const uint32_t sb = staged ? 0u : i * a.L;
          sweep_range<PG>(a.src[s].ew, a.src[s].wt, a.ew_lo[s], p0 + (lo - vo), p0 + (hi - vo), g,
                          sb, a.lb, acc, rot, a.outdeg);
        }
        vo += len;
      }
    }
    if constexpr (K == PK_PROBE) {  // keep the loads alive, skip everything after them
      __syncthreads();
      if (threadIdx.x == 0 && acc.hi[0] == 12345.678f) static_cast<float*>(a.vnew)[0] = acc.hi[0];
      return;
    }
    // FromHub (Algorithm 6, 7): fold hub entries of pieces (i, t), i in [hub_lo, hub_hi)
    if (a.mode == 0 && it.sub == 0 && a.hub_lo < a.hub_hi) {
      for (int s = 0; s < a.nsrc; ++s) {
        const V* hv = static_cast<const V*>(a.hubs[s]);
        const uint64_t* ho = a.hub_off[s];
        const uint16_t* hd = a.hub_dst[s];
        for (uint32_t i = a.hub_lo; i < a.hub_hi; ++i) {
          if (a.act_in && !a.act_in[i]) continue;
          const uint64_t pc = piece_index(a.P, tb, nt, i, t);
          const uint64_t h0 = ho[pc], h1 = ho[pc + 1];
          for (uint64_t k = h0 + threadIdx.x; k < h1; k += kThreads) PG::emit(acc, hd[k], hv[k]);
        }
      }
    }
    __syncthreads();

    if (it.nsplit > 1) {  // combine the blocks of a split tile in slot order
      // slot q holds hi[tile_max] (+ lo[tile_max] for sums)
      const uint64_t slot_len = (uint64_t)a.tile_max * (PG::compensated ? 2 : 1);
      V* sp = static_cast<V*>(a.split);
      V* mine = sp + (uint64_t)(it.slot + it.sub) * slot_len;
      for (uint32_t k = threadIdx.x; k < T; k += kThreads) {
        mine[k] = acc.hi[k];
        if (PG::compensated) reinterpret_cast<float*>(mine)[a.tile_max + k] = acc.lo[k];
      }
      __threadfence();
      __syncthreads();
      // one completion counter per (tile, DSSS of a row-pass item)
      const uint32_t tix = t + (a.mode == 1 ? it.pad * a.col_tb[a.P] : 0u);
      if (threadIdx.x == 0) s_flag = (atomicAdd(&a.tile_ticket[tix], 1u) == it.nsplit - 1);
      __syncthreads();
      if (!s_flag) return;
      __threadfence();
      if (threadIdx.x == 0) a.tile_ticket[tix] = 0;
      for (uint32_t k = threadIdx.x; k < T; k += kThreads) {
        if constexpr (PG::compensated) {
          double v = 0.0;  // fixed slot order, double precision
          for (uint32_t q = 0; q < it.nsplit; ++q) {
            const float* sq = reinterpret_cast<const float*>(sp + (uint64_t)(it.slot + q) * slot_len);
            v += (double)__ldcg(sq + k) + (double)__ldcg(sq + a.tile_max + k);
          }
          const float hi = (float)v;
          acc.hi[k] = hi;
          acc.lo[k] = (float)(v - (double)hi);
        } else {
          V v = PG::identity();
          for (uint32_t q = 0; q < it.nsplit; ++q)
            v = PG::op(v, __ldcg(sp + (uint64_t)(it.slot + q) * slot_len + k));
          acc.hi[k] = v;
        }
      }
      __syncthreads();
    }
  }

  if (a.mode == 1) {  // row pass of one source interval (Algorithm 6 ToHub / 7 lines 9-14)
    const uint32_t i = it.row;
    const uint32_t sx = it.pad;
    const uint64_t pc = piece_index(a.P, tb, nt, i, t);
    const uint64_t* ho = a.hub_off[sx];
    const uint16_t* hd = a.hub_dst[sx];
    const uint64_t h0 = ho[pc], h1 = ho[pc + 1];
    if (j < a.q_res) {  // destination resident: update it in place
      V* ar = static_cast<V*>(a.accres) + (ts - a.acc_base);
      for (uint64_t k = h0 + threadIdx.x; k < h1; k += kThreads) {
        const uint32_t o = hd[k];
        PG::emit_global(ar + o, PG::read(acc, o));
      }
    } else {  // destination on the host side: write the hub
      V* hv = static_cast<V*>(a.hubs[sx]);
      for (uint64_t k = h0 + threadIdx.x; k < h1; k += kThreads) hv[k] = PG::read(acc, hd[k]);
    }
    return;
  }
  if (a.mode == 2) {
    V* ar = static_cast<V*>(a.accres) + (ts - a.acc_base);
    for (uint32_t k = threadIdx.x; k < T; k += kThreads) ar[k] = PG::read(acc, k);
    return;
  }

  // ---- epilogue (modes 0 and 3)
  if constexpr (K == PK_ADJ) {
    // lambda' = g + a (acc + [dangling] S / n); the fold sums lambda' over all vertices
    const float alpha = a.alpha;
    const float sn = (float)(*a.dm_in) / (float)a.n;
    float* ln = static_cast<float*>(a.vnew);
    double part = 0.0;
    for (uint32_t k = threadIdx.x; k < T; k += kThreads) {
      const uint32_t v = ts + k;
      const float dang = a.outdeg[v] == 0 ? sn : 0.0f;
      const float l = a.tele[v] + alpha * (PG::read(acc, k) + dang);
      ln[v] = l;
      part += (double)l;
    }
    const double tot = block_sum_d(part, red);
    if (threadIdx.x == 0) a.tile_part[t] = tot;
  } else if constexpr (K == PK_PR || K == PK_WPR || K == PK_PRD) {
    const float alpha = a.alpha;
    const float inv_n = 1.0f / (float)a.n;
    const float dm = (float)(*a.dm_in);
    float* rn = static_cast<float*>(a.vnew);
    double part = 0.0;
    for (uint32_t k = threadIdx.x; k < T; k += kThreads) {
      const uint32_t v = ts + k;
      const float tv = a.tele ? a.tele[v] : inv_n;
      const float spread = a.dang_by_tele ? tv : inv_n;
      const float r = (1.0f - alpha) * tv + alpha * (PG::read(acc, k) + dm * spread);
      rn[v - a.out_base] = r;
      const uint32_t od = a.outdeg[v];
      if (a.cnew) a.cnew[v - a.out_base] = od ? r / (float)od : 0.0f;
      if (od == 0) part += (double)r;
    }
    const double tot = block_sum_d(part, red);
    if (threadIdx.x == 0) a.tile_part[t] = tot;
  } else {
    const uint32_t* vo = static_cast<const uint32_t*>(a.vold);
    uint32_t* vn = static_cast<uint32_t*>(a.vnew);
    bool changed = false;
    for (uint32_t k = threadIdx.x; k < T; k += kThreads) {
      const uint32_t v = ts + k - a.out_base;
      const uint32_t o = vo[v];
      const uint32_t ak = acc.hi[k];
      uint32_t nv;
      if constexpr (K == PK_SCCF) {  // assigned vertices keep their mark
        nv = (o == kInf || ak >= o) ? o : ak;
      } else if constexpr (K == PK_SCCB) {  // reached once an out-neighbour of its color is
        const uint32_t c = a.aux_u32[ts + k];
        nv = (o == 0u && c != kInf && ak == c + 1u) ? ak : o;
      } else {
        nv = ak < o ? ak : o;
      }
      vn[v] = nv;
      changed |= nv != o;
    }
    if (__syncthreads_or(changed) && threadIdx.x == 0) a.act_out[j] = 1u;
  }

  // ---- iteration completion: the last epilogue of the iteration folds the
  // per-tile dangling mass (fixed order) / counts active intervals.
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_flag = (atomicAdd(a.ticket, 1u) == a.n_epi - 1);
  __syncthreads();
  if (!s_flag) return;
  __threadfence();
  if constexpr (K == PK_PR || K == PK_WPR || K == PK_PRD || K == PK_ADJ) {
    const uint32_t ntiles = a.col_tb[a.P];
    double s = 0.0;
    for (uint32_t q = threadIdx.x; q < ntiles; q += kThreads) s += __ldcg(a.tile_part + q);
    const double tot = block_sum_d(s, red);
    if (threadIdx.x == 0) *a.dm_out = tot;
  } else {
    uint32_t c = 0;
    for (uint32_t q = threadIdx.x; q < a.P; q += kThreads) c += __ldcg(a.act_out + q) ? 1u : 0u;
    for (int d = 16; d > 0; d >>= 1) c += __shfl_down_sync(0xffffffffu, c, d);
    __shared__ uint32_t cnt[kWarps];
    if ((threadIdx.x & 31) == 0) cnt[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t tot = 0;
      for (int q = 0; q < kWarps; ++q) tot += cnt[q];
      *a.act_count = tot;
    }
    // the flags read this iteration become the next iteration's output flags
    if (a.act_in)
      for (uint32_t q = threadIdx.x; q < a.P; q += kThreads) const_cast<uint32_t*>(a.act_in)[q] = 0u;
  }
  if (threadIdx.x == 0) *a.ticket = 0u;
}

// Blocks per SM the register budget is set for: five (48 registers) --
// PageRank's sweep ran 4.3% faster at R-MAT scale 26 (5.38 vs 5.62 ms), BFS /
// WCC 1-3% faster and the weighted programs 2-3% faster with the fifth
// block's gathers in flight -- and four (64 registers) for the r/outdeg
// gather, which carries a second gathered value per edge.
template <int K>
constexpr int sweep_min_blocks() {
  return K == PK_PRD ? 4 : 5;
}

template <int K>
__global__ void __launch_bounds__(kThreads, sweep_min_blocks<K>()) k_sweep(const __grid_constant__ SweepArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Item it;
  if (a.items) {
    it = a.items[blockIdx.x];
  } else {  // one block per tile, whole tile
    it.tile = blockIdx.x;
    it.nsplit = 1;
    it.slot = 0;
    it.sub = 0;
    it.vbeg = 0;
    it.vend = ~0ull;
    it.row = 0;
    it.pad = 0;
  }
  sweep_item<K>(a, it, smem_raw);
}

// ---------------------------------------------------------------- many graphs
// Persistent kernel over several independent graphs: every iteration, blocks
// pull (graph, item) pairs from a shared counter, sweep them with the graph's
// own arguments (args[2*gid + parity]), then meet at a grid barrier before the
// next iteration. The barrier spins a bounded number of cycles; on expiry it
// sets *err and every block returns.
__device__ __forceinline__ bool grid_barrier(MultiSync* sy, unsigned nblocks, long long limit) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    volatile unsigned* gen = &sy->gen;
    const unsigned g0 = *gen;
    __threadfence();
    if (atomicAdd(&sy->count, 1u) == nblocks - 1) {
      sy->count = 0;
      __threadfence();
      atomicAdd(&sy->gen, 1u);
      s_ok = 1;
    } else {
      const long long t0 = clock64();
      s_ok = 1;
      while (*gen == g0) {
        if (*(volatile unsigned*)&sy->err) {
          s_ok = 0;
          break;
        }
        if (clock64() - t0 > limit) {
          atomicExch(&sy->err, 1u);
          s_ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return s_ok != 0;
}

// The persistent kernel's register budget is set for five blocks per SM
// (48 registers; the programs spill a little there, but the extra warps win:
// 256 R-MAT graphs, PageRank x20 16.9 vs 19.7 ms at three blocks, BFS / WCC
// x40 9.0 / 17.1 vs 12.2 / 22.7 ms; six blocks lost on PageRank), and for
// three for weighted PageRank, which spills badly below 80 registers.
template <int K>
__global__ void __launch_bounds__(kThreads, K == PK_WPR ? 3 : 5) k_multi(const SweepArgs* __restrict__ args,
                                                    const MItem* __restrict__ items,
                                                    uint32_t nitems, uint32_t iters,
                                                    uint32_t* __restrict__ ctr, MultiSync* sy,
                                                    long long limit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t s_idx;
  // the item's arguments live in shared memory: reading them through a global
  // reference would reload them after every store the sweep makes
  __shared__ __align__(16) SweepArgs s_args;
  for (uint32_t itn = 0; itn < iters; ++itn) {
    const uint32_t par = itn & 1u;
    for (;;) {
      __syncthreads();
      if (threadIdx.x == 0) s_idx = atomicAdd(ctr + itn, 1u);
      __syncthreads();
      const uint32_t q = s_idx;
      if (q >= nitems) break;
      const MItem mi = items[q];
      {
        const uint32_t* srcw = reinterpret_cast<const uint32_t*>(args + 2 * mi.gid + par);
        uint32_t* dstw = reinterpret_cast<uint32_t*>(&s_args);
        for (uint32_t w = threadIdx.x; w < sizeof(SweepArgs) / 4; w += blockDim.x) dstw[w] = srcw[w];
      }
      __syncthreads();
      sweep_item<K>(s_args, mi.it, smem_raw);
    }
    if (!grid_barrier(sy, gridDim.x, limit)) return;
  }
}

}  // namespace

nx_status launch_multi(ProgKind kind, const SweepArgs* args, const MItem* items, uint32_t nitems,
                       uint32_t iters, uint32_t* ctr, MultiSync* sy, uint32_t tile_max,
                       uint32_t nblocks, long long limit, cudaStream_t s) {
  const bool sums = (kind == PK_PR || kind == PK_WPR);
  const size_t smem = (size_t)tile_max * (sums ? 8 : 4) + (size_t)(kThreads + 1) * sizeof(FlatEnt);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.gridDim = dim3(nblocks);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  switch (kind) {
    case PK_PR: NX_CUDA(cudaLaunchKernelEx(&cfg, k_multi<PK_PR>, args, items, nitems, iters, ctr, sy, limit)); break;
    case PK_WPR: NX_CUDA(cudaLaunchKernelEx(&cfg, k_multi<PK_WPR>, args, items, nitems, iters, ctr, sy, limit)); break;
    case PK_BFS: NX_CUDA(cudaLaunchKernelEx(&cfg, k_multi<PK_BFS>, args, items, nitems, iters, ctr, sy, limit)); break;
    case PK_WCC: NX_CUDA(cudaLaunchKernelEx(&cfg, k_multi<PK_WCC>, args, items, nitems, iters, ctr, sy, limit)); break;
    default: return invalid("launch_multi: program not supported");
  }
  return NX_OK;
}

nx_status multi_blocks(ProgKind kind, uint32_t tile_max, uint32_t* nblocks) {
  const bool sums = (kind == PK_PR || kind == PK_WPR);
  const size_t smem = (size_t)tile_max * (sums ? 8 : 4) + (size_t)(kThreads + 1) * sizeof(FlatEnt);
  if (smem > 40 * 1024) {  // tiles above the default cap: opt in to more shared memory
    const void* fn = kind == PK_PR ? reinterpret_cast<const void*>(k_multi<PK_PR>)
                   : kind == PK_WPR ? reinterpret_cast<const void*>(k_multi<PK_WPR>)
                   : kind == PK_BFS ? reinterpret_cast<const void*>(k_multi<PK_BFS>)
                                    : reinterpret_cast<const void*>(k_multi<PK_WCC>);
    NX_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  }
  int per_sm = 0;
  switch (kind) {
    case PK_PR: NX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_multi<PK_PR>, kThreads, smem)); break;
    case PK_WPR: NX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_multi<PK_WPR>, kThreads, smem)); break;
    case PK_BFS: NX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_multi<PK_BFS>, kThreads, smem)); break;
    case PK_WCC: NX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_multi<PK_WCC>, kThreads, smem)); break;
    default: return invalid("multi_blocks: program not supported");
  }
  if (per_sm < 1) return invalid("multi_blocks: kernel does not fit on an SM");
  *nblocks = (uint32_t)per_sm * (uint32_t)num_sms();
  return NX_OK;
}

size_t flat_table_bytes(const SweepArgs& a) {
  return a.flat_cap ? (size_t)(a.flat_cap + 1) * sizeof(FlatEnt) : 0;
}

const void* sweep_fn(ProgKind kind) {
  switch (kind) {
    case PK_PR: return reinterpret_cast<const void*>(k_sweep<PK_PR>);
    case PK_WPR: return reinterpret_cast<const void*>(k_sweep<PK_WPR>);
    case PK_BFS: return reinterpret_cast<const void*>(k_sweep<PK_BFS>);
    case PK_WCC: return reinterpret_cast<const void*>(k_sweep<PK_WCC>);
    case PK_PRD: return reinterpret_cast<const void*>(k_sweep<PK_PRD>);
    case PK_ADJ: return reinterpret_cast<const void*>(k_sweep<PK_ADJ>);
    case PK_SCCF: return reinterpret_cast<const void*>(k_sweep<PK_SCCF>);
    case PK_PROBE: return reinterpret_cast<const void*>(k_sweep<PK_PROBE>);
    case PK_SCCB: return reinterpret_cast<const void*>(k_sweep<PK_SCCB>);
  }
  return nullptr;
}

// Function attributes of a sweep kernel for `smem` bytes of dynamic shared
// memory: the opt-in limit when dynamic + static shared memory pass the 48 KB
// default (per device), and the smallest shared-memory carveout that still
// holds the blocks an SM can run (the registers allow four or five), so the rest
// of the unified L1 caches the random source gathers. The driver's own choice
// reserved more: PageRank ran 0-6% slower with it (R-MAT scales 22-26,
// P = 8-64).
nx_status configure_sweep(ProgKind kind, size_t smem) {
  const void* fn = sweep_fn(kind);
  if (smem > 40 * 1024) {
    static std::mutex mu;
    static std::set<std::pair<int, int>> raised;
    int dev = 0;
    NX_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    if (raised.insert(std::make_pair(dev, (int)kind)).second)
      NX_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  }
  return prefer_l1(fn, kThreads, smem);
}

nx_status launch_sweep(ProgKind kind, const SweepArgs& a, uint32_t nitems, cudaStream_t s) {
  if (nitems == 0) return NX_OK;
  const bool sums = (kind == PK_PR || kind == PK_WPR || kind == PK_PRD || kind == PK_ADJ ||
                     kind == PK_PROBE);
  const size_t smem = (size_t)a.tile_max * (sums ? 8 : 4) + flat_table_bytes(a);
  NX_TRY(configure_sweep(kind, smem));
  switch (kind) {
    case PK_PR: k_sweep<PK_PR><<<nitems, kThreads, smem, s>>>(a); break;
    case PK_WPR: k_sweep<PK_WPR><<<nitems, kThreads, smem, s>>>(a); break;
    case PK_BFS: k_sweep<PK_BFS><<<nitems, kThreads, smem, s>>>(a); break;
    case PK_WCC: k_sweep<PK_WCC><<<nitems, kThreads, smem, s>>>(a); break;
    case PK_PRD: k_sweep<PK_PRD><<<nitems, kThreads, smem, s>>>(a); break;
    case PK_ADJ: k_sweep<PK_ADJ><<<nitems, kThreads, smem, s>>>(a); break;
    case PK_SCCF: k_sweep<PK_SCCF><<<nitems, kThreads, smem, s>>>(a); break;
    case PK_PROBE: k_sweep<PK_PROBE><<<nitems, kThreads, smem, s>>>(a); break;
    case PK_SCCB: k_sweep<PK_SCCB><<<nitems, kThreads, smem, s>>>(a); break;
  }
  NX_LAUNCH_CHECK();
  return NX_OK;
}

}  // namespace nx
