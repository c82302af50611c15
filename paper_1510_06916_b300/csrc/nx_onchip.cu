// The Double-Phase Update (Algorithm 6) with intervals sized to shared memory.
//
// The paper keeps intervals in main memory and writes hubs to disk; on the
// B300 the level that holds an interval is the SM's shared memory and the
// level that holds hubs is HBM. ToHub walks the edges row by row (source
// interval i of 2^15 vertices): a block stages I_i's contributions c in shared
// memory, so every gather is an on-chip load, and reduces each run of equal
// destination into one hub value, written once, in order. FromHub walks the
// hubs column by column (destination interval j of 2^14 vertices): a block
// folds every hub entry of column j into a compensated shared-memory
// accumulator (TwoSum, Knuth TAOCP vol. 2 4.2.2) and applies the PageRank
// epilogue. Both phases stream HBM sequentially; with degree-ordered ids the
// hubs hold 15-25% as many entries as there are edges.
#include <algorithm>
#include <cstring>
#include <vector>

#include "nx_internal.cuh"

namespace nx {
namespace {

constexpr int kOcThreads = 1024;
constexpr int kOcWarps = kOcThreads / 32;
constexpr uint32_t kSrcLen = 1u << kOcSrcBits;  // source interval (ToHub)
constexpr uint32_t kDstLen = 1u << kOcDstBits;  // destination interval (FromHub)
constexpr uint32_t kChunk = 256;                // hub entries per FromHub chunk
constexpr uint32_t kSegsPerItem = 256;          // ToHub segments per block (8 per warp)

// ---------------------------------------------------------------- build
__global__ void k_oc_keys(const uint32_t* __restrict__ s, const uint32_t* __restrict__ d,
                          uint64_t m, uint64_t* __restrict__ key) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    const uint64_t u = s[e], v = d[e];
    key[e] = ((u >> kOcSrcBits) << 45) | ((v >> kOcDstBits) << 29) |
             ((v & (kDstLen - 1)) << 15) | (u & (kSrcLen - 1));
  }
}

// Hub-entry starts (a new (i, j, destination), or a cut every kOcSeg edges)
// and the 16-bit edge entries ToHub reads: src_local | start << 15.
__global__ void k_oc_words(const uint64_t* __restrict__ key, uint64_t m,
                           uint16_t* __restrict__ ew, uint32_t* __restrict__ head) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    const uint64_t k = key[e];
    const bool h = e == 0 || (k >> 15) != (key[e - 1] >> 15) || e % kOcSeg == 0;
    ew[e] = (uint16_t)((k & (kSrcLen - 1)) | (h ? 0x8000u : 0u));
    head[e] = h ? 1u : 0u;
  }
}

// Hub destinations and entries per piece (row-major i * PB + j).
__global__ void k_oc_hubs(const uint64_t* __restrict__ key, const uint32_t* __restrict__ head,
                          const uint32_t* __restrict__ hidx, uint64_t m, uint32_t PB,
                          uint16_t* __restrict__ hub_dst, uint32_t* __restrict__ cnt) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) {
    if (!head[e]) continue;
    const uint64_t k = key[e];
    hub_dst[hidx[e]] = (uint16_t)((k >> 15) & (kDstLen - 1));
    atomicAdd(cnt + (k >> 45) * PB + ((k >> 29) & 0xFFFFu), 1u);
  }
}

// First edge of each row (source interval) in the sorted keys: rs[r] = the
// first e with key[e] >> 45 >= r (a binary search per row).
__global__ void k_oc_row_starts(const uint64_t* __restrict__ key, uint64_t m, uint32_t PA,
                                uint64_t* __restrict__ rs) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r > PA) return;
  uint64_t lo = 0, hi = m;
  while (lo < hi) {
    const uint64_t mid = lo + ((hi - lo) >> 1);
    if ((key[mid] >> 45) < r) lo = mid + 1;
    else hi = mid;
  }
  rs[r] = lo;
}

__global__ void k_oc_seg_hub(const uint64_t* __restrict__ seg_e, uint32_t nseg,
                             const uint32_t* __restrict__ hidx, uint64_t* __restrict__ seg_h) {
  const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nseg) seg_h[q] = hidx[seg_e[q]];
}

unsigned grid_n(uint64_t work) {
  return (unsigned)std::min<uint64_t>(ceil_div(work ? work : 1, 256), (uint64_t)num_sms() * 16);
}

// ---------------------------------------------------------------- ToHub
struct ArgsA {
  const uint16_t* ew;
  const uint64_t* seg_e;
  const uint64_t* seg_h;
  const OcItemA* items;
  const float* c_in;
  float* hub_val;
  uint64_t H;
  uint32_t n, nseg;
};

// One 256-edge step of a segment (see oc_segment): lane l holds the 16-bit
// entries of edges base + 8 l .. + 7 (source offset, and bit 15 set where a
// hub entry starts). FULL: every edge of the step lies inside the segment.
template <bool FULL>
__device__ __forceinline__ void oc_step(const uint4 w, uint64_t base, uint64_t e0, uint64_t e1,
                                        const float* __restrict__ csh, float* __restrict__ hv,
                                        uint32_t hlim, uint32_t& cnt, float& csum) {
  const int lane = threadIdx.x & 31;
  const uint32_t wv[4] = {w.x, w.y, w.z, w.w};
  float val[8];
  uint32_t hm = 0;
  const uint64_t p0 = base + (uint64_t)lane * 8;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint32_t e = (wv[k >> 1] >> (16 * (k & 1))) & 0xFFFFu;
    const bool valid = FULL || (p0 + k >= e0 && p0 + k < e1);
    val[k] = valid ? csh[e & (kSrcLen - 1)] : 0.f;
    hm |= (valid ? (e >> 15) : 0u) << k;
  }
  const uint32_t hc = __popc(hm);
  uint32_t incl = hc;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += y;
  }
  const uint32_t hb = cnt + incl - hc;  // entries of the segment started before this lane
  const uint32_t htot = __shfl_sync(0xffffffffu, incl, 31);
  // in-lane runs: F before the first head, the open run from the last head;
  // runs between two heads of the lane are complete and written here
  float run = 0.f, F = 0.f;
  uint32_t nh = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    if ((hm >> k) & 1u) {
      if (nh == 0) {
        F = run;
      } else {
        const uint32_t idx = hb + nh - 1;
        if (idx < hlim) hv[idx] = run;
      }
      ++nh;
      run = 0.f;
    }
    run += val[k];
  }
  if (nh == 0) F = run;
  // runs across lanes: segmented inclusive scan of the lanes' open partials
  float x = nh ? run : F;
  if (lane == 0 && nh == 0) x += csum;
  const uint32_t starts = __ballot_sync(0xffffffffu, nh != 0);
  const uint32_t le = starts & (0xffffffffu >> (31 - lane));
  const int seg0 = le ? 31 - __clz(le) : 0;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane - d >= seg0) x += y;
  }
  float prev = __shfl_up_sync(0xffffffffu, x, 1);
  if (lane == 0) prev = csum;
  // the run that ends just before this lane's first head (if a run is open)
  if (nh && hb > 0) {
    const uint32_t idx = hb - 1;
    if (idx < hlim) hv[idx] = prev + F;
  }
  csum = __shfl_sync(0xffffffffu, x, 31);
  cnt += htot;
}

// One warp, one segment: 256-edge steps (one 16-byte load per lane, the next
// step prefetched), source values from shared memory, runs reduced in
// registers and across lanes; every hub entry is written once, the run open
// at the end of a step carried to the next step.
__device__ __forceinline__ void oc_segment(const ArgsA& a, const float* __restrict__ csh,
                                           uint32_t q) {
  const int lane = threadIdx.x & 31;
  const uint64_t e0 = a.seg_e[q], e1 = a.seg_e[q + 1], h0 = a.seg_h[q];
  const uint64_t h1 = (q + 1 < a.nseg) ? a.seg_h[q + 1] : a.H;
  const uint32_t hlim = h1 > h0 ? (uint32_t)(h1 - h0) : 0u;  // entries of this segment
  float* hv = a.hub_val + h0;
  uint64_t base = e0 & ~7ull;
  uint4 nx = make_uint4(0, 0, 0, 0);
  {
    const uint64_t p = base + (uint64_t)lane * 8;
    if (p < e1) nx = __ldcs(reinterpret_cast<const uint4*>(a.ew + p));
  }
  uint32_t cnt = 0;  // hub entries started so far (> 0: a run is open)
  float csum = 0.f;  // the open run's partial sum
  while (base < e1) {
    const uint4 w = nx;
    const uint64_t nbase = base + 256;
    {
      const uint64_t p = nbase + (uint64_t)lane * 8;
      if (p < e1) nx = __ldcs(reinterpret_cast<const uint4*>(a.ew + p));
    }
    if (base >= e0 && nbase <= e1)
      oc_step<true>(w, base, e0, e1, csh, hv, hlim, cnt, csum);
    else
      oc_step<false>(w, base, e0, e1, csh, hv, hlim, cnt, csum);
    base = nbase;
  }
  if (lane == 0 && cnt && cnt - 1 < hlim) hv[cnt - 1] = csum;  // the segment's last run
}

__global__ void __launch_bounds__(kOcThreads, 1) k_oc_tohub(const __grid_constant__ ArgsA a) {
  extern __shared__ __align__(16) float csh[];
  const OcItemA it = a.items[blockIdx.x];
  const uint64_t v0 = (uint64_t)it.row << kOcSrcBits;
  const uint32_t len = (uint32_t)std::min<uint64_t>(kSrcLen, a.n - v0);
  // stage the source interval's contributions
  const uint32_t n4 = len / 4;
  const float4* src4 = reinterpret_cast<const float4*>(a.c_in + v0);
  float4* dst4 = reinterpret_cast<float4*>(csh);
  for (uint32_t k = threadIdx.x; k < n4; k += kOcThreads) dst4[k] = __ldg(src4 + k);
  for (uint32_t k = 4 * n4 + threadIdx.x; k < len; k += kOcThreads) csh[k] = a.c_in[v0 + k];
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  for (uint32_t q = it.s0 + warp; q < it.s1; q += kOcWarps) oc_segment(a, csh, q);
}

// ---------------------------------------------------------------- FromHub
struct ArgsB {
  const uint64_t* chunks;
  const OcItemB* items;
  const float* hub_val;
  const uint16_t* hub_dst;
  const uint32_t* outdeg;
  const float* tele;
  int dang_by_tele;
  float alpha;
  uint32_t n, PB;
  const double* dm_in;
  double* dm_out;
  double* part;      // [PB] dangling partial per column
  uint32_t* ticket;  // [0]: iteration; [1 + group]: split columns
  float* split;      // [slots][2 * kDstLen]
  float* r_out;
  float* c_out;
};

__device__ __forceinline__ void twosum_add(float* hi, float* lo, uint32_t k, float v) {
  const float old = atomicAdd(hi + k, v);
  const float s = old + v;
  const float bb = s - old;
  atomicAdd(lo + k, (old - (s - bb)) + (v - bb));
}

__global__ void __launch_bounds__(kOcThreads, 1) k_oc_fromhub(const __grid_constant__ ArgsB a) {
  extern __shared__ __align__(16) float acc[];  // hi [kDstLen], lo [kDstLen]
  float* hi = acc;
  float* lo = acc + kDstLen;
  __shared__ double red[kOcWarps];
  __shared__ int s_last;
  const OcItemB it = a.items[blockIdx.x];
  const uint64_t v0 = (uint64_t)it.col << kOcDstBits;
  const uint32_t T = (uint32_t)std::min<uint64_t>(kDstLen, a.n - v0);
  for (uint32_t k = threadIdx.x; k < kDstLen; k += kOcThreads) {
    hi[k] = 0.f;
    lo[k] = 0.f;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // a chunk (<= 256 entries): every lane issues its loads first, then folds
  static_assert(kChunk == 8 * 32, "eight entries per lane per chunk");
  // the warp's chunks are c0 + warp + 32 t; lane l loads the descriptor of
  // t = t0 + l for a batch of 32, handed out by shuffles; a chunk's loads are
  // all issued before its folds
  uint64_t batch = 0;
  for (uint32_t t = 0;; ++t) {
    const uint64_t c = (uint64_t)it.c0 + warp + (uint64_t)kOcWarps * t;
    if (c >= it.c1) break;
    if ((t & 31) == 0) {
      const uint64_t cl = c + (uint64_t)kOcWarps * lane;
      batch = cl < it.c1 ? a.chunks[cl] : 0ull;
    }
    const uint64_t ch = __shfl_sync(0xffffffffu, batch, t & 31);
    const uint64_t h0 = ch >> 32;
    const uint32_t len = (uint32_t)(ch & 0xFFFFFFFFull);
    uint32_t o[8];
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint32_t x = lane + 32 * q;
      o[q] = kDstLen;
      v[q] = 0.f;
      if (x < len) {
        o[q] = a.hub_dst[h0 + x];
        v[q] = __ldcs(a.hub_val + h0 + x);
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (o[q] < kDstLen) twosum_add(hi, lo, o[q], v[q]);
  }
  __syncthreads();
  if (it.nsplit > 1) {  // combine the blocks of a split column in slot order
    float* mine = a.split + (uint64_t)(it.slot + it.part) * 2 * kDstLen;
    for (uint32_t k = threadIdx.x; k < T; k += kOcThreads) {
      mine[k] = hi[k];
      mine[kDstLen + k] = lo[k];
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(a.ticket + 1 + it.group, 1u) == it.nsplit - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) a.ticket[1 + it.group] = 0;
    for (uint32_t k = threadIdx.x; k < T; k += kOcThreads) {
      double v = 0.0;
      for (uint32_t q = 0; q < it.nsplit; ++q) {
        const float* sq = a.split + (uint64_t)(it.slot + q) * 2 * kDstLen;
        v += (double)__ldcg(sq + k) + (double)__ldcg(sq + kDstLen + k);
      }
      const float h = (float)v;
      hi[k] = h;
      lo[k] = (float)(v - (double)h);
    }
    __syncthreads();
  }
  // epilogue: r' = (1-a) t + a (acc + Dm s), c' = r' / outdeg
  const float alpha = a.alpha;
  const float inv_n = 1.0f / (float)a.n;
  const float dm = (float)(*a.dm_in);
  double dpart = 0.0;
  for (uint32_t k = threadIdx.x; k < T; k += kOcThreads) {
    const uint64_t v = v0 + k;
    const float tv = a.tele ? a.tele[v] : inv_n;
    const float spread = a.dang_by_tele ? tv : inv_n;
    const float r = (1.0f - alpha) * tv + alpha * ((hi[k] + lo[k]) + dm * spread);
    a.r_out[v] = r;
    const uint32_t od = a.outdeg[v];
    a.c_out[v] = od ? r / (float)od : 0.0f;
    if (od == 0) dpart += (double)r;
  }
  for (int d = 16; d > 0; d >>= 1) dpart += __shfl_down_sync(0xffffffffu, dpart, d);
  if (lane == 0) red[warp] = dpart;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kOcWarps; ++q) t += red[q];
    a.part[it.col] = t;
    __threadfence();
    s_last = (atomicAdd(a.ticket, 1u) == a.PB - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // the last column of the iteration folds the dangling partials in order
  double t = 0.0;
  for (uint32_t q = threadIdx.x; q < a.PB; q += kOcThreads) t += __ldcg(a.part + q);
  for (int d = 16; d > 0; d >>= 1) t += __shfl_down_sync(0xffffffffu, t, d);
  __syncthreads();
  if (lane == 0) red[warp] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int q = 0; q < kOcWarps; ++q) tot += red[q];
    *a.dm_out = tot;
    *a.ticket = 0;
  }
}

}  // namespace

nx_status build_onchip(nx_graph* g, const uint32_t* s, const uint32_t* d, uint64_t m) {
  OnChip& oc = g->oc;
  const uint32_t n = g->geo.n;
  cudaStream_t st = stream();
  oc.m = m;
  oc.PA = (uint32_t)ceil_div(n, kSrcLen);
  oc.PB = (uint32_t)ceil_div(n, kDstLen);
  if ((uint64_t)oc.PA * oc.PB > (1ull << 26))
    return invalid("nx_build_dsss: NX_ONCHIP_HUBS supports n up to about 9.5e7 vertices");
  const uint64_t words = round_up(m, kEdgeAlign) + kEdgeAlign;  // 16-bit entries
  NX_TRY(oc.ew.alloc(words * 2));
  NX_CUDA(cudaMemsetAsync(oc.ew.p, 0, words * 2, st));
  std::vector<uint32_t> cnt((size_t)oc.PA * oc.PB, 0);
  std::vector<uint64_t> row_start(oc.PA + 1, 0);
  if (m) {
    DevBuf key, head, hidx, dcnt, drows, tot;
    NX_TRY(key.alloc(m * 8));
    k_oc_keys<<<grid_n(m), 256, 0, st>>>(s, d, m, key.as<uint64_t>());
    NX_LAUNCH_CHECK();
    NX_TRY(radix_sort_u64(key, nullptr, m, 45 + std::max<uint32_t>(1, bits_for(oc.PA))));
    NX_TRY(head.alloc(m * 4));
    k_oc_words<<<grid_n(m), 256, 0, st>>>(key.as<uint64_t>(), m, oc.ew.as<uint16_t>(),
                                          head.as<uint32_t>());
    NX_LAUNCH_CHECK();
    NX_TRY(hidx.alloc(m * 4));
    NX_TRY(tot.alloc(4));
    NX_TRY(exclusive_scan_u32(head.as<uint32_t>(), hidx.as<uint32_t>(), m, tot.as<uint32_t>()));
    uint32_t H = 0;
    NX_CUDA(cudaMemcpyAsync(&H, tot.p, 4, cudaMemcpyDeviceToHost, st));
    NX_CUDA(cudaStreamSynchronize(st));
    oc.H = H;
    NX_TRY(oc.hub_dst.alloc(std::max<uint64_t>(H, 1) * 2));
    NX_TRY(oc.hub_val.alloc(std::max<uint64_t>(H, 1) * 4));
    NX_TRY(dcnt.alloc(cnt.size() * 4));
    NX_CUDA(cudaMemsetAsync(dcnt.p, 0, cnt.size() * 4, st));
    k_oc_hubs<<<grid_n(m), 256, 0, st>>>(key.as<uint64_t>(), head.as<uint32_t>(),
                                         hidx.as<uint32_t>(), m, oc.PB, oc.hub_dst.as<uint16_t>(),
                                         dcnt.as<uint32_t>());
    NX_LAUNCH_CHECK();
    NX_TRY(drows.alloc(((size_t)oc.PA + 1) * 8));
    k_oc_row_starts<<<(unsigned)ceil_div(oc.PA + 1, 256), 256, 0, st>>>(key.as<uint64_t>(), m, oc.PA,
                                                                        drows.as<uint64_t>());
    NX_LAUNCH_CHECK();
    NX_CUDA(cudaMemcpyAsync(cnt.data(), dcnt.p, cnt.size() * 4, cudaMemcpyDeviceToHost, st));
    NX_CUDA(cudaMemcpyAsync(row_start.data(), drows.p, row_start.size() * 8, cudaMemcpyDeviceToHost, st));
    NX_CUDA(cudaStreamSynchronize(st));
    key.release();
    head.release();
    // segments: windows between multiples of kOcSeg and row starts
    std::vector<uint64_t> seg_e;
    std::vector<OcItemA> items_a;
    for (uint32_t r = 0; r < oc.PA; ++r) {
      const uint64_t rs = row_start[r], re = row_start[r + 1];
      uint32_t first = (uint32_t)seg_e.size();
      for (uint64_t e = rs; e < re;) {
        seg_e.push_back(e);
        e = std::min<uint64_t>(re, (e / kOcSeg + 1) * kOcSeg);
      }
      const uint32_t last = (uint32_t)seg_e.size();
      for (uint32_t q = first; q < last; q += kSegsPerItem)
        items_a.push_back(OcItemA{r, q, std::min<uint32_t>(last, q + kSegsPerItem), 0});
    }
    oc.nseg = (uint32_t)seg_e.size();
    seg_e.push_back(m);
    NX_TRY(oc.seg_e.alloc(seg_e.size() * 8));
    NX_TRY(oc.seg_h.alloc(std::max<size_t>(oc.nseg, 1) * 8));
    NX_CUDA(cudaMemcpyAsync(oc.seg_e.p, seg_e.data(), seg_e.size() * 8, cudaMemcpyHostToDevice, st));
    k_oc_seg_hub<<<(unsigned)ceil_div(std::max<uint32_t>(oc.nseg, 1), 256), 256, 0, st>>>(
        oc.seg_e.as<uint64_t>(), oc.nseg, hidx.as<uint32_t>(), oc.seg_h.as<uint64_t>());
    NX_LAUNCH_CHECK();
    // largest first (each block stages its row's 128 KB once, whatever its length)
    std::stable_sort(items_a.begin(), items_a.end(), [&](const OcItemA& x, const OcItemA& y) {
      return seg_e[x.s1] - seg_e[x.s0] > seg_e[y.s1] - seg_e[y.s0];
    });
    oc.na = (uint32_t)items_a.size();
    NX_TRY(oc.items_a.alloc(std::max<size_t>(items_a.size(), 1) * sizeof(OcItemA)));
    if (!items_a.empty())
      NX_CUDA(cudaMemcpyAsync(oc.items_a.p, items_a.data(), items_a.size() * sizeof(OcItemA),
                              cudaMemcpyHostToDevice, st));
    NX_CUDA(cudaStreamSynchronize(st));  // host vectors and hidx are released below
  }
  // FromHub: the nonempty pieces of each column as chunks of <= kChunk entries
  // (hub entries are ordered row-major, so piece (i, j) starts at the
  // row-major prefix of the counts), and work items that split heavy columns
  std::vector<uint64_t> start(cnt.size());
  {
    uint64_t acc = 0;
    for (size_t q = 0; q < cnt.size(); ++q) {
      start[q] = acc;
      acc += cnt[q];
    }
  }
  std::vector<uint64_t> chunks;
  std::vector<uint32_t> col_c0(oc.PB + 1, 0);
  std::vector<uint64_t> col_tot(oc.PB, 0);
  for (uint32_t j = 0; j < oc.PB; ++j) {
    col_c0[j] = (uint32_t)chunks.size();
    for (uint32_t i = 0; i < oc.PA; ++i) {
      const size_t q = (size_t)i * oc.PB + j;
      for (uint64_t x = 0; x < cnt[q]; x += kChunk) {
        const uint64_t len = std::min<uint64_t>(kChunk, cnt[q] - x);
        chunks.push_back(((start[q] + x) << 32) | len);
      }
      col_tot[j] += cnt[q];
    }
  }
  col_c0[oc.PB] = (uint32_t)chunks.size();
  oc.nchunks = chunks.size();
  const uint64_t target = std::max<uint64_t>(1u << 16, oc.H / ((uint64_t)num_sms() * 2));
  std::vector<OcItemB> items_b;
  uint32_t slots = 0, groups = 0;
  for (uint32_t j = 0; j < oc.PB; ++j) {
    const uint32_t c0 = col_c0[j], c1 = col_c0[j + 1];
    const uint32_t k = (uint32_t)std::max<uint64_t>(
        1, std::min<uint64_t>(c1 - c0, ceil_div(col_tot[j], target)));
    if (k == 1) {
      items_b.push_back(OcItemB{j, c0, c1, 1, 0, 0, 0, 0});
      continue;
    }
    // k parts with about equal entries (chunk boundaries)
    uint64_t acc = 0;
    uint32_t part = 0, cs = c0;
    for (uint32_t c = c0; c < c1 && part + 1 < k; ++c) {
      acc += chunks[c] & 0xFFFFFFFFull;
      if (acc * k >= col_tot[j] * (part + 1)) {
        items_b.push_back(OcItemB{j, cs, c + 1, k, part, slots, groups, 0});
        cs = c + 1;
        ++part;
      }
    }
    while (part < k) {  // the rest (and any empty parts)
      items_b.push_back(OcItemB{j, cs, c1, k, part, slots, groups, 0});
      cs = c1;
      ++part;
    }
    slots += k;
    ++groups;
  }
  {  // heaviest work first
    std::vector<std::pair<uint64_t, OcItemB>> w(items_b.size());
    for (size_t q = 0; q < items_b.size(); ++q) {
      uint64_t e = 0;
      for (uint32_t c = items_b[q].c0; c < items_b[q].c1; ++c) e += chunks[c] & 0xFFFFFFFFull;
      w[q] = {e, items_b[q]};
    }
    std::stable_sort(w.begin(), w.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    for (size_t q = 0; q < w.size(); ++q) items_b[q] = w[q].second;
  }
  oc.nb = (uint32_t)items_b.size();
  oc.slots = slots;
  oc.groups = groups;
  NX_TRY(oc.chunks.alloc(std::max<size_t>(chunks.size(), 1) * 8));
  if (!chunks.empty())
    NX_CUDA(cudaMemcpyAsync(oc.chunks.p, chunks.data(), chunks.size() * 8, cudaMemcpyHostToDevice, st));
  NX_TRY(oc.items_b.alloc(std::max<size_t>(items_b.size(), 1) * sizeof(OcItemB)));
  NX_CUDA(cudaMemcpyAsync(oc.items_b.p, items_b.data(), items_b.size() * sizeof(OcItemB),
                          cudaMemcpyHostToDevice, st));
  NX_TRY(oc.split.alloc(std::max<uint64_t>(slots, 1) * 2 * kDstLen * 4));
  NX_TRY(oc.ticket.alloc((1 + (size_t)groups) * 4));
  NX_CUDA(cudaMemsetAsync(oc.ticket.p, 0, (1 + (size_t)groups) * 4, st));
  NX_TRY(oc.part.alloc((size_t)oc.PB * 8));
  NX_CUDA(cudaStreamSynchronize(st));
  oc.built = true;
  return NX_OK;
}

nx_status onchip_iteration(nx_graph* g, const OcRun& r, cudaStream_t s) {
  const OnChip& oc = g->oc;
  const size_t smem_a = kSrcLen * 4, smem_b = 2 * kDstLen * 4;
  // 128 KB of dynamic shared memory each (per device; cheap to repeat)
  NX_CUDA(cudaFuncSetAttribute(k_oc_tohub, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_a));
  NX_CUDA(cudaFuncSetAttribute(k_oc_fromhub, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b));
  if (oc.na) {
    ArgsA a{};
    a.ew = oc.ew.as<uint16_t>();
    a.seg_e = oc.seg_e.as<uint64_t>();
    a.seg_h = oc.seg_h.as<uint64_t>();
    a.items = oc.items_a.as<OcItemA>();
    a.c_in = r.c_in;
    a.hub_val = oc.hub_val.as<float>();
    a.H = oc.H;
    a.n = g->geo.n;
    a.nseg = oc.nseg;
    k_oc_tohub<<<oc.na, kOcThreads, smem_a, s>>>(a);
    NX_LAUNCH_CHECK();
  }
  ArgsB b{};
  b.chunks = oc.chunks.as<uint64_t>();
  b.items = oc.items_b.as<OcItemB>();
  b.hub_val = oc.hub_val.as<float>();
  b.hub_dst = oc.hub_dst.as<uint16_t>();
  b.outdeg = g->outdeg.as<uint32_t>();
  b.tele = r.tele;
  b.dang_by_tele = r.dang_by_tele;
  b.alpha = r.alpha;
  b.n = g->geo.n;
  b.PB = oc.PB;
  b.dm_in = r.dm_in;
  b.dm_out = r.dm_out;
  b.part = oc.part.as<double>();
  b.ticket = oc.ticket.as<uint32_t>();
  b.split = oc.split.as<float>();
  b.r_out = r.r_out;
  b.c_out = r.c_out;
  k_oc_fromhub<<<oc.nb, kOcThreads, smem_b, s>>>(b);
  NX_LAUNCH_CHECK();
  return NX_OK;
}

}  // namespace nx
