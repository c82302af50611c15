// Error state, buffers, and the device-wide primitives the DSSS builder uses:
// exclusive scans and a stable LSD radix sort of 64-bit keys. All written for
// this library (no CUB / Thrust).
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <atomic>
#include <mutex>

#include "nx_internal.cuh"

namespace nx {

// ---------------------------------------------------------------- errors
static thread_local std::string t_err;
void set_error(const std::string& msg) { t_err = msg; }
const char* get_error() { return t_err.c_str(); }

nx_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof buf, "CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e),
           what, file, line);
  set_error(buf);
  if (e == cudaErrorMemoryAllocation) return NX_ERR_OOM;
  return NX_ERR_CUDA;
}

nx_status invalid(const std::string& msg) {
  set_error(msg);
  return NX_ERR_INVALID_ARG;
}

// ---------------------------------------------------------------- stream
static cudaStream_t g_stream = nullptr;
cudaStream_t stream() { return g_stream; }

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || !sms)
      sms = 148;
  }
  return sms;
}

// ---------------------------------------------------------------- buffers
// The pool keeps freed memory for reuse, up to half of the device's memory
// (graphs built and run one after another reuse it instead of mapping new
// pages: at R-MAT scale 26 a build and its first run allocate about 40 GB of
// temporaries); memory above that goes back to the driver at the next
// synchronisation, and nx_trim_memory() returns all of it.
static std::mutex g_pool_mu;
static cudaMemPool_t g_pools[64] = {};

static cudaError_t pool_of_current_device(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pools[dev]) {
    size_t free_b = 0, total_b = 0;
    e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) return e;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    e = cudaMemPoolCreate(&g_pools[dev], &props);
    if (e != cudaSuccess) {
      g_pools[dev] = nullptr;
      return e;
    }
    uint64_t keep = total_b / 2;
    e = cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) return e;
  }
  *out = g_pools[dev];
  return cudaSuccess;
}

void DevBuf::release() {
  if (p) {
    if (!pooled) {
      cudaFree(p);
    } else {
      if (owner != stream()) cudaDeviceSynchronize();  // the allocating stream may still use it
      cudaFreeAsync(p, stream());
    }
  }
  p = nullptr;
  bytes = 0;
}
// nx_debug_fail_alloc: allocations left before the injected failure (-1: off)
static std::atomic<long long> g_fail_after{-1};

nx_status DevBuf::alloc(size_t n) {
  release();
  if (n == 0) return NX_OK;
  if (g_fail_after.load() >= 0 && g_fail_after.fetch_sub(1) == 0) {
    g_fail_after.store(-1);
    set_error("device allocation failed: injected by nx_debug_fail_alloc");
    return NX_ERR_OOM;
  }
  cudaMemPool_t pool = nullptr;
  cudaError_t e = pool_of_current_device(&pool);
  pooled = (e == cudaSuccess);
  if (pooled) {
    e = cudaMallocFromPoolAsync(&p, n, pool, stream());
  } else {
    cudaGetLastError();
    e = cudaMalloc(&p, n);
  }
  owner = stream();
  if (e != cudaSuccess) {
    p = nullptr;
    cudaGetLastError();
    char buf[160];
    snprintf(buf, sizeof buf, "device allocation of %zu bytes failed: %s", n,
             cudaGetErrorString(e));
    set_error(buf);
    return NX_ERR_OOM;
  }
  bytes = n;
  return NX_OK;
}
static std::mutex g_pinned_mu;
static std::vector<std::pair<void*, size_t>> g_pinned_free;  // cached blocks
static size_t g_pinned_cached = 0;
constexpr size_t kPinnedCacheMax = 512ull << 20;

void* pinned_take(size_t bytes, size_t* got) {
  bytes = std::max<size_t>(bytes, 64);
  {
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    for (size_t q = 0; q < g_pinned_free.size(); ++q) {
      const auto blk = g_pinned_free[q];
      if (blk.second >= bytes && blk.second <= 2 * bytes) {
        g_pinned_free.erase(g_pinned_free.begin() + q);
        g_pinned_cached -= blk.second;
        *got = blk.second;
        return blk.first;
      }
    }
  }
  void* p = nullptr;
  if (cudaMallocHost(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    char buf[160];
    snprintf(buf, sizeof buf, "pinned host allocation of %zu bytes failed", bytes);
    set_error(buf);
    return nullptr;
  }
  *got = bytes;
  return p;
}

void pinned_give(void* p, size_t bytes) {
  if (!p) return;
  {
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    if (g_pinned_cached + bytes <= kPinnedCacheMax) {
      g_pinned_free.push_back({p, bytes});
      g_pinned_cached += bytes;
      return;
    }
  }
  cudaFreeHost(p);
}

void PinnedBuf::release() {
  if (p) cudaFreeHost(p);
  p = nullptr;
  bytes = 0;
}
nx_status PinnedBuf::alloc(size_t n) {
  release();
  if (n == 0) return NX_OK;
  cudaError_t e = cudaMallocHost(&p, n);
  if (e != cudaSuccess) {
    p = nullptr;
    cudaGetLastError();
    char buf[160];
    snprintf(buf, sizeof buf, "pinned host allocation of %zu bytes failed: %s", n,
             cudaGetErrorString(e));
    set_error(buf);
    return NX_ERR_OOM;
  }
  bytes = n;
  return NX_OK;
}

nx_status EventPair::create() {
  NX_CUDA(cudaEventCreate(&e0));
  NX_CUDA(cudaEventCreate(&e1));
  return NX_OK;
}
nx_status EventPair::elapsed(float* ms) {
  NX_CUDA(cudaEventSynchronize(e1));
  NX_CUDA(cudaEventElapsedTime(ms, e0, e1));
  return NX_OK;
}

// ---------------------------------------------------------------- scan
namespace {
constexpr int SC_THREADS = 256;
constexpr int SC_ITEMS = 8;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

template <class T>
__device__ T block_exclusive(T v, T* total) {
  __shared__ T warp_tot[SC_THREADS / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    T t = lane < SC_THREADS / 32 ? warp_tot[lane] : T(0);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, t, d);
      if (lane >= d) t += y;
    }
    if (lane < SC_THREADS / 32) warp_tot[lane] = t;
  }
  __syncthreads();
  T before = (w > 0 ? warp_tot[w - 1] : T(0)) + x - v;
  if (total) *total = warp_tot[SC_THREADS / 32 - 1];
  __syncthreads();
  return before;
}

template <class T>
__global__ void scan_reduce(const T* in, uint64_t n, T* part) {
  uint64_t base = (uint64_t)blockIdx.x * SC_TILE + (uint64_t)threadIdx.x * SC_ITEMS;
  T s = 0;
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k)
    if (base + k < n) s += in[base + k];
  T tot;
  block_exclusive<T>(s, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

template <class T>
__global__ void scan_tiles(const T* in, T* out, uint64_t n, const T* part_scanned, T* total) {
  uint64_t base = (uint64_t)blockIdx.x * SC_TILE + (uint64_t)threadIdx.x * SC_ITEMS;
  T v[SC_ITEMS];
  T s = 0;
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k) {
    v[k] = base + k < n ? in[base + k] : T(0);
    s += v[k];
  }
  T tot;
  T run = block_exclusive<T>(s, &tot) + (part_scanned ? part_scanned[blockIdx.x] : T(0));
#pragma unroll
  for (int k = 0; k < SC_ITEMS; ++k)
    if (base + k < n) {
      out[base + k] = run;
      run += v[k];
    }
  if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
    *total = (part_scanned ? part_scanned[blockIdx.x] : T(0)) + tot;
}

template <class T>
nx_status exclusive_scan(const T* in, T* out, uint64_t n, T* total) {
  if (n == 0) {
    if (total) NX_CUDA(cudaMemsetAsync(total, 0, sizeof(T), stream()));
    return NX_OK;
  }
  uint64_t nb = ceil_div(n, SC_TILE);
  if (nb == 1) {
    scan_tiles<T><<<1, SC_THREADS, 0, stream()>>>(in, out, n, nullptr, total);
    NX_LAUNCH_CHECK();
    return NX_OK;
  }
  DevBuf part;
  NX_TRY(part.alloc(nb * sizeof(T)));
  scan_reduce<T><<<(unsigned)nb, SC_THREADS, 0, stream()>>>(in, n, part.as<T>());
  NX_LAUNCH_CHECK();
  NX_TRY(exclusive_scan<T>(part.as<T>(), part.as<T>(), nb, nullptr));
  scan_tiles<T><<<(unsigned)nb, SC_THREADS, 0, stream()>>>(in, out, n, part.as<T>(), total);
  NX_LAUNCH_CHECK();
  NX_CUDA(cudaStreamSynchronize(stream()));  // `part` is freed on return
  return NX_OK;
}
}  // namespace

nx_status exclusive_scan_u32(const uint32_t* in, uint32_t* out, uint64_t n, uint32_t* total) {
  return exclusive_scan<uint32_t>(in, out, n, total);
}
nx_status exclusive_scan_u64(const uint64_t* in, uint64_t* out, uint64_t n, uint64_t* total) {
  return exclusive_scan<uint64_t>(in, out, n, total);
}

// ---------------------------------------------------------------- L1 carveout
// Smallest shared-memory carveout that still holds the blocks of `fn` an SM
// can run with `smem` bytes of dynamic shared memory, so the rest of the
// unified L1 caches global loads. Computed once per (device, kernel, size)
// with the whole unified memory offered to shared memory, and re-applied
// whenever the size in use for the kernel changes.
nx_status prefer_l1(const void* fn, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, size_t>, int> pct_of;
  static std::map<std::pair<int, const void*>, int> applied;
  int dev = 0;
  NX_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_tuple(dev, fn, smem);
  auto hit = pct_of.find(key);
  if (hit == pct_of.end()) {
    NX_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    applied[std::make_pair(dev, fn)] = 100;
    int nb = 0, per_sm = 0;
    cudaFuncAttributes fa;
    NX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem));
    NX_CUDA(cudaFuncGetAttributes(&fa, fn));
    NX_CUDA(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    int pct = 100;
    if (nb > 0 && per_sm > 0) {
      const uint64_t need = (uint64_t)nb * (smem + fa.sharedSizeBytes + 1024);  // 1 KB reserved per block
      pct = (int)std::min<uint64_t>(100, ceil_div(100 * need, (uint64_t)per_sm));
    }
    hit = pct_of.emplace(key, pct).first;
  }
  int& cur = applied[std::make_pair(dev, fn)];
  if (cur != hit->second) {
    NX_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, hit->second));
    cur = hit->second;
  }
  return NX_OK;
}

// ---------------------------------------------------------------- radix sort
// Stable LSD radix sort in passes of at most 9 bits: per pass one kernel
// counts each tile's digits, a scan turns the counts into the first output
// slot of every (digit, tile), and one kernel ranks and scatters each tile.
namespace {
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 16;                     // keys per lane
constexpr int RS_WARP_KEYS = 32 * RS_ROUNDS;      // 512
constexpr int RS_TILE = RS_WARPS * RS_WARP_KEYS;  // 4096
constexpr uint32_t RS_MAX_BITS = 9;

// counts[d * nb + tile] = keys of the tile whose digit (key >> shift) & mask is d.
template <int BITS>
__global__ void __launch_bounds__(RS_THREADS) rs_hist(const uint64_t* __restrict__ keys, uint64_t n,
                                                      uint32_t shift, uint32_t mask,
                                                      uint32_t* __restrict__ counts, uint32_t nb) {
  constexpr int NB = 1 << BITS;
  __shared__ uint32_t h[RS_WARPS][NB];
  for (int k = threadIdx.x; k < RS_WARPS * NB; k += RS_THREADS) (&h[0][0])[k] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint64_t base = (uint64_t)blockIdx.x * RS_TILE + (uint64_t)w * RS_WARP_KEYS + lane;
  uint64_t k[RS_ROUNDS];
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {  // every load in flight before the first count
    const uint64_t idx = base + (uint64_t)r * 32;
    k[r] = idx < n ? keys[idx] : ~0ull;
  }
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r)
    if (base + (uint64_t)r * 32 < n) atomicAdd(&h[w][(uint32_t)(k[r] >> shift) & mask], 1u);
  __syncthreads();
  for (uint32_t d = threadIdx.x; d <= mask; d += RS_THREADS) {
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < RS_WARPS; ++q) s += h[q][d];
    counts[(uint64_t)d * nb + blockIdx.x] = s;
  }
}

// Lanes of the warp whose NBITS-bit value d equals this lane's, from one
// ballot per bit.
template <int NBITS>
__device__ __forceinline__ uint32_t rs_peers(uint32_t d) {
  uint32_t peers = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < NBITS; ++b) {
    const bool bit = (d >> b) & 1u;
    const uint32_t bal = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? bal : ~bal;
  }
  return peers;
}

// Stable scatter of one digit of at most BITS bits. Keys are ranked per warp
// (lane order within a round, rounds in order, warps in order = input order),
// placed in shared memory in digit order, and written out from there so that
// consecutive threads store consecutive addresses of one digit's run.
// Dynamic shared memory: RS_TILE keys (+ RS_TILE values when vin != nullptr).
template <int BITS>
__global__ void __launch_bounds__(RS_THREADS) rs_scatter(
    const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint64_t* __restrict__ kout,
    uint32_t* __restrict__ vout, uint64_t n, uint32_t shift, uint32_t mask,
    const uint32_t* __restrict__ offs, uint32_t nb) {
  constexpr int NB = 1 << BITS;
  constexpr int PER = NB / RS_THREADS > 0 ? NB / RS_THREADS : 1;  // digits per thread
  static_assert(NB <= RS_THREADS * PER, "digit tables");
  extern __shared__ __align__(16) unsigned char rs_smem[];
  uint64_t* sk = reinterpret_cast<uint64_t*>(rs_smem);       // [RS_TILE]
  uint32_t* sv = reinterpret_cast<uint32_t*>(sk + RS_TILE);  // [RS_TILE] (values)
  __shared__ uint32_t wc[RS_WARPS][NB + 1];
  __shared__ uint32_t dstart[NB];  // first local slot of each digit
  __shared__ uint32_t gbase[NB];   // first global slot of this block's run of each digit
  __shared__ uint32_t wsum[RS_WARPS];
  for (int k = threadIdx.x; k < RS_WARPS * (NB + 1); k += RS_THREADS) (&wc[0][0])[k] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  const uint64_t tile0 = (uint64_t)blockIdx.x * RS_TILE;
  const uint64_t base = tile0 + (uint64_t)w * RS_WARP_KEYS + lane;
  const uint32_t cnt = (uint32_t)((n - tile0) < (uint64_t)RS_TILE ? (n - tile0) : (uint64_t)RS_TILE);
  uint64_t key[RS_ROUNDS];
  uint32_t rank[RS_ROUNDS];
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    uint64_t idx = base + (uint64_t)r * 32;
    bool valid = idx < n;
    key[r] = valid ? kin[idx] : 0ull;
    uint32_t d = valid ? ((uint32_t)(key[r] >> shift) & mask) : (uint32_t)NB;
    // the match pipe for one round in three, one ballot per bit otherwise:
    // either alone saturates its pipe
    uint32_t peers = (r % 3) ? rs_peers<BITS + 1>(d) : __match_any_sync(0xffffffffu, d);
    uint32_t before = wc[w][d];
    __syncwarp();
    if ((peers & lt_mask) == 0) wc[w][d] = before + __popc(peers);
    __syncwarp();
    rank[r] = before + __popc(peers & lt_mask);
  }
  __syncthreads();
  // per digit: block total, then per-warp starts inside the digit's local run
  uint32_t tot[PER];
  uint32_t tsum = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const uint32_t d = threadIdx.x * PER + q;
    tot[q] = 0;
    if (d < (uint32_t)NB) {
#pragma unroll
      for (int v = 0; v < RS_WARPS; ++v) tot[q] += wc[v][d];
      gbase[d] = d <= mask ? offs[(uint64_t)d * nb + blockIdx.x] : 0u;
    }
    tsum += tot[q];
  }
  // exclusive scan of the per-thread sums (digits in thread order)
  uint32_t x = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  uint32_t pre = 0;
  for (int q = 0; q < w; ++q) pre += wsum[q];
  uint32_t st = pre + x - tsum;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const uint32_t d = threadIdx.x * PER + q;
    if (d < (uint32_t)NB) {
      dstart[d] = st;
#pragma unroll
      for (int v = 0; v < RS_WARPS; ++v) {
        const uint32_t t = wc[v][d];
        wc[v][d] = st;
        st += t;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_ROUNDS; ++r) {
    uint64_t idx = base + (uint64_t)r * 32;
    if (idx < n) {
      const uint32_t d = (uint32_t)(key[r] >> shift) & mask;
      const uint32_t lp = wc[w][d] + rank[r];
      sk[lp] = key[r];
      if (vin) sv[lp] = vin[idx];
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < cnt; i += RS_THREADS) {
    const uint64_t k = sk[i];
    const uint32_t d = (uint32_t)(k >> shift) & mask;
    const uint32_t pos = gbase[d] + (i - dstart[d]);
    kout[pos] = k;
    if (vin) vout[pos] = sv[i];
  }
}
}  // namespace

uint64_t radix_sort_count_words(uint64_t n) {
  return ceil_div(std::max<uint64_t>(n, 1), RS_TILE) << RS_MAX_BITS;
}

nx_status radix_sort_u64_raw(uint64_t* a, uint64_t* b, uint32_t* va, uint32_t* vb, uint32_t* counts,
                             uint64_t n, uint32_t key_bits, bool* in_b) {
  *in_b = false;
  if (n <= 1 || key_bits == 0) return NX_OK;
  if (n >= (1ull << 32)) return invalid("radix_sort_u64: n must be < 2^32");
  key_bits = std::min<uint32_t>(key_bits, 64);
  const uint32_t nb = (uint32_t)ceil_div(n, RS_TILE);
  // passes of at most 9 bits, as even as possible (52 bits: 9,9,9,9,8,8)
  const uint32_t npass = (key_bits + RS_MAX_BITS - 1) / RS_MAX_BITS;
  const size_t smem = (size_t)RS_TILE * (sizeof(uint64_t) + (va ? sizeof(uint32_t) : 0));
  // dynamic + static shared memory exceed 48 KB: opt in (per device, so every call)
  NX_CUDA(cudaFuncSetAttribute(rs_scatter<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  NX_CUDA(cudaFuncSetAttribute(rs_scatter<9>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  uint64_t* ka = a;
  uint64_t* kb = b;
  uint32_t* vx = va;
  uint32_t* vy = vb;
  uint32_t shift = 0;
  for (uint32_t p = 0; p < npass; ++p) {
    const uint32_t width = key_bits / npass + (p < key_bits % npass ? 1u : 0u);
    const uint32_t mask = (1u << width) - 1u;
    const uint64_t nc = (uint64_t)nb << width;
    if (width > 8) {
      rs_hist<9><<<nb, RS_THREADS, 0, stream()>>>(ka, n, shift, mask, counts, nb);
    } else {
      rs_hist<8><<<nb, RS_THREADS, 0, stream()>>>(ka, n, shift, mask, counts, nb);
    }
    NX_LAUNCH_CHECK();
    NX_TRY(exclusive_scan_u32(counts, counts, nc, nullptr));
    if (width > 8) {
      rs_scatter<9><<<nb, RS_THREADS, smem, stream()>>>(ka, vx, kb, vy, n, shift, mask, counts, nb);
    } else {
      rs_scatter<8><<<nb, RS_THREADS, smem, stream()>>>(ka, vx, kb, vy, n, shift, mask, counts, nb);
    }
    NX_LAUNCH_CHECK();
    std::swap(ka, kb);
    std::swap(vx, vy);
    shift += width;
  }
  *in_b = (npass & 1) != 0;
  return NX_OK;
}

nx_status radix_sort_u64(DevBuf& keys, DevBuf* vals, uint64_t n, uint32_t key_bits) {
  if (n <= 1 || key_bits == 0) return NX_OK;
  DevBuf k2, v2, counts;
  NX_TRY(k2.alloc(n * sizeof(uint64_t)));
  if (vals) NX_TRY(v2.alloc(n * sizeof(uint32_t)));
  NX_TRY(counts.alloc(radix_sort_count_words(n) * sizeof(uint32_t)));
  bool in_b = false;
  NX_TRY(radix_sort_u64_raw(keys.as<uint64_t>(), k2.as<uint64_t>(), vals ? vals->as<uint32_t>() : nullptr,
                            vals ? v2.as<uint32_t>() : nullptr, counts.as<uint32_t>(), n, key_bits,
                            &in_b));
  if (in_b) {  // the result sits in the scratch buffers: hand them to the caller
    std::swap(keys, k2);
    if (vals) std::swap(*vals, v2);
  }
  // scratch is freed on return: make sure the stream is done with it
  NX_CUDA(cudaStreamSynchronize(stream()));
  return NX_OK;
}

// ---------------------------------------------------------------- merge
// Stable merge of two sorted runs (ties: the first run's keys first) by merge
// path: a partition pass finds, for every output tile of MG_TILE keys, how
// many of its predecessors come from the first run (a binary search along the
// tile's cross diagonal); each block then stages its tile's inputs in shared
// memory, each thread finds its own split there and merges MG_ITEMS keys
// (keeping the two candidate keys in registers, so one shared load per key),
// and the block writes the tile out in order. Shared memory holds one spare
// slot per 16 keys, so the threads' strided stores of their MG_ITEMS results
// (and the warps' linear reads) hit 16 distinct 8-byte bank pairs.
constexpr int MG_THREADS = 256;
constexpr int MG_ITEMS = 8;
constexpr int MG_TILE = MG_THREADS * MG_ITEMS;  // 2048

__device__ __forceinline__ uint32_t mg_pad(uint32_t x) { return x + (x >> 4); }

// Keys of `a` among the first `diag` outputs.
template <class I>
__device__ __forceinline__ I merge_split(const uint64_t* a, I na, const uint64_t* b, I nb, I diag) {
  I lo = diag > nb ? diag - nb : 0, hi = diag < na ? diag : na;
  while (lo < hi) {
    const I mid = (lo + hi) >> 1;
    if (a[mid] <= b[diag - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__global__ void k_merge_part(const uint64_t* __restrict__ a, uint64_t na, const uint64_t* __restrict__ b,
                             uint64_t nb, uint64_t ntiles, uint64_t* __restrict__ split) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= ntiles; t += stride)
    split[t] = merge_split<uint64_t>(a, na, b, nb, std::min<uint64_t>(t * MG_TILE, na + nb));
}

__global__ void __launch_bounds__(MG_THREADS) k_merge(const uint64_t* __restrict__ a, uint64_t na,
                                                      const uint64_t* __restrict__ b, uint64_t nb,
                                                      const uint64_t* __restrict__ split,
                                                      uint64_t* __restrict__ out) {
  __shared__ uint64_t sm[MG_TILE + MG_TILE / 16];
  const uint64_t k0 = (uint64_t)blockIdx.x * MG_TILE;
  const uint64_t k1 = std::min<uint64_t>(k0 + MG_TILE, na + nb);
  const uint64_t a0 = split[blockIdx.x], a1 = split[blockIdx.x + 1];
  const uint64_t b0 = k0 - a0, b1 = k1 - a1;
  const uint32_t la = (uint32_t)(a1 - a0), lb = (uint32_t)(b1 - b0), cnt = la + lb;
  for (uint32_t x = threadIdx.x; x < la; x += MG_THREADS) sm[mg_pad(x)] = a[a0 + x];
  for (uint32_t x = threadIdx.x; x < lb; x += MG_THREADS) sm[mg_pad(la + x)] = b[b0 + x];
  __syncthreads();
  const uint32_t diag = std::min<uint32_t>(threadIdx.x * MG_ITEMS, cnt);
  uint32_t i, j;
  {  // this thread's split: binary search along its diagonal
    uint32_t lo = diag > lb ? diag - lb : 0, hi = diag < la ? diag : la;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (sm[mg_pad(mid)] <= sm[mg_pad(la + diag - 1 - mid)]) lo = mid + 1;
      else hi = mid;
    }
    i = lo;
    j = diag - lo;
  }
  uint64_t va = i < la ? sm[mg_pad(i)] : 0ull, vb = j < lb ? sm[mg_pad(la + j)] : 0ull;
  uint64_t v[MG_ITEMS];
#pragma unroll
  for (int q = 0; q < MG_ITEMS; ++q) {
    const bool take_a = i < la && (j >= lb || va <= vb);
    v[q] = take_a ? va : vb;
    i += take_a ? 1u : 0u;
    j += take_a ? 0u : 1u;
    // the next key of the run just taken (one shared load)
    const uint32_t nx = take_a ? i : la + j;
    const bool more = take_a ? i < la : j < lb;
    const uint64_t y = more ? sm[mg_pad(nx)] : 0ull;
    va = take_a ? y : va;
    vb = take_a ? vb : y;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < MG_ITEMS; ++q)
    if (diag + q < cnt) sm[mg_pad(diag + q)] = v[q];
  __syncthreads();
  for (uint32_t x = threadIdx.x; x < cnt; x += MG_THREADS) out[k0 + x] = sm[mg_pad(x)];
}

nx_status merge_u64(const uint64_t* a, uint64_t na, const uint64_t* b, uint64_t nb, uint64_t* out,
                    uint64_t* split) {
  const uint64_t total = na + nb;
  if (!total) return NX_OK;
  const uint64_t ntiles = ceil_div(total, MG_TILE);
  if (ntiles >= (1ull << 31)) return invalid("merge_u64: too many keys");
  k_merge_part<<<(unsigned)std::min<uint64_t>(ceil_div(ntiles + 1, 256), (uint64_t)num_sms() * 16), 256, 0,
                 stream()>>>(a, na, b, nb, ntiles, split);
  NX_LAUNCH_CHECK();
  k_merge<<<(unsigned)ntiles, MG_THREADS, 0, stream()>>>(a, na, b, nb, split, out);
  NX_LAUNCH_CHECK();
  return NX_OK;
}

uint64_t merge_split_words(uint64_t n) { return ceil_div(std::max<uint64_t>(n, 1), MG_TILE) + 2; }

nx_status RunMerger::init(DevBuf& k, uint64_t n) {
  keys = &k;
  st.clear();
  NX_TRY(tmp.alloc(std::max<uint64_t>(n, 1) * sizeof(uint64_t)));
  NX_TRY(split.alloc(merge_split_words(n) * sizeof(uint64_t)));
  return NX_OK;
}

nx_status RunMerger::merge_top() {
  const Run b = st.back();
  st.pop_back();
  const Run a = st.back();
  st.pop_back();
  DevBuf* bufs[2] = {keys, &tmp};
  if (a.in_tmp != b.in_tmp)  // both inputs in one buffer, the output in the other
    NX_CUDA(cudaMemcpyAsync(bufs[a.in_tmp]->as<uint64_t>() + b.x0, bufs[b.in_tmp]->as<uint64_t>() + b.x0,
                            (b.x1 - b.x0) * sizeof(uint64_t), cudaMemcpyDeviceToDevice, stream()));
  const uint64_t* in = bufs[a.in_tmp]->as<uint64_t>();
  uint64_t* out = bufs[!a.in_tmp]->as<uint64_t>();
  NX_TRY(merge_u64(in + a.x0, a.x1 - a.x0, in + b.x0, b.x1 - b.x0, out + a.x0, split.as<uint64_t>()));
  st.push_back(Run{a.x0, b.x1, std::max(a.level, b.level) + 1, !a.in_tmp});
  return NX_OK;
}

nx_status RunMerger::push(uint64_t x0, uint64_t x1) {
  if (x1 <= x0) return NX_OK;
  st.push_back(Run{x0, x1, 0, false});
  while (st.size() >= 2 && st[st.size() - 1].level == st[st.size() - 2].level) NX_TRY(merge_top());
  return NX_OK;
}

nx_status RunMerger::finish() {
  while (st.size() >= 2) NX_TRY(merge_top());
  if (!st.empty() && st[0].in_tmp) std::swap(*keys, tmp);
  NX_CUDA(cudaStreamSynchronize(stream()));  // the scratch is freed with the merger
  return NX_OK;
}

}  // namespace nx

extern "C" nx_status nx_debug_fail_alloc(int64_t after) {
  nx::g_fail_after.store(after < 0 ? -1 : (long long)after);
  return NX_OK;
}

extern "C" nx_status nx_set_stream(void* s) {
  nx::g_stream = (cudaStream_t)s;
  return NX_OK;
}

extern "C" nx_status nx_trim_memory(void) {
  int dev = 0;
  NX_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return NX_OK;
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lock(nx::g_pool_mu);
    pool = nx::g_pools[dev];
  }
  if (!pool) return NX_OK;
  NX_CUDA(cudaDeviceSynchronize());  // frees still queued on streams reach the pool
  NX_CUDA(cudaMemPoolTrimTo(pool, 0));
  return NX_OK;
}

extern "C" void nx_last_error(char* buf, size_t len) {
  if (!buf || !len) return;
  const char* e = nx::get_error();
  size_t k = strlen(e);
  if (k >= len) k = len - 1;
  memcpy(buf, e, k);
  buf[k] = 0;
}
