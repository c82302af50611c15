// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/nxgraph.h"
#include <nvtx3/nvToolsExt.h>

namespace nx {

// A named range on the NVTX timeline for the library's phases (builds, runs,
// their plan and iteration loops), for Nsight tools; with no tool attached a
// push and a pop cost a few nanoseconds.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
const char* get_error();

struct Status {
  nx_status code = NX_OK;
  bool ok() const { return code == NX_OK; }
};

#define NX_TRY(expr)                    \
  do {                                  \
    nx_status _s = (expr);              \
    if (_s != NX_OK) return _s;         \
  } while (0)

nx_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);
#define NX_CUDA(call)                                                  \
  do {                                                                 \
    cudaError_t _e = (call);                                           \
    if (_e != cudaSuccess) return nx::cuda_fail(_e, #call, __FILE__, __LINE__); \
  } while (0)
#define NX_LAUNCH_CHECK() NX_CUDA(cudaGetLastError())

nx_status invalid(const std::string& msg);

// ---------------------------------------------------------------- stream
cudaStream_t stream();

// ---------------------------------------------------------------- device buffers
// Device memory from the library's stream-ordered pool (one per device):
// allocated and freed in the order of the stream that was current at
// allocation, so buffers of one graph are reused without device-wide
// synchronisation. A buffer released while another stream is current first
// waits for the whole device (the older stream may still use it).
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t owner = nullptr;  // stream current at allocation
  bool pooled = false;           // false: plain cudaMalloc (no pool on this device)
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes), owner(o.owner), pooled(o.pooled) {
    o.p = nullptr;
    o.bytes = 0;
  }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p;
      bytes = o.bytes;
      owner = o.owner;
      pooled = o.pooled;
      o.p = nullptr;
      o.bytes = 0;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  void release();
  nx_status alloc(size_t n);  // frees first; n == 0 allocates nothing
  template <class T> T* as() const { return static_cast<T*>(p); }
};

struct PinnedBuf {
  void* p = nullptr;
  size_t bytes = 0;
  PinnedBuf() = default;
  PinnedBuf(const PinnedBuf&) = delete;
  PinnedBuf& operator=(const PinnedBuf&) = delete;
  ~PinnedBuf() { release(); }
  void release();
  nx_status alloc(size_t n);
  template <class T> T* as() const { return static_cast<T*>(p); }
};

// Pinned host blocks from a process-wide cache: a freed block is kept (up to
// 512 MB in all) for the next request of about its size, so a graph built
// after another one reuses pinned pages instead of pinning and zeroing new ones.
void* pinned_take(size_t bytes, size_t* got);
void pinned_give(void* p, size_t bytes);

// Host array in a cached pinned block (device-to-host copies into it run at
// full speed); resize() leaves the contents undefined.
template <class T> struct PinnedArray {
  T* p = nullptr;
  size_t n = 0, cap = 0;  // cap: bytes of the block
  PinnedArray() = default;
  PinnedArray(const PinnedArray&) = delete;
  PinnedArray& operator=(const PinnedArray&) = delete;
  ~PinnedArray() { release(); }
  void release() {
    if (p) pinned_give(p, cap);
    p = nullptr;
    n = cap = 0;
  }
  nx_status resize(size_t count) {
    if (count * sizeof(T) > cap) {
      release();
      size_t got = 0;
      p = static_cast<T*>(pinned_take(count * sizeof(T), &got));
      if (!p) return NX_ERR_OOM;
      cap = got;
    }
    n = count;
    return NX_OK;
  }
  T& operator[](size_t i) { return p[i]; }
  const T& operator[](size_t i) const { return p[i]; }
  T* data() { return p; }
  const T* data() const { return p; }
  size_t size() const { return n; }
  bool empty() const { return n == 0; }
};

// Two timing events, destroyed on every exit path.
struct EventPair {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  EventPair() = default;
  EventPair(const EventPair&) = delete;
  EventPair& operator=(const EventPair&) = delete;
  ~EventPair() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
  nx_status create();
  nx_status elapsed(float* ms);  // waits for e1
};

inline uint32_t bits_for(uint64_t x) {  // bits to hold values in [0, x)
  uint32_t b = 0;
  while (b < 64 && (x - 1) >> b) ++b;
  return x <= 1 ? 0 : b;
}
inline uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }
inline uint64_t round_up(uint64_t a, uint64_t b) { return ceil_div(a, b) * b; }

int num_sms();

// Edge arrays are padded and streamed staging copies aligned to this many
// words, so a lane's vector loads past the end of a range stay in the buffer.
constexpr uint64_t kEdgeAlign = 16;

// ---------------------------------------------------------------- primitives
// Exclusive scan of in[0..n) into out[0..n); *total (device, nullable) gets the
// sum. out may alias in. Scratch is allocated internally.
nx_status exclusive_scan_u32(const uint32_t* in, uint32_t* out, uint64_t n, uint32_t* total);
nx_status exclusive_scan_u64(const uint64_t* in, uint64_t* out, uint64_t n, uint64_t* total);
// LSD radix sort of 64-bit keys over bits [0, key_bits), stable, with an
// optional uint32 payload. On return keys/vals hold the sorted data, possibly
// in buffers swapped in from the sort's scratch (at least n elements), so
// pointers taken from them before the call are stale.
nx_status radix_sort_u64(DevBuf& keys, DevBuf* vals, uint64_t n, uint32_t key_bits);
// The same on caller buffers, stream-ordered, no allocation: keys a[0..n)
// (payload va, nullable) with scratch b (vb) of n elements and `counts` of
// radix_sort_count_words(n) words; *in_b tells whether the result ended in b.
nx_status radix_sort_u64_raw(uint64_t* a, uint64_t* b, uint32_t* va, uint32_t* vb, uint32_t* counts,
                             uint64_t n, uint32_t key_bits, bool* in_b);
uint64_t radix_sort_count_words(uint64_t n);
// Stable merge (ties: the earlier run first) of sorted runs laid end to end in
// `keys` into one sorted sequence, pairwise by merge path, stream-ordered.
// Runs are pushed in order as they become sorted and neighbours of equal rank
// are merged at once (a binary counter), so most of the merging overlaps the
// work that produces the later runs; finish() merges the rest, leaving the
// result in keys (possibly swapped with the scratch buffer, as in
// radix_sort_u64) and synchronising the stream.
struct RunMerger {
  nx_status init(DevBuf& keys, uint64_t n);
  nx_status push(uint64_t x0, uint64_t x1);  // keys[x0, x1) is sorted
  nx_status finish();

 private:
  struct Run {
    uint64_t x0, x1;
    int level;
    bool in_tmp;
  };
  nx_status merge_top();
  DevBuf* keys = nullptr;
  DevBuf tmp, split;
  std::vector<Run> st;
};
// Smallest shared-memory carveout that keeps the occupancy of kernel `fn`
// (`threads` per block, `smem` dynamic bytes); the rest of L1 caches loads.
nx_status prefer_l1(const void* fn, int threads, size_t smem);

// ---------------------------------------------------------------- DSSS
// One destination-sorted structure over the graph's tile geometry. The
// transpose DSSS is the same structure built with source and destination
// swapped (its "destination" is the original source).
struct Dsss {
  uint64_t m = 0;
  uint64_t words = 0;  // edge words with padding: round_up(m, kEdgeAlign) + kEdgeAlign
  DevBuf ew;         // uint32 [dev_words]: ((dst - tile_start) << lb) | src_local
  DevBuf wt;         // float  [words]: normalised weight of each edge (weighted graphs)
  DevBuf piece_off;  // uint64 [npieces+1]
  DevBuf hub_off;    // uint64 [npieces+1]: hub entries before each piece
  DevBuf hub_dst;    // uint16 [D]: destination offset in its tile of each hub entry
  uint64_t D = 0;
  PinnedArray<uint64_t> h_piece_off;  // host copy of piece_off
  // Residency under a device budget: words [0, dev_words) of the edge array
  // are on the device; the pinned host image h_ew holds words
  // [h_ew_first, words) (h_ew_first <= dev_words, so together they hold every
  // word). Without a budget dev_words == words and h_ew is empty.
  uint64_t dev_words = 0;
  PinnedBuf h_ew;
  uint64_t h_ew_first = 0;
  // Arrays moved whole to pinned host memory while a budgeted run does not
  // need them on the device (hub index, weights).
  PinnedBuf h_hub_dst, h_wt;
  PinnedBuf h_piece_pin, h_hub_off;  // piece and hub offsets while the DSSS is unread
};

// The on-chip double-phase structure (NX_ONCHIP_HUBS): the paper's DPU
// (Algorithm 6) with source intervals of 2^kOcSrcBits vertices, small enough
// to stage in shared memory for ToHub, and destination intervals of
// 2^kOcDstBits vertices, whose compensated accumulators fit shared memory for
// FromHub. Edges are sorted by (source interval i, destination interval j,
// destination, source), rows (i) outermost. A hub entry is a run of equal
// (i, j, destination), also cut at every multiple of kOcSeg edges; a segment
// is a window of the edge array between cuts and row starts, so no hub entry
// crosses a segment. ToHub needs only the source and where entries start, so
// each edge is stored as 16 bits: src_local | (entry start) << 15.
constexpr uint32_t kOcSrcBits = 15;
constexpr uint32_t kOcDstBits = 14;
constexpr uint32_t kOcSeg = 2048;
struct OcItemA {   // ToHub work item: segments [s0, s1) of row `row`
  uint32_t row, s0, s1, pad;
};
struct OcItemB {   // FromHub work item: hub chunks [c0, c1) of column `col`
  uint32_t col, c0, c1;
  uint32_t nsplit, part, slot;  // blocks sharing the column, this block, first split slot
  uint32_t group, pad;          // completion counter of a split column
};
struct OnChip {
  bool built = false;
  uint32_t PA = 0, PB = 0;     // source (row) and destination (column) intervals
  uint64_t m = 0, H = 0;       // edges, hub entries
  DevBuf ew;                   // uint16 [round_up(m, 16) + 16]
  DevBuf seg_e;                // uint64 [nseg + 1]: first edge of each segment
  DevBuf seg_h;                // uint64 [nseg]: first hub entry of each segment
  DevBuf hub_dst;              // uint16 [H]: destination offset in its column
  DevBuf hub_val;              // float [H]
  DevBuf chunks;               // uint64 [nchunks]: (first hub entry << 32) | entries (<= 256),
                               // the nonempty pieces (i, j) column by column
  DevBuf items_a, items_b;     // OcItemA [na], OcItemB [nb]
  DevBuf split, ticket, part;  // split-column slots, completion counters, dangling partials
  PinnedBuf h_ew, h_hub_dst;   // host copies while a budgeted run holds them off the device
  uint32_t na = 0, nb = 0, nseg = 0, slots = 0, groups = 0;
  uint64_t nchunks = 0;
};

struct Geometry {
  uint32_t n = 0, P = 0, L = 0, lb = 0, tile_max = 0, ntiles = 0;
  DevBuf tile_start;  // uint32 [ntiles+1]
  DevBuf col_tb;      // uint32 [P+1]: first tile of each column
  std::vector<uint32_t> h_tile_start, h_col_tb;
};

// One thread block's work: a destination tile, or a contiguous part of the
// tile's "virtual edge sequence" (its pieces (i, t) for i = 0..P-1, over each
// DSSS in the sweep, concatenated) when the tile is too heavy for one block.
struct Item {
  uint32_t tile;
  uint32_t nsplit;  // blocks sharing this tile (1: not split)
  uint32_t slot;    // first split slot of the tile (split tiles only)
  uint32_t sub;     // this block's index among them
  uint64_t vbeg, vend;
  uint32_t row;     // mode 1: the source interval i of the piece
  uint32_t pad;     // mode 1: the DSSS of the piece (0 forward, 1 transpose)
};

// Piece (i, t) of tile t in column j: P*tb_j + i*nt_j + (t - tb_j).
__host__ __device__ inline uint64_t piece_index(uint32_t P, uint32_t tb_j, uint32_t nt_j,
                                                uint32_t i, uint32_t t) {
  return (uint64_t)P * tb_j + (uint64_t)i * nt_j + (t - tb_j);
}

}  // namespace nx

// ---------------------------------------------------------------- the graph
struct nx_graph {
  uint64_t m = 0;
  nx::Geometry geo;
  nx::Dsss fwd, tr;
  bool has_tr = false, has_w = false;
  nx::DevBuf outdeg;   // uint32 [n]
  nx::DevBuf wsum;     // float [n]  W_u (weighted)
  nx::DevBuf orig_src, orig_dst;  // uint32 [m] caller order (weighted: edge grads)
  nx::PinnedBuf h_orig_src, h_orig_dst;  // their host copies while offloaded
  // Degree-ordered ids (NX_RELABEL): internal id k holds caller vertex
  // old_of_new[k]; every vertex-indexed input and output is mapped at the ABI.
  bool relabeled = false;
  nx::DevBuf old_of_new, new_of_old;  // uint32 [n]
  float build_ms = 0.f;
  // values
  int last_prog = -1;
  int values_set_for = -1;  // program whose values were set by nx_set_values
  nx::DevBuf val[2];        // ping-pong value arrays [n] (float or uint32)
  nx::DevBuf aux[2];        // PR: contribution arrays c = r / outdeg
  int cur = 0;              // index of the current values
  nx::DevBuf act[2];        // uint32 [P+1] interval activity (+ counter slot)
  nx::DevBuf scal;          // doubles / counters used by the sweeps
  nx::DevBuf tile_part;     // double [ntiles] per-tile dangling partials
  nx::DevBuf split_buf;     // split-tile partial accumulators
  nx::DevBuf tile_ticket;   // uint32 [ntiles]
  nx::DevBuf hubs;          // hub values [D] (forward DSSS)
  nx::DevBuf hubs_t;        // hub values [D_t] (transpose DSSS, WCC)
  // Work plans (item lists) cached by strategy / DSSS set / placement.
  struct Plan {
    nx::DevBuf items;
    std::vector<uint64_t> h_cost;  // per item: its share of edges (host)
    std::vector<nx::Item> h_items;
    uint32_t na = 0, nb = 0, slots = 0;
    std::vector<uint32_t> off;  // item offsets of each launch of the plan
  };
  std::map<int, std::unique_ptr<Plan>> plans;
  nx::DevBuf init_part;     // per-block partial sums of the init kernel
  uint64_t split_floats = 0;
  nx::DevBuf tele;          // float [n] teleport copy (PPR/WPR)
  nx::DevBuf lam[2], ybuf;  // adjoint scratch
  nx::OnChip oc;            // the on-chip double-phase structure (NX_ONCHIP_HUBS)
  float wpr_alpha = 0.85f;  // damping of the last weighted PageRank run
  uint32_t ppr_rows = 4;    // batched PPR: source rows in flight per lane group
  uint32_t ppr_sub = 128;   // batched PPR: destinations per sub-tile
  nx::DevBuf stage[2];      // staging for streamed shards
  nx::DevBuf vstage[8];     // staging for non-resident intervals (MPU), double-buffered
  nx::PinnedBuf hval[2];    // pinned host values of non-resident intervals
  nx::PinnedBuf hact;       // pinned host copy of the activity count + flags [P + 1]
  nx::DevBuf accres;        // MPU resident-column accumulators
  uint64_t device_bytes() const;
  uint64_t host_bytes() const;
};

namespace nx {
// Table IV ablation run (nx_push.cu): source-sorted sub-shards with atomic
// pushes; values start from g->val/aux[g->cur] and dm[g->cur].
struct PushRun {
  bool coarse;         // one block per sub-shard (else edge-balanced chunks)
  uint32_t iters;
  float alpha;
  const float* tele;   // nullable: uniform 1/n
  int dang_by_tele;    // PPR: dangling mass spread by the teleport
  double* dm;          // [2] dangling mass ping-pong
};
nx_status push_run(nx_graph* g, const PushRun& r, uint32_t* launches, float* ms);

// The on-chip double-phase structure (nx_onchip.cu): built from the internal
// edge arrays; one iteration of PageRank / personalized PageRank over it.
nx_status build_onchip(nx_graph* g, const uint32_t* s, const uint32_t* d, uint64_t m);
struct OcRun {
  const float* c_in;     // contributions r / outdeg of the current values
  float* r_out;          // new ranks
  float* c_out;          // new contributions
  const float* tele;     // teleport (nullptr: uniform 1/n)
  int dang_by_tele;
  float alpha;
  const double* dm_in;   // dangling mass of the current values
  double* dm_out;        // of the new values
};
nx_status onchip_iteration(nx_graph* g, const OcRun& r, cudaStream_t s);

// Relabel (nx_relabel.cu). relabel_edges computes the vertex order (out-degree
// descending, ties by caller id) into g from the caller ids' out-degrees
// `outdeg` and, when s_out is not NULL, writes the renamed endpoints (s_out /
// d_out may alias s / d).
// gather_u32: out[k] = in[idx[k]] for k < n.
nx_status relabel_edges(nx_graph* g, const uint32_t* s, const uint32_t* d, uint64_t m,
                        uint32_t* s_out, uint32_t* d_out, const uint32_t* outdeg);
nx_status gather_u32(const uint32_t* idx, const void* in, void* out, uint64_t n);
// Endpoints renamed to the new ids of g in place (caller ids -> internal ids).
nx_status rename_edges(const nx_graph* g, uint32_t* s, uint32_t* d, uint64_t m);
// Vertex arrays across the ABI: caller order -> internal order (to_internal)
// or back; a plain copy for graphs that were not relabeled. `in` and `out`
// are device pointers and must not alias.
nx_status vertex_to_internal(const nx_graph* g, const void* in, void* out);
nx_status vertex_to_caller(const nx_graph* g, const void* in, void* out);

// Residency (nx_engine.cu). set_edge_residency keeps words [0, dev_words) of
// d's edge array on the device and words [host_first, words) in pinned host
// memory (host_first <= dev_words), moving data between the two as needed.
// ensure_resident brings every array of the graph back to the device and
// frees the host copies (entry points that read the whole graph call it).
nx_status set_edge_residency(Dsss& d, uint64_t dev_words, uint64_t host_first);
nx_status ensure_resident(nx_graph* g);
bool fully_resident(const nx_graph* g);
nx_status move_to_host(DevBuf& d, PinnedBuf& h);
nx_status move_to_device(PinnedBuf& h, DevBuf& d);
}  // namespace nx

