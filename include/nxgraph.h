/*
 * nxgraph.h — C ABI of the B300 (sm_103a) DSSS update-sweep library.
 *
 * Method: NXgraph (Chi, Dai, Wang, Sun, Li, Yang; arXiv 1510.06916).
 * Vertices are split into P equal intervals I_0..I_{P-1} of L = ceil(n/P)
 * vertices; edges into P x P sub-shards SS_ij (source in I_i, destination in
 * I_j), each sorted by destination and then by source: the Destination-Sorted
 * Sub-Shard structure (Section II-A, Section III-A "Sharding"). One iteration
 * updates every destination interval from the previous iteration's values of
 * every source interval (Algorithm 1, synchronous consistency of Section II-B)
 * under one of three schedules: Single-Phase Update (Algorithm 5), Double-Phase
 * Update with per-sub-shard hubs (Algorithm 6) or Mixed-Phase Update
 * (Algorithm 7, Q resident intervals with Q <= B_M * P / (2 n B_a), Section
 * III-B3).
 *
 * Conventions for every function below:
 *  - The return value is an nx_status; 0 (NX_OK) is success. No function
 *    throws, aborts or exits the process. On failure, nx_last_error() returns
 *    a one-line description (thread-local).
 *  - "device pointer" means memory on the current CUDA device; "host pointer"
 *    means ordinary or pinned host memory. Flags or *_is_device arguments say
 *    which; pointers are never owned by the library unless stated.
 *  - All GPU work is issued on the stream set by nx_set_stream (default: the
 *    legacy default stream) and the calls return after that work is complete
 *    unless stated otherwise.
 *  - Vertex ids are uint32 in [0, n), n <= 2^30; edge counts m < 2^32.
 */
#ifndef NXGRAPH_H
#define NXGRAPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t nx_status;
#define NX_OK 0
#define NX_ERR_INVALID_ARG 1      /* bad size, id >= n, missing structure, ... */
#define NX_ERR_OOM 2              /* device or pinned-host allocation failed   */
#define NX_ERR_BUDGET_TOO_SMALL 3 /* budget below what the strategy needs      */
#define NX_ERR_CUDA 4             /* a CUDA call failed (message has the text) */
#define NX_ERR_TIMEOUT 5          /* a bounded device-side wait ran out        */

/* Vertex programs (Section II-B "Update Scheme"). */
typedef enum {
  NX_PR = 0,  /* PageRank: r' = (1-a)/n + a (sum_{u->v} r_u/outdeg_u + Dm/n)      */
  NX_PPR = 1, /* personalized PageRank: teleport t, r0 = t, dangling mass by t    */
  NX_WPR = 2, /* weighted PageRank: p_uv = w_uv / W_u (needs NX_WITH_WEIGHTS)     */
  NX_BFS = 3, /* Algorithms 2-4: depth(root) = 0, min over in-edges of depth+1    */
  NX_WCC = 4, /* min-label propagation along both edge directions (needs
                 NX_WITH_TRANSPOSE); label = smallest vertex id in the component */
  NX_SCC = 5  /* strongly connected components (Section IV-D; needs
                 NX_WITH_TRANSPOSE; SPU, no budget): label = smallest vertex id
                 of the component, by rounds of forward color propagation over
                 the DSSS and backward reach over its transpose. `iters` bounds
                 the sweeps of all rounds; vertices still unassigned when it
                 runs out keep 0xFFFFFFFF. stats: iters_done = sweeps,
                 Q = coloring rounds                                           */
} nx_program;

/* Update strategies (Section III-B). */
typedef enum {
  NX_SPU = 0,  /* Algorithm 5: all intervals resident (ping-pong), one pass      */
  NX_DPU = 1,  /* Algorithm 6: ToHub pass writes per-sub-shard hubs, FromHub pass
                  combines them per destination interval                           */
  NX_MPU = 2,  /* Algorithm 7: Q intervals resident from the budget; the (P-Q)^2
                  sub-shards among the others go through hubs                      */
  NX_AUTO = 3, /* the fastest the graph and budget allow: NX_DPU_ONCHIP for PR /
                  PPR on a graph built with NX_ONCHIP_HUBS and no budget, else
                  SPU when the budget holds all intervals, else MPU             */
  /* Exp 1 / Table IV ablation (PR and PPR only; needs NX_WITH_TRANSPOSE; budget
     0): the same sub-shards read in source order from the transpose DSSS, each
     edge pushing its contribution to the destination with an atomic add.      */
  NX_SRC_COARSE = 4, /* one thread block per sub-shard (coarse-grained model)  */
  NX_SRC_FINE = 5,   /* edge-balanced chunks of the source-sorted order         */
  /* Algorithm 6 with intervals held in shared memory (PR and PPR; the graph
     built with NX_ONCHIP_HUBS; budget 0): ToHub streams the edges row by row
     with the source interval (2^15 vertices) staged on chip and writes one hub
     value per (row, destination) run; FromHub folds the hubs column by column
     into a destination interval (2^14 vertices) accumulated on chip.          */
  NX_DPU_ONCHIP = 6
} nx_strategy;

/* nx_build_dsss flags. */
#define NX_HOST_PTRS 0u          /* src/dst/w are host pointers                     */
#define NX_DEV_PTRS 1u           /* src/dst/w are device pointers                   */
#define NX_WITH_TRANSPOSE 2u     /* also build the source-sorted (transpose) DSSS  */
#define NX_WITH_WEIGHTS 4u       /* w (float, > 0) is given: weighted PageRank     */
#define NX_RELABEL 8u            /* degree-ordered internal ids (Section III-A
                                    "degreeing"): see nx_get_relabel              */
#define NX_ONCHIP_HUBS 16u       /* also build the row-major structure of
                                    NX_DPU_ONCHIP (n up to about 9.5e7)          */
/* Tile shape (below the interval level; nx_autotune_shape searches it):
 * destination tiles of at most 2^k vertices (8 <= k <= 13; default 2^11), and
 * a tile also ends where its in-edges pass a multiple of 2^e (10 <= e <= 20;
 * default m / (8 x SMs) clamped to [2^14, 2^20], m doubled with the
 * transpose). 0 = the default.                                               */
#define NX_TILE_CAP_LOG2(k) ((uint32_t)(k) << 8)
#define NX_TILE_EDGES_LOG2(e) ((uint32_t)(e) << 12)

typedef struct nx_graph nx_graph; /* opaque; owns all its device and pinned memory */

typedef struct {
  float alpha;            /* damping (PageRank family), e.g. 0.85              */
  uint32_t root;          /* BFS root vertex                                   */
  const float* teleport;  /* PPR/WPR teleport vector [n], or NULL = uniform 1/n */
  int32_t teleport_is_device;
  int32_t use_graph;      /* reserved, set to 0                                  */
  uint32_t band_intervals;/* SPU: source intervals per launch (0 = all P in one
                             launch); with fewer, the sweep runs one launch per
                             band of source intervals and the accumulators carry
                             between bands in device memory                     */
} nx_params;

typedef struct {
  uint32_t iters_done;    /* sweeps performed                                   */
  uint32_t Q;             /* resident intervals used (MPU; P for SPU and
                             NX_DPU_ONCHIP, 0 for DPU); NX_SCC: coloring rounds;
                             nx_run_multi: 1 if the kept CUDA graph was replayed */
  uint32_t strategy;      /* the strategy that ran (after NX_AUTO)              */
  uint32_t streamed_cols; /* shards streamed from pinned host per iteration     */
  float ms;               /* wall time of the iteration loop (CUDA events)      */
  uint64_t edges_swept;   /* edges read by all sweeps (inactive sources skipped) */
  uint64_t bytes_model;   /* algorithmic device bytes of the loop: per sweep 4 B
                             per edge read (8 B weighted) + 16 n (PageRank family:
                             gather, outdeg, new values, contributions) or 12 n
                             (BFS / WCC / SCC); DPU adds 12 B per hub entry;
                             NX_DPU_ONCHIP: 2 B per edge + 10 B per hub entry
                             (H_onchip) + 16 n                                 */
  uint64_t h2d_bytes;     /* host->device bytes of the loop (streaming)         */
  uint64_t d2h_bytes;     /* device->host bytes of the loop                     */
  uint32_t launches;      /* kernels launched by the loop                       */
  uint32_t intervals_skipped; /* BFS / WCC under SPU, DPU, MPU: source intervals
                             skipped as inactive, summed over the sweeps (each
                             skips its sub-shards SS_i*, Algorithm 1); else 0  */
} nx_run_stats;

typedef struct {
  uint32_t n, P, L;       /* vertices, intervals, interval length ceil(n/P)     */
  uint32_t ntiles;        /* destination tiles (a tile never crosses an interval) */
  uint32_t tile_max;      /* max vertices in a tile                             */
  uint32_t lb;            /* bits of a source offset inside an interval         */
  uint64_t m;             /* edges                                              */
  uint64_t D;             /* distinct (sub-shard, destination) pairs = hub size */
  uint64_t D_t;           /* same for the transpose DSSS (0 if not built)       */
  uint64_t device_bytes;  /* device memory held by the graph now (after a run
                             with a budget: what that budget left resident)    */
  float build_ms;         /* time of nx_build_dsss on the device                */
  int32_t has_transpose, has_weights;
  uint64_t host_bytes;    /* pinned host memory held by the graph (offloaded
                             edges and indexes, staged intervals)             */
  uint64_t H_onchip;      /* hub entries of the NX_ONCHIP_HUBS structure (0 if
                             not built): runs of equal (source interval of
                             2^15, destination), cut every 2048 edges         */
} nx_graph_info;

/* Stream for all later calls (a cudaStream_t; NULL = legacy default stream). */
nx_status nx_set_stream(void* stream);

/* Device memory cache. The library allocates from a stream-ordered pool of its
 * own per device that keeps freed blocks (up to half of the device's memory)
 * for the next build or run, the way a caching allocator does. This call
 * synchronises the device and returns every cached, unused block of the
 * current device's pool to the driver (memory held by live graphs stays).
 * Errors: NX_ERR_CUDA if the device cannot be synchronised. */
nx_status nx_trim_memory(void);

/* Copies the last error message of this thread into buf (always terminated). */
void nx_last_error(char* buf, size_t len);

/* Test hook for the error paths: the library's device allocation made `after`
 * allocations from now (0: the next one) fails as if the device were out of
 * memory, so the call that made it returns NX_ERR_OOM (nx_last_error says the
 * failure was injected). A negative `after` disarms the hook; it disarms
 * itself once it fires. The countdown is process-wide and counts the
 * library's own device allocations only. A graph whose call failed stays
 * valid: a later call may use or free it. Always NX_OK. */
nx_status nx_debug_fail_alloc(int64_t after);

/*
 * Builds the DSSS of Section II-A / III-A on the device: equal intervals of
 * L = ceil(n/P) vertices, P*P sub-shards sorted by (destination, source), the
 * per-sub-shard hub index (Table I, H_ij), out-degrees, and optionally the
 * transpose (source-sorted) DSSS and per-source normalised weights.
 *   src, dst : edge endpoints [m] (uint32 ids < n); host or device per flags
 *   m, n, P  : edges, vertices (1 <= n <= 2^30), intervals (1 <= P <= min(n, 1024))
 *   w        : edge weights [m] (> 0) when NX_WITH_WEIGHTS, else ignored
 *   out      : receives the new graph (caller frees with nx_graph_free)
 * Input arrays are copied; the caller keeps ownership. Host edges without
 * weights are sorted chunk by chunk while they cross the host link (all source
 * chunks first, then the destination chunks) and the sorted chunks merged;
 * from page-locked (pinned) host memory every copy is queued at once, from
 * pageable memory each chunk is staged by the calling thread in turn. The
 * result does not depend on the path taken.
 * NX_RELABEL renames the vertices before sharding: internal id k is the
 * caller vertex with the k-th largest out-degree (ties by caller id), so
 * heavily read source values cluster. No vertex is dropped and n is kept.
 * Every vertex-indexed argument and result of nx_run, nx_get_values,
 * nx_set_values, nx_run_ppr_batch and nx_adjoint_wpr stays in caller ids
 * (BFS root, teleports, ranks, depths, WCC labels = smallest caller id of the
 * component, gradients; edge gradients stay in caller edge order). Only
 * nx_dsss_export reports internal ids. nx_run_multi and
 * nx_pagerank_step_noalloc reject relabeled graphs.
 * NX_ONCHIP_HUBS also builds the row-major structure of NX_DPU_ONCHIP (its
 * edges sorted by source interval of 2^15 vertices, destination interval of
 * 2^14, destination, source; one 16-bit entry per edge and one hub entry per
 * run of equal (source interval, destination), cut every 2048 edges).
 * NX_TILE_CAP_LOG2 / NX_TILE_EDGES_LOG2 choose the tile shape.
 * Errors: INVALID_ARG (an id >= n, P out of range, m >= 2^32, n > 2^30,
 * missing w, tile shape out of range, unknown flag bits, NX_ONCHIP_HUBS with
 * more than about 9.5e7 vertices), OOM, CUDA.
 */
nx_status nx_build_dsss(const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n,
                        uint32_t P, uint32_t flags, const float* w, nx_graph** out);

nx_status nx_graph_get_info(const nx_graph* g, nx_graph_info* info);

/*
 * The vertex order of a graph built with NX_RELABEL: old_of_new[k] is the
 * caller id of internal vertex k (a permutation of [0, n)).
 *   old_of_new : [count] uint32, device if out_is_device else host
 * Errors: INVALID_ARG (NULL, count != n, graph built without NX_RELABEL), CUDA.
 */
nx_status nx_get_relabel(const nx_graph* g, uint32_t* old_of_new, uint64_t count,
                         int32_t out_is_device);

/*
 * Exports a DSSS in its storage order (Section II-A): edge k of the output is
 * the k-th stored edge, sub-shard by sub-shard (shard j = destination
 * interval outer, source interval i inner), each sorted by destination then
 * source. sub_off[j*P + i] is where SS_ij starts (P*P + 1 entries).
 *   transpose : 0 = forward DSSS, 1 = the transpose DSSS (its "destination"
 *               is the original source; the output gives original src/dst)
 * Ids are the internal ones (after NX_RELABEL, map them with nx_get_relabel).
 *   src, dst  : host uint32 [m]; sub_off: host uint64 [P*P + 1] (nullable)
 * Errors: INVALID_ARG (transpose not built), CUDA.
 */
nx_status nx_dsss_export(const nx_graph* g, int32_t transpose, uint32_t* src, uint32_t* dst,
                         uint64_t* sub_off);

/*
 * Runs `iters` synchronous iterations of `program` (BFS/WCC: at most `iters`,
 * stopping when no interval is active — Algorithm 1) under `strategy` with a
 * device-memory budget of mem_budget_bytes (0 = unlimited).
 * The budget B_M is accounted as in Section III-B: the ping-pong intervals
 * (2 n B_a, B_a = 4) plus the edge words held on the device.
 *  - B_M >= 2 n B_a (SPU, and MPU / AUTO with Q = P): shards [0, Jc) and the
 *    head of shard Jc that fit stay on the device; the rest of the edge words
 *    live only in pinned host memory and stream through two staging buffers
 *    on a side stream every iteration, in bands of at most 64 MB (consecutive
 *    sub-shards of a shard, or ranges of the tiles of one larger sub-shard; a
 *    band exceeds 64 MB only when a single tile does). DSSS the program does
 *    not read, the hub index and (except for NX_WPR) the weights move to
 *    pinned host memory too. The device then holds the budget plus:
 *    out-degrees and PageRank contributions (12 n bytes), the id maps of
 *    NX_RELABEL (8 n), piece offsets (16 bytes per piece per DSSS), tile
 *    tables, one column of accumulators and the staging buffers. The
 *    layout persists after the run (nx_graph_get_info: device_bytes,
 *    host_bytes); a later call that needs more on the device (a run without a
 *    budget, nx_run_ppr_batch, nx_adjoint_wpr, nx_run_multi, nx_dsss_export)
 *    uploads it again first. Shrinking copies the kept prefix once, so the
 *    old and the new prefix coexist for the length of that copy.
 *  - 2 L B_a <= B_M < 2 n B_a (MPU with Q < P, Algorithm 7; DPU): intervals
 *    [Q, P) live in pinned host memory and are staged per row and column;
 *    the edge words and hubs stay on the device.
 *   params : nullable (alpha 0.85, root 0, uniform teleport)
 *   stats  : nullable; filled on success
 * Every run starts from the program's Initialize (Algorithm 2 for BFS), with
 * one exception that serves resuming: when nx_set_values was called for this
 * program since the graph's last run, the run continues from those values.
 * The values a run leaves stay in the graph for nx_get_values.
 * Errors: INVALID_ARG (program needs a structure the graph lacks, root >= n,
 * an NX_SRC_* strategy with another program or a budget), BUDGET_TOO_SMALL
 * (SPU without room for 2 n B_a; MPU/DPU below one interval pair), OOM, CUDA.
 */
nx_status nx_run(nx_graph* g, nx_program program, const nx_params* params, uint32_t iters,
                 nx_strategy strategy, uint64_t mem_budget_bytes, nx_run_stats* stats);

/*
 * Copies the current values of the last program run (float ranks for the
 * PageRank family; uint32 depths / labels for BFS / WCC) into out[count],
 * count == n. out is device memory if out_is_device, else host memory.
 */
nx_status nx_get_values(const nx_graph* g, void* out, uint64_t count, int32_t out_is_device);

/*
 * Replaces the current values of `program` (same layout as nx_get_values) so
 * that the next nx_run of that program continues from them (resume; for BFS
 * and WCC every interval is marked active).
 */
nx_status nx_set_values(nx_graph* g, nx_program program, const void* in, uint64_t count,
                        int32_t in_is_device);

/*
 * Batched personalized PageRank: B teleport vectors solved together, one
 * sweep per iteration over the DSSS with B values per vertex.
 *   teleport : [n][B] row-major float (vertex-major), host or device
 *   ranks    : output [n][B] float, host or device (same flag)
 * r0 = t and dangling mass spread by each column's t; damping `alpha`
 * (iters = 0 returns r0 = t).
 * Errors: INVALID_ARG (NULL pointers, B not in [1, 64], alpha outside
 * [0, 1)), OOM, CUDA.
 */
nx_status nx_run_ppr_batch(nx_graph* g, const float* teleport, uint32_t B, uint32_t iters,
                           float alpha, float* ranks, int32_t ptrs_are_device,
                           nx_run_stats* stats);

/*
 * Adjoint of weighted PageRank (an extension; the paper has no counterpart).
 * Uses the ranks r of the last NX_WPR run (fwd iterations) and the transpose
 * DSSS: lambda^0 = grad_r, lambda' = a (W^ lambda + d (1^T lambda)/n) + grad_r
 * for adj_terms-1 updates, then
 *   grad_t[v]  = (1-a) lambda_v
 *   grad_w[e]  = a r_u / W_u (lambda_v - sum_v' w^_uv' lambda_v'),  e = (u, v)
 * with grad_w in the caller's original edge order.
 *   grad_r : [n] float; grad_w : [m] float; grad_t : [n] float (nullable)
 *   all three on the device if ptrs_are_device, else host.
 * Errors: INVALID_ARG (no weights/transpose, no prior WPR run), OOM, CUDA.
 */
nx_status nx_adjoint_wpr(nx_graph* g, const float* grad_r, uint32_t adj_terms, float* grad_w,
                         float* grad_t, int32_t ptrs_are_device, nx_run_stats* stats);

/*
 * Runs `program` on `count` independent graphs in one persistent kernel per
 * call (blocks pull (graph, tile) work items from a counter and meet at a
 * grid barrier after every iteration), the whole iteration loop captured in a
 * CUDA graph. The launch has parallelism across graphs, so graphs built for it
 * with larger tiles (NX_TILE_EDGES_LOG2(16)) run faster here (256 R-MAT graphs
 * of scales 10..18: 1.4x) and slower when swept alone. The executable graph
 * is kept (a few per process) and replayed by a later call with the same
 * graphs, program, iteration count, damping and barrier limit whose graphs
 * have not reallocated any buffer since (stats->Q is then 1, else 0);
 * nx_graph_free of a member drops it. Each graph keeps its own values (read
 * them with nx_get_values). BFS uses root 0.
 * Errors: INVALID_ARG (NULL or repeated graphs, PPR, WCC on a graph without
 * transpose, WPR without weights, a graph built with NX_RELABEL), TIMEOUT (a
 * grid barrier waited longer than its limit, see nx_set_barrier_limit; the
 * kernel then ends without touching memory beyond its graphs, the values are
 * undefined and the graphs' completion counters are reset for later runs),
 * OOM, CUDA.
 */
nx_status nx_run_multi(nx_graph** graphs, uint32_t count, nx_program program, float alpha,
                       uint32_t iters, nx_run_stats* stats);

/*
 * Output of BFS (Algorithm 4): the largest finite depth among the graph's
 * current BFS values (the number of levels below the root), or -1 if none is
 * finite.
 *   max_depth : host int64
 * Errors: INVALID_ARG (NULL, the graph's last run was not NX_BFS), CUDA.
 */
nx_status nx_bfs_max_depth(const nx_graph* g, int64_t* max_depth);

/*
 * Measurement aid (no counterpart in the paper): times `sweeps` passes of the
 * PageRank SPU sweep's memory access pattern alone over the forward DSSS --
 * the same thread blocks, launches, edge-word loads and one 4-byte source
 * gather per edge, but no reduction, accumulation or epilogue -- and returns
 * the mean time of one pass. It bounds from below the time of any sweep that
 * gathers one value per edge in DSSS order on this GPU.
 *   ms_per_sweep : host float
 * Errors: INVALID_ARG (NULL, sweeps == 0), OOM, CUDA.
 */
nx_status nx_gather_probe(nx_graph* g, uint32_t sweeps, float* ms_per_sweep);

/*
 * How long a thread block of nx_run_multi's persistent kernel waits at a grid
 * barrier before it gives up, in GPU clock cycles (0 = the default, 4e9
 * cycles: about two seconds at 2 GHz). Applies to later calls in the whole
 * process. A short limit makes the barrier give up on purpose, which is how
 * the TIMEOUT path is tested (no block ever waits without a limit).
 * Errors: INVALID_ARG (cycles > 2^62).
 */
nx_status nx_set_barrier_limit(uint64_t cycles);

void nx_graph_free(nx_graph* g);

/*
 * nx_pagerank_step_noalloc — one synchronous PageRank step that allocates no
 * memory (the paper has no counterpart; this serves callers of the library).
 * It is for callers that cannot call cudaMalloc when they step the iteration:
 * an application that has already given the whole device to its own memory
 * pool, or a latency-critical loop that must not pay for an allocation or for
 * the device-wide synchronisation of cudaFree. It computes
 *   r_out[v] = (1-alpha)/n + alpha * (sum_{u->v} r_in[u]/outdeg(u) + Dm/n),
 *   Dm = sum over vertices without out-edges of r_in[u],
 * the same step as one NX_PR iteration of nx_run, with one thread block per
 * destination tile (heavy tiles are not split).
 *   g     : a graph from nx_build_dsss (only its forward DSSS is used)
 *   r_in  : device float [n], the current ranks (not modified)
 *   r_out : device float [n], receives the next ranks (must not alias r_in)
 * Scratch: a file-scope 4 MiB device array (held by every GPU that loads the
 * library until the process exits) instead of cudaMalloc; graphs with more
 * than 523,232 destination tiles are rejected with NX_ERR_INVALID_ARG. The
 * first call on a device looks up the array's device address once for that
 * device; make that first call before any stream capture. All calls share the
 * array: calls whose GPU work overlaps (different streams or threads) race on
 * it and must be serialised by the caller. Runs on the stream of
 * nx_set_stream and returns when the step is complete.
 * Errors: INVALID_ARG (NULL pointers, r_in == r_out, alpha outside [0, 1),
 * too many tiles, a graph built with NX_RELABEL, a graph whose arrays a run
 * with a device budget moved to host memory), CUDA.
 */
nx_status nx_pagerank_step_noalloc(const nx_graph* g, float alpha, const float* r_in,
                                   float* r_out);

/* A partition and tile shape: P intervals, tiles of at most 2^tile_cap_log2
 * vertices ending where their in-edges pass multiples of 2^tile_edges_log2
 * (0 = the default of each; the NX_TILE_* flags). */
typedef struct {
  uint32_t P, tile_cap_log2, tile_edges_log2, pad_;
} nx_shape;

/*
 * Autotuner over the partition and the tile shape (Exp 2, Section IV-B2: the
 * paper finds P = 12..48 good on its CPU): builds the DSSS for every
 * candidate, times `iters` iterations of `program` under SPU (after one
 * warm-up run) and returns the index of the fastest candidate.
 *   src, dst, m, n, flags, w : as nx_build_dsss (the candidates' shapes
 *                              replace any NX_TILE_* bits of flags)
 *   candidates, count        : shapes to try
 *   best                     : receives the fastest candidate's index
 *   ms_per_iter              : [count] measured ms per iteration (nullable)
 *   cache_path               : text file of earlier results keyed by GPU name,
 *                              n, m, flags, program and candidates (nullable:
 *                              none). A hit returns the stored index without
 *                              timing (ms_per_iter then holds -1).
 * Errors: as nx_build_dsss and nx_run.
 */
nx_status nx_autotune_shape(const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n,
                            uint32_t flags, const float* w, nx_program program,
                            const nx_shape* candidates, uint32_t count, uint32_t iters,
                            uint32_t* best, float* ms_per_iter, const char* cache_path);

/*
 * nx_autotune_shape over P alone (tile shape from flags): best_P receives the
 * fastest of candidates[count].
 */
nx_status nx_autotune(const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n,
                      uint32_t flags, const float* w, nx_program program,
                      const uint32_t* candidates, uint32_t count, uint32_t iters,
                      uint32_t* best_P, float* ms_per_iter, const char* cache_path);

/* Shape of the batched PPR sweep: source rows each lane group keeps in
 * flight (2, 4 or 8) and destinations per sub-tile (32, 64, 128 or 256; a
 * block's shared-memory rows). Default {4, 128}. */
typedef struct {
  uint32_t rows, sub;
} nx_batch_shape;

/* Sets the batched-PPR shape used by later nx_run_ppr_batch calls on g.
 * Errors: INVALID_ARG (NULL, a value outside the sets above). */
nx_status nx_set_batch_shape(nx_graph* g, uint32_t rows, uint32_t sub);

/*
 * Autotuner of the batched-PPR shape: runs nx_run_ppr_batch with each
 * candidate (a warm-up run, then a timed one), keeps the fastest on the graph
 * (as nx_set_batch_shape) and returns its index. Arguments as
 * nx_run_ppr_batch (the ranks go to a scratch buffer the tuner allocates);
 * ms_per_iter, cache_path as nx_autotune_shape (the key holds the GPU name,
 * n, m, P, tile count, padded B and the candidates).
 * Errors: INVALID_ARG (NULL, no candidates, iters == 0, a shape out of
 * range), and those of nx_run_ppr_batch.
 */
nx_status nx_autotune_ppr_batch(nx_graph* g, const float* teleport, uint32_t B, uint32_t iters,
                                float alpha, int32_t ptrs_are_device,
                                const nx_batch_shape* candidates, uint32_t count, uint32_t* best,
                                float* ms_per_iter, const char* cache_path);

/* Planner model of Section III-B (Table II): bytes read / written per
 * iteration for strategy s with n vertices, m edges, P intervals, budget B_M,
 * attribute/id/edge sizes B_a, B_v, B_e and average hub in-degree d.
 * Q (resident intervals) = min(P, floor(B_M * P / (2 n B_a))) for MPU.
 * Host arithmetic only (no device is touched).
 * Errors: INVALID_ARG (n, P, B_a or d not positive; a strategy other than
 * SPU, DPU, MPU or AUTO, which the paper's model does not cover). */
nx_status nx_io_model(nx_strategy s, double n, double m, double P, double B_M, double B_a,
                      double B_v, double B_e, double d, double* Q, double* bytes_read,
                      double* bytes_write);

#ifdef __cplusplus
}
#endif
#endif /* NXGRAPH_H */
