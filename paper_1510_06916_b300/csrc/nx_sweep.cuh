// Sweep kernels' host-visible interface: work items and launch arguments.
#pragma once
#include "nx_internal.cuh"

namespace nx {

struct SweepSrc {
  const uint32_t* ew = nullptr;        // edge words; index e addresses edge e of the DSSS
  const float* wt = nullptr;           // normalised weights (weighted PageRank), same indexing
  const uint64_t* piece_off = nullptr; // [npieces+1]
};

// PK_PRD: PageRank that gathers r[u] / outdeg[u] directly (no contribution
// array), used by the allocation-free single-step entry point.
// PK_ADJ: the weighted-PageRank adjoint step over the transpose DSSS,
// lambda'_u = g_u + a (sum_v w^_uv lambda_v + [outdeg(u) = 0] S / n), S = sum lambda.
// PK_SCCF / PK_SCCB: the two propagations of strongly connected components
// (coloring): the forward min-color sweep over unassigned vertices (color
// 0xFFFFFFFF = assigned, never updated) and the backward max-reach sweep over
// the transpose DSSS (value 0 = not reached, color + 1 = reached; a vertex is
// reached when an out-neighbour of its own color is; aux_u32 = the colors).
enum ProgKind : int {
  PK_PR = 0, PK_WPR = 1, PK_BFS = 2, PK_WCC = 3, PK_PRD = 4, PK_ADJ = 5, PK_SCCF = 6, PK_SCCB = 7,
  PK_PROBE = 8  // the PageRank sweep's edge loads and gathers alone (a measurement)
};

struct SweepArgs {
  SweepSrc src[2];
  int nsrc = 1;
  uint32_t src_lo = 0, src_hi = 0;  // source intervals swept: [src_lo, src_hi)
  // Banded sweeps: when non-null, the tile accumulator starts from acc_in
  // (the bands before this one) instead of the identity (block 0 of a split
  // tile only).
  const void* acc_in = nullptr;
  // Items whose piece count (DSSS x source intervals) is at most flat_cap
  // (<= 256) are swept as one flattened step sequence; the table takes
  // 16 B x (flat_cap + 1) of dynamic shared memory. 0: per-piece loop.
  uint32_t flat_cap = 0;
  const Item* items = nullptr;  // nullptr: block b sweeps the whole tile b
  const uint32_t* tile_start = nullptr;
  const uint32_t* col_tb = nullptr;
  uint32_t P = 0, L = 0, lb = 0, n = 0, tile_max = 0;
  // interval activity (min programs); nullptr = every source interval active
  const uint32_t* act_in = nullptr;
  uint32_t* act_out = nullptr;
  uint32_t* act_count = nullptr;
  // values
  const void* gsrc = nullptr;  // gathered per source: c (PR), r (WPR), depth/label
  const void* vold = nullptr;  // previous values (min programs)
  void* vnew = nullptr;        // new values
  float* cnew = nullptr;       // PR: next contributions r / outdeg (nullable)
  const uint32_t* outdeg = nullptr;
  const float* tele = nullptr;  // teleport vector or nullptr (uniform 1/n)
  int dang_by_tele = 0;
  float alpha = 0.85f;
  const double* dm_in = nullptr;  // dangling mass of the previous values
  double* dm_out = nullptr;       // dangling mass of the new values
  double* tile_part = nullptr;    // [ntiles]
  uint32_t* ticket = nullptr;     // completion counter of the iteration
  uint32_t n_epi = 0;             // tile epilogues in the whole iteration
  void* split = nullptr;          // split-tile partial accumulators
  uint32_t* tile_ticket = nullptr;
  // Modes. 0: sweep [src_lo, src_hi) (+ FromHub over [hub_lo, hub_hi)) then
  // the epilogue; 1: row pass over single pieces of source interval src_lo —
  // columns < q_res accumulate into accres, the others write their hub
  // (ToHub); 2: sweep then store the raw accumulator into accres; 3: epilogue
  // from accres (no edges).
  int mode = 0;
  uint32_t q_res = 0;
  // hubs of each DSSS of the sweep (row-pass items name theirs in Item::pad)
  const uint64_t* hub_off[2] = {nullptr, nullptr};
  const uint16_t* hub_dst[2] = {nullptr, nullptr};
  void* hubs[2] = {nullptr, nullptr};  // hub values [D_s]
  uint32_t hub_lo = 0, hub_hi = 0;
  void* accres = nullptr;             // accumulators of resident columns [n_res]
  uint32_t acc_base = 0;              // vertex id of accres[0] (acc_in too)
  const uint32_t* aux_u32 = nullptr;  // PK_SCCB: the forward colors
  // staged (non-resident) intervals: the source interval stage_i is read from
  // gstage[0..L); epilogue values of a staged column go to vnew/cnew at
  // v - out_base and previous values come from vold at v - out_base.
  const void* gstage = nullptr;
  uint32_t stage_i = 0xFFFFFFFFu;
  uint32_t out_base = 0;
  // debug/robustness: number of items and edge words addressable by ew[]
  uint64_t ew_lo[2] = {0, 0};         // first edge index held by src[s].ew
};

// Launches one sweep over `nitems` items (kind selects the program).
nx_status launch_sweep(ProgKind kind, const SweepArgs& a, uint32_t nitems, cudaStream_t s);

// Persistent multi-graph run: item q of iteration i sweeps graph items[q].gid
// with args[2 * gid + (i & 1)].
struct MItem {
  uint32_t gid, pad;
  Item it;
};
struct MultiSync {
  unsigned count, gen, err, pad;
};
// `limit`: clock cycles a block waits at a grid barrier before it gives up,
// sets sy->err and returns.
nx_status launch_multi(ProgKind kind, const SweepArgs* args, const MItem* items, uint32_t nitems,
                       uint32_t iters, uint32_t* ctr, MultiSync* sy, uint32_t tile_max,
                       uint32_t nblocks, long long limit, cudaStream_t s);
// Grid-barrier wait limit of nx_run_multi in clock cycles (nx_set_barrier_limit).
long long barrier_limit();
// Co-resident blocks of the multi-graph kernel (occupancy x SMs).
nx_status multi_blocks(ProgKind kind, uint32_t tile_max, uint32_t* nblocks);

}  // namespace nx
