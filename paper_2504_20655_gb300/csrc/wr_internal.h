// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "wroute.h"

namespace wr {

constexpr uint32_t INF_U = 0x7FFFFFFFu;       // unreachable distance (= WR_INF)
constexpr uint32_t NO_CARRY = 0x80000000u;    // carry weight of a node without a chain arc
constexpr uint32_t GLOBAL_REF = 0x80000000u;  // arc source not staged: low 31 bits = node id
constexpr uint32_t TOUR_CAP = 1u << 27;       // unreachable legs are clamped to this in tour sums
constexpr int DSTRIDE = 13;                   // D blocks are 13 x 13
constexpr int DBLOCK = DSTRIDE * DSTRIDE;
constexpr int TAIL = 5;                       // tail walked by one compile-time unrolled walk
constexpr int UNIT_TAIL = 6;                  // the 720 orderings of six picks are walked from register tables
constexpr int HK_MAX_K = 20;                  // orders of WR_MAX_K+1 .. 20 picks: Held-Karp
// Held-Karp D blocks: entry (i, j), i, j in 0..HK_MAX_K, at i * HK_DSTRIDE + HK_DOFF + j, so
// that the pick legs of a row (j = 1..HK_MAX_K) start on a 16-byte boundary
constexpr int HK_DSTRIDE = 24;
constexpr int HK_DOFF = 3;
constexpr int HK_DBLOCK = (HK_MAX_K + 1) * HK_DSTRIDE;
static_assert(HK_MAX_K % 4 == 0 && (HK_DOFF + 1) % 4 == 0 && HK_DSTRIDE % 4 == 0 && HK_DOFF + HK_MAX_K < HK_DSTRIDE,
              "Held-Karp D rows: pick legs on 16-byte boundaries, inside the row");
constexpr int ORDER_FLAG_RANGE = 1;
constexpr int32_t RUN_SIMPLE = 1;             // run's extra arcs fit the tile buffer, halo fully staged
constexpr uint32_t IX_EXTRA = 1u << 24;       // node has arcs beyond the inline ones
constexpr int32_t RUN_COMPACT = 2;            // every node's arcs are staged: compact descriptors + extras (warp tiling)
constexpr int32_t RUN_PRIORITY = 8;           // feeds at least PRIORITY_FEEDS runs: listed first in every sweep
constexpr int PRIORITY_FEEDS = 6;
// extra arcs a compact run may have (they are staged with the tile): tile_cap / 2 entries, so
// that a 128-slot warp tile takes 20.5 KB of shared memory and 11 of them fit one SM
__host__ __device__ constexpr int wx_cap(int tile_cap) { return tile_cap / 2; }

// --------------------------------------------------------------------------
// graph preprocessing (host, wr_graph.cpp)
// --------------------------------------------------------------------------

// In-arc (pull) CSR: arcs into v are [in_ptr[v], in_ptr[v+1]), sorted by
// source, one arc per (u, v) pair (the lightest), no self loops.
struct HostGraph {
    int32_t V = 0;
    int64_t E = 0;
    int32_t depot = 0;
    std::vector<int64_t> in_ptr;
    std::vector<int32_t> in_src;
    std::vector<int32_t> in_w;
};

// Sweep tiles ("runs"): one or two segments of consecutive node ids (two when
// a segment and the one holding most of its halo fit one tile together, e.g.
// both faces of an aisle), whose own rows plus the rows of their outside
// in-neighbours (the halo) fit tile_cap shared-memory slots.  Tile slots:
// the first segment's nodes, then the second's, then the staged halo.
struct HostPartition {
    int32_t V = 0, n_runs = 0, tile_cap = 0, max_len = 0;
    std::vector<int4> run_seg;          // n_runs: {a0, alen, b0, blen}: nodes a0.. then b0.. (blen may be 0)
    std::vector<int32_t> halo_ptr;      // n_runs + 1 (staged halo only)
    std::vector<int32_t> halo_nodes;
    std::vector<int32_t> rin_ptr;       // runs with an arc into the run
    std::vector<int32_t> rin_list;
    std::vector<int32_t> rout_ptr;      // runs the run has an arc into (rin transposed)
    std::vector<int32_t> rout_list;
    std::vector<int32_t> run_of_node;   // V
    std::vector<int32_t> slot_of_node;  // V: tile slot in its own run
    // per node v (plus a sentinel at V): x = weight of the carry arc from the
    // previous tile slot (node v-1, NO_CARRY if none), y = from the next slot
    // (node v+1), z = first forward arc, w = first backward arc; backward arcs
    // end at desc[v+1].z (arc lists are in node id order).  Forward arcs come
    // from lower tile slots or the halo, backward arcs from higher slots.
    std::vector<int4> node_desc;
    std::vector<uint32_t> arc_ref;      // tile slot of the arc's source, or GLOBAL_REF | node
    std::vector<uint32_t> arc_w;
    // Inline form of the same arcs for the CTA tiling, two uint4 per node:
    // a = {fw carry w, bw carry w, fw0 w, fw1 w}, b = {bw0 w, fw0 slot | fw1
    // slot << 16, bw0 slot | n_fw_extra << 16 | IX_EXTRA | n_bw_extra << 25,
    // first extra}.  Absent inline arcs use slot 0 and weight NO_CARRY.  Arcs
    // beyond the inline ones are the run's extras, xarc2[run_x.x ..
    // run_x.y), forward then backward per node; "first extra" is relative to
    // run_x.x.
    std::vector<uint4> node_ix;
    std::vector<uint2> xarc2;
    std::vector<int2> run_x;
    std::vector<int64_t> run_meta_bytes;  // 8 * in-arcs + 8 * nodes of the run
    std::vector<int32_t> run_flags;       // RUN_SIMPLE | RUN_COMPACT
    // Compact descriptors of the warp tiling, 2 per node: forward {carry weight,
    // o0 | o1 << 16, w0, w1} and backward {carry weight, o0 | o1 << 16, w0, w1},
    // o = tile slot x 128 (byte offset of the slot's line in the slot-major
    // tile).  Up to two non-carry arcs per pass; absent ones o = 0, w = NO_CARRY.
    std::vector<uint4> cdesc;
    // A node's non-carry arcs beyond two per pass go to its run's extras, folded
    // into the tile before the pass (an upper bound, like every stale read):
    // wx entries {dst o | src o << 16, w}, per run forward extras then backward
    // extras from run_wx = {first entry, forward count, backward count, 0}; each
    // run's list starts at an even entry (16-byte copies).
    std::vector<uint2> wx;
    std::vector<int4> run_wx;
    int64_t n_global_refs = 0;
};

int build_host_graph(int32_t V, int64_t E, const int64_t* row_ptr, const int32_t* col,
                     const int32_t* w, int32_t depot, HostGraph& g);
void build_partition(const HostGraph& g, int run_target, int tile_cap, HostPartition& p);

// --------------------------------------------------------------------------
// device-side structures
// --------------------------------------------------------------------------

struct alignas(8) GridBar {  // one 64-bit word: count (low), generation (high)
    unsigned int count;
    unsigned int gen;
};

struct DevGraph {
    int32_t V = 0, n_runs = 0, tile_cap = 0, depot = 0;
    int4* node_desc = nullptr;
    uint32_t* arc_ref = nullptr;
    uint32_t* arc_w = nullptr;
    uint2* arc2 = nullptr;  // (arc_ref, arc_w) interleaved
    uint4* node_ix = nullptr;  // inline descriptors, 2 per node
    uint2* xarc2 = nullptr;    // extra arcs
    int4* run_seg = nullptr;   // {a0, alen, b0, blen} per run
    int2* run_x = nullptr;     // the run's extras in xarc2
    int32_t* halo_ptr = nullptr;
    int32_t* halo_nodes = nullptr;
    int32_t* rin_ptr = nullptr;
    int32_t* rin_list = nullptr;
    int32_t* rout_ptr = nullptr;   // runs fed by each run (rin transposed)
    int32_t* rout_list = nullptr;
    int32_t* run_of_node = nullptr;
    int64_t* run_meta_bytes = nullptr;
    int32_t* run_flags = nullptr;
    uint4* cdesc = nullptr;    // compact descriptors, 2 per node
    uint2* wx = nullptr;       // compact form: extra arcs per run
    int4* run_wx = nullptr;
};

// One source segment of Bellman-Ford: rows[v * ld + b] holds
// dist(src[first + b], v) for lanes b < min(count, n_src - first).
struct BfSegment {
    uint32_t* rows;
    int64_t ld;
    const int32_t* src;        // source node ids (index space of n_src)
    const int32_t* n_src_dev;  // device count of sources, or nullptr to use n_src_host
    int32_t n_src_host;
    int32_t first;
    int32_t lanes;             // lane capacity (multiple of 32)
    // optional: group g (lanes 32g .. 32g+31) lives in row columns
    // [32 gcol[g], 32 gcol[g] + 32) instead of [32g, 32g + 32) (a row cache
    // whose free column groups are scattered); nullptr = contiguous
    const int32_t* gcol = nullptr;
    // the sources are sorted by node id (the distinct sources of a batch of orders), so the 32
    // sources of a group are neighbours when they are dense enough; see BfWork::prio
    bool sorted = false;
    // optional: node -> index in src (-1: not a source), so that the init kernel writes the
    // seeds d(s, s) = 0 with the fill; nullptr = a separate seed kernel
    const int32_t* src_index = nullptr;
};

struct BfWork {
    int32_t* stamp;   // n_runs * Gcap
    int32_t* run_stamp;  // n_runs: the last sweep whose byte count took the run's descriptors
    int32_t* list0;   // n_runs * Gcap
    int32_t* list1;
    int32_t* list2;   // third frontier list (warp sweeps: sweep s reads list s mod 3)
    int32_t* counts;  // 16: list sizes, claim counters, priority list sizes (warp sweeps)
    // warp sweeps: list the items of RUN_PRIORITY runs first in every sweep.  Taken for sorted
    // sources with at least one lane per 64 nodes: a group's 32 sources then lie within a few
    // aisles, its distances spread out from there through the cross-aisles, and relaxing the
    // cross-aisle tiles first lets each sweep's aisle tiles read their new values (and keeps those
    // long tiles from ending the sweep last).  Sparse or scattered sources (the scale rows) reach
    // the cross-aisles from every aisle at once, and there it cost more tile visits.
    int prio;
    int32_t gcap;
    GridBar* bar;
    int* err;
    unsigned long long max_spins;
    unsigned long long* stats;  // [0] sweeps [1] tiles [2] node visits [3] bytes [5] descriptor re-read bytes
    long long* trace;           // optional: per sweep t < trace_cap, [2t] = frontier tiles, [2t+1] = ns
    int trace_cap;
    // asynchronous worklist (bf_tiling 3): stamp holds each item's state
    int32_t* ring;                // 2 * n_runs * Gcap slots: queued items
    unsigned long long* ring_seq;  // per slot: the ring position it serves next (see wr_bf_warp.cu)
    unsigned long long* qctl;      // [0] pop counter, [1] push counter, [2] items queued or running
    int async;                  // 1: the worklist kernel runs this segment (init fills the ring)
};

// launchers (wr_bf.cu)
struct BfLaunchInfo {
    int blocks;
    int threads;
    size_t smem;
    const void* fn;
};
// picks the sweep kernel for (tile_cap, warps per CTA; 0 = default) and its co-resident grid
int bf_prepare(int tile_cap, int warps, int device, BfLaunchInfo* info);
// the warp-per-tile kernel (wr_bf_warp.cu) for tile_cap 128 or 256: sweeps with grid barriers
// (WARP_SWEEPS), the same with two source groups per warp (WARP_PAIRS, tile_cap 128), or one
// asynchronous worklist without sweeps (WARP_ASYNC)
constexpr int WARP_SWEEPS = 0, WARP_ASYNC = 1, WARP_PAIRS = 2;
int bf_prepare_warp(int tile_cap, int mode, int device, BfLaunchInfo* info);
cudaError_t bf_launch_init(const DevGraph& g, const BfSegment& seg, const BfWork& w, cudaStream_t s);
cudaError_t bf_launch_sweeps(const DevGraph& g, const BfSegment& seg, const BfWork& w,
                             const BfLaunchInfo& info, cudaStream_t s);
cudaError_t bf_launch_rows_out(const BfSegment& seg, int32_t V, int32_t* out, int64_t ld_out,
                               cudaStream_t s);
cudaError_t bf_launch_submatrix(const BfSegment& seg, int32_t V, int32_t n_dst, const int32_t* dst,
                                int32_t* sub, unsigned long long* check, cudaStream_t s);

// launchers (wr_tour.cu)
struct TourBufs {
    const int64_t* offs;
    const int32_t* picks;
    int32_t* order_status;   // n
    int32_t* order_flags;    // n
    uint32_t* D;             // n * DBLOCK
    long long* unit_off;     // n + 1 (exclusive prefix of units)
    unsigned long long* best;  // n
    unsigned long long* unit_ctr;  // scheduling counter
    long long* seq_count;    // sequences evaluated (stat)
};
cudaError_t tour_launch_select(int32_t n, const int64_t* offs, const int32_t* picks, int32_t V,
                               int32_t depot, int32_t max_k, uint8_t* node_flag,
                               int32_t* order_status, cudaStream_t s);
// Node flags (and order flags, when given) cleared, select, compact: one launch for small calls.
cudaError_t tour_launch_select_compact(int32_t n, const int64_t* offs, const int32_t* picks, int32_t V, int32_t depot,
                                       int32_t max_k, uint8_t* node_flag, int32_t* order_status, int32_t* order_flags,
                                       int32_t* src_index, int32_t* src_list, int32_t* n_src, int32_t* block_sums,
                                       cudaStream_t s, int* launches);
cudaError_t tour_launch_compact(int32_t V, const uint8_t* node_flag, int32_t* src_index,
                                int32_t* src_list, int32_t* n_src, int32_t* block_sums,
                                cudaStream_t s, int* launches);
// open_path: the depot's legs are free (the route is the path through the picks)
cudaError_t tour_launch_gather(int32_t n, const TourBufs& t, int32_t depot, const int32_t* src_index,
                               const BfSegment& seg, int open_path, cudaStream_t s);
cudaError_t tour_launch_prepare_given(int32_t n, const int32_t* k, const int32_t* Din, int32_t max_k,
                                      const TourBufs& t, cudaStream_t s);
cudaError_t tour_launch_units(int32_t n, const int32_t* k_given, const TourBufs& t, cudaStream_t s,
                              int* launches);
cudaError_t tour_launch_enum(int32_t n, const int32_t* k_given, const TourBufs& t, long long u_begin,
                             long long u_end, int units_per_thread, int blocks, cudaStream_t s);
cudaError_t tour_launch_finish(int32_t n, const int32_t* k_given, const TourBufs& t, int32_t* cost,
                               int32_t* perm, int perm_stride, int32_t* status, cudaStream_t s);
int tour_enum_blocks(int device);

// Node-level routes (wr_paths.cu)
struct PathsLaunch {
    int32_t n;
    const int64_t* offs;
    const int32_t* picks;
    const int32_t* perm;
    const int32_t* order_status;
    int open_path;
    int32_t depot;
    const int32_t* src_index;
    const int64_t* in_ptr;  // in-arc CSR with node ids
    const int32_t* in_src;
    const int32_t* in_w;
    const int4* in4;        // per node 2 x int4: up to 4 in-arcs (u, w); u0 = -2: more, in the CSR
    int32_t V;
    int32_t* leg_len;       // offs[n] + n entries
    int32_t* leg_cache;     // (offs[n] + n) x cache_cap node ids: the legs of at most cache_cap nodes
    int32_t cache_cap;      // 0: no cache
};
// mode 0 (count walk over the legs whose source lies in *seg; a leg longer than the cache sets
// *seg_long), 1 (write walk of those legs that are longer than the cache) or 2 (copy of every
// cached leg; seg unused)
cudaError_t paths_launch(const PathsLaunch& l, const BfSegment* seg, int mode, int32_t* seg_long, int32_t* nodes,
                         const int64_t* node_offs, cudaStream_t s);
cudaError_t paths_launch_offsets(const PathsLaunch& l, int64_t* node_offs, cudaStream_t s);

// Cluster-patched approximate routing (wr_cluster.cu); xy: 2 int32 plan coordinates per node.
// Order o's clusters are sub-orders o*m .. o*m + m-1 routed by the exhaustive enumeration.
constexpr int CL_MAX = 10;   // stops per cluster
constexpr int CL_MAX_M = 6;  // clusters per order
struct ClusterBufs {
    int32_t* sub_k;               // n*m: stops of each cluster (0: empty slot)
    int32_t* sub_status;          // n*m: WR_ORDER_OK for a cluster, else BAD (no units)
    int32_t* sub_flags;           // n*m: 0
    uint32_t* sub_D;              // n*m * DBLOCK: the cluster's legs, free depot legs
    unsigned long long* members;  // n*m: pick indices (4 bits each) | count << 60
    int32_t* sub_perm;            // n*m * WR_MAX_K: the clusters' routes (sub-order sequences)
    int32_t* order_state;         // n: the order's status before patching
    int32_t* n_clusters;          // n
};
cudaError_t cluster_launch_split(int32_t n, const TourBufs& t, const int32_t* xy, int32_t m, const ClusterBufs& cb,
                                 cudaStream_t s);
cudaError_t cluster_launch_patch(int32_t n, const TourBufs& t, int32_t m, int open_path, const ClusterBufs& cb,
                                 int32_t* cost, int32_t* perm, int32_t* status, cudaStream_t s);

// Held-Karp for orders of WR_MAX_K+1 .. max_k picks (wr_hk.cu)
cudaError_t hk_launch_select(int32_t n, const TourBufs& t, int32_t max_k, int32_t* list, int32_t* count,
                             cudaStream_t s);
cudaError_t hk_launch_gather(int32_t n, const int32_t* list, const int32_t* count, const TourBufs& t, int32_t depot,
                             const int32_t* src_index, const BfSegment& seg, uint32_t* D21, int open_path,
                             cudaStream_t s);
int hk_blocks(int device);
cudaError_t hk_launch_solve(const int32_t* list, const int32_t* count, const uint32_t* D21, uint32_t* h,
                            unsigned long long h_words, const TourBufs& t, int32_t* cost, int32_t* perm,
                            int32_t* status, GridBar* bar, int* err, unsigned long long max_spins, int blocks,
                            cudaStream_t s);

}  // namespace wr
