// Internal: the library context behind the C ABI and the host-side steps of
// the launch sequence shared by the API calls, the batching plans and the
// serving loop.
#pragma once

#include <cstdio>
#include <cstdlib>
#include <string>
#include <utility>
#include <vector>

#include "wr_internal.h"

namespace wrc {

struct DBuf {
    void* p = nullptr;
    size_t bytes = 0;
    bool ensure(size_t need) {
        if (need <= bytes) return true;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        size_t want = need + need / 4 + 256;
        if (cudaMalloc(&p, want) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        bytes = want;
        return true;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <class T>
    T* as() const { return static_cast<T*>(p); }
};

constexpr unsigned long long DEFAULT_SPINS = 1ull << 24;  // x 64 ns sleeps: about a second
// node-level routes: legs of at most LEG_CACHE_NODES nodes keep their walk for the output, in
// a cache of at most LEG_CACHE_WORDS node ids (256 MiB)
constexpr size_t LEG_CACHE_NODES = 256;
constexpr size_t LEG_CACHE_WORDS = size_t(1) << 26;
constexpr uint64_t DEFAULT_BUDGET = 2ull << 30;

}  // namespace wrc

struct wr_ctx {
    int device = 0;
    wr_config cfg{};
    wr_tuning tune{};
    bool has_graph = false;
    wr::HostGraph hg;
    wr::HostPartition hp;
    wr::DevGraph dg;
    wrc::DBuf g_desc, g_ref, g_w, g_arc2, g_run_ptr, g_run_x, g_halo_ptr, g_halo_nodes, g_rin_ptr, g_rin_list, g_rout_ptr, g_rout_list, g_wx, g_run_wx, g_run_of, g_meta, g_flags, g_ix, g_xarc, g_cdesc;
    wr::BfLaunchInfo bf_info{};
    int enum_blocks = 0;
    // working buffers
    wrc::DBuf rows, stamp, run_stamp, list0, list1, list2, counts, bar, err, stats, ring, ring_seq, qctl;
    wrc::DBuf node_flag, src_index, src_list, n_src, block_sums;
    wrc::DBuf offs, picks, order_status, order_flags, D, unit_off, best, unit_ctr;
    wrc::DBuf out_cost, out_perm, out_status, kbuf, dgiven, src_in, sub, check;
    wrc::DBuf hk_list, hk_count, hk_D, hk_h;  // Held-Karp orders (k > WR_MAX_K)
    int hk_blocks = 0;
    int route_mode = WR_ROUTE_TOUR;
    wrc::DBuf g_in_ptr, g_in_src, g_in_w, g_in4, leg_len, leg_cache, seg_long, perm_in, node_offs_d, nodes_d;  // node-level routes
    bool in_csr_uploaded = false;
    bool positive_weights = false;  // every arc weight > 0: node-level routes are defined
    int32_t cluster_m = 0;          // > 0: cluster-patched approximate routing with at most this many clusters
    std::vector<int32_t> coords;    // plan coordinates (2 per node), host copy
    wrc::DBuf g_coords;
    // clustered routing: per order and cluster slot (n * cluster_m sub-orders)
    wrc::DBuf cl_k, cl_status, cl_flags, cl_D, cl_mem, cl_perm, cl_state, cl_nc, cl_unit_off, cl_best, cl_cost,
        cl_ostatus;
    wrc::DBuf trace;          // sweep trace of the last Bellman-Ford segment
    int32_t trace_cap = 0;
    bool capturing = false;  // enqueueing into a CUDA graph: no host syncs, external timing events
    bool untimed = false;    // no phase events (work from several streams at once: the serving loop)
    std::string tune_path;   // autotuner table: read at creation, written by wr_autotune
    // stats
    wr_stats last{};
    std::vector<cudaEvent_t> events;
    int n_events_used = 0;
    int ev_call_begin = -1, ev_call_end = -1;
    int64_t* h_offs = nullptr;   // pinned: offs[0], offs[n] of a call with device buffers
    cudaEvent_t ev_offs = nullptr;
    std::vector<std::pair<int, int>> ev_phase[6];  // select, init, bf, gather, enum, finish
    int launches = 0;
    cudaStream_t last_stream = nullptr;
};

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            if (getenv("WROUTE_DEBUG")) fprintf(stderr, "wroute: %s at %s:%d: %s\n", #call, __FILE__, \
                                                __LINE__, cudaGetErrorString(e_));            \
            return WR_ECUDA;                                                                  \
        }                                                                                     \
    } while (0)

#define RC(call)                      \
    do {                              \
        int r_ = (call);              \
        if (r_ != WR_OK) return r_;   \
    } while (0)

namespace wrc {

int ensure(DBuf& b, size_t bytes);
int set_device(wr_ctx* c);
int record(wr_ctx* c, cudaStream_t s, int* idx);

// Times one phase of a call with a pair of events on the call's stream.
struct PhaseTimer {
    wr_ctx* c;
    cudaStream_t s;
    int phase;
    int b = -1;
    PhaseTimer(wr_ctx* c_, cudaStream_t s_, int ph) : c(c_), s(s_), phase(ph) { record(c, s, &b); }
    ~PhaseTimer() {
        int e = -1;
        if (b >= 0 && record(c, s, &e) == WR_OK) c->ev_phase[phase].push_back({b, e});
    }
};

int begin_call(wr_ctx* c, cudaStream_t s);
int end_call(wr_ctx* c, cudaStream_t s);
int take_device_error(wr_ctx* c);
int32_t budget_lanes(const wr_ctx* c);
// frontier arrays for segments of seg_lanes lanes, and the segment row buffer unless the rows live elsewhere
int ensure_bf(wr_ctx* c, int32_t seg_lanes, bool with_rows = true);
wr::BfWork bf_work(wr_ctx* c, int32_t seg_lanes);
int run_bf_segment(wr_ctx* c, const wr::BfSegment& seg, cudaStream_t s);
int run_tours(wr_ctx* c, int32_t n, const int32_t* k_dev, const wr::TourBufs& tb, int32_t* cost, int32_t* perm,
              int perm_stride, int32_t* status, cudaStream_t s);
int ensure_tour_bufs(wr_ctx* c, int32_t n, wr::TourBufs& tb);
int finish_graph(wr_ctx* c);
int enqueue_select(wr_ctx* c, int32_t n, const int64_t* d_offs, const int32_t* d_picks, cudaStream_t s);
// selected: enqueue_select already queued for this call
int enqueue_route(wr_ctx* c, int32_t n, const int64_t* d_offs, const int32_t* d_picks, int64_t np_bound,
                  int32_t* o_cost, int32_t* o_perm, int32_t* o_status, cudaStream_t s, bool selected = false);

}  // namespace wrc
