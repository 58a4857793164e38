// C ABI (include/wroute.h): context, buffers and the launch sequence of the
// routing path.  Every step of the path runs in the kernels of wr_bf.cu and
// wr_tour.cu; this file only sizes buffers, plans source segments and
// enqueues work on the caller's stream.
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "wr_ctx.h"

namespace wrc {

int ensure(DBuf& b, size_t bytes) { return b.ensure(bytes) ? WR_OK : WR_ENOMEM; }

int set_device(wr_ctx* c) { return cudaSetDevice(c->device) == cudaSuccess ? WR_OK : WR_ECUDA; }

cudaEvent_t next_event(wr_ctx* c, int* idx) {
    if (c->n_events_used >= static_cast<int>(c->events.size())) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        c->events.push_back(e);
    }
    *idx = c->n_events_used;
    return c->events[c->n_events_used++];
}

int record(wr_ctx* c, cudaStream_t s, int* idx) {
    if (c->untimed) {
        *idx = -1;
        return WR_OK;
    }
    cudaEvent_t e = next_event(c, idx);
    if (!e) return WR_ECUDA;
    // inside a capture the record becomes a node of the graph that stamps the event at replay
    if (c->capturing) CK(cudaEventRecordWithFlags(e, s, cudaEventRecordExternal));
    else CK(cudaEventRecord(e, s));
    return WR_OK;
}


int begin_call(wr_ctx* c, cudaStream_t s) {
    c->n_events_used = 0;
    c->ev_call_end = -1;  // a call that fails after this point reports no total
    for (auto& v : c->ev_phase) v.clear();
    c->launches = 0;
    c->last_stream = s;
    std::memset(&c->last, 0, sizeof(c->last));
    RC(ensure(c->stats, 8 * sizeof(unsigned long long)));
    RC(ensure(c->err, sizeof(int)));
    CK(cudaMemsetAsync(c->stats.p, 0, 8 * sizeof(unsigned long long), s));
    return record(c, s, &c->ev_call_begin);
}

int end_call(wr_ctx* c, cudaStream_t s) { return record(c, s, &c->ev_call_end); }

// Returns the recorded device error (and clears it); the stream must be idle.
int take_device_error(wr_ctx* c) {
    int h = 0;
    if (!c->err.p) return WR_OK;
    CK(cudaMemcpy(&h, c->err.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (h != 0) CK(cudaMemset(c->err.p, 0, sizeof(int)));
    return h;
}

int upload(DBuf& b, const void* src, size_t bytes) {
    RC(ensure(b, bytes == 0 ? 4 : bytes));
    if (bytes) CK(cudaMemcpy(b.p, src, bytes, cudaMemcpyHostToDevice));
    return WR_OK;
}

// Tiling in effect: the tuned one, else warp tiles up to 256 slots and CTA tiles above.
int resolved_tiling(const wr_ctx* c) {
    return c->tune.bf_tiling != 0 ? c->tune.bf_tiling : (c->hp.tile_cap <= 256 ? 1 : 2);
}

// Sweep kernel for the context's tiling and tile size.
int prepare_sweeps(wr_ctx* c) {
    const int tiling = resolved_tiling(c);
    if (tiling == 1 || tiling == 3 || tiling == 4)
        return wr::bf_prepare_warp(c->hp.tile_cap,
                                   tiling == 3 ? wr::WARP_ASYNC : tiling == 4 ? wr::WARP_PAIRS : wr::WARP_SWEEPS,
                                   c->device, &c->bf_info);
    return wr::bf_prepare(c->hp.tile_cap, c->tune.bf_warps, c->device, &c->bf_info);
}

int upload_partition(wr_ctx* c) {
    const wr::HostPartition& p = c->hp;
    RC(upload(c->g_desc, p.node_desc.data(), p.node_desc.size() * sizeof(int4)));
    RC(upload(c->g_ref, p.arc_ref.data(), p.arc_ref.size() * 4));
    RC(upload(c->g_w, p.arc_w.data(), p.arc_w.size() * 4));
    {
        std::vector<uint2> a2(p.arc_ref.size());
        for (size_t i = 0; i < a2.size(); ++i) a2[i] = make_uint2(p.arc_ref[i], p.arc_w[i]);
        RC(upload(c->g_arc2, a2.data(), a2.size() * sizeof(uint2)));
    }
    RC(upload(c->g_run_ptr, p.run_seg.data(), p.run_seg.size() * sizeof(int4)));
    RC(upload(c->g_run_x, p.run_x.data(), p.run_x.size() * sizeof(int2)));
    RC(upload(c->g_halo_ptr, p.halo_ptr.data(), p.halo_ptr.size() * 4));
    RC(upload(c->g_halo_nodes, p.halo_nodes.data(), p.halo_nodes.size() * 4));
    RC(upload(c->g_rin_ptr, p.rin_ptr.data(), p.rin_ptr.size() * 4));
    RC(upload(c->g_rin_list, p.rin_list.data(), p.rin_list.size() * 4));
    RC(upload(c->g_wx, p.wx.data(), p.wx.size() * sizeof(uint2)));
    RC(upload(c->g_run_wx, p.run_wx.data(), p.run_wx.size() * sizeof(int4)));
    RC(upload(c->g_rout_ptr, p.rout_ptr.data(), p.rout_ptr.size() * 4));
    RC(upload(c->g_rout_list, p.rout_list.data(), p.rout_list.size() * 4));
    RC(upload(c->g_run_of, p.run_of_node.data(), p.run_of_node.size() * 4));
    RC(upload(c->g_meta, p.run_meta_bytes.data(), p.run_meta_bytes.size() * 8));
    RC(upload(c->g_flags, p.run_flags.data(), p.run_flags.size() * 4));
    RC(upload(c->g_ix, p.node_ix.data(), p.node_ix.size() * sizeof(uint4)));
    RC(upload(c->g_xarc, p.xarc2.data(), p.xarc2.size() * sizeof(uint2)));
    RC(upload(c->g_cdesc, p.cdesc.data(), p.cdesc.size() * sizeof(uint4)));
    wr::DevGraph& g = c->dg;
    g.V = p.V;
    g.n_runs = p.n_runs;
    g.tile_cap = p.tile_cap;
    g.depot = c->hg.depot;
    g.node_desc = c->g_desc.as<int4>();
    g.arc_ref = c->g_ref.as<uint32_t>();
    g.arc_w = c->g_w.as<uint32_t>();
    g.arc2 = c->g_arc2.as<uint2>();
    g.run_seg = c->g_run_ptr.as<int4>();
    g.run_x = c->g_run_x.as<int2>();
    g.halo_ptr = c->g_halo_ptr.as<int32_t>();
    g.halo_nodes = c->g_halo_nodes.as<int32_t>();
    g.rin_ptr = c->g_rin_ptr.as<int32_t>();
    g.rin_list = c->g_rin_list.as<int32_t>();
    g.wx = c->g_wx.as<uint2>();
    g.run_wx = c->g_run_wx.as<int4>();
    g.rout_ptr = c->g_rout_ptr.as<int32_t>();
    g.rout_list = c->g_rout_list.as<int32_t>();
    g.run_of_node = c->g_run_of.as<int32_t>();
    g.run_meta_bytes = c->g_meta.as<int64_t>();
    g.run_flags = c->g_flags.as<int32_t>();
    g.node_ix = c->g_ix.as<uint4>();
    g.xarc2 = c->g_xarc.as<uint2>();
    g.cdesc = c->g_cdesc.as<uint4>();
    return prepare_sweeps(c);
}

int partition(wr_ctx* c) {
    wr::build_partition(c->hg, c->tune.run_target, c->tune.tile_cap, c->hp);
    return upload_partition(c);
}

int32_t budget_lanes(const wr_ctx* c) {
    const uint64_t per_lane = static_cast<uint64_t>(c->dg.V) * 4ull;
    uint64_t lanes = c->cfg.mem_budget_bytes / per_lane;
    lanes = (lanes / 32) * 32;
    if (lanes > (1u << 30)) lanes = 1u << 30;
    return static_cast<int32_t>(lanes);
}

// Size the row buffer and frontier arrays for segments of seg_lanes lanes.
int ensure_bf(wr_ctx* c, int32_t seg_lanes, bool with_rows) {
    const size_t rows_bytes = static_cast<size_t>(seg_lanes) * static_cast<size_t>(c->dg.V) * 4;
    if (with_rows) RC(ensure(c->rows, rows_bytes));
    const size_t items = static_cast<size_t>(c->dg.n_runs) * static_cast<size_t>(seg_lanes / 32);
    RC(ensure(c->stamp, items * 4));
    RC(ensure(c->run_stamp, static_cast<size_t>(c->dg.n_runs) * 4));
    RC(ensure(c->list0, items * 4));
    RC(ensure(c->list1, items * 4));
    RC(ensure(c->list2, items * 4));
    RC(ensure(c->counts, 64));
    RC(ensure(c->bar, sizeof(wr::GridBar)));
    RC(ensure(c->ring, 2 * items * 4));
    RC(ensure(c->ring_seq, 2 * items * 8));
    RC(ensure(c->qctl, 4 * sizeof(unsigned long long)));
    return WR_OK;
}

wr::BfWork bf_work(wr_ctx* c, int32_t seg_lanes) {
    wr::BfWork w;
    w.stamp = c->stamp.as<int32_t>();
    w.run_stamp = c->run_stamp.as<int32_t>();
    w.list0 = c->list0.as<int32_t>();
    w.list1 = c->list1.as<int32_t>();
    w.list2 = c->list2.as<int32_t>();
    w.counts = c->counts.as<int32_t>();
    w.prio = 0;
    w.gcap = seg_lanes / 32;
    w.bar = c->bar.as<wr::GridBar>();
    w.err = c->err.as<int>();
    w.max_spins = c->cfg.barrier_max_spins ? c->cfg.barrier_max_spins : DEFAULT_SPINS;
    w.stats = c->stats.as<unsigned long long>();
    w.trace = c->trace_cap > 0 ? c->trace.as<long long>() : nullptr;
    w.trace_cap = c->trace_cap > 0 ? c->trace_cap : 0;
    w.ring = c->ring.as<int32_t>();
    w.ring_seq = c->ring_seq.as<unsigned long long>();
    w.qctl = c->qctl.as<unsigned long long>();
    w.async = resolved_tiling(c) == 3;
    return w;
}

// One Bellman-Ford segment: init + sweeps.
int run_bf_segment(wr_ctx* c, const wr::BfSegment& seg, cudaStream_t s) {
    wr::BfWork w = bf_work(c, seg.lanes);
    w.prio = seg.sorted && static_cast<int64_t>(seg.lanes) * 64 >= static_cast<int64_t>(c->dg.V);
    if (w.trace) CK(cudaMemsetAsync(w.trace, 0xFF, static_cast<size_t>(w.trace_cap) * 16, s));
    {
        PhaseTimer t(c, s, 1);
        CK(wr::bf_launch_init(c->dg, seg, w, s));
        c->launches += seg.src_index ? 1 : 2;
    }
    {
        PhaseTimer t(c, s, 2);
        CK(wr::bf_launch_sweeps(c->dg, seg, w, c->bf_info, s));
        c->launches++;
    }
    return WR_OK;
}

float elapsed(wr_ctx* c, int a, int b) {
    float ms = 0.f;
    if (a < 0 || b < 0) return 0.f;
    if (cudaEventElapsedTime(&ms, c->events[a], c->events[b]) != cudaSuccess) {
        cudaGetLastError();
        return 0.f;
    }
    return ms;
}

// Enumeration (a5, a6) over the prepared D blocks, then decode (a7).
int run_tours(wr_ctx* c, int32_t n, const int32_t* k_dev, const wr::TourBufs& tb, int32_t* cost, int32_t* perm,
              int perm_stride, int32_t* status, cudaStream_t s) {
    {
        PhaseTimer t(c, s, 4);
        CK(wr::tour_launch_units(n, k_dev, tb, s, &c->launches));
        const int upt = c->tune.enum_units > 0 ? c->tune.enum_units : 2;
        if (c->tune.enum_max_units_per_launch > 0 && !c->capturing) {
            long long total = 0;
            CK(cudaMemcpyAsync(&total, tb.unit_off + n, sizeof(long long), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            const long long step = c->tune.enum_max_units_per_launch;
            for (long long b = 0; b < total; b += step) {
                CK(cudaMemsetAsync(tb.unit_ctr, 0, sizeof(unsigned long long), s));
                CK(wr::tour_launch_enum(n, k_dev, tb, b, b + step < total ? b + step : total, upt, c->enum_blocks, s));
                c->launches += 2;  // two builds, one of which returns at once
            }
        } else {
            CK(wr::tour_launch_enum(n, k_dev, tb, 0, 1ll << 62, upt, c->enum_blocks, s));
            c->launches += 2;
        }
    }
    {
        PhaseTimer t(c, s, 5);
        CK(wr::tour_launch_finish(n, k_dev, tb, cost, perm, perm_stride, status, s));
        c->launches++;
    }
    return WR_OK;
}

int ensure_tour_bufs(wr_ctx* c, int32_t n, wr::TourBufs& tb) {
    RC(ensure(c->order_status, static_cast<size_t>(n) * 4 + 4));
    RC(ensure(c->order_flags, static_cast<size_t>(n) * 4 + 4));
    RC(ensure(c->D, static_cast<size_t>(n) * wr::DBLOCK * 4 + 4));
    RC(ensure(c->unit_off, (static_cast<size_t>(n) + 1) * 8));
    RC(ensure(c->best, static_cast<size_t>(n) * 8 + 8));
    RC(ensure(c->unit_ctr, 16));
    tb.order_status = c->order_status.as<int32_t>();
    tb.order_flags = c->order_flags.as<int32_t>();
    tb.D = c->D.as<uint32_t>();
    tb.unit_off = c->unit_off.as<long long>();
    tb.best = c->best.as<unsigned long long>();
    tb.unit_ctr = c->unit_ctr.as<unsigned long long>();
    tb.seq_count = reinterpret_cast<long long*>(c->stats.as<unsigned long long>() + 4);
    return WR_OK;
}

int finish_host_call(wr_ctx* c, cudaStream_t s) {
    CK(cudaStreamSynchronize(s));
    return take_device_error(c);
}

int check_ptr_kind(int k) { return (k == WR_HOST || k == WR_DEVICE) ? WR_OK : WR_EINVAL; }

bool valid_tuning(const wr_tuning* t) {
    if (t->run_target < 1 || (t->tile_cap != 128 && t->tile_cap != 256 && t->tile_cap != 512) || t->enum_units < 1 ||
        t->enum_max_units_per_launch < 0 || t->run_target > t->tile_cap)
        return false;
    if (t->bf_warps != 0 && t->bf_warps != 4 && t->bf_warps != 8) return false;
    if (t->tile_cap >= 512 && t->bf_warps == 4) return false;
    if (t->bf_tiling < 0 || t->bf_tiling > 4 || ((t->bf_tiling == 1 || t->bf_tiling == 3) && t->tile_cap > 256) ||
        (t->bf_tiling == 4 && t->tile_cap != 128))
        return false;
    return true;
}

// Tuning table file: one "name value" pair per line, unknown names ignored.
bool read_tuning_file(const std::string& path, wr_tuning* t) {
    FILE* f = std::fopen(path.c_str(), "r");
    if (!f) return false;
    char key[64];
    long long v = 0;
    int n = 0;
    while (std::fscanf(f, "%63s %lld", key, &v) == 2) {
        const std::string k(key);
        if (k == "run_target") t->run_target = static_cast<int32_t>(v);
        else if (k == "tile_cap") t->tile_cap = static_cast<int32_t>(v);
        else if (k == "enum_units") t->enum_units = static_cast<int32_t>(v);
        else if (k == "enum_max_units_per_launch") t->enum_max_units_per_launch = static_cast<int32_t>(v);
        else if (k == "bf_warps") t->bf_warps = static_cast<int32_t>(v);
        else if (k == "bf_tiling") t->bf_tiling = static_cast<int32_t>(v);
        else continue;
        ++n;
    }
    std::fclose(f);
    return n > 0;
}

bool write_tuning_file(const std::string& path, const wr_tuning* t) {
    FILE* f = std::fopen(path.c_str(), "w");
    if (!f) return false;
    std::fprintf(f, "run_target %d\ntile_cap %d\nenum_units %d\nenum_max_units_per_launch %d\nbf_warps %d\nbf_tiling %d\n",
                 t->run_target, t->tile_cap, t->enum_units, t->enum_max_units_per_launch, t->bf_warps, t->bf_tiling);
    return std::fclose(f) == 0;
}

// Partition and upload c->hg, size the per-node work arrays.
int finish_graph(wr_ctx* c) {
    const int32_t V = c->hg.V;
    c->has_graph = false;
    RC(partition(c));
    RC(ensure(c->node_flag, static_cast<size_t>(V) + 16));
    RC(ensure(c->src_index, static_cast<size_t>(V) * 4 + 16));
    RC(ensure(c->src_list, static_cast<size_t>(V) * 4 + 16));
    RC(ensure(c->n_src, 16));
    RC(ensure(c->block_sums, (static_cast<size_t>(V) / 4096 + 2) * 4));
    c->has_graph = true;
    return WR_OK;
}

// a1-a7 for n orders whose offs/picks are on the device, np_bound >= offs[n]:
// enqueues everything on s with no host synchronisation (the segments are
// planned for the worst case of np_bound + 1 distinct sources).
// a2: sources = depot + distinct pick nodes of valid orders (needs no host-side pick count)
int enqueue_select(wr_ctx* c, int32_t n, const int64_t* d_offs, const int32_t* d_picks, cudaStream_t s) {
    const int32_t V = c->dg.V;
    wr::TourBufs tb{};
    tb.offs = d_offs;
    tb.picks = d_picks;
    RC(ensure_tour_bufs(c, n, tb));
    PhaseTimer t(c, s, 0);
    CK(wr::tour_launch_select_compact(n, d_offs, d_picks, V, c->dg.depot, c->cfg.max_k, c->node_flag.as<uint8_t>(),
                                      tb.order_status, c->order_flags.as<int32_t>(), c->src_index.as<int32_t>(),
                                      c->src_list.as<int32_t>(), c->n_src.as<int32_t>(), c->block_sums.as<int32_t>(),
                                      s, &c->launches));
    return WR_OK;
}

int enqueue_route(wr_ctx* c, int32_t n, const int64_t* d_offs, const int32_t* d_picks, int64_t np_bound,
                  int32_t* o_cost, int32_t* o_perm, int32_t* o_status, cudaStream_t s, bool selected) {
    const int32_t V = c->dg.V;
    wr::TourBufs tb{};
    tb.offs = d_offs;
    tb.picks = d_picks;
    RC(ensure_tour_bufs(c, n, tb));
    if (!selected) RC(enqueue_select(c, n, d_offs, d_picks, s));
    // orders above WR_MAX_K picks (when the context admits them): Held-Karp; the clustered
    // approximation takes at most WR_MAX_K picks
    const bool clustered = c->cluster_m > 0;
    if (clustered && c->coords.size() != 2 * static_cast<size_t>(V)) return WR_EINVAL;
    const bool hk = c->cfg.max_k > WR_MAX_K && !clustered;
    if (hk) {
        RC(ensure(c->hk_list, static_cast<size_t>(n) * 4 + 4));
        RC(ensure(c->hk_count, 16));
        RC(ensure(c->hk_D, static_cast<size_t>(n) * wr::HK_DBLOCK * 4 + 4));
        // tables of a batch of orders solved together: at least one of max_k picks, up to the budget
        const size_t one = (static_cast<size_t>(1) << (c->cfg.max_k - 1)) * static_cast<size_t>(c->cfg.max_k) * 4;
        RC(ensure(c->hk_h, one > c->cfg.mem_budget_bytes ? one : static_cast<size_t>(c->cfg.mem_budget_bytes)));
        CK(cudaMemsetAsync(c->hk_count.p, 0, 4, s));
        CK(wr::hk_launch_select(n, tb, c->cfg.max_k, c->hk_list.as<int32_t>(), c->hk_count.as<int32_t>(), s));
        c->launches++;
    }
    // segments of the worst-case source count; empty ones exit on the device
    const int64_t worst = np_bound + 1 < V ? np_bound + 1 : V;
    const int32_t lanes_needed = static_cast<int32_t>((worst + 31) / 32 * 32);
    const int32_t blanes = budget_lanes(c);
    if (blanes < 32) return WR_ENOMEM;
    const int32_t seg_lanes = lanes_needed < blanes ? lanes_needed : blanes;
    const int32_t n_seg = (lanes_needed + seg_lanes - 1) / seg_lanes;
    RC(ensure_bf(c, seg_lanes));
    for (int32_t sg = 0; sg < n_seg; ++sg) {
        wr::BfSegment seg;
        seg.rows = c->rows.as<uint32_t>();
        seg.ld = seg_lanes;
        seg.src = c->src_list.as<int32_t>();
        seg.sorted = true;  // the distinct sources of the orders, in node id order
        seg.src_index = c->src_index.as<int32_t>();
        seg.n_src_dev = c->n_src.as<int32_t>();
        seg.n_src_host = 0;
        seg.first = sg * seg_lanes;
        seg.lanes = seg_lanes;
        RC(run_bf_segment(c, seg, s));
        PhaseTimer t(c, s, 3);
        CK(wr::tour_launch_gather(n, tb, c->dg.depot, c->src_index.as<int32_t>(), seg, c->route_mode == WR_ROUTE_OPEN,
                                  s));
        c->launches++;
        if (hk) {
            CK(wr::hk_launch_gather(n, c->hk_list.as<int32_t>(), c->hk_count.as<int32_t>(), tb, c->dg.depot,
                                    c->src_index.as<int32_t>(), seg, c->hk_D.as<uint32_t>(),
                                    c->route_mode == WR_ROUTE_OPEN, s));
            c->launches++;
        }
    }
    c->last.n_segments = n_seg;
    if (clustered) {
        // every cluster an order has becomes a sub-order with free depot legs, routed by the
        // exhaustive enumeration; then the patching of the cluster routes
        const int32_t m = c->cluster_m;
        const size_t ns = static_cast<size_t>(n) * static_cast<size_t>(m);
        RC(ensure(c->cl_k, ns * 4 + 4));
        RC(ensure(c->cl_status, ns * 4 + 4));
        RC(ensure(c->cl_flags, ns * 4 + 4));
        RC(ensure(c->cl_D, ns * wr::DBLOCK * 4 + 4));
        RC(ensure(c->cl_mem, ns * 8 + 8));
        RC(ensure(c->cl_perm, ns * WR_MAX_K * 4 + 4));
        RC(ensure(c->cl_state, static_cast<size_t>(n) * 4 + 4));
        RC(ensure(c->cl_nc, static_cast<size_t>(n) * 4 + 4));
        RC(ensure(c->cl_unit_off, (ns + 1) * 8));
        RC(ensure(c->cl_best, ns * 8 + 8));
        RC(ensure(c->cl_cost, ns * 4 + 4));
        RC(ensure(c->cl_ostatus, ns * 4 + 4));
        wr::ClusterBufs cb{c->cl_k.as<int32_t>(), c->cl_status.as<int32_t>(), c->cl_flags.as<int32_t>(),
                           c->cl_D.as<uint32_t>(), c->cl_mem.as<unsigned long long>(), c->cl_perm.as<int32_t>(),
                           c->cl_state.as<int32_t>(), c->cl_nc.as<int32_t>()};
        {
            PhaseTimer t(c, s, 3);
            CK(wr::cluster_launch_split(n, tb, c->g_coords.as<int32_t>(), m, cb, s));
            c->launches++;
        }
        wr::TourBufs sb{};
        sb.order_status = cb.sub_status;
        sb.order_flags = cb.sub_flags;
        sb.D = cb.sub_D;
        sb.unit_off = c->cl_unit_off.as<long long>();
        sb.best = c->cl_best.as<unsigned long long>();
        sb.unit_ctr = tb.unit_ctr;
        sb.seq_count = tb.seq_count;
        RC(run_tours(c, static_cast<int32_t>(ns), cb.sub_k, sb, c->cl_cost.as<int32_t>(), cb.sub_perm, WR_MAX_K,
                     c->cl_ostatus.as<int32_t>(), s));
        {
            PhaseTimer t(c, s, 5);
            CK(wr::cluster_launch_patch(n, tb, m, c->route_mode == WR_ROUTE_OPEN, cb, o_cost, o_perm, o_status, s));
            c->launches++;
        }
        return WR_OK;
    }
    RC(run_tours(c, n, nullptr, tb, o_cost, o_perm, 0, o_status, s));
    if (hk) {
        // after the decode of the other orders: these write their own cost, perm and status
        PhaseTimer t(c, s, 4);
        RC(ensure(c->bar, sizeof(wr::GridBar)));
        CK(cudaMemsetAsync(c->bar.p, 0, sizeof(wr::GridBar), s));
        CK(wr::hk_launch_solve(c->hk_list.as<int32_t>(), c->hk_count.as<int32_t>(), c->hk_D.as<uint32_t>(),
                               c->hk_h.as<uint32_t>(), c->hk_h.bytes / 4, tb, o_cost, o_perm, o_status,
                               c->bar.as<wr::GridBar>(),
                               c->err.as<int>(), c->cfg.barrier_max_spins ? c->cfg.barrier_max_spins : DEFAULT_SPINS,
                               c->hk_blocks, s));
        c->launches++;
    }
    return WR_OK;
}

}  // namespace wrc

using namespace wrc;

extern "C" {

const char* wr_strerror(int code) {
    switch (code) {
        case WR_OK: return "ok";
        case WR_EINVAL: return "invalid argument";
        case WR_ENOMEM: return "out of memory or memory budget too small";
        case WR_ECUDA: return "CUDA runtime error";
        case WR_ETIMEOUT: return "device-side wait timed out";
        case WR_ENOGRAPH: return "no graph loaded";
        case WR_EINTERNAL: return "Bellman-Ford sweep cap exceeded";
        default: return "unknown error";
    }
}

int wr_create(const wr_config* cfg, wr_ctx** out) {
    if (!out) return WR_EINVAL;
    *out = nullptr;
    wr_config c{};
    c.device = 0;
    c.mem_budget_bytes = DEFAULT_BUDGET;
    c.max_k = WR_MAX_K;
    c.barrier_max_spins = DEFAULT_SPINS;
    c.tune_path = nullptr;
    if (cfg) c = *cfg;
    if (c.max_k < 1 || c.max_k > WR_MAX_K_EXACT || c.device < 0) return WR_EINVAL;
    if (c.mem_budget_bytes == 0) return WR_ENOMEM;
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || c.device >= n_dev) {
        cudaGetLastError();
        return WR_ECUDA;
    }
    if (cudaSetDevice(c.device) != cudaSuccess) return WR_ECUDA;
    wr_ctx* ctx = new (std::nothrow) wr_ctx();
    if (!ctx) return WR_ENOMEM;
    ctx->device = c.device;
    ctx->cfg = c;
    ctx->cfg.tune_path = nullptr;
    ctx->tune.run_target = 60;  // two segments of ~60 nodes (aisle faces) share a 128-slot tile
    ctx->tune.tile_cap = 128;
    ctx->tune.enum_units = 2;
    ctx->tune.enum_max_units_per_launch = 0;
    ctx->tune.bf_warps = 0;
    ctx->tune.bf_tiling = 0;
    ctx->enum_blocks = wr::tour_enum_blocks(c.device);
    ctx->hk_blocks = wr::hk_blocks(c.device);
    if (cfg && cfg->tune_path) {
        ctx->tune_path = cfg->tune_path;
        wr_tuning t = ctx->tune;
        if (read_tuning_file(ctx->tune_path, &t) && valid_tuning(&t)) ctx->tune = t;
    }
    if (ctx->err.ensure(sizeof(int)) == false || cudaMemset(ctx->err.p, 0, sizeof(int)) != cudaSuccess) {
        delete ctx;
        return WR_ENOMEM;
    }
    *out = ctx;
    return WR_OK;
}

void wr_destroy(wr_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    if (c->h_offs) cudaFreeHost(c->h_offs);
    if (c->ev_offs) cudaEventDestroy(c->ev_offs);
    DBuf* bufs[] = {&c->g_desc, &c->g_ref, &c->g_w, &c->g_arc2, &c->g_run_ptr, &c->g_run_x, &c->g_halo_ptr, &c->g_halo_nodes, &c->g_rin_ptr,
                    &c->g_rin_list, &c->g_rout_ptr, &c->g_rout_list, &c->g_wx, &c->g_run_wx, &c->g_run_of, &c->g_meta, &c->g_flags, &c->g_ix, &c->g_xarc, &c->g_cdesc, &c->rows, &c->stamp, &c->run_stamp, &c->list0, &c->list1, &c->list2,
                    &c->counts, &c->bar, &c->ring, &c->ring_seq, &c->qctl, &c->err, &c->stats, &c->node_flag, &c->src_index, &c->src_list,
                    &c->n_src, &c->block_sums, &c->offs, &c->picks, &c->order_status, &c->order_flags, &c->D,
                    &c->unit_off, &c->best, &c->unit_ctr, &c->out_cost, &c->out_perm, &c->out_status, &c->kbuf,
                    &c->dgiven, &c->src_in, &c->sub, &c->check, &c->trace,
                    &c->hk_list, &c->hk_count, &c->hk_D, &c->hk_h, &c->g_in_ptr, &c->g_in_src, &c->g_in_w, &c->g_in4,
                    &c->leg_len, &c->leg_cache, &c->seg_long, &c->perm_in, &c->node_offs_d, &c->nodes_d, &c->g_coords,
                    &c->cl_k, &c->cl_status, &c->cl_flags, &c->cl_D, &c->cl_mem, &c->cl_perm, &c->cl_state, &c->cl_nc,
                    &c->cl_unit_off, &c->cl_best, &c->cl_cost, &c->cl_ostatus};
    for (DBuf* b : bufs) b->release();
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    delete c;
}

int wr_sync(wr_ctx* c) {
    if (!c) return WR_EINVAL;
    RC(set_device(c));
    CK(cudaDeviceSynchronize());
    return take_device_error(c);
}

int wr_load_graph(wr_ctx* c, int32_t V, int64_t E, const int64_t* row_ptr, const int32_t* col, const int32_t* w,
                  int32_t depot, int ptr_kind) {
    if (!c || V < 1 || E < 0 || !row_ptr) return WR_EINVAL;
    RC(check_ptr_kind(ptr_kind));
    RC(set_device(c));
    std::vector<int64_t> rp;
    std::vector<int32_t> cl, wt;
    const int64_t* hrp = row_ptr;
    const int32_t* hcol = col;
    const int32_t* hw = w;
    if (ptr_kind == WR_DEVICE) {
        rp.resize(static_cast<size_t>(V) + 1);
        CK(cudaDeviceSynchronize());  // no stream argument: wait for all work writing the inputs
        CK(cudaMemcpy(rp.data(), row_ptr, rp.size() * 8, cudaMemcpyDeviceToHost));
        cl.resize(static_cast<size_t>(E));
        wt.resize(static_cast<size_t>(E));
        if (E) {
            CK(cudaMemcpy(cl.data(), col, static_cast<size_t>(E) * 4, cudaMemcpyDeviceToHost));
            CK(cudaMemcpy(wt.data(), w, static_cast<size_t>(E) * 4, cudaMemcpyDeviceToHost));
        }
        hrp = rp.data();
        hcol = cl.data();
        hw = wt.data();
    }
    wr::HostGraph g;
    RC(wr::build_host_graph(V, E, hrp, hcol, hw, depot, g));
    c->hg.in_ptr.swap(g.in_ptr);
    c->hg.in_src.swap(g.in_src);
    c->hg.in_w.swap(g.in_w);
    c->hg.V = g.V;
    c->hg.E = g.E;
    c->hg.depot = g.depot;
    c->in_csr_uploaded = false;
    c->coords.clear();  // coordinates belong to the previous graph
    c->positive_weights = std::all_of(c->hg.in_w.begin(), c->hg.in_w.end(), [](int32_t x) { return x > 0; });
    return finish_graph(c);
}

int wr_route_orders(wr_ctx* c, int32_t n, const int64_t* offs, const int32_t* picks, int32_t* cost, int32_t* perm,
                    int32_t* status, int ptr_kind, void* stream) {
    if (!c || n < 0 || !offs) return WR_EINVAL;
    RC(check_ptr_kind(ptr_kind));
    if (!c->has_graph) return WR_ENOGRAPH;
    if (n > 0 && (!cost || !status)) return WR_EINVAL;
    RC(set_device(c));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // total picks
    int64_t np = 0, first = 0;
    bool selected = false;
    if (ptr_kind == WR_HOST) {
        first = offs[0];
        np = offs[n];
        for (int32_t i = 0; i < n; ++i)
            if (offs[i + 1] < offs[i]) return WR_EINVAL;
    } else if (n > 0 && picks) {
        // offs[0] and offs[n] come back through pinned memory, ordered after the caller's work on
        // its stream; the source selection, which needs neither, is queued before the host waits
        if (!c->h_offs) {
            void* h = nullptr;
            CK(cudaMallocHost(&h, 16));
            c->h_offs = static_cast<int64_t*>(h);
        }
        if (!c->ev_offs) CK(cudaEventCreateWithFlags(&c->ev_offs, cudaEventDisableTiming));
        CK(cudaMemcpyAsync(c->h_offs, offs, 8, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(c->h_offs + 1, offs + n, 8, cudaMemcpyDeviceToHost, s));
        CK(cudaEventRecord(c->ev_offs, s));
        RC(begin_call(c, s));
        RC(enqueue_select(c, n, offs, picks, s));
        selected = true;
        CK(cudaEventSynchronize(c->ev_offs));
        first = c->h_offs[0];
        np = c->h_offs[1];
    } else {
        CK(cudaMemcpyAsync(&first, offs, 8, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&np, offs + n, 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    if (first != 0 || np < 0) return WR_EINVAL;
    if (np > 0 && (!picks || !perm)) return WR_EINVAL;
    if (n == 0) return WR_OK;
    if (!selected) RC(begin_call(c, s));
    // inputs on the device
    const int64_t* d_offs = offs;
    const int32_t* d_picks = picks;
    if (ptr_kind == WR_HOST) {
        RC(ensure(c->offs, (static_cast<size_t>(n) + 1) * 8));
        RC(ensure(c->picks, static_cast<size_t>(np) * 4 + 4));
        CK(cudaMemcpyAsync(c->offs.p, offs, (static_cast<size_t>(n) + 1) * 8, cudaMemcpyHostToDevice, s));
        if (np) CK(cudaMemcpyAsync(c->picks.p, picks, static_cast<size_t>(np) * 4, cudaMemcpyHostToDevice, s));
        d_offs = c->offs.as<int64_t>();
        d_picks = c->picks.as<int32_t>();
    }
    int32_t* o_cost = cost;
    int32_t* o_perm = perm;
    int32_t* o_status = status;
    if (ptr_kind == WR_HOST) {
        RC(ensure(c->out_cost, static_cast<size_t>(n) * 4));
        RC(ensure(c->out_status, static_cast<size_t>(n) * 4));
        RC(ensure(c->out_perm, static_cast<size_t>(np) * 4 + 4));
        o_cost = c->out_cost.as<int32_t>();
        o_status = c->out_status.as<int32_t>();
        o_perm = c->out_perm.as<int32_t>();
    }
    RC(enqueue_route(c, n, d_offs, d_picks, np, o_cost, o_perm, o_status, s, selected));
    RC(end_call(c, s));
    c->last.n_orders = n;
    if (ptr_kind == WR_HOST) {
        CK(cudaMemcpyAsync(cost, o_cost, static_cast<size_t>(n) * 4, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(status, o_status, static_cast<size_t>(n) * 4, cudaMemcpyDeviceToHost, s));
        if (np) CK(cudaMemcpyAsync(perm, o_perm, static_cast<size_t>(np) * 4, cudaMemcpyDeviceToHost, s));
        return finish_host_call(c, s);
    }
    return WR_OK;
}

// Shared driver of wr_bf_rows / wr_distance_rows / wr_submatrix.
typedef int (*seg_fn)(wr_ctx* c, const wr::BfSegment& seg, void* user, cudaStream_t s);

static int rows_driver(wr_ctx* c, int32_t n_src, const int32_t* src, int ptr_kind, seg_fn fn, void* user,
                       cudaStream_t s) {
    if (!c || n_src < 0 || (n_src > 0 && !src)) return WR_EINVAL;
    RC(check_ptr_kind(ptr_kind));
    if (!c->has_graph) return WR_ENOGRAPH;
    RC(set_device(c));
    if (n_src == 0) return WR_OK;
    std::vector<int32_t> hsrc;
    const int32_t* hs = src;
    if (ptr_kind == WR_DEVICE) {
        hsrc.resize(static_cast<size_t>(n_src));
        CK(cudaMemcpyAsync(hsrc.data(), src, static_cast<size_t>(n_src) * 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        hs = hsrc.data();
    }
    for (int32_t i = 0; i < n_src; ++i)
        if (hs[i] < 0 || hs[i] >= c->dg.V) return WR_EINVAL;
    RC(ensure(c->src_in, static_cast<size_t>(n_src) * 4));
    CK(cudaMemcpyAsync(c->src_in.p, hs, static_cast<size_t>(n_src) * 4, cudaMemcpyHostToDevice, s));
    const int32_t lanes_needed = (n_src + 31) / 32 * 32;
    const int32_t blanes = budget_lanes(c);
    if (blanes < 32) return WR_ENOMEM;
    const int32_t seg_lanes = lanes_needed < blanes ? lanes_needed : blanes;
    const int32_t n_seg = (lanes_needed + seg_lanes - 1) / seg_lanes;
    RC(ensure_bf(c, seg_lanes));
    for (int32_t sg = 0; sg < n_seg; ++sg) {
        wr::BfSegment seg;
        seg.rows = c->rows.as<uint32_t>();
        seg.ld = seg_lanes;
        seg.src = c->src_in.as<int32_t>();
        seg.n_src_dev = nullptr;
        seg.n_src_host = n_src;
        seg.first = sg * seg_lanes;
        seg.lanes = seg_lanes;
        RC(run_bf_segment(c, seg, s));
        RC(fn(c, seg, user, s));
    }
    c->last.n_segments = n_seg;
    c->last.n_sources = n_src;
    return WR_OK;
}

struct RowsOut {
    int32_t* rows;
    int64_t ld;
    int host;
};

static int rows_out_fn(wr_ctx* c, const wr::BfSegment& seg, void* user, cudaStream_t s) {
    RowsOut* ro = static_cast<RowsOut*>(user);
    const int32_t V = c->dg.V;
    if (!ro->host) {
        CK(wr::bf_launch_rows_out(seg, V, ro->rows, ro->ld, s));
        c->launches++;
        return WR_OK;
    }
    // host: transpose into a device staging block, then one 2-D copy
    const size_t blk = static_cast<size_t>(seg.lanes) * static_cast<size_t>(V) * 4;
    RC(ensure(c->sub, blk));
    wr::BfSegment shifted = seg;
    shifted.first = 0;
    // lanes of this segment: min(lanes, n_src - first)
    const int32_t count = seg.n_src_host - seg.first < seg.lanes ? seg.n_src_host - seg.first : seg.lanes;
    shifted.n_src_host = count;
    shifted.src = seg.src + seg.first;
    CK(wr::bf_launch_rows_out(shifted, V, c->sub.as<int32_t>(), V, s));
    c->launches++;
    CK(cudaMemcpy2DAsync(ro->rows + static_cast<int64_t>(seg.first) * ro->ld, static_cast<size_t>(ro->ld) * 4,
                         c->sub.p, static_cast<size_t>(V) * 4, static_cast<size_t>(V) * 4,
                         static_cast<size_t>(count), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return WR_OK;
}

int wr_bf_rows(wr_ctx* c, int32_t n_src, const int32_t* src, int32_t* rows, int64_t ld, int ptr_kind, void* stream) {
    if (!c || !rows) return WR_EINVAL;
    if (c->has_graph && ld < c->dg.V) return WR_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    RC(begin_call(c, s));
    RowsOut ro{rows, ld, ptr_kind == WR_HOST};
    RC(rows_driver(c, n_src, src, ptr_kind, rows_out_fn, &ro, s));
    RC(end_call(c, s));
    if (ptr_kind == WR_HOST) return finish_host_call(c, s);
    return WR_OK;
}

struct ConsumeCtx {
    wr_consume_fn fn;
    void* user;
};

static int consume_fn(wr_ctx* c, const wr::BfSegment& seg, void* user, cudaStream_t) {
    ConsumeCtx* cc = static_cast<ConsumeCtx*>(user);
    const int32_t count = seg.n_src_host - seg.first < seg.lanes ? seg.n_src_host - seg.first : seg.lanes;
    (void)c;
    return cc->fn(cc->user, seg.first, count, reinterpret_cast<const int32_t*>(seg.rows), seg.ld);
}

int wr_distance_rows(wr_ctx* c, int32_t n_src, const int32_t* src, int ptr_kind, wr_consume_fn consume, void* user,
                     void* stream) {
    if (!c || !consume) return WR_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    RC(begin_call(c, s));
    ConsumeCtx cc{consume, user};
    RC(rows_driver(c, n_src, src, ptr_kind, consume_fn, &cc, s));
    return end_call(c, s);
}

struct SubCtx {
    int32_t n_dst;
    const int32_t* dst;
    int32_t* sub;
    unsigned long long* check;
};

static int sub_fn(wr_ctx* c, const wr::BfSegment& seg, void* user, cudaStream_t s) {
    SubCtx* sc = static_cast<SubCtx*>(user);
    CK(wr::bf_launch_submatrix(seg, c->dg.V, sc->n_dst, sc->dst, sc->sub, sc->check, s));
    c->launches++;
    return WR_OK;
}

int wr_submatrix(wr_ctx* c, int32_t n_src, const int32_t* src, int32_t n_dst, const int32_t* dst, int32_t* sub,
                 uint64_t* check, int ptr_kind, void* stream) {
    if (!c || n_src < 0 || n_dst < 0 || (n_dst > 0 && !dst) || !sub || !check) return WR_EINVAL;
    RC(check_ptr_kind(ptr_kind));
    if (!c->has_graph) return WR_ENOGRAPH;
    RC(set_device(c));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    RC(begin_call(c, s));
    SubCtx sc{n_dst, dst, sub, reinterpret_cast<unsigned long long*>(check)};
    const int32_t* d_dst = dst;
    if (ptr_kind == WR_HOST) {
        for (int32_t j = 0; j < n_dst; ++j)
            if (dst[j] < 0 || dst[j] >= c->dg.V) return WR_EINVAL;
        RC(ensure(c->kbuf, static_cast<size_t>(n_dst) * 4 + 4));
        RC(ensure(c->dgiven, static_cast<size_t>(n_src) * static_cast<size_t>(n_dst) * 4 + 4));
        RC(ensure(c->check, static_cast<size_t>(n_src) * 8 + 8));
        CK(cudaMemcpyAsync(c->kbuf.p, dst, static_cast<size_t>(n_dst) * 4, cudaMemcpyHostToDevice, s));
        d_dst = c->kbuf.as<int32_t>();
        sc.sub = c->dgiven.as<int32_t>();
        sc.check = c->check.as<unsigned long long>();
    }
    sc.dst = d_dst;
    CK(cudaMemsetAsync(sc.check, 0, static_cast<size_t>(n_src) * 8, s));
    RC(rows_driver(c, n_src, src, ptr_kind, sub_fn, &sc, s));
    RC(end_call(c, s));
    if (ptr_kind == WR_HOST) {
        CK(cudaMemcpyAsync(sub, sc.sub, static_cast<size_t>(n_src) * static_cast<size_t>(n_dst) * 4,
                           cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(check, sc.check, static_cast<size_t>(n_src) * 8, cudaMemcpyDeviceToHost, s));
        return finish_host_call(c, s);
    }
    return WR_OK;
}

int wr_tour_eval(wr_ctx* c, int32_t n, const int32_t* k, const int32_t* D, int32_t* cost, int32_t* perm,
                 int32_t* status, int ptr_kind, void* stream) {
    if (!c || n < 0 || (n > 0 && (!k || !D || !cost || !perm || !status))) return WR_EINVAL;
    RC(check_ptr_kind(ptr_kind));
    RC(set_device(c));
    if (n == 0) return WR_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    RC(begin_call(c, s));
    const int32_t* d_k = k;
    const int32_t* d_D = D;
    const size_t dbytes = static_cast<size_t>(n) * wr::DBLOCK * 4;
    if (ptr_kind == WR_HOST) {
        RC(ensure(c->kbuf, static_cast<size_t>(n) * 4));
        RC(ensure(c->dgiven, dbytes));
        CK(cudaMemcpyAsync(c->kbuf.p, k, static_cast<size_t>(n) * 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(c->dgiven.p, D, dbytes, cudaMemcpyHostToDevice, s));
        d_k = c->kbuf.as<int32_t>();
        d_D = c->dgiven.as<int32_t>();
    }
    wr::TourBufs tb{};
    RC(ensure_tour_bufs(c, n, tb));
    {
        PhaseTimer t(c, s, 3);
        // given 13 x 13 blocks: exhaustive orders only
        CK(wr::tour_launch_prepare_given(n, d_k, d_D, c->cfg.max_k < WR_MAX_K ? c->cfg.max_k : WR_MAX_K, tb, s));
        c->launches++;
    }
    int32_t* o_cost = cost;
    int32_t* o_perm = perm;
    int32_t* o_status = status;
    if (ptr_kind == WR_HOST) {
        RC(ensure(c->out_cost, static_cast<size_t>(n) * 4));
        RC(ensure(c->out_status, static_cast<size_t>(n) * 4));
        RC(ensure(c->out_perm, static_cast<size_t>(n) * WR_MAX_K * 4));
        o_cost = c->out_cost.as<int32_t>();
        o_status = c->out_status.as<int32_t>();
        o_perm = c->out_perm.as<int32_t>();
    }
    RC(run_tours(c, n, d_k, tb, o_cost, o_perm, WR_MAX_K, o_status, s));
    RC(end_call(c, s));
    c->last.n_orders = n;
    if (ptr_kind == WR_HOST) {
        CK(cudaMemcpyAsync(cost, o_cost, static_cast<size_t>(n) * 4, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(status, o_status, static_cast<size_t>(n) * 4, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(perm, o_perm, static_cast<size_t>(n) * WR_MAX_K * 4, cudaMemcpyDeviceToHost, s));
        return finish_host_call(c, s);
    }
    return WR_OK;
}

int wr_get_stats(wr_ctx* c, wr_stats* out) {
    if (!c || !out) return WR_EINVAL;
    RC(set_device(c));
    CK(cudaStreamSynchronize(c->last_stream));
    wr_stats st = c->last;
    unsigned long long h[8] = {0};
    if (c->stats.p) CK(cudaMemcpy(h, c->stats.p, sizeof(h), cudaMemcpyDeviceToHost));
    st.sweeps = static_cast<int64_t>(h[0]);
    st.tile_visits = static_cast<int64_t>(h[1]);
    st.node_visits = static_cast<int64_t>(h[2]);
    st.bytes_alg = static_cast<int64_t>(h[3]);
    st.bytes_reread = static_cast<int64_t>(h[5]);
    st.sequences = static_cast<int64_t>(h[4]);
    st.kernel_launches = c->launches;
    if (c->n_src.p && st.n_sources == 0 && st.n_orders > 0) {
        int32_t ns = 0;
        CK(cudaMemcpy(&ns, c->n_src.p, 4, cudaMemcpyDeviceToHost));
        st.n_sources = ns;
    }
    float* slots[6] = {&st.ms_select, &st.ms_init, &st.ms_bf, &st.ms_gather, &st.ms_enum, &st.ms_finish};
    for (int ph = 0; ph < 6; ++ph) {
        float sum = 0.f;
        for (auto& pr : c->ev_phase[ph]) sum += elapsed(c, pr.first, pr.second);
        *slots[ph] = sum;
    }
    st.ms_total = elapsed(c, c->ev_call_begin, c->ev_call_end);
    *out = st;
    return WR_OK;
}

int wr_set_trace(wr_ctx* c, int32_t max_sweeps) {
    if (!c || max_sweeps < 0 || max_sweeps > (1 << 20)) return WR_EINVAL;
    RC(set_device(c));
    if (max_sweeps > 0) RC(ensure(c->trace, static_cast<size_t>(max_sweeps) * 16));
    c->trace_cap = max_sweeps;
    return WR_OK;
}

int wr_get_trace(wr_ctx* c, int64_t* out, int32_t max_entries, int32_t* n_out) {
    if (!c || !n_out || max_entries < 0 || (max_entries > 0 && !out)) return WR_EINVAL;
    RC(set_device(c));
    *n_out = 0;
    if (c->trace_cap <= 0) return WR_OK;
    CK(cudaStreamSynchronize(c->last_stream));
    std::vector<long long> h(static_cast<size_t>(c->trace_cap) * 2);
    CK(cudaMemcpy(h.data(), c->trace.p, h.size() * 8, cudaMemcpyDeviceToHost));
    int n = 0;
    while (n < c->trace_cap && h[2 * n] >= 0) ++n;
    for (int i = 0; i < n && i < max_entries; ++i) {
        out[2 * i] = h[2 * i];
        out[2 * i + 1] = h[2 * i + 1];
    }
    *n_out = n;
    return WR_OK;
}

int wr_route_nodes(wr_ctx* c, int32_t n, const int64_t* offs, const int32_t* picks, const int32_t* perm,
                   int64_t* node_offs, int32_t* nodes, int64_t max_nodes, int ptr_kind, void* stream) {
    if (!c || n < 0 || !offs || !node_offs || max_nodes < 0) return WR_EINVAL;
    RC(check_ptr_kind(ptr_kind));
    if (!c->has_graph) return WR_ENOGRAPH;
    if (!c->positive_weights) return WR_EINVAL;  // zero-weight arcs: the predecessor rule may cycle
    RC(set_device(c));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int64_t np = 0, first = 0;
    if (ptr_kind == WR_HOST) {
        first = offs[0];
        np = offs[n];
        for (int32_t i = 0; i < n; ++i)
            if (offs[i + 1] < offs[i]) return WR_EINVAL;
    } else {
        CK(cudaMemcpyAsync(&first, offs, 8, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&np, offs + n, 8, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    if (first != 0 || np < 0 || (np > 0 && (!picks || !perm))) return WR_EINVAL;
    if (n == 0) {
        if (ptr_kind == WR_HOST) node_offs[0] = 0;
        else CK(cudaMemsetAsync(node_offs, 0, 8, s));
        return WR_OK;
    }
    const int32_t V = c->dg.V;
    if (!c->in_csr_uploaded) {
        RC(upload(c->g_in_ptr, c->hg.in_ptr.data(), c->hg.in_ptr.size() * 8));
        RC(upload(c->g_in_src, c->hg.in_src.data(), c->hg.in_src.size() * 4));
        RC(upload(c->g_in_w, c->hg.in_w.data(), c->hg.in_w.size() * 4));
        // fixed records of up to 4 in-arcs per node (u = -1 pads; u0 = -2: more arcs, in the CSR)
        std::vector<int32_t> in4(static_cast<size_t>(V) * 8, -1);
        for (int32_t v = 0; v < V; ++v) {
            const int64_t e0 = c->hg.in_ptr[static_cast<size_t>(v)], e1 = c->hg.in_ptr[static_cast<size_t>(v) + 1];
            int32_t* r = in4.data() + static_cast<size_t>(v) * 8;
            if (e1 - e0 > 4) {
                r[0] = -2;
                continue;
            }
            for (int64_t e = e0; e < e1; ++e) {
                r[2 * (e - e0)] = c->hg.in_src[static_cast<size_t>(e)];
                r[2 * (e - e0) + 1] = c->hg.in_w[static_cast<size_t>(e)];
            }
        }
        RC(upload(c->g_in4, in4.data(), in4.size() * 4));
        c->in_csr_uploaded = true;
    }
    RC(begin_call(c, s));
    const int64_t* d_offs = offs;
    const int32_t* d_picks = picks;
    const int32_t* d_perm = perm;
    if (ptr_kind == WR_HOST) {
        RC(ensure(c->offs, (static_cast<size_t>(n) + 1) * 8));
        RC(ensure(c->picks, static_cast<size_t>(np) * 4 + 4));
        RC(ensure(c->perm_in, static_cast<size_t>(np) * 4 + 4));
        CK(cudaMemcpyAsync(c->offs.p, offs, (static_cast<size_t>(n) + 1) * 8, cudaMemcpyHostToDevice, s));
        if (np) {
            CK(cudaMemcpyAsync(c->picks.p, picks, static_cast<size_t>(np) * 4, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(c->perm_in.p, perm, static_cast<size_t>(np) * 4, cudaMemcpyHostToDevice, s));
        }
        d_offs = c->offs.as<int64_t>();
        d_picks = c->picks.as<int32_t>();
        d_perm = c->perm_in.as<int32_t>();
    }
    wr::TourBufs tb{};
    RC(ensure_tour_bufs(c, n, tb));
    const size_t n_legs = static_cast<size_t>(np) + static_cast<size_t>(n);
    RC(ensure(c->leg_len, n_legs * 4 + 4));
    RC(ensure(c->node_offs_d, (static_cast<size_t>(n) + 1) * 8));
    // leg cache: up to LEG_CACHE_NODES nodes per leg, at most LEG_CACHE_WORDS words in all
    const size_t per_leg = LEG_CACHE_WORDS / n_legs;
    const int32_t cache_cap = static_cast<int32_t>(per_leg < LEG_CACHE_NODES ? per_leg : LEG_CACHE_NODES);
    if (cache_cap > 0) RC(ensure(c->leg_cache, n_legs * static_cast<size_t>(cache_cap) * 4));
    CK(wr::tour_launch_select_compact(n, d_offs, d_picks, V, c->dg.depot, c->cfg.max_k, c->node_flag.as<uint8_t>(),
                                      tb.order_status, nullptr, c->src_index.as<int32_t>(), c->src_list.as<int32_t>(),
                                      c->n_src.as<int32_t>(), c->block_sums.as<int32_t>(), s, &c->launches));
    const int64_t worst = np + 1 < V ? np + 1 : V;
    const int32_t lanes_needed = static_cast<int32_t>((worst + 31) / 32 * 32);
    const int32_t blanes = budget_lanes(c);
    if (blanes < 32) return WR_ENOMEM;
    const int32_t seg_lanes = lanes_needed < blanes ? lanes_needed : blanes;
    const int32_t n_seg = (lanes_needed + seg_lanes - 1) / seg_lanes;
    RC(ensure_bf(c, seg_lanes));
    wr::PathsLaunch pl{n, d_offs, d_picks, d_perm, tb.order_status, c->route_mode == WR_ROUTE_OPEN, c->dg.depot,
                       c->src_index.as<int32_t>(), c->g_in_ptr.as<int64_t>(), c->g_in_src.as<int32_t>(),
                       c->g_in_w.as<int32_t>(), c->g_in4.as<int4>(), V, c->leg_len.as<int32_t>(),
                       cache_cap > 0 ? c->leg_cache.as<int32_t>() : nullptr, cache_cap};
    RC(ensure(c->seg_long, static_cast<size_t>(n_seg) * 4));
    CK(cudaMemsetAsync(c->seg_long.p, 0, static_cast<size_t>(n_seg) * 4, s));
    auto segment = [&](int32_t sg) {
        wr::BfSegment seg;
        seg.rows = c->rows.as<uint32_t>();
        seg.ld = seg_lanes;
        seg.src = c->src_list.as<int32_t>();
        seg.sorted = true;  // the distinct sources of the orders, in node id order
        seg.src_index = c->src_index.as<int32_t>();
        seg.n_src_dev = c->n_src.as<int32_t>();
        seg.n_src_host = 0;
        seg.first = sg * seg_lanes;
        seg.lanes = seg_lanes;
        return seg;
    };
    // count walk: every leg's length, in the segment holding its source; short legs cached
    for (int32_t sg = 0; sg < n_seg; ++sg) {
        const wr::BfSegment seg = segment(sg);
        RC(run_bf_segment(c, seg, s));
        PhaseTimer t(c, s, 5);  // the walks are the decode of routes into nodes
        CK(wr::paths_launch(pl, &seg, 0, c->seg_long.as<int32_t>() + sg, nullptr, nullptr, s));
        c->launches++;
    }
    {
        PhaseTimer t(c, s, 5);
        CK(wr::paths_launch_offsets(pl, c->node_offs_d.as<int64_t>(), s));
        c->launches++;
    }
    int64_t total = 0;
    std::vector<int32_t> seg_long(static_cast<size_t>(n_seg));
    CK(cudaMemcpyAsync(&total, c->node_offs_d.as<int64_t>() + n, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(seg_long.data(), c->seg_long.p, static_cast<size_t>(n_seg) * 4, cudaMemcpyDeviceToHost, s));
    if (ptr_kind == WR_HOST)
        CK(cudaMemcpyAsync(node_offs, c->node_offs_d.p, (static_cast<size_t>(n) + 1) * 8, cudaMemcpyDeviceToHost, s));
    else
        CK(cudaMemcpyAsync(node_offs, c->node_offs_d.p, (static_cast<size_t>(n) + 1) * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    RC(take_device_error(c));
    if (!nodes) return WR_OK;
    if (total > max_nodes) return WR_ENOMEM;
    int32_t* d_nodes = nodes;
    if (ptr_kind == WR_HOST) {
        RC(ensure(c->nodes_d, static_cast<size_t>(total) * 4 + 4));
        d_nodes = c->nodes_d.as<int32_t>();
    }
    // cached legs (and each route's first node) straight into the output
    {
        PhaseTimer t(c, s, 5);
        CK(wr::paths_launch(pl, nullptr, 2, nullptr, d_nodes, c->node_offs_d.as<int64_t>(), s));
        c->launches++;
    }
    // legs longer than the cache are walked again in their segment: the last segment's rows are
    // still in place, earlier ones are computed again
    for (int32_t sg = n_seg - 1; sg >= 0; --sg) {
        if (!seg_long[static_cast<size_t>(sg)]) continue;
        const wr::BfSegment seg = segment(sg);
        if (sg != n_seg - 1) RC(run_bf_segment(c, seg, s));
        PhaseTimer t(c, s, 5);
        CK(wr::paths_launch(pl, &seg, 1, nullptr, d_nodes, c->node_offs_d.as<int64_t>(), s));
        c->launches++;
    }
    RC(end_call(c, s));
    if (ptr_kind == WR_HOST) {
        if (total) CK(cudaMemcpyAsync(nodes, d_nodes, static_cast<size_t>(total) * 4, cudaMemcpyDeviceToHost, s));
        return finish_host_call(c, s);
    }
    return WR_OK;
}

int wr_set_node_coords(wr_ctx* c, const int32_t* xy, int ptr_kind) {
    if (!c || !xy) return WR_EINVAL;
    RC(check_ptr_kind(ptr_kind));
    if (!c->has_graph) return WR_ENOGRAPH;
    RC(set_device(c));
    const size_t n = 2 * static_cast<size_t>(c->dg.V);
    c->coords.resize(n);
    if (ptr_kind == WR_HOST) {
        std::memcpy(c->coords.data(), xy, n * 4);
    } else {
        CK(cudaDeviceSynchronize());
        CK(cudaMemcpy(c->coords.data(), xy, n * 4, cudaMemcpyDeviceToHost));
    }
    for (size_t i = 0; i < n; ++i)
        if (c->coords[i] < -(1 << 20) || c->coords[i] > (1 << 20)) {
            c->coords.clear();
            return WR_EINVAL;
        }
    return upload(c->g_coords, c->coords.data(), n * 4);
}

int wr_set_clusters(wr_ctx* c, int32_t m) {
    if (!c || m < 0 || m > 6) return WR_EINVAL;
    c->cluster_m = m;
    return WR_OK;
}

int wr_set_route_mode(wr_ctx* c, int mode) {
    if (!c || (mode != WR_ROUTE_TOUR && mode != WR_ROUTE_OPEN)) return WR_EINVAL;
    c->route_mode = mode;
    return WR_OK;
}

int wr_get_tuning(wr_ctx* c, wr_tuning* out) {
    if (!c || !out) return WR_EINVAL;
    *out = c->tune;
    return WR_OK;
}

int wr_set_tuning(wr_ctx* c, const wr_tuning* t) {
    if (!c || !t || !valid_tuning(t)) return WR_EINVAL;
    RC(set_device(c));
    const bool repart = t->run_target != c->tune.run_target || t->tile_cap != c->tune.tile_cap;
    const bool relaunch = t->bf_warps != c->tune.bf_warps || t->bf_tiling != c->tune.bf_tiling;
    c->tune = *t;
    if (repart && c->has_graph) {
        CK(cudaDeviceSynchronize());
        RC(partition(c));
    } else if (relaunch && c->has_graph) {
        RC(prepare_sweeps(c));
    }
    return WR_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: times the path on a sample batch for candidate tunings.

int wr_autotune(wr_ctx* c, int32_t n, const int64_t* offs, const int32_t* picks, int ptr_kind, int32_t reps,
                wr_tuning* out) {
    if (!c || n < 1 || !offs || reps < 1 || reps > 100) return WR_EINVAL;
    RC(check_ptr_kind(ptr_kind));
    if (!c->has_graph) return WR_ENOGRAPH;
    RC(set_device(c));
    int64_t np = 0;
    if (ptr_kind == WR_HOST) np = offs[n];
    else CK(cudaMemcpy(&np, offs + n, 8, cudaMemcpyDeviceToHost));
    if (np < 0) return WR_EINVAL;
    // outputs of the trial calls, of the inputs' kind
    std::vector<int32_t> h_cost, h_perm, h_status;
    DBuf d_out;
    int32_t *cost, *perm, *status;
    if (ptr_kind == WR_HOST) {
        h_cost.resize(n);
        h_status.resize(n);
        h_perm.resize(static_cast<size_t>(np) + 1);
        cost = h_cost.data();
        perm = h_perm.data();
        status = h_status.data();
    } else {
        RC(ensure(d_out, (2 * static_cast<size_t>(n) + static_cast<size_t>(np) + 1) * 4));
        cost = d_out.as<int32_t>();
        status = cost + n;
        perm = status + n;
    }
    const wr_tuning start = c->tune;
    // median of reps timed calls (after one warm-up), device time of the whole call
    auto trial = [&](float* ms) -> int {
        std::vector<float> t;
        for (int i = 0; i <= reps; ++i) {
            RC(wr_route_orders(c, n, offs, picks, cost, perm, status, ptr_kind, nullptr));
            if (ptr_kind == WR_DEVICE) RC(wr_sync(c));
            wr_stats st;
            RC(wr_get_stats(c, &st));
            if (i > 0) t.push_back(st.ms_total);
        }
        std::sort(t.begin(), t.end());
        *ms = t[t.size() / 2];
        return WR_OK;
    };
    struct BfCand { int tiling, tile_cap, run_target; };
    // run_target about half the tile lets two segments (the faces of an aisle) share one tile
    const BfCand bf[] = {{1, 256, 120}, {1, 128, 60}, {4, 128, 60}, {1, 256, 200}, {3, 128, 60}, {2, 256, 120}, {2, 256, 200}, {2, 512, 240}};
    wr_tuning best = start;
    float best_ms = 3.4e38f;
    int rc = WR_OK;
    for (const BfCand& b : bf) {
        wr_tuning t = start;
        t.bf_tiling = b.tiling;
        t.tile_cap = b.tile_cap;
        t.run_target = b.run_target;
        t.bf_warps = 0;
        if (!valid_tuning(&t)) continue;
        rc = wr_set_tuning(c, &t);
        float ms = 0.f;
        if (rc == WR_OK) rc = trial(&ms);
        if (rc != WR_OK) break;
        if (ms < best_ms) {
            best_ms = ms;
            best = t;
        }
    }
    const int units[] = {1, 2, 4, 8, 16};
    if (rc == WR_OK) rc = wr_set_tuning(c, &best);
    for (int u : units) {
        if (rc != WR_OK) break;
        if (u == best.enum_units) continue;
        wr_tuning t = best;
        t.enum_units = u;
        rc = wr_set_tuning(c, &t);
        float ms = 0.f;
        if (rc == WR_OK) rc = trial(&ms);
        if (rc == WR_OK && ms < best_ms) {
            best_ms = ms;
            best = t;
        }
    }
    const int rc2 = wr_set_tuning(c, rc == WR_OK ? &best : &start);
    if (rc != WR_OK) return rc;
    RC(rc2);
    if (out) *out = best;
    if (!c->tune_path.empty() && !write_tuning_file(c->tune_path, &best)) return WR_EINVAL;
    return WR_OK;
}

// ---------------------------------------------------------------------------
// Batching: the whole path for one fixed-size batch, captured into a CUDA graph.

struct wr_plan {
    wr_ctx* c = nullptr;      // private context: its own graph copy, tuning and work buffers
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int32_t n = 0;
    int64_t max_picks = 0;
    const int64_t* offs = nullptr;
    const int32_t* picks = nullptr;
    int32_t *cost = nullptr, *perm = nullptr, *status = nullptr;
};

void wr_plan_destroy(wr_plan* p) {
    if (!p) return;
    if (p->c) cudaSetDevice(p->c->device);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->c) wr_destroy(p->c);
    delete p;
}

int wr_plan_create(wr_ctx* parent, int32_t n, int64_t max_picks, const int64_t* offs, const int32_t* picks,
                   int32_t* cost, int32_t* perm, int32_t* status, wr_plan** out) {
    if (!parent || !out || n < 1 || max_picks < 0 || !offs || !cost || !status) return WR_EINVAL;
    if (max_picks > 0 && (!picks || !perm)) return WR_EINVAL;
    *out = nullptr;
    if (!parent->has_graph) return WR_ENOGRAPH;
    RC(set_device(parent));
    wr_plan* p = new (std::nothrow) wr_plan();
    if (!p) return WR_ENOMEM;
    p->n = n;
    p->max_picks = max_picks;
    p->offs = offs;
    p->picks = picks;
    p->cost = cost;
    p->perm = perm;
    p->status = status;
    int rc = wr_create(&parent->cfg, &p->c);
    if (rc == WR_OK) {
        wr_ctx* c = p->c;
        c->tune = parent->tune;
        c->route_mode = parent->route_mode;
        c->cluster_m = parent->cluster_m;
        c->hg = parent->hg;  // host copy of the in-arc graph; re-partitioned and uploaded privately
        rc = finish_graph(c);
        if (rc == WR_OK && !parent->coords.empty()) rc = wr_set_node_coords(c, parent->coords.data(), WR_HOST);
    }
    if (rc == WR_OK && cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess) rc = WR_ECUDA;
    // one plain run sizes every buffer, so the captured run allocates nothing
    if (rc == WR_OK) {
        wr_ctx* c = p->c;
        rc = begin_call(c, p->cap);
        if (rc == WR_OK) rc = enqueue_route(c, n, offs, picks, max_picks, cost, perm, status, p->cap);
        if (rc == WR_OK) rc = end_call(c, p->cap);
        if (rc == WR_OK && cudaStreamSynchronize(p->cap) != cudaSuccess) rc = WR_ECUDA;
        if (rc == WR_OK) rc = take_device_error(c);
    }
    if (rc == WR_OK) {
        wr_ctx* c = p->c;
        c->capturing = true;
        if (cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            rc = WR_ECUDA;
        } else {
            rc = begin_call(c, p->cap);
            if (rc == WR_OK) rc = enqueue_route(c, n, offs, picks, max_picks, cost, perm, status, p->cap);
            if (rc == WR_OK) rc = end_call(c, p->cap);
            cudaGraph_t g = nullptr;
            const cudaError_t e = cudaStreamEndCapture(p->cap, &g);
            if (rc == WR_OK && e != cudaSuccess) rc = WR_ECUDA;
            p->graph = g;
        }
        c->capturing = false;
        if (rc == WR_OK && cudaGraphInstantiate(&p->exec, p->graph, 0) != cudaSuccess) rc = WR_ECUDA;
    }
    if (rc != WR_OK) {
        cudaGetLastError();
        wr_plan_destroy(p);
        return rc;
    }
    *out = p;
    return WR_OK;
}

int wr_plan_launch(wr_plan* p, void* stream) {
    if (!p || !p->exec) return WR_EINVAL;
    RC(set_device(p->c));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaGraphLaunch(p->exec, s));
    p->c->last_stream = s;
    return WR_OK;
}

int wr_plan_sync(wr_plan* p) {
    if (!p) return WR_EINVAL;
    RC(set_device(p->c));
    CK(cudaStreamSynchronize(p->c->last_stream));
    return take_device_error(p->c);
}

int wr_plan_get_stats(wr_plan* p, wr_stats* out) {
    if (!p || !out) return WR_EINVAL;
    p->c->last.n_orders = p->n;  // the capture saw no host-side order count
    RC(wr_get_stats(p->c, out));
    return WR_OK;
}

}  // extern "C"
