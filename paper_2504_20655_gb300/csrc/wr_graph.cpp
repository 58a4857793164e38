// Graph load (row a1): validate the out-arc CSR, build the in-arc (pull) CSR
// and partition the nodes into sweep tiles.
//
// Sec. 4.7 stores the graph as an arc list (u, v, w) and relaxes every arc in
// every round.  The sweep kernel instead pulls: node v takes
// min(d[v], d[u] + w) over its in-arcs, so each row element has one writer
// and no atomics are needed.  Nodes are grouped into runs of consecutive ids;
// a run plus the nodes feeding it from outside (its halo) is staged in shared
// memory and swept forward and backward in id order, so improvements travel
// along increasing- or decreasing-id paths inside a run within one sweep.
#include <algorithm>
#include <cstring>
#include <numeric>

#include "wr_internal.h"

namespace wr {

int build_host_graph(int32_t V, int64_t E, const int64_t* row_ptr, const int32_t* col,
                     const int32_t* w, int32_t depot, HostGraph& g) {
    if (V < 1 || E < 0 || !row_ptr || (E > 0 && (!col || !w))) return WR_EINVAL;
    if (depot < 0 || depot >= V) return WR_EINVAL;
    if (row_ptr[0] != 0 || row_ptr[V] != E) return WR_EINVAL;
    for (int32_t u = 0; u < V; ++u)
        if (row_ptr[u + 1] < row_ptr[u]) return WR_EINVAL;
    for (int64_t a = 0; a < E; ++a)
        if (col[a] < 0 || col[a] >= V || w[a] < 0) return WR_EINVAL;

    std::vector<int64_t> cnt(static_cast<size_t>(V) + 1, 0);
    for (int32_t u = 0; u < V; ++u)
        for (int64_t a = row_ptr[u]; a < row_ptr[u + 1]; ++a)
            if (col[a] != u) cnt[static_cast<size_t>(col[a]) + 1]++;
    for (int32_t v = 0; v < V; ++v) cnt[v + 1] += cnt[v];
    std::vector<int32_t> src(static_cast<size_t>(cnt[V])), wt(static_cast<size_t>(cnt[V]));
    std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
    // sources are visited in increasing u, so each in-list comes out sorted by source
    for (int32_t u = 0; u < V; ++u)
        for (int64_t a = row_ptr[u]; a < row_ptr[u + 1]; ++a) {
            int32_t v = col[a];
            if (v == u) continue;  // a self loop never shortens a path (w >= 0)
            int64_t p = pos[v]++;
            src[p] = u;
            wt[p] = w[a];
        }
    // keep the lightest of parallel arcs
    g.V = V;
    g.depot = depot;
    g.in_ptr.assign(static_cast<size_t>(V) + 1, 0);
    g.in_src.clear();
    g.in_w.clear();
    g.in_src.reserve(src.size());
    g.in_w.reserve(src.size());
    for (int32_t v = 0; v < V; ++v) {
        for (int64_t a = cnt[v]; a < cnt[v + 1]; ++a) {
            if (!g.in_src.empty() && static_cast<int64_t>(g.in_src.size()) > g.in_ptr[v] &&
                g.in_src.back() == src[a]) {
                g.in_w.back() = std::min(g.in_w.back(), wt[a]);
                continue;
            }
            g.in_src.push_back(src[a]);
            g.in_w.push_back(wt[a]);
        }
        g.in_ptr[v + 1] = static_cast<int64_t>(g.in_src.size());
    }
    g.E = E;
    return WR_OK;
}

void build_partition(const HostGraph& g, int run_target, int tile_cap, HostPartition& p) {
    const int32_t V = g.V;
    p = HostPartition();
    p.V = V;
    p.tile_cap = tile_cap;
    p.run_of_node.assign(static_cast<size_t>(V), 0);
    p.run_ptr.push_back(0);
    p.halo_ptr.push_back(0);
    p.rin_ptr.push_back(0);
    p.node_desc.resize(static_cast<size_t>(V) + 1);
    p.node_ix.resize(2 * (static_cast<size_t>(V) + 1));
    p.cdesc.assign(2 * (static_cast<size_t>(V) + 1), make_uint4(NO_CARRY, 0u, NO_CARRY, NO_CARRY));

    std::vector<int32_t> halo_mark(static_cast<size_t>(V), -1);  // run id whose halo holds the node
    std::vector<int32_t> slot(static_cast<size_t>(V), 0);        // tile slot within the current run
    std::vector<int32_t> halo_tmp, halo_all, rin_tmp;
    int32_t run = 0;
    int32_t s = 0;
    while (s < V) {
        int32_t len = 0, halo_cnt = 0;
        int64_t n_arcs = 0;  // arcs kept in the run's arc list (all in-arcs but the two carries)
        halo_tmp.clear();
        while (s + len < V && len < run_target) {
            const int32_t v = s + len;
            const bool v_in_halo = halo_mark[v] == run;
            int32_t add = 0;
            int64_t listed = 0;
            for (int64_t a = g.in_ptr[v]; a < g.in_ptr[v + 1]; ++a) {
                int32_t u = g.in_src[a];
                if ((u < s || u > v) && halo_mark[u] != run) ++add;
                if (!(u == v - 1 && u >= s)) ++listed;  // may count the backward carry: conservative
            }
            const int32_t new_cnt = halo_cnt - (v_in_halo ? 1 : 0) + add;
            // extra arcs beyond the inline ones (at most 3 inline), counted conservatively
            const int64_t extra = listed > 3 ? listed - 2 : 0;
            if (len > 0 && len + 1 + new_cnt > tile_cap) break;
            if (len > 0 && n_arcs + extra > static_cast<int64_t>(tile_cap)) break;
            n_arcs += extra;
            if (v_in_halo) {
                halo_mark[v] = -1;
                --halo_cnt;
            }
            for (int64_t a = g.in_ptr[v]; a < g.in_ptr[v + 1]; ++a) {
                int32_t u = g.in_src[a];
                if ((u < s || u > v) && halo_mark[u] != run) {
                    halo_mark[u] = run;
                    ++halo_cnt;
                    halo_tmp.push_back(u);
                }
            }
            ++len;
        }
        const int32_t e = s + len;
        // halo nodes still outside the run, in order of first use
        halo_all.clear();
        for (int32_t u : halo_tmp)
            if (halo_mark[u] == run && (u < s || u >= e)) halo_all.push_back(u);
        const int32_t staged = std::min<int32_t>(static_cast<int32_t>(halo_all.size()),
                                                 std::max(0, tile_cap - len));
        for (int32_t i = 0; i < staged; ++i) {
            slot[halo_all[i]] = len + i;
            p.halo_nodes.push_back(halo_all[i]);
        }
        for (int32_t i = staged; i < static_cast<int32_t>(halo_all.size()); ++i)
            slot[halo_all[i]] = -1;  // read from global memory
        // node descriptors and arcs
        int64_t arcs_in_run = 0;
        bool any_not_inline = false;
        bool compact = true;
        const uint32_t x_first = static_cast<uint32_t>(p.xarc2.size());
        for (int32_t v = s; v < e; ++v) {
            p.run_of_node[v] = run;
            uint32_t fw_cw = NO_CARRY, bw_cw = NO_CARRY;
            std::vector<std::pair<uint32_t, uint32_t>> fw, bw;
            for (int64_t a = g.in_ptr[v]; a < g.in_ptr[v + 1]; ++a) {
                const int32_t u = g.in_src[a];
                const uint32_t wt = static_cast<uint32_t>(g.in_w[a]);
                ++arcs_in_run;
                if (u == v - 1 && u >= s) {
                    fw_cw = wt;
                } else if (u == v + 1 && u < e) {
                    bw_cw = wt;
                } else if (u >= s && u < v) {
                    fw.emplace_back(static_cast<uint32_t>(u - s), wt);
                } else if (u > v && u < e) {
                    bw.emplace_back(static_cast<uint32_t>(u - s), wt);
                } else {
                    const int32_t sl = slot[u];
                    if (sl >= 0) {
                        fw.emplace_back(static_cast<uint32_t>(sl), wt);
                    } else {
                        fw.emplace_back(GLOBAL_REF | static_cast<uint32_t>(u), wt);
                        ++p.n_global_refs;
                    }
                }
            }
            int4 d;
            d.x = static_cast<int>(fw_cw);
            d.y = static_cast<int>(bw_cw);
            d.z = static_cast<int>(p.arc_ref.size());
            for (auto& pr : fw) {
                p.arc_ref.push_back(pr.first);
                p.arc_w.push_back(pr.second);
            }
            d.w = static_cast<int>(p.arc_ref.size());
            for (auto& pr : bw) {
                p.arc_ref.push_back(pr.first);
                p.arc_w.push_back(pr.second);
            }
            p.node_desc[v] = d;
            // inline form: up to two forward and one backward non-carry arcs
            uint4 a, b;
            a.x = fw_cw;
            a.y = bw_cw;
            a.z = fw.size() > 0 ? fw[0].second : NO_CARRY;
            a.w = fw.size() > 1 ? fw[1].second : NO_CARRY;
            const uint32_t s0 = fw.size() > 0 ? fw[0].first : 0u, s1 = fw.size() > 1 ? fw[1].first : 0u;
            const uint32_t sb = bw.size() > 0 ? bw[0].first : 0u;
            b.x = bw.size() > 0 ? bw[0].second : NO_CARRY;
            b.y = (s0 & 0xFFFFu) | (s1 << 16);
            const uint32_t nfx = fw.size() > 2 ? static_cast<uint32_t>(fw.size() - 2) : 0u;
            const uint32_t nbx = bw.size() > 1 ? static_cast<uint32_t>(bw.size() - 1) : 0u;
            const bool inline_ok = s0 < 0x10000u && s1 < 0x10000u && sb < 0x10000u && nfx < 256u &&
                                   !((s0 | s1) & GLOBAL_REF);
            b.z = (sb & 0xFFFFu) | (nfx << 16) | ((nfx + nbx) ? IX_EXTRA : 0u);
            b.w = static_cast<uint32_t>(p.xarc2.size());
            for (size_t q = 2; q < fw.size(); ++q) p.xarc2.push_back(make_uint2(fw[q].first, fw[q].second));
            for (size_t q = 1; q < bw.size(); ++q) p.xarc2.push_back(make_uint2(bw[q].first, bw[q].second));
            if (!inline_ok) any_not_inline = true;
            // compact form: <= 2 non-carry arcs per pass, all in staged tile slots
            auto off = [](uint32_t slot) { return slot * 128u; };
            bool c_ok = fw.size() <= 2 && bw.size() <= 2;
            for (auto& pr : fw) c_ok = c_ok && !(pr.first & GLOBAL_REF) && pr.first < static_cast<uint32_t>(tile_cap);
            for (auto& pr : bw) c_ok = c_ok && pr.first < static_cast<uint32_t>(tile_cap);
            if (c_ok) {
                uint4 f, bk;
                f.x = fw_cw;
                f.y = (fw.size() > 0 ? off(fw[0].first) : 0u) | ((fw.size() > 1 ? off(fw[1].first) : 0u) << 16);
                f.z = fw.size() > 0 ? fw[0].second : NO_CARRY;
                f.w = fw.size() > 1 ? fw[1].second : NO_CARRY;
                bk.x = bw_cw;
                bk.y = (bw.size() > 0 ? off(bw[0].first) : 0u) | ((bw.size() > 1 ? off(bw[1].first) : 0u) << 16);
                bk.z = bw.size() > 0 ? bw[0].second : NO_CARRY;
                bk.w = bw.size() > 1 ? bw[1].second : NO_CARRY;
                p.cdesc[2 * static_cast<size_t>(v)] = f;
                p.cdesc[2 * static_cast<size_t>(v) + 1] = bk;
            } else {
                compact = false;
            }
            p.node_ix[2 * static_cast<size_t>(v)] = a;
            p.node_ix[2 * static_cast<size_t>(v) + 1] = b;
        }
        p.run_meta_bytes.push_back(8 * arcs_in_run + 8 * static_cast<int64_t>(len));
        {
            const int64_t extras = static_cast<int64_t>(p.xarc2.size()) - x_first;
            const bool simple = extras <= static_cast<int64_t>(tile_cap) &&
                                staged == static_cast<int32_t>(halo_all.size()) && !any_not_inline;
            const bool all_staged = staged == static_cast<int32_t>(halo_all.size());
            p.run_flags.push_back((simple ? RUN_SIMPLE : 0) | (compact && all_staged && tile_cap <= 512 ? RUN_COMPACT : 0));
        }
        p.run_ptr.push_back(e);
        p.halo_ptr.push_back(static_cast<int32_t>(p.halo_nodes.size()));
        p.max_len = std::max(p.max_len, len);
        // in-neighbour runs (every halo node lies in an earlier or later run)
        rin_tmp.clear();
        for (int32_t u : halo_all) rin_tmp.push_back(u);
        p.rin_list.insert(p.rin_list.end(), rin_tmp.begin(), rin_tmp.end());  // node ids for now
        p.rin_ptr.push_back(static_cast<int32_t>(p.rin_list.size()));
        ++run;
        s = e;
    }
    p.n_runs = run;
    int4 sentinel;
    sentinel.x = static_cast<int>(NO_CARRY);
    sentinel.y = static_cast<int>(NO_CARRY);
    sentinel.z = static_cast<int>(p.arc_ref.size());
    sentinel.w = sentinel.z;
    p.node_desc[V] = sentinel;
    p.node_ix[2 * static_cast<size_t>(V)] = make_uint4(NO_CARRY, NO_CARRY, NO_CARRY, NO_CARRY);
    p.node_ix[2 * static_cast<size_t>(V) + 1] = make_uint4(NO_CARRY, 0u, 0u, static_cast<uint32_t>(p.xarc2.size()));
    // turn halo node ids into distinct run ids
    std::vector<int32_t> out_ptr(1, 0), out_list;
    for (int32_t r = 0; r < p.n_runs; ++r) {
        rin_tmp.clear();
        for (int32_t i = p.rin_ptr[r]; i < p.rin_ptr[r + 1]; ++i) rin_tmp.push_back(p.run_of_node[p.rin_list[i]]);
        std::sort(rin_tmp.begin(), rin_tmp.end());
        rin_tmp.erase(std::unique(rin_tmp.begin(), rin_tmp.end()), rin_tmp.end());
        for (int32_t q : rin_tmp)
            if (q != r) out_list.push_back(q);
        out_ptr.push_back(static_cast<int32_t>(out_list.size()));
    }
    p.rin_ptr.swap(out_ptr);
    p.rin_list.swap(out_list);
}

}  // namespace wr
