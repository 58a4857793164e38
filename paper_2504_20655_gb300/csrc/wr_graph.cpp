// Graph load (row a1): validate the out-arc CSR, build the in-arc (pull) CSR
// and partition the nodes into sweep tiles.
//
// Sec. 4.7 stores the graph as an arc list (u, v, w) and relaxes every arc in
// every round.  The sweep kernels instead pull: node v takes
// min(d[v], d[u] + w) over its in-arcs, so each row element has one writer
// and no atomics are needed.  Nodes are grouped into segments of consecutive
// ids, and a tile holds one segment or two that feed each other (both faces
// of an aisle); the tile plus the nodes feeding it from outside (its halo) is
// staged in shared memory and swept forward and backward in slot order, so
// improvements travel along consecutive-id chains inside a tile within one
// sweep, and across the two segments through their shared arcs.
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
    // Distances are int32 with WR_INF = 2^31 - 1 meaning unreachable.  A shortest
    // path is simple (w >= 0), so it has at most V - 1 arcs and uses each arc at most
    // once: its length is at most min((V - 1) * max w, sum of all w).  The graph is
    // accepted only when that bound stays below WR_INF, so every finite distance is
    // exact and none can be mistaken for unreachable.  The bound is taken over the arcs
    // as given (self loops and parallel arcs included).
    int64_t max_w = 0, sum_w = 0;
    for (int64_t a = 0; a < E; ++a) {
        if (col[a] < 0 || col[a] >= V || w[a] < 0) return WR_EINVAL;
        max_w = std::max<int64_t>(max_w, w[a]);
        sum_w = std::min<int64_t>(sum_w + w[a], int64_t(1) << 40);  // saturate: only "< WR_INF" matters
    }
    if (std::min<int64_t>(static_cast<int64_t>(V - 1) * max_w, sum_w) >= WR_INF) return WR_EINVAL;

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

namespace {

// A segment: consecutive node ids [s, e) and the nodes outside it that feed
// it (its halo), in order of first use.
struct Seg {
    int32_t s = 0, e = 0;
    int64_t extra = 0;  // arcs beyond the three inline ones (conservative count)
    std::vector<int32_t> halo;
};

// Segments.  A chain is a maximal range of consecutive ids joined by arcs
// between neighbours (v-1 -> v or v -> v-1); an aisle face is one.  A long
// chain (at least run_target / 2 nodes) is cut into near-equal pieces of at
// most run_target nodes, so two faces of equal length are cut alike and their
// pieces can pair up; short chains are grouped greedily.  Every segment keeps
// own nodes plus halo within tile_cap slots and its extra arcs within tile_cap.
std::vector<Seg> build_segments(const HostGraph& g, int run_target, int tile_cap) {
    const int32_t V = g.V;
    std::vector<char> joined(static_cast<size_t>(V) + 1, 0);  // joined[v]: an arc between v-1 and v
    for (int32_t v = 1; v < V; ++v) {
        for (int64_t a = g.in_ptr[v]; a < g.in_ptr[v + 1] && !joined[v]; ++a)
            if (g.in_src[a] == v - 1) joined[v] = 1;
        for (int64_t a = g.in_ptr[v - 1]; a < g.in_ptr[v] && !joined[v]; ++a)
            if (g.in_src[a] == v) joined[v] = 1;
    }
    std::vector<int32_t> chain_end(static_cast<size_t>(V));
    for (int32_t v = V - 1; v >= 0; --v) chain_end[v] = (v + 1 < V && joined[v + 1]) ? chain_end[v + 1] : v + 1;
    const int32_t long_chain = std::max(2, run_target / 2);
    auto starts_long = [&](int32_t v) { return (v == 0 || !joined[v]) && chain_end[v] - v >= long_chain; };
    std::vector<int32_t> next_long(static_cast<size_t>(V) + 1, V);  // first long-chain start at or after v
    for (int32_t v = V - 1; v >= 0; --v) next_long[v] = starts_long(v) ? v : next_long[v + 1];

    std::vector<Seg> segs;
    std::vector<int32_t> halo_mark(static_cast<size_t>(V), -1);
    std::vector<int32_t> halo_tmp;
    int32_t id = 0, s = 0;
    // grow one segment from s: at most target nodes, not past stop
    auto grow = [&](int32_t target, int32_t stop) {
        int32_t len = 0, halo_cnt = 0;
        int64_t n_extra = 0;
        halo_tmp.clear();
        while (s + len < stop && len < target) {
            const int32_t v = s + len;
            const bool v_in_halo = halo_mark[v] == id;
            int32_t add = 0;
            int64_t listed = 0;
            for (int64_t a = g.in_ptr[v]; a < g.in_ptr[v + 1]; ++a) {
                const int32_t u = g.in_src[a];
                if ((u < s || u > v) && halo_mark[u] != id) ++add;
                if (!(u == v - 1 && u >= s)) ++listed;  // may count the backward carry: conservative
            }
            const int32_t new_cnt = halo_cnt - (v_in_halo ? 1 : 0) + add;
            const int64_t extra = listed > 3 ? listed - 2 : 0;
            if (len > 0 && len + 1 + new_cnt > tile_cap) break;
            if (len > 0 && n_extra + extra > static_cast<int64_t>(tile_cap)) break;
            n_extra += extra;
            if (v_in_halo) {
                halo_mark[v] = -1;
                --halo_cnt;
            }
            for (int64_t a = g.in_ptr[v]; a < g.in_ptr[v + 1]; ++a) {
                const int32_t u = g.in_src[a];
                if ((u < s || u > v) && halo_mark[u] != id) {
                    halo_mark[u] = id;
                    ++halo_cnt;
                    halo_tmp.push_back(u);
                }
            }
            ++len;
        }
        Seg sg;
        sg.s = s;
        sg.e = s + len;
        sg.extra = n_extra;
        for (int32_t u : halo_tmp)
            if (halo_mark[u] == id && (u < sg.s || u >= sg.e)) sg.halo.push_back(u);
        segs.push_back(std::move(sg));
        ++id;
        s += len;
    };
    while (s < V) {
        if (starts_long(s)) {
            const int32_t ce = chain_end[s];
            const int32_t pieces = (ce - s + run_target - 1) / run_target;
            const int32_t piece = (ce - s + pieces - 1) / pieces;
            while (s < ce) grow(piece, ce);
        } else {
            // short chains up to the next long chain
            grow(run_target, next_long[s + 1]);
        }
    }
    return segs;
}

// Pairs of segments that share one tile: a segment and the one holding most
// of its halo (both faces of an aisle, say), when the pair with its merged
// halo fits tile_cap and saves a useful part of the halo.  partner[i] = j or -1.
std::vector<int32_t> pair_segments(const std::vector<Seg>& segs, int32_t V, int tile_cap) {
    const int32_t n = static_cast<int32_t>(segs.size());
    std::vector<int32_t> partner(static_cast<size_t>(n), -1), seg_of(static_cast<size_t>(V));
    for (int32_t i = 0; i < n; ++i)
        for (int32_t v = segs[i].s; v < segs[i].e; ++v) seg_of[v] = i;
    std::vector<int32_t> mark(static_cast<size_t>(V), -1);
    std::vector<std::pair<int32_t, int32_t>> cnt;
    int32_t stamp = 0;
    for (int32_t i = 0; i < n; ++i) {
        if (partner[i] >= 0) continue;
        const Seg& A = segs[i];
        // candidate partners by the number of A's halo nodes they hold
        cnt.clear();
        for (int32_t u : A.halo) cnt.emplace_back(seg_of[u], 1);
        std::sort(cnt.begin(), cnt.end());
        std::vector<std::pair<int32_t, int32_t>> agg;
        for (auto& c : cnt) {
            if (!agg.empty() && agg.back().first == c.first) ++agg.back().second;
            else agg.push_back(c);
        }
        std::sort(agg.begin(), agg.end(), [](auto& x, auto& y) { return x.second > y.second || (x.second == y.second && x.first < y.first); });
        const int32_t lenA = A.e - A.s;
        for (size_t q = 0; q < agg.size() && q < 4; ++q) {
            const int32_t j = agg[q].first;
            if (j == i || partner[j] >= 0) continue;
            const Seg& B = segs[j];
            const int32_t lenB = B.e - B.s;
            if (A.extra + B.extra > static_cast<int64_t>(tile_cap)) continue;
            // merged halo: the union of both halos outside both segments
            ++stamp;
            int32_t merged = 0, shared = 0;
            for (const Seg* X : {&A, &B})
                for (int32_t u : X->halo) {
                    const int32_t su = seg_of[u];
                    if (su == i || su == j) {
                        ++shared;
                        continue;
                    }
                    if (mark[u] != stamp) {
                        mark[u] = stamp;
                        ++merged;
                    }
                }
            if (lenA + lenB + merged > tile_cap) continue;
            if (shared < 8 || 8 * shared < lenA + lenB) continue;
            partner[i] = j;
            partner[j] = i;
            break;
        }
    }
    return partner;
}

}  // namespace

void build_partition(const HostGraph& g, int run_target, int tile_cap, HostPartition& p) {
    const int32_t V = g.V;
    p = HostPartition();
    p.V = V;
    p.tile_cap = tile_cap;
    const std::vector<Seg> segs = build_segments(g, run_target, tile_cap);
    const std::vector<int32_t> partner = pair_segments(segs, V, tile_cap);
    // runs (tiles) in order of their first segment; a paired segment joins its partner's run
    std::vector<std::pair<int32_t, int32_t>> runs;
    for (int32_t i = 0; i < static_cast<int32_t>(segs.size()); ++i)
        if (partner[i] < 0 || partner[i] > i) runs.emplace_back(i, partner[i]);
    const int32_t T = static_cast<int32_t>(runs.size());
    p.n_runs = T;
    p.run_of_node.assign(static_cast<size_t>(V), 0);
    p.slot_of_node.assign(static_cast<size_t>(V), 0);
    p.run_seg.resize(static_cast<size_t>(T));
    std::vector<int32_t> own;
    for (int32_t t = 0; t < T; ++t) {
        const Seg& A = segs[runs[t].first];
        int4 rs = make_int4(A.s, A.e - A.s, 0, 0);
        if (runs[t].second >= 0) {
            const Seg& B = segs[runs[t].second];
            rs.z = B.s;
            rs.w = B.e - B.s;
        }
        p.run_seg[t] = rs;
        for (int32_t i = 0; i < rs.y + rs.w; ++i) {
            const int32_t v = i < rs.y ? rs.x + i : rs.z + (i - rs.y);
            p.run_of_node[v] = t;
            p.slot_of_node[v] = i;
        }
        p.max_len = std::max(p.max_len, rs.y + rs.w);
    }
    // carries: the arc from the previous (next) tile slot when that slot holds node v-1 (v+1)
    auto fw_carry = [&](int32_t v, int32_t u) {
        return u == v - 1 && p.run_of_node[u] == p.run_of_node[v] && p.slot_of_node[u] + 1 == p.slot_of_node[v];
    };
    auto bw_carry = [&](int32_t v, int32_t u) {
        return u == v + 1 && p.run_of_node[u] == p.run_of_node[v] && p.slot_of_node[u] == p.slot_of_node[v] + 1;
    };
    // listed arcs (all in-arcs but the carries) at positions in node id order
    std::vector<int64_t> astart(static_cast<size_t>(V) + 1, 0);
    for (int32_t v = 0; v < V; ++v) {
        int64_t c = 0;
        for (int64_t a = g.in_ptr[v]; a < g.in_ptr[v + 1]; ++a) {
            const int32_t u = g.in_src[a];
            if (!fw_carry(v, u) && !bw_carry(v, u)) ++c;
        }
        astart[v + 1] = astart[v] + c;
    }
    p.node_desc.resize(static_cast<size_t>(V) + 1);
    p.arc_ref.resize(static_cast<size_t>(astart[V]));
    p.arc_w.resize(static_cast<size_t>(astart[V]));
    p.node_ix.assign(2 * (static_cast<size_t>(V) + 1), make_uint4(NO_CARRY, NO_CARRY, NO_CARRY, NO_CARRY));
    p.cdesc.assign(2 * (static_cast<size_t>(V) + 1), make_uint4(NO_CARRY, 0u, NO_CARRY, NO_CARRY));
    p.run_x.resize(static_cast<size_t>(T));
    p.halo_ptr.push_back(0);
    p.rin_ptr.push_back(0);
    std::vector<int32_t> htile(static_cast<size_t>(V), -1), hslot(static_cast<size_t>(V), -1);
    std::vector<int32_t> halo_all, rin_tmp;
    std::vector<uint2> xt;
    std::vector<std::pair<uint32_t, uint32_t>> fw, bw;
    std::vector<uint2> wxf, wxb;
    auto off = [](uint32_t slot) { return slot * 128u; };
    for (int32_t t = 0; t < T; ++t) {
        const int4 rs = p.run_seg[t];
        const int32_t len = rs.y + rs.w;
        own.clear();
        for (int32_t i = 0; i < len; ++i) own.push_back(i < rs.y ? rs.x + i : rs.z + (i - rs.y));
        // halo in order of first use (own nodes in slot order, in-arcs in CSR order)
        halo_all.clear();
        for (int32_t v : own)
            for (int64_t a = g.in_ptr[v]; a < g.in_ptr[v + 1]; ++a) {
                const int32_t u = g.in_src[a];
                if (p.run_of_node[u] != t && htile[u] != t) {
                    htile[u] = t;
                    halo_all.push_back(u);
                }
            }
        const int32_t staged = std::min<int32_t>(static_cast<int32_t>(halo_all.size()), std::max(0, tile_cap - len));
        for (int32_t h = 0; h < static_cast<int32_t>(halo_all.size()); ++h) {
            hslot[halo_all[h]] = h < staged ? len + h : -1;
            if (h < staged) p.halo_nodes.push_back(halo_all[h]);
        }
        p.halo_ptr.push_back(static_cast<int32_t>(p.halo_nodes.size()));
        xt.clear();
        bool any_not_inline = false, compact = staged == static_cast<int32_t>(halo_all.size()) && tile_cap <= 512;
        int64_t arcs_in_run = 0;
        for (int32_t v : own) {
            const uint32_t sv = static_cast<uint32_t>(p.slot_of_node[v]);
            uint32_t fw_cw = NO_CARRY, bw_cw = NO_CARRY;
            fw.clear();
            bw.clear();
            for (int64_t a = g.in_ptr[v]; a < g.in_ptr[v + 1]; ++a) {
                const int32_t u = g.in_src[a];
                const uint32_t wt = static_cast<uint32_t>(g.in_w[a]);
                ++arcs_in_run;
                if (fw_carry(v, u)) {
                    fw_cw = wt;
                } else if (bw_carry(v, u)) {
                    bw_cw = wt;
                } else if (p.run_of_node[u] == t) {
                    const uint32_t su = static_cast<uint32_t>(p.slot_of_node[u]);
                    (su < sv ? fw : bw).emplace_back(su, wt);
                } else if (hslot[u] >= 0) {
                    fw.emplace_back(static_cast<uint32_t>(hslot[u]), wt);
                } else {
                    fw.emplace_back(GLOBAL_REF | static_cast<uint32_t>(u), wt);
                    ++p.n_global_refs;
                }
            }
            // generic form: forward arcs then backward arcs, at the node's id-order position
            int64_t q = astart[v];
            int4 d;
            d.x = static_cast<int>(fw_cw);
            d.y = static_cast<int>(bw_cw);
            d.z = static_cast<int>(q);
            for (auto& pr : fw) {
                p.arc_ref[q] = pr.first;
                p.arc_w[q++] = pr.second;
            }
            d.w = static_cast<int>(q);
            for (auto& pr : bw) {
                p.arc_ref[q] = pr.first;
                p.arc_w[q++] = pr.second;
            }
            p.node_desc[v] = d;
            // inline form (CTA tiling): two forward and one backward non-carry arcs, the rest in the run's extras
            const uint32_t nfx = fw.size() > 2 ? static_cast<uint32_t>(fw.size() - 2) : 0u;
            const uint32_t nbx = bw.size() > 1 ? static_cast<uint32_t>(bw.size() - 1) : 0u;
            const uint32_t s0 = fw.size() > 0 ? fw[0].first : 0u, s1 = fw.size() > 1 ? fw[1].first : 0u;
            const uint32_t sb = bw.size() > 0 ? bw[0].first : 0u;
            const bool inline_ok = s0 < 0x10000u && s1 < 0x10000u && sb < 0x10000u && nfx < 256u && nbx < 128u &&
                                   !((s0 | s1) & GLOBAL_REF);
            if (!inline_ok) any_not_inline = true;
            uint4 ia, ib;
            ia.x = fw_cw;
            ia.y = bw_cw;
            ia.z = fw.size() > 0 ? fw[0].second : NO_CARRY;
            ia.w = fw.size() > 1 ? fw[1].second : NO_CARRY;
            ib.x = bw.size() > 0 ? bw[0].second : NO_CARRY;
            ib.y = (s0 & 0xFFFFu) | (s1 << 16);
            ib.z = (sb & 0xFFFFu) | ((nfx & 0xFFu) << 16) | ((nfx + nbx) ? IX_EXTRA : 0u) | ((nbx & 0x7Fu) << 25);
            ib.w = static_cast<uint32_t>(xt.size());
            for (size_t k = 2; k < fw.size(); ++k) xt.push_back(make_uint2(fw[k].first, fw[k].second));
            for (size_t k = 1; k < bw.size(); ++k) xt.push_back(make_uint2(bw[k].first, bw[k].second));
            p.node_ix[2 * static_cast<size_t>(v)] = ia;
            p.node_ix[2 * static_cast<size_t>(v) + 1] = ib;
            // compact form (warp tiling): two non-carry arcs per pass in the
            // descriptor, the rest in the run's extras; all in staged slots
            bool c_ok = true;
            for (auto& pr : fw) c_ok = c_ok && !(pr.first & GLOBAL_REF) && pr.first < static_cast<uint32_t>(tile_cap);
            for (auto& pr : bw) c_ok = c_ok && pr.first < static_cast<uint32_t>(tile_cap);
            for (size_t k = 2; c_ok && k < fw.size(); ++k)
                wxf.push_back(make_uint2(off(sv) | (off(fw[k].first) << 16), fw[k].second));
            for (size_t k = 2; c_ok && k < bw.size(); ++k)
                wxb.push_back(make_uint2(off(sv) | (off(bw[k].first) << 16), bw[k].second));
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
        }
        // warp tiling extras: at most wx_cap(tile_cap) entries fit the warp's shared memory
        if (wxf.size() + wxb.size() > static_cast<size_t>(wx_cap(tile_cap))) compact = false;
        p.run_wx.push_back(compact ? make_int4(static_cast<int>(p.wx.size()), static_cast<int>(wxf.size()),
                                               static_cast<int>(wxb.size()), 0)
                                   : make_int4(static_cast<int>(p.wx.size()), 0, 0, 0));
        if (compact) {
            p.wx.insert(p.wx.end(), wxf.begin(), wxf.end());
            p.wx.insert(p.wx.end(), wxb.begin(), wxb.end());
            if (p.wx.size() & 1u) p.wx.push_back(make_uint2(0u, NO_CARRY));  // whole 16-byte pairs per run
        }
        wxf.clear();
        wxb.clear();
        p.run_x[t] = make_int2(static_cast<int>(p.xarc2.size()), static_cast<int>(p.xarc2.size() + xt.size()));
        p.xarc2.insert(p.xarc2.end(), xt.begin(), xt.end());
        p.run_meta_bytes.push_back(8 * arcs_in_run + 8 * static_cast<int64_t>(len));
        const bool simple = static_cast<int64_t>(xt.size()) <= static_cast<int64_t>(tile_cap) &&
                            staged == static_cast<int32_t>(halo_all.size()) && !any_not_inline;
        p.run_flags.push_back((simple ? RUN_SIMPLE : 0) | (compact ? RUN_COMPACT : 0));
        // runs feeding this one: the runs of its halo nodes
        rin_tmp.clear();
        for (int32_t u : halo_all) rin_tmp.push_back(p.run_of_node[u]);
        std::sort(rin_tmp.begin(), rin_tmp.end());
        rin_tmp.erase(std::unique(rin_tmp.begin(), rin_tmp.end()), rin_tmp.end());
        p.rin_list.insert(p.rin_list.end(), rin_tmp.begin(), rin_tmp.end());
        p.rin_ptr.push_back(static_cast<int32_t>(p.rin_list.size()));
    }
    // runs fed by each run: rin transposed, ascending
    p.rout_ptr.assign(static_cast<size_t>(p.n_runs) + 1, 0);
    p.rout_list.assign(p.rin_list.size(), 0);
    for (int32_t r = 0; r < p.n_runs; ++r)
        for (int32_t q = p.rin_ptr[r]; q < p.rin_ptr[r + 1]; ++q) ++p.rout_ptr[p.rin_list[q] + 1];
    for (int32_t r = 0; r < p.n_runs; ++r) p.rout_ptr[r + 1] += p.rout_ptr[r];
    {
        std::vector<int32_t> fill(p.rout_ptr.begin(), p.rout_ptr.end() - 1);
        for (int32_t r = 0; r < p.n_runs; ++r)
            for (int32_t q = p.rin_ptr[r]; q < p.rin_ptr[r + 1]; ++q) p.rout_list[fill[p.rin_list[q]]++] = r;
    }
    // runs that feed many others (the cross-aisle pieces, which feed every aisle they cross)
    // are listed first in every sweep of the warp tiling
    for (int32_t r = 0; r < p.n_runs; ++r)
        if (p.rout_ptr[r + 1] - p.rout_ptr[r] >= PRIORITY_FEEDS) p.run_flags[r] |= RUN_PRIORITY;
    int4 sentinel;
    sentinel.x = static_cast<int>(NO_CARRY);
    sentinel.y = static_cast<int>(NO_CARRY);
    sentinel.z = static_cast<int>(astart[V]);
    sentinel.w = sentinel.z;
    p.node_desc[V] = sentinel;
}


}  // namespace wr
