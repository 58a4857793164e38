// Sequential CPU model of the Bellman-Ford sweep kernel, for the CPU tests.
// It runs the library's own graph preprocessing (wr_graph.cpp) and replays
// the kernel's per-tile forward/backward passes and frontier rules one tile
// at a time, so the algorithm (not the GPU) can be checked against the
// oracle without a device.  It also checks the partition's invariants.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "wr_internal.h"

using namespace wr;

// One tile visit of item (run, 32-source group), as the kernel does it:
// stage, forward pass, backward pass, write back.  Returns 1 if a row
// dropped, 0 if not, 98 if the tile does not fit.
static int relax_item(const HostPartition& p, std::vector<uint32_t>& rows, size_t ld, int G, int tile_cap, int item,
                      std::vector<uint32_t>& tile) {
    const int r = item / G, gg = item % G;
    const int4 rs = p.run_seg[r];
    const int len = rs.y + rs.w;
    auto node = [&](int i) { return i < rs.y ? rs.x + i : rs.z + (i - rs.y); };
    const int h0 = p.halo_ptr[r], hn = p.halo_ptr[r + 1] - h0;
    if (len + hn > tile_cap) return 98;
    bool changed = false;
    for (int lane = 0; lane < 32; ++lane) {
        const size_t c = static_cast<size_t>(gg) * 32 + lane;
        for (int i = 0; i < len; ++i) tile[i] = rows[static_cast<size_t>(node(i)) * ld + c];
        for (int h = 0; h < hn; ++h) tile[len + h] = rows[static_cast<size_t>(p.halo_nodes[h0 + h]) * ld + c];
        std::vector<char> dirty(static_cast<size_t>(len), 0);
        // The kernel walks each pass in chunks of SPAN node ids aligned to
        // multiples of SPAN (ascending forward, descending backward): a node's non-carry
        // arcs read the tile as it was when its chunk started, then
        // the carry chain is solved in pass order.
        constexpr int SPAN = 64;
        std::vector<uint32_t> oth(static_cast<size_t>(len));
        auto src = [&](uint32_t ref) {
            return (ref & GLOBAL_REF) ? rows[static_cast<size_t>(ref & ~GLOBAL_REF) * ld + c] : tile[ref];
        };
        for (int c0 = 0; c0 < len; c0 += SPAN) {
            const int c1 = std::min(len, c0 + SPAN);
            for (int i = c0; i < c1; ++i) {
                const int4 d = p.node_desc[node(i)];
                uint32_t o = 0xFFFFFFFFu;
                for (int a = d.z; a < d.w; ++a) o = std::min(src(p.arc_ref[a]) + p.arc_w[a], o);
                oth[i] = o;
            }
            for (int i = c0; i < c1; ++i) {
                const uint32_t cw = std::min(static_cast<uint32_t>(p.node_desc[node(i)].x), INF_U);
                uint32_t best = std::min(tile[i], oth[i]);
                if (i > 0) best = std::min(tile[i - 1] + cw, best);
                if (best < tile[i]) { tile[i] = best; dirty[i] = 1; changed = true; }
            }
        }
        for (int cb = ((len - 1) / SPAN) * SPAN; cb >= 0; cb -= SPAN) {
            const int top = std::min(len - 1, cb + SPAN - 1), bot = cb - 1;
            for (int i = top; i > bot; --i) {
                const int4 d = p.node_desc[node(i)];
                uint32_t o = 0xFFFFFFFFu;
                for (int a = d.w; a < p.node_desc[node(i) + 1].z; ++a) o = std::min(tile[p.arc_ref[a]] + p.arc_w[a], o);
                oth[i] = o;
            }
            for (int i = top; i > bot; --i) {
                const uint32_t cw = std::min(static_cast<uint32_t>(p.node_desc[node(i)].y), INF_U);
                uint32_t best = std::min(tile[i], oth[i]);
                if (i + 1 < len) best = std::min(tile[i + 1] + cw, best);
                if (best < tile[i]) { tile[i] = best; dirty[i] = 1; changed = true; }
            }
        }
        for (int i = 0; i < len; ++i)
            if (dirty[i]) rows[static_cast<size_t>(node(i)) * ld + c] = tile[i];
    }
    return changed ? 1 : 0;
}

// One tile visit as the warp tiling (wr_bf_warp.cu) does it, lane by lane:
// compact runs fold their forward extras, run the forward pass in blocks of 4
// nodes whose loads precede the previous block's carry chain, fold the
// backward extras, then the backward pass; other runs take the generic path
// (descriptors and arcs in node order, sources past the tile from the rows).
static int relax_item_warp(const HostPartition& p, std::vector<uint32_t>& rows, size_t ld, int G, int tile_cap,
                           int item, std::vector<uint32_t>& tile) {
    constexpr int B = 4;
    const int r = item / G, gg = item % G;
    const int4 rs = p.run_seg[r];
    const int len = rs.y + rs.w;
    auto node = [&](int i) { return i < rs.y ? rs.x + i : rs.z + (i - rs.y); };
    const int h0 = p.halo_ptr[r], hn = p.halo_ptr[r + 1] - h0;
    if (len + hn > tile_cap) return 98;
    const bool compact = (p.run_flags[r] & RUN_COMPACT) != 0;
    const int4 rx = p.run_wx[r];
    if (compact && rx.y + rx.z > wx_cap(tile_cap)) return 97;
    bool changed = false;
    for (int lane = 0; lane < 32; ++lane) {
        const size_t c = static_cast<size_t>(gg) * 32 + lane;
        for (int i = 0; i < len; ++i) tile[i] = rows[static_cast<size_t>(node(i)) * ld + c];
        for (int h = 0; h < hn; ++h) tile[len + h] = rows[static_cast<size_t>(p.halo_nodes[h0 + h]) * ld + c];
        uint32_t chg = 0;
        auto addmin = [](uint32_t a, uint32_t b, uint32_t m) { return std::min(a + b, m); };
        if (compact) {
            auto fold = [&](int e0, int n) {
                for (int e = e0; e < e0 + n; ++e) {
                    const uint2 x = p.wx[static_cast<size_t>(rx.x + e)];
                    const uint32_t d = (x.x & 0xFFFFu) / 128u, sidx = (x.x >> 16) / 128u;
                    if (d >= static_cast<uint32_t>(len) || sidx >= static_cast<uint32_t>(len + hn)) return false;
                    const uint32_t v = addmin(tile[sidx], x.y, tile[d]);
                    chg |= v ^ tile[d];
                    tile[d] = v;
                }
                return true;
            };
            auto pass = [&](bool fwd) {
                const int nf = len / B;
                uint32_t xprev = INF_U;
                struct Blk { uint32_t cur[B], m[B], cw[B]; bool valid[B]; };
                auto load = [&](int b, Blk& k) {
                    const int ib = fwd ? b * B : len - 1 - b * B;
                    for (int j = 0; j < B; ++j) {
                        const int i = fwd ? ib + j : ib - j;
                        k.valid[j] = i >= 0 && i < len;
                        if (!k.valid[j]) {
                            k.cur[j] = INF_U;
                            k.m[j] = INF_U;
                            k.cw[j] = NO_CARRY;
                            continue;
                        }
                        const uint4 d = p.cdesc[2 * static_cast<size_t>(node(i)) + (fwd ? 0 : 1)];
                        k.cur[j] = tile[i];
                        const uint32_t s0 = tile[(d.y & 0xFFFFu) / 128u], s1 = tile[(d.y >> 16) / 128u];
                        k.cw[j] = d.x;
                        k.m[j] = addmin(s1, d.w, addmin(s0, d.z, k.cur[j]));
                    }
                };
                auto chain = [&](int b, const Blk& k) {
                    const int ib = fwd ? b * B : len - 1 - b * B;
                    for (int j = 0; j < B; ++j) {
                        const uint32_t x = addmin(xprev, k.cw[j], k.m[j]);
                        if (k.valid[j]) {
                            tile[fwd ? ib + j : ib - j] = x;
                            chg |= x ^ k.cur[j];
                        }
                        xprev = x;
                    }
                };
                Blk a, nb;
                if (nf > 0) load(0, a);
                for (int b = 0; b < nf; ++b) {
                    if (b + 1 < nf) load(b + 1, nb);
                    chain(b, a);
                    a = nb;
                }
                if (nf * B < len) {
                    load(nf, a);
                    chain(nf, a);
                }
            };
            if (!fold(0, rx.y)) return 96;
            pass(true);
            if (!fold(rx.y, rx.z)) return 96;
            pass(false);
        } else {
            uint32_t carry = INF_U;
            for (int i = 0; i < len; ++i) {
                const int4 d = p.node_desc[node(i)];
                const uint32_t cur = tile[i];
                uint32_t best = addmin(carry, static_cast<uint32_t>(d.x), cur);
                for (int a = d.z; a < d.w; ++a) {
                    const uint32_t ref = p.arc_ref[a];
                    const uint32_t x = (ref & GLOBAL_REF) ? rows[static_cast<size_t>(ref & ~GLOBAL_REF) * ld + c] : tile[ref];
                    best = addmin(x, p.arc_w[a], best);
                }
                tile[i] = best;
                chg |= best ^ cur;
                carry = best;
            }
            carry = INF_U;
            for (int i = len - 1; i >= 0; --i) {
                const int4 d = p.node_desc[node(i)];
                const int end = p.node_desc[node(i) + 1].z;
                const uint32_t cur = tile[i];
                uint32_t best = addmin(carry, static_cast<uint32_t>(d.y), cur);
                for (int a = d.w; a < end; ++a) best = addmin(tile[p.arc_ref[a]], p.arc_w[a], best);
                tile[i] = best;
                chg |= best ^ cur;
                carry = best;
            }
        }
        if (chg) {
            changed = true;
            for (int i = 0; i < len; ++i) rows[static_cast<size_t>(node(i)) * ld + c] = tile[i];
        }
    }
    return changed ? 1 : 0;
}

static void setup(int V, long long E, const long long* rp, const int* col, const int* w, int run_target, int tile_cap,
                  HostGraph& g, HostPartition& p, int& rc) {
    rc = build_host_graph(V, E, reinterpret_cast<const int64_t*>(rp), col, w, 0, g);
    if (!rc) build_partition(g, run_target, tile_cap, p);
}

static void copy_out(const std::vector<uint32_t>& rows, size_t ld, int V, int n_src, int* out) {
    for (int b = 0; b < n_src; ++b)
        for (int v = 0; v < V; ++v) out[static_cast<size_t>(b) * V + v] = static_cast<int>(rows[static_cast<size_t>(v) * ld + b]);
}

extern "C" int bfm_rows(int V, long long E, const long long* rp, const int* col, const int* w, int n_src,
                        const int* src, int run_target, int tile_cap, int* out, int* sweeps_out) {
    HostGraph g;
    HostPartition p;
    int rc = 0;
    setup(V, E, rp, col, w, run_target, tile_cap, g, p, rc);
    if (rc) return rc;
    const int G = (n_src + 31) / 32;
    const size_t ld = static_cast<size_t>(G) * 32;
    std::vector<uint32_t> rows(static_cast<size_t>(V) * ld, INF_U);
    for (int b = 0; b < n_src; ++b) rows[static_cast<size_t>(src[b]) * ld + b] = 0;
    std::vector<int> stamp(static_cast<size_t>(p.n_runs) * G, 0);
    for (int b = 0; b < n_src; ++b) stamp[static_cast<size_t>(p.run_of_node[src[b]]) * G + b / 32] = 1;
    auto build = [&](int match) {
        std::vector<int> l;
        for (int it = 0; it < p.n_runs * G; ++it) {
            const int r = it / G, gg = it % G;
            bool act = stamp[it] == match;
            for (int q = p.rin_ptr[r]; !act && q < p.rin_ptr[r + 1]; ++q)
                act = stamp[static_cast<size_t>(p.rin_list[q]) * G + gg] == match;
            if (act) l.push_back(it);
        }
        return l;
    };
    std::vector<int> list = build(1);
    int sweep = 1;
    std::vector<uint32_t> tile(static_cast<size_t>(tile_cap));
    for (;; ++sweep) {
        if (list.empty()) break;
        if (sweep > V + 1) return 99;
        for (int item : list) {
            const int c = relax_item(p, rows, ld, G, tile_cap, item, tile);
            if (c > 1) return c;
            if (c) stamp[item] = sweep + 1;
        }
        list = build(sweep + 1);
    }
    *sweeps_out = sweep - 1;
    copy_out(rows, ld, V, n_src, out);
    return 0;
}

// The warp tiling's sweeps (default tiling): the frontier of each sweep is
// the tiles that changed in the previous one and the tiles of the runs they
// feed (the kernel pushes them; the set is the same), visited one at a time.
// compact_out: the share of runs on the compact path.
extern "C" int bfm_rows_warp(int V, long long E, const long long* rp, const int* col, const int* w, int n_src,
                             const int* src, int run_target, int tile_cap, int* out, int* sweeps_out,
                             double* compact_out) {
    HostGraph g;
    HostPartition p;
    int rc = 0;
    setup(V, E, rp, col, w, run_target, tile_cap, g, p, rc);
    if (rc) return rc;
    const int G = (n_src + 31) / 32;
    const size_t ld = static_cast<size_t>(G) * 32;
    std::vector<uint32_t> rows(static_cast<size_t>(V) * ld, INF_U);
    for (int b = 0; b < n_src; ++b) rows[static_cast<size_t>(src[b]) * ld + b] = 0;
    const size_t n_items = static_cast<size_t>(p.n_runs) * G;
    std::vector<int> stamp(n_items, 0), list;
    auto push = [&](int item, int s, std::vector<int>& l) {
        if (stamp[item] < s) {
            stamp[item] = s;
            l.push_back(item);
        }
    };
    for (int b = 0; b < n_src; ++b) {
        const int r = p.run_of_node[src[b]];
        push(r * G + b / 32, 1, list);
        for (int k = p.rout_ptr[r]; k < p.rout_ptr[r + 1]; ++k) push(p.rout_list[k] * G + b / 32, 1, list);
    }
    std::vector<uint32_t> tile(static_cast<size_t>(tile_cap));
    int sweep = 1;
    for (;; ++sweep) {
        if (list.empty()) break;
        if (sweep > V + 1) return 99;
        std::vector<int> next;
        for (int item : list) {
            const int c = relax_item_warp(p, rows, ld, G, tile_cap, item, tile);
            if (c > 1) return c;
            if (c) {
                push(item, sweep + 1, next);
                const int r = item / G;
                for (int k = p.rout_ptr[r]; k < p.rout_ptr[r + 1]; ++k) push(p.rout_list[k] * G + item % G, sweep + 1, next);
            }
        }
        list.swap(next);
    }
    *sweeps_out = sweep - 1;
    int compact = 0;
    for (int r = 0; r < p.n_runs; ++r) compact += (p.run_flags[r] & RUN_COMPACT) ? 1 : 0;
    *compact_out = static_cast<double>(compact) / p.n_runs;
    copy_out(rows, ld, V, n_src, out);
    return 0;
}

// The asynchronous worklist (bf_tiling 3) replayed one visit at a time: the
// seeds are each source's run and the runs it feeds (rout); a visit that
// drops a row requests the item itself and the items of the runs it feeds;
// an item already waiting is not queued twice.  Visits are taken from the
// waiting set in a seeded random order (order = 0: first in, first out), so
// the fixpoint must not depend on the order.  visits_out: tile visits.
// seed_fed = 0 leaves the fed runs out of the seeds (a planted omission).
extern "C" int bfm_rows_worklist(int V, long long E, const long long* rp, const int* col, const int* w, int n_src,
                                 const int* src, int run_target, int tile_cap, unsigned long long order,
                                 int seed_fed, int* out, long long* visits_out) {
    HostGraph g;
    HostPartition p;
    int rc = 0;
    setup(V, E, rp, col, w, run_target, tile_cap, g, p, rc);
    if (rc) return rc;
    const int G = (n_src + 31) / 32;
    const size_t ld = static_cast<size_t>(G) * 32;
    const long long n_items = static_cast<long long>(p.n_runs) * G;
    std::vector<uint32_t> rows(static_cast<size_t>(V) * ld, INF_U);
    for (int b = 0; b < n_src; ++b) rows[static_cast<size_t>(src[b]) * ld + b] = 0;
    std::vector<char> queued(static_cast<size_t>(n_items), 0);
    std::vector<int> q;
    auto push = [&](int item) {
        if (!queued[item]) {
            queued[item] = 1;
            q.push_back(item);
        }
    };
    auto push_fed = [&](int r, int gg) {
        for (int k = p.rout_ptr[r]; k < p.rout_ptr[r + 1]; ++k) push(p.rout_list[k] * G + gg);
    };
    for (int b = 0; b < n_src; ++b) {
        const int r = p.run_of_node[src[b]];
        push(r * G + b / 32);
        if (seed_fed) push_fed(r, b / 32);  // 0: a planted omission for the tests
    }
    std::vector<uint32_t> tile(static_cast<size_t>(tile_cap));
    unsigned long long x = order;
    size_t head = 0;
    long long visits = 0;
    while (head < q.size()) {
        if (visits > (static_cast<long long>(V) + 2) * n_items) return 99;
        if (order) {  // swap a random waiting item to the front
            x ^= x << 13;
            x ^= x >> 7;
            x ^= x << 17;
            std::swap(q[head], q[head + x % (q.size() - head)]);
        }
        const int item = q[head++];
        queued[item] = 0;
        const int c = relax_item(p, rows, ld, G, tile_cap, item, tile);
        if (c > 1) return c;
        ++visits;
        if (c) {
            push(item);
            push_fed(item / G, item % G);
        }
    }
    *visits_out = visits;
    copy_out(rows, ld, V, n_src, out);
    return 0;
}

// Partition invariants; returns 0 or a non-zero code naming the broken rule.
extern "C" int bfm_check_partition(int V, long long E, const long long* rp, const int* col, const int* w,
                                   int run_target, int tile_cap, int* n_runs_out) {
    HostGraph g;
    if (build_host_graph(V, E, reinterpret_cast<const int64_t*>(rp), col, w, 0, g)) return 1;
    HostPartition p;
    build_partition(g, run_target, tile_cap, p);
    *n_runs_out = p.n_runs;
    // the runs' segments cover every node once, slots in segment order
    std::vector<int> seen(static_cast<size_t>(V), 0);
    for (int r = 0; r < p.n_runs; ++r) {
        const int4 rs = p.run_seg[r];
        if (rs.y < 1 || rs.y > run_target || rs.w < 0 || rs.w > run_target) return 3;
        for (int i = 0; i < rs.y + rs.w; ++i) {
            const int v = i < rs.y ? rs.x + i : rs.z + (i - rs.y);
            if (v < 0 || v >= V || seen[v]++) return 2;
            if (p.run_of_node[v] != r || p.slot_of_node[v] != i) return 5;
        }
    }
    for (int v = 0; v < V; ++v)
        if (!seen[v]) return 2;
    for (int r = 0; r < p.n_runs; ++r) {
        const int4 rs = p.run_seg[r];
        const int len = rs.y + rs.w;
        auto node = [&](int i) { return i < rs.y ? rs.x + i : rs.z + (i - rs.y); };
        const int hn = p.halo_ptr[r + 1] - p.halo_ptr[r];
        if (len + hn > tile_cap) return 4;
        // every in-arc of the run's nodes appears exactly once, with its weight
        std::vector<int> halo(p.halo_nodes.begin() + p.halo_ptr[r], p.halo_nodes.begin() + p.halo_ptr[r + 1]);
        std::vector<int> runs_in;
        for (int i = 0; i < len; ++i) {
            const int v = node(i);
            const int4 d = p.node_desc[v];
            std::vector<std::pair<int, uint32_t>> got;
            // carries come from the neighbouring slots, which must hold v - 1 / v + 1
            if (static_cast<uint32_t>(d.x) != NO_CARRY) {
                if (i == 0 || node(i - 1) != v - 1) return 17;
                got.emplace_back(v - 1, static_cast<uint32_t>(d.x));
            }
            if (static_cast<uint32_t>(d.y) != NO_CARRY) {
                if (i + 1 >= len || node(i + 1) != v + 1) return 17;
                got.emplace_back(v + 1, static_cast<uint32_t>(d.y));
            }
            const int end = p.node_desc[v + 1].z;
            for (int a = d.z; a < end; ++a) {
                const uint32_t ref = p.arc_ref[a];
                int u;
                const bool fw = a < d.w;
                if (ref & GLOBAL_REF) {
                    u = static_cast<int>(ref & ~GLOBAL_REF);
                    if (!fw) return 9;
                } else if (static_cast<int>(ref) < len) {
                    u = node(static_cast<int>(ref));
                    if (fw && !(static_cast<int>(ref) < i)) return 7;   // forward arcs come from lower slots
                    if (!fw && !(static_cast<int>(ref) > i)) return 8;  // backward arcs from higher slots
                } else {
                    if (static_cast<int>(ref) - len >= hn) return 6;
                    if (!fw) return 9;  // out-of-run sources are read in the forward pass
                    u = halo[ref - len];
                }
                got.emplace_back(u, p.arc_w[a]);
            }
            std::vector<std::pair<int, uint32_t>> want;
            for (int64_t a = g.in_ptr[v]; a < g.in_ptr[v + 1]; ++a)
                want.emplace_back(g.in_src[a], static_cast<uint32_t>(g.in_w[a]));
            std::sort(got.begin(), got.end());
            if (got != want) return 10;
            for (auto& pr : want)
                if (p.run_of_node[pr.first] != r) runs_in.push_back(p.run_of_node[pr.first]);
        }
        // the inline descriptors of a fast-path run hold the same arcs
        if (p.run_flags[r] & RUN_SIMPLE) {
            const int2 rx = p.run_x[r];
            if (rx.y - rx.x > tile_cap) return 12;
            for (int i = 0; i < len; ++i) {
                const int v = node(i);
                const uint4 a = p.node_ix[2 * static_cast<size_t>(v)], b = p.node_ix[2 * static_cast<size_t>(v) + 1];
                const int4 d = p.node_desc[v];
                if (a.x != static_cast<uint32_t>(d.x) || a.y != static_cast<uint32_t>(d.y)) return 13;
                std::vector<std::pair<uint32_t, uint32_t>> fw_ix, bw_ix, fw_l, bw_l;
                if (a.z != NO_CARRY) fw_ix.emplace_back(b.y & 0xFFFFu, a.z);
                if (a.w != NO_CARRY) fw_ix.emplace_back(b.y >> 16, a.w);
                if (b.x != NO_CARRY) bw_ix.emplace_back(b.z & 0xFFFFu, b.x);
                const uint32_t nfx = (b.z >> 16) & 0xFFu, nbx = (b.z >> 25) & 0x7Fu;
                if (!(b.z & IX_EXTRA) && (nfx || nbx)) return 14;
                const uint32_t x0 = static_cast<uint32_t>(rx.x) + b.w;
                if (x0 + nfx + nbx > static_cast<uint32_t>(rx.y)) return 14;
                for (uint32_t q = x0; q < x0 + nfx; ++q) fw_ix.emplace_back(p.xarc2[q].x, p.xarc2[q].y);
                for (uint32_t q = x0 + nfx; q < x0 + nfx + nbx; ++q) bw_ix.emplace_back(p.xarc2[q].x, p.xarc2[q].y);
                for (int q = d.z; q < d.w; ++q) fw_l.emplace_back(p.arc_ref[q], p.arc_w[q]);
                for (int q = d.w; q < p.node_desc[v + 1].z; ++q) bw_l.emplace_back(p.arc_ref[q], p.arc_w[q]);
                std::sort(fw_ix.begin(), fw_ix.end());
                std::sort(bw_ix.begin(), bw_ix.end());
                std::sort(fw_l.begin(), fw_l.end());
                std::sort(bw_l.begin(), bw_l.end());
                if (fw_ix != fw_l || bw_ix != bw_l) return 15;
                for (auto& pr : fw_ix)
                    if (pr.first >= static_cast<uint32_t>(tile_cap)) return 16;
            }
        }
        // the compact descriptors of a warp-tiling run, with the run's extras,
        // hold the same arcs
        if (p.run_flags[r] & RUN_COMPACT) {
            const int4 rx = p.run_wx[r];
            if (rx.x & 1 || rx.y + rx.z > wx_cap(tile_cap) || rx.x + rx.y + rx.z > static_cast<int>(p.wx.size())) return 20;
            std::vector<std::vector<std::pair<uint32_t, uint32_t>>> xf(static_cast<size_t>(len)), xb(static_cast<size_t>(len));
            for (int e = 0; e < rx.y + rx.z; ++e) {
                const uint2 x = p.wx[static_cast<size_t>(rx.x + e)];
                const uint32_t dst = (x.x & 0xFFFFu) / 128u;
                if ((x.x & 127u) || dst >= static_cast<uint32_t>(len)) return 21;
                (e < rx.y ? xf : xb)[dst].emplace_back((x.x >> 16) / 128u, x.y);
            }
            for (int i = 0; i < len; ++i) {
                const int v = node(i);
                const uint4 f = p.cdesc[2 * static_cast<size_t>(v)], bk = p.cdesc[2 * static_cast<size_t>(v) + 1];
                const int4 d = p.node_desc[v];
                if (f.x != static_cast<uint32_t>(d.x) || bk.x != static_cast<uint32_t>(d.y)) return 18;
                std::vector<std::pair<uint32_t, uint32_t>> fc, bc, fw_l, bw_l;
                if (f.z != NO_CARRY) fc.emplace_back((f.y & 0xFFFFu) / 128u, f.z);
                if (f.w != NO_CARRY) fc.emplace_back((f.y >> 16) / 128u, f.w);
                if (bk.z != NO_CARRY) bc.emplace_back((bk.y & 0xFFFFu) / 128u, bk.z);
                if (bk.w != NO_CARRY) bc.emplace_back((bk.y >> 16) / 128u, bk.w);
                if (!xf[i].empty() && fc.size() < 2) return 22;  // extras only beyond two arcs
                if (!xb[i].empty() && bc.size() < 2) return 22;
                fc.insert(fc.end(), xf[i].begin(), xf[i].end());
                bc.insert(bc.end(), xb[i].begin(), xb[i].end());
                for (int q = d.z; q < d.w; ++q) fw_l.emplace_back(p.arc_ref[q], p.arc_w[q]);
                for (int q = d.w; q < p.node_desc[v + 1].z; ++q) bw_l.emplace_back(p.arc_ref[q], p.arc_w[q]);
                std::sort(fc.begin(), fc.end());
                std::sort(bc.begin(), bc.end());
                std::sort(fw_l.begin(), fw_l.end());
                std::sort(bw_l.begin(), bw_l.end());
                if (fc != fw_l || bc != bw_l) return 19;
            }
        }
        std::sort(runs_in.begin(), runs_in.end());
        runs_in.erase(std::unique(runs_in.begin(), runs_in.end()), runs_in.end());
        std::vector<int> rin(p.rin_list.begin() + p.rin_ptr[r], p.rin_list.begin() + p.rin_ptr[r + 1]);
        std::sort(rin.begin(), rin.end());
        if (rin != runs_in) return 11;
    }
    // the runs listed first in the warp sweeps feed at least PRIORITY_FEEDS runs
    for (int r = 0; r < p.n_runs; ++r)
        if (((p.run_flags[r] & RUN_PRIORITY) != 0) != (p.rout_ptr[r + 1] - p.rout_ptr[r] >= PRIORITY_FEEDS)) return 23;
    return 0;
}

// Share of runs that take the kernel's fast path.
extern "C" double bfm_fast_fraction(int V, long long E, const long long* rp, const int* col, const int* w,
                                    int run_target, int tile_cap) {
    HostGraph g;
    if (build_host_graph(V, E, reinterpret_cast<const int64_t*>(rp), col, w, 0, g)) return -1.0;
    HostPartition p;
    build_partition(g, run_target, tile_cap, p);
    int simple = 0;
    for (int r = 0; r < p.n_runs; ++r) simple += (p.run_flags[r] & RUN_SIMPLE) ? 1 : 0;
    return static_cast<double>(simple) / p.n_runs;
}

// Pairing statistics: out[0] = share of runs with two segments, out[1] = staged
// halo slots per own node, out[2] = share of runs with compact descriptors.
extern "C" void bfm_pair_stats(int V, long long E, const long long* rp, const int* col, const int* w, int run_target,
                               int tile_cap, double* out) {
    HostGraph g;
    out[0] = out[1] = out[2] = -1.0;
    if (build_host_graph(V, E, reinterpret_cast<const int64_t*>(rp), col, w, 0, g)) return;
    HostPartition p;
    build_partition(g, run_target, tile_cap, p);
    int paired = 0, compact = 0;
    for (int r = 0; r < p.n_runs; ++r) {
        paired += p.run_seg[r].w > 0 ? 1 : 0;
        compact += (p.run_flags[r] & RUN_COMPACT) ? 1 : 0;
    }
    out[0] = static_cast<double>(paired) / p.n_runs;
    out[1] = static_cast<double>(p.halo_nodes.size()) / V;
    out[2] = static_cast<double>(compact) / p.n_runs;
}
