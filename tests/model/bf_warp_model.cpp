// Warp-exact CPU model of the sweep kernel's fast path, for the CPU tests.
//
// It replays, lane by lane and quad by quad, what one warp of
// bf_sweeps_kernel does for a tile: the quad-major shared-memory tile with
// its position permutation, the 64-node chunks of both passes, the per-lane
// 2-node carry chains, the (min, +) shuffle scan with its saturated weight
// prefixes, and the unsigned 32-bit wrap-around of every add.  Before each
// tile the shared memory is filled with adversarial stale contents, so a
// read of a slot the kernel did not stage shows up as a wrong distance.
// Keep it in step with scan_pass / sweep_tile in wr_bf.cu.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "wr_internal.h"

using namespace wr;

namespace {

constexpr int TILE = 256;
constexpr int SEG = 2;
constexpr int SPAN = 32 * SEG;

int pos_of(int i) { return (i & ~(SPAN - 1)) | ((i % SEG) << 5) | ((i / SEG) & 31); }

struct Q4 {
    uint32_t v[4];
};

// min(x + w, m) in 32-bit unsigned arithmetic (the add wraps like the GPU's)
uint32_t am(uint32_t x, uint32_t w, uint32_t m) {
    const uint32_t s = x + w;
    return s < m ? s : m;
}
Q4 addmin4(const Q4& x, uint32_t w, const Q4& m) {
    Q4 r;
    for (int c = 0; c < 4; ++c) r.v[c] = am(x.v[c], w, m.v[c]);
    return r;
}

struct Smem {
    Q4 rows[8][TILE];
    uint4 ix[2 * (TILE + 1)];
    uint2 xarcs[TILE];
    uint8_t dirtyb[TILE];
};

struct Lane {
    int p_own[SEG], p0[SEG], p1[SEG];
    bool valid[SEG];
    uint32_t w[SEG], S[SEG], w0[SEG], w1[SEG], xb[SEG], xe[SEG];
};

}  // namespace

namespace {

// One pass over a staged tile (the kernel's scan_pass, all 32 lanes at once).
bool scan_pass(Smem& sm, bool fwd, int len) {
    bool changed = false;
    const int nchunks = (len + SPAN - 1) / SPAN;
    for (int cc = 0; cc < nchunks; ++cc) {
        const int c = fwd ? cc : nchunks - 1 - cc;
        Lane L[32];
        for (int l = 0; l < 32; ++l) {
            for (int j = 0; j < SEG; ++j) {
                const int node = fwd ? c * SPAN + SEG * l + j : c * SPAN + (SPAN - 1) - SEG * l - j;
                L[l].valid[j] = node < len;
                const int ii = L[l].valid[j] ? node : 0;
                L[l].p_own[j] = fwd ? c * SPAN + j * 32 + l : c * SPAN + (SEG - 1 - j) * 32 + 31 - l;
                const uint4 a = sm.ix[2 * ii], b = sm.ix[2 * ii + 1];
                L[l].w[j] = L[l].valid[j] ? std::min(fwd ? a.x : a.y, INF_U) : INF_U;
                L[l].S[j] = j == 0 ? L[l].w[0] : std::min(L[l].S[j - 1] + L[l].w[j], INF_U);
                L[l].p0[j] = pos_of(fwd ? static_cast<int>(b.y & 0xFFFFu) : static_cast<int>(b.z & 0xFFFFu));
                L[l].p1[j] = pos_of(static_cast<int>(b.y >> 16));
                L[l].w0[j] = L[l].valid[j] ? (fwd ? a.z : b.x) : NO_CARRY;
                L[l].w1[j] = L[l].valid[j] ? a.w : NO_CARRY;
                L[l].xb[j] = L[l].xe[j] = 0u;
                if (L[l].valid[j] && (b.z & IX_EXTRA)) {
                    const uint32_t nfx = (b.z >> 16) & 0xFFu;
                    L[l].xb[j] = fwd ? b.w : b.w + nfx;
                    L[l].xe[j] = b.w + nfx + (fwd ? 0u : (b.z >> 25) & 0x7Fu);
                }
            }
        }
        uint32_t W[32][5], acc[32];
        for (int l = 0; l < 32; ++l) acc[l] = L[l].S[SEG - 1];
        for (int k = 0; k < 5; ++k) {
            uint32_t o[32];
            for (int l = 0; l < 32; ++l) {
                W[l][k] = l >= (1 << k) ? acc[l] : INF_U;
                o[l] = acc[l >= (1 << k) ? l - (1 << k) : l];
            }
            for (int l = 0; l < 32; ++l)
                if (l >= (1 << k)) acc[l] = std::min(acc[l] + o[l], INF_U);
        }
        const int prev = fwd ? c * SPAN - 1 : (c + 1) * SPAN;
        const bool has_prev = fwd ? prev >= 0 : prev < len;
        const int p_prev = pos_of(has_prev ? prev : 0);
        uint32_t drop[32][SEG];
        std::memset(drop, 0, sizeof(drop));
        for (int q = 0; q < 8; ++q) {
            Q4 cur[32][SEG], Lc[32][SEG], A[32], cin;
            for (int l = 0; l < 32; ++l) {
                for (int j = 0; j < SEG; ++j) {
                    cur[l][j] = sm.rows[q][L[l].p_own[j]];
                    Q4 cv = addmin4(sm.rows[q][L[l].p0[j]], L[l].w0[j], cur[l][j]);
                    if (fwd) cv = addmin4(sm.rows[q][L[l].p1[j]], L[l].w1[j], cv);
                    for (uint32_t e = L[l].xb[j]; e < L[l].xe[j]; ++e)
                        cv = addmin4(sm.rows[q][pos_of(static_cast<int>(sm.xarcs[e].x))], sm.xarcs[e].y, cv);
                    Lc[l][j] = j == 0 ? cv : addmin4(Lc[l][j - 1], L[l].w[j], cv);
                }
                A[l] = Lc[l][SEG - 1];
            }
            for (int t = 0; t < 4; ++t) cin.v[t] = INF_U;
            if (has_prev) {
                cin = sm.rows[q][p_prev];
                A[0] = addmin4(cin, L[0].S[SEG - 1], A[0]);
            }
            for (int k = 0; k < 5; ++k) {
                Q4 o[32];
                for (int l = 0; l < 32; ++l) o[l] = A[l >= (1 << k) ? l - (1 << k) : l];
                for (int l = 0; l < 32; ++l) A[l] = addmin4(o[l], W[l][k], A[l]);
            }
            for (int l = 0; l < 32; ++l) {
                const Q4 xin = l == 0 ? cin : A[l - 1];
                for (int j = 0; j < SEG; ++j) {
                    const Q4 x = addmin4(xin, L[l].S[j], Lc[l][j]);
                    if (L[l].valid[j]) sm.rows[q][L[l].p_own[j]] = x;
                    for (int t = 0; t < 4; ++t) drop[l][j] |= x.v[t] ^ cur[l][j].v[t];
                }
            }
        }
        for (int l = 0; l < 32; ++l)
            for (int j = 0; j < SEG; ++j)
                if (L[l].valid[j] && drop[l][j]) {
                    const int node = fwd ? c * SPAN + SEG * l + j : c * SPAN + (SPAN - 1) - SEG * l - j;
                    sm.dirtyb[node] = 1;
                    changed = true;
                }
    }
    return changed;
}

}  // namespace

// Rows of n_src sources, sweeping like the kernel (one tile at a time).
// stale: 0 = shared memory starts clean; 1 = before every tile, every slot the
// tile does not stage holds a mix of values above 2^31 and small values (what
// earlier kernels or tiles may have left).  inf_fill: the kernel's INF fill of
// the unstaged slots of the last 64-block (0 plants its omission).
extern "C" int bwm_rows(int V, long long E, const long long* rp, const int* col, const int* w, int n_src,
                        const int* src, int run_target, int stale, int inf_fill, int* out, int* sweeps_out) {
    HostGraph g;
    if (build_host_graph(V, E, reinterpret_cast<const int64_t*>(rp), col, w, 0, g)) return 1;
    HostPartition p;
    build_partition(g, run_target, TILE, p);
    static Smem sm;
    std::memset(&sm, 0, sizeof(sm));
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
    for (;; ++sweep) {
        if (list.empty()) break;
        if (sweep > V + 1) return 99;
        for (int item : list) {
            const int r = item / G, gg = item % G;
            if (!(p.run_flags[r] & RUN_SIMPLE)) return 97;  // the generic path is not modelled
            const int4 rs = p.run_seg[r];
            const int len = rs.y + rs.w;
            auto node = [&](int i) { return i < rs.y ? rs.x + i : rs.z + (i - rs.y); };
            const int h0 = p.halo_ptr[r], hn = p.halo_ptr[r + 1] - h0;
            const int2 rx = p.run_x[r];
            if (stale)
                for (int q = 0; q < 8; ++q)
                    for (int i = len + hn; i < TILE; ++i)
                        for (int c = 0; c < 4; ++c)
                            sm.rows[q][pos_of(i)].v[c] = (i % 3 == 0) ? 0x80010000u + static_cast<uint32_t>(i) : 5u;
            for (int i = 0; i < 2 * len; ++i) sm.ix[i] = p.node_ix[2 * static_cast<size_t>(node(i >> 1)) + (i & 1)];
            for (int q = rx.x; q < rx.y; ++q) sm.xarcs[q - rx.x] = p.xarc2[q];
            const size_t off = static_cast<size_t>(gg) * 32;
            for (int i = 0; i < hn; ++i)
                for (int q = 0; q < 8; ++q)
                    for (int c = 0; c < 4; ++c)
                        sm.rows[q][pos_of(len + i)].v[c] = rows[static_cast<size_t>(p.halo_nodes[h0 + i]) * ld + off + q * 4 + c];
            for (int i = 0; i < len; ++i)
                for (int q = 0; q < 8; ++q)
                    for (int c = 0; c < 4; ++c)
                        sm.rows[q][pos_of(i)].v[c] = rows[static_cast<size_t>(node(i)) * ld + off + q * 4 + c];
            for (int i = 0; i < len; ++i) sm.dirtyb[i] = 0;
            if (inf_fill)
                for (int t = len + hn; t < ((len + SPAN - 1) / SPAN) * SPAN; ++t)
                    for (int q = 0; q < 8; ++q)
                        for (int c = 0; c < 4; ++c) sm.rows[q][pos_of(t)].v[c] = INF_U;
            const bool f = scan_pass(sm, true, len);
            const bool b = scan_pass(sm, false, len);
            if (f || b) {
                for (int i = 0; i < len; ++i)
                    if (sm.dirtyb[i])
                        for (int q = 0; q < 8; ++q)
                            for (int c = 0; c < 4; ++c)
                                rows[static_cast<size_t>(node(i)) * ld + off + q * 4 + c] = sm.rows[q][pos_of(i)].v[c];
                stamp[item] = sweep + 1;
            }
        }
        list = build(sweep + 1);
    }
    *sweeps_out = sweep - 1;
    for (int b = 0; b < n_src; ++b)
        for (int v = 0; v < V; ++v) out[static_cast<size_t>(b) * V + v] = static_cast<int>(rows[static_cast<size_t>(v) * ld + b]);
    return 0;
}
