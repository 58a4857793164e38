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
constexpr int SPAN = 64;

int pos_of(int i) { return (i & ~63) | ((i & 1) << 5) | ((i >> 1) & 31); }

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
    int p_own[2], p0[2], p1[2];
    bool valid[2];
    uint32_t w[2], S[2], w0[2], w1[2], xb[2], xe[2];
};

}  // namespace

namespace {

// One pass over a staged tile (the kernel's scan_pass, all 32 lanes at once).
bool scan_pass(Smem& sm, bool fwd, int len, uint32_t x0) {
    bool changed = false;
    const int nchunks = (len + SPAN - 1) / SPAN;
    for (int cc = 0; cc < nchunks; ++cc) {
        const int c = fwd ? cc : nchunks - 1 - cc;
        Lane L[32];
        for (int l = 0; l < 32; ++l) {
            for (int j = 0; j < 2; ++j) {
                const int node = fwd ? c * SPAN + 2 * l + j : c * SPAN + 63 - 2 * l - j;
                L[l].valid[j] = node < len;
                const int ii = L[l].valid[j] ? node : 0;
                L[l].p_own[j] = fwd ? c * SPAN + j * 32 + l : c * SPAN + (1 - j) * 32 + 31 - l;
                const uint4 a = sm.ix[2 * ii], b = sm.ix[2 * ii + 1];
                L[l].w[j] = L[l].valid[j] ? std::min(fwd ? a.x : a.y, INF_U) : INF_U;
                L[l].S[j] = j == 0 ? L[l].w[0] : std::min(L[l].S[0] + L[l].w[1], INF_U);
                L[l].p0[j] = pos_of(fwd ? static_cast<int>(b.y & 0xFFFFu) : static_cast<int>(b.z & 0xFFFFu));
                L[l].p1[j] = pos_of(static_cast<int>(b.y >> 16));
                L[l].w0[j] = L[l].valid[j] ? (fwd ? a.z : b.x) : NO_CARRY;
                L[l].w1[j] = L[l].valid[j] ? a.w : NO_CARRY;
                L[l].xb[j] = L[l].xe[j] = 0u;
                if (L[l].valid[j] && (b.z & IX_EXTRA)) {
                    const uint32_t nfx = (b.z >> 16) & 0xFFu;
                    L[l].xb[j] = fwd ? b.w : b.w + nfx;
                    L[l].xe[j] = fwd ? b.w + nfx : sm.ix[2 * ii + 3].w;
                }
            }
        }
        uint32_t W[32][5], acc[32];
        for (int l = 0; l < 32; ++l) acc[l] = L[l].S[1];
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
        uint32_t drop[32][2] = {{0u}};
        for (int q = 0; q < 8; ++q) {
            Q4 cur0[32], cur1[32], L0[32], L1[32], A[32], cin;
            for (int l = 0; l < 32; ++l) {
                cur0[l] = sm.rows[q][L[l].p_own[0]];
                cur1[l] = sm.rows[q][L[l].p_own[1]];
                Q4 a0 = addmin4(sm.rows[q][L[l].p0[0]], L[l].w0[0], cur0[l]);
                Q4 c1 = addmin4(sm.rows[q][L[l].p0[1]], L[l].w0[1], cur1[l]);
                if (fwd) {
                    a0 = addmin4(sm.rows[q][L[l].p1[0]], L[l].w1[0], a0);
                    c1 = addmin4(sm.rows[q][L[l].p1[1]], L[l].w1[1], c1);
                }
                for (uint32_t e = L[l].xb[0]; e < L[l].xe[0]; ++e)
                    a0 = addmin4(sm.rows[q][pos_of(static_cast<int>(sm.xarcs[e - x0].x))], sm.xarcs[e - x0].y, a0);
                for (uint32_t e = L[l].xb[1]; e < L[l].xe[1]; ++e)
                    c1 = addmin4(sm.rows[q][pos_of(static_cast<int>(sm.xarcs[e - x0].x))], sm.xarcs[e - x0].y, c1);
                L0[l] = a0;
                L1[l] = addmin4(a0, L[l].w[1], c1);
                A[l] = L1[l];
            }
            for (int t = 0; t < 4; ++t) cin.v[t] = INF_U;
            if (has_prev) {
                cin = sm.rows[q][p_prev];
                A[0] = addmin4(cin, L[0].S[1], A[0]);
            }
            for (int k = 0; k < 5; ++k) {
                Q4 o[32];
                for (int l = 0; l < 32; ++l) o[l] = A[l >= (1 << k) ? l - (1 << k) : l];
                for (int l = 0; l < 32; ++l) A[l] = addmin4(o[l], W[l][k], A[l]);
            }
            for (int l = 0; l < 32; ++l) {
                const Q4 xin = l == 0 ? cin : A[l - 1];
                const Q4 x0v = addmin4(xin, L[l].S[0], L0[l]);
                const Q4 x1v = addmin4(xin, L[l].S[1], L1[l]);
                if (L[l].valid[0]) sm.rows[q][L[l].p_own[0]] = x0v;
                if (L[l].valid[1]) sm.rows[q][L[l].p_own[1]] = x1v;
                for (int t = 0; t < 4; ++t) {
                    drop[l][0] |= x0v.v[t] ^ cur0[l].v[t];
                    drop[l][1] |= x1v.v[t] ^ cur1[l].v[t];
                }
            }
        }
        for (int l = 0; l < 32; ++l) {
            const int n0 = fwd ? c * SPAN + 2 * l : c * SPAN + 63 - 2 * l;
            if (L[l].valid[0] && drop[l][0]) { sm.dirtyb[n0] = 1; changed = true; }
            if (L[l].valid[1] && drop[l][1]) { sm.dirtyb[fwd ? n0 + 1 : n0 - 1] = 1; changed = true; }
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
            const int r0 = p.run_ptr[r], len = p.run_ptr[r + 1] - r0;
            const int h0 = p.halo_ptr[r], hn = p.halo_ptr[r + 1] - h0;
            const uint32_t x0 = p.node_ix[2 * static_cast<size_t>(r0) + 1].w;
            const uint32_t x1 = p.node_ix[2 * static_cast<size_t>(r0 + len) + 1].w;
            if (stale)
                for (int q = 0; q < 8; ++q)
                    for (int i = len + hn; i < TILE; ++i)
                        for (int c = 0; c < 4; ++c)
                            sm.rows[q][pos_of(i)].v[c] = (i % 3 == 0) ? 0x80010000u + static_cast<uint32_t>(i) : 5u;
            for (int i = 0; i < 2 * (len + 1); ++i) sm.ix[i] = p.node_ix[2 * static_cast<size_t>(r0) + i];
            for (uint32_t q = x0; q < x1; ++q) sm.xarcs[q - x0] = p.xarc2[q];
            const size_t off = static_cast<size_t>(gg) * 32;
            for (int i = 0; i < hn; ++i)
                for (int q = 0; q < 8; ++q)
                    for (int c = 0; c < 4; ++c)
                        sm.rows[q][pos_of(len + i)].v[c] = rows[static_cast<size_t>(p.halo_nodes[h0 + i]) * ld + off + q * 4 + c];
            for (int i = 0; i < len; ++i)
                for (int q = 0; q < 8; ++q)
                    for (int c = 0; c < 4; ++c)
                        sm.rows[q][pos_of(i)].v[c] = rows[static_cast<size_t>(r0 + i) * ld + off + q * 4 + c];
            for (int i = 0; i < len; ++i) sm.dirtyb[i] = 0;
            if (inf_fill)
                for (int t = len + hn; t < ((len + SPAN - 1) / SPAN) * SPAN; ++t)
                    for (int q = 0; q < 8; ++q)
                        for (int c = 0; c < 4; ++c) sm.rows[q][pos_of(t)].v[c] = INF_U;
            const bool f = scan_pass(sm, true, len, x0);
            const bool b = scan_pass(sm, false, len, x0);
            if (f || b) {
                for (int i = 0; i < len; ++i)
                    if (sm.dirtyb[i])
                        for (int q = 0; q < 8; ++q)
                            for (int c = 0; c < 4; ++c)
                                rows[static_cast<size_t>(r0 + i) * ld + off + q * 4 + c] = sm.rows[q][pos_of(i)].v[c];
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
