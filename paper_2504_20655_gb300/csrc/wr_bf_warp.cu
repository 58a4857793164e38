// Row a3, warp tiling of the multi-source Bellman-Ford sweeps (Sec. 4.7).
//
// Same rows layout, frontier and sweep loop as the CTA tiling in wr_bf.cu;
// the difference is who owns a (run, 32-source group) tile: here one warp,
// with lane b holding source b of the group.  Shared memory keeps the tile
// slot-major (rows[slot][b], one 128-byte line per node), so a lane only
// ever reads and writes its own column: the relaxation passes need no
// shuffles, no warp barriers and have no bank conflicts (32 lanes read one
// line).  Per node and pass a lane does the min-plus step of the paper for
// the node's in-arcs -- the carry arc from the previous node in pass order
// through a register, up to two other arcs from the staged tile, addressed
// by byte offsets precomputed on the host (compact descriptors).
//
// Staging: cp.async copies of 16 bytes, 8 lanes per 128-byte line (4 lines
// per instruction), in two commit groups -- the descriptors, the halo and the
// first segment, then the second segment -- so the forward pass starts on the
// first segment while the second is in flight.  Write-back: every own line
// of a tile that changed, 16-byte stores from 8 lanes per line.  The warp
// fetches its next tile's index and run metadata while it relaxes the
// current one.
//
// The loads of a block of BLK nodes are issued before the previous block's
// carry chain runs, so a non-carry arc from a node of the previous block
// reads the value from before that block: an upper bound, which only defers
// the improvement to the next sweep (the tile changed, so it is in the next
// frontier).  The fixpoint, and hence every distance, is unchanged.
#include "wr_bf_common.cuh"

namespace wr {

// GPW source groups per warp: lane b holds source b of each group, the
// groups' lines side by side in one slot (a 128 x GPW-byte row per slot).
template <int TILE, int GPW = 1>
struct __align__(128) WarpTile {
    uint32_t rows[TILE][32 * GPW];  // slot-major: rows[i][32 g + b] = source b of group g at tile slot i
    uint4 desc[2 * TILE];           // compact descriptors of the run's nodes: forward, backward
    uint2 wx[wx_cap(TILE)];         // the run's extra arcs: forward, then backward
};

constexpr int BLK = 4;  // nodes per pipelined block

// Run metadata of one work item (the same in every lane).
struct TileMeta {
    int item, r, g, len, h0, hn, flags;
    int hid;    // this lane's halo node (lane < hn), loaded with the metadata when hn <= 32
    bool hids;  // hid holds the halo
    int q0, nq, rq;  // the runs fed: rout_list[q0 .. q0 + nq); rq = this lane's (lane < nq <= 32)
    bool rqp;        // run rq is a priority run
    int ng;   // source groups of the item (GPW, or fewer for the last item of a run)
    int4 rs;  // {a0, alen, b0, blen}
    int4 rx;  // extras {first entry, forward count, backward count, 0}
};

// Item = run x items_per_run + j, its groups GPW j .. GPW j + GPW - 1 (those below G).
template <int GPW>
__device__ __forceinline__ TileMeta load_meta(const BfParams& p, int32_t item, int G, int lane) {
    const int ipr = (G + GPW - 1) / GPW;
    TileMeta m;
    m.item = item;
    m.r = m.item / ipr;
    m.g = (m.item - m.r * ipr) * GPW;
    m.ng = min(GPW, G - m.g);
    m.rs = __ldg(p.g.run_seg + m.r);
    m.len = m.rs.y + m.rs.w;
    m.h0 = __ldg(p.g.halo_ptr + m.r);
    m.hn = __ldg(p.g.halo_ptr + m.r + 1) - m.h0;
    m.flags = __ldg(p.g.run_flags + m.r);
    m.rx = __ldg(p.g.run_wx + m.r);
    // the halo's node ids, one per lane, so that staging needs no dependent load for them
    m.hids = m.hn <= 32;
    m.hid = (m.hids && lane < m.hn) ? __ldg(p.g.halo_nodes + m.h0 + lane) : 0;
    // the runs it feeds, for the frontier pushes after the tile
    m.q0 = __ldg(p.g.rout_ptr + m.r);
    m.nq = __ldg(p.g.rout_ptr + m.r + 1) - m.q0;
    m.rq = lane < m.nq ? __ldg(p.g.rout_list + m.q0 + lane) : 0;
    m.rqp = p.w.prio && lane < m.nq && (__ldg(p.g.run_flags + m.rq) & RUN_PRIORITY) != 0;
    return m;
}

// Byte offset of a descriptor's slot offset (slot x 128) in a GPW-group tile.
template <int GPW>
__device__ __forceinline__ uint32_t line_off(uint32_t o) {
    return GPW == 1 ? o : o * GPW;
}

// Fold n extra arcs into the tile before a pass: each {dst | src << 16, w}
// lowers line dst by line src + w in this lane's columns; changed bits per group.
template <int TILE, int GPW>
__device__ __forceinline__ void fold_extras(WarpTile<TILE, GPW>& t, int e0, int n, int lane, uint32_t (&chg)[GPW]) {
    char* cb = reinterpret_cast<char*>(&t.rows[0][lane]);
#pragma unroll 1
    for (int e = e0; e < e0 + n; ++e) {
        const uint2 x = t.wx[e];
        char* dp = cb + line_off<GPW>(x.x & 0xFFFFu);
        const char* sp = cb + line_off<GPW>(x.x >> 16);
#pragma unroll
        for (int g = 0; g < GPW; ++g) {
            uint32_t* dst = reinterpret_cast<uint32_t*>(dp + 128 * g);
            const uint32_t cur = *dst;
            const uint32_t v = __viaddmin_u32(*reinterpret_cast<const uint32_t*>(sp + 128 * g), x.y, cur);
            *dst = v;
            chg[g] |= v ^ cur;
        }
    }
}

// One block's inputs: current values, the best over the non-carry arcs, carry weight.
template <int GPW>
struct BlkIn {
    uint32_t cur[BLK][GPW], m[BLK][GPW], cw[BLK];
};

// Block b of a pass: nodes ib, ib +- 1, ... (ib = b * BLK forward, len - 1 - b * BLK
// backward).  PART: the block runs past the run's end and its missing nodes
// are neutral (infinite value, blocking weights, no loads).  The descriptor
// and the arc addresses of a node serve all GPW groups.
template <int TILE, int GPW, bool FWD, bool PART>
__device__ __forceinline__ void load_blk(const WarpTile<TILE, GPW>& t, const char* cb, int len, int b,
                                         BlkIn<GPW>& in) {
    constexpr int LINE = 128 * GPW;
    const int ib = FWD ? b * BLK : len - 1 - b * BLK;
    const uint4* dp = &t.desc[2 * ib + (FWD ? 0 : 1)];
    const char* rp = cb + LINE * ib;
    uint4 d[BLK];
    uint32_t s0[BLK][GPW], s1[BLK][GPW];
#pragma unroll
    for (int j = 0; j < BLK; ++j) {
        const int st = FWD ? j : -j;
        const bool valid = !PART || (FWD ? ib + j < len : ib - j >= 0);
        d[j] = valid ? dp[2 * st] : make_uint4(NO_CARRY, 0u, NO_CARRY, NO_CARRY);
    }
#pragma unroll
    for (int j = 0; j < BLK; ++j) {
        const int st = FWD ? j : -j;
        const bool valid = !PART || (FWD ? ib + j < len : ib - j >= 0);
        const char* a0 = cb + line_off<GPW>(d[j].y & 0xFFFFu);
        const char* a1 = cb + line_off<GPW>(d[j].y >> 16);
#pragma unroll
        for (int g = 0; g < GPW; ++g) {
            in.cur[j][g] = valid ? *reinterpret_cast<const uint32_t*>(rp + LINE * st + 128 * g) : INF_U;
            s0[j][g] = valid ? *reinterpret_cast<const uint32_t*>(a0 + 128 * g) : 0u;
            s1[j][g] = valid ? *reinterpret_cast<const uint32_t*>(a1 + 128 * g) : 0u;
        }
        in.cw[j] = d[j].x;
    }
#pragma unroll
    for (int j = 0; j < BLK; ++j)
#pragma unroll
        for (int g = 0; g < GPW; ++g)
            in.m[j][g] = __viaddmin_u32(s1[j][g], d[j].w, __viaddmin_u32(s0[j][g], d[j].z, in.cur[j][g]));
}

// Carry chains of one block (one per group); stores the new values, folds the
// changed bits into chg (per group).
template <int GPW, bool FWD, bool PART>
__device__ __forceinline__ void chain_blk(char* cb, int len, int b, const BlkIn<GPW>& in, uint32_t (&xprev)[GPW],
                                          uint32_t (&chg)[GPW]) {
    constexpr int LINE = 128 * GPW;
    const int ib = FWD ? b * BLK : len - 1 - b * BLK;
    char* rp = cb + LINE * ib;
#pragma unroll
    for (int j = 0; j < BLK; ++j) {
        const int st = FWD ? j : -j;
#pragma unroll
        for (int g = 0; g < GPW; ++g) {
            const uint32_t x = __viaddmin_u32(xprev[g], in.cw[j], in.m[j][g]);
            if (!PART || (FWD ? ib + j < len : ib - j >= 0)) {
                *reinterpret_cast<uint32_t*>(rp + LINE * st + 128 * g) = x;
                chg[g] |= x ^ in.cur[j][g];
            }
            xprev[g] = x;
        }
    }
}

// One pass over the run: whole blocks of BLK nodes in pass order, the loads
// of block b + 1 issued before the chain of block b, then the partial block.
template <int TILE, int GPW, bool FWD>
__device__ __forceinline__ void warp_pass(WarpTile<TILE, GPW>& t, int len, int alen, int lane, uint32_t (&chg)[GPW]) {
    char* cb = reinterpret_cast<char*>(&t.rows[0][lane]);
    const int nf = len / BLK;
    uint32_t xprev[GPW];
#pragma unroll
    for (int g = 0; g < GPW; ++g) xprev[g] = INF_U;
    BlkIn<GPW> a, c;
    // forward: the second segment's lines are waited for before the first block that reaches them
    bool second = !FWD || alen >= len;
    auto need = [&](int b) {
        if (!second && (b + 1) * BLK > alen) {
            cp_async_wait_pending(0);
            __syncwarp();
            second = true;
        }
    };
    if (nf > 0) {
        need(0);
        load_blk<TILE, GPW, FWD, false>(t, cb, len, 0, a);
    }
#pragma unroll 1
    for (int b = 0; b < nf; b += 2) {
        if (b + 1 < nf) {
            need(b + 1);
            load_blk<TILE, GPW, FWD, false>(t, cb, len, b + 1, c);
        }
        chain_blk<GPW, FWD, false>(cb, len, b, a, xprev, chg);
        if (b + 2 < nf) {
            need(b + 2);
            load_blk<TILE, GPW, FWD, false>(t, cb, len, b + 2, a);
        }
        if (b + 1 < nf) chain_blk<GPW, FWD, false>(cb, len, b + 1, c, xprev, chg);
    }
    if (nf * BLK < len) {
        need(nf);
        load_blk<TILE, GPW, FWD, true>(t, cb, len, nf, a);
        chain_blk<GPW, FWD, true>(cb, len, nf, a, xprev, chg);
    }
}

// Runs without compact descriptors (a node with more than two non-carry arcs
// in a pass, or a halo larger than the tile): descriptors and arcs from global
// memory, sources from the tile or, past its capacity, from the rows in L2.
template <int TILE, int GPW>
__device__ __noinline__ uint32_t warp_passes_generic(const BfParams& p, WarpTile<TILE, GPW>& t, int4 rs, int len,
                                                     int lane, const TileMeta& m, int G) {
    const uint32_t* rows = p.seg.rows;
    const int64_t ld = p.seg.ld;
    uint32_t chg = 0;
#pragma unroll 1
    for (int g = 0; g < m.ng; ++g) {
        uint32_t* col = &t.rows[0][32 * g + lane];
        const int64_t lane_off = seg_col0(p.seg, m.g + g);
        uint32_t carry = INF_U;
        for (int i = 0; i < len; ++i) {
            const int4 d = __ldg(p.g.node_desc + run_node(rs, i));
            const uint32_t cur = col[32 * GPW * i];
            uint32_t best = __viaddmin_u32(carry, static_cast<uint32_t>(d.x), cur);
            for (int q = d.z; q < d.w; ++q) {
                const uint2 e = __ldg(p.g.arc2 + q);
                const uint32_t x = (e.x & GLOBAL_REF)
                                       ? ld_l2(rows + static_cast<int64_t>(e.x & ~GLOBAL_REF) * ld + lane_off + lane)
                                       : col[32 * GPW * e.x];
                best = __viaddmin_u32(x, e.y, best);
            }
            col[32 * GPW * i] = best;
            chg |= best ^ cur;
            carry = best;
        }
        carry = INF_U;
        for (int i = len - 1; i >= 0; --i) {
            const int4 d = __ldg(p.g.node_desc + run_node(rs, i));
            const int end = __ldg(&p.g.node_desc[run_node(rs, i) + 1].z);
            const uint32_t cur = col[32 * GPW * i];
            uint32_t best = __viaddmin_u32(carry, static_cast<uint32_t>(d.y), cur);
            for (int q = d.w; q < end; ++q) {
                const uint2 e = __ldg(p.g.arc2 + q);
                best = __viaddmin_u32(col[32 * GPW * e.x], e.y, best);
            }
            col[32 * GPW * i] = best;
            chg |= best ^ cur;
            carry = best;
        }
    }
    return chg;
}

// One tile by one warp: stage, forward pass, backward pass, write back the
// own lines.  Returns true (warp-uniform) if a row dropped.  A group slot
// past G (ng < GPW) is neither staged nor written back; its columns hold
// stale values that only feed its own discarded chains.
__device__ __forceinline__ void prefetch_l2(const void* a) { asm volatile("prefetch.global.L2 [%0];" ::"l"(a)); }

template <int TILE, int GPW>
__device__ __forceinline__ bool warp_tile(const BfParams& p, const TileMeta& m, WarpTile<TILE, GPW>& t, int lane,
                                          const TileMeta* next = nullptr) {
    const int64_t ld = p.seg.ld;
    uint32_t* rows = p.seg.rows;
    const bool compact = (m.flags & RUN_COMPACT) != 0;
    // 8 lanes x 16 bytes per 128-byte line; 4 / GPW slots per instruction
    constexpr int LPS = 8 * GPW;  // lanes per slot
    const int sub = lane / LPS, gq = (lane % LPS) / 8, part = (lane & 7) * 4;
    constexpr int SPI = 32 / LPS;  // slots per instruction
    const bool act = gq < m.ng;
    const int64_t col0 = act ? seg_col0(p.seg, m.g + gq) : 0;
    const int cpart = 32 * gq + part;
    // group A: descriptors, extras, halo lines, the first segment's lines
    const int nx = m.rx.y + m.rx.z;
    if (compact) {
        for (int e = lane; e < 2 * m.len; e += 32)
            cp_async16(&t.desc[e], p.g.cdesc + 2 * static_cast<int64_t>(run_node(m.rs, e >> 1)) + (e & 1));
        for (int e = lane; 2 * e < nx; e += 32) cp_async16(&t.wx[2 * e], p.g.wx + m.rx.x + 2 * e);
    }
    if (m.hids) {
        for (int hb = 0; hb < m.hn; hb += SPI) {  // the same trip count in every lane
            const int h = hb + sub;
            const int node = __shfl_sync(FULL_MASK, m.hid, h & 31);
            if (act && h < m.hn)
                cp_async16(&t.rows[m.len + h][cpart], rows + static_cast<int64_t>(node) * ld + col0 + part);
        }
    } else if (act) {
        for (int h = sub; h < m.hn; h += SPI) {
            const int node = __ldg(p.g.halo_nodes + m.h0 + h);
            cp_async16(&t.rows[m.len + h][cpart], rows + static_cast<int64_t>(node) * ld + col0 + part);
        }
    }
    if (act) {
        const uint32_t* gp = rows + static_cast<int64_t>(m.rs.x + sub) * ld + col0 + part;
        for (int i = sub; i < m.rs.y; i += SPI, gp += SPI * ld) cp_async16(&t.rows[i][cpart], gp);
    }
    cp_async_commit();
    // group B: the second segment's lines
    if (act) {
        const uint32_t* gp = rows + static_cast<int64_t>(m.rs.z + sub) * ld + col0 + part;
        for (int i = sub; i < m.rs.w; i += SPI, gp += SPI * ld) cp_async16(&t.rows[m.rs.y + i][cpart], gp);
    }
    cp_async_commit();
    // the next tile's own lines and descriptors towards L2 while this one is relaxed
    if (next != nullptr && next->len > 0) {
        for (int g = 0; g < next->ng; ++g) {
            const int64_t c1 = seg_col0(p.seg, next->g + g);
            for (int i = lane; i < next->len; i += 32)
                prefetch_l2(rows + static_cast<int64_t>(run_node(next->rs, i)) * ld + c1);
        }
        if (next->flags & RUN_COMPACT)
            for (int i = 4 * lane; i < next->len; i += 128)
                prefetch_l2(p.g.cdesc + 2 * static_cast<int64_t>(run_node(next->rs, i)));
    }

    uint32_t chg = 0;
    if (compact) {
        uint32_t cg[GPW];
#pragma unroll
        for (int g = 0; g < GPW; ++g) cg[g] = 0;
        int alen = m.rs.y;
        if (m.rx.y > 0) {
            // forward extras may touch either segment: everything lands first
            cp_async_wait_pending(0);
            __syncwarp();
            fold_extras<TILE, GPW>(t, 0, m.rx.y, lane, cg);
            alen = m.len;
        } else {
            cp_async_wait_pending(1);  // group A landed: the forward pass starts on the first segment
            __syncwarp();
        }
        warp_pass<TILE, GPW, true>(t, m.len, alen, lane, cg);
        if (m.rx.z > 0) fold_extras<TILE, GPW>(t, m.rx.y, m.rx.z, lane, cg);
        warp_pass<TILE, GPW, false>(t, m.len, m.rs.y, lane, cg);
        // an absent group's columns hold stale values: only the present groups count
#pragma unroll
        for (int g = 0; g < GPW; ++g)
            if (g < m.ng) chg |= cg[g];
    } else {
        cp_async_wait_pending(0);
        __syncwarp();
        chg = warp_passes_generic<TILE, GPW>(p, t, m.rs, m.len, lane, m, 0);
    }
    const bool changed = __any_sync(FULL_MASK, chg != 0u);
    if (changed) {
        // every own line goes back (a visited line is read and written once per sweep)
        __syncwarp();
        if (act)
            for (int i = sub; i < m.len; i += SPI)
                __stcg(reinterpret_cast<uint4*>(rows + static_cast<int64_t>(run_node(m.rs, i)) * ld + col0 + part),
                       *reinterpret_cast<const uint4*>(&t.rows[i][cpart]));
    }
    __syncwarp();  // every lane's reads of the tile done before the next staging overwrites it
    return changed;
}

// Push-based frontier of the warp sweeps: sweep s visits list s mod 3.  A
// tile that changed in sweep s adds itself and the tiles of the runs it feeds
// (same group) to list s+1; stamp[item] = the last sweep it was listed for,
// raised with atomicMax, so an item is listed once per sweep.  List s+2 (read
// in sweep s-1) is cleared during sweep s, before anyone appends to it in
// sweep s+1.  One grid barrier per sweep.
__device__ __forceinline__ int32_t* frontier_list(const BfParams& p, int s) {
    const int i = s % 3;
    return i == 0 ? p.w.list0 : i == 1 ? p.w.list1 : p.w.list2;
}

// Items of runs that feed many others (RUN_PRIORITY: the cross-aisle pieces) are
// listed first: they fill each list from its end (count counts[6 + s % 3]), the
// others from its start (counts[s % 3]), and claim c takes the c-th priority item
// while there are any.  So a sweep relaxes the cross-aisle tiles in its first
// wave, and the aisle tiles claimed after them already read their new values.
// cap = items of the segment (no list holds an item twice, so the two ends never meet).
__device__ __forceinline__ int32_t list_item(const int32_t* list, int c, int n_prio, int cap) {
    return __ldcg(list + (c < n_prio ? cap - 1 - c : c - n_prio));
}

__device__ __forceinline__ bool item_priority(const BfParams& p, int32_t item, int ipr) {
    return p.w.prio && (__ldg(p.g.run_flags + item / ipr) & RUN_PRIORITY) != 0;
}

// One thread lists one item for sweep s (seeding).
__device__ __forceinline__ void frontier_push(const BfParams& p, int32_t item, int s, int ipr, int cap) {
    if (atomicMax(p.w.stamp + item, s) < s) {
        int32_t* list = frontier_list(p, s);
        if (item_priority(p, item, ipr)) list[cap - 1 - atomicAdd(p.w.counts + 6 + s % 3, 1)] = item;
        else list[atomicAdd(p.w.counts + s % 3, 1)] = item;
    }
}

// The warp lists up to n items cand(j) for sweep s: one item per lane and
// round, one reservation per list end and round.
template <class Cand, class Prio>
__device__ __forceinline__ void frontier_push_warp(const BfParams& p, int n, int s, int lane, int ipr, int cap, Cand cand,
                                                   Prio prio) {
    int32_t* list = frontier_list(p, s);
    for (int base = 0; base < n; base += 32) {
        const int j = base + lane;
        int32_t item = -1;
        bool add = false, pr = false;
        if (j < n) {
            item = cand(j);
            add = atomicMax(p.w.stamp + item, s) < s;
            pr = add && prio(j, item);
        }
        const unsigned mn = __ballot_sync(FULL_MASK, add && !pr), mp = __ballot_sync(FULL_MASK, pr);
        if ((mn | mp) == 0u) continue;
        int pn = 0, pp = 0;
        if (lane == 0) {
            if (mn) pn = atomicAdd(p.w.counts + s % 3, __popc(mn));
            if (mp) pp = atomicAdd(p.w.counts + 6 + s % 3, __popc(mp));
        }
        pn = __shfl_sync(FULL_MASK, pn, 0);
        pp = __shfl_sync(FULL_MASK, pp, 0);
        if (pr) list[cap - 1 - (pp + __popc(mp & lanemask_lt()))] = item;
        else if (add) list[pn + __popc(mn & lanemask_lt())] = item;
    }
}

template <int TILE, int NW, int GPW>
__global__ void __launch_bounds__(32 * NW, 1) bf_warp_kernel(BfParams p) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpTile<TILE, GPW>& t = reinterpret_cast<WarpTile<TILE, GPW>*>(smem_raw)[warp];

    const int n_lanes = segment_lanes(p.seg);
    const int G = (n_lanes + 31) >> 5;
    if (G == 0) return;  // same decision in every block
    const int ipr = (G + GPW - 1) / GPW;  // items per run: GPW groups each
    const int cap = p.g.n_runs * ipr;     // items of the segment: the lists' length
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthreads = gridDim.x * blockDim.x;

    // seeds: writing d[s][s] = 0 was the change of "sweep 0": sweep 1 visits
    // the tile holding each source and the tiles it feeds
    for (int b = gtid; b < n_lanes; b += nthreads) {
        const int r = __ldg(p.g.run_of_node + p.seg.src[p.seg.first + b]);
        const int g = (b >> 5) / GPW;
        frontier_push(p, r * ipr + g, 1, ipr, cap);
        const int q1 = __ldg(p.g.rout_ptr + r + 1);
        for (int q = __ldg(p.g.rout_ptr + r); q < q1; ++q) frontier_push(p, __ldg(p.g.rout_list + q) * ipr + g, 1, ipr, cap);
    }
    if (!grid_sync(p.w.bar, p.w.err, p.w.max_spins)) return;

    unsigned long long tiles = 0, nodes = 0, bytes = 0, reread = 0;
    int sweep = 1;
    for (;; ++sweep) {
        const int cur = sweep % 3;
        const int n_prio = ld_volatile(p.w.counts + 6 + cur);
        const int cnt = ld_volatile(p.w.counts + cur) + n_prio;
        if (gtid == 0 && sweep <= p.w.trace_cap) {
            long long tm;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(tm));
            p.w.trace[2 * (sweep - 1)] = cnt;
            p.w.trace[2 * (sweep - 1) + 1] = tm;
        }
        if (cnt == 0) break;
        if (sweep > p.g.V + 1) {
            if (gtid == 0) atomicCAS(p.w.err, 0, WR_EINTERNAL);
            break;
        }
        if (gtid == 0) {
            const int nx = (sweep + 2) % 3;  // the list sweep s+2 fills; sweep s-1 read it
            p.w.counts[nx] = 0;
            p.w.counts[3 + nx] = 0;
            p.w.counts[6 + nx] = 0;
        }
        const int32_t* list = frontier_list(p, sweep);
        int* claim = p.w.counts + 3 + cur;
        // dynamic tile scheduling, per warp: the item two ahead is claimed and
        // the next item's run metadata loaded while the current tile is relaxed.
        // A sweep with no more items than warps claims one item per warp instead,
        // so that no warp relaxes two tiles one after the other while others idle
        const bool ahead = cnt > static_cast<int>(gridDim.x) * NW;
        int it = 0, it1 = 0;
        if (lane == 0) {
            it = atomicAdd(claim, 1);
            it1 = ahead ? atomicAdd(claim, 1) : cnt;
        }
        it = __shfl_sync(FULL_MASK, it, 0);
        it1 = __shfl_sync(FULL_MASK, it1, 0);
        TileMeta m{};
        if (it < cnt) m = load_meta<GPW>(p, list_item(list, it, n_prio, cap), G, lane);
        while (it < cnt) {
            int it2 = 0;
            if (lane == 0) it2 = ahead ? atomicAdd(claim, 1) : cnt;
            TileMeta m1{};
            if (it1 < cnt) m1 = load_meta<GPW>(p, list_item(list, it1, n_prio, cap), G, lane);
            // algorithmic bytes take a run's descriptors once per sweep, whichever of its
            // groups comes first; the answer is used after the tile, so the atomic's latency
            // hides behind it
            int first_visit = 0;
            if (lane == 0) first_visit = atomicMax(p.w.run_stamp + m.r, sweep) < sweep;
            const bool ch = warp_tile<TILE, GPW>(p, m, t, lane, it1 < cnt ? &m1 : nullptr);
            if (ch) {
                // the tile itself and the runs it feeds, for the next sweep; up to 31 fed runs
                // come from the registers loaded with the metadata
                const int q0 = m.q0, nq = m.nq;
                const int item = m.item, g = m.g / GPW;
                const int fed = __shfl_sync(FULL_MASK, m.rq, (lane + 31) & 31) * ipr + g;  // lane j: fed run j - 1
                const bool fedp = __shfl_sync(FULL_MASK, m.rqp, (lane + 31) & 31);
                const bool selfp = p.w.prio && (m.flags & RUN_PRIORITY) != 0;
                if (nq < 32)
                    frontier_push_warp(p, nq + 1, sweep + 1, lane, ipr, cap, [&](int j) { return j == 0 ? item : fed; },
                                       [&](int j, int32_t) { return j == 0 ? selfp : fedp; });
                else
                    frontier_push_warp(p, nq + 1, sweep + 1, lane, ipr, cap,
                                       [&](int j) { return j == 0 ? item : __ldg(p.g.rout_list + q0 + j - 1) * ipr + g; },
                                       [&](int, int32_t it) { return item_priority(p, it, ipr); });
            }
            if (lane == 0) {
                ++tiles;
                nodes += static_cast<unsigned long long>(m.len) * m.ng;
                const unsigned long long meta = static_cast<unsigned long long>(__ldg(p.g.run_meta_bytes + m.r));
                bytes += 256ull * static_cast<unsigned long long>(m.len) * m.ng + (first_visit ? meta : 0ull);
                reread += first_visit ? 0ull : meta;
            }
            it = it1;
            m = m1;
            it1 = __shfl_sync(FULL_MASK, it2, 0);
        }
        if (!grid_sync(p.w.bar, p.w.err, p.w.max_spins)) break;
    }
    if (lane == 0 && tiles) {
        atomicAdd(p.w.stats + 1, tiles);
        atomicAdd(p.w.stats + 2, nodes);
        atomicAdd(p.w.stats + 3, bytes);
        atomicAdd(p.w.stats + 5, reread);
    }
    if (gtid == 0) atomicAdd(p.w.stats + 0, static_cast<unsigned long long>(sweep - 1));
}

// ---------------------------------------------------------------------------
// Asynchronous worklist (bf_tiling 3): the same warp tiles with no sweeps and
// no grid barriers after seeding.  Each (run, group) item is idle, queued,
// running, or running and dirty (an input changed while it ran).  A warp pops
// an item, relaxes its tile, and when a row dropped pushes the item itself
// and the items of the runs it feeds (same group); an idle item is queued
// once (its state is the dedup), a running one is marked dirty and requeued
// by its runner when it finishes.  So no two warps ever hold the same tile,
// and each own line has a single writer.  The pending count (queued plus
// running items) rises before every push and falls only after the finished
// item's pushes: it reaches zero exactly when nothing can change any more,
// the fixpoint, which is when every warp stops.
//
// The queue is a ring of 2 x items slots with a sequence number per slot:
// the producer of position t waits for seq == t, writes the item and
// releases seq = t + 1; the consumer of position h waits for seq == h + 1,
// takes the item and releases seq = h + cap for the producer one lap later.
// Consumers may claim positions far ahead of the producers (idle warps); a
// slot still serves its positions in order.  At most `items` entries wait at
// any time, so the consumer of position t - cap has always claimed it when
// the producer of t arrives, and every wait ends.  Every wait is also
// bounded by max_spins (WR_ETIMEOUT), the kernel by a wall-clock limit, and
// the total work by (V + 2) x items visits (WR_EINTERNAL).
// ---------------------------------------------------------------------------
enum : int32_t { Q_IDLE = 0, Q_QUEUED = 1, Q_RUNNING = 2, Q_DIRTY = 3 };

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p) {
    return *reinterpret_cast<const volatile unsigned long long*>(p);
}

__device__ __forceinline__ bool q_fail(const BfParams& p, int code) {
    atomicCAS(p.w.err, 0, code);
    return false;
}

// Put an item (already counted as pending) into the next ring position.
__device__ bool q_enqueue(const BfParams& p, int32_t item, unsigned long long cap) {
    const unsigned long long t = atomicAdd(p.w.qctl + 1, 1ull);
    const unsigned long long k = t % cap;
    unsigned long long spins = 0;
    while (ld_acquire_u64(p.w.ring_seq + k) != t) {  // the slot's previous lap is being taken
        if (ld_volatile(p.w.err) != 0) return false;
        if (++spins > p.w.max_spins) return q_fail(p, WR_ETIMEOUT);
        __nanosleep(32);
    }
    *reinterpret_cast<volatile int32_t*>(p.w.ring + k) = item;
    st_release_u64(p.w.ring_seq + k, t + 1);
    return true;
}

// Request a (re)visit of an item: queue it if idle, mark it dirty if running.
__device__ bool q_push(const BfParams& p, int32_t item, unsigned long long cap) {
    int32_t* st = p.w.stamp + item;
    for (int tries = 0; tries < 64; ++tries) {
        const int32_t s = atomicCAS(st, Q_IDLE, Q_QUEUED);
        if (s == Q_IDLE) {
            atomicAdd(p.w.qctl + 2, 1ull);
            return q_enqueue(p, item, cap);
        }
        if (s != Q_RUNNING) return true;  // queued or dirty: a visit is already due
        if (atomicCAS(st, Q_RUNNING, Q_DIRTY) == Q_RUNNING) return true;
        // it finished between the two steps: try again from idle
    }
    return q_fail(p, WR_EINTERNAL);
}

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Next item for this warp (lane 0), or -1 when the worklist is exhausted or
// failed.  Past t_stop (a wall-clock bound far above any legitimate run) the
// kernel gives up with WR_ETIMEOUT rather than run on.
__device__ int32_t q_pop(const BfParams& p, unsigned long long cap, unsigned long long limit, long long t_stop) {
    const unsigned long long h = atomicAdd(p.w.qctl + 0, 1ull);
    if (h >= limit) {
        q_fail(p, WR_EINTERNAL);
        return -1;
    }
    if (global_ns() > t_stop) {
        q_fail(p, WR_ETIMEOUT);
        return -1;
    }
    const unsigned long long k = h % cap;
    unsigned long long spins = 0;
    for (;;) {
        if (ld_acquire_u64(p.w.ring_seq + k) == h + 1) {
            const int32_t v = *reinterpret_cast<volatile int32_t*>(p.w.ring + k);
            st_release_u64(p.w.ring_seq + k, h + cap);
            atomicExch(p.w.stamp + v, Q_RUNNING);  // no one else writes a queued item's state
            __threadfence();  // the producer's row stores are visible before the tile is staged
            return v;
        }
        if (ld_volatile_u64(p.w.qctl + 2) == 0ull || ld_volatile(p.w.err) != 0) return -1;
        if (++spins > p.w.max_spins) {
            q_fail(p, WR_ETIMEOUT);
            return -1;
        }
        __nanosleep(32);
    }
}

// The whole warp requests visits of up to n items (cand(j), j < n), one per
// lane and round: state changes in parallel, then one pending and one ring
// reservation for all newly queued items of the round.
template <class Cand>
__device__ bool q_push_warp(const BfParams& p, int n, unsigned long long cap, int lane, Cand cand) {
    for (int base = 0; base < n; base += 32) {
        const int j = base + lane;
        int32_t item = -1;
        bool enq = false, ok = true;
        if (j < n) {
            item = cand(j);
            int32_t* st = p.w.stamp + item;
            int tries = 0;
            for (; tries < 64; ++tries) {
                const int32_t s = atomicCAS(st, Q_IDLE, Q_QUEUED);
                if (s == Q_IDLE) {
                    enq = true;
                    break;
                }
                if (s != Q_RUNNING) break;  // queued or dirty: a visit is already due
                if (atomicCAS(st, Q_RUNNING, Q_DIRTY) == Q_RUNNING) break;
            }
            if (tries == 64) ok = q_fail(p, WR_EINTERNAL);
        }
        const unsigned m = __ballot_sync(FULL_MASK, enq);
        if (!__all_sync(FULL_MASK, ok)) return false;
        if (m == 0u) continue;
        unsigned long long t0 = 0;
        if (lane == 0) {
            atomicAdd(p.w.qctl + 2, static_cast<unsigned long long>(__popc(m)));
            t0 = atomicAdd(p.w.qctl + 1, static_cast<unsigned long long>(__popc(m)));
        }
        t0 = __shfl_sync(FULL_MASK, t0, 0);
        if (enq) {
            const unsigned long long t = t0 + static_cast<unsigned long long>(__popc(m & lanemask_lt()));
            const unsigned long long k = t % cap;
            unsigned long long spins = 0;
            while (ld_acquire_u64(p.w.ring_seq + k) != t) {
                if (ld_volatile(p.w.err) != 0) {
                    ok = false;
                    break;
                }
                if (++spins > p.w.max_spins) {
                    ok = q_fail(p, WR_ETIMEOUT);
                    break;
                }
                __nanosleep(32);
            }
            if (ok) {
                *reinterpret_cast<volatile int32_t*>(p.w.ring + k) = item;
                st_release_u64(p.w.ring_seq + k, t + 1);
            }
        }
        if (!__all_sync(FULL_MASK, ok)) return false;
    }
    return true;
}

// After the visit: requeue a dirty item, else retire it from the pending count.
__device__ bool q_finish(const BfParams& p, int32_t item, unsigned long long cap) {
    const int32_t s = atomicCAS(p.w.stamp + item, Q_RUNNING, Q_IDLE);
    if (s == Q_DIRTY) {
        atomicExch(p.w.stamp + item, Q_QUEUED);
        return q_enqueue(p, item, cap);
    }
    atomicAdd(p.w.qctl + 2, ~0ull);  // -1
    return true;
}

template <int TILE, int NW>
__global__ void __launch_bounds__(32 * NW, 1) bf_warp_async_kernel(BfParams p) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpTile<TILE, 1>& t = reinterpret_cast<WarpTile<TILE, 1>*>(smem_raw)[warp];

    const int n_lanes = segment_lanes(p.seg);
    const int G = (n_lanes + 31) >> 5;
    if (G == 0) return;  // same decision in every block
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthreads = gridDim.x * blockDim.x;
    const unsigned long long n_items = static_cast<unsigned long long>(p.g.n_runs) * static_cast<unsigned long long>(G);
    const unsigned long long cap = 2ull * n_items;
    // pops: at most (V + 2) visits per item, plus one last empty pop per warp
    const unsigned long long limit = (static_cast<unsigned long long>(p.g.V) + 2ull) * n_items +
                                     static_cast<unsigned long long>(gridDim.x) * (blockDim.x >> 5);

    // seeds: d[s][s] = 0 was written by the init; the tile holding each source
    // and every tile it feeds get a first visit
    for (int b = gtid; b < n_lanes; b += nthreads) {
        const int r = __ldg(p.g.run_of_node + p.seg.src[p.seg.first + b]);
        const int g = b >> 5;
        if (!q_push(p, r * G + g, cap)) break;
        const int q1 = __ldg(p.g.rout_ptr + r + 1);
        for (int q = __ldg(p.g.rout_ptr + r); q < q1; ++q)
            if (!q_push(p, __ldg(p.g.rout_list + q) * G + g, cap)) break;
    }
    if (!grid_sync(p.w.bar, p.w.err, p.w.max_spins)) return;

    // wall-clock bound: 1024 ns per allowed spin (about 17 s by default)
    const long long t_stop = global_ns() + static_cast<long long>(min(p.w.max_spins, 1ull << 40) * 1024ull);
    unsigned long long tiles = 0, nodes = 0, bytes = 0;
    for (;;) {
        int32_t item = -1;
        if (lane == 0 && ld_volatile(p.w.err) == 0) item = q_pop(p, cap, limit, t_stop);
        item = __shfl_sync(FULL_MASK, item, 0);
        if (item < 0) break;
        __syncwarp();
        TileMeta m;
        m.item = item;
        m.r = item / G;
        m.g = item - m.r * G;
        m.ng = 1;
        m.rs = __ldg(p.g.run_seg + m.r);
        m.len = m.rs.y + m.rs.w;
        m.h0 = __ldg(p.g.halo_ptr + m.r);
        m.hn = __ldg(p.g.halo_ptr + m.r + 1) - m.h0;
        m.flags = __ldg(p.g.run_flags + m.r);
        m.rx = __ldg(p.g.run_wx + m.r);
        m.hids = false;  // the halo's node ids are read while staging
        m.hid = 0;
        const bool ch = warp_tile<TILE, 1>(p, m, t, lane);
        bool ok = true;
        if (ch) {
            __threadfence();  // this lane's row stores before the pushes that announce them
            __syncwarp();
            // the item itself (running: marked dirty, so it is visited again) and the runs it feeds
            const int q0 = __ldg(p.g.rout_ptr + m.r), nq = __ldg(p.g.rout_ptr + m.r + 1) - q0;
            ok = q_push_warp(p, nq + 1, cap, lane,
                             [&](int j) { return j == 0 ? item : __ldg(p.g.rout_list + q0 + j - 1) * G + m.g; });
        }
        if (lane == 0) {
            if (ok) q_finish(p, item, cap);
            ++tiles;
            nodes += static_cast<unsigned long long>(m.len);
            bytes += static_cast<unsigned long long>(__ldg(p.g.run_meta_bytes + m.r)) +
                     256ull * static_cast<unsigned long long>(m.len);
        }
    }
    if (lane == 0 && tiles) {
        atomicAdd(p.w.stats + 1, tiles);
        atomicAdd(p.w.stats + 2, nodes);
        atomicAdd(p.w.stats + 3, bytes);
    }
}

template <int TILE, int NW, bool ASYNC, int GPW = 1>
static int prepare_warp_one(int device, BfLaunchInfo* info) {
    const size_t smem = sizeof(WarpTile<TILE, GPW>) * NW;
    auto* fn = ASYNC ? bf_warp_async_kernel<TILE, NW> : bf_warp_kernel<TILE, NW, GPW>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
        return WR_ECUDA;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 32 * NW, smem) != cudaSuccess || occ < 1)
        return WR_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return WR_ECUDA;
    info->blocks = occ * sms;
    info->threads = 32 * NW;
    info->smem = smem;
    info->fn = reinterpret_cast<const void*>(fn);
    return WR_OK;
}

// Warps per CTA: as many warp tiles as fit 227 KB of shared memory: 128-slot
// tiles of one source group (11 warps of 20.5 KB) or two (6 warps), 256-slot tiles of one (5).
int bf_prepare_warp(int tile_cap, int mode, int device, BfLaunchInfo* info) {
    switch (tile_cap) {
        case 128:
            if (mode == WARP_ASYNC) return prepare_warp_one<128, 11, true>(device, info);
            if (mode == WARP_PAIRS) return prepare_warp_one<128, 6, false, 2>(device, info);
            return prepare_warp_one<128, 11, false>(device, info);
        case 256:
            if (mode == WARP_ASYNC) return prepare_warp_one<256, 5, true>(device, info);
            if (mode == WARP_PAIRS) return WR_EINVAL;
            return prepare_warp_one<256, 5, false>(device, info);
        default: return WR_EINVAL;
    }
}

}  // namespace wr
