// Row a3: multi-source Bellman-Ford sweeps (Sec. 4.7), with the source
// batching of Sec. 4.7 (N sources processed together, dist is V x N).
//
// Layout: one source segment keeps rows[v * ld + b] = current bound on
// dist(src_b, v): the B sources of a node are contiguous, so one 128-byte
// line of a node row serves a group of 32 sources.  Work items are
// (run, group) tiles.  A warp stages the tile's own rows and its halo rows
// in shared memory (cp.async through L2), relaxes every in-arc once per
// sweep -- arcs from lower ids in a forward pass, from higher ids in a
// backward pass, each pass in place -- and writes back the rows that
// dropped.  The relaxation is the min-plus step d[v] = min(d[v], d[u] + w)
// of the paper; every value stays an upper bound on the true distance, so
// the in-place order and the concurrency of tiles cannot change the
// fixpoint, only how many sweeps reach it.
//
// Frontier: a tile is processed in sweep t+1 only if it or a run feeding
// it changed in sweep t (stamps, compacted into a list with warp-aggregated
// appends).  The sweep loop lives in one cooperative persistent kernel with
// bounded grid barriers and stops at the first sweep that changes nothing
// (early exit on a converged frontier), capped at V+1 sweeps.
#include "wr_bf_common.cuh"

namespace wr {

// rows := INF; stamps := 0; counters := 0.  A warp fills whole rows with
// 16-byte stores (32 lanes x 4 sources per instruction).  The sources' zeros
// go in with the fill when the segment maps nodes to its sources (src_index),
// else bf_seed_kernel writes them after it.
__global__ void bf_init_kernel(BfParams p) {
    const int n_lanes = segment_lanes(p.seg);
    const int G = (n_lanes + 31) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    const int64_t w0 = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint4 inf = make_uint4(INF_U, INF_U, INF_U, INF_U);
    for (int64_t v = w0; v < p.g.V; v += warps) {
        uint32_t* row = p.seg.rows + v * p.seg.ld;
        // the lane of this segment whose source is v, if any: its entry gets the seed 0
        int sl = -1;
        if (p.seg.src_index) {
            const int b = __ldg(p.seg.src_index + v) - p.seg.first;
            if (b >= 0 && b < n_lanes) sl = b;
        }
        for (int q = lane; q < 8 * G; q += 32) {  // uint4 q: group q / 8, lanes 4 (q % 8) ..
            uint4 x = inf;
            if (q == (sl >> 2)) {
                const int comp = sl & 3;
                x.x = comp == 0 ? 0u : INF_U;
                x.y = comp == 1 ? 0u : INF_U;
                x.z = comp == 2 ? 0u : INF_U;
                x.w = comp == 3 ? 0u : INF_U;
            }
            __stcg(reinterpret_cast<uint4*>(row + seg_col0(p.seg, q >> 3) + 4 * (q & 7)), x);
        }
    }
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t n_items = static_cast<int64_t>(p.g.n_runs) * G;
    for (int64_t i = t0; i < n_items; i += stride) p.w.stamp[i] = 0;
    for (int64_t i = t0; i < p.g.n_runs; i += stride) p.w.run_stamp[i] = 0;
    if (t0 < 16) p.w.counts[t0] = 0;
    if (p.w.async) {
        for (int64_t i = t0; i < 2 * n_items; i += stride) p.w.ring_seq[i] = static_cast<unsigned long long>(i);
        if (t0 < 4) p.w.qctl[t0] = 0ull;
    }
    if (t0 == 0) {
        p.w.bar->count = 0;
        p.w.bar->gen = 0;
    }
}

// dist(src_b, src_b) = 0, after the fill.
__global__ void bf_seed_kernel(BfParams p) {
    const int n_lanes = segment_lanes(p.seg);
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n_lanes)
        p.seg.rows[static_cast<int64_t>(p.seg.src[p.seg.first + b]) * p.seg.ld + seg_col0(p.seg, b >> 5) + (b & 31)] = 0u;
}

// Shared memory of one warp: the tile's rows (own nodes then halo), the
// run's inline node descriptors and extra arcs, and a dirty bit per own node.
// Each quad plane is padded by one 16-byte slot, so the 8 planes' copies of
// one position fall in 8 different bank groups (the write-back reads all 8
// quads of a node in one phase).
template <int TILE>
struct TileSmem {
    static constexpr int PLANE = TILE + 1;
    uint4 rows[8][PLANE];  // quad-major: rows[q][pos(i)] = sources 4q..4q+3 of tile slot i
    uint4 ix[2 * (TILE + 1)];
    uint2 xarcs[TILE];
    uint8_t dirtyb[TILE];
};

// Scan chunks cover SPAN = 32 * SEG consecutive node ids, aligned to
// multiples of SPAN, in both passes; a lane owns SEG consecutive nodes of a
// chunk.  Within each SPAN-slot block, slot o = SEG * l + j sits at position
// 32 j + l, so the 32 lanes reading "their" j-th node touch 32 consecutive
// 16-byte positions: no bank conflicts and a constant offset per quad.
constexpr int SEG = 2;
constexpr int SPAN = 32 * SEG;
__device__ __forceinline__ int pos_of(int i) { return (i & ~(SPAN - 1)) | ((i % SEG) << 5) | ((i / SEG) & 31); }

__device__ __forceinline__ uint4 addmin4(uint4 x, uint32_t w, uint4 m) {
    return make_uint4(__viaddmin_u32(x.x, w, m.x), __viaddmin_u32(x.y, w, m.y), __viaddmin_u32(x.z, w, m.z),
                      __viaddmin_u32(x.w, w, m.w));
}
__device__ __forceinline__ uint4 shfl_up4(uint4 v, int d) {
    return make_uint4(__shfl_up_sync(FULL_MASK, v.x, d), __shfl_up_sync(FULL_MASK, v.y, d),
                      __shfl_up_sync(FULL_MASK, v.z, d), __shfl_up_sync(FULL_MASK, v.w, d));
}
__device__ __forceinline__ uint32_t diff4(uint4 a, uint4 b) {
    return (a.x ^ b.x) | (a.y ^ b.y) | (a.z ^ b.z) | (a.w ^ b.w);
}

// Fast pass (every arc source a staged tile slot).  The run is walked in
// SPAN-node chunks (ascending forward, descending backward); lane l owns SEG
// consecutive nodes of the chunk in pass order and handles 4 sources at a
// time.  Per node,
//   c_v = min(d[v], min over non-carry arcs u -> v of d[u] + w)
// with sources in earlier chunks (or the halo) already final for this pass
// and sources in the same chunk as they were at the chunk's start.  Then the
// carry chain x_v = min(c_v, x_prev + w(prev, v)) is solved exactly: each
// lane runs it over its own nodes (x = min(L, x_in + S) with L the chain
// from infinity and S the summed carry weights), a (min, +) warp scan over
// the lanes' (L_last, S_last) pairs gives every lane its x_in, and a fix-up
// writes min(L, x_in + S).  The forward pass takes arcs from lower ids, the
// backward pass from higher ids, so every arc is relaxed once per sweep.
template <int TILE, bool FWD, int NQ>
__device__ __forceinline__ bool scan_pass(TileSmem<TILE>& sm, int len, int lane, int q0) {
    constexpr int NCH = TILE / 32;
    const uint2* xa = sm.xarcs;
    bool changed = false;
    const int nchunks = (len + SPAN - 1) / SPAN;
    for (int cc = 0; cc < nchunks; ++cc) {
        const int c = FWD ? cc : nchunks - 1 - cc;  // chunk covers ids [SPAN c, SPAN c + SPAN)
        if (FWD) {
            const int last_grp = min(NCH - 1, (min(len, (c + 1) * SPAN) - 1) >> 5);
            cp_async_wait_pending(NCH - 1 - last_grp);  // own rows of the chunk have landed
            __syncwarp();
        }
        int p_own[SEG], p0[SEG], p1[SEG];
        bool valid[SEG];
        uint32_t w[SEG], S[SEG], w0[SEG], w1[SEG], xb[SEG], xe[SEG];
#pragma unroll
        for (int j = 0; j < SEG; ++j) {
            // pass order: forward node SPAN c + SEG l + j, backward node SPAN c + SPAN - 1 - SEG l - j
            const int node = FWD ? c * SPAN + SEG * lane + j : c * SPAN + (SPAN - 1) - SEG * lane - j;
            valid[j] = node < len;
            const int ii = valid[j] ? node : 0;
            p_own[j] = FWD ? c * SPAN + j * 32 + lane : c * SPAN + (SEG - 1 - j) * 32 + 31 - lane;
            const uint4 a = sm.ix[2 * ii];
            const uint4 b = sm.ix[2 * ii + 1];
            w[j] = valid[j] ? min(FWD ? a.x : a.y, INF_U) : INF_U;
            S[j] = j == 0 ? w[0] : min(S[j > 0 ? j - 1 : 0] + w[j], INF_U);
            p0[j] = pos_of(FWD ? static_cast<int>(b.y & 0xFFFFu) : static_cast<int>(b.z & 0xFFFFu));
            p1[j] = pos_of(static_cast<int>(b.y >> 16));
            w0[j] = valid[j] ? (FWD ? a.z : b.x) : NO_CARRY;
            w1[j] = valid[j] ? a.w : NO_CARRY;
            xb[j] = 0u;
            xe[j] = 0u;
            if (valid[j] && (b.z & IX_EXTRA)) {
                const uint32_t nfx = (b.z >> 16) & 0xFFu;
                xb[j] = FWD ? b.w : b.w + nfx;
                xe[j] = b.w + nfx + (FWD ? 0u : (b.z >> 25) & 0x7Fu);
            }
        }
        // carry-weight prefixes over the lanes: W[k] = summed S over lanes
        // (lane - 2^k, lane]; lanes below 2^k get INF_U, which never wins
        uint32_t W[5];
        {
            uint32_t acc = S[SEG - 1];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                W[k] = lane >= (1 << k) ? acc : INF_U;
                const uint32_t o = __shfl_up_sync(FULL_MASK, acc, 1 << k);
                if (lane >= (1 << k)) acc = min(acc + o, INF_U);
            }
        }
        // the node before the chunk in pass order feeds lane 0 (already final)
        const int prev = FWD ? c * SPAN - 1 : (c + 1) * SPAN;
        const bool has_prev = lane == 0 && (FWD ? prev >= 0 : prev < len);
        const int p_prev = pos_of(has_prev ? prev : 0);
        uint32_t drop[SEG];
#pragma unroll
        for (int j = 0; j < SEG; ++j) drop[j] = 0u;
#pragma unroll
        for (int qq = 0; qq < NQ; ++qq) {
            const int q = q0 + qq;
            const uint4* rq = sm.rows[q];
            uint4 cur[SEG], L[SEG];
#pragma unroll
            for (int j = 0; j < SEG; ++j) {
                cur[j] = rq[p_own[j]];
                uint4 cv = addmin4(rq[p0[j]], w0[j], cur[j]);
                if constexpr (FWD) cv = addmin4(rq[p1[j]], w1[j], cv);
                for (uint32_t e = xb[j]; e < xe[j]; ++e) cv = addmin4(rq[pos_of(xa[e].x)], xa[e].y, cv);
                L[j] = j == 0 ? cv : addmin4(L[j > 0 ? j - 1 : 0], w[j], cv);
            }
            uint4 cin = make_uint4(INF_U, INF_U, INF_U, INF_U);
            uint4 A = L[SEG - 1];
            if (has_prev) {
                cin = rq[p_prev];
                A = addmin4(cin, S[SEG - 1], A);
            }
#pragma unroll
            for (int k = 0; k < 5; ++k) A = addmin4(shfl_up4(A, 1 << k), W[k], A);
            uint4 xin = shfl_up4(A, 1);
            if (lane == 0) xin = cin;
#pragma unroll
            for (int j = 0; j < SEG; ++j) {
                // x <= cur always; store where valid, note any change
                const uint4 x = addmin4(xin, S[j], L[j]);
                if (valid[j]) sm.rows[q][p_own[j]] = x;
                drop[j] |= diff4(x, cur[j]);
            }
        }
        bool any = false;
#pragma unroll
        for (int j = 0; j < SEG; ++j) any |= valid[j] && drop[j] != 0u;
        if (__any_sync(FULL_MASK, any)) {
            changed = true;
#pragma unroll
            for (int j = 0; j < SEG; ++j) {
                if (valid[j] && drop[j] != 0u) {
                    const int node = FWD ? c * SPAN + SEG * lane + j : c * SPAN + (SPAN - 1) - SEG * lane - j;
                    sm.dirtyb[node] = 1;
                }
            }
        }
        __syncwarp();  // stores of this chunk visible before the next chunk reads them
    }
    return changed;
}

template <int TILE, int NQ>
__device__ __forceinline__ bool passes_fast(TileSmem<TILE>& sm, int len, int lane, int q0) {
    const bool f = scan_pass<TILE, true, NQ>(sm, len, lane, q0);
    cp_async_wait_pending(0);
    __syncwarp();
    const bool b = scan_pass<TILE, false, NQ>(sm, len, lane, q0);
    return f || b;
}

// Generic passes for runs the fast path cannot take (a single node with more
// in-neighbours than the tile holds): descriptors and arcs from global memory,
// sources from the tile or, past its capacity, from the rows in L2.
template <int TILE>
__device__ __noinline__ bool passes_generic(const BfParams& p, TileSmem<TILE>& sm, int4 rs, int len, int lane,
                                            int64_t lane_off) {
    uint32_t* words = reinterpret_cast<uint32_t*>(&sm.rows[0][0]);
    // word of source lane `lane` of tile slot i in the quad-major layout
    auto at = [&](int i) -> uint32_t& {
        return words[((lane >> 2) * TileSmem<TILE>::PLANE + pos_of(i)) * 4 + (lane & 3)];
    };
    const uint32_t* rows = p.seg.rows;
    const int64_t ld = p.seg.ld;
    bool changed = false;
    cp_async_wait_pending(0);
    __syncwarp();
    uint32_t carry = INF_U;
    for (int i = 0; i < len; ++i) {
        const int4 d = __ldg(p.g.node_desc + run_node(rs, i));
        const uint32_t cur = at(i);
        uint32_t best = __viaddmin_u32(carry, static_cast<uint32_t>(d.x), cur);
        for (int q = d.z; q < d.w; ++q) {
            const uint2 e = __ldg(p.g.arc2 + q);
            const uint32_t x = (e.x & GLOBAL_REF) ? ld_l2(rows + static_cast<int64_t>(e.x & ~GLOBAL_REF) * ld + lane_off + lane)
                                                  : at(static_cast<int>(e.x));
            best = __viaddmin_u32(x, e.y, best);
        }
        const bool dropped = best < cur;
        if (dropped) at(i) = best;
        const unsigned m = __ballot_sync(FULL_MASK, dropped);
        if (m) {
            changed = true;
            if (lane == 0) sm.dirtyb[i] = 1;
        }
        carry = best;
    }
    carry = INF_U;
    for (int i = len - 1; i >= 0; --i) {
        const int4 d = __ldg(p.g.node_desc + run_node(rs, i));
        const int end = __ldg(&p.g.node_desc[run_node(rs, i) + 1].z);
        const uint32_t cur = at(i);
        uint32_t best = __viaddmin_u32(carry, static_cast<uint32_t>(d.y), cur);
        for (int q = d.w; q < end; ++q) {
            const uint2 e = __ldg(p.g.arc2 + q);
            best = __viaddmin_u32(at(static_cast<int>(e.x)), e.y, best);
        }
        const bool dropped = best < cur;
        if (dropped) at(i) = best;
        const unsigned m = __ballot_sync(FULL_MASK, dropped);
        if (m) {
            changed = true;
            if (lane == 0) sm.dirtyb[i] = 1;
        }
        carry = best;
    }
    return changed;
}

// One tile, processed by the whole CTA: NQW warps, warp w owning the 8 / NQW
// quads (4 sources each) starting at quad w * (8 / NQW).  Every warp stages
// its own quads of the halo and of the own rows (own rows in 32-node chunks,
// so the forward pass can start on the first chunk while the rest is in
// flight); the run's descriptors and extra arcs are staged by all threads.
// Then each warp runs the forward and backward passes over its quads, and
// the CTA writes back the rows that dropped.  Returns true (CTA-uniform) if
// any row dropped.  Each pass relaxes every arc of its direction once.
template <int TILE, int NQW>
__device__ __forceinline__ bool sweep_tile(const BfParams& p, int r, int g, TileSmem<TILE>& sm,
                                           unsigned long long& node_visits) {
    constexpr int NCH = TILE / 32;
    constexpr int NQ = 8 / NQW;      // quads per warp
    constexpr int NPI = 32 / NQ;     // nodes per warp instruction when staging
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int q0 = warp * NQ;
    // Staging: lanes [NPI m', NPI m' + NPI) stage quad q0 + m' of NPI nodes; a
    // lane's node offset interleaves parities (even nodes on the low half), so
    // the 8 lanes of a 16-byte access phase hit 8 consecutive positions.
    const int qs = q0 + lane / NPI;  // the quad this lane stages
    const int soff = 2 * (lane % (NPI / 2)) + (lane % NPI) / (NPI / 2);
    const int4 rs = __ldg(p.g.run_seg + r);
    const int len = rs.y + rs.w;
    const int h0 = __ldg(p.g.halo_ptr + r);
    const int hn = __ldg(p.g.halo_ptr + r + 1) - h0;
    const bool simple = (__ldg(p.g.run_flags + r) & RUN_SIMPLE) != 0;
    const int64_t ld = p.seg.ld;
    const int64_t lane_off = seg_col0(p.seg, g);
    uint32_t* rows = p.seg.rows;
    const int2 rx = __ldg(p.g.run_x + r);

    // group 0: descriptors and extra arcs (all threads), this warp's quads of the halo rows
    if (simple) {
        for (int i = tid; i < 2 * len; i += 32 * NQW)
            cp_async16(&sm.ix[i], &p.g.node_ix[2 * static_cast<int64_t>(run_node(rs, i >> 1)) + (i & 1)]);
        for (int q = rx.x + tid; q < rx.y; q += 32 * NQW) cp_async8_ca(&sm.xarcs[q - rx.x], &p.g.xarc2[q]);
    }
    for (int i0 = 0; i0 < hn; i0 += NPI) {
        const int i = i0 + soff;
        if (i >= hn) break;
        const int node = __ldg(p.g.halo_nodes + h0 + i);
        cp_async16(&sm.rows[qs][pos_of(len + i)], rows + static_cast<int64_t>(node) * ld + lane_off + qs * 4);
    }
    cp_async_commit();
    // groups 1..NCH: this warp's quads of the own rows, 32 nodes each (empty groups complete at once)
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        const int base = c * 32;
        if (base < len) {
#pragma unroll
            for (int t = 0; t < NQ; ++t) {
                const int i = base + t * NPI + soff;
                if (i < len)
                    cp_async16(&sm.rows[qs][pos_of(i)],
                               rows + static_cast<int64_t>(run_node(rs, i)) * ld + lane_off + qs * 4);
            }
        }
        cp_async_commit();
    }
    for (int i = tid; i < len; i += 32 * NQW) sm.dirtyb[i] = 0;
    // Slots of the last SPAN-block past the staged rows are read (as nodes that
    // do not exist) by the chunk scans; they must hold INF, not whatever the
    // shared memory held before: a value above 2^31 plus a blocking INF
    // weight would wrap to a small number.
    {
        const int top = ((len + SPAN - 1) / SPAN) * SPAN;
        for (int t = len + hn + soff; t < top; t += NPI)
            sm.rows[qs][pos_of(t)] = make_uint4(INF_U, INF_U, INF_U, INF_U);
    }
    cp_async_wait_pending(NCH - 1);  // group 0 and the first row chunk of this thread landed
    __syncthreads();                 // descriptors staged by other warps are visible

    bool mine = false;
    if (simple) {
        mine = passes_fast<TILE, NQ>(sm, len, lane, q0);
    } else {
        cp_async_wait_pending(0);
        __syncthreads();  // every quad staged
        if (warp == 0) mine = passes_generic<TILE>(p, sm, rs, len, lane, lane_off);
    }
    const bool changed = __syncthreads_or(mine) != 0;
    if (tid == 0) node_visits += static_cast<unsigned long long>(len);
    if (changed) {
        // 4 * NQW nodes per step, 8 threads x 16 bytes per node row
        const int sub = tid >> 3, q = tid & 7;
        for (int i0 = 0; i0 < len; i0 += 4 * NQW) {
            const int i = i0 + sub;
            if (i < len && sm.dirtyb[i])
                __stcg(reinterpret_cast<uint4*>(rows + static_cast<int64_t>(run_node(rs, i)) * ld + lane_off + q * 4),
                       sm.rows[q][pos_of(i)]);
        }
    }
    __syncthreads();  // shared memory free for the next tile
    return changed;
}

template <int TILE, int NQW>
// NQW warps per CTA, each owning 8 / NQW quads of a tile's 32 sources.
__global__ void __launch_bounds__(32 * NQW, NQW == 8 ? 2 : 5) bf_sweeps_kernel(BfParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem<TILE>& sm = *reinterpret_cast<TileSmem<TILE>*>(smem_raw);
    __shared__ int s_item;

    const int n_lanes = segment_lanes(p.seg);
    const int G = (n_lanes + 31) >> 5;
    if (G == 0) return;  // same decision in every block
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthreads = gridDim.x * blockDim.x;

    // seeds: writing d[s][s] = 0 is the change of "sweep 0": the tile holding
    // each source gets stamp 1, and sweep 1 visits it and the tiles it feeds
    for (int b = gtid; b < n_lanes; b += nthreads) {
        const int r = __ldg(p.g.run_of_node + p.seg.src[p.seg.first + b]);
        p.w.stamp[static_cast<int64_t>(r) * G + (b >> 5)] = 1;
    }
    if (!grid_sync(p.w.bar, p.w.err, p.w.max_spins)) return;
    build_list(p, G, 1, true, p.w.list0, p.w.counts + 0);
    if (!grid_sync(p.w.bar, p.w.err, p.w.max_spins)) return;

    unsigned long long tiles = 0, nodes = 0, bytes = 0, reread = 0;
    int cur = 0;
    int sweep = 1;
    for (;; ++sweep) {
        const int cnt = ld_volatile(p.w.counts + cur);
        if (gtid == 0 && sweep <= p.w.trace_cap) {
            // frontier of this sweep and when it started (the last entry, 0 tiles, is the end)
            long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            p.w.trace[2 * (sweep - 1)] = cnt;
            p.w.trace[2 * (sweep - 1) + 1] = t;
        }
        if (cnt == 0) break;
        if (sweep > p.g.V + 1) {
            if (gtid == 0) atomicCAS(p.w.err, 0, WR_EINTERNAL);
            break;
        }
        if (gtid == 0) {
            p.w.counts[cur ^ 1] = 0;
            p.w.counts[2 + (cur ^ 1)] = 0;
        }
        const int32_t* list = cur ? p.w.list1 : p.w.list0;
        for (;;) {
            if (threadIdx.x == 0) s_item = atomicAdd(p.w.counts + 2 + cur, 1);  // dynamic tile scheduling
            __syncthreads();
            const int it = s_item;
            __syncthreads();
            if (it >= cnt) break;
            const int item = __ldcg(list + it);
            const int r = item / G;
            const int g = item - r * G;
            // the run's descriptors count once per sweep, whichever of its groups comes first
            int first_visit = 0;
            if (threadIdx.x == 0) first_visit = atomicMax(p.w.run_stamp + r, sweep) < sweep;
            const bool ch = sweep_tile<TILE, NQW>(p, r, g, sm, nodes);
            if (threadIdx.x == 0) {
                if (ch) p.w.stamp[item] = sweep + 1;
                ++tiles;
                const unsigned long long meta = static_cast<unsigned long long>(__ldg(p.g.run_meta_bytes + r));
                bytes += (first_visit ? meta : 0ull) +
                         256ull * static_cast<unsigned long long>(__ldg(&p.g.run_seg[r].y) + __ldg(&p.g.run_seg[r].w));
                reread += first_visit ? 0ull : meta;
            }
        }
        if (!grid_sync(p.w.bar, p.w.err, p.w.max_spins)) break;
        build_list(p, G, sweep + 1, true, cur ? p.w.list0 : p.w.list1, p.w.counts + (cur ^ 1));
        if (!grid_sync(p.w.bar, p.w.err, p.w.max_spins)) break;
        cur ^= 1;
    }
    if (threadIdx.x == 0 && tiles) {
        atomicAdd(p.w.stats + 1, tiles);
        atomicAdd(p.w.stats + 2, nodes);
        atomicAdd(p.w.stats + 3, bytes);
        atomicAdd(p.w.stats + 5, reread);
    }
    if (gtid == 0) atomicAdd(p.w.stats + 0, static_cast<unsigned long long>(sweep - 1));
}

// ---------------------------------------------------------------------------

template <int TILE, int NQW>
static int prepare_one(int device, BfLaunchInfo* info) {
    const size_t smem = sizeof(TileSmem<TILE>);
    auto* fn = bf_sweeps_kernel<TILE, NQW>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
        return WR_ECUDA;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 32 * NQW, smem) != cudaSuccess || occ < 1)
        return WR_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return WR_ECUDA;
    info->blocks = occ * sms;
    info->threads = 32 * NQW;
    info->smem = smem;
    info->fn = reinterpret_cast<const void*>(fn);
    return WR_OK;
}

int bf_prepare(int tile_cap, int warps, int device, BfLaunchInfo* info) {
    if (warps == 0) warps = tile_cap >= 512 ? 8 : 4;
    if (warps != 4 && warps != 8) return WR_EINVAL;
    switch (tile_cap * 16 + warps) {
        case 128 * 16 + 4: return prepare_one<128, 4>(device, info);
        case 128 * 16 + 8: return prepare_one<128, 8>(device, info);
        case 256 * 16 + 4: return prepare_one<256, 4>(device, info);
        case 256 * 16 + 8: return prepare_one<256, 8>(device, info);
        case 512 * 16 + 8: return prepare_one<512, 8>(device, info);
        default: return WR_EINVAL;
    }
}

cudaError_t bf_launch_init(const DevGraph& g, const BfSegment& seg, const BfWork& w, cudaStream_t s) {
    BfParams p{g, seg, w};
    bf_init_kernel<<<1216, 256, 0, s>>>(p);  // 8 blocks per SM
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || seg.src_index) return e;  // seeds written with the fill
    bf_seed_kernel<<<(seg.lanes + 255) / 256 + (seg.lanes == 0), 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t bf_launch_sweeps(const DevGraph& g, const BfSegment& seg, const BfWork& w, const BfLaunchInfo& info,
                             cudaStream_t s) {
    BfParams p{g, seg, w};
    void* args[] = {&p};
    if (!info.fn) return cudaErrorInvalidValue;
    return cudaLaunchCooperativeKernel(info.fn, dim3(info.blocks), dim3(info.threads), args, info.smem, s);
}

// out[b * ld_out + v] = rows[v * ld + b]: 32 x 32 tiles through shared memory.
__global__ void bf_rows_out_kernel(BfSegment seg, int32_t V, int32_t* out, int64_t ld_out) {
    __shared__ uint32_t t[32][33];
    const int n_lanes = segment_lanes(seg);
    const int vb = blockIdx.x * 32, bb = blockIdx.y * 32;
    if (bb >= n_lanes) return;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int v = vb + i, b = bb + threadIdx.x;
        if (v < V && b < n_lanes) t[i][threadIdx.x] = seg.rows[static_cast<int64_t>(v) * seg.ld + b];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int b = bb + i, v = vb + threadIdx.x;
        if (v < V && b < n_lanes) out[static_cast<int64_t>(seg.first + b) * ld_out + v] = static_cast<int32_t>(t[threadIdx.x][i]);
    }
}

cudaError_t bf_launch_rows_out(const BfSegment& seg, int32_t V, int32_t* out, int64_t ld_out, cudaStream_t s) {
    dim3 grid((V + 31) / 32, (seg.lanes + 31) / 32);
    bf_rows_out_kernel<<<grid, dim3(32, 8), 0, s>>>(seg, V, out, ld_out);
    return cudaGetLastError();
}

// Scale-workload consumer: sub[(first+b) * n_dst + j] = rows[dst[j] * ld + b] and
// check[first+b] += sum over v of rows[v * ld + b] * (2v + 1)  (mod 2^64).
__global__ void bf_submatrix_kernel(BfSegment seg, int32_t V, int32_t n_dst, const int32_t* dst, int32_t* sub,
                                    unsigned long long* check) {
    const int n_lanes = segment_lanes(seg);
    const int b = blockIdx.y * 32 + (threadIdx.x & 31);
    const int sub_row = threadIdx.x >> 5;  // 8 node strips per block
    if (blockIdx.y * 32 >= n_lanes) return;
    unsigned long long acc = 0;
    const int64_t per = (static_cast<int64_t>(V) + gridDim.x - 1) / gridDim.x;
    const int64_t v0 = per * blockIdx.x, v1 = min(static_cast<int64_t>(V), v0 + per);
    if (b < n_lanes) {
        for (int64_t v = v0 + sub_row; v < v1; v += 8)
            acc += static_cast<unsigned long long>(__ldcg(seg.rows + v * seg.ld + b)) *
                   static_cast<unsigned long long>(2 * v + 1);
        atomicAdd(check + seg.first + b, acc);
    }
    // the submatrix entries, spread over every block of this lane group (a few loads per thread)
    if (b < n_lanes) {
        for (int j = blockIdx.x * 8 + sub_row; j < n_dst; j += gridDim.x * 8)
            sub[static_cast<int64_t>(seg.first + b) * n_dst + j] =
                static_cast<int32_t>(__ldcg(seg.rows + static_cast<int64_t>(dst[j]) * seg.ld + b));
    }
}

cudaError_t bf_launch_submatrix(const BfSegment& seg, int32_t V, int32_t n_dst, const int32_t* dst, int32_t* sub,
                                unsigned long long* check, cudaStream_t s) {
    dim3 grid(256, (seg.lanes + 31) / 32);
    bf_submatrix_kernel<<<grid, 256, 0, s>>>(seg, V, n_dst, dst, sub, check);
    return cudaGetLastError();
}

}  // namespace wr
