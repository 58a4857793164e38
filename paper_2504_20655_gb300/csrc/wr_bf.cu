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
#include "wr_device.cuh"

namespace wr {

struct BfParams {
    DevGraph g;
    BfSegment seg;
    BfWork w;
};

__device__ __forceinline__ int segment_lanes(const BfSegment& seg) {
    const int n_src = seg.n_src_dev ? ld_l2(seg.n_src_dev) : seg.n_src_host;
    return min(max(n_src - seg.first, 0), seg.lanes);
}

// rows := INF except dist(src_b, src_b) = 0; stamps := 0; counters := 0.
__global__ void bf_init_kernel(BfParams p) {
    const int n_lanes = segment_lanes(p.seg);
    const int G = (n_lanes + 31) >> 5;
    const int64_t width = static_cast<int64_t>(G) * 32;
    const int64_t n = static_cast<int64_t>(p.g.V) * width;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    // 4 lanes per thread (16-byte stores); width is a multiple of 32
    for (int64_t e = t0 * 4; e < n; e += stride * 4) {
        const int64_t v = e / width;
        const int b = static_cast<int>(e - v * width);
        uint4 val = make_uint4(INF_U, INF_U, INF_U, INF_U);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int lane = b + q;
            if (lane < n_lanes && p.seg.src[p.seg.first + lane] == v) (&val.x)[q] = 0u;
        }
        __stcg(reinterpret_cast<uint4*>(p.seg.rows + v * p.seg.ld + b), val);
    }
    const int64_t n_items = static_cast<int64_t>(p.g.n_runs) * G;
    for (int64_t i = t0; i < n_items; i += stride) p.w.stamp[i] = 0;
    if (t0 < 4) p.w.counts[t0] = 0;
    if (t0 == 0) {
        p.w.bar->count = 0;
        p.w.bar->gen = 0;
    }
}

// Append the items whose stamp (or, with nbrs, an in-neighbour run's stamp
// in the same group) equals match.
__device__ __forceinline__ void build_list(const BfParams& p, int G, int match, bool nbrs, int32_t* out,
                                           int32_t* count) {
    const int64_t n_items = static_cast<int64_t>(p.g.n_runs) * G;
    const int lane = threadIdx.x & 31;
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x; base < n_items;
         base += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t item = base + threadIdx.x;
        bool act = false;
        if (item < n_items) {
            act = ld_l2(p.w.stamp + item) == match;
            if (!act && nbrs) {
                const int r = static_cast<int>(item / G);
                const int g = static_cast<int>(item - static_cast<int64_t>(r) * G);
                const int q1 = __ldg(p.g.rin_ptr + r + 1);
                for (int q = __ldg(p.g.rin_ptr + r); q < q1; ++q) {
                    const int rr = __ldg(p.g.rin_list + q);
                    if (ld_l2(p.w.stamp + static_cast<int64_t>(rr) * G + g) == match) {
                        act = true;
                        break;
                    }
                }
            }
        }
        const unsigned m = __ballot_sync(FULL_MASK, act);
        if (m) {
            const int leader = __ffs(m) - 1;
            int pos = 0;
            if (lane == leader) pos = atomicAdd(count, __popc(m));
            pos = __shfl_sync(FULL_MASK, pos, leader);
            if (act) out[pos + __popc(m & lanemask_lt())] = static_cast<int32_t>(item);
        }
    }
}

// One tile: stage, forward pass, backward pass, write back dropped rows.
// Returns true (warp-uniform) if any row of the tile dropped.
template <int TILE>
__device__ __forceinline__ bool sweep_tile(const BfParams& p, int r, int g, uint32_t* tile, uint32_t* dirty,
                                           int lane, unsigned long long& node_visits) {
    const int r0 = __ldg(p.g.run_ptr + r);
    const int len = __ldg(p.g.run_ptr + r + 1) - r0;
    const int h0 = __ldg(p.g.halo_ptr + r);
    const int hn = __ldg(p.g.halo_ptr + r + 1) - h0;
    const int64_t ld = p.seg.ld;
    const int64_t lane_off = static_cast<int64_t>(g) * 32;
    uint32_t* rows = p.seg.rows;

    // stage: 8 threads x 16 bytes per node row of the group
    const int total = len + hn;
    for (int i0 = 0; i0 < total; i0 += 4) {
        const int i = i0 + (lane >> 3);
        if (i < total) {
            const int node = i < len ? r0 + i : __ldg(p.g.halo_nodes + h0 + (i - len));
            cp_async16(tile + i * 32 + (lane & 7) * 4, rows + static_cast<int64_t>(node) * ld + lane_off + (lane & 7) * 4);
        }
    }
    if (lane < TILE / 32) dirty[lane] = 0u;
    cp_async_wait_all();
    __syncwarp();

    bool changed = false;
    // forward: arcs from lower ids (and the halo); carry = arc v-1 -> v
    uint32_t carry = INF_U;
#pragma unroll 2
    for (int i = 0; i < len; ++i) {
        const int4 d = __ldg(p.g.node_desc + r0 + i);
        const uint32_t cur = tile[i * 32 + lane];
        uint32_t best = __viaddmin_u32(carry, static_cast<uint32_t>(d.x), cur);
        for (int a = d.z; a < d.w; ++a) {
            const uint32_t ref = __ldg(p.g.arc_ref + a);
            const uint32_t wt = __ldg(p.g.arc_w + a);
            const uint32_t x = (ref & GLOBAL_REF)
                                   ? ld_l2(rows + static_cast<int64_t>(ref & ~GLOBAL_REF) * ld + lane_off + lane)
                                   : tile[ref * 32 + lane];
            best = __viaddmin_u32(x, wt, best);
        }
        const bool dropped = best < cur;
        if (dropped) tile[i * 32 + lane] = best;
        const unsigned m = __ballot_sync(FULL_MASK, dropped);
        if (m) {
            changed = true;
            if (lane == 0) dirty[i >> 5] |= 1u << (i & 31);
        }
        carry = best;
    }
    // backward: arcs from higher ids; carry = arc v+1 -> v
    carry = INF_U;
    int next_begin = __ldg(&p.g.node_desc[r0 + len].z);
#pragma unroll 2
    for (int i = len - 1; i >= 0; --i) {
        const int4 d = __ldg(p.g.node_desc + r0 + i);
        const uint32_t cur = tile[i * 32 + lane];
        uint32_t best = __viaddmin_u32(carry, static_cast<uint32_t>(d.y), cur);
        for (int a = d.w; a < next_begin; ++a) {
            const uint32_t ref = __ldg(p.g.arc_ref + a);
            const uint32_t wt = __ldg(p.g.arc_w + a);
            best = __viaddmin_u32(tile[ref * 32 + lane], wt, best);
        }
        next_begin = d.z;
        const bool dropped = best < cur;
        if (dropped) tile[i * 32 + lane] = best;
        const unsigned m = __ballot_sync(FULL_MASK, dropped);
        if (m) {
            changed = true;
            if (lane == 0) dirty[i >> 5] |= 1u << (i & 31);
        }
        carry = best;
    }
    node_visits += static_cast<unsigned long long>(len);
    __syncwarp();
    if (changed) {
        for (int wd = 0; wd < (len + 31) / 32; ++wd) {
            uint32_t bits = dirty[wd];
            while (bits) {
                const int i = wd * 32 + __ffs(bits) - 1;
                bits &= bits - 1;
                __stcg(rows + static_cast<int64_t>(r0 + i) * ld + lane_off + lane, tile[i * 32 + lane]);
            }
        }
    }
    __syncwarp();
    return changed;
}

template <int TILE, int NW>
__global__ void __launch_bounds__(NW * 32) bf_sweeps_kernel(BfParams p) {
    extern __shared__ uint32_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t* tile = smem + warp * TILE * 32;
    uint32_t* dirty = smem + NW * TILE * 32 + warp * (TILE / 32);

    const int n_lanes = segment_lanes(p.seg);
    const int G = (n_lanes + 31) >> 5;
    if (G == 0) return;  // same decision in every block
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nthreads = gridDim.x * blockDim.x;
    const int gwarp = blockIdx.x * NW + warp;
    const int nwarps = gridDim.x * NW;

    // seeds: writing d[s][s] = 0 is the change of "sweep 0": the tile holding
    // each source gets stamp 1, and sweep 1 visits it and the tiles it feeds
    for (int b = gtid; b < n_lanes; b += nthreads) {
        const int r = __ldg(p.g.run_of_node + p.seg.src[p.seg.first + b]);
        p.w.stamp[static_cast<int64_t>(r) * G + (b >> 5)] = 1;
    }
    if (!grid_sync(p.w.bar, p.w.err, p.w.max_spins)) return;
    build_list(p, G, 1, true, p.w.list0, p.w.counts + 0);
    if (!grid_sync(p.w.bar, p.w.err, p.w.max_spins)) return;

    unsigned long long tiles = 0, nodes = 0, bytes = 0;
    int cur = 0;
    int sweep = 1;
    for (;; ++sweep) {
        const int cnt = ld_volatile(p.w.counts + cur);
        if (cnt == 0) break;
        if (sweep > p.g.V + 1) {
            if (gtid == 0) atomicCAS(p.w.err, 0, WR_EINTERNAL);
            break;
        }
        if (gtid == 0) p.w.counts[cur ^ 1] = 0;
        const int32_t* list = cur ? p.w.list1 : p.w.list0;
        for (int it = gwarp; it < cnt; it += nwarps) {
            const int item = __ldcg(list + it);
            const int r = item / G;
            const int g = item - r * G;
            const bool ch = sweep_tile<TILE>(p, r, g, tile, dirty, lane, nodes);
            if (ch && lane == 0) p.w.stamp[item] = sweep + 1;
            ++tiles;
            bytes += static_cast<unsigned long long>(__ldg(p.g.run_meta_bytes + r)) +
                     256ull * static_cast<unsigned long long>(__ldg(p.g.run_ptr + r + 1) - __ldg(p.g.run_ptr + r));
        }
        if (!grid_sync(p.w.bar, p.w.err, p.w.max_spins)) break;
        build_list(p, G, sweep + 1, true, cur ? p.w.list0 : p.w.list1, p.w.counts + (cur ^ 1));
        if (!grid_sync(p.w.bar, p.w.err, p.w.max_spins)) break;
        cur ^= 1;
    }
    if (lane == 0 && tiles) {
        atomicAdd(p.w.stats + 1, tiles);
        atomicAdd(p.w.stats + 2, nodes);
        atomicAdd(p.w.stats + 3, bytes);
    }
    if (gtid == 0) atomicAdd(p.w.stats + 0, static_cast<unsigned long long>(sweep - 1));
}

// ---------------------------------------------------------------------------

template <int TILE, int NW>
static size_t sweep_smem() {
    return static_cast<size_t>(NW) * (TILE * 32 * sizeof(uint32_t) + (TILE / 32) * sizeof(uint32_t));
}

template <int TILE, int NW>
static int prepare_one(int device, BfLaunchInfo* info) {
    const size_t smem = sweep_smem<TILE, NW>();
    if (cudaFuncSetAttribute(bf_sweeps_kernel<TILE, NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem)) != cudaSuccess)
        return WR_ECUDA;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bf_sweeps_kernel<TILE, NW>, NW * 32, smem) !=
            cudaSuccess ||
        occ < 1)
        return WR_ECUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return WR_ECUDA;
    info->blocks = occ * sms;
    info->threads = NW * 32;
    info->smem = smem;
    return WR_OK;
}

constexpr int BF_NW = 4;

int bf_prepare(int tile_cap, int device, BfLaunchInfo* info) {
    switch (tile_cap) {
        case 64: return prepare_one<64, BF_NW>(device, info);
        case 128: return prepare_one<128, BF_NW>(device, info);
        case 256: return prepare_one<256, BF_NW>(device, info);
        default: return WR_EINVAL;
    }
}

cudaError_t bf_launch_init(const DevGraph& g, const BfSegment& seg, const BfWork& w, cudaStream_t s) {
    BfParams p{g, seg, w};
    bf_init_kernel<<<1024, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t bf_launch_sweeps(const DevGraph& g, const BfSegment& seg, const BfWork& w, const BfLaunchInfo& info,
                             cudaStream_t s) {
    BfParams p{g, seg, w};
    void* args[] = {&p};
    const void* fn = nullptr;
    switch (g.tile_cap) {
        case 64: fn = reinterpret_cast<const void*>(bf_sweeps_kernel<64, BF_NW>); break;
        case 128: fn = reinterpret_cast<const void*>(bf_sweeps_kernel<128, BF_NW>); break;
        case 256: fn = reinterpret_cast<const void*>(bf_sweeps_kernel<256, BF_NW>); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaLaunchCooperativeKernel(fn, dim3(info.blocks), dim3(info.threads), args, info.smem, s);
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
    if (blockIdx.x == 0 && b < n_lanes) {
        for (int j = sub_row; j < n_dst; j += 8)
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
