// Node-level routes: the nodes a route passes, leg by leg.
//
// A leg s -> t of an order's route is the shortest path whose node sequence,
// read backward from t, is lexicographically smallest: walking back from t,
// the predecessor of v is the smallest node id u with an arc u -> v and
// dist(s, u) + w(u, v) = dist(s, v).  With positive arc weights every such
// walk reaches s in at most V - 1 steps.  dist(s, .) is the row of s in the
// current Bellman-Ford segment, so each leg is walked in the segment that
// holds its source.
//
// A route is the depot, then each leg's nodes after its first (closed tour:
// depot -> picks in the given order -> depot), or in open-path mode the
// first pick and then the legs between consecutive picks.
//
// Three kinds of launch: the count walk (every leg's length, in the segment
// holding its source; a leg of at most cache_cap nodes also leaves its nodes
// in the leg cache), the copy (cached legs into the output, any segment) and
// the write walk (legs longer than the cache, in their segment).  A walk step
// issues the loads of all of a node's in-arcs before it compares them.
#include "wr_bf_common.cuh"

namespace wr {

enum PathMode { PATH_COUNT = 0, PATH_WRITE = 1, PATH_COPY = 2 };

struct PathArgs {
    int32_t n;
    const int64_t* offs;
    const int32_t* picks;
    const int32_t* perm;          // per order, 0-based indices into its picks
    const int32_t* order_status;  // from the source selection
    int open_path;
    int32_t depot;
    const int32_t* src_index;
    BfSegment seg;
    const int64_t* in_ptr;        // in-arc CSR with node ids
    const int32_t* in_src;
    const int32_t* in_w;
    const int4* in4;              // per node 2 x int4: up to 4 in-arcs {u0, w0, u1, w1}, {u2, w2, u3, w3}
    int32_t V;
    int32_t* leg_len;             // offs[o] + o + q: nodes of leg q after its first; -1 unreachable, -2 invalid
    int32_t* leg_cache;           // slot * cache_cap: a short leg's nodes, walk order (t first)
    int32_t cache_cap;
    int32_t* seg_long;            // count walk: set to 1 when a leg of this segment outgrows the cache
    int mode;
    const int64_t* node_offs;     // write / copy: where each order's nodes start
    int32_t* nodes;               // write / copy: output
};

// Legs of order o: closed tour k + 1 (depot first and last), open path k - 1.
__device__ __forceinline__ int n_legs(const PathArgs& a, int k) { return a.open_path ? max(k - 1, 0) : k + 1; }

__device__ __forceinline__ void leg_ends(const PathArgs& a, int64_t b, int k, int q, int32_t& s, int32_t& t) {
    if (a.open_path) {
        s = a.picks[b + a.perm[b + q]];
        t = a.picks[b + a.perm[b + q + 1]];
    } else {
        s = q == 0 ? a.depot : a.picks[b + a.perm[b + q - 1]];
        t = q == k ? a.depot : a.picks[b + a.perm[b + q]];
    }
}

// Walk one leg backward from t.  Node i of the walk (t is i = 0, s is not
// stored) goes to walk[i] when i < walk_cap and, when out != nullptr, to
// out[len_known - 1 - i] (forward order).  Returns len, -1 if t is
// unreachable, -3 on rows that are not a fixpoint.
constexpr int WALK_ARCS = 4;  // in-arcs whose loads are issued together

__device__ int walk_leg(const PathArgs& a, int32_t s, int32_t t, int32_t lane_s, int32_t* walk, int32_t walk_cap,
                        int32_t* out, int32_t len_known) {
    const uint32_t* rows = a.seg.rows;
    const int64_t ld = a.seg.ld;
    uint32_t dv = __ldcg(rows + static_cast<int64_t>(t) * ld + lane_s);
    if (dv == INF_U) return -1;
    int32_t v = t, len = 0;
    while (v != s && len < a.V) {
        if (len < walk_cap) walk[len] = v;
        if (out) out[len_known - 1 - len] = v;
        ++len;
        int32_t best_u = -1;
        uint32_t best_d = 0;
        // a node of at most 4 in-arcs: its arcs in one 32-byte record (u = -1 pads; u0 = -2
        // marks a node of more, read from the CSR)
        int4 r0 = make_int4(-2, 0, 0, 0), r1 = r0;
        if (a.in4) {
            r0 = __ldg(a.in4 + 2 * static_cast<int64_t>(v));
            r1 = __ldg(a.in4 + 2 * static_cast<int64_t>(v) + 1);
        }
        if (r0.x != -2) {
            const int32_t u[WALK_ARCS] = {r0.x, r0.z, r1.x, r1.z};
            const uint32_t w[WALK_ARCS] = {static_cast<uint32_t>(r0.y), static_cast<uint32_t>(r0.w),
                                           static_cast<uint32_t>(r1.y), static_cast<uint32_t>(r1.w)};
            uint32_t du[WALK_ARCS];
#pragma unroll
            for (int j = 0; j < WALK_ARCS; ++j)
                du[j] = u[j] >= 0 ? __ldcg(rows + static_cast<int64_t>(u[j]) * ld + lane_s) : INF_U;
#pragma unroll
            for (int j = 0; j < WALK_ARCS; ++j)
                if (du[j] != INF_U && static_cast<uint64_t>(du[j]) + w[j] == dv && (best_u < 0 || u[j] < best_u)) {
                    best_u = u[j];
                    best_d = du[j];
                }
        }
        const int64_t e0 = r0.x == -2 ? __ldg(a.in_ptr + v) : 0, e1 = r0.x == -2 ? __ldg(a.in_ptr + v + 1) : 0;
        for (int64_t eb = e0; eb < e1; eb += WALK_ARCS) {
            int32_t u[WALK_ARCS];
            uint32_t w[WALK_ARCS], du[WALK_ARCS];
#pragma unroll
            for (int j = 0; j < WALK_ARCS; ++j) {
                const bool in = eb + j < e1;
                u[j] = in ? __ldg(a.in_src + eb + j) : -1;
                w[j] = in ? static_cast<uint32_t>(__ldg(a.in_w + eb + j)) : 0u;
            }
#pragma unroll
            for (int j = 0; j < WALK_ARCS; ++j)
                du[j] = u[j] >= 0 ? __ldcg(rows + static_cast<int64_t>(u[j]) * ld + lane_s) : INF_U;
#pragma unroll
            for (int j = 0; j < WALK_ARCS; ++j)
                if (du[j] != INF_U && static_cast<uint64_t>(du[j]) + w[j] == dv && (best_u < 0 || u[j] < best_u)) {
                    best_u = u[j];
                    best_d = du[j];
                }
        }
        if (best_u < 0) return -3;  // inconsistent rows (cannot happen at the fixpoint)
        v = best_u;
        dv = best_d;
    }
    return v == s ? len : -3;
}

// One warp per order, one lane per leg.
__global__ void paths_kernel(PathArgs a) {
    const int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (o >= a.n) return;
    const int64_t b = a.offs[o];
    const int k = static_cast<int>(a.offs[o + 1] - b);
    const int64_t lb = b + o;  // leg slots of this order
    bool ok = a.order_status[o] == WR_ORDER_OK;
    if (ok) {
        // the sequence must be a permutation of the order's picks
        unsigned seen = 0;
        for (int q = 0; q < k; ++q) {
            const int32_t j = a.perm[b + q];
            if (j < 0 || j >= k || (seen >> j) & 1u) ok = false;
            else seen |= 1u << j;
        }
    }
    const int nl = n_legs(a, k);
    if (!ok) {
        if (a.mode == PATH_COUNT)
            for (int q = lane; q < nl; q += 32) a.leg_len[lb + q] = -2;
        return;
    }
    // write / copy: this order's leg offsets (a warp-wide prefix over at most 21 legs)
    int64_t start = 0;
    if (a.mode != PATH_COUNT) {
        if (a.node_offs[o + 1] == a.node_offs[o]) return;  // an unreachable leg: no nodes
        int32_t len = lane < nl ? a.leg_len[lb + lane] : 0;
        int32_t inc = len;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t y = __shfl_up_sync(FULL_MASK, inc, d);
            if (lane >= d) inc += y;
        }
        start = a.node_offs[o] + 1 + (inc - len);
        if (lane == 0 && a.mode == PATH_COPY) a.nodes[a.node_offs[o]] = a.open_path ? a.picks[b + a.perm[b]] : a.depot;
    }
    if (a.mode == PATH_COPY) {
        // the warp copies one cached leg at a time, lanes over its nodes (reversed: walk order is t first)
        for (int q = 0; q < nl; ++q) {
            const int64_t sq = __shfl_sync(FULL_MASK, start, q & 31);  // nl <= 21: lane q holds leg q
            const int32_t len = a.leg_len[lb + q];
            if (len > a.cache_cap) continue;
            const int32_t* cache = a.leg_cache + (lb + q) * static_cast<int64_t>(a.cache_cap);
            for (int i = lane; i < len; i += 32) a.nodes[sq + len - 1 - i] = cache[i];
        }
        return;
    }
    for (int q = lane; q < nl; q += 32) {
        int32_t* cache = a.leg_cache + (lb + q) * static_cast<int64_t>(a.cache_cap);
        int32_t s, t;
        leg_ends(a, b, k, q, s, t);
        const int32_t lane_s = a.src_index[s] - a.seg.first;
        if (lane_s < 0 || lane_s >= a.seg.lanes) continue;  // another segment holds s
        if (a.mode == PATH_WRITE) {
            const int32_t len = a.leg_len[lb + q];
            if (len > a.cache_cap) walk_leg(a, s, t, lane_s, cache, 0, a.nodes + start, len);
        } else {
            const int32_t len = walk_leg(a, s, t, lane_s, cache, a.cache_cap, nullptr, 0);
            a.leg_len[lb + q] = len;
            if (len > a.cache_cap) *a.seg_long = 1;
        }
    }
}

// node_offs: exclusive prefix of the orders' node counts (0 for an order with
// an invalid sequence or an unreachable leg); one block.
__global__ void paths_offsets_kernel(int32_t n, const int64_t* offs, int open_path, const int32_t* leg_len,
                                     int64_t* node_offs) {
    __shared__ long long ws[32];
    __shared__ long long tot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long carry = 0;
    for (int base = 0; base < n; base += blockDim.x) {
        const int o = base + threadIdx.x;
        long long x = 0;
        if (o < n) {
            const int k = static_cast<int>(offs[o + 1] - offs[o]);
            const int nl = open_path ? max(k - 1, 0) : k + 1;
            const int64_t lb = offs[o] + o;
            x = 1;
            for (int q = 0; q < nl; ++q) {
                const int32_t l = leg_len[lb + q];
                if (l < 0) {
                    x = 0;
                    break;
                }
                x += l;
            }
            if (k < 1) x = 0;
        }
        long long inc = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const long long y = __shfl_up_sync(FULL_MASK, inc, d);
            if (lane >= d) inc += y;
        }
        if (lane == 31) ws[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const long long w0 = lane < (blockDim.x >> 5) ? ws[lane] : 0;
            long long wi = w0;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const long long y = __shfl_up_sync(FULL_MASK, wi, d);
                if (lane >= d) wi += y;
            }
            if (lane < (blockDim.x >> 5)) ws[lane] = wi - w0;
            if (lane == 31) tot = wi;
        }
        __syncthreads();
        if (o < n) node_offs[o] = carry + ws[warp] + inc - x;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) node_offs[n] = carry;
}

cudaError_t paths_launch(const PathsLaunch& l, const BfSegment* seg, int mode, int32_t* seg_long, int32_t* nodes,
                         const int64_t* node_offs, cudaStream_t s) {
    PathArgs a{};
    a.n = l.n;
    a.offs = l.offs;
    a.picks = l.picks;
    a.perm = l.perm;
    a.order_status = l.order_status;
    a.open_path = l.open_path;
    a.depot = l.depot;
    a.src_index = l.src_index;
    if (seg) a.seg = *seg;
    a.in_ptr = l.in_ptr;
    a.in_src = l.in_src;
    a.in_w = l.in_w;
    a.in4 = l.in4;
    a.V = l.V;
    a.leg_len = l.leg_len;
    a.leg_cache = l.leg_cache;
    a.cache_cap = l.cache_cap;
    a.seg_long = seg_long;
    a.mode = mode;
    a.node_offs = node_offs;
    a.nodes = nodes;
    paths_kernel<<<(l.n + 7) / 8, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t paths_launch_offsets(const PathsLaunch& l, int64_t* node_offs, cudaStream_t s) {
    paths_offsets_kernel<<<1, 1024, 0, s>>>(l.n, l.offs, l.open_path, l.leg_len, node_offs);
    return cudaGetLastError();
}

}  // namespace wr
