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
#include "wr_bf_common.cuh"

namespace wr {

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
    int32_t V;
    int32_t* leg_len;             // offs[o] + o + q: nodes of leg q after its first; -1 unreachable, -2 invalid
    const int64_t* node_offs;     // write pass: where each order's nodes start
    int32_t* nodes;               // write pass: output (nullptr in the count pass)
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

// Walk one leg backward from t; writes the nodes after s (forward order) into
// out[0 .. len) when out != nullptr.  Returns len, or -1 if t is unreachable.
__device__ int walk_leg(const PathArgs& a, int32_t s, int32_t t, int32_t lane_s, int32_t* out, int32_t len_known) {
    const uint32_t* rows = a.seg.rows;
    const int64_t ld = a.seg.ld;
    uint32_t dv = __ldcg(rows + static_cast<int64_t>(t) * ld + lane_s);
    if (dv == INF_U) return -1;
    int32_t v = t, len = 0;
    while (v != s && len < a.V) {
        if (out) out[len_known - 1 - len] = v;
        ++len;
        int32_t best_u = -1;
        uint32_t best_d = 0;
        for (int64_t e = a.in_ptr[v]; e < a.in_ptr[v + 1]; ++e) {
            const int32_t u = a.in_src[e];
            const uint32_t du = __ldcg(rows + static_cast<int64_t>(u) * ld + lane_s);
            if (du != INF_U && static_cast<uint64_t>(du) + static_cast<uint32_t>(a.in_w[e]) == dv &&
                (best_u < 0 || u < best_u)) {
                best_u = u;
                best_d = du;
            }
        }
        if (best_u < 0) return -3;  // inconsistent rows (cannot happen at the fixpoint)
        v = best_u;
        dv = best_d;
    }
    return v == s ? len : -3;
}

// One warp per order, one lane per leg: legs whose source lies in this segment.
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
        if (!a.nodes)
            for (int q = lane; q < nl; q += 32) a.leg_len[lb + q] = -2;
        return;
    }
    // write pass: this order's leg offsets (a warp-wide prefix over at most 21 legs)
    int64_t start = 0;
    if (a.nodes) {
        if (a.node_offs[o + 1] == a.node_offs[o]) return;  // an unreachable leg: no nodes
        int32_t len = lane < nl ? a.leg_len[lb + lane] : 0;
        int32_t inc = len;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t y = __shfl_up_sync(FULL_MASK, inc, d);
            if (lane >= d) inc += y;
        }
        start = a.node_offs[o] + 1 + (inc - len);
        if (lane == 0) {
            int32_t first;
            if (a.open_path) first = a.picks[b + a.perm[b]];
            else first = a.depot;
            a.nodes[a.node_offs[o]] = first;
        }
    }
    for (int q = lane; q < nl; q += 32) {
        int32_t s, t;
        leg_ends(a, b, k, q, s, t);
        const int32_t lane_s = a.src_index[s] - a.seg.first;
        if (lane_s < 0 || lane_s >= a.seg.lanes) continue;  // another segment holds s
        if (a.nodes) walk_leg(a, s, t, lane_s, a.nodes + start, a.leg_len[lb + q]);
        else a.leg_len[lb + q] = walk_leg(a, s, t, lane_s, nullptr, 0);
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

cudaError_t paths_launch(const PathsLaunch& l, const BfSegment& seg, int32_t* nodes, const int64_t* node_offs,
                         cudaStream_t s) {
    PathArgs a;
    a.n = l.n;
    a.offs = l.offs;
    a.picks = l.picks;
    a.perm = l.perm;
    a.order_status = l.order_status;
    a.open_path = l.open_path;
    a.depot = l.depot;
    a.src_index = l.src_index;
    a.seg = seg;
    a.in_ptr = l.in_ptr;
    a.in_src = l.in_src;
    a.in_w = l.in_w;
    a.V = l.V;
    a.leg_len = l.leg_len;
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
