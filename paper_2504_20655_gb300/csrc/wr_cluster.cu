// Cluster-patched approximate routing (Sec. 3): the paper's own way to route
// large orders.  The stops of an order are grouped into at most m clusters
// by k-means on their plan coordinates, an optimal open route is found inside
// every cluster, and the cluster routes are patched into one global route by
// trying every order of the clusters and every travel direction of each
// (m! x 2^m candidates; Sec. 3 counts the m! x 2^(m-1) undirected ones).
//
// The steps and their tie rules, in the paper's order:
//   k-means   centres start at stop 0 and then, one by one, at the stop
//             farthest (squared Euclidean) from the centres so far (ties to
//             the lowest stop index), up to m; Lloyd steps assign each stop to
//             its nearest centre (ties to the lowest centre) and move every
//             non-empty centre to the mean of its stops until no assignment
//             changes (at most 64 steps).  Distances to a mean (Sx/c, Sy/c)
//             are compared exactly in integers: (c x - Sx)^2 + (c y - Sy)^2
//             over c^2, by cross multiplication.
//   cluster   the lexicographically first optimal open route over the
//             cluster's stops (legs between its stops only), at most 10 stops.
//   patching  the cheapest global route (depot legs included for closed
//             tours, free for open paths), ties to the lexicographically
//             first stop sequence.
//
// Three stages on the device:
//   split     one thread per order: k-means, then one sub-order per cluster,
//             its stops in increasing index and a D block whose depot legs
//             are zero, so that a tour of the sub-order costs exactly the open
//             route through the cluster;
//   routes    the sub-orders go through the exhaustive enumeration (units,
//             enum, finish): the first optimal sequence of each is the
//             cluster's route;
//   patch     one warp per order: the m! x 2^m candidates spread over the
//             lanes, each lane's best kept by (cost, stop sequence), then a
//             warp reduction in the same order.
#include "wr_bf_common.cuh"

namespace wr {

constexpr unsigned long long CL_BIG = 1ull << 62;

__device__ __forceinline__ unsigned long long cl_leg(const uint32_t* Dm, int a, int b) {
    const uint32_t v = Dm[a * DSTRIDE + b];
    return v >= TOUR_CAP ? CL_BIG : v;  // the gather stores unreachable legs as TOUR_CAP
}

// Sub-order slot c of order o holds cluster c: member pick indices (4 bits
// each, increasing, first in the low bits) and the member count in bits 60..63.
__device__ __forceinline__ int cl_size(unsigned long long mem) { return static_cast<int>(mem >> 60); }
__device__ __forceinline__ int cl_member(unsigned long long mem, int i) { return static_cast<int>((mem >> (4 * i)) & 15u); }

__global__ void cluster_split_kernel(int32_t n, TourBufs t, const int32_t* __restrict__ xy_all, int32_t m,
                                     ClusterBufs cb) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const int64_t b = t.offs[o];
    const int k = static_cast<int>(t.offs[o + 1] - b);
    const int64_t s0 = static_cast<int64_t>(o) * m;
    for (int c = 0; c < m; ++c) {
        cb.sub_k[s0 + c] = 0;
        cb.sub_status[s0 + c] = WR_ORDER_BAD;  // empty slot: no units
        cb.sub_flags[s0 + c] = 0;
        cb.members[s0 + c] = 0ull;
    }
    int st = t.order_status[o];
    if (st == WR_ORDER_OK && (t.order_flags[o] & ORDER_FLAG_RANGE)) st = WR_ORDER_RANGE;
    if (st == WR_ORDER_OK && k > WR_MAX_K) st = WR_ORDER_BAD;
    if (st != WR_ORDER_OK) {
        cb.order_state[o] = st;
        return;
    }
    long long x[WR_MAX_K], y[WR_MAX_K];
    for (int i = 0; i < k; ++i) {
        const int32_t node = t.picks[b + i];
        x[i] = xy_all[2 * static_cast<int64_t>(node)];
        y[i] = xy_all[2 * static_cast<int64_t>(node) + 1];
    }
    // k-means: farthest-first centres, then Lloyd steps
    long long Sx[CL_MAX_M], Sy[CL_MAX_M], cnt[CL_MAX_M];
    int nc = 1;
    Sx[0] = x[0];
    Sy[0] = y[0];
    cnt[0] = 1;
    while (nc < m && nc < k) {
        int best_i = -1;
        long long best_d = -1;
        for (int i = 0; i < k; ++i) {
            long long dmin = -1;
            for (int c = 0; c < nc; ++c) {
                const long long dx = x[i] - Sx[c], dy = y[i] - Sy[c];
                const long long d = dx * dx + dy * dy;
                if (dmin < 0 || d < dmin) dmin = d;
            }
            if (dmin > best_d) {
                best_d = dmin;
                best_i = i;
            }
        }
        if (best_d <= 0) break;
        Sx[nc] = x[best_i];
        Sy[nc] = y[best_i];
        cnt[nc] = 1;
        ++nc;
    }
    int assign[WR_MAX_K];
    for (int i = 0; i < k; ++i) assign[i] = -1;
    for (int it = 0; it < 64; ++it) {
        bool changed = false;
        for (int i = 0; i < k; ++i) {
            int bc = 0;
            long long bnum = 0, bden = 1;
            for (int c = 0; c < nc; ++c) {
                const long long dx = cnt[c] * x[i] - Sx[c], dy = cnt[c] * y[i] - Sy[c];
                const long long num = dx * dx + dy * dy, den = cnt[c] * cnt[c];
                if (c == 0 || num * bden < bnum * den) {
                    bc = c;
                    bnum = num;
                    bden = den;
                }
            }
            if (assign[i] != bc) {
                assign[i] = bc;
                changed = true;
            }
        }
        if (!changed) break;
        for (int c = 0; c < nc; ++c) {
            long long sx = 0, sy = 0, ct = 0;
            for (int i = 0; i < k; ++i)
                if (assign[i] == c) {
                    sx += x[i];
                    sy += y[i];
                    ++ct;
                }
            if (ct > 0) {
                Sx[c] = sx;
                Sy[c] = sy;
                cnt[c] = ct;
            }
        }
    }
    // clusters in centre order, stops in increasing index: one sub-order each
    const uint32_t* Dm = t.D + static_cast<int64_t>(o) * DBLOCK;
    int M = 0;
    for (int c = 0; c < nc; ++c) {
        unsigned long long mem = 0;
        int sz = 0;
        for (int i = 0; i < k; ++i)
            if (assign[i] == c) {
                if (sz == CL_MAX) {
                    cb.order_state[o] = WR_ORDER_BAD;
                    for (int q = 0; q < m; ++q) {
                        cb.sub_k[s0 + q] = 0;
                        cb.sub_status[s0 + q] = WR_ORDER_BAD;
                    }
                    return;
                }
                mem |= static_cast<unsigned long long>(i) << (4 * sz);
                ++sz;
            }
        if (sz == 0) continue;
        const int64_t q = s0 + M;
        uint32_t* Dq = cb.sub_D + q * DBLOCK;
        for (int i = 0; i <= sz; ++i)
            for (int j = 0; j <= sz; ++j) {
                uint32_t v = 0u;  // the sub-order's depot: free entry and exit
                if (i > 0 && j > 0) {
                    const int a = static_cast<int>((mem >> (4 * (i - 1))) & 15u) + 1;
                    const int e = static_cast<int>((mem >> (4 * (j - 1))) & 15u) + 1;
                    v = Dm[a * DSTRIDE + e];
                }
                Dq[i * DSTRIDE + j] = v;
            }
        cb.members[q] = mem | (static_cast<unsigned long long>(sz) << 60);
        cb.sub_k[q] = sz;
        cb.sub_status[q] = WR_ORDER_OK;
        ++M;
    }
    cb.order_state[o] = WR_ORDER_OK;
    cb.n_clusters[o] = M;
}

// Candidate key for ties: the stop sequence, first stop in the highest nibble.
struct PatchBest {
    unsigned long long cost, key;
};

__device__ __forceinline__ bool patch_less(unsigned long long c1, unsigned long long k1, unsigned long long c2,
                                           unsigned long long k2) {
    return c1 < c2 || (c1 == c2 && k1 < k2);
}

__global__ void cluster_patch_kernel(int32_t n, TourBufs t, int32_t m, int open_path, ClusterBufs cb, int32_t* cost,
                                     int32_t* perm, int32_t* status) {
    const int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (o >= n) return;
    const int64_t b = t.offs[o];
    const int k = static_cast<int>(t.offs[o + 1] - b);
    int32_t* pp = perm + b;
    const int st = cb.order_state[o];
    auto fail = [&](int s) {
        if (lane != 0) return;
        status[o] = s;
        cost[o] = WR_INF;
        for (int i = 0; i < k && b >= 0 && t.offs[o + 1] <= t.offs[n]; ++i) pp[i] = i;
    };
    if (st != WR_ORDER_OK) {
        fail(st);
        return;
    }
    const uint32_t* Dm = t.D + static_cast<int64_t>(o) * DBLOCK;
    const int M = cb.n_clusters[o];
    const int64_t s0 = static_cast<int64_t>(o) * m;
    // each cluster's route (pick indices), its cost forward and backward
    int route[CL_MAX_M][CL_MAX], size[CL_MAX_M];
    unsigned long long fwd[CL_MAX_M], rev[CL_MAX_M];
#pragma unroll 1
    for (int c = 0; c < M; ++c) {
        const unsigned long long mem = cb.members[s0 + c];
        const int sz = cl_size(mem);
        size[c] = sz;
        const int32_t* sp = cb.sub_perm + (s0 + c) * WR_MAX_K;
        for (int i = 0; i < sz; ++i) route[c][i] = cl_member(mem, sp[i]);
        unsigned long long f = 0, r = 0;
        for (int i = 0; i + 1 < sz; ++i) {
            const unsigned long long lf = cl_leg(Dm, route[c][i] + 1, route[c][i + 1] + 1);
            const unsigned long long lr = cl_leg(Dm, route[c][i + 1] + 1, route[c][i] + 1);
            f = (f >= CL_BIG || lf >= CL_BIG) ? CL_BIG : f + lf;
            r = (r >= CL_BIG || lr >= CL_BIG) ? CL_BIG : r + lr;
        }
        fwd[c] = f;
        rev[c] = r;
    }
    // candidates: cluster order (Lehmer code of idx >> M) x travel directions (idx & mask)
    int fact = 1;
    for (int i = 2; i <= M; ++i) fact *= i;
    const int n_cand = fact << M;
    unsigned long long best_c = CL_BIG, best_k = ~0ull;
#pragma unroll 1
    for (int idx = lane; idx < n_cand; idx += 32) {
        int code = idx >> M;
        const unsigned dir = static_cast<unsigned>(idx) & ((1u << M) - 1u);
        unsigned avail = (1u << M) - 1u;
        int f = fact;
        unsigned long long tt = 0, key = 0;
        int prev = -1;  // last stop so far (pick index); -1 = depot
        bool ok = true;
        for (int q = 0; q < M; ++q) {
            f /= (M - q);
            const int dgt = code / f;
            code -= dgt * f;
            unsigned mm = avail;
            for (int s = 0; s < dgt; ++s) mm &= mm - 1;
            const int c = __ffs(mm) - 1;
            avail &= ~(1u << c);
            const bool r = (dir >> q) & 1u;
            const int head = r ? route[c][size[c] - 1] : route[c][0];
            const unsigned long long link =
                prev < 0 ? (open_path ? 0ull : cl_leg(Dm, 0, head + 1)) : cl_leg(Dm, prev + 1, head + 1);
            const unsigned long long inner = r ? rev[c] : fwd[c];
            if (link >= CL_BIG || inner >= CL_BIG) {
                ok = false;
                break;
            }
            tt += link + inner;
            for (int i = 0; i < size[c]; ++i) {
                const int stop = r ? route[c][size[c] - 1 - i] : route[c][i];
                key = (key << 4) | static_cast<unsigned long long>(stop);
            }
            prev = r ? route[c][0] : route[c][size[c] - 1];
        }
        if (ok && !open_path) {
            const unsigned long long back = cl_leg(Dm, prev + 1, 0);
            if (back >= CL_BIG) ok = false;
            else tt += back;
        }
        if (ok && patch_less(tt, key, best_c, best_k)) {
            best_c = tt;
            best_k = key;
        }
    }
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        const unsigned long long oc = __shfl_xor_sync(FULL_MASK, best_c, d);
        const unsigned long long ok2 = __shfl_xor_sync(FULL_MASK, best_k, d);
        if (patch_less(oc, ok2, best_c, best_k)) {
            best_c = oc;
            best_k = ok2;
        }
    }
    if (best_c >= CL_BIG) {
        fail(WR_ORDER_UNREACHABLE);
        return;
    }
    if (lane == 0) {
        status[o] = WR_ORDER_OK;
        cost[o] = static_cast<int32_t>(best_c);
        for (int i = 0; i < k; ++i) pp[i] = static_cast<int32_t>((best_k >> (4 * (k - 1 - i))) & 15u);
    }
}

cudaError_t cluster_launch_split(int32_t n, const TourBufs& t, const int32_t* xy, int32_t m, const ClusterBufs& cb,
                                 cudaStream_t s) {
    cluster_split_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, t, xy, m, cb);
    return cudaGetLastError();
}

cudaError_t cluster_launch_patch(int32_t n, const TourBufs& t, int32_t m, int open_path, const ClusterBufs& cb,
                                 int32_t* cost, int32_t* perm, int32_t* status, cudaStream_t s) {
    cluster_patch_kernel<<<(n + 7) / 8, 256, 0, s>>>(n, t, m, open_path, cb, cost, perm, status);
    return cudaGetLastError();
}

}  // namespace wr
