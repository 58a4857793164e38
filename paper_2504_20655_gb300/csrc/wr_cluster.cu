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
// One thread per order; D is the order's gathered 13 x 13 block.
#include "wr_bf_common.cuh"

namespace wr {

constexpr int CL_MAX = 10;
constexpr int CL_MAX_M = 6;
constexpr unsigned long long CL_BIG = 1ull << 62;

__device__ __forceinline__ unsigned long long cl_leg(const uint32_t* Dm, int a, int b) {
    const uint32_t v = Dm[a * DSTRIDE + b];
    return v >= TOUR_CAP ? CL_BIG : v;  // the gather stores unreachable legs as TOUR_CAP
}

__device__ bool cl_next_perm(int* p, int n) {
    int i = n - 2;
    while (i >= 0 && p[i] >= p[i + 1]) --i;
    if (i < 0) return false;
    int j = n - 1;
    while (p[j] <= p[i]) --j;
    const int tmp = p[i];
    p[i] = p[j];
    p[j] = tmp;
    for (int a = i + 1, b = n - 1; a < b; ++a, --b) {
        const int x = p[a];
        p[a] = p[b];
        p[b] = x;
    }
    return true;
}

__global__ void cluster_kernel(int32_t n, TourBufs t, const int32_t* __restrict__ xy_all, int32_t m, int open_path,
                               int32_t* cost, int32_t* perm, int32_t* status) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const int64_t b = t.offs[o];
    const int k = static_cast<int>(t.offs[o + 1] - b);
    int32_t* pp = perm + b;
    int st = t.order_status[o];
    if (st == WR_ORDER_OK && (t.order_flags[o] & ORDER_FLAG_RANGE)) st = WR_ORDER_RANGE;
    if (st == WR_ORDER_OK && k > WR_MAX_K) st = WR_ORDER_BAD;
    auto fail = [&](int s) {
        status[o] = s;
        cost[o] = WR_INF;
        for (int i = 0; i < k && b >= 0 && t.offs[o + 1] <= t.offs[n]; ++i) pp[i] = i;
    };
    if (st != WR_ORDER_OK) {
        fail(st);
        return;
    }
    const uint32_t* Dm = t.D + static_cast<int64_t>(o) * DBLOCK;
    long long x[WR_MAX_K], y[WR_MAX_K];
    for (int i = 0; i < k; ++i) {
        const int32_t node = t.picks[b + i];
        x[i] = xy_all[2 * static_cast<int64_t>(node)];
        y[i] = xy_all[2 * static_cast<int64_t>(node) + 1];
    }
    // k-means
    long long Sx[WR_MAX_K], Sy[WR_MAX_K], cnt[WR_MAX_K];
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
    // clusters in centre order, stops in increasing index
    int members[CL_MAX_M][CL_MAX], size[CL_MAX_M], M = 0;
    for (int c = 0; c < nc; ++c) {
        int sz = 0;
        for (int i = 0; i < k; ++i)
            if (assign[i] == c) {
                if (sz == CL_MAX) {
                    fail(WR_ORDER_BAD);
                    return;
                }
                members[M][sz++] = i;
            }
        if (sz > 0) size[M++] = sz;
    }
    // the first optimal open route inside every cluster, and the cost of its reverse
    int route[CL_MAX_M][CL_MAX];
    unsigned long long fwd[CL_MAX_M], rev[CL_MAX_M];
    for (int c = 0; c < M; ++c) {
        const int sz = size[c];
        int p[CL_MAX], best_p[CL_MAX];
        for (int i = 0; i < sz; ++i) p[i] = best_p[i] = i;
        unsigned long long best = CL_BIG + 1;
        do {
            unsigned long long tt = 0;
            for (int i = 0; i + 1 < sz && tt < CL_BIG; ++i) {
                const unsigned long long l = cl_leg(Dm, members[c][p[i]] + 1, members[c][p[i + 1]] + 1);
                tt = l >= CL_BIG ? CL_BIG : tt + l;
            }
            if (tt < best) {
                best = tt;
                for (int i = 0; i < sz; ++i) best_p[i] = p[i];
            }
        } while (cl_next_perm(p, sz));
        for (int i = 0; i < sz; ++i) route[c][i] = members[c][best_p[i]];
        fwd[c] = best;
        unsigned long long r = 0;
        for (int i = sz - 1; i > 0 && r < CL_BIG; --i) {
            const unsigned long long l = cl_leg(Dm, route[c][i] + 1, route[c][i - 1] + 1);
            r = l >= CL_BIG ? CL_BIG : r + l;
        }
        rev[c] = r;
    }
    // patching
    int order[CL_MAX_M], seq[WR_MAX_K], best_seq[WR_MAX_K];
    for (int c = 0; c < M; ++c) order[c] = c;
    unsigned long long best = CL_BIG;
    bool have = false;
    do {
        for (unsigned dir = 0; dir < (1u << M); ++dir) {
            int len = 0;
            unsigned long long tt = 0;
            for (int q = 0; q < M; ++q) {
                const int c = order[q];
                const bool r = (dir >> q) & 1u;
                const int head = r ? route[c][size[c] - 1] : route[c][0];
                const unsigned long long inner = r ? rev[c] : fwd[c];
                const unsigned long long link =
                    q == 0 ? (open_path ? 0ull : cl_leg(Dm, 0, head + 1)) : cl_leg(Dm, seq[len - 1] + 1, head + 1);
                if (inner >= CL_BIG || link >= CL_BIG) {
                    tt = CL_BIG;
                    break;
                }
                tt += link + inner;
                for (int i = 0; i < size[c]; ++i) seq[len++] = r ? route[c][size[c] - 1 - i] : route[c][i];
            }
            if (tt < CL_BIG && !open_path) {
                const unsigned long long back = cl_leg(Dm, seq[k - 1] + 1, 0);
                tt = back >= CL_BIG ? CL_BIG : tt + back;
            }
            if (tt >= CL_BIG) continue;
            bool better = !have || tt < best;
            if (!better && tt == best) {
                for (int i = 0; i < k; ++i)
                    if (seq[i] != best_seq[i]) {
                        better = seq[i] < best_seq[i];
                        break;
                    }
            }
            if (better) {
                best = tt;
                have = true;
                for (int i = 0; i < k; ++i) best_seq[i] = seq[i];
            }
        }
    } while (cl_next_perm(order, M));
    if (!have) {
        fail(WR_ORDER_UNREACHABLE);
        return;
    }
    status[o] = WR_ORDER_OK;
    cost[o] = static_cast<int32_t>(best);
    for (int i = 0; i < k; ++i) pp[i] = best_seq[i];
}

cudaError_t cluster_launch(int32_t n, const TourBufs& t, const int32_t* xy, int32_t m, int open_path, int32_t* cost,
                           int32_t* perm, int32_t* status, cudaStream_t s) {
    cluster_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, t, xy, m, open_path, cost, perm, status);
    return cudaGetLastError();
}

}  // namespace wr
