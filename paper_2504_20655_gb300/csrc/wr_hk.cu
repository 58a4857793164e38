// Orders of 13..20 picks (beyond exhaustive enumeration): exact Held-Karp.
//
// The paper scores a route by the cost of a pick sequence (Sec. 2.4, Sec. 4.6)
// and uses the exact optimum as the reference its clustered routes are
// measured against (Sec. 3).  For k <= 12 the library enumerates all k!
// sequences; above that it computes the same optimum, with the same
// tie rule (the lexicographically first optimal sequence), by dynamic
// programming over pick subsets:
//   h(S, c) = D[c][depot]                                   if S = all picks
//   h(S, c) = min over j not in S of D[c][j] + h(S + j, j)  otherwise,
// for every subset S and pick c in S (c = last pick visited), then
//   cost = min over j of D[depot][j] + h({j}, j)
// and the sequence is rebuilt from the depot by taking, at every step, the
// smallest pick index j whose D[cur][j] + h(S + j, j) equals what remains.
//
// One cooperative persistent kernel fills the tables (2^k x k words per order)
// level by level (subsets of k picks, then k-1, ... 1) for a whole batch of
// orders at once, all blocks sharing each level, with one bounded grid
// barrier per level; then every order's sequence is rebuilt by one thread.
// Arithmetic is uint32 with WR_INF saturation; finite sums stay below
// 21 x WR_LEG_MAX < 2^31.
#include "wr_bf_common.cuh"

namespace wr {

// Orders to solve here: valid, k in (WR_MAX_K, max_k].  list gets their ids (any order).
__global__ void hk_select_kernel(int32_t n, TourBufs t, int32_t max_k, int32_t* list, int32_t* count) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const long long k = t.offs[o + 1] - t.offs[o];
    if (t.order_status[o] == WR_ORDER_OK && k > WR_MAX_K && k <= max_k) list[atomicAdd(count, 1)] = o;
}

// D of the listed orders, (k+1) x (k+1) at stride HK_DSTRIDE, from one source segment's rows.
__global__ void hk_gather_kernel(const int32_t* __restrict__ list, const int32_t* __restrict__ count, TourBufs t,
                                 int32_t depot, const int32_t* __restrict__ src_index, BfSegment seg, uint32_t* D21,
                                 int open_path) {
    const int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (q >= ld_volatile(count)) return;
    const int o = list[q];
    const int64_t b = t.offs[o];
    const int k = static_cast<int>(t.offs[o + 1] - b);
    const int m = k + 1;
    bool range = false;
    for (int e = lane; e < m * m; e += 32) {
        const int i = e / m, j = e - i * m;
        if (open_path && (i == 0 || j == 0)) {  // open path: free entrance/exit legs
            D21[static_cast<int64_t>(q) * HK_DBLOCK + i * HK_DSTRIDE + j] = 0u;
            continue;
        }
        const int32_t pi = i == 0 ? depot : t.picks[b + i - 1];
        const int32_t si = src_index[pi] - seg.first;
        if (si < 0 || si >= seg.lanes) continue;
        const int32_t pj = j == 0 ? depot : t.picks[b + j - 1];
        const uint32_t val = __ldcg(seg.rows + static_cast<int64_t>(pj) * seg.ld + si);
        if (val != INF_U && val > static_cast<uint32_t>(WR_LEG_MAX) && i != j) range = true;
        D21[static_cast<int64_t>(q) * HK_DBLOCK + i * HK_DSTRIDE + j] = val;
    }
    if (__any_sync(FULL_MASK, range) && lane == 0) atomicOr(t.order_flags + o, ORDER_FLAG_RANGE);
}

__device__ __forceinline__ uint32_t sat_add(uint32_t a, uint32_t b) { return min(a + b, INF_U); }

struct HkParams {
    const int32_t* list;
    const int32_t* count;
    const uint32_t* D21;
    uint32_t* h;                 // table buffer
    unsigned long long h_words;  // its capacity in words (at least one table of max_k picks)
    TourBufs t;
    int32_t* cost;
    int32_t* perm;
    int32_t* status;
    GridBar* bar;
    int* err;
    unsigned long long max_spins;
};

constexpr int HK_BATCH = 512;  // orders solved together, at most

// Picks of listed order q (0 for an order whose D holds an out-of-range leg:
// its status comes from the decode of the other orders).
__device__ __forceinline__ int hk_k(const HkParams& p, int q) {
    const int o = p.list[q];
    if (p.t.order_flags[o] & ORDER_FLAG_RANGE) return 0;
    return static_cast<int>(p.t.offs[o + 1] - p.t.offs[o]);
}

// Orders are solved in batches whose tables (2^k x k words each) fit the buffer;
// within a batch all orders share every level: level L holds, for every order of
// k >= L picks, its C(k, L) subsets S of size L, in increasing bitmask order per
// order, orders one after another.  Consecutive threads take consecutive items
// (grid-stride), each unranking its subset (combinatorial number system), and a
// table is pick-major, h[c][S], so the lanes of a warp read and write
// neighbouring words.  One grid barrier per level; then one thread per order
// rebuilds its first optimal sequence.
__global__ void __launch_bounds__(256) hk_solve_kernel(HkParams p) {
    __shared__ uint32_t binom[HK_MAX_K + 1][HK_MAX_K + 1];
    __shared__ unsigned long long pre[HK_BATCH + 1];  // level prefix of C(k_q, L)
    __shared__ unsigned long long base[HK_BATCH + 1];  // table offsets (words)
    __shared__ int kq[HK_BATCH];
    __shared__ int nb_s;
    for (int i = threadIdx.x; i < (HK_MAX_K + 1) * (HK_MAX_K + 1); i += blockDim.x) {
        const int n = i / (HK_MAX_K + 1), r = i % (HK_MAX_K + 1);
        unsigned long long c = 1;  // C(n, r) by the multiplicative formula (exact at each step)
        if (r > n) c = 0;
        for (int j = 1; j <= r && j <= n; ++j) c = c * static_cast<unsigned long long>(n - r + j) / j;
        binom[n][r] = static_cast<uint32_t>(c);
    }
    const int n_big = ld_volatile(p.count);
    const long long gtid = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    const long long nthreads = static_cast<long long>(gridDim.x) * blockDim.x;
    int q0 = 0;
    while (q0 < n_big) {
        // the batch: orders q0 .. q1-1 whose tables fit (the same in every block)
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long acc = 0;
            int q = q0;
            base[0] = 0;
            while (q < n_big && q - q0 < HK_BATCH) {
                const int k = hk_k(p, q);
                const unsigned long long sz = k > 0 ? (1ull << k) * static_cast<unsigned long long>(k) : 0ull;
                if (q > q0 && acc + sz > p.h_words) break;
                kq[q - q0] = k;
                acc += sz;
                base[q - q0 + 1] = acc;
                ++q;
            }
            nb_s = q - q0;  // batch size
        }
        __syncthreads();
        const int nb = nb_s;
        int kmax = 0;
        for (int i = 0; i < nb; ++i) kmax = max(kmax, kq[i]);
        for (int L = kmax; L >= 1; --L) {
            __syncthreads();
            if (threadIdx.x == 0) {
                pre[0] = 0;
                for (int i = 0; i < nb; ++i) pre[i + 1] = pre[i] + (kq[i] >= L ? binom[kq[i]][L] : 0u);
            }
            __syncthreads();
            const unsigned long long total = pre[nb];
            int qi = 0;
            for (unsigned long long w = static_cast<unsigned long long>(gtid); w < total;
                 w += static_cast<unsigned long long>(nthreads)) {
                while (pre[qi + 1] <= w) ++qi;  // the order holding item w
                const int k = kq[qi];
                // unrank: the subset of rank w - pre[qi] among the L-subsets of k picks
                unsigned s = 0;
                unsigned long long rr = w - pre[qi];
                for (int i = L; i >= 1; --i) {
                    int c = i - 1;
                    while (c + 1 < k && binom[c + 1][i] <= rr) ++c;
                    s |= 1u << c;
                    rr -= binom[c][i];
                }
                const unsigned full = (1u << k) - 1u;
                const int64_t side = static_cast<int64_t>(1) << k;  // words per pick in the table
                const uint32_t* D = p.D21 + static_cast<int64_t>(q0 + qi) * HK_DBLOCK;
                uint32_t* hq = p.h + base[qi];
                // h(S + j, j) for every pick j outside S, all loads in flight together
                uint32_t hv[HK_MAX_K];
#pragma unroll
                for (int j = 0; j < HK_MAX_K; ++j)
                    hv[j] = (j < k && !((s >> j) & 1u)) ? __ldcg(hq + j * side + (s | (1u << j))) : INF_U;
                for (unsigned cm = s; cm; cm &= cm - 1) {
                    const int c = __ffs(cm) - 1;
                    const uint32_t* Dr = D + (c + 1) * HK_DSTRIDE;
                    uint32_t best;
                    if (s == full) {
                        best = __ldg(Dr);
                    } else {
                        best = INF_U;
#pragma unroll
                        for (int j = 0; j < HK_MAX_K; ++j)
                            if (j < k && !((s >> j) & 1u)) best = min(best, sat_add(__ldg(Dr + j + 1), hv[j]));
                    }
                    __stcg(hq + c * side + s, best);
                }
            }
            if (!grid_sync(p.bar, p.err, p.max_spins)) return;
        }
        // rebuild: one thread per order, lexicographically first optimal sequence
        for (long long qi = gtid; qi < nb; qi += nthreads) {
            const int q = q0 + static_cast<int>(qi);
            const int k = kq[qi];
            if (k == 0) continue;
            const int o = p.list[q];
            const int64_t b = p.t.offs[o];
            const uint32_t* D = p.D21 + static_cast<int64_t>(q) * HK_DBLOCK;
            const uint32_t* hq = p.h + base[qi];
            const int64_t side = static_cast<int64_t>(1) << k;
            uint32_t best = INF_U;
            for (int j = 0; j < k; ++j) best = min(best, sat_add(__ldg(D + j + 1), __ldcg(hq + j * side + (1u << j))));
            int32_t* pp = p.perm + b;
            if (best >= INF_U) {
                p.cost[o] = WR_INF;
                p.status[o] = WR_ORDER_UNREACHABLE;
                for (int i = 0; i < k; ++i) pp[i] = i;
            } else {
                p.cost[o] = static_cast<int32_t>(best);
                p.status[o] = WR_ORDER_OK;
                unsigned s = 0;
                int cur = 0;  // matrix index of the current stop (0 = depot)
                uint32_t rem = best;
                for (int pos = 0; pos < k; ++pos) {
                    for (int j = 0; j < k; ++j) {
                        if (s & (1u << j)) continue;
                        const uint32_t r = __ldcg(hq + j * side + (s | (1u << j)));
                        if (sat_add(__ldg(D + cur * HK_DSTRIDE + j + 1), r) == rem) {
                            pp[pos] = j;
                            s |= 1u << j;
                            rem = r;
                            cur = j + 1;
                            break;
                        }
                    }
                }
            }
        }
        // the table buffer is reused by the next batch
        if (!grid_sync(p.bar, p.err, p.max_spins)) return;
        q0 += nb;
    }
}

cudaError_t hk_launch_select(int32_t n, const TourBufs& t, int32_t max_k, int32_t* list, int32_t* count,
                             cudaStream_t s) {
    hk_select_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, t, max_k, list, count);
    return cudaGetLastError();
}

cudaError_t hk_launch_gather(int32_t n, const int32_t* list, const int32_t* count, const TourBufs& t, int32_t depot,
                             const int32_t* src_index, const BfSegment& seg, uint32_t* D21, int open_path,
                             cudaStream_t s) {
    hk_gather_kernel<<<(n + 7) / 8, 256, 0, s>>>(list, count, t, depot, src_index, seg, D21, open_path);
    return cudaGetLastError();
}

int hk_blocks(int device) {
    int occ = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hk_solve_kernel, 256, 0) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    return occ * sms;
}

cudaError_t hk_launch_solve(const int32_t* list, const int32_t* count, const uint32_t* D21, uint32_t* h,
                            unsigned long long h_words, const TourBufs& t, int32_t* cost, int32_t* perm,
                            int32_t* status, GridBar* bar, int* err, unsigned long long max_spins, int blocks,
                            cudaStream_t s) {
    HkParams p{list, count, D21, h, h_words, t, cost, perm, status, bar, err, max_spins};
    void* args[] = {&p};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(hk_solve_kernel), dim3(blocks), dim3(256), args, 0,
                                       s);
}

}  // namespace wr
