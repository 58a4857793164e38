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
// One cooperative persistent kernel works through the orders one at a time:
// the table of an order (2^k x k words) is filled level by level (subsets of
// k picks, then k-1, ... 1), all blocks sharing each level, with a bounded
// grid barrier between levels; block 0 rebuilds the sequence.  Arithmetic is
// uint32 with WR_INF saturation; finite sums stay below 21 x WR_LEG_MAX < 2^31.
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
    uint32_t* h;  // 2^max_k x max_k words
    TourBufs t;
    int32_t* cost;
    int32_t* perm;
    int32_t* status;
    GridBar* bar;
    int* err;
    unsigned long long max_spins;
};

__global__ void __launch_bounds__(256) hk_solve_kernel(HkParams p) {
    __shared__ uint32_t D[HK_DBLOCK];
    const int n_big = ld_volatile(p.count);
    const long long gtid = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    const long long nthreads = static_cast<long long>(gridDim.x) * blockDim.x;
    for (int q = 0; q < n_big; ++q) {
        const int o = p.list[q];
        const int64_t b = p.t.offs[o];
        const int k = static_cast<int>(p.t.offs[o + 1] - b);
        if (p.t.order_flags[o] & ORDER_FLAG_RANGE) continue;  // decided by the decode of the other orders
        for (int e = threadIdx.x; e < HK_DBLOCK; e += blockDim.x) D[e] = p.D21[static_cast<int64_t>(q) * HK_DBLOCK + e];
        __syncthreads();
        const unsigned full = (1u << k) - 1u;
        for (int L = k; L >= 1; --L) {
            for (long long S = gtid; S <= full; S += nthreads) {
                const unsigned s = static_cast<unsigned>(S);
                if (__popc(s) != L) continue;
                uint32_t* hs = p.h + static_cast<int64_t>(s) * k;
                for (unsigned cm = s; cm; cm &= cm - 1) {
                    const int c = __ffs(cm) - 1;
                    uint32_t best;
                    if (s == full) {
                        best = D[(c + 1) * HK_DSTRIDE];
                    } else {
                        best = INF_U;
                        for (unsigned jm = full & ~s; jm; jm &= jm - 1) {
                            const int j = __ffs(jm) - 1;
                            best = min(best, sat_add(D[(c + 1) * HK_DSTRIDE + j + 1],
                                                     __ldcg(p.h + static_cast<int64_t>(s | (1u << j)) * k + j)));
                        }
                    }
                    __stcg(hs + c, best);
                }
            }
            if (!grid_sync(p.bar, p.err, p.max_spins)) return;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            uint32_t best = INF_U;
            for (int j = 0; j < k; ++j) best = min(best, sat_add(D[j + 1], __ldcg(p.h + static_cast<int64_t>(1u << j) * k + j)));
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
                        const uint32_t r = __ldcg(p.h + static_cast<int64_t>(s | (1u << j)) * k + j);
                        if (sat_add(D[cur * HK_DSTRIDE + j + 1], r) == rem) {
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
        // the table and the shared matrix are reused by the next order
        if (!grid_sync(p.bar, p.err, p.max_spins)) return;
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
                            const TourBufs& t, int32_t* cost, int32_t* perm, int32_t* status, GridBar* bar, int* err,
                            unsigned long long max_spins, int blocks, cudaStream_t s) {
    HkParams p{list, count, D21, h, t, cost, perm, status, bar, err, max_spins};
    void* args[] = {&p};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(hk_solve_kernel), dim3(blocks), dim3(256), args, 0,
                                       s);
}

}  // namespace wr
