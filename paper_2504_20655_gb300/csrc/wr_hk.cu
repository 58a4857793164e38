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
// One cooperative persistent kernel fills the tables (k x 2^(k-1) words per
// order) level by level (subsets of k picks, then k-1, ... 1) for a whole batch
// of orders at once, all blocks sharing each level, with one bounded grid
// barrier per level; then every order's sequence is rebuilt by one thread.
//
// Table layout: plane c (one per pick, 2^(k-1) words) holds h(S, c) for the
// subsets S that contain c, indexed by T = S - c with c's bit squeezed out (a
// subset of the other k-1 picks): first by |T| (blocks of C(k-1, l) words),
// then by the colex rank of T.  Colex order of equal-size subsets is their
// numeric order, and squeezing out a bit every subset lacks keeps that order,
// so the threads that take consecutive subsets S of a level read consecutive
// words of each plane j (h(S + j, j)) and write consecutive words of each
// plane c (h(S, c)).  A thread gets both ranks from running prefix sums of
// binomial terms over the bits of S.
// Arithmetic is uint32 on values of at most WR_INF = 2^31 - 1 (unreachable):
// a sum of two does not wrap, and a minimum started at WR_INF stays at most
// WR_INF, so a transition is one fused add-min; finite sums stay below
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

// D of the listed orders, (k+1) x (k+1) at stride HK_DSTRIDE (column j at HK_DOFF + j), from one
// source segment's rows.
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
            D21[static_cast<int64_t>(q) * HK_DBLOCK + i * HK_DSTRIDE + HK_DOFF + j] = 0u;
            continue;
        }
        const int32_t pi = i == 0 ? depot : t.picks[b + i - 1];
        const int32_t si = src_index[pi] - seg.first;
        if (si < 0 || si >= seg.lanes) continue;
        const int32_t pj = j == 0 ? depot : t.picks[b + j - 1];
        const uint32_t val = __ldcg(seg.rows + static_cast<int64_t>(pj) * seg.ld + si);
        if (val != INF_U && val > static_cast<uint32_t>(WR_LEG_MAX) && i != j) range = true;
        D21[static_cast<int64_t>(q) * HK_DBLOCK + i * HK_DSTRIDE + HK_DOFF + j] = val;
    }
    if (__any_sync(FULL_MASK, range) && lane == 0) atomicOr(t.order_flags + o, ORDER_FLAG_RANGE);
    // the rest of the block is unreachable: the solve's transitions then run over every
    // pick slot with no test (a leg of WR_INF plus any table value never wins a minimum)
    for (int e = lane; e < HK_DBLOCK; e += 32) {
        const int i = e / HK_DSTRIDE, j = e - i * HK_DSTRIDE - HK_DOFF;
        if (i >= m || j < 0 || j >= m) D21[static_cast<int64_t>(q) * HK_DBLOCK + e] = INF_U;
    }
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

// One subset S of a level: its order (index in the batch), S, and h(S + j, j) for the picks j outside S.
struct HkItem {
    int qi;
    unsigned s;
    uint32_t pc_tot;
    uint32_t hv[HK_MAX_K];
};

// Picks of listed order q (0 for an order whose D holds an out-of-range leg:
// its status comes from the decode of the other orders).
__device__ __forceinline__ int hk_k(const HkParams& p, int q) {
    const int o = p.list[q];
    if (p.t.order_flags[o] & ORDER_FLAG_RANGE) return 0;
    return static_cast<int>(p.t.offs[o + 1] - p.t.offs[o]);
}

// Orders are solved in batches whose tables (k x 2^(k-1) words each) fit the
// buffer; within a batch all orders share every level: level L holds, for every
// order of k >= L picks, its C(k, L) subsets S of size L, in increasing bitmask
// order per order, orders one after another.  Consecutive threads take
// consecutive items (grid-stride; in a level with four or more items per thread,
// consecutive pairs), unranking a subset in the combinatorial number system or
// stepping to the next one in colex order.  One grid barrier per level; then
// one warp per order rebuilds its first optimal sequence.
__global__ void __launch_bounds__(256) hk_solve_kernel(HkParams p) {
    __shared__ uint32_t binom[HK_MAX_K + 1][HK_MAX_K + 1];
    __shared__ uint32_t binx[HK_MAX_K + 2][HK_MAX_K + 2];  // binx[n + 1][r] = C(n, r); C(-1, r) = 0
    __shared__ uint32_t loff[HK_MAX_K + 1][HK_MAX_K + 2];  // loff[k][l]: sum of C(k-1, l') over l' < l
    __shared__ unsigned long long pre[HK_BATCH + 1];  // level prefix of C(k_q, L)
    __shared__ unsigned long long base[HK_BATCH + 1];  // table offsets (words)
    __shared__ int kq[HK_BATCH];
    __shared__ int nb_s, kmax_s;
    for (int i = threadIdx.x; i < (HK_MAX_K + 1) * (HK_MAX_K + 1); i += blockDim.x) {
        const int n = i / (HK_MAX_K + 1), r = i % (HK_MAX_K + 1);
        // C(n, r) by the multiplicative formula: exact at each step, C(n - r + j, j) * (n - r + j + 1)
        // stays below C(20, 10) * 21 < 2^32
        uint32_t c = 1;
        if (r > n) c = 0;
        for (int j = 1; j <= r && j <= n; ++j) c = c * static_cast<uint32_t>(n - r + j) / static_cast<uint32_t>(j);
        binom[n][r] = c;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < (HK_MAX_K + 2) * (HK_MAX_K + 2); i += blockDim.x) {
        const int n = i / (HK_MAX_K + 2) - 1, r = i % (HK_MAX_K + 2);
        binx[n + 1][r] = (n < 0 || r > HK_MAX_K) ? 0u : binom[n][r];
    }
    for (int k = threadIdx.x; k <= HK_MAX_K; k += blockDim.x) {
        loff[k][0] = 0;
        for (int l = 0; l <= HK_MAX_K; ++l) loff[k][l + 1] = loff[k][l] + (k >= 1 ? binom[k - 1][l] : 0u);
    }
    const int n_big = ld_volatile(p.count);
    const long long gtid = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    const long long nthreads = static_cast<long long>(gridDim.x) * blockDim.x;
    int q0 = 0;
    while (q0 < n_big) {
        // the batch: orders q0 .. q1-1 whose tables fit (the same in every block); every thread
        // reads the picks of its share of the candidates, then one thread sums the sizes
        __syncthreads();
        for (int i = threadIdx.x; i < HK_BATCH && q0 + i < n_big; i += blockDim.x) kq[i] = hk_k(p, q0 + i);
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long acc = 0;
            int q = q0, km = 0;
            base[0] = 0;
            while (q < n_big && q - q0 < HK_BATCH) {
                const int k = kq[q - q0];
                const unsigned long long sz = k > 0 ? (1ull << (k - 1)) * static_cast<unsigned long long>(k) : 0ull;
                if (q > q0 && acc + sz > p.h_words) break;
                acc += sz;
                base[q - q0 + 1] = acc;
                km = max(km, k);
                ++q;
            }
            nb_s = q - q0;  // batch size
            kmax_s = km;
        }
        __syncthreads();
        const int nb = nb_s;
        const int kmax = kmax_s;
        for (int L = kmax; L >= 1; --L) {
            __syncthreads();
            if (threadIdx.x < 32) {
                // pre[i] = items of the batch's orders before i at this level: a warp scan, lane l
                // over orders [l * per, (l + 1) * per)
                const int lane = threadIdx.x;
                const int per = (nb + 31) / 32;
                const int i0 = min(lane * per, nb), i1 = min(i0 + per, nb);
                unsigned long long sum = 0;
                for (int i = i0; i < i1; ++i) sum += kq[i] >= L ? binom[kq[i]][L] : 0u;
                unsigned long long inc = sum;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const unsigned long long y = __shfl_up_sync(FULL_MASK, inc, d);
                    if (lane >= d) inc += y;
                }
                unsigned long long run = inc - sum;
                for (int i = i0; i < i1; ++i) {
                    pre[i] = run;
                    run += kq[i] >= L ? binom[kq[i]][L] : 0u;
                }
                if (lane == 31) pre[nb] = inc;
            }
            __syncthreads();
            const unsigned long long total = pre[nb];
            int qi = 0;
            // unrank item w, then issue the loads h(S + j, j) for every pick j outside S (plane j,
            // block |S|, rank of S with bit j squeezed out = its bits below j as they are plus
            // its bits above j one lower)
            // h(S + j, j) for the picks j outside S: plane j (2^(k-1) words), block |S|, at the
            // rank of S with bit j squeezed out: over the bits b of S, C(b, t + 1) below j and
            // C(b - 1, t + 1) above, = pb_tot + the sum over the bits below j of C(b - 1, t)
            // (Pascal).  Offsets within the order's table fit 32 bits (20 x 2^19 words at most)
            auto load_succ = [&](HkItem& it, uint32_t pb_tot) {
                const int k = kq[it.qi];
                const unsigned s = it.s;
                const uint32_t* hq = p.h + base[it.qi];
                const uint32_t off0 = loff[k][L] + pb_tot;
                uint32_t pcr = 0;
                int m = 0;
#pragma unroll
                for (int j = 0; j < HK_MAX_K; ++j) {
                    it.hv[j] = INF_U;
                    if (j < k) {
                        if ((s >> j) & 1u) {
                            pcr += binx[j][m];
                            ++m;
                        } else {
                            it.hv[j] = __ldcg(hq + ((static_cast<uint32_t>(j) << (k - 1)) + off0 + pcr));
                        }
                    }
                }
            };
            // the subset after it.s in colex order (the next item of the same order): Gosper's
            // step to the next larger word with as many bits, then its two rank prefixes
            auto next_item = [&](HkItem& it) {
                const unsigned s = it.s;
                const unsigned u = s & (0u - s);
                const unsigned v = s + u;
                const unsigned nx = v | (((v ^ s) >> 2) >> (__ffs(u) - 1));
                uint32_t pb_tot = 0, pc_tot = 0;
                int t = 0;
                for (unsigned m = nx; m; m &= m - 1, ++t) {
                    const int b = __ffs(m) - 1;
                    pb_tot += binx[b][t + 1];
                    pc_tot += binx[b][t];
                }
                it.s = nx;
                it.pc_tot = pc_tot;
                load_succ(it, pb_tot);
            };
            auto load_item = [&](unsigned long long w, HkItem& it) {
                // the order holding item w: the last i with pre[i] <= w (an order with no items at
                // this level shares its pre with the next, so the last one holds w), by bisection
                // from the order of the thread's previous item
                {
                    int hi = nb - 1;
                    while (qi < hi) {
                        const int mid = (qi + hi + 1) >> 1;
                        if (pre[mid] <= w) qi = mid; else hi = mid - 1;
                    }
                }
                const int k = kq[qi];
                it.qi = qi;
                // the subset of rank w - pre[qi] (below C(20, 10): 32-bit) among the L-subsets of k
                // picks, bits from the top: each the largest c below the previous one with
                // C(c, i) <= rr.  Bit c is bit t = i - 1 from the bottom, so the same pass sums,
                // over the bits b_0 < b_1 < ... of S, pb = sum C(b_t - 1, t + 1) and
                // pc = sum C(b_t - 1, t)
                unsigned s = 0;
                uint32_t rr = static_cast<uint32_t>(w - pre[qi]);
                uint32_t pb_tot = 0, pc_tot = 0;
                int c = k - 1;
                for (int i = L; i >= 1; --i, --c) {
                    while (binx[c + 1][i] > rr) --c;  // ends by c = i - 1: C(i - 1, i) = 0
                    s |= 1u << c;
                    rr -= binx[c + 1][i];
                    pb_tot += binx[c][i];
                    pc_tot += binx[c][i - 1];
                }
                it.s = s;
                it.pc_tot = pc_tot;
                load_succ(it, pb_tot);
            };
            // h(S, c) for every c in S: plane c, block |S| - 1, rank of S - c with c's bit squeezed out
            auto store_item = [&](const HkItem& it) {
                const int k = kq[it.qi];
                const unsigned s = it.s, full = (1u << k) - 1u;
                const uint32_t* D = p.D21 + static_cast<int64_t>(q0 + it.qi) * HK_DBLOCK;
                uint32_t* hq = p.h + base[it.qi];
                const uint32_t lo = loff[k][L - 1];
                uint32_t pa = 0, pc = 0;
                int t = 0;
                for (unsigned cm = s; cm; cm &= cm - 1, ++t) {
                    const int c = __ffs(cm) - 1;
                    const uint32_t* Dr = D + (c + 1) * HK_DSTRIDE + HK_DOFF;
                    uint32_t best;
                    if (s == full) {
                        best = __ldg(Dr);
                    } else {
                        // D and h are at most INF_U = 2^31 - 1, so D + h does not wrap, and a minimum
                        // started at INF_U stays at most INF_U: one fused add-min per transition.
                        // hv[j] is INF_U for the picks j in S and past k, and the legs past k are
                        // INF_U, so their terms never win and need no test
                        // the row's pick legs D[c][1..HK_MAX_K] as 16-byte loads
                        const uint4* D4 = reinterpret_cast<const uint4*>(Dr + 1);
                        best = INF_U;
#pragma unroll
                        for (int j4 = 0; j4 < HK_MAX_K / 4; ++j4) {
                            const uint4 d = __ldg(D4 + j4);
                            best = __viaddmin_u32(d.x, it.hv[4 * j4], best);
                            best = __viaddmin_u32(d.y, it.hv[4 * j4 + 1], best);
                            best = __viaddmin_u32(d.z, it.hv[4 * j4 + 2], best);
                            best = __viaddmin_u32(d.w, it.hv[4 * j4 + 3], best);
                        }
                    }
                    const uint32_t cc = binx[c][t];  // C(c - 1, t)
                    __stcg(hq + ((static_cast<uint32_t>(c) << (k - 1)) + lo + (pa + it.pc_tot - pc - cc)), best);
                    pa += binx[c + 1][t + 1];
                    pc += cc;
                }
            };
            // a level with at least four items per thread: two adjacent items per thread and
            // round, the second, when it lies in the same order, one colex step after the first
            // instead of an unranking; a smaller level: one item per thread, so that its items
            // spread over every thread
            const unsigned long long per = total >= 4ull * static_cast<unsigned long long>(nthreads) ? 2ull : 1ull;
            const unsigned long long step = per * static_cast<unsigned long long>(nthreads);
            for (unsigned long long w = per * static_cast<unsigned long long>(gtid); w < total; w += step) {
                HkItem it;
                load_item(w, it);
                store_item(it);
                if (per == 2 && w + 1 < total) {
                    if (w + 1 < pre[it.qi + 1]) next_item(it);
                    else load_item(w + 1, it);
                    store_item(it);
                }
            }
            if (!grid_sync(p.bar, p.err, p.max_spins)) return;
        }
        // rebuild: one warp per order, lanes over the candidate next picks; the
        // lexicographically first optimal sequence takes at every step the smallest j
        // whose leg plus what remains after it equals what remains now
        {
            const int lane = threadIdx.x & 31;
            const long long nw = nthreads >> 5;
            for (long long qi = gtid >> 5; qi < nb; qi += nw) {
                const int q = q0 + static_cast<int>(qi);
                const int k = kq[qi];
                if (k == 0) continue;
                const int o = p.list[q];
                const int64_t b = p.t.offs[o];
                const uint32_t* D = p.D21 + static_cast<int64_t>(q) * HK_DBLOCK;
                const uint32_t* hq = p.h + base[qi];
                const int64_t half = static_cast<int64_t>(1) << (k - 1);
                // h(set + j, j) for j outside set: plane j, block |set|, rank of set with bit j squeezed out
                auto h_at = [&](unsigned set, int j) {
                    uint32_t r = 0;
                    int i = 0;
                    for (unsigned m = set; m; m &= m - 1, ++i) {
                        const int bb = __ffs(m) - 1;
                        r += binom[bb > j ? bb - 1 : bb][i + 1];
                    }
                    return __ldcg(hq + j * half + loff[k][__popc(set)] + r);
                };
                uint32_t best = lane < k ? sat_add(__ldg(D + HK_DOFF + lane + 1), h_at(0u, lane)) : INF_U;
#pragma unroll
                for (int d = 16; d >= 1; d >>= 1) best = min(best, __shfl_xor_sync(FULL_MASK, best, d));
                int32_t* pp = p.perm + b;
                if (best >= INF_U) {
                    if (lane == 0) {
                        p.cost[o] = WR_INF;
                        p.status[o] = WR_ORDER_UNREACHABLE;
                    }
                    if (lane < k) pp[lane] = lane;
                    continue;
                }
                unsigned s = 0;
                int cur = 0;  // matrix index of the current stop (0 = depot)
                uint32_t rem = best;
                bool ok = true;
                for (int pos = 0; pos < k; ++pos) {
                    uint32_t r = INF_U;
                    bool hit = false;
                    if (lane < k && !((s >> lane) & 1u)) {
                        r = h_at(s, lane);
                        hit = sat_add(__ldg(D + cur * HK_DSTRIDE + HK_DOFF + lane + 1), r) == rem;
                    }
                    const unsigned m = __ballot_sync(FULL_MASK, hit);
                    if (m == 0u) {  // cannot happen on a consistent table
                        ok = false;
                        break;
                    }
                    const int j = __ffs(m) - 1;
                    rem = __shfl_sync(FULL_MASK, r, j);
                    if (lane == 0) pp[pos] = j;
                    s |= 1u << j;
                    cur = j + 1;
                }
                if (lane == 0) {
                    p.cost[o] = ok ? static_cast<int32_t>(best) : WR_INF;
                    p.status[o] = ok ? WR_ORDER_OK : WR_ORDER_UNREACHABLE;
                    if (!ok) atomicCAS(p.err, 0, WR_EINTERNAL);
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

constexpr int HK_BLOCKS_PER_SM = 4;  // measured: 3.37 ms at 4 blocks per SM (the register limit), 3.53 at 3, 4.44 at 2

int hk_blocks(int device) {
    int occ = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hk_solve_kernel, 256, 0) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
    return (occ < HK_BLOCKS_PER_SM ? occ : HK_BLOCKS_PER_SM) * sms;
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
