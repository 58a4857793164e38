// Rows a2 and a4-a7: source selection, D gather, exhaustive sequence
// evaluation with rank-range segments, reduction and result decode.
//
// Sec. 4.6 evaluates all n! route permutations, one thread per permutation
// and an inner loop over the transitions.  Here a thread owns a contiguous
// range of "units": for k >= 7 a unit fixes the first k-7 picks of the
// sequence (its prefix, decoded from the unit index in the factorial number
// system) and covers the 5040 orderings of the remaining seven: each of the
// seven next, then the 720 orderings of the other six, costed in registers
// from tables of the legs among those six.  Every one of the k! sequences
// still gets its own cost computed and compared; shared partial sums only
// avoid re-adding the same legs.  A thread keeps the minimum of each block of
// 120 sequences; only when a block beats the thread's best does it look for
// the lowest-rank sequence attaining it.  Blocks are visited in increasing
// rank, so the first match keeps the lowest rank.  Segment minima are merged
// into one 64-bit word per order, (cost << 32) | rank, with atomicMin: the
// lexicographic (cost, rank) minimum, independent of scheduling.
#include "wr_device.cuh"

namespace wr {

// ---------------------------------------------------------------------------
// a2: source selection
// ---------------------------------------------------------------------------

// Order o: its status, and node_flag set at its picks when it is valid.
__device__ __forceinline__ void select_order(int o, int32_t n, const int64_t* __restrict__ offs,
                                             const int32_t* __restrict__ picks, int32_t V, int32_t max_k,
                                             uint8_t* node_flag, int32_t* order_status) {
    const int64_t b = offs[o], e = offs[o + 1];
    const int64_t k = e - b;
    int st = WR_ORDER_OK;
    // offsets that do not start at 0 make the whole call invalid: no pick is read (the host
    // returns WR_EINVAL once it has read them back)
    if (k < 1 || k > max_k || b < 0 || e > offs[n] || offs[0] != 0) {
        st = WR_ORDER_BAD;
    } else {
        for (int64_t i = b; i < e; ++i)
            if (picks[i] < 0 || picks[i] >= V) st = WR_ORDER_BAD;
        if (st == WR_ORDER_OK)
            for (int64_t i = b; i < e; ++i) node_flag[picks[i]] = 1;
    }
    order_status[o] = st;
}

__global__ void select_kernel(int32_t n, const int64_t* __restrict__ offs, const int32_t* __restrict__ picks,
                              int32_t V, int32_t depot, int32_t max_k, uint8_t* node_flag, int32_t* order_status) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o == 0) node_flag[depot] = 1;
    if (o < n) select_order(o, n, offs, picks, V, max_k, node_flag, order_status);
}

cudaError_t tour_launch_select(int32_t n, const int64_t* offs, const int32_t* picks, int32_t V, int32_t depot,
                               int32_t max_k, uint8_t* node_flag, int32_t* order_status, cudaStream_t s) {
    select_kernel<<<(n + 255) / 256 + (n == 0), 256, 0, s>>>(n, offs, picks, V, depot, max_k, node_flag,
                                                              order_status);
    return cudaGetLastError();
}

// Compaction of node_flag into the ascending source list and node -> source index.
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int block_exclusive_scan(int x, int* warp_sums, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(FULL_MASK, inc, d);
        if (lane >= d) inc += y;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int ws = lane < (blockDim.x >> 5) ? warp_sums[lane] : 0;
        int wi = ws;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(FULL_MASK, wi, d);
            if (lane >= d) wi += y;
        }
        warp_sums[lane] = wi - ws;
        if (lane == 31) *total = wi;
    }
    __syncthreads();
    const int r = warp_sums[warp] + inc - x;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SCAN_THREADS) compact_count_kernel(int32_t V, const uint8_t* __restrict__ flag,
                                                                       int32_t* block_sums) {
    __shared__ int ws[32];
    __shared__ int tot;
    const int64_t base = static_cast<int64_t>(blockIdx.x) * SCAN_CHUNK + threadIdx.x * SCAN_ITEMS;
    int c = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q)
        if (base + q < V) c += flag[base + q];
    block_exclusive_scan(c, ws, &tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_THREADS) compact_top_kernel(int32_t nb, int32_t* block_sums, int32_t* n_src) {
    __shared__ int ws[32];
    __shared__ int tot;
    int carry = 0;
    for (int base = 0; base < nb; base += SCAN_THREADS) {
        const int i = base + threadIdx.x;
        const int x = i < nb ? block_sums[i] : 0;
        const int ex = block_exclusive_scan(x, ws, &tot);
        if (i < nb) block_sums[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *n_src = carry;
}

__global__ void __launch_bounds__(SCAN_THREADS) compact_apply_kernel(int32_t V, const uint8_t* __restrict__ flag,
                                                                       const int32_t* __restrict__ block_sums,
                                                                       int32_t* src_index, int32_t* src_list) {
    __shared__ int ws[32];
    __shared__ int tot;
    const int64_t base = static_cast<int64_t>(blockIdx.x) * SCAN_CHUNK + threadIdx.x * SCAN_ITEMS;
    int f[SCAN_ITEMS];
    int c = 0;
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        f[q] = (base + q < V) ? flag[base + q] : 0;
        c += f[q];
    }
    int pos = block_sums[blockIdx.x] + block_exclusive_scan(c, ws, &tot);
#pragma unroll
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        if (base + q < V) {
            const int32_t v = static_cast<int32_t>(base + q);
            if (f[q]) {
                src_index[v] = pos;
                src_list[pos] = v;
                ++pos;
            } else {
                src_index[v] = -1;
            }
        }
    }
}

// The same compaction by one block walking the chunks in order with a running
// carry: one launch instead of three for graphs of up to SINGLE_MAX_CHUNKS chunks.
constexpr int SINGLE_MAX_CHUNKS = 64;

__device__ __forceinline__ void compact_block(int32_t V, const uint8_t* __restrict__ flag, int32_t* src_index,
                                              int32_t* src_list, int32_t* n_src) {
    __shared__ int ws[32];
    __shared__ int tot;
    int carry = 0;
    for (int64_t chunk = 0; chunk < V; chunk += SCAN_CHUNK) {
        const int64_t base = chunk + threadIdx.x * SCAN_ITEMS;
        int f[SCAN_ITEMS];
        int c = 0;
#pragma unroll
        for (int q = 0; q < SCAN_ITEMS; ++q) {
            f[q] = (base + q < V) ? flag[base + q] : 0;
            c += f[q];
        }
        int pos = carry + block_exclusive_scan(c, ws, &tot);
#pragma unroll
        for (int q = 0; q < SCAN_ITEMS; ++q) {
            if (base + q < V) {
                const int32_t v = static_cast<int32_t>(base + q);
                if (f[q]) {
                    src_index[v] = pos;
                    src_list[pos] = v;
                    ++pos;
                } else {
                    src_index[v] = -1;
                }
            }
        }
        carry += tot;  // every thread reads the chunk's total before the next scan overwrites it
    }
    if (threadIdx.x == 0) *n_src = carry;
}

__global__ void __launch_bounds__(SCAN_THREADS) compact_single_kernel(int32_t V, const uint8_t* __restrict__ flag,
                                                                        int32_t* src_index, int32_t* src_list,
                                                                        int32_t* n_src) {
    compact_block(V, flag, src_index, src_list, n_src);
}

// Selection and compaction of a small call in one block: clear the node flags
// (and the order flags), select every order, then compact.  Global writes of
// the block's threads are visible to each other after __syncthreads.
__global__ void __launch_bounds__(SCAN_THREADS) select_compact_kernel(int32_t n, const int64_t* __restrict__ offs,
                                                                        const int32_t* __restrict__ picks, int32_t V,
                                                                        int32_t depot, int32_t max_k, uint8_t* node_flag,
                                                                        int32_t* order_status, int32_t* order_flags,
                                                                        int32_t* src_index, int32_t* src_list,
                                                                        int32_t* n_src) {
    for (int v = threadIdx.x; v < V; v += SCAN_THREADS) node_flag[v] = 0;
    if (order_flags)
        for (int o = threadIdx.x; o < n; o += SCAN_THREADS) order_flags[o] = 0;
    __syncthreads();
    if (threadIdx.x == 0) node_flag[depot] = 1;
    for (int o = threadIdx.x; o < n; o += SCAN_THREADS) select_order(o, n, offs, picks, V, max_k, node_flag, order_status);
    __syncthreads();
    compact_block(V, node_flag, src_index, src_list, n_src);
}

// One block: graphs of up to SINGLE_MAX_CHUNKS chunks and calls of up to this many orders.
constexpr int FUSED_MAX_ORDERS = 4 * SCAN_THREADS;

cudaError_t tour_launch_select_compact(int32_t n, const int64_t* offs, const int32_t* picks, int32_t V, int32_t depot,
                                       int32_t max_k, uint8_t* node_flag, int32_t* order_status, int32_t* order_flags,
                                       int32_t* src_index, int32_t* src_list, int32_t* n_src, int32_t* block_sums,
                                       cudaStream_t s, int* launches) {
    const int nb = (V + SCAN_CHUNK - 1) / SCAN_CHUNK;
    if (nb <= SINGLE_MAX_CHUNKS && n <= FUSED_MAX_ORDERS) {
        select_compact_kernel<<<1, SCAN_THREADS, 0, s>>>(n, offs, picks, V, depot, max_k, node_flag, order_status,
                                                          order_flags, src_index, src_list, n_src);
        *launches += 1;
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(node_flag, 0, static_cast<size_t>(V), s);
    if (e == cudaSuccess && order_flags) e = cudaMemsetAsync(order_flags, 0, static_cast<size_t>(n) * 4, s);
    if (e == cudaSuccess) e = tour_launch_select(n, offs, picks, V, depot, max_k, node_flag, order_status, s);
    if (e != cudaSuccess) return e;
    *launches += 1;
    return tour_launch_compact(V, node_flag, src_index, src_list, n_src, block_sums, s, launches);
}

cudaError_t tour_launch_compact(int32_t V, const uint8_t* node_flag, int32_t* src_index, int32_t* src_list,
                                int32_t* n_src, int32_t* block_sums, cudaStream_t s, int* launches) {
    const int nb = (V + SCAN_CHUNK - 1) / SCAN_CHUNK;
    if (nb <= SINGLE_MAX_CHUNKS) {
        compact_single_kernel<<<1, SCAN_THREADS, 0, s>>>(V, node_flag, src_index, src_list, n_src);
        *launches += 1;
        return cudaGetLastError();
    }
    compact_count_kernel<<<nb, SCAN_THREADS, 0, s>>>(V, node_flag, block_sums);
    compact_top_kernel<<<1, SCAN_THREADS, 0, s>>>(nb, block_sums, n_src);
    compact_apply_kernel<<<nb, SCAN_THREADS, 0, s>>>(V, node_flag, block_sums, src_index, src_list);
    *launches += 3;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a4: D gather.  D[i][j] = dist(P_i, P_j), P_0 = depot; the row of P_i lives
// in the segment holding its source index.  Unreachable legs become TOUR_CAP;
// a finite leg above WR_LEG_MAX flags the order.
// ---------------------------------------------------------------------------

__global__ void gather_kernel(int32_t n, TourBufs t, int32_t depot, const int32_t* __restrict__ src_index,
                              BfSegment seg, int open_path) {
    const int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (o >= n) return;
    if (t.order_status[o] != WR_ORDER_OK) return;
    const int64_t b = t.offs[o];
    const int k = static_cast<int>(t.offs[o + 1] - b);
    if (k > WR_MAX_K) return;  // Held-Karp orders gather into their own blocks
    const int m = k + 1;
    bool range = false;
    for (int e = lane; e < m * m; e += 32) {
        const int i = e / m, j = e - i * m;
        if (open_path && (i == 0 || j == 0)) {
            // open path: the entrance/exit is not part of the route, its legs are free
            t.D[static_cast<int64_t>(o) * DBLOCK + i * DSTRIDE + j] = 0u;
            continue;
        }
        const int32_t pi = i == 0 ? depot : t.picks[b + i - 1];
        const int32_t si = src_index[pi] - seg.first;
        if (si < 0 || si >= seg.lanes) continue;
        const int32_t pj = j == 0 ? depot : t.picks[b + j - 1];
        uint32_t val = __ldcg(seg.rows + static_cast<int64_t>(pj) * seg.ld + si);
        if (val == INF_U) {
            val = TOUR_CAP;
        } else if (val > static_cast<uint32_t>(WR_LEG_MAX) && i != j) {
            range = true;
        }
        t.D[static_cast<int64_t>(o) * DBLOCK + i * DSTRIDE + j] = val;
    }
    if (__any_sync(FULL_MASK, range) && lane == 0) atomicOr(t.order_flags + o, ORDER_FLAG_RANGE);
}

cudaError_t tour_launch_gather(int32_t n, const TourBufs& t, int32_t depot, const int32_t* src_index,
                               const BfSegment& seg, int open_path, cudaStream_t s) {
    gather_kernel<<<(n + 7) / 8, 256, 0, s>>>(n, t, depot, src_index, seg, open_path);
    return cudaGetLastError();
}

// Given matrices (wr_tour_eval): validate k, clamp, flag range.
__global__ void prepare_given_kernel(int32_t n, const int32_t* __restrict__ kk, const int32_t* __restrict__ Din,
                                     int32_t max_k, TourBufs t) {
    const int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (o >= n) return;
    const int k = kk[o];
    if (k < 1 || k > max_k) {
        if (lane == 0) {
            t.order_status[o] = WR_ORDER_BAD;
            t.order_flags[o] = 0;
        }
        return;
    }
    const int m = k + 1;
    bool range = false;
    for (int e = lane; e < m * m; e += 32) {
        const int i = e / m, j = e - i * m;
        uint32_t val = static_cast<uint32_t>(Din[static_cast<int64_t>(o) * DBLOCK + i * DSTRIDE + j]);
        if (val == INF_U) {
            val = TOUR_CAP;
        } else if (i != j && val > static_cast<uint32_t>(WR_LEG_MAX)) {  // negatives land here too
            range = true;
        }
        t.D[static_cast<int64_t>(o) * DBLOCK + i * DSTRIDE + j] = val;
    }
    const bool any = __any_sync(FULL_MASK, range);
    if (lane == 0) {
        t.order_status[o] = WR_ORDER_OK;
        t.order_flags[o] = any ? ORDER_FLAG_RANGE : 0;
    }
}

cudaError_t tour_launch_prepare_given(int32_t n, const int32_t* k, const int32_t* Din, int32_t max_k,
                                      const TourBufs& t, cudaStream_t s) {
    prepare_given_kernel<<<(n + 7) / 8, 256, 0, s>>>(n, k, Din, max_k, t);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// units per order and their exclusive prefix (one block)
// ---------------------------------------------------------------------------

__device__ __forceinline__ int order_k(const TourBufs& t, const int32_t* k_given, int o) {
    return k_given ? k_given[o] : static_cast<int>(t.offs[o + 1] - t.offs[o]);
}

// Orders of at least this many picks enumerate in set units, smaller ones in
// prefix units (see enum_order_range), in a call with at least SET_UNITS_MIN_ORDERS
// such orders.  A set unit of 11 or 12 picks holds 17,280 sequences (a prefix
// unit 5,040): fewer large orders leave too few of them to end close together.
constexpr int SET_UNITS_FROM = 11;
constexpr int SET_UNITS_MIN_ORDERS = 32;

__device__ __forceinline__ long long units_of(int k, bool sets) {
    // k <= 6: 1.  Prefix units, 7 <= k < SET_UNITS_FROM: k! / 7! (a unit is an ordered prefix of
    // k - 7 picks and the 5040 orderings of the last seven).  Set units: C(k, q) sets of the
    // first q = k - 7 picks x 7 picks next x (q = 5) 5 first picks.  Orders above WR_MAX_K are
    // solved by Held-Karp instead
    if (k > WR_MAX_K) return 0;
    if (k <= UNIT_TAIL) return 1;
    const int q = k - UNIT_TAIL - 1;
    if (!sets || k < SET_UNITS_FROM) {
        long long u = 1;
        for (int i = UNIT_TAIL + 2; i <= k; ++i) u *= i;
        return u;
    }
    long long c = 1;  // C(k, q)
    for (int j = 1; j <= q; ++j) c = c * (k - q + j) / j;
    return c * 7 * (q == 5 ? 5 : 1);
}

__global__ void __launch_bounds__(SCAN_THREADS) units_kernel(int32_t n, const int32_t* k_given, TourBufs t) {
    __shared__ long long ws[32];
    __shared__ long long tot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long carry = 0;
    // set units when the call holds enough orders of SET_UNITS_FROM .. WR_MAX_K picks
    int big = 0;
    for (int o = threadIdx.x; o < n; o += SCAN_THREADS)
        if (t.order_status[o] == WR_ORDER_OK && !(t.order_flags[o] & ORDER_FLAG_RANGE)) {
            const int k = order_k(t, k_given, o);
            big += k >= SET_UNITS_FROM && k <= WR_MAX_K;
        }
    __shared__ int n_big;
    if (threadIdx.x == 0) n_big = 0;
    __syncthreads();
    big = __reduce_add_sync(FULL_MASK, big);
    if (lane == 0 && big) atomicAdd(&n_big, big);
    __syncthreads();
    const bool sets = n_big >= SET_UNITS_MIN_ORDERS;
    for (int base = 0; base < n; base += SCAN_THREADS) {
        const int o = base + threadIdx.x;
        long long x = 0;
        if (o < n) {
            t.best[o] = ~0ull;
            if (t.order_status[o] == WR_ORDER_OK && !(t.order_flags[o] & ORDER_FLAG_RANGE))
                x = units_of(order_k(t, k_given, o), sets);
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
            const long long w0 = ws[lane];
            long long wi = w0;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const long long y = __shfl_up_sync(FULL_MASK, wi, d);
                if (lane >= d) wi += y;
            }
            ws[lane] = wi - w0;
            if (lane == 31) tot = wi;
        }
        __syncthreads();
        if (o < n) t.unit_off[o] = carry + ws[warp] + inc - x;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        t.unit_off[n] = carry;
        t.unit_ctr[0] = 0ull;
        t.unit_ctr[1] = sets ? 1ull : 0ull;  // which enumeration kernel runs
    }
}

cudaError_t tour_launch_units(int32_t n, const int32_t* k_given, const TourBufs& t, cudaStream_t s, int* launches) {
    units_kernel<<<1, SCAN_THREADS, 0, s>>>(n, k_given, t);
    *launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a5/a6: enumeration
// ---------------------------------------------------------------------------

// Leg tables of one unit, indexed by tail position (compile-time indices only,
// so everything lives in registers).
template <int L>
struct Tab {
    uint32_t x[L];        // D[x][t_i], x = last prefix node (or the depot)
    uint32_t d[L][L];     // D[t_i][t_j]
    uint32_t h[L];        // D[t_i][0]
    uint32_t t3[L][L][L];  // D[t_a][t_b] + D[t_b][t_c] + D[t_c][0] (distinct a, b, c)
};

template <unsigned M>
struct Bits {
    static constexpr int count = (M & 1u) + Bits<(M >> 1)>::count;
    static constexpr int low = (M & 1u) ? 0 : 1 + Bits<(M >> 1)>::low;
};
template <>
struct Bits<0u> {
    static constexpr int count = 0;
    static constexpr int low = 64;
};

__host__ __device__ constexpr int cfact(int n) { return n <= 1 ? 1 : n * cfact(n - 1); }

// Walks of the prefix tree below a node: M = tail positions still to visit,
// CUR = tail position just visited (-1: the prefix end x), IDX = lexicographic
// index of the subtree's first sequence within the walk.  Children are visited
// in increasing position, i.e. lexicographic order of the sequences.
// Scan folds every leaf's cost into one of NACC accumulators with one fused
// add-min; accumulator a takes the a-th contiguous range of leaves, so the
// first accumulator holding a block's minimum names the range that holds its
// lowest-rank minimiser.  Find sets idx to the index of the first leaf whose
// cost equals target.
constexpr int NACC = 4;

template <int L>
struct AccSpan {
    static constexpr int value = (cfact(L) + NACC - 1) / NACC;  // leaves per accumulator
};

template <int L, unsigned M, int CUR, int IDX>
struct Scan;

template <int L, unsigned M, unsigned REST, int CUR, int IDX>
struct ScanChildren {
    static __device__ __forceinline__ void run(uint32_t acc, const Tab<L>& T, uint32_t (&mn)[NACC]) {
        if constexpr (REST != 0u) {
            constexpr int i = Bits<REST>::low;
            uint32_t leg;
            if constexpr (CUR < 0) leg = T.x[i];
            else leg = T.d[CUR][i];
            Scan<L, (M & ~(1u << i)), i, IDX>::run(acc + leg, T, mn);
            ScanChildren<L, M, (REST & ~(1u << i)), CUR, IDX + cfact(Bits<M>::count - 1)>::run(acc, T, mn);
        }
    }
};

template <int L, unsigned M, int CUR, int IDX>
struct Scan {
    static __device__ __forceinline__ void run(uint32_t acc, const Tab<L>& T, uint32_t (&mn)[NACC]) {
        constexpr int n = Bits<M>::count;
        constexpr int S = AccSpan<L>::value;
        if constexpr (n == 0) {
            mn[IDX / S] = __viaddmin_u32(acc, T.h[CUR], mn[IDX / S]);
        } else if constexpr (n == 2 && CUR >= 0) {
            constexpr int b = Bits<M>::low;
            constexpr int c = Bits<(M & ~(1u << b))>::low;
            mn[IDX / S] = __viaddmin_u32(acc, T.t3[CUR][b][c], mn[IDX / S]);
            mn[(IDX + 1) / S] = __viaddmin_u32(acc, T.t3[CUR][c][b], mn[(IDX + 1) / S]);
        } else {
            ScanChildren<L, M, M, CUR, IDX>::run(acc, T, mn);
        }
    }
};

template <int L, unsigned M, int CUR, int IDX>
struct Find;

template <int L, unsigned M, unsigned REST, int CUR, int IDX>
struct FindChildren {
    static __device__ __forceinline__ void run(uint32_t acc, const Tab<L>& T, uint32_t target, int& idx) {
        if constexpr (REST != 0u) {
            constexpr int i = Bits<REST>::low;
            uint32_t leg;
            if constexpr (CUR < 0) leg = T.x[i];
            else leg = T.d[CUR][i];
            Find<L, (M & ~(1u << i)), i, IDX>::run(acc + leg, T, target, idx);
            FindChildren<L, M, (REST & ~(1u << i)), CUR, IDX + cfact(Bits<M>::count - 1)>::run(acc, T, target, idx);
        }
    }
};

template <int L, unsigned M, int CUR, int IDX>
struct Find {
    static __device__ __forceinline__ void run(uint32_t acc, const Tab<L>& T, uint32_t target, int& idx) {
        constexpr int n = Bits<M>::count;
        if constexpr (n == 0) {
            if (idx < 0 && acc + T.h[CUR] == target) idx = IDX;
        } else if constexpr (n == 2 && CUR >= 0) {
            constexpr int b = Bits<M>::low;
            constexpr int c = Bits<(M & ~(1u << b))>::low;
            if (idx < 0 && acc + T.t3[CUR][b][c] == target) idx = IDX;
            if (idx < 0 && acc + T.t3[CUR][c][b] == target) idx = IDX + 1;
        } else {
            FindChildren<L, M, M, CUR, IDX>::run(acc, T, target, idx);
        }
    }
};

template <int L>
__device__ __forceinline__ void load_tab(Tab<L>& T, const uint32_t* __restrict__ Dm, int x, const int (&t)[TAIL]) {
#pragma unroll
    for (int i = 0; i < L; ++i) {
        T.x[i] = __ldg(Dm + x * DSTRIDE + t[i]);
        T.h[i] = __ldg(Dm + t[i] * DSTRIDE);
#pragma unroll
        for (int j = 0; j < L; ++j)
            if (i != j) T.d[i][j] = __ldg(Dm + t[i] * DSTRIDE + t[j]);
    }
    if constexpr (L >= 3) {
#pragma unroll
        for (int b = 0; b < L; ++b)
#pragma unroll
            for (int c = 0; c < L; ++c) {
                if (b == c) continue;
                const uint32_t tail2 = T.d[b][c] + T.h[c];
#pragma unroll
                for (int a = 0; a < L; ++a)
                    if (a != b && a != c) T.t3[a][b][c] = T.d[a][b] + tail2;
            }
    }
}

__device__ __forceinline__ uint32_t min_of(const uint32_t (&mn)[NACC]) {
    uint32_t m = mn[0];
#pragma unroll
    for (int i = 1; i < NACC; ++i) m = min(m, mn[i]);
    return m;
}

// An order of k <= 5 picks: the L! orderings of all picks after the depot.
// Folds (cost, rank) into (best_c, best_r) when the order holds a sequence
// that is lexicographically smaller in (cost, rank).
template <int L>
__device__ __forceinline__ void unit_eval(const uint32_t* __restrict__ Dm, const int (&t)[TAIL], uint32_t& best_c,
                                          unsigned& best_r) {
    Tab<L> T;
    load_tab<L>(T, Dm, 0, t);
    uint32_t mins[NACC];
#pragma unroll
    for (int i = 0; i < NACC; ++i) mins[i] = 0xFFFFFFFFu;
    Scan<L, (1u << L) - 1u, -1, 0>::run(0u, T, mins);
    const uint32_t mn = min_of(mins);
    if (mn < best_c || (mn == best_c && 0u < best_r)) {
        int idx = -1;
        Find<L, (1u << L) - 1u, -1, 0>::run(0u, T, mn, idx);
        const unsigned r = static_cast<unsigned>(idx);
        if (mn < best_c || r < best_r) {
            best_c = mn;
            best_r = r;
        }
    }
}

__device__ __forceinline__ void unit_eval_dispatch(int L, const uint32_t* Dm, const int (&t)[TAIL], uint32_t& best_c,
                                                   unsigned& best_r) {
    switch (L) {
        case 1: unit_eval<1>(Dm, t, best_c, best_r); break;
        case 2: unit_eval<2>(Dm, t, best_c, best_r); break;
        case 3: unit_eval<3>(Dm, t, best_c, best_r); break;
        case 4: unit_eval<4>(Dm, t, best_c, best_r); break;
        default: unit_eval<5>(Dm, t, best_c, best_r); break;
    }
}

// n-th (0-based) set bit of m.
__device__ __forceinline__ int nth_bit(unsigned m, int n) {
    for (int i = 0; i < n; ++i) m &= m - 1;
    return __ffs(m) - 1;
}

// Lexicographic index, within [lo, hi), of the first ordering of the five
// picks packed in `five` (4-bit matrix indices, increasing) whose cost after
// a prefix of cost acc ending at s, back to the depot, equals target.  Runs
// at most once per thread and unit range, for the block range that recorded
// the thread's best, so it is a plain loop over D: small code, off the hot
// path.  Its sums are the hot path's sums regrouped, and exact (no term
// reaches 2^28, at most 13 terms).
__device__ __noinline__ int first_of_five(const uint32_t* __restrict__ Dm, uint32_t acc, int s, unsigned five,
                                          uint32_t target, int lo, int hi) {
    for (int idx = lo; idx < hi; ++idx) {
        unsigned rest = five;
        int r = idx, f = 24, prev = s;
        uint32_t c = acc;
        for (int pos = 0; pos < 5; ++pos) {
            const int d = r / f;
            r -= d * f;
            const int e = static_cast<int>((rest >> (4 * d)) & 15u);
            rest = (rest & ((1u << (4 * d)) - 1u)) | ((rest >> (4 * d + 4)) << (4 * d));
            c += __ldg(Dm + prev * DSTRIDE + e);
            prev = e;
            if (pos < 3) f /= (4 - pos);
        }
        c += __ldg(Dm + prev * DSTRIDE);
        if (c == target) return idx;
    }
    return lo;  // not reached: target is the cost of one of these orderings
}

// The block range that holds a thread's best so far: the five picks after s_J
// and the cost through s_J, to find the exact rank once at the end.
struct BlockRec {
    uint32_t acc;
    unsigned five, rank0;
    int sj, lo;
    bool have;
};

// k-th smallest of 0..4 outside the bit set used (compile-time relabeling).
__host__ __device__ constexpr int kth_free5(unsigned used, int k) {
    for (int i = 0; i < 5; ++i)
        if (!(used & (1u << i))) {
            if (k == 0) return i;
            --k;
        }
    return -1;
}

// One block of 120 sequences of a 720-sequence unit: the six remaining picks
// s_0 < ... < s_5 (matrix indices packed in sp), s_J next, then the 120
// orderings of the other five, costed from compile-time views of the six's
// tables: legs between them (d6) and every three-leg suffix ending at the
// depot (t3f[a][b][c] = D[s_a][s_b] + D[s_b][s_c] + D[s_c][0]).  acc = cost
// of the sequence through s_J.  The five subtrees below the first of the five
// (24 sequences each, SUB24) are walked side by side: each step does the same
// relative move in all five, so the five running minima (one per subtree)
// form five independent add-min chains instead of one long one.
constexpr int SUB24 = 24;

template <int J>
__device__ __forceinline__ void tail6_block(const uint32_t (&d6)[6][6], const uint32_t (&t3f)[6][6][6], unsigned sp,
                                            uint32_t acc, unsigned rank0, uint32_t& cur_c, unsigned& cur_r,
                                            BlockRec& rec) {
    Tab<5> T;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const int ri = i < J ? i : i + 1;
        T.x[i] = d6[J][ri];
        T.h[i] = 0u;  // the 5-tail never ends above a three-leg suffix
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const int rq = q < J ? q : q + 1;
            if (i != q) T.d[i][q] = d6[ri][rq];
        }
    }
#pragma unroll
    for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int b = 0; b < 5; ++b)
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                if (a == b || a == c || b == c) continue;
                T.t3[a][b][c] = t3f[a < J ? a : a + 1][b < J ? b : b + 1][c < J ? c : c + 1];
            }
    uint32_t mn[5], a0[5];
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        mn[s] = 0xFFFFFFFFu;
        a0[s] = acc + T.x[s];
    }
#pragma unroll
    for (int i1 = 0; i1 < 4; ++i1) {
        uint32_t a1[5];
#pragma unroll
        for (int s = 0; s < 5; ++s) a1[s] = a0[s] + T.d[s][kth_free5(1u << s, i1)];
#pragma unroll
        for (int i2 = 0; i2 < 3; ++i2) {
            uint32_t a2[5];
#pragma unroll
            for (int s = 0; s < 5; ++s) {
                const int p1 = kth_free5(1u << s, i1);
                a2[s] = a1[s] + T.d[p1][kth_free5((1u << s) | (1u << p1), i2)];
            }
            // the two orderings of the last two picks b < c: (b, c) first, then (c, b)
#pragma unroll
            for (int s = 0; s < 5; ++s) {
                const int p1 = kth_free5(1u << s, i1);
                const unsigned u2 = (1u << s) | (1u << p1);
                const int p2 = kth_free5(u2, i2);
                const unsigned u3 = u2 | (1u << p2);
                mn[s] = __viaddmin_u32(a2[s], T.t3[p2][kth_free5(u3, 0)][kth_free5(u3, 1)], mn[s]);
            }
#pragma unroll
            for (int s = 0; s < 5; ++s) {
                const int p1 = kth_free5(1u << s, i1);
                const unsigned u2 = (1u << s) | (1u << p1);
                const int p2 = kth_free5(u2, i2);
                const unsigned u3 = u2 | (1u << p2);
                mn[s] = __viaddmin_u32(a2[s], T.t3[p2][kth_free5(u3, 1)][kth_free5(u3, 0)], mn[s]);
            }
        }
    }
    uint32_t m = mn[0];
#pragma unroll
    for (int s = 1; s < 5; ++s) m = min(m, mn[s]);
    // cur_r: the exact rank of the order's best, or the first rank of the
    // recorded subtree; every later block starts above both
    if (m < cur_c || (m == cur_c && rank0 < cur_r)) {
        int a = 4;
#pragma unroll
        for (int s = 3; s >= 0; --s)
            if (mn[s] == m) a = s;
        cur_c = m;
        cur_r = rank0 + static_cast<unsigned>(a * SUB24);
        rec.acc = acc;
        rec.five = (sp & ((1u << (4 * J)) - 1u)) | ((sp >> (4 * J + 4)) << (4 * J));
        rec.sj = static_cast<int>((sp >> (4 * J)) & 15u);
        rec.rank0 = rank0;
        rec.lo = a * SUB24;
        rec.have = true;
    }
}

template <int J>
struct Tail6 {
    static __device__ __forceinline__ void run(const uint32_t (&d6)[6][6], const uint32_t (&t3f)[6][6][6],
                                               const uint32_t (&xl)[6], unsigned sp, uint32_t P, unsigned rank0,
                                               uint32_t& cur_c, unsigned& cur_r, BlockRec& rec) {
        if constexpr (J < 6) {
            tail6_block<J>(d6, t3f, sp, P + xl[J], rank0 + 120u * J, cur_c, cur_r, rec);
            Tail6<J + 1>::run(d6, t3f, xl, sp, P, rank0, cur_c, cur_r, rec);
        }
    }
};

// One 720-sequence unit: a prefix of cost P ending at x (0: the depot), then
// the 720 orderings of the six picks in `six` (a bit set of matrix indices);
// rank0 = rank of its first sequence.
// Register tables of a 720-sequence part: the six picks after x (packed in
// sp), legs from x to them, legs among them, and their three-leg suffixes.
struct PartTab {
    uint32_t d6[6][6], t3f[6][6][6], xl[6];
    unsigned sp;
};

__device__ __forceinline__ void part_tables(const uint32_t* __restrict__ Dm, int x, unsigned six, PartTab& T) {
    int sx[UNIT_TAIL];
    unsigned sp = 0;
#pragma unroll
    for (int i = 0; i < UNIT_TAIL; ++i) {
        sx[i] = __ffs(six) - 1;
        six &= six - 1;
        sp |= static_cast<unsigned>(sx[i]) << (4 * i);
    }
    T.sp = sp;
    uint32_t h6[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const uint32_t* row = Dm + sx[i] * DSTRIDE;
        T.xl[i] = __ldg(Dm + x * DSTRIDE + sx[i]);
        h6[i] = __ldg(row);
#pragma unroll
        for (int q = 0; q < 6; ++q)
            if (q != i) T.d6[i][q] = __ldg(row + sx[q]);
    }
#pragma unroll
    for (int b = 0; b < 6; ++b)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            if (b == c) continue;
            const uint32_t tail2 = T.d6[b][c] + h6[c];
#pragma unroll
            for (int a = 0; a < 6; ++a)
                if (a != b && a != c) T.t3f[a][b][c] = T.d6[a][b] + tail2;
        }
}

__device__ __forceinline__ void unit720(const uint32_t* __restrict__ Dm, uint32_t P, int x, unsigned six,
                                        unsigned rank0, uint32_t& cur_c, unsigned& cur_r, BlockRec& rec) {
    int sx[UNIT_TAIL];
    unsigned sp = 0;
#pragma unroll
    for (int i = 0; i < UNIT_TAIL; ++i) {
        sx[i] = __ffs(six) - 1;
        six &= six - 1;
        sp |= static_cast<unsigned>(sx[i]) << (4 * i);
    }
    uint32_t d6[6][6], xl[6], h6[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const uint32_t* row = Dm + sx[i] * DSTRIDE;
        xl[i] = __ldg(Dm + x * DSTRIDE + sx[i]);
        h6[i] = __ldg(row);
#pragma unroll
        for (int q = 0; q < 6; ++q)
            if (q != i) d6[i][q] = __ldg(row + sx[q]);
    }
    uint32_t t3f[6][6][6];
#pragma unroll
    for (int b = 0; b < 6; ++b)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            if (b == c) continue;
            const uint32_t tail2 = d6[b][c] + h6[c];
#pragma unroll
            for (int a = 0; a < 6; ++a)
                if (a != b && a != c) t3f[a][b][c] = d6[a][b] + tail2;
        }
    Tail6<0>::run(d6, t3f, xl, sp, P, rank0, cur_c, cur_r, rec);
}

// Small tables of the enumeration kernel (shared memory).
struct EnumTabs {
    const uint32_t* cb;    // cb[6 n + r] = C(n, r), n <= 12, r <= 5
    const uint32_t* fact;  // fact[n] = n!, n <= 12
    // perm[24 (n - 1) + r] = the r-th ordering (lexicographic) of n <= 4 items: nibble i holds
    // the item at position i (bits 0-1) and how many of the items before it are smaller (bits 2-3)
    const uint16_t* perm;
};

// Enumerate the units [ulo, uhi) of one order (k picks, D block Dm); fold
// the best (cost, rank) into *out.  k <= 5: one unit of k! sequences; k = 6:
// one unit of 720.  For k >= 7 let q = k - 7, the picks before the last seven.
// Prefix units (k < SET_UNITS_FROM): unit u fixes the first q picks in the
// order of its factorial digits and covers the 5040 orderings of the other
// seven, as seven 720-sequence parts (each of the seven, in increasing order,
// next).  Set units (k >= SET_UNITS_FROM): a unit is a set Q of q picks, one
// pick x of the other seven and, for q = 5, the first pick of Q; it covers
// every ordering of Q (of the rest of Q after that first pick) followed by x
// and the 720 orderings of the other six.  A part's leg and suffix tables
// depend only on x and the six, so a set unit builds them once for all its
// orderings of Q, each of which adds its own prefix cost and rank.  Either way
// every sequence is costed and compared on its own.
template <bool SETS>
__device__ void enum_order_range(const uint32_t* __restrict__ Dm, int k, unsigned ulo, unsigned uhi,
                                 unsigned long long* out, long long& seqs, const EnumTabs& tb) {
    // start from the order's current best (a stale read is only larger, so safe)
    const unsigned long long g0 = __ldcg(out);
    uint32_t best_c = static_cast<uint32_t>(g0 >> 32);
    unsigned best_r = static_cast<unsigned>(g0 & 0xFFFFFFFFull);
    if (k < UNIT_TAIL) {
        int t[TAIL];
#pragma unroll
        for (int i = 0; i < TAIL; ++i) t[i] = i < k ? i + 1 : 0;
        unit_eval_dispatch(k, Dm, t, best_c, best_r);
        seqs += k == 1 ? 1 : k == 2 ? 2 : k == 3 ? 6 : k == 4 ? 24 : 120;
    } else {
        const unsigned all = ((1u << k) - 1u) << 1;
        BlockRec rec;
        rec.have = false;
        if (!SETS || k < SET_UNITS_FROM) {
            // prefix units: the first q picks in the order of the unit index, then seven
            // 720-sequence parts (each of the seven next)
            const int q = k - UNIT_TAIL - 1;  // picks fixed by the unit index; -1 for k = 6
            const int nsub = q < 0 ? 1 : UNIT_TAIL + 1;
#pragma unroll 1
            for (unsigned u = ulo; u < uhi; ++u) {
                unsigned avail = all;
                uint32_t S = 0;
                int last = 0;
                if (q > 0) {
                    // factorial digits of u, position i in radix k - i
                    unsigned digits = 0, v = u;
                    for (int i = q - 1; i >= 0; --i) {
                        const unsigned r = static_cast<unsigned>(k - i);
                        digits |= (v % r) << (4 * i);
                        v /= r;
                    }
                    for (int i = 0; i < q; ++i) {
                        const int e = nth_bit(avail, static_cast<int>((digits >> (4 * i)) & 15u));
                        S += __ldg(Dm + last * DSTRIDE + e);
                        avail &= ~(1u << e);
                        last = e;
                    }
                }
                unsigned m = avail;
#pragma unroll 1
                for (int j = 0; j < nsub; ++j) {
                    int x = 0;
                    unsigned six = all;
                    uint32_t P = 0;
                    if (q >= 0) {
                        x = __ffs(m) - 1;
                        m &= m - 1;
                        six = avail & ~(1u << x);
                        P = S + __ldg(Dm + last * DSTRIDE + x);
                    }
                    unit720(Dm, P, x, six, (u * static_cast<unsigned>(nsub) + static_cast<unsigned>(j)) * 720u,
                            best_c, best_r, rec);
                }
            }
            seqs += static_cast<long long>(uhi - ulo) * 720 * nsub;
        } else {
        const int q = k - UNIT_TAIL - 1;  // picks before the last seven: -1 (k = 6) .. 5
        // prefix units (k <= SET_UNITS_FROM - 1): the first q picks in the order the unit index
        // gives, then seven parts (each of the seven next); set units (k >= SET_UNITS_FROM):
        // one part, walked after every ordering of the set
        const bool sets = SETS && k >= SET_UNITS_FROM;
        const int nf = sets && q == 5 ? 5 : 1;  // q = 5: the unit fixes the first pick too
        const int qr = !sets ? 0 : q == 5 ? 4 : q;  // picks whose orderings a set unit walks
        const int nperm = qr == 4 ? 24 : qr == 3 ? 6 : qr == 2 ? 2 : 1;
        const int lvl0 = nf == 5 ? 1 : 0;  // position of the first walked pick
        const int nsub = sets || q < 0 ? 1 : UNIT_TAIL + 1;
#pragma unroll 1
        for (unsigned u = ulo; u < uhi; ++u) {
            unsigned avail = all;  // picks after the prefix
            uint32_t S = 0;        // prefix cost (prefix units; set units: the fixed first pick)
            int last = 0;          // last prefix pick (0: the depot)
            unsigned base = 0;     // rank of the unit's first sequence, less the walked digits
            int xi = -1;           // set units: the index of x among the seven
            unsigned qpack = 0;    // set units: the walked picks in increasing order, 4 bits each
            if (!sets) {
                if (q > 0) {
                    // factorial digits of u, position i in radix k - i
                    unsigned digits = 0, v = u;
                    for (int i = q - 1; i >= 0; --i) {
                        const unsigned r = static_cast<unsigned>(k - i);
                        digits |= (v % r) << (4 * i);
                        v /= r;
                    }
                    for (int i = 0; i < q; ++i) {
                        const int e = nth_bit(avail, static_cast<int>((digits >> (4 * i)) & 15u));
                        S += __ldg(Dm + last * DSTRIDE + e);
                        avail &= ~(1u << e);
                        last = e;
                    }
                }
                base = u * static_cast<unsigned>(nsub) * 720u;
            } else {
                unsigned tt = u;
                const int fi = static_cast<int>(tt % static_cast<unsigned>(nf));
                tt /= static_cast<unsigned>(nf);
                xi = static_cast<int>(tt % 7u);
                tt /= 7u;
                // Q: the q-subset of colex rank tt of the picks (matrix indices 1..k), bits from
                // the top: each the largest c below the previous one with C(c, i) <= rr
                unsigned Q = 0, rr = tt;
                int c = k - 1;
                for (int i = q; i >= 1; --i, --c) {
                    while (tb.cb[6 * c + i] > rr) --c;  // ends by c = i - 1: C(i - 1, i) = 0
                    Q |= 2u << c;
                    rr -= tb.cb[6 * c + i];
                }
                avail = all & ~Q;
                base = static_cast<unsigned>(xi) * 720u;  // x: digit xi at position q
                if (nf == 5) {  // the fixed first pick: digit f - 1 at position 0
                    last = nth_bit(Q, fi);
                    Q &= ~(1u << last);
                    S = __ldg(Dm + last);
                    base += static_cast<unsigned>(last - 1) * tb.fact[k - 1];
                }
                int i = 0;
                for (unsigned m = Q; m; m &= m - 1, ++i) qpack |= static_cast<unsigned>(__ffs(m) - 1) << (4 * i);
            }
            const int f = nf == 5 ? last : 0;
            unsigned m = avail;
#pragma unroll 1
            for (int j = 0; j < nsub; ++j) {
                // one part: the six picks after x, its tables, then each walked ordering
                int x;
                if (sets) x = nth_bit(avail, xi);
                else if (q >= 0) {
                    x = __ffs(m) - 1;
                    m &= m - 1;
                } else x = 0;
                PartTab T;
                part_tables(Dm, x, x ? avail & ~(1u << x) : avail, T);
#pragma unroll 1
                for (int r = 0; r < nperm; ++r) {
                    const unsigned pat = qr > 0 ? tb.perm[24 * (qr - 1) + r] : 0u;
                    uint32_t P = S;
                    int lp = last;
                    unsigned rank = base + static_cast<unsigned>(j) * 720u;
                    for (int i = 0; i < qr; ++i) {
                        const unsigned nib = (pat >> (4 * i)) & 15u;
                        const int p = static_cast<int>((qpack >> (4 * (nib & 3u))) & 15u);
                        P += __ldg(Dm + lp * DSTRIDE + p);
                        lp = p;
                        // rank digit: the unused picks below p (picks 1..p-1 less those used)
                        const unsigned digit = static_cast<unsigned>(p - 1) - (nib >> 2) - (f != 0 && f < p ? 1u : 0u);
                        rank += digit * tb.fact[k - 1 - lvl0 - i];
                    }
                    if (x) P += __ldg(Dm + lp * DSTRIDE + x);
                    Tail6<0>::run(T.d6, T.t3f, T.xl, T.sp, P, rank, best_c, best_r, rec);
                }
            }
        }
        seqs += static_cast<long long>(uhi - ulo) * 720 * nsub * nperm;
        }
        if (rec.have) {
            // when another thread has meanwhile published a cheaper sequence of this order, this
            // range cannot hold the result: no search, nothing to publish
            if (static_cast<uint32_t>(__ldcg(out) >> 32) < best_c) return;
            best_r = rec.rank0 + static_cast<unsigned>(first_of_five(Dm, rec.acc, rec.sj, rec.five, best_c, rec.lo,
                                                                     rec.lo + SUB24));
        }
    }
    const unsigned long long packed = (static_cast<unsigned long long>(best_c) << 32) | best_r;
    if (packed < g0) atomicMin(out, packed);
}

constexpr int ENUM_THREADS = 128;
constexpr bool ENUM_GUIDED = true;  // chunk sizes shrink as the unit counter nears the end

// Two builds: SETS walks both unit kinds, the other prefix units only (without
// the set-unit code it keeps fewer registers live); the units kernel's flag in
// unit_ctr[1] says which one a call needs, and the other returns at once.
template <bool SETS>
__global__ void __launch_bounds__(ENUM_THREADS) enum_kernel(int32_t n, const int32_t* __restrict__ k_given, TourBufs t,
                                                            long long u_begin, long long u_end, int upt) {
    if ((__ldcg(t.unit_ctr + 1) != 0ull) != SETS) return;  // the other build runs this call
    __shared__ uint32_t s_cb[13 * 6], s_fact[13];
    __shared__ uint16_t s_perm[4 * 24];
    for (int i = threadIdx.x; i < 13 * 6; i += blockDim.x) {
        const int nn = i / 6, r = i % 6;
        uint32_t c = r > nn ? 0u : 1u;  // C(nn, r), multiplicative: exact at each step
        for (int j = 1; j <= r && j <= nn; ++j) c = c * static_cast<uint32_t>(nn - r + j) / static_cast<uint32_t>(j);
        s_cb[i] = c;
    }
    for (int i = threadIdx.x; i < 13; i += blockDim.x) {
        uint32_t f = 1;
        for (int j = 2; j <= i; ++j) f *= static_cast<uint32_t>(j);
        s_fact[i] = f;
    }
    for (int i = threadIdx.x; i < 4 * 24; i += blockDim.x) {
        const int nn = i / 24 + 1, r = i % 24;
        int nf = 1;
        for (int j = 2; j <= nn; ++j) nf *= j;
        unsigned pat = 0;
        if (r < nf) {
            unsigned used = 0;
            int rr = r, f = nf;
            for (int pos = 0; pos < nn; ++pos) {
                f /= nn - pos;
                const int d = rr / f;  // the d-th unused item
                rr -= d * f;
                const int item = nth_bit(~used & ((1u << nn) - 1u), d);
                pat |= static_cast<unsigned>(item | (__popc(used & ((1u << item) - 1u)) << 2)) << (4 * pos);
                used |= 1u << item;
            }
        }
        s_perm[i] = static_cast<uint16_t>(pat);
    }
    __syncthreads();
    const EnumTabs tb{s_cb, s_fact, s_perm};
    const int lane = threadIdx.x & 31;
    const long long total = min(u_end, static_cast<long long>(__ldcg(t.unit_off + n)));
    const long long warps = static_cast<long long>(gridDim.x) * (blockDim.x >> 5);
    long long seqs = 0;
    for (;;) {
        // guided claims: upt units per lane while at least 4 such chunks per warp remain, then
        // fewer, down to one, so that the last chunks end close together
        long long c0 = 0;
        int per = upt;
        if (lane == 0) {
            if (ENUM_GUIDED) {
                const long long left = total - u_begin - static_cast<long long>(__ldcg(t.unit_ctr));
                const long long fair = left / (32ll * 4ll * warps);
                per = fair >= upt ? upt : (fair < 1 ? 1 : static_cast<int>(fair));
            }
            c0 = static_cast<long long>(atomicAdd(t.unit_ctr, 32ull * static_cast<unsigned long long>(per)));
        }
        c0 = __shfl_sync(FULL_MASK, c0, 0) + u_begin;
        per = __shfl_sync(FULL_MASK, per, 0);
        if (c0 >= total) break;
        long long u = c0 + static_cast<long long>(lane) * per;
        const long long ue = min(u + per, total);
        while (u < ue) {
            // order holding unit u: last o with unit_off[o] <= u
            int lo = 0, hi = n - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (__ldg(t.unit_off + mid) <= u) lo = mid; else hi = mid - 1;
            }
            const int o = lo;
            const long long ob = __ldg(t.unit_off + o), oe = __ldg(t.unit_off + o + 1);
            const long long stop = min(ue, oe);
            const int k = order_k(t, k_given, o);
            enum_order_range<SETS>(t.D + static_cast<int64_t>(o) * DBLOCK, k, static_cast<unsigned>(u - ob),
                             static_cast<unsigned>(stop - ob), t.best + o, seqs, tb);
            u = stop;
        }
    }
    if (seqs) atomicAdd(reinterpret_cast<unsigned long long*>(t.seq_count), static_cast<unsigned long long>(seqs));
}

int tour_enum_blocks(int device) {
    int occ = 0, sms = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, enum_kernel<true>, ENUM_THREADS, 0);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    return (occ < 1 ? 1 : occ) * (sms < 1 ? 1 : sms);
}

cudaError_t tour_launch_enum(int32_t n, const int32_t* k_given, const TourBufs& t, long long u_begin, long long u_end,
                             int units_per_thread, int blocks, cudaStream_t s) {
    enum_kernel<false><<<blocks, ENUM_THREADS, 0, s>>>(n, k_given, t, u_begin, u_end, units_per_thread);
    enum_kernel<true><<<blocks, ENUM_THREADS, 0, s>>>(n, k_given, t, u_begin, u_end, units_per_thread);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a7: decode rank -> permutation, status
// ---------------------------------------------------------------------------

__global__ void finish_kernel(int32_t n, const int32_t* __restrict__ k_given, TourBufs t, int32_t* cost, int32_t* perm,
                              int perm_stride, int32_t* status) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const long long k64 = k_given ? k_given[o] : (t.offs[o + 1] - t.offs[o]);
    int32_t* pp = perm + (perm_stride > 0 ? static_cast<int64_t>(o) * perm_stride : t.offs[o]);
    long long kw = perm_stride > 0 ? min(k64, static_cast<long long>(perm_stride)) : k64;
    // an inconsistent pick range (only possible with device inputs) gets no perm writes
    if (perm_stride == 0 && (t.offs[o] < 0 || t.offs[o + 1] > t.offs[n])) kw = 0;
    int st = t.order_status[o];
    if (st == WR_ORDER_OK && (t.order_flags[o] & ORDER_FLAG_RANGE)) st = WR_ORDER_RANGE;
    uint32_t c = 0xFFFFFFFFu;
    unsigned rank = 0;
    if (st == WR_ORDER_OK) {
        const unsigned long long b = t.best[o];
        c = static_cast<uint32_t>(b >> 32);
        rank = static_cast<unsigned>(b & 0xFFFFFFFFull);
        if (c >= TOUR_CAP) st = WR_ORDER_UNREACHABLE;
    }
    status[o] = st;
    if (st != WR_ORDER_OK) {
        cost[o] = WR_INF;
        for (long long i = 0; i < kw; ++i) pp[i] = static_cast<int32_t>(i);
        return;
    }
    cost[o] = static_cast<int32_t>(c);
    const int k = static_cast<int>(k64);
    unsigned fact = 1;
    for (int i = 2; i < k; ++i) fact *= i;  // (k-1)!
    unsigned avail = (1u << k) - 1u;
    for (int i = 0; i < k; ++i) {
        const unsigned d = rank / fact;
        rank -= d * fact;
        if (k - 1 - i > 0) fact /= (k - 1 - i);
        const int e = nth_bit(avail, static_cast<int>(d));
        avail &= ~(1u << e);
        pp[i] = e;
    }
}

cudaError_t tour_launch_finish(int32_t n, const int32_t* k_given, const TourBufs& t, int32_t* cost, int32_t* perm,
                               int perm_stride, int32_t* status, cudaStream_t s) {
    finish_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, k_given, t, cost, perm, perm_stride, status);
    return cudaGetLastError();
}

}  // namespace wr
