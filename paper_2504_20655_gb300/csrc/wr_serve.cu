// Serving loop (no counterpart in the paper): orders arrive over time and are
// routed exactly, with the graph and a cache of distance rows resident on the
// device.
//
// Continuous batching.  Whenever a slot is free, every order that has
// arrived so far (up to the slot's capacity and the cache's room) forms one
// batch.  A batch runs in two stages:
//   stage 1, on one stream shared by all batches (in admission order):
//     upload the batch, compute the rows of the sources the cache lacks
//     (multi-source Bellman-Ford straight into free cache columns), and
//     gather every order's distance matrix from the cache;
//   stage 2, on the slot's own stream: enumerate, reduce, decode, copy the
//     results back.
// Stage 2 of one batch overlaps stage 1 of the next and stage 2 of others.
// Stage 1 being in order on one stream is what makes eviction safe: a column
// group is only reused by a later batch, after every earlier gather that read
// it has run.
//
// Row cache.  A [V][C] matrix of distances (C columns, one per cached source,
// in groups of 32 that Bellman-Ford fills together), a host directory
// node -> column, and least-recently-used eviction of whole groups, never of
// a group the batch being admitted reads.  Admission stops growing a batch
// when its new sources would not fit the groups it may evict.
//
// The plain mode is the baseline the loop is measured against: every order
// alone, one at a time, with its own rows computed from scratch.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <thread>
#include <vector>

#include "wr_ctx.h"

using namespace wrc;

namespace {

// dir[nodes[i]] = cols[i]: directory entries of the sources a batch adds.
__global__ void dir_scatter_kernel(int32_t n, const int32_t* __restrict__ nodes, const int32_t* __restrict__ cols,
                                   int32_t* dir) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dir[nodes[i]] = cols[i];
}

template <class T>
T* host_alloc(size_t count) {
    void* p = nullptr;
    if (cudaHostAlloc(&p, count * sizeof(T) + 16, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return static_cast<T*>(p);
}

struct Slot {
    cudaStream_t s = nullptr;
    cudaEvent_t ev_in = nullptr, ev_done = nullptr;
    // pinned host staging: the batch in, the results out
    int64_t* h_offs = nullptr;
    int32_t *h_picks = nullptr, *h_status_in = nullptr, *h_miss = nullptr, *h_mcol = nullptr, *h_gcol = nullptr;
    int32_t *h_cost = nullptr, *h_perm = nullptr, *h_status = nullptr;
    DBuf offs, picks, miss, mcol, gcol, cost, perm, status;
    DBuf order_status, order_flags, D, unit_off, best, unit_ctr;
    std::vector<int32_t> orders;  // caller's indices of the batch's orders
    int32_t n = 0;
    int64_t np = 0;
    bool busy = false;
};

}  // namespace

struct wr_server {
    wr_ctx* c = nullptr;  // private context: graph copy, Bellman-Ford work buffers
    wr_serve_config cfg{};
    int32_t V = 0, C = 0, NG = 0;
    DBuf cache, dir;
    std::vector<int32_t> col_of;        // node -> cache column, -1 if absent
    std::vector<int32_t> group_nodes;   // NG * 32: the node in each column, -1 if free
    std::vector<int64_t> group_used;    // last batch that read or filled the group
    std::vector<int64_t> group_pin;     // batch being admitted that reads the group
    std::vector<int64_t> node_mark;     // batch that already listed the node as a new source
    cudaStream_t s0 = nullptr;          // stage 1 stream
    std::vector<Slot> slots;
    wr_serve_stats st{};
    int64_t batch_id = 0;
};

namespace {

void free_slot(Slot& sl) {
    if (sl.s) cudaStreamDestroy(sl.s);
    if (sl.ev_in) cudaEventDestroy(sl.ev_in);
    if (sl.ev_done) cudaEventDestroy(sl.ev_done);
    void* hp[] = {sl.h_offs, sl.h_picks, sl.h_status_in, sl.h_miss, sl.h_mcol, sl.h_gcol, sl.h_cost, sl.h_perm, sl.h_status};
    for (void* p : hp)
        if (p) cudaFreeHost(p);
    DBuf* db[] = {&sl.offs, &sl.picks, &sl.miss, &sl.mcol, &sl.gcol, &sl.cost, &sl.perm, &sl.status, &sl.order_status,
                  &sl.order_flags, &sl.D, &sl.unit_off, &sl.best, &sl.unit_ctr};
    for (DBuf* b : db) b->release();
}

int init_slot(Slot& sl, int32_t max_batch, int64_t max_picks, int32_t n_groups) {
    const size_t nb = static_cast<size_t>(max_batch), np = static_cast<size_t>(max_picks);
    const size_t ns = np + 1;  // distinct sources of a batch: depot + picks
    if (cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) != cudaSuccess) return WR_ECUDA;
    if (cudaEventCreateWithFlags(&sl.ev_in, cudaEventDisableTiming) != cudaSuccess) return WR_ECUDA;
    if (cudaEventCreateWithFlags(&sl.ev_done, cudaEventDisableTiming) != cudaSuccess) return WR_ECUDA;
    sl.h_offs = host_alloc<int64_t>(nb + 1);
    sl.h_picks = host_alloc<int32_t>(np);
    sl.h_status_in = host_alloc<int32_t>(nb);
    sl.h_miss = host_alloc<int32_t>(ns);
    sl.h_mcol = host_alloc<int32_t>(ns);
    sl.h_gcol = host_alloc<int32_t>(static_cast<size_t>(n_groups));
    sl.h_cost = host_alloc<int32_t>(nb);
    sl.h_perm = host_alloc<int32_t>(np);
    sl.h_status = host_alloc<int32_t>(nb);
    if (!sl.h_offs || !sl.h_picks || !sl.h_status_in || !sl.h_miss || !sl.h_mcol || !sl.h_gcol || !sl.h_cost ||
        !sl.h_perm || !sl.h_status)
        return WR_ENOMEM;
    RC(ensure(sl.offs, (nb + 1) * 8));
    RC(ensure(sl.picks, np * 4 + 4));
    RC(ensure(sl.miss, ns * 4));
    RC(ensure(sl.mcol, ns * 4));
    RC(ensure(sl.gcol, static_cast<size_t>(n_groups) * 4 + 4));
    RC(ensure(sl.cost, nb * 4));
    RC(ensure(sl.perm, np * 4 + 4));
    RC(ensure(sl.status, nb * 4));
    RC(ensure(sl.order_status, nb * 4 + 4));
    RC(ensure(sl.order_flags, nb * 4 + 4));
    RC(ensure(sl.D, nb * wr::DBLOCK * 4 + 4));
    RC(ensure(sl.unit_off, (nb + 1) * 8));
    RC(ensure(sl.best, nb * 8 + 8));
    RC(ensure(sl.unit_ctr, 16));
    return WR_OK;
}

wr::TourBufs slot_tour_bufs(wr_server* sv, Slot& sl) {
    wr::TourBufs tb{};
    tb.offs = sl.offs.as<int64_t>();
    tb.picks = sl.picks.as<int32_t>();
    tb.order_status = sl.order_status.as<int32_t>();
    tb.order_flags = sl.order_flags.as<int32_t>();
    tb.D = sl.D.as<uint32_t>();
    tb.unit_off = sl.unit_off.as<long long>();
    tb.best = sl.best.as<unsigned long long>();
    tb.unit_ctr = sl.unit_ctr.as<unsigned long long>();
    tb.seq_count = reinterpret_cast<long long*>(sv->c->stats.as<unsigned long long>() + 4);
    return tb;
}

double seconds_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

bool order_valid(const wr_server* sv, const int64_t* offs, const int32_t* picks, int32_t i) {
    const int64_t k = offs[i + 1] - offs[i];
    if (k < 1 || k > sv->c->cfg.max_k || k > WR_MAX_K) return false;  // the loop routes exhaustive orders
    for (int64_t q = offs[i]; q < offs[i + 1]; ++q)
        if (picks[q] < 0 || picks[q] >= sv->V) return false;
    return true;
}

// Enqueue both stages of the batch held in sl (host staging filled, n_miss new sources).
int launch_batch(wr_server* sv, Slot& sl, int32_t n_miss, int32_t n_new_groups) {
    wr_ctx* c = sv->c;
    cudaStream_t s0 = sv->s0;
    const size_t n = static_cast<size_t>(sl.n);
    RC(begin_call(c, s0));
    CK(cudaMemcpyAsync(sl.offs.p, sl.h_offs, (n + 1) * 8, cudaMemcpyHostToDevice, s0));
    if (sl.np) CK(cudaMemcpyAsync(sl.picks.p, sl.h_picks, static_cast<size_t>(sl.np) * 4, cudaMemcpyHostToDevice, s0));
    CK(cudaMemcpyAsync(sl.order_status.p, sl.h_status_in, n * 4, cudaMemcpyHostToDevice, s0));
    CK(cudaMemsetAsync(sl.order_flags.p, 0, n * 4, s0));
    if (n_miss > 0) {
        CK(cudaMemcpyAsync(sl.miss.p, sl.h_miss, static_cast<size_t>(n_miss) * 4, cudaMemcpyHostToDevice, s0));
        CK(cudaMemcpyAsync(sl.mcol.p, sl.h_mcol, static_cast<size_t>(n_miss) * 4, cudaMemcpyHostToDevice, s0));
        CK(cudaMemcpyAsync(sl.gcol.p, sl.h_gcol, static_cast<size_t>(n_new_groups) * 4, cudaMemcpyHostToDevice, s0));
        dir_scatter_kernel<<<(n_miss + 255) / 256, 256, 0, s0>>>(n_miss, sl.miss.as<int32_t>(), sl.mcol.as<int32_t>(),
                                                                   sv->dir.as<int32_t>());
        CK(cudaGetLastError());
        wr::BfSegment seg;
        seg.rows = sv->cache.as<uint32_t>();
        seg.ld = sv->C;
        seg.src = sl.miss.as<int32_t>();
        seg.n_src_dev = nullptr;
        seg.n_src_host = n_miss;
        seg.first = 0;
        seg.lanes = n_new_groups * 32;
        seg.gcol = sl.gcol.as<int32_t>();
        RC(ensure_bf(c, seg.lanes, false));
        RC(run_bf_segment(c, seg, s0));
        sv->st.bf_launches += 1;
    }
    wr::TourBufs tb = slot_tour_bufs(sv, sl);
    wr::BfSegment all;
    all.rows = sv->cache.as<uint32_t>();
    all.ld = sv->C;
    all.src = nullptr;
    all.n_src_dev = nullptr;
    all.n_src_host = sv->C;
    all.first = 0;
    all.lanes = sv->C;
    CK(wr::tour_launch_gather(sl.n, tb, c->dg.depot, sv->dir.as<int32_t>(), all, c->route_mode == WR_ROUTE_OPEN, s0));
    CK(cudaEventRecord(sl.ev_in, s0));
    // stage 2
    CK(cudaStreamWaitEvent(sl.s, sl.ev_in, 0));
    RC(run_tours(c, sl.n, nullptr, tb, sl.cost.as<int32_t>(), sl.perm.as<int32_t>(), 0, sl.status.as<int32_t>(), sl.s));
    CK(cudaMemcpyAsync(sl.h_cost, sl.cost.p, n * 4, cudaMemcpyDeviceToHost, sl.s));
    CK(cudaMemcpyAsync(sl.h_status, sl.status.p, n * 4, cudaMemcpyDeviceToHost, sl.s));
    if (sl.np) CK(cudaMemcpyAsync(sl.h_perm, sl.perm.p, static_cast<size_t>(sl.np) * 4, cudaMemcpyDeviceToHost, sl.s));
    CK(cudaEventRecord(sl.ev_done, sl.s));
    sl.busy = true;
    return WR_OK;
}

// Admit arrived orders [*next, ...) into slot sl; returns WR_OK with sl.n = 0 if none.
int admit(wr_server* sv, Slot& sl, int32_t n_total, const double* arrival, double now, const int64_t* offs,
          const int32_t* picks, int32_t* next) {
    const int64_t bid = ++sv->batch_id;
    const int32_t depot = sv->c->dg.depot;
    std::vector<int32_t> miss;
    int32_t pinned = 0;
    sl.orders.clear();
    sl.n = 0;
    sl.np = 0;
    sl.h_offs[0] = 0;
    auto pin = [&](int32_t node) {
        const int32_t g = sv->col_of[node] / 32;
        if (sv->group_pin[g] != bid) {
            sv->group_pin[g] = bid;
            ++pinned;
        }
        sv->group_used[g] = bid;
    };
    while (*next < n_total && arrival[*next] <= now && sl.n < sv->cfg.max_batch) {
        const int32_t i = *next;
        const int64_t k = offs[i + 1] - offs[i];
        if (k < 0 || sl.np + k > sv->cfg.max_batch_picks) break;
        const bool ok = order_valid(sv, offs, picks, i);
        if (ok) {
            // the order's sources the cache lacks, and the groups it reads
            int32_t fresh = 0;
            for (int64_t q = -1; q < k; ++q) {
                const int32_t node = q < 0 ? depot : picks[offs[i] + q];
                if (sv->col_of[node] < 0 && sv->node_mark[node] != bid) ++fresh;
            }
            int32_t pins_new = 0;
            for (int64_t q = -1; q < k; ++q) {
                const int32_t node = q < 0 ? depot : picks[offs[i] + q];
                if (sv->col_of[node] >= 0 && sv->group_pin[sv->col_of[node] / 32] != bid) ++pins_new;
            }
            const int64_t groups_needed = (static_cast<int64_t>(miss.size()) + fresh + 31) / 32;
            if (groups_needed > sv->NG - pinned - pins_new) {
                if (sl.n == 0) return WR_ENOMEM;  // one order's sources exceed the cache
                break;
            }
            for (int64_t q = -1; q < k; ++q) {
                const int32_t node = q < 0 ? depot : picks[offs[i] + q];
                if (sv->col_of[node] >= 0) {
                    pin(node);
                    sv->st.cache_hits += 1;
                } else if (sv->node_mark[node] != bid) {
                    sv->node_mark[node] = bid;
                    miss.push_back(node);
                } else {
                    sv->st.cache_hits += 1;  // listed by an earlier order of this batch
                }
            }
        }
        for (int64_t q = 0; q < k; ++q) sl.h_picks[sl.np + q] = picks[offs[i] + q];
        sl.np += k;
        sl.h_offs[sl.n + 1] = sl.np;
        sl.h_status_in[sl.n] = ok ? WR_ORDER_OK : WR_ORDER_BAD;
        sl.orders.push_back(i);
        ++sl.n;
        ++*next;
    }
    if (sl.n == 0) return WR_OK;
    // columns for the new sources: least recently used groups this batch does not read
    const int32_t n_miss = static_cast<int32_t>(miss.size());
    const int32_t n_groups = (n_miss + 31) / 32;
    std::vector<int32_t> cand;
    cand.reserve(sv->NG);
    for (int32_t g = 0; g < sv->NG; ++g)
        if (sv->group_pin[g] != bid) cand.push_back(g);
    if (static_cast<int32_t>(cand.size()) < n_groups) return WR_EINTERNAL;  // admission guarantees room
    std::partial_sort(cand.begin(), cand.begin() + n_groups, cand.end(),
                      [&](int32_t a, int32_t b) { return sv->group_used[a] < sv->group_used[b]; });
    for (int32_t q = 0; q < n_groups; ++q) {
        const int32_t g = cand[q];
        bool had = false;
        for (int32_t j = 0; j < 32; ++j) {
            int32_t& old = sv->group_nodes[g * 32 + j];
            if (old >= 0) {
                if (sv->col_of[old] == g * 32 + j) sv->col_of[old] = -1;
                had = true;
            }
            old = -1;
        }
        if (had) sv->st.evicted_groups += 1;
        sv->group_used[g] = bid;
        sv->group_pin[g] = bid;
        sl.h_gcol[q] = g;
    }
    for (int32_t b = 0; b < n_miss; ++b) {
        const int32_t col = sl.h_gcol[b / 32] * 32 + (b % 32);
        sl.h_miss[b] = miss[b];
        sl.h_mcol[b] = col;
        sv->col_of[miss[b]] = col;
        sv->group_nodes[col] = miss[b];
    }
    sv->st.rows_computed += n_miss;
    sv->st.batches += 1;
    sv->st.orders += sl.n;
    return launch_batch(sv, sl, n_miss, n_groups);
}

// Results of a finished slot into the caller's arrays.
void retire(Slot& sl, const int64_t* offs, int32_t* cost, int32_t* perm, int32_t* status, double* done_s, double now) {
    for (int32_t j = 0; j < sl.n; ++j) {
        const int32_t i = sl.orders[j];
        cost[i] = sl.h_cost[j];
        status[i] = sl.h_status[j];
        const int64_t k = offs[i + 1] - offs[i];
        if (perm)
            for (int64_t q = 0; q < k; ++q) perm[offs[i] + q] = sl.h_perm[sl.h_offs[j] + q];
        done_s[i] = now;
    }
    sl.busy = false;
}

}  // namespace

extern "C" {

void wr_serve_destroy(wr_server* sv) {
    if (!sv) return;
    if (sv->c) cudaSetDevice(sv->c->device);
    cudaDeviceSynchronize();
    for (Slot& sl : sv->slots) free_slot(sl);
    if (sv->s0) cudaStreamDestroy(sv->s0);
    sv->cache.release();
    sv->dir.release();
    if (sv->c) wr_destroy(sv->c);
    delete sv;
}

int wr_serve_create(wr_ctx* parent, const wr_serve_config* cfg, wr_server** out) {
    if (!parent || !cfg || !out) return WR_EINVAL;
    *out = nullptr;
    if (!parent->has_graph) return WR_ENOGRAPH;
    if (parent->cluster_m > 0) return WR_EINVAL;  // the loop routes exactly
    if (!cfg->plain && (cfg->max_batch < 1 || cfg->max_batch_picks < WR_MAX_K || cfg->n_slots < 1 || cfg->n_slots > 8))
        return WR_EINVAL;
    RC(set_device(parent));
    wr_server* sv = new (std::nothrow) wr_server();
    if (!sv) return WR_ENOMEM;
    sv->cfg = *cfg;
    if (cfg->plain) {
        sv->cfg.max_batch = 1;
        sv->cfg.max_batch_picks = WR_MAX_K;
        sv->cfg.n_slots = 1;
    }
    int rc = wr_create(&parent->cfg, &sv->c);
    if (rc == WR_OK) {
        sv->c->tune = parent->tune;
        sv->c->route_mode = parent->route_mode;
        sv->c->tune.enum_max_units_per_launch = 0;  // no host syncs inside a batch
        if (sv->c->cfg.max_k > WR_MAX_K) sv->c->cfg.max_k = WR_MAX_K;  // the loop routes exhaustive orders
        sv->c->hg = parent->hg;
        rc = finish_graph(sv->c);
    }
    if (rc == WR_OK) {
        sv->c->untimed = true;
        sv->V = sv->c->dg.V;
        if (!cfg->plain) {
            const uint64_t per_col = static_cast<uint64_t>(sv->V) * 4ull;
            uint64_t cols = cfg->cache_bytes / per_col / 32 * 32;
            if (cols > (1u << 20)) cols = 1u << 20;
            if (cols < 512) rc = WR_ENOMEM;  // 16 groups: any one order (<= 13 sources) always fits
            sv->C = static_cast<int32_t>(cols);
            sv->NG = sv->C / 32;
            if (rc == WR_OK) rc = ensure(sv->cache, static_cast<size_t>(cols) * per_col);
            if (rc == WR_OK) rc = ensure(sv->dir, static_cast<size_t>(sv->V) * 4);
            sv->col_of.assign(static_cast<size_t>(sv->V), -1);
            sv->node_mark.assign(static_cast<size_t>(sv->V), 0);
            sv->group_nodes.assign(static_cast<size_t>(sv->C), -1);
            sv->group_used.assign(static_cast<size_t>(sv->NG), 0);
            sv->group_pin.assign(static_cast<size_t>(sv->NG), 0);
        }
    }
    if (rc == WR_OK && !cfg->plain) {
        // frontier arrays for the largest set of new sources one batch can bring
        const int64_t groups = std::min<int64_t>((sv->cfg.max_batch_picks + 1 + 31) / 32, sv->NG);
        rc = ensure_bf(sv->c, static_cast<int32_t>(groups) * 32, false);
    }
    if (rc == WR_OK && cudaStreamCreateWithFlags(&sv->s0, cudaStreamNonBlocking) != cudaSuccess) rc = WR_ECUDA;
    if (rc == WR_OK) {
        sv->slots.resize(static_cast<size_t>(sv->cfg.n_slots));
        for (Slot& sl : sv->slots) {
            rc = init_slot(sl, sv->cfg.max_batch, sv->cfg.max_batch_picks, std::max(sv->NG, 1));
            if (rc != WR_OK) break;
        }
    }
    if (rc != WR_OK) {
        cudaGetLastError();
        wr_serve_destroy(sv);
        return rc;
    }
    *out = sv;
    return WR_OK;
}

int wr_serve_run(wr_server* sv, int32_t n, const double* arrival, const int64_t* offs, const int32_t* picks,
                 int32_t* cost, int32_t* perm, int32_t* status, double* done_s) {
    if (!sv || n < 0 || (n > 0 && (!arrival || !offs || !cost || !status || !done_s))) return WR_EINVAL;
    if (n > 0 && offs[0] != 0) return WR_EINVAL;
    for (int32_t i = 0; i < n; ++i) {
        if (offs[i + 1] < offs[i] || offs[i + 1] - offs[i] > sv->cfg.max_batch_picks) return WR_EINVAL;
        if (i > 0 && arrival[i] < arrival[i - 1]) return WR_EINVAL;
    }
    if (n > 0 && offs[n] > 0 && (!picks || !perm)) return WR_EINVAL;
    RC(set_device(sv->c));
    std::memset(&sv->st, 0, sizeof(sv->st));
    const auto t0 = std::chrono::steady_clock::now();
    int32_t next = 0, done = 0;
    int rc = WR_OK;
    while (done < n && rc == WR_OK) {
        bool progressed = false;
        for (Slot& sl : sv->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.ev_done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                rc = WR_ECUDA;
                break;
            }
            retire(sl, offs, cost, perm, status, done_s, seconds_since(t0));
            done += sl.n;
            progressed = true;
        }
        if (rc != WR_OK) break;
        const double now = seconds_since(t0);
        if (next < n && arrival[next] <= now) {
            for (Slot& sl : sv->slots) {
                if (sl.busy || next >= n || arrival[next] > now) continue;
                if (sv->cfg.plain) {
                    // the baseline: this order alone, its own rows from scratch
                    const int32_t i = next++;
                    const int64_t k = offs[i + 1] - offs[i];
                    sl.n = 1;
                    sl.np = k;
                    sl.orders.assign(1, i);
                    sl.h_offs[0] = 0;
                    sl.h_offs[1] = k;
                    for (int64_t q = 0; q < k; ++q) sl.h_picks[q] = picks[offs[i] + q];
                    CK(cudaMemcpyAsync(sl.offs.p, sl.h_offs, 16, cudaMemcpyHostToDevice, sl.s));
                    if (k) CK(cudaMemcpyAsync(sl.picks.p, sl.h_picks, static_cast<size_t>(k) * 4, cudaMemcpyHostToDevice, sl.s));
                    rc = begin_call(sv->c, sl.s);
                    if (rc == WR_OK)
                        rc = enqueue_route(sv->c, 1, sl.offs.as<int64_t>(), sl.picks.as<int32_t>(), k,
                                           sl.cost.as<int32_t>(), sl.perm.as<int32_t>(), sl.status.as<int32_t>(), sl.s);
                    if (rc != WR_OK) break;
                    CK(cudaMemcpyAsync(sl.h_cost, sl.cost.p, 4, cudaMemcpyDeviceToHost, sl.s));
                    CK(cudaMemcpyAsync(sl.h_status, sl.status.p, 4, cudaMemcpyDeviceToHost, sl.s));
                    if (k) CK(cudaMemcpyAsync(sl.h_perm, sl.perm.p, static_cast<size_t>(k) * 4, cudaMemcpyDeviceToHost, sl.s));
                    CK(cudaEventRecord(sl.ev_done, sl.s));
                    sl.busy = true;
                    sv->st.orders += 1;
                    sv->st.batches += 1;
                    sv->st.rows_computed += k + 1;
                } else {
                    rc = admit(sv, sl, n, arrival, now, offs, picks, &next);
                    if (rc != WR_OK) break;
                }
                progressed = true;
            }
        }
        if (!progressed) std::this_thread::yield();
    }
    if (rc != WR_OK) {
        cudaDeviceSynchronize();
        for (Slot& sl : sv->slots) sl.busy = false;
        cudaGetLastError();
        return rc;
    }
    sv->st.wall_s = seconds_since(t0);
    CK(cudaStreamSynchronize(sv->s0));
    return take_device_error(sv->c);
}

int wr_serve_get_stats(wr_server* sv, wr_serve_stats* out) {
    if (!sv || !out) return WR_EINVAL;
    *out = sv->st;
    return WR_OK;
}

}  // extern "C"
