// wr_tour_eval_static: tour evaluation over caller-given distance matrices
// that allocates no device memory.
//
// Some callers cannot call cudaMalloc: a serving process whose device memory
// belongs to another allocator (a framework's caching allocator or a fixed
// arena sized at start-up) must not have memory allocated, grown or freed
// behind that allocator's back, and a latency-critical loop cannot afford
// the device-wide synchronisation that cudaMalloc / cudaFree may imply.
// This entry point serves them: its scratch (the clamped matrices, unit
// offsets, per-order minima and counters) lives in the file-scope array
// below, which the CUDA runtime places on every device that loads the
// library and which stays there until the process exits.
#include <mutex>

#include "wr_internal.h"

namespace {

struct StaticScratch {
    uint32_t D[WR_STATIC_MAX_ORDERS * wr::DBLOCK];
    long long unit_off[WR_STATIC_MAX_ORDERS + 1];
    unsigned long long best[WR_STATIC_MAX_ORDERS];
    int32_t order_status[WR_STATIC_MAX_ORDERS];
    int32_t order_flags[WR_STATIC_MAX_ORDERS];
    unsigned long long unit_ctr[2];
    long long seq_count;
};

}  // namespace

// The scratch itself: about 2.9 MB per device (WR_STATIC_MAX_ORDERS = 4096 orders).
static __device__ __align__(256) unsigned char g_static_scratch[sizeof(StaticScratch)];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
StaticScratch* g_scratch_addr[MAX_DEVICES] = {nullptr};
int g_enum_blocks[MAX_DEVICES] = {0};

// With the device current: the device address of the scratch array (in host
// code its name is only a host-side stand-in).  A call outside stream capture
// looks the address up again every time, so a context that was torn down and
// created anew (cudaDeviceReset) never leaves a stale address behind; otherwise
// the address an earlier call found is used.
int setup_device(int dev, bool capturing, StaticScratch** out, int* blocks) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!capturing) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return WR_ECUDA;
        }
        if (!g_enum_blocks[dev]) g_enum_blocks[dev] = wr::tour_enum_blocks(dev);
        g_scratch_addr[dev] = static_cast<StaticScratch*>(p);
    }
    if (!g_scratch_addr[dev]) return WR_ECUDA;  // first call inside a capture: no address yet
    *out = g_scratch_addr[dev];
    *blocks = g_enum_blocks[dev];
    return WR_OK;
}

}  // namespace

extern "C" int wr_tour_eval_static(int32_t n_orders, const int32_t* k, const int32_t* D, int32_t* cost, int32_t* perm,
                                   int32_t* status, void* cuda_stream) {
    if (n_orders < 0 || n_orders > WR_STATIC_MAX_ORDERS) return WR_EINVAL;
    if (n_orders == 0) return WR_OK;
    if (!k || !D || !cost || !perm || !status) return WR_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return WR_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return WR_ECUDA;
    StaticScratch* s = nullptr;
    int blocks = 0;
    const int rc = setup_device(dev, cap != cudaStreamCaptureStatusNone, &s, &blocks);
    if (rc != WR_OK) return rc;
    wr::TourBufs tb{};
    tb.order_status = s->order_status;
    tb.order_flags = s->order_flags;
    tb.D = s->D;
    tb.unit_off = s->unit_off;
    tb.best = s->best;
    tb.unit_ctr = s->unit_ctr;
    tb.seq_count = &s->seq_count;
    // Every call reuses the same array.  The kernels below rewrite the
    // statuses, flags, clamped matrices, unit offsets, minima and the
    // scheduling counter before reading them; only the sequence counter is
    // cleared here.
    if (cudaMemsetAsync(&s->seq_count, 0, sizeof(long long), st) != cudaSuccess) return WR_ECUDA;
    int launches = 0;
    if (wr::tour_launch_prepare_given(n_orders, k, D, WR_MAX_K, tb, st) != cudaSuccess) return WR_ECUDA;
    if (wr::tour_launch_units(n_orders, k, tb, st, &launches) != cudaSuccess) return WR_ECUDA;
    if (wr::tour_launch_enum(n_orders, k, tb, 0, 1ll << 62, 4, blocks, st) != cudaSuccess) return WR_ECUDA;
    if (wr::tour_launch_finish(n_orders, k, tb, cost, perm, WR_MAX_K, status, st) != cudaSuccess) return WR_ECUDA;
    return WR_OK;
}
