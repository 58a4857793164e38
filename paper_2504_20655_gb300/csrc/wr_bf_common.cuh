// Shared pieces of the Bellman-Ford sweep kernels: launch parameters, the
// frontier list builder and cp.async helpers.
#pragma once

#include "wr_device.cuh"

namespace wr {

struct BfParams {
    DevGraph g;
    BfSegment seg;
    BfWork w;
};

// Node held by tile slot i < alen + blen of a run {a0, alen, b0, blen}.
__device__ __forceinline__ int run_node(const int4& rs, int i) { return i < rs.y ? rs.x + i : rs.z + (i - rs.y); }

// First row column of the segment's 32-source group g.
__device__ __forceinline__ int64_t seg_col0(const BfSegment& seg, int g) {
    return seg.gcol ? static_cast<int64_t>(__ldg(seg.gcol + g)) * 32 : static_cast<int64_t>(g) * 32;
}

__device__ __forceinline__ int segment_lanes(const BfSegment& seg) {
    const int n_src = seg.n_src_dev ? ld_l2(seg.n_src_dev) : seg.n_src_host;
    return min(max(n_src - seg.first, 0), seg.lanes);
}

// Append the items whose stamp (or, with nbrs, an in-neighbour run's stamp
// in the same group) equals match.
__device__ __forceinline__ void build_list(const BfParams& p, int G, int match, bool nbrs, int32_t* out,
                                           int32_t* count) {
    const int64_t n_items = static_cast<int64_t>(p.g.n_runs) * G;
    const int lane = threadIdx.x & 31;
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x; base < n_items;
         base += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t item = base + threadIdx.x;
        bool act = false;
        if (item < n_items) {
            act = ld_l2(p.w.stamp + item) == match;
            if (!act && nbrs) {
                const int r = static_cast<int>(item / G);
                const int g = static_cast<int>(item - static_cast<int64_t>(r) * G);
                const int q1 = __ldg(p.g.rin_ptr + r + 1);
                for (int q = __ldg(p.g.rin_ptr + r); q < q1; ++q) {
                    const int rr = __ldg(p.g.rin_list + q);
                    if (ld_l2(p.w.stamp + static_cast<int64_t>(rr) * G + g) == match) {
                        act = true;
                        break;
                    }
                }
            }
        }
        const unsigned m = __ballot_sync(FULL_MASK, act);
        if (m) {
            const int leader = __ffs(m) - 1;
            int pos = 0;
            if (lane == leader) pos = atomicAdd(count, __popc(m));
            pos = __shfl_sync(FULL_MASK, pos, leader);
            if (act) out[pos + __popc(m & lanemask_lt())] = static_cast<int32_t>(item);
        }
    }
}

// cp.async.wait_group takes an immediate: dispatch on the pending count.
__device__ __forceinline__ void cp_async_wait_pending(int n) {
    switch (n) {
        case 0: asm volatile("cp.async.wait_group 0;\n" ::: "memory"); break;
        case 1: asm volatile("cp.async.wait_group 1;\n" ::: "memory"); break;
        case 2: asm volatile("cp.async.wait_group 2;\n" ::: "memory"); break;
        case 3: asm volatile("cp.async.wait_group 3;\n" ::: "memory"); break;
        case 4: asm volatile("cp.async.wait_group 4;\n" ::: "memory"); break;
        case 5: asm volatile("cp.async.wait_group 5;\n" ::: "memory"); break;
        case 6: asm volatile("cp.async.wait_group 6;\n" ::: "memory"); break;
        case 7: asm volatile("cp.async.wait_group 7;\n" ::: "memory"); break;
        case 8: asm volatile("cp.async.wait_group 8;\n" ::: "memory"); break;
        case 9: asm volatile("cp.async.wait_group 9;\n" ::: "memory"); break;
        case 10: asm volatile("cp.async.wait_group 10;\n" ::: "memory"); break;
        case 11: asm volatile("cp.async.wait_group 11;\n" ::: "memory"); break;
        case 12: asm volatile("cp.async.wait_group 12;\n" ::: "memory"); break;
        case 13: asm volatile("cp.async.wait_group 13;\n" ::: "memory"); break;
        case 14: asm volatile("cp.async.wait_group 14;\n" ::: "memory"); break;
        case 15: asm volatile("cp.async.wait_group 15;\n" ::: "memory"); break;
        default: asm volatile("cp.async.wait_group 16;\n" ::: "memory"); break;
    }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async8_ca(void* smem, const void* gmem) {
    unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}

}  // namespace wr
