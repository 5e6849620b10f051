// kpx_batch.cu -- one Kino-PAX+ iteration for many independent problems at
// once: every phase is one launch over the whole batch (propagate and append
// once per dynamics class), so the launch count per iteration does not grow
// with the number of problems.
//
// Each problem keeps its own workspace laid out exactly as a single planner's,
// its own counters, Philox keys, tile words and propagate order; work units (32-slot chunks,
// regions, scan tiles, winners, prune tiles) are numbered across problems by
// prefix sums recomputed every iteration, and a unit finds its problem by a
// binary search.  Nothing couples two problems, so each result is the one the
// problem would get alone.
#include <cuda_runtime.h>

#include "kpx_phases.cuh"

namespace kpx {

namespace {

// largest p in [lo, hi) with prefix[p] <= v (that problem owns unit v)
__device__ __forceinline__ int find_problem(const int64_t* __restrict__ prefix, int lo, int hi, int64_t v) {
    int a = lo, b = hi - 1;
    while (a < b) {
        const int mid = (a + b + 1) >> 1;
        if (prefix[mid] <= v)
            a = mid;
        else
            b = mid - 1;
    }
    return a;
}

// block-wide running prefix: out[p] = sum of vals before p, out[B] = total
template <typename F>
__device__ void block_prefix(int B, int64_t* out, F value_of) {
    __shared__ uint32_t s_warp[32];
    __shared__ unsigned long long s_carry;
    if (threadIdx.x == 0) s_carry = 0ull;
    __syncthreads();
    for (int base = 0; base < B; base += 1024) {
        const int p = base + threadIdx.x;
        const uint32_t v = p < B ? (uint32_t)value_of(p) : 0u;
        uint32_t agg;
        const uint32_t excl = block_exclusive_scan<1024>(v, agg, s_warp);
        if (p < B) out[p] = (int64_t)(s_carry + excl);
        __syncthreads();
        if (threadIdx.x == 0) s_carry += agg;
        __syncthreads();
    }
    if (threadIdx.x == 0) out[B] = (int64_t)s_carry;
    __syncthreads();
}

// per-problem counters, then the chunk and scan-tile numbering
__global__ void __launch_bounds__(1024) k_b_begin(BatchParams BP) {
    for (int p = threadIdx.x; p < BP.B; p += blockDim.x) begin_counters(BP.Ps[p], BP.Ps[p].hdr);
    __syncthreads();
    block_prefix(BP.B, BP.chunk_prefix, [&](int p) {  // each problem's propagate units
        return propagate_units(BP.Ps[p].hdr->n_slots, BP.Ps[p].slot_order != nullptr);
    });
    block_prefix(BP.B, BP.order_prefix, [&](int p) {
        const DevParams& P = BP.Ps[p];
        return P.hdr->active && P.slot_order ? (P.hdr->n_slots + ORDER_CHUNK - 1) / ORDER_CHUNK : (int64_t)0;
    });
    block_prefix(BP.B, BP.scan_prefix, [&](int p) {
        const int64_t words = (BP.Ps[p].hdr->n_slots + 31) / 32;
        return (words + WIN_TILE_WORDS - 1) / WIN_TILE_WORDS;
    });
    if (threadIdx.x == 0) {
        for (int c = 0; c < 6; ++c) BP.bh->prop_ticket[c] = 0ull;
        BP.bh->scan_ticket = 0u;
    }
}

// region snapshot where the capacity rule could trigger (grid.y = problem),
// and the propagate order of every problem's slots (each 128-slot chunk
// sorted by the single planner's key): the chunks of all problems are
// spread over all warps of the grid, so that a few large problems (a
// request loop's) do not wait on their own blocks alone
__global__ void k_b_snapshot(BatchParams BP) {
    const int64_t total = BP.order_prefix[BP.B];
    const int64_t warps = ((int64_t)gridDim.x * gridDim.y * blockDim.x) >> 5;
    const int64_t w0 = (((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    for (int64_t g = w0; g < total; g += warps) {
        const int p = find_problem(BP.order_prefix, 0, BP.B, g);
        const DevParams& Q = BP.Ps[p];
        const kpx_device_header* HQ = Q.hdr;
        const int64_t c = g - BP.order_prefix[p];
        if (Q.m == 4)
            order_chunk<4>(Q, va_current(Q, HQ), HQ->lambda, (uint32_t)HQ->iter, HQ->n_slots, c);
        else
            order_chunk<3>(Q, va_current(Q, HQ), HQ->lambda, (uint32_t)HQ->iter, HQ->n_slots, c);
    }
    const DevParams& P = BP.Ps[blockIdx.y];
    if (!begin_needs_snapshot(P, P.hdr)) return;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < P.R; r += gridDim.x * blockDim.x)
        P.region_snap[r] = P.region_key[r];
}

template <int DYN>
struct BatchPropOccupancy {
    static constexpr int blocks = DYN == KPX_QUAD12 ? 3 : 4;
};

// propagate over the chunks of the class's problems [lo, hi)
template <int DYN, int INTEG>
__global__ void __launch_bounds__(PROP_THREADS, BatchPropOccupancy<DYN>::blocks) k_b_propagate(BatchParams BP) {
    const int64_t c_lo = BP.chunk_prefix[BP.lo], c_hi = BP.chunk_prefix[BP.hi];
    const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    int64_t chunk = c_lo + (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const kpx_debug_records no_rec{};
    int cur = -1;
    uint32_t steps = 0, tests = 0, n_valid = 0;
    while (chunk < c_hi) {
        const int p = find_problem(BP.chunk_prefix, BP.lo, BP.hi, chunk);
        const DevParams& P = BP.Ps[p];
        if (p != cur) {
            if (cur >= 0) flush_propagate_counters(BP.Ps[cur].hdr, steps, tests, n_valid);
            cur = p;
        }
        const kpx_device_header* H = P.hdr;
        const bool early = (P.flags & KPX_FLAG_EARLY_REJECT) != 0;
        const int64_t unit = propagate_unit_chunk(chunk - BP.chunk_prefix[p], H->n_slots, P.slot_order != nullptr);
        propagate_chunk<DYN, INTEG>(P, H->n_slots, H->lambda, (uint32_t)H->iter, va_current(P, H), early, unit,
                                    no_rec, 0, steps, tests, n_valid, P.slot_order);
        unsigned long long t = 0ull;
        if ((threadIdx.x & 31) == 0) t = atomicAdd(&BP.bh->prop_ticket[BP.cls], 1ull);
        chunk = c_lo + n_warps + (int64_t)__shfl_sync(FULL, t, 0);
    }
    if (cur >= 0) flush_propagate_counters(BP.Ps[cur].hdr, steps, tests, n_valid);
}

__global__ void k_b_mark(BatchParams BP) {
    const DevParams& P = BP.Ps[blockIdx.y];
    if (!P.hdr->active) return;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < P.R; r += gridDim.x * blockDim.x) mark_region(P, r);
}

__global__ void __launch_bounds__(WIN_THREADS) k_b_scan(BatchParams BP) {
    __shared__ uint32_t s_tile, s_prefix;
    __shared__ uint32_t s_warp[WIN_THREADS / 32];
    const int64_t total = BP.scan_prefix[BP.B];
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&BP.bh->scan_ticket, 1u);
        __syncthreads();
        const int64_t t = s_tile;
        __syncthreads();
        if (t >= total) return;
        const int p = find_problem(BP.scan_prefix, 0, BP.B, t);
        const DevParams& P = BP.Ps[p];
        kpx_device_header* H = P.hdr;
        const int64_t n_tiles = BP.scan_prefix[p + 1] - BP.scan_prefix[p];
        scan_tile(P, H, (uint32_t)(t - BP.scan_prefix[p]), n_tiles, (H->n_slots + 31) / 32, s_warp, s_prefix);
    }
}

// winners kept (capacity rule), then the winner and prune-tile numbering
__global__ void __launch_bounds__(1024) k_b_prefix(BatchParams BP) {
    for (int p = threadIdx.x; p < BP.B; p += blockDim.x) {
        kpx_device_header* H = BP.Ps[p].hdr;
        if (!H->active) continue;
        const int W = H->n_win;
        const int room = BP.Ps[p].N - H->n_nodes;
        const int kept = W < room ? W : room;
        H->n_kept = kept;
        if (W > kept) set_status(H, KPX_TREE_FULL);
    }
    __syncthreads();
    block_prefix(BP.B, BP.win_prefix, [&](int p) {
        const kpx_device_header* H = BP.Ps[p].hdr;
        return H->active ? (int64_t)H->n_win : (int64_t)0;
    });
    block_prefix(BP.B, BP.prune_prefix, [&](int p) {
        const kpx_device_header* H = BP.Ps[p].hdr;
        return H->active ? (int64_t)((H->n_nodes + H->n_kept + PRUNE_TILE - 1) / PRUNE_TILE) : (int64_t)0;
    });
    if (threadIdx.x == 0) BP.bh->prune_ticket = 0u;
}

template <int DYN, int INTEG>
__global__ void __launch_bounds__(128) k_b_append(BatchParams BP) {
    const int64_t w_lo = BP.win_prefix[BP.lo], w_hi = BP.win_prefix[BP.hi];
    for (int64_t g = w_lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < w_hi;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int p = find_problem(BP.win_prefix, BP.lo, BP.hi, g);
        const DevParams& P = BP.Ps[p];
        kpx_device_header* H = P.hdr;
        append_winner<DYN, INTEG>(P, H, (int)(g - BP.win_prefix[p]), H->n_kept, H->n_nodes, H->lambda,
                                  (uint32_t)H->iter, va_current(P, H));
    }
}

__global__ void __launch_bounds__(PRUNE_THREADS) k_b_prune(BatchParams BP) {
    __shared__ uint32_t s_tile, s_prefix;
    __shared__ int32_t s_parent[PRUNE_TILE];
    __shared__ uint8_t s_set[PRUNE_TILE];
    __shared__ uint8_t s_icount[PRUNE_TILE];
    __shared__ uint32_t s_counts[PRUNE_ROUND_WARPS];
    const int64_t total_tiles = BP.prune_prefix[BP.B];
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&BP.bh->prune_ticket, 1u);
        __syncthreads();
        const int64_t t = s_tile;
        __syncthreads();
        if (t >= total_tiles) return;
        const int p = find_problem(BP.prune_prefix, 0, BP.B, t);
        const DevParams& P = BP.Ps[p];
        kpx_device_header* H = P.hdr;
        const int n_old = H->n_nodes;
        const int n_tiles = (int)(BP.prune_prefix[p + 1] - BP.prune_prefix[p]);
        int cA = 0, cI = 0, cT = 0;
        prune_tile(P, H, (uint32_t)(t - BP.prune_prefix[p]), n_tiles, n_old, n_old + H->n_kept, (uint32_t)H->epoch,
                   va_following(P, H), s_parent, s_set, s_icount, s_counts, s_prefix, cA, cI, cT);
        flush_prune_counters(H, cA, cI, cT);
    }
}

__global__ void k_b_end(BatchParams BP) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < BP.B) end_counters(BP.Ps[p], BP.Ps[p].hdr);
}

__global__ void k_b_poll(BatchParams BP) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= BP.B) return;
    const kpx_device_header* H = BP.Ps[p].hdr;
    SlotState st;
    st.status = BP.Ps[p].iter_limit < 0 ? -1 : H->status;
    st.iter = H->iter;
    st.n_nodes = H->n_nodes;
    st.first_solution_iter = H->first_solution_iter;
    st.goal_key = H->goal_key;
    st.t_start_ns = H->t_start_ns;
    st.t_first_solution_ns = H->first_solution_iter >= 0 ? H->t_first_solution_ns : 0ull;
    st.t_last_ns = H->t_last_ns;
    st.t_poll_ns = globaltimer_ns();
    BP.slots[p] = st;
}

int b_sm_count() {
    static int cached[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = sms > 0 ? sms : 1;
    }
    return cached[dev];
}

template <int DYN, int INTEG>
cudaError_t launch_b_propagate_t(const BatchParams& BP, int bps, cudaStream_t s) {
    static int per_sm = 0;
    if (!per_sm) {
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_b_propagate<DYN, INTEG>, PROP_THREADS, 0);
        per_sm = v < 1 ? 1 : v;
    }
    const int use = bps > 0 && bps < per_sm ? bps : per_sm;
    k_b_propagate<DYN, INTEG><<<b_sm_count() * use, PROP_THREADS, 0, s>>>(BP);
    return cudaGetLastError();
}

template <int DYN, int INTEG>
cudaError_t launch_b_append_t(const BatchParams& BP, cudaStream_t s) {
    k_b_append<DYN, INTEG><<<b_sm_count() * 4, 128, 0, s>>>(BP);
    return cudaGetLastError();
}

#define KPX_CLASS_DISPATCH(FN, KIND, ...)                                          \
    switch (KIND) {                                                                \
        case KPX_DI6 * 2 + KPX_EULER: return FN<KPX_DI6, KPX_EULER>(__VA_ARGS__);         \
        case KPX_DI6 * 2 + KPX_RK4: return FN<KPX_DI6, KPX_RK4>(__VA_ARGS__);             \
        case KPX_DUBINS6 * 2 + KPX_EULER: return FN<KPX_DUBINS6, KPX_EULER>(__VA_ARGS__); \
        case KPX_DUBINS6 * 2 + KPX_RK4: return FN<KPX_DUBINS6, KPX_RK4>(__VA_ARGS__);     \
        case KPX_QUAD12 * 2 + KPX_EULER: return FN<KPX_QUAD12, KPX_EULER>(__VA_ARGS__);   \
        case KPX_QUAD12 * 2 + KPX_RK4: return FN<KPX_QUAD12, KPX_RK4>(__VA_ARGS__);       \
        default: return cudaErrorInvalidValue;                                    \
    }

}  // namespace

cudaError_t launch_batch_poll(const BatchParams& base, cudaStream_t s) {
    k_b_poll<<<(base.B + 255) / 256, 256, 0, s>>>(base);
    return cudaGetLastError();
}

// One batched iteration: begin, snapshot, propagate per class, mark, scan,
// prefix, append per class, prune, end.
cudaError_t launch_batch_iteration(const BatchParams& base, int n_classes, const int* cls_kind, const int* cls_lo,
                                   const int* cls_hi, const int* cls_bps, cudaStream_t s) {
    k_b_begin<<<1, 1024, 0, s>>>(base);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_b_snapshot<<<dim3(8, base.B), 256, 0, s>>>(base);
    for (int c = 0; c < n_classes && e == cudaSuccess; ++c) {
        BatchParams bp = base;
        bp.lo = cls_lo[c];
        bp.hi = cls_hi[c];
        bp.cls = c;
        e = [&]() -> cudaError_t { KPX_CLASS_DISPATCH(launch_b_propagate_t, cls_kind[c], bp, cls_bps[c], s); }();
    }
    if (e != cudaSuccess) return e;
    k_b_mark<<<dim3(8, base.B), 256, 0, s>>>(base);
    k_b_scan<<<b_sm_count() * 8, WIN_THREADS, 0, s>>>(base);
    k_b_prefix<<<1, 1024, 0, s>>>(base);
    for (int c = 0; c < n_classes && e == cudaSuccess; ++c) {
        BatchParams bp = base;
        bp.lo = cls_lo[c];
        bp.hi = cls_hi[c];
        bp.cls = c;
        e = [&]() -> cudaError_t { KPX_CLASS_DISPATCH(launch_b_append_t, cls_kind[c], bp, s); }();
    }
    if (e != cudaSuccess) return e;
    k_b_prune<<<b_sm_count() * 6, PRUNE_THREADS, 0, s>>>(base);  // 40 registers: 6 blocks per SM
    k_b_end<<<(base.B + 255) / 256, 256, 0, s>>>(base);
    return cudaGetLastError();
}

}  // namespace kpx
