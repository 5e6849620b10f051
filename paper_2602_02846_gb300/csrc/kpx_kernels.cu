// kpx_kernels.cu -- the sm_103a kernels of one Kino-PAX+ iteration.
//
// Launch order per iteration (all counts are read from device memory, so
// the sequence has a fixed launch shape and can be captured in a graph):
//   begin      lambda (fixed or floor(t_e/|V_A|)), slot count, tickets,
//              region-key snapshot when the capacity rule could trigger
//   propagate  Alg. 2: one thread per (active node, sample) slot
//   mark       V_U filter: a region whose key holds a candidate id marks
//              that candidate's slot in a bitmask
//   scan       winners ranked in ascending slot order (decoupled look-back)
//   append     UpdateTree (Alg. 4): winners appended at n_nodes + rank
//              (everything but the end states); capacity rule
//   stage      the kept winners re-materialised from Philox: their end
//              states and the solution update (beside append and prune in
//              the graphs)
//   prune      PruneNodes (Alg. 3) over the pre-append tree, fused with the
//              compaction of the next V_A list (Alg. 5)
//   end        counters
#include <cuda_runtime.h>

#include "kpx_phases.cuh"

namespace kpx {

#define KPX_DISPATCH(FN, P, ...)                                                         \
    switch ((P).dyn * 2 + (P).integ) {                                                  \
        case KPX_DI6 * 2 + KPX_EULER: return FN<KPX_DI6, KPX_EULER>(P, __VA_ARGS__);         \
        case KPX_DI6 * 2 + KPX_RK4: return FN<KPX_DI6, KPX_RK4>(P, __VA_ARGS__);             \
        case KPX_DUBINS6 * 2 + KPX_EULER: return FN<KPX_DUBINS6, KPX_EULER>(P, __VA_ARGS__); \
        case KPX_DUBINS6 * 2 + KPX_RK4: return FN<KPX_DUBINS6, KPX_RK4>(P, __VA_ARGS__);     \
        case KPX_QUAD12 * 2 + KPX_EULER: return FN<KPX_QUAD12, KPX_EULER>(P, __VA_ARGS__);   \
        case KPX_QUAD12 * 2 + KPX_RK4: return FN<KPX_QUAD12, KPX_RK4>(P, __VA_ARGS__);       \
        default: return cudaErrorInvalidValue;                                          \
    }

namespace {

// ---------------------------------------------------------------------------
// init / reset: Alg. 1 initialisation.
// ---------------------------------------------------------------------------
template <int N>
__global__ void k_init(DevParams P, int first_time) {
    float xs[N];
#pragma unroll
    for (int d = 0; d < N; ++d) xs[d] = P.start[d];
    const int root_region = region_of<N>(P, xs);
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const uint64_t root_key = pack_key(0.0f, 0u);
    for (int64_t r = tid; r < P.R; r += stride) {
        P.region_key[r] = (r == root_region) ? root_key : KEY_INF;
        P.region_owner[r] = (r == root_region) ? 0 : -1;
    }
    for (int64_t w = tid; w < P.mask_words; w += stride) P.win_mask[w] = 0u;
    if (first_time) {
        for (int64_t t = tid; t < P.n_win_tiles; t += stride) P.win_tiles[t] = 0ull;
        for (int64_t t = tid; t < P.n_prune_tiles; t += stride) P.prune_tiles[t] = 0ull;
        for (int64_t i = tid; i < P.N; i += stride) P.clean[i] = 0u;  // epoch 0 is never current
    }
    if (tid == 0) {
        kpx_device_header* H = P.hdr;
        const int32_t epoch = first_time ? 0 : H->epoch;
        memset(H, 0, sizeof(kpx_device_header));
        H->epoch = epoch;
        H->status = KPX_OK;
        H->n_nodes = 1;
        H->count_A = 1;
        H->first_solution_iter = -1;
        H->goal_key = KEY_INF;
        if (in_goal(P, xs[0], xs[1], xs[2])) {
            H->goal_key = root_key;
            H->first_solution_iter = 0;
        }
#pragma unroll
        for (int d = 0; d < N; ++d) P.x[(int64_t)d * P.N] = xs[d];
        for (int d = 0; d < P.m; ++d) P.u[(int64_t)d * P.N] = 0.0f;
        P.K[0] = 0;
        P.parent[0] = -1;
        P.key[0] = root_key;
        P.region[0] = root_region;
        P.set[0] = SET_A;
        P.icount[0] = 0;
        P.va0[0] = 0;
    }
}

// ---------------------------------------------------------------------------
// obstacle grid (broad phase), built once per create: per-box cell ranges,
// per-cell counts (one warp per cell, boxes in index order), a scan into CSR
// offsets, then the fill.  Deterministic: each cell lists its boxes in
// ascending box index.
// ---------------------------------------------------------------------------
__global__ void k_box_cells(DevParams P) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= P.n_obs) return;
    const float4 lo = P.obs[2 * b], hi = P.obs[2 * b + 1];
    const float l[3] = {lo.x, lo.y, lo.z}, h[3] = {hi.x, hi.y, hi.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        P.box_cells[6 * b + a] = grid_cell(l[a], P.ws_lo[a], P.grid_inv[a], P.grid_n[a]);
        P.box_cells[6 * b + 3 + a] = grid_cell(h[a], P.ws_lo[a], P.grid_inv[a], P.grid_n[a]);
    }
}

__device__ __forceinline__ bool box_overlaps_cell(const DevParams& P, int b, int cx, int cy, int cz) {
    const int* bc = P.box_cells + 6 * b;
    return cx >= bc[0] && cx <= bc[3] && cy >= bc[1] && cy <= bc[4] && cz >= bc[2] && cz <= bc[5];
}

template <bool FILL>
__global__ void k_grid_cells(DevParams P) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < P.n_cells; c += warps) {
        const int cx = c % P.grid_n[0];
        const int cy = (c / P.grid_n[0]) % P.grid_n[1];
        const int cz = c / (P.grid_n[0] * P.grid_n[1]);
        int count = 0;
        const int start = FILL ? P.cell_start[c] : 0;
        for (int base = 0; base < P.n_obs; base += 32) {
            const int b = base + lane;
            const bool in = b < P.n_obs && box_overlaps_cell(P, b, cx, cy, cz);
            const uint32_t bal = __ballot_sync(FULL, in);
            if (FILL && in) {
                const int pos = start + count + __popc(bal & ((1u << lane) - 1u));
                if (pos < P.grid_cap) {
                    P.cell_box[2 * pos] = P.obs[2 * b];
                    P.cell_box[2 * pos + 1] = P.obs[2 * b + 1];
                }
            }
            count += __popc(bal);
        }
        if (!FILL && lane == 0) P.cell_start[c + 1] = count;
        if (FILL && lane == 0) P.cell_pair[c] = make_int2(start, min(P.cell_start[c + 1], P.grid_cap));
    }
    if (!FILL && blockIdx.x == 0 && threadIdx.x == 0) P.cell_start[0] = 0;
}

// in-place inclusive scan of cell_start[1..n_cells] (one block)
__global__ void __launch_bounds__(1024) k_grid_scan(DevParams P) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < P.n_cells; base += 1024) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < P.n_cells ? (uint32_t)P.cell_start[i + 1] : 0u;
        uint32_t agg;
        const uint32_t excl = block_exclusive_scan<1024>(v, agg, s_warp);
        if (i < P.n_cells) P.cell_start[i + 1] = (int32_t)(s_carry + excl + v);
        __syncthreads();
        if (threadIdx.x == 0) s_carry += agg;
        __syncthreads();
    }
    if (threadIdx.x == 0 && (int64_t)s_carry > (int64_t)P.grid_cap) {
        set_status(P.hdr, KPX_E_INTERNAL);
        P.hdr->err_info[2] = s_carry;
    }
}

// ---------------------------------------------------------------------------
// begin: branching factor, slot count, tickets; region snapshot for the
// capacity rule (only when an overflow is possible this iteration).
// ---------------------------------------------------------------------------
// In the loop body of a planner's graph (loop = 1) an iteration runs only
// while iterations are owed (graph_pending > 0); otherwise every kernel of
// the iteration is a no-op.
// Every warp also sorts chunks of the iteration's slots by their order key
// (order_chunk: K, or the quadcopter's predicted step count) for the
// propagate kernel (slot_order); the slot count and lambda it uses are read
// from counters begin_counters leaves alone (|V_A|, the iteration, the V_A
// buffer), exactly as begin_counters derives them.
__global__ void k_begin(DevParams P, int loop) {
    kpx_device_header* H = P.hdr;
    const bool allowed = !loop || H->graph_pending > 0;
    const bool snap = begin_needs_snapshot(P, H, allowed);  // reads counters begin_counters leaves alone
    const bool runs = allowed && problem_runs(P, H);
    const int count_A = H->count_A;
    const uint32_t iter = (uint32_t)H->iter;
    const int32_t* va = va_current(P, H);
    if (blockIdx.x == 0 && threadIdx.x == 0) begin_counters(P, H, allowed);
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (snap)
        for (int64_t r = tid; r < P.R; r += stride) P.region_snap[r] = P.region_key[r];
    if (runs && P.slot_order) {
        const int lam = begin_lambda(P, count_A);
        const int64_t n_slots = (int64_t)count_A * lam;
        const int64_t n_chunks = (n_slots + ORDER_CHUNK - 1) / ORDER_CHUNK;
        const int64_t warps = stride >> 5;
        for (int64_t c = tid >> 5; c < n_chunks; c += warps) {
            if (P.m == 4)
                order_chunk<4>(P, va, lam, iter, n_slots, c);
            else
                order_chunk<3>(P, va, lam, iter, n_slots, c);
        }
    }
}

// ---------------------------------------------------------------------------
// propagate (Alg. 2): warps take 32-slot chunks; a warp's first chunk is
// fixed (warp-major across blocks, no atomic), later chunks come from a
// ticket, so warps that drew short rollouts take more work.
// ---------------------------------------------------------------------------
#ifndef KPX_QUAD_MIN_BLOCKS
#define KPX_QUAD_MIN_BLOCKS 3
#endif
// resident blocks per SM requested from the register allocator: the 12D
// quadcopter's RK4 would otherwise need ~100 registers (two blocks per SM)
template <int DYN>
struct PropOccupancy {
    static constexpr int blocks = DYN == KPX_QUAD12 ? KPX_QUAD_MIN_BLOCKS : 4;
};

template <int DYN, int INTEG, bool SYM>
__global__ void __launch_bounds__(PROP_THREADS, PropOccupancy<DYN>::blocks)
    k_propagate(DevParams P, kpx_debug_records rec, int rec_on) {
    kpx_device_header* H = P.hdr;
    if (!H->active) return;
    const int64_t n_slots = H->n_slots;
    const int lam = H->lambda;
    const uint32_t iter = (uint32_t)H->iter;
    const int32_t* va = va_current(P, H);
    const bool early = (P.flags & KPX_FLAG_EARLY_REJECT) && !rec_on;
    const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const bool ordered = P.slot_order != nullptr;
    const int64_t n_units = propagate_units(n_slots, ordered);  // longest first when ordered
    int64_t q = (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    uint32_t steps = 0, tests = 0, n_valid = 0;
    while (q < n_units) {
        const int64_t chunk = propagate_unit_chunk(q, n_slots, ordered);
        propagate_chunk<DYN, INTEG, SYM>(P, n_slots, lam, iter, va, early, chunk, rec, rec_on, steps, tests, n_valid,
                                         P.slot_order);
        unsigned long long t = 0ull;
        if ((threadIdx.x & 31) == 0) t = atomicAdd((unsigned long long*)&H->prop_ticket, 1ull);
        q = n_warps + (int64_t)__shfl_sync(FULL, t, 0);
    }
    flush_propagate_counters(H, steps, tests, n_valid);
}

__global__ void k_mark(DevParams P) {
    if (!P.hdr->active) return;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < P.R; r += gridDim.x * blockDim.x) mark_region(P, r);
}

__global__ void __launch_bounds__(WIN_THREADS) k_scan(DevParams P) {
    __shared__ uint32_t s_tile, s_prefix;
    __shared__ uint32_t s_warp[WIN_THREADS / 32];
    kpx_device_header* H = P.hdr;
    if (!H->active) return;
    const int64_t live_words = (H->n_slots + 31) / 32;
    const int64_t n_tiles = (live_words + WIN_TILE_WORDS - 1) / WIN_TILE_WORDS;
    if ((int64_t)blockIdx.x >= n_tiles) return;  // the other blocks take every tile
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&H->win_ticket, 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        __syncthreads();
        if ((int64_t)tile >= n_tiles) return;
        scan_tile(P, H, tile, n_tiles, live_words, s_warp, s_prefix);
    }
}

template <int DYN, int INTEG>
__global__ void __launch_bounds__(128) k_append(DevParams P) {
    kpx_device_header* H = P.hdr;
    if (!H->active) return;
    const int W = H->n_win;
    const int n_old = H->n_nodes;
    const int room = P.N - n_old;
    const int kept = W < room ? W : room;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        H->n_kept = kept;
        if (W > kept) set_status(H, KPX_TREE_FULL);
    }
    const int lam = H->lambda;
    const uint32_t iter = (uint32_t)H->iter;
    const int32_t* va = va_current(P, H);
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < W; w += gridDim.x * blockDim.x)
        append_meta<DYN, INTEG>(P, H, w, kept, n_old, lam, iter, va);
}

// The kept winners' end states (one thread per winner, re-materialised) and
// the solution update; in the planner's graphs beside append and prune.
template <int DYN, int INTEG>
__global__ void __launch_bounds__(128) k_stage(DevParams P) {
    kpx_device_header* H = P.hdr;
    if (!H->active) return;
    const int W = H->n_win;
    const int n_old = H->n_nodes;  // end_counters advances it only after both halves
    const int room = P.N - n_old;
    const int kept = W < room ? W : room;
    const int lam = H->lambda;
    const uint32_t iter = (uint32_t)H->iter;
    const int32_t* va = va_current(P, H);
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < kept; w += gridDim.x * blockDim.x)
        stage_winner<DYN, INTEG>(P, H, w, n_old, lam, iter, va);
}

__global__ void __launch_bounds__(PRUNE_THREADS, 8) k_prune(DevParams P) {
    __shared__ uint32_t s_tile, s_prefix;
    __shared__ int32_t s_parent[PRUNE_TILE];
    __shared__ uint8_t s_set[PRUNE_TILE];
    __shared__ uint8_t s_icount[PRUNE_TILE];
    __shared__ uint32_t s_counts[PRUNE_ROUND_WARPS];
    kpx_device_header* H = P.hdr;
    if (!H->active) return;
    const int n_old = H->n_nodes;
    const int total = n_old + H->n_kept;
    const int n_tiles = (total + PRUNE_TILE - 1) / PRUNE_TILE;
    if ((int)blockIdx.x >= n_tiles) return;  // the other blocks take every tile
    const uint32_t epoch = (uint32_t)H->epoch;
    int32_t* va_next = va_following(P, H);
    int cA = 0, cI = 0, cT = 0;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&H->prune_ticket, 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        __syncthreads();
        if ((int)tile >= n_tiles) break;
        prune_tile(P, H, tile, n_tiles, n_old, total, epoch, va_next, s_parent, s_set, s_icount, s_counts, s_prefix,
                   cA, cI, cT);
    }
    flush_prune_counters(H, cA, cI, cT);
}

__global__ void k_end(DevParams P) { end_counters(P, P.hdr); }

// The end of an iteration in the loop body of a planner's graph: an
// iteration that ran (graph_pending > 0, as k_begin saw it) ends and is
// counted off; once the problem has stopped (tree full, an error, its
// iteration limit) the iterations still owed would be no-ops and are
// dropped.  The body's last iteration lets the loop run again while
// iterations are owed.  graph_pending only falls, so the loop ends.
__global__ void k_end_loop(DevParams P, cudaGraphConditionalHandle h, int last) {
    kpx_device_header* H = P.hdr;
    if (H->graph_pending > 0) {
        end_counters(P, H);
        H->graph_pending = problem_runs(P, H) ? H->graph_pending - 1 : 0;
    }
    if (last) cudaGraphSetConditional(h, H->graph_pending > 0 ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// solution extraction: parent walk from the best goal node.
// ---------------------------------------------------------------------------
__global__ void k_path(DevParams P) {
    kpx_device_header* H = P.hdr;
    const uint64_t gk = H->goal_key;
    if (gk == KEY_INF) {
        H->traj_len = -1;
        return;
    }
    const int id = (int)(uint32_t)gk;
    int len = 0;
    for (int p = id; P.parent[p] >= 0 && len < P.N; p = P.parent[p]) ++len;
    H->traj_len = len;
    int p = id;
    for (int k = len; k >= 0; --k) {
        P.path[k] = p;
        p = P.parent[p];
    }
}

__global__ void k_gather(DevParams P, int first, int rows) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const int node = P.path[first + r];
    const int w = P.n + P.m + 1;
    float* row = P.traj + (int64_t)r * w;
    for (int d = 0; d < P.n; ++d) row[d] = P.x[(int64_t)d * P.N + node];
    for (int d = 0; d < P.m; ++d) row[P.n + d] = P.u[(int64_t)d * P.N + node];
    row[P.n + P.m] = __int_as_float((int)P.K[node]);
}

// ---------------------------------------------------------------------------
// a new region decomposition (adaptive delta): every node's region under
// the new grid; each region's key = the minimum key of its non-terminal
// nodes; a non-terminal node that does not hold its region's key is
// dominated; the memoised ancestor bits are cleared for PruneNodes to
// re-derive.  Terminal nodes keep their set byte.
// ---------------------------------------------------------------------------
__global__ void k_remap_clear(DevParams P) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < P.R; r += (int64_t)gridDim.x * blockDim.x) {
        P.region_key[r] = KEY_INF;
        P.region_owner[r] = -1;
    }
}

template <int N>
__global__ void k_remap_assign(DevParams P) {
    const int n_nodes = P.hdr->n_nodes;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += gridDim.x * blockDim.x) {
        float x[N];
#pragma unroll
        for (int d = 0; d < N; ++d) x[d] = P.x[(int64_t)d * P.N + i];
        const int r = region_of<N>(P, x);
        P.region[i] = r;
        if ((P.set[i] & SET_MASK) != SET_T) atomicMin((unsigned long long*)&P.region_key[r], (unsigned long long)P.key[i]);
    }
}

__global__ void k_remap_mark(DevParams P) {
    const int n_nodes = P.hdr->n_nodes;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += gridDim.x * blockDim.x) {
        const uint8_t sb = P.set[i];
        if ((sb & SET_MASK) == SET_T) continue;
        const int r = P.region[i];
        const bool owner = P.key[i] == P.region_key[r];
        if (owner) P.region_owner[r] = i;
        P.set[i] = (uint8_t)((sb & SET_MASK) | (owner ? 0 : SET_DOM));
    }
}

int sm_count() {
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

// a persistent grid: enough resident blocks to fill the GPU, never more than the work
int persistent_blocks(int64_t work_blocks, int per_sm) {
    int64_t g = (int64_t)sm_count() * per_sm;
    if (g > work_blocks) g = work_blocks;
    return (int)(g < 1 ? 1 : g);
}

template <int DYN, int INTEG, bool SYM>
int propagate_blocks_per_sm() {
    static int per_sm = 0;
    if (!per_sm) {
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_propagate<DYN, INTEG, SYM>, PROP_THREADS, 0);
        per_sm = v < 1 ? 1 : v;
    }
    return per_sm;
}

template <int DYN, int INTEG>
int propagate_occupancy_t(const DevParams& P, int) {
    return P.sym_bounds ? propagate_blocks_per_sm<DYN, INTEG, true>() : propagate_blocks_per_sm<DYN, INTEG, false>();
}

int propagate_occupancy(const DevParams& P) { KPX_DISPATCH(propagate_occupancy_t, P, 0); }

template <int DYN, int INTEG>
cudaError_t launch_propagate_t(const DevParams& P, const kpx_debug_records* rec, cudaStream_t s) {
    const int fit = propagate_occupancy_t<DYN, INTEG>(P, 0);
    const int per_sm = P.prop_bps > 0 && P.prop_bps < fit ? P.prop_bps : fit;
    const int grid = persistent_blocks((P.slot_cap + PROP_THREADS - 1) / PROP_THREADS, per_sm);
    kpx_debug_records r{};
    int on = 0;
    if (rec && rec->valid) {
        r = *rec;
        on = 1;
    }
    if (P.sym_bounds)
        k_propagate<DYN, INTEG, true><<<grid, PROP_THREADS, 0, s>>>(P, r, on);
    else
        k_propagate<DYN, INTEG, false><<<grid, PROP_THREADS, 0, s>>>(P, r, on);
    return cudaGetLastError();
}

template <int DYN, int INTEG>
cudaError_t launch_append_t(const DevParams& P, cudaStream_t s) {
    k_append<DYN, INTEG><<<persistent_blocks((P.R + 127) / 128, 4), 128, 0, s>>>(P);
    return cudaGetLastError();
}

template <int DYN, int INTEG>
cudaError_t launch_stage_t(const DevParams& P, cudaStream_t s) {
    k_stage<DYN, INTEG><<<persistent_blocks((P.R + 127) / 128, 4), 128, 0, s>>>(P);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_init(const DevParams& P, bool first_time, cudaStream_t s) {
    int64_t work = P.R > P.mask_words ? P.R : P.mask_words;
    int blocks = (int)((work + 255) / 256);
    if (blocks > 2048) blocks = 2048;
    if (blocks < 1) blocks = 1;
    if (P.n == 12)
        k_init<12><<<blocks, 256, 0, s>>>(P, first_time ? 1 : 0);
    else
        k_init<6><<<blocks, 256, 0, s>>>(P, first_time ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_grid_build(const DevParams& P, cudaStream_t s) {
    if (P.n_obs == 0) return cudaSuccess;
    k_box_cells<<<(P.n_obs + 127) / 128, 128, 0, s>>>(P);
    const int cell_blocks = persistent_blocks((P.n_cells + 7) / 8, 8);
    k_grid_cells<false><<<cell_blocks, 256, 0, s>>>(P);
    k_grid_scan<<<1, 1024, 0, s>>>(P);
    k_grid_cells<true><<<cell_blocks, 256, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_begin(const DevParams& P, cudaStream_t s, bool loop) {
    // the snapshot wants a few blocks per SM; the propagate order one warp
    // per 128-slot chunk (up to 6 blocks of 8 warps per SM at 40 registers)
    int64_t work = (P.R + 255) / 256;
    int per_sm = 2;
    if (P.slot_order) {
        const int64_t order_blocks = (P.slot_cap + ORDER_CHUNK * 8 - 1) / (ORDER_CHUNK * 8);
        if (order_blocks > work) work = order_blocks;
        per_sm = 6;
    }
    k_begin<<<persistent_blocks(work, per_sm), 256, 0, s>>>(P, loop ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_propagate(const DevParams& P, const kpx_debug_records* rec, cudaStream_t s) {
    KPX_DISPATCH(launch_propagate_t, P, rec, s);
}

cudaError_t launch_mark(const DevParams& P, cudaStream_t s) {
    k_mark<<<persistent_blocks((P.R + 255) / 256, 8), 256, 0, s>>>(P);
    return cudaGetLastError();
}

// every tile of a large iteration in flight at once (31 registers: 8 blocks per SM)
cudaError_t launch_scan(const DevParams& P, cudaStream_t s) {
    k_scan<<<persistent_blocks(P.n_win_tiles, 8), WIN_THREADS, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_append(const DevParams& P, cudaStream_t s) { KPX_DISPATCH(launch_append_t, P, s); }

cudaError_t launch_stage(const DevParams& P, cudaStream_t s) { KPX_DISPATCH(launch_stage_t, P, s); }

cudaError_t launch_prune(const DevParams& P, cudaStream_t s) {
    // a tile's time is its deepest ancestor walk: as many tiles in flight as fit
    // (32 registers and 6 KB of shared memory a block: 8 blocks per SM)
    k_prune<<<persistent_blocks(P.n_prune_tiles, 8), PRUNE_THREADS, 0, s>>>(P);
    return cudaGetLastError();
}

// A look-back wait that nothing will release: tile 1 of `tiles` waits on
// tile 0 at an epoch no tile word carries.  The wait gives up after its poll
// limit and records KPX_E_TIMEOUT (err_info[0] = 0x10000 | 1): a test that the
// bounded waits end and report without faulting.
__global__ void k_wait_timeout(DevParams P, uint64_t* tiles) {
    kpx_device_header* H = P.hdr;
    uint32_t epoch = ((uint32_t)H->epoch + (1u << 29)) & 0x3FFFFFFFu;
    if (epoch == 0) epoch = 1;
    lookback(tiles, 1u, 0u, epoch, H);
}

cudaError_t launch_wait_timeout(const DevParams& P, cudaStream_t s) {
    uint64_t* tiles = P.n_win_tiles >= 2 ? P.win_tiles : (P.n_prune_tiles >= 2 ? P.prune_tiles : nullptr);
    if (!tiles) return cudaErrorInvalidValue;
    k_wait_timeout<<<1, 1, 0, s>>>(P, tiles);
    return cudaGetLastError();
}

cudaError_t launch_end_loop(const DevParams& P, cudaGraphConditionalHandle h, bool last, cudaStream_t s) {
    k_end_loop<<<1, 1, 0, s>>>(P, h, last ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_end(const DevParams& P, cudaStream_t s) {
    k_end<<<1, 1, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_remap_regions(const DevParams& P, cudaStream_t s) {
    k_remap_clear<<<persistent_blocks((P.R + 255) / 256, 4), 256, 0, s>>>(P);
    const int blocks = persistent_blocks((P.N + 255) / 256, 4);
    if (P.n == 12)
        k_remap_assign<12><<<blocks, 256, 0, s>>>(P);
    else
        k_remap_assign<6><<<blocks, 256, 0, s>>>(P);
    k_remap_mark<<<blocks, 256, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_path(const DevParams& P, cudaStream_t s) {
    k_path<<<1, 1, 0, s>>>(P);
    return cudaGetLastError();
}

void prepare_launches(const DevParams& P) {
    (void)sm_count();
    propagate_occupancy(P);
}

cudaError_t launch_gather(const DevParams& P, int32_t first_row, int32_t rows, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    k_gather<<<(rows + 127) / 128, 128, 0, s>>>(P, first_row, rows);
    return cudaGetLastError();
}

}  // namespace kpx
