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
//   append     UpdateTree (Alg. 4): winners re-materialised from Philox and
//              appended at n_nodes + rank; capacity rule; solution update
//   prune      PruneNodes (Alg. 3) over the pre-append tree, fused with the
//              compaction of the next V_A list (Alg. 5)
//   end        counters
#include <cuda_runtime.h>

#include "kpx_device.cuh"

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

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr uint32_t LOOKBACK_POLL_LIMIT = 1u << 20;

// ---------------------------------------------------------------------------
// Block-wide exclusive scan of one value per thread.
// ---------------------------------------------------------------------------
template <int THREADS>
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t& total, uint32_t* s_warp) {
    constexpr int NW = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NW ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NW) s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t excl = x - v + (warp > 0 ? s_warp[warp - 1] : 0u);
    total = s_warp[NW - 1];
    __syncthreads();
    return excl;
}

// Single-pass chained scan across tiles ("decoupled look-back"): each tile
// publishes its aggregate, then walks back over predecessors until it meets
// an inclusive prefix.  Tile ids come from an atomic ticket, so every
// predecessor of a waiting tile is already running.  Status word:
// epoch (30 bits) << 34 | flag (1 aggregate, 2 prefix) << 32 | value.
// The wait is bounded: after LOOKBACK_POLL_LIMIT polls the kernel records
// KPX_E_TIMEOUT and continues with the partial prefix.
__device__ uint32_t lookback(uint64_t* tiles, uint32_t tile, uint32_t agg, uint32_t epoch, kpx_device_header* H) {
    const uint64_t E = (uint64_t)(epoch & 0x3FFFFFFFu);
    if (tile == 0) {
        st_relaxed_u64(&tiles[0], (E << 34) | (2ull << 32) | agg);
        return 0u;
    }
    st_relaxed_u64(&tiles[tile], (E << 34) | (1ull << 32) | agg);
    uint32_t excl = 0u;
    int t = (int)tile - 1;
    uint32_t polls = 0;
    while (t >= 0) {
        const uint64_t w = ld_relaxed_u64(&tiles[t]);
        const uint32_t flag = (uint32_t)(w >> 32) & 3u;
        if ((w >> 34) == E && flag != 0u) {
            excl += (uint32_t)w;
            if (flag == 2u) break;
            --t;
        } else {
            if (++polls > LOOKBACK_POLL_LIMIT) {
                set_status(H, KPX_E_TIMEOUT);
                H->err_info[0] = 0x10000u | tile;
                break;
            }
            __nanosleep(32);
        }
    }
    st_relaxed_u64(&tiles[tile], (E << 34) | (2ull << 32) | (excl + agg));
    return excl;
}

__device__ __forceinline__ const int32_t* va_current(const DevParams& P, const kpx_device_header* H) {
    return H->va_sel ? P.va1 : P.va0;
}

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
__global__ void k_begin(DevParams P) {
    kpx_device_header* H = P.hdr;
    const bool active = H->status == KPX_OK;
    const int count_A = H->count_A;
    const int lam = P.lambda_fixed > 0 ? P.lambda_fixed : (count_A > 0 ? max(1, P.N / count_A) : 0);
    const int64_t n_slots = active ? (int64_t)count_A * lam : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        H->active = active ? 1 : 0;
        H->lambda = lam;
        H->n_slots = n_slots;
        H->prop_ticket = 0ull;
        H->win_ticket = 0u;
        H->prune_ticket = 0u;
        H->n_win = 0;
        H->n_kept = 0;
        H->count_A_next = 0;
        H->last_valid = 0ull;
        H->n_active = H->n_inactive = H->n_terminal = 0;
        if (active) {
            H->epoch = (H->epoch + 1) & 0x3FFFFFFF;
            if (H->epoch == 0) H->epoch = 1;
            if (H->t_start_ns == 0ull) H->t_start_ns = globaltimer_ns();
        }
    }
    if (!active) return;
    const int64_t max_new = n_slots < P.R ? n_slots : P.R;
    if ((int64_t)H->n_nodes + max_new <= P.N) return;  // capacity rule cannot trigger
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = tid; r < P.R; r += stride) P.region_snap[r] = P.region_key[r];
}

// ---------------------------------------------------------------------------
// propagate (Alg. 2).  Slot = rank j of the parent in V_A times lambda plus
// sample s; one lane per slot.  A warp's first chunk of 32 slots is fixed
// (warp-major across blocks, no atomic); later chunks come from a ticket, so
// warps that drew short rollouts take more work.
// ---------------------------------------------------------------------------
// resident blocks per SM requested from the register allocator: the 12D
// quadcopter's RK4 would otherwise need ~100 registers (two blocks per SM)
#ifndef KPX_QUAD_MIN_BLOCKS
#define KPX_QUAD_MIN_BLOCKS 3
#endif
template <int DYN>
struct PropOccupancy {
    static constexpr int blocks = DYN == KPX_QUAD12 ? KPX_QUAD_MIN_BLOCKS : 4;
};

template <int DYN, int INTEG>
__global__ void __launch_bounds__(PROP_THREADS, PropOccupancy<DYN>::blocks)
    k_propagate(DevParams P, kpx_debug_records rec, int rec_on) {
    constexpr int n = Dims<DYN>::n, m = Dims<DYN>::m;
    kpx_device_header* H = P.hdr;
    if (!H->active) return;
    const int64_t n_slots = H->n_slots;
    const int lam = H->lambda;
    const uint32_t iter = (uint32_t)H->iter;
    const int32_t* va = va_current(P, H);
    const bool early = (P.flags & KPX_FLAG_EARLY_REJECT) && !rec_on;
    const int lane = threadIdx.x & 31;
    const uint32_t cand_base = (uint32_t)P.N;
    const int64_t n_warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    int64_t chunk = (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    uint32_t steps = 0, tests = 0, n_valid = 0;
    for (;;) {
        const int64_t base = chunk * 32;
        if (base >= n_slots) break;
        const int64_t slot = base + lane;
        if (slot < n_slots) {
            LaneRollout<DYN, INTEG> R;
            R.start(P, va, lam, iter, slot);
            bool ok = true;
            while (ok && R.k < R.K) {
                ++steps;
                ok = early ? R.template advance<false>(P, tests) : R.template advance<true>(P, tests);
            }
            int r = -1;
            uint64_t key = KEY_INF;
            if (ok) {
                r = region_of<n>(P, R.x);
                key = pack_key(R.cost(P), cand_base + (uint32_t)slot);
                if (early) {
                    // collision-after-cost: only a possible winner is checked against obstacles
                    ok = key < __ldcg(&P.region_key[r]);
                    if (ok) {
                        float x0[n];
#pragma unroll
                        for (int d = 0; d < n; ++d) x0[d] = P.x[(int64_t)d * P.N + R.node];
                        ok = obstacle_pass<DYN, INTEG>(P, x0, R.u, R.K, steps, tests);
                    }
                }
                if (ok && key < __ldcg(&P.region_key[r]))
                    atomicMin((unsigned long long*)&P.region_key[r], (unsigned long long)key);
            }
            n_valid += ok ? 1u : 0u;
            if (rec_on && slot < rec.capacity) {
                rec.valid[slot] = ok ? 1 : 0;
                rec.region[slot] = ok ? r : -1;
                rec.key[slot] = ok ? key : KEY_INF;
                rec.K[slot] = R.K;
#pragma unroll
                for (int d = 0; d < n; ++d) rec.x[(int64_t)d * rec.capacity + slot] = R.x[d];
#pragma unroll
                for (int d = 0; d < m; ++d) rec.u[(int64_t)d * rec.capacity + slot] = R.u[d];
            }
        }
        unsigned long long t = 0ull;
        if (lane == 0) t = atomicAdd((unsigned long long*)&H->prop_ticket, 1ull);
        chunk = n_warps + (int64_t)__shfl_sync(FULL, t, 0);
    }
    // work counters (one atomic each per warp)
    unsigned long long st = steps, te = tests, nv = n_valid;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        st += __shfl_down_sync(FULL, st, o);
        te += __shfl_down_sync(FULL, te, o);
        nv += __shfl_down_sync(FULL, nv, o);
    }
    if (lane == 0 && st) {
        atomicAdd((unsigned long long*)&H->total_steps, st);
        atomicAdd((unsigned long long*)&H->total_box_tests, te);
        if (nv) atomicAdd((unsigned long long*)&H->last_valid, nv);
    }
}

// ---------------------------------------------------------------------------
// mark: a region whose key carries a candidate id (>= N) names the slot of
// the winner of that region (the V_U filter: "cost(x) = cost(R_i)").
// ---------------------------------------------------------------------------
__global__ void k_mark(DevParams P) {
    const kpx_device_header* H = P.hdr;
    if (!H->active) return;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < P.R; r += gridDim.x * blockDim.x) {
        const uint64_t k = P.region_key[r];
        if (k == KEY_INF) continue;
        const uint32_t id = (uint32_t)k;
        if (id < (uint32_t)P.N) continue;
        const uint32_t slot = id - (uint32_t)P.N;
        if ((int64_t)slot >= P.slot_cap) {  // a stale candidate id: cannot happen in a consistent state
            set_status(P.hdr, KPX_E_INTERNAL);
            continue;
        }
        atomicOr(&P.win_mask[slot >> 5], 1u << (slot & 31));
    }
}

// ---------------------------------------------------------------------------
// scan: ranks of the marked slots in ascending slot order -> win_slot[rank];
// clears the mask for the next iteration.
// ---------------------------------------------------------------------------
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
        const int64_t w0 = (int64_t)tile * WIN_TILE_WORDS + (int64_t)threadIdx.x * WIN_WORDS_PER_THREAD;
        uint32_t w[WIN_WORDS_PER_THREAD];
        uint32_t cnt = 0;
#pragma unroll
        for (int i = 0; i < WIN_WORDS_PER_THREAD; ++i) {
            w[i] = (w0 + i < live_words) ? P.win_mask[w0 + i] : 0u;
            cnt += __popc(w[i]);
        }
        uint32_t agg;
        const uint32_t excl = block_exclusive_scan<WIN_THREADS>(cnt, agg, s_warp);
        if (threadIdx.x == 0) {
            s_prefix = lookback(P.win_tiles, tile, agg, (uint32_t)H->epoch, H);
            if ((int64_t)tile == n_tiles - 1) H->n_win = (int32_t)(s_prefix + agg);
        }
        __syncthreads();
        uint32_t rank = s_prefix + excl;
#pragma unroll
        for (int i = 0; i < WIN_WORDS_PER_THREAD; ++i) {
            uint32_t word = w[i];
            while (word) {
                const int b = __ffs(word) - 1;
                word &= word - 1;
                if (rank < (uint32_t)P.R)
                    P.win_slot[rank] = (int32_t)((w0 + i) * 32 + b);
                else
                    set_status(H, KPX_E_INTERNAL);
                ++rank;
            }
            if (w[i]) P.win_mask[w0 + i] = 0u;
        }
    }
}

// ---------------------------------------------------------------------------
// append (UpdateTree, Alg. 4): each winner's rollout is re-materialised from
// (seed, iteration, node, sample) with the propagate kernel's arithmetic,
// written to T at n_nodes + rank, and its region key rewritten with the new
// id.  Winners beyond the capacity restore their region from the snapshot
// and mark the planner KPX_TREE_FULL.  Goal nodes lower the solution key.
// ---------------------------------------------------------------------------
template <int DYN, int INTEG>
__global__ void __launch_bounds__(128) k_append(DevParams P) {
    constexpr int n = Dims<DYN>::n, m = Dims<DYN>::m;
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
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < W; w += gridDim.x * blockDim.x) {
        const int slot = P.win_slot[w];
        LaneRollout<DYN, INTEG> Rw;
        Rw.start(P, va, lam, iter, (int64_t)slot);
        uint32_t te_unused = 0;
        for (int k = 0; k < Rw.K; ++k) Rw.template advance<false>(P, te_unused);
        const float c = Rw.cost(P);
        const int node = Rw.node;
        float (&x)[n] = Rw.x;
        float (&u)[m] = Rw.u;
        const int K = Rw.K;
        const int r = region_of<n>(P, x);
        const uint64_t cand_key = pack_key(c, (uint32_t)P.N + (uint32_t)slot);
        if (P.region_key[r] != cand_key) {
            set_status(H, KPX_E_INTERNAL);
            H->err_info[1] = (uint32_t)slot;
            continue;
        }
        if (w < kept) {
            const int id = n_old + w;
#pragma unroll
            for (int d = 0; d < n; ++d) P.x[(int64_t)d * P.N + id] = x[d];
#pragma unroll
            for (int d = 0; d < m; ++d) P.u[(int64_t)d * P.N + id] = u[d];
            P.K[id] = (uint16_t)K;
            P.parent[id] = node;
            const uint64_t k = pack_key(c, (uint32_t)id);
            P.key[id] = k;
            P.region[id] = r;
            P.set[id] = SET_A;
            P.icount[id] = 0;
            P.region_key[r] = k;
            // the previous owner of r loses its region (one winner per region,
            // so this thread is the only writer of that node's set byte)
            const int old = P.region_owner[r];
            if (old >= 0) P.set[old] = (uint8_t)(P.set[old] | SET_DOM);
            P.region_owner[r] = id;
            if (in_goal(P, x[0], x[1], x[2])) atomicMin((unsigned long long*)&H->goal_key, (unsigned long long)k);
        } else {
            P.region_key[r] = P.region_snap[r];
        }
    }
}

// ---------------------------------------------------------------------------
// prune (PruneNodes, Alg. 3) over nodes [0, n_nodes) in the literal rule
// order, then the compaction of V_A (Alg. 5) over [0, n_nodes + kept): new
// winners are active by Alg. 4.  A tile of PRUNE_TILE consecutive ids keeps
// ascending order; tiles are chained by the look-back scan.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PRUNE_THREADS) k_prune(DevParams P) {
    __shared__ uint32_t s_tile, s_prefix;
    __shared__ uint32_t s_warp[PRUNE_THREADS / 32];
    // the tile's parent ids and set bytes: ancestor walks that stay inside
    // the tile read shared memory (parents precede children)
    __shared__ int32_t s_parent[PRUNE_TILE];
    __shared__ uint8_t s_set[PRUNE_TILE];
    kpx_device_header* H = P.hdr;
    if (!H->active) return;
    const int n_old = H->n_nodes;
    const int total = n_old + H->n_kept;
    const int n_tiles = (total + PRUNE_TILE - 1) / PRUNE_TILE;
    if ((int)blockIdx.x >= n_tiles) return;  // the other blocks take every tile
    int cA = 0, cI = 0, cT = 0;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(&H->prune_ticket, 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        __syncthreads();
        if ((int)tile >= n_tiles) break;
        const int i_max = P.i_max;
        const int tile0 = (int)tile * PRUNE_TILE;
        for (int k = threadIdx.x; k < PRUNE_TILE; k += PRUNE_THREADS) {
            const int i = tile0 + k;
            s_parent[k] = i < n_old ? P.parent[i] : -1;
            s_set[k] = i < n_old ? P.set[i] : 0;
        }
        __syncthreads();
        const int base = tile0 + threadIdx.x * PRUNE_PER_THREAD;
        uint32_t amask = 0;
#pragma unroll
        for (int q = 0; q < PRUNE_PER_THREAD; ++q) {
            const int i = base + q;
            if (i >= total) break;
            if (i >= n_old) {  // appended this iteration: in V_A
                amask |= 1u << q;
                ++cA;
                continue;
            }
            const uint8_t sb = P.set[i];
            const int st = sb & SET_MASK;
            if (st == SET_T) {  // V_T is permanent
                ++cT;
                continue;
            }
            // key(i) >= key(region(i)) always, with equality only for the
            // region's owner: "best" is "not dominated"
            const bool dominated = (sb & SET_DOM) != 0;
            const bool best = !dominated;
            int ic = P.icount[i];
            const int ic0 = ic;
            int nst = st;
            bool anc = (sb & SET_ANC) != 0;
            bool done = false;
            if (best && st == SET_I) {  // rule 1: region best while inactive
                ++ic;
                if (ic > i_max) {
                    nst = SET_A;
                    done = true;
                }
            }
            if (!done && ic > i_max && best) done = true;  // rule 2
            if (!done && dominated) {                       // rule 3: dominated
                nst = SET_T;
                done = true;
            }
            if (!done) {  // rule 4: any strict ancestor dominated
                if (!anc) {
                    int p = s_parent[i - tile0];
                    while (p >= tile0) {  // inside the tile: shared memory (a stale
                        // set byte only lacks a monotone flag, which the walk re-derives)
                        const uint8_t sp = s_set[p - tile0];
                        if (sp & (SET_DOM | SET_ANC)) {
                            anc = true;
                            break;
                        }
                        p = s_parent[p - tile0];
                    }
                    for (; !anc && p >= 0; p = P.parent[p]) {
                        const uint8_t sp = *(volatile const uint8_t*)&P.set[p];
                        if (sp & (SET_DOM | SET_ANC)) anc = true;
                    }
                }
                if (anc) nst = SET_I;
            }
            const uint8_t nb = (uint8_t)(nst | (anc ? SET_ANC : 0) | (sb & SET_DOM));
            if (nb != sb) P.set[i] = nb;
            if (ic != ic0) P.icount[i] = (uint8_t)ic;
            if (nst == SET_A) {
                amask |= 1u << q;
                ++cA;
            } else if (nst == SET_I) {
                ++cI;
            } else {
                ++cT;
            }
        }
        uint32_t agg;
        const uint32_t excl = block_exclusive_scan<PRUNE_THREADS>((uint32_t)__popc(amask), agg, s_warp);
        if (threadIdx.x == 0) {
            s_prefix = lookback(P.prune_tiles, tile, agg, (uint32_t)H->epoch, H);
            if ((int)tile == n_tiles - 1) H->count_A_next = (int32_t)(s_prefix + agg);
        }
        __syncthreads();
        int32_t* va_next = H->va_sel ? P.va0 : P.va1;
        uint32_t pos = s_prefix + excl;
#pragma unroll
        for (int q = 0; q < PRUNE_PER_THREAD; ++q) {
            if (amask & (1u << q)) {
                // at most one active node per region, so pos < min(N, R) = va_cap
                if (pos < (uint32_t)P.va_cap)
                    va_next[pos] = base + q;
                else
                    set_status(H, KPX_E_INTERNAL);
                ++pos;
            }
        }
        __syncthreads();
    }
    // set sizes for the statistics
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cA += __shfl_down_sync(FULL, cA, o);
        cI += __shfl_down_sync(FULL, cI, o);
        cT += __shfl_down_sync(FULL, cT, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (cA) atomicAdd(&H->n_active, cA);
        if (cI) atomicAdd(&H->n_inactive, cI);
        if (cT) atomicAdd(&H->n_terminal, cT);
    }
}

// ---------------------------------------------------------------------------
// end: commit the counters of the iteration.
// ---------------------------------------------------------------------------
__global__ void k_end(DevParams P) {
    kpx_device_header* H = P.hdr;
    if (!H->active) return;
    H->n_nodes += H->n_kept;
    H->count_A = H->count_A_next;
    H->va_sel ^= 1;
    H->last_candidates = (uint64_t)H->n_slots;
    H->last_winners = (uint64_t)H->n_kept;
    H->total_candidates += (uint64_t)H->n_slots;
    H->total_valid += H->last_valid;
    H->total_winners += (uint64_t)H->n_kept;
    const uint64_t now = globaltimer_ns();
    if (H->goal_key != KEY_INF && H->first_solution_iter < 0) {
        H->first_solution_iter = H->iter;
        H->t_first_solution_ns = now;
    }
    H->iter += 1;
    H->t_last_ns = now;
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

template <int DYN, int INTEG>
int propagate_blocks_per_sm() {
    static int per_sm = 0;
    if (!per_sm) {
        int v = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_propagate<DYN, INTEG>, PROP_THREADS, 0);
        per_sm = v < 1 ? 1 : v;
    }
    return per_sm;
}

template <int DYN, int INTEG>
int propagate_occupancy_t(const DevParams&, int) {
    return propagate_blocks_per_sm<DYN, INTEG>();
}

int propagate_occupancy(const DevParams& P) { KPX_DISPATCH(propagate_occupancy_t, P, 0); }

template <int DYN, int INTEG>
cudaError_t launch_propagate_t(const DevParams& P, const kpx_debug_records* rec, cudaStream_t s) {
    const int per_sm = propagate_blocks_per_sm<DYN, INTEG>();
    const int grid = persistent_blocks((P.slot_cap + PROP_THREADS - 1) / PROP_THREADS, per_sm);
    kpx_debug_records r{};
    int on = 0;
    if (rec && rec->valid) {
        r = *rec;
        on = 1;
    }
    k_propagate<DYN, INTEG><<<grid, PROP_THREADS, 0, s>>>(P, r, on);
    return cudaGetLastError();
}

template <int DYN, int INTEG>
cudaError_t launch_append_t(const DevParams& P, cudaStream_t s) {
    k_append<DYN, INTEG><<<persistent_blocks((P.R + 127) / 128, 4), 128, 0, s>>>(P);
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

cudaError_t launch_begin(const DevParams& P, cudaStream_t s) {
    k_begin<<<persistent_blocks((P.R + 255) / 256, 2), 256, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_propagate(const DevParams& P, const kpx_debug_records* rec, cudaStream_t s) {
    KPX_DISPATCH(launch_propagate_t, P, rec, s);
}

cudaError_t launch_mark(const DevParams& P, cudaStream_t s) {
    k_mark<<<persistent_blocks((P.R + 255) / 256, 4), 256, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_scan(const DevParams& P, cudaStream_t s) {
    k_scan<<<persistent_blocks(P.n_win_tiles, 2), WIN_THREADS, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_append(const DevParams& P, cudaStream_t s) { KPX_DISPATCH(launch_append_t, P, s); }

cudaError_t launch_prune(const DevParams& P, cudaStream_t s) {
    k_prune<<<persistent_blocks(P.n_prune_tiles, 4), PRUNE_THREADS, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_end(const DevParams& P, cudaStream_t s) {
    k_end<<<1, 1, 0, s>>>(P);
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
