// kpx_fused.cu -- whole Kino-PAX+ iterations in one launch while the problem
// is small.
//
// With a few thousand slots per iteration, the eight phase kernels are
// bound by launch and dependency latency rather than by work: every kernel
// boundary costs a few microseconds, while the iteration's rollouts need a
// few in total.  This kernel runs whole iterations inside one thread-block
// cluster (up to 16 CTAs on 16 SMs).  A hardware cluster barrier
// (barrier.cluster, release/acquire) stands where the phase kernels have a
// kernel boundary, and the kernel loops over the iterations of one graph
// launch on the device.  The rollouts, the row writes of UpdateTree and
// PruneNodes are the functions the phase kernels call (kpx_phases.cuh), so
// the results are bit-identical to theirs.  Two things differ in how the
// work is arranged.  Each lane keeps its candidate's rollout in registers,
// and a winner appends its own row at its rank: no re-materialisation.  The
// V_U filter reads one region key per candidate, and the ranks in slot order
// come from a prefix over the warps' winner counts, exchanged through
// distributed shared memory: no region loop, no bitmask scan.
//
// A small obstacle grid is copied into shared memory at the start: the
// cluster barriers discard the L1 cache, and every rollout step reads the grid.
//
// Before each iteration the leader thread checks that the iteration fits: at
// most one 32-slot chunk per warp, and a tree of at most FUSED_MAX_NODES
// nodes.  When it does not fit, the kernel stops and leaves the number of
// iterations still owed to this graph launch in the header (graph_pending).
// It then sets the graph's conditional handle, so that the loop of phase
// kernels that follows it runs them (build_loop_graph in kpx_api.cu).
#include <cuda_runtime.h>

#include "kpx_phases.cuh"

namespace kpx {

namespace {

constexpr int FUSED_THREADS = 256;  // = WIN_THREADS = PRUNE_THREADS (block-wide units)
constexpr int FUSED_MAX_CLUSTER = 16;
constexpr int FUSED_MAX_NODES = 32768;
// obstacle grids up to this size are copied into shared memory: every cluster
// barrier (acquire) discards the L1 cache, and the rollouts read the grid at
// every step
constexpr size_t FUSED_GRID_SMEM_MAX = 180 * 1024;

__host__ __device__ inline size_t grid_start_bytes(int32_t n_cells) {
    return ((size_t)(n_cells + 1) * sizeof(int32_t) + 15) / 16 * 16;
}
static_assert(FUSED_THREADS == WIN_THREADS && FUSED_THREADS == PRUNE_THREADS, "block-wide units");

__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// distributed shared memory: a generic pointer to CTA `cta`'s copy of a
// shared variable (plain loads, stores and atomics reach it)
template <typename T>
__device__ __forceinline__ T* dsmem_generic(T* p, uint32_t cta) {
    uint64_t remote;
    asm volatile("mapa.u64 %0, %1, %2;" : "=l"(remote) : "l"(reinterpret_cast<uint64_t>(p)), "r"(cta));
    return reinterpret_cast<T*>(remote);
}

// distributed shared memory: a word of CTA `cta`'s copy of a shared array
__device__ __forceinline__ uint32_t dsmem_addr(const uint32_t* p, uint32_t cta) {
    const uint32_t local = (uint32_t)__cvta_generic_to_shared(p);
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(local), "r"(cta));
    return remote;
}

__device__ __forceinline__ void dsmem_store(const uint32_t* p, uint32_t cta, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(dsmem_addr(p, cta)), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t warp_sum_u32(uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// warp-wide, once per launch: add the launch's propagate counters to the
// header (the totals, and the last iteration's valid candidates)
__device__ __forceinline__ void flush_launch_counters(kpx_device_header* H, uint64_t steps, uint64_t tests,
                                                      uint32_t valid, uint32_t last) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        steps += __shfl_down_sync(FULL, steps, o);
        tests += __shfl_down_sync(FULL, tests, o);
        valid += __shfl_down_sync(FULL, valid, o);
        last += __shfl_down_sync(FULL, last, o);
    }
    if ((threadIdx.x & 31) == 0 && steps) {
        atomicAdd((unsigned long long*)&H->total_steps, (unsigned long long)steps);
        atomicAdd((unsigned long long*)&H->total_box_tests, (unsigned long long)tests);
        if (valid) atomicAdd((unsigned long long*)&H->total_valid, (unsigned long long)valid);
        if (last) atomicAdd((unsigned long long*)&H->last_valid, (unsigned long long)last);
    }
}

// An iteration's parameters as the leader's begin leaves them in the header.
// The leader's warp copies them into every CTA's shared memory before the
// barrier that publishes them, so that after it each warp reads them from
// its own SM instead of all warps of the cluster reading CTA 0's.
struct IterParams {
    int64_t n_slots;
    int32_t ctl, lambda, iter, n_nodes, va_sel, epoch;
};
static_assert(sizeof(IterParams) == 32, "two 16-byte words");

// warp 0 of CTA 0, after the leader's begin: lane c writes CTA c's copy
__device__ __forceinline__ void publish_iteration(const kpx_device_header* H, IterParams* s_it, int n_cta) {
    __syncwarp();
    const int lane = threadIdx.x & 31;
    if (lane < n_cta) {
        IterParams v;
        v.n_slots = H->n_slots;
        v.ctl = H->graph_ctl;
        v.lambda = H->lambda;
        v.iter = H->iter;
        v.n_nodes = H->n_nodes;
        v.va_sel = H->va_sel;
        v.epoch = H->epoch;
        *dsmem_generic(s_it, (uint32_t)lane) = v;
    }
}

// Leader only: decide whether the next iteration runs here; if so, begin it.
// remaining: iterations this graph launch still owes (including this one).
__device__ __forceinline__ void fused_begin(const DevParams& P, kpx_device_header* H, int remaining,
                                            int64_t max_slots) {
    int ctl = 0;
    if (remaining <= 0 || !problem_runs(P, H)) {
        H->graph_pending = 0;  // done, or every further iteration is a no-op
    } else {
        const int64_t n_slots = (int64_t)H->count_A * begin_lambda(P, H->count_A);
        if (n_slots > max_slots || H->n_nodes > FUSED_MAX_NODES) {
            H->graph_pending = remaining;  // too large: the phase kernels take over
        } else {
            ctl = 1 | (begin_needs_snapshot(P, H) ? 2 : 0);
            begin_counters(P, H);
        }
    }
    H->graph_ctl = ctl;
}

template <int DYN, int INTEG>
__global__ void __launch_bounds__(FUSED_THREADS, 1)
    k_fused(DevParams P, int n_iter, cudaGraphConditionalHandle handle, int use_handle, int grid_smem) {
    extern __shared__ __align__(16) unsigned char fused_grid[];
    __shared__ uint32_t s_prefix;
    __shared__ int32_t s_parent[PRUNE_TILE];
    __shared__ uint8_t s_set[PRUNE_TILE];
    __shared__ uint8_t s_icount[PRUNE_TILE];
    __shared__ uint32_t s_counts[PRUNE_ROUND_WARPS];
    __shared__ uint32_t s_cnt[FUSED_MAX_CLUSTER * (FUSED_THREADS / 32)];  // winners per chunk (every CTA's copy)
    // While the launch runs, the header lives in CTA 0's shared memory: the
    // leader's bookkeeping stays on the SM, and the few header updates of
    // other CTAs (a status, the goal key) reach it over distributed shared
    // memory instead of L2 (each cluster barrier's acquire would otherwise
    // send header reads back to L2).  What every warp needs in each iteration
    // comes from its own CTA's copy of the parameters (s_it), and the
    // counters stay in registers until the launch ends.  The header is copied
    // in here and written back before the kernel exits.
    __shared__ __align__(16) kpx_device_header s_hdr;
    __shared__ __align__(16) IterParams s_it;  // this CTA's copy of the iteration's parameters
    constexpr int HDR_WORDS = (int)(sizeof(kpx_device_header) / sizeof(uint32_t));
    static_assert(sizeof(kpx_device_header) % sizeof(uint32_t) == 0, "header size");
    if (blockIdx.x == 0) {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(P.hdr);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&s_hdr);
        for (int i = threadIdx.x; i < HDR_WORDS; i += FUSED_THREADS) dst[i] = src[i];
        __syncthreads();
    }
    kpx_device_header* H = dsmem_generic(&s_hdr, 0);
    const int lane = threadIdx.x & 31;
    const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
    const int n_cta = (int)gridDim.x;  // the grid is one cluster
    const int64_t gtid = (int64_t)blockIdx.x * FUSED_THREADS + threadIdx.x;
    const int64_t gthreads = (int64_t)n_cta * FUSED_THREADS;
    const int n_chunks = n_cta * (FUSED_THREADS / 32);  // one per warp of the cluster
    const bool early = (P.flags & KPX_FLAG_EARLY_REJECT) != 0;
    GridView G{P.cell_start, P.cell_box};
    if (grid_smem) {  // the obstacle grid is read-only while planning
        int32_t* sc = reinterpret_cast<int32_t*>(fused_grid);
        float4* sb = reinterpret_cast<float4*>(fused_grid + grid_start_bytes(P.n_cells));
        for (int i = threadIdx.x; i <= P.n_cells; i += FUSED_THREADS) sc[i] = P.cell_start[i];
        for (int i = threadIdx.x; i < 2 * P.grid_entries; i += FUSED_THREADS) sb[i] = P.cell_box[i];
        __syncthreads();
        G = GridView{sc, sb};
    }
    if (n_iter < 0) n_iter = s_hdr.graph_pending;  // read by the leader (CTA 0) only
    const bool lead_warp = blockIdx.x == 0 && threadIdx.x < 32;
    // the leader's warp keeps the books through CTA 0's own window
    kpx_device_header* HL = &s_hdr;
    if (lead_warp) {
        if (leader) fused_begin(P, HL, n_iter, gthreads);
        publish_iteration(HL, &s_it, n_cta);
    }
    int done = 0;
    // the propagate counters (integration steps, box tests, valid candidates)
    // stay in registers for the whole launch and reach the header once at its
    // end: they are statistics, and no decision of the leader reads them
    uint64_t acc_steps = 0, acc_tests = 0;
    uint32_t acc_valid = 0, last_valid = 0;
    int pA = 0, pI = 0, pT = 0;  // V_A, V_I, V_T sizes of this thread's nodes in the latest iteration
    bool merged = false;  // the last barrier already published this iteration's parameters
    for (;;) {
        if (!merged) cluster_barrier();
        // this iteration's parameters, published by the barrier (this CTA's
        // copy): all of them are taken here, so the leader's warp may write
        // the next iteration's while the cluster is still in this one
        const IterParams it = s_it;
        const int ctl = it.ctl;
        if (!(ctl & 1)) break;
        const int64_t n_slots = it.n_slots;
        const int lam = it.lambda;
        const uint32_t iter = (uint32_t)it.iter;
        const int n_old = it.n_nodes;  // the tree's size before this iteration's appends
        const int32_t* va = it.va_sel ? P.va1 : P.va0;
        int32_t* va_next = it.va_sel ? P.va0 : P.va1;
        const uint32_t epoch = (uint32_t)it.epoch;
        if (ctl & 2) {  // region snapshot for the capacity rule
            for (int64_t r = gtid; r < P.R; r += gthreads) P.region_snap[r] = P.region_key[r];
            cluster_barrier();
        }
        // propagate (Alg. 2): one chunk of 32 / g slots per warp, warp-major
        // across the CTAs; g lanes share a rollout when the slots fill at
        // most half of the cluster's threads.  The lane that keeps a
        // candidate holds it in registers.
        const int g = early ? 1 : coop_lanes(n_slots, gthreads);
        const int64_t chunk = (int64_t)(threadIdx.x >> 5) * n_cta + blockIdx.x;
        const int64_t slot = chunk * (32 / g) + lane / g;
        Candidate<DYN, INTEG> C;
        C.ok = false;
        {
            uint32_t steps = 0, tests = 0, n_valid = 0;
            const bool live = slot < n_slots;
            if (g > 1) {  // all lanes of the warp take part
                if (grid_smem)
                    roll_candidate_coop<DYN, INTEG, true>(P, G, lam, iter, va, live, slot, g, C, steps, tests);
                else
                    roll_candidate_coop<DYN, INTEG, false>(P, G, lam, iter, va, live, slot, g, C, steps, tests);
            } else if (live) {
                if (early) {
                    if (grid_smem)
                        roll_candidate<DYN, INTEG, true>(P, G, lam, iter, va, true, slot, C, steps, tests);
                    else
                        roll_candidate<DYN, INTEG, false>(P, G, lam, iter, va, true, slot, C, steps, tests);
                } else if (DYN == KPX_DI6) {  // a short step: nothing to overlap
                    if (grid_smem)
                        roll_candidate<DYN, INTEG, true>(P, G, lam, iter, va, false, slot, C, steps, tests);
                    else
                        roll_candidate<DYN, INTEG, false>(P, G, lam, iter, va, false, slot, C, steps, tests);
                } else if (grid_smem) {
                    roll_candidate_ahead<DYN, INTEG, true>(P, G, lam, iter, va, slot, C, steps, tests);
                } else {
                    roll_candidate_ahead<DYN, INTEG, false>(P, G, lam, iter, va, slot, C, steps, tests);
                }
            }
            n_valid = C.ok ? 1u : 0u;
            acc_steps += steps;
            acc_tests += tests;
            acc_valid += n_valid;
            last_valid = n_valid;
        }
        cluster_barrier();
        // the V_U filter and the winner ranks in slot order: a valid
        // candidate is its region's winner when the region holds its key;
        // each warp publishes its winner count to every CTA of the cluster
        // (lane c stores it into CTA c's array, over distributed shared
        // memory), indexed by chunk, so that the ranks read local words
        // (a valid candidate also reads its region's key node, which only
        // the region's winner rewrites, in the append phase: one L2 round
        // trip fewer there)
        bool won = false;
        int owner = -1;
        if (C.ok) {
            const uint64_t rk = __ldcg(&P.region_key[C.r]);
            owner = __ldcg(&P.region_owner[C.r]);
            won = rk == C.key;
        }
        // CTA 0 prunes tile 0: it stages the tile now, in the same round
        // trip, and the winners that take a region from one of its nodes
        // write that node's new set byte into the staged copy as well
        if (blockIdx.x == 0) stage_tile(P, 0, n_old, s_parent, s_set, s_icount);
        const uint32_t word = __ballot_sync(FULL, won);
        if (lane < n_cta) dsmem_store(s_cnt + chunk, (uint32_t)lane, (uint32_t)__popc(word));
        cluster_barrier();
        // the winners kept: every thread derives them alike (prune uses them
        // too, so it reads no header field the leader may rewrite at its end)
        int kept;
        {
            uint32_t before = 0, total = 0;
            for (int k = lane; k < n_chunks; k += 32) {
                const uint32_t v = *(volatile const uint32_t*)&s_cnt[k];
                total += v;
                if (k < chunk) before += v;
            }
            before = warp_sum_u32(before);
            total = warp_sum_u32(total);
            const int W = (int)total;
            const int room = P.N - n_old;
            kept = W < room ? W : room;
            if (leader) {
                H->n_win = W;
                H->n_kept = kept;
                if (W > kept) set_status(H, KPX_TREE_FULL);
            }
            // UpdateTree (Alg. 4): each winner appends itself at its rank
            if (won) {
                const int rank = (int)(before + __popc(word & ((1u << lane) - 1u)));
                append_row<DYN, INTEG>(P, H, rank, kept, n_old, C.R, C.c, C.r, owner, dsmem_generic(s_set, 0));
            }
        }
        cluster_barrier();
        // prune (Alg. 3) + compaction of the next V_A
        const int total = n_old + kept;
        const int n_tiles = (total + PRUNE_TILE - 1) / PRUNE_TILE;
        // one tile: CTA 0 prunes it alone, and its leader ends this iteration
        // and begins the next before the barrier, which then also publishes
        // the next iteration's parameters (no barrier at the top)
        merged = n_tiles <= 1;
        // the set sizes stay in registers: every begin resets the header's,
        // so only the launch's last iteration reaches it, at the end
        pA = pI = pT = 0;
        for (int t = blockIdx.x; t < n_tiles; t += n_cta)
            prune_tile(P, H, (uint32_t)t, n_tiles, n_old, total, epoch, va_next, s_parent, s_set, s_icount, s_counts,
                       s_prefix, pA, pI, pT, t == 0);
        ++done;
        if (merged && lead_warp) {  // prune_tile ended with a CTA barrier
            if (leader) {
                end_counters(P, HL, false);
                HL->fused_iterations += 1;
                fused_begin(P, HL, n_iter - done, gthreads);
            }
            publish_iteration(HL, &s_it, n_cta);
        }
        cluster_barrier();
        if (!merged && lead_warp) {
            if (leader) {
                end_counters(P, HL, false);
                HL->fused_iterations += 1;
                fused_begin(P, HL, n_iter - done, gthreads);
            }
            publish_iteration(HL, &s_it, n_cta);
        }
    }
    if (leader && done > 0) H->t_last_ns = globaltimer_ns();  // the last iteration's end
    // every begin reset last_valid, so the header holds the sums over the
    // launch's iterations (total_valid) and over its last one (last_valid)
    flush_launch_counters(H, acc_steps, acc_tests, acc_valid, last_valid);
    flush_prune_counters(H, pA, pI, pT);
    // every CTA has read the header for the last time; CTA 0 writes it back
    cluster_barrier();
    if (blockIdx.x == 0) {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(&s_hdr);
        uint32_t* dst = reinterpret_cast<uint32_t*>(P.hdr);
        for (int i = threadIdx.x; i < HDR_WORDS; i += FUSED_THREADS) dst[i] = src[i];
        if (leader && use_handle) cudaGraphSetConditional(handle, s_hdr.graph_pending > 0 ? 1u : 0u);
    }
}

template <int DYN, int INTEG>
int fused_cluster_size_t(const DevParams&, int) {
    static int size = -1;
    if (size < 0) {
        size = 0;
        if (cudaFuncSetAttribute(k_fused<DYN, INTEG>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess) {
            cudaGetLastError();
        }
        if (cudaFuncSetAttribute(k_fused<DYN, INTEG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)FUSED_GRID_SMEM_MAX) != cudaSuccess) {
            cudaGetLastError();
            return size;  // 0: unavailable
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(FUSED_MAX_CLUSTER);
        cfg.blockDim = dim3(FUSED_THREADS);
        cfg.dynamicSmemBytes = FUSED_GRID_SMEM_MAX;  // the cluster must fit with a staged grid
        int cl = 0;
        if (cudaOccupancyMaxPotentialClusterSize(&cl, (const void*)k_fused<DYN, INTEG>, &cfg) != cudaSuccess) {
            cudaGetLastError();
            cl = 0;
        }
        // a power of two up to 16 (the grid is one cluster)
        int c = 1;
        while (c * 2 <= cl && c * 2 <= FUSED_MAX_CLUSTER) c *= 2;
        size = c >= 4 ? c : 0;
    }
    return size;
}

template <int DYN, int INTEG>
cudaError_t launch_fused_t(const DevParams& P, int n_iter, cudaGraphConditionalHandle handle, int use_handle,
                           cudaStream_t s) {
    const int cl = fused_cluster_size_t<DYN, INTEG>(P, 0);
    if (cl == 0) return cudaErrorNotSupported;
    const size_t grid_bytes = grid_start_bytes(P.n_cells) + (size_t)P.grid_entries * 2 * sizeof(float4);
    const int grid_smem = P.n_obs > 0 && grid_bytes <= FUSED_GRID_SMEM_MAX ? 1 : 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(FUSED_THREADS);
    cfg.dynamicSmemBytes = grid_smem ? grid_bytes : 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_fused<DYN, INTEG>, P, n_iter, handle, use_handle, grid_smem);
}

#define KPX_FUSED_DISPATCH(FN, P, ...)                                                   \
    switch ((P).dyn * 2 + (P).integ) {                                                  \
        case KPX_DI6 * 2 + KPX_EULER: return FN<KPX_DI6, KPX_EULER>(P, __VA_ARGS__);         \
        case KPX_DI6 * 2 + KPX_RK4: return FN<KPX_DI6, KPX_RK4>(P, __VA_ARGS__);             \
        case KPX_DUBINS6 * 2 + KPX_EULER: return FN<KPX_DUBINS6, KPX_EULER>(P, __VA_ARGS__); \
        case KPX_DUBINS6 * 2 + KPX_RK4: return FN<KPX_DUBINS6, KPX_RK4>(P, __VA_ARGS__);     \
        case KPX_QUAD12 * 2 + KPX_EULER: return FN<KPX_QUAD12, KPX_EULER>(P, __VA_ARGS__);   \
        case KPX_QUAD12 * 2 + KPX_RK4: return FN<KPX_QUAD12, KPX_RK4>(P, __VA_ARGS__);       \
        default: break;                                                                 \
    }

}  // namespace

int fused_cluster_size(const DevParams& P) {
    KPX_FUSED_DISPATCH(fused_cluster_size_t, P, 0);
    return 0;
}

cudaError_t launch_fused(const DevParams& P, int n_iter, cudaGraphConditionalHandle handle, int use_handle,
                         cudaStream_t s) {
    KPX_FUSED_DISPATCH(launch_fused_t, P, n_iter, handle, use_handle, s);
    return cudaErrorInvalidValue;
}

}  // namespace kpx
