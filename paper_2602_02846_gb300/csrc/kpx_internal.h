// kpx_internal.h -- private declarations shared by the kernels and the C ABI.
//
// Everything here is an implementation detail of libkpx.so: the kernel
// parameter block, the workspace layout, and the launchers of the per-phase
// kernels.  The public surface is include/kpx.h.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "kpx.h"

namespace kpx {

constexpr uint64_t KEY_INF = ~0ull;

// node-set byte: bits 0-1 the set; bit 2 the memoised "a strict ancestor is
// dominated" flag; bit 3 "dominated": the node no longer holds its region's
// key (set by the append that replaces it as the region's owner).  Both flags
// are monotone: region keys only decrease.
enum : uint8_t { SET_A = 1, SET_I = 2, SET_T = 3, SET_MASK = 3, SET_ANC = 4, SET_DOM = 8 };

// work partitioning constants
constexpr int PROP_THREADS = 256;
constexpr int WIN_THREADS = 256;
constexpr int WIN_WORDS_PER_THREAD = 8;
constexpr int WIN_TILE_WORDS = WIN_THREADS * WIN_WORDS_PER_THREAD;   // 2048 words = 65536 slots
constexpr int PRUNE_THREADS = 256;
constexpr int PRUNE_PER_THREAD = 4;
constexpr int PRUNE_TILE = PRUNE_THREADS * PRUNE_PER_THREAD;         // 1024 nodes
constexpr int TRAJ_STAGE_ROWS = 65536;                               // trajectory gather chunk
// propagate order: each aligned chunk of ORDER_CHUNK slots (one node's
// samples at lambda = 128) is rolled out in ascending step count K
constexpr int ORDER_CHUNK = 128;
// obstacle broad phase: a uniform grid over the workspace box
constexpr int GRID_MAX_CELLS = 65536;
// Default obstacle-grid cell edge as a multiple of the mean box extent per
// axis: finer than the boxes themselves, so that a cell lists fewer boxes
// (measured: the Dubins forest 3 % and the quadcopter building 1 % faster at
// 0.75 than at 1; finer still is slower on the forest)
constexpr float GRID_SCALE_DEFAULT = 0.75f;
constexpr int GRID_MAX_AXIS = 64;
inline int64_t grid_entry_budget(int32_t n_obs) { return 32 * (int64_t)n_obs + 4096; }

// Parameter block passed by value to every kernel.
struct DevParams {
    // problem (FP32 throughout, as given by the caller)
    int32_t dyn, integ, n, m;
    float h;
    int32_t k_min, k_max;
    float u_lo[8], u_hi[8];
    float x_lo[16], x_hi[16];
    float param[8];
    float ws_lo[3], ws_hi[3];
    float goal_c[3], goal_r2;
    int32_t cost_kind;
    float w_effort;
    float mg, inv_mg, inv_tau_max, inv_mass;
    float inv_J[3], J[3];
    float dJ[3];                 // J[2] - J[1], J[0] - J[2], J[1] - J[0] (FP32, as the device would round them)
    int32_t iso_inertia;         // quadcopter: J[0] = J[1] = J[2] exactly (omega' = tau / J)
    int32_t sym_bounds;          // x_lo[d] = -x_hi[d] for every state component d >= 3 (bounds_ok<SYM>)
    float pos_lo[3], pos_hi[3];  // the workspace box intersected with the state bounds of x, y, z
    int32_t n_axes;
    int32_t ax_dim[8], ax_bins[8], ax_wrap[8];
    float ax_lo[8], ax_scale[8];
    // the same grid indexed by state component (0 bins: not a region axis);
    // id = sum over axes of cell * stride, stride = product of later axes' bins
    int32_t rg_bins[16], rg_wrap[16], rg_stride[16];
    float rg_lo[16], rg_scale[16];
    float start[16];
    // planner
    int32_t N, R, lambda_fixed, i_max;
    uint32_t seed_lo, seed_hi;
    int32_t flags, n_obs;
    int32_t va_cap;
    int32_t iter_limit;   // batch slots: iterate while iter < iter_limit (0: no limit, -1: vacant)
    int32_t prop_bps;     // host side: propagate blocks per SM (0: as many as fit)
    int64_t slot_cap, mask_words;
    int32_t n_win_tiles, n_prune_tiles;
    // obstacle grid: cell(c, axis a) = clamp(floor((c - ws_lo[a]) * grid_inv[a]), 0, grid_n[a] - 1)
    int32_t grid_n[3];
    float grid_inv[3];
    int32_t n_cells;
    int32_t grid_cap;     // entries reserved in cell_box
    int32_t grid_entries; // entries the grid build writes (computed on the host, <= grid_cap)
    // device arrays (inside the caller's workspace)
    kpx_device_header* hdr;
    float* x;
    float* u;
    uint16_t* K;
    int32_t* parent;
    uint64_t* key;
    int32_t* region;
    uint8_t* set;
    uint8_t* icount;
    uint64_t* region_key;
    uint64_t* region_snap;
    int32_t* region_owner;  // [R]: tree id holding the region's key, -1 if none
    int32_t* va0;
    int32_t* va1;
    int32_t* win_slot;
    uint32_t* win_mask;
    uint64_t* win_tiles;
    uint64_t* prune_tiles;
    float4* obs;          // [2*n_obs]: lo (x,y,z,0), hi (x,y,z,0)
    int32_t* box_cells;   // [6*n_obs]: per box cell range lo x,y,z, hi x,y,z
    int32_t* cell_start;  // [n_cells + 1]: CSR offsets into cell_box
    int2* cell_pair;      // [n_cells]: (cell_start[c], min(cell_start[c + 1], grid_cap)), one 8-byte load
    float4* cell_box;     // [2*grid_cap]: boxes of each cell, in box order
    uint32_t* clean;      // [N]: the epoch of the prune that found the node's strict ancestors not dominated
    int32_t* slot_region; // [slot_cap]: region of a winning slot (written by mark)
    uint8_t* slot_order;  // [slot_cap rounded up to ORDER_CHUNK]: per chunk, the slots (offsets in the chunk)
                          // in ascending K; null: slots in index order
    int32_t* path;        // [N] node ids root -> goal
    float* traj;          // staging: states [(TRAJ_STAGE_ROWS+1) n], controls [TRAJ_STAGE_ROWS m], steps
};

// FP32 cell index along one axis, identical on host and device (one
// rounding per operation, no contraction).  Monotone in c, so a box that
// contains a point always lists the point's cell.  t is clamped to
// [0, n - 1] in floating point first (fmaxf maps NaN to 0), so truncation
// equals floor and every input, NaN and infinities included, lands in a
// cell: the same index as clamp(floor(t), 0, n - 1).
__host__ __device__ inline int grid_cell(float c, float lo, float inv, int n) {
#ifdef __CUDA_ARCH__
    const float t = __fmul_rn(__fsub_rn(c, lo), inv);
#else
    volatile float d = c - lo;
    const float t = d * inv;
#endif
    return (int)fminf(fmaxf(t, 0.0f), (float)(n - 1));
}

// Workspace layout (byte offsets from the workspace base).
struct Layout {
    size_t hdr, obs, box_cells, cell_start, cell_pair, cell_box, x, u, K, parent, key, region, set, icount;
    size_t region_key, region_snap, region_owner, va0, va1, win_slot, win_mask, win_tiles, prune_tiles, clean,
        slot_region, slot_order, path, traj;
    size_t total;
    int32_t va_cap;
    int64_t slot_cap, mask_words;
    int32_t n_win_tiles, n_prune_tiles;
    int32_t traj_rows;
    int64_t region_cap;  // regions the arrays hold
};

// fills the per-component region fields from the per-axis ones
inline void fill_region_by_component(DevParams& P) {
    for (int d = 0; d < 16; ++d) {
        P.rg_bins[d] = 0;
        P.rg_wrap[d] = 0;
        P.rg_stride[d] = 0;
        P.rg_lo[d] = 0.0f;
        P.rg_scale[d] = 0.0f;
    }
    int stride = 1;
    for (int a = P.n_axes - 1; a >= 0; --a) {
        const int d = P.ax_dim[a];
        P.rg_bins[d] = P.ax_bins[a];
        P.rg_wrap[d] = P.ax_wrap[a];
        P.rg_lo[d] = P.ax_lo[a];
        P.rg_scale[d] = P.ax_scale[a];
        P.rg_stride[d] = stride;
        stride *= P.ax_bins[a];
    }
}

// The dynamics fields of the parameter block (kind, integrator, step, control
// and state boxes, constants); the planner and the refinement kernels share
// them, so their FP32 rollouts are the same arithmetic.
inline void fill_dynamics(DevParams& P, const kpx_dynamics* dyn) {
    const int n = dyn->kind == KPX_QUAD12 ? 12 : 6, m = dyn->kind == KPX_QUAD12 ? 4 : 3;
    P.dyn = dyn->kind;
    P.integ = dyn->integ;
    P.n = n;
    P.m = m;
    P.h = dyn->h;
    P.k_min = dyn->k_min;
    P.k_max = dyn->k_max;
    for (int i = 0; i < 8; ++i) {
        P.u_lo[i] = i < m ? dyn->u_lo[i] : 0.0f;
        P.u_hi[i] = i < m ? dyn->u_hi[i] : 0.0f;
        P.param[i] = dyn->param[i];
    }
    for (int i = 0; i < 16; ++i) {
        P.x_lo[i] = i < n ? dyn->x_lo[i] : -__builtin_huge_valf();
        P.x_hi[i] = i < n ? dyn->x_hi[i] : __builtin_huge_valf();
    }
    P.sym_bounds = 1;
    for (int i = 3; i < n; ++i)
        if (!(P.x_lo[i] == -P.x_hi[i])) P.sym_bounds = 0;  // a NaN bound is not symmetric
    if (dyn->kind == KPX_QUAD12) {
        P.mg = dyn->param[0] * dyn->param[1];
        P.inv_mg = 1.0f / P.mg;
        P.inv_mass = 1.0f / dyn->param[0];
        P.inv_tau_max = 1.0f / dyn->param[5];
        for (int i = 0; i < 3; ++i) {
            P.J[i] = dyn->param[2 + i];
            P.inv_J[i] = 1.0f / dyn->param[2 + i];
        }
        P.dJ[0] = P.J[2] - P.J[1];
        P.dJ[1] = P.J[0] - P.J[2];
        P.dJ[2] = P.J[1] - P.J[0];
        P.iso_inertia = (P.J[0] == P.J[1] && P.J[1] == P.J[2]) ? 1 : 0;
    }
}

// The position test of X_valid in one box per axis: x >= max(ws_lo, x_lo)
// holds exactly when x >= ws_lo and x >= x_lo (a NaN bound stays NaN, so
// every comparison with it still fails).  Call after the workspace and the
// state bounds are set.
inline void set_position_box(DevParams& P) {
    for (int a = 0; a < 3; ++a) {
        const float wl = P.ws_lo[a], wh = P.ws_hi[a], xl = P.x_lo[a], xh = P.x_hi[a];
        P.pos_lo[a] = (wl != wl || xl != xl) ? __builtin_nanf("") : (wl > xl ? wl : xl);
        P.pos_hi[a] = (wh != wh || xh != xh) ? __builtin_nanf("") : (wh < xh ? wh : xh);
    }
}

// Many problems in one launch per phase (kpx_batch.cu).
struct BatchHeader {
    unsigned long long prop_ticket[6];  // per dynamics class
    uint32_t scan_ticket, prune_ticket;
};

// Per-slot summary gathered by kpx_batch_poll (mirrors kpx_slot_state).
struct SlotState {
    int32_t status, iter, n_nodes, first_solution_iter;
    uint64_t goal_key;
    // device clock (ns): first active iteration, first solution (0: none),
    // end of the last iteration, and the poll itself
    uint64_t t_start_ns, t_first_solution_ns, t_last_ns, t_poll_ns;
};

struct BatchParams {
    int32_t B;       // problems, ordered by class
    int32_t lo, hi;  // class range for the per-class launches
    int32_t cls;     // class index (its ticket)
    const DevParams* Ps;     // [B] device copy of every problem's parameters
    BatchHeader* bh;
    int64_t* chunk_prefix;   // [B+1] propagate chunks (32 slots) before problem p
    int64_t* scan_prefix;    // [B+1] winner-scan tiles before p
    int64_t* win_prefix;     // [B+1] winners before p
    int64_t* prune_prefix;   // [B+1] prune tiles before p
    int64_t* order_prefix;   // [B+1] 128-slot order chunks before p (0 for a problem without the order)
    SlotState* slots;        // [B] poll staging
};

cudaError_t launch_batch_poll(const BatchParams& base, cudaStream_t s);

// cls_bps: per class, propagate blocks per SM (0: as many as fit)
cudaError_t launch_batch_iteration(const BatchParams& base, int n_classes, const int* cls_kind, const int* cls_lo,
                                   const int* cls_hi, const int* cls_bps, cudaStream_t s);

// launchers (kpx_kernels.cu); each returns the launch status
cudaError_t launch_init(const DevParams& P, bool first_time, cudaStream_t s);
cudaError_t launch_grid_build(const DevParams& P, cudaStream_t s);
// loop: in the loop body of a planner's graph (runs only while graph_pending > 0)
cudaError_t launch_begin(const DevParams& P, cudaStream_t s, bool loop = false);
cudaError_t launch_propagate(const DevParams& P, const kpx_debug_records* rec, cudaStream_t s);
cudaError_t launch_mark(const DevParams& P, cudaStream_t s);
cudaError_t launch_scan(const DevParams& P, cudaStream_t s);
// UpdateTree in two halves (kpx_phases.cuh): append (rows, keys, owners,
// capacity rule) and stage (the kept winners' end states and the goal test)
cudaError_t launch_append(const DevParams& P, cudaStream_t s);
cudaError_t launch_stage(const DevParams& P, cudaStream_t s);
cudaError_t launch_prune(const DevParams& P, cudaStream_t s);
cudaError_t launch_end(const DevParams& P, cudaStream_t s);
// the end of an iteration in the loop body of a planner's graph: counts the
// iteration off graph_pending; the body's last sets the loop's handle (1: run
// again)
cudaError_t launch_end_loop(const DevParams& P, cudaGraphConditionalHandle h, bool last, cudaStream_t s);
cudaError_t launch_path(const DevParams& P, cudaStream_t s);
// one bounded look-back wait that nothing releases (tests): records KPX_E_TIMEOUT
cudaError_t launch_wait_timeout(const DevParams& P, cudaStream_t s);
// a new region decomposition (already in P): node regions, region keys and
// owners, dominated bits (kpx_set_regions)
cudaError_t launch_remap_regions(const DevParams& P, cudaStream_t s);
cudaError_t launch_gather(const DevParams& P, int32_t first_row, int32_t rows, cudaStream_t s);
// computes the cached launch shapes (SM count, occupancy) outside any capture
void prepare_launches(const DevParams& P);

// fused iterations (kpx_fused.cu): CTAs of the single cluster that runs
// them for this problem's dynamics (0: unavailable on this device)
int fused_cluster_size(const DevParams& P);
// up to n_iter iterations in one launch while the problem stays small
// (n_iter < 0: the count the header's graph_pending holds at launch); the
// rest go to the phase kernels through graph_pending and, when use_handle,
// the graph's conditional handle (1: phase kernels needed)
cudaError_t launch_fused(const DevParams& P, int n_iter, cudaGraphConditionalHandle handle, int use_handle,
                         cudaStream_t s);

// trajectory refinement (kpx_adjoint.cu: objective, adjoint gradient and
// optimiser kernels; kpx_refine.cu: re-validation and the C ABI)
constexpr int REFINE_CKPT_STEPS = 32;  // integration steps per checkpoint interval
constexpr int REFINE_CKPT_WORDS = 16;  // 12 state floats, segment index, step in segment, pad
constexpr int REFINE_MAX_OBS = 4096;   // boxes staged in shared memory

struct RefineParams {
    // dynamics (the quadcopter's constants)
    float h, inv_mass, g, J[3], inv_J[3], mg, tau_max;
    // objective
    float w_obs, beta, inv_beta, margin, w_goal, goal[3], w_effort;
    int32_t count, max_segments, n_obs, max_total_steps, n_ckpt;
    const float* obs;       // [n_obs][6]
    const float* x0;        // [count][12]
    const float* u;         // [count][max_segments][4]
    const int32_t* steps;   // [count][max_segments]
    const int32_t* n_seg;   // [count]
    const int32_t* order;   // [count] processing order (null: index order)
    float* cost;            // [count]
    float* grad;            // [count][max_segments][4] (null: objective only)
    float* ckpt;            // [count][n_ckpt][REFINE_CKPT_WORDS]
    // broad phase of the box sum (null: every box at every step)
    struct RefineGridHeader* grid;
    int32_t* grid_off;      // [REFINE_GRID_CELLS + 1]
    uint16_t* grid_ids;     // [REFINE_GRID_ENTRIES]
};

// The box grid of the refinement objective: a uniform grid of
// REFINE_GRID_AXIS^3 cells over the boxes grown by the distance beyond which
// a box's term is dropped; cell c lists, in index order, every box whose
// grown box meets it.  Built on the device at each kpx_refine_eval call; the
// counters count the box tests of the call's kernels.
constexpr int REFINE_GRID_AXIS = 16;
constexpr int REFINE_GRID_CELLS = REFINE_GRID_AXIS * REFINE_GRID_AXIS * REFINE_GRID_AXIS;
constexpr int REFINE_GRID_ENTRIES = 1 << 22;
struct RefineGridHeader {
    float lo[3], inv_cs[3];
    int32_t ok, total;
    unsigned long long tests[4];  // forward candidates, forward near, backward candidates, backward near
};
static_assert(sizeof(RefineGridHeader) <= 256, "the grid header's slot");
constexpr size_t REFINE_GRID_BYTES = 256 + (size_t)(REFINE_GRID_CELLS + 1) * 4 + (size_t)REFINE_GRID_ENTRIES * 2;

struct AdamParams {
    int32_t count, max_segments;
    const int32_t* n_seg;
    float* u;
    const float* grad;
    float* m1;
    float* m2;
    float lo[4], hi[4];
    float lr, b1, b2, eps, c1, c2;  // c1 = 1 - b1^t, c2 = 1 - b2^t
};

cudaError_t launch_refine_eval(const RefineParams& R, cudaStream_t s);
cudaError_t launch_refine_adam(const AdamParams& A, cudaStream_t s);
cudaError_t launch_refine_keep_best(int32_t count, int32_t max_segments, const float* u, const float* cost,
                                    float* u_best, float* cost_best, cudaStream_t s);

}  // namespace kpx
