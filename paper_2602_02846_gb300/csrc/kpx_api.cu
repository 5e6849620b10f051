// kpx_api.cu -- host side of the C ABI declared in include/kpx.h.
//
// Validates the problem, lays the planner's arrays out in the caller's
// device workspace, and enqueues the per-phase kernels on the caller's
// stream.  Allocates no device memory.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <algorithm>
#include <atomic>
#include <vector>

#include <cuda_runtime.h>

#include "kpx_internal.h"

using namespace kpx;

// The second stream and the two events with which a captured iteration forks
// the winners' re-integration off the main chain and joins it again.
struct SideBranch {
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
};

struct kpx_planner {
    DevParams P;
    Layout L;
    cudaStream_t stream;
    char* ws;
    size_t ws_bytes;
    std::string err;
    // kpx_iterate's CUDA graph (built on first use; launched on `stream`)
    int graph_state = 0;  // 0 not decided, 1 graph, -1 unavailable (plain launches)
    bool graph_fused = false;  // the graph starts with the fused kernel
    cudaStream_t capture_stream = nullptr;
    SideBranch side;                       // used while capturing the loop body
    cudaGraph_t loop_graph = nullptr;      // kept: its count node is updated before each launch
    cudaGraphExec_t loop_exec = nullptr;
    cudaGraphNode_t count_node = nullptr;  // memset node: the launch's iteration count
    int32_t count_value = 1;               // the count node's current value
    float grid_scale = GRID_SCALE_DEFAULT;  // obstacle-grid cell edge / mean box extent
    std::vector<float> host_obs; // the boxes (lo xyz, hi xyz), to rebuild the grid
    std::vector<float4> upload;  // source of kpx_create's obstacle copy, alive until destroy
};

// Many problems iterated together (one launch per phase for all of them).
struct kpx_batch {
    int B = 0;
    std::vector<kpx_planner*> members;   // ordered by dynamics class
    std::vector<int> member_of_index;    // caller's index -> position in members
    int n_classes = 0;
    int cls_kind[6] = {}, cls_lo[6] = {}, cls_hi[6] = {};
    int cls_bps[6] = {};  // propagate blocks per SM per class (0: as many as fit)
    kpx::BatchParams BP{};
    cudaStream_t stream = nullptr;
    std::string err;
    int graph_state = 0;  // 0 not tried, 1 ready, -1 plain launches
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph_one = nullptr;
    cudaGraphExec_t graph_many = nullptr;
    std::vector<std::vector<float4>> staging;  // per member: obstacles of the last (re)assignment
    std::vector<kpx::SlotState> poll_buf;
    kpx_device_header* parking = nullptr;     // [B] headers that vacant slots point at
    std::vector<DevParams> parked;             // host source of a vacant slot's device parameters
};

namespace {

thread_local std::string g_create_error;

constexpr int kStateDim[3] = {6, 6, 12};
constexpr int kControlDim[3] = {3, 3, 4};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool finite(float v) { return std::isfinite(v); }

// Validates a region decomposition for an n-dimensional state; sets R to
// its region count.  Returns an empty string when valid.
std::string check_axes(int n, int32_t n_axes, const kpx_region_axis* axis, int64_t& R) {
    if (n_axes < 1 || n_axes > 8 || !axis) return "n_axes must be in [1, 8]";
    R = 1;
    for (int a = 0; a < n_axes; ++a) {
        const kpx_region_axis& ax = axis[a];
        if (ax.state_dim < 0 || ax.state_dim >= n) return "region axis state_dim out of range";
        if (ax.bins < 1 || ax.bins > (1 << 20)) return "region axis bins out of range";
        if (!finite(ax.lo) || !finite(ax.hi) || !(ax.hi > ax.lo)) return "region axis needs finite lo < hi";
        for (int b = 0; b < a; ++b)
            if (axis[b].state_dim == ax.state_dim) return "a state component may appear in one region axis only";
        R *= ax.bins;
        if (R > (1 << 28)) return "too many regions (> 2^28)";
    }
    return "";
}

// the per-axis region fields of the parameter block
void fill_axes(DevParams& P, int32_t n_axes, const kpx_region_axis* axis) {
    P.n_axes = n_axes;
    int64_t R = 1;
    for (int a = 0; a < n_axes; ++a) {
        const kpx_region_axis& ax = axis[a];
        P.ax_dim[a] = ax.state_dim;
        P.ax_bins[a] = ax.bins;
        P.ax_wrap[a] = ax.wrap ? 1 : 0;
        P.ax_lo[a] = ax.lo;
        const float width = ax.hi - ax.lo;
        P.ax_scale[a] = (float)ax.bins / width;
        R *= ax.bins;
    }
    fill_region_by_component(P);
    P.R = (int32_t)R;
}

// Validates the scalar configuration; returns an empty string when valid.
std::string check_config(const kpx_dynamics* dyn, const kpx_config* cfg, int32_t n_obs) {
    if (!dyn || !cfg) return "null dynamics or config";
    if (dyn->kind < 0 || dyn->kind > 2) return "unknown dynamics kind";
    if (dyn->integ != KPX_EULER && dyn->integ != KPX_RK4) return "unknown integrator";
    if (!(dyn->h > 0.0f) || !finite(dyn->h)) return "integration step h must be positive and finite";
    if (dyn->k_min < 1 || dyn->k_max < dyn->k_min || dyn->k_max > 4096) return "need 1 <= k_min <= k_max <= 4096";
    const int n = kStateDim[dyn->kind], m = kControlDim[dyn->kind];
    for (int i = 0; i < m; ++i)
        if (!finite(dyn->u_lo[i]) || !finite(dyn->u_hi[i]) || dyn->u_lo[i] > dyn->u_hi[i])
            return "control bounds must be finite with lo <= hi";
    for (int i = 0; i < n; ++i)
        if (std::isnan(dyn->x_lo[i]) || std::isnan(dyn->x_hi[i]) || dyn->x_lo[i] > dyn->x_hi[i])
            return "state bounds must satisfy lo <= hi";
    if (dyn->kind == KPX_QUAD12) {
        for (int i = 0; i < 6; ++i)
            if (!finite(dyn->param[i])) return "quadcopter parameters must be finite";
        if (!(dyn->param[0] > 0.0f) || !(dyn->param[2] > 0.0f) || !(dyn->param[3] > 0.0f) ||
            !(dyn->param[4] > 0.0f) || !(dyn->param[5] > 0.0f))
            return "quadcopter mass, inertia and tau_max must be positive";
    }
    if (cfg->tree_cap < 1 || cfg->tree_cap > (1 << 28)) return "tree_cap must be in [1, 2^28]";
    if (cfg->samples_per_node < 0 || cfg->samples_per_node > 65536) return "samples_per_node must be in [0, 65536]";
    int64_t R = 0;
    std::string msg = check_axes(n, cfg->n_axes, cfg->axis, R);
    if (!msg.empty()) return msg;
    if (cfg->region_capacity != 0 && (cfg->region_capacity < R || cfg->region_capacity > (1 << 28)))
        return "region_capacity must be 0 or in [the grid's region count, 2^28]";
    if (cfg->i_max < 0 || cfg->i_max > 254) return "i_max must be in [0, 254]";
    if (n_obs < 0 || n_obs > 6000) return "obstacle count must be in [0, 6000]";
    return "";
}

Layout make_layout(const kpx_dynamics* dyn, const kpx_config* cfg, int32_t n_obs) {
    Layout L{};
    const int n = kStateDim[dyn->kind], m = kControlDim[dyn->kind];
    const int64_t N = cfg->tree_cap;
    int64_t R = 1;
    for (int a = 0; a < cfg->n_axes; ++a) R *= cfg->axis[a].bins;
    if (cfg->region_capacity > R) R = cfg->region_capacity;  // room for a finer grid later
    L.region_cap = R;
    L.va_cap = (int32_t)(N < R ? N : R);
    L.slot_cap = cfg->samples_per_node > 0 ? (int64_t)L.va_cap * cfg->samples_per_node : N;
    L.mask_words = (L.slot_cap + 31) / 32;
    L.n_win_tiles = (int32_t)((L.mask_words + WIN_TILE_WORDS - 1) / WIN_TILE_WORDS);
    L.n_prune_tiles = (int32_t)((N + PRUNE_TILE - 1) / PRUNE_TILE);
    L.traj_rows = (int32_t)(N < TRAJ_STAGE_ROWS ? N + 1 : TRAJ_STAGE_ROWS);
    size_t off = 0;
    auto seg = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    L.hdr = seg(sizeof(kpx_device_header));
    L.obs = seg((size_t)(n_obs > 0 ? n_obs : 1) * 2 * sizeof(float4));
    L.box_cells = seg((size_t)(n_obs > 0 ? n_obs : 1) * 6 * sizeof(int32_t));
    L.cell_start = seg((size_t)(GRID_MAX_CELLS + 1) * sizeof(int32_t));
    L.cell_pair = seg((size_t)GRID_MAX_CELLS * sizeof(int2));
    L.cell_box = seg((size_t)grid_entry_budget(n_obs) * 2 * sizeof(float4));
    L.x = seg((size_t)n * N * sizeof(float));
    L.u = seg((size_t)m * N * sizeof(float));
    L.K = seg((size_t)N * sizeof(uint16_t));
    L.parent = seg((size_t)N * sizeof(int32_t));
    L.key = seg((size_t)N * sizeof(uint64_t));
    L.region = seg((size_t)N * sizeof(int32_t));
    L.set = seg((size_t)N);
    L.icount = seg((size_t)N);
    L.region_key = seg((size_t)R * sizeof(uint64_t));
    L.region_snap = seg((size_t)R * sizeof(uint64_t));
    L.region_owner = seg((size_t)R * sizeof(int32_t));
    L.va0 = seg((size_t)L.va_cap * sizeof(int32_t));
    L.va1 = seg((size_t)L.va_cap * sizeof(int32_t));
    L.win_slot = seg((size_t)R * sizeof(int32_t));
    L.win_mask = seg((size_t)L.mask_words * sizeof(uint32_t));
    L.win_tiles = seg((size_t)L.n_win_tiles * sizeof(uint64_t));
    L.prune_tiles = seg((size_t)L.n_prune_tiles * sizeof(uint64_t));
    L.clean = seg((size_t)N * sizeof(uint32_t));
    L.slot_region = seg((size_t)L.slot_cap * sizeof(int32_t));
    L.slot_order = seg((size_t)((L.slot_cap + ORDER_CHUNK - 1) / ORDER_CHUNK) * ORDER_CHUNK);
    L.path = seg((size_t)N * sizeof(int32_t));
    L.traj = seg((size_t)L.traj_rows * (n + m + 1) * sizeof(float));
    L.total = off;
    return L;
}

// FP32 membership of x in X_valid, with the same comparisons as the kernels.
bool host_point_valid(const DevParams& P, const float* x, const float* obs, int n_obs) {
    for (int d = 0; d < P.n; ++d)
        if (!(x[d] >= P.x_lo[d] && x[d] <= P.x_hi[d])) return false;
    for (int a = 0; a < 3; ++a)
        if (!(x[a] >= P.ws_lo[a] && x[a] <= P.ws_hi[a])) return false;
    for (int b = 0; b < n_obs; ++b) {
        const float* o = obs + 6 * b;
        if (x[0] >= o[0] && x[0] <= o[3] && x[1] >= o[1] && x[1] <= o[4] && x[2] >= o[2] && x[2] <= o[5])
            return false;
    }
    return true;
}

// Resolution of the obstacle grid: cells about the mean box extent per axis
// (at most GRID_MAX_AXIS per axis and GRID_MAX_CELLS in all), coarsened until
// the cell lists fit the reserved entries.  Uses the same FP32 cell map as
// the device, so the entry count here is the one the device build produces.
// Obstacle grid: cells of about `scale` x the mean box extent per axis
// (capped by GRID_MAX_AXIS, GRID_MAX_CELLS and the entry budget).  Any grid
// gives the same verdicts (the broad phase is exact); the scale only moves
// work between cell lookups and box tests.
void choose_grid(DevParams& P, const float* aabb, int n_obs, float scale = GRID_SCALE_DEFAULT) {
    P.grid_cap = (int32_t)grid_entry_budget(n_obs);
    int g[3] = {1, 1, 1};
    float W[3];
    for (int a = 0; a < 3; ++a) W[a] = P.ws_hi[a] - P.ws_lo[a];
    if (n_obs > 0) {
        for (int a = 0; a < 3; ++a) {
            if (!(W[a] > 0.0f)) continue;
            double sum = 0.0;
            for (int b = 0; b < n_obs; ++b) {
                double e = (double)aabb[6 * b + 3 + a] - (double)aabb[6 * b + a];
                sum += e < (double)W[a] ? e : (double)W[a];
            }
            double mean = sum / n_obs * (double)scale;
            if (mean < (double)W[a] / GRID_MAX_AXIS) mean = (double)W[a] / GRID_MAX_AXIS;
            int ga = (int)((double)W[a] / mean);
            g[a] = ga < 1 ? 1 : (ga > GRID_MAX_AXIS ? GRID_MAX_AXIS : ga);
        }
    }
    for (;;) {
        while ((int64_t)g[0] * g[1] * g[2] > GRID_MAX_CELLS) {
            int big = g[0] >= g[1] && g[0] >= g[2] ? 0 : (g[1] >= g[2] ? 1 : 2);
            g[big] = (g[big] + 1) / 2;
        }
        for (int a = 0; a < 3; ++a) {
            P.grid_n[a] = g[a];
            P.grid_inv[a] = W[a] > 0.0f ? (float)g[a] / W[a] : 0.0f;
        }
        int64_t entries = 0;
        for (int b = 0; b < n_obs; ++b) {
            int64_t cells = 1;
            for (int a = 0; a < 3; ++a) {
                const int c0 = grid_cell(aabb[6 * b + a], P.ws_lo[a], P.grid_inv[a], g[a]);
                const int c1 = grid_cell(aabb[6 * b + 3 + a], P.ws_lo[a], P.grid_inv[a], g[a]);
                cells *= (int64_t)(c1 - c0 + 1);
            }
            entries += cells;
        }
        P.grid_entries = (int32_t)(entries < P.grid_cap ? entries : P.grid_cap);
        if (entries <= P.grid_cap || (g[0] == 1 && g[1] == 1 && g[2] == 1)) break;
        int big = g[0] >= g[1] && g[0] >= g[2] ? 0 : (g[1] >= g[2] ? 1 : 2);
        g[big] = (g[big] + 1) / 2;
    }
    P.n_cells = g[0] * g[1] * g[2];
}

kpx_status fail(kpx_planner* p, kpx_status st, const std::string& msg) {
    if (p) p->err = msg;
    return st;
}

kpx_status cuda_fail(kpx_planner* p, cudaError_t e, const char* where) {
    std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
    if (p) p->err = msg;
    return KPX_E_CUDA;
}

void bind_pointers(kpx_planner* p) {
    char* b = p->ws;
    const Layout& L = p->L;
    DevParams& P = p->P;
    P.hdr = reinterpret_cast<kpx_device_header*>(b + L.hdr);
    P.obs = reinterpret_cast<float4*>(b + L.obs);
    P.box_cells = reinterpret_cast<int32_t*>(b + L.box_cells);
    P.cell_start = reinterpret_cast<int32_t*>(b + L.cell_start);
    P.cell_pair = reinterpret_cast<int2*>(b + L.cell_pair);
    P.cell_box = reinterpret_cast<float4*>(b + L.cell_box);
    P.x = reinterpret_cast<float*>(b + L.x);
    P.u = reinterpret_cast<float*>(b + L.u);
    P.K = reinterpret_cast<uint16_t*>(b + L.K);
    P.parent = reinterpret_cast<int32_t*>(b + L.parent);
    P.key = reinterpret_cast<uint64_t*>(b + L.key);
    P.region = reinterpret_cast<int32_t*>(b + L.region);
    P.set = reinterpret_cast<uint8_t*>(b + L.set);
    P.icount = reinterpret_cast<uint8_t*>(b + L.icount);
    P.region_key = reinterpret_cast<uint64_t*>(b + L.region_key);
    P.region_snap = reinterpret_cast<uint64_t*>(b + L.region_snap);
    P.region_owner = reinterpret_cast<int32_t*>(b + L.region_owner);
    P.va0 = reinterpret_cast<int32_t*>(b + L.va0);
    P.va1 = reinterpret_cast<int32_t*>(b + L.va1);
    P.win_slot = reinterpret_cast<int32_t*>(b + L.win_slot);
    P.win_mask = reinterpret_cast<uint32_t*>(b + L.win_mask);
    P.win_tiles = reinterpret_cast<uint64_t*>(b + L.win_tiles);
    P.prune_tiles = reinterpret_cast<uint64_t*>(b + L.prune_tiles);
    P.clean = reinterpret_cast<uint32_t*>(b + L.clean);
    P.slot_region = reinterpret_cast<int32_t*>(b + L.slot_region);
    P.slot_order = (P.flags & KPX_FLAG_NO_SLOT_ORDER) ? nullptr : reinterpret_cast<uint8_t*>(b + L.slot_order);
    P.path = reinterpret_cast<int32_t*>(b + L.path);
    P.traj = reinterpret_cast<float*>(b + L.traj);
}

kpx_status read_header(kpx_planner* p, kpx_device_header* h) {
    cudaError_t e = cudaMemcpyAsync(h, p->P.hdr, sizeof(*h), cudaMemcpyDeviceToHost, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "reading planner counters");
    return KPX_OK;
}

// One iteration of the phase kernels (plain launches, one stream).
cudaError_t enqueue_iteration(const DevParams& P, cudaStream_t s) {
    cudaError_t e = launch_begin(P, s);
    if (e == cudaSuccess) e = launch_propagate(P, nullptr, s);
    if (e == cudaSuccess) e = launch_mark(P, s);
    if (e == cudaSuccess) e = launch_scan(P, s);
    if (e == cudaSuccess) e = launch_append(P, s);
    if (e == cudaSuccess) e = launch_stage(P, s);
    if (e == cudaSuccess) e = launch_prune(P, s);
    if (e == cudaSuccess) e = launch_end(P, s);
    return e;
}

// Iterations of the phase kernels per trip of the graph's loop: a trip
// costs a few microseconds on top of its kernels, so it carries several
// iterations (those past graph_pending are no-ops).  Behind the fused
// kernel the loop runs only once a problem has outgrown it, where an
// iteration costs tens of microseconds or more; there a shorter body keeps
// the graph, which every new planner builds, small.
constexpr int kLoopIterations = 8;
constexpr int kLoopIterationsFused = 2;

// One iteration of the phase kernels in the body of the graph's loop: it
// runs only while iterations are owed, and its last kernel counts it off
// graph_pending (the body's last iteration sets the loop's handle).
// The kept winners' re-integration (stage) forks onto the side stream after
// the winner scan and joins before the iteration's end, so that it runs
// beside append and prune (which need no end state).
cudaError_t enqueue_loop_iteration(const DevParams& P, cudaGraphConditionalHandle h, bool last, cudaStream_t s,
                                   const SideBranch& side) {
    cudaError_t e = launch_begin(P, s, true);
    if (e == cudaSuccess) e = launch_propagate(P, nullptr, s);
    if (e == cudaSuccess) e = launch_mark(P, s);
    if (e == cudaSuccess) e = launch_scan(P, s);
    if (e == cudaSuccess) e = cudaEventRecord(side.fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side.stream, side.fork, 0);
    if (e == cudaSuccess) e = launch_stage(P, side.stream);
    if (e == cudaSuccess) e = cudaEventRecord(side.join, side.stream);
    if (e == cudaSuccess) e = launch_append(P, s);
    if (e == cudaSuccess) e = launch_prune(P, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, side.join, 0);
    if (e == cudaSuccess) e = launch_end_loop(P, h, last, s);
    return e;
}

// The count node's parameters: n written to the header's graph_pending.
cudaMemsetParams count_params(const kpx_planner* p, int n) {
    cudaMemsetParams m = {};
    m.dst = &p->P.hdr->graph_pending;
    m.value = (unsigned int)n;
    m.elementSize = sizeof(int32_t);
    m.width = 1;
    m.height = 1;
    m.pitch = sizeof(int32_t);
    return m;
}

// kpx_iterate(n) is one launch of one graph per planner:
//   count node (memset: graph_pending = n)
//   -> the fused kernel (kpx_fused.cu), when the device can run its cluster:
//      iterations while the problem is small; the rest stay in graph_pending
//   -> WHILE node: up to kLoopIterations (kLoopIterationsFused behind the
//      fused kernel) iterations of the phase kernels per trip, until
//      graph_pending is 0 (each iteration's last kernel
//      counts it off).
// With the fused kernel the loop's handle starts at 0 and the fused kernel
// sets it; without it the handle starts at 1 (n >= 1).  Only the count
// node changes between launches.
cudaError_t build_loop_graph(kpx_planner* p, bool fused) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle h = 0;
    cudaGraphNode_t count = nullptr, dep = nullptr, loop = nullptr;
    cudaError_t le = cudaSuccess;
    e = cudaGraphConditionalHandleCreate(&h, g, fused ? 0u : 1u, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
        const cudaMemsetParams m = count_params(p, 1);
        e = cudaGraphAddMemsetNode(&count, g, nullptr, 0, &m);
    }
    dep = count;
    if (e == cudaSuccess && fused) {
        e = cudaStreamBeginCaptureToGraph(p->capture_stream, g, &count, nullptr, 1, cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            le = launch_fused(p->P, -1, h, 1, p->capture_stream);
            cudaGraph_t out = nullptr;
            e = cudaStreamEndCapture(p->capture_stream, &out);
            if (le != cudaSuccess) e = le;
        }
        // the captured fused kernel: the graph's only kernel node
        cudaGraphNode_t nodes[2] = {};
        size_t n_nodes = 2;
        if (e == cudaSuccess) e = cudaGraphGetNodes(g, nodes, &n_nodes);
        if (e == cudaSuccess && n_nodes != 2) e = cudaErrorUnknown;
        for (size_t k = 0; e == cudaSuccess && k < n_nodes; ++k) {
            cudaGraphNodeType t;
            e = cudaGraphNodeGetType(nodes[k], &t);
            if (e == cudaSuccess && t == cudaGraphNodeTypeKernel) dep = nodes[k];
        }
        if (e == cudaSuccess && dep == count) e = cudaErrorUnknown;
    }
    cudaGraphNodeParams cp = {};
    if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&loop, g, &dep, nullptr, 1, &cp);
    }
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(p->capture_stream, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            const int unroll = fused ? kLoopIterationsFused : kLoopIterations;
            for (int u = 0; u < unroll && le == cudaSuccess; ++u)
                le = enqueue_loop_iteration(p->P, h, u == unroll - 1, p->capture_stream, p->side);
            cudaGraph_t out = nullptr;
            e = cudaStreamEndCapture(p->capture_stream, &out);
            if (le != cudaSuccess) e = le;
        }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->loop_exec, g, 0);
    if (e != cudaSuccess) {
        p->loop_exec = nullptr;
        cudaGraphDestroy(g);
        return e;
    }
    p->loop_graph = g;
    p->count_node = count;
    p->count_value = 1;
    return cudaSuccess;
}

void drop_graphs(kpx_planner* p) {
    if (p->loop_exec) cudaGraphExecDestroy(p->loop_exec);
    if (p->loop_graph) cudaGraphDestroy(p->loop_graph);
    p->loop_exec = nullptr;
    p->loop_graph = nullptr;
    p->count_node = nullptr;
}

// The stream that planners' graphs are captured on: one per host thread and
// device, made on first use and kept (a capture leaves it idle), so that a
// planner neither creates nor destroys one.  nullptr when none can be made.
struct CaptureStreams {
    static constexpr int kDevices = 64;
    cudaStream_t s[kDevices] = {};
    SideBranch side[kDevices];
    ~CaptureStreams() {  // each call fails harmlessly once the context is gone
        for (int d = 0; d < kDevices; ++d) {
            if (s[d]) cudaStreamDestroy(s[d]);
            if (side[d].stream) cudaStreamDestroy(side[d].stream);
            if (side[d].fork) cudaEventDestroy(side[d].fork);
            if (side[d].join) cudaEventDestroy(side[d].join);
        }
    }
};

// The capture stream and side branch of this host thread on the current
// device (made on first use and kept); false when they cannot be made.
bool capture_resources_here(cudaStream_t* stream, SideBranch* side) {
    thread_local CaptureStreams streams;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= CaptureStreams::kDevices) {
        cudaGetLastError();
        return false;
    }
    SideBranch& b = streams.side[dev];
    bool ok = true;
    if (!streams.s[dev]) ok = cudaStreamCreateWithFlags(&streams.s[dev], cudaStreamNonBlocking) == cudaSuccess;
    if (ok && !b.stream) ok = cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking) == cudaSuccess;
    if (ok && !b.fork) ok = cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming) == cudaSuccess;
    if (ok && !b.join) ok = cudaEventCreateWithFlags(&b.join, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return false;
    }
    *stream = streams.s[dev];
    *side = b;
    return true;
}

// Decides once how kpx_iterate launches: a graph that starts with the fused
// kernel when the device can run its cluster (and KPX_FLAG_NO_FUSED is
// clear), else a graph of the phase kernels alone; plain launches (same
// kernels, same order) when no graph can be made.
void ensure_graphs(kpx_planner* p) {
    if (p->graph_state != 0) return;
    p->graph_state = -1;
    prepare_launches(p->P);
    p->graph_fused = !(p->P.flags & KPX_FLAG_NO_FUSED) && fused_cluster_size(p->P) > 0;
    cudaGetLastError();
    if (!capture_resources_here(&p->capture_stream, &p->side)) {
        p->capture_stream = nullptr;
        return;
    }
    p->graph_state = 1;
}

// The planner's graph, built on first use (nullptr: none can be made; the
// planner falls back to plain launches).
cudaGraphExec_t get_graph(kpx_planner* p) {
    if (p->loop_exec) return p->loop_exec;
    if (p->graph_fused) {
        if (build_loop_graph(p, true) == cudaSuccess) return p->loop_exec;
        cudaGetLastError();
        p->graph_fused = false;  // the fused form is unavailable: the phase kernels alone
    }
    if (build_loop_graph(p, false) == cudaSuccess) return p->loop_exec;
    cudaGetLastError();
    p->graph_state = -1;
    return nullptr;
}

kpx_status run_phase(kpx_planner* p, int phase, const kpx_debug_records* rec) {
    cudaError_t e = cudaSuccess;
    switch (phase) {
        case KPX_PHASE_BEGIN: e = launch_begin(p->P, p->stream); break;
        case KPX_PHASE_PROPAGATE: e = launch_propagate(p->P, rec, p->stream); break;
        case KPX_PHASE_MARK: e = launch_mark(p->P, p->stream); break;
        case KPX_PHASE_SCAN: e = launch_scan(p->P, p->stream); break;
        case KPX_PHASE_APPEND:  // both halves of UpdateTree
            e = launch_append(p->P, p->stream);
            if (e == cudaSuccess) e = launch_stage(p->P, p->stream);
            break;
        case KPX_PHASE_PRUNE: e = launch_prune(p->P, p->stream); break;
        case KPX_PHASE_END: e = launch_end(p->P, p->stream); break;
        default: return fail(p, KPX_E_INVALID, "unknown phase");
    }
    if (e != cudaSuccess) return cuda_fail(p, e, "kernel launch");
    return KPX_OK;
}

// Checks one problem's arguments and computes its workspace layout (no device
// work; nothing is allocated unless a message is returned).  kpx_create, the
// batch calls and kpx_plan_static all go through it.
kpx_status validate_problem(const kpx_dynamics* dyn, const kpx_workspace* ws, const kpx_obstacles* obs,
                            const float* start, const kpx_goal* goal, const kpx_cost* cost, const kpx_config* cfg,
                            Layout& L, std::string& err) {
    auto reject = [&](kpx_status st, const std::string& msg) {
        err = msg;
        return st;
    };
    if (!ws || !obs || !start || !goal || !cost) return reject(KPX_E_INVALID, "null argument");
    const int32_t n_obs = obs->count;
    std::string msg = check_config(dyn, cfg, n_obs);
    if (!msg.empty()) return reject(KPX_E_INVALID, msg);
    if (n_obs > 0 && !obs->aabb) return reject(KPX_E_INVALID, "obstacle array is null");
    for (int a = 0; a < 3; ++a)
        if (!finite(ws->lo[a]) || !finite(ws->hi[a]) || !(ws->hi[a] >= ws->lo[a]))
            return reject(KPX_E_INVALID, "workspace box needs finite lo <= hi");
    for (int i = 0; i < 6 * n_obs; ++i)
        if (!finite(obs->aabb[i])) return reject(KPX_E_INVALID, "obstacle coordinates must be finite");
    for (int b = 0; b < n_obs; ++b)
        for (int a = 0; a < 3; ++a)
            if (obs->aabb[6 * b + a] > obs->aabb[6 * b + 3 + a]) return reject(KPX_E_INVALID, "obstacle box with lo > hi");
    for (int a = 0; a < 3; ++a)
        if (!finite(goal->center[a])) return reject(KPX_E_INVALID, "goal centre must be finite");
    if (!finite(goal->radius) || goal->radius < 0.0f) return reject(KPX_E_INVALID, "goal radius must be >= 0");
    if (cost->kind < 0 || cost->kind > 2) return reject(KPX_E_INVALID, "unknown cost kind");
    if (!finite(cost->w_effort) || cost->w_effort < 0.0f) return reject(KPX_E_INVALID, "w_effort must be >= 0");
    if (cost->kind == KPX_COST_EFFORT_DURATION && dyn->kind != KPX_QUAD12)
        return reject(KPX_E_INVALID, "effort+duration cost needs the quadcopter");
    const int n = kStateDim[dyn->kind];
    for (int i = 0; i < n; ++i)
        if (!finite(start[i])) return reject(KPX_E_INVALID, "start state must be finite");
    L = make_layout(dyn, cfg, n_obs);
    if ((uint64_t)cfg->tree_cap + (uint64_t)L.slot_cap >= 0xFFFFFFFFull)
        return reject(KPX_E_INVALID, "tree_cap + candidate slots must stay below 2^32");
    return KPX_OK;
}

// Fills the parameter block of a validated problem laid out by L in the
// device memory at p->ws: problem fields, planner fields, device pointers and
// the obstacle grid (cell edge = grid_scale x the mean box extent), then
// checks that the start lies in X_valid.
kpx_status fill_problem(const kpx_dynamics* dyn, const kpx_workspace* ws, const kpx_obstacles* obs,
                        const float* start, const kpx_goal* goal, const kpx_cost* cost, const kpx_config* cfg,
                        const Layout& L, float grid_scale, kpx_planner* p, std::string& err) {
    const int32_t n_obs = obs->count;
    const int n = kStateDim[dyn->kind];
    p->L = L;
    DevParams& P = p->P;
    memset(&P, 0, sizeof(P));
    fill_dynamics(P, dyn);
    for (int i = 0; i < 16; ++i) P.start[i] = i < n ? start[i] : 0.0f;
    for (int a = 0; a < 3; ++a) {
        P.ws_lo[a] = ws->lo[a];
        P.ws_hi[a] = ws->hi[a];
        P.goal_c[a] = goal->center[a];
    }
    set_position_box(P);
    P.goal_r2 = goal->radius * goal->radius;
    P.cost_kind = cost->kind;
    P.w_effort = cost->w_effort;
    fill_axes(P, cfg->n_axes, cfg->axis);
    P.N = cfg->tree_cap;
    P.lambda_fixed = cfg->samples_per_node;
    P.i_max = cfg->i_max;
    P.seed_lo = (uint32_t)(cfg->seed & 0xFFFFFFFFull);
    P.seed_hi = (uint32_t)(cfg->seed >> 32);
    P.flags = cfg->flags;
    P.n_obs = n_obs;
    P.va_cap = L.va_cap;
    P.slot_cap = L.slot_cap;
    P.mask_words = L.mask_words;
    P.n_win_tiles = L.n_win_tiles;
    P.n_prune_tiles = L.n_prune_tiles;
    bind_pointers(p);
    choose_grid(P, obs->aabb, n_obs, grid_scale);
    if (!host_point_valid(P, P.start, obs->aabb, n_obs)) {
        err = "start state is not in X_valid";
        return KPX_E_INVALID;
    }
    return KPX_OK;
}

// Validates one problem and lays it out in `device_workspace` (no device
// work): fills p->P, p->L, p->ws.  On failure returns the status and a message.
kpx_status setup_member(const kpx_dynamics* dyn, const kpx_workspace* ws, const kpx_obstacles* obs,
                        const float* start, const kpx_goal* goal, const kpx_cost* cost, const kpx_config* cfg,
                        void* device_workspace, size_t workspace_bytes, kpx_planner* p, std::string& err) {
    Layout L;
    kpx_status st = validate_problem(dyn, ws, obs, start, goal, cost, cfg, L, err);
    if (st != KPX_OK) return st;
    if (!device_workspace) {
        err = "device workspace is null";
        return KPX_E_INVALID;
    }
    if (reinterpret_cast<uintptr_t>(device_workspace) % 256 != 0) {
        err = "device workspace must be 256-byte aligned";
        return KPX_E_INVALID;
    }
    if (workspace_bytes < L.total) {
        err = "device workspace smaller than kpx_workspace_size()";
        return KPX_E_NOMEM;
    }
    p->ws = reinterpret_cast<char*>(device_workspace);
    p->ws_bytes = workspace_bytes;
    st = fill_problem(dyn, ws, obs, start, goal, cost, cfg, L, p->grid_scale, p, err);
    if (st != KPX_OK) return st;
    p->host_obs.assign(obs->aabb, obs->aabb + 6 * (size_t)obs->count);
    return KPX_OK;
}

// Copies the obstacles (staged in `ob`, which must outlive the copy) and
// enqueues the initialisation and the obstacle grid build.
cudaError_t upload_and_init(kpx_planner* p, const kpx_obstacles* obs, std::vector<float4>& ob) {
    const int n_obs = obs->count;
    ob.assign((size_t)2 * (n_obs > 0 ? n_obs : 1), make_float4(0.0f, 0.0f, 0.0f, 0.0f));
    for (int b = 0; b < n_obs; ++b) {
        const float* o = obs->aabb + 6 * b;
        ob[2 * b] = make_float4(o[0], o[1], o[2], 0.0f);
        ob[2 * b + 1] = make_float4(o[3], o[4], o[5], 0.0f);
    }
    cudaError_t e = cudaSuccess;
    if (n_obs > 0)
        e = cudaMemcpyAsync(p->P.obs, ob.data(), (size_t)2 * n_obs * sizeof(float4), cudaMemcpyHostToDevice,
                            p->stream);
    if (e == cudaSuccess) e = launch_init(p->P, true, p->stream);
    if (e == cudaSuccess) e = launch_grid_build(p->P, p->stream);
    return e;
}

size_t batch_header_bytes(int B) {
    size_t off = align_up(sizeof(BatchHeader), 256);
    off += align_up((size_t)B * sizeof(DevParams), 256);
    off += 5 * align_up((size_t)(B + 1) * sizeof(int64_t), 256);
    off += align_up((size_t)B * sizeof(SlotState), 256);
    off += align_up((size_t)B * sizeof(kpx_device_header), 256);
    return off;
}

void drop_member_graphs(kpx_planner* p) {
    drop_graphs(p);
    p->graph_state = 0;
}

// batched iterations go out as graphs of kGraphIterations iterations (and
// single iterations for the remainder)
constexpr int kGraphIterations = 8;

cudaError_t capture_batch(kpx_batch* b, int count, cudaGraphExec_t* exec) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    cudaError_t le = cudaSuccess;
    for (int i = 0; i < count && le == cudaSuccess; ++i)
        le = launch_batch_iteration(b->BP, b->n_classes, b->cls_kind, b->cls_lo, b->cls_hi, b->cls_bps,
                                    b->capture_stream);
    e = cudaStreamEndCapture(b->capture_stream, &g);
    if (le != cudaSuccess) e = le;
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
    if (g) cudaGraphDestroy(g);
    return e;
}

}  // namespace

extern "C" {

size_t kpx_workspace_size(const kpx_dynamics* dyn, const kpx_config* cfg, int32_t n_obstacles) {
    if (!check_config(dyn, cfg, n_obstacles).empty()) return 0;
    return make_layout(dyn, cfg, n_obstacles).total;
}

kpx_status kpx_create(const kpx_dynamics* dyn, const kpx_workspace* ws, const kpx_obstacles* obs,
                      const float* start, const kpx_goal* goal, const kpx_cost* cost, const kpx_config* cfg,
                      void* device_workspace, size_t workspace_bytes, void* cuda_stream, kpx_planner** out) {
    g_create_error.clear();
    if (!out) {
        g_create_error = "out is null";
        return KPX_E_INVALID;
    }
    *out = nullptr;
    kpx_planner* p = new (std::nothrow) kpx_planner();
    if (!p) {
        g_create_error = "host allocation failed";
        return KPX_E_NOMEM;
    }
    p->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    std::string msg;
    kpx_status st = setup_member(dyn, ws, obs, start, goal, cost, cfg, device_workspace, workspace_bytes, p, msg);
    if (st != KPX_OK) {
        g_create_error = msg;
        delete p;
        return st;
    }
    // enqueued only: the copy's source lives as long as the planner, and
    // every later call runs on the same stream
    cudaError_t e = upload_and_init(p, obs, p->upload);
    if (e != cudaSuccess) {
        g_create_error = std::string("kpx_create: ") + cudaGetErrorString(e);
        delete p;
        return KPX_E_CUDA;
    }
    *out = p;
    return KPX_OK;
}

kpx_status kpx_iterate(kpx_planner* p, int32_t n_iters, kpx_iter_stats* out_last) {
    if (!p) return KPX_E_INVALID;
    if (n_iters < 0) return fail(p, KPX_E_INVALID, "n_iters must be >= 0");
    if (n_iters > 0) ensure_graphs(p);
    int32_t it = 0;
    if (p->graph_state == 1 && n_iters > 0) {
        cudaGraphExec_t g = get_graph(p);
        if (g) {
            cudaError_t e = cudaSuccess;
            if (n_iters != p->count_value) {  // the update costs a few microseconds: only on a change
                const cudaMemsetParams m = count_params(p, n_iters);
                e = cudaGraphExecMemsetNodeSetParams(g, p->count_node, &m);
                if (e == cudaSuccess) p->count_value = n_iters;
            }
            if (e == cudaSuccess) e = cudaGraphLaunch(g, p->stream);
            if (e != cudaSuccess) return cuda_fail(p, e, "graph launch");
            it = n_iters;
        }
    }
    for (; it < n_iters; ++it) {  // plain launches when no graph can be made
        cudaError_t e = enqueue_iteration(p->P, p->stream);
        if (e != cudaSuccess) return cuda_fail(p, e, "kernel launch");
    }
    if (!out_last) return KPX_OK;
    kpx_device_header h;
    kpx_status st = read_header(p, &h);
    if (st != KPX_OK) return st;
    memset(out_last, 0, sizeof(*out_last));
    out_last->status = h.status;
    out_last->iter = h.iter;
    out_last->n_nodes = h.n_nodes;
    out_last->n_active = h.count_A;
    out_last->n_inactive = h.n_inactive;
    out_last->n_terminal = h.n_terminal;
    out_last->lambda = h.lambda;
    out_last->first_solution_iter = h.first_solution_iter;
    out_last->candidates = (int64_t)h.last_candidates;
    out_last->valid = (int64_t)h.last_valid;
    out_last->winners = (int64_t)h.last_winners;
    out_last->total_candidates = (int64_t)h.total_candidates;
    out_last->total_valid = (int64_t)h.total_valid;
    out_last->total_winners = (int64_t)h.total_winners;
    if (h.goal_key == KEY_INF) {
        out_last->best_cost = INFINITY;
    } else {
        uint32_t bits = (uint32_t)(h.goal_key >> 32);
        float c;
        memcpy(&c, &bits, sizeof c);
        out_last->best_cost = c;
    }
    out_last->first_solution_ns =
        (h.first_solution_iter >= 0 && h.t_first_solution_ns > h.t_start_ns) ? h.t_first_solution_ns - h.t_start_ns : 0;
    out_last->elapsed_ns = h.t_last_ns > h.t_start_ns ? h.t_last_ns - h.t_start_ns : 0;
    out_last->total_steps = h.total_steps;
    out_last->total_box_tests = h.total_box_tests;
    if (h.status == KPX_E_TIMEOUT || h.status == KPX_E_INTERNAL) {
        char buf[128];
        snprintf(buf, sizeof buf, "device status %d (info %08x %08x)", h.status, h.err_info[0], h.err_info[1]);
        p->err = buf;
    }
    return (kpx_status)h.status;
}

kpx_status kpx_best_trajectory(kpx_planner* p, int32_t capacity, float* states, float* controls, int32_t* steps,
                               int32_t* out_len, float* out_cost) {
    if (!p || !out_len) return KPX_E_INVALID;
    *out_len = 0;
    cudaError_t e = launch_path(p->P, p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "path kernel");
    kpx_device_header h;
    kpx_status st = read_header(p, &h);
    if (st != KPX_OK) return st;
    if (h.traj_len < 0) return KPX_NO_SOLUTION;
    const int len = h.traj_len;
    *out_len = len;
    if (len > capacity) return fail(p, KPX_E_INVALID, "trajectory capacity too small (see *out_len)");
    if (!states || (len > 0 && (!controls || !steps))) return fail(p, KPX_E_INVALID, "null output array");
    const int n = p->P.n, m = p->P.m, w = n + m + 1;
    std::vector<float> buf((size_t)p->L.traj_rows * w);
    for (int first = 0; first <= len; first += p->L.traj_rows) {
        const int rows = (len + 1 - first) < p->L.traj_rows ? (len + 1 - first) : p->L.traj_rows;
        e = launch_gather(p->P, first, rows, p->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(buf.data(), p->P.traj, (size_t)rows * w * sizeof(float), cudaMemcpyDeviceToHost,
                                p->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
        if (e != cudaSuccess) return cuda_fail(p, e, "trajectory gather");
        for (int r = 0; r < rows; ++r) {
            const int g = first + r;
            const float* row = buf.data() + (size_t)r * w;
            memcpy(states + (size_t)g * n, row, n * sizeof(float));
            if (g >= 1) {
                memcpy(controls + (size_t)(g - 1) * m, row + n, m * sizeof(float));
                int k;
                memcpy(&k, row + n + m, sizeof k);
                steps[g - 1] = k;
            }
        }
    }
    if (out_cost) {
        uint32_t bits = (uint32_t)(h.goal_key >> 32);
        memcpy(out_cost, &bits, sizeof(float));
    }
    return KPX_OK;
}

kpx_status kpx_set_regions(kpx_planner* p, int32_t n_axes, const kpx_region_axis* axes) {
    if (!p) return KPX_E_INVALID;
    int64_t R = 0;
    std::string msg = check_axes(p->P.n, n_axes, axes, R);
    if (!msg.empty()) return fail(p, KPX_E_INVALID, msg);
    if (R > p->L.region_cap) return fail(p, KPX_E_INVALID, "the new grid needs more regions than the workspace holds "
                                                          "(kpx_config.region_capacity)");
    fill_axes(p->P, n_axes, axes);
    drop_graphs(p);  // the graphs hold the parameter block by value
    p->graph_state = 0;
    cudaError_t e = launch_remap_regions(p->P, p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "region remap");
    return KPX_OK;
}

// Re-chooses the obstacle grid at `scale` and enqueues its rebuild (the
// boxes are already on the device); no-op when the scale is unchanged.
cudaError_t regrid(kpx_planner* p, float scale) {
    if (scale == p->grid_scale) return cudaSuccess;
    p->grid_scale = scale;
    choose_grid(p->P, p->host_obs.data(), p->P.n_obs, scale);
    return launch_grid_build(p->P, p->stream);
}

bool launch_config_ok(const kpx_launch_config* lc) {
    return lc && lc->propagate_blocks_per_sm >= 0 && lc->propagate_blocks_per_sm <= 64 &&
           std::isfinite(lc->grid_scale) && lc->grid_scale >= 0.0f && lc->grid_scale <= 64.0f;
}

kpx_status kpx_set_launch(kpx_planner* p, const kpx_launch_config* lc) {
    if (!p || !launch_config_ok(lc)) return KPX_E_INVALID;
    if (lc->grid_scale > 0.0f) {
        cudaError_t e = regrid(p, lc->grid_scale);
        if (e != cudaSuccess) return cuda_fail(p, e, "grid rebuild");
    }
    if (lc->propagate_blocks_per_sm != p->P.prop_bps) {
        p->P.prop_bps = lc->propagate_blocks_per_sm;
        drop_graphs(p);  // the captured launch shapes and parameters change
        p->graph_state = 0;
    } else if (lc->grid_scale > 0.0f) {
        drop_graphs(p);  // the graphs hold the parameter block by value
        p->graph_state = 0;
    }
    return KPX_OK;
}

kpx_status kpx_graph_info(kpx_planner* p, int32_t* max_iterations_per_launch, int32_t* fused) {
    if (!p || !max_iterations_per_launch || !fused) return KPX_E_INVALID;
    ensure_graphs(p);
    *max_iterations_per_launch = p->graph_state == 1 ? INT32_MAX : 0;
    *fused = p->graph_state == 1 && p->graph_fused ? 1 : 0;
    return KPX_OK;
}

kpx_status kpx_reset(kpx_planner* p) {
    if (!p) return KPX_E_INVALID;
    cudaError_t e = launch_init(p->P, false, p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "reset");
    return KPX_OK;
}

kpx_status kpx_destroy(kpx_planner* p) {
    if (!p) return KPX_OK;
    cudaError_t e = cudaStreamSynchronize(p->stream);
    drop_graphs(p);
    delete p;
    return e == cudaSuccess ? KPX_OK : KPX_E_CUDA;
}

const char* kpx_status_str(kpx_status s) {
    switch (s) {
        case KPX_OK: return "ok";
        case KPX_E_INVALID: return "invalid argument";
        case KPX_E_NOMEM: return "workspace too small";
        case KPX_E_CUDA: return "CUDA error";
        case KPX_TREE_FULL: return "tree full";
        case KPX_NO_SOLUTION: return "no solution";
        case KPX_E_TIMEOUT: return "device wait timed out";
        case KPX_E_INTERNAL: return "internal consistency check failed";
    }
    return "unknown status";
}

const char* kpx_last_error(const kpx_planner* p) { return p ? p->err.c_str() : g_create_error.c_str(); }

kpx_status kpx_get_layout(const kpx_planner* p, kpx_layout* out) {
    if (!p || !out) return KPX_E_INVALID;
    const DevParams& P = p->P;
    memset(out, 0, sizeof(*out));
    out->header = P.hdr;
    out->x = P.x;
    out->u = P.u;
    out->K = P.K;
    out->parent = P.parent;
    out->key = P.key;
    out->region = P.region;
    out->set = P.set;
    out->icount = P.icount;
    out->region_key = P.region_key;
    out->region_snap = P.region_snap;
    out->va[0] = P.va0;
    out->va[1] = P.va1;
    out->win_slot = P.win_slot;
    out->win_mask = P.win_mask;
    out->obstacles = reinterpret_cast<float*>(P.obs);
    out->n = P.n;
    out->m = P.m;
    out->N = P.N;
    out->R = P.R;
    out->va_cap = P.va_cap;
    out->n_obstacles = P.n_obs;
    out->slot_cap = P.slot_cap;
    out->mask_words = P.mask_words;
    out->workspace_bytes = p->L.total;
    out->slot_order = P.slot_order;
    return KPX_OK;
}

kpx_status kpx_debug_wait_timeout(kpx_planner* p) {
    if (!p) return KPX_E_INVALID;
    cudaError_t e = launch_wait_timeout(p->P, p->stream);
    if (e == cudaErrorInvalidValue) return fail(p, KPX_E_INVALID, "the planner has fewer than two scan tiles");
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "bounded wait test");
    return KPX_OK;
}

kpx_status kpx_debug_step(kpx_planner* p, int32_t phase, const kpx_debug_records* records) {
    if (!p) return KPX_E_INVALID;
    if (records && records->valid && records->capacity < p->P.slot_cap)
        return fail(p, KPX_E_INVALID, "debug record capacity below the slot capacity");
    return run_phase(p, phase, phase == KPX_PHASE_PROPAGATE ? records : nullptr);
}

kpx_status kpx_snapshot(kpx_planner* p, void* dst) {
    if (!p || !dst) return KPX_E_INVALID;
    cudaError_t e = cudaMemcpyAsync(dst, p->ws, p->L.total, cudaMemcpyDefault, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    return e == cudaSuccess ? KPX_OK : cuda_fail(p, e, "snapshot");
}

size_t kpx_batch_workspace_size(int32_t count, const kpx_problem* problems) {
    if (count < 1 || count > 65535 || !problems) return 0;
    size_t total = batch_header_bytes(count);
    for (int i = 0; i < count; ++i) {
        const kpx_problem& q = problems[i];
        if (!q.obs || !check_config(q.dyn, q.cfg, q.obs->count).empty()) return 0;
        total += align_up(make_layout(q.dyn, q.cfg, q.obs->count).total, 256);
    }
    return total;
}

kpx_status kpx_batch_create(int32_t count, const kpx_problem* problems, void* device_workspace, size_t workspace_bytes,
                            void* cuda_stream, kpx_batch** out) {
    g_create_error.clear();
    if (!out || !problems || count < 1 || count > 65535) {
        g_create_error = "need 1 <= count <= 65535 problems and an output handle";
        return KPX_E_INVALID;
    }
    *out = nullptr;
    if (!device_workspace || reinterpret_cast<uintptr_t>(device_workspace) % 256 != 0) {
        g_create_error = "device workspace must be non-null and 256-byte aligned";
        return KPX_E_INVALID;
    }
    const size_t need = kpx_batch_workspace_size(count, problems);
    if (need == 0) {
        g_create_error = "a problem of the batch has an invalid configuration";
        return KPX_E_INVALID;
    }
    if (workspace_bytes < need) {
        g_create_error = "device workspace smaller than kpx_batch_workspace_size()";
        return KPX_E_NOMEM;
    }
    kpx_batch* b = new (std::nothrow) kpx_batch();
    if (!b) {
        g_create_error = "host allocation failed";
        return KPX_E_NOMEM;
    }
    b->B = count;
    b->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    // order problems by dynamics class (stable), one propagate/append launch per class
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    auto kind_of = [&](int i) { return problems[i].dyn->kind * 2 + problems[i].dyn->integ; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return kind_of(a) < kind_of(c); });
    b->member_of_index.assign(count, 0);
    char* base = reinterpret_cast<char*>(device_workspace);
    size_t off = batch_header_bytes(count);
    b->staging.assign(count, std::vector<float4>());
    std::vector<std::vector<float4>>& staging = b->staging;
    std::vector<DevParams> host_ps(count);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < count && e == cudaSuccess; ++k) {
        const int i = order[k];
        const kpx_problem& q = problems[i];
        kpx_planner* p = new (std::nothrow) kpx_planner();
        if (!p) {
            g_create_error = "host allocation failed";
            kpx_batch_destroy(b);
            return KPX_E_NOMEM;
        }
        p->stream = b->stream;
        b->members.push_back(p);
        b->member_of_index[i] = k;
        const size_t bytes = align_up(make_layout(q.dyn, q.cfg, q.obs->count).total, 256);
        std::string msg;
        kpx_status st = setup_member(q.dyn, q.ws, q.obs, q.start, q.goal, q.cost, q.cfg, base + off, bytes, p, msg);
        if (st != KPX_OK) {
            g_create_error = "problem " + std::to_string(i) + ": " + msg;
            kpx_batch_destroy(b);
            return st;
        }
        off += bytes;
        host_ps[k] = p->P;
        e = upload_and_init(p, q.obs, staging[k]);
        const int kind = kind_of(i);
        if (b->n_classes == 0 || b->cls_kind[b->n_classes - 1] != kind) {
            b->cls_kind[b->n_classes] = kind;
            b->cls_lo[b->n_classes] = k;
            ++b->n_classes;
        }
        b->cls_hi[b->n_classes - 1] = k + 1;
    }
    BatchParams& BP = b->BP;
    size_t h = 0;
    BP.B = count;
    BP.bh = reinterpret_cast<BatchHeader*>(base + h);
    h += align_up(sizeof(BatchHeader), 256);
    BP.Ps = reinterpret_cast<const DevParams*>(base + h);
    h += align_up((size_t)count * sizeof(DevParams), 256);
    int64_t* pre[5];
    for (int t = 0; t < 5; ++t) {
        pre[t] = reinterpret_cast<int64_t*>(base + h);
        h += align_up((size_t)(count + 1) * sizeof(int64_t), 256);
    }
    BP.chunk_prefix = pre[0];
    BP.scan_prefix = pre[1];
    BP.win_prefix = pre[2];
    BP.prune_prefix = pre[3];
    BP.order_prefix = pre[4];
    BP.slots = reinterpret_cast<SlotState*>(base + h);
    h += align_up((size_t)count * sizeof(SlotState), 256);
    b->poll_buf.assign(count, SlotState{});
    b->parking = reinterpret_cast<kpx_device_header*>(base + h);
    h += align_up((size_t)count * sizeof(kpx_device_header), 256);
    b->parked.assign(count, DevParams{});
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(const_cast<DevParams*>(BP.Ps), host_ps.data(), (size_t)count * sizeof(DevParams),
                            cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(BP.bh, 0, sizeof(BatchHeader), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->parking, 0, (size_t)count * sizeof(kpx_device_header), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // staging buffers are local
    if (e != cudaSuccess) {
        g_create_error = std::string("kpx_batch_create: ") + cudaGetErrorString(e);
        kpx_batch_destroy(b);
        return KPX_E_CUDA;
    }
    *out = b;
    return KPX_OK;
}

kpx_status kpx_batch_iterate(kpx_batch* b, int32_t n_iters) {
    if (!b) return KPX_E_INVALID;
    if (n_iters < 0) {
        b->err = "n_iters must be >= 0";
        return KPX_E_INVALID;
    }
    int32_t it = 0;
    cudaError_t e = cudaSuccess;
    if (b->graph_state == 0 && n_iters > 0) {
        // the first iteration runs plainly (it also computes the launch shapes),
        // then the iteration is captured once as a graph
        e = launch_batch_iteration(b->BP, b->n_classes, b->cls_kind, b->cls_lo, b->cls_hi, b->cls_bps, b->stream);
        ++it;
        b->graph_state = -1;
        if (e == cudaSuccess && cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking) == cudaSuccess) {
            if (capture_batch(b, 1, &b->graph_one) == cudaSuccess &&
                capture_batch(b, kGraphIterations, &b->graph_many) == cudaSuccess)
                b->graph_state = 1;
            else
                cudaGetLastError();
        }
    }
    if (b->graph_state == 1) {
        for (; e == cudaSuccess && it + kGraphIterations <= n_iters; it += kGraphIterations)
            e = cudaGraphLaunch(b->graph_many, b->stream);
        for (; e == cudaSuccess && it < n_iters; ++it) e = cudaGraphLaunch(b->graph_one, b->stream);
    }
    for (; e == cudaSuccess && it < n_iters; ++it)
        e = launch_batch_iteration(b->BP, b->n_classes, b->cls_kind, b->cls_lo, b->cls_hi, b->cls_bps, b->stream);
    if (e != cudaSuccess) {
        b->err = std::string("batch iteration: ") + cudaGetErrorString(e);
        return KPX_E_CUDA;
    }
    return KPX_OK;
}

kpx_status kpx_batch_member(kpx_batch* b, int32_t index, kpx_planner** out) {
    if (!b || !out || index < 0 || index >= b->B) return KPX_E_INVALID;
    *out = b->members[b->member_of_index[index]];
    return KPX_OK;
}

kpx_status kpx_batch_assign(kpx_batch* b, int32_t index, const kpx_problem* problem, int32_t iter_limit,
                            void* device_workspace, size_t workspace_bytes) {
    if (!b || !problem || index < 0 || index >= b->B || iter_limit < 0) return KPX_E_INVALID;
    const int k = b->member_of_index[index];
    kpx_planner* p = b->members[k];
    if (!problem->dyn || problem->dyn->kind * 2 + problem->dyn->integ != p->P.dyn * 2 + p->P.integ) {
        b->err = "the slot holds another dynamics class";
        return KPX_E_INVALID;
    }
    kpx_planner tmp;
    tmp.stream = b->stream;
    tmp.grid_scale = p->grid_scale;  // the class's launch settings stay with the slot
    std::string msg;
    void* ws = device_workspace ? device_workspace : p->ws;
    const size_t ws_bytes = device_workspace ? workspace_bytes : p->ws_bytes;
    kpx_status st = setup_member(problem->dyn, problem->ws, problem->obs, problem->start, problem->goal,
                                 problem->cost, problem->cfg, ws, ws_bytes, &tmp, msg);
    if (st != KPX_OK) {
        b->err = msg;
        return st;
    }
    drop_member_graphs(p);
    p->P = tmp.P;
    p->L = tmp.L;
    p->ws = tmp.ws;
    p->ws_bytes = tmp.ws_bytes;
    p->host_obs = std::move(tmp.host_obs);
    p->P.iter_limit = iter_limit;
    cudaError_t e = upload_and_init(p, problem->obs, b->staging[k]);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(const_cast<DevParams*>(b->BP.Ps) + k, &p->P, sizeof(DevParams), cudaMemcpyHostToDevice,
                            b->stream);
    if (e != cudaSuccess) {
        b->err = std::string("batch assign: ") + cudaGetErrorString(e);
        return KPX_E_CUDA;
    }
    return KPX_OK;
}

kpx_status kpx_batch_release(kpx_batch* b, int32_t index) {
    if (!b || index < 0 || index >= b->B) return KPX_E_INVALID;
    const int k = b->member_of_index[index];
    kpx_planner* p = b->members[k];
    p->P.iter_limit = -1;
    // the device copy points at a parking header: from here on (in stream
    // order) no batch kernel touches the slot's workspace
    b->parked[k] = p->P;
    b->parked[k].hdr = b->parking + k;
    cudaError_t e = cudaMemcpyAsync(const_cast<DevParams*>(b->BP.Ps) + k, &b->parked[k], sizeof(DevParams),
                                    cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) {
        b->err = std::string("batch release: ") + cudaGetErrorString(e);
        return KPX_E_CUDA;
    }
    return KPX_OK;
}

kpx_status kpx_batch_poll(kpx_batch* b, kpx_slot_state* out) {
    if (!b || !out) return KPX_E_INVALID;
    cudaError_t e = launch_batch_poll(b->BP, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->poll_buf.data(), b->BP.slots, (size_t)b->B * sizeof(SlotState), cudaMemcpyDeviceToHost,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        b->err = std::string("batch poll: ") + cudaGetErrorString(e);
        return KPX_E_CUDA;
    }
    static_assert(sizeof(SlotState) == sizeof(kpx_slot_state), "slot state layouts differ");
    for (int i = 0; i < b->B; ++i) memcpy(&out[i], &b->poll_buf[b->member_of_index[i]], sizeof(kpx_slot_state));
    return KPX_OK;
}

kpx_status kpx_batch_set_launch(kpx_batch* b, int32_t kind, int32_t integ, const kpx_launch_config* lc) {
    if (!b || !launch_config_ok(lc)) return KPX_E_INVALID;
    int c = 0;
    while (c < b->n_classes && b->cls_kind[c] != kind * 2 + integ) ++c;
    if (c == b->n_classes) {
        b->err = "the batch has no problem of that dynamics class";
        return KPX_E_INVALID;
    }
    if (lc->grid_scale > 0.0f) {
        for (int k = b->cls_lo[c]; k < b->cls_hi[c]; ++k) {
            kpx_planner* p = b->members[k];
            if (lc->grid_scale == p->grid_scale) continue;
            cudaError_t e = cudaSuccess;
            if (p->P.iter_limit < 0) {  // vacant slot: the next assignment builds its grid
                p->grid_scale = lc->grid_scale;
            } else {
                e = regrid(p, lc->grid_scale);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(const_cast<DevParams*>(b->BP.Ps) + k, &p->P, sizeof(DevParams),
                                        cudaMemcpyHostToDevice, b->stream);
            }
            if (e != cudaSuccess) {
                b->err = std::string("batch set_launch: ") + cudaGetErrorString(e);
                return KPX_E_CUDA;
            }
            drop_member_graphs(p);
        }
    }
    if (lc->propagate_blocks_per_sm != b->cls_bps[c]) {
        b->cls_bps[c] = lc->propagate_blocks_per_sm;
        if (b->graph_one) cudaGraphExecDestroy(b->graph_one);
        if (b->graph_many) cudaGraphExecDestroy(b->graph_many);
        b->graph_one = b->graph_many = nullptr;
        b->graph_state = 0;
    }
    return KPX_OK;
}

kpx_status kpx_batch_reset(kpx_batch* b) {
    if (!b) return KPX_E_INVALID;
    for (kpx_planner* p : b->members) {
        if (p->P.iter_limit < 0) continue;  // vacant slot
        cudaError_t e = launch_init(p->P, false, b->stream);
        if (e != cudaSuccess) {
            b->err = std::string("batch reset: ") + cudaGetErrorString(e);
            return KPX_E_CUDA;
        }
    }
    return KPX_OK;
}

kpx_status kpx_batch_destroy(kpx_batch* b) {
    if (!b) return KPX_OK;
    cudaError_t e = b->stream ? cudaStreamSynchronize(b->stream) : cudaSuccess;
    for (kpx_planner* p : b->members) kpx_destroy(p);
    if (b->graph_one) cudaGraphExecDestroy(b->graph_one);
    if (b->graph_many) cudaGraphExecDestroy(b->graph_many);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    delete b;
    return e == cudaSuccess ? KPX_OK : KPX_E_CUDA;
}

const char* kpx_batch_last_error(const kpx_batch* b) { return b ? b->err.c_str() : g_create_error.c_str(); }

kpx_status kpx_restore(kpx_planner* p, const void* src) {
    if (!p || !src) return KPX_E_INVALID;
    cudaError_t e = cudaMemcpyAsync(p->ws, src, p->L.total, cudaMemcpyDefault, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    return e == cudaSuccess ? KPX_OK : cuda_fail(p, e, "restore");
}

}  // extern "C"

// ===========================================================================
// kpx_plan_static: one planning run without any allocation.
//
// For callers that may not allocate device memory: real-time control loops
// that must never wait on an allocator or see an out-of-memory error
// mid-flight, and plugins whose host application owns the whole device
// memory pool.  Their device memory is this file-scope array, reserved when
// the library is loaded and held by every GPU that loads it until the
// process exits.  The call synchronises its stream, so it refuses to run
// while that stream is being captured into a CUDA graph.  Validation and the
// parameter block are kpx_create's (validate_problem, fill_problem), and the
// iterations are the phase kernels of enqueue_iteration.
// ===========================================================================
namespace {

constexpr size_t kStaticScratchBytes = (size_t)KPX_STATIC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch, looked up once per device with that
// device current (the host-side symbol is only a stand-in, never a device
// address).  Threads that race on a device's first call both look it up and
// store the same address.
constexpr int kMaxDevices = 64;
std::atomic<void*> g_static_addr[kMaxDevices];

cudaError_t static_scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    void* ptr = g_static_addr[dev].load(std::memory_order_acquire);
    if (!ptr) {
        e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_static_addr[dev].store(ptr, std::memory_order_release);
    }
    *out = ptr;
    return cudaSuccess;
}

}  // namespace

extern "C" kpx_status kpx_plan_static(const kpx_dynamics* dyn, const kpx_workspace* ws, const kpx_obstacles* obs,
                                      const float* start, const kpx_goal* goal, const kpx_cost* cost,
                                      const kpx_config* cfg, int32_t n_iters, void* cuda_stream, int32_t capacity,
                                      float* states, float* controls, int32_t* steps, int32_t* out_len,
                                      float* out_cost) {
    g_create_error.clear();
    auto reject = [&](kpx_status st, const char* msg) {
        g_create_error = msg;
        return st;
    };
    if (!out_len) return reject(KPX_E_INVALID, "out_len is null");
    *out_len = 0;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    {
        // the call copies to the host and synchronises the stream, neither of
        // which a capturing stream allows: refuse before any stream work
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        const cudaError_t ce = cudaStreamIsCapturing(stream, &cs);
        if (ce == cudaErrorStreamCaptureImplicit || (ce == cudaSuccess && cs != cudaStreamCaptureStatusNone))
            return reject(KPX_E_INVALID, "kpx_plan_static synchronises its stream and cannot run while the stream "
                                         "is being captured into a CUDA graph");
        if (ce != cudaSuccess) {
            g_create_error = std::string("kpx_plan_static: cudaStreamIsCapturing: ") + cudaGetErrorString(ce);
            return KPX_E_CUDA;
        }
    }
    if (n_iters < 0) return reject(KPX_E_INVALID, "n_iters must be >= 0");
    Layout L;
    {
        std::string msg;
        const kpx_status st = validate_problem(dyn, ws, obs, start, goal, cost, cfg, L, msg);
        if (st != KPX_OK) {
            g_create_error = msg;
            return st;
        }
    }
    if (L.total > kStaticScratchBytes)
        return reject(KPX_E_NOMEM, "problem needs more device memory than the static scratch of "
                                   "kpx_plan_static (KPX_STATIC_SCRATCH_BYTES); use kpx_create with a workspace");
    const int n = kStateDim[dyn->kind], m = kControlDim[dyn->kind];
    const int32_t n_obs = obs->count;

    kpx_planner pl;  // host handle on the stack: nothing is allocated
    pl.stream = stream;
    void* scratch = nullptr;
    cudaError_t e = static_scratch_address(&scratch);
    if (e != cudaSuccess) {
        g_create_error = std::string("kpx_plan_static: cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return KPX_E_CUDA;
    }
    pl.ws = reinterpret_cast<char*>(scratch);
    pl.ws_bytes = kStaticScratchBytes;
    {
        std::string msg;
        const kpx_status st = fill_problem(dyn, ws, obs, start, goal, cost, cfg, L, pl.grid_scale, &pl, msg);
        if (st != KPX_OK) {
            g_create_error = msg;
            return st;
        }
    }
    const DevParams& P = pl.P;

    // obstacles: lo and hi corners copied straight from the caller's
    // float[M][6] into the float4 pairs the kernels read (no staging buffer)
    if (n_obs > 0) {
        e = cudaMemcpy2DAsync(P.obs, 2 * sizeof(float4), obs->aabb, 6 * sizeof(float), 3 * sizeof(float), n_obs,
                              cudaMemcpyHostToDevice, pl.stream);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(reinterpret_cast<char*>(P.obs) + sizeof(float4), 2 * sizeof(float4), obs->aabb + 3,
                                  6 * sizeof(float), 3 * sizeof(float), n_obs, cudaMemcpyHostToDevice, pl.stream);
    }
    // every array that must start at zero is cleared by the first-time init
    if (e == cudaSuccess) e = launch_init(P, true, pl.stream);
    if (e == cudaSuccess) e = launch_grid_build(P, pl.stream);
    for (int32_t it = 0; e == cudaSuccess && it < n_iters; ++it) e = enqueue_iteration(P, pl.stream);
    if (e == cudaSuccess) e = launch_path(P, pl.stream);
    kpx_device_header h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, P.hdr, sizeof(h), cudaMemcpyDeviceToHost, pl.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(pl.stream);
    if (e != cudaSuccess) {
        g_create_error = std::string("kpx_plan_static: ") + cudaGetErrorString(e);
        return KPX_E_CUDA;
    }
    if (h.status == KPX_E_TIMEOUT || h.status == KPX_E_INTERNAL) return reject((kpx_status)h.status, "device status");
    if (h.traj_len < 0) return KPX_NO_SOLUTION;
    const int len = h.traj_len;
    *out_len = len;
    if (len > capacity) return reject(KPX_E_INVALID, "trajectory capacity too small (see *out_len)");
    if (!states || (len > 0 && (!controls || !steps))) return reject(KPX_E_INVALID, "null output array");
    const size_t w = (size_t)(n + m + 1) * sizeof(float);
    for (int first = 0; e == cudaSuccess && first <= len; first += L.traj_rows) {
        const int rows = (len + 1 - first) < L.traj_rows ? (len + 1 - first) : L.traj_rows;
        e = launch_gather(P, first, rows, pl.stream);
        // staging row r holds node path[first + r]: its state, then the
        // control and step count of the segment that ends at it
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(states + (size_t)first * n, n * sizeof(float), P.traj, w, n * sizeof(float), rows,
                                  cudaMemcpyDeviceToHost, pl.stream);
        const int skip = first == 0 ? 1 : 0;  // the root has no incoming segment
        if (e == cudaSuccess && rows > skip) {
            e = cudaMemcpy2DAsync(controls + (size_t)(first + skip - 1) * m, m * sizeof(float),
                                  P.traj + (size_t)skip * (n + m + 1) + n, w, m * sizeof(float), rows - skip,
                                  cudaMemcpyDeviceToHost, pl.stream);
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(steps + (first + skip - 1), sizeof(int32_t),
                                      P.traj + (size_t)skip * (n + m + 1) + n + m, w, sizeof(int32_t), rows - skip,
                                      cudaMemcpyDeviceToHost, pl.stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(pl.stream);
    }
    if (e != cudaSuccess) {
        g_create_error = std::string("kpx_plan_static: ") + cudaGetErrorString(e);
        return KPX_E_CUDA;
    }
    if (out_cost) {
        uint32_t bits = (uint32_t)(h.goal_key >> 32);
        memcpy(out_cost, &bits, sizeof(float));
    }
    return KPX_OK;
}
