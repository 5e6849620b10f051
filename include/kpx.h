/*
 * kpx.h -- C ABI of the GB300 (sm_103a) Kino-PAX+ planning library.
 *
 * The library runs the per-iteration hot path of Kino-PAX+ (Alg. 1: the
 * Propagate / PruneNodes / UpdateTree loop) entirely on one GPU:
 *   - Propagate (Alg. 2): lambda Philox-sampled (control, duration) pairs per
 *     active node, Euler or RK4 integration in FP32, a validity check after
 *     every integration step, region map, and a packed 64-bit (cost | id)
 *     atomic minimum per region;
 *   - the V_U filter and UpdateTree (Alg. 4): winners are the candidates
 *     still holding their region's key; they are appended in slot order and
 *     the best goal-reaching node is tracked;
 *   - PruneNodes (Alg. 3) over the whole tree, fused with the compaction of
 *     the next active set (Alg. 5, exclusiveScan + GraphSearch).
 *
 * Conventions shared by every entry point:
 *   - No function throws; every one returns a kpx_status.
 *   - Host inputs are read during the call and copied; the caller keeps
 *     ownership of every pointer it passes.
 *   - Device memory: the library allocates none.  The caller provides one
 *     device buffer ("workspace") of kpx_workspace_size() bytes, aligned to
 *     256 bytes, that must stay valid until kpx_destroy().  The opaque
 *     planner handle itself lives in host memory (malloc).
 *   - Work is enqueued on the caller's CUDA stream (a cudaStream_t passed as
 *     void*; NULL = the legacy default stream).  kpx_iterate() does not wait
 *     for the GPU unless statistics are requested.
 *   - Errors: invalid arguments return KPX_E_INVALID with a message in
 *     kpx_last_error(); a CUDA runtime failure returns KPX_E_CUDA with the
 *     CUDA message.  KPX_TREE_FULL is sticky: once the tree capacity is
 *     reached every further iteration is a no-op, but the best solution
 *     stays readable.
 *   - Thread safety: one planner must not be used from two host threads at
 *     once; distinct planners are independent.
 */
#ifndef KPX_H
#define KPX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KPX_OK = 0,
    KPX_E_INVALID = 1,     /* bad argument (message in kpx_last_error) */
    KPX_E_NOMEM = 2,       /* workspace too small */
    KPX_E_CUDA = 3,        /* CUDA runtime error */
    KPX_TREE_FULL = 4,     /* tree capacity t_e reached (sticky; not an error) */
    KPX_NO_SOLUTION = 5,   /* no goal-reaching node yet */
    KPX_E_TIMEOUT = 6,     /* a bounded device-side wait gave up */
    KPX_E_INTERNAL = 7     /* a device-side consistency check failed */
} kpx_status;

/* The three systems of Sec. V (6D double integrator, 6D Dubins airplane,
 * 12D quadcopter).  State / control layouts:
 *   KPX_DI6      x = (p_x, p_y, p_z, v_x, v_y, v_z), u = (a_x, a_y, a_z)
 *   KPX_DUBINS6  x = (x, y, z, yaw, pitch, speed), u = (yaw rate, pitch rate, accel)
 *   KPX_QUAD12   x = (p, roll, pitch, yaw (ZYX), v, body rates), u = (thrust, tau_x, tau_y, tau_z)
 */
typedef enum { KPX_DI6 = 0, KPX_DUBINS6 = 1, KPX_QUAD12 = 2 } kpx_dyn_kind;
typedef enum { KPX_EULER = 0, KPX_RK4 = 1 } kpx_integrator;
/* Edge costs satisfying Assumption 1 (additive, monotone). */
typedef enum {
    KPX_COST_PATH_LENGTH = 0,     /* sum of |p_k - p_{k-1}| over the checked points */
    KPX_COST_DURATION = 1,        /* K h */
    KPX_COST_EFFORT_DURATION = 2  /* K h (1 + w e(u)), e = ((T-mg)/mg)^2 + sum (tau_i/tau_max)^2 */
} kpx_cost_kind;

/* Dynamics x' = f(x, u) (Sec. III) with the compact control box U and the
 * state constraints that, with the workspace and obstacles, define X_valid.
 * A segment has K steps of length h, K uniform in [k_min, k_max]
 * ("duration dt in (0, T_prop]" of Sec. IV with dt = K h).
 * Unconstrained state components use x_lo = -inf, x_hi = +inf.
 * param (quadcopter): mass, g, Jx, Jy, Jz, tau_max. */
typedef struct {
    int32_t kind;          /* kpx_dyn_kind */
    int32_t integ;         /* kpx_integrator */
    float h;               /* integration step (s), > 0 */
    int32_t k_min, k_max;  /* 1 <= k_min <= k_max <= 4096 */
    float u_lo[8], u_hi[8];
    float x_lo[16], x_hi[16];
    float param[8];
} kpx_dynamics;

/* Workspace W (Sec. III): a closed box; the robot's position must stay in it. */
typedef struct {
    float lo[3], hi[3];
} kpx_workspace;

/* Obstacle set O: count closed axis-aligned boxes, aabb = host float[count][6]
 * (lo x, y, z, hi x, y, z).  Copied at create. */
typedef struct {
    const float* aabb;
    int32_t count;
} kpx_obstacles;

/* Goal set X_goal: closed ball on the position. */
typedef struct {
    float center[3];
    float radius;
} kpx_goal;

typedef struct {
    int32_t kind;          /* kpx_cost_kind */
    float w_effort;
} kpx_cost;

/* One axis of the region decomposition R (hyper-cubes of Sec. IV): state
 * component, bin count and range; wrap != 0 maps an angle into [-pi, pi)
 * first.  Region ids are mixed radix in axis order. */
typedef struct {
    int32_t state_dim;
    int32_t bins;
    float lo, hi;
    int32_t wrap;
} kpx_region_axis;

enum {
    /* Reject a candidate whose key cannot win its region before checking
     * obstacles (the collision-after-cost remark of the appendix).  Results
     * are identical; only the "valid" statistic then counts fewer rollouts.
     * That count and the step and box-test counts then depend on the order
     * in which candidates reach the check, so they can differ between runs
     * and launch paths. */
    KPX_FLAG_EARLY_REJECT = 1,
    /* Never run whole iterations in the single-launch cluster kernel (used
     * while an iteration has at most a few thousand slots); every iteration
     * then launches the eight phase kernels.  Results are identical. */
    KPX_FLAG_NO_FUSED = 2,
    /* Roll the propagate kernel's slots out in index order instead of in
     * ascending order key (the step count K; the 12D quadcopter's predicted
     * step count) within each aligned chunk of 128 slots, longest quarter
     * first.
     * Results are identical (every slot's outcome is independent of the
     * lane that computes it); only the time changes. */
    KPX_FLAG_NO_SLOT_ORDER = 4
};

/* Planner hyperparameters (appendix "Hyperparameters"): tree capacity t_e,
 * branching factor lambda (0 = adaptive lambda = floor(t_e / |V_A|)),
 * region grid, inactivity threshold I_max (0..254), Philox seed. */
typedef struct {
    int32_t tree_cap;
    int32_t samples_per_node;
    int32_t n_axes;
    kpx_region_axis axis[8];
    int32_t i_max;
    uint64_t seed;
    int32_t flags;         /* KPX_FLAG_* */
    int32_t region_capacity; /* regions the workspace holds (0: this grid's count); room for a finer grid
                                given later to kpx_set_regions */
} kpx_config;

/* Counters after the last completed iteration. */
typedef struct {
    int32_t status;              /* kpx_status held by the planner */
    int32_t iter;                /* iterations completed */
    int32_t n_nodes;             /* |T| */
    int32_t n_active;            /* |V_A| for the next iteration */
    int32_t n_inactive, n_terminal;
    int32_t lambda;              /* branching factor of the last iteration */
    int32_t first_solution_iter; /* -1 until a goal node exists */
    int64_t candidates, valid, winners;            /* last iteration */
    int64_t total_candidates, total_valid, total_winners;
    float best_cost;             /* +inf without a solution */
    float pad;
    uint64_t first_solution_ns;  /* device clock: first solution - first iterate launch, 0 if none */
    uint64_t elapsed_ns;         /* device clock: last iteration end - first iterate launch */
    uint64_t total_steps;        /* integration steps executed by Propagate */
    uint64_t total_box_tests;    /* point-in-box tests executed by Propagate */
} kpx_iter_stats;

typedef struct kpx_planner kpx_planner;

/* Bytes of device workspace kpx_create needs for this problem size
 * (0 if the arguments are invalid). */
size_t kpx_workspace_size(const kpx_dynamics* dyn, const kpx_config* cfg, int32_t n_obstacles);

/* Problem statement of Sec. III + Alg. 1 initialisation: root node x_init,
 * V_A = {root}, every region at infinite cost except the root's region,
 * which holds the root's key; no solution (unless x_init is already in the
 * goal).  start = host float[n] with n the state dimension of dyn->kind; it
 * must lie in X_valid.  device_workspace: caller-owned device memory of at
 * least kpx_workspace_size() bytes, 256-byte aligned.  cuda_stream: the
 * stream all work of this planner is enqueued on.  On success *out receives
 * the planner; the device work that sets it up (obstacle upload, reset,
 * obstacle grid) is enqueued on the stream, not waited for, and a fault in
 * it is reported by the next call that waits for the stream.  The host
 * arrays may be reused as soon as the call returns.  Errors: KPX_E_INVALID
 * (inconsistent or non-finite inputs, start not valid, sizes out of range),
 * KPX_E_NOMEM (workspace too small), KPX_E_CUDA (a launch or copy that
 * could not be enqueued). */
kpx_status kpx_create(const kpx_dynamics* dyn, const kpx_workspace* ws, const kpx_obstacles* obs,
                      const float* start, const kpx_goal* goal, const kpx_cost* cost,
                      const kpx_config* cfg, void* device_workspace, size_t workspace_bytes,
                      void* cuda_stream, kpx_planner** out);

/* Runs n_iters iterations of Alg. 1's loop body (Propagate, PruneNodes,
 * UpdateTree) asynchronously on the planner's stream.  If out_last is not
 * NULL the call waits for the stream and fills it; the return value is then
 * the planner's status (KPX_OK or KPX_TREE_FULL or a device error).
 * Without out_last the call returns KPX_OK once the work is enqueued (or a
 * launch error). */
kpx_status kpx_iterate(kpx_planner* p, int32_t n_iters, kpx_iter_stats* out_last);

/* The best solution trajectory (Alg. 1 returns it): root-to-goal node
 * states, the control and step count of each segment.  Host outputs of
 * capacity segments: states float[capacity+1][n], controls float[capacity][m],
 * steps int32[capacity].  Waits for the planner's stream.  Returns
 * KPX_NO_SOLUTION when no goal node exists (*out_len = 0), KPX_E_INVALID with
 * *out_len = required segments when capacity is too small. */
kpx_status kpx_best_trajectory(kpx_planner* p, int32_t capacity, float* states, float* controls,
                               int32_t* steps, int32_t* out_len, float* out_cost);

/* Re-initialises the planner to its kpx_create state on the device (same
 * problem, same workspace), without host copies.  Asynchronous. */
kpx_status kpx_reset(kpx_planner* p);

/* Launch choices that leave every result unchanged (an autotuner picks
 * them by timing):
 *   propagate_blocks_per_sm: resident propagate blocks per SM of the
 *     persistent grid (0: as many as fit; capped at that);
 *   grid_scale: obstacle-grid cell edge as a multiple of the mean box extent
 *     per axis (0.75: the default; 0: keep the current).  The broad phase is
 *     exact at any cell size, so only the split between cell lookups and
 *     box tests moves.
 * kpx_set_launch applies them to one planner; kpx_batch_set_launch to every
 * problem of dynamics class (kind, integ) in a batch (KPX_E_INVALID if there
 * is none).  A new grid is rebuilt asynchronously on the stream, between
 * iterations. */
typedef struct {
    int32_t propagate_blocks_per_sm;
    float grid_scale;
} kpx_launch_config;
kpx_status kpx_set_launch(kpx_planner* p, const kpx_launch_config* lc);

/* Replaces the region decomposition between iterations (adaptive delta:
 * the paper's remark on non-uniform and adaptive decompositions allows the
 * grid to be refined over time).  The new grid (same axis rules as
 * kpx_config) must have at most the planner's region capacity (else
 * KPX_E_INVALID).  On the device, asynchronously:
 *   - every node's region becomes its state's region under the new grid;
 *   - each region's key becomes the minimum key over the non-terminal nodes
 *     (V_A and V_I) in it; a region with none is empty;
 *   - a non-terminal node is dominated when its key is not its region's key
 *     (the next PruneNodes sends it to V_T); terminal nodes stay terminal;
 *   - the memoised "ancestor dominated" bits are cleared, so PruneNodes
 *     re-derives them;
 *   - the sets and the next V_A list are left to the next PruneNodes.
 * Under a refinement (each new region inside one old region) no
 * non-terminal node becomes dominated.  kpx_reset keeps the new grid. */
kpx_status kpx_set_regions(kpx_planner* p, int32_t n_axes, const kpx_region_axis* axes);

/* How kpx_iterate launches (the graph is built on first use): each call
 * kpx_iterate(n) is one launch of one CUDA graph per planner
 * (*max_iterations_per_launch = INT32_MAX; 0 when no graph can be made and
 * every iteration is eight plain launches).  The graph's first node writes
 * n into the header's graph_pending.  *fused = 1 when a fused
 * single-launch kernel follows: it runs iterations in one thread-block
 * cluster while an iteration has at most one 32-slot chunk per warp of the
 * cluster and the tree at most 32,768 nodes, and leaves the iterations it
 * did not run in graph_pending.  A loop (a WHILE conditional node) then runs
 * the eight phase kernels once per iteration left, counting graph_pending
 * down to 0.  A launch of n iterations thus starts 1 + 8 m kernels, m = the
 * iterations the fused kernel left (the header's fused_iterations counts the
 * ones it ran); without the fused kernel, 7 n. */
kpx_status kpx_graph_info(kpx_planner* p, int32_t* max_iterations_per_launch, int32_t* fused);

/* Waits for the planner's stream and releases the host handle; the device
 * workspace is the caller's to free afterwards. */
kpx_status kpx_destroy(kpx_planner* p);

const char* kpx_status_str(kpx_status s);
/* Message of the last failing call on this planner ("" if none); with
 * p == NULL the message of the last failing kpx_create in this thread. */
const char* kpx_last_error(const kpx_planner* p);

/* ------------------------------------------------------------------------
 * Batches: many independent problems iterated together.  Every phase of an
 * iteration is one launch over the whole batch (propagate and append once
 * per dynamics class present), so launch overhead does not grow with the
 * number of problems.  Problems may differ in dynamics, obstacles, grid,
 * capacity and lambda; each keeps its own tree, counters and Philox stream,
 * and its result is the one it would get planned alone with kpx_create.
 * ---------------------------------------------------------------------- */
typedef struct {
    const kpx_dynamics* dyn;
    const kpx_workspace* ws;
    const kpx_obstacles* obs;
    const float* start;
    const kpx_goal* goal;
    const kpx_cost* cost;
    const kpx_config* cfg;
} kpx_problem;

typedef struct kpx_batch kpx_batch;

/* Device bytes for the batch (0 if count is out of [1, 65535] or a problem is invalid). */
size_t kpx_batch_workspace_size(int32_t count, const kpx_problem* problems);
/* Validates and initialises every problem (as kpx_create does) inside one
 * caller-owned workspace (256-byte aligned, >= kpx_batch_workspace_size bytes).
 * Errors as kpx_create, with the failing problem's index in
 * kpx_batch_last_error(NULL). */
kpx_status kpx_batch_create(int32_t count, const kpx_problem* problems, void* device_workspace, size_t workspace_bytes,
                            void* cuda_stream, kpx_batch** out);
/* n_iters iterations of every problem (asynchronous; CUDA graphs after the first). */
kpx_status kpx_batch_iterate(kpx_batch* b, int32_t n_iters);
/* Borrowed handle of problem `index` (caller's order) for kpx_iterate(.., 0, &stats),
 * kpx_best_trajectory, kpx_get_layout, kpx_snapshot; owned by the batch (do not destroy). */
kpx_status kpx_batch_member(kpx_batch* b, int32_t index, kpx_planner** out);
/* Every problem back to its create state (asynchronous). */
kpx_status kpx_batch_reset(kpx_batch* b);

/* Continuous batching: a request loop admits problems into slots as they
 * free up, each in device memory sized for it.
 *
 * kpx_batch_assign re-initialises slot `index` with a new problem of the
 * slot's dynamics class (else KPX_E_INVALID), asynchronously on the batch's
 * stream.  device_workspace (256-byte aligned, >= kpx_workspace_size() of the
 * problem, else KPX_E_NOMEM; caller-owned, kept alive until the slot is
 * released or reassigned) holds the slot's tree; NULL keeps the slot's
 * current workspace (the one from kpx_batch_create or the last assign) and
 * workspace_bytes is ignored.  The slot then iterates with the batch while
 * its iteration count is below iter_limit (0: no limit; < 0 KPX_E_INVALID)
 * and idles after; its result equals that of the problem planned alone with
 * kpx_create for the same number of iterations.
 *
 * kpx_batch_release marks slot `index` vacant.  Work enqueued on the batch's
 * stream after it never touches the slot's workspace, so the caller may
 * reuse that memory in stream order (its arrays stay readable until then).
 * kpx_batch_reset skips vacant slots.
 *
 * kpx_batch_poll waits for the batch's stream and fills out[count] with every
 * slot's state (status -1 for a vacant slot).  KPX_E_CUDA on a CUDA error. */
typedef struct {
    int32_t status, iter, n_nodes, first_solution_iter;
    uint64_t goal_key;            /* (FP32 cost bits << 32) | node id; all ones: no solution */
    /* device clock (%globaltimer, ns): the slot's first iteration, its first
     * solution (0: none), the end of its last iteration, and the poll itself
     * (t_poll_ns maps device times onto a host clock read right after). */
    uint64_t t_start_ns, t_first_solution_ns, t_last_ns, t_poll_ns;
} kpx_slot_state;
kpx_status kpx_batch_assign(kpx_batch* b, int32_t index, const kpx_problem* problem, int32_t iter_limit,
                            void* device_workspace, size_t workspace_bytes);
kpx_status kpx_batch_release(kpx_batch* b, int32_t index);
kpx_status kpx_batch_set_launch(kpx_batch* b, int32_t kind, int32_t integ, const kpx_launch_config* lc);
kpx_status kpx_batch_poll(kpx_batch* b, kpx_slot_state* out);
kpx_status kpx_batch_destroy(kpx_batch* b);
const char* kpx_batch_last_error(const kpx_batch* b);

/* One complete planning run that allocates nothing (the paper has no
 * counterpart: this is a deployment convenience of this library).
 *
 * Some callers cannot call cudaMalloc: real-time control loops that must
 * never block on an allocator or meet an out-of-memory error mid-plan, and
 * plugins whose host application already owns the device's memory pool and
 * hands out no device memory of its own.  This entry point plans with device
 * memory reserved inside the library instead: a static device array of
 * KPX_STATIC_SCRATCH_BYTES that every GPU loading the library holds until the
 * process exits.  It runs kpx_create + kpx_iterate(n_iters) +
 * kpx_best_trajectory in one call, with the same arguments and outputs as
 * those calls (host inputs; host outputs of capacity segments), and the same
 * validation as kpx_create.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *
 * The call enqueues its work on cuda_stream, copies the result to the host
 * and synchronises cuda_stream before it returns.  So it must not be called
 * while cuda_stream is being captured into a CUDA graph (nor, in global
 * capture mode, while any stream is): it then returns KPX_E_INVALID without
 * enqueuing anything.
 *
 * Limits and caveats:
 *   - problems whose kpx_workspace_size() exceeds KPX_STATIC_SCRATCH_BYTES
 *     are rejected with KPX_E_NOMEM (message in kpx_last_error(NULL));
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current;
 *   - every call, from any thread or stream, uses the same array, and the
 *     array keeps the last call's contents (each call re-initialises what it
 *     reads); calls that overlap on the GPU race and corrupt each other.
 * Returns KPX_OK, KPX_NO_SOLUTION (*out_len = 0), KPX_E_INVALID (bad input,
 * a capturing stream, or capacity too small with *out_len = required
 * segments), KPX_E_NOMEM, KPX_E_CUDA, or a device status (KPX_E_TIMEOUT /
 * KPX_E_INTERNAL). */
#define KPX_STATIC_SCRATCH_BYTES (16u << 20)
kpx_status kpx_plan_static(const kpx_dynamics* dyn, const kpx_workspace* ws, const kpx_obstacles* obs,
                           const float* start, const kpx_goal* goal, const kpx_cost* cost, const kpx_config* cfg,
                           int32_t n_iters, void* cuda_stream, int32_t capacity, float* states, float* controls,
                           int32_t* steps, int32_t* out_len, float* out_cost);

/* ------------------------------------------------------------------------
 * Trajectory refinement (an optional post-pass over returned trajectories;
 * the paper has none, and the planner never calls it).  For the 12D
 * quadcopter with RK4 only (else KPX_E_INVALID).
 *
 * A trajectory is a control sequence u[s] (thrust, 3 torques) held for
 * steps[s] RK4 steps each, s < n_segments, from the state x0.  Its
 * objective, with p_k the position after step k and N = sum of the steps:
 *   J = sum_s steps[s] h (1 + w_effort e(u[s]))              effort + duration
 *     + w_obs sum_{k=1..N} sum_b sp(margin - d_b(p_k))       obstacle penalty
 *     + w_goal |p_N - goal|^2                                goal pull
 * where e is the planner's effort term, sp(z) = log(1 + exp(beta z)) / beta,
 * and d_b is the signed distance from p_k to box b (negative inside).  Box
 * terms with beta (margin - d) < -30 are dropped (each is below 1e-13/beta).
 * ---------------------------------------------------------------------- */
typedef struct {
    float w_obs;      /* weight of the obstacle penalty */
    float beta;       /* softplus sharpness (1 / length), > 0 */
    float margin;     /* clearance at which the penalty is log(2)/beta per box */
    float w_goal;     /* weight of |p_N - goal|^2 */
    float goal[3];
    float w_effort;   /* effort weight of the edge cost */
} kpx_refine_cost;

/* Device bytes of the workspace kpx_refine_eval needs for a gradient of
 * count trajectories of at most max_total_steps steps: the box grid (below)
 * followed by the checkpoints.  kpx_refine_workspace_size(0, 0) is the box
 * grid alone, enough for an objective without a gradient. */
size_t kpx_refine_workspace_size(int32_t count, int32_t max_total_steps);

/* J (cost_out[count]) and, when grad_u != NULL, dJ/du (grad_u[count]
 * [max_segments][4]; rows past n_segments are 0) for count trajectories, on
 * cuda_stream, asynchronously.  Device arrays: obstacles[n_obstacles][6]
 * (lo xyz, hi xyz; n_obstacles <= 4096), x0[count][12], u[count]
 * [max_segments][4] (16-byte aligned, as is grad_u), steps[count]
 * [max_segments], n_segments[count].  The gradient is the adjoint
 * (reverse-mode) rollout with the state checkpointed every 32 steps in
 * workspace (256-byte aligned, caller-owned; >= kpx_refine_workspace_size
 * (count, max_total_steps) bytes with a gradient; without one it may be NULL,
 * or >= kpx_refine_workspace_size(0, 0) bytes for the box grid).
 * The box grid: every call that has it builds, on the device, a uniform
 * 16^3 grid over the boxes grown by the distance beyond which a box's term
 * is dropped, each cell listing in index order the boxes that can reach it;
 * a point then tests only its cell's boxes.  The terms kept are the same as
 * with every box tested; the summation order differs, so results equal those
 * of a call without the grid up to FP32 rounding, and calls with the grid
 * equal one another exactly.  A trajectory with more than max_total_steps
 * steps or an invalid segment count gets J = NaN and a zero gradient.  order
 * (device, may be NULL): a permutation of 0..count-1 giving the order in
 * which the trajectories are taken up; the results stay in index order.
 * Longest first (by total steps) balances the launch. */
kpx_status kpx_refine_eval(const kpx_dynamics* dyn, const kpx_refine_cost* cost, const float* obstacles,
                           int32_t n_obstacles, int32_t count, int32_t max_segments, const float* x0,
                           const float* u, const int32_t* steps, const int32_t* n_segments, const int32_t* order,
                           int32_t max_total_steps, float* cost_out, float* grad_u, void* workspace,
                           size_t workspace_bytes, void* cuda_stream);

/* The box tests of the last kpx_refine_eval call that used the box grid in
 * this workspace: counters[0] candidate boxes tested by the objective,
 * [1] those within the far distance (terms evaluated), [2] and [3] the same
 * for the gradient.  Synchronises cuda_stream. */
kpx_status kpx_refine_counters(const void* workspace, uint64_t counters[4], void* cuda_stream);

/* Re-validation of count trajectories with the planner's own FP32 RK4
 * stepper from x0: valid[i] = 1 when every state after a step satisfies the
 * state bounds, lies in the workspace box and in no obstacle box, and the
 * final position lies in the goal ball; cost_out[i] = the sum of all the
 * segments' effort+duration edge costs accumulated in FP64 (w_effort);
 * x_end[count][12] (may be NULL) = the final states.  Same array layouts as
 * kpx_refine_eval; asynchronous on cuda_stream. */
kpx_status kpx_refine_validate(const kpx_dynamics* dyn, const kpx_workspace* ws, const float* obstacles,
                               int32_t n_obstacles, const kpx_goal* goal, float w_effort, int32_t count,
                               int32_t max_segments, const float* x0, const float* u, const int32_t* steps,
                               const int32_t* n_segments, int32_t* valid, double* cost_out, float* x_end,
                               void* cuda_stream);

/* One projected Adam step (b1 0.9, b2 0.999, eps 1e-8, step t >= 1, rate lr)
 * on the controls u[count][max_segments][4], each scaled to [-1, 1] by the
 * control box of dyn: z = (u - mid) / half; z -= lr mhat / (sqrt(vhat) +
 * eps); z is clipped to [-1, 1].  m1, m2: the moment arrays (same shape,
 * zero before step 1), updated in place.  Rows past n_segments are left as
 * they are.  Asynchronous on cuda_stream. */
kpx_status kpx_refine_adam(const kpx_dynamics* dyn, int32_t count, int32_t max_segments, const int32_t* n_segments,
                           float* u, const float* grad_u, float* m1, float* m2, int32_t t, float lr,
                           void* cuda_stream);

/* Where cost[i] < cost_best[i], copies the row u[i] to u_best[i] and cost[i]
 * to cost_best[i] (NaN never wins).  Asynchronous on cuda_stream. */
kpx_status kpx_refine_keep_best(int32_t count, int32_t max_segments, const float* u, const float* cost,
                                float* u_best, float* cost_best, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Measurement.
 * ---------------------------------------------------------------------- */

/* The device's FP32 fused multiply-add throughput, measured: one launch of
 * 4 blocks of 256 threads per SM, each thread running 16 independent FMA
 * chains of `iters` steps (1 <= iters <= 2^20), timed with CUDA events on
 * cuda_stream after one untimed launch.  *tflops = 2 x FMAs / seconds / 1e12.
 * Synchronises the stream; allocates no device memory.  The reference for
 * the planner kernels' FP32 roofline beside the peak derived from unit
 * counts and the clock. */
kpx_status kpx_fp32_fma_rate(int32_t iters, double* tflops, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Introspection and step-by-step API (tests, debugging, checkpointing).
 * ---------------------------------------------------------------------- */

/* Device-resident counters at the head of the workspace. */
typedef struct {
    int32_t status, active, iter, n_nodes;
    int32_t count_A, lambda, va_sel, first_solution_iter;
    int64_t n_slots;
    uint64_t goal_key;
    int32_t n_win, n_kept, count_A_next, epoch;
    uint64_t prop_ticket;
    uint32_t win_ticket, prune_ticket;
    int32_t n_active, n_inactive, n_terminal;
    int32_t graph_pending;     /* iterations of the current graph launch left to the phase kernels */
    uint64_t last_candidates, last_valid, last_winners;
    uint64_t total_candidates, total_valid, total_winners;
    uint64_t t_start_ns, t_first_solution_ns, t_last_ns;
    int32_t traj_len;
    int32_t graph_ctl;         /* internal: the fused iteration's control word */
    uint64_t total_steps;      /* integration steps executed by Propagate since create/reset */
    uint64_t total_box_tests;  /* point-in-box tests executed by Propagate since create/reset */
    uint32_t err_info[4];
    uint64_t fused_iterations; /* iterations run by the fused single-launch kernel since create/reset */
} kpx_device_header;

/* Device addresses of the planner's arrays inside the workspace (SoA):
 * x: float[n][N] (component d of node i at x[d*N + i]), u: float[m][N],
 * K: uint16[N], parent: int32[N] (root: -1), key: uint64[N] ((FP32 cost
 * bits << 32) | id), region: int32[N], set: uint8[N] (bits 0-1: 1 = V_A,
 * 2 = V_I, 3 = V_T; bit 2: a strict ancestor is dominated; bit 3: the node
 * no longer holds its region's key), icount: uint8[N],
 * region_key: uint64[R], region_snap: uint64[R], va[2]: int32[va_cap] each
 * (the current V_A list is va[header.va_sel]), win_slot: int32[R],
 * win_mask: uint32[mask_words], obstacles: float[M][8] (lo x, y, z, 0,
 * hi x, y, z, 0). */
typedef struct {
    kpx_device_header* header;
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
    int32_t* va[2];
    int32_t* win_slot;
    uint32_t* win_mask;
    float* obstacles;
    int32_t n, m, N, R;
    int32_t va_cap, n_obstacles;
    int64_t slot_cap;
    int64_t mask_words;
    size_t workspace_bytes;
    /* propagate order of the current iteration (written by the begin phase):
     * uint8[slot_cap rounded up to 128]; entry c * 128 + p is the offset in
     * chunk c of the slot with the p-th smallest (key, offset), the key
     * being the step count K (for the 12D quadcopter: K, or fewer steps when
     * the velocity, extrapolated at the sampled thrust along the parent's
     * body z axis, leaves its bounds); null when KPX_FLAG_NO_SLOT_ORDER is
     * set */
    uint8_t* slot_order;
} kpx_layout;

kpx_status kpx_get_layout(const kpx_planner* p, kpx_layout* out);

/* Phases of one iteration, in launch order. */
typedef enum {
    KPX_PHASE_BEGIN = 0,      /* lambda, |V_A| lambda slots, region snapshot */
    KPX_PHASE_PROPAGATE = 1,  /* Alg. 2 */
    KPX_PHASE_MARK = 2,       /* V_U filter: regions holding a candidate key mark its slot */
    KPX_PHASE_SCAN = 3,       /* winners ranked in slot order */
    KPX_PHASE_APPEND = 4,     /* UpdateTree: winners written to T (capacity rule) */
    KPX_PHASE_PRUNE = 5,      /* Alg. 3 + compaction of the next V_A */
    KPX_PHASE_END = 6         /* counters */
} kpx_phase;

/* Per-slot record of PROPAGATE for parity checks (device arrays of
 * capacity slots): valid uint8, region int32, key uint64, K int32,
 * x_end float[n][capacity], u float[m][capacity]. */
typedef struct {
    uint8_t* valid;
    int32_t* region;
    uint64_t* key;
    int32_t* K;
    float* x;
    float* u;
    int64_t capacity;
} kpx_debug_records;

/* Launches one phase of the current iteration (records: PROPAGATE only,
 * nullable; with records every slot is checked in full and recorded). */
kpx_status kpx_debug_step(kpx_planner* p, int32_t phase, const kpx_debug_records* records);

/* Runs one look-back wait (the bounded spin of the decoupled scans) that
 * nothing will release: a scan tile waits on a predecessor word at an epoch
 * no tile carries.  The wait gives up after its poll limit (2^20 polls, well
 * under a second), records KPX_E_TIMEOUT in the planner's status with
 * err_info[0] = 0x10000 | 1, and returns; the planner then stays stopped and
 * the CUDA context usable.  Synchronises the stream.  For tests of the
 * failure path: KPX_E_INVALID if the planner has fewer than two tiles. */
kpx_status kpx_debug_wait_timeout(kpx_planner* p);

/* Copies the whole workspace (every array and counter) to / from dst/src,
 * host or device memory of layout.workspace_bytes bytes.  Waits for the
 * planner's stream.  A restored planner continues bit-identically. */
kpx_status kpx_snapshot(kpx_planner* p, void* dst);
kpx_status kpx_restore(kpx_planner* p, const void* src);

#ifdef __cplusplus
}
#endif
#endif /* KPX_H */
