/*
 * kpx_oracle.h -- plain, single-threaded FP64 reference ("oracle") for the
 * Kino-PAX+ planning iteration (Alg. 1 main loop, Alg. 2 Propagate, Alg. 3
 * PruneNodes, Alg. 4 UpdateTree; Appendix "Atomic Operations" for the GPU
 * form of the V_U filter and the ordered transfer into the tree).
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA planner.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code, header, table or helper with the CUDA
 * planner; the two meet only through the seeded scene description.
 *
 * Precision: states, dynamics, costs and margins are FP64.  Two operations
 * are defined in FP32 by the adopted reading of the paper (and are therefore
 * FP32 here as well): the control sample u = lo + (hi - lo) * f, and the
 * region map, which is applied to (float)x.  Region keys pack the FP32 cost
 * bits above a 32-bit node id, so that "cost(x) = cost(R_i)" of Alg. 2-4 is
 * an exact key comparison with a deterministic tie-break.
 *
 * Parity pins: every function here is pinned by CPU tests (closed forms,
 * brute force, hand-computed values, Philox known-answer vectors, the
 * paper's compaction example).  Nothing is "parity unpinned".
 */
#ifndef KPX_ORACLE_H
#define KPX_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { KPO_DI6 = 0, KPO_DUBINS6 = 1, KPO_QUAD12 = 2 };
enum { KPO_EULER = 0, KPO_RK4 = 1 };
enum { KPO_COST_PATH_LENGTH = 0, KPO_COST_DURATION = 1, KPO_COST_EFFORT_DURATION = 2 };
/* node sets (Sec. IV): active, inactive, terminal */
enum { KPO_SET_A = 1, KPO_SET_I = 2, KPO_SET_T = 3 };
enum { KPO_OK = 0, KPO_TREE_FULL = 4, KPO_NO_SOLUTION = 5, KPO_INVALID = 1 };

#define KPO_KEY_INF 0xFFFFFFFFFFFFFFFFull

typedef struct {
    int32_t dyn, integ, n, m;
    double h;
    int32_t k_min, k_max;
    float u_lo[8], u_hi[8];
    double x_lo[16], x_hi[16];
    double param[8];
    double ws_lo[3], ws_hi[3];
    double goal_c[3], goal_r;
    int32_t cost_kind, pad0;
    double w_effort;
    int32_t n_axes, pad1;
    int32_t ax_dim[8], ax_bins[8], ax_wrap[8];
    float ax_lo[8], ax_hi[8];
    int32_t tree_cap, lambda, i_max, n_obs;
    uint64_t seed;
    const double* obs; /* [n_obs][6]: lo x,y,z then hi x,y,z */
} kpo_problem;

/* Philox4x32-10 block function (Salmon et al., SC'11). */
void kpo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* "Randomly sample u and dt" (Alg. 2), keyed by (seed, iteration, node, sample). */
void kpo_sample_control(const kpo_problem* P, uint32_t iter, uint32_t node, uint32_t sample,
                        float* u, int32_t* K);

/* x' = f(x, u) of the three systems named in Sec. V (textbook equations, stated in the .c file). */
void kpo_deriv(const kpo_problem* P, const double* x, const double* u, double* dx);
/* One integration step of PropagateODE (forward Euler or classic RK4). */
void kpo_step(const kpo_problem* P, const double* x, const double* u, double* x_next);

/* X_valid membership of one state (Sec. III): state bounds, closed workspace, closed boxes. */
int32_t kpo_point_valid(const kpo_problem* P, const double* x);
/* Smallest L-infinity distance from x to a state where that verdict flips. */
double kpo_point_margin(const kpo_problem* P, const double* x);
/* Signed clearance: >= 0 inside X_valid, < 0 inside an obstacle or out of bounds. */
double kpo_point_clearance(const kpo_problem* P, const double* x);

/* PropagateODE + validity of the segment + edge cost (Alg. 2). */
int32_t kpo_rollout(const kpo_problem* P, const double* x0, const float* u, int32_t K,
                    double* x_end, double* edge_cost, int32_t* first_bad, double* min_margin,
                    double* traj /* nullable, [K+1][n] */);

/* "Map x' to region R_i" (Alg. 2): FP32 grid map of (float)x.  margin: FP64
 * distance of x to the nearest cell boundary that changes the id. */
int32_t kpo_region(const kpo_problem* P, const double* x, double* margin);

/* Goal set test on the position ball: ||p - c||^2 <= r^2; margin = | ||p-c|| - r |. */
int32_t kpo_in_goal(const kpo_problem* P, const double* x, double* margin);

uint64_t kpo_pack_key(float cost, uint32_t id);

/* Alg. 2 for a list of (rank, sample) slots of one iteration. */
void kpo_propagate(const kpo_problem* P, uint32_t iter, int32_t lambda,
                   const double* tree_x, const double* tree_cost,
                   const int32_t* VA, int32_t count_A,
                   int64_t n_slots, const int64_t* slots /* NULL = 0..count_A*lambda-1 */,
                   uint8_t* valid, double* x_end, double* cost, int32_t* region, uint64_t* key,
                   int32_t* K, float* u, double* vmargin, double* rmargin,
                   uint8_t* in_goal, double* gmargin);

/* Region argmin of Alg. 2 plus the V_U filter of Alg. 4 and the capacity
 * rule (winners beyond the free tree slots are dropped in slot order and
 * their regions restored).  Candidates in ascending slot order.  Returns 1
 * if the tree became full. */
int32_t kpo_select_winners(int32_t R, uint64_t* region_key, const uint64_t* region_snap,
                           int64_t n_cand, const uint8_t* valid, const int32_t* region,
                           const uint64_t* key, int32_t n_nodes, int32_t tree_cap,
                           int64_t* winners, int64_t* n_win, int64_t* n_kept);

/* PruneNodes (Alg. 3), literal order. */
void kpo_prune(int32_t n_nodes, const uint64_t* key, const int32_t* region, const int32_t* parent,
               uint8_t* set, uint8_t* icount, const uint64_t* region_key, int32_t i_max);

/* UpdateTree (Alg. 4), one iteration's appends.  The first n_kept winners,
 * given in slot order (cx[k][n] end state, cu[k][m] control, cK, cparent,
 * ccost accumulated cost, cregion, cgoal = end state in the goal set), become
 * nodes n_nodes + k: their rows are written, their key is pack(cost, id),
 * that key becomes their region's key, their set is V_A with icount 0, and
 * an appended goal node lowers *goal_key.  Tree arrays are row-major
 * (x[N][n], u[N][m]).  Returns 1 when *goal_key went from infinity to a
 * solution, else 0. */
int32_t kpo_append(const kpo_problem* P, int32_t n_nodes, int32_t n_kept, const double* cx, const float* cu,
                   const int32_t* cK, const int32_t* cparent, const double* ccost, const int32_t* cregion,
                   const uint8_t* cgoal, double* x, float* u, int32_t* K, int32_t* parent, double* cost,
                   uint64_t* key, int32_t* region, uint8_t* set, uint8_t* icount, uint64_t* region_key,
                   uint64_t* goal_key);

/* Exclusive scan + GraphSearch compaction (Alg. 5): I = [i : mask[i]] and
 * the count S[n-1] + mask[n-1] (the last element of an exclusive scan alone
 * misses the last mask entry).  S may be NULL. */
int32_t kpo_compact(int32_t n, const uint8_t* mask, int32_t* S, int32_t* I);

/* ---------------- full planner (Alg. 1) ---------------- */
typedef struct kpo_planner kpo_planner;

typedef struct {
    int32_t N, R, n, m;
    int32_t n_nodes, count_A, iter, tree_full;
    int32_t first_solution_iter, last_lambda;
    uint64_t goal_key;
    int64_t last_candidates, last_valid, last_winners;
    int64_t total_candidates, total_valid, total_winners;
    double* x;          /* [N][n] */
    float* u;           /* [N][m] */
    int32_t* K;         /* [N] */
    int32_t* parent;    /* [N] */
    double* cost;       /* [N] */
    uint64_t* key;      /* [N] */
    int32_t* region;    /* [N] */
    uint8_t* set;       /* [N] */
    uint8_t* icount;    /* [N] */
    uint64_t* region_key; /* [R] */
    int32_t* VA;        /* [N] */
} kpo_view;

kpo_planner* kpo_create(const kpo_problem* P, const double* start);
int32_t kpo_iterate(kpo_planner* pl, int32_t n_iters);
void kpo_view_state(const kpo_planner* pl, kpo_view* out);
int32_t kpo_best_trajectory(const kpo_planner* pl, int32_t cap, double* states, float* controls,
                            int32_t* steps, int32_t* out_len, double* out_cost);
void kpo_destroy(kpo_planner* pl);

/* FP64 re-validation of a returned trajectory (states[len+1][n], controls[len][m]):
 * 1 when the start and every re-rolled point have clearance >= -1e-4, the
 * last stored state lies within goal_r + 1e-4 of the goal centre, and each
 * segment re-rolled from its stored start reaches the next stored state to
 * 1e-4 relative (Sec. III: dynamics, X_valid, X_goal). */
int32_t kpo_revalidate(const kpo_problem* P, int32_t len, const double* states, const float* controls,
                       const int32_t* steps, double* max_seg_err, double* min_clearance,
                       double* goal_slack, double* cost, double* openloop_err);

/* A new region decomposition between iterations (adaptive delta; the
 * paper's remark on adaptive decompositions).  Reading: with P's grid, every
 * node's region is its state's region; a region's key is the minimum key
 * over its non-terminal nodes (set 1 or 2; KPO key order); a non-terminal
 * node whose key is not its region's key is dominated; terminal nodes keep
 * their set.  x[n_nodes][n]; region_key[R] with R = P's region count;
 * margin[i] = the node's distance to a cell boundary (as kpo_region). */
void kpo_remap_regions(const kpo_problem* P, int32_t n_nodes, const double* x, const uint64_t* key,
                       const uint8_t* set, int32_t* region, uint64_t* region_key, uint8_t* dominated,
                       double* margin);

/* ------------------------------------------------------------------------
 * Refinement objective of a control sequence (the adjoint post-pass; the
 * paper has no refinement, so the objective is a reading):
 *   J = sum_s K_s h (1 + w_effort e(u_s))                     effort + duration
 *     + w_obs sum_{k=1..N} sum_b sp(margin - d_b(p_k))        obstacle penalty
 *     + w_goal |p_N - goal|^2                                  goal pull
 * sp(z) = log(1 + exp(beta z)) / beta; d_b = signed distance from the
 * position p_k after RK4 step k to box b (negative inside); N = sum_s K_s.
 * ---------------------------------------------------------------------- */
typedef struct {
    double w_obs, beta, margin, w_goal;
    double goal[3];
    double w_effort;
} kpo_refine;

double kpo_box_distance(const double* box, const double* p, double* grad);
double kpo_refine_cost(const kpo_problem* P, const kpo_refine* R, const double* obs, int32_t n_obs,
                       const double* x0, const double* u, const int32_t* K, int32_t S);
double kpo_refine_grad(const kpo_problem* P, const kpo_refine* R, const double* obs, int32_t n_obs,
                       const double* x0, const double* u, const int32_t* K, int32_t S, double* grad_u);
/* Open-loop FP64 re-validation of a control sequence from x0: 1 when every
 * point after a step is valid and the last position lies in the goal ball. */
int32_t kpo_validate_controls(const kpo_problem* P, const double* x0, const float* u, const int32_t* K,
                              int32_t S, double* min_clearance, double* goal_dist, double* cost,
                              double* x_end);

#ifdef __cplusplus
}
#endif
#endif
