/*
 * kpx_oracle.c -- plain, single-threaded FP64 reference for the Kino-PAX+
 * planning iteration.  TEST INFRASTRUCTURE ONLY (see kpx_oracle.h): only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg load it.
 *
 * The code follows the paper's pseudocode in its order and notation:
 *   Alg. 1  main loop: Propagate, PruneNodes, UpdateTree
 *   Alg. 2  Propagate: sample u and dt, PropagateODE, validity, region map,
 *           cumulative cost, region min, provisional V_U
 *   Alg. 3  PruneNodes: I_count / I_max reactivation, terminal, inactive
 *   Alg. 4  UpdateTree: keep region-best V_U nodes, append, solution update
 *   Alg. 5  GraphSearch compaction over an exclusive scan
 * Where the paper is silent or ambiguous, the reading adopted is stated at
 * the place it is used, marked "Reading:".
 *
 * Build flags must include -ffp-contract=off: FP32 steps that are defined op
 * by op (control sample, region map) must not be fused.
 */
#include "kpx_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#if !defined(FLT_EVAL_METHOD) || (FLT_EVAL_METHOD != 0)
#error "the oracle needs IEEE single-precision evaluation of float expressions"
#endif

/* ------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11).  Ten rounds of the 4x32 S-box built from two
 * 32x32->64 multiplications; the 2x32 key is bumped by the Weyl constants
 * between rounds.
 * ---------------------------------------------------------------------- */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void kpo_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(M0, c0, &hi0, &lo0);
        mulhilo32(M1, c2, &hi1, &lo1);
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------
 * Sampling (Alg. 2, "randomly sample u and dt").  Reading:
 * key = (seed low word, seed high word), counter = (iteration, node, sample,
 * block).  Words in order: u_0..u_{m-1} then the step count K; for m = 4 the
 * K word is word 0 of block 1.  u_i = lo + (hi - lo) * f with f = (w >> 8) *
 * 2^-24, evaluated in FP32 with one rounding per operation; dt = K * h with
 * K = k_min + floor(w * (k_max - k_min + 1) / 2^32).
 * ---------------------------------------------------------------------- */
void kpo_sample_control(const kpo_problem* P, uint32_t iter, uint32_t node, uint32_t sample,
                        float* u, int32_t* K) {
    uint32_t key[2] = {(uint32_t)(P->seed & 0xFFFFFFFFu), (uint32_t)(P->seed >> 32)};
    uint32_t ctr[4] = {iter, node, sample, 0u};
    uint32_t w[8];
    kpo_philox4x32_10(ctr, key, w);
    ctr[3] = 1u;
    kpo_philox4x32_10(ctr, key, w + 4);
    for (int i = 0; i < P->m; ++i) {
        float f = (float)(w[i] >> 8) * 0x1p-24f;
        float span = P->u_hi[i] - P->u_lo[i];
        float t = span * f;
        u[i] = P->u_lo[i] + t;
    }
    uint64_t range = (uint64_t)(P->k_max - P->k_min + 1);
    *K = P->k_min + (int32_t)(((uint64_t)w[P->m] * range) >> 32);
}

/* ------------------------------------------------------------------------
 * Dynamics x' = f(x, u).  Sec. V names the systems (6D double integrator,
 * 6D Dubins airplane, 12D quadcopter) without equations.  Reading (textbook forms):
 *   DI:     p' = v, v' = a
 *   Dubins: (x,y,z,psi,gamma,v)' = (v cos psi cos gamma, v sin psi cos gamma,
 *           v sin gamma, u0, u1, u2)
 *   Quad:   state (p, phi, theta, psi, v, omega), control (T, tau):
 *           p' = v;  v' = (T/m) R(phi,theta,psi) e3 - g e3 with R = Rz Ry Rx;
 *           (phi,theta,psi)' = W(phi,theta) omega,
 *           W = [[1, s_phi t_theta, c_phi t_theta], [0, c_phi, -s_phi],
 *                [0, s_phi/c_theta, c_phi/c_theta]];
 *           omega' = J^-1 (tau - omega x J omega), J diagonal.
 * param = (m, g, Jx, Jy, Jz, tau_max, -, -).
 * ---------------------------------------------------------------------- */
void kpo_deriv(const kpo_problem* P, const double* x, const double* u, double* dx) {
    if (P->dyn == KPO_DI6) {
        for (int i = 0; i < 3; ++i) {
            dx[i] = x[3 + i];
            dx[3 + i] = u[i];
        }
    } else if (P->dyn == KPO_DUBINS6) {
        double psi = x[3], gam = x[4], v = x[5];
        dx[0] = v * cos(psi) * cos(gam);
        dx[1] = v * sin(psi) * cos(gam);
        dx[2] = v * sin(gam);
        dx[3] = u[0];
        dx[4] = u[1];
        dx[5] = u[2];
    } else {
        double mass = P->param[0], g = P->param[1];
        double Jx = P->param[2], Jy = P->param[3], Jz = P->param[4];
        double phi = x[3], th = x[4], psi = x[5];
        double p = x[9], q = x[10], r = x[11];
        double cphi = cos(phi), sphi = sin(phi);
        double cth = cos(th), sth = sin(th), tth = tan(th);
        double cpsi = cos(psi), spsi = sin(psi);
        double a = u[0] / mass;
        /* third column of R = Rz(psi) Ry(theta) Rx(phi) */
        double r13 = cpsi * sth * cphi + spsi * sphi;
        double r23 = spsi * sth * cphi - cpsi * sphi;
        double r33 = cth * cphi;
        dx[0] = x[6];
        dx[1] = x[7];
        dx[2] = x[8];
        dx[3] = p + sphi * tth * q + cphi * tth * r;
        dx[4] = cphi * q - sphi * r;
        dx[5] = (sphi * q + cphi * r) / cth;
        dx[6] = a * r13;
        dx[7] = a * r23;
        dx[8] = a * r33 - g;
        dx[9] = (u[1] - (Jz - Jy) * q * r) / Jx;
        dx[10] = (u[2] - (Jx - Jz) * r * p) / Jy;
        dx[11] = (u[3] - (Jy - Jx) * p * q) / Jz;
    }
}

/* PropagateODE integration step (the paper names no integrator): forward Euler or classic RK4,
 * control held constant over the segment. */
void kpo_step(const kpo_problem* P, const double* x, const double* u, double* x_next) {
    const int n = P->n;
    const double h = P->h;
    double k1[16], k2[16], k3[16], k4[16], tmp[16];
    kpo_deriv(P, x, u, k1);
    if (P->integ == KPO_EULER) {
        for (int i = 0; i < n; ++i) x_next[i] = x[i] + h * k1[i];
        return;
    }
    for (int i = 0; i < n; ++i) tmp[i] = x[i] + 0.5 * h * k1[i];
    kpo_deriv(P, tmp, u, k2);
    for (int i = 0; i < n; ++i) tmp[i] = x[i] + 0.5 * h * k2[i];
    kpo_deriv(P, tmp, u, k3);
    for (int i = 0; i < n; ++i) tmp[i] = x[i] + h * k3[i];
    kpo_deriv(P, tmp, u, k4);
    for (int i = 0; i < n; ++i)
        x_next[i] = x[i] + (h / 6.0) * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

/* ------------------------------------------------------------------------
 * Validity (Sec. III: X_valid = collision-free states satisfying the state
 * constraints).  Reading: a point robot at p = x[0..2]; invalid when a
 * state bound is violated, p leaves the closed workspace box, or p lies in
 * any closed obstacle box.  NaN compares false and is therefore invalid.
 * ---------------------------------------------------------------------- */
int32_t kpo_point_valid(const kpo_problem* P, const double* x) {
    for (int d = 0; d < P->n; ++d)
        if (!(x[d] >= P->x_lo[d] && x[d] <= P->x_hi[d])) return 0;
    for (int a = 0; a < 3; ++a)
        if (!(x[a] >= P->ws_lo[a] && x[a] <= P->ws_hi[a])) return 0;
    for (int b = 0; b < P->n_obs; ++b) {
        const double* o = P->obs + 6 * b;
        if (x[0] >= o[0] && x[0] <= o[3] && x[1] >= o[1] && x[1] <= o[4] &&
            x[2] >= o[2] && x[2] <= o[5])
            return 0;
    }
    return 1;
}

/* Chebyshev signed distance of p to a closed box: > 0 outside, <= 0 inside. */
static double box_cheb(const double* o, const double* p) {
    double d = -INFINITY;
    for (int a = 0; a < 3; ++a) {
        double lo = o[a] - p[a];
        double hi = p[a] - o[3 + a];
        double e = lo > hi ? lo : hi;
        if (e > d) d = e;
    }
    return d;
}

double kpo_point_clearance(const kpo_problem* P, const double* x) {
    double c = INFINITY;
    for (int d = 0; d < P->n; ++d) {
        if (isfinite(P->x_lo[d]) && x[d] - P->x_lo[d] < c) c = x[d] - P->x_lo[d];
        if (isfinite(P->x_hi[d]) && P->x_hi[d] - x[d] < c) c = P->x_hi[d] - x[d];
    }
    for (int a = 0; a < 3; ++a) {
        if (x[a] - P->ws_lo[a] < c) c = x[a] - P->ws_lo[a];
        if (P->ws_hi[a] - x[a] < c) c = P->ws_hi[a] - x[a];
    }
    for (int b = 0; b < P->n_obs; ++b) {
        double e = box_cheb(P->obs + 6 * b, x);
        if (e < c) c = e;
    }
    return c;
}

double kpo_point_margin(const kpo_problem* P, const double* x) {
    double c = INFINITY;
    for (int d = 0; d < P->n; ++d) {
        if (isfinite(P->x_lo[d])) c = fmin(c, fabs(x[d] - P->x_lo[d]));
        if (isfinite(P->x_hi[d])) c = fmin(c, fabs(P->x_hi[d] - x[d]));
    }
    for (int a = 0; a < 3; ++a) {
        c = fmin(c, fabs(x[a] - P->ws_lo[a]));
        c = fmin(c, fabs(P->ws_hi[a] - x[a]));
    }
    for (int b = 0; b < P->n_obs; ++b) c = fmin(c, fabs(box_cheb(P->obs + 6 * b, x)));
    return c;
}

/* ------------------------------------------------------------------------
 * Edge cost (Assumption 1: additive, monotone).  Reading:
 *   path length      sum_k ||p_k - p_{k-1}|| over the checked points
 *   duration         K h
 *   effort+duration  K h (1 + w e(u)), e(u) = ((T - m g)/(m g))^2 + sum_i (tau_i/tau_max)^2
 * ---------------------------------------------------------------------- */
static double effort(const kpo_problem* P, const double* u) {
    double mg = P->param[0] * P->param[1];
    double tmax = P->param[5];
    double e = (u[0] - mg) / mg;
    e = e * e;
    for (int i = 1; i < 4; ++i) {
        double t = u[i] / tmax;
        e += t * t;
    }
    return e;
}

/* PropagateODE over K steps with the validity check after every step
 * (Reading: checked at steps 1..K, not at RK4 stages). */
int32_t kpo_rollout(const kpo_problem* P, const double* x0, const float* u, int32_t K,
                    double* x_end, double* edge_cost, int32_t* first_bad, double* min_margin,
                    double* traj) {
    const int n = P->n;
    double x[16], xn[16], ud[8];
    for (int i = 0; i < P->m; ++i) ud[i] = (double)u[i];
    for (int i = 0; i < n; ++i) x[i] = x0[i];
    if (traj)
        for (int i = 0; i < n; ++i) traj[i] = x[i];
    double len = 0.0, mm = INFINITY;
    int32_t valid = 1, fb = -1;
    for (int k = 1; k <= K; ++k) {
        kpo_step(P, x, ud, xn);
        double dx = xn[0] - x[0], dy = xn[1] - x[1], dz = xn[2] - x[2];
        len += sqrt(dx * dx + dy * dy + dz * dz);
        double mk = kpo_point_margin(P, xn);
        if (mk < mm) mm = mk;
        for (int i = 0; i < n; ++i) x[i] = xn[i];
        if (traj)
            for (int i = 0; i < n; ++i) traj[k * n + i] = x[i];
        if (!kpo_point_valid(P, x)) {
            valid = 0;
            fb = k;
            break;
        }
    }
    for (int i = 0; i < n; ++i) x_end[i] = x[i];
    double c;
    if (P->cost_kind == KPO_COST_PATH_LENGTH)
        c = len;
    else if (P->cost_kind == KPO_COST_DURATION)
        c = (double)K * P->h;
    else
        c = (double)K * P->h * (1.0 + P->w_effort * effort(P, ud));
    *edge_cost = c;
    if (first_bad) *first_bad = fb;
    if (min_margin) *min_margin = mm;
    return valid;
}

/* ------------------------------------------------------------------------
 * Region map (Alg. 2; decomposition R of Sec. IV).  Reading: per
 * axis c = clamp(floor((x - lo) * (bins / (hi - lo))), 0, bins - 1) in FP32,
 * one rounding per operation, on (float)x; a wrapped axis first maps
 * psi -> psi - 2 pi floor((psi + pi) / (2 pi)) in FP32; the id is mixed radix
 * in axis order.  The margin is computed in FP64 from the same boundaries.
 * ---------------------------------------------------------------------- */
static const float KPO_PI_F = 3.14159265358979323846f;
static const float KPO_TWO_PI_F = 6.28318530717958647692f;

int32_t kpo_region(const kpo_problem* P, const double* x, double* margin) {
    int32_t id = 0;
    double mg = INFINITY;
    for (int a = 0; a < P->n_axes; ++a) {
        int bins = P->ax_bins[a];
        float lo = P->ax_lo[a], hi = P->ax_hi[a];
        float width = hi - lo;
        float scale = (float)bins / width;
        float xf = (float)x[P->ax_dim[a]];
        double xd = x[P->ax_dim[a]];
        if (P->ax_wrap[a]) {
            float t = (xf + KPO_PI_F) / KPO_TWO_PI_F;
            float fl = floorf(t);
            float w = KPO_TWO_PI_F * fl;
            xf = xf - w;
            xd = xd - 2.0 * M_PI * floor((xd + M_PI) / (2.0 * M_PI));
        }
        float t = (xf - lo) * scale;
        int c = (int)floorf(t);
        if (c < 0) c = 0;
        if (c > bins - 1) c = bins - 1;
        id = id * bins + c;
        /* FP64 distance to the boundaries that change this axis' cell */
        double cw = ((double)hi - (double)lo) / (double)bins;
        int b_first = P->ax_wrap[a] ? 0 : 1;
        int b_last = P->ax_wrap[a] ? bins : bins - 1;
        for (int b = b_first; b <= b_last; ++b) {
            double edge = (double)lo + cw * (double)b;
            double d = fabs(xd - edge);
            if (d < mg) mg = d;
        }
    }
    if (margin) *margin = mg;
    return id;
}

int32_t kpo_in_goal(const kpo_problem* P, const double* x, double* margin) {
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double e = x[a] - P->goal_c[a];
        d2 += e * e;
    }
    if (margin) *margin = fabs(sqrt(d2) - P->goal_r);
    return d2 <= P->goal_r * P->goal_r;
}

/* Reading: key = (IEEE bits of the FP32 cost << 32) | id.  Costs are >= 0,
 * so key order is (cost, id) lexicographic order. */
uint64_t kpo_pack_key(float cost, uint32_t id) {
    uint32_t bits;
    memcpy(&bits, &cost, sizeof bits);
    return ((uint64_t)bits << 32) | (uint64_t)id;
}

/* ------------------------------------------------------------------------
 * Alg. 2 over an explicit list of slots.  Slot = j * lambda + s, j = rank of
 * the parent in the ascending-id V_A list, s = sample index (Reading).
 * Candidate id = tree_cap + slot (Reading: tree nodes beat candidates of
 * equal cost; lower slots beat higher ones).
 * ---------------------------------------------------------------------- */
void kpo_propagate(const kpo_problem* P, uint32_t iter, int32_t lambda,
                   const double* tree_x, const double* tree_cost,
                   const int32_t* VA, int32_t count_A,
                   int64_t n_slots, const int64_t* slots,
                   uint8_t* valid, double* x_end, double* cost, int32_t* region, uint64_t* key,
                   int32_t* K, float* u, double* vmargin, double* rmargin,
                   uint8_t* in_goal, double* gmargin) {
    const int n = P->n, m = P->m;
    if (!slots) n_slots = (int64_t)count_A * lambda;
    for (int64_t i = 0; i < n_slots; ++i) {
        int64_t slot = slots ? slots[i] : i;
        int32_t j = (int32_t)(slot / lambda), s = (int32_t)(slot % lambda);
        int32_t node = VA[j];
        float ui[8];
        int32_t Ki;
        kpo_sample_control(P, iter, (uint32_t)node, (uint32_t)s, ui, &Ki);
        double xe[16], ec, vm;
        int32_t fb;
        int32_t v = kpo_rollout(P, tree_x + (int64_t)node * n, ui, Ki, xe, &ec, &fb, &vm, NULL);
        double c = tree_cost[node] + ec;
        double rm, gm;
        int32_t r = kpo_region(P, xe, &rm);
        int32_t g = kpo_in_goal(P, xe, &gm);
        valid[i] = (uint8_t)v;
        for (int d = 0; d < n; ++d) x_end[i * n + d] = xe[d];
        for (int d = 0; d < m; ++d) u[i * m + d] = ui[d];
        cost[i] = c;
        region[i] = r;
        key[i] = kpo_pack_key((float)c, (uint32_t)((int64_t)P->tree_cap + slot));
        K[i] = Ki;
        vmargin[i] = vm;
        rmargin[i] = rm;
        in_goal[i] = (uint8_t)g;
        gmargin[i] = gm;
    }
}

/* Alg. 2 (region min and provisional V_U, sequential here), the
 * V_U filter of the GPU form (keep x only if cost(x) still equals cost(R_i)),
 * and, as the Reading for capacity (the paper only sizes lambda so
 * as not to overflow): keep the first tree_cap - n_nodes winners in slot order; restore the regions of the dropped ones from the snapshot taken
 * before Propagate. */
int32_t kpo_select_winners(int32_t R, uint64_t* region_key, const uint64_t* region_snap,
                           int64_t n_cand, const uint8_t* valid, const int32_t* region,
                           const uint64_t* key, int32_t n_nodes, int32_t tree_cap,
                           int64_t* winners, int64_t* n_win, int64_t* n_kept) {
    (void)R;
    int64_t* vu = (int64_t*)malloc((size_t)(n_cand > 0 ? n_cand : 1) * sizeof(int64_t));
    int64_t n_vu = 0;
    for (int64_t c = 0; c < n_cand; ++c) {
        if (!valid[c]) continue;
        int32_t r = region[c];
        if (key[c] < region_key[r]) region_key[r] = key[c];
        if (key[c] == region_key[r]) vu[n_vu++] = c;
    }
    int64_t w = 0;
    for (int64_t i = 0; i < n_vu; ++i) {
        int64_t c = vu[i];
        if (key[c] == region_key[region[c]]) winners[w++] = c;
    }
    free(vu);
    int64_t room = (int64_t)tree_cap - n_nodes;
    int64_t kept = w < room ? w : room;
    for (int64_t i = kept; i < w; ++i) {
        int32_t r = region[winners[i]];
        region_key[r] = region_snap[r];
    }
    *n_win = w;
    *n_kept = kept;
    return w > kept;
}

/* ------------------------------------------------------------------------
 * PruneNodes (Alg. 3) in its literal order, first match wins (reading where
 * the text is terse): nodes in V_T are permanent and skipped; "ancestor" means every strict
 * ancestor up to the root; a node is dominated when its key is above its
 * region's key.
 * ---------------------------------------------------------------------- */
void kpo_prune(int32_t n_nodes, const uint64_t* key, const int32_t* region, const int32_t* parent,
               uint8_t* set, uint8_t* icount, const uint64_t* region_key, int32_t i_max) {
    for (int32_t i = 0; i < n_nodes; ++i) {
        if (set[i] == KPO_SET_T) continue;
        uint64_t rk = region_key[region[i]];
        int best = key[i] == rk;
        if (best && set[i] == KPO_SET_I) {
            icount[i] = (uint8_t)(icount[i] + 1);
            if (icount[i] > i_max) {
                set[i] = KPO_SET_A;
                continue;
            }
        }
        if (icount[i] > i_max && best) continue;
        if (key[i] > rk) {
            set[i] = KPO_SET_T;
            continue;
        }
        for (int32_t p = parent[i]; p >= 0; p = parent[p]) {
            if (key[p] > region_key[region[p]]) {
                set[i] = KPO_SET_I;
                break;
            }
        }
    }
}

/* Exclusive scan S of the mask, then GraphSearch: I[S[i]] = i where mask[i]. */
int32_t kpo_compact(int32_t n, const uint8_t* mask, int32_t* S, int32_t* I) {
    int32_t run = 0;
    for (int32_t i = 0; i < n; ++i) {
        if (S) S[i] = run;
        run += mask[i] ? 1 : 0;
    }
    int32_t acc = 0;
    for (int32_t i = 0; i < n; ++i) {
        if (mask[i]) I[acc++] = i;
    }
    return acc;
}

/* ------------------------------------------------------------------------
 * Full planner (Alg. 1).
 * ---------------------------------------------------------------------- */
typedef struct {
    int64_t slot;
    int32_t parent, K, region, goal;
    double cost;
    uint64_t key;
    double x[16];
    float u[8];
} kpo_cand;

struct kpo_planner {
    kpo_problem P;
    double* obs;
    kpo_view v;
    uint64_t* region_snap;
    kpo_cand* vu;
    int64_t vu_cap;
};

static void* xcalloc(size_t n, size_t s) {
    void* p = calloc(n ? n : 1, s);
    return p;
}

/* Alg. 1: root node, V_A = {root}, regions at infinite cost,
 * solution null.  Reading: the root's region holds the root's key.
 * The root is tested against the goal like any appended node. */
kpo_planner* kpo_create(const kpo_problem* P, const double* start) {
    if (P->tree_cap < 1 || P->n_axes < 1) return NULL;
    kpo_planner* pl = (kpo_planner*)xcalloc(1, sizeof(kpo_planner));
    pl->P = *P;
    pl->obs = (double*)xcalloc((size_t)(P->n_obs * 6), sizeof(double));
    memcpy(pl->obs, P->obs, (size_t)P->n_obs * 6 * sizeof(double));
    pl->P.obs = pl->obs;
    kpo_view* v = &pl->v;
    int32_t R = 1;
    for (int a = 0; a < P->n_axes; ++a) R *= P->ax_bins[a];
    v->N = P->tree_cap;
    v->R = R;
    v->n = P->n;
    v->m = P->m;
    size_t N = (size_t)P->tree_cap;
    v->x = (double*)xcalloc(N * P->n, sizeof(double));
    v->u = (float*)xcalloc(N * P->m, sizeof(float));
    v->K = (int32_t*)xcalloc(N, sizeof(int32_t));
    v->parent = (int32_t*)xcalloc(N, sizeof(int32_t));
    v->cost = (double*)xcalloc(N, sizeof(double));
    v->key = (uint64_t*)xcalloc(N, sizeof(uint64_t));
    v->region = (int32_t*)xcalloc(N, sizeof(int32_t));
    v->set = (uint8_t*)xcalloc(N, 1);
    v->icount = (uint8_t*)xcalloc(N, 1);
    v->VA = (int32_t*)xcalloc(N, sizeof(int32_t));
    v->region_key = (uint64_t*)xcalloc((size_t)R, sizeof(uint64_t));
    pl->region_snap = (uint64_t*)xcalloc((size_t)R, sizeof(uint64_t));
    for (int32_t r = 0; r < R; ++r) v->region_key[r] = KPO_KEY_INF;
    for (int d = 0; d < P->n; ++d) v->x[d] = start[d];
    v->parent[0] = -1;
    v->cost[0] = 0.0;
    v->key[0] = kpo_pack_key(0.0f, 0u);
    v->region[0] = kpo_region(&pl->P, start, NULL);
    v->region_key[v->region[0]] = v->key[0];
    v->set[0] = KPO_SET_A;
    v->n_nodes = 1;
    v->VA[0] = 0;
    v->count_A = 1;
    v->goal_key = KPO_KEY_INF;
    v->first_solution_iter = -1;
    if (kpo_in_goal(&pl->P, start, NULL)) {
        v->goal_key = v->key[0];
        v->first_solution_iter = 0;
    }
    return pl;
}

/* UpdateTree (Alg. 4): each kept winner, in slot order, becomes the next
 * node; its key (cost, id) is written to its region (the winner holds the
 * region's least key, so this is the region's new best node); appended goal
 * nodes lower the solution key (Reading: the solution is the least key over
 * appended goal nodes). */
int32_t kpo_append(const kpo_problem* P, int32_t n_nodes, int32_t n_kept, const double* cx, const float* cu,
                   const int32_t* cK, const int32_t* cparent, const double* ccost, const int32_t* cregion,
                   const uint8_t* cgoal, double* x, float* u, int32_t* K, int32_t* parent, double* cost,
                   uint64_t* key, int32_t* region, uint8_t* set, uint8_t* icount, uint64_t* region_key,
                   uint64_t* goal_key) {
    const int n = P->n, m = P->m;
    int32_t first = 0;
    for (int32_t k = 0; k < n_kept; ++k) {
        const int32_t id = n_nodes + k;
        for (int d = 0; d < n; ++d) x[(int64_t)id * n + d] = cx[(int64_t)k * n + d];
        for (int d = 0; d < m; ++d) u[(int64_t)id * m + d] = cu[(int64_t)k * m + d];
        K[id] = cK[k];
        parent[id] = cparent[k];
        cost[id] = ccost[k];
        key[id] = kpo_pack_key((float)ccost[k], (uint32_t)id);
        region[id] = cregion[k];
        set[id] = KPO_SET_A;
        icount[id] = 0;
        region_key[cregion[k]] = key[id];
        if (cgoal[k] && key[id] < *goal_key) {
            if (*goal_key == KPO_KEY_INF) first = 1;
            *goal_key = key[id];
        }
    }
    return first;
}

static void vu_push(kpo_planner* pl, int64_t* n, const kpo_cand* c) {
    if (*n == pl->vu_cap) {
        pl->vu_cap = pl->vu_cap ? 2 * pl->vu_cap : 1024;
        pl->vu = (kpo_cand*)realloc(pl->vu, (size_t)pl->vu_cap * sizeof(kpo_cand));
    }
    pl->vu[(*n)++] = *c;
}

static int32_t iterate_once(kpo_planner* pl) {
    kpo_problem* P = &pl->P;
    kpo_view* v = &pl->v;
    const int n = P->n, m = P->m;
    if (v->tree_full) return KPO_TREE_FULL;
    /* branching factor: fixed, or lambda = floor(t_e / |V_A|) (Eq. for lambda) */
    int32_t lambda = P->lambda > 0 ? P->lambda : (v->count_A > 0 ? P->tree_cap / v->count_A : 0);
    if (lambda < 1) lambda = 1;
    v->last_lambda = lambda;
    memcpy(pl->region_snap, v->region_key, (size_t)v->R * sizeof(uint64_t));

    /* ---- Propagate (Alg. 2) ---- */
    int64_t n_vu = 0, n_valid = 0;
    const int32_t count_before = v->count_A;
    for (int32_t j = 0; j < count_before; ++j) {
        int32_t node = v->VA[j];
        for (int32_t s = 0; s < lambda; ++s) {
            kpo_cand c;
            c.slot = (int64_t)j * lambda + s;
            c.parent = node;
            kpo_sample_control(P, (uint32_t)v->iter, (uint32_t)node, (uint32_t)s, c.u, &c.K);
            double ec;
            int32_t fb;
            if (!kpo_rollout(P, v->x + (int64_t)node * n, c.u, c.K, c.x, &ec, &fb, NULL, NULL))
                continue;
            n_valid++;
            c.region = kpo_region(P, c.x, NULL);
            c.cost = v->cost[node] + ec;
            c.key = kpo_pack_key((float)c.cost, (uint32_t)((int64_t)P->tree_cap + c.slot));
            c.goal = kpo_in_goal(P, c.x, NULL);
            if (c.key < v->region_key[c.region]) v->region_key[c.region] = c.key;
            if (c.key == v->region_key[c.region]) vu_push(pl, &n_vu, &c);
        }
    }
    /* ---- V_U filter + capacity (Alg. 4; capacity rule below) ---- */
    int64_t w = 0;
    for (int64_t i = 0; i < n_vu; ++i)
        if (pl->vu[i].key == v->region_key[pl->vu[i].region]) pl->vu[w++] = pl->vu[i];
    int64_t room = (int64_t)v->N - v->n_nodes;
    int64_t kept = w < room ? w : room;
    for (int64_t i = kept; i < w; ++i) v->region_key[pl->vu[i].region] = pl->region_snap[pl->vu[i].region];
    if (w > kept) v->tree_full = 1;

    /* ---- PruneNodes (Alg. 3) on the tree as it was before this iteration's appends ---- */
    kpo_prune(v->n_nodes, v->key, v->region, v->parent, v->set, v->icount, v->region_key, P->i_max);

    /* ---- UpdateTree (Alg. 4): append in slot order, solution update ---- */
    if (kept > 0) {
        double* cx = (double*)malloc((size_t)kept * n * sizeof(double));
        float* cu = (float*)malloc((size_t)kept * m * sizeof(float));
        int32_t* ci = (int32_t*)malloc((size_t)kept * 3 * sizeof(int32_t));
        double* cc = (double*)malloc((size_t)kept * sizeof(double));
        uint8_t* cg = (uint8_t*)malloc((size_t)kept);
        for (int64_t i = 0; i < kept; ++i) {
            const kpo_cand* c = &pl->vu[i];
            for (int d = 0; d < n; ++d) cx[i * n + d] = c->x[d];
            for (int d = 0; d < m; ++d) cu[i * m + d] = c->u[d];
            ci[i] = c->K;
            ci[kept + i] = c->parent;
            ci[2 * kept + i] = c->region;
            cc[i] = c->cost;
            cg[i] = (uint8_t)(c->goal != 0);
        }
        if (kpo_append(P, v->n_nodes, (int32_t)kept, cx, cu, ci, ci + kept, cc, ci + 2 * kept, cg, v->x, v->u,
                       v->K, v->parent, v->cost, v->key, v->region, v->set, v->icount, v->region_key,
                       &v->goal_key))
            v->first_solution_iter = v->iter;
        free(cx);
        free(cu);
        free(ci);
        free(cc);
        free(cg);
    }
    v->n_nodes += (int32_t)kept;
    /* next V_A: ascending ids (Alg. 5 compaction of the V_A mask) */
    int32_t cnt = 0;
    for (int32_t i = 0; i < v->n_nodes; ++i)
        if (v->set[i] == KPO_SET_A) v->VA[cnt++] = i;
    v->last_candidates = (int64_t)count_before * lambda;
    v->last_valid = n_valid;
    v->last_winners = kept;
    v->total_candidates += v->last_candidates;
    v->total_valid += n_valid;
    v->total_winners += kept;
    v->count_A = cnt;
    v->iter += 1;
    return v->tree_full ? KPO_TREE_FULL : KPO_OK;
}

/* Runs n_iters iterations of Alg. 1's loop body; once the tree is full every
 * further iteration is a no-op that reports KPO_TREE_FULL (Reading: tree exhaustion ends the run). */
int32_t kpo_iterate(kpo_planner* pl, int32_t n_iters) {
    int32_t st = pl->v.tree_full ? KPO_TREE_FULL : KPO_OK;
    for (int32_t it = 0; it < n_iters && !pl->v.tree_full; ++it) st = iterate_once(pl);
    return st;
}

void kpo_view_state(const kpo_planner* pl, kpo_view* out) { *out = pl->v; }

/* Solution extraction: walk parents from the best goal node (Alg. 1 "return"). */
int32_t kpo_best_trajectory(const kpo_planner* pl, int32_t cap, double* states, float* controls,
                            int32_t* steps, int32_t* out_len, double* out_cost) {
    const kpo_view* v = &pl->v;
    if (v->goal_key == KPO_KEY_INF) {
        *out_len = 0;
        return KPO_NO_SOLUTION;
    }
    int32_t id = (int32_t)(v->goal_key & 0xFFFFFFFFu);
    int32_t len = 0;
    for (int32_t p = id; v->parent[p] >= 0; p = v->parent[p]) len++;
    *out_len = len;
    *out_cost = v->cost[id];
    if (len > cap) return KPO_INVALID;
    int32_t p = id;
    for (int32_t k = len; k >= 0; --k) {
        for (int d = 0; d < v->n; ++d) states[(int64_t)k * v->n + d] = v->x[(int64_t)p * v->n + d];
        if (k > 0) {
            for (int d = 0; d < v->m; ++d) controls[(int64_t)(k - 1) * v->m + d] = v->u[(int64_t)p * v->m + d];
            steps[k - 1] = v->K[p];
            p = v->parent[p];
        }
    }
    return KPO_OK;
}

void kpo_destroy(kpo_planner* pl) {
    if (!pl) return;
    kpo_view* v = &pl->v;
    free(v->x); free(v->u); free(v->K); free(v->parent); free(v->cost); free(v->key);
    free(v->region); free(v->set); free(v->icount); free(v->VA); free(v->region_key);
    free(pl->region_snap); free(pl->vu); free(pl->obs);
    free(pl);
}

/* ------------------------------------------------------------------------
 * FP64 re-validation of a trajectory returned by a planner: every segment is
 * re-rolled in FP64 from its stored start state with its stored control and
 * step count (state mismatch, clearance and cost are accumulated), and the
 * whole control sequence is re-rolled open loop from the start state.
 * A solution of Sec. III follows the dynamics, stays in X_valid and ends in
 * X_goal, so the verdict is 1 exactly when
 *   - every re-rolled point (and the start) has clearance >= -1e-4,
 *   - the final stored state is within goal_r + 1e-4 of the goal centre, and
 *   - every segment's re-rolled end state matches the next stored state to
 *     1e-4 relative (|a - b| / max(1, |b|) per component).
 * The open-loop error is reported only: FP32 and FP64 rollouts of an
 * unstable system drift apart over many segments without either being wrong.
 * ---------------------------------------------------------------------- */
int32_t kpo_revalidate(const kpo_problem* P, int32_t len, const double* states, const float* controls,
                       const int32_t* steps, double* max_seg_err, double* min_clearance,
                       double* goal_slack, double* cost, double* openloop_err) {
    const int n = P->n;
    double worst = 0.0, clear = INFINITY, total = 0.0, olerr = 0.0;
    double xo[16];
    for (int d = 0; d < n; ++d) xo[d] = states[d];
    clear = fmin(clear, kpo_point_clearance(P, states));
    for (int32_t i = 0; i < len; ++i) {
        const double* xs = states + (int64_t)i * n;
        const double* xe_ref = states + (int64_t)(i + 1) * n;
        int32_t K = steps[i];
        double* traj = (double*)malloc((size_t)(K + 1) * n * sizeof(double));
        double xe[16], ec, mm;
        int32_t fb;
        /* the segment's own validity is judged by clearance below, so the
         * rollout is asked for the full trajectory even past a violation */
        kpo_rollout(P, xs, controls + (int64_t)i * P->m, K, xe, &ec, &fb, &mm, traj);
        int32_t kdone = fb > 0 ? fb : K;
        for (int k = 1; k <= kdone; ++k) clear = fmin(clear, kpo_point_clearance(P, traj + (int64_t)k * n));
        if (fb > 0) {
            /* a violation: clearance already negative unless within tolerance; continue
             * the re-roll to measure the end-state mismatch */
            double xx[16], xn[16], ud[8];
            for (int d = 0; d < P->m; ++d) ud[d] = controls[(int64_t)i * P->m + d];
            for (int d = 0; d < n; ++d) xx[d] = traj[(int64_t)fb * n + d];
            for (int k = fb + 1; k <= K; ++k) {
                kpo_step(P, xx, ud, xn);
                for (int d = 0; d < n; ++d) xx[d] = xn[d];
                clear = fmin(clear, kpo_point_clearance(P, xx));
            }
            for (int d = 0; d < n; ++d) xe[d] = xx[d];
        }
        for (int d = 0; d < n; ++d) {
            double den = fabs(xe_ref[d]) > 1.0 ? fabs(xe_ref[d]) : 1.0;
            double e = fabs(xe[d] - xe_ref[d]) / den;
            if (e > worst) worst = e;
        }
        total += ec;
        /* open-loop re-roll */
        {
            double ud[8], xn[16];
            for (int d = 0; d < P->m; ++d) ud[d] = controls[(int64_t)i * P->m + d];
            for (int k = 1; k <= K; ++k) {
                kpo_step(P, xo, ud, xn);
                for (int d = 0; d < n; ++d) xo[d] = xn[d];
            }
            for (int d = 0; d < n; ++d) {
                double den = fabs(xe_ref[d]) > 1.0 ? fabs(xe_ref[d]) : 1.0;
                double e = fabs(xo[d] - xe_ref[d]) / den;
                if (e > olerr) olerr = e;
            }
        }
        free(traj);
    }
    const double* xl = states + (int64_t)len * n;
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double e = xl[a] - P->goal_c[a];
        d2 += e * e;
    }
    *max_seg_err = worst;
    *min_clearance = clear;
    *goal_slack = P->goal_r - sqrt(d2);
    *cost = total;
    *openloop_err = olerr;
    return (clear >= -1e-4 && *goal_slack >= -1e-4 && worst <= 1e-4) ? 1 : 0;
}

/* ------------------------------------------------------------------------
 * Region remap (adaptive delta): the definition in kpx_oracle.h, written
 * out node by node.
 * ---------------------------------------------------------------------- */
void kpo_remap_regions(const kpo_problem* P, int32_t n_nodes, const double* x, const uint64_t* key,
                       const uint8_t* set, int32_t* region, uint64_t* region_key, uint8_t* dominated,
                       double* margin) {
    int64_t R = 1;
    for (int a = 0; a < P->n_axes; ++a) R *= P->ax_bins[a];
    for (int64_t r = 0; r < R; ++r) region_key[r] = KPO_KEY_INF;
    for (int32_t i = 0; i < n_nodes; ++i) {
        double mg;
        region[i] = kpo_region(P, x + (int64_t)i * P->n, &mg);
        if (margin) margin[i] = mg;
        if (set[i] != KPO_SET_T && key[i] < region_key[region[i]]) region_key[region[i]] = key[i];
    }
    for (int32_t i = 0; i < n_nodes; ++i)
        dominated[i] = (set[i] != KPO_SET_T && key[i] != region_key[region[i]]) ? 1 : 0;
}

/* ------------------------------------------------------------------------
 * Refinement objective and its gradient (TEST INFRASTRUCTURE: the reference
 * for the adjoint kernel).  The objective is defined in kpx_oracle.h.  The
 * gradient is plain reverse mode: the forward pass keeps every state, the
 * reverse pass walks the steps backwards through the RK4 stages with the
 * hand-derived vector-Jacobian product of the quadcopter dynamics below.
 * ---------------------------------------------------------------------- */

/* signed distance from p to the closed box (lo, hi); grad (may be NULL)
 * receives its gradient: (p - q)/|p - q| outside (q = nearest box point),
 * the outward normal of the nearest face inside. */
double kpo_box_distance(const double* box, const double* p, double* grad) {
    double q[3], o2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        q[a] = p[a] < box[a] ? box[a] : (p[a] > box[3 + a] ? box[3 + a] : p[a]);
        o2 += (p[a] - q[a]) * (p[a] - q[a]);
    }
    if (o2 > 0.0) {
        double d = sqrt(o2);
        if (grad)
            for (int a = 0; a < 3; ++a) grad[a] = (p[a] - q[a]) / d;
        return d;
    }
    /* inside: depth to the nearest face */
    double best = INFINITY;
    int axis = 0, side = 0;
    for (int a = 0; a < 3; ++a) {
        double dl = p[a] - box[a], dh = box[3 + a] - p[a];
        if (dl < best) { best = dl; axis = a; side = -1; }
        if (dh < best) { best = dh; axis = a; side = 1; }
    }
    if (grad) {
        for (int a = 0; a < 3; ++a) grad[a] = 0.0;
        grad[axis] = (double)side;
    }
    return -best;
}

static double softplus_b(double z, double beta) {
    double t = beta * z;
    return (t > 0.0 ? t + log1p(exp(-t)) : log1p(exp(t))) / beta;
}

static double sigmoid_b(double z, double beta) {
    double t = beta * z;
    if (t >= 0.0) return 1.0 / (1.0 + exp(-t));
    double e = exp(t);
    return e / (1.0 + e);
}

/* obstacle penalty at position p, and its gradient (added into g3) */
static double obstacle_penalty(const kpo_refine* R, const double* obs, int32_t n_obs, const double* p, double* g3) {
    double sum = 0.0;
    for (int32_t b = 0; b < n_obs; ++b) {
        double gd[3];
        double d = kpo_box_distance(obs + 6 * b, p, g3 ? gd : NULL);
        double z = R->margin - d;
        sum += softplus_b(z, R->beta);
        if (g3) {
            double s = sigmoid_b(z, R->beta) * R->w_obs;
            for (int a = 0; a < 3; ++a) g3[a] -= s * gd[a];
        }
    }
    return R->w_obs * sum;
}

/* a^T df/dx and a^T df/du of the quadcopter dynamics (kpo_deriv), by hand */
static void quad_vjp(const kpo_problem* P, const double* x, const double* u, const double* a, double* gx,
                     double* gu) {
    double mass = P->param[0];
    double Jx = P->param[2], Jy = P->param[3], Jz = P->param[4];
    double phi = x[3], th = x[4], psi = x[5];
    double p = x[9], q = x[10], r = x[11];
    double cphi = cos(phi), sphi = sin(phi);
    double cth = cos(th), sth = sin(th), tth = tan(th);
    double cpsi = cos(psi), spsi = sin(psi);
    double A = u[0] / mass;
    double r13 = cpsi * sth * cphi + spsi * sphi;
    double r23 = spsi * sth * cphi - cpsi * sphi;
    double r33 = cth * cphi;
    double w = sphi * q + cphi * r; /* appears in the theta derivatives */
    for (int i = 0; i < 12; ++i) gx[i] = 0.0;
    /* p' = v */
    gx[6] += a[0];
    gx[7] += a[1];
    gx[8] += a[2];
    /* phi' = p + sphi tth q + cphi tth r */
    gx[3] += a[3] * (cphi * tth * q - sphi * tth * r);
    gx[4] += a[3] * w / (cth * cth);
    gx[9] += a[3];
    gx[10] += a[3] * sphi * tth;
    gx[11] += a[3] * cphi * tth;
    /* theta' = cphi q - sphi r */
    gx[3] += a[4] * (-sphi * q - cphi * r);
    gx[10] += a[4] * cphi;
    gx[11] += a[4] * (-sphi);
    /* psi' = (sphi q + cphi r) / cth */
    gx[3] += a[5] * (cphi * q - sphi * r) / cth;
    gx[4] += a[5] * w * sth / (cth * cth);
    gx[10] += a[5] * sphi / cth;
    gx[11] += a[5] * cphi / cth;
    /* v' = A (r13, r23, r33) - g e3 */
    gx[3] += A * (a[6] * (-cpsi * sth * sphi + spsi * cphi) + a[7] * (-spsi * sth * sphi - cpsi * cphi) +
                  a[8] * (-cth * sphi));
    gx[4] += A * (a[6] * cpsi * cth * cphi + a[7] * spsi * cth * cphi + a[8] * (-sth * cphi));
    gx[5] += A * (a[6] * (-spsi * sth * cphi + cpsi * sphi) + a[7] * (cpsi * sth * cphi + spsi * sphi));
    gu[0] = (a[6] * r13 + a[7] * r23 + a[8] * r33) / mass;
    /* omega' = J^-1 (tau - omega x J omega), J diagonal */
    gx[10] += -a[9] * (Jz - Jy) * r / Jx;
    gx[11] += -a[9] * (Jz - Jy) * q / Jx;
    gx[11] += -a[10] * (Jx - Jz) * p / Jy;
    gx[9] += -a[10] * (Jx - Jz) * r / Jy;
    gx[9] += -a[11] * (Jy - Jx) * q / Jz;
    gx[10] += -a[11] * (Jy - Jx) * p / Jz;
    gu[1] = a[9] / Jx;
    gu[2] = a[10] / Jy;
    gu[3] = a[11] / Jz;
}

static double effort_cost(const kpo_problem* P, const kpo_refine* R, const double* u, int32_t K, double* g4) {
    double mg = P->param[0] * P->param[1], tmax = P->param[5];
    double dur = (double)K * P->h;
    double e = ((u[0] - mg) / mg) * ((u[0] - mg) / mg);
    for (int i = 1; i < 4; ++i) e += (u[i] / tmax) * (u[i] / tmax);
    if (g4) {
        g4[0] += dur * R->w_effort * 2.0 * (u[0] - mg) / (mg * mg);
        for (int i = 1; i < 4; ++i) g4[i] += dur * R->w_effort * 2.0 * u[i] / (tmax * tmax);
    }
    return dur * (1.0 + R->w_effort * e);
}

static int32_t total_steps(const int32_t* K, int32_t S) {
    int32_t n = 0;
    for (int32_t s = 0; s < S; ++s) n += K[s];
    return n;
}

double kpo_refine_cost(const kpo_problem* P, const kpo_refine* R, const double* obs, int32_t n_obs,
                       const double* x0, const double* u, const int32_t* K, int32_t S) {
    double x[16], xn[16], J = 0.0;
    for (int d = 0; d < 12; ++d) x[d] = x0[d];
    for (int32_t s = 0; s < S; ++s) {
        J += effort_cost(P, R, u + 4 * s, K[s], NULL);
        for (int32_t k = 0; k < K[s]; ++k) {
            kpo_step(P, x, u + 4 * s, xn);
            for (int d = 0; d < 12; ++d) x[d] = xn[d];
            J += obstacle_penalty(R, obs, n_obs, x, NULL);
        }
    }
    for (int a = 0; a < 3; ++a) J += R->w_goal * (x[a] - R->goal[a]) * (x[a] - R->goal[a]);
    return J;
}

double kpo_refine_grad(const kpo_problem* P, const kpo_refine* R, const double* obs, int32_t n_obs,
                       const double* x0, const double* u, const int32_t* K, int32_t S, double* grad_u) {
    const int32_t N = total_steps(K, S);
    const double h = P->h;
    double* xs = (double*)malloc((size_t)(N + 1) * 12 * sizeof(double));
    int32_t* seg = (int32_t*)malloc((size_t)(N > 0 ? N : 1) * sizeof(int32_t));
    for (int d = 0; d < 12; ++d) xs[d] = x0[d];
    double J = 0.0;
    int32_t k = 0;
    for (int32_t s = 0; s < S; ++s) {
        for (int i = 0; i < 4; ++i) grad_u[4 * s + i] = 0.0;
        J += effort_cost(P, R, u + 4 * s, K[s], grad_u + 4 * s);
        for (int32_t j = 0; j < K[s]; ++j, ++k) {
            kpo_step(P, xs + 12 * k, u + 4 * s, xs + 12 * (k + 1));
            seg[k] = s;
            J += obstacle_penalty(R, obs, n_obs, xs + 12 * (k + 1), NULL);
        }
    }
    /* adjoint of the last state: goal pull + the penalty at p_N */
    double lam[12] = {0.0};
    for (int a = 0; a < 3; ++a) {
        double e = xs[12 * N + a] - R->goal[a];
        J += R->w_goal * e * e;
        lam[a] = 2.0 * R->w_goal * e;
    }
    for (k = N - 1; k >= 0; --k) {
        const double* xk = xs + 12 * k;
        const double* uk = u + 4 * seg[k];
        if (k + 1 <= N) obstacle_penalty(R, obs, n_obs, xs + 12 * (k + 1), lam); /* d/dp of the penalty at p_{k+1} */
        /* RK4 stages of step k */
        double k1[12], k2[12], k3[12], k4[12], x2[12], x3[12], x4[12];
        kpo_deriv(P, xk, uk, k1);
        for (int i = 0; i < 12; ++i) x2[i] = xk[i] + 0.5 * h * k1[i];
        kpo_deriv(P, x2, uk, k2);
        for (int i = 0; i < 12; ++i) x3[i] = xk[i] + 0.5 * h * k2[i];
        kpo_deriv(P, x3, uk, k3);
        for (int i = 0; i < 12; ++i) x4[i] = xk[i] + h * k3[i];
        kpo_deriv(P, x4, uk, k4);
        (void)k4;
        /* x_{k+1} = x_k + h/6 (k1 + 2 k2 + 2 k3 + k4): adjoints of the stage derivatives */
        double ak1[12], ak2[12], ak3[12], ak4[12], g[12], gu[4], ax[12];
        for (int i = 0; i < 12; ++i) {
            ak1[i] = h / 6.0 * lam[i];
            ak2[i] = h / 3.0 * lam[i];
            ak3[i] = h / 3.0 * lam[i];
            ak4[i] = h / 6.0 * lam[i];
            ax[i] = lam[i];
        }
        double* gus = grad_u + 4 * seg[k];
        /* k4 = f(x4), x4 = x_k + h k3 */
        quad_vjp(P, x4, uk, ak4, g, gu);
        for (int i = 0; i < 12; ++i) { ak3[i] += h * g[i]; ax[i] += g[i]; }
        for (int i = 0; i < 4; ++i) gus[i] += gu[i];
        /* k3 = f(x3), x3 = x_k + h/2 k2 */
        quad_vjp(P, x3, uk, ak3, g, gu);
        for (int i = 0; i < 12; ++i) { ak2[i] += 0.5 * h * g[i]; ax[i] += g[i]; }
        for (int i = 0; i < 4; ++i) gus[i] += gu[i];
        /* k2 = f(x2), x2 = x_k + h/2 k1 */
        quad_vjp(P, x2, uk, ak2, g, gu);
        for (int i = 0; i < 12; ++i) { ak1[i] += 0.5 * h * g[i]; ax[i] += g[i]; }
        for (int i = 0; i < 4; ++i) gus[i] += gu[i];
        /* k1 = f(x_k) */
        quad_vjp(P, xk, uk, ak1, g, gu);
        for (int i = 0; i < 12; ++i) ax[i] += g[i];
        for (int i = 0; i < 4; ++i) gus[i] += gu[i];
        for (int i = 0; i < 12; ++i) lam[i] = ax[i];
    }
    free(xs);
    free(seg);
    return J;
}

int32_t kpo_validate_controls(const kpo_problem* P, const double* x0, const float* u, const int32_t* K,
                              int32_t S, double* min_clearance, double* goal_dist, double* cost,
                              double* x_end) {
    const int n = P->n;
    double x[16], xn[16], ud[8], clear = INFINITY, total = 0.0;
    int32_t ok = 1;
    for (int d = 0; d < n; ++d) x[d] = x0[d];
    for (int32_t s = 0; s < S; ++s) {
        for (int d = 0; d < P->m; ++d) ud[d] = u[(int64_t)s * P->m + d];
        total += (double)K[s] * P->h * (1.0 + P->w_effort * effort(P, ud));
        for (int32_t k = 0; k < K[s]; ++k) {
            kpo_step(P, x, ud, xn);
            for (int d = 0; d < n; ++d) x[d] = xn[d];
            if (!kpo_point_valid(P, x)) ok = 0;
            clear = fmin(clear, kpo_point_clearance(P, x));
        }
    }
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) d2 += (x[a] - P->goal_c[a]) * (x[a] - P->goal_c[a]);
    *min_clearance = clear;
    *goal_dist = sqrt(d2);
    *cost = total;
    for (int d = 0; d < n; ++d) x_end[d] = x[d];
    return (ok && sqrt(d2) <= P->goal_r) ? 1 : 0;
}

