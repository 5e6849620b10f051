// kpx_adjoint.cu -- trajectory refinement for the 12D quadcopter: the
// objective of a control sequence and its gradient by a hand-written adjoint
// (reverse-mode) rollout with checkpoints, plus the optimiser step.  The
// objective is defined in include/kpx.h (kpx_refine_cost); the paper has no
// refinement step.
//
// Layout: one warp per trajectory, taken in the caller's order (longest
// first balances the launch).  The state integration is sequential, so
// every lane integrates the same RK4 step (registers, no broadcast), and the
// launch takes as long as the longest trajectory's chain of dependent steps.
// The obstacle terms are kept off that chain: the forward pass integrates 32
// steps while lane t keeps the point after step t, then every lane sums the
// box terms of its own point; the backward pass re-integrates an interval,
// then lane t computes the penalty gradient at step t + 1 into shared memory
// before the serial adjoint recursion reads it.  The boxes sit in shared
// memory in SoA form.  A box whose softplus term is negligible (beta (margin
// - d) < -30) is rejected on the squared distance, without a square root.
//
// Gradient: the forward pass stores the state every REFINE_CKPT_STEPS steps.
// The backward pass walks the checkpoint intervals from the last one back,
// re-integrates each interval from its checkpoint into shared memory, then
// runs the adjoint recursion through the RK4 stages of each step with the
// vector-Jacobian product of the dynamics, written out by hand below.
//
// This file is compiled with FMA contraction: nothing else has to reproduce
// its arithmetic bit for bit.  The re-validation (kpx_refine.cu) uses the
// planner's own stepper and the planner's compile flags.
#include <cuda_runtime.h>

#include "kpx_device.cuh"

namespace kpx {

namespace {

constexpr int ADJ_WARPS = 4;            // warps (trajectories) per block
constexpr float SOFTPLUS_CUT = -30.0f;  // beta (margin - d) below this: exp() < 1e-13, the box is skipped

// sin and cos of the three Euler angles
struct Trig {
    float sphi, cphi, sth, cth, spsi, cpsi, ic;  // ic = 1 / cos(theta)
};

// Roll and pitch of a quadcopter trajectory stay within a few radians, where
// the hardware sine and cosine need no range reduction (absolute error grows
// like |angle| 1e-7); yaw keeps the reduction.  1 / cos(theta) is the
// hardware's approximate reciprocal (about 1 ulp).  The flush-to-zero forms
// differ only on subnormal values, which these angles and cos(theta) are not.
__device__ __forceinline__ Trig trig_of(const float (&x)[12]) {
    Trig T;
    sincos_sfu(x[3], T.sphi, T.cphi);
    sincos_sfu(x[4], T.sth, T.cth);
    fast_sincos(x[5], T.spsi, T.cpsi);
    T.ic = rcp_sfu(T.cth);
    return T;
}

// ---------------------------------------------------------------------------
// dynamics: x' = f(x, u) (p, ZYX Euler angles, v, body rates; u = thrust,
// torques) and a^T df/dx, a^T df/du
// ---------------------------------------------------------------------------
// f at a state whose angles' sine and cosine are T
__device__ __forceinline__ void quad_f_t(const RefineParams& R, const Trig& T, const float (&x)[12],
                                         const float (&u)[4], float (&dx)[12]) {
    const float tth = T.sth * T.ic;
    const float p = x[9], q = x[10], r = x[11];
    const float A = u[0] * R.inv_mass;
    const float w = T.sphi * q + T.cphi * r;
    dx[0] = x[6];
    dx[1] = x[7];
    dx[2] = x[8];
    dx[3] = p + tth * w;
    dx[4] = T.cphi * q - T.sphi * r;
    dx[5] = w * T.ic;
    dx[6] = A * (T.cpsi * T.sth * T.cphi + T.spsi * T.sphi);
    dx[7] = A * (T.spsi * T.sth * T.cphi - T.cpsi * T.sphi);
    dx[8] = A * (T.cth * T.cphi) - R.g;
    dx[9] = (u[1] - (R.J[2] - R.J[1]) * q * r) * R.inv_J[0];
    dx[10] = (u[2] - (R.J[0] - R.J[2]) * r * p) * R.inv_J[1];
    dx[11] = (u[3] - (R.J[1] - R.J[0]) * p * q) * R.inv_J[2];
}

__device__ __forceinline__ void quad_f(const RefineParams& R, const float (&x)[12], const float (&u)[4],
                                       float (&dx)[12]) {
    quad_f_t(R, trig_of(x), x, u, dx);
}

// a^T df/dx and a^T df/du at a state with angle sine/cosine T and body rates (p, q, r)
__device__ __forceinline__ void quad_vjp_t(const RefineParams& R, const Trig& T, float p, float q, float r,
                                           const float (&u)[4], const float (&a)[12], float (&gx)[12],
                                           float (&gu)[4]) {
    const float sphi = T.sphi, cphi = T.cphi, sth = T.sth, cth = T.cth, spsi = T.spsi, cpsi = T.cpsi, ic = T.ic;
    const float tth = sth * ic;
    const float A = u[0] * R.inv_mass;
    const float w = sphi * q + cphi * r;   // psi' cos(theta)
    const float wp = cphi * q - sphi * r;  // d w / d phi
    const float r13 = cpsi * sth * cphi + spsi * sphi;
    const float r23 = spsi * sth * cphi - cpsi * sphi;
    const float r33 = cth * cphi;
    gx[0] = 0.0f;
    gx[1] = 0.0f;
    gx[2] = 0.0f;
    // d/dphi: the Euler-rate rows and the thrust direction
    gx[3] = a[3] * tth * wp + a[4] * (-sphi * q - cphi * r) + a[5] * wp * ic +
            A * (a[6] * (-cpsi * sth * sphi + spsi * cphi) + a[7] * (-spsi * sth * sphi - cpsi * cphi) -
                 a[8] * cth * sphi);
    // d/dtheta
    gx[4] = (a[3] + a[5] * sth) * w * ic * ic + A * cphi * (a[6] * cpsi * cth + a[7] * spsi * cth - a[8] * sth);
    // d/dpsi
    gx[5] = A * (a[6] * (-spsi * sth * cphi + cpsi * sphi) + a[7] * (cpsi * sth * cphi + spsi * sphi));
    // d/dv: p' = v
    gx[6] = a[0];
    gx[7] = a[1];
    gx[8] = a[2];
    // d/d(p, q, r): Euler rates and the gyroscopic term
    const float kx = (R.J[2] - R.J[1]) * R.inv_J[0];
    const float ky = (R.J[0] - R.J[2]) * R.inv_J[1];
    const float kz = (R.J[1] - R.J[0]) * R.inv_J[2];
    gx[9] = a[3] - a[10] * ky * r - a[11] * kz * q;
    gx[10] = a[3] * sphi * tth + a[4] * cphi + a[5] * sphi * ic - a[9] * kx * r - a[11] * kz * p;
    gx[11] = a[3] * cphi * tth - a[4] * sphi + a[5] * cphi * ic - a[9] * kx * q - a[10] * ky * p;
    gu[0] = (a[6] * r13 + a[7] * r23 + a[8] * r33) * R.inv_mass;
    gu[1] = a[9] * R.inv_J[0];
    gu[2] = a[10] * R.inv_J[1];
    gu[3] = a[11] * R.inv_J[2];
}

// classic RK4 with the control held over the step (the stage sums two
// components per packed FP32 instruction)
__device__ __forceinline__ void rk4_step(const RefineParams& R, float (&x)[12], const float (&u)[4]) {
    const float h = R.h;
    float k[12], acc[12], xs[12];
    quad_f(R, x, u, k);
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = k[i];
    fma_pairs(xs, 0.5f * h, k, x);
    quad_f(R, xs, u, k);
    fma_pairs(acc, 2.0f, k, acc);
    fma_pairs(xs, 0.5f * h, k, x);
    quad_f(R, xs, u, k);
    fma_pairs(acc, 2.0f, k, acc);
    fma_pairs(xs, h, k, x);
    quad_f(R, xs, u, k);
    add_pairs(acc, acc, k);
    fma_pairs(x, h / 6.0f, acc, x);
}

// One RK4 stage as the adjoint needs it: the sine/cosine of the stage state's
// angles (and 1 / cos(theta)) and its body rates.
constexpr int STAGE_WORDS = 10;

__device__ __forceinline__ void put_stage(float* w, const Trig& T, const float (&x)[12]) {
    w[0] = T.sphi;
    w[1] = T.cphi;
    w[2] = T.sth;
    w[3] = T.cth;
    w[4] = T.spsi;
    w[5] = T.cpsi;
    w[6] = T.ic;
    w[7] = x[9];
    w[8] = x[10];
    w[9] = x[11];
}

// rk4_step() that also writes its four stages to rec[4 * STAGE_WORDS] (lane 0)
__device__ __forceinline__ void rk4_step_rec(const RefineParams& R, float (&x)[12], const float (&u)[4], float* rec,
                                             bool writer) {
    const float h = R.h;
    float k[12], acc[12], xs[12];
    Trig T = trig_of(x);
    if (writer) put_stage(rec, T, x);
    quad_f_t(R, T, x, u, k);
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = k[i];
    fma_pairs(xs, 0.5f * h, k, x);
    T = trig_of(xs);
    if (writer) put_stage(rec + STAGE_WORDS, T, xs);
    quad_f_t(R, T, xs, u, k);
    fma_pairs(acc, 2.0f, k, acc);
    fma_pairs(xs, 0.5f * h, k, x);
    T = trig_of(xs);
    if (writer) put_stage(rec + 2 * STAGE_WORDS, T, xs);
    quad_f_t(R, T, xs, u, k);
    fma_pairs(acc, 2.0f, k, acc);
    fma_pairs(xs, h, k, x);
    T = trig_of(xs);
    if (writer) put_stage(rec + 3 * STAGE_WORDS, T, xs);
    quad_f_t(R, T, xs, u, k);
    add_pairs(acc, acc, k);
    fma_pairs(x, h / 6.0f, acc, x);
}

__device__ __forceinline__ void vjp_stage(const RefineParams& R, const float* w, const float (&u)[4],
                                          const float (&a)[12], float (&gx)[12], float (&gu)[4]) {
    Trig T;
    T.sphi = w[0];
    T.cphi = w[1];
    T.sth = w[2];
    T.cth = w[3];
    T.spsi = w[4];
    T.cpsi = w[5];
    T.ic = w[6];
    quad_vjp_t(R, T, w[7], w[8], w[9], u, a, gx, gu);
}

// Adjoint of one RK4 step: lam (dJ/dx_{k+1}) becomes dJ/dx_k; gu gets dJ/du
// through this step.  The four stages come from rk4_step_rec(), so no stage
// is re-evaluated on the serial chain of the backward pass.  The
// component-wise sums run two per packed FP32 instruction.
__device__ __forceinline__ void rk4_adjoint_rec(const RefineParams& R, const float* rec, const float (&u)[4],
                                                float (&lam)[12], float (&gu)[4]) {
    const float h = R.h;
    float ax[12], ak[12], g[12], t[12], gus[4];
#pragma unroll
    for (int i = 0; i < 12; ++i) ax[i] = lam[i];
    mul_pairs(ak, h / 6.0f, lam);                        // adjoint of k4
    vjp_stage(R, rec + 3 * STAGE_WORDS, u, ak, g, gus);  // k4 = f(x + h k3)
    add_pairs(ax, ax, g);
    mul_pairs(t, h / 3.0f, lam);
    fma_pairs(ak, h, g, t);  // adjoint of k3
#pragma unroll
    for (int i = 0; i < 4; ++i) gu[i] += gus[i];
    vjp_stage(R, rec + 2 * STAGE_WORDS, u, ak, g, gus);  // k3 = f(x + h/2 k2)
    add_pairs(ax, ax, g);
    fma_pairs(ak, 0.5f * h, g, t);  // adjoint of k2
#pragma unroll
    for (int i = 0; i < 4; ++i) gu[i] += gus[i];
    vjp_stage(R, rec + STAGE_WORDS, u, ak, g, gus);  // k2 = f(x + h/2 k1)
    add_pairs(ax, ax, g);
    mul_pairs(t, h / 6.0f, lam);
    fma_pairs(ak, 0.5f * h, g, t);  // adjoint of k1
#pragma unroll
    for (int i = 0; i < 4; ++i) gu[i] += gus[i];
    vjp_stage(R, rec, u, ak, g, gus);  // k1 = f(x)
    add_pairs(lam, ax, g);
#pragma unroll
    for (int i = 0; i < 4; ++i) gu[i] += gus[i];
}

// ---------------------------------------------------------------------------
// obstacle penalty: sum_b sp(margin - d_b(p)), sp(z) = log(1 + exp(beta z))/beta,
// d_b the signed distance to box b.  Each lane takes boxes lane, lane+32, ...
// ---------------------------------------------------------------------------
struct ObsSmem {
    const float* lo[3];
    const float* hi[3];
};

// the box's squared outside distance and the offsets behind it
__device__ __forceinline__ float box_offset(float px, float py, float pz, const ObsSmem& O, int b, float& dx, float& dy,
                                            float& dz) {
    dx = px - fminf(fmaxf(px, O.lo[0][b]), O.hi[0][b]);
    dy = py - fminf(fmaxf(py, O.lo[1][b]), O.hi[1][b]);
    dz = pz - fminf(fmaxf(pz, O.lo[2][b]), O.hi[2][b]);
    return dx * dx + dy * dy + dz * dz;
}

// inside a box: depth to the nearest face (first in the order x-lo, x-hi,
// y-lo, ... on ties) and the gradient of d = -depth
__device__ __forceinline__ float inside_distance(float px, float py, float pz, const ObsSmem& O, int b, float& gx,
                                                 float& gy, float& gz) {
    float best = px - O.lo[0][b];
    gx = -1.0f;
    gy = 0.0f;
    gz = 0.0f;
    float c = O.hi[0][b] - px;
    if (c < best) { best = c; gx = 1.0f; }
    c = py - O.lo[1][b];
    if (c < best) { best = c; gx = 0.0f; gy = -1.0f; }
    c = O.hi[1][b] - py;
    if (c < best) { best = c; gx = 0.0f; gy = 1.0f; }
    c = pz - O.lo[2][b];
    if (c < best) { best = c; gx = 0.0f; gy = 0.0f; gz = -1.0f; }
    c = O.hi[2][b] - pz;
    if (c < best) { best = c; gx = 0.0f; gy = 0.0f; gz = 1.0f; }
    return -best;
}

// beta * sp = log(1 + exp(t)), t = beta (margin - d)
__device__ __forceinline__ float softplus_t(float t) { return fmaxf(t, 0.0f) + log1pf(__expf(-fabsf(t))); }

__device__ __forceinline__ float sigmoid_t(float t) {
    const float e = __expf(-fabsf(t));
    const float r = __frcp_rn(1.0f + e);
    return t >= 0.0f ? r : e * r;
}

// the squared distance beyond which beta (margin - d) < SOFTPLUS_CUT
__device__ __forceinline__ float far_distance2(const RefineParams& R) {
    const float d = R.margin - SOFTPLUS_CUT * R.inv_beta;
    return d > 0.0f ? d * d : 0.0f;
}

// ---------------------------------------------------------------------------
// broad phase of the box sum.  The grid covers the boxes grown by the far
// distance (a little more, so that rounding never drops a box a point
// reaches); cell c lists in index order every box whose grown box meets it,
// so a point's cell holds every box whose term survives the cutoff.  The
// exact squared-distance test still decides each candidate, and a cell's
// list keeps index order, so the sum is the same on every call.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float grid_grow(const RefineParams& R) {
    const float d = R.margin - SOFTPLUS_CUT * R.inv_beta;
    return d > 0.0f ? d * 1.0001f + 1e-6f : 0.0f;
}

__device__ __forceinline__ int grid_axis_cell(float v, float lo, float inv) {
    return (int)fminf(fmaxf((v - lo) * inv, 0.0f), (float)(REFINE_GRID_AXIS - 1));
}

// whether box b's grown box meets cell (cx, cy, cz)
__device__ __forceinline__ bool grid_covers(const RefineParams& R, const RefineGridHeader& H, float grow, int b,
                                            int cx, int cy, int cz) {
    const int c[3] = {cx, cy, cz};
    bool in = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int c0 = grid_axis_cell(R.obs[6 * b + a] - grow, H.lo[a], H.inv_cs[a]);
        const int c1 = grid_axis_cell(R.obs[6 * b + 3 + a] + grow, H.lo[a], H.inv_cs[a]);
        in &= c[a] >= c0 && c[a] <= c1;
    }
    return in;
}

// one block: the grid's extent (zeroes the counters)
__global__ void k_grid_bounds(RefineParams R) {
    __shared__ float s_mn[3][32], s_mx[3][32];
    const float INF = __int_as_float(0x7F800000);
    float mn[3] = {INF, INF, INF}, mx[3] = {-INF, -INF, -INF};
    for (int b = threadIdx.x; b < R.n_obs; b += blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            mn[a] = fminf(mn[a], R.obs[6 * b + a]);
            mx[a] = fmaxf(mx[a], R.obs[6 * b + 3 + a]);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(0xFFFFFFFFu, mn[a], o));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xFFFFFFFFu, mx[a], o));
        }
        if (lane == 0) {
            s_mn[a][warp] = mn[a];
            s_mx[a][warp] = mx[a];
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    RefineGridHeader* H = R.grid;
    const float grow = grid_grow(R);
    for (int a = 0; a < 3; ++a) {
        float lo = INF, hi = -INF;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            lo = fminf(lo, s_mn[a][w]);
            hi = fmaxf(hi, s_mx[a][w]);
        }
        if (!(lo <= hi)) lo = hi = 0.0f;  // no boxes
        lo -= grow;
        hi += grow;
        H->lo[a] = lo;
        H->inv_cs[a] = hi > lo ? (float)REFINE_GRID_AXIS / (hi - lo) : 0.0f;
    }
    H->ok = 0;
    H->total = 0;
    for (int k = 0; k < 4; ++k) H->tests[k] = 0ull;
}

// one thread per cell: the number of boxes the cell lists
__global__ void k_grid_count(RefineParams R) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= REFINE_GRID_CELLS) return;
    const RefineGridHeader H = *R.grid;
    const float grow = grid_grow(R);
    const int cx = c % REFINE_GRID_AXIS, cy = (c / REFINE_GRID_AXIS) % REFINE_GRID_AXIS,
              cz = c / (REFINE_GRID_AXIS * REFINE_GRID_AXIS);
    int n = 0;
    for (int b = 0; b < R.n_obs; ++b) n += grid_covers(R, H, grow, b, cx, cy, cz) ? 1 : 0;
    R.grid_off[c] = n;
}

// one block of 1024 threads: counts -> offsets; the grid is used only when
// every entry fits
__global__ void __launch_bounds__(1024) k_grid_scan(RefineParams R) {
    constexpr int PER = REFINE_GRID_CELLS / 1024;
    __shared__ int s_warp[32];
    int v[PER], sum = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        v[q] = R.grid_off[threadIdx.x * PER + q];
        sum += v[q];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    int run = x - sum + (warp > 0 ? s_warp[warp - 1] : 0);
    __syncthreads();  // every count is read before any offset is written
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        R.grid_off[threadIdx.x * PER + q] = run;
        run += v[q];
    }
    if (threadIdx.x == 1023) {
        R.grid_off[REFINE_GRID_CELLS] = run;
        R.grid->total = run;
        R.grid->ok = run <= REFINE_GRID_ENTRIES ? 1 : 0;
    }
}

// one thread per cell: the cell's boxes in index order
__global__ void k_grid_fill(RefineParams R) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= REFINE_GRID_CELLS) return;
    const RefineGridHeader H = *R.grid;
    if (!H.ok) return;
    const float grow = grid_grow(R);
    const int cx = c % REFINE_GRID_AXIS, cy = (c / REFINE_GRID_AXIS) % REFINE_GRID_AXIS,
              cz = c / (REFINE_GRID_AXIS * REFINE_GRID_AXIS);
    int pos = R.grid_off[c];
    for (int b = 0; b < R.n_obs; ++b)
        if (grid_covers(R, H, grow, b, cx, cy, cz)) R.grid_ids[pos++] = (uint16_t)b;
}

// where a point's candidate boxes come from: its grid cell, or every box
// (the grid's extent is read from the header, L1-resident, at each use)
struct BoxSource {
    const RefineGridHeader* H;
    const int32_t* off;
    const uint16_t* ids;
    bool grid;
};

__device__ __forceinline__ BoxSource box_source(const RefineParams& R) {
    BoxSource S;
    S.grid = R.grid && R.grid->ok;
    S.H = R.grid;
    S.off = R.grid_off;
    S.ids = R.grid_ids;
    return S;
}

__device__ __forceinline__ void candidates(const BoxSource& S, int n_obs, float px, float py, float pz, int& e0,
                                           int& e1) {
    if (!S.grid) {
        e0 = 0;
        e1 = n_obs;
        return;
    }
    const RefineGridHeader* H = S.H;
    const int c = (grid_axis_cell(pz, H->lo[2], H->inv_cs[2]) * REFINE_GRID_AXIS +
                   grid_axis_cell(py, H->lo[1], H->inv_cs[1])) *
                      REFINE_GRID_AXIS +
                  grid_axis_cell(px, H->lo[0], H->inv_cs[0]);
    e0 = S.off[c];
    e1 = S.off[c + 1];
}

__device__ __forceinline__ int box_of(const BoxSource& S, int e) { return S.grid ? (int)S.ids[e] : e; }

// beta * sum_b sp(margin - d_b(p)) at one point, every candidate box of its
// cell in order; far2 = the squared distance beyond which a box's term is
// dropped
__device__ __forceinline__ float penalty_point(const RefineParams& R, const ObsSmem& O, const BoxSource& S, float px,
                                               float py, float pz, float far2, uint32_t& n_test, uint32_t& n_near) {
    float acc = 0.0f;
    int e0, e1;
    candidates(S, R.n_obs, px, py, pz, e0, e1);
    for (int e = e0; e < e1; ++e) {
        const int b = box_of(S, e);
        float dx, dy, dz;
        const float o2 = box_offset(px, py, pz, O, b, dx, dy, dz);
        ++n_test;
        if (o2 >= far2) continue;
        ++n_near;
        float gx, gy, gz;
        const float d = o2 > 0.0f ? sqrtf(o2) : inside_distance(px, py, pz, O, b, gx, gy, gz);
        acc += softplus_t(R.beta * (R.margin - d));
    }
    return acc;
}

// d/dp sum_b sp(margin - d_b(p)) = -sum_b sigma(t) grad d_b at one point
__device__ __forceinline__ void penalty_grad_point(const RefineParams& R, const ObsSmem& O, const BoxSource& S,
                                                   float px, float py, float pz, float far2, float& ox, float& oy,
                                                   float& oz, uint32_t& n_test, uint32_t& n_near) {
    ox = oy = oz = 0.0f;
    int e0, e1;
    candidates(S, R.n_obs, px, py, pz, e0, e1);
    for (int e = e0; e < e1; ++e) {
        const int b = box_of(S, e);
        float dx, dy, dz;
        const float o2 = box_offset(px, py, pz, O, b, dx, dy, dz);
        ++n_test;
        if (o2 >= far2) continue;
        ++n_near;
        float gx, gy, gz, d;
        if (o2 > 0.0f) {
            d = sqrtf(o2);
            const float id = __frcp_rn(d);
            gx = dx * id;
            gy = dy * id;
            gz = dz * id;
        } else {
            d = inside_distance(px, py, pz, O, b, gx, gy, gz);
        }
        const float s = sigmoid_t(R.beta * (R.margin - d));
        ox -= s * gx;
        oy -= s * gy;
        oz -= s * gz;
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// the warp's box tests into the grid header's counters k, k + 1
__device__ __forceinline__ void count_tests(const RefineParams& R, int k, uint32_t n_test, uint32_t n_near) {
    unsigned long long t = n_test, n = n_near;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
        n += __shfl_xor_sync(0xFFFFFFFFu, n, o);
    }
    if ((threadIdx.x & 31) == 0 && R.grid) {
        atomicAdd(&R.grid->tests[k], t);
        atomicAdd(&R.grid->tests[k + 1], n);
    }
}

// stages the boxes (SoA) into shared memory; returns the views
__device__ __forceinline__ ObsSmem stage_obstacles(const RefineParams& R, float* smem) {
    ObsSmem O;
    const int M = R.n_obs;
    for (int a = 0; a < 3; ++a) {
        O.lo[a] = smem + a * M;
        O.hi[a] = smem + (3 + a) * M;
    }
    for (int i = threadIdx.x; i < 6 * M; i += blockDim.x) {
        const int b = i / 6, c = i - 6 * b;
        smem[c * M + b] = R.obs[i];
    }
    __syncthreads();
    return O;
}

__device__ __forceinline__ float effort_cost(const RefineParams& R, const float (&u)[4], int K, float (&g)[4]) {
    const float dur = (float)K * R.h;
    const float et = (u[0] - R.mg) / R.mg;
    const float it2 = 1.0f / (R.tau_max * R.tau_max);
    const float e = et * et + (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) * it2;
    g[0] = dur * R.w_effort * 2.0f * (u[0] - R.mg) / (R.mg * R.mg);
#pragma unroll
    for (int i = 1; i < 4; ++i) g[i] = dur * R.w_effort * 2.0f * u[i] * it2;
    return dur * (1.0f + R.w_effort * e);
}

__device__ __forceinline__ void load_u(const RefineParams& R, int64_t tr, int s, float (&u)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(R.u + (tr * R.max_segments + s) * 4);
    u[0] = v.x;
    u[1] = v.y;
    u[2] = v.z;
    u[3] = v.w;
}

// ---------------------------------------------------------------------------
// forward: the objective of each trajectory; with a gradient requested, the
// state every REFINE_CKPT_STEPS steps (and the segment position there)
// ---------------------------------------------------------------------------
template <bool CKPT>
__global__ void __launch_bounds__(ADJ_WARPS * 32) k_refine_forward(RefineParams R) {
    extern __shared__ float smem[];
    const ObsSmem O = stage_obstacles(R, smem);
    const int lane = threadIdx.x & 31;
    const int64_t slot = (int64_t)blockIdx.x * ADJ_WARPS + (threadIdx.x >> 5);
    if (slot >= R.count) return;
    const int64_t tr = R.order ? R.order[slot] : slot;
    const int S = R.n_seg[tr];
    int total = 0;
    for (int s = 0; s < S && s < R.max_segments; ++s) total += R.steps[tr * R.max_segments + s];
    if (S < 0 || S > R.max_segments || total > R.max_total_steps) {
        if (lane == 0) R.cost[tr] = __int_as_float(0x7FC00000);  // NaN: the trajectory does not fit
        return;
    }
    const float far2 = far_distance2(R);
    const BoxSource BS = box_source(R);
    uint32_t n_test = 0, n_near = 0;
    float x[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) x[i] = R.x0[tr * 12 + i];
    float effort = 0.0f, pen = 0.0f;
    float px = 0.0f, py = 0.0f, pz = 0.0f;  // this lane's point of the current block of 32 steps
    int step = 0;
    for (int s = 0; s < S; ++s) {
        float u[4], gdummy[4];
        load_u(R, tr, s, u);
        const int K = R.steps[tr * R.max_segments + s];
        effort += effort_cost(R, u, K, gdummy);
        for (int j = 0; j < K; ++j, ++step) {
            if (CKPT && step % REFINE_CKPT_STEPS == 0) {
                float* c = R.ckpt + (tr * R.n_ckpt + step / REFINE_CKPT_STEPS) * REFINE_CKPT_WORDS;
#pragma unroll
                for (int i = 0; i < 12; ++i)
                    if (lane == i) c[i] = x[i];
                if (lane == 12) c[12] = __int_as_float(s);
                if (lane == 13) c[13] = __int_as_float(j);
            }
            rk4_step(R, x, u);
            const int t = step & 31;
            if (lane == t) {
                px = x[0];
                py = x[1];
                pz = x[2];
            }
            if (t == 31) pen += penalty_point(R, O, BS, px, py, pz, far2, n_test, n_near);  // 32 points, one a lane
        }
    }
    if (lane < (step & 31)) pen += penalty_point(R, O, BS, px, py, pz, far2, n_test, n_near);  // the last block
    count_tests(R, 0, n_test, n_near);
    pen = warp_sum(pen);
    if (lane == 0) {
        float goal = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) goal += (x[a] - R.goal[a]) * (x[a] - R.goal[a]);
        R.cost[tr] = effort + R.w_obs * R.inv_beta * pen + R.w_goal * goal;
    }
}

// ---------------------------------------------------------------------------
// backward: dJ/du by the adjoint recursion, interval by interval
// ---------------------------------------------------------------------------
// per warp: the interval's states, segment ids, penalty gradients and RK4 stages
constexpr int BWD_WARP_FLOATS =
    (REFINE_CKPT_STEPS + 1) * 12 + REFINE_CKPT_STEPS + 3 * REFINE_CKPT_STEPS + 4 * STAGE_WORDS * REFINE_CKPT_STEPS;

__global__ void __launch_bounds__(ADJ_WARPS * 32) k_refine_backward(RefineParams R) {
    extern __shared__ float smem[];
    const ObsSmem O = stage_obstacles(R, smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // per-warp scratch after the boxes: the interval's states, segment ids and
    // the penalty gradient at each step's end point
    float* xs = smem + 6 * R.n_obs + warp * BWD_WARP_FLOATS;
    int* seg_of = reinterpret_cast<int*>(xs + (REFINE_CKPT_STEPS + 1) * 12);
    float* pg = xs + (REFINE_CKPT_STEPS + 1) * 12 + REFINE_CKPT_STEPS;
    float* stages = pg + 3 * REFINE_CKPT_STEPS;  // [step][4 stages][STAGE_WORDS]
    const int64_t slot = (int64_t)blockIdx.x * ADJ_WARPS + warp;
    if (slot >= R.count) return;
    const int64_t tr = R.order ? R.order[slot] : slot;
    const int S = R.n_seg[tr];
    int total = 0;
    for (int s = 0; s < S && s < R.max_segments; ++s) total += R.steps[tr * R.max_segments + s];
    float* G = R.grad + tr * R.max_segments * 4;
    if (S < 0 || S > R.max_segments || total > R.max_total_steps) {
        for (int i = lane; i < R.max_segments * 4; i += 32) G[i] = 0.0f;
        return;
    }
    const float far2 = far_distance2(R);
    const BoxSource BS = box_source(R);
    uint32_t n_test = 0, n_near = 0;
    // the effort part of every segment's gradient (padding rows: 0)
    for (int s = lane; s < R.max_segments; s += 32) {
        float u[4], g[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (s < S) {
            load_u(R, tr, s, u);
            effort_cost(R, u, R.steps[tr * R.max_segments + s], g);
        }
        *reinterpret_cast<float4*>(G + 4 * s) = make_float4(g[0], g[1], g[2], g[3]);
    }
    __syncwarp();
    float lam[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) lam[i] = 0.0f;
    float gu[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    int cur_seg = -1;
    float u[4];
    const int n_ck = (total + REFINE_CKPT_STEPS - 1) / REFINE_CKPT_STEPS;
    for (int c = n_ck - 1; c >= 0; --c) {
        const int c0 = c * REFINE_CKPT_STEPS;
        const int len = min(REFINE_CKPT_STEPS, total - c0);
        // re-integrate the interval from its checkpoint
        const float* ck = R.ckpt + (tr * R.n_ckpt + c) * REFINE_CKPT_WORDS;
        float x[12];
#pragma unroll
        for (int i = 0; i < 12; ++i) x[i] = ck[i];
        int s = __float_as_int(ck[12]), j = __float_as_int(ck[13]);
        load_u(R, tr, s, u);
        for (int t = 0; t < len; ++t) {
            while (j >= R.steps[tr * R.max_segments + s]) {  // next non-empty segment
                ++s;
                j = 0;
                load_u(R, tr, s, u);
            }
#pragma unroll
            for (int i = 0; i < 12; ++i)
                if (lane == i) xs[t * 12 + i] = x[i];
            if (lane == 0) seg_of[t] = s;
            rk4_step_rec(R, x, u, stages + t * 4 * STAGE_WORDS, lane == 0);
            ++j;
        }
#pragma unroll
        for (int i = 0; i < 12; ++i)
            if (lane == i) xs[len * 12 + i] = x[i];
        __syncwarp();
        // the penalty at p_{k+1} of every step of the interval, one step a
        // lane: d/dp w_obs sp(margin - d) = -w_obs sigma grad d (it depends on
        // the stored states only, not on the adjoint)
        if (lane < len) {
            float ox, oy, oz;
            penalty_grad_point(R, O, BS, xs[(lane + 1) * 12 + 0], xs[(lane + 1) * 12 + 1], xs[(lane + 1) * 12 + 2],
                               far2, ox, oy, oz, n_test, n_near);
            pg[3 * lane] = ox;
            pg[3 * lane + 1] = oy;
            pg[3 * lane + 2] = oz;
        }
        __syncwarp();
        if (c == n_ck - 1) {  // dJ/dx_N of the goal pull
#pragma unroll
            for (int a = 0; a < 3; ++a) lam[a] = 2.0f * R.w_goal * (x[a] - R.goal[a]);
        }
        for (int t = len - 1; t >= 0; --t) {
            lam[0] += R.w_obs * pg[3 * t];
            lam[1] += R.w_obs * pg[3 * t + 1];
            lam[2] += R.w_obs * pg[3 * t + 2];
            const int sk = seg_of[t];
            if (sk != cur_seg) {  // entering an earlier segment: commit the later one
                if (cur_seg >= 0 && lane == 0) {
                    float4* q = reinterpret_cast<float4*>(G + 4 * cur_seg);
                    const float4 v = *q;
                    *q = make_float4(v.x + gu[0], v.y + gu[1], v.z + gu[2], v.w + gu[3]);
                }
                gu[0] = gu[1] = gu[2] = gu[3] = 0.0f;
                cur_seg = sk;
                load_u(R, tr, sk, u);
            }
            rk4_adjoint_rec(R, stages + t * 4 * STAGE_WORDS, u, lam, gu);
        }
        __syncwarp();
    }
    if (cur_seg >= 0 && lane == 0) {
        float4* q = reinterpret_cast<float4*>(G + 4 * cur_seg);
        const float4 v = *q;
        *q = make_float4(v.x + gu[0], v.y + gu[1], v.z + gu[2], v.w + gu[3]);
    }
    count_tests(R, 2, n_test, n_near);
}

// ---------------------------------------------------------------------------
// optimiser: one projected Adam step on the controls scaled to [-1, 1] by
// the control box, and the best iterate per trajectory
// ---------------------------------------------------------------------------
__global__ void k_refine_adam(AdamParams A) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = (int64_t)A.count * A.max_segments * 4;
    if (i >= n) return;
    const int c = (int)(i & 3);
    const int64_t row = i >> 2;
    const int64_t tr = row / A.max_segments;
    const int s = (int)(row - tr * A.max_segments);
    if (s >= A.n_seg[tr]) return;
    // the component's box, selected without indexing the parameter arrays
    const float lo = c == 0 ? A.lo[0] : (c == 1 ? A.lo[1] : (c == 2 ? A.lo[2] : A.lo[3]));
    const float hi = c == 0 ? A.hi[0] : (c == 1 ? A.hi[1] : (c == 2 ? A.hi[2] : A.hi[3]));
    const float half = 0.5f * (hi - lo);
    const float mid = 0.5f * (hi + lo);
    const float g = A.grad[i] * half;  // gradient in the scaled coordinate
    const float m = A.b1 * A.m1[i] + (1.0f - A.b1) * g;
    const float v = A.b2 * A.m2[i] + (1.0f - A.b2) * g * g;
    A.m1[i] = m;
    A.m2[i] = v;
    float z = (A.u[i] - mid) / half;
    z -= A.lr * (m / A.c1) / (sqrtf(v / A.c2) + A.eps);
    z = fminf(fmaxf(z, -1.0f), 1.0f);
    A.u[i] = mid + half * z;
}

__global__ void k_refine_keep_best(int32_t count, int32_t max_segments, const float* u, const float* J,
                                   float* u_best, float* J_best) {
    const int64_t tr = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (tr >= count) return;
    const float j = J[tr];
    if (!(j < J_best[tr])) return;  // NaN never wins
    const int lane = threadIdx.x & 31;
    for (int k = lane; k < max_segments * 4; k += 32) u_best[tr * max_segments * 4 + k] = u[tr * max_segments * 4 + k];
    if (lane == 0) J_best[tr] = j;
}

cudaError_t set_smem(const void* fn, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

cudaError_t launch_refine_eval(const RefineParams& R, cudaStream_t s) {
    if (R.count == 0) return cudaSuccess;
    const int blocks = (R.count + ADJ_WARPS - 1) / ADJ_WARPS;
    const size_t smem_obs = (size_t)6 * R.n_obs * sizeof(float);
    cudaError_t e = cudaSuccess;
    if (R.grid) {  // the box grid of this call's boxes and cost
        k_grid_bounds<<<1, 1024, 0, s>>>(R);
        k_grid_count<<<REFINE_GRID_CELLS / 256, 256, 0, s>>>(R);
        k_grid_scan<<<1, 1024, 0, s>>>(R);
        k_grid_fill<<<REFINE_GRID_CELLS / 256, 256, 0, s>>>(R);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (!R.grad) {
        e = set_smem((const void*)k_refine_forward<false>, smem_obs);
        if (e == cudaSuccess) {
            k_refine_forward<false><<<blocks, ADJ_WARPS * 32, smem_obs, s>>>(R);
            e = cudaGetLastError();
        }
        return e;
    }
    e = set_smem((const void*)k_refine_forward<true>, smem_obs);
    if (e == cudaSuccess) {
        k_refine_forward<true><<<blocks, ADJ_WARPS * 32, smem_obs, s>>>(R);
        e = cudaGetLastError();
    }
    const size_t smem_bwd = smem_obs + (size_t)ADJ_WARPS * BWD_WARP_FLOATS * sizeof(float);
    if (e == cudaSuccess) e = set_smem((const void*)k_refine_backward, smem_bwd);
    if (e == cudaSuccess) {
        k_refine_backward<<<blocks, ADJ_WARPS * 32, smem_bwd, s>>>(R);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_refine_adam(const AdamParams& A, cudaStream_t s) {
    const int64_t n = (int64_t)A.count * A.max_segments * 4;
    if (n == 0) return cudaSuccess;
    k_refine_adam<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_refine_keep_best(int32_t count, int32_t max_segments, const float* u, const float* cost,
                                    float* u_best, float* cost_best, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    k_refine_keep_best<<<(count + 7) / 8, 256, 0, s>>>(count, max_segments, u, cost, u_best, cost_best);
    return cudaGetLastError();
}

}  // namespace kpx
