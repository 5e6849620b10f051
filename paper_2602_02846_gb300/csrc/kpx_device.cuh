// kpx_device.cuh -- device-side arithmetic of one Kino-PAX+ rollout.
//
// Compiled with -fmad=false: every FP32 operation rounds once, and fused
// multiply-adds appear only where written as fmaf().  The propagate kernel
// and the append kernel inline the same functions, so a winner's rollout is
// re-materialised bit-identically from (seed, iteration, node, sample).
#pragma once

#include <cstdint>

#include "kpx_internal.h"

namespace kpx {

// --------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 products per 4-word counter, key bumped by the Weyl constants.
// --------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// "Randomly sample u and dt" (Alg. 2): counter (iteration, node, sample,
// block), key = seed words.  u_i = lo + (hi - lo) * f, f = (w >> 8) 2^-24,
// one FP32 rounding per operation; K from word m (block 1 word 0 when m = 4).
__device__ __forceinline__ int steps_from_word(const DevParams& P, uint32_t wk) {
    const uint64_t range = (uint64_t)(P.k_max - P.k_min + 1);
    return P.k_min + (int)(((uint64_t)wk * range) >> 32);
}

template <int M>
__device__ __forceinline__ void sample_control(const DevParams& P, uint32_t iter, uint32_t node, uint32_t s,
                                               float (&u)[M], int& K) {
    const uint2 key = make_uint2(P.seed_lo, P.seed_hi);
    const uint4 w0 = philox4x32_10(make_uint4(iter, node, s, 0u), key);
    const uint32_t w[4] = {w0.x, w0.y, w0.z, w0.w};
    uint32_t wk;
    if (M == 4) {
        const uint4 w1 = philox4x32_10(make_uint4(iter, node, s, 1u), key);
        wk = w1.x;
    } else {
        wk = w[M];
    }
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const float f = __fmul_rn(__uint2float_rn(w[i] >> 8), 0x1p-24f);
        u[i] = __fadd_rn(P.u_lo[i], __fmul_rn(__fsub_rn(P.u_hi[i], P.u_lo[i]), f));
    }
    K = steps_from_word(P, wk);
}

// The step count K of sample_control() alone (the same Philox word).
template <int M>
__device__ __forceinline__ int sample_steps(const DevParams& P, uint32_t iter, uint32_t node, uint32_t s) {
    const uint2 key = make_uint2(P.seed_lo, P.seed_hi);
    const uint4 w = philox4x32_10(make_uint4(iter, node, s, M == 4 ? 1u : 0u), key);
    return steps_from_word(P, M == 4 ? w.x : (M == 3 ? w.w : w.z));
}

// --------------------------------------------------------------------------
// Dynamics (the three systems of Sec. V; textbook equations).
// --------------------------------------------------------------------------
template <int DYN>
struct Dims;
template <>
struct Dims<KPX_DI6> {
    static constexpr int n = 6, m = 3;
};
template <>
struct Dims<KPX_DUBINS6> {
    static constexpr int n = 6, m = 3;
};
template <>
struct Dims<KPX_QUAD12> {
    static constexpr int n = 12, m = 4;
};

// sin and cos through the special-function unit after a two-constant
// Cody-Waite reduction of the angle to [-pi, pi] (the hardware sine and
// cosine are accurate to about 4e-7 absolute on that interval).
__device__ __forceinline__ float reduce_angle(float a) {
    constexpr float INV_TWO_PI = 0.15915494309189535f;
    constexpr float TWO_PI_HI = 6.28125f;                   // few significant bits: k * TWO_PI_HI is exact
    constexpr float TWO_PI_LO = 1.9353071795864769e-3f;     // 2 pi - TWO_PI_HI
    const float k = rintf(a * INV_TWO_PI);
    const float r = fmaf(-k, TWO_PI_HI, a);
    return fmaf(-k, TWO_PI_LO, r);
}

__device__ __forceinline__ void fast_sincos(float a, float& s, float& c) { __sincosf(reduce_angle(a), &s, &c); }

// The special-function unit's approximate sine and cosine and reciprocal in
// their flush-to-zero forms (PTX sin / cos / rcp.approx.ftz.f32): they differ
// from the non-flushing forms only for subnormal arguments or results, which
// the quadcopter's angles (a subnormal angle is flushed to 0, whose sine is
// 0 either way) and cos(theta) >= cos(pi/4) do not produce.
__device__ __forceinline__ void sincos_sfu(float a, float& s, float& c) {
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(a));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c) : "f"(a));
}

__device__ __forceinline__ float rcp_sfu(float a) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

// The quadcopter's x' = f(x, u) with the sine and cosine of the yaw given:
// p' = v; v' = (T/m) R(phi,theta,psi) e3 - g e3 (R = Rz Ry Rx);
// (phi,theta,psi)' = W(phi,theta) omega; omega' = J^-1 (tau - omega x J omega).
// Roll and pitch stay near the state bounds' range (|phi|, |theta| <= pi/4 at
// every checked point; a stage point passes it by at most h |rate|), where the
// hardware sine and cosine need no range reduction.
template <bool ISO>
__device__ __forceinline__ void quad_deriv(const DevParams& P, const float (&x)[12], float sps, float cps,
                                           const float (&u)[4], float (&dx)[12]) {
    // The products and sums are paired into packed FP32 operations (two per
    // instruction, each component rounded as its scalar form; a negated
    // factor is exact), so the values are those of the scalar expressions
    //   r13 = cps (sth cph) + sps sph,  r23 = sps (sth cph) - cps sph,
    //   r33 = cth cph,  t1 = sph q + cph r,  theta' = cph q - sph r,
    //   phi' = (sth / cth) t1 + p,  psi' = t1 / cth,  v' = a (r13, r23, r33) - g e3.
    float sph, cph, sth, cth;
    sincos_sfu(x[3], sph, cph);
    sincos_sfu(x[4], sth, cth);
    const float inv_cth = rcp_sfu(cth);
    const float p = x[9], q = x[10], r = x[11];
    const float a = u[0] * P.inv_mass;
    const float2 sc_c = __fmul2_rn(make_float2(sth, cth), make_float2(cph, cph));      // (sth cph, r33)
    const float2 ss_c = __fmul2_rn(make_float2(sps, -cps), make_float2(sph, sph));     // (sps sph, -cps sph)
    const float2 rr = __ffma2_rn(make_float2(cps, sps), make_float2(sc_c.x, sc_c.x), ss_c);  // (r13, r23)
    const float2 cr = __fmul2_rn(make_float2(cph, -sph), make_float2(r, r));           // (cph r, -sph r)
    const float2 tq = __ffma2_rn(make_float2(sph, cph), make_float2(q, q), cr);        // (t1, theta')
    const float2 td = __fmul2_rn(make_float2(sth, tq.x), make_float2(inv_cth, inv_cth));  // (tan theta, psi')
    const float2 av = __fmul2_rn(make_float2(a, a), rr);                               // v'_x, v'_y
    dx[0] = x[6];
    dx[1] = x[7];
    dx[2] = x[8];
    dx[3] = fmaf(td.x, tq.x, p);
    dx[4] = tq.y;
    dx[5] = td.y;
    dx[6] = av.x;
    dx[7] = av.y;
    dx[8] = fmaf(a, sc_c.y, -P.param[1]);
    if constexpr (ISO) {
        dx[9] = u[1] * P.inv_J[0];
        dx[10] = u[2] * P.inv_J[1];
        dx[11] = u[3] * P.inv_J[2];
    } else {
        dx[9] = fmaf(-P.dJ[0] * q, r, u[1]) * P.inv_J[0];
        dx[10] = fmaf(-P.dJ[1] * r, p, u[2]) * P.inv_J[1];
        dx[11] = fmaf(-P.dJ[2] * p, q, u[3]) * P.inv_J[2];
    }
}

// ISO (quadcopter only): the inertia is isotropic (J_x = J_y = J_z), so the
// gyroscopic term omega x J omega is zero and omega' = tau / J.  With J
// isotropic both forms give the same FP32 values for finite states.
template <int DYN, bool ISO = false>
__device__ __forceinline__ void deriv(const DevParams& P, const float (&x)[Dims<DYN>::n],
                                      const float (&u)[Dims<DYN>::m], float (&dx)[Dims<DYN>::n]) {
    if constexpr (DYN == KPX_DI6) {
        // p' = v, v' = a
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            dx[i] = x[3 + i];
            dx[3 + i] = u[i];
        }
    } else if constexpr (DYN == KPX_DUBINS6) {
        // (x, y, z)' = v (cos psi cos gamma, sin psi cos gamma, sin gamma); angles and speed follow u
        float sp, cp, sg, cg;
        fast_sincos(x[3], sp, cp);
        fast_sincos(x[4], sg, cg);
        const float vc = x[5] * cg;
        dx[0] = vc * cp;
        dx[1] = vc * sp;
        dx[2] = x[5] * sg;
        dx[3] = u[0];
        dx[4] = u[1];
        dx[5] = u[2];
    } else {
        float sps, cps;
        fast_sincos(x[5], sps, cps);  // yaw is unbounded
        quad_deriv<ISO>(P, x, sps, cps, u, dx);
    }
}

// One PropagateODE step: forward Euler or classic RK4, control held constant.
template <int DYN, int INTEG, bool ISO = false>
__device__ __forceinline__ void step(const DevParams& P, float (&x)[Dims<DYN>::n], const float (&u)[Dims<DYN>::m]) {
    constexpr int n = Dims<DYN>::n;
    const float h = P.h;
    float k1[n];
    deriv<DYN, ISO>(P, x, u, k1);
    if constexpr (INTEG == KPX_EULER) {
#pragma unroll
        for (int i = 0; i < n; ++i) x[i] = fmaf(h, k1[i], x[i]);
    } else {
        // one accumulator: acc = k1 + 2 k2 + 2 k3 + k4, stages evaluated into k
        const float hh = 0.5f * h;
        const float h6 = h * (1.0f / 6.0f);
        float xt[n], acc[n];
#pragma unroll
        for (int i = 0; i < n; ++i) {
            acc[i] = k1[i];
            xt[i] = fmaf(hh, k1[i], x[i]);
        }
        deriv<DYN, ISO>(P, xt, u, k1);
#pragma unroll
        for (int i = 0; i < n; ++i) {
            acc[i] = fmaf(2.0f, k1[i], acc[i]);
            xt[i] = fmaf(hh, k1[i], x[i]);
        }
        deriv<DYN, ISO>(P, xt, u, k1);
#pragma unroll
        for (int i = 0; i < n; ++i) {
            acc[i] = fmaf(2.0f, k1[i], acc[i]);
            xt[i] = fmaf(h, k1[i], x[i]);
        }
        deriv<DYN, ISO>(P, xt, u, k1);
#pragma unroll
        for (int i = 0; i < n; ++i) x[i] = fmaf(h6, acc[i] + k1[i], x[i]);
    }
}

// --------------------------------------------------------------------------
// Validity of one checked point (X_valid of Sec. III): state bounds, the
// closed workspace box, and no closed obstacle box containing the position.
// NaN fails every comparison and is therefore invalid.
// --------------------------------------------------------------------------
// SYM: every non-position state bound is symmetric (x_lo[d] = -x_hi[d],
// infinities included, checked on the host), so x_lo[d] <= x <= x_hi[d] is
// exactly |x| <= x_hi[d] (NaN fails both forms): one comparison, not two.
template <int N, bool SYM = false>
__device__ __forceinline__ bool bounds_ok(const DevParams& P, const float (&x)[N]) {
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) ok &= (x[a] >= P.pos_lo[a]) & (x[a] <= P.pos_hi[a]);  // workspace and bounds
#pragma unroll
    for (int d = 3; d < N; ++d) {
        if constexpr (SYM)
            ok &= fabsf(x[d]) <= P.x_hi[d];
        else
            ok &= (x[d] >= P.x_lo[d]) & (x[d] <= P.x_hi[d]);
    }
    return ok;
}

// Obstacle test through the uniform grid: only the boxes listed for the
// point's cell are tested (the list holds every box overlapping the cell,
// so the verdict equals testing all boxes).  The point must lie in the
// workspace box.  `tests` accumulates the number of boxes examined.
// Where the grid is read from: the workspace (global memory, read-only path)
// or a copy in shared memory (the fused kernel stages small grids).
struct GridView {
    const int32_t* cell_start;
    const float4* cell_box;
};

template <bool SMEM, typename T>
__device__ __forceinline__ T grid_ld(const T* p) {
    if constexpr (SMEM)
        return *p;
    else
        return __ldg(p);
}

// The entry range [e0, e1) of the point's cell.  Every coordinate, NaN and
// infinities included, maps to a cell of the grid, so the read stays in
// range for any point.
template <bool SMEM>
__device__ __forceinline__ void cell_range(const DevParams& P, const GridView& G, float px, float py, float pz,
                                           int& e0, int& e1) {
    const int cx = grid_cell(px, P.ws_lo[0], P.grid_inv[0], P.grid_n[0]);
    const int cy = grid_cell(py, P.ws_lo[1], P.grid_inv[1], P.grid_n[1]);
    const int cz = grid_cell(pz, P.ws_lo[2], P.grid_inv[2], P.grid_n[2]);
    const int c = (cz * P.grid_n[1] + cy) * P.grid_n[0] + cx;
    // the build keeps every offset within grid_entries <= grid_cap; a
    // shared-memory copy holds exactly grid_entries boxes
    e0 = grid_ld<SMEM>(G.cell_start + c);
    e1 = min(grid_ld<SMEM>(G.cell_start + c + 1), SMEM ? P.grid_entries : P.grid_cap);
}

// cell_range() for a point inside the workspace box (bounds_ok() passed:
// c >= pos_lo >= ws_lo on each axis), where (c - lo) * inv >= 0 needs no
// lower clamp; x and y in one packed pair.  The cell is cell_range()'s.
template <bool SMEM>
__device__ __forceinline__ void cell_range_ws(const DevParams& P, const GridView& G, float px, float py, float pz,
                                              int& e0, int& e1) {
    const float2 txy = __fmul2_rn(__fadd2_rn(make_float2(px, py), make_float2(-P.ws_lo[0], -P.ws_lo[1])),
                                  make_float2(P.grid_inv[0], P.grid_inv[1]));
    const float tz = __fmul_rn(__fsub_rn(pz, P.ws_lo[2]), P.grid_inv[2]);
    const int cx = (int)fminf(txy.x, (float)(P.grid_n[0] - 1));
    const int cy = (int)fminf(txy.y, (float)(P.grid_n[1] - 1));
    const int cz = (int)fminf(tz, (float)(P.grid_n[2] - 1));
    const int c = (cz * P.grid_n[1] + cy) * P.grid_n[0] + cx;
    if constexpr (SMEM) {
        e0 = G.cell_start[c];
        e1 = min(G.cell_start[c + 1], P.grid_entries);
    } else {  // the cell's (start, clamped end) pair, one load
        const int2 r = __ldg(P.cell_pair + c);
        e0 = r.x;
        e1 = r.y;
    }
}

// Tests the point against the boxes e0..e1-1 in order and stops at the
// first that contains it; `tests` accumulates the boxes examined.
template <bool SMEM>
__device__ __forceinline__ bool walk_cell(const GridView& G, float px, float py, float pz, int e0, int e1,
                                          uint32_t& tests) {
    for (int e = e0; e < e1; ++e) {
        const float4 lo = grid_ld<SMEM>(G.cell_box + 2 * e);
        const float4 hi = grid_ld<SMEM>(G.cell_box + 2 * e + 1);
        const bool in = (px >= lo.x) & (px <= hi.x) & (py >= lo.y) & (py <= hi.y) & (pz >= lo.z) & (pz <= hi.z);
        if (in) {
            tests += (uint32_t)(e - e0 + 1);
            return true;
        }
    }
    tests += (uint32_t)(e1 > e0 ? e1 - e0 : 0);
    return false;
}

template <bool SMEM = false>
__device__ __forceinline__ bool hits_obstacle_in(const DevParams& P, const GridView& G, float px, float py, float pz,
                                                 uint32_t& tests) {
    if (P.n_obs == 0) return false;
    int e0, e1;
    cell_range<SMEM>(P, G, px, py, pz, e0, e1);
    return walk_cell<SMEM>(G, px, py, pz, e0, e1, tests);
}

__device__ __forceinline__ bool hits_obstacle(const DevParams& P, float px, float py, float pz, uint32_t& tests) {
    return hits_obstacle_in<false>(P, GridView{P.cell_start, P.cell_box}, px, py, pz, tests);
}

// --------------------------------------------------------------------------
// Edge cost (Assumption 1): path length accumulated per step, duration K h,
// or effort+duration K h (1 + w e(u)).
// --------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ float edge_cost(const DevParams& P, int K, float path_len, const float (&u)[M]) {
    if (P.cost_kind == KPX_COST_PATH_LENGTH) return path_len;
    const float dur = __fmul_rn(__int2float_rn(K), P.h);
    if (P.cost_kind == KPX_COST_DURATION || M < 4) return dur;
    const float dt = (u[0] - P.mg) * P.inv_mg;
    float e = dt * dt;
#pragma unroll
    for (int i = 1; i < M; ++i) {
        const float t = u[i] * P.inv_tau_max;
        e = fmaf(t, t, e);
    }
    return dur * fmaf(P.w_effort, e, 1.0f);
}

// One integrator per (system, scheme).  The generic stepper applies step().
// The Dubins RK4 stepper uses that yaw and pitch turn at a constant rate
// under a constant control: the two RK4 midpoint stages coincide (k2 = k3),
// and the sine and cosine at the midpoint and at the end of a step follow
// from those at its start by two rotations through the half-step angle,
// whose sine and cosine are evaluated once per rollout.  A step thus needs
// no sine or cosine evaluation; the angles of the state itself are still
// advanced by one rounding per step.
template <int DYN, int INTEG>
struct Stepper {
    static constexpr int n = Dims<DYN>::n, m = Dims<DYN>::m;
    __device__ __forceinline__ void init(const DevParams&, const float (&)[n], const float (&)[m]) {}
    template <int ISO = -1>
    __device__ __forceinline__ void advance(const DevParams& P, float (&x)[n], const float (&u)[m]) {
        step<DYN, INTEG>(P, x, u);
    }
};

// d[i] = a b[i] + c[i], d[i] = a b[i] and d[i] = b[i] + c[i] over the
// components, two per packed FP32 instruction (sm_100 and later): each
// component rounds as the scalar fmaf / mul / add does, so the results are
// those of the scalar loops.
template <int N>
__device__ __forceinline__ void fma_pairs(float (&d)[N], float a, const float (&b)[N], const float (&c)[N]) {
    static_assert(N % 2 == 0, "pairs");
    const float2 a2 = make_float2(a, a);
#pragma unroll
    for (int i = 0; i < N; i += 2) {
        const float2 r = __ffma2_rn(a2, make_float2(b[i], b[i + 1]), make_float2(c[i], c[i + 1]));
        d[i] = r.x;
        d[i + 1] = r.y;
    }
}

template <int N>
__device__ __forceinline__ void mul_pairs(float (&d)[N], float a, const float (&b)[N]) {
    static_assert(N % 2 == 0, "pairs");
    const float2 a2 = make_float2(a, a);
#pragma unroll
    for (int i = 0; i < N; i += 2) {
        const float2 r = __fmul2_rn(a2, make_float2(b[i], b[i + 1]));
        d[i] = r.x;
        d[i + 1] = r.y;
    }
}

template <int N>
__device__ __forceinline__ void add_pairs(float (&d)[N], const float (&b)[N], const float (&c)[N]) {
    static_assert(N % 2 == 0, "pairs");
#pragma unroll
    for (int i = 0; i < N; i += 2) {
        const float2 r = __fadd2_rn(make_float2(b[i], b[i + 1]), make_float2(c[i], c[i + 1]));
        d[i] = r.x;
        d[i + 1] = r.y;
    }
}

// The quadcopter's RK4.  The yaw enters f only through its sine and cosine,
// so the stepper carries beside x[5] a copy yr of the yaw reduced to
// [-pi, pi] when the rollout starts and advanced by the same RK4 increments;
// a step that takes it past pi folds it back by 2 pi.  The stage yaws
// yr + c k then lie within [-pi, pi] widened by one stage's turn (about
// 0.02 rad), where the hardware sine and cosine need no reduction: four
// reductions fewer per step.  The copy rounds differently from a reduction
// of x[5] (both approximate the same angle to a few FP32 ulps of pi).  With
// isotropic inertia (flag set by the host when J_x = J_y = J_z exactly) the
// body rates' derivative is the constant tau / J, which the compiler keeps
// out of the step loop.  The stage sums run two components per packed FP32
// instruction.
template <bool ISO>
__device__ __forceinline__ void quad_rk4_step(const DevParams& P, float (&x)[12], float& yr, const float (&u)[4]) {
    constexpr float PI_F = 3.14159265358979323846f;
    constexpr float TWO_PI_F = 6.28318530717958647692f;
    const float h = P.h;
    const float hh = 0.5f * h;
    const float h6 = h * (1.0f / 6.0f);
    float k[12], acc[12], xt[12];
    float s, c;
    sincos_sfu(yr, s, c);
    quad_deriv<ISO>(P, x, s, c, u, k);
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = k[i];
    fma_pairs(xt, hh, k, x);
    sincos_sfu(fmaf(hh, k[5], yr), s, c);
    quad_deriv<ISO>(P, xt, s, c, u, k);
    fma_pairs(acc, 2.0f, k, acc);
    fma_pairs(xt, hh, k, x);
    sincos_sfu(fmaf(hh, k[5], yr), s, c);
    quad_deriv<ISO>(P, xt, s, c, u, k);
    fma_pairs(acc, 2.0f, k, acc);
    fma_pairs(xt, h, k, x);
    sincos_sfu(fmaf(h, k[5], yr), s, c);
    quad_deriv<ISO>(P, xt, s, c, u, k);
    add_pairs(acc, acc, k);  // acc + k4
    yr = fmaf(h6, acc[5], yr);
    fma_pairs(x, h6, acc, x);
    if (fabsf(yr) > PI_F) yr -= copysignf(TWO_PI_F, yr);
}

template <>
struct Stepper<KPX_QUAD12, KPX_RK4> {
    static constexpr int n = 12, m = 4;
    float yr;  // the yaw x[5] reduced to [-pi, pi]
    __device__ __forceinline__ void init(const DevParams&, const float (&x)[n], const float (&)[m]) {
        yr = reduce_angle(x[5]);
    }
    // ISO: 1 or 0 when the caller has read P.iso_inertia already, -1 to read it here
    template <int ISO = -1>
    __device__ __forceinline__ void advance(const DevParams& P, float (&x)[n], const float (&u)[m]) {
        if (ISO == 1 || (ISO < 0 && P.iso_inertia))
            quad_rk4_step<true>(P, x, yr, u);
        else
            quad_rk4_step<false>(P, x, yr, u);
    }
};

template <>
struct Stepper<KPX_DUBINS6, KPX_RK4> {
    static constexpr int n = 6, m = 3;
    float sp, cp, sg, cg;      // sin/cos of yaw and pitch at the current state
    float sdp, cdp, sdg, cdg;  // sin/cos of the half-step turns h u0 / 2 and h u1 / 2
    __device__ __forceinline__ void init(const DevParams& P, const float (&x)[n], const float (&u)[m]) {
        fast_sincos(x[3], sp, cp);
        fast_sincos(x[4], sg, cg);
        const float hh = 0.5f * P.h;
        sincosf(hh * u[0], &sdp, &cdp);
        sincosf(hh * u[1], &sdg, &cdg);
    }
    // (s, c) = sin and cos of (a + d) from those of a and of d:
    // (s cd + c sd, c cd - s sd), one packed FP32 multiply and one packed FMA
    __device__ __forceinline__ static float2 rotate2(float2 sc, float sd, float cd) {
        const float2 t = __fmul2_rn(make_float2(sc.y, -sc.x), make_float2(sd, sd));
        return __ffma2_rn(sc, make_float2(cd, cd), t);
    }
    template <int ISO = -1>
    __device__ __forceinline__ void advance(const DevParams& P, float (&x)[n], const float (&u)[m]) {
        const float h = P.h;
        const float hh = 0.5f * h;
        const float h6 = h * (1.0f / 6.0f);
        const float vs = x[5];
        const float vm = fmaf(hh, u[2], x[5]), ve = fmaf(h, u[2], x[5]);
        const float2 pm = rotate2(make_float2(sp, cp), sdp, cdp);  // yaw at the midpoint
        const float2 gm = rotate2(make_float2(sg, cg), sdg, cdg);  // pitch at the midpoint
        const float2 pe = rotate2(pm, sdp, cdp);                    // and at the end
        const float2 ge = rotate2(gm, sdg, cdg);
        // f = v (cos yaw cos pitch, sin yaw cos pitch, sin pitch) at start, mid, end;
        // (fx, fy) in packed pairs, (cos yaw, sin yaw) swapped into (x, y) order
        const float as = vs * cg, am = vm * gm.y, ae = ve * ge.y;
        const float2 fe = __fmul2_rn(make_float2(ae, ae), make_float2(pe.y, pe.x));
        const float2 fs = __ffma2_rn(make_float2(as, as), make_float2(cp, sp), fe);
        const float2 fm = __fmul2_rn(make_float2(am, am), make_float2(pm.y, pm.x));
        const float2 fxy = __ffma2_rn(make_float2(4.0f, 4.0f), fm, fs);
        const float fz = fmaf(4.0f, vm * gm.x, fmaf(vs, sg, ve * ge.x));
        const float2 pxy = __ffma2_rn(make_float2(h6, h6), fxy, make_float2(x[0], x[1]));
        x[0] = pxy.x;
        x[1] = pxy.y;
        x[2] = fmaf(h6, fz, x[2]);
        x[3] = fmaf(h, u[0], x[3]);
        x[4] = fmaf(h, u[1], x[4]);
        x[5] = ve;
        sp = pe.x;
        cp = pe.y;
        sg = ge.x;
        cg = ge.y;
    }
};

// Obstacle pass alone over a re-integrated segment (used after an early cost
// check; same integration arithmetic as rollout()).
template <int DYN, int INTEG, bool SMEM = false>
__device__ __forceinline__ bool obstacle_pass(const DevParams& P, const GridView& G, float (&x)[Dims<DYN>::n],
                                              const float (&u)[Dims<DYN>::m], int K, uint32_t& steps,
                                              uint32_t& tests) {
    Stepper<DYN, INTEG> st;
    st.init(P, x, u);
    for (int k = 0; k < K; ++k) {
        st.advance(P, x, u);
        ++steps;
        if (hits_obstacle_in<SMEM>(P, G, x[0], x[1], x[2], tests)) return false;
    }
    return true;
}

// --------------------------------------------------------------------------
// Region map (decomposition R of Sec. IV): per axis
// c = clamp(floor((x - lo) * scale), 0, bins - 1) in FP32, one rounding per
// operation; a wrapped axis first maps psi -> psi - 2 pi floor((psi + pi) / 2 pi).
// --------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ int region_of(const DevParams& P, const float (&x)[N]) {
    constexpr float PI_F = 3.14159265358979323846f;
    constexpr float TWO_PI_F = 6.28318530717958647692f;
    int id = 0;
#pragma unroll
    for (int d = 0; d < N; ++d) {  // components in a fixed order: no indexed access to x
        const int bins = P.rg_bins[d];
        if (bins > 0) {
            float xv = x[d];
            if (P.rg_wrap[d]) {
                const float t = __fdiv_rn(__fadd_rn(xv, PI_F), TWO_PI_F);
                xv = __fsub_rn(xv, __fmul_rn(TWO_PI_F, floorf(t)));
            }
            const float t = __fmul_rn(__fsub_rn(xv, P.rg_lo[d]), P.rg_scale[d]);
            int c = (int)floorf(t);
            c = c < 0 ? 0 : c;
            c = c > bins - 1 ? bins - 1 : c;
            id += c * P.rg_stride[d];
        }
    }
    return id;
}

__device__ __forceinline__ bool in_goal(const DevParams& P, float px, float py, float pz) {
    const float dx = px - P.goal_c[0], dy = py - P.goal_c[1], dz = pz - P.goal_c[2];
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= P.goal_r2;
}

__device__ __forceinline__ uint64_t pack_key(float cost, uint32_t id) {
    return ((uint64_t)__float_as_uint(cost) << 32) | (uint64_t)id;
}

__device__ __forceinline__ float key_cost(uint64_t k) { return __uint_as_float((uint32_t)(k >> 32)); }

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// first device error wins; TREE_FULL only replaces OK
__device__ __forceinline__ void set_status(kpx_device_header* h, int code) {
    atomicCAS(&h->status, (int)KPX_OK, code);
}

// One rollout held by one lane: started from a slot, advanced one
// integration step at a time.  The propagate kernel interleaves many of
// these per warp (a lane takes a new slot as soon as its rollout ends); the
// append kernel replays a winner through the same advance(), which makes the
// re-materialised end state and cost bit-identical.
template <int DYN, int INTEG>
struct LaneRollout {
    static constexpr int n = Dims<DYN>::n, m = Dims<DYN>::m;
    float x[n], u[m];
    Stepper<DYN, INTEG> st;
    float len, cost0;
    int K, k, node;

    __device__ __forceinline__ void start(const DevParams& P, const int32_t* va, int lam, uint32_t iter,
                                          int64_t slot) {
        // slot < 2^32 (create checks tree_cap + slot capacity): 32-bit division
        const uint32_t su = (uint32_t)slot;
        const int j = (int)(su / (uint32_t)lam);
        const int s = (int)(su - (uint32_t)j * (uint32_t)lam);
        node = va[j];
#pragma unroll
        for (int d = 0; d < n; ++d) x[d] = P.x[(int64_t)d * P.N + node];
        cost0 = key_cost(P.key[node]);
        sample_control<m>(P, iter, (uint32_t)node, (uint32_t)s, u, K);
        st.init(P, x, u);
        len = 0.0f;
        k = 0;
    }

    // One integration step and its path length, no checks.  PL and ISO: 1 or
    // 0 when the caller has read the cost kind (path length or not) and the
    // inertia flag already, so that its loop tests neither; -1 to read them.
    template <int PL = -1, int ISO = -1>
    __device__ __forceinline__ void integrate(const DevParams& P) {
        const float p0 = x[0], p1 = x[1], p2 = x[2];
        st.template advance<ISO>(P, x, u);
        ++k;
        if (PL == 1 || (PL < 0 && P.cost_kind == KPX_COST_PATH_LENGTH)) {
            const float dx = x[0] - p0, dy = x[1] - p1, dz = x[2] - p2;
            len = len + sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
        }
    }

    // One step; returns whether the new point is valid (bounds, and the
    // obstacles when OBST).
    template <bool OBST, bool SMEM = false, bool SYM = false, int PL = -1, int ISO = -1>
    __device__ __forceinline__ bool advance_in(const DevParams& P, const GridView& G, uint32_t& tests) {
        integrate<PL, ISO>(P);
        if (!bounds_ok<n, SYM>(P, x)) return false;
        if (OBST && P.n_obs > 0) {  // hits_obstacle_in() for a point in the workspace
            int e0, e1;
            cell_range_ws<SMEM>(P, G, x[0], x[1], x[2], e0, e1);
            if (walk_cell<SMEM>(G, x[0], x[1], x[2], e0, e1, tests)) return false;
        }
        return true;
    }

    template <bool OBST>
    __device__ __forceinline__ bool advance(const DevParams& P, uint32_t& tests) {
        return advance_in<OBST, false>(P, GridView{P.cell_start, P.cell_box}, tests);
    }

    __device__ __forceinline__ float cost(const DevParams& P) const { return cost0 + edge_cost<m>(P, K, len, u); }
};

}  // namespace kpx
