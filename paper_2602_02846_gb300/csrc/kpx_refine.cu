// kpx_refine.cu -- the C ABI of the trajectory refinement post-pass
// (include/kpx.h) and its re-validation kernel.
//
// Re-validation re-rolls each control sequence from its start state with the
// planner's own FP32 RK4 stepper.  This file has the planner's compile flags,
// so a trajectory the planner returned re-rolls to the same states bit for
// bit.  A sequence is valid when every state after a step satisfies the state
// bounds, lies in the workspace box and in no obstacle box, and the last
// position lies in the goal ball.  The edge costs are summed in FP64: FP64
// appears on the GPU only here.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "kpx_device.cuh"

namespace kpx {

namespace {

constexpr int VAL_WARPS = 4;  // trajectories per block

struct ValidateParams {
    int32_t count, max_segments, n_obs;
    const float* obs;
    const float* x0;
    const float* u;
    const int32_t* steps;
    const int32_t* n_seg;
    int32_t* valid;
    double* cost;
    float* x_end;
};

// one warp per trajectory: every lane integrates, the box tests are split
// across the lanes
__global__ void __launch_bounds__(VAL_WARPS * 32) k_refine_validate(DevParams P, ValidateParams V) {
    extern __shared__ float smem[];
    const int M = V.n_obs;
    for (int i = threadIdx.x; i < 6 * M; i += blockDim.x) smem[i] = V.obs[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t tr = (int64_t)blockIdx.x * VAL_WARPS + (threadIdx.x >> 5);
    if (tr >= V.count) return;
    const int S = V.n_seg[tr];
    float x[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) x[i] = V.x0[tr * 12 + i];
    bool ok = S >= 0 && S <= V.max_segments;
    // the edge costs of every segment, in FP64 from the FP32 controls:
    // K h (1 + w e(u)); they do not depend on the states
    double total = 0.0;
    const double mg = (double)P.param[0] * (double)P.param[1];
    const double tm = (double)P.param[5];
    for (int s = 0; ok && s < S; ++s) {
        const float* uv = V.u + (tr * V.max_segments + s) * 4;
        const double et = ((double)uv[0] - mg) / mg;
        const double e = et * et + ((double)uv[1] * uv[1] + (double)uv[2] * uv[2] + (double)uv[3] * uv[3]) / (tm * tm);
        total += (double)V.steps[tr * V.max_segments + s] * (double)P.h * (1.0 + (double)P.w_effort * e);
    }
    Stepper<KPX_QUAD12, KPX_RK4> st;
    for (int s = 0; ok && s < S; ++s) {
        const float4 uv = *reinterpret_cast<const float4*>(V.u + (tr * V.max_segments + s) * 4);
        const float u[4] = {uv.x, uv.y, uv.z, uv.w};
        const int K = V.steps[tr * V.max_segments + s];
        st.init(P, x, u);
        for (int k = 0; ok && k < K; ++k) {
            st.advance(P, x, u);
            bool hit = false;
            for (int b = lane; b < M; b += 32) {
                const float* o = smem + 6 * b;
                hit |= x[0] >= o[0] && x[0] <= o[3] && x[1] >= o[1] && x[1] <= o[4] && x[2] >= o[2] && x[2] <= o[5];
            }
            ok = bounds_ok<12>(P, x) && !__any_sync(0xFFFFFFFFu, hit);
        }
    }
    if (ok) ok = in_goal(P, x[0], x[1], x[2]);
    if (lane == 0) {
        V.valid[tr] = ok ? 1 : 0;
        V.cost[tr] = total;
    }
    if (V.x_end && lane < 12) {
#pragma unroll
        for (int i = 0; i < 12; ++i)
            if (lane == i) V.x_end[tr * 12 + i] = x[i];
    }
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

int n_checkpoints(int32_t max_total_steps) { return (max_total_steps + REFINE_CKPT_STEPS - 1) / REFINE_CKPT_STEPS + 1; }

bool quad_rk4(const kpx_dynamics* dyn) { return dyn && dyn->kind == KPX_QUAD12 && dyn->integ == KPX_RK4; }

bool aligned16(const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; }

// workspace: the box grid first, then the checkpoints
size_t grid_region() { return align256(REFINE_GRID_BYTES); }

}  // namespace
}  // namespace kpx

using namespace kpx;

extern "C" size_t kpx_refine_workspace_size(int32_t count, int32_t max_total_steps) {
    if (count < 0 || max_total_steps < 0) return 0;
    return grid_region() +
           align256((size_t)count * n_checkpoints(max_total_steps) * REFINE_CKPT_WORDS * sizeof(float));
}

extern "C" kpx_status kpx_refine_eval(const kpx_dynamics* dyn, const kpx_refine_cost* cost, const float* obstacles,
                                      int32_t n_obstacles, int32_t count, int32_t max_segments, const float* x0,
                                      const float* u, const int32_t* steps, const int32_t* n_segments,
                                      const int32_t* order, int32_t max_total_steps, float* cost_out, float* grad_u,
                                      void* workspace, size_t workspace_bytes, void* cuda_stream) {
    if (!quad_rk4(dyn) || !cost || count < 0 || max_segments < 1 || max_total_steps < 0 || n_obstacles < 0 ||
        n_obstacles > REFINE_MAX_OBS || (n_obstacles > 0 && !obstacles) || !x0 || !u || !steps || !n_segments ||
        !cost_out)
        return KPX_E_INVALID;
    if (!(cost->beta > 0.0f) || !std::isfinite(cost->beta)) return KPX_E_INVALID;
    if (!aligned16(u) || (grad_u && !aligned16(grad_u))) return KPX_E_INVALID;  // float4 rows
    if (count == 0) return KPX_OK;
    if (grad_u && (!workspace || workspace_bytes < kpx_refine_workspace_size(count, max_total_steps)))
        return KPX_E_NOMEM;
    if (workspace && reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return KPX_E_INVALID;
    RefineParams R;
    memset(&R, 0, sizeof(R));
    R.h = dyn->h;
    R.inv_mass = 1.0f / dyn->param[0];
    R.g = dyn->param[1];
    for (int i = 0; i < 3; ++i) {
        R.J[i] = dyn->param[2 + i];
        R.inv_J[i] = 1.0f / dyn->param[2 + i];
    }
    R.mg = dyn->param[0] * dyn->param[1];
    R.tau_max = dyn->param[5];
    R.w_obs = cost->w_obs;
    R.beta = cost->beta;
    R.inv_beta = 1.0f / cost->beta;
    R.margin = cost->margin;
    R.w_goal = cost->w_goal;
    for (int a = 0; a < 3; ++a) R.goal[a] = cost->goal[a];
    R.w_effort = cost->w_effort;
    R.count = count;
    R.max_segments = max_segments;
    R.n_obs = n_obstacles;
    R.max_total_steps = max_total_steps;
    R.n_ckpt = n_checkpoints(max_total_steps);
    R.obs = obstacles;
    R.x0 = x0;
    R.u = u;
    R.steps = steps;
    R.n_seg = n_segments;
    R.order = order;
    R.cost = cost_out;
    R.grad = grad_u;
    // the box grid when the workspace holds it (with a gradient it always does)
    if (workspace && workspace_bytes >= grid_region()) {
        char* w = reinterpret_cast<char*>(workspace);
        R.grid = reinterpret_cast<RefineGridHeader*>(w);
        R.grid_off = reinterpret_cast<int32_t*>(w + 256);
        R.grid_ids = reinterpret_cast<uint16_t*>(w + 256 + (size_t)(REFINE_GRID_CELLS + 1) * 4);
    }
    R.ckpt = workspace ? reinterpret_cast<float*>(reinterpret_cast<char*>(workspace) + grid_region()) : nullptr;
    return launch_refine_eval(R, reinterpret_cast<cudaStream_t>(cuda_stream)) == cudaSuccess ? KPX_OK : KPX_E_CUDA;
}

extern "C" kpx_status kpx_refine_validate(const kpx_dynamics* dyn, const kpx_workspace* ws, const float* obstacles,
                                          int32_t n_obstacles, const kpx_goal* goal, float w_effort, int32_t count,
                                          int32_t max_segments, const float* x0, const float* u,
                                          const int32_t* steps, const int32_t* n_segments, int32_t* valid,
                                          double* cost_out, float* x_end, void* cuda_stream) {
    if (!quad_rk4(dyn) || !ws || !goal || count < 0 || max_segments < 1 || n_obstacles < 0 ||
        n_obstacles > REFINE_MAX_OBS || (n_obstacles > 0 && !obstacles) || !x0 || !u || !steps || !n_segments ||
        !valid || !cost_out)
        return KPX_E_INVALID;
    if (!aligned16(u)) return KPX_E_INVALID;
    if (count == 0) return KPX_OK;
    DevParams P;
    memset(&P, 0, sizeof(P));
    fill_dynamics(P, dyn);
    for (int a = 0; a < 3; ++a) {
        P.ws_lo[a] = ws->lo[a];
        P.ws_hi[a] = ws->hi[a];
        P.goal_c[a] = goal->center[a];
    }
    set_position_box(P);
    P.goal_r2 = goal->radius * goal->radius;
    P.cost_kind = KPX_COST_EFFORT_DURATION;
    P.w_effort = w_effort;
    ValidateParams V;
    V.count = count;
    V.max_segments = max_segments;
    V.n_obs = n_obstacles;
    V.obs = obstacles;
    V.x0 = x0;
    V.u = u;
    V.steps = steps;
    V.n_seg = n_segments;
    V.valid = valid;
    V.cost = cost_out;
    V.x_end = x_end;
    const size_t smem = (size_t)6 * n_obstacles * sizeof(float);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_refine_validate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return KPX_E_CUDA;
    k_refine_validate<<<(count + VAL_WARPS - 1) / VAL_WARPS, VAL_WARPS * 32, smem,
                        reinterpret_cast<cudaStream_t>(cuda_stream)>>>(P, V);
    return cudaGetLastError() == cudaSuccess ? KPX_OK : KPX_E_CUDA;
}

extern "C" kpx_status kpx_refine_adam(const kpx_dynamics* dyn, int32_t count, int32_t max_segments,
                                      const int32_t* n_segments, float* u, const float* grad_u, float* m1, float* m2,
                                      int32_t t, float lr, void* cuda_stream) {
    if (!quad_rk4(dyn) || count < 0 || max_segments < 1 || !n_segments || !u || !grad_u || !m1 || !m2 || t < 1 ||
        !(lr >= 0.0f))
        return KPX_E_INVALID;
    if (count == 0) return KPX_OK;
    AdamParams A;
    A.count = count;
    A.max_segments = max_segments;
    A.n_seg = n_segments;
    A.u = u;
    A.grad = grad_u;
    A.m1 = m1;
    A.m2 = m2;
    for (int c = 0; c < 4; ++c) {
        A.lo[c] = dyn->u_lo[c];
        A.hi[c] = dyn->u_hi[c];
        if (!(A.hi[c] > A.lo[c])) return KPX_E_INVALID;
    }
    A.lr = lr;
    A.b1 = 0.9f;
    A.b2 = 0.999f;
    A.eps = 1e-8f;
    A.c1 = (float)(1.0 - std::pow(0.9, (double)t));
    A.c2 = (float)(1.0 - std::pow(0.999, (double)t));
    return launch_refine_adam(A, reinterpret_cast<cudaStream_t>(cuda_stream)) == cudaSuccess ? KPX_OK : KPX_E_CUDA;
}

extern "C" kpx_status kpx_refine_keep_best(int32_t count, int32_t max_segments, const float* u, const float* cost,
                                           float* u_best, float* cost_best, void* cuda_stream) {
    if (count < 0 || max_segments < 1 || !u || !cost || !u_best || !cost_best) return KPX_E_INVALID;
    return launch_refine_keep_best(count, max_segments, u, cost, u_best, cost_best,
                                   reinterpret_cast<cudaStream_t>(cuda_stream)) == cudaSuccess
               ? KPX_OK
               : KPX_E_CUDA;
}

extern "C" kpx_status kpx_refine_counters(const void* workspace, uint64_t counters[4], void* cuda_stream) {
    if (!workspace || !counters) return KPX_E_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    const RefineGridHeader* H = reinterpret_cast<const RefineGridHeader*>(workspace);
    unsigned long long t[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(t, H->tests, sizeof(t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return KPX_E_CUDA;
    for (int k = 0; k < 4; ++k) counters[k] = t[k];
    return KPX_OK;
}
