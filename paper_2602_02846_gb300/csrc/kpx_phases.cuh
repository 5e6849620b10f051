// kpx_phases.cuh -- one unit of work of each phase of a Kino-PAX+ iteration,
// shared by the single-problem kernels (kpx_kernels.cu) and the batched
// kernels (kpx_batch.cu).  A unit is a 32-slot chunk (propagate), a region
// (mark), a tile of the winner bitmask (scan), a winner (append) or a tile of
// node ids (prune); the kernels only decide which units a block or warp takes.
#pragma once

#include "kpx_device.cuh"

namespace kpx {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr uint32_t LOOKBACK_POLL_LIMIT = 1u << 20;

// ---------------------------------------------------------------------------
// Block-wide exclusive scan of one value per thread.
// ---------------------------------------------------------------------------
template <int THREADS, typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T& total, T* s_warp) {
    constexpr int NW = THREADS / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < NW ? s_warp[lane] : (T)0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(FULL, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NW) s_warp[lane] = w;
    }
    __syncthreads();
    const T excl = x - v + (warp > 0 ? s_warp[warp - 1] : (T)0);
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
__device__ __forceinline__ uint32_t lookback(uint64_t* tiles, uint32_t tile, uint32_t agg, uint32_t epoch,
                                             kpx_device_header* H) {
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

// goal_key = min(goal_key, k) by compare-and-swap.  The header may live in
// another CTA's shared memory (the fused kernel); there a 64-bit atomicMin
// through a generic address lost updates under contention on GB300, while
// 64-bit compare-and-swap held.  Each failed swap means another thread
// lowered the key, so the loop ends; it is bounded all the same.
__device__ __forceinline__ void goal_key_min(kpx_device_header* H, uint64_t k) {
    unsigned long long* p = reinterpret_cast<unsigned long long*>(&H->goal_key);
    unsigned long long old = *reinterpret_cast<volatile unsigned long long*>(p);
    for (int it = 0; k < old; ++it) {
        if (it == (1 << 20)) {
            set_status(H, KPX_E_INTERNAL);
            H->err_info[0] = 0x20000u;
            break;
        }
        const unsigned long long prev = atomicCAS(p, old, (unsigned long long)k);
        if (prev == old) break;
        old = prev;
    }
}

__device__ __forceinline__ const int32_t* va_current(const DevParams& P, const kpx_device_header* H) {
    return H->va_sel ? P.va1 : P.va0;
}

// the buffer that receives the next V_A (the compaction's output)
__device__ __forceinline__ int32_t* va_following(const DevParams& P, const kpx_device_header* H) {
    return H->va_sel ? P.va0 : P.va1;
}

// ---------------------------------------------------------------------------
// begin: branching factor (fixed, or floor(t_e/|V_A|)), slot count, tickets.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int begin_lambda(const DevParams& P, int count_A) {
    return P.lambda_fixed > 0 ? P.lambda_fixed : (count_A > 0 ? max(1, P.N / count_A) : 0);
}

// one thread per problem
__device__ __forceinline__ bool problem_runs(const DevParams& P, const kpx_device_header* H) {
    return H->status == KPX_OK && P.iter_limit >= 0 && (P.iter_limit == 0 || H->iter < P.iter_limit);
}

__device__ __forceinline__ void begin_counters(const DevParams& P, kpx_device_header* H, bool allowed = true) {
    if (!allowed || !problem_runs(P, H)) {
        // a stopped (tree full) or idle planner is a no-op: its header stays
        // as its last iteration left it
        H->active = 0;
        H->n_slots = 0;
        return;
    }
    const int lam = begin_lambda(P, H->count_A);
    H->active = 1;
    H->lambda = lam;
    H->n_slots = (int64_t)H->count_A * lam;
    H->prop_ticket = 0ull;
    H->win_ticket = 0u;
    H->prune_ticket = 0u;
    H->n_win = 0;
    H->n_kept = 0;
    H->count_A_next = 0;
    H->last_valid = 0ull;
    H->n_active = H->n_inactive = H->n_terminal = 0;
    H->epoch = (H->epoch + 1) & 0x3FFFFFFF;
    if (H->epoch == 0) H->epoch = 1;
    if (H->t_start_ns == 0ull) H->t_start_ns = globaltimer_ns();
}

// The capacity rule can only trigger when the largest possible number of
// winners (one per region, at most one per slot) overflows the tree.
// Computed from counters that begin_counters does not write.
__device__ __forceinline__ bool begin_needs_snapshot(const DevParams& P, const kpx_device_header* H,
                                                     bool allowed = true) {
    if (!allowed || !problem_runs(P, H)) return false;
    const int64_t n_slots = (int64_t)H->count_A * begin_lambda(P, H->count_A);
    const int64_t max_new = n_slots < P.R ? n_slots : P.R;
    return (int64_t)H->n_nodes + max_new > P.N;
}

// ---------------------------------------------------------------------------
// propagate order: the slots of each aligned ORDER_CHUNK-slot chunk sorted by
// an order key, their step count K or the quadcopter's predicted step count
// (one warp per chunk, a bitonic network over the warp's registers and
// shuffles).  Only the lane that computes a slot changes, not the slot's
// result.
// ---------------------------------------------------------------------------
// Ascending sort of the 128 values v[e] of all lanes, element i = lane + 32 e.
__device__ __forceinline__ void warp_sort128(uint32_t (&v)[4]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 128; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {  // partner in this lane's registers: e ^ (j / 32)
                const int je = j >> 5;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if ((e & je) == 0) {
                        const int f = e | je;
                        const bool asc = ((lane + 32 * e) & k) == 0;
                        const uint32_t lo = min(v[e], v[f]), hi = max(v[e], v[f]);
                        v[e] = asc ? lo : hi;
                        v[f] = asc ? hi : lo;
                    }
                }
            } else {  // partner in lane ^ j, same register
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const uint32_t o = __shfl_xor_sync(FULL, v[e], j);
                    const bool lower = (lane & j) == 0;
                    const bool asc = ((lane + 32 * e) & k) == 0;  // bit k is the pair's common bit
                    v[e] = (lower == asc) ? min(v[e], o) : max(v[e], o);
                }
            }
        }
    }
}

// The sort key of a quadcopter slot: K, or fewer steps when the velocity,
// extrapolated from the parent's at the start's acceleration (the sampled
// thrust along the parent's body z axis, gravity), leaves its bounds first.
// Most quadcopter rollouts end on a velocity bound, so this predicts a
// rollout's length better than K alone; only the order in which the slots
// are rolled out depends on it, not any result.  The parent's part (its
// body z axis and velocity) is computed once per parent.
struct QuadOrderParent {
    float zx, zy, zz, v[3];
};

__device__ __forceinline__ QuadOrderParent quad_order_parent(const DevParams& P, int node) {
    const int64_t N = P.N;
    float sph, cph, sth, cth, sps, cps;
    __sincosf(P.x[3 * N + node], &sph, &cph);
    __sincosf(P.x[4 * N + node], &sth, &cth);
    fast_sincos(P.x[5 * N + node], sps, cps);
    QuadOrderParent q;
    q.zx = fmaf(cps, sth * cph, sps * sph);
    q.zy = fmaf(sps, sth * cph, -(cps * sph));
    q.zz = cth * cph;
#pragma unroll
    for (int i = 0; i < 3; ++i) q.v[i] = P.x[(6 + i) * N + node];
    return q;
}

__device__ __forceinline__ uint32_t quad_order_key(const DevParams& P, const QuadOrderParent& q, int node,
                                                   uint32_t iter, uint32_t s) {
    // the thrust (word 0 of block 0) and K (word 0 of block 1), as sample_control() draws them
    const uint2 key = make_uint2(P.seed_lo, P.seed_hi);
    const uint32_t w0 = philox4x32_10(make_uint4(iter, (uint32_t)node, s, 0u), key).x;
    const uint32_t w1 = philox4x32_10(make_uint4(iter, (uint32_t)node, s, 1u), key).x;
    const float f = __fmul_rn(__uint2float_rn(w0 >> 8), 0x1p-24f);
    const float thrust = __fadd_rn(P.u_lo[0], __fmul_rn(__fsub_rn(P.u_hi[0], P.u_lo[0]), f));
    const int K = steps_from_word(P, w1);
    const float ah = thrust * P.inv_mass * P.h;  // velocity change per step along the body z axis
    const float dv[3] = {ah * q.zx, ah * q.zy, fmaf(ah, q.zz, -P.param[1] * P.h)};
    float n = (float)K;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        if (dv[i] > 0.0f) n = fminf(n, __fdividef(P.x_hi[6 + i] - q.v[i], dv[i]));
        if (dv[i] < 0.0f) n = fminf(n, __fdividef(P.x_lo[6 + i] - q.v[i], dv[i]));
    }
    return (uint32_t)fmaxf(n, 0.0f);  // <= K < 2^16
}

// Chunk c of this iteration's slots: order[c * 128 + p] = offset in the
// chunk of the slot with the p-th smallest (key, offset), the key being K
// (the quadcopter's: K or its predicted step count, quad_order_key).  Slots past n_slots
// take keys above every live slot's, so they sort to the chunk's end.
template <int M>
__device__ __forceinline__ void order_chunk(const DevParams& P, const int32_t* va, int lam, uint32_t iter,
                                            int64_t n_slots, int64_t c) {
    static_assert(ORDER_CHUNK == 128, "one warp sorts 4 slots per lane");
    const int lane = threadIdx.x & 31;
    uint32_t v[4];
    int j_parent = -1;  // the parent whose part of the quadcopter key qp holds
    QuadOrderParent qp;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const uint32_t off = (uint32_t)(lane + 32 * e);
        const int64_t slot = c * ORDER_CHUNK + off;
        if (slot < n_slots) {
            const uint32_t su = (uint32_t)slot;  // < 2^32, as in LaneRollout::start
            const int j = (int)(su / (uint32_t)lam);
            const int s = (int)(su - (uint32_t)j * (uint32_t)lam);
            uint32_t key;
            if constexpr (M == 4) {
                if (j != j_parent) {
                    qp = quad_order_parent(P, va[j]);
                    j_parent = j;
                }
                key = quad_order_key(P, qp, va[j], iter, (uint32_t)s);
            } else {
                key = (uint32_t)sample_steps<M>(P, iter, (uint32_t)va[j], (uint32_t)s);
            }
            v[e] = (key << 7) | off;  // key < 2^16
        } else {
            v[e] = 0xFFFFFF80u | off;
        }
    }
    warp_sort128(v);
#pragma unroll
    for (int e = 0; e < 4; ++e) P.slot_order[c * ORDER_CHUNK + lane + 32 * e] = (uint8_t)(v[e] & 127u);
}

// ---------------------------------------------------------------------------
// propagate (Alg. 2): 32 consecutive slots, one per lane.  Slot = rank j of
// the parent in V_A times lambda plus sample s.
// ---------------------------------------------------------------------------
// One slot's rollout: the candidate's validity, region, cost and packed
// key, with the region's atomicMin done.  Kept by the caller (the fused
// kernel appends a winner straight from it).
template <int DYN, int INTEG>
struct Candidate {
    LaneRollout<DYN, INTEG> R;
    bool ok;
    int r;
    float c;
    uint64_t key;
};

// The steps of a started rollout until its K-th or its first invalid point;
// returns whether every point was valid.
template <bool OBST, bool SMEM, bool SYM, int PL = -1, int ISO = -1, int DYN, int INTEG>
__device__ __forceinline__ bool rollout_steps(const DevParams& P, const GridView& G, LaneRollout<DYN, INTEG>& R,
                                              uint32_t& steps, uint32_t& tests) {
    bool ok = true;
    while (ok && R.k < R.K) {
        ++steps;
        ok = R.template advance_in<OBST, SMEM, SYM, PL, ISO>(P, G, tests);
    }
    return ok;
}

// G: where the obstacle grid is read (SMEM: a shared-memory copy)
// SYM: the state bounds are symmetric (bounds_ok's one-comparison form)
template <int DYN, int INTEG, bool SMEM = false, bool SYM = false>
__device__ __forceinline__ void roll_candidate(const DevParams& P, const GridView& G, int lam, uint32_t iter,
                                               const int32_t* va, bool early, int64_t slot, Candidate<DYN, INTEG>& C,
                                               uint32_t& steps, uint32_t& tests) {
    constexpr int n = Dims<DYN>::n;
    C.R.start(P, va, lam, iter, slot);
    bool ok = true;
    if (early) {  // one loop per mode: no per-step test of the flag
        while (ok && C.R.k < C.R.K) {
            ++steps;
            ok = C.R.template advance_in<false, SMEM, SYM>(P, G, tests);
        }
    } else if (DYN == KPX_QUAD12 && INTEG == KPX_RK4) {  // the cost kind and inertia flag read once
        const bool pl = P.cost_kind == KPX_COST_PATH_LENGTH;
        if (P.iso_inertia) {
            if (pl)
                ok = rollout_steps<true, SMEM, SYM, 1, 1>(P, G, C.R, steps, tests);
            else
                ok = rollout_steps<true, SMEM, SYM, 0, 1>(P, G, C.R, steps, tests);
        } else {
            if (pl)
                ok = rollout_steps<true, SMEM, SYM, 1, 0>(P, G, C.R, steps, tests);
            else
                ok = rollout_steps<true, SMEM, SYM, 0, 0>(P, G, C.R, steps, tests);
        }
    } else {
        ok = rollout_steps<true, SMEM, SYM>(P, G, C.R, steps, tests);
    }
    C.r = -1;
    C.c = 0.0f;
    C.key = KEY_INF;
    if (ok) {
        C.r = region_of<n>(P, C.R.x);
        C.c = C.R.cost(P);
        C.key = pack_key(C.c, (uint32_t)P.N + (uint32_t)slot);
        if (early) {
            // collision-after-cost: only a possible winner is checked against obstacles
            ok = C.key < __ldcg(&P.region_key[C.r]);
            if (ok) {
                float x0[n];
#pragma unroll
                for (int d = 0; d < n; ++d) x0[d] = P.x[(int64_t)d * P.N + C.R.node];
                ok = obstacle_pass<DYN, INTEG, SMEM>(P, G, x0, C.R.u, C.R.K, steps, tests);
            }
        }
        if (ok && C.key < __ldcg(&P.region_key[C.r]))
            atomicMin((unsigned long long*)&P.region_key[C.r], (unsigned long long)C.key);
    }
    C.ok = ok;
}

// roll_candidate() with early reject off, for one lane whose warp waits on
// its longest rollout (the fused kernel): step k+1 is integrated before step
// k's point is checked, so that the integration and the check, which both
// depend only on step k's state, overlap instead of the check's verdict
// gating the next integration.  The bounds test does not short-circuit the
// obstacle walk (whose box count is then dropped for an out-of-bounds point).
// One integration beyond the last step is thus discarded; the end state,
// path length, verdict and the step and box-test counts equal
// roll_candidate()'s (K >= 1).
template <int DYN, int INTEG, bool SMEM>
__device__ __forceinline__ void roll_candidate_ahead(const DevParams& P, const GridView& G, int lam, uint32_t iter,
                                                     const int32_t* va, int64_t slot, Candidate<DYN, INTEG>& C,
                                                     uint32_t& steps, uint32_t& tests) {
    constexpr int n = Dims<DYN>::n;
    C.R.start(P, va, lam, iter, slot);
    C.R.integrate(P);  // step 1
    bool ok = true;
    for (int k = 1;; ++k) {
        float xc[n];  // step k's point
#pragma unroll
        for (int d = 0; d < n; ++d) xc[d] = C.R.x[d];
        const float len_c = C.R.len;
        C.R.integrate(P);  // step k+1 (discarded after the last step)
        ++steps;
        const bool inb = bounds_ok(P, xc);
        uint32_t t = 0;
        const bool hit = hits_obstacle_in<SMEM>(P, G, xc[0], xc[1], xc[2], t);
        tests += inb ? t : 0u;
        if (!inb || hit) {
            ok = false;
            break;
        }
        if (k == C.R.K) {
#pragma unroll
            for (int d = 0; d < n; ++d) C.R.x[d] = xc[d];
            C.R.len = len_c;
            C.R.k = k;
            break;
        }
    }
    C.r = -1;
    C.c = 0.0f;
    C.key = KEY_INF;
    if (ok) {
        C.r = region_of<n>(P, C.R.x);
        C.c = C.R.cost(P);
        C.key = pack_key(C.c, (uint32_t)P.N + (uint32_t)slot);
        if (C.key < __ldcg(&P.region_key[C.r]))
            atomicMin((unsigned long long*)&P.region_key[C.r], (unsigned long long)C.key);
    }
    C.ok = ok;
}

// Lanes per rollout for n_slots rollouts on `threads` threads: the largest
// power of two up to 32 with n_slots * g <= threads (1 when the slots fill
// more than half of the threads).
__device__ __forceinline__ int coop_lanes(int64_t n_slots, int64_t threads) {
    int g = 1;
    while (g < 32 && n_slots * (int64_t)(2 * g) <= threads) g *= 2;
    return g;
}

// Rollouts shared by the g lanes of aligned groups of a warp (g a power of
// two, 2..32; called by all 32 lanes, `live` false for a group without a
// slot): every lane of a group integrates the group's rollout, and after
// each block of g steps lane gl = lane % g checks the block's step gl
// (bounds, then obstacles).  The block's first failing step ends the
// rollout.  A rollout of K steps thus waits on ceil(K / g) rounds of checks
// instead of K.  The blocks are warp-uniform (the warp runs until its
// longest rollout ends, the groups predicated) so that the warp never splits
// into groups that would then issue one after another.  Verdict, end state,
// cost and the step and box-test counts equal those of roll_candidate()
// with early reject off; lane 0 of a group keeps the candidate and the
// counts, the other lanes neither.
template <int DYN, int INTEG, bool SMEM>
__device__ __forceinline__ void roll_candidate_coop(const DevParams& P, const GridView& G, int lam, uint32_t iter,
                                                    const int32_t* va, bool live, int64_t slot, int g,
                                                    Candidate<DYN, INTEG>& C, uint32_t& steps, uint32_t& tests) {
    constexpr int n = Dims<DYN>::n;
    const int lane = threadIdx.x & 31;
    const int gl = lane & (g - 1);
    const int base = lane - gl;
    const uint32_t gbits = g == 32 ? FULL : (1u << g) - 1u;
    C.R.K = 0;
    C.R.k = 0;
    if (live) C.R.start(P, va, lam, iter, slot);
    bool run = live;  // the group's rollout has not ended
    bool ok = live;
    uint32_t n_steps = 0, n_tests = 0;
    const int k_warp = (int)__reduce_max_sync(FULL, (uint32_t)(live ? C.R.K : 0));
    for (int k0 = 0; k0 < k_warp; k0 += g) {  // warp-uniform
        const int nb = run ? min(g, C.R.K - k0) : 0;  // uniform within the group
        float mx[n];
#pragma unroll
        for (int d = 0; d < n; ++d) mx[d] = 0.0f;
        for (int i = 0; i < nb; ++i) {
            C.R.integrate(P);
#pragma unroll
            for (int d = 0; d < n; ++d) mx[d] = i == gl ? C.R.x[d] : mx[d];
        }
        bool bad = false;
        uint32_t t = 0;
        if (gl < nb) bad = !bounds_ok(P, mx) || hits_obstacle_in<SMEM>(P, G, mx[0], mx[1], mx[2], t);
        const uint32_t b = (__ballot_sync(FULL, bad) >> base) & gbits;
        const int f = b ? __ffs(b) - 1 : nb;  // the block's first failing step
        uint32_t tt = gl <= f ? t : 0u;
        for (int o = g >> 1; o > 0; o >>= 1) tt += __shfl_xor_sync(FULL, tt, o);
        if (run) {
            n_tests += tt;
            if (f < nb) {
                n_steps += (uint32_t)(f + 1);
                ok = false;
                run = false;
            } else {
                n_steps += (uint32_t)nb;
                run = C.R.k < C.R.K;
            }
        }
    }
    C.r = -1;
    C.c = 0.0f;
    C.key = KEY_INF;
    ok = ok && gl == 0;
    if (gl == 0) {
        steps += n_steps;
        tests += n_tests;
    }
    if (ok) {
        C.r = region_of<n>(P, C.R.x);
        C.c = C.R.cost(P);
        C.key = pack_key(C.c, (uint32_t)P.N + (uint32_t)slot);
        if (C.key < __ldcg(&P.region_key[C.r]))
            atomicMin((unsigned long long*)&P.region_key[C.r], (unsigned long long)C.key);
    }
    C.ok = ok;
}

// Lane l of a warp takes position chunk * 32 + l of the slot sequence: the
// slot itself, or with `order` (written by the begin kernel) the slot at that
// position of its ORDER_CHUNK-slot chunk sorted by the order key (K, or the
// quadcopter's predicted step count), so that a warp's lanes run similar
// step counts.  The slots past n_slots sort last in the final chunk, so a
// position below n_slots always names a live slot.
template <int DYN, int INTEG, bool SYM = false>
__device__ __forceinline__ void propagate_chunk(const DevParams& P, int64_t n_slots, int lam, uint32_t iter,
                                                const int32_t* va, bool early, int64_t chunk,
                                                const kpx_debug_records& rec, int rec_on, uint32_t& steps,
                                                uint32_t& tests, uint32_t& n_valid, const uint8_t* order = nullptr) {
    constexpr int n = Dims<DYN>::n, m = Dims<DYN>::m;
    const int64_t pos = chunk * 32 + (threadIdx.x & 31);
    if (pos >= n_slots) return;
    const int64_t slot = order ? (pos & ~(int64_t)(ORDER_CHUNK - 1)) + order[pos] : pos;
    Candidate<DYN, INTEG> C;
    roll_candidate<DYN, INTEG, false, SYM>(P, GridView{P.cell_start, P.cell_box}, lam, iter, va, early, slot, C, steps,
                                           tests);
    n_valid += C.ok ? 1u : 0u;
    if (rec_on && slot < rec.capacity) {
        rec.valid[slot] = C.ok ? 1 : 0;
        rec.region[slot] = C.ok ? C.r : -1;
        rec.key[slot] = C.ok ? C.key : KEY_INF;
        rec.K[slot] = C.R.K;
#pragma unroll
        for (int d = 0; d < n; ++d) rec.x[(int64_t)d * rec.capacity + slot] = C.R.x[d];
#pragma unroll
        for (int d = 0; d < m; ++d) rec.u[(int64_t)d * rec.capacity + slot] = C.R.u[d];
    }
}

// The propagate's work units: 32 slots each.  With the slots of each
// 128-slot chunk sorted by the order key (ordered) they are handed out longest quarter
// first: unit q is quarter 3 - q / n128 of 128-slot chunk q % n128, so that
// a launch ends on the short rollouts (a longest-first schedule); units past
// n_slots are empty.  Otherwise unit q is slots [32 q, 32 q + 32).
__device__ __forceinline__ int64_t propagate_units(int64_t n_slots, bool ordered) {
    return ordered ? (n_slots + ORDER_CHUNK - 1) / ORDER_CHUNK * (ORDER_CHUNK / 32) : (n_slots + 31) / 32;
}

__device__ __forceinline__ int64_t propagate_unit_chunk(int64_t q, int64_t n_slots, bool ordered) {
    if (!ordered) return q;
    const int64_t n128 = (n_slots + ORDER_CHUNK - 1) / ORDER_CHUNK;
    return (q % n128) * (ORDER_CHUNK / 32) + (ORDER_CHUNK / 32 - 1 - q / n128);
}

// warp-wide: add the lane counters to the problem's header (one atomic each)
__device__ __forceinline__ void flush_propagate_counters(kpx_device_header* H, uint32_t& steps, uint32_t& tests,
                                                         uint32_t& n_valid) {
    unsigned long long st = steps, te = tests, nv = n_valid;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        st += __shfl_down_sync(FULL, st, o);
        te += __shfl_down_sync(FULL, te, o);
        nv += __shfl_down_sync(FULL, nv, o);
    }
    if ((threadIdx.x & 31) == 0 && st) {
        atomicAdd((unsigned long long*)&H->total_steps, st);
        atomicAdd((unsigned long long*)&H->total_box_tests, te);
        if (nv) atomicAdd((unsigned long long*)&H->last_valid, nv);
    }
    steps = tests = n_valid = 0;
}

// ---------------------------------------------------------------------------
// mark: a region whose key carries a candidate id (>= N) names the slot of
// the winner of that region (the V_U filter: "cost(x) = cost(R_i)").
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mark_region(const DevParams& P, int r) {
    const uint64_t k = P.region_key[r];
    if (k == KEY_INF) return;
    const uint32_t id = (uint32_t)k;
    if (id < (uint32_t)P.N) return;
    const uint32_t slot = id - (uint32_t)P.N;
    if ((int64_t)slot >= P.slot_cap) {  // a stale candidate id: cannot happen in a consistent state
        set_status(P.hdr, KPX_E_INTERNAL);
        return;
    }
    atomicOr(&P.win_mask[slot >> 5], 1u << (slot & 31));
    P.slot_region[slot] = r;
}

// ---------------------------------------------------------------------------
// scan (block-wide): one tile of the winner bitmask; ranks in ascending slot
// order -> win_slot[rank]; clears the words.  The problem's last tile writes
// its winner count.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void scan_tile(const DevParams& P, kpx_device_header* H, uint32_t tile, int64_t n_tiles,
                                          int64_t live_words, uint32_t* s_warp, uint32_t& s_prefix) {
    const int64_t w0 = (int64_t)tile * WIN_TILE_WORDS + (int64_t)threadIdx.x * WIN_WORDS_PER_THREAD;
    static_assert(WIN_WORDS_PER_THREAD == 8, "two 16-byte loads a thread");
    uint32_t w[WIN_WORDS_PER_THREAD];
    uint32_t cnt = 0;
    if (w0 + WIN_WORDS_PER_THREAD <= live_words) {  // w0 is a multiple of 8 words: 32-byte aligned
        const uint4 a = *reinterpret_cast<const uint4*>(P.win_mask + w0);
        const uint4 b = *reinterpret_cast<const uint4*>(P.win_mask + w0 + 4);
        w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
        w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
    } else {
#pragma unroll
        for (int i = 0; i < WIN_WORDS_PER_THREAD; ++i) w[i] = (w0 + i < live_words) ? P.win_mask[w0 + i] : 0u;
    }
#pragma unroll
    for (int i = 0; i < WIN_WORDS_PER_THREAD; ++i) cnt += __popc(w[i]);
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
    __syncthreads();
}

// ---------------------------------------------------------------------------
// append (UpdateTree, Alg. 4) of winner w: its rollout is re-materialised
// from (seed, iteration, node, sample) with the propagate arithmetic, written
// to T at n_old + w, and its region key rewritten with the new id; the
// previous owner of the region becomes dominated.  Winners beyond the
// capacity restore their region from the snapshot.  Goal nodes lower the
// solution key.
// ---------------------------------------------------------------------------
// The row writes of winner w (rank in slot order) with rollout Rw, cost c,
// region r, whose key node is `old` (region_owner[r], read by the caller;
// -1 for none): appended at n_old + w when w < kept, else the capacity rule
// restores the region's key.
// set_mirror: where the fused kernel keeps tile 0's staged set bytes (CTA
// 0's shared memory), which receive the previous owner's new byte too; null
// elsewhere.
template <int DYN, int INTEG>
__device__ __forceinline__ void append_row(const DevParams& P, kpx_device_header* H, int w, int kept, int n_old,
                                           const LaneRollout<DYN, INTEG>& Rw, float c, int r, int old,
                                           uint8_t* set_mirror = nullptr) {
    constexpr int n = Dims<DYN>::n, m = Dims<DYN>::m;
    if (w < kept) {
        const int id = n_old + w;
#pragma unroll
        for (int d = 0; d < n; ++d) P.x[(int64_t)d * P.N + id] = Rw.x[d];
#pragma unroll
        for (int d = 0; d < m; ++d) P.u[(int64_t)d * P.N + id] = Rw.u[d];
        P.K[id] = (uint16_t)Rw.K;
        P.parent[id] = Rw.node;
        const uint64_t k = pack_key(c, (uint32_t)id);
        P.key[id] = k;
        P.region[id] = r;
        P.set[id] = SET_A;
        P.icount[id] = 0;
        P.region_key[r] = k;
        // the previous owner of r loses its region (one winner per region,
        // so this thread is the only writer of that node's set byte)
        if (old >= 0) {
            const uint8_t nb = (uint8_t)(P.set[old] | SET_DOM);
            P.set[old] = nb;
            if (set_mirror && old < PRUNE_TILE) set_mirror[old] = nb;
        }
        P.region_owner[r] = id;
        if (in_goal(P, Rw.x[0], Rw.x[1], Rw.x[2])) goal_key_min(H, k);
    } else {
        P.region_key[r] = P.region_snap[r];
    }
}

template <int DYN, int INTEG>
__device__ __forceinline__ void append_winner(const DevParams& P, kpx_device_header* H, int w, int kept, int n_old,
                                              int lam, uint32_t iter, const int32_t* va) {
    constexpr int n = Dims<DYN>::n;
    const int slot = P.win_slot[w];
    LaneRollout<DYN, INTEG> Rw;
    Rw.start(P, va, lam, iter, (int64_t)slot);
    uint32_t te_unused = 0;
    for (int k = 0; k < Rw.K; ++k) Rw.template advance<false>(P, te_unused);
    const float c = Rw.cost(P);
    const int r = region_of<n>(P, Rw.x);
    const uint64_t cand_key = pack_key(c, (uint32_t)P.N + (uint32_t)slot);
    if (P.region_key[r] != cand_key) {
        set_status(H, KPX_E_INTERNAL);
        H->err_info[1] = (uint32_t)slot;
        return;
    }
    append_row<DYN, INTEG>(P, H, w, kept, n_old, Rw, c, r, P.region_owner[r]);
}

// UpdateTree split in two for the planner's graphs, which run the halves on
// two branches after the winner scan:
// - append_meta writes everything that needs no end state: the row's parent,
//   control, step count, key, region and sets, the region's key and owner,
//   the previous owner's dominated mark, and the capacity rule's restores.
//   The winner's region comes from mark (slot_region), its cost from the
//   region's key.  PruneNodes needs only these.
// - stage_winner re-materialises a kept winner's rollout from Philox (the
//   propagate kernel's arithmetic, bit for bit), writes its end state into
//   the tree row and lowers the solution key for a goal node.  It checks the
//   rollout's region and cost against the region's key, whose cost bits the
//   other half leaves as they are.
template <int DYN, int INTEG>
__device__ __forceinline__ void append_meta(const DevParams& P, kpx_device_header* H, int w, int kept, int n_old,
                                            int lam, uint32_t iter, const int32_t* va) {
    constexpr int m = Dims<DYN>::m;
    const int slot = P.win_slot[w];
    const int r = P.slot_region[slot];
    // the mapped region must hold this slot's key (a stale entry would not)
    if (r < 0 || r >= P.R || (uint32_t)P.region_key[r] != (uint32_t)P.N + (uint32_t)slot) {
        set_status(H, KPX_E_INTERNAL);
        H->err_info[1] = (uint32_t)slot;
        return;
    }
    if (w >= kept) {  // dropped by the capacity rule: the region's key before this iteration
        P.region_key[r] = P.region_snap[r];
        return;
    }
    const uint32_t su = (uint32_t)slot;  // < 2^32, as in LaneRollout::start
    const int j = (int)(su / (uint32_t)lam);
    const int s = (int)(su - (uint32_t)j * (uint32_t)lam);
    const int node = va[j];
    float u[m];
    int K;
    sample_control<m>(P, iter, (uint32_t)node, (uint32_t)s, u, K);
    const int id = n_old + w;
#pragma unroll
    for (int d = 0; d < m; ++d) P.u[(int64_t)d * P.N + id] = u[d];
    P.K[id] = (uint16_t)K;
    P.parent[id] = node;
    const uint64_t k = pack_key(key_cost(P.region_key[r]), (uint32_t)id);
    P.key[id] = k;
    P.region[id] = r;
    P.set[id] = SET_A;
    P.icount[id] = 0;
    const int old = P.region_owner[r];
    P.region_key[r] = k;
    if (old >= 0) P.set[old] = (uint8_t)(P.set[old] | SET_DOM);  // one winner per region: the only writer
    P.region_owner[r] = id;
}

template <int DYN, int INTEG>
__device__ __forceinline__ void stage_winner(const DevParams& P, kpx_device_header* H, int w, int n_old, int lam,
                                             uint32_t iter, const int32_t* va) {
    constexpr int n = Dims<DYN>::n;
    const int slot = P.win_slot[w];
    const int r = P.slot_region[slot];
    if (r < 0 || r >= P.R) return;  // append_meta reports it
    LaneRollout<DYN, INTEG> Rw;
    Rw.start(P, va, lam, iter, (int64_t)slot);
    uint32_t te_unused = 0;
    for (int k = 0; k < Rw.K; ++k) Rw.template advance<false>(P, te_unused);
    const float c = Rw.cost(P);
    if ((uint32_t)(P.region_key[r] >> 32) != __float_as_uint(c) || region_of<n>(P, Rw.x) != r) {
        set_status(H, KPX_E_INTERNAL);
        H->err_info[1] = (uint32_t)slot;
        return;
    }
    const int id = n_old + w;
#pragma unroll
    for (int d = 0; d < n; ++d) P.x[(int64_t)d * P.N + id] = Rw.x[d];
    if (in_goal(P, Rw.x[0], Rw.x[1], Rw.x[2])) goal_key_min(H, pack_key(c, (uint32_t)id));
}

// Rules 1-3 of Alg. 3 (literal order, first match wins) for a node that is
// not terminal: set byte sb, inactivity count ic and set nst in/out.
// Returns whether a rule decided the node; false leaves it to rule 4.
// key(i) >= key(region(i)) always, with equality only for the region's
// owner: "best" is "not dominated".
__device__ __forceinline__ bool prune_rules_123(uint8_t sb, int i_max, int& ic, int& nst) {
    const bool dominated = (sb & SET_DOM) != 0;
    const bool best = !dominated;
    if (best && nst == SET_I) {  // rule 1: region best while inactive
        ++ic;
        if (ic > i_max) {
            nst = SET_A;
            return true;
        }
    }
    if (ic > i_max && best) return true;  // rule 2
    if (dominated) {                      // rule 3: dominated
        nst = SET_T;
        return true;
    }
    return false;
}

// ---------------------------------------------------------------------------
// prune (block-wide): PruneNodes (Alg. 3) over the tile's nodes below n_old,
// literal rule order, then the tile's part of the compaction of V_A (Alg. 5)
// over [0, total): nodes appended this iteration are active by Alg. 4.
// epoch and va_next are the iteration's (the header's epoch, and the V_A
// buffer that va_sel does not select), read by the caller.
// ---------------------------------------------------------------------------
// The tile's parent ids, set bytes and inactivity counts below n_old, read in
// one pass: ancestor walks that stay inside the tile read shared memory
// (parents precede children), and a node's own bytes come from here.
__device__ __forceinline__ void stage_tile(const DevParams& P, int tile0, int n_old, int32_t* s_parent,
                                           uint8_t* s_set, uint8_t* s_icount) {
    for (int k = threadIdx.x; k < PRUNE_TILE; k += PRUNE_THREADS) {
        const int i = tile0 + k;
        const bool in = i < n_old;
        s_parent[k] = in ? P.parent[i] : -1;
        s_set[k] = in ? P.set[i] : 0;
        s_icount[k] = in ? P.icount[i] : 0;
    }
}

// staged: the caller staged the tile already (the fused kernel stages tile 0
// before the append phase, whose dominated marks it then receives directly).
// One pass, one node per thread in each of PRUNE_PER_THREAD rounds (node
// tile0 + round * PRUNE_THREADS + thread): rules 1-3, then rule 4's walk
// for the nodes they leave undecided, so that a small tree's nodes spread
// over the block's warps.  The compaction keeps id order, which runs round
// by round, then warp by warp, then lane by lane: each warp ballots its
// active nodes of each round, and one warp scans the (round, warp) counts,
// PRUNE_ROUND_WARPS of them, in that order (s_counts) and takes the tile's
// look-back.
constexpr int PRUNE_ROUND_WARPS = PRUNE_PER_THREAD * (PRUNE_THREADS / 32);
static_assert(PRUNE_ROUND_WARPS <= 32, "one warp scans the (round, warp) counts");

__device__ __forceinline__ void prune_tile(const DevParams& P, kpx_device_header* H, uint32_t tile, int n_tiles,
                                           int n_old, int total, uint32_t epoch, int32_t* va_next,
                                           int32_t* s_parent, uint8_t* s_set, uint8_t* s_icount,
                                           uint32_t* s_counts, uint32_t& s_prefix, int& cA, int& cI, int& cT,
                                           bool staged = false) {
    const int i_max = P.i_max;
    const int tile0 = (int)tile * PRUNE_TILE;
    if (!staged) stage_tile(P, tile0, n_old, s_parent, s_set, s_icount);
    __syncthreads();
    uint32_t fields = 0;  // bit q: this thread's node of round q stays in V_A
#pragma unroll
    for (int q = 0; q < PRUNE_PER_THREAD; ++q) {
        const int k = threadIdx.x + q * PRUNE_THREADS;
        const int i = tile0 + k;
        if (i >= total) continue;
        if (i >= n_old) {  // appended this iteration: in V_A
            fields |= 1u << q;
            ++cA;
            continue;
        }
        const uint8_t sb = s_set[k];
        if ((sb & SET_MASK) == SET_T) {  // V_T is permanent
            ++cT;
            continue;
        }
        int ic = s_icount[k];
        const int ic0 = ic;
        int nst = sb & SET_MASK;
        bool anc = (sb & SET_ANC) != 0;
        if (!prune_rules_123(sb, i_max, ic, nst)) {
            // rule 4: whether a strict ancestor is dominated.  The ANC flag
            // memoises a positive answer (it is monotone); clean[] memoises a
            // negative one for this prune only: a walk that finds no dominated
            // strict ancestor stamps its node with the epoch, and a later walk
            // stops at a stamped ancestor that is not dominated itself.  The
            // dominated bits do not change during prune, so a stamp seen in
            // this epoch stays true; a stamp not yet visible only means a
            // longer walk.
            if (!anc) {
                int p = s_parent[k];
                while (p >= tile0) {  // inside the tile: shared memory (a stale set byte
                    // only lacks a monotone flag, which the walk re-derives)
                    const uint8_t sp = s_set[p - tile0];
                    if (sp & (SET_DOM | SET_ANC)) {
                        anc = true;
                        break;
                    }
                    p = s_parent[p - tile0];
                }
                for (; !anc && p >= 0; p = P.parent[p]) {
                    const uint8_t sp = *(volatile const uint8_t*)&P.set[p];
                    if (sp & (SET_DOM | SET_ANC)) {
                        anc = true;
                    } else if (*(volatile const uint32_t*)&P.clean[p] == epoch) {
                        break;  // p's strict ancestors are clean, and p is not dominated
                    }
                }
                if (!anc) P.clean[i] = epoch;
            }
            if (anc) nst = SET_I;
        }
        const uint8_t nb = (uint8_t)(nst | (anc ? SET_ANC : 0) | (sb & SET_DOM));
        if (nb != sb) P.set[i] = nb;
        if (ic != ic0) P.icount[i] = (uint8_t)ic;
        if (nst == SET_A) {
            fields |= 1u << q;
            ++cA;
        } else if (nst == SET_I) {
            ++cI;
        } else {
            ++cT;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t ball[PRUNE_PER_THREAD];
#pragma unroll
    for (int q = 0; q < PRUNE_PER_THREAD; ++q) {
        ball[q] = __ballot_sync(FULL, (fields >> q) & 1u);
        if (lane == 0) s_counts[q * (PRUNE_THREADS / 32) + warp] = (uint32_t)__popc(ball[q]);
    }
    __syncthreads();
    if (warp == 0) {
        // exclusive prefix of the (round, warp) counts, then the tile's
        // place among the tiles (look-back)
        const uint32_t v = lane < PRUNE_ROUND_WARPS ? s_counts[lane] : 0u;
        uint32_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        const uint32_t agg = __shfl_sync(FULL, x, 31);
        __syncwarp();
        if (lane < PRUNE_ROUND_WARPS) s_counts[lane] = x - v;
        if (lane == 0) {
            s_prefix = lookback(P.prune_tiles, tile, agg, epoch, H);
            if ((int)tile == n_tiles - 1) H->count_A_next = (int32_t)(s_prefix + agg);
        }
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;  // lanes below this one
#pragma unroll
    for (int q = 0; q < PRUNE_PER_THREAD; ++q) {
        if ((fields >> q) & 1u) {
            // at most one active node per region, so pos < min(N, R) = va_cap
            const uint32_t pos =
                s_prefix + s_counts[q * (PRUNE_THREADS / 32) + warp] + (uint32_t)__popc(ball[q] & lt);
            if (pos < (uint32_t)P.va_cap)
                va_next[pos] = tile0 + (int)threadIdx.x + q * PRUNE_THREADS;
            else
                set_status(H, KPX_E_INTERNAL);
        }
    }
    __syncthreads();
}

// warp-wide: add the set sizes to the problem's header
__device__ __forceinline__ void flush_prune_counters(kpx_device_header* H, int& cA, int& cI, int& cT) {
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
    cA = cI = cT = 0;
}

// ---------------------------------------------------------------------------
// end (one thread per problem): commit the counters of the iteration.
// stamp_last: take the end-of-iteration time now; the fused kernel passes
// false and stamps it once when its launch ends (its header is private to the
// launch until then), keeping the global timer off the iteration's chain.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void end_counters(const DevParams& P, kpx_device_header* H, bool stamp_last = true) {
    if (!H->active) return;
    H->n_nodes += H->n_kept;
    H->count_A = H->count_A_next;
    H->va_sel ^= 1;
    H->last_candidates = (uint64_t)H->n_slots;
    H->last_winners = (uint64_t)H->n_kept;
    H->total_candidates += (uint64_t)H->n_slots;
    H->total_valid += H->last_valid;
    H->total_winners += (uint64_t)H->n_kept;
    uint64_t now = 0ull;
    if (H->goal_key != KEY_INF && H->first_solution_iter < 0) {
        now = globaltimer_ns();
        H->first_solution_iter = H->iter;
        H->t_first_solution_ns = now;
    }
    H->iter += 1;
    if (stamp_last) H->t_last_ns = now ? now : globaltimer_ns();
}

}  // namespace kpx
