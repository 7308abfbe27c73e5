// env_split.cuh -- the 4-robot Navigation rollout (binary32, scripted position control or policy
// actions, no traces) with the per-step outputs taken off the dynamics' dependency chain.
//
// Same method and results (up to rounding) as run_env_small<true>.  Each block holds 8 warps on
// one SM: warps 0-3 run the dynamics of their envs (nominal velocity, barrier QP, unicycle step,
// auto-reset), warps 4-7 the outputs of the same envs (collision and arena flags, the team
// reward, the observations, the reward and done streams).  Warp w and warp w + 4 form a pair on
// the same SM sub-partition, with the same team layout (lane i of team k holds robot i of the
// k-th env of the pair).  Every step the dynamics warp publishes, per robot, the projected point
// after the Euler step (the flags' and the reward's point), its reward term, and the pose and
// goal after any auto-reset (the observation's) into a shared-memory slot, then goes on with the
// next step; the output warp reads the slot and writes the step's outputs while the dynamics
// warp computes the next step.  The two warps hand the slot over with a pair of named barriers
// (bar.arrive by the writer, bar.sync by the reader, one pair per warp pair), so the handover
// costs the dynamics warp one barrier arrival and two shared stores per step.
//
// The output warp also takes two state-independent pieces of the step off the dynamics warp:
//  * the action noise: it draws the Philox words of a launch's first three steps before the
//    dynamics warp starts (one extra handover arrival releases it), then after reading step s
//    those of step s + 3, into a ring of four steps that the dynamics warp reads;
//  * the auto-reset sample: after reading the step that began an episode (or before reading the
//    launch's first step, for its first episode) it samples the next episode's initial poses,
//    goals and levels into its own team record, which the dynamics warp reads at the episode's
//    end.
// Apart from the first three steps' noise, which the extra arrival orders, both are read at least
// three steps after they were written; the barriers of the two steps in between order the
// accesses (the writer has passed them only after finishing the write, the reader waits on
// them), and a slot is rewritten only after the reader has arrived past its read.  An episode
// end closer than that (episodes shorter than three steps, or the first one ending before step
// 2) is sampled by the dynamics warp itself.
//
// Both warps of a pair run the same T steps over the same envs, every lane of both warps
// executing every barrier (teams without an env skip only the work), so every barrier completes.
#pragma once
#include "env_small.cuh"

namespace rl {

// One step's handover from a dynamics warp to its output warp.
struct SplitSlot {
    float4 r[8][4][2];  // [team][robot]: (npx, npy, reward term, gy), (x, y, th, gx)
    int done[8];        // [team]: the episode ended (the pose above is the new episode's)
    uint2 noise[4][8][4];  // [step & 3][team][robot]: Philox words of the robot's action noise
};

// Noise words of robot i for step t of episode ep (robots 2m and 2m + 1 share the block of
// pair m, as in the other 4-robot kernels).
__device__ __forceinline__ uint2 split_noise(uint64_t seed, int e, int ep, int i, int t) {
    const Words4 w = draw(seed, e, ep, kNoise, i >> 1, (uint32_t)t);
    return (i & 1) ? make_uint2(w.w[2], w.w[3]) : make_uint2(w.w[0], w.w[1]);
}

// Named barriers of warp pair p (ids 1..8; id 0 is left to __syncthreads).  Both warps count:
// 64 threads.
__device__ __forceinline__ void split_arrive(int id) {
    asm volatile("barrier.cta.arrive %0, 64;" ::"r"(id) : "memory");
}
__device__ __forceinline__ void split_wait(int id) {
    asm volatile("barrier.cta.sync %0, 64;" ::"r"(id) : "memory");
}
__device__ __forceinline__ int split_full_id(int p) { return 1 + 2 * p; }
__device__ __forceinline__ int split_empty_id(int p) { return 2 + 2 * p; }

// The dynamics warp of a pair: live teams step their env T times; every lane executes the
// handover of every step.
static __device__ __forceinline__ void split_dynamics(const LaunchArgs<float>& A, const Team<4>& tm,
                                                      TeamSmem<float, 4>& S,
                                                      const TeamSmem<float, 4>& So, SplitSlot& slot,
                                                      int p, int tiw, int e, unsigned wm) {
    const StepConsts<float>& k = A.k;
    const bool live = e >= 0;
    const int N = live ? A.s.nrob[e] : 0;
    const int i = tm.lane;
    const bool own = i < N;
    const int off = live ? A.s.off[e] : 0;
    const int row = off + (own ? i : 0);

    QPConsts<float> qc;
    qc.gamma = k.gamma; qc.r2 = k.r2; qc.kg = k.kg; qc.half_r = k.half_r;
    qc.xmin = k.xmin; qc.xmax = k.xmax; qc.ymin = k.ymin; qc.ymax = k.ymax;
    qc.h_flag = k.h_flag;
    qc.max_iter = k.max_iter;
    qc.tol_abs = 2e-7f; qc.tol_rel = 1e-6f; qc.eps_dep = 1e-5f; qc.tol_lam = 1e-6f;

    float x = 0.f, y = 0.f, th = 0.f, gx = 0.f, gy = 0.f, gth = 0.f;
    int lv = 0, t = 0, ep = 0;
    if (live) {
        x = A.s.x[row]; y = A.s.y[row]; th = A.s.th[row];
        gx = A.s.gx[row]; gy = A.s.gy[row]; gth = A.s.gth[row];
        lv = A.s.level[row];
        t = A.s.t[e];
        ep = A.s.ep[e];
    }
    float sn, cs;
    __sincosf(th, &sn, &cs);
    int c_succ = 0, c_act = 0, c_flag = 0, c_inf = 0, c_ep = 0, c_it = 0;
    int last_reset = -1;  // the step of the last episode end (-1: none in this launch)
    // the output warp has drawn the noise of the launch's first three steps
    if (A.T > 0) split_wait(split_empty_id(p));

    for (int step = 0; step < A.T; ++step) {
        float npx = 0.f, npy = 0.f, dterm = 0.f;
        int done = 0;
        if (live) {
            // ---- projected point and nominal SI velocity: the policy's action, or go to goal,
            // cap, noise; then the cap
            const float px = x + k.l * cs, py = y + k.l * sn;
            float ux, uy;
            if (A.io.actions) {
                ux = A.io.actions[2 * row];
                uy = A.io.actions[2 * row + 1];
                screen_action(A.io.status, ux, uy);
            } else {
                ux = k.k_si * (gx - px);
                uy = k.k_si * (gy - py);
                cap_fast(ux, uy, k.vmax);
                // the noise words, drawn ahead by the output warp
                const uint2 w = slot.noise[step & 3][tiw][i];
                {
                    const float ex = __fmul_rn(__fsub_rn(unit24(w.x), 0.5f), k.noise_scale);
                    const float ey = __fmul_rn(__fsub_rn(unit24(w.y), 0.5f), k.noise_scale);
                    ux += k.noise_on ? ex : 0.f;
                    uy += k.noise_on ? ey : 0.f;
                }
            }
            cap_fast(ux, uy, k.vmax);
            const float dold = fast_norm(px - gx, py - gy);

            // ---- the barrier QP: every lane solves the team's QP in registers (at most six
            // active rows); a larger active set, and the binary64 re-solve of a flagged QP, by
            // the warp's live lanes (or by the team when it is alone in its warp)
            float usx, usy;
            QPResult res = small_filter_all(tm, S, N, px, py, ux, uy, qc, usx, usy, wm != 0u);
            bool rare64 = false;
            if (wm != 0u) {
                const unsigned rare = __ballot_sync(
                    wm, i == 0 && (res.status == 3 || (k.resolve_f64 && res.flag)));
                if (rare) {
                    const int nl = __popc(wm);
                    const int wl = threadIdx.x & 31;
                    unsigned need = __ballot_sync(wm, i == 0 && res.status == 3);
                    while (need) {
                        const int src = __ffs(need) - 1;  // the team's first lane
                        need &= need - 1u;
                        const int Ns = __shfl_sync(wm, N, src);
                        float Px[4], Py[4], U0[8];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            Px[j] = __shfl_sync(wm, px, src + j);
                            Py[j] = __shfl_sync(wm, py, src + j);
                            U0[2 * j] = __shfl_sync(wm, ux, src + j);
                            U0[2 * j + 1] = __shfl_sync(wm, uy, src + j);
                        }
                        float um;
                        const QPResult r = warp_qp<float>(wm, nl, Ns, Px, Py, U0, qc, um);
                        const float ox = __shfl_sync(wm, um, 2 * (wl & 3));
                        const float oy = __shfl_sync(wm, um, 2 * (wl & 3) + 1);
                        if (tm.base == src) {
                            res = r;
                            usx = own ? ox : 0.f;
                            usy = own ? oy : 0.f;
                        }
                    }
                    need = __ballot_sync(wm, i == 0 && k.resolve_f64 && res.flag);
                    if (need) {
                        float sf, cf;
                        sincosf(th, &sf, &cf);
                        const double pxd = (double)x + (double)k.l * (double)cf;
                        const double pyd = (double)y + (double)k.l * (double)sf;
                        QPConsts<double> dc;
                        dc.gamma = (double)k.gamma; dc.r2 = (double)k.r2; dc.kg = (double)k.kg;
                        dc.half_r = (double)k.half_r; dc.xmin = (double)k.xmin;
                        dc.xmax = (double)k.xmax; dc.ymin = (double)k.ymin; dc.ymax = (double)k.ymax;
                        dc.h_flag = (double)k.h_flag;
                        dc.max_iter = 8 * 4 + 16;
                        dc.tol_abs = 1e-12; dc.tol_rel = 1e-12; dc.eps_dep = 1e-12;
                        dc.tol_lam = 1e-10;
                        while (need) {
                            const int src = __ffs(need) - 1;
                            need &= need - 1u;
                            const int Ns = __shfl_sync(wm, N, src);
                            double Px[4], Py[4], U0[8];
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                Px[j] = __shfl_sync(wm, pxd, src + j);
                                Py[j] = __shfl_sync(wm, pyd, src + j);
                                U0[2 * j] = (double)__shfl_sync(wm, ux, src + j);
                                U0[2 * j + 1] = (double)__shfl_sync(wm, uy, src + j);
                            }
                            double um;
                            const QPResult r64 = warp_qp<double>(wm, nl, Ns, Px, Py, U0, dc, um);
                            const double ox = __shfl_sync(wm, um, 2 * (wl & 3));
                            const double oy = __shfl_sync(wm, um, 2 * (wl & 3) + 1);
                            if (tm.base == src) {
                                res.status = r64.status;
                                res.q = r64.q;
                                res.iters += r64.iters;
                                usx = own ? (float)ox : 0.f;
                                usy = own ? (float)oy : 0.f;
                                rare64 = true;
                            }
                        }
                    }
                }
            } else if (k.resolve_f64 && res.flag) {
                const QPResult r64 = small_resolve_f64(tm, S, k, N, x, y, th, ux, uy);
                res.status = r64.status;
                res.q = r64.q;
                res.iters += r64.iters;
                usx = own ? (float)S.qp.d.ux[i] : 0.f;
                usy = own ? (float)S.qp.d.uy[i] : 0.f;
                tm.sync();
                rare64 = true;
            }
            const int qflags = ((res.q > 0 || res.status != 0) ? 1 : 0) | (rare64 ? 2 : 0);

            // ---- SI -> unicycle, wheel clip, Euler step
            float v = cs * usx + sn * usy;
            float om = (cs * usy - sn * usx) * k.inv_l;
            const float wr = fminf(fmaxf(v + k.half_track * om, -k.vmax), k.vmax);
            const float wl = fminf(fmaxf(v - k.half_track * om, -k.vmax), k.vmax);
            v = 0.5f * (wr + wl);
            om = (wr - wl) * k.inv_track;
            x += k.dt * v * cs;
            y += k.dt * v * sn;
            th = wrap_pi_f(th + k.dt * om);
            __sincosf(th, &sn, &cs);
            npx = x + k.l * cs;
            npy = y + k.l * sn;
            dterm = own ? dold - fast_norm(npx - gx, npy - gy) : 0.f;
            if (k.waypoint && own) {
                const float ex = npx - gx, ey = npy - gy;
                if (ex * ex + ey * ey < k.goal_eps2) {
                    const float3 g = waypoint_goal(A.sc, A.seed, e, ep, i, t + 1);
                    gx = g.x;
                    gy = g.y;
                    gth = g.z;
                    ++c_succ;
                }
            }
            c_act += qflags & 1;
            c_flag += (qflags >> 1) & 1;
            c_inf += (res.status == 1) ? 1 : 0;
            c_it += res.iters;

            // ---- episode end and auto-reset
            t += 1;
            if (t >= k.episode_len) {
                done = 1;
                c_ep += 1;
                ep += 1;
                t = 0;
                if (step >= last_reset + 3) {
                    // sampled ahead by the output warp
                    if (own) {
                        x = So.fx[i]; y = So.fy[i]; th = So.fth[i];
                        gx = So.sx[i]; gy = So.sy[i]; gth = So.sth[i]; lv = So.slevel[i];
                    }
                } else {
                    small_reset(tm, S, A, e, ep, N);
                    if (own) {
                        x = S.fx[i]; y = S.fy[i]; th = S.fth[i];
                        gx = S.sx[i]; gy = S.sy[i]; gth = S.sth[i]; lv = S.slevel[i];
                    }
                    tm.sync();
                }
                last_reset = step;
                __sincosf(th, &sn, &cs);
            }
        }
        // ---- hand the step over to the output warp (slot free once it has read the last one)
        __syncwarp();
        if (step > 0) split_wait(split_empty_id(p));
        slot.r[tiw][i][0] = make_float4(npx, npy, dterm, gy);
        slot.r[tiw][i][1] = make_float4(x, y, th, gx);
        if (i == 0) slot.done[tiw] = done;
        split_arrive(split_full_id(p));
    }
    if (A.T > 0) split_wait(split_empty_id(p));
    if (live) {
        if (own) {
            A.s.x[row] = x; A.s.y[row] = y; A.s.th[row] = th;
            A.s.gx[row] = gx; A.s.gy[row] = gy; A.s.gth[row] = gth; A.s.level[row] = lv;
        }
        c_succ = tm.sum(c_succ);  // arrivals were counted per robot
        if (i == 0) {
            A.s.t[e] = t;
            A.s.ep[e] = ep;
            // collisions and arena exits are the output warp's; reductions without a returned
            // value, so that the warp does not wait for the old counts before it exits
            int32_t* cn = A.s.counters + e * kNCount;
            atomicAdd(cn + 2, c_succ); atomicAdd(cn + 3, c_act); atomicAdd(cn + 4, c_flag);
            atomicAdd(cn + 5, c_inf); atomicAdd(cn + 6, c_ep); atomicAdd(cn + 7, c_it);
        }
    }
}

// The output warp of a pair: per step, the flags, the team reward, the observations and the
// reward and done streams of the pair's envs, from the dynamics warp's slot.
static __device__ __forceinline__ void split_outputs(const LaunchArgs<float>& A, const Team<4>& tm,
                                                     TeamSmem<float, 4>& So, SplitSlot& slot,
                                                     int p, int tiw, int e) {
    const StepConsts<float>& k = A.k;
    const bool live = e >= 0;
    const int N = live ? A.s.nrob[e] : 0;
    const int i = tm.lane;
    const bool own = i < N;
    const int row = (live ? A.s.off[e] : 0) + (own ? i : 0);
    int jo[3];  // the others in index order: observation slot s holds robot s + (s >= i)
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) jo[sl] = sl + (sl >= i ? 1 : 0);
    int c_col = 0, c_oob = 0;
    float ret_acc = 0.f;
    const int od = A.io.obs_dim;
    const bool scripted = A.io.actions == nullptr;
    // the env's episode clock (the dynamics warp's, advanced by the published done flags)
    int t = live ? A.s.t[e] : 0, ep = live ? A.s.ep[e] : 0;
    // the noise of the launch's first three steps, then one handover arrival that releases the
    // dynamics warp (every later arrival follows the reading of a step's slot)
    if (live && scripted) {
        int ts = t, es = ep;
        for (int s0 = 0; s0 < 3 && s0 < A.T; ++s0) {
            if (own) slot.noise[s0][tiw][i] = split_noise(A.seed, e, es, i, ts);
            if (++ts >= k.episode_len) { ts = 0; ++es; }
        }
    }
    if (A.T > 0) split_arrive(split_empty_id(p));
    // the launch's first episode end (read at step 2 or later: short launches skip it)
    if (live && A.T > 2) small_reset(tm, So, A, e, ep + 1, N);

    for (int step = 0; step < A.T; ++step) {
        __syncwarp();
        split_wait(split_full_id(p));
        float4 a[4], b[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            a[r] = slot.r[tiw][r][0];
            b[r] = slot.r[tiw][r][1];
        }
        const int done = slot.done[tiw];
        split_arrive(split_empty_id(p));
        if (!live) continue;
        // the episode clock at the start of step + 1, then the noise of step + 3 and, after an
        // episode end, the next episode's initial state
        if (done) { t = 0; ++ep; } else { ++t; }
        if (scripted && step + 3 < A.T) {
            int t3 = t + 1, ep3 = ep;
            if (t3 >= k.episode_len) { t3 = 0; ++ep3; }
            if (++t3 >= k.episode_len) { t3 = 0; ++ep3; }
            if (own) slot.noise[(step + 3) & 3][tiw][i] = split_noise(A.seed, e, ep3, i, t3);
        }
        if (done && step + 3 < A.T) small_reset(tm, So, A, e, ep + 1, N);
        // collisions and arena exits of the projected points after the Euler step (before any
        // reset), the team reward
        int col = 0, oob = 0;
        float rew = 0.f;
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (r < N) {
                rew += a[r].z;
                oob += (a[r].x < k.xmin || a[r].x > k.xmax || a[r].y < k.ymin || a[r].y > k.ymax)
                           ? 1 : 0;
            }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = r + 1; q < 4; ++q) {
                const float dx = a[r].x - a[q].x, dy = a[r].y - a[q].y;
                col += (q < N && dx * dx + dy * dy < k.r2) ? 1 : 0;
            }
        rew -= k.c_col * (float)col;
        c_col += col;
        c_oob += oob;
        ret_acc += rew;
        // ---- observation of the own robot: [x, y, th, gx, gy], then the others in index order
        // relative to it (after any reset: the new episode's)
        if (A.io.obs && own) {
            const float4 me = pick4(b, i);
            const float myg = pick4(a, i).w;
            float rel[9];
#pragma unroll
            for (int sl = 0; sl < 3; ++sl) {
                const float4 o = pick4(b, jo[sl]);
                const bool lv2 = jo[sl] < N;
                rel[3 * sl] = lv2 ? o.x - me.x : 0.f;
                rel[3 * sl + 1] = lv2 ? o.y - me.y : 0.f;
                rel[3 * sl + 2] = lv2 ? wrap_pi_f(o.z - me.z) : 0.f;
            }
            float* ob = A.io.obs + (long long)step * A.io.obs_step + (long long)row * od;
            if (od == 14) {
                float2* o2 = reinterpret_cast<float2*>(ob);
                o2[0] = make_float2(me.x, me.y);
                o2[1] = make_float2(me.z, me.w);
                o2[2] = make_float2(myg, rel[0]);
                o2[3] = make_float2(rel[1], rel[2]);
                o2[4] = make_float2(rel[3], rel[4]);
                o2[5] = make_float2(rel[5], rel[6]);
                o2[6] = make_float2(rel[7], rel[8]);
            } else {
                const float head[5] = {me.x, me.y, me.z, me.w, myg};
#pragma unroll
                for (int s2 = 0; s2 < 5; ++s2)
                    if (s2 < od) ob[s2] = head[s2];
#pragma unroll
                for (int s2 = 0; s2 < 9; ++s2)
                    if (5 + s2 < od) ob[5 + s2] = rel[s2];
                for (int s2 = 14; s2 < od; ++s2) ob[s2] = 0.f;
            }
        }
        if (i == 0) {
            if (A.io.reward) A.io.reward[(long long)step * A.io.E + e] = rew;
            if (A.io.done) A.io.done[(long long)step * A.io.E + e] = (uint8_t)done;
        }
    }
    if (live && i == 0) {
        if (A.io.ret) A.io.ret[e] = ret_acc;
        int32_t* cn = A.s.counters + e * kNCount;
        atomicAdd(cn, c_col);
        atomicAdd(cn + 1, c_oob);
    }
}

// One block of 8 warps per SM: warps 0-3 dynamics, warps 4-7 outputs, the envs of the launch
// divided evenly over the grid's 4 * gridDim.x dynamics warps (at most 8 per warp: the launcher
// guarantees it).
__global__ void __launch_bounds__(256, 1) env_kernel_split(LaunchArgs<float> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ SplitSlot slots[4];
    const Team<4> tm;
    const int warp_in_block = threadIdx.x >> 5;
    const int p = warp_in_block & 3;
    const int tiw = (threadIdx.x & 31) >> 2;
    const long long n = A.n_list;
    const int dw = blockIdx.x * 4 + p, dws = gridDim.x * 4;
    const int lo = (int)(dw * n / dws), hi = (int)((dw + 1) * n / dws);
    const int idx = lo + tiw;
    const int e = idx < hi ? (A.env_list ? A.env_list[idx] : A.env_begin + idx) : -1;
    if (warp_in_block < 4) {
        TeamSmem<float, 4>* S = reinterpret_cast<TeamSmem<float, 4>*>(smem_raw) + (threadIdx.x >> 2);
        const TeamSmem<float, 4>* So = S + 32;  // the partner output team's record
        const int nw = hi - lo;  // the warp's live teams, for the warp-wide rare QPs
        const unsigned wm = nw >= 8 ? 0xffffffffu : (nw >= 2 ? (1u << (4 * nw)) - 1u : 0u);
        split_dynamics(A, tm, *S, *So, slots[p], p, tiw, e, wm);
    } else {
        TeamSmem<float, 4>* So = reinterpret_cast<TeamSmem<float, 4>*>(smem_raw) + (threadIdx.x >> 2);
        split_outputs(A, tm, *So, slots[p], p, tiw, e);
    }
}

}  // namespace rl
