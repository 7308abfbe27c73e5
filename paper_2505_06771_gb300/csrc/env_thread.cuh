// env_thread.cuh -- one thread per environment for Navigation batches of at most 4 robots.
//
// Same method and results (up to rounding) as run_env in env_step.cuh.  A thread owns all four
// robots, the 22 barrier rows and the whole QP in registers: no step crosses lanes (a dependent
// warp shuffle costs about 48-66 cycles on GB300 against about 4.5 for a dependent FMA), and the
// four robots give the compiler independent work to interleave.  The price is four times the
// per-thread work and a quarter of the warps of the 4-lane team kernel; on 4096 envs that leaves
// most schedulers idle and the team kernel is faster, so this kernel is an autotuner candidate
// (lanes = 1) rather than the default.
//
// The QP of an env is thread_qp (qp_regs.cuh).  A flagged QP is re-solved in binary64 by the
// shared-memory solver of env_step.cuh, the thread acting as a one-lane team.
#pragma once
#include "qp_regs.cuh"

namespace rl {

// Reset sampler of one env of N <= 4 robots in one thread (binary32, one rounding per
// operation; the same draws as team_sample).
struct ThreadPose {
    float x[4], y[4], th[4], gx[4], gy[4], gth[4];
};

static __device__ __noinline__ ThreadPose thread_sample(const SamplerConsts sc, uint64_t seed,
                                                        int max_att, int e, int ep, int N) {
    ThreadPose P;
#pragma unroll
    for (int i = 0; i < 4; ++i) P.x[i] = P.y[i] = P.th[i] = P.gx[i] = P.gy[i] = P.gth[i] = 0.f;
    {
        const Words4 w = draw(seed, e, ep, kPos, 0, 0u);
        P.x[0] = __fadd_rn(sc.lox, __fmul_rn(unit24(w.w[0]), sc.wx));
        P.y[0] = __fadd_rn(sc.loy, __fmul_rn(unit24(w.w[1]), sc.wy));
        P.th[0] = __fadd_rn(-sc.pif, __fmul_rn(unit24(w.w[2]), sc.twopif));
    }
    int first = 1;
    if (N >= 2 && sc.near_on) {
        const Words4 w = draw(seed, e, ep, kNear, 0, 0u);
        if (unit24(w.w[0]) < sc.near_frac) {
            for (int a = 0; a < max_att; ++a) {
                const Words4 v = draw(seed, e, ep, kNear, 1, (uint32_t)a);
                const float d = __fadd_rn(sc.dmin, __fmul_rn(unit24(v.w[0]), sc.dspan));
                const float cx = __fsub_rn(__fmul_rn(2.0f, unit24(v.w[1])), 1.0f);
                const float cy = __fsub_rn(__fmul_rn(2.0f, unit24(v.w[2])), 1.0f);
                const float rr = __fadd_rn(__fmul_rn(cx, cx), __fmul_rn(cy, cy));
                if (rr < 0.0625f || rr > 1.0f) continue;
                const float nrm = __fsqrt_rn(rr);
                const float x1 = __fadd_rn(P.x[0], __fdiv_rn(__fmul_rn(d, cx), nrm));
                const float y1 = __fadd_rn(P.y[0], __fdiv_rn(__fmul_rn(d, cy), nrm));
                if (x1 < sc.lox || x1 > sc.hix || y1 < sc.loy || y1 > sc.hiy) continue;
                P.x[1] = x1;
                P.y[1] = y1;
                P.th[1] = P.th[0];
                first = 2;
                break;
            }
        }
    }
#pragma unroll
    for (int i = 1; i < 4; ++i) {
        if (i >= first && i < N) {
            float cx = 0.f, cy = 0.f, cth = 0.f;
            for (int a = 0; a < max_att; ++a) {
                const Words4 v = draw(seed, e, ep, kPos, i, (uint32_t)a);
                cx = __fadd_rn(sc.lox, __fmul_rn(unit24(v.w[0]), sc.wx));
                cy = __fadd_rn(sc.loy, __fmul_rn(unit24(v.w[1]), sc.wy));
                cth = __fadd_rn(-sc.pif, __fmul_rn(unit24(v.w[2]), sc.twopif));
                bool ok = true;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (j < i) {
                        const float dx = __fsub_rn(cx, P.x[j]), dy = __fsub_rn(cy, P.y[j]);
                        const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
                        if (d2 < sc.sep2) ok = false;
                    }
                }
                if (ok) break;  // after max_att attempts the last candidate is kept
            }
            P.x[i] = cx;
            P.y[i] = cy;
            P.th[i] = cth;
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (i < N) {
            const Words4 w = draw(seed, e, ep, kGoal, i, 0u);
            P.gx[i] = __fadd_rn(sc.lox, __fmul_rn(unit24(w.w[0]), sc.wx));
            P.gy[i] = __fadd_rn(sc.loy, __fmul_rn(unit24(w.w[1]), sc.wy));
            P.gth[i] = __fadd_rn(-sc.pif, __fmul_rn(unit24(w.w[2]), sc.twopif));
        }
    }
    return P;
}

__device__ __forceinline__ float twrap(float a) {
    a = (a > CUDART_PI_F) ? a - 2.f * CUDART_PI_F : a;
    return (a <= -CUDART_PI_F) ? a + 2.f * CUDART_PI_F : a;
}

__device__ __forceinline__ void tcap(float& ux, float& uy, float m) {
    const float s = fminf(1.f, m * rsqrtf(ux * ux + uy * uy));
    ux *= s;
    uy *= s;
}

__device__ __forceinline__ float tnorm(float a, float b) {
    const float n2 = a * a + b * b;
    return n2 > 0.f ? n2 * rsqrtf(n2) : 0.f;
}

// One Navigation env of N <= 4 robots for T scripted steps, all in this thread.  W: this
// thread's shared-memory workspace for the binary64 re-solve.
__device__ void run_env_thread(const LaunchArgs<float>& A, int e, QPWork<double, 4>& W) {
    const StepConsts<float>& k = A.k;
    const int off = A.s.off[e];
    const int N = A.s.nrob[e];
    QPConsts<float> qc;
    qc.gamma = k.gamma; qc.r2 = k.r2; qc.kg = k.kg; qc.half_r = k.half_r;
    qc.xmin = k.xmin; qc.xmax = k.xmax; qc.ymin = k.ymin; qc.ymax = k.ymax;
    qc.h_flag = k.h_flag;
    qc.max_iter = k.max_iter;
    qc.tol_abs = 2e-7f; qc.tol_rel = 1e-6f; qc.eps_dep = 1e-5f; qc.tol_lam = 1e-6f;

    float x[4], y[4], th[4], gx[4], gy[4], gth[4], cs[4], sn[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int row = off + (i < N ? i : 0);
        x[i] = A.s.x[row]; y[i] = A.s.y[row]; th[i] = A.s.th[row];
        gx[i] = A.s.gx[row]; gy[i] = A.s.gy[row]; gth[i] = A.s.gth[row];
        __sincosf(th[i], &sn[i], &cs[i]);
    }
    int t = A.s.t[e], ep = A.s.ep[e];
    int c_col = 0, c_oob = 0, c_succ = 0, c_act = 0, c_flag = 0, c_inf = 0, c_ep = 0, c_it = 0;
    float ret_acc = 0.f;
    const int od = A.io.obs_dim;

    for (int step = 0; step < A.T; ++step) {
        // ---- projected points, nominal SI velocities (go to goal, noise, cap)
        float px[4], py[4], U0[8], dold[4];
        const Words4 w01 = draw(A.seed, e, ep, kNoise, 0, (uint32_t)t);
        const Words4 w23 = draw(A.seed, e, ep, kNoise, 1, (uint32_t)t);
        const uint32_t nw[8] = {w01.w[0], w01.w[1], w01.w[2], w01.w[3],
                                w23.w[0], w23.w[1], w23.w[2], w23.w[3]};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            px[i] = x[i] + k.l * cs[i];
            py[i] = y[i] + k.l * sn[i];
            float ux = k.k_si * (gx[i] - px[i]), uy = k.k_si * (gy[i] - py[i]);
            tcap(ux, uy, k.vmax);
            const float ex = __fmul_rn(__fsub_rn(unit24(nw[2 * i]), 0.5f), k.noise_scale);
            const float ey = __fmul_rn(__fsub_rn(unit24(nw[2 * i + 1]), 0.5f), k.noise_scale);
            ux += k.noise_on ? ex : 0.f;
            uy += k.noise_on ? ey : 0.f;
            tcap(ux, uy, k.vmax);
            U0[2 * i] = ux;
            U0[2 * i + 1] = uy;
            dold[i] = tnorm(px[i] - gx[i], py[i] - gy[i]);
        }
        // ---- barrier QP
        float U[8];
        bool overflow;
        QPResult res = thread_qp<float, kThreadRows>(px, py, N, U0, qc, U, overflow);
        int qflags = (res.q > 0 || res.status != 0) ? 1 : 0;
        if (k.resolve_f64 && res.flag) {
            // binary64 re-solve with the shared-memory solver, this thread as a 1-lane team
            QPConsts<double> dc;
            dc.gamma = (double)k.gamma; dc.r2 = (double)k.r2; dc.kg = (double)k.kg;
            dc.half_r = (double)k.half_r; dc.xmin = (double)k.xmin; dc.xmax = (double)k.xmax;
            dc.ymin = (double)k.ymin; dc.ymax = (double)k.ymax; dc.h_flag = (double)k.h_flag;
            dc.max_iter = 8 * 4 + 16;
            dc.tol_abs = 1e-12; dc.tol_rel = 1e-12; dc.eps_dep = 1e-12; dc.tol_lam = 1e-10;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                double sd, cd;
                sincos((double)th[i], &sd, &cd);
                W.px[i] = (double)x[i] + (double)k.l * cd;
                W.py[i] = (double)y[i] + (double)k.l * sd;
                W.u0x[i] = W.ux[i] = (double)U0[2 * i];
                W.u0y[i] = W.uy[i] = (double)U0[2 * i + 1];
            }
            const Team<1> solo;
            const QPResult r64 = qp_solve<double, 1, 4>(solo, W, N, dc);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                U[2 * i] = (float)W.ux[i];
                U[2 * i + 1] = (float)W.uy[i];
            }
            res.status = r64.status;
            res.q = r64.q;
            res.iters += r64.iters;
            qflags |= 2;
        }
        // ---- SI -> unicycle, wheel clip, Euler step, new projected points
        float npx[4], npy[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float v = cs[i] * U[2 * i] + sn[i] * U[2 * i + 1];
            float om = (cs[i] * U[2 * i + 1] - sn[i] * U[2 * i]) * k.inv_l;
            const float wr = fminf(fmaxf(v + k.half_track * om, -k.vmax), k.vmax);
            const float wl = fminf(fmaxf(v - k.half_track * om, -k.vmax), k.vmax);
            v = 0.5f * (wr + wl);
            om = (wr - wl) * k.inv_track;
            x[i] += k.dt * v * cs[i];
            y[i] += k.dt * v * sn[i];
            th[i] = twrap(th[i] + k.dt * om);
            __sincosf(th[i], &sn[i], &cs[i]);
            npx[i] = x[i] + k.l * cs[i];
            npy[i] = y[i] + k.l * sn[i];
        }
        // ---- flags and reward
        int col = 0, oob = 0;
        float rew = 0.f;
#pragma unroll
        for (int r = 0; r < 6; ++r) {
            const int a = slot_a(r), b = slot_b(r);
            const float dx = npx[a] - npx[b], dy = npy[a] - npy[b];
            col += (b < N && dx * dx + dy * dy < k.r2) ? 1 : 0;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (i < N) {
                oob += (npx[i] < k.xmin || npx[i] > k.xmax || npy[i] < k.ymin || npy[i] > k.ymax) ? 1 : 0;
                rew += dold[i] - tnorm(npx[i] - gx[i], npy[i] - gy[i]);
                if (k.waypoint) {
                    const float ex = npx[i] - gx[i], ey = npy[i] - gy[i];
                    if (ex * ex + ey * ey < k.goal_eps2) {
                        const float3 g = waypoint_goal(A.sc, A.seed, e, ep, i, t + 1);
                        gx[i] = g.x;
                        gy[i] = g.y;
                        gth[i] = g.z;
                        ++c_succ;
                    }
                }
            }
        }
        rew -= k.c_col * (float)col;
        c_col += col;
        c_oob += oob;
        c_act += qflags & 1;
        c_flag += (qflags >> 1) & 1;
        c_inf += (res.status == 1) ? 1 : 0;
        c_it += res.iters;
        // ---- episode end and auto-reset
        t += 1;
        const bool done = t >= k.episode_len;
        if (done) {
            c_ep += 1;
            ep += 1;
            t = 0;
            const ThreadPose P = thread_sample(A.sc, A.seed, k.max_attempts, e, ep, N);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                x[i] = P.x[i]; y[i] = P.y[i]; th[i] = P.th[i]; gx[i] = P.gx[i]; gy[i] = P.gy[i];
                gth[i] = P.gth[i];
                __sincosf(th[i], &sn[i], &cs[i]);
            }
        }
        // ---- observations: [x, y, th, gx, gy] + others [dx, dy, dth] in index order
        if (A.io.obs) {
            float* ob = A.io.obs + (long long)step * A.io.obs_step + (long long)off * od;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (i < N) {
                    float rel[9];
#pragma unroll
                    for (int sl = 0; sl < 3; ++sl) {
                        const int j = sl + (sl >= i ? 1 : 0);
                        const bool live = j < N;
                        rel[3 * sl] = live ? x[j] - x[i] : 0.f;
                        rel[3 * sl + 1] = live ? y[j] - y[i] : 0.f;
                        rel[3 * sl + 2] = live ? twrap(th[j] - th[i]) : 0.f;
                    }
                    float* o = ob + i * od;
                    if (od == 14) {
                        float2* o2 = reinterpret_cast<float2*>(o);
                        o2[0] = make_float2(x[i], y[i]);
                        o2[1] = make_float2(th[i], gx[i]);
                        o2[2] = make_float2(gy[i], rel[0]);
                        o2[3] = make_float2(rel[1], rel[2]);
                        o2[4] = make_float2(rel[3], rel[4]);
                        o2[5] = make_float2(rel[5], rel[6]);
                        o2[6] = make_float2(rel[7], rel[8]);
                    } else {
                        const float head[5] = {x[i], y[i], th[i], gx[i], gy[i]};
#pragma unroll
                        for (int s2 = 0; s2 < 5; ++s2)
                            if (s2 < od) o[s2] = head[s2];
#pragma unroll
                        for (int s2 = 0; s2 < 9; ++s2)
                            if (5 + s2 < od) o[5 + s2] = rel[s2];
                        for (int s2 = 14; s2 < od; ++s2) o[s2] = 0.f;
                    }
                }
            }
        }
        if (A.io.reward) A.io.reward[(long long)step * A.io.E + e] = rew;
        if (A.io.done) A.io.done[(long long)step * A.io.E + e] = done ? 1 : 0;
        ret_acc += rew;
    }
    if (A.io.ret) A.io.ret[e] = ret_acc;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (i < N) {
            A.s.x[off + i] = x[i]; A.s.y[off + i] = y[i]; A.s.th[off + i] = th[i];
            A.s.gx[off + i] = gx[i]; A.s.gy[off + i] = gy[i]; A.s.gth[off + i] = gth[i];
        }
    }
    A.s.t[e] = t;
    A.s.ep[e] = ep;
    int32_t* cn = A.s.counters + e * kNCount;
    cn[0] += c_col; cn[1] += c_oob; cn[2] += c_succ; cn[3] += c_act; cn[4] += c_flag; cn[5] += c_inf;
    cn[6] += c_ep; cn[7] += c_it;
}

// A.warp_envs lanes of each 32-lane warp take one env each (fewer envs per warp: less
// divergence between envs and more warps in flight); the other lanes idle.
__global__ void __launch_bounds__(128, 1) env_kernel_thread(LaunchArgs<float> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int per = A.warp_envs;
    if (lane >= per) return;
    QPWork<double, 4>& W = reinterpret_cast<QPWork<double, 4>*>(smem_raw)[threadIdx.x];
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int idx = warp * per + lane; idx < A.n_list; idx += warps * per) {
        const int e = A.env_list ? A.env_list[idx] : A.env_begin + idx;
        run_env_thread(A, e, W);
    }
}

}  // namespace rl
