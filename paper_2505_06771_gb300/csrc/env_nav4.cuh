// env_nav4.cuh -- the Navigation step for envs of at most 4 robots (binary32, scripted nominal
// control, no traces): the hot path of the 4096 x 4 rollout and of the single-env waypoint run.
//
// Same method and results (up to rounding) as run_env_small, for either scripted controller
// (position, or the unicycle pose controller).  A team of 4 lanes runs one env,
// lane i owning robot i, and the step is organised around two all-gathers -- one batch of
// independent shuffles each, so the team pays one shuffle latency per batch:
//   1. after the nominal velocities are formed, every lane gathers all four (u_nom);
//   2. after the Euler step, every lane gathers all poses and projected points.
// Everything else is either redundant in every lane, computed from the gathered values -- the
// collision and arena flags, the team reward, the relative poses of the observation, the
// closed-form first active-set step -- or split by rows: each lane evaluates its own barrier
// rows (its circulant pair rows and its four arena rows) and the team picks the most violated
// row with one warp reduction (redux.sync max) over keys that pack the violation with the row's
// slot.  Most QPs (Sec. 3 barrier QP, dual active set) end there or after one closed-form step;
// a second violated row hands the QP to the register solver of qp_regs.cuh, which every lane
// runs on the whole 8-variable problem, and beyond its capacity to the shared-memory solver.
#pragma once
#include "env_small.cuh"

namespace rl {

// The rows a lane owns in one QP: pair rows with its circulant partners (slot in the tie-break
// order, sign of the lane's robot in the row, p_a - p_b, gamma h^3, threshold) and its robot's
// four arena rows.  Thresholds are +inf for rows that do not exist (partner beyond the lane's
// pair count, absent robot).
struct Nav4Rows {
    int pslot[2];
    float sg[2];             // +1 when the lane's robot is a, -1 when it is b
    float dx[2], dy[2], bp[2], pthr[2];
    int bslot0;              // slot of the lane's +x arena row
    float bb[4], bthr[4];
    int hneg;                // pair rows with h < 0 (colliding projected points)
};

__device__ __forceinline__ void nav4_rows(int i, int N, int ndi, const int (&jn)[2], float px,
                                          float py, const float (&qx)[2], const float (&qy)[2],
                                          const QPConsts<float>& c, Nav4Rows& R) {
    const int P = N * (N - 1) / 2;
    R.hneg = 0;
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        const int j = jn[d];
        const int a = min(i, j), b = max(i, j);
        R.pslot[d] = pair_index(a, b, N);
        R.sg[d] = (a == i) ? 1.f : -1.f;
        R.dx[d] = R.sg[d] * (px - qx[d]);
        R.dy[d] = R.sg[d] * (py - qy[d]);
        const float h = R.dx[d] * R.dx[d] + R.dy[d] * R.dy[d] - c.r2;
        R.bp[d] = c.gamma * h * h * h;
        R.pthr[d] = (d < ndi) ? c.tol_abs + c.tol_rel * fabsf(R.bp[d]) : CUDART_INF_F;
    }
    const bool own = i < N;
    const float d4[4] = {c.xmax - c.half_r - px, px - c.xmin - c.half_r,
                         c.ymax - c.half_r - py, py - c.ymin - c.half_r};
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        R.bb[s] = c.kg * d4[s] * d4[s] * d4[s];
        R.bthr[s] = own ? c.tol_abs + c.tol_rel * fabsf(R.bb[s]) : CUDART_INF_F;
    }
    R.bslot0 = P + 4 * i;
}

// A violated row as a key: the violation's bits with the low five replaced by 31 - slot.  For
// positive violations the unsigned order is the float order, so the team's unsigned maximum is
// the most violated row (to 2^-18 relative) with ties to the lowest slot.  The tie rule only
// orders the active-set iterations; the minimiser they reach is unique.
__device__ __forceinline__ unsigned nav4_key(float v, float thr, int slot, int act) {
    return (v > thr && slot != act) ? ((__float_as_uint(v) & 0xFFFFFFE0u) | (unsigned)(31 - slot))
                                    : 0u;
}

// The team's most violated row at u (own robot's u, the pair partners' u), excluding slot act.
__device__ __forceinline__ unsigned nav4_scan(const Team<4>& tm, const Nav4Rows& R, float uix,
                                              float uiy, const float (&wx)[2],
                                              const float (&wy)[2], int act) {
    unsigned k0 = 0u, k1 = 0u;
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        const float dux = R.sg[d] * (uix - wx[d]), duy = R.sg[d] * (uiy - wy[d]);
        const float v = -2.f * (R.dx[d] * dux + R.dy[d] * duy) - R.bp[d];
        k0 = max(k0, nav4_key(v, R.pthr[d], R.pslot[d], act));
    }
    const float au[4] = {uix, -uix, uiy, -uiy};
#pragma unroll
    for (int s = 0; s < 4; ++s)
        k1 = max(k1, nav4_key(au[s] - R.bb[s], R.bthr[s], R.bslot0 + s, act));
    return __reduce_max_sync(tm.mask, max(k0, k1));
}

// Robots a < b of pair slot s < N(N-1)/2.
__device__ __forceinline__ void nav4_pair(int s, int N, int& a, int& b) {
    int k = 0;
    a = 0;
    b = 1;
#pragma unroll
    for (int aa = 0; aa < 4; ++aa)
#pragma unroll
        for (int bb = aa + 1; bb < 4; ++bb)
            if (bb < N) {
                if (k == s) { a = aa; b = bb; }
                ++k;
            }
}

// The whole QP in registers (qp_regs.cuh), out of line: reached by the few QPs with a second
// violated row after the closed-form step.  Operands come from the team's published values.
static __device__ __noinline__ QPResult nav4_full(const TeamSmem<float, 4>& S, int cb, int N,
                                                  const QPConsts<float> c, bool& overflow,
                                                  float& usx, float& usy, int i) {
    float px[4], py[4], u0[8], u[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        px[j] = S.g4[cb][j][0].w;
        py[j] = S.g4[cb][j][1].x;
        u0[2 * j] = S.g2[j].x;
        u0[2 * j + 1] = S.g2[j].y;
    }
    const QPResult r = thread_qp<float, kRegRows>(px, py, N, u0, c, u, overflow);
    usx = (i == 0) ? u[0] : (i == 1) ? u[2] : (i == 2) ? u[4] : u[6];
    usy = (i == 0) ? u[1] : (i == 1) ? u[3] : (i == 2) ? u[5] : u[7];
    return r;
}

static __device__ __forceinline__ void run_env_nav4(const LaunchArgs<float>& A, const Team<4>& tm,
                                                    TeamSmem<float, 4>& S, int e) {
    const StepConsts<float>& k = A.k;
    const int off = A.s.off[e];
    const int N = A.s.nrob[e];
    const int i = tm.lane;
    const bool own = i < N;
    const int row = off + (own ? i : 0);

    QPConsts<float> qc;
    qc.gamma = k.gamma; qc.r2 = k.r2; qc.kg = k.kg; qc.half_r = k.half_r;
    qc.xmin = k.xmin; qc.xmax = k.xmax; qc.ymin = k.ymin; qc.ymax = k.ymax;
    qc.h_flag = k.h_flag;
    qc.max_iter = k.max_iter;
    qc.tol_abs = 2e-7f; qc.tol_rel = 1e-6f; qc.eps_dep = 1e-5f; qc.tol_lam = 1e-6f;

    float x = A.s.x[row], y = A.s.y[row], th = A.s.th[row];
    float gx = A.s.gx[row], gy = A.s.gy[row], gth = A.s.gth[row];
    const int lv = A.s.level[row];
    float sn, cs;
    __sincosf(th, &sn, &cs);
    int t = A.s.t[e], ep = A.s.ep[e];
    int c_col = 0, c_oob = 0, c_succ = 0, c_act = 0, c_flag = 0, c_inf = 0, c_ep = 0, c_it = 0;
    const int nd = (N - 1) / 2;
    const int ndi = own ? nd + (((N & 1) == 0 && i < N / 2) ? 1 : 0) : 0;
    int jn[2];  // the robots of the lane's circulant pair rows (offsets 1 and 2)
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        int j = i + d + 1;
        while (j >= N) j -= N;
        jn[d] = own ? j : i;
    }
    int jo[3];  // the others in index order: observation slot s holds robot s + (s >= i)
#pragma unroll
    for (int sl = 0; sl < 3; ++sl) jo[sl] = sl + (sl >= i ? 1 : 0);

    // Every lane publishes its robot's pose and projected point (g4[cb][i][0] = x, y, th, p_x;
    // g4[cb][i][1] = p_y, reward term, out-of-arena flag, arrival flag) once per step, and its
    // nominal velocity (g2[i]) once per QP, each write followed by a __syncwarp over the team.
    // The state alternates between two buffers, so every write is separated from the last
    // reads of the values it replaces by the other publication's __syncwarp.
    int cb = 1;
    auto publish = [&](float npx, float npy, float dterm, int oob_i, int arr_i) {
        cb ^= 1;
        S.g4[cb][i][0] = make_float4(x, y, th, npx);
        S.g4[cb][i][1] = make_float4(npy, dterm, (float)oob_i, (float)arr_i);
        tm.sync();
    };
    float npx = x + k.l * cs, npy = y + k.l * sn;
    publish(npx, npy, 0.f, 0, 0);

    // Noise words of the own robot for the coming step, drawn one step ahead (the draw
    // depends on the counters only, so it overlaps the previous step's work).  Robots 2m and
    // 2m+1 share the Philox block (pair m, step t); their two lanes draw the blocks of steps t
    // and t + 1 at once and swap them, so each lane runs Philox every other step (the words of
    // step t + 1 are kept while the episode continues).  Measured on one env: Philox is 8% of
    // the step.
    int nz_t = -2, nz_ep = -1;  // the kept words are those of step nz_t + 1 of episode nz_ep
    uint32_t nz_nx = 0u, nz_ny = 0u;
    auto noise_words = [&](uint32_t& nwx, uint32_t& nwy) {
        if (nz_ep == ep && nz_t + 1 == t) {
            nwx = nz_nx;
            nwy = nz_ny;
            nz_t = -2;
            return;
        }
        const Words4 w = draw(A.seed, e, ep, kNoise, i >> 1, (uint32_t)(t + (i & 1)));
        uint32_t o[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) o[m] = __shfl_xor_sync(tm.mask, w.w[m], 1, 4);
        // block of step t: the even lane's; of step t + 1: the odd lane's
        nwx = (i & 1) ? o[2] : w.w[0];
        nwy = (i & 1) ? o[3] : w.w[1];
        nz_nx = (i & 1) ? w.w[2] : o[0];
        nz_ny = (i & 1) ? w.w[3] : o[1];
        nz_t = t;
        nz_ep = ep;
    };
    uint32_t nwx, nwy;
    noise_words(nwx, nwy);

    float ret_acc = 0.f;

    for (int step = 0; step < A.T; ++step) {
        // ---- nominal SI velocity of the own robot (go to goal, cap, noise, cap)
        const float px = npx, py = npy;
        const float dold = fast_norm(px - gx, py - gy);
        float ux, uy;
        if (k.controller == 1) {
            pose_nominal<float>(k, x, y, th, gx, gy, gth, ux, uy);
        } else {
            ux = k.k_si * (gx - px);
            uy = k.k_si * (gy - py);
        }
        cap_fast(ux, uy, k.vmax);
        {
            const float ex = __fmul_rn(__fsub_rn(unit24(nwx), 0.5f), k.noise_scale);
            const float ey = __fmul_rn(__fsub_rn(unit24(nwy), 0.5f), k.noise_scale);
            ux += k.noise_on ? ex : 0.f;
            uy += k.noise_on ? ey : 0.f;
        }
        cap_fast(ux, uy, k.vmax);

        // ---- the barrier QP: own rows, partners' projected points and u_nom, team maximum
        S.g2[i] = make_float2(ux, uy);
        tm.sync();
        float qx[2], qy[2], wx[2], wy[2];
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            qx[d] = S.g4[cb][jn[d]][0].w;
            qy[d] = S.g4[cb][jn[d]][1].x;
            const float2 w = S.g2[jn[d]];
            wx[d] = w.x;
            wy[d] = w.y;
        }
        Nav4Rows R;
        nav4_rows(i, N, ndi, jn, px, py, qx, qy, qc, R);
        QPResult res;
        res.status = 0;
        res.q = 0;
        res.iters = 0;
        res.flag = false;
        float usx = ux, usy = uy;
        unsigned K = nav4_scan(tm, R, ux, uy, wx, wy, -1);
        if (K != 0u) {
            // first iteration, closed form: u <- u - (v / |a|^2) a, in every lane
            const int s1 = 31 - (int)(K & 31u);
            const int P = N * (N - 1) / 2;
            int a, b = -1;
            float cx, cy, bv, h = 1e30f;
            if (s1 < P) {
                nav4_pair(s1, N, a, b);
                const float dx = S.g4[cb][a][0].w - S.g4[cb][b][0].w;
                const float dy = S.g4[cb][a][1].x - S.g4[cb][b][1].x;
                h = dx * dx + dy * dy - qc.r2;
                bv = qc.gamma * h * h * h;
                cx = -2.f * dx;
                cy = -2.f * dy;
            } else {
                const int m = s1 - P, sd = m & 3;
                a = m >> 2;
                const float pa = (sd < 2) ? S.g4[cb][a][0].w : S.g4[cb][a][1].x;
                const float dd = (sd == 0) ? qc.xmax - qc.half_r - pa
                               : (sd == 1) ? pa - qc.xmin - qc.half_r
                               : (sd == 2) ? qc.ymax - qc.half_r - pa
                                           : pa - qc.ymin - qc.half_r;
                bv = qc.kg * dd * dd * dd;
                cx = (sd == 0) ? 1.f : ((sd == 1) ? -1.f : 0.f);
                cy = (sd == 2) ? 1.f : ((sd == 3) ? -1.f : 0.f);
            }
            const float2 ua = S.g2[a];
            const float2 ub = (b >= 0) ? S.g2[b] : make_float2(0.f, 0.f);
            const float v = cx * (ua.x - ub.x) + cy * (ua.y - ub.y) - bv;
            const float app = (b >= 0 ? 2.f : 1.f) * (cx * cx + cy * cy);
            const float st = v / app;
            // the lane's copies of u (own robot, pair partners) move with the step
            const float si = (i == a) ? st : ((i == b) ? -st : 0.f);
            usx -= si * cx;
            usy -= si * cy;
#pragma unroll
            for (int d = 0; d < 2; ++d) {
                const float sj = (jn[d] == a) ? st : ((jn[d] == b) ? -st : 0.f);
                wx[d] -= sj * cx;
                wy[d] -= sj * cy;
            }
            res.q = 1;
            res.iters = 1;
            res.flag = (b >= 0 && h < qc.h_flag);
            K = nav4_scan(tm, R, usx, usy, wx, wy, s1);
            if (K != 0u) {
                // a second violated row: the whole QP again, in registers
                bool overflow;
                res = nav4_full(S, cb, N, qc, overflow, usx, usy, i);
                if (overflow) {
                    res = small_general(tm, S, N, px, py, ux, uy, qc);
                    usx = own ? S.qp.s.f.ux[i] : 0.f;
                    usy = own ? S.qp.s.f.uy[i] : 0.f;
                    tm.sync();
                }
            }
        }
        int qflags = (res.q > 0 || res.status != 0) ? 1 : 0;
        if (k.resolve_f64 && res.flag) {
            const QPResult r64 = small_resolve_f64(tm, S, k, N, x, y, th, ux, uy);
            res.status = r64.status;
            res.q = r64.q;
            res.iters += r64.iters;
            usx = own ? (float)S.qp.d.ux[i] : 0.f;
            usy = own ? (float)S.qp.d.uy[i] : 0.f;
            tm.sync();
            qflags |= 2;
        }

        // ---- SI -> unicycle, wheel clip, Euler step
        {
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
        }
        npx = x + k.l * cs;
        npy = y + k.l * sn;

        // ---- own flags and reward term, publish, then the team's totals in every lane
        const float gex = npx - gx, gey = npy - gy;
        const float dterm = dold - fast_norm(gex, gey);
        const int oob_i = (own && (npx < k.xmin || npx > k.xmax || npy < k.ymin || npy > k.ymax)) ? 1 : 0;
        const int arr_i = (own && k.waypoint && gex * gex + gey * gey < k.goal_eps2) ? 1 : 0;
        publish(npx, npy, own ? dterm : 0.f, oob_i, arr_i);
        float4 oa[3], ob[3];
#pragma unroll
        for (int sl = 0; sl < 3; ++sl) {
            oa[sl] = S.g4[cb][jo[sl]][0];
            ob[sl] = S.g4[cb][jo[sl]][1];
        }
        int col = 0, oob = oob_i, narr = arr_i;
        float rew = own ? dterm : 0.f;
        const float ppx[4] = {npx, oa[0].w, oa[1].w, oa[2].w};
        const float ppy[4] = {npy, ob[0].x, ob[1].x, ob[2].x};
        const bool live[4] = {own, jo[0] < N, jo[1] < N, jo[2] < N};
#pragma unroll
        for (int sl = 0; sl < 3; ++sl) {
            if (live[sl + 1]) {
                rew += ob[sl].y;
                oob += (int)ob[sl].z;
                narr += (int)ob[sl].w;
            }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = a + 1; b < 4; ++b) {
                const float dx = ppx[a] - ppx[b], dy = ppy[a] - ppy[b];
                col += (live[a] && live[b] && dx * dx + dy * dy < k.r2) ? 1 : 0;
            }
        rew -= k.c_col * (float)col;
        if (arr_i) {
            // Random Waypoint Navigation: a new goal for the robot that arrived
            const float3 g = waypoint_goal(A.sc, A.seed, e, ep, i, t + 1);
            gx = g.x;
            gy = g.y;
            gth = g.z;
        }
        c_col += col;
        c_oob += oob;
        c_succ += narr;
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
            small_reset(tm, S, A, e, ep, N);
            if (own) {
                x = S.fx[i]; y = S.fy[i]; th = S.fth[i];
                gx = S.sx[i]; gy = S.sy[i]; gth = S.sth[i];
            }
            __sincosf(th, &sn, &cs);
            npx = x + k.l * cs;
            npy = y + k.l * sn;
            // republish into the current buffer once every lane is done reading it
            tm.sync();
            S.g4[cb][i][0] = make_float4(x, y, th, npx);
            S.g4[cb][i][1] = make_float4(npy, 0.f, 0.f, 0.f);
            tm.sync();
#pragma unroll
            for (int sl = 0; sl < 3; ++sl) oa[sl] = S.g4[cb][jo[sl]][0];
        }
        noise_words(nwx, nwy);

        // ---- observations of the own robot: [x, y, th, gx, gy], then the others in index
        // order relative to it
        if (A.io.obs && own) {
            const int od = A.io.obs_dim;
            float* o = A.io.obs + (long long)step * A.io.obs_step + (long long)row * od;
            float rel[9];
#pragma unroll
            for (int sl = 0; sl < 3; ++sl) {
                const bool lv2 = jo[sl] < N;
                rel[3 * sl] = lv2 ? oa[sl].x - x : 0.f;
                rel[3 * sl + 1] = lv2 ? oa[sl].y - y : 0.f;
                rel[3 * sl + 2] = lv2 ? wrap_pi_f(oa[sl].z - th) : 0.f;
            }
            if (od == 14) {
                float2* o2 = reinterpret_cast<float2*>(o);
                o2[0] = make_float2(x, y);
                o2[1] = make_float2(th, gx);
                o2[2] = make_float2(gy, rel[0]);
                o2[3] = make_float2(rel[1], rel[2]);
                o2[4] = make_float2(rel[3], rel[4]);
                o2[5] = make_float2(rel[5], rel[6]);
                o2[6] = make_float2(rel[7], rel[8]);
            } else {
                const float head[5] = {x, y, th, gx, gy};
#pragma unroll
                for (int s2 = 0; s2 < 5; ++s2)
                    if (s2 < od) o[s2] = head[s2];
#pragma unroll
                for (int s2 = 0; s2 < 9; ++s2)
                    if (5 + s2 < od) o[5 + s2] = rel[s2];
                for (int s2 = 14; s2 < od; ++s2) o[s2] = 0.f;
            }
        }
        if (i == 0) {
            if (A.io.reward) A.io.reward[(long long)step * A.io.E + e] = rew;
            if (A.io.done) A.io.done[(long long)step * A.io.E + e] = done ? 1 : 0;
        }
        ret_acc += rew;
    }
    if (A.io.ret && i == 0) A.io.ret[e] = ret_acc;
    if (own) {
        A.s.x[row] = x; A.s.y[row] = y; A.s.th[row] = th;
        A.s.gx[row] = gx; A.s.gy[row] = gy; A.s.gth[row] = gth; A.s.level[row] = lv;
    }
    if (i == 0) {
        A.s.t[e] = t;
        A.s.ep[e] = ep;
        int32_t* cn = A.s.counters + e * kNCount;
        cn[0] += c_col; cn[1] += c_oob; cn[2] += c_succ; cn[3] += c_act;
        cn[4] += c_flag; cn[5] += c_inf; cn[6] += c_ep; cn[7] += c_it;
    }
    tm.sync();
}

// A.warp_envs teams (envs) per 32-lane warp, 1..8 (0: 4); with fewer than 8 the other lanes
// idle, which trades SIMD width for less divergence between envs and more warps per scheduler.
// MODE 0: any scenario, policy actions, traces (run_env_small<false>).  Navigation with scripted
// nominal control and no traces: MODE 1 reduces across the team with shuffles
// (run_env_small<true>), MODE 2 publishes robot state in shared memory (run_env_nav4).
template <int MODE>
__global__ void __launch_bounds__(128, 1) env_kernel_small(LaunchArgs<float> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Team<4> tm;
    const int tiw = (threadIdx.x & 31) >> 2;  // team in warp
    const int tib = threadIdx.x / 4;
    TeamSmem<float, 4>* S = reinterpret_cast<TeamSmem<float, 4>*>(smem_raw) + tib;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    // The team's list entries -- spread: warp w takes [w n / W, (w + 1) n / W), at most 8 (the
    // launcher guarantees it), one per team; else a grid stride of per envs per warp.  One call
    // site: a second inlined copy of the step measured 2-7% slower (instruction footprint).
    int idx, end, stride;
    unsigned wm = 0u;
    if (A.warp_envs <= 0) {
        const long long n = A.n_list;
        const int lo = (int)(warp * n / warps), hi = (int)((warp + 1) * n / warps);
        idx = lo + tiw;
        end = hi;
        stride = 8;
        const int nw = hi - lo;  // the warp's live teams, for the warp-wide rare QPs
        wm = nw >= 8 ? 0xffffffffu : (nw >= 2 ? (1u << (4 * nw)) - 1u : 0u);
    } else {
        const int per = A.warp_envs <= 8 ? A.warp_envs : 4;
        if (tiw >= per) return;
        idx = warp * per + tiw;
        end = A.n_list;
        stride = warps * per;
    }
    for (; idx < end; idx += stride) {
        const int e = A.env_list ? A.env_list[idx] : A.env_begin + idx;
        if constexpr (MODE == 2) run_env_nav4(A, tm, *S, e);
        else if constexpr (MODE == 1) run_env_small<true>(A, tm, *S, e, wm);
        else run_env_small<false>(A, tm, *S, e);
    }
}

}  // namespace rl
