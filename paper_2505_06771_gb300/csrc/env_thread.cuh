// env_thread.cuh -- one thread per environment for Navigation batches of at most 4 robots.
//
// Same method and results (up to rounding) as run_env in env_step.cuh.  On GB300 a dependent warp
// shuffle costs about 48-66 cycles against about 4.5 for a dependent FMA, so for 4-robot envs a
// thread that owns all four robots, the 22 barrier rows and the whole QP in registers beats any
// multi-lane team: no step of the environment crosses lanes, and the four robots and 22 rows
// give the compiler independent work to interleave.
//
// Rows are compile-time slots in the method's tie-break order: pairs (a, b), a < b,
// lexicographic, then per robot the arena rows [+x, -x, +y, -y]; a slot is valid when its robots
// exist (index < N).  The active set is a bitmask over slots plus dense 8-vector copies of at most
// kThreadRows active rows with their multipliers and Cholesky factor.  The dual active-set
// iteration is the one of qp_solve (Goldfarb-Idnani on H = I); its first step, the projection
// onto the most violated row's half-plane, is closed form.  A flagged QP is re-solved in binary64
// by the shared-memory solver of env_step.cuh, the thread acting as a one-lane team.
#pragma once
#include "env_step.cuh"

namespace rl {

constexpr int kThreadRows = 4;   // active rows held in binary32 registers (more: binary64 re-solve)
constexpr int kSlots = 22;       // 6 pair slots + 16 arena slots (N <= 4)

__device__ __forceinline__ constexpr int slot_a(int r) { return r < 1 ? 0 : r < 2 ? 0 : r < 3 ? 0 : r < 4 ? 1 : r < 5 ? 1 : 2; }
__device__ __forceinline__ constexpr int slot_b(int r) { return r == 0 ? 1 : r == 1 ? 2 : r == 2 ? 3 : r == 3 ? 2 : r == 4 ? 3 : 3; }

template <typename Q>
struct TRows {
    Q dx[6], dy[6], bp[6];   // pair rows: p_a - p_b and gamma h^3
    Q bb[16];                // arena rows: kappa gamma d^3
    unsigned valid;          // bit per slot
};

// Violations of every valid inactive slot at u; returns the most violated (ties: lowest slot)
// or -1.  Three in-order chains (pair rows; arena rows of robots 0-1; of robots 2-3) run in
// parallel and are merged in slot order, so the lowest slot wins every tie.
template <typename Q>
__device__ __forceinline__ int tscan(const TRows<Q>& R, const Q (&U)[8], unsigned act,
                                     const QPConsts<Q>& c, Q& vbest) {
    Q v0 = (Q)0, v1 = (Q)0, v2 = (Q)0;
    int i0 = -1, i1 = -1, i2 = -1;
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        const int a = slot_a(r), b = slot_b(r);
        const Q du = U[2 * a] - U[2 * b], dv = U[2 * a + 1] - U[2 * b + 1];
        const Q vv = (Q)-2 * (R.dx[r] * du + R.dy[r] * dv) - R.bp[r];
        const bool ok = ((R.valid >> r) & 1u) && !((act >> r) & 1u) &&
                        vv > c.tol_abs + c.tol_rel * fabs(R.bp[r]);
        if (ok && vv > v0) { v0 = vv; i0 = r; }
    }
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const int r = 6 + m;
        const int i = m >> 2, s = m & 3;
        const Q au = (s == 0) ? U[2 * i] : (s == 1) ? -U[2 * i] : (s == 2) ? U[2 * i + 1] : -U[2 * i + 1];
        const Q vv = au - R.bb[m];
        const bool ok = ((R.valid >> r) & 1u) && !((act >> r) & 1u) &&
                        vv > c.tol_abs + c.tol_rel * fabs(R.bb[m]);
        if (m < 8) {
            if (ok && vv > v1) { v1 = vv; i1 = r; }
        } else {
            if (ok && vv > v2) { v2 = vv; i2 = r; }
        }
    }
    if (v1 > v0) { v0 = v1; i0 = i1; }
    if (v2 > v0) { v0 = v2; i0 = i2; }
    vbest = v0;
    return i0;
}

// Dense coefficient vector and bound of slot r; h of a pair row (arena rows: +inf).
template <typename Q>
__device__ __forceinline__ void trow(const TRows<Q>& R, int r, Q (&a)[8], Q& b, Q& h, Q r2) {
#pragma unroll
    for (int m = 0; m < 8; ++m) a[m] = (Q)0;
    h = (Q)1e30;
    if (r < 6) {
        Q dx = 0, dy = 0, bp = 0;
        int pa = 0, pb = 1;
#pragma unroll
        for (int s = 0; s < 6; ++s)
            if (s == r) { dx = R.dx[s]; dy = R.dy[s]; bp = R.bp[s]; pa = slot_a(s); pb = slot_b(s); }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            a[2 * m] = (m == pa) ? (Q)-2 * dx : ((m == pb) ? (Q)2 * dx : a[2 * m]);
            a[2 * m + 1] = (m == pa) ? (Q)-2 * dy : ((m == pb) ? (Q)2 * dy : a[2 * m + 1]);
        }
        b = bp;
        h = dx * dx + dy * dy - r2;
    } else {
        const int m = r - 6, i = m >> 2, s = m & 3;
        Q bb = 0;
#pragma unroll
        for (int t = 0; t < 16; ++t)
            if (t == m) bb = R.bb[t];
        const Q sg = (s & 1) ? (Q)-1 : (Q)1;
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (k == 2 * i + (s >> 1)) a[k] = sg;
        b = bb;
    }
}

template <typename Q>
__device__ __forceinline__ Q tdot(const Q (&a)[8], const Q (&b)[8]) {
    Q s = (Q)0;
#pragma unroll
    for (int m = 0; m < 8; ++m) s += a[m] * b[m];
    return s;
}

__device__ __forceinline__ int ttri(int i, int k) { return i * (i + 1) / 2 + k; }

// The QP of one env from its projected points and nominal velocities (dense u over 4 robots).
template <typename Q, int CAP>
__device__ __forceinline__ QPResult thread_qp(const Q (&Px)[4], const Q (&Py)[4], int N,
                                              const Q (&U0)[8], const QPConsts<Q>& c,
                                              Q (&U)[8]) {
    QPResult res;
    res.status = 0;
    res.q = 0;
    res.iters = 0;
    res.flag = false;
    TRows<Q> R;
    R.valid = 0u;
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        const int a = slot_a(r), b = slot_b(r);
        R.dx[r] = Px[a] - Px[b];
        R.dy[r] = Py[a] - Py[b];
        const Q h = R.dx[r] * R.dx[r] + R.dy[r] * R.dy[r] - c.r2;
        R.bp[r] = c.gamma * h * h * h;
        if (b < N) R.valid |= 1u << r;
    }
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const int i = m >> 2, s = m & 3;
        const Q d = (s == 0) ? c.xmax - c.half_r - Px[i]
                  : (s == 1) ? Px[i] - c.xmin - c.half_r
                  : (s == 2) ? c.ymax - c.half_r - Py[i]
                             : Py[i] - c.ymin - c.half_r;
        R.bb[m] = c.kg * d * d * d;
        if (i < N) R.valid |= 1u << (6 + m);
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) U[m] = U0[m];
    Q vb;
    int r = tscan(R, U, 0u, c, vb);
    if (r < 0) return res;

    Q AR[CAP][8], lam[CAP], L[CAP * (CAP + 1) / 2],
        dinv[CAP], hs[CAP];
    int slot[CAP];
    unsigned act = 0u;
    int q = 0;
    {
        // first iteration in closed form: u <- u - (v / |a|^2) a
        Q a[8], b, h;
        trow(R, r, a, b, h, c.r2);
        const Q app = tdot(a, a);
        const Q st = vb / app;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            U[m] -= st * a[m];
            AR[0][m] = a[m];
        }
        lam[0] = st;
        L[0] = sqrt(app);
        dinv[0] = (Q)1 / L[0];
        hs[0] = h;
        slot[0] = r;
        act = 1u << r;
        q = 1;
        res.iters = 1;
    }
    bool overflow = false;
    r = tscan(R, U, act, c, vb);
    while (r >= 0) {
        if (++res.iters > c.max_iter) { res.status = 2; break; }
        Q ap[8], bp, hp;
        trow(R, r, ap, bp, hp, c.r2);
        const Q app = tdot(ap, ap);
        Q lam_p = (Q)0;
        bool added = false;
        for (int guard = 0; guard <= CAP + 1 && !added; ++guard) {
            Q y[CAP], rr[CAP];
#pragma unroll
            for (int t = 0; t < CAP; ++t) {
                y[t] = (Q)0;
                if (t < q) {
                    Q s = tdot(AR[t], ap);
#pragma unroll
                    for (int m = 0; m < t; ++m) s -= L[ttri(t, m)] * y[m];
                    y[t] = s * dinv[t];
                }
            }
#pragma unroll
            for (int t = CAP - 1; t >= 0; --t) {
                rr[t] = (Q)0;
                if (t < q) {
                    Q s = y[t];
#pragma unroll
                    for (int m = t + 1; m < CAP; ++m)
                        if (m < q) s -= L[ttri(m, t)] * rr[m];
                    rr[t] = s * dinv[t];
                }
            }
            Q z[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) z[m] = ap[m];
#pragma unroll
            for (int t = 0; t < CAP; ++t)
                if (t < q) {
#pragma unroll
                    for (int m = 0; m < 8; ++m) z[m] -= rr[t] * AR[t][m];
                }
            const Q zz = tdot(z, z);
            Q td = (Q)CUDART_INF;
            int jb = -1;
#pragma unroll
            for (int t = 0; t < CAP; ++t)
                if (t < q && rr[t] > (Q)0) {
                    const Q tj = lam[t] / rr[t];
                    if (tj < td) { td = tj; jb = t; }
                }
            const Q sp = tdot(ap, U) - bp;
            const bool indep = zz > c.eps_dep * app;
            if (!indep) res.flag = true;
            const Q tf = indep ? sp / zz : (Q)CUDART_INF;
            if (!(tf < (Q)CUDART_INF) && !(td < (Q)CUDART_INF)) {
                res.status = 1;
                break;
            }
            const Q st = tf < td ? tf : td;
            if (tf < (Q)CUDART_INF) {
#pragma unroll
                for (int m = 0; m < 8; ++m) U[m] -= st * z[m];
            }
#pragma unroll
            for (int t = 0; t < CAP; ++t)
                if (t < q) lam[t] -= st * rr[t];
            lam_p += st;
            if (tf <= td) {
                if (q == CAP) { overflow = true; break; }
                const Q dg = sqrt(zz);
#pragma unroll
                for (int t = 0; t < CAP; ++t) {
                    if (t == q) {
#pragma unroll
                        for (int m = 0; m < t; ++m) L[ttri(t, m)] = y[m];
                        L[ttri(t, t)] = dg;
                        dinv[t] = (Q)1 / dg;
#pragma unroll
                        for (int m = 0; m < 8; ++m) AR[t][m] = ap[m];
                        lam[t] = lam_p;
                        hs[t] = hp;
                        slot[t] = r;
                    }
                }
                act |= 1u << r;
                ++q;
                added = true;
            } else {
                int js = 0;
#pragma unroll
                for (int t = 0; t < CAP; ++t)
                    if (t == jb) js = slot[t];
                act &= ~(1u << js);
#pragma unroll
                for (int t = 0; t < CAP - 1; ++t)
                    if (t >= jb) {
#pragma unroll
                        for (int m = 0; m < 8; ++m) AR[t][m] = AR[t + 1][m];
                        lam[t] = lam[t + 1];
                        hs[t] = hs[t + 1];
                        slot[t] = slot[t + 1];
                    }
                --q;
                bool ok = true;
#pragma unroll
                for (int t = 0; t < CAP; ++t)
                    if (t < q) {
#pragma unroll
                        for (int m = 0; m <= t; ++m) {
                            Q g = tdot(AR[t], AR[m]);
#pragma unroll
                            for (int n = 0; n < m; ++n) g -= L[ttri(t, n)] * L[ttri(m, n)];
                            if (m == t) {
                                ok = ok && (g > (Q)0);
                                const Q dg = sqrt(g > (Q)1e-30 ? g : (Q)1e-30);
                                L[ttri(t, t)] = dg;
                                dinv[t] = (Q)1 / dg;
                            } else {
                                L[ttri(t, m)] = g * dinv[m];
                            }
                        }
                    }
                if (!ok) { res.status = 2; break; }
            }
        }
        if (res.status != 0) break;
        if (overflow) { res.status = 2; break; }  // more active rows than registers: re-solve
        if (!added) { res.status = 2; break; }
        r = tscan(R, U, act, c, vb);
    }
    res.q = q;
    if (res.status == 0) {
#pragma unroll
        for (int t = 0; t < CAP; ++t)
            if (t < q && hs[t] < c.h_flag) res.flag = true;  // near-degenerate pair row
    } else {
        res.flag = true;
        if (res.status == 1) {
#pragma unroll
            for (int m = 0; m < 8; ++m) U[m] = (Q)0;
        }
    }
    return res;
}

// Reset sampler of one env of N <= 4 robots in one thread (binary32, one rounding per
// operation; the same draws as team_sample).
struct ThreadPose {
    float x[4], y[4], th[4], gx[4], gy[4];
};

static __device__ __noinline__ ThreadPose thread_sample(const SamplerConsts sc, uint64_t seed,
                                                        int max_att, int e, int ep, int N) {
    ThreadPose P;
#pragma unroll
    for (int i = 0; i < 4; ++i) P.x[i] = P.y[i] = P.th[i] = P.gx[i] = P.gy[i] = 0.f;
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

    float x[4], y[4], th[4], gx[4], gy[4], cs[4], sn[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int row = off + (i < N ? i : 0);
        x[i] = A.s.x[row]; y[i] = A.s.y[row]; th[i] = A.s.th[row];
        gx[i] = A.s.gx[row]; gy[i] = A.s.gy[row];
        __sincosf(th[i], &sn[i], &cs[i]);
    }
    int t = A.s.t[e], ep = A.s.ep[e];
    int c_col = 0, c_oob = 0, c_act = 0, c_flag = 0, c_inf = 0, c_ep = 0, c_it = 0;
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
        QPResult res = thread_qp<float, kThreadRows>(px, py, N, U0, qc, U);
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
            A.s.gx[off + i] = gx[i]; A.s.gy[off + i] = gy[i];
        }
    }
    A.s.t[e] = t;
    A.s.ep[e] = ep;
    int32_t* cn = A.s.counters + e * kNCount;
    cn[0] += c_col; cn[1] += c_oob; cn[3] += c_act; cn[4] += c_flag; cn[5] += c_inf;
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
