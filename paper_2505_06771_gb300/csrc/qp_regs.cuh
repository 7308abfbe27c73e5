// qp_regs.cuh -- the barrier QP of one env of at most 4 robots, whole in registers.
//
// Rows are compile-time slots in the method's tie-break order: pairs (a, b), a < b,
// lexicographic, then per robot the arena rows [+x, -x, +y, -y]; a slot is valid when its robots
// exist (index < N).  The active set is a bitmask over slots plus dense 8-vector copies of at most
// CAP active rows with their multipliers and Cholesky factor.  The dual active-set iteration is
// the one of qp_solve in env_step.cuh (Goldfarb-Idnani on H = I, Sec. 3 barrier QP); its first
// step, the projection onto the most violated row's half-plane, is closed form.
// Used by the one-thread-per-env kernel (env_thread.cuh) and by the gather team kernel's second
// violated row (env_nav4.cuh); the register team kernels use team_qp (qp_team.cuh), the same
// iteration with the pair rows taken first.
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
    Q thr[22];               // violation threshold per slot (+inf: the slot's robots are absent)
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
        const bool ok = !((act >> r) & 1u) && vv > R.thr[r];
        if (ok && vv > v0) { v0 = vv; i0 = r; }
    }
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const int r = 6 + m;
        const int i = m >> 2, s = m & 3;
        const Q au = (s == 0) ? U[2 * i] : (s == 1) ? -U[2 * i] : (s == 2) ? U[2 * i + 1] : -U[2 * i + 1];
        const Q vv = au - R.bb[m];
        const bool ok = !((act >> r) & 1u) && vv > R.thr[r];
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
// overflow: the active set outgrew CAP rows (status 2; the caller re-solves).
template <typename Q, int CAP>
__device__ __forceinline__ QPResult thread_qp(const Q (&Px)[4], const Q (&Py)[4], int N,
                                              const Q (&U0)[8], const QPConsts<Q>& c,
                                              Q (&U)[8], bool& overflow) {
    overflow = false;
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
        R.thr[r] = (b < N) ? c.tol_abs + c.tol_rel * fabs(R.bp[r]) : (Q)CUDART_INF;
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
        R.thr[6 + m] = (i < N) ? c.tol_abs + c.tol_rel * fabs(R.bb[m]) : (Q)CUDART_INF;
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
    r = tscan(R, U, act, c, vb);
    while (r >= 0) {
        if (++res.iters > c.max_iter) { res.status = 2; break; }
        Q ap[8], bp, hp;
        trow(R, r, ap, bp, hp, c.r2);
        const Q app = tdot(ap, ap);
        Q lam_p = (Q)0;
        bool added = false;
        if constexpr (CAP >= 2) if (q == 1) {
            // The common second row, written out: with one active row the Cholesky solves are
            // scalar, and the row is added when the full primal step is feasible (tf <= td).
            // Otherwise (a drop, a dependent row) the general pass below takes it.
            const Q y0 = tdot(AR[0], ap) * dinv[0];
            const Q r0 = y0 * dinv[0];
            Q z[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) z[m] = ap[m] - r0 * AR[0][m];
            const Q zz = tdot(z, z);
            const Q td = r0 > (Q)0 ? lam[0] / r0 : (Q)CUDART_INF;
            const Q tf = (tdot(ap, U) - bp) / zz;
            if (zz > c.eps_dep * app && tf <= td) {
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    U[m] -= tf * z[m];
                    AR[1][m] = ap[m];
                }
                lam[0] -= tf * r0;
                const Q dg = sqrt(zz);
                L[1] = y0;
                L[2] = dg;
                dinv[1] = (Q)1 / dg;
                lam[1] = tf;
                hs[1] = hp;
                slot[1] = r;
                act |= 1u << r;
                q = 2;
                added = true;
            }
        }
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

}  // namespace rl
