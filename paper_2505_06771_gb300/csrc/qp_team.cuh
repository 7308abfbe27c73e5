// qp_team.cuh -- the barrier QP of one env of at most 4 robots, solved in registers by every lane
// of the env's 4-lane team, pair rows first.
//
// The problem and the iteration are those of thread_qp (qp_regs.cuh): min |u - u_nom|^2 over the
// 8 velocities subject to the pair rows -2 (p_a - p_b).(u_a - u_b) <= gamma h^3 and the arena
// rows +-u <= kappa gamma (d - r/2)^3 (Sec. 4.1, barrier certificates), by the dual active-set
// method on H = I (Goldfarb-Idnani 1983) with the first iteration in closed form.  What differs
// is the order in which rows enter:
//  * the dual method may take violated constraints in any order from any dual-feasible start
//    (the current minimiser of a subset of the rows, with nonnegative multipliers), and the
//    minimiser is unique;
//  * arena rows are seldom active (in the 4096 x 4 Navigation batch about 1e-4 of the
//    env-steps, against 0.28 with an active pair row).
// So the solver first minimises over the 6 pair rows alone, scanning only those; at that
// minimiser (where the envs of a warp meet again) it builds and checks the 16 arena rows once.
// With none violated the point is the minimiser of the whole problem (it minimises a
// relaxation and meets every row).  Otherwise the same iteration goes on over all 22 rows
// from the current active set.
// Room for kTeamRows = 6 active rows: every active set of the pair rows alone fits, so the
// jammed envs whose robots press against each other (five active pair rows) stay in registers.
#pragma once
#include "qp_regs.cuh"

namespace rl {

constexpr int kTeamRows = 6;
// Quotients, square roots and their reciprocals here are the hardware approximations
// (__fdividef, rsqrtf: about 2 ulp), not the correctly rounded ones: they only scale steps and
// factors, so their error stays at binary32 rounding level in the minimiser.  A divisor must be
// above kTinyPos (a multiplier ratio with a smaller positive divisor is an unbounded step).
constexpr float kTinyPos = 1e-30f;

// Bound of arena side s (0 +x, 1 -x, 2 +y, 3 -y) of a robot at projected point (px, py).
template <typename Q>
__device__ __forceinline__ Q arena_bound(const QPConsts<Q>& c, int s, Q px, Q py) {
    const Q d = (s == 0) ? c.xmax - c.half_r - px
              : (s == 1) ? px - c.xmin - c.half_r
              : (s == 2) ? c.ymax - c.half_r - py
                         : py - c.ymin - c.half_r;
    return c.kg * d * d * d;
}

// Violations of the valid inactive pair rows at u; the most violated (ties: lowest slot) or -1.
template <typename Q>
__device__ __forceinline__ int pair_scan(const TRows<Q>& R, const Q (&U)[8], unsigned act,
                                         Q& vbest) {
    Q v0 = (Q)0;
    int i0 = -1;
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        const int a = slot_a(r), b = slot_b(r);
        const Q du = U[2 * a] - U[2 * b], dv = U[2 * a + 1] - U[2 * b + 1];
        const Q vv = (Q)-2 * (R.dx[r] * du + R.dy[r] * dv) - R.bp[r];
        const bool ok = !((act >> r) & 1u) && vv > R.thr[r];
        if (ok && vv > v0) { v0 = vv; i0 = r; }
    }
    vbest = v0;
    return i0;
}

// Violations of the valid inactive arena rows at u (bounds bb, thresholds computed here); the
// most violated (ties: lowest slot) merged into (v0, i0), which holds the pair rows' best.
template <typename Q>
__device__ __forceinline__ int arena_scan(const Q (&bb)[16], const Q (&U)[8], unsigned act, int N,
                                          const QPConsts<Q>& c, Q& v0, int i0) {
    Q v1 = (Q)0, v2 = (Q)0;
    int i1 = -1, i2 = -1;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const int r = 6 + m;
        const int i = m >> 2, s = m & 3;
        const Q au = (s == 0) ? U[2 * i] : (s == 1) ? -U[2 * i] : (s == 2) ? U[2 * i + 1] : -U[2 * i + 1];
        const Q vv = au - bb[m];
        const bool ok = i < N && !((act >> r) & 1u) && vv > c.tol_abs + c.tol_rel * fabs(bb[m]);
        if (m < 8) {
            if (ok && vv > v1) { v1 = vv; i1 = r; }
        } else {
            if (ok && vv > v2) { v2 = vv; i2 = r; }
        }
    }
    if (v1 > v0) { v0 = v1; i0 = i1; }
    if (v2 > v0) { v0 = v2; i0 = i2; }
    return i0;
}

// Whether any valid arena row is violated at u (the check of the common path: no argmax).
template <typename Q>
__device__ __forceinline__ bool arena_any(const Q (&bb)[16], const Q (&U)[8], int N,
                                          const QPConsts<Q>& c) {
    bool v = false;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        const int i = m >> 2, s = m & 3;
        const Q au = (s == 0) ? U[2 * i] : (s == 1) ? -U[2 * i] : (s == 2) ? U[2 * i + 1] : -U[2 * i + 1];
        v |= (i < N) & (au - bb[m] > c.tol_abs + c.tol_rel * fabs(bb[m]));
    }
    return v;
}

// Dense coefficients, bound and h (arena rows: +inf) of slot r: a pair row from the cached
// differences, an arena row from its bound.
template <typename Q>
__device__ __forceinline__ void team_row(const TRows<Q>& R, int r, Q (&a)[8], Q& b, Q& h, Q r2) {
#pragma unroll
    for (int m = 0; m < 8; ++m) a[m] = (Q)0;
    h = (Q)1e30;
    if (r < 6) {
        Q dx = 0, dy = 0, bp = 0;
#pragma unroll
        for (int s = 0; s < 6; ++s)
            if (s == r) { dx = R.dx[s]; dy = R.dy[s]; bp = R.bp[s]; }
        const int pa = (r < 3) ? 0 : (r < 5) ? 1 : 2;
        const int pb = (r < 3) ? r + 1 : (r < 5) ? r - 1 : 3;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            a[2 * m] = (m == pa) ? (Q)-2 * dx : ((m == pb) ? (Q)2 * dx : (Q)0);
            a[2 * m + 1] = (m == pa) ? (Q)-2 * dy : ((m == pb) ? (Q)2 * dy : (Q)0);
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

// The QP of one env from the team's all-gathered projected points Px, Py and nominal velocities
// U0, in every lane of the team (same operands, same branches).  overflow: the active set
// outgrew CAP rows (status 2; the caller re-solves).
template <int CAP>
__device__ __forceinline__ QPResult team_qp(const float (&Px)[4], const float (&Py)[4], int N,
                                            const float (&U0)[8], const QPConsts<float>& c,
                                            float (&U)[8], bool& overflow) {
    using Q = float;
    overflow = false;
    QPResult res;
    res.status = 0;
    res.q = 0;
    res.iters = 0;
    res.flag = false;
    TRows<Q> R;  // thr holds the pair rows' thresholds; bb the arena bounds once built
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        const int a = slot_a(r), b = slot_b(r);
        R.dx[r] = Px[a] - Px[b];
        R.dy[r] = Py[a] - Py[b];
        const Q h = R.dx[r] * R.dx[r] + R.dy[r] * R.dy[r] - c.r2;
        R.bp[r] = c.gamma * h * h * h;
        R.thr[r] = (b < N) ? c.tol_abs + c.tol_rel * fabsf(R.bp[r]) : CUDART_INF_F;
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) U[m] = U0[m];

    Q AR[CAP][8], lam[CAP], L[CAP * (CAP + 1) / 2], dinv[CAP];
    unsigned slots = 0u;  // slot of active row t in bits [5t, 5t + 5)
    unsigned hlow = 0u;   // bit t: active row t is a pair row with h below the re-solve flag
    unsigned act = 0u;
    int q = 0;
    Q vb;
    int r = pair_scan(R, U, act, vb);
    {
        // first row in closed form: u <- u - (v / |a|^2) a.  Every team runs it, a team with no
        // violated row as a zero step on slot 0 that it does not keep (the teams of a warp then
        // take no divergent branch here; measured faster on GB300 than a branch around it)
        const bool has = r >= 0;
        const int r0 = has ? r : 0;
        Q a[8], b, h;
        team_row(R, r0, a, b, h, c.r2);
        const Q app = tdot(a, a);
        const Q st = has ? __fdividef(vb, app) : (Q)0;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            U[m] -= st * a[m];
            AR[0][m] = a[m];
        }
        lam[0] = st;
        dinv[0] = rsqrtf(app);
        L[0] = app * dinv[0];
        hlow = (has && h < c.h_flag) ? 1u : 0u;
        slots = (unsigned)r0;
        act = has ? (1u << r0) : 0u;
        q = has ? 1 : 0;
        res.iters = has ? 1 : 0;
        r = pair_scan(R, U, act, vb);  // u is unchanged without a row: -1 again
    }
    bool all_rows = false;  // the arena rows are built and scanned
    for (;;) {
        while (r >= 0) {
            if (++res.iters > c.max_iter) { res.status = 2; break; }
            Q ap[8], bp, hp;
            team_row(R, r, ap, bp, hp, c.r2);
            const Q app = tdot(ap, ap);
            Q lam_p = (Q)0;
            bool added = false;
            if (q == 1) {
                // the common second row, written out (scalar Cholesky solves); taken when the
                // full primal step is feasible, else the general pass below
                const Q y0 = tdot(AR[0], ap) * dinv[0];
                const Q r0 = y0 * dinv[0];
                Q z[8];
#pragma unroll
                for (int m = 0; m < 8; ++m) z[m] = ap[m] - r0 * AR[0][m];
                const Q zz = tdot(z, z);
                const Q td = r0 > kTinyPos ? __fdividef(lam[0], r0) : CUDART_INF_F;
                const Q tf = __fdividef(tdot(ap, U) - bp, zz);
                if (zz > c.eps_dep * app && tf <= td) {
#pragma unroll
                    for (int m = 0; m < 8; ++m) {
                        U[m] -= tf * z[m];
                        AR[1][m] = ap[m];
                    }
                    lam[0] -= tf * r0;
                    dinv[1] = rsqrtf(zz);
                    L[1] = y0;
                    L[2] = zz * dinv[1];
                    lam[1] = tf;
                    hlow |= (hp < c.h_flag) ? 2u : 0u;
                    slots |= (unsigned)r << 5;
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
                Q td = CUDART_INF_F;
                int jb = -1;
#pragma unroll
                for (int t = 0; t < CAP; ++t)
                    if (t < q && rr[t] > kTinyPos) {
                        const Q tj = __fdividef(lam[t], rr[t]);
                        if (tj < td) { td = tj; jb = t; }
                    }
                const Q sp = tdot(ap, U) - bp;
                const bool indep = zz > c.eps_dep * app;
                if (!indep) res.flag = true;
                const Q tf = indep ? __fdividef(sp, zz) : CUDART_INF_F;
                if (!(tf < CUDART_INF_F) && !(td < CUDART_INF_F)) {
                    res.status = 1;
                    break;
                }
                const Q st = tf < td ? tf : td;
                if (tf < CUDART_INF_F) {
#pragma unroll
                    for (int m = 0; m < 8; ++m) U[m] -= st * z[m];
                }
#pragma unroll
                for (int t = 0; t < CAP; ++t)
                    if (t < q) lam[t] -= st * rr[t];
                lam_p += st;
                if (tf <= td) {
                    if (q == CAP) { overflow = true; break; }
                    const Q di = rsqrtf(zz);
#pragma unroll
                    for (int t = 0; t < CAP; ++t) {
                        if (t == q) {
#pragma unroll
                            for (int m = 0; m < t; ++m) L[ttri(t, m)] = y[m];
                            L[ttri(t, t)] = zz * di;
                            dinv[t] = di;
#pragma unroll
                            for (int m = 0; m < 8; ++m) AR[t][m] = ap[m];
                            lam[t] = lam_p;
                        }
                    }
                    hlow |= (hp < c.h_flag) ? (1u << q) : 0u;
                    slots |= (unsigned)r << (5 * q);
                    act |= 1u << r;
                    ++q;
                    added = true;
                } else {
                    const int js = (int)((slots >> (5 * jb)) & 31u);
                    act &= ~(1u << js);
                    {
                        const unsigned lo5 = (1u << (5 * jb)) - 1u, lo1 = (1u << jb) - 1u;
                        slots = (slots & lo5) | ((slots >> 5) & ~lo5);
                        hlow = (hlow & lo1) | ((hlow >> 1) & ~lo1);
                    }
#pragma unroll
                    for (int t = 0; t < CAP - 1; ++t)
                        if (t >= jb) {
#pragma unroll
                            for (int m = 0; m < 8; ++m) AR[t][m] = AR[t + 1][m];
                            lam[t] = lam[t + 1];
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
                                    const Q gp = g > (Q)1e-30 ? g : (Q)1e-30;
                                    dinv[t] = rsqrtf(gp);
                                    L[ttri(t, t)] = gp * dinv[t];
                                } else {
                                    L[ttri(t, m)] = g * dinv[m];
                                }
                            }
                        }
                    if (!ok) { res.status = 2; break; }
                }
            }
            if (res.status != 0) break;
            if (overflow) { res.status = 2; break; }  // more active rows than registers
            if (!added) { res.status = 2; break; }
            r = pair_scan(R, U, act, vb);
            if (all_rows) r = arena_scan(R.bb, U, act, N, c, vb, r);
        }
        if (all_rows) break;
        // the pair rows' minimiser (the envs of a warp meet here): the arena rows, once
        if (res.status != 0) break;
        all_rows = true;
#pragma unroll
        for (int m = 0; m < 16; ++m) R.bb[m] = arena_bound(c, m & 3, Px[m >> 2], Py[m >> 2]);
        if (!arena_any(R.bb, U, N, c)) break;
        vb = (Q)0;
        r = arena_scan(R.bb, U, act, N, c, vb, -1);
        if (r < 0) break;
    }
    res.q = q;
    if (res.status == 0) {
        if (hlow & ((1u << q) - 1u)) res.flag = true;  // near-degenerate pair row
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
