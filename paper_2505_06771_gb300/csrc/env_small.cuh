// env_small.cuh -- the step for environments of at most 4 robots (binary32), register-resident.
//
// Same method and same results (up to rounding) as run_env in env_step.cuh, specialised for the
// 4-robot class: a team of 4 lanes, lane i owning robot i, pose and heading in registers for the
// whole launch.  After the nominal velocities are formed the team all-gathers the projected
// points and nominal velocities with warp shuffles; the barrier rows are evaluated in registers
// (lane i takes its circulant pair rows and its four arena rows) and reduced with shuffles.
// Most QPs end with no active row or exactly one; the dual active-set method's first iteration
// is then the closed-form projection onto that row's half-plane, confirmed by a second scan.
// Only when a second row is violated does the team hand the QP to the general shared-memory
// solver.  Rare work -- the auto-reset sampler and the binary64 re-solve of a flagged QP --
// also goes through the shared-memory code of env_step.cuh.
#pragma once
#include "env_step.cuh"
#include "qp_regs.cuh"
#include "qp_team.cuh"
#include "qp_warp.cuh"

namespace rl {

template <typename T>
__device__ __forceinline__ T pick4(const T (&a)[4], int k) {
    T r = a[0];
    if (k == 1) r = a[1];
    if (k == 2) r = a[2];
    if (k == 3) r = a[3];
    return r;
}

constexpr int kRegRows = 4;  // active rows the register solver holds (more: shared memory)

// One barrier row: coefficient (cx, cy) on u_a and, for a pair row (b >= 0), (-cx, -cy) on u_b;
// bound bv; key = row index * 4 + the lane that evaluates it (ties order by row index).
struct RowD {
    int a, b, key;
    float cx, cy, bv;
};

__device__ __forceinline__ void own_coef(const RowD& r, int i, float& ox, float& oy) {
    ox = (i == r.a) ? r.cx : ((i == r.b) ? -r.cx : 0.f);
    oy = (i == r.a) ? r.cy : ((i == r.b) ? -r.cy : 0.f);
}

__device__ __forceinline__ float rowdot(const RowD& r1, const RowD& r2) {
    return row_dot<float>(r1.a, r1.b, r1.cx, r1.cy, r2.a, r2.b, r2.cx, r2.cy);
}

__device__ __forceinline__ RowD bcast_row(const Team<4>& tm, const RowD& r, int src) {
    RowD o;
    o.a = __shfl_sync(tm.mask, r.a, src, 4);
    o.b = __shfl_sync(tm.mask, r.b, src, 4);
    o.key = __shfl_sync(tm.mask, r.key, src, 4);
    o.cx = __shfl_sync(tm.mask, r.cx, src, 4);
    o.cy = __shfl_sync(tm.mask, r.cy, src, 4);
    o.bv = __shfl_sync(tm.mask, r.bv, src, 4);
    return o;
}

// The lane's own rows for one QP: its circulant pair rows with robots jd[0] (offset 1) and
// jd[1] (offset 2) -- key, orientation, p_a - p_b, bound -- and its four arena rows' bounds.
struct OwnRows {
    int pkey[2], bkey[4], pa[2];
    float sgn[2], dx[2], dy[2], bp[2], bb[4];
    int npair;
};

__device__ __forceinline__ void own_rows(int i, int N, int P, int ndi, const int (&jd)[2],
                                         float px, float py, const float (&qx)[2],
                                         const float (&qy)[2], const QPConsts<float>& c,
                                         OwnRows& R) {
    R.npair = (i < N) ? ndi : 0;
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        const int j = jd[d];
        const int a = min(i, j), b = max(i, j);
        R.pa[d] = j;
        R.pkey[d] = pair_index(a, b, N) * 4 + i;
        R.sgn[d] = (a == i) ? 1.f : -1.f;
        R.dx[d] = R.sgn[d] * (px - qx[d]);
        R.dy[d] = R.sgn[d] * (py - qy[d]);
        const float h = R.dx[d] * R.dx[d] + R.dy[d] * R.dy[d] - c.r2;
        R.bp[d] = c.gamma * h * h * h;
    }
    const float bx0 = c.xmax - c.half_r - px, bx1 = px - c.xmin - c.half_r;
    const float by0 = c.ymax - c.half_r - py, by1 = py - c.ymin - c.half_r;
    R.bb[0] = c.kg * bx0 * bx0 * bx0;
    R.bb[1] = c.kg * bx1 * bx1 * bx1;
    R.bb[2] = c.kg * by0 * by0 * by0;
    R.bb[3] = c.kg * by1 * by1 * by1;
#pragma unroll
    for (int s = 0; s < 4; ++s) R.bkey[s] = (P + 4 * i + s) * 4 + i;
}

// Most violated inactive row over the team at u (own ux, uy; the pair partners' nux, nuy),
// ties to the lowest row index; the lane owning the winner broadcasts its descriptor.
__device__ __forceinline__ void small_scan(const Team<4>& tm, int i, int N, const OwnRows& R,
                                           float ux, float uy, const float (&nux)[2],
                                           const float (&nuy)[2], const QPConsts<float>& c,
                                           const int (&akey)[kRegRows], int q, float& vb,
                                           RowD& win) {
    vb = 0.f;
    RowD best;
    best.a = best.b = -1;
    best.key = 0x7fffffff;
    best.cx = best.cy = best.bv = 0.f;
    if (i < N) {
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            bool act = false;
#pragma unroll
            for (int t = 0; t < kRegRows; ++t) act |= (t < q && akey[t] == R.pkey[d]);
            const float dux = R.sgn[d] * (ux - nux[d]), duy = R.sgn[d] * (uy - nuy[d]);
            const float v = -2.f * (R.dx[d] * dux + R.dy[d] * duy) - R.bp[d];
            if (d < R.npair && !act && v > c.tol_abs + c.tol_rel * fabsf(R.bp[d]) &&
                (v > vb || (v == vb && R.pkey[d] < best.key))) {
                vb = v;
                best.key = R.pkey[d];
                best.cx = -2.f * R.dx[d];
                best.cy = -2.f * R.dy[d];
                best.bv = R.bp[d];
                best.a = min(i, R.pa[d]);
                best.b = max(i, R.pa[d]);
            }
        }
        const float aus[4] = {ux, -ux, uy, -uy};
        const float cxs[4] = {1.f, -1.f, 0.f, 0.f}, cys[4] = {0.f, 0.f, 1.f, -1.f};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            bool act = false;
#pragma unroll
            for (int t = 0; t < kRegRows; ++t) act |= (t < q && akey[t] == R.bkey[s]);
            const float v = aus[s] - R.bb[s];
            if (!act && v > c.tol_abs + c.tol_rel * fabsf(R.bb[s]) &&
                (v > vb || (v == vb && R.bkey[s] < best.key))) {
                vb = v;
                best.a = i; best.b = -1; best.key = R.bkey[s];
                best.cx = cxs[s]; best.cy = cys[s]; best.bv = R.bb[s];
            }
        }
    }
    int kb = best.key;
    tm.argmax(vb, kb);
    if (kb == 0x7fffffff) {
        win.key = kb;
        return;
    }
    win = bcast_row(tm, best, kb & 3);
}

__device__ __forceinline__ int ltri(int i, int k) { return i * (i + 1) / 2 + k; }

// General shared-memory solver for the QPs whose active set outgrows the register solver (out
// of line, so the hot loop stays small).
static __device__ __noinline__ QPResult small_general(const Team<4> tm, TeamSmem<float, 4>& S, int N,
                                               float px, float py, float u0x, float u0y,
                                               const QPConsts<float> c) {
    QPWork<float, 4>& W = S.qp.s.f;
    const int i = tm.lane;
    if (i < N) {
        W.px[i] = px;
        W.py[i] = py;
        W.u0x[i] = W.ux[i] = u0x;
        W.u0y[i] = W.uy[i] = u0y;
    }
    tm.sync();
    return qp_solve<float, 4, 4>(tm, W, N, c);  // the minimiser is left in W.ux / W.uy
}

// The barrier QP of one env of N <= 4 robots; (usx, usy) receives the lane's own robot's
// filtered velocity.  The dual active-set method runs with u distributed over the lanes (lane i
// holds u_i), the active rows' descriptors, multipliers and Cholesky factor replicated in
// registers (at most kRegRows rows), dot products over u as team sums.  The first iteration is
// the closed-form projection onto the first row's half-plane: its violation is the scan's
// maximum and |a|^2 is known.  A larger active set goes to the shared-memory solver.
__device__ __forceinline__ QPResult small_filter(const Team<4>& tm, TeamSmem<float, 4>& S, int N,
                                                 const int (&jd)[2], int ndi, float px,
                                                 float py, float u0x, float u0y,
                                                 const QPConsts<float>& c, float& usx,
                                                 float& usy) {
    QPResult res;
    res.status = 0;
    res.q = 0;
    res.iters = 0;
    res.flag = false;
    const int i = tm.lane;
    const int P = N * (N - 1) / 2;
    float qx[2], qy[2], nux[2], nuy[2];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        qx[d] = __shfl_sync(tm.mask, px, jd[d], 4);
        qy[d] = __shfl_sync(tm.mask, py, jd[d], 4);
        nux[d] = __shfl_sync(tm.mask, u0x, jd[d], 4);
        nuy[d] = __shfl_sync(tm.mask, u0y, jd[d], 4);
    }
    OwnRows R;
    own_rows(i, N, P, ndi, jd, px, py, qx, qy, c, R);
    float ux = u0x, uy = u0y;
    int akey[kRegRows];
#pragma unroll
    for (int t = 0; t < kRegRows; ++t) akey[t] = -1;
    float vb;
    RowD p;
    small_scan(tm, i, N, R, ux, uy, nux, nuy, c, akey, 0, vb, p);
    usx = ux;
    usy = uy;
    if (p.key == 0x7fffffff) return res;

    // first iteration, closed form: u <- u - (v / |a|^2) a
    RowD A[kRegRows];
    float lam[kRegRows], L[kRegRows * (kRegRows + 1) / 2], dinv[kRegRows];
    {
        const float app = (p.b >= 0 ? 2.f : 1.f) * (p.cx * p.cx + p.cy * p.cy);
        const float st = vb / app;
        float ox, oy;
        own_coef(p, i, ox, oy);
        ux -= st * ox;
        uy -= st * oy;
#pragma unroll
        for (int d = 0; d < 2; ++d) {  // the partners' u change the same way: no re-fetch
            own_coef(p, jd[d], ox, oy);
            nux[d] -= st * ox;
            nuy[d] -= st * oy;
        }
        A[0] = p;
        akey[0] = p.key;
        lam[0] = st;
        L[0] = sqrtf(app);
        dinv[0] = 1.f / L[0];
    }
    int q = 1;
    res.iters = 1;
    small_scan(tm, i, N, R, ux, uy, nux, nuy, c, akey, q, vb, p);
    bool overflow = false;
    while (p.key != 0x7fffffff) {
        if (++res.iters > c.max_iter) { res.status = 2; break; }
        const float app = (p.b >= 0 ? 2.f : 1.f) * (p.cx * p.cx + p.cy * p.cy);
        float pox, poy;
        own_coef(p, i, pox, poy);
        float lam_p = 0.f;
        bool added = false;
        for (int guard = 0; guard <= kRegRows + 1 && !added; ++guard) {
            // r = G^-1 N^T a_p, z = a_p - N r (own robot's two components)
            float y[kRegRows], r[kRegRows];
#pragma unroll
            for (int t = 0; t < kRegRows; ++t) {
                y[t] = 0.f;
                if (t < q) {
                    float s = rowdot(A[t], p);
#pragma unroll
                    for (int m = 0; m < t; ++m) s -= L[ltri(t, m)] * y[m];
                    y[t] = s * dinv[t];
                }
            }
#pragma unroll
            for (int t = kRegRows - 1; t >= 0; --t) {
                r[t] = 0.f;
                if (t < q) {
                    float s = y[t];
#pragma unroll
                    for (int m = t + 1; m < kRegRows; ++m)
                        if (m < q) s -= L[ltri(m, t)] * r[m];
                    r[t] = s * dinv[t];
                }
            }
            float zx = pox, zy = poy;
#pragma unroll
            for (int t = 0; t < kRegRows; ++t)
                if (t < q) {
                    float ox, oy;
                    own_coef(A[t], i, ox, oy);
                    zx -= r[t] * ox;
                    zy -= r[t] * oy;
                }
            const float zz = tm.sum(zx * zx + zy * zy);
            float td = CUDART_INF_F;
            int jb = -1;
#pragma unroll
            for (int t = 0; t < kRegRows; ++t)
                if (t < q && r[t] > 0.f) {
                    const float tj = lam[t] / r[t];
                    if (tj < td) { td = tj; jb = t; }
                }
            const float sp = tm.sum(pox * ux + poy * uy) - p.bv;
            const bool indep = zz > c.eps_dep * app;
            if (!indep) res.flag = true;
            const float tf = indep ? sp / zz : CUDART_INF_F;
            if (!(tf < CUDART_INF_F) && !(td < CUDART_INF_F)) {
                res.status = 1;
                break;
            }
            const float st = tf < td ? tf : td;
            if (tf < CUDART_INF_F) {
                ux -= st * zx;
                uy -= st * zy;
            }
#pragma unroll
            for (int t = 0; t < kRegRows; ++t)
                if (t < q) lam[t] -= st * r[t];
            lam_p += st;
            if (tf <= td) {
                if (q == kRegRows) { overflow = true; break; }
                const float dg = sqrtf(zz);
#pragma unroll
                for (int t = 0; t < kRegRows; ++t) {
                    if (t == q) {
#pragma unroll
                        for (int m = 0; m < t; ++m) L[ltri(t, m)] = y[m];
                        L[ltri(t, t)] = dg;
                        dinv[t] = 1.f / dg;
                        A[t] = p;
                        akey[t] = p.key;
                        lam[t] = lam_p;
                    }
                }
                ++q;
                added = true;
            } else {
                // drop row jb and refactor the Gram matrix of the remaining rows
#pragma unroll
                for (int t = 0; t < kRegRows - 1; ++t)
                    if (t >= jb) {
                        A[t] = A[t + 1];
                        akey[t] = akey[t + 1];
                        lam[t] = lam[t + 1];
                    }
                --q;
#pragma unroll
                for (int t = 0; t < kRegRows; ++t)
                    if (t >= q) akey[t] = -1;
                bool ok = true;
#pragma unroll
                for (int t = 0; t < kRegRows; ++t)
                    if (t < q) {
#pragma unroll
                        for (int m = 0; m <= t; ++m) {
                            float g = rowdot(A[t], A[m]);
#pragma unroll
                            for (int n = 0; n < m; ++n) g -= L[ltri(t, n)] * L[ltri(m, n)];
                            if (m == t) {
                                ok = ok && (g > 0.f);
                                const float dg = sqrtf(fmaxf(g, 1e-30f));
                                L[ltri(t, t)] = dg;
                                dinv[t] = 1.f / dg;
                            } else {
                                L[ltri(t, m)] = g * dinv[m];
                            }
                        }
                    }
                if (!ok) { res.status = 2; break; }
            }
        }
        if (res.status != 0 || overflow) break;
        if (!added) { res.status = 2; break; }
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            nux[d] = __shfl_sync(tm.mask, ux, jd[d], 4);
            nuy[d] = __shfl_sync(tm.mask, uy, jd[d], 4);
        }
        small_scan(tm, i, N, R, ux, uy, nux, nuy, c, akey, q, vb, p);
    }
    if (overflow) {
        res = small_general(tm, S, N, px, py, u0x, u0y, c);
        usx = (i < N) ? S.qp.s.f.ux[i] : 0.f;
        usy = (i < N) ? S.qp.s.f.uy[i] : 0.f;
        tm.sync();
        return res;
    }
    res.q = q;
    if (res.status == 0) {
#pragma unroll
        for (int t = 0; t < kRegRows; ++t)
            if (t < q && A[t].b >= 0 &&
                0.25f * (A[t].cx * A[t].cx + A[t].cy * A[t].cy) - c.r2 < c.h_flag)
                res.flag = true;  // near-degenerate pair row
    } else {
        res.flag = true;
        if (res.status == 1) { ux = 0.f; uy = 0.f; }
    }
    usx = ux;
    usy = uy;
    return res;
}

// The barrier QP of one env of N <= 4 robots, solved redundantly by every lane of the team.
// One round of shuffles all-gathers the projected points and nominal velocities; then each lane
// runs the register dual active-set solver (team_qp: pair rows first, then the arena rows
// checked once; closed-form first iteration) on the whole 8-variable QP, with no cross-lane
// traffic inside the solve, and keeps its own robot's u.  Every lane takes the same branches,
// so the team never diverges; an active set beyond kTeamRows rows goes to the shared-memory
// solver.  defer: an active set beyond kTeamRows rows is not solved here but returned as
// status 3 (the caller hands it to the whole warp).
__device__ __forceinline__ QPResult small_filter_all(const Team<4>& tm, TeamSmem<float, 4>& S,
                                                     int N, float px, float py, float u0x,
                                                     float u0y, const QPConsts<float>& c,
                                                     float& usx, float& usy, bool defer = false) {
    float Px[4], Py[4], U0[8], U[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        Px[j] = __shfl_sync(tm.mask, px, j, 4);
        Py[j] = __shfl_sync(tm.mask, py, j, 4);
        U0[2 * j] = __shfl_sync(tm.mask, u0x, j, 4);
        U0[2 * j + 1] = __shfl_sync(tm.mask, u0y, j, 4);
    }
    bool overflow;
    QPResult res = team_qp<kTeamRows>(Px, Py, N, U0, c, U, overflow);
    if (overflow && defer) {
        res.status = 3;
        usx = u0x;
        usy = u0y;
        return res;
    }
    if (overflow) {
        res = small_general(tm, S, N, px, py, u0x, u0y, c);
        const int i = tm.lane;
        usx = (i < N) ? S.qp.s.f.ux[i] : 0.f;
        usy = (i < N) ? S.qp.s.f.uy[i] : 0.f;
        tm.sync();
        return res;
    }
    const int i = tm.lane;
    usx = (i == 0) ? U[0] : (i == 1) ? U[2] : (i == 2) ? U[4] : U[6];
    usy = (i == 0) ? U[1] : (i == 1) ? U[3] : (i == 2) ? U[5] : U[7];
    return res;
}

// binary64 re-solve of a flagged QP by the team, through the shared-memory solver.
static __device__ __noinline__ QPResult small_resolve_f64(const Team<4> tm, TeamSmem<float, 4>& S,
                                                   const StepConsts<float> k, int N, float x,
                                                   float y, float th, float u0x, float u0y) {
    QPWork<double, 4>& D = S.qp.d;
    QPConsts<double> dc;
    dc.gamma = (double)k.gamma; dc.r2 = (double)k.r2; dc.kg = (double)k.kg;
    dc.half_r = (double)k.half_r; dc.xmin = (double)k.xmin; dc.xmax = (double)k.xmax;
    dc.ymin = (double)k.ymin; dc.ymax = (double)k.ymax; dc.h_flag = (double)k.h_flag;
    dc.max_iter = 8 * 4 + 16;
    dc.tol_abs = 1e-12; dc.tol_rel = 1e-12; dc.eps_dep = 1e-12; dc.tol_lam = 1e-10;
    const int i = tm.lane;
    if (i < N) {
        double sd, cd;
        sincos((double)th, &sd, &cd);
        D.px[i] = (double)x + (double)k.l * cd;
        D.py[i] = (double)y + (double)k.l * sd;
        D.u0x[i] = (double)u0x;
        D.u0y[i] = (double)u0y;
        D.ux[i] = D.u0x[i];
        D.uy[i] = D.u0y[i];
    }
    tm.sync();
    return qp_solve<double, 4, 4>(tm, D, N, dc);  // the minimiser is left in D.ux / D.uy
}

// Auto-reset: samples episode ep into S.fx/fy/fth (poses), S.sx/sy/sth (goal positions and
// headings), S.slevel (levels) and the resources; returns the resource count.
static __device__ __noinline__ int small_reset(const Team<4> tm, TeamSmem<float, 4>& S,
                                        const LaunchArgs<float> A, int e, int ep, int N) {
    int n_res = 0;
    team_sample<float, 4, 4>(tm, S, A, e, ep, N, n_res);
    const int i = tm.lane;
    if (i < N) {
        float gx, gy, gth;
        int lv;
        robot_goal_level<float>(A, e, ep, i, gx, gy, gth, lv);
        S.sx[i] = gx;
        S.sy[i] = gy;
        S.sth[i] = gth;
        S.slevel[i] = lv;
    }
    tm.sync();
    return n_res;
}

__device__ __forceinline__ float wrap_pi_f(float a) {
    a = (a > CUDART_PI_F) ? a - 2.f * CUDART_PI_F : a;
    return (a <= -CUDART_PI_F) ? a + 2.f * CUDART_PI_F : a;
}

// |(a, b)| through the reciprocal square root (relative error a few 1e-7).
__device__ __forceinline__ float fast_norm(float a, float b) {
    const float n2 = a * a + b * b;
    return n2 > 0.f ? n2 * rsqrtf(n2) : 0.f;
}

// |u| <= m by scaling, without a branch: s = min(1, m / |u|).
__device__ __forceinline__ void cap_fast(float& ux, float& uy, float m) {
    const float s = fminf(1.f, m * rsqrtf(ux * ux + uy * uy));
    ux *= s;
    uy *= s;
}

// Out-of-line rare paths of the foraging scenario.
static __device__ __noinline__ void small_forage_target(const TeamSmem<float, 4>& S, int n_res, float px,
                                                 float py, float& tx, float& ty) {
    int best = -1;
    float bd = 0.f;
    for (int r = 0; r < n_res; ++r) {
        if (!S.qactive[r]) continue;
        const float dx = S.qx[r] - px, dy = S.qy[r] - py;
        const float d2 = dx * dx + dy * dy;
        if (best < 0 || d2 < bd) { best = r; bd = d2; }
    }
    if (best >= 0) { tx = S.qx[best]; ty = S.qy[best]; }
    else { tx = px; ty = py; }
}

static __device__ __noinline__ void small_forage_obs(const TeamSmem<float, 4>& S, const StepConsts<float> k,
                                              float* o, int i, int N, int n_res, float x, float y,
                                              float th, int lv, const float (&X)[4],
                                              const float (&Y)[4], const float (&TH)[4],
                                              const int (&LV)[4]) {
    o[0] = x; o[1] = y; o[2] = th; o[3] = (float)lv;
    int c = 4;
    for (int j = 0; j < N; ++j) {
        if (j == i) continue;
        o[c] = pick4(X, j) - x;
        o[c + 1] = pick4(Y, j) - y;
        o[c + 2] = wrap_pi_f(pick4(TH, j) - th);
        o[c + 3] = (float)pick4(LV, j);
        c += 4;
    }
    const int rbase = 4 + 4 * (k.n_max_obs - 1);
    for (; c < rbase; ++c) o[c] = 0.f;
    for (int r = 0; r < k.r_max; ++r) {
        if (r < n_res) {
            o[c] = S.qx[r] - x;
            o[c + 1] = S.qy[r] - y;
            o[c + 2] = (float)S.qlevel[r];
            o[c + 3] = (float)S.qactive[r];
        } else {
            o[c] = o[c + 1] = o[c + 2] = o[c + 3] = 0.f;
        }
        c += 4;
    }
}

// Discovery observation of robot i: own pose and capability, the others' relative poses and
// capabilities, the landmarks (relative position, sensed, tagged; a stand-in point outside the
// arena while unsensed).
static __device__ __noinline__ void small_disc_obs(const TeamSmem<float, 4>& S, const StepConsts<float> k,
                                            float* o, int i, int N, int n_res, float x, float y,
                                            float th, int lv, const float (&X)[4],
                                            const float (&Y)[4], const float (&TH)[4],
                                            const int (&LV)[4]) {
    o[0] = x; o[1] = y; o[2] = th;
    o[3] = lv == 1 ? k.sense_r : 0.f;
    o[4] = lv == 2 ? k.tag_r : 0.f;
    int c = 5;
    for (int j = 0; j < N; ++j) {
        if (j == i) continue;
        const int lj = pick4(LV, j);
        o[c] = pick4(X, j) - x;
        o[c + 1] = pick4(Y, j) - y;
        o[c + 2] = wrap_pi_f(pick4(TH, j) - th);
        o[c + 3] = lj == 1 ? k.sense_r : 0.f;
        o[c + 4] = lj == 2 ? k.tag_r : 0.f;
        c += 5;
    }
    const int rbase = 5 + 5 * (k.n_max_obs - 1);
    for (; c < rbase; ++c) o[c] = 0.f;
    for (int r = 0; r < k.r_max; ++r) {
        if (r < n_res && S.qlevel[r]) {
            o[c] = S.qx[r] - x;
            o[c + 1] = S.qy[r] - y;
            o[c + 2] = 1.f;
            o[c + 3] = S.qactive[r] ? 0.f : 1.f;
        } else if (r < n_res) {
            o[c] = k.xo - x;
            o[c + 1] = k.yo - y;
            o[c + 2] = o[c + 3] = 0.f;
        } else {
            o[c] = o[c + 1] = o[c + 2] = o[c + 3] = 0.f;
        }
        c += 4;
    }
}

// One env of at most 4 robots for T steps (team of 4 lanes).  FAST: the Navigation scenario with
// scripted nominal control and no traces, every such branch folded away at compile time.
// SCEN >= 0 fixes the scenario at compile time and LEAN drops policy actions and traces (the
// one-launch kernel's scripted rollouts).
// wm (scripted Navigation): the lanes of the warp's live teams, all running the same steps in
// step with each other, when there are at least two; the rare QPs (an active set beyond the
// register solver's, the binary64 re-solve) are then solved by the whole warp (qp_warp.cuh).
// 0: each team solves its own in shared memory.  (The general kernel keeps the team solvers:
// measured on GB300, the warp path's code slowed its common path by about 2%.)
template <bool FAST, int SCEN = -1, bool LEAN = false>
__device__ void run_env_small(const LaunchArgs<float>& A, const Team<4>& tm,
                              TeamSmem<float, 4>& S, int e, unsigned wm = 0u) {
    const StepConsts<float>& k = A.k;
    const int off = A.s.off[e];
    const int N = A.s.nrob[e];
    const bool forage = !FAST && ((SCEN < 0) ? (k.scenario == 1) : (SCEN == 1));
    const bool disc = !FAST && ((SCEN < 0) ? (k.scenario == 2) : (SCEN == 2));
    const bool resv = forage || disc;  // per-env resources / landmarks
    const float* actions = (FAST || LEAN) ? nullptr : A.io.actions;
    float* tr_unom = (FAST || LEAN) ? nullptr : A.io.u_nom;
    float* tr_ustar = (FAST || LEAN) ? nullptr : A.io.u_star;
    float* tr_vw = (FAST || LEAN) ? nullptr : A.io.vw;
    int32_t* tr_qp = (FAST || LEAN) ? nullptr : A.io.qp_info;
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
    int lv = A.s.level[row];
    float sn, cs;
    __sincosf(th, &sn, &cs);
    int t = A.s.t[e], ep = A.s.ep[e];
    int n_res = 0;
    if (resv) {
        n_res = A.s.n_res[e];
        for (int r = i; r < k.r_max; r += 4) {
            S.qx[r] = A.s.qx[e * k.r_max + r];
            S.qy[r] = A.s.qy[e * k.r_max + r];
            S.qlevel[r] = A.s.qlevel[e * k.r_max + r];
            S.qactive[r] = A.s.qactive[e * k.r_max + r];
        }
    }
    // counters, kept by lane 0
    int c_col = 0, c_oob = 0, c_succ = 0, c_act = 0, c_flag = 0, c_inf = 0, c_ep = 0, c_it = 0;
    tm.sync();
    const int nd = (N - 1) / 2;
    const int ndi = own ? nd + (((N & 1) == 0 && i < N / 2) ? 1 : 0) : 0;
    int jn[2];  // the robots of the lane's circulant pair rows (offsets 1 and 2)
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        int j = i + d + 1;
        while (j >= N) j -= N;
        jn[d] = own ? j : i;
    }
    const float* acts = actions;
    float ret_acc = 0.f;
    int nz_t = -2, nz_ep = -1;   // noise words cached for step nz_t + 1 of episode nz_ep
    uint32_t nz_nx = 0u, nz_ny = 0u;

    for (int step = 0; step < A.T; ++step) {
        // ---- projected point and nominal SI velocity of the own robot
        const float px = x + k.l * cs, py = y + k.l * sn;
        float ux, uy;
        if (!FAST && acts) {
            ux = acts[2 * row];
            uy = acts[2 * row + 1];
            screen_action(A.io.status, ux, uy);
        } else {
            float tx = gx, ty = gy;
            if (forage) small_forage_target(S, n_res, px, py, tx, ty);
            if (disc && !discovery_target<float>(S.qx, S.qy, S.qlevel, S.qactive, n_res, lv, px, py,
                                                 tx, ty)) {
                tx = px;
                ty = py;
            }
            if (!FAST && !resv && k.controller == 1) {
                pose_nominal<float>(k, x, y, th, gx, gy, gth, ux, uy);
            } else {
                ux = k.k_si * (tx - px);
                uy = k.k_si * (ty - py);
            }
            cap_fast(ux, uy, k.vmax);
            // Noise words of this robot for step t.  Robots 2m and 2m+1 share the Philox block
            // (pair m, step t); their two lanes compute the blocks of steps t and t+1 at once
            // and swap them, so each lane runs Philox every other step.
            uint32_t wx, wy;
            if (nz_ep == ep && nz_t + 1 == t) {
                wx = nz_nx;
                wy = nz_ny;
                nz_t = -2;
            } else {
                const Words4 w = draw(A.seed, e, ep, kNoise, i >> 1, (uint32_t)(t + (i & 1)));
                uint32_t o[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) o[m] = __shfl_xor_sync(tm.mask, w.w[m], 1, 4);
                // block of step t: the even lane's; of step t+1: the odd lane's
                wx = (i & 1) ? o[2] : w.w[0];
                wy = (i & 1) ? o[3] : w.w[1];
                nz_nx = (i & 1) ? w.w[2] : o[0];
                nz_ny = (i & 1) ? w.w[3] : o[1];
                nz_t = t;
                nz_ep = ep;
            }
            const float ex = __fmul_rn(__fsub_rn(unit24(wx), 0.5f), k.noise_scale);
            const float ey = __fmul_rn(__fsub_rn(unit24(wy), 0.5f), k.noise_scale);
            ux += k.noise_on ? ex : 0.f;
            uy += k.noise_on ? ey : 0.f;
        }
        cap_fast(ux, uy, k.vmax);
        const float dold = fast_norm(px - gx, py - gy);
        // ---- the barrier QP
        float usx, usy;
        const bool by_warp = FAST && wm != 0u;
        QPResult res = small_filter_all(tm, S, N, px, py, ux, uy, qc, usx, usy, by_warp);
        int qflags = (res.q > 0 || res.status != 0) ? 1 : 0;
        // rare QPs of the warp's envs (one vote when there are none), one env at a time by all
        // live lanes
        if (by_warp && __ballot_sync(wm, i == 0 && (res.status == 3 || (k.resolve_f64 && res.flag)))) {
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
                // binary64: projected points from the binary32 pose (the heading's sine and
                // cosine to binary32 accuracy, a few 1e-9 m at the look-ahead distance)
                float sf, cf;
                sincosf(th, &sf, &cf);
                const double pxd = (double)x + (double)k.l * (double)cf;
                const double pyd = (double)y + (double)k.l * (double)sf;
                QPConsts<double> dc;
                dc.gamma = (double)k.gamma; dc.r2 = (double)k.r2; dc.kg = (double)k.kg;
                dc.half_r = (double)k.half_r; dc.xmin = (double)k.xmin; dc.xmax = (double)k.xmax;
                dc.ymin = (double)k.ymin; dc.ymax = (double)k.ymax; dc.h_flag = (double)k.h_flag;
                dc.max_iter = 8 * 4 + 16;
                dc.tol_abs = 1e-12; dc.tol_rel = 1e-12; dc.eps_dep = 1e-12; dc.tol_lam = 1e-10;
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
                        qflags |= 2;
                    }
                }
            }
        } else if (!by_warp && k.resolve_f64 && res.flag) {
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
        float v = cs * usx + sn * usy;
        float om = (cs * usy - sn * usx) * k.inv_l;
        const float wr = fminf(fmaxf(v + k.half_track * om, -k.vmax), k.vmax);
        const float wl = fminf(fmaxf(v - k.half_track * om, -k.vmax), k.vmax);
        v = 0.5f * (wr + wl);
        om = (wr - wl) * k.inv_track;
        if (!FAST && own) {
            if (tr_unom) { tr_unom[2 * row] = ux; tr_unom[2 * row + 1] = uy; }
            if (tr_ustar) { tr_ustar[2 * row] = usx; tr_ustar[2 * row + 1] = usy; }
            if (tr_vw) { tr_vw[2 * row] = v; tr_vw[2 * row + 1] = om; }
        }
        x += k.dt * v * cs;
        y += k.dt * v * sn;
        th = wrap_pi_f(th + k.dt * om);
        __sincosf(th, &sn, &cs);
        const float npx = x + k.l * cs, npy = y + k.l * sn;
        // ---- flags, reward, scenario transition
        int flags_l = 0;  // collisions in the low half, out-of-arena in the high half
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            const float qx = __shfl_sync(tm.mask, npx, jn[d], 4);
            const float qy = __shfl_sync(tm.mask, npy, jn[d], 4);
            const float dx = npx - qx, dy = npy - qy;
            flags_l += (d < ndi && dx * dx + dy * dy < k.r2) ? 1 : 0;
        }
        flags_l += (own && (npx < k.xmin || npx > k.xmax || npy < k.ymin || npy > k.ymax)) ? 65536 : 0;
        // flags_l: collisions in bits 0..7, waypoint arrivals in 8..15, out-of-arena from 16
        float rew_l = (!resv && own) ? dold - fast_norm(npx - gx, npy - gy) : 0.f;
        if (!resv && k.waypoint && own) {
            const float ex = npx - gx, ey = npy - gy;
            if (ex * ex + ey * ey < k.goal_eps2) {
                const float3 g = waypoint_goal(A.sc, A.seed, e, ep, i, t + 1);
                gx = g.x;
                gy = g.y;
                gth = g.z;
                flags_l += 256;  // arrivals in bits 8..15
            }
        }
        const int flags = tm.sum(flags_l);
        float rew = tm.sum(rew_l);
        const int col = flags & 0xff, oob = flags >> 16;
        bool all_foraged = false;
        int succ = (flags >> 8) & 0xff;
        if (forage) {
            int remaining = 0;
            for (int r = 0; r < n_res; ++r) {
                if (!S.qactive[r]) continue;
                int ls = 0;
                if (own) {
                    const float dx = npx - S.qx[r], dy = npy - S.qy[r];
                    if (dx * dx + dy * dy < k.rho2) ls = lv;
                }
                ls = tm.sum(ls);
                if (ls >= S.qlevel[r]) {
                    rew += (float)S.qlevel[r];
                    ++succ;
                    tm.sync();
                    if (i == 0) S.qactive[r] = 0;
                    tm.sync();
                } else {
                    ++remaining;
                }
            }
            all_foraged = (n_res > 0 && remaining == 0);
        }
        if (disc) {
            // Discovery: sensing robots sense landmarks within their radius, tagging robots tag
            // sensed ones within theirs (in the same step too); a penalty while one is left
            int remaining = 0;
            for (int r = 0; r < n_res; ++r) {
                const float dx = npx - S.qx[r], dy = npy - S.qy[r];
                const float d2 = dx * dx + dy * dy;
                const bool hs = tm.any(own && lv == 1 && d2 < k.sense_r2);
                const bool ht = tm.any(own && lv == 2 && d2 < k.tag_r2);
                int sensed = S.qlevel[r], tagged = S.qactive[r] ? 0 : 1;
                if (!sensed && hs) { sensed = 1; rew += k.sense_rew; }
                if (sensed && !tagged && ht) { tagged = 1; rew += k.tag_rew; ++succ; }
                remaining += tagged ? 0 : 1;
                tm.sync();
                if (i == 0) { S.qlevel[r] = sensed; S.qactive[r] = tagged ? 0 : 1; }
                tm.sync();
            }
            if (remaining > 0) rew -= k.step_pen;
        }
        rew -= k.c_col * (float)col;
        c_col += col;
        c_oob += oob;
        c_succ += succ;
        c_act += qflags & 1;
        c_flag += (qflags >> 1) & 1;
        c_inf += (res.status == 1) ? 1 : 0;
        c_it += res.iters;
        if (!FAST && tr_qp && i == 0) {
            tr_qp[4 * e + 0] = res.status;
            tr_qp[4 * e + 1] = res.q;
            tr_qp[4 * e + 2] = res.iters;
            tr_qp[4 * e + 3] = qflags;
        }
        // ---- episode end and auto-reset
        t += 1;
        const bool done = (t >= k.episode_len) || all_foraged;
        if (done) {
            c_ep += 1;
            ep += 1;
            t = 0;
            n_res = small_reset(tm, S, A, e, ep, N);
            if (own) {
                x = S.fx[i]; y = S.fy[i]; th = S.fth[i];
                gx = S.sx[i]; gy = S.sy[i]; gth = S.sth[i]; lv = S.slevel[i];
            }
            tm.sync();
            __sincosf(th, &sn, &cs);
        }
        // ---- observations of the own robot
        if (A.io.obs) {
            const int od = A.io.obs_dim;
            float* o = A.io.obs + (long long)step * A.io.obs_step + (long long)row * od;
            if (!resv) {
                // others in index order: slot s holds robot s + (s >= i)
                float rel[9];
#pragma unroll
                for (int sl = 0; sl < 3; ++sl) {
                    const int j = sl + (sl >= i ? 1 : 0);
                    const bool live = j < N;
                    const float xj = __shfl_sync(tm.mask, x, j, 4);
                    const float yj = __shfl_sync(tm.mask, y, j, 4);
                    const float tj = __shfl_sync(tm.mask, th, j, 4);
                    rel[3 * sl] = live ? xj - x : 0.f;
                    rel[3 * sl + 1] = live ? yj - y : 0.f;
                    rel[3 * sl + 2] = live ? wrap_pi_f(tj - th) : 0.f;
                }
                if (own) {
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
            } else {
                float X[4], Y[4], TH[4];
                int LV[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    X[r] = __shfl_sync(tm.mask, x, r, 4);
                    Y[r] = __shfl_sync(tm.mask, y, r, 4);
                    TH[r] = __shfl_sync(tm.mask, th, r, 4);
                    LV[r] = __shfl_sync(tm.mask, lv, r, 4);
                }
                if (own && disc) small_disc_obs(S, k, o, i, N, n_res, x, y, th, lv, X, Y, TH, LV);
                else if (own) small_forage_obs(S, k, o, i, N, n_res, x, y, th, lv, X, Y, TH, LV);
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
    if (resv) {
        tm.sync();
        for (int r = i; r < k.r_max; r += 4) {
            A.s.qx[e * k.r_max + r] = S.qx[r];
            A.s.qy[e * k.r_max + r] = S.qy[r];
            A.s.qlevel[e * k.r_max + r] = S.qlevel[r];
            A.s.qactive[e * k.r_max + r] = S.qactive[r];
        }
    }
    if (i == 0) {
        A.s.t[e] = t;
        A.s.ep[e] = ep;
        if (resv) A.s.n_res[e] = n_res;
        int32_t* cn = A.s.counters + e * kNCount;
        cn[0] += c_col; cn[1] += c_oob; cn[2] += c_succ; cn[3] += c_act;
        cn[4] += c_flag; cn[5] += c_inf; cn[6] += c_ep; cn[7] += c_it;
    }
}

}  // namespace rl
