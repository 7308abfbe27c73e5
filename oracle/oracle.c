/*
 * oracle.c -- FP64 CPU oracle of the batched multi-robot environment step (JaxRobotarium,
 * arXiv 2505.06771).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, by the smoke check and by the benchmark's CPU
 * baseline leg; never by the product path.  Written from the paper's description of the
 * method; it shares no code with the CUDA library.
 *
 * What one step of one environment computes (paper Sec. 4.1 and Sec. 6.1, App. B):
 *   1. projected points p_i = (x_i + l cos th_i, y_i + l sin th_i) on which the
 *      single-integrator (SI) layer acts (SI controller + SI<->unicycle map, Sec. 4.1);
 *   2. nominal SI velocity u_nom: the policy action, or the scripted go-to-target law
 *      k (target - p) capped to v_max plus uniform action noise (Sec. 7 domain randomisation),
 *      then capped to v_max;
 *   3. the barrier-certificate QP (Sec. 4.1, the robust-CBF QP it cites):
 *          min |u - u_nom|^2  s.t.  -2 (p_i - p_j).(u_i - u_j) <= gamma h_ij^3,
 *          h_ij = |p_i - p_j|^2 - r^2   for every pair i < j,
 *          and four arena rows per robot  +-u_{x,y} <= kappa gamma (distance to wall - r/2)^3;
 *      solved exactly (Goldfarb-Idnani dual active set on H = I, then the equality-constrained
 *      KKT system on the final active set);
 *   4. SI -> unicycle map v = cos th u_x + sin th u_y, omega = (-sin th u_x + cos th u_y) / l;
 *   5. differential-drive wheel clip (GRITSBot actuator limits, Sec. 1 "dynamic constraints");
 *   6. explicit Euler unicycle step with heading wrapped by atan2(sin, cos);
 *   7. collision / boundary flags, team reward, scenario transition, done, auto-reset, and
 *      per-robot observations (App. B Navigation and Foraging).
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC 2011), implemented here from that definition.  Counter = (env, episode,
 * purpose << 24 | index, step or attempt); key = the 64-bit seed.  The reset sampler and the
 * noise draw are specified in binary32 arithmetic (round-to-nearest, no fused multiply-add) so
 * that any implementation reproduces the same bits; build with -ffp-contract=off.
 */
#include "oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#if !defined(FLT_EVAL_METHOD) || FLT_EVAL_METHOD != 0
#error "the oracle's binary32 sampler needs FLT_EVAL_METHOD == 0"
#endif

#define MMAX (ORC_NMAX * (ORC_NMAX - 1) / 2 + 4 * ORC_NMAX)
#define VMAX (2 * ORC_NMAX)

enum { P_NOISE = 1, P_POS = 2, P_GOAL = 3, P_NEAR = 4, P_LEVEL = 5, P_RES = 6, P_NRES = 7 };

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11): 10 rounds of two 32x32->64 multiplies, the key bumped by the Weyl   */
/* constants between rounds.                                                                  */
/* ------------------------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw(uint64_t seed, int e, int ep, int purpose, int index, uint32_t step,
                 uint32_t out[4]) {
    uint32_t ctr[4] = {(uint32_t)e, (uint32_t)ep, ((uint32_t)purpose << 24) | (uint32_t)index,
                       step};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* uniform in [0, 1) on the 2^-24 grid: exact in binary32 and binary64 */
static float u01(uint32_t w) { return (float)(w >> 8) * 0x1p-24f; }

/* floor(w * k / 2^32): an integer in [0, k) */
static int32_t below(uint32_t w, uint32_t k) { return (int32_t)(((uint64_t)w * k) >> 32); }

int orc_obs_dim(const orc_cfg* c) {
    if (c->scenario == ORC_FORAGE) return 4 + 4 * (c->n_max - 1) + 4 * c->r_max;
    if (c->scenario == ORC_DISCOVERY) return 5 + 5 * (c->n_max - 1) + 4 * c->r_max;
    return 5 + 3 * (c->n_max - 1);
}

/* ------------------------------------------------------------------------------------------ */
/* Environment state of one env                                                               */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int n, t, ep, n_res;
    double x[ORC_NMAX], y[ORC_NMAX], th[ORC_NMAX], gx[ORC_NMAX], gy[ORC_NMAX], gth[ORC_NMAX];
    int32_t level[ORC_NMAX];
    double qx[ORC_RMAX], qy[ORC_RMAX];
    int32_t qlevel[ORC_RMAX], qactive[ORC_RMAX];
} env_t;

static void load_env(const orc_cfg* c, const orc_batch* b, int e, int off, int n, env_t* s) {
    s->n = n;
    s->t = b->t[e];
    s->ep = b->ep[e];
    s->n_res = b->n_res[e];
    for (int i = 0; i < n; ++i) {
        s->x[i] = b->x[off + i]; s->y[i] = b->y[off + i]; s->th[i] = b->th[off + i];
        s->gx[i] = b->gx[off + i]; s->gy[i] = b->gy[off + i]; s->level[i] = b->level[off + i];
        s->gth[i] = b->gth[off + i];
    }
    for (int k = 0; k < c->r_max; ++k) {
        s->qx[k] = b->qx[e * c->r_max + k]; s->qy[k] = b->qy[e * c->r_max + k];
        s->qlevel[k] = b->qlevel[e * c->r_max + k]; s->qactive[k] = b->qactive[e * c->r_max + k];
    }
}

static void store_env(const orc_cfg* c, orc_batch* b, int e, int off, const env_t* s) {
    b->t[e] = s->t;
    b->ep[e] = s->ep;
    b->n_res[e] = s->n_res;
    for (int i = 0; i < s->n; ++i) {
        b->x[off + i] = s->x[i]; b->y[off + i] = s->y[i]; b->th[off + i] = s->th[i];
        b->gx[off + i] = s->gx[i]; b->gy[off + i] = s->gy[i]; b->level[off + i] = s->level[i];
        b->gth[off + i] = s->gth[i];
    }
    for (int k = 0; k < c->r_max; ++k) {
        b->qx[e * c->r_max + k] = s->qx[k]; b->qy[e * c->r_max + k] = s->qy[k];
        b->qlevel[e * c->r_max + k] = s->qlevel[k]; b->qactive[e * c->r_max + k] = s->qactive[k];
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Reset sampler (binary32): poses uniform in the arena shrunk by init_margin with pairwise   */
/* separation >= min_sep by rejection; headings uniform; goals uniform in the same region.    */
/* A near_frac share of envs (selected by one draw) places robot 1 at a distance uniform in   */
/* [near_dmin, near_dmax] from robot 0 with robot 0's heading, so that their projected points */
/* are that far apart too (a near-degenerate barrier row, h close to 0).                      */
/* Foraging: robot levels and resource levels uniform in {1,2,3}, resource count uniform in   */
/* [n_res_min, n_res_max], resource positions uniform in the same region.                     */
/* ------------------------------------------------------------------------------------------ */
static void sample_env(const orc_cfg* c, uint64_t seed, int e, int ep, int n, env_t* s) {
    const float lox = (float)c->xmin + (float)c->init_margin;
    const float hix = (float)c->xmax - (float)c->init_margin;
    const float loy = (float)c->ymin + (float)c->init_margin;
    const float hiy = (float)c->ymax - (float)c->init_margin;
    const float wx = hix - lox, wy = hiy - loy;
    const float sep2 = (float)c->min_sep * (float)c->min_sep;
    const float pif = (float)M_PI, twopif = (float)(2.0 * M_PI);
    float fx[ORC_NMAX], fy[ORC_NMAX], fth[ORC_NMAX];
    uint32_t w[4];

    memset(s, 0, sizeof(*s));
    s->n = n;
    s->t = 0;
    s->ep = ep;

    int first = 0;
    /* robot 0 */
    draw(seed, e, ep, P_POS, 0, 0, w);
    fx[0] = lox + u01(w[0]) * wx;
    fy[0] = loy + u01(w[1]) * wy;
    fth[0] = -pif + u01(w[2]) * twopif;
    first = 1;

    if (n >= 2 && c->near_frac > 0.0) {
        draw(seed, e, ep, P_NEAR, 0, 0, w);
        if (u01(w[0]) < (float)c->near_frac) {
            const float dmin = (float)c->near_dmin, dspan = (float)c->near_dmax - (float)c->near_dmin;
            for (int a = 0; a < c->max_attempts; ++a) {
                draw(seed, e, ep, P_NEAR, 1, (uint32_t)a, w);
                float d = dmin + u01(w[0]) * dspan;
                float cx = 2.0f * u01(w[1]) - 1.0f;
                float cy = 2.0f * u01(w[2]) - 1.0f;
                float rr = cx * cx + cy * cy;
                if (rr < 0.0625f || rr > 1.0f) continue;
                float nrm = sqrtf(rr);
                float ox = (d * cx) / nrm, oy = (d * cy) / nrm;
                float x1 = fx[0] + ox, y1 = fy[0] + oy;
                if (x1 < lox || x1 > hix || y1 < loy || y1 > hiy) continue;
                fx[1] = x1;
                fy[1] = y1;
                fth[1] = fth[0]; /* same heading: the projected points keep distance d */
                first = 2;
                break;
            }
        }
    }
    for (int i = first; i < n; ++i) {
        for (int a = 0; a < c->max_attempts; ++a) {
            draw(seed, e, ep, P_POS, i, (uint32_t)a, w);
            float cx = lox + u01(w[0]) * wx;
            float cy = loy + u01(w[1]) * wy;
            int ok = 1;
            for (int j = 0; j < i; ++j) {
                float dx = cx - fx[j], dy = cy - fy[j];
                float d2 = dx * dx + dy * dy;
                if (d2 < sep2) { ok = 0; break; }
            }
            fx[i] = cx;
            fy[i] = cy;
            fth[i] = -pif + u01(w[2]) * twopif;
            if (ok) break; /* after max_attempts the last candidate is kept */
        }
    }
    for (int i = 0; i < n; ++i) {
        s->x[i] = (double)fx[i];
        s->y[i] = (double)fy[i];
        s->th[i] = (double)fth[i];
        draw(seed, e, ep, P_GOAL, i, 0, w);
        s->gx[i] = (double)(lox + u01(w[0]) * wx);
        s->gy[i] = (double)(loy + u01(w[1]) * wy);
        s->gth[i] = (double)(-pif + u01(w[2]) * twopif);  /* goal heading (pose controller) */
        s->level[i] = 0;
    }
    s->n_res = 0;
    if (c->scenario == ORC_DISCOVERY) {
        /* Discovery (App. B): the first ceil(n/2) robots sense (role 1), the others tag (role
           2); K landmarks uniform in the arena region, none sensed (qlevel 0) or tagged
           (qactive 1 = still to tag) */
        for (int i = 0; i < n; ++i) s->level[i] = (i < (n + 1) / 2) ? 1 : 2;
        draw(seed, e, ep, P_NRES, 0, 0, w);
        s->n_res = c->n_res_min + below(w[0], (uint32_t)(c->n_res_max - c->n_res_min + 1));
        for (int k = 0; k < s->n_res; ++k) {
            draw(seed, e, ep, P_RES, k, 0, w);
            s->qx[k] = (double)(lox + u01(w[0]) * wx);
            s->qy[k] = (double)(loy + u01(w[1]) * wy);
            s->qlevel[k] = 0;
            s->qactive[k] = 1;
        }
    }
    if (c->scenario == ORC_FORAGE) {
        for (int i = 0; i < n; ++i) {
            draw(seed, e, ep, P_LEVEL, i, 0, w);
            s->level[i] = 1 + below(w[0], 3);
        }
        draw(seed, e, ep, P_NRES, 0, 0, w);
        s->n_res = c->n_res_min + below(w[0], (uint32_t)(c->n_res_max - c->n_res_min + 1));
        for (int k = 0; k < s->n_res; ++k) {
            draw(seed, e, ep, P_RES, k, 0, w);
            s->qx[k] = (double)(lox + u01(w[0]) * wx);
            s->qy[k] = (double)(loy + u01(w[1]) * wy);
            s->qlevel[k] = 1 + below(w[2], 3);
            s->qactive[k] = 1;
        }
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Dense linear algebra helpers                                                               */
/* ------------------------------------------------------------------------------------------ */
static double dot(int n, const double* a, const double* b) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Solve G x = rhs with G symmetric positive definite (q x q) by a Cholesky factorisation
   computed from scratch.  Returns 0 on success, 1 if G is not numerically positive definite. */
static int chol_solve(int q, const double* G, const double* rhs, double* x) {
    double L[VMAX * VMAX];
    for (int i = 0; i < q; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = G[i * q + j];
            for (int k = 0; k < j; ++k) s -= L[i * VMAX + k] * L[j * VMAX + k];
            if (i == j) {
                if (!(s > 0.0)) return 1;
                L[i * VMAX + i] = sqrt(s);
            } else {
                L[i * VMAX + j] = s / L[j * VMAX + j];
            }
        }
    }
    double yv[VMAX];
    for (int i = 0; i < q; ++i) {
        double s = rhs[i];
        for (int k = 0; k < i; ++k) s -= L[i * VMAX + k] * yv[k];
        yv[i] = s / L[i * VMAX + i];
    }
    for (int i = q - 1; i >= 0; --i) {
        double s = yv[i];
        for (int k = i + 1; k < q; ++k) s -= L[k * VMAX + i] * x[k];
        x[i] = s / L[i * VMAX + i];
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* QP: min 1/2 |u - u0|^2 s.t. A u <= b.  Goldfarb & Idnani's dual active-set method          */
/* (Math. Programming 27, 1983) with Hessian I: start at the unconstrained minimiser u0, add  */
/* the most violated row (ties: lowest index), step in primal direction z = (I - N G^-1 N^T) */
/* a_p and dual direction r = G^-1 N^T a_p (N: active rows, G = N^T N), drop a row whose      */
/* multiplier would turn negative.  Finally the KKT system of the final active set is solved */
/* directly (G lam = N^T u0 - b_A, u = u0 - N lam) and kept if it is feasible and dual        */
/* feasible.                                                                                  */
/* ------------------------------------------------------------------------------------------ */
int orc_qp_project(int n, int m, const double* A, const double* bvec, const double* u0,
                   double* u, double* lam, int32_t* n_active, int32_t* iters) {
    int act[VMAX];
    double lam_act[VMAX];
    int in_set[MMAX > 1024 ? MMAX : 1024];
    int q = 0, it = 0, status = 0;
    const int max_iter = 10 * m + 100;
    double G[VMAX * VMAX], w[VMAX], r[VMAX], z[VMAX];

    if (n > VMAX || m > (int)(sizeof(in_set) / sizeof(in_set[0]))) return 3;
    for (int k = 0; k < m; ++k) in_set[k] = 0;
    for (int i = 0; i < n; ++i) u[i] = u0[i];

    for (;;) {
        /* most violated inactive row */
        int p = -1;
        double worst = 0.0;
        for (int k = 0; k < m; ++k) {
            if (in_set[k]) continue;
            double s = dot(n, A + (size_t)k * n, u) - bvec[k];
            double tol = 1e-12 * (1.0 + fabs(bvec[k]));
            if (s > tol && (p < 0 || s > worst)) { p = k; worst = s; }
        }
        if (p < 0) break;
        if (++it > max_iter) { status = 2; break; }

        const double* ap = A + (size_t)p * n;
        double lam_p = 0.0;
        int added = 0;
        while (!added) {
            /* r = G^-1 N^T a_p ; z = a_p - N r */
            for (int j = 0; j < q; ++j) {
                w[j] = dot(n, A + (size_t)act[j] * n, ap);
                for (int k = 0; k < q; ++k)
                    G[j * q + k] = dot(n, A + (size_t)act[j] * n, A + (size_t)act[k] * n);
            }
            if (q > 0 && chol_solve(q, G, w, r)) { status = 2; goto finish; }
            for (int i = 0; i < n; ++i) {
                double zi = ap[i];
                for (int j = 0; j < q; ++j) zi -= r[j] * A[(size_t)act[j] * n + i];
                z[i] = zi;
            }
            double zz = dot(n, z, z);
            double app = dot(n, ap, ap);
            /* largest dual step keeping the active multipliers non-negative */
            double t_dual = INFINITY;
            int jblock = -1;
            for (int j = 0; j < q; ++j) {
                if (r[j] > 0.0) {
                    double tj = lam_act[j] / r[j];
                    if (tj < t_dual) { t_dual = tj; jblock = j; }
                }
            }
            double s = dot(n, ap, u) - bvec[p];
            double t_full = (zz > 1e-12 * app) ? s / zz : INFINITY;
            if (isinf(t_full) && isinf(t_dual)) { status = 1; goto finish; }
            double t = t_full < t_dual ? t_full : t_dual;
            if (!isinf(t_full)) {
                for (int i = 0; i < n; ++i) u[i] -= t * z[i];
            }
            for (int j = 0; j < q; ++j) lam_act[j] -= t * r[j];
            lam_p += t;
            if (t_full <= t_dual) {
                act[q] = p;
                lam_act[q] = lam_p;
                in_set[p] = 1;
                ++q;
                added = 1;
            } else {
                /* drop the blocking row */
                in_set[act[jblock]] = 0;
                for (int j = jblock; j < q - 1; ++j) {
                    act[j] = act[j + 1];
                    lam_act[j] = lam_act[j + 1];
                }
                --q;
            }
        }
    }

    /* exact solve on the final active set */
    if (status == 0 && q > 0) {
        double rhs[VMAX], lp[VMAX], up[VMAX];
        for (int j = 0; j < q; ++j) {
            rhs[j] = dot(n, A + (size_t)act[j] * n, u0) - bvec[act[j]];
            for (int k = 0; k < q; ++k)
                G[j * q + k] = dot(n, A + (size_t)act[j] * n, A + (size_t)act[k] * n);
        }
        if (chol_solve(q, G, rhs, lp) == 0) {
            for (int i = 0; i < n; ++i) {
                double ui = u0[i];
                for (int j = 0; j < q; ++j) ui -= lp[j] * A[(size_t)act[j] * n + i];
                up[i] = ui;
            }
            int ok = 1;
            for (int j = 0; j < q; ++j)
                if (lp[j] < -1e-10) ok = 0;
            for (int k = 0; k < m && ok; ++k) {
                double sk = dot(n, A + (size_t)k * n, up) - bvec[k];
                if (sk > 1e-10 * (1.0 + fabs(bvec[k]))) ok = 0;
            }
            if (ok) {
                for (int i = 0; i < n; ++i) u[i] = up[i];
                for (int j = 0; j < q; ++j) lam_act[j] = lp[j] > 0.0 ? lp[j] : 0.0;
            }
        }
    }
finish:
    if (lam) {
        for (int k = 0; k < m; ++k) lam[k] = 0.0;
        for (int j = 0; j < q; ++j) lam[act[j]] = lam_act[j];
    }
    if (n_active) *n_active = q;
    if (iters) *iters = it;
    return status;
}

/* Rows of the barrier QP for one env over the stacked SI velocity u = [u_0x, u_0y, u_1x, ...].
   Pairs i < j in lexicographic order, then per robot the arena rows [+x, -x, +y, -y]. */
int orc_build_cbf_rows(const orc_cfg* c, int N, const double* px, const double* py, double* A,
                       double* bvec) {
    const int n = 2 * N;
    const int m = N * (N - 1) / 2 + 4 * N;
    for (int k = 0; k < m * n; ++k) A[k] = 0.0;
    int row = 0;
    for (int i = 0; i < N; ++i) {
        for (int j = i + 1; j < N; ++j) {
            double dx = px[i] - px[j], dy = py[i] - py[j];
            double h = dx * dx + dy * dy - c->r * c->r;
            double* a = A + (size_t)row * n;
            a[2 * i] = -2.0 * dx;
            a[2 * i + 1] = -2.0 * dy;
            a[2 * j] = 2.0 * dx;
            a[2 * j + 1] = 2.0 * dy;
            bvec[row] = c->gamma * h * h * h;
            ++row;
        }
    }
    const double kg = c->kappa * c->gamma, half_r = 0.5 * c->r;
    for (int i = 0; i < N; ++i) {
        double d[4] = {c->xmax - half_r - px[i], px[i] - c->xmin - half_r,
                       c->ymax - half_r - py[i], py[i] - c->ymin - half_r};
        double sgn[4] = {1.0, -1.0, 1.0, -1.0};
        int col[4] = {2 * i, 2 * i, 2 * i + 1, 2 * i + 1};
        for (int s = 0; s < 4; ++s) {
            A[(size_t)row * n + col[s]] = sgn[s];
            bvec[row] = kg * d[s] * d[s] * d[s];
            ++row;
        }
    }
    return m;
}

static double wrap_angle(double a) { return atan2(sin(a), cos(a)); }

/* Posture regulation of a unicycle in polar coordinates (Aicardi, Casalino, Bicchi, Balestrino,
   "Closed loop steering of unicycle-like vehicles via Lyapunov techniques", IEEE Robotics &
   Automation Magazine 1995).  In the goal's frame the robot sits at (xr, yr) with heading thr;
   rho is its distance to the goal, gam the angle from its heading to the direction of the goal,
   del the angle of that direction in the goal's frame.  The law
       v = k1 rho cos(gam),  omega = k2 gam + k1 (sin(gam) cos(gam) / gam) (gam + k3 del)
   makes V = (rho^2 + gam^2 + k3 del^2) / 2 non-increasing: dV/dt = -k1 cos^2(gam) rho^2 - k2 gam^2.
   The paper evaluates a unicycle pose controller (Sec. 4.2, Table 2) without giving its law;
   this published one stands for it (a reading). */
void orc_pose_control(const orc_cfg* c, const double* pose, const double* goal, double* vw) {
    const double cg = cos(goal[2]), sg = sin(goal[2]);
    const double dx = pose[0] - goal[0], dy = pose[1] - goal[1];
    const double xr = cg * dx + sg * dy, yr = -sg * dx + cg * dy;
    const double thr = wrap_angle(pose[2] - goal[2]);
    const double rho = hypot(xr, yr);
    if (rho == 0.0) {  /* on the goal point: turn in place towards the goal heading */
        vw[0] = 0.0;
        vw[1] = -c->pose_k2 * thr;
        return;
    }
    const double gam = wrap_angle(atan2(yr, xr) + M_PI - thr);
    const double del = wrap_angle(gam + thr);
    const double sinc = (gam == 0.0) ? 1.0 : sin(gam) / gam;
    vw[0] = c->pose_k1 * rho * cos(gam);
    vw[1] = c->pose_k2 * gam + c->pose_k1 * sinc * cos(gam) * (gam + c->pose_k3 * del);
}

void orc_unicycle_update(const orc_cfg* c, double ux, double uy, double* pose, double* vw) {
    double cs = cos(pose[2]), sn = sin(pose[2]);
    /* SI -> unicycle map for the point l ahead of the wheel axle */
    double v = cs * ux + sn * uy;
    double om = (-sn * ux + cs * uy) / c->l;
    /* differential-drive wheel clip: track width L chosen so that (vmax, 0) and (0, wmax) are
       the extreme points; each wheel's speed is clipped to [-vmax, vmax] */
    double L = 2.0 * c->vmax / c->wmax;
    double wr = v + 0.5 * L * om, wl = v - 0.5 * L * om;
    if (wr > c->vmax) wr = c->vmax;
    if (wr < -c->vmax) wr = -c->vmax;
    if (wl > c->vmax) wl = c->vmax;
    if (wl < -c->vmax) wl = -c->vmax;
    v = 0.5 * (wr + wl);
    om = (wr - wl) / L;
    /* explicit Euler with the pre-step heading */
    pose[0] += c->dt * v * cs;
    pose[1] += c->dt * v * sn;
    pose[2] = wrap_angle(pose[2] + c->dt * om);
    if (vw) { vw[0] = v; vw[1] = om; }
}

static void cap_norm(double* ux, double* uy, double m) {
    double nrm = sqrt(*ux * *ux + *uy * *uy);
    if (nrm > m) {
        *ux *= m / nrm;
        *uy *= m / nrm;
    }
}

static void write_obs(const orc_cfg* c, const env_t* s, double* obs) {
    const int od = orc_obs_dim(c);
    for (int i = 0; i < s->n; ++i) {
        double* o = obs + (size_t)i * od;
        for (int k = 0; k < od; ++k) o[k] = 0.0;
        int base;
        if (c->scenario == ORC_DISCOVERY) {
            /* own pose and capability [sensing radius, tagging radius]; the others' relative
               poses and capabilities; landmarks: relative position, sensed, tagged once sensed,
               else the relative position of a point outside the arena and zeros (App. B) */
            const double xo = c->xmax + (c->xmax - c->xmin), yo = c->ymax + (c->ymax - c->ymin);
            o[0] = s->x[i]; o[1] = s->y[i]; o[2] = s->th[i];
            o[3] = s->level[i] == 1 ? c->sense_radius : 0.0;
            o[4] = s->level[i] == 2 ? c->tag_radius : 0.0;
            int slot = 0;
            for (int j = 0; j < s->n; ++j) {
                if (j == i) continue;
                double* q = o + 5 + 5 * slot;
                q[0] = s->x[j] - s->x[i];
                q[1] = s->y[j] - s->y[i];
                q[2] = wrap_angle(s->th[j] - s->th[i]);
                q[3] = s->level[j] == 1 ? c->sense_radius : 0.0;
                q[4] = s->level[j] == 2 ? c->tag_radius : 0.0;
                ++slot;
            }
            base = 5 + 5 * (c->n_max - 1);
            for (int k = 0; k < s->n_res; ++k) {
                double* q = o + base + 4 * k;
                if (s->qlevel[k]) {
                    q[0] = s->qx[k] - s->x[i];
                    q[1] = s->qy[k] - s->y[i];
                    q[2] = 1.0;
                    q[3] = s->qactive[k] ? 0.0 : 1.0;
                } else {
                    q[0] = xo - s->x[i];
                    q[1] = yo - s->y[i];
                }
            }
        } else if (c->scenario == ORC_FORAGE) {
            o[0] = s->x[i]; o[1] = s->y[i]; o[2] = s->th[i]; o[3] = (double)s->level[i];
            base = 4;
            int slot = 0;
            for (int j = 0; j < s->n; ++j) {
                if (j == i) continue;
                double* q = o + base + 4 * slot;
                q[0] = s->x[j] - s->x[i];
                q[1] = s->y[j] - s->y[i];
                q[2] = wrap_angle(s->th[j] - s->th[i]);
                q[3] = (double)s->level[j];
                ++slot;
            }
            base = 4 + 4 * (c->n_max - 1);
            for (int k = 0; k < s->n_res; ++k) {
                double* q = o + base + 4 * k;
                q[0] = s->qx[k] - s->x[i];
                q[1] = s->qy[k] - s->y[i];
                q[2] = (double)s->qlevel[k];
                q[3] = (double)s->qactive[k];
            }
        } else {
            o[0] = s->x[i]; o[1] = s->y[i]; o[2] = s->th[i]; o[3] = s->gx[i]; o[4] = s->gy[i];
            base = 5;
            int slot = 0;
            for (int j = 0; j < s->n; ++j) {
                if (j == i) continue;
                double* q = o + base + 3 * slot;
                q[0] = s->x[j] - s->x[i];
                q[1] = s->y[j] - s->y[i];
                q[2] = wrap_angle(s->th[j] - s->th[i]);
                ++slot;
            }
        }
    }
}

typedef struct {
    double A[MMAX * VMAX];
    double b[MMAX];
    double lam[MMAX];
} qp_ws;

/* One step of one env.  act: [2n] or NULL.  Outputs of this env only. */
static void env_step(const orc_cfg* c, uint64_t seed, int e, env_t* s, const double* act,
                     qp_ws* ws, double* obs, double* reward, uint8_t* done, int32_t* cnt,
                     double* tr_unom, double* tr_ustar, double* tr_vw, int32_t* tr_qp,
                     double* tr_kkt) {
    const int N = s->n;
    const int n = 2 * N;
    double cs[ORC_NMAX], sn[ORC_NMAX], px[ORC_NMAX], py[ORC_NMAX];
    double unom[VMAX], ustar[VMAX];

    for (int i = 0; i < N; ++i) {
        cs[i] = cos(s->th[i]);
        sn[i] = sin(s->th[i]);
        px[i] = s->x[i] + c->l * cs[i];
        py[i] = s->y[i] + c->l * sn[i];
    }

    /* nominal single-integrator velocity */
    for (int i = 0; i < N; ++i) {
        double ux, uy;
        if (act) {
            ux = act[2 * i];
            uy = act[2 * i + 1];
        } else {
            double tx = s->gx[i], ty = s->gy[i];
            if (c->scenario == ORC_DISCOVERY) {
                /* sensing robots: the nearest landmark not yet sensed; tagging robots: the
                   nearest sensed one not yet tagged (ties: lowest index); none: hold */
                int best = -1;
                double bd = 0.0;
                for (int k = 0; k < s->n_res; ++k) {
                    const int want = (s->level[i] == 1) ? !s->qlevel[k]
                                                        : (s->qlevel[k] && s->qactive[k]);
                    if (!want) continue;
                    double dx = s->qx[k] - px[i], dy = s->qy[k] - py[i];
                    double d2 = dx * dx + dy * dy;
                    if (best < 0 || d2 < bd) { best = k; bd = d2; }
                }
                if (best >= 0) { tx = s->qx[best]; ty = s->qy[best]; }
                else { tx = px[i]; ty = py[i]; }
            }
            if (c->scenario == ORC_FORAGE) {
                /* nearest active resource (ties: lowest index); none: hold position */
                int best = -1;
                double bd = 0.0;
                for (int k = 0; k < s->n_res; ++k) {
                    if (!s->qactive[k]) continue;
                    double dx = s->qx[k] - px[i], dy = s->qy[k] - py[i];
                    double d2 = dx * dx + dy * dy;
                    if (best < 0 || d2 < bd) { best = k; bd = d2; }
                }
                if (best >= 0) { tx = s->qx[best]; ty = s->qy[best]; }
                else { tx = px[i]; ty = py[i]; }
            }
            if (c->scenario == ORC_NAV && c->controller == ORC_CTRL_POSE) {
                /* unicycle pose controller, then its command as the projected point's velocity
                   (the SI <-> unicycle map at distance l, c2) */
                const double pose[3] = {s->x[i], s->y[i], s->th[i]};
                const double goal[3] = {s->gx[i], s->gy[i], s->gth[i]};
                double vw[2];
                orc_pose_control(c, pose, goal, vw);
                ux = vw[0] * cs[i] - c->l * vw[1] * sn[i];
                uy = vw[0] * sn[i] + c->l * vw[1] * cs[i];
            } else {
                ux = c->k_si * (tx - px[i]);
                uy = c->k_si * (ty - py[i]);
            }
            cap_norm(&ux, &uy, c->vmax);
            if (c->noise_amp > 0.0) {
                uint32_t w[4];
                draw(seed, e, s->ep, P_NOISE, i >> 1, (uint32_t)s->t, w);
                const float scale = 2.0f * (float)c->noise_amp;
                float ex = (u01(w[2 * (i & 1)]) - 0.5f) * scale;
                float ey = (u01(w[2 * (i & 1) + 1]) - 0.5f) * scale;
                ux += (double)ex;
                uy += (double)ey;
            }
        }
        cap_norm(&ux, &uy, c->vmax);
        unom[2 * i] = ux;
        unom[2 * i + 1] = uy;
    }

    /* barrier-certificate QP */
    int m = orc_build_cbf_rows(c, N, px, py, ws->A, ws->b);
    int32_t q = 0, iters = 0;
    int status = orc_qp_project(n, m, ws->A, ws->b, unom, ustar, ws->lam, &q, &iters);
    if (status != 0) {
        for (int i = 0; i < n; ++i) ustar[i] = 0.0; /* infeasible: the env stops */
    }
    int any_active = (q > 0) || status != 0;
    if (tr_kkt) {
        /* stationarity u - u0 + A^T lam = 0, feasibility, complementarity */
        double res = 0.0;
        if (status == 0) {
            for (int i = 0; i < n; ++i) {
                double g = ustar[i] - unom[i];
                for (int k = 0; k < m; ++k) g += ws->A[(size_t)k * n + i] * ws->lam[k];
                if (fabs(g) > res) res = fabs(g);
            }
            for (int k = 0; k < m; ++k) {
                double sk = dot(n, ws->A + (size_t)k * n, ustar) - ws->b[k];
                if (sk > res) res = sk;
                if (-ws->lam[k] > res) res = -ws->lam[k];
                if (fabs(ws->lam[k] * sk) > res) res = fabs(ws->lam[k] * sk);
            }
        }
        *tr_kkt = res;
    }

    double d_old[ORC_NMAX];
    for (int i = 0; i < N; ++i) d_old[i] = hypot(px[i] - s->gx[i], py[i] - s->gy[i]);

    /* unicycle map, wheel clip, integration */
    for (int i = 0; i < N; ++i) {
        double pose[3] = {s->x[i], s->y[i], s->th[i]}, vw[2];
        orc_unicycle_update(c, ustar[2 * i], ustar[2 * i + 1], pose, vw);
        s->x[i] = pose[0];
        s->y[i] = pose[1];
        s->th[i] = pose[2];
        if (tr_vw) { tr_vw[2 * i] = vw[0]; tr_vw[2 * i + 1] = vw[1]; }
    }
    for (int i = 0; i < N; ++i) {
        px[i] = s->x[i] + c->l * cos(s->th[i]);
        py[i] = s->y[i] + c->l * sin(s->th[i]);
    }

    /* flags on the new projected points */
    int col = 0, oob = 0;
    for (int i = 0; i < N; ++i)
        for (int j = i + 1; j < N; ++j) {
            double dx = px[i] - px[j], dy = py[i] - py[j];
            if (dx * dx + dy * dy < c->r * c->r) ++col;
        }
    for (int i = 0; i < N; ++i)
        if (px[i] < c->xmin || px[i] > c->xmax || py[i] < c->ymin || py[i] > c->ymax) ++oob;

    /* reward and scenario transition */
    double rew = 0.0;
    int all_foraged = 0;
    if (c->scenario == ORC_FORAGE) {
        const double rho2 = c->forage_radius * c->forage_radius;
        int remaining = 0;
        for (int k = 0; k < s->n_res; ++k) {
            if (!s->qactive[k]) continue;
            int lsum = 0;
            for (int i = 0; i < N; ++i) {
                double dx = px[i] - s->qx[k], dy = py[i] - s->qy[k];
                if (dx * dx + dy * dy < rho2) lsum += s->level[i];
            }
            if (lsum >= s->qlevel[k]) {
                s->qactive[k] = 0;
                rew += (double)s->qlevel[k];
                cnt[ORC_CNT_SUCCESS] += 1;
            } else {
                ++remaining;
            }
        }
        all_foraged = (s->n_res > 0 && remaining == 0);
    } else if (c->scenario == ORC_DISCOVERY) {
        /* a landmark within the sensing radius of a sensing robot becomes sensed; a sensed
           landmark within the tagging radius of a tagging robot becomes tagged (in the same
           step too); rewards per landmark sensed and tagged, a penalty for every step that
           ends with a landmark still to tag (App. B); each tag counts as a success */
        const double rs2 = c->sense_radius * c->sense_radius, rt2 = c->tag_radius * c->tag_radius;
        int remaining = 0;
        for (int k = 0; k < s->n_res; ++k) {
            if (!s->qlevel[k]) {
                for (int i = 0; i < N; ++i) {
                    double dx = px[i] - s->qx[k], dy = py[i] - s->qy[k];
                    if (s->level[i] == 1 && dx * dx + dy * dy < rs2) { s->qlevel[k] = 1; break; }
                }
                if (s->qlevel[k]) rew += c->sense_reward;
            }
            if (s->qlevel[k] && s->qactive[k]) {
                for (int i = 0; i < N; ++i) {
                    double dx = px[i] - s->qx[k], dy = py[i] - s->qy[k];
                    if (s->level[i] == 2 && dx * dx + dy * dy < rt2) { s->qactive[k] = 0; break; }
                }
                if (!s->qactive[k]) {
                    rew += c->tag_reward;
                    cnt[ORC_CNT_SUCCESS] += 1;
                }
            }
            remaining += s->qactive[k];
        }
        if (remaining > 0) rew -= c->step_penalty;
    } else {
        for (int i = 0; i < N; ++i) {
            double d_new = hypot(px[i] - s->gx[i], py[i] - s->gy[i]);
            rew -= d_new - d_old[i];
        }
        /* Random Waypoint Navigation (Sec. 4.2): a robot whose projected point ends the step
           strictly within goal_eps of its goal is assigned a new goal (after the reward, which
           uses the goal it was heading to), drawn from the reset's goal distribution under the
           counter (env, episode, goal | robot, steps taken in the episode including this one).
           Each arrival counts as a success. */
        if (c->goal_eps > 0.0) {
            const float lox = (float)c->xmin + (float)c->init_margin;
            const float hix = (float)c->xmax - (float)c->init_margin;
            const float loy = (float)c->ymin + (float)c->init_margin;
            const float hiy = (float)c->ymax - (float)c->init_margin;
            const float wx = hix - lox, wy = hiy - loy;
            for (int i = 0; i < N; ++i) {
                double dx = px[i] - s->gx[i], dy = py[i] - s->gy[i];
                if (dx * dx + dy * dy < c->goal_eps * c->goal_eps) {
                    uint32_t w[4];
                    draw(seed, e, s->ep, P_GOAL, i, (uint32_t)(s->t + 1), w);
                    s->gx[i] = (double)(lox + u01(w[0]) * wx);
                    s->gy[i] = (double)(loy + u01(w[1]) * wy);
                    s->gth[i] = (double)(-(float)M_PI + u01(w[2]) * (float)(2.0 * M_PI));
                    cnt[ORC_CNT_SUCCESS] += 1;
                }
            }
        }
    }
    rew -= c->c_col * (double)col;

    cnt[ORC_CNT_COLLISIONS] += col;
    cnt[ORC_CNT_OOB] += oob;
    cnt[ORC_CNT_QP_ACTIVE] += any_active;
    cnt[ORC_CNT_QP_INFEASIBLE] += (status == 1);
    cnt[ORC_CNT_QP_ITERS] += iters;

    s->t += 1;
    int d = (s->t >= c->episode_len) || all_foraged;
    if (d) {
        cnt[ORC_CNT_EPISODES] += 1;
        sample_env(c, seed, e, s->ep + 1, N, s);
    }
    *reward = rew;
    *done = (uint8_t)d;
    if (obs) write_obs(c, s, obs);
    if (tr_unom) for (int i = 0; i < n; ++i) tr_unom[i] = unom[i];
    if (tr_ustar) for (int i = 0; i < n; ++i) tr_ustar[i] = ustar[i];
    if (tr_qp) { tr_qp[0] = status; tr_qp[1] = q; tr_qp[2] = iters; tr_qp[3] = any_active; }
}

static int check_cfg(const orc_cfg* c, int E, const int32_t* n_robots) {
    if (E < 0 || c->n_max < 1 || c->n_max > ORC_NMAX || c->r_max < 0 || c->r_max > ORC_RMAX)
        return 1;
    if (c->scenario != ORC_NAV && c->scenario != ORC_FORAGE && c->scenario != ORC_DISCOVERY)
        return 1;
    if (c->scenario != ORC_NAV && (c->n_res_min < 0 || c->n_res_max > c->r_max ||
                                   c->n_res_min > c->n_res_max))
        return 1;
    if (!(c->goal_eps >= 0.0) || (c->goal_eps > 0.0 && c->scenario != ORC_NAV)) return 1;
    if (c->controller != ORC_CTRL_POSITION && c->controller != ORC_CTRL_POSE) return 1;
    if (c->controller == ORC_CTRL_POSE &&
        (c->scenario != ORC_NAV || !(c->pose_k1 > 0.0) || !(c->pose_k2 > 0.0) || !(c->pose_k3 > 0.0)))
        return 1;
    for (int e = 0; e < E; ++e)
        if (n_robots[e] < 1 || n_robots[e] > c->n_max) return 1;
    return 0;
}

int orc_reset_batch(const orc_cfg* c, uint64_t seed, int E, const int32_t* n_robots,
                    const int32_t* ep, orc_batch* b) {
    if (check_cfg(c, E, n_robots)) return 1;
    int off = 0;
    for (int e = 0; e < E; ++e) {
        env_t s;
        sample_env(c, seed, e, ep ? ep[e] : 0, n_robots[e], &s);
        store_env(c, b, e, off, &s);
        for (int k = 0; k < ORC_NCOUNT; ++k) b->counters[e * ORC_NCOUNT + k] = 0;
        off += n_robots[e];
    }
    return 0;
}

int orc_step_batch(const orc_cfg* c, uint64_t seed, int E, const int32_t* n_robots, orc_batch* b,
                   const double* actions, double* obs, double* reward, uint8_t* done,
                   orc_trace* tr, int n_threads) {
    if (check_cfg(c, E, n_robots)) return 1;
    const int od = orc_obs_dim(c);
    int32_t* offs = (int32_t*)malloc(sizeof(int32_t) * (size_t)(E + 1));
    if (!offs) return 2;
    offs[0] = 0;
    for (int e = 0; e < E; ++e) offs[e + 1] = offs[e] + n_robots[e];
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
#endif
    {
        qp_ws* ws = (qp_ws*)malloc(sizeof(qp_ws));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int e = 0; e < E; ++e) {
            env_t s;
            int off = offs[e];
            load_env(c, b, e, off, n_robots[e], &s);
            env_step(c, seed, e, &s, actions ? actions + 2 * (size_t)off : NULL, ws,
                     obs ? obs + (size_t)off * od : NULL, &reward[e], &done[e],
                     b->counters + e * ORC_NCOUNT,
                     tr && tr->u_nom ? tr->u_nom + 2 * (size_t)off : NULL,
                     tr && tr->u_star ? tr->u_star + 2 * (size_t)off : NULL,
                     tr && tr->vw ? tr->vw + 2 * (size_t)off : NULL,
                     tr && tr->qp ? tr->qp + 4 * (size_t)e : NULL,
                     tr && tr->kkt ? tr->kkt + e : NULL);
            store_env(c, b, e, off, &s);
        }
        free(ws);
    }
    free(offs);
    return 0;
}

int orc_rollout(const orc_cfg* c, uint64_t seed, int E, const int32_t* n_robots, orc_batch* b,
                int T, double* obs_traj, double* rew_traj, uint8_t* done_traj, int n_threads) {
    if (check_cfg(c, E, n_robots) || T < 0) return 1;
    const int od = orc_obs_dim(c);
    int32_t* offs = (int32_t*)malloc(sizeof(int32_t) * (size_t)(E + 1));
    if (!offs) return 2;
    offs[0] = 0;
    for (int e = 0; e < E; ++e) offs[e + 1] = offs[e] + n_robots[e];
    const size_t total = (size_t)offs[E];
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
#endif
    {
        qp_ws* ws = (qp_ws*)malloc(sizeof(qp_ws));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 4)
#endif
        for (int e = 0; e < E; ++e) {
            env_t s;
            int off = offs[e];
            load_env(c, b, e, off, n_robots[e], &s);
            for (int t = 0; t < T; ++t) {
                double rw;
                uint8_t dn;
                env_step(c, seed, e, &s, NULL, ws,
                         obs_traj ? obs_traj + ((size_t)t * total + (size_t)off) * od : NULL, &rw,
                         &dn, b->counters + e * ORC_NCOUNT, NULL, NULL, NULL, NULL, NULL);
                if (rew_traj) rew_traj[(size_t)t * E + e] = rw;
                if (done_traj) done_traj[(size_t)t * E + e] = dn;
            }
            store_env(c, b, e, off, &s);
        }
        free(ws);
    }
    free(offs);
    return 0;
}
