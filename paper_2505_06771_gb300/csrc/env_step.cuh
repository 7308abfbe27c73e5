// env_step.cuh -- device code of the batched multi-robot environment step (sm_103a).
//
// One environment is handled by a *team* of G consecutive lanes of a warp (G in 1..32, a power
// of two).  Robot i of the env is owned by lane i mod G, which keeps its pose, goal and cached
// heading sine/cosine in registers for the whole launch (a rollout of T steps never round-trips
// the state through global memory).  What lanes need from each other -- projected points, the
// QP iterate, the active set and its Cholesky factor -- sits in a per-team slice of shared
// memory; team-wide reductions use warp shuffles over width G.
//
// The step (JaxRobotarium, arXiv 2505.06771, Sec. 4.1 and 6.1, App. B):
//   projected points -> nominal SI velocity (policy action, or go-to-target + noise) -> speed cap
//   -> barrier-certificate QP -> SI-to-unicycle map -> wheel clip -> Euler step -> flags, reward,
//   scenario transition -> done and auto-reset -> observations.
//
// The QP, min |u - u_nom|^2 s.t. A u <= b, is a Euclidean projection (Hessian 2I), solved by the
// dual active-set method of Goldfarb and Idnani (1983): start at u_nom, add the most violated row,
// step along z = (I - N G^-1 N^T) a_p in the primal and r = G^-1 N^T a_p in the dual, drop rows
// whose multiplier would go negative.  G = N^T N (Gram of the active rows, at most 2N of them) is
// kept as a Cholesky factor that grows by one row per added constraint.  Row j's violation is
// evaluated on the fly from the projected points, so the m = N(N-1)/2 + 4N rows are never stored.
// Pair rows are spread over the lanes by a circulant schedule (robot i owns pairs (i, i+d mod N),
// d = 1..floor((N-1)/2), plus d = N/2 for i < N/2 when N is even), which balances them with no
// index table.  In binary32 a QP that hits the iteration cap, meets a nearly dependent row, is
// infeasible, or keeps an active pair with h < h_flag is re-solved in binary64 by the same team.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <math_constants.h>
#include <type_traits>

#include "philox.cuh"

namespace rl {

constexpr int kMaxRobots = 32;
constexpr int kMaxRes = 16;
constexpr int kNCount = 8;

template <typename R>
struct StepConsts {
    R gamma, r2, l, inv_l, vmax, half_track, inv_track, dt, kg, half_r, k_si, c_col, rho2;
    R xmin, xmax, ymin, ymax, h_flag;
    R goal_eps2;        // Navigation waypoints: squared arrival radius (waypoint != 0)
    R pk1, pk2, pk3;    // pose controller gains (controller == 1)
    R sense_r2, tag_r2, sense_rew, tag_rew, step_pen;  // Discovery (scenario 2)
    R sense_r, tag_r, xo, yo;  // capability radii and the unsensed landmarks' stand-in point
    int scenario, scripted, episode_len, max_iter, n_res_min, n_res_max, r_max, n_max_obs;
    int max_attempts, resolve_f64, noise_on, waypoint, controller;
    float noise_scale;  // 2 * noise amplitude, binary32 (the noise draw is binary32)
};

// Reset-sampler constants, binary32, computed on the host with one rounding each.
struct SamplerConsts {
    float lox, hix, loy, hiy, wx, wy, sep2, pif, twopif, near_frac, dmin, dspan;
    int near_on;
};

template <typename R>
struct StateView {
    R *x, *y, *th, *gx, *gy;
    R* gth;  // goal heading (pose controller)
    int32_t* level;
    int32_t *t, *ep, *n_res;
    R *qx, *qy;
    int32_t *qlevel, *qactive;
    int32_t* counters;
    const int32_t* off;   // [E + 1] first row of each env
    const int32_t* nrob;  // [E]
};

template <typename R>
struct StepIO {
    const R* actions;  // [rows][2] (T == 1 only)
    R* obs;            // [T][rows][obs_dim]
    R* reward;         // [T][E]
    uint8_t* done;     // [T][E]
    R* u_nom;          // [rows][2] traces (T == 1 only)
    R* u_star;
    R* vw;
    int32_t* qp_info;  // [E][4]
    R* ret;            // [E] sum of the rewards of this launch (serving), or NULL
    int32_t* status;   // device status word (host-mapped), or NULL; see flag_status
    long long obs_step;  // rows * obs_dim
    int E;
    int obs_dim;
};

// Bits of the device status word.  Set by any lane, read and cleared by the host.
constexpr int32_t kStatusNonFiniteAction = 1;
constexpr int32_t kStatusWaitTimeout = 2;  // a bounded wait in a kernel ran out (policy kernel)

// A non-finite policy action is replaced by zero (the robot's nominal velocity is zero, the
// barrier QP still applies) and reported through the status word.
template <typename R>
__device__ __forceinline__ void screen_action(int32_t* status, R& ux, R& uy) {
    if (!(isfinite(ux) && isfinite(uy))) {
        ux = (R)0;
        uy = (R)0;
        if (status) *(volatile int32_t*)status = kStatusNonFiniteAction;
    }
}

template <typename R>
struct LaunchArgs {
    StateView<R> s;
    StepIO<R> io;
    StepConsts<R> k;
    SamplerConsts sc;
    const int32_t* env_list;  // env ids of this launch (NULL: env_begin + index)
    int n_list;
    int env_begin;
    int T;
    int warp_envs;  // envs per 32-lane warp; 4-robot team kernels: <= 0 spreads the envs evenly
                    // over all warps of the grid (at most 8 per warp, one pass)
    int variant;    // 4-robot binary32 Navigation fast path: 1 shuffle team, 2 gather team
    uint64_t seed;
};

// ------------------------------------------------------------------------------------------
// Team of G lanes
// ------------------------------------------------------------------------------------------
template <int G>
struct Team {
    static_assert(G >= 1 && G <= 32 && (G & (G - 1)) == 0, "team size must be a power of two");
    int lane;
    int base;
    unsigned mask;
    __device__ __forceinline__ Team() {
        const int wl = threadIdx.x & 31;
        lane = wl & (G - 1);
        base = wl & ~(G - 1);
        mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << base);
    }
    __device__ __forceinline__ void sync() const { __syncwarp(mask); }
    template <typename T>
    __device__ __forceinline__ T sum(T v) const {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
        return v;
    }
    __device__ __forceinline__ unsigned ballot(bool p) const {
        const unsigned b = __ballot_sync(mask, p);
        return (G == 32) ? b : ((b >> base) & ((1u << G) - 1u));
    }
    __device__ __forceinline__ bool any(bool p) const { return ballot(p) != 0u; }
    // max of v, ties to the smallest key (all lanes get the result)
    template <typename T>
    __device__ __forceinline__ void argmax(T& v, int& key) const {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const T ov = __shfl_xor_sync(mask, v, o, G);
            const int ok = __shfl_xor_sync(mask, key, o, G);
            if (ov > v || (ov == v && ok < key)) { v = ov; key = ok; }
        }
    }
    template <typename T>
    __device__ __forceinline__ void argmin(T& v, int& key) const {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const T ov = __shfl_xor_sync(mask, v, o, G);
            const int ok = __shfl_xor_sync(mask, key, o, G);
            if (ov < v || (ov == v && ok < key)) { v = ov; key = ok; }
        }
    }
};

// ------------------------------------------------------------------------------------------
// Shared-memory workspace of one team
// ------------------------------------------------------------------------------------------
template <typename Q, int NMAX>
struct QPWork {
    static constexpr int A = 2 * NMAX;                          // active rows at most
    static constexpr int M = NMAX * (NMAX - 1) / 2 + 4 * NMAX;  // rows
    Q px[NMAX], py[NMAX];
    Q ux[NMAX], uy[NMAX];
    Q u0x[NMAX], u0y[NMAX];
    Q lam[A], w[A], yv[A], rv[A], rb[A], rax[A], ray[A];
    Q L[A * A];
    int ria[A], rib[A], rk[A];
    unsigned actbits[(M + 31) / 32];
    int fail;
};

// Explicit-inverse workspace of qp_solve_inv (see there): Q the precision, AS the slots (the
// most active rows it holds; 2 NMAX, the variables, in binary32).
template <int NMAX, typename Q = float, int AS = 2 * NMAX>
struct InvWork {
    static constexpr int A = AS;                                // slots (active rows at most)
    static constexpr int V = 2 * NMAX;                          // variables
    static_assert(AS <= 64, "free slots are a 64-bit mask");
    // rows padded to A + 1 words: lanes walking their own rows hit distinct banks
    Q Mi[V][A + 1];          // M = N G^-1, variable x slot
    Q Bi[A][A + 1];          // B = G^-1, slot x slot
    Q r[A];
    Q lam[A], sax[A], say[A], sb[A];
    int sia[A], sib[A], sk[A];
    int act[A];              // active slots in order of addition
    Q zx[NMAX], zy[NMAX];                // z = a_p - N r per robot (for the factor updates)
    unsigned long long inc[NMAX];        // per robot: the active slots whose row touches it
    unsigned long long free_slots;
};

struct NoInvWork {};

// Slots of the binary64 explicit-inverse re-solve: enough for the active sets met (a QP that
// needs more falls back to the Cholesky form) while its workspace stays within the binary32
// one for 16 to 32 robots, so that the union below does not grow there (8 robots: about 1 KB
// more per team).
template <int NMAX>
constexpr int f64_inv_slots() { return NMAX <= 8 ? 2 * NMAX : (NMAX <= 20 ? 24 : 32); }

// binary64 explicit-inverse re-solve work: the QP data the solver reads (points, u) and its
// factors.
template <int NMAX>
struct F64Inv {
    double px[NMAX], py[NMAX], ux[NMAX], uy[NMAX], u0x[NMAX], u0y[NMAX];
    InvWork<NMAX, double, f64_inv_slots<NMAX>()> inv;
};

// binary32 work (the QP data and, for teams over 4 robots, the explicit-inverse factors)
// overlays the binary64 re-solve work: the re-solve starts after the binary32 result is read.
template <int NMAX>
struct F32Work {
    QPWork<float, NMAX> f;
    typename std::conditional<(NMAX > 4), InvWork<NMAX>, NoInvWork>::type inv;
};

template <int NMAX>
union QPUnion {
    F32Work<NMAX> s;
    QPWork<double, NMAX> d;
    typename std::conditional<(NMAX > 4), F64Inv<NMAX>, NoInvWork>::type di;
};

template <typename R, int NMAX>
struct TeamSmem {
    float4 g4[2][4][2];  // 4-robot Navigation kernel: per-robot state published each step
    float2 g2[4];        // (two buffers, alternating) and nominal velocities
    QPUnion<NMAX> qp;
    R sx[NMAX], sy[NMAX], sth[NMAX];
    int slevel[NMAX];
    R qx[kMaxRes], qy[kMaxRes];
    int qlevel[kMaxRes], qactive[kMaxRes];
    float fx[NMAX], fy[NMAX], fth[NMAX];
};

template <typename Q, int NMAX>
struct WorkSel;
template <int NMAX>
struct WorkSel<float, NMAX> {
    static __device__ __forceinline__ QPWork<float, NMAX>& get(QPUnion<NMAX>& u) { return u.s.f; }
};
template <int NMAX>
struct WorkSel<double, NMAX> {
    static __device__ __forceinline__ QPWork<double, NMAX>& get(QPUnion<NMAX>& u) { return u.d; }
};

template <typename Q>
struct QPConsts {
    Q gamma, r2, kg, half_r, xmin, xmax, ymin, ymax, tol_abs, tol_rel, eps_dep, tol_lam, h_flag;
    int max_iter;
};

struct QPResult {
    int status;  // 0 ok, 1 infeasible, 2 iteration cap or numerical failure
    int q;       // active rows
    int iters;
    bool flag;   // needs the binary64 re-solve (binary32 only)
};

template <typename Q>
__device__ __forceinline__ Q qinf() { return (Q)CUDART_INF; }
template <>
__device__ __forceinline__ float qinf<float>() { return CUDART_INF_F; }

__device__ __forceinline__ float qsqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ double qsqrt(double v) { return sqrt(v); }

// Coefficients of one QP row: (ax, ay) on u_ia and, for a pair row, (-ax, -ay) on u_ib.
template <typename Q>
__device__ __forceinline__ Q row_dot(int ia1, int ib1, Q ax1, Q ay1, int ia2, int ib2, Q ax2,
                                     Q ay2) {
    const Q cc = ax1 * ax2 + ay1 * ay2;
    Q d = (Q)0;
    if (ia1 == ia2) d += cc;
    if (ib1 >= 0 && ib1 == ia2) d -= cc;
    if (ib2 >= 0 && ia1 == ib2) d -= cc;
    if (ib1 >= 0 && ib1 == ib2) d += cc;
    return d;
}

__device__ __forceinline__ int pair_index(int a, int b, int N) {
    return a * N - (a * (a + 1)) / 2 + (b - a - 1);
}

// Pair (a, b), a < b, of the lexicographic index k < N(N-1)/2.
__device__ __forceinline__ void pair_of(int k, int N, int& a, int& b) {
    int rem = k, i = 0;
    while (rem >= N - 1 - i) {
        rem -= N - 1 - i;
        ++i;
    }
    a = i;
    b = i + 1 + rem;
}

template <typename Q>
struct RowInfo {
    int k, ia, ib;
    Q ax, ay, b;
};

template <typename Q, int NMAX>
__device__ __forceinline__ RowInfo<Q> decode_row(const QPWork<Q, NMAX>& W, int k, int N,
                                                 const QPConsts<Q>& c) {
    RowInfo<Q> r;
    r.k = k;
    const int P = N * (N - 1) / 2;
    if (k < P) {
        int a, b;
        pair_of(k, N, a, b);
        const Q dx = W.px[a] - W.px[b], dy = W.py[a] - W.py[b];
        const Q h = dx * dx + dy * dy - c.r2;
        r.ia = a;
        r.ib = b;
        r.ax = (Q)-2 * dx;
        r.ay = (Q)-2 * dy;
        r.b = c.gamma * h * h * h;
    } else {
        const int i = (k - P) >> 2, s = (k - P) & 3;
        r.ia = i;
        r.ib = -1;
        Q d;
        if (s == 0) { r.ax = (Q)1; r.ay = (Q)0; d = c.xmax - c.half_r - W.px[i]; }
        else if (s == 1) { r.ax = (Q)-1; r.ay = (Q)0; d = W.px[i] - c.xmin - c.half_r; }
        else if (s == 2) { r.ax = (Q)0; r.ay = (Q)1; d = c.ymax - c.half_r - W.py[i]; }
        else { r.ax = (Q)0; r.ay = (Q)-1; d = W.py[i] - c.ymin - c.half_r; }
        r.b = c.kg * d * d * d;
    }
    return r;
}

// Most violated inactive row (violation beyond tolerance); key INT_MAX if none.
template <typename Q, int G, int NMAX>
__device__ __forceinline__ void scan_rows(const Team<G>& tm, const QPWork<Q, NMAX>& W, int N,
                                          const QPConsts<Q>& c, Q& vbest, int& kbest) {
    constexpr int RPL = (NMAX + G - 1) / G;
    const int P = N * (N - 1) / 2;
    vbest = (Q)0;
    kbest = 0x7fffffff;
    const int nd = (N - 1) / 2;
#pragma unroll
    for (int s = 0; s < RPL; ++s) {
        const int i = tm.lane + s * G;
        if (i < N) {
            const int ndi = nd + (((N & 1) == 0 && i < N / 2) ? 1 : 0);
            for (int d = 1; d <= ndi; ++d) {
                int j = i + d;
                if (j >= N) j -= N;
                const int a = min(i, j), b = max(i, j);
                const int k = pair_index(a, b, N);
                if ((W.actbits[k >> 5] >> (k & 31)) & 1u) continue;
                const Q dx = W.px[a] - W.px[b], dy = W.py[a] - W.py[b];
                const Q h = dx * dx + dy * dy - c.r2;
                const Q bv = c.gamma * h * h * h;
                const Q au = (Q)-2 * (dx * (W.ux[a] - W.ux[b]) + dy * (W.uy[a] - W.uy[b]));
                const Q v = au - bv;
                if (v > c.tol_abs + c.tol_rel * fabs(bv) && (v > vbest || (v == vbest && k < kbest))) {
                    vbest = v;
                    kbest = k;
                }
            }
            const Q bx0 = c.xmax - c.half_r - W.px[i], bx1 = W.px[i] - c.xmin - c.half_r;
            const Q by0 = c.ymax - c.half_r - W.py[i], by1 = W.py[i] - c.ymin - c.half_r;
            const Q bvs[4] = {c.kg * bx0 * bx0 * bx0, c.kg * bx1 * bx1 * bx1,
                              c.kg * by0 * by0 * by0, c.kg * by1 * by1 * by1};
            const Q aus[4] = {W.ux[i], -W.ux[i], W.uy[i], -W.uy[i]};
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) {
                const int k = P + 4 * i + q4;
                if ((W.actbits[k >> 5] >> (k & 31)) & 1u) continue;
                const Q v = aus[q4] - bvs[q4];
                if (v > c.tol_abs + c.tol_rel * fabs(bvs[q4]) &&
                    (v > vbest || (v == vbest && k < kbest))) {
                    vbest = v;
                    kbest = k;
                }
            }
        }
    }
    tm.argmax(vbest, kbest);
}

// Cholesky factor of the Gram matrix of the active rows, from scratch (leader lane only).
template <typename Q, int NMAX>
__device__ bool refactor(QPWork<Q, NMAX>& W, int q) {
    constexpr int A = QPWork<Q, NMAX>::A;
    for (int i = 0; i < q; ++i) {
        for (int j = 0; j <= i; ++j) {
            Q s = row_dot(W.ria[i], W.rib[i], W.rax[i], W.ray[i], W.ria[j], W.rib[j], W.rax[j],
                          W.ray[j]);
            for (int k = 0; k < j; ++k) s -= W.L[i * A + k] * W.L[j * A + k];
            if (i == j) {
                if (!(s > (Q)0)) return false;
                W.L[i * A + i] = qsqrt(s);
            } else {
                W.L[i * A + j] = s / W.L[j * A + j];
            }
        }
    }
    return true;
}

// L y = w, then L^T r = y (leader lane only).
template <typename Q, int NMAX>
__device__ __forceinline__ void chol_solve(QPWork<Q, NMAX>& W, int q, const Q* rhs, Q* y, Q* r) {
    constexpr int A = QPWork<Q, NMAX>::A;
    for (int i = 0; i < q; ++i) {
        Q s = rhs[i];
        for (int k = 0; k < i; ++k) s -= W.L[i * A + k] * y[k];
        y[i] = s / W.L[i * A + i];
    }
    for (int i = q - 1; i >= 0; --i) {
        Q s = y[i];
        for (int k = i + 1; k < q; ++k) s -= W.L[k * A + i] * r[k];
        r[i] = s / W.L[i * A + i];
    }
}

// Solve the team's QP.  On entry W.px/py, W.u0x/u0y and W.ux/uy (= u0) hold all N robots and
// the team is synchronised; on exit W.ux/uy hold the minimiser (zero if infeasible), synced.
template <typename Q, int G, int NMAX>
__device__ QPResult qp_solve(const Team<G>& tm, QPWork<Q, NMAX>& W, int N, const QPConsts<Q>& c) {
    constexpr int RPL = (NMAX + G - 1) / G;
    constexpr int A = QPWork<Q, NMAX>::A;
    const int P = N * (N - 1) / 2;
    const int M = P + 4 * N;
    for (int wd = tm.lane; wd < (M + 31) / 32; wd += G) W.actbits[wd] = 0u;
    if (tm.lane == 0) W.fail = 0;
    tm.sync();

    QPResult res;
    res.status = 0;
    res.q = 0;
    res.iters = 0;
    res.flag = false;
    int q = 0;
    const Q INF = qinf<Q>();

    for (;;) {
        Q vbest;
        int kbest;
        scan_rows<Q, G, NMAX>(tm, W, N, c, vbest, kbest);
        if (kbest == 0x7fffffff) break;
        if (++res.iters > c.max_iter || q >= A) {
            res.status = 2;
            break;
        }
        const RowInfo<Q> p = decode_row<Q, NMAX>(W, kbest, N, c);
        const Q app = (p.ib >= 0 ? (Q)2 : (Q)1) * (p.ax * p.ax + p.ay * p.ay);
        Q lam_p = (Q)0;
        bool added = false;
        for (int guard = 0; guard <= A + 1 && !added; ++guard) {
            for (int j = tm.lane; j < q; j += G)
                W.w[j] = row_dot(W.ria[j], W.rib[j], W.rax[j], W.ray[j], p.ia, p.ib, p.ax, p.ay);
            tm.sync();
            if (tm.lane == 0) chol_solve<Q, NMAX>(W, q, W.w, W.yv, W.rv);
            tm.sync();
            // primal direction z on the lane's own robots
            Q zx[RPL], zy[RPL];
            Q zzl = (Q)0;
#pragma unroll
            for (int s = 0; s < RPL; ++s) {
                const int i = tm.lane + s * G;
                Q ax = (Q)0, ay = (Q)0;
                if (i < N) {
                    if (p.ia == i) { ax += p.ax; ay += p.ay; }
                    if (p.ib == i) { ax -= p.ax; ay -= p.ay; }
                    for (int j = 0; j < q; ++j) {
                        const Q rj = W.rv[j];
                        if (W.ria[j] == i) { ax -= rj * W.rax[j]; ay -= rj * W.ray[j]; }
                        if (W.rib[j] == i) { ax += rj * W.rax[j]; ay += rj * W.ray[j]; }
                    }
                }
                zx[s] = ax;
                zy[s] = ay;
                zzl += ax * ax + ay * ay;
            }
            const Q zz = tm.sum(zzl);
            // dual step bound
            Q td = INF;
            int jb = 0x7fffffff;
            for (int j = tm.lane; j < q; j += G) {
                const Q rj = W.rv[j];
                if (rj > (Q)0) {
                    const Q tj = W.lam[j] / rj;
                    if (tj < td || (tj == td && j < jb)) { td = tj; jb = j; }
                }
            }
            tm.argmin(td, jb);
            // current violation of row p
            Q ap_u;
            if (p.ib >= 0)
                ap_u = p.ax * (W.ux[p.ia] - W.ux[p.ib]) + p.ay * (W.uy[p.ia] - W.uy[p.ib]);
            else
                ap_u = p.ax * W.ux[p.ia] + p.ay * W.uy[p.ia];
            const Q sp = ap_u - p.b;
            const bool indep = zz > c.eps_dep * app;
            if (!indep) res.flag = true;
            const Q tf = indep ? sp / zz : INF;
            if (!(tf < INF) && !(td < INF)) {
                res.status = 1;
                break;
            }
            const Q t = tf < td ? tf : td;
            tm.sync();  // everyone has read W.ux / W.rv / W.lam
            if (tf < INF) {
#pragma unroll
                for (int s = 0; s < RPL; ++s) {
                    const int i = tm.lane + s * G;
                    if (i < N) {
                        W.ux[i] -= t * zx[s];
                        W.uy[i] -= t * zy[s];
                    }
                }
            }
            for (int j = tm.lane; j < q; j += G) W.lam[j] -= t * W.rv[j];
            lam_p += t;
            if (tf <= td) {
                if (tm.lane == 0) {
                    for (int jj = 0; jj < q; ++jj) W.L[q * A + jj] = W.yv[jj];
                    W.L[q * A + q] = qsqrt(zz);
                    W.ria[q] = p.ia;
                    W.rib[q] = p.ib;
                    W.rax[q] = p.ax;
                    W.ray[q] = p.ay;
                    W.rb[q] = p.b;
                    W.rk[q] = p.k;
                    W.lam[q] = lam_p;
                    W.actbits[p.k >> 5] |= 1u << (p.k & 31);
                }
                ++q;
                added = true;
            } else {
                tm.sync();
                if (tm.lane == 0) {
                    W.actbits[W.rk[jb] >> 5] &= ~(1u << (W.rk[jb] & 31));
                    for (int j = jb; j < q - 1; ++j) {
                        W.ria[j] = W.ria[j + 1];
                        W.rib[j] = W.rib[j + 1];
                        W.rax[j] = W.rax[j + 1];
                        W.ray[j] = W.ray[j + 1];
                        W.rb[j] = W.rb[j + 1];
                        W.rk[j] = W.rk[j + 1];
                        W.lam[j] = W.lam[j + 1];
                    }
                    if (!refactor<Q, NMAX>(W, q - 1)) W.fail = 1;
                }
                --q;
            }
            tm.sync();
            if (W.fail) {
                res.status = 2;
                break;
            }
        }
        if (res.status != 0) break;
        if (!added) {
            res.status = 2;
            break;
        }
    }
    res.q = q;

    if (std::is_same<Q, double>::value && res.status == 0 && q > 0) {
        // binary64: exact solve on the final active set, G lam = N^T u0 - b_A, u = u0 - N lam
        // (in binary32 the active-set iterate is already as accurate as this re-solve)
        for (int j = tm.lane; j < q; j += G) {
            Q au0;
            if (W.rib[j] >= 0)
                au0 = W.rax[j] * (W.u0x[W.ria[j]] - W.u0x[W.rib[j]]) +
                      W.ray[j] * (W.u0y[W.ria[j]] - W.u0y[W.rib[j]]);
            else
                au0 = W.rax[j] * W.u0x[W.ria[j]] + W.ray[j] * W.u0y[W.ria[j]];
            W.w[j] = au0 - W.rb[j];
        }
        tm.sync();
        if (tm.lane == 0) {
            chol_solve<Q, NMAX>(W, q, W.w, W.yv, W.rv);
            int bad = 0;
            for (int j = 0; j < q; ++j)
                if (W.rv[j] < -c.tol_lam) bad = 1;
            W.fail = bad;
        }
        tm.sync();
        const bool dual_ok = (W.fail == 0);
        Q keepx[RPL], keepy[RPL];
        if (dual_ok) {
#pragma unroll
            for (int s = 0; s < RPL; ++s) {
                const int i = tm.lane + s * G;
                keepx[s] = (Q)0;
                keepy[s] = (Q)0;
                if (i < N) {
                    Q ux = W.u0x[i], uy = W.u0y[i];
                    for (int j = 0; j < q; ++j) {
                        const Q lj = W.rv[j];
                        if (W.ria[j] == i) { ux -= lj * W.rax[j]; uy -= lj * W.ray[j]; }
                        if (W.rib[j] == i) { ux += lj * W.rax[j]; uy += lj * W.ray[j]; }
                    }
                    keepx[s] = W.ux[i];
                    keepy[s] = W.uy[i];
                    W.ux[i] = ux;
                    W.uy[i] = uy;
                }
            }
            tm.sync();
            // the polished point must stay feasible; otherwise keep the active-set iterate
            for (int wd = tm.lane; wd < (M + 31) / 32; wd += G) W.actbits[wd] = 0u;
            tm.sync();
            Q vb;
            int kb;
            scan_rows<Q, G, NMAX>(tm, W, N, c, vb, kb);
            tm.sync();
            if (kb != 0x7fffffff) {
#pragma unroll
                for (int s = 0; s < RPL; ++s) {
                    const int i = tm.lane + s * G;
                    if (i < N) {
                        W.ux[i] = keepx[s];
                        W.uy[i] = keepy[s];
                    }
                }
            }
        }
    }
    if (res.status == 0 && q > 0) {
        // an active pair with h below h_flag marks the QP near-degenerate
        bool small_h = false;
        for (int j = tm.lane; j < q; j += G) {
            if (W.rib[j] >= 0) {
                const Q dx = W.px[W.ria[j]] - W.px[W.rib[j]], dy = W.py[W.ria[j]] - W.py[W.rib[j]];
                if (dx * dx + dy * dy - c.r2 < c.h_flag) small_h = true;
            }
        }
        if (tm.any(small_h)) res.flag = true;
    }
    if (res.status == 1) {
#pragma unroll
        for (int s = 0; s < RPL; ++s) {
            const int i = tm.lane + s * G;
            if (i < N) {
                W.ux[i] = (Q)0;
                W.uy[i] = (Q)0;
            }
        }
    }
    if (res.status != 0) res.flag = true;
    tm.sync();
    return res;
}

// ------------------------------------------------------------------------------------------
// The same dual active-set method in explicit-inverse form (teams of 8..32 lanes: the binary32
// solve, and the binary64 re-solve of the 8..20-robot classes).
// With N the active rows (as columns) and G = N^T N, it keeps B = G^-1 and M = N B in shared
// memory, indexed by slot.  Then r = G^-1 N^T a_p = M^T a_p needs only the (at most four)
// non-zeros of a_p -- one lane per active row, no sequential triangular solve -- and the block-
// inverse identities update both in O(n q):
//   add a_p (z = a_p - N r, s = |z|^2):  M <- [M - z r^T / s, z / s],
//                                        B <- [[B + r r^T / s, -r / s], [-r^T / s, 1 / s]];
//   drop row j:  M <- M_{:,-j} - M_{:,j} B_{j,-j} / B_jj,  B <- B_{-j,-j} - B_{-j,j} B_{j,-j} / B_jj.
// ------------------------------------------------------------------------------------------

// The barrier rows one lane evaluates in qp_solve_inv (teams with one robot per lane): its
// circulant pair rows (partner, p_i - p_j, bound, key) and its four arena rows, computed once per
// QP; a row in the active set (or absent) carries an infinite threshold.  key = row index * 32 +
// lane: it names the row in the active set and the lane holding it.
template <int NMAX, typename Q = float>
struct LaneRows {
    static constexpr int PR = NMAX / 2 > 0 ? NMAX / 2 : 1;
    // dx, dy: p_i - p_j (the lane's robot first); thr: the violation threshold, +inf for a row
    // that is absent or in the active set (so that a scan skips it without a test)
    Q dx[PR], dy[PR], bp[PR], thr[PR];
    int j[PR], key[PR];
    Q bb[4], bthr[4];
    int bkey[4];
    int np;
};

template <int NMAX, typename Q>
__device__ __forceinline__ void lane_rows_init(LaneRows<NMAX, Q>& R, int i, int N, const Q* px,
                                               const Q* py, const QPConsts<Q>& c) {
    const int nd = (N - 1) / 2;
    R.np = (i < N) ? nd + (((N & 1) == 0 && i < N / 2) ? 1 : 0) : 0;
    const int P = N * (N - 1) / 2;
#pragma unroll
    for (int d = 0; d < LaneRows<NMAX, Q>::PR; ++d) {
        int j = i + d + 1;
        while (j >= N) j -= N;
        if (d >= R.np) j = i;
        const int a = min(i, j), b = max(i, j);
        R.j[d] = j;
        R.key[d] = (d < R.np) ? pair_index(a, b, N) * 32 + (i & 31) : 0x7fffffff;
        R.dx[d] = px[i < N ? i : 0] - px[j < N ? j : 0];
        R.dy[d] = py[i < N ? i : 0] - py[j < N ? j : 0];
        const Q h = R.dx[d] * R.dx[d] + R.dy[d] * R.dy[d] - c.r2;
        R.bp[d] = c.gamma * h * h * h;
        R.thr[d] = (d < R.np) ? c.tol_abs + c.tol_rel * fabs(R.bp[d]) : qinf<Q>();
    }
    const Q pxi = px[i < N ? i : 0], pyi = py[i < N ? i : 0];
    const Q bx0 = c.xmax - c.half_r - pxi, bx1 = pxi - c.xmin - c.half_r;
    const Q by0 = c.ymax - c.half_r - pyi, by1 = pyi - c.ymin - c.half_r;
    R.bb[0] = c.kg * bx0 * bx0 * bx0;
    R.bb[1] = c.kg * bx1 * bx1 * bx1;
    R.bb[2] = c.kg * by0 * by0 * by0;
    R.bb[3] = c.kg * by1 * by1 * by1;
#pragma unroll
    for (int s = 0; s < 4; ++s) R.bthr[s] = (i < N) ? c.tol_abs + c.tol_rel * fabs(R.bb[s]) : qinf<Q>();
#pragma unroll
    for (int s = 0; s < 4; ++s) R.bkey[s] = (i < N) ? (P + 4 * i + s) * 32 + (i & 31) : 0x7fffffff;
}

// Most violated inactive row of the team at u (shared memory), its descriptor broadcast from
// the lane that holds it.  Returns false when every row holds.
template <typename Q, int G, int NMAX>
__device__ __forceinline__ bool scan_cached(const Team<G>& tm, const LaneRows<NMAX, Q>& R, int i,
                                            const Q* ux, const Q* uy, const QPConsts<Q>& c,
                                            RowInfo<Q>& p, Q& vbest) {
    constexpr int PR = LaneRows<NMAX, Q>::PR;
    // the lane's most violated row: pair row d, or PR + arena side (ties: the first in that
    // order; only the order of the iterations depends on it)
    Q vb = (Q)0;
    int db = -1;
    if (R.np > 0 || (R.bkey[0] != 0x7fffffff)) {
        const Q uxi = ux[i], uyi = uy[i];
#pragma unroll
        for (int d = 0; d < PR; ++d) {
            const int j = R.j[d];
            const Q v = (Q)-2 * (R.dx[d] * (uxi - ux[j]) + R.dy[d] * (uyi - uy[j])) - R.bp[d];
            if (v > (R.thr[d] > vb ? R.thr[d] : vb)) {
                vb = v;
                db = d;
            }
        }
        const Q aus[4] = {uxi, -uxi, uyi, -uyi};
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const Q v = aus[s] - R.bb[s];
            if (v > (R.bthr[s] > vb ? R.bthr[s] : vb)) {
                vb = v;
                db = PR + s;
            }
        }
    }
    // the chosen row's descriptor: key, robots a < b, p_a - p_b and bound (arena side s:
    // b = -1 - s)
    int kb = 0x7fffffff, ba = i, bbv = -1;
    Q bdx = (Q)0, bdy = (Q)0, bbound = (Q)0;
#pragma unroll
    for (int d = 0; d < PR; ++d)
        if (d == db) {
            const int j = R.j[d];
            const Q sg = (i < j) ? (Q)1 : (Q)-1;
            kb = R.key[d];
            ba = min(i, j);
            bbv = max(i, j);
            bdx = sg * R.dx[d];
            bdy = sg * R.dy[d];
            bbound = R.bp[d];
        }
#pragma unroll
    for (int s = 0; s < 4; ++s)
        if (db == PR + s) {
            kb = R.bkey[s];
            bbv = -1 - s;
            bbound = R.bb[s];
        }
    // the team's largest violation (non-negative floats order as their bits; a binary64 one is
    // compared rounded to binary32, which only orders the iterations), held by the lowest lane
    // that has it
    const unsigned vbits = __float_as_uint((float)vb);
    const unsigned vmax = __reduce_max_sync(tm.mask, vbits);
    if (vmax == 0u) return false;
    const int own = (__ffs(__ballot_sync(tm.mask, vbits == vmax)) - 1) & (G - 1);
    vbest = __shfl_sync(tm.mask, vb, own, G);
    kb = __shfl_sync(tm.mask, kb, own, G);
    const int a = __shfl_sync(tm.mask, ba, own, G), b = __shfl_sync(tm.mask, bbv, own, G);
    const Q dx = __shfl_sync(tm.mask, bdx, own, G), dy = __shfl_sync(tm.mask, bdy, own, G);
    p.b = __shfl_sync(tm.mask, bbound, own, G);
    p.k = kb;
    p.ia = a;
    if (b >= 0) {
        p.ib = b;
        p.ax = (Q)-2 * dx;
        p.ay = (Q)-2 * dy;
    } else {
        const int s = -1 - b;
        p.ib = -1;
        p.ax = (s == 0) ? (Q)1 : (s == 1) ? (Q)-1 : (Q)0;
        p.ay = (s == 2) ? (Q)1 : (s == 3) ? (Q)-1 : (Q)0;
    }
    return true;
}

// Mark row key k active (its threshold +inf: the scans skip it) or inactive (its threshold
// back) in the lane that holds it.
template <int NMAX, typename Q>
__device__ __forceinline__ void lane_rows_mark(LaneRows<NMAX, Q>& R, int k, bool on,
                                               const QPConsts<Q>& c) {
#pragma unroll
    for (int d = 0; d < LaneRows<NMAX, Q>::PR; ++d)
        if (R.key[d] == k) R.thr[d] = on ? qinf<Q>() : c.tol_abs + c.tol_rel * fabs(R.bp[d]);
#pragma unroll
    for (int s = 0; s < 4; ++s)
        if (R.bkey[s] == k) R.bthr[s] = on ? qinf<Q>() : c.tol_abs + c.tol_rel * fabs(R.bb[s]);
}

// a / b for a step length: the hardware quotient in binary32 (about 2 ulp; a length only
// scales a step), the correctly rounded one in binary64.
__device__ __forceinline__ float step_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double step_div(double a, double b) { return a / b; }

// Order-preserving map of a float to an unsigned key (for redux.sync minima).
__device__ __forceinline__ unsigned float_order_key(float v) {
    const unsigned b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Every lane of the team gets the minimum of v over the team and the team lane that holds it
// (the lowest such lane).
template <int G>
__device__ __forceinline__ int team_min_lane(const Team<G>& tm, float v) {
    const unsigned k = float_order_key(v);
    const unsigned m = __reduce_min_sync(tm.mask, k);
    return (__ffs(__ballot_sync(tm.mask, k == m)) - 1) & (G - 1);
}

// Warm start of the dual active-set method from a given active set A (used by the binary64
// re-solve of a flagged QP, started from the binary32 solve's final active set: each binary64
// iteration is costly, and that set is the answer or close to it).  The method may start from
// any active set of independent rows whose equality-constrained minimiser has nonnegative
// multipliers (Goldfarb-Idnani 1983): here the rows of A at the current points (lane i holds row
// i: robots wa < wb, or arena side wside of robot wa when wb < 0, and its key), their Gram matrix
// G = N^T N inverted in place by Gauss-Jordan elimination (one row per lane; the pivots are the
// |z|^2 the iteration tests for dependence), lam = G^-1 (N^T u0 - b), M = N G^-1,
// u = u0 - N lam.  A dependent row or a negative multiplier rejects the start (returns 0: the
// solve begins from the empty set, nothing of it kept); else the factors, multipliers, slots,
// incidence masks and row marks are those the iteration would hold with A active, and it
// returns |A|.
template <typename Q, int G, int NMAX, int AS, class UW>
__device__ int qp_warm_start(const Team<G>& tm, InvWork<NMAX, Q, AS>& W, int N,
                             const QPConsts<Q>& c, UW& Wscan, LaneRows<NMAX, Q>& LR, int q0,
                             int wa, int wb, int wside, int wkey) {
    const int i = tm.lane;  // row i of A (i < q0) and robot i (i < N)
    Q rax = (Q)0, ray = (Q)0, rbd = (Q)0;
    if (i < q0) {
        if (wb >= 0) {
            const Q dx = Wscan.px[wa] - Wscan.px[wb], dy = Wscan.py[wa] - Wscan.py[wb];
            const Q h = dx * dx + dy * dy - c.r2;
            rax = (Q)-2 * dx;
            ray = (Q)-2 * dy;
            rbd = c.gamma * h * h * h;
        } else {
            const Q pxi = Wscan.px[wa], pyi = Wscan.py[wa];
            rax = (wside == 0) ? (Q)1 : (wside == 1) ? (Q)-1 : (Q)0;
            ray = (wside == 2) ? (Q)1 : (wside == 3) ? (Q)-1 : (Q)0;
            const Q d = (wside == 0) ? c.xmax - c.half_r - pxi
                      : (wside == 1) ? pxi - c.xmin - c.half_r
                      : (wside == 2) ? c.ymax - c.half_r - pyi
                                     : pyi - c.ymin - c.half_r;
            rbd = c.kg * d * d * d;
        }
        W.sia[i] = wa;
        W.sib[i] = wb;
        W.sk[i] = wkey;
        W.sax[i] = rax;
        W.say[i] = ray;
        W.sb[i] = rbd;
        W.act[i] = i;
    }
    tm.sync();
    // G (row i per lane): a_t = e_t at robot sia_t and -e_t at sib_t
    if (i < q0) {
        for (int u = 0; u < q0; ++u) {
            const int ua = W.sia[u], ub = W.sib[u];
            const int sg = (wa == ua ? 1 : 0) - (wa == ub ? 1 : 0) +
                           (wb >= 0 ? ((wb == ub ? 1 : 0) - (wb == ua ? 1 : 0)) : 0);
            W.Bi[i][u] = (Q)sg * (rax * W.sax[u] + ray * W.say[u]);
        }
        W.r[i] = W.Bi[i][i];  // |a_i|^2, the scale of the pivot test
    }
    tm.sync();
    bool ok = true;
    for (int kk = 0; kk < q0 && ok; ++kk) {
        const Q pv = W.Bi[kk][kk];
        ok = pv > c.eps_dep * W.r[kk];
        const Q d = (Q)1 / pv;
        tm.sync();
        if (ok && i == kk) {
            for (int j = 0; j < q0; ++j) W.Bi[kk][j] *= d;
            W.Bi[kk][kk] = d;
        }
        tm.sync();
        if (ok && i < q0 && i != kk) {
            const Q f = W.Bi[i][kk];
            W.Bi[i][kk] = (Q)0;
            for (int j = 0; j < q0; ++j) W.Bi[i][j] -= f * W.Bi[kk][j];
        }
        tm.sync();
    }
    if (!ok) return 0;
    // lam = G^-1 (N^T u0 - b): u still holds u0
    if (i < q0) {
        Q au = rax * Wscan.ux[wa] + ray * Wscan.uy[wa];
        if (wb >= 0) au -= rax * Wscan.ux[wb] + ray * Wscan.uy[wb];
        W.r[i] = au - rbd;
    }
    tm.sync();
    Q lam = (Q)0;
    if (i < q0)
        for (int u = 0; u < q0; ++u) lam += W.Bi[i][u] * W.r[u];
    if (__any_sync(tm.mask, i < q0 && lam < -c.tol_lam)) return 0;
    lam = lam > (Q)0 ? lam : (Q)0;
    // M = N G^-1 (column i per lane), the multipliers, the incidence masks
    if (i < q0) {
        for (int v = 0; v < 2 * N; ++v) W.Mi[v][i] = (Q)0;
        for (int u = 0; u < q0; ++u) {
            const Q w = W.Bi[u][i];
            const int ua = W.sia[u], ub = W.sib[u];
            const Q ex = w * W.sax[u], ey = w * W.say[u];
            W.Mi[2 * ua][i] += ex;
            W.Mi[2 * ua + 1][i] += ey;
            if (ub >= 0) {
                W.Mi[2 * ub][i] -= ex;
                W.Mi[2 * ub + 1][i] -= ey;
            }
        }
        W.lam[i] = lam;
        atomicOr(&W.inc[wa], 1ull << i);
        if (wb >= 0) atomicOr(&W.inc[wb], 1ull << i);
    }
    if (i == 0) W.free_slots &= ~((q0 >= 64) ? ~0ull : ((1ull << q0) - 1ull));
    tm.sync();
    // u = u0 - N lam on the lane's robot
    if (i < N) {
        Q ux = Wscan.ux[i], uy = Wscan.uy[i];
        for (unsigned long long m = W.inc[i]; m; m &= m - 1ull) {
            const int t = __ffsll((long long)m) - 1;
            const Q lt = W.sia[t] == i ? W.lam[t] : -W.lam[t];
            ux -= lt * W.sax[t];
            uy -= lt * W.say[t];
        }
        Wscan.ux[i] = ux;
        Wscan.uy[i] = uy;
    }
    // the rows of A marked active in the lanes that hold them (key: row index * 32 + lane)
    for (int u = 0; u < q0; ++u) {
        const int k = W.sk[u];
        if ((k & 31) == (i & 31)) lane_rows_mark<NMAX, Q>(LR, k, true, c);
    }
    tm.sync();
    return q0;
}

// The work of one iteration is spread so that no lane walks the active set serially: the team
// maxima and minima are redux.sync reductions; z, a robot's share of a_p - N r, comes from that
// robot's own incident active rows (a bit mask per robot); the rank-one updates of M and B run
// one active slot per lane over the variables.
// Q: binary32 (the step's solver) or binary64 (the re-solve of a flagged QP); UW holds the
// points and u (px, py, ux, uy per robot).  A QP whose active set outgrows the AS slots ends
// with status 2.  warm_q > 0 (binary64 only): start from the active set of warm_q rows that the
// lanes hold (qp_warm_start) instead of the empty set.
template <typename Q, int G, int NMAX, int AS, class UW>
__device__ QPResult qp_solve_inv(const Team<G>& tm, InvWork<NMAX, Q, AS>& W, int N,
                                 const QPConsts<Q>& c, UW& Wscan, int warm_q = 0, int wa = 0,
                                 int wb = -1, int wside = 0, int wkey = 0x7fffffff) {
    static_assert(G >= NMAX, "qp_solve_inv holds one robot per lane");
    const int i = tm.lane;  // the lane's robot
    if (i == 0) W.free_slots = (AS >= 64) ? ~0ull : ((1ull << AS) - 1ull);
    if (i < NMAX) W.inc[i] = 0ull;
    tm.sync();
    QPResult res;
    res.status = 0;
    res.q = 0;
    res.iters = 0;
    res.flag = false;
    int q = 0;
    LaneRows<NMAX, Q> LR;
    lane_rows_init<NMAX, Q>(LR, i, N, Wscan.px, Wscan.py, c);
    if constexpr (!std::is_same<Q, float>::value) {
        if (warm_q > 0 && warm_q <= G && warm_q <= AS)
            q = qp_warm_start<Q, G, NMAX, AS, UW>(tm, W, N, c, Wscan, LR, warm_q, wa, wb, wside,
                                                  wkey);
    }
    for (;;) {
        Q vbest;
        RowInfo<Q> p;
        if (!scan_cached<Q, G, NMAX>(tm, LR, i, Wscan.ux, Wscan.uy, c, p, vbest)) break;
        if (++res.iters > c.max_iter || q >= AS) { res.status = 2; break; }
        const Q app = (p.ib >= 0 ? (Q)2 : (Q)1) * (p.ax * p.ax + p.ay * p.ay);
        // non-zeros of a_p: (variable, value)
        const int v0 = 2 * p.ia, v1 = 2 * p.ia + 1;
        const int v2 = p.ib >= 0 ? 2 * p.ib : v0, v3 = p.ib >= 0 ? 2 * p.ib + 1 : v1;
        const Q a0 = p.ax, a1 = p.ay, a2 = p.ib >= 0 ? -p.ax : (Q)0, a3 = p.ib >= 0 ? -p.ay : (Q)0;
        Q lam_p = (Q)0;
        bool added = false;
        for (int guard = 0; guard <= AS + 1 && !added; ++guard) {
            // r = M^T a_p over the active slots, one slot per lane
            for (int idx = i; idx < q; idx += G) {
                const int t = W.act[idx];
                W.r[t] = W.Mi[v0][t] * a0 + W.Mi[v1][t] * a1 + W.Mi[v2][t] * a2 + W.Mi[v3][t] * a3;
            }
            tm.sync();
            // z = a_p - N r on the lane's robot: a_t is (sax, say) at robot sia, minus that at sib
            Q zx = (Q)0, zy = (Q)0;
            if (i < N) {
                if (p.ia == i) { zx += p.ax; zy += p.ay; }
                if (p.ib == i) { zx -= p.ax; zy -= p.ay; }
                unsigned long long m = W.inc[i];
                while (m) {
                    const int t = __ffsll((long long)m) - 1;
                    m &= m - 1ull;
                    const Q rt = W.sia[t] == i ? -W.r[t] : W.r[t];
                    zx += rt * W.sax[t];
                    zy += rt * W.say[t];
                }
            }
            const Q zz = tm.sum(zx * zx + zy * zy);
            // the blocking multiplier: min over active slots with r > 0 of lam / r
            Q td = qinf<Q>();
            int jb = 0x7fffffff;
            for (int idx = i; idx < q; idx += G) {
                const int t = W.act[idx];
                const Q rt = W.r[t];
                if (rt > (Q)1e-30) {  // a smaller positive r blocks only an unbounded step
                    const Q tj = step_div(W.lam[t], rt);
                    if (tj < td || (tj == td && idx < jb)) { td = tj; jb = idx; }
                }
            }
            if constexpr (std::is_same<Q, float>::value) {
                const int own = team_min_lane(tm, td);
                td = __shfl_sync(tm.mask, td, own, G);
                jb = __shfl_sync(tm.mask, jb, own, G);
            } else {
                tm.argmin(td, jb);
            }
            Q apu;
            if (p.ib >= 0)
                apu = p.ax * (Wscan.ux[p.ia] - Wscan.ux[p.ib]) + p.ay * (Wscan.uy[p.ia] - Wscan.uy[p.ib]);
            else
                apu = p.ax * Wscan.ux[p.ia] + p.ay * Wscan.uy[p.ia];
            const Q sp = apu - p.b;
            const bool indep = zz > c.eps_dep * app;
            if (!indep) res.flag = true;
            const Q tf = indep ? step_div(sp, zz) : qinf<Q>();
            if (!(tf < qinf<Q>()) && !(td < qinf<Q>())) { res.status = 1; break; }
            const Q st = tf < td ? tf : td;
            tm.sync();  // every lane is done reading u, r, lam
            if (tf < qinf<Q>() && i < N) {
                Wscan.ux[i] -= st * zx;
                Wscan.uy[i] -= st * zy;
            }
            for (int idx = i; idx < q; idx += G) {
                const int t = W.act[idx];
                W.lam[t] -= st * W.r[t];
            }
            lam_p += st;
            if (tf <= td) {
                // add a_p in a free slot
                const int sn = __ffsll((long long)W.free_slots) - 1;
                const Q inv = (Q)1 / zz;
                if (i < N) {
                    W.zx[i] = zx;
                    W.zy[i] = zy;
                    W.Mi[2 * i][sn] = zx * inv;      // the new column z / zz
                    W.Mi[2 * i + 1][sn] = zy * inv;
                }
                // the robots where z is non-zero (z and r are sparse: rows of other clusters
                // of robots keep exact zeros in M, B and r, so skipping them changes nothing)
                unsigned zm = __ballot_sync(tm.mask, i < N && (zx != (Q)0 || zy != (Q)0));
                zm = (G == 32) ? zm : ((zm >> tm.base) & ((1u << G) - 1u));
                tm.sync();
                // M <- [M - z r^T / zz, z / zz] and B <- [[B + r r^T / zz, -r / zz], ...],
                // one active slot per lane
                for (int idx = i; idx < q; idx += G) {
                    const int t = W.act[idx];
                    const Q rt = W.r[t] * inv;
                    if (rt != (Q)0) {
                        for (unsigned m = zm; m; m &= m - 1u) {
                            const int k = __ffs(m) - 1;
                            W.Mi[2 * k][t] -= W.zx[k] * rt;
                            W.Mi[2 * k + 1][t] -= W.zy[k] * rt;
                        }
#pragma unroll 4
                        for (int jdx = 0; jdx < q; ++jdx) {
                            const int u = W.act[jdx];
                            W.Bi[t][u] += rt * W.r[u];
                        }
                    }
                    W.Bi[t][sn] = -rt;
                    W.Bi[sn][t] = -rt;
                }
                if (i < N && (i == p.ia || i == p.ib)) W.inc[i] |= 1ull << sn;
                tm.sync();
                if (i == 0) {
                    W.Bi[sn][sn] = inv;
                    W.sia[sn] = p.ia;
                    W.sib[sn] = p.ib;
                    W.sax[sn] = p.ax;
                    W.say[sn] = p.ay;
                    W.sb[sn] = p.b;
                    W.sk[sn] = p.k;
                    W.lam[sn] = lam_p;
                    W.act[q] = sn;
                    W.free_slots &= ~(1ull << sn);
                }
                lane_rows_mark<NMAX, Q>(LR, p.k, true, c);
                ++q;
                added = true;
            } else {
                // drop the blocking row (list position jb, slot j)
                const int j = W.act[jb];
                tm.sync();
                const Q bjj = W.Bi[j][j];
                const Q ibjj = (Q)1 / bjj;
                // the robots where column j of M is non-zero (as above: exact zeros elsewhere)
                unsigned mm = __ballot_sync(tm.mask, i < N && (W.Mi[2 * i][j] != (Q)0 ||
                                                               W.Mi[2 * i + 1][j] != (Q)0));
                mm = (G == 32) ? mm : ((mm >> tm.base) & ((1u << G) - 1u));
                // M <- M_{:,-j} - M_{:,j} B_{j,-j} / B_jj and
                // B <- B_{-j,-j} - B_{-j,j} B_{j,-j} / B_jj, one slot t != j per lane (column and
                // row j are only read)
                for (int idx = i; idx < q; idx += G) {
                    const int t = W.act[idx];
                    if (t == j) continue;
                    const Q bjt = W.Bi[j][t] * ibjj;
                    if (bjt != (Q)0) {
                        for (unsigned m = mm; m; m &= m - 1u) {
                            const int k = __ffs(m) - 1;
                            W.Mi[2 * k][t] -= W.Mi[2 * k][j] * bjt;
                            W.Mi[2 * k + 1][t] -= W.Mi[2 * k + 1][j] * bjt;
                        }
                    }
                    const Q btj = W.Bi[t][j] * ibjj;
                    if (btj != (Q)0) {
#pragma unroll 4
                        for (int jdx = 0; jdx < q; ++jdx) {
                            const int u = W.act[jdx];
                            if (u != j) W.Bi[t][u] -= btj * W.Bi[j][u];
                        }
                    }
                }
                if (i < N && (i == W.sia[j] || i == W.sib[j])) W.inc[i] &= ~(1ull << j);
                lane_rows_mark<NMAX, Q>(LR, W.sk[j], false, c);
                tm.sync();
                if (i == 0) {
                    for (int idx = jb; idx < q - 1; ++idx) W.act[idx] = W.act[idx + 1];
                    W.free_slots |= 1ull << j;
                }
                --q;
                if (!(bjj > (Q)0)) res.status = 2;
            }
            tm.sync();
            if (res.status != 0) break;
        }
        if (res.status != 0) break;
        if (!added) { res.status = 2; break; }
    }
    res.q = q;
    if (res.status == 0 && q > 0) {
        bool small_h = false;
        for (int idx = i; idx < q; idx += G) {
            const int t = W.act[idx];
            if (W.sib[t] >= 0) {
                const Q dx = Wscan.px[W.sia[t]] - Wscan.px[W.sib[t]];
                const Q dy = Wscan.py[W.sia[t]] - Wscan.py[W.sib[t]];
                if (dx * dx + dy * dy - c.r2 < c.h_flag) small_h = true;
            }
        }
        if (tm.any(small_h)) res.flag = true;
    }
    if (res.status == 1 && i < N) {
        Wscan.ux[i] = (Q)0;
        Wscan.uy[i] = (Q)0;
    }
    if (res.status != 0) res.flag = true;
    tm.sync();
    return res;
}

// ------------------------------------------------------------------------------------------
// Small helpers
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void sc_(float v, float* s, float* c) { sincosf(v, s, c); }
__device__ __forceinline__ void sc_(double v, double* s, double* c) { sincos(v, s, c); }

template <typename R>
__device__ __forceinline__ void cap_norm(R& ux, R& uy, R m) {
    const R n2 = ux * ux + uy * uy;
    if (n2 > m * m) {
        const R s = m / qsqrt(n2);
        ux *= s;
        uy *= s;
    }
}

template <typename R>
__device__ __forceinline__ R wrap_pi(R a) {
    const R pi = (R)CUDART_PI, two_pi = (R)(2.0 * CUDART_PI);
    if (a > pi) a -= two_pi;
    else if (a <= -pi) a += two_pi;
    return a;
}

template <typename R>
__device__ __forceinline__ R hyp(R a, R b) { return qsqrt(a * a + b * b); }

// ------------------------------------------------------------------------------------------
// Reset sampler (binary32, every operation rounded on its own)
// ------------------------------------------------------------------------------------------
template <typename R, int G, int NMAX>
__device__ void team_sample(const Team<G>& tm, TeamSmem<R, NMAX>& S, const LaunchArgs<R>& A,
                            int e, int ep, int N, int& n_res) {
    const SamplerConsts& sc = A.sc;
    const uint64_t seed = A.seed;
    const int max_att = A.k.max_attempts;
    if (tm.lane == 0) {
        const Words4 w = draw(seed, e, ep, kPos, 0, 0u);
        S.fx[0] = __fadd_rn(sc.lox, __fmul_rn(unit24(w.w[0]), sc.wx));
        S.fy[0] = __fadd_rn(sc.loy, __fmul_rn(unit24(w.w[1]), sc.wy));
        S.fth[0] = __fadd_rn(-sc.pif, __fmul_rn(unit24(w.w[2]), sc.twopif));
    }
    tm.sync();
    int first = 1;
    if (N >= 2 && sc.near_on) {
        const Words4 w = draw(seed, e, ep, kNear, 0, 0u);
        if (unit24(w.w[0]) < sc.near_frac) {
            for (int base = 0; base < max_att; base += G) {
                const int a = base + tm.lane;
                bool ok = false;
                float x1 = 0.f, y1 = 0.f;
                if (a < max_att) {
                    const Words4 v = draw(seed, e, ep, kNear, 1, (uint32_t)a);
                    const float d = __fadd_rn(sc.dmin, __fmul_rn(unit24(v.w[0]), sc.dspan));
                    const float cx = __fsub_rn(__fmul_rn(2.0f, unit24(v.w[1])), 1.0f);
                    const float cy = __fsub_rn(__fmul_rn(2.0f, unit24(v.w[2])), 1.0f);
                    const float rr = __fadd_rn(__fmul_rn(cx, cx), __fmul_rn(cy, cy));
                    if (!(rr < 0.0625f || rr > 1.0f)) {
                        const float nrm = __fsqrt_rn(rr);
                        const float ox = __fdiv_rn(__fmul_rn(d, cx), nrm);
                        const float oy = __fdiv_rn(__fmul_rn(d, cy), nrm);
                        x1 = __fadd_rn(S.fx[0], ox);
                        y1 = __fadd_rn(S.fy[0], oy);
                        ok = !(x1 < sc.lox || x1 > sc.hix || y1 < sc.loy || y1 > sc.hiy);
                    }
                }
                const unsigned bal = tm.ballot(ok);
                if (bal) {
                    const int win = __ffs(bal) - 1;
                    if (tm.lane == win) {
                        S.fx[1] = x1;
                        S.fy[1] = y1;
                        S.fth[1] = S.fth[0];
                    }
                    first = 2;
                    break;
                }
            }
            tm.sync();
        }
    }
    for (int i = first; i < N; ++i) {
        for (int base = 0; base < max_att; base += G) {
            const int a = base + tm.lane;
            bool ok = false;
            float cx = 0.f, cy = 0.f, cth = 0.f;
            if (a < max_att) {
                const Words4 v = draw(seed, e, ep, kPos, i, (uint32_t)a);
                cx = __fadd_rn(sc.lox, __fmul_rn(unit24(v.w[0]), sc.wx));
                cy = __fadd_rn(sc.loy, __fmul_rn(unit24(v.w[1]), sc.wy));
                cth = __fadd_rn(-sc.pif, __fmul_rn(unit24(v.w[2]), sc.twopif));
                ok = true;
                for (int j = 0; j < i; ++j) {
                    const float dx = __fsub_rn(cx, S.fx[j]), dy = __fsub_rn(cy, S.fy[j]);
                    const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
                    if (d2 < sc.sep2) { ok = false; break; }
                }
            }
            const unsigned bal = tm.ballot(ok);
            int writer = -1;
            if (bal) writer = __ffs(bal) - 1;
            else if (base + G >= max_att) writer = (max_att - 1) - base;  // keep the last candidate
            if (writer >= 0) {
                if (tm.lane == writer) {
                    S.fx[i] = cx;
                    S.fy[i] = cy;
                    S.fth[i] = cth;
                }
                break;
            }
        }
        tm.sync();
    }
    n_res = 0;
    if (A.k.scenario != 0) {
        // Foraging resources (level U{1,2,3}) or Discovery landmarks (none sensed: level 0)
        const Words4 w = draw(seed, e, ep, kNRes, 0, 0u);
        n_res = A.k.n_res_min + below(w.w[0], (uint32_t)(A.k.n_res_max - A.k.n_res_min + 1));
        for (int r = tm.lane; r < A.k.r_max; r += G) {
            if (r < n_res) {
                const Words4 v = draw(seed, e, ep, kRes, r, 0u);
                S.qx[r] = (R)__fadd_rn(sc.lox, __fmul_rn(unit24(v.w[0]), sc.wx));
                S.qy[r] = (R)__fadd_rn(sc.loy, __fmul_rn(unit24(v.w[1]), sc.wy));
                S.qlevel[r] = (A.k.scenario == 1) ? 1 + below(v.w[2], 3u) : 0;
                S.qactive[r] = 1;
            } else {
                S.qx[r] = (R)0;
                S.qy[r] = (R)0;
                S.qlevel[r] = 0;
                S.qactive[r] = 0;
            }
        }
    }
    tm.sync();
}

// New goal of a robot that arrived at its goal (Random Waypoint Navigation, Sec. 4.2): the
// reset's goal distribution under the counter (env, episode, goal | robot, steps taken in the
// episode including this one), so it never repeats the reset's draw (counter word 3 = 0).
// Out of line: arrivals are rare and the hot loop stays small.
static __device__ __noinline__ float3 waypoint_goal(const SamplerConsts sc, uint64_t seed, int e,
                                                    int ep, int i, int t_after) {
    const Words4 w = draw(seed, e, ep, kGoal, i, (uint32_t)t_after);
    return make_float3(__fadd_rn(sc.lox, __fmul_rn(unit24(w.w[0]), sc.wx)),
                       __fadd_rn(sc.loy, __fmul_rn(unit24(w.w[1]), sc.wy)),
                       __fadd_rn(-sc.pif, __fmul_rn(unit24(w.w[2]), sc.twopif)));
}

// Unicycle pose controller: posture regulation in polar coordinates (Aicardi, Casalino, Bicchi,
// Balestrino 1995), standing for the pose controller the paper evaluates (Sec. 4.2, Table 2).
// In the goal's frame rho is the distance to the goal, gam the angle from the heading to the
// goal's direction and del that direction's angle; v = k1 rho cos(gam) and
// omega = k2 gam + k1 (sin(gam) cos(gam) / gam)(gam + k3 del) decrease
// V = (rho^2 + gam^2 + k3 del^2) / 2.  Returned as the projected point's SI velocity.  In
// binary32 the headings' sines and cosines use the hardware approximation (absolute error
// below 4e-7 on (-pi, pi]); gam's go through the accurate library function, since
// sin(gam) / gam would amplify an absolute error near gam = 0.  The nominal velocity stays
// within about 1e-6 of the binary64 oracle's.
__device__ __forceinline__ void sincos_r(float a, float* s, float* c) { __sincosf(a, s, c); }
__device__ __forceinline__ void sincos_r(double a, double* s, double* c) { sincos(a, s, c); }

template <typename R>
__device__ __forceinline__ void pose_nominal(const StepConsts<R>& k, R x, R y, R th, R gx, R gy,
                                             R gth, R& ux, R& uy) {
    const R pi = (R)CUDART_PI, two_pi = (R)(2.0 * CUDART_PI);
    R cs, sn, cg, sg;
    sincos_r(th, &sn, &cs);
    sincos_r(gth, &sg, &cg);
    auto wrap = [&](R a) { return a > pi ? a - two_pi : (a <= -pi ? a + two_pi : a); };
    const R dx = x - gx, dy = y - gy;
    const R xr = cg * dx + sg * dy, yr = -sg * dx + cg * dy;
    const R thr = wrap(th - gth);
    const R rho = hypot(xr, yr);
    R v = (R)0, w = -k.pk2 * thr;  // on the goal point: turn towards the goal heading
    if (rho > (R)0) {
        const R gam = wrap(atan2(yr, xr) + pi - thr);
        const R del = wrap(gam + thr);
        R sgm, cgm;
        sincos(gam, &sgm, &cgm);
        const R sinc = (gam == (R)0) ? (R)1 : sgm / gam;
        v = k.pk1 * rho * cgm;
        w = k.pk2 * gam + k.pk1 * sinc * cgm * (gam + k.pk3 * del);
    }
    ux = v * cs - k.l * w * sn;
    uy = v * sn + k.l * w * cs;
}

// Goal and level of robot i for episode ep (owner lane).
template <typename R>
__device__ __forceinline__ void robot_goal_level(const LaunchArgs<R>& A, int e, int ep, int i,
                                                 R& gx, R& gy, R& gth, int& lv) {
    const Words4 w = draw(A.seed, e, ep, kGoal, i, 0u);
    gx = (R)__fadd_rn(A.sc.lox, __fmul_rn(unit24(w.w[0]), A.sc.wx));
    gy = (R)__fadd_rn(A.sc.loy, __fmul_rn(unit24(w.w[1]), A.sc.wy));
    gth = (R)__fadd_rn(-A.sc.pif, __fmul_rn(unit24(w.w[2]), A.sc.twopif));
    lv = 0;
    if (A.k.scenario == 1) {
        const Words4 v = draw(A.seed, e, ep, kLevel, i, 0u);
        lv = 1 + below(v.w[0], 3u);
    }
    // Discovery roles: the first ceil(N/2) robots sense (1), the others tag (2)
    if (A.k.scenario == 2) lv = (i < (A.s.nrob[e] + 1) / 2) ? 1 : 2;
}

// Scripted target of a Discovery robot: a sensing robot (role 1) heads for the nearest landmark
// not yet sensed, a tagging robot for the nearest sensed one not yet tagged (ties: lowest index);
// false when there is none (the robot holds its position).
template <typename R>
__device__ __forceinline__ bool discovery_target(const R* qx, const R* qy, const int* qlevel,
                                                 const int* qactive, int n_res, int role, R px,
                                                 R py, R& tx, R& ty) {
    int best = -1;
    R bd = (R)0;
    for (int r = 0; r < n_res; ++r) {
        const bool want = (role == 1) ? (qlevel[r] == 0) : (qlevel[r] != 0 && qactive[r] != 0);
        if (!want) continue;
        const R dx = qx[r] - px, dy = qy[r] - py;
        const R d2 = dx * dx + dy * dy;
        if (best < 0 || d2 < bd) { best = r; bd = d2; }
    }
    if (best < 0) return false;
    tx = qx[best];
    ty = qy[best];
    return true;
}

// ------------------------------------------------------------------------------------------
// One env for T steps
// ------------------------------------------------------------------------------------------
// SCEN >= 0 fixes the scenario at compile time and LEAN drops policy actions and traces (a
// scripted rollout): the one-launch kernel instantiates the step it needs, nothing more, which
// keeps its code -- every class's loop in one kernel -- small for the instruction cache.
template <typename R, int G, int NMAX, int SCEN = -1, bool LEAN = false>
__device__ void run_env(const LaunchArgs<R>& A, const Team<G>& tm, TeamSmem<R, NMAX>& S, int e) {
    constexpr int RPL = (NMAX + G - 1) / G;
    const StepConsts<R>& k = A.k;
    const int off = A.s.off[e];
    const int N = A.s.nrob[e];
    const bool forage = (SCEN < 0) ? (k.scenario == 1) : (SCEN == 1);
    const bool disc = (SCEN < 0) ? (k.scenario == 2) : (SCEN == 2);
    const bool resv = forage || disc;  // per-env resources / landmarks
    const R* actions = LEAN ? nullptr : A.io.actions;
    R* tr_unom = LEAN ? nullptr : A.io.u_nom;
    R* tr_ustar = LEAN ? nullptr : A.io.u_star;
    R* tr_vw = LEAN ? nullptr : A.io.vw;
    int32_t* tr_qp = LEAN ? nullptr : A.io.qp_info;
    QPWork<R, NMAX>& W = WorkSel<R, NMAX>::get(S.qp);

    QPConsts<R> qc;
    qc.gamma = k.gamma; qc.r2 = k.r2; qc.kg = k.kg; qc.half_r = k.half_r;
    qc.xmin = k.xmin; qc.xmax = k.xmax; qc.ymin = k.ymin; qc.ymax = k.ymax;
    qc.h_flag = k.h_flag;
    qc.max_iter = k.max_iter;
    if (std::is_same<R, float>::value) {
        qc.tol_abs = (R)2e-7; qc.tol_rel = (R)1e-6; qc.eps_dep = (R)1e-5; qc.tol_lam = (R)1e-6;
    } else {
        qc.tol_abs = (R)1e-12; qc.tol_rel = (R)1e-12; qc.eps_dep = (R)1e-12; qc.tol_lam = (R)1e-10;
    }

    R x[RPL], y[RPL], th[RPL], gx[RPL], gy[RPL], gth[RPL], cs[RPL], sn[RPL];
    int lv[RPL];
#pragma unroll
    for (int s = 0; s < RPL; ++s) {
        const int i = tm.lane + s * G;
        x[s] = y[s] = th[s] = gx[s] = gy[s] = cs[s] = sn[s] = (R)0;
        lv[s] = 0;
        if (i < N) {
            x[s] = A.s.x[off + i]; y[s] = A.s.y[off + i]; th[s] = A.s.th[off + i];
            gx[s] = A.s.gx[off + i]; gy[s] = A.s.gy[off + i]; lv[s] = A.s.level[off + i];
            gth[s] = A.s.gth[off + i];
            sc_(th[s], &sn[s], &cs[s]);
        }
    }
    int t = A.s.t[e], ep = A.s.ep[e];
    int n_res = 0;
    if (resv) {
        n_res = A.s.n_res[e];
        for (int r = tm.lane; r < k.r_max; r += G) {
            S.qx[r] = A.s.qx[e * k.r_max + r];
            S.qy[r] = A.s.qy[e * k.r_max + r];
            S.qlevel[r] = A.s.qlevel[e * k.r_max + r];
            S.qactive[r] = A.s.qactive[e * k.r_max + r];
        }
    }
    int cnt[kNCount];
#pragma unroll
    for (int c = 0; c < kNCount; ++c) cnt[c] = (tm.lane == 0) ? A.s.counters[e * kNCount + c] : 0;
    tm.sync();

    R ret_acc = (R)0;
    for (int step = 0; step < A.T; ++step) {
        // ---- projected points and nominal SI velocity
        R dold[RPL], u0x[RPL], u0y[RPL];
#pragma unroll
        for (int s = 0; s < RPL; ++s) {
            const int i = tm.lane + s * G;
            dold[s] = u0x[s] = u0y[s] = (R)0;
            if (i < N) {
                const R px = x[s] + k.l * cs[s], py = y[s] + k.l * sn[s];
                R ux, uy;
                if (actions) {
                    ux = actions[2 * (off + i)];
                    uy = actions[2 * (off + i) + 1];
                    screen_action(A.io.status, ux, uy);
                } else {
                    R tx = gx[s], ty = gy[s];
                    if (forage) {
                        int best = -1;
                        R bd = (R)0;
                        for (int r = 0; r < n_res; ++r) {
                            if (!S.qactive[r]) continue;
                            const R dx = S.qx[r] - px, dy = S.qy[r] - py;
                            const R d2 = dx * dx + dy * dy;
                            if (best < 0 || d2 < bd) { best = r; bd = d2; }
                        }
                        if (best >= 0) { tx = S.qx[best]; ty = S.qy[best]; }
                        else { tx = px; ty = py; }
                    }
                    if (disc && !discovery_target<R>(S.qx, S.qy, S.qlevel, S.qactive, n_res,
                                                     lv[s], px, py, tx, ty)) {
                        tx = px;
                        ty = py;
                    }
                    if (!resv && k.controller == 1) {
                        pose_nominal<R>(k, x[s], y[s], th[s], gx[s], gy[s], gth[s], ux, uy);
                    } else {
                        ux = k.k_si * (tx - px);
                        uy = k.k_si * (ty - py);
                    }
                    cap_norm(ux, uy, k.vmax);
                    if (k.noise_on) {
                        const Words4 w = draw(A.seed, e, ep, kNoise, i >> 1, (uint32_t)t);
                        const float ex = __fmul_rn(__fsub_rn(unit24(w.w[2 * (i & 1)]), 0.5f), k.noise_scale);
                        const float ey = __fmul_rn(__fsub_rn(unit24(w.w[2 * (i & 1) + 1]), 0.5f), k.noise_scale);
                        ux += (R)ex;
                        uy += (R)ey;
                    }
                }
                cap_norm(ux, uy, k.vmax);
                u0x[s] = ux;
                u0y[s] = uy;
                if (!resv) dold[s] = hyp(px - gx[s], py - gy[s]);
                W.px[i] = px; W.py[i] = py;
                W.u0x[i] = ux; W.u0y[i] = uy;
                W.ux[i] = ux; W.uy[i] = uy;
            }
        }
        tm.sync();

        // ---- barrier-certificate QP (binary32: explicit-inverse form; binary64: Cholesky form)
        QPResult res;
        if constexpr (std::is_same<R, float>::value && (NMAX > 4))
            res = qp_solve_inv<float, G, NMAX>(tm, S.qp.s.inv, N, qc, W);
        else
            res = qp_solve<R, G, NMAX>(tm, W, N, qc);
        int qflags = (res.q > 0 || res.status != 0) ? 1 : 0;
        R usx[RPL], usy[RPL];
        bool resolved = false;
        if (std::is_same<R, float>::value && k.resolve_f64 && res.flag) {
            tm.sync();  // every lane is done with the binary32 workspace that D overlays
            QPWork<double, NMAX>& D = S.qp.d;
            QPConsts<double> dc;
            dc.gamma = (double)k.gamma; dc.r2 = (double)k.r2; dc.kg = (double)k.kg;
            dc.half_r = (double)k.half_r; dc.xmin = (double)k.xmin; dc.xmax = (double)k.xmax;
            dc.ymin = (double)k.ymin; dc.ymax = (double)k.ymax; dc.h_flag = (double)k.h_flag;
            dc.max_iter = 8 * NMAX + 16;
            dc.tol_abs = 1e-12; dc.tol_rel = 1e-12; dc.eps_dep = 1e-12; dc.tol_lam = 1e-10;
            double pxd[RPL], pyd[RPL];
#pragma unroll
            for (int s = 0; s < RPL; ++s) {
                double sd, cd;
                sincos((double)th[s], &sd, &cd);
                pxd[s] = (double)x[s] + (double)k.l * cd;
                pyd[s] = (double)y[s] + (double)k.l * sd;
            }
            QPResult r64;
            r64.status = 2;
            const double* rux = D.ux;
            const double* ruy = D.uy;
            if constexpr (NMAX > 4 && NMAX <= 20 && G >= NMAX) {
                // the explicit-inverse form (binary64 issue is slow: its rank-one updates spread
                // over the lanes need far fewer instructions than the Cholesky form's
                // triangular solves); an active set beyond its slots falls back below, and so
                // does the 32-robot class (its binary64 lane rows would not fit in registers)
                // the binary32 solve's final active rows, the binary64 solve's start (read before
                // the binary64 work overwrites them)
                const int q32 = (res.status == 0) ? res.q : 0;
                int wa = 0, wb = -1, wside = 0, wkey = 0x7fffffff;
                if (tm.lane < q32) {
                    const InvWork<NMAX>& W32 = S.qp.s.inv;
                    const int t = W32.act[tm.lane];
                    wa = W32.sia[t];
                    wb = W32.sib[t];
                    wkey = W32.sk[t];
                    const float ax = W32.sax[t], ay = W32.say[t];
                    wside = ax > 0.f ? 0 : ax < 0.f ? 1 : ay > 0.f ? 2 : 3;
                }
                tm.sync();
                F64Inv<NMAX>& F = S.qp.di;
#pragma unroll
                for (int s = 0; s < RPL; ++s) {
                    const int i = tm.lane + s * G;
                    if (i < N) {
                        F.px[i] = pxd[s];
                        F.py[i] = pyd[s];
                        F.u0x[i] = F.ux[i] = (double)u0x[s];
                        F.u0y[i] = F.uy[i] = (double)u0y[s];
                    }
                }
                tm.sync();
                r64 = qp_solve_inv<double, G, NMAX>(tm, F.inv, N, dc, F, q32, wa, wb, wside, wkey);
                rux = F.ux;
                ruy = F.uy;
            }
            if (r64.status == 2) {
                tm.sync();
#pragma unroll
                for (int s = 0; s < RPL; ++s) {
                    const int i = tm.lane + s * G;
                    if (i < N) {
                        D.px[i] = pxd[s];
                        D.py[i] = pyd[s];
                        D.u0x[i] = (double)u0x[s];
                        D.u0y[i] = (double)u0y[s];
                        D.ux[i] = D.u0x[i];
                        D.uy[i] = D.u0y[i];
                    }
                }
                tm.sync();
                const int it = r64.iters;
                r64 = qp_solve<double, G, NMAX>(tm, D, N, dc);
                r64.iters += it;
                rux = D.ux;
                ruy = D.uy;
            }
            res.status = r64.status;
            res.q = r64.q;
            res.iters += r64.iters;
            resolved = true;
            qflags |= 2;
#pragma unroll
            for (int s = 0; s < RPL; ++s) {
                const int i = tm.lane + s * G;
                usx[s] = usy[s] = (R)0;
                if (i < N) { usx[s] = (R)rux[i]; usy[s] = (R)ruy[i]; }
            }
        }
        if (!resolved) {
#pragma unroll
            for (int s = 0; s < RPL; ++s) {
                const int i = tm.lane + s * G;
                usx[s] = usy[s] = (R)0;
                if (i < N) { usx[s] = W.ux[i]; usy[s] = W.uy[i]; }
            }
        }
        tm.sync();  // the workspace is reused below

        // ---- SI -> unicycle, wheel clip, Euler step
#pragma unroll
        for (int s = 0; s < RPL; ++s) {
            const int i = tm.lane + s * G;
            if (i < N) {
                R v = cs[s] * usx[s] + sn[s] * usy[s];
                R om = (cs[s] * usy[s] - sn[s] * usx[s]) * k.inv_l;
                R wr = v + k.half_track * om, wl = v - k.half_track * om;
                wr = fmin(fmax(wr, -k.vmax), k.vmax);
                wl = fmin(fmax(wl, -k.vmax), k.vmax);
                v = (R)0.5 * (wr + wl);
                om = (wr - wl) * k.inv_track;
                if (tr_unom) {
                    tr_unom[2 * (off + i)] = u0x[s];
                    tr_unom[2 * (off + i) + 1] = u0y[s];
                }
                if (tr_ustar) {
                    tr_ustar[2 * (off + i)] = usx[s];
                    tr_ustar[2 * (off + i) + 1] = usy[s];
                }
                if (tr_vw) {
                    tr_vw[2 * (off + i)] = v;
                    tr_vw[2 * (off + i) + 1] = om;
                }
                x[s] += k.dt * v * cs[s];
                y[s] += k.dt * v * sn[s];
                th[s] = wrap_pi(th[s] + k.dt * om);
                sc_(th[s], &sn[s], &cs[s]);
                W.px[i] = x[s] + k.l * cs[s];
                W.py[i] = y[s] + k.l * sn[s];
            }
        }
        tm.sync();

        // ---- flags and reward
        int col_l = 0, oob_l = 0, arr_l = 0;
        R rew_l = (R)0;
        const int nd = (N - 1) / 2;
#pragma unroll
        for (int s = 0; s < RPL; ++s) {
            const int i = tm.lane + s * G;
            if (i < N) {
                const R pxi = W.px[i], pyi = W.py[i];
                const int ndi = nd + (((N & 1) == 0 && i < N / 2) ? 1 : 0);
                for (int d = 1; d <= ndi; ++d) {
                    int j = i + d;
                    if (j >= N) j -= N;
                    const R dx = pxi - W.px[j], dy = pyi - W.py[j];
                    if (dx * dx + dy * dy < k.r2) ++col_l;
                }
                if (pxi < k.xmin || pxi > k.xmax || pyi < k.ymin || pyi > k.ymax) ++oob_l;
                if (!resv) rew_l -= hyp(pxi - gx[s], pyi - gy[s]) - dold[s];
                if (!resv && k.waypoint) {
                    const R ex = pxi - gx[s], ey = pyi - gy[s];
                    if (ex * ex + ey * ey < k.goal_eps2) {
                        const float3 g = waypoint_goal(A.sc, A.seed, e, ep, i, t + 1);
                        gx[s] = (R)g.x;
                        gy[s] = (R)g.y;
                        gth[s] = (R)g.z;
                        ++arr_l;
                    }
                }
            }
        }
        const int col = tm.sum(col_l);
        const int oob = tm.sum(oob_l);
        R rew = tm.sum(rew_l);
        bool all_foraged = false;
        int succ = k.waypoint ? tm.sum(arr_l) : 0;
        if (forage) {
            const R rho2 = k.rho2;
            int remaining = 0;
            for (int r = 0; r < n_res; ++r) {
                const bool act = S.qactive[r] != 0;
                if (!act) continue;
                int ls = 0;
#pragma unroll
                for (int s = 0; s < RPL; ++s) {
                    const int i = tm.lane + s * G;
                    if (i < N) {
                        const R dx = W.px[i] - S.qx[r], dy = W.py[i] - S.qy[r];
                        if (dx * dx + dy * dy < rho2) ls += lv[s];
                    }
                }
                ls = tm.sum(ls);
                if (ls >= S.qlevel[r]) {
                    rew += (R)S.qlevel[r];
                    ++succ;
                    tm.sync();
                    if (tm.lane == 0) S.qactive[r] = 0;
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
                int sensed = S.qlevel[r], tagged = S.qactive[r] ? 0 : 1;
                int hs = 0, ht = 0;
#pragma unroll
                for (int s = 0; s < RPL; ++s) {
                    const int i = tm.lane + s * G;
                    if (i < N) {
                        const R dx = W.px[i] - S.qx[r], dy = W.py[i] - S.qy[r];
                        const R d2 = dx * dx + dy * dy;
                        hs |= (lv[s] == 1 && d2 < k.sense_r2) ? 1 : 0;
                        ht |= (lv[s] == 2 && d2 < k.tag_r2) ? 1 : 0;
                    }
                }
                hs = tm.any(hs != 0) ? 1 : 0;
                ht = tm.any(ht != 0) ? 1 : 0;
                if (!sensed && hs) { sensed = 1; rew += k.sense_rew; }
                if (sensed && !tagged && ht) { tagged = 1; rew += k.tag_rew; ++succ; }
                remaining += tagged ? 0 : 1;
                tm.sync();
                if (tm.lane == 0) { S.qlevel[r] = sensed; S.qactive[r] = tagged ? 0 : 1; }
                tm.sync();
            }
            if (remaining > 0) rew -= k.step_pen;
        }
        rew -= k.c_col * (R)col;
        if (tm.lane == 0) {
            cnt[0] += col;
            cnt[1] += oob;
            cnt[2] += succ;
            cnt[3] += (qflags & 1);
            cnt[4] += (qflags >> 1) & 1;
            cnt[5] += (res.status == 1) ? 1 : 0;
            cnt[7] += res.iters;
        }
        if (tr_qp && tm.lane == 0) {
            tr_qp[4 * e + 0] = res.status;
            tr_qp[4 * e + 1] = res.q;
            tr_qp[4 * e + 2] = res.iters;
            tr_qp[4 * e + 3] = qflags;
        }

        // ---- episode end and auto-reset
        t += 1;
        const bool done = (t >= k.episode_len) || all_foraged;
        if (done) {
            if (tm.lane == 0) cnt[6] += 1;
            ep += 1;
            t = 0;
            tm.sync();
            team_sample<R, G, NMAX>(tm, S, A, e, ep, N, n_res);
#pragma unroll
            for (int s = 0; s < RPL; ++s) {
                const int i = tm.lane + s * G;
                if (i < N) {
                    x[s] = (R)S.fx[i];
                    y[s] = (R)S.fy[i];
                    th[s] = (R)S.fth[i];
                    sc_(th[s], &sn[s], &cs[s]);
                    robot_goal_level<R>(A, e, ep, i, gx[s], gy[s], gth[s], lv[s]);
                }
            }
            tm.sync();
        }

        // ---- observations
        if (A.io.obs) {
#pragma unroll
            for (int s = 0; s < RPL; ++s) {
                const int i = tm.lane + s * G;
                if (i < N) {
                    S.sx[i] = x[s]; S.sy[i] = y[s]; S.sth[i] = th[s]; S.slevel[i] = lv[s];
                }
            }
            tm.sync();
            const int od = A.io.obs_dim;
#pragma unroll
            for (int s = 0; s < RPL; ++s) {
                const int i = tm.lane + s * G;
                if (i < N) {
                    R* o = A.io.obs + (long long)step * A.io.obs_step + (long long)(off + i) * od;
                    int c = 0;
                    if (disc) {
                        o[0] = x[s]; o[1] = y[s]; o[2] = th[s];
                        o[3] = lv[s] == 1 ? k.sense_r : (R)0;
                        o[4] = lv[s] == 2 ? k.tag_r : (R)0;
                        c = 5;
                        for (int j = 0; j < N; ++j) {
                            if (j == i) continue;
                            o[c] = S.sx[j] - x[s];
                            o[c + 1] = S.sy[j] - y[s];
                            o[c + 2] = wrap_pi(S.sth[j] - th[s]);
                            o[c + 3] = S.slevel[j] == 1 ? k.sense_r : (R)0;
                            o[c + 4] = S.slevel[j] == 2 ? k.tag_r : (R)0;
                            c += 5;
                        }
                        const int rbase = 5 + 5 * (k.n_max_obs - 1);
                        for (; c < rbase; ++c) o[c] = (R)0;
                        for (int r = 0; r < k.r_max; ++r) {
                            if (r < n_res && S.qlevel[r]) {
                                o[c] = S.qx[r] - x[s];
                                o[c + 1] = S.qy[r] - y[s];
                                o[c + 2] = (R)1;
                                o[c + 3] = S.qactive[r] ? (R)0 : (R)1;
                            } else if (r < n_res) {
                                o[c] = k.xo - x[s];
                                o[c + 1] = k.yo - y[s];
                                o[c + 2] = o[c + 3] = (R)0;
                            } else {
                                o[c] = o[c + 1] = o[c + 2] = o[c + 3] = (R)0;
                            }
                            c += 4;
                        }
                    } else if (!forage) {
                        o[0] = x[s]; o[1] = y[s]; o[2] = th[s]; o[3] = gx[s]; o[4] = gy[s];
                        c = 5;
                        for (int j = 0; j < N; ++j) {
                            if (j == i) continue;
                            o[c] = S.sx[j] - x[s];
                            o[c + 1] = S.sy[j] - y[s];
                            o[c + 2] = wrap_pi(S.sth[j] - th[s]);
                            c += 3;
                        }
                        for (; c < od; ++c) o[c] = (R)0;
                    } else {
                        o[0] = x[s]; o[1] = y[s]; o[2] = th[s]; o[3] = (R)lv[s];
                        c = 4;
                        for (int j = 0; j < N; ++j) {
                            if (j == i) continue;
                            o[c] = S.sx[j] - x[s];
                            o[c + 1] = S.sy[j] - y[s];
                            o[c + 2] = wrap_pi(S.sth[j] - th[s]);
                            o[c + 3] = (R)S.slevel[j];
                            c += 4;
                        }
                        const int rbase = 4 + 4 * (k.n_max_obs - 1);
                        for (; c < rbase; ++c) o[c] = (R)0;
                        for (int r = 0; r < k.r_max; ++r) {
                            if (r < n_res) {
                                o[c] = S.qx[r] - x[s];
                                o[c + 1] = S.qy[r] - y[s];
                                o[c + 2] = (R)S.qlevel[r];
                                o[c + 3] = (R)S.qactive[r];
                            } else {
                                o[c] = o[c + 1] = o[c + 2] = o[c + 3] = (R)0;
                            }
                            c += 4;
                        }
                    }
                }
            }
            tm.sync();
        }
        if (tm.lane == 0) {
            if (A.io.reward) A.io.reward[(long long)step * A.io.E + e] = rew;
            if (A.io.done) A.io.done[(long long)step * A.io.E + e] = done ? 1 : 0;
        }
        ret_acc += rew;
    }
    if (A.io.ret && tm.lane == 0) A.io.ret[e] = ret_acc;

    // ---- state back to global memory
#pragma unroll
    for (int s = 0; s < RPL; ++s) {
        const int i = tm.lane + s * G;
        if (i < N) {
            A.s.x[off + i] = x[s]; A.s.y[off + i] = y[s]; A.s.th[off + i] = th[s];
            A.s.gx[off + i] = gx[s]; A.s.gy[off + i] = gy[s]; A.s.level[off + i] = lv[s];
            A.s.gth[off + i] = gth[s];
        }
    }
    if (resv) {
        for (int r = tm.lane; r < k.r_max; r += G) {
            A.s.qx[e * k.r_max + r] = S.qx[r];
            A.s.qy[e * k.r_max + r] = S.qy[r];
            A.s.qlevel[e * k.r_max + r] = S.qlevel[r];
            A.s.qactive[e * k.r_max + r] = S.qactive[r];
        }
    }
    if (tm.lane == 0) {
        A.s.t[e] = t;
        A.s.ep[e] = ep;
        if (resv) A.s.n_res[e] = n_res;
#pragma unroll
        for (int c = 0; c < kNCount; ++c) A.s.counters[e * kNCount + c] = cnt[c];
    }
}

// Reset env e to episode ep (state written to global memory).
template <typename R, int G, int NMAX>
__device__ void reset_env(const LaunchArgs<R>& A, const Team<G>& tm, TeamSmem<R, NMAX>& S, int e,
                          int ep) {
    constexpr int RPL = (NMAX + G - 1) / G;
    const int off = A.s.off[e];
    const int N = A.s.nrob[e];
    int n_res = 0;
    team_sample<R, G, NMAX>(tm, S, A, e, ep, N, n_res);
#pragma unroll
    for (int s = 0; s < RPL; ++s) {
        const int i = tm.lane + s * G;
        if (i < N) {
            R gx, gy, gth;
            int lv;
            robot_goal_level<R>(A, e, ep, i, gx, gy, gth, lv);
            A.s.x[off + i] = (R)S.fx[i];
            A.s.y[off + i] = (R)S.fy[i];
            A.s.th[off + i] = (R)S.fth[i];
            A.s.gx[off + i] = gx;
            A.s.gy[off + i] = gy;
            A.s.gth[off + i] = gth;
            A.s.level[off + i] = lv;
        }
    }
    if (A.k.scenario != 0) {
        for (int r = tm.lane; r < A.k.r_max; r += G) {
            A.s.qx[e * A.k.r_max + r] = S.qx[r];
            A.s.qy[e * A.k.r_max + r] = S.qy[r];
            A.s.qlevel[e * A.k.r_max + r] = S.qlevel[r];
            A.s.qactive[e * A.k.r_max + r] = S.qactive[r];
        }
    }
    if (tm.lane == 0) {
        A.s.t[e] = 0;
        A.s.ep[e] = ep;
        A.s.n_res[e] = n_res;
        for (int c = 0; c < kNCount; ++c) A.s.counters[e * kNCount + c] = 0;
    }
    tm.sync();
}

template <typename R, int G, int NMAX>
__global__ void __launch_bounds__(256, 1) env_kernel(LaunchArgs<R> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Team<G> tm;
    const int teams_per_block = blockDim.x / G;
    const int tib = threadIdx.x / G;
    TeamSmem<R, NMAX>* S = reinterpret_cast<TeamSmem<R, NMAX>*>(smem_raw) + tib;
    const int total_teams = gridDim.x * teams_per_block;
    for (int idx = blockIdx.x * teams_per_block + tib; idx < A.n_list; idx += total_teams) {
        const int e = A.env_list ? A.env_list[idx] : A.env_begin + idx;
        run_env<R, G, NMAX>(A, tm, *S, e);
    }
}

template <typename R, int G, int NMAX>
__global__ void __launch_bounds__(256) reset_kernel(LaunchArgs<R> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Team<G> tm;
    const int teams_per_block = blockDim.x / G;
    const int tib = threadIdx.x / G;
    TeamSmem<R, NMAX>* S = reinterpret_cast<TeamSmem<R, NMAX>*>(smem_raw) + tib;
    const int total_teams = gridDim.x * teams_per_block;
    for (int idx = blockIdx.x * teams_per_block + tib; idx < A.n_list; idx += total_teams) {
        const int e = A.env_list ? A.env_list[idx] : A.env_begin + idx;
        reset_env<R, G, NMAX>(A, tm, *S, e, 0);
    }
}

}  // namespace rl
