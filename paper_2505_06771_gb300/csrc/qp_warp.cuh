// qp_warp.cuh -- the barrier QP of one env of at most 4 robots, solved by all live lanes of a
// warp at once.
//
// The 4-robot team kernels solve almost every QP inside the team (qp_regs.cuh).  Two rare
// cases are far slower there: an active set of more than four rows (the register solver's
// capacity) and the binary64 re-solve of a flagged QP.  Both come in bursts, from the few envs
// whose robots are jammed or in contact, and the rollout ends when the slowest env does.  On
// GB300 a binary64 instruction costs about 64 cycles of issue whether 4 or 32 lanes run it, so
// these solves are bound by the number of instructions on their critical path.  Here the 22
// row slots (6 pairs, then the 16 arena rows, the method's tie-break order) are spread over the
// lanes, the unknowns u (8 values) over lanes 0..7, and the multiplier ratios of the dual step
// over the active rows' lanes; the short sequential parts (triangular solves on at most 8 rows)
// run in every lane.  The iteration is the one of thread_qp / qp_solve (Goldfarb-Idnani dual
// active set on H = I, Sec. 3 barrier QP): add the most violated inactive row (ties: lowest
// slot), step by min(tf, td), drop a row whose multiplier reaches zero.  Its result is
// rounded to binary32 by the caller, so the binary64 iterate is not polished by an exact solve
// on the final active set as the binary64 kernels' qp_solve does (the two differ by binary64
// rounding).
#pragma once
#include "qp_regs.cuh"

namespace rl {

constexpr int kWarpRows = 8;  // at most 8 independent rows in 8 unknowns

template <typename Q>
__device__ __forceinline__ Q wsel4(const Q (&a)[4], int k) {
    return k == 0 ? a[0] : (k == 1 ? a[1] : (k == 2 ? a[2] : a[3]));
}
template <typename Q>
__device__ __forceinline__ Q wsel8(const Q (&a)[8], int k) {
    Q r = a[0];
#pragma unroll
    for (int m = 1; m < 8; ++m)
        if (k == m) r = a[m];
    return r;
}

// Reciprocal, quotient and square root for the dual step.  binary32: the IEEE operations.
// binary64: a binary32 estimate refined by Newton's method (one step for the reciprocal,
// r <- r + r (1 - b r); Heron's step s <- s + (x - s^2) / (2 s) for the root), about 2^-46
// relative, in 2 or 3 binary64 instructions instead of the 10 or more of the IEEE sequences;
// operands outside the binary32 normal range take the IEEE operation.
__device__ __forceinline__ float wrcp(float b) { return 1.f / b; }
__device__ __forceinline__ float wdiv(float a, float b) { return a / b; }
__device__ __forceinline__ float wsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ bool wnormal(double b) {
    const double m = fabs(b);
    return m > 1e-30 && m < 1e30;
}
__device__ __forceinline__ double wrcp(double b) {
    if (!wnormal(b)) return 1.0 / b;
    const double r = (double)(1.f / (float)b);
    return fma(r, fma(-b, r, 1.0), r);
}
__device__ __forceinline__ double wdiv(double a, double b) { return a * wrcp(b); }
__device__ __forceinline__ double wsqrt(double x) {
    if (!wnormal(x) || x < 0.0) return sqrt(x);
    const float sf = sqrtf((float)x);
    const double s = (double)sf;
    return fma(fma(-s, s, x), (double)(0.5f / sf), s);
}

// Orderable bits of a value >= 0 (0 for "none").
__device__ __forceinline__ unsigned long long wkey(double v) {
    return v > 0.0 ? (unsigned long long)__double_as_longlong(v) : 0ull;
}
__device__ __forceinline__ unsigned long long wkey(float v) {
    return v > 0.f ? (unsigned long long)__float_as_uint(v) : 0ull;
}

// Over the lanes of wm: the idx of the largest key (ties: smallest idx), -1 when all are 0.
__device__ __forceinline__ int warp_argmax_key(unsigned wm, unsigned long long key, int idx) {
    const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
    const unsigned mh = __reduce_max_sync(wm, hi);
    const unsigned ml = __reduce_max_sync(wm, hi == mh ? lo : 0u);
    if (mh == 0u && ml == 0u) return -1;
    const bool top = (hi == mh && lo == ml);
    return (int)__reduce_min_sync(wm, top ? (unsigned)idx : 0x7fffffffu);
}
// Over the lanes of wm: the idx of the smallest key (ties: smallest idx).
__device__ __forceinline__ int warp_argmin_key(unsigned wm, unsigned long long key, int idx) {
    const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
    const unsigned mh = __reduce_min_sync(wm, hi);
    const unsigned ml = __reduce_min_sync(wm, hi == mh ? lo : 0xffffffffu);
    const bool bot = (hi == mh && lo == ml);
    return (int)__reduce_min_sync(wm, bot ? (unsigned)idx : 0x7fffffffu);
}

// Sum over lanes 0..7 (lanes 8.. hold zeros), returned in every lane of wm.
template <typename Q>
__device__ __forceinline__ Q warp_sum8(unsigned wm, Q v) {
    v += __shfl_xor_sync(wm, v, 4);
    v += __shfl_xor_sync(wm, v, 2);
    v += __shfl_xor_sync(wm, v, 1);
    return __shfl_sync(wm, v, 0);
}

// Slot s of the QP: pair rows 0..5 as (a, b) with coefficient (cx, cy) on u_a and (-cx, -cy)
// on u_b; arena rows 6 + 4 i + t with b = -1.  Branch-free, so that the lanes holding pair rows
// and those holding arena rows run one instruction stream: a pair row's h = dx^2 + dy^2 - r^2
// and an arena row's wall distance d are both a difference e1 - e2 (less e3 for the arena),
// then the bound is gamma h^3 or kappa gamma d^3.
template <typename Q>
__device__ __forceinline__ void warp_row(int s, int N, const Q (&Px)[4], const Q (&Py)[4],
                                         const QPConsts<Q>& c, int& a, int& b, Q& cx, Q& cy,
                                         Q& bv, bool& ok) {
    const bool pr = s < 6;
    const int m = pr ? 0 : s - 6, i = m >> 2, t = m & 3;
    a = pr ? slot_a(s) : i;
    b = pr ? slot_b(s) : -1;
    const Q pax = wsel4(Px, a), pay = wsel4(Py, a);
    const Q pbx = wsel4(Px, pr ? b : 0), pby = wsel4(Py, pr ? b : 0);
    const Q own = (t < 2) ? pax : pay;
    // pair: e1 - e2 = dx; arena t = 0: (xmax - half_r) - px, 1: (px - xmin) - half_r,
    // 2: (ymax - half_r) - py, 3: (py - ymin) - half_r
    const Q e1 = pr ? pax : ((t & 1) ? own : (t == 0 ? c.xmax : c.ymax));
    const Q e2 = pr ? pbx : ((t & 1) ? (t == 1 ? c.xmin : c.ymin) : c.half_r);
    const Q e3 = (t & 1) ? c.half_r : own;
    const Q d1 = e1 - e2;
    const Q dy = pay - pby;
    const Q val = pr ? d1 * d1 + dy * dy - c.r2 : d1 - e3;
    bv = (pr ? c.gamma : c.kg) * val * val * val;
    cx = pr ? (Q)-2 * d1 : ((t == 0) ? (Q)1 : ((t == 1) ? (Q)-1 : (Q)0));
    cy = pr ? (Q)-2 * dy : ((t == 2) ? (Q)1 : ((t == 3) ? (Q)-1 : (Q)0));
    ok = s < 22 && (pr ? b < N : i < N);
}

// Coefficient of a row on unknown m = 2 i + d.
template <typename Q>
__device__ __forceinline__ Q warp_coef(int a, int b, Q cx, Q cy, int m) {
    const int i = m >> 1;
    const Q v = (m & 1) ? cy : cx;
    return (a == i) ? v : ((b >= 0 && b == i) ? -v : (Q)0);
}

// The QP of one env, by the lanes of wm (lanes 0..nl-1, 8 <= nl <= 32).  Px, Py, U0 are the
// same in every lane.  On return lane m < 8 holds u_m in um; the result is the same in every
// lane (status 0 ok, 1 infeasible (u = 0), 2 iteration cap or numerical failure).
template <typename Q>
__device__ __noinline__ QPResult warp_qp(unsigned wm, int nl, int N, const Q (&Px)[4],
                                         const Q (&Py)[4], const Q (&U0)[8],
                                         const QPConsts<Q> c, Q& um) {
    const int l = threadIdx.x & 31;
    const Q INF = qinf<Q>();
    QPResult res;
    res.status = 0;
    res.q = 0;
    res.iters = 0;
    res.flag = false;
    // the lane's row slots s = l + k nl, k < K <= 3 (nl >= 8)
    const int K = (22 + nl - 1) / nl;
    int ra[3], rb[3];
    Q rcx[3], rcy[3], rbv[3], rthr[3];
    bool rok[3];
    unsigned myact = 0u;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        ra[k] = 0;
        rb[k] = -1;
        rcx[k] = rcy[k] = rbv[k] = rthr[k] = (Q)0;
        rok[k] = false;
        if (k >= K) continue;
        const int s = l + k * nl;
        warp_row<Q>(s < 22 ? s : 21, N, Px, Py, c, ra[k], rb[k], rcx[k], rcy[k], rbv[k],
                    rok[k]);
        rok[k] = rok[k] && s < 22 && l < nl;
        rthr[k] = c.tol_abs + c.tol_rel * fabs(rbv[k]);
    }
    um = (l < 8) ? wsel8(U0, l) : (Q)0;

    // most violated inactive row at the current u: slot and violation (the same in all lanes)
    auto scan = [&](Q& vb) -> int {
        unsigned long long best = 0ull;
        int bslot = 0x7fffffff;
        Q bv_own = (Q)0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (k >= K) continue;
            const int bs = rb[k] >= 0 ? rb[k] : 0;
            const Q uax = __shfl_sync(wm, um, 2 * ra[k]);
            const Q uay = __shfl_sync(wm, um, 2 * ra[k] + 1);
            const Q ubx = __shfl_sync(wm, um, 2 * bs);
            const Q uby = __shfl_sync(wm, um, 2 * bs + 1);
            const Q v = (rb[k] >= 0) ? rcx[k] * (uax - ubx) + rcy[k] * (uay - uby) - rbv[k]
                                     : rcx[k] * uax + rcy[k] * uay - rbv[k];
            const bool cand = rok[k] && !((myact >> k) & 1u) && v > rthr[k];
            const unsigned long long key = cand ? wkey(v) : 0ull;
            if (key > best) {
                best = key;
                bslot = l + k * nl;
                bv_own = v;
            }
        }
        const int s = warp_argmax_key(wm, best, bslot);
        if (s < 0) return -1;
        vb = __shfl_sync(wm, bv_own, s % nl);
        return s;
    };

    // active rows, replicated in every lane
    int As[kWarpRows], Aa[kWarpRows], Ab[kWarpRows];
    Q Acx[kWarpRows], Acy[kWarpRows], Abv[kWarpRows], lam[kWarpRows], dinv[kWarpRows];
    Q L[kWarpRows * (kWarpRows + 1) / 2];
    int q = 0;
    Q vb = (Q)0;
    int sp_slot = scan(vb);
    while (sp_slot >= 0) {
        if (++res.iters > c.max_iter) { res.status = 2; break; }
        // the new row, from its owner
        const int own = sp_slot % nl, kk = sp_slot / nl;
        const int pa = __shfl_sync(wm, kk == 0 ? ra[0] : (kk == 1 ? ra[1] : ra[2]), own);
        const int pb = __shfl_sync(wm, kk == 0 ? rb[0] : (kk == 1 ? rb[1] : rb[2]), own);
        const Q pcx = __shfl_sync(wm, kk == 0 ? rcx[0] : (kk == 1 ? rcx[1] : rcx[2]), own);
        const Q pcy = __shfl_sync(wm, kk == 0 ? rcy[0] : (kk == 1 ? rcy[1] : rcy[2]), own);
        const Q pbv = __shfl_sync(wm, kk == 0 ? rbv[0] : (kk == 1 ? rbv[1] : rbv[2]), own);
        const Q app = (pb >= 0 ? (Q)2 : (Q)1) * (pcx * pcx + pcy * pcy);
        Q lam_p = (Q)0;
        bool added = false;
        for (int guard = 0; guard <= kWarpRows + 1 && !added; ++guard) {
            // w = N a_p (lane t < q), y = L^-1 w, r = L^-T y
            Q wl = (Q)0;
            if (l < q) wl = row_dot<Q>(Aa[l], Ab[l], Acx[l], Acy[l], pa, pb, pcx, pcy);
            Q y[kWarpRows], r[kWarpRows];
            for (int t = 0; t < q; ++t) {
                Q s = __shfl_sync(wm, wl, t);
                for (int m = 0; m < t; ++m) s -= L[t * (t + 1) / 2 + m] * y[m];
                y[t] = s * dinv[t];
            }
            for (int t = q - 1; t >= 0; --t) {
                Q s = y[t];
                for (int m = t + 1; m < q; ++m) s -= L[m * (m + 1) / 2 + t] * r[m];
                r[t] = s * dinv[t];
            }
            // z = a_p - N^T r on lanes 0..7
            Q zm = (Q)0;
            if (l < 8) {
                zm = warp_coef<Q>(pa, pb, pcx, pcy, l);
                for (int t = 0; t < q; ++t) zm -= r[t] * warp_coef<Q>(Aa[t], Ab[t], Acx[t], Acy[t], l);
            }
            const Q zz = warp_sum8<Q>(wm, zm * zm);
            // dual step bound: min lam_t / r_t over r_t > 0 (lane t), ties to the lowest t
            Q tl = INF;
            if (l < q && r[l] > (Q)0) {
                tl = wdiv(lam[l], r[l]);
                if (tl < (Q)0) tl = (Q)0;
            }
            const int jb = warp_argmin_key(wm, l < q ? wkey(tl) : ~0ull, l);
            const Q td = (jb >= 0 && jb < q) ? __shfl_sync(wm, tl, jb) : INF;
            // current violation of the new row
            const int pbs = pb >= 0 ? pb : 0;
            const Q uax = __shfl_sync(wm, um, 2 * pa), uay = __shfl_sync(wm, um, 2 * pa + 1);
            const Q ubx = __shfl_sync(wm, um, 2 * pbs), uby = __shfl_sync(wm, um, 2 * pbs + 1);
            const Q sp = (pb >= 0) ? pcx * (uax - ubx) + pcy * (uay - uby) - pbv
                                   : pcx * uax + pcy * uay - pbv;
            const bool indep = zz > c.eps_dep * app;
            if (!indep) res.flag = true;
            const Q tf = indep ? wdiv(sp, zz) : INF;
            if (!(tf < INF) && !(td < INF)) {
                res.status = 1;
                break;
            }
            const Q st = tf < td ? tf : td;
            if (tf < INF && l < 8) um -= st * zm;
            for (int t = 0; t < q; ++t) lam[t] -= st * r[t];
            lam_p += st;
            if (tf <= td) {
                if (q == kWarpRows) { res.status = 2; break; }
                const Q dg = wsqrt(zz);
                for (int m = 0; m < q; ++m) L[q * (q + 1) / 2 + m] = y[m];
                L[q * (q + 1) / 2 + q] = dg;
                dinv[q] = wrcp(dg);
                As[q] = sp_slot;
                Aa[q] = pa;
                Ab[q] = pb;
                Acx[q] = pcx;
                Acy[q] = pcy;
                Abv[q] = pbv;
                lam[q] = lam_p;
                if (l == own) myact |= 1u << kk;
                ++q;
                added = true;
            } else {
                // drop row jb and refactor the Gram matrix of the remaining rows
                const int js = As[jb];
                if (l == js % nl) myact &= ~(1u << (js / nl));
                for (int t = jb; t < q - 1; ++t) {
                    As[t] = As[t + 1];
                    Aa[t] = Aa[t + 1];
                    Ab[t] = Ab[t + 1];
                    Acx[t] = Acx[t + 1];
                    Acy[t] = Acy[t + 1];
                    Abv[t] = Abv[t + 1];
                    lam[t] = lam[t + 1];
                }
                --q;
                bool okf = true;
                for (int t = 0; t < q; ++t)
                    for (int m = 0; m <= t; ++m) {
                        Q g = row_dot<Q>(Aa[t], Ab[t], Acx[t], Acy[t], Aa[m], Ab[m], Acx[m], Acy[m]);
                        for (int n = 0; n < m; ++n)
                            g -= L[t * (t + 1) / 2 + n] * L[m * (m + 1) / 2 + n];
                        if (m == t) {
                            okf = okf && (g > (Q)0);
                            const Q d2 = sqrt(g > (Q)1e-30 ? g : (Q)1e-30);
                            L[t * (t + 1) / 2 + t] = d2;
                            dinv[t] = (Q)1 / d2;
                        } else {
                            L[t * (t + 1) / 2 + m] = g * dinv[m];
                        }
                    }
                if (!okf) { res.status = 2; break; }
            }
        }
        if (res.status != 0) break;
        if (!added) { res.status = 2; break; }
        sp_slot = scan(vb);
    }
    res.q = q;
    if (res.status == 0) {
        for (int t = 0; t < q; ++t)
            if (Ab[t] >= 0) {
                const Q dx = wsel4(Px, Aa[t]) - wsel4(Px, Ab[t]);
                const Q dy = wsel4(Py, Aa[t]) - wsel4(Py, Ab[t]);
                if (dx * dx + dy * dy - c.r2 < c.h_flag) res.flag = true;  // near-degenerate pair
            }
    } else {
        res.flag = true;
        if (res.status == 1) um = (Q)0;
    }
    return res;
}

}  // namespace rl
