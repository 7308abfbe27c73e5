"""Accuracy of the binary32 barrier QP when an active pair row is nearly degenerate (h < 1e-3 m²).

The dual active-set method (Goldfarb-Idnani on H = I; the Sec. 3 barrier QP) is run in emulated
binary32 -- every operation on numpy float32 scalars, rows formed in binary32 from binary32
projected points, the kernels' tolerances -- on QPs met along FP64 oracle rollouts, and compared
with the oracle's binary64 minimiser.  QPs with an active pair near contact (h < 1e-3 m², some with
h < 0) come out as close as the ordinary active QPs: a binary64 re-solve triggered by small h
alone would buy nothing, which is why rl_config.h_flag is off by default.  The emulation is test
code, written from the method's definition; it shares nothing with the CUDA kernels."""
import numpy as np

import oracle

F = np.float32


def rows32(c, px, py, N):
    g, r2 = F(c["gamma"]), F(c["r"]) * F(c["r"])
    kg, hr = F(c["kappa"]) * F(c["gamma"]), F(c["r"]) / F(2)
    A, b = [], []
    for a in range(N):
        for q in range(a + 1, N):
            dx, dy = px[a] - px[q], py[a] - py[q]
            h = dx * dx + dy * dy - r2
            row = np.zeros(2 * N, F)
            row[2 * a], row[2 * a + 1] = F(-2) * dx, F(-2) * dy
            row[2 * q], row[2 * q + 1] = F(2) * dx, F(2) * dy
            A.append(row)
            b.append(g * h * h * h)
    for i in range(N):
        d = [F(c["xmax"]) - hr - px[i], px[i] - F(c["xmin"]) - hr,
             F(c["ymax"]) - hr - py[i], py[i] - F(c["ymin"]) - hr]
        for s in range(4):
            row = np.zeros(2 * N, F)
            row[2 * i + (s >> 1)] = F(1) if s % 2 == 0 else F(-1)
            A.append(row)
            b.append(kg * d[s] * d[s] * d[s])
    return A, b


def solve32(A, b, u0, max_iter=60):
    """Dual active set in binary32: add the most violated row (ties: lowest index), step by
    min(tf, td), drop a row whose multiplier reaches zero."""
    n, m = len(u0), len(A)
    u = u0.copy()
    act, lam = [], []
    tol_abs, tol_rel, eps_dep = F(2e-7), F(1e-6), F(1e-5)
    for _ in range(max_iter):
        best, kb = F(0), -1
        for j in range(m):
            if j in act:
                continue
            v = F(np.dot(A[j], u)) - b[j]
            if v > tol_abs + tol_rel * abs(b[j]) and v > best:
                best, kb = v, j
        if kb < 0:
            return u, 0
        ap = A[kb]
        lam_p = F(0)
        while True:
            if act:
                Nm = np.array([A[j] for j in act], F)
                G = (Nm @ Nm.T).astype(F)
                r = np.linalg.solve(G, (Nm @ ap).astype(F)).astype(F)
                z = (ap - Nm.T @ r).astype(F)
            else:
                r, z = np.zeros(0, F), ap.copy()
            zz = F(np.dot(z, z))
            td, jb = F(np.inf), -1
            for t in range(len(act)):
                if r[t] > 0 and F(lam[t] / r[t]) < td:
                    td, jb = F(lam[t] / r[t]), t
            sp = F(np.dot(ap, u)) - b[kb]
            tf = sp / zz if zz > eps_dep * F(np.dot(ap, ap)) else F(np.inf)
            if not np.isfinite(tf) and not np.isfinite(td):
                return np.zeros(n, F), 1
            st = min(tf, td)
            if np.isfinite(tf):
                u = (u - st * z).astype(F)
            lam = [F(lv - st * r[t]) for t, lv in enumerate(lam)]
            lam_p = F(lam_p + st)
            if tf <= td:
                act.append(kb)
                lam.append(lam_p)
                break
            del act[jb]
            del lam[jb]
    return u, 2


def test_binary32_small_h_as_accurate_as_others():
    c = oracle.default_cfg(0, n_max=4)
    E, T = 4096, 720
    s = oracle.reset(c, 0, np.full(E, 4, np.int32))
    rng = np.random.default_rng(5)
    small, other = [], []
    for t in range(T):
        x, y, th = s.x.copy(), s.y.copy(), s.th.copy()
        _, _, _, tr = oracle.step(c, 0, s, trace=True)
        for e in np.nonzero(tr["qp"][:, 1] > 0)[0]:
            o = 4 * e
            px = x[o:o + 4] + c["l"] * np.cos(th[o:o + 4])
            py = y[o:o + 4] + c["l"] * np.sin(th[o:o + 4])
            hmin = min((px[a] - px[q]) ** 2 + (py[a] - py[q]) ** 2 - c["r"] ** 2
                       for a in range(4) for q in range(a + 1, 4))
            near = hmin < 1e-3
            if not near and (len(other) >= 1500 or rng.random() > 0.004):
                continue
            A, b = rows32(c, px.astype(F), py.astype(F), 4)
            u, st = solve32(A, b, tr["u_nom"][o:o + 4].reshape(-1).astype(F))
            err = np.abs(u.astype(np.float64) - tr["u_star"][o:o + 4].reshape(-1)).max()
            (small if near else other).append((err, st))
    es = np.array([e for e, _ in small])
    eo = np.array([e for e, _ in other])
    print(f"\nh < 1e-3: {len(es)} QPs, max {es.max():.2e}; others: {len(eo)} QPs, max {eo.max():.2e}")
    assert len(es) >= 20 and len(eo) >= 500
    assert all(st == 0 for _, st in small + other)
    # binary32 accuracy of a unit-scale minimiser: well inside the 1e-5 control tolerance, and
    # the near-contact QPs no worse than the others
    assert eo.max() < 1e-6
    assert es.max() <= max(2 * eo.max(), 1e-7)


def solve32_vec(A, b, u0, max_iter=200):
    """solve32 with the row scan vectorised (A u - b in binary32), for 40-variable QPs."""
    A = np.asarray(A, F)
    b = np.asarray(b, F)
    n, m = len(u0), len(A)
    u = u0.copy()
    act, lam = [], []
    tol_abs, tol_rel, eps_dep = F(2e-7), F(1e-6), F(1e-5)
    thr = (tol_abs + tol_rel * np.abs(b)).astype(F)
    for _ in range(max_iter):
        v = (A @ u).astype(F) - b
        v[act] = F(0)
        ok = v > thr
        if not ok.any():
            return u, 0
        kb = int(np.argmax(np.where(ok, v, F(-np.inf))))  # ties: lowest index
        ap = A[kb]
        lam_p = F(0)
        while True:
            if act:
                Nm = A[act]
                G = (Nm @ Nm.T).astype(F)
                r = np.linalg.solve(G, (Nm @ ap).astype(F)).astype(F)
                z = (ap - Nm.T @ r).astype(F)
            else:
                r, z = np.zeros(0, F), ap.copy()
            zz = F(np.dot(z, z))
            td, jb = F(np.inf), -1
            for t in range(len(act)):
                if r[t] > 0 and F(lam[t] / r[t]) < td:
                    td, jb = F(lam[t] / r[t]), t
            sp = F(np.dot(ap, u)) - b[kb]
            tf = sp / zz if zz > eps_dep * F(np.dot(ap, ap)) else F(np.inf)
            if not np.isfinite(tf) and not np.isfinite(td):
                return np.zeros(n, F), 1
            st = min(tf, td)
            if np.isfinite(tf):
                u = (u - st * z).astype(F)
            lam = [F(lv - st * r[t]) for t, lv in enumerate(lam)]
            lam_p = F(lam_p + st)
            if tf <= td:
                act.append(kb)
                lam.append(lam_p)
                break
            del act[jb]
            del lam[jb]
    return u, 2


def test_binary32_small_h_largen_near_pairs():
    """The 20-robot configuration with near pairs (1024 envs, 30% starting with a pair at
    0.18-0.20 m), the case the "h close to 0" re-solve was meant for: the active QPs met over
    the first 100 steps of an FP64 oracle rollout, those whose active set keeps a pair row with
    h < 1e-3 m^2 against a sample of the others, each solved in emulated binary32 and compared
    with the oracle's binary64 minimiser."""
    c = oracle.default_cfg(0, n_max=20, near_frac=0.3)
    N, E, T = 20, 1024, 100
    s = oracle.reset(c, 0, np.full(E, N, np.int32))
    rng = np.random.default_rng(11)
    near, other = [], []
    pairs = [(a, q) for a in range(N) for q in range(a + 1, N)]
    for t in range(T):
        x, y, th = s.x.copy(), s.y.copy(), s.th.copy()
        _, _, _, tr = oracle.step(c, 0, s, trace=True)
        if t % 4:
            continue  # every fourth step: QPs of the whole rollout, not one stretch of it
        for e in np.nonzero(tr["qp"][:, 1] > 0)[0]:
            if len(near) >= 60 and len(other) >= 60:
                break
            o = N * e
            px = x[o:o + N] + c["l"] * np.cos(th[o:o + N])
            py = y[o:o + N] + c["l"] * np.sin(th[o:o + N])
            A, b = rows32(c, px.astype(F), py.astype(F), N)
            u0 = tr["u_nom"][o:o + N].reshape(-1)
            us = tr["u_star"][o:o + N].reshape(-1)
            # the oracle's active pair rows: tight at its minimiser
            hs = [(px[a] - px[q]) ** 2 + (py[a] - py[q]) ** 2 - c["r"] ** 2 for a, q in pairs]
            slack = [np.dot(np.asarray(A[k], np.float64), us) - float(b[k]) for k in range(len(pairs))]
            h_act = min([h for h, sl in zip(hs, slack) if abs(sl) < 1e-6] or [np.inf])
            is_near = h_act < 1e-3
            if is_near and len(near) >= 60:
                continue
            if not is_near and (len(other) >= 60 or rng.random() > 0.05):
                continue
            u, st = solve32_vec(A, b, u0.astype(F))
            err = np.abs(u.astype(np.float64) - us).max()
            (near if is_near else other).append((err, st, h_act))
    en = np.array([e for e, _, _ in near])
    eo = np.array([e for e, _, _ in other])
    print(f"\nlargen near pairs: active pair h < 1e-3: {len(en)} QPs (min h "
          f"{min(h for _, _, h in near):.2e}), max err {en.max():.2e}; others: {len(eo)} QPs, "
          f"max err {eo.max():.2e}")
    assert len(en) >= 30 and len(eo) >= 30
    assert all(st == 0 for _, st, _ in near + other)
    # both inside the 1e-5 control tolerance, near contact no worse than the others
    assert eo.max() < 1e-5 and en.max() < 1e-5
    assert en.max() <= max(2 * eo.max(), 1e-6)
