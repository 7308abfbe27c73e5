"""Pins of the oracle's barrier-certificate QP (paper Sec. 4.1: the robust-CBF QP).

min |u - u_nom|^2 s.t. A u <= b is a Euclidean projection onto a polyhedron: its minimiser is
unique, so every exact solver must return the same u.  Pins: (i) u = u_nom bit for bit when
u_nom is feasible; (ii) brute-force enumeration of all active sets on 2- and 3-robot QPs;
(iii) KKT residuals on the QPs met along rollouts; (iv) the 2-robot head-on case, a projection
onto one half-plane with a closed form; (v) the row layout against the constraint definition.
"""
import itertools

import numpy as np
import pytest

import oracle

C = oracle.default_cfg()


def _brute_force(A, b, u0, tol=1e-9):
    """Every subset S of rows with independent normals: solve the equality-constrained projection,
    keep it if primal and dual feasible.  Returns the list of KKT points found."""
    m, n = A.shape
    sols = []
    for k in range(0, n + 1):
        for S in itertools.combinations(range(m), k):
            if k == 0:
                u = u0.copy()
                lam = np.zeros(0)
            else:
                AS = A[list(S)]
                G = AS @ AS.T
                if np.linalg.matrix_rank(G, tol=1e-10) < k:
                    continue
                lam = np.linalg.solve(G, AS @ u0 - b[list(S)])
                u = u0 - AS.T @ lam
            if np.all(lam >= -tol) and np.all(A @ u - b <= tol * (1 + np.abs(b))):
                sols.append(u)
    return sols


def _instance(rng, N, spread, speed):
    """Projected points clustered in a small box near a wall, nominal velocities pointing
    towards the cluster centre and the wall so that many rows are active."""
    cx, cy = rng.uniform(0.9, 1.35), rng.uniform(-0.5, 0.5)
    for _ in range(1000):
        px = cx + rng.uniform(-spread, spread, N)
        py = cy + rng.uniform(-spread, spread, N)
        d = np.hypot(px[:, None] - px[None], py[:, None] - py[None]) + 9 * np.eye(N)
        if d.min() > 0.175:
            break
    ang = rng.uniform(-np.pi, np.pi, N)
    u0 = np.empty(2 * N)
    u0[0::2] = speed * (np.cos(ang) + 0.8 * (cx - px) / spread + 0.5)
    u0[1::2] = speed * (np.sin(ang) + 0.8 * (cy - py) / spread)
    return px, py, u0


@pytest.mark.parametrize("N,cases", [(2, 60), (3, 25)])
def test_qp_matches_brute_force_enumeration(N, cases):
    rng = np.random.default_rng(100 + N)
    n_active_seen = set()
    for _ in range(cases):
        px, py, u0 = _instance(rng, N, spread=0.25, speed=0.2)
        A, b = oracle.cbf_rows(C, px, py)
        u, lam, st, q, _ = oracle.qp_project(A, b, u0)
        assert st == 0
        n_active_seen.add(q)
        sols = _brute_force(A, b, u0)
        assert len(sols) >= 1
        for s in sols:
            assert np.max(np.abs(s - sols[0])) < 1e-9  # uniqueness
        assert np.max(np.abs(u - sols[0])) < 1e-10
    assert max(n_active_seen) >= 2  # the instances exercise multi-row active sets


def test_qp_inactive_returns_nominal_bit_exact():
    rng = np.random.default_rng(1)
    for _ in range(200):
        N = int(rng.integers(2, 8))
        ang = np.linspace(0, 2 * np.pi, N, endpoint=False)
        px, py = 0.6 * np.cos(ang) * 1.5, 0.6 * np.sin(ang)
        u0 = rng.uniform(-0.02, 0.02, 2 * N)
        A, b = oracle.cbf_rows(C, px, py)
        assert np.all(A @ u0 <= b)
        u, lam, st, q, it = oracle.qp_project(A, b, u0)
        assert st == 0 and q == 0 and it == 0
        assert np.array_equal(u, u0)


def test_qp_head_on_half_plane_projection():
    # two robots on the x axis approaching each other: only the pair row can be active
    for gap, v in [(0.3, 0.2), (0.2, 0.15), (0.18, 0.05), (0.5, 0.2)]:
        px, py = np.array([-gap / 2, gap / 2]), np.array([0.0, 0.0])
        u0 = np.array([v, 0.01, -v, -0.02])
        A, b = oracle.cbf_rows(C, px, py)
        a, bb = A[0], b[0]
        h = gap ** 2 - 0.17 ** 2
        assert np.allclose(a, [2 * gap, 0, -2 * gap, 0]) and abs(bb - 100 * h ** 3) < 1e-15
        expect = u0 - max(0.0, a @ u0 - bb) / (a @ a) * a
        u, lam, st, q, _ = oracle.qp_project(A, b, u0)
        assert st == 0
        assert np.max(np.abs(u - expect)) < 1e-14


def test_cbf_row_layout():
    N = 4
    rng = np.random.default_rng(3)
    px, py = rng.uniform(-1.2, 1.2, N), rng.uniform(-0.7, 0.7, N)
    A, b = oracle.cbf_rows(C, px, py)
    assert A.shape == (6 + 16, 8)
    k = 0
    for i in range(N):
        for j in range(i + 1, N):
            d = np.array([px[i] - px[j], py[i] - py[j]])
            u = rng.normal(size=8)
            # -2 (p_i - p_j) . (u_i - u_j)
            assert abs(A[k] @ u - (-2 * d @ (u[2 * i:2 * i + 2] - u[2 * j:2 * j + 2]))) < 1e-12
            assert abs(b[k] - 100 * (d @ d - 0.17 ** 2) ** 3) < 1e-12
            k += 1
    for i in range(N):
        dists = [1.6 - 0.085 - px[i], px[i] + 1.6 - 0.085, 1.0 - 0.085 - py[i], py[i] + 1.0 - 0.085]
        for s, (col, sgn) in enumerate([(2 * i, 1), (2 * i, -1), (2 * i + 1, 1), (2 * i + 1, -1)]):
            row = np.zeros(8)
            row[col] = sgn
            assert np.array_equal(A[k], row)
            assert abs(b[k] - 0.4 * 100 * dists[s] ** 3) < 1e-12
            k += 1


@pytest.mark.parametrize("N,near", [(4, 0.0), (10, 0.0), (20, 0.3)])
def test_qp_kkt_residuals_along_rollouts(N, near):
    c = oracle.default_cfg(n_max=N, near_frac=near)
    E = 32 if N <= 10 else 16
    s = oracle.reset(c, 21, [N] * E)
    worst = 0.0
    active = 0
    for _ in range(60):
        _, _, _, tr = oracle.step(c, 21, s, trace=True)
        assert np.all(tr["qp"][:, 0] == 0)
        worst = max(worst, tr["kkt"].max())
        active += tr["qp"][:, 1].sum()
    assert active > 0
    assert worst < 1e-10


@pytest.mark.parametrize("arena", ["default", "crowded"])
def test_pair_rows_first_reaches_the_same_minimiser(arena):
    """The 4-robot team QP of the GPU kernels solves over the pair rows alone first and checks
    the arena rows only at that point: a minimiser of the relaxation that meets every row is the
    minimiser of the whole QP.  Checked with the oracle's own solver on the QPs met along a
    4-robot rollout: wherever the pair rows' minimiser meets the arena rows it equals the full
    minimiser.  In the default arena the pair rows alone decide nearly every QP with an active
    row; a crowded arena (1.2 m x 1.0 m, weak arena gain, strong noise) also meets QPs whose
    relaxation leaves an arena row violated, where the full solve must go on."""
    kw = {} if arena == "default" else dict(xmin=-0.6, xmax=0.6, ymin=-0.5, ymax=0.5,
                                            kappa=0.05, noise_amp=0.3, init_margin=0.15)
    c = oracle.default_cfg(oracle.NAV, n_max=4, **kw)
    E, N = 256, 4
    s = oracle.reset(c, 21, [N] * E)
    P = N * (N - 1) // 2
    checked = active = needs_arena = 0
    for t in range(40):
        x, y, th = s.x.reshape(E, N), s.y.reshape(E, N), s.th.reshape(E, N)
        px, py = x + c["l"] * np.cos(th), y + c["l"] * np.sin(th)
        _, _, _, tr = oracle.step(c, 21, s, trace=True)
        u0 = tr["u_nom"].reshape(E, 2 * N)
        for e in range(0, E, 4):
            A, b = oracle.cbf_rows(c, px[e], py[e])
            u_full, _, st, q, _ = oracle.qp_project(A, b, u0[e])
            if st != 0 or q == 0:
                continue
            active += 1
            u_pair, _, st_p, _, _ = oracle.qp_project(A[:P], b[:P], u0[e])
            assert st_p == 0
            viol = A[P:] @ u_pair - b[P:]
            if np.all(viol <= 1e-12 * (1 + np.abs(b[P:]))):
                checked += 1
                assert np.abs(u_pair - u_full).max() < 1e-12
            else:
                needs_arena += 1
                assert np.all(A @ u_full - b <= 1e-10 * (1 + np.abs(b)))
    assert checked > 100
    if arena == "default":
        assert needs_arena <= 0.05 * active
    else:
        assert needs_arena > 0
