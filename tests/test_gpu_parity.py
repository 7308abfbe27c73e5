"""Parity of the CUDA step (through the C ABI) with the FP64 oracle.

Bars: integer outputs (done flags, counters, levels, resource states, sampled initial states)
bit-exact; binary64 GPU path within 1e-9 of the oracle; binary32 path: filtered controls within
1e-5 per step (teacher-forced: both sides step from the same state), poses within 1e-4 after
100 free-running steps.  Max errors are printed per case.
"""
import numpy as np
import pytest

import oracle
from pairing import make_pair, obs_diff, to_oracle_state, wrap

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U_TOL = 1e-5      # filtered SI velocity, binary32
POSE_TOL = 1e-4   # poses after 100 free-running steps, binary32
# pose error of one step from the same state, for kernels that write no control traces: a
# filtered-velocity error e moves the projected point by dt * e, so U_TOL * dt bounds it
POSE_STEP_TOL = 3e-7


@pytest.fixture(scope="module")
def rl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2505_06771_gb300 as m
    m.build()
    return m


def _alloc(env, T=None):
    dt = env.dtype
    R, E, od = env.total_robots, env.n_envs, env.obs_dim
    if T is None:
        return dict(obs=torch.zeros(R, od, dtype=dt, device="cuda"),
                    reward=torch.zeros(E, dtype=dt, device="cuda"),
                    done=torch.zeros(E, dtype=torch.uint8, device="cuda"),
                    u_nom=torch.zeros(R, 2, dtype=dt, device="cuda"),
                    u_star=torch.zeros(R, 2, dtype=dt, device="cuda"),
                    vw=torch.zeros(R, 2, dtype=dt, device="cuda"),
                    qp_info=torch.zeros(E, 4, dtype=torch.int32, device="cuda"))
    return dict(obs=torch.zeros(T, R, od, dtype=dt, device="cuda"),
                reward=torch.zeros(T, E, dtype=dt, device="cuda"),
                done=torch.zeros(T, E, dtype=torch.uint8, device="cuda"))


def _check_reset_state(g, o, st, n_robots, seed):
    s = oracle.reset(o, seed, n_robots)
    for k in ("x", "y", "th", "gx", "gy", "gth"):
        assert np.array_equal(st[k].astype(np.float64), getattr(s, k)), k
    assert np.array_equal(st["level"], s.level)
    assert np.array_equal(st["n_res"], s.n_res)
    if o["r_max"] > 0:
        assert np.array_equal(st["qx"].astype(np.float64), s.qx)
        assert np.array_equal(st["qlevel"], s.qlevel)
        assert np.array_equal(st["qactive"], s.qactive)


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("case", ["nav4", "nav20_near", "forage_uneven", "nav_edge", "disc_uneven"])
def test_reset_sampler_bit_exact(rl, prec, case):
    if case == "nav4":
        g, o = make_pair(0, 4, prec)
        n = [4] * 300
    elif case == "nav20_near":
        g, o = make_pair(0, 20, prec, near_frac=0.3)
        n = [20] * 64
    elif case == "forage_uneven":
        g, o = make_pair(1, 10, prec)
        n = list(np.random.default_rng(5).integers(2, 11, 257))
    elif case == "disc_uneven":
        g, o = make_pair(2, 10, prec)
        n = list(np.random.default_rng(6).integers(1, 11, 130))
    else:
        g, o = make_pair(0, 32, prec)
        n = [1, 2, 3, 5, 8, 9, 16, 17, 31, 32, 4]
    seed = 0xC0FFEE
    env = rl.Env(g, len(n), n, seed)
    _check_reset_state(g, o, env.state_arrays(), n, seed)
    env.close()


def _teacher_forced(rl, g, o, n, seed, steps, actions=False, traces=True):
    """Both sides step from the same state.  traces=False calls the step with observations,
    rewards and done flags only, which selects the kernels that write no traces (the 4-robot
    Navigation fast paths the configuration names)."""
    env = rl.Env(g, len(n), n, seed)
    b = _alloc(env)
    if not traces:
        for k in ("u_nom", "u_star", "vw", "qp_info"):
            b[k] = None
    err = dict(u_nom=0.0, u_star=0.0, v=0.0, w=0.0, pose=0.0, th=0.0, rew=0.0, obs=0.0)
    rng = np.random.default_rng(seed)
    flagged = 0
    for t in range(steps):
        st = env.state_arrays()
        s = to_oracle_state(o, st)
        act_t = None
        act_o = None
        if actions:
            a = rng.uniform(-0.3, 0.3, (env.total_robots, 2)).astype(env.np_dtype)
            act_t = torch.from_numpy(a).cuda()
            act_o = a.astype(np.float64)
        obs_o, rew_o, done_o, tr = oracle.step(o, seed, s, actions=act_o, trace=True)
        env.step(actions=act_t, **b)
        torch.cuda.synchronize()
        st2 = env.state_arrays()
        done_g = b["done"].cpu().numpy()
        assert np.array_equal(done_g, done_o), f"done differs at step {t}"
        if traces:
            err["u_nom"] = max(err["u_nom"], np.abs(b["u_nom"].cpu().numpy() - tr["u_nom"]).max())
            err["u_star"] = max(err["u_star"],
                                np.abs(b["u_star"].cpu().numpy() - tr["u_star"]).max())
            vw = b["vw"].cpu().numpy()
            err["v"] = max(err["v"], np.abs(vw[:, 0] - tr["vw"][:, 0]).max())
            err["w"] = max(err["w"], np.abs(vw[:, 1] - tr["vw"][:, 1]).max())
        err["pose"] = max(err["pose"], np.abs(st2["x"] - s.x).max(), np.abs(st2["y"] - s.y).max())
        err["th"] = max(err["th"], np.abs(wrap(st2["th"] - s.th)).max())
        err["rew"] = max(err["rew"], np.abs(b["reward"].cpu().numpy() - rew_o).max())
        err["obs"] = max(err["obs"], obs_diff(b["obs"].cpu().numpy(), obs_o, g["scenario"],
                                              g["n_max"], g["r_max"]))
        assert np.array_equal(st2["t"], s.t) and np.array_equal(st2["ep"], s.ep)
        assert np.array_equal(st2["level"], s.level)
        # goals change only through exact draws (reset, waypoint arrival)
        assert np.array_equal(st2["gx"].astype(np.float64), s.gx), f"goals differ at step {t}"
        assert np.array_equal(st2["gy"].astype(np.float64), s.gy), f"goals differ at step {t}"
        assert np.array_equal(st2["gth"].astype(np.float64), s.gth), f"goal headings differ at {t}"
        if o["r_max"] > 0:
            assert np.array_equal(st2["qactive"], s.qactive), f"resources differ at step {t}"
            assert np.array_equal(st2["qlevel"], s.qlevel), f"resource levels differ at {t}"
        cg, co = st2["counters"], s.counters.reshape(-1, 8)
        for c in (0, 1, 2, 6):
            assert np.array_equal(cg[:, c], co[:, c]), f"counter {c} differs at step {t}"
        if traces:
            qi = b["qp_info"].cpu().numpy()
            flagged += int(((qi[:, 3] >> 1) & 1).sum())
    if not traces:
        flagged = int(env.state_arrays()["counters"][:, 4].sum())
    env.close()
    return err, flagged


@pytest.mark.parametrize("case", ["nav4_scripted", "nav4_policy", "nav10", "forage_uneven",
                                  "nav20_near", "disc4", "disc_uneven"])
def test_teacher_forced_binary32(rl, case):
    seed = 77
    if case == "nav4_scripted":
        g, o = make_pair(0, 4)
        n, steps, act = [4] * 300, 40, False
    elif case == "nav4_policy":
        g, o = make_pair(0, 4, scripted=0)
        n, steps, act = [4] * 300, 30, True
    elif case == "nav10":
        g, o = make_pair(0, 10)
        n, steps, act = [10] * 96, 30, False
    elif case == "forage_uneven":
        g, o = make_pair(1, 10, episode_len=30)
        n, steps, act = list(np.random.default_rng(2).integers(2, 11, 200)), 40, False
    elif case == "disc4":
        g, o = make_pair(2, 4, episode_len=30)
        n, steps, act = [4] * 300, 40, False
    elif case == "disc_uneven":
        g, o = make_pair(2, 10, episode_len=30)
        n, steps, act = list(np.random.default_rng(4).integers(1, 11, 200)), 40, False
    else:
        g, o = make_pair(0, 20, near_frac=0.3)
        n, steps, act = [20] * 40, 25, False
    err, flagged = _teacher_forced(rl, g, o, n, seed, steps, actions=act)
    print(f"\n{case}: max errors {err}  fp64-resolved QPs {flagged}")
    assert err["u_nom"] < 1e-6
    assert err["u_star"] < U_TOL
    assert err["v"] < U_TOL and err["w"] < U_TOL / g["l"]
    assert err["pose"] < POSE_STEP_TOL and err["th"] < 1e-5
    assert err["rew"] < 1e-5 and err["obs"] < 1e-5


@pytest.mark.parametrize("case", ["nav8", "nav20_near", "forage_uneven"])
def test_teacher_forced_large_binary64_resolve(rl, case):
    """The binary64 re-solve of the classes over four robots (the explicit-inverse form in
    binary64, with the Cholesky form behind it for active sets beyond its slots): h_flag = 10 m^2
    flags every QP that keeps an active pair row, so most steps are re-solved; the minimisers
    against the oracle's, stepped from the same states."""
    seed = 91
    if case == "nav8":
        g, o = make_pair(0, 8, h_flag=10.0)
        n, steps = [8] * 128, 20
    elif case == "nav20_near":
        g, o = make_pair(0, 20, near_frac=0.3, h_flag=10.0)
        n, steps = [20] * 40, 20
    else:
        g, o = make_pair(1, 10, episode_len=30, h_flag=10.0)
        n, steps = list(np.random.default_rng(8).integers(5, 11, 200)), 20
    err, flagged = _teacher_forced(rl, g, o, n, seed, steps)
    print(f"\n{case} (h_flag 10): max errors {err}  fp64-resolved QPs {flagged}")
    assert flagged > 0
    assert err["u_star"] < U_TOL
    assert err["pose"] < POSE_STEP_TOL and err["rew"] < 1e-5 and err["obs"] < 1e-5


def test_largen_near_contact_default_flag(rl):
    """The 20-robot configuration at full size (1024 envs, 30% with a near pair) under the
    default re-solve flag (no binary64 re-solve for small h alone): after 30 scripted steps
    (mid-episode, when near pairs have closed in), traced steps with the filtered controls u* against the oracle's binary64 minimiser, reported
    separately for the QPs whose active set keeps a pair row with h < 1e-3 m^2."""
    N, E, seed = 20, 1024, 1000
    g, o = make_pair(0, N, near_frac=0.3)
    env = rl.Env(g, E, N, seed)
    env.rollout(30)
    b = _alloc(env)
    pairs = [(a, q) for a in range(N) for q in range(a + 1, N)]
    err_near, err_all, n_near = 0.0, 0.0, 0
    for t in range(4):
        st = env.state_arrays()
        s = to_oracle_state(o, st)
        _, _, _, tr = oracle.step(o, seed, s, trace=True)
        env.step(**b)
        torch.cuda.synchronize()
        du = np.abs(b["u_star"].cpu().numpy() - tr["u_star"]).reshape(E, 2 * N).max(1)
        err_all = max(err_all, float(du.max()))
        px = (st["x"] + g["l"] * np.cos(st["th"].astype(np.float64))).reshape(E, N)
        py = (st["y"] + g["l"] * np.sin(st["th"].astype(np.float64))).reshape(E, N)
        us = tr["u_star"].reshape(E, N, 2)
        for e in np.nonzero(tr["qp"][:, 1] > 0)[0]:
            for a, q in pairs:
                dx, dy = px[e, a] - px[e, q], py[e, a] - py[e, q]
                h = dx * dx + dy * dy - g["r"] ** 2
                if h >= 1e-3:
                    continue
                # pair row tight at the oracle's minimiser
                v = -2 * (dx * (us[e, a, 0] - us[e, q, 0]) + dy * (us[e, a, 1] - us[e, q, 1]))
                if abs(v - g["gamma"] * h ** 3) < 1e-6:
                    n_near += 1
                    err_near = max(err_near, float(du[e]))
                    break
    flagged = int(env.state_arrays()["counters"][:, 4].sum())
    print(f"\nlargen default flag: {n_near} QPs with an active pair at h < 1e-3, max u* error "
          f"{err_near:.2e}; all QPs {err_all:.2e}; binary64 re-solves {flagged}")
    assert n_near >= 30
    assert err_all < U_TOL and err_near < U_TOL
    env.close()


FAST_KERNELS = dict(shuffle=dict(small_variant=1), gather=dict(small_variant=2),
                    split=dict(small_variant=3), thread=dict(lanes=1))


# E = 1: the spread launch's single block; E = 5000: more envs than 8 per warp of one block per
# SM (4864 on 152 SMs), so the team kernels fall back to a grid stride
@pytest.mark.parametrize("kern", list(FAST_KERNELS))
@pytest.mark.parametrize("N,E", [(4, 600), (3, 300), (2, 200), (4, 1), (4, 5000)])
def test_teacher_forced_fast_kernels(rl, kern, N, E):
    """The Navigation fast paths (scripted nominal control, no traces): the 4-lane team kernel
    that reduces with shuffles, the one that publishes robot state in shared memory, and one
    thread per env.  Poses, observations and rewards against the oracle stepped from the same
    state.  A pose error within U_TOL * dt = 3e-7 m per step bounds the filtered-control
    error by the control tolerance 1e-5 (an active-set mistake moves a robot by ~1e-4 m per
    step)."""
    g, o = make_pair(0, N, episode_len=30, **FAST_KERNELS[kern])
    err, _ = _teacher_forced(rl, g, o, [N] * E, 91, 40, traces=False)
    print(f"\n{kern} kernel N={N}: max errors {err}")
    assert err["pose"] < POSE_STEP_TOL and err["th"] < 2e-5
    assert err["rew"] < 1e-5 and err["obs"] < 1e-5


@pytest.mark.parametrize("N,E", [(4, 600), (3, 300), (4, 1)])
def test_teacher_forced_policy_actions_split_kernel(rl, N, E):
    """Policy actions without traces (the policy-in-the-loop step) run the split kernel, its
    dynamics taking the actions as nominal velocities: poses, observations and rewards against
    the oracle stepped from the same state with the same actions."""
    g, o = make_pair(0, N, scripted=0, episode_len=30)
    err, _ = _teacher_forced(rl, g, o, [N] * E, 63, 35, actions=True, traces=False)
    print(f"\nsplit kernel, policy actions, N={N} E={E}: max errors {err}")
    assert err["pose"] < POSE_STEP_TOL and err["th"] < 2e-5
    assert err["rew"] < 1e-5 and err["obs"] < 1e-5


# Crowded arena: with a weak wall barrier and strong noise about 5% of the QPs keep five or more
# active rows (up to seven); h_flag = 10 m^2 flags every QP with an active pair row for the
# binary64 re-solve.
CROWDED = dict(xmin=-0.6, xmax=0.6, ymin=-0.5, ymax=0.5, kappa=0.05, noise_amp=0.3)
WARP_CASES = dict(binary64=(0, dict(h_flag=10.0), False),
                  crowded=(0, CROWDED, False),
                  crowded_binary64=(0, dict(CROWDED, h_flag=10.0), False),
                  # 4 envs per warp with a grid stride: the teams' own shared-memory solvers
                  crowded_binary64_team=(0, dict(CROWDED, h_flag=10.0, warp_envs=4), False),
                  # with traces: the general 4-robot kernel and its team solvers, filtered
                  # controls compared too
                  crowded_binary64_traces=(0, dict(CROWDED, h_flag=10.0), True),
                  # the split kernel: active sets beyond four rows solved in the team with
                  # room for eight rows
                  crowded_split=(0, dict(CROWDED, small_variant=3), False),
                  crowded_split_binary64=(0, dict(CROWDED, h_flag=10.0, small_variant=3), False),
                  discovery_binary64=(2, dict(CROWDED, h_flag=10.0), True))


@pytest.mark.parametrize("case", list(WARP_CASES))
def test_teacher_forced_warp_rare_qps(rl, case):
    """2048 envs spread over one block of 4 warps per SM put 3-4 envs in each warp of the shuffle
    kernel, which then solves its rare QPs -- an active set beyond the four rows of the register
    solver, and the binary64 re-solve of a flagged QP -- with the whole warp; the same crowded
    batches through the teams' own solvers as controls.  Poses, observations and rewards (and
    with traces the filtered controls) against the oracle stepped from the same state."""
    scen, kw, traces = WARP_CASES[case]
    extra = {} if traces or "small_variant" in kw else dict(small_variant=1)
    g, o = make_pair(scen, 4, episode_len=30, **extra, **kw)
    err, flagged = _teacher_forced(rl, g, o, [4] * 2048, 57, 30, traces=traces)
    print(f"\nwarp-solved rare QPs, {case}: max errors {err}  binary64 re-solves {flagged}")
    if "binary64" in case:
        assert flagged > 1000
    if traces:
        assert err["u_star"] < U_TOL
    assert err["pose"] < POSE_STEP_TOL and err["th"] < 2e-5
    assert err["rew"] < 1e-5 and err["obs"] < 1e-5


@pytest.mark.parametrize("case", ["nav4", "nav4_shuffle", "nav4_gather", "nav4_split",
                                  "nav4_thread", "nav3", "nav10", "nav4_f64"])
def test_teacher_forced_waypoints(rl, case):
    """Random Waypoint Navigation (goal reassigned on arrival): every kernel that runs 4-robot,
    3-robot, 10-robot and binary64 Navigation against the oracle stepped from the same state.
    The arrival radius is large so that arrivals happen within the 40 steps; goals, arrival
    counts and done flags are compared exactly."""
    N = 10 if case == "nav10" else (3 if case == "nav3" else 4)
    prec = 64 if case == "nav4_f64" else 32
    kern = case.split("_")[1] if case in ("nav4_shuffle", "nav4_gather", "nav4_split",
                                          "nav4_thread") else None
    g, o = make_pair(0, N, prec, goal_eps=0.35, episode_len=10_000,
                     **(FAST_KERNELS[kern] if kern else {}))
    E = 96 if N == 10 else 300
    err, _ = _teacher_forced(rl, g, o, [N] * E, 23, 40, traces=kern is None)
    print(f"\nwaypoints {case}: max errors {err}")
    tol = 1e-5 if prec == 64 else 1.0
    assert err["pose"] < POSE_STEP_TOL * tol and err["rew"] < 1e-5 * tol and err["obs"] < 1e-5 * tol


def test_waypoint_arrivals_counted_in_rollout(rl):
    """Rollout (persistent kernel) and step-at-a-time agree in waypoint mode, and arrivals are
    counted: the success counter equals the number of goal changes seen in the observations."""
    g, _ = make_pair(0, 4, goal_eps=0.2, episode_len=10_000)
    n, T = [4] * 64, 120
    a = rl.Env(g, 64, n, 4)
    bt = _alloc(a, T)
    a.rollout(T, **bt)
    b = rl.Env(g, 64, n, 4)
    for t in range(T):
        bs = _alloc(b)
        b.step(obs=bs["obs"], reward=bs["reward"], done=bs["done"])
        assert torch.equal(bs["obs"], bt["obs"][t]) and torch.equal(bs["done"], bt["done"][t])
    assert a.get_state() == b.get_state()
    goals = bt["obs"][:, :, 3:5].cpu().numpy()
    changes = (np.abs(np.diff(goals, axis=0)).sum(-1) > 0).reshape(T - 1, 64, 4).sum()
    first = a.state_arrays()  # counters include the arrivals of step 0 as well
    succ = int(first["counters"][:, 2].sum())
    assert succ >= changes > 0
    a.close()
    b.close()


@pytest.mark.parametrize("case", ["nav4", "nav4_fast_path_off", "nav10", "nav4_f64",
                                  "nav4_waypoint"])
def test_teacher_forced_pose_controller(rl, case):
    """Navigation under the unicycle pose controller (goal heading drawn with the goal): the
    nominal command, the filtered command and the step against the oracle stepped from the same
    state, for the 4-robot register kernel, the 10-robot team kernel, binary64 and waypoint
    mode (goal pose redrawn on arrival).  Without traces the step takes the gather kernel, the
    one Navigation fast path that implements the pose controller."""
    N = 10 if case == "nav10" else 4
    prec = 64 if case == "nav4_f64" else 32
    kw = dict(controller=1, episode_len=30)
    if case == "nav4_waypoint":
        kw.update(goal_eps=0.35, episode_len=10_000)
    g, o = make_pair(0, N, prec, **kw)
    E = 96 if N == 10 else 300
    err, _ = _teacher_forced(rl, g, o, [N] * E, 29, 40, traces=(case != "nav4_fast_path_off"))
    print(f"\npose controller {case}: max errors {err}")
    # the pose law is a chain of trigonometric functions: in binary32 its nominal velocity is
    # held to the control tolerance (1e-5), not the 1e-6 of the position law
    tol = 1e-8 if prec == 64 else 1.0
    assert err["u_nom"] < U_TOL * tol and err["u_star"] < U_TOL * tol
    assert err["pose"] < 1e-6 * tol and err["th"] < 1e-5 * tol
    assert err["rew"] < 1e-5 * tol and err["obs"] < 1e-5 * tol


@pytest.mark.parametrize("scenario", [0, 2])
def test_teacher_forced_binary64(rl, scenario):
    g, o = make_pair(scenario, 4, 64, episode_len=30)
    err, _ = _teacher_forced(rl, g, o, [4] * 64, 5, 40)
    print(f"\nfp64 teacher-forced, scenario {scenario}: {err}")
    for k, v in err.items():
        assert v < 1e-11, (k, v)


def test_tiny_config_free_run_binary64(rl):
    """16 envs x 4 robots, 100 steps, binary64: one full episode, ending in auto-reset."""
    g, o = make_pair(0, 4, 64)
    n, seed, T = [4] * 16, 0, 100
    env = rl.Env(g, 16, n, seed)
    b = _alloc(env, T)
    env.rollout(T, **b)
    torch.cuda.synchronize()
    s = oracle.reset(o, seed, n)
    obs_o, rew_o, done_o = oracle.rollout(o, seed, s, T)
    d_obs = obs_diff(b["obs"].cpu().numpy(), obs_o, 0, 4, 0)
    d_rew = np.abs(b["reward"].cpu().numpy() - rew_o).max()
    print(f"\ntiny fp64 free run: obs {d_obs:.3e} reward {d_rew:.3e}")
    assert np.array_equal(b["done"].cpu().numpy(), done_o)
    assert done_o[-1].all() and not done_o[:-1].any()
    assert d_obs < 1e-9 and d_rew < 1e-9
    assert np.array_equal(env.counters()[:, [0, 1, 2, 6]], s.counters.reshape(-1, 8)[:, [0, 1, 2, 6]])
    env.close()


@pytest.mark.parametrize("N,E", [(4, 16), (4, 257), (10, 64)])
def test_free_run_binary32_poses_after_100_steps(rl, N, E):
    g, o = make_pair(0, N, episode_len=1000)
    n, seed = [N] * E, 3
    env = rl.Env(g, E, n, seed)
    env.rollout(100)
    st = env.state_arrays()
    s = oracle.reset(o, seed, n)
    oracle.rollout(o, seed, s, 100, want_obs=False)
    dp = max(np.abs(st["x"] - s.x).max(), np.abs(st["y"] - s.y).max())
    dth = np.abs(wrap(st["th"] - s.th)).max()
    print(f"\nN={N} E={E} fp32 free run 100 steps: max pose err {dp:.3e} m, heading {dth:.3e}")
    assert dp < POSE_TOL
    env.close()


@pytest.mark.parametrize("scenario", [1, 0])
def test_free_run_uneven_one_launch_100_steps(rl, scenario):
    """The one persistent launch over every size class (the uneven benchmark's kernel), free
    running for 100 steps from the sampled start (one whole episode) on 2..10 robots per env,
    against the FP64 oracle: done flags, counters and resource states exact, positions within
    1e-4 m over the 100 steps, and the 100 rewards of every env."""
    from synth_inputs import uneven_robot_counts
    n = uneven_robot_counts(3, 600, 2, 10)
    g, o = make_pair(scenario, 10)
    E, seed, T = len(n), 17, 100
    env = rl.Env(g, E, n, seed)
    env.set_class_launch(1)
    b = _alloc(env, T)
    env.rollout(T, **b)
    torch.cuda.synchronize()
    st = env.state_arrays()
    s = oracle.reset(o, seed, n)
    obs_o, rew_o, done_o = oracle.rollout(o, seed, s, T)
    assert np.array_equal(b["done"].cpu().numpy(), done_o)
    for c in (0, 1, 2, 6):
        assert np.array_equal(st["counters"][:, c], s.counters.reshape(-1, 8)[:, c]), c
    if o["r_max"] > 0:
        assert np.array_equal(st["qactive"], s.qactive)
    # the state after step 99 is the auto-reset of episode 1 (exact draws), so the poses are
    # compared in the observations' own pose columns (x, y, heading) of steps 0..98; the
    # positions against the 1e-4 m bar, the heading reported (an active-set switch within
    # rounding can turn a heading by ~1e-3 rad, as in the 257-env case above)
    og, oo = b["obs"].cpu().numpy()[:T - 1].astype(np.float64), obs_o[:T - 1]
    d_pos = float(np.abs(og[..., :2] - oo[..., :2]).max())
    d_head = float(np.abs(wrap(og[..., 2] - oo[..., 2])).max())
    d_rew = np.abs(b["reward"].cpu().numpy() - rew_o).max()
    print(f"\none launch free run, scenario {scenario}: positions {d_pos:.3e} m, headings "
          f"{d_head:.3e} rad over 99 steps, reward {d_rew:.3e}")
    assert d_pos < POSE_TOL and d_rew < 1e-4
    env.close()


def test_rollout_equals_steps_and_plain_form(rl):
    g, _ = make_pair(0, 4, episode_len=20)
    n, T = [4] * 130, 45
    a = rl.Env(g, 130, n, 9)
    bt = _alloc(a, T)
    a.rollout(T, **bt)
    b = rl.Env(g, 130, n, 9)
    for t in range(T):
        bs = _alloc(b)
        b.step(obs=bs["obs"], reward=bs["reward"], done=bs["done"])
        assert torch.equal(bs["obs"], bt["obs"][t]) and torch.equal(bs["reward"], bt["reward"][t])
        assert torch.equal(bs["done"], bt["done"][t])
    c = rl.Env(g, 130, n, 9)
    bp = _alloc(c, T)
    c.rollout(T, plain=True, **bp)
    assert torch.equal(bp["obs"], bt["obs"]) and torch.equal(bp["done"], bt["done"])
    assert a.get_state() == b.get_state() == c.get_state()
    for e in (a, b, c):
        e.close()


def test_split_rollout_equals_steps_crowded(rl):
    """The split kernel in a crowded arena (many jammed envs, whose QPs keep more active rows
    than the team's register solver holds): one 30-step launch and 30 one-step launches give
    the same trajectories and state bit for bit."""
    g, _ = make_pair(0, 4, episode_len=20, small_variant=3, **CROWDED)
    n, T = [4] * 2048, 30
    a = rl.Env(g, 2048, n, 19)
    bt = _alloc(a, T)
    a.rollout(T, **bt)
    b = rl.Env(g, 2048, n, 19)
    for t in range(T):
        bs = _alloc(b)
        b.step(obs=bs["obs"], reward=bs["reward"], done=bs["done"])
        assert torch.equal(bs["obs"], bt["obs"][t]) and torch.equal(bs["reward"], bt["reward"][t])
        assert torch.equal(bs["done"], bt["done"][t])
    assert a.get_state() == b.get_state()
    c = a.counters()
    print(f"\nsplit crowded: {int(c[:, 3].sum())} active QPs, {int(c[:, 4].sum())} re-solved in "
          "binary64")
    a.close()
    b.close()


@pytest.mark.parametrize("episode_len", [1, 2, 3, 4, 7])
def test_split_rollout_equals_steps_episode_ends(rl, episode_len):
    """The split kernel's output warps draw the action noise three steps ahead and sample each
    next episode's start ahead of its end; the dynamics warps draw and sample themselves where
    that is too close (the first three steps of a launch, episodes shorter than three steps, a
    first episode end before step 2).  Launches of 29 steps started mid-episode give the same
    trajectories and state as 29 one-step launches (which take only the dynamics warps' own
    draws), bit for bit, for episode lengths around that limit."""
    g, _ = make_pair(0, 4, episode_len=episode_len, small_variant=3)
    n, T = [4] * 300 + [3] * 40 + [2] * 17, 29
    E = len(n)
    a = rl.Env(g, E, n, 31)
    a.rollout(5)
    b = rl.Env(g, E, n, 31)
    b.set_state(a.get_state())
    bt = _alloc(a, T)
    a.rollout(T, **bt)
    for t in range(T):
        bs = _alloc(b)
        b.step(obs=bs["obs"], reward=bs["reward"], done=bs["done"])
        assert torch.equal(bs["obs"], bt["obs"][t]) and torch.equal(bs["reward"], bt["reward"][t])
        assert torch.equal(bs["done"], bt["done"][t])
    assert int(bt["done"].sum()) > 0
    assert a.get_state() == b.get_state()
    a.close()
    b.close()


def test_uneven_classes_in_one_batch(rl):
    """Envs of 2..32 robots (every size class, ragged class sizes) in one handle."""
    n = [2, 3, 4, 5, 7, 8, 9, 12, 16, 17, 25, 32] * 5
    g, o = make_pair(0, 32)
    err, _ = _teacher_forced(rl, g, o, n, 4, 12)
    print(f"\nuneven classes: {err}")
    assert err["u_star"] < U_TOL and err["pose"] < 1e-6


def test_checkpoint_resume_bit_identical(rl):
    g, _ = make_pair(1, 8)
    n = list(np.random.default_rng(1).integers(2, 9, 100))
    env = rl.Env(g, 100, n, 12)
    env.rollout(37)
    blob = env.get_state()
    b1 = _alloc(env, 50)
    env.rollout(50, **b1)
    s1 = env.get_state()
    env.set_state(blob)
    b2 = _alloc(env, 50)
    env.rollout(50, **b2)
    assert env.get_state() == s1
    assert torch.equal(b1["obs"], b2["obs"]) and torch.equal(b1["reward"], b2["reward"])
    env.close()


def test_rollout_host_matches_device(rl):
    g, _ = make_pair(0, 4)
    env = rl.Env(g, 64, 4, 21)
    blob = env.get_state()
    T = 30
    b = _alloc(env, T)
    env.rollout(T, **b)
    ho = np.zeros((T, env.total_robots, env.obs_dim), np.float32)
    hr = np.zeros((T, 64), np.float32)
    hd = np.zeros((T, 64), np.uint8)
    env.rollout_host(T, state=blob, obs=ho, reward=hr, done=hd)
    assert np.array_equal(ho, b["obs"].cpu().numpy())
    assert np.array_equal(hr, b["reward"].cpu().numpy())
    env.close()


def test_determinism_same_seed(rl):
    g, _ = make_pair(0, 20, near_frac=0.3)
    outs = []
    for _ in range(2):
        env = rl.Env(g, 50, 20, 123)
        b = _alloc(env, 20)
        env.rollout(20, **b)
        outs.append((b["obs"].cpu().numpy(), env.get_state()))
        env.close()
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


def test_argument_errors(rl):
    g, _ = make_pair(0, 4)
    env = rl.Env(g, 8, 4, 0)
    with pytest.raises(rl.RLError):
        env.step(actions=torch.zeros(32, 2, device="cuda"))  # scripted handle takes no actions
    with pytest.raises(rl.RLError):
        env.set_state(b"\0" * env.state_bytes())
    env.close()
    with pytest.raises(rl.RLError):
        rl.Env(dict(g, episode_len=0), 8, 4, 0)
    with pytest.raises(rl.RLError):
        rl.Env(g, 8, 33, 0)


@pytest.mark.parametrize("n_robots", [4, 10])
def test_nonfinite_action_zeroed_and_reported(rl, n_robots):
    """A NaN or infinite policy action is taken as zero for that robot (the step is the same as
    with a zero action) and the next synchronising call reports it once as RL_ERR_ARG."""
    g, _ = make_pair(0, n_robots, scripted=0)
    E = 8
    bad = rl.Env(g, E, n_robots, 5)
    ref = rl.Env(g, E, n_robots, 5)
    gen = torch.Generator().manual_seed(2)
    act = ((torch.rand(E * n_robots, 2, generator=gen) - 0.5) * 0.3).cuda()
    a_bad, a_ref = act.clone(), act.clone()
    a_bad[3, 0] = float("nan")
    a_bad[n_robots + 1, 1] = float("inf")
    a_ref[3] = 0.0
    a_ref[n_robots + 1] = 0.0
    ob, orf = _alloc(bad), _alloc(ref)
    bad.step(actions=a_bad, **ob)
    ref.step(actions=a_ref, **orf)
    with pytest.raises(rl.RLError) as ei:
        bad.sync()
    assert ei.value.status == 1 and "non-finite" in str(ei.value)
    ref.sync()
    bad.sync()  # reported once, then cleared
    assert torch.equal(ob["obs"], orf["obs"]) and torch.equal(ob["reward"], orf["reward"])
    assert torch.isfinite(ob["obs"]).all()
    bad.step(actions=a_bad, **ob)
    with pytest.raises(rl.RLError):
        bad.counters()
    bad.sync()
    bad.close()
    ref.close()


@pytest.mark.parametrize("scenario", [0, 1, 2])
def test_uneven_one_launch_matches_steps(rl, scenario):
    """Uneven robot counts (2..10, every class up to 16 robots) in one persistent launch match
    one step at a time through the per-class launches: done flags and integer state exactly,
    values to rounding (the same device code compiled into two kernels may contract multiply-
    adds differently)."""
    from synth_inputs import uneven_robot_counts
    n = uneven_robot_counts(8, 333, 2, 10)
    g, _ = make_pair(scenario, 10, episode_len=25)
    T = 40
    a = rl.Env(g, 333, n, 31)
    bt = _alloc(a, T)
    a.rollout(T, **bt)
    b = rl.Env(g, 333, n, 31)
    worst = 0.0
    for t in range(T):
        bs = _alloc(b)
        b.step(obs=bs["obs"], reward=bs["reward"], done=bs["done"])
        worst = max(worst, (bs["obs"] - bt["obs"][t]).abs().max().item(),
                    (bs["reward"] - bt["reward"][t]).abs().max().item())
        assert torch.equal(bs["done"], bt["done"][t]), f"done differs at step {t}"
    sa, sb = a.state_arrays(), b.state_arrays()
    print(f"\none launch vs steps, scenario {scenario}: max |diff| {worst:.3e}")
    for k in ("t", "ep", "level", "qactive", "counters"):
        assert np.array_equal(sa[k], sb[k]), k
    assert worst < 1e-5
    a.close()
    b.close()


def test_uneven_parallel_classes_equal_sequential(rl):
    """One launch per class on parallel streams gives the same trajectories and state as one
    launch per class in sequence, bit for bit (the same kernels on the same data)."""
    from synth_inputs import uneven_robot_counts
    n = uneven_robot_counts(9, 700, 2, 10)
    g, _ = make_pair(1, 10, episode_len=30)
    T = 45
    outs = []
    for mode in (0, 2):
        env = rl.Env(g, 700, n, 13)
        env.set_class_launch(mode)
        b = _alloc(env, T)
        env.rollout(T, **b)
        env.rollout(T, **b)  # the cached graph replayed
        torch.cuda.synchronize()
        outs.append((b, env.get_state()))
        env.close()
    (b0, s0), (b2, s2) = outs
    assert torch.equal(b0["obs"], b2["obs"]) and torch.equal(b0["reward"], b2["reward"])
    assert torch.equal(b0["done"], b2["done"]) and s0 == s2


def test_tuner_keeps_state_and_results(rl):
    n = [2, 3, 4, 6, 8, 12, 16, 20] * 16
    g, _ = make_pair(0, 20)
    env = rl.Env(g, len(n), n, 5)
    ref = rl.Env(g, len(n), n, 5)
    before = env.get_state()
    choice = env.tune(10)
    print(f"\ntuner choice: {choice}")
    assert env.get_state() == before
    assert len(choice["classes"]) == 4
    T = 30
    b1, b2 = _alloc(env, T), _alloc(ref, T)
    env.rollout(T, **b1)
    ref.rollout(T, **b2)
    assert torch.equal(b1["done"], b2["done"])
    assert (b1["obs"] - b2["obs"]).abs().max().item() < 1e-4
    env.close()
    ref.close()
