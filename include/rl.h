/*
 * rl.h -- C ABI of the GB300 (sm_103a) batched multi-robot environment step.
 *
 * The method: JaxRobotarium (arXiv 2505.06771).  Each step of each environment
 *   - forms the projected points p_i = (x_i + l cos th_i, y_i + l sin th_i) that the
 *     single-integrator (SI) layer drives (Sec. 4.1: "single integrator and unicycle
 *     controllers");
 *   - takes a nominal SI velocity per robot: the policy's action, or the scripted go-to-target
 *     law (Sec. 6.1 ControllerManager: waypoint -> controller) with uniform action noise
 *     (Sec. 7, domain randomisation), capped to v_max;
 *   - filters it through the barrier-certificate QP (Sec. 4.1: "control barrier certificates
 *     ... solve the quadratic program"), min |u - u_nom|^2 subject to
 *     -2 (p_i - p_j).(u_i - u_j) <= gamma h_ij^3, h_ij = |p_i - p_j|^2 - r^2, for every pair, and
 *     four arena rows per robot, +-u_{x,y} <= kappa gamma (distance to the wall - r/2)^3;
 *   - maps SI to unicycle velocities, clips the wheel speeds (Sec. 1: GRITSBot "dynamic
 *     constraints"), integrates the unicycle model (Sec. 4.1) with explicit Euler;
 *   - computes collision / boundary flags, the team reward, the scenario transition, done and
 *     auto-reset, and the per-robot observations (App. B: Navigation, Foraging).
 * The calls follow the Dec-POMDP reading of the Scenario interface (Sec. 6.1): per-agent
 * observations, one shared team reward per environment, one done flag per environment.
 *
 * Conventions.
 *   Ownership: every d_* pointer is device memory owned by the caller; host pointers are named
 *   h_*.  Environment state lives in device memory owned by the handle.
 *   Precision: a handle computes in binary32 (RL_PREC_F32) or binary64 (RL_PREC_F64); every
 *   real-valued buffer of a call (actions, observations, rewards, traces) has that type.
 *   Layout: the robots of env e occupy rows [off_e, off_e + n_e) of every per-robot buffer,
 *   off_e = n_0 + ... + n_{e-1}; per-robot observations are rows of obs_dim values; per-env
 *   buffers have one entry per env.  Trajectories are [T][rows...] with step t outermost.
 *   Streams: calls are enqueued on the handle's stream and return before the GPU finishes.
 *   Errors: argument errors are returned at once; CUDA errors are returned by the call that
 *   sees them; rl_last_error() holds a one-line message.  Nothing aborts and no C++ exception
 *   crosses this boundary.
 */
#ifndef ROBO_GB300_RL_H
#define ROBO_GB300_RL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rl_env rl_env;

typedef enum {
    RL_OK = 0,
    RL_ERR_ARG = 1,      /* invalid argument (size, pointer, configuration) */
    RL_ERR_CUDA = 2,     /* a CUDA runtime call failed */
    RL_ERR_OOM = 3,      /* device allocation failed */
    RL_ERR_STATE = 4,    /* call not valid in the handle's state */
    RL_ERR_TIMEOUT = 5,  /* a bounded device wait ran out */
    RL_ERR_BUDGET = 6    /* a request can never fit the memory budget */
} rl_status;

typedef enum { RL_SCEN_NAVIGATION = 0, RL_SCEN_FORAGING = 1, RL_SCEN_DISCOVERY = 2 } rl_scenario;
typedef enum { RL_CTRL_POSITION = 0, RL_CTRL_POSE = 1 } rl_controller;

typedef enum { RL_PREC_F32 = 32, RL_PREC_F64 = 64 } rl_precision;

/* Counters per env (int32, cumulative since rl_create / rl_reset). */
enum {
    RL_CNT_COLLISIONS = 0,   /* colliding pairs summed over steps: |p_i - p_j|^2 < r^2 */
    RL_CNT_OOB = 1,          /* robots whose projected point left the arena, summed over steps */
    RL_CNT_SUCCESS = 2,      /* foraged resources; Navigation with goal_eps > 0: arrivals */
    RL_CNT_QP_ACTIVE = 3,    /* steps whose QP had at least one active row */
    RL_CNT_QP_FLAGGED = 4,   /* steps whose binary32 QP was flagged and re-solved in binary64 */
    RL_CNT_QP_INFEASIBLE = 5,/* steps whose QP was infeasible (the env's robots then stop) */
    RL_CNT_EPISODES = 6,     /* completed episodes */
    RL_CNT_QP_ITERS = 7,     /* active-set iterations summed over steps */
    RL_NCOUNT = 8
};

/* Configuration.  rl_config_default() fills the constants of the paper's setting. */
typedef struct {
    int32_t scenario;       /* rl_scenario */
    int32_t precision;      /* rl_precision */
    int32_t scripted;       /* 1: scripted nominal control; 0: rl_step takes policy actions */
    int32_t episode_len;    /* steps per episode (App. B: 100) */
    int32_t n_res_min;      /* foraging: resources per episode, uniform in [min, max] */
    int32_t n_res_max;
    int32_t r_max;          /* foraging: resource slots in the observation (>= n_res_max) */
    int32_t n_max;          /* robot slots in the observation (0: the largest n_e) */
    int32_t max_attempts;   /* rejection-sampling attempts per robot at reset */
    int32_t qp_max_iter;    /* active-set iteration cap (0: 8 * n_max + 16) */
    int32_t resolve_f64;    /* 1: re-solve flagged binary32 QPs in binary64 */
    int32_t lanes;          /* lanes per environment (0: the class default or rl_tune's pick) */
    int32_t block_threads;  /* threads per block, a multiple of 32 up to 256 (0: default) */
    int32_t warp_envs;      /* 4-robot binary32 class: envs per 32-lane warp (0: default: for
                               scripted Navigation the envs are spread evenly over one block of 4
                               warps per SM when that leaves at most 8 per warp, else 6 per warp
                               for the shuffle kernel and 4 otherwise) */
    int32_t small_variant;  /* 4-robot binary32 Navigation, scripted, without traces: 1 the team
                               kernel that reduces across lanes with shuffles (faster on large
                               batches), 2 the team kernel that publishes each robot's state in
                               shared memory (lower latency per step), 3 the shuffle team kernel
                               with the flags, reward and observations in a second warp per
                               dynamics warp (position controller, spread launch); 0 picks by
                               batch size */
    int32_t controller;     /* Navigation scripted nominal control: RL_CTRL_POSITION (go to the
                               goal point, k_si) or RL_CTRL_POSE (unicycle posture regulation to
                               the goal pose: position and goal heading, pose_k1..3) */
    double gamma;           /* barrier gain (100) */
    double r;               /* safety radius [m] (0.17) */
    double l;               /* projection distance [m] (0.05) */
    double vmax;            /* speed cap and wheel-speed limit [m/s] (0.2) */
    double wmax;            /* turn-rate limit [rad/s] (3.6) */
    double dt;              /* step [s] (0.033) */
    double kappa;           /* arena-row gain factor (0.4) */
    double k_si;            /* SI go-to-target gain (1.0) */
    double noise_amp;       /* action noise U(-a, a) per component (0.05) */
    double c_col;           /* collision penalty (1 Navigation, 0 Foraging) */
    double forage_radius;   /* [m] (0.25) */
    double xmin, xmax, ymin, ymax;   /* arena [m] (3.2 x 2.0 centred) */
    double init_margin;     /* reset: distance of sampled points from the walls [m] (0.2) */
    double min_sep;         /* reset: pairwise separation of robot centres [m] (0.3) */
    double near_frac;       /* reset: share of envs with one near pair (0) */
    double near_dmin, near_dmax;     /* reset: distance of the near pair [m] (0.18, 0.20) */
    double h_flag;          /* also re-solve in binary64 a binary32 QP with an active pair whose
                               h < h_flag (m^2); default -1: never (h >= -r^2) */
    double goal_eps;        /* Navigation: > 0 gives a robot a new goal when its projected point
                               ends a step within goal_eps of its goal (Random Waypoint
                               Navigation, Sec. 4.2); 0 (default) keeps goals for the episode */
    double pose_k1, pose_k2, pose_k3;  /* pose controller gains: approach, heading, final
                                          orientation weight (1, 2, 1), all > 0 */
    double sense_radius, tag_radius;   /* Discovery capabilities (App. B: 0.45 m, 0.25 m) */
    double sense_reward, tag_reward, step_penalty;  /* Discovery rewards (App. B: 1, 5, 0.05) */
} rl_config;

/* Optional outputs of one step (any pointer may be NULL). */
typedef struct {
    const void* d_actions;  /* [rows][2] policy SI velocities; NULL in scripted mode */
    void* d_obs;            /* [rows][obs_dim] observations after the step (after auto-reset) */
    void* d_reward;         /* [E] team reward of the transition */
    uint8_t* d_done;        /* [E] 1 if the episode ended (the env was reset) */
    void* d_u_nom;          /* [rows][2] nominal SI velocity after the speed cap */
    void* d_u_star;         /* [rows][2] QP minimiser (filtered SI velocity) */
    void* d_vw;             /* [rows][2] unicycle (v, omega) after the wheel clip */
    int32_t* d_qp_info;     /* [E][4] status (0 ok, 1 infeasible, 2 iteration cap), active rows,
                               iterations, flags (bit0 any active row, bit1 re-solved in FP64) */
} rl_step_io;

/* Fill *out with the defaults of a scenario.  RL_ERR_ARG on an unknown scenario. */
rl_status rl_config_default(int32_t scenario, rl_config* out);

/* Create a batch of n_envs environments and reset them (episode 0) with seed.
   Passage: Sec. 6.1 (RobotariumEnv holds a batch of robots; a Scenario defines their reset,
   step, reward and observation) and App. B (the scenarios' initial distributions).
   h_n_robots: host array [n_envs] of robot counts in [1, 32], or NULL to give every env
   n_robots_uniform robots.  stream: a cudaStream_t; NULL makes the handle create its own
   stream, which is ordered with the legacy default stream.
   The handle allocates and owns the device state.  RL_ERR_ARG on bad sizes or configuration,
   RL_ERR_OOM when the state does not fit. */
rl_status rl_create(const rl_config* cfg, int32_t n_envs, const int32_t* h_n_robots,
                    int32_t n_robots_uniform, uint64_t seed, void* stream, rl_env** out);

/* Reset every env to episode 0 under a new seed and zero the counters.
   Passage: Sec. 6.1 (Scenario reset: robots and goals drawn anew for each episode). */
rl_status rl_reset(rl_env* env, uint64_t seed);

/* One step of every env (Dec-POMDP step: joint action -> per-agent observations, team reward,
   done).  d_actions is required unless the handle is scripted; the others may be NULL.
   A non-finite action (NaN or infinity) is taken as zero for that robot and raises a bit in
   the handle's device status word, which the next rl_sync or rl_get_counters reports (once)
   as RL_ERR_ARG. */
rl_status rl_step(rl_env* env, const void* d_actions, void* d_obs, void* d_reward,
                  uint8_t* d_done);

/* rl_step with the optional traces of rl_step_io. */
rl_status rl_step_io_call(rl_env* env, const rl_step_io* io);

/* T scripted steps of every env in one persistent launch (replayed from a CUDA graph), the
   state kept on chip across steps.  Passage: Sec. 4.1 (the step jit-compiled and vmapped over
   environments, whole rollouts run on the accelerator); here that batching is one launch.  d_obs_traj [T][rows][obs_dim], d_rew_traj [T][E],
   d_done_traj [T][E]; any may be NULL.  RL_ERR_STATE if the handle is not scripted. */
rl_status rl_rollout(rl_env* env, int32_t T, void* d_obs_traj, void* d_rew_traj,
                     uint8_t* d_done_traj);

/* The same T steps in the plain form: one kernel launch per env per step, state through
   global memory.  Same results as rl_rollout; kept as the per-env baseline. */
rl_status rl_rollout_plain(rl_env* env, int32_t T, void* d_obs_traj, void* d_rew_traj,
                           uint8_t* d_done_traj);

/* Autotuner: times T_probe-step rollouts of the handle's own batch (from a saved copy of its
   state, restored afterwards) for every launch shape -- lanes per environment and threads per
   block for each robot-count class, and for an uneven batch one persistent launch over all
   classes against one launch per class -- and keeps the fastest for later rollouts.
   h_choice (NULL or 26 ints): [class launch mode (rl_set_class_launch), then per robot-count
   class (nmax, lanes, block threads, envs per warp, 4-robot kernel variant)].
   The probes write their trajectories to scratch memory the call allocates and frees.
   Synchronises the stream.  RL_ERR_STATE if the handle is not scripted. */
rl_status rl_tune(rl_env* env, int32_t T_probe, int32_t* h_choice);

/* Uneven binary32 batches (more than one robot-count class): how rl_rollout launches the
   classes.  mode 1: one persistent launch over every class (the default); 0: one launch per
   class, in sequence; 2: one launch per class, each on its own stream forked from and joined
   back to the handle's stream, so that the classes run at the same time (parallel branches of
   the rollout's CUDA graph).  rl_tune picks among the three.  Same results in every mode up to
   rounding.  RL_ERR_STATE for a batch with one class or a binary64 handle, RL_ERR_ARG for other
   modes. */
rl_status rl_set_class_launch(rl_env* env, int32_t mode);

/* End to end through host memory: upload h_state (rl_state_bytes() bytes, or NULL to keep the
   device state), run the T steps, and copy the trajectories to the host buffers (pinned memory
   recommended; any may be NULL).  The steps run in up to 16 chunks, one launch each; each
   chunk's slice of the observations is downloaded on a second stream while the next chunk
   runs (rewards and done flags once, after the last chunk).  Same results as rl_rollout.  Returns after the copies completed. */
rl_status rl_rollout_host(rl_env* env, const void* h_state, int32_t T, void* h_obs_traj,
                          void* h_rew_traj, uint8_t* h_done_traj);

/* Checkpoint: the full state (poses, goals, levels, step and episode counters, resources,
   counters) as a self-describing blob.  Copies complete before return. */
size_t    rl_state_bytes(const rl_env* env);
rl_status rl_get_state(rl_env* env, void* h_dst, size_t bytes);
rl_status rl_set_state(rl_env* env, const void* h_src, size_t bytes);

/* Counters [E][RL_NCOUNT] to host memory (synchronises the stream).  RL_ERR_ARG if the
   device status word was raised (non-finite action, see rl_step); the counters are copied
   all the same. */
rl_status rl_get_counters(rl_env* env, int32_t* h_dst);

/* Wait for the handle's stream; RL_ERR_CUDA if the device reported a CUDA error, RL_ERR_ARG
   if a non-finite action was seen since the last report (the word is then cleared). */
rl_status rl_sync(rl_env* env);

/* Allocation-free reset + rollout.  The paper has no counterpart: this is a service for callers
   that cannot allocate device memory -- code running while another component owns the device
   allocator (a caching allocator that must see every allocation, a framework enforcing a fixed
   memory budget), or code that must avoid the synchronisation a cudaMalloc/cudaFree can imply.
   It resets n_envs envs of n_robots robots each (episode 0, seed) and runs T scripted steps,
   with the same kernels and results as rl_create + rl_rollout on a fresh handle; the caller
   passes the trajectory buffers (layout of rl_rollout, any may be NULL) and a stream (NULL: the
   legacy default stream).  The environment state lives in one file-scope device array of
   RL_NOALLOC_MAX_BYTES (8 MiB) that every GPU loading the library holds until the process
   exits; rl_noalloc_state_bytes() gives a batch's need, and a batch that needs more returns
   RL_ERR_ARG before any GPU work.  Nothing is allocated: no cudaMalloc, cudaFree or allocating
   library call.  The first call on a device looks the array's device address up
   (cudaGetSymbolAddress) with that device current and caches it, so make that first call before
   any stream capture.  Every call reuses the same array and overwrites what it reads (the
   previous call's contents never leak into a result), so calls that overlap on the GPU --
   concurrent streams, other threads, or a capture replayed while another call runs -- race.
   Returns after enqueueing; RL_ERR_CUDA if a launch failed. */
#define RL_NOALLOC_MAX_BYTES ((size_t)8 << 20)
rl_status rl_rollout_noalloc(const rl_config* cfg, int32_t n_envs, int32_t n_robots,
                             uint64_t seed, int32_t T, void* d_obs_traj, void* d_rew_traj,
                             uint8_t* d_done_traj, void* stream);
size_t    rl_noalloc_state_bytes(const rl_config* cfg, int32_t n_envs, int32_t n_robots);

/* ---- Serving: continuous batching of rollout requests ------------------------------------
   A server runs scripted rollout requests (n_envs environments of n_robots robots, horizon
   steps, seed) with the configuration given at creation.  An engine thread admits queued
   requests in arrival order whenever one of max_slots slots is free and the device bytes the
   request holds fit in what the budget has left; each admitted request runs as one persistent
   rollout launch on its slot's stream, so requests admitted at different times run on the GPU
   at the same time.  Its environment state stays on the device for the whole horizon; only the
   per-env returns and counters come back.  A request's result is the same alone or in any mix
   (the same kernels on the same data).  Latency = finish - submit on the host steady clock. */
typedef struct rl_server rl_server;
typedef struct {
    int32_t n_envs;     /* >= 1 */
    int32_t n_robots;   /* 1..32 (and <= the config's n_max when that is set) */
    int32_t horizon;    /* steps, >= 0 */
    uint64_t seed;
} rl_request;
typedef struct {
    uint64_t id;
    int32_t status;     /* 0 queued, 1 running, 2 done, 3 failed */
    int32_t n_envs, n_robots, horizon;
    double submit_s, start_s, finish_s;   /* seconds since the server was created */
    double mean_return;                   /* mean over envs of the summed team reward */
    int32_t counters[RL_NCOUNT];          /* summed over the request's envs */
} rl_result;

/* hbm_budget_bytes: device bytes all running requests may hold together.  The server uses the
   current device. */
rl_status rl_server_create(const rl_config* cfg, size_t hbm_budget_bytes, int32_t max_slots,
                           rl_server** out);
/* Queue a request; *id identifies it.  RL_ERR_BUDGET if it can never fit the budget,
   RL_ERR_ARG on bad sizes.  Thread-safe; returns at once. */
rl_status rl_server_submit(rl_server* srv, const rl_request* req, uint64_t* id);
/* Status of a request; h_returns (NULL or n_envs floats) gets the per-env returns once done.
   RL_ERR_ARG for an unknown id, RL_ERR_CUDA if the request failed. */
rl_status rl_server_result(rl_server* srv, uint64_t id, rl_result* out, float* h_returns);
/* out[6]: bytes in use, peak bytes in use, requests done, running, queued, env-steps done. */
rl_status rl_server_stats(rl_server* srv, int64_t* out);
/* Wait (host side, at most timeout_s seconds) until every submitted request has finished;
   RL_ERR_TIMEOUT if they have not. */
rl_status rl_server_drain(rl_server* srv, double timeout_s);
/* Stop the engine, wait for running requests, free everything.  NULL-safe. */
rl_status rl_server_destroy(rl_server* srv);

/* ---- Policy in the loop ------------------------------------------------------------------
   A recurrent policy evaluated on the GPU between steps, of the shape the paper trains (App. A:
   a one-layer MLP with ReLU, a GRU, a linear layer; widths 128-512):
       h1 = ReLU(W1 o + b1),  GRU(h1, h) -> h,  a = v_max tanh(Wo h + bo)
   with the GRU's gates r = sigma(Wi_r h1 + bi_r + Wh_r h + bh_r), z (likewise) and
   n = tanh(Wi_n h1 + bi_n + r * (Wh_n h + bh_n)), h <- (1 - z) n + z h.  The action a is the
   robot's SI velocity (rl_step's policy actions).  Each policy step is one kernel on the
   5th-generation tensor cores (tcgen05 MMA with the accumulators in tensor memory, operands
   staged by TMA), 128 robots per CTA, with the observation's conversion, the first layer's bias
   and ReLU, the gates, the new state and the head fused around the two products.  Operands of
   the products are bf16 (W1, b1, Wi, Wh and the inputs o, h1 and the previous h rounded to
   bf16, nearest-even), accumulation binary32; gates, state and the head are binary32, the
   gates' sigma and tanh from the hardware tanh approximation (relative error about 2^-11).  The
   recurrent state is per robot, reset to zero when its env's episode ends.  Binary32 handles
   with policy actions (scripted = 0) and observations of at most 16 values (up to 4 robots) only.
   A bounded wait inside the kernel that runs out raises the handle's status word (rl_sync then
   returns RL_ERR_TIMEOUT). */
typedef struct rl_policy rl_policy;

/* Passage: App. A (policy architecture).  hidden: H, a multiple of 64 up to 512.  Host arrays, row-major: h_w1 [H][obs_dim], h_b1 [H],
   h_wi [3H][H], h_bi [3H], h_wh [3H][H], h_bh [3H] (gate blocks in the order r, z, n),
   h_wo [2][H], h_bo [2].  Copies the weights to the device; the recurrent state starts at 0. */
rl_status rl_policy_create(rl_env* env, int32_t hidden, const float* h_w1, const float* h_b1,
                           const float* h_wi, const float* h_bi, const float* h_wh,
                           const float* h_bh, const float* h_wo, const float* h_bo,
                           rl_policy** out);
/* Zero the recurrent state of every robot. */
rl_status rl_policy_reset_hidden(rl_policy* pol);
/* T policy-driven steps of every env, captured once in a CUDA graph and replayed: observation
   -> policy -> action -> rl_step.  d_obs0 [rows][obs_dim]: the observation of the current state
   (rl_observe, or the last step's).  d_obs_traj [T][rows][obs_dim] and d_done_traj [T][E] are
   required (step t's observation and done flags feed step t + 1); d_rew_traj [T][E] and
   d_act_traj [T][rows][2] may be NULL. */
rl_status rl_policy_rollout(rl_env* env, rl_policy* pol, int32_t T, const void* d_obs0,
                            void* d_obs_traj, void* d_rew_traj, uint8_t* d_done_traj,
                            void* d_act_traj);
void      rl_policy_destroy(rl_policy* pol);   /* NULL-safe; waits for the handle's stream */

/* The observation of the current state without stepping ([rows][obs_dim], binary32 Navigation
   handles; RL_ERR_ARG otherwise). */
rl_status rl_observe(rl_env* env, void* d_obs);

int32_t     rl_obs_dim(const rl_env* env);      /* values per robot observation row */
int32_t     rl_n_envs(const rl_env* env);       /* environments E */
int32_t     rl_total_robots(const rl_env* env); /* robot rows, the sum of n_e */
int32_t     rl_lanes(const rl_env* env);        /* lanes per env the handle runs with */
const char* rl_last_error(const rl_env* env);   /* never NULL */
void        rl_destroy(rl_env* env);            /* NULL-safe; waits for the stream */

#ifdef __cplusplus
}
#endif
#endif
