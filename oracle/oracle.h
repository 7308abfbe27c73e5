/*
 * oracle.h -- FP64 CPU oracle of the batched multi-robot environment step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load this library.  It shares no code, header, table or constant with the CUDA
 * library under paper_2505_06771_gb300/; the two agree only through the written definition of
 * the method (JaxRobotarium, arXiv 2505.06771: Sec. 4.1 "Design" for the unicycle simulator,
 * the single-integrator controller and the barrier-certificate QP; Sec. 6.1 for the
 * ControllerManager ordering; App. B for the Navigation and Foraging scenarios).
 *
 * Everything here is plain double precision, except the reset sampler and the action-noise
 * draw, which the method specifies in binary32 so that both implementations draw identical
 * initial states and noise (see oracle.c).
 */
#ifndef ROBO_ORACLE_H
#define ROBO_ORACLE_H
#include <stdint.h>

#define ORC_NMAX 32   /* robots per environment */
#define ORC_RMAX 16   /* foraging resources per environment */
#define ORC_NCOUNT 8  /* int32 counters per environment */

enum { ORC_NAV = 0, ORC_FORAGE = 1, ORC_DISCOVERY = 2 };
enum { ORC_CTRL_POSITION = 0, ORC_CTRL_POSE = 1 };
enum { ORC_CNT_COLLISIONS = 0, ORC_CNT_OOB = 1, ORC_CNT_SUCCESS = 2, ORC_CNT_QP_ACTIVE = 3,
       ORC_CNT_QP_FLAGGED = 4, ORC_CNT_QP_INFEASIBLE = 5, ORC_CNT_EPISODES = 6,
       ORC_CNT_QP_ITERS = 7 };

typedef struct {
    int32_t scenario;      /* ORC_NAV or ORC_FORAGE */
    int32_t scripted;      /* 1: scripted go-to-target nominal control + noise; 0: policy actions */
    int32_t episode_len;   /* steps per episode (App. B: max steps 100) */
    int32_t n_res_min, n_res_max;   /* foraging resources per episode */
    int32_t max_attempts;  /* rejection-sampling attempts per robot */
    int32_t n_max, r_max;  /* observation padding (robots, resources) */
    int32_t controller;    /* Navigation scripted control: ORC_CTRL_POSITION or ORC_CTRL_POSE */
    double gamma, r, l, vmax, wmax, dt, kappa, k_si, noise_amp, c_col, forage_radius;
    double xmin, xmax, ymin, ymax, init_margin, min_sep;
    double near_frac, near_dmin, near_dmax;
    double goal_eps;       /* Navigation: > 0 assigns a new goal on arrival (Random Waypoint
                              Navigation, Sec. 4.2); 0 keeps the goals for the episode */
    double pose_k1, pose_k2, pose_k3;  /* pose controller gains (approach, heading, final
                                          orientation weight), all > 0 */
    double sense_radius, tag_radius;   /* Discovery: capability radii (App. B: 0.45, 0.25) */
    double sense_reward, tag_reward, step_penalty;  /* Discovery rewards (App. B: 1, 5, 0.05) */
} orc_cfg;

/* Batched structure-of-arrays state.  Robots of env e occupy [off_e, off_e + n_e). */
typedef struct {
    double *x, *y, *th, *gx, *gy;     /* [sum n] */
    double *gth;                      /* [sum n] goal heading (pose controller) */
    int32_t *level;                   /* [sum n] foraging level */
    int32_t *t, *ep, *n_res;          /* [E] */
    double *qx, *qy;                  /* [E * r_max] */
    int32_t *qlevel, *qactive;        /* [E * r_max] */
    int32_t *counters;                /* [E * ORC_NCOUNT] */
} orc_batch;

/* Optional per-step trace (any pointer may be NULL). */
typedef struct {
    double *u_nom;    /* [sum n * 2] nominal SI velocity after the speed cap */
    double *u_star;   /* [sum n * 2] QP minimiser */
    double *vw;       /* [sum n * 2] unicycle (v, omega) after the wheel clip */
    int32_t *qp;      /* [E * 4]: status, active rows, iterations, any-active flag */
    double *kkt;      /* [E] max KKT residual of the QP */
} orc_trace;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

int orc_obs_dim(const orc_cfg* c);

/* Sample the initial state of each env for episode ep[e] (ep may be NULL: episode 0). */
int orc_reset_batch(const orc_cfg* c, uint64_t seed, int E, const int32_t* n_robots,
                    const int32_t* ep, orc_batch* b);

/* One step of every env.  actions: [sum n * 2] or NULL (scripted).  obs: [sum n * obs_dim]. */
int orc_step_batch(const orc_cfg* c, uint64_t seed, int E, const int32_t* n_robots, orc_batch* b,
                   const double* actions, double* obs, double* reward, uint8_t* done,
                   orc_trace* tr, int n_threads);

/* T steps of every env in scripted mode; trajectory buffers may be NULL. */
int orc_rollout(const orc_cfg* c, uint64_t seed, int E, const int32_t* n_robots, orc_batch* b,
                int T, double* obs_traj, double* rew_traj, uint8_t* done_traj, int n_threads);

/* min 1/2 |u - u0|^2  s.t.  A u <= b  (A: m x n row-major).  Returns 0 ok, 1 infeasible,
   2 iteration cap.  lam[m] gets the multipliers (0 off the active set). */
int orc_qp_project(int n, int m, const double* A, const double* bvec, const double* u0,
                   double* u, double* lam, int32_t* n_active, int32_t* iters);

/* Barrier-certificate QP rows of one env from its projected points: m = N(N-1)/2 + 4N rows. */
int orc_build_cbf_rows(const orc_cfg* c, int N, const double* px, const double* py,
                       double* A, double* bvec);

/* Unicycle pose controller (posture regulation in polar coordinates, Aicardi et al. 1995):
   the nominal (v, omega) driving pose [x, y, th] to goal [gx, gy, gth]. */
void orc_pose_control(const orc_cfg* c, const double* pose, const double* goal, double* vw);

/* Single-integrator velocity -> unicycle command -> wheel clip -> Euler step, one robot.
   pose: in/out [x, y, th]; vw: out [v, omega] after the clip. */
void orc_unicycle_update(const orc_cfg* c, double ux, double uy, double* pose, double* vw);

#endif
