// rl_api.cu -- the C ABI of include/rl.h: handles, device state, launches, CUDA-graph replay.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/rl.h"
#include "internal.h"
#include "launch.h"

namespace {

constexpr uint32_t kMagic = 0x31534C52u;  // "RLS1"
constexpr uint32_t kVersion = 2u;
constexpr int kSegs = 17;
constexpr int kHostChunks = 16;  // rl_rollout_host: chunks of the rollout, one launch each
enum Seg { S_X = 0, S_Y, S_TH, S_GX, S_GY, S_LEVEL, S_T, S_EP, S_NRES, S_QX, S_QY, S_QLEVEL,
           S_QACTIVE, S_COUNTERS, S_NROB, S_OFF, S_GTH };

struct StateHeader {
    uint32_t magic, version;
    int32_t precision, scenario, n_envs, total_robots, r_max, n_max;
    uint64_t seed, image_bytes;
    uint8_t pad[16];
};
static_assert(sizeof(StateHeader) == 64, "state header is 64 bytes");

struct Class {
    int nmax, lanes, begin, count, block_threads;
    int warp_envs;  // envs per warp for the 4-robot binary32 kernels (0: default)
    int variant;    // 4-robot binary32 Navigation fast path (0: by batch size)
};

}  // namespace

struct rl_env {
    rl_config cfg;
    int E = 0, total = 0, n_max = 0, r_max = 0, obs_dim = 0, prec = 32, esz = 4;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    uint64_t seed = 0;
    unsigned char* d_img = nullptr;
    size_t img_bytes = 0;
    size_t seg_off[kSegs] = {};
    size_t seg_len[kSegs] = {};
    int32_t* d_lists = nullptr;
    std::vector<int32_t> h_nrob, h_off;
    Class cls[rl::kNumClasses];
    int ncls = 0;
    std::string err;
    // rollout graph cache
    cudaGraphExec_t gexec = nullptr;
    int g_T = -1;
    void *g_obs = nullptr, *g_rew = nullptr;
    uint8_t* g_done = nullptr;
    // device scratch of rl_rollout_host, its copy stream and chunk events
    void* d_scratch = nullptr;
    size_t scratch_bytes = 0;
    cudaStream_t copy_st = nullptr;
    cudaEvent_t chunk_ev[kHostChunks] = {};
    // uneven batches: 1 one persistent launch over all classes (binary32), 0 one launch per class
    // in sequence, 2 one launch per class on parallel streams (parallel branches of the graph)
    int use_multi = 0;
    cudaStream_t side[rl::kNumClasses] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[rl::kNumClasses] = {};
    int n_items = 0;
    int4* d_items = nullptr;
    unsigned* d_head = nullptr;
    unsigned class_mask = 0;
    // device status word (rl::kStatusNonFiniteAction ...), read by the synchronising calls
    int32_t* d_status = nullptr;
};

namespace rl {
cudaStream_t env_stream(const rl_env* h) { return h->st; }
const std::vector<int32_t>& env_offsets(const rl_env* h) { return h->h_off; }
const rl_config& env_config(const rl_env* h) { return h->cfg; }
void env_set_error(rl_env* h, const std::string& msg) { h->err = msg; }

bool valid_config(const rl_config& c, std::string& why) {
    if (c.scenario != RL_SCEN_NAVIGATION && c.scenario != RL_SCEN_FORAGING &&
        c.scenario != RL_SCEN_DISCOVERY) { why = "scenario"; return false; }
    if (c.precision != RL_PREC_F32 && c.precision != RL_PREC_F64) { why = "precision"; return false; }
    if (c.episode_len < 1) { why = "episode_len"; return false; }
    if (c.max_attempts < 1) { why = "max_attempts"; return false; }
    if (!(c.l > 0) || !(c.vmax > 0) || !(c.wmax > 0) || !(c.dt > 0) || !(c.r >= 0)) { why = "constants"; return false; }
    if (!(c.xmax > c.xmin) || !(c.ymax > c.ymin)) { why = "arena"; return false; }
    if (c.scenario != RL_SCEN_NAVIGATION) {
        if (c.r_max < 1 || c.r_max > kMaxRes) { why = "r_max"; return false; }
        if (c.n_res_min < 0 || c.n_res_max > c.r_max || c.n_res_min > c.n_res_max) { why = "n_res"; return false; }
    }
    if (c.n_max < 0 || c.n_max > kMaxRobots) { why = "n_max"; return false; }
    if (c.block_threads < 0 || c.block_threads % 32 != 0 || c.block_threads > 256) {
        why = "block_threads";
        return false;
    }
    if (c.lanes < 0 || c.warp_envs < 0) { why = "lanes / warp_envs"; return false; }
    if (!(c.goal_eps >= 0.0) || (c.goal_eps > 0.0 && c.scenario != RL_SCEN_NAVIGATION)) {
        why = "goal_eps";
        return false;
    }
    if ((c.controller != RL_CTRL_POSITION && c.controller != RL_CTRL_POSE) ||
        (c.controller == RL_CTRL_POSE &&
         (c.scenario != RL_SCEN_NAVIGATION || !(c.pose_k1 > 0) || !(c.pose_k2 > 0) ||
          !(c.pose_k3 > 0)))) {
        why = "controller";
        return false;
    }
    return true;
}
}  // namespace rl

namespace {
template <typename R>
void fill_args(const rl_env* h, rl::LaunchArgs<R>& a);
}  // namespace

namespace rl {
bool env_args_f32(const rl_env* h, LaunchArgs<float>& a) {
    if (h->prec != 32) return false;
    fill_args<float>(h, a);
    return true;
}
}  // namespace rl

namespace {

rl_status fail(rl_env* h, rl_status s, const std::string& msg) {
    if (h) h->err = msg;
    return s;
}

rl_status cuda_fail(rl_env* h, cudaError_t e, const char* where) {
    return fail(h, RL_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <typename R>
void fill_args(const rl_env* h, rl::LaunchArgs<R>& a) {
    const rl_config& c = h->cfg;
    auto seg = [&](int s) { return (void*)(h->d_img + h->seg_off[s]); };
    a.s.x = (R*)seg(S_X); a.s.y = (R*)seg(S_Y); a.s.th = (R*)seg(S_TH);
    a.s.gx = (R*)seg(S_GX); a.s.gy = (R*)seg(S_GY); a.s.gth = (R*)seg(S_GTH);
    a.s.level = (int32_t*)seg(S_LEVEL);
    a.s.t = (int32_t*)seg(S_T); a.s.ep = (int32_t*)seg(S_EP); a.s.n_res = (int32_t*)seg(S_NRES);
    a.s.qx = (R*)seg(S_QX); a.s.qy = (R*)seg(S_QY);
    a.s.qlevel = (int32_t*)seg(S_QLEVEL); a.s.qactive = (int32_t*)seg(S_QACTIVE);
    a.s.counters = (int32_t*)seg(S_COUNTERS);
    a.s.off = (const int32_t*)seg(S_OFF);
    a.s.nrob = (const int32_t*)seg(S_NROB);
    std::memset(&a.io, 0, sizeof(a.io));
    a.io.status = h->d_status;
    a.io.E = h->E;
    a.io.obs_dim = h->obs_dim;
    a.io.obs_step = (long long)h->total * h->obs_dim;
    rl::StepConsts<R>& k = a.k;
    const double track = 2.0 * c.vmax / c.wmax;
    k.gamma = (R)c.gamma; k.r2 = (R)(c.r * c.r); k.l = (R)c.l; k.inv_l = (R)(1.0 / c.l);
    k.vmax = (R)c.vmax; k.half_track = (R)(0.5 * track); k.inv_track = (R)(1.0 / track);
    k.dt = (R)c.dt; k.kg = (R)(c.kappa * c.gamma); k.half_r = (R)(0.5 * c.r); k.k_si = (R)c.k_si;
    k.c_col = (R)c.c_col; k.rho2 = (R)(c.forage_radius * c.forage_radius);
    k.xmin = (R)c.xmin; k.xmax = (R)c.xmax; k.ymin = (R)c.ymin; k.ymax = (R)c.ymax;
    k.h_flag = (R)c.h_flag;
    k.goal_eps2 = (R)(c.goal_eps * c.goal_eps);
    k.waypoint = (c.scenario == RL_SCEN_NAVIGATION && c.goal_eps > 0.0) ? 1 : 0;
    k.controller = c.controller;
    k.pk1 = (R)c.pose_k1; k.pk2 = (R)c.pose_k2; k.pk3 = (R)c.pose_k3;
    k.sense_r = (R)c.sense_radius; k.tag_r = (R)c.tag_radius;
    k.sense_r2 = (R)(c.sense_radius * c.sense_radius); k.tag_r2 = (R)(c.tag_radius * c.tag_radius);
    k.sense_rew = (R)c.sense_reward; k.tag_rew = (R)c.tag_reward; k.step_pen = (R)c.step_penalty;
    k.xo = (R)(c.xmax + (c.xmax - c.xmin)); k.yo = (R)(c.ymax + (c.ymax - c.ymin));
    k.scenario = c.scenario; k.scripted = c.scripted; k.episode_len = c.episode_len;
    k.max_iter = c.qp_max_iter > 0 ? c.qp_max_iter : 8 * h->n_max + 16;
    k.n_res_min = c.n_res_min; k.n_res_max = c.n_res_max; k.r_max = h->r_max;
    k.n_max_obs = h->n_max; k.max_attempts = c.max_attempts; k.resolve_f64 = c.resolve_f64;
    k.noise_on = c.noise_amp > 0.0 ? 1 : 0;
    k.noise_scale = 2.0f * (float)c.noise_amp;
    rl::SamplerConsts& s = a.sc;
    s.lox = (float)c.xmin + (float)c.init_margin;
    s.hix = (float)c.xmax - (float)c.init_margin;
    s.loy = (float)c.ymin + (float)c.init_margin;
    s.hiy = (float)c.ymax - (float)c.init_margin;
    s.wx = s.hix - s.lox;
    s.wy = s.hiy - s.loy;
    s.sep2 = (float)c.min_sep * (float)c.min_sep;
    s.pif = (float)M_PI;
    s.twopif = (float)(2.0 * M_PI);
    s.near_frac = (float)c.near_frac;
    s.dmin = (float)c.near_dmin;
    s.dspan = (float)c.near_dmax - (float)c.near_dmin;
    s.near_on = c.near_frac > 0.0 ? 1 : 0;
    a.env_list = nullptr;
    a.n_list = 0;
    a.env_begin = 0;
    a.T = 1;
    a.seed = h->seed;
}

template <typename R>
cudaError_t launch_class(const rl_env* h, const Class& c, rl::LaunchArgs<R> a, bool reset,
                         int max_blocks = 0, cudaStream_t st = nullptr) {
    if (!st) st = h->st;
    a.env_list = h->d_lists + c.begin;
    a.n_list = c.count;
    a.warp_envs = c.warp_envs;
    a.variant = c.variant;
    if constexpr (std::is_same<R, double>::value) {
        return rl::launch_f64(a, c.nmax, c.lanes, c.block_threads, max_blocks, st, reset);
    } else {
        if (c.nmax == 4)
            return rl::launch_f32_small(a, c.lanes, c.block_threads, max_blocks, st, reset);
        return rl::launch_f32_large(a, c.nmax, c.lanes, c.block_threads, max_blocks, st, reset);
    }
}

// Side streams and events of the parallel per-class launch, made on first use.
cudaError_t ensure_side_streams(rl_env* h) {
    if (h->fork_ev) return cudaSuccess;
    cudaError_t e = cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming);
    for (int c = 0; c < rl::kNumClasses && e == cudaSuccess; ++c) {
        e = cudaStreamCreateWithFlags(&h->side[c], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join_ev[c], cudaEventDisableTiming);
    }
    return e;
}

// One launch per class, each on its own stream forked from and joined back to the handle's
// stream: the classes' kernels run at the same time (in a captured graph: parallel branches).
template <typename R>
rl_status run_parallel(rl_env* h, rl::LaunchArgs<R>& a, const char* what) {
    cudaError_t e = ensure_side_streams(h);
    if (e == cudaSuccess) e = cudaEventRecord(h->fork_ev, h->st);
    for (int i = 0; i < h->ncls && e == cudaSuccess; ++i) {
        e = cudaStreamWaitEvent(h->side[i], h->fork_ev, 0);
        if (e == cudaSuccess) e = launch_class<R>(h, h->cls[i], a, false, 0, h->side[i]);
        if (e == cudaSuccess) e = cudaEventRecord(h->join_ev[i], h->side[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->st, h->join_ev[i], 0);
    }
    return e == cudaSuccess ? RL_OK : cuda_fail(h, e, what);
}

template <typename R>
rl_status run_all(rl_env* h, rl::LaunchArgs<R>& a, bool reset, const char* what) {
    for (int i = 0; i < h->ncls; ++i) {
        cudaError_t e = launch_class<R>(h, h->cls[i], a, reset);
        if (e != cudaSuccess) return cuda_fail(h, e, what);
    }
    return RL_OK;
}

rl_status do_reset(rl_env* h) {
    if (h->prec == 64) {
        rl::LaunchArgs<double> a;
        fill_args(h, a);
        return run_all(h, a, true, "reset");
    }
    rl::LaunchArgs<float> a;
    fill_args(h, a);
    return run_all(h, a, true, "reset");
}

template <typename R>
rl_status do_step(rl_env* h, const rl_step_io* io) {
    rl::LaunchArgs<R> a;
    fill_args(h, a);
    a.T = 1;
    a.io.actions = (const R*)io->d_actions;
    a.io.obs = (R*)io->d_obs;
    a.io.reward = (R*)io->d_reward;
    a.io.done = io->d_done;
    a.io.u_nom = (R*)io->d_u_nom;
    a.io.u_star = (R*)io->d_u_star;
    a.io.vw = (R*)io->d_vw;
    a.io.qp_info = io->d_qp_info;
    return run_all(h, a, false, "step");
}

template <typename R>
rl_status do_rollout_launch(rl_env* h, int T, void* obs, void* rew, uint8_t* done) {
    rl::LaunchArgs<R> a;
    fill_args(h, a);
    a.T = T;
    a.io.obs = (R*)obs;
    a.io.reward = (R*)rew;
    a.io.done = done;
    if constexpr (std::is_same<R, float>::value) {
        if (h->use_multi == 1 && h->n_items > 0) {
            rl::MultiArgs m;
            std::memset(&m, 0, sizeof(m));
            m.a = a;
            m.a.env_list = h->d_lists;
            for (int i = 0; i < h->ncls; ++i) {
                m.cls[i].nmax = h->cls[i].nmax;
                m.cls[i].list_begin = h->cls[i].begin;
                m.cls[i].count = h->cls[i].count;
            }
            m.items = h->d_items;
            m.n_items = h->n_items;
            m.head = h->d_head;
            m.fast = h->cfg.scenario == RL_SCEN_NAVIGATION ? 1 : 0;
            cudaError_t e = rl::launch_multi(m, h->class_mask, 0, h->st);
            if (e != cudaSuccess) return cuda_fail(h, e, "rollout (one launch)");
            return RL_OK;
        }
    }
    if (h->use_multi == 2 && h->ncls > 1) return run_parallel<R>(h, a, "rollout (parallel classes)");
    return run_all(h, a, false, "rollout");
}

template <typename R>
rl_status do_rollout_returns(rl_env* h, int T, void* ret) {
    rl::LaunchArgs<R> a;
    fill_args(h, a);
    a.T = T;
    a.io.ret = (R*)ret;
    if constexpr (std::is_same<R, float>::value) {
        if (h->use_multi == 1 && h->n_items > 0) {
            rl::MultiArgs m;
            std::memset(&m, 0, sizeof(m));
            m.a = a;
            m.a.env_list = h->d_lists;
            for (int i = 0; i < h->ncls; ++i) {
                m.cls[i].nmax = h->cls[i].nmax;
                m.cls[i].list_begin = h->cls[i].begin;
                m.cls[i].count = h->cls[i].count;
            }
            m.items = h->d_items;
            m.n_items = h->n_items;
            m.head = h->d_head;
            m.fast = h->cfg.scenario == RL_SCEN_NAVIGATION ? 1 : 0;
            cudaError_t e = rl::launch_multi(m, h->class_mask, 0, h->st);
            return e == cudaSuccess ? RL_OK : cuda_fail(h, e, "serving rollout");
        }
    }
    if (h->use_multi == 2 && h->ncls > 1) return run_parallel<R>(h, a, "serving rollout");
    return run_all(h, a, false, "serving rollout");
}

rl_status rollout_enqueue(rl_env* h, int T, void* obs, void* rew, uint8_t* done) {
    return h->prec == 64 ? do_rollout_launch<double>(h, T, obs, rew, done)
                         : do_rollout_launch<float>(h, T, obs, rew, done);
}

// Wait for the stream, then report (once) what the kernels raised in the status word.
rl_status sync_and_take_status(rl_env* h, const char* what) {
    int32_t v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, h->d_status, sizeof(v), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, what);
    if (v == 0) return RL_OK;
    e = cudaMemsetAsync(h->d_status, 0, sizeof(v), h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, what);
    if (v & rl::kStatusWaitTimeout)
        return fail(h, RL_ERR_TIMEOUT, std::string(what) +
                                           ": a kernel's bounded wait ran out (its results are not valid)");
    if (v & rl::kStatusNonFiniteAction)
        return fail(h, RL_ERR_ARG, std::string(what) +
                                       ": a non-finite action reached the device (that robot's "
                                       "nominal velocity was taken as zero)");
    return fail(h, RL_ERR_STATE, std::string(what) + ": device status word set");
}

void drop_graph(rl_env* h) {
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    h->g_T = -1;
}

}  // namespace

extern "C" {

rl_status rl_config_default(int32_t scenario, rl_config* out) {
    if (!out) return RL_ERR_ARG;
    if (scenario != RL_SCEN_NAVIGATION && scenario != RL_SCEN_FORAGING &&
        scenario != RL_SCEN_DISCOVERY)
        return RL_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    out->scenario = scenario;
    out->precision = RL_PREC_F32;
    out->scripted = 1;
    out->episode_len = 100;
    out->n_res_min = 2;
    out->n_res_max = 6;
    out->r_max = scenario == RL_SCEN_NAVIGATION ? 0 : 6;
    out->n_max = 0;
    out->max_attempts = 4096;
    out->qp_max_iter = 0;
    out->resolve_f64 = 1;
    out->lanes = 0;
    out->block_threads = 0;
    out->warp_envs = 0;
    out->gamma = 100.0;
    out->r = 0.17;
    out->l = 0.05;
    out->vmax = 0.2;
    out->wmax = 3.6;
    out->dt = 0.033;
    out->kappa = 0.4;
    out->k_si = 1.0;
    out->noise_amp = 0.05;
    out->c_col = scenario == RL_SCEN_NAVIGATION ? 1.0 : 0.0;
    out->forage_radius = 0.25;
    out->xmin = -1.6;
    out->xmax = 1.6;
    out->ymin = -1.0;
    out->ymax = 1.0;
    out->init_margin = 0.2;
    out->min_sep = 0.3;
    out->near_frac = 0.0;
    out->near_dmin = 0.18;
    out->near_dmax = 0.20;
    // No small-h trigger by default (h >= -r^2 > -1): on 278 active QPs with h < 1e-3 m^2 met in
    // 16.4 M oracle env-steps, a binary32 solve was as close to the binary64 minimiser (6.9e-8)
    // as on the others (tests/test_binary32_small_h.py)
    out->h_flag = -1.0;
    out->goal_eps = 0.0;
    out->controller = RL_CTRL_POSITION;
    out->pose_k1 = 1.0;
    out->pose_k2 = 2.0;
    out->pose_k3 = 1.0;
    out->sense_radius = 0.45;
    out->tag_radius = 0.25;
    out->sense_reward = 1.0;
    out->tag_reward = 5.0;
    out->step_penalty = 0.05;
    return RL_OK;
}

rl_status rl_create(const rl_config* cfg, int32_t n_envs, const int32_t* h_n_robots,
                    int32_t n_robots_uniform, uint64_t seed, void* stream, rl_env** out) {
    if (!cfg || !out || n_envs < 1) return RL_ERR_ARG;
    *out = nullptr;
    std::string why;
    if (!rl::valid_config(*cfg, why)) return RL_ERR_ARG;
    rl_env* h = new (std::nothrow) rl_env();
    if (!h) return RL_ERR_OOM;
    h->cfg = *cfg;
    h->E = n_envs;
    h->prec = cfg->precision;
    h->esz = cfg->precision == 64 ? 8 : 4;
    h->seed = seed;
    h->h_nrob.resize(n_envs);
    h->h_off.resize(n_envs + 1);
    int nmax_seen = 0;
    h->h_off[0] = 0;
    for (int e = 0; e < n_envs; ++e) {
        const int n = h_n_robots ? h_n_robots[e] : n_robots_uniform;
        if (n < 1 || n > rl::kMaxRobots) { delete h; return RL_ERR_ARG; }
        h->h_nrob[e] = n;
        h->h_off[e + 1] = h->h_off[e] + n;
        nmax_seen = std::max(nmax_seen, n);
    }
    h->total = h->h_off[n_envs];
    h->n_max = cfg->n_max > 0 ? cfg->n_max : nmax_seen;
    if (h->n_max < nmax_seen) { delete h; return RL_ERR_ARG; }
    h->r_max = cfg->scenario != RL_SCEN_NAVIGATION ? cfg->r_max : 0;
    h->obs_dim = cfg->scenario == RL_SCEN_DISCOVERY ? 5 + 5 * (h->n_max - 1) + 4 * h->r_max
               : cfg->scenario == RL_SCEN_FORAGING ? 4 + 4 * (h->n_max - 1) + 4 * h->r_max
                                                   : 5 + 3 * (h->n_max - 1);
    // segments of the state image
    const size_t E = (size_t)n_envs, T = (size_t)h->total, RM = (size_t)h->r_max * E;
    const size_t lens[kSegs] = {T * h->esz, T * h->esz, T * h->esz, T * h->esz, T * h->esz,
                                T * 4, E * 4, E * 4, E * 4, RM * h->esz, RM * h->esz, RM * 4,
                                RM * 4, E * rl::kNCount * 4, E * 4, (E + 1) * 4, T * h->esz};
    size_t pos = 0;
    for (int s = 0; s < kSegs; ++s) {
        h->seg_off[s] = pos;
        h->seg_len[s] = lens[s];
        pos += (lens[s] + 255) & ~(size_t)255;
    }
    h->img_bytes = pos;
    if (stream) {
        h->st = (cudaStream_t)stream;
    } else {
        // a blocking stream: ordered with the legacy default stream, as the caller expects
        cudaError_t e = cudaStreamCreate(&h->st);
        if (e != cudaSuccess) { delete h; return RL_ERR_CUDA; }
        h->own_stream = true;
    }
    if (cudaMallocAsync((void**)&h->d_img, h->img_bytes, h->st) != cudaSuccess) {
        cudaGetLastError();
        rl_destroy(h);
        return RL_ERR_OOM;
    }
    // classes by robot count
    std::vector<int32_t> lists;
    for (int c = 0; c < rl::kNumClasses; ++c) {
        const int nm = rl::kClassNmax[c];
        const int lo = c == 0 ? 1 : rl::kClassNmax[c - 1] + 1;
        Class k;
        k.nmax = nm;
        k.begin = (int)lists.size();
        for (int e = 0; e < n_envs; ++e)
            if (h->h_nrob[e] >= lo && h->h_nrob[e] <= nm) lists.push_back(e);
        k.count = (int)lists.size() - k.begin;
        if (k.count == 0) continue;
        const unsigned ok = rl::supported_lanes(h->prec, nm);
        int lanes = cfg->lanes > 0 ? cfg->lanes : rl::kClassLanes[c];
        if (!(lanes > 0 && (ok & (unsigned)lanes))) lanes = rl::kClassLanes[c];
        k.lanes = lanes;
        k.block_threads = nm <= 16 ? 64 : 32;
        k.warp_envs = cfg->warp_envs > 0 ? std::min(32, cfg->warp_envs) : 0;
        k.variant = (cfg->small_variant >= 1 && cfg->small_variant <= 3) ? cfg->small_variant : 0;
        if (cfg->block_threads > 0) {
            if (cfg->block_threads % 32 != 0 || cfg->block_threads > 256) { rl_destroy(h); return RL_ERR_ARG; }
            k.block_threads = std::max(cfg->block_threads, lanes);
        }
        h->cls[h->ncls++] = k;
    }
    cudaError_t ce = cudaMallocAsync((void**)&h->d_lists, lists.size() * sizeof(int32_t), h->st);
    if (ce != cudaSuccess) { cudaGetLastError(); rl_destroy(h); return RL_ERR_OOM; }
    ce = cudaMallocAsync((void**)&h->d_status, 256, h->st);
    if (ce != cudaSuccess) { cudaGetLastError(); rl_destroy(h); return RL_ERR_OOM; }
    ce = cudaMemsetAsync(h->d_status, 0, 256, h->st);
    if (ce != cudaSuccess) { rl_destroy(h); return RL_ERR_CUDA; }
    // work items of the one-launch path, largest class first
    std::vector<int4> items;
    if (h->prec == 32 && h->ncls > 1) {
        for (int c = h->ncls - 1; c >= 0; --c) {
            int ci = 0;
            while (rl::kClassNmax[ci] != h->cls[c].nmax) ++ci;
            const int tpb = 64 / rl::kClassLanes[ci];
            for (int b = 0; b < h->cls[c].count; b += tpb)
                items.push_back(make_int4(c, b, std::min(tpb, h->cls[c].count - b), 0));
            h->class_mask |= 1u << ci;
        }
        ce = cudaMallocAsync((void**)&h->d_items, items.size() * sizeof(int4) + 256, h->st);
        if (ce != cudaSuccess) { cudaGetLastError(); rl_destroy(h); return RL_ERR_OOM; }
        h->d_head = (unsigned*)((char*)h->d_items + ((items.size() * sizeof(int4) + 255) & ~(size_t)255));
        h->n_items = (int)items.size();
        h->use_multi = 1;
    }
    ce = cudaMemsetAsync(h->d_img, 0, h->img_bytes, h->st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(h->d_lists, lists.data(), lists.size() * sizeof(int32_t),
                             cudaMemcpyHostToDevice, h->st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(h->d_img + h->seg_off[S_NROB], h->h_nrob.data(), E * 4,
                             cudaMemcpyHostToDevice, h->st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(h->d_img + h->seg_off[S_OFF], h->h_off.data(), (E + 1) * 4,
                             cudaMemcpyHostToDevice, h->st);
    if (ce == cudaSuccess && h->n_items > 0)
        ce = cudaMemcpyAsync(h->d_items, items.data(), items.size() * sizeof(int4),
                             cudaMemcpyHostToDevice, h->st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->st);
    if (ce != cudaSuccess) { rl_destroy(h); return RL_ERR_CUDA; }
    rl_status s = do_reset(h);
    if (s != RL_OK) { rl_destroy(h); return s; }
    *out = h;
    return RL_OK;
}

rl_status rl_reset(rl_env* h, uint64_t seed) {
    if (!h) return RL_ERR_ARG;
    h->seed = seed;
    drop_graph(h);
    return do_reset(h);
}

rl_status rl_step_io_call(rl_env* h, const rl_step_io* io) {
    if (!h || !io) return RL_ERR_ARG;
    if (!h->cfg.scripted && !io->d_actions)
        return fail(h, RL_ERR_ARG, "rl_step: actions are required for a policy-driven handle");
    if (h->cfg.scripted && io->d_actions)
        return fail(h, RL_ERR_ARG, "rl_step: a scripted handle takes no actions");
    return h->prec == 64 ? do_step<double>(h, io) : do_step<float>(h, io);
}

rl_status rl_step(rl_env* h, const void* d_actions, void* d_obs, void* d_reward,
                  uint8_t* d_done) {
    rl_step_io io;
    std::memset(&io, 0, sizeof(io));
    io.d_actions = d_actions;
    io.d_obs = d_obs;
    io.d_reward = d_reward;
    io.d_done = d_done;
    return rl_step_io_call(h, &io);
}

rl_status rl_rollout(rl_env* h, int32_t T, void* d_obs, void* d_rew, uint8_t* d_done) {
    if (!h || T < 0) return RL_ERR_ARG;
    if (!h->cfg.scripted) return fail(h, RL_ERR_STATE, "rl_rollout: the handle takes policy actions");
    if (T == 0) return RL_OK;
    if (!(h->gexec && h->g_T == T && h->g_obs == d_obs && h->g_rew == d_rew &&
          h->g_done == d_done)) {
        drop_graph(h);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(h->st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(h, e, "rollout capture");
        rl_status s = rollout_enqueue(h, T, d_obs, d_rew, d_done);
        e = cudaStreamEndCapture(h->st, &g);
        if (s != RL_OK) { if (g) cudaGraphDestroy(g); return s; }
        if (e != cudaSuccess) return cuda_fail(h, e, "rollout capture");
        e = cudaGraphInstantiate(&h->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { h->gexec = nullptr; return cuda_fail(h, e, "graph instantiate"); }
        h->g_T = T;
        h->g_obs = d_obs;
        h->g_rew = d_rew;
        h->g_done = d_done;
    }
    cudaError_t e = cudaGraphLaunch(h->gexec, h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "graph launch");
    return RL_OK;
}

rl_status rl_rollout_plain(rl_env* h, int32_t T, void* d_obs, void* d_rew, uint8_t* d_done) {
    if (!h || T < 0) return RL_ERR_ARG;
    if (!h->cfg.scripted) return fail(h, RL_ERR_STATE, "rl_rollout_plain: the handle takes policy actions");
    const size_t ostep = (size_t)h->total * h->obs_dim * h->esz;
    for (int t = 0; t < T; ++t) {
        for (int c = 0; c < h->ncls; ++c) {
            Class one = h->cls[c];
            for (int i = 0; i < h->cls[c].count; ++i) {
                one.begin = h->cls[c].begin + i;
                one.count = 1;
                one.block_threads = 32 > one.lanes ? 32 : one.lanes;
                cudaError_t e;
                void* o = d_obs ? (char*)d_obs + t * ostep : nullptr;
                if (h->prec == 64) {
                    rl::LaunchArgs<double> a;
                    fill_args(h, a);
                    a.io.obs = (double*)o;
                    a.io.reward = d_rew ? (double*)d_rew + (size_t)t * h->E : nullptr;
                    a.io.done = d_done ? d_done + (size_t)t * h->E : nullptr;
                    e = launch_class<double>(h, one, a, false);
                } else {
                    rl::LaunchArgs<float> a;
                    fill_args(h, a);
                    a.io.obs = (float*)o;
                    a.io.reward = d_rew ? (float*)d_rew + (size_t)t * h->E : nullptr;
                    a.io.done = d_done ? d_done + (size_t)t * h->E : nullptr;
                    e = launch_class<float>(h, one, a, false);
                }
                if (e != cudaSuccess) return cuda_fail(h, e, "plain step");
            }
        }
    }
    return RL_OK;
}

rl_status rl_tune(rl_env* h, int32_t T_probe, int32_t* h_choice) {
    if (!h || T_probe < 1) return RL_ERR_ARG;
    if (!h->cfg.scripted) return fail(h, RL_ERR_STATE, "rl_tune: the handle takes policy actions");
    // the probes run from a saved copy of the state, which is restored afterwards
    void* saved = nullptr;
    cudaError_t e = cudaMallocAsync(&saved, h->img_bytes, h->st);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(h, RL_ERR_OOM, "rl_tune: state copy"); }
    e = cudaMemcpyAsync(saved, h->d_img, h->img_bytes, cudaMemcpyDeviceToDevice, h->st);
    // the probes write trajectories like a real rollout: kernels differ most in their stores
    const size_t pob = (size_t)T_probe * h->total * h->obs_dim * h->esz;
    const size_t prb = ((size_t)T_probe * h->E * h->esz + 255) & ~(size_t)255;
    const size_t pdb = (size_t)T_probe * h->E;
    void* probe_out = nullptr;
    if (e == cudaSuccess) {
        e = cudaMallocAsync(&probe_out, ((pob + 255) & ~(size_t)255) + prb + pdb, h->st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaFreeAsync(saved, h->st);
            return fail(h, RL_ERR_OOM, "rl_tune: probe trajectories");
        }
    }
    char* po = (char*)probe_out;
    void* p_obs = po;
    void* p_rew = po + ((pob + 255) & ~(size_t)255);
    uint8_t* p_done = (uint8_t*)(po + ((pob + 255) & ~(size_t)255) + prb);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    auto probe = [&](float& ms) -> rl_status {
        float best = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaError_t ee = cudaMemcpyAsync(h->d_img, saved, h->img_bytes, cudaMemcpyDeviceToDevice, h->st);
            if (ee != cudaSuccess) return cuda_fail(h, ee, "rl_tune");
            cudaEventRecord(e0, h->st);
            rl_status st = rollout_enqueue(h, T_probe, p_obs, p_rew, p_done);
            if (st != RL_OK) return st;
            cudaEventRecord(e1, h->st);
            ee = cudaEventSynchronize(e1);
            if (ee != cudaSuccess) return cuda_fail(h, ee, "rl_tune");
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            best = std::min(best, t);
        }
        ms = best;
        return RL_OK;
    };
    rl_status st = e == cudaSuccess ? RL_OK : cuda_fail(h, e, "rl_tune");
    const int bts[3] = {32, 64, 128};
    // per class: the fastest (lanes, block) with only that class launched
    const int keep_multi = h->use_multi;
    h->use_multi = 0;
    for (int c = 0; c < h->ncls && st == RL_OK; ++c) {
        const int nc = h->ncls;
        Class all[rl::kNumClasses];
        for (int i = 0; i < nc; ++i) all[i] = h->cls[i];
        h->cls[0] = all[c];
        h->ncls = 1;
        const unsigned ok = rl::supported_lanes(h->prec, all[c].nmax);
        float best = 1e30f;
        Class pick = all[c];
        // candidates (lanes, block threads, envs per warp, 4-robot kernel variant)
        int cand[32][4];
        int nc_ = 0;
        if (h->prec == 32 && all[c].nmax == 4) {
            // envs per warp; 0: spread evenly over one block per SM
            const int we4[6] = {0, 2, 4, 6, 7, 8}, we1[3] = {8, 16, 32};
            for (int var = 1; var <= 2; ++var)
                for (int w = 0; w < 6; ++w) {
                    cand[nc_][0] = 4; cand[nc_][1] = 128; cand[nc_][2] = we4[w]; cand[nc_][3] = var;
                    ++nc_;
                }
            // dynamics and output warps (spread launch only)
            cand[nc_][0] = 4; cand[nc_][1] = 128; cand[nc_][2] = 0; cand[nc_][3] = 3; ++nc_;
            for (int w = 0; w < 3; ++w) {
                cand[nc_][0] = 1; cand[nc_][1] = 4 * we1[w]; cand[nc_][2] = 0; cand[nc_][3] = 0;
                ++nc_;
            }
            cand[nc_][0] = 2; cand[nc_][1] = 64; cand[nc_][2] = 0; cand[nc_][3] = 0; ++nc_;
        } else {
            for (int lanes = 1; lanes <= 32; lanes <<= 1) {
                if (!(ok & (unsigned)lanes)) continue;
                for (int b = 0; b < 3; ++b)
                    if (bts[b] >= lanes) {
                        cand[nc_][0] = lanes; cand[nc_][1] = bts[b]; cand[nc_][2] = 0; cand[nc_][3] = 0;
                        ++nc_;
                    }
            }
        }
        for (int ci = 0; ci < nc_ && st == RL_OK; ++ci) {
            h->cls[0].lanes = cand[ci][0];
            h->cls[0].block_threads = cand[ci][1];
            h->cls[0].warp_envs = cand[ci][2];
            h->cls[0].variant = cand[ci][3];
            float ms = 0.f;
            st = probe(ms);
            if (st == RL_OK && ms < best) { best = ms; pick = h->cls[0]; }
        }
        for (int i = 0; i < nc; ++i) h->cls[i] = all[i];
        h->ncls = nc;
        h->cls[c] = pick;
    }
    // uneven batches: one launch over every class, one launch per class in sequence, or one per
    // class on parallel streams
    if (st == RL_OK && h->n_items > 0) {
        float t_mode[3] = {0.f, 0.f, 0.f};
        for (int m = 0; m < 3 && st == RL_OK; ++m) {
            h->use_multi = m;
            st = probe(t_mode[m]);
        }
        int best_m = 1;
        for (int m = 0; m < 3; ++m)
            if (t_mode[m] < t_mode[best_m]) best_m = m;
        h->use_multi = st == RL_OK ? best_m : keep_multi;
    } else {
        h->use_multi = keep_multi;
    }
    cudaError_t er = cudaMemcpyAsync(h->d_img, saved, h->img_bytes, cudaMemcpyDeviceToDevice, h->st);
    if (er == cudaSuccess) er = cudaStreamSynchronize(h->st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(saved, h->st);
    if (probe_out) cudaFreeAsync(probe_out, h->st);
    drop_graph(h);
    if (st != RL_OK) return st;
    if (er != cudaSuccess) return cuda_fail(h, er, "rl_tune restore");
    if (h_choice) {
        h_choice[0] = h->use_multi;
        for (int c = 0; c < rl::kNumClasses; ++c) {
            h_choice[1 + 5 * c] = c < h->ncls ? h->cls[c].nmax : 0;
            h_choice[2 + 5 * c] = c < h->ncls ? h->cls[c].lanes : 0;
            h_choice[3 + 5 * c] = c < h->ncls ? h->cls[c].block_threads : 0;
            h_choice[4 + 5 * c] = c < h->ncls ? h->cls[c].warp_envs : 0;
            h_choice[5 + 5 * c] = c < h->ncls ? h->cls[c].variant : 0;
        }
    }
    return RL_OK;
}

rl_status rl_set_class_launch(rl_env* h, int32_t mode) {
    if (!h || mode < 0 || mode > 2) return RL_ERR_ARG;
    if (h->n_items == 0)
        return fail(h, RL_ERR_STATE, "rl_set_class_launch: the batch has one size class (or is binary64)");
    if (h->use_multi != mode) drop_graph(h);
    h->use_multi = mode;
    return RL_OK;
}

size_t rl_state_bytes(const rl_env* h) { return h ? sizeof(StateHeader) + h->img_bytes : 0; }

rl_status rl_get_state(rl_env* h, void* dst, size_t bytes) {
    if (!h || !dst || bytes < rl_state_bytes(h)) return RL_ERR_ARG;
    StateHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    hd.magic = kMagic;
    hd.version = kVersion;
    hd.precision = h->prec;
    hd.scenario = h->cfg.scenario;
    hd.n_envs = h->E;
    hd.total_robots = h->total;
    hd.r_max = h->r_max;
    hd.n_max = h->n_max;
    hd.seed = h->seed;
    hd.image_bytes = h->img_bytes;
    std::memcpy(dst, &hd, sizeof(hd));
    cudaError_t e = cudaMemcpyAsync((char*)dst + sizeof(hd), h->d_img, h->img_bytes,
                                    cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "get_state");
    return RL_OK;
}

rl_status rl_set_state(rl_env* h, const void* src, size_t bytes) {
    if (!h || !src || bytes < rl_state_bytes(h)) return RL_ERR_ARG;
    StateHeader hd;
    std::memcpy(&hd, src, sizeof(hd));
    if (hd.magic != kMagic || hd.version != kVersion || hd.precision != h->prec ||
        hd.scenario != h->cfg.scenario || hd.n_envs != h->E || hd.total_robots != h->total ||
        hd.r_max != h->r_max || hd.image_bytes != h->img_bytes)
        return fail(h, RL_ERR_ARG, "set_state: the blob does not match this handle");
    const char* img = (const char*)src + sizeof(hd);
    if (std::memcmp(img + h->seg_off[S_NROB], h->h_nrob.data(), h->E * 4) != 0 ||
        std::memcmp(img + h->seg_off[S_OFF], h->h_off.data(), (h->E + 1) * 4) != 0)
        return fail(h, RL_ERR_ARG, "set_state: robot counts differ from this handle");
    h->seed = hd.seed;
    cudaError_t e = cudaMemcpyAsync(h->d_img, img, h->img_bytes, cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "set_state");
    drop_graph(h);
    return RL_OK;
}

rl_status rl_rollout_host(rl_env* h, const void* h_state, int32_t T, void* h_obs, void* h_rew,
                          uint8_t* h_done) {
    if (!h || T < 0) return RL_ERR_ARG;
    if (h_state) {
        StateHeader hd;
        std::memcpy(&hd, h_state, sizeof(hd));
        if (hd.magic != kMagic || hd.image_bytes != h->img_bytes)
            return fail(h, RL_ERR_ARG, "rollout_host: bad state blob");
        const char* img = (const char*)h_state + sizeof(hd);
        cudaError_t e = cudaMemcpyAsync(h->d_img, img, h->img_bytes, cudaMemcpyHostToDevice, h->st);
        if (e != cudaSuccess) return cuda_fail(h, e, "rollout_host upload");
    }
    const size_t ob = h_obs ? (size_t)T * h->total * h->obs_dim * h->esz : 0;
    const size_t rb = h_rew ? (size_t)T * h->E * h->esz : 0;
    const size_t db = h_done ? (size_t)T * h->E : 0;
    const size_t need = ((ob + 255) & ~(size_t)255) + ((rb + 255) & ~(size_t)255) + db + 256;
    if (need > h->scratch_bytes) {
        if (h->d_scratch) { cudaFreeAsync(h->d_scratch, h->st); h->d_scratch = nullptr; h->scratch_bytes = 0; }
        drop_graph(h);
        if (cudaMallocAsync(&h->d_scratch, need, h->st) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, RL_ERR_OOM, "rollout_host: scratch allocation");
        }
        h->scratch_bytes = need;
    }
    char* base = (char*)h->d_scratch;
    void* d_obs = h_obs ? base : nullptr;
    void* d_rew = h_rew ? base + ((ob + 255) & ~(size_t)255) : nullptr;
    uint8_t* d_done = h_done ? (uint8_t*)(base + ((ob + 255) & ~(size_t)255) + ((rb + 255) & ~(size_t)255)) : nullptr;
    if (T == 0) return RL_OK;
    // The rollout in chunks of steps, each chunk one launch on the handle's stream; after a
    // chunk's launch an event, on which the copy stream waits before downloading that chunk's
    // slice of the observations.  Chunk k's download overlaps chunk k + 1's compute, so the call
    // takes about max(compute, copy) instead of their sum.  Chunking gives the same results:
    // the kernels write the state back after a chunk and read it at the next.
    cudaError_t e = cudaSuccess;
    if (!h->copy_st) {
        e = cudaStreamCreateWithFlags(&h->copy_st, cudaStreamNonBlocking);
        for (int k = 0; k < kHostChunks && e == cudaSuccess; ++k)
            e = cudaEventCreateWithFlags(&h->chunk_ev[k], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(h, e, "rollout_host streams");
    }
    const int nck = std::min(kHostChunks, (int)T);
    const size_t ostep = (size_t)h->total * h->obs_dim * h->esz, rstep = (size_t)h->E * h->esz;
    for (int k = 0; k < nck && e == cudaSuccess; ++k) {
        const size_t t0 = (size_t)T * k / nck, t1 = (size_t)T * (k + 1) / nck;
        rl_status s = rollout_enqueue(h, (int)(t1 - t0), d_obs ? (char*)d_obs + t0 * ostep : nullptr,
                                      d_rew ? (char*)d_rew + t0 * rstep : nullptr,
                                      d_done ? d_done + t0 * h->E : nullptr);
        if (s != RL_OK) return s;
        e = cudaEventRecord(h->chunk_ev[k], h->st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy_st, h->chunk_ev[k], 0);
        if (e == cudaSuccess && h_obs)
            e = cudaMemcpyAsync((char*)h_obs + t0 * ostep, (char*)d_obs + t0 * ostep,
                                (t1 - t0) * ostep, cudaMemcpyDeviceToHost, h->copy_st);
    }
    // rewards and done flags (a few percent of the bytes) in one copy each, after the last chunk
    if (e == cudaSuccess && h_rew)
        e = cudaMemcpyAsync(h_rew, d_rew, rb, cudaMemcpyDeviceToHost, h->copy_st);
    if (e == cudaSuccess && h_done)
        e = cudaMemcpyAsync(h_done, d_done, db, cudaMemcpyDeviceToHost, h->copy_st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->copy_st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "rollout_host download");
    return RL_OK;
}

rl_status rl_get_counters(rl_env* h, int32_t* dst) {
    if (!h || !dst) return RL_ERR_ARG;
    cudaError_t e = cudaMemcpyAsync(dst, h->d_img + h->seg_off[S_COUNTERS],
                                    h->seg_len[S_COUNTERS], cudaMemcpyDeviceToHost, h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "get_counters");
    return sync_and_take_status(h, "get_counters");
}

rl_status rl_sync(rl_env* h) {
    if (!h) return RL_ERR_ARG;
    return sync_and_take_status(h, "sync");
}

int32_t rl_obs_dim(const rl_env* h) { return h ? h->obs_dim : 0; }
int32_t rl_n_envs(const rl_env* h) { return h ? h->E : 0; }
int32_t rl_total_robots(const rl_env* h) { return h ? h->total : 0; }
int32_t rl_lanes(const rl_env* h) { return (h && h->ncls > 0) ? h->cls[0].lanes : 0; }
const char* rl_last_error(const rl_env* h) { return h ? h->err.c_str() : "null handle"; }

void rl_destroy(rl_env* h) {
    if (!h) return;
    if (h->st) cudaStreamSynchronize(h->st);
    drop_graph(h);
    // stream-ordered frees: no device-wide synchronisation
    if (h->d_scratch) cudaFreeAsync(h->d_scratch, h->st);
    for (int c = 0; c < rl::kNumClasses; ++c) {
        if (h->side[c]) cudaStreamDestroy(h->side[c]);
        if (h->join_ev[c]) cudaEventDestroy(h->join_ev[c]);
    }
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->copy_st) {
        cudaStreamSynchronize(h->copy_st);
        for (int k = 0; k < kHostChunks; ++k)
            if (h->chunk_ev[k]) cudaEventDestroy(h->chunk_ev[k]);
        cudaStreamDestroy(h->copy_st);
    }
    if (h->d_lists) cudaFreeAsync(h->d_lists, h->st);
    if (h->d_items) cudaFreeAsync(h->d_items, h->st);
    if (h->d_img) cudaFreeAsync(h->d_img, h->st);
    if (h->d_status) cudaFreeAsync(h->d_status, h->st);
    if (h->own_stream && h->st) cudaStreamDestroy(h->st);
    delete h;
}

}  // extern "C"

// ================================================================================================
// Serving: continuous batching of rollout requests under a device-memory budget
// ================================================================================================
namespace {

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

// Device bytes a request holds while it runs (state image, class lists, work items, returns).
size_t request_bytes(const rl_config& c, const rl_request& r) {
    const size_t E = (size_t)r.n_envs, rows = E * (size_t)r.n_robots;
    const size_t es = c.precision == RL_PREC_F64 ? 8 : 4;
    const size_t RM = c.scenario != RL_SCEN_NAVIGATION ? E * (size_t)c.r_max : 0;
    auto a = [](size_t v) { return (v + 255) & ~(size_t)255; };
    return 6 * a(rows * es) + a(rows * 4) + 3 * a(E * 4) + 2 * a(RM * es) + 2 * a(RM * 4) +
           a(E * rl::kNCount * 4) + a(E * 4) + a((E + 1) * 4) + a(E * 4) + a(E * es) + 4096;
}

struct SrvReq {
    uint64_t id;
    rl_request r;
    double t_submit;
    size_t bytes;
};

struct SrvSlot {
    bool busy = false;
    SrvReq req{};
    rl_env* env = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    void* d_ret = nullptr;
    double t_start = 0.0;
};

struct SrvResult {
    int status = 0;  // 0 queued, 1 running, 2 done, 3 failed
    rl_request r{};
    double t_submit = 0, t_start = 0, t_finish = 0;
    std::vector<float> returns;
    int32_t counters[RL_NCOUNT] = {};
};

}  // namespace

struct rl_server {
    rl_config cfg;
    size_t budget = 0, used = 0, peak = 0;
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<SrvReq> queue;
    std::vector<SrvSlot> slots;
    std::unordered_map<uint64_t, SrvResult> results;
    uint64_t next_id = 1;
    int64_t n_done = 0, env_steps_done = 0;
    bool stop = false;
    std::string err;
    std::thread engine;
};

namespace {

// Start a request in a free slot (engine thread, lock held).
bool srv_start(rl_server* S, SrvSlot& sl, const SrvReq& q) {
    rl_config c = S->cfg;
    c.scripted = 1;
    rl_env* env = nullptr;
    if (rl_create(&c, q.r.n_envs, nullptr, q.r.n_robots, q.r.seed, sl.st, &env) != RL_OK) return false;
    const size_t es = c.precision == RL_PREC_F64 ? 8 : 4;
    if (cudaMallocAsync(&sl.d_ret, (size_t)q.r.n_envs * es, sl.st) != cudaSuccess) {
        cudaGetLastError();
        rl_destroy(env);
        return false;
    }
    rl_status st = c.precision == RL_PREC_F64 ? do_rollout_returns<double>(env, q.r.horizon, sl.d_ret)
                                              : do_rollout_returns<float>(env, q.r.horizon, sl.d_ret);
    if (st != RL_OK || cudaEventRecord(sl.ev, sl.st) != cudaSuccess) {
        cudaFreeAsync(sl.d_ret, sl.st);
        rl_destroy(env);
        return false;
    }
    sl.env = env;
    sl.req = q;
    sl.busy = true;
    sl.t_start = now_s(S->t0);
    return true;
}

// Collect a finished request (engine thread, lock held).
void srv_finish(rl_server* S, SrvSlot& sl, bool ok) {
    SrvResult& R = S->results[sl.req.id];
    R.t_finish = now_s(S->t0);
    R.t_start = sl.t_start;
    R.status = 3;
    if (ok) {
        const size_t E = (size_t)sl.req.r.n_envs;
        R.returns.assign(E, 0.f);
        std::vector<int32_t> cnt(E * RL_NCOUNT);
        bool good = rl_get_counters(sl.env, cnt.data()) == RL_OK;
        if (S->cfg.precision == RL_PREC_F64) {
            std::vector<double> tmp(E);
            good = good && cudaMemcpyAsync(tmp.data(), sl.d_ret, E * 8, cudaMemcpyDeviceToHost, sl.st) == cudaSuccess;
            good = good && cudaStreamSynchronize(sl.st) == cudaSuccess;
            for (size_t i = 0; i < E; ++i) R.returns[i] = (float)tmp[i];
        } else {
            good = good && cudaMemcpyAsync(R.returns.data(), sl.d_ret, E * 4, cudaMemcpyDeviceToHost, sl.st) == cudaSuccess;
            good = good && cudaStreamSynchronize(sl.st) == cudaSuccess;
        }
        for (size_t e = 0; e < E; ++e)
            for (int k = 0; k < RL_NCOUNT; ++k) R.counters[k] += cnt[e * RL_NCOUNT + k];
        if (good) {
            R.status = 2;
            S->n_done += 1;
            S->env_steps_done += (int64_t)sl.req.r.n_envs * sl.req.r.horizon;
        }
    }
    cudaFreeAsync(sl.d_ret, sl.st);
    sl.d_ret = nullptr;
    rl_destroy(sl.env);
    sl.env = nullptr;
    sl.busy = false;
    S->used -= sl.req.bytes;
}

void srv_engine(rl_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        bool busy = false;
        for (SrvSlot& sl : S->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaSuccess) srv_finish(S, sl, true);
            else if (q != cudaErrorNotReady) { cudaGetLastError(); srv_finish(S, sl, false); }
            else busy = true;
        }
        // admit in arrival order while a slot and the budget allow
        while (!S->queue.empty() && S->used + S->queue.front().bytes <= S->budget) {
            SrvSlot* free_slot = nullptr;
            for (SrvSlot& sl : S->slots)
                if (!sl.busy) { free_slot = &sl; break; }
            if (!free_slot) break;
            SrvReq q = S->queue.front();
            S->queue.pop_front();
            S->used += q.bytes;
            S->peak = std::max(S->peak, S->used);
            S->results[q.id].status = 1;
            if (srv_start(S, *free_slot, q)) {
                busy = true;
            } else {
                S->used -= q.bytes;
                SrvResult& R = S->results[q.id];
                R.status = 3;
                R.t_finish = now_s(S->t0);
            }
        }
        S->cv.notify_all();
        if (busy) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        } else {
            S->cv.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
}

}  // namespace

extern "C" {

rl_status rl_server_create(const rl_config* cfg, size_t hbm_budget_bytes, int32_t max_slots,
                           rl_server** out) {
    if (!cfg || !out || max_slots < 1 || hbm_budget_bytes == 0) return RL_ERR_ARG;
    std::string why;
    if (!rl::valid_config(*cfg, why)) return RL_ERR_ARG;
    rl_server* S = new (std::nothrow) rl_server();
    if (!S) return RL_ERR_OOM;
    S->cfg = *cfg;
    S->budget = hbm_budget_bytes;
    S->t0 = std::chrono::steady_clock::now();
    if (cudaGetDevice(&S->device) != cudaSuccess) { delete S; return RL_ERR_CUDA; }
    S->slots.resize(max_slots);
    for (SrvSlot& sl : S->slots) {
        if (cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
            rl_server_destroy(S);
            return RL_ERR_CUDA;
        }
    }
    S->engine = std::thread(srv_engine, S);
    *out = S;
    return RL_OK;
}

rl_status rl_server_submit(rl_server* S, const rl_request* r, uint64_t* id) {
    if (!S || !r || !id) return RL_ERR_ARG;
    if (r->n_envs < 1 || r->n_robots < 1 || r->n_robots > rl::kMaxRobots || r->horizon < 0)
        return RL_ERR_ARG;
    if (S->cfg.n_max > 0 && r->n_robots > S->cfg.n_max) return RL_ERR_ARG;
    const size_t b = request_bytes(S->cfg, *r);
    if (b > S->budget) return RL_ERR_BUDGET;
    std::lock_guard<std::mutex> lk(S->mu);
    SrvReq q{S->next_id++, *r, now_s(S->t0), b};
    SrvResult& R = S->results[q.id];
    R.status = 0;
    R.r = *r;
    R.t_submit = q.t_submit;
    S->queue.push_back(q);
    *id = q.id;
    S->cv.notify_all();
    return RL_OK;
}

rl_status rl_server_result(rl_server* S, uint64_t id, rl_result* out, float* h_returns) {
    if (!S || !out) return RL_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->results.find(id);
    if (it == S->results.end()) return RL_ERR_ARG;
    const SrvResult& R = it->second;
    std::memset(out, 0, sizeof(*out));
    out->id = id;
    out->status = R.status;
    out->n_envs = R.r.n_envs;
    out->n_robots = R.r.n_robots;
    out->horizon = R.r.horizon;
    out->submit_s = R.t_submit;
    out->start_s = R.t_start;
    out->finish_s = R.t_finish;
    for (int k = 0; k < RL_NCOUNT; ++k) out->counters[k] = R.counters[k];
    double sum = 0.0;
    for (float v : R.returns) sum += v;
    out->mean_return = R.returns.empty() ? 0.0 : sum / (double)R.returns.size();
    if (h_returns && R.status == 2) std::memcpy(h_returns, R.returns.data(), R.returns.size() * 4);
    return R.status == 3 ? RL_ERR_CUDA : RL_OK;
}

rl_status rl_server_stats(rl_server* S, int64_t* out) {
    if (!S || !out) return RL_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    int64_t running = 0;
    for (const SrvSlot& sl : S->slots) running += sl.busy ? 1 : 0;
    out[0] = (int64_t)S->used;
    out[1] = (int64_t)S->peak;
    out[2] = S->n_done;
    out[3] = running;
    out[4] = (int64_t)S->queue.size();
    out[5] = S->env_steps_done;
    return RL_OK;
}

rl_status rl_server_drain(rl_server* S, double timeout_s) {
    if (!S) return RL_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::microseconds((int64_t)(timeout_s * 1e6));
    for (;;) {
        bool idle = S->queue.empty();
        for (const SrvSlot& sl : S->slots) idle = idle && !sl.busy;
        if (idle) return RL_OK;
        if (std::chrono::steady_clock::now() >= deadline) return RL_ERR_TIMEOUT;
        S->cv.wait_until(lk, deadline);
    }
}

rl_status rl_server_destroy(rl_server* S) {
    if (!S) return RL_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->engine.joinable()) S->engine.join();
    for (SrvSlot& sl : S->slots) {
        if (sl.busy) {
            cudaStreamSynchronize(sl.st);
            if (sl.d_ret) cudaFreeAsync(sl.d_ret, sl.st);
            rl_destroy(sl.env);
        }
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.st) {
            cudaStreamSynchronize(sl.st);
            cudaStreamDestroy(sl.st);
        }
    }
    delete S;
    return RL_OK;
}

}  // extern "C"
