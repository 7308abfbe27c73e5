// rl_noalloc.cu -- rl_rollout_noalloc: a reset + rollout that allocates no memory.
//
// Some callers cannot allocate device memory: code that runs while another component owns the
// device allocator (a caching allocator that must see every allocation, a process with a fixed
// memory budget enforced by its framework), or code that must not trigger the implicit
// synchronisation a cudaMalloc/cudaFree can cause.  For them this entry point keeps the whole
// environment state in one file-scope device array instead of a handle's cudaMalloc'd buffer.
// The kernels are the same ones rl_rollout launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>

#include "../../include/rl.h"
#include "internal.h"
#include "launch.h"

namespace {

constexpr size_t kStaticBytes = RL_NOALLOC_MAX_BYTES;
static_assert(kStaticBytes % 256 == 0, "the static state array holds 256-byte segments");
static __device__ __align__(256) unsigned char g_noalloc_state[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_lookup_mu;
void* g_state_ptr[kMaxDevices] = {};

// Device address of the static state array on the current device (looked up once per device).
cudaError_t state_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_lookup_mu);
    if (!g_state_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_state);
        if (e != cudaSuccess) return e;
        g_state_ptr[dev] = p;
    }
    *out = g_state_ptr[dev];
    return cudaSuccess;
}

// Robot offsets and counts of a batch with the same robot count in every env.
__global__ void fill_layout(int32_t* off, int32_t* nrob, int n_envs, int n_robots) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e <= n_envs; e += gridDim.x * blockDim.x) {
        off[e] = e * n_robots;
        if (e < n_envs) nrob[e] = n_robots;
    }
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

template <typename R>
rl_status run(const rl_config& c, int E, int N, uint64_t seed, int T, void* obs, void* rew,
              uint8_t* done, cudaStream_t st, unsigned char* base) {
    const int n_max = c.n_max > 0 ? c.n_max : N;
    const int r_max = c.scenario != RL_SCEN_NAVIGATION ? c.r_max : 0;
    const size_t rows = (size_t)E * N, RM = (size_t)E * r_max, es = sizeof(R);
    // state segments, each 256-byte aligned
    size_t pos = 0;
    auto take = [&](size_t bytes) { size_t p = pos; pos += align256(bytes); return base + p; };
    rl::LaunchArgs<R> a;
    std::memset(&a, 0, sizeof(a));
    a.s.x = (R*)take(rows * es);
    a.s.y = (R*)take(rows * es);
    a.s.th = (R*)take(rows * es);
    a.s.gx = (R*)take(rows * es);
    a.s.gy = (R*)take(rows * es);
    a.s.gth = (R*)take(rows * es);
    a.s.level = (int32_t*)take(rows * 4);
    a.s.t = (int32_t*)take((size_t)E * 4);
    a.s.ep = (int32_t*)take((size_t)E * 4);
    a.s.n_res = (int32_t*)take((size_t)E * 4);
    a.s.qx = (R*)take(RM * es);
    a.s.qy = (R*)take(RM * es);
    a.s.qlevel = (int32_t*)take(RM * 4);
    a.s.qactive = (int32_t*)take(RM * 4);
    a.s.counters = (int32_t*)take((size_t)E * rl::kNCount * 4);
    int32_t* nrob = (int32_t*)take((size_t)E * 4);
    int32_t* off = (int32_t*)take((size_t)(E + 1) * 4);
    a.s.nrob = nrob;
    a.s.off = off;

    const int od = c.scenario == RL_SCEN_DISCOVERY ? 5 + 5 * (n_max - 1) + 4 * r_max
                 : c.scenario == RL_SCEN_FORAGING ? 4 + 4 * (n_max - 1) + 4 * r_max
                                                  : 5 + 3 * (n_max - 1);
    a.io.E = E;
    a.io.obs_dim = od;
    a.io.obs_step = (long long)rows * od;
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
    k.scenario = c.scenario; k.scripted = 1; k.episode_len = c.episode_len;
    k.max_iter = c.qp_max_iter > 0 ? c.qp_max_iter : 8 * n_max + 16;
    k.n_res_min = c.n_res_min; k.n_res_max = c.n_res_max; k.r_max = r_max;
    k.n_max_obs = n_max; k.max_attempts = c.max_attempts; k.resolve_f64 = c.resolve_f64;
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
    a.env_list = nullptr;  // env = index
    a.n_list = E;
    a.env_begin = 0;
    a.seed = seed;

    // the robot-count class this batch runs in, with the launch shape rl_create would give it
    // (the configuration's lanes, block size, envs per warp and 4-robot variant, else the
    // class defaults)
    int ci = 0;
    while (ci + 1 < rl::kNumClasses && N > rl::kClassNmax[ci]) ++ci;
    const int nmax_class = rl::kClassNmax[ci];
    const unsigned ok = rl::supported_lanes(c.precision, nmax_class);
    int lanes = c.lanes > 0 ? c.lanes : rl::kClassLanes[ci];
    if (!(ok & (unsigned)lanes)) lanes = rl::kClassLanes[ci];
    int bt = nmax_class <= 16 ? 64 : 32;
    if (c.block_threads > 0) bt = std::max(c.block_threads, lanes);
    a.warp_envs = c.warp_envs > 0 ? std::min(32, c.warp_envs) : 0;
    a.variant = (c.small_variant >= 1 && c.small_variant <= 3) ? c.small_variant : 0;
    auto launch = [&](bool reset) -> cudaError_t {
        if constexpr (std::is_same<R, double>::value) {
            return rl::launch_f64(a, nmax_class, lanes, bt, 0, st, reset);
        } else {
            if (nmax_class == 4) return rl::launch_f32_small(a, lanes, bt, 0, st, reset);
            return rl::launch_f32_large(a, nmax_class, lanes, bt, 0, st, reset);
        }
    };
    // every byte the kernels read is written first: layout, then the reset of every env
    fill_layout<<<(E + 256) / 256, 256, 0, st>>>(off, nrob, E, N);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        a.T = 1;
        e = launch(true);
    }
    if (e == cudaSuccess && T > 0) {
        a.T = T;
        a.io.obs = (R*)obs;
        a.io.reward = (R*)rew;
        a.io.done = done;
        e = launch(false);
    }
    return e == cudaSuccess ? RL_OK : RL_ERR_CUDA;
}

}  // namespace

extern "C" size_t rl_noalloc_state_bytes(const rl_config* c, int32_t n_envs, int32_t n_robots) {
    if (!c || n_envs < 1 || n_robots < 1) return 0;
    const size_t E = (size_t)n_envs, rows = E * (size_t)n_robots;
    const size_t es = c->precision == RL_PREC_F64 ? 8 : 4;
    const size_t RM = c->scenario != RL_SCEN_NAVIGATION ? E * (size_t)c->r_max : 0;
    return 6 * align256(rows * es) + align256(rows * 4) + 3 * align256(E * 4) +
           2 * align256(RM * es) + 2 * align256(RM * 4) + align256(E * rl::kNCount * 4) +
           align256(E * 4) + align256((E + 1) * 4);
}

extern "C" rl_status rl_rollout_noalloc(const rl_config* cfg, int32_t n_envs, int32_t n_robots,
                                        uint64_t seed, int32_t T, void* d_obs_traj,
                                        void* d_rew_traj, uint8_t* d_done_traj, void* stream) {
    if (!cfg || n_envs < 1 || n_robots < 1 || n_robots > rl::kMaxRobots || T < 0) return RL_ERR_ARG;
    const rl_config& c = *cfg;
    std::string why;
    if (!rl::valid_config(c, why)) return RL_ERR_ARG;  // the checks rl_create makes
    if (!c.scripted) return RL_ERR_ARG;
    if (c.n_max != 0 && c.n_max < n_robots) return RL_ERR_ARG;
    if (rl_noalloc_state_bytes(cfg, n_envs, n_robots) > kStaticBytes) return RL_ERR_ARG;
    void* base = nullptr;
    if (state_address(&base) != cudaSuccess) return RL_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    if (c.precision == RL_PREC_F64)
        return run<double>(c, n_envs, n_robots, seed, T, d_obs_traj, d_rew_traj, d_done_traj, st,
                           (unsigned char*)base);
    return run<float>(c, n_envs, n_robots, seed, T, d_obs_traj, d_rew_traj, d_done_traj, st,
                      (unsigned char*)base);
}
