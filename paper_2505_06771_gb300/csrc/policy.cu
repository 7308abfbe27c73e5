// policy.cu -- a recurrent policy evaluated on the GPU between environment steps (include/rl.h,
// "Policy in the loop"), and rl_observe.
//
// One policy step over all robots of the batch is one launch of policy_step_tc (policy_tc.cuh):
// the observation in bf16, h1 = ReLU(W1 o + b1) on the tensor cores, the GRU's gate products
// on the tensor cores (tcgen05, accumulators in tensor memory, operands by TMA), the gates, the
// new state and the two-output head, for 128 robots per CTA; then the environment step with
// those actions (rl_step).  The T steps are captured in a CUDA graph once and replayed.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rl.h"
#include "internal.h"
#include "policy_tc.cuh"

namespace {

// Navigation observation of the current state, one thread per robot (the definition the step
// kernels write after each step).
__global__ void observe_nav(rl::LaunchArgs<float> A, const int32_t* __restrict__ row_env,
                            int rows, float* __restrict__ obs) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const int e = row_env[r];
    const int off = A.s.off[e], N = A.s.nrob[e], i = r - off;
    const int od = A.io.obs_dim;
    float* o = obs + (size_t)r * od;
    const float x = A.s.x[r], y = A.s.y[r], th = A.s.th[r];
    const float head[5] = {x, y, th, A.s.gx[r], A.s.gy[r]};
    int c = 0;
    for (; c < 5 && c < od; ++c) o[c] = head[c];
    for (int j = 0; j < N; ++j) {
        if (j == i) continue;
        float d = A.s.th[off + j] - th;
        d = (d > CUDART_PI_F) ? d - 2.f * CUDART_PI_F : d;
        d = (d <= -CUDART_PI_F) ? d + 2.f * CUDART_PI_F : d;
        const float rel[3] = {A.s.x[off + j] - x, A.s.y[off + j] - y, d};
        for (int q = 0; q < 3; ++q, ++c)
            if (c < od) o[c] = rel[q];
    }
    for (; c < od; ++c) o[c] = 0.f;
}

__global__ void to_bf16(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, size_t n) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        dst[k] = __float2bfloat16_rn(src[k]);
}

int grid_for(size_t work, int threads) {
    size_t b = (work + threads - 1) / threads;
    if (b > 4096) b = 4096;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

struct rl_policy {
    rl_env* env = nullptr;
    int H = 0, U = 0, od = 0, rows = 0, E = 0;
    float vmax = 0.f;
    cudaStream_t st = nullptr;
    __nv_bfloat16 *w1 = nullptr, *wcat = nullptr, *cat = nullptr;
    float *b1 = nullptr, *bias = nullptr, *wo = nullptr, *bo = nullptr, *h = nullptr, *act = nullptr;
    int32_t* row_env = nullptr;
    int32_t* status = nullptr;   // the handle's device status word (a wait that ran out)
    uint8_t* done0 = nullptr;    // [E] episode ended at the last step of the previous rollout
    CUtensorMap tmA{}, tmB{};    // A = cat [rows][2H]; B = the gate weights [4H][2H]
    size_t smem = 0;
    cudaGraphExec_t gexec = nullptr;
    int g_T = -1;
    const void* g_ptr[5] = {};
};

namespace {

void policy_free(rl_policy* p) {
    if (!p) return;
    if (p->st) cudaStreamSynchronize(p->st);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    void* bufs[] = {p->w1, p->b1, p->wcat, p->bias, p->wo, p->bo, p->cat, p->h, p->act,
                    p->row_env, p->done0};
    for (void* b : bufs)
        if (b) cudaFreeAsync(b, p->st);
    if (p->st) cudaStreamSynchronize(p->st);
    delete p;
}

// A 2-D bf16 tensor map [rows][cols] (row-major) with boxes of 64 columns x box_rows rows and
// the 128-byte swizzle the MMA descriptors expect.
bool make_map(CUtensorMap* map, const void* base, uint64_t cols, uint64_t rows, uint32_t box_rows,
              std::string& why) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
            why = "cuTensorMapEncodeTiled unavailable";
            return false;
        }
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[2] = {cols, rows};
    const cuuint64_t strides[1] = {cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)rl::ptc::kKc, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                              strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        why = "tensor map encode failed (" + std::to_string((int)r) + ")";
        return false;
    }
    return true;
}

rl_status fail(rl_env* env, rl_policy* p, rl_status s, const std::string& msg) {
    if (env) rl::env_set_error(env, msg);
    policy_free(p);
    return s;
}

// T policy steps enqueued on the handle's stream (captured into a graph by the caller).
rl_status enqueue_rollout(rl_env* env, rl_policy* p, int T, const float* obs0, float* obs,
                          float* rew, uint8_t* done, float* act) {
    const size_t ob = (size_t)p->rows * p->od;
    rl::ptc::Params P;
    P.row_env = p->row_env;
    P.cat = p->cat;
    P.h = p->h;
    P.w1 = p->w1;
    P.b1 = p->b1;
    P.bias = p->bias;
    P.wo = p->wo;
    P.bo = p->bo;
    P.status = p->status;
    P.rows = p->rows;
    P.od = p->od;
    P.H = p->H;
    P.U = p->U;
    P.vmax = p->vmax;
    const int grid = (p->rows + rl::ptc::kM - 1) / rl::ptc::kM;
    for (int t = 0; t < T; ++t) {
        P.obs = (t == 0) ? obs0 : obs + (size_t)(t - 1) * ob;
        P.done_prev = (t == 0) ? p->done0 : done + (size_t)(t - 1) * p->E;
        P.act = act ? act + (size_t)t * p->rows * 2 : p->act;
        rl::ptc::policy_step_tc<<<grid, rl::ptc::kThreads, p->smem, p->st>>>(p->tmA, p->tmB, P);
        if (cudaGetLastError() != cudaSuccess) return RL_ERR_CUDA;
        const rl_status s = rl_step(env, P.act, obs + (size_t)t * ob,
                                    rew ? rew + (size_t)t * p->E : nullptr,
                                    done + (size_t)t * p->E);
        if (s != RL_OK) return s;
    }
    if (cudaMemcpyAsync(p->done0, done + (size_t)(T - 1) * p->E, p->E, cudaMemcpyDeviceToDevice,
                        p->st) != cudaSuccess)
        return RL_ERR_CUDA;
    return RL_OK;
}

}  // namespace

extern "C" {

rl_status rl_policy_create(rl_env* env, int32_t hidden, const float* h_w1, const float* h_b1,
                           const float* h_wi, const float* h_bi, const float* h_wh,
                           const float* h_bh, const float* h_wo, const float* h_bo,
                           rl_policy** out) {
    if (!env || !out || !h_w1 || !h_b1 || !h_wi || !h_bi || !h_wh || !h_bh || !h_wo || !h_bo)
        return RL_ERR_ARG;
    *out = nullptr;
    const rl_config& c = rl::env_config(env);
    if (c.precision != RL_PREC_F32 || c.scripted)
        return fail(env, nullptr, RL_ERR_ARG, "rl_policy_create: needs a binary32 handle that takes policy actions");
    if (hidden < 64 || hidden > 512 || hidden % 64 != 0)
        return fail(env, nullptr, RL_ERR_ARG, "rl_policy_create: hidden must be a multiple of 64 up to 512");
    if (rl_obs_dim(env) > 16)
        return fail(env, nullptr, RL_ERR_ARG, "rl_policy_create: observations of at most 16 values (4 robots)");
    rl_policy* p = new (std::nothrow) rl_policy();
    if (!p) return RL_ERR_OOM;
    p->env = env;
    p->H = hidden;
    // hidden units per block of gate accumulators (shared memory: 2 stages of 3 gate slots of
    // U x 64 bf16 each, beside the resident A of H <= 256)
    p->U = (hidden == 128 || (hidden > rl::ptc::kResidentH && hidden % 128 == 0)) ? 128 : 64;
    p->od = rl_obs_dim(env);
    p->rows = rl_total_robots(env);
    p->E = rl_n_envs(env);
    p->vmax = (float)c.vmax;
    p->st = rl::env_stream(env);
    p->smem = rl::ptc::smem_bytes(p->U, p->H);
    {
        rl::LaunchArgs<float> a;
        rl::env_args_f32(env, a);
        p->status = a.io.status;  // the policy kernel reports into the handle's status word
    }
    const int H = p->H, od = p->od, rows = p->rows;
    // weights on the host in their device layouts: W1 [H][16] (observation padded), the gate
    // weights [4H][2H] = [[Wi_r, Wh_r], [Wi_z, Wh_z], [Wi_n, 0], [0, Wh_n]], biases [4H]
    std::vector<float> w1((size_t)H * 16, 0.f), wcat((size_t)4 * H * 2 * H, 0.f), bias(4 * H), b1(H);
    for (int u = 0; u < H; ++u)
        for (int q = 0; q < od; ++q) w1[(size_t)u * 16 + q] = h_w1[(size_t)u * od + q];
    for (int gte = 0; gte < 3; ++gte)
        for (int u = 0; u < H; ++u) {
            const size_t src = (size_t)(gte * H + u) * H;
            float* dst_i = &wcat[(size_t)(gte * H + u) * 2 * H];
            float* dst_h = &wcat[(size_t)((gte == 2 ? 3 : gte) * H + u) * 2 * H + H];
            for (int v = 0; v < H; ++v) {
                dst_i[v] = h_wi[src + v];
                dst_h[v] = h_wh[src + v];
            }
        }
    for (int u = 0; u < H; ++u) {
        bias[u] = h_bi[u] + h_bh[u];
        bias[H + u] = h_bi[H + u] + h_bh[H + u];
        bias[2 * H + u] = h_bi[2 * H + u];
        bias[3 * H + u] = h_bh[2 * H + u];
        // the first layer's bias enters in bf16 (rounded to nearest even)
        uint32_t bits;
        std::memcpy(&bits, &h_b1[u], 4);
        bits = (bits + 0x7FFFu + ((bits >> 16) & 1u)) & 0xFFFF0000u;
        std::memcpy(&b1[u], &bits, 4);
    }
    std::vector<int32_t> row_env(rows);
    const std::vector<int32_t>& off = rl::env_offsets(env);
    for (int e = 0; e < p->E; ++e)
        for (int r = off[e]; r < off[e + 1]; ++r) row_env[r] = e;
    // device buffers (the state per tile of 128 robots, unit-major)
    const size_t h_bytes = (size_t)((rows + rl::ptc::kM - 1) / rl::ptc::kM) * rl::ptc::kM * H * 4;
    float* staging = nullptr;
    const size_t stage_n = std::max(w1.size(), wcat.size());
    bool ok = cudaMallocAsync((void**)&p->w1, w1.size() * 2, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->b1, (size_t)H * 4, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->wcat, wcat.size() * 2, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->bias, bias.size() * 4, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->wo, (size_t)2 * H * 4, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->bo, 2 * 4, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->cat, (size_t)rows * 2 * H * 2, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->h, h_bytes, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->act, (size_t)rows * 2 * 4, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->row_env, (size_t)rows * 4, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->done0, (size_t)p->E, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&staging, stage_n * 4, p->st) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        if (staging) cudaFreeAsync(staging, p->st);
        return fail(env, p, RL_ERR_OOM, "rl_policy_create: device memory");
    }
    auto up_bf16 = [&](const float* src, size_t n, __nv_bfloat16* dst) {
        if (cudaMemcpyAsync(staging, src, n * 4, cudaMemcpyHostToDevice, p->st) != cudaSuccess)
            return false;
        to_bf16<<<grid_for(n, 256), 256, 0, p->st>>>(staging, dst, n);
        return cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(p->st) == cudaSuccess;
    };
    ok = up_bf16(w1.data(), w1.size(), p->w1) && up_bf16(wcat.data(), wcat.size(), p->wcat) &&
         cudaMemcpyAsync(p->b1, b1.data(), (size_t)H * 4, cudaMemcpyHostToDevice, p->st) == cudaSuccess &&
         cudaMemcpyAsync(p->bias, bias.data(), bias.size() * 4, cudaMemcpyHostToDevice, p->st) == cudaSuccess &&
         cudaMemcpyAsync(p->wo, h_wo, (size_t)2 * H * 4, cudaMemcpyHostToDevice, p->st) == cudaSuccess &&
         cudaMemcpyAsync(p->bo, h_bo, 2 * 4, cudaMemcpyHostToDevice, p->st) == cudaSuccess &&
         cudaMemcpyAsync(p->row_env, row_env.data(), (size_t)rows * 4, cudaMemcpyHostToDevice, p->st) == cudaSuccess &&
         cudaMemsetAsync(p->h, 0, h_bytes, p->st) == cudaSuccess &&
         cudaMemsetAsync(p->cat, 0, (size_t)rows * 2 * H * 2, p->st) == cudaSuccess &&
         cudaMemsetAsync(p->done0, 0, (size_t)p->E, p->st) == cudaSuccess &&
         cudaStreamSynchronize(p->st) == cudaSuccess;
    cudaFreeAsync(staging, p->st);
    if (!ok) return fail(env, p, RL_ERR_CUDA, "rl_policy_create: upload");
    std::string why;
    if (!make_map(&p->tmA, p->cat, 2 * (uint64_t)H, (uint64_t)rows, rl::ptc::kM, why) ||
        !make_map(&p->tmB, p->wcat, 2 * (uint64_t)H, 4 * (uint64_t)H, (uint32_t)p->U, why))
        return fail(env, p, RL_ERR_CUDA, "rl_policy_create: " + why);
    if (cudaFuncSetAttribute(rl::ptc::policy_step_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)p->smem) != cudaSuccess)
        return fail(env, p, RL_ERR_CUDA, "rl_policy_create: shared memory");
    *out = p;
    return RL_OK;
}

rl_status rl_policy_reset_hidden(rl_policy* p) {
    if (!p) return RL_ERR_ARG;
    const size_t h_bytes = (size_t)((p->rows + rl::ptc::kM - 1) / rl::ptc::kM) * rl::ptc::kM * p->H * 4;
    if (cudaMemsetAsync(p->h, 0, h_bytes, p->st) != cudaSuccess ||
        cudaMemsetAsync(p->cat, 0, (size_t)p->rows * 2 * p->H * 2, p->st) != cudaSuccess ||
        cudaMemsetAsync(p->done0, 0, (size_t)p->E, p->st) != cudaSuccess)
        return RL_ERR_CUDA;
    return RL_OK;
}

rl_status rl_policy_rollout(rl_env* env, rl_policy* p, int32_t T, const void* d_obs0,
                            void* d_obs_traj, void* d_rew_traj, uint8_t* d_done_traj,
                            void* d_act_traj) {
    if (!env || !p || p->env != env || T < 0 || !d_obs0 || !d_obs_traj || !d_done_traj)
        return RL_ERR_ARG;
    if (T == 0) return RL_OK;
    const void* key[5] = {d_obs0, d_obs_traj, d_rew_traj, d_done_traj, d_act_traj};
    bool same = p->gexec && p->g_T == T;
    for (int q = 0; q < 5 && same; ++q) same = (p->g_ptr[q] == key[q]);
    if (!same) {
        if (p->gexec) cudaGraphExecDestroy(p->gexec);
        p->gexec = nullptr;
        p->g_T = -1;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { rl::env_set_error(env, "policy rollout capture"); return RL_ERR_CUDA; }
        const rl_status s = enqueue_rollout(env, p, T, (const float*)d_obs0, (float*)d_obs_traj,
                                            (float*)d_rew_traj, d_done_traj, (float*)d_act_traj);
        e = cudaStreamEndCapture(p->st, &g);
        if (s != RL_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            rl::env_set_error(env, "policy rollout capture");
            return s != RL_OK ? s : RL_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&p->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            p->gexec = nullptr;
            rl::env_set_error(env, std::string("policy rollout graph instantiate: ") +
                                       cudaGetErrorString(e));
            return RL_ERR_CUDA;
        }
        p->g_T = T;
        for (int q = 0; q < 5; ++q) p->g_ptr[q] = key[q];
    }
    if (cudaGraphLaunch(p->gexec, p->st) != cudaSuccess) {
        rl::env_set_error(env, "policy rollout graph launch");
        return RL_ERR_CUDA;
    }
    return RL_OK;
}

void rl_policy_destroy(rl_policy* p) { policy_free(p); }

rl_status rl_observe(rl_env* env, void* d_obs) {
    if (!env || !d_obs) return RL_ERR_ARG;
    rl::LaunchArgs<float> a;
    if (!rl::env_args_f32(env, a) || rl::env_config(env).scenario != RL_SCEN_NAVIGATION) {
        rl::env_set_error(env, "rl_observe: binary32 Navigation handles only");
        return RL_ERR_ARG;
    }
    const int rows = rl_total_robots(env);
    const std::vector<int32_t>& off = rl::env_offsets(env);
    std::vector<int32_t> row_env(rows);
    for (int e = 0; e + 1 < (int)off.size(); ++e)
        for (int r = off[e]; r < off[e + 1]; ++r) row_env[r] = e;
    cudaStream_t st = rl::env_stream(env);
    int32_t* d_map = nullptr;
    if (cudaMallocAsync((void**)&d_map, (size_t)rows * 4, st) != cudaSuccess) {
        cudaGetLastError();
        return RL_ERR_OOM;
    }
    cudaError_t e = cudaMemcpyAsync(d_map, row_env.data(), (size_t)rows * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        observe_nav<<<(rows + 127) / 128, 128, 0, st>>>(a, d_map, rows, (float*)d_obs);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamSynchronize(st);  // the host map is freed on return
    cudaFreeAsync(d_map, st);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        rl::env_set_error(env, "rl_observe");
        return RL_ERR_CUDA;
    }
    return RL_OK;
}

}  // extern "C"
