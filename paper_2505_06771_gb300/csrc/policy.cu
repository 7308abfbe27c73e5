// policy.cu -- a recurrent policy evaluated on the GPU between environment steps (include/rl.h,
// "Policy in the loop"), and rl_observe.
//
// One policy step over all robots of the batch:
//   1. policy_input: the observation to bf16 (padded to a multiple of 16 columns); robots whose
//      env ended its episode at the previous step get a zero recurrent state;
//   2. tensor cores (cuBLASLt): h1 = ReLU(W1 o + b1), written in bf16 into the first half of
//      each robot's [h1, h_prev] row;
//   3. tensor cores (cuBLASLt): the gate pre-activations of r, z and the two halves of n from
//      [h1, h_prev] with one block weight [[Wi_r, Wh_r], [Wi_z, Wh_z], [Wi_n, 0], [0, Wh_n]]
//      (one GEMM with K = 2H instead of two);
//   4. policy_gates: gates, the new state (binary32, and its bf16 copy for the next GEMM), and the
//      two-output head reduced across a warp per robot;
//   5. the environment step with those actions (rl_step).
// The T steps are captured in a CUDA graph once and replayed.
#include <cublasLt.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/rl.h"
#include "internal.h"

namespace {

constexpr size_t kLtWorkspace = size_t(32) << 20;

__global__ void policy_input(const float* __restrict__ obs, int rows, int od, int odp, int H,
                             const int32_t* __restrict__ row_env,
                             const uint8_t* __restrict__ done_prev, __nv_bfloat16* __restrict__ x,
                             __nv_bfloat16* __restrict__ cat, float* __restrict__ h) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int r = warp; r < rows; r += nwarps) {
        for (int c = lane; c < odp; c += 32)
            x[(size_t)r * odp + c] = __float2bfloat16_rn(c < od ? obs[(size_t)r * od + c] : 0.f);
        if (done_prev && done_prev[row_env[r]]) {
            for (int u = lane; u < H; u += 32) {
                h[(size_t)r * H + u] = 0.f;
                cat[(size_t)r * 2 * H + H + u] = __float2bfloat16_rn(0.f);
            }
        }
    }
}

// Gate nonlinearities on the special-function unit: tanh.approx.f32 (relative error about
// 2^-11, below the bf16 rounding of the GEMM operands) and sigma(v) = (1 + tanh(v / 2)) / 2.
__device__ __forceinline__ float tanh_sfu(float v) {
    float r;
    asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float sigmoid_f(float v) { return fmaf(0.5f, tanh_sfu(0.5f * v), 0.5f); }

// One warp per robot: gates from the pre-activations g [rows][4H] (r, z, n from h1, n from
// h_prev), the new state, and a = v_max tanh(Wo h + bo).
__global__ void policy_gates(const float* __restrict__ g, const float* __restrict__ bias,
                             const float* __restrict__ wo, const float* __restrict__ bo, int rows,
                             int H, float vmax, float* __restrict__ h,
                             __nv_bfloat16* __restrict__ cat, float* __restrict__ act) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int r = warp; r < rows; r += nwarps) {
        const float* gr = g + (size_t)r * 4 * H;
        float a0 = 0.f, a1 = 0.f;
        for (int u = lane; u < H; u += 32) {
            const float rg = sigmoid_f(gr[u] + bias[u]);
            const float zg = sigmoid_f(gr[H + u] + bias[H + u]);
            const float ng = tanh_sfu(gr[2 * H + u] + bias[2 * H + u] + rg * (gr[3 * H + u] + bias[3 * H + u]));
            const float hp = h[(size_t)r * H + u];
            const float hn = (1.f - zg) * ng + zg * hp;
            h[(size_t)r * H + u] = hn;
            cat[(size_t)r * 2 * H + H + u] = __float2bfloat16_rn(hn);
            a0 += wo[u] * hn;
            a1 += wo[H + u] * hn;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        }
        if (lane == 0) {
            act[2 * (size_t)r] = vmax * tanhf(a0 + bo[0]);
            act[2 * (size_t)r + 1] = vmax * tanhf(a1 + bo[1]);
        }
    }
}

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
    int H = 0, od = 0, odp = 0, rows = 0, E = 0;
    float vmax = 0.f;
    cudaStream_t st = nullptr;
    cublasLtHandle_t lt = nullptr;
    __nv_bfloat16 *w1 = nullptr, *b1 = nullptr, *wcat = nullptr;
    float *bias = nullptr, *wo = nullptr, *bo = nullptr;
    __nv_bfloat16 *x = nullptr, *cat = nullptr;
    float *g = nullptr, *h = nullptr, *act = nullptr;
    int32_t* row_env = nullptr;
    uint8_t* done0 = nullptr;  // [E] episode ended at the last step of the previous rollout
    void* ws = nullptr;
    cublasLtMatmulDesc_t d1 = nullptr, d2 = nullptr;
    cublasLtMatrixLayout_t la1 = nullptr, lb1 = nullptr, lc1 = nullptr;
    cublasLtMatrixLayout_t la2 = nullptr, lb2 = nullptr, lc2 = nullptr;
    cublasLtMatmulAlgo_t algo1{}, algo2{};
    cudaGraphExec_t gexec = nullptr;
    int g_T = -1;
    const void* g_ptr[5] = {};
};

namespace {

void policy_free(rl_policy* p) {
    if (!p) return;
    if (p->st) cudaStreamSynchronize(p->st);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->d1) cublasLtMatmulDescDestroy(p->d1);
    if (p->d2) cublasLtMatmulDescDestroy(p->d2);
    for (cublasLtMatrixLayout_t l : {p->la1, p->lb1, p->lc1, p->la2, p->lb2, p->lc2})
        if (l) cublasLtMatrixLayoutDestroy(l);
    if (p->lt) cublasLtDestroy(p->lt);
    void* bufs[] = {p->w1, p->b1, p->wcat, p->bias, p->wo, p->bo, p->x, p->cat, p->g,
                    p->h, p->act, p->row_env, p->done0, p->ws};
    for (void* b : bufs)
        if (b) cudaFreeAsync(b, p->st);
    if (p->st) cudaStreamSynchronize(p->st);
    delete p;
}

// One cuBLASLt matmul description: column-major D [m][n] = op_T(A) B with A stored [k][m].
bool make_gemm(cublasLtHandle_t lt, int m, int n, int k, int lda, int ldb, int ldc,
               cudaDataType_t ctype, cublasLtEpilogue_t epi, const void* bias,
               cudaDataType_t bias_type,
               cublasLtMatmulDesc_t* desc, cublasLtMatrixLayout_t* la, cublasLtMatrixLayout_t* lb,
               cublasLtMatrixLayout_t* lc, cublasLtMatmulAlgo_t* algo, std::string& why) {
    if (cublasLtMatmulDescCreate(desc, CUBLAS_COMPUTE_32F, CUDA_R_32F) != CUBLAS_STATUS_SUCCESS) {
        why = "matmul description";
        return false;
    }
    const cublasOperation_t ta = CUBLAS_OP_T, tb = CUBLAS_OP_N;
    cublasLtMatmulDescSetAttribute(*desc, CUBLASLT_MATMUL_DESC_TRANSA, &ta, sizeof(ta));
    cublasLtMatmulDescSetAttribute(*desc, CUBLASLT_MATMUL_DESC_TRANSB, &tb, sizeof(tb));
    cublasLtMatmulDescSetAttribute(*desc, CUBLASLT_MATMUL_DESC_EPILOGUE, &epi, sizeof(epi));
    if (bias) {
        cublasLtMatmulDescSetAttribute(*desc, CUBLASLT_MATMUL_DESC_BIAS_POINTER, &bias, sizeof(bias));
        cublasLtMatmulDescSetAttribute(*desc, CUBLASLT_MATMUL_DESC_BIAS_DATA_TYPE, &bias_type,
                                       sizeof(bias_type));
    }
    if (cublasLtMatrixLayoutCreate(la, CUDA_R_16BF, k, m, lda) != CUBLAS_STATUS_SUCCESS ||
        cublasLtMatrixLayoutCreate(lb, CUDA_R_16BF, k, n, ldb) != CUBLAS_STATUS_SUCCESS ||
        cublasLtMatrixLayoutCreate(lc, ctype, m, n, ldc) != CUBLAS_STATUS_SUCCESS) {
        why = "matrix layout";
        return false;
    }
    cublasLtMatmulPreference_t pref = nullptr;
    cublasLtMatmulPreferenceCreate(&pref);
    size_t wsb = kLtWorkspace;
    cublasLtMatmulPreferenceSetAttribute(pref, CUBLASLT_MATMUL_PREF_MAX_WORKSPACE_BYTES, &wsb,
                                         sizeof(wsb));
    cublasLtMatmulHeuristicResult_t hr{};
    int found = 0;
    const cublasStatus_t s =
        cublasLtMatmulAlgoGetHeuristic(lt, *desc, *la, *lb, *lc, *lc, pref, 1, &hr, &found);
    cublasLtMatmulPreferenceDestroy(pref);
    if (s != CUBLAS_STATUS_SUCCESS || found < 1) {
        why = "no cuBLASLt algorithm for the policy GEMM";
        return false;
    }
    *algo = hr.algo;
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
    const float one = 1.f, zero = 0.f;
    const size_t ob = (size_t)p->rows * p->od;
    const int threads = 256;
    const int gw = grid_for((size_t)p->rows * 32, threads);
    for (int t = 0; t < T; ++t) {
        const float* o_in = (t == 0) ? obs0 : obs + (size_t)(t - 1) * ob;
        const uint8_t* d_prev = (t == 0) ? p->done0 : done + (size_t)(t - 1) * p->E;
        float* a_t = act ? act + (size_t)t * p->rows * 2 : p->act;
        policy_input<<<gw, threads, 0, p->st>>>(o_in, p->rows, p->od, p->odp, p->H, p->row_env,
                                                d_prev, p->x, p->cat, p->h);
        if (cudaGetLastError() != cudaSuccess) return RL_ERR_CUDA;
        if (cublasLtMatmul(p->lt, p->d1, &one, p->w1, p->la1, p->x, p->lb1, &zero, p->cat,
                           p->lc1, p->cat, p->lc1, &p->algo1, p->ws, kLtWorkspace,
                           p->st) != CUBLAS_STATUS_SUCCESS)
            return RL_ERR_CUDA;
        if (cublasLtMatmul(p->lt, p->d2, &one, p->wcat, p->la2, p->cat, p->lb2, &zero, p->g,
                           p->lc2, p->g, p->lc2, &p->algo2, p->ws, kLtWorkspace,
                           p->st) != CUBLAS_STATUS_SUCCESS)
            return RL_ERR_CUDA;
        policy_gates<<<gw, threads, 0, p->st>>>(p->g, p->bias, p->wo, p->bo, p->rows, p->H,
                                                p->vmax, p->h, p->cat, a_t);
        if (cudaGetLastError() != cudaSuccess) return RL_ERR_CUDA;
        const rl_status s = rl_step(env, a_t, obs + (size_t)t * ob,
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
    if (hidden < 32 || hidden > 512 || hidden % 32 != 0)
        return fail(env, nullptr, RL_ERR_ARG, "rl_policy_create: hidden must be a multiple of 32 up to 512");
    rl_policy* p = new (std::nothrow) rl_policy();
    if (!p) return RL_ERR_OOM;
    p->env = env;
    p->H = hidden;
    p->od = rl_obs_dim(env);
    p->odp = (p->od + 15) / 16 * 16;
    p->rows = rl_total_robots(env);
    p->E = rl_n_envs(env);
    p->vmax = (float)c.vmax;
    p->st = rl::env_stream(env);
    const int H = p->H, od = p->od, odp = p->odp, rows = p->rows;
    // weights on the host in their device layouts
    std::vector<float> w1((size_t)H * odp, 0.f), wcat((size_t)4 * H * 2 * H, 0.f), bias(4 * H);
    for (int u = 0; u < H; ++u)
        for (int q = 0; q < od; ++q) w1[(size_t)u * odp + q] = h_w1[(size_t)u * od + q];
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
    }
    std::vector<int32_t> row_env(rows);
    const std::vector<int32_t>& off = rl::env_offsets(env);
    for (int e = 0; e < p->E; ++e)
        for (int r = off[e]; r < off[e + 1]; ++r) row_env[r] = e;
    // device buffers
    float* staging = nullptr;
    const size_t stage_n = std::max(w1.size(), wcat.size());
    bool ok = cudaMallocAsync((void**)&p->w1, w1.size() * 2, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->b1, (size_t)H * 2, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->wcat, wcat.size() * 2, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->bias, bias.size() * 4, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->wo, (size_t)2 * H * 4, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->bo, 2 * 4, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->x, (size_t)rows * odp * 2, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->cat, (size_t)rows * 2 * H * 2, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->g, (size_t)rows * 4 * H * 4, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->h, (size_t)rows * H * 4, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->act, (size_t)rows * 2 * 4, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->row_env, (size_t)rows * 4, p->st) == cudaSuccess &&
              cudaMallocAsync((void**)&p->done0, (size_t)p->E, p->st) == cudaSuccess &&
              cudaMallocAsync(&p->ws, kLtWorkspace, p->st) == cudaSuccess &&
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
    ok = up_bf16(w1.data(), w1.size(), p->w1) && up_bf16(h_b1, H, p->b1) &&
         up_bf16(wcat.data(), wcat.size(), p->wcat) &&
         cudaMemcpyAsync(p->bias, bias.data(), bias.size() * 4, cudaMemcpyHostToDevice, p->st) == cudaSuccess &&
         cudaMemcpyAsync(p->wo, h_wo, (size_t)2 * H * 4, cudaMemcpyHostToDevice, p->st) == cudaSuccess &&
         cudaMemcpyAsync(p->bo, h_bo, 2 * 4, cudaMemcpyHostToDevice, p->st) == cudaSuccess &&
         cudaMemcpyAsync(p->row_env, row_env.data(), (size_t)rows * 4, cudaMemcpyHostToDevice, p->st) == cudaSuccess &&
         cudaMemsetAsync(p->h, 0, (size_t)rows * H * 4, p->st) == cudaSuccess &&
         cudaMemsetAsync(p->cat, 0, (size_t)rows * 2 * H * 2, p->st) == cudaSuccess &&
         cudaMemsetAsync(p->done0, 0, (size_t)p->E, p->st) == cudaSuccess &&
         cudaStreamSynchronize(p->st) == cudaSuccess;
    cudaFreeAsync(staging, p->st);
    if (!ok) return fail(env, p, RL_ERR_CUDA, "rl_policy_create: upload");
    if (cublasLtCreate(&p->lt) != CUBLAS_STATUS_SUCCESS)
        return fail(env, p, RL_ERR_CUDA, "rl_policy_create: cuBLASLt");
    std::string why;
    // h1 (bf16, into the first H rows of each [2H] column of cat) = ReLU(W1 x + b1)
    if (!make_gemm(p->lt, H, rows, odp, odp, odp, 2 * H, CUDA_R_16BF, CUBLASLT_EPILOGUE_RELU_BIAS,
                   p->b1, CUDA_R_16BF, &p->d1, &p->la1, &p->lb1, &p->lc1, &p->algo1, why) ||
        !make_gemm(p->lt, 4 * H, rows, 2 * H, 2 * H, 2 * H, 4 * H, CUDA_R_32F,
                   CUBLASLT_EPILOGUE_DEFAULT, nullptr, CUDA_R_32F, &p->d2, &p->la2, &p->lb2,
                   &p->lc2, &p->algo2, why))
        return fail(env, p, RL_ERR_CUDA, "rl_policy_create: " + why);
    *out = p;
    return RL_OK;
}

rl_status rl_policy_reset_hidden(rl_policy* p) {
    if (!p) return RL_ERR_ARG;
    if (cudaMemsetAsync(p->h, 0, (size_t)p->rows * p->H * 4, p->st) != cudaSuccess ||
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
            rl::env_set_error(env, "policy rollout graph instantiate");
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
