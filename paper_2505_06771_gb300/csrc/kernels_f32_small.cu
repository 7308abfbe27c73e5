// Binary32 kernels of the 4-robot class: one thread per env (Navigation, scripted, no traces),
// the register-resident team kernel (4 lanes per env), and the generic shared-memory kernel with
// 2 lanes per env (a tuner candidate).
#include "env_nav4.cuh"
#include "env_split.cuh"
#include "env_thread.cuh"
#include "launch.h"

namespace rl {

static bool is_fast(const LaunchArgs<float>& a);

// Dynamic shared memory of a spread launch: more than half of an SM's 228 KB, so one block
// per SM.
constexpr size_t kSpreadSmem = 116 * 1024;

static cudaError_t launch_small_regs(const LaunchArgs<float>& a, int block_threads,
                                     int max_blocks, cudaStream_t st) {
    if (block_threads < 32 || block_threads % 32 != 0) return cudaErrorInvalidValue;
    if (block_threads > 128) block_threads = 128;  // the kernel's launch bound
    const int tpb = block_threads / 4;
    const size_t smem = (size_t)tpb * sizeof(TeamSmem<float, 4>);
    const bool fast = is_fast(a);
    int variant = a.variant;
    if (fast && a.k.controller != 0) variant = 2;  // the pose controller: gather kernel only
    // policy actions without traces (the policy-in-the-loop step): the split kernel, whose
    // dynamics take the actions as nominal velocities
    const bool split_ok = fast || (a.k.scenario == 0 && a.k.controller == 0 && a.io.u_nom == nullptr &&
                                   a.io.u_star == nullptr && a.io.vw == nullptr &&
                                   a.io.qp_info == nullptr);
    if (!fast && split_ok && variant == 0) variant = 3;
    if (split_ok && variant == 3 && a.warp_envs <= 0 && max_blocks <= 0) {
        // dynamics and output warps (env_split.cuh): one block of 4 + 4 warps per SM, the envs
        // spread evenly over the dynamics warps when that leaves at most 8 per warp
        int dev = 0, sms = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        const int blocks = std::min(sms, (a.n_list + 3) / 4);
        if (blocks >= 1 && a.n_list <= 8 * 4 * blocks) {
            const size_t sp = (size_t)64 * sizeof(TeamSmem<float, 4>);  // dynamics + output teams
            e = cudaFuncSetAttribute(env_kernel_split, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sp);
            if (e != cudaSuccess) return e;
            LaunchArgs<float> b = a;
            b.warp_envs = 0;
            env_kernel_split<<<blocks, 256, sp, st>>>(b);
            return cudaGetLastError();
        }
    }
    if (variant == 3) variant = 1;  // beyond the split launch's reach: the shuffle team kernel
    if (fast && variant != 1 && variant != 2) {
        // auto: the gather kernel (lower latency per step) for small batches, the shuffle
        // kernel (fewer instructions per env-step) for large ones; measured on GB300, 4096
        // envs run 10% faster with the shuffle kernel, one env 20% faster with the gather one
        variant = a.n_list <= 1024 ? 2 : 1;
    }
    void (*kern)(LaunchArgs<float>) = !fast ? env_kernel_small<0>
                                      : (variant == 2 ? env_kernel_small<2> : env_kernel_small<1>);
    if (fast && a.warp_envs <= 0 && max_blocks <= 0) {
        // Spread: one block of 4 warps per SM, so that each warp scheduler runs one warp, and
        // the envs divided evenly over the warps (at most 8 per warp).  The kernel time is the
        // slowest warp's: with a fixed number of envs per warp (6 on 4096 envs) some schedulers
        // get two warps and run them at about half speed.  The shared-memory request keeps a
        // second block off each SM.
        int dev = 0, sms = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        const int blocks = std::min(sms, (a.n_list + 3) / 4);
        if (blocks >= 1 && a.n_list <= 8 * 4 * blocks) {
            const size_t sp = std::max((size_t)32 * sizeof(TeamSmem<float, 4>), kSpreadSmem);
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sp);
            if (e != cudaSuccess) return e;
            LaunchArgs<float> b = a;
            b.warp_envs = 0;
            kern<<<blocks, 128, sp, st>>>(b);
            return cudaGetLastError();
        }
    }
    // envs per warp: 6 for the shuffle kernel (fastest on 4096 envs: 2.60 ms against 2.71 ms
    // with 8 and 2.85 ms with 5), 4 otherwise
    const int per = (a.warp_envs >= 1 && a.warp_envs <= 8) ? a.warp_envs
                                                             : ((fast && variant == 1) ? 6 : 4);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int envs_per_block = (block_threads / 32) * per;
    int blocks = (a.n_list + envs_per_block - 1) / envs_per_block;
    if (max_blocks > 0 && blocks > max_blocks) blocks = max_blocks;
    if (blocks <= 0) return cudaSuccess;
    LaunchArgs<float> b = a;
    b.warp_envs = per;  // the kernel walks the envs with the same stride
    kern<<<blocks, block_threads, smem, st>>>(b);
    return cudaGetLastError();
}

// One thread per env: block_threads / 4 envs per warp (8, 16 or 32), one warp per block.
static cudaError_t launch_thread(const LaunchArgs<float>& a, int block_threads, int max_blocks,
                                 cudaStream_t st) {
    LaunchArgs<float> b = a;
    b.warp_envs = std::min(32, std::max(1, block_threads / 4));
    int blocks = (a.n_list + b.warp_envs - 1) / b.warp_envs;
    if (max_blocks > 0 && blocks > max_blocks) blocks = max_blocks;
    if (blocks <= 0) return cudaSuccess;
    env_kernel_thread<<<blocks, 32, 32 * sizeof(QPWork<double, 4>), st>>>(b);
    return cudaGetLastError();
}

static bool is_fast(const LaunchArgs<float>& a) {
    return a.k.scenario == 0 && a.io.actions == nullptr && a.io.u_nom == nullptr &&
           a.io.u_star == nullptr && a.io.vw == nullptr && a.io.qp_info == nullptr;
}

cudaError_t launch_f32_small(const LaunchArgs<float>& a, int lanes, int block_threads,
                             int max_blocks, cudaStream_t st, bool reset) {
    switch (lanes) {
        case 1:
            // Navigation, scripted, no traces: one thread per env; otherwise the 4-lane team
            if (reset) return launch_one<float, 4, 4>(a, 64, max_blocks, st, true);
            if (is_fast(a) && a.k.controller == 0) return launch_thread(a, block_threads, max_blocks, st);
            return launch_small_regs(a, 64, max_blocks, st);
        case 2: return launch_one<float, 2, 4>(a, block_threads, max_blocks, st, reset);
        case 4:
            if (reset) return launch_one<float, 4, 4>(a, block_threads, max_blocks, st, true);
            return launch_small_regs(a, block_threads, max_blocks, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rl
