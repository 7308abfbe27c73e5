// Binary32 kernels of the 4-robot class: the register-resident team kernel (4 lanes per env)
// and the generic shared-memory kernel with 1 or 2 lanes per env (tuner candidates).
#include "env_small.cuh"
#include "launch.h"

namespace rl {

static cudaError_t launch_small_regs(const LaunchArgs<float>& a, int block_threads,
                                     int max_blocks, cudaStream_t st) {
    if (block_threads < 32 || block_threads % 32 != 0) return cudaErrorInvalidValue;
    if (block_threads > 128) block_threads = 128;  // the kernel's launch bound
    const int tpb = block_threads / 4;
    const size_t smem = (size_t)tpb * sizeof(TeamSmem<float, 4>);
    const bool fast = a.k.scenario == 0 && a.io.actions == nullptr && a.io.u_nom == nullptr &&
                      a.io.u_star == nullptr && a.io.vw == nullptr && a.io.qp_info == nullptr;
    void (*kern)(LaunchArgs<float>) = fast ? env_kernel_small<true> : env_kernel_small<false>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    int blocks = (a.n_list + tpb - 1) / tpb;
    if (max_blocks > 0 && blocks > max_blocks) blocks = max_blocks;
    if (blocks <= 0) return cudaSuccess;
    kern<<<blocks, block_threads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_f32_small(const LaunchArgs<float>& a, int lanes, int block_threads,
                             int max_blocks, cudaStream_t st, bool reset) {
    switch (lanes) {
        case 1: return launch_one<float, 1, 4>(a, block_threads, max_blocks, st, reset);
        case 2: return launch_one<float, 2, 4>(a, block_threads, max_blocks, st, reset);
        case 4:
            if (reset) return launch_one<float, 4, 4>(a, block_threads, max_blocks, st, true);
            return launch_small_regs(a, block_threads, max_blocks, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rl
