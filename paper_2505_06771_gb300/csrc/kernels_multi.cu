// kernels_multi.cu -- one persistent launch over environments of uneven robot counts (binary32).
//
// The envs of a batch are bucketed by robot count into classes (<= 4, <= 8, <= 16, <= 20,
// <= 32 robots), each with its own team size (4, 8, 16, 32, 32 lanes).  A block of 64 threads repeatedly
// takes the next work item -- a run of envs of one class, one env per team -- from a device-wide
// queue (one atomic counter), and runs those envs for all T steps.  Items are ordered largest
// class first, so the longest jobs start first and the short ones fill the tail.
#include "env_nav4.cuh"
#include "launch.h"

namespace rl {

// SCEN: the batch's scenario, fixed at compile time (Navigation takes the gather fast path for
// its 4-robot class; the others the lean scripted steps).
template <int SCEN>
__global__ void __launch_bounds__(64, 1) env_kernel_multi(MultiArgs M) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(M.head, 1u);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= M.n_items) break;
        const int4 w = M.items[it];  // class, first list index, count
        const MultiClass& c = M.cls[w.x];
        const int* list = M.a.env_list + c.list_begin + w.y;
        switch (c.nmax) {
            case 4: {
                const Team<4> tm;
                const int tib = threadIdx.x / 4;
                TeamSmem<float, 4>* S = reinterpret_cast<TeamSmem<float, 4>*>(smem_raw) + tib;
                if (tib < w.z) {
                    if constexpr (SCEN == 0) run_env_nav4(M.a, tm, *S, list[tib]);
                    else run_env_small<false, SCEN, true>(M.a, tm, *S, list[tib]);
                }
                break;
            }
            case 8: {
                const Team<8> tm;
                const int tib = threadIdx.x / 8;
                TeamSmem<float, 8>* S = reinterpret_cast<TeamSmem<float, 8>*>(smem_raw) + tib;
                if (tib < w.z) run_env<float, 8, 8, SCEN, true>(M.a, tm, *S, list[tib]);
                break;
            }
            case 16: {
                const Team<16> tm;
                const int tib = threadIdx.x / 16;
                TeamSmem<float, 16>* S = reinterpret_cast<TeamSmem<float, 16>*>(smem_raw) + tib;
                if (tib < w.z) run_env<float, 16, 16, SCEN, true>(M.a, tm, *S, list[tib]);
                break;
            }
            case 20: {
                const Team<32> tm;
                const int tib = threadIdx.x / 32;
                TeamSmem<float, 20>* S = reinterpret_cast<TeamSmem<float, 20>*>(smem_raw) + tib;
                if (tib < w.z) run_env<float, 32, 20, SCEN, true>(M.a, tm, *S, list[tib]);
                break;
            }
            default: {
                const Team<32> tm;
                const int tib = threadIdx.x / 32;
                TeamSmem<float, 32>* S = reinterpret_cast<TeamSmem<float, 32>*>(smem_raw) + tib;
                if (tib < w.z) run_env<float, 32, 32, SCEN, true>(M.a, tm, *S, list[tib]);
                break;
            }
        }
        __syncthreads();
    }
}

size_t multi_smem_bytes(unsigned class_mask) {
    size_t m = 0;
    if (class_mask & 1u) m = std::max(m, (size_t)(64 / 4) * sizeof(TeamSmem<float, 4>));
    if (class_mask & 2u) m = std::max(m, (size_t)(64 / 8) * sizeof(TeamSmem<float, 8>));
    if (class_mask & 4u) m = std::max(m, (size_t)(64 / 16) * sizeof(TeamSmem<float, 16>));
    if (class_mask & 8u) m = std::max(m, (size_t)(64 / 32) * sizeof(TeamSmem<float, 20>));
    if (class_mask & 16u) m = std::max(m, (size_t)(64 / 32) * sizeof(TeamSmem<float, 32>));
    return m;
}

cudaError_t launch_multi(const MultiArgs& m, unsigned class_mask, int max_blocks, cudaStream_t st) {
    const size_t smem = multi_smem_bytes(class_mask);
    const int scen = m.a.k.scenario;
    if (scen < 0 || scen > 2) return cudaErrorInvalidValue;
    void (*kern)(MultiArgs) = scen == 0 ? env_kernel_multi<0>
                              : (scen == 1 ? env_kernel_multi<1> : env_kernel_multi<2>);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 64, smem);
    if (e != cudaSuccess) return e;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int blocks = std::max(1, per_sm) * sms;
    if (blocks > m.n_items) blocks = m.n_items;
    if (max_blocks > 0 && blocks > max_blocks) blocks = max_blocks;
    if (blocks <= 0) return cudaSuccess;
    e = cudaMemsetAsync(m.head, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    kern<<<blocks, 64, smem, st>>>(m);
    return cudaGetLastError();
}

}  // namespace rl
