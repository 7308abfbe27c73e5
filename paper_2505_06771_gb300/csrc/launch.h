// launch.h -- host-side launchers of the environment kernels (one translation unit per
// precision / size class so that the library builds in parallel).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>

#include "env_step.cuh"

namespace rl {

// Robot-count classes: an env with n robots runs in the smallest class with n <= nmax; the
// team of a class has kClassLanes lanes (a power of two >= nmax).
constexpr int kNumClasses = 5;
constexpr int kClassNmax[kNumClasses] = {4, 8, 16, 20, 32};
constexpr int kClassLanes[kNumClasses] = {4, 8, 16, 32, 32};

// Launch the step (reset == false) or reset (reset == true) kernel of one class.
// lanes: team size; block_threads: a multiple of 32; max_blocks <= 0: one team per env.
cudaError_t launch_f32_small(const LaunchArgs<float>& a, int lanes, int block_threads,
                             int max_blocks, cudaStream_t st, bool reset);
cudaError_t launch_f32_large(const LaunchArgs<float>& a, int nmax, int lanes, int block_threads,
                             int max_blocks, cudaStream_t st, bool reset);
cudaError_t launch_f64(const LaunchArgs<double>& a, int nmax, int lanes, int block_threads,
                       int max_blocks, cudaStream_t st, bool reset);

// One persistent launch over every class of an uneven batch (binary32).
struct MultiClass {
    int nmax, list_begin, count;
};
struct MultiArgs {
    LaunchArgs<float> a;  // a.env_list: the class lists, concatenated
    MultiClass cls[kNumClasses];
    const int4* items;    // (class, first index in the class list, envs)
    int n_items;
    unsigned* head;       // work-queue counter, zeroed by launch_multi
    int fast;             // Navigation, scripted, no traces
};
cudaError_t launch_multi(const MultiArgs& m, unsigned class_mask, int max_blocks,
                         cudaStream_t st);
size_t multi_smem_bytes(unsigned class_mask);

// Shared memory per team of a class.
size_t team_smem_bytes(int precision, int nmax);
// Lanes a class supports (bitmask of powers of two).
unsigned supported_lanes(int precision, int nmax);

template <typename R, int G, int NMAX>
cudaError_t launch_one(const LaunchArgs<R>& a, int block_threads, int max_blocks,
                       cudaStream_t st, bool reset) {
    if (block_threads < G || block_threads % 32 != 0 || block_threads > 256)
        return cudaErrorInvalidValue;
    // fewer teams per block when their shared memory would exceed the 227 KB per-block limit
    while (block_threads > 32 && (size_t)(block_threads / G) * sizeof(TeamSmem<R, NMAX>) > 227 * 1024)
        block_threads -= 32;
    const int tpb = block_threads / G;
    const size_t smem = (size_t)tpb * sizeof(TeamSmem<R, NMAX>);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    void (*kern)(LaunchArgs<R>) = reset ? reset_kernel<R, G, NMAX> : env_kernel<R, G, NMAX>;
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

}  // namespace rl
