// Binary32 kernels of the 4-robot class (lanes 1, 2 or 4 per env).
#include "launch.h"

namespace rl {

cudaError_t launch_f32_small(const LaunchArgs<float>& a, int lanes, int block_threads,
                             int max_blocks, cudaStream_t st, bool reset) {
    switch (lanes) {
        case 1: return launch_one<float, 1, 4>(a, block_threads, max_blocks, st, reset);
        case 2: return launch_one<float, 2, 4>(a, block_threads, max_blocks, st, reset);
        case 4: return launch_one<float, 4, 4>(a, block_threads, max_blocks, st, reset);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rl
