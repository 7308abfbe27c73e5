// Binary64 kernels (every class, one lane per robot).
#include "launch.h"

namespace rl {

cudaError_t launch_f64(const LaunchArgs<double>& a, int nmax, int lanes, int block_threads,
                       int max_blocks, cudaStream_t st, bool reset) {
    if (lanes != (nmax == 20 ? 32 : nmax)) return cudaErrorInvalidValue;
    switch (nmax) {
        case 4: return launch_one<double, 4, 4>(a, block_threads, max_blocks, st, reset);
        case 8: return launch_one<double, 8, 8>(a, block_threads, max_blocks, st, reset);
        case 16: return launch_one<double, 16, 16>(a, block_threads, max_blocks, st, reset);
        case 20: return launch_one<double, 32, 20>(a, block_threads, max_blocks, st, reset);
        case 32: return launch_one<double, 32, 32>(a, block_threads, max_blocks, st, reset);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rl
