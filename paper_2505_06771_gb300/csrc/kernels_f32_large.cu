// Binary32 kernels of the 8-, 16- and 32-robot classes.
#include "launch.h"

namespace rl {

cudaError_t launch_f32_large(const LaunchArgs<float>& a, int nmax, int lanes, int block_threads,
                             int max_blocks, cudaStream_t st, bool reset) {
    if (nmax == 8 && lanes == 8) return launch_one<float, 8, 8>(a, block_threads, max_blocks, st, reset);
    if (nmax == 16 && lanes == 16) return launch_one<float, 16, 16>(a, block_threads, max_blocks, st, reset);
    if (nmax == 20 && lanes == 32) return launch_one<float, 32, 20>(a, block_threads, max_blocks, st, reset);
    if (nmax == 32 && lanes == 32) return launch_one<float, 32, 32>(a, block_threads, max_blocks, st, reset);
    return cudaErrorInvalidValue;
}

size_t team_smem_bytes(int precision, int nmax) {
    if (precision == 64) {
        switch (nmax) {
            case 4: return sizeof(TeamSmem<double, 4>);
            case 8: return sizeof(TeamSmem<double, 8>);
            case 16: return sizeof(TeamSmem<double, 16>);
            case 20: return sizeof(TeamSmem<double, 20>);
            case 32: return sizeof(TeamSmem<double, 32>);
        }
    } else {
        switch (nmax) {
            case 4: return sizeof(TeamSmem<float, 4>);
            case 8: return sizeof(TeamSmem<float, 8>);
            case 16: return sizeof(TeamSmem<float, 16>);
            case 20: return sizeof(TeamSmem<float, 20>);
            case 32: return sizeof(TeamSmem<float, 32>);
        }
    }
    return 0;
}

unsigned supported_lanes(int precision, int nmax) {
    if (precision == 32 && nmax == 4) return 1u | 2u | 4u;
    return nmax == 20 ? 32u : (unsigned)nmax;
}

}  // namespace rl
