// internal.h -- what the policy and allocation-free modules need from the handle code (not part
// of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/rl.h"
#include "env_step.cuh"

namespace rl {

cudaStream_t env_stream(const rl_env* h);
const std::vector<int32_t>& env_offsets(const rl_env* h);  // [E + 1] first row of each env
const rl_config& env_config(const rl_env* h);
void env_set_error(rl_env* h, const std::string& msg);
// Checks a configuration (scenario, precision, constants, arena, resource and robot slots,
// tuning fields, controller); false with a one-word reason in why.
bool valid_config(const rl_config& c, std::string& why);
// The launch arguments of a binary32 handle (state views, constants); false for binary64.
bool env_args_f32(const rl_env* h, LaunchArgs<float>& a);

}  // namespace rl
