// Gaussian-mixture SMC sampler kernels (Sec. 5.2).
#pragma once

#include "weight_reduce.cuh"

namespace smc {

constexpr bool kGmmEnabled = false;
constexpr int kGmmMaxComp = 8;
constexpr int64_t kGmmMaxData = 8192;

}  // namespace smc
