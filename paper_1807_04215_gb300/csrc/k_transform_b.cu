// Transform kernels instantiated for N = 128, 192 (see k_transform.cuh).
#include "k_transform.cuh"

namespace gridspt {
GRIDSPT_TRANSFORM_SIZE(128)
GRIDSPT_TRANSFORM_SIZE(192)
}  // namespace gridspt
