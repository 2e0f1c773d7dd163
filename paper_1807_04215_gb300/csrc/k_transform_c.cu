// Transform kernels instantiated for N = 256, 384 (see k_transform.cuh).
#include "k_transform.cuh"

namespace gridspt {
GRIDSPT_TRANSFORM_SIZE(256)
GRIDSPT_TRANSFORM_SIZE(384)
}  // namespace gridspt
