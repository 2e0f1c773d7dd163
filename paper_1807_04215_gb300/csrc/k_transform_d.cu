// Transform kernels instantiated for N = 512 (see k_transform.cuh).
#include "k_transform.cuh"

namespace gridspt {
GRIDSPT_TRANSFORM_SIZE(512)
}  // namespace gridspt
