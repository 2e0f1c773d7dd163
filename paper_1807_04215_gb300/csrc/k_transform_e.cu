// Transform kernels instantiated for N = 768, 1024 (see k_transform.cuh).
#include "k_transform.cuh"

namespace gridspt {
GRIDSPT_TRANSFORM_SIZE(768)
GRIDSPT_TRANSFORM_SIZE(1024)
}  // namespace gridspt
