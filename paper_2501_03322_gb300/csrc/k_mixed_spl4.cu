// Kernel instance: mixed FP32/FP64 root iterations, 4 new limb sample(s) per lane per iteration.
#include "kernels.cuh"

namespace tw {
TW_DEFINE_LAUNCHER(1, 4)
}
