// Kernel instance: mixed FP32/FP64 root iterations, 4 warps integrate each position, one new limb
// sample per lane per iteration (128 per iteration).
#include "kernels.cuh"

namespace tw {
TW_DEFINE_LAUNCHER_W(1, 4)
}
