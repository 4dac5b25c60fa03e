// Kernel instance: limb-darkened sources, mixed FP32/FP64 root iterations.
#include "kernels.cuh"

namespace tw {
TW_DEFINE_LD_LAUNCHER(1)
}
