// Kernel instance: limb-darkened sources, FP64 root iterations.
#include "kernels.cuh"

namespace tw {
TW_DEFINE_LD_LAUNCHER(0)
}
